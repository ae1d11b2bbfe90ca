// Fused power-iteration kernel (Algorithm 1 body with the operator M of Sec. 2).
//
// The iterate is kept in embedding coordinates z = D^-1/2 x.  Since
// D^-1/2 M D^1/2 = (I + D^-1 A) / 2, one step is
//     z_out[i] = (z_in[i] + (1/d_i) * sum_j w_ij z_in[j]) / 2,
// which gathers only z rows (no per-neighbour degree load), and the final
// D^-1/2 of Algorithm 2 comes for free: after t steps z_t = D^-1/2 M^t x_0.
//
// Layout: z is n x LP row-major (LP = padded l, rows of 4..64 bytes).  A group
// of G lanes owns one row: lanes stride over the row's column indices
// (coalesced int32 loads), unroll U independent gathers of LP-wide rows, then
// a shuffle-xor tree reduces the group.  Accumulation is float32.
//
// Optional per-column power-of-two rescale: the previous launch's column
// max-abs (cm_in, float bits) gives e_c = floor(log2 max); outputs are
// multiplied by 2^-e_c (exact), block 0 adds e_c into expo[c], and the final
// launch (last = 1) multiplies by 2^expo[c], so the result equals the
// unscaled iteration except for under/overflow.
#pragma once

#include "fsc_internal.cuh"

namespace fsc {

__device__ __forceinline__ float pow2i(int e) {
    e = e < -126 ? -126 : (e > 127 ? 127 : e);
    return __int_as_float((e + 127) << 23);
}

// Loads of the iterate: through the read-only path when it is not written during the launch
// (NC = true), else through L2 only (the batch kernel rewrites it between block barriers).
template <int LP, typename T, bool NC>
__device__ __forceinline__ void load_z(const T* p, float (&v)[LP]) {
    if (NC) {
        load_row<LP, T>(p, v);
    } else {
        constexpr int BYTES = LP * (int)sizeof(T);
        constexpr int CB = BYTES < 16 ? BYTES : 16;
        using C = typename Chunk<CB>::type;
        constexpr int NCH = BYTES / CB;
        C buf[NCH];
#pragma unroll
        for (int i = 0; i < NCH; ++i) buf[i] = __ldcg(reinterpret_cast<const C*>(p) + i);
        const T* e = reinterpret_cast<const T*>(buf);
#pragma unroll
        for (int c = 0; c < LP; ++c) v[c] = to_f32(e[c]);
    }
}

// sum_j w_ij z_j of one row, computed by the G lanes `sub` = 0..G-1 of a group and reduced with
// full-warp shuffles (every lane of the warp must call it).  `row` indexes rp; column ids are
// shifted by col_off to index zin, which has nz rows.  After the call every lane of the group holds
// the sum.  A row with more than max_row entries is left to the long-row kernels (longrows.cu):
// returns false for it (and for an inactive row).
template <int LP, typename TI, int G, int U, bool W, bool NC>
__device__ __forceinline__ bool row_gather(bool active, long long row, int sub, const int64_t* __restrict__ rp,
                                           const int32_t* __restrict__ col, const float* __restrict__ w,
                                           const TI* zin, long long col_off, long long nz, long long max_row,
                                           float (&acc)[LP]) {
#pragma unroll
    for (int c = 0; c < LP; ++c) acc[c] = 0.f;
    bool own = false;
    if (active) {
        const int64_t s = rp[row], e = rp[row + 1];
        own = e - s <= max_row;
        for (int64_t p = s + sub; own && p < e; p += G * U) {
            long long j[U];
            float wv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t q = p + (int64_t)u * G;
                const bool ok = q < e;
                j[u] = ok ? (long long)__ldg(col + q) - col_off : -1;
                if (ok && !in_range(j[u], 0, nz, BS_GATHER)) j[u] = -1;
                if (W) wv[u] = ok ? __ldg(w + q) : 0.f;
            }
            float v[U][LP];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (j[u] >= 0) {
                    load_z<LP, TI, NC>(zin + (size_t)j[u] * LP, v[u]);
                } else {
#pragma unroll
                    for (int c = 0; c < LP; ++c) v[u][c] = 0.f;
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int c = 0; c < LP; ++c) acc[c] = W ? fmaf(wv[u], v[u][c], acc[c]) : acc[c] + v[u][c];
        }
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1)
#pragma unroll
        for (int c = 0; c < LP; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
    return own;
}

// One output row of the power step, y = scale * (z_in[row] + (1/d) sum_j w_ij z_in[j]) / 2,
// written by lane sub == 0 of the group (which returns true, with the row in y).
template <int LP, typename TI, typename TO, int G, int U, bool W, bool NC>
__device__ __forceinline__ bool power_row(bool active, long long row, int sub, const int64_t* __restrict__ rp,
                                          const int32_t* __restrict__ col, const float* __restrict__ w,
                                          const float* __restrict__ invdeg, const TI* zin, TO* zout,
                                          long long col_off, long long nz, long long max_row,
                                          const float (&scale)[LP], float (&y)[LP]) {
    float acc[LP];
    const bool own = row_gather<LP, TI, G, U, W, NC>(active, row, sub, rp, col, w, zin, col_off, nz, max_row, acc);
    if (own && sub == 0) {
        float self[LP];
        load_z<LP, TI, NC>(zin + (size_t)row * LP, self);
        const float id = invdeg[row];
#pragma unroll
        for (int c = 0; c < LP; ++c) y[c] = scale[c] * (0.5f * fmaf(id, acc[c], self[c]));
        store_row<LP, TO>(zout + (size_t)row * LP, y);
        return true;
    }
    return false;
}

template <int LP, typename TI, typename TO, int G, int U, bool W>
__global__ void __launch_bounds__(256)
k_power_step(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const float* __restrict__ w,
             const float* __restrict__ invdeg, const TI* __restrict__ zin, TO* __restrict__ zout,
             const unsigned* __restrict__ cm_in, unsigned* __restrict__ cm_out, unsigned* __restrict__ cm_zero,
             int* __restrict__ expo, int last, long long col_off, long long max_row) {
    static_assert(32 % G == 0, "G must divide the warp");
    constexpr int RPW = 32 / G;
    __shared__ unsigned s_cm[LP];
    const int lane = threadIdx.x & 31;
    const int sub = lane % G;
    const int grp = lane / G;

    float scale[LP];
#pragma unroll
    for (int c = 0; c < LP; ++c) {
        if (last) scale[c] = expo ? pow2i(expo[c]) : 1.f;
        else scale[c] = cm_in ? pow2i(-exponent_of(__uint_as_float(cm_in[c]))) : 1.f;
    }
    if (cm_out && threadIdx.x < LP) s_cm[threadIdx.x] = 0u;
    if (blockIdx.x == 0 && threadIdx.x < LP) {
        if (cm_zero) cm_zero[threadIdx.x] = 0u;
        if (!last && cm_in && expo) expo[threadIdx.x] += exponent_of(__uint_as_float(cm_in[threadIdx.x]));
    }
    __syncthreads();

    float cmx[LP];   // this lane's running column max |y| (reduced once, at the end)
#pragma unroll
    for (int c = 0; c < LP; ++c) cmx[c] = 0.f;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long base = warp * RPW; base < n; base += nwarps * RPW) {
        const long long row = base + grp;
        float y[LP];
        if (power_row<LP, TI, TO, G, U, W, true>(row < n, row, sub, rp, col, w, invdeg, zin, zout, col_off, n, max_row,
                                                  scale, y)) {
#pragma unroll
            for (int c = 0; c < LP; ++c) cmx[c] = fmaxf(cmx[c], fabsf(y[c]));
        }
    }
    if (cm_out) {
#pragma unroll
        for (int c = 0; c < LP; ++c) {
            float m = cmx[c];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
            if (lane == 0 && m > 0.f) atomicMax(&s_cm[c], __float_as_uint(m));
        }
        __syncthreads();
        if (threadIdx.x < LP && s_cm[threadIdx.x]) atomicMax(cm_out + threadIdx.x, s_cm[threadIdx.x]);
    }
}

struct StepArgs {
    int n;
    const int64_t* rp;
    const int32_t* col;
    const float* w;
    const float* invdeg;
    const void* zin;
    void* zout;
    const unsigned* cm_in;
    unsigned* cm_out;
    unsigned* cm_zero;
    int* expo;
    int last;
    long long col_off;   // subtracted from column ids (graphs that are a slice of a larger CSR)
    long long max_row = 0x7fffffffffffffffLL;   // rows with more entries are left to longrows.cu
    int unroll = 0;      // neighbour rows in flight per lane: 0 = the default for the lane count, or 3 with 4 lanes
};

template <int LP, typename TI, typename TO, int G, int U, bool W>
cudaError_t launch_step(const StepArgs& a, cudaStream_t s) {
    auto kern = k_power_step<LP, TI, TO, G, U, W>;
    static int blocks_per_sm = 0;
    if (blocks_per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, 256, 0);
        if (e != cudaSuccess || blocks_per_sm < 1) blocks_per_sm = 4;
    }
    constexpr int RPW = 32 / G;
    const long long warps = ((long long)a.n + RPW - 1) / RPW;
    long long blocks = (warps + 7) / 8;
    const long long cap = (long long)device_props().num_sms * blocks_per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, 256, 0, s>>>(a.n, a.rp, a.col, a.w, a.invdeg, static_cast<const TI*>(a.zin),
                                         static_cast<TO*>(a.zout), a.cm_in, a.cm_out, a.cm_zero, a.expo, a.last,
                                         a.col_off, a.max_row);
    return cudaGetLastError();
}

template <int LP, typename TI, typename TO, bool W>
cudaError_t launch_step_g(int G, const StepArgs& a, cudaStream_t s) {
    switch (G) {
        case 4: return a.unroll == 3 ? launch_step<LP, TI, TO, 4, 3, W>(a, s) : launch_step<LP, TI, TO, 4, 4, W>(a, s);
        case 8: return launch_step<LP, TI, TO, 8, 4, W>(a, s);
        case 16: return launch_step<LP, TI, TO, 16, 2, W>(a, s);
        case 32: return launch_step<LP, TI, TO, 32, 2, W>(a, s);
    }
    return cudaErrorInvalidValue;
}

template <typename TI, typename TO>
cudaError_t launch_step_any(int LP, int G, bool weighted, const StepArgs& a, cudaStream_t s) {
    switch (LP) {
        case 1: return weighted ? launch_step_g<1, TI, TO, true>(G, a, s) : launch_step_g<1, TI, TO, false>(G, a, s);
        case 2: return weighted ? launch_step_g<2, TI, TO, true>(G, a, s) : launch_step_g<2, TI, TO, false>(G, a, s);
        case 4: return weighted ? launch_step_g<4, TI, TO, true>(G, a, s) : launch_step_g<4, TI, TO, false>(G, a, s);
        case 8: return weighted ? launch_step_g<8, TI, TO, true>(G, a, s) : launch_step_g<8, TI, TO, false>(G, a, s);
    }
    return cudaErrorInvalidValue;
}

// Defined in spmm_f32.cu / spmm_bf16.cu (one instantiation set per translation unit).
cudaError_t launch_step_f32(int LP, int G, bool weighted, const StepArgs& a, cudaStream_t s);
cudaError_t launch_step_bf16(int LP, int G, bool weighted, const StepArgs& a, cudaStream_t s);
cudaError_t launch_step_bf16_to_f32(int LP, int G, bool weighted, const StepArgs& a, cudaStream_t s);
// The long rows of g after a row-split power step with the same arguments (longrows.cu); store_in /
// store_out 0 = float32, 1 = bfloat16.  Nothing to do for a graph without long rows.
cudaError_t long_rows_power(const fsc_graph* g, int LP, int store_in, int store_out, const StepArgs& a, cudaStream_t s);

}  // namespace fsc
