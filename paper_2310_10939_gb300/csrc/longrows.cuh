// Long rows of the sparse steps: device code shared by longrows.cu (power step) and filter.cu
// (Chebyshev step); the decomposition is described in longrows.cu.
#pragma once

#include "spmm.cuh"

namespace fsc {

// One warp per segment: sum over its entries of w * z_in[col - col_off] (float32, lanes striding
// over the entries, then a shuffle tree), written to part[seg * 8 + c].
template <int LP, typename TI, bool W>
__global__ void __launch_bounds__(256)
k_seg_partial(int64_t nseg, const int64_t* __restrict__ seg_lo, const int64_t* __restrict__ seg_hi,
              const int32_t* __restrict__ col, const float* __restrict__ w, const TI* __restrict__ zin,
              long long col_off, long long nz, float* __restrict__ part) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sg = warp; sg < nseg; sg += nwarps) {
        float acc[LP];
#pragma unroll
        for (int c = 0; c < LP; ++c) acc[c] = 0.f;
        const int64_t lo = seg_lo[sg], hi = seg_hi[sg];
        for (int64_t p = lo + lane; p < hi; p += 4 * 32) {
            float v[4][LP], wv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t q = p + (int64_t)u * 32;
                long long j = q < hi ? (long long)__ldg(col + q) - col_off : -1;
                if (q < hi && !in_range(j, 0, nz, BS_GATHER)) j = -1;
                wv[u] = W ? (q < hi ? __ldg(w + q) : 0.f) : 1.f;
                if (j >= 0) {
                    load_row<LP, TI>(zin + (size_t)j * LP, v[u]);
                } else {
#pragma unroll
                    for (int c = 0; c < LP; ++c) v[u][c] = 0.f;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int c = 0; c < LP; ++c) acc[c] = W ? fmaf(wv[u], v[u][c], acc[c]) : acc[c] + v[u][c];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int c = 0; c < LP; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], off);
        if (lane == 0)
#pragma unroll
            for (int c = 0; c < LP; ++c) part[sg * 8 + c] = acc[c];
    }
}

template <int LP, typename TI>
void seg_partial_launch(const fsc_graph* g, const TI* zin, cudaStream_t s) {
    const int64_t ns = g->n_seg;
    int64_t blocks = (ns * 32 + 255) / 256;
    const int64_t lim = (int64_t)device_props().num_sms * 8;
    if (blocks > lim) blocks = lim;
    if (g->w)
        k_seg_partial<LP, TI, true><<<(unsigned)blocks, 256, 0, s>>>(ns, g->seg_lo, g->seg_hi, g->col, g->w, zin,
                                                                     g->col_off, g->n, g->seg_part);
    else
        k_seg_partial<LP, TI, false><<<(unsigned)blocks, 256, 0, s>>>(ns, g->seg_lo, g->seg_hi, g->col, g->w, zin,
                                                                      g->col_off, g->n, g->seg_part);
}

// The sum of long row h: its segments' partial sums, in segment order.
__device__ __forceinline__ void long_row_sum(int64_t h, const int32_t* seg0, const int32_t* nseg, const float* part,
                                             int LPr, float* acc) {
    for (int c = 0; c < LPr; ++c) acc[c] = 0.f;
    const int64_t s0 = seg0[h], ns = nseg[h];
    for (int64_t q = 0; q < ns; ++q)
        for (int c = 0; c < LPr; ++c) acc[c] += part[(s0 + q) * 8 + c];
}

}  // namespace fsc
