// Measurement aid (not part of the method): the neighbour gathers of one power step with no row
// structure.  Every entry p of the CSR's column array is read once, in order and coalesced, and
// the iterate row z[col[p]] it names is loaded; the rows are summed so that the loads stay live.
// The memory work is that of the power step's gathers (Algorithm 1 body: one row of the iterate
// per stored entry), without row_ptr, the per-row reduction, 1/d or the output rows, so its
// duration is a floor for k_power_step / k_cheb_step on the same graph, row width and type.
#include "fsc_internal.cuh"

namespace fsc {

template <int LP, typename T, int U>
__global__ void __launch_bounds__(256)
k_gather_floor(long long nnz, const int32_t* __restrict__ col, const T* __restrict__ z, long long col_off,
               float* __restrict__ out) {
    float acc = 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride * U) {
        long long j[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long q = p + (long long)u * stride;
            j[u] = q < nnz ? (long long)__ldg(col + q) - col_off : -1;
        }
        float v[U][LP];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (j[u] >= 0) {
                load_row<LP, T>(z + (size_t)j[u] * LP, v[u]);
            } else {
#pragma unroll
                for (int c = 0; c < LP; ++c) v[u][c] = 0.f;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < LP; ++c) acc += v[u][c];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

template <int LP, typename T>
static cudaError_t launch_floor(const fsc_graph* g, const void* z, float* out, cudaStream_t s) {
    auto kern = k_gather_floor<LP, T, 4>;
    const int per_sm = kernel_occupancy((const void*)kern, 256, 0);
    long long blocks = (long long)device_props().num_sms * (per_sm > 0 ? per_sm : 4);
    const long long need = (g->nnz + 255) / 256;
    if (blocks > need) blocks = need;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, 256, 0, s>>>(g->nnz, g->col, static_cast<const T*>(z), g->col_off, out);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_floor_lp(int LP, const fsc_graph* g, const void* z, float* out, cudaStream_t s) {
    switch (LP) {
        case 1: return launch_floor<1, T>(g, z, out, s);
        case 2: return launch_floor<2, T>(g, z, out, s);
        case 4: return launch_floor<4, T>(g, z, out, s);
        case 8: return launch_floor<8, T>(g, z, out, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fsc

using namespace fsc;

extern "C" fsc_status fsc_gather_floor(const fsc_graph* g, int l, fsc_dtype store, const void* z, float* sum_out,
                                       void* stream) {
    if (!g || !z || !sum_out || l < 1 || l > 8 || (store != FSC_F32 && store != FSC_BF16 && store != FSC_F16))
        return FSC_ERR_INVALID_ARG;
    const int LP = pad_l(l);
    const size_t es = store == FSC_F32 ? 4 : 2;
    const size_t al = LP * es < 16 ? LP * es : 16;
    if (reinterpret_cast<uintptr_t>(z) % al) return FSC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    FSC_CUDA(cudaMemsetAsync(sum_out, 0, sizeof(float), s));
    if (g->nnz == 0) return FSC_OK;
    if (store == FSC_F32) FSC_CUDA(launch_floor_lp<float>(LP, g, z, sum_out, s));
    else if (store == FSC_F16) FSC_CUDA(launch_floor_lp<__half>(LP, g, z, sum_out, s));
    else FSC_CUDA(launch_floor_lp<__nv_bfloat16>(LP, g, z, sum_out, s));
    return FSC_OK;
}
