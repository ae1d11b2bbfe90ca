// Batched-mode kernels with bfloat16 iterates, one per row width and weighting.
#include "batch_device.cuh"

namespace fsc {

const void* batch_kernel_bf16(int LP, bool weighted) {
    switch (LP) {
        case 1: return weighted ? (const void*)k_batch_embed<1, __nv_bfloat16, true> : (const void*)k_batch_embed<1, __nv_bfloat16, false>;
        case 2: return weighted ? (const void*)k_batch_embed<2, __nv_bfloat16, true> : (const void*)k_batch_embed<2, __nv_bfloat16, false>;
        case 4: return weighted ? (const void*)k_batch_embed<4, __nv_bfloat16, true> : (const void*)k_batch_embed<4, __nv_bfloat16, false>;
        default: return weighted ? (const void*)k_batch_embed<8, __nv_bfloat16, true> : (const void*)k_batch_embed<8, __nv_bfloat16, false>;
    }
}

FSC_BOUNDS_READER(batch_bf16)
}  // namespace fsc
