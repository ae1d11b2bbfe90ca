// Batched-mode kernels with float32 iterates, one per row width and weighting.
#include "batch_device.cuh"

namespace fsc {

const void* batch_kernel_f32(int LP, bool weighted) {
    switch (LP) {
        case 1: return weighted ? (const void*)k_batch<1, float, true> : (const void*)k_batch<1, float, false>;
        case 2: return weighted ? (const void*)k_batch<2, float, true> : (const void*)k_batch<2, float, false>;
        case 4: return weighted ? (const void*)k_batch<4, float, true> : (const void*)k_batch<4, float, false>;
        default: return weighted ? (const void*)k_batch<8, float, true> : (const void*)k_batch<8, float, false>;
    }
}

}  // namespace fsc
