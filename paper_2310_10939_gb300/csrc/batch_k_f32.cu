// Batched-mode kernels with float32 iterates, one per row width and weighting.
#include "batch_device.cuh"

namespace fsc {

const void* batch_kernel_f32(int LP, bool weighted) {
    switch (LP) {
        case 1: return weighted ? (const void*)k_batch_embed<1, float, true> : (const void*)k_batch_embed<1, float, false>;
        case 2: return weighted ? (const void*)k_batch_embed<2, float, true> : (const void*)k_batch_embed<2, float, false>;
        case 4: return weighted ? (const void*)k_batch_embed<4, float, true> : (const void*)k_batch_embed<4, float, false>;
        default: return weighted ? (const void*)k_batch_embed<8, float, true> : (const void*)k_batch_embed<8, float, false>;
    }
}

const void* batch_kmeans_kernel(int LP) {
    switch (LP) {
        case 1: return (const void*)k_batch_kmeans<1>;
        case 2: return (const void*)k_batch_kmeans<2>;
        case 4: return (const void*)k_batch_kmeans<4>;
        default: return (const void*)k_batch_kmeans<8>;
    }
}

FSC_BOUNDS_READER(batch_f32)
}  // namespace fsc
