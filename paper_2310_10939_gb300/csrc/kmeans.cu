// k-means++ seeding and Lloyd iterations on the embedding rows (Sec. 2.2, Algorithm 2 last step).
//
// Both phases run as one cooperative (co-resident) persistent launch each.  Blocks own
// contiguous chunks of points; cross-block steps are separated by a bounded grid barrier
// (grid_sync), after which every block reads the other blocks' partial results through L2.
//
// Decisions follow fixed rules so that a float64 CPU restatement can reproduce them:
//  * squared distances: float32, columns in order, no fused multiply-add;
//  * k-means++: first centre floor(u0 * n); round r picks the smallest index whose float64
//    prefix of D^2 exceeds u_r * sum(D^2) (prefix taken over block chunks, then 512-point
//    tiles, then a block scan - the same index order as a sequential scan); sum(D^2) = 0
//    picks the lowest index not chosen yet; a target beyond the computed prefix (rounding)
//    picks the last index with D^2 > 0;
//  * Lloyd: strict '<' over centroids in index order (ties -> lowest index); float64 sums
//    per block, reduced over blocks in a fixed order; an empty cluster keeps its centroid;
//    stop when no label changes or after max_iter steps.
#include <limits.h>
#include <math.h>

#include "fsc_internal.cuh"

namespace fsc {

constexpr int KM_THREADS = 512;
constexpr int KM_WARPS = KM_THREADS / 32;
constexpr int KM_MAX_BLOCKS = 1024;

struct KmDevStats {
    int iterations;
    int changed;
    int empty_events;
    int status;
    double inertia;
    double potential;
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Block-wide sum with a fixed reduction tree; result valid in every thread.
__device__ double block_sum_d(double v, double* s_red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum_d(v);
    __syncthreads();
    if (lane == 0) s_red[wid] = v;
    __syncthreads();
    double t = lane < KM_WARPS ? s_red[lane] : 0.0;
    t = warp_sum_d(t);
    return t;
}
__device__ int block_sum_i(int v, int* s_red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum_i(v);
    __syncthreads();
    if (lane == 0) s_red[wid] = v;
    __syncthreads();
    int t = lane < KM_WARPS ? s_red[lane] : 0;
    return warp_sum_i(t);
}

// Inclusive block scan (fixed tree) of one double per thread.
__device__ double block_scan_incl(double v, double* s_red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double u = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += u;
    }
    __syncthreads();
    if (lane == 31) s_red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double t = lane < KM_WARPS ? s_red[lane] : 0.0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const double u = __shfl_up_sync(0xffffffffu, t, off);
            if (lane >= off) t += u;
        }
        if (lane < KM_WARPS) s_red[lane] = t;
    }
    __syncthreads();
    if (wid > 0) v += s_red[wid - 1];
    return v;
}

template <int LP>
__device__ __forceinline__ void load_point(const float* __restrict__ X, long long i, int l, float (&x)[LP]) {
    load_row<LP, float>(X + (size_t)i * LP, x);
#pragma unroll
    for (int c = 0; c < LP; ++c)
        if (c >= l) x[c] = 0.f;
}

struct KppArgs {
    const float* X;
    int n, l, k;
    unsigned long long seed;
    float* d2[2];
    double* bsum[2];
    double* tsum[2];
    int max_tiles;
    int64_t* seeds;
    float* c32;
    double* c64;
    GridBarrier* bar;
    int* status;
    long long limit;
};

template <int LP>
__global__ void __launch_bounds__(KM_THREADS) k_kmeanspp(KppArgs a) {
    extern __shared__ int s_chosen[];   // k entries
    __shared__ float s_c[LP];
    __shared__ double s_red[KM_WARPS];
    __shared__ double s_pref[KM_MAX_BLOCKS];
    __shared__ double s_T, s_base;
    __shared__ int s_bstar, s_tile, s_idx, s_fallback;
    const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const long long n = a.n;
    const long long chunk = (n + G - 1) / G;
    const long long lo = min(n, (long long)b * chunk), hi = min(n, lo + chunk);

    if (tid == 0) {
        const U64x4 r = philox4x64_10(U64x4{0ull, 0ull, 0ull, 0ull}, a.seed, STREAM_KMEANSPP);
        long long i0 = (long long)floor(uniform53(r.x) * (double)n);
        if (i0 > n - 1) i0 = n - 1;
        s_chosen[0] = (int)i0;
        if (b == 0) a.seeds[0] = i0;
    }
    __syncthreads();

    for (int r = 1; r < a.k; ++r) {
        const int cur = s_chosen[r - 1];
        if (tid < LP) s_c[tid] = tid < a.l ? a.X[(size_t)cur * LP + tid] : 0.f;
        __syncthreads();
        float* d2n = a.d2[r & 1];
        const float* d2o = a.d2[(r - 1) & 1];
        double* bs = a.bsum[r & 1];
        double* ts = a.tsum[r & 1] + (size_t)b * a.max_tiles;
        // ---- phase A: D^2 update over this block's chunk, in 512-point tiles
        double bacc = 0.0;
        int tile = 0;
        for (long long t0 = lo; t0 < hi; t0 += KM_THREADS, ++tile) {
            const long long i = t0 + tid;
            double v = 0.0;
            if (i < hi) {
                float x[LP];
                load_point<LP>(a.X, i, a.l, x);
                float dd = sqdist<LP>(x, s_c);
                if (r > 1) dd = fminf(dd, d2o[i]);
                d2n[i] = dd;
                v = (double)dd;
            }
            const double tsv = block_sum_d(v, s_red);
            if (tid == 0) {
                ts[tile] = tsv;
                bacc += tsv;
            }
        }
        if (tid == 0) bs[b] = bacc;
        if (!grid_sync(a.bar, a.status, a.limit)) return;

        // ---- selection (identical in every block)
        if (wid == 0) {
            const int per = (G + 31) / 32;
            const int q0 = min(G, lane * per), q1 = min(G, q0 + per);
            double seg = 0.0;
            for (int q = q0; q < q1; ++q) seg += __ldcg(bs + q);
            double incl = seg;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const double u = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += u;
            }
            double run = __shfl_up_sync(0xffffffffu, incl, 1);
            if (lane == 0) run = 0.0;
            for (int q = q0; q < q1; ++q) {
                run += __ldcg(bs + q);
                s_pref[q] = run;
            }
        }
        __syncthreads();
        if (wid == 0) {
            const double total = s_pref[G - 1];
            if (!(total > 0.0)) {
                if (lane == 0) {
                    s_bstar = -1;
                    s_fallback = 0;
                    s_idx = -1;
                }
            } else {
                const U64x4 rr = philox4x64_10(U64x4{(unsigned long long)r, 0ull, 0ull, 0ull}, a.seed, STREAM_KMEANSPP);
                const double T = uniform53(rr.x) * total;
                const int per = (G + 31) / 32;
                const int q0 = min(G, lane * per), q1 = min(G, q0 + per);
                int found = -1;
                for (int q = q0; q < q1; ++q)
                    if (s_pref[q] > T) { found = q; break; }
                const unsigned m = __ballot_sync(0xffffffffu, found >= 0);
                int bstar, fb = 0;
                if (m) {
                    bstar = __shfl_sync(0xffffffffu, found, __ffs(m) - 1);
                } else {
                    int lastpos = -1;
                    for (int q = q1 - 1; q >= q0; --q)
                        if (__ldcg(bs + q) > 0.0) { lastpos = q; break; }
                    const unsigned m2 = __ballot_sync(0xffffffffu, lastpos >= 0);
                    bstar = m2 ? __shfl_sync(0xffffffffu, lastpos, 31 - __clz(m2)) : 0;
                    fb = 1;
                }
                if (lane == 0) {
                    s_bstar = bstar;
                    s_fallback = fb;
                    s_idx = -1;
                    s_base = bstar > 0 ? s_pref[bstar - 1] : 0.0;
                    s_T = T;
                }
            }
        }
        __syncthreads();
        if (s_bstar < 0) {
            // sum(D^2) = 0: the lowest index not chosen yet
            if (tid == 0) {
                int cand = 0;
                for (;; ++cand) {
                    bool taken = false;
                    for (int q = 0; q < r; ++q)
                        if (s_chosen[q] == cand) { taken = true; break; }
                    if (!taken) break;
                }
                s_idx = cand;
            }
        } else {
            const int bs_ = s_bstar;
            const long long blo = min(n, (long long)bs_ * chunk), bhi = min(n, blo + chunk);
            const double* tsb = a.tsum[r & 1] + (size_t)bs_ * a.max_tiles;
            const int ntiles = (int)((bhi - blo + KM_THREADS - 1) / KM_THREADS);
            if (tid == 0) {
                double run = s_base;
                int tl = -1;
                if (!s_fallback) {
                    for (int q = 0; q < ntiles; ++q) {
                        const double v = __ldcg(tsb + q);
                        if (run + v > s_T) { tl = q; break; }
                        run += v;
                    }
                }
                s_tile = tl;
                s_base = run;
            }
            __syncthreads();
            if (s_tile >= 0) {
                const long long i = blo + (long long)s_tile * KM_THREADS + tid;
                const double v = i < bhi ? (double)__ldcg(d2n + i) : 0.0;
                const double incl = block_scan_incl(v, s_red) + s_base;
                if (tid == 0) s_idx = INT_MAX;
                __syncthreads();
                if (i < bhi && v > 0.0 && incl > s_T) atomicMin(&s_idx, (int)i);
                __syncthreads();
                if (s_idx == INT_MAX) s_idx = -1;   // rounding: fall through to the last positive
                __syncthreads();
            }
            if (s_idx < 0) {
                // last index of the chunk with D^2 > 0
                if (tid == 0) s_idx = -1;
                __syncthreads();
                for (long long i = blo + tid; i < bhi; i += KM_THREADS)
                    if (__ldcg(d2n + i) > 0.f) atomicMax(&s_idx, (int)i);
                __syncthreads();
                if (tid == 0 && s_idx < 0) {
                    // nothing positive in the chunk (rounding only): the lowest index not chosen yet
                    int cand = 0;
                    for (;; ++cand) {
                        bool taken = false;
                        for (int q = 0; q < r; ++q)
                            if (s_chosen[q] == cand) { taken = true; break; }
                        if (!taken) break;
                    }
                    s_idx = cand;
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            s_chosen[r] = s_idx;
            if (b == 0) a.seeds[r] = s_idx;
        }
        __syncthreads();
    }
    // centres: block 0 writes the k seed rows (float32 copy and float64 master)
    if (b == 0) {
        for (int q = tid; q < a.k * LP; q += KM_THREADS) {
            const int j = q / LP, c = q % LP;
            const float v = c < a.l ? a.X[(size_t)s_chosen[j] * LP + c] : 0.f;
            a.c32[q] = v;
            a.c64[q] = (double)v;
        }
    }
}

struct LloydArgs {
    const float* X;
    int n, l, k, max_iter;
    int32_t* labels;
    float* c32;
    double* c64;
    double* partials;
    double* inertia_part;
    int* changed_part;
    KmDevStats* st;
    GridBarrier* bar;
    int* status;
    long long limit;
};

template <int LP>
__global__ void __launch_bounds__(KM_THREADS) k_lloyd(LloydArgs a) {
    extern __shared__ __align__(16) unsigned char km_smem[];
    const int k = a.k;
    float* s_c = reinterpret_cast<float*>(km_smem);
    double* s_sum = reinterpret_cast<double*>(km_smem + (((size_t)k * LP * 4 + 15) & ~(size_t)15));
    unsigned long long* s_cnt = reinterpret_cast<unsigned long long*>(s_sum + (size_t)k * LP);
    __shared__ double s_red[KM_WARPS];
    __shared__ int s_redi[KM_WARPS];
    __shared__ int s_stop, s_changed;
    const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const long long n = a.n;
    const long long chunk = (n + G - 1) / G;
    const long long lo = min(n, (long long)b * chunk), hi = min(n, lo + chunk);
    const size_t pstride = (size_t)k * LP + k;

    for (int it = 1; it <= a.max_iter; ++it) {
        for (int q = tid; q < k * LP; q += KM_THREADS) {
            s_c[q] = __ldcg(a.c32 + q);
            s_sum[q] = 0.0;
        }
        for (int q = tid; q < k; q += KM_THREADS) s_cnt[q] = 0ull;
        __syncthreads();
        double inert = 0.0;
        int changed = 0;
        // ---- phase A: assignment and per-block float64 sums
        for (long long base = lo + (long long)wid * 32; base < hi; base += KM_THREADS) {
            const long long i = base + lane;
            const bool valid = i < hi;
            float x[LP];
            int bj = 0;
            if (valid) {
                load_point<LP>(a.X, i, a.l, x);
                float best = sqdist<LP>(x, s_c);
                for (int j = 1; j < k; ++j) {
                    const float d = sqdist<LP>(x, s_c + j * LP);
                    if (d < best) { best = d; bj = j; }
                }
                const int old = a.labels[i];
                changed += old != bj;
                a.labels[i] = bj;
                inert += (double)best;
            } else {
#pragma unroll
                for (int c = 0; c < LP; ++c) x[c] = 0.f;
            }
            const unsigned vmask = __ballot_sync(0xffffffffu, valid);
            const int lab0 = __shfl_sync(0xffffffffu, bj, 0);
            const bool uniform = __all_sync(0xffffffffu, !valid || bj == lab0);
            if (uniform) {
#pragma unroll
                for (int c = 0; c < LP; ++c) {
                    const double v = warp_sum_d((double)x[c]);
                    if (lane == 0) atomicAdd(&s_sum[lab0 * LP + c], v);
                }
                if (lane == 0) atomicAdd(&s_cnt[lab0], (unsigned long long)__popc(vmask));
            } else if (valid) {
#pragma unroll
                for (int c = 0; c < LP; ++c) atomicAdd(&s_sum[bj * LP + c], (double)x[c]);
                atomicAdd(&s_cnt[bj], 1ull);
            }
        }
        __syncthreads();
        double* P = a.partials + (size_t)b * pstride;
        for (int q = tid; q < k * LP; q += KM_THREADS) P[q] = s_sum[q];
        for (int q = tid; q < k; q += KM_THREADS) P[(size_t)k * LP + q] = (double)s_cnt[q];
        inert = block_sum_d(inert, s_red);
        changed = block_sum_i(changed, s_redi);
        if (tid == 0) {
            a.inertia_part[b] = inert;
            a.changed_part[b] = changed;
        }
        if (!grid_sync(a.bar, a.status, a.limit)) return;
        // ---- phase B: convergence test (every block) and centroid means (one warp per cluster)
        if (wid == 0) {
            int c = 0;
            for (int q = lane; q < G; q += 32) c += __ldcg(a.changed_part + q);
            c = warp_sum_i(c);
            if (lane == 0) {
                s_changed = c;
                s_stop = (c == 0 || it == a.max_iter) ? 1 : 0;
            }
        }
        for (int j = b * KM_WARPS + wid; j < k; j += G * KM_WARPS) {
            double acc[LP + 1];
#pragma unroll
            for (int c = 0; c <= LP; ++c) acc[c] = 0.0;
            for (int q = lane; q < G; q += 32) {
                const double* Pq = a.partials + (size_t)q * pstride;
#pragma unroll
                for (int c = 0; c < LP; ++c) acc[c] += __ldcg(Pq + (size_t)j * LP + c);
                acc[LP] += __ldcg(Pq + (size_t)k * LP + j);
            }
#pragma unroll
            for (int c = 0; c <= LP; ++c) acc[c] = warp_sum_d(acc[c]);
            if (lane == 0) {
                const double cnt = acc[LP];
                if (cnt > 0.0) {
#pragma unroll
                    for (int c = 0; c < LP; ++c) {
                        const double m = acc[c] / cnt;
                        a.c64[(size_t)j * LP + c] = m;
                        a.c32[(size_t)j * LP + c] = (float)m;
                    }
                } else {
                    atomicAdd(&a.st->empty_events, 1);
                }
            }
        }
        if (b == 0 && wid == 1) {
            double v = 0.0;
            for (int q = lane; q < G; q += 32) v += __ldcg(a.inertia_part + q);
            v = warp_sum_d(v);
            if (lane == 0) {
                a.st->inertia = v;
                if (it == 1) a.st->potential = v;
            }
        }
        __syncthreads();
        if (b == 0 && tid == 0) {
            a.st->iterations = it;
            a.st->changed = s_changed;
        }
        if (s_stop) return;
        if (!grid_sync(a.bar, a.status, a.limit)) return;
    }
}

__global__ void k_merge_status(const int* __restrict__ call_status, int* __restrict__ dev_status) {
    if (*call_status) atomicOr(dev_status, *call_status);
}

template <typename K>
static int coop_blocks(K kern, size_t smem) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, KM_THREADS, smem) != cudaSuccess) return 0;
    if (per_sm > 2) per_sm = 2;
    return per_sm * device_props().num_sms;
}

template <int LP>
static fsc_status kmeans_lp(const float* emb, int n, int l, int k, uint64_t seed, int max_iter, int32_t* labels,
                            double* centroids, int64_t* seed_idx, fsc_kmeans_stats* stats, cudaStream_t s) {
    const size_t kpp_smem = (size_t)k * sizeof(int);
    const size_t lloyd_smem = (((size_t)k * LP * 4 + 15) & ~(size_t)15) + (size_t)k * LP * 8 + (size_t)k * 8;
    auto kpp = k_kmeanspp<LP>;
    auto lly = k_lloyd<LP>;
    FSC_CUDA(cudaFuncSetAttribute(kpp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kpp_smem));
    FSC_CUDA(cudaFuncSetAttribute(lly, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lloyd_smem));
    int G = coop_blocks(kpp, kpp_smem);
    const int G2 = coop_blocks(lly, lloyd_smem);
    if (G2 < G) G = G2;
    if (G < 1) return FSC_ERR_CUDA;
    const long long need = ((long long)n + KM_THREADS - 1) / KM_THREADS;
    if (G > need) G = (int)need;
    if (G > KM_MAX_BLOCKS) G = KM_MAX_BLOCKS;
    const long long chunk = ((long long)n + G - 1) / G;
    const int max_tiles = (int)((chunk + KM_THREADS - 1) / KM_THREADS);

    // workspace layout (256-byte aligned pieces)
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0;
    const size_t o_hdr = off; off += up(sizeof(KmDevStats) + sizeof(GridBarrier) + 2 * sizeof(int));
    const size_t o_d2 = off; off += 2 * up((size_t)n * 4);
    const size_t o_bs = off; off += 2 * up((size_t)G * 8);
    const size_t o_ts = off; off += 2 * up((size_t)G * max_tiles * 8);
    const size_t o_part = off; off += up((size_t)G * ((size_t)k * LP + k) * 8);
    const size_t o_inert = off; off += up((size_t)G * 8);
    const size_t o_chg = off; off += up((size_t)G * 4);
    const size_t o_c64 = off; off += up((size_t)k * LP * 8);
    const size_t o_c32 = off; off += up((size_t)k * LP * 4);
    const size_t o_seed = off; off += up((size_t)k * 8);
    char* ws = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&ws), off, s);
    if (e != cudaSuccess) return cuda_status(e);
    fsc_status rc = FSC_OK;
    KmDevStats* st = reinterpret_cast<KmDevStats*>(ws + o_hdr);
    GridBarrier* bar = reinterpret_cast<GridBarrier*>(ws + o_hdr + sizeof(KmDevStats));
    int* call_status = reinterpret_cast<int*>(ws + o_hdr + sizeof(KmDevStats) + sizeof(GridBarrier));
    do {
        if ((e = cudaMemsetAsync(ws + o_hdr, 0, up(sizeof(KmDevStats) + sizeof(GridBarrier) + 2 * sizeof(int)), s)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(labels, 0xff, (size_t)n * 4, s)) != cudaSuccess) break;
        KppArgs ka{};
        ka.X = emb;
        ka.n = n;
        ka.l = l;
        ka.k = k;
        ka.seed = seed;
        ka.d2[0] = reinterpret_cast<float*>(ws + o_d2);
        ka.d2[1] = reinterpret_cast<float*>(ws + o_d2 + up((size_t)n * 4));
        ka.bsum[0] = reinterpret_cast<double*>(ws + o_bs);
        ka.bsum[1] = reinterpret_cast<double*>(ws + o_bs + up((size_t)G * 8));
        ka.tsum[0] = reinterpret_cast<double*>(ws + o_ts);
        ka.tsum[1] = reinterpret_cast<double*>(ws + o_ts + up((size_t)G * max_tiles * 8));
        ka.max_tiles = max_tiles;
        ka.seeds = reinterpret_cast<int64_t*>(ws + o_seed);
        ka.c32 = reinterpret_cast<float*>(ws + o_c32);
        ka.c64 = reinterpret_cast<double*>(ws + o_c64);
        ka.bar = bar;
        ka.status = call_status;
        ka.limit = wait_limit_ns();
        void* kargs[] = {&ka};
        if ((e = cudaLaunchCooperativeKernel((const void*)kpp, dim3(G), dim3(KM_THREADS), kargs, kpp_smem, s)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s)) != cudaSuccess) break;
        LloydArgs la{};
        la.X = emb;
        la.n = n;
        la.l = l;
        la.k = k;
        la.max_iter = max_iter;
        la.labels = labels;
        la.c32 = ka.c32;
        la.c64 = ka.c64;
        la.partials = reinterpret_cast<double*>(ws + o_part);
        la.inertia_part = reinterpret_cast<double*>(ws + o_inert);
        la.changed_part = reinterpret_cast<int*>(ws + o_chg);
        la.st = st;
        la.bar = bar;
        la.status = call_status;
        la.limit = ka.limit;
        void* largs[] = {&la};
        if ((e = cudaLaunchCooperativeKernel((const void*)lly, dim3(G), dim3(KM_THREADS), largs, lloyd_smem, s)) != cudaSuccess) break;
        if (centroids)
            if ((e = cudaMemcpy2DAsync(centroids, (size_t)l * 8, ka.c64, (size_t)LP * 8, (size_t)l * 8, (size_t)k,
                                       cudaMemcpyDeviceToDevice, s)) != cudaSuccess) break;
        if (seed_idx)
            if ((e = cudaMemcpyAsync(seed_idx, ka.seeds, (size_t)k * 8, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) break;
        if (stats) {
            KmDevStats hst{};
            int hstatus = 0;
            if ((e = cudaMemcpyAsync(&hst, st, sizeof(hst), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
            if ((e = cudaMemcpyAsync(&hstatus, call_status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
            rc = status_from_bits(hstatus);
            stats->iterations = hst.iterations;
            stats->changed = hst.changed;
            stats->empty_events = hst.empty_events;
            stats->device_status = (int32_t)rc;
            stats->inertia = hst.inertia;
            stats->seeding_potential = hst.potential;
        } else {
            int* word = device_status_word();
            if (word) {
                k_merge_status<<<1, 1, 0, s>>>(call_status, word);
                if ((e = cudaGetLastError()) != cudaSuccess) break;
            }
        }
    } while (0);
    cudaError_t ef = cudaFreeAsync(ws, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (ef != cudaSuccess) return cuda_status(ef);
    return rc;
}

}  // namespace fsc

using namespace fsc;

extern "C" fsc_status fsc_kmeans(const float* emb, int64_t n, int l, int ld, int k, uint64_t seed, int max_iter,
                                 int32_t* labels, double* centroids, int64_t* seed_idx, fsc_kmeans_stats* stats,
                                 void* stream) {
    if (!emb || !labels || n < 1 || n > 2147483647LL || l < 1 || l > ld || k < 1 || (int64_t)k > n || k > 1024 ||
        max_iter < 1)
        return FSC_ERR_INVALID_ARG;
    if (ld != 1 && ld != 2 && ld != 4 && ld != 8) return FSC_ERR_INVALID_ARG;
    if ((int64_t)k * ld > 4096) return FSC_ERR_INVALID_ARG;
    const size_t al = (size_t)ld * 4 < 16 ? (size_t)ld * 4 : 16;
    if (reinterpret_cast<uintptr_t>(emb) % al) return FSC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    switch (ld) {
        case 1: return kmeans_lp<1>(emb, (int)n, l, k, seed, max_iter, labels, centroids, seed_idx, stats, s);
        case 2: return kmeans_lp<2>(emb, (int)n, l, k, seed, max_iter, labels, centroids, seed_idx, stats, s);
        case 4: return kmeans_lp<4>(emb, (int)n, l, k, seed, max_iter, labels, centroids, seed_idx, stats, s);
        case 8: return kmeans_lp<8>(emb, (int)n, l, k, seed, max_iter, labels, centroids, seed_idx, stats, s);
    }
    return FSC_ERR_INVALID_ARG;
}

extern "C" fsc_status fsc_cluster(const fsc_graph* g, int k, int l, int t, uint64_t seed, fsc_dtype store,
                                  int max_iter, int32_t* labels, fsc_kmeans_stats* stats, const fsc_embed_opts* opts,
                                  void* stream) {
    if (!g || !labels || l < 1 || l > 8 || k < 1 || (int64_t)k > g->n) return FSC_ERR_INVALID_ARG;
    const int LP = pad_l(l);
    cudaStream_t s = as_stream(stream);
    float* emb = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&emb), (size_t)g->n * LP * 4, s);
    if (e != cudaSuccess) return cuda_status(e);
    fsc_kmeans_stats local{};
    fsc_status rc = fsc_embed(g, l, t, seed, store, emb, opts, stream);
    if (rc == FSC_OK)
        rc = fsc_kmeans(emb, g->n, l, LP, k, seed, max_iter, labels, nullptr, nullptr, stats ? stats : &local, stream);
    cudaError_t ef = cudaFreeAsync(emb, s);
    if (rc == FSC_OK && ef != cudaSuccess) rc = cuda_status(ef);
    if (rc == FSC_OK) {
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) rc = cuda_status(e);
    }
    return rc;
}
