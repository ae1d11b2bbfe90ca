// k-means++ and Lloyd on rows of 16 .. 128 float32 (ld = 16, 32, 64, 128): the clustering step of
// Algorithm 2 (Sec. 2.2) for the wide embeddings of the "PM k Vectors" and "k Eigenvectors"
// variants (l = k columns, Sec. 4).
//
// Decision rules and sums are those of kmeans.cu (a point's float32 squared distance summed over
// the columns in order without fused multiply-add; k-means++ takes the smallest index whose exact
// fixed-point prefix of D^2 exceeds floor(U * total / 2^53); Lloyd moves a point only to a strictly
// nearer centroid, ties to the lowest index; centroids are float64 means of exact fixed-point
// sums, an empty cluster keeps its centroid).  The layout differs: a point's row is too wide to
// keep several per thread, so every k-means++ round is one pass kernel (blocks own contiguous
// point ranges and write exact block totals) and one single-block selection kernel, and every
// Lloyd iteration an assignment kernel (one point per thread, its row in registers, centroids in
// shared memory, running sums updated by the points that change cluster) and an update kernel;
// the host stops the loop when an iteration changes no label.  k-means++ skips the distance of a
// point the new centre cannot reach (triangle inequality on the half distance to its nearest
// chosen centre, widened by 1e-5 as in kmeans.cu).
#include <math.h>

#include "kmeans_common.cuh"

namespace fsc {

constexpr int KW_PASS = 256;     // threads of the pass kernels
constexpr int KW_ASSIGN = 128;   // threads of the assignment kernel (a 128-float row in registers)
constexpr int KW_SELECT = 1024;  // threads of the selection kernel (one per pass block at most)
constexpr float KW_EPS = 1e-5f;

struct WideKm {
    const float* X;
    int n, l, k, LP;
    long long chunk;           // points per pass block (contiguous, in index order)
    unsigned long long seed;
    unsigned* amax;            // max |x| over the used columns (float bits)
    float* d2;                 // D^2 per point
    int* near;                 // per point: selection index of its nearest chosen centre
    long long* btot;           // per pass block: exact D^2 total
    int64_t* seeds;
    float* c32;                // k x LP
    double* c64;               // k x LP
    unsigned long long* tot;   // k x (LP + 1): exact running sums of coordinates, then the count
    unsigned long long* misc;  // [0] labels changed, [1] inertia (fixed point), [2] empty-cluster events
    double* dstat;             // [0] inertia of the last assignment, [1] of the first
    int32_t* labels;
};

// float32 squared distance of a row to a centre, columns 0 .. LP-1 in order, no contraction
// (the row in memory, or in registers for the second form)
template <int LP>
__device__ __forceinline__ float dist_rowc(const float* __restrict__ x, const float* __restrict__ c) {
    float acc = 0.f;
#pragma unroll 8
    for (int q = 0; q < LP; ++q) {
        const float d = __fsub_rn(x[q], c[q]);
        acc = __fadd_rn(acc, __fmul_rn(d, d));
    }
    return acc;
}
template <int LP>
__device__ __forceinline__ float dist_reg(const float (&x)[LP], const float* __restrict__ c) {
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < LP; ++q) {
        const float d = __fsub_rn(x[q], c[q]);
        acc = __fadd_rn(acc, __fmul_rn(d, d));
    }
    return acc;
}

template <int LP>
__device__ __forceinline__ void load_wide(const float* __restrict__ X, long long i, int l, float (&x)[LP]) {
#pragma unroll
    for (int q = 0; q < LP / 4; ++q) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(X + (size_t)i * LP) + q);
        x[4 * q] = v.x;
        x[4 * q + 1] = v.y;
        x[4 * q + 2] = v.z;
        x[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int q = 0; q < LP; ++q)
        if (q >= l) x[q] = 0.f;
}

// max |x| over the used columns; the first centre floor(u_0 n)
template <int LP>
__global__ void __launch_bounds__(KW_PASS) k_wkm_start(WideKm a) {
    float m = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (long long)gridDim.x * blockDim.x) {
        float x[LP];
        load_wide<LP>(a.X, i, a.l, x);
#pragma unroll
        for (int q = 0; q < LP; ++q) m = fmaxf(m, fabsf(x[q]));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(a.amax, __float_as_uint(m));
    if (blockIdx.x == 0) {
        __shared__ long long s_i0;
        if (threadIdx.x == 0) {
            const U64x4 r = philox4x64_10(U64x4{0ull, 0ull, 0ull, 0ull}, a.seed, STREAM_KMEANSPP);
            long long i0 = (long long)floor(uniform53(r.x) * (double)a.n);
            if (i0 > a.n - 1) i0 = a.n - 1;
            s_i0 = i0;
            a.seeds[0] = i0;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < LP; q += blockDim.x)
            a.c32[q] = q < a.l ? a.X[(size_t)s_i0 * LP + q] : 0.f;
    }
}

// k-means++ round r >= 1: D^2 against the centre chosen last round, exact block totals
template <int LP>
__global__ void __launch_bounds__(KW_PASS) k_wkm_pass(WideKm a, int r) {
    extern __shared__ float s_half2[];       // r - 1 floats
    __shared__ float s_c[LP];
    __shared__ long long s_red[KW_PASS / 32];
    const float* cnew = a.c32 + (size_t)(r - 1) * LP;
    for (int q = threadIdx.x; q < LP; q += blockDim.x) s_c[q] = __ldcg(cnew + q);
    __syncthreads();
    for (int j = threadIdx.x; j < r - 1; j += blockDim.x) {
        const float h = 0.5f * sqrtf(dist_rowc<LP>(a.c32 + (size_t)j * LP, s_c)) * (1.0f - KW_EPS);
        s_half2[j] = h * h;
    }
    __syncthreads();
    const Scales sc = scales_for(__uint_as_float(__ldcg(a.amax)), a.n, a.l);
    const long long lo = (long long)blockIdx.x * a.chunk, hi = min((long long)a.n, lo + a.chunk);
    long long v = 0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        float dd = 0.f;
        bool need = true;
        if (r > 1) {
            dd = a.d2[i];
            const int na = a.near[i];
            need = !in_range(na, 0, r - 1, BS_WIDE_NEAR) || dd * (1.0f + KW_EPS) * (1.0f + KW_EPS) >= s_half2[na];
        }
        if (need) {
            float x[LP];
            load_wide<LP>(a.X, i, a.l, x);
            const float dn = dist_reg<LP>(x, s_c);
            if (r == 1 || dn < dd) {
                dd = dn;
                a.d2[i] = dn;
                a.near[i] = r - 1;
            }
        }
        v += fixq(dd, sc.Sd);
    }
    v = warp_sum_ll(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) s_red[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < KW_PASS / 32; ++w) t += s_red[w];
        a.btot[blockIdx.x] = t;
    }
}

// One block: the block whose range holds the target (block totals in index order), then the point
// inside it (its D^2 in index order), 1024 points per step; sum(D^2) = 0 picks the lowest index
// not chosen yet.  Writes the pick and its coordinates as centre r.
template <int LP>
__global__ void __launch_bounds__(KW_SELECT) k_wkm_select(WideKm a, int r, int nb) {
    __shared__ long long s_red[KW_SELECT / 32];
    __shared__ long long s_T, s_base, s_run;
    __shared__ int s_blk, s_idx;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const Scales sc = scales_for(__uint_as_float(__ldcg(a.amax)), a.n, a.l);
    const long long v = tid < nb ? __ldcg(a.btot + tid) : 0;
    // inclusive block scan of the block totals
    long long incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += u;
    }
    if (lane == 31) s_red[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        long long t = lane < KW_SELECT / 32 ? s_red[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, t, off);
            if (lane >= off) t += u;
        }
        s_red[lane] = t;
    }
    __syncthreads();
    if (wid > 0) incl += s_red[wid - 1];
    const long long total = s_red[KW_SELECT / 32 - 1];
    if (tid == 0) {
        s_blk = -1;
        s_idx = INT_MAX;
        if (total > 0) {
            const U64x4 rr = philox4x64_10(U64x4{(unsigned long long)r, 0ull, 0ull, 0ull}, a.seed, STREAM_KMEANSPP);
            const unsigned long long U = rr.x >> 11, P = (unsigned long long)total;
            const unsigned long long hi64 = __umul64hi(U, P), lo64 = U * P;
            s_T = (long long)((hi64 << 11) | (lo64 >> 53));   // floor(U * P / 2^53) < P
        }
    }
    __syncthreads();
    if (total > 0) {
        const long long T = s_T;
        if (tid < nb && v > 0 && incl - v <= T && T < incl) {   // exactly one block
            s_blk = tid;
            s_base = incl - v;
        }
        __syncthreads();
        const long long lo = (long long)s_blk * a.chunk, hi = min((long long)a.n, lo + a.chunk);
        if (tid == 0) s_run = s_base;
        __syncthreads();
        for (long long i0 = lo; i0 < hi; i0 += KW_SELECT) {
            const long long i = i0 + tid;
            const long long q = i < hi ? fixq(__ldcg(a.d2 + i), sc.Sd) : 0;
            long long s = q;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const long long u = __shfl_up_sync(0xffffffffu, s, off);
                if (lane >= off) s += u;
            }
            __syncthreads();
            if (lane == 31) s_red[wid] = s;
            __syncthreads();
            if (wid == 0) {
                long long t = s_red[lane];
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const long long u = __shfl_up_sync(0xffffffffu, t, off);
                    if (lane >= off) t += u;
                }
                s_red[lane] = t;
            }
            __syncthreads();
            if (wid > 0) s += s_red[wid - 1];
            const long long run = s_run + s;
            if (q > 0 && run > T && run - q <= T) atomicMin(&s_idx, (int)i);
            __syncthreads();
            if (s_idx != INT_MAX) break;
            if (tid == 0) s_run += s_red[KW_SELECT / 32 - 1];
            __syncthreads();
        }
    }
    __syncthreads();
    if (tid == 0 && s_idx == INT_MAX) {   // sum(D^2) = 0: the lowest index not chosen yet
        long long cand = 0;
        for (;; ++cand) {
            bool taken = false;
            for (int q = 0; q < r; ++q)
                if (a.seeds[q] == cand) { taken = true; break; }
            if (!taken) break;
        }
        s_idx = (int)cand;
    }
    __syncthreads();
    if (tid == 0) a.seeds[r] = s_idx;
    for (int q = tid; q < LP; q += blockDim.x)
        a.c32[(size_t)r * LP + q] = q < a.l ? a.X[(size_t)s_idx * LP + q] : 0.f;
}

// Lloyd assignment: nearest centroid of each point (strict '<' in index order), two centroids per
// pass over the row for two independent add chains; a point that changes cluster moves its exact
// coordinates between the running sums; the fixed-point inertia of the assignment accumulates.
template <int LP>
__global__ void __launch_bounds__(KW_ASSIGN) k_wkm_assign(WideKm a) {
    extern __shared__ float s_cen[];   // k x LP
    __shared__ long long s_ri[KW_ASSIGN / 32];
    __shared__ int s_rc[KW_ASSIGN / 32];
    const int k = a.k;
    for (int q = threadIdx.x; q < k * LP; q += blockDim.x) s_cen[q] = __ldcg(a.c32 + q);
    __syncthreads();
    const Scales sc = scales_for(__uint_as_float(__ldcg(a.amax)), a.n, a.l);
    long long inert = 0;
    int changed = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (long long)gridDim.x * blockDim.x) {
        float x[LP];
        load_wide<LP>(a.X, i, a.l, x);
        float best = dist_reg<LP>(x, s_cen);
        int bj = 0;
        int j = 1;
        for (; j + 1 < k; j += 2) {
            const float* c0 = s_cen + (size_t)j * LP;
            const float* c1 = c0 + LP;
            float d0 = 0.f, d1 = 0.f;
#pragma unroll
            for (int q = 0; q < LP; ++q) {
                const float e0 = __fsub_rn(x[q], c0[q]), e1 = __fsub_rn(x[q], c1[q]);
                d0 = __fadd_rn(d0, __fmul_rn(e0, e0));
                d1 = __fadd_rn(d1, __fmul_rn(e1, e1));
            }
            if (d0 < best) {
                best = d0;
                bj = j;
            }
            if (d1 < best) {
                best = d1;
                bj = j + 1;
            }
        }
        if (j < k) {
            const float d0 = dist_reg<LP>(x, s_cen + (size_t)j * LP);
            if (d0 < best) {
                best = d0;
                bj = j;
            }
        }
        inert += fixq(best, sc.Sd);
        const int old = a.labels[i];
        if (old != bj) {
            a.labels[i] = bj;
            ++changed;
            unsigned long long* to = a.tot + (size_t)bj * (LP + 1);
            unsigned long long* from =
                old >= 0 && in_range(old, 0, k, BS_WIDE_LABEL) ? a.tot + (size_t)old * (LP + 1) : nullptr;
#pragma unroll
            for (int q = 0; q < LP; ++q) {
                const long long v = q < a.l ? fixq(x[q], sc.Sx) : 0;
                if (v) {
                    atomicAdd(to + q, (unsigned long long)v);
                    if (from) atomicAdd(from + q, (unsigned long long)(-v));
                }
            }
            atomicAdd(to + LP, 1ull);
            if (from) atomicAdd(from + LP, ~0ull);   // -1
        }
    }
    inert = warp_sum_ll(inert);
    for (int off = 16; off > 0; off >>= 1) changed += __shfl_xor_sync(0xffffffffu, changed, off);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s_ri[wid] = inert;
        s_rc[wid] = changed;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long ti = 0;
        int tc = 0;
        for (int w = 0; w < KW_ASSIGN / 32; ++w) {
            ti += s_ri[w];
            tc += s_rc[w];
        }
        if (ti) atomicAdd(a.misc + 1, (unsigned long long)ti);
        if (tc) atomicAdd(a.misc, (unsigned long long)tc);
    }
}

// Centroid update: c_j = (exact sum) / count in float64, then float32; an empty cluster keeps its
// centroid.  Also turns the assignment's exact inertia into float64 (and keeps the first one).
__global__ void k_wkm_update(WideKm a, int it) {
    const int LP = a.LP;
    const Scales sc = scales_for(__uint_as_float(__ldcg(a.amax)), a.n, a.l);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < a.k * LP; q += gridDim.x * blockDim.x) {
        const int j = q / LP, c = q - j * LP;
        const long long cnt = (long long)__ldcg(a.tot + (size_t)j * (LP + 1) + LP);
        if (cnt > 0 && c < a.l) {
            const long long s = (long long)__ldcg(a.tot + (size_t)j * (LP + 1) + c);
            const double m = ((double)s * pow2d(-sc.Sx)) / (double)cnt;
            a.c64[q] = m;
            a.c32[q] = (float)m;
        }
        if (c == 0 && cnt == 0) atomicAdd(a.misc + 2, 1ull);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double in = (double)(long long)__ldcg(a.misc + 1) * pow2d(-sc.Sd);
        a.dstat[0] = in;
        if (it == 1) a.dstat[1] = in;
    }
}

__global__ void k_wkm_c64_init(WideKm a) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < a.k * a.LP; q += gridDim.x * blockDim.x)
        a.c64[q] = (double)__ldcg(a.c32 + q);
}

template <int LP>
static fsc_status kmeans_wide_lp(const float* emb, int n, int l, int k, uint64_t seed, int max_iter, int32_t* labels,
                                 double* centroids, int64_t* seed_idx, fsc_kmeans_stats* stats, cudaStream_t s) {
    const int nsm = device_props().num_sms;
    int nb = nsm * 4;
    if (nb > KW_SELECT) nb = KW_SELECT;
    long long chunk = ((long long)n + nb - 1) / nb;
    nb = (int)(((long long)n + chunk - 1) / chunk);
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t b_misc = up(8 * 8), b_amax = 256, b_d2 = up((size_t)n * 4), b_near = up((size_t)n * 4),
                 b_btot = up((size_t)nb * 8), b_seed = up((size_t)k * 8), b_c32 = up((size_t)k * LP * 4),
                 b_c64 = up((size_t)k * LP * 8), b_tot = up((size_t)k * (LP + 1) * 8);
    char* ws = nullptr;
    cudaError_t e = pool_malloc(reinterpret_cast<void**>(&ws),
                                b_misc + b_amax + b_d2 + b_near + b_btot + b_seed + b_c32 + b_c64 + b_tot, s);
    if (e != cudaSuccess) return cuda_status(e);
    WideKm a{};
    char* p = ws;
    a.misc = reinterpret_cast<unsigned long long*>(p);
    a.dstat = reinterpret_cast<double*>(p + 32);
    p += b_misc;
    a.amax = reinterpret_cast<unsigned*>(p);
    p += b_amax;
    a.d2 = reinterpret_cast<float*>(p);
    p += b_d2;
    a.near = reinterpret_cast<int*>(p);
    p += b_near;
    a.btot = reinterpret_cast<long long*>(p);
    p += b_btot;
    a.seeds = reinterpret_cast<int64_t*>(p);
    p += b_seed;
    a.c32 = reinterpret_cast<float*>(p);
    p += b_c32;
    a.c64 = reinterpret_cast<double*>(p);
    p += b_c64;
    a.tot = reinterpret_cast<unsigned long long*>(p);
    a.X = emb;
    a.n = n;
    a.l = l;
    a.k = k;
    a.LP = LP;
    a.chunk = chunk;
    a.seed = seed;
    a.labels = labels;
    fsc_status rc = FSC_OK;
    const size_t cen_smem = (size_t)k * LP * 4;
    do {
        if ((e = cudaMemsetAsync(ws, 0, b_misc + b_amax, s)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(a.tot, 0, b_tot, s)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(a.c32, 0, b_c32, s)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(labels, 0xff, (size_t)n * 4, s)) != cudaSuccess) break;
        int sb = (n + KW_PASS - 1) / KW_PASS;
        if (sb > nsm * 8) sb = nsm * 8;
        k_wkm_start<LP><<<sb, KW_PASS, 0, s>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((size_t)k * 4 > 48 * 1024 &&
            (e = cudaFuncSetAttribute(k_wkm_pass<LP>, cudaFuncAttributeMaxDynamicSharedMemorySize, k * 4)) != cudaSuccess)
            break;
        for (int r = 1; r < k && e == cudaSuccess; ++r) {
            k_wkm_pass<LP><<<nb, KW_PASS, (size_t)(r - 1 > 0 ? r - 1 : 1) * 4, s>>>(a, r);
            k_wkm_select<LP><<<1, KW_SELECT, 0, s>>>(a, r, nb);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) break;
        k_wkm_c64_init<<<(k * LP + 255) / 256, 256, 0, s>>>(a);
        if (cen_smem > 48 * 1024 &&
            (e = cudaFuncSetAttribute(k_wkm_assign<LP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cen_smem)) !=
                cudaSuccess)
            break;
        int ab = (n + KW_ASSIGN - 1) / KW_ASSIGN;
        if (ab > nsm * 16) ab = nsm * 16;
        unsigned long long hm[3] = {0, 0, 0};
        int it = 0;
        for (it = 1; it <= max_iter; ++it) {
            if ((e = cudaMemsetAsync(a.misc, 0, 16, s)) != cudaSuccess) break;
            k_wkm_assign<LP><<<ab, KW_ASSIGN, cen_smem, s>>>(a);
            k_wkm_update<<<(k * LP + 255) / 256, 256, 0, s>>>(a, it);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            if ((e = cudaMemcpyAsync(hm, a.misc, sizeof(hm), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
            if (hm[0] == 0 || it == max_iter) break;
        }
        if (e != cudaSuccess) break;
        double ds[2] = {0.0, 0.0};
        if ((e = cudaMemcpyAsync(ds, a.dstat, sizeof(ds), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
        if (centroids &&
            (e = cudaMemcpy2DAsync(centroids, (size_t)l * 8, a.c64, (size_t)LP * 8, (size_t)l * 8, (size_t)k,
                                   cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            break;
        if (seed_idx && (e = cudaMemcpyAsync(seed_idx, a.seeds, (size_t)k * 8, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
            break;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
        if (stats) {
            stats->iterations = it > max_iter ? max_iter : it;
            stats->changed = (int32_t)hm[0];
            stats->empty_events = (int32_t)hm[2];
            stats->device_status = FSC_OK;
            stats->inertia = ds[0];
            stats->seeding_potential = ds[1];
        }
    } while (0);
    const cudaError_t ef = pool_free(ws, s);
    if (e != cudaSuccess) rc = cuda_status(e);
    else if (ef != cudaSuccess) rc = cuda_status(ef);
    return rc;
}

fsc_status kmeans_wide(const float* emb, int n, int l, int ld, int k, uint64_t seed, int max_iter, int32_t* labels,
                       double* centroids, int64_t* seed_idx, fsc_kmeans_stats* stats, cudaStream_t s) {
    switch (ld) {
        case 16: return kmeans_wide_lp<16>(emb, n, l, k, seed, max_iter, labels, centroids, seed_idx, stats, s);
        case 32: return kmeans_wide_lp<32>(emb, n, l, k, seed, max_iter, labels, centroids, seed_idx, stats, s);
        case 64: return kmeans_wide_lp<64>(emb, n, l, k, seed, max_iter, labels, centroids, seed_idx, stats, s);
        case 128: return kmeans_wide_lp<128>(emb, n, l, k, seed, max_iter, labels, centroids, seed_idx, stats, s);
    }
    return FSC_ERR_INVALID_ARG;
}

FSC_BOUNDS_READER(kmeans_wide)

}  // namespace fsc
