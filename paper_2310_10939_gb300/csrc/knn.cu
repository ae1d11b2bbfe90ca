// k-nearest-neighbour graph of a point set (the Sec. 4.2 pre-processing: the paper clusters the
// 10-NN graph of each dataset).  Reading (the paper gives no more than "the k nearest neighbour
// graph"): float32 squared distances summed over the columns in order without fused multiply-add,
// the knn points j != i of smallest distance (ties to the lower index), symmetrised by union, and
// weights exp(-d2 / sigma^2) with sigma the median of the n * knn directed distances.
//
// Kernels: brute-force neighbour search, one thread per query with its point in registers and
// candidate tiles staged in shared memory (every thread reads the same candidate: broadcast);
// an exact radix selection of the median on the float bits of d2 (non-negative floats order as
// their bit patterns); reverse lists by counting; the union per row; sorted rows and weights.
#include <math.h>

#include "fsc_internal.cuh"

namespace fsc {

constexpr int KNN_THREADS = 256;
constexpr int KNN_TILE = 128;     // candidate points per shared tile
constexpr int KNN_MAX = 16;       // largest neighbour count (list kept in registers)

template <int DIMP>
__global__ void __launch_bounds__(KNN_THREADS) k_knn(const float* __restrict__ X, int n, int dim, int knn,
                                                     int32_t* __restrict__ nbr, float* __restrict__ nd2) {
    __shared__ float s_p[KNN_TILE][DIMP];
    const long long qi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = qi < n;
    float q[DIMP];
#pragma unroll
    for (int c = 0; c < DIMP; ++c) q[c] = (act && c < dim) ? X[qi * dim + c] : 0.f;
    float bd[KNN_MAX];
    int bi[KNN_MAX];
#pragma unroll
    for (int s = 0; s < KNN_MAX; ++s) {
        bd[s] = __int_as_float(0x7f800000);
        bi[s] = 0x7fffffff;
    }
    for (long long t0 = 0; t0 < n; t0 += KNN_TILE) {
        __syncthreads();
        for (int e = threadIdx.x; e < KNN_TILE * DIMP; e += blockDim.x) {
            const int p = e / DIMP, c = e - p * DIMP;
            const long long j = t0 + p;
            s_p[p][c] = (j < n && c < dim) ? X[j * dim + c] : 0.f;
        }
        __syncthreads();
        if (!act) continue;
        const int cnt = (int)min((long long)KNN_TILE, n - t0);
        for (int p = 0; p < cnt; ++p) {
            float d = 0.f;
#pragma unroll
            for (int c = 0; c < DIMP; ++c) {   // padded columns add +0 exactly
                const float df = __fsub_rn(s_p[p][c], q[c]);
                d = __fadd_rn(d, __fmul_rn(df, df));
            }
            const int j = (int)(t0 + p);
            if (j == qi || !(d < bd[KNN_MAX - 1])) continue;
            // sorted insert: candidates arrive in increasing index, so an equal distance never
            // displaces an earlier one (ties stay with the lower index)
            float cd = d;
            int cj = j;
#pragma unroll
            for (int s = 0; s < KNN_MAX; ++s) {
                if (cd < bd[s]) {
                    const float td = bd[s];
                    const int tj = bi[s];
                    bd[s] = cd;
                    bi[s] = cj;
                    cd = td;
                    cj = tj;
                }
            }
        }
    }
    if (act) {
#pragma unroll
        for (int s = 0; s < KNN_MAX; ++s)
            if (s < knn) {
                nbr[qi * knn + s] = bi[s];
                nd2[qi * knn + s] = bd[s];
            }
    }
}

// ---- exact order statistic of the d2 values (radix selection, 8 bits per pass) ----------------
// state: [0] prefix bits, [1] mask of decided bits, [2] rank still to find inside the prefix
__global__ void __launch_bounds__(256) k_sel_hist(const float* __restrict__ v, long long m, int shift,
                                                  const unsigned* __restrict__ state, unsigned* __restrict__ hist) {
    __shared__ unsigned s_h[256];
    s_h[threadIdx.x] = 0u;
    __syncthreads();
    const unsigned prefix = state[0], mask = state[1];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
        const unsigned b = __float_as_uint(v[i]);
        if ((b & mask) == prefix) atomicAdd(&s_h[(b >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (s_h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], s_h[threadIdx.x]);
}

__global__ void k_sel_pick(unsigned* __restrict__ hist, int shift, unsigned* __restrict__ state) {
    if (threadIdx.x != 0) return;
    unsigned r = state[2];
    int bin = 255;
    for (int q = 0; q < 256; ++q) {
        if (r < hist[q]) { bin = q; break; }
        r -= hist[q];
    }
    state[0] |= (unsigned)bin << shift;
    state[1] |= 255u << shift;
    state[2] = r;
    for (int q = 0; q < 256; ++q) hist[q] = 0u;
}

// sigma = mean of the two middle values (or the middle one) of sqrt(d2), float32 square roots
__global__ void k_sigma(const unsigned* __restrict__ lo_state, const unsigned* __restrict__ hi_state, int even,
                        double* __restrict__ sigma) {
    const double a = (double)sqrtf(__uint_as_float(lo_state[0]));
    const double b = (double)sqrtf(__uint_as_float(hi_state[0]));
    *sigma = even ? 0.5 * (a + b) : b;
}

// ---- union of the neighbour lists -----------------------------------------------------------
__global__ void __launch_bounds__(256) k_rev_count(const int32_t* __restrict__ nbr, long long m,
                                                   int* __restrict__ cnt) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (long long)gridDim.x * blockDim.x)
        atomicAdd(&cnt[nbr[e]], 1);
}

// exclusive prefix sums of n counts into out[0..n] (one block, chunks of its width)
__global__ void __launch_bounds__(1024) k_scan(const int* __restrict__ in, long long n, long long* __restrict__ out) {
    __shared__ long long s_w[32];
    __shared__ long long s_carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (long long base = 0; base < n; base += blockDim.x) {
        const long long i = base + threadIdx.x;
        long long v = i < n ? (long long)in[i] : 0;
        long long x = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) s_w[wid] = x;
        __syncthreads();
        if (wid == 0) {
            long long t = lane < (int)(blockDim.x >> 5) ? s_w[lane] : 0;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const long long y = __shfl_up_sync(0xffffffffu, t, off);
                if (lane >= off) t += y;
            }
            s_w[lane] = t;
        }
        __syncthreads();
        const long long incl = x + (wid > 0 ? s_w[wid - 1] : 0) + s_carry;
        if (i < n) out[i] = incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = s_carry;
}

__global__ void __launch_bounds__(256) k_rev_fill(const int32_t* __restrict__ nbr, long long m, int knn,
                                                  const long long* __restrict__ roff, int* __restrict__ fill,
                                                  int32_t* __restrict__ rev) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (long long)gridDim.x * blockDim.x) {
        const int j = nbr[e];
        rev[roff[j] + atomicAdd(&fill[j], 1)] = (int32_t)(e / knn);
    }
}

// per row: its own list plus the reverse entries not already in it
__global__ void __launch_bounds__(256) k_union_count(int n, int knn, const int32_t* __restrict__ nbr,
                                                     const long long* __restrict__ roff,
                                                     const int32_t* __restrict__ rev, int* __restrict__ ucnt) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int own[KNN_MAX];
#pragma unroll
        for (int s = 0; s < KNN_MAX; ++s) own[s] = s < knn ? nbr[i * knn + s] : -1;
        int c = knn;
        for (long long p = roff[i]; p < roff[i + 1]; ++p) {
            const int r = rev[p];
            bool dup = false;
#pragma unroll
            for (int s = 0; s < KNN_MAX; ++s) dup |= own[s] == r;
            c += !dup;
        }
        ucnt[i] = c;
    }
}

__device__ __forceinline__ float sqdist_rows(const float* __restrict__ X, int dim, long long a, long long b) {
    float d = 0.f;
    for (int c = 0; c < dim; ++c) {
        const float df = __fsub_rn(X[b * dim + c], X[a * dim + c]);
        d = __fadd_rn(d, __fmul_rn(df, df));
    }
    return d;
}

// per row: write the union, sort it (insertion sort: rows hold knn plus the reverse entries), and
// the weights exp(-d2 / sigma^2)
__global__ void __launch_bounds__(256) k_union_write(int n, int knn, const float* __restrict__ X, int dim,
                                                     const int32_t* __restrict__ nbr, const long long* __restrict__ roff,
                                                     const int32_t* __restrict__ rev,
                                                     const long long* __restrict__ row_ptr,
                                                     const double* __restrict__ sigma, int32_t* __restrict__ col,
                                                     float* __restrict__ w) {
    const float inv_s2 = (float)(1.0 / (*sigma * *sigma));
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int own[KNN_MAX];
#pragma unroll
        for (int s = 0; s < KNN_MAX; ++s) own[s] = s < knn ? nbr[i * knn + s] : -1;
        const long long o = row_ptr[i];
        long long len = 0;
        for (int s = 0; s < knn; ++s) col[o + len++] = own[s];
        for (long long p = roff[i]; p < roff[i + 1]; ++p) {
            const int r = rev[p];
            bool dup = false;
#pragma unroll
            for (int s = 0; s < KNN_MAX; ++s) dup |= own[s] == r;
            if (!dup) col[o + len++] = r;
        }
        for (long long a = 1; a < len; ++a) {
            const int key = col[o + a];
            long long b = a - 1;
            while (b >= 0 && col[o + b] > key) {
                col[o + b + 1] = col[o + b];
                --b;
            }
            col[o + b + 1] = key;
        }
        if (w)
            for (long long a = 0; a < len; ++a) w[o + a] = expf(-sqdist_rows(X, dim, i, col[o + a]) * inv_s2);
    }
}

template <int DIMP>
static cudaError_t launch_knn(const float* X, int n, int dim, int knn, int32_t* nbr, float* nd2, cudaStream_t s) {
    const unsigned blocks = (unsigned)(((long long)n + KNN_THREADS - 1) / KNN_THREADS);
    k_knn<DIMP><<<blocks, KNN_THREADS, 0, s>>>(X, n, dim, knn, nbr, nd2);
    return cudaGetLastError();
}

}  // namespace fsc

using namespace fsc;

extern "C" fsc_status fsc_knn_graph(const float* points, int64_t n, int dim, int knn, int64_t* row_ptr, int32_t* col,
                                    float* w, int64_t capacity, int64_t* nnz, double* sigma, void* stream) {
    NvtxRange nvtx_range("fsc_knn_graph");
    if (!points || !row_ptr || !col || !nnz || n < 2 || n > 2147483647LL || dim < 1 || dim > 64 || knn < 1 ||
        knn > KNN_MAX || knn >= n || capacity < 2 * n * (int64_t)knn || n * (int64_t)knn > 2147483647LL)
        return FSC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    const long long m = n * (long long)knn;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t b_nbr = up((size_t)m * 4), b_nd2 = up((size_t)m * 4), b_cnt = up((size_t)(n + 1) * 4),
                 b_off = up((size_t)(n + 1) * 8), b_rev = up((size_t)m * 4), b_sel = 256 * 4 + 64;
    char* ws = nullptr;
    cudaError_t e = pool_malloc(reinterpret_cast<void**>(&ws), b_nbr + b_nd2 + 3 * b_cnt + b_off + b_rev + b_sel + 256, s);
    if (e != cudaSuccess) return cuda_status(e);
    int32_t* nbr = reinterpret_cast<int32_t*>(ws);
    float* nd2 = reinterpret_cast<float*>(ws + b_nbr);
    int* cnt = reinterpret_cast<int*>(ws + b_nbr + b_nd2);
    int* fill = reinterpret_cast<int*>(ws + b_nbr + b_nd2 + b_cnt);
    int* ucnt = reinterpret_cast<int*>(ws + b_nbr + b_nd2 + 2 * b_cnt);
    long long* roff = reinterpret_cast<long long*>(ws + b_nbr + b_nd2 + 3 * b_cnt);
    int32_t* rev = reinterpret_cast<int32_t*>(ws + b_nbr + b_nd2 + 3 * b_cnt + b_off);
    char* sel = ws + b_nbr + b_nd2 + 3 * b_cnt + b_off + b_rev;
    unsigned* hist = reinterpret_cast<unsigned*>(sel);
    unsigned* st_lo = reinterpret_cast<unsigned*>(sel + 256 * 4);
    unsigned* st_hi = st_lo + 4;
    double* d_sigma = reinterpret_cast<double*>(sel + 256 * 4 + 32);
    const long long gcap = (long long)device_props().num_sms * 8;
    auto grid = [&](long long items) {
        long long b = (items + 255) / 256;
        return (unsigned)(b < 1 ? 1 : (b > gcap ? gcap : b));
    };
    fsc_status rc = FSC_OK;
    do {
        // 1. neighbours
        if (dim <= 8) e = launch_knn<8>(points, (int)n, dim, knn, nbr, nd2, s);
        else if (dim <= 16) e = launch_knn<16>(points, (int)n, dim, knn, nbr, nd2, s);
        else if (dim <= 32) e = launch_knn<32>(points, (int)n, dim, knn, nbr, nd2, s);
        else e = launch_knn<64>(points, (int)n, dim, knn, nbr, nd2, s);
        if (e != cudaSuccess) break;
        // 2. sigma: ranks m/2 - 1 and m/2 (m even) or m/2 (m odd) of the directed d2
        const unsigned rank_hi = (unsigned)(m / 2), rank_lo = (unsigned)(m % 2 == 0 ? m / 2 - 1 : m / 2);
        unsigned init_lo[4] = {0u, 0u, rank_lo, 0u}, init_hi[4] = {0u, 0u, rank_hi, 0u};
        if ((e = cudaMemsetAsync(hist, 0, 256 * 4, s)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(st_lo, init_lo, 16, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(st_hi, init_hi, 16, cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
        for (unsigned* st : {st_lo, st_hi}) {
            for (int shift = 24; shift >= 0; shift -= 8) {
                k_sel_hist<<<grid(m), 256, 0, s>>>(nd2, m, shift, st, hist);
                k_sel_pick<<<1, 32, 0, s>>>(hist, shift, st);
            }
        }
        k_sigma<<<1, 1, 0, s>>>(st_lo, st_hi, m % 2 == 0 ? 1 : 0, d_sigma);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        // 3. reverse lists
        if ((e = cudaMemsetAsync(cnt, 0, 2 * b_cnt, s)) != cudaSuccess) break;   // cnt and fill
        k_rev_count<<<grid(m), 256, 0, s>>>(nbr, m, cnt);
        k_scan<<<1, 1024, 0, s>>>(cnt, n, roff);
        k_rev_fill<<<grid(m), 256, 0, s>>>(nbr, m, knn, roff, fill, rev);
        // 4. union: counts, row offsets, rows
        k_union_count<<<grid(n), 256, 0, s>>>((int)n, knn, nbr, roff, rev, ucnt);
        k_scan<<<1, 1024, 0, s>>>(ucnt, n, reinterpret_cast<long long*>(row_ptr));
        k_union_write<<<grid(n), 256, 0, s>>>((int)n, knn, points, dim, nbr, roff, rev,
                                             reinterpret_cast<const long long*>(row_ptr), d_sigma, col, w);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        long long hn = 0;
        double hs = 0.0;
        if ((e = cudaMemcpyAsync(&hn, row_ptr + n, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(&hs, d_sigma, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
        *nnz = hn;
        if (sigma) *sigma = hs;
    } while (0);
    pool_free(ws, s);
    if (e != cudaSuccess) rc = cuda_status(e);
    return rc;
}
