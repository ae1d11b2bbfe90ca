// Batched Algorithm 2: thousands of graphs of uneven size in one persistent launch.
//
// The batch is the disjoint union of its graphs, given as one CSR with global vertex ids.
// A persistent kernel takes graphs from an atomic work queue, largest first (longest
// processing time order), and one 512-thread CTA runs a whole graph: Gaussian start block,
// t power iterations separated by block barriers, then block-local k-means++ and Lloyd.  CTAs
// never wait on each other, so the launch has no inter-CTA spin wait at all.  Each graph uses
// the same per-row power step (power_row) and the same exact fixed-point k-means rules as the
// single-graph entry points, so its labels equal those of fsc_cluster with the same lanes per
// row.  The launch sequence (queue reset, stats reset, kernel) is captured once into a CUDA
// graph and replayed by fsc_batch_run.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "kmeans_common.cuh"
#include "spmm.cuh"

namespace fsc {

int choose_threads_per_row(const fsc_graph* g, int requested, int LP, int store);
int tuned_threads_per_row(double avg_degree, int LP, int store, bool weighted);   // 0 = no entry
fsc_status autotune_graph(fsc_graph* g, int l, fsc_dtype store, int* best, float* us, cudaStream_t s);

struct BatchGraph {
    long long v0;        // first global vertex
    long long zoff;      // offset (elements of the storage type) of the two iterate buffers
    long long eoff;      // offset (floats) of the float32 embedding
    long long doff;      // offset (floats) of the D^2 scratch
    long long toff;      // offset (int64) of the tile sums
    long long soff;      // offset (int64) of the k k-means++ picks
    long long coff;      // offset (doubles) of the k x LP centroids
    unsigned long long seed;
    int n, k, l, LP, t, tpr, ntab, gid;
};

struct BatchArgs {
    const BatchGraph* graphs;
    int num_graphs;
    int* queue;
    const int64_t* row_ptr;
    const int32_t* col;
    const float* w;
    const float* dinv;
    const float* invdeg;
    void* zarena;
    float* earena;
    float* darena;
    long long* tarena;
    int64_t* seeds;
    double* cents;
    int32_t* labels;
    KmDevStats* stats;
    int max_iter;
};

// ---- block-local Algorithm 2 pieces ---------------------------------------------------------

template <int LP, typename TS>
__device__ void init_block(const BatchGraph& g, const float* __restrict__ dinv, TS* z, float* cm) {
    const int tid = threadIdx.x;
    const long long n = g.n, total = n * g.l, nblk = (total + 3) / 4;
    const long long work = nblk > n ? nblk : n;
    for (long long b = tid; b < work; b += KM_THREADS) {
        if (b < nblk) {
            const U64x4 r = philox4x64_10(U64x4{(unsigned long long)b, 0ull, 0ull, 0ull}, g.seed, STREAM_X0);
            const unsigned long long wd[4] = {r.x, r.y, r.z, r.w};
            float zz[4];
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const float u1 = uniform24(wd[2 * p]);
                const float u2 = uniform24(wd[2 * p + 1]);
                const float rad = sqrtf(-2.0f * logf(u1));
                float sn, cs;
                sincospif(2.0f * u2, &sn, &cs);
                zz[2 * p] = rad * cs;
                zz[2 * p + 1] = rad * sn;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const long long e = 4 * b + j;
                if (e < total) {
                    const int c = (int)(e / n);
                    const long long i = e - (long long)c * n;
                    const float v = dinv[i] * zz[j];
                    z[i * LP + c] = from_f32<TS>(v);
                    atomicMax(reinterpret_cast<unsigned*>(cm) + c, __float_as_uint(fabsf(v)));
                }
            }
        }
        if (b < n)
            for (int c = g.l; c < LP; ++c) z[b * LP + c] = from_f32<TS>(0.f);
    }
}

template <int LP, typename TS, int G, bool W>
__device__ void power_block(const BatchGraph& g, const BatchArgs& a, TS* zA, TS* zB, float* emb, float* s_cm,
                            int* s_E) {
    constexpr int U = G <= 8 ? 4 : 2;
    constexpr int RPW = 32 / G;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, sub = lane % G, grp = lane / G;
    const int64_t* rp = a.row_ptr + g.v0;
    const float* invdeg = a.invdeg + g.v0;
    for (int it = 0; it < g.t; ++it) {
        const bool last = it == g.t - 1;
        float scale[LP];
#pragma unroll
        for (int c = 0; c < LP; ++c)
            scale[c] = last ? pow2i(s_E[c]) : pow2i(-exponent_of(s_cm[c]));
        __syncthreads();
        if (!last && tid < LP) {
            s_E[tid] += exponent_of(s_cm[tid]);
            s_cm[tid] = 0.f;
        }
        __syncthreads();
        const TS* zin = (it & 1) ? zB : zA;
        TS* zout = (it & 1) ? zA : zB;
        float cmx[LP];
#pragma unroll
        for (int c = 0; c < LP; ++c) cmx[c] = 0.f;
        for (long long base = (long long)wid * RPW; base < g.n; base += (long long)KM_WARPS * RPW) {
            const long long row = base + grp;
            float y[LP];
            bool wrote;
            if (last)
                wrote = power_row<LP, TS, float, G, U, W, false>(row < g.n, row, sub, rp, a.col, a.w, invdeg, zin,
                                                                 emb, g.v0, scale, y);
            else
                wrote = power_row<LP, TS, TS, G, U, W, false>(row < g.n, row, sub, rp, a.col, a.w, invdeg, zin,
                                                              zout, g.v0, scale, y);
            if (wrote) {
#pragma unroll
                for (int c = 0; c < LP; ++c) cmx[c] = fmaxf(cmx[c], fabsf(y[c]));
            }
        }
        if (!last) {
#pragma unroll
            for (int c = 0; c < LP; ++c) {
                float m = cmx[c];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
                if (lane == 0 && m > 0.f) atomicMax(reinterpret_cast<unsigned*>(s_cm) + c, __float_as_uint(m));
            }
        }
        __syncthreads();
    }
}

template <int LP>
__device__ float block_absmax(const float* X, int n, int l) {
    __shared__ unsigned s_amax;
    if (threadIdx.x == 0) s_amax = 0u;
    __syncthreads();
    float m = 0.f;
    for (long long i = threadIdx.x; i < n; i += KM_THREADS) {
#pragma unroll
        for (int c = 0; c < LP; ++c)
            if (c < l) m = fmaxf(m, fabsf(__ldcg(X + (size_t)i * LP + c)));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(&s_amax, __float_as_uint(m));
    __syncthreads();
    const float A = __uint_as_float(s_amax);
    __syncthreads();
    return A;
}

template <int LP>
__device__ __forceinline__ void load_point_cg(const float* X, long long i, int l, float (&x)[LP]) {
#pragma unroll
    for (int c = 0; c < LP; ++c) x[c] = c < l ? __ldcg(X + (size_t)i * LP + c) : 0.f;
}

template <int LP>
__device__ void kpp_block(const float* X, int n, int l, int k, unsigned long long seed, const Scales& sc, float* D2,
                          long long* tiles, int* chosen, float* cent, int64_t* seeds_out) {
    __shared__ long long s_red[KM_WARPS];
    __shared__ float s_c[LP];
    __shared__ long long s_total, s_T, s_base;
    __shared__ int s_tile, s_idx;
    const int tid = threadIdx.x;
    if (tid == 0) {
        const U64x4 r = philox4x64_10(U64x4{0ull, 0ull, 0ull, 0ull}, seed, STREAM_KMEANSPP);
        long long i0 = (long long)floor(uniform53(r.x) * (double)n);
        if (i0 > n - 1) i0 = n - 1;
        chosen[0] = (int)i0;
    }
    __syncthreads();
    const int ntiles = (n + KM_TILE - 1) / KM_TILE;
    for (int r = 1; r < k; ++r) {
        if (tid < LP) s_c[tid] = tid < l ? __ldcg(X + (size_t)chosen[r - 1] * LP + tid) : 0.f;
        if (tid == 0) s_total = 0;
        __syncthreads();
        for (int tl = 0; tl < ntiles; ++tl) {
            const long long i0 = (long long)tl * KM_TILE + (long long)KM_PPT * tid;
            long long v = 0;
#pragma unroll
            for (int u = 0; u < KM_PPT; ++u) {
                if (i0 + u < n) {
                    float x[LP];
                    load_point_cg<LP>(X, i0 + u, l, x);
                    float dd = sqdist<LP>(x, s_c);
                    if (r > 1) dd = fminf(dd, D2[i0 + u]);
                    D2[i0 + u] = dd;
                    v += fixq(dd, sc.Sd);
                }
            }
            const long long ts = block_sum_ll(v, s_red);
            if (tid == 0) {
                tiles[tl] = ts;
                s_total += ts;
            }
        }
        __syncthreads();
        if (tid == 0) {
            const long long total = s_total;
            if (total <= 0) {
                s_idx = lowest_unchosen(chosen, r);
                s_tile = -1;
            } else {
                const U64x4 rr = philox4x64_10(U64x4{(unsigned long long)r, 0ull, 0ull, 0ull}, seed, STREAM_KMEANSPP);
                const unsigned long long U = rr.x >> 11, P = (unsigned long long)total;
                const unsigned long long hi64 = __umul64hi(U, P), lo64 = U * P;
                const long long T = (long long)((hi64 << 11) | (lo64 >> 53));
                long long run = 0;
                int tsel = ntiles - 1;
                for (int q = 0; q < ntiles; ++q) {
                    const long long v = tiles[q];
                    if (run + v > T) { tsel = q; break; }
                    run += v;
                }
                s_tile = tsel;
                s_base = run;
                s_T = T;
                s_idx = INT_MAX;
            }
        }
        __syncthreads();
        if (s_tile >= 0) {
            const long long i0 = (long long)s_tile * KM_TILE + (long long)KM_PPT * tid;
            long long q[KM_PPT];
            long long v = 0;
#pragma unroll
            for (int u = 0; u < KM_PPT; ++u) {
                q[u] = i0 + u < n ? fixq(__ldcg(D2 + i0 + u), sc.Sd) : 0;
                v += q[u];
            }
            long long run = block_scan_ll(v, s_red) - v + s_base;
#pragma unroll
            for (int u = 0; u < KM_PPT; ++u) {
                run += q[u];
                if (q[u] > 0 && run > s_T) {
                    atomicMin(&s_idx, (int)(i0 + u));
                    break;
                }
            }
            __syncthreads();
            if (tid == 0 && s_idx == INT_MAX) s_idx = lowest_unchosen(chosen, r);
        }
        __syncthreads();
        if (tid == 0) chosen[r] = s_idx;
        __syncthreads();
    }
    for (int q = tid; q < k * LP; q += KM_THREADS) {
        const int j = q / LP, c = q % LP;
        cent[q] = c < l ? __ldcg(X + (size_t)chosen[j] * LP + c) : 0.f;
    }
    for (int q = tid; q < k; q += KM_THREADS) seeds_out[q] = chosen[q];
    __syncthreads();
}

template <int LP>
__device__ void lloyd_block(const float* X, int n, int l, int k, int max_iter, const Scales& sc, int32_t* labels,
                            float* s_c, double* s_c64, unsigned long long* s_tab, int ntab, KmDevStats* st) {
    __shared__ long long s_red[KM_WARPS];
    __shared__ int s_redi[KM_WARPS];
    const int tid = threadIdx.x, wid = tid >> 5;
    const size_t rowlen = (size_t)k * (LP + 1);
    unsigned long long* my_tab = s_tab + (size_t)(wid % ntab) * rowlen;
    for (long long i = tid; i < n; i += KM_THREADS) labels[i] = -1;
    for (int q = tid; q < k * LP; q += KM_THREADS) s_c64[q] = (double)s_c[q];
    int empty = 0;
    const int ntiles = (n + KM_TILE - 1) / KM_TILE;
    for (int it = 1; it <= max_iter; ++it) {
        for (size_t q = tid; q < (size_t)ntab * rowlen; q += KM_THREADS) s_tab[q] = 0ull;
        __syncthreads();
        long long inert = 0;
        int changed = 0;
        Slot<LP> sl[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            sl[q].j = -1;
            sl[q].cnt = 0;
#pragma unroll
            for (int c = 0; c < LP; ++c) sl[q].s[c] = 0;
        }
        for (int tl = 0; tl < ntiles; ++tl) {
            const long long i0 = (long long)tl * KM_TILE + (long long)KM_PPT * tid;
            float x[KM_PPT][LP];
            int old[KM_PPT];
#pragma unroll
            for (int u = 0; u < KM_PPT; ++u) {
                if (i0 + u < n) {
                    load_point_cg<LP>(X, i0 + u, l, x[u]);
                    old[u] = __ldcg(labels + i0 + u);
                } else {
#pragma unroll
                    for (int c = 0; c < LP; ++c) x[u][c] = 0.f;
                    old[u] = 0;
                }
            }
            float best[KM_PPT];
            int bj[KM_PPT];
#pragma unroll
            for (int u = 0; u < KM_PPT; ++u) {
                best[u] = __int_as_float(0x7f800000);
                bj[u] = 0;
            }
            for (int j = 0; j < k; ++j) {
                float cj[LP];
#pragma unroll
                for (int c = 0; c < LP; ++c) cj[c] = s_c[j * LP + c];
#pragma unroll
                for (int u = 0; u < KM_PPT; ++u) {
                    const float d = sqdist<LP>(x[u], cj);
                    if (d < best[u]) { best[u] = d; bj[u] = j; }
                }
            }
#pragma unroll
            for (int u = 0; u < KM_PPT; ++u) {
                if (i0 + u >= n) break;
                const int lab = bj[u];
                changed += old[u] != lab;
                labels[i0 + u] = lab;
                inert += fixq(best[u], sc.Sd);
                int q;
                if (sl[0].j == lab) q = 0;
                else if (sl[1].j == lab) q = 1;
                else {
                    slot_flush<LP>(sl[1], my_tab);
                    sl[1] = sl[0];
                    sl[0].j = lab;
                    sl[0].cnt = 0;
#pragma unroll
                    for (int c = 0; c < LP; ++c) sl[0].s[c] = 0;
                    q = 0;
                }
                if (q == 1) {
                    const Slot<LP> t = sl[0];
                    sl[0] = sl[1];
                    sl[1] = t;
                }
#pragma unroll
                for (int c = 0; c < LP; ++c) sl[0].s[c] += fixq(x[u][c], sc.Sx);
                ++sl[0].cnt;
            }
        }
        slot_flush_warp<LP>(sl[0], my_tab);
        slot_flush_warp<LP>(sl[1], my_tab);
        __syncthreads();
        for (size_t q = tid; q < rowlen; q += KM_THREADS) {
            unsigned long long v = s_tab[q];
            for (int t = 1; t < ntab; ++t) v += s_tab[(size_t)t * rowlen + q];
            s_tab[q] = v;
        }
        inert = block_sum_ll(inert, s_red);
        changed = block_sum_i(changed, s_redi);
        __syncthreads();
        for (int q = tid; q < k * LP; q += KM_THREADS) {
            const int j = q / LP, c = q % LP;
            const long long cnt = (long long)s_tab[(size_t)j * (LP + 1) + LP];
            if (cnt > 0) {
                const double m = ((double)(long long)s_tab[(size_t)j * (LP + 1) + c] * pow2d(-sc.Sx)) / (double)cnt;
                s_c64[q] = m;
                s_c[q] = (float)m;
            } else if (c == 0) {
                ++empty;
            }
        }
        __syncthreads();
        if (tid == 0) {
            const double iv = (double)inert * pow2d(-sc.Sd);
            st->inertia = iv;
            if (it == 1) st->potential = iv;
            st->iterations = it;
            st->changed = changed;
        }
        if (changed == 0 || it == max_iter) break;
    }
    const int e = block_sum_i(empty, s_redi);
    if (tid == 0) st->empty_events = e;
    __syncthreads();
}

template <int LP, typename TS, bool W>
__device__ void run_graph(const BatchArgs& a, const BatchGraph& g, unsigned char* smem) {
    __shared__ float s_cm[8];
    __shared__ int s_E[8];
    const int tid = threadIdx.x;
    TS* zA = static_cast<TS*>(a.zarena) + g.zoff;
    TS* zB = zA + (size_t)g.n * LP;
    float* emb = a.earena + g.eoff;
    if (tid < 8) {
        s_cm[tid] = 0.f;
        s_E[tid] = 0;
    }
    __syncthreads();
    // 1. Gaussian start block in embedding coordinates, Z0 = D^-1/2 X0
    if (g.t == 0) init_block<LP, float>(g, a.dinv + g.v0, emb, s_cm);   // t = 0: D^-1/2 X0 itself
    else init_block<LP, TS>(g, a.dinv + g.v0, zA, s_cm);
    __syncthreads();
    // 2. t power iterations; the last one writes the float32 embedding
    if (g.t > 0) {
        switch (g.tpr) {
            case 4: power_block<LP, TS, 4, W>(g, a, zA, zB, emb, s_cm, s_E); break;
            case 8: power_block<LP, TS, 8, W>(g, a, zA, zB, emb, s_cm, s_E); break;
            case 16: power_block<LP, TS, 16, W>(g, a, zA, zB, emb, s_cm, s_E); break;
            default: power_block<LP, TS, 32, W>(g, a, zA, zB, emb, s_cm, s_E); break;
        }
    }
    __syncthreads();
    // 3. k-means++ and Lloyd on the embedding rows
    const float A = block_absmax<LP>(emb, g.n, g.l);
    const Scales sc = scales_for(A, g.n, g.l);
    float* s_c = reinterpret_cast<float*>(smem);
    double* s_c64 = reinterpret_cast<double*>(smem + (((size_t)g.k * LP * 4 + 15) & ~(size_t)15));
    int* s_chosen = reinterpret_cast<int*>(s_c64 + (size_t)g.k * LP);
    unsigned long long* s_tab =
        reinterpret_cast<unsigned long long*>(smem + ((((size_t)g.k * LP * 4 + 15) & ~(size_t)15) +
                                                      (size_t)g.k * LP * 8 + (((size_t)g.k * 4 + 15) & ~(size_t)15)));
    KmDevStats* st = a.stats + g.gid;
    kpp_block<LP>(emb, g.n, g.l, g.k, g.seed, sc, a.darena + g.doff, a.tarena + g.toff, s_chosen, s_c,
                  a.seeds + g.soff);
    lloyd_block<LP>(emb, g.n, g.l, g.k, a.max_iter, sc, a.labels + g.v0, s_c, s_c64, s_tab, g.ntab, st);
    for (int q = tid; q < g.k * LP; q += KM_THREADS) a.cents[g.coff + q] = s_c64[q];
    __syncthreads();
}

template <typename TS, bool W>
__global__ void __launch_bounds__(KM_THREADS, 1) k_batch(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char bsmem[];
    __shared__ int s_q;
    for (;;) {
        if (threadIdx.x == 0) s_q = atomicAdd(a.queue, 1);
        __syncthreads();
        const int q = s_q;
        __syncthreads();
        if (q >= a.num_graphs) break;
        const BatchGraph g = a.graphs[q];
        switch (g.LP) {
            case 1: run_graph<1, TS, W>(a, g, bsmem); break;
            case 2: run_graph<2, TS, W>(a, g, bsmem); break;
            case 4: run_graph<4, TS, W>(a, g, bsmem); break;
            default: run_graph<8, TS, W>(a, g, bsmem); break;
        }
    }
}

// Every edge of a row of graph g must stay inside graph g's vertex range (block-diagonal union).
__global__ void __launch_bounds__(256) k_batch_check(long long nv, const int64_t* __restrict__ rp,
                                                     const int32_t* __restrict__ col,
                                                     const long long* __restrict__ voff, int G,
                                                     int* __restrict__ status) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
        int lo = 0, hi = G;                      // graph of row i: largest g with voff[g] <= i
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (voff[mid] <= i) lo = mid; else hi = mid;
        }
        const long long a = voff[lo], b = voff[lo + 1];
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            const long long j = col[p];
            if (j < a || j >= b) { atomicOr(status, ST_INDEX_RANGE); break; }
        }
    }
}

__global__ void k_gather_boundaries(const int64_t* __restrict__ rp, const long long* __restrict__ voff, int G,
                                    long long* __restrict__ out) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g <= G) out[g] = rp[voff[g]];
}

}  // namespace fsc

using namespace fsc;

struct fsc_batch {
    int device = 0;
    int num_graphs = 0;
    fsc_graph* uni = nullptr;            // the union graph (degrees, validation)
    BatchGraph* d_graphs = nullptr;
    int* d_queue = nullptr;
    void* zarena = nullptr;
    float* earena = nullptr;
    float* darena = nullptr;
    long long* tarena = nullptr;
    int64_t* seeds = nullptr;
    double* cents = nullptr;
    KmDevStats* stats = nullptr;
    int32_t* labels = nullptr;
    std::vector<BatchGraph> h_graphs;    // in queue order
    std::vector<long long> seed_off;     // by graph id
    std::vector<long long> cent_off;     // by graph id
    std::vector<int> k_of;
    std::vector<int> l_of;
    long long seeds_total = 0, cents_total = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int store = 0;
    size_t smem = 0;
};

static void batch_free(fsc_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->d_graphs);
    cudaFree(b->d_queue);
    cudaFree(b->zarena);
    cudaFree(b->earena);
    cudaFree(b->darena);
    cudaFree(b->tarena);
    cudaFree(b->seeds);
    cudaFree(b->cents);
    cudaFree(b->stats);
    if (b->uni) fsc_destroy_graph(b->uni);
    delete b;
}

extern "C" fsc_status fsc_batch_create(const fsc_batch_desc* d, void* stream, fsc_batch** out) {
    if (!d || !out || d->num_graphs < 1 || !d->vertex_offset || !d->row_ptr || !d->k || !d->seed || !d->labels)
        return FSC_ERR_INVALID_ARG;
    if ((d->store != FSC_F32 && d->store != FSC_BF16) || d->max_iter < 1) return FSC_ERR_INVALID_ARG;
    if (d->flags & ~(FSC_BATCH_AUTOTUNE | FSC_VALIDATE_SYMMETRY)) return FSC_ERR_INVALID_ARG;
    const int G = d->num_graphs;
    const long long* voff = reinterpret_cast<const long long*>(d->vertex_offset);
    if (voff[0] != 0) return FSC_ERR_INVALID_ARG;
    for (int g = 0; g < G; ++g) {
        const long long n = voff[g + 1] - voff[g];
        const int k = d->k[g];
        const int l = d->l ? d->l[g] : 0;
        if (n < 1 || k < 1 || k > n || k > 256 || l < 0 || l > 8 || (d->t && d->t[g] < 0)) return FSC_ERR_INVALID_ARG;
    }
    const long long nv = voff[G];
    if (nv > 2147483647LL) return FSC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    fsc_batch* b = new (std::nothrow) fsc_batch();
    if (!b) return FSC_ERR_OOM;
    b->num_graphs = G;
    b->labels = d->labels;
    b->store = d->store;
    cudaGetDevice(&b->device);
    fsc_status rc = FSC_OK;
    cudaError_t e = cudaSuccess;
    long long* d_voff = nullptr;
    do {
        // nnz of the union and of each graph (row_ptr values at the graph boundaries)
        if ((e = cudaMalloc(&d_voff, sizeof(long long) * (G + 1))) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(d_voff, voff, sizeof(long long) * (G + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
        long long* d_bound = nullptr;
        if ((e = cudaMalloc(&d_bound, sizeof(long long) * (G + 1))) != cudaSuccess) break;
        k_gather_boundaries<<<(G + 256) / 256, 256, 0, s>>>(d->row_ptr, d_voff, G, d_bound);
        std::vector<long long> bound(G + 1);
        e = cudaMemcpyAsync(bound.data(), d_bound, sizeof(long long) * (G + 1), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(d_bound);
        if (e != cudaSuccess) break;
        const long long nnz = bound[G];
        // the union graph: validation and degrees of every vertex
        rc = fsc_create_graph(nv, nnz, d->row_ptr, d->col_idx, d->w, d->flags & FSC_VALIDATE_SYMMETRY, stream, &b->uni);
        if (rc != FSC_OK) break;
        int* d_status = nullptr;
        if ((e = cudaMalloc(&d_status, sizeof(int))) != cudaSuccess) break;
        cudaMemsetAsync(d_status, 0, sizeof(int), s);
        k_batch_check<<<device_props().num_sms * 8, 256, 0, s>>>(nv, d->row_ptr, d->col_idx, d_voff, G, d_status);
        int hst = 0;
        e = cudaMemcpyAsync(&hst, d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(d_status);
        if (e != cudaSuccess) break;
        if (hst) { rc = status_from_bits(hst); break; }

        // per-graph parameters, arenas and the largest-first work order
        const size_t es = d->store == FSC_F32 ? 4 : 2;
        std::vector<BatchGraph> gs(G);
        b->seed_off.assign(G, 0);
        b->cent_off.assign(G, 0);
        b->k_of.assign(G, 0);
        b->l_of.assign(G, 0);
        long long zoff = 0, eoff = 0, doff = 0, toff = 0, soff = 0, coff = 0;
        size_t smem = 0;
        std::vector<long long> gnnz(G);
        for (int g = 0; g < G; ++g) {
            BatchGraph& x = gs[g];
            const long long n = voff[g + 1] - voff[g];
            int l = d->l ? d->l[g] : 0, t = d->t ? d->t[g] : -1;
            int ld = 0, td = 0;
            fsc_default_params(n, d->k[g], 0, &ld, &td);
            if (l == 0) l = ld;
            if (t < 0) t = td;
            x.v0 = voff[g];
            x.n = (int)n;
            x.k = d->k[g];
            x.l = l;
            x.LP = pad_l(l);
            x.t = t;
            x.seed = d->seed[g];
            x.gid = g;
            gnnz[g] = bound[g + 1] - bound[g];
            const double avg = (double)gnnz[g] / (double)n;
            int tpr = tuned_threads_per_row(avg, x.LP, d->store, d->w != nullptr);
            if (!tpr) {
                fsc_graph tmp{};
                tmp.n = n;
                tmp.nnz = gnnz[g];
                tpr = choose_threads_per_row(&tmp, 0, x.LP, d->store);
            }
            x.tpr = tpr;
            const size_t tab = (size_t)x.k * (x.LP + 1) * 8;
            int ntab = (int)(32768 / tab);
            x.ntab = ntab < 1 ? 1 : (ntab > KM_WARPS ? KM_WARPS : ntab);
            const size_t need = (((size_t)x.k * x.LP * 4 + 15) & ~(size_t)15) + (size_t)x.k * x.LP * 8 +
                                (((size_t)x.k * 4 + 15) & ~(size_t)15) + (size_t)x.ntab * tab;
            smem = std::max(smem, need);
            // every per-graph base is rounded to 64 elements (>= 128 bytes), so the row vectors of
            // any LP stay aligned whatever the previous graphs' sizes were
            auto round64 = [](long long v) { return (v + 63) / 64 * 64; };
            x.zoff = zoff;
            zoff += round64(2 * n * x.LP);     // two iterate buffers; the second starts at n*LP
            x.eoff = eoff;
            eoff += round64(n * x.LP);
            x.doff = doff;
            doff += n;
            x.toff = toff;
            toff += (n + KM_TILE - 1) / KM_TILE;
            x.soff = soff;
            soff += x.k;
            x.coff = coff;
            coff += (long long)x.k * x.LP;
            b->seed_off[g] = x.soff;
            b->cent_off[g] = x.coff;
            b->k_of[g] = x.k;
            b->l_of[g] = x.l;
        }
        // autotune (optional): time the lane counts on the largest graph of each (degree bucket, LP)
        if (d->flags & FSC_BATCH_AUTOTUNE) {
            std::vector<int> order(G);
            for (int g = 0; g < G; ++g) order[g] = g;
            std::sort(order.begin(), order.end(), [&](int x, int y) { return gnnz[x] > gnnz[y]; });
            for (int g : order) {
                const double avg = (double)gnnz[g] / (double)gs[g].n;
                if (tuned_threads_per_row(avg, gs[g].LP, d->store, d->w != nullptr)) continue;
                fsc_graph view{};
                view.device = b->device;
                view.n = gs[g].n;
                view.nnz = gnnz[g];
                view.row_ptr = d->row_ptr + gs[g].v0;
                view.col = d->col_idx;
                view.w = d->w;
                view.deg = b->uni->deg + gs[g].v0;
                view.dinv = b->uni->dinv + gs[g].v0;
                view.invdeg = b->uni->invdeg + gs[g].v0;
                view.col_off = gs[g].v0;
                int best = 0;
                float us = 0.f;
                rc = autotune_graph(&view, gs[g].l, (fsc_dtype)d->store, &best, &us, s);
                if (view.ws) pool_free(view.ws, s);
                if (rc != FSC_OK) break;
            }
            if (rc != FSC_OK) break;
            for (int g = 0; g < G; ++g) {
                const int tpr = tuned_threads_per_row((double)gnnz[g] / (double)gs[g].n, gs[g].LP, d->store,
                                                      d->w != nullptr);
                if (tpr) gs[g].tpr = tpr;
            }
        }
        std::vector<int> order(G);
        for (int g = 0; g < G; ++g) order[g] = g;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            return gnnz[x] * (long long)gs[x].t > gnnz[y] * (long long)gs[y].t;
        });
        b->h_graphs.resize(G);
        for (int q = 0; q < G; ++q) b->h_graphs[q] = gs[order[q]];
        b->smem = smem;
        if ((e = cudaMalloc(&b->d_graphs, sizeof(BatchGraph) * G)) != cudaSuccess) break;
        if ((e = cudaMemcpy(b->d_graphs, b->h_graphs.data(), sizeof(BatchGraph) * G, cudaMemcpyHostToDevice)) != cudaSuccess) break;
        if ((e = cudaMalloc(&b->d_queue, 256)) != cudaSuccess) break;
        if ((e = cudaMalloc(&b->zarena, (size_t)zoff * es + 256)) != cudaSuccess) break;
        if ((e = cudaMalloc(&b->earena, (size_t)eoff * 4 + 256)) != cudaSuccess) break;
        if ((e = cudaMalloc(&b->darena, (size_t)doff * 4 + 256)) != cudaSuccess) break;
        if ((e = cudaMalloc(&b->tarena, (size_t)toff * 8 + 256)) != cudaSuccess) break;
        if ((e = cudaMalloc(&b->seeds, (size_t)soff * 8 + 256)) != cudaSuccess) break;
        if ((e = cudaMalloc(&b->cents, (size_t)coff * 8 + 256)) != cudaSuccess) break;
        b->seeds_total = soff;
        b->cents_total = coff;
        if ((e = cudaMalloc(&b->stats, sizeof(KmDevStats) * G)) != cudaSuccess) break;

        // capture queue reset + stats reset + the persistent launch into a CUDA graph
        BatchArgs a{};
        a.graphs = b->d_graphs;
        a.num_graphs = G;
        a.queue = b->d_queue;
        a.row_ptr = d->row_ptr;
        a.col = d->col_idx;
        a.w = d->w;
        a.dinv = b->uni->dinv;
        a.invdeg = b->uni->invdeg;
        a.zarena = b->zarena;
        a.earena = b->earena;
        a.darena = b->darena;
        a.tarena = b->tarena;
        a.seeds = b->seeds;
        a.cents = b->cents;
        a.labels = d->labels;
        a.stats = b->stats;
        a.max_iter = d->max_iter;
        const void* kern;
        if (d->store == FSC_F32) kern = d->w ? (const void*)k_batch<float, true> : (const void*)k_batch<float, false>;
        else kern = d->w ? (const void*)k_batch<__nv_bfloat16, true> : (const void*)k_batch<__nv_bfloat16, false>;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) break;
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, KM_THREADS, smem)) != cudaSuccess) break;
        if (per_sm < 1) { rc = FSC_ERR_INVALID_ARG; break; }
        long long grid = (long long)per_sm * device_props().num_sms;
        if (grid > G) grid = G;
        cudaStream_t cs = nullptr;
        if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) break;
        void* args[] = {&a};
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemsetAsync(b->d_queue, 0, sizeof(int), cs);
            cudaMemsetAsync(b->stats, 0, sizeof(KmDevStats) * G, cs);
            cudaLaunchKernel(kern, dim3((unsigned)grid), dim3(KM_THREADS), args, smem, cs);
            e = cudaStreamEndCapture(cs, &b->graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) break;
    } while (0);
    cudaFree(d_voff);
    if (e != cudaSuccess && rc == FSC_OK) rc = cuda_status(e);
    if (rc != FSC_OK) {
        batch_free(b);
        return rc;
    }
    *out = b;
    return FSC_OK;
}

extern "C" fsc_status fsc_batch_run(fsc_batch* b, void* stream) {
    if (!b || !b->exec) return FSC_ERR_INVALID_ARG;
    FSC_CUDA(cudaGraphLaunch(b->exec, as_stream(stream)));
    return FSC_OK;
}

extern "C" fsc_status fsc_batch_results(fsc_batch* b, fsc_kmeans_stats* stats, int64_t* seed_idx, double* centroids,
                                        void* stream) {
    if (!b) return FSC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    FSC_CUDA(cudaStreamSynchronize(s));
    const int G = b->num_graphs;
    if (stats) {
        std::vector<KmDevStats> h(G);
        FSC_CUDA(cudaMemcpy(h.data(), b->stats, sizeof(KmDevStats) * G, cudaMemcpyDeviceToHost));
        for (int g = 0; g < G; ++g) {
            stats[g].iterations = h[g].iterations;
            stats[g].changed = h[g].changed;
            stats[g].empty_events = h[g].empty_events;
            stats[g].device_status = 0;
            stats[g].inertia = h[g].inertia;
            stats[g].seeding_potential = h[g].potential;
        }
    }
    if (seed_idx || centroids) {
        std::vector<int64_t> hs(b->seeds_total + 1);
        std::vector<double> hc(b->cents_total + 1);
        if (seed_idx) FSC_CUDA(cudaMemcpy(hs.data(), b->seeds, sizeof(int64_t) * b->seeds_total, cudaMemcpyDeviceToHost));
        if (centroids) FSC_CUDA(cudaMemcpy(hc.data(), b->cents, sizeof(double) * b->cents_total, cudaMemcpyDeviceToHost));
        long long so = 0, co = 0;
        for (int g = 0; g < G; ++g) {
            const int k = b->k_of[g], l = b->l_of[g], LP = pad_l(l);
            if (seed_idx)
                for (int j = 0; j < k; ++j) seed_idx[so + j] = hs[b->seed_off[g] + j];
            if (centroids)
                for (int j = 0; j < k; ++j)
                    for (int c = 0; c < l; ++c) centroids[co + (long long)j * l + c] = hc[b->cent_off[g] + (long long)j * LP + c];
            so += k;
            co += (long long)k * l;
        }
    }
    return FSC_OK;
}

extern "C" fsc_status fsc_batch_embedding(fsc_batch* b, int graph, float* out, void* stream) {
    if (!b || !out || graph < 0 || graph >= b->num_graphs) return FSC_ERR_INVALID_ARG;
    for (const BatchGraph& x : b->h_graphs) {
        if (x.gid != graph) continue;
        FSC_CUDA(cudaMemcpyAsync(out, b->earena + x.eoff, sizeof(float) * (size_t)x.n * x.LP, cudaMemcpyDeviceToDevice,
                                 as_stream(stream)));
        return FSC_OK;
    }
    return FSC_ERR_INVALID_ARG;
}

extern "C" fsc_status fsc_batch_destroy(fsc_batch* b) {
    if (!b) return FSC_OK;
    cudaDeviceSynchronize();
    batch_free(b);
    return FSC_OK;
}
