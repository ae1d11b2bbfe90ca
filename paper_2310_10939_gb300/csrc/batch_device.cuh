// Device side of the batched mode: per-graph pieces of Algorithm 2 run by one CTA, and the two
// persistent kernels (embedding, k-means), one instantiation per row width l_pad (graphs are
// grouped by it, so each kernel's registers follow its own width instead of the widest one).
#pragma once

#include <math.h>
#include <string.h>
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

// row_gather (spmm.cuh) for R rows at once, their loads interleaved: one block per SM has a third
// of the warps the single-graph kernel keeps in flight, so each lane group carries R rows to keep
// as many gathers outstanding.  Each row's sum is formed exactly as row_gather forms it (the same
// passes, entries and order; a row adds nothing in the passes after its own last one).
template <int LP, typename TI, int G, int U, bool W, int R>
__device__ __forceinline__ void rows_gather(const bool (&active)[R], const long long (&row)[R], int sub,
                                            const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                            const float* __restrict__ w, const TI* zin, long long col_off,
                                            long long nz, float (&acc)[R][LP]) {
    int64_t p[R], e[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int c = 0; c < LP; ++c) acc[r][c] = 0.f;
        p[r] = active[r] ? rp[row[r]] + sub : 0;
        e[r] = active[r] ? rp[row[r] + 1] : 0;
    }
    for (;;) {
        bool live[R], any = false;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            live[r] = p[r] < e[r];
            any |= live[r];
        }
        if (!any) break;
        long long j[R][U];
        float wv[R][U];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t q = p[r] + (int64_t)u * G;
                const bool ok = live[r] && q < e[r];
                j[r][u] = ok ? (long long)__ldg(col + q) - col_off : -1;
                if (ok && !in_range(j[r][u], 0, nz, BS_GATHER)) j[r][u] = -1;
                if (W) wv[r][u] = ok ? __ldg(w + q) : 0.f;
            }
        float v[R][U][LP];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (j[r][u] >= 0) {
                    load_z<LP, TI, false>(zin + (size_t)j[r][u] * LP, v[r][u]);
                } else {
#pragma unroll
                    for (int c = 0; c < LP; ++c) v[r][u][c] = 0.f;
                }
            }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (live[r]) {
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int c = 0; c < LP; ++c)
                        acc[r][c] = W ? fmaf(wv[r][u], v[r][u][c], acc[r][c]) : acc[r][c] + v[r][u][c];
            }
            p[r] += (int64_t)G * U;
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1)
#pragma unroll
            for (int c = 0; c < LP; ++c) acc[r][c] += __shfl_xor_sync(0xffffffffu, acc[r][c], off);
}

template <int LP, typename TS, int G, bool W>
__device__ void power_block(const BatchGraph& g, const BatchArgs& a, TS* zA, TS* zB, float* emb, float* s_cm,
                            int* s_E) {
    constexpr int U = G <= 8 ? 4 : 2;
    constexpr int RPW = 32 / G;
    // rows in flight per lane group (the 64-register budget of two CTAs per SM holds two rows of
    // up to 4 columns)
    constexpr int R = LP <= 4 ? 2 : 1;
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
        for (long long base = (long long)wid * RPW * R; base < g.n; base += (long long)KM_WARPS * RPW * R) {
            long long row[R];
            bool act[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                row[r] = base + (long long)r * RPW + grp;
                act[r] = row[r] < g.n;
            }
            float acc[R][LP];
            rows_gather<LP, TS, G, U, W, R>(act, row, sub, rp, a.col, a.w, zin, g.v0, g.n, acc);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (act[r] && sub == 0) {   // the same epilogue as power_row
                    float self[LP], y[LP];
                    load_z<LP, TS, false>(zin + (size_t)row[r] * LP, self);
                    const float id = invdeg[row[r]];
#pragma unroll
                    for (int c = 0; c < LP; ++c) y[c] = scale[c] * (0.5f * fmaf(id, acc[r][c], self[c]));
                    if (last) store_row<LP, float>(emb + (size_t)row[r] * LP, y);
                    else store_row<LP, TS>(zout + (size_t)row[r] * LP, y);
#pragma unroll
                    for (int c = 0; c < LP; ++c) cmx[c] = fmaxf(cmx[c], fabsf(y[c]));
                }
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

// Lloyd in one CTA with the same exact arithmetic as k_lloyd: the cluster sums are running
// totals (s_S) that only points changing cluster update, and the inertia is taken in the first
// iteration and, for the last assignment, by one pass after the loop with the centroids that
// assignment used.
template <int LP>
__device__ void lloyd_block(const float* X, int n, int l, int k, int max_iter, const Scales& sc, int32_t* labels,
                            float* s_c, double* s_c64, unsigned long long* s_tab, int ntab, long long* s_S,
                            KmDevStats* st) {
    __shared__ long long s_red[KM_WARPS];
    __shared__ int s_redi[KM_WARPS];
    const int tid = threadIdx.x, wid = tid >> 5;
    const size_t rowlen = (size_t)k * (LP + 1);
    unsigned long long* my_tab = s_tab + (size_t)(wid % ntab) * rowlen;
    for (long long i = tid; i < n; i += KM_THREADS) labels[i] = -1;
    for (int q = tid; q < k * LP; q += KM_THREADS) s_c64[q] = (double)s_c[q];
    for (size_t q = tid; q < rowlen; q += KM_THREADS) s_S[q] = 0;
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
                if (it == 1) inert += fixq(best[u], sc.Sd);
                if (old[u] != lab) {   // leaves its old cluster (none in iteration 1), joins the new
                    ++changed;
                    labels[i0 + u] = lab;
                    long long qx[LP];
#pragma unroll
                    for (int c = 0; c < LP; ++c) qx[c] = fixq(x[u][c], sc.Sx);
                    slot_add<LP>(sl, lab, qx, false, my_tab);
                    if (old[u] >= 0) slot_add<LP>(sl, old[u], qx, true, my_tab);
                }
            }
        }
        slot_flush_warp<LP>(sl[0], my_tab);
        slot_flush_warp<LP>(sl[1], my_tab);
        __syncthreads();
        for (size_t q = tid; q < rowlen; q += KM_THREADS) {
            unsigned long long v = s_tab[q];
            for (int t = 1; t < ntab; ++t) v += s_tab[(size_t)t * rowlen + q];
            s_S[q] += (long long)v;   // exact running totals
        }
        inert = block_sum_ll(inert, s_red);
        changed = block_sum_i(changed, s_redi);
        __syncthreads();
        // on the last iteration s_c keeps the centroids its assignment used (for the inertia)
        const bool stop = changed == 0 || it == max_iter;
        for (int q = tid; q < k * LP; q += KM_THREADS) {
            const int j = q / LP, c = q % LP;
            const long long cnt = s_S[(size_t)j * (LP + 1) + LP];
            if (cnt > 0) {
                const double m = ((double)s_S[(size_t)j * (LP + 1) + c] * pow2d(-sc.Sx)) / (double)cnt;
                s_c64[q] = m;
                if (!stop) s_c[q] = (float)m;
            } else if (c == 0) {
                ++empty;
            }
        }
        __syncthreads();
        if (tid == 0) {
            if (it == 1) st->potential = (double)inert * pow2d(-sc.Sd);
            st->iterations = it;
            st->changed = changed;
        }
        if (stop) break;
    }
    long long inert = 0;
    for (int tl = 0; tl < ntiles; ++tl) {
        const long long i0 = (long long)tl * KM_TILE + (long long)KM_PPT * tid;
#pragma unroll
        for (int u = 0; u < KM_PPT; ++u) {
            if (i0 + u < n) {
                float x[LP];
                load_point_cg<LP>(X, i0 + u, l, x);
                const int lab = __ldcg(labels + i0 + u);
                inert += fixq(sqdist<LP>(x, s_c + lab * LP), sc.Sd);
            }
        }
    }
    inert = block_sum_ll(inert, s_red);
    const int e = block_sum_i(empty, s_redi);
    if (tid == 0) {
        st->empty_events = e;
        st->inertia = (double)inert * pow2d(-sc.Sd);
    }
    __syncthreads();
}

// Steps 1-2 of Algorithm 2 for one graph: the start block and the t power steps; the last one
// writes the float32 embedding.
template <int LP, typename TS, bool W>
__device__ void embed_graph(const BatchArgs& a, const BatchGraph& g) {
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
}

// Step 3 for one graph: k-means++ and Lloyd on the embedding rows.
template <int LP>
__device__ void kmeans_graph(const BatchArgs& a, const BatchGraph& g, unsigned char* smem) {
    const int tid = threadIdx.x;
    const float* emb = a.earena + g.eoff;
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
    long long* s_S = reinterpret_cast<long long*>(s_tab + (size_t)g.ntab * g.k * (LP + 1));
    lloyd_block<LP>(emb, g.n, g.l, g.k, a.max_iter, sc, a.labels + g.v0, s_c, s_c64, s_tab, g.ntab, s_S, st);
    for (int q = tid; q < g.k * LP; q += KM_THREADS) a.cents[g.coff + q] = s_c64[q];
    __syncthreads();
}

// The two persistent kernels of a row-width group, run one after the other: each CTA pops a
// graph from the group's queue counter and runs that graph's part with block barriers only, so
// no CTA ever waits on another.  The power steps are latency-bound gathers, so their kernel
// runs two CTAs per SM (64 registers); k-means needs ~120 registers and runs one.
template <int LP, typename TS, bool W>
__global__ void __launch_bounds__(KM_THREADS, 2) k_batch_embed(BatchArgs a) {
    __shared__ int s_q;
    for (;;) {
        if (threadIdx.x == 0) s_q = atomicAdd(a.queue, 1);
        __syncthreads();
        const int q = s_q;
        __syncthreads();
        if (q >= a.num_graphs) break;
        embed_graph<LP, TS, W>(a, a.graphs[q]);
    }
}

template <int LP>
__global__ void __launch_bounds__(KM_THREADS, 1) k_batch_kmeans(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char bsmem[];
    __shared__ int s_q;
    for (;;) {
        if (threadIdx.x == 0) s_q = atomicAdd(a.queue, 1);
        __syncthreads();
        const int q = s_q;
        __syncthreads();
        if (q >= a.num_graphs) break;
        kmeans_graph<LP>(a, a.graphs[q], bsmem);
    }
}

// Kernel entry points: the embedding kernels of one storage type (batch_k_f32.cu,
// batch_k_bf16.cu) and the k-means kernels (batch_k_f32.cu).
const void* batch_kernel_f32(int LP, bool weighted);
const void* batch_kernel_bf16(int LP, bool weighted);
const void* batch_kmeans_kernel(int LP);

}  // namespace fsc
