// k-means++ seeding and Lloyd iterations on the embedding rows (Sec. 2.2, last step of Algorithm 2).
//
// Both phases run as one cooperative (co-resident) persistent launch each.  Chunks of KM_CHUNK
// points (one warp's work) are dealt round-robin over the blocks; cross-block steps are separated
// by a bounded grid barrier (grid_sync), after which every block reads the other blocks' partial
// results through L2.  Lloyd keeps the exact cluster sums as running totals that only points changing
// cluster update, and skips points by Hamerly's bounds (see k_lloyd).
//
// Decisions follow fixed rules that a float64 CPU restatement reproduces:
//  * squared distances: float32, columns in order, no fused multiply-add;
//  * k-means++: first centre floor(u0 * n); round r picks the smallest index whose prefix sum
//    of D^2 exceeds u_r * sum(D^2); sum(D^2) = 0 picks the lowest index not chosen yet;
//  * Lloyd: strict '<' over centroids in index order (ties -> lowest index); centroids are
//    means; an empty cluster keeps its centroid; stop when no label changes or after max_iter.
//
// High-precision sums without float64 arithmetic in the loops: float64 runs at a small
// fraction of the float32 rate on this GPU, so centroid sums, D^2 prefix sums and the
// inertia are accumulated EXACTLY as 64-bit fixed-point integers (order independent,
// deterministic).  With A = max |x| over the used columns, 2^Ex > A and 2^N >= n:
//    coordinates:  q(x) = trunc(x * 2^Sx),  Sx = 62 - Ex - N
//    distances:    q(d) = trunc(d * 2^Sd),  Sd = 62 - Ed - N,  Ed = 2 Ex + ceil(log2 l) + 3
// so no sum of n terms can exceed 2^62.  Each term loses less than one unit 2^-S, i.e. the
// sums carry an absolute error below n 2^-S (about 1e-13 A for the centroid means at
// n = 2^20), smaller than the rounding of a sequential float64 sum.  Means and inertia are
// formed in float64 from the exact integer sums.  The k-means++ target is compared exactly:
// with U = w >> 11 (53 bits), index i qualifies iff P_i > floor(U * P_total / 2^53), which is
// the same as P_i > u * P_total for u = U / 2^53.
#include <limits.h>
#include <math.h>

#include <mutex>

#include "kmeans_common.cuh"

namespace fsc {

struct KppArgs {
    const float* X;
    int n, l, k;
    unsigned long long seed;
    float* d2[2];        // D^2 per point, two buffers; cfl names the one holding a chunk's current values
    long long* ttot[3];  // per tile: exact D^2 total (its chunks' totals, atomics), three in rotation
    unsigned* tmask[3];  // per tile: bit w = the d2 buffer of its chunk w (atomics), three in rotation
    long long* ctot[2];  // per chunk: exact D^2 total after round r: ctot[r & 1]
    unsigned* cdmax[2];  // per chunk: largest D^2 (float bits) after round r: cdmax[r & 1]
    int* cfl[2];         // per chunk: the d2 buffer holding its D^2 after round r is cfl[r & 1][chunk]
    float* ccen;         // per chunk: centre of its points (LP floats)
    float* crad;         // per chunk: largest distance of its points from that centre, widened
    float* clb;          // per chunk: lower bound on its points' distances to the centres it was carried past
    float* lb2;          // per point: lower bound on its distance to every chosen centre but its nearest
    unsigned* amax;      // max |x| (float bits), output for the Lloyd launch
    int* near;           // per point: index (selection order) of its nearest chosen centre
    int64_t* seeds;
    float* c32;
    GridBarrier* bar;
    int* status;
    long long limit;
    int stall;
    // optional: the learned filter's energy guard (see fsc_cluster_filtered).  When *guard / guard_lk
    // is not <= guard_thr the filtered embedding will be replaced by the plain one, and the launch
    // returns at once (the same double division and comparison as the host's decision).
    const double* guard;
    double guard_lk, guard_thr;
};

// The guard test of KppArgs / LloydArgs: true when the clustering is not wanted.
__device__ __forceinline__ bool guard_rejects(const double* guard, double lk, double thr) {
    return guard && !(__ldcg(guard) / lk <= thr);
}

// A point whose D^2 = |x - c_a|^2 (c_a its nearest chosen centre) satisfies
// sqrt(D^2) < |c - c_a| / 2 cannot move closer to a new centre c (triangle inequality:
// |x - c| >= |c - c_a| - |x - c_a| > sqrt(D^2)), so its D^2 is carried over without loading
// the point.  Both sides of the test are widened by KPP_EPS relative, far above float32
// rounding of the distances, so a skipped point is one whose min(D^2, d) is D^2 exactly.
// The same argument for a whole chunk of KM_CHUNK points with centre m and radius rho (every point
// within rho of m) whose largest D^2 is Dmax: if |c - m| - rho > sqrt(Dmax), then for every point x
// of the chunk |x - c| >= |c - m| - |x - m| > sqrt(Dmax) >= sqrt(D^2(x)), so no D^2 of the chunk
// changes and the chunk is carried over (its D^2, nearest centres and exact total) without reading
// any of its per-point state.  rho is widened when it is stored, |c - m| shrunk and sqrt(Dmax)
// grown by KPP_EPS relative, so a carried chunk is one the per-point rule would leave unchanged.
// The draw sums the chunks' totals per tile of KM_TILE points (tile totals, atomics).
constexpr float KPP_EPS = 1e-5f;
constexpr int KPP_CACHE = 4;   // tile totals per thread kept in registers by the selection

template <int LP>
__global__ void __launch_bounds__(KM_THREADS) k_kmeanspp(KppArgs a) {
    unsigned epoch = 0;   // grid barriers passed
    // k chosen indices, k floats (|c_new - c_j| / 2)^2 shrunk, the chosen centres (k x LP floats)
    extern __shared__ int s_chosen[];
    __shared__ long long s_red[KM_WARPS];
    __shared__ long long s_T, s_base, s_tile;
    __shared__ unsigned s_amax;
    __shared__ int s_bstar, s_idx;
    __shared__ unsigned s_src;   // the drawn tile's buffer mask
    __shared__ int s_live[KM_THREADS], s_nlive;   // phase A: a group's live chunks
    const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const long long n = a.n;
    const long long ntiles = (n + KM_TILE - 1) / KM_TILE;
    const long long nch = (n + KM_CHUNK - 1) / KM_CHUNK;   // chunks of KM_CHUNK points (see phase A)
    if (guard_rejects(a.guard, a.guard_lk, a.guard_thr)) return;   // every block alike: before any barrier

    // ---- phase 0: A = max |x| over the used columns (sets the fixed-point scales), and for each
    // chunk (one warp each, dealt as in phase A) the mean of its points and their largest distance
    // from it
    if (tid == 0) s_amax = 0u;
    __syncthreads();
    {
        float m = 0.f;
        for (long long ch = b + (long long)G * wid; ch < nch; ch += (long long)G * KM_WARPS) {
            const long long i0 = ch * KM_CHUNK + (long long)KM_PPT * lane;
            float x[KM_PPT][LP];
            float sum[LP];
#pragma unroll
            for (int c = 0; c < LP; ++c) sum[c] = 0.f;
#pragma unroll
            for (int u = 0; u < KM_PPT; ++u) {
                if (i0 + u < n) {
                    load_point<LP>(a.X, i0 + u, a.l, x[u]);
#pragma unroll
                    for (int c = 0; c < LP; ++c) {
                        m = fmaxf(m, fabsf(x[u][c]));
                        sum[c] += x[u][c];
                    }
                }
            }
            const float cnt = (float)min((long long)KM_CHUNK, n - ch * KM_CHUNK);
            float mc[LP];
#pragma unroll
            for (int c = 0; c < LP; ++c) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) sum[c] += __shfl_xor_sync(0xffffffffu, sum[c], off);
                mc[c] = sum[c] / cnt;
            }
            float r2 = 0.f;
#pragma unroll
            for (int u = 0; u < KM_PPT; ++u)
                if (i0 + u < n) r2 = fmaxf(r2, sqdist<LP>(x[u], mc));
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) r2 = fmaxf(r2, __shfl_xor_sync(0xffffffffu, r2, off));
            float mine = 0.f;   // lane c writes column c (selects: no dynamically indexed array)
#pragma unroll
            for (int c = 0; c < LP; ++c)
                if (lane == c) mine = mc[c];
            if (lane < LP) a.ccen[ch * LP + lane] = mine;
            if (lane == 0) {
                a.crad[ch] = sqrtf(r2) * (1.0f + KPP_EPS);
                a.clb[ch] = __int_as_float(0x7f800000);   // +inf
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        if (lane == 0 && m > 0.f) atomicMax(&s_amax, __float_as_uint(m));
        __syncthreads();
        if (tid == 0 && s_amax) atomicMax(a.amax, s_amax);
    }
    if (!grid_sync(a.bar, a.status, a.limit, a.stall, epoch)) return;
    const float A = __uint_as_float(__ldcg(a.amax));
    const Scales sc = scales_for(A, n, a.l);

    float* s_half2 = reinterpret_cast<float*>(s_chosen + a.k);
    float* s_cent = s_half2 + a.k;   // centre j at s_cent[j * LP], unused columns 0
    if (tid == 0) {
        const U64x4 r = philox4x64_10(U64x4{0ull, 0ull, 0ull, 0ull}, a.seed, STREAM_KMEANSPP);
        long long i0 = (long long)floor(uniform53(r.x) * (double)n);
        if (i0 > n - 1) i0 = n - 1;
        s_chosen[0] = (int)i0;
        if (b == 0) a.seeds[0] = i0;
    }
    __syncthreads();
    if (tid < LP) s_cent[tid] = tid < a.l ? a.X[(size_t)s_chosen[0] * LP + tid] : 0.f;
    __syncthreads();

    for (int r = 1; r <= a.k; ++r) {
        const float* s_c = s_cent + (size_t)(r - 1) * LP;   // the centre chosen last round
        // squared half-distances from the new centre to the earlier ones, shrunk by the margin
        for (int j = tid; j < r - 1; j += KM_THREADS) {
            float cj[LP];
#pragma unroll
            for (int c = 0; c < LP; ++c) cj[c] = s_cent[(size_t)j * LP + c];
            const float h = 0.5f * sqrtf(sqdist<LP>(cj, s_c)) * (1.0f - KPP_EPS);
            s_half2[j] = h * h;
        }
        __syncthreads();
        long long* tt = a.ttot[r % 3];              // exact D^2 total per tile (atomics)
        long long* tz = a.ttot[(r + 1) % 3];        // cleared here for round r + 1
        unsigned* tmk = a.tmask[r % 3];             // per tile: its chunks' buffer bits (atomics)
        unsigned* tmz = a.tmask[(r + 1) % 3];       // cleared here for round r + 1
        long long* ct = a.ctot[r & 1];              // per chunk, this round (one writer per chunk)
        const long long* cp = a.ctot[(r + 1) & 1];  // per chunk, after round r - 1
        unsigned* dm = a.cdmax[r & 1];
        const unsigned* dp = a.cdmax[(r + 1) & 1];
        int* fl = a.cfl[r & 1];
        const int* fp = a.cfl[(r + 1) & 1];
        // ---- phase A: D^2 update.  The points are dealt in chunks of KM_CHUNK (one warp, four
        // consecutive points per lane): chunk c goes to block c mod G.  The points that cannot
        // skip the new centre are its neighbourhood, a contiguous run of vertices in a clustered
        // graph, and dealing chunks spreads them over every block instead of loading a few while
        // the others wait at the barrier.  A block tests up to KM_THREADS of its chunks at once
        // (one thread per chunk, which also carries a far chunk's state and adds its total to its
        // tile's), lists the live chunks in shared memory and deals them over its warps, each of
        // which works its share in order, the next chunk's D^2, nearest-centre indices and lower
        // bounds (and for l_pad <= 4 its points) loading while one computes.  A chunk's D^2 is read
        // from the buffer holding it and written to the other one (the selection of the previous
        // round may still read the first).
        constexpr bool kPre = LP <= 4;
        for (long long m0 = 0; b + (long long)G * m0 < nch; m0 += KM_THREADS) {
            const long long ch_t = b + (long long)G * (m0 + tid);   // this thread's chunk of the group
            bool live = false;
            int src_t = 0;                                           // the buffer holding its D^2
            if (ch_t < nch && r == 1) {
                live = true;   // the first centre: every point's D^2 is set
            } else if (ch_t < nch) {
                const long long t = ch_t / KM_CHUNKS_PER_TILE;
                // every load of the test and of a carry issued together (one memory latency)
                float mc[LP];
#pragma unroll
                for (int c = 0; c < LP; ++c) mc[c] = __ldcg(a.ccen + ch_t * LP + c);
                const unsigned dmb = __ldcg(dp + ch_t);
                const float rad = __ldcg(a.crad + ch_t);
                const int fpv = __ldcg(fp + ch_t);
                const long long ctp = __ldcg(cp + ch_t);
                const float clbv = a.clb[ch_t];
                const float dc = sqrtf(sqdist<LP>(mc, s_c));
                // a chunk the new centre cannot reach (the rule above KPP_EPS) keeps its state; dcr
                // is |c - m|, shrunk, minus the chunk's radius: a lower bound on the distance from
                // any point of the chunk to the new centre
                const float dcr = dc * (1.0f - KPP_EPS) - rad;
                if (!(dcr > sqrtf(__uint_as_float(dmb)) * (1.0f + KPP_EPS))) {
                    live = true;
                    src_t = fpv & 1;
                } else {
                    // every point of the chunk is at least dcr from the new centre
                    a.clb[ch_t] = fminf(clbv, fmaxf(0.f, dcr) * (1.0f - KPP_EPS));
                    ct[ch_t] = ctp;
                    dm[ch_t] = dmb;
                    fl[ch_t] = fpv;
                    if (ctp) atomicAdd(reinterpret_cast<unsigned long long*>(tt + t), (unsigned long long)ctp);
                    if (fpv & 1) atomicOr(tmk + t, 1u << (ch_t % KM_CHUNKS_PER_TILE));
                    if (ch_t % KM_CHUNKS_PER_TILE == 0) {
                        tz[t] = 0;
                        tmz[t] = 0u;
                    }
                }
            }
            const int incl = (int)block_scan_ll(live ? 1 : 0, s_red);
            if (live) s_live[incl - 1] = tid | (src_t << 30);
            if (tid == KM_THREADS - 1) s_nlive = incl;
            __syncthreads();
            const int nlive = s_nlive;
            auto live_chunk = [&](int e, int& src) -> long long {   // the e-th live chunk of the group
                const int v = s_live[e];
                src = v >> 30;
                return b + (long long)G * (m0 + (v & 0x3fffffff));
            };
            // loads of one live chunk's per-point state (D^2, nearest centre, lower bound)
            auto load_state = [&](long long ch, int src, float (&old)[KM_PPT], int (&na)[KM_PPT], float (&lb)[KM_PPT],
                                  float (&x)[KM_PPT][LP]) {
                const long long i0 = ch * KM_CHUNK + (long long)KM_PPT * lane;
                if (r > 1 && i0 + KM_PPT <= n) {
                    const float4 dv = *reinterpret_cast<const float4*>(a.d2[src] + i0);
                    const int4 nv = *reinterpret_cast<const int4*>(a.near + i0);
                    const float4 lv = *reinterpret_cast<const float4*>(a.lb2 + i0);
                    old[0] = dv.x; old[1] = dv.y; old[2] = dv.z; old[3] = dv.w;
                    na[0] = nv.x; na[1] = nv.y; na[2] = nv.z; na[3] = nv.w;
                    lb[0] = lv.x; lb[1] = lv.y; lb[2] = lv.z; lb[3] = lv.w;
                } else {
#pragma unroll
                    for (int u = 0; u < KM_PPT; ++u) {
                        const bool in = r > 1 && i0 + u < n;
                        old[u] = in ? a.d2[src][i0 + u] : 0.f;
                        na[u] = in ? a.near[i0 + u] : 0;
                        lb[u] = in ? a.lb2[i0 + u] : 0.f;
                    }
                }
                if constexpr (kPre) {
#pragma unroll
                    for (int u = 0; u < KM_PPT; ++u)
                        if (i0 + u < n) load_point<LP>(a.X, i0 + u, a.l, x[u]);
                }
            };
            float old_n[KM_PPT], lb_n[KM_PPT];
            int na_n[KM_PPT];
            float x_n[KM_PPT][LP];
            int src_n = 0;
            long long ch_n = wid < nlive ? live_chunk(wid, src_n) : nch;
            if (wid < nlive) load_state(ch_n, src_n, old_n, na_n, lb_n, x_n);
            for (int e = wid; e < nlive; e += KM_WARPS) {
                const long long ch = ch_n;
                const int src = src_n;
                const bool more = e + KM_WARPS < nlive;
                if (more) ch_n = live_chunk(e + KM_WARPS, src_n);
                float old[KM_PPT], lb[KM_PPT];
                int na[KM_PPT];
                float x[KM_PPT][LP];
#pragma unroll
                for (int u = 0; u < KM_PPT; ++u) {
                    old[u] = old_n[u];
                    na[u] = na_n[u];
                    lb[u] = lb_n[u];
                    if constexpr (kPre) {
#pragma unroll
                        for (int c = 0; c < LP; ++c) x[u][c] = x_n[u][c];
                    }
                }
                if (more) load_state(ch_n, src_n, old_n, na_n, lb_n, x_n);
                const long long tile = ch / KM_CHUNKS_PER_TILE;
                float* d2n = a.d2[src ^ 1];
                const long long i0 = ch * KM_CHUNK + (long long)KM_PPT * lane;
                bool need[KM_PPT];
#pragma unroll
                for (int u = 0; u < KM_PPT; ++u) {
                    const bool in = i0 + u < n;
                    const bool nok = r == 1 || !in || in_range(na[u], 0, r - 1, BS_KPP_NEAR);
                    need[u] = in && (r == 1 || !nok || old[u] * (1.0f + KPP_EPS) * (1.0f + KPP_EPS) >= s_half2[na[u]]);
                }
                if constexpr (!kPre) {
#pragma unroll
                    for (int u = 0; u < KM_PPT; ++u)
                        if (need[u]) load_point<LP>(a.X, i0 + u, a.l, x[u]);
                }
                long long v = 0;
                float dmx = 0.f;
#pragma unroll
                for (int u = 0; u < KM_PPT; ++u) {
                    if (i0 + u < n) {
                        float dd = old[u];
                        // lower bound on the distance to the centre that is not (or no longer) the nearest
                        float lbc = __int_as_float(0x7f800000);
                        if (need[u]) {
                            const float dn = sqdist<LP>(x[u], s_c);
                            if (r == 1 || dn < old[u]) {
                                dd = dn;
                                a.near[i0 + u] = r - 1;
                                if (r > 1) lbc = sqrtf(old[u]);
                            } else {
                                lbc = sqrtf(dn);
                            }
                        } else {   // |x - c| >= |c - c_a| - |x - c_a| (the skip's own margins kept)
                            lbc = 2.0f * sqrtf(s_half2[na[u]]) - sqrtf(old[u]) * (1.0f + KPP_EPS);
                        }
                        const float lbn = fminf(r == 1 ? __int_as_float(0x7f800000) : lb[u],
                                                fmaxf(0.f, lbc) * (1.0f - KPP_EPS));
                        if (r == 1 || lbn < lb[u]) a.lb2[i0 + u] = lbn;
                        d2n[i0 + u] = dd;
                        v += fixq(dd, sc.Sd);
                        dmx = fmaxf(dmx, dd);
                    }
                }
                v = warp_sum_ll(v);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) dmx = fmaxf(dmx, __shfl_xor_sync(0xffffffffu, dmx, off));
                if (lane == 0) {
                    ct[ch] = v;
                    dm[ch] = __float_as_uint(dmx);
                    fl[ch] = src ^ 1;
                    if (v) atomicAdd(reinterpret_cast<unsigned long long*>(tt + tile), (unsigned long long)v);
                    if ((src ^ 1) & 1) atomicOr(tmk + tile, 1u << (ch % KM_CHUNKS_PER_TILE));
                    if (ch % KM_CHUNKS_PER_TILE == 0) {   // once per tile (its first chunk)
                        tz[tile] = 0;
                        tmz[tile] = 0u;
                    }
                }
            }
            __syncthreads();   // s_live is rewritten by the next group
        }
        // after the last pick one more pass (r = k) folds it into D^2 and the nearest centres, which
        // Lloyd's first assignment then reads; no selection follows it
        if (r == a.k) break;
        if (!grid_sync(a.bar, a.status, a.limit, a.stall, epoch)) return;

        // ---- selection (identical in every block, exact integer arithmetic).  The tile: every
        // thread sums a contiguous range of the tile totals, one block scan gives the total (which
        // sets the target) and each range's offset, and the thread whose range holds the target
        // walks it.  The point: the tile's D^2 in point order, one block scan.
        const long long per = (ntiles + KM_THREADS - 1) / KM_THREADS;
        const long long q_lo = min(ntiles, per * tid), q_hi = min(ntiles, q_lo + per);
        // the first KPP_CACHE totals of the range, and their tiles' buffer masks, stay in registers
        // for the walk below
        long long tcache[KPP_CACHE];
        unsigned fcache[KPP_CACHE];
        long long rsum = 0;
#pragma unroll
        for (int q = 0; q < KPP_CACHE; ++q) {
            const bool in = q_lo + q < q_hi;
            tcache[q] = in ? __ldcg(tt + q_lo + q) : 0;
            fcache[q] = in ? __ldcg(tmk + q_lo + q) : 0u;
            rsum += tcache[q];
        }
        for (long long q = q_lo + KPP_CACHE; q < q_hi; ++q) rsum += __ldcg(tt + q);
        const long long rincl = block_scan_ll(rsum, s_red);
        const long long total = s_red[KM_WARPS - 1];
        if (tid == 0) {
            if (total <= 0) {
                s_bstar = -1;
            } else {
                const U64x4 rr = philox4x64_10(U64x4{(unsigned long long)r, 0ull, 0ull, 0ull}, a.seed,
                                               STREAM_KMEANSPP);
                const unsigned long long U = rr.x >> 11, P = (unsigned long long)total;
                const unsigned long long hi64 = __umul64hi(U, P), lo64 = U * P;
                s_T = (long long)((hi64 << 11) | (lo64 >> 53));   // floor(U * P / 2^53) < P
                s_bstar = 0;
            }
            s_tile = -1;
            s_idx = INT_MAX;
        }
        __syncthreads();
        if (s_bstar == 0) {
            const long long T = s_T;
            const long long rex = rincl - rsum;
            if (rsum > 0 && rex <= T && T < rincl) {   // exactly one thread
                long long base = rex;
                bool found = false;
#pragma unroll
                for (int q = 0; q < KPP_CACHE; ++q) {
                    const long long v = tcache[q];
                    if (!found && v > 0 && base + v > T) {
                        s_tile = q_lo + q;
                        s_base = base;
                        s_src = fcache[q];
                        found = true;
                    }
                    if (!found) base += v;
                }
                for (long long q = q_lo + KPP_CACHE; !found && q < q_hi; ++q) {
                    const long long v = __ldcg(tt + q);
                    if (v > 0 && base + v > T) {
                        s_tile = q;
                        s_base = base;
                        s_src = __ldcg(tmk + q);
                        found = true;
                    }
                    base += v;
                }
            }
            __syncthreads();
            const long long tq = s_tile;
            if (tq >= 0) {   // always (exact sums cross the target); block-uniform
                // warp w's points are the tile's chunk w, whose buffer is bit w of the tile's mask
                static_assert(KM_CHUNKS_PER_TILE == KM_WARPS, "one chunk of the drawn tile per warp");
                const float* d2n = a.d2[(s_src >> wid) & 1];
                const long long i0 = tq * KM_TILE + (long long)KM_PPT * tid;
                long long qv[KM_PPT];
                long long v = 0;
#pragma unroll
                for (int u = 0; u < KM_PPT; ++u) {
                    qv[u] = i0 + u < n ? fixq(__ldcg(d2n + i0 + u), sc.Sd) : 0;
                    v += qv[u];
                }
                const long long incl = block_scan_ll(v, s_red);
                long long run = s_base + incl - v;   // exclusive prefix of this thread's points
#pragma unroll
                for (int u = 0; u < KM_PPT; ++u) {
                    run += qv[u];
                    if (qv[u] > 0 && run > T) {
                        atomicMin(&s_idx, (int)(i0 + u));
                        break;
                    }
                }
            }
        }
        __syncthreads();
        if (tid == 0 && s_idx == INT_MAX) s_idx = lowest_unchosen(s_chosen, r);   // sum(D^2) = 0
        __syncthreads();
        if (tid == 0) {
            s_chosen[r] = s_idx;
            if (b == 0) a.seeds[r] = s_idx;
        }
        const bool pick_ok = in_range(s_idx, 0, n, BS_KPP_PICK);
        if (tid < LP) s_cent[(size_t)r * LP + tid] = tid < a.l && pick_ok ? a.X[(size_t)s_idx * LP + tid] : 0.f;
        __syncthreads();
    }
    if (b == 0) {
        for (int q = tid; q < a.k * LP; q += KM_THREADS) a.c32[q] = s_cent[q];
    }
}

// k_lloyd's dynamic shared memory: centroids (16-byte aligned), ntab private tables, half the
// separation of each centroid (k floats, padded to 8 bytes), the running totals k (LP + 1), the
// last move of each centroid (k floats), then (16-byte aligned) the per-warp point queues of
// KM_QUEUE entries (index, old label, lower bound).
constexpr int KM_QUEUE = 256;
__host__ __device__ inline size_t lloyd_queue_offset(int k, int LP, int ntab) {
    const size_t rowlen = (size_t)k * (LP + 1);
    const size_t end = (((size_t)k * LP * 4 + 15) & ~(size_t)15) + (size_t)ntab * rowlen * 8 +
                       (((size_t)k + 1) / 2) * 8 + rowlen * 8 + (size_t)k * 4;
    return (end + 15) & ~(size_t)15;
}

struct LloydArgs {
    const float* X;
    int n, l, k, max_iter;
    int32_t* labels;
    float* c32;                 // in: the k-means++ centres; out: the final centroids (float32)
    double* c64;                // out: the final centroids (float64)
    unsigned long long* tot;    // 3 accumulators of k*(LP+1) exact sums (coordinates, count), zeroed
    unsigned long long* cnt3;   // 3 x (inertia sum, changed count, 2 unused), then the final inertia; zeroed
    const unsigned* amax;
    int ntab;
    float* lbound;       // per point: lower bound on the distance to every other centroid (pruning)
    float* ubound;       // per point: upper bound on the distance to its own centroid (pruning)
    int prune;           // 1: skip the k-way scan of points whose bounds prove the label unchanged
    // The first assignment from the seeding (seeded = 1): each point's nearest of the k chosen
    // centres (near),
    // its D^2 (in the buffer dfl[chunk] names) and a lower bound on the distance to every other centre
    // (min of lb2 and the chunk's carried bound tlb[chunk]), instead of a k-way scan.  (d2s0 / d2s1:
    // the two D^2 buffers; chunks of KM_CHUNK points.)
    int seeded;
    const int* near;
    // after the first iteration `near` is free: each block lists there the points that need the k-way
    // scan, in its own region (see k_lloyd's phase A); pend is the same buffer, writable
    int* pend;
    const float* d2s0;
    const float* d2s1;
    const int* dfl;
    const float* lb2;
    const float* tlb;
    KmDevStats* st;
    GridBarrier* bar;
    int* status;
    long long limit;
    int stall;
    const double* guard;   // as in KppArgs
    double guard_lk, guard_thr;
};

// Exact pruning (Hamerly's bounds): a point whose distance to its current centroid is below
// max(s(a), lb) - where s(a) is half the distance from centroid a to its nearest other centroid
// and lb a lower bound on the distance to every other centroid - keeps its label without the
// k-way scan (triangle inequality).  The bounds are computed in float32 and widened by the
// relative margin PRUNE_EPS, far above the float32 rounding of the distances (< 1e-6), so a
// skipped point is exactly one the full scan would leave in place (no tie is possible).
constexpr float PRUNE_EPS = 1e-5f;
// From this k on, k_lloyd runs with BLIST: the points that fail the tight test go to the block-wide
// scan list.  Below it each warp scans its own (a scan of few centroids is cheap, and the list's
// block barrier and the split of the scans from the chunk pass cost more than the balance gains:
// measured 0.2 ms slower per clustering on a 154 K-point graph at k = 8, 0.3 ms faster on 4 M points
// at k = 100).  A template parameter, not a runtime test: both paths in one kernel spill registers.
constexpr int KM_BLOCK_LIST_MIN_K = 16;
constexpr float PRUNE_GROW2 = (1.0f + PRUNE_EPS) * (1.0f + PRUNE_EPS);   // the test runs on squares
// The upper bound u on a point's distance to its own centroid is carried from one iteration to
// the next by adding that centroid's movement (itself computed with a PRUNE_EPS margin), and the
// sum is grown by 4 ulp so its own float rounding can only raise it.
constexpr float UBOUND_GROW = 1.0f + 4.0f / 8388608.0f;

// Settles a point that went through the k-way scan: lower bound, label, changed count and, in the
// first iteration, its distance in the inertia.  The centroid sums are running totals, so only a
// point whose label changes contributes: its coordinates leave the old cluster and join the new
// one (in the first iteration every label changes from -1).  Labels are written only when they
// change.
template <int LP>
__device__ __forceinline__ void lloyd_commit(const LloydArgs& a, long long i, const float (&x)[LP], int oldl, int lab,
                                             float dist, float lbn, bool first, const Scales& sc, Slot<LP> (&sl)[2],
                                             unsigned long long* tab, long long& inert, int& changed) {
    if (a.prune) a.lbound[i] = lbn;
    if (first) inert += fixq(dist, sc.Sd);
    if (oldl != lab) {
        ++changed;
        a.labels[i] = lab;
        long long q[LP];
#pragma unroll
        for (int c = 0; c < LP; ++c) q[c] = fixq(x[c], sc.Sx);
        slot_add<LP>(sl, lab, q, false, tab);
        if (oldl >= 0) slot_add<LP>(sl, oldl, q, true, tab);
    }
}

template <int LP, bool BLIST>
__global__ void __launch_bounds__(KM_THREADS, 1) k_lloyd(LloydArgs a) {
    extern __shared__ __align__(16) unsigned char km_smem[];
    unsigned epoch = 0;   // grid barriers passed
    const int k = a.k;
    const int ntab = a.ntab;                              // private tables (warp w uses w % ntab)
    const size_t rowlen = (size_t)k * (LP + 1);
    float* s_c = reinterpret_cast<float*>(km_smem);
    unsigned long long* s_tab =
        reinterpret_cast<unsigned long long*>(km_smem + (((size_t)k * LP * 4 + 15) & ~(size_t)15));
    float* s_sep = reinterpret_cast<float*>(s_tab + (size_t)ntab * rowlen);   // k floats
    // running exact sums and counts of every cluster (the same in every block)
    long long* s_S = reinterpret_cast<long long*>(s_tab + (size_t)ntab * rowlen + (((size_t)k + 1) / 2));
    float* s_mv = reinterpret_cast<float*>(s_S + rowlen);   // k floats: each centroid's last move, grown
    // per-warp queues of points whose loose test failed: index, old label, decayed lower bound
    int* s_qidx = reinterpret_cast<int*>(km_smem + lloyd_queue_offset(k, LP, ntab));
    int* s_qold = s_qidx + KM_WARPS * KM_QUEUE;
    float* s_qlw = reinterpret_cast<float*>(s_qold + KM_WARPS * KM_QUEUE);
    // the new centroids, formed after the grid barrier in the queue indices' space (idle then; k LP
    // floats <= KM_WARPS KM_QUEUE since k ld <= 4096)
    float* s_cn = reinterpret_cast<float*>(s_qidx);
    __shared__ long long s_red[KM_WARPS];
    __shared__ int s_redi[KM_WARPS];
    __shared__ long long s_inert;
    __shared__ int s_changed;
    __shared__ unsigned s_pmax;
    __shared__ int s_pend;   // points in the block's list for the k-way scan (phase A)

    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const long long n = a.n;
    // a seeding that stopped on an error (a barrier timeout) left its per-point results
    // unwritten: report its status and leave
    if (*reinterpret_cast<volatile int*>(a.status) != 0) return;
    if (guard_rejects(a.guard, a.guard_lk, a.guard_thr)) return;   // every block alike: before any barrier
    // tiles of KM_TILE points, dealt round-robin (block b takes b, b + G, ...) in the final
    // inertia pass
    const long long ntl = (n + KM_TILE - 1) / KM_TILE;
    const int G = gridDim.x;
    const Scales sc = scales_for(__uint_as_float(__ldcg(a.amax)), n, a.l);
    unsigned long long* my_tab = s_tab + (size_t)(wid % ntab) * rowlen;

    for (int q = tid; q < k * LP; q += KM_THREADS) {
        const float v = __ldcg(a.c32 + q);
        s_c[q] = v;
        if (b == 0) a.c64[q] = (double)v;   // float64 masters of the k-means++ centres
    }
    for (size_t q = tid; q < rowlen; q += KM_THREADS) s_S[q] = 0;
    for (size_t q = tid; q < (size_t)ntab * rowlen; q += KM_THREADS) s_tab[q] = 0ull;   // then after each push
    if (tid == 0) {
        s_pmax = 0u;
        s_pend = 0;
    }
    __syncthreads();
    // The block's region of the scan list: its chunks' points, counted exactly (chunk c belongs to
    // block c mod G; the last chunk may be partial), so the regions of all blocks tile [0, n)
    long long pstart;
    {
        const long long nch0 = (n + KM_CHUNK - 1) / KM_CHUNK;
        const long long q_ = nch0 / G, r_ = nch0 % G, owner = (nch0 - 1) % G, missing = nch0 * KM_CHUNK - n;
        pstart = (long long)KM_CHUNK * ((long long)b * q_ + min((long long)b, r_)) - (owner < b ? missing : 0);
    }
    int* pend = a.pend + pstart;
    // One grid barrier per iteration: blocks add the changes of their clusters' exact sums into
    // the iteration's accumulator (one of three, used in rotation), and after the barrier every
    // block adds them to its running totals and forms all k centroids itself, so the centroids
    // never travel through global memory between blocks.  A point whose bounds prove its label
    // unchanged costs one distance and one store.
    for (int it = 1; it <= a.max_iter; ++it) {
        const int cur = it % 3;
        unsigned long long* T = a.tot + (size_t)cur * rowlen;
        const bool pr = a.prune && it > 1;
        // the tables are clear and (with pruning, from the second iteration on) s_sep holds half the
        // distance of each centroid to its nearest other one: both prepared by the previous update
        const float pmax = pr ? __uint_as_float(s_pmax) * (1.0f + PRUNE_EPS) : 0.f;
        long long inert = 0;
        int changed = 0;
        // ---- phase A.  Each thread takes KM_PPT consecutive points of a chunk and settles, from
        // its label and bounds alone, those whose upper bound u (carried forward by the centroid's
        // move) is below max(s(a), lower bound): Hamerly's test, without loading the point.  The
        // others go to a per-warp queue that the warp then works one point per lane with the exact
        // distance to the own centroid (the same test, tight); those it does not settle go to the
        // block's scan list, whose k-way scans all warps of the block share after the chunk pass.
        // Centroid sums are exact integers, so which lane adds a point changes no result.
        // Points are dealt in chunks of KM_CHUNK (one warp, four consecutive points per lane):
        // chunk c goes to block c mod G, warp (c / G) mod KM_WARPS, so the chunks of any vertex
        // range (a planted cluster's, whose boundary points all need the scan) spread over every
        // block instead of loading a few
        const long long nch = (n + KM_CHUNK - 1) / KM_CHUNK;
        auto chunk = [&](long long sq) -> long long {
            return (long long)b + (long long)G * ((long long)wid + (long long)KM_WARPS * sq);
        };
        Slot<LP> sl[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            sl[q].j = -1;
            sl[q].cnt = 0;
#pragma unroll
            for (int c = 0; c < LP; ++c) sl[q].s[c] = 0;
        }
        int* qidx = s_qidx + wid * KM_QUEUE;
        int* qold = s_qold + wid * KM_QUEUE;
        float* qlw = s_qlw + wid * KM_QUEUE;
        int qn = 0;   // queue length (warp-uniform)
        // the k-way scan of one point per lane (act: the lane has one): label, bounds, sums
        auto scan_point = [&](bool act, long long i, int oldl) {
            float xv[LP];
            load_point<LP>(a.X, i, a.l, xv);
            float best = __int_as_float(0x7f800000), sec = __int_as_float(0x7f800000);
            int bj = 0;
#pragma unroll 4
            for (int j = 0; j < k; ++j) {
                const float d = sqdist<LP>(xv, s_c + j * LP);
                if (d < best) {
                    sec = best;
                    best = d;
                    bj = j;
                } else if (d < sec) {
                    sec = d;
                }
            }
            if (act) {
                lloyd_commit<LP>(a, i, xv, oldl, bj, best, sqrtf(sec) * (1.0f - PRUNE_EPS), it == 1, sc, sl, my_tab,
                                 inert, changed);
                if (a.prune) a.ubound[i] = sqrtf(best) * (1.0f + PRUNE_EPS);
            }
        };
        // works the queued points: the tight test (the exact distance to the own centroid), 32 at a
        // time.  With BLIST the points it does not settle join the block's scan list, which all warps
        // of the block work together once the chunks are done, so a warp whose chunks hold many such
        // points does not hold up the block (the k-way scan, bound by its float32 issue, is most of
        // the work in the heavy iterations, and dealt by chunks the most loaded warp of a block
        // scanned about twice the mean).  Without, they are moved in place to the queue's front and
        // the warp scans them itself, every lane busy.
        auto flush = [&]() {
            __syncwarp();
            int nq = 0;   // without BLIST: points left for the warp's own scan (warp-uniform)
            for (int q0 = 0; q0 < qn; q0 += 32) {
                const int q = q0 + lane;
                const bool act = q < qn;
                const long long i = act ? qidx[q] : 0;
                const int oldl = act ? qold[q] : 0;
                const float lw = act ? qlw[q] : 0.f;
                bool settled = false;
                if (pr && act && in_range(oldl, 0, k, BS_LLOYD_LABEL)) {
                    float xv[LP];
                    load_point<LP>(a.X, i, a.l, xv);
                    const float da = sqdist<LP>(xv, s_c + oldl * LP);
                    const float bnd = fmaxf(s_sep[oldl], lw);
                    settled = da * PRUNE_GROW2 < bnd * bnd;
                    if (settled) {
                        a.lbound[i] = lw;
                        a.ubound[i] = sqrtf(da) * (1.0f + PRUNE_EPS);
                    }
                }
                const bool keep = act && !settled;
                const unsigned m = __ballot_sync(0xffffffffu, keep);
                if constexpr (BLIST) {
                    int base = 0;
                    if (lane == 0 && m) base = atomicAdd(&s_pend, __popc(m));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    // a point joins the list at most once per iteration, so the list stays within
                    // the block's region (its chunks' points)
                    if (keep) pend[base + __popc(m & ((1u << lane) - 1u))] = (int)i;
                } else {
                    __syncwarp();   // every lane has read its entry before any is overwritten
                    if (keep) {     // pos <= q: only entries already read are overwritten
                        const int pos = nq + __popc(m & ((1u << lane) - 1u));
                        qidx[pos] = (int)i;
                        qold[pos] = oldl;
                    }
                    nq += __popc(m);
                    __syncwarp();
                }
            }
            for (int q0 = 0; q0 < nq; q0 += 32) {
                const int q = q0 + lane;
                const bool act = q < nq;
                scan_point(act, act ? qidx[q] : 0, act ? qold[q] : 0);
            }
            __syncwarp();
            qn = 0;
        };
        if (it == 1 && a.seeded) {
            // The first assignment is the seeding's (near, D^2 and the lower bound come from
            // k-means++; see LloydArgs), and every label changes (from -1, the launcher's fill).
            // Every thread settles its own four points directly; their coordinates join the
            // centroid sums through table_add_grouped (one shared add per label where a warp's
            // points carry few labels, per-lane adds where they carry many).  Per-lane run caches
            // were slower (0.26 against 0.15 ms on 2^22 points): when the label changes at a chunk
            // boundary all 32 lanes evict into the same table row at once.
            const bool lab16 = (reinterpret_cast<uintptr_t>(a.labels) & 15) == 0;
            long long ch = chunk(0);
            int fl_n = ch < nch ? __ldcg(a.dfl + ch) : 0;
            for (long long sq = 0; ch < nch; ch = chunk(++sq)) {
                const long long i0 = ch * KM_CHUNK + (long long)KM_PPT * lane;
                const bool full4 = i0 + KM_PPT <= n;
                const float* d2s = (fl_n & 1) ? a.d2s1 : a.d2s0;
                const float tl = __ldcg(a.tlb + ch);
                const long long chn = chunk(sq + 1);
                fl_n = chn < nch ? __ldcg(a.dfl + chn) : 0;
                int nr[KM_PPT];
                float dd[KM_PPT], lbs[KM_PPT], x[KM_PPT][LP];
                if (full4) {
                    const int4 v = *reinterpret_cast<const int4*>(a.near + i0);
                    const float4 dv = *reinterpret_cast<const float4*>(d2s + i0);
                    const float4 lv = *reinterpret_cast<const float4*>(a.lb2 + i0);
                    nr[0] = v.x; nr[1] = v.y; nr[2] = v.z; nr[3] = v.w;
                    dd[0] = dv.x; dd[1] = dv.y; dd[2] = dv.z; dd[3] = dv.w;
                    lbs[0] = lv.x; lbs[1] = lv.y; lbs[2] = lv.z; lbs[3] = lv.w;
                } else {
#pragma unroll
                    for (int u = 0; u < KM_PPT; ++u) {
                        const bool in = i0 + u < n;
                        nr[u] = in ? a.near[i0 + u] : 0;
                        dd[u] = in ? d2s[i0 + u] : 0.f;
                        lbs[u] = in ? a.lb2[i0 + u] : 0.f;
                    }
                }
#pragma unroll
                for (int u = 0; u < KM_PPT; ++u) {
                    if (i0 + u < n) load_point<LP>(a.X, i0 + u, a.l, x[u]);
                    else
#pragma unroll
                        for (int c = 0; c < LP; ++c) x[u][c] = 0.f;
                }
                float lbo[KM_PPT], ubo[KM_PPT];
#pragma unroll
                for (int u = 0; u < KM_PPT; ++u) {
                    int bj = nr[u];
                    if (i0 + u < n && !in_range(bj, 0, k, BS_LLOYD_LABEL)) bj = 0;
                    nr[u] = min(max(bj, 0), k - 1);   // memory safety whatever the seeding left
                }
                // where every lane's four points share a label, a lane adds their sum (one grouped
                // add per chunk instead of four; |sum| < 2^62 since n >= 4 here)
                if (__all_sync(0xffffffffu, full4 && nr[0] == nr[1] && nr[1] == nr[2] && nr[2] == nr[3])) {
                    long long q[LP];
#pragma unroll
                    for (int c = 0; c < LP; ++c)
                        q[c] = fixq(x[0][c], sc.Sx) + fixq(x[1][c], sc.Sx) + fixq(x[2][c], sc.Sx) + fixq(x[3][c], sc.Sx);
                    table_add_grouped<LP>(nr[0], q, KM_PPT, my_tab);
                } else {
#pragma unroll
                    for (int u = 0; u < KM_PPT; ++u) {
                        const bool in = i0 + u < n;
                        long long q[LP];
#pragma unroll
                        for (int c = 0; c < LP; ++c) q[c] = in ? fixq(x[u][c], sc.Sx) : 0;
                        table_add_grouped<LP>(in ? nr[u] : -1, q, 1, my_tab);
                    }
                }
#pragma unroll
                for (int u = 0; u < KM_PPT; ++u) {
                    const bool in = i0 + u < n;
                    if (in) {
                        inert += fixq(dd[u], sc.Sd);
                        ++changed;
                    }
                    lbo[u] = fminf(lbs[u], tl);
                    ubo[u] = sqrtf(dd[u]) * (1.0f + PRUNE_EPS);
                }
                // lbound and ubound share the D^2 buffers: these points' D^2 were read above
                if (full4) {
                    if (lab16) *reinterpret_cast<int4*>(a.labels + i0) = make_int4(nr[0], nr[1], nr[2], nr[3]);
                    else
#pragma unroll
                        for (int u = 0; u < KM_PPT; ++u) a.labels[i0 + u] = nr[u];
                    if (a.prune) {
                        *reinterpret_cast<float4*>(a.lbound + i0) = make_float4(lbo[0], lbo[1], lbo[2], lbo[3]);
                        *reinterpret_cast<float4*>(a.ubound + i0) = make_float4(ubo[0], ubo[1], ubo[2], ubo[3]);
                    }
                } else {
#pragma unroll
                    for (int u = 0; u < KM_PPT; ++u)
                        if (i0 + u < n) {
                            a.labels[i0 + u] = nr[u];
                            if (a.prune) {
                                a.lbound[i0 + u] = lbo[u];
                                a.ubound[i0 + u] = ubo[u];
                            }
                        }
                }
            }
        }
        // labels and bounds of the chunks two steps ahead load while a chunk is settled (16-byte
        // loads where the rows allow: workspace bounds always, labels when the caller's array is
        // 16-byte aligned)
        const bool lab16 = (reinterpret_cast<uintptr_t>(a.labels) & 15) == 0;
        auto fetch = [&](long long ch, int (&o)[KM_PPT], float (&lbv)[KM_PPT], float (&ubv)[KM_PPT]) {
            const long long i0 = ch * KM_CHUNK + (long long)KM_PPT * lane;
            if (ch < nch && i0 + KM_PPT <= n) {
                if (lab16) {
                    const int4 v = *reinterpret_cast<const int4*>(a.labels + i0);
                    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
                } else {
#pragma unroll
                    for (int u = 0; u < KM_PPT; ++u) o[u] = a.labels[i0 + u];
                }
                if (pr) {
                    const float4 lv = *reinterpret_cast<const float4*>(a.lbound + i0);
                    const float4 uv = *reinterpret_cast<const float4*>(a.ubound + i0);
                    lbv[0] = lv.x; lbv[1] = lv.y; lbv[2] = lv.z; lbv[3] = lv.w;
                    ubv[0] = uv.x; ubv[1] = uv.y; ubv[2] = uv.z; ubv[3] = uv.w;
                } else {
#pragma unroll
                    for (int u = 0; u < KM_PPT; ++u) lbv[u] = ubv[u] = 0.f;
                }
            } else {
#pragma unroll
                for (int u = 0; u < KM_PPT; ++u) {
                    const bool in = ch < nch && i0 + u < n;
                    o[u] = in ? a.labels[i0 + u] : 0;
                    lbv[u] = in && pr ? a.lbound[i0 + u] : 0.f;
                    ubv[u] = in && pr ? a.ubound[i0 + u] : 0.f;
                }
            }
        };
        static_assert(KM_PPT == 4, "the 16-byte loads and stores take four points");
        int old_a[KM_PPT], old_b[KM_PPT];
        float lbv_a[KM_PPT], ubv_a[KM_PPT], lbv_b[KM_PPT], ubv_b[KM_PPT];
        const long long sq0 = (it == 1 && a.seeded) ? nch : 0;   // the seeded pass settled every point
        fetch(chunk(sq0), old_a, lbv_a, ubv_a);
        fetch(chunk(sq0 + 1), old_b, lbv_b, ubv_b);
        for (long long sq = sq0, ch = chunk(sq0); ch < nch; ch = chunk(++sq)) {
            const long long i0 = ch * KM_CHUNK + (long long)KM_PPT * lane;
            int old[KM_PPT];
            float lbv[KM_PPT], ubv[KM_PPT];
#pragma unroll
            for (int u = 0; u < KM_PPT; ++u) {
                old[u] = old_a[u];
                lbv[u] = lbv_a[u];
                ubv[u] = ubv_a[u];
                old_a[u] = old_b[u];
                lbv_a[u] = lbv_b[u];
                ubv_a[u] = ubv_b[u];
            }
            fetch(chunk(sq + 2), old_b, lbv_b, ubv_b);
            if (qn > KM_QUEUE - KM_PPT * 32) flush();   // room for this chunk's points
            float lw_s[KM_PPT], ub_s[KM_PPT];
            bool set_s[KM_PPT];
#pragma unroll
            for (int u = 0; u < KM_PPT; ++u) {
                bool need = i0 + u < n;
                float lw = 0.f;
                set_s[u] = false;
                lw_s[u] = ub_s[u] = 0.f;
                if (pr && need && in_range(old[u], 0, k, BS_LLOYD_LABEL)) {
                    const int ca = old[u];
                    lw = fmaxf(0.f, lbv[u] - pmax);
                    const float bnd = fmaxf(s_sep[ca], lw);
                    const float ub = (ubv[u] + s_mv[ca]) * UBOUND_GROW;
                    if (ub < bnd) {
                        set_s[u] = true;
                        lw_s[u] = lw;
                        ub_s[u] = ub;
                        need = false;
                    }
                }
                const unsigned m = __ballot_sync(0xffffffffu, need);
                if (need) {
                    const int pos = qn + __popc(m & ((1u << lane) - 1u));
                    qidx[pos] = (int)(i0 + u);
                    qold[pos] = old[u];
                    qlw[pos] = lw;
                }
                qn += __popc(m);
            }
            // the bounds of the points settled without their coordinates
            if (set_s[0] && set_s[1] && set_s[2] && set_s[3]) {
                *reinterpret_cast<float4*>(a.lbound + i0) = make_float4(lw_s[0], lw_s[1], lw_s[2], lw_s[3]);
                *reinterpret_cast<float4*>(a.ubound + i0) = make_float4(ub_s[0], ub_s[1], ub_s[2], ub_s[3]);
            } else {
#pragma unroll
                for (int u = 0; u < KM_PPT; ++u)
                    if (set_s[u]) {
                        a.lbound[i0 + u] = lw_s[u];
                        a.ubound[i0 + u] = ub_s[u];
                    }
            }
        }
        flush();
        if constexpr (BLIST) {
            __syncthreads();   // the block's scan list is complete (global writes of this block: visible)
            // the k-way scan of the listed points, 32 per warp at a time over all warps; a point's
            // label is still the one this iteration started from (a commit writes only its own)
            const int P = s_pend;
            for (int q0 = wid * 32; q0 < P; q0 += KM_WARPS * 32) {
                const int q = q0 + lane;
                const bool act = q < P;
                const long long i = act ? __ldcg(pend + q) : 0;
                scan_point(act, i, act ? a.labels[i] : 0);
            }
        }
        slot_flush_warp<LP>(sl[0], my_tab);
        slot_flush_warp<LP>(sl[1], my_tab);
        __syncthreads();
        // block totals -> the iteration's accumulator (two's-complement sums: order-free, exact)
        for (size_t q = tid; q < rowlen; q += KM_THREADS) {
            unsigned long long v = 0;
            for (int t = 0; t < ntab; ++t) v += s_tab[(size_t)t * rowlen + q];
            if (v) atomicAdd(T + q, v);
        }
        inert = block_sum_ll(inert, s_red);
        changed = block_sum_i(changed, s_redi);
        if (tid == 0) {
            if (inert) atomicAdd(a.cnt3 + 4 * cur, (unsigned long long)inert);
            if (changed) atomicAdd(a.cnt3 + 4 * cur + 1, (unsigned long long)changed);
        }
        // the tables were read before the block sums' barriers: clear them for the next iteration
        // while the grid gathers
        for (size_t q = tid; q < (size_t)ntab * rowlen; q += KM_THREADS) s_tab[q] = 0ull;
        if (!grid_sync(a.bar, a.status, a.limit, a.stall, epoch)) return;
        // ---- update, in every block: running totals += this iteration's changes (exact integer
        // adds, so every block holds the same totals); c_j = (exact sum of its points) / count,
        // rounded to float64 then float32; an empty cluster keeps its centroid
        for (size_t q = tid; q < rowlen; q += KM_THREADS) s_S[q] += (long long)__ldcg(T + q);
        if (tid == 0) {
            s_inert = (long long)__ldcg(a.cnt3 + 4 * cur);
            s_changed = (int)__ldcg(a.cnt3 + 4 * cur + 1);
            s_pmax = 0u;
            s_pend = 0;   // every warp has finished phase A's scans (the barriers above)
        }
        __syncthreads();
        for (int q = tid; q < k * LP; q += KM_THREADS) {
            const int j = q / LP, c = q - j * LP;
            const long long cntj = s_S[(size_t)j * (LP + 1) + LP];
            float v = s_c[q];
            if (cntj > 0) {
                const long long sj = s_S[(size_t)j * (LP + 1) + c];
                const double m = ((double)sj * pow2d(-sc.Sx)) / (double)cntj;
                v = (float)m;
                if (b == 0) a.c64[q] = m;
            }
            s_cn[q] = v;
        }
        __syncthreads();
        // on the last iteration s_c keeps the centroids its assignment used (for the inertia)
        const bool stop = s_changed == 0 || it == a.max_iter;
        // how far each centroid moved (bounds of the next assignment), empty-cluster events; and
        // for the next assignment half the distance of each new centroid to its nearest other one:
        // centroid j's candidates are dealt into `parts` interleaved subsets, one thread each, whose
        // minima one thread per centroid combines below (no shared atomics; (a - b)^2 = (b - a)^2
        // exactly, so d(j, jj) = d(jj, j) and the result equals a scan over pairs)
        for (int j = tid; j < k; j += KM_THREADS) {
            float mv = 0.f;
#pragma unroll
            for (int c = 0; c < LP; ++c) {
                const float dlt = __fsub_rn(s_cn[j * LP + c], s_c[j * LP + c]);
                mv = __fadd_rn(mv, __fmul_rn(dlt, dlt));
            }
            s_mv[j] = sqrtf(mv) * (1.0f + PRUNE_EPS);
            atomicMax(&s_pmax, __float_as_uint(s_mv[j]));
            if (b == 0 && s_S[(size_t)j * (LP + 1) + LP] == 0) atomicAdd(&a.st->empty_events, 1);
        }
        const bool sep_next = a.prune && !stop;
        const int parts = k >= KM_THREADS ? 1 : KM_THREADS / k;
        float* s_part = s_qlw;   // the point queues are idle until phase A
        if (sep_next) {
            for (int q = tid; q < k * parts; q += KM_THREADS) {
                const int j = q / parts, p = q - j * parts;
                float cj[LP];
#pragma unroll
                for (int c = 0; c < LP; ++c) cj[c] = s_cn[j * LP + c];
                float m = __int_as_float(0x7f800000);   // +inf: k = 1 has no other centroid
                for (int jj = p; jj < k; jj += parts)
                    if (jj != j) m = fminf(m, sqdist<LP>(cj, s_cn + jj * LP));
                if (parts == 1) s_sep[j] = 0.5f * sqrtf(m) * (1.0f - PRUNE_EPS);
                else s_part[q] = m;
            }
        }
        // the accumulator of iteration it+2 was last read after the previous barrier: clear it
        if (b == 0) {
            unsigned long long* Tz = a.tot + (size_t)((it + 2) % 3) * rowlen;
            for (size_t q = tid; q < rowlen; q += KM_THREADS) Tz[q] = 0ull;
            if (tid < 4) a.cnt3[4 * ((it + 2) % 3) + tid] = 0ull;
        }
        if (b == 0 && tid == 0) {
            if (it == 1) a.st->potential = (double)s_inert * pow2d(-sc.Sd);
            a.st->iterations = it;
            a.st->changed = s_changed;
        }
        __syncthreads();
        if (stop) break;
        if (sep_next && parts > 1) {
            for (int j = tid; j < k; j += KM_THREADS) {
                float m = s_part[j * parts];
                for (int p = 1; p < parts; ++p) m = fminf(m, s_part[j * parts + p]);
                s_sep[j] = 0.5f * sqrtf(m) * (1.0f - PRUNE_EPS);
            }
        }
        for (int q = tid; q < k * LP; q += KM_THREADS) s_c[q] = s_cn[q];
        __syncthreads();
    }
    // ---- inertia of the last assignment: each point's float32 distance to the centroid it was
    // assigned to (the same value the assignment computed), summed exactly in fixed point
    long long inert = 0;
    for (long long tile = b; tile < ntl; tile += G) {
        const long long t0 = tile * KM_TILE, hi = min(n, t0 + KM_TILE);
        const long long i0 = t0 + (long long)KM_PPT * tid;
#pragma unroll
        for (int u = 0; u < KM_PPT; ++u) {
            if (i0 + u < hi) {
                float x[LP];
                load_point<LP>(a.X, i0 + u, a.l, x);
                const int lab = a.labels[i0 + u];
                if (in_range(lab, 0, k, BS_LLOYD_LABEL)) inert += fixq(sqdist<LP>(x, s_c + lab * LP), sc.Sd);
            }
        }
    }
    inert = block_sum_ll(inert, s_red);
    if (tid == 0 && inert) atomicAdd(a.cnt3 + 12, (unsigned long long)inert);
    if (!grid_sync(a.bar, a.status, a.limit, a.stall, epoch)) return;
    if (b == 0) {
        if (tid == 0) a.st->inertia = (double)(long long)__ldcg(a.cnt3 + 12) * pow2d(-sc.Sd);
        for (int q = tid; q < k * LP; q += KM_THREADS) a.c32[q] = s_cn[q];
    }
}

__global__ void k_merge_status(const int* __restrict__ call_status, int* __restrict__ dev_status) {
    if (*call_status) atomicOr(dev_status, *call_status);
}

static size_t lloyd_smem_bytes(int k, int LP, int ntab) {
    return lloyd_queue_offset(k, LP, ntab) + (size_t)KM_WARPS * KM_QUEUE * 12;
}

// Workspace of one k-means call: header (stats, grid barrier, status, max |x|) and the Lloyd
// accumulators (zeroed together), the two D^2 buffers, the per-tile k-means++ state (zeroed: exact
// totals x 3, buffer masks x 3), the per-chunk state (zeroed: buffer flags x 2; not zeroed: totals
// x 2, largest D^2 x 2, centres, radii, carried bounds), the centroids (float64, float32), the
// k-means++ picks and each point's nearest chosen centre and lower bound.
struct KmLayout {
    size_t hdr, acc, o_d2, o_tt, tt_bytes, o_cs, cs_zero, o_c64, o_c32, o_seed, o_near, o_lb2, total;
    size_t d2_stride, tt8, tt4, c8, c4, ccen;
};

static size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

static KmLayout km_layout(long long n, int k, int LP) {
    KmLayout L{};
    const long long ntiles = (n + KM_TILE - 1) / KM_TILE;
    const long long nch = (n + KM_CHUNK - 1) / KM_CHUNK;
    L.hdr = up256(sizeof(KmDevStats) + sizeof(GridBarrier) + 2 * sizeof(int) + sizeof(unsigned));
    L.acc = up256((size_t)3 * k * (LP + 1) * 8 + 16 * 8);
    L.d2_stride = up256((size_t)n * 4);
    L.tt8 = up256((size_t)ntiles * 8);
    L.tt4 = up256((size_t)ntiles * 4);
    L.c8 = up256((size_t)nch * 8);
    L.c4 = up256((size_t)nch * 4);
    L.ccen = up256((size_t)nch * LP * 4);
    size_t off = L.hdr + L.acc;
    L.o_d2 = off; off += 2 * L.d2_stride;
    L.o_tt = off; L.tt_bytes = 3 * L.tt8 + 3 * L.tt4; off += L.tt_bytes;
    L.o_cs = off; L.cs_zero = 2 * L.c4; off += 2 * L.c4 + 2 * L.c8 + 2 * L.c4 + L.ccen + 2 * L.c4;
    L.o_c64 = off; off += up256((size_t)k * LP * 8);
    L.o_c32 = off; off += up256((size_t)k * LP * 4);
    L.o_seed = off; off += up256((size_t)k * 8);
    L.o_near = off; off += up256((size_t)n * 4);
    L.o_lb2 = off; off += up256((size_t)n * 4);
    L.total = off;
    return L;
}

// Points the k-means++ arguments at the buffers of a workspace laid out by km_layout.
static void kpp_buffers(KppArgs& ka, char* ws, const KmLayout& L) {
    ka.d2[0] = reinterpret_cast<float*>(ws + L.o_d2);
    ka.d2[1] = reinterpret_cast<float*>(ws + L.o_d2 + L.d2_stride);
    char* t = ws + L.o_tt;
    for (int q = 0; q < 3; ++q) ka.ttot[q] = reinterpret_cast<long long*>(t + q * L.tt8);
    t += 3 * L.tt8;
    for (int q = 0; q < 3; ++q) ka.tmask[q] = reinterpret_cast<unsigned*>(t + q * L.tt4);
    char* c = ws + L.o_cs;
    for (int q = 0; q < 2; ++q) ka.cfl[q] = reinterpret_cast<int*>(c + q * L.c4);
    c += 2 * L.c4;
    for (int q = 0; q < 2; ++q) ka.ctot[q] = reinterpret_cast<long long*>(c + q * L.c8);
    c += 2 * L.c8;
    for (int q = 0; q < 2; ++q) ka.cdmax[q] = reinterpret_cast<unsigned*>(c + q * L.c4);
    c += 2 * L.c4;
    ka.ccen = reinterpret_cast<float*>(c);
    c += L.ccen;
    ka.crad = reinterpret_cast<float*>(c);
    ka.clb = reinterpret_cast<float*>(c + L.c4);
    ka.lb2 = reinterpret_cast<float*>(ws + L.o_lb2);
    ka.seeds = reinterpret_cast<int64_t*>(ws + L.o_seed);
    ka.near = reinterpret_cast<int*>(ws + L.o_near);
    ka.c32 = reinterpret_cast<float*>(ws + L.o_c32);
}

template <typename K>
static int coop_blocks(K kern, size_t smem) {
    int per_sm = kernel_occupancy((const void*)kern, KM_THREADS, smem);
    if (per_sm > 2) per_sm = 2;
    return per_sm * device_props().num_sms;
}

template <int LP>
static fsc_status kmeans_lp(const float* emb, int n, int l, int k, uint64_t seed, int max_iter, int32_t* labels,
                            double* centroids, int64_t* seed_idx, fsc_kmeans_stats* stats, cudaStream_t s,
                            const double* guard = nullptr, double guard_thr = 0.0) {
    const size_t kpp_smem = (size_t)k * (sizeof(int) + sizeof(float) + LP * sizeof(float));
    // private accumulation tables: as many as fit in 64 KB (at least one, at most one per warp)
    const size_t tab_bytes = (size_t)k * (LP + 1) * 8;
    int ntab = (int)(65536 / tab_bytes);
    if (ntab > KM_WARPS) ntab = KM_WARPS;
    if (ntab < 1) ntab = 1;
    const size_t lloyd_smem = lloyd_smem_bytes(k, LP, ntab);
    auto kpp = k_kmeanspp<LP>;
    auto lly = k >= KM_BLOCK_LIST_MIN_K ? k_lloyd<LP, true> : k_lloyd<LP, false>;
    int G = coop_blocks(kpp, kpp_smem);
    const int G2 = coop_blocks(lly, lloyd_smem);
    if (G2 < G) G = G2;
    if (G < 1) return FSC_ERR_CUDA;
    if (G > KM_MAX_BLOCKS) G = KM_MAX_BLOCKS;
    // no more blocks than tiles of KM_TILE points (the unit of the final inertia pass)
    const long long ntiles = ((long long)n + KM_TILE - 1) / KM_TILE;
    if (G > ntiles) G = (int)ntiles;

    const KmLayout Lw = km_layout(n, k, LP);
    char* ws = nullptr;
    cudaError_t e = pool_malloc(reinterpret_cast<void**>(&ws), Lw.total, s);
    if (e != cudaSuccess) return cuda_status(e);
    fsc_status rc = FSC_OK;
    KmDevStats* st = reinterpret_cast<KmDevStats*>(ws);
    GridBarrier* bar = reinterpret_cast<GridBarrier*>(ws + sizeof(KmDevStats));
    int* call_status = reinterpret_cast<int*>(ws + sizeof(KmDevStats) + sizeof(GridBarrier));
    unsigned* amax = reinterpret_cast<unsigned*>(ws + sizeof(KmDevStats) + sizeof(GridBarrier) + 8);
    do {
        if ((e = cudaMemsetAsync(ws, 0, Lw.hdr + Lw.acc, s)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(labels, 0xff, (size_t)n * 4, s)) != cudaSuccess) break;
        KppArgs ka{};
        ka.X = emb;
        ka.n = n;
        ka.l = l;
        ka.k = k;
        ka.seed = seed;
        kpp_buffers(ka, ws, Lw);
        if ((e = cudaMemsetAsync(ws + Lw.o_tt, 0, Lw.tt_bytes, s)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(ws + Lw.o_cs, 0, Lw.cs_zero, s)) != cudaSuccess) break;
        ka.amax = amax;
        ka.bar = bar;
        ka.status = call_status;
        ka.limit = wait_limit_ns();
        ka.stall = barrier_stall();
        ka.guard = guard;
        ka.guard_lk = (double)l * (double)k;
        ka.guard_thr = guard_thr;
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
        la.c64 = reinterpret_cast<double*>(ws + Lw.o_c64);
        la.tot = reinterpret_cast<unsigned long long*>(ws + Lw.hdr);
        la.cnt3 = la.tot + (size_t)3 * k * (LP + 1);
        la.amax = amax;
        la.ntab = ntab;
        la.lbound = ka.d2[0];          // the k-means++ D^2 buffers are free once seeding is done
        la.ubound = ka.d2[1];
        la.prune = k <= 256 ? 1 : 0;
        la.seeded = 1;
        la.near = ka.near;
        la.pend = ka.near;
        la.d2s0 = ka.d2[0];
        la.d2s1 = ka.d2[1];
        la.dfl = ka.cfl[k & 1];   // the chunk flags after the final pass (r = k)
        la.lb2 = ka.lb2;
        la.tlb = ka.clb;
        la.st = st;
        la.bar = bar;
        la.status = call_status;
        la.limit = ka.limit;
        la.stall = ka.stall;
        la.guard = ka.guard;
        la.guard_lk = ka.guard_lk;
        la.guard_thr = ka.guard_thr;
        void* largs[] = {&la};
        if ((e = cudaLaunchCooperativeKernel((const void*)lly, dim3(G), dim3(KM_THREADS), largs, lloyd_smem, s)) != cudaSuccess) break;
        if (centroids)
            if ((e = cudaMemcpy2DAsync(centroids, (size_t)l * 8, la.c64, (size_t)LP * 8, (size_t)l * 8, (size_t)k,
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
    cudaError_t ef = pool_free(ws, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (ef != cudaSuccess) return cuda_status(ef);
    return rc;
}

FSC_BOUNDS_READER(kmeans)

// rows of 16 .. 128 floats (kmeans_wide.cu)
fsc_status kmeans_wide(const float* emb, int n, int l, int ld, int k, uint64_t seed, int max_iter, int32_t* labels,
                       double* centroids, int64_t* seed_idx, fsc_kmeans_stats* stats, cudaStream_t s);

// fsc_kmeans for rows of at most 8 floats whose launches return at once when the learned filter's
// energy guard rejects the embedding (energy / (l k) not <= thr, read on the device): the caller
// then discards labels and stats (labels are left at -1).  guard = nullptr: plain fsc_kmeans.
fsc_status kmeans_guarded(const float* emb, int64_t n, int l, int ld, int k, uint64_t seed, int max_iter,
                          int32_t* labels, fsc_kmeans_stats* stats, const double* guard, double guard_thr,
                          cudaStream_t s) {
    switch (ld) {
        case 1: return kmeans_lp<1>(emb, (int)n, l, k, seed, max_iter, labels, nullptr, nullptr, stats, s, guard, guard_thr);
        case 2: return kmeans_lp<2>(emb, (int)n, l, k, seed, max_iter, labels, nullptr, nullptr, stats, s, guard, guard_thr);
        case 4: return kmeans_lp<4>(emb, (int)n, l, k, seed, max_iter, labels, nullptr, nullptr, stats, s, guard, guard_thr);
        case 8: return kmeans_lp<8>(emb, (int)n, l, k, seed, max_iter, labels, nullptr, nullptr, stats, s, guard, guard_thr);
    }
    return FSC_ERR_INVALID_ARG;
}

}  // namespace fsc

using namespace fsc;

extern "C" fsc_status fsc_kmeans(const float* emb, int64_t n, int l, int ld, int k, uint64_t seed, int max_iter,
                                 int32_t* labels, double* centroids, int64_t* seed_idx, fsc_kmeans_stats* stats,
                                 void* stream) {
    NvtxRange nvtx_range("fsc_kmeans");
    if (!emb || !labels || n < 1 || n > 2147483647LL || l < 1 || l > ld || k < 1 || (int64_t)k > n || k > 1024 ||
        max_iter < 1)
        return FSC_ERR_INVALID_ARG;
    if (ld != 1 && ld != 2 && ld != 4 && ld != 8 && ld != 16 && ld != 32 && ld != 64 && ld != 128)
        return FSC_ERR_INVALID_ARG;
    if ((int64_t)k * ld > (ld <= 8 ? 4096 : 32768)) return FSC_ERR_INVALID_ARG;
    const size_t al = (size_t)ld * 4 < 16 ? (size_t)ld * 4 : 16;
    if (reinterpret_cast<uintptr_t>(emb) % al) return FSC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if (ld > 8) return kmeans_wide(emb, (int)n, l, ld, k, seed, max_iter, labels, centroids, seed_idx, stats, s);
    switch (ld) {
        case 1: return kmeans_lp<1>(emb, (int)n, l, k, seed, max_iter, labels, centroids, seed_idx, stats, s);
        case 2: return kmeans_lp<2>(emb, (int)n, l, k, seed, max_iter, labels, centroids, seed_idx, stats, s);
        case 4: return kmeans_lp<4>(emb, (int)n, l, k, seed, max_iter, labels, centroids, seed_idx, stats, s);
        case 8: return kmeans_lp<8>(emb, (int)n, l, k, seed, max_iter, labels, centroids, seed_idx, stats, s);
    }
    return FSC_ERR_INVALID_ARG;
}

// Restarts: run r seeds k-means++ with seed + r; the run of lowest inertia wins (ties: lowest r).
// Two label (and centroid / seed) buffers swap roles, so the winner is copied at most once.
extern "C" fsc_status fsc_kmeans_best(const float* emb, int64_t n, int l, int ld, int k, uint64_t seed, int n_init,
                                      int max_iter, int32_t* labels, double* centroids, int64_t* seed_idx,
                                      fsc_kmeans_stats* stats, int32_t* best_run, void* stream) {
    NvtxRange nvtx_range("fsc_kmeans_best");
    if (n_init < 1 || n_init > 1000000 || !labels || n < 1 || n > 2147483647LL || k < 1 || l < 1 || l > 128)
        return FSC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    char* spare = nullptr;
    const size_t lab_b = ((size_t)n * 4 + 255) & ~(size_t)255;
    const size_t cen_b = (((size_t)k * l * 8) + 255) & ~(size_t)255;
    const size_t sd_b = (((size_t)k * 8) + 255) & ~(size_t)255;
    if (n_init > 1) {
        cudaError_t e = pool_malloc(reinterpret_cast<void**>(&spare), lab_b + cen_b + sd_b, s);
        if (e != cudaSuccess) return cuda_status(e);
    }
    int32_t* lab_buf[2] = {labels, reinterpret_cast<int32_t*>(spare)};
    double* cen_buf[2] = {centroids, centroids ? reinterpret_cast<double*>(spare + lab_b) : nullptr};
    int64_t* sd_buf[2] = {seed_idx, seed_idx ? reinterpret_cast<int64_t*>(spare + lab_b + cen_b) : nullptr};
    int best = -1, cur = 0, best_buf = 0;
    fsc_kmeans_stats best_st{};
    fsc_status rc = FSC_OK;
    for (int r = 0; r < n_init && rc == FSC_OK; ++r) {
        fsc_kmeans_stats st{};
        rc = fsc_kmeans(emb, n, l, ld, k, seed + (uint64_t)r, max_iter, lab_buf[cur], cen_buf[cur], sd_buf[cur], &st,
                        stream);
        if (rc != FSC_OK) break;
        if (best < 0 || st.inertia < best_st.inertia) {
            best = r;
            best_st = st;
            best_buf = cur;
            cur ^= 1;   // keep the winner, run the next restart in the other buffer
        }
    }
    if (rc == FSC_OK && best_buf == 1) {
        cudaError_t e = cudaMemcpyAsync(labels, lab_buf[1], (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && centroids)
            e = cudaMemcpyAsync(centroids, cen_buf[1], (size_t)k * l * 8, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess && seed_idx)
            e = cudaMemcpyAsync(seed_idx, sd_buf[1], (size_t)k * 8, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_status(e);
    }
    if (spare) {
        pool_free(spare, s);
        cudaStreamSynchronize(s);
    }
    if (rc == FSC_OK) {
        if (stats) *stats = best_st;
        if (best_run) *best_run = best;
    }
    return rc;
}

extern "C" fsc_status fsc_cluster(const fsc_graph* g, int k, int l, int t, uint64_t seed, fsc_dtype store,
                                  int max_iter, int32_t* labels, fsc_kmeans_stats* stats, const fsc_embed_opts* opts,
                                  void* stream) {
    NvtxRange nvtx_range("fsc_cluster");
    if (!g || !labels || l < 1 || l > 8 || k < 1 || (int64_t)k > g->n) return FSC_ERR_INVALID_ARG;
    const int LP = pad_l(l);
    cudaStream_t s = as_stream(stream);
    float* emb = nullptr;
    cudaError_t e = pool_malloc(reinterpret_cast<void**>(&emb), (size_t)g->n * LP * 4, s);
    if (e != cudaSuccess) return cuda_status(e);
    fsc_kmeans_stats local{};
    fsc_status rc = fsc_embed(g, l, t, seed, store, emb, opts, stream);
    if (rc == FSC_OK)
        rc = fsc_kmeans(emb, g->n, l, LP, k, seed, max_iter, labels, nullptr, nullptr, stats ? stats : &local, stream);
    cudaError_t ef = pool_free(emb, s);
    if (rc == FSC_OK && ef != cudaSuccess) rc = cuda_status(ef);
    if (rc == FSC_OK) {
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) rc = cuda_status(e);
    }
    return rc;
}

// ---------------------------------------------------------------------------------------------
// fsc_kmeans_static: the same k-means++ and Lloyd kernels, with every scratch buffer carved out
// of one fixed device array instead of a stream-ordered allocation.  For callers that must not
// allocate device memory while they run (code inside a memory-capped or pre-sized runtime, or a
// real-time loop whose memory is reserved up front): the array below is part of the library's
// device image, so it exists on every GPU that loads the library and stays reserved until the
// process exits.
// ---------------------------------------------------------------------------------------------
namespace fsc {

static __device__ __align__(256) unsigned char g_kmeans_static_scratch[FSC_KMEANS_STATIC_SCRATCH_BYTES];

namespace {
// Host code cannot use the array's name as a device address.  The address is looked up on every
// call, with the caller's device current: the lookup allocates nothing and costs little next to
// the synchronous k-means, and an address kept from an earlier call could outlive its context
// (cudaDeviceReset, or a caller that switches primary contexts) or keep a failed first lookup.
cudaError_t static_scratch(void** out) {
    *out = nullptr;
    return cudaGetSymbolAddress(out, g_kmeans_static_scratch);
}
}  // namespace

template <int LP>
static fsc_status kmeans_lp_static(const float* emb, int n, int l, int k, uint64_t seed, int max_iter,
                                   int32_t* labels, double* centroids, int64_t* seed_idx, fsc_kmeans_stats* stats,
                                   cudaStream_t s) {
    // the call ends with a host wait and host copies, which a stream capture cannot hold
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FSC_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) return FSC_ERR_INVALID_ARG;
    void* basep = nullptr;
    FSC_CUDA(static_scratch(&basep));
    char* ws = static_cast<char*>(basep);
    if (!ws) return FSC_ERR_CUDA;

    const size_t kpp_smem = (size_t)k * (sizeof(int) + sizeof(float) + LP * sizeof(float));
    const size_t tab_bytes = (size_t)k * (LP + 1) * 8;
    int ntab = (int)(65536 / tab_bytes);
    if (ntab > KM_WARPS) ntab = KM_WARPS;
    if (ntab < 1) ntab = 1;
    const size_t lloyd_smem = lloyd_smem_bytes(k, LP, ntab);
    auto kpp = k_kmeanspp<LP>;
    auto lly = k >= KM_BLOCK_LIST_MIN_K ? k_lloyd<LP, true> : k_lloyd<LP, false>;
    int G = coop_blocks(kpp, kpp_smem);
    const int G2 = coop_blocks(lly, lloyd_smem);
    if (G2 < G) G = G2;
    if (G < 1) return FSC_ERR_CUDA;
    if (G > KM_MAX_BLOCKS) G = KM_MAX_BLOCKS;
    const long long ntiles = ((long long)n + KM_TILE - 1) / KM_TILE;   // no more blocks than tiles
    if (G > ntiles) G = (int)ntiles;

    const KmLayout Lw = km_layout(n, k, LP);
    if (Lw.total > (size_t)FSC_KMEANS_STATIC_SCRATCH_BYTES) return FSC_ERR_TOO_LARGE;

    KmDevStats* st = reinterpret_cast<KmDevStats*>(ws);
    GridBarrier* bar = reinterpret_cast<GridBarrier*>(ws + sizeof(KmDevStats));
    int* call_status = reinterpret_cast<int*>(ws + sizeof(KmDevStats) + sizeof(GridBarrier));
    unsigned* amax = reinterpret_cast<unsigned*>(ws + sizeof(KmDevStats) + sizeof(GridBarrier) + 8);
    // the array keeps the previous call's contents: clear what the kernels expect to start at zero
    FSC_CUDA(cudaMemsetAsync(ws, 0, Lw.hdr + Lw.acc, s));
    FSC_CUDA(cudaMemsetAsync(labels, 0xff, (size_t)n * 4, s));
    KppArgs ka{};
    ka.X = emb;
    ka.n = n;
    ka.l = l;
    ka.k = k;
    ka.seed = seed;
    kpp_buffers(ka, ws, Lw);
    FSC_CUDA(cudaMemsetAsync(ws + Lw.o_tt, 0, Lw.tt_bytes, s));
    FSC_CUDA(cudaMemsetAsync(ws + Lw.o_cs, 0, Lw.cs_zero, s));
    ka.amax = amax;
    ka.bar = bar;
    ka.status = call_status;
    ka.limit = wait_limit_ns();
    ka.stall = barrier_stall();
    void* kargs[] = {&ka};
    FSC_CUDA(cudaLaunchCooperativeKernel((const void*)kpp, dim3(G), dim3(KM_THREADS), kargs, kpp_smem, s));
    FSC_CUDA(cudaMemsetAsync(bar, 0, sizeof(GridBarrier), s));
    LloydArgs la{};
    la.X = emb;
    la.n = n;
    la.l = l;
    la.k = k;
    la.max_iter = max_iter;
    la.labels = labels;
    la.c32 = ka.c32;
    la.c64 = reinterpret_cast<double*>(ws + Lw.o_c64);
    la.tot = reinterpret_cast<unsigned long long*>(ws + Lw.hdr);
    la.cnt3 = la.tot + (size_t)3 * k * (LP + 1);
    la.amax = amax;
    la.ntab = ntab;
    la.lbound = ka.d2[0];
    la.ubound = ka.d2[1];
    la.prune = k <= 256 ? 1 : 0;
    la.seeded = 1;
    la.near = ka.near;
    la.pend = ka.near;
    la.d2s0 = ka.d2[0];
    la.d2s1 = ka.d2[1];
    la.dfl = ka.cfl[k & 1];   // the chunk flags after the final pass (r = k)
    la.lb2 = ka.lb2;
    la.tlb = ka.clb;
    la.st = st;
    la.bar = bar;
    la.status = call_status;
    la.limit = ka.limit;
    la.stall = ka.stall;
    void* largs[] = {&la};
    FSC_CUDA(cudaLaunchCooperativeKernel((const void*)lly, dim3(G), dim3(KM_THREADS), largs, lloyd_smem, s));
    if (centroids)
        FSC_CUDA(cudaMemcpy2DAsync(centroids, (size_t)l * 8, la.c64, (size_t)LP * 8, (size_t)l * 8, (size_t)k,
                                   cudaMemcpyDeviceToDevice, s));
    if (seed_idx) FSC_CUDA(cudaMemcpyAsync(seed_idx, ka.seeds, (size_t)k * 8, cudaMemcpyDeviceToDevice, s));
    KmDevStats hst{};
    int hstatus = 0;
    FSC_CUDA(cudaMemcpyAsync(&hst, st, sizeof(hst), cudaMemcpyDeviceToHost, s));
    FSC_CUDA(cudaMemcpyAsync(&hstatus, call_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    FSC_CUDA(cudaStreamSynchronize(s));
    const fsc_status rc = status_from_bits(hstatus);
    if (stats) {
        stats->iterations = hst.iterations;
        stats->changed = hst.changed;
        stats->empty_events = hst.empty_events;
        stats->device_status = (int32_t)rc;
        stats->inertia = hst.inertia;
        stats->seeding_potential = hst.potential;
    }
    return rc;
}

}  // namespace fsc

extern "C" fsc_status fsc_kmeans_static(const float* emb, int64_t n, int l, int ld, int k, uint64_t seed,
                                        int max_iter, int32_t* labels, double* centroids, int64_t* seed_idx,
                                        fsc_kmeans_stats* stats, void* stream) {
    NvtxRange nvtx_range("fsc_kmeans_static");
    if (!emb || !labels || n < 1 || n > 2147483647LL || l < 1 || l > ld || k < 1 || (int64_t)k > n || k > 1024 ||
        max_iter < 1)
        return FSC_ERR_INVALID_ARG;
    if (ld != 1 && ld != 2 && ld != 4 && ld != 8) return FSC_ERR_INVALID_ARG;
    if ((int64_t)k * ld > 4096) return FSC_ERR_INVALID_ARG;
    const size_t al = (size_t)ld * 4 < 16 ? (size_t)ld * 4 : 16;
    if (reinterpret_cast<uintptr_t>(emb) % al) return FSC_ERR_INVALID_ARG;
    cudaStream_t s = fsc::as_stream(stream);
    switch (ld) {
        case 1: return fsc::kmeans_lp_static<1>(emb, (int)n, l, k, seed, max_iter, labels, centroids, seed_idx, stats, s);
        case 2: return fsc::kmeans_lp_static<2>(emb, (int)n, l, k, seed, max_iter, labels, centroids, seed_idx, stats, s);
        case 4: return fsc::kmeans_lp_static<4>(emb, (int)n, l, k, seed, max_iter, labels, centroids, seed_idx, stats, s);
        case 8: return fsc::kmeans_lp_static<8>(emb, (int)n, l, k, seed, max_iter, labels, centroids, seed_idx, stats, s);
    }
    return FSC_ERR_INVALID_ARG;
}
