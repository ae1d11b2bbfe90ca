// Helpers shared by the k-means kernels: fixed-point scales and conversions, block
// reductions and scans, point loads, and the per-thread run accumulators of Lloyd.
// The fixed-point scheme is described in kmeans.cu.
#pragma once

#include <limits.h>

#include "fsc_internal.cuh"

namespace fsc {

constexpr int KM_THREADS = 512;
constexpr int KM_WARPS = KM_THREADS / 32;
constexpr int KM_MAX_BLOCKS = 1024;
constexpr int KM_PPT = 4;                          // consecutive points per lane in a chunk or tile
constexpr int KM_TILE = KM_THREADS * KM_PPT;       // points per tile (one block's four points per thread)
constexpr int KM_CHUNK = 32 * KM_PPT;              // points per warp chunk (Lloyd's unit of work)
constexpr int KM_CHUNKS_PER_TILE = KM_TILE / KM_CHUNK;

struct KmDevStats {
    int iterations;
    int changed;
    int empty_events;
    int status;
    double inertia;
    double potential;
};

// ---- fixed-point helpers ---------------------------------------------------------------
__device__ __forceinline__ long long fixq(float x, int S) {
    const unsigned b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xffu);
    if (e == 0 || e == 0xff) return 0;                     // zero / subnormal (below resolution)
    const long long m = (long long)((b & 0x7fffffu) | 0x800000u);   // |x| = m * 2^(e - 150)
    const int sh = e - 150 + S;
    long long v;
    if (sh >= 0) v = sh < 39 ? (m << sh) : (m << 38);      // sh < 39 whenever |x| < 2^(62-S)
    else v = sh > -25 ? (m >> -sh) : 0;
    return (b >> 31) ? -v : v;
}
__device__ __forceinline__ double pow2d(int e) {          // 2^e as a double, e in [-1022, 1023]
    return __longlong_as_double((long long)(1023 + e) << 52);
}
__device__ __forceinline__ int ceil_log2(long long v) {    // smallest c with 2^c >= v (v >= 1)
    int c = 0;
    while ((1LL << c) < v) ++c;
    return c;
}
struct Scales {
    int Sx, Sd;
};
__device__ __forceinline__ Scales scales_for(float A, long long n, int l) {
    const int N = ceil_log2(n < 2 ? 2 : n);
    const int Ex = A > 0.f ? exponent_of(A) + 1 : 0;
    const int Ed = 2 * Ex + ceil_log2(l) + 3;
    Scales s;
    s.Sx = 62 - Ex - N;
    s.Sd = 62 - Ed - N;
    return s;
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}
__device__ __forceinline__ long long block_sum_ll(long long v, long long* s_red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum_ll(v);
    __syncthreads();
    if (lane == 0) s_red[wid] = v;
    __syncthreads();
    long long t = lane < KM_WARPS ? s_red[lane] : 0;
    return warp_sum_ll(t);
}
__device__ __forceinline__ int block_sum_i(int v, int* s_red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum_i(v);
    __syncthreads();
    if (lane == 0) s_red[wid] = v;
    __syncthreads();
    int t = lane < KM_WARPS ? s_red[lane] : 0;
    return warp_sum_i(t);
}
// inclusive block scan of one int64 per thread
__device__ __forceinline__ long long block_scan_ll(long long v, long long* s_red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const long long u = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += u;
    }
    __syncthreads();
    if (lane == 31) s_red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        long long t = lane < KM_WARPS ? s_red[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const long long u = __shfl_up_sync(0xffffffffu, t, off);
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

__device__ __forceinline__ int lowest_unchosen(const int* chosen, int r) {
    int cand = 0;
    for (;; ++cand) {
        bool taken = false;
        for (int q = 0; q < r; ++q)
            if (chosen[q] == cand) { taken = true; break; }
        if (!taken) return cand;
    }
}

// Per-thread accumulation: two register slots (cluster id, exact coordinate sums, count) absorb
// runs of one label and alternation between two labels; a third label evicts the older slot
// into the warp's private shared table (no contention between warps).  At the end of the
// phase a slot that every lane of the warp holds for the same cluster is reduced in registers.
template <int LP>
struct Slot {
    int j;
    long long cnt;
    long long s[LP];
};

// A slot may hold signed contributions (a point leaving a cluster subtracts its coordinates), so
// a zero count does not mean zero sums: only an unused slot (j < 0) is skipped.
template <int LP>
__device__ __forceinline__ void slot_flush(const Slot<LP>& sl, unsigned long long* tab) {
    if (sl.j < 0) return;
    unsigned long long* row = tab + (size_t)sl.j * (LP + 1);
#pragma unroll
    for (int c = 0; c < LP; ++c) atomicAdd(row + c, (unsigned long long)sl.s[c]);
    atomicAdd(row + LP, (unsigned long long)sl.cnt);
}

// Adds sign * q (a point's exact coordinates) and sign to cluster lab through the two-slot run
// cache in front of the warp's shared table (slot 0 holds the most recent label).
template <int LP>
__device__ __forceinline__ void slot_add(Slot<LP> (&sl)[2], int lab, const long long (&q)[LP], bool minus,
                                         unsigned long long* tab) {
    if (sl[0].j != lab) {
        if (sl[1].j == lab) {
            const Slot<LP> t = sl[0];
            sl[0] = sl[1];
            sl[1] = t;
        } else {
            slot_flush<LP>(sl[1], tab);   // evict the older run
            sl[1] = sl[0];
            sl[0].j = lab;
            sl[0].cnt = 0;
#pragma unroll
            for (int c = 0; c < LP; ++c) sl[0].s[c] = 0;
        }
    }
#pragma unroll
    for (int c = 0; c < LP; ++c) sl[0].s[c] += minus ? -q[c] : q[c];
    sl[0].cnt += minus ? -1 : 1;
}

// Adds exact coordinates q (a point's, or the sum of a lane's points) and a count cnt to row `key`
// of the warp's table, for all 32 lanes at once (key < 0: nothing).  Lanes holding the same key
// form a group (match.any).  With few groups (vertex orders that keep clusters together give one
// to three), each 64-bit value is split into limbs of 21, 21 and 22 bits (two unsigned, the top one
// signed), whose sums over at most 32 lanes fit 32 bits and are formed by one warp reduction
// (redux.sync) per limb; the group's lowest lane recombines them, exactly (the values are sums of
// distinct points, and a sum of at most n fixed-point terms fits 62 bits), and adds them to the
// table.  A reduction over a lane subset runs once per group, so with many groups (points in random
// order: ~27 labels among 32 lanes at k = 100) each lane adds its own value with shared atomics
// instead (measured on 2^22 points, k = 100: 0.15 ms for the pass either way, against 2.0 ms for
// the reductions in random order).  Integer sums: both routes give the same table.
constexpr int KM_GROUPED_MAX = 3;
template <int LP>
__device__ __forceinline__ void table_add_grouped(int key, const long long (&q)[LP], int cnt, unsigned long long* tab) {
    const int lane = threadIdx.x & 31;
    const unsigned grp = __match_any_sync(0xffffffffu, key);
    const bool first = lane == __ffs(grp) - 1;
    const bool lead = key >= 0 && first;
    unsigned long long* row = tab + (size_t)(key < 0 ? 0 : key) * (LP + 1);
    if (__popc(__ballot_sync(0xffffffffu, first)) > KM_GROUPED_MAX) {
        if (key >= 0) {
#pragma unroll
            for (int c = 0; c < LP; ++c) atomicAdd(row + c, (unsigned long long)q[c]);
            atomicAdd(row + LP, (unsigned long long)cnt);
        }
        return;
    }
#pragma unroll
    for (int c = 0; c < LP; ++c) {
        const long long v = key >= 0 ? q[c] : 0;
        const unsigned long long u = (unsigned long long)v;
        const unsigned lo = __reduce_add_sync(grp, (unsigned)(u & 0x1fffffu));
        const unsigned mid = __reduce_add_sync(grp, (unsigned)((u >> 21) & 0x1fffffu));
        const int hi = __reduce_add_sync(grp, (int)(v >> 42));
        if (lead) {
            const unsigned long long t = ((unsigned long long)(long long)hi << 42) + ((unsigned long long)mid << 21) +
                                         (unsigned long long)lo;
            atomicAdd(row + c, t);
        }
    }
    if (lead) atomicAdd(row + LP, (unsigned long long)cnt * __popc(grp));
}

template <int LP>
__device__ __forceinline__ void slot_flush_warp(const Slot<LP>& sl, unsigned long long* tab) {
    // all 32 lanes call this: lanes holding the same label are summed by warp reductions, one
    // label after another, and the label's lowest lane adds the totals (one set of shared
    // atomics per label present instead of one per lane)
    const int lane = threadIdx.x & 31;
    unsigned pending = __ballot_sync(0xffffffffu, sl.j >= 0);
    while (pending) {
        const int src = __ffs(pending) - 1;
        const int jj = __shfl_sync(0xffffffffu, sl.j, src);
        const bool mine = ((pending >> lane) & 1u) && sl.j == jj;
        const unsigned members = __ballot_sync(0xffffffffu, mine);
        unsigned long long* row = tab + (size_t)jj * (LP + 1);
#pragma unroll
        for (int c = 0; c < LP; ++c) {
            const long long v = warp_sum_ll(mine ? sl.s[c] : 0ll);
            if (lane == src) atomicAdd(row + c, (unsigned long long)v);
        }
        const long long cn = warp_sum_ll(mine ? sl.cnt : 0ll);
        if (lane == src) atomicAdd(row + LP, (unsigned long long)cn);
        pending &= ~members;
    }
}

}  // namespace fsc
