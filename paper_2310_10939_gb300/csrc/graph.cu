// Graph ingest: validation and degrees d(v) = sum_{u != v} w(u, v) (Sec. 2), plus host utilities.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include <cuda.h>   // driver types only: the two driver calls below are fetched through the runtime

#include "fsc_internal.cuh"

namespace fsc {

// The unique id of the calling thread's current CUDA context (0 if it cannot be had).  The
// library's per-device caches (memory pool, status word, launch attributes) belong to one context
// and are rebuilt when the id changes, e.g. after cudaDeviceReset replaced the primary context:
// their old handles and addresses are dropped, never used.
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    });
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS || !c) {
        cudaFree(nullptr);   // makes the device's primary context current (no allocation)
        if (get_current(&c) != CUDA_SUCCESS || !c) return 0;
    }
    unsigned long long id = 0;
    return get_id(c, &id) == CUDA_SUCCESS ? id : 0;
}

// long rows (longrows.cu)
cudaError_t launch_long_rows(int64_t n, const int64_t* rp, int64_t cap, unsigned long long* count, int64_t* rows,
                             cudaStream_t s);
fsc_status build_long_rows(fsc_graph* g, int64_t count, const int64_t* d_rows, cudaStream_t s);

namespace {
constexpr int kMaxDevices = 64;
DeviceProps g_props[kMaxDevices];
int* g_status_word[kMaxDevices];
unsigned long long g_status_ctx[kMaxDevices];
std::once_flag g_props_once[kMaxDevices];
std::mutex g_status_mu;
std::atomic<long long> g_wait_limit{2000000000LL};
std::atomic<int> g_stall{0};
}  // namespace

const DeviceProps& device_props() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= kMaxDevices) dev = 0;
    std::call_once(g_props_once[dev], [dev] {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g_props[dev] = DeviceProps{dev, sms > 0 ? sms : 1};
    });
    return g_props[dev];
}

int* device_status_word() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_status_mu);
    bool stale = g_status_ctx[dev] != ctx;   // one of a former context
    if (g_status_word[dev] && !stale && ctx == 0) {
        // no context id to compare: check that the address still names device memory
        cudaPointerAttributes pa{};
        stale = cudaPointerGetAttributes(&pa, g_status_word[dev]) != cudaSuccess || pa.type != cudaMemoryTypeDevice;
        cudaGetLastError();
    }
    if (!g_status_word[dev] || stale) {
        int* p = nullptr;
        if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return nullptr;
        g_status_word[dev] = p;
        g_status_ctx[dev] = ctx;
    }
    return g_status_word[dev];
}

namespace {
cudaMemPool_t g_pool[kMaxDevices];
unsigned long long g_pool_ctx[kMaxDevices];
std::mutex g_pool_mu;
std::mutex g_occ_mu;
// keyed by context id as well: a kernel's dynamic shared-memory opt-in is per context
std::map<std::tuple<unsigned long long, int, const void*, int, size_t>, int> g_occ;
std::map<std::tuple<unsigned long long, int, const void*>, size_t> g_smem_attr;
}  // namespace

static cudaMemPool_t library_pool(int dev) {
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_pool_mu);
    bool stale = g_pool_ctx[dev] != ctx;   // one of a former context
    if (g_pool[dev] && !stale && ctx == 0) {
        // no context id to compare: check that the pool still answers
        unsigned long long v = 0;
        stale = cudaMemPoolGetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &v) != cudaSuccess;
        cudaGetLastError();
    }
    if (!g_pool[dev] || stale) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = p;
        g_pool_ctx[dev] = ctx;
    }
    return g_pool[dev];
}

cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaMemPool_t pool = library_pool(dev);
    if (!pool) return cudaErrorMemoryAllocation;
    return cudaMallocFromPoolAsync(p, bytes < 256 ? 256 : bytes, pool, s);
}

cudaError_t pool_free(void* p, cudaStream_t s) { return p ? cudaFreeAsync(p, s) : cudaSuccess; }

int kernel_occupancy(const void* fn, int threads, size_t smem) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    const unsigned long long ctx = current_context_id();
    std::lock_guard<std::mutex> lock(g_occ_mu);
    const auto key = std::make_tuple(ctx, dev, fn, threads, smem);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) return it->second;
    // the opt-in limit covers dynamic bytes on top of the kernel's static shared memory, so it is
    // raised for every size above the largest one set so far
    size_t& attr = g_smem_attr[std::make_tuple(ctx, dev, fn)];
    if (smem > attr) {
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
        attr = smem;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess) return 0;
    g_occ[key] = per_sm;
    return per_sm;
}

long long wait_limit_ns() { return g_wait_limit.load(); }
int barrier_stall() { return g_stall.load(); }

fsc_status cuda_status(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) return FSC_ERR_OOM;
    return FSC_ERR_CUDA;
}

fsc_status status_from_bits(int bits) {
    if (bits == 0) return FSC_OK;
    if (bits & (ST_INDEX_RANGE | ST_BAD_ROWPTR)) return FSC_ERR_INDEX_RANGE;
    if (bits & ST_SELF_LOOP) return FSC_ERR_SELF_LOOP;
    if (bits & ST_BAD_WEIGHT) return FSC_ERR_BAD_WEIGHT;
    if (bits & ST_UNSORTED) return FSC_ERR_UNSORTED;
    if (bits & ST_NOT_SYMMETRIC) return FSC_ERR_NOT_SYMMETRIC;
    if (bits & ST_TIMEOUT) return FSC_ERR_TIMEOUT;
    return FSC_ERR_CUDA;
}

// float64 value of an integer below 2^53, built with integer operations only (the float64 pipe
// is a small fraction of the integer one on this GPU).
__device__ __forceinline__ double exact_u64_to_f64(unsigned long long c) {
    if (c == 0) return 0.0;
    const int e = 63 - __clzll((long long)c);
    const unsigned long long mant = (c << (52 - e)) & ((1ull << 52) - 1);
    return __longlong_as_double((long long)((((unsigned long long)(1023 + e)) << 52) | mant));
}

// Per-thread degree statistics to the graph header: warp shuffles, then the block's warps through
// shared memory, then one atomic per block and statistic (per-warp atomics on five single
// addresses serialised at L2 and dominated the kernel).  Blocks of 256 threads.
__device__ __forceinline__ void degree_block_totals(int bad, unsigned iso, double vol_part, double vsq,
                                                    double vmax, unsigned long long* n_iso, double* vol,
                                                    int* status, double* sumsq,
                                                    unsigned long long* dmax_bits) {
    const int lane = threadIdx.x & 31;
    for (int off = 16; off > 0; off >>= 1) {
        bad |= __shfl_xor_sync(0xffffffffu, bad, off);
        iso += __shfl_xor_sync(0xffffffffu, iso, off);
        vol_part += __shfl_xor_sync(0xffffffffu, vol_part, off);
        vsq += __shfl_xor_sync(0xffffffffu, vsq, off);
        vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
    }
    __shared__ double s_sq[8], s_mx[8], s_vol[8];
    __shared__ int s_bad[8];
    __shared__ unsigned s_iso[8];
    const int wid = threadIdx.x >> 5;
    if (lane == 0) {
        s_sq[wid] = vsq;
        s_mx[wid] = vmax;
        s_vol[wid] = vol_part;
        s_bad[wid] = bad;
        s_iso[wid] = iso;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tsq = 0.0, tmx = 0.0, tvol = 0.0;
        int tbad = 0;
        unsigned tiso = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            tsq += s_sq[q];
            tmx = fmax(tmx, s_mx[q]);
            tvol += s_vol[q];
            tbad |= s_bad[q];
            tiso += s_iso[q];
        }
        if (tsq != 0.0) atomicAdd(sumsq, tsq);
        if (tmx > 0.0) atomicMax(dmax_bits, (unsigned long long)__double_as_longlong(tmx));
        if (tbad) atomicOr(status, tbad);
        if (tiso) atomicAdd(n_iso, (unsigned long long)tiso);
        if (tvol != 0.0) atomicAdd(vol, tvol);
    }
}

// Unit weights: d(v) is the row length, so the degrees come from row_ptr alone and col is read
// only to validate it.  A block takes a tile of `rows` consecutive rows (dynamic shared memory
// holds the tile's rows + 1 row_ptr values): one thread per row writes the degrees (coalesced),
// then the block streams the tile's entries as one flat range of VEC-entry vectors, kDegUnroll
// independent loads in flight per thread.  No entry needs its own row: a self-loop (i, i) has i
// in the tile, and then the entry's position lies in row i's range, two shared-memory reads
// away.  Only the optional sortedness check looks a row up (a binary search in the shared
// row_ptr), and only at an inversion col[p-1] >= col[p], which is a row start or an unsorted
// row.  The tile size is chosen so the grid is about one wave of resident blocks; HBM traffic
// is row_ptr, col and the three n-vectors once.
constexpr int kDegUnroll = 4;
// k_degree_unit with a 16-byte aligned col streams the tile's entries through a ring of kDegRingS
// stages in shared memory, each stage kDegRingU vectors per thread, filled by asynchronous copies
// (cp.async, every thread copying and later reading only its own slots): kDegRingS - 1 stages are in
// flight while one is checked, without holding them in registers.
constexpr int kDegThreads = 256, kDegRingS = 4, kDegRingU = 2;
constexpr size_t kDegRingBytes = (size_t)kDegRingS * kDegRingU * kDegThreads * 16;
// dynamic shared memory of k_degree_unit: the tile's row_ptr (int64, 16-byte padded; in the lean
// scan below it is rewritten in place as each row's entry range relative to the tile's first entry,
// int32 pairs), then the ring
constexpr int kDegMaxRows = 2048;   // rows per tile at most (kDegMaxRows / kDegThreads per thread)
__host__ __device__ inline size_t deg_unit_smem(int rows) {
    return (((size_t)rows + 1) * 8 + 15) / 16 * 16 + kDegRingBytes;
}

template <int VEC>
__device__ __forceinline__ void load_entries(const int32_t* __restrict__ col, long long v, long long nnz,
                                             int32_t (&x)[VEC]) {
    const long long base = v * VEC;
    if (VEC == 4 && base + 3 < nnz) {
        const int4 t = __ldg(reinterpret_cast<const int4*>(col) + v);
        x[0] = t.x;
        x[VEC > 1 ? 1 : 0] = t.y;
        x[VEC > 2 ? 2 : 0] = t.z;
        x[VEC > 3 ? 3 : 0] = t.w;
    } else {
#pragma unroll
        for (int u = 0; u < VEC; ++u) x[u] = base + u < nnz ? __ldg(col + base + u) : 0;
    }
}

template <int VEC>
__global__ void __launch_bounds__(256) k_degree_unit(int64_t n, int64_t nnz, const int64_t* __restrict__ rp,
                                                     const int32_t* __restrict__ col, int rows, int check_sorted,
                                                     double* __restrict__ deg, float* __restrict__ dinv,
                                                     float* __restrict__ invdeg,
                                                     unsigned long long* __restrict__ n_iso,
                                                     double* __restrict__ vol, int* __restrict__ status,
                                                     double* __restrict__ sumsq,
                                                     unsigned long long* __restrict__ dmax_bits) {
    extern __shared__ __align__(16) long long s_rp[];   // rows + 1, then (VEC = 4) the copy ring
    if (blockIdx.x == 0 && threadIdx.x == 0 && (rp[0] != 0 || rp[n] != nnz)) atomicOr(status, ST_BAD_ROWPTR);
    int bad = 0;
    unsigned iso = 0;
    long long cnt_total = 0;
    double vsq = 0.0;
    unsigned long long usq = 0, umax = 0;   // sum of d^2 (below 2^64: it is at most nnz * max d) and max d
    const int64_t ntiles = (n + rows - 1) / rows;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r0 = tile * rows;
        const int nr = (int)(n - r0 < rows ? n - r0 : rows);
        for (int q = threadIdx.x; q <= nr; q += blockDim.x) s_rp[q] = rp[r0 + q];
        __syncthreads();
        int tile_bad = 0;
        for (int q = threadIdx.x; q < nr; q += blockDim.x) {
            const long long s = s_rp[q], e = s_rp[q + 1];
            if (s < 0 || e < s || e > nnz) {
                tile_bad = 1;
                continue;
            }
            const unsigned long long c = (unsigned long long)(e - s);
            const int64_t i = r0 + q;
            deg[i] = exact_u64_to_f64(c);
            cnt_total += (long long)c;
            if (c < (1ull << 26)) usq += c * c;
            else vsq += (double)c * (double)c;
            umax = umax > c ? umax : c;
            if (c) {
                const float df = (float)c;
                dinv[i] = 1.0f / sqrtf(df);
                invdeg[i] = 1.0f / df;
            } else {
                dinv[i] = 0.0f;
                invdeg[i] = 0.0f;
                ++iso;
            }
        }
        // a tile with a bad row_ptr is not scanned (its rows would not be monotone); the barrier
        // also ends every read of s_rp before the next tile overwrites it
        if (__syncthreads_or(tile_bad)) {
            bad |= ST_BAD_ROWPTR;
            continue;
        }
        const long long P0 = s_rp[0], P1 = s_rp[nr];   // 0 <= P0 <= P1 <= nnz, rows non-decreasing
        const long long v0 = P0 / VEC, v1 = (P1 + VEC - 1) / VEC;
        const int r0i = (int)r0;                        // r0 < n <= 2^31 - 1
        // the checks of one vector of entries (positions base .. base + VEC - 1) of the tile
        auto check = [&](long long base, const int32_t (&x)[VEC]) {
            const bool interior = base >= P0 && base + VEC <= P1;
            if (interior && !check_sorted) {
                // the common case in a few instructions: the largest column (as unsigned, so a
                // negative one is out of range too) against n, and the smallest offset from the
                // tile's first row against the tile; only a vector holding a column of a tile row
                // takes the per-entry self-loop test below
                unsigned mx = (unsigned)x[0], mt = (unsigned)(x[0] - r0i);
#pragma unroll
                for (int u = 1; u < VEC; ++u) {
                    mx = max(mx, (unsigned)x[u]);
                    mt = min(mt, (unsigned)(x[u] - r0i));
                }
                if (mx >= (unsigned long long)n) bad |= ST_INDEX_RANGE;
                if (mt >= (unsigned)nr) return;
            }
#pragma unroll
            for (int u = 0; u < VEC; ++u) {
                const long long p = base + u;
                if (!interior && (p < P0 || p >= P1)) continue;
                const int j = x[u];
                const int jl = j - r0i;   // j's row within the tile, if it is one
                // a self-loop (i, i) needs i in the tile: then p lies in row i's range
                if ((unsigned)j >= (unsigned)n) bad |= ST_INDEX_RANGE;
                else if ((unsigned)jl < (unsigned)nr && s_rp[jl] <= p && p < s_rp[jl + 1]) bad |= ST_SELF_LOOP;
                if (check_sorted && p > P0) {
                    // an inversion col[p-1] >= col[p] is either a row start or an unsorted row
                    const int prev = u > 0 ? x[u > 0 ? u - 1 : 0] : __ldg(col + p - 1);
                    if (prev >= j) {
                        int lo = 0, hi = nr - 1;   // last row whose start is <= p (s_rp[nr] = P1 > p)
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (s_rp[mid] <= p) lo = mid;
                            else hi = mid - 1;
                        }
                        if (p > s_rp[lo]) bad |= ST_UNSORTED;
                    }
                }
            }
        };
        if constexpr (VEC == 4) {
            int4* ring = reinterpret_cast<int4*>(reinterpret_cast<char*>(s_rp) + deg_unit_smem(rows) - kDegRingBytes);
            // Without the sortedness check, and when the tile's entries fit int32 offsets, a vector's
            // checks run branch-free on every lane (an entry whose column is a tile row is a rare
            // case per lane, but over 32 lanes nearly every warp meets one): the largest column
            // against n, and per entry the own-row range test against the tile's row ranges relative
            // to P0 (s_rng), whose row is the column's only if the column is a tile row.
            int2* s_rng = reinterpret_cast<int2*>(s_rp);   // replaces s_rp (same bytes) in the lean scan
            const bool lean = !check_sorted && P1 - P0 < 0x7ffffff0LL;
            if (lean) {
                constexpr int kPer = kDegMaxRows / kDegThreads;
                int2 rg[kPer];
#pragma unroll
                for (int k = 0; k < kPer; ++k) {
                    const int q = threadIdx.x + k * kDegThreads;
                    if (q < nr) rg[k] = make_int2((int)(s_rp[q] - P0), (int)(s_rp[q + 1] - P0));
                }
                __syncthreads();   // every read of s_rp is done before it is overwritten
#pragma unroll
                for (int k = 0; k < kPer; ++k) {
                    const int q = threadIdx.x + k * kDegThreads;
                    if (q < nr) s_rng[q] = rg[k];
                }
                __syncthreads();
            }
            const int span = (int)(lean ? P1 - P0 : 0);
            auto lean_check = [&](long long base, const int4& t) {
                const int32_t x[4] = {t.x, t.y, t.z, t.w};
                const int pr0 = (int)(base - P0);   // base >= P0 - 3 and base < P1: fits int
                bool range = false, self = false;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int pr = pr0 + u;
                    const bool valid = (unsigned)pr < (unsigned)span;   // the entry belongs to the tile
                    const unsigned jl = (unsigned)(x[u] - r0i);
                    const bool in = jl < (unsigned)nr;
                    const int q = in ? (int)jl : 0;
                    range |= valid && (unsigned)x[u] >= (unsigned long long)n;
                    const int2 rg = s_rng[q];
                    self |= valid && in && rg.x <= pr && pr < rg.y;
                }
                if (range) bad |= ST_INDEX_RANGE;
                if (self) bad |= ST_SELF_LOOP;
            };
            const long long per_stage = (long long)kDegRingU * kDegThreads;
            const long long nstages = (v1 - v0 + per_stage - 1) / per_stage;
            auto issue = [&](long long st) {   // stage st into slot st mod kDegRingS (own slots only)
                if (st < nstages) {
                    const int slot = (int)(st % kDegRingS);
#pragma unroll
                    for (int h = 0; h < kDegRingU; ++h) {
                        const long long vv = v0 + st * per_stage + (long long)h * kDegThreads + threadIdx.x;
                        if (vv < v1) {
                            const long long rem = nnz - vv * 4;   // >= 1: vv < v1 <= ceil(nnz / 4)
                            cp_async16(ring + ((size_t)slot * kDegRingU + h) * kDegThreads + threadIdx.x,
                                       reinterpret_cast<const int4*>(col) + vv, rem >= 4 ? 16 : (int)rem * 4);
                        }
                    }
                }
                cp_async_commit();   // every thread commits one group per stage, empty or not
            };
#pragma unroll
            for (int st = 0; st < kDegRingS - 1; ++st) issue(st);
            for (long long st = 0; st < nstages; ++st) {
                cp_async_wait<kDegRingS - 2>();   // this thread's copies of stage st have landed
                issue(st + kDegRingS - 1);          // into the slot of stage st - 1, already checked
                const int slot = (int)(st % kDegRingS);
#pragma unroll
                for (int h = 0; h < kDegRingU; ++h) {
                    const long long vv = v0 + st * per_stage + (long long)h * kDegThreads + threadIdx.x;
                    if (vv < v1) {
                        const int4 t = ring[((size_t)slot * kDegRingU + h) * kDegThreads + threadIdx.x];
                        if (lean) {
                            lean_check(vv * VEC, t);
                        } else {
                            const int32_t x[VEC] = {t.x, t.y, t.z, t.w};
                            check(vv * VEC, x);
                        }
                    }
                }
            }
            cp_async_wait<0>();
            __syncthreads();
            continue;
        }
        for (long long v = v0 + threadIdx.x; v < v1; v += (long long)kDegUnroll * blockDim.x) {
            int32_t x[kDegUnroll][VEC];
#pragma unroll
            for (int h = 0; h < kDegUnroll; ++h) {
                const long long vv = v + (long long)h * blockDim.x;
                if (vv < v1) load_entries<VEC>(col, vv, nnz, x[h]);
            }
#pragma unroll
            for (int h = 0; h < kDegUnroll; ++h) {
                const long long vv = v + (long long)h * blockDim.x;
                if (vv < v1) check(vv * VEC, x[h]);
            }
        }
        __syncthreads();
    }
    degree_block_totals(bad, iso, (double)cnt_total, vsq + (double)usq, (double)umax, n_iso, vol, status,
                        sumsq, dmax_bits);
}

// Weighted graphs: the same tiles as k_degree_unit.  The flat scan over the tile's entries
// validates col and w and stages the weights in shared memory (coalesced loads, kDegUnroll in
// flight per thread); then one thread per row sums its row's weights in float64 in entry order
// (deterministic; the same order as a sequential sum).  A tile with more than `cap` entries (a
// few very long rows) sums from global memory instead.
template <int U>
__global__ void __launch_bounds__(256) k_degree_weighted(int64_t n, int64_t nnz, const int64_t* __restrict__ rp,
                                                         const int32_t* __restrict__ col, const float* __restrict__ w,
                                                         int rows, int cap, int check_sorted, double* __restrict__ deg,
                                                         float* __restrict__ dinv, float* __restrict__ invdeg,
                                                         unsigned long long* __restrict__ n_iso,
                                                         double* __restrict__ vol, int* __restrict__ status,
                                                         double* __restrict__ sumsq,
                                                         unsigned long long* __restrict__ dmax_bits) {
    extern __shared__ long long s_rpw[];   // rows + 1 row_ptr values, then cap weights
    long long* s_rp = s_rpw;
    float* s_w = reinterpret_cast<float*>(s_rpw + rows + 1);
    if (blockIdx.x == 0 && threadIdx.x == 0 && (rp[0] != 0 || rp[n] != nnz)) atomicOr(status, ST_BAD_ROWPTR);
    int bad = 0;
    unsigned iso = 0;
    double vsum = 0.0, vsq = 0.0, vmax = 0.0;
    const int64_t ntiles = (n + rows - 1) / rows;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r0 = tile * rows;
        const int nr = (int)(n - r0 < rows ? n - r0 : rows);
        for (int q = threadIdx.x; q <= nr; q += blockDim.x) s_rp[q] = rp[r0 + q];
        __syncthreads();
        int tile_bad = 0;
        for (int q = threadIdx.x; q < nr; q += blockDim.x) {
            const long long s = s_rp[q], e = s_rp[q + 1];
            if (s < 0 || e < s || e > nnz) tile_bad = 1;
        }
        if (__syncthreads_or(tile_bad)) {
            bad |= ST_BAD_ROWPTR;
            continue;
        }
        const long long P0 = s_rp[0], P1 = s_rp[nr];   // 0 <= P0 <= P1 <= nnz, rows non-decreasing
        const bool staged = P1 - P0 <= (long long)cap;
        const int r0i = (int)r0;
        for (long long p0 = P0 + threadIdx.x; p0 < P1; p0 += (long long)U * blockDim.x) {
            int jv[U];
            float wv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long p = p0 + (long long)u * blockDim.x;
                jv[u] = p < P1 ? __ldg(col + p) : 0;
                wv[u] = p < P1 ? __ldg(w + p) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long p = p0 + (long long)u * blockDim.x;
                if (p >= P1) break;
                const int j = jv[u];
                const int jl = j - r0i;
                if ((unsigned)j >= (unsigned)n) bad |= ST_INDEX_RANGE;
                else if ((unsigned)jl < (unsigned)nr && s_rp[jl] <= p && p < s_rp[jl + 1]) bad |= ST_SELF_LOOP;
                if (!(wv[u] >= 0.0f) || isinf(wv[u])) bad |= ST_BAD_WEIGHT;
                if (staged) s_w[p - P0] = wv[u];
                if (check_sorted && p > P0 && __ldg(col + p - 1) >= j) {
                    int lo = 0, hi = nr - 1;   // last row whose start is <= p
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (s_rp[mid] <= p) lo = mid;
                        else hi = mid - 1;
                    }
                    if (p > s_rp[lo]) bad |= ST_UNSORTED;
                }
            }
        }
        __syncthreads();
        for (int q = threadIdx.x; q < nr; q += blockDim.x) {
            const long long s = s_rp[q], e = s_rp[q + 1];
            double d = 0.0;
            if (staged)
                for (long long p = s; p < e; ++p) d += (double)s_w[p - P0];
            else
                for (long long p = s; p < e; ++p) d += (double)__ldg(w + p);
            const int64_t i = r0 + q;
            deg[i] = d;
            vsum += d;
            vsq += d * d;
            vmax = fmax(vmax, d);
            if (d > 0.0) {
                const float df = (float)d;
                dinv[i] = 1.0f / sqrtf(df);
                invdeg[i] = 1.0f / df;
            } else {
                dinv[i] = 0.0f;
                invdeg[i] = 0.0f;
                ++iso;
            }
        }
        __syncthreads();
    }
    degree_block_totals(bad, iso, vsum, vsq, vmax, n_iso, vol, status, sumsq, dmax_bits);
}

// One warp per row: each entry (i, j, w) must have its mirror (j, i, w) (binary search, sorted rows).
__global__ void __launch_bounds__(256) k_symmetry(int64_t n, const int64_t* __restrict__ rp,
                                                  const int32_t* __restrict__ col, const float* __restrict__ w,
                                                  int* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < n; i += nwarps) {
        for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) {
            const int j = col[p];
            int64_t lo = rp[j], hi = rp[j + 1];
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (col[mid] < (int)i) lo = mid + 1; else hi = mid;
            }
            const bool found = lo < rp[j + 1] && col[lo] == (int)i &&
                               (w == nullptr || __float_as_uint(w[lo]) == __float_as_uint(w[p]));
            if (!found) atomicOr(status, ST_NOT_SYMMETRIC);
        }
    }
}

}  // namespace fsc

using namespace fsc;

extern "C" fsc_status fsc_create_graph(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                                       const float* w, uint32_t flags, void* stream, fsc_graph** out) {
    if (!out || n < 1 || n > 2147483647LL || nnz < 0 || !row_ptr || (nnz > 0 && !col_idx))
        return FSC_ERR_INVALID_ARG;
    if (flags & ~(FSC_VALIDATE_SYMMETRY | FSC_COPY)) return FSC_ERR_INVALID_ARG;
    NvtxRange nvtx_range("fsc_create_graph");
    cudaStream_t s = as_stream(stream);
    int dev = 0;
    FSC_CUDA(cudaGetDevice(&dev));
    fsc_graph* g = new (std::nothrow) fsc_graph();
    if (!g) return FSC_ERR_OOM;
    memset(g, 0, sizeof(*g));
    g->max_row = 0x7fffffffffffffffLL;
    g->device = dev;
    g->n = n;
    g->nnz = nnz;
    g->row_ptr = row_ptr;
    g->col = col_idx;
    g->w = w;
    if (flags & FSC_COPY) {   // the graph's own CSR: row_ptr | col | w, each 256-byte aligned
        const size_t brp = ((size_t)(n + 1) * 8 + 255) & ~(size_t)255, bcol = ((size_t)nnz * 4 + 255) & ~(size_t)255;
        const size_t bw = w ? (size_t)nnz * 4 : 0;
        char* cb = nullptr;
        cudaError_t ce = pool_malloc(reinterpret_cast<void**>(&cb), brp + bcol + bw + 256, s);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(cb, row_ptr, (size_t)(n + 1) * 8, cudaMemcpyDeviceToDevice, s);
        if (ce == cudaSuccess && nnz > 0)
            ce = cudaMemcpyAsync(cb + brp, col_idx, (size_t)nnz * 4, cudaMemcpyDeviceToDevice, s);
        if (ce == cudaSuccess && w && nnz > 0)
            ce = cudaMemcpyAsync(cb + brp + bcol, w, (size_t)nnz * 4, cudaMemcpyDeviceToDevice, s);
        if (ce != cudaSuccess) {
            if (cb) pool_free(cb, s);
            delete g;
            return cuda_status(ce);
        }
        g->copy_base = cb;
        g->row_ptr = reinterpret_cast<const int64_t*>(cb);
        g->col = reinterpret_cast<const int32_t*>(cb + brp);
        g->w = w ? reinterpret_cast<const float*>(cb + brp + bcol) : nullptr;
        row_ptr = g->row_ptr;
        col_idx = g->col;
        w = g->w;
    }
    // one allocation: deg (n doubles) | header (256 B: volume, n_iso, status, sumsq, max bits,
    //                 long-row count) | dinv (n floats) | invdeg (n floats) | colmax 24 u32 | expo 8 int |
    //                 long-row triples (at most nnz / kLongRow rows can be longer than kLongRow)
    const size_t n8 = (size_t)n * 8, n4 = ((size_t)n * 4 + 255) & ~(size_t)255;
    const int64_t lcap = nnz / kLongRow + 1;
    const size_t bytes = n8 + 256 + 2 * n4 + 256 + (size_t)lcap * 24;
    char* base = nullptr;
    cudaError_t e = pool_malloc(reinterpret_cast<void**>(&base), bytes, s);
    if (e != cudaSuccess) {
        if (g->copy_base) pool_free(g->copy_base, s);
        cudaStreamSynchronize(s);
        delete g;
        return cuda_status(e);
    }
    struct Header {           // device layout of the 256-byte header
        double vol;
        unsigned long long niso;
        int status, pad;
        double pad2;
        double sumsq;
        unsigned long long dmax_bits;
        unsigned long long nlong;
    };
    Header* hdr = reinterpret_cast<Header*>(base + n8);
    g->deg = reinterpret_cast<double*>(base);
    g->dinv = reinterpret_cast<float*>(base + n8 + 256);
    g->invdeg = reinterpret_cast<float*>(base + n8 + 256 + n4);
    g->colmax = reinterpret_cast<unsigned*>(base + n8 + 256 + 2 * n4);
    g->expo = reinterpret_cast<int*>(base + n8 + 256 + 2 * n4 + 128);
    int64_t* long_list = reinterpret_cast<int64_t*>(base + n8 + 256 + 2 * n4 + 256);
    fsc_status rc = FSC_OK;
    do {
        if ((e = cudaMemsetAsync(base + n8, 0, 256, s)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(base + n8 + 256 + 2 * n4, 0, 256, s)) != cudaSuccess) break;
        const int threads = kDegThreads;   // the copy ring of k_degree_unit is sized for it
        const int check_sorted = (flags & FSC_VALIDATE_SYMMETRY) ? 1 : 0;
        if (w == nullptr) {
            // tiles of 64 .. 2048 rows, sized so the grid is about one wave of resident blocks
            const bool vec4 = (reinterpret_cast<uintptr_t>(col_idx) & 15) == 0;
            const void* fn = vec4 ? (const void*)k_degree_unit<4> : (const void*)k_degree_unit<1>;
            constexpr int64_t kMaxRows = kDegMaxRows, kMinRows = 64;
            int per_sm = kernel_occupancy(fn, threads, deg_unit_smem((int)kMaxRows));
            if (per_sm < 1) per_sm = 1;
            const int64_t slots = (int64_t)device_props().num_sms * per_sm;
            int64_t rows = ((n + slots - 1) / slots + 31) / 32 * 32;
            rows = rows < kMinRows ? kMinRows : (rows > kMaxRows ? kMaxRows : rows);
            const int64_t ntiles = (n + rows - 1) / rows;
            const int blocks = (int)(ntiles < slots ? ntiles : slots);
            const size_t smem = deg_unit_smem((int)rows);
            if (vec4)
                k_degree_unit<4><<<blocks, threads, smem, s>>>(n, nnz, row_ptr, col_idx, (int)rows, check_sorted,
                                                               g->deg, g->dinv, g->invdeg, &hdr->niso, &hdr->vol,
                                                               &hdr->status, &hdr->sumsq, &hdr->dmax_bits);
            else
                k_degree_unit<1><<<blocks, threads, smem, s>>>(n, nnz, row_ptr, col_idx, (int)rows, check_sorted,
                                                               g->deg, g->dinv, g->invdeg, &hdr->niso, &hdr->vol,
                                                               &hdr->status, &hdr->sumsq, &hdr->dmax_bits);
        } else {
            // tiles sized so that the staged weights of an average tile fill at most half of the
            // 32 KB weight buffer, and the grid is about one wave of resident blocks
            constexpr int kCap = 8192;
            constexpr int64_t kMaxRows = 2048, kMinRows = 32;
            const void* fn = (const void*)k_degree_weighted<4>;
            int per_sm = kernel_occupancy(fn, threads, (size_t)(kMaxRows + 1) * 8 + (size_t)kCap * 4);
            if (per_sm < 1) per_sm = 1;
            const int64_t slots = (int64_t)device_props().num_sms * per_sm;
            const double avg = n > 0 ? (double)nnz / (double)n : 0.0;
            int64_t rows = ((n + slots - 1) / slots + 31) / 32 * 32;
            const int64_t by_cap = avg > 0.0 ? (int64_t)((kCap / 2) / avg) / 32 * 32 : kMaxRows;
            if (rows > by_cap) rows = by_cap;
            rows = rows < kMinRows ? kMinRows : (rows > kMaxRows ? kMaxRows : rows);
            const int64_t ntiles = (n + rows - 1) / rows;
            const int blocks = (int)(ntiles < slots ? ntiles : slots);
            const size_t smem = (size_t)(rows + 1) * 8 + (size_t)kCap * 4;
            k_degree_weighted<4><<<blocks, threads, smem, s>>>(n, nnz, row_ptr, col_idx, w, (int)rows, kCap, check_sorted,
                                                               g->deg, g->dinv, g->invdeg, &hdr->niso, &hdr->vol,
                                                               &hdr->status, &hdr->sumsq, &hdr->dmax_bits);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = launch_long_rows(n, row_ptr, lcap, &hdr->nlong, long_list, s)) != cudaSuccess) break;
        Header h{};
        if ((e = cudaMemcpyAsync(&h, hdr, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
        int bits = h.status;
        if (bits == 0 && check_sorted) {
            const int64_t want = (n + threads / 32 - 1) / (threads / 32), cap = (int64_t)device_props().num_sms * 32;
            k_symmetry<<<(int)(want < cap ? want : cap), threads, 0, s>>>(n, row_ptr, col_idx, w, &hdr->status);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            if ((e = cudaMemcpyAsync(&bits, &hdr->status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
        }
        if (bits) { rc = status_from_bits(bits); break; }
        const int64_t nlong = (int64_t)h.nlong < lcap ? (int64_t)h.nlong : lcap;
        if (nlong > 0 && (rc = build_long_rows(g, nlong, long_list, s)) != FSC_OK) break;
        g->n_isolated = (int64_t)h.niso;
        g->volume = h.vol;
        g->deg_sumsq = h.sumsq;
        memcpy(&g->deg_max, &h.dmax_bits, 8);
    } while (0);
    if (e != cudaSuccess) rc = cuda_status(e);
    if (rc != FSC_OK) {
        pool_free(base, s);
        if (g->long_base) pool_free(g->long_base, s);
        if (g->copy_base) pool_free(g->copy_base, s);
        cudaStreamSynchronize(s);
        delete g;
        return rc;
    }
    *out = g;
    return FSC_OK;
}

extern "C" fsc_status fsc_destroy_graph(fsc_graph* g) {
    NvtxRange nvtx_range("fsc_destroy_graph");
    if (!g) return FSC_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(g->device);
    // all work that may still read the graph's buffers ends here; the blocks go back to the
    // library pool (no unmapping), ordered on the legacy stream after that point
    cudaError_t e = cudaDeviceSynchronize();
    pool_free(g->ws, 0);
    pool_free(g->deg, 0);
    if (g->long_base) pool_free(g->long_base, 0);
    if (g->copy_base) pool_free(g->copy_base, 0);
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    if (g->ev_join) cudaEventDestroy(g->ev_join);
    if (g->side) cudaStreamDestroy(g->side);
    cudaSetDevice(prev);
    delete g;
    return e == cudaSuccess ? FSC_OK : cuda_status(e);
}

extern "C" fsc_status fsc_release_cached_memory(void) {
    int prev = 0;
    cudaGetDevice(&prev);
    std::lock_guard<std::mutex> lock(g_pool_mu);
    cudaError_t first = cudaSuccess;
    for (int d = 0; d < kMaxDevices; ++d) {
        if (!g_pool[d]) continue;
        cudaSetDevice(d);
        if (g_pool_ctx[d] != current_context_id()) continue;   // a former context's pool is gone
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemPoolTrimTo(g_pool[d], 0);
        if (first == cudaSuccess) first = e;
    }
    cudaSetDevice(prev);
    return first == cudaSuccess ? FSC_OK : cuda_status(first);
}

extern "C" fsc_status fsc_graph_info(const fsc_graph* g, fsc_graph_info_t* info) {
    if (!g || !info) return FSC_ERR_INVALID_ARG;
    info->n = g->n;
    info->nnz = g->nnz;
    info->n_isolated = g->n_isolated;
    info->weighted = g->w != nullptr;
    info->volume = g->volume;
    info->deg_sumsq = g->deg_sumsq;
    info->deg_max = g->deg_max;
    info->deg = g->deg;
    info->dinv = g->dinv;
    info->invdeg = g->invdeg;
    return FSC_OK;
}

extern "C" int fsc_pad_l(int l) { return pad_l(l); }

#ifdef FSC_BOUNDS_CHECK
namespace fsc {
cudaError_t bounds_read_spmm_f32(BoundsRecord*, bool);
cudaError_t bounds_read_spmm_bf16(BoundsRecord*, bool);
cudaError_t bounds_read_filter(BoundsRecord*, bool);
cudaError_t bounds_read_batch_f32(BoundsRecord*, bool);
cudaError_t bounds_read_batch_bf16(BoundsRecord*, bool);
cudaError_t bounds_read_kmeans(BoundsRecord*, bool);
cudaError_t bounds_read_kmeans_wide(BoundsRecord*, bool);
cudaError_t bounds_read_wide(BoundsRecord*, bool);
}  // namespace fsc
#endif

extern "C" fsc_status fsc_bounds_report(int32_t* site, int64_t* index, int64_t* lo, int64_t* hi, int clear) {
    if (!site) return FSC_ERR_INVALID_ARG;
#ifdef FSC_BOUNDS_CHECK
    cudaError_t (*readers[])(BoundsRecord*, bool) = {bounds_read_spmm_f32, bounds_read_spmm_bf16, bounds_read_filter,
                                                     bounds_read_batch_f32, bounds_read_batch_bf16, bounds_read_kmeans,
                                                     bounds_read_kmeans_wide, bounds_read_wide};
    *site = 0;
    for (auto rd : readers) {
        BoundsRecord r{};
        const cudaError_t e = rd(&r, clear != 0);
        if (e != cudaSuccess) return cuda_status(e);
        if (r.site && *site == 0) {
            *site = r.site;
            if (index) *index = r.index;
            if (lo) *lo = r.lo;
            if (hi) *hi = r.hi;
        }
    }
    return FSC_OK;
#else
    (void)index;
    (void)lo;
    (void)hi;
    (void)clear;
    *site = -1;   // built without bounds checks
    return FSC_OK;
#endif
}

extern "C" fsc_status fsc_default_params(int64_t n, int k, int mode, int* l, int* t) {
    if (!l || !t || n < 1 || k < 1 || k > n || (mode != 0 && mode != 1)) return FSC_ERR_INVALID_ARG;
    if (mode == 0) {
        int lv = 0;
        while ((1LL << lv) < k) ++lv;
        int tv = 0;
        while ((1LL << tv) < n) ++tv;
        *l = lv < 1 ? 1 : lv;
        *t = tv;
    } else {
        const double lk = k > 1 ? ceil(log((double)k)) : 1.0;
        *l = lk < 1.0 ? 1 : (int)lk;
        *t = n > k ? (int)ceil(10.0 * log((double)n / (double)k)) : 0;
    }
    return FSC_OK;
}

extern "C" fsc_status fsc_sync_status(void* stream) {
    int* word = device_status_word();
    if (!word) return FSC_ERR_CUDA;
    cudaStream_t s = as_stream(stream);
    int bits = 0;
    FSC_CUDA(cudaMemcpyAsync(&bits, word, sizeof(int), cudaMemcpyDeviceToHost, s));
    FSC_CUDA(cudaStreamSynchronize(s));
    if (bits) {
        FSC_CUDA(cudaMemsetAsync(word, 0, sizeof(int), s));
        FSC_CUDA(cudaStreamSynchronize(s));
    }
    return status_from_bits(bits);
}

extern "C" void fsc_set_wait_limit_ns(int64_t ns) { g_wait_limit.store(ns < 0 ? 0 : ns); }

extern "C" void fsc_inject_barrier_stall(int enable) { g_stall.store(enable ? 1 : 0); }

extern "C" const char* fsc_status_string(fsc_status s) {
    switch (s) {
        case FSC_OK: return "ok";
        case FSC_ERR_INVALID_ARG: return "invalid argument";
        case FSC_ERR_INDEX_RANGE: return "column index out of range or malformed row_ptr";
        case FSC_ERR_NOT_SYMMETRIC: return "adjacency matrix is not symmetric";
        case FSC_ERR_SELF_LOOP: return "self-loop in the graph";
        case FSC_ERR_BAD_WEIGHT: return "negative, NaN or infinite edge weight";
        case FSC_ERR_OOM: return "device out of memory";
        case FSC_ERR_CUDA: return "CUDA runtime error";
        case FSC_ERR_TIMEOUT: return "device-side wait timed out";
        case FSC_ERR_UNSORTED: return "row columns not increasing (required by the symmetry check)";
        case FSC_ERR_TOO_LARGE: return "problem exceeds the fixed scratch array of fsc_kmeans_static";
    }
    return "unknown status";
}

extern "C" const char* fsc_version(void) { return "0.1.0"; }
