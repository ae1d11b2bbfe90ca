// Graph ingest: validation and degrees d(v) = sum_{u != v} w(u, v) (Sec. 2), plus host utilities.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <tuple>

#include "fsc_internal.cuh"

namespace fsc {

namespace {
constexpr int kMaxDevices = 64;
DeviceProps g_props[kMaxDevices];
int* g_status_word[kMaxDevices];
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
    std::lock_guard<std::mutex> lock(g_status_mu);
    if (!g_status_word[dev]) {
        int* p = nullptr;
        if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return nullptr;
        g_status_word[dev] = p;
    }
    return g_status_word[dev];
}

namespace {
cudaMemPool_t g_pool[kMaxDevices];
std::mutex g_pool_mu;
std::mutex g_occ_mu;
std::map<std::tuple<int, const void*, int, size_t>, int> g_occ;
std::map<std::pair<int, const void*>, size_t> g_smem_attr;
}  // namespace

static cudaMemPool_t library_pool(int dev) {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
        unsigned long long keep = ~0ull;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = p;
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
    std::lock_guard<std::mutex> lock(g_occ_mu);
    const auto key = std::make_tuple(dev, fn, threads, smem);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) return it->second;
    // the opt-in limit covers dynamic bytes on top of the kernel's static shared memory, so it is
    // raised for every size above the largest one set so far
    size_t& attr = g_smem_attr[std::make_pair(dev, fn)];
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

// Validation and degrees, kDegLanes lanes per row: the lanes of a row read its entries side by
// side (coalesced), each keeps a partial count (unit weights, exact) or a float64 partial sum
// (weights), and the partials meet in a shuffle tree.  D^-1/2 and 1/d are formed in float32 from
// the float64 degree (correctly rounded sqrt and division, within 1-2 ulp of the exact values);
// float64 arithmetic stays out of the unit-weight path, which it would slow down on this GPU.
constexpr int kDegLanes = 8;

// float64 value of an integer below 2^53, built with integer operations only (the float64 pipe
// is a small fraction of the integer one on this GPU, and it bounded the unit-weight kernel).
__device__ __forceinline__ double exact_u64_to_f64(unsigned long long c) {
    if (c == 0) return 0.0;
    const int e = 63 - __clzll((long long)c);
    const unsigned long long mant = (c << (52 - e)) & ((1ull << 52) - 1);
    return __longlong_as_double((long long)((((unsigned long long)(1023 + e)) << 52) | mant));
}
__global__ void __launch_bounds__(256) k_degree(int64_t n, int64_t nnz, const int64_t* __restrict__ rp,
                                                const int32_t* __restrict__ col, const float* __restrict__ w,
                                                int check_sorted, double* __restrict__ deg,
                                                float* __restrict__ dinv, float* __restrict__ invdeg,
                                                unsigned long long* __restrict__ n_iso, double* __restrict__ vol,
                                                int* __restrict__ status, double* __restrict__ sumsq,
                                                unsigned long long* __restrict__ dmax_bits) {
    constexpr int G = kDegLanes, RPW = 32 / G;
    const int lane = threadIdx.x & 31, sub = lane % G, grp = lane / G;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0 && (rp[0] != 0 || rp[n] != nnz)) atomicOr(status, ST_BAD_ROWPTR);
    int bad = 0;
    unsigned iso = 0;
    double vsum = 0.0, vsq = 0.0, vmax = 0.0;
    long long cnt_total = 0;
    unsigned long long usq = 0, umax = 0;   // unit weights: sum of d^2 and max d as integers
    for (int64_t base = warp * RPW; base < n; base += nwarps * RPW) {   // warp-uniform trip count
        const int64_t i = base + grp;
        const bool active = i < n;
        int64_t s = 0, e = 0;
        if (active) {
            s = rp[i];
            e = rp[i + 1];
            if (s < 0 || e < s || e > nnz) {
                bad |= ST_BAD_ROWPTR;
                s = e = 0;
            }
        }
        double d = 0.0;
        long long cnt = 0;
        for (int64_t p = s + sub; p < e; p += G) {
            const int j = col[p];
            if (j < 0 || (int64_t)j >= n) { bad |= ST_INDEX_RANGE; continue; }
            if ((int64_t)j == i) { bad |= ST_SELF_LOOP; continue; }
            if (check_sorted && p > s && col[p - 1] >= j) bad |= ST_UNSORTED;
            if (w) {
                const float wv = w[p];
                if (!(wv >= 0.0f) || isinf(wv)) { bad |= ST_BAD_WEIGHT; continue; }
                d += (double)wv;
            } else {
                ++cnt;
            }
        }
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
        if (w) {
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
        }
        if (active && sub == 0 && !w) {
            // unit weights: d is the exact count; everything stays in integer registers
            const unsigned long long c = (unsigned long long)cnt;
            cnt_total += cnt;
            deg[i] = exact_u64_to_f64(c);
            if (c < (1ull << 26)) usq += c * c;          // a thread's few rows cannot overflow
            else vsq += (double)c * (double)c;            // only with repeated entries
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
        } else if (active && sub == 0) {
            vsum += d;
            deg[i] = d;
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
    }
    for (int off = 16; off > 0; off >>= 1) {
        bad |= __shfl_xor_sync(0xffffffffu, bad, off);
        iso += __shfl_xor_sync(0xffffffffu, iso, off);
        cnt_total += __shfl_xor_sync(0xffffffffu, cnt_total, off);
    }
    if (w) {
        for (int off = 16; off > 0; off >>= 1) vsum += __shfl_xor_sync(0xffffffffu, vsum, off);
    }
    if (!w) {   // fold the integer statistics in once per thread
        vsq += (double)usq;
        vmax = (double)umax;
    }
    for (int off = 16; off > 0; off >>= 1) {
        vsq += __shfl_xor_sync(0xffffffffu, vsq, off);
        vmax = fmax(vmax, __shfl_xor_sync(0xffffffffu, vmax, off));
    }
    // block totals first: one atomic per block and statistic (per-warp atomics on five single
    // addresses serialised at L2 and dominated the kernel)
    __shared__ double s_sq[8], s_mx[8], s_vol[8];
    __shared__ int s_bad[8];
    __shared__ unsigned s_iso[8];
    const int wid = threadIdx.x >> 5;
    if (lane == 0) {
        s_sq[wid] = vsq;
        s_mx[wid] = vmax;
        s_vol[wid] = w ? vsum : (double)cnt_total;
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
    if (flags & ~FSC_VALIDATE_SYMMETRY) return FSC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    int dev = 0;
    FSC_CUDA(cudaGetDevice(&dev));
    fsc_graph* g = new (std::nothrow) fsc_graph();
    if (!g) return FSC_ERR_OOM;
    memset(g, 0, sizeof(*g));
    g->device = dev;
    g->n = n;
    g->nnz = nnz;
    g->row_ptr = row_ptr;
    g->col = col_idx;
    g->w = w;
    // one allocation: deg (n doubles) | header (256 B: volume, n_iso, status, sumsq, max bits) |
    //                 dinv (n floats) | invdeg (n floats) | colmax 24 u32 | expo 8 int
    const size_t n8 = (size_t)n * 8, n4 = ((size_t)n * 4 + 255) & ~(size_t)255;
    const size_t bytes = n8 + 256 + 2 * n4 + 256;
    char* base = nullptr;
    cudaError_t e = pool_malloc(reinterpret_cast<void**>(&base), bytes, s);
    if (e != cudaSuccess) {
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
    };
    Header* hdr = reinterpret_cast<Header*>(base + n8);
    g->deg = reinterpret_cast<double*>(base);
    g->dinv = reinterpret_cast<float*>(base + n8 + 256);
    g->invdeg = reinterpret_cast<float*>(base + n8 + 256 + n4);
    g->colmax = reinterpret_cast<unsigned*>(base + n8 + 256 + 2 * n4);
    g->expo = reinterpret_cast<int*>(base + n8 + 256 + 2 * n4 + 128);
    fsc_status rc = FSC_OK;
    do {
        if ((e = cudaMemsetAsync(base + n8, 0, 256, s)) != cudaSuccess) break;
        if ((e = cudaMemsetAsync(base + n8 + 256 + 2 * n4, 0, 256, s)) != cudaSuccess) break;
        const int threads = 256;
        constexpr int rows_per_block = threads / 32 * (32 / kDegLanes);
        const int64_t want = (n + rows_per_block - 1) / rows_per_block;
        // enough warps that each walks only a few rows: every row is a dependent row_ptr -> col
        // load chain, so the kernel is latency-bound with fewer warps in flight
        const int64_t cap = (int64_t)device_props().num_sms * 32;
        const int blocks = (int)(want < cap ? want : cap);
        const int check_sorted = (flags & FSC_VALIDATE_SYMMETRY) ? 1 : 0;
        k_degree<<<blocks, threads, 0, s>>>(n, nnz, row_ptr, col_idx, w, check_sorted, g->deg, g->dinv,
                                            g->invdeg, &hdr->niso, &hdr->vol, &hdr->status, &hdr->sumsq,
                                            &hdr->dmax_bits);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        Header h{};
        if ((e = cudaMemcpyAsync(&h, hdr, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
        int bits = h.status;
        if (bits == 0 && check_sorted) {
            k_symmetry<<<blocks, threads, 0, s>>>(n, row_ptr, col_idx, w, &hdr->status);
            if ((e = cudaGetLastError()) != cudaSuccess) break;
            if ((e = cudaMemcpyAsync(&bits, &hdr->status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
        }
        if (bits) { rc = status_from_bits(bits); break; }
        g->n_isolated = (int64_t)h.niso;
        g->volume = h.vol;
        g->deg_sumsq = h.sumsq;
        memcpy(&g->deg_max, &h.dmax_bits, 8);
    } while (0);
    if (e != cudaSuccess) rc = cuda_status(e);
    if (rc != FSC_OK) {
        pool_free(base, s);
        cudaStreamSynchronize(s);
        delete g;
        return rc;
    }
    *out = g;
    return FSC_OK;
}

extern "C" fsc_status fsc_destroy_graph(fsc_graph* g) {
    if (!g) return FSC_OK;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(g->device);
    // all work that may still read the graph's buffers ends here; the blocks go back to the
    // library pool (no unmapping), ordered on the legacy stream after that point
    cudaError_t e = cudaDeviceSynchronize();
    pool_free(g->ws, 0);
    pool_free(g->deg, 0);
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

extern "C" int fsc_pad_l(int l) { return (l >= 1 && l <= 8) ? pad_l(l) : 0; }

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
