// Internal definitions shared by the libfsc translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda/atomic>
#include <nvtx3/nvToolsExt.h>

#include "../../include/fsc.h"

namespace fsc {

// ---- device status word ---------------------------------------------------------------
// Bits OR-ed into a device int by kernels; translated to fsc_status on the host.
enum : int {
    ST_INDEX_RANGE = 1 << 0,
    ST_SELF_LOOP = 1 << 1,
    ST_BAD_WEIGHT = 1 << 2,
    ST_NOT_SYMMETRIC = 1 << 3,
    ST_UNSORTED = 1 << 4,
    ST_TIMEOUT = 1 << 5,
    ST_BAD_ROWPTR = 1 << 6,
};

fsc_status status_from_bits(int bits);

// ---- optional bounds checking (compile flag FSC_BOUNDS_CHECK) ----------------------------------
// With the flag, an index that a kernel derives from its inputs (a column index, a label, the index
// of a chosen centre) is tested against its range before the access it addresses; the first index
// found outside is recorded (site, value, range) in the translation unit's record, the access is
// skipped, and fsc_bounds_report() returns the record.  Nothing traps.  Without the flag the test
// is the constant true and compiles away.
enum BoundsSite : int {
    BS_GATHER = 1,        // neighbour row of a sparse step (column index, minus the graph's first vertex)
    BS_GATHER_WIDE = 2,   // neighbour row of the wide power step
    BS_KPP_NEAR = 3,      // k-means++: a point's nearest-centre index
    BS_LLOYD_LABEL = 4,   // Lloyd: a point's label
    BS_WIDE_NEAR = 5,     // wide k-means++: a point's nearest-centre index
    BS_WIDE_LABEL = 6,    // wide Lloyd: a point's previous label
    BS_KPP_PICK = 7,      // k-means++: the chosen point
};
struct BoundsRecord {
    int site;
    int unused;
    long long index, lo, hi;
};
#ifdef FSC_BOUNDS_CHECK
static __device__ BoundsRecord g_bounds;   // one per translation unit
__device__ __forceinline__ bool in_range(long long i, long long lo, long long hi, int site) {
    if (i >= lo && i < hi) return true;
    if (atomicCAS(&g_bounds.site, 0, site) == 0) {
        g_bounds.index = i;
        g_bounds.lo = lo;
        g_bounds.hi = hi;
    }
    return false;
}
// Host reader of one translation unit's record (defined by FSC_BOUNDS_READER in that unit).
#define FSC_BOUNDS_READER(name)                                                              \
    cudaError_t bounds_read_##name(BoundsRecord* r, bool clear) {                           \
        cudaError_t e = cudaMemcpyFromSymbol(r, g_bounds, sizeof(BoundsRecord));            \
        if (e == cudaSuccess && clear) {                                                     \
            const BoundsRecord z{};                                                          \
            e = cudaMemcpyToSymbol(g_bounds, &z, sizeof(BoundsRecord));                      \
        }                                                                                    \
        return e;                                                                            \
    }
#else
__device__ __forceinline__ constexpr bool in_range(long long, long long, long long, int) { return true; }
#define FSC_BOUNDS_READER(name)
#endif

// ---- host helpers ---------------------------------------------------------------------
struct DeviceProps {
    int device;
    int num_sms;
};
const DeviceProps& device_props();        // of the current device (cached per device)
int* device_status_word();                // per-device error word (allocated once)
long long wait_limit_ns();
int barrier_stall();                      // testing hook: nonzero = never release grid barriers
fsc_status cuda_status(cudaError_t e);    // records and maps a CUDA error
// Device memory for the library's own buffers comes from one stream-ordered pool per device that
// keeps freed blocks mapped (release threshold = max), so repeated create / cluster / destroy
// cycles neither map nor unmap memory; fsc_release_cached_memory() returns it to the driver.
cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t s);
cudaError_t pool_free(void* p, cudaStream_t s);
// Blocks per SM of a kernel at (threads, dynamic shared bytes), with the opt-in shared-memory
// attribute raised as needed; cached per (device, kernel, threads, bytes).  0 on error.
int kernel_occupancy(const void* fn, int threads, size_t smem);

#define FSC_CUDA(call)                                            \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return ::fsc::cuda_status(e_);     \
    } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ---- asynchronous copies global -> shared (cp.async): each thread's copies are visible to that
// thread after its wait; the copies of one commit group complete together ----------------------
// 16 bytes; bytes < 16 copies that many and zero-fills the rest
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    const size_t ga = __cvta_generic_to_global(gmem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(ga), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// An NVTX range for the lifetime of a C-ABI call (seen by Nsight tools; costs nothing without one).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---- row vectors: LP elements of type T, loaded/stored as aligned chunks ---------------
template <int B> struct Chunk;
template <> struct Chunk<2> { using type = unsigned short; };
template <> struct Chunk<4> { using type = unsigned int; };
template <> struct Chunk<8> { using type = uint2; };
template <> struct Chunk<16> { using type = uint4; };

__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float to_f32(__half x) { return __half2float(x); }
template <typename T> __device__ __forceinline__ T from_f32(float x);
template <> __device__ __forceinline__ float from_f32<float>(float x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float x) {
    return __float2bfloat16_rn(x);
}
template <> __device__ __forceinline__ __half from_f32<__half>(float x) { return __float2half_rn(x); }

// p must point to global memory: the row is read through the read-only data path (__ldg)
template <int LP, typename T>
__device__ __forceinline__ void load_row(const T* __restrict__ p, float (&v)[LP]) {
    constexpr int BYTES = LP * (int)sizeof(T);
    constexpr int CB = BYTES < 16 ? BYTES : 16;
    using C = typename Chunk<CB>::type;
    constexpr int NC = BYTES / CB;
    C buf[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) buf[i] = __ldg(reinterpret_cast<const C*>(p) + i);
    const T* e = reinterpret_cast<const T*>(buf);
#pragma unroll
    for (int c = 0; c < LP; ++c) v[c] = to_f32(e[c]);
}

template <int LP, typename T>
__device__ __forceinline__ void store_row(T* __restrict__ p, const float (&v)[LP]) {
    constexpr int BYTES = LP * (int)sizeof(T);
    constexpr int CB = BYTES < 16 ? BYTES : 16;
    using C = typename Chunk<CB>::type;
    constexpr int NC = BYTES / CB;
    C buf[NC];
    T* e = reinterpret_cast<T*>(buf);
#pragma unroll
    for (int c = 0; c < LP; ++c) e[c] = from_f32<T>(v[c]);
#pragma unroll
    for (int i = 0; i < NC; ++i) reinterpret_cast<C*>(p)[i] = buf[i];
}

// ---- Philox4x64-10 (Salmon et al., SC'11) ----------------------------------------------
struct U64x4 {
    unsigned long long x, y, z, w;
};

__device__ __forceinline__ U64x4 philox4x64_10(U64x4 c, unsigned long long k0, unsigned long long k1) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long hi0 = __umul64hi(M0, c.x), lo0 = M0 * c.x;
        const unsigned long long hi1 = __umul64hi(M1, c.z), lo1 = M1 * c.z;
        c = U64x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += W0;
        k1 += W1;
    }
    return c;
}

// uniform in (0, 1] from the top 24 bits (exact in float)
__device__ __forceinline__ float uniform24(unsigned long long w) {
    return (float)((unsigned)(w >> 40) + 1u) * 0x1p-24f;
}
// uniform in [0, 1) from the top 53 bits (exact in double)
__device__ __forceinline__ double uniform53(unsigned long long w) { return (double)(w >> 11) * 0x1p-53; }

constexpr unsigned long long STREAM_X0 = 1, STREAM_KMEANSPP = 2;

// ---- bounded grid-wide barrier for cooperative launches --------------------------------
struct GridBarrier {
    unsigned int count;        // arrivals so far (starts at 0)
    unsigned int reserved;
};

__device__ __forceinline__ long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return (long long)t;
}

// All blocks of a cooperative launch call this, each with its own count of the barriers it has
// passed (`epoch`, starting at 0; the counter starts at 0 too).  Arrivals only ever increase the
// counter, so barrier e releases once it reaches e * gridDim.x and no block has to reset or
// re-arm anything.  Returns false (for every thread of the block) if the device error word is
// set or the wait exceeded `limit_ns`; the caller then returns.  With `stall` set, block 0
// never arrives (test hook for the timeout path).
__device__ __forceinline__ bool grid_sync(GridBarrier* bar, int* status, long long limit_ns, int stall,
                                          unsigned& epoch) {
    __shared__ int s_ok;
    __syncthreads();
    epoch += 1;
    if (threadIdx.x == 0) {
        cuda::atomic_ref<unsigned int, cuda::thread_scope_device> cnt(bar->count);
        cuda::atomic_ref<int, cuda::thread_scope_device> st(*status);
        int ok = st.load(cuda::memory_order_relaxed) == 0;
        if (ok) {
            const unsigned target = epoch * gridDim.x;
            __threadfence();
            if (!(stall && blockIdx.x == 0)) cnt.fetch_add(1u, cuda::memory_order_release);
            const long long t0 = global_ns();
            unsigned spins = 0;
            while ((int)(cnt.load(cuda::memory_order_acquire) - target) < 0) {
                if (st.load(cuda::memory_order_relaxed) != 0) { ok = 0; break; }
                if (++spins > 64) __nanosleep(32);
                if ((spins & 15u) == 0 && global_ns() - t0 > limit_ns) {
                    st.fetch_or(ST_TIMEOUT, cuda::memory_order_relaxed);
                    ok = 0;
                    break;
                }
            }
            __threadfence();
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---- misc --------------------------------------------------------------------------------
__device__ __forceinline__ int exponent_of(float m) {   // floor(log2 m) for normal m > 0, else 0
    const unsigned b = __float_as_uint(m);
    const int e = (int)((b >> 23) & 0xff);
    return (e == 0 || e == 0xff) ? 0 : e - 127;
}

// float32 squared distance in a fixed order, no contraction (mirrors the oracle's decision rule)
template <int LP>
__device__ __forceinline__ float sqdist(const float (&x)[LP], const float* __restrict__ c) {
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < LP; ++j) {
        const float d = __fsub_rn(x[j], c[j]);
        acc = __fadd_rn(acc, __fmul_rn(d, d));
    }
    return acc;
}

// Row width of an l-column block: 1, 2, 4, 8 for l <= 8 (every entry point); 16, 32, 64, 128 for
// l = 9 .. 128 (orthogonal iteration, Ritz vectors, k-means); 0 beyond.
// Rows with more stored entries than kLongRow are summed in segments of kSegLen entries by their
// own kernels (longrows.cu); the row-split kernels skip them.
constexpr int64_t kLongRow = 1024;
constexpr int64_t kSegLen = 1024;

inline int pad_l(int l) {
    return l < 1 ? 0 : l == 1 ? 1 : l == 2 ? 2 : l <= 4 ? 4 : l <= 8 ? 8 : l <= 16 ? 16 : l <= 32 ? 32 : l <= 64 ? 64
                                                                                         : l <= 128 ? 128 : 0;
}

}  // namespace fsc

// The graph object behind the opaque handle.
struct fsc_graph {
    int device;
    int64_t n, nnz;
    const int64_t* row_ptr;
    const int32_t* col;
    const float* w;
    double* deg;
    float* dinv;
    float* invdeg;
    int64_t n_isolated;
    double volume;
    double deg_sumsq;   // sum of d(v)^2
    double deg_max;     // max d(v)
    // embedding workspace (grown on demand)
    void* ws;
    size_t ws_bytes;
    unsigned* colmax;   // 3 x 8 unsigned
    int* expo;          // 8 ints
    long long col_off;  // subtracted from column ids (0, or the first vertex of a graph inside a batch)
    // long rows (longrows.cu): max_row = kLongRow when there are any, else no limit
    long long max_row = 0x7fffffffffffffffLL;
    int64_t n_long, n_seg;
    void* long_base;             // one allocation holding the tables below
    int64_t* long_rows;          // the long rows, increasing
    int32_t* long_seg0;          // per long row: its first segment
    int32_t* long_nseg;          // per long row: its number of segments
    int64_t* seg_lo;             // per segment: first entry
    int64_t* seg_hi;             // per segment: one past its last entry
    float* seg_part;             // per segment: partial sums, 8 floats
    void* copy_base;             // FSC_COPY: the graph's own copy of the CSR
    // the learned filter's side stream (its coefficients run beside the later sparse steps) and the
    // two events joining it, made on first use
    cudaStream_t side;
    cudaEvent_t ev_fork, ev_join;
};
