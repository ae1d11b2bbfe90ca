// Algorithm 2 up to k-means: Gaussian start block, t power iterations, D^-1/2 scaling.
#include <math.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>

#include "spmm.cuh"

namespace fsc {

// Z0 = D^-1/2 X0 with X0 ~ N(0, I) from Philox4x64-10 (key (seed, 1)) and Box-Muller.
// Element (i, c) of X0 has index e = c*n + i; one thread per Philox block b = e/4 produces
// the four elements 4b..4b+3.  Pad columns l..LP-1 are zeroed.  Optionally records the
// per-column max |Z0| for the rescale protocol.
template <int LP, typename TO>
__global__ void __launch_bounds__(256) k_gauss_init(int n, int l, unsigned long long seed,
                                                    const float* __restrict__ dinv, TO* __restrict__ out,
                                                    unsigned* __restrict__ cm_out) {
    __shared__ unsigned s_cm[LP];
    if (threadIdx.x < LP) s_cm[threadIdx.x] = 0u;
    __syncthreads();
    const long long total = (long long)n * l;
    const long long nblk = (total + 3) / 4;
    const long long work = nblk > n ? nblk : n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < work; b += stride) {
        if (b < nblk) {
            const U64x4 r = philox4x64_10(U64x4{(unsigned long long)b, 0ull, 0ull, 0ull}, seed, STREAM_X0);
            const unsigned long long wd[4] = {r.x, r.y, r.z, r.w};
            float z[4];
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const float u1 = uniform24(wd[2 * p]);
                const float u2 = uniform24(wd[2 * p + 1]);
                const float rad = sqrtf(-2.0f * logf(u1));
                float sn, cs;
                sincospif(2.0f * u2, &sn, &cs);
                z[2 * p] = rad * cs;
                z[2 * p + 1] = rad * sn;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const long long e = 4 * b + j;
                if (e < total) {
                    const int c = (int)(e / n);
                    const long long i = e - (long long)c * n;
                    const float v = dinv[i] * z[j];
                    out[i * LP + c] = from_f32<TO>(v);
                    if (cm_out) atomicMax(&s_cm[c], __float_as_uint(fabsf(v)));
                }
            }
        }
        if (b < n) {
            for (int c = l; c < LP; ++c) out[b * LP + c] = from_f32<TO>(0.f);
        }
    }
    if (cm_out) {
        __syncthreads();
        if (threadIdx.x < LP && s_cm[threadIdx.x]) atomicMax(cm_out + threadIdx.x, s_cm[threadIdx.x]);
    }
}

// The four normals of Philox block b (Box-Muller on its two word pairs), as k_gauss_init forms them.
__device__ __forceinline__ void gauss_block(unsigned long long b, unsigned long long seed, float (&z)[4]) {
    const U64x4 r = philox4x64_10(U64x4{b, 0ull, 0ull, 0ull}, seed, STREAM_X0);
    const unsigned long long wd[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const float u1 = uniform24(wd[2 * p]);
        const float u2 = uniform24(wd[2 * p + 1]);
        const float rad = sqrtf(-2.0f * logf(u1));
        float sn, cs;
        sincospif(2.0f * u2, &sn, &cs);
        z[2 * p] = rad * cs;
        z[2 * p + 1] = rad * sn;
    }
}

// The same start block for rows of at most 8 entries, written row-wise: a thread takes four
// consecutive rows and every column of them (element (i, c) is draw c n + i, as above), so each
// thread stores 4 whole rows (one contiguous run) and reads 1/sqrt(d) once.  Element c n + i0 .. +3
// spans one Philox block, or two when n is not a multiple of 4.
template <int LP, typename TO>
__global__ void __launch_bounds__(256) k_gauss_init_rows(int n, int l, unsigned long long seed,
                                                         const float* __restrict__ dinv, TO* __restrict__ out,
                                                         unsigned* __restrict__ cm_out) {
    __shared__ unsigned s_cm[LP];
    if (threadIdx.x < LP) s_cm[threadIdx.x] = 0u;
    __syncthreads();
    const long long groups = ((long long)n + 3) / 4;
    float cmx[LP];   // this thread's largest |value| per column
#pragma unroll
    for (int c = 0; c < LP; ++c) cmx[c] = 0.f;
    for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < groups;
         g += (long long)gridDim.x * blockDim.x) {
        const long long i0 = 4 * g;
        float dv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) dv[q] = i0 + q < n ? dinv[i0 + q] : 0.f;
        float v[4][LP];
#pragma unroll
        for (int c = 0; c < LP; ++c) {
            if (c < l) {
                const long long e0 = (long long)c * n + i0;
                float za[4], zb[4];
                gauss_block((unsigned long long)(e0 >> 2), seed, za);
                const int off = (int)(e0 & 3);
                if (off) gauss_block((unsigned long long)(e0 >> 2) + 1, seed, zb);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    // draw e0 + q: word off + q of block e0 / 4, or of the next block (selects, not
                    // a dynamically indexed array, which would live in local memory)
                    const int w = off + q;
                    float z = za[q];
                    if (off) {
                        z = w == 1 ? za[1] : w == 2 ? za[2] : w == 3 ? za[3] : w == 4 ? zb[0] : w == 5 ? zb[1] : zb[2];
                    }
                    v[q][c] = dv[q] * z;
                    if (i0 + q < n) cmx[c] = fmaxf(cmx[c], fabsf(v[q][c]));
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q][c] = 0.f;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (i0 + q < n) store_row<LP, TO>(out + (size_t)(i0 + q) * LP, v[q]);
    }
    if (cm_out) {
#pragma unroll
        for (int c = 0; c < LP; ++c) {
            float m = cmx[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(&s_cm[c], __float_as_uint(m));
        }
        __syncthreads();
        if (threadIdx.x < LP && s_cm[threadIdx.x]) atomicMax(cm_out + threadIdx.x, s_cm[threadIdx.x]);
    }
}

template <typename TO>
cudaError_t launch_init(int LP, int n, int l, unsigned long long seed, const float* dinv, TO* out,
                        unsigned* cm_out, cudaStream_t s) {
    if (LP <= 8) {
        long long blocks = ((long long)n + 1023) / 1024;   // 256 threads x 4 rows
        const long long cap = (long long)device_props().num_sms * 8;
        if (blocks > cap) blocks = cap;
        switch (LP) {
            case 1: k_gauss_init_rows<1, TO><<<(unsigned)blocks, 256, 0, s>>>(n, l, seed, dinv, out, cm_out); break;
            case 2: k_gauss_init_rows<2, TO><<<(unsigned)blocks, 256, 0, s>>>(n, l, seed, dinv, out, cm_out); break;
            case 4: k_gauss_init_rows<4, TO><<<(unsigned)blocks, 256, 0, s>>>(n, l, seed, dinv, out, cm_out); break;
            case 8: k_gauss_init_rows<8, TO><<<(unsigned)blocks, 256, 0, s>>>(n, l, seed, dinv, out, cm_out); break;
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    const long long total = (long long)n * l;
    const long long work = (total + 3) / 4 > n ? (total + 3) / 4 : n;
    long long blocks = (work + 255) / 256;
    const long long cap = (long long)device_props().num_sms * 8;
    if (blocks > cap) blocks = cap;
    switch (LP) {
        case 1: k_gauss_init<1, TO><<<(unsigned)blocks, 256, 0, s>>>(n, l, seed, dinv, out, cm_out); break;
        case 2: k_gauss_init<2, TO><<<(unsigned)blocks, 256, 0, s>>>(n, l, seed, dinv, out, cm_out); break;
        case 4: k_gauss_init<4, TO><<<(unsigned)blocks, 256, 0, s>>>(n, l, seed, dinv, out, cm_out); break;
        case 8: k_gauss_init<8, TO><<<(unsigned)blocks, 256, 0, s>>>(n, l, seed, dinv, out, cm_out); break;
        case 16: k_gauss_init<16, TO><<<(unsigned)blocks, 256, 0, s>>>(n, l, seed, dinv, out, cm_out); break;
        case 32: k_gauss_init<32, TO><<<(unsigned)blocks, 256, 0, s>>>(n, l, seed, dinv, out, cm_out); break;
        case 64: k_gauss_init<64, TO><<<(unsigned)blocks, 256, 0, s>>>(n, l, seed, dinv, out, cm_out); break;
        case 128: k_gauss_init<128, TO><<<(unsigned)blocks, 256, 0, s>>>(n, l, seed, dinv, out, cm_out); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_init_any(int LP, int n, int l, unsigned long long seed, const float* dinv, void* out, int store,
                            cudaStream_t s) {
    if (store == FSC_F32) return launch_init<float>(LP, n, l, seed, dinv, static_cast<float*>(out), nullptr, s);
    if (store == FSC_F16) return launch_init<__half>(LP, n, l, seed, dinv, static_cast<__half*>(out), nullptr, s);
    return launch_init<__nv_bfloat16>(LP, n, l, seed, dinv, static_cast<__nv_bfloat16*>(out), nullptr, s);
}

// ---- lanes per row: explicit request > autotuned table > degree heuristic ------------------
namespace {
std::mutex g_tune_mu;
// (LP, store, weighted, degree bucket) -> lanes per row | unroll << 8
std::map<std::tuple<int, int, int, int>, int> g_tune;
int degree_bucket(double avg) { return (int)floor(2.0 * log2(avg < 1.0 ? 1.0 : avg)); }   // half octaves
}  // namespace

static int tuned_code(double avg_degree, int LP, int store, bool weighted) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(LP, store, weighted ? 1 : 0, degree_bucket(avg_degree)));
    return it == g_tune.end() ? 0 : it->second;
}

int tuned_threads_per_row(double avg_degree, int LP, int store, bool weighted) {
    return tuned_code(avg_degree, LP, store, weighted) & 0xff;
}

// The autotuned number of neighbour rows each lane keeps in flight (0: the kernel's default), for
// calls that let the library choose the lane count.
int tuned_unroll(const fsc_graph* g, int requested_threads, int LP, int store) {
    if (requested_threads) return 0;
    const double avg = g->n > 0 ? (double)g->nnz / (double)g->n : 0.0;
    return tuned_code(avg, LP, store, g->w != nullptr) >> 8;
}

int choose_threads_per_row(const fsc_graph* g, int requested, int LP, int store) {
    if (requested == 4 || requested == 8 || requested == 16 || requested == 32) return requested;
    const double avg = g->n > 0 ? (double)g->nnz / (double)g->n : 0.0;
    const int tuned = tuned_threads_per_row(avg, LP, store, g->w != nullptr);
    if (tuned) return tuned;
    if (avg <= 40.0) return 4;      // measured fastest at average degree ~22 (random 16-byte row gathers)
    if (avg <= 96.0) return 8;
    if (avg <= 256.0) return 16;
    return 32;
}

int choose_threads_per_row(const fsc_graph* g, int requested) { return choose_threads_per_row(g, requested, 4, 0); }

// Times one power step for each (lane count, rows in flight per lane) candidate on scratch
// iterates and records the fastest for the graph's (row width, storage type, weighting, degree
// bucket).
fsc_status autotune_graph(fsc_graph* g, int l, fsc_dtype store, int* best, float* best_us, cudaStream_t s) {
    const int LP = pad_l(l);
    const size_t es = store == FSC_F32 ? 4 : 2;
    const size_t bytes = (size_t)g->n * LP * es;
    void* buf = nullptr;
    FSC_CUDA(pool_malloc(&buf, 2 * bytes + 256, s));
    char* zin = static_cast<char*>(buf);
    char* zout = zin + ((bytes + 255) & ~(size_t)255);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMemsetAsync(zin, 0, bytes, s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int bestG = 0, bestU = 0;
    float bestT = 1e30f;
    const int cands[5] = {4, 4, 8, 16, 32}, unrolls[5] = {0, 3, 0, 0, 0};
    for (int ci = 0; ci < 5 && e == cudaSuccess; ++ci) {
        StepArgs a{};
        a.unroll = unrolls[ci];
        a.max_row = g->max_row;
        a.n = (int)g->n;
        a.rp = g->row_ptr;
        a.col = g->col;
        a.w = g->w;
        a.invdeg = g->invdeg;
        a.zin = zin;
        a.zout = zout;
        a.col_off = g->col_off;
        auto launch = [&]() {
            return store == FSC_F32 ? launch_step_f32(LP, cands[ci], g->w != nullptr, a, s)
                                    : launch_step_bf16(LP, cands[ci], g->w != nullptr, a, s);
        };
        if ((e = launch()) != cudaSuccess) break;
        if ((e = cudaEventRecord(e0, s)) != cudaSuccess) break;
        for (int r = 0; r < 5 && e == cudaSuccess; ++r) e = launch();
        if (e != cudaSuccess) break;
        if ((e = cudaEventRecord(e1, s)) != cudaSuccess) break;
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
        float ms = 0.f;
        if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
        if (ms < bestT) { bestT = ms; bestG = cands[ci]; bestU = unrolls[ci]; }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    pool_free(buf, s);
    cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        const double avg = g->n > 0 ? (double)g->nnz / (double)g->n : 0.0;
        g_tune[std::make_tuple(LP, (int)store, g->w ? 1 : 0, degree_bucket(avg))] = bestG | (bestU << 8);
    }
    if (best) *best = bestG;
    if (best_us) *best_us = bestT * 1000.f / 5.f;
    return FSC_OK;
}

fsc_status ensure_workspace(fsc_graph* g, size_t bytes, cudaStream_t s) {
    if (g->ws_bytes >= bytes) return FSC_OK;
    if (g->ws) {   // calls on one graph are stream-ordered, so the old block is free after them
        cudaError_t e = pool_free(g->ws, s);
        g->ws = nullptr;
        g->ws_bytes = 0;
        if (e != cudaSuccess) return cuda_status(e);
    }
    void* p = nullptr;
    cudaError_t e = pool_malloc(&p, bytes, s);
    if (e != cudaSuccess) return cuda_status(e);
    g->ws = p;
    g->ws_bytes = bytes;
    return FSC_OK;
}

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace fsc

using namespace fsc;

extern "C" fsc_status fsc_embed(const fsc_graph* gc, int l, int t, uint64_t seed, fsc_dtype store, float* emb,
                                const fsc_embed_opts* opts, void* stream) {
    NvtxRange nvtx_range("fsc_embed");
    fsc_graph* g = const_cast<fsc_graph*>(gc);
    if (!g || !emb || l < 1 || l > 8 || t < 0 || (store != FSC_F32 && store != FSC_BF16)) return FSC_ERR_INVALID_ARG;
    const int LP = pad_l(l);
    if (!aligned(emb, (size_t)(LP * 4 < 16 ? LP * 4 : 16))) return FSC_ERR_INVALID_ARG;
    const uint32_t flags = opts ? opts->flags : 0u;
    if (flags & ~FSC_EMBED_RESCALE) return FSC_ERR_INVALID_ARG;
    const bool rescale = (flags & FSC_EMBED_RESCALE) != 0;
    const int G = choose_threads_per_row(g, opts ? opts->threads_per_row : 0, LP, (int)store);
    cudaStream_t s = as_stream(stream);
    const int n = (int)g->n;
    if (t == 0) {
        FSC_CUDA(launch_init<float>(LP, n, l, seed, g->dinv, emb, nullptr, s));
        if (opts && opts->ev_spmm_begin) FSC_CUDA(cudaEventRecord((cudaEvent_t)opts->ev_spmm_begin, s));
        if (opts && opts->ev_spmm_end) FSC_CUDA(cudaEventRecord((cudaEvent_t)opts->ev_spmm_end, s));
        return FSC_OK;
    }
    fsc_status rc = ensure_workspace(g, (size_t)n * LP * 4 + 256, s);
    if (rc != FSC_OK) return rc;
    unsigned* cm = g->colmax;   // three buffers of 8
    int* expo = rescale ? g->expo : nullptr;
    if (rescale) FSC_CUDA(cudaMemsetAsync(g->colmax, 0, 256, s));   // 3 x 8 column maxima + 8 exponents

    StepArgs a{};
    a.n = n;
    a.rp = g->row_ptr;
    a.col = g->col;
    a.w = g->w;
    a.invdeg = g->invdeg;
    a.expo = expo;
    a.col_off = g->col_off;
    a.max_row = g->max_row;
    a.unroll = tuned_unroll(g, opts ? opts->threads_per_row : 0, LP, (int)store);
    const bool weighted = g->w != nullptr;

    if (store == FSC_F32) {
        float* buf[2];
        buf[t % 2] = emb;
        buf[(t + 1) % 2] = static_cast<float*>(g->ws);
        FSC_CUDA(launch_init<float>(LP, n, l, seed, g->dinv, buf[0], rescale ? cm : nullptr, s));
        if (opts && opts->ev_spmm_begin) FSC_CUDA(cudaEventRecord((cudaEvent_t)opts->ev_spmm_begin, s));
        for (int it = 0; it < t; ++it) {
            const bool last = it == t - 1;
            a.zin = buf[it % 2];
            a.zout = buf[(it + 1) % 2];
            a.cm_in = (rescale && !last) ? cm + 8 * (it % 3) : nullptr;
            a.cm_out = (rescale && it < t - 2) ? cm + 8 * ((it + 1) % 3) : nullptr;
            a.cm_zero = (rescale && !last) ? cm + 8 * ((it + 2) % 3) : nullptr;
            a.last = last ? 1 : 0;
            FSC_CUDA(launch_step_f32(LP, G, weighted, a, s));
            FSC_CUDA(long_rows_power(g, LP, 0, 0, a, s));
        }
    } else {
        __nv_bfloat16* wb[2];
        wb[0] = static_cast<__nv_bfloat16*>(g->ws);
        wb[1] = wb[0] + (size_t)n * LP;
        FSC_CUDA(launch_init<__nv_bfloat16>(LP, n, l, seed, g->dinv, wb[0], rescale ? cm : nullptr, s));
        if (opts && opts->ev_spmm_begin) FSC_CUDA(cudaEventRecord((cudaEvent_t)opts->ev_spmm_begin, s));
        for (int it = 0; it < t; ++it) {
            const bool last = it == t - 1;
            a.zin = wb[it % 2];
            a.zout = last ? static_cast<void*>(emb) : static_cast<void*>(wb[(it + 1) % 2]);
            a.cm_in = (rescale && !last) ? cm + 8 * (it % 3) : nullptr;
            a.cm_out = (rescale && it < t - 2) ? cm + 8 * ((it + 1) % 3) : nullptr;
            a.cm_zero = (rescale && !last) ? cm + 8 * ((it + 2) % 3) : nullptr;
            a.last = last ? 1 : 0;
            if (last) FSC_CUDA(launch_step_bf16_to_f32(LP, G, weighted, a, s));
            else FSC_CUDA(launch_step_bf16(LP, G, weighted, a, s));
            FSC_CUDA(long_rows_power(g, LP, 1, last ? 0 : 1, a, s));
        }
    }
    if (opts && opts->ev_spmm_end) FSC_CUDA(cudaEventRecord((cudaEvent_t)opts->ev_spmm_end, s));
    return FSC_OK;
}

extern "C" fsc_status fsc_power_step(const fsc_graph* g, int l, fsc_dtype store, const void* z_in, void* z_out,
                                     int threads_per_row, void* stream) {
    NvtxRange nvtx_range("fsc_power_step");
    if (!g || !z_in || !z_out || z_in == z_out || l < 1 || l > 8 || (store != FSC_F32 && store != FSC_BF16))
        return FSC_ERR_INVALID_ARG;
    const int LP = pad_l(l);
    const size_t es = store == FSC_F32 ? 4 : 2;
    const size_t al = LP * es < 16 ? LP * es : 16;
    if (!aligned(z_in, al) || !aligned(z_out, al)) return FSC_ERR_INVALID_ARG;
    StepArgs a{};
    a.n = (int)g->n;
    a.rp = g->row_ptr;
    a.col = g->col;
    a.w = g->w;
    a.invdeg = g->invdeg;
    a.zin = z_in;
    a.zout = z_out;
    a.col_off = g->col_off;
    a.max_row = g->max_row;
    a.unroll = tuned_unroll(g, threads_per_row, LP, (int)store);
    const int G = choose_threads_per_row(g, threads_per_row, LP, (int)store);
    cudaStream_t s = as_stream(stream);
    if (store == FSC_F32) FSC_CUDA(launch_step_f32(LP, G, g->w != nullptr, a, s));
    else FSC_CUDA(launch_step_bf16(LP, G, g->w != nullptr, a, s));
    FSC_CUDA(long_rows_power(g, LP, store == FSC_F32 ? 0 : 1, store == FSC_F32 ? 0 : 1, a, s));
    return FSC_OK;
}

extern "C" fsc_status fsc_autotune(const fsc_graph* g, int l, fsc_dtype store, int* best_threads_per_row,
                                   float* best_us, void* stream) {
    NvtxRange nvtx_range("fsc_autotune");
    if (!g || l < 1 || l > 8 || (store != FSC_F32 && store != FSC_BF16)) return FSC_ERR_INVALID_ARG;
    return autotune_graph(const_cast<fsc_graph*>(g), l, store, best_threads_per_row, best_us, as_stream(stream));
}
