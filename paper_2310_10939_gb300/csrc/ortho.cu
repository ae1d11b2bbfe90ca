// Orthogonal iteration: the power method of Algorithm 1 on a block of l vectors kept
// orthonormal, so that the columns do not all collapse onto the top eigenvector (with l = k it
// is the "PM k Vectors" variant compared in Sec. 4).
//
// The block is kept in embedding coordinates z = D^-1/2 x, so the x-space inner product is
// <x_a, x_b> = sum_v d(v) z_a(v) z_b(v).  Orthonormalising is CholeskyQR2: the l x l Gram
// G = Z^T D Z (float32 per thread, float64 per block and in total), G = R^T R with R upper
// triangular and positive diagonal (float64, one block), Z <- Z R^-1, and the same once more to
// restore orthogonality lost to rounding in the first pass.  The result is the unique basis with
// positive-diagonal R; orthonormalising never changes the span, so after t steps the columns
// span M^t X0 exactly as the plain method's do.
#include <math.h>

#include "spmm.cuh"

namespace fsc {

fsc_status ensure_workspace(fsc_graph* g, size_t bytes, cudaStream_t s);
cudaError_t launch_init_any(int LP, int n, int l, unsigned long long seed, const float* dinv, void* out, int store,
                            cudaStream_t s);
int choose_threads_per_row(const fsc_graph* g, int requested, int LP, int store);

constexpr int kOrthoThreads = 256;

// l = 9 .. 128 (wide.cu)
fsc_status embed_orthogonal_wide(fsc_graph* g, int l, int t, int every, uint64_t seed, float* emb,
                                 const fsc_embed_opts* opts, cudaStream_t s);
fsc_status ritz_wide(fsc_graph* g, int l, float* emb, double* values, cudaStream_t s);

// Per-block partial Gram sums (upper triangle, row-major index a * LP + b, a <= b).
template <int LP>
__global__ void __launch_bounds__(kOrthoThreads) k_gram(int n, const float* __restrict__ z,
                                                        const double* __restrict__ deg, double* __restrict__ part) {
    constexpr int NT = LP * (LP + 1) / 2;
    __shared__ float s_w[kOrthoThreads / 32][NT];
    float acc[NT];
#pragma unroll
    for (int e = 0; e < NT; ++e) acc[e] = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float v[LP];
        load_row<LP, float>(z + (size_t)i * LP, v);
        const float d = (float)deg[i];
        int e = 0;
#pragma unroll
        for (int a = 0; a < LP; ++a) {
            const float da = d * v[a];
#pragma unroll
            for (int b = a; b < LP; ++b) {
                acc[e] = fmaf(da, v[b], acc[e]);
                ++e;
            }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < NT; ++e) {
        float x = acc[e];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (lane == 0) s_w[wid][e] = x;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NT; e += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < kOrthoThreads / 32; ++w) t += (double)s_w[w][e];
        part[(size_t)blockIdx.x * NT + e] = t;
    }
}

// One block: total Gram of the leading l columns, Cholesky G = R^T R, and R^-1 (LP x LP floats,
// identity on the padded columns).  A column whose pivot falls below 1e-14 of the largest
// diagonal entry is linearly dependent on the earlier ones (or zero): its column of R^-1 is set
// to zero, so it leaves the block as a zero column.
template <int LP>
__global__ void k_chol_inv(const double* __restrict__ part, int nb, int l, float* __restrict__ rinv) {
    constexpr int NT = LP * (LP + 1) / 2;
    __shared__ double s_g[NT];
    for (int e = threadIdx.x; e < NT; e += blockDim.x) {
        double t = 0.0;
        for (int q = 0; q < nb; ++q) t += part[(size_t)q * NT + e];
        s_g[e] = t;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double G[LP][LP], R[LP][LP], Ri[LP][LP];
    int e = 0;
    for (int a = 0; a < LP; ++a)
        for (int b = a; b < LP; ++b) {
            G[a][b] = s_g[e];
            G[b][a] = s_g[e];
            ++e;
        }
    double gmax = 0.0;
    for (int a = 0; a < l; ++a) gmax = fmax(gmax, G[a][a]);
    bool dead[LP];
    for (int a = 0; a < LP; ++a)
        for (int b = 0; b < LP; ++b) R[a][b] = 0.0;
    for (int a = 0; a < l; ++a) {
        double p = G[a][a];
        for (int c = 0; c < a; ++c) p -= R[c][a] * R[c][a];
        dead[a] = !(p > 1e-14 * gmax) || gmax <= 0.0;
        R[a][a] = dead[a] ? 1.0 : sqrt(p);
        for (int b = a + 1; b < l; ++b) {
            double q = G[a][b];
            for (int c = 0; c < a; ++c) q -= R[c][a] * R[c][b];
            R[a][b] = dead[a] ? 0.0 : q / R[a][a];
        }
    }
    // R^-1 by back substitution, column by column (upper triangular)
    for (int a = 0; a < LP; ++a)
        for (int b = 0; b < LP; ++b) Ri[a][b] = 0.0;
    for (int c = 0; c < l; ++c) {
        Ri[c][c] = 1.0 / R[c][c];
        for (int a = c - 1; a >= 0; --a) {
            double s = 0.0;
            for (int b = a + 1; b <= c; ++b) s += R[a][b] * Ri[b][c];
            Ri[a][c] = -s / R[a][a];
        }
    }
    for (int c = 0; c < l; ++c)
        if (dead[c])
            for (int a = 0; a < LP; ++a) Ri[a][c] = 0.0;
    for (int a = 0; a < LP; ++a)
        for (int b = 0; b < LP; ++b)
            rinv[a * LP + b] = (a >= l || b >= l) ? (a == b && a >= l ? 1.f : 0.f) : (float)Ri[a][b];
}

// z_v <- z_v R^-1 for every row (row vector times upper-triangular matrix), in place.
template <int LP>
__global__ void __launch_bounds__(kOrthoThreads) k_apply(int n, float* __restrict__ z, const float* __restrict__ rinv) {
    __shared__ float s_r[LP * LP];
    for (int q = threadIdx.x; q < LP * LP; q += blockDim.x) s_r[q] = rinv[q];
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float v[LP], o[LP];
        load_row<LP, float>(z + (size_t)i * LP, v);
#pragma unroll
        for (int c = 0; c < LP; ++c) {
            float t = 0.f;
#pragma unroll
            for (int a = 0; a <= c; ++a) t = fmaf(v[a], s_r[a * LP + c], t);
            o[c] = t;
        }
        store_row<LP, float>(z + (size_t)i * LP, o);
    }
}

template <int LP>
static cudaError_t orthonormalize_lp(int n, int l, float* z, const double* deg, double* part, int nb, float* rinv,
                                     cudaStream_t s) {
    for (int pass = 0; pass < 2; ++pass) {   // CholeskyQR2
        k_gram<LP><<<nb, kOrthoThreads, 0, s>>>(n, z, deg, part);
        k_chol_inv<LP><<<1, 64, 0, s>>>(part, nb, l, rinv);
        k_apply<LP><<<nb, kOrthoThreads, 0, s>>>(n, z, rinv);
    }
    return cudaGetLastError();
}

static cudaError_t orthonormalize(int LP, int n, int l, float* z, const double* deg, double* part, int nb,
                                  float* rinv, cudaStream_t s) {
    switch (LP) {
        case 1: return orthonormalize_lp<1>(n, l, z, deg, part, nb, rinv, s);
        case 2: return orthonormalize_lp<2>(n, l, z, deg, part, nb, rinv, s);
        case 4: return orthonormalize_lp<4>(n, l, z, deg, part, nb, rinv, s);
        default: return orthonormalize_lp<8>(n, l, z, deg, part, nb, rinv, s);
    }
}

// ---- Rayleigh-Ritz ---------------------------------------------------------------------------
// Per-block partial sums of the cross Gram sum_v d(v) a_v b_v^T (full LP x LP, row-major).
template <int LP>
__global__ void __launch_bounds__(kOrthoThreads) k_gram2(int n, const float* __restrict__ za,
                                                         const float* __restrict__ zb, const double* __restrict__ deg,
                                                         double* __restrict__ part) {
    constexpr int NT = LP * LP;
    __shared__ float s_w[kOrthoThreads / 32][NT];
    float acc[NT];
#pragma unroll
    for (int e = 0; e < NT; ++e) acc[e] = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float a[LP], b[LP];
        load_row<LP, float>(za + (size_t)i * LP, a);
        load_row<LP, float>(zb + (size_t)i * LP, b);
        const float d = (float)deg[i];
#pragma unroll
        for (int x = 0; x < LP; ++x) {
            const float dx = d * a[x];
#pragma unroll
            for (int y = 0; y < LP; ++y) acc[x * LP + y] = fmaf(dx, b[y], acc[x * LP + y]);
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < NT; ++e) {
        float x = acc[e];
        for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (lane == 0) s_w[wid][e] = x;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < NT; e += blockDim.x) {
        double t = 0.0;
        for (int w = 0; w < kOrthoThreads / 32; ++w) t += (double)s_w[w][e];
        part[(size_t)blockIdx.x * NT + e] = t;
    }
}

// One block: H = (G + G^T) / 2 over the leading l x l, eigenpairs by cyclic Jacobi (float64),
// sorted by decreasing value; each vector's sign fixed so that its largest component is
// positive.  Writes V (LP x LP floats, identity on the padding) and the values.
template <int LP>
__global__ void k_ritz(const double* __restrict__ part, int nb, int l, float* __restrict__ vout,
                       double* __restrict__ values) {
    constexpr int NT = LP * LP;
    __shared__ double s_g[NT];
    for (int e = threadIdx.x; e < NT; e += blockDim.x) {
        double t = 0.0;
        for (int q = 0; q < nb; ++q) t += part[(size_t)q * NT + e];
        s_g[e] = t;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double A[LP][LP], V[LP][LP];
    for (int a = 0; a < LP; ++a)
        for (int b = 0; b < LP; ++b) {
            A[a][b] = (a < l && b < l) ? 0.5 * (s_g[a * LP + b] + s_g[b * LP + a]) : 0.0;
            V[a][b] = a == b ? 1.0 : 0.0;
        }
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int a = 0; a < l; ++a)
            for (int b = 0; b < l; ++b) {
                tot += A[a][b] * A[a][b];
                if (a != b) off += A[a][b] * A[a][b];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < l - 1; ++p)
            for (int q = p + 1; q < l; ++q) {
                if (A[p][q] == 0.0) continue;
                const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                const double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(tt * tt + 1.0), sn = tt * c;
                for (int r = 0; r < l; ++r) {   // A <- J^T A J, V <- V J
                    const double arp = A[r][p], arq = A[r][q];
                    A[r][p] = c * arp - sn * arq;
                    A[r][q] = sn * arp + c * arq;
                }
                for (int r = 0; r < l; ++r) {
                    const double apr = A[p][r], aqr = A[q][r];
                    A[p][r] = c * apr - sn * aqr;
                    A[q][r] = sn * apr + c * aqr;
                }
                for (int r = 0; r < l; ++r) {
                    const double vrp = V[r][p], vrq = V[r][q];
                    V[r][p] = c * vrp - sn * vrq;
                    V[r][q] = sn * vrp + c * vrq;
                }
            }
    }
    int order[LP];
    for (int a = 0; a < LP; ++a) order[a] = a;
    for (int a = 0; a < l; ++a)   // selection sort by decreasing eigenvalue (stable in index)
        for (int b = a + 1; b < l; ++b)
            if (A[order[b]][order[b]] > A[order[a]][order[a]]) {
                const int t = order[a];
                order[a] = order[b];
                order[b] = t;
            }
    for (int a = 0; a < LP; ++a)
        for (int b = 0; b < LP; ++b) vout[a * LP + b] = (a == b && a >= l) ? 1.f : 0.f;
    for (int c = 0; c < l; ++c) {
        const int src = order[c];
        int big = 0;
        for (int r = 1; r < l; ++r)
            if (fabs(V[r][src]) > fabs(V[big][src])) big = r;
        const double sgn = V[big][src] < 0 ? -1.0 : 1.0;
        for (int r = 0; r < l; ++r) vout[r * LP + c] = (float)(sgn * V[r][src]);
        values[c] = A[src][src];
    }
}

// z_v <- z_v V for every row (full LP x LP matrix), in place.
template <int LP>
__global__ void __launch_bounds__(kOrthoThreads) k_apply_full(int n, float* __restrict__ z, const float* __restrict__ m) {
    __shared__ float s_m[LP * LP];
    for (int q = threadIdx.x; q < LP * LP; q += blockDim.x) s_m[q] = m[q];
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float v[LP], o[LP];
        load_row<LP, float>(z + (size_t)i * LP, v);
#pragma unroll
        for (int c = 0; c < LP; ++c) {
            float t = 0.f;
#pragma unroll
            for (int a = 0; a < LP; ++a) t = fmaf(v[a], s_m[a * LP + c], t);
            o[c] = t;
        }
        store_row<LP, float>(z + (size_t)i * LP, o);
    }
}

template <int LP>
static cudaError_t ritz_lp(int n, int l, float* z, const float* mz, const double* deg, double* part, int nb,
                           float* vmat, double* values, cudaStream_t s) {
    k_gram2<LP><<<nb, kOrthoThreads, 0, s>>>(n, z, mz, deg, part);
    k_ritz<LP><<<1, 64, 0, s>>>(part, nb, l, vmat, values);
    k_apply_full<LP><<<nb, kOrthoThreads, 0, s>>>(n, z, vmat);
    return cudaGetLastError();
}

}  // namespace fsc

using namespace fsc;

extern "C" fsc_status fsc_embed_orthogonal(const fsc_graph* gc, int l, int t, int every, uint64_t seed, float* emb,
                                           const fsc_embed_opts* opts, void* stream);

extern "C" fsc_status fsc_top_eigenvectors(const fsc_graph* gc, int l, int t, int every, uint64_t seed, float* emb,
                                           double* values, const fsc_embed_opts* opts, void* stream) {
    NvtxRange nvtx_range("fsc_top_eigenvectors");
    fsc_graph* g = const_cast<fsc_graph*>(gc);
    if (!g || !emb || !values || l < 1 || l > 128 || t < 0 || every < 1) return FSC_ERR_INVALID_ARG;
    fsc_status rc = fsc_embed_orthogonal(gc, l, t, every, seed, emb, opts, stream);
    if (rc != FSC_OK) return rc;
    if (l > 8) return ritz_wide(g, l, emb, values, as_stream(stream));
    const int LP = pad_l(l);
    const int n = (int)g->n;
    cudaStream_t s = as_stream(stream);
    long long nb = ((long long)n + kOrthoThreads - 1) / kOrthoThreads;
    const long long cap = (long long)device_props().num_sms * 8;
    if (nb > cap) nb = cap;
    if (nb < 1) nb = 1;
    const size_t part_bytes = ((size_t)nb * 64 * 8 + 255) & ~(size_t)255;
    char* scratch = nullptr;
    cudaError_t e = pool_malloc(reinterpret_cast<void**>(&scratch), part_bytes + 512, s);
    if (e != cudaSuccess) return cuda_status(e);
    double* part = reinterpret_cast<double*>(scratch);
    float* vmat = reinterpret_cast<float*>(scratch + part_bytes);
    double* dvals = reinterpret_cast<double*>(scratch + part_bytes + 256);
    do {
        // M Q in embedding coordinates: one power step of the basis into the workspace
        StepArgs a{};
        a.n = n;
        a.rp = g->row_ptr;
        a.col = g->col;
        a.w = g->w;
        a.invdeg = g->invdeg;
        a.col_off = g->col_off;
        a.max_row = g->max_row;
        a.zin = emb;
        a.zout = g->ws;
        const int G = choose_threads_per_row(g, opts ? opts->threads_per_row : 0, LP, (int)FSC_F32);
        if ((e = launch_step_f32(LP, G, g->w != nullptr, a, s)) != cudaSuccess) break;
        if ((e = long_rows_power(g, LP, 0, 0, a, s)) != cudaSuccess) break;
        const float* mz = static_cast<const float*>(g->ws);
        switch (LP) {
            case 1: e = ritz_lp<1>(n, l, emb, mz, g->deg, part, (int)nb, vmat, dvals, s); break;
            case 2: e = ritz_lp<2>(n, l, emb, mz, g->deg, part, (int)nb, vmat, dvals, s); break;
            case 4: e = ritz_lp<4>(n, l, emb, mz, g->deg, part, (int)nb, vmat, dvals, s); break;
            default: e = ritz_lp<8>(n, l, emb, mz, g->deg, part, (int)nb, vmat, dvals, s); break;
        }
        if (e != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(values, dvals, sizeof(double) * l, cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
        e = cudaStreamSynchronize(s);
    } while (0);
    pool_free(scratch, s);
    return e == cudaSuccess ? FSC_OK : cuda_status(e);
}

extern "C" fsc_status fsc_embed_orthogonal(const fsc_graph* gc, int l, int t, int every, uint64_t seed, float* emb,
                                           const fsc_embed_opts* opts, void* stream) {
    NvtxRange nvtx_range("fsc_embed_orthogonal");
    fsc_graph* g = const_cast<fsc_graph*>(gc);
    if (!g || !emb || l < 1 || l > 128 || t < 0 || every < 1) return FSC_ERR_INVALID_ARG;
    if (opts && opts->flags) return FSC_ERR_INVALID_ARG;
    const int LP = pad_l(l);
    if (reinterpret_cast<uintptr_t>(emb) % (size_t)(LP * 4 < 16 ? LP * 4 : 16)) return FSC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if (l > 8) return embed_orthogonal_wide(g, l, t, every, seed, emb, opts, s);
    const int n = (int)g->n;
    fsc_status rc = ensure_workspace(g, (size_t)n * LP * 4 + 256, s);
    if (rc != FSC_OK) return rc;
    long long nb = ((long long)n + kOrthoThreads - 1) / kOrthoThreads;
    const long long cap = (long long)device_props().num_sms * 8;
    if (nb > cap) nb = cap;
    if (nb < 1) nb = 1;
    char* scratch = nullptr;
    const size_t part_bytes = ((size_t)nb * 36 * 8 + 255) & ~(size_t)255;
    cudaError_t e = pool_malloc(reinterpret_cast<void**>(&scratch), part_bytes + 256, s);
    if (e != cudaSuccess) return cuda_status(e);
    double* part = reinterpret_cast<double*>(scratch);
    float* rinv = reinterpret_cast<float*>(scratch + part_bytes);
    float* buf[2];
    buf[t % 2] = emb;
    buf[(t + 1) % 2] = static_cast<float*>(g->ws);
    do {
        if ((e = launch_init_any(LP, n, l, seed, g->dinv, buf[0], (int)FSC_F32, s)) != cudaSuccess) break;
        if (opts && opts->ev_spmm_begin && (e = cudaEventRecord((cudaEvent_t)opts->ev_spmm_begin, s)) != cudaSuccess) break;
        StepArgs a{};
        a.n = n;
        a.rp = g->row_ptr;
        a.col = g->col;
        a.w = g->w;
        a.invdeg = g->invdeg;
        a.col_off = g->col_off;
        a.max_row = g->max_row;
        const int G = choose_threads_per_row(g, opts ? opts->threads_per_row : 0, LP, (int)FSC_F32);
        for (int it = 0; it < t && e == cudaSuccess; ++it) {
            a.zin = buf[it % 2];
            a.zout = buf[(it + 1) % 2];
            a.last = 0;
            if ((e = launch_step_f32(LP, G, g->w != nullptr, a, s)) != cudaSuccess) break;
            if ((e = long_rows_power(g, LP, 0, 0, a, s)) != cudaSuccess) break;
            if ((it + 1) % every == 0 || it == t - 1)
                e = orthonormalize(LP, n, l, buf[(it + 1) % 2], g->deg, part, (int)nb, rinv, s);
        }
        if (e == cudaSuccess && t == 0) e = orthonormalize(LP, n, l, emb, g->deg, part, (int)nb, rinv, s);
        if (e == cudaSuccess && opts && opts->ev_spmm_end) e = cudaEventRecord((cudaEvent_t)opts->ev_spmm_end, s);
    } while (0);
    pool_free(scratch, s);
    return e == cudaSuccess ? FSC_OK : cuda_status(e);
}
