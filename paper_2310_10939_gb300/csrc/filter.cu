// Learned polynomial filter: p(M) X = sum_{j=0..8} c_j T_j(A_hat) X with A_hat = 2M - I, chosen per
// graph by a small MLP fed 16 graph features.  Not in the paper: an extension that replaces the
// t power iterations of Algorithm 2; it is judged by the quantity Lemma 3.1 bounds,
// ||p(M) x_0 - P x_0|| with P the projector on the top-k eigenvectors of M.
//
// Everything runs in embedding coordinates z = D^-1/2 x, where D^-1/2 T_j(A_hat) D^1/2 =
// T_j(D^-1 A): T_0 = z, T_1 = D^-1 A z, T_{j+1} = 2 D^-1 A T_j - T_{j-1}, and the filtered block
// sum_j c_j T_j is already D^-1/2 p(M) X, the embedding of Algorithm 2.
//
// Features (computed on the device, no host round trip): log n, log mean degree, degree std /
// mean, log(max degree / mean), log k, log(n / k), l / 8, isolated fraction, and the Chebyshev
// moments mu_j = sum_c x_c^T T_j(A_hat) x_c / sum_c x_c^T x_c (j = 1..8) of the start block.  In
// z coordinates x^T T_j x = <z, T_j z>_D (D-weighted), and the product rule T_a T_b =
// (T_{a+b} + T_{|a-b|}) / 2 gives mu_{2j} = 2 <T_j, T_j>_D / <T_0, T_0>_D - 1 and
// mu_{2j+1} = 2 <T_{j+1}, T_j>_D / <T_0, T_0>_D - mu_1, so the moments come from inner products
// fused into the first four recurrence steps.
//
// MLP (float32): h1 = gelu(W1 f + b1), h2 = gelu(W2 h1 + b2), c = W3 h2 + b3, 16 -> 64 -> 64 -> 9,
// gelu(x) = x * Phi(x); parameters flattened as W1 (64x16 row-major), b1, W2 (64x64), b2,
// W3 (9x64), b3: 5833 floats.  Training minimises the per-graph quadratic
// c^T Gn c - 2 bn^T c + 1 (= ||sum_j c_j K_j - PX||^2 / ||PX||^2) with Adam.
#include <math.h>

#include "longrows.cuh"

namespace fsc {

constexpr int FDEG = 8, NFEAT = 16, HID = 64, NCOEF = FDEG + 1;
constexpr int OW1 = 0, OB1 = OW1 + HID * NFEAT, OW2 = OB1 + HID, OB2 = OW2 + HID * HID, OW3 = OB2 + HID,
              OB3 = OW3 + NCOEF * HID, NPARAM = OB3 + NCOEF;
static_assert(NPARAM == 5833, "parameter count");

cudaError_t launch_init_any(int LP, int n, int l, unsigned long long seed, const float* dinv, void* out, int store,
                            cudaStream_t s);
int choose_threads_per_row(const fsc_graph* g, int requested, int LP, int store);
fsc_status ensure_workspace(fsc_graph* g, size_t bytes, cudaStream_t s);

// ---- Chebyshev step -----------------------------------------------------------------------------
template <int LP, typename TS, int G, int U, bool W>
__global__ void __launch_bounds__(256)
k_cheb_step(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const float* __restrict__ w,
            const float* __restrict__ invdeg, const double* __restrict__ deg, const TS* __restrict__ cur,
            const TS* __restrict__ prev, TS* __restrict__ out, float* __restrict__ mom, long long col_off, int first,
            long long max_row) {
    constexpr int RPW = 32 / G;
    const int lane = threadIdx.x & 31, sub = lane % G, grp = lane / G, wid = threadIdx.x >> 5;
    float s_oc = 0.f, s_oo = 0.f, s_cc = 0.f;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long base = warp * RPW; base < n; base += nwarps * RPW) {
        const long long row = base + grp;
        const bool active = row < n;
        float acc[LP];
        const bool own = row_gather<LP, TS, G, U, W, true>(active, row, sub, rp, col, w, cur, col_off, n, max_row, acc);
        if (own && sub == 0) {
            const float id = invdeg[row];
            float y[LP];
            if (first) {
#pragma unroll
                for (int c = 0; c < LP; ++c) y[c] = id * acc[c];
            } else {
                float pv[LP];
                load_row<LP, TS>(prev + (size_t)row * LP, pv);
#pragma unroll
                for (int c = 0; c < LP; ++c) y[c] = fmaf(2.0f * id, acc[c], -pv[c]);
            }
            store_row<LP, TS>(out + (size_t)row * LP, y);
            if (mom) {
                float cv[LP];
                load_row<LP, TS>(cur + (size_t)row * LP, cv);
                const float d = (float)deg[row];
#pragma unroll
                for (int c = 0; c < LP; ++c) {
                    const float yr = to_f32(from_f32<TS>(y[c]));   // the value T_{j+1} holds
                    s_oc = fmaf(d * yr, cv[c], s_oc);
                    s_oo = fmaf(d * yr, yr, s_oo);
                    s_cc = fmaf(d * cv[c], cv[c], s_cc);
                }
            }
        }
    }
    if (mom) {
        __shared__ float s_r[3][8];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            s_oc += __shfl_xor_sync(0xffffffffu, s_oc, off);
            s_oo += __shfl_xor_sync(0xffffffffu, s_oo, off);
            s_cc += __shfl_xor_sync(0xffffffffu, s_cc, off);
        }
        if (lane == 0) {
            s_r[0][wid] = s_oc;
            s_r[1][wid] = s_oo;
            s_r[2][wid] = s_cc;
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            float v = 0.f;
            for (int q = 0; q < 8; ++q) v += s_r[threadIdx.x][q];
            mom[3 * blockIdx.x + threadIdx.x] = v;
        }
    }
}

struct ChebArgs {
    int n;
    const int64_t* rp;
    const int32_t* col;
    const float* w;
    const float* invdeg;
    const double* deg;
    const void* cur;
    const void* prev;
    void* out;
    float* mom;
    long long col_off;
    int first;
    long long max_row;
};

template <int LP, typename TS, int G, int U, bool W>
static cudaError_t launch_cheb(const ChebArgs& a, int blocks, cudaStream_t s) {
    k_cheb_step<LP, TS, G, U, W><<<blocks, 256, 0, s>>>(a.n, a.rp, a.col, a.w, a.invdeg, a.deg,
                                                        static_cast<const TS*>(a.cur), static_cast<const TS*>(a.prev),
                                                        static_cast<TS*>(a.out), a.mom, a.col_off, a.first,
                                                        a.max_row);
    return cudaGetLastError();
}

template <int LP, typename TS, bool W>
static cudaError_t launch_cheb_g(int G, const ChebArgs& a, int blocks, cudaStream_t s) {
    switch (G) {
        case 4: return launch_cheb<LP, TS, 4, 4, W>(a, blocks, s);
        case 8: return launch_cheb<LP, TS, 8, 4, W>(a, blocks, s);
        case 16: return launch_cheb<LP, TS, 16, 2, W>(a, blocks, s);
        default: return launch_cheb<LP, TS, 32, 2, W>(a, blocks, s);
    }
}

template <typename TS>
static cudaError_t launch_cheb_any(int LP, int G, bool weighted, const ChebArgs& a, int blocks, cudaStream_t s) {
    switch (LP) {
        case 1: return weighted ? launch_cheb_g<1, TS, true>(G, a, blocks, s) : launch_cheb_g<1, TS, false>(G, a, blocks, s);
        case 2: return weighted ? launch_cheb_g<2, TS, true>(G, a, blocks, s) : launch_cheb_g<2, TS, false>(G, a, blocks, s);
        case 4: return weighted ? launch_cheb_g<4, TS, true>(G, a, blocks, s) : launch_cheb_g<4, TS, false>(G, a, blocks, s);
        default: return weighted ? launch_cheb_g<8, TS, true>(G, a, blocks, s) : launch_cheb_g<8, TS, false>(G, a, blocks, s);
    }
}

// The Chebyshev step of the long rows (longrows.cu's decomposition): their segments' partial sums
// added in order, the step's epilogue, and their moment terms summed in a fixed order by one block
// into the launch's extra moment slot.
template <int LP, typename TS>
__global__ void __launch_bounds__(256)
k_long_cheb(int64_t nl, const int64_t* __restrict__ rows, const int32_t* __restrict__ seg0,
            const int32_t* __restrict__ nseg, const float* __restrict__ part, const float* __restrict__ invdeg,
            const double* __restrict__ deg, const TS* __restrict__ cur, const TS* __restrict__ prev,
            TS* __restrict__ out, float* __restrict__ mom_slot, int first) {
    float s_oc = 0.f, s_oo = 0.f, s_cc = 0.f;
    for (int64_t h = threadIdx.x; h < nl; h += blockDim.x) {
        const int64_t row = rows[h];
        float acc[LP], y[LP];
        long_row_sum(h, seg0, nseg, part, LP, acc);
        const float id = invdeg[row];
        if (first) {
#pragma unroll
            for (int c = 0; c < LP; ++c) y[c] = id * acc[c];
        } else {
            float pv[LP];
            load_row<LP, TS>(prev + (size_t)row * LP, pv);
#pragma unroll
            for (int c = 0; c < LP; ++c) y[c] = fmaf(2.0f * id, acc[c], -pv[c]);
        }
        store_row<LP, TS>(out + (size_t)row * LP, y);
        if (mom_slot) {
            float cv[LP];
            load_row<LP, TS>(cur + (size_t)row * LP, cv);
            const float d = (float)deg[row];
#pragma unroll
            for (int c = 0; c < LP; ++c) {
                const float yr = to_f32(from_f32<TS>(y[c]));
                s_oc = fmaf(d * yr, cv[c], s_oc);
                s_oo = fmaf(d * yr, yr, s_oo);
                s_cc = fmaf(d * cv[c], cv[c], s_cc);
            }
        }
    }
    if (mom_slot) {
        __shared__ float s_r[3][8];
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            s_oc += __shfl_xor_sync(0xffffffffu, s_oc, off);
            s_oo += __shfl_xor_sync(0xffffffffu, s_oo, off);
            s_cc += __shfl_xor_sync(0xffffffffu, s_cc, off);
        }
        if (lane == 0) {
            s_r[0][wid] = s_oc;
            s_r[1][wid] = s_oo;
            s_r[2][wid] = s_cc;
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            float v = 0.f;
            for (int q = 0; q < 8; ++q) v += s_r[threadIdx.x][q];
            mom_slot[threadIdx.x] = v;
        }
    }
}

template <int LP, typename TS>
static cudaError_t long_cheb_lp(const fsc_graph* g, const ChebArgs& a, float* mom_slot, cudaStream_t s) {
    seg_partial_launch<LP, TS>(g, static_cast<const TS*>(a.cur), s);
    k_long_cheb<LP, TS><<<1, 256, 0, s>>>(g->n_long, g->long_rows, g->long_seg0, g->long_nseg, g->seg_part, g->invdeg,
                                          g->deg, static_cast<const TS*>(a.cur), static_cast<const TS*>(a.prev),
                                          static_cast<TS*>(a.out), mom_slot, a.first);
    return cudaGetLastError();
}

template <typename TS>
static cudaError_t long_cheb(const fsc_graph* g, int LP, const ChebArgs& a, float* mom_slot, cudaStream_t s) {
    if (g->n_long == 0) return cudaSuccess;
    switch (LP) {
        case 1: return long_cheb_lp<1, TS>(g, a, mom_slot, s);
        case 2: return long_cheb_lp<2, TS>(g, a, mom_slot, s);
        case 4: return long_cheb_lp<4, TS>(g, a, mom_slot, s);
        default: return long_cheb_lp<8, TS>(g, a, mom_slot, s);
    }
}


// ---- the MLP --------------------------------------------------------------------------------------
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// Forward pass of one feature vector by a block of >= 64 threads; f, a1, h1, a2, h2, c in shared memory.
__device__ void mlp_forward_block(const float* __restrict__ P, const float* f, float* a1, float* h1, float* a2,
                                  float* h2, float* c) {
    const int t = threadIdx.x;
    if (t < HID) {
        float v = P[OB1 + t];
#pragma unroll
        for (int i = 0; i < NFEAT; ++i) v = fmaf(P[OW1 + t * NFEAT + i], f[i], v);
        a1[t] = v;
        h1[t] = gelu(v);
    }
    __syncthreads();
    if (t < HID) {
        float v = P[OB2 + t];
        for (int i = 0; i < HID; ++i) v = fmaf(P[OW2 + t * HID + i], h1[i], v);
        a2[t] = v;
        h2[t] = gelu(v);
    }
    __syncthreads();
    if (t < NCOEF) {
        float v = P[OB3 + t];
        for (int i = 0; i < HID; ++i) v = fmaf(P[OW3 + t * HID + i], h2[i], v);
        c[t] = v;
    }
    __syncthreads();
}

// Features from the degree statistics and the fused moment sums, then the coefficients.
__global__ void __launch_bounds__(256) k_filter_coeffs(const float* __restrict__ mom, int nb, double n, double vol,
                                                       double sumsq, double dmax, double niso, int k, int l,
                                                       const float* __restrict__ params,
                                                       const float* __restrict__ override_c, float* feats_out,
                                                       float* coeffs_out) {
    __shared__ double s_sum[12];
    __shared__ float f[NFEAT], a1[HID], h1[HID], a2[HID], h2[HID], c[NCOEF];
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    for (int q = wid; q < 12; q += 8) {      // 4 steps x (oc, oo, cc), summed over the blocks in float64
        double v = 0.0;
        for (int b = lane; b < nb; b += 32) v += (double)mom[(size_t)(q / 3) * nb * 3 + 3 * b + (q % 3)];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) s_sum[q] = v;
    }
    __syncthreads();
    if (t == 0) {
        const double S00 = s_sum[2];
        const double S10 = s_sum[0], S11 = s_sum[1], S21 = s_sum[3], S22 = s_sum[4];
        const double S32 = s_sum[6], S33 = s_sum[7], S43 = s_sum[9], S44 = s_sum[10];
        const double mu1 = S10 / S00;
        const double mean = vol / n;
        const double var = sumsq / n - mean * mean;
        f[0] = (float)log(n);
        f[1] = (float)log(mean);
        f[2] = (float)(sqrt(var > 0.0 ? var : 0.0) / mean);
        f[3] = (float)log(dmax / mean);
        f[4] = (float)log((double)k);
        f[5] = (float)log(n / (double)k);
        f[6] = (float)l / 8.0f;
        f[7] = (float)(niso / n);
        f[8] = (float)mu1;
        f[9] = (float)(2.0 * S11 / S00 - 1.0);
        f[10] = (float)(2.0 * S21 / S00 - mu1);
        f[11] = (float)(2.0 * S22 / S00 - 1.0);
        f[12] = (float)(2.0 * S32 / S00 - mu1);
        f[13] = (float)(2.0 * S33 / S00 - 1.0);
        f[14] = (float)(2.0 * S43 / S00 - mu1);
        f[15] = (float)(2.0 * S44 / S00 - 1.0);
    }
    __syncthreads();
    if (override_c) {
        if (t < NCOEF) c[t] = override_c[t];
        __syncthreads();
    } else {
        mlp_forward_block(params, f, a1, h1, a2, h2, c);
    }
    if (t < NFEAT && feats_out) feats_out[t] = f[t];
    if (t < NCOEF) coeffs_out[t] = c[t];
}

template <int LP, typename TS>
__global__ void __launch_bounds__(256) k_cheb_combine(int n, const TS* __restrict__ T, size_t stride,
                                                      const float* __restrict__ coeffs, const double* __restrict__ deg,
                                                      float* __restrict__ out, double* __restrict__ energy) {
    __shared__ float s_c[NCOEF];
    __shared__ float s_e[8];
    if (threadIdx.x < NCOEF) s_c[threadIdx.x] = coeffs[threadIdx.x];
    __syncthreads();
    float e_loc = 0.f;   // sum over this thread's rows of d(v) |y_v|^2 (x-space energy)
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float acc[LP];
#pragma unroll
        for (int c = 0; c < LP; ++c) acc[c] = 0.f;
#pragma unroll
        for (int j = 0; j < NCOEF; ++j) {
            float v[LP];
            load_row<LP, TS>(T + j * stride + (size_t)i * LP, v);
#pragma unroll
            for (int c = 0; c < LP; ++c) acc[c] = fmaf(s_c[j], v[c], acc[c]);
        }
        store_row<LP, float>(out + (size_t)i * LP, acc);
        if (energy) {
            float q = 0.f;
#pragma unroll
            for (int c = 0; c < LP; ++c) q = fmaf(acc[c], acc[c], q);
            e_loc = fmaf((float)deg[i], q, e_loc);
        }
    }
    if (energy) {
        for (int off = 16; off > 0; off >>= 1) e_loc += __shfl_xor_sync(0xffffffffu, e_loc, off);
        if ((threadIdx.x & 31) == 0) s_e[threadIdx.x >> 5] = e_loc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += (double)s_e[w];
            atomicAdd(energy, t);
        }
    }
}

template <typename TS>
static cudaError_t launch_combine(int LP, unsigned blocks, int n, const void* T, size_t stride, const float* coeffs,
                                  const double* deg, float* out, double* energy, cudaStream_t s) {
    const TS* t = static_cast<const TS*>(T);
    switch (LP) {
        case 1: k_cheb_combine<1, TS><<<blocks, 256, 0, s>>>(n, t, stride, coeffs, deg, out, energy); break;
        case 2: k_cheb_combine<2, TS><<<blocks, 256, 0, s>>>(n, t, stride, coeffs, deg, out, energy); break;
        case 4: k_cheb_combine<4, TS><<<blocks, 256, 0, s>>>(n, t, stride, coeffs, deg, out, energy); break;
        default: k_cheb_combine<8, TS><<<blocks, 256, 0, s>>>(n, t, stride, coeffs, deg, out, energy); break;
    }
    return cudaGetLastError();
}

// ---- training: one block of 64 threads per graph of the minibatch ------------------------------------
__global__ void __launch_bounds__(64) k_mlp_grad(const float* __restrict__ P, const float* __restrict__ F,
                                                 const float* __restrict__ Gn, const float* __restrict__ bn, int B,
                                                 float* __restrict__ grad, float* __restrict__ loss_sum) {
    __shared__ float f[NFEAT], a1[HID], h1[HID], a2[HID], h2[HID], c[NCOEF], dc[NCOEF], da2[HID];
    const int g = blockIdx.x, t = threadIdx.x;
    if (t < NFEAT) f[t] = F[(size_t)g * NFEAT + t];
    __syncthreads();
    mlp_forward_block(P, f, a1, h1, a2, h2, c);
    const float* G = Gn + (size_t)g * NCOEF * NCOEF;
    const float* b = bn + (size_t)g * NCOEF;
    const float invB = 1.0f / (float)B;
    if (t < NCOEF) {
        float v = 0.f;
        for (int j = 0; j < NCOEF; ++j) v = fmaf(G[t * NCOEF + j], c[j], v);
        dc[t] = 2.0f * (v - b[t]) * invB;
    }
    if (t == 0 && loss_sum) {
        float q = 1.0f;
        for (int i = 0; i < NCOEF; ++i) {
            float gi = 0.f;
            for (int j = 0; j < NCOEF; ++j) gi = fmaf(G[i * NCOEF + j], c[j], gi);
            q += c[i] * gi - 2.0f * b[i] * c[i];
        }
        atomicAdd(loss_sum, q * invB);
    }
    __syncthreads();
    // layer 3
    for (int q = 0; q < NCOEF; ++q) atomicAdd(&grad[OW3 + q * HID + t], dc[q] * h2[t]);
    if (t < NCOEF) atomicAdd(&grad[OB3 + t], dc[t]);
    float dh2 = 0.f;
    for (int q = 0; q < NCOEF; ++q) dh2 = fmaf(P[OW3 + q * HID + t], dc[q], dh2);
    const float d2 = dh2 * gelu_grad(a2[t]);
    da2[t] = d2;
    __syncthreads();
    // layer 2
    for (int i = 0; i < HID; ++i) atomicAdd(&grad[OW2 + t * HID + i], d2 * h1[i]);
    atomicAdd(&grad[OB2 + t], d2);
    float dh1 = 0.f;
    for (int r = 0; r < HID; ++r) dh1 = fmaf(P[OW2 + r * HID + t], da2[r], dh1);
    const float d1 = dh1 * gelu_grad(a1[t]);
    // layer 1
    for (int i = 0; i < NFEAT; ++i) atomicAdd(&grad[OW1 + t * NFEAT + i], d1 * f[i]);
    atomicAdd(&grad[OB1 + t], d1);
}

__global__ void k_adam(float* __restrict__ P, float* __restrict__ grad, float* __restrict__ m, float* __restrict__ v,
                       float lr, float beta1, float beta2, float eps, float wd, float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const float g = grad[i] + wd * P[i];
    const float mi = beta1 * m[i] + (1.0f - beta1) * g;
    const float vi = beta2 * v[i] + (1.0f - beta2) * g * g;
    m[i] = mi;
    v[i] = vi;
    P[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    grad[i] = 0.f;
}

__global__ void __launch_bounds__(64) k_mlp_forward(const float* __restrict__ P, const float* __restrict__ F, int B,
                                                    float* __restrict__ out) {
    __shared__ float f[NFEAT], a1[HID], h1[HID], a2[HID], h2[HID], c[NCOEF];
    const int g = blockIdx.x, t = threadIdx.x;
    if (t < NFEAT) f[t] = F[(size_t)g * NFEAT + t];
    __syncthreads();
    mlp_forward_block(P, f, a1, h1, a2, h2, c);
    if (t < NCOEF) out[(size_t)g * NCOEF + t] = c[t];
}

static bool is_aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

FSC_BOUNDS_READER(filter)

// kmeans.cu: fsc_kmeans (rows of <= 8 floats, no centroids or seeds) whose launches return at once
// when the energy guard rejects the embedding
fsc_status kmeans_guarded(const float* emb, int64_t n, int l, int ld, int k, uint64_t seed, int max_iter,
                          int32_t* labels, fsc_kmeans_stats* stats, const double* guard, double guard_thr,
                          cudaStream_t s);

}  // namespace fsc

using namespace fsc;

extern "C" fsc_status fsc_mlp_forward(const float* params, const float* feats, int batch, float* coeffs, void* stream) {
    if (!params || !feats || !coeffs || batch < 1) return FSC_ERR_INVALID_ARG;
    k_mlp_forward<<<batch, 64, 0, as_stream(stream)>>>(params, feats, batch, coeffs);
    FSC_CUDA(cudaGetLastError());
    return FSC_OK;
}

extern "C" fsc_status fsc_mlp_train_step(float* params, float* grad, float* adam_m, float* adam_v, int step, float lr,
                                         float weight_decay, const float* feats, const float* Gn, const float* bn,
                                         int batch, float* loss_out, int apply_update, void* stream) {
    if (!params || !grad || !feats || !Gn || !bn || batch < 1 || step < 1) return FSC_ERR_INVALID_ARG;
    if (apply_update && (!adam_m || !adam_v)) return FSC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    if (loss_out) FSC_CUDA(cudaMemsetAsync(loss_out, 0, sizeof(float), s));
    k_mlp_grad<<<batch, 64, 0, s>>>(params, feats, Gn, bn, batch, grad, loss_out);
    FSC_CUDA(cudaGetLastError());
    if (apply_update) {
        const float b1 = 0.9f, b2 = 0.999f;
        const float bc1 = 1.0f - powf(b1, (float)step), bc2 = 1.0f - powf(b2, (float)step);
        k_adam<<<(NPARAM + 255) / 256, 256, 0, s>>>(params, grad, adam_m, adam_v, lr, b1, b2, 1e-8f, weight_decay,
                                                     bc1, bc2);
        FSC_CUDA(cudaGetLastError());
    }
    return FSC_OK;
}

extern "C" fsc_status fsc_filter_embed(const fsc_graph* gc, int l, int k, uint64_t seed, fsc_dtype store,
                                       const float* params, const float* coeffs_override, float* emb, float* feats_out,
                                       float* coeffs_out, double* energy_out, const fsc_embed_opts* opts,
                                       void* stream) {
    NvtxRange nvtx_range("fsc_filter_embed");
    fsc_graph* g = const_cast<fsc_graph*>(gc);
    if (!g || !emb || l < 1 || l > 8 || k < 1 || (int64_t)k > g->n ||
        (store != FSC_F32 && store != FSC_BF16 && store != FSC_F16))
        return FSC_ERR_INVALID_ARG;
    if (!params && !coeffs_override) return FSC_ERR_INVALID_ARG;
    const int LP = pad_l(l);
    if (!is_aligned(emb, (size_t)(LP * 4 < 16 ? LP * 4 : 16))) return FSC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    const int n = (int)g->n;
    const size_t es = store == FSC_F32 ? 4 : 2;
    const size_t blk = ((size_t)n * LP * es + 255) & ~(size_t)255;
    const int G = choose_threads_per_row(g, opts ? opts->threads_per_row : 0, LP, (int)store);
    const int RPW = 32 / G;
    long long blocks = (((long long)n + RPW - 1) / RPW + 7) / 8;
    const long long cap = (long long)device_props().num_sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    // workspace: 9 basis blocks | 4 x 3 x (blocks + 1) moment sums (the last slot of each launch holds
    // the long rows' terms) | coefficients (16) | features (16)
    const long long mslots = blocks + 1;
    const size_t mom_bytes = (size_t)4 * 3 * mslots * 4;
    fsc_status rc = ensure_workspace(g, NCOEF * blk + mom_bytes + 256, s);
    if (rc != FSC_OK) return rc;
    char* ws = static_cast<char*>(g->ws);
    float* mom = reinterpret_cast<float*>(ws + NCOEF * blk);
    float* coeffs = reinterpret_cast<float*>(ws + NCOEF * blk + mom_bytes);
    // the side stream that computes the coefficients once the moments are in (after the fourth
    // step), beside the later steps; the combination waits for it
    if (!g->side) {
        FSC_CUDA(cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking));
        FSC_CUDA(cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming));
        FSC_CUDA(cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming));
    }
    FSC_CUDA(launch_init_any(LP, n, l, seed, g->dinv, ws, (int)store, s));
    FSC_CUDA(cudaMemsetAsync(mom, 0, mom_bytes, s));
    if (opts && opts->ev_spmm_begin) FSC_CUDA(cudaEventRecord((cudaEvent_t)opts->ev_spmm_begin, s));
    ChebArgs a{};
    a.max_row = g->max_row;
    a.n = n;
    a.rp = g->row_ptr;
    a.col = g->col;
    a.w = g->w;
    a.invdeg = g->invdeg;
    a.deg = g->deg;
    a.col_off = g->col_off;
    for (int j = 0; j < FDEG; ++j) {
        a.cur = ws + (size_t)j * blk;
        a.prev = j > 0 ? ws + (size_t)(j - 1) * blk : nullptr;
        a.out = ws + (size_t)(j + 1) * blk;
        a.mom = j < 4 ? mom + (size_t)j * 3 * mslots : nullptr;
        a.first = j == 0;
        float* mslot = j < 4 ? mom + (size_t)j * 3 * mslots + 3 * blocks : nullptr;
        if (store == FSC_F32) {
            FSC_CUDA(launch_cheb_any<float>(LP, G, g->w != nullptr, a, (int)blocks, s));
            FSC_CUDA(long_cheb<float>(g, LP, a, mslot, s));
        } else if (store == FSC_F16) {
            FSC_CUDA(launch_cheb_any<__half>(LP, G, g->w != nullptr, a, (int)blocks, s));
            FSC_CUDA(long_cheb<__half>(g, LP, a, mslot, s));
        } else {
            FSC_CUDA(launch_cheb_any<__nv_bfloat16>(LP, G, g->w != nullptr, a, (int)blocks, s));
            FSC_CUDA(long_cheb<__nv_bfloat16>(g, LP, a, mslot, s));
        }
        if (j == 3) {   // the moments are complete: the coefficients on the side stream
            static_assert(FDEG > 4, "the coefficients are formed after the fourth step");
            FSC_CUDA(cudaEventRecord(g->ev_fork, s));
            FSC_CUDA(cudaStreamWaitEvent(g->side, g->ev_fork, 0));
            k_filter_coeffs<<<1, 256, 0, g->side>>>(mom, (int)mslots, (double)n, g->volume, g->deg_sumsq, g->deg_max,
                                                    (double)g->n_isolated, k, l, params, coeffs_override, feats_out,
                                                    coeffs);
            FSC_CUDA(cudaGetLastError());
            FSC_CUDA(cudaEventRecord(g->ev_join, g->side));
        }
    }
    if (opts && opts->ev_spmm_end) FSC_CUDA(cudaEventRecord((cudaEvent_t)opts->ev_spmm_end, s));
    FSC_CUDA(cudaStreamWaitEvent(s, g->ev_join, 0));   // the coefficients
    long long cb = ((long long)n + 255) / 256;
    if (cb > cap * 2) cb = cap * 2;
    const size_t stride = blk / es;
    if (energy_out) FSC_CUDA(cudaMemsetAsync(energy_out, 0, sizeof(double), s));
    if (store == FSC_F32) FSC_CUDA(launch_combine<float>(LP, (unsigned)cb, n, ws, stride, coeffs, g->deg, emb, energy_out, s));
    else if (store == FSC_F16) FSC_CUDA(launch_combine<__half>(LP, (unsigned)cb, n, ws, stride, coeffs, g->deg, emb, energy_out, s));
    else FSC_CUDA(launch_combine<__nv_bfloat16>(LP, (unsigned)cb, n, ws, stride, coeffs, g->deg, emb, energy_out, s));
    if (coeffs_out) FSC_CUDA(cudaMemcpyAsync(coeffs_out, coeffs, NCOEF * sizeof(float), cudaMemcpyDeviceToDevice, s));
    return FSC_OK;
}

extern "C" fsc_status fsc_cluster_filtered(const fsc_graph* g, int k, int l, uint64_t seed, fsc_dtype store,
                                           const float* params, int max_iter, int32_t* labels,
                                           fsc_kmeans_stats* stats, fsc_filter_report* report,
                                           const fsc_embed_opts* opts, void* stream) {
    NvtxRange nvtx_range("fsc_cluster_filtered");
    if (!g || !labels || !params || l < 1 || l > 8 || k < 1 || (int64_t)k > g->n) return FSC_ERR_INVALID_ARG;
    const int LP = pad_l(l);
    cudaStream_t s = as_stream(stream);
    const bool guard = !(opts && (opts->flags & FSC_FILTER_NO_FALLBACK));
    fsc_embed_opts eo{};
    if (opts) eo = *opts;
    eo.flags = 0;
    float* emb = nullptr;
    cudaError_t e = pool_malloc(reinterpret_cast<void**>(&emb), (size_t)g->n * LP * 4 + 256, s);
    if (e != cudaSuccess) return cuda_status(e);
    double* d_energy = reinterpret_cast<double*>(reinterpret_cast<char*>(emb) + (((size_t)g->n * LP * 4 + 127) & ~(size_t)127));
    fsc_kmeans_stats local{};
    fsc_filter_report rep{};
    rep.threshold = 1.25 + 3.0 * sqrt(2.0 / ((double)l * (double)k));
    fsc_status rc = fsc_filter_embed(g, l, k, seed, store, params, nullptr, emb, nullptr, nullptr, d_energy, &eo, stream);
    // k-means runs on the filtered embedding straight away (no host round trip between the two);
    // the guard's energy is read once k-means has synchronised, and when it calls for the fallback
    // the plain embedding and its k-means replace the results.  The k-means launches read the
    // energy themselves and return at once when the guard will reject the embedding (the same test
    // as below), so a fallback costs the filter and the plain method, not a wasted k-means too
    // (a graph without a spectral gap falls back on every call).
    const bool guarded_ok = guard && g->n <= 2147483647LL && k <= 1024 && (int64_t)k * LP <= 4096 && max_iter >= 1;
    if (rc == FSC_OK)
        rc = guarded_ok ? kmeans_guarded(emb, g->n, l, LP, k, seed, max_iter, labels, stats ? stats : &local, d_energy,
                                         rep.threshold, s)
                        : fsc_kmeans(emb, g->n, l, LP, k, seed, max_iter, labels, nullptr, nullptr, stats ? stats : &local,
                                     stream);
    if (rc == FSC_OK) {
        double energy = 0.0;
        if ((e = cudaMemcpyAsync(&energy, d_energy, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            rc = cuda_status(e);
        rep.energy_ratio = energy / ((double)l * (double)k);
    }
    if (rc == FSC_OK && guard && !(rep.energy_ratio <= rep.threshold)) {
        int lp = 0, t = 0;
        fsc_default_params(g->n, k, 0, &lp, &t);
        rep.fallback = 1;
        rep.fallback_t = t;
        fsc_embed_opts po = eo;
        po.flags = store == FSC_F32 ? 0u : FSC_EMBED_RESCALE;
        rc = fsc_embed(g, l, t, seed, store == FSC_F32 ? FSC_F32 : FSC_BF16, emb, &po, stream);
        if (rc == FSC_OK)
            rc = fsc_kmeans(emb, g->n, l, LP, k, seed, max_iter, labels, nullptr, nullptr, stats ? stats : &local,
                            stream);
    }
    cudaError_t ef = pool_free(emb, s);
    if (rc == FSC_OK && ef != cudaSuccess) rc = cuda_status(ef);
    if (rc == FSC_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) rc = cuda_status(e);
    if (report) *report = rep;
    return rc;
}
