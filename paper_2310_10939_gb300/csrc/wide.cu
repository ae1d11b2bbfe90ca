// Wide blocks: orthogonal iteration and Rayleigh-Ritz for l = 9 .. 128 columns (l_pad = 16, 32,
// 64 or 128 float32 per row), the block sizes of the "PM k Vectors" and "k Eigenvectors"
// variants the paper compares against (Sec. 4) when k > 8.
//
// Same arithmetic as the l <= 8 kernels of ortho.cu, laid out for rows of 64 .. 512 bytes:
//  * power step (Algorithm 1 body, embedding coordinates z = D^-1/2 x):
//        z_out[i] = (z_in[i] + (1/d_i) sum_j w_ij z_in[j]) / 2,
//    one group of l_pad/4 lanes per row, each lane owning 4 columns (16 bytes), so every
//    neighbour row is gathered as one coalesced l_pad*4-byte access; the group reads the row's
//    column indices l_pad/4 at a time and broadcasts them by shuffles;
//  * Gram G = A^T D B (A = B for orthonormalising, B = M A for Ritz): 16 x 16 threads each own an
//    (l_pad/16)^2 tile of G; rows are staged 32 at a time in shared memory; float32 products
//    summed over 32 rows, then added into float64 per thread; float64 per block in fixed order;
//  * Cholesky G = R^T R and R^-1 in float64 by one block (a column whose pivot falls below 1e-14
//    of the largest diagonal entry is dependent and comes out zero, as for l <= 8);
//  * Z <- Z M (M = R^-1, or the Ritz vectors V) with M in shared memory, sums in column order;
//  * the l x l Ritz problem H = Q^T M Q by parallel cyclic Jacobi in float64: each step rotates
//    l/2 disjoint index pairs at once (round-robin pairing), which commute; sweeps stop when the
//    off-diagonal mass is below 1e-30 of the total, as the one-thread version for l <= 8 does.
#include <math.h>

#include "spmm.cuh"

namespace fsc {

fsc_status ensure_workspace(fsc_graph* g, size_t bytes, cudaStream_t s);

constexpr int kWideThreads = 256;

// ---- power step -------------------------------------------------------------------------------
template <int LP, bool W>
__global__ void __launch_bounds__(kWideThreads)
k_power_step_wide(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                  const float* __restrict__ w, const float* __restrict__ invdeg, const float* __restrict__ zin,
                  float* __restrict__ zout, long long col_off) {
    constexpr int L = LP / 4;          // lanes per row, 4 columns each
    constexpr int RPW = 32 / L;        // rows per warp
    const int lane = threadIdx.x & 31, sub = lane % L, grp = lane / L;
    const unsigned gmask = L == 32 ? 0xffffffffu : (((1u << L) - 1u) << (grp * L));
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long base = warp * RPW; base < n; base += nwarps * RPW) {
        const long long row = base + grp;
        if (row >= n) continue;                       // whole groups leave together
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        const int64_t s = rp[row], e = rp[row + 1];
        for (int64_t p = s; p < e; p += L) {
            const int cnt = (int)(e - p < L ? e - p : L);
            const int jl = sub < cnt ? (int)((long long)__ldg(col + p + sub) - col_off) : 0;
            const float wl = W ? (sub < cnt ? __ldg(w + p + sub) : 0.f) : 1.f;
            for (int q = 0; q < cnt; q += 4) {
                float4 v[4];
                float wq[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int src = q + u < cnt ? q + u : q;
                    int j = __shfl_sync(gmask, jl, src, L);
                    wq[u] = q + u < cnt ? (W ? __shfl_sync(gmask, wl, src, L) : 1.f) : 0.f;
                    if (!in_range(j, 0, n, BS_GATHER_WIDE)) {
                        j = 0;
                        wq[u] = 0.f;
                    }
                    v[u] = __ldg(reinterpret_cast<const float4*>(zin + (size_t)j * LP) + sub);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    acc.x = fmaf(wq[u], v[u].x, acc.x);
                    acc.y = fmaf(wq[u], v[u].y, acc.y);
                    acc.z = fmaf(wq[u], v[u].z, acc.z);
                    acc.w = fmaf(wq[u], v[u].w, acc.w);
                }
            }
        }
        const float4 self = __ldg(reinterpret_cast<const float4*>(zin + (size_t)row * LP) + sub);
        const float id = invdeg[row];
        float4 y;
        y.x = 0.5f * fmaf(id, acc.x, self.x);
        y.y = 0.5f * fmaf(id, acc.y, self.y);
        y.z = 0.5f * fmaf(id, acc.z, self.z);
        y.w = 0.5f * fmaf(id, acc.w, self.w);
        reinterpret_cast<float4*>(zout + (size_t)row * LP)[sub] = y;
    }
}

template <int LP>
static cudaError_t launch_power_wide(const fsc_graph* g, const float* zin, float* zout, cudaStream_t s) {
    constexpr int RPW = 32 / (LP / 4);
    long long blocks = (((long long)g->n + RPW - 1) / RPW + 7) / 8;
    const long long cap = (long long)device_props().num_sms * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (g->w)
        k_power_step_wide<LP, true><<<(unsigned)blocks, kWideThreads, 0, s>>>((int)g->n, g->row_ptr, g->col, g->w,
                                                                          g->invdeg, zin, zout, g->col_off);
    else
        k_power_step_wide<LP, false><<<(unsigned)blocks, kWideThreads, 0, s>>>((int)g->n, g->row_ptr, g->col, g->w,
                                                                           g->invdeg, zin, zout, g->col_off);
    return cudaGetLastError();
}

cudaError_t power_step_wide(int LP, const fsc_graph* g, const float* zin, float* zout, cudaStream_t s) {
    switch (LP) {
        case 16: return launch_power_wide<16>(g, zin, zout, s);
        case 32: return launch_power_wide<32>(g, zin, zout, s);
        case 64: return launch_power_wide<64>(g, zin, zout, s);
        case 128: return launch_power_wide<128>(g, zin, zout, s);
    }
    return cudaErrorInvalidValue;
}

// ---- Gram A^T D B, per-block float64 partials ------------------------------------------------------
constexpr int kGramRows = 32;   // rows staged per round

template <int LP>
__global__ void __launch_bounds__(kWideThreads, 1)
k_gram_wide(int n, const float* __restrict__ za, const float* __restrict__ zb, const double* __restrict__ deg,
            double* __restrict__ part) {
    constexpr int MT = LP / 16;              // each thread owns rows ty*MT.. and columns tx*MT.. of G
    constexpr int PAD = LP + 4;              // keeps 16-byte alignment, staggers the rows over banks
    __shared__ __align__(16) float s_a[kGramRows][PAD];
    __shared__ __align__(16) float s_b[kGramRows][PAD];
    __shared__ float s_d[kGramRows];
    const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
    float a32[MT][MT];
    double a64[MT][MT];
#pragma unroll
    for (int x = 0; x < MT; ++x)
#pragma unroll
        for (int y = 0; y < MT; ++y) a64[x][y] = 0.0;
    const long long ntile = ((long long)n + kGramRows - 1) / kGramRows;
    for (long long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const long long r0 = tile * kGramRows;
        __syncthreads();
        for (int q = tid; q < kGramRows * (LP / 4); q += kWideThreads) {
            const int r = q / (LP / 4), c4 = q % (LP / 4);
            const long long i = r0 + r;
            float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = va;
            if (i < n) {
                va = __ldg(reinterpret_cast<const float4*>(za + (size_t)i * LP) + c4);
                vb = __ldg(reinterpret_cast<const float4*>(zb + (size_t)i * LP) + c4);
            }
            *reinterpret_cast<float4*>(&s_a[r][c4 * 4]) = va;
            *reinterpret_cast<float4*>(&s_b[r][c4 * 4]) = vb;
        }
        if (tid < kGramRows) s_d[tid] = r0 + tid < n ? (float)deg[r0 + tid] : 0.f;
        __syncthreads();
#pragma unroll
        for (int x = 0; x < MT; ++x)
#pragma unroll
            for (int y = 0; y < MT; ++y) a32[x][y] = 0.f;
        for (int r = 0; r < kGramRows; ++r) {
            const float d = s_d[r];
            float av[MT], bv[MT];
#pragma unroll
            for (int x = 0; x < MT; ++x) av[x] = d * s_a[r][ty * MT + x];
#pragma unroll
            for (int y = 0; y < MT; ++y) bv[y] = s_b[r][tx * MT + y];
#pragma unroll
            for (int x = 0; x < MT; ++x)
#pragma unroll
                for (int y = 0; y < MT; ++y) a32[x][y] = fmaf(av[x], bv[y], a32[x][y]);
        }
#pragma unroll
        for (int x = 0; x < MT; ++x)
#pragma unroll
            for (int y = 0; y < MT; ++y) a64[x][y] += (double)a32[x][y];
    }
#pragma unroll
    for (int x = 0; x < MT; ++x)
#pragma unroll
        for (int y = 0; y < MT; ++y)
            part[(size_t)blockIdx.x * LP * LP + (size_t)(ty * MT + x) * LP + tx * MT + y] = a64[x][y];
}

static cudaError_t gram_wide(int LP, int n, const float* za, const float* zb, const double* deg, double* part, int nb,
                             cudaStream_t s) {
    switch (LP) {
        case 16: k_gram_wide<16><<<nb, kWideThreads, 0, s>>>(n, za, zb, deg, part); break;
        case 32: k_gram_wide<32><<<nb, kWideThreads, 0, s>>>(n, za, zb, deg, part); break;
        case 64: k_gram_wide<64><<<nb, kWideThreads, 0, s>>>(n, za, zb, deg, part); break;
        case 128: k_gram_wide<128><<<nb, kWideThreads, 0, s>>>(n, za, zb, deg, part); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Sum of the nb block partials (fixed order) into smem, one LP x LP float64 matrix.
__device__ void sum_partials(const double* __restrict__ part, int nb, int LP, double* s_g) {
    const int NT = LP * LP;
    for (int e = threadIdx.x; e < NT; e += blockDim.x) {
        double t = 0.0;
        for (int q = 0; q < nb; ++q) t += part[(size_t)q * NT + e];
        s_g[e] = t;
    }
    __syncthreads();
}

// ---- Cholesky and R^-1 (one block, float64) --------------------------------------------------------
// Shared memory: one LP x LP float64 array holding G's upper triangle, overwritten row by row by R
// (R[a][b] at [a][b], a < b), and then R^-1 transposed in the strict lower triangle (R^-1[a][c] at
// [c][a], a < c); the two diagonals live in their own arrays.
__global__ void __launch_bounds__(kWideThreads)
k_chol_inv_wide(const double* __restrict__ part, int nb, int l, int LP, float* __restrict__ rinv) {
    extern __shared__ double s_g[];
    double* s_rd = s_g + (size_t)LP * LP;   // diagonal of R
    double* s_id = s_rd + LP;               // diagonal of R^-1
    __shared__ int s_dead[128];
    __shared__ double s_gmax;
    sum_partials(part, nb, LP, s_g);
    if (threadIdx.x == 0) {
        double gmax = 0.0;
        for (int a = 0; a < l; ++a) gmax = fmax(gmax, s_g[(size_t)a * LP + a]);
        s_gmax = gmax;
    }
    __syncthreads();
    const double gmax = s_gmax;
    for (int a = 0; a < l; ++a) {
        if (threadIdx.x == 0) {
            double p = s_g[(size_t)a * LP + a];
            for (int c = 0; c < a; ++c) p -= s_g[(size_t)c * LP + a] * s_g[(size_t)c * LP + a];
            const int dead = !(p > 1e-14 * gmax) || gmax <= 0.0;
            s_dead[a] = dead;
            s_rd[a] = dead ? 1.0 : sqrt(p);
        }
        __syncthreads();
        for (int b = a + 1 + threadIdx.x; b < l; b += blockDim.x) {
            double q = s_g[(size_t)a * LP + b];
            for (int c = 0; c < a; ++c) q -= s_g[(size_t)c * LP + a] * s_g[(size_t)c * LP + b];
            s_g[(size_t)a * LP + b] = s_dead[a] ? 0.0 : q / s_rd[a];
        }
        __syncthreads();
    }
    // column c of R^-1 by back substitution, one thread per column
    for (int c = threadIdx.x; c < l; c += blockDim.x) {
        s_id[c] = 1.0 / s_rd[c];
        for (int a = c - 1; a >= 0; --a) {
            double t = s_g[(size_t)a * LP + c] * s_id[c];
            for (int b = a + 1; b < c; ++b) t += s_g[(size_t)a * LP + b] * s_g[(size_t)c * LP + b];
            s_g[(size_t)c * LP + a] = -t / s_rd[a];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < LP * LP; e += blockDim.x) {
        const int a = e / LP, b = e % LP;
        double v;
        if (a >= l || b >= l) v = (a == b && a >= l) ? 1.0 : 0.0;
        else if (s_dead[b]) v = 0.0;
        else if (a < b) v = s_g[(size_t)b * LP + a];
        else if (a == b) v = s_id[a];
        else v = 0.0;
        rinv[e] = (float)v;
    }
}

// ---- Z <- Z M, in place ----------------------------------------------------------------------------
// Tiles of 32 rows are staged in shared memory; thread (r, g) forms row r's columns g*LP/8 .. of
// the product, sum over a in increasing order (the order of the l <= 8 kernels), and the tile is
// written back coalesced.
constexpr int kApplyRows = 32;

template <int LP>
__global__ void __launch_bounds__(kWideThreads) k_apply_wide(int n, float* __restrict__ z, const float* __restrict__ m) {
    constexpr int CG = LP / 8;               // columns per thread
    extern __shared__ float s_m[];           // LP x LP
    float* s_z = s_m + LP * LP;              // kApplyRows x (LP + 1)
    for (int q = threadIdx.x; q < LP * LP; q += blockDim.x) s_m[q] = m[q];
    const int r = threadIdx.x % kApplyRows, g = threadIdx.x / kApplyRows;
    const long long ntile = ((long long)n + kApplyRows - 1) / kApplyRows;
    for (long long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const long long r0 = tile * kApplyRows;
        __syncthreads();
        for (int q = threadIdx.x; q < kApplyRows * LP; q += blockDim.x) {
            const int rr = q / LP, c = q % LP;
            s_z[rr * (LP + 1) + c] = r0 + rr < n ? z[(size_t)(r0 + rr) * LP + c] : 0.f;
        }
        __syncthreads();
        float acc[CG];
#pragma unroll
        for (int q = 0; q < CG; ++q) acc[q] = 0.f;
        for (int a = 0; a < LP; ++a) {
            const float za = s_z[r * (LP + 1) + a];
#pragma unroll
            for (int q = 0; q < CG; ++q) acc[q] = fmaf(za, s_m[a * LP + g * CG + q], acc[q]);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < CG; ++q) s_z[r * (LP + 1) + g * CG + q] = acc[q];
        __syncthreads();
        for (int q = threadIdx.x; q < kApplyRows * LP; q += blockDim.x) {
            const int rr = q / LP, c = q % LP;
            if (r0 + rr < n) z[(size_t)(r0 + rr) * LP + c] = s_z[rr * (LP + 1) + c];
        }
    }
}

static size_t apply_smem(int LP) { return ((size_t)LP * LP + (size_t)kApplyRows * (LP + 1)) * sizeof(float); }

template <int LP>
static cudaError_t launch_apply_wide(int n, float* z, const float* m, int nb, cudaStream_t s) {
    const size_t smem = apply_smem(LP);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_apply_wide<LP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_apply_wide<LP><<<nb, kWideThreads, smem, s>>>(n, z, m);
    return cudaGetLastError();
}

static cudaError_t apply_wide(int LP, int n, float* z, const float* m, int nb, cudaStream_t s) {
    switch (LP) {
        case 16: return launch_apply_wide<16>(n, z, m, nb, s);
        case 32: return launch_apply_wide<32>(n, z, m, nb, s);
        case 64: return launch_apply_wide<64>(n, z, m, nb, s);
        case 128: return launch_apply_wide<128>(n, z, m, nb, s);
    }
    return cudaErrorInvalidValue;
}

static size_t chol_smem(int LP) { return ((size_t)LP * LP + 2 * (size_t)LP) * sizeof(double); }

static cudaError_t chol_inv_wide(const double* part, int nb, int l, int LP, float* rinv, cudaStream_t s) {
    const size_t smem = chol_smem(LP);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k_chol_inv_wide, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_chol_inv_wide<<<1, kWideThreads, smem, s>>>(part, nb, l, LP, rinv);
    return cudaGetLastError();
}

// ---- Rayleigh-Ritz: H = (G + G^T) / 2, eigenpairs by parallel cyclic Jacobi (one block) -------------
// A in shared memory (LP x LP float64), the accumulated rotations V in global memory (vwork).
// Round-robin pairing: positions 0 .. m-1 (m = l rounded up to even), position 0 fixed and the
// others turning by one each step, so that every pair meets once in the m - 1 steps of a sweep.
// Output as for l <= 8: columns sorted by decreasing value, each with its largest component
// positive; identity on the padding.
__global__ void __launch_bounds__(kWideThreads)
k_ritz_wide(const double* __restrict__ part, int nb, int l, int LP, double* __restrict__ V, float* __restrict__ vout,
            double* __restrict__ values) {
    extern __shared__ double s_a[];
    __shared__ double s_c[64], s_s[64];
    __shared__ int s_p[64], s_q[64];
    __shared__ double s_r1[kWideThreads / 32], s_r2[kWideThreads / 32];
    __shared__ int s_order[128];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    sum_partials(part, nb, LP, s_a);
    for (int e = tid; e < LP * LP; e += blockDim.x) {
        const int a = e / LP, b = e % LP;
        if (a < b && b < l) {
            const double v = 0.5 * (s_a[(size_t)a * LP + b] + s_a[(size_t)b * LP + a]);
            s_a[(size_t)a * LP + b] = v;
            s_a[(size_t)b * LP + a] = v;
        } else if (a >= l || b >= l) {
            s_a[e] = 0.0;
        }
        V[e] = a == b ? 1.0 : 0.0;
    }
    __syncthreads();
    const int m = l + (l & 1), half = m / 2;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int e = tid; e < l * l; e += blockDim.x) {
            const double v = s_a[(size_t)(e / l) * LP + e % l];
            tot += v * v;
            if (e / l != e % l) off += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if (lane == 0) {
            s_r1[wid] = off;
            s_r2[wid] = tot;
        }
        __syncthreads();
        off = 0.0;
        tot = 0.0;
        for (int w = 0; w < kWideThreads / 32; ++w) {
            off += s_r1[w];
            tot += s_r2[w];
        }
        __syncthreads();
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int step = 0; step < m - 1; ++step) {
            if (tid < half) {
                const int pa = tid, pb = m - 1 - tid;
                const int xa = pa == 0 ? 0 : 1 + (pa - 1 + step) % (m - 1);
                const int xb = pb == 0 ? 0 : 1 + (pb - 1 + step) % (m - 1);
                const int p = xa < xb ? xa : xb, q = xa < xb ? xb : xa;
                double c = 1.0, sn = 0.0;
                const double apq = q < l ? s_a[(size_t)p * LP + q] : 0.0;
                if (apq != 0.0) {
                    const double theta = (s_a[(size_t)q * LP + q] - s_a[(size_t)p * LP + p]) / (2.0 * apq);
                    const double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                    c = 1.0 / sqrt(tt * tt + 1.0);
                    sn = tt * c;
                }
                s_p[tid] = p;
                s_q[tid] = q;
                s_c[tid] = c;
                s_s[tid] = sn;
            }
            __syncthreads();
            for (int idx = tid; idx < half * l; idx += blockDim.x) {   // A <- A J
                const int j = idx / l, r = idx % l;
                if (s_s[j] == 0.0) continue;
                const int p = s_p[j], q = s_q[j];
                const double arp = s_a[(size_t)r * LP + p], arq = s_a[(size_t)r * LP + q];
                s_a[(size_t)r * LP + p] = s_c[j] * arp - s_s[j] * arq;
                s_a[(size_t)r * LP + q] = s_s[j] * arp + s_c[j] * arq;
            }
            __syncthreads();
            for (int idx = tid; idx < half * l; idx += blockDim.x) {   // A <- J^T A
                const int j = idx / l, r = idx % l;
                if (s_s[j] == 0.0) continue;
                const int p = s_p[j], q = s_q[j];
                const double apr = s_a[(size_t)p * LP + r], aqr = s_a[(size_t)q * LP + r];
                s_a[(size_t)p * LP + r] = s_c[j] * apr - s_s[j] * aqr;
                s_a[(size_t)q * LP + r] = s_s[j] * apr + s_c[j] * aqr;
            }
            for (int idx = tid; idx < half * l; idx += blockDim.x) {   // V <- V J
                const int j = idx / l, r = idx % l;
                if (s_s[j] == 0.0) continue;
                const int p = s_p[j], q = s_q[j];
                const double vrp = V[(size_t)r * LP + p], vrq = V[(size_t)r * LP + q];
                V[(size_t)r * LP + p] = s_c[j] * vrp - s_s[j] * vrq;
                V[(size_t)r * LP + q] = s_s[j] * vrp + s_c[j] * vrq;
            }
            __syncthreads();
        }
    }
    if (tid == 0) {   // selection sort by decreasing eigenvalue (stable in index)
        for (int a = 0; a < l; ++a) s_order[a] = a;
        for (int a = 0; a < l; ++a)
            for (int b = a + 1; b < l; ++b)
                if (s_a[(size_t)s_order[b] * LP + s_order[b]] > s_a[(size_t)s_order[a] * LP + s_order[a]]) {
                    const int t = s_order[a];
                    s_order[a] = s_order[b];
                    s_order[b] = t;
                }
    }
    __syncthreads();
    for (int e = tid; e < LP * LP; e += blockDim.x) {
        const int a = e / LP, b = e % LP;
        if (a >= l || b >= l) vout[e] = (a == b && a >= l) ? 1.f : 0.f;
    }
    for (int c = tid; c < l; c += blockDim.x) {
        const int src = s_order[c];
        int big = 0;
        for (int r = 1; r < l; ++r)
            if (fabs(V[(size_t)r * LP + src]) > fabs(V[(size_t)big * LP + src])) big = r;
        const double sgn = V[(size_t)big * LP + src] < 0 ? -1.0 : 1.0;
        for (int r = 0; r < l; ++r) vout[(size_t)r * LP + c] = (float)(sgn * V[(size_t)r * LP + src]);
        values[c] = s_a[(size_t)src * LP + src];
    }
}

// ---- host: orthonormalising and Ritz on wide blocks -------------------------------------------------
struct WideScratch {
    double* part;    // nb x LP x LP
    float* mat;      // LP x LP (R^-1 or V)
    double* vwork;   // LP x LP
    int nb;
};

static size_t wide_scratch_bytes(int LP, int nb) {
    return (((size_t)nb * LP * LP * 8 + 255) & ~(size_t)255) + (((size_t)LP * LP * 4 + 255) & ~(size_t)255) +
           (size_t)LP * LP * 8 + 256;
}

static WideScratch carve_wide(char* p, int LP, int nb) {
    WideScratch w{};
    w.nb = nb;
    w.part = reinterpret_cast<double*>(p);
    p += ((size_t)nb * LP * LP * 8 + 255) & ~(size_t)255;
    w.mat = reinterpret_cast<float*>(p);
    p += ((size_t)LP * LP * 4 + 255) & ~(size_t)255;
    w.vwork = reinterpret_cast<double*>(p);
    return w;
}

static cudaError_t orthonormalize_wide(int LP, int n, int l, float* z, const double* deg, const WideScratch& w,
                                       cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {   // CholeskyQR2
        if ((e = gram_wide(LP, n, z, z, deg, w.part, w.nb, s)) != cudaSuccess) break;
        if ((e = chol_inv_wide(w.part, w.nb, l, LP, w.mat, s)) != cudaSuccess) break;
        e = apply_wide(LP, n, z, w.mat, w.nb, s);
    }
    return e;
}

cudaError_t launch_init_any(int LP, int n, int l, unsigned long long seed, const float* dinv, void* out, int store,
                            cudaStream_t s);

// Orthogonal iteration on l = 9 .. 128 columns (fsc_embed_orthogonal's wide branch).
fsc_status embed_orthogonal_wide(fsc_graph* g, int l, int t, int every, uint64_t seed, float* emb,
                                 const fsc_embed_opts* opts, cudaStream_t s) {
    const int LP = pad_l(l);
    const int n = (int)g->n;
    fsc_status rc = ensure_workspace(g, (size_t)n * LP * 4 + 256, s);
    if (rc != FSC_OK) return rc;
    const int nb = device_props().num_sms;
    char* scratch = nullptr;
    cudaError_t e = pool_malloc(reinterpret_cast<void**>(&scratch), wide_scratch_bytes(LP, nb), s);
    if (e != cudaSuccess) return cuda_status(e);
    const WideScratch w = carve_wide(scratch, LP, nb);
    float* buf[2];
    buf[t % 2] = emb;
    buf[(t + 1) % 2] = static_cast<float*>(g->ws);
    do {
        if ((e = launch_init_any(LP, n, l, seed, g->dinv, buf[0], (int)FSC_F32, s)) != cudaSuccess) break;
        if (opts && opts->ev_spmm_begin && (e = cudaEventRecord((cudaEvent_t)opts->ev_spmm_begin, s)) != cudaSuccess) break;
        for (int it = 0; it < t && e == cudaSuccess; ++it) {
            if ((e = power_step_wide(LP, g, buf[it % 2], buf[(it + 1) % 2], s)) != cudaSuccess) break;
            if ((it + 1) % every == 0 || it == t - 1) e = orthonormalize_wide(LP, n, l, buf[(it + 1) % 2], g->deg, w, s);
        }
        if (e != cudaSuccess) break;
        if (t == 0) e = orthonormalize_wide(LP, n, l, emb, g->deg, w, s);
        if (e != cudaSuccess) break;
        if (opts && opts->ev_spmm_end) e = cudaEventRecord((cudaEvent_t)opts->ev_spmm_end, s);
    } while (0);
    const cudaError_t ef = pool_free(scratch, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (ef != cudaSuccess) return cuda_status(ef);
    return FSC_OK;
}

// Ritz pairs on the orthonormal wide block emb (fsc_top_eigenvectors' wide branch): M Q by one power
// step into the workspace, the cross Gram Q^T D (M Q), Jacobi, and the rotation emb <- emb V.
fsc_status ritz_wide(fsc_graph* g, int l, float* emb, double* values, cudaStream_t s) {
    const int LP = pad_l(l);
    const int n = (int)g->n;
    const int nb = device_props().num_sms;
    char* scratch = nullptr;
    cudaError_t e = pool_malloc(reinterpret_cast<void**>(&scratch), wide_scratch_bytes(LP, nb) + 1024, s);
    if (e != cudaSuccess) return cuda_status(e);
    const WideScratch w = carve_wide(scratch, LP, nb);
    double* dvals = reinterpret_cast<double*>(scratch + wide_scratch_bytes(LP, nb));
    float* mz = static_cast<float*>(g->ws);
    do {
        if ((e = power_step_wide(LP, g, emb, mz, s)) != cudaSuccess) break;
        if ((e = gram_wide(LP, n, emb, mz, g->deg, w.part, nb, s)) != cudaSuccess) break;
        const size_t smem = (size_t)LP * LP * sizeof(double);
        if (smem > 48 * 1024 &&
            (e = cudaFuncSetAttribute(k_ritz_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            break;
        k_ritz_wide<<<1, kWideThreads, smem, s>>>(w.part, nb, l, LP, w.vwork, w.mat, dvals);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = apply_wide(LP, n, emb, w.mat, nb, s)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(values, dvals, (size_t)l * 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
        e = cudaStreamSynchronize(s);
    } while (0);
    const cudaError_t ef = pool_free(scratch, s);
    if (e != cudaSuccess) return cuda_status(e);
    if (ef != cudaSuccess) return cuda_status(ef);
    return FSC_OK;
}

FSC_BOUNDS_READER(wide)

}  // namespace fsc
