/*
 * The float64 oracle of Algorithm 2 restated in plain C with OpenMP loops, for timing the
 * method on all host cores.  TEST INFRASTRUCTURE: only tests, smoke() and the benchmark's CPU
 * legs use it; it shares no code with the CUDA library.  Built by build() with
 *     gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC
 * (-ffp-contract=off: the float32 distances below must be rounded after every operation,
 * as the module doc of oracle/kmeans.py fixes).
 *
 * It follows the numpy oracle step for step (oracle/spectral.py, oracle/kmeans.py,
 * oracle/rng.py) and is pinned against it on small graphs by the CPU tests:
 *   - degrees d(v) = sum over u != v of w(u, v) (Sec. 2); D^-1/2 := 0 for d(v) = 0;
 *   - start block: Philox4x64-10 (Salmon et al., SC'11) key (seed, 1), element (i, c) has linear
 *     index e = c n + i, block e / 4, Box-Muller on U24 words (cosine for even e % 4, sine for
 *     odd), U24(w) = ((w >> 40) + 1) 2^-24;
 *   - Algorithm 1: x <- M x, M = I - N / 2, N = D^-1/2 (D - A) D^-1/2, t times, no
 *     normalisation; the embedding is D^-1/2 Y (Algorithm 2), rounded to float32 for k-means;
 *   - k-means++ (Sec. 2.2): first centre floor(u_0 n); round r: smallest i with float64 prefix
 *     (index order) of D^2 above u_r sum(D^2), u_r = U53 of word 0 of Philox counter (r, 0, 0, 0)
 *     under key (seed, 2); sum 0 -> lowest index not chosen; no prefix above -> largest index
 *     with D^2 > 0;
 *   - Lloyd: nearest centroid by float32 squared distance (columns in order, ties to the lowest
 *     index), centroids are float64 means in point order (an empty cluster keeps its centroid),
 *     stop when no label changes or after max_iter steps.
 * Loops over points and rows run in parallel; every sum whose order matters (prefix, centroid
 * sums, inertia) runs sequentially in index order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---- Philox4x64-10 ---------------------------------------------------------------------- */
static void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    for (int r = 0; r < 10; ++r) {
        const u128 p0 = (u128)c[0] * M0, p1 = (u128)c[2] * M1;
        const uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        const uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += W0;
        k1 += W1;
    }
}

static double u24(uint64_t w) { return ((double)(w >> 40) + 1.0) * 0x1p-24; }
static double u53(uint64_t w) { return (double)(w >> 11) * 0x1p-53; }

/* n x l start block, row-major out[i * l + c]. */
void orc_gaussian_block(int64_t n, int l, uint64_t seed, double* out) {
    const int64_t total = n * (int64_t)l, nblk = (total + 3) / 4;
#pragma omp parallel for schedule(static)
    for (int64_t b = 0; b < nblk; ++b) {
        uint64_t c[4] = {(uint64_t)b, 0, 0, 0};
        philox4x64_10(c, seed, 1);
        double z[4];
        for (int p = 0; p < 2; ++p) {
            const double r = sqrt(-2.0 * log(u24(c[2 * p])));
            const double a = 2.0 * 3.141592653589793 * u24(c[2 * p + 1]);
            z[2 * p] = r * cos(a);
            z[2 * p + 1] = r * sin(a);
        }
        for (int j = 0; j < 4; ++j) {
            const int64_t e = 4 * b + j;
            if (e < total) out[(e % n) * l + e / n] = z[j];
        }
    }
}

double orc_kmeanspp_uniform(uint64_t seed, int64_t r) {
    uint64_t c[4] = {(uint64_t)r, 0, 0, 0};
    philox4x64_10(c, seed, 2);
    return u53(c[0]);
}

/* ---- graph operator --------------------------------------------------------------------- */
void orc_degrees(int64_t n, const int64_t* rp, const int32_t* col, const float* w, double* deg, double* dinv) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double d = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
            if (col[p] != i) d += w ? (double)w[p] : 1.0;
        deg[i] = d;
        dinv[i] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
    }
}

/* t steps x <- M x on the n x l block x (row-major), tmp of the same size; result in x. */
void orc_power_method(int64_t n, const int64_t* rp, const int32_t* col, const float* w, const double* deg,
                      const double* dinv, int l, int t, double* x, double* tmp) {
    for (int s = 0; s < t; ++s) {
#pragma omp parallel for schedule(dynamic, 1024)
        for (int64_t i = 0; i < n; ++i) {
            double ax[64];                              /* (A D^-1/2 x)_i, l <= 64 */
            for (int c = 0; c < l; ++c) ax[c] = 0.0;
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
                const int64_t j = col[p];
                const double a = (w ? (double)w[p] : 1.0) * dinv[j];
                for (int c = 0; c < l; ++c) ax[c] += a * x[j * l + c];
            }
            for (int c = 0; c < l; ++c) {
                /* (N x)_i = d^-1/2_i (d_i d^-1/2_i x_i - sum_j w_ij d^-1/2_j x_j); y = x - N x / 2 */
                const double nx = dinv[i] * (deg[i] * dinv[i] * x[i * l + c] - ax[c]);
                tmp[i * l + c] = x[i * l + c] - 0.5 * nx;
            }
        }
        memcpy(x, tmp, sizeof(double) * (size_t)n * (size_t)l);
    }
}

/* B = D^-1/2 Y rounded to float32, n x l row-major. */
void orc_embedding_f32(int64_t n, int l, const double* dinv, const double* y, float* out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < l; ++c) out[i * l + c] = (float)(dinv[i] * y[i * l + c]);
}

/* ---- k-means ---------------------------------------------------------------------------- */
static float dist32(const float* x, const float* c, int l) {
    float acc = 0.0f;
    for (int j = 0; j < l; ++j) {
        const float d = x[j] - c[j];
        const float q = d * d;
        acc = acc + q;
    }
    return acc;
}

/* The first `rounds` picks (rounds <= k) of k-means++ on X (n x l float32); D2 is scratch (n). */
void orc_kmeanspp(int64_t n, int l, const float* X, int k, int rounds, uint64_t seed, int64_t* seeds, float* D2,
                  double* prefix) {
    int64_t first = (int64_t)floor(orc_kmeanspp_uniform(seed, 0) * (double)n);
    if (first > n - 1) first = n - 1;
    seeds[0] = first;
    for (int r = 1; r < rounds && r < k; ++r) {
        const float* c = X + seeds[r - 1] * l;
        const int init = r == 1;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) {
            const float d = dist32(X + i * l, c, l);
            D2[i] = (init || d < D2[i]) ? d : D2[i];
        }
        double acc = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            acc += (double)D2[i];
            prefix[i] = acc;
        }
        int64_t nxt = -1;
        if (acc == 0.0) {
            for (int64_t i = 0; i < n && nxt < 0; ++i) {
                int taken = 0;
                for (int q = 0; q < r; ++q) taken |= seeds[q] == i;
                if (!taken) nxt = i;
            }
        } else {
            const double target = orc_kmeanspp_uniform(seed, r) * acc;
            int64_t lo = 0, hi = n;                     /* smallest i with prefix[i] > target */
            while (lo < hi) {
                const int64_t mid = lo + (hi - lo) / 2;
                if (prefix[mid] > target) hi = mid;
                else lo = mid + 1;
            }
            if (lo < n) nxt = lo;
            else
                for (int64_t i = n - 1; i >= 0 && nxt < 0; --i)
                    if (D2[i] > 0.0f) nxt = i;
        }
        seeds[r] = nxt;
    }
}

/* Lloyd from the centres X[seeds]; returns the iteration count, writes labels, float64
 * centroids (k x l), the last assignment's inertia and the number of labels it changed, and each
 * point's nearest and second-nearest float32 distances in that assignment. */
int orc_lloyd(int64_t n, int l, const float* X, int k, const int64_t* seeds, int max_iter, int32_t* labels,
              double* c64, double* inertia, int64_t* changed, float* best, float* second) {
    float* c32 = (float*)malloc(sizeof(float) * (size_t)k * (size_t)l);
    double* sum = (double*)malloc(sizeof(double) * (size_t)k * (size_t)l);
    int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
    for (int j = 0; j < k; ++j)
        for (int c = 0; c < l; ++c) {
            c64[j * l + c] = (double)X[seeds[j] * l + c];
            c32[j * l + c] = (float)c64[j * l + c];
        }
    for (int64_t i = 0; i < n; ++i) labels[i] = -1;
    int it = 0;
    int64_t ch = n;
    for (it = 1; it <= max_iter; ++it) {
        ch = 0;
#pragma omp parallel for schedule(static) reduction(+ : ch)
        for (int64_t i = 0; i < n; ++i) {
            int bj = 0;
            float bd = dist32(X + i * l, c32, l), sd = INFINITY;
            for (int j = 1; j < k; ++j) {
                const float d = dist32(X + i * l, c32 + j * l, l);
                if (d < bd) {
                    sd = bd;
                    bd = d;
                    bj = j;
                } else if (d < sd) {
                    sd = d;
                }
            }
            ch += labels[i] != bj;
            labels[i] = bj;
            best[i] = bd;
            second[i] = sd;
        }
        double in = 0.0;
        for (int64_t i = 0; i < n; ++i) in += (double)best[i];
        *inertia = in;
        memset(sum, 0, sizeof(double) * (size_t)k * (size_t)l);
        memset(cnt, 0, sizeof(int64_t) * (size_t)k);
        for (int64_t i = 0; i < n; ++i) {
            const int j = labels[i];
            cnt[j] += 1;
            for (int c = 0; c < l; ++c) sum[j * l + c] += (double)X[i * l + c];
        }
        for (int j = 0; j < k; ++j)
            if (cnt[j] > 0)
                for (int c = 0; c < l; ++c) {
                    c64[j * l + c] = sum[j * l + c] / (double)cnt[j];
                    c32[j * l + c] = (float)c64[j * l + c];
                }
        if (ch == 0) break;
    }
    if (it > max_iter) it = max_iter;
    *changed = ch;
    free(c32);
    free(sum);
    free(cnt);
    return it;
}
