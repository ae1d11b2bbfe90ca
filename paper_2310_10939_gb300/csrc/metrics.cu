// Partition comparison (the accuracy measures of Sec. 4): the contingency table of two labelings
// on the device, then the adjusted Rand index and the normalised mutual information from it.
//
// ARI: pair counts C(x, 2) summed over table cells, row and column totals in exact 64-bit
// integers; the final ratio (index - expected) / (max - expected) in float64.
// NMI: mutual information over the table divided by the arithmetic mean of the two entropies
// (natural logarithms, float64).  Empty rows or columns contribute nothing to either.
#include <math.h>

#include "fsc_internal.cuh"

namespace fsc {

// Counts n_xy over all i.  Small tables are counted per block in shared memory (32-bit) and
// added once per cell; larger ones go straight to the global 64-bit table.
__global__ void __launch_bounds__(256) k_contingency(const int32_t* __restrict__ a, const int32_t* __restrict__ b,
                                                     long long n, int ka, int kb, int shared_ok,
                                                     unsigned long long* __restrict__ table, int* __restrict__ bad) {
    extern __shared__ unsigned s_tab[];
    const int cells = ka * kb;
    if (shared_ok) {
        for (int q = threadIdx.x; q < cells; q += blockDim.x) s_tab[q] = 0u;
        __syncthreads();
    }
    int flag = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = a[i], y = b[i];
        if (x < 0 || x >= ka || y < 0 || y >= kb) {
            flag = 1;
            continue;
        }
        if (shared_ok) atomicAdd(&s_tab[x * kb + y], 1u);
        else atomicAdd(&table[(size_t)x * kb + y], 1ull);
    }
    if (flag) atomicOr(bad, 1);
    if (shared_ok) {
        __syncthreads();
        for (int q = threadIdx.x; q < cells; q += blockDim.x)
            if (s_tab[q]) atomicAdd(&table[q], (unsigned long long)s_tab[q]);
    }
}

__device__ __forceinline__ unsigned long long pairs(unsigned long long x) { return x ? x * (x - 1) / 2 : 0ull; }

__device__ double block_sum_d(double v, double* s_red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
    return t;
}

__device__ unsigned long long block_sum_u(unsigned long long v, unsigned long long* s_red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
    return t;
}

// One block: row and column totals (kept in rt, ct), the three pair sums, the entropies and the
// mutual information.
__global__ void __launch_bounds__(256) k_scores(const unsigned long long* __restrict__ table, int ka, int kb,
                                                long long n, unsigned long long* __restrict__ rt,
                                                unsigned long long* __restrict__ ct, double* __restrict__ out) {
    __shared__ double s_rd[8];
    __shared__ unsigned long long s_ru[8];
    const double dn = (double)n;
    unsigned long long p_ij = 0, p_a = 0, p_b = 0;
    double mi = 0.0, ha = 0.0, hb = 0.0;
    for (int x = threadIdx.x; x < ka; x += blockDim.x) {
        unsigned long long r = 0;
        for (int y = 0; y < kb; ++y) r += table[(size_t)x * kb + y];
        rt[x] = r;
        p_a += pairs(r);
        if (r) ha -= ((double)r / dn) * log((double)r / dn);
    }
    for (int y = threadIdx.x; y < kb; y += blockDim.x) {
        unsigned long long c = 0;
        for (int x = 0; x < ka; ++x) c += table[(size_t)x * kb + y];
        ct[y] = c;
        p_b += pairs(c);
        if (c) hb -= ((double)c / dn) * log((double)c / dn);
    }
    __syncthreads();   // rt, ct complete (global writes of this block)
    for (int q = threadIdx.x; q < ka * kb; q += blockDim.x) {
        const unsigned long long v = table[q];
        if (!v) continue;
        p_ij += pairs(v);
        const int x = q / kb, y = q - x * kb;
        const double pij = (double)v / dn;
        mi += pij * log(((double)v * dn) / ((double)rt[x] * (double)ct[y]));
    }
    p_ij = block_sum_u(p_ij, s_ru);
    p_a = block_sum_u(p_a, s_ru);
    p_b = block_sum_u(p_b, s_ru);
    mi = block_sum_d(mi, s_rd);
    ha = block_sum_d(ha, s_rd);
    hb = block_sum_d(hb, s_rd);
    if (threadIdx.x == 0) {
        const unsigned long long total = pairs((unsigned long long)n);
        double ari = 1.0;
        if (total) {
            const double expected = (double)p_a * (double)p_b / (double)total;
            const double maximum = 0.5 * ((double)p_a + (double)p_b);
            if (maximum != expected) ari = ((double)p_ij - expected) / (maximum - expected);
        }
        out[0] = ari;
        out[1] = (ha + hb == 0.0) ? 1.0 : 2.0 * mi / (ha + hb);
    }
}

}  // namespace fsc

using namespace fsc;

extern "C" fsc_status fsc_partition_scores(const int32_t* labels_a, const int32_t* labels_b, int64_t n, int ka,
                                           int kb, double* ari_nmi, void* stream) {
    if (!labels_a || !labels_b || !ari_nmi || n < 1 || ka < 1 || kb < 1 || ka > 65536 || kb > 65536 ||
        (long long)ka * kb > (1LL << 24))
        return FSC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    const size_t cells = (size_t)ka * kb;
    char* buf = nullptr;
    const size_t bytes = (cells + (size_t)ka + (size_t)kb) * 8 + 256;
    cudaError_t e = pool_malloc(reinterpret_cast<void**>(&buf), bytes, s);
    if (e != cudaSuccess) return cuda_status(e);
    unsigned long long* table = reinterpret_cast<unsigned long long*>(buf);
    unsigned long long* rt = table + cells;
    unsigned long long* ct = rt + ka;
    char* tail = reinterpret_cast<char*>(ct + kb);
    int* bad = reinterpret_cast<int*>(tail);
    double* dout = reinterpret_cast<double*>(tail + 128);
    fsc_status rc = FSC_OK;
    do {
        if ((e = cudaMemsetAsync(buf, 0, bytes, s)) != cudaSuccess) break;
        const size_t smem = cells * 4;
        const int shared_ok = smem <= 32 * 1024 ? 1 : 0;
        long long blocks = (n + 255) / 256;
        const long long cap = (long long)device_props().num_sms * 4;
        if (blocks > cap) blocks = cap;
        k_contingency<<<(unsigned)blocks, 256, shared_ok ? smem : 0, s>>>(labels_a, labels_b, n, ka, kb, shared_ok,
                                                                        table, bad);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        k_scores<<<1, 256, 0, s>>>(table, ka, kb, n, rt, ct, dout);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        int hbad = 0;
        if ((e = cudaMemcpyAsync(ari_nmi, dout, 2 * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
        if (hbad) rc = FSC_ERR_INDEX_RANGE;
    } while (0);
    pool_free(buf, s);
    if (e != cudaSuccess) return cuda_status(e);
    return rc;
}
