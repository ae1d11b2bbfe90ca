// Long rows of the sparse steps (Algorithm 1 body and the filter's Chebyshev step).
//
// The row-split kernels give each row a group of a few lanes, which walk the row's entries in
// dependent passes: a row with d entries costs about d / 16 memory latencies, so one hub row (a
// star's centre, a kNN hub) holds back the whole launch.  Rows with more than kLongRow entries are
// therefore split, as a merge-path decomposition would split them, into segments of kSegLen
// consecutive entries: fsc_create_graph lists them (rows sorted, segments in entry order), the
// row-split kernels skip them, one warp per segment sums its entries' gathered rows (coalesced
// column reads), and one thread per long row adds its segments' partial sums in segment order and
// applies the step's epilogue.  The sums of a row are therefore formed in a fixed order: results
// do not depend on scheduling.
#include <algorithm>
#include <vector>

#include "longrows.cuh"

namespace fsc {

// rows longer than kLongRow entries: count, and (row, first entry, length) triples in [0, cap)
__global__ void k_long_rows(int64_t n, const int64_t* __restrict__ rp, int64_t cap,
                            unsigned long long* __restrict__ count, int64_t* __restrict__ rows) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lo = rp[i], len = rp[i + 1] - lo;
        if (len > kLongRow) {
            const unsigned long long slot = atomicAdd(count, 1ull);
            if ((int64_t)slot < cap) {   // (row, first entry, length)
                rows[3 * slot] = i;
                rows[3 * slot + 1] = lo;
                rows[3 * slot + 2] = len;
            }
        }
    }
}

cudaError_t launch_long_rows(int64_t n, const int64_t* rp, int64_t cap, unsigned long long* count, int64_t* rows,
                             cudaStream_t s) {
    int64_t blocks = (n + 255) / 256;
    const int64_t lim = (int64_t)device_props().num_sms * 8;
    if (blocks > lim) blocks = lim;
    k_long_rows<<<(unsigned)blocks, 256, 0, s>>>(n, rp, cap, count, rows);
    return cudaGetLastError();
}

// Host: the segment tables of the listed long rows (rows sorted, so the layout does not depend on
// the order the listing kernel found them in).  Allocates g->long_base.
fsc_status build_long_rows(fsc_graph* g, int64_t count, const int64_t* d_rows, cudaStream_t s) {
    std::vector<int64_t> trip((size_t)count * 3);
    cudaError_t e = cudaMemcpyAsync(trip.data(), d_rows, (size_t)count * 24, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
    std::vector<size_t> order((size_t)count);
    for (size_t q = 0; q < order.size(); ++q) order[q] = q;
    std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return trip[3 * a] < trip[3 * b]; });
    std::vector<int64_t> lrow, slo, shi;
    std::vector<int32_t> seg0, nseg;
    for (size_t q : order) {
        const int64_t r = trip[3 * q], lo = trip[3 * q + 1], len = trip[3 * q + 2];
        lrow.push_back(r);
        seg0.push_back((int32_t)slo.size());
        const int64_t ns = (len + kSegLen - 1) / kSegLen;
        nseg.push_back((int32_t)ns);
        for (int64_t k = 0; k < ns; ++k) {
            slo.push_back(lo + k * kSegLen);
            shi.push_back(std::min(lo + len, lo + (k + 1) * kSegLen));
        }
    }
    const int64_t nl = (int64_t)lrow.size(), ns = (int64_t)slo.size();
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t b_rows = up((size_t)nl * 8), b_s0 = up((size_t)nl * 4), b_ns = up((size_t)nl * 4),
                 b_lo = up((size_t)ns * 8), b_hi = up((size_t)ns * 8), b_part = up((size_t)ns * 8 * 4);
    char* base = nullptr;
    if ((e = pool_malloc(reinterpret_cast<void**>(&base), b_rows + b_s0 + b_ns + b_lo + b_hi + b_part, s)) != cudaSuccess)
        return cuda_status(e);
    g->long_base = base;
    g->long_rows = reinterpret_cast<int64_t*>(base);
    g->long_seg0 = reinterpret_cast<int32_t*>(base + b_rows);
    g->long_nseg = reinterpret_cast<int32_t*>(base + b_rows + b_s0);
    g->seg_lo = reinterpret_cast<int64_t*>(base + b_rows + b_s0 + b_ns);
    g->seg_hi = reinterpret_cast<int64_t*>(base + b_rows + b_s0 + b_ns + b_lo);
    g->seg_part = reinterpret_cast<float*>(base + b_rows + b_s0 + b_ns + b_lo + b_hi);
    g->n_long = nl;
    g->n_seg = ns;
    g->max_row = kLongRow;
    e = cudaMemcpyAsync(g->long_rows, lrow.data(), (size_t)nl * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->long_seg0, seg0.data(), (size_t)nl * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->long_nseg, nseg.data(), (size_t)nl * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->seg_lo, slo.data(), (size_t)ns * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->seg_hi, shi.data(), (size_t)ns * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host vectors go out of scope
    return e == cudaSuccess ? FSC_OK : cuda_status(e);
}

// The power step's epilogue for the long rows (as power_row, with the launch's column scale).
template <int LP, typename TI, typename TO>
__global__ void __launch_bounds__(256)
k_long_power(int64_t nl, const int64_t* __restrict__ rows, const int32_t* __restrict__ seg0,
             const int32_t* __restrict__ nseg, const float* __restrict__ part, const float* __restrict__ invdeg,
             const TI* __restrict__ zin, TO* __restrict__ zout, const unsigned* __restrict__ cm_in,
             unsigned* __restrict__ cm_out, const int* __restrict__ expo, int last) {
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < nl; h += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = rows[h];
        float acc[LP];
        long_row_sum(h, seg0, nseg, part, LP, acc);
        float self[LP], y[LP];
        load_row<LP, TI>(zin + (size_t)row * LP, self);
        const float id = invdeg[row];
#pragma unroll
        for (int c = 0; c < LP; ++c) {
            float scale;
            if (last) scale = expo ? pow2i(expo[c]) : 1.f;
            else scale = cm_in ? pow2i(-exponent_of(__uint_as_float(cm_in[c]))) : 1.f;
            y[c] = scale * (0.5f * fmaf(id, acc[c], self[c]));
        }
        store_row<LP, TO>(zout + (size_t)row * LP, y);
        if (cm_out)
#pragma unroll
            for (int c = 0; c < LP; ++c)
                if (fabsf(y[c]) > 0.f) atomicMax(cm_out + c, __float_as_uint(fabsf(y[c])));
    }
}

template <int LP, typename TI, typename TO>
static cudaError_t long_power_lp(const fsc_graph* g, const StepArgs& a, cudaStream_t s) {
    seg_partial_launch<LP, TI>(g, static_cast<const TI*>(a.zin), s);
    const int64_t nl = g->n_long;
    k_long_power<LP, TI, TO><<<(unsigned)((nl + 255) / 256), 256, 0, s>>>(
        nl, g->long_rows, g->long_seg0, g->long_nseg, g->seg_part, g->invdeg, static_cast<const TI*>(a.zin),
        static_cast<TO*>(a.zout), a.cm_in, a.cm_out, a.expo, a.last);
    return cudaGetLastError();
}

// After a power step on g (row-split kernel, long rows skipped): the long rows.  store_in / store_out:
// 0 float32, 1 bfloat16.
cudaError_t long_rows_power(const fsc_graph* g, int LP, int store_in, int store_out, const StepArgs& a, cudaStream_t s) {
    if (g->n_long == 0) return cudaSuccess;
#define FSC_LP_CASES(TI, TO)                                         \
    switch (LP) {                                                    \
        case 1: return long_power_lp<1, TI, TO>(g, a, s);            \
        case 2: return long_power_lp<2, TI, TO>(g, a, s);            \
        case 4: return long_power_lp<4, TI, TO>(g, a, s);            \
        case 8: return long_power_lp<8, TI, TO>(g, a, s);            \
    }
    if (store_in == 0) { FSC_LP_CASES(float, float) }
    else if (store_out == 0) { FSC_LP_CASES(__nv_bfloat16, float) }
    else { FSC_LP_CASES(__nv_bfloat16, __nv_bfloat16) }
#undef FSC_LP_CASES
    return cudaErrorInvalidValue;
}


}  // namespace fsc
