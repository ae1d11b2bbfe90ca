// Batched Algorithm 2: thousands of graphs of uneven size in a few persistent launches.
//
// The batch is the disjoint union of its graphs, given as one CSR with global vertex ids.
// Graphs are grouped by row width l_pad; per group two persistent kernels run one after the
// other, each taking graphs from its own atomic work queue, largest first (longest processing
// time order), with one 512-thread CTA per graph: k_batch_embed (Gaussian start block, t power
// iterations separated by block barriers; two CTAs per SM) and k_batch_kmeans (block-local
// k-means++ and Lloyd; one CTA per SM).  CTAs never wait on each other, so no launch has an
// inter-CTA spin wait at all.  Each graph uses the same per-row power step arithmetic
// (row_gather) and the same exact fixed-point k-means rules as the single-graph entry points,
// so its labels equal those of fsc_cluster with the same lanes per row.  The launch sequence
// (queue reset, stats reset, the kernels) is captured once into a CUDA graph and replayed by
// fsc_batch_run.
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "batch_device.cuh"

namespace fsc {

// Every edge of a row of graph g must stay inside graph g's vertex range (block-diagonal union).
__global__ void __launch_bounds__(256) k_batch_check(long long nv, const int64_t* __restrict__ rp,
                                                     const int32_t* __restrict__ col,
                                                     const long long* __restrict__ voff, int G,
                                                     int* __restrict__ status) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
        int lo = 0, hi = G;                      // graph of row i: largest g with voff[g] <= i
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (voff[mid] <= i) lo = mid; else hi = mid;
        }
        const long long a = voff[lo], b = voff[lo + 1];
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            const long long j = col[p];
            if (j < a || j >= b) { atomicOr(status, ST_INDEX_RANGE); break; }
        }
    }
}

__global__ void k_gather_boundaries(const int64_t* __restrict__ rp, const long long* __restrict__ voff, int G,
                                    long long* __restrict__ out) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g <= G) out[g] = rp[voff[g]];
}

}  // namespace fsc

using namespace fsc;

struct BatchGroup {
    int LP, first, count;
};

struct fsc_batch {
    int device = 0;
    int num_graphs = 0;
    fsc_graph* uni = nullptr;            // the union graph (degrees, validation)
    BatchGraph* d_graphs = nullptr;
    int* d_queue = nullptr;
    void* zarena = nullptr;
    float* earena = nullptr;
    float* darena = nullptr;
    long long* tarena = nullptr;
    int64_t* seeds = nullptr;
    double* cents = nullptr;
    KmDevStats* stats = nullptr;
    int32_t* labels = nullptr;
    std::vector<BatchGraph> h_graphs;    // in queue order, grouped by row width
    std::vector<BatchGroup> groups;      // two persistent launches each (embedding, k-means)
    std::vector<long long> seed_off;     // by graph id
    std::vector<long long> cent_off;     // by graph id
    std::vector<int> k_of;
    std::vector<int> l_of;
    long long seeds_total = 0, cents_total = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int store = 0;
    size_t smem = 0;
};

static void batch_free(fsc_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->d_graphs);
    cudaFree(b->d_queue);
    cudaFree(b->zarena);
    cudaFree(b->earena);
    cudaFree(b->darena);
    cudaFree(b->tarena);
    cudaFree(b->seeds);
    cudaFree(b->cents);
    cudaFree(b->stats);
    if (b->uni) fsc_destroy_graph(b->uni);
    delete b;
}

extern "C" fsc_status fsc_batch_create(const fsc_batch_desc* d, void* stream, fsc_batch** out) {
    NvtxRange nvtx_range("fsc_batch_create");
    if (!d || !out || d->num_graphs < 1 || !d->vertex_offset || !d->row_ptr || !d->k || !d->seed || !d->labels)
        return FSC_ERR_INVALID_ARG;
    if ((d->store != FSC_F32 && d->store != FSC_BF16) || d->max_iter < 1) return FSC_ERR_INVALID_ARG;
    if (d->flags & ~(FSC_BATCH_AUTOTUNE | FSC_VALIDATE_SYMMETRY)) return FSC_ERR_INVALID_ARG;
    const int G = d->num_graphs;
    const long long* voff = reinterpret_cast<const long long*>(d->vertex_offset);
    if (voff[0] != 0) return FSC_ERR_INVALID_ARG;
    for (int g = 0; g < G; ++g) {
        const long long n = voff[g + 1] - voff[g];
        const int k = d->k[g];
        const int l = d->l ? d->l[g] : 0;
        if (n < 1 || k < 1 || k > n || k > 256 || l < 0 || l > 8 || (d->t && d->t[g] < 0)) return FSC_ERR_INVALID_ARG;
    }
    const long long nv = voff[G];
    if (nv > 2147483647LL) return FSC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    fsc_batch* b = new (std::nothrow) fsc_batch();
    if (!b) return FSC_ERR_OOM;
    b->num_graphs = G;
    b->labels = d->labels;
    b->store = d->store;
    cudaGetDevice(&b->device);
    fsc_status rc = FSC_OK;
    cudaError_t e = cudaSuccess;
    long long* d_voff = nullptr;
    do {
        // nnz of the union and of each graph (row_ptr values at the graph boundaries)
        if ((e = cudaMalloc(&d_voff, sizeof(long long) * (G + 1))) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(d_voff, voff, sizeof(long long) * (G + 1), cudaMemcpyHostToDevice, s)) != cudaSuccess) break;
        long long* d_bound = nullptr;
        if ((e = cudaMalloc(&d_bound, sizeof(long long) * (G + 1))) != cudaSuccess) break;
        k_gather_boundaries<<<(G + 256) / 256, 256, 0, s>>>(d->row_ptr, d_voff, G, d_bound);
        std::vector<long long> bound(G + 1);
        e = cudaMemcpyAsync(bound.data(), d_bound, sizeof(long long) * (G + 1), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(d_bound);
        if (e != cudaSuccess) break;
        const long long nnz = bound[G];
        // the union graph: validation and degrees of every vertex
        rc = fsc_create_graph(nv, nnz, d->row_ptr, d->col_idx, d->w, d->flags & FSC_VALIDATE_SYMMETRY, stream, &b->uni);
        if (rc != FSC_OK) break;
        int* d_status = nullptr;
        if ((e = cudaMalloc(&d_status, sizeof(int))) != cudaSuccess) break;
        cudaMemsetAsync(d_status, 0, sizeof(int), s);
        k_batch_check<<<device_props().num_sms * 8, 256, 0, s>>>(nv, d->row_ptr, d->col_idx, d_voff, G, d_status);
        int hst = 0;
        e = cudaMemcpyAsync(&hst, d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(d_status);
        if (e != cudaSuccess) break;
        if (hst) { rc = status_from_bits(hst); break; }

        // per-graph parameters, arenas and the largest-first work order
        const size_t es = d->store == FSC_F32 ? 4 : 2;
        std::vector<BatchGraph> gs(G);
        b->seed_off.assign(G, 0);
        b->cent_off.assign(G, 0);
        b->k_of.assign(G, 0);
        b->l_of.assign(G, 0);
        long long zoff = 0, eoff = 0, doff = 0, toff = 0, soff = 0, coff = 0;
        size_t smem = 0;
        std::vector<long long> gnnz(G);
        for (int g = 0; g < G; ++g) {
            BatchGraph& x = gs[g];
            const long long n = voff[g + 1] - voff[g];
            int l = d->l ? d->l[g] : 0, t = d->t ? d->t[g] : -1;
            int ld = 0, td = 0;
            fsc_default_params(n, d->k[g], 0, &ld, &td);
            if (l == 0) l = ld;
            if (t < 0) t = td;
            x.v0 = voff[g];
            x.n = (int)n;
            x.k = d->k[g];
            x.l = l;
            x.LP = pad_l(l);
            x.t = t;
            x.seed = d->seed[g];
            x.gid = g;
            gnnz[g] = bound[g + 1] - bound[g];
            const double avg = (double)gnnz[g] / (double)n;
            int tpr = tuned_threads_per_row(avg, x.LP, d->store, d->w != nullptr);
            if (!tpr) {
                fsc_graph tmp{};
                tmp.n = n;
                tmp.nnz = gnnz[g];
                tpr = choose_threads_per_row(&tmp, 0, x.LP, d->store);
            }
            x.tpr = tpr;
            const size_t tab = (size_t)x.k * (x.LP + 1) * 8;
            int ntab = (int)(32768 / tab);
            x.ntab = ntab < 1 ? 1 : (ntab > KM_WARPS ? KM_WARPS : ntab);
            // centroids (float32, float64), chosen indices, ntab tables and the running totals
            const size_t need = (((size_t)x.k * x.LP * 4 + 15) & ~(size_t)15) + (size_t)x.k * x.LP * 8 +
                                (((size_t)x.k * 4 + 15) & ~(size_t)15) + (size_t)(x.ntab + 1) * tab;
            smem = std::max(smem, need);
            // every per-graph base is rounded to 64 elements (>= 128 bytes), so the row vectors of
            // any LP stay aligned whatever the previous graphs' sizes were
            auto round64 = [](long long v) { return (v + 63) / 64 * 64; };
            x.zoff = zoff;
            zoff += round64(2 * n * x.LP);     // two iterate buffers; the second starts at n*LP
            x.eoff = eoff;
            eoff += round64(n * x.LP);
            x.doff = doff;
            doff += n;
            x.toff = toff;
            toff += (n + KM_TILE - 1) / KM_TILE;
            x.soff = soff;
            soff += x.k;
            x.coff = coff;
            coff += (long long)x.k * x.LP;
            b->seed_off[g] = x.soff;
            b->cent_off[g] = x.coff;
            b->k_of[g] = x.k;
            b->l_of[g] = x.l;
        }
        // autotune (optional): time the lane counts on the largest graph of each (degree bucket, LP)
        if (d->flags & FSC_BATCH_AUTOTUNE) {
            std::vector<int> order(G);
            for (int g = 0; g < G; ++g) order[g] = g;
            std::sort(order.begin(), order.end(), [&](int x, int y) { return gnnz[x] > gnnz[y]; });
            for (int g : order) {
                const double avg = (double)gnnz[g] / (double)gs[g].n;
                if (tuned_threads_per_row(avg, gs[g].LP, d->store, d->w != nullptr)) continue;
                fsc_graph view{};
                view.device = b->device;
                view.n = gs[g].n;
                view.nnz = gnnz[g];
                view.row_ptr = d->row_ptr + gs[g].v0;
                view.col = d->col_idx;
                view.w = d->w;
                view.deg = b->uni->deg + gs[g].v0;
                view.dinv = b->uni->dinv + gs[g].v0;
                view.invdeg = b->uni->invdeg + gs[g].v0;
                view.col_off = gs[g].v0;
                int best = 0;
                float us = 0.f;
                rc = autotune_graph(&view, gs[g].l, (fsc_dtype)d->store, &best, &us, s);
                if (view.ws) pool_free(view.ws, s);
                if (rc != FSC_OK) break;
            }
            if (rc != FSC_OK) break;
            for (int g = 0; g < G; ++g) {
                const int tpr = tuned_threads_per_row((double)gnnz[g] / (double)gs[g].n, gs[g].LP, d->store,
                                                      d->w != nullptr);
                if (tpr) gs[g].tpr = tpr;
            }
        }
        std::vector<int> order(G);
        for (int g = 0; g < G; ++g) order[g] = g;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            return gnnz[x] * (long long)gs[x].t > gnnz[y] * (long long)gs[y].t;
        });
        // one group per row width (l_pad 8, 4, 2, 1), largest first inside each group
        b->h_graphs.clear();
        b->groups.clear();
        for (int lp : {8, 4, 2, 1}) {
            const int first = (int)b->h_graphs.size();
            for (int q = 0; q < G; ++q)
                if (gs[order[q]].LP == lp) b->h_graphs.push_back(gs[order[q]]);
            const int count = (int)b->h_graphs.size() - first;
            if (count > 0) b->groups.push_back({lp, first, count});
        }
        b->smem = smem;
        if ((e = cudaMalloc(&b->d_graphs, sizeof(BatchGraph) * G)) != cudaSuccess) break;
        if ((e = cudaMemcpy(b->d_graphs, b->h_graphs.data(), sizeof(BatchGraph) * G, cudaMemcpyHostToDevice)) != cudaSuccess) break;
        if ((e = cudaMalloc(&b->d_queue, 256)) != cudaSuccess) break;
        if ((e = cudaMalloc(&b->zarena, (size_t)zoff * es + 256)) != cudaSuccess) break;
        if ((e = cudaMalloc(&b->earena, (size_t)eoff * 4 + 256)) != cudaSuccess) break;
        if ((e = cudaMalloc(&b->darena, (size_t)doff * 4 + 256)) != cudaSuccess) break;
        if ((e = cudaMalloc(&b->tarena, (size_t)toff * 8 + 256)) != cudaSuccess) break;
        if ((e = cudaMalloc(&b->seeds, (size_t)soff * 8 + 256)) != cudaSuccess) break;
        if ((e = cudaMalloc(&b->cents, (size_t)coff * 8 + 256)) != cudaSuccess) break;
        b->seeds_total = soff;
        b->cents_total = coff;
        if ((e = cudaMalloc(&b->stats, sizeof(KmDevStats) * G)) != cudaSuccess) break;

        // capture queue reset + stats reset + the persistent launches into a CUDA graph
        BatchArgs a{};
        a.graphs = b->d_graphs;
        a.num_graphs = G;
        a.queue = b->d_queue;
        a.row_ptr = d->row_ptr;
        a.col = d->col_idx;
        a.w = d->w;
        a.dinv = b->uni->dinv;
        a.invdeg = b->uni->invdeg;
        a.zarena = b->zarena;
        a.earena = b->earena;
        a.darena = b->darena;
        a.tarena = b->tarena;
        a.seeds = b->seeds;
        a.cents = b->cents;
        a.labels = d->labels;
        a.stats = b->stats;
        a.max_iter = d->max_iter;
        // per group: its kernel, grid (persistent CTAs) and arguments (its slice of the work
        // list and its own queue counter)
        struct Launch {
            const void* kern;
            long long grid;
            size_t smem;
            BatchArgs args;
        };
        std::vector<Launch> launches;
        for (size_t gi = 0; gi < b->groups.size() && e == cudaSuccess && rc == FSC_OK; ++gi) {
            const BatchGroup& grp = b->groups[gi];
            // the group's embedding kernel, then its k-means kernel, each with its own queue counter
            for (int part = 0; part < 2; ++part) {
                Launch L{};
                if (part == 0)
                    L.kern = d->store == FSC_F32 ? batch_kernel_f32(grp.LP, d->w != nullptr)
                                                 : batch_kernel_bf16(grp.LP, d->w != nullptr);
                else
                    L.kern = batch_kmeans_kernel(grp.LP);
                L.smem = part == 0 ? 0 : smem;
                const int per_sm = kernel_occupancy(L.kern, KM_THREADS, L.smem);
                if (per_sm < 1) { rc = FSC_ERR_INVALID_ARG; break; }
                L.grid = (long long)per_sm * device_props().num_sms;
                if (L.grid > grp.count) L.grid = grp.count;
                L.args = a;
                L.args.graphs = b->d_graphs + grp.first;
                L.args.num_graphs = grp.count;
                L.args.queue = b->d_queue + 2 * gi + part;
                launches.push_back(L);
            }
        }
        if (e != cudaSuccess || rc != FSC_OK) break;
        cudaStream_t cs = nullptr;
        if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) break;
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaMemsetAsync(b->d_queue, 0, 8 * sizeof(int), cs);
            cudaMemsetAsync(b->stats, 0, sizeof(KmDevStats) * G, cs);
            for (Launch& L : launches) {
                void* args[] = {&L.args};
                cudaLaunchKernel(L.kern, dim3((unsigned)L.grid), dim3(KM_THREADS), args, L.smem, cs);
            }
            e = cudaStreamEndCapture(cs, &b->graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) break;
    } while (0);
    cudaFree(d_voff);
    if (e != cudaSuccess && rc == FSC_OK) rc = cuda_status(e);
    if (rc != FSC_OK) {
        batch_free(b);
        return rc;
    }
    *out = b;
    return FSC_OK;
}

extern "C" fsc_status fsc_batch_run(fsc_batch* b, void* stream) {
    NvtxRange nvtx_range("fsc_batch_run");
    if (!b || !b->exec) return FSC_ERR_INVALID_ARG;
    FSC_CUDA(cudaGraphLaunch(b->exec, as_stream(stream)));
    return FSC_OK;
}

extern "C" fsc_status fsc_batch_results(fsc_batch* b, fsc_kmeans_stats* stats, int64_t* seed_idx, double* centroids,
                                        void* stream) {
    if (!b) return FSC_ERR_INVALID_ARG;
    cudaStream_t s = as_stream(stream);
    FSC_CUDA(cudaStreamSynchronize(s));
    const int G = b->num_graphs;
    if (stats) {
        std::vector<KmDevStats> h(G);
        FSC_CUDA(cudaMemcpy(h.data(), b->stats, sizeof(KmDevStats) * G, cudaMemcpyDeviceToHost));
        for (int g = 0; g < G; ++g) {
            stats[g].iterations = h[g].iterations;
            stats[g].changed = h[g].changed;
            stats[g].empty_events = h[g].empty_events;
            stats[g].device_status = 0;
            stats[g].inertia = h[g].inertia;
            stats[g].seeding_potential = h[g].potential;
        }
    }
    if (seed_idx || centroids) {
        std::vector<int64_t> hs(b->seeds_total + 1);
        std::vector<double> hc(b->cents_total + 1);
        if (seed_idx) FSC_CUDA(cudaMemcpy(hs.data(), b->seeds, sizeof(int64_t) * b->seeds_total, cudaMemcpyDeviceToHost));
        if (centroids) FSC_CUDA(cudaMemcpy(hc.data(), b->cents, sizeof(double) * b->cents_total, cudaMemcpyDeviceToHost));
        long long so = 0, co = 0;
        for (int g = 0; g < G; ++g) {
            const int k = b->k_of[g], l = b->l_of[g], LP = pad_l(l);
            if (seed_idx)
                for (int j = 0; j < k; ++j) seed_idx[so + j] = hs[b->seed_off[g] + j];
            if (centroids)
                for (int j = 0; j < k; ++j)
                    for (int c = 0; c < l; ++c) centroids[co + (long long)j * l + c] = hc[b->cent_off[g] + (long long)j * LP + c];
            so += k;
            co += (long long)k * l;
        }
    }
    return FSC_OK;
}

extern "C" fsc_status fsc_batch_embedding(fsc_batch* b, int graph, float* out, void* stream) {
    if (!b || !out || graph < 0 || graph >= b->num_graphs) return FSC_ERR_INVALID_ARG;
    for (const BatchGraph& x : b->h_graphs) {
        if (x.gid != graph) continue;
        FSC_CUDA(cudaMemcpyAsync(out, b->earena + x.eoff, sizeof(float) * (size_t)x.n * x.LP, cudaMemcpyDeviceToDevice,
                                 as_stream(stream)));
        return FSC_OK;
    }
    return FSC_ERR_INVALID_ARG;
}

extern "C" fsc_status fsc_batch_destroy(fsc_batch* b) {
    if (!b) return FSC_OK;
    cudaDeviceSynchronize();
    batch_free(b);
    return FSC_OK;
}
