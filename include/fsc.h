/*
 * fsc.h - C ABI of the GB300 fast spectral clustering library (libfsc.so).
 *
 * The library implements Algorithm 2 (FastSpectralCluster) of Macgregor,
 * "Fast and Simple Spectral Clustering in Theory and Practice" (NeurIPS 2023):
 * l Gaussian vectors are pushed through t unnormalised power iterations
 * (Algorithm 1) of the signless Laplacian M = I - N/2 = (I + D^-1/2 A D^-1/2)/2
 * (Sec. 2), the result is scaled by D^-1/2, and its rows are clustered with
 * k-means++ seeding and Lloyd iterations (Sec. 2.2).
 *
 * Conventions for every entry point:
 *  - Array arguments are DEVICE pointers on the current CUDA device unless a
 *    comment says "host".  `stream` is a cudaStream_t passed as void*
 *    (NULL = the legacy default stream).
 *  - Matrices are row-major.  An embedding of l columns is stored with
 *    ld = fsc_pad_l(l) floats per row (1, 2, 4 or 8 for l <= 8; 16, 32, 64 or
 *    128 for l = 9 .. 128, accepted by fsc_embed_orthogonal, fsc_top_eigenvectors,
 *    fsc_kmeans and fsc_kmeans_best); columns l..ld-1 are written as zero by
 *    the embeddings and ignored by fsc_kmeans.
 *  - No C++ exception crosses the ABI.  Every call returns an fsc_status;
 *    outputs are defined only when it returns FSC_OK.  Calls marked
 *    "asynchronous" only enqueue work on `stream`; errors detected on the
 *    device during such work are reported by the next synchronous call that
 *    reads them (fsc_kmeans with non-NULL stats, fsc_cluster) or by
 *    fsc_sync_status().
 *  - Thread safety: a graph handle may be used by one stream at a time.
 *  - Contexts: the library's per-device state (its memory pool, status word and kernel launch
 *    attributes) is made in the CUDA context current at first use and made again when a call
 *    finds another context current (for example after cudaDeviceReset).  Handles (graphs,
 *    batches) are not: destroy them before resetting a device.
 */
#ifndef FSC_H
#define FSC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fsc_status {
    FSC_OK = 0,
    FSC_ERR_INVALID_ARG = 1,    /* bad size, null pointer, unsupported l/k, ... */
    FSC_ERR_INDEX_RANGE = 2,    /* column index outside [0, n) or row_ptr not monotone */
    FSC_ERR_NOT_SYMMETRIC = 3,  /* edge (i,j,w) without its mirror (j,i,w) */
    FSC_ERR_SELF_LOOP = 4,      /* an entry (i, i) */
    FSC_ERR_BAD_WEIGHT = 5,     /* negative, NaN or infinite weight */
    FSC_ERR_OOM = 6,            /* device allocation failed */
    FSC_ERR_CUDA = 7,           /* a CUDA runtime call failed */
    FSC_ERR_TIMEOUT = 8,        /* a bounded device-side wait gave up */
    FSC_ERR_UNSORTED = 9,       /* symmetry check asked for, but a row's columns are not increasing */
    FSC_ERR_TOO_LARGE = 10      /* problem needs more scratch than fsc_kmeans_static's fixed array */
} fsc_status;

typedef enum fsc_dtype {
    FSC_F32 = 0,                /* power-iteration block stored in float32 */
    FSC_BF16 = 1,               /* stored in bfloat16, accumulated in float32 */
    FSC_F16 = 2                 /* stored in float16 (learned-filter basis only), accumulated in float32 */
} fsc_dtype;

/* fsc_create_graph flags */
#define FSC_VALIDATE_SYMMETRY 0x1u  /* also check that A is symmetric (rows must be sorted) */
#define FSC_COPY 0x4u               /* the graph keeps its own copy of the CSR (no borrowing) */

/* fsc_embed_opts.flags */
#define FSC_EMBED_RESCALE 0x1u      /* per-column power-of-two rescale every iteration */

typedef struct fsc_graph fsc_graph;   /* opaque */

typedef struct fsc_graph_info_t {
    int64_t n;                  /* vertices */
    int64_t nnz;                /* stored entries = 2m (both directions of each edge) */
    int64_t n_isolated;         /* vertices with d(v) = 0 */
    int32_t weighted;           /* 1 if the graph has a weight array */
    double volume;              /* vol(V) = sum of degrees (Sec. 2) */
    const double* deg;          /* device, n: d(v) = sum_{u != v} w(u, v), float64 */
    const float* dinv;          /* device, n: d(v)^-1/2 rounded to float (0 if isolated) */
    const float* invdeg;        /* device, n: 1/d(v) rounded to float (0 if isolated) */
    double deg_sumsq;           /* sum of d(v)^2 */
    double deg_max;             /* max d(v) */
} fsc_graph_info_t;

typedef struct fsc_embed_opts {
    uint32_t flags;             /* FSC_EMBED_* */
    int32_t threads_per_row;    /* 0 = choose automatically; else 4, 8, 16 or 32 */
    void* ev_spmm_begin;        /* optional cudaEvent_t recorded on `stream` before the first power iteration */
    void* ev_spmm_end;          /* optional cudaEvent_t recorded after the last power iteration */
} fsc_embed_opts;

typedef struct fsc_kmeans_stats {
    int32_t iterations;         /* Lloyd assignment steps run */
    int32_t changed;            /* labels changed in the last step (0 = converged) */
    int32_t empty_events;       /* cluster-steps in which a cluster had no point */
    int32_t device_status;      /* fsc_status of the device-side work */
    double inertia;             /* float64 sum of the last step's float32 squared distances */
    double seeding_potential;   /* sum of D^2 after the last k-means++ round */
} fsc_kmeans_stats;

/*
 * fsc_create_graph - wrap a CSR graph and compute its degrees (Sec. 2).
 *
 * row_ptr: int64[n+1], row_ptr[0] = 0, row_ptr[n] = nnz, non-decreasing.
 * col_idx: int32[nnz], each in [0, n), no (i, i) entries.
 * w:       float[nnz] non-negative finite weights, or NULL for unit weights.
 * The CSR must hold both directions of every undirected edge with equal
 * weights (checked only with FSC_VALIDATE_SYMMETRY, which also requires
 * increasing columns within each row).
 * The graph BORROWS row_ptr, col_idx and w: the caller keeps them alive and
 * unchanged until fsc_destroy_graph, unless flags holds FSC_COPY, in which case
 * the graph copies them (stream-ordered, device to device) into memory it owns
 * and the caller's arrays may be reused once the call returns.  The library owns
 * the degree arrays and the embedding workspace.  n must be in [1, 2^31 - 1].
 * Degrees: d(v) = sum over u != v of w(u,v) in float64; D^-1/2 of an
 * isolated vertex is taken as 0 (its embedding row is then 0).
 * Rows with more than 1024 stored entries (hubs) are listed and cut into
 * 1024-entry segments here; every sparse step sums a segment with one warp and
 * a row's segments in segment order (results do not depend on scheduling), so
 * a hub does not hold back the row-split kernels.
 * Synchronous: returns after validation; on error *out is left unchanged and
 * nothing is allocated.
 */
fsc_status fsc_create_graph(int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                            const float* w, uint32_t flags, void* stream, fsc_graph** out);

/* Frees the library-owned arrays of g (synchronises the device first). NULL is a no-op. */
fsc_status fsc_destroy_graph(fsc_graph* g);

/*
 * Device memory.  The library's own buffers (degree arrays, workspaces, k-means scratch) come
 * from one stream-ordered pool per device that keeps freed blocks mapped, so repeated
 * create / cluster / destroy cycles neither map nor unmap memory.  fsc_release_cached_memory
 * synchronises every device the pool has used and returns the cached blocks to the driver
 * (blocks still owned by live graphs stay).  Host call.
 */
fsc_status fsc_release_cached_memory(void);

/* Host call: fills *info (pointers stay valid until fsc_destroy_graph). */
fsc_status fsc_graph_info(const fsc_graph* g, fsc_graph_info_t* info);

/* Row stride of an l-column embedding: 1, 2, 4 or 8 (0 if l is not in [1, 8]). */
int fsc_pad_l(int l);

/*
 * fsc_embed - Algorithm 2 up to k-means: B = D^-1/2 [PowerMethod(M, x_i, t)]_{i=1..l}.
 *
 * x_1..x_l are N(0, I) vectors drawn by Philox4x64-10 (key = (seed, 1)):
 * element (i, c) of the n x l start block has index e = c*n + i; Philox
 * counter (e/4, 0, 0, 0) gives four words; element slot j = e%4 takes the
 * Box-Muller pair (u1, u2) = (U(w[2*(j/2)]), U(w[2*(j/2)+1])),
 * U(w) = ((w >> 40) + 1) * 2^-24, cosine branch for even j, sine for odd.
 * PowerMethod (Algorithm 1) applies M t times without normalisation.
 * emb: float[n * fsc_pad_l(l)] output, pad columns set to 0.
 * store: dtype of the iterated block (FSC_BF16 = bfloat16 storage with
 * float32 accumulation; degrees and weights stay float32/float64).
 * 1 <= l <= 8, t >= 0 (t = 0 returns D^-1/2 X0).  opts may be NULL.
 * Asynchronous.
 */
fsc_status fsc_embed(const fsc_graph* g, int l, int t, uint64_t seed, fsc_dtype store, float* emb,
                     const fsc_embed_opts* opts, void* stream);

/*
 * fsc_power_step - one power iteration (Algorithm 1 body) in embedding coordinates.
 *
 * With z = D^-1/2 x, computes z_out = D^-1/2 M D^1/2 z_in = (z_in + D^-1 A z_in) / 2,
 * i.e. D^-1/2 of M x.  z_in/z_out: n * fsc_pad_l(l) elements of `store`
 * type (float or bfloat16 bits), must not overlap.  Accumulation in float32.
 * This is the kernel fsc_embed runs t times, with the same launch shape.
 * Asynchronous.
 */
fsc_status fsc_power_step(const fsc_graph* g, int l, fsc_dtype store, const void* z_in, void* z_out,
                          int threads_per_row, void* stream);

/*
 * fsc_gather_floor - a measurement aid, not a step of the method: the neighbour gathers of one
 * power step (Algorithm 1 body: one iterate row per stored entry) with no row structure.  Reads
 * every column index of g once, in order, loads the row of z it names and adds the rows up into
 * *sum_out (device float, overwritten; the value itself means nothing).  z: n * fsc_pad_l(l)
 * elements of `store` (FSC_F32, FSC_BF16 or FSC_F16), aligned like an embedding.  Its duration
 * is the floor that random row gathers set for fsc_power_step (and the filter's sparse steps) on
 * the same graph, row width and type: row_ptr, the per-row sums, 1/d and the output rows are
 * left out.  Asynchronous.
 */
fsc_status fsc_gather_floor(const fsc_graph* g, int l, fsc_dtype store, const void* z, float* sum_out, void* stream);

/*
 * fsc_kmeans - k-means++ seeding and Lloyd iterations on the rows of emb (Sec. 2.2).
 *
 * emb: float[n * ld], row i = point i, first l columns used (1 <= l <= ld, ld in {1, 2, 4, 8,
 * 16, 32, 64, 128}; the rows of 16 .. 128 floats are the wide embeddings of
 * fsc_embed_orthogonal / fsc_top_eigenvectors with l = k, and need 16-byte alignment).
 * Seeding: first centre floor(u_0 * n); round r picks the smallest i whose
 * float64 prefix sum of D^2 (float32 squared distance to the nearest chosen
 * centre) exceeds u_r * sum(D^2); u_r from Philox4x64-10 key (seed, 2),
 * counter (r, 0, 0, 0), word 0, U(w) = (w >> 11) * 2^-53.  If sum(D^2) = 0,
 * the lowest index not chosen yet.
 * Lloyd: nearest centroid by float32 squared distance (ties -> lowest
 * index), centroids are float64 means (an empty cluster keeps its centroid),
 * stop when no label changes or after max_iter steps.
 * labels: int32[n] output.  centroids: float64[k * l] output or NULL.
 * seed_idx: int64[k] output (the k-means++ picks) or NULL.
 * stats: host struct or NULL.  With stats != NULL the call synchronises
 * `stream` and reports device-side errors (e.g. FSC_ERR_TIMEOUT) in its
 * return value; with NULL it is asynchronous.
 * Limits: 1 <= k <= n, k <= 1024, k * ld <= 4096 (ld <= 8) or 32768 (ld >= 16), 1 <= max_iter.
 * Workspace is allocated stream-ordered (cudaMallocAsync) and freed on return.  With ld >= 16
 * the same rules and results come from per-round / per-iteration launches (no pruning), and
 * the call synchronises `stream` once per Lloyd iteration whether or not stats is given.
 */
fsc_status fsc_kmeans(const float* emb, int64_t n, int l, int ld, int k, uint64_t seed, int max_iter,
                      int32_t* labels, double* centroids, int64_t* seed_idx, fsc_kmeans_stats* stats,
                      void* stream);

/*
 * fsc_kmeans_static - fsc_kmeans without any device allocation.
 *
 * No counterpart in the paper: an engineering variant for callers that cannot allocate
 * device memory once they are running, e.g. code inside a runtime that hands out a fixed
 * memory budget up front, or a latency-critical loop where an allocation could block or
 * fail.  Same arguments, same kernels and same results as fsc_kmeans; the scratch space
 * (16 bytes per point: two D^2 buffers, reused by Lloyd for its bounds, each point's nearest
 * chosen centre and a lower bound on its distance to the others; plus per-tile and per-chunk
 * state and the centroids) lives in one fixed array of
 * FSC_KMEANS_STATIC_SCRATCH_BYTES compiled into the library, which every GPU that loads the
 * library keeps reserved until the process exits.
 *  - Size limit, independent of the GPU and of the launch shape: about
 *      16 n + 36 ceil(n / 2048) + (40 + 4 ld) ceil(n / 128) + 24 k (ld + 1) + 12 k ld + 8 k + 1 KB  (each part
 *    rounded up to 256 bytes) must not exceed FSC_KMEANS_STATIC_SCRATCH_BYTES; larger problems
 *    return FSC_ERR_TOO_LARGE.  With k = 64 and ld = 8 that admits up to about 1.01 million points.
 *  - All calls on a device share the one array, which keeps the last call's contents (the
 *    call clears what must start at zero): calls that may run at the same time on the GPU
 *    (different streams, threads or processes sharing the context) race; serialise them.
 *  - Every call looks up the array's device address (cudaGetSymbolAddress) on the current
 *    device; nothing is cached, so the call also works after cudaDeviceReset.
 *  - Always synchronous: it waits for `stream` and copies results to the host, so it cannot be
 *    used inside a stream capture (a call on a capturing stream returns FSC_ERR_INVALID_ARG
 *    without touching the capture).  stats may be NULL.
 *  - Device-side errors (e.g. FSC_ERR_TIMEOUT) are reported in the return value only; unlike
 *    fsc_kmeans they are not added to the status word that fsc_sync_status() reads.
 */
#define FSC_KMEANS_STATIC_SCRATCH_BYTES (16u * 1024u * 1024u)
fsc_status fsc_kmeans_static(const float* emb, int64_t n, int l, int ld, int k, uint64_t seed, int max_iter,
                             int32_t* labels, double* centroids, int64_t* seed_idx, fsc_kmeans_stats* stats,
                             void* stream);

/*
 * fsc_embed_orthogonal - orthogonal iteration: t power steps of M (Algorithm 1) on a block of l
 * vectors that is D-orthonormalised after every `every` steps and after the last (CholeskyQR2,
 * the unique basis with positive-diagonal R).  With l = k it is the "PM k Vectors" variant the
 * paper compares against (Sec. 4); the span after t steps is that of M^t X0, so only the basis,
 * not the subspace, differs from fsc_embed.  emb: n x fsc_pad_l(l) floats = D^-1/2 Q (columns
 * orthonormal in x-space).  Float32 only; opts->flags must be 0.  A column linearly dependent on
 * the earlier ones comes out zero.  Same start block as fsc_embed(seed).  1 <= l <= 128: blocks of
 * 16 .. 128 columns (l > 8, "PM k Vectors" for k up to 128) use their own kernels for the power
 * step (a lane group per row, 16 bytes per lane), the Gram, the Cholesky factor and Z R^-1.
 * Asynchronous.
 */
fsc_status fsc_embed_orthogonal(const fsc_graph* g, int l, int t, int every, uint64_t seed, float* emb,
                                const fsc_embed_opts* opts, void* stream);

/*
 * fsc_knn_graph - the k-nearest-neighbour graph of a point set (the Sec. 4.2 pre-processing,
 * where the paper clusters the 10-NN graph of each dataset).  points: device float32 n x dim,
 * row-major; dim <= 64, 1 <= knn <= 16, knn < n, n * knn < 2^31.  Distances: float32
 * sum over columns in order of (x_i[c] - x_j[c])^2, no fused multiply-add; neighbours of i: the
 * knn points j != i of smallest distance, ties to the lower index; symmetrised by union; weight
 * of {i, j}: exp(-d2 / sigma^2), sigma = median (mean of the two middle values for an even
 * count) of the n * knn directed distances sqrt(d2), found exactly.  Output CSR (both
 * directions, columns increasing in each row): row_ptr (device int64, n + 1), col (device
 * int32) and w (device float32, may be NULL) with room for capacity >= 2 * n * knn entries;
 * *nnz (host) receives the entry count, *sigma (host, optional) sigma.  Synchronous.  The
 * result can be passed to fsc_create_graph (FSC_VALIDATE_SYMMETRY accepts it).
 */
fsc_status fsc_knn_graph(const float* points, int64_t n, int dim, int knn, int64_t* row_ptr, int32_t* col, float* w,
                         int64_t capacity, int64_t* nnz, double* sigma, void* stream);

/*
 * fsc_top_eigenvectors - Rayleigh-Ritz on the fsc_embed_orthogonal basis: with Q that basis
 * (x-space, orthonormal), H = Q^T M Q (one more power step and a D-weighted Gram), H = V diag(theta)
 * V^T by cyclic Jacobi (float64; one thread for l <= 8, the block's threads rotating l/2 disjoint
 * pairs at a time for l = 9 .. 128), and emb <- D^-1/2 Q V, columns in decreasing theta, each
 * column's largest entry of V positive.  For t large enough the pairs converge to the top l
 * eigenpairs of M: the "k Eigs" embedding of the paper's comparison (Sec. 4) when l = k <= 128.
 * values: host double[l] <- theta.  Synchronous.
 */
fsc_status fsc_top_eigenvectors(const fsc_graph* g, int l, int t, int every, uint64_t seed, float* emb,
                                double* values, const fsc_embed_opts* opts, void* stream);

/*
 * fsc_kmeans_best - k-means with restarts (not in the paper; the usual library practice of
 * keeping the best of several k-means runs).  Run r (r = 0 .. n_init-1) is fsc_kmeans with
 * seed + r (its own k-means++ draws); the run of lowest inertia is kept, ties going to the
 * lowest r.  Outputs as fsc_kmeans for that run; *best_run (host, optional) receives r.
 * Synchronous; allocates one spare labels/centroids/seeds set from the library pool when
 * n_init > 1.
 */
fsc_status fsc_kmeans_best(const float* emb, int64_t n, int l, int ld, int k, uint64_t seed, int n_init,
                           int max_iter, int32_t* labels, double* centroids, int64_t* seed_idx,
                           fsc_kmeans_stats* stats, int32_t* best_run, void* stream);

/*
 * fsc_partition_scores - adjusted Rand index and normalised mutual information of two labelings
 * (the accuracy measures of Sec. 4).  labels_a (values in [0, ka)) and labels_b (in [0, kb)):
 * device int32 arrays of n entries.  The contingency table is built on the device; ARI uses
 * exact 64-bit pair counts, NMI the arithmetic-mean normalisation (natural logs).
 * ari_nmi: host double[2] <- {ARI, NMI}.  ka * kb <= 2^24.  A label outside its range gives
 * FSC_ERR_INDEX_RANGE.  Synchronous.
 */
fsc_status fsc_partition_scores(const int32_t* labels_a, const int32_t* labels_b, int64_t n, int ka, int kb,
                                double* ari_nmi, void* stream);

/*
 * fsc_cluster - Algorithm 2 end to end: fsc_embed then fsc_kmeans on its output.
 * labels: int32[n] output.  stats: host struct or NULL.  opts may be NULL.
 * Synchronous (returns after the device work and reports its status).
 */
fsc_status fsc_cluster(const fsc_graph* g, int k, int l, int t, uint64_t seed, fsc_dtype store, int max_iter,
                       int32_t* labels, fsc_kmeans_stats* stats, const fsc_embed_opts* opts, void* stream);

/*
 * fsc_autotune - time launch shapes of the power step on g: 4 lanes per row with 4 or 3
 * neighbour rows in flight per lane, and 8, 16, 32 lanes per row.
 *
 * No counterpart in the paper (a tuning aid).  Runs one warm-up and five timed power steps per
 * candidate on scratch iterates, records the fastest in a process-wide table keyed by (row
 * width fsc_pad_l(l), storage type, weighted or not, half-octave bucket of the average degree)
 * and returns its lane count (*best_threads_per_row) and time.  Later fsc_embed / fsc_cluster /
 * fsc_power_step calls with threads_per_row = 0 use the table's shape for graphs in the same
 * bucket, batch plans its lane count.  Rows with more than 1024 entries are not timed: every
 * sparse step splits them into 1024-entry segments summed by their own kernels (see
 * fsc_create_graph).  Synchronous; allocates its scratch.
 */
fsc_status fsc_autotune(const fsc_graph* g, int l, fsc_dtype store, int* best_threads_per_row, float* best_us,
                        void* stream);

/*
 * Batched Algorithm 2 (no counterpart in the paper: many independent graphs at once).
 *
 * The batch is the disjoint union of num_graphs graphs in one CSR with global vertex ids:
 * graph g owns vertices [vertex_offset[g], vertex_offset[g+1]) and every edge of its rows must
 * stay inside that range (checked).  Each graph gets its own k, l, t and seed; l or t NULL
 * (or l[g] = 0, t[g] < 0) take fsc_default_params mode 0.  fsc_batch_create validates the
 * union, computes degrees, assigns lanes per row (autotuned with FSC_BATCH_AUTOTUNE), orders
 * the graphs largest first, allocates the per-graph workspace and captures the work (a queue
 * reset and, per row width, two persistent kernels in which one CTA runs one graph's embedding,
 * then one graph's k-means) into a CUDA graph.
 * fsc_batch_run replays that graph on `stream` (asynchronous); labels[v] receives the local
 * cluster id (0..k_g-1) of global vertex v.  Per graph the result equals fsc_cluster with the
 * same parameters and lanes per row.  The plan borrows row_ptr, col_idx, w and labels.
 * Limits: k_g <= 256, l_g <= 8, total vertices < 2^31.
 */
#define FSC_BATCH_AUTOTUNE 0x2u
typedef struct fsc_batch fsc_batch;   /* opaque */
typedef struct fsc_batch_desc {
    int32_t num_graphs;
    const int64_t* vertex_offset;   /* host, num_graphs + 1, vertex_offset[0] = 0 */
    const int64_t* row_ptr;         /* device, vertex_offset[num_graphs] + 1 entries */
    const int32_t* col_idx;         /* device, global vertex ids */
    const float* w;                 /* device or NULL (unit weights) */
    const int32_t* k;               /* host, clusters per graph */
    const int32_t* l;               /* host or NULL */
    const int32_t* t;               /* host or NULL */
    const uint64_t* seed;           /* host */
    int32_t* labels;                /* device output, vertex_offset[num_graphs] entries */
    int32_t store;                  /* fsc_dtype of the iterates */
    int32_t max_iter;               /* Lloyd iteration cap per graph */
    uint32_t flags;                 /* FSC_BATCH_AUTOTUNE | FSC_VALIDATE_SYMMETRY */
} fsc_batch_desc;

fsc_status fsc_batch_create(const fsc_batch_desc* desc, void* stream, fsc_batch** out);
fsc_status fsc_batch_run(fsc_batch* batch, void* stream);
/* Synchronises `stream`; any output may be NULL.  stats: host, num_graphs entries.
 * seed_idx: host, sum of k_g (graph by graph).  centroids: host, sum of k_g * l_g doubles. */
fsc_status fsc_batch_results(fsc_batch* batch, fsc_kmeans_stats* stats, int64_t* seed_idx, double* centroids,
                             void* stream);
/* Copies graph `graph`'s float32 embedding D^-1/2 M^t X0 of the last run into out (device,
 * n_g * fsc_pad_l(l_g) floats).  Asynchronous on `stream`. */
fsc_status fsc_batch_embedding(fsc_batch* batch, int graph, float* out, void* stream);
fsc_status fsc_batch_destroy(fsc_batch* batch);

/*
 * Learned polynomial filter (no counterpart in the paper: an extension of Algorithm 2).
 *
 * p(M) X = sum_{j=0..8} c_j T_j(A_hat) X, A_hat = 2M - I = D^-1/2 A D^-1/2, replaces M^t X
 * (Chebyshev three-term recurrence: 8 sparse products instead of t).  The coefficients come
 * from an MLP 16 -> 64 -> 64 -> 9 (GELU, float32, 5833 parameters: W1 64x16, b1, W2 64x64, b2,
 * W3 9x64, b3, row-major, in that order) fed 16 features of the graph and its start block:
 * log n, log mean degree, degree std / mean, log(max degree / mean), log k, log(n/k), l/8,
 * isolated fraction, and the Chebyshev moments mu_j = sum_c x_c^T T_j(A_hat) x_c / sum_c
 * x_c^T x_c, j = 1..8 (from inner products fused into the recurrence).  It is trained to
 * minimise ||p(M) X - P X||^2 / ||P X||^2, P the top-k eigenprojector of M (the quantity
 * Lemma 3.1 bounds for M^t).
 *
 * fsc_filter_embed: the filtered embedding D^-1/2 p(M) X (emb: n x fsc_pad_l(l) floats), with
 *   X the same start block as fsc_embed(seed).  params: device MLP parameters, or NULL when
 *   coeffs_override (device, 9 floats) gives the coefficients.  feats_out (16) and coeffs_out
 *   (9) are optional device outputs.  opts: threads_per_row and the events bracketing the 8
 *   sparse steps (flags ignored).  store is the type the basis T_j X is held in: FSC_F32, or
 *   FSC_F16 for half the bytes.  The coefficients alternate in sign and cancel the bulk of
 *   the spectrum, so rounding in the basis does not cancel with it and the recurrence carries
 *   it forward: FSC_BF16 (8-bit significand) raises the leakage ||(I - P) Y||^2 / ||P Y||^2
 *   of an SBM (n = 1e5, k = 20, mean degree 33) from 1.3e-3 to 1.7e-2 and k-means lands in
 *   worse optima; FSC_F16 (11-bit significand, 64x smaller squared error) keeps it near the
 *   float32 value.  FSC_F16 needs the entries of D^-1/2 X inside float16's normal range
 *   (about 6e-5 .. 6e4): degrees between about 1e-8 and 1e8.  energy_out (device double,
 *   optional) receives ||p(M) X||^2 in x-space (sum over v of d(v) |y_v|^2).  Asynchronous.
 * fsc_cluster_filtered: fsc_filter_embed then fsc_kmeans; synchronous.  Guard (the plain
 *   method as fallback): for Gaussian X, E ||P X||^2 = l k, so a good filter gives
 *   ||p(M) X||^2 / (l k) near 1 and leakage into the bulk raises it; above
 *   1.25 + 3 sqrt(2 / (l k)) (leakage beyond a quarter of the signal, allowing for the chi^2
 *   spread of ||P X||^2) the block is recomputed by fsc_embed with t = ceil(log2 n) (float32,
 *   or bfloat16 with rescaling for the 2-byte stores) and that block is clustered instead.
 *   opts->flags may hold FSC_FILTER_NO_FALLBACK.  report (optional) tells what happened.
 * fsc_mlp_forward: coefficients (batch x 9) of features (batch x 16), device arrays.
 * fsc_mlp_train_step: adds the gradient of the mean loss c^T Gn c - 2 bn^T c + 1 over the
 *   batch (feats batch x 16, Gn batch x 81, bn batch x 9, device float32) to grad (5833);
 *   with apply_update != 0 then takes an Adam step (beta 0.9 / 0.999, eps 1e-8, step >= 1
 *   for bias correction, weight decay added to the gradient) and zeroes grad.  loss_out
 *   (device scalar) receives the mean loss, may be NULL.  Asynchronous.
 */
typedef struct fsc_filter_report {
    double energy_ratio;        /* ||p(M) X||^2 / (l k), x-space energy of the filtered block */
    double threshold;           /* the ratio above which the plain method replaces the filter */
    int32_t fallback;           /* 1: the labels come from the plain power method */
    int32_t fallback_t;         /* its number of iterations, ceil(log2 n) */
} fsc_filter_report;

#define FSC_FILTER_NO_FALLBACK 0x100u   /* fsc_embed_opts.flags bit for fsc_cluster_filtered */

fsc_status fsc_filter_embed(const fsc_graph* g, int l, int k, uint64_t seed, fsc_dtype store, const float* params,
                            const float* coeffs_override, float* emb, float* feats_out, float* coeffs_out,
                            double* energy_out, const fsc_embed_opts* opts, void* stream);
fsc_status fsc_cluster_filtered(const fsc_graph* g, int k, int l, uint64_t seed, fsc_dtype store, const float* params,
                                int max_iter, int32_t* labels, fsc_kmeans_stats* stats, fsc_filter_report* report,
                                const fsc_embed_opts* opts, void* stream);
fsc_status fsc_mlp_forward(const float* params, const float* feats, int batch, float* coeffs, void* stream);
fsc_status fsc_mlp_train_step(float* params, float* grad, float* adam_m, float* adam_v, int step, float lr,
                              float weight_decay, const float* feats, const float* Gn, const float* bn, int batch,
                              float* loss_out, int apply_update, void* stream);

/*
 * fsc_default_params - l and t for n vertices and k clusters (host, no device work).
 * mode 0: l = max(1, ceil(log2 k)), t = ceil(log2 n).
 * mode 1: the paper's practical remark after Theorem 3.2, l = max(1, ceil(ln k)),
 *         t = ceil(10 ln(n / k)).
 */
fsc_status fsc_default_params(int64_t n, int k, int mode, int* l, int* t);

/* Synchronises `stream`, returns and clears the device-side error word of the current device. */
fsc_status fsc_sync_status(void* stream);

/* Testing hook: bound on every device-side wait, in nanoseconds (default 2e9). Host call. */
void fsc_set_wait_limit_ns(int64_t ns);

/* Testing hook (failure injection without a GPU fault): with enable != 0, kernels launched
 * afterwards never release their grid barriers, so every wait runs into the limit above and
 * the call reports FSC_ERR_TIMEOUT.  Host call; 0 restores normal operation. */
void fsc_inject_barrier_stall(int enable);

/*
 * fsc_bounds_report - the first out-of-range index found by a library built with the compile flag
 * FSC_BOUNDS_CHECK (python -m paper_2310_10939_gb300.build --bounds-check: libfsc_checked.so).  Such
 * a build tests every index a kernel derives from its inputs before the access it addresses (a
 * neighbour's column index against the rows of the iterate, a point's label or nearest-centre
 * index against the centres, a chosen point against n), records the first one outside its range
 * and skips the access; nothing traps.  Host call, synchronising the device.  *site: 0 = nothing
 * recorded, -1 = this library has no checks, else the kernel site (1 sparse-step gather, 2 wide
 * power-step gather, 3 k-means++ nearest centre, 4 Lloyd label, 5 wide k-means++ nearest centre,
 * 6 wide Lloyd label, 7 k-means++ pick); *index, *lo, *hi (optional) the value and its range
 * [lo, hi).  clear != 0 resets the records.
 */
fsc_status fsc_bounds_report(int32_t* site, int64_t* index, int64_t* lo, int64_t* hi, int clear);

/* Static, human-readable name of a status code. */
const char* fsc_status_string(fsc_status s);

/* Library version, e.g. "0.1.0". */
const char* fsc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FSC_H */
