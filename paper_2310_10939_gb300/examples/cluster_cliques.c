/*
 * Algorithm 2 end to end through the C ABI alone: k disjoint cliques of s vertices, each of
 * which must come out as one cluster.  The component indicators of a disconnected graph span
 * the eigenvalue-1 eigenspace of M (Sec. 2); on K_s every other eigenvalue of M is
 * (1 - 1/(s-1))/2, so after t = 30 power iterations the embedding rows of a clique coincide to
 * float32 precision.  The points are then k distinct point masses, and k-means++ puts one centre
 * on each (a mass that already holds a centre has D^2 = 0).  With the default t = ceil(log2 n)
 * = 9 the rows still differ by about 2e-3 relative, and a few seeds land in a merged optimum.
 *
 * Build from the repository root after the library (python -m paper_2310_10939_gb300.build):
 *   gcc -O2 -Iinclude -I/usr/local/cuda/include paper_2310_10939_gb300/examples/cluster_cliques.c \
 *       -Lpaper_2310_10939_gb300 -lfsc -L/usr/local/cuda/lib64 -lcudart \
 *       -Wl,-rpath,paper_2310_10939_gb300 -o cluster_cliques
 * Run: ./cluster_cliques    (exit status 0 when every clique is one cluster)
 */
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>

#include "fsc.h"

#define CK(call)                                                                   \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            fprintf(stderr, "%s: %s\n", #call, cudaGetErrorString(e_));            \
            return 2;                                                              \
        }                                                                          \
    } while (0)
#define FK(call)                                                                   \
    do {                                                                           \
        fsc_status s_ = (call);                                                    \
        if (s_ != FSC_OK) {                                                        \
            fprintf(stderr, "%s: %s\n", #call, fsc_status_string(s_));             \
            return 3;                                                              \
        }                                                                          \
    } while (0)

int main(void) {
    const int k = 8, s = 64;
    const int64_t n = (int64_t)k * s, nnz = n * (s - 1);
    int64_t* row_ptr = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
    int32_t* col = (int32_t*)malloc((size_t)nnz * sizeof(int32_t));
    int32_t* labels = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!row_ptr || !col || !labels) return 4;
    /* CSR with increasing columns: vertex v joins the other s - 1 vertices of its clique */
    int64_t p = 0;
    for (int64_t v = 0; v < n; ++v) {
        row_ptr[v] = p;
        const int64_t c0 = v / s * s;
        for (int64_t u = c0; u < c0 + s; ++u)
            if (u != v) col[p++] = (int32_t)u;
    }
    row_ptr[n] = p;

    int64_t* d_row_ptr;
    int32_t *d_col, *d_labels;
    CK(cudaMalloc((void**)&d_row_ptr, (size_t)(n + 1) * sizeof(int64_t)));
    CK(cudaMalloc((void**)&d_col, (size_t)nnz * sizeof(int32_t)));
    CK(cudaMalloc((void**)&d_labels, (size_t)n * sizeof(int32_t)));
    CK(cudaMemcpy(d_row_ptr, row_ptr, (size_t)(n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_col, col, (size_t)nnz * sizeof(int32_t), cudaMemcpyHostToDevice));

    fsc_graph* g = NULL;
    FK(fsc_create_graph(n, nnz, d_row_ptr, d_col, NULL, FSC_VALIDATE_SYMMETRY, NULL, &g));
    int l = 0, t = 0;
    FK(fsc_default_params(n, k, 0, &l, &t));   /* l = ceil(log2 k) */
    t = 30;
    fsc_kmeans_stats st;
    FK(fsc_cluster(g, k, l, t, 7, FSC_F32, 100, d_labels, &st, NULL, NULL));
    CK(cudaMemcpy(labels, d_labels, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost));

    /* every clique one label, and the k labels distinct */
    int ok = 1, seen[64] = {0};
    for (int c = 0; c < k && ok; ++c) {
        const int lab = labels[(int64_t)c * s];
        if (lab < 0 || lab >= k || seen[lab]++) ok = 0;
        for (int64_t v = (int64_t)c * s; v < (int64_t)(c + 1) * s; ++v)
            if (labels[v] != lab) ok = 0;
    }
    printf("n = %lld, k = %d, l = %d, t = %d: %d Lloyd iterations, inertia %.3e, cliques recovered: %s\n",
           (long long)n, k, l, t, st.iterations, st.inertia, ok ? "yes" : "no");

    FK(fsc_destroy_graph(g));
    CK(cudaFree(d_row_ptr));
    CK(cudaFree(d_col));
    CK(cudaFree(d_labels));
    free(row_ptr);
    free(col);
    free(labels);
    return ok ? 0 : 1;
}
