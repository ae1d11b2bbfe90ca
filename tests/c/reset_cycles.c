/*
 * Three create / cluster / destroy cycles of the disjoint-cliques problem (see
 * examples/cluster_cliques.c) with cudaDeviceReset between them: the library's per-device state
 * (memory pool, status word, launch attributes) belongs to the context it was made in and must be
 * rebuilt in the next one.  Each cycle also runs fsc_embed + fsc_kmeans without stats (so the
 * k-means status goes to the library's status word) and reads it back with fsc_sync_status.
 * Exit status 0 when every cycle recovers the cliques and every call succeeds.
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

static int cliques_ok(const int32_t* labels, int k, int s) {
    int seen[64] = {0};
    for (int c = 0; c < k; ++c) {
        const int lab = labels[(int64_t)c * s];
        if (lab < 0 || lab >= k || seen[lab]++) return 0;
        for (int64_t v = (int64_t)c * s; v < (int64_t)(c + 1) * s; ++v)
            if (labels[v] != lab) return 0;
    }
    return 1;
}

static int cycle(const int64_t* row_ptr, const int32_t* col, int64_t n, int64_t nnz, int k, int s, int32_t* labels) {
    int64_t* d_row_ptr;
    int32_t *d_col, *d_labels;
    float* d_emb;
    CK(cudaMalloc((void**)&d_row_ptr, (size_t)(n + 1) * sizeof(int64_t)));
    CK(cudaMalloc((void**)&d_col, (size_t)nnz * sizeof(int32_t)));
    CK(cudaMalloc((void**)&d_labels, (size_t)n * sizeof(int32_t)));
    CK(cudaMalloc((void**)&d_emb, (size_t)n * 4 * sizeof(float)));
    CK(cudaMemcpy(d_row_ptr, row_ptr, (size_t)(n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_col, col, (size_t)nnz * sizeof(int32_t), cudaMemcpyHostToDevice));
    fsc_graph* g = NULL;
    FK(fsc_create_graph(n, nnz, d_row_ptr, d_col, NULL, FSC_COPY, NULL, &g));
    /* asynchronous embed + k-means without stats: the status goes to the library's status word */
    FK(fsc_embed(g, 3, 30, 7, FSC_F32, d_emb, NULL, NULL));
    FK(fsc_kmeans(d_emb, n, 3, 4, k, 7, 100, d_labels, NULL, NULL, NULL, NULL));
    FK(fsc_sync_status(NULL));
    CK(cudaMemcpy(labels, d_labels, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (!cliques_ok(labels, k, s)) return 1;
    fsc_kmeans_stats st;
    FK(fsc_cluster(g, k, 3, 30, 9, FSC_F32, 100, d_labels, &st, NULL, NULL));
    CK(cudaMemcpy(labels, d_labels, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (!cliques_ok(labels, k, s)) return 1;
    FK(fsc_destroy_graph(g));
    CK(cudaFree(d_row_ptr));
    CK(cudaFree(d_col));
    CK(cudaFree(d_labels));
    CK(cudaFree(d_emb));
    return 0;
}

int main(void) {
    const int k = 8, s = 64;
    const int64_t n = (int64_t)k * s, nnz = n * (s - 1);
    int64_t* row_ptr = (int64_t*)malloc((size_t)(n + 1) * sizeof(int64_t));
    int32_t* col = (int32_t*)malloc((size_t)nnz * sizeof(int32_t));
    int32_t* labels = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    if (!row_ptr || !col || !labels) return 4;
    int64_t p = 0;
    for (int64_t v = 0; v < n; ++v) {
        row_ptr[v] = p;
        const int64_t c0 = v / s * s;
        for (int64_t u = c0; u < c0 + s; ++u)
            if (u != v) col[p++] = (int32_t)u;
    }
    row_ptr[n] = p;
    int rc = 0;
    for (int c = 0; c < 3 && rc == 0; ++c) {
        rc = cycle(row_ptr, col, n, nnz, k, s, labels);
        printf("cycle %d: %s\n", c, rc == 0 ? "cliques recovered" : "failed");
        if (rc == 0) CK(cudaDeviceReset());
    }
    free(row_ptr);
    free(col);
    free(labels);
    return rc;
}
