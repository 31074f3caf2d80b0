/* A plain C program on the library's C ABI -- test infrastructure only.  It sketches a small
 * CSR batch held in host memory through dm_sketch_host (k minhash keys, seed 1) and prints one
 * key per line in hexadecimal, set by set.  Usage: c_abi_example k < batch.txt, where batch.txt
 * holds n, then n + 1 indptr values, then indptr[n] (index, weight) pairs. */
#include <inttypes.h>
#include <stdio.h>
#include <stdlib.h>

#include "dartminhash.h"

int main(int argc, char **argv) {
    int k = argc > 1 ? atoi(argv[1]) : 64;
    long long n = 0;
    if (scanf("%lld", &n) != 1 || n < 0) return 2;
    int64_t *indptr = malloc(sizeof(int64_t) * (size_t)(n + 1));
    for (long long s = 0; s <= n; ++s)
        if (scanf("%" SCNd64, &indptr[s]) != 1) return 2;
    const int64_t nnz = indptr[n];
    uint32_t *indices = malloc(sizeof(uint32_t) * (size_t)(nnz > 0 ? nnz : 1));
    float *weights = malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    for (int64_t i = 0; i < nnz; ++i)
        if (scanf("%" SCNu32 " %f", &indices[i], &weights[i]) != 2) return 2;
    uint64_t *keys = malloc(sizeof(uint64_t) * (size_t)(n * k > 0 ? n * k : 1));
    dm_ctx *ctx = NULL;
    int rc = dm_create(&ctx, 0, 0);
    if (rc != DM_OK) {
        fprintf(stderr, "dm_create: %s\n", dm_strerror(rc));
        return 1;
    }
    rc = dm_sketch_host(ctx, indptr, indices, weights, n, k, 0, 1, keys, NULL, NULL);
    if (rc == DM_OK) rc = dm_sync_status(ctx, NULL);
    if (rc != DM_OK) {
        fprintf(stderr, "dm_sketch_host: %s\n", dm_strerror(rc));
        dm_destroy(ctx);
        return 1;
    }
    for (long long i = 0; i < n * k; ++i) printf("%016" PRIx64 "\n", keys[i]);
    dm_destroy(ctx);
    free(keys);
    free(weights);
    free(indices);
    free(indptr);
    return 0;
}
