/* The C ABI used from plain C99 (no C++ and no Python): compress a small
 * Gaussian matrix given only through an entry callback, read its figures,
 * round-trip a checkpoint, check the documented error codes, free.  Needs no
 * GPU (compression runs on the host). */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "gofmm.h"

typedef struct {
    int64_t n;
    const double* x; /* n x 3 */
} points;

static int gaussian(void* ctx, const int64_t* I, int64_t nI, const int64_t* J, int64_t nJ, double* out) {
    const points* p = (const points*)ctx;
    for (int64_t a = 0; a < nI; ++a)
        for (int64_t b = 0; b < nJ; ++b) {
            double d2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double t = p->x[3 * I[a] + k] - p->x[3 * J[b] + k];
                d2 += t * t;
            }
            out[a * nJ + b] = exp(-d2 / (2.0 * 0.3 * 0.3)) + (I[a] == J[b] ? 1e-3 : 0.0);
        }
    return 0;
}

int main(int argc, char** argv) {
    const char* ckpt = argc > 1 ? argv[1] : "abi_from_c.bin";
    const int64_t n = 700;
    double* x = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    uint64_t s = 12345;
    for (int64_t i = 0; i < 3 * n; ++i) { /* a small LCG: any points will do */
        s = s * 6364136223846793005ULL + 1442695040888963407ULL;
        x[i] = (double)(s >> 11) / 9007199254740992.0;
    }
    points pts = {n, x};
    gofmm_entries K;
    memset(&K, 0, sizeof K);
    K.kind = GOFMM_GEN_CALLBACK;
    K.n = n;
    K.fn = gaussian;
    K.ctx = &pts;
    gofmm_params p;
    gofmm_default_params(&p);
    p.leaf_size = 32;
    p.max_rank = 32;
    gofmm_handle* h = NULL;
    int rc = gofmm_compress(&K, &p, &h);
    if (rc != GOFMM_OK || !h) { printf("compress failed: %d %s\n", rc, gofmm_last_error()); return 1; }
    gofmm_stats_t st;
    if (gofmm_stats(h, &st) != GOFMM_OK || st.n != n || st.n_leaves < 2 || st.max_rank < 1 || st.max_rank > 32) {
        printf("bad stats\n");
        return 1;
    }
    if (gofmm_export(h, ckpt) != GOFMM_OK) { printf("export failed: %s\n", gofmm_last_error()); return 1; }
    gofmm_handle* h2 = NULL;
    if (gofmm_import(ckpt, &K, GOFMM_CACHE_BLOCKS, 0, &h2) != GOFMM_OK || !h2) {
        printf("import failed: %s\n", gofmm_last_error());
        return 1;
    }
    gofmm_stats_t st2;
    gofmm_stats(h2, &st2);
    if (st2.near_pairs != st.near_pairs || st2.far_pairs != st.far_pairs || st2.skel_total != st.skel_total) {
        printf("checkpoint changed the structure\n");
        return 1;
    }
    /* documented errors */
    p.leaf_size = 0;
    gofmm_handle* bad = NULL;
    if (gofmm_compress(&K, &p, &bad) != GOFMM_ERR_ARG || bad != NULL || strlen(gofmm_last_error()) == 0) {
        printf("missing ERR_ARG\n");
        return 1;
    }
    if (gofmm_set_tc_config(h, GOFMM_PREC_BF16X3, 100, GOFMM_SCHED_FUSED, GOFMM_ORDER_CRITICAL) != GOFMM_ERR_ARG) {
        printf("missing ERR_ARG for a bad piece height\n");
        return 1;
    }
    gofmm_free(h2);
    gofmm_free(h);
    free(x);
    printf("c abi ok: n %lld, leaves %lld, near pairs %lld, far pairs %lld, max rank %lld\n", (long long)st.n,
           (long long)st.n_leaves, (long long)st.near_pairs, (long long)st.far_pairs, (long long)st.max_rank);
    return 0;
}
