/* A plain C11 caller of the library (include/frnn.h): a self-query of five
 * points on a line from host memory.  Exit status 0: results as expected;
 * 3: no usable CUDA device (frnn_create failed cleanly); 1: wrong result or
 * another error. */
#include <stdio.h>

#include "frnn.h"

int main(void) {
    frnn_ctx* ctx = NULL;
    frnn_status s = frnn_create(&ctx, NULL, 0);
    if (s != FRNN_OK) {
        printf("frnn_create: %d (%s)\n", (int)s, frnn_last_error(NULL));
        return ctx == NULL ? 3 : 1;
    }
    /* D = 1; r = 0.25: pairs (0, 1) at 0.125 and (1, 2) at 0.25 (inclusive) */
    const float pts[5] = {0.0f, 0.125f, 0.375f, 2.0f, 4.0f};
    enum { N = 5, K = 2 };
    int32_t counts[N], idx[N * K];
    float dist2[N * K];
    s = frnn_self_query_host(ctx, pts, N, 1, 0.25f, K, 0, counts, idx, dist2);
    if (s == FRNN_OK) s = frnn_sync(ctx);
    if (s != FRNN_OK) {
        printf("query: %d (%s)\n", (int)s, frnn_last_error(ctx));
        frnn_destroy(ctx);
        return 1;
    }
    const int32_t want_counts[N] = {1, 2, 1, 0, 0};
    const int32_t want_idx[N * K] = {1, -1, 0, 2, 1, -1, -1, -1, -1, -1};
    int ok = 1;
    for (int i = 0; i < N; ++i) ok &= counts[i] == want_counts[i];
    for (int i = 0; i < N * K; ++i) ok &= idx[i] == want_idx[i];
    ok &= dist2[0] == 0.015625f && dist2[2] == 0.015625f && dist2[3] == 0.0625f;
    printf("%s\n", ok ? "ok" : "wrong result");
    frnn_destroy(ctx);
    return ok ? 0 : 1;
}
