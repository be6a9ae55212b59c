/*
 * A plain C caller of libch.so, written against include/ch.h only: the three
 * steps of the hull path (ch_reduce, then ch_chain, then ch_hull, each with
 * the workspace its size query asks for) and the chain step without a
 * workspace (ch_chain_noalloc), on points read from a text file.
 *
 * Input file:  "n p" then n lines "x y".
 * Output (stdout): "L x ly hy" for every column, "lower x y" / "upper x y"
 * for the chains of ch_chain, "nlower x y" / "nupper x y" for those of
 * ch_chain_noalloc, "hull x y" for every hull vertex, then "status s" (the
 * value of ch_sync_status) and "ok".  Exit status 0 on success.
 */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "ch.h"

#define CK(call)                                                                   \
    do {                                                                           \
        int rc_ = (int)(call);                                                     \
        if (rc_ != 0) {                                                            \
            fprintf(stderr, "%s failed: %d (line %d)\n", #call, rc_, __LINE__);    \
            return 1;                                                              \
        }                                                                          \
    } while (0)

static void *dalloc(size_t bytes)
{
    void *p = NULL;
    if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess)
        return NULL;
    return p;
}

int main(int argc, char **argv)
{
    if (argc != 2) {
        fprintf(stderr, "usage: %s points.txt\n", argv[0]);
        return 2;
    }
    FILE *f = fopen(argv[1], "r");
    if (!f)
        return 2;
    long long n = 0;
    int p = 0;
    if (fscanf(f, "%lld %d", &n, &p) != 2 || n < 0 || p < 1)
        return 2;
    int32_t *pts = (int32_t *)malloc((size_t)(n ? n : 1) * 8);
    for (long long i = 0; i < n; ++i)
        if (fscanf(f, "%d %d", &pts[2 * i], &pts[2 * i + 1]) != 2)
            return 2;
    fclose(f);

    size_t ws_r = 0, ws_c = 0, ws_h = 0;
    CK(ch_reduce_workspace_size(n, p, &ws_r));
    CK(ch_chain_workspace_size(p, &ws_c));
    CK(ch_hull_workspace_size(p, &ws_h));
    const size_t mask_words = ((size_t)p + 31) / 32;
    int32_t *d_pts = (int32_t *)dalloc((size_t)n * 8);
    int32_t *d_L = (int32_t *)dalloc((size_t)p * 8);
    int32_t *d_lo = (int32_t *)dalloc((size_t)p * 8), *d_up = (int32_t *)dalloc((size_t)p * 8);
    int32_t *d_nlo = (int32_t *)dalloc((size_t)p * 8), *d_nup = (int32_t *)dalloc((size_t)p * 8);
    int32_t *d_cnt = (int32_t *)dalloc(8), *d_ncnt = (int32_t *)dalloc(8);
    uint32_t *d_mask = (uint32_t *)dalloc(mask_words * 4);
    int32_t *d_hull = (int32_t *)dalloc((size_t)p * 16), *d_hc = (int32_t *)dalloc(4);
    void *w_r = dalloc(ws_r), *w_c = dalloc(ws_c), *w_h = dalloc(ws_h);
    if (!d_pts || !d_L || !d_lo || !d_up || !d_nlo || !d_nup || !d_cnt || !d_ncnt || !d_mask ||
        !d_hull || !d_hc || !w_r || !w_c || !w_h)
        return 3;
    CK(cudaMemcpy(d_pts, pts, (size_t)n * 8, cudaMemcpyHostToDevice));

    /* the three steps, stream-ordered on the legacy default stream */
    CK(ch_reduce(d_pts, n, p, d_L, w_r, ws_r, NULL));
    CK(ch_chain(d_L, p, d_lo, d_up, d_cnt, d_mask, w_c, ws_c, NULL));
    CK(ch_hull(d_lo, d_up, d_cnt, p, d_hull, d_hc, w_h, ws_h, NULL));
    /* the chain step again, with the library's own scratch */
    CK(ch_chain_noalloc(d_L, p, d_nlo, d_nup, d_ncnt, NULL, NULL));
    const int status = ch_sync_status(NULL);

    int32_t *L = (int32_t *)malloc((size_t)p * 8), *lo = (int32_t *)malloc((size_t)p * 8);
    int32_t *up = (int32_t *)malloc((size_t)p * 8), *nlo = (int32_t *)malloc((size_t)p * 8);
    int32_t *nup = (int32_t *)malloc((size_t)p * 8), *hull = (int32_t *)malloc((size_t)p * 16);
    int32_t cnt[2], ncnt[2], hc = 0;
    CK(cudaMemcpy(L, d_L, (size_t)p * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(cnt, d_cnt, 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(ncnt, d_ncnt, 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&hc, d_hc, 4, cudaMemcpyDeviceToHost));
    for (int k = 0; k < 2; ++k)
        if (cnt[k] < 0 || cnt[k] > p || ncnt[k] < 0 || ncnt[k] > p)
            return 4;
    if (hc < 0 || hc > 2 * p)
        return 4;
    CK(cudaMemcpy(lo, d_lo, (size_t)cnt[0] * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(up, d_up, (size_t)cnt[1] * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(nlo, d_nlo, (size_t)ncnt[0] * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(nup, d_nup, (size_t)ncnt[1] * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hull, d_hull, (size_t)hc * 8, cudaMemcpyDeviceToHost));

    for (int x = 0; x < p; ++x)
        printf("L %d %d %d\n", x + 1, L[2 * x], L[2 * x + 1]);
    for (int i = 0; i < cnt[0]; ++i)
        printf("lower %d %d\n", lo[2 * i], lo[2 * i + 1]);
    for (int i = 0; i < cnt[1]; ++i)
        printf("upper %d %d\n", up[2 * i], up[2 * i + 1]);
    for (int i = 0; i < ncnt[0]; ++i)
        printf("nlower %d %d\n", nlo[2 * i], nlo[2 * i + 1]);
    for (int i = 0; i < ncnt[1]; ++i)
        printf("nupper %d %d\n", nup[2 * i], nup[2 * i + 1]);
    for (int i = 0; i < hc; ++i)
        printf("hull %d %d\n", hull[2 * i], hull[2 * i + 1]);
    printf("status %d\nok\n", status);
    return 0;
}
