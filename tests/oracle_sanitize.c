/* Sanitizer run of the CPU oracle (test infrastructure, built and run by
 * tests/test_oracle_sanitize.py with AddressSanitizer and
 * UndefinedBehaviorSanitizer).  Random and edge-case inputs go through every
 * entry point of oracle.c with heap buffers of exactly the documented
 * capacity, so any read or write past a buffer, any signed overflow and any
 * leak ends the run; the independent routes to the same hull (sort + Andrew
 * on all points, Andrew on the Lemma 1 polyline, Melkman on that polyline,
 * brute force from the edge definition, and Steps 1-2 on translated points)
 * must agree, and the bit array M must count the valid columns. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

int oracle_reduce(const int32_t *pts, int64_t n, int32_t p, int32_t *L);
int oracle_reduce_from(const int32_t *pts, int64_t n, int32_t p, const int32_t *Linit, int32_t *L);
int64_t oracle_chain(const int32_t *L, int32_t p, int32_t *lower, int32_t *upper);
void oracle_mask(const int32_t *L, int32_t p, uint32_t *M);
int64_t oracle_polyline(const int32_t *L, int32_t p, int32_t *out);
int64_t oracle_hull_points(const int32_t *pts, int64_t n, int32_t *out);
int64_t oracle_hull_chain(const int32_t *L, int32_t p, int32_t *out);
int64_t oracle_hull_brute(const int32_t *pts, int64_t n, int32_t *out);
int oracle_polygon_init(const int32_t *poly, int32_t m, int32_t p, int32_t *Linit);
void oracle_chain_from(const int32_t *L, const int32_t *Linit, int32_t p, int32_t *lower,
                       int32_t *upper, int64_t *cnt);
void oracle_best_offsets(const int32_t *H, int64_t h, int K, int sub, int rounds, float *out);
int64_t oracle_melkman(const int32_t *v, int64_t m, int32_t *out);
int64_t oracle_hull_box(const int32_t *pts, int64_t n, int32_t *out);
void oracle_reduce_rows(const int32_t *L, int32_t p, int32_t *R);

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;

static uint64_t next64(void) /* xorshift64 */
{
    rng_state ^= rng_state << 13;
    rng_state ^= rng_state >> 7;
    rng_state ^= rng_state << 17;
    return rng_state;
}

static int64_t rnd(int64_t lo, int64_t hi) /* uniform in [lo, hi] */
{
    return lo + (int64_t)(next64() % (uint64_t)(hi - lo + 1));
}

static int32_t *pairs(int64_t k) /* k int32 pairs; malloc(0) avoided */
{
    return (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(k > 0 ? k : 0) + (k > 0 ? 0 : 1));
}

static int same(const int32_t *a, int64_t na, const int32_t *b, int64_t nb)
{
    return na == nb && (na == 0 || memcmp(a, b, sizeof(int32_t) * 2 * (size_t)na) == 0);
}

#define CHECK(cond, ...)                                                                           \
    do {                                                                                           \
        if (!(cond)) {                                                                             \
            fprintf(stderr, "trial %d: ", trial);                                                  \
            fprintf(stderr, __VA_ARGS__);                                                          \
            fprintf(stderr, "\n");                                                                 \
            return 1;                                                                              \
        }                                                                                          \
    } while (0)

static int one_trial(int trial)
{
    const int32_t p = (int32_t)rnd(1, trial % 3 == 0 ? 8 : 300);
    const int64_t n = rnd(0, trial % 5 == 0 ? 3 : 400);
    int32_t *P = pairs(n);
    const int line = trial % 7 == 0; /* all points on one line now and then */
    for (int64_t i = 0; i < n; ++i) {
        P[2 * i] = (int32_t)rnd(1, p);
        P[2 * i + 1] = line ? P[2 * i] : (int32_t)rnd(1, p);
    }
    int32_t *L = pairs(p);
    CHECK(oracle_reduce(P, n, p, L) == 0, "reduce failed");

    int32_t *lo = pairs(p), *up = pairs(p);
    const int64_t s = oracle_chain(L, p, lo, up);
    uint32_t *M = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)((p + 31) / 32));
    oracle_mask(L, p, M);
    int64_t bits = 0;
    for (int32_t w = 0; w < (p + 31) / 32; ++w)
        bits += __builtin_popcount(M[w]);
    CHECK(bits == s, "mask counts %lld of %lld columns", (long long)bits, (long long)s);

    int32_t *poly = pairs(2 * (int64_t)p); /* s <= 2p */
    const int64_t sp = oracle_polyline(L, p, poly);
    CHECK(sp <= 2 * (int64_t)p, "polyline longer than 2p");

    int32_t *h1 = pairs(n);
    const int64_t k1 = oracle_hull_points(P, n, h1);
    int32_t *h2 = pairs(2 * (int64_t)p);
    const int64_t k2 = oracle_hull_chain(L, p, h2);
    CHECK(same(h1, k1, h2, k2), "hull of the chains differs from the hull of the points");
    int32_t *h3 = pairs((sp > 0 ? sp : 1) + 1);
    const int64_t k3 = oracle_melkman(poly, sp, h3);
    CHECK(same(h1, k1, h3, k3), "Melkman on the polyline differs");
    if (n <= 64) {
        int32_t *h4 = pairs(n);
        const int64_t k4 = oracle_hull_brute(P, n, h4);
        CHECK(same(h1, k1, h4, k4), "brute force differs");
        free(h4);
    }

    int32_t *R = pairs(p);
    oracle_reduce_rows(L, p, R);

    /* culling start array from the hull itself, then the culled reduction */
    int32_t *Li = pairs(p), *L2 = pairs(p), *lo2 = pairs(p), *up2 = pairs(p);
    int64_t cnt[2];
    CHECK(oracle_polygon_init(h1, (int32_t)k1, p, Li) == 0, "polygon_init failed");
    CHECK(oracle_reduce_from(P, n, p, Li, L2) == 0, "reduce_from failed");
    oracle_chain_from(L2, Li, p, lo2, up2, cnt);
    CHECK(cnt[0] <= s && cnt[1] <= s, "culled chains longer than the plain ones");
    if (k1 >= 1) {
        float off[16];
        oracle_best_offsets(h1, k1, 16, 3, 2, off);
        for (int k = 0; k < 16; ++k)
            CHECK(off[k] >= -1.0f && off[k] <= 1.0f, "label offset out of range");
    }

    /* Steps 1-2: the same points translated anywhere in int32 */
    if (n > 0) {
        const int64_t dx = rnd(-2147483647ll, 2147483647ll - p), dy = rnd(-2147483647ll, 2147483647ll - p);
        int32_t *Q = pairs(n);
        int64_t xmin = INT64_MAX, xmax = INT64_MIN, ymin = INT64_MAX, ymax = INT64_MIN;
        for (int64_t i = 0; i < n; ++i) {
            Q[2 * i] = (int32_t)(P[2 * i] + dx);
            Q[2 * i + 1] = (int32_t)(P[2 * i + 1] + dy);
            if (Q[2 * i] < xmin) xmin = Q[2 * i];
            if (Q[2 * i] > xmax) xmax = Q[2 * i];
            if (Q[2 * i + 1] < ymin) ymin = Q[2 * i + 1];
            if (Q[2 * i + 1] > ymax) ymax = Q[2 * i + 1];
        }
        const int64_t side = (xmax - xmin < ymax - ymin ? xmax - xmin : ymax - ymin) + 1;
        int32_t *hb = pairs(2 * side + 2);
        const int64_t kb = oracle_hull_box(Q, n, hb);
        CHECK(kb == k1, "Steps 1-2 hull has %lld vertices, not %lld", (long long)kb, (long long)k1);
        for (int64_t i = 0; i < kb; ++i)
            CHECK(hb[2 * i] == (int32_t)(h1[2 * i] + dx) && hb[2 * i + 1] == (int32_t)(h1[2 * i + 1] + dy),
                  "Steps 1-2 hull is not the translated hull");
        free(hb);
        free(Q);
    }

    free(P), free(L), free(lo), free(up), free(M), free(poly), free(h1), free(h2), free(h3), free(R);
    free(Li), free(L2), free(lo2), free(up2);
    return 0;
}

int main(int argc, char **argv)
{
    const int trials = argc > 1 ? atoi(argv[1]) : 3000;
    for (int t = 0; t < trials; ++t)
        if (one_trial(t))
            return 1;
    /* a point outside [1,p]^2 is an error, not an out-of-bounds write */
    int32_t bad[4] = {1, 1, 9, 2}, L[16];
    if (oracle_reduce(bad, 2, 8, L) == 0) {
        fprintf(stderr, "out-of-range point accepted\n");
        return 1;
    }
    printf("oracle sanitize ok: %d trials\n", trials);
    return 0;
}
