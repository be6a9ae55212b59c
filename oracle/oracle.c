/*
 * Plain, slow, obviously-correct CPU oracle for the integer convex-hull
 * preconditioner of Cadenas & Megson, "An Empirical Evaluation of
 * Preconditioning Data for Accelerating Convex Hull Computations".
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this
 * file; only the tests, the smoke check and the benchmark's CPU-baseline leg
 * do.  It shares no code, header or table with the CUDA library.
 *
 * Conventions (readings of the paper, each one stated where it is used):
 *   - points are int32 pairs (x, y), 1 <= x, y <= p (Section 2.1, the square
 *     of side p); anything else is rejected with ORC_ERR_RANGE.
 *   - L is stored 0-based: column x lives at L[2*(x-1)], L[2*(x-1)+1]
 *     (the paper indexes L[1..p]).
 *   - hulls are listed as strict vertices (collinear points dropped),
 *     counter-clockwise, starting at the lexicographic minimum (min x, then
 *     min y).  The paper says collinear points are removed (Section 2.1 and
 *     the Appendix) and fixes no start vertex or orientation.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_RANGE (-2)

/* ------------------------------------------------------------------------ */
/* Algorithm 1 (Reduction of Points), Section 2.1.                          */
/* L starts as p copies of (p+1, -1); each point (x, y) replaces L[x] by    */
/* (min(y, L[x].ly), max(y, L[x].hy)).                                      */
/* ------------------------------------------------------------------------ */
int oracle_reduce(const int32_t *pts, int64_t n, int32_t p, int32_t *L)
{
    if (p < 1 || n < 0 || (n > 0 && pts == NULL) || L == NULL)
        return ORC_ERR_ARG;
    for (int64_t i = 0; i < p; ++i) {
        L[2 * i] = p + 1;
        L[2 * i + 1] = -1;
    }
    for (int64_t k = 0; k < n; ++k) {
        int32_t x = pts[2 * k], y = pts[2 * k + 1];
        if (x < 1 || x > p || y < 1 || y > p)
            return ORC_ERR_RANGE;
        int32_t yv = L[2 * (x - 1)], yu = L[2 * (x - 1) + 1];
        int32_t ly = y < yv ? y : yv;
        int32_t hy = y > yu ? y : yu;
        L[2 * (x - 1)] = ly;
        L[2 * (x - 1) + 1] = hy;
    }
    return ORC_OK;
}

/* Algorithm 1 with a caller-given starting array instead of (p+1, -1).     */
/* Used for the culled reduction: the update rule is the same.              */
int oracle_reduce_from(const int32_t *pts, int64_t n, int32_t p,
                       const int32_t *Linit, int32_t *L)
{
    if (p < 1 || n < 0 || (n > 0 && pts == NULL) || L == NULL || Linit == NULL)
        return ORC_ERR_ARG;
    memcpy(L, Linit, sizeof(int32_t) * 2 * (size_t)p);
    for (int64_t k = 0; k < n; ++k) {
        int32_t x = pts[2 * k], y = pts[2 * k + 1];
        if (x < 1 || x > p || y < 1 || y > p)
            return ORC_ERR_RANGE;
        int32_t yv = L[2 * (x - 1)], yu = L[2 * (x - 1) + 1];
        L[2 * (x - 1)] = y < yv ? y : yv;
        L[2 * (x - 1) + 1] = y > yu ? y : yu;
    }
    return ORC_OK;
}

/* An entry is valid when it differs from the initial (p+1, -1)            */
/* (Lemma 1: "one different to (p+1, -1)").                                 */
static int entry_valid(const int32_t *L, int32_t p, int64_t i)
{
    return !(L[2 * i] == p + 1 && L[2 * i + 1] == -1);
}

/* ------------------------------------------------------------------------ */
/* Lower and upper chains: scanning L along x (Lemma 1) and keeping the     */
/* valid entries gives (x, ly) and (x, hy) in increasing x.  Returns s_cols */
/* (number of valid columns); both chains have that many points.            */
/* ------------------------------------------------------------------------ */
int64_t oracle_chain(const int32_t *L, int32_t p, int32_t *lower, int32_t *upper)
{
    int64_t s = 0;
    for (int64_t i = 0; i < p; ++i) {
        if (!entry_valid(L, p, i))
            continue;
        lower[2 * s] = (int32_t)(i + 1);
        lower[2 * s + 1] = L[2 * i];
        upper[2 * s] = (int32_t)(i + 1);
        upper[2 * s + 1] = L[2 * i + 1];
        ++s;
    }
    return s;
}

/* Bit array M of the "Extraction using an array of bits" passage: column i */
/* (1-based) is bit (i-1) & 31 of word (i-1) >> 5, set iff L[i] is valid.   */
void oracle_mask(const int32_t *L, int32_t p, uint32_t *M)
{
    int64_t words = ((int64_t)p + 31) / 32;
    memset(M, 0, sizeof(uint32_t) * (size_t)words);
    for (int64_t i = 1; i <= p; ++i)
        if (entry_valid(L, p, i - 1))
            M[(i - 1) >> 5] |= (uint32_t)1 << ((i - 1) & 31);
}

/* Lemma 1 polyline: for each valid column, (i, ly) then (i, hy) when the   */
/* two differ; consecutive columns are joined hy -> next ly.  Returns the   */
/* number of points s written to out (s <= 2p).                             */
int64_t oracle_polyline(const int32_t *L, int32_t p, int32_t *out)
{
    int64_t s = 0;
    for (int64_t i = 0; i < p; ++i) {
        if (!entry_valid(L, p, i))
            continue;
        out[2 * s] = (int32_t)(i + 1);
        out[2 * s + 1] = L[2 * i];
        ++s;
        if (L[2 * i + 1] != L[2 * i]) {
            out[2 * s] = (int32_t)(i + 1);
            out[2 * s + 1] = L[2 * i + 1];
            ++s;
        }
    }
    return s;
}

/* ------------------------------------------------------------------------ */
/* Hull: Andrew's monotone chain (a Graham-scan variant) on points that are */
/* already in increasing (x, y) order with no duplicates.                   */
/* ------------------------------------------------------------------------ */
static int64_t cross3(const int32_t *o, const int32_t *a, const int32_t *b)
{
    return ((int64_t)a[0] - o[0]) * ((int64_t)b[1] - o[1]) -
           ((int64_t)a[1] - o[1]) * ((int64_t)b[0] - o[0]);
}

static int64_t andrew_sorted(const int32_t *q, int64_t m, int32_t *out)
{
    if (m == 0)
        return 0;
    if (m == 1) {
        out[0] = q[0];
        out[1] = q[1];
        return 1;
    }
    int32_t *h = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(2 * m + 2));
    int64_t k = 0;
    /* lower hull, left to right: keep strict counter-clockwise turns */
    for (int64_t i = 0; i < m; ++i) {
        while (k >= 2 && cross3(&h[2 * (k - 2)], &h[2 * (k - 1)], &q[2 * i]) <= 0)
            --k;
        h[2 * k] = q[2 * i];
        h[2 * k + 1] = q[2 * i + 1];
        ++k;
    }
    /* upper hull, right to left */
    int64_t t = k + 1;
    for (int64_t i = m - 2; i >= 0; --i) {
        while (k >= t && cross3(&h[2 * (k - 2)], &h[2 * (k - 1)], &q[2 * i]) <= 0)
            --k;
        h[2 * k] = q[2 * i];
        h[2 * k + 1] = q[2 * i + 1];
        ++k;
    }
    /* the last point repeats the first */
    int64_t hn = k - 1;
    memcpy(out, h, sizeof(int32_t) * 2 * (size_t)hn);
    free(h);
    return hn;
}

static int cmp_xy(const void *a, const void *b)
{
    const int32_t *u = (const int32_t *)a, *v = (const int32_t *)b;
    if (u[0] != v[0])
        return u[0] < v[0] ? -1 : 1;
    if (u[1] != v[1])
        return u[1] < v[1] ? -1 : 1;
    return 0;
}

/* Hull of all n points: sort, drop duplicates, Andrew.  This is the       */
/* paper's "hull on the original n points" (t_n in Section 3).             */
int64_t oracle_hull_points(const int32_t *pts, int64_t n, int32_t *out)
{
    if (n <= 0)
        return 0;
    int32_t *q = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)n);
    memcpy(q, pts, sizeof(int32_t) * 2 * (size_t)n);
    qsort(q, (size_t)n, 2 * sizeof(int32_t), cmp_xy);
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (m > 0 && q[2 * (m - 1)] == q[2 * i] && q[2 * (m - 1) + 1] == q[2 * i + 1])
            continue;
        q[2 * m] = q[2 * i];
        q[2 * m + 1] = q[2 * i + 1];
        ++m;
    }
    int64_t h = andrew_sorted(q, m, out);
    free(q);
    return h;
}

/* Hull of the reduced set: the Lemma 1 polyline is already in (x, y)      */
/* order, so Andrew's scan runs on it with no sort (the paper's point that */
/* L can be "directly pipelined" into a hull algorithm).                   */
int64_t oracle_hull_chain(const int32_t *L, int32_t p, int32_t *out)
{
    int32_t *q = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(2 * (int64_t)p + 1));
    int64_t s = oracle_polyline(L, p, q);
    int64_t h = andrew_sorted(q, s, out);
    free(q);
    return h;
}

/* ------------------------------------------------------------------------ */
/* Brute force, O(m^3) on the distinct points, from the definition of a    */
/* hull edge: the directed pair (a, b), a != b, is an edge of the          */
/* counter-clockwise hull iff every point c is strictly left of a->b or    */
/* lies on the closed segment [a, b].  Strict vertices are the edge        */
/* endpoints; the list is walked along the edges from the lexicographic    */
/* minimum.  Independent of Andrew's algorithm.  Small inputs only.        */
/* ------------------------------------------------------------------------ */
int64_t oracle_hull_brute(const int32_t *pts, int64_t n, int32_t *out)
{
    if (n <= 0)
        return 0;
    int32_t *q = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)n);
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        int dup = 0;
        for (int64_t j = 0; j < m; ++j)
            if (q[2 * j] == pts[2 * i] && q[2 * j + 1] == pts[2 * i + 1]) {
                dup = 1;
                break;
            }
        if (!dup) {
            q[2 * m] = pts[2 * i];
            q[2 * m + 1] = pts[2 * i + 1];
            ++m;
        }
    }
    if (m == 1) {
        out[0] = q[0];
        out[1] = q[1];
        free(q);
        return 1;
    }
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)m);
    for (int64_t a = 0; a < m; ++a) {
        next[a] = -1;
        for (int64_t b = 0; b < m; ++b) {
            if (a == b)
                continue;
            int ok = 1;
            for (int64_t c = 0; c < m && ok; ++c) {
                int64_t cr = cross3(&q[2 * a], &q[2 * b], &q[2 * c]);
                if (cr > 0)
                    continue;
                if (cr < 0) {
                    ok = 0;
                    break;
                }
                /* collinear: c must lie on the closed segment [a, b] */
                int32_t lox = q[2 * a] < q[2 * b] ? q[2 * a] : q[2 * b];
                int32_t hix = q[2 * a] < q[2 * b] ? q[2 * b] : q[2 * a];
                int32_t loy = q[2 * a + 1] < q[2 * b + 1] ? q[2 * a + 1] : q[2 * b + 1];
                int32_t hiy = q[2 * a + 1] < q[2 * b + 1] ? q[2 * b + 1] : q[2 * a + 1];
                if (q[2 * c] < lox || q[2 * c] > hix || q[2 * c + 1] < loy || q[2 * c + 1] > hiy)
                    ok = 0;
            }
            if (ok) {
                next[a] = b;
                break;
            }
        }
    }
    int64_t start = 0;
    for (int64_t i = 1; i < m; ++i)
        if (cmp_xy(&q[2 * i], &q[2 * start]) < 0)
            start = i;
    int64_t h = 0, cur = start;
    do {
        out[2 * h] = q[2 * cur];
        out[2 * h + 1] = q[2 * cur + 1];
        ++h;
        cur = next[cur];
    } while (cur >= 0 && cur != start && h <= m);
    free(next);
    free(q);
    return h;
}

/* ------------------------------------------------------------------------ */
/* Culling polygon -> starting array for Algorithm 1.                      */
/* poly: a convex polygon, strict vertices counter-clockwise from the      */
/* lexicographic minimum (m >= 3), vertices inside [1,p]^2.  For a column  */
/* x strictly inside its x-range, with lower boundary b(x) and upper      */
/* boundary u(x), the                                                      */
/* entry starts at (floor(b(x)) + 1, ceil(u(x)) - 1): a point is left out  */
/* by Algorithm 1's min/max exactly when floor(b)+1 <= y <= ceil(u)-1,     */
/* i.e. when b(x) < y < u(x), strictly inside the polygon.  Columns        */
/* outside the x-range start at (p+1, -1) as in Algorithm 1.               */
/* ------------------------------------------------------------------------ */
static int64_t floor_div(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b) != 0 && a < 0)
        --q;
    return q;
}

static int64_t ceil_div(int64_t a, int64_t b) /* b > 0 */
{
    return -floor_div(-a, b);
}

/* Boundary value at column x along the edge (x0,y0)-(x1,y1), x0 < x1, as  */
/* the rational num/den with den = x1 - x0 > 0.                            */
static void edge_at(const int32_t *v0, const int32_t *v1, int64_t x, int64_t *num, int64_t *den)
{
    *den = (int64_t)v1[0] - v0[0];
    *num = (int64_t)v0[1] * (*den) + ((int64_t)v1[1] - v0[1]) * (x - v0[0]);
}

int oracle_polygon_init(const int32_t *poly, int32_t m, int32_t p, int32_t *Linit)
{
    for (int64_t i = 0; i < p; ++i) {
        Linit[2 * i] = p + 1;
        Linit[2 * i + 1] = -1;
    }
    if (m < 3)
        return ORC_OK;
    /* vertex 0 is the lexicographic minimum; the lower boundary runs       */
    /* counter-clockwise from it to the rightmost vertex (largest x, then  */
    /* largest y), the upper boundary continues from there back to 0.      */
    int32_t r = 0;
    for (int32_t i = 1; i < m; ++i)
        if (poly[2 * i] > poly[2 * r] || (poly[2 * i] == poly[2 * r] && poly[2 * i + 1] > poly[2 * r + 1]))
            r = i;
    int32_t xmin = poly[0], xmax = poly[2 * r];
    /* the interior of the polygon meets only the columns strictly between  */
    /* its extreme x values; the end columns hold boundary points only      */
    for (int64_t x = (int64_t)xmin + 1; x < xmax; ++x) {
        /* lower boundary: the chain 0 -> r, take the lowest y at column x */
        int64_t lo_num = 0, lo_den = 1, hi_num = 0, hi_den = 1;
        int have_lo = 0, have_hi = 0;
        for (int32_t i = 0; i < r; ++i) {
            const int32_t *a = &poly[2 * i], *b = &poly[2 * (i + 1)];
            if (a[0] == b[0]) {
                if (a[0] == x) {
                    int64_t yy = a[1] < b[1] ? a[1] : b[1];
                    if (!have_lo || yy * lo_den < lo_num) { lo_num = yy; lo_den = 1; have_lo = 1; }
                }
                continue;
            }
            if (x < a[0] || x > b[0])
                continue;
            int64_t nu, de;
            edge_at(a, b, x, &nu, &de);
            if (!have_lo || nu * lo_den < lo_num * de) { lo_num = nu; lo_den = de; have_lo = 1; }
        }
        /* upper boundary: the chain r -> m-1 -> 0 (x decreasing) */
        for (int32_t i = r; i < m; ++i) {
            const int32_t *a = &poly[2 * i], *b = &poly[2 * ((i + 1) % m)];
            /* orient the edge left to right */
            const int32_t *l = a[0] <= b[0] ? a : b, *rr = a[0] <= b[0] ? b : a;
            if (l[0] == rr[0]) {
                if (l[0] == x) {
                    int64_t yy = l[1] > rr[1] ? l[1] : rr[1];
                    if (!have_hi || yy * hi_den > hi_num) { hi_num = yy; hi_den = 1; have_hi = 1; }
                }
                continue;
            }
            if (x < l[0] || x > rr[0])
                continue;
            int64_t nu, de;
            edge_at(l, rr, x, &nu, &de);
            if (!have_hi || nu * hi_den > hi_num * de) { hi_num = nu; hi_den = de; have_hi = 1; }
        }
        if (!have_lo || !have_hi)
            continue;
        int64_t lo0 = floor_div(lo_num, lo_den) + 1;
        int64_t hi0 = ceil_div(hi_num, hi_den) - 1;
        Linit[2 * (x - 1)] = (int32_t)lo0;
        Linit[2 * (x - 1) + 1] = (int32_t)hi0;
    }
    return ORC_OK;
}

/* Chains of a culled reduction: column x has a lower point (x, L.ly) when  */
/* ly fell below the start value, an upper point (x, L.hy) when hy rose     */
/* above it.  Returns the counts in cnt[0] (lower), cnt[1] (upper).         */
void oracle_chain_from(const int32_t *L, const int32_t *Linit, int32_t p,
                       int32_t *lower, int32_t *upper, int64_t *cnt)
{
    int64_t nl = 0, nu = 0;
    for (int64_t i = 0; i < p; ++i) {
        if (L[2 * i] < Linit[2 * i]) {
            lower[2 * nl] = (int32_t)(i + 1);
            lower[2 * nl + 1] = L[2 * i];
            ++nl;
        }
        if (L[2 * i + 1] > Linit[2 * i + 1]) {
            upper[2 * nu] = (int32_t)(i + 1);
            upper[2 * nu + 1] = L[2 * i + 1];
            ++nu;
        }
    }
    cnt[0] = nl;
    cnt[1] = nu;
}

/* ------------------------------------------------------------------------ */
/* Training labels of the learned culling proposal (not in the paper).      */
/* For a hull H (strict vertices, counter-clockwise) and K sectors of        */
/* directions [2*pi*k/K - pi/K, 2*pi*k/K + pi/K], choose one direction per   */
/* sector (`sub` evenly spaced candidates) so that the polygon of the hull   */
/* vertices extreme in those directions has the largest area; coordinate    */
/* ascent, `rounds` sweeps from the sector centres.  out[k] = offset of the  */
/* chosen direction from the sector centre in units of pi/K, in [-1, 1].     */
/* ------------------------------------------------------------------------ */
#include <math.h>

static int64_t extreme_vertex(const int32_t *H, int64_t h, double c, double s)
{
    int64_t best = 0;
    double bv = -1e300;
    for (int64_t i = 0; i < h; ++i) {
        double v = c * H[2 * i] + s * H[2 * i + 1];
        if (v > bv) {
            bv = v;
            best = i;
        }
    }
    return best;
}

/* Twice the area of the polygon of the distinct chosen vertices, visited in
 * the hull's counter-clockwise order. */
static double chosen_area2(const int32_t *H, int64_t h, const int64_t *idx, int K)
{
    int64_t sel[64];
    int m = 0;
    for (int k = 0; k < K && m < 64; ++k) {
        int dup = 0;
        for (int j = 0; j < m; ++j)
            if (sel[j] == idx[k])
                dup = 1;
        if (!dup)
            sel[m++] = idx[k];
    }
    /* sort by hull order */
    for (int a = 1; a < m; ++a) {
        int64_t v = sel[a];
        int b = a - 1;
        while (b >= 0 && sel[b] > v) {
            sel[b + 1] = sel[b];
            --b;
        }
        sel[b + 1] = v;
    }
    double s = 0;
    for (int j = 0; j < m; ++j) {
        const int32_t *u = &H[2 * sel[j]], *w = &H[2 * sel[(j + 1) % m]];
        s += (double)u[0] * w[1] - (double)u[1] * w[0];
    }
    (void)h;
    return s;
}

void oracle_best_offsets(const int32_t *H, int64_t h, int K, int sub, int rounds, float *out)
{
    int64_t idx[64];
    double off[64];
    if (K > 64)
        K = 64;
    for (int k = 0; k < K; ++k) {
        off[k] = 0.0;
        if (h == 0) {
            idx[k] = 0;
            continue;
        }
        double a = 2.0 * M_PI * k / K;
        idx[k] = extreme_vertex(H, h, cos(a), sin(a));
    }
    if (h >= 3) {
        for (int r = 0; r < rounds; ++r) {
            for (int k = 0; k < K; ++k) {
                double best_area = -1, best_off = off[k];
                int64_t best_idx = idx[k];
                for (int j = 0; j < sub; ++j) {
                    double o = sub == 1 ? 0.0 : -1.0 + 2.0 * j / (sub - 1);
                    double a = 2.0 * M_PI * k / K + o * M_PI / K;
                    int64_t keep = idx[k];
                    idx[k] = extreme_vertex(H, h, cos(a), sin(a));
                    double ar = chosen_area2(H, h, idx, K);
                    /* prefer the centre on ties */
                    if (ar > best_area + 1e-9 || (ar > best_area - 1e-9 && fabs(o) < fabs(best_off))) {
                        best_area = ar;
                        best_off = o;
                        best_idx = idx[k];
                    }
                    idx[k] = keep;
                }
                off[k] = best_off;
                idx[k] = best_idx;
            }
        }
    }
    for (int k = 0; k < K; ++k)
        out[k] = (float)off[k];
}

/* Labels of B sets: set s = pts[off[s], off[s+1]) of side ps[s]; its hull
 * from Algorithm 1 + Andrew on the reduced set, then oracle_best_offsets. */
int oracle_label_batch(const int32_t *pts, const int64_t *off, const int32_t *ps, int64_t B, int K,
                       int sub, int rounds, float *out, int64_t *hull_sizes)
{
    int32_t *L = NULL, *Hb = NULL;
    int64_t capL = 0;
    for (int64_t s = 0; s < B; ++s) {
        int32_t p = ps[s];
        if ((int64_t)p > capL) {
            free(L);
            free(Hb);
            capL = p;
            L = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)p);
            Hb = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(2 * p + 2));
        }
        int rc = oracle_reduce(pts + 2 * off[s], off[s + 1] - off[s], p, L);
        if (rc != ORC_OK) {
            free(L);
            free(Hb);
            return rc;
        }
        int64_t h = oracle_hull_chain(L, p, Hb);
        if (hull_sizes)
            hull_sizes[s] = h;
        oracle_best_offsets(Hb, h, K, sub, rounds, out + (size_t)s * K);
    }
    free(L);
    free(Hb);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Melkman's on-line hull of a simple polyline, the hull algorithm the     */
/* paper applies to its reduced set in Section 3 (Fig. 10): a deque holds  */
/* the hull of the vertices seen so far, counter-clockwise from its bottom */
/* to its top, with the last vertex at both ends.  A new vertex u that is  */
/* on or inside the hull (left of or on both edges at the deque's ends) is */
/* skipped; otherwise vertices are popped from the top while u is not      */
/* strictly left of the top edge and from the bottom while the bottom edge */
/* is not strictly left-turning into u, and u is pushed at both ends.      */
/* Popping on "not strictly left" and skipping on "left or on" drop        */
/* collinear points, so the hull lists strict vertices.  The input must be */
/* a simple polyline with distinct vertices, as the Lemma 1 polyline is.   */
/* A collinear prefix becomes the segment between its lexicographic        */
/* extremes before the first vertex off its line starts the deque.         */
/* Output as every hull here: counter-clockwise from the lexicographic     */
/* minimum.                                                                */
/* ------------------------------------------------------------------------ */
static void put_rotated(const int32_t *ring, int64_t h, int32_t *out)
{
    int64_t s = 0;
    for (int64_t i = 1; i < h; ++i)
        if (cmp_xy(&ring[2 * i], &ring[2 * s]) < 0)
            s = i;
    for (int64_t i = 0; i < h; ++i) {
        out[2 * i] = ring[2 * ((s + i) % h)];
        out[2 * i + 1] = ring[2 * ((s + i) % h) + 1];
    }
}

int64_t oracle_melkman(const int32_t *v, int64_t m, int32_t *out)
{
    if (m <= 0)
        return 0;
    /* the collinear prefix v[0..k-1] and its extremes a (min), b (max) */
    int64_t a = 0, b = 0, k = 1;
    for (; k < m; ++k) {
        if (k >= 2 && cross3(&v[2 * a], &v[2 * b], &v[2 * k]) != 0)
            break;
        if (cmp_xy(&v[2 * k], &v[2 * a]) < 0)
            a = k;
        if (cmp_xy(&v[2 * k], &v[2 * b]) > 0)
            b = k;
    }
    if (k == m) { /* every vertex on one line (or a single vertex) */
        out[0] = v[2 * a];
        out[1] = v[2 * a + 1];
        if (a == b)
            return 1;
        out[2] = v[2 * b];
        out[3] = v[2 * b + 1];
        return 2;
    }
    /* deque as a plain array indexed bot..top, room for m pushes each way */
    int64_t cap = 2 * m + 8, mid = m + 4;
    int32_t *D = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)cap);
#define DQ(i) (&D[2 * (i)])
#define SETDQ(i, p)              \
    do {                         \
        D[2 * (i)] = (p)[0];     \
        D[2 * (i) + 1] = (p)[1]; \
    } while (0)
    int64_t bot = mid, top = mid + 3;
    const int32_t *vk = &v[2 * k];
    SETDQ(bot, vk);
    SETDQ(top, vk);
    if (cross3(&v[2 * a], &v[2 * b], vk) > 0) {
        SETDQ(bot + 1, &v[2 * a]);
        SETDQ(bot + 2, &v[2 * b]);
    } else {
        SETDQ(bot + 1, &v[2 * b]);
        SETDQ(bot + 2, &v[2 * a]);
    }
    for (int64_t i = k + 1; i < m; ++i) {
        const int32_t *u = &v[2 * i];
        if (cross3(DQ(top - 1), DQ(top), u) >= 0 && cross3(DQ(bot), DQ(bot + 1), u) >= 0)
            continue; /* on or inside the current hull */
        while (top - bot > 1 && cross3(DQ(top - 1), DQ(top), u) <= 0)
            --top;
        ++top;
        SETDQ(top, u);
        while (top - bot > 1 && cross3(u, DQ(bot), DQ(bot + 1)) <= 0)
            ++bot;
        --bot;
        SETDQ(bot, u);
    }
#undef DQ
#undef SETDQ
    /* D[bot..top-1] is the hull, counter-clockwise */
    int64_t h = top - bot;
    put_rotated(&D[2 * bot], h, out);
    free(D);
    return h;
}

/* ------------------------------------------------------------------------ */
/* Steps 1 and 2 of the paper's general procedure (Section 2,              */
/* "Implementation of the proposed heuristic") for int32 points anywhere:  */
/* the bounding box [xmin, xmax] x [ymin, ymax]; the translation           */
/* x' = x - xmin + 1, y' = y - ymin + 1 into a p x q box (the printed     */
/* formula is garbled; this is the reading that maps the box onto          */
/* [1, p] x [1, q]); Algorithm 1 with the columns along the shorter side   */
/* (when q < p the roles of x and y swap, the sweep along min(p, q));     */
/* the hull of the reduced set on its Lemma 1 polyline; the vertices       */
/* mapped back.  Swapping x and y reverses the orientation, so the list is */
/* then reversed before it is rotated to start at the lexicographic min.   */
/* Sides above 2^30 are rejected (ORC_ERR_ARG), as for p.                  */
/* ------------------------------------------------------------------------ */
int64_t oracle_hull_box(const int32_t *pts, int64_t n, int32_t *out)
{
    if (n <= 0)
        return 0;
    int64_t xmin = pts[0], xmax = pts[0], ymin = pts[1], ymax = pts[1];
    for (int64_t i = 1; i < n; ++i) {
        if (pts[2 * i] < xmin) xmin = pts[2 * i];
        if (pts[2 * i] > xmax) xmax = pts[2 * i];
        if (pts[2 * i + 1] < ymin) ymin = pts[2 * i + 1];
        if (pts[2 * i + 1] > ymax) ymax = pts[2 * i + 1];
    }
    const int64_t p = xmax - xmin + 1, q = ymax - ymin + 1;
    if (p > (1 << 30) || q > (1 << 30))
        return ORC_ERR_ARG;
    const int tr = q < p;
    const int64_t nc = tr ? q : p, nr = tr ? p : q;
    /* Algorithm 1 on the translated (and, if tr, swapped) points; the     */
    /* empty entry is (nr + 1, -1), the sentinel of the longer side        */
    int32_t *L = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)nc);
    for (int64_t i = 0; i < nc; ++i) {
        L[2 * i] = (int32_t)(nr + 1);
        L[2 * i + 1] = -1;
    }
    for (int64_t i = 0; i < n; ++i) {
        const int64_t x = pts[2 * i] - xmin + 1, y = pts[2 * i + 1] - ymin + 1;
        const int64_t c = tr ? y : x, r = tr ? x : y;
        if (r < L[2 * (c - 1)]) L[2 * (c - 1)] = (int32_t)r;
        if (r > L[2 * (c - 1) + 1]) L[2 * (c - 1) + 1] = (int32_t)r;
    }
    /* Lemma 1 polyline (a column is valid when ly <= hy), then Andrew */
    int32_t *poly = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(2 * nc + 1));
    int64_t s = 0;
    for (int64_t i = 0; i < nc; ++i) {
        if (L[2 * i] > L[2 * i + 1])
            continue;
        poly[2 * s] = (int32_t)(i + 1);
        poly[2 * s + 1] = L[2 * i];
        ++s;
        if (L[2 * i + 1] != L[2 * i]) {
            poly[2 * s] = (int32_t)(i + 1);
            poly[2 * s + 1] = L[2 * i + 1];
            ++s;
        }
    }
    int32_t *hf = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(2 * nc + 2));
    const int64_t h = andrew_sorted(poly, s, hf);
    /* back to the input's coordinates (reversed when swapped) */
    int32_t *ring = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(h + 1));
    for (int64_t i = 0; i < h; ++i) {
        const int64_t j = tr ? h - 1 - i : i;
        const int64_t c = hf[2 * j], r = hf[2 * j + 1];
        const int64_t x = (tr ? r : c) + xmin - 1, y = (tr ? c : r) + ymin - 1;
        ring[2 * i] = (int32_t)x;
        ring[2 * i + 1] = (int32_t)y;
    }
    put_rotated(ring, h, out);
    free(ring);
    free(hf);
    free(poly);
    free(L);
    return h;
}

/* ------------------------------------------------------------------------ */
/* The second scan along y (Section 2, Fig. 4: rx -> rxy): Algorithm 1 run */
/* again over the rx points, the surviving (x, ly) and (x, hy) of L, with  */
/* the roles of x and y exchanged.  R is indexed by y, 0-based; entry      */
/* y - 1 becomes (min x, max x) over the rx points with that y, or stays   */
/* (p + 1, -1) (the square of side p, so q = p).  The rxy points are the   */
/* (lo, y) and (hi, y) of the valid rows: a subset of the rx points that   */
/* keeps every point extreme in its row, hence every hull vertex.          */
/* ------------------------------------------------------------------------ */
void oracle_reduce_rows(const int32_t *L, int32_t p, int32_t *R)
{
    for (int64_t i = 0; i < p; ++i) {
        R[2 * i] = p + 1;
        R[2 * i + 1] = -1;
    }
    for (int64_t i = 0; i < p; ++i) {
        if (!entry_valid(L, p, i))
            continue;
        const int32_t x = (int32_t)(i + 1);
        for (int k = 0; k < 2; ++k) {
            const int32_t y = L[2 * i + k];
            if (x < R[2 * (y - 1)])
                R[2 * (y - 1)] = x;
            if (x > R[2 * (y - 1) + 1])
                R[2 * (y - 1) + 1] = x;
        }
    }
}
