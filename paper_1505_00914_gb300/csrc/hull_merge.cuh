// CTA-level pieces of the exact hull of x-ordered chains: bridge finding,
// in-place pairwise merging, peeling and stitching.  Shared by the single-set
// final kernel and the batched kernel.
#pragma once

#include "ch_internal.cuh"
#include "hull_filter.cuh"

namespace ch {
namespace {

constexpr int HS = 16;        // points per thread run of the merge fallback
constexpr int SMALL = 32;     // pairs with na + nb <= SMALL merge on one thread
constexpr int FT = 1024;      // threads of a CTA running the final steps
constexpr int PEEL_MAX = 24;  // peeling rounds before the merge fallback


// Index of the tangent point from a (left of every point of B) to the lower
// hull B: the vertex of least slope, the farthest one on ties.
__device__ __forceinline__ int tangent(const int2 *B, int nb, int2 a)
{
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cross3(a, B[mid], B[mid + 1]) <= 0)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Bridge (u, v) of lower hulls A (left) and B (right); called by a full warp.
// u is the first i for which a_{i+1} is not strictly below the line from a_i
// to its tangent point on B.
__device__ void warp_bridge(const int2 *A, int na, const int2 *B, int nb, int lane, int &u, int &v)
{
    int lo = 0, hi = na - 1;
    while (lo < hi) {
        const int span = hi - lo;
        const int i = lo + (int)(((long long)span * lane) >> 5);
        bool q = false;
        if (i < na - 1) {
            const int2 ai = A[i];
            q = cross3(ai, B[tangent(B, nb, ai)], A[i + 1]) < 0;
        }
        const unsigned fb = __ballot_sync(0xFFFFFFFFu, !q);
        const int f = fb ? __ffs(fb) - 1 : 31;
        const int i_f = __shfl_sync(0xFFFFFFFFu, i, f);
        const int i_p = __shfl_sync(0xFFFFFFFFu, i, f > 0 ? f - 1 : 0);
        if (fb) {
            hi = i_f;
            if (f > 0)
                lo = i_p + 1;
        } else {
            lo = i_f + 1;
        }
    }
    u = lo;
    v = tangent(B, nb, A[u]);
}

// One thread: continue Andrew's scan of the hull at D[a..a+na) over the hull
// at D[b..b+nb) (b >= a + na), in place.  Returns the merged length.
__device__ int thread_merge(int2 *D, int a, int na, int b, int nb)
{
    int top = na;
    int2 t1 = D[a + top - 1];
    int2 t0 = top >= 2 ? D[a + top - 2] : t1;
    for (int k = 0; k < nb; ++k) {
        const int2 q = D[b + k];
        while (top >= 2 && cross3(t0, t1, q) <= 0) {
            --top;
            t1 = t0;
            if (top >= 2)
                t0 = D[a + top - 2];
        }
        D[a + top] = q;
        ++top;
        t0 = t1;
        t1 = q;
    }
    return top;
}

// In-place exclusive scan of a[0..n) by a group of NT threads (t = the
// thread's index in the group, BAR its barrier); returns the total.
template <int NT, int BAR = 0>
__device__ int block_excl_scan(int *a, int n, int *s_warp, int *s_total, int t = threadIdx.x)
{
    const int lane = t & 31, w = t >> 5;
    const int per = (n + NT - 1) / NT;
    const int b = min(n, t * per), e = min(n, b + per);
    int sum = 0;
    for (int i = b; i < e; ++i)
        sum += a[i];
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o)
            incl += x;
    }
    if (lane == 31)
        s_warp[w] = incl;
    group_sync<BAR, NT>();
    if (w == 0) {
        const int v = lane < NT / 32 ? s_warp[lane] : 0;
        int inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o)
                inc += x;
        }
        if (lane < NT / 32)
            s_warp[lane] = inc - v;
        if (lane == 31)
            *s_total = inc;
    }
    group_sync<BAR, NT>();
    int run = s_warp[w] + incl - sum;
    for (int i = b; i < e; ++i) {
        const int v = a[i];
        a[i] = run;
        run += v;
    }
    const int total = *s_total;
    group_sync<BAR, NT>();
    return total;
}

// In-place pairwise merge tree.  Segments [0, c0) belong to chain 0 and
// [c0, c0 + c1) to chain 1; segment s is D[S[s] .. S[s] + L[s]), and each
// segment starts at or after the end of the previous one.  On return the
// index arrays (swapped as needed) describe one hull per non-empty chain.
struct Tree {
    int2 *D;
    int *S, *L, *S2, *L2;
    int c0, c1;
};

template <int NT, int BAR = 0>
__device__ void merge_tree(Tree &t, int tid = threadIdx.x)
{
    const int lane = tid & 31, warp = tid >> 5;
    while (t.c0 > 1 || t.c1 > 1) {
        const int d0 = (t.c0 + 1) >> 1, d1 = (t.c1 + 1) >> 1, nd = d0 + d1;
        // small pairs and carries: one thread each
        for (int j = tid; j < nd; j += NT) {
            const int chain = j >= d0;
            const int jj = j - (chain ? d0 : 0);
            const int cc = chain ? t.c1 : t.c0;
            const int ia = (chain ? t.c0 : 0) + 2 * jj, ib = ia + 1;
            const int la = t.L[ia];
            if (2 * jj + 1 >= cc) {
                t.S2[j] = t.S[ia];
                t.L2[j] = la;
            } else if (la + t.L[ib] <= SMALL) {
                t.S2[j] = t.S[ia];
                t.L2[j] = thread_merge(t.D, t.S[ia], la, t.S[ib], t.L[ib]);
            }
        }
        // large pairs: one warp each
        for (int j = warp; j < nd; j += NT / 32) {
            const int chain = j >= d0;
            const int jj = j - (chain ? d0 : 0);
            const int cc = chain ? t.c1 : t.c0;
            const int ia = (chain ? t.c0 : 0) + 2 * jj, ib = ia + 1;
            if (2 * jj + 1 >= cc || t.L[ia] + t.L[ib] <= SMALL)
                continue;
            const int sa = t.S[ia], sb = t.S[ib], lb = t.L[ib];
            int u, v;
            warp_bridge(t.D + sa, t.L[ia], t.D + sb, lb, lane, u, v);
            const int cnt = lb - v;
            int2 *dst = t.D + sa + u + 1;
            const int2 *src = t.D + sb + v;
            for (int k0 = 0; k0 < cnt; k0 += 32) {
                const int k = k0 + lane;
                int2 q;
                if (k < cnt)
                    q = src[k];
                __syncwarp();
                if (k < cnt)
                    dst[k] = q;
                __syncwarp();
            }
            if (lane == 0) {
                t.S2[j] = sa;
                t.L2[j] = u + 1 + cnt;
            }
        }
        group_sync<BAR, NT>();
        int *x = t.S;
        t.S = t.S2;
        t.S2 = x;
        x = t.L;
        t.L = t.L2;
        t.L2 = x;
        t.c0 = d0;
        t.c1 = d1;
    }
}

// True when point i of the chain stored at D[cs..ce) lies on or above a
// segment between two of its neighbours: any of the pairs at most two places
// away, or the pairs three and four places away on both sides (those end a
// long concave run in fewer rounds).
template <bool NARROW = false>
__device__ __forceinline__ bool peel_drops(const int2 *D, int cs, int ce, int i)
{
    if (i - 1 < cs || i + 1 >= ce)
        return false;
    const int2 q = D[i], l1 = D[i - 1], r1 = D[i + 1];
    if (orient<NARROW>(l1, r1, q) >= 0)
        return true;
    const bool l2 = i - 2 >= cs, r2 = i + 2 < ce;
    const int2 a2 = l2 ? D[i - 2] : l1, b2 = r2 ? D[i + 2] : r1;
    if ((r2 && orient<NARROW>(l1, b2, q) >= 0) || (l2 && orient<NARROW>(a2, r1, q) >= 0) ||
        (l2 && r2 && orient<NARROW>(a2, b2, q) >= 0))
        return true;
    const bool l3 = i - 3 >= cs, r3 = i + 3 < ce, l4 = i - 4 >= cs, r4 = i + 4 < ce;
    const int2 a3 = l3 ? D[i - 3] : a2, b3 = r3 ? D[i + 3] : b2;
    const int2 a4 = l4 ? D[i - 4] : a3, b4 = r4 ? D[i + 4] : b3;
    return (l3 && r3 && orient<NARROW>(a3, b3, q) >= 0) || (l4 && r4 && orient<NARROW>(a4, b4, q) >= 0);
}

// Peel, merge fallback and stitch, run by a whole CTA of FT threads.  A holds
// the survivors: the lower chain in A[0..T0), the mirrored upper chain in
// A[T0..T).  B (T points), F (T ints) and ix (4 * (T / HS + 2) ints) are
// scratch.  Peeling drops, round after round, every point that lies on or
// above a segment between its current neighbours, until a round drops
// nothing: an x-monotone chain that turns strictly counter-clockwise at every
// point is its own strict lower hull.  If PEEL_MAX rounds do not get there,
// the rest goes through runs of HS points and the pairwise merge tree.  The
// stitched hull (counter-clockwise from the lexicographic minimum) goes to
// hull[0..*hull_count).
// NT, BAR, tid: run by a group of NT threads (whole warps) with its own
// barrier BAR instead of the whole CTA; tid is the thread's index in the
// group and s_warp holds NT / 32 + 1 ints of the group's own.
template <int NT = FT, int BAR = 0, bool NARROW = false>
__device__ void peel_merge_stitch(int2 *A, int2 *B, int *F, int *ix, int T0, int T, int2 *hull,
                                  int *hull_count, int *s_warp, int *s_total, int tid = threadIdx.x)
{
    static_assert(NT % 32 == 0 && NT <= 1024, "whole warps");
    const int t = tid, lane = t & 31, w = t >> 5;
    bool done = false;
    for (int round = 0; round < PEEL_MAX && !done; ++round) {
        if (T <= NT) {  // one point per thread: a ballot scan, three block barriers
            const bool c1 = t >= T0;
            const bool keep = t < T && !peel_drops<NARROW>(A, c1 ? T0 : 0, c1 ? T : T0, t);
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
            if (lane == 0)
                s_warp[w] = __popc(bal);
            group_sync<BAR, NT>();
            if (w == 0) {
                const int v = lane < NT / 32 ? s_warp[lane] : 0;
                int incl = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                    if (lane >= o)
                        incl += x;
                }
                if (lane < NT / 32)
                    s_warp[lane] = incl - v;
                if (lane == 31)
                    *s_total = incl;
            }
            group_sync<BAR, NT>();
            const int kept = *s_total;
            if (kept == T) {
                done = true;  // block-uniform
                break;
            }
            const int pos = s_warp[w] + __popc(bal & ((1u << lane) - 1u));
            if (keep)
                B[pos] = A[t];
            if (t == T0 && T0 < T)
                F[0] = pos;  // points kept before the upper chain
            group_sync<BAR, NT>();
            T0 = T0 < T ? F[0] : kept;
            T = kept;
            int2 *x = A;
            A = B;
            B = x;
            continue;
        }
        for (int i = t; i < T; i += NT) {
            const bool c1 = i >= T0;
            F[i] = peel_drops<NARROW>(A, c1 ? T0 : 0, c1 ? T : T0, i) ? 0 : 1;
        }
        group_sync<BAR, NT>();
        const int kept = block_excl_scan<NT, BAR>(F, T, s_warp, s_total, t);
        if (kept == T) {
            done = true;  // block-uniform
            break;
        }
        for (int i = t; i < T; i += NT) {
            const int next = i + 1 < T ? F[i + 1] : kept;
            if (next != F[i])
                B[F[i]] = A[i];
        }
        const int nT0 = T0 < T ? F[T0] : kept;
        group_sync<BAR, NT>();
        int2 *x = A;
        A = B;
        B = x;
        T = kept;
        T0 = nT0;
    }

    int hl, hu;
    const int2 *LH, *UH;
    if (done) {
        hl = T0;
        hu = T - T0;
        LH = A;
        UH = A + T0;
    } else {
        // fallback: Andrew's scan over runs of HS points, then the merge tree
        const int T1 = T - T0;
        const int r0 = (T0 + HS - 1) / HS, r1 = (T1 + HS - 1) / HS, nr = r0 + r1;
        for (int r = t; r < nr; r += NT) {
            const bool c1 = r >= r0;
            const int st = c1 ? T0 + (r - r0) * HS : r * HS;
            const int cnt = min(HS, (c1 ? T : T0) - st);
            int top = 0;
            int2 a0 = make_int2(0, 0), a1 = make_int2(0, 0);
            for (int i = 0; i < cnt; ++i) {
                const int2 q = A[st + i];
                while (top >= 2 && orient<NARROW>(a0, a1, q) <= 0) {
                    --top;
                    a1 = a0;
                    if (top >= 2)
                        a0 = A[st + top - 2];
                }
                A[st + top] = q;
                ++top;
                a0 = a1;
                a1 = q;
            }
            ix[r] = st;
            ix[nr + r] = top;
        }
        group_sync<BAR, NT>();
        Tree tr;
        tr.D = A;
        tr.S = ix;
        tr.L = ix + nr;
        tr.S2 = ix + 2 * nr;
        tr.L2 = ix + 3 * nr;
        tr.c0 = r0;
        tr.c1 = r1;
        merge_tree<NT, BAR>(tr, t);
        hl = tr.c0 ? tr.L[0] : 0;
        hu = tr.c1 ? tr.L[tr.c0] : 0;
        LH = A + (tr.c0 ? tr.S[0] : 0);
        UH = A + (tr.c1 ? tr.S[tr.c0] : 0);
    }

    // Stitch: lower hull left to right, then the upper hull right to left,
    // without repeating the shared end points.
    int kl = hu - 1, kf = 0;
    if (hl > 0 && hu > 0) {
        const int2 ul = UH[hu - 1], ll = LH[hl - 1];
        if (ul.x == ll.x && -ul.y == ll.y)
            --kl;
        const int2 uf = UH[0], lf = LH[0];
        if (kl >= 0 && uf.x == lf.x && -uf.y == lf.y)
            kf = 1;
    }
    const int nup = max(0, kl - kf + 1);
    for (int k = t; k < hl; k += NT)
        hull[k] = LH[k];
    for (int k = t; k < nup; k += NT) {
        const int2 q = UH[kl - k];
        hull[hl + k] = make_int2(q.x, -q.y);
    }
    if (t == 0)
        *hull_count = hl + nup;
    group_sync<BAR, NT>();
}


}  // namespace
}  // namespace ch
