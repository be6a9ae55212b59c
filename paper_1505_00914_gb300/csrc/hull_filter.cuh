// Exact pre-filter of a lower chain held in shared memory, shared by the
// fused chain kernel and the hull kernels.
//
// For a run of n <= 1024 consecutive points of an x-ordered chain, thread i
// decides whether point i can be a strict vertex of the lower hull.  It drops
// the point when it lies on or above the segment between two other points of
// the run, one on each side: the lowest points of the blocks left and right
// of i's block at every level of a binary min-tree over the run, or its
// neighbours at most two places away.  A dropped point
// is a convex combination of two input points, so it is not a strict vertex:
// every drop is exact, whichever tests are chosen; the tests only decide how
// many non-vertices are left for the exact merge that follows.
#pragma once

#include "ch_internal.cuh"

namespace ch {

constexpr int RUN = 1024;      // points per filtered run (= threads of the CTA)
constexpr int RUN_LOG = 10;

// Level k >= 1 of the tree (node j covers [j << k, (j+1) << k)) starts at
// tree_off(k); 2 * RUN shorts hold every level.
__device__ __forceinline__ int tree_off(int k) { return 2 * RUN - ((2 * RUN) >> (k - 1)); }

// Barrier of a group of NT threads (whole warps): the whole CTA when BAR is
// 0, else the named barrier BAR, which exactly those NT threads use.
template <int BAR, int NT>
__device__ __forceinline__ void group_sync()
{
    if constexpr (BAR == 0)
        __syncthreads();
    else
        asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(NT) : "memory");
}

// Builds the min-y index trees of two runs, P0[0..n0) and P1[0..n1), level by
// level; every thread of the CTA calls it (or, with NT and BAR, every thread
// of a group of NT >= RUN / 2 threads with barrier BAR, tid its index in the
// group).  Levels 5 and up have at most 32 nodes and read only nodes that
// warp 0 wrote, so warp 0 builds them alone with warp barriers between levels.
template <int NT = RUN, int BAR = 0>
__device__ __forceinline__ void build_min_trees(const int2 *P0, short *M0, int n0, const int2 *P1,
                                                short *M1, int n1, int tid = threadIdx.x)
{
    static_assert(NT >= RUN / 2, "one thread per node of the lowest level");
    const int i = tid;
    auto level = [&](int k) {
        if (i < (RUN >> k)) {
            int a0, b0, a1, b1;
            if (k == 1) {
                a0 = a1 = 2 * i;
                b0 = b1 = 2 * i + 1;
            } else {
                a0 = M0[tree_off(k - 1) + 2 * i];
                b0 = M0[tree_off(k - 1) + 2 * i + 1];
                a1 = M1[tree_off(k - 1) + 2 * i];
                b1 = M1[tree_off(k - 1) + 2 * i + 1];
            }
            const bool va0 = a0 >= 0 && a0 < n0, vb0 = b0 >= 0 && b0 < n0;
            const bool va1 = a1 >= 0 && a1 < n1, vb1 = b1 >= 0 && b1 < n1;
            const int ya0 = va0 ? P0[a0].y : 0, yb0 = vb0 ? P0[b0].y : 0;
            const int ya1 = va1 ? P1[a1].y : 0, yb1 = vb1 ? P1[b1].y : 0;
            M0[tree_off(k) + i] = (short)(va0 ? ((vb0 && yb0 < ya0) ? b0 : a0) : (vb0 ? b0 : -1));
            M1[tree_off(k) + i] = (short)(va1 ? ((vb1 && yb1 < ya1) ? b1 : a1) : (vb1 ? b1 : -1));
        }
    };
    constexpr int WARP_LEVEL = 5;  // RUN >> 5 = 32 nodes
    static_assert((RUN >> WARP_LEVEL) == 32, "levels from WARP_LEVEL on fit one warp");
    for (int k = 1; k < WARP_LEVEL; ++k) {
        level(k);
        group_sync<BAR, NT>();
    }
    if (i < 32) {
        // lane i holds node i of the current level as (index of its lowest
        // point, that point's y; INT_MAX when the node is empty) for both
        // runs; the next level combines lanes 2j and 2j + 1 by shuffles
        constexpr int EMPTY_Y = 0x7FFFFFFF;
        auto node = [&](const int2 *P, const short *M, int n, int &m, int &y) {
            const int a = M[tree_off(WARP_LEVEL - 1) + 2 * i];
            const int b = M[tree_off(WARP_LEVEL - 1) + 2 * i + 1];
            const bool va = a >= 0 && a < n, vb = b >= 0 && b < n;
            const int ya = va ? P[a].y : EMPTY_Y, yb = vb ? P[b].y : EMPTY_Y;
            m = va ? ((vb && yb < ya) ? b : a) : (vb ? b : -1);
            y = yb < ya ? yb : ya;
        };
        int m0, y0, m1, y1;
        node(P0, M0, n0, m0, y0);
        node(P1, M1, n1, m1, y1);
        M0[tree_off(WARP_LEVEL) + i] = (short)m0;
        M1[tree_off(WARP_LEVEL) + i] = (short)m1;
#pragma unroll
        for (int k = WARP_LEVEL + 1; k <= RUN_LOG; ++k) {
            const int sa = (2 * i) & 31, sb = (2 * i + 1) & 31;
            const int ma0 = __shfl_sync(0xFFFFFFFFu, m0, sa), ya0 = __shfl_sync(0xFFFFFFFFu, y0, sa);
            const int mb0 = __shfl_sync(0xFFFFFFFFu, m0, sb), yb0 = __shfl_sync(0xFFFFFFFFu, y0, sb);
            const int ma1 = __shfl_sync(0xFFFFFFFFu, m1, sa), ya1 = __shfl_sync(0xFFFFFFFFu, y1, sa);
            const int mb1 = __shfl_sync(0xFFFFFFFFu, m1, sb), yb1 = __shfl_sync(0xFFFFFFFFu, y1, sb);
            // the left child wins ties; an empty child (y = INT_MAX) never wins
            m0 = yb0 < ya0 ? mb0 : ma0;
            y0 = yb0 < ya0 ? yb0 : ya0;
            m1 = yb1 < ya1 ? mb1 : ma1;
            y1 = yb1 < ya1 ? yb1 : ya1;
            if (i < (RUN >> k)) {
                M0[tree_off(k) + i] = (short)m0;
                M1[tree_off(k) + i] = (short)m1;
            }
        }
    }
    group_sync<BAR, NT>();
}

// True when point i of P[0..n) may be a strict lower-hull vertex.  The anchor
// loads of three levels at a time are issued before their orientation tests.
// At each level only the pair (lowest point of the left sibling block,
// lowest point of the right one) is tested: pairing an anchor with a direct
// neighbour as well dropped 7 % more points but cost a third more time than
// the final hull saved.
// SPARSE_EXIT: the variant the batched kernel uses, where most tiles are
// short-lived: a warp stops testing once all its points are dropped, and the
// lowest level (blocks of two points, next to the +-2 neighbour tests) is
// left out; the chain kernel's dense tiles are faster without the vote.
// NARROW: 32-bit orientation tests (see orient; chain points of p <= 16384).
template <bool SPARSE_EXIT = false, bool NARROW = false>
__device__ __forceinline__ bool run_keeps(const int2 *P, const short *M, int n, int i)
{
    const bool alive = i < n;
    const int2 q = alive ? P[i] : make_int2(0, 0);
    const bool h1 = alive && i >= 1 && i + 1 < n, l2 = i >= 2, r2 = i + 2 < n;
    const int2 nl1 = alive && i >= 1 ? P[i - 1] : q, nr1 = alive && i + 1 < n ? P[i + 1] : q;
    const int2 nl2 = alive && l2 ? P[i - 2] : q, nr2 = alive && r2 ? P[i + 2] : q;
    bool drop = !alive || (h1 && (orient<NARROW>(nl1, nr1, q) >= 0 ||
                                  (r2 && orient<NARROW>(nl1, nr2, q) >= 0) ||
                                  (l2 && orient<NARROW>(nl2, nr1, q) >= 0)));
    constexpr int CH = 3;  // levels per batch; levels 1..RUN_LOG-1 have siblings
#pragma unroll
    for (int k0 = SPARSE_EXIT ? 2 : 1; k0 < RUN_LOG; k0 += CH) {
        if (SPARSE_EXIT && __all_sync(0xFFFFFFFFu, drop))
            break;
        int la[CH], ra[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const int k = k0 + u, node = i >> k;
            la[u] = k < RUN_LOG && node >= 1 ? M[tree_off(k) + node - 1] : -1;
            ra[u] = k < RUN_LOG && (node + 1) < (RUN >> k) ? M[tree_off(k) + node + 1] : -1;
        }
        int2 A[CH], B[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            A[u] = la[u] >= 0 ? P[la[u]] : q;
            B[u] = ra[u] >= 0 ? P[ra[u]] : q;
        }
#pragma unroll
        for (int u = 0; u < CH; ++u)
            drop |= la[u] >= 0 && ra[u] >= 0 && orient<NARROW>(A[u], B[u], q) >= 0;
    }
    return !drop;
}

// run_keeps<true, NARROW> for point i of two runs at once (P0/M0 and P1/M1
// of the same length n, the two chains of one tile): the same tests, their
// shared-memory loads interleaved so that the two chains' latencies overlap,
// and a warp stops once every point of both is dropped.
template <bool NARROW>
__device__ __forceinline__ void run_keeps_pair(const int2 *P0, const short *M0, const int2 *P1,
                                               const short *M1, int n, int i, bool &keep0,
                                               bool &keep1)
{
    const bool alive = i < n;
    const bool h1 = alive && i >= 1 && i + 1 < n, l2 = i >= 2, r2 = i + 2 < n;
    const int2 q0 = alive ? P0[i] : make_int2(0, 0), q1 = alive ? P1[i] : make_int2(0, 0);
    const int2 a1 = alive && i >= 1 ? P0[i - 1] : q0, b1 = alive && i + 1 < n ? P0[i + 1] : q0;
    const int2 c1 = alive && i >= 1 ? P1[i - 1] : q1, d1 = alive && i + 1 < n ? P1[i + 1] : q1;
    const int2 a2 = alive && l2 ? P0[i - 2] : q0, b2 = alive && r2 ? P0[i + 2] : q0;
    const int2 c2 = alive && l2 ? P1[i - 2] : q1, d2 = alive && r2 ? P1[i + 2] : q1;
    bool drop0 = !alive || (h1 && (orient<NARROW>(a1, b1, q0) >= 0 ||
                                   (r2 && orient<NARROW>(a1, b2, q0) >= 0) ||
                                   (l2 && orient<NARROW>(a2, b1, q0) >= 0)));
    bool drop1 = !alive || (h1 && (orient<NARROW>(c1, d1, q1) >= 0 ||
                                   (r2 && orient<NARROW>(c1, d2, q1) >= 0) ||
                                   (l2 && orient<NARROW>(c2, d1, q1) >= 0)));
    constexpr int CH = 3;  // levels per batch; levels 2..RUN_LOG-1 have siblings
#pragma unroll
    for (int k0 = 2; k0 < RUN_LOG; k0 += CH) {
        if (__all_sync(0xFFFFFFFFu, drop0 && drop1))
            break;
        int la0[CH], ra0[CH], la1[CH], ra1[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const int k = k0 + u, node = i >> k;
            const bool hl = k < RUN_LOG && node >= 1, hr = k < RUN_LOG && (node + 1) < (RUN >> k);
            la0[u] = hl ? M0[tree_off(k) + node - 1] : -1;
            ra0[u] = hr ? M0[tree_off(k) + node + 1] : -1;
            la1[u] = hl ? M1[tree_off(k) + node - 1] : -1;
            ra1[u] = hr ? M1[tree_off(k) + node + 1] : -1;
        }
        int2 A0[CH], B0[CH], A1[CH], B1[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            A0[u] = la0[u] >= 0 ? P0[la0[u]] : q0;
            B0[u] = ra0[u] >= 0 ? P0[ra0[u]] : q0;
            A1[u] = la1[u] >= 0 ? P1[la1[u]] : q1;
            B1[u] = ra1[u] >= 0 ? P1[ra1[u]] : q1;
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            drop0 |= la0[u] >= 0 && ra0[u] >= 0 && orient<NARROW>(A0[u], B0[u], q0) >= 0;
            drop1 |= la1[u] >= 0 && ra1[u] >= 0 && orient<NARROW>(A1[u], B1[u], q1) >= 0;
        }
    }
    keep0 = !drop0;
    keep1 = !drop1;
}

// Writes the kept points of P[0..n), in order, to out; returns their number.
// `keep` is this thread's decision for point threadIdx.x; s_wc holds
// RUN / 32 ints of scratch.  Every thread of the CTA calls it.
__device__ __forceinline__ int compact_run(const int2 *P, bool keep, int2 *out, int *s_wc)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
    __syncthreads();  // s_wc may still be read by a previous call
    if (lane == 0)
        s_wc[w] = __popc(bal);
    __syncthreads();
    if (w == 0) {
        const int v = s_wc[lane];
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o)
                incl += x;
        }
        s_wc[lane] = incl - v;
        if (lane == 31)
            s_wc[RUN / 32] = incl;
    }
    __syncthreads();
    if (keep)
        out[s_wc[w] + __popc(bal & ((1u << lane) - 1u))] = P[threadIdx.x];
    return s_wc[RUN / 32];
}

// compact_run for two runs at once: one scan over both counts (packed in
// 16-bit halves; each is at most RUN).  Returns (kept of P0, kept of P1).
// LEAD = false when no thread can still be reading s_wc (a block barrier
// since its last read).
template <bool LEAD = true>
__device__ __forceinline__ int2 compact_runs(const int2 *P0, bool keep0, int2 *out0, const int2 *P1,
                                             bool keep1, int2 *out1, int *s_wc)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned b0 = __ballot_sync(0xFFFFFFFFu, keep0), b1 = __ballot_sync(0xFFFFFFFFu, keep1);
    if (LEAD)
        __syncthreads();  // s_wc may still be read by a previous call
    if (lane == 0)
        s_wc[w] = __popc(b0) | (__popc(b1) << 16);
    __syncthreads();
    if (w == 0) {
        const int v = s_wc[lane];
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o)
                incl += x;
        }
        s_wc[lane] = incl - v;
        if (lane == 31)
            s_wc[RUN / 32] = incl;
    }
    __syncthreads();
    const int base = s_wc[w];
    const unsigned below = (1u << lane) - 1u;
    if (keep0)
        out0[(base & 0xFFFF) + __popc(b0 & below)] = P0[threadIdx.x];
    if (keep1)
        out1[(base >> 16) + __popc(b1 & below)] = P1[threadIdx.x];
    const int tot = s_wc[RUN / 32];
    return make_int2(tot & 0xFFFF, tot >> 16);
}

}  // namespace ch
