// Exact pre-filter of a lower chain held in shared memory, shared by the
// fused chain kernel and the hull kernels.
//
// For a run of n <= 1024 consecutive points of an x-ordered chain, thread i
// decides whether point i can be a strict vertex of the lower hull.  It drops
// the point when it lies on or above the segment between two other points of
// the run, one on each side: the lowest points of the sibling sub-runs of i at
// every level of a binary min-tree over the run, its immediate neighbours, and
// the points at distances d, e in {s, 2s}, s = 1, 2, 4, ...  A dropped point
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

// Builds the min-y index tree of P[0..n); every thread of the CTA calls it.
__device__ __forceinline__ void build_min_tree(const int2 *P, short *M, int n)
{
    const int i = threadIdx.x;
    for (int k = 1; k <= RUN_LOG; ++k) {
        if (i < (RUN >> k)) {
            int a, b;
            if (k == 1) {
                a = 2 * i;
                b = 2 * i + 1;
            } else {
                a = M[tree_off(k - 1) + 2 * i];
                b = M[tree_off(k - 1) + 2 * i + 1];
            }
            int best = (a >= 0 && a < n) ? a : -1;
            if (b >= 0 && b < n && (best < 0 || P[b].y < P[best].y))
                best = b;
            M[tree_off(k) + i] = (short)best;
        }
        __syncthreads();
    }
}

// True when point i of P[0..n) may be a strict lower-hull vertex.
__device__ __forceinline__ bool run_keeps(const int2 *P, const short *M, int n, int i)
{
    if (i >= n)
        return false;
    const int2 q = P[i];
    for (int k = 1; k < RUN_LOG; ++k) {
        const int node = i >> k;
        const int la = node >= 1 ? M[tree_off(k) + node - 1] : -1;
        const int ra = (node + 1) < (RUN >> k) ? M[tree_off(k) + node + 1] : -1;
        if (la >= 0 && ra >= 0 && cross3(P[la], P[ra], q) >= 0)
            return false;
        if (la >= 0 && i + 1 < n && cross3(P[la], P[i + 1], q) >= 0)
            return false;
        if (ra >= 0 && i >= 1 && cross3(P[i - 1], P[ra], q) >= 0)
            return false;
    }
    for (int s = 1; i - s >= 0 || i + s < n; s <<= 1) {
        const bool l1 = i - s >= 0, r1 = i + s < n, l2 = i - 2 * s >= 0, r2 = i + 2 * s < n;
        if ((l1 && r1 && cross3(P[i - s], P[i + s], q) >= 0) ||
            (l1 && r2 && cross3(P[i - s], P[i + 2 * s], q) >= 0) ||
            (l2 && r1 && cross3(P[i - 2 * s], P[i + s], q) >= 0))
            return false;
    }
    return true;
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

}  // namespace ch
