// Step 3: strict convex hull of the x-ordered chains, with no sort.
//
// The lower hull of the lower chain and the upper hull of the upper chain,
// stitched counter-clockwise from the lexicographic minimum, give the hull of
// the reduced set, which by the correctness argument of the Appendix is the
// hull of the input.  The upper chain is mirrored (y -> -y) so that one
// lower-hull routine serves both.
//
// Parallel monotone chain:
//   k_hull_seg   - every thread runs Andrew's scan (pop while the turn is not
//                  strictly counter-clockwise, int64 orientation) over a
//                  segment of 32 consecutive chain points.  A point that is
//                  not a strict vertex of its segment's hull lies on or above
//                  a segment between two other points, so it is not a strict
//                  vertex of the whole hull either: dropping it is exact.
//   k_hull_final - one CTA merges adjacent segment hulls pairwise, level by
//                  level.  Two x-separated lower hulls A (left) and B (right)
//                  merge into A[0..u] ++ B[v..] where (a_u, b_v) is their
//                  bridge; a warp finds it by a 32-way search over A, each
//                  lane locating the tangent from its a_i to B by binary
//                  search.  Ties are resolved towards the strict hull: the
//                  tangent takes the farthest of collinear B points, the
//                  bridge the leftmost of collinear A points.
#include "ch_internal.cuh"

namespace ch {
namespace {

constexpr int HS = 32;    // chain points per segment
constexpr int HT = 128;   // threads per CTA of the segment kernel
constexpr int FT = 1024;  // threads of the final CTA
constexpr int PCAP = 6144;  // points per shared-memory buffer (two buffers)
constexpr int SCAP = 4096;  // segments per shared-memory index array (six arrays)
constexpr size_t FINAL_SMEM = 2 * PCAP * sizeof(int2) + 6 * SCAP * sizeof(int);

__global__ void __launch_bounds__(HT)
    k_hull_seg(const int2 *__restrict__ lower, const int2 *__restrict__ upper,
               const int *__restrict__ counts, int p, int nsegmax, int2 *cand, int *segcnt)
{
    __shared__ int2 stk[HS][HT];
    const int gid = blockIdx.x * HT + threadIdx.x;
    if (gid >= 2 * nsegmax)
        return;
    const int chain = gid >= nsegmax;
    const int seg = gid - chain * nsegmax;
    const int m = max(0, min(counts[chain], p));
    const int b = seg * HS;
    if (b >= m)
        return;
    const int e = min(m, b + HS);
    const int2 *src = chain ? upper : lower;
    const int sg = chain ? -1 : 1;
    int top = 0;
    for (int i = b; i < e; ++i) {
        int2 q = src[i];
        q.y *= sg;
        while (top >= 2 && cross3(stk[top - 2][threadIdx.x], stk[top - 1][threadIdx.x], q) <= 0)
            --top;
        stk[top][threadIdx.x] = q;
        ++top;
    }
    int2 *out = cand + (size_t)gid * HS;
    for (int k = 0; k < top; ++k)
        out[k] = stk[k][threadIdx.x];
    segcnt[gid] = top;
}

// Index of the tangent point from a (left of every point of B) to the lower
// hull B: the vertex of least slope, the farthest one on ties.
__device__ __forceinline__ int tangent(const int2 *B, int nb, int2 a)
{
    int lo = 0, hi = nb - 1;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
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
__device__ void warp_bridge(const int2 *A, int na, const int2 *B, int nb, int lane, int &u,
                            int &v)
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

// In-place exclusive scan of a[0..n) by the whole CTA; returns the total.
__device__ int block_excl_scan(int *a, int n, int *s_warp, int *s_total)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int per = (n + FT - 1) / FT;
    const int b = min(n, t * per), e = min(n, b + per);
    int sum = 0;
    for (int i = b; i < e; ++i)
        sum += a[i];
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o)
            incl += x;
    }
    if (lane == 31)
        s_warp[w] = incl;
    __syncthreads();
    if (w == 0) {
        int v = s_warp[lane], inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int x = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o)
                inc += x;
        }
        s_warp[lane] = inc - v;
        if (lane == 31)
            *s_total = inc;
    }
    __syncthreads();
    int run = s_warp[w] + incl - sum;
    for (int i = b; i < e; ++i) {
        int v = a[i];
        a[i] = run;
        run += v;
    }
    const int total = *s_total;
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(FT, 1)
    k_hull_final(const int2 *__restrict__ cand, const int *__restrict__ segcnt,
                 const int *__restrict__ counts, int p, int nsegmax, int2 *gA, int2 *gB,
                 int *gseg, int2 *hull, int *hull_count)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_warp[32];
    __shared__ int s_total;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;

    const int m0 = max(0, min(counts[0], p)), m1 = max(0, min(counts[1], p));
    const int n0 = (m0 + HS - 1) / HS, n1 = (m1 + HS - 1) / HS, ns = n0 + n1;

    int *ix[6];
    const bool seg_smem = ns <= SCAP;
    for (int r = 0; r < 6; ++r)
        ix[r] = seg_smem ? reinterpret_cast<int *>(smem + 2 * PCAP * sizeof(int2)) + r * SCAP
                         : gseg + (size_t)r * 2 * nsegmax;
    int *segS = ix[0], *segL = ix[1], *nS = ix[2], *nL = ix[3], *U = ix[4], *V = ix[5];

    for (int s = t; s < ns; s += FT) {
        const int chain = s >= n0, seg = s - (chain ? n0 : 0);
        const int len = segcnt[chain * nsegmax + seg];
        segL[s] = len;
        segS[s] = len;
    }
    __syncthreads();
    const int total = block_excl_scan(segS, ns, s_warp, &s_total);
    const bool pt_smem = total <= PCAP;
    int2 *A = pt_smem ? reinterpret_cast<int2 *>(smem) : gA;
    int2 *B = pt_smem ? reinterpret_cast<int2 *>(smem) + PCAP : gB;

    for (int idx = t; idx < ns * HS; idx += FT) {
        const int s = idx / HS, k = idx - s * HS;
        if (k < segL[s]) {
            const int chain = s >= n0, seg = s - (chain ? n0 : 0);
            A[segS[s] + k] = cand[((size_t)chain * nsegmax + seg) * HS + k];
        }
    }
    __syncthreads();

    int c0 = n0, c1 = n1;
    while (c0 > 1 || c1 > 1) {
        const int d0 = (c0 + 1) >> 1, d1 = (c1 + 1) >> 1, nd = d0 + d1;
        for (int j = warp; j < nd; j += FT / 32) {
            const int chain = j >= d0;
            const int jj = j - (chain ? d0 : 0);
            const int cc = chain ? c1 : c0;
            const int ia = (chain ? c0 : 0) + 2 * jj, ib = ia + 1;
            if (2 * jj + 1 < cc) {
                int u, v;
                warp_bridge(A + segS[ia], segL[ia], A + segS[ib], segL[ib], lane, u, v);
                if (lane == 0) {
                    U[j] = u;
                    V[j] = v;
                    nL[j] = u + 1 + segL[ib] - v;
                }
            } else if (lane == 0) {
                U[j] = segL[ia] - 1;
                V[j] = -1;
                nL[j] = segL[ia];
            }
        }
        __syncthreads();
        for (int j = t; j < nd; j += FT)
            nS[j] = nL[j];
        __syncthreads();
        block_excl_scan(nS, nd, s_warp, &s_total);
        for (int j = warp; j < nd; j += FT / 32) {
            const int chain = j >= d0;
            const int jj = j - (chain ? d0 : 0);
            const int ia = (chain ? c0 : 0) + 2 * jj, ib = ia + 1;
            const int u = U[j], v = V[j];
            int2 *dst = B + nS[j];
            const int2 *sa = A + segS[ia];
            for (int k = lane; k <= u; k += 32)
                dst[k] = sa[k];
            if (v >= 0) {
                const int2 *sb = A + segS[ib];
                const int lb = segL[ib];
                for (int k = v + lane; k < lb; k += 32)
                    dst[u + 1 + k - v] = sb[k];
            }
        }
        __syncthreads();
        int2 *tp = A;
        A = B;
        B = tp;
        int *ti = segS;
        segS = nS;
        nS = ti;
        ti = segL;
        segL = nL;
        nL = ti;
        c0 = d0;
        c1 = d1;
    }

    // Stitch: lower hull left to right, then the upper hull right to left,
    // without repeating the shared end points.
    const int hl = c0 ? segL[0] : 0, hu = c1 ? segL[c0] : 0;
    const int2 *LH = A + (c0 ? segS[0] : 0);
    const int2 *UH = A + (c1 ? segS[c0] : 0);
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
    for (int k = t; k < hl; k += FT)
        hull[k] = LH[k];
    for (int k = t; k < nup; k += FT) {
        const int2 q = UH[kl - k];
        hull[hl + k] = make_int2(q.x, -q.y);
    }
    if (t == 0)
        *hull_count = hl + nup;
}

struct HullWs {
    size_t cand, segcnt, gA, gB, gseg, end;
};

HullWs hull_layout(int p)
{
    const size_t nsegmax = ((size_t)p + HS - 1) / HS;
    WsLayout w;
    HullWs h;
    h.cand = w.take(2 * nsegmax * HS * sizeof(int2));
    h.segcnt = w.take(2 * nsegmax * sizeof(int));
    h.gA = w.take(2 * nsegmax * HS * sizeof(int2));
    h.gB = w.take(2 * nsegmax * HS * sizeof(int2));
    h.gseg = w.take(6 * 2 * nsegmax * sizeof(int));
    h.end = w.off;
    return h;
}

}  // namespace

size_t hull_ws_bytes(int p) { return hull_layout(p).end; }

cudaError_t hull_launch(const int32_t *lower, const int32_t *upper, const int32_t *counts, int p,
                        int32_t *hull, int32_t *hull_count, void *ws, unsigned *status,
                        cudaStream_t s)
{
    (void)status;
    const HullWs h = hull_layout(p);
    const int nsegmax = (p + HS - 1) / HS;
    char *b = reinterpret_cast<char *>(ws);
    int2 *cand = reinterpret_cast<int2 *>(b + h.cand);
    int *segcnt = reinterpret_cast<int *>(b + h.segcnt);
    k_hull_seg<<<(2 * nsegmax + HT - 1) / HT, HT, 0, s>>>(
        reinterpret_cast<const int2 *>(lower), reinterpret_cast<const int2 *>(upper), counts, p,
        nsegmax, cand, segcnt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    e = cudaFuncSetAttribute(k_hull_final, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)FINAL_SMEM);
    if (e != cudaSuccess)
        return e;
    k_hull_final<<<1, FT, FINAL_SMEM, s>>>(cand, segcnt, counts, p, nsegmax,
                                           reinterpret_cast<int2 *>(b + h.gA),
                                           reinterpret_cast<int2 *>(b + h.gB),
                                           reinterpret_cast<int *>(b + h.gseg),
                                           reinterpret_cast<int2 *>(hull), hull_count);
    return cudaGetLastError();
}

}  // namespace ch
