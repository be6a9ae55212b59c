// Step 3: strict convex hull of the x-ordered chains, with no sort.
//
// The lower hull of the lower chain and the upper hull of the upper chain,
// stitched counter-clockwise from the lexicographic minimum, give the hull of
// the reduced set, which by the correctness argument of the Appendix is the
// hull of the input.  The upper chain is mirrored (y -> -y) so that one
// lower-hull routine serves both.
//
// k_hull_filter - per block of 1024 consecutive chain points (in shared
//                 memory), the exact pre-filter of hull_filter.cuh: a point
//                 on or above a segment between two other points of the
//                 block, one on each side, is not a strict vertex and goes;
//                 on chains of real data nearly all non-vertices go.
//                 Survivors of each block are compacted in order.
// k_hull_final  - one CTA gathers the survivors, runs Andrew's scan (pop while
//                 the turn is not strictly counter-clockwise, int64
//                 orientation) over runs of 16 of them per thread, merges the
//                 run hulls pairwise, level by level, and stitches the result.
// A merge of two x-separated lower hulls A (left) and B (right) happens in
// place, B's survivors moving left to follow A's.  Small pairs are merged by
// one thread continuing Andrew's scan over B; large pairs by a warp that
// finds the bridge (a_u, b_v) - the result being A[0..u] ++ B[v..] - with a
// 32-way search over A, each lane locating the tangent from its a_i to B by
// binary search.  Ties resolve towards the strict hull: the tangent takes the
// farthest of collinear B points, the bridge the leftmost of collinear A
// points.
#include "ch_internal.cuh"
#include "hull_filter.cuh"
#include "hull_merge.cuh"
#include "lookback.cuh"

namespace ch {
namespace {

constexpr int PCAP = 8192;    // survivors held in shared memory by the final CTA
constexpr size_t FINAL_SMEM =
    2 * PCAP * sizeof(int2) + PCAP * sizeof(int) + 4 * (PCAP / HS + 2) * sizeof(int);

// Survivors of chain run b (RUN consecutive chain points) of chain c.
__global__ void __launch_bounds__(RUN)
    k_hull_filter(const int2 *__restrict__ lower, const int2 *__restrict__ upper,
                  const int *__restrict__ counts, int p, int nblk, int2 *cand, int *ccnt)
{
    pdl_wait();
    pdl_trigger();
    __shared__ int2 P[RUN];
    __shared__ short M[2 * RUN];
    __shared__ int s_wc[RUN / 32 + 1];
    const int chain = blockIdx.x >= nblk;
    const int blk = blockIdx.x - chain * nblk;
    const int m = max(0, min(counts[chain], p));
    const int b0 = blk * RUN;
    const int nin = max(0, min(RUN, m - b0));
    if (threadIdx.x < nin) {
        int2 q = (chain ? upper : lower)[b0 + threadIdx.x];
        q.y = chain ? -q.y : q.y;
        P[threadIdx.x] = q;
    }
    __syncthreads();
    build_min_trees(P, M, nin, P, M, nin);
    const bool keep = run_keeps(P, M, nin, threadIdx.x);
    const int n = compact_run(P, keep, cand + (size_t)blockIdx.x * RUN, s_wc);
    if (threadIdx.x == 0)
        ccnt[blockIdx.x] = n;
}

// With many runs (long chains: large p or sparse data) the survivors are
// filtered once more before the final CTA: they are packed per chain
// (k_cand_compact: one warp per run, the runs' offsets by a look-back over
// tiles of 32 runs, the upper chain un-mirrored) and go through
// k_hull_filter again as chains of their own.  A point the second pass drops
// lies on or above a segment between two other points, as in the first, so
// every drop stays exact; the final CTA then sees a few survivors per 1024
// instead of the local hulls of every run.
constexpr int REFILTER_MIN_BLK = 128;  // runs per chain from which the second pass runs

__global__ void __launch_bounds__(1024)
    k_cand_compact(const int2 *__restrict__ cand, const int *__restrict__ ccnt, int nblk, int2 *out,
                   int *counts2, unsigned long long *state, int ntile, unsigned *status)
{
    pdl_wait();
    pdl_trigger();
    const int chain = blockIdx.y;
    unsigned long long *st = state + (size_t)chain * (ntile + 1);
    __shared__ int s_tile;
    __shared__ int s_off[32];
    __shared__ long long s_prefix;
    if (threadIdx.x == 0)
        s_tile = (int)atomicAdd(st, 1ull);
    __syncthreads();
    const int tile = s_tile, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        const int r = tile * 32 + lane;
        const int v = r < nblk ? ccnt[(size_t)chain * nblk + r] : 0;
        int inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if (lane >= o)
                inc += x;
        }
        s_off[lane] = inc - v;
        const int tot = __shfl_sync(0xFFFFFFFFu, inc, 31);
        if (lane == 0)
            publish_aggregate(st + 1, tile, tot);
        const long long pre = warp_look_back(st + 1, tile, tot, lane, status);
        if (lane == 0) {
            s_prefix = pre;
            if (tile == ntile - 1)
                counts2[chain] = (int)(pre + tot);
        }
    }
    __syncthreads();
    const int run = tile * 32 + warp;
    if (run >= nblk)
        return;
    const int len = ccnt[(size_t)chain * nblk + run];
    const int2 *src = cand + ((size_t)chain * nblk + run) * RUN;
    int2 *dst = out + (size_t)chain * nblk * RUN + s_prefix + s_off[warp];
    for (int k = lane; k < len; k += 32) {
        int2 q = src[k];
        if (chain)
            q.y = -q.y;
        dst[k] = q;
    }
}

// The final CTA: gathers the survivors of every run (chain 0 first) into A,
// then peels, merges and stitches them (hull_merge.cuh).
template <bool SM, bool NARROW>
__device__ __forceinline__ void final_body(const int2 *__restrict__ cand, const int *__restrict__ ccnt,
                                           const int *offs, int nblk, int T0, int T, int2 *gA,
                                           int2 *gB, int *gF, int *gix, int2 *hull, int *hull_count,
                                           int *s_warp, int *s_total)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    int2 *A = SM ? reinterpret_cast<int2 *>(smem) : gA;
    int2 *B = SM ? reinterpret_cast<int2 *>(smem) + PCAP : gB;
    int *F = SM ? reinterpret_cast<int *>(reinterpret_cast<int2 *>(smem) + 2 * PCAP) : gF;
    int *ix = SM ? reinterpret_cast<int *>(reinterpret_cast<int2 *>(smem) + 2 * PCAP) + PCAP : gix;

    // gather
    for (int s = warp; s < 2 * nblk; s += FT / 32) {
        const int2 *src = cand + (size_t)s * RUN;
        const int len = ccnt[s], st = offs[s];
        for (int k0 = 0; k0 < len; k0 += 128) {
            int2 q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (k0 + u * 32 + lane < len)
                    q[u] = src[k0 + u * 32 + lane];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (k0 + u * 32 + lane < len)
                    A[st + k0 + u * 32 + lane] = q[u];
        }
    }
    __syncthreads();

    peel_merge_stitch<FT, 0, NARROW>(A, B, F, ix, T0, T, hull, hull_count, s_warp, s_total);
}

// NARROW: 32-bit orientation tests in the peeling (the survivors of chains of
// a frame of side and rows at most 16384).
template <bool NARROW>
__global__ void __launch_bounds__(FT, 1)
    k_hull_final(const int2 *__restrict__ cand, const int *__restrict__ ccnt, int nblk, int2 *gA,
                 int2 *gB, int *gF, int *gix, int2 *hull, int *hull_count)
{
    pdl_wait();
    pdl_trigger();
    __shared__ int s_warp[32];
    __shared__ int s_total, s_t0;
    __shared__ int s_offs[2 * 128 + 1];
    const int t = threadIdx.x, nb = 2 * nblk;
    int *offs = nb <= 2 * 128 ? s_offs : gix;  // global scratch reused before the fallback
    for (int s = t; s < nb; s += FT)
        offs[s] = ccnt[s];
    __syncthreads();
    const int total = block_excl_scan<FT>(offs, nb, s_warp, &s_total);
    if (t == 0)
        s_t0 = offs[nblk];
    __syncthreads();
    const int T0 = s_t0;
    if (total <= PCAP)
        final_body<true, NARROW>(cand, ccnt, offs, nblk, T0, total, gA, gB, gF, gix + nb + 1, hull,
                         hull_count, s_warp, &s_total);
    else
        final_body<false, NARROW>(cand, ccnt, offs, nblk, T0, total, gA, gB, gF, gix + nb + 1, hull,
                          hull_count, s_warp, &s_total);
}

}  // namespace

HullLayout hull_layout(int p)
{
    const size_t nblk = ((size_t)p + RUN - 1) / RUN;
    const size_t cap = 2 * nblk * RUN;  // survivors of both chains, at most
    WsLayout w;
    HullLayout h;
    h.nblk = (int)nblk;
    h.cand = w.take(cap * sizeof(int2));
    h.ccnt = w.take(2 * nblk * sizeof(int));
    h.gA = w.take(cap * sizeof(int2));
    h.gB = w.take(cap * sizeof(int2));
    h.gF = w.take(cap * sizeof(int));
    h.gix = w.take((2 * nblk + 1 + 4 * (cap / HS + 2)) * sizeof(int));
    // second pass (packed survivors in gA, its survivors in gB)
    h.refilter = nblk >= (size_t)REFILTER_MIN_BLK;
    const size_t ntile = (nblk + 31) / 32;
    h.ccnt2 = w.take(h.refilter ? 2 * nblk * sizeof(int) : 0);
    h.counts2 = w.take(h.refilter ? 8 : 0);
    h.state2 = w.take(h.refilter ? 2 * (ntile + 1) * 8 : 0);
    h.end = w.off;
    return h;
}

namespace {

cudaError_t set_attrs()
{
    static bool attrs_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64)
        return cudaErrorInvalidDevice;
    if (!attrs_set[dev]) {
        cudaError_t a = cudaFuncSetAttribute(k_hull_final<false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)FINAL_SMEM);
        if (a == cudaSuccess)
            a = cudaFuncSetAttribute(k_hull_final<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)FINAL_SMEM);
        if (a != cudaSuccess)
            return a;
        attrs_set[dev] = true;
    }
    return cudaSuccess;
}

}  // namespace

size_t hull_ws_bytes(int p) { return hull_layout(p).end; }

cudaError_t hull_final_launch(const HullLayout &h, void *ws, int32_t *hull, int32_t *hull_count,
                              cudaStream_t s, bool narrow)
{
    cudaError_t e = set_attrs();
    if (e != cudaSuccess)
        return e;
    char *b = reinterpret_cast<char *>(ws);
    size_t cand = h.cand, ccnt = h.ccnt;
    if (h.refilter) {
        unsigned *status = device_status_ptr(s);
        if (!status)
            return cudaErrorUnknown;
        const int ntile = (h.nblk + 31) / 32;
        e = cudaMemsetAsync(b + h.state2, 0, (size_t)2 * (ntile + 1) * 8, s);
        if (e != cudaSuccess)
            return e;
        int2 *packed = reinterpret_cast<int2 *>(b + h.gA);
        int *counts2 = reinterpret_cast<int *>(b + h.counts2);
        launch(k_cand_compact, dim3(ntile, 2), 1024, 0, s, reinterpret_cast<const int2 *>(b + h.cand),
               reinterpret_cast<const int *>(b + h.ccnt), h.nblk, packed, counts2,
               reinterpret_cast<unsigned long long *>(b + h.state2), ntile, status);
        const size_t half = (size_t)h.nblk * RUN;
        launch(k_hull_filter, 2 * h.nblk, RUN, 0, s, (const int2 *)packed, (const int2 *)(packed + half),
               (const int *)counts2, (int)half, h.nblk, reinterpret_cast<int2 *>(b + h.gB),
               reinterpret_cast<int *>(b + h.ccnt2));
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
        cand = h.gB;  // gathered by the final CTA before it reuses gB
        ccnt = h.ccnt2;
    }
    launch(narrow ? k_hull_final<true> : k_hull_final<false>, 1, FT, FINAL_SMEM, s,
        reinterpret_cast<const int2 *>(b + cand), reinterpret_cast<const int *>(b + ccnt), h.nblk,
        reinterpret_cast<int2 *>(b + h.gA), reinterpret_cast<int2 *>(b + h.gB),
        reinterpret_cast<int *>(b + h.gF), reinterpret_cast<int *>(b + h.gix),
        reinterpret_cast<int2 *>(hull), hull_count);
    return cudaGetLastError();
}

cudaError_t hull_launch(const int32_t *lower, const int32_t *upper, const int32_t *counts, int p,
                        int32_t *hull, int32_t *hull_count, void *ws, unsigned *status,
                        cudaStream_t s)
{
    (void)status;
    const HullLayout h = hull_layout(p);
    char *b = reinterpret_cast<char *>(ws);
    launch(k_hull_filter, 2 * h.nblk, RUN, 0, s, reinterpret_cast<const int2 *>(lower),
                                             reinterpret_cast<const int2 *>(upper), counts, p,
                                             h.nblk, reinterpret_cast<int2 *>(b + h.cand),
                                             reinterpret_cast<int *>(b + h.ccnt));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    return hull_final_launch(h, ws, hull, hull_count, s);
}

}  // namespace ch
