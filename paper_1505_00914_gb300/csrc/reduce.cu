// Step 1: Algorithm 1 (Reduction of Points, Section 2.1) on sm_103a.
//
// Each point (x, y) folds into column x of L as (min(y, ly), max(y, hy)).
// Min and max commute, so the GPU may fold in any order and into any number
// of partial arrays that are merged column by column afterwards.  Only the
// native 32-bit shared-memory atomicMin/atomicMax run at streaming speed on
// GB300 (compare-and-swap and cluster-remote atomics are an order of
// magnitude slower), which fixes the two forms used here:
//
// Private form (8p bytes of shared memory, p <= 20480):
//   every CTA (one per SM) keeps int32 lo[p], hi[p] in shared memory, folds
//   its slice of the points with unconditional shared atomics and writes its
//   copy as one row of a partial array, packed as ((lo-1) << 16) | (hi-1)
//   (0xFFFF0000 for an empty column); the chain step merges the rows.
//
// Filtered form (larger p): L lives in global memory and every CTA keeps a
//   16-bit filter per column in shared memory: a row bin (y-1) >> shift for
//   each of L's two extremes.  Every value a filter ever holds is the row bin
//   of some input point, so the point(s) with a column's least y always have
//   a bin <= the filter's lo bin and always pass, and a point whose bin is
//   strictly above the lo bin cannot be that least y (likewise for the
//   greatest y).  A point whose bin lies strictly between the two bins is
//   therefore dropped after one shared load; any other point is folded into
//   L with a global red.min / red.max and tightens the CTA's filter (plain,
//   racing byte stores are safe: whichever lands, the value is still some
//   point's bin).
//   The filters start warm: k_filter_warm has each CTA build a filter from
//   the first sixteenth of the slice it will reduce and store it as one row
//   of a slot array; k_filter_merge folds the rows column-wise into one
//   filter G (and fills L with (p+1, -1)); k_reduce_filtered starts from G
//   and folds the whole slice (the warm-up part again, from L2).  About one
//   point in fifty reaches global memory.
//   Filters need 2p bytes of shared memory (p <= 116224); beyond that every
//   point takes a read-then-atomic test against the global L.
#include <map>
#include <mutex>
#include <tuple>

#include "ch_internal.cuh"

namespace ch {
namespace {

#ifndef CH_RU
#define CH_RU 4
#endif
constexpr int RU = CH_RU;        // 16-byte loads in flight per thread per iteration

// The point array is read as 16-byte vectors from the first 16-byte
// boundary: two int32 (x, y) points per vector, or four packed 16-bit points
// (FM 3, one 32-bit word (x - 1) | (y - 1) << 16 per point).  The points
// before the boundary (head) and after the last whole vector (tail) are
// taken one by one.
template <int FM>
constexpr int WPP = FM == 3 ? 1 : 2;  // 32-bit words per point
template <int FM>
constexpr int PPV = 4 / WPP<FM>;  // points per 16-byte vector

struct VecView {
    const int4 *p4;
    int64_t nvec;
    int head;  // points before the first vector (0 .. PPV - 1)
    int tail;  // points after the last vector (0 .. PPV - 1)
};

template <int FM>
__device__ __forceinline__ VecView vec_view(const int32_t *pts, int64_t n)
{
    VecView v;
    const int64_t h = (int64_t)(((16 - ((uintptr_t)pts & 15)) & 15) / (4 * WPP<FM>));
    v.head = (int)min(h, n);
    v.nvec = (n - v.head) / PPV<FM>;
    v.tail = (int)(n - v.head - v.nvec * PPV<FM>);
    v.p4 = reinterpret_cast<const int4 *>(pts + WPP<FM> * v.head);
    return v;
}

// Point k of the array.
template <int FM>
__device__ __forceinline__ void point_at(const int32_t *pts, int64_t k, int &x, int &y)
{
    if constexpr (FM == 3) {
        const uint32_t w = (uint32_t)pts[k];
        x = (int)(w & 0xFFFFu) + 1;
        y = (int)(w >> 16) + 1;
    } else {
        x = pts[2 * k];
        y = pts[2 * k + 1];
    }
}

// fold(x, y) for every point of one vector.
template <int FM, typename Fold>
__device__ __forceinline__ void each_point(const int4 &v, Fold &&fold)
{
    if constexpr (FM == 3) {
        const uint32_t w[4] = {(uint32_t)v.x, (uint32_t)v.y, (uint32_t)v.z, (uint32_t)v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            fold((int)(w[k] & 0xFFFFu) + 1, (int)(w[k] >> 16) + 1);
    } else {
        fold(v.x, v.y);
        fold(v.z, v.w);
    }
}

// The head points (first CTA) and tail points (last CTA), one thread each.
template <int FM, typename Fold>
__device__ __forceinline__ void fold_edges(const int32_t *pts, int64_t n, const VecView &v,
                                           Fold &&fold)
{
    if (threadIdx.x != 0)
        return;
    int x, y;
    if (blockIdx.x == 0)
        for (int k = 0; k < v.head; ++k) {
            point_at<FM>(pts, k, x, y);
            fold(x, y);
        }
    if (blockIdx.x == gridDim.x - 1)
        for (int k = 0; k < v.tail; ++k) {
            point_at<FM>(pts, n - v.tail + k, x, y);
            fold(x, y);
        }
}

// Streams the 16-byte vectors [s0, e0) of a CTA's slice: each thread keeps
// RU loads in flight and issues its next RU before folding the current ones
// (register double buffering), so the loads never wait for the folding.
// fold(v) takes one vector of points.  KEEP: load through L2 with the
// normal policy (the data is read again soon) instead of evict-first.
// The same over 64-bit indices.
template <int RT, bool KEEP, typename Fold>
__device__ __forceinline__ void stream_pairs_wide(const int4 *__restrict__ p4, int64_t s0,
                                                  int64_t e0, Fold &fold)
{
    auto ld = [&](int64_t j) { return KEEP ? __ldcg(p4 + j) : __ldcs(p4 + j); };
    int4 v[RU];
#pragma unroll
    for (int u = 0; u < RU; ++u) {
        const int64_t j = s0 + threadIdx.x + (int64_t)u * RT;
        v[u] = j < e0 ? ld(j) : make_int4(0, 0, 0, 0);
    }
    for (int64_t i = s0 + threadIdx.x; i < e0; i += (int64_t)RT * RU) {
        int4 w[RU];
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            const int64_t j = i + (int64_t)(RU + u) * RT;
            w[u] = j < e0 ? ld(j) : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < RU; ++u)
            if (i + (int64_t)u * RT < e0)
                fold(v[u]);
#pragma unroll
        for (int u = 0; u < RU; ++u)
            v[u] = w[u];
    }
}

#ifndef CH_STREAM32
#define CH_STREAM32 1  // index a slice with 32-bit offsets from its first vector
#endif
template <int RT, bool KEEP = false, typename Fold>
__device__ __forceinline__ void stream_pairs(const int4 *__restrict__ p4, int64_t s0, int64_t e0,
                                             Fold &&fold)
{
#if CH_STREAM32
    // a slice below 2^31 - 2 RU RT vectors (any that fits in memory at one
    // CTA per SM) is indexed by 32-bit offsets from its start, which keeps the
    // loop's index tests and address sums single-word
    if (e0 - s0 > (int64_t)(0x7FFFFFFF - 2 * RU * RT)) {
        stream_pairs_wide<RT, KEEP>(p4, s0, e0, fold);
        return;
    }
    const int4 *__restrict__ q = p4 + s0;
    const int len = (int)(e0 - s0);
    auto ld = [&](int j) { return KEEP ? __ldcg(q + j) : __ldcs(q + j); };
    int4 v[RU];
#pragma unroll
    for (int u = 0; u < RU; ++u) {
        const int j = (int)threadIdx.x + u * RT;
        v[u] = j < len ? ld(j) : make_int4(0, 0, 0, 0);
    }
    for (int i = (int)threadIdx.x; i < len; i += RT * RU) {
        int4 w[RU];
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            const int j = i + (RU + u) * RT;
            w[u] = j < len ? ld(j) : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < RU; ++u)
            if (i + u * RT < len)
                fold(v[u]);
#pragma unroll
        for (int u = 0; u < RU; ++u)
            v[u] = w[u];
    }
#else
    stream_pairs_wide<RT, KEEP>(p4, s0, e0, fold);
#endif
}

// ---------------------------------------------------------------- private
template <int RT, int FM>
__global__ void __launch_bounds__(RT)
    k_reduce_private(const int32_t *__restrict__ pts, int64_t n, Frame f,
                     uint32_t *__restrict__ part, unsigned *status)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) int sI[];
    const int nc = f.nc;
    int *slo = sI, *shi = sI + nc;
    for (int i = threadIdx.x; i < nc; i += RT) {
        slo[i] = f.nr + 1;
        shi[i] = -1;
    }
    __syncthreads();
    bool bad = false;
    auto fold = [&](int x, int y) {
        uint32_t c, rr;
        frame_map<FM>(f, x, y, c, rr);
        if (c >= (uint32_t)nc || rr >= (uint32_t)f.nr) {
            bad = true;
            return;
        }
        const int r = (int)rr + 1;
        // a read first: the entry only ever tightens, so a point that cannot
        // improve the value read cannot improve the current one either
        if (r < slo[c])
            atomicMin(slo + c, r);
        if (r > shi[c])
            atomicMax(shi + c, r);
    };
    const VecView pv = vec_view<FM>(pts, n);
    fold_edges<FM>(pts, n, pv, fold);
    const int64_t per = (pv.nvec + gridDim.x - 1) / gridDim.x;
    const int64_t s0 = (int64_t)blockIdx.x * per;
    const int64_t e0 = min(pv.nvec, s0 + per);
    stream_pairs<RT>(pv.p4, s0, e0, [&](const int4 &v) { each_point<FM>(v, fold); });
    __syncthreads();
    uint32_t *out = part + (size_t)blockIdx.x * nc;
    for (int i = threadIdx.x; i < nc; i += RT)  // rows <= 65536 in this form
        out[i] = slo[i] <= f.nr ? ((uint32_t)(slo[i] - 1) << 16) | (uint32_t)(shi[i] - 1)
                                : 0xFFFF0000u;
    if (__syncthreads_or(bad) && threadIdx.x == 0)
        atomicOr(status, ST_RANGE);
}

// --------------------------------------------------------------- filtered
__global__ void k_fill_empty(int2 *L, int nc, int nr, unsigned long long *zero, int nzero)
{
    pdl_wait();
    pdl_trigger();
    if (zero && blockIdx.x == 0)
        for (int i = threadIdx.x; i < nzero; i += blockDim.x)
            zero[i] = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
        L[i] = make_int2(nr + 1, -1);
}

// Read-then-atomic fold of one point into the global L.
template <int FM>
__device__ __forceinline__ bool fold_global(int2 *L, const Frame &f, int x, int y)
{
    uint32_t c, rr;
    frame_map<FM>(f, x, y, c, rr);
    if (c >= (uint32_t)f.nc || rr >= (uint32_t)f.nr)
        return false;
    const int r = (int)rr + 1;
    const int2 e = L[c];
    if (r < e.x)
        atomicMin(&L[c].x, r);
    if (r > e.y)
        atomicMax(&L[c].y, r);
    return true;
}

// Whole input through the read-then-atomic test (too many columns for a filter).
template <int FM>
__global__ void __launch_bounds__(256)
    k_reduce_global(const int32_t *__restrict__ pts, int64_t n, Frame f, int2 *L, unsigned *status)
{
    pdl_wait();
    pdl_trigger();
    const VecView pv = vec_view<FM>(pts, n);
    bool bad = false;
    auto fold = [&](int x, int y) { bad |= !fold_global<FM>(L, f, x, y); };
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < pv.nvec;
         j += (int64_t)gridDim.x * blockDim.x)
        each_point<FM>(__ldcs(pv.p4 + j), fold);
    fold_edges<FM>(pts, n, pv, fold);
    if (__syncthreads_or(bad) && threadIdx.x == 0)
        atomicOr(status, ST_RANGE);
}


#ifndef CH_WARM_DIV
#define CH_WARM_DIV 16
#endif
constexpr int WARM_DIV = CH_WARM_DIV;  // the warm-up reads the first 1/WARM_DIV of each slice

// Slice of point vectors [s0, e0) reduced by CTA `b` of `grid`.
__device__ __forceinline__ void slice_of(int64_t nvec, int b, int grid, int64_t &s0, int64_t &e0)
{
    const int64_t per = (nvec + grid - 1) / grid;
    s0 = (int64_t)b * per;
    e0 = min(nvec, s0 + per);
}

// Filter words are (lo bin << 8) | hi bin; "tighter of" two packed words is
// a byte-wise min on the lo bytes and max on the hi bytes.
__device__ __forceinline__ uint32_t tighter2(uint32_t a, uint32_t b)
{
    return (__vminu4(a, b) & 0xFF00FF00u) | (__vmaxu4(a, b) & 0x00FF00FFu);
}

__device__ __forceinline__ uint4 tighter8(uint4 a, uint4 b)
{
    return make_uint4(tighter2(a.x, b.x), tighter2(a.y, b.y), tighter2(a.z, b.z), tighter2(a.w, b.w));
}

// Thread-block cluster helpers (a launch without clusters is a cluster of one).
__device__ __forceinline__ unsigned cluster_ctas()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Every thread of every CTA of the cluster; orders the shared-memory writes
// before it with the reads after it, cluster-wide.
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}
// 16 bytes at the same shared-memory offset as `p`, in CTA `rank` of the cluster.
__device__ __forceinline__ uint4 ld_cluster_v4(const void *p, unsigned rank)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    unsigned ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    uint4 v;
    asm volatile("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(ra)
                 : "memory");
    return v;
}

// Each CTA builds a filter from the first 1/WARM_DIV of its slice.  Launched
// in clusters of C CTAs, the C filters of a cluster are merged through
// distributed shared memory (CTA rank r merges the r-th C-th of the columns
// over all C) and the cluster writes one slot row, so the merge kernel reads
// grid / C rows instead of grid.
template <int RT, int FM>
__global__ void __launch_bounds__(RT)
    k_filter_warm(const int32_t *__restrict__ pts, int64_t n, Frame fr, int shift, int grid,
                  uint16_t *__restrict__ slots)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) uint16_t F[];
    unsigned char *fb = reinterpret_cast<unsigned char *>(F);
    const int words = (fr.nc + 7) / 8;
    uint4 *F4 = reinterpret_cast<uint4 *>(F);
    for (int i = threadIdx.x; i < words; i += RT)
        F4[i] = make_uint4(0xFF00FF00u, 0xFF00FF00u, 0xFF00FF00u, 0xFF00FF00u);
    __syncthreads();
    auto learn = [&](int x, int y) {
        uint32_t c, rr;
        frame_map<FM>(fr, x, y, c, rr);
        if (c >= (uint32_t)fr.nc || rr >= (uint32_t)fr.nr)
            return;
        const uint32_t f = F[c], b = rr >> shift;
        if (b < (f >> 8))
            fb[2 * c + 1] = (unsigned char)b;
        if (b > (f & 0xFFu))
            fb[2 * c] = (unsigned char)b;
    };
    const VecView pv = vec_view<FM>(pts, n);
    int64_t s0, e0;
    slice_of(pv.nvec, blockIdx.x, grid, s0, e0);
    const int64_t warm = s0 + (e0 - s0) / WARM_DIV;
    stream_pairs<RT, true>(pv.p4, s0, warm, [&](const int4 &v) { each_point<FM>(v, learn); });
    const unsigned C = cluster_ctas();
    uint4 *out = reinterpret_cast<uint4 *>(slots) + (size_t)(blockIdx.x / C) * words;
    if (C == 1) {
        __syncthreads();
        for (int i = threadIdx.x; i < words; i += RT)
            __stcg(out + i, F4[i]);
        return;
    }
    cluster_sync();  // every filter of the cluster is complete
    const unsigned r = cluster_rank();
    const int per = (int)((words + C - 1) / C);
    const int i1 = min(words, (int)(r + 1) * per);
    for (int i = (int)r * per + threadIdx.x; i < i1; i += RT) {
        uint4 acc = F4[i];
        for (unsigned k = 1; k < C; ++k)
            acc = tighter8(acc, ld_cluster_v4(F4 + i, (r + k) % C));
        __stcg(out + i, acc);
    }
    cluster_sync();  // no CTA exits while another may still read its filter
}

// G = column-wise tighter-of over the `rows` slot rows; also L = (p+1, -1).
// A CTA has MG_GROUPS thread groups over the same MG_V uint4 words (8
// columns each); group g folds rows g, g + MG_GROUPS, ...
constexpr int MG_V = 32, MG_GROUPS = 32;

__global__ void __launch_bounds__(MG_V *MG_GROUPS)
    k_filter_merge(const uint16_t *__restrict__ slots, int rows, int p, int nr, uint16_t *__restrict__ G,
                   int2 *__restrict__ L, unsigned long long *zero, int nzero)
{
    pdl_wait();
    pdl_trigger();
    if (zero && blockIdx.x == 0)
        for (int i = threadIdx.x; i < nzero; i += blockDim.x)
            zero[i] = 0;
    __shared__ uint4 part[MG_GROUPS][MG_V];
    const int words = (p + 7) / 8;
    const int v = threadIdx.x % MG_V, g = threadIdx.x / MG_V;
    const int i = blockIdx.x * MG_V + v;
    uint4 acc = make_uint4(0xFF00FF00u, 0xFF00FF00u, 0xFF00FF00u, 0xFF00FF00u);
    if (i < words) {
        const uint4 *s4 = reinterpret_cast<const uint4 *>(slots) + i;
        int r = g;
        for (; r + 7 * MG_GROUPS < rows; r += 8 * MG_GROUPS) {
            uint4 w[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                w[u] = __ldcg(s4 + (size_t)(r + u * MG_GROUPS) * words);
#pragma unroll
            for (int u = 0; u < 8; ++u)
                acc = tighter8(acc, w[u]);
        }
        for (; r < rows; r += MG_GROUPS)
            acc = tighter8(acc, __ldcg(s4 + (size_t)r * words));
    }
    part[g][v] = acc;
    __syncthreads();
    if (g == 0 && i < words) {
#pragma unroll
        for (int h = 1; h < MG_GROUPS; ++h)
            acc = tighter8(acc, part[h][v]);
        reinterpret_cast<uint4 *>(G)[i] = acc;
    }
    const int c0 = blockIdx.x * MG_V * 8;
    for (int c = c0 + threadIdx.x; c < min(p, c0 + MG_V * 8); c += MG_V * MG_GROUPS)
        L[c] = make_int2(nr + 1, -1);
}

template <int RT, int FM>
__global__ void __launch_bounds__(RT)
    k_reduce_filtered(const int32_t *__restrict__ pts, int64_t n, Frame fr, int shift,
                      const uint16_t *__restrict__ G, int2 *L, unsigned *status)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) uint16_t F[];
    unsigned char *fb = reinterpret_cast<unsigned char *>(F);
    {
        const int words = (fr.nc + 7) / 8;
        const uint4 *G4 = reinterpret_cast<const uint4 *>(G);
        uint4 *F4 = reinterpret_cast<uint4 *>(F);
        for (int i0 = threadIdx.x; i0 < words; i0 += RT * 8) {
            uint4 g[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (i0 + u * RT < words)
                    g[u] = __ldcg(G4 + i0 + u * RT);
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (i0 + u * RT < words)
                    F4[i0 + u * RT] = g[u];
        }
    }
    __syncthreads();
    bool bad = false;
    auto fold = [&](int x, int y) {
        uint32_t c, rr;
        frame_map<FM>(fr, x, y, c, rr);
        if constexpr (FM == 3) {
            // packed 16-bit points, four per load, leave the fold issue-bound:
            // no early exit for a point outside the frame (it reads column 0's
            // filter and passes no test), which drops a branch per point
            // (bench: 729 -> 781 Gpoints/s; with int32 pairs it gains nothing)
            const bool ok = c < (uint32_t)fr.nc && rr < (uint32_t)fr.nr;
            bad |= !ok;
            c = ok ? c : 0u;
            const int r = (int)rr + 1;
            const uint32_t f = F[c], b = rr >> shift;
            const uint32_t qlo = f >> 8, qhi = f & 0xFFu;
            if (ok && b <= qlo) {
                atomicMin(&L[c].x, r);
                if (b < qlo)
                    fb[2 * c + 1] = (unsigned char)b;
            }
            if (ok && b >= qhi) {
                atomicMax(&L[c].y, r);
                if (b > qhi)
                    fb[2 * c] = (unsigned char)b;
            }
        } else {
            if (c >= (uint32_t)fr.nc || rr >= (uint32_t)fr.nr) {
                bad = true;
                return;
            }
            const int r = (int)rr + 1;
            const uint32_t f = F[c], b = rr >> shift;
            const uint32_t qlo = f >> 8, qhi = f & 0xFFu;
            if (b <= qlo) {
                atomicMin(&L[c].x, r);
                if (b < qlo)
                    fb[2 * c + 1] = (unsigned char)b;
            }
            if (b >= qhi) {
                atomicMax(&L[c].y, r);
                if (b > qhi)
                    fb[2 * c] = (unsigned char)b;
            }
        }
    };
    const VecView pv = vec_view<FM>(pts, n);
    fold_edges<FM>(pts, n, pv, fold);
    int64_t s0, e0;
    slice_of(pv.nvec, blockIdx.x, gridDim.x, s0, e0);
    stream_pairs<RT>(pv.p4, s0, e0, [&](const int4 &v) { each_point<FM>(v, fold); });
    if (__syncthreads_or(bad) && threadIdx.x == 0)
        atomicOr(status, ST_RANGE);
}

// L = column-wise merge of the packed partial rows.  A CTA covers 32 columns
// with 32 thread groups; group g folds rows g, g + 32, ... (all loads of a
// thread in flight together), and the groups combine through shared memory.
__global__ void __launch_bounds__(1024)
    k_merge_partials(const uint32_t *__restrict__ part, int copies, int p, int nr, int2 *L,
                     unsigned long long *zero, int nzero, const int2 *__restrict__ Linit)
{
    pdl_wait();
    pdl_trigger();
    if (zero && blockIdx.x == 0)
        for (int i = threadIdx.x; i < nzero; i += blockDim.x)
            zero[i] = 0;
    __shared__ uint32_t s_lo[32][33], s_hi[32][33];
    const int v = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int c = blockIdx.x * 32 + v;
    uint32_t lo = 0xFFFFu, hi = 0;
    if (c < p) {
        int r = g;
        for (; r + 7 * 32 < copies; r += 8 * 32) {
            uint32_t w[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                w[u] = __ldcg(part + (size_t)(r + u * 32) * p + c);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                lo = min(lo, w[u] >> 16);
                hi = max(hi, w[u] & 0xFFFFu);
            }
        }
        for (; r < copies; r += 32) {
            const uint32_t w = __ldcg(part + (size_t)r * p + c);
            lo = min(lo, w >> 16);
            hi = max(hi, w & 0xFFFFu);
        }
    }
    s_lo[g][v] = lo;
    s_hi[g][v] = hi;
    __syncthreads();
    if (g == 0 && c < p) {
#pragma unroll 8
        for (int h = 1; h < 32; ++h) {
            lo = min(lo, s_lo[h][v]);
            hi = max(hi, s_hi[h][v]);
        }
        int2 r = lo <= hi ? make_int2((int)lo + 1, (int)hi + 1) : make_int2(nr + 1, -1);
        if (Linit) {  // a culled reduction starts from Linit instead of (p+1, -1)
            const int2 li = Linit[c];
            r = make_int2(min(r.x, li.x), max(r.y, li.y));
        }
        L[c] = r;
    }
}

// Per-device facts the plan needs, computed once: the opt-in shared memory
// limit, kernel attributes raised to it, and the private kernels' occupancy
// at each shared-memory size class.
struct DevInfo {
    bool ready = false;
    int optin = 0;
};
std::mutex g_dev_mu;
DevInfo g_dev[64];
std::map<std::pair<int, size_t>, int> g_bps;  // (device, smem) -> CTAs/SM of the private kernel

int dev_setup(int *dev_out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return -1;
    *dev_out = dev;
    std::lock_guard<std::mutex> g(g_dev_mu);
    DevInfo &d = g_dev[dev];
    if (!d.ready) {
        if (cudaDeviceGetAttribute(&d.optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess)
            return -1;
        const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
        cudaFuncSetAttribute(k_reduce_private<1024, 0>, a, d.optin);
        cudaFuncSetAttribute(k_reduce_private<1024, 1>, a, d.optin);
        cudaFuncSetAttribute(k_reduce_private<1024, 2>, a, d.optin);
        cudaFuncSetAttribute(k_reduce_filtered<1024, 0>, a, d.optin);
        cudaFuncSetAttribute(k_reduce_filtered<1024, 1>, a, d.optin);
        cudaFuncSetAttribute(k_reduce_filtered<1024, 2>, a, d.optin);
        cudaFuncSetAttribute(k_filter_warm<1024, 0>, a, d.optin);
        cudaFuncSetAttribute(k_filter_warm<1024, 1>, a, d.optin);
        cudaFuncSetAttribute(k_filter_warm<1024, 2>, a, d.optin);
        cudaFuncSetAttribute(k_reduce_private<1024, 3>, a, d.optin);
        cudaFuncSetAttribute(k_reduce_filtered<1024, 3>, a, d.optin);
        cudaFuncSetAttribute(k_filter_warm<1024, 3>, a, d.optin);
        d.ready = true;
    }
    return d.optin;
}

int private_bps(int dev, size_t smem)
{
    std::lock_guard<std::mutex> g(g_dev_mu);
    auto key = std::make_pair(dev, smem);
    auto it = g_bps.find(key);
    if (it != g_bps.end())
        return it->second;
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_reduce_private<1024, 0>, 1024,
                                                      smem) != cudaSuccess)
        return -1;
    g_bps[key] = bps;
    return bps;
}

// Shared memory the private form may use.  Above it the filtered form is
// faster: a private copy of 8p bytes leaves the SM too little L1 for the
// loads in flight (a whole call on 2^26 points: p = 16384 private 115.9 us
// against filtered 120.5; p = 24576 126.5 against 123.8; p = 29056 155.6
// against 122.8).
#ifndef CH_PRIVATE_SMEM_MAX
#define CH_PRIVATE_SMEM_MAX 163840u  // p <= 20480
#endif
#ifndef CH_FILTER_SMEM_MAX
#define CH_FILTER_SMEM_MAX (1u << 30)  // the filtered form up to the opt-in limit (the global form is slower)
#endif
#ifndef CH_WARM_CLUSTER_MAX
#define CH_WARM_CLUSTER_MAX 8  // largest cluster of the filter warm-up (portable limit)
#endif
std::map<std::tuple<int, size_t, int>, int> g_wcl;  // (device, smem, grid) -> cluster size

// Largest cluster size C <= CH_WARM_CLUSTER_MAX (a power of two dividing the
// grid) for which the whole warm-up grid is resident at once, so that no
// cluster waits for a second wave; 1 if none.
int warm_cluster(int dev, size_t smem, int grid)
{
    std::lock_guard<std::mutex> g(g_dev_mu);
    const auto key = std::make_tuple(dev, smem, grid);
    auto it = g_wcl.find(key);
    if (it != g_wcl.end())
        return it->second;
    int best = 1;
    for (int C = CH_WARM_CLUSTER_MAX; C >= 2; C /= 2) {
        if (grid % C)
            continue;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(1024);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_filter_warm<1024, 0>, &cfg) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if ((long long)nclusters * C >= grid) {
            best = C;
            break;
        }
    }
    g_wcl[key] = best;
    return best;
}

int filter_shift(int p)
{
    int s = 0;
    while (((p - 1) >> s) > 255)
        ++s;
    return s;
}

}  // namespace

int reduce_plan(int64_t n, int nc, int nr, ReducePlan *pl)
{
    const int sms = sm_count();
    if (sms <= 0)
        return CH_ERR_CUDA;
    int dev = 0;
    const int optin_i = dev_setup(&dev);
    if (optin_i <= 0)
        return CH_ERR_CUDA;
    const size_t optin = (size_t)optin_i;
    const int64_t npairs = n / 2;
    pl->cluster = 1;
    pl->threads = 1024;
    if ((size_t)nc * 8 <= std::min<size_t>(optin, CH_PRIVATE_SMEM_MAX) && nr <= 65536) {
        pl->mode = 0;  // private copies (rows packed in 16 bits for the merge)
        pl->smem = (size_t)nc * 8;
        // at least ~16K points per CTA so a private copy pays for its merge
        const int64_t want = std::max<int64_t>(1, (npairs + 8191) / 8192);
        const int bps = private_bps(dev, pl->smem);
        if (bps < 0)
            return CH_ERR_CUDA;
        pl->grid = (int)std::min<int64_t>(want, (int64_t)std::max(1, std::min(bps, 1)) * sms);
        pl->copies = pl->grid;
    } else {
        pl->mode = (size_t)nc * 2 <= std::min<size_t>(optin, CH_FILTER_SMEM_MAX) ? 1 : 2;  // filtered / read-then-atomic
        pl->smem = pl->mode == 1 ? (((size_t)nc * 2 + 15) & ~size_t(15)) : 0;
        pl->grid = sms;
        pl->copies = 0;
        pl->shift = filter_shift(nr);
        if (pl->mode == 1)
            pl->cluster = warm_cluster(dev, pl->smem, pl->grid);
    }
    return CH_OK;
}

int reduce_filter_shift(int p) { return filter_shift(p); }

int reduce_kernel_count(const ReducePlan &pl)
{
    return pl.mode == 0 ? 1 : (pl.mode == 1 ? 3 : 2);
}

size_t reduce_partials_bytes(const ReducePlan &pl, int nc)
{
    if (pl.mode == 0)
        return (size_t)pl.copies * (size_t)nc * 4;
    if (pl.mode == 1)  // merged filter G, then one slot row per CTA
        return (((size_t)nc * 2 + 255) & ~size_t(255)) + (size_t)pl.grid * (((size_t)nc + 7) / 8) * 16;
    return 0;
}

namespace {

template <int FM>
void launch_warm(const ReducePlan &pl, const int32_t *pts, int64_t n, const Frame &f, void *part,
                 int2 *L2, cudaStream_t s, unsigned long long *zero, int nzero)
{
    uint16_t *G = reinterpret_cast<uint16_t *>(part);
    uint16_t *slots = reinterpret_cast<uint16_t *>(reinterpret_cast<char *>(part) +
                                                   ((((size_t)f.nc * 2) + 255) & ~size_t(255)));
    if (pl.cluster > 1)
        launch_cluster(k_filter_warm<1024, FM>, pl.grid, 1024, pl.smem, s, pl.cluster, pts, n, f,
                       pl.shift, pl.grid, slots);
    else
        launch(k_filter_warm<1024, FM>, pl.grid, 1024, pl.smem, s, pts, n, f, pl.shift, pl.grid,
               slots);
    const int words = (f.nc + 7) / 8;
    launch(k_filter_merge, (words + MG_V - 1) / MG_V, MG_V * MG_GROUPS, 0, s, slots,
           pl.grid / pl.cluster, f.nc, f.nr, G, L2, zero, nzero);
}

template <int FM>
void launch_main(const ReducePlan &pl, const int32_t *pts, int64_t n, const Frame &f, void *part,
                 int2 *L2, unsigned *status, cudaStream_t s)
{
    if (pl.mode == 0)
        launch(k_reduce_private<1024, FM>, pl.grid, 1024, pl.smem, s, pts, n, f,
               reinterpret_cast<uint32_t *>(part), status);
    else if (pl.mode == 2)
        launch(k_reduce_global<FM>, sm_count() * 8, 256, 0, s, pts, n, f, L2, status);
    else
        launch(k_reduce_filtered<1024, FM>, pl.grid, 1024, pl.smem, s, pts, n, f, pl.shift,
               reinterpret_cast<const uint16_t *>(part), L2, status);
}

void launch_fill(const Frame &f, int2 *L2, cudaStream_t s, unsigned long long *zero, int nzero)
{
    launch(k_fill_empty, std::max(1, std::min((f.nc + 255) / 256, sm_count() * 4)), 256, 0, s, L2,
           f.nc, f.nr, zero, nzero);
}

}  // namespace

cudaError_t reduce_launch(const ReducePlan &pl, const int32_t *pts, int64_t n, const Frame &f,
                          void *part, int32_t *L, unsigned *status, cudaStream_t s,
                          unsigned long long *zero, int nzero, cudaEvent_t ev0, cudaEvent_t ev1,
                          bool prefilled)
{
    auto mark = [&](cudaEvent_t ev) { return ev ? cudaEventRecord(ev, s) : cudaSuccess; };
    int2 *L2 = reinterpret_cast<int2 *>(L);
    if (!prefilled && pl.mode == 2)
        launch_fill(f, L2, s, zero, nzero);
    const int fm = frame_mode(f);
    if (!prefilled && pl.mode == 1)
        (fm == 0   ? launch_warm<0>
         : fm == 1 ? launch_warm<1>
         : fm == 2 ? launch_warm<2>
                   : launch_warm<3>)(pl, pts, n, f, part, L2, s, zero, nzero);
    mark(ev0);
    (fm == 0   ? launch_main<0>
     : fm == 1 ? launch_main<1>
     : fm == 2 ? launch_main<2>
               : launch_main<3>)(pl, pts, n, f, part, L2, status, s);
    mark(ev1);
    return cudaGetLastError();
}

cudaError_t reduce_warm_launch(const ReducePlan &pl, const int32_t *pts, int64_t n, const Frame &f,
                               void *part, int32_t *L, cudaStream_t s, unsigned long long *zero,
                               int nzero)
{
    int2 *L2 = reinterpret_cast<int2 *>(L);
    if (pl.mode == 2)
        launch_fill(f, L2, s, zero, nzero);
    else if (pl.mode == 1) {
        const int fm = frame_mode(f);
        (fm == 0   ? launch_warm<0>
         : fm == 1 ? launch_warm<1>
         : fm == 2 ? launch_warm<2>
                   : launch_warm<3>)(pl, pts, n, f, part, L2, s, zero, nzero);
    }
    return cudaGetLastError();
}

cudaError_t reduce_merge_launch(const void *part, int copies, int nc, int nr, int32_t *L,
                                cudaStream_t s, unsigned long long *zero, int nzero,
                                const int32_t *Linit)
{
    launch(k_merge_partials, (nc + 31) / 32, 1024, 0, s, reinterpret_cast<const uint32_t *>(part),
           copies, nc, nr, reinterpret_cast<int2 *>(L), zero, nzero,
           reinterpret_cast<const int2 *>(Linit));
    return cudaGetLastError();
}

}  // namespace ch
