// Lemma 1's polyline (Section 2.1) and Melkman's hull of a simple polyline,
// the linear hull algorithm the paper runs directly on its reduced set
// (Section 3, Fig. 10).
//
// k_polyline  the valid columns of L in increasing x, each as (x, ly) and
//             then (x, hy) when the two differ: a compaction with weights
//             0, 1 or 2 per column in one pass over 1024-column tiles
//             (decoupled look-back).  Joining consecutive vertices gives the
//             simple chain of Lemma 1.  The filtered form drops, tile by
//             tile, the vertices the exact pre-filter of the hull step rules
//             out, which leaves a shorter simple polyline for Melkman.
// k_melkman   one warp runs Melkman's algorithm.  A deque holds the hull of
//             the vertices seen so far, counter-clockwise from its bottom to
//             its top, with the newest vertex at both ends; only the two
//             entries at each end take part in the tests, so they live in
//             registers and the deque itself in shared memory (global memory
//             when the hull can outgrow it).  The vertex stream is staged in
//             shared memory 1024 at a time.  The next vertex is tested on
//             its own; after one that is inside, the 32 lanes test the next
//             32 vertices against the current hull at once (a skipped vertex
//             leaves the hull unchanged, so every test of the batch up to the
//             first vertex outside is the sequential test).  The update for
//             a vertex outside is sequential, executed by all lanes alike.
//             Skipping on "left of or on" and popping on "not strictly left"
//             drop collinear points: the hull lists strict vertices,
//             counter-clockwise from the lexicographic minimum.
#include <climits>
#include <type_traits>

#include "ch_internal.cuh"
#include "hull_filter.cuh"
#include "lookback.cuh"

namespace ch {
namespace {

constexpr int PL_TILE = 1024;
constexpr unsigned FULL = 0xFFFFFFFFu;

struct PolyFilterSmem {
    int2 P[2][PL_TILE];  // the tile's lower chain and mirrored upper chain
    short M[2][2 * PL_TILE];
};

// FILTER: a column's ly (hy) vertex is kept only when the exact in-tile
// pre-filter of hull_filter.cuh keeps it on the tile's lower (upper) chain;
// a column with ly == hy keeps its one vertex when either chain keeps it.
// The result is the Lemma 1 polyline of a sub-array of L (each column
// holding a subset of its two points), so it is still simple, and it keeps
// every hull vertex.
template <bool FILTER>
__global__ void __launch_bounds__(PL_TILE)
    k_polyline(const int2 *__restrict__ L, int p, int nr, int2 *poly, int *count,
               unsigned long long *state, int ntiles, unsigned *status)
{
    pdl_wait();
    pdl_trigger();
    __shared__ int s_tile, s_tot;
    __shared__ int s_wsum[PL_TILE / 32 + 1];
    __shared__ long long s_prefix;
    __shared__ typename std::conditional<FILTER, PolyFilterSmem, int>::type fs;
    if (threadIdx.x == 0)
        s_tile = (int)atomicAdd(state, 1ull);
    __syncthreads();
    const int tile = s_tile;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int c = tile * PL_TILE + threadIdx.x;  // 0-based column
    int2 e = c < p ? L[c] : make_int2(nr + 1, -1);
    bool valid = c < p && !(e.x == nr + 1 && e.y == -1);
    int wt;
    bool emit_lo = valid, emit_hi = valid && e.x != e.y;
    if constexpr (FILTER) {
        // rank the valid columns, filter their two chains in shared memory;
        // from here on thread r speaks for the tile's r-th valid column
        const unsigned bal = __ballot_sync(FULL, valid);
        if (lane == 0)
            s_wsum[w] = __popc(bal);
        __syncthreads();
        if (w == 0) {
            const int v = s_wsum[lane];
            int inc = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(FULL, inc, o);
                if (lane >= o)
                    inc += t;
            }
            s_wsum[lane] = inc - v;
            if (lane == 31)
                s_wsum[PL_TILE / 32] = inc;
        }
        __syncthreads();
        const int cnt = s_wsum[PL_TILE / 32];
        if (valid) {
            const int r = s_wsum[w] + __popc(bal & ((1u << lane) - 1u));
            fs.P[0][r] = make_int2(c + 1, e.x);
            fs.P[1][r] = make_int2(c + 1, -e.y);
        }
        __syncthreads();
        build_min_trees(fs.P[0], fs.M[0], cnt, fs.P[1], fs.M[1], cnt);
        const bool k0 = run_keeps(fs.P[0], fs.M[0], cnt, threadIdx.x);
        const bool k1 = run_keeps(fs.P[1], fs.M[1], cnt, threadIdx.x);
        valid = (int)threadIdx.x < cnt;
        if (valid) {
            c = fs.P[0][threadIdx.x].x - 1;
            e = make_int2(fs.P[0][threadIdx.x].y, -fs.P[1][threadIdx.x].y);
        }
        emit_lo = valid && (e.x != e.y ? k0 : (k0 || k1));
        emit_hi = valid && e.x != e.y && k1;
        __syncthreads();  // s_wsum is reused below
    }
    wt = (int)emit_lo + (int)emit_hi;
    int incl = wt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o)
            incl += t;
    }
    if (lane == 31)
        s_wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int v = s_wsum[lane];
        int inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, inc, o);
            if (lane >= o)
                inc += t;
        }
        s_wsum[lane] = inc - v;
        if (lane == 31) {
            s_tot = inc;
            publish_aggregate(state + 1, tile, inc);
        }
    }
    __syncthreads();
    const int agg = s_tot;
    const int excl = s_wsum[w] + incl - wt;
    if (w == 0) {
        const long long pre = warp_look_back(state + 1, tile, agg, lane, status);
        if (lane == 0) {
            s_prefix = pre;
            if (tile == ntiles - 1)
                *count = (int)(pre + agg);
        }
    }
    __syncthreads();
    long long pos = s_prefix + excl;
    if (emit_lo)
        poly[pos++] = make_int2(c + 1, e.x);
    if (emit_hi)
        poly[pos] = make_int2(c + 1, e.y);
}

constexpr int MK_STAGE = 1024;  // polyline vertices staged per round

__device__ __forceinline__ bool lex_less(int2 a, int2 b)
{
    return a.x < b.x || (a.x == b.x && a.y < b.y);
}

// Key whose unsigned order is the lexicographic order of (x, y).
__device__ __forceinline__ unsigned long long lex_key(int2 q)
{
    return ((unsigned long long)((unsigned)q.x ^ 0x80000000u) << 32) |
           (unsigned long long)((unsigned)q.y ^ 0x80000000u);
}

// Orientation of (o, a, b) in 32-bit arithmetic when every coordinate lies
// in [1, 2^15]: each product is below 2^30 in magnitude and their difference
// below 2^31, so the sign is exact; else in 64-bit arithmetic.
template <bool SMALL>
__device__ __forceinline__ long long orient(int2 o, int2 a, int2 b)
{
    if constexpr (SMALL)
        return (a.x - o.x) * (b.y - o.y) - (a.y - o.y) * (b.x - o.x);
    else
        return cross3(o, a, b);
}

// poly: *count vertices of a simple polyline, distinct, in [1, p]^2.
// GDQ: the deque is dq_global (it does not fit in shared memory), else it
// follows the staging buffer in shared memory; dq_cap: its capacity (a power
// of two above the largest hull plus one).
template <bool GDQ, bool SMALL>
__global__ void __launch_bounds__(32)
    k_melkman(const int2 *__restrict__ poly, const int *count, int p, int2 *dq_global,
              unsigned dq_cap, int2 *hull, int *hull_count, unsigned *status)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ int2 sm[];
    int2 *stage = sm;
    int2 *dq = GDQ ? dq_global : sm + MK_STAGE;
    const unsigned mask = dq_cap - 1;
    const int lane = threadIdx.x;
    const int m = *count;
    int phase = 0;                 // 0: collinear prefix, 1: deque running
    int k = 0;                     // vertices of the collinear prefix
    int2 a = make_int2(0, 0), b = a;  // its lexicographic extremes
    int top = 0, bot = 0;          // deque ends, taken modulo dq_cap
    int2 t1 = a, t0 = a, b0 = a, b1 = a;  // D[top-1], D[top], D[bot], D[bot+1]
    bool bad = false;
    for (int base = 0; base < m && !bad; base += MK_STAGE) {
        const int cnt = min(MK_STAGE, m - base);
        __syncwarp();
        bool oob = false;
        for (int i = lane; i < cnt; i += 32) {
            const int2 v = poly[base + i];
            oob |= (unsigned)(v.x - 1) >= (unsigned)p || (unsigned)(v.y - 1) >= (unsigned)p;
            stage[i] = v;
        }
        if (__any_sync(FULL, oob)) {
            if (lane == 0)
                atomicOr(status, ST_RANGE);
            bad = true;
            break;
        }
        __syncwarp();
        int i = 0;
        if (phase == 0) {
            for (; i < cnt; ++i) {
                const int2 u = stage[i];
                if (k == 0) {
                    a = b = u;
                    k = 1;
                    continue;
                }
                const long long o = orient<SMALL>(a, b, u);
                if (k >= 2 && o != 0) {
                    // the first vertex off the prefix's line: the deque starts
                    // as the counter-clockwise triangle (u, a, b) or (u, b, a)
                    const int2 q1 = o > 0 ? a : b, q2 = o > 0 ? b : a;
                    dq[0] = u;
                    dq[1] = q1;
                    dq[2] = q2;
                    dq[3] = u;
                    bot = 0;
                    top = 3;
                    b0 = u;
                    b1 = q1;
                    t1 = q2;
                    t0 = u;
                    phase = 1;
                    ++i;
                    break;
                }
                if (lex_less(u, a))
                    a = u;
                if (lex_less(b, u))
                    b = u;
                ++k;
            }
        }
        if (phase == 1) {
            while (i < cnt) {
                // the next vertex alone first: on a polyline that keeps
                // leaving the hull (as Lemma 1's does) that is the common case
                int2 u = stage[i];
                if (orient<SMALL>(t1, t0, u) >= 0 && orient<SMALL>(b0, b1, u) >= 0) {
                    // inside: skip on, testing 32 vertices at a time
                    ++i;
                    bool found = false;
                    while (i < cnt) {
                        const int j = i + lane;
                        bool out = false;
                        if (j < cnt) {
                            const int2 v = stage[j];
                            out = !(orient<SMALL>(t1, t0, v) >= 0 && orient<SMALL>(b0, b1, v) >= 0);
                        }
                        const unsigned ob = __ballot_sync(FULL, out);
                        if (ob) {
                            i += __ffs(ob) - 1;
                            found = true;
                            break;
                        }
                        i += 32;
                    }
                    if (!found)
                        break;
                    u = stage[i];
                }
                ++i;
                // top: pop while u is not strictly left of the top edge
                while (top - bot > 1 && orient<SMALL>(t1, t0, u) <= 0) {
                    --top;
                    t0 = t1;
                    t1 = dq[(unsigned)(top - 1) & mask];
                }
                if (top + 1 - bot + 1 > (int)dq_cap) {
                    bad = true;
                    break;
                }
                ++top;
                dq[(unsigned)top & mask] = u;  // every lane stores the same value
                t1 = t0;
                t0 = u;
                // bottom: pop while (u, D[bot], D[bot+1]) is not a strict left turn
                while (top - bot > 1 && orient<SMALL>(u, b0, b1) <= 0) {
                    ++bot;
                    b0 = b1;
                    b1 = dq[(unsigned)(bot + 1) & mask];
                }
                if (top - (bot - 1) + 1 > (int)dq_cap) {
                    bad = true;
                    break;
                }
                --bot;
                dq[(unsigned)bot & mask] = u;
                b1 = b0;
                b0 = u;
            }
            if (bad && lane == 0)
                atomicOr(status, ST_CAPACITY);
        }
    }
    if (bad) {
        if (lane == 0)
            *hull_count = 0;
        return;
    }
    if (phase == 0) {  // no vertex, one, or all on one line: [min, max]
        if (lane == 0) {
            int h = 0;
            if (m > 0) {
                hull[0] = a;
                h = 1;
                if (a.x != b.x || a.y != b.y) {
                    hull[1] = b;
                    h = 2;
                }
            }
            *hull_count = h;
        }
        return;
    }
    // D[bot .. top-1] is the hull, counter-clockwise; start it at its
    // lexicographic minimum (the vertices are distinct).  A simple polyline
    // in [1, p]^2 has at most min(2p, m) hull vertices (two per column); a
    // longer list means the input was not simple and is not written.
    const int h = top - bot;
    if ((long long)h > min(2ll * p, (long long)m)) {
        if (lane == 0) {
            atomicOr(status, ST_CAPACITY);
            *hull_count = 0;
        }
        return;
    }
    unsigned long long best = ULLONG_MAX;
    for (int r = lane; r < h; r += 32)
        best = min(best, lex_key(dq[(unsigned)(bot + r) & mask]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        best = min(best, __shfl_xor_sync(FULL, best, o));
    int rs = INT_MAX;
    for (int r = lane; r < h; r += 32)
        if (lex_key(dq[(unsigned)(bot + r) & mask]) == best)
            rs = r;
    rs = __reduce_min_sync(FULL, rs);
    for (int r = lane; r < h; r += 32) {
        const int q = rs + r < h ? rs + r : rs + r - h;
        hull[r] = dq[(unsigned)(bot + q) & mask];
    }
    if (lane == 0)
        *hull_count = h;
}

constexpr size_t MK_SMEM_MAX_DQ = 16384;  // deque entries kept in shared memory at most

cudaError_t set_melkman_smem()
{
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64)
        return cudaErrorInvalidDevice;
    if (!done[dev]) {
        const int bytes = (int)((MK_STAGE + MK_SMEM_MAX_DQ) * sizeof(int2));
        cudaError_t e = cudaFuncSetAttribute(k_melkman<false, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_melkman<false, true>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess)
            return e;
        done[dev] = true;
    }
    return cudaSuccess;
}

}  // namespace

// Most vertices a strictly convex polygon with vertices in [1, p]^2 can
// have.  Its edge vectors are nonzero integer vectors of distinct directions
// whose L1 lengths add up to at most 4(p - 1), the L1 perimeter of the box;
// there are 4r integer vectors of L1 length r, so the count is largest when
// the shortest vectors are taken first.  At most 2 per column, so also 2p.
long long lattice_hull_bound(int p)
{
    long long budget = 4 * ((long long)p - 1), cnt = 0;
    for (long long r = 1; budget >= r; ++r) {
        const long long take = std::min(4 * r, budget / r);
        cnt += take;
        budget -= take * r;
    }
    return std::max(2ll, std::min(cnt, 2 * (long long)p));
}

// Deque capacity for side p: a power of two above the largest hull + 1.
size_t melkman_deque_cap(int p)
{
    const long long need = lattice_hull_bound(p) + 2;
    size_t cap = 1024;
    while ((long long)cap < need)
        cap <<= 1;
    return cap;
}

size_t melkman_ws_bytes(int p)
{
    const size_t cap = melkman_deque_cap(p);
    return cap <= MK_SMEM_MAX_DQ ? 0 : cap * sizeof(int2);
}

size_t polyline_state_bytes(int p) { return chain_state_bytes(p); }

cudaError_t polyline_launch(const int32_t *L, int p, int nr, int32_t *poly, int32_t *count,
                            void *state, bool state_zeroed, unsigned *status, cudaStream_t s,
                            bool filter)
{
    const int nt = (p + PL_TILE - 1) / PL_TILE;
    if (!state_zeroed) {
        const cudaError_t e = cudaMemsetAsync(state, 0, polyline_state_bytes(p), s);
        if (e != cudaSuccess)
            return e;
    }
    launch(filter ? k_polyline<true> : k_polyline<false>, nt, PL_TILE, 0, s,
           reinterpret_cast<const int2 *>(L), p, nr > 0 ? nr : p, reinterpret_cast<int2 *>(poly),
           count, reinterpret_cast<unsigned long long *>(state), nt, status);
    return cudaGetLastError();
}

cudaError_t melkman_launch(const int32_t *poly, const int32_t *count, int p, int32_t *hull,
                           int32_t *hull_count, void *ws, unsigned *status, cudaStream_t s)
{
    cudaError_t e = set_melkman_smem();
    if (e != cudaSuccess)
        return e;
    const size_t cap = melkman_deque_cap(p);
    const bool in_smem = cap <= MK_SMEM_MAX_DQ;
    const size_t smem = (MK_STAGE + (in_smem ? cap : 0)) * sizeof(int2);
    const bool small = p <= (1 << 15);
    launch(in_smem ? (small ? k_melkman<false, true> : k_melkman<false, false>)
                   : k_melkman<true, false>,
           1, 32, smem, s,
           reinterpret_cast<const int2 *>(poly), count, p,
           in_smem ? nullptr : reinterpret_cast<int2 *>(ws), (unsigned)cap,
           reinterpret_cast<int2 *>(hull), hull_count, status);
    return cudaGetLastError();
}

}  // namespace ch
