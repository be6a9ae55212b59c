// Step 2: the valid columns of L as x-ordered lower and upper chains
// (Lemma 1, Section 2.1), via the bit array M of Section 4.
//
// Each warp's __ballot_sync over 32 consecutive columns is exactly one 32-bit
// word of M (column i at bit (i-1) & 31 of word (i-1) >> 5, the paper's
// block/bit indexing with w = 32).  Where the paper walks set bits with ctz,
// the GPU ranks them: a column's output slot is the number of valid columns
// before it, popc of the lower bits of its word plus an exclusive scan over
// words.  The scan runs in one pass over 1024-column tiles of L: each tile
// publishes its count and looks back at its predecessors' (decoupled
// look-back), with tiles handed out in launch order by an atomic ticket so
// that every tile it waits on is already running; every wait is bounded.
//
// The fused form used by the whole path also runs the exact hull pre-filter
// (hull_filter.cuh) on the tile's own stretch of both chains while it is in
// shared memory, and writes the survivors of each tile for the final hull.
#include <type_traits>

#include "ch_internal.cuh"
#include "hull_filter.cuh"
#include "lookback.cuh"

namespace ch {
namespace {

constexpr int TILE = RUN;         // columns per tile (one per thread)
constexpr int WPB = TILE / 32;    // words of M per tile

struct FilterSmem {
    int2 P[2][TILE];     // the tile's stretch of the lower chain and mirrored upper chain
    short M[2][2 * TILE];
};

// CULL: the chains of a culled reduction (L started from a culling start
// array Linit): column c has a lower point when L[c].lo < Linit[c].lo and an
// upper point when L[c].hi > Linit[c].hi, so the two chains are ranked
// separately; the look-back then carries both counts in one word
// ((lower << 31) | upper, no carry since each total is below 2^31).  Without
// culling Linit is (p+1, -1) everywhere and both tests reduce to "column
// non-empty".
constexpr int CNT_SHIFT = 31;
constexpr int SPARSE_TILE = 64;  // tiles with at most this many points per chain skip the pre-filter
constexpr long long CNT_LOW = (1ll << CNT_SHIFT) - 1;

// CHAINS = false (with FILTER): only the pre-filter's survivors are wanted
// (the hull path when the caller asks for no chain outputs), so the tile
// skips the look-back and the chain writes.  NARROW: 32-bit orientation tests
// in the pre-filter (sides and rows of at most 16384), and without culling
// both chains' keep tests interleaved (run_keeps_pair).
template <bool FILTER, bool CULL, bool CHAINS = true, bool NARROW = false>
__global__ void __launch_bounds__(TILE)
    k_chain(const int2 *__restrict__ L, const int2 *__restrict__ Linit, int p, int nr, int2 *lower,
            int2 *upper, int *counts, uint32_t *mask, unsigned long long *state, int ntiles,
            int2 *cand, int *ccnt, unsigned *status)
{
    pdl_wait();
    pdl_trigger();
    __shared__ int s_tile, s_cnt0, s_cnt1;
    __shared__ int s_wc[2][WPB + 1];
    __shared__ long long s_prefix;
    __shared__ typename std::conditional<FILTER, FilterSmem, int>::type fs;
    if (threadIdx.x == 0)
        s_tile = (int)atomicAdd(state, 1ull);
    __syncthreads();
    const int tile = s_tile;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = tile * TILE + threadIdx.x;  // 0-based column
    const int2 e = c < p ? L[c] : make_int2(nr + 1, -1);
    bool v0, v1;
    if constexpr (CULL) {
        const int2 li = c < p ? Linit[c] : make_int2(nr + 1, -1);
        v0 = c < p && e.x < li.x;
        v1 = c < p && e.y > li.y;
    } else {
        v0 = v1 = c < p && !(e.x == nr + 1 && e.y == -1);
    }
    const unsigned bal0 = __ballot_sync(0xFFFFFFFFu, v0);
    const unsigned bal1 = CULL ? __ballot_sync(0xFFFFFFFFu, v1) : bal0;
    if (lane == 0) {
        s_wc[0][w] = __popc(bal0);
        if (CULL)
            s_wc[1][w] = __popc(bal1);
        if (mask && c < p)
            mask[c >> 5] = bal0;
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int ch = 0; ch < (CULL ? 2 : 1); ++ch) {
            const int v = s_wc[ch][lane];
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o)
                    incl += t;
            }
            s_wc[ch][lane] = incl - v;
            if (lane == 31)
                (ch == 0 ? s_cnt0 : s_cnt1) = incl;
        }
        if (lane == 31) {
            const long long agg = CULL ? ((long long)s_cnt0 << CNT_SHIFT) | s_cnt1 : s_cnt0;
            publish_aggregate(state + 1, tile, agg);  // early: successors need only this
        }
    }
    __syncthreads();
    const int cnt0 = s_cnt0, cnt1 = CULL ? s_cnt1 : cnt0;
    const unsigned below = (1u << lane) - 1u;
    const int r0 = s_wc[0][w] + __popc(bal0 & below);  // ranks within the tile
    const int r1 = CULL ? s_wc[1][w] + __popc(bal1 & below) : r0;
    if constexpr (FILTER) {
        // the hull pre-filter needs no global position: run it before waiting
        if (cnt0 <= SPARSE_TILE && cnt1 <= SPARSE_TILE) {
            // few points (a culled chain): all of them are candidates, the
            // final merge copes, and the tile skips the trees
            if (v0)
                cand[(size_t)tile * TILE + r0] = make_int2(c + 1, e.x);
            if (v1)
                cand[((size_t)ntiles + tile) * TILE + r1] = make_int2(c + 1, -e.y);
            if (threadIdx.x == 0) {
                ccnt[tile] = cnt0;
                ccnt[ntiles + tile] = cnt1;
            }
        } else {
            if (v0)
                fs.P[0][r0] = make_int2(c + 1, e.x);
            if (v1)
                fs.P[1][r1] = make_int2(c + 1, -e.y);
            __syncthreads();
            build_min_trees(fs.P[0], fs.M[0], cnt0, fs.P[1], fs.M[1], cnt1);
            bool k0, k1;
            if constexpr (NARROW && !CULL) {
                run_keeps_pair<true>(fs.P[0], fs.M[0], fs.P[1], fs.M[1], cnt0, threadIdx.x, k0, k1);
            } else {
                k0 = run_keeps<false, NARROW>(fs.P[0], fs.M[0], cnt0, threadIdx.x);
                k1 = run_keeps<false, NARROW>(fs.P[1], fs.M[1], cnt1, threadIdx.x);
            }
            __shared__ int s_cw[WPB + 1];
            const int2 nk = compact_runs<false>(fs.P[0], k0, cand + (size_t)tile * TILE, fs.P[1], k1,
                                         cand + ((size_t)ntiles + tile) * TILE, s_cw);
            if (threadIdx.x == 0) {
                ccnt[tile] = nk.x;
                ccnt[ntiles + tile] = nk.y;
            }
        }
    }
    if constexpr (FILTER && !CHAINS)
        return;
    if (w == 0) {
        const long long agg = CULL ? ((long long)cnt0 << CNT_SHIFT) | cnt1 : cnt0;
        const long long pre = warp_look_back(state + 1, tile, agg, lane, status);
        if (lane == 0) {
            s_prefix = pre;
            if (tile == ntiles - 1) {
                const long long tot = pre + agg;
                counts[0] = (int)(CULL ? tot >> CNT_SHIFT : tot);
                counts[1] = (int)(CULL ? tot & CNT_LOW : tot);
            }
        }
    }
    __syncthreads();
    const long long pre0 = CULL ? s_prefix >> CNT_SHIFT : s_prefix;
    const long long pre1 = CULL ? s_prefix & CNT_LOW : s_prefix;
    if (v0)
        lower[pre0 + r0] = make_int2(c + 1, e.x);
    if (v1)
        upper[pre1 + r1] = make_int2(c + 1, e.y);
}

}  // namespace

int chain_tiles(int p) { return (p + TILE - 1) / TILE; }

size_t chain_state_bytes(int p) { return (size_t)(chain_tiles(p) + 1) * 8; }

cudaError_t chain_launch(const int32_t *L, int p, int32_t *lower, int32_t *upper, int32_t *counts,
                         uint32_t *mask, void *state, bool state_zeroed, int2 *cand, int *ccnt,
                         unsigned *status, cudaStream_t s, const int32_t *Linit, int nr)
{
    if (nr <= 0)
        nr = p;
    const int nt = chain_tiles(p);
    if (!state_zeroed) {
        cudaError_t e = cudaMemsetAsync(state, 0, chain_state_bytes(p), s);
        if (e != cudaSuccess)
            return e;
    }
    auto *st = reinterpret_cast<unsigned long long *>(state);
    const int2 *L2 = reinterpret_cast<const int2 *>(L), *Li = reinterpret_cast<const int2 *>(Linit);
    int2 *lo = reinterpret_cast<int2 *>(lower), *up = reinterpret_cast<int2 *>(upper);
    const bool narrow = p <= 16384 && nr <= 16384;
    const bool chains = lower || upper || counts || mask;
    if (cand && Linit)
        launch(chains ? (narrow ? k_chain<true, true, true, true> : k_chain<true, true>)
                      : (narrow ? k_chain<true, true, false, true> : k_chain<true, true, false>),
               nt, TILE, 0, s, L2, Li, p, nr, lo, up, counts, mask, st, nt, cand, ccnt, status);
    else if (cand)
        launch(chains ? (narrow ? k_chain<true, false, true, true> : k_chain<true, false>)
                      : (narrow ? k_chain<true, false, false, true> : k_chain<true, false, false>),
               nt, TILE, 0, s, L2, nullptr, p, nr, lo, up, counts, mask, st, nt, cand, ccnt, status);
    else if (Linit)
        launch(k_chain<false, true>, nt, TILE, 0, s, L2, Li, p, nr, lo, up, counts, mask, st, nt, nullptr,
                                                 nullptr, status);
    else
        launch(k_chain<false, false>, nt, TILE, 0, s, L2, nullptr, p, nr, lo, up, counts, mask, st, nt,
                                                  nullptr, nullptr, status);
    return cudaGetLastError();
}

}  // namespace ch
