// The sparse regime p > n (Section 4, "Extraction using a tree structure"
// and "For all practical purposes"): the bit array M grows into a w-ary tree
// of 32-bit words, so that extraction visits only non-empty words and the
// whole path costs O(n) instead of O(p).
//
// Persistent part of the workspace (zero-filled once by the caller; every
// call that ends without an error leaves it zero-filled again):
//   Lz   int2[p]: column c holds (INT_MAX - ly, hy) once it has a point and
//        (0, 0) while empty, so the zero fill is the empty array and both
//        halves of Algorithm 1's update are atomic maxima;
//   M_0 .. M_{H-1}: level 0 has one bit per column (word c >> 5, bit c & 31,
//        the paper's block/bit indexing with w = 32); level k + 1 has one bit
//        per word of level k, set when that word is non-zero; the top level
//        is a single word.
//
// k_sparse_reduce  Algorithm 1 into Lz (a read first, then an atomic max only
//                  when it improves the entry) and the tree's insert: set the
//                  column's bit, and the parent's bit whenever a word goes
//                  from zero to non-zero.
// k_tree_expand    level k -> level k - 1, top down: the list of non-empty
//                  words of level k (increasing index) becomes the list of
//                  non-empty words of level k - 1, each word's set bits in
//                  increasing order (the positions the ctz walk of Table I
//                  visits, ranked by 32 lanes at once); a compaction with one
//                  look-back pass.  The words it read are cleared.
//                  Its leaf form takes the non-empty words of level 0 to
//                  the lower and upper chains in increasing x (Lemma 1),
//                  clearing Lz and level 0.
// The hull then runs on the chains as in the plain path, sized by min(p, n).
#include <climits>

#include "ch_internal.cuh"
#include "lookback.cuh"

namespace ch {
namespace {

constexpr int SP_RED_T = 512;     // threads per reduction block
constexpr unsigned FULL = 0xFFFFFFFFu;

__global__ void __launch_bounds__(SP_RED_T)
    k_sparse_reduce(const int4 *__restrict__ pts2, const int2 *__restrict__ head,
                    const int2 *__restrict__ tail, long long npairs, int p, int2 *Lz, TreeLevels t,
                    unsigned *status)
{
    pdl_wait();
    pdl_trigger();
    bool bad = false;
    auto put = [&](int x, int y) {
        if ((unsigned)(x - 1) >= (unsigned)p || (unsigned)(y - 1) >= (unsigned)p) {
            bad = true;
            return;
        }
        const int c = x - 1;
        const int2 e = Lz[c];
        const int A = INT_MAX - y;
        if (A > e.x)
            atomicMax(&Lz[c].x, A);
        if (y > e.y)
            atomicMax(&Lz[c].y, y);
        unsigned idx = (unsigned)c;
#pragma unroll
        for (int k = 0; k < TREE_MAX_LEVELS; ++k) {  // unrolled: t.M stays in registers
            if (k >= t.levels)
                break;
            const unsigned bit = 1u << (idx & 31);
            idx >>= 5;
            if (t.M[k][idx] & bit)
                break;
            if (atomicOr(&t.M[k][idx], bit) != 0)
                break;  // the word was non-empty: its ancestors are set
        }
    };
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < npairs; i += stride) {
        const int4 q = __ldcs(pts2 + i);
        put(q.x, q.y);
        put(q.z, q.w);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (head) {
            const int2 q = *head;
            put(q.x, q.y);
        }
        if (tail) {
            const int2 q = *tail;
            put(q.x, q.y);
        }
    }
    if (__any_sync(FULL, bad) && (threadIdx.x & 31) == 0)
        atomicOr(status, ST_RANGE);
}

// Block-wide exclusive scan of v over the 1024 threads (32 warps) of a CTA; returns the
// block total in *tot (all threads).
__device__ __forceinline__ int block_excl_scan(int v, int *s_w, int *tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o)
            incl += t;
    }
    if (lane == 31)
        s_w[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int x = s_w[lane];
        int inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, inc, o);
            if (lane >= o)
                inc += t;
        }
        s_w[lane] = inc - x;
        if (lane == 31)
            s_w[32] = inc;
    }
    __syncthreads();
    *tot = s_w[32];
    return s_w[w] + incl - v;
}

constexpr int XW = 8;             // list words per warp
constexpr int XT = 32 * XW;       // list words per tile (a CTA of 32 warps)

// LEAF = false: in = non-empty words of level k (top: the single word 0),
// out = non-empty words of level k - 1.  LEAF = true: in = non-empty words of
// level 0, out = the chains.  A warp takes XW consecutive words of the list;
// lane b speaks for bit b of each, so the children of a word are ranked by
// popc of the lower bits (the ctz walk of Table I, done by 32 lanes at once)
// and a leaf word's 32 entries of Lz are read and cleared as one coalesced
// 256-byte access.
// in_cap, out_cap: capacities of the two lists (out: of the chains for LEAF);
// child_limit: words of level k - 1 (LEAF: p).  With a workspace that was
// zero-filled as required none of them is ever reached; otherwise the
// excess is dropped and recorded as CH_ERR_CAPACITY instead of written.
template <bool LEAF>
__global__ void __launch_bounds__(1024)
    k_tree_expand(uint32_t *Mk, const int *__restrict__ in, const int *in_cnt, int top, int *out,
                  int *out_cnt, int2 *Lz, int2 *lower, int2 *upper, int *counts,
                  unsigned long long *state, int in_cap, int out_cap, int child_limit,
                  unsigned *status)
{
    pdl_wait();
    pdl_trigger();
    __shared__ int s_tile;
    __shared__ int s_w[33];
    __shared__ long long s_prefix;
    if (threadIdx.x == 0)
        s_tile = (int)atomicAdd(state, 1ull);
    __syncthreads();
    const int tile = s_tile;
    const int cnt = top ? 1 : min(*in_cnt, in_cap);
    const int ntiles = (cnt + XT - 1) / XT;
    if (tile >= max(ntiles, 1))
        return;  // a later ticket: nothing waits on it
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int w0 = tile * XT + warp * XW;  // this warp's first list position
    int my_idx = -1;
    uint32_t my_word = 0;
    if (lane < XW && w0 + lane < cnt) {
        my_idx = top ? 0 : in[w0 + lane];
        my_word = Mk[my_idx];
    }
    int idx[XW];
    uint32_t word[XW];
    int wtot = 0;
#pragma unroll
    for (int k = 0; k < XW; ++k) {
        idx[k] = __shfl_sync(FULL, my_idx, k);
        word[k] = __shfl_sync(FULL, my_word, k);
        wtot += __popc(word[k]);
    }
    int2 e[XW];
    if constexpr (LEAF) {
#pragma unroll
        for (int k = 0; k < XW; ++k) {
            const int child = idx[k] * 32 + lane;
            e[k] = make_int2(0, 0);
            if (((word[k] >> lane) & 1u) && child < child_limit)
                e[k] = Lz[child];
        }
    }
    int tot;
    const int wexcl = block_excl_scan(lane == 0 ? wtot : 0, s_w, &tot);
    const int woff = __shfl_sync(FULL, wexcl, 0);
    if (threadIdx.x == 0)
        publish_aggregate(state + 1, tile, tot);
    if (threadIdx.x < 32) {
        const long long pre = warp_look_back(state + 1, tile, tot, threadIdx.x, status);
        if (threadIdx.x == 0) {
            s_prefix = pre;
            if (tile == max(ntiles, 1) - 1) {
                const int total = (int)min(pre + tot, (long long)out_cap);
                if (pre + tot > out_cap)
                    atomicOr(status, ST_CAPACITY);
                if (LEAF) {
                    counts[0] = total;
                    counts[1] = total;
                } else {
                    *out_cnt = total;
                }
            }
        }
    }
    __syncthreads();
    // the clears come after the look-back: a release or acquire of the
    // look-back waits for this thread's earlier stores, which would put their
    // latency on the path between consecutive tiles
    if (my_idx >= 0)
        Mk[my_idx] = 0;
    long long run = s_prefix + woff;
    const unsigned below = (1u << lane) - 1u;
    bool over = false;
#pragma unroll
    for (int k = 0; k < XW; ++k) {
        if ((word[k] >> lane) & 1u) {
            const long long pos = run + __popc(word[k] & below);
            const int child = idx[k] * 32 + lane;
            if (pos >= out_cap || child >= child_limit) {
                over = true;
            } else if (LEAF) {
                lower[pos] = make_int2(child + 1, INT_MAX - e[k].x);
                upper[pos] = make_int2(child + 1, e[k].y);
                Lz[child] = make_int2(0, 0);
            } else {
                out[pos] = child;
            }
        }
        run += __popc(word[k]);
    }
    if (__any_sync(FULL, over) && lane == 0)
        atomicOr(status, ST_CAPACITY);
}

}  // namespace

int tree_levels(int p, size_t *words)
{
    int H = 0;
    long long n = p;
    do {
        n = (n + 31) / 32;
        if (words)
            words[H] = (size_t)n;
        ++H;
    } while (n > 1);
    return H;
}

SparseLayout sparse_layout(int64_t n, int p)
{
    SparseLayout L;
    size_t words[TREE_MAX_LEVELS];
    L.levels = tree_levels(p, words);
    const long long cap_chain = std::max<long long>(1, std::min<long long>(p, n));
    L.chain_cap = (int)cap_chain;
    WsLayout w;
    // persistent, zero-filled
    L.Lz = w.take((size_t)p * 8);
    for (int k = 0; k < L.levels; ++k) {
        L.M[k] = w.take(words[k] * 4);
        L.words[k] = words[k];
    }
    L.persistent_end = w.off;
    // per call
    size_t lmax = 1;
    for (int k = 0; k < L.levels; ++k) {
        L.list_cap[k] = (size_t)std::max<long long>(1, std::min<long long>((long long)words[k], n));
        lmax = std::max(lmax, L.list_cap[k]);
    }
    L.list[0] = w.take(lmax * 4);
    L.list[1] = w.take(lmax * 4);
    L.cnt = w.take(2 * 4 + 8);
    L.state_words = 0;
    for (int k = 0; k < L.levels; ++k) {
        L.state_off[k] = L.state_words;
        // tiles of the expansion from level k (its input list)
        L.state_words += (int)((L.list_cap[k] + XT - 1) / XT) + 1;
    }
    L.state = w.take((size_t)L.state_words * 8);
    L.lower = w.take((size_t)cap_chain * 8);
    L.upper = w.take((size_t)cap_chain * 8);
    L.counts = w.take(8);
    L.hull = w.take(hull_ws_bytes((int)cap_chain));
    L.end = w.off;
    return L;
}

cudaError_t sparse_launch(const SparseLayout &L, const int32_t *pts, int64_t n, int p, void *ws,
                          int32_t *lower, int32_t *upper, int32_t *counts, int32_t *hull,
                          int32_t *hull_count, unsigned *status, cudaStream_t s, cudaEvent_t ev0,
                          cudaEvent_t ev1)
{
    char *b = reinterpret_cast<char *>(ws);
    cudaError_t e = cudaMemsetAsync(b + L.state, 0, (size_t)L.state_words * 8, s);
    if (e != cudaSuccess)
        return e;
    TreeLevels t = {};
    t.levels = L.levels;
    for (int k = 0; k < L.levels; ++k)
        t.M[k] = reinterpret_cast<uint32_t *>(b + L.M[k]);
    int2 *Lz = reinterpret_cast<int2 *>(b + L.Lz);
    // int4 loads of point pairs need 16-byte alignment: an 8-byte aligned
    // array starts with one point taken alone
    const int2 *p2 = reinterpret_cast<const int2 *>(pts);
    const int head = (n > 0 && ((uintptr_t)pts & 15)) ? 1 : 0;
    const long long npairs = (n - head) / 2;
    const int has_tail = (int)((n - head) & 1);
    const int blocks = (int)std::max<long long>(
        1, std::min<long long>((npairs + SP_RED_T - 1) / SP_RED_T, (long long)sm_count() * 4));
    if (ev0)
        cudaEventRecord(ev0, s);
    launch(k_sparse_reduce, blocks, SP_RED_T, 0, s, reinterpret_cast<const int4 *>(p2 + head),
           head ? p2 : nullptr, has_tail ? p2 + (n - 1) : nullptr, npairs, p, Lz, t, status);
    if (ev1)
        cudaEventRecord(ev1, s);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    int *list[2] = {reinterpret_cast<int *>(b + L.list[0]), reinterpret_cast<int *>(b + L.list[1])};
    int *cnt = reinterpret_cast<int *>(b + L.cnt);
    auto *st = reinterpret_cast<unsigned long long *>(b + L.state);
    // top level: its single word; then down to level 1
    int cur = 0;
    for (int k = L.levels - 1; k >= 1; --k) {
        const bool top = k == L.levels - 1;
        const int grid = (int)((L.list_cap[k] + XT - 1) / XT);
        launch(k_tree_expand<false>, std::max(grid, 1), 1024, 0, s, t.M[k], list[cur], cnt + cur,
               (int)top, list[cur ^ 1], cnt + (cur ^ 1), Lz, nullptr, nullptr, nullptr,
               st + L.state_off[k], (int)L.list_cap[k], (int)L.list_cap[k - 1],
               (int)L.words[k - 1], status);
        if ((e = cudaGetLastError()) != cudaSuccess)
            return e;
        cur ^= 1;
    }
    const int grid0 = (int)((L.list_cap[0] + XT - 1) / XT);
    launch(k_tree_expand<true>, std::max(grid0, 1), 1024, 0, s, t.M[0], list[cur], cnt + cur,
           (int)(L.levels == 1), nullptr, nullptr, Lz, reinterpret_cast<int2 *>(lower),
           reinterpret_cast<int2 *>(upper), counts, st + L.state_off[0], (int)L.list_cap[0],
           L.chain_cap, p, status);
    if ((e = cudaGetLastError()) != cudaSuccess)
        return e;
    return hull_launch(lower, upper, counts, L.chain_cap, hull, hull_count, b + L.hull, status, s);
}

// the reduction, one expansion per level, the hull filter and final CTA (and
// the second filter pass for long chains)
int sparse_kernel_count(const SparseLayout &L)
{
    return 1 + L.levels + 2 + (hull_layout(L.chain_cap).refilter ? 2 : 0);
}

}  // namespace ch
