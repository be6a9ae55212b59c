// Many independent point sets in one persistent launch: Algorithm 1, the
// chains and the hull (Section 2.1) for each set.
//
// A host-side planner cuts every set into chunks (work items) and sorts the
// items longest first.  Persistent CTAs take items from an atomic queue.  For
// an item the CTA folds its chunk into a private L in shared memory with
// native shared atomicMin / atomicMax (int32 lo[p], hi[p]).  A set of one
// chunk is finished by that CTA at once; a set of several chunks has each
// chunk write its L as a packed partial row, and the CTA that completes the
// last chunk (per-set atomic ticket) merges the rows and finishes the set.
// Finishing scans L in 1024-column tiles: the valid columns of a tile with
// more than SPARSE_TILE of them go through the exact hull pre-filter
// (hull_filter.cuh), those of the other tiles are kept as they are, and both
// are appended to per-chain lists; the lists are then peeled, merged and
// stitched (hull_merge.cuh) straight into the set's slice of the ragged
// output.  L never leaves shared memory for one-chunk sets.
#include <algorithm>
#include <vector>

#include "ch_internal.cuh"
#include "hull_filter.cuh"
#include "hull_merge.cuh"

namespace ch {
namespace {

constexpr int BT = 1024;       // threads per CTA (= RUN, one column per thread in a tile)
constexpr int BPCAP = 2048;    // survivors (both chains) finished in shared memory (more: global
                               // scratch; a smaller region leaves more L1 for loads in flight)

struct BItem {
    long long start, end;  // global point range [start, end)
    int set, chunk;
};
struct BSet {
    long long part_off;  // first packed partial row (uint32 units), sets with nchunks > 1
    int nchunks, p;
};

// Dynamic shared memory: [L: 8 * BMAX_P][A: BPCAP int2][tile runs + trees].
// After the tiles the L region holds B (BPCAP int2), F (BPCAP int), ix.
constexpr size_t SM_L = 8 * (size_t)BATCH_MAX_P;
constexpr size_t SM_A = BPCAP * sizeof(int2);
constexpr size_t SM_RUNS = 2 * RUN * sizeof(int2) + 2 * 2 * RUN * sizeof(short);
constexpr size_t BATCH_SMEM = SM_L + SM_A + SM_RUNS;
static_assert(BPCAP * (sizeof(int2) + sizeof(int)) + 4 * (BPCAP / HS + 2) * sizeof(int) <= SM_L,
              "peel scratch fits the L region");

// Per-CTA global scratch (used when a set's survivors exceed BPCAP).
constexpr size_t SCR_PTS = 2 * (size_t)BATCH_MAX_P;  // points, both chains
constexpr size_t SCR_BYTES = 2 * SCR_PTS * sizeof(int2) + SCR_PTS * sizeof(int) +
                             4 * (SCR_PTS / HS + 2) * sizeof(int) + 256;

__device__ __forceinline__ void fold(int *slo, int *shi, uint32_t up, int x, int y, bool &bad)
{
    const uint32_t c = (uint32_t)(x - 1);
    if (c >= up || (uint32_t)(y - 1) >= up) {
        bad = true;
        return;
    }
    atomicMin(slo + c, y);
    atomicMax(shi + c, y);
}

// Folds points [0, n) of `base` (8-byte aligned) into slo/shi; a group of NT
// threads (tid: the thread's index in the group), by default the whole CTA.
template <int NT = BT>
__device__ void fold_range(const int32_t *__restrict__ base, int64_t n, int p, int *slo, int *shi,
                           bool &bad, int tid = threadIdx.x)
{
    const uint32_t up = (uint32_t)p;
    const int64_t head = (((uintptr_t)base & 15) != 0 && n > 0) ? 1 : 0;
    const int64_t npairs = (n - head) >> 1;
    if (tid == 0) {
        if (head)
            fold(slo, shi, up, base[0], base[1], bad);
        if ((n - head) & 1)
            fold(slo, shi, up, base[2 * (n - 1)], base[2 * (n - 1) + 1], bad);
    }
    const int4 *p4 = reinterpret_cast<const int4 *>(base + 2 * head);
    // U loads in flight per thread; the next U are issued before the current
    // ones are folded (register double buffering).  A work item holds at most
    // 2^22 points (and a small problem's slice fewer), so the vector indices
    // are 32-bit, which keeps the loop's tests and address sums single-word.
#ifndef CH_FOLD_U
#define CH_FOLD_U 5  // 10,000-set batch, 640/384 split: 4 2.257, 5 2.236 ms per replay; 6 spills
#endif
    constexpr int U = CH_FOLD_U;
    const int m = (int)npairs;
    int4 v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int j = tid + u * NT;
        v[u] = j < m ? __ldcs(p4 + j) : make_int4(0, 0, 0, 0);
    }
    for (int i = tid; i < m; i += NT * U) {
        int4 nx[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = i + (U + u) * NT;
            nx[u] = j < m ? __ldcs(p4 + j) : make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (i + u * NT < m) {
                fold(slo, shi, up, v[u].x, v[u].y, bad);
                fold(slo, shi, up, v[u].z, v[u].w, bad);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            v[u] = nx[u];
    }
}

// Tiles with at most this many valid columns skip the pre-filter: below it
// the peeling rounds remove their non-vertices for less than the trees cost.
// Swept on the 10,000-set batch with the split CTA (ms per replay): 64 2.625,
// 128 2.588, 192 2.574, 256 2.553, 384 2.568, 512 2.587, 768 2.704, 1024
// (no tile filtered) 3.996.
#ifndef CH_SPARSE_TILE
#define CH_SPARSE_TILE 256
#endif
constexpr int SPARSE_TILE = CH_SPARSE_TILE;

// What the tile pre-filter leaves of a set: the survivors at D, the lower
// chain in D[0..T0) and the mirrored upper chain in D[T0..T).
struct Survivors {
    int2 *D;
    int T0, T;
    bool in_smem;
};

// The tile phase of finishing a set (a whole CTA of RUN threads): the valid
// columns of L (slo/shi, p columns), 1024-column tile by tile, through the
// exact pre-filter (tiles with more than SPARSE_TILE valid columns) or kept
// as they are, appended to the per-CTA global lists in scr; then copied
// compactly to Ds when they fit `cap` points, else to the global scratch
// behind the lists.  runs: the tile buffers P0, P1 (RUN int2 each) and M0,
// M1 (2 RUN shorts each), contiguous.
__device__ Survivors collect_survivors(int p, const int *slo, const int *shi, unsigned char *runs,
                                       int2 *Ds, int cap, int2 *scr, int *s_warp, int *s_cnt)
{
    int2 *P0 = reinterpret_cast<int2 *>(runs);
    int2 *P1 = P0 + RUN;
    short *M0 = reinterpret_cast<short *>(P1 + RUN);
    short *M1 = M0 + 2 * RUN;
    // survivors are appended to the per-CTA global lists first (capacity p each)
    int2 *glo = scr, *gup = scr + BATCH_MAX_P;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int T0 = 0, T1 = 0;
    int *const s_warp2 = s_warp;
    for (int t0 = 0; t0 < p; t0 += RUN) {
        // consecutive tiles alternate between two scan buffers, so a tile
        // needs no closing barrier: every other shared value it reads is
        // rewritten only after the next tile's first two barriers
        s_warp = s_warp2 + ((t0 / RUN) & 1) * (RUN / 32 + 1);
        const int c = t0 + threadIdx.x;
        const bool valid = c < p && slo[c] <= shi[c];
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, valid);
        if (lane == 0)
            s_warp[w] = __popc(bal);
        __syncthreads();
        if (w == 0) {
            const int v = s_warp[lane];
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o)
                    incl += x;
            }
            s_warp[lane] = incl - v;
            if (lane == 31)
                *s_cnt = incl;
        }
        __syncthreads();
        const int cnt = *s_cnt;
        if (cnt <= SPARSE_TILE) {  // few columns: keep them all, the merge copes
            if (valid) {
                const int r = s_warp[w] + __popc(bal & ((1u << lane) - 1u));
                glo[T0 + r] = make_int2(c + 1, slo[c]);
                gup[T1 + r] = make_int2(c + 1, -shi[c]);
            }
            T0 += cnt;
            T1 += cnt;
            continue;
        }
        if (valid) {
            const int r = s_warp[w] + __popc(bal & ((1u << lane) - 1u));
            P0[r] = make_int2(c + 1, slo[c]);
            P1[r] = make_int2(c + 1, -shi[c]);
        }
        __syncthreads();
        build_min_trees(P0, M0, cnt, P1, M1, cnt);
        bool k0, k1;
        run_keeps_pair<true>(P0, M0, P1, M1, cnt, threadIdx.x, k0, k1);
        const int2 nk = compact_runs<false>(P0, k0, glo + T0, P1, k1, gup + T1, s_warp);
        T0 += nk.x;
        T1 += nk.y;
    }
    __syncthreads();  // the last tile's survivor lists are copied below by other threads
    const int T = T0 + T1;
    const bool in_smem = T <= cap;
    int2 *D = in_smem ? Ds : scr + 2 * BATCH_MAX_P;  // compact: lower then upper
    for (int k = threadIdx.x; k < T0; k += BT)
        D[k] = __ldcg(glo + k);
    for (int k = threadIdx.x; k < T1; k += BT)
        D[T0 + k] = __ldcg(gup + k);
    __syncthreads();
    return Survivors{D, T0, T, in_smem};
}

// Peel scratch in the per-CTA global scratch, for survivors beyond the
// shared-memory capacity: lists [0, 2P), D [2P, 4P), F, ix (P = BATCH_MAX_P).
__device__ __forceinline__ void global_peel_scratch(int2 *scr, int2 *&B, int *&F, int *&ix)
{
    B = scr;  // the survivor lists were copied to D already
    F = reinterpret_cast<int *>(scr + 4 * BATCH_MAX_P);
    ix = F + 2 * BATCH_MAX_P;
}

// Hull of the set whose L is in slo/shi (p columns); whole CTA.
// Layout of the shared memory a set is finished in: L at `smem` (which holds
// the peel scratch once the tiles are done: cap int2 + cap int + the merge
// tree's index arrays), the tile buffers at `runs`, up to `cap` survivors at
// Ds; more survivors peel in the CTA's global scratch.
__device__ void finish_set_at(int p, int *slo, int *shi, unsigned char *smem, unsigned char *runs,
                              int2 *Ds, int cap, int2 *scr, int2 *hull, int *hull_count,
                              int *s_warp, int *s_total, int *s_cnt)
{
    const Survivors sv = collect_survivors(p, slo, shi, runs, Ds, cap, scr, s_warp, s_cnt);
    int2 *B;
    int *F, *ix;
    if (sv.in_smem) {  // L is no longer needed: its region holds the peel scratch
        B = reinterpret_cast<int2 *>(smem);
        F = reinterpret_cast<int *>(B + cap);
        ix = F + cap;
    } else {
        global_peel_scratch(scr, B, F, ix);
    }
    peel_merge_stitch<FT, 0, true>(sv.D, B, F, ix, sv.T0, sv.T, hull, hull_count, s_warp, s_total);
}

// The batched kernels' layout: [L: SM_L][survivors: BPCAP int2][tile buffers].
__device__ void finish_set(int p, int *slo, int *shi, unsigned char *smem, int2 *scr,
                           int2 *hull, int *hull_count, int *s_warp, int *s_total, int *s_cnt)
{
    finish_set_at(p, slo, shi, smem, smem + SM_L + SM_A, reinterpret_cast<int2 *>(smem + SM_L),
                  BPCAP, scr, hull, hull_count, s_warp, s_total, s_cnt);
}

// k_small's layout, sized for its p: [L or peel scratch][survivors: SCAP
// int2][tile buffers].  Less shared memory leaves more of the SM to L1,
// which holds the folding threads' loads in flight.
constexpr int SCAP = 2048;
__host__ __device__ constexpr size_t small_lreg(int p)
{
    return ((8 * (size_t)p > (size_t)SCAP * 12 + 4 * (SCAP / HS + 2) * 4
                 ? 8 * (size_t)p
                 : (size_t)SCAP * 12 + 4 * (SCAP / HS + 2) * 4) +
            15) & ~size_t(15);
}
__host__ __device__ constexpr size_t small_smem(int p)
{
    return small_lreg(p) + (size_t)SCAP * sizeof(int2) + SM_RUNS;
}
static_assert(small_smem(BATCH_MAX_P) <= BATCH_SMEM, "k_small never needs more than the batched kernels");

// WRITE_L: instead of finishing a set, write its L (Algorithm 1's array,
// (p+1, -1) for an empty column) to L_out[L_offsets[set] ...].
template <bool WRITE_L>
__global__ void __launch_bounds__(BT, 1)
    k_batched(const int32_t *__restrict__ pts, const BItem *__restrict__ items, int nitems,
              const BSet *__restrict__ sets, int *queue, int *set_done, uint32_t *part,
              int2 *hull_out, const int64_t *__restrict__ hull_offsets, int *hull_counts,
              int2 *L_out, const int64_t *__restrict__ L_offsets, unsigned char *scratch,
              unsigned *status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item, s_ticket, s_total, s_cnt;
    __shared__ int s_warp[2 * (RUN / 32 + 1)];
    int *slo = reinterpret_cast<int *>(smem);
    int2 *scr = reinterpret_cast<int2 *>(scratch + (size_t)blockIdx.x * SCR_BYTES);
    bool bad = false;
    for (;;) {
        if (threadIdx.x == 0)
            s_item = atomicAdd(queue, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems)
            break;
        const BItem item = items[it];
        const BSet st = sets[item.set];
        const int p = st.p;
        int *shi = slo + p;
        for (int i = threadIdx.x; i < p; i += BT) {
            slo[i] = p + 1;
            shi[i] = -1;
        }
        __syncthreads();
        fold_range(pts + 2 * item.start, item.end - item.start, p, slo, shi, bad);
        __syncthreads();
        bool last = true;
        if (st.nchunks > 1) {
            uint32_t *row = part + st.part_off + (size_t)item.chunk * p;
            for (int i = threadIdx.x; i < p; i += BT)
                __stcg(row + i, slo[i] <= p ? ((uint32_t)(slo[i] - 1) << 16) | (uint32_t)(shi[i] - 1)
                                            : 0xFFFF0000u);
            __threadfence();
            __syncthreads();
            if (threadIdx.x == 0)
                s_ticket = atomicAdd(set_done + item.set, 1);
            __syncthreads();
            last = s_ticket == st.nchunks - 1;
            if (last) {
                __threadfence();
                const uint32_t *rows = part + st.part_off;
                for (int i = threadIdx.x; i < p; i += BT) {
                    uint32_t lo = 0xFFFFu, hi = 0;
                    for (int r = 0; r < st.nchunks; ++r) {
                        const uint32_t w = __ldcg(rows + (size_t)r * p + i);
                        lo = min(lo, w >> 16);
                        hi = max(hi, w & 0xFFFFu);
                    }
                    slo[i] = lo <= hi ? (int)lo + 1 : p + 1;
                    shi[i] = lo <= hi ? (int)hi + 1 : -1;
                }
                __syncthreads();
            }
        }
        if (last) {
            if constexpr (WRITE_L) {
                int2 *Lo = L_out + L_offsets[item.set];
                for (int i = threadIdx.x; i < p; i += BT)
                    Lo[i] = make_int2(slo[i], shi[i]);
            } else {
                finish_set(p, slo, shi, smem, scr, hull_out + hull_offsets[item.set],
                           hull_counts + item.set, s_warp, &s_total, &s_cnt);
            }
        }
        __syncthreads();
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0)
        atomicOr(status, ST_RANGE);
}

// ---------------------------------------------------------------- split CTA
// The hull mode of k_batched with the CTA split in two groups of whole warps.
// FW "fold" threads take items from the queue and fold them into L.  When a
// set is complete, the whole CTA runs its tile phase (collect_survivors needs
// L and one thread per column of a 1024-column tile); then the BT - FW
// "finish" threads peel, merge and stitch its survivors on a named barrier of
// their own while the fold threads already fold the next item into L.  The
// survivors and the peel buffers lie outside L, and the next tile phase
// begins only at a whole-CTA barrier the finish threads reach after their
// peel, so the two groups never use the same scratch at once.  (Running the
// tile pre-filter in the finish threads as well, on the set's valid columns
// extracted from L by the whole CTA, measured slower: 3.18 against 2.62 ms
// on the 10,000-set batch at a 512/512 split.)
// The survivor capacity BPW sets how much of the SM's 256 KB of combined
// L1 and shared memory is left to L1, which holds the fold threads' loads in
// flight: 4096 survivors (212 KB of shared memory, 28 KB of L1) against 2048
// (170 KB, 60 KB of L1): 2.55 against 2.27 ms per replay of the 10,000-set
// batch (1536: no further gain); a set with more survivors peels them in
// global scratch.
constexpr int WS_BAR_FOLD = 1, WS_BAR_FINISH = 2;  // named barriers (0 is the whole CTA)
#ifndef CH_BPW
#define CH_BPW 2048
#endif
constexpr int BPW = CH_BPW;  // survivors (both chains) peeled in shared memory
constexpr size_t WS_D = SM_L;                          // survivors (with B: the tile buffers at a hand-over)
constexpr size_t WS_B = WS_D + BPW * sizeof(int2);     // peel buffer B
constexpr size_t WS_F = WS_B + BPW * sizeof(int2);     // peel flags F
constexpr size_t WS_IX = WS_F + BPW * sizeof(int);     // merge-tree index arrays
constexpr size_t WS_SMEM = WS_IX + 4 * (BPW / HS + 2) * sizeof(int);
static_assert(SM_RUNS <= WS_F - WS_D, "the tile buffers fit the survivor and peel buffers D and B");
static_assert(WS_SMEM <= 227 * 1024, "one CTA's shared memory");

template <int FW>
__global__ void __launch_bounds__(BT, 1)
    k_batched_ws(const int32_t *__restrict__ pts, const BItem *__restrict__ items, int nitems,
                 const BSet *__restrict__ sets, int *queue, int *set_done, uint32_t *part,
                 int2 *hull_out, const int64_t *__restrict__ hull_offsets, int *hull_counts,
                 unsigned char *scratch, unsigned *status)
{
    constexpr int HW = BT - FW;
    static_assert(FW % 32 == 0 && HW % 32 == 0 && HW >= 64 && FW >= 256, "whole warps");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item, s_ticket, s_cnt, s_set, s_done;
    __shared__ int s_warp[2 * (RUN / 32 + 1)];  // tile phase (whole CTA)
    __shared__ int h_warp[HW / 32 + 1];         // peel (finish threads)
    __shared__ int h_total;
    int *slo = reinterpret_cast<int *>(smem);
    int2 *Ds = reinterpret_cast<int2 *>(smem + WS_D);
    int2 *scr = reinterpret_cast<int2 *>(scratch + (size_t)blockIdx.x * SCR_BYTES);
    bool bad = false;
    const int t = threadIdx.x;
    if (t < FW) {
        for (;;) {
            if (t == 0)
                s_item = atomicAdd(queue, 1);
            group_sync<WS_BAR_FOLD, FW>();
            const int it = s_item;
            if (it >= nitems)
                break;
            const BItem item = items[it];
            const BSet st = sets[item.set];
            const int p = st.p;
            int *shi = slo + p;
            for (int i = t; i < p; i += FW) {
                slo[i] = p + 1;
                shi[i] = -1;
            }
            group_sync<WS_BAR_FOLD, FW>();
            fold_range<FW>(pts + 2 * item.start, item.end - item.start, p, slo, shi, bad, t);
            group_sync<WS_BAR_FOLD, FW>();
            bool last = true;
            if (st.nchunks > 1) {
                uint32_t *row = part + st.part_off + (size_t)item.chunk * p;
                for (int i = t; i < p; i += FW)
                    __stcg(row + i, slo[i] <= p ? ((uint32_t)(slo[i] - 1) << 16) | (uint32_t)(shi[i] - 1)
                                                : 0xFFFF0000u);
                __threadfence();
                group_sync<WS_BAR_FOLD, FW>();
                if (t == 0)
                    s_ticket = atomicAdd(set_done + item.set, 1);
                group_sync<WS_BAR_FOLD, FW>();
                last = s_ticket == st.nchunks - 1;
                if (last) {
                    __threadfence();
                    const uint32_t *rows = part + st.part_off;
                    for (int i = t; i < p; i += FW) {
                        uint32_t lo = 0xFFFFu, hi = 0;
                        for (int r = 0; r < st.nchunks; ++r) {
                            const uint32_t w = __ldcg(rows + (size_t)r * p + i);
                            lo = min(lo, w >> 16);
                            hi = max(hi, w & 0xFFFFu);
                        }
                        slo[i] = lo <= hi ? (int)lo + 1 : p + 1;
                        shi[i] = lo <= hi ? (int)hi + 1 : -1;
                    }
                    group_sync<WS_BAR_FOLD, FW>();
                }
            }
            if (last) {
                if (t == 0) {
                    s_set = item.set;
                    s_done = 0;
                }
                group_sync<0, BT>();  // hand-over: the finish threads are done with the last set
                collect_survivors(p, slo, shi, smem + WS_D, Ds, BPW, scr, s_warp, &s_cnt);
            }
        }
        if (t == 0)
            s_done = 1;
        group_sync<0, BT>();  // the last hand-over: nothing more to finish
    } else {
        const int ht = t - FW;
        for (;;) {
            group_sync<0, BT>();  // hand-over from the fold threads
            if (s_done)
                break;
            const int set = s_set;  // read before the tile phase: s_set changes only after it
            const int p = sets[set].p;
            const Survivors sv =
                collect_survivors(p, slo, slo + p, smem + WS_D, Ds, BPW, scr, s_warp, &s_cnt);
            int2 *B;
            int *F, *ix;
            if (sv.in_smem) {
                B = reinterpret_cast<int2 *>(smem + WS_B);
                F = reinterpret_cast<int *>(smem + WS_F);
                ix = reinterpret_cast<int *>(smem + WS_IX);
            } else {
                global_peel_scratch(scr, B, F, ix);
            }
            peel_merge_stitch<HW, WS_BAR_FINISH, true>(sv.D, B, F, ix, sv.T0, sv.T,
                                                       hull_out + hull_offsets[set],
                                                       hull_counts + set, h_warp, &h_total, ht);
        }
    }
    if (__syncthreads_or(bad) && t == 0)
        atomicOr(status, ST_RANGE);
}

// Chains of every set from its L (as ch_chain does for one set): set s has
// side ps[s] and L at L[L_offsets[s] ...]; its k-th valid column (an entry
// other than (p+1, -1)) x gives lower[L_offsets[s] + k] = (x, ly) and
// upper[L_offsets[s] + k] = (x, hy); counts[2s] = counts[2s+1] = the number of
// valid columns.  CTAs stride over the sets; a set is scanned in tiles of BT
// columns (ballot, block scan).  Consecutive tiles, across sets too,
// alternate between two scan buffers, so no tile needs a closing barrier.
__global__ void __launch_bounds__(BT)
    k_chain_batched(const int2 *__restrict__ L, const int64_t *__restrict__ L_offsets,
                    const int *__restrict__ ps, int B, int2 *lower, int2 *upper, int *counts)
{
    __shared__ int s_buf[2][RUN / 32 + 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int k = 0;
    for (int set = blockIdx.x; set < B; set += gridDim.x) {
        const int p = ps[set];
        const int64_t base = L_offsets[set];
        int T = 0;
        for (int t0 = 0; t0 < p; t0 += BT, ++k) {
            int *sw = s_buf[k & 1];
            const int c = t0 + threadIdx.x;
            const int2 e = c < p ? L[base + c] : make_int2(p + 1, -1);
            const bool valid = c < p && !(e.x == p + 1 && e.y == -1);
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, valid);
            if (lane == 0)
                sw[w] = __popc(bal);
            __syncthreads();
            if (w == 0) {
                const int v = sw[lane];
                int incl = v;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                    if (lane >= o)
                        incl += x;
                }
                sw[lane] = incl - v;
                if (lane == 31)
                    sw[RUN / 32] = incl;
            }
            __syncthreads();
            if (valid) {
                const int64_t r = base + T + sw[w] + __popc(bal & ((1u << lane) - 1u));
                lower[r] = make_int2(c + 1, e.x);
                upper[r] = make_int2(c + 1, e.y);
            }
            T += sw[RUN / 32];
        }
        if (threadIdx.x == 0) {
            counts[2 * set] = T;
            counts[2 * set + 1] = T;
        }
    }
}

// ---------------------------------------------------------------- one small set
// One set in one launch: G CTAs fold consecutive slices of the points into
// private copies of L in shared memory; with G > 1 each writes its copy as a
// packed partial row and takes a ticket, and the CTA that takes the last one
// merges the rows.  That CTA (the only one when G = 1) then finishes the set
// as the batched kernel does (chains, exact pre-filter, peel/merge/stitch)
// and resets the ticket for the next call.  L_out (optional) receives L.
__global__ void __launch_bounds__(BT, 1)
    k_small(const int32_t *__restrict__ pts, int64_t n, int p, uint32_t *part, unsigned *ticket,
            unsigned char *scratch, int2 *L_out, int2 *hull, int *hull_count, unsigned *status)
{
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_total, s_cnt;
    __shared__ unsigned s_ticket;
    __shared__ int s_warp[2 * (RUN / 32 + 1)];
    int *slo = reinterpret_cast<int *>(smem), *shi = slo + p;
    for (int i = threadIdx.x; i < p; i += BT) {
        slo[i] = p + 1;
        shi[i] = -1;
    }
    __syncthreads();
    const int G = gridDim.x;
    const int64_t per = (((n + G - 1) / G) + 1) & ~(int64_t)1;  // even: slices keep pts' alignment
    const int64_t a = min(n, (int64_t)blockIdx.x * per), e = min(n, a + per);
    bool bad = false;
    fold_range(pts + 2 * a, e - a, p, slo, shi, bad);
    if (__syncthreads_or(bad) && threadIdx.x == 0)
        atomicOr(status, ST_RANGE);
    if (G > 1) {
        uint32_t *row = part + (size_t)blockIdx.x * p;
        for (int i = threadIdx.x; i < p; i += BT)
            __stcg(row + i, slo[i] <= p ? ((uint32_t)(slo[i] - 1) << 16) | (uint32_t)(shi[i] - 1)
                                        : 0xFFFF0000u);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0)
            s_ticket = atomicAdd(ticket, 1u);
        __syncthreads();
        if (s_ticket != (unsigned)(G - 1))
            return;  // block-uniform: another CTA finishes the set
        __threadfence();
        for (int i = threadIdx.x; i < p; i += BT) {
            uint32_t lo = 0xFFFFu, hi = 0;
            int r = 0;
            for (; r + 8 <= G; r += 8) {  // eight loads in flight
                uint32_t w[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    w[u] = __ldcg(part + (size_t)(r + u) * p + i);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    lo = min(lo, w[u] >> 16);
                    hi = max(hi, w[u] & 0xFFFFu);
                }
            }
            for (; r < G; ++r) {
                const uint32_t w = __ldcg(part + (size_t)r * p + i);
                lo = min(lo, w >> 16);
                hi = max(hi, w & 0xFFFFu);
            }
            slo[i] = lo <= hi ? (int)lo + 1 : p + 1;
            shi[i] = lo <= hi ? (int)hi + 1 : -1;
        }
        if (threadIdx.x == 0)
            *ticket = 0;  // every CTA of this launch has taken its ticket
        __syncthreads();
    }
    if (L_out)
        for (int i = threadIdx.x; i < p; i += BT)
            L_out[i] = make_int2(slo[i], shi[i]);
    const size_t lreg = small_lreg(p);
    finish_set_at(p, slo, shi, smem, smem + lreg + (size_t)SCAP * sizeof(int2),
                  reinterpret_cast<int2 *>(smem + lreg), SCAP, reinterpret_cast<int2 *>(scratch),
                  hull, hull_count, s_warp, &s_total, &s_cnt);
}

constexpr int SMALL_PPC = 8192;                // points per CTA of k_small
constexpr long long SMALL_ROW_WORDS = 1 << 16;  // partial-row words the last CTA merges

struct BatchWs {
    size_t head, items, sets, part, scratch, end;
};

// Workspace of a prepared batch: [queue, set_done[B]][items][sets][partials][scratch].
BatchWs batch_layout(int B, size_t nitems, size_t part_words, int grid)
{
    WsLayout w;
    BatchWs b;
    b.head = w.take((size_t)(B + 2) * sizeof(int));
    b.items = w.take(nitems * sizeof(BItem));
    b.sets = w.take((size_t)B * sizeof(BSet));
    b.part = w.take(part_words * sizeof(uint32_t));
    b.scratch = w.take((size_t)grid * SCR_BYTES);
    b.end = w.off;
    return b;
}

void build_plan(int B, const int64_t *off, const int32_t *ps, int chunk_mult,
                std::vector<BItem> &items, std::vector<BSet> &sets, long long &part_words)
{
    items.clear();
    sets.assign(B, BSet{0, 1, 1});
    part_words = 0;
    for (int s = 0; s < B; ++s) {
        const long long n = off[s + 1] - off[s];
        const int p = ps[s];
        // chunk: chunk_mult points per column, at least 64K, at most 4M points
        const long long chunk = std::min<long long>(std::max<long long>((long long)chunk_mult * p, 65536),
                                                    1ll << 22);
        const int nch = (int)std::max<long long>(1, (n + chunk - 1) / chunk);
        sets[s].p = p;
        sets[s].nchunks = nch;
        sets[s].part_off = 0;
        if (nch > 1) {
            sets[s].part_off = part_words;
            part_words += (long long)nch * p;
        }
        for (int c = 0; c < nch; ++c) {
            const long long a = off[s] + (long long)c * chunk;
            const long long e = std::min<long long>(off[s + 1], a + chunk);
            items.push_back(BItem{a, e, s, c});
        }
    }
    std::stable_sort(items.begin(), items.end(), [](const BItem &a, const BItem &b) {
        return (a.end - a.start) > (b.end - b.start);
    });
}

}  // namespace

size_t batch_smem() { return BATCH_SMEM; }

int small_ctas(int64_t n, int p)
{
    if (n < 0 || p < 1 || p > BATCH_MAX_P)
        return 0;
    const long long g = std::max<long long>(1, (n + SMALL_PPC - 1) / SMALL_PPC);
    const long long gmax = std::max<long long>(1, SMALL_ROW_WORDS / p);
    const int sms = sm_count();
    if (sms <= 0 || g > gmax || g > sms)
        return 0;
    return (int)g;
}

size_t small_ws_bytes(int G, int p)
{
    WsLayout w;
    w.take(G > 1 ? (size_t)G * p * sizeof(uint32_t) : 0);
    w.take(SCR_BYTES);
    return w.off;
}

cudaError_t small_launch(const int32_t *pts, int64_t n, int p, int G, void *ws, unsigned *ticket,
                         int32_t *L_out, int32_t *hull, int32_t *hull_count, unsigned *status,
                         cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1)
{
    static bool attr[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return cudaErrorUnknown;
    if (dev >= 0 && dev < 64 && !attr[dev]) {
        const cudaError_t e = cudaFuncSetAttribute(
            k_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BATCH_SMEM);
        if (e != cudaSuccess)
            return e;
        attr[dev] = true;
    }
    WsLayout w;
    char *b = reinterpret_cast<char *>(ws);
    uint32_t *part = reinterpret_cast<uint32_t *>(
        b + w.take(G > 1 ? (size_t)G * p * sizeof(uint32_t) : 0));
    unsigned char *scratch = reinterpret_cast<unsigned char *>(b + w.take(SCR_BYTES));
    if (ev0)
        cudaEventRecord(ev0, s);
    launch(k_small, G, BT, small_smem(p), s, pts, n, p, part, ticket, scratch,
           reinterpret_cast<int2 *>(L_out), reinterpret_cast<int2 *>(hull), hull_count, status);
    if (ev1)
        cudaEventRecord(ev1, s);
    return cudaGetLastError();
}

int batch_sizes(int B, const int64_t *off, const int32_t *ps, int chunk_mult, size_t *ws_bytes,
                BatchPlanInfo *info)
{
    std::vector<BItem> items;
    std::vector<BSet> sets;
    long long pw = 0;
    build_plan(B, off, ps, chunk_mult, items, sets, pw);
    const int grid = sm_count();
    if (grid <= 0)
        return CH_ERR_CUDA;
    const BatchWs l = batch_layout(B, items.size(), (size_t)pw, grid);
    *ws_bytes = l.end;
    if (info) {
        info->B = B;
        info->nitems = (int)items.size();
        info->grid = grid;
        info->part_words = pw;
        info->fold = 0;
    }
    return CH_OK;
}

int batch_prepare(int B, const int64_t *off, const int32_t *ps, int chunk_mult, void *ws,
                  size_t ws_bytes, cudaStream_t s, BatchPlanInfo *info)
{
    std::vector<BItem> items;
    std::vector<BSet> sets;
    long long pw = 0;
    build_plan(B, off, ps, chunk_mult, items, sets, pw);
    const int grid = sm_count();
    if (grid <= 0)
        return CH_ERR_CUDA;
    const BatchWs l = batch_layout(B, items.size(), (size_t)pw, grid);
    if (ws_bytes < l.end)
        return CH_ERR_WORKSPACE;
    char *b = reinterpret_cast<char *>(ws);
    if (cudaMemcpyAsync(b + l.items, items.data(), items.size() * sizeof(BItem),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(b + l.sets, sets.data(), sets.size() * sizeof(BSet),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)  // the host vectors die on return
        return CH_ERR_CUDA;
    info->B = B;
    info->nitems = (int)items.size();
    info->grid = grid;
    info->part_words = pw;
    info->fold = 0;
    return CH_OK;
}

int batch_launch(const int32_t *pts, int2 *hull_out, const int64_t *hull_offsets, int *hull_counts,
                 int2 *L_out, const int64_t *L_offsets, void *ws, size_t ws_bytes,
                 const BatchPlanInfo &info, unsigned *status, cudaStream_t s)
{
    const BatchWs l = batch_layout(info.B, (size_t)info.nitems, (size_t)info.part_words, info.grid);
    if (ws_bytes < l.end)
        return CH_ERR_WORKSPACE;
    static bool attr[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr[dev]) {
        const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
        if (cudaFuncSetAttribute(k_batched<false>, a, (int)BATCH_SMEM) != cudaSuccess ||
            cudaFuncSetAttribute(k_batched<true>, a, (int)BATCH_SMEM) != cudaSuccess ||
            cudaFuncSetAttribute(k_batched_ws<384>, a, (int)WS_SMEM) != cudaSuccess ||
            cudaFuncSetAttribute(k_batched_ws<512>, a, (int)WS_SMEM) != cudaSuccess ||
            cudaFuncSetAttribute(k_batched_ws<640>, a, (int)WS_SMEM) != cudaSuccess ||
            cudaFuncSetAttribute(k_batched_ws<768>, a, (int)WS_SMEM) != cudaSuccess ||
            cudaFuncSetAttribute(k_batched_ws<896>, a, (int)WS_SMEM) != cudaSuccess)
            return CH_ERR_CUDA;
        attr[dev] = true;
    }
    char *b = reinterpret_cast<char *>(ws);
    int *head = reinterpret_cast<int *>(b + l.head);
    if (cudaMemsetAsync(head, 0, (size_t)(info.B + 2) * sizeof(int), s) != cudaSuccess)
        return CH_ERR_CUDA;
    if (!L_out && info.fold > 0) {
        if (!batch_fold_ok(info.fold))
            return CH_ERR_ARG;
        auto ws_kern = info.fold == 384   ? k_batched_ws<384>
                       : info.fold == 512 ? k_batched_ws<512>
                       : info.fold == 640 ? k_batched_ws<640>
                       : info.fold == 768 ? k_batched_ws<768>
                                          : k_batched_ws<896>;
        ws_kern<<<info.grid, BT, WS_SMEM, s>>>(
            pts, reinterpret_cast<const BItem *>(b + l.items), info.nitems,
            reinterpret_cast<const BSet *>(b + l.sets), head, head + 1,
            reinterpret_cast<uint32_t *>(b + l.part), hull_out, hull_offsets, hull_counts,
            reinterpret_cast<unsigned char *>(b + l.scratch), status);
        return cudaGetLastError() == cudaSuccess ? CH_OK : CH_ERR_CUDA;
    }
    auto kern = L_out ? k_batched<true> : k_batched<false>;
    // writing L needs only L's region of the layout (the rest would take L1)
    kern<<<info.grid, BT, L_out ? SM_L : BATCH_SMEM, s>>>(
        pts, reinterpret_cast<const BItem *>(b + l.items), info.nitems,
        reinterpret_cast<const BSet *>(b + l.sets), head, head + 1,
        reinterpret_cast<uint32_t *>(b + l.part), hull_out, hull_offsets, hull_counts, L_out,
        L_offsets, reinterpret_cast<unsigned char *>(b + l.scratch), status);
    return cudaGetLastError() == cudaSuccess ? CH_OK : CH_ERR_CUDA;
}

int chain_batched_launch(const int2 *L, const int64_t *L_offsets, const int *ps, int B, int2 *lower,
                         int2 *upper, int *counts, cudaStream_t s)
{
    const int sms = sm_count();
    if (sms <= 0)
        return CH_ERR_CUDA;
    const int grid = std::max(1, std::min(B, 2 * sms));
    k_chain_batched<<<grid, BT, 0, s>>>(L, L_offsets, ps, B, lower, upper, counts);
    return cudaGetLastError() == cudaSuccess ? CH_OK : CH_ERR_CUDA;
}

}  // namespace ch
