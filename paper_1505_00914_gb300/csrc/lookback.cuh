// Decoupled look-back over tiles (a single-pass exclusive scan across the
// thread blocks of one grid), shared by the compaction kernels.  Tile j's
// word ts[j] holds 0 (nothing yet), FLAG_AGG | count (its own count) or
// FLAG_PRE | inclusive prefix.  Tiles take their index from an atomic ticket
// in launch order, so every tile a tile waits on is already running; every
// wait is bounded by SPIN_LIMIT and reports CH_ERR_TIMEOUT when it runs out.
#pragma once

#include <cuda/atomic>

#include "ch_internal.cuh"

namespace ch {
namespace {

constexpr unsigned long long FLAG_AGG = 1ull << 62;
constexpr unsigned long long FLAG_PRE = 2ull << 62;
constexpr unsigned long long VAL_MASK = (1ull << 62) - 1;

using aref = cuda::atomic_ref<unsigned long long, cuda::thread_scope_device>;

// Exclusive prefix of tile `tile` by decoupled look-back, run by a full warp.
// A window covers LB_W * 32 predecessors (lane l, slot k inspects tile
// base - l - 32k), all loads in flight at once; the window moves back until
// it meets a tile that has published its inclusive prefix.  Waiting tiles are
// running (ticket order), so the spin polls without sleeping; it is bounded.
constexpr int LB_W = 8;

// Publishes the tile's own count (tile 0: its inclusive prefix); one thread.
__device__ __forceinline__ void publish_aggregate(unsigned long long *ts, int tile, long long agg)
{
    aref(ts[tile]).store((tile == 0 ? FLAG_PRE : FLAG_AGG) | (unsigned long long)agg,
                         cuda::memory_order_release);
}

// The tile's exclusive prefix; its aggregate was published earlier.
__device__ long long warp_look_back(unsigned long long *ts, int tile, long long agg, int lane,
                                    unsigned *status)
{
    if (tile == 0)
        return 0;
    long long excl = 0;
    int base = tile - 1;
    int spins = 0;
    bool timed_out = false;
    while (base >= 0) {
        unsigned long long v[LB_W];
#pragma unroll
        for (int k = 0; k < LB_W; ++k) {
            const int j = base - lane - 32 * k;
            v[k] = j >= 0 ? aref(ts[j]).load(cuda::memory_order_acquire) : FLAG_PRE;
        }
#pragma unroll
        for (int k = 0; k < LB_W; ++k) {
            const int j = base - lane - 32 * k;
            while ((v[k] & ~VAL_MASK) == 0) {
                if (++spins > SPIN_LIMIT) {
                    timed_out = true;
                    v[k] = FLAG_PRE;
                    break;
                }
                v[k] = aref(ts[j]).load(cuda::memory_order_acquire);
            }
        }
        // nearest inclusive prefix in the window: slot k, lane l <-> distance 32k + l
        int stop = 32 * LB_W;
#pragma unroll
        for (int k = LB_W - 1; k >= 0; --k) {
            const unsigned pre = __ballot_sync(0xFFFFFFFFu, (v[k] & ~VAL_MASK) == FLAG_PRE);
            if (pre)
                stop = 32 * k + __ffs(pre) - 1;
        }
        long long val = 0;
#pragma unroll
        for (int k = 0; k < LB_W; ++k)
            if (32 * k + lane <= stop)
                val += (long long)(v[k] & VAL_MASK);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            val += __shfl_xor_sync(0xFFFFFFFFu, val, o);
        excl += val;
        if (stop < 32 * LB_W)
            break;
        base -= 32 * LB_W;
    }
    if (__any_sync(0xFFFFFFFFu, timed_out) && lane == 0)
        atomicOr(status, ST_TIMEOUT);
    if (lane == 0)
        aref(ts[tile]).store(FLAG_PRE | (unsigned long long)(excl + agg), cuda::memory_order_release);
    return excl;
}

}  // namespace
}  // namespace ch
