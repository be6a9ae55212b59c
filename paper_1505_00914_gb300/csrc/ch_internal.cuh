// Internal declarations shared by the translation units of libch.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "ch.h"

namespace ch {

// Bits of the per-device sticky status word.
enum : unsigned {
    ST_RANGE = 1u,
    ST_CAPACITY = 2u,
    ST_TIMEOUT = 4u,
};

// Iteration cap of every inter-block spin (decoupled look-back).  Each
// iteration sleeps ~0.1-1 us, so the cap is well above any legal wait and
// far below a hang.
constexpr int SPIN_LIMIT = 1 << 22;

// Packed private column word of the reduction: (lo16 << 16) | hi16 with
// lo16 = min(y) - 1 and hi16 = max(y) - 1; an empty column is lo16 = 0xFFFF,
// hi16 = 0.  A column is non-empty iff lo16 <= hi16 (a column whose only y is
// p = 65536 holds lo16 = hi16 = 0xFFFF).  Usable for p <= 65536.
constexpr uint32_t PACK_EMPTY = 0xFFFF0000u;
constexpr int PACK_MAX_P = 65536;

// 64-bit orientation of (o, a, b): > 0 for a counter-clockwise turn.
__device__ __forceinline__ long long cross3(int2 o, int2 a, int2 b)
{
    return (long long)(a.x - o.x) * (long long)(b.y - o.y) -
           (long long)(a.y - o.y) * (long long)(b.x - o.x);
}

// Bump allocator for workspace layouts (256-byte aligned regions).
struct WsLayout {
    size_t off = 0;
    size_t take(size_t bytes)
    {
        size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return o;
    }
};

// ---- reduction (reduce.cu) ----
struct ReducePlan {
    int mode;      // 0: private packed copies, 1: global atomics (p > 65536)
    int cluster;   // CTAs sharing one private copy (1 or 2)
    int grid;      // CTAs launched
    int copies;    // grid / cluster = number of partial arrays
    int cols;      // columns held per CTA
    size_t smem;   // dynamic shared memory per CTA
};
int reduce_plan(int64_t n, int p, ReducePlan *plan);
size_t reduce_partials_bytes(const ReducePlan &plan, int p);
// Writes plan.copies packed partial arrays of p words each (mode 0), or the
// final L directly (mode 1).
cudaError_t reduce_launch(const ReducePlan &plan, const int32_t *pts, int64_t n, int p,
                          uint32_t *partials, int32_t *L, unsigned *status, cudaStream_t s);
// L = column-wise merge of `copies` packed partial arrays.
cudaError_t reduce_merge_launch(const uint32_t *partials, int copies, int p, int32_t *L,
                                cudaStream_t s);

// ---- chain (chain.cu) ----
int chain_tiles(int p);
size_t chain_state_bytes(int p);
// If partials != nullptr, merges `copies` packed arrays into L first (and
// writes L if L_out != nullptr); otherwise reads L_in.
cudaError_t chain_launch(const int32_t *L_in, const uint32_t *partials, int copies, int p,
                         int32_t *L_out, int32_t *lower, int32_t *upper, int32_t *counts,
                         uint32_t *mask, void *state, unsigned *status, cudaStream_t s);

// ---- hull (hull.cu) ----
size_t hull_ws_bytes(int p);
cudaError_t hull_launch(const int32_t *lower, const int32_t *upper, const int32_t *counts, int p,
                        int32_t *hull, int32_t *hull_count, void *ws, unsigned *status,
                        cudaStream_t s);

// ---- api.cu ----
unsigned *device_status_ptr();  // this device's status word (nullptr on failure)
int sm_count();

}  // namespace ch
