// Step 2: the valid columns of L as x-ordered lower and upper chains
// (Lemma 1, Section 2.1), via the bit array M of Section 4.
//
// Each warp's __ballot_sync over 32 consecutive columns is exactly one 32-bit
// word of M (column i at bit (i-1) & 31 of word (i-1) >> 5, the paper's
// block/bit indexing with w = 32).  Where the paper walks set bits with ctz,
// the GPU ranks them: a column's output slot is the number of valid columns
// before it, popc of the lower bits of its word plus an exclusive scan over
// words.  The scan runs in one pass over the tiles of L: each tile publishes
// its count and looks back at its predecessors' (decoupled look-back), with
// tiles handed out in launch order by an atomic ticket so that every tile it
// waits on is already running; every wait is bounded.
#include <cuda/atomic>

#include "ch_internal.cuh"

namespace ch {
namespace {

constexpr int CT = 256;           // threads per CTA
constexpr int CPT = 4;            // columns per thread
constexpr int WPB = CT / 32;      // warps per CTA
constexpr int TILE = CT * CPT;    // columns per tile (= 32 words of M)
static_assert(CPT * WPB == 32, "one warp scans the tile's words");

constexpr unsigned long long FLAG_AGG = 1ull << 62;
constexpr unsigned long long FLAG_PRE = 2ull << 62;
constexpr unsigned long long VAL_MASK = (1ull << 62) - 1;

using aref = cuda::atomic_ref<unsigned long long, cuda::thread_scope_device>;

__device__ long long look_back(unsigned long long *ts, int tile, long long agg, unsigned *status)
{
    if (tile == 0) {
        aref(ts[0]).store(FLAG_PRE | (unsigned long long)agg, cuda::memory_order_release);
        return 0;
    }
    aref(ts[tile]).store(FLAG_AGG | (unsigned long long)agg, cuda::memory_order_release);
    long long excl = 0;
    int j = tile - 1, spins = 0;
    while (j >= 0) {
        unsigned long long v = aref(ts[j]).load(cuda::memory_order_acquire);
        unsigned long long f = v & ~VAL_MASK;
        if (f == 0) {
            if (++spins > SPIN_LIMIT) {
                atomicOr(status, ST_TIMEOUT);
                break;
            }
            __nanosleep(100);
            continue;
        }
        excl += (long long)(v & VAL_MASK);
        if (f == FLAG_PRE)
            break;
        --j;
    }
    aref(ts[tile]).store(FLAG_PRE | (unsigned long long)(excl + agg), cuda::memory_order_release);
    return excl;
}

template <bool FROM_PART>
__global__ void __launch_bounds__(CT)
    k_chain(const int2 *__restrict__ Lin, const uint32_t *__restrict__ part, int copies, int p,
            int2 *Lout, int2 *lower, int2 *upper, int *counts, uint32_t *mask,
            unsigned long long *state, int ntiles, unsigned *status)
{
    __shared__ int s_tile;
    __shared__ int s_wc[CPT * WPB];
    __shared__ long long s_prefix;
    if (threadIdx.x == 0)
        s_tile = (int)atomicAdd(state, 1ull);
    __syncthreads();
    const int tile = s_tile;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;

    int2 e[CPT];
    unsigned bal[CPT];
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        const int c = tile * TILE + k * CT + threadIdx.x;  // 0-based column
        const bool inr = c < p;
        bool valid;
        if constexpr (FROM_PART) {
            uint32_t lo = 0xFFFFu, hi = 0;
            if (inr) {
                const uint32_t *q = part + c;
                int j = 0;
                for (; j + 4 <= copies; j += 4) {
                    uint32_t a0 = __ldcg(q + (size_t)(j + 0) * p), a1 = __ldcg(q + (size_t)(j + 1) * p);
                    uint32_t a2 = __ldcg(q + (size_t)(j + 2) * p), a3 = __ldcg(q + (size_t)(j + 3) * p);
                    lo = min(min(lo, a0 >> 16), min(a1 >> 16, min(a2 >> 16, a3 >> 16)));
                    hi = max(max(hi, a0 & 0xFFFFu), max(a1 & 0xFFFFu, max(a2 & 0xFFFFu, a3 & 0xFFFFu)));
                }
                for (; j < copies; ++j) {
                    uint32_t a = __ldcg(q + (size_t)j * p);
                    lo = min(lo, a >> 16);
                    hi = max(hi, a & 0xFFFFu);
                }
            }
            valid = inr && lo <= hi;
            e[k] = valid ? make_int2((int)lo + 1, (int)hi + 1) : make_int2(p + 1, -1);
            if (inr && Lout)
                Lout[c] = e[k];
        } else {
            e[k] = inr ? Lin[c] : make_int2(p + 1, -1);
            valid = inr && !(e[k].x == p + 1 && e[k].y == -1);
        }
        bal[k] = __ballot_sync(0xFFFFFFFFu, valid);
        if (lane == 0) {
            s_wc[k * WPB + w] = __popc(bal[k]);
            if (mask && c < p)
                mask[c >> 5] = bal[k];
        }
    }
    __syncthreads();
    if (w == 0) {
        int v = s_wc[lane];
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o)
                incl += t;
        }
        s_wc[lane] = incl - v;
        const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        if (lane == 0) {
            long long pre = look_back(state + 1, tile, total, status);
            s_prefix = pre;
            if (tile == ntiles - 1) {
                counts[0] = (int)(pre + total);
                counts[1] = (int)(pre + total);
            }
        }
    }
    __syncthreads();
    const long long pre = s_prefix;
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
        if ((bal[k] >> lane) & 1u) {
            const int c = tile * TILE + k * CT + threadIdx.x;
            const long long pos = pre + s_wc[k * WPB + w] + __popc(bal[k] & lt);
            lower[pos] = make_int2(c + 1, e[k].x);
            upper[pos] = make_int2(c + 1, e[k].y);
        }
    }
}

}  // namespace

int chain_tiles(int p) { return (p + TILE - 1) / TILE; }

size_t chain_state_bytes(int p) { return (size_t)(chain_tiles(p) + 1) * 8; }

cudaError_t chain_launch(const int32_t *L_in, const uint32_t *partials, int copies, int p,
                         int32_t *L_out, int32_t *lower, int32_t *upper, int32_t *counts,
                         uint32_t *mask, void *state, unsigned *status, cudaStream_t s)
{
    const int nt = chain_tiles(p);
    cudaError_t e = cudaMemsetAsync(state, 0, chain_state_bytes(p), s);
    if (e != cudaSuccess)
        return e;
    auto *st = reinterpret_cast<unsigned long long *>(state);
    if (partials)
        k_chain<true><<<nt, CT, 0, s>>>(nullptr, partials, copies, p,
                                        reinterpret_cast<int2 *>(L_out),
                                        reinterpret_cast<int2 *>(lower),
                                        reinterpret_cast<int2 *>(upper), counts, mask, st, nt,
                                        status);
    else
        k_chain<false><<<nt, CT, 0, s>>>(reinterpret_cast<const int2 *>(L_in), nullptr, 0, p,
                                         nullptr, reinterpret_cast<int2 *>(lower),
                                         reinterpret_cast<int2 *>(upper), counts, mask, st, nt,
                                         status);
    return cudaGetLastError();
}

}  // namespace ch
