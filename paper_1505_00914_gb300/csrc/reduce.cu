// Step 1: Algorithm 1 (Reduction of Points, Section 2.1) on sm_103a.
//
// Each point (x, y) folds into column x of L as (min(y, ly), max(y, hy)).
// Min and max commute, so any order of folding gives the same L; the GPU
// folds in parallel into private copies of L and merges them afterwards.
//
// Private copies live in shared memory as one packed 32-bit word per column
// (lo16 = min y - 1, hi16 = max y - 1), so p <= 65536 columns need at most
// 256 KB.  When that exceeds one CTA's shared memory (227 KB on GB300), two
// CTAs of a thread-block cluster split the x range and fold the other half's
// points into their partner's shared memory (distributed shared memory).
// Every fold first reads the column word and only issues a compare-and-swap
// when y falls outside [lo, hi]: the word only ever widens, so a stale read
// can only cause a redundant CAS, never a missed update.
//
// Each copy ends as one row of a partial array in the workspace; the chain
// step (or reduce_merge below) combines the rows column by column.
// p > 65536 uses a global-memory L with the same read-then-atomic rule.
#include <cooperative_groups.h>

#include "ch_internal.cuh"

namespace cg = cooperative_groups;

namespace ch {
namespace {

constexpr int RT = 512;  // threads per CTA
constexpr int RU = 4;    // 16-byte loads in flight per thread per iteration

__device__ __forceinline__ void fold(uint32_t *a, uint32_t v)
{
    uint32_t w = *reinterpret_cast<volatile uint32_t *>(a);
    uint32_t lo = w >> 16, hi = w & 0xFFFFu;
    while (v < lo || v > hi) {
        uint32_t nw = (min(lo, v) << 16) | max(hi, v);
        uint32_t prev = atomicCAS(a, w, nw);
        if (prev == w)
            return;
        w = prev;
        lo = w >> 16;
        hi = w & 0xFFFFu;
    }
}

template <int CL>
__global__ void __launch_bounds__(RT, 1)
    k_reduce_packed(const int32_t *__restrict__ pts, int64_t n, int p, int cols,
                    uint32_t *__restrict__ part, unsigned *status)
{
    extern __shared__ __align__(16) uint32_t sL[];
    for (int i = threadIdx.x; i < cols; i += RT)
        sL[i] = PACK_EMPTY;

    uint32_t *base0 = sL, *base1 = sL;
    int rank = 0;
    if constexpr (CL == 1) {
        __syncthreads();
    } else {
        cg::cluster_group cl = cg::this_cluster();
        rank = (int)cl.block_rank();
        cl.sync();  // partner's words initialised before any remote fold
        base0 = cl.map_shared_rank(sL, 0);
        base1 = cl.map_shared_rank(sL, 1);
    }

    const uint32_t up = (uint32_t)p, ucols = (uint32_t)cols;
    bool bad = false;
    auto proc = [&](int x, int y) {
        uint32_t c = (uint32_t)(x - 1), v = (uint32_t)(y - 1);
        if (c >= up || v >= up) {
            bad = true;
            return;
        }
        uint32_t *a;
        if constexpr (CL == 1)
            a = sL + c;
        else
            a = c < ucols ? base0 + c : base1 + (c - ucols);
        fold(a, v);
    };

    // 16-byte loads need a 16-byte aligned start; an 8-byte aligned array
    // has its first point handled on its own, and an odd tail likewise.
    const int64_t head = (((uintptr_t)pts & 15) != 0 && n > 0) ? 1 : 0;
    const int64_t npairs = (n - head) >> 1;
    if (blockIdx.x == 0 && threadIdx.x == 0 && head)
        proc(pts[0], pts[1]);
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0 && ((n - head) & 1))
        proc(pts[2 * (n - 1)], pts[2 * (n - 1) + 1]);
    const int4 *p4 = reinterpret_cast<const int4 *>(pts + 2 * head);

    const int64_t per = (npairs + gridDim.x - 1) / gridDim.x;
    const int64_t s0 = (int64_t)blockIdx.x * per;
    const int64_t e0 = min(npairs, s0 + per);
    for (int64_t i = s0 + threadIdx.x; i < e0; i += (int64_t)RT * RU) {
        int4 v[RU];
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            int64_t j = i + (int64_t)u * RT;
            if (j < e0)
                v[u] = __ldcs(p4 + j);
        }
#pragma unroll
        for (int u = 0; u < RU; ++u) {
            int64_t j = i + (int64_t)u * RT;
            if (j < e0) {
                proc(v[u].x, v[u].y);
                proc(v[u].z, v[u].w);
            }
        }
    }

    if constexpr (CL == 1)
        __syncthreads();
    else
        cg::this_cluster().sync();  // every remote fold has landed

    const int copy = blockIdx.x / CL;
    const int c0 = rank * cols;
    const int mine = min(cols, p - c0);
    uint32_t *out = part + (size_t)copy * p + c0;
    for (int i = threadIdx.x; i < mine; i += RT)
        out[i] = sL[i];
    if (__syncthreads_or(bad) && threadIdx.x == 0)
        atomicOr(status, ST_RANGE);
}

__global__ void k_fill_empty(int2 *L, int p)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < p; i += gridDim.x * blockDim.x)
        L[i] = make_int2(p + 1, -1);
}

// Large-p form: L in global memory (L2-resident for moderate p).
__global__ void __launch_bounds__(256)
    k_reduce_global(const int2 *__restrict__ pts, int64_t n, int p, int2 *L, unsigned *status)
{
    bool bad = false;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int2 q = __ldcs(pts + k);
        uint32_t c = (uint32_t)(q.x - 1), v = (uint32_t)(q.y - 1);
        if (c >= (uint32_t)p || v >= (uint32_t)p) {
            bad = true;
            continue;
        }
        volatile int *e = reinterpret_cast<volatile int *>(L + c);
        if (q.y < e[0])
            atomicMin(&L[c].x, q.y);
        if (q.y > e[1])
            atomicMax(&L[c].y, q.y);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0)
        atomicOr(status, ST_RANGE);
}

__global__ void __launch_bounds__(256)
    k_merge_partials(const uint32_t *__restrict__ part, int copies, int p, int2 *L)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < p; c += gridDim.x * blockDim.x) {
        uint32_t lo = 0xFFFFu, hi = 0;
        for (int j = 0; j < copies; ++j) {
            uint32_t w = __ldcg(part + (size_t)j * p + c);
            lo = min(lo, w >> 16);
            hi = max(hi, w & 0xFFFFu);
        }
        L[c] = lo <= hi ? make_int2((int)lo + 1, (int)hi + 1) : make_int2(p + 1, -1);
    }
}

int optin_smem()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

}  // namespace

int reduce_plan(int64_t n, int p, ReducePlan *pl)
{
    const int sms = sm_count();
    if (sms <= 0)
        return CH_ERR_CUDA;
    if (p > PACK_MAX_P) {
        pl->mode = 1;
        pl->cluster = 1;
        pl->copies = 0;
        pl->cols = 0;
        pl->smem = 0;
        int64_t want = (n + 255) / 256;
        pl->grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
        return CH_OK;
    }
    const int optin = optin_smem();
    pl->mode = 0;
    pl->cluster = ((size_t)p * 4 <= (size_t)optin) ? 1 : 2;
    pl->cols = (p + pl->cluster - 1) / pl->cluster;
    pl->smem = (size_t)pl->cols * 4;
    const int64_t npairs = n / 2;
    // at least ~8K points per CTA so the private copy pays for itself
    const int64_t want = std::max<int64_t>(1, (npairs + RT * RU * 2 - 1) / (RT * RU * 2));
    int resident = 0;
    if (pl->cluster == 1) {
        cudaFuncSetAttribute(k_reduce_packed<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pl->smem);
        int bps = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_reduce_packed<1>, RT, pl->smem) !=
            cudaSuccess)
            return CH_ERR_CUDA;
        resident = std::max(1, bps) * sms;
        pl->grid = (int)std::min<int64_t>(want, resident);
    } else {
        cudaFuncSetAttribute(k_reduce_packed<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pl->smem);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(2 * sms);
        cfg.blockDim = dim3(RT);
        cfg.dynamicSmemBytes = pl->smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 2;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, k_reduce_packed<2>, &cfg) != cudaSuccess)
            return CH_ERR_CUDA;
        nc = std::max(1, nc);
        int64_t clusters = std::min<int64_t>((want + 1) / 2, nc);
        pl->grid = (int)std::max<int64_t>(1, clusters) * 2;
    }
    pl->copies = pl->grid / pl->cluster;
    return CH_OK;
}

size_t reduce_partials_bytes(const ReducePlan &pl, int p)
{
    return pl.mode == 0 ? (size_t)pl.copies * (size_t)p * 4 : 0;
}

cudaError_t reduce_launch(const ReducePlan &pl, const int32_t *pts, int64_t n, int p,
                          uint32_t *part, int32_t *L, unsigned *status, cudaStream_t s)
{
    if (pl.mode == 1) {
        int2 *L2 = reinterpret_cast<int2 *>(L);
        k_fill_empty<<<std::min((p + 255) / 256, 4096), 256, 0, s>>>(L2, p);
        if (n > 0)
            k_reduce_global<<<pl.grid, 256, 0, s>>>(reinterpret_cast<const int2 *>(pts), n, p, L2,
                                                   status);
        return cudaGetLastError();
    }
    if (pl.cluster == 1) {
        k_reduce_packed<1><<<pl.grid, RT, pl.smem, s>>>(pts, n, p, pl.cols, part, status);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(pl.grid);
    cfg.blockDim = dim3(RT);
    cfg.dynamicSmemBytes = pl.smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_reduce_packed<2>, pts, n, p, pl.cols, part, status);
}

cudaError_t reduce_merge_launch(const uint32_t *part, int copies, int p, int32_t *L,
                                cudaStream_t s)
{
    int blocks = std::min((p + 255) / 256, sm_count() * 8);
    k_merge_partials<<<std::max(1, blocks), 256, 0, s>>>(part, copies, p,
                                                         reinterpret_cast<int2 *>(L));
    return cudaGetLastError();
}

}  // namespace ch
