// Internal declarations shared by the translation units of libch.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "ch.h"

namespace ch {

// Bits of the per-stream sticky status word.
enum : unsigned {
    ST_RANGE = 1u,
    ST_CAPACITY = 2u,
    ST_TIMEOUT = 4u,
};

// Iteration cap of every inter-block spin (decoupled look-back).  An
// iteration is one L2 round trip (~1 us at most), so the cap is well above
// any legal wait and far below a hang.
constexpr int SPIN_LIMIT = 1 << 22;

// 64-bit orientation of (o, a, b): > 0 for a counter-clockwise turn.
__device__ __forceinline__ long long cross3(int2 o, int2 a, int2 b)
{
    return (long long)(a.x - o.x) * (long long)(b.y - o.y) -
           (long long)(a.y - o.y) * (long long)(b.x - o.x);
}

// The same orientation in 32-bit arithmetic (NARROW = true), exact when
// every coordinate difference is below 2^14 in magnitude, so that each
// product is below 2^28: the batched and single-launch kernels take sets of
// side p <= 16384, whose chain points differ by at most p - 1 in x and in y
// (lower chains (x, y), upper chains mirrored to (x, -y), never mixed).
template <bool NARROW>
__device__ __forceinline__ long long orient(int2 o, int2 a, int2 b)
{
    if constexpr (NARROW)
        return (long long)((a.x - o.x) * (b.y - o.y) - (a.y - o.y) * (b.x - o.x));
    else
        return cross3(o, a, b);
}

// Launch with programmatic dependent launch allowed: the grid may be
// scheduled while the previous kernel of the stream finishes, which hides the
// launch latency between the dependent kernels of the path.  Every kernel
// launched this way calls pdl_wait() before it touches global memory, so it
// still sees (and does not overwrite) anything its predecessor works on, and
// pdl_trigger() to let its own successor be scheduled.
template <typename... KArgs, typename... Args>
inline cudaError_t launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                         cudaStream_t s, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// launch() for a grid of thread-block clusters of `cluster` CTAs along x
// (the grid's x extent a multiple of it).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_cluster(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                  cudaStream_t s, int cluster, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    at[1].id = cudaLaunchAttributeClusterDimension;
    at[1].val.clusterDim.x = (unsigned)cluster;
    at[1].val.clusterDim.y = 1;
    at[1].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Waits until the previous grid of the stream has completed and its memory
// operations are visible (a no-op for a grid launched without the attribute).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the next grid of the stream be scheduled once every CTA of this grid
// has issued it (or exited).
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;"); }

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

// ---- frame of Algorithm 1 ----
// The columns of L run along x (tr = 0) or along y (tr = 1, the sweep along
// the shorter side of the bounding box); a point (x, y) with u = tr ? y : x,
// v = tr ? x : y lands in column u - c0 (0-based, < nc) at row v - r0 + 1
// (1-based, <= nr).  The square of side p of Section 2.1 is {1, 1, p, p, 0}.
// pk = 1: the points are packed 16-bit pairs, one 32-bit word per point,
// (x - 1) | (y - 1) << 16, in the square of side p <= 65536.
struct Frame {
    int c0, r0;
    int nc, nr;
    int tr;
    int pk;
};
inline Frame square_frame(int p) { return Frame{1, 1, p, p, 0, 0}; }
inline Frame square_frame_u16(int p) { return Frame{1, 1, p, p, 0, 1}; }

// Column c (0-based) and row index rr = row - 1 of point (x, y); unsigned
// arithmetic, so that any out-of-frame point gives c >= nc or rr >= nr.
// FM: 0 the square (offsets 1, known at compile time), 1 a translated frame,
// 2 a translated and transposed frame, 3 the square with packed 16-bit points.
template <int FM>
__device__ __forceinline__ void frame_map(const Frame &f, int x, int y, uint32_t &c, uint32_t &rr)
{
    const int u = FM == 2 ? y : x, v = FM == 2 ? x : y;
    c = (uint32_t)u - (uint32_t)(FM == 0 || FM == 3 ? 1 : f.c0);
    rr = (uint32_t)v - (uint32_t)(FM == 0 || FM == 3 ? 1 : f.r0);
}
inline int frame_mode(const Frame &f)
{
    return f.pk ? 3 : f.tr ? 2 : (f.c0 == 1 && f.r0 == 1 ? 0 : 1);
}

// ---- reduction (reduce.cu) ----
struct ReducePlan {
    int mode;      // 0: private copies, 1: filtered global L, 2: global L only
    int cluster;   // mode 1: CTAs per cluster of the filter warm-up (1, 2, 4 or 8)
    int grid;      // CTAs of the main reduction kernel
    int threads;   // threads per CTA of the main reduction kernel
    int copies;    // mode 0: number of int2[p] partial arrays
    int shift;     // modes 1-2: row-bin shift of the filter
    size_t smem;   // dynamic shared memory per CTA
};
// Plan for nc columns of nr rows (the square: nc = nr = p).
int reduce_plan(int64_t n, int nc, int nr, ReducePlan *plan);
inline int reduce_plan(int64_t n, int p, ReducePlan *plan) { return reduce_plan(n, p, p, plan); }
size_t reduce_partials_bytes(const ReducePlan &plan, int nc);
// Mode 0 writes plan.copies packed uint32[p] partial arrays to `scratch`
// (((lo-1) << 16) | (hi-1), 0xFFFF0000 when empty); modes 1-2 write the final
// L (mode 1 keeps its global filter in `scratch`).
// zero/nzero: words (the chain look-back state) that the last kernel before
// the main pass clears, or nullptr.  ev0/ev1: events recorded right before
// and after the main reduction kernel (the dominant one), or nullptr.
// prefilled: the culling step has already written L (modes 1-2) and the
// filter (mode 1, at the start of `scratch`), so the warm-up is skipped.
cudaError_t reduce_launch(const ReducePlan &plan, const int32_t *pts, int64_t n, const Frame &f,
                          void *scratch, int32_t *L, unsigned *status, cudaStream_t s,
                          unsigned long long *zero = nullptr, int nzero = 0,
                          cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr,
                          bool prefilled = false);
int reduce_kernel_count(const ReducePlan &plan);
// The part of reduce_launch before the main pass: mode 1 the filter warm-up
// and merge (L = (p+1, -1), G ready), mode 2 the fill of L; both clear
// zero/nzero.  Mode 0 launches nothing.
cudaError_t reduce_warm_launch(const ReducePlan &plan, const int32_t *pts, int64_t n,
                               const Frame &f, void *scratch, int32_t *L, cudaStream_t s,
                               unsigned long long *zero, int nzero);
// L = column-wise merge of `copies` packed partial arrays (folded with the
// culling start array Linit when given).
cudaError_t reduce_merge_launch(const void *partials, int copies, int nc, int nr, int32_t *L,
                                cudaStream_t s, unsigned long long *zero = nullptr, int nzero = 0,
                                const int32_t *Linit = nullptr);
// Filter shift of the filtered form: (p - 1) >> shift <= 255.
int reduce_filter_shift(int p);

// ---- chain (chain.cu) ----
int chain_tiles(int p);
size_t chain_state_bytes(int p);
// Chains of L.  With cand != nullptr also runs the exact hull pre-filter on
// each 1024-column tile and writes its survivors in the hull layout (so that
// hull_final_launch can follow directly).  state: chain_state_bytes(p),
// zeroed here unless state_zeroed.
// With cand, lower, upper, counts and mask may all be nullptr: the step then
// writes only the candidates (no look-back).  NARROW orientation tests are
// taken when p and nr are at most 16384.
// Linit != nullptr: chains of a culled reduction (see k_chain); counts[0] and
// counts[1] then differ.  nr: rows of the frame (empty columns hold
// (nr + 1, -1)); 0 means p.
cudaError_t chain_launch(const int32_t *L, int p, int32_t *lower, int32_t *upper, int32_t *counts,
                         uint32_t *mask, void *state, bool state_zeroed, int2 *cand, int *ccnt,
                         unsigned *status, cudaStream_t s, const int32_t *Linit = nullptr,
                         int nr = 0);

// ---- hull (hull.cu) ----
struct HullLayout {
    int nblk;  // runs of 1024 chain points (or chain tiles) per chain
    bool refilter;  // survivors filtered a second time before the final CTA
    size_t cand, ccnt, gA, gB, gF, gix, ccnt2, counts2, state2, end;
};
HullLayout hull_layout(int p);
size_t hull_ws_bytes(int p);
// Filter + final CTA from the chains.
cudaError_t hull_launch(const int32_t *lower, const int32_t *upper, const int32_t *counts, int p,
                        int32_t *hull, int32_t *hull_count, void *ws, unsigned *status,
                        cudaStream_t s);
// Final CTA only, from survivors already in the hull workspace.  narrow:
// the survivors come from a frame whose columns and rows are at most 16384
// (32-bit orientation tests are exact there).
cudaError_t hull_final_launch(const HullLayout &h, void *ws, int32_t *hull, int32_t *hull_count,
                              cudaStream_t s, bool narrow = false);

// ---- batched (batched.cu) ----
constexpr int BATCH_MAX_P = 16384;  // largest p of a set in a batch
struct BatchPlanInfo {
    int B, nitems, grid;
    long long part_words;
    int fold;  // threads of a CTA that fold while the others finish (0: the whole CTA does both)
};
// The CTA splits the batched hull kernel is built for (threads that fold).
inline bool batch_fold_ok(int fold)
{
    return fold == 0 || fold == 384 || fold == 512 || fold == 640 || fold == 768 || fold == 896;
}
size_t batch_smem();
// One set of n points and side p in one launch (k_small): the number of CTAs
// it takes, or 0 when the set is too large for that path.
int small_ctas(int64_t n, int p);
size_t small_ws_bytes(int G, int p);
// ticket: a zero word that no other launch uses meanwhile (left zero);
// L_out optional; ev0/ev1 recorded around the launch when given.
cudaError_t small_launch(const int32_t *pts, int64_t n, int p, int G, void *ws, unsigned *ticket,
                         int32_t *L_out, int32_t *hull, int32_t *hull_count, unsigned *status,
                         cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1);
int batch_sizes(int B, const int64_t *off, const int32_t *ps, int chunk_mult, size_t *ws_bytes,
                BatchPlanInfo *info);
int batch_prepare(int B, const int64_t *off, const int32_t *ps, int chunk_mult, void *ws,
                  size_t ws_bytes, cudaStream_t s, BatchPlanInfo *info);
// L_out == nullptr: hulls into hull_out; otherwise each set's L into
// L_out[L_offsets[s] ...] and no hull.
int batch_launch(const int32_t *pts, int2 *hull_out, const int64_t *hull_offsets, int *hull_counts,
                 int2 *L_out, const int64_t *L_offsets, void *ws, size_t ws_bytes,
                 const BatchPlanInfo &info, unsigned *status, cudaStream_t s);
int chain_batched_launch(const int2 *L, const int64_t *L_offsets, const int *ps, int B, int2 *lower,
                         int2 *upper, int *counts, cudaStream_t s);

// ---- MLP (mlp.cu) ----
// C[M x N] = epi(A[M x K] B[K x N] (+ bias)) (+ beta * C); element (r, c) of A
// at A[r * a_sr + c * a_sc], likewise B.  epi: 0 plain, 1 ReLU, 2 times
// (mask[r * ldm + c] > 0).
cudaError_t gemm_launch(const float *A, long long a_sr, long long a_sc, const float *B, long long b_sr,
                        long long b_sc, float *C, long long ldc, int M, int N, int K,
                        const float *bias, int epi, const float *mask, long long ldm, float beta,
                        cudaStream_t s);
cudaError_t colsum_launch(const float *X, long long ld, int M, int N, float *out, cudaStream_t s);
cudaError_t tanh_mse_launch(const float *Y, const float *T, int count, float *dY, float *loss,
                            cudaStream_t s);
cudaError_t adam_launch(float *w, const float *g, float *m, float *v, long long n, float lr_t,
                        float b1, float b2, float eps, cudaStream_t s);

// ---- learned culling (cull.cu) ----
size_t cull_ws_bytes(int p);
// Sample histogram -> network (params != nullptr; else the K sector centres)
// -> extreme sample points -> culling polygon -> Linit for every column.  L
// and G (filter words) are written too when given (G_warm: G holds the
// warm-up filter, which is tightened rather than replaced); zero/nzero as in
// reduce_launch.  features, y_out, dirs_out, poly_out, poly_count, ext_out,
// chosen are optional diagnostic outputs (of the polygon used: the network's
// or the sector centres', whichever has the larger area).
cudaError_t cull_launch(const int32_t *pts, int64_t n, int p, const float *params, void *ws,
                        int32_t *Linit, int32_t *L, uint16_t *G, bool G_warm, int shift,
                        unsigned long long *zero, int nzero, float *features, float *y_out,
                        float *dirs_out, int32_t *poly_out, int32_t *poly_count, int64_t *ext_out,
                        int32_t *chosen, cudaStream_t s);
int cull_kernel_count(bool net);
// *culled += the points strictly inside the culling polygon of Linit
// (Linit.lo <= y <= Linit.hi in their column); no launch when n = 0.
cudaError_t cull_count_launch(const int32_t *pts, int64_t n, int p, const int32_t *Linit,
                              unsigned long long *culled, cudaStream_t s);

// ---- bounding box and frames (box.cu) ----
int bbox_parts();
// box[4] = (xmin, xmax, ymin, ymax) of pts; ws: bbox_parts() * 16 bytes.
cudaError_t bbox_launch(const int32_t *pts, int64_t n, int32_t *box, void *ws, cudaStream_t s);
// Hull from frame coordinates back to the input's (see k_unframe).
cudaError_t unframe_launch(const int32_t *hull_in, const int32_t *count_in, const Frame &f,
                           int32_t *hull_out, int32_t *count_out, cudaStream_t s);

// ---- Lemma 1 polyline and Melkman's hull (polyline.cu) ----
size_t polyline_state_bytes(int p);
// poly: the Lemma 1 polyline of L (columns of nr rows; 0 means p), *count
// its vertices.  state: polyline_state_bytes(p), zeroed here unless
// state_zeroed.  filter: drop the vertices the in-tile hull pre-filter rules
// out (still a simple polyline with every hull vertex).
cudaError_t polyline_launch(const int32_t *L, int p, int nr, int32_t *poly, int32_t *count,
                            void *state, bool state_zeroed, unsigned *status, cudaStream_t s,
                            bool filter = false);
long long lattice_hull_bound(int p);
size_t melkman_ws_bytes(int p);  // 0 when the deque fits in shared memory
cudaError_t melkman_launch(const int32_t *poly, const int32_t *count, int p, int32_t *hull,
                           int32_t *hull_count, void *ws, unsigned *status, cudaStream_t s);

// ---- sparse regime: w-ary tree of bit words (sparse.cu) ----
constexpr int TREE_MAX_LEVELS = 7;  // 32^6 >= 2^30
struct TreeLevels {
    int levels;
    uint32_t *M[TREE_MAX_LEVELS];
};
struct SparseLayout {
    int levels, chain_cap, state_words;
    size_t words[TREE_MAX_LEVELS], list_cap[TREE_MAX_LEVELS];
    int state_off[TREE_MAX_LEVELS];
    size_t Lz, M[TREE_MAX_LEVELS], persistent_end;  // zero-filled between calls
    size_t list[2], cnt, state, lower, upper, counts, hull, end;
};
// Levels of the tree for side p (words[k] = words of level k, optional).
int tree_levels(int p, size_t *words);
SparseLayout sparse_layout(int64_t n, int p);
cudaError_t sparse_launch(const SparseLayout &L, const int32_t *pts, int64_t n, int p, void *ws,
                          int32_t *lower, int32_t *upper, int32_t *counts, int32_t *hull,
                          int32_t *hull_count, unsigned *status, cudaStream_t s, cudaEvent_t ev0,
                          cudaEvent_t ev1);
int sparse_kernel_count(const SparseLayout &L);

// ---- second scan along y (rows.cu) ----
// R (int32[p][2]) = Algorithm 1 along y over the rx points of L; an entry
// of L that no in-range input can produce is skipped as CH_ERR_RANGE.
cudaError_t rows_launch(const int32_t *L, int p, int32_t *R, unsigned *status, cudaStream_t s);

// ---- api.cu ----
// The status word of stream s on the current device (nullptr on failure).
unsigned *device_status_ptr(cudaStream_t s);
// A ticket word of stream s on the current device for the single-launch path
// (zero between calls), or nullptr (also for the streams beyond the ones with
// words of their own, whose calls take the multi-kernel path).
unsigned *device_ticket_ptr(cudaStream_t s);
int sm_count();

}  // namespace ch
