// C ABI of libch.so (declared in include/ch.h): argument checks, workspace
// layouts, the per-stream status words and launch sequencing.  No entry point
// allocates device memory; every launch goes to the caller's stream.
#include <cmath>
#include <map>
#include <mutex>

#include "ch_internal.cuh"

// Sticky error words written by the kernels (ST_* bits), one per stream: a
// call's kernels record into the word of the stream the call was made on, so
// an error is reported to the caller of ch_sync_status on that stream only.
// Slots are handed out to streams in order of first use and never recycled;
// streams beyond the STATUS_SLOTS-th distinct one share the last word.
constexpr int STATUS_SLOTS = 1024;
__device__ unsigned g_ch_status[STATUS_SLOTS + 1];
// ch_sync_status moves a stream's word here (atomic exchange with 0, on that
// stream) and reads it back with a copy ordered on the same stream.
__device__ unsigned g_ch_taken[STATUS_SLOTS + 1];
// Ticket of the single-launch path, one per stream slot: zero between calls
// (the launch that counts it up resets it), so calls on one stream, which
// never overlap, never share it.  The shared overflow slot has none.
__device__ unsigned g_ch_ticket[STATUS_SLOTS];

namespace ch {

namespace {
constexpr int MAX_DEV = 64;
std::mutex g_mu;
unsigned *g_status_base[MAX_DEV] = {};
unsigned *g_taken_base[MAX_DEV] = {};
unsigned *g_ticket_base[MAX_DEV] = {};
std::map<cudaStream_t, int> g_slot_of[MAX_DEV];
int g_sms[MAX_DEV] = {};

inline bool aligned8(const void *p) { return ((uintptr_t)p & 7) == 0; }
// Workspaces start on a 256-byte boundary (as cudaMalloc returns them): the
// kernels put 16-byte vectors and 8-byte words at offsets inside them.
inline bool ws_aligned(const void *w) { return ((uintptr_t)w & 255) == 0; }

// ch_trace_set ring of event pairs around the reduction kernel.
std::mutex g_trace_mu;
cudaEvent_t g_trace[2 * 1024];
int g_trace_n = 0, g_trace_next = 0;

// The next traced event pair, or (nullptr, nullptr) when tracing is off.
void next_trace(cudaEvent_t *e0, cudaEvent_t *e1)
{
    std::lock_guard<std::mutex> g(g_trace_mu);
    *e0 = *e1 = nullptr;
    if (g_trace_n > 0) {
        const int i = g_trace_next;
        g_trace_next = (g_trace_next + 1) % g_trace_n;
        *e0 = g_trace[2 * i];
        *e1 = g_trace[2 * i + 1];
    }
}
inline int cuda_rc(cudaError_t e) { return e == cudaSuccess ? CH_OK : CH_ERR_CUDA; }

// Slot index of stream s on the current device (-1 on failure); the device
// addresses of both word arrays are resolved on the device's first use.
int status_slot(cudaStream_t s, unsigned **word, unsigned **taken)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV)
        return -1;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_status_base[dev]) {
        void *a = nullptr, *b = nullptr, *c = nullptr;
        if (cudaGetSymbolAddress(&a, g_ch_status) != cudaSuccess ||
            cudaGetSymbolAddress(&b, g_ch_taken) != cudaSuccess ||
            cudaGetSymbolAddress(&c, g_ch_ticket) != cudaSuccess)
            return -1;
        g_status_base[dev] = reinterpret_cast<unsigned *>(a);
        g_taken_base[dev] = reinterpret_cast<unsigned *>(b);
        g_ticket_base[dev] = reinterpret_cast<unsigned *>(c);
    }
    auto &m = g_slot_of[dev];
    auto it = m.find(s);
    int k;
    if (it != m.end()) {
        k = it->second;
    } else {
        k = std::min((int)m.size(), STATUS_SLOTS);
        m.emplace(s, k);
    }
    if (word)
        *word = g_status_base[dev] + k;
    if (taken)
        *taken = g_taken_base[dev] + k;
    return k;
}

// Moves the stream's status word to its read-back word (stream-ordered).
__global__ void k_status_take(unsigned *word, unsigned *taken) { *taken = atomicExch(word, 0u); }
}  // namespace

unsigned *device_status_ptr(cudaStream_t s)
{
    unsigned *w = nullptr;
    return status_slot(s, &w, nullptr) < 0 ? nullptr : w;
}

unsigned *device_ticket_ptr(cudaStream_t s)
{
    const int k = status_slot(s, nullptr, nullptr);
    if (k < 0 || k >= STATUS_SLOTS)
        return nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return nullptr;
    std::lock_guard<std::mutex> g(g_mu);
    return g_ticket_base[dev] + k;
}

int sm_count()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEV)
        return 0;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_sms[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return 0;
        g_sms[dev] = v;
    }
    return g_sms[dev];
}

namespace {

// Workspace of the whole path: chain look-back state, partial arrays (or L
// for p > 65536), optional chain outputs, hull scratch.
struct PathWs {
    ReducePlan plan;
    size_t state, part, L, lower, upper, counts, hull, end;
};

// nc columns of nr rows (the square: nc = nr = p).
int path_layout(int64_t n, int nc, int nr, PathWs *w)
{
    int rc = reduce_plan(n, nc, nr, &w->plan);
    if (rc != CH_OK)
        return rc;
    WsLayout l;
    w->state = l.take(chain_state_bytes(nc));
    w->part = l.take(reduce_partials_bytes(w->plan, nc));
    w->L = l.take((size_t)nc * 8);
    w->lower = l.take((size_t)nc * 8);
    w->upper = l.take((size_t)nc * 8);
    w->counts = l.take(8);
    w->hull = l.take(hull_ws_bytes(nc));
    w->end = l.off;
    return CH_OK;
}

int path_layout(int64_t n, int p, PathWs *w) { return path_layout(n, p, p, w); }

// Workspace of ch_convex_hull: the multi-kernel layout, or the single-launch
// path's rows and scratch, whichever is larger (the call may take either).
size_t plain_ws_bytes(const PathWs &w, int64_t n, int p)
{
    const int G = small_ctas(n, p);
    return G > 0 ? std::max(w.end, small_ws_bytes(G, p)) : w.end;
}

// The frame of a bounding box (xmin, xmax, ymin, ymax): columns along the
// shorter side; CH_ERR_ARG for an empty box or a side above CH_MAX_P.
int box_frame(const int32_t *box, Frame *f)
{
    const int64_t p = (int64_t)box[1] - box[0] + 1, q = (int64_t)box[3] - box[2] + 1;
    if (p < 1 || q < 1 || p > CH_MAX_P || q > CH_MAX_P)
        return CH_ERR_ARG;
    f->tr = q < p;
    f->pk = 0;
    f->c0 = f->tr ? box[2] : box[0];
    f->r0 = f->tr ? box[0] : box[2];
    f->nc = (int)std::min(p, q);
    f->nr = (int)std::max(p, q);
    return CH_OK;
}

int check_np(int64_t n, int32_t p)
{
    if (n < 0 || p < 1 || p > CH_MAX_P)
        return CH_ERR_ARG;
    return CH_OK;
}

}  // namespace
}  // namespace ch

using namespace ch;

extern "C" {

const char *ch_strerror(int code)
{
    switch (code) {
    case CH_OK: return "ok";
    case CH_ERR_ARG: return "invalid argument";
    case CH_ERR_RANGE: return "a point lies outside [1,p]^2";
    case CH_ERR_CAPACITY: return "output or workspace capacity exceeded";
    case CH_ERR_TIMEOUT: return "a bounded inter-block wait ran out";
    case CH_ERR_CUDA: return "CUDA runtime error";
    case CH_ERR_WORKSPACE: return "workspace smaller than the size query";
    default: return "unknown status";
    }
}

int ch_version(void) { return (1 << 16) | 0; }

int ch_sync_status(ch_stream_t stream)
{
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned *word = nullptr, *taken = nullptr;
    if (status_slot(s, &word, &taken) < 0)
        return CH_ERR_CUDA;
    // exchange and read-back are ordered after the stream's earlier work and
    // touch only this stream's word; other streams keep running
    k_status_take<<<1, 1, 0, s>>>(word, taken);
    unsigned v = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&v, taken, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CH_ERR_CUDA;
    if (v & ST_RANGE)
        return CH_ERR_RANGE;
    if (v & ST_CAPACITY)
        return CH_ERR_CAPACITY;
    if (v & ST_TIMEOUT)
        return CH_ERR_TIMEOUT;
    return CH_OK;
}

int ch_clear_status(ch_stream_t stream)
{
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned *st = device_status_ptr(s);
    if (!st)
        return CH_ERR_CUDA;
    return cuda_rc(cudaMemsetAsync(st, 0, sizeof(unsigned), s));
}

int ch_trace_set(void *const *events, int npairs)
{
    if (npairs < 0 || npairs > 1024 || (npairs > 0 && !events))
        return CH_ERR_ARG;
    std::lock_guard<std::mutex> g(g_trace_mu);
    for (int i = 0; i < 2 * npairs; ++i)
        g_trace[i] = reinterpret_cast<cudaEvent_t>(events[i]);
    g_trace_n = npairs;
    g_trace_next = 0;
    return CH_OK;
}

int ch_plan_info(int64_t n, int32_t p, int32_t *form, int32_t *kernels)
{
    if (check_np(n, p) != CH_OK)
        return CH_ERR_ARG;
    ReducePlan pl;
    int rc = reduce_plan(n, p, &pl);
    if (rc != CH_OK)
        return rc;
    if (small_ctas(n, p) > 0) {  // the whole path in one launch
        if (form)
            *form = 3;
        if (kernels)
            *kernels = 1;
        return CH_OK;
    }
    if (form)
        *form = pl.mode;
    if (kernels)  // reduction (+ merge of private copies), chain, (second filter pass), final hull
        *kernels = reduce_kernel_count(pl) + (pl.mode == 0 ? 1 : 0) + 2 +
                   (hull_layout(p).refilter ? 2 : 0);
    return CH_OK;
}

int ch_reduce_workspace_size(int64_t n, int32_t p, size_t *bytes)
{
    if (!bytes || check_np(n, p) != CH_OK)
        return CH_ERR_ARG;
    ReducePlan pl;
    int rc = reduce_plan(n, p, &pl);
    if (rc != CH_OK)
        return rc;
    WsLayout l;
    l.take(reduce_partials_bytes(pl, p));
    *bytes = l.off;
    return CH_OK;
}

int ch_reduce(const int32_t *pts, int64_t n, int32_t p, int32_t *L, void *workspace,
              size_t ws_bytes, ch_stream_t stream)
{
    if (check_np(n, p) != CH_OK || !L || (n > 0 && !pts) || !aligned8(pts) || !aligned8(L))
        return CH_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    ReducePlan pl;
    int rc = reduce_plan(n, p, &pl);
    if (rc != CH_OK)
        return rc;
    const size_t need = reduce_partials_bytes(pl, p);
    if (!ws_aligned(workspace))
        return CH_ERR_ARG;
    if (ws_bytes < need || (need > 0 && !workspace))
        return CH_ERR_WORKSPACE;
    unsigned *st = device_status_ptr(reinterpret_cast<cudaStream_t>(stream));
    if (!st)
        return CH_ERR_CUDA;
    void *part = workspace;
    cudaEvent_t ev0, ev1;
    next_trace(&ev0, &ev1);
    cudaError_t e = reduce_launch(pl, pts, n, square_frame(p), part, L, st, s, nullptr, 0, ev0, ev1);
    if (e == cudaSuccess && pl.mode == 0)
        e = reduce_merge_launch(part, pl.copies, p, p, L, s);
    return cuda_rc(e);
}

int ch_chain_workspace_size(int32_t p, size_t *bytes)
{
    if (!bytes || p < 1 || p > CH_MAX_P)
        return CH_ERR_ARG;
    WsLayout l;
    l.take(chain_state_bytes(p));
    *bytes = l.off;
    return CH_OK;
}

int ch_chain(const int32_t *L, int32_t p, int32_t *lower, int32_t *upper, int32_t *counts,
             uint32_t *mask, void *workspace, size_t ws_bytes, ch_stream_t stream)
{
    if (p < 1 || p > CH_MAX_P || !L || !lower || !upper || !counts || !aligned8(L) ||
        !aligned8(lower) || !aligned8(upper))
        return CH_ERR_ARG;
    size_t need = 0;
    ch_chain_workspace_size(p, &need);
    if (!ws_aligned(workspace))
        return CH_ERR_ARG;
    if (ws_bytes < need || !workspace)
        return CH_ERR_WORKSPACE;
    unsigned *st = device_status_ptr(reinterpret_cast<cudaStream_t>(stream));
    if (!st)
        return CH_ERR_CUDA;
    return cuda_rc(chain_launch(L, p, lower, upper, counts, mask, workspace, false, nullptr,
                                nullptr, st, reinterpret_cast<cudaStream_t>(stream)));
}

int ch_hull_workspace_size(int32_t p, size_t *bytes)
{
    if (!bytes || p < 1 || p > CH_MAX_P)
        return CH_ERR_ARG;
    *bytes = hull_ws_bytes(p);
    return CH_OK;
}

int ch_hull(const int32_t *lower, const int32_t *upper, const int32_t *counts, int32_t p,
            int32_t *hull, int32_t *hull_count, void *workspace, size_t ws_bytes,
            ch_stream_t stream)
{
    if (p < 1 || p > CH_MAX_P || !lower || !upper || !counts || !hull || !hull_count ||
        !aligned8(lower) || !aligned8(upper) || !aligned8(hull))
        return CH_ERR_ARG;
    if (!ws_aligned(workspace))
        return CH_ERR_ARG;
    if (ws_bytes < hull_ws_bytes(p) || !workspace)
        return CH_ERR_WORKSPACE;
    unsigned *st = device_status_ptr(reinterpret_cast<cudaStream_t>(stream));
    if (!st)
        return CH_ERR_CUDA;
    return cuda_rc(hull_launch(lower, upper, counts, p, hull, hull_count, workspace, st,
                               reinterpret_cast<cudaStream_t>(stream)));
}

int ch_convex_hull_workspace_size(int64_t n, int32_t p, size_t *bytes)
{
    if (!bytes || check_np(n, p) != CH_OK)
        return CH_ERR_ARG;
    PathWs w;
    int rc = path_layout(n, p, &w);
    if (rc != CH_OK)
        return rc;
    *bytes = plain_ws_bytes(w, n, p);
    return CH_OK;
}

}  // extern "C"

namespace ch {
namespace {
// The fused path over the square of side p; frame = square_frame(p) for
// int32 points, square_frame_u16(p) for packed 16-bit points.
int convex_hull_square(const int32_t *pts, int64_t n, int32_t p, const Frame &frame, int32_t *L,
                       int32_t *lower, int32_t *upper, int32_t *counts, int32_t *hull,
                       int32_t *hull_count, void *workspace, size_t ws_bytes, ch_stream_t stream)
{
    // the caller checks the alignment of pts for its point format
    if (check_np(n, p) != CH_OK || (n > 0 && !pts) || !hull || !hull_count || !aligned8(L) ||
        !aligned8(lower) || !aligned8(upper) || !aligned8(hull))
        return CH_ERR_ARG;
    PathWs w;
    int rc = path_layout(n, p, &w);
    if (rc != CH_OK)
        return rc;
    const bool int32_pts = frame_mode(frame) == 0;
    if (!ws_aligned(workspace))
        return CH_ERR_ARG;
    if (ws_bytes < (int32_pts ? plain_ws_bytes(w, n, p) : w.end) || !workspace)
        return CH_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned *st = device_status_ptr(s);
    if (!st)
        return CH_ERR_CUDA;
    // small problems without chain outputs: the whole path in one launch
    const int G = int32_pts && !lower && !upper && !counts ? small_ctas(n, p) : 0;
    unsigned *ticket = G > 0 ? device_ticket_ptr(s) : nullptr;
    if (ticket) {
        cudaEvent_t ev0, ev1;
        next_trace(&ev0, &ev1);
        return cuda_rc(small_launch(pts, n, p, G, workspace, ticket, L, hull, hull_count, st, s,
                                    ev0, ev1));
    }
    char *b = reinterpret_cast<char *>(workspace);
    if (!L && w.plan.mode != 0)
        L = reinterpret_cast<int32_t *>(b + w.L);  // the filtered forms write L directly
    if (lower || upper || counts) {  // else the chain step writes only the hull's candidates
        if (!lower)
            lower = reinterpret_cast<int32_t *>(b + w.lower);
        if (!upper)
            upper = reinterpret_cast<int32_t *>(b + w.upper);
        if (!counts)
            counts = reinterpret_cast<int32_t *>(b + w.counts);
    }
    void *part = b + w.part;
    cudaEvent_t ev0, ev1;
    next_trace(&ev0, &ev1);
    unsigned long long *zero = reinterpret_cast<unsigned long long *>(b + w.state);
    const int nzero = (int)(chain_state_bytes(p) / 8);
    // the look-back state is cleared by the last kernel before the chain step
    cudaError_t e = reduce_launch(w.plan, pts, n, frame, part, L, st, s,
                                  w.plan.mode == 0 ? nullptr : zero, nzero, ev0, ev1);
    if (e != cudaSuccess)
        return CH_ERR_CUDA;
    if (w.plan.mode == 0) {
        if (!L)
            L = reinterpret_cast<int32_t *>(b + w.L);
        e = reduce_merge_launch(part, w.plan.copies, p, p, L, s, zero, nzero);
        if (e != cudaSuccess)
            return CH_ERR_CUDA;
    }
    const HullLayout hl = hull_layout(p);
    char *hw = b + w.hull;
    e = chain_launch(L, p, lower, upper, counts, nullptr, b + w.state, true,
                     reinterpret_cast<int2 *>(hw + hl.cand), reinterpret_cast<int *>(hw + hl.ccnt),
                     st, s);
    if (e != cudaSuccess)
        return CH_ERR_CUDA;
    return cuda_rc(hull_final_launch(hl, hw, hull, hull_count, s, p <= 16384));
}
}  // namespace
}  // namespace ch

extern "C" {

int ch_convex_hull(const int32_t *pts, int64_t n, int32_t p, int32_t *L, int32_t *lower,
                   int32_t *upper, int32_t *counts, int32_t *hull, int32_t *hull_count,
                   void *workspace, size_t ws_bytes, ch_stream_t stream)
{
    if (!aligned8(pts))
        return CH_ERR_ARG;
    return convex_hull_square(pts, n, p, square_frame(p), L, lower, upper, counts, hull,
                              hull_count, workspace, ws_bytes, stream);
}

int ch_convex_hull_u16(const uint32_t *pts, int64_t n, int32_t p, int32_t *L, int32_t *lower,
                       int32_t *upper, int32_t *counts, int32_t *hull, int32_t *hull_count,
                       void *workspace, size_t ws_bytes, ch_stream_t stream)
{
    if (p > 65536 || ((uintptr_t)pts & 3))
        return CH_ERR_ARG;
    return convex_hull_square(reinterpret_cast<const int32_t *>(pts), n, p, square_frame_u16(p), L,
                              lower, upper, counts, hull, hull_count, workspace, ws_bytes, stream);
}

int ch_reduce_u16(const uint32_t *pts, int64_t n, int32_t p, int32_t *L, void *workspace,
                  size_t ws_bytes, ch_stream_t stream)
{
    if (check_np(n, p) != CH_OK || p > 65536 || !L || (n > 0 && !pts) || ((uintptr_t)pts & 3) ||
        !aligned8(L))
        return CH_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    ReducePlan pl;
    int rc = reduce_plan(n, p, &pl);
    if (rc != CH_OK)
        return rc;
    const size_t need = reduce_partials_bytes(pl, p);
    if (!ws_aligned(workspace))
        return CH_ERR_ARG;
    if (ws_bytes < need || (need > 0 && !workspace))
        return CH_ERR_WORKSPACE;
    unsigned *st = device_status_ptr(reinterpret_cast<cudaStream_t>(stream));
    if (!st)
        return CH_ERR_CUDA;
    cudaEvent_t ev0, ev1;
    next_trace(&ev0, &ev1);
    cudaError_t e = reduce_launch(pl, reinterpret_cast<const int32_t *>(pts), n,
                                  square_frame_u16(p), workspace, L, st, s, nullptr, 0, ev0, ev1);
    if (e == cudaSuccess && pl.mode == 0)
        e = reduce_merge_launch(workspace, pl.copies, p, p, L, s);
    return cuda_rc(e);
}

namespace {
std::mutex g_batch_mu;
std::map<const void *, BatchPlanInfo> g_batch_plans;  // workspace -> prepared plan

int check_batch(int32_t B, const int64_t *off, const int32_t *ps, int32_t chunk_mult)
{
    if (B < 0 || (B > 0 && (!off || !ps)) || chunk_mult < 1)
        return CH_ERR_ARG;
    if (B > 0 && off[0] < 0)
        return CH_ERR_ARG;
    for (int s = 0; s < B; ++s)
        if (off[s + 1] < off[s] || ps[s] < 1 || ps[s] > BATCH_MAX_P)
            return CH_ERR_ARG;
    return CH_OK;
}
}  // namespace

int ch_batched_workspace_size(int32_t B, const int64_t *host_offsets, const int32_t *host_ps,
                              int32_t chunk_mult, size_t *bytes)
{
    if (!bytes)
        return CH_ERR_ARG;
    int rc = check_batch(B, host_offsets, host_ps, chunk_mult);
    if (rc != CH_OK)
        return rc;
    return batch_sizes(B, host_offsets, host_ps, chunk_mult, bytes, nullptr);
}

int ch_batched_prepare_shape(int32_t B, const int64_t *host_offsets, const int32_t *host_ps,
                             int32_t chunk_mult, int32_t fold_threads, void *workspace,
                             size_t ws_bytes, ch_stream_t stream)
{
    int rc = check_batch(B, host_offsets, host_ps, chunk_mult);
    if (rc != CH_OK)
        return rc;
    if (!batch_fold_ok(fold_threads))
        return CH_ERR_ARG;
    if (!ws_aligned(workspace))
        return CH_ERR_ARG;
    if (!workspace)
        return CH_ERR_WORKSPACE;
    BatchPlanInfo info;
    rc = batch_prepare(B, host_offsets, host_ps, chunk_mult, workspace, ws_bytes,
                       reinterpret_cast<cudaStream_t>(stream), &info);
    if (rc != CH_OK)
        return rc;
    info.fold = fold_threads;
    std::lock_guard<std::mutex> g(g_batch_mu);
    g_batch_plans[workspace] = info;
    return CH_OK;
}

int ch_batched_prepare(int32_t B, const int64_t *host_offsets, const int32_t *host_ps,
                       int32_t chunk_mult, void *workspace, size_t ws_bytes, ch_stream_t stream)
{
    return ch_batched_prepare_shape(B, host_offsets, host_ps, chunk_mult, CH_BATCH_FOLD_DEFAULT,
                                    workspace, ws_bytes, stream);
}

int ch_hull_batched(const int32_t *pts, const int64_t *offsets, const int32_t *ps, int32_t B,
                    int32_t *hull_out, const int64_t *hull_offsets, int32_t *hull_counts,
                    void *workspace, size_t ws_bytes, ch_stream_t stream)
{
    (void)offsets;
    (void)ps;
    if (B < 0 || (B > 0 && (!pts || !hull_out || !hull_offsets || !hull_counts)) ||
        !aligned8(pts) || !aligned8(hull_out))
        return CH_ERR_ARG;
    if (B == 0)
        return CH_OK;
    BatchPlanInfo info;
    {
        std::lock_guard<std::mutex> g(g_batch_mu);
        auto it = g_batch_plans.find(workspace);
        if (it == g_batch_plans.end() || it->second.B != B)
            return CH_ERR_ARG;  // no plan prepared in this workspace for B sets
        info = it->second;
    }
    unsigned *st = device_status_ptr(reinterpret_cast<cudaStream_t>(stream));
    if (!st)
        return CH_ERR_CUDA;
    return batch_launch(pts, reinterpret_cast<int2 *>(hull_out), hull_offsets, hull_counts, nullptr,
                        nullptr, workspace, ws_bytes, info, st, reinterpret_cast<cudaStream_t>(stream));
}

int ch_reduce_batched(const int32_t *pts, const int64_t *offsets, const int32_t *ps, int32_t B,
                      int32_t *L_out, const int64_t *L_offsets, void *workspace, size_t ws_bytes,
                      ch_stream_t stream)
{
    (void)offsets;
    (void)ps;
    if (B < 0 || (B > 0 && (!pts || !L_out || !L_offsets)) || !aligned8(pts) || !aligned8(L_out))
        return CH_ERR_ARG;
    if (B == 0)
        return CH_OK;
    BatchPlanInfo info;
    {
        std::lock_guard<std::mutex> g(g_batch_mu);
        auto it = g_batch_plans.find(workspace);
        if (it == g_batch_plans.end() || it->second.B != B)
            return CH_ERR_ARG;  // no plan prepared in this workspace for B sets
        info = it->second;
    }
    unsigned *st = device_status_ptr(reinterpret_cast<cudaStream_t>(stream));
    if (!st)
        return CH_ERR_CUDA;
    return batch_launch(pts, nullptr, nullptr, nullptr, reinterpret_cast<int2 *>(L_out), L_offsets,
                        workspace, ws_bytes, info, st, reinterpret_cast<cudaStream_t>(stream));
}

int ch_chain_batched(const int32_t *L, const int64_t *L_offsets, const int32_t *ps, int32_t B,
                     int32_t *lower, int32_t *upper, int32_t *counts, ch_stream_t stream)
{
    if (B < 0 || (B > 0 && (!L || !L_offsets || !ps || !lower || !upper || !counts)) ||
        !aligned8(L) || !aligned8(lower) || !aligned8(upper))
        return CH_ERR_ARG;
    if (B == 0)
        return CH_OK;
    return chain_batched_launch(reinterpret_cast<const int2 *>(L), L_offsets, ps, B,
                                reinterpret_cast<int2 *>(lower), reinterpret_cast<int2 *>(upper),
                                counts, reinterpret_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------- MLP
namespace {
constexpr long long OFF_W1 = 0, OFF_B1 = OFF_W1 + (long long)CH_MLP_IN * CH_MLP_HID;
constexpr long long OFF_W2 = OFF_B1 + CH_MLP_HID, OFF_B2 = OFF_W2 + (long long)CH_MLP_HID * CH_MLP_HID;
constexpr long long OFF_W3 = OFF_B2 + CH_MLP_HID, OFF_B3 = OFF_W3 + (long long)CH_MLP_HID * CH_MLP_K;
static_assert(OFF_B3 + CH_MLP_K == CH_MLP_PARAMS, "parameter layout");
}  // namespace

int ch_mlp_forward(const float *params, const float *X, int32_t M, float *H1, float *H2, float *Y,
                   ch_stream_t stream)
{
    if (M < 0 || (M > 0 && (!params || !X || !H1 || !H2 || !Y)))
        return CH_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float *w = params;
    const int I = CH_MLP_IN, H = CH_MLP_HID, K = CH_MLP_K;
    cudaError_t e = gemm_launch(X, I, 1, w + OFF_W1, H, 1, H1, H, M, H, I, w + OFF_B1, 1, nullptr, 0,
                                0.f, s);
    if (e == cudaSuccess)
        e = gemm_launch(H1, H, 1, w + OFF_W2, H, 1, H2, H, M, H, H, w + OFF_B2, 1, nullptr, 0, 0.f, s);
    if (e == cudaSuccess)
        e = gemm_launch(H2, H, 1, w + OFF_W3, K, 1, Y, K, M, K, H, w + OFF_B3, 0, nullptr, 0, 0.f, s);
    return cuda_rc(e);
}

int ch_mlp_loss(const float *Y, const float *T, int32_t M, float *dY, float *loss,
                ch_stream_t stream)
{
    if (M < 0 || (M > 0 && (!Y || !T || !dY || !loss)))
        return CH_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), s);
    if (e == cudaSuccess && M > 0)
        e = tanh_mse_launch(Y, T, M * CH_MLP_K, dY, loss, s);
    return cuda_rc(e);
}

int ch_mlp_backward_workspace_size(int32_t M, size_t *bytes)
{
    if (!bytes || M < 0)
        return CH_ERR_ARG;
    *bytes = 2 * (size_t)M * CH_MLP_HID * sizeof(float);
    return CH_OK;
}

int ch_mlp_backward(const float *params, const float *X, const float *H1, const float *H2,
                    const float *dY, int32_t M, float *grads, void *workspace, size_t ws_bytes,
                    ch_stream_t stream)
{
    if (M < 1 || !params || !X || !H1 || !H2 || !dY || !grads)
        return CH_ERR_ARG;
    if (!ws_aligned(workspace))
        return CH_ERR_ARG;
    if (ws_bytes < 2 * (size_t)M * CH_MLP_HID * sizeof(float) || !workspace)
        return CH_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int I = CH_MLP_IN, H = CH_MLP_HID, K = CH_MLP_K;
    const float *w = params;
    float *g = grads;
    float *dH2 = reinterpret_cast<float *>(workspace), *dH1 = dH2 + (size_t)M * H;
    cudaError_t e = gemm_launch(H2, 1, H, dY, K, 1, g + OFF_W3, K, H, K, M, nullptr, 0, nullptr, 0,
                                0.f, s);  // dW3 = H2^T dY
    if (e == cudaSuccess)
        e = colsum_launch(dY, K, M, K, g + OFF_B3, s);
    if (e == cudaSuccess)  // dH2 = (dY W3^T) . [H2 > 0]
        e = gemm_launch(dY, K, 1, w + OFF_W3, 1, K, dH2, H, M, H, K, nullptr, 2, H2, H, 0.f, s);
    if (e == cudaSuccess)
        e = gemm_launch(H1, 1, H, dH2, H, 1, g + OFF_W2, H, H, H, M, nullptr, 0, nullptr, 0, 0.f, s);
    if (e == cudaSuccess)
        e = colsum_launch(dH2, H, M, H, g + OFF_B2, s);
    if (e == cudaSuccess)  // dH1 = (dH2 W2^T) . [H1 > 0]
        e = gemm_launch(dH2, H, 1, w + OFF_W2, 1, H, dH1, H, M, H, H, nullptr, 2, H1, H, 0.f, s);
    if (e == cudaSuccess)
        e = gemm_launch(X, 1, I, dH1, H, 1, g + OFF_W1, H, I, H, M, nullptr, 0, nullptr, 0, 0.f, s);
    if (e == cudaSuccess)
        e = colsum_launch(dH1, H, M, H, g + OFF_B1, s);
    return cuda_rc(e);
}

int ch_mlp_adam(float *params, const float *grads, float *m, float *v, int32_t step, float lr,
                float beta1, float beta2, float eps, ch_stream_t stream)
{
    if (!params || !grads || !m || !v || step < 1)
        return CH_ERR_ARG;
    const double c1 = 1.0 - std::pow((double)beta1, step), c2 = 1.0 - std::pow((double)beta2, step);
    const float lr_t = (float)(lr * std::sqrt(c2) / c1);
    return cuda_rc(adam_launch(params, grads, m, v, CH_MLP_PARAMS, lr_t, beta1, beta2, eps,
                               reinterpret_cast<cudaStream_t>(stream)));
}

// ---------------------------------------------------------------- learned culling
namespace {
struct LearnedWs {
    PathWs path;
    size_t cull, Linit, end;
};

int learned_layout(int64_t n, int p, LearnedWs *w)
{
    int rc = path_layout(n, p, &w->path);
    if (rc != CH_OK)
        return rc;
    WsLayout l;
    l.off = w->path.end;
    w->cull = l.take(cull_ws_bytes(p));
    w->Linit = l.take((size_t)p * 8);
    w->end = l.off;
    return CH_OK;
}
}  // namespace

int ch_cull_workspace_size(int32_t p, size_t *bytes)
{
    if (!bytes || p < 1 || p > CH_MAX_P)
        return CH_ERR_ARG;
    *bytes = cull_ws_bytes(p);
    return CH_OK;
}

int ch_cull_propose(const int32_t *pts, int64_t n, int32_t p, const float *params, int32_t *Linit,
                    float *features, float *net_out, float *dirs, int32_t *poly,
                    int32_t *poly_count, int64_t *extremes, int32_t *chosen, void *workspace,
                    size_t ws_bytes, ch_stream_t stream)
{
    if (check_np(n, p) != CH_OK || (n > 0 && !pts) || !Linit || !aligned8(pts) ||
        !aligned8(Linit) || !aligned8(poly))
        return CH_ERR_ARG;
    if (!ws_aligned(workspace))
        return CH_ERR_ARG;
    if (ws_bytes < cull_ws_bytes(p) || !workspace)
        return CH_ERR_WORKSPACE;
    return cuda_rc(cull_launch(pts, n, p, params, workspace, Linit, nullptr, nullptr, false, 0,
                               nullptr, 0, features, net_out, dirs, poly, poly_count, extremes,
                               chosen,
                               reinterpret_cast<cudaStream_t>(stream)));
}

int ch_hull_learned_workspace_size(int64_t n, int32_t p, size_t *bytes)
{
    if (!bytes || check_np(n, p) != CH_OK)
        return CH_ERR_ARG;
    LearnedWs w;
    int rc = learned_layout(n, p, &w);
    if (rc != CH_OK)
        return rc;
    *bytes = w.end;
    return CH_OK;
}

int ch_hull_learned_kernel_count(int64_t n, int32_t p, int32_t with_net, int32_t *kernels)
{
    if (!kernels || check_np(n, p) != CH_OK)
        return CH_ERR_ARG;
    ReducePlan pl;
    int rc = reduce_plan(n, p, &pl);
    if (rc != CH_OK)
        return rc;
    // warm-up (filtered forms), culling step, the reduction (+ merge of
    // private copies), chain, (second filter pass), final hull
    *kernels = reduce_kernel_count(pl) + cull_kernel_count(with_net != 0) +
               (pl.mode == 0 ? 1 : 0) + 2 + (hull_layout(p).refilter ? 2 : 0);
    return CH_OK;
}

int ch_hull_learned(const int32_t *pts, int64_t n, int32_t p, const float *params, int32_t *L,
                    int32_t *Linit, int32_t *lower, int32_t *upper, int32_t *counts, int32_t *hull,
                    int32_t *hull_count, ch_cull_stats *stats, void *workspace, size_t ws_bytes,
                    ch_stream_t stream)
{
    if (check_np(n, p) != CH_OK || (n > 0 && !pts) || !hull || !hull_count || !aligned8(pts) ||
        !aligned8(L) || !aligned8(Linit) || !aligned8(lower) || !aligned8(upper) ||
        !aligned8(hull) || !aligned8(stats))
        return CH_ERR_ARG;
    LearnedWs w;
    int rc = learned_layout(n, p, &w);
    if (rc != CH_OK)
        return rc;
    if (!ws_aligned(workspace))
        return CH_ERR_ARG;
    if (ws_bytes < w.end || !workspace)
        return CH_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned *st = device_status_ptr(s);
    if (!st)
        return CH_ERR_CUDA;
    char *b = reinterpret_cast<char *>(workspace);
    const PathWs &pw = w.path;
    if (!L)
        L = reinterpret_cast<int32_t *>(b + pw.L);
    if (!Linit)
        Linit = reinterpret_cast<int32_t *>(b + w.Linit);
    if (lower || upper || counts) {  // else the chain step writes only the hull's candidates
        if (!lower)
            lower = reinterpret_cast<int32_t *>(b + pw.lower);
        if (!upper)
            upper = reinterpret_cast<int32_t *>(b + pw.upper);
        if (!counts)
            counts = reinterpret_cast<int32_t *>(b + pw.counts);
    }
    void *part = b + pw.part;
    unsigned long long *zero = reinterpret_cast<unsigned long long *>(b + pw.state);
    const int nzero = (int)(chain_state_bytes(p) / 8);
    const int mode = pw.plan.mode;
    // the filtered forms warm their filter up as the plain path does (and
    // clear the chain's look-back state); the culling step then writes
    // Linit, the start of L (filtered forms) and tightens the filter with
    // the polygon (mode 1); in mode 0 it clears the look-back state itself
    cudaError_t e = reduce_warm_launch(pw.plan, pts, n, square_frame(p), part, L, s, zero, nzero);
    if (e == cudaSuccess && stats)
        e = cudaMemsetAsync(&stats->culled, 0, sizeof(stats->culled), s);
    if (e == cudaSuccess)
        e = cull_launch(pts, n, p, params, b + w.cull, Linit, mode != 0 ? L : nullptr,
                        mode == 1 ? reinterpret_cast<uint16_t *>(part) : nullptr, mode == 1,
                        pw.plan.shift, mode == 0 ? zero : nullptr, mode == 0 ? nzero : 0, nullptr,
                        nullptr, nullptr, nullptr, stats ? &stats->poly_vertices : nullptr,
                        nullptr, stats ? &stats->chosen : nullptr, s);
    if (e != cudaSuccess)
        return CH_ERR_CUDA;
    cudaEvent_t ev0, ev1;
    next_trace(&ev0, &ev1);
    e = reduce_launch(pw.plan, pts, n, square_frame(p), part, L, st, s, nullptr, 0, ev0, ev1, true);
    if (e == cudaSuccess && mode == 0)
        e = reduce_merge_launch(part, pw.plan.copies, p, p, L, s, nullptr, 0, Linit);
    if (e != cudaSuccess)
        return CH_ERR_CUDA;
    const HullLayout hl = hull_layout(p);
    char *hw = b + pw.hull;
    e = chain_launch(L, p, lower, upper, counts, nullptr, zero, true,
                     reinterpret_cast<int2 *>(hw + hl.cand), reinterpret_cast<int *>(hw + hl.ccnt),
                     st, s, Linit);
    if (e != cudaSuccess)
        return CH_ERR_CUDA;
    e = hull_final_launch(hl, hw, hull, hull_count, s, p <= 16384);
    if (e == cudaSuccess && stats)
        e = cull_count_launch(pts, n, p, Linit, reinterpret_cast<unsigned long long *>(&stats->culled),
                              s);
    return cuda_rc(e);
}

// ---------------------------------------------------------------- any integer points
int ch_bbox_workspace_size(size_t *bytes)
{
    if (!bytes)
        return CH_ERR_ARG;
    *bytes = (size_t)bbox_parts() * 16;
    return CH_OK;
}

int ch_bbox(const int32_t *pts, int64_t n, int32_t *box, void *workspace, size_t ws_bytes,
            ch_stream_t stream)
{
    if (n < 0 || (n > 0 && !pts) || !box || !aligned8(pts))
        return CH_ERR_ARG;
    if (!ws_aligned(workspace))
        return CH_ERR_ARG;
    if (ws_bytes < (size_t)bbox_parts() * 16 || !workspace)
        return CH_ERR_WORKSPACE;
    return cuda_rc(bbox_launch(pts, n, box, workspace, reinterpret_cast<cudaStream_t>(stream)));
}

namespace {
struct BoxWs {
    PathWs path;
    size_t hull, count, end;
};

int box_layout(int64_t n, const Frame &f, BoxWs *w)
{
    int rc = path_layout(n, f.nc, f.nr, &w->path);
    if (rc != CH_OK)
        return rc;
    WsLayout l;
    l.off = w->path.end;
    w->hull = l.take((size_t)(2 * f.nc + 2) * 8);
    w->count = l.take(8);
    w->end = l.off;
    return CH_OK;
}
}  // namespace

int ch_convex_hull_box_workspace_size(int64_t n, const int32_t *host_box, size_t *bytes)
{
    Frame f;
    if (!bytes || !host_box || n < 0 || box_frame(host_box, &f) != CH_OK)
        return CH_ERR_ARG;
    BoxWs w;
    int rc = box_layout(n, f, &w);
    if (rc != CH_OK)
        return rc;
    *bytes = w.end;
    return CH_OK;
}

int ch_convex_hull_box(const int32_t *pts, int64_t n, const int32_t *host_box, int32_t *hull,
                       int32_t *hull_count, void *workspace, size_t ws_bytes, ch_stream_t stream)
{
    Frame f;
    if (n < 0 || (n > 0 && !pts) || !host_box || !hull || !hull_count || !aligned8(pts) ||
        !aligned8(hull) || box_frame(host_box, &f) != CH_OK)
        return CH_ERR_ARG;
    BoxWs w;
    int rc = box_layout(n, f, &w);
    if (rc != CH_OK)
        return rc;
    if (!ws_aligned(workspace))
        return CH_ERR_ARG;
    if (ws_bytes < w.end || !workspace)
        return CH_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned *st = device_status_ptr(s);
    if (!st)
        return CH_ERR_CUDA;
    char *b = reinterpret_cast<char *>(workspace);
    const PathWs &pw = w.path;
    int32_t *L = reinterpret_cast<int32_t *>(b + pw.L);
    void *part = b + pw.part;
    unsigned long long *zero = reinterpret_cast<unsigned long long *>(b + pw.state);
    const int nzero = (int)(chain_state_bytes(f.nc) / 8);
    cudaEvent_t ev0, ev1;
    next_trace(&ev0, &ev1);
    cudaError_t e = reduce_launch(pw.plan, pts, n, f, part, L, st, s,
                                  pw.plan.mode == 0 ? nullptr : zero, nzero, ev0, ev1);
    if (e == cudaSuccess && pw.plan.mode == 0)
        e = reduce_merge_launch(part, pw.plan.copies, f.nc, f.nr, L, s, zero, nzero);
    if (e != cudaSuccess)
        return CH_ERR_CUDA;
    const HullLayout hl = hull_layout(f.nc);
    char *hw = b + pw.hull;
    // only the hull's candidates: no chain outputs
    e = chain_launch(L, f.nc, nullptr, nullptr, nullptr, nullptr, zero, true,
                     reinterpret_cast<int2 *>(hw + hl.cand), reinterpret_cast<int *>(hw + hl.ccnt),
                     st, s, nullptr, f.nr);
    if (e == cudaSuccess)
        e = hull_final_launch(hl, hw, reinterpret_cast<int32_t *>(b + w.hull),
                              reinterpret_cast<int32_t *>(b + w.count), s,
                              f.nc <= 16384 && f.nr <= 16384);
    if (e == cudaSuccess)
        e = unframe_launch(reinterpret_cast<int32_t *>(b + w.hull),
                           reinterpret_cast<int32_t *>(b + w.count), f, hull, hull_count, s);
    return cuda_rc(e);
}

int ch_convex_hull_host_workspace_size(int64_t n, int32_t p, size_t *bytes)
{
    if (!bytes || check_np(n, p) != CH_OK)
        return CH_ERR_ARG;
    PathWs w;
    int rc = path_layout(n, p, &w);
    if (rc != CH_OK)
        return rc;
    WsLayout l;
    l.take((size_t)n * 8);
    l.take((size_t)p * 16);
    l.take(8);
    l.take(plain_ws_bytes(w, n, p));
    *bytes = l.off;
    return CH_OK;
}

int ch_convex_hull_host(const int32_t *host_pts, int64_t n, int32_t p, int32_t *host_hull,
                        int32_t *host_hull_count, void *workspace, size_t ws_bytes,
                        ch_stream_t stream)
{
    if (check_np(n, p) != CH_OK || (n > 0 && !host_pts) || !host_hull || !host_hull_count)
        return CH_ERR_ARG;
    size_t need = 0;
    int rc = ch_convex_hull_host_workspace_size(n, p, &need);
    if (rc != CH_OK)
        return rc;
    if (!ws_aligned(workspace))
        return CH_ERR_ARG;
    if (ws_bytes < need || !workspace)
        return CH_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    WsLayout l;
    char *b = reinterpret_cast<char *>(workspace);
    int32_t *d_pts = reinterpret_cast<int32_t *>(b + l.take((size_t)n * 8));
    int32_t *d_hull = reinterpret_cast<int32_t *>(b + l.take((size_t)p * 16));
    int32_t *d_cnt = reinterpret_cast<int32_t *>(b + l.take(8));
    const size_t inner_off = l.take(0);
    void *inner = b + inner_off;
    const size_t inner_bytes = ws_bytes - inner_off;
    if (n > 0 && cudaMemcpyAsync(d_pts, host_pts, (size_t)n * 8, cudaMemcpyHostToDevice, s) !=
                     cudaSuccess)
        return CH_ERR_CUDA;
    rc = ch_convex_hull(d_pts, n, p, nullptr, nullptr, nullptr, nullptr, d_hull, d_cnt, inner,
                        inner_bytes, stream);
    if (rc != CH_OK)
        return rc;
    int32_t h = 0;
    if (cudaMemcpyAsync(&h, d_cnt, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CH_ERR_CUDA;
    if (h < 0 || h > 2 * p)
        return CH_ERR_CAPACITY;
    if (h > 0 && cudaMemcpyAsync(host_hull, d_hull, (size_t)h * 8, cudaMemcpyDeviceToHost, s) !=
                     cudaSuccess)
        return CH_ERR_CUDA;
    *host_hull_count = h;
    return ch_sync_status(stream);
}

// ---- Lemma 1 polyline and Melkman's hull ----

int ch_polyline_workspace_size(int32_t p, size_t *bytes)
{
    if (!bytes || p < 1 || p > CH_MAX_P)
        return CH_ERR_ARG;
    *bytes = polyline_state_bytes(p);
    return CH_OK;
}

int ch_polyline(const int32_t *L, int32_t p, int32_t *poly, int32_t *count, void *workspace,
                size_t ws_bytes, ch_stream_t stream)
{
    if (p < 1 || p > CH_MAX_P || !L || !poly || !count || !aligned8(L) || !aligned8(poly))
        return CH_ERR_ARG;
    if (!ws_aligned(workspace))
        return CH_ERR_ARG;
    if (ws_bytes < polyline_state_bytes(p) || !workspace)
        return CH_ERR_WORKSPACE;
    unsigned *st = device_status_ptr(reinterpret_cast<cudaStream_t>(stream));
    if (!st)
        return CH_ERR_CUDA;
    return cuda_rc(polyline_launch(L, p, p, poly, count, workspace, false, st,
                                   reinterpret_cast<cudaStream_t>(stream)));
}

int ch_hull_melkman_workspace_size(int32_t p, size_t *bytes)
{
    if (!bytes || p < 1 || p > CH_MAX_P)
        return CH_ERR_ARG;
    *bytes = melkman_ws_bytes(p);
    return CH_OK;
}

int ch_hull_melkman(const int32_t *poly, const int32_t *count, int32_t p, int32_t *hull,
                    int32_t *hull_count, void *workspace, size_t ws_bytes, ch_stream_t stream)
{
    if (p < 1 || p > CH_MAX_P || !poly || !count || !hull || !hull_count || !aligned8(poly) ||
        !aligned8(hull))
        return CH_ERR_ARG;
    const size_t need = melkman_ws_bytes(p);
    if (!ws_aligned(workspace))
        return CH_ERR_ARG;
    if (ws_bytes < need || (need && !workspace))
        return CH_ERR_WORKSPACE;
    unsigned *st = device_status_ptr(reinterpret_cast<cudaStream_t>(stream));
    if (!st)
        return CH_ERR_CUDA;
    return cuda_rc(melkman_launch(poly, count, p, hull, hull_count, workspace, st,
                                  reinterpret_cast<cudaStream_t>(stream)));
}

namespace {
struct MelkmanWs {
    ReducePlan plan;
    size_t state, part, L, poly, count, dq, end;
};
int melkman_layout(int64_t n, int p, MelkmanWs *w)
{
    int rc = reduce_plan(n, p, &w->plan);
    if (rc != CH_OK)
        return rc;
    WsLayout l;
    w->state = l.take(polyline_state_bytes(p));
    w->part = l.take(reduce_partials_bytes(w->plan, p));
    w->L = l.take((size_t)p * 8);
    w->poly = l.take((size_t)p * 16);
    w->count = l.take(8);
    w->dq = l.take(melkman_ws_bytes(p));
    w->end = l.off;
    return CH_OK;
}
}  // namespace

int ch_convex_hull_melkman_workspace_size(int64_t n, int32_t p, size_t *bytes)
{
    if (!bytes || check_np(n, p) != CH_OK)
        return CH_ERR_ARG;
    MelkmanWs w;
    const int rc = melkman_layout(n, p, &w);
    if (rc != CH_OK)
        return rc;
    *bytes = w.end;
    return CH_OK;
}

int ch_convex_hull_melkman(const int32_t *pts, int64_t n, int32_t p, int32_t *L, int32_t *poly,
                           int32_t *poly_count, int32_t *hull, int32_t *hull_count,
                           void *workspace, size_t ws_bytes, ch_stream_t stream)
{
    if (check_np(n, p) != CH_OK || (n > 0 && !pts) || !hull || !hull_count || !aligned8(pts) ||
        !aligned8(L) || !aligned8(poly) || !aligned8(hull))
        return CH_ERR_ARG;
    MelkmanWs w;
    int rc = melkman_layout(n, p, &w);
    if (rc != CH_OK)
        return rc;
    if (!ws_aligned(workspace))
        return CH_ERR_ARG;
    if (ws_bytes < w.end || !workspace)
        return CH_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned *st = device_status_ptr(s);
    if (!st)
        return CH_ERR_CUDA;
    char *b = reinterpret_cast<char *>(workspace);
    if (!L)
        L = reinterpret_cast<int32_t *>(b + w.L);
    if (!poly)
        poly = reinterpret_cast<int32_t *>(b + w.poly);
    if (!poly_count)
        poly_count = reinterpret_cast<int32_t *>(b + w.count);
    cudaEvent_t ev0, ev1;
    next_trace(&ev0, &ev1);
    unsigned long long *zero = reinterpret_cast<unsigned long long *>(b + w.state);
    const int nzero = (int)(polyline_state_bytes(p) / 8);
    cudaError_t e = reduce_launch(w.plan, pts, n, square_frame(p), b + w.part, L, st, s,
                                  w.plan.mode == 0 ? nullptr : zero, nzero, ev0, ev1);
    if (e == cudaSuccess && w.plan.mode == 0)
        e = reduce_merge_launch(b + w.part, w.plan.copies, p, p, L, s, zero, nzero);
    if (e == cudaSuccess)
        e = polyline_launch(L, p, p, poly, poly_count, zero, true, st, s, true);
    if (e == cudaSuccess)
        e = melkman_launch(poly, poly_count, p, hull, hull_count, b + w.dq, st, s);
    return cuda_rc(e);
}

// ---- sparse regime (p > n): the w-ary tree of bit words ----

int ch_sparse_workspace_size(int64_t n, int32_t p, size_t *bytes, size_t *persistent_bytes)
{
    if (!bytes || check_np(n, p) != CH_OK)
        return CH_ERR_ARG;
    const SparseLayout L = sparse_layout(n, p);
    *bytes = L.end;
    if (persistent_bytes)
        *persistent_bytes = L.persistent_end;
    return CH_OK;
}

int ch_sparse_kernel_count(int64_t n, int32_t p, int32_t *kernels)
{
    if (!kernels || check_np(n, p) != CH_OK)
        return CH_ERR_ARG;
    *kernels = sparse_kernel_count(sparse_layout(n, p));
    return CH_OK;
}

int ch_convex_hull_sparse(const int32_t *pts, int64_t n, int32_t p, int32_t *lower,
                          int32_t *upper, int32_t *counts, int32_t *hull, int32_t *hull_count,
                          void *workspace, size_t ws_bytes, ch_stream_t stream)
{
    if (check_np(n, p) != CH_OK || (n > 0 && !pts) || !hull || !hull_count || !aligned8(pts) ||
        !aligned8(lower) || !aligned8(upper) || !aligned8(hull))
        return CH_ERR_ARG;
    const SparseLayout L = sparse_layout(n, p);
    if (!ws_aligned(workspace))
        return CH_ERR_ARG;
    if (ws_bytes < L.end || !workspace)
        return CH_ERR_WORKSPACE;
    unsigned *st = device_status_ptr(reinterpret_cast<cudaStream_t>(stream));
    if (!st)
        return CH_ERR_CUDA;
    char *b = reinterpret_cast<char *>(workspace);
    if (!lower)
        lower = reinterpret_cast<int32_t *>(b + L.lower);
    if (!upper)
        upper = reinterpret_cast<int32_t *>(b + L.upper);
    if (!counts)
        counts = reinterpret_cast<int32_t *>(b + L.counts);
    cudaEvent_t ev0, ev1;
    next_trace(&ev0, &ev1);
    return cuda_rc(sparse_launch(L, pts, n, p, workspace, lower, upper, counts, hull, hull_count,
                                 st, reinterpret_cast<cudaStream_t>(stream), ev0, ev1));
}

// ---- the second scan along y (rx -> rxy) ----

int ch_reduce_rows(const int32_t *L, int32_t p, int32_t *R, ch_stream_t stream)
{
    if (p < 1 || p > CH_MAX_P || !L || !R || !aligned8(L) || !aligned8(R))
        return CH_ERR_ARG;
    unsigned *st = device_status_ptr(reinterpret_cast<cudaStream_t>(stream));
    if (!st)
        return CH_ERR_CUDA;
    return cuda_rc(rows_launch(L, p, R, st, reinterpret_cast<cudaStream_t>(stream)));
}

namespace {
struct RxyWs {
    PathWs path;
    size_t R, hull_t, count_t, end;
};
int rxy_layout(int64_t n, int p, RxyWs *w)
{
    int rc = path_layout(n, p, &w->path);
    if (rc != CH_OK)
        return rc;
    WsLayout l;
    l.off = w->path.end;
    w->R = l.take((size_t)p * 8);
    w->hull_t = l.take((size_t)p * 16);
    w->count_t = l.take(8);
    w->end = l.off;
    return CH_OK;
}
}  // namespace

int ch_convex_hull_rxy_workspace_size(int64_t n, int32_t p, size_t *bytes)
{
    if (!bytes || check_np(n, p) != CH_OK)
        return CH_ERR_ARG;
    RxyWs w;
    const int rc = rxy_layout(n, p, &w);
    if (rc != CH_OK)
        return rc;
    *bytes = w.end;
    return CH_OK;
}

int ch_convex_hull_rxy(const int32_t *pts, int64_t n, int32_t p, int32_t *L, int32_t *R,
                       int32_t *hull, int32_t *hull_count, void *workspace, size_t ws_bytes,
                       ch_stream_t stream)
{
    if (check_np(n, p) != CH_OK || (n > 0 && !pts) || !hull || !hull_count || !aligned8(pts) ||
        !aligned8(L) || !aligned8(R) || !aligned8(hull))
        return CH_ERR_ARG;
    RxyWs w;
    int rc = rxy_layout(n, p, &w);
    if (rc != CH_OK)
        return rc;
    if (!ws_aligned(workspace))
        return CH_ERR_ARG;
    if (ws_bytes < w.end || !workspace)
        return CH_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned *st = device_status_ptr(s);
    if (!st)
        return CH_ERR_CUDA;
    char *b = reinterpret_cast<char *>(workspace);
    const PathWs &pw = w.path;
    if (!L)
        L = reinterpret_cast<int32_t *>(b + pw.L);
    if (!R)
        R = reinterpret_cast<int32_t *>(b + w.R);
    cudaEvent_t ev0, ev1;
    next_trace(&ev0, &ev1);
    cudaError_t e = reduce_launch(pw.plan, pts, n, square_frame(p), b + pw.part, L, st, s, nullptr,
                                  0, ev0, ev1);
    if (e == cudaSuccess && pw.plan.mode == 0)
        e = reduce_merge_launch(b + pw.part, pw.plan.copies, p, p, L, s);
    if (e == cudaSuccess)
        e = rows_launch(L, p, R, st, s);
    // the rxy points as chains along y: the transposed frame of the plain path
    const HullLayout hl = hull_layout(p);
    char *hw = b + pw.hull;
    int32_t *hull_t = reinterpret_cast<int32_t *>(b + w.hull_t);
    int32_t *count_t = reinterpret_cast<int32_t *>(b + w.count_t);
    if (e == cudaSuccess)
        e = chain_launch(R, p, nullptr, nullptr, nullptr, nullptr, b + pw.state, false,
                         reinterpret_cast<int2 *>(hw + hl.cand), reinterpret_cast<int *>(hw + hl.ccnt),
                         st, s);
    if (e == cudaSuccess)
        e = hull_final_launch(hl, hw, hull_t, count_t, s, p <= 16384);
    if (e == cudaSuccess)
        e = unframe_launch(hull_t, count_t, Frame{1, 1, p, p, 1, 0}, hull, hull_count, s);
    return cuda_rc(e);
}

}  // extern "C"
