/*
 * ch.h - C ABI of libch.so, a GB300 (sm_103a) implementation of the integer
 * convex-hull preconditioner of Cadenas & Megson, "An Empirical Evaluation of
 * Preconditioning Data for Accelerating Convex Hull Computations".
 *
 * The hot path has three steps, each a CUDA kernel family:
 *   1. ch_reduce - Algorithm 1 (Reduction of Points, Section 2.1): n integer
 *      points in [1,p]^2 become one (min y, max y) pair per x column, held in
 *      an array L of p entries that start at (p+1, -1).
 *   2. ch_chain  - the scan of Lemma 1 (Section 2.1) and the bit array M of
 *      the "Extraction using an array of bits" passage (Section 4): the valid
 *      columns (entries that left (p+1, -1)) become the x-ordered lower chain
 *      (x, ly) and upper chain (x, hy).
 *   3. ch_hull   - a monotone-chain hull on the two chains, so nothing is
 *      sorted.  Output: the strict vertices (collinear points removed, as in
 *      the Appendix) counter-clockwise from the lexicographic minimum.
 *
 * Conventions shared by every entry point
 *   - Points are int32 pairs (x, y), interleaved: pts[2k] = x, pts[2k+1] = y.
 *     Every point must satisfy 1 <= x, y <= p (the square of side p).
 *   - L is int32[p][2], 0-based: column x is L[2(x-1)] = ly, L[2(x-1)+1] = hy;
 *     an empty column holds (p+1, -1).
 *   - Array arguments are DEVICE pointers owned by the caller, unless the name
 *     says host.  int32 pairs must be 8-byte aligned; 16-byte alignment of the
 *     point array gives the fastest loads.
 *   - Nothing allocates device memory inside a call: each call that needs
 *     scratch takes a caller-owned device workspace whose size is returned by
 *     the matching *_workspace_size query.  A workspace starts on a 256-byte
 *     boundary (as cudaMalloc returns memory); a misaligned one is refused
 *     with CH_ERR_ARG.  A workspace may be reused by any later call on the
 *     same stream; two calls in flight at once need two.
 *   - Calls are asynchronous and stream-ordered on `stream` (NULL = legacy
 *     default stream).  The return value reports argument and launch errors
 *     only.  Errors that depend on the data (a point outside [1,p]^2, a
 *     capacity overflow, a bounded wait that ran out) are recorded in a sticky
 *     status word of the stream the call was made on (a call captured in a
 *     CUDA graph records into the word of the stream it was captured on);
 *     ch_sync_status(stream) waits for that stream and returns (and clears)
 *     its word, so an error is reported only to the stream whose call made
 *     it.  After such an error the outputs of that call are unspecified but
 *     every kernel has returned: no call ever hangs.
 *   - p must satisfy 1 <= p <= 2^30 (so int64 cross products of coordinate
 *     differences cannot overflow); n >= 0.
 */
#ifndef CH_H
#define CH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; declared here so this header needs no CUDA. */
typedef struct CUstream_st *ch_stream_t;

/* Status codes. */
#define CH_OK 0
#define CH_ERR_ARG (-1)       /* bad argument: null pointer, n < 0, p out of range, misalignment */
#define CH_ERR_RANGE (-2)     /* some point outside [1,p]^2 (recorded by a kernel) */
#define CH_ERR_CAPACITY (-3)  /* an output or workspace region was too small (recorded by a kernel) */
#define CH_ERR_TIMEOUT (-4)   /* a bounded inter-block wait ran out (recorded by a kernel) */
#define CH_ERR_CUDA (-5)      /* a CUDA runtime call or kernel launch failed */
#define CH_ERR_WORKSPACE (-6) /* ws_bytes smaller than the *_workspace_size query */

#define CH_MAX_P (1 << 30)

/* Text for a status code (static storage, never NULL). */
const char *ch_strerror(int code);

/* ABI version, (major << 16) | minor. */
int ch_version(void);

/* Read and clear the status word of `stream` on the current device, then
 * wait for the stream.  The word is taken by an atomic exchange with zero that
 * runs on `stream` after the work queued there before, and is copied back on
 * the same stream, so calls on other streams neither wait nor lose their own
 * errors.  Returns CH_OK or a recorded error (RANGE before CAPACITY before
 * TIMEOUT when several bits are set), or CH_ERR_CUDA if the stream itself
 * failed.  A device keeps a word of its own for each of the first 1024
 * distinct stream handles used on it; later handles share one further word.
 * Two host threads reading the same stream's word at once race. */
int ch_sync_status(ch_stream_t stream);

/* Clear the status word of `stream` (stream-ordered, does not wait). */
int ch_clear_status(ch_stream_t stream);

/* Profiling aid (not part of the method).  events: npairs pairs of
 * cudaEvent_t handles created by the caller with timing enabled.  While set,
 * every ch_reduce / ch_convex_hull call records the next pair (round robin)
 * on its stream immediately before and after its main reduction kernel (the
 * one that reads every point), so the caller can time that kernel inside a
 * longer stream of work.  npairs = 0
 * (or events = NULL) turns it off.  Process-wide; the handles must outlive
 * the calls that use them. */
int ch_trace_set(void *const *events, int npairs);

/* How ch_convex_hull will run n points of side p on the current device
 * when it is not asked for the chains (lower, upper and counts NULL):
 * *form = 0 (private shared-memory copies of L, p <= 20480), 1 (filtered
 * global L, p <= 116224), 2 (global L with a read-then-atomic test) or 3
 * (small problems: p <= 16384, at most 8192 points per thread block and
 * the blocks' partial copies of L at most 65536 words in all, the whole path
 * in one launch), and *kernels = the number of kernels one ch_convex_hull
 * call launches (with the second filter pass of the hull step from 128 runs
 * of 1024 columns on).  A call that asks for the chains never takes form 3.
 * Either pointer may be NULL. */
int ch_plan_info(int64_t n, int32_t p, int32_t *form, int32_t *kernels);

/* ---------------------------------------------------------------------- */
/* Step 1: Algorithm 1, Reduction of Points (Section 2.1).                 */
/* ---------------------------------------------------------------------- */

/* Workspace bytes ch_reduce needs for n points and side p on the current
 * device (it holds one private L per resident thread block). */
int ch_reduce_workspace_size(int64_t n, int32_t p, size_t *bytes);

/* L[x-1] = (min y, max y) over the points with that x, (p+1, -1) for columns
 * with no point.  pts: int32[n][2] (read only).  L: int32[p][2], written in
 * full.  Points outside [1,p]^2 are skipped and recorded as CH_ERR_RANGE. */
int ch_reduce(const int32_t *pts, int64_t n, int32_t p, int32_t *L,
              void *workspace, size_t ws_bytes, ch_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Step 2: chains of the valid columns (Lemma 1; bit array M, Section 4).  */
/* ---------------------------------------------------------------------- */

int ch_chain_workspace_size(int32_t p, size_t *bytes);

/* From L (int32[p][2], as written by ch_reduce): a column is valid when its
 * entry differs from (p+1, -1).  Writes, in increasing x, lower[k] = (x, ly)
 * and upper[k] = (x, hy) for the k-th valid column (capacity p pairs each),
 * counts[0] = counts[1] = number of valid columns (device int32[2]), and, if
 * mask is not NULL, the bit array M: uint32[(p+31)/32], column i (1-based) at
 * bit (i-1) & 31 of word (i-1) >> 5. */
int ch_chain(const int32_t *L, int32_t p, int32_t *lower, int32_t *upper,
             int32_t *counts, uint32_t *mask,
             void *workspace, size_t ws_bytes, ch_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Step 3: hull of the chains (monotone chain; strictness per Appendix).   */
/* ---------------------------------------------------------------------- */

int ch_hull_workspace_size(int32_t p, size_t *bytes);

/* lower: int32[counts[0]][2], upper: int32[counts[1]][2], both strictly
 * increasing in x, with lower[k].y <= upper[j].y where they share a column
 * (as written by ch_chain).  counts is a DEVICE int32[2] (the host need not
 * know it).  Writes the strict hull vertices counter-clockwise from the
 * lexicographic minimum to hull (capacity 2p pairs) and their number to
 * *hull_count (device int32).  Empty chains give hull_count = 0. */
int ch_hull(const int32_t *lower, const int32_t *upper, const int32_t *counts,
            int32_t p, int32_t *hull, int32_t *hull_count,
            void *workspace, size_t ws_bytes, ch_stream_t stream);

/* ---------------------------------------------------------------------- */
/* The three steps in one call, back to back on the stream (each kernel   */
/* launched with programmatic dependent launch), with the chain step and   */
/* the hull's pre-filter fused into one kernel.                            */
/* ---------------------------------------------------------------------- */

int ch_convex_hull_workspace_size(int64_t n, int32_t p, size_t *bytes);

/* Same outputs as ch_reduce + ch_chain + ch_hull; L, lower, upper, counts
 * may each be NULL, in which case the workspace holds them.  When lower,
 * upper and counts are all NULL the chains are not ranked or written at all:
 * the chain step writes only the candidates of the hull.  A small problem
 * (ch_plan_info form 3) called with lower, upper and counts all NULL runs
 * as one kernel: its thread blocks fold slices of the points into private
 * copies of L, and the block that finishes last (a ticket word kept per
 * stream, zero between calls) merges them and computes the hull, so calls
 * made on one stream must not overlap (as stream order ensures). */
int ch_convex_hull(const int32_t *pts, int64_t n, int32_t p, int32_t *L,
                   int32_t *lower, int32_t *upper, int32_t *counts,
                   int32_t *hull, int32_t *hull_count,
                   void *workspace, size_t ws_bytes, ch_stream_t stream);

/* The same two calls for points stored as packed 16-bit pairs (the int16x2
 * point format): pts is uint32[n], point k = (x, y) with x - 1 in the low
 * and y - 1 in the high 16 bits of pts[k] (little-endian uint16 pairs
 * (x - 1, y - 1)), 4-byte aligned; p <= 65536 (else CH_ERR_ARG).  Half the
 * bytes of int32 pairs per point.  Workspaces: ch_reduce_workspace_size and
 * ch_convex_hull_workspace_size for the same n and p.  Outputs and errors
 * as for ch_reduce and ch_convex_hull. */
int ch_reduce_u16(const uint32_t *pts, int64_t n, int32_t p, int32_t *L, void *workspace,
                  size_t ws_bytes, ch_stream_t stream);
int ch_convex_hull_u16(const uint32_t *pts, int64_t n, int32_t p, int32_t *L, int32_t *lower,
                       int32_t *upper, int32_t *counts, int32_t *hull, int32_t *hull_count,
                       void *workspace, size_t ws_bytes, ch_stream_t stream);

int ch_convex_hull_host_workspace_size(int64_t n, int32_t p, size_t *bytes);

/* End to end from HOST memory: copies host_pts (int32[n][2]; pinned memory
 * gives full copy speed) to the device workspace, runs ch_convex_hull, copies
 * the hull to host_hull (capacity 2p pairs) and its size to
 * *host_hull_count, and waits for the stream.  Returns the data status too
 * (it calls ch_sync_status). */
int ch_convex_hull_host(const int32_t *host_pts, int64_t n, int32_t p,
                        int32_t *host_hull, int32_t *host_hull_count,
                        void *workspace, size_t ws_bytes, ch_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Lemma 1's polyline and Melkman's hull of it (Section 2.1; Section 3,    */
/* Fig. 10: the reduced set is a simple polyline, so Melkman's linear      */
/* algorithm for simple polylines applies without a sort).                 */
/* ---------------------------------------------------------------------- */

int ch_polyline_workspace_size(int32_t p, size_t *bytes);

/* From L (int32[p][2], as written by ch_reduce): for each valid column in
 * increasing x, the vertex (x, ly) and then (x, hy) when hy != ly, written to
 * poly (capacity 2p pairs); *count (device int32) = the number of vertices.
 * Joining consecutive vertices gives the simple chain of Lemma 1. */
int ch_polyline(const int32_t *L, int32_t p, int32_t *poly, int32_t *count,
                void *workspace, size_t ws_bytes, ch_stream_t stream);

/* Bytes of the deque ch_hull_melkman keeps in global memory: 0 (workspace
 * may be NULL) unless the largest convex lattice polygon in [1,p]^2 has more
 * than 16382 vertices (p above about 2^17). */
int ch_hull_melkman_workspace_size(int32_t p, size_t *bytes);

/* Melkman's algorithm on the polyline poly[0 .. *count) (count: DEVICE
 * int32), which must be simple with distinct vertices in [1,p]^2 - the Lemma 1
 * polyline is.  Writes the strict hull vertices counter-clockwise from the
 * lexicographic minimum to hull (capacity min(2p, *count) pairs) and their
 * number to *hull_count (device int32).  A vertex outside [1,p]^2 records
 * CH_ERR_RANGE (hull_count 0).  For a polyline that is not simple the result
 * is unspecified, but nothing is written beyond min(2p, *count) pairs (a
 * longer vertex list records CH_ERR_CAPACITY instead).  One warp: the
 * algorithm is sequential. */
int ch_hull_melkman(const int32_t *poly, const int32_t *count, int32_t p, int32_t *hull,
                    int32_t *hull_count, void *workspace, size_t ws_bytes, ch_stream_t stream);

int ch_convex_hull_melkman_workspace_size(int64_t n, int32_t p, size_t *bytes);

/* ch_reduce, the polyline and ch_hull_melkman in one call; L, poly and
 * poly_count may each be NULL (the workspace holds them).  Same hull as
 * ch_convex_hull.  The polyline written to poly (capacity 2p pairs) is
 * ch_polyline's with the vertices that the exact in-tile pre-filter of the
 * hull step rules out (on or above a segment between two other chain points)
 * removed, column by column: the Lemma 1 polyline of a sub-array of L, so
 * still simple, and holding every hull vertex. */
int ch_convex_hull_melkman(const int32_t *pts, int64_t n, int32_t p, int32_t *L, int32_t *poly,
                           int32_t *poly_count, int32_t *hull, int32_t *hull_count,
                           void *workspace, size_t ws_bytes, ch_stream_t stream);

/* ---------------------------------------------------------------------- */
/* The sparse regime p > n (Section 4, "Extraction using a tree structure" */
/* and "For all practical purposes"): the bit array M becomes a w-ary tree */
/* of 32-bit words (one bit per non-empty word of the level below), L is   */
/* kept in a form whose empty entry is all-zero, and each call clears what */
/* it touched, so that a call costs O(n + s) and never O(p).               */
/* ---------------------------------------------------------------------- */

/* *bytes: workspace for n points of side p; *persistent_bytes (optional):
 * its leading part, which must be zero-filled (cudaMemsetAsync) before the
 * first call and which every call that records no error leaves zero-filled
 * again (it depends on p only, so one workspace sized for the largest n
 * serves any smaller n of the same p).  After a recorded error, zero it
 * again. */
int ch_sparse_workspace_size(int64_t n, int32_t p, size_t *bytes, size_t *persistent_bytes);

/* Number of kernels one ch_convex_hull_sparse call launches. */
int ch_sparse_kernel_count(int64_t n, int32_t p, int32_t *kernels);

/* Same results as ch_convex_hull (chains and hull; L is not materialised):
 * lower, upper (capacity min(p, n) pairs each) and counts may be NULL, in
 * which case the workspace holds them.  Points outside [1,p]^2 are skipped
 * and recorded as CH_ERR_RANGE. */
int ch_convex_hull_sparse(const int32_t *pts, int64_t n, int32_t p, int32_t *lower,
                          int32_t *upper, int32_t *counts, int32_t *hull, int32_t *hull_count,
                          void *workspace, size_t ws_bytes, ch_stream_t stream);

/* ---------------------------------------------------------------------- */
/* The second scan along y (Section 2, Fig. 4: rx -> rxy).                 */
/* ---------------------------------------------------------------------- */

/* From L (int32[p][2], as written by ch_reduce): Algorithm 1 once more over
 * its rx points - the valid (x, ly) and (x, hy) - with x and y exchanged.
 * R: int32[p][2], written in full; row y (1-based) at R[2(y-1)] = min x,
 * R[2(y-1)+1] = max x over the rx points with that y, (p+1, -1) for none.
 * The rxy points are the (min x, y) and (max x, y) of the valid rows: a
 * subset of rx that keeps every hull vertex.  An entry of L outside
 * 1 <= ly <= hy <= p (other than the empty one) is skipped and recorded as
 * CH_ERR_RANGE. */
int ch_reduce_rows(const int32_t *L, int32_t p, int32_t *R, ch_stream_t stream);

int ch_convex_hull_rxy_workspace_size(int64_t n, int32_t p, size_t *bytes);

/* ch_reduce, ch_reduce_rows, then the chains and hull of the rxy points (the
 * plain path's kernels in the transposed frame, the hull mapped back).  L and
 * R may be NULL (the workspace holds them).  Same hull as ch_convex_hull. */
int ch_convex_hull_rxy(const int32_t *pts, int64_t n, int32_t p, int32_t *L, int32_t *R,
                       int32_t *hull, int32_t *hull_count, void *workspace, size_t ws_bytes,
                       ch_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Many independent sets in one persistent launch (the three steps per     */
/* set, Section 2.1).                                                      */
/* ---------------------------------------------------------------------- */

/* Largest side p of a set in a batch. */
#define CH_BATCH_MAX_P 16384

/* Set s holds points [offsets[s], offsets[s+1]) of one interleaved int32
 * point array and has side ps[s] (1 <= ps[s] <= CH_BATCH_MAX_P).  The plan
 * cuts each set into chunks of about chunk_mult * ps[s] points (at least
 * 65536, at most 2^22): the tuning knob.  host_offsets (int64[B+1]) and
 * host_ps (int32[B]) are HOST arrays. */
int ch_batched_workspace_size(int32_t B, const int64_t *host_offsets, const int32_t *host_ps,
                              int32_t chunk_mult, size_t *bytes);

/* Builds the work plan on the host and stores it in the device workspace
 * (waits for `stream`).  The workspace then belongs to this plan: any number
 * of ch_hull_batched calls with the same B may follow (and may be captured in
 * a CUDA graph); prepare again after a change of sizes. */
int ch_batched_prepare(int32_t B, const int64_t *host_offsets, const int32_t *host_ps,
                       int32_t chunk_mult, void *workspace, size_t ws_bytes, ch_stream_t stream);

/* The CTA shape of ch_hull_batched's persistent kernel (1024 threads):
 * fold_threads = 0 has every thread fold a set's points and then finish it
 * (chains, exact pre-filter, peel/merge/stitch); 384, 512, 640, 768 or 896
 * splits the CTA: that many threads fold the next set's points while the
 * other 1024 - fold_threads peel, merge and stitch the previous set (the
 * pre-filter, which reads the set's L in shared memory, is run by all of
 * them).  The hulls are the same for every shape. */
#define CH_BATCH_FOLD_DEFAULT 512

/* ch_batched_prepare with the CTA shape (fold_threads: 0, 384, 512, 640, 768 or 896;
 * anything else is CH_ERR_ARG).  ch_batched_prepare uses
 * CH_BATCH_FOLD_DEFAULT; the autotuner times the others. */
int ch_batched_prepare_shape(int32_t B, const int64_t *host_offsets, const int32_t *host_ps,
                             int32_t chunk_mult, int32_t fold_threads, void *workspace,
                             size_t ws_bytes, ch_stream_t stream);

/* Hulls of the B sets of the prepared plan in one launch.  pts: the device
 * point array; offsets, ps: device copies of the sizes the plan was built
 * from (kept in the signature; the plan carries them).  hull_out: int32 pairs,
 * set s writing hull_out[hull_offsets[s] ...] (device int64[B+1]; capacity at
 * least min(n_s, 2 * ps[s]) pairs per set); hull_counts: device int32[B].
 * Each hull lists strict vertices counter-clockwise from the lexicographic
 * minimum.  Returns CH_ERR_ARG if no plan for B sets was prepared in
 * `workspace`. */
int ch_hull_batched(const int32_t *pts, const int64_t *offsets, const int32_t *ps, int32_t B,
                    int32_t *hull_out, const int64_t *hull_offsets, int32_t *hull_counts,
                    void *workspace, size_t ws_bytes, ch_stream_t stream);

/* Algorithm 1 (Section 2.1) for each set of the prepared plan in the same
 * persistent launch as ch_hull_batched, stopping after the reduction: set s
 * writes its L, int32[ps[s]][2] (L[x-1] = (min y, max y), (ps[s]+1, -1) for a
 * column with no point), to L_out[L_offsets[s] ...] (device int64[B+1]
 * offsets counted in pairs; capacity at least ps[s] pairs per set).  Points
 * outside [1, ps[s]]^2 are skipped and recorded as CH_ERR_RANGE.  Returns
 * CH_ERR_ARG if no plan for B sets was prepared in `workspace`. */
int ch_reduce_batched(const int32_t *pts, const int64_t *offsets, const int32_t *ps, int32_t B,
                      int32_t *L_out, const int64_t *L_offsets, void *workspace, size_t ws_bytes,
                      ch_stream_t stream);

/* Chains of every set (Lemma 1; ch_chain for B sets in one launch).  L and
 * L_offsets as written by ch_reduce_batched; ps: device int32[B] (any side
 * >= 1).  A column is valid when its entry differs from (ps[s]+1, -1).  Set s
 * writes, in increasing x, lower[L_offsets[s] + k] = (x, ly) and
 * upper[L_offsets[s] + k] = (x, hy) for its k-th valid column, and
 * counts[2s] = counts[2s+1] = its number of valid columns (device
 * int32[B][2]).  No workspace. */
int ch_chain_batched(const int32_t *L, const int64_t *L_offsets, const int32_t *ps, int32_t B,
                     int32_t *lower, int32_t *upper, int32_t *counts, ch_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Integer points anywhere in int32: Steps 1 and 2 of the paper's general   */
/* procedure (Section 2, "Implementation of the proposed heuristic": find   */
/* the bounding box, translate the points into it, then Algorithm 1), with  */
/* the columns of L along the shorter side of the box (the sweep along      */
/* min(p, q) recommended in the same passage).                              */
/* ---------------------------------------------------------------------- */

int ch_bbox_workspace_size(size_t *bytes);

/* box: device int32[4] = (xmin, xmax, ymin, ymax) of the n points (for
 * n = 0: (INT32_MAX, INT32_MIN, INT32_MAX, INT32_MIN)).  pts 8-byte aligned. */
int ch_bbox(const int32_t *pts, int64_t n, int32_t *box, void *workspace, size_t ws_bytes,
            ch_stream_t stream);

/* host_box: HOST int32[4] = (xmin, xmax, ymin, ymax) enclosing every point
 * (typically ch_bbox's result copied to the host); each side
 * (max - min + 1) must be 1 .. CH_MAX_P, else CH_ERR_ARG.  A point outside
 * the box is reported as CH_ERR_RANGE by ch_sync_status. */
int ch_convex_hull_box_workspace_size(int64_t n, const int32_t *host_box, size_t *bytes);

/* The strict hull of the points in their own coordinates, counter-clockwise
 * from the lexicographic minimum: hull capacity 2 * min(p, q) + 2 points
 * (p, q the box sides). */
int ch_convex_hull_box(const int32_t *pts, int64_t n, const int32_t *host_box, int32_t *hull,
                       int32_t *hull_count, void *workspace, size_t ws_bytes, ch_stream_t stream);

/* ch_chain without a workspace (the paper has no counterpart: it is an     */
/* interface for callers that cannot allocate device memory, e.g. plain C  */
/* code without a device allocator, or loops that must not call cudaMalloc */
/* / cudaFree because those synchronise the device).  Same arguments and   */
/* results as ch_chain; the look-back scratch is a fixed device array of    */
/* the library sized for p <= CH_CHAIN_NOALLOC_MAX_P (128 KiB); larger p    */
/* returns CH_ERR_CAPACITY.  Nothing needs to be zeroed by the caller: each */
/* call clears the scratch words it uses on `stream` before its kernel.     */
/* The first call on a device looks up the array's address with            */
/* cudaGetSymbolAddress, so make it before any stream capture begins.  One  */
/* array serves all calls on a device: calls that overlap in time race on   */
/* it and must be serialised by the caller. */
#define CH_CHAIN_NOALLOC_MAX_P (1 << 24)
int ch_chain_noalloc(const int32_t *L, int32_t p, int32_t *lower, int32_t *upper, int32_t *counts,
                     uint32_t *mask, ch_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Learned culling proposal: MLP 1024 -> 256 -> 256 -> K on a 32x32        */
/* occupancy histogram (not in the paper; the hull stays exact whatever    */
/* the network outputs, see ch_hull_learned).  All pointers are device     */
/* pointers to row-major float32 arrays; GEMMs run on the tensor cores with */
/* bf16 operands and fp32 accumulation.                                     */
/* ---------------------------------------------------------------------- */

#define CH_MLP_IN 1024
#define CH_MLP_HID 256
#define CH_MLP_K 16
/* Parameter vector: W1[1024][256], b1[256], W2[256][256], b2[256],
 * W3[256][16], b3[16] (W[i][j]: input i to output j), 332304 floats. */
#define CH_MLP_PARAMS (1024 * 256 + 256 + 256 * 256 + 256 + 256 * 16 + 16)

/* X[M][1024] -> H1 = relu(X W1 + b1), H2 = relu(H1 W2 + b2), Y = H2 W3 + b3
 * (H1, H2: [M][256], kept for the backward pass; Y: [M][16]). */
int ch_mlp_forward(const float *params, const float *X, int32_t M, float *H1, float *H2, float *Y,
                   ch_stream_t stream);

/* Loss of the direction offsets against targets T[M][16] in [-1, 1]:
 * *loss = mean((tanh(Y) - T)^2) (device float), dY = dloss/dY. */
int ch_mlp_loss(const float *Y, const float *T, int32_t M, float *dY, float *loss,
                ch_stream_t stream);

int ch_mlp_backward_workspace_size(int32_t M, size_t *bytes);

/* Gradients of the loss with respect to every parameter (same layout as
 * params) from the forward activations and dY. */
int ch_mlp_backward(const float *params, const float *X, const float *H1, const float *H2,
                    const float *dY, int32_t M, float *grads, void *workspace, size_t ws_bytes,
                    ch_stream_t stream);

/* One Adam step (step counts from 1) on params with moments m, v. */
int ch_mlp_adam(float *params, const float *grads, float *m, float *v, int32_t step, float lr,
                float beta1, float beta2, float eps, ch_stream_t stream);

/* ---------------------------------------------------------------------- */
/* Learned culling (not in the paper; it serves the culling idea that a    */
/* convex polygon with input points as vertices lies inside the hull, so   */
/* that the points strictly inside it are no hull vertices).               */
/*                                                                          */
/* Sample: runs of CH_CULL_RUN consecutive points starting at j * (n /      */
/* CH_CULL_RUNS), j < CH_CULL_RUNS (all points when n <= their product).   */
/* Features: 32 x 32 occupancy histogram of the sample, cell (bx, by) =    */
/* ((x-1)*32/p, (y-1)*32/p) at index by*32+bx, value count * (1024/m) in   */
/* float32 (m = sample size).  Network: ch_mlp_forward's, for one vector,  */
/* giving y[16]; directions theta_k = 2*pi*k/16 + (pi/16)*tanh(y_k) (the    */
/* sector centres when params is NULL).  Extremes: per direction the sample */
/* point maximising fl32(fl32(cos*x) + fl32(sin*y)), ties to the smaller    */
/* index.  Polygon: strict hull of the extremes; with a network, the larger */
/* (exact area, ties to the centres) of the network's and the sector        */
/* centres' polygons, so the network can only enlarge the culled region.    */
/* Start array Linit: for                                                   */
/* columns strictly between the polygon's extreme x values, (floor(b(x))+1, */
/* ceil(u(x))-1) with b, u its lower and upper boundary; (p+1, -1) else.    */
/* ---------------------------------------------------------------------- */

#define CH_CULL_RUN 1024
#define CH_CULL_RUNS 256

int ch_cull_workspace_size(int32_t p, size_t *bytes);

/* The culling proposal alone, with its intermediate results.  Linit: device
 * int32[p][2] (required).  Optional (NULL to skip) device outputs: features
 * float[1024], net_out float[16] (y), for both direction sets (set 0 the
 * sector centres, set 1 the network's, zero / -1 without a network) dirs
 * float[2][32] (16 cosines then 16 sines) and extremes int64[2][16] (point
 * indices, -1 if none), and for the polygon used poly int32[16][2] +
 * poly_count (counter-clockwise from the lexicographic minimum) and chosen
 * int32 (1: the network's polygon, 0: the sector centres', -1: no network).
 * params: device float[CH_MLP_PARAMS]
 * or NULL.  Workspace: device memory of ch_cull_workspace_size bytes, no
 * initial contents. */
int ch_cull_propose(const int32_t *pts, int64_t n, int32_t p, const float *params, int32_t *Linit,
                    float *features, float *net_out, float *dirs, int32_t *poly,
                    int32_t *poly_count, int64_t *extremes, int32_t *chosen, void *workspace,
                    size_t ws_bytes, ch_stream_t stream);

/* Quality of one culling step, written by the kernels of ch_hull_learned
 * (device memory, 16 bytes). */
typedef struct ch_cull_stats {
    int64_t culled;         /* input points strictly inside the culling polygon, i.e.
                               Linit.lo <= y <= Linit.hi in their column (points
                               outside [1,p]^2 are not counted); cull rate = culled / n */
    int32_t poly_vertices;  /* strict vertices of the polygon used (0 .. 16) */
    int32_t chosen;         /* 1: the network's polygon, 0: the sector centres',
                               -1: no network (params NULL) */
} ch_cull_stats;

int ch_hull_learned_workspace_size(int64_t n, int32_t p, size_t *bytes);

/* Kernels one ch_hull_learned call launches (with_net != 0: params given)
 * when stats is NULL; a non-NULL stats adds one counting kernel. */
int ch_hull_learned_kernel_count(int64_t n, int32_t p, int32_t with_net, int32_t *kernels);

/* The whole path with culling: the proposal above, Algorithm 1 started from
 * Linit (L = column-wise (min, max) of Linit and the points), chains of the
 * columns where L moved past Linit (lower: L.lo < Linit.lo, upper: L.hi >
 * Linit.hi; counts[0], counts[1] may differ), and the strict hull, which is
 * the same as ch_convex_hull's for every params (NULL included).  Arguments
 * as in ch_convex_hull; L, Linit, lower, upper, counts may be NULL.
 * stats: NULL, or a device ch_cull_stats filled in by this call (the count
 * of culled points costs one more pass over the points, after the hull). */
int ch_hull_learned(const int32_t *pts, int64_t n, int32_t p, const float *params, int32_t *L,
                    int32_t *Linit, int32_t *lower, int32_t *upper, int32_t *counts, int32_t *hull,
                    int32_t *hull_count, ch_cull_stats *stats, void *workspace, size_t ws_bytes,
                    ch_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* CH_H */
