// Steps 1 and 2 of the paper's general procedure (Section 2, "Implementation
// of the proposed heuristic") for integer points anywhere in int32: the
// bounding box (Step 1), then Algorithm 1 on the points translated into it
// (Step 2, fused into the reduction as a column/row offset), with the columns
// along the shorter side of the box (the sweep along min(p, q) that the same
// passage recommends), and the hull mapped back to the input coordinates.
//
// k_bbox        per-CTA minima and maxima of x and y over its slice;
// k_bbox_final  one CTA folds the per-CTA results into box[4];
// k_unframe     the hull from frame coordinates back to the input's: a
//               translation, and for a transposed frame a reflection, which
//               reverses the orientation, so the list is read backwards from
//               the input's lexicographic minimum.
#include <climits>

#include "ch_internal.cuh"

namespace ch {
namespace {

constexpr int BB_T = 512;

__device__ __forceinline__ int4 box_fold(int4 a, int4 b)
{
    return make_int4(min(a.x, b.x), max(a.y, b.y), min(a.z, b.z), max(a.w, b.w));
}

__device__ __forceinline__ int4 warp_box(int4 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        int4 w;
        w.x = __shfl_xor_sync(0xFFFFFFFFu, v.x, o);
        w.y = __shfl_xor_sync(0xFFFFFFFFu, v.y, o);
        w.z = __shfl_xor_sync(0xFFFFFFFFu, v.z, o);
        w.w = __shfl_xor_sync(0xFFFFFFFFu, v.w, o);
        v = box_fold(v, w);
    }
    return v;
}

// box = (xmin, xmax, ymin, ymax); the empty box is (INT_MAX, INT_MIN, ...).
__global__ void __launch_bounds__(BB_T) k_bbox(const int2 *__restrict__ pts, long long n, int4 *part)
{
    pdl_wait();
    pdl_trigger();
    __shared__ int4 s_w[BB_T / 32];
    int4 b = make_int4(INT_MAX, INT_MIN, INT_MAX, INT_MIN);
    const long long stride = (long long)gridDim.x * BB_T;
    for (long long i0 = (long long)blockIdx.x * BB_T + threadIdx.x; i0 < n; i0 += 4 * stride) {
        int2 q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long i = i0 + u * stride;
            q[u] = i < n ? __ldcs(pts + i) : make_int2(0, 0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (i0 + u * stride < n)
                b = box_fold(b, make_int4(q[u].x, q[u].x, q[u].y, q[u].y));
    }
    b = warp_box(b);
    if ((threadIdx.x & 31) == 0)
        s_w[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x < 32) {
        b = threadIdx.x < BB_T / 32 ? s_w[threadIdx.x] : make_int4(INT_MAX, INT_MIN, INT_MAX, INT_MIN);
        b = warp_box(b);
        if (threadIdx.x == 0)
            part[blockIdx.x] = b;
    }
}

__global__ void __launch_bounds__(32) k_bbox_final(const int4 *part, int nparts, int *box)
{
    pdl_wait();
    pdl_trigger();
    int4 b = make_int4(INT_MAX, INT_MIN, INT_MAX, INT_MIN);
    for (int i = threadIdx.x; i < nparts; i += 32)
        b = box_fold(b, part[i]);
    b = warp_box(b);
    if (threadIdx.x == 0) {
        box[0] = b.x;
        box[1] = b.y;
        box[2] = b.z;
        box[3] = b.w;
    }
}

constexpr int UF_T = 1024;

// hull_in: h frame points (column + 1, row), counter-clockwise from the
// frame's lexicographic minimum; hull_out: the same vertices in the input's
// coordinates, counter-clockwise from the input's lexicographic minimum.
__global__ void __launch_bounds__(UF_T)
    k_unframe(const int2 *__restrict__ hull_in, const int *hull_count, Frame f, int2 *hull_out,
              int *count_out)
{
    pdl_wait();
    pdl_trigger();
    __shared__ unsigned long long s_best[UF_T / 32];
    __shared__ int s_j;
    const int h = *hull_count;
    auto map = [&](int2 q) {
        const int u = q.x - 1 + f.c0, v = q.y - 1 + f.r0;  // in range: the hull's points are inputs
        return f.tr ? make_int2(v, u) : make_int2(u, v);
    };
    if (!f.tr) {
        for (int k = threadIdx.x; k < h; k += UF_T)
            hull_out[k] = map(hull_in[k]);
        if (threadIdx.x == 0)
            *count_out = h;
        return;
    }
    // position of the input's lexicographic minimum (x, then y) in the list;
    // key: x and y with their sign bits flipped (signed order as unsigned
    // order), x in the high word; the vertices are distinct, so are the keys
    auto key_of = [](int2 q) {
        return ((unsigned long long)((unsigned)q.x ^ 0x80000000u) << 32) |
               (unsigned long long)((unsigned)q.y ^ 0x80000000u);
    };
    unsigned long long best = ULLONG_MAX;
    for (int k = threadIdx.x; k < h; k += UF_T)
        best = min(best, key_of(map(hull_in[k])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        best = min(best, __shfl_xor_sync(0xFFFFFFFFu, best, o));
    if ((threadIdx.x & 31) == 0)
        s_best[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x < 32) {
        best = s_best[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            best = min(best, __shfl_xor_sync(0xFFFFFFFFu, best, o));
        if (threadIdx.x == 0)
            s_best[0] = best;
    }
    __syncthreads();
    best = s_best[0];
    for (int k = threadIdx.x; k < h; k += UF_T)
        if (key_of(map(hull_in[k])) == best)
            s_j = k;
    __syncthreads();
    const int j = s_j;
    for (int k = threadIdx.x; k < h; k += UF_T)
        hull_out[k] = map(hull_in[(j - k + h) % h]);
    if (threadIdx.x == 0)
        *count_out = h;
}

}  // namespace

int bbox_parts() { return std::max(1, sm_count() * 2); }

cudaError_t bbox_launch(const int32_t *pts, int64_t n, int32_t *box, void *ws, cudaStream_t s)
{
    const int parts = bbox_parts();
    int4 *part = reinterpret_cast<int4 *>(ws);
    launch(k_bbox, parts, BB_T, 0, s, reinterpret_cast<const int2 *>(pts), (long long)n, part);
    launch(k_bbox_final, 1, 32, 0, s, part, parts, box);
    return cudaGetLastError();
}

cudaError_t unframe_launch(const int32_t *hull_in, const int32_t *count_in, const Frame &f,
                           int32_t *hull_out, int32_t *count_out, cudaStream_t s)
{
    launch(k_unframe, 1, UF_T, 0, s, reinterpret_cast<const int2 *>(hull_in), count_in, f,
           reinterpret_cast<int2 *>(hull_out), count_out);
    return cudaGetLastError();
}

}  // namespace ch
