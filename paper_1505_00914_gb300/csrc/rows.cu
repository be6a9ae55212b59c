// The second scan along y (Section 2, Fig. 4: rx -> rxy): Algorithm 1 again,
// over the rx points that L holds (its valid (x, ly) and (x, hy)), with the
// roles of x and y exchanged.  R[y - 1] = (min x, max x) over the rx points
// with that y, (p + 1, -1) for a row with none.
//
// k_rows_fill    R = (p + 1, -1) everywhere;
// k_rows_reduce  one thread per column of L: its one or two points go to
//                their rows by atomic min / max (read first, so an entry
//                that cannot improve costs no atomic).
// The rxy points, as chains along y, then take the plain path's chain and
// hull kernels in the transposed frame, and the hull is mapped back.
#include "ch_internal.cuh"

namespace ch {
namespace {

constexpr int RW_T = 256;

__global__ void __launch_bounds__(RW_T) k_rows_fill(int2 *R, int p)
{
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * RW_T + threadIdx.x;
    if (i < p)
        R[i] = make_int2(p + 1, -1);
}

__device__ __forceinline__ void row_put(int2 *R, int y, int x)
{
    const int2 e = R[y - 1];
    if (x < e.x)
        atomicMin(&R[y - 1].x, x);
    if (x > e.y)
        atomicMax(&R[y - 1].y, x);
}

__global__ void __launch_bounds__(RW_T)
    k_rows_reduce(const int2 *__restrict__ L, int p, int2 *R, unsigned *status)
{
    pdl_wait();
    pdl_trigger();
    const int c = blockIdx.x * RW_T + threadIdx.x;
    if (c >= p)
        return;
    const int2 e = L[c];
    if (e.x == p + 1 && e.y == -1)
        return;
    // Algorithm 1 on points in range leaves 1 <= ly <= hy <= p; any other
    // entry is not an array L and is reported instead of used
    if (e.x < 1 || e.x > e.y || e.y > p) {
        atomicOr(status, ST_RANGE);
        return;
    }
    row_put(R, e.x, c + 1);
    if (e.y != e.x)
        row_put(R, e.y, c + 1);
}

}  // namespace

cudaError_t rows_launch(const int32_t *L, int p, int32_t *R, unsigned *status, cudaStream_t s)
{
    const int g = (p + RW_T - 1) / RW_T;
    launch(k_rows_fill, g, RW_T, 0, s, reinterpret_cast<int2 *>(R), p);
    launch(k_rows_reduce, g, RW_T, 0, s, reinterpret_cast<const int2 *>(L), p,
           reinterpret_cast<int2 *>(R), status);
    return cudaGetLastError();
}

}  // namespace ch
