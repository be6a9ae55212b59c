// The learned culling proposal: a small MLP (1024 -> 256 -> 256 -> K) that
// reads a 32x32 occupancy histogram and proposes K culling directions, with
// its own training kernels.  The paper has no learned part; the network only
// chooses which input points span the culling polygon, so the hull stays
// exact whatever it outputs.
//
// Every layer is one GEMM on the tensor cores: operand tiles are converted to
// bf16 in shared memory and multiplied with mma.sync m16n8k16 (bf16 x bf16 ->
// fp32); bias, ReLU and the ReLU gradient mask are fused into the epilogue.
// Operands are addressed through strides, so the backward products
// (X^T dH, dH W^T) use the same kernel.  Master weights and Adam moments are
// fp32.
#include <cuda_bf16.h>

#include "ch_internal.cuh"

namespace ch {
namespace {

constexpr int GM = 64, GN = 64, GK = 32;  // CTA tile
constexpr int GT = 128;                  // 4 warps, each a 32x32 sub-tile

struct Mat {  // element (r, c) at p[r * sr + c * sc]
    const float *p;
    long long sr, sc;
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// C[M x N] = epilogue(A[M x K] * B[K x N] (+ bias[n])), fp32 out.
// epi: 0 plain, 1 ReLU, 2 multiply by (mask(r, c) > 0) (ReLU gradient).
__global__ void __launch_bounds__(GT)
    k_gemm(Mat A, Mat B, float *C, long long ldc, int M, int N, int K, const float *bias, int epi,
           const float *mask, long long ldm, float beta)
{
    __shared__ __nv_bfloat16 As[GM][GK + 8];
    __shared__ __nv_bfloat16 Bs[GK][GN + 8];
    const int m0 = blockIdx.y * GM, n0 = blockIdx.x * GN;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, tg = lane & 3;
    float acc[2][4][4] = {};
    for (int k0 = 0; k0 < K; k0 += GK) {
        for (int i = threadIdx.x; i < GM * GK; i += GT) {
            const int r = i / GK, c = i % GK;
            const int gr = m0 + r, gc = k0 + c;
            const float v = (gr < M && gc < K) ? A.p[gr * A.sr + gc * A.sc] : 0.f;
            As[r][c] = __float2bfloat16_rn(v);
        }
        for (int i = threadIdx.x; i < GK * GN; i += GT) {
            const int r = i / GN, c = i % GN;
            const int gr = k0 + r, gc = n0 + c;
            const float v = (gr < K && gc < N) ? B.p[gr * B.sr + gc * B.sc] : 0.f;
            Bs[r][c] = __float2bfloat16_rn(v);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; kk += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int r = wm + mi * 16 + g;
                const int c = kk + tg * 2;
                af[mi][0] = *reinterpret_cast<const uint32_t *>(&As[r][c]);
                af[mi][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][c]);
                af[mi][2] = *reinterpret_cast<const uint32_t *>(&As[r][c + 8]);
                af[mi][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][c + 8]);
            }
#pragma unroll
            for (int ni = 0; ni < 4; ++ni) {
                const int n = wn + ni * 8 + g;
                const int k = kk + tg * 2;
                bfr[ni][0] = pack_bf16(__bfloat162float(Bs[k][n]), __bfloat162float(Bs[k + 1][n]));
                bfr[ni][1] = pack_bf16(__bfloat162float(Bs[k + 8][n]), __bfloat162float(Bs[k + 9][n]));
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                        : "+f"(acc[mi][ni][0]), "+f"(acc[mi][ni][1]), "+f"(acc[mi][ni][2]),
                          "+f"(acc[mi][ni][3])
                        : "r"(af[mi][0]), "r"(af[mi][1]), "r"(af[mi][2]), "r"(af[mi][3]),
                          "r"(bfr[ni][0]), "r"(bfr[ni][1]));
        }
        __syncthreads();
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int r = m0 + wm + mi * 16 + g + (h >= 2 ? 8 : 0);
                const int c = n0 + wn + ni * 8 + tg * 2 + (h & 1);
                if (r >= M || c >= N)
                    continue;
                float v = acc[mi][ni][h];
                if (bias)
                    v += bias[c];
                if (epi == 1)
                    v = fmaxf(v, 0.f);
                else if (epi == 2)
                    v = mask[r * ldm + c] > 0.f ? v : 0.f;
                float *dst = C + r * ldc + c;
                *dst = beta != 0.f ? beta * *dst + v : v;
            }
}

// Column sums: out[c] = sum_r X[r * ld + c] (bias gradients).
__global__ void k_colsum(const float *X, long long ld, int M, int N, float *out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N)
        return;
    float s = 0.f;
    for (int r = 0; r < M; ++r)
        s += X[r * ld + c];
    out[c] = s;
}

// Loss of the direction offsets: mean over the batch and the K outputs of
// (tanh(y) - t)^2; writes dL/dy and accumulates the loss.
__global__ void k_tanh_mse(const float *Y, const float *T, int count, float *dY, float *loss)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count)
        return;
    const float th = tanhf(Y[i]);
    const float d = th - T[i];
    dY[i] = 2.f * d * (1.f - th * th) / (float)count;
    atomicAdd(loss, d * d / (float)count);
}

// Adam on the flat parameter vector (bias-corrected step size lr_t).
__global__ void k_adam(float *w, const float *g, float *m, float *v, long long n, float lr_t,
                       float b1, float b2, float eps)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr_t * mi / (sqrtf(vi) + eps);
    }
}

}  // namespace

cudaError_t gemm_launch(const float *A, long long a_sr, long long a_sc, const float *B, long long b_sr,
                        long long b_sc, float *C, long long ldc, int M, int N, int K,
                        const float *bias, int epi, const float *mask, long long ldm, float beta,
                        cudaStream_t s)
{
    if (M <= 0 || N <= 0)
        return cudaSuccess;
    dim3 grid((N + GN - 1) / GN, (M + GM - 1) / GM);
    k_gemm<<<grid, GT, 0, s>>>(Mat{A, a_sr, a_sc}, Mat{B, b_sr, b_sc}, C, ldc, M, N, K, bias, epi,
                               mask, ldm, beta);
    return cudaGetLastError();
}

cudaError_t colsum_launch(const float *X, long long ld, int M, int N, float *out, cudaStream_t s)
{
    k_colsum<<<(N + 127) / 128, 128, 0, s>>>(X, ld, M, N, out);
    return cudaGetLastError();
}

cudaError_t tanh_mse_launch(const float *Y, const float *T, int count, float *dY, float *loss,
                            cudaStream_t s)
{
    k_tanh_mse<<<(count + 255) / 256, 256, 0, s>>>(Y, T, count, dY, loss);
    return cudaGetLastError();
}

cudaError_t adam_launch(float *w, const float *g, float *m, float *v, long long n, float lr_t,
                        float b1, float b2, float eps, cudaStream_t s)
{
    k_adam<<<std::max(1, std::min((int)((n + 255) / 256), sm_count() * 4)), 256, 0, s>>>(
        w, g, m, v, n, lr_t, b1, b2, eps);
    return cudaGetLastError();
}

}  // namespace ch
