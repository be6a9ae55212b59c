// The learned culling proposal (no counterpart in the paper; it serves the
// paper's culling idea): a convex polygon whose vertices are input points
// lies inside the hull, so points strictly inside it are not hull vertices
// and Algorithm 1 may start each column of L from the polygon's interior
// span instead of (p+1, -1).  Whatever the polygon, the hull is unchanged.
//
// k_sample_hist  occupancy histogram of a sample of the input (runs of
//                CH_CULL_RUN consecutive points at CH_CULL_RUNS evenly spaced
//                starts): 32 x 32 cells, one row of counts per CTA;
// k_gemv1/2      the network's two hidden layers for one input vector
//                (operands rounded to bf16, fp32 accumulation, as the
//                training GEMMs do; a CTA owns 32 outputs x 64 inputs and
//                writes a partial sum, summed in fixed order by the next
//                layer, so the result is deterministic);
// k_extremes     output layer, directions theta_k = 2 pi k / K +
//                (pi / K) tanh(y_k), and per CTA the sample point with the
//                largest fl32(c_k x + s_k y) (two rounded products, one
//                rounded sum; ties to the smaller index) for each k, for the
//                network's directions and for the sector centres;
// k_cull_init    every CTA folds the per-CTA winners, takes the strict hull
//                of each set's K winners in one warp (exact int64
//                orientation), keeps the polygon of larger area (exact, ties
//                to the sector centres), and writes for its columns the
//                start array Linit, L = Linit and
//                the filtered reduction's row-bin filter (tightening the
//                warm-up filter when there is one).
// The reduction then runs unchanged from that filter and start array, and
// the chain step keeps a lower (upper) point only where L moved below
// (above) Linit.
#include <cuda_bf16.h>
#include <math_constants.h>

#include "ch_internal.cuh"

namespace ch {
namespace {

constexpr int SR = CH_CULL_RUN, SJ = CH_CULL_RUNS;
constexpr int NI = CH_MLP_IN, NH = CH_MLP_HID, NK = CH_MLP_K;
constexpr int HB = 32;                   // histogram CTAs (rows of counts)
constexpr int HU = (SJ + HB - 1) / HB;   // runs per histogram CTA
constexpr int KC = 64;                   // inputs per CTA of a hidden layer
constexpr int KS1 = NI / KC, KS2 = NH / KC;
constexpr int EXB = 32, EXT = 256;       // extremes CTAs x threads (k_cull_init folds EXB candidates per direction)
constexpr int EXU = 8;                   // sample points in flight per thread
constexpr long long NONE = 0x7FFFFFFFFFFFFFFFll;
static_assert(SR == NI, "one histogram cell per thread");
static_assert(NK == 16 && NH == 256, "layer shapes");

// parameter offsets (same layout as the C ABI's parameter vector)
constexpr long long OFF_W1 = 0, OFF_B1 = OFF_W1 + (long long)NI * NH;
constexpr long long OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + (long long)NH * NH;
constexpr long long OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + (long long)NH * NK;

struct Cand {
    float score;
    int pad;
    long long idx;
};

__host__ __device__ __forceinline__ void sample_shape(long long n, long long &nruns, long long &step)
{
    if (n <= (long long)SR * SJ) {
        nruns = (n + SR - 1) / SR;
        step = SR;
    } else {
        nruns = SJ;
        step = n / SJ;
    }
}

__host__ __device__ __forceinline__ long long sample_size(long long n)
{
    return n <= (long long)SR * SJ ? n : (long long)SR * SJ;
}

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__device__ __forceinline__ bool better(float s, long long i, float bs, long long bi)
{
    return s > bs || (s == bs && i < bi);
}

// ------------------------------------------------------------- histogram
__global__ void __launch_bounds__(SR) k_sample_hist(const int2 *__restrict__ pts, long long n, int p,
                                                    int *__restrict__ rows)
{
    pdl_wait();
    pdl_trigger();
    __shared__ int h[NI];
    h[threadIdx.x] = 0;
    __syncthreads();
    long long nruns, step;
    sample_shape(n, nruns, step);
    int2 q[HU];
    bool have[HU];
#pragma unroll
    for (int u = 0; u < HU; ++u) {
        const long long r = blockIdx.x + (long long)u * HB;
        const long long i = r * step + threadIdx.x;
        have[u] = r < nruns && i < n && threadIdx.x < SR;
        q[u] = have[u] ? pts[i] : make_int2(0, 0);
    }
    const unsigned up = (unsigned)p;
#pragma unroll
    for (int u = 0; u < HU; ++u) {
        // points outside [1,p]^2 are left out here; the reduction reports them
        if (have[u] && (unsigned)(q[u].x - 1) < up && (unsigned)(q[u].y - 1) < up) {
            int bx, by;
            if (up <= (1u << 27)) {  // (x-1) * 32 fits 32 bits: the cheap division
                bx = (int)(((unsigned)(q[u].x - 1) * 32u) / up);
                by = (int)(((unsigned)(q[u].y - 1) * 32u) / up);
            } else {
                bx = (int)(((unsigned long long)(q[u].x - 1) * 32ull) / up);
                by = (int)(((unsigned long long)(q[u].y - 1) * 32ull) / up);
            }
            atomicAdd(&h[by * 32 + bx], 1);
        }
    }
    __syncthreads();
    rows[blockIdx.x * NI + threadIdx.x] = h[threadIdx.x];
}

// features[i] = fl32(count_i * fl32(1024 / m)) (diagnostic output only)
__global__ void k_features(const int *__restrict__ rows, float scale, float *__restrict__ X)
{
    pdl_wait();
    pdl_trigger();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NI)
        return;
    int c = 0;
#pragma unroll
    for (int r = 0; r < HB; ++r)
        c += rows[r * NI + i];
    X[i] = (float)c * scale;
}

// ------------------------------------------------------------- network
// Layer 1: partial[kc][j] = sum over the 64 inputs of chunk kc of
// bf16(x_k) * bf16(W1[k][j]), x_k = count_k * scale.
__global__ void __launch_bounds__(256)
    k_gemv1(const int *__restrict__ rows, float scale, const float *__restrict__ W,
            float *__restrict__ part)
{
    pdl_wait();
    pdl_trigger();
    __shared__ float xs[KC];
    __shared__ float red[8][32];
    const int jc = blockIdx.x, kc = blockIdx.y;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t < KC) {
        const int k = kc * KC + t;
        int c[HB];
#pragma unroll
        for (int r = 0; r < HB; ++r)
            c[r] = rows[r * NI + k];
        int s = 0;
#pragma unroll
        for (int r = 0; r < HB; ++r)
            s += c[r];
        xs[t] = bf16r((float)s * scale);
    }
    const int j = jc * 32 + lane;
    float wv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
        wv[u] = bf16r(W[OFF_W1 + (long long)(kc * KC + w * 8 + u) * NH + j]);
    __syncthreads();
    float acc = 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u)
        acc = fmaf(xs[w * 8 + u], wv[u], acc);
    red[w][lane] = acc;
    __syncthreads();
    if (t < 32) {
        float s = 0.f;
#pragma unroll
        for (int v = 0; v < 8; ++v)
            s += red[v][t];
        part[kc * NH + jc * 32 + t] = s;
    }
}

// Layer 2 from layer 1's partials: h1 = relu(sum + b1), same scheme.
__global__ void __launch_bounds__(256)
    k_gemv2(const float *__restrict__ part1, const float *__restrict__ W, float *__restrict__ part2)
{
    pdl_wait();
    pdl_trigger();
    __shared__ float hs[KC];
    __shared__ float red[8][32];
    const int jc = blockIdx.x, kc = blockIdx.y;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t < KC) {
        const int k = kc * KC + t;
        float v[KS1];
#pragma unroll
        for (int q = 0; q < KS1; ++q)
            v[q] = part1[q * NH + k];
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < KS1; ++q)
            s += v[q];
        hs[t] = bf16r(fmaxf(s + W[OFF_B1 + k], 0.f));
    }
    const int j = jc * 32 + lane;
    float wv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
        wv[u] = bf16r(W[OFF_W2 + (long long)(kc * KC + w * 8 + u) * NH + j]);
    __syncthreads();
    float acc = 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u)
        acc = fmaf(hs[w * 8 + u], wv[u], acc);
    red[w][lane] = acc;
    __syncthreads();
    if (t < 32) {
        float s = 0.f;
#pragma unroll
        for (int v = 0; v < 8; ++v)
            s += red[v][t];
        part2[kc * NH + jc * 32 + t] = s;
    }
}

// ------------------------------------------------------------- extremes
// Direction set 0 is the sector centres theta_k = 2 pi k / K; set 1 (only
// with a network) adds (pi / K) tanh(y_k).  Each set's winners go to
// cand[(set * gridDim.x + CTA) * K + k] and its directions to dirs[set].
__global__ void __launch_bounds__(EXT)
    k_extremes(const int2 *__restrict__ pts, long long n, const float *__restrict__ part2,
               const float *__restrict__ W, Cand *__restrict__ cand, float *y_out, float *dirs)
{
    pdl_wait();
    pdl_trigger();
    __shared__ float h2[NH];
    __shared__ float red[16][NK];
    __shared__ float s_c[2][NK], s_s[2][NK];
    __shared__ float s_best[EXT / 32][NK];
    __shared__ long long s_idx[EXT / 32][NK];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int nsets = W ? 2 : 1;
    if (W) {
        float v[KS2];
#pragma unroll
        for (int q = 0; q < KS2; ++q)
            v[q] = part2[q * NH + t];
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < KS2; ++q)
            s += v[q];
        h2[t] = bf16r(fmaxf(s + W[OFF_B2 + t], 0.f));
        __syncthreads();
        const int k = t & (NK - 1), js = t >> 4;
        float acc = 0.f;
#pragma unroll
        for (int u = 0; u < 16; ++u)
            acc = fmaf(h2[js * 16 + u], bf16r(W[OFF_W3 + (long long)(js * 16 + u) * NK + k]), acc);
        red[js][k] = acc;
        __syncthreads();
    }
    if (t < 2 * NK) {
        const int set = t / NK, k = t % NK;
        float th = 0.f;
        if (set == 1 && W) {
            float y = 0.f;
#pragma unroll
            for (int js = 0; js < 16; ++js)
                y += red[js][k];
            y += W[OFF_B3 + k];
            th = tanhf(y);
            if (!(fabsf(th) <= 1.f))
                th = 0.f;  // a non-finite output falls back to the sector centre
            if (blockIdx.x == 0 && y_out)
                y_out[k] = y;
        }
        const float theta = (float)(2.0 * CUDART_PI / NK) * (float)k + (float)(CUDART_PI / NK) * th;
        float sn, cs;
        sincosf(theta, &sn, &cs);
        s_c[set][k] = cs;
        s_s[set][k] = sn;
        if (blockIdx.x == 0 && set < nsets) {
            dirs[set * 2 * NK + k] = cs;
            dirs[set * 2 * NK + NK + k] = sn;
        }
    }
    __syncthreads();
    long long nruns, step;
    sample_shape(n, nruns, step);
    const long long m = sample_size(n);
    const long long stride = (long long)gridDim.x * EXT;
    for (int set = 0; set < nsets; ++set) {
        float c[NK], s[NK], best[NK];
        long long bi[NK];
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            c[k] = s_c[set][k];
            s[k] = s_s[set][k];
            best[k] = -CUDART_INF_F;
            bi[k] = NONE;
        }
        for (long long q0 = (long long)blockIdx.x * EXT + t; q0 < m; q0 += stride * EXU) {
            int2 v[EXU];
            long long gi[EXU];
#pragma unroll
            for (int u = 0; u < EXU; ++u) {
                const long long q = q0 + u * stride;
                gi[u] = (q / SR) * step + (q % SR);
                v[u] = q < m ? pts[gi[u]] : make_int2(0, 0);
            }
#pragma unroll
            for (int u = 0; u < EXU; ++u) {
                if (q0 + u * stride >= m)
                    break;
                const float xf = __int2float_rn(v[u].x), yf = __int2float_rn(v[u].y);
#pragma unroll
                for (int k = 0; k < NK; ++k) {
                    const float sc = __fadd_rn(__fmul_rn(c[k], xf), __fmul_rn(s[k], yf));
                    if (sc > best[k]) {  // visits increase in index: ties keep the first
                        best[k] = sc;
                        bi[k] = gi[u];
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NK; ++k) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xFFFFFFFFu, best[k], o);
                const long long oi = __shfl_xor_sync(0xFFFFFFFFu, bi[k], o);
                if (better(ob, oi, best[k], bi[k])) {
                    best[k] = ob;
                    bi[k] = oi;
                }
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                s_best[w][k] = best[k];
                s_idx[w][k] = bi[k];
            }
        }
        __syncthreads();
        if (t < NK) {
            float b = s_best[0][t];
            long long i = s_idx[0][t];
            for (int v = 1; v < EXT / 32; ++v)
                if (better(s_best[v][t], s_idx[v][t], b, i)) {
                    b = s_best[v][t];
                    i = s_idx[v][t];
                }
            cand[((size_t)set * gridDim.x + blockIdx.x) * NK + t] = Cand{b, 0, i};
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------- polygon
__device__ __forceinline__ long long floor_div(long long a, long long b)  // b > 0
{
    const long long q = a / b;
    return (a % b != 0 && a < 0) ? q - 1 : q;
}

__device__ __forceinline__ long long ceil_div(long long a, long long b)  // b > 0
{
    const long long q = a / b;
    return (a % b != 0 && a > 0) ? q + 1 : q;
}

// Value of the chain V[0..nv) (x non-decreasing, V[0].x < x < V[nv-1].x) at
// column x as a fraction num / den, den > 0.
__device__ __forceinline__ void chain_at(const int2 *V, int nv, int x, long long &num, long long &den)
{
    int j = 0;
    for (int k = 1; k < nv - 1; ++k)
        if (V[k].x <= x)
            j = k;
    const int2 a = V[j], b = V[j + 1];
    den = (long long)b.x - a.x;
    num = (long long)a.y * ((long long)b.x - x) + (long long)b.y * ((long long)x - a.x);
}

// Twice the signed area of the polygon s_lo[0..nlo) ++ s_up[nup-2..1]
// (counter-clockwise), exact.
__device__ __forceinline__ __int128 area2(const int2 *lo, int nlo, const int2 *up, int nup)
{
    __int128 a = 0;
    const int nv = nlo + nup - 2;
    if (nv < 3)
        return 0;
    const int2 o = lo[0];
    auto vert = [&](int i) { return i < nlo ? lo[i] : up[nup - 2 - (i - nlo)]; };
    for (int i = 0; i < nv; ++i) {
        const int2 u = vert(i), v = vert(i + 1 < nv ? i + 1 : 0);
        a += (__int128)((long long)u.x - o.x) * ((long long)v.y - o.y) -
             (__int128)((long long)u.y - o.y) * ((long long)v.x - o.x);
    }
    return a;
}

// nsets = 1: the sector-centre polygon; nsets = 2: also the network's, and
// the one of larger area is used (ties: the sector centres), so the network
// can only enlarge the culled region.
__global__ void __launch_bounds__(256)
    k_cull_init(const int2 *__restrict__ pts, const Cand *__restrict__ cand, int ncand, int nsets,
                int p, int2 *Linit, int2 *L, uint16_t *G, bool G_warm, int shift,
                unsigned long long *zero, int nzero, const float *dirs_in, float *dirs_out,
                int2 *poly_out, int *poly_count, long long *ext_out, int *chosen)
{
    pdl_wait();
    pdl_trigger();
    __shared__ long long s_idx[2][NK];
    __shared__ int2 s_sorted[2][NK];
    __shared__ int2 s_lo2[2][NK], s_up2[2][NK];
    __shared__ int s_nlo[2], s_nup[2], s_m[2];
    __shared__ int s_sel;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (zero && blockIdx.x == 0)
        for (int i = t; i < nzero; i += blockDim.x)
            zero[i] = 0;
    // winner of each direction over the extremes CTAs: warp w takes k = 2w, 2w+1
    for (int set = 0; set < nsets; ++set) {
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            const int k = 2 * w + kk;
            float b = -CUDART_INF_F;
            long long bi = NONE;
            for (int r = lane; r < ncand; r += 32) {
                const Cand cd = cand[((size_t)set * ncand + r) * NK + k];
                if (better(cd.score, cd.idx, b, bi)) {
                    b = cd.score;
                    bi = cd.idx;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xFFFFFFFFu, b, o);
                const long long oi = __shfl_xor_sync(0xFFFFFFFFu, bi, o);
                if (better(ob, oi, b, bi)) {
                    b = ob;
                    bi = oi;
                }
            }
            if (lane == 0)
                s_idx[set][k] = bi;
        }
    }
    __syncthreads();
    // strict hull of each set's winners (warp `set`; lane k holds winner k)
    if (w < nsets) {
        const int set = w;
        int2 *srt = s_sorted[set];
        const long long my = lane < NK ? s_idx[set][lane] : NONE;
        const bool have = my != NONE;
        const int2 P = have ? pts[my] : make_int2(0, 0);
        const unsigned hv = __ballot_sync(0xFFFFFFFFu, have);
        bool dup = false;
        for (int j = 0; j < NK; ++j) {
            const int qx = __shfl_sync(0xFFFFFFFFu, P.x, j), qy = __shfl_sync(0xFFFFFFFFu, P.y, j);
            dup |= have && ((hv >> j) & 1u) && j < lane && qx == P.x && qy == P.y;
        }
        const bool keep = have && !dup;
        const unsigned kv = __ballot_sync(0xFFFFFFFFu, keep);
        int rank = 0;
        for (int j = 0; j < NK; ++j) {
            const int qx = __shfl_sync(0xFFFFFFFFu, P.x, j), qy = __shfl_sync(0xFFFFFFFFu, P.y, j);
            rank += keep && ((kv >> j) & 1u) && (qx < P.x || (qx == P.x && qy < P.y));
        }
        if (keep)
            srt[rank] = P;
        __syncwarp();
        const int m = __popc(kv);
        // lane i (< m): sorted point i is a strict lower (upper) hull vertex
        // when it lies strictly below (above) every segment joining a point
        // before it to a point after it; the end points belong to both
        bool lo = false, upf = false;
        if (lane < m) {
            const int2 q = srt[lane];
            lo = upf = true;
            if (lane > 0 && lane < m - 1) {
                for (int a = 0; a < lane; ++a)
                    for (int b = lane + 1; b < m; ++b) {
                        const long long cr = cross3(srt[a], srt[b], q);
                        lo &= cr < 0;
                        upf &= cr > 0;
                    }
            }
        }
        const unsigned bl = __ballot_sync(0xFFFFFFFFu, lo), bu = __ballot_sync(0xFFFFFFFFu, upf);
        const unsigned below = (1u << lane) - 1u;
        if (lo)
            s_lo2[set][__popc(bl & below)] = srt[lane];
        if (upf)
            s_up2[set][__popc(bu & below)] = srt[lane];
        if (lane == 0) {
            s_nlo[set] = __popc(bl);
            s_nup[set] = __popc(bu);
            s_m[set] = m;
        }
    }
    __syncthreads();
    if (t == 0) {
        int sel = 0;
        if (nsets == 2 && area2(s_lo2[1], s_m[1] <= 1 ? 0 : s_nlo[1], s_up2[1], s_nup[1]) >
                              area2(s_lo2[0], s_m[0] <= 1 ? 0 : s_nlo[0], s_up2[0], s_nup[0]))
            sel = 1;
        s_sel = sel;
    }
    __syncthreads();
    const int sel = s_sel;
    const int2 *s_lo = s_lo2[sel], *s_up = s_up2[sel];
    const int nlo = s_nlo[sel], nup = s_nup[sel], m = s_m[sel];
    const int nv = m <= 1 ? m : nlo + nup - 2;  // strict vertices of the polygon
    if (blockIdx.x == 0) {
        if (t < 2 * NK && ext_out) {  // both sets: [set][k]
            const int set = t / NK;
            ext_out[t] = set >= nsets || s_idx[set][t % NK] == NONE ? -1 : s_idx[set][t % NK];
        }
        if (t < 4 * NK && dirs_out)  // both sets: [set][cos k | sin k]
            dirs_out[t] = t < nsets * 2 * NK ? dirs_in[t] : 0.f;
        if (poly_out && t == 0) {
            // counter-clockwise from the lexicographic minimum
            int o = 0;
            for (int i = 0; i < (m <= 1 ? m : nlo); ++i)
                poly_out[o++] = s_lo[i];
            for (int i = nup - 2; i >= 1; --i)
                poly_out[o++] = s_up[i];
        }
        if (poly_count && t == 0)
            *poly_count = nv;
        if (chosen && t == 0)
            *chosen = nsets == 2 ? sel : -1;
    }
    const int c = blockIdx.x * blockDim.x + t;
    if (c >= p)
        return;
    const int x = c + 1;
    int2 li = make_int2(p + 1, -1);
    if (nv >= 3 && x > s_lo[0].x && x < s_lo[nlo - 1].x) {
        long long num, den;
        chain_at(s_lo, nlo, x, num, den);
        const long long lo0 = floor_div(num, den) + 1;
        chain_at(s_up, nup, x, num, den);
        const long long hi0 = ceil_div(num, den) - 1;
        li = make_int2((int)lo0, (int)hi0);
    }
    if (Linit)
        Linit[c] = li;
    if (L)
        L[c] = li;
    if (G) {
        // pass every point that could move L below li.x or above li.y; the
        // warm-up filter already in G is another such bound, so keep the
        // tighter of the two (each is the bin of a value every point that
        // can set the final L.lo is at or below, likewise for L.hi)
        const unsigned top = (unsigned)(p - 1) >> shift;
        unsigned qlo = li.x <= 1 ? 0u : (unsigned)(li.x - 2) >> shift;
        unsigned qhi = li.y + 1 < 1 ? 0u : (li.y + 1 > p ? top : (unsigned)li.y >> shift);
        if (G_warm) {
            const unsigned g = G[c];
            qlo = min(qlo, g >> 8);
            qhi = max(qhi, g & 0xFFu);
        }
        G[c] = (uint16_t)((qlo << 8) | qhi);
    }
}

// Points strictly inside the culling polygon (Linit.lo <= y <= Linit.hi in
// their column); points outside [1,p]^2 are not counted.  Adds to *culled.
__global__ void __launch_bounds__(256)
    k_cull_count(const int2 *__restrict__ pts, long long n, int p, const int2 *__restrict__ Linit,
                 unsigned long long *culled)
{
    pdl_wait();
    pdl_trigger();
    unsigned long long k = 0;
    const unsigned up = (unsigned)p;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int2 q = __ldcs(pts + i);
        const unsigned c = (unsigned)(q.x - 1);
        if (c < up && (unsigned)(q.y - 1) < up) {
            const int2 li = __ldg(Linit + c);
            k += (li.x <= q.y && q.y <= li.y) ? 1ull : 0ull;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        k += __shfl_xor_sync(0xFFFFFFFFu, k, o);
    if ((threadIdx.x & 31) == 0 && k)
        atomicAdd(culled, k);
}

}  // namespace

cudaError_t cull_count_launch(const int32_t *pts, int64_t n, int p, const int32_t *Linit,
                              unsigned long long *culled, cudaStream_t s)
{
    const long long blocks = std::min<long long>((n + 255) / 256, (long long)sm_count() * 8);
    if (blocks > 0)
        launch(k_cull_count, (int)blocks, 256, 0, s, reinterpret_cast<const int2 *>(pts), (long long)n,
               p, reinterpret_cast<const int2 *>(Linit), culled);
    return cudaGetLastError();
}

size_t cull_ws_bytes(int p)
{
    (void)p;
    WsLayout l;
    l.take((size_t)HB * NI * sizeof(int));
    l.take((size_t)KS1 * NH * sizeof(float));
    l.take((size_t)KS2 * NH * sizeof(float));
    l.take((size_t)2 * EXB * NK * sizeof(Cand));
    l.take((size_t)2 * 2 * NK * sizeof(float));
    return l.off;
}

cudaError_t cull_launch(const int32_t *pts, int64_t n, int p, const float *params, void *ws,
                        int32_t *Linit, int32_t *L, uint16_t *G, bool G_warm, int shift,
                        unsigned long long *zero, int nzero, float *features, float *y_out,
                        float *dirs_out, int32_t *poly_out, int32_t *poly_count, int64_t *ext_out,
                        int32_t *chosen, cudaStream_t s)
{
    WsLayout l;
    char *b = reinterpret_cast<char *>(ws);
    int *rows = reinterpret_cast<int *>(b + l.take((size_t)HB * NI * sizeof(int)));
    float *part1 = reinterpret_cast<float *>(b + l.take((size_t)KS1 * NH * sizeof(float)));
    float *part2 = reinterpret_cast<float *>(b + l.take((size_t)KS2 * NH * sizeof(float)));
    Cand *cand = reinterpret_cast<Cand *>(b + l.take((size_t)2 * EXB * NK * sizeof(Cand)));
    float *dirs = reinterpret_cast<float *>(b + l.take((size_t)2 * 2 * NK * sizeof(float)));
    const int2 *P = reinterpret_cast<const int2 *>(pts);
    const long long m = sample_size(n);
    const float scale = m > 0 ? 1024.0f / (float)m : 0.f;
    if (params || features) {
        launch(k_sample_hist, HB, SR, 0, s, P, n, p, rows);
        if (features)
            launch(k_features, NI / 256, 256, 0, s, rows, scale, features);
    }
    if (params) {
        launch(k_gemv1, dim3(NH / 32, KS1), 256, 0, s, rows, scale, params, part1);
        launch(k_gemv2, dim3(NH / 32, KS2), 256, 0, s, part1, params, part2);
    }
    launch(k_extremes, EXB, EXT, 0, s, P, n, part2, params, cand, y_out, dirs);
    launch(k_cull_init, (p + 255) / 256, 256, 0, s, P, cand, EXB, params ? 2 : 1, p,
           reinterpret_cast<int2 *>(Linit), reinterpret_cast<int2 *>(L), G, G_warm, shift, zero,
           nzero, dirs, dirs_out, reinterpret_cast<int2 *>(poly_out), poly_count,
           reinterpret_cast<long long *>(ext_out), chosen);
    return cudaGetLastError();
}

int cull_kernel_count(bool net) { return net ? 5 : 2; }

}  // namespace ch
