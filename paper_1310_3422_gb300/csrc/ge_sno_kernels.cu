// ge_sno_kernels.cu -- kernels of the spectral neural operator (the learned
// surrogate that jumps K GE steps ahead): a batched tensor-core GEMM with
// fused epilogues, and the elementwise pieces of the forward and backward
// passes and of Adam.
//
// GEMM: C[b] = alpha * (op(A[b]) op(B[b]) [+ op(A2[b]) op(B2[b])]) + beta *
// C0[b] + bias, FP32 in global memory, operands rounded to BF16 (round to
// nearest even) while staged into shared memory (float4 loads along the
// unit-stride dimension where the layout allows), products on the tensor
// cores (mma.sync m16n8k16, FP32 accumulate).  The second product lets two
// GEMMs into the same output (the inverse DFT and the pointwise path of a
// layer) run as one pass; the epilogue can multiply by GELU' of a stored
// pre-activation (backward) and store GELU of the result (forward), so no
// separate activation pass touches HBM.  Split mode (SPLIT = true) also
// stages the BF16 residual of every operand and adds the two cross products
// (x = hi + lo, x*y ~ hi*hi + hi*lo + lo*hi), which is accurate to about
// 1e-5 relative: it lets the network's gradients be checked against an FP64
// reference.
#include <cuda_bf16.h>
#include <cstdint>

#include "ge_sno_internal.h"

namespace ge {
namespace {

constexpr int BM = 64, BN = 64, BK = 32, PADK = BK + 8;  // bf16 elements per smem row
constexpr int NT = 128;                                  // threads per GEMM CTA

__device__ __forceinline__ float gelu(float x)
{
    // tanh form of GELU
    const float k0 = 0.7978845608028654f, k1 = 0.044715f;
    return 0.5f * x * (1.0f + tanhf(k0 * (x + k1 * x * x * x)));
}

__device__ __forceinline__ float gelu_grad(float x)
{
    const float k0 = 0.7978845608028654f, k1 = 0.044715f;
    const float u = k0 * (x + k1 * x * x * x);
    const float th = tanhf(u);
    const float du = k0 * (1.0f + 3.0f * k1 * x * x);
    return 0.5f * (1.0f + th) + 0.5f * x * (1.0f - th * th) * du;
}

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    const uint16_t a = *reinterpret_cast<const uint16_t *>(&lo);
    const uint16_t b = *reinterpret_cast<const uint16_t *>(&hi);
    return (uint32_t)a | ((uint32_t)b << 16);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <bool SPLIT>
__device__ __forceinline__ void put(__nv_bfloat16 (*S)[BM][PADK], int r, int kk, float x)
{
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    S[0][r][kk] = h;
    if (SPLIT)
        S[SPLIT ? 1 : 0][r][kk] = __float2bfloat16_rn(x - __bfloat162float(h));
}

// Stage the 64 x BK tile of an operand whose element (row, k) is
// X[row * s_r + k * s_k] (rows r0.., rows < rmax and k0.. < kend are read,
// the rest is zero) as S[.][row - r0][k - k0].  The element order follows
// the unit-stride dimension so a warp's loads coalesce; `vec` (checked by
// the launcher: that dimension's extent, the other stride and the base all
// multiples of 4 floats / 16 bytes) loads four elements at once.
template <bool SPLIT>
__device__ __forceinline__ void stage(__nv_bfloat16 (*S)[BM][PADK], const float *__restrict__ X, long long s_r,
                                      long long s_k, int r0, int rmax, int k0, int kend, bool vec, int t)
{
    if (s_k == 1) {
        if (vec) {
            for (int e = t; e < BM * BK / 4; e += NT) {
                const int r = e / (BK / 4), kk = (e % (BK / 4)) * 4;
                const int row = r0 + r, k = k0 + kk;
                float4 x = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (row < rmax && k < kend)
                    x = __ldg(reinterpret_cast<const float4 *>(X + (long long)row * s_r + k));
                put<SPLIT>(S, r, kk, x.x);
                put<SPLIT>(S, r, kk + 1, x.y);
                put<SPLIT>(S, r, kk + 2, x.z);
                put<SPLIT>(S, r, kk + 3, x.w);
            }
        } else {
            for (int e = t; e < BM * BK; e += NT) {
                const int r = e / BK, kk = e % BK;
                const int row = r0 + r, k = k0 + kk;
                put<SPLIT>(S, r, kk, (row < rmax && k < kend) ? __ldg(X + (long long)row * s_r + k) : 0.0f);
            }
        }
    } else {
        if (vec) {
            for (int e = t; e < BM * BK / 4; e += NT) {
                const int r = (e % (BM / 4)) * 4, kk = e / (BM / 4);
                const int row = r0 + r, k = k0 + kk;
                float4 x = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (row < rmax && k < kend)
                    x = __ldg(reinterpret_cast<const float4 *>(X + row + (long long)k * s_k));
                put<SPLIT>(S, r, kk, x.x);
                put<SPLIT>(S, r + 1, kk, x.y);
                put<SPLIT>(S, r + 2, kk, x.z);
                put<SPLIT>(S, r + 3, kk, x.w);
            }
        } else {
            for (int e = t; e < BM * BK; e += NT) {
                const int r = e % BM, kk = e / BM;
                const int row = r0 + r, k = k0 + kk;
                put<SPLIT>(S, r, kk,
                           (row < rmax && k < kend) ? __ldg(X + (long long)row * s_r + (long long)k * s_k) : 0.0f);
            }
        }
    }
}

// 64x64 output tile per CTA, 4 warps (2 x 2), each warp 32x32 = 2 x 4 mma tiles.
template <bool SPLIT>
__global__ void __launch_bounds__(NT) gemm_kernel(GemmArgs g)
{
    __shared__ __nv_bfloat16 As[SPLIT ? 2 : 1][BM][PADK];
    __shared__ __nv_bfloat16 Bs[SPLIT ? 2 : 1][BN][PADK];
    const int ks_n = g.ksplit > 1 ? g.ksplit : 1;
    const int bz = blockIdx.z / ks_n, kslice = blockIdx.z % ks_n;
    const int i0 = blockIdx.y * BM, j0 = blockIdx.x * BN;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int grp = lane >> 2, tig = lane & 3;

    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c)
                acc[a][b][c] = 0.0f;

    for (int seg = 0; seg < 2; ++seg) {
        const float *A, *Bm;
        long long la_i, la_k, lb_k, lb_j;
        int kbeg, kend;
        bool va, vb;
        if (seg == 0) {
            const int kchunk = ((g.K + ks_n - 1) / ks_n + BK - 1) / BK * BK;
            kbeg = kslice * kchunk;
            kend = (kbeg + kchunk < g.K) ? kbeg + kchunk : g.K;
            A = g.A + (long long)bz * g.sA;
            Bm = g.B + (long long)bz * g.sB;
            la_i = g.lda_i, la_k = g.lda_k, lb_k = g.ldb_k, lb_j = g.ldb_j;
            va = g.vec[0] != 0, vb = g.vec[1] != 0;
        } else {
            if (!g.A2 || g.K2 <= 0)
                break;
            kbeg = 0;
            kend = g.K2;
            A = g.A2 + (long long)bz * g.sA2;
            Bm = g.B2 + (long long)bz * g.sB2;
            la_i = g.lda2_i, la_k = g.lda2_k, lb_k = g.ldb2_k, lb_j = g.ldb2_j;
            va = g.vec[2] != 0, vb = g.vec[3] != 0;
        }
        for (int k0 = kbeg; k0 < kend; k0 += BK) {
            stage<SPLIT>(As, A, la_i, la_k, i0, g.M, k0, kend, va, t);
            stage<SPLIT>(Bs, Bm, lb_j, lb_k, j0, g.N, k0, kend, vb, t);
            __syncthreads();
#pragma unroll
            for (int ks = 0; ks < BK; ks += 16) {
                uint32_t af[SPLIT ? 2 : 1][2][4], bf[SPLIT ? 2 : 1][4][2];
#pragma unroll
                for (int s = 0; s < (SPLIT ? 2 : 1); ++s) {
#pragma unroll
                    for (int mi = 0; mi < 2; ++mi) {
                        const int r = wm + mi * 16 + grp;
                        const int kc = ks + tig * 2;
                        af[s][mi][0] = pack_bf16(As[s][r][kc], As[s][r][kc + 1]);
                        af[s][mi][1] = pack_bf16(As[s][r + 8][kc], As[s][r + 8][kc + 1]);
                        af[s][mi][2] = pack_bf16(As[s][r][kc + 8], As[s][r][kc + 9]);
                        af[s][mi][3] = pack_bf16(As[s][r + 8][kc + 8], As[s][r + 8][kc + 9]);
                    }
#pragma unroll
                    for (int ni = 0; ni < 4; ++ni) {
                        const int c = wn + ni * 8 + grp;
                        const int kc = ks + tig * 2;
                        bf[s][ni][0] = pack_bf16(Bs[s][c][kc], Bs[s][c][kc + 1]);
                        bf[s][ni][1] = pack_bf16(Bs[s][c][kc + 8], Bs[s][c][kc + 9]);
                    }
                }
#pragma unroll
                for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                    for (int ni = 0; ni < 4; ++ni) {
                        mma_bf16(acc[mi][ni], af[0][mi], bf[0][ni]);
                        if (SPLIT) {
                            mma_bf16(acc[mi][ni], af[0][mi], bf[SPLIT ? 1 : 0][ni]);
                            mma_bf16(acc[mi][ni], af[SPLIT ? 1 : 0][mi], bf[0][ni]);
                        }
                    }
            }
            __syncthreads();
        }
    }
    // epilogue: alpha * acc + beta * C0 + bias[j], then GELU' / store / GELU
    float *C = g.C ? g.C + (long long)bz * g.sC : nullptr;
    const float *C0 = g.C0 ? g.C0 + (long long)bz * g.sC0 : nullptr;
    const float *Dg = g.dgelu_pre ? g.dgelu_pre + (long long)bz * g.sDg : nullptr;
    float *act = g.act ? g.act + (long long)bz * g.sAct : nullptr;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int i = i0 + wm + mi * 16 + grp + (h >= 2 ? 8 : 0);
                const int j = j0 + wn + ni * 8 + tig * 2 + (h & 1);
                if (i < g.M && j < g.N) {
                    float v = g.alpha * acc[mi][ni][h];
                    const long long off = (long long)i * g.ldc + j;
                    if (ks_n > 1) {
                        atomicAdd(&C[off], v);
                        continue;
                    }
                    if (C0)
                        v += g.beta * C0[off];
                    if (g.bias)
                        v += g.bias[j];
                    if (Dg)
                        v *= gelu_grad(Dg[off]);
                    if (C)
                        C[off] = v;
                    if (act)
                        act[off] = gelu(v);
                }
            }
}

// Input features per point: (u0, x, r, wall profile beta_l + (beta_r - beta_l) x).
__global__ void features_kernel(const float *__restrict__ u0, const float *__restrict__ r,
                                const float *__restrict__ bl, const float *__restrict__ br, float *__restrict__ f,
                                int batch, int n)
{
    const long long total = (long long)batch * n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / n), j = (int)(i % n);
        const float x = (float)(j + 1) / (float)(n + 1);
        f[i * 4 + 0] = u0[i];
        f[i * 4 + 1] = x;
        f[i * 4 + 2] = r[b];
        f[i * 4 + 3] = bl[b] + (br[b] - bl[b]) * x;
    }
}

// Spectral weights: for mode m, the real 2C x 2C matrix acting on the row
// vector (re, im): [[Rr^T, Ri^T], [-Ri^T, Rr^T]] with R = Rr + i Ri (C x C,
// out x in).  Layout of rr/ri: [m][out][in]; of w: [m][2C][2C].
__global__ void spec_assemble_kernel(const float *__restrict__ rr, const float *__restrict__ ri,
                                     float *__restrict__ w, int modes, int c)
{
    const long long total = (long long)modes * 2 * c * 2 * c;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(e / (4LL * c * c));
        const int rem = (int)(e % (4LL * c * c));
        const int row = rem / (2 * c), col = rem % (2 * c);
        const int in = row % c, out = col % c;
        const bool row_im = row >= c, col_im = col >= c;
        const long long ro = ((long long)m * c + out) * c + in;
        float v;
        if (!row_im && !col_im)
            v = rr[ro];
        else if (!row_im && col_im)
            v = ri[ro];
        else if (row_im && !col_im)
            v = -ri[ro];
        else
            v = rr[ro];
        w[e] = v;
    }
}

// Gradient of the spectral weights from the gradient of the assembled matrix.
__global__ void spec_reduce_kernel(const float *__restrict__ dw, float *__restrict__ drr, float *__restrict__ dri,
                                   int modes, int c)
{
    const long long total = (long long)modes * c * c;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(e / ((long long)c * c));
        const int rem = (int)(e % ((long long)c * c));
        const int out = rem / c, in = rem % c;
        const float *d = dw + (long long)m * 4 * c * c;
        const int C2 = 2 * c;
        drr[e] = d[in * C2 + out] + d[(c + in) * C2 + (c + out)];
        dri[e] = d[in * C2 + (c + out)] - d[(c + in) * C2 + out];
    }
}

// Column sums (bias gradients): out[j] = sum_i x[i, j], x is rows x cols.
__global__ void colsum_kernel(const float *__restrict__ x, float *__restrict__ out, long long rows, int cols)
{
    const int j = blockIdx.x;
    float s = 0.0f;
    for (long long i = threadIdx.x; i < rows; i += blockDim.x)
        s += x[i * cols + j];
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        out[j] = red[0];
}

// Relative L2 loss per sample and its gradient: loss_b = ||p - y|| / ||y||,
// mean over the batch; dp = (p - y) / (||p - y|| ||y|| batch).
__global__ void rel_l2_kernel(const float *__restrict__ pred, const float *__restrict__ target,
                              float *__restrict__ dpred, float *__restrict__ loss_per_sample, int n, int batch)
{
    const int b = blockIdx.x;
    const float *p = pred + (long long)b * n;
    const float *y = target + (long long)b * n;
    float se = 0.0f, sy = 0.0f;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const float d = p[j] - y[j];
        se += d * d;
        sy += y[j] * y[j];
    }
    __shared__ float r1[256], r2[256];
    r1[threadIdx.x] = se;
    r2[threadIdx.x] = sy;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            r1[threadIdx.x] += r1[threadIdx.x + w];
            r2[threadIdx.x] += r2[threadIdx.x + w];
        }
        __syncthreads();
    }
    const float ne = sqrtf(r1[0]), ny = fmaxf(sqrtf(r2[0]), 1e-30f);
    if (threadIdx.x == 0)
        loss_per_sample[b] = ne / ny;
    if (dpred) {
        const float sc = 1.0f / (fmaxf(ne, 1e-30f) * ny * (float)batch);
        for (int j = threadIdx.x; j < n; j += blockDim.x)
            dpred[(long long)b * n + j] = (p[j] - y[j]) * sc;
    }
}

// Adam (bias-corrected), FP32 master parameters.
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Round to the nearest BF16 value (kept in FP32 storage): the network's
// weights as the BF16 model sees them.
__global__ void round_bf16_kernel(const float *__restrict__ x, float *__restrict__ y, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __bfloat162float(__float2bfloat16_rn(x[i]));
}

int grid_for(long long n)
{
    long long b = (n + 255) / 256;
    return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

}  // namespace

namespace {

// float4 staging is allowed when the unit-stride dimension's extent, the
// other stride, the batch stride and the base are all multiples of 4 floats.
int vec_ok(const float *X, long long s_r, long long s_k, int rmax, int kdim, long long sbatch, int batch)
{
    if (!X || (reinterpret_cast<uintptr_t>(X) & 15) != 0 || (batch > 1 && sbatch % 4 != 0))
        return 0;
    if (s_k == 1)
        return (kdim % 4 == 0 && s_r % 4 == 0) ? 1 : 0;
    if (s_r == 1)
        return (rmax % 4 == 0 && s_k % 4 == 0) ? 1 : 0;
    return 0;
}

}  // namespace

cudaError_t sno_gemm(const GemmArgs &g0, int batch, bool split, cudaStream_t s)
{
    if (g0.M <= 0 || g0.N <= 0 || batch <= 0)
        return cudaSuccess;
    GemmArgs g = g0;
    const int ks = g.ksplit > 1 ? g.ksplit : 1;
    if (ks > 1 && (g.A2 || g.C0 || g.bias || g.dgelu_pre || g.act || !g.C))
        return cudaErrorInvalidValue;
    g.vec[0] = vec_ok(g.A, g.lda_i, g.lda_k, g.M, g.K, g.sA, batch);
    g.vec[1] = vec_ok(g.B, g.ldb_j, g.ldb_k, g.N, g.K, g.sB, batch);
    g.vec[2] = g.A2 ? vec_ok(g.A2, g.lda2_i, g.lda2_k, g.M, g.K2, g.sA2, batch) : 0;
    g.vec[3] = g.A2 ? vec_ok(g.B2, g.ldb2_j, g.ldb2_k, g.N, g.K2, g.sB2, batch) : 0;
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, batch * ks);
    if (split)
        gemm_kernel<true><<<grid, NT, 0, s>>>(g);
    else
        gemm_kernel<false><<<grid, NT, 0, s>>>(g);
    return cudaGetLastError();
}

cudaError_t sno_features(const float *u0, const float *r, const float *bl, const float *br, float *f, int batch, int n,
                         cudaStream_t s)
{
    features_kernel<<<grid_for((long long)batch * n), 256, 0, s>>>(u0, r, bl, br, f, batch, n);
    return cudaGetLastError();
}

cudaError_t sno_spec_assemble(const float *rr, const float *ri, float *w, int modes, int c, cudaStream_t s)
{
    spec_assemble_kernel<<<grid_for(4LL * modes * c * c), 256, 0, s>>>(rr, ri, w, modes, c);
    return cudaGetLastError();
}

cudaError_t sno_spec_reduce(const float *dw, float *drr, float *dri, int modes, int c, cudaStream_t s)
{
    spec_reduce_kernel<<<grid_for((long long)modes * c * c), 256, 0, s>>>(dw, drr, dri, modes, c);
    return cudaGetLastError();
}

cudaError_t sno_colsum(const float *x, float *out, long long rows, int cols, cudaStream_t s)
{
    colsum_kernel<<<cols, 256, 0, s>>>(x, out, rows, cols);
    return cudaGetLastError();
}

cudaError_t sno_rel_l2(const float *pred, const float *target, float *dpred, float *loss, int n, int batch, cudaStream_t s)
{
    rel_l2_kernel<<<batch, 256, 0, s>>>(pred, target, dpred, loss, n, batch);
    return cudaGetLastError();
}

cudaError_t sno_adam(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2, float eps,
                     float c1, float c2, cudaStream_t s)
{
    adam_kernel<<<grid_for(n), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t sno_round_bf16(const float *x, float *y, long long n, cudaStream_t s)
{
    round_bf16_kernel<<<grid_for(n), 256, 0, s>>>(x, y, n);
    return cudaGetLastError();
}

}  // namespace ge
