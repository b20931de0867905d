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

#include "ge_f32x2.cuh"
#include "ge_sno_internal.h"

namespace ge {
namespace {

constexpr int BM = 64, BN = 64, BK = 32, PADK = BK + 8;  // bf16 elements per smem row
constexpr int NT = 128;                                  // threads per GEMM CTA

// tanh: the library function (EXACT, split mode) or the hardware
// approximation (tanh.approx.f32, relative error about 2^-11, below the
// 2^-8 of the BF16 operands it feeds in the plain mode).
template <bool EXACT>
__device__ __forceinline__ float tanh_sel(float x)
{
    if (EXACT)
        return tanhf(x);
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// tanh form of GELU and its derivative
template <bool EXACT>
__device__ __forceinline__ float gelu(float x)
{
    const float k0 = 0.7978845608028654f, k1 = 0.044715f;
    return 0.5f * x * (1.0f + tanh_sel<EXACT>(k0 * (x + k1 * x * x * x)));
}

template <bool EXACT>
__device__ __forceinline__ float gelu_grad(float x)
{
    const float k0 = 0.7978845608028654f, k1 = 0.044715f;
    const float u = k0 * (x + k1 * x * x * x);
    const float th = tanh_sel<EXACT>(u);
    const float du = k0 * (1.0f + 3.0f * k1 * x * x);
    return 0.5f * (1.0f + th) + 0.5f * x * (1.0f - th * th) * du;
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Shared-memory tile of one operand: 64 rows x BK k-values in BF16, stored
// k-contiguous ([row][PADK]) when the operand is k-contiguous in global
// memory and row-contiguous ([k][PADT]) otherwise.  Both are written with
// packed 8-byte stores and read with ldmatrix (.trans for the second); the
// row pitches (80 and 144 bytes) keep ldmatrix free of bank conflicts.
constexpr int PADT = BM + 8;
constexpr int TILE = BM * PADK;
static_assert(BK * PADT <= TILE, "both tile layouts fit one buffer");

__device__ __forceinline__ int at_k(int r, int k) { return r * PADK + k; }
__device__ __forceinline__ int at_r(int r, int k) { return k * PADT + r; }

template <bool SPLIT>
__device__ __forceinline__ void put1(__nv_bfloat16 (*S)[TILE], int idx, float x)
{
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    S[0][idx] = h;
    if (SPLIT)
        S[SPLIT ? 1 : 0][idx] = __float2bfloat16_rn(x - __bfloat162float(h));
}

// Four values that are adjacent in the tile's contiguous dimension (idx a
// multiple of 4): two packed BF16 pairs, one 8-byte store per part.
template <bool SPLIT>
__device__ __forceinline__ void put4(__nv_bfloat16 (*S)[TILE], int idx, float a, float b, float c, float d)
{
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(a, b), h1 = __floats2bfloat162_rn(c, d);
    uint2 w;
    w.x = *reinterpret_cast<const uint32_t *>(&h0);
    w.y = *reinterpret_cast<const uint32_t *>(&h1);
    *reinterpret_cast<uint2 *>(&S[0][idx]) = w;
    if (SPLIT) {
        const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
        const __nv_bfloat162 l0 = __floats2bfloat162_rn(a - f0.x, b - f0.y);
        const __nv_bfloat162 l1 = __floats2bfloat162_rn(c - f1.x, d - f1.y);
        w.x = *reinterpret_cast<const uint32_t *>(&l0);
        w.y = *reinterpret_cast<const uint32_t *>(&l1);
        *reinterpret_cast<uint2 *>(&S[SPLIT ? 1 : 0][idx]) = w;
    }
}

// Tiles of an operand whose element (row, k) is X[row * s_r + k * s_k]:
// rows r0.. (< rmax) and k0.. (< kend) are read, the rest is zero.  Each
// thread holds 16 values between the global load (`load`) and the
// shared-memory store (`store`), so the next tile's loads are in flight
// while the current one is multiplied.  The element order follows the
// unit-stride dimension so a warp's loads coalesce; VEC (checked by the
// launcher: that dimension's extent, the other stride and the base all
// multiples of 4 floats / 16 bytes) loads four elements at once.
constexpr int PER_T = BM * BK / NT;  // 16 values per thread and tile

template <bool VEC>
__device__ __forceinline__ void load(float (&x)[PER_T], const float *__restrict__ X, long long s_r, long long s_k,
                                     int r0, int rmax, int k0, int kend, int t)
{
    if (s_k == 1) {
        if (VEC) {
#pragma unroll
            for (int q = 0; q < PER_T / 4; ++q) {
                const int e = t + q * NT;
                const int row = r0 + e / (BK / 4), k = k0 + (e % (BK / 4)) * 4;
                float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (row < rmax && k < kend)
                    v = __ldg(reinterpret_cast<const float4 *>(X + (long long)row * s_r + k));
                x[4 * q] = v.x, x[4 * q + 1] = v.y, x[4 * q + 2] = v.z, x[4 * q + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < PER_T; ++q) {
                const int e = t + q * NT;
                const int row = r0 + e / BK, k = k0 + e % BK;
                x[q] = (row < rmax && k < kend) ? __ldg(X + (long long)row * s_r + k) : 0.0f;
            }
        }
    } else {
        if (VEC) {
#pragma unroll
            for (int q = 0; q < PER_T / 4; ++q) {
                const int e = t + q * NT;
                const int row = r0 + (e % (BM / 4)) * 4, k = k0 + e / (BM / 4);
                float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (row < rmax && k < kend)
                    v = __ldg(reinterpret_cast<const float4 *>(X + row + (long long)k * s_k));
                x[4 * q] = v.x, x[4 * q + 1] = v.y, x[4 * q + 2] = v.z, x[4 * q + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < PER_T; ++q) {
                const int e = t + q * NT;
                const int row = r0 + e % BM, k = k0 + e / BM;
                x[q] = (row < rmax && k < kend) ? __ldg(X + (long long)row * s_r + (long long)k * s_k) : 0.0f;
            }
        }
    }
}

template <bool SPLIT, bool VEC>
__device__ __forceinline__ void store(__nv_bfloat16 (*S)[TILE], const float (&x)[PER_T], bool kfast, int t)
{
    if (kfast) {
        if (VEC) {
#pragma unroll
            for (int q = 0; q < PER_T / 4; ++q) {
                const int e = t + q * NT;
                put4<SPLIT>(S, at_k(e / (BK / 4), (e % (BK / 4)) * 4), x[4 * q], x[4 * q + 1], x[4 * q + 2],
                            x[4 * q + 3]);
            }
        } else {
#pragma unroll
            for (int q = 0; q < PER_T; ++q) {
                const int e = t + q * NT;
                put1<SPLIT>(S, at_k(e / BK, e % BK), x[q]);
            }
        }
    } else {
        if (VEC) {
#pragma unroll
            for (int q = 0; q < PER_T / 4; ++q) {
                const int e = t + q * NT;
                put4<SPLIT>(S, at_r((e % (BM / 4)) * 4, e / (BM / 4)), x[4 * q], x[4 * q + 1], x[4 * q + 2],
                            x[4 * q + 3]);
            }
        } else {
#pragma unroll
            for (int q = 0; q < PER_T; ++q) {
                const int e = t + q * NT;
                put1<SPLIT>(S, at_r(e % BM, e / BM), x[q]);
            }
        }
    }
}

// Four 8x8 BF16 matrices from shared memory (one 16-byte row address per lane).
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p)
{
    const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

// The same, each 8x8 matrix transposed.
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void *p)
{
    const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

// Products of one staged BK slice: the warp's 32x32 block of the tile.  The
// fragments of m16n8k16 come from ldmatrix: A as 16x16 blocks (rows, k), B
// as pairs of n8 x k16 blocks; a row-contiguous tile is read transposed.
template <bool SPLIT>
__device__ __forceinline__ void mma_tile(const __nv_bfloat16 (*As)[TILE], const __nv_bfloat16 (*Bs)[TILE],
                                         float (&acc)[2][4][4], int wm, int wn, int lane, bool a_kfast, bool b_kfast)
{
    const int q = lane >> 3, l8 = lane & 7;
#pragma unroll
    for (int ks = 0; ks < BK; ks += 16) {
        uint32_t af[SPLIT ? 2 : 1][2][4], bf[SPLIT ? 2 : 1][4][2];
#pragma unroll
        for (int s = 0; s < (SPLIT ? 2 : 1); ++s) {
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                if (a_kfast)
                    ldsm_x4(af[s][mi], &As[s][at_k(wm + mi * 16 + (lane & 15), ks + (lane >> 4) * 8)]);
                else
                    ldsm_x4_t(af[s][mi], &As[s][at_r(wm + mi * 16 + (q & 1) * 8, ks + (q >> 1) * 8 + l8)]);
            }
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                uint32_t r4[4];
                if (b_kfast)
                    ldsm_x4(r4, &Bs[s][at_k(wn + p * 16 + l8 + ((lane >> 4) << 3), ks + (q & 1) * 8)]);
                else
                    ldsm_x4_t(r4, &Bs[s][at_r(wn + p * 16 + (q >> 1) * 8, ks + (q & 1) * 8 + l8)]);
                bf[s][2 * p][0] = r4[0];
                bf[s][2 * p][1] = r4[1];
                bf[s][2 * p + 1][0] = r4[2];
                bf[s][2 * p + 1][1] = r4[3];
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
}

// ---- BF16 operands: 16-byte cp.async chunks (8 elements along the
// unit-stride dimension, zero-filled outside the operand) or 2-byte loads
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One BK slice of a BF16 operand into the tile S (layout as in `store`).
// `chunk` (checked by the launcher: the unit-stride extent, the other
// stride and the batch stride multiples of 8, the base 16-byte aligned)
// copies whole 16-byte chunks asynchronously; otherwise 2-byte loads.
__device__ __forceinline__ void stage_bf16(__nv_bfloat16 *S, const __nv_bfloat16 *__restrict__ X, long long s_r,
                                           long long s_k, int r0, int rmax, int k0, int kend, bool chunk, int t)
{
    if (s_k == 1) {
        if (chunk) {
#pragma unroll
            for (int q = 0; q < BM * BK / 8 / NT; ++q) {
                const int e = t + q * NT;
                const int r = e / (BK / 8), kc = (e % (BK / 8)) * 8;
                const int row = r0 + r, k = k0 + kc;
                const bool ok = row < rmax && k < kend;
                cp_async16(&S[at_k(r, kc)], ok ? X + (long long)row * s_r + k : X, ok);
            }
        } else {
            for (int e = t; e < BM * BK; e += NT) {
                const int r = e / BK, kk = e % BK;
                const int row = r0 + r, k = k0 + kk;
                S[at_k(r, kk)] = (row < rmax && k < kend) ? X[(long long)row * s_r + k] : __float2bfloat16_rn(0.0f);
            }
        }
    } else {
        if (chunk) {
#pragma unroll
            for (int q = 0; q < BM * BK / 8 / NT; ++q) {
                const int e = t + q * NT;
                const int r = (e % (BM / 8)) * 8, kk = e / (BM / 8);
                const int row = r0 + r, k = k0 + kk;
                const bool ok = row < rmax && k < kend;
                cp_async16(&S[at_r(r, kk)], ok ? X + row + (long long)k * s_k : X, ok);
            }
        } else {
            for (int e = t; e < BM * BK; e += NT) {
                const int r = e % BM, kk = e / BM;
                const int row = r0 + r, k = k0 + kk;
                S[at_r(r, kk)] = (row < rmax && k < kend) ? X[(long long)row * s_r + (long long)k * s_k]
                                                          : __float2bfloat16_rn(0.0f);
            }
        }
    }
}

// Operands of one product (segment) of the GEMM for batch entry bz.
struct Seg {
    const void *A, *B;
    long long la_i, la_k, lb_k, lb_j;
    int kbeg, kend;
    int va, vb;
};

__device__ __forceinline__ Seg segment(const GemmArgs &g, int seg, int bz, int kslice, int ks_n, int esize)
{
    Seg s;
    if (seg == 0) {
        const int kchunk = ((g.K + ks_n - 1) / ks_n + BK - 1) / BK * BK;
        s.kbeg = kslice * kchunk;
        s.kend = (s.kbeg + kchunk < g.K) ? s.kbeg + kchunk : g.K;
        s.A = static_cast<const char *>(g.A) + (long long)bz * g.sA * esize;
        s.B = static_cast<const char *>(g.B) + (long long)bz * g.sB * esize;
        s.la_i = g.lda_i, s.la_k = g.lda_k, s.lb_k = g.ldb_k, s.lb_j = g.ldb_j;
        s.va = g.vec[0], s.vb = g.vec[1];
    } else {
        s.kbeg = 0;
        s.kend = (g.A2 && g.K2 > 0) ? g.K2 : 0;
        s.A = g.A2 ? static_cast<const char *>(g.A2) + (long long)bz * g.sA2 * esize : nullptr;
        s.B = g.B2 ? static_cast<const char *>(g.B2) + (long long)bz * g.sB2 * esize : nullptr;
        s.la_i = g.lda2_i, s.la_k = g.lda2_k, s.lb_k = g.ldb2_k, s.lb_j = g.ldb2_j;
        s.va = g.vec[2], s.vb = g.vec[3];
    }
    return s;
}

// Main loop, FP32 operands: staged as BF16 (and split residuals) through
// registers; VEC: float4 loads of the next slice overlap this slice's MMAs.
template <bool SPLIT, bool VEC>
__device__ __forceinline__ void mainloop_f32(const GemmArgs &g, int bz, int kslice, int ks_n, int i0, int j0,
                                             float (&acc)[2][4][4], __nv_bfloat16 (*As)[TILE],
                                             __nv_bfloat16 (*Bs)[TILE], int t, int wm, int wn, int lane)
{
    for (int seg = 0; seg < 2; ++seg) {
        const Seg sg = segment(g, seg, bz, kslice, ks_n, 4);
        if (sg.kbeg >= sg.kend)
            continue;
        const float *A = static_cast<const float *>(sg.A), *Bm = static_cast<const float *>(sg.B);
        float xa[PER_T], xb[PER_T];
        if (VEC) {
            load<VEC>(xa, A, sg.la_i, sg.la_k, i0, g.M, sg.kbeg, sg.kend, t);
            load<VEC>(xb, Bm, sg.lb_j, sg.lb_k, j0, g.N, sg.kbeg, sg.kend, t);
        }
        for (int k0 = sg.kbeg; k0 < sg.kend; k0 += BK) {
            if (!VEC) {  // scalar staging: no prefetch (registers)
                load<VEC>(xa, A, sg.la_i, sg.la_k, i0, g.M, k0, sg.kend, t);
                load<VEC>(xb, Bm, sg.lb_j, sg.lb_k, j0, g.N, k0, sg.kend, t);
            }
            store<SPLIT, VEC>(As, xa, sg.la_k == 1, t);
            store<SPLIT, VEC>(Bs, xb, sg.lb_k == 1, t);
            __syncthreads();
            if (VEC && k0 + BK < sg.kend) {
                load<VEC>(xa, A, sg.la_i, sg.la_k, i0, g.M, k0 + BK, sg.kend, t);
                load<VEC>(xb, Bm, sg.lb_j, sg.lb_k, j0, g.N, k0 + BK, sg.kend, t);
            }
            mma_tile<SPLIT>(As, Bs, acc, wm, wn, lane, sg.la_k == 1, sg.lb_k == 1);
            __syncthreads();
        }
    }
}

// Main loop, BF16 operands: the slices of both products run through two
// shared-memory stages; the copies of slice i+1 are in flight while slice i
// is multiplied.
__device__ __forceinline__ void mainloop_bf16(const GemmArgs &g, int bz, int kslice, int ks_n, int i0, int j0,
                                              float (&acc)[2][4][4], __nv_bfloat16 (*As)[TILE],
                                              __nv_bfloat16 (*Bs)[TILE], int t, int wm, int wn, int lane)
{
    const Seg s0 = segment(g, 0, bz, kslice, ks_n, 2), s1 = segment(g, 1, bz, kslice, ks_n, 2);
    const int n0 = s0.kend > s0.kbeg ? (s0.kend - s0.kbeg + BK - 1) / BK : 0;
    const int n1 = s1.kend > s1.kbeg ? (s1.kend - s1.kbeg + BK - 1) / BK : 0;
    const int nt = n0 + n1;
    auto issue = [&](int i) {
        const Seg &sg = i < n0 ? s0 : s1;
        const int k0 = sg.kbeg + (i < n0 ? i : i - n0) * BK;
        __nv_bfloat16 *as = As[i & 1], *bs = Bs[i & 1];
        stage_bf16(as, static_cast<const __nv_bfloat16 *>(sg.A), sg.la_i, sg.la_k, i0, g.M, k0, sg.kend, sg.va, t);
        stage_bf16(bs, static_cast<const __nv_bfloat16 *>(sg.B), sg.lb_j, sg.lb_k, j0, g.N, k0, sg.kend, sg.vb, t);
        cp_async_commit();
    };
    if (nt > 0)
        issue(0);
    for (int i = 0; i < nt; ++i) {
        if (i + 1 < nt) {
            issue(i + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const Seg &sg = i < n0 ? s0 : s1;
        mma_tile<false>(As + (i & 1), Bs + (i & 1), acc, wm, wn, lane, sg.la_k == 1, sg.lb_k == 1);
        __syncthreads();
    }
}

// Two adjacent outputs (columns j, j+1) in FP32 or BF16 storage.
__device__ __forceinline__ float2 ld2(const void *base, long long off, bool bf16)
{
    if (bf16)
        return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(static_cast<const __nv_bfloat16 *>(base) + off));
    return *reinterpret_cast<const float2 *>(static_cast<const float *>(base) + off);
}

__device__ __forceinline__ void st2(void *base, long long off, float a, float b, bool bf16)
{
    if (bf16)
        *reinterpret_cast<__nv_bfloat162 *>(static_cast<__nv_bfloat16 *>(base) + off) = __floats2bfloat162_rn(a, b);
    else
        *reinterpret_cast<float2 *>(static_cast<float *>(base) + off) = make_float2(a, b);
}

__device__ __forceinline__ float ld1(const void *base, long long off, bool bf16)
{
    return bf16 ? __bfloat162float(static_cast<const __nv_bfloat16 *>(base)[off]) : static_cast<const float *>(base)[off];
}

__device__ __forceinline__ void st1(void *base, long long off, float a, bool bf16)
{
    if (bf16)
        static_cast<__nv_bfloat16 *>(base)[off] = __float2bfloat16_rn(a);
    else
        static_cast<float *>(base)[off] = a;
}

// Epilogue: alpha * acc + beta * C0 + bias[j], then GELU' / store / GELU,
// one row and two adjacent columns at a time (paired accesses when the
// launcher found every epilogue array aligned with an even pitch).
template <bool SPLIT>
__device__ __forceinline__ void epilogue(const GemmArgs &g, int bz, int ks_n, int i0, int j0, const float (&acc)[2][4][4],
                                         int wm, int wn, int grp, int tig)
{
    const bool ob = g.out_bf16 != 0, db = g.dg_bf16 != 0;
    const int oes = ob ? 2 : 4, des = db ? 2 : 4;
    void *C = g.C ? static_cast<char *>(g.C) + (long long)bz * g.sC * oes : nullptr;
    const float *C0 = g.C0 ? g.C0 + (long long)bz * g.sC0 : nullptr;
    const void *Dg = g.dgelu_pre ? static_cast<const char *>(g.dgelu_pre) + (long long)bz * g.sDg * des : nullptr;
    void *act = g.act ? static_cast<char *>(g.act) + (long long)bz * g.sAct * oes : nullptr;
    if (g.dot_w) {
        // per row: sum over this CTA's columns of GELU(value) * dot_w[j]
#pragma unroll
        for (int mi = 0; mi < 2; ++mi)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int i = i0 + wm + mi * 16 + grp + hh * 8;
                float part = 0.0f;
#pragma unroll
                for (int ni = 0; ni < 4; ++ni)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const int j = j0 + wn + ni * 8 + tig * 2 + c;
                        if (i < g.M && j < g.N) {
                            float w = g.alpha * acc[mi][ni][2 * hh + c];
                            if (g.bias)
                                w += g.bias[j];
                            part += gelu<SPLIT>(w) * g.dot_w[j];
                        }
                    }
                // the four lanes of a row group (tig) hold the warp's 32 columns
                part += __shfl_xor_sync(0xffffffffu, part, 1);
                part += __shfl_xor_sync(0xffffffffu, part, 2);
                if (tig == 0 && i < g.M && j0 + wn < g.N)
                    g.dot_out[((long long)bz * g.M + i) * g.dot_slots + (j0 + wn) / 32] = part;
            }
        return;
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int i = i0 + wm + mi * 16 + grp + hh * 8;
                const int j = j0 + wn + ni * 8 + tig * 2;
                if (i >= g.M || j >= g.N)
                    continue;
                const long long off = (long long)i * g.ldc + j;
                float v[2] = {g.alpha * acc[mi][ni][2 * hh], g.alpha * acc[mi][ni][2 * hh + 1]};
                if (ks_n > 1) {
                    float *Cf = static_cast<float *>(C);
                    atomicAdd(&Cf[off], v[0]);
                    if (j + 1 < g.N)
                        atomicAdd(&Cf[off + 1], v[1]);
                    continue;
                }
                if (g.pairs && j + 1 < g.N) {
                    if (C0) {
                        const float2 c = *reinterpret_cast<const float2 *>(C0 + off);
                        v[0] += g.beta * c.x;
                        v[1] += g.beta * c.y;
                    }
                    if (g.bias) {
                        const float2 b = *reinterpret_cast<const float2 *>(g.bias + j);
                        v[0] += b.x;
                        v[1] += b.y;
                    }
                    if (Dg) {
                        const float2 d = ld2(Dg, off, db);
                        v[0] *= gelu_grad<SPLIT>(d.x);
                        v[1] *= gelu_grad<SPLIT>(d.y);
                    }
                    if (C)
                        st2(C, off, v[0], v[1], ob);
                    if (act)
                        st2(act, off, gelu<SPLIT>(v[0]), gelu<SPLIT>(v[1]), ob);
                    continue;
                }
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (j + c >= g.N)
                        break;
                    float w = v[c];
                    if (C0)
                        w += g.beta * C0[off + c];
                    if (g.bias)
                        w += g.bias[j + c];
                    if (Dg)
                        w *= gelu_grad<SPLIT>(ld1(Dg, off + c, db));
                    if (C)
                        st1(C, off + c, w, ob);
                    if (act)
                        st1(act, off + c, gelu<SPLIT>(w), ob);
                }
            }
}

// 64x64 output tile per CTA, 4 warps (2 x 2), each warp 32x32 = 2 x 4 mma
// tiles.  MODE 0: FP32 operands, scalar loads; 1: FP32 operands, float4
// loads (the launcher checks every operand allows it); 2: BF16 operands.
template <bool SPLIT, int MODE>
__global__ void __launch_bounds__(NT, MODE == 0 ? 1 : 4) gemm_kernel(GemmArgs g)
{
    constexpr int NS = (SPLIT || MODE == 2) ? 2 : 1;  // split parts, or pipeline stages
    __shared__ __align__(16) __nv_bfloat16 As[NS][TILE];
    __shared__ __align__(16) __nv_bfloat16 Bs[NS][TILE];
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
    if constexpr (MODE == 2)
        mainloop_bf16(g, bz, kslice, ks_n, i0, j0, acc, As, Bs, t, wm, wn, lane);
    else
        mainloop_f32<SPLIT, MODE == 1>(g, bz, kslice, ks_n, i0, j0, acc, As, Bs, t, wm, wn, lane);
    epilogue<SPLIT>(g, bz, ks_n, i0, j0, acc, wm, wn, grp, tig);
}

// Input features per point: (u0, x, r, wall profile beta_l + (beta_r - beta_l) x).
// FP32 rows of 4, or BF16 rows of 8 (the last 4 zero, so rows stay 16 bytes).
__global__ void features_kernel(const float *__restrict__ u0, const float *__restrict__ r,
                                const float *__restrict__ bl, const float *__restrict__ br, void *__restrict__ f,
                                int batch, int n, int bf16)
{
    const long long total = (long long)batch * n;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / n), j = (int)(i % n);
        const float x = (float)(j + 1) / (float)(n + 1);
        const float v[4] = {u0[i], x, r[b], bl[b] + (br[b] - bl[b]) * x};
        if (bf16) {
            __nv_bfloat16 *fb = static_cast<__nv_bfloat16 *>(f) + i * 8;
#pragma unroll
            for (int c = 0; c < 8; ++c)
                fb[c] = __float2bfloat16_rn(c < 4 ? v[c] : 0.0f);
        } else {
            float *ff = static_cast<float *>(f) + i * 4;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                ff[c] = v[c];
        }
    }
}

// Spectral weights: for mode m, the real 2C x 2C matrix acting on the row
// vector (re, im): [[Rr^T, Ri^T], [-Ri^T, Rr^T]] with R = Rr + i Ri (C x C,
// out x in).  Layout of rr/ri: [m][out][in]; of w: [m][2C][2C].
__global__ void spec_assemble_kernel(const float *__restrict__ rr, const float *__restrict__ ri,
                                     void *__restrict__ w, int modes, int c, int bf16, int k_major)
{
    // k_major: store each mode's matrix transposed, [2C out][2C in] (the
    // K-major B operand of the tensor-core mixing)
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
        const long long o = k_major ? (long long)m * 4 * c * c + (long long)col * 2 * c + row : e;
        if (bf16)
            static_cast<__nv_bfloat16 *>(w)[o] = __float2bfloat16_rn(v);
        else
            static_cast<float *>(w)[o] = v;
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

// Column sums (bias gradients): out[j] = sum_i x[i, j], x is rows x cols
// (FP32 or BF16).
__global__ void colsum_kernel(const void *__restrict__ x, float *__restrict__ out, long long rows, int cols, int bf16)
{
    const int j = blockIdx.x;
    float s = 0.0f;
    for (long long i = threadIdx.x; i < rows; i += blockDim.x)
        s += bf16 ? __bfloat162float(static_cast<const __nv_bfloat16 *>(x)[i * cols + j])
                  : static_cast<const float *>(x)[i * cols + j];
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
                              void *__restrict__ dpred, float *__restrict__ loss_per_sample, int n, int batch, int bf16)
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
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const float d = (p[j] - y[j]) * sc;
            if (bf16)
                static_cast<__nv_bfloat16 *>(dpred)[(long long)b * n + j] = __float2bfloat16_rn(d);
            else
                static_cast<float *>(dpred)[(long long)b * n + j] = d;
        }
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

// Round to the nearest BF16 value: the network's weights as the BF16 model
// sees them, kept in FP32 storage (y) and, when y16 is set, as BF16.
__global__ void round_bf16_kernel(const float *__restrict__ x, float *__restrict__ y, __nv_bfloat16 *__restrict__ y16,
                                  long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x[i]);
        y[i] = __bfloat162float(h);
        if (y16)
            y16[i] = h;
    }
}

// Lift without a GEMM (K = 4): one thread per point and 8 channels.
constexpr int kLiftMaxC = 256;

template <typename T, typename I>
__global__ void lift_kernel(const float *__restrict__ u0, const float *__restrict__ r, const float *__restrict__ bl,
                            const float *__restrict__ br, const T *__restrict__ w0, const float *__restrict__ b0,
                            T *__restrict__ v0, int batch, int n, int c, int bf16)
{
    // I: index type of the point and work counters (32-bit when they fit:
    // 64-bit divisions cost more than the rest of the work); the activation
    // index i * c is formed in 64 bits
    // the lift's weights and bias, once per CTA (c <= kLiftMaxC; else from global)
    __shared__ float sw[4 * kLiftMaxC], sb[kLiftMaxC];
    const bool staged = c <= kLiftMaxC;
    if (staged) {
        for (int k = threadIdx.x; k < 4 * c; k += blockDim.x)
            sw[k] = (float)w0[k];
        for (int k = threadIdx.x; k < c; k += blockDim.x)
            sb[k] = b0[k];
        __syncthreads();
    }
    const int cg = (c + 7) / 8;
    const I total = (I)batch * n * cg;
    for (I e = (I)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (I)gridDim.x * blockDim.x) {
        const I i = e / cg;
        const int c0 = (int)(e - i * cg) * 8;
        const int b = (int)(i / n), j = (int)(i - (I)b * n);
        const float x = (float)(j + 1) / (float)(n + 1);
        float f[4] = {u0[i], x, r[b], bl[b] + (br[b] - bl[b]) * x};
        if (bf16) {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                f[k] = __bfloat162float(__float2bfloat16_rn(f[k]));
        }
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int ch = c0 + q < c ? c0 + q : c - 1;
            float a = staged ? sb[ch] : b0[ch];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                a = fmaf(f[k], staged ? sw[k * c + ch] : (float)w0[k * c + ch], a);
            v[q] = a;
        }
        if (bf16 && c % 8 == 0) {
            // eight BF16 channels in one 16-byte store
            __nv_bfloat162 h[4];
#pragma unroll
            for (int q = 0; q < 4; ++q)
                h[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
            *reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(v0) + (long long)i * c + c0) =
                *reinterpret_cast<const uint4 *>(h);
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (c0 + q < c)
                    v0[(long long)i * c + c0 + q] = (T)v[q];
        }
    }
}

// The same lift with a warp per 32 consecutive points, when the number of
// channel groups cg divides 32: lane l forms the features of point l once
// (one division by n, the BF16 roundings), then cg rounds each hand 32 / cg
// points' features to the lanes by shuffles, lane l computing channel group
// l % cg of point l / cg of the round.  Each lane's channel group is fixed,
// so its 8 channels' weights live in registers, as channel pairs for packed
// FMAs.  The per-point scalar work is done once per point instead of once
// per channel group.  Same fused products in the same order as lift_kernel,
// so the two give the same bits.
template <typename T, typename I>
__global__ void __launch_bounds__(256) lift_fixed_kernel(const float *__restrict__ u0, const float *__restrict__ r,
                                                         const float *__restrict__ bl, const float *__restrict__ br,
                                                         const T *__restrict__ w0, const float *__restrict__ b0,
                                                         T *__restrict__ v0, int batch, int n, int c, int bf16)
{
    const int cg = (c + 7) / 8;  // lanes per point
    const int per_round = 32 / cg;
    const int lane = threadIdx.x & 31;
    const int c0 = (lane % cg) * 8;
    // the weights and biases of channel pairs (q, q + 1), for packed FMAs
    uint64_t w2[4][4], bias2[4];
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
        const int ch0 = c0 + q < c ? c0 + q : c - 1, ch1 = c0 + q + 1 < c ? c0 + q + 1 : c - 1;
        bias2[q / 2] = f2(b0[ch0], b0[ch1]);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            w2[k][q / 2] = f2((float)w0[k * c + ch0], (float)w0[k * c + ch1]);
    }
    const I points = (I)batch * n;
    const I warp0 = ((I)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const I warps = (I)gridDim.x * (blockDim.x / 32);
    // the loads of point p0 + lane of the next pass are issued before this
    // pass's stores, so their latency hides behind them
    float nu = 0.0f, nr = 0.0f, nl = 0.0f, nrt = 0.0f;
    int nj = 0;
    auto fetch = [&](I p) {
        const I ip = p + lane;
        if (ip < points) {
            const int b = (int)(ip / n);
            nj = (int)(ip - (I)b * n);
            nu = u0[ip];
            nr = r[b];
            nl = bl[b];
            nrt = br[b];
        }
    };
    fetch(warp0 * 32);
    for (I p0 = warp0 * 32; p0 < points; p0 += warps * 32) {
        // the features of point p0 + lane
        float g[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        if (p0 + lane < points) {
            const float x = (float)(nj + 1) / (float)(n + 1);
            g[0] = nu;
            g[1] = x;
            g[2] = nr;
            g[3] = nl + (nrt - nl) * x;
            if (bf16) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    g[k] = __bfloat162float(__float2bfloat16_rn(g[k]));
            }
        }
        fetch(p0 + warps * 32);
        for (int rd = 0; rd < cg; ++rd) {
            const int src = rd * per_round + lane / cg;
            uint64_t f[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float fk = __shfl_sync(0xffffffffu, g[k], src);
                f[k] = f2(fk, fk);
            }
            const I i = p0 + src;
            if (i >= points)
                continue;
            float v[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint64_t a = bias2[q];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    a = f2_fma(f[k], w2[k][q], a);
                const float2 aq = f2_split(a);
                v[2 * q] = aq.x;
                v[2 * q + 1] = aq.y;
            }
            if (bf16 && c % 8 == 0) {
                __nv_bfloat162 h[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    h[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                *reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(v0) + (long long)i * c + c0) =
                    *reinterpret_cast<const uint4 *>(h);
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (c0 + q < c)
                        v0[(long long)i * c + c0 + q] = (T)v[q];
            }
        }
    }
}

__global__ void dot_finish_kernel(const float *__restrict__ u0, const float *__restrict__ q2,
                                  const float *__restrict__ part, int slots, float *__restrict__ out, long long n)
{
    const float b = q2[0];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        float acc = 0.0f;
        for (int k = 0; k < slots; ++k)
            acc += part[i * slots + k];
        out[i] = u0[i] + (b + acc);
    }
}

// --- fallback arbiter helpers: rows of n FP32 values -----------------------

// Block-wide sum of a double (blockDim.x = 256); valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
            t += red[w];
    __syncthreads();
    return t;
}

// flags[i] = 1 when row i holds a NaN or an infinity (one block per row).
__global__ void rows_nonfinite_kernel(const float *__restrict__ u, long long rows, int n, int *__restrict__ flags)
{
    for (long long i = blockIdx.x; i < rows; i += gridDim.x) {
        const float *row = u + i * (long long)n;
        int bad = 0;
        for (int j = threadIdx.x; j < n; j += blockDim.x)
            bad |= !isfinite(row[j]);
        const int any = __syncthreads_or(bad);
        if (threadIdx.x == 0)
            flags[i] = any;
    }
}

// dst row i <- src row idx[i] (gather) or dst row idx[i] <- src row i
// (scatter); an index outside [0, rows) is skipped.
__global__ void rows_move_kernel(const float *__restrict__ src, float *__restrict__ dst, const long long *__restrict__ idx,
                                 long long count, int n, long long rows, int scatter)
{
    const long long total = count * (long long)n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / n;
        const int j = (int)(e % n);
        const long long k = idx[i];
        if (k < 0 || k >= rows)
            continue;
        if (scatter)
            dst[k * n + j] = src[e];
        else
            dst[e] = src[k * n + j];
    }
}

// err[i] = ||a[idx[i]] - ref[i]|| / ||ref[i]|| (sums in FP64; +inf when the
// result is not finite or ref is zero with a difference; NaN for an index
// outside [0, a_rows)).  One block per row.
__global__ void rows_rel_err_kernel(const float *__restrict__ a, long long a_rows, const long long *__restrict__ idx,
                                    const float *__restrict__ ref, long long count, int n, float *__restrict__ err)
{
    __shared__ double red[32];
    for (long long i = blockIdx.x; i < count; i += gridDim.x) {
        const long long k = idx[i];
        if (k < 0 || k >= a_rows) {
            if (threadIdx.x == 0)
                err[i] = __int_as_float(0x7fc00000);
            continue;  // uniform across the block
        }
        const float *ar = a + k * (long long)n;
        const float *rr = ref + i * (long long)n;
        double d2 = 0.0, r2 = 0.0;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const double d = (double)ar[j] - (double)rr[j];
            d2 += d * d;
            r2 += (double)rr[j] * (double)rr[j];
        }
        d2 = block_sum(d2, red);
        r2 = block_sum(r2, red);
        if (threadIdx.x == 0) {
            double e;
            if (!isfinite(d2) || !isfinite(r2))
                e = INFINITY;
            else if (r2 == 0.0)
                e = d2 == 0.0 ? 0.0 : INFINITY;
            else
                e = sqrt(d2 / r2);
            err[i] = (float)e;
        }
    }
}

int grid_for(long long n)
{
    long long b = (n + 255) / 256;
    return (int)(b > 4096 ? 4096 : (b < 1 ? 1 : b));
}

}  // namespace

namespace {

// Vector staging (16 bytes: 4 floats or 8 BF16 values along the unit-stride
// dimension) is allowed when that dimension's extent, the other stride, the
// batch stride and the base are all whole multiples of 16 bytes.
int vec_ok(const void *X, long long s_r, long long s_k, int rmax, int kdim, long long sbatch, int batch, int q)
{
    if (!X || (reinterpret_cast<uintptr_t>(X) & 15) != 0 || (batch > 1 && sbatch % q != 0))
        return 0;
    if (s_k == 1)
        return (kdim % q == 0 && s_r % q == 0) ? 1 : 0;
    if (s_r == 1)
        return (rmax % q == 0 && s_k % q == 0) ? 1 : 0;
    return 0;
}

}  // namespace

cudaError_t sno_gemm(const GemmArgs &g0, int batch, bool split, cudaStream_t s)
{
    if (g0.M <= 0 || g0.N <= 0 || batch <= 0)
        return cudaSuccess;
    GemmArgs g = g0;
    const int ks = g.ksplit > 1 ? g.ksplit : 1;
    if (ks > 1 && (g.A2 || g.C0 || g.bias || g.dgelu_pre || g.act || !g.C || g.out_bf16 || g.dot_w))
        return cudaErrorInvalidValue;
    if (g.dot_w && (g.C || g.act || g.C0 || g.dgelu_pre || !g.dot_out || g.dot_slots < (g.N + 31) / 32))
        return cudaErrorInvalidValue;
    if (g.in_bf16 && split)
        return cudaErrorInvalidValue;
    const int q = g.in_bf16 ? 8 : 4;
    g.vec[0] = vec_ok(g.A, g.lda_i, g.lda_k, g.M, g.K, g.sA, batch, q);
    g.vec[1] = vec_ok(g.B, g.ldb_j, g.ldb_k, g.N, g.K, g.sB, batch, q);
    g.vec[2] = g.A2 ? vec_ok(g.A2, g.lda2_i, g.lda2_k, g.M, g.K2, g.sA2, batch, q) : 0;
    g.vec[3] = g.A2 ? vec_ok(g.B2, g.ldb2_j, g.ldb2_k, g.N, g.K2, g.sB2, batch, q) : 0;
    const bool vec = g.vec[0] && g.vec[1] && (!g.A2 || (g.vec[2] && g.vec[3]));
    auto al8 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7) == 0; };
    g.pairs = (g.ldc % 2 == 0) && al8(g.C) && al8(g.C0) && al8(g.dgelu_pre) && al8(g.act) && al8(g.bias) &&
              (batch == 1 || (g.sC % 2 == 0 && g.sC0 % 2 == 0 && g.sDg % 2 == 0 && g.sAct % 2 == 0));
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, batch * ks);
    if (g.in_bf16)
        gemm_kernel<false, 2><<<grid, NT, 0, s>>>(g);
    else if (split)
        vec ? gemm_kernel<true, 1><<<grid, NT, 0, s>>>(g) : gemm_kernel<true, 0><<<grid, NT, 0, s>>>(g);
    else
        vec ? gemm_kernel<false, 1><<<grid, NT, 0, s>>>(g) : gemm_kernel<false, 0><<<grid, NT, 0, s>>>(g);
    return cudaGetLastError();
}

cudaError_t sno_features(const float *u0, const float *r, const float *bl, const float *br, void *f, int batch, int n,
                         int bf16, cudaStream_t s)
{
    features_kernel<<<grid_for((long long)batch * n), 256, 0, s>>>(u0, r, bl, br, f, batch, n, bf16);
    return cudaGetLastError();
}

cudaError_t sno_spec_assemble(const float *rr, const float *ri, void *w, int modes, int c, int bf16, cudaStream_t s,
                              bool k_major)
{
    spec_assemble_kernel<<<grid_for(4LL * modes * c * c), 256, 0, s>>>(rr, ri, w, modes, c, bf16, k_major ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t sno_spec_reduce(const float *dw, float *drr, float *dri, int modes, int c, cudaStream_t s)
{
    spec_reduce_kernel<<<grid_for((long long)modes * c * c), 256, 0, s>>>(dw, drr, dri, modes, c);
    return cudaGetLastError();
}

cudaError_t sno_colsum(const void *x, float *out, long long rows, int cols, int bf16, cudaStream_t s)
{
    colsum_kernel<<<cols, 256, 0, s>>>(x, out, rows, cols, bf16);
    return cudaGetLastError();
}

cudaError_t sno_rel_l2(const float *pred, const float *target, void *dpred, float *loss, int n, int batch, int bf16,
                       cudaStream_t s)
{
    rel_l2_kernel<<<batch, 256, 0, s>>>(pred, target, dpred, loss, n, batch, bf16);
    return cudaGetLastError();
}

cudaError_t sno_adam(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2, float eps,
                     float c1, float c2, cudaStream_t s)
{
    adam_kernel<<<grid_for(n), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t sno_lift(const float *u0, const float *r, const float *bl, const float *br, const void *w0,
                     const float *b0, void *v0, int batch, int n, int c, int bf16, cudaStream_t s)
{
    const long long total = (long long)batch * n * ((c + 7) / 8);
    if (32 % ((c + 7) / 8) == 0) {
        // 32-bit indices when the loop's point counter (up to the points plus
        // one grid stride of 32 points a warp) cannot overflow them
        const bool small = (long long)batch * n < (1LL << 31) - 2LL * 32 * 8 * 4096;
        // one wave of resident blocks, each warp looping over many points
        // (the weights are loaded once per thread)
        static int resident = 0;
        if (resident == 0) {
            int dev = 0, sms = 0, per_sm = 0;
            cudaError_t e = cudaGetDevice(&dev);
            if (e == cudaSuccess)
                e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lift_fixed_kernel<__nv_bfloat16, int>, 256,
                                                                  0);
            if (e != cudaSuccess)
                return e;
            resident = sms * (per_sm < 1 ? 1 : per_sm);
        }
        long long blocks = ((long long)batch * n + 255) / 256;
        if (blocks > resident)
            blocks = resident;
        if (blocks > 4096)
            blocks = 4096;
        const int grid = (int)(blocks < 1 ? 1 : blocks);
        if (bf16 && small)
            lift_fixed_kernel<__nv_bfloat16, int><<<grid, 256, 0, s>>>(
                u0, r, bl, br, static_cast<const __nv_bfloat16 *>(w0), b0, static_cast<__nv_bfloat16 *>(v0), batch, n,
                c, 1);
        else if (bf16)
            lift_fixed_kernel<__nv_bfloat16, long long><<<grid, 256, 0, s>>>(
                u0, r, bl, br, static_cast<const __nv_bfloat16 *>(w0), b0, static_cast<__nv_bfloat16 *>(v0), batch, n,
                c, 1);
        else if (small)
            lift_fixed_kernel<float, int><<<grid, 256, 0, s>>>(u0, r, bl, br, static_cast<const float *>(w0),
                                                                          b0, static_cast<float *>(v0), batch, n, c, 0);
        else
            lift_fixed_kernel<float, long long><<<grid, 256, 0, s>>>(
                u0, r, bl, br, static_cast<const float *>(w0), b0, static_cast<float *>(v0), batch, n, c, 0);
    } else {
        // 32-bit indices when the grid-stride loop cannot overflow them
        const bool small = total < (1LL << 31) - 2LL * 256 * 4096;
        if (bf16 && small)
            lift_kernel<__nv_bfloat16, int><<<grid_for(total), 256, 0, s>>>(
                u0, r, bl, br, static_cast<const __nv_bfloat16 *>(w0), b0, static_cast<__nv_bfloat16 *>(v0), batch, n,
                c, 1);
        else if (bf16)
            lift_kernel<__nv_bfloat16, long long><<<grid_for(total), 256, 0, s>>>(
                u0, r, bl, br, static_cast<const __nv_bfloat16 *>(w0), b0, static_cast<__nv_bfloat16 *>(v0), batch, n,
                c, 1);
        else if (small)
            lift_kernel<float, int><<<grid_for(total), 256, 0, s>>>(u0, r, bl, br, static_cast<const float *>(w0), b0,
                                                                    static_cast<float *>(v0), batch, n, c, 0);
        else
            lift_kernel<float, long long><<<grid_for(total), 256, 0, s>>>(
                u0, r, bl, br, static_cast<const float *>(w0), b0, static_cast<float *>(v0), batch, n, c, 0);
    }
    return cudaGetLastError();
}

cudaError_t sno_dot_finish(const float *u0, const float *q2, const float *part, int slots, float *out, long long n,
                           cudaStream_t s)
{
    dot_finish_kernel<<<grid_for(n), 256, 0, s>>>(u0, q2, part, slots, out, n);
    return cudaGetLastError();
}

cudaError_t sno_round_bf16(const float *x, float *y, void *y16, long long n, cudaStream_t s)
{
    round_bf16_kernel<<<grid_for(n), 256, 0, s>>>(x, y, static_cast<__nv_bfloat16 *>(y16), n);
    return cudaGetLastError();
}

cudaError_t sno_rows_nonfinite(const float *u, long long rows, int n, int *flags, cudaStream_t s)
{
    if (rows <= 0)
        return cudaSuccess;
    const int grid = (int)(rows < 8192 ? rows : 8192);
    rows_nonfinite_kernel<<<grid, 256, 0, s>>>(u, rows, n, flags);
    return cudaGetLastError();
}

cudaError_t sno_rows_move(const float *src, float *dst, const long long *idx, long long count, int n, long long rows,
                          bool scatter, cudaStream_t s)
{
    if (count <= 0)
        return cudaSuccess;
    rows_move_kernel<<<grid_for(count * (long long)n), 256, 0, s>>>(src, dst, idx, count, n, rows, scatter ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t sno_rows_rel_err(const float *a, long long a_rows, const long long *idx, const float *ref, long long count,
                             int n, float *err, cudaStream_t s)
{
    if (count <= 0)
        return cudaSuccess;
    const int grid = (int)(count < 8192 ? count : 8192);
    rows_rel_err_kernel<<<grid, 256, 0, s>>>(a, a_rows, idx, ref, count, n, err);
    return cudaGetLastError();
}

}  // namespace ge
