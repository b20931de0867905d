// ge_df.cuh -- double-float arithmetic on the FP32 pipes for the FP64
// contexts' double-float kernels (ge_tb_df.cu, ge_tbb_df.cu): every value an
// unevaluated sum hi + lo of two floats (Dekker's double-length arithmetic,
// 1971), operations built from error-free transformations.
#pragma once

#include <cuda_runtime.h>

#include "ge_internal.h"
#include "ge_tb_dev.cuh"

namespace ge {
namespace {

// --- error-free transformations (round-to-nearest intrinsics: never
// contracted into FMAs or reassociated by the compiler) ---

// s + e == a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e == a + b exactly when the exponent of a is not below that of b
// (Dekker's Fast2Sum); renormalises a pair.
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// Low-order part of a * p beyond q = fl(a_hi p_hi), qe = a_hi p_hi - q
// (exact).  With a_lo != 0 (GL), the two terms that depend on p_hi alone,
// a_lo p_hi and qe, are summed exactly (TwoProd, TwoSum): both follow p_hi
// through the fixed constant a, so rounding their sum errs in the same
// direction step after step (for a = 2r = 0.6 the error of a long smooth run
// grew linearly, about 0.02 units of 2^-48 per step, to 1e-12 in 10^4 steps).
// Roundings that involve p_lo are unbiased and stay.  a_lo p_lo is below the
// format's resolution.
template <bool GL>
__device__ __forceinline__ float df_prod_lo(float ah, float al, float ph, float pl, float qe)
{
    if constexpr (GL) {
        const float r1 = __fmul_rn(al, ph);
        const float r1e = __fmaf_rn(al, ph, -r1);
        float s, se;
        two_sum(r1, qe, s, se);
        return __fadd_rn(s, __fmaf_rn(ah, pl, __fadd_rn(se, r1e)));
    } else {
        return __fmaf_rn(ah, pl, qe);
    }
}

// (oh, ol) = x + g * p, every operand a (hi, lo) pair; GL: g_lo != 0.
// g_hi p_hi = q + qe exactly (one FMA gives the product's rounding error);
// x_hi + q = s + e exactly (TwoSum); the low-order terms join e in FP32.
// NORM: renormalise (s, rest) by Fast2Sum.  Without it the pair stays an
// unevaluated sum whose low part may exceed half an ulp of the high part;
// every operation above takes such pairs.  With g_lo = 0 the fast step loop
// renormalises every second step only (over 2e4 smooth steps no loss:
// 2-3e-14 for r = 0.125 ... 3).  With g_lo != 0 it renormalises every step:
// skipping it there brought the systematic error back (2.0e-12 at r = 0.3
// against 1.4e-13), the unnormalised high parts feeding the same fixed-
// pattern products.
template <bool GL, bool NORM = true>
__device__ __forceinline__ void df_axpy(float xh, float xl, float gh, float gl, float ph, float pl, float &oh,
                                        float &ol)
{
    const float q = __fmul_rn(gh, ph);
    const float qe = __fmaf_rn(gh, ph, -q);
    const float c = df_prod_lo<GL>(gh, gl, ph, pl, qe);
    float s, e;
    two_sum(xh, q, s, e);
    if constexpr (NORM) {
        fast_two_sum(s, __fadd_rn(e, __fadd_rn(xl, c)), oh, ol);
    } else {
        oh = s;
        ol = __fadd_rn(e, __fadd_rn(xl, c));
    }
}

// (oh, ol) = a * x.
__device__ __forceinline__ void df_mul(float ah, float al, float xh, float xl, float &oh, float &ol)
{
    const float q = __fmul_rn(ah, xh);
    const float qe = __fmaf_rn(ah, xh, -q);
    fast_two_sum(q, df_prod_lo<true>(ah, al, xh, xl, qe), oh, ol);
}

// (oh, ol) = a + b.
__device__ __forceinline__ void df_add(float ah, float al, float bh, float bl, float &oh, float &ol)
{
    float s, e;
    two_sum(ah, bh, s, e);
    fast_two_sum(s, __fadd_rn(e, __fadd_rn(al, bl)), oh, ol);
}

// Split a double into (hi, lo): hi = fl32(x), lo = fl32(x - hi) (x - hi is
// exact in double).
__device__ __forceinline__ void df_split(double x, float &h, float &l)
{
    h = __double2float_rn(x);
    l = __double2float_rn(x - (double)h);
}

// The smallest e with |x| < 2^e for a finite nonzero double, from its bits.
__device__ __forceinline__ int df_exponent_bound(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
    const int field = (int)(b >> 52);
    if (field != 0)
        return field - 1022;
    const int top = 63 - __clzll((long long)b);  // subnormal: highest mantissa bit
    return top - 1073;
}


// CTA-row layout of the double-float kernels: one 128-byte row (16 points as
// (hi, lo) pairs or doubles) per thread, kTileRows threads.
constexpr int kDfNT = kTileRows;  // one 128-byte row (16 points) per thread
constexpr int kDfK = kRowBytes / 8;
constexpr int kDfNW = kDfNT / 32;
#ifndef GE_TB_MINBLOCKS_DF
#define GE_TB_MINBLOCKS_DF 2
#endif

struct DfC {
    float h, l;
};

// Cross-thread exchange of (hi, lo) pairs: L = left thread's last point,
// R = right thread's first point.  Warp edges go through a double-buffered
// shared slot and one CTA barrier.
struct DfExch {
    float2 (*slot)[kDfNW][2];
    int eb, lane, warp;
};

__device__ __forceinline__ void df_exchange(const float (&h)[kDfK], const float (&l)[kDfK], DfC &L, DfC &R,
                                            DfExch &x)
{
    L.h = __shfl_up_sync(0xffffffffu, h[kDfK - 1], 1);
    L.l = __shfl_up_sync(0xffffffffu, l[kDfK - 1], 1);
    R.h = __shfl_down_sync(0xffffffffu, h[0], 1);
    R.l = __shfl_down_sync(0xffffffffu, l[0], 1);
    if (x.lane == 0)
        x.slot[x.eb][x.warp][0] = make_float2(h[0], l[0]);
    if (x.lane == 31)
        x.slot[x.eb][x.warp][1] = make_float2(h[kDfK - 1], l[kDfK - 1]);
    __syncthreads();
    if (x.lane == 0 && x.warp > 0) {
        const float2 v = x.slot[x.eb][x.warp - 1][1];
        L = DfC{v.x, v.y};
    }
    if (x.lane == 31 && x.warp < kDfNW - 1) {
        const float2 v = x.slot[x.eb][x.warp + 1][0];
        R = DfC{v.x, v.y};
    }
    x.eb ^= 1;
}

// Partner value of register j under grouping Q (j - 1 = -1 is L, j + 1 = K
// is R).
template <int Q>
__device__ __forceinline__ DfC df_partner(const float (&h)[kDfK], const float (&l)[kDfK], int j, DfC L, DfC R)
{
    const int pj = partner_reg<Q>(j);
    if (pj < 0)
        return L;
    if (pj >= kDfK)
        return R;
    return DfC{h[pj], l[pj]};
}

// One stage with every check: group members get A x + B x_partner (mid:
// A = 1, the scaled map), singletons S x, the wall points add fl / fr
// (WALLS), points outside the grid keep their value.
template <int Q, bool MID, bool WALLS, bool GL = true>
__device__ __forceinline__ void df_stage_checked(float (&h)[kDfK], float (&l)[kDfK], DfC A, DfC B, DfC S, DfC fl,
                                                 DfC fr, Span sp, DfExch &x)
{
    DfC L{0.0f, 0.0f}, R{0.0f, 0.0f};
    if constexpr (Q == 1)
        df_exchange(h, l, L, R, x);
    float nh[kDfK], nl[kDfK];
#pragma unroll
    for (int j = 0; j < kDfK; ++j) {
        const int pj = partner_reg<Q>(j);
        const bool inside = (j >= sp.jlo) && (j < sp.jhi);
        const bool paired = (pj >= sp.jlo) && (pj < sp.jhi);
        const DfC p = df_partner<Q>(h, l, j, L, R);
        float vh, vl;
        if (paired) {
            if constexpr (MID) {
                df_axpy<GL>(h[j], l[j], B.h, B.l, p.h, p.l, vh, vl);
            } else {
                float ah, al;
                df_mul(A.h, A.l, h[j], l[j], ah, al);
                df_axpy<true>(ah, al, B.h, B.l, p.h, p.l, vh, vl);
            }
        } else {
            df_mul(S.h, S.l, h[j], l[j], vh, vl);
        }
        if constexpr (WALLS) {
            if (j == sp.jlo)
                df_add(vh, vl, fl.h, fl.l, vh, vl);
            if (j == sp.jhi - 1)
                df_add(vh, vl, fr.h, fr.l, vh, vl);
        }
        nh[j] = inside ? vh : h[j];
        nl[j] = inside ? vl : l[j];
    }
#pragma unroll
    for (int j = 0; j < kDfK; ++j) {
        h[j] = nh[j];
        l[j] = nl[j];
    }
}

// One scaled block step x <- x + g x_partner on a thread whose points and
// partners all lie inside the grid, none a wall point.
template <int Q, bool GL, bool NORM>
__device__ __forceinline__ void df_mid_fast(float (&h)[kDfK], float (&l)[kDfK], DfC g, DfExch &x)
{
    if constexpr (Q == 0) {
#pragma unroll
        for (int j = 0; j < kDfK; j += 2) {
            float ah, al, bh, bl;
            df_axpy<GL, NORM>(h[j], l[j], g.h, g.l, h[j + 1], l[j + 1], ah, al);
            df_axpy<GL, NORM>(h[j + 1], l[j + 1], g.h, g.l, h[j], l[j], bh, bl);
            h[j] = ah;
            l[j] = al;
            h[j + 1] = bh;
            l[j + 1] = bl;
        }
    } else {
        DfC L, R;
        df_exchange(h, l, L, R, x);
        float fh, fl, kh, kl;
        df_axpy<GL, NORM>(h[0], l[0], g.h, g.l, L.h, L.l, fh, fl);
        df_axpy<GL, NORM>(h[kDfK - 1], l[kDfK - 1], g.h, g.l, R.h, R.l, kh, kl);
#pragma unroll
        for (int j = 1; j + 1 < kDfK; j += 2) {
            float ah, al, bh, bl;
            df_axpy<GL, NORM>(h[j], l[j], g.h, g.l, h[j + 1], l[j + 1], ah, al);
            df_axpy<GL, NORM>(h[j + 1], l[j + 1], g.h, g.l, h[j], l[j], bh, bl);
            h[j] = ah;
            l[j] = al;
            h[j + 1] = bh;
            l[j + 1] = bl;
        }
        h[0] = fh;
        l[0] = fl;
        h[kDfK - 1] = kh;
        l[kDfK - 1] = kl;
    }
}

}  // namespace
}  // namespace ge
