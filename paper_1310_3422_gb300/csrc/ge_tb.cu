// ge_tb.cu -- tiled multi-step GE kernel (GE_KERNEL_TEMPORAL, and
// GE_KERNEL_ONESTEP as its one-step-per-launch case).
//
// The scheme (arXiv:1310.3422 Sec. 2, sub-domain width 1) advances u by
//     (I + r G_p) u^{s+1} = (I - r G_{1-p}) u^s + f,   p = s mod 2,
// where G_p is the block diagonal of [[1,-1],[-1,1]] on the parity-p groups
// and [1] on singletons, and f = r beta_l e_0 + r beta_r e_{n-1} holds the
// wall terms.  Solving each group's 2x2 system is Eqs. (cc)/(dd).
//
// This kernel carries the right-hand side w^s = (I - r G_{1-p}) u^s + f of
// each step instead of u.  Then
//     w^{s+1} = (I - r G_p)(I + r G_p)^{-1} w^s + f,
// and the block map on one group is [[1, 2r], [2r, 1]] / (1+2r) (on a
// singleton (1-r)/(1+r)): one fused multiply-add per point and step when the
// common factor 1/(1+2r) is kept out of the data (scaled form: every point is
// x <- x + 2r x_partner; the scale sigma = (1+2r)^m is a scalar kept by the
// host, brought back by exact powers of two and folded into the exit).  Entry and exit:
//     w = (1-r) u_i + r u_partner(1-p) [+ r beta at the walls],
//     u = ((1+r) w_i + r w_partner(p)) / (1+2r)   (singleton: w_i/(1+r)).
// This is the same linear map as the step-by-step scheme, reassociated.
//
// Layout.  A tile is kTileRows rows of 128 bytes (8192 floats or 4096
// doubles), loaded by a 2D TMA copy (cp.async.bulk.tensor, 128-byte swizzle
// so that a thread's row read is bank-conflict free) into one of two shared
// buffers while the previous tile is computed.  Each thread holds RPT
// consecutive rows in registers (its first point has an even index, so
// parity-0 groups never cross threads and parity-1 groups cross one thread
// boundary, bridged by warp shuffles).  Two layouts (chosen per precision):
//  * CTA rows: thread t owns row t; warp edges go through shared memory with
//    one CTA barrier per parity-1 step; the halo sits only at the tile ends;
//  * warp windows: every warp owns a window of 32*RPT rows with its own halo
//    (windows of neighbouring warps overlap), so the step loop has no barrier.
// The halo H >= (stages in the launch) points per side: the dependency cone
// grows one point per stage, so after the launch the corrupted margin is
// still inside the halo.  Results go back through the same buffer and leave
// with coalesced 16-byte stores.
//
// Compensated FP32 (GE_F32_COMP): the block map is applied in normalised
// form x <- x + d (x_partner - x), d = 2r/(1+2r), and each point's updates
// are Kahan-summed into (hi, lo); lo lives in registers for the launch.
#include <cuda.h>
#include <cstdint>

#include "ge_internal.h"

namespace ge {
namespace {

constexpr long long kWaitLimitCycles = 4000000000LL;  // about 2 s of SM clock

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the barrier; give up after kWaitLimitCycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitLimitCycles)
            return false;
    }
    return true;
}

// 2D tiled TMA load: box origin (x = 0, y = row), completes on `bar`.
__device__ __forceinline__ void tma_load_rows(void *dst, const CUtensorMap *map, uint64_t *bar,
                                              int row)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(row), "r"(smem_addr(bar))
        : "memory");
}

// 16-byte chunk c of a thread's registers <-> shared memory.
template <int K>
__device__ __forceinline__ void chunk_to_regs(const unsigned char *p, float (&v)[K], int c)
{
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[4 * c + 0] = q.x;
    v[4 * c + 1] = q.y;
    v[4 * c + 2] = q.z;
    v[4 * c + 3] = q.w;
}
template <int K>
__device__ __forceinline__ void chunk_to_regs(const unsigned char *p, double (&v)[K], int c)
{
    const double2 q = *reinterpret_cast<const double2 *>(p);
    v[2 * c + 0] = q.x;
    v[2 * c + 1] = q.y;
}
template <int K>
__device__ __forceinline__ void regs_to_chunk(unsigned char *p, const float (&v)[K], int c)
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
}
template <int K>
__device__ __forceinline__ void regs_to_chunk(unsigned char *p, const double (&v)[K], int c)
{
    *reinterpret_cast<double2 *>(p) = make_double2(v[2 * c], v[2 * c + 1]);
}

// Value of the partner of register j under grouping Q.  The thread's first
// point has an even global index, so register parity = point parity: the
// partner is point+1 when (j + Q) is even, else point-1.  L / R are the left
// thread's last and the right thread's first value.
template <int Q, int K, typename Real>
__device__ __forceinline__ Real pval(const Real (&v)[K], int j, Real L, Real R)
{
    if (((j + Q) & 1) == 0)
        return (j + 1 < K) ? v[j + 1] : R;
    return (j >= 1) ? v[j - 1] : L;
}

// The thread's registers in local coordinates: register j is grid point
// g0 + j; points jlo..jhi-1 (clamped to [-1, K+1]) lie inside the grid, so
// register jlo is grid point 0 and register jhi-1 grid point n-1 when they
// fall in 0..K-1.  A partner register j +- 1 is inside iff jlo <= j +- 1 < jhi.
struct Span {
    int jlo, jhi;
};

template <int K>
__device__ __forceinline__ Span make_span(long long g0, long long n)
{
    long long lo = -g0, hi = n - g0;
    lo = lo < -1 ? -1 : (lo > K + 1 ? K + 1 : lo);
    hi = hi < -1 ? -1 : (hi > K + 1 ? K + 1 : hi);
    return Span{(int)lo, (int)hi};
}

template <int Q>
__device__ __forceinline__ int partner_reg(int j)
{
    return (((j + Q) & 1) == 0) ? j + 1 : j - 1;
}

// Cross-thread neighbour exchange.  Warp-window layout (WT): every warp
// carries its own halo, so neighbours come from warp shuffles only (lanes 0
// and 31 get their own value back: garbage that stays inside the halo).
// CTA-row layout: warp edges go through a double-buffered shared slot and
// one CTA barrier per exchange.
template <typename Real, int NW, bool WT>
struct Exch {
    Real (*slot)[NW][2];
    int eb;
    int lane;
    int warp;
};

// L = left thread's last value, R = right thread's first value (parity-1
// groups cross thread boundaries).
template <typename Real, int K, int NW, bool WT>
__device__ __forceinline__ void exchange(const Real (&v)[K], Real &L, Real &R, Exch<Real, NW, WT> &x)
{
    L = __shfl_up_sync(0xffffffffu, v[K - 1], 1);
    R = __shfl_down_sync(0xffffffffu, v[0], 1);
    if constexpr (!WT) {
        if (x.lane == 0)
            x.slot[x.eb][x.warp][0] = v[0];
        if (x.lane == 31)
            x.slot[x.eb][x.warp][1] = v[K - 1];
        __syncthreads();
        if (x.lane == 0 && x.warp > 0)
            L = x.slot[x.eb][x.warp - 1][1];
        if (x.lane == 31 && x.warp < NW - 1)
            R = x.slot[x.eb][x.warp + 1][0];
        x.eb ^= 1;
    }
}

enum StageKind { kEntry = 0, kMid = 1, kExit = 2, kMidN = 3 };

template <typename Real>
struct StageC {
    Real a, b, s, fl, fr;
};

// One stage on a thread's K registers.
//   entry: v <- (1-r) v + r v_p      (a = r, b = 1-r; singleton: b v)
//   mid:   v <- v + 2r v_p           (a = 2r;         singleton: s v)  scaled form
//   midN:  v <- v + d (v_p - v)      (a = 2r/(1+2r);  singleton: s v)  normalised form
//   exit:  v <- x1 v + x2 v_p        (a = x1, b = x2; singleton: s v)
// Entry and mid add the wall terms fl / fr at points 0 and n-1.  With
// EDGE = false every point of the thread and every partner lies inside the
// grid and none is a wall point, so no checks are compiled.  With EDGE = true
// singletons and wall terms are applied and points outside [0, n) keep their
// value (see Span).
template <int Q, int KIND, bool EDGE, int K, typename Real>
__device__ __forceinline__ void stage(Real (&v)[K], Real L, Real R, Span sp, const StageC<Real> &c)
{
    Real nv[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const Real p = pval<Q>(v, j, L, R);
        if (KIND == kEntry)
            nv[j] = fma(c.a, p, c.b * v[j]);
        else if (KIND == kMid)
            nv[j] = fma(c.a, p, v[j]);
        else if (KIND == kMidN)
            nv[j] = fma(c.a, p - v[j], v[j]);
        else
            nv[j] = fma(c.a, v[j], c.b * p);
    }
    if constexpr (EDGE) {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int pj = partner_reg<Q>(j);
            const bool inside = (j >= sp.jlo) && (j < sp.jhi);
            const bool paired = (pj >= sp.jlo) && (pj < sp.jhi);
            Real val;
            if (KIND == kEntry)
                val = paired ? nv[j] : c.b * v[j];
            else
                val = paired ? nv[j] : c.s * v[j];
            if (KIND != kExit) {
                if (j == sp.jlo)
                    val += c.fl;
                if (j == sp.jhi - 1)
                    val += c.fr;
            }
            nv[j] = inside ? val : v[j];
        }
    }
#pragma unroll
    for (int j = 0; j < K; ++j)
        v[j] = nv[j];
}

// Exact 2^-e (0 <= e <= 1022 for double, 0 <= e <= 126 for float).
template <typename Real>
__device__ __forceinline__ Real pow2neg(int e);
template <>
__device__ __forceinline__ double pow2neg<double>(int e)
{
    return __longlong_as_double(static_cast<long long>(1023 - e) << 52);
}
template <>
__device__ __forceinline__ float pow2neg<float>(int e)
{
    return __int_as_float((127 - e) << 23);
}

// Scaled block step of this launch.  Only warps on the checked path (EDGE)
// need the wall terms; they carry the scale sigma of the right-hand side in
// double, with the same recurrence the host runs (see TbParams).
template <int Q, bool EDGE, typename Real, int K, int NW, bool WT>
__device__ __forceinline__ void mid_scaled(Real (&v)[K], double &sig, const TbParams &P, Exch<Real, NW, WT> &x,
                                           Span sp, Real g, Real kap)
{
    Real L = 0, R = 0;
    if (Q == 1)
        exchange(v, L, R, x);
    StageC<Real> c{g, (Real)0, kap, (Real)0, (Real)0};
    if constexpr (EDGE) {
        sig *= P.onepg;
        c.fl = (Real)(sig * P.f_l);
        c.fr = (Real)(sig * P.f_r);
    }
    stage<Q, kMid, EDGE>(v, L, R, sp, c);
}

// `count` block steps m0 .. m0+count-1, step m having grouping parity
// (p_first + m) & 1: an odd first step alone, then pairs, then an even
// trailing step.  No rescaling inside.
template <bool EDGE, typename Real, int K, int NW, bool WT>
__device__ __forceinline__ void mid_run(Real (&v)[K], int m0, int count, double &sig, const TbParams &P,
                                        Exch<Real, NW, WT> &x, Span sp, Real g, Real kap)
{
    int m = m0;
    const int end = m0 + count;
    if (m < end && ((P.p_first + m) & 1)) {
        mid_scaled<1, EDGE>(v, sig, P, x, sp, g, kap);
        ++m;
    }
    for (; m + 1 < end; m += 2) {
        mid_scaled<0, EDGE>(v, sig, P, x, sp, g, kap);
        mid_scaled<1, EDGE>(v, sig, P, x, sp, g, kap);
    }
    if (m < end)
        mid_scaled<0, EDGE>(v, sig, P, x, sp, g, kap);
}

// Entry, the launch's block steps (in runs between rescalings) and exit on
// one tile (scaled form).
template <bool EDGE, typename Real, int K, int NW, bool WT>
__device__ __forceinline__ void run_scaled(Real (&v)[K], const TbParams &P, Exch<Real, NW, WT> &x, Span sp)
{
    Real L = 0, R = 0;
    if (P.do_entry) {
        const StageC<Real> c{(Real)P.r, (Real)P.omr, (Real)0, (Real)P.f_l, (Real)P.f_r};
        if (((1 - P.p_first) & 1) == 1) {
            exchange(v, L, R, x);
            stage<1, kEntry, EDGE>(v, L, R, sp, c);
        } else {
            stage<0, kEntry, EDGE>(v, L, R, sp, c);
        }
    }
    const Real g = (Real)P.g, kap = (Real)P.kappa;
    double sig = P.sigma_in;  // used on the checked path only
    int until = P.rescale_phase, ev = 0, m = 0;
    while (m < P.n_mid) {
        int count = P.n_mid - m;
        if (until > 0 && until < count)
            count = until;
        mid_run<EDGE>(v, m, count, sig, P, x, sp, g, kap);
        m += count;
        if (until > 0) {
            until -= count;
            if (until == 0) {
                until = P.rescale_every;
                const int e = P.rs_exp[ev++];
                const Real s = pow2neg<Real>(e);
#pragma unroll
                for (int j = 0; j < K; ++j)
                    v[j] *= s;
                if constexpr (EDGE)
                    sig *= pow2neg<double>(e);
            }
        }
    }
    if (P.do_exit) {
        // x1, x2, xs arrive divided by the final scale
        const StageC<Real> c{(Real)P.x1, (Real)P.x2, (Real)P.xs, (Real)0, (Real)0};
        if (((P.p_first + P.n_mid) & 1) == 1) {
            exchange(v, L, R, x);
            stage<1, kExit, EDGE>(v, L, R, sp, c);
        } else {
            stage<0, kExit, EDGE>(v, L, R, sp, c);
        }
    }
}

// Kahan sum of an update into (hi, lo).
__device__ __forceinline__ void kahan_add(float &hi, float &lo, float delta)
{
    const float y = delta + lo;
    const float s = hi + y;
    lo = y - (s - hi);
    hi = s;
}

// Update of register j in the checked compensated step: d (x_p - x) for a
// group member, (kappa - 1)(hi + lo) for a singleton, plus the wall terms;
// zero outside the grid.
template <int Q>
__device__ __forceinline__ float comp_delta(int j, float self, float lself, float partner, float d,
                                            float km1, float fl, float fr, Span sp)
{
    const int pj = partner_reg<Q>(j);
    const bool inside = (j >= sp.jlo) && (j < sp.jhi);
    const bool paired = (pj >= sp.jlo) && (pj < sp.jhi);
    float val = paired ? d * (partner - self) : km1 * (self + lself);
    if (j == sp.jlo)
        val += fl;
    if (j == sp.jhi - 1)
        val += fr;
    return inside ? val : 0.0f;
}

// Compensated block step: normalised form x <- x + d (x_p - x), the update
// Kahan-summed into (hi, lo); singleton x <- x + (kappa - 1) x + wall term.
// The members of a group get opposite updates t and -t.
template <int Q, bool EDGE, int K, int NW, bool WT>
__device__ __forceinline__ void mid_comp(float (&v)[K], float (&lo)[K], const TbParams &P, float d,
                                         float km1, float fl, float fr, Exch<float, NW, WT> &x, Span sp)
{
    float L = 0.0f, R = 0.0f;
    if (Q == 1)
        exchange(v, L, R, x);
    if constexpr (!EDGE) {
        if (Q == 0) {
#pragma unroll
            for (int j = 0; j < K; j += 2) {
                const float t = d * (v[j + 1] - v[j]);
                kahan_add(v[j], lo[j], t);
                kahan_add(v[j + 1], lo[j + 1], -t);
            }
        } else {
            const float t0 = d * (L - v[0]);
            const float tk = d * (R - v[K - 1]);
#pragma unroll
            for (int j = 1; j + 1 < K; j += 2) {
                const float t = d * (v[j + 1] - v[j]);
                kahan_add(v[j], lo[j], t);
                kahan_add(v[j + 1], lo[j + 1], -t);
            }
            kahan_add(v[0], lo[0], t0);
            kahan_add(v[K - 1], lo[K - 1], tk);
        }
    } else {
        // checked path, still pair by pair from the old values
        if (Q == 0) {
#pragma unroll
            for (int j = 0; j < K; j += 2) {
                const float a = comp_delta<Q>(j, v[j], lo[j], v[j + 1], d, km1, fl, fr, sp);
                const float b = comp_delta<Q>(j + 1, v[j + 1], lo[j + 1], v[j], d, km1, fl, fr, sp);
                kahan_add(v[j], lo[j], a);
                kahan_add(v[j + 1], lo[j + 1], b);
            }
        } else {
            const float a0 = comp_delta<Q>(0, v[0], lo[0], L, d, km1, fl, fr, sp);
            const float ak = comp_delta<Q>(K - 1, v[K - 1], lo[K - 1], R, d, km1, fl, fr, sp);
#pragma unroll
            for (int j = 1; j + 1 < K; j += 2) {
                const float a = comp_delta<Q>(j, v[j], lo[j], v[j + 1], d, km1, fl, fr, sp);
                const float b = comp_delta<Q>(j + 1, v[j + 1], lo[j + 1], v[j], d, km1, fl, fr, sp);
                kahan_add(v[j], lo[j], a);
                kahan_add(v[j + 1], lo[j + 1], b);
            }
            kahan_add(v[0], lo[0], a0);
            kahan_add(v[K - 1], lo[K - 1], ak);
        }
    }
}

template <bool EDGE, int K, int NW, bool WT>
__device__ __forceinline__ void run_comp(float (&v)[K], const TbParams &P, Exch<float, NW, WT> &x, Span sp)
{
    float L = 0.0f, R = 0.0f;
    if (P.do_entry) {
        const StageC<float> c{(float)P.r, (float)P.omr, 0.0f, (float)P.f_l, (float)P.f_r};
        if (((1 - P.p_first) & 1) == 1) {
            exchange(v, L, R, x);
            stage<1, kEntry, EDGE>(v, L, R, sp, c);
        } else {
            stage<0, kEntry, EDGE>(v, L, R, sp, c);
        }
    }
    float lo[K];
#pragma unroll
    for (int j = 0; j < K; ++j)
        lo[j] = 0.0f;
    const float d = (float)P.d, km1 = (float)(P.kappa - 1.0);
    const float fl = (float)P.f_l, fr = (float)P.f_r;
    int m = 0;
    if (P.n_mid > 0 && (P.p_first & 1)) {
        mid_comp<1, EDGE>(v, lo, P, d, km1, fl, fr, x, sp);
        m = 1;
    }
    for (; m + 1 < P.n_mid; m += 2) {
        mid_comp<0, EDGE>(v, lo, P, d, km1, fl, fr, x, sp);
        mid_comp<1, EDGE>(v, lo, P, d, km1, fl, fr, x, sp);
    }
    if (m < P.n_mid)
        mid_comp<0, EDGE>(v, lo, P, d, km1, fl, fr, x, sp);
    // fold the compensation word in (one rounding, below the final FP32 store's)
#pragma unroll
    for (int j = 0; j < K; ++j)
        v[j] += lo[j];
    if (P.do_exit) {
        const StageC<float> c{(float)P.x1, (float)P.x2, (float)P.xs, 0.0f, 0.0f};
        if (((P.p_first + P.n_mid) & 1) == 1) {
            exchange(v, L, R, x);
            stage<1, kExit, EDGE>(v, L, R, sp, c);
        } else {
            stage<0, kExit, EDGE>(v, L, R, sp, c);
        }
    }
}

// Compile-time layout of the tiled kernel (tuning knobs).
//   GE_TB_WT_*: 1 = warp windows (each warp carries its own halo; no barrier
//             in the step loop), 0 = CTA rows (one CTA barrier per parity-1
//             step, halo only at the tile's two ends).
//   GE_TB_RPT_*: 128-byte rows per thread (warp windows only).
//   GE_TB_MINBLOCKS_*: CTAs per SM the register budget is sized for.
#ifndef GE_TB_WT_F64
#define GE_TB_WT_F64 0
#endif
#ifndef GE_TB_WT_F32
#define GE_TB_WT_F32 1
#endif
#ifndef GE_TB_WT_COMP
#define GE_TB_WT_COMP 0
#endif
#ifndef GE_TB_RPT_F64
#define GE_TB_RPT_F64 2
#endif
#ifndef GE_TB_RPT_F32
#define GE_TB_RPT_F32 1
#endif
#ifndef GE_TB_RPT_COMP
#define GE_TB_RPT_COMP 1
#endif
#ifndef GE_TB_MINBLOCKS_F64
#define GE_TB_MINBLOCKS_F64 2
#endif
#ifndef GE_TB_MINBLOCKS_F32
#define GE_TB_MINBLOCKS_F32 2
#endif
#ifndef GE_TB_MINBLOCKS_COMP
#define GE_TB_MINBLOCKS_COMP 2
#endif

template <typename Real, bool COMP>
struct Layout {
    static constexpr bool WT =
        (sizeof(Real) == 8 ? GE_TB_WT_F64 : (COMP ? GE_TB_WT_COMP : GE_TB_WT_F32)) != 0;
    static constexpr int RPT = !WT ? 1 : (sizeof(Real) == 8 ? GE_TB_RPT_F64 : (COMP ? GE_TB_RPT_COMP : GE_TB_RPT_F32));
    static constexpr int NT = kTileRows / RPT;                  // threads per CTA
    static constexpr int KR = kRowBytes / (int)sizeof(Real);    // elements per row
    static constexpr int KT = KR * RPT;                          // elements per thread
    static constexpr int MINB =
        sizeof(Real) == 8 ? GE_TB_MINBLOCKS_F64 : (COMP ? GE_TB_MINBLOCKS_COMP : GE_TB_MINBLOCKS_F32);
};

template <typename Real, bool COMP>
__global__ void __launch_bounds__(Layout<Real, COMP>::NT, Layout<Real, COMP>::MINB)
    tb_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ TbParams P)
{
    using LY = Layout<Real, COMP>;
    constexpr bool WT = LY::WT;
    constexpr int RPT = LY::RPT, NT = LY::NT, KR = LY::KR, K = LY::KT;
    constexpr int NW = NT / 32;
    constexpr int CH = kRowBytes / 16;
    constexpr uint32_t kTileBytes = kTileRows * kRowBytes;

    extern __shared__ unsigned char smem_raw[];
    unsigned char *tiles = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ Real slot[2][NW][2];

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int hr = P.H / KR;  // halo rows of the tile
    const int ur = P.U / KR;  // output rows of the tile
    // first tile row of this thread: CTA rows -> row t; warp windows ->
    // warp w starts where warp w-1's output ends (windows overlap by 2 halos)
    const int ht = P.H / K;                                   // halo threads per warp side
    const int my_row = WT ? (warp * (32 - 2 * ht) + lane) * RPT : t;
    const bool writes = WT ? (lane >= ht && lane < 32 - ht) : true;
    Exch<Real, NW, WT> x{slot, 0, lane, warp};

    if (t == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    long long tile = blockIdx.x;
    if (t == 0 && tile < P.n_tiles) {
        mbar_arrive_expect_tx(&mbar[0], kTileBytes);
        tma_load_rows(tiles, &tmap, &mbar[0], (int)(tile * ur - hr));
    }
    for (long long it = 0; tile < P.n_tiles; ++it, tile += gridDim.x) {
        const int b = (int)(it & 1);
        unsigned char *cur = tiles + b * kTileBytes;
        const long long next = tile + gridDim.x;
        const bool prefetch = next < P.n_tiles;
        if (t == 0 && prefetch) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&mbar[b ^ 1], kTileBytes);
            tma_load_rows(tiles + (b ^ 1) * kTileBytes, &tmap, &mbar[b ^ 1], (int)(next * ur - hr));
        }
        const bool ok = mbar_wait_bounded(&mbar[b], (uint32_t)((it >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            if (t == 0) {
                atomicExch(P.err, kDevTimeout);
                if (prefetch)  // let our own copy in flight land before leaving
                    mbar_wait_bounded(&mbar[b ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
            }
            return;
        }

        Real v[K];
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
            const int row = my_row + i;
            const unsigned char *rp = cur + row * kRowBytes;
#pragma unroll
            for (int c = 0; c < CH; ++c)
                chunk_to_regs<K>(rp + ((c ^ (row & 7)) << 4), v, i * CH + c);
        }
        if constexpr (WT)
            __syncthreads();  // windows overlap: every load before any write-back
        const long long g0 = tile * P.U - P.H + (long long)my_row * KR;
        // the whole warp takes the checked path if any lane holds a wall
        // point, a point outside the grid, or a partner outside it
        const bool edge_thr = !(g0 >= 1 && g0 + K <= P.n - 1);
        const bool edge_warp = __any_sync(0xffffffffu, edge_thr);
        const Span sp = make_span<K>(g0, P.n);
        if constexpr (!COMP) {
            if (edge_warp)
                run_scaled<true>(v, P, x, sp);
            else
                run_scaled<false>(v, P, x, sp);
        } else {
            if (edge_warp)
                run_comp<true>(v, P, x, sp);
            else
                run_comp<false>(v, P, x, sp);
        }

        // write back the output rows, then copy them out with coalesced stores
        if (writes) {
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
                const int row = my_row + i;
                unsigned char *rp = cur + row * kRowBytes;
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    regs_to_chunk<K>(rp + ((c ^ (row & 7)) << 4), v, i * CH + c);
            }
        }
        __syncthreads();
        {
            const long long grow0 = tile * ur;
            unsigned char *out = static_cast<unsigned char *>(P.out);
            for (int ch = t; ch < ur * CH; ch += NT) {
                const int lr = hr + ch / CH;
                const int c = ch % CH;
                const long long gr = grow0 + ch / CH;
                if (gr < P.n_rows) {
                    const uint4 val = *reinterpret_cast<const uint4 *>(cur + lr * kRowBytes +
                                                                       ((c ^ (lr & 7)) << 4));
                    *reinterpret_cast<uint4 *>(out + gr * kRowBytes + c * 16) = val;
                }
            }
        }
        __syncthreads();
    }
}

template <typename Real, bool COMP>
cudaError_t launch_one(const void *tmap, const TbParams &p, int grid, cudaStream_t s)
{
    const CUtensorMap *m = static_cast<const CUtensorMap *>(tmap);
    tb_kernel<Real, COMP><<<grid, Layout<Real, COMP>::NT, tb_smem_bytes(), s>>>(*m, p);
    return cudaGetLastError();
}

template <typename Real, bool COMP>
cudaError_t set_attr_and_occupancy(int *blocks)
{
    cudaError_t e = cudaFuncSetAttribute(tb_kernel<Real, COMP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, tb_smem_bytes());
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, tb_kernel<Real, COMP>,
                                                         Layout<Real, COMP>::NT, tb_smem_bytes());
}

template <typename Real, bool COMP>
bool geometry(int reach, int *H, int *U)
{
    using LY = Layout<Real, COMP>;
    const int ht = (reach + LY::KT - 1) / LY::KT;  // halo, in threads
    if (LY::WT) {
        if (2 * ht >= 32)
            return false;
        *H = ht * LY::KT;
        *U = (LY::NT / 32) * (32 - 2 * ht) * LY::KT;
    } else {
        *H = ht * LY::KT;
        *U = LY::NT * LY::KT - 2 * *H;
        if (*U <= 0)
            return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Batched kernel: many independent problems packed back to back in one
// buffer, each starting on a 128-byte row.  The tiles run over the packed
// buffer exactly as for one long problem; every thread looks its problem up
// (row -> problem id), takes that problem's constants and walls, and treats
// points of other problems like points outside its grid.  Normalised block
// map, so no scale bookkeeping: every launch starts and ends unscaled.
// CTA-row layout (one row per thread).

// Entry, block steps and exit of one tile, batched form.
template <bool EDGE, typename Real, int K, int NW, bool WT>
__device__ __forceinline__ void run_batch(Real (&v)[K], const TbbParams &P, const BatchDesc &bd,
                                          Exch<Real, NW, WT> &x, Span sp)
{
    Real L = 0, R = 0;
    if (P.do_entry) {
        const StageC<Real> c{(Real)bd.r, (Real)bd.omr, (Real)0, (Real)bd.f_l, (Real)bd.f_r};
        if (((1 - P.p_first) & 1) == 1) {
            exchange(v, L, R, x);
            stage<1, kEntry, EDGE>(v, L, R, sp, c);
        } else {
            stage<0, kEntry, EDGE>(v, L, R, sp, c);
        }
    }
    const StageC<Real> cm{(Real)bd.d, (Real)0, (Real)bd.kappa, (Real)bd.f_l, (Real)bd.f_r};
    int m = 0;
    if (P.n_mid > 0 && (P.p_first & 1)) {
        exchange(v, L, R, x);
        stage<1, kMidN, EDGE>(v, L, R, sp, cm);
        m = 1;
    }
    for (; m + 1 < P.n_mid; m += 2) {
        stage<0, kMidN, EDGE>(v, L, R, sp, cm);
        exchange(v, L, R, x);
        stage<1, kMidN, EDGE>(v, L, R, sp, cm);
    }
    if (m < P.n_mid)
        stage<0, kMidN, EDGE>(v, L, R, sp, cm);
    if (P.do_exit) {
        const StageC<Real> c{(Real)bd.x1, (Real)bd.x2, (Real)bd.xs, (Real)0, (Real)0};
        if (((P.p_first + P.n_mid) & 1) == 1) {
            exchange(v, L, R, x);
            stage<1, kExit, EDGE>(v, L, R, sp, c);
        } else {
            stage<0, kExit, EDGE>(v, L, R, sp, c);
        }
    }
}

template <bool EDGE, int K, int NW, bool WT>
__device__ __forceinline__ void run_batch_comp(float (&v)[K], const TbbParams &P, const BatchDesc &bd,
                                               Exch<float, NW, WT> &x, Span sp)
{
    float L = 0.0f, R = 0.0f;
    if (P.do_entry) {
        const StageC<float> c{(float)bd.r, (float)bd.omr, 0.0f, (float)bd.f_l, (float)bd.f_r};
        if (((1 - P.p_first) & 1) == 1) {
            exchange(v, L, R, x);
            stage<1, kEntry, EDGE>(v, L, R, sp, c);
        } else {
            stage<0, kEntry, EDGE>(v, L, R, sp, c);
        }
    }
    float lo[K];
#pragma unroll
    for (int j = 0; j < K; ++j)
        lo[j] = 0.0f;
    const float d = (float)bd.d, km1 = (float)(bd.kappa - 1.0);
    const float fl = (float)bd.f_l, fr = (float)bd.f_r;
    TbParams dummy{};
    dummy.n = 0;
    int m = 0;
    if (P.n_mid > 0 && (P.p_first & 1)) {
        mid_comp<1, EDGE>(v, lo, dummy, d, km1, fl, fr, x, sp);
        m = 1;
    }
    for (; m + 1 < P.n_mid; m += 2) {
        mid_comp<0, EDGE>(v, lo, dummy, d, km1, fl, fr, x, sp);
        mid_comp<1, EDGE>(v, lo, dummy, d, km1, fl, fr, x, sp);
    }
    if (m < P.n_mid)
        mid_comp<0, EDGE>(v, lo, dummy, d, km1, fl, fr, x, sp);
#pragma unroll
    for (int j = 0; j < K; ++j)
        v[j] += lo[j];
    if (P.do_exit) {
        const StageC<float> c{(float)bd.x1, (float)bd.x2, (float)bd.xs, 0.0f, 0.0f};
        if (((P.p_first + P.n_mid) & 1) == 1) {
            exchange(v, L, R, x);
            stage<1, kExit, EDGE>(v, L, R, sp, c);
        } else {
            stage<0, kExit, EDGE>(v, L, R, sp, c);
        }
    }
}

// Scaled batched form (FP64 and plain FP32).  The thread's problem is
// shifted by its linear wall profile u* (an exact fixed point of the step:
// the shifted problem has zero walls, so no wall terms and no scale in the
// edge warps), advanced with the scaled block map x <- x + g x_partner (one
// FMA per point and step; singletons x <- kap_s x), multiplied by the
// problem's power of two 2^-e after every R block steps, and brought back to
// the normalised state at the launch end by the factor endf (the inverse of
// the accumulated scale, computed in double-double by batch_endf_kernel).
// Only points inside the problem change: padding keeps its values.
template <bool EDGE, typename Real, int K, int NW, bool WT>
__device__ __forceinline__ void run_batch_scaled(Real (&v)[K], const TbbParams &P, const BatchDesc &bd, int pid,
                                                 long long g0, Exch<Real, NW, WT> &x, Span sp)
{
    Real L = 0, R = 0;
    const Real ua = (Real)bd.ustar_a, ub = (Real)bd.ustar_b;
    if (P.do_entry) {
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (!EDGE || (j >= sp.jlo && j < sp.jhi))
                v[j] -= ua + ub * (Real)(g0 + j + 1);
        const StageC<Real> c{(Real)bd.r, (Real)bd.omr, (Real)0, (Real)0, (Real)0};
        if (((1 - P.p_first) & 1) == 1) {
            exchange(v, L, R, x);
            stage<1, kEntry, EDGE>(v, L, R, sp, c);
        } else {
            stage<0, kEntry, EDGE>(v, L, R, sp, c);
        }
    }
    const StageC<Real> cm{(Real)bd.g, (Real)0, (Real)bd.kap_s, (Real)0, (Real)0};
    int m = 0, q = 0;
    while (m < P.n_mid) {
        const int cnt = (P.n_mid - m < P.R) ? P.n_mid - m : P.R;
        int i = 0;
        if (((P.p_first + m) & 1) == 1) {
            exchange(v, L, R, x);
            stage<1, kMid, EDGE>(v, L, R, sp, cm);
            i = 1;
        }
        for (; i + 1 < cnt; i += 2) {
            stage<0, kMid, EDGE>(v, L, R, sp, cm);
            exchange(v, L, R, x);
            stage<1, kMid, EDGE>(v, L, R, sp, cm);
        }
        if (i < cnt)
            stage<0, kMid, EDGE>(v, L, R, sp, cm);
        m += cnt;
        if (cnt == P.R && pid >= 0) {
            const Real sc = pow2neg<Real>(P.exps[(long long)pid * P.Q + q]);
#pragma unroll
            for (int j = 0; j < K; ++j)
                if (!EDGE || (j >= sp.jlo && j < sp.jhi))
                    v[j] *= sc;
        }
        ++q;
    }
    if (pid >= 0) {
        Real fh, fl;
        if constexpr (sizeof(Real) == 4) {
            const float2 f = reinterpret_cast<const float2 *>(P.endf)[pid];
            fh = f.x, fl = f.y;
        } else {
            fh = reinterpret_cast<const double *>(P.endf)[pid];
            fl = 0;
        }
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (!EDGE || (j >= sp.jlo && j < sp.jhi))
                v[j] = fma(v[j], fh, v[j] * fl);
    }
    if (P.do_exit) {
        const StageC<Real> c{(Real)bd.x1, (Real)bd.x2, (Real)bd.xs, (Real)0, (Real)0};
        if (((P.p_first + P.n_mid) & 1) == 1) {
            exchange(v, L, R, x);
            stage<1, kExit, EDGE>(v, L, R, sp, c);
        } else {
            stage<0, kExit, EDGE>(v, L, R, sp, c);
        }
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (!EDGE || (j >= sp.jlo && j < sp.jhi))
                v[j] += ua + ub * (Real)(g0 + j + 1);
    }
}

// Layout of the batched kernel: GE_TBB_WT_F32 = 1 gives plain FP32 warp
// windows (no barrier in the step loop); FP64 and compensated FP32 use CTA
// rows.
#ifndef GE_TBB_WT_F32
#define GE_TBB_WT_F32 0
#endif

#ifndef GE_TBB_MINB_F32
#define GE_TBB_MINB_F32 3
#endif

template <typename Real, bool COMP>
struct BatchLayout {
    static constexpr bool WT = sizeof(Real) == 4 && !COMP && GE_TBB_WT_F32 != 0;
    static constexpr int MINB = (sizeof(Real) == 4 && !COMP) ? GE_TBB_MINB_F32 : 2;
};

template <typename Real, bool COMP>
__global__ void __launch_bounds__(kTileRows, BatchLayout<Real, COMP>::MINB)
    tbb_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ TbbParams P)
{
    constexpr bool WT = BatchLayout<Real, COMP>::WT;
    constexpr int NT = kTileRows;
    constexpr int K = kRowBytes / (int)sizeof(Real);
    constexpr int NW = NT / 32;
    constexpr int CH = kRowBytes / 16;
    constexpr uint32_t kTileBytes = kTileRows * kRowBytes;

    extern __shared__ unsigned char smem_raw[];
    unsigned char *tiles = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ Real slot[2][NW][2];

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int hr = P.H / K, ur = P.U / K;
    // tile row of this thread: CTA rows -> row t; warp windows -> warp w
    // starts where warp w-1's output ends (windows overlap by 2 halos)
    const int my_row = WT ? warp * (32 - 2 * hr) + lane : t;
    const bool writes = WT ? (lane >= hr && lane < 32 - hr) : true;
    Exch<Real, NW, WT> x{slot, 0, lane, warp};

    if (t == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    long long tile = blockIdx.x;
    if (t == 0 && tile < P.n_tiles) {
        mbar_arrive_expect_tx(&mbar[0], kTileBytes);
        tma_load_rows(tiles, &tmap, &mbar[0], (int)(tile * ur - hr));
    }
    for (long long it = 0; tile < P.n_tiles; ++it, tile += gridDim.x) {
        const int b = (int)(it & 1);
        unsigned char *cur = tiles + b * kTileBytes;
        const long long next = tile + gridDim.x;
        const bool prefetch = next < P.n_tiles;
        if (t == 0 && prefetch) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&mbar[b ^ 1], kTileBytes);
            tma_load_rows(tiles + (b ^ 1) * kTileBytes, &tmap, &mbar[b ^ 1], (int)(next * ur - hr));
        }
        const bool ok = mbar_wait_bounded(&mbar[b], (uint32_t)((it >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            if (t == 0) {
                atomicExch(P.err, kDevTimeout);
                if (prefetch)
                    mbar_wait_bounded(&mbar[b ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
            }
            return;
        }

        Real v[K];
        {
            const unsigned char *rp = cur + my_row * kRowBytes;
#pragma unroll
            for (int c = 0; c < CH; ++c)
                chunk_to_regs<K>(rp + ((c ^ (my_row & 7)) << 4), v, c);
        }
        if constexpr (WT)
            __syncthreads();  // windows overlap: every load before any write-back
        // this thread's problem: rows outside the buffer or in padding have none
        const long long grow = tile * ur - hr + my_row;
        const int pid = (grow >= 0 && grow < P.n_rows) ? __ldg(P.row_pid + grow) : -1;
        BatchDesc bd{};
        Span sp{K + 1, K + 1};  // no point of this thread is inside a grid
        if (pid >= 0) {
            bd = P.desc[pid];
            sp = make_span<K>(grow * K - bd.off, bd.n);
        }
        const bool edge_thr = !(sp.jlo <= -1 && sp.jhi >= K + 1);
        const bool edge_warp = __any_sync(0xffffffffu, edge_thr);
        if constexpr (!COMP) {
            const long long g0 = pid >= 0 ? grow * K - bd.off : 0;
            if (P.scaled) {
                if (edge_warp)
                    run_batch_scaled<true>(v, P, bd, pid, g0, x, sp);
                else
                    run_batch_scaled<false>(v, P, bd, pid, g0, x, sp);
            } else if (edge_warp) {
                run_batch<true>(v, P, bd, x, sp);
            } else {
                run_batch<false>(v, P, bd, x, sp);
            }
        } else {
            if (edge_warp)
                run_batch_comp<true>(v, P, bd, x, sp);
            else
                run_batch_comp<false>(v, P, bd, x, sp);
        }

        if (writes) {
            unsigned char *rp = cur + my_row * kRowBytes;
#pragma unroll
            for (int c = 0; c < CH; ++c)
                regs_to_chunk<K>(rp + ((c ^ (my_row & 7)) << 4), v, c);
        }
        __syncthreads();
        {
            const long long grow0 = tile * ur;
            unsigned char *out = static_cast<unsigned char *>(P.out);
            for (int ch = t; ch < ur * CH; ch += NT) {
                const int lr = hr + ch / CH;
                const int c = ch % CH;
                const long long gr = grow0 + ch / CH;
                if (gr < P.n_rows) {
                    const uint4 val = *reinterpret_cast<const uint4 *>(cur + lr * kRowBytes +
                                                                       ((c ^ (lr & 7)) << 4));
                    *reinterpret_cast<uint4 *>(out + gr * kRowBytes + c * 16) = val;
                }
            }
        }
        __syncthreads();
    }
}

template <typename Real, bool COMP>
cudaError_t launch_batch_one(const void *tmap, const TbbParams &p, int grid, cudaStream_t s)
{
    const CUtensorMap *m = static_cast<const CUtensorMap *>(tmap);
    tbb_kernel<Real, COMP><<<grid, kTileRows, tb_smem_bytes(), s>>>(*m, p);
    return cudaGetLastError();
}

template <typename Real, bool COMP>
cudaError_t batch_attr_and_occupancy(int *blocks)
{
    cudaError_t e = cudaFuncSetAttribute(tbb_kernel<Real, COMP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, tb_smem_bytes());
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, tbb_kernel<Real, COMP>, kTileRows,
                                                         tb_smem_bytes());
}

// Scale bookkeeping of the batched scaled form, one thread per problem, in
// double-double so no rounding drift enters the end factors.  The growth
// per block step is exactly 1 + g with g the coefficient the kernel holds
// (FP32-rounded on the FP32 path).
__device__ __forceinline__ void dd_mul_dev(double &h, double &l, double bh, double bl)
{
    const double p = __dmul_rn(h, bh);
    const double e = __fma_rn(h, bh, -p);
    const double t = __dadd_rn(e, __dadd_rn(__dmul_rn(h, bl), __dmul_rn(l, bh)));
    h = __dadd_rn(p, t);
    l = __dsub_rn(t, __dsub_rn(h, p));
}

__device__ __forceinline__ void growth_dev(const BatchDesc &d, int f32, double &gh, double &gl)
{
    const double g = f32 ? (double)__double2float_rn(d.g) : d.g;
    gh = __dadd_rn(1.0, g);
    gl = __dadd_rn(__dsub_rn(1.0, gh), g);  // exact: 1 + g == gh + gl
}

// exps[b][q]: after block q of R steps (scale starting at 1) the scale is
// brought back into [1, 2) by 2^-exps[b][q].
__global__ void batch_exps_kernel(const BatchDesc *__restrict__ desc, int np, int R, int Q, int f32,
                                  short *__restrict__ exps)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= np)
        return;
    double gh, gl, sh = 1.0, sl = 0.0;
    growth_dev(desc[b], f32, gh, gl);
    for (int q = 0; q < Q; ++q) {
        for (int i = 0; i < R; ++i)
            dd_mul_dev(sh, sl, gh, gl);
        int e2 = 0;
        frexp(sh, &e2);
        const int e = e2 - 1;
        sh = ldexp(sh, -e);
        sl = ldexp(sl, -e);
        exps[(long long)b * Q + q] = (short)e;
    }
}

// endf[b] = 1 / (scale after n_mid block steps with the rescalings above):
// float2 (hi, lo) on the FP32 path, double on the FP64 path.
__global__ void batch_endf_kernel(const BatchDesc *__restrict__ desc, const short *__restrict__ exps, int np, int R,
                                  int Q, int n_mid, int f32, void *endf)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= np)
        return;
    double gh, gl, sh = 1.0, sl = 0.0;
    growth_dev(desc[b], f32, gh, gl);
    for (int m = 0; m < n_mid; ++m) {
        dd_mul_dev(sh, sl, gh, gl);
        if ((m + 1) % R == 0) {
            const int e = exps[(long long)b * Q + (m + 1) / R - 1];
            sh = ldexp(sh, -e);
            sl = ldexp(sl, -e);
        }
    }
    const double ih = __ddiv_rn(1.0, sh);
    const double inv = __dsub_rn(ih, __dmul_rn(ih, __ddiv_rn(sl, sh)));
    if (f32) {
        const float hi = __double2float_rn(inv);
        reinterpret_cast<float2 *>(endf)[b] = make_float2(hi, __double2float_rn(__dsub_rn(inv, (double)hi)));
    } else {
        reinterpret_cast<double *>(endf)[b] = inv;
    }
}

}  // namespace

cudaError_t batch_exps(const BatchDesc *desc, int n_problems, int R, int Q, int f32, short *exps, cudaStream_t s)
{
    batch_exps_kernel<<<(n_problems + 127) / 128, 128, 0, s>>>(desc, n_problems, R, Q, f32, exps);
    return cudaGetLastError();
}

cudaError_t batch_endf(const BatchDesc *desc, const short *exps, int n_problems, int R, int Q, int n_mid, int f32,
                       void *endf, cudaStream_t s)
{
    batch_endf_kernel<<<(n_problems + 127) / 128, 128, 0, s>>>(desc, exps, n_problems, R, Q, n_mid, f32, endf);
    return cudaGetLastError();
}

int tb_smem_bytes() { return 2 * kTileRows * kRowBytes + 1024; }

bool tb_geometry(int prec, int reach, int *H, int *U)
{
    if (prec == 0)
        return geometry<double, false>(reach, H, U);
    if (prec == 1)
        return geometry<float, false>(reach, H, U);
    return geometry<float, true>(reach, H, U);
}

cudaError_t tb_occupancy(int prec, int *blocks)
{
    if (prec == 0)
        return set_attr_and_occupancy<double, false>(blocks);
    if (prec == 1)
        return set_attr_and_occupancy<float, false>(blocks);
    return set_attr_and_occupancy<float, true>(blocks);
}

bool tbb_geometry(int prec, int reach, int *H, int *U)
{
    const int K = kRowBytes / (prec == 0 ? 8 : 4);
    const int ht = (reach + K - 1) / K;
    const bool wt = prec == 1 ? BatchLayout<float, false>::WT : false;
    *H = ht * K;
    if (wt) {
        if (2 * ht >= 32)
            return false;
        *U = (kTileRows / 32) * (32 - 2 * ht) * K;
        return true;
    }
    *U = kTileRows * K - 2 * *H;
    return *U > 0;
}

int tbb_max_depth(int prec)
{
    int H, U, d = kMaxTableSteps;
    while (d > 1 && !tbb_geometry(prec, d + 2, &H, &U))
        --d;
    return d;
}

cudaError_t tbb_occupancy(int prec, int *blocks)
{
    if (prec == 0)
        return batch_attr_and_occupancy<double, false>(blocks);
    if (prec == 1)
        return batch_attr_and_occupancy<float, false>(blocks);
    return batch_attr_and_occupancy<float, true>(blocks);
}

cudaError_t launch_tbb(int prec, const void *tmap, const TbbParams &p, int grid, cudaStream_t s)
{
    if (prec == 0)
        return launch_batch_one<double, false>(tmap, p, grid, s);
    if (prec == 1)
        return launch_batch_one<float, false>(tmap, p, grid, s);
    return launch_batch_one<float, true>(tmap, p, grid, s);
}

cudaError_t launch_tb(int prec, const void *tmap, const TbParams &p, int grid, cudaStream_t s)
{
    if (prec == 0)
        return launch_one<double, false>(tmap, p, grid, s);
    if (prec == 1)
        return launch_one<float, false>(tmap, p, grid, s);
    return launch_one<float, true>(tmap, p, grid, s);
}

}  // namespace ge
