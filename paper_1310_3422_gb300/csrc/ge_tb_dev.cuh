// ge_tb_dev.cuh -- device helpers shared by the tiled kernel (ge_tb.cu) and
// the batched kernel (ge_tbb.cu): bounded mbarrier waits and 2D TMA tile
// loads, register <-> shared-memory chunks, the partner of a register, the
// cross-thread exchange, one stage of the block map, and the compensated
// (Kahan) step.  The scheme itself is described in ge_tb.cu.
#pragma once

#include <cuda.h>
#include <cstdint>

#include "ge_dfma_emu.cuh"
#include "ge_f32x2.cuh"
#include "ge_internal.h"

namespace ge {
namespace {


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

// One arrival on the barrier (release: this thread's earlier shared-memory
// accesses are ordered before the phase completes).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
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

// Wait for phase `parity` of the barrier; give up after `limit` SM cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit)
            return false;
    }
    return true;
}

// The same for a producer lane whose waits last about a tile's compute: it
// sleeps between polls, so that it takes no issue slots from the warps that
// compute on its SM sub-partition.
__device__ __forceinline__ bool mbar_wait_backoff(uint64_t *bar, uint32_t parity, long long limit)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit)
            return false;
        __nanosleep(128);
    }
    return true;
}

// Wait for the tile in buffer b (phase from the iteration).  With the
// diagnostic `stall` > 0 the wait polls `never`, a barrier no thread or copy
// arrives on, and so runs out after `stall` cycles: the failure path below
// then runs exactly as for a tile load that never completes.
__device__ __forceinline__ bool tile_wait(uint64_t *mbar, uint64_t *never, int b, long long it, long long stall)
{
    if (stall > 0)
        return mbar_wait_bounded(never, 0, stall);
    return mbar_wait_bounded(&mbar[b], (uint32_t)((it >> 1) & 1), kWaitLimitCycles);
}

// A tile wait gave up: record GE_ETIMEOUT and let this CTA's own TMA copies
// still in flight (the tile waited for, and the prefetch) land before the
// CTA leaves, each within the default limit.  Called by thread 0 only.
__device__ __forceinline__ void tile_wait_failed(int *err, uint64_t *mbar, int b, long long it, bool prefetch)
{
    atomicExch(err, kDevTimeout);
    mbar_wait_bounded(&mbar[b], (uint32_t)((it >> 1) & 1), kWaitLimitCycles);
    if (prefetch)
        mbar_wait_bounded(&mbar[b ^ 1], (uint32_t)(((it + 1) >> 1) & 1), kWaitLimitCycles);
}

// Tile at position k of a launch's dynamic tile queue.  The two edge tiles
// (the only ones with warps on the checked path, several times slower) go
// first, so the CTAs that take them take fewer tiles in all; then the
// interior tiles in order.
__device__ __forceinline__ long long queue_tile(long long k, long long n_tiles)
{
    if (n_tiles <= 2 || k >= n_tiles)
        return k;
    if (k == 0)
        return 0;
    if (k == 1)
        return n_tiles - 1;
    return k - 1;
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
// groups cross thread boundaries), from the thread's first and last values.
template <typename Real, int NW, bool WT>
__device__ __forceinline__ void exchange_ends(Real first, Real last, Real &L, Real &R, Exch<Real, NW, WT> &x)
{
    L = __shfl_up_sync(0xffffffffu, last, 1);
    R = __shfl_down_sync(0xffffffffu, first, 1);
    if constexpr (!WT) {
        if (x.lane == 0)
            x.slot[x.eb][x.warp][0] = first;
        if (x.lane == 31)
            x.slot[x.eb][x.warp][1] = last;
        __syncthreads();
        if (x.lane == 0 && x.warp > 0)
            L = x.slot[x.eb][x.warp - 1][1];
        if (x.lane == 31 && x.warp < NW - 1)
            R = x.slot[x.eb][x.warp + 1][0];
        x.eb ^= 1;
    }
}

template <typename Real, int K, int NW, bool WT>
__device__ __forceinline__ void exchange(const Real (&v)[K], Real &L, Real &R, Exch<Real, NW, WT> &x)
{
    exchange_ends(v[0], v[K - 1], L, R, x);
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

// Paired FP32 block steps for threads whose points and partners all lie
// inside one problem (no singletons, no walls): register j and register
// j + K/2 share one 64-bit register, a pair, and one fma.rn.f32x2 advances
// both points (two FP32 FMAs, each rounded as fmaf: the scalar step's bits
// with half the issue slots).  With K/2 even both halves of a pair have the
// same grouping parity, so a pair's partner is the neighbouring pair, except
// at the ends under grouping 1: pair 0 takes (L, v[K/2 - 1]) and pair
// K/2 - 1 takes (v[K/2], R).
template <int K>
__device__ __forceinline__ void to_pairs(const float (&v)[K], uint64_t (&p)[K / 2])
{
#pragma unroll
    for (int j = 0; j < K / 2; ++j)
        p[j] = f2(v[j], v[j + K / 2]);
}

template <int K>
__device__ __forceinline__ void from_pairs(const uint64_t (&p)[K / 2], float (&v)[K])
{
#pragma unroll
    for (int j = 0; j < K / 2; ++j) {
        const float2 t = f2_split(p[j]);
        v[j] = t.x;
        v[j + K / 2] = t.y;
    }
}

// x <- x + g x_partner on the pairs (g2 = (g, g)): the scaled mid stage.
template <int Q, int H>
__device__ __forceinline__ void pair_mid(uint64_t (&p)[H], float L, float R, uint64_t g2)
{
    static_assert(H % 2 == 0, "paired steps need an even number of pairs");
    uint64_t np[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        uint64_t q;
        if (((j + Q) & 1) == 0)
            q = (j + 1 < H) ? p[j + 1] : f2(f2_split(p[0]).y, R);
        else
            q = (j >= 1) ? p[j - 1] : f2(L, f2_split(p[H - 1]).x);
        np[j] = f2_fma(g2, q, p[j]);
    }
#pragma unroll
    for (int j = 0; j < H; ++j)
        p[j] = np[j];
}

// FP64 registers per thread whose scaled update runs on the integer pipes
// (emu_fma) instead of the FP64 unit, in the interior warps' block steps of
// the tiled and the batched FP64 kernels.
#ifndef GE_EMU_F64
#define GE_EMU_F64 7
#endif

// Register j is one of the E emulated ones of K, spread evenly: j is taken
// where floor(j E / K) steps up (E = 7 of K = 16: registers 2, 4, 6, 9, 11, 13, 15).
template <int K, int E>
__device__ __forceinline__ constexpr bool emu_reg(int j)
{
    return E > 0 && ((j + 1) * E) / K > (j * E) / K;
}

// The scaled mid stage x <- x + g x_partner in FP64 on a warp whose points
// and partners all lie inside the grid, E registers per thread on the
// integer pipes.  If any lane's emulated update leaves the fast path (or a
// lane passes usable = false), the warp recomputes its emulated registers on
// the FP64 unit, so the result is always the FP64 unit's fma, bit for bit.
template <int Q, int E, int K>
__device__ __forceinline__ void stage_mid_hybrid(double (&v)[K], double L, double R, double g, const EmuG &eg,
                                                 bool usable = true)
{
    double nv[K];
    bool ok = usable;
    // the cheaper, narrower form when every lane's emulated updates are
    // additions (the product and x of the same sign: a smooth field of one
    // sign); taken for g > 0 only, where that is sign(x_partner) == sign(x)
    uint32_t diff = eg.s << 31;
#pragma unroll
    for (int j = 0; j < K; ++j)
        if (emu_reg<K, E>(j))
            diff |= (uint32_t)__double2hiint(pval<Q>(v, j, L, R)) ^ (uint32_t)__double2hiint(v[j]);
    if (__any_sync(0xffffffffu, (diff >> 31) != 0u)) {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const double p = pval<Q>(v, j, L, R);
            if (emu_reg<K, E>(j)) {
                bool o;
                nv[j] = emu_fma(eg, p, v[j], o);
                ok = ok && o;
            } else {
                nv[j] = fma(g, p, v[j]);
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const double p = pval<Q>(v, j, L, R);
            if (emu_reg<K, E>(j)) {
                bool o;
                nv[j] = emu_fma_add(eg, p, v[j], o);
                ok = ok && o;
            } else {
                nv[j] = fma(g, p, v[j]);
            }
        }
    }
    if (!__all_sync(0xffffffffu, ok)) {
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (emu_reg<K, E>(j))
                nv[j] = fma(g, pval<Q>(v, j, L, R), v[j]);
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

// v[j] <- v[j] * 2^-e for the registers in [jlo, jhi) (all with ALL).  In
// double, a power-of-two scaling of a normal number whose result stays
// normal only lowers its exponent field: when every such value of the warp
// has an exponent field in (e, 2047), the scaling is an integer subtraction
// on the ALU pipe instead of a multiply on the FP64 pipe (the one DFMA per
// point and step is what bounds the FP64 kernels); the results are the same
// bits.  Otherwise (zeros, subnormal results, infinities) the multiply.
template <bool ALL, int K>
__device__ __forceinline__ void scale_pow2(double (&v)[K], int e, int jlo = 0, int jhi = K)
{
    const long long sh = (long long)e << 52;
    bool ok = true;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int ex = (int)((__double_as_longlong(v[j]) >> 52) & 0x7FF);
        if (ALL || (j >= jlo && j < jhi))
            ok = ok && ex > e && ex < 2047;
    }
    if (__all_sync(0xffffffffu, ok)) {
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (ALL || (j >= jlo && j < jhi))
                v[j] = __longlong_as_double(__double_as_longlong(v[j]) - sh);
    } else {
        const double s = pow2neg<double>(e);
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (ALL || (j >= jlo && j < jhi))
                v[j] *= s;
    }
}
template <bool ALL, int K>
__device__ __forceinline__ void scale_pow2(float (&v)[K], int e, int jlo = 0, int jhi = K)
{
    const float s = pow2neg<float>(e);
#pragma unroll
    for (int j = 0; j < K; ++j)
        if (ALL || (j >= jlo && j < jhi))
            v[j] *= s;
}

// Kahan sum of an update into (hi, lo).  The updates that reach it are
// explicitly rounded products (__fmul_rn), so the compiler can never fuse a
// product into the sum: every kernel instantiation and tile geometry then
// gives the same bits.
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
    float val = paired ? __fmul_rn(d, partner - self) : __fmul_rn(km1, self + lself);
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
                const float t = __fmul_rn(d, v[j + 1] - v[j]);
                kahan_add(v[j], lo[j], t);
                kahan_add(v[j + 1], lo[j + 1], -t);
            }
        } else {
            const float t0 = __fmul_rn(d, L - v[0]);
            const float tk = __fmul_rn(d, R - v[K - 1]);
#pragma unroll
            for (int j = 1; j + 1 < K; j += 2) {
                const float t = __fmul_rn(d, v[j + 1] - v[j]);
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

// Compensated block steps on register pairs (threads whose points and
// partners all lie inside one problem): the same deltas and Kahan sums as
// mid_comp, two points per packed instruction, the same bits.  A group's
// second member takes its update -t as lo - t (the number the scalar sum
// (-t) + lo gives).  Under grouping 1 the end pairs take their partners
// across the halves: pair 0 = (v[0], v[K/2]) pairs with (L, v[K/2 - 1]),
// pair K/2 - 1 = (v[K/2 - 1], v[K - 1]) with (v[K/2], R); the group
// (K/2 - 1, K/2) so gets d (v[K/2] - v[K/2 - 1]) on one side and its exact
// negative on the other, as in the scalar step.
__device__ __forceinline__ void kahan2(uint64_t &hi, uint64_t &lo, uint64_t delta)
{
    const uint64_t y = f2_add(delta, lo);
    const uint64_t s = f2_add(hi, y);
    lo = f2_sub(y, f2_sub(s, hi));
    hi = s;
}
__device__ __forceinline__ void kahan2_neg(uint64_t &hi, uint64_t &lo, uint64_t t)
{
    const uint64_t y = f2_sub(lo, t);
    const uint64_t s = f2_add(hi, y);
    lo = f2_sub(y, f2_sub(s, hi));
    hi = s;
}

template <int Q, int H, int NW, bool WT>
__device__ __forceinline__ void pair_mid_comp(uint64_t (&p)[H], uint64_t (&lo)[H], uint64_t d2, uint64_t nz,
                                              Exch<float, NW, WT> &x)
{
    static_assert(H % 2 == 0, "paired steps need an even number of pairs");
    if (Q == 0) {
#pragma unroll
        for (int j = 0; j < H; j += 2) {
            const uint64_t t = f2_mul_alone(d2, f2_sub(p[j + 1], p[j]), nz);
            kahan2(p[j], lo[j], t);
            kahan2_neg(p[j + 1], lo[j + 1], t);
        }
    } else {
        const float2 a = f2_split(p[0]), b = f2_split(p[H - 1]);
        float L = 0.0f, R = 0.0f;
        exchange_ends(a.x, b.y, L, R, x);
        const uint64_t t0 = f2_mul_alone(d2, f2_sub(f2(L, b.x), p[0]), nz);
        const uint64_t tk = f2_mul_alone(d2, f2_sub(f2(a.y, R), p[H - 1]), nz);
#pragma unroll
        for (int j = 1; j + 1 < H; j += 2) {
            const uint64_t t = f2_mul_alone(d2, f2_sub(p[j + 1], p[j]), nz);
            kahan2(p[j], lo[j], t);
            kahan2_neg(p[j + 1], lo[j + 1], t);
        }
        kahan2(p[0], lo[0], t0);
        kahan2(p[H - 1], lo[H - 1], tk);
    }
}

// n_mid compensated block steps from grouping parity p_first, the
// compensation word folded in at the end (v += lo), on pairs.
template <int K, int NW, bool WT>
__device__ __forceinline__ void comp_steps_pairs(float (&v)[K], int p_first, int n_mid, float d,
                                                 Exch<float, NW, WT> &x)
{
    constexpr int H = K / 2;
    uint64_t p[H], lo[H];
    to_pairs(v, p);
#pragma unroll
    for (int j = 0; j < H; ++j)
        lo[j] = f2(0.0f, 0.0f);
    const uint64_t d2 = f2(d, d), nz = f2_neg_zero(d);  // d = 2r / (1 + 2r) >= 0
    int m = 0;
    if (n_mid > 0 && (p_first & 1)) {
        pair_mid_comp<1>(p, lo, d2, nz, x);
        m = 1;
    }
    for (; m + 1 < n_mid; m += 2) {
        pair_mid_comp<0>(p, lo, d2, nz, x);
        pair_mid_comp<1>(p, lo, d2, nz, x);
    }
    if (m < n_mid)
        pair_mid_comp<0>(p, lo, d2, nz, x);
#pragma unroll
    for (int j = 0; j < H; ++j)
        p[j] = f2_add(p[j], lo[j]);
    from_pairs(p, v);
}

}  // namespace
}  // namespace ge
