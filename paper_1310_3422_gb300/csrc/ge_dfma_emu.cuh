// ge_dfma_emu.cuh -- the FP64 multiply-add x + g p on the 32-bit integer
// pipes, exact (the IEEE 754 round-to-nearest-even result, the bits the FP64
// unit's fma gives), for the common case; the caller falls back to the FP64
// unit for everything else.
//
// Why: a GB300 SM issues about two FP64 FMAs per clock but 128 integer or
// FP32 lane-operations; the tiled FP64 kernel is bound by the FP64 unit.
// Moving a fraction of a thread's updates to the integer pipes lets both run
// at once.  Written from the IEEE 754 definition of fusedMultiplyAdd (exact
// product, exact sum, one rounding), not from any library's code.
//
// The fast path (ok == true) takes normal nonzero p and x, g normal (a
// launch constant), with x's lowest bit 0 .. 74 bit positions above the
// product's lowest bit (x within about 2^-53 .. 2^21 of |g p|: the sum of a
// smooth field and its scaled neighbour lies well inside), a sum whose
// leading bit is at position 96 or above of the 128-bit frame (no deep
// cancellation) and a normal result.  In that range the whole computation is
// exact integer arithmetic:
//   - the 106-bit product of the two 53-bit significands, as four 32-bit
//     limbs (IMAD.WIDE partial products);
//   - x's significand shifted to its place in the same 128-bit frame (no bit
//     of it is lost), added or subtracted in two's complement, then made
//     positive;
//   - the top 53 bits below the leading one, rounded to nearest-even from the
//     next bit and the OR of all bits below it;
//   - the exponent from the product's and the leading bit's positions, packed
//     so that a carry out of the rounding moves into the exponent field.
// Anything else (zeros, subnormals, infinities, NaNs, far-apart magnitudes,
// results that cancel below bit 96 or leave the normal range) clears ok.
#pragma once

#include <cstdint>

namespace ge {

// g split once per launch: significand limbs, biased exponent, sign.
struct EmuG {
    uint32_t gh, gl;
    int eb;
    uint32_t s;
};

__device__ __forceinline__ EmuG emu_g(double g)
{
    const uint32_t hi = (uint32_t)__double2hiint(g), lo = (uint32_t)__double2loint(g);
    return EmuG{(hi & 0xfffffu) | 0x100000u, lo, (int)((hi >> 20) & 0x7ff), hi >> 31};
}

// g must be normal and nonzero for the fast path.
__device__ __forceinline__ bool emu_g_usable(const EmuG &g) { return (unsigned)(g.eb - 1) < 0x7feu; }

// The result's bits from its sign s, the biased exponent eb of its leading
// bit, the 53-bit significand (mhi:mlo, leading 1 at bit 52) and the
// rounding increment up.  The exponent field goes in as eb - 1 and the
// significand's leading 1 adds the missing one; a carry out of the rounded
// significand (all ones + 1 = 2^53) moves into the exponent field by itself
// and leaves a zero fraction, so rounding needs no separate renormalisation.
// ok stays set for eb in [1, 2045] (normal even after such a carry).
__device__ __forceinline__ double emu_pack(uint32_t s, int eb, uint32_t mhi, uint32_t mlo, uint32_t up, bool &ok)
{
    ok = ok & ((unsigned)(eb - 1) < 0x7fdu);
    uint32_t lo, hi;
    asm("add.cc.u32 %0, %2, %3;\n\t"
        "addc.u32 %1, %4, %5;"
        : "=r"(lo), "=r"(hi)
        : "r"(mlo), "r"(up), "r"(mhi), "r"((s << 31) + ((uint32_t)(eb - 1) << 20)));
    return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ double emu_fma(const EmuG &g, double p, double x, bool &ok)
{
    const uint32_t Ph = (uint32_t)__double2hiint(p), Pl = (uint32_t)__double2loint(p);
    const uint32_t Xh = (uint32_t)__double2hiint(x), Xl = (uint32_t)__double2loint(x);
    const int ep = (int)((Ph >> 20) & 0x7ff), ex = (int)((Xh >> 20) & 0x7ff);
    const uint32_t ph = (Ph & 0xfffffu) | 0x100000u, xh = (Xh & 0xfffffu) | 0x100000u;
    // the product's significand M = mg * mp in [2^104, 2^106), four limbs
    const uint64_t t = (uint64_t)g.gl * Pl;
    const uint64_t t2 = (uint64_t)g.gh * Pl + (t >> 32);
    const uint64_t t3 = (uint64_t)g.gl * ph + (uint32_t)t2;
    const uint64_t t4 = (uint64_t)g.gh * ph + (t2 >> 32) + (t3 >> 32);
    const uint32_t m0 = (uint32_t)t, m1 = (uint32_t)t3, m2 = (uint32_t)t4, m3 = (uint32_t)(t4 >> 32);
    // x's significand at bit D of the product's frame (M's lowest bit is
    // worth 2^(e_g + e_p - 2150), x's 2^(e_x - 1075))
    const int D = ex - g.eb - ep + 1075;
    ok = ((unsigned)(ep - 1) < 0x7feu) & ((unsigned)(ex - 1) < 0x7feu) & ((unsigned)D <= 74u);
    const uint32_t b = (uint32_t)D & 31u, q = (uint32_t)D >> 5;
    const uint32_t v0 = Xl << b, v1 = __funnelshift_l(Xl, xh, b), v2 = b ? (xh >> (32u - b)) : 0u;
    uint32_t x0 = q == 0 ? v0 : 0u;
    uint32_t x1 = q == 0 ? v1 : (q == 1 ? v0 : 0u);
    uint32_t x2 = q == 0 ? v2 : (q == 1 ? v1 : v0);
    uint32_t x3 = q == 0 ? 0u : (q == 1 ? v2 : v1);
    // R = M + X, or M - X when the signs differ (two's complement), then |R|
    const uint32_t sprod = (Ph >> 31) ^ g.s, sub = sprod ^ (Xh >> 31), inv = 0u - sub;
    x0 ^= inv;
    x1 ^= inv;
    x2 ^= inv;
    x3 ^= inv;
    uint32_t r0, r1, r2, r3;
    asm("add.cc.u32 %0, %4, %8;\n\t"
        "addc.cc.u32 %1, %5, %9;\n\t"
        "addc.cc.u32 %2, %6, %10;\n\t"
        "addc.u32 %3, %7, %11;"
        : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
        : "r"(m0), "r"(m1), "r"(m2), "r"(m3), "r"(x0), "r"(x1), "r"(x2), "r"(x3));
    asm("add.cc.u32 %0, %0, %4;\n\t"
        "addc.cc.u32 %1, %1, 0;\n\t"
        "addc.cc.u32 %2, %2, 0;\n\t"
        "addc.u32 %3, %3, 0;"
        : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3)
        : "r"(sub));
    const uint32_t neg = 0u - (r3 >> 31);
    r0 ^= neg;
    r1 ^= neg;
    r2 ^= neg;
    r3 ^= neg;
    asm("add.cc.u32 %0, %0, %4;\n\t"
        "addc.cc.u32 %1, %1, 0;\n\t"
        "addc.cc.u32 %2, %2, 0;\n\t"
        "addc.u32 %3, %3, 0;"
        : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3)
        : "r"(neg & 1u));
    const uint32_t s = sprod ^ (neg & 1u);
    ok = ok & (r3 != 0u);
    const int L = 127 - __clz((int)r3);  // the leading bit, 96 .. 126
    // significand = bits L-52 .. L, from the window (r3:r2:r1) >> (L - 84)
    const int sh = L - 84;
    uint32_t mlo, mhi;
    if (sh < 32) {
        mlo = __funnelshift_r(r1, r2, (uint32_t)sh);
        mhi = __funnelshift_r(r2, r3, (uint32_t)sh);
    } else {
        mlo = __funnelshift_r(r2, r3, (uint32_t)(sh - 32));
        mhi = r3 >> (sh - 32);
    }
    // the rounding bit L-53 and the OR of every bit below it
    const int rb = L - 53;
    uint32_t guard, sticky;
    if (rb < 64) {
        const uint32_t k = (uint32_t)(rb - 32);
        guard = (r1 >> k) & 1u;
        sticky = r0 | (r1 & ((1u << k) - 1u));
    } else {
        const uint32_t k = (uint32_t)(rb - 64);
        guard = (r2 >> k) & 1u;
        sticky = r0 | r1 | (r2 & ((1u << k) - 1u));
    }
    const uint32_t up = guard & ((sticky != 0u) | (mlo & 1u));
    return emu_pack(s, g.eb + ep + L - 1127, mhi, mlo, up, ok);
}

// The addition-only form for the common case, narrower still: the product
// and x of the same sign (the caller checked) and x's lowest bit 32 .. 62
// positions above the product's (x between about 2^-21 and 2^9 of g p, where
// a smooth field and its scaled neighbour sit).  Then x's significand fills
// limbs 1 .. 3 with one shift amount and no selects, limb 0 of the sum is the
// product's, the leading bit lies in 104 .. 115, so the significand window and
// the rounding bit need no branch.  ok = false outside that range.
__device__ __forceinline__ double emu_fma_add(const EmuG &g, double p, double x, bool &ok)
{
    const uint32_t Ph = (uint32_t)__double2hiint(p), Pl = (uint32_t)__double2loint(p);
    const uint32_t Xh = (uint32_t)__double2hiint(x), Xl = (uint32_t)__double2loint(x);
    const int ep = (int)((Ph >> 20) & 0x7ff), ex = (int)((Xh >> 20) & 0x7ff);
    const uint32_t ph = (Ph & 0xfffffu) | 0x100000u, xh = (Xh & 0xfffffu) | 0x100000u;
    const uint64_t t = (uint64_t)g.gl * Pl;
    const uint64_t t2 = (uint64_t)g.gh * Pl + (t >> 32);
    const uint64_t t3 = (uint64_t)g.gl * ph + (uint32_t)t2;
    const uint64_t t4 = (uint64_t)g.gh * ph + (t2 >> 32) + (t3 >> 32);
    const uint32_t r0 = (uint32_t)t, m1 = (uint32_t)t3, m2 = (uint32_t)t4, m3 = (uint32_t)(t4 >> 32);
    const int D = ex - g.eb - ep + 1075;
    ok = ((unsigned)(ep - 1) < 0x7feu) & ((unsigned)(ex - 1) < 0x7feu) & ((unsigned)(D - 32) <= 30u);
    const uint32_t b = (uint32_t)(D - 32) & 31u;
    // x's significand << D: limbs 1, 2, 3 (limb 0 is zero)
    const uint32_t x1 = Xl << b, x2 = __funnelshift_l(Xl, xh, b), x3 = __funnelshift_l(xh, 0u, b);
    uint32_t r1, r2, r3;
    asm("add.cc.u32 %0, %3, %6;\n\t"
        "addc.cc.u32 %1, %4, %7;\n\t"
        "addc.u32 %2, %5, %8;"
        : "=r"(r1), "=r"(r2), "=r"(r3)
        : "r"(m1), "r"(m2), "r"(m3), "r"(x1), "r"(x2), "r"(x3));
    const int L = 127 - __clz((int)r3);  // 104 .. 115 in range
    const uint32_t sh = (uint32_t)(L - 84) & 31u;
    const uint32_t mlo = __funnelshift_r(r1, r2, sh), mhi = __funnelshift_r(r2, r3, sh);
    const uint32_t k = (uint32_t)(L - 85) & 31u;  // the rounding bit L - 53 sits in limb 1
    const uint32_t guard = (r1 >> k) & 1u, sticky = r0 | (r1 & ((1u << k) - 1u));
    const uint32_t up = guard & ((sticky != 0u) | (mlo & 1u));
    return emu_pack((Ph >> 31) ^ g.s, g.eb + ep + L - 1127, mhi, mlo, up, ok);
}

}  // namespace ge
