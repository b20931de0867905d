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
// x <- x + 2r x_partner; the scale sigma = (1+2r)^m is a scalar, brought back
// by exact powers of two and folded into the exit).  Entry and exit:
//     w = (1-r) u_i + r u_partner(1-p) [+ r beta at the walls],
//     u = ((1+r) w_i + r w_partner(p)) / (1+2r)   (singleton: w_i/(1+r)).
// This is the same linear map as the step-by-step scheme, reassociated.
//
// Layout.  A tile is kTileThreads rows of 128 bytes (8192 floats or 4096
// doubles); thread t owns row t in registers, so parity-0 groups never cross
// threads and parity-1 groups cross one thread boundary (warp shuffles, and a
// shared-memory slot between warps, one CTA barrier per parity-1 step).  The
// tile is the tile's output range plus a halo of H >= (steps in the launch
// + 1) points per side: after the launch's steps, the corrupted margin (the
// dependency cone grows one point per step) is still inside the halo.  The
// tile is loaded by a 2D TMA copy (cp.async.bulk.tensor, 128-byte swizzle so
// each thread's row read is bank-conflict free) into one of two shared
// buffers while the previous tile is computed; results go back through the
// same buffer and leave with coalesced 16-byte stores.
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

// 16-byte chunk c of a thread's register row <-> shared memory.
template <typename Real, int K>
__device__ __forceinline__ void chunk_to_regs(const unsigned char *p, Real (&v)[K], int c);
template <>
__device__ __forceinline__ void chunk_to_regs<float, 32>(const unsigned char *p, float (&v)[32], int c)
{
    const float4 q = *reinterpret_cast<const float4 *>(p);
    v[4 * c + 0] = q.x;
    v[4 * c + 1] = q.y;
    v[4 * c + 2] = q.z;
    v[4 * c + 3] = q.w;
}
template <>
__device__ __forceinline__ void chunk_to_regs<double, 16>(const unsigned char *p, double (&v)[16], int c)
{
    const double2 q = *reinterpret_cast<const double2 *>(p);
    v[2 * c + 0] = q.x;
    v[2 * c + 1] = q.y;
}
template <typename Real, int K>
__device__ __forceinline__ void regs_to_chunk(unsigned char *p, const Real (&v)[K], int c);
template <>
__device__ __forceinline__ void regs_to_chunk<float, 32>(unsigned char *p, const float (&v)[32], int c)
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
}
template <>
__device__ __forceinline__ void regs_to_chunk<double, 16>(unsigned char *p, const double (&v)[16], int c)
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

template <int Q>
__device__ __forceinline__ long long partner_of(long long gi, int j)
{
    return (((j + Q) & 1) == 0) ? gi + 1 : gi - 1;
}

// Neighbour values across thread boundaries for a parity-1 grouping.
template <typename Real, int K, int NW>
__device__ __forceinline__ void exchange(const Real (&v)[K], Real &L, Real &R, Real (*edge)[NW][2],
                                         int &eb, int lane, int warp)
{
    L = __shfl_up_sync(0xffffffffu, v[K - 1], 1);
    R = __shfl_down_sync(0xffffffffu, v[0], 1);
    if (lane == 0)
        edge[eb][warp][0] = v[0];
    if (lane == 31)
        edge[eb][warp][1] = v[K - 1];
    __syncthreads();
    if (lane == 0 && warp > 0)
        L = edge[eb][warp - 1][1];
    if (lane == 31 && warp < NW - 1)
        R = edge[eb][warp + 1][0];
    eb ^= 1;
}

enum StageKind { kEntry = 0, kMid = 1, kExit = 2 };

template <typename Real>
struct StageC {
    Real a, b, s, fl, fr;
};

// One stage on a thread's K registers (scaled form).
//   entry: v <- (1-r) v + r v_p          (a = r, b = 1-r; singleton: b v)
//   mid:   v <- v + 2r v_p               (a = 2r;         singleton: s v)
//   exit:  v <- x1 v + x2 v_p            (a = x1, b = x2; singleton: s v)
// Entry and mid add the wall terms fl / fr at points 0 and n-1.  Points
// outside [0, n) keep their value.  `edge` is false when every point of the
// thread and every partner is inside the grid and none is at a wall.
template <int Q, int KIND, int K, typename Real>
__device__ __forceinline__ void stage(Real (&v)[K], Real L, Real R, bool edge, long long g0, long long n,
                                      const StageC<Real> &c)
{
    Real nv[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const Real p = pval<Q>(v, j, L, R);
        if (KIND == kEntry)
            nv[j] = fma(c.a, p, c.b * v[j]);
        else if (KIND == kMid)
            nv[j] = fma(c.a, p, v[j]);
        else
            nv[j] = fma(c.a, v[j], c.b * p);
    }
    if (edge) {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const long long gi = g0 + j;
            const long long pg = partner_of<Q>(gi, j);
            const bool inside = (gi >= 0) && (gi < n);
            const bool paired = (pg >= 0) && (pg < n);
            Real val;
            if (KIND == kEntry)
                val = paired ? nv[j] : c.b * v[j];
            else
                val = paired ? nv[j] : c.s * v[j];
            if (KIND != kExit) {
                if (gi == 0)
                    val += c.fl;
                if (gi == n - 1)
                    val += c.fr;
            }
            nv[j] = inside ? val : v[j];
        }
    }
#pragma unroll
    for (int j = 0; j < K; ++j)
        v[j] = nv[j];
}

// Compensated block step (normalised form, Kahan sum of each point's update).
template <int Q, int K>
__device__ __forceinline__ void mid_comp(float (&v)[K], float (&lo)[K], float L, float R, bool edge,
                                         long long g0, long long n, float d, float kappa_m1, float fl,
                                         float fr)
{
    float dl[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const float p = pval<Q>(v, j, L, R);
        dl[j] = d * (p - v[j]);
    }
    if (edge) {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const long long gi = g0 + j;
            const long long pg = partner_of<Q>(gi, j);
            const bool inside = (gi >= 0) && (gi < n);
            const bool paired = (pg >= 0) && (pg < n);
            float val = paired ? dl[j] : kappa_m1 * (v[j] + lo[j]);
            if (gi == 0)
                val += fl;
            if (gi == n - 1)
                val += fr;
            dl[j] = inside ? val : 0.0f;
        }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const float y = dl[j] + lo[j];
        const float s = v[j] + y;
        lo[j] = y - (s - v[j]);
        v[j] = s;
    }
}

template <typename Real, bool COMP>
__global__ void __launch_bounds__(kTileThreads, 2)
    tb_kernel(const __grid_constant__ CUtensorMap tmap, const TbParams P)
{
    constexpr int NT = kTileThreads;
    constexpr int K = kRowBytes / (int)sizeof(Real);
    constexpr int NW = NT / 32;
    constexpr int CH = kRowBytes / 16;
    constexpr uint32_t kTileBytes = NT * kRowBytes;

    extern __shared__ unsigned char smem_raw[];
    unsigned char *tiles = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ Real edge[2][NW][2];

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int hr = P.H / K;  // halo rows
    const int ur = P.U / K;  // output rows

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
    int eb = 0;
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
        {
            const unsigned char *row = cur + t * kRowBytes;
#pragma unroll
            for (int c = 0; c < CH; ++c)
                chunk_to_regs<Real, K>(row + ((c ^ (t & 7)) << 4), v, c);
        }
        const long long g0 = tile * P.U - P.H + (long long)t * K;
        const bool edge_thr = !(g0 >= 1 && g0 + K <= P.n - 1);
        Real L = 0, R = 0;

        if constexpr (!COMP) {
            double sigma = 1.0;
            int until_rescale = P.rescale_every;
            if (P.do_entry) {
                StageC<Real> c{(Real)P.r, (Real)P.omr, (Real)0, (Real)P.f_l, (Real)P.f_r};
                if (((1 - P.p_first) & 1) == 1) {
                    exchange<Real, K, NW>(v, L, R, edge, eb, lane, warp);
                    stage<1, kEntry>(v, L, R, edge_thr, g0, P.n, c);
                } else {
                    stage<0, kEntry>(v, L, R, edge_thr, g0, P.n, c);
                }
            }
            for (int m = 0; m < P.n_mid; ++m) {
                sigma *= (1.0 + P.g);
                StageC<Real> c{(Real)P.g, (Real)0, (Real)P.kappa, (Real)(sigma * P.f_l),
                               (Real)(sigma * P.f_r)};
                if (((P.p_first + m) & 1) == 1) {
                    exchange<Real, K, NW>(v, L, R, edge, eb, lane, warp);
                    stage<1, kMid>(v, L, R, edge_thr, g0, P.n, c);
                } else {
                    stage<0, kMid>(v, L, R, edge_thr, g0, P.n, c);
                }
                if (until_rescale > 0 && --until_rescale == 0) {
                    until_rescale = P.rescale_every;
                    int e;
                    frexp(sigma, &e);
                    const double s = ldexp(1.0, 1 - e);  // sigma * s in [1, 2)
                    sigma *= s;
#pragma unroll
                    for (int j = 0; j < K; ++j)
                        v[j] *= (Real)s;
                }
            }
            const double inv = 1.0 / sigma;
            if (P.do_exit) {
                StageC<Real> c{(Real)(P.x1 * inv), (Real)(P.x2 * inv), (Real)(P.xs * inv), (Real)0,
                               (Real)0};
                if (((P.p_first + P.n_mid) & 1) == 1) {
                    exchange<Real, K, NW>(v, L, R, edge, eb, lane, warp);
                    stage<1, kExit>(v, L, R, edge_thr, g0, P.n, c);
                } else {
                    stage<0, kExit>(v, L, R, edge_thr, g0, P.n, c);
                }
            } else if (sigma != 1.0) {
#pragma unroll
                for (int j = 0; j < K; ++j)
                    v[j] *= (Real)inv;
            }
        } else {
            float lo[K];
#pragma unroll
            for (int j = 0; j < K; ++j)
                lo[j] = 0.0f;
            if (P.do_entry) {
                StageC<Real> c{(Real)P.r, (Real)P.omr, (Real)0, (Real)P.f_l, (Real)P.f_r};
                if (((1 - P.p_first) & 1) == 1) {
                    exchange<Real, K, NW>(v, L, R, edge, eb, lane, warp);
                    stage<1, kEntry>(v, L, R, edge_thr, g0, P.n, c);
                } else {
                    stage<0, kEntry>(v, L, R, edge_thr, g0, P.n, c);
                }
            }
            const float d = (float)P.d, km1 = (float)(P.kappa - 1.0);
            const float fl = (float)P.f_l, fr = (float)P.f_r;
            for (int m = 0; m < P.n_mid; ++m) {
                if (((P.p_first + m) & 1) == 1) {
                    exchange<Real, K, NW>(v, L, R, edge, eb, lane, warp);
                    mid_comp<1, K>(v, lo, L, R, edge_thr, g0, P.n, d, km1, fl, fr);
                } else {
                    mid_comp<0, K>(v, lo, L, R, edge_thr, g0, P.n, d, km1, fl, fr);
                }
            }
            if (P.do_exit) {
                // u = x1 (hi + lo) + x2 hi_partner; singleton: xs (hi + lo)
                StageC<Real> c{(Real)P.x1, (Real)P.x2, (Real)P.xs, (Real)0, (Real)0};
                const int q = (P.p_first + P.n_mid) & 1;
                if (q == 1) {
                    exchange<Real, K, NW>(v, L, R, edge, eb, lane, warp);
                    stage<1, kExit>(v, L, R, edge_thr, g0, P.n, c);
                } else {
                    stage<0, kExit>(v, L, R, edge_thr, g0, P.n, c);
                }
                const float x1 = (float)P.x1, xs = (float)P.xs;
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    float w = x1;
                    if (edge_thr) {
                        const long long gi = g0 + j;
                        const long long pg = (((j + q) & 1) == 0) ? gi + 1 : gi - 1;
                        const bool inside = (gi >= 0) && (gi < P.n);
                        const bool paired = (pg >= 0) && (pg < P.n);
                        w = inside ? (paired ? x1 : xs) : 0.0f;
                    }
                    v[j] = fmaf(w, lo[j], v[j]);
                }
            } else {
#pragma unroll
                for (int j = 0; j < K; ++j)
                    v[j] += lo[j];
            }
        }

        // write back (own row), then coalesced copy of the output rows
        {
            unsigned char *row = cur + t * kRowBytes;
#pragma unroll
            for (int c = 0; c < CH; ++c)
                regs_to_chunk<Real, K>(row + ((c ^ (t & 7)) << 4), v, c);
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
    tb_kernel<Real, COMP><<<grid, kTileThreads, tb_smem_bytes(), s>>>(*m, p);
    return cudaGetLastError();
}

template <typename Real, bool COMP>
cudaError_t set_attr_and_occupancy(int *blocks)
{
    cudaError_t e = cudaFuncSetAttribute(tb_kernel<Real, COMP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, tb_smem_bytes());
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, tb_kernel<Real, COMP>, kTileThreads,
                                                         tb_smem_bytes());
}

}  // namespace

int tb_smem_bytes() { return 2 * kTileThreads * kRowBytes + 1024; }

cudaError_t tb_occupancy(int prec, int *blocks)
{
    if (prec == 0)
        return set_attr_and_occupancy<double, false>(blocks);
    if (prec == 1)
        return set_attr_and_occupancy<float, false>(blocks);
    return set_attr_and_occupancy<float, true>(blocks);
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
