// ge_tb_df.cu -- the tiled GE kernel for FP64 contexts evaluated on the FP32
// pipes in double-float arithmetic (GE_KERNEL_TEMPORAL_DF).
//
// Same scheme, tile and CTA-row layout as the FP64 tiled kernel (ge_tb.cu):
// the kernel carries the right-hand side w of each step's group systems in
// scaled form, one block step being x <- x + g x_partner (g = 2r, Sec. 2's
// 2x2 solve reassociated), with the scale sigma kept by the host and brought
// back by exact powers of two.  Here every value is an unevaluated sum
// hi + lo of two floats, about 48 significant bits (Dekker's double-length
// arithmetic, 1971), and one step is evaluated with error-free
// transformations: the product g * x_partner exactly by one FMA (TwoProd),
// the sum of the high parts exactly by Knuth's TwoSum, the low parts added
// in FP32, and the pair renormalised by Fast2Sum.  That is 15 FP32
// operations per point and step where the FP64 kernel needs one DFMA; an SM
// issues 128 FP32 operations per clock and only 2 FP64 FMAs.
//
// Storage and range.  The context's buffers hold doubles between calls.  A
// call starts with a reduction that finds the power of two 2^e0 just above
// the largest |u| and wall value (df_exponent_kernel); its first launch
// loads doubles and splits u * 2^-e0 into (hi, lo), so any double data fit
// the float exponent range; later launches of the call keep (hi, lo) pairs
// in the buffers (8 bytes per point, like a double); the last launch joins
// each pair back into a double and multiplies by 2^e0.  Both conversions
// are exact up to the 48-bit rounding of the split.
#include <cuda.h>
#include <cstdint>

#include "ge_internal.h"
#include "ge_df.cuh"
#include "ge_tb_dev.cuh"

namespace ge {
namespace {



// Prescale code of the data (see kDfCodeBias): the largest over the values
// and walls_code, raised into *code by atomicMax.
__global__ void df_exponent_kernel(const double *__restrict__ u, long long n, int walls_code, int *code)
{
    int best = walls_code;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double x = u[i];
        if (x != 0.0) {
            const int c = df_exponent_bound(x) + kDfCodeBias;
            best = c > best ? c : best;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int other = __shfl_xor_sync(0xffffffffu, best, o);
        best = other > best ? other : best;
    }
    if ((threadIdx.x & 31) == 0 && best > 0)
        atomicMax(code, best);
}


__device__ __forceinline__ DfC dfc(const TbParams &P, int i) { return DfC{P.dfc[i][0], P.dfc[i][1]}; }

// Block steps m0 .. m0+count-1 (step m has grouping parity (p_first + m) & 1).
// The checked path carries the scale sigma in double for its wall terms.
// One block step of grouping Q; the checked path updates sigma and forms
// the scaled wall terms.
template <int Q, bool EDGE, bool GL, bool NORM>
__device__ __forceinline__ void df_mid_step(float (&h)[kDfK], float (&l)[kDfK], const TbParams &P, DfExch &x,
                                            Span sp, DfC g, DfC kap, double &sig, double fls, double frs)
{
    if constexpr (EDGE) {
        const DfC zero{0.0f, 0.0f};
        sig *= P.onepg;
        DfC fl, fr;
        df_split(sig * fls, fl.h, fl.l);
        df_split(sig * frs, fr.h, fr.l);
        df_stage_checked<Q, true, true, GL>(h, l, zero, g, kap, fl, fr, sp, x);
    } else {
        df_mid_fast<Q, GL, NORM>(h, l, g, x);
    }
}

// Block steps m0 .. m0+count-1, step m having grouping parity
// (p_first + m) & 1: an odd first step alone, then (even, odd) pairs (with
// g_lo = 0 the even one not renormalised), then an even trailing step.
template <bool EDGE, bool GL>
__device__ __forceinline__ void df_mid_run(float (&h)[kDfK], float (&l)[kDfK], int m0, int count, const TbParams &P,
                                           DfExch &x, Span sp, DfC g, DfC kap, double &sig, double fls, double frs)
{
    int m = m0;
    const int end = m0 + count;
    if (m < end && ((P.p_first + m) & 1)) {
        df_mid_step<1, EDGE, GL, true>(h, l, P, x, sp, g, kap, sig, fls, frs);
        ++m;
    }
    for (; m + 1 < end; m += 2) {
        df_mid_step<0, EDGE, GL, GL>(h, l, P, x, sp, g, kap, sig, fls, frs);
        df_mid_step<1, EDGE, GL, true>(h, l, P, x, sp, g, kap, sig, fls, frs);
    }
    if (m < end)
        df_mid_step<0, EDGE, GL, true>(h, l, P, x, sp, g, kap, sig, fls, frs);
}

// Entry, the launch's block steps (in runs between rescalings) and exit on
// one tile.  e0: the call's prescale exponent (walls scaled by 2^-e0 like
// the data).  GL: g = 2r has a nonzero low part.
template <bool EDGE, bool GL>
__device__ __forceinline__ void df_run(float (&h)[kDfK], float (&l)[kDfK], const TbParams &P, DfExch &x, Span sp,
                                       int e0)
{
    const DfC zero{0.0f, 0.0f};
    const DfC g = dfc(P, 0), kap = dfc(P, 1), rr = dfc(P, 2), omr = dfc(P, 3);
    double fls = 0.0, frs = 0.0;
    if constexpr (EDGE) {
        fls = ldexp(P.f_l, -e0);
        frs = ldexp(P.f_r, -e0);
    }
    if (P.do_entry) {
        // w = (1-r) u + r u_partner (singleton (1-r) u) plus the wall terms
        DfC fl = zero, fr = zero;
        if constexpr (EDGE) {
            df_split(fls, fl.h, fl.l);
            df_split(frs, fr.h, fr.l);
        }
        if (((1 - P.p_first) & 1) == 1)
            df_stage_checked<1, false, true>(h, l, omr, rr, omr, fl, fr, sp, x);
        else
            df_stage_checked<0, false, true>(h, l, omr, rr, omr, fl, fr, sp, x);
    }
    double sig = P.sigma_in;  // used on the checked path only
    int until = P.rescale_phase, ev = 0, m = 0;
    while (m < P.n_mid) {
        int count = P.n_mid - m;
        if (until > 0 && until < count)
            count = until;
        df_mid_run<EDGE, GL>(h, l, m, count, P, x, sp, g, kap, sig, fls, frs);
        m += count;
        if (until > 0) {
            until -= count;
            if (until == 0) {
                until = P.rescale_every;
                const int e = P.rs_exp[ev++];
                const float s = pow2neg<float>(e);
#pragma unroll
                for (int j = 0; j < kDfK; ++j) {
                    h[j] *= s;
                    l[j] *= s;
                }
                if constexpr (EDGE)
                    sig *= pow2neg<double>(e);
            }
        }
    }
    if (P.do_exit) {
        // u = x1 w + x2 w_partner (singleton xs w), x1, x2, xs divided by the
        // final scale
        const DfC x1 = dfc(P, 4), x2 = dfc(P, 5), xs = dfc(P, 6);
        if (((P.p_first + P.n_mid) & 1) == 1)
            df_stage_checked<1, false, false>(h, l, x1, x2, xs, zero, zero, sp, x);
        else
            df_stage_checked<0, false, false>(h, l, x1, x2, xs, zero, zero, sp, x);
    }
}

// GL: the pair of g = 2r has a nonzero low part (one kernel per form keeps
// each kernel's unrolled step loop small).
template <bool GL>
__global__ void __launch_bounds__(kDfNT, GE_TB_MINBLOCKS_DF)
    tb_df_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ TbParams P)
{
    constexpr int K = kDfK;
    constexpr int CH = kRowBytes / 16;  // 16-byte chunks per row: two points each
    constexpr uint32_t kTileBytes = kTileRows * kRowBytes;

    extern __shared__ unsigned char smem_raw[];
    unsigned char *tiles = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    __shared__ __align__(8) uint64_t mbar[3];  // two tile buffers, and one nothing arrives on
    __shared__ float2 slot[2][kDfNW][2];

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int hr = P.H / K;  // halo rows of the tile
    const int ur = P.U / K;  // output rows of the tile
    DfExch x{slot, 0, lane, warp};
    const int code = *P.df_code;
    const int e0 = code ? code - kDfCodeBias : 0;

    if (t == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_init(&mbar[2], 1);
        fence_mbar_init();
        // the next launch's tile queue starts empty (it runs after this one)
        if (blockIdx.x == 0 && P.tile_ctr_next)
            *P.tile_ctr_next = 0;
    }
    __syncthreads();

    // tiles come from the launch's dynamic queue (queue_tile): thread 0
    // takes the next position while the current tile is computed
    __shared__ long long s_next;
    long long k = blockIdx.x;
    if (t == 0 && k < P.n_tiles) {
        mbar_arrive_expect_tx(&mbar[0], kTileBytes);
        tma_load_rows(tiles, &tmap, &mbar[0], (int)(queue_tile(k, P.n_tiles) * ur - hr));
    }
    for (long long it = 0; k < P.n_tiles; ++it) {
        const int b = (int)(it & 1);
        unsigned char *cur = tiles + b * kTileBytes;
        const long long tile = queue_tile(k, P.n_tiles);
        bool prefetch = false;
        if (t == 0) {
            const long long nk = (long long)gridDim.x + atomicAdd(P.tile_ctr, 1);
            s_next = nk;
            prefetch = nk < P.n_tiles;
            if (prefetch) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&mbar[b ^ 1], kTileBytes);
                tma_load_rows(tiles + (b ^ 1) * kTileBytes, &tmap, &mbar[b ^ 1],
                              (int)(queue_tile(nk, P.n_tiles) * ur - hr));
            }
        }
        const bool ok = tile_wait(mbar, &mbar[2], b, it, P.stall);
        if (__syncthreads_or(!ok)) {
            if (t == 0)
                tile_wait_failed(P.err, mbar, b, it, prefetch);
            return;
        }
        const long long next = s_next;  // written by thread 0 before the barrier

        float h[K], l[K];
        unsigned char *rp = cur + t * kRowBytes;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const unsigned char *p = rp + ((c ^ (t & 7)) << 4);
            if (P.df_in) {
                const double2 q = *reinterpret_cast<const double2 *>(p);
                df_split(ldexp(q.x, -e0), h[2 * c], l[2 * c]);
                df_split(ldexp(q.y, -e0), h[2 * c + 1], l[2 * c + 1]);
            } else {
                const float4 q = *reinterpret_cast<const float4 *>(p);
                h[2 * c] = q.x;
                l[2 * c] = q.y;
                h[2 * c + 1] = q.z;
                l[2 * c + 1] = q.w;
            }
        }
        const long long g0 = tile * P.U - P.H + (long long)t * K;
        // the whole warp takes the checked path if any lane holds a wall
        // point, a point outside the grid, or a partner outside it
        const bool edge_thr = !(g0 >= 1 && g0 + K <= P.n - 1);
        const bool edge_warp = __any_sync(0xffffffffu, edge_thr);
        const Span sp = make_span<K>(g0, P.n);
        if (edge_warp)
            df_run<true, GL>(h, l, P, x, sp, e0);
        else
            df_run<false, GL>(h, l, P, x, sp, e0);

        // write back every row, then copy the output rows out with coalesced
        // stores
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            unsigned char *p = rp + ((c ^ (t & 7)) << 4);
            if (P.df_out)
                *reinterpret_cast<double2 *>(p) =
                    make_double2(ldexp((double)h[2 * c] + (double)l[2 * c], e0),
                                 ldexp((double)h[2 * c + 1] + (double)l[2 * c + 1], e0));
            else
                *reinterpret_cast<float4 *>(p) = make_float4(h[2 * c], l[2 * c], h[2 * c + 1], l[2 * c + 1]);
        }
        __syncthreads();
        {
            const long long grow0 = tile * ur;
            unsigned char *out = static_cast<unsigned char *>(P.out);
            for (int ch = t; ch < ur * CH; ch += kDfNT) {
                const int lr = hr + ch / CH;
                const int c = ch % CH;
                const long long gr = grow0 + ch / CH;
                if (gr < P.n_rows) {
                    const uint4 val = *reinterpret_cast<const uint4 *>(cur + lr * kRowBytes + ((c ^ (lr & 7)) << 4));
                    *reinterpret_cast<uint4 *>(out + gr * kRowBytes + c * 16) = val;
                }
            }
        }
        __syncthreads();
        k = next;
    }
}

}  // namespace

cudaError_t df_prescale(const void *u, long long n, int walls_code, int *code, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(code, 0, sizeof(int), s);
    if (e != cudaSuccess)
        return e;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096)
        blocks = 4096;
    if (blocks < 1)
        blocks = 1;
    df_exponent_kernel<<<(int)blocks, 256, 0, s>>>(static_cast<const double *>(u), n, walls_code, code);
    return cudaGetLastError();
}

bool tb_df_geometry(int reach, int *H, int *U)
{
    const int ht = (reach + kDfK - 1) / kDfK;  // halo, in threads
    *H = ht * kDfK;
    *U = kDfNT * kDfK - 2 * *H;
    return *U > 0;
}

cudaError_t tb_df_occupancy(int *blocks)
{
    int b[2] = {0, 0};
    cudaError_t e = cudaFuncSetAttribute(tb_df_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         tb_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tb_df_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tb_smem_bytes());
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b[0], tb_df_kernel<false>, kDfNT, tb_smem_bytes());
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b[1], tb_df_kernel<true>, kDfNT, tb_smem_bytes());
    *blocks = b[0] < b[1] ? b[0] : b[1];
    return e;
}

cudaError_t launch_tb_df(const void *tmap, const TbParams &p, int grid, cudaStream_t s)
{
    const CUtensorMap *m = static_cast<const CUtensorMap *>(tmap);
    if (p.df_gl)
        tb_df_kernel<true><<<grid, kDfNT, tb_smem_bytes(), s>>>(*m, p);
    else
        tb_df_kernel<false><<<grid, kDfNT, tb_smem_bytes(), s>>>(*m, p);
    return cudaGetLastError();
}

}  // namespace ge
