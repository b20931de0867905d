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
#include "ge.h"
#include "ge_tb_dev.cuh"

namespace ge {
namespace {

// Scaled block step of this launch.  Only warps on the checked path (EDGE)
// need the wall terms; they carry the scale sigma of the right-hand side in
// double, with the same recurrence the host runs (see TbParams).
template <int Q, bool EDGE, typename Real, int K, int NW, bool WT>
__device__ __forceinline__ void mid_scaled(Real (&v)[K], double &sig, const TbParams &P, Exch<Real, NW, WT> &x,
                                           Span sp, Real g, Real kap, const EmuG &eg)
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
    if constexpr (!EDGE && sizeof(Real) == 8 && GE_EMU_F64 > 0 && GE_EMU_F64 < K) {
        if (P.emu && emu_g_usable(eg)) {
            stage_mid_hybrid<Q, GE_EMU_F64>(v, L, R, g, eg);
            return;
        }
    }
    stage<Q, kMid, EDGE>(v, L, R, sp, c);
}

// `count` block steps m0 .. m0+count-1, step m having grouping parity
// (p_first + m) & 1: an odd first step alone, then pairs, then an even
// trailing step.  No rescaling inside.
template <bool EDGE, typename Real, int K, int NW, bool WT>
__device__ __forceinline__ void mid_run(Real (&v)[K], int m0, int count, double &sig, const TbParams &P,
                                        Exch<Real, NW, WT> &x, Span sp, Real g, Real kap, const EmuG &eg)
{
    int m = m0;
    const int end = m0 + count;
    if (m < end && ((P.p_first + m) & 1)) {
        mid_scaled<1, EDGE>(v, sig, P, x, sp, g, kap, eg);
        ++m;
    }
    for (; m + 1 < end; m += 2) {
        mid_scaled<0, EDGE>(v, sig, P, x, sp, g, kap, eg);
        mid_scaled<1, EDGE>(v, sig, P, x, sp, g, kap, eg);
    }
    if (m < end)
        mid_scaled<0, EDGE>(v, sig, P, x, sp, g, kap, eg);
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
    const EmuG eg = emu_g(P.g);  // FP64: the integer-pipe share of the updates
    double sig = P.sigma_in;  // used on the checked path only
    int until = P.rescale_phase, ev = 0, m = 0;
    if constexpr (!EDGE && sizeof(Real) == 4 && K % 4 == 0) {
        // interior FP32 tiles: the same steps and rescalings on register
        // pairs (packed FMAs; the same bits)
        constexpr int H = K / 2;
        uint64_t pr[H];
        to_pairs(v, pr);
        const uint64_t g2 = f2((float)g, (float)g);
        auto pair_step = [&](int q) {
            if (q == 1) {
                exchange_ends(f2_split(pr[0]).x, f2_split(pr[H - 1]).y, L, R, x);
                pair_mid<1>(pr, L, R, g2);
            } else {
                pair_mid<0>(pr, L, R, g2);
            }
        };
        while (m < P.n_mid) {
            int count = P.n_mid - m;
            if (until > 0 && until < count)
                count = until;
            int mm = m;
            const int end = m + count;
            if (mm < end && ((P.p_first + mm) & 1)) {
                pair_step(1);
                ++mm;
            }
            for (; mm + 1 < end; mm += 2) {
                pair_step(0);
                pair_step(1);
            }
            if (mm < end)
                pair_step(0);
            m += count;
            if (until > 0) {
                until -= count;
                if (until == 0) {
                    until = P.rescale_every;
                    const float sc = pow2neg<float>(P.rs_exp[ev++]);
                    const uint64_t s2 = f2(sc, sc);
#pragma unroll
                    for (int j = 0; j < H; ++j)
                        pr[j] = f2_mul(pr[j], s2);
                }
            }
        }
        from_pairs(pr, v);
    } else {
    while (m < P.n_mid) {
        int count = P.n_mid - m;
        if (until > 0 && until < count)
            count = until;
        mid_run<EDGE>(v, m, count, sig, P, x, sp, g, kap, eg);
        m += count;
        if (until > 0) {
            until -= count;
            if (until == 0) {
                until = P.rescale_every;
                const int e = P.rs_exp[ev++];
                scale_pow2<true>(v, e);
                if constexpr (EDGE)
                    sig *= pow2neg<double>(e);
            }
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
    if constexpr (!EDGE && K % 4 == 0) {
        // interior tiles: the same steps on register pairs (the same bits)
        comp_steps_pairs(v, P.p_first, P.n_mid, (float)P.d, x);
    } else {
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
    }
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
    __shared__ __align__(8) uint64_t mbar[3];  // two tile buffers, and one nothing arrives on
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
        k = next;
    }
}

// One block step of a launch that does nothing else: no entry or exit
// conversion, n_mid = 1 (the middle launches of the one-step-per-launch
// path).  Such a launch moves 2 x 4 bytes per point for one multiply-add in
// FP32, so it is an HBM stream: no tiles, shared memory or barriers.  (In
// FP64 the same stream ran slower than the tiled kernel, 0.54 against 0.66
// of the HBM roofline, so the FP64 one-step launches keep the TMA-fed tiled
// kernel.  The FP64 kernels' profiles show DFMA issue waiting on the
// tex_throttle queue, which the stream's global loads and stores also use.)
// A warp takes 4 KB blocks; lane l holds the 16-byte chunks l, 32 + l, ...,
// 224 + l of the block (every load and store of the warp is 512 contiguous
// bytes).  A chunk starts on an even point, so grouping 0 pairs points inside
// a chunk; under grouping 1 a chunk's first point pairs with the previous
// chunk's last (the lane below, or lane 31 of the row before) and its last
// with the next chunk's first, by shuffles, and a block's two outer
// neighbours come from global memory.  Each chunk then takes exactly the
// tiled kernel's stage (same arithmetic, same bits), the checked stage for a
// chunk that holds a wall point, a singleton or a point outside the grid.
constexpr int kStreamChunks = 8;  // 16-byte chunks per lane per block
constexpr int kStreamThreads = 256;

template <int Q, typename Real>
__global__ void __launch_bounds__(kStreamThreads) onestep_stream_kernel(const Real *__restrict__ in,
                                                                        Real *__restrict__ out,
                                                                        const __grid_constant__ TbParams P)
{
    constexpr int E = 16 / (int)sizeof(Real);       // points per chunk
    constexpr int BLK = 32 * kStreamChunks * E;     // points per warp block
    const int lane = threadIdx.x & 31;
    const long long total = P.n_rows * (kRowBytes / (long long)sizeof(Real));  // whole rows
    const long long n_blocks = (total + BLK - 1) / BLK;
    const long long warp0 = ((long long)blockIdx.x * kStreamThreads + threadIdx.x) >> 5;
    const long long warps = ((long long)gridDim.x * kStreamThreads) >> 5;
    const Real g = (Real)P.g, kap = (Real)P.kappa;
    const StageC<Real> c{g, (Real)0, kap, (Real)0, (Real)0};
    const bool rescale = P.rescale_every > 0 && P.rescale_phase == 1;
    const Real rs = rescale ? pow2neg<Real>(P.rs_exp[0]) : (Real)1;
    for (long long blk = warp0; blk < n_blocks; blk += warps) {
        const long long base = blk * BLK;
        Real v[kStreamChunks][E];
#pragma unroll
        for (int i = 0; i < kStreamChunks; ++i) {
            const long long e0 = base + (long long)(i * 32 + lane) * E;
            if (e0 < total) {
                if constexpr (E == 2) {
                    const double2 q = *reinterpret_cast<const double2 *>(in + e0);
                    v[i][0] = q.x;
                    v[i][1] = q.y;
                } else {
                    const float4 q = *reinterpret_cast<const float4 *>(in + e0);
                    v[i][0] = q.x;
                    v[i][1] = q.y;
                    v[i][2] = q.z;
                    v[i][3] = q.w;
                }
            } else {
#pragma unroll
                for (int j = 0; j < E; ++j)
                    v[i][j] = (Real)0;
            }
        }
        // outer neighbours of the block (grouping 1 only)
        Real before = (Real)0, after = (Real)0;
        if (Q == 1) {
            if (lane == 0 && base > 0)
                before = in[base - 1];
            if (lane == 31 && base + BLK < total)
                after = in[base + BLK];
        }
        Real nv[kStreamChunks][E];
#pragma unroll
        for (int i = 0; i < kStreamChunks; ++i) {
            Real L = 0, R = 0;
            if (Q == 1) {
                L = __shfl_up_sync(0xffffffffu, v[i][E - 1], 1);
                const Real wrapL = __shfl_sync(0xffffffffu, i > 0 ? v[i - 1][E - 1] : before, 31);
                if (lane == 0)
                    L = i > 0 ? wrapL : before;
                R = __shfl_down_sync(0xffffffffu, v[i][0], 1);
                const Real wrapR = __shfl_sync(0xffffffffu, i + 1 < kStreamChunks ? v[i + 1][0] : after, 0);
                if (lane == 31)
                    R = i + 1 < kStreamChunks ? wrapR : after;
            }
            const long long g0 = base + (long long)(i * 32 + lane) * E;
#pragma unroll
            for (int j = 0; j < E; ++j)
                nv[i][j] = v[i][j];
            if (g0 >= 1 && g0 + E <= P.n - 1) {
                stage<Q, kMid, false>(nv[i], L, R, Span{-1, E + 1}, c);
            } else {
                // the wall terms of this step, scaled by sigma after it
                // (double arithmetic only here: FP64 is slow on this GPU)
                const double sig = P.sigma_in * P.onepg;
                const StageC<Real> ce{g, (Real)0, kap, (Real)(sig * P.f_l), (Real)(sig * P.f_r)};
                stage<Q, kMid, true>(nv[i], L, R, make_span<E>(g0, P.n), ce);
            }
            if (rescale) {
#pragma unroll
                for (int j = 0; j < E; ++j)
                    nv[i][j] *= rs;
            }
        }
#pragma unroll
        for (int i = 0; i < kStreamChunks; ++i) {
            const long long e0 = base + (long long)(i * 32 + lane) * E;
            if (e0 < total) {
                if constexpr (E == 2)
                    *reinterpret_cast<double2 *>(out + e0) = make_double2(nv[i][0], nv[i][1]);
                else
                    *reinterpret_cast<float4 *>(out + e0) = make_float4(nv[i][0], nv[i][1], nv[i][2], nv[i][3]);
            }
        }
    }
}

template <typename Real>
cudaError_t launch_stream(const void *in, void *out, const TbParams &p, cudaStream_t s)
{
    constexpr int E = 16 / (int)sizeof(Real);
    constexpr long long BLK = 32LL * kStreamChunks * E;
    const long long total = p.n_rows * (kRowBytes / (long long)sizeof(Real));
    const long long n_blocks = (total + BLK - 1) / BLK;
    const long long warps_per_cta = kStreamThreads / 32;
    // one warp per block: the CTAs of a stream start as others finish, with no
    // partial second wave of a capped grid
    long long grid = (n_blocks + warps_per_cta - 1) / warps_per_cta;
    if (grid > (1LL << 30))
        grid = 1LL << 30;  // grid-stride beyond that
    if (grid < 1)
        grid = 1;
    const Real *src = static_cast<const Real *>(in);
    Real *dst = static_cast<Real *>(out);
    if (p.p_first & 1)
        onestep_stream_kernel<1, Real><<<(int)grid, kStreamThreads, 0, s>>>(src, dst, p);
    else
        onestep_stream_kernel<0, Real><<<(int)grid, kStreamThreads, 0, s>>>(src, dst, p);
    return cudaGetLastError();
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

}  // namespace

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

cudaError_t launch_tb_stream(int prec, const void *in, void *out, const TbParams &p, cudaStream_t s)
{
    if (prec == 1)
        return launch_stream<float>(in, out, p, s);
    return cudaErrorInvalidValue;  // FP64 and compensated FP32 keep the tiled kernel
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

extern "C" ge_status ge_fp64_int_share(double *share)
{
    if (!share) {
        ge::set_last_error("ge_fp64_int_share: NULL share");
        return GE_EINVAL;
    }
    constexpr int K = ge::Layout<double, false>::KT;  // FP64 values per thread
    *share = (GE_EMU_F64 > 0 && GE_EMU_F64 < K) ? (double)GE_EMU_F64 / K : 0.0;
    return GE_OK;
}
