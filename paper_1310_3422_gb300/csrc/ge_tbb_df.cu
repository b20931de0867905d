// ge_tbb_df.cu -- the batched tiled kernel for FP64 plans in double-float
// arithmetic on the FP32 pipes (ge_batch_set_kernel with
// GE_KERNEL_TEMPORAL_DF).
//
// Same plan and scheme as the batched scaled form of tbb_kernel (ge_tbb.cu):
// problems packed row-aligned in one buffer, a row -> problem table, each
// problem shifted by its linear wall profile u* (an exact fixed point of the
// step, so the shifted problem has zero walls), the one-FMA scaled block map
// x <- x + g x_partner with per-problem rescalings by 2^-exps and an end
// factor that brings every launch back to the normalised state, a dynamic
// tile queue.  The arithmetic is that of the single-problem double-float
// kernel (ge_tb_df.cu, ge_df.cuh): pairs hi + lo of floats, error-free
// transformations, the low-order product terms summed exactly.
//
// Storage: the plan's buffers hold doubles between calls.  The first launch
// of a call converts each point of a problem, shifted by u* and prescaled by
// 2^-e0 of its problem (e0 from a per-problem reduction at the start of the
// call), to a pair; points of no problem (padding) are never written back,
// so the tile passes on the raw 64 bits it loaded and they come back
// exactly.  The last launch joins the pairs, scales back and adds u*.
#include <cuda.h>
#include <cstdint>

#include "ge_internal.h"
#include "ge_df.cuh"
#include "ge_tb_dev.cuh"

namespace ge {
namespace {

constexpr int K = kDfK;

// codes[b] = the walls' code of problem b.
__global__ void df_codes_init_kernel(const BatchDesc *__restrict__ desc, int np, int *__restrict__ codes)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < np)
        codes[b] = desc[b].walls_code;
}

// Raise codes[pid] to the code of every value of problem pid (one thread
// per 128-byte row of 16 doubles).
__global__ void df_codes_rows_kernel(const double *__restrict__ u, const int *__restrict__ row_pid,
                                     const BatchDesc *__restrict__ desc, long long n_rows, int *__restrict__ codes)
{
    for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < n_rows;
         row += (long long)gridDim.x * blockDim.x) {
        const int pid = row_pid[row];
        if (pid < 0)
            continue;
        const long long lo = desc[pid].off, hi = lo + desc[pid].n;
        int best = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const long long e = row * K + j;
            if (e >= lo && e < hi) {
                const double x = u[e];
                if (x != 0.0) {
                    const int c = df_exponent_bound(x) + kDfCodeBias;
                    best = c > best ? c : best;
                }
            }
        }
        if (best > codes[pid])  // a stale read only costs an extra atomic
            atomicMax(&codes[pid], best);
    }
}

// Boundary fix-ups of one thread (as BatchFix in ge_tbb.cu): registers from
// `keep` on are padding, `tail` is the problem's last point in this row
// (-1: none), `head` marks the problem's first point at register 0.
struct DfFix {
    int keep, tail;
    bool head;
};

__device__ __forceinline__ DfFix df_fix(int pid, Span sp)
{
    DfFix f;
    if (pid < 0) {
        f.keep = 0;
        f.tail = -1;
        f.head = false;
        return f;
    }
    f.keep = sp.jhi < K ? (sp.jhi < 0 ? 0 : sp.jhi) : K;
    f.tail = (sp.jhi >= 1 && sp.jhi <= K) ? sp.jhi - 1 : -1;
    f.head = sp.jlo == 0;
    return f;
}

// One scaled block step on a warp that holds problem boundaries: every lane
// runs the update (padding registers too: no point of a problem reads them,
// and the write-back skips them), then singletons become x <- kap_s x.
template <int Q>
__device__ __forceinline__ void df_batch_fixed(float (&h)[K], float (&l)[K], DfC g, DfC kap, const DfFix &f,
                                               DfExch &x)
{
    DfC L{0.0f, 0.0f}, R{0.0f, 0.0f};
    if constexpr (Q == 1)
        df_exchange(h, l, L, R, x);
    float nh[K], nl[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const DfC p = df_partner<Q>(h, l, j, L, R);
        df_axpy<true>(h[j], l[j], g.h, g.l, p.h, p.l, nh[j], nl[j]);
    }
    if (Q == 1 && f.head && f.keep > 0)
        df_mul(kap.h, kap.l, h[0], l[0], nh[0], nl[0]);
    // the last point's partner under grouping Q is tail + 1 when (tail + Q) is even
    if (f.tail >= 0 && ((f.tail + Q) & 1) == 0) {
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (j == f.tail)
                df_mul(kap.h, kap.l, h[j], l[j], nh[j], nl[j]);
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
        h[j] = nh[j];
        l[j] = nl[j];
    }
}

template <int Q, bool EDGE>
__device__ __forceinline__ void df_batch_step(float (&h)[K], float (&l)[K], DfC g, DfC kap, const DfFix &f,
                                              DfExch &x)
{
    if constexpr (EDGE)
        df_batch_fixed<Q>(h, l, g, kap, f, x);
    else
        df_mid_fast<Q, true, true>(h, l, g, x);
}

__device__ __forceinline__ DfC dpair(const BatchDesc &d, int i) { return DfC{d.dfc[i][0], d.dfc[i][1]}; }

// Entry, the launch's block steps in runs of R between the problem's
// rescalings, the end factor and the exit, on one tile (zero walls: the
// problem is shifted by u*).
template <bool EDGE>
__device__ __forceinline__ void df_batch_run(float (&h)[K], float (&l)[K], const TbbParams &P, const BatchDesc &bd,
                                             int pid, const DfFix &fx, Span sp, DfExch &x)
{
    const DfC zero{0.0f, 0.0f};
    auto inside = [&](int j) { return !EDGE || (j >= sp.jlo && j < sp.jhi); };
    if (P.do_entry) {
        // w = (1-r) u + r u_partner, singleton (1-r) u
        const DfC rr = dpair(bd, 2), omr = dpair(bd, 3);
        if (((1 - P.p_first) & 1) == 1)
            df_stage_checked<1, false, false>(h, l, omr, rr, omr, zero, zero, sp, x);
        else
            df_stage_checked<0, false, false>(h, l, omr, rr, omr, zero, zero, sp, x);
    }
    const DfC g = dpair(bd, 0), kap = dpair(bd, 1);
    int m = 0, q = 0;
    while (m < P.n_mid) {
        const int cnt = (P.n_mid - m < P.R) ? P.n_mid - m : P.R;
        int i = 0;
        if (((P.p_first + m) & 1) == 1) {
            df_batch_step<1, EDGE>(h, l, g, kap, fx, x);
            i = 1;
        }
        for (; i + 1 < cnt; i += 2) {
            df_batch_step<0, EDGE>(h, l, g, kap, fx, x);
            df_batch_step<1, EDGE>(h, l, g, kap, fx, x);
        }
        if (i < cnt)
            df_batch_step<0, EDGE>(h, l, g, kap, fx, x);
        m += cnt;
        if (cnt == P.R && pid >= 0) {
            const float sc = pow2neg<float>(P.exps[(long long)pid * P.Q + q]);
#pragma unroll
            for (int j = 0; j < K; ++j)
                if (inside(j)) {
                    h[j] *= sc;
                    l[j] *= sc;
                }
        }
        ++q;
    }
    if (pid >= 0) {
        const float2 f = reinterpret_cast<const float2 *>(P.endf)[pid];
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (inside(j))
                df_mul(f.x, f.y, h[j], l[j], h[j], l[j]);
    }
    if (P.do_exit) {
        const DfC x1 = dpair(bd, 4), x2 = dpair(bd, 5), xs = dpair(bd, 6);
        if (((P.p_first + P.n_mid) & 1) == 1)
            df_stage_checked<1, false, false>(h, l, x1, x2, xs, zero, zero, sp, x);
        else
            df_stage_checked<0, false, false>(h, l, x1, x2, xs, zero, zero, sp, x);
    }
}

// Raw 64 bits of a double in a pair's registers (padding: never used in
// arithmetic that reaches a problem's points, never written back).
__device__ __forceinline__ void raw_to_pair(double x, float &h, float &l)
{
    const long long b = __double_as_longlong(x);
    h = __int_as_float((int)(b & 0xffffffffLL));
    l = __int_as_float((int)(b >> 32));
}

__global__ void __launch_bounds__(kDfNT, 2)
    tbb_df_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ TbbParams P)
{
    constexpr int CH = kRowBytes / 16;  // 16-byte chunks per row: two points each
    constexpr uint32_t kTileBytes = kTileRows * kRowBytes;

    extern __shared__ unsigned char smem_raw[];
    unsigned char *tiles = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    __shared__ __align__(8) uint64_t mbar[3];  // two tile buffers, and one nothing arrives on
    __shared__ float2 slot[2][kDfNW][2];
    __shared__ long long s_next;

    const int t = threadIdx.x;
    const int hr = P.H / K, ur = P.U / K;
    DfExch x{slot, 0, t & 31, t >> 5};

    if (t == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_init(&mbar[2], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // tiles come from the launch's dynamic queue in order: thread 0 takes the
    // next one while the current tile is computed
    long long tile = blockIdx.x;
    if (t == 0 && tile < P.n_tiles) {
        mbar_arrive_expect_tx(&mbar[0], kTileBytes);
        tma_load_rows(tiles, &tmap, &mbar[0], (int)(tile * ur - hr));
    }
    for (long long it = 0; tile < P.n_tiles; ++it) {
        const int b = (int)(it & 1);
        unsigned char *cur = tiles + b * kTileBytes;
        bool prefetch = false;
        if (t == 0) {
            const long long next = (long long)gridDim.x + atomicAdd(P.tile_ctr, 1);
            s_next = next;
            prefetch = next < P.n_tiles;
            if (prefetch) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&mbar[b ^ 1], kTileBytes);
                tma_load_rows(tiles + (b ^ 1) * kTileBytes, &tmap, &mbar[b ^ 1], (int)(next * ur - hr));
            }
        }
        const bool ok = tile_wait(mbar, &mbar[2], b, it, P.stall);
        if (__syncthreads_or(!ok)) {
            if (t == 0)
                tile_wait_failed(P.err, mbar, b, it, prefetch);
            return;
        }
        const long long next_tile = s_next;  // written by thread 0 before the barrier

        // this thread's problem: rows outside the buffer or in padding have none
        const long long grow = tile * ur - hr + t;
        const int pid = (grow >= 0 && grow < P.n_rows) ? __ldg(P.row_pid + grow) : -1;
        BatchDesc bd{};
        Span sp{K + 1, K + 1};  // no point of this thread is inside a problem
        long long g0 = 0;
        int e0 = 0;
        if (pid >= 0) {
            bd = P.desc[pid];
            g0 = grow * K - bd.off;
            sp = make_span<K>(g0, bd.n);
            const int code = P.df_codes[pid];
            e0 = code ? code - kDfCodeBias : 0;
        }
        float h[K], l[K];
        unsigned char *rp = cur + t * kRowBytes;
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const unsigned char *p = rp + ((c ^ (t & 7)) << 4);
            if (P.df_in) {
                const double2 q = *reinterpret_cast<const double2 *>(p);
                const double v2[2] = {q.x, q.y};
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int j = 2 * c + i;
                    if (j >= sp.jlo && j < sp.jhi)
                        df_split(ldexp(v2[i] - (bd.ustar_a + bd.ustar_b * (double)(g0 + j + 1)), -e0), h[j], l[j]);
                    else
                        raw_to_pair(v2[i], h[j], l[j]);
                }
            } else {
                const float4 q = *reinterpret_cast<const float4 *>(p);
                h[2 * c] = q.x;
                l[2 * c] = q.y;
                h[2 * c + 1] = q.z;
                l[2 * c + 1] = q.w;
            }
        }
        const bool edge_thr = !(sp.jlo <= -1 && sp.jhi >= K + 1);
        const bool edge_warp = __any_sync(0xffffffffu, edge_thr);
        const DfFix fx = df_fix(pid, sp);
        if (edge_warp)
            df_batch_run<true>(h, l, P, bd, pid, fx, sp, x);
        else
            df_batch_run<false>(h, l, P, bd, pid, fx, sp, x);

        // write back the points of the thread's problem (padding and rows of
        // no problem keep the raw bits the tile loaded), then copy the output
        // rows out with coalesced stores
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            unsigned char *p = rp + ((c ^ (t & 7)) << 4);
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int j = 2 * c + i;
                if (j >= sp.jlo && j < sp.jhi) {
                    if (P.df_out)
                        reinterpret_cast<double *>(p)[i] = ldexp((double)h[j] + (double)l[j], e0) +
                                                           (bd.ustar_a + bd.ustar_b * (double)(g0 + j + 1));
                    else
                        reinterpret_cast<float2 *>(p)[i] = make_float2(h[j], l[j]);
                }
            }
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
        tile = next_tile;
    }
}

}  // namespace

cudaError_t batch_df_prescale(const double *u, const int *row_pid, const BatchDesc *desc, long long n_rows,
                              int n_problems, int *codes, cudaStream_t s)
{
    df_codes_init_kernel<<<(n_problems + 255) / 256, 256, 0, s>>>(desc, n_problems, codes);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || n_rows <= 0)
        return e;
    long long blocks = (n_rows + 255) / 256;
    if (blocks > 8192)
        blocks = 8192;
    df_codes_rows_kernel<<<(int)blocks, 256, 0, s>>>(u, row_pid, desc, n_rows, codes);
    return cudaGetLastError();
}

cudaError_t tbb_df_occupancy(int *blocks)
{
    cudaError_t e = cudaFuncSetAttribute(tbb_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tb_smem_bytes());
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, tbb_df_kernel, kDfNT, tb_smem_bytes());
}

cudaError_t launch_tbb_df(const void *tmap, const TbbParams &p, int grid, cudaStream_t s)
{
    const CUtensorMap *m = static_cast<const CUtensorMap *>(tmap);
    tbb_df_kernel<<<grid, kDfNT, tb_smem_bytes(), s>>>(*m, p);
    return cudaGetLastError();
}

}  // namespace ge
