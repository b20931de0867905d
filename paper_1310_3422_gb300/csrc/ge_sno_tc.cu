// ge_sno_tc.cu -- the surrogate's inference GEMMs on the fifth-generation
// tensor cores: tcgen05.mma with the accumulator in tensor memory (TMEM),
// operands staged in shared memory by 2D TMA copies, and the epilogue fused.
// The paper has no counterpart (the surrogate is a deployment variant of the
// GE solve; see ge_sno.h for the model).
//
// Three kernels: two of one template, each over 128-row tiles of the activation
// rows (all problems' grid points, [rows][64] BF16, channel last):
//   layer (MODE 0):  pre = G y + v W + b, then GELU (not after the last
//       layer), written as the next BF16 activation.  G [n][2M] is the
//       inverse truncated DFT, y [2M][C] the mode-mixed spectrum of the
//       tile's problem, v the tile's activations, W [C][C] the pointwise
//       weights.  Two products accumulate into one TMEM tile: K = 2M = 32
//       (G y) and K = C = 64 (v W).
//   projection (MODE 1): out = u0 + q2 + sum_h GELU(v Q1 + q1)_h Q2_h, one
//       FP32 value per row; the hidden layer (N = H = 128) lives in TMEM
//       only, and each thread sums its row in a fixed order;
// and the truncated DFT vh[b] = F v[b] of a layer's input (sno_tc_dft_kernel,
// described where it is defined).
//
// A operands are K-major with 128-byte (C = 64 BF16) or 64-byte (2M = 32
// BF16) rows, TMA-swizzled (SWIZZLE_128B / SWIZZLE_64B) as the tensor cores
// read them.  B operands: the spectrum y [2M][C] and the activations v (in
// the DFT) are read as stored, MN-major (N = 64 channels contiguous, one
// 128-byte swizzle atom wide); W and Q1 go through transposed copies W^T
// [C][C] and Q1^T [H][C] (K-major; a small kernel below writes them when
// the parameters change).  One MMA instruction covers 128 rows x N columns
// x 16 of K.
//
// Warp roles (160 threads): warp 4 lane 0 is the producer: it issues the TMA
// loads of a stage (two stages) and, once they land, the MMAs of the tile
// into a TMEM accumulator (two in the layer, one in the projection), then
// commits them to an mbarrier.
// Warps 0-3 drain the accumulator of a finished tile (warp w reads TMEM
// lanes 32w .. 32w + 31, i.e. tile rows) with tcgen05.ld, hand it back, and
// run the epilogue.  So the loads of tile i+1 (and, in the layer, its MMAs)
// run under the epilogue of tile i.  The layer's output leaves through a
// small per-warp staging buffer and TMA stores (whole 128-byte lines).
//
// Every wait is bounded: on expiry the kernel records GE_ETIMEOUT in the
// device error word, stops every role at its next wait, lets its own copies
// and MMAs in flight finish (each wait bounded again), frees its TMEM and
// returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "ge_f32x2.cuh"
#include "ge_internal.h"
#include "ge_sno_internal.h"

namespace ge {
namespace {

__device__ __forceinline__ uint32_t saddr(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void bar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool bar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity`; false after `limit` cycles or once the CTA aborts.
__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity, long long limit, volatile int *abort)
{
    const long long t0 = clock64();
    while (!bar_try(bar, parity)) {
        if (*abort || clock64() - t0 > limit)
            return false;
    }
    return true;
}

// Same, ignoring the abort flag (draining this CTA's own work before exit).
__device__ __forceinline__ void bar_drain(uint64_t *bar, uint32_t parity, long long limit)
{
    const long long t0 = clock64();
    while (!bar_try(bar, parity) && clock64() - t0 <= limit) {
    }
}

__device__ __forceinline__ void tma_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(saddr(bar))
        : "memory");
}

// 2D tensor store of a shared-memory box to global memory (bulk-group
// completion), and the bulk-group waits: .read = the box has been read out of
// shared memory (the buffer may be rewritten), plain = the writes are done.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, const void *src, int x, int y)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(saddr(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// generic-proxy writes to shared memory made visible to the async proxy (TMA)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ---- tcgen05 -------------------------------------------------------------

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(dst)), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] B[smem]^T, BF16 x BF16 -> FP32, one CTA.
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

// Arrive on `bar` once every MMA this thread issued so far has completed.
__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand tile whose rows of
// `row_bytes` (128 or 64) are TMA-swizzled with the same width: groups of 8
// rows lie 8 * row_bytes apart (stride byte offset), the leading byte offset
// is unused for a swizzled K-major tile, bits 46-47 hold the descriptor
// version (1), bits 61-63 the swizzle (2: 128-byte, 4: 64-byte).  The tile
// starts on a 1024-byte boundary; a K step of 16 BF16 (32 bytes) inside the
// swizzle row advances the start address.
__device__ __forceinline__ uint64_t smem_desc(const void *tile, uint32_t row_bytes)
{
    const uint64_t addr = saddr(tile);
    const uint64_t layout = row_bytes == 128 ? 2 : 4;
    return ((addr & 0x3FFFF) >> 4) | (1ull << 16) | ((uint64_t)((8 * row_bytes) >> 4) << 32) | (1ull << 46) |
           (layout << 61);
}

// Instruction descriptor of kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// B operand descriptor, MN-major with a 128-byte swizzle, for a tile of K
// rows of 64 BF16 N values (one swizzle atom wide, as TMA stores a box 128
// bytes wide): 8-row K groups 1024 bytes apart (the same stride in both
// offset fields: with one atom across N, only the K direction has a stride).
// The instruction descriptor marks B MN-major with bit 16.
constexpr uint32_t kIdescBMn = 1u << 16;
__device__ __forceinline__ uint64_t smem_desc_mn128(const void *tile)
{
    const uint64_t addr = saddr(tile);
    return ((addr & 0x3FFFF) >> 4) | ((uint64_t)(1024 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

// GELU, tanh form: GELU(x) = x (1 + tanh(k0 (x + k1 x^3))) / 2
constexpr float kGeluK0 = 0.7978845608028654f, kGeluK0K1 = 0.7978845608028654f * 0.044715f;

__device__ __forceinline__ float gelu_hw(float x)
{
    const float k0 = 0.7978845608028654f, k1 = 0.044715f;
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(k0 * (x + k1 * x * x * x)));
    return 0.5f * x * (1.0f + t);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // .x = a (low half), .y = b
    return *reinterpret_cast<const uint32_t *>(&h);
}

constexpr int kTcThreads = 160;
constexpr int kTileM = 128;

template <int MODE>
struct TcShape {
    static constexpr int N = MODE == 0 ? 64 : 128;                  // output columns (TMEM columns per stage)
    static constexpr uint32_t kA2 = kTileM * 128;                    // v tile: 128 rows x 64 BF16
    static constexpr uint32_t kA1 = MODE == 0 ? kTileM * 64 : 0;     // G tile: 128 rows x 32 BF16
    static constexpr uint32_t kB1 = MODE == 0 ? 32 * 128 : 0;        // y: 32 rows x 64 BF16
    static constexpr uint32_t kStage = kA2 + kA1 + kB1;              // bytes of one stage (x1024)
    static constexpr uint32_t kB2 = N * 128;                         // W^T (64 rows) or Q1^T (128 rows)
    // TMEM accumulators: the layer keeps two (the next tile's MMAs run under
    // this tile's epilogue); the projection one, so that four CTAs fit an SM
    // (4 x 128 of the 512 columns) and their 16 epilogue warps hide the
    // latency of its GELU arithmetic
    static constexpr int kAccs = MODE == 0 ? 2 : 1;
    static constexpr uint32_t kTmemCols = kAccs * N;
    // layer: per epilogue warp a 2 KB staging buffer of its 32 output rows x
    // 32 columns (64-byte swizzle), written to global memory by a TMA store
    static constexpr uint32_t kOut = MODE == 0 ? 4 * 2048 : 0;
    static constexpr int kSmem = (int)(2 * kStage + kB2 + kOut + 1024);
};

template <int MODE>
__global__ void __launch_bounds__(kTcThreads) sno_tc_kernel(const __grid_constant__ CUtensorMap tmA1,
                                                            const __grid_constant__ CUtensorMap tmB1,
                                                            const __grid_constant__ CUtensorMap tmA2,
                                                            const __grid_constant__ CUtensorMap tmB2,
                                                            const __grid_constant__ CUtensorMap tmOut,
                                                            const __grid_constant__ SnoTcArgs P)
{
    using S = TcShape<MODE>;
    constexpr int N = S::N;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char *b2 = sm + 2 * S::kStage;
    __shared__ __align__(8) uint64_t full[2], mma_done[2], acc_empty[2], b2_full;
    __shared__ uint32_t tmem_base_sh;
    __shared__ __align__(16) float s_bias[N];
    __shared__ __align__(16) float s_q2[N];
    __shared__ volatile int s_abort;

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (t == 0) {
        for (int s = 0; s < 2; ++s) {
            bar_init(&full[s], 1);
            bar_init(&mma_done[s], 1);
            bar_init(&acc_empty[s], 4);
        }
        bar_init(&b2_full, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base_sh, S::kTmemCols);
        tmem_relinquish();
    }
    for (int i = t; i < N; i += kTcThreads) {
        s_bias[i] = P.bias[i];
        // the projection keeps Q2 / 2 (exact): GELU's factor 1/2 moves onto it
        s_q2[i] = MODE == 1 ? 0.5f * P.q2w[i] : 0.0f;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_base_sh;
    const long long my_tiles =
        P.n_tiles > (long long)blockIdx.x ? (P.n_tiles - 1 - (long long)blockIdx.x) / gridDim.x + 1 : 0;

    if (warp == 4) {
        if (lane == 0 && my_tiles > 0) {
            // ---- producer: TMA loads and MMA issue ----------------------
            constexpr uint32_t idesc = idesc_bf16(kTileM, N);
            auto load_stage = [&](int s, long long i) {
                const long long g = (long long)blockIdx.x + i * gridDim.x;
                unsigned char *st = sm + s * S::kStage;
                bar_expect_tx(&full[s], S::kStage);
                tma_2d(st, &tmA2, 0, (int)(g * kTileM), &full[s]);
                if (MODE == 0) {
                    const long long b = g / P.tiles_per_problem, tt = g % P.tiles_per_problem;
                    tma_2d(st + S::kA2, &tmA1, 0, (int)(tt * kTileM), &full[s]);
                    tma_2d(st + S::kA2 + S::kA1, &tmB1, 0, (int)(b * 32), &full[s]);
                }
            };
            bar_expect_tx(&b2_full, S::kB2);
            tma_2d(b2, &tmB2, 0, P.b2_row, &b2_full);
            load_stage(0, 0);
            long long issued = 0, committed = 0;  // stages loaded, tiles committed
            bool ok = bar_wait(&b2_full, 0, P.limit, &s_abort);
            for (long long i = 0; ok && i < my_tiles; ++i) {
                const int s = (int)(i & 1);
                if (i + 1 < my_tiles) {
                    const int s1 = (int)((i + 1) & 1);
                    // stage s1 is free once the MMAs of tile i - 1 (which read it) are done
                    if (i >= 1 && !(ok = bar_wait(&mma_done[s1], (uint32_t)(((i - 1) >> 1) & 1), P.limit, &s_abort)))
                        break;
                    load_stage(s1, i + 1);
                    issued = i + 1;
                }
                if (!(ok = bar_wait(&full[s], (uint32_t)((i >> 1) & 1), P.limit, &s_abort)))
                    break;
                // accumulator i % kAccs is free once the epilogue of tile
                // i - kAccs has read it
                const int ac = (int)(i % S::kAccs);
                if (i >= S::kAccs && !(ok = bar_wait(&acc_empty[ac], (uint32_t)(((i - S::kAccs) / S::kAccs) & 1),
                                                      P.limit, &s_abort)))
                    break;
                tc_fence_after();
                const uint32_t acc = tbase + (uint32_t)(ac * N);
                unsigned char *st = sm + s * S::kStage;
                const uint64_t a2 = smem_desc(st, 128), bw = smem_desc(b2, 128);
                if (MODE == 0) {
                    // G y: the spectrum y[b] [2M][C] is read as stored (channels
                    // contiguous: an MN-major B operand, K steps of 16 rows =
                    // 2048 bytes); G's K step is 32 bytes inside its swizzle row
                    const uint64_t a1 = smem_desc(st + S::kA2, 64), b1 = smem_desc_mn128(st + S::kA2 + S::kA1);
                    tc_mma(acc, a1, b1, idesc | kIdescBMn, 0);
                    tc_mma(acc, a1 + 2, b1 + (2048 >> 4), idesc | kIdescBMn, 1);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    tc_mma(acc, a2 + 2 * k, bw + 2 * k, idesc, (MODE == 0 || k > 0) ? 1u : 0u);
                tc_commit(&mma_done[s]);
                committed = i + 1;
            }
            if (!ok) {
                atomicExch(P.err, kDevTimeout);
                s_abort = 1;
                // this CTA's own work in flight: the loads it issued and the
                // MMAs it committed
                bar_drain(&b2_full, 0, kWaitLimitCycles);
                for (long long j = committed; j <= issued; ++j)
                    bar_drain(&full[j & 1], (uint32_t)((j >> 1) & 1), kWaitLimitCycles);
                if (committed > 0)
                    bar_drain(&mma_done[(committed - 1) & 1], (uint32_t)(((committed - 1) >> 1) & 1),
                              kWaitLimitCycles);
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue warps 0-3: TMEM lanes 32 warp .. 32 warp + 31 ------
        for (long long i = 0; i < my_tiles; ++i) {
            const int s = (int)(i & 1);
            const bool ok = bar_wait(&mma_done[s], (uint32_t)((i >> 1) & 1), P.limit, &s_abort);
            if (__any_sync(0xffffffffu, !ok)) {
                if (lane == 0 && !s_abort) {
                    atomicExch(P.err, kDevTimeout);
                    s_abort = 1;
                }
                break;
            }
            tc_fence_after();
            const long long g = (long long)blockIdx.x + i * gridDim.x;
            const long long row = g * kTileM + warp * 32 + lane;
            const int ac = (int)(i % S::kAccs);
            const uint32_t taddr = tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ac * N);
            if (MODE == 0) {
                uint32_t r0[32], r1[32];
                tmem_ld32(taddr, r0);
                tmem_ld32(taddr + 32, r1);
                tmem_wait_ld();
                tc_fence_before();
                __syncwarp();
                if (lane == 0)
                    bar_arrive(&acc_empty[ac]);
                // the warp's 32 rows leave through its staging buffer, 32
                // columns (64 bytes a row) at a time: the 16-byte chunk q of
                // row `lane` sits at chunk q ^ ((lane >> 1) & 3), the 64-byte
                // swizzle the store's tensor map reads
                unsigned char *stg = sm + 2 * S::kStage + S::kB2 + warp * 2048;
                const long long row0 = g * kTileM + warp * 32;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint32_t *r = h ? r1 : r0;
                    uint32_t w[16];
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        float a = __uint_as_float(r[2 * c]) + s_bias[32 * h + 2 * c];
                        float b = __uint_as_float(r[2 * c + 1]) + s_bias[32 * h + 2 * c + 1];
                        if (P.gelu) {
                            a = gelu_hw(a);
                            b = gelu_hw(b);
                        }
                        w[c] = pack_bf16(a, b);
                    }
                    // the buffer is free once the previous store has read it
                    if (lane == 0)
                        bulk_wait_read0();
                    __syncwarp();
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        *reinterpret_cast<uint4 *>(stg + lane * 64 + ((q ^ ((lane >> 1) & 3)) << 4)) =
                            make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
                    fence_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        tma_store_2d(&tmOut, stg, 32 * h, (int)row0);
                        bulk_commit();
                    }
                }
            } else {
                // sum_h GELU(x_h) Q2_h with x_h = acc_h + q1_h, on column pairs
                // in packed FP32: GELU(x) Q2 = (x + x tanh(a)) (Q2 / 2) with
                // a = x (k0 + k0 k1 x^2).  Pair p of the row goes to partial
                // sum p % 4 (four short dependency chains); the partial sums
                // and their two lanes are added at the end in a fixed order.
                // TMEM is read 64 columns at a time (two loads, one wait).
                const uint64_t c_lo = f2(kGeluK0, kGeluK0), c_hi = f2(kGeluK0K1, kGeluK0K1);
                uint64_t part[4];
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    part[k] = f2(0.0f, 0.0f);
#pragma unroll
                for (int h = 0; h < N / 64; ++h) {
                    uint32_t r[2][32];
                    tmem_ld32(taddr + 64 * h, r[0]);
                    tmem_ld32(taddr + 64 * h + 32, r[1]);
                    tmem_wait_ld();
#pragma unroll
                    for (int c = 0; c < 64; c += 2) {
                        const int col = 64 * h + c;
                        const float2 bq = *reinterpret_cast<const float2 *>(&s_bias[col]);
                        const float2 wq = *reinterpret_cast<const float2 *>(&s_q2[col]);
                        const uint32_t *rr = r[c >> 5];
                        const uint64_t x =
                            f2_add(f2(__uint_as_float(rr[c & 31]), __uint_as_float(rr[(c & 31) + 1])), f2(bq.x, bq.y));
                        const uint64_t a = f2_mul(x, f2_fma(f2_mul(x, x), c_hi, c_lo));
                        const float2 af = f2_split(a);
                        float t0, t1;
                        asm("tanh.approx.f32 %0, %1;" : "=f"(t0) : "f"(af.x));
                        asm("tanh.approx.f32 %0, %1;" : "=f"(t1) : "f"(af.y));
                        part[(c >> 1) & 3] = f2_fma(f2_fma(x, f2(t0, t1), x), f2(wq.x, wq.y), part[(c >> 1) & 3]);
                    }
                }
                const float2 accf = f2_split(f2_add(f2_add(part[0], part[1]), f2_add(part[2], part[3])));
                const float sum = accf.x + accf.y;
                tc_fence_before();
                __syncwarp();
                if (lane == 0)
                    bar_arrive(&acc_empty[ac]);
                float *out = static_cast<float *>(P.out);
                out[row] = P.u0[row] + P.q2b[0] + sum;
            }
        }
    }
    // the layer's output stores have landed before the CTA exits
    if (MODE == 0 && warp < 4 && lane == 0)
        bulk_wait0();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        tmem_dealloc(tbase, S::kTmemCols);
}

// ---- truncated DFT on the tensor cores ------------------------------------
//
// vh[b] = F v[b]: F [2M][n] (the truncated transform, 2M = 32 rows), v[b]
// [n][C] the problem's activations (C = 64).  One MMA takes M = 128 rows of
// A: A is F's 32 rows of a 128-point chunk of the grid (K-major, 128-byte
// swizzle); its rows 32 .. 127 are whatever shared memory of the same stage
// follows them, and the accumulator rows they produce are never read.  B is the activation
// tile exactly as the layer kernel loads it ([128 points][64 channels]): the
// channels (N) are contiguous, so B is MN-major, with 8-point groups 1024
// bytes apart and 16 points (one K step) 2048 bytes on.  A CTA takes whole
// problems: the n / 128 chunks (8 MMAs each) accumulate into one TMEM tile,
// then warp 0 (TMEM lanes 0 .. 31 = the 2M transform rows) writes vh[b] as
// BF16 [2M][C].  Warp 1's lane 0 is the producer (two stages of TMA loads,
// the MMAs, commits); two accumulators, so the next problem's MMAs run
// under the previous one's write-out.  Bounded waits as in sno_tc_kernel.
constexpr int kDftThreads = 64;
constexpr uint32_t kDftAtom = 32 * 128;              // F rows of one 64-point half of a chunk
constexpr uint32_t kDftV = 128 * 128;                // the activation tile
constexpr uint32_t kDftStage = 2 * kDftAtom + kDftV;  // 24 KB: F halves first, so A's unused rows stay inside
constexpr int kDftSmem = (int)(2 * kDftStage) + 1024;

__global__ void __launch_bounds__(kDftThreads) sno_tc_dft_kernel(const __grid_constant__ CUtensorMap tmF,
                                                                 const __grid_constant__ CUtensorMap tmV,
                                                                 const __grid_constant__ SnoTcArgs P)
{
    const int kChunks = P.tiles_per_problem;  // 128-point chunks of a problem
    constexpr uint32_t idesc = idesc_bf16(128, 64) | kIdescBMn;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    __shared__ __align__(8) uint64_t full[2], freed[2], done[2], acc_empty[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int s_abort;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (t == 0) {
        for (int s = 0; s < 2; ++s) {
            bar_init(&full[s], 1);
            bar_init(&freed[s], 1);
            bar_init(&done[s], 1);
            bar_init(&acc_empty[s], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base_sh, 128);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_base_sh;
    const long long problems = P.n_tiles / P.tiles_per_problem;
    const long long mine = problems > (long long)blockIdx.x ? (problems - 1 - (long long)blockIdx.x) / gridDim.x + 1 : 0;

    if (warp == 1) {
        if (lane == 0 && mine > 0) {
            // ---- producer: loads and MMAs, item = (problem, chunk) ----------
            const long long items = mine * kChunks;
            auto load = [&](long long it) {
                const int s = (int)(it & 1);
                const long long b = (long long)blockIdx.x + (it / kChunks) * gridDim.x;
                const int ch = (int)(it % kChunks);
                unsigned char *st = sm + s * kDftStage;
                bar_expect_tx(&full[s], 2 * kDftAtom + kDftV);
                tma_2d(st, &tmF, ch * 128, 0, &full[s]);
                tma_2d(st + kDftAtom, &tmF, ch * 128 + 64, 0, &full[s]);
                tma_2d(st + 2 * kDftAtom, &tmV, 0, (int)((b * kChunks + ch) * 128), &full[s]);
            };
            long long issued = 0, committed = 0;
            bool ok = true;
            load(0);
            issued = 1;
            for (long long it = 0; ok && it < items; ++it) {
                const int s = (int)(it & 1);
                const long long prob = it / kChunks;
                const int ch = (int)(it % kChunks);
                if (it + 1 < items) {
                    // stage (it + 1) & 1 is free once the MMAs of item it - 1 are done
                    if (it >= 1 && !(ok = bar_wait(&freed[(it + 1) & 1], (uint32_t)(((it - 1) >> 1) & 1), P.limit,
                                                    &s_abort)))
                        break;
                    load(it + 1);
                    issued = it + 2;
                }
                if (!(ok = bar_wait(&full[s], (uint32_t)((it >> 1) & 1), P.limit, &s_abort)))
                    break;
                const int a = (int)(prob & 1);  // accumulator of this problem
                if (ch == 0 && prob >= 2 &&
                    !(ok = bar_wait(&acc_empty[a], (uint32_t)(((prob - 2) >> 1) & 1), P.limit, &s_abort)))
                    break;
                tc_fence_after();
                unsigned char *st = sm + s * kDftStage;
                const uint32_t acc = tbase + (uint32_t)(a * 64);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    // K step k: points 16k .. 16k + 15 of the chunk
                    const uint64_t ad = smem_desc(st + (k >> 2) * kDftAtom, 128) + (uint64_t)(2 * (k & 3));
                    const uint64_t bd = smem_desc_mn128(st + 2 * kDftAtom) + (uint64_t)(k * (2048 >> 4));
                    tc_mma(acc, ad, bd, idesc, (ch > 0 || k > 0) ? 1u : 0u);
                }
                tc_commit(&freed[s]);
                if (ch == kChunks - 1)
                    tc_commit(&done[a]);
                committed = it + 1;
            }
            if (!ok) {
                atomicExch(P.err, kDevTimeout);
                s_abort = 1;
                for (long long j = committed; j < issued; ++j)
                    bar_drain(&full[j & 1], (uint32_t)((j >> 1) & 1), kWaitLimitCycles);
                if (committed > 0)
                    bar_drain(&freed[(committed - 1) & 1], (uint32_t)(((committed - 1) >> 1) & 1), kWaitLimitCycles);
            }
        }
        __syncwarp();
    } else {
        // ---- warp 0: TMEM lanes 0 .. 31 (transform rows) -> vh[b] ----------
        for (long long prob = 0; prob < mine; ++prob) {
            const int a = (int)(prob & 1);
            const bool ok = bar_wait(&done[a], (uint32_t)((prob >> 1) & 1), P.limit, &s_abort);
            if (__any_sync(0xffffffffu, !ok)) {
                if (lane == 0 && !s_abort) {
                    atomicExch(P.err, kDevTimeout);
                    s_abort = 1;
                }
                break;
            }
            tc_fence_after();
            uint32_t r0[32], r1[32];
            const uint32_t taddr = tbase + (uint32_t)(a * 64);
            tmem_ld32(taddr, r0);
            tmem_ld32(taddr + 32, r1);
            tmem_wait_ld();
            tc_fence_before();
            __syncwarp();
            if (lane == 0)
                bar_arrive(&acc_empty[a]);
            const long long b = (long long)blockIdx.x + prob * gridDim.x;
            uint4 *dst = reinterpret_cast<uint4 *>(static_cast<unsigned char *>(P.out) + (b * 32 + lane) * 128);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint32_t *r = h ? r1 : r0;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    dst[4 * h + q] = make_uint4(pack_bf16(__uint_as_float(r[8 * q]), __uint_as_float(r[8 * q + 1])),
                                                pack_bf16(__uint_as_float(r[8 * q + 2]), __uint_as_float(r[8 * q + 3])),
                                                pack_bf16(__uint_as_float(r[8 * q + 4]), __uint_as_float(r[8 * q + 5])),
                                                pack_bf16(__uint_as_float(r[8 * q + 6]), __uint_as_float(r[8 * q + 7])));
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        tmem_dealloc(tbase, 128);
}

// ---- per-mode complex mixing on the tensor cores ---------------------------
//
// y[b, m] = vh[b, m] Wspec_m for every mode m: vh[b, m] is the 2C = 128 values
// (real and imaginary parts of the C channels) of mode m of problem b, Wspec_m
// the [2C][2C] real form of the complex mode weights.  A CTA takes 128
// problems of one mode: A = those problems' vh[., m] rows (K-major, two
// 64-wide 128-byte-swizzled boxes), B = Wspec_m^T [N][K] (K-major, written so
// by the K-major variant of the spectral-weight assembly), one 128 x 128 FP32
// accumulator in TMEM after 8 MMAs of K = 16.  Thread 0 issues the four loads
// and the MMAs; the four warps then read back their 32 rows each and write
// y[b, m] as BF16 (rows past the batch are not written).
constexpr int kMixThreads = 128;
constexpr uint32_t kMixHalf = 128 * 128;  // one 64-wide box of 128 rows
constexpr int kMixSmem = (int)(4 * kMixHalf) + 1024;

__global__ void __launch_bounds__(kMixThreads) sno_tc_mix_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                 const __grid_constant__ CUtensorMap tmB,
                                                                 const __grid_constant__ SnoTcMixArgs P)
{
    constexpr uint32_t idesc = idesc_bf16(128, 128);
    extern __shared__ unsigned char smem_raw[];
    unsigned char *sm = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char *sa = sm, *sb = sm + 2 * kMixHalf;
    __shared__ __align__(8) uint64_t full, done;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int s_abort;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int m = blockIdx.y;
    const int row0 = blockIdx.x * 128;
    if (t == 0) {
        bar_init(&full, 1);
        bar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 0) {
        tmem_alloc(&tmem_base_sh, 128);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = tmem_base_sh;
    if (t == 0) {
        bar_expect_tx(&full, 4 * kMixHalf);
        tma_2d(sa, &tmA, m * 128, row0, &full);
        tma_2d(sa + kMixHalf, &tmA, m * 128 + 64, row0, &full);
        tma_2d(sb, &tmB, 0, P.b_row0 + m * 128, &full);
        tma_2d(sb + kMixHalf, &tmB, 64, P.b_row0 + m * 128, &full);
        if (bar_wait(&full, 0, P.limit, &s_abort)) {
            tc_fence_after();
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint64_t ad = smem_desc(sa + h * kMixHalf, 128), bd = smem_desc(sb + h * kMixHalf, 128);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    tc_mma(tbase, ad + 2 * k, bd + 2 * k, idesc, (h > 0 || k > 0) ? 1u : 0u);
            }
            tc_commit(&done);
        } else {
            atomicExch(P.err, kDevTimeout);
            s_abort = 1;
            bar_drain(&full, 0, kWaitLimitCycles);  // the loads in flight land before the CTA exits
        }
    }
    const bool ok = bar_wait(&done, 0, P.limit, &s_abort);
    if (__any_sync(0xffffffffu, !ok)) {
        if (lane == 0 && !s_abort) {
            atomicExch(P.err, kDevTimeout);
            s_abort = 1;
        }
        if (t == 0)
            bar_drain(&done, 0, kWaitLimitCycles);  // MMAs it issued finish before TMEM is freed
    } else {
        tc_fence_after();
        const int b = row0 + warp * 32 + lane;
        uint4 *dst = reinterpret_cast<uint4 *>(static_cast<unsigned char *>(P.y) +
                                               ((long long)b * P.row_elems + (long long)m * 128) * 2);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            uint32_t r[32];
            tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(32 * h), r);
            tmem_wait_ld();
            if (b < P.batch) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    dst[4 * h + q] = make_uint4(pack_bf16(__uint_as_float(r[8 * q]), __uint_as_float(r[8 * q + 1])),
                                                pack_bf16(__uint_as_float(r[8 * q + 2]), __uint_as_float(r[8 * q + 3])),
                                                pack_bf16(__uint_as_float(r[8 * q + 4]), __uint_as_float(r[8 * q + 5])),
                                                pack_bf16(__uint_as_float(r[8 * q + 6]), __uint_as_float(r[8 * q + 7])));
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        tmem_dealloc(tbase, 128);
}

// yT[b][c][k] = y[b][k][c]  (BF16, K = 2M rows, C columns per problem);
// 32-bit indices (the caller checks that every index fits)
__global__ void transpose_rows_kernel(const __nv_bfloat16 *__restrict__ y, __nv_bfloat16 *__restrict__ yt,
                                      int batch, int k_rows, int c_cols)
{
    const int per = k_rows * c_cols;
    const int total = batch * per;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int b = e / per;
        const int rem = e - b * per;
        const int c = rem / k_rows, k = rem - c * k_rows;
        yt[e] = y[b * per + k * c_cols + c];
    }
}

template <int MODE>
cudaError_t launch_tc(const SnoTcMaps &m, const SnoTcArgs &a, int sms, cudaStream_t s)
{
    using S = TcShape<MODE>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(sno_tc_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             S::kSmem);
        // the largest shared-memory carve-out, so that as many CTAs fit as
        // TMEM allows (3 layer CTAs of 74 KB need about 225 KB)
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(sno_tc_kernel<MODE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess)
            return e;
        attr_set = true;
    }
    // co-resident CTAs per SM: what shared memory holds (the kernel's static
    // and dynamic bytes plus the driver's reserve per CTA), capped so that
    // their TMEM columns (at most 512 per SM) all fit
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaFuncAttributes fa{};
        int dev = 0, sm_bytes = 0, reserve = 0;
        cudaError_t e = cudaFuncGetAttributes(&fa, sno_tc_kernel<MODE>);
        if (e == cudaSuccess)
            e = cudaGetDevice(&dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&reserve, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        if (e != cudaSuccess)
            return e;
        int fit = sm_bytes / (S::kSmem + (int)fa.sharedSizeBytes + reserve);
        const int tmem_cap = 512 / (int)S::kTmemCols;
        per_sm = fit < tmem_cap ? fit : tmem_cap;
        if (per_sm < 1)
            return cudaErrorInvalidConfiguration;
    }
    long long grid = (long long)sms * per_sm;
    if (grid > a.n_tiles)
        grid = a.n_tiles;
    if (grid < 1)
        return cudaSuccess;
    if (!m.a2 || !m.b2 || (MODE == 0 && (!m.a1 || !m.b1 || !m.out)))
        return cudaErrorInvalidValue;
    // the projection has no first product and no output map: those
    // parameters repeat a2
    const CUtensorMap *a1 = static_cast<const CUtensorMap *>(MODE == 0 ? m.a1 : m.a2);
    const CUtensorMap *b1 = static_cast<const CUtensorMap *>(MODE == 0 ? m.b1 : m.a2);
    const CUtensorMap *o = static_cast<const CUtensorMap *>(MODE == 0 ? m.out : m.a2);
    sno_tc_kernel<MODE><<<(int)grid, kTcThreads, S::kSmem, s>>>(*a1, *b1, *static_cast<const CUtensorMap *>(m.a2),
                                                              *static_cast<const CUtensorMap *>(m.b2), *o, a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t sno_tc_layer(const SnoTcMaps &m, const SnoTcArgs &a, int sms, cudaStream_t s)
{
    return launch_tc<0>(m, a, sms, s);
}

cudaError_t sno_tc_projection(const SnoTcMaps &m, const SnoTcArgs &a, int sms, cudaStream_t s)
{
    return launch_tc<1>(m, a, sms, s);
}

cudaError_t sno_tc_dft(const void *map_f, const void *map_v, const SnoTcArgs &a, int sms, cudaStream_t s)
{
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(sno_tc_dft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kDftSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(sno_tc_dft_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
        cudaFuncAttributes fa{};
        int dev = 0, sm_bytes = 0, reserve = 0;
        if (e == cudaSuccess)
            e = cudaFuncGetAttributes(&fa, sno_tc_dft_kernel);
        if (e == cudaSuccess)
            e = cudaGetDevice(&dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&reserve, cudaDevAttrReservedSharedMemoryPerBlock, dev);
        if (e != cudaSuccess)
            return e;
        const int fit = sm_bytes / (kDftSmem + (int)fa.sharedSizeBytes + reserve);
        per_sm = fit < 4 ? fit : 4;  // 128 TMEM columns each
        if (per_sm < 1)
            return cudaErrorInvalidConfiguration;
    }
    if (!map_f || !map_v || a.tiles_per_problem < 1)
        return cudaErrorInvalidValue;
    const long long problems = a.n_tiles / a.tiles_per_problem;
    long long grid = (long long)sms * per_sm;
    if (grid > problems)
        grid = problems;
    if (grid < 1)
        return cudaSuccess;
    sno_tc_dft_kernel<<<(int)grid, kDftThreads, kDftSmem, s>>>(*static_cast<const CUtensorMap *>(map_f),
                                                              *static_cast<const CUtensorMap *>(map_v), a);
    return cudaGetLastError();
}

cudaError_t sno_tc_mix(const void *map_vh, const void *map_wst, const SnoTcMixArgs &a, int modes, cudaStream_t s)
{
    static bool ready = false;
    if (!ready) {
        cudaError_t e = cudaFuncSetAttribute(sno_tc_mix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kMixSmem);
        if (e != cudaSuccess)
            return e;
        ready = true;
    }
    if (!map_vh || !map_wst || modes < 1 || a.batch < 0)
        return cudaErrorInvalidValue;
    if (a.batch == 0)
        return cudaSuccess;
    const dim3 grid((unsigned)((a.batch + 127) / 128), (unsigned)modes);
    sno_tc_mix_kernel<<<grid, kMixThreads, kMixSmem, s>>>(*static_cast<const CUtensorMap *>(map_vh),
                                                          *static_cast<const CUtensorMap *>(map_wst), a);
    return cudaGetLastError();
}

cudaError_t sno_transpose_rows(const void *y, void *yt, long long batch, int k_rows, int c_cols, cudaStream_t s)
{
    const long long total = batch * k_rows * c_cols;
    if (total >= (1LL << 31) - 256LL * 4096)
        return cudaErrorInvalidValue;
    long long blocks = (total + 255) / 256;
    if (blocks > 4096)
        blocks = 4096;
    if (blocks < 1)
        return cudaSuccess;
    transpose_rows_kernel<<<(int)blocks, 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(y),
                                                       static_cast<__nv_bfloat16 *>(yt), (int)batch, k_rows, c_cols);
    return cudaGetLastError();
}

}  // namespace ge
