// ge_tbb.cu -- batched tiled GE kernel: many independent problems of
// uneven size and mesh ratio packed back to back in one buffer, each
// starting on a 128-byte row (arXiv:1310.3422 Sec. 2 for every problem, the
// right-hand-side scheme of ge_tb.cu).
#include "ge_tb_dev.cuh"

namespace ge {
namespace {

// The tiles run over the packed buffer exactly as for one long problem;
// every thread looks its problem up (row -> problem id), takes that
// problem's constants, and treats points of other problems like points
// outside its grid.  Two forms: the scaled one (FP64 and plain FP32, below:
// run_batch_scaled) and the normalised one x <- x + d (x_partner - x) with
// per-problem walls (run_batch, run_batch_comp; the compensated path, and
// any launch whose end factor has no table slot).  Every launch starts and
// ends with the normalised state in the buffer.  Two kernels: tbb_kernel
// (CTA rows; FP64 and compensated FP32) and tbb_ws_kernel (plain FP32:
// warp windows fed by a TMA producer warp).

// The per-launch fields of a tile's steps: one launch of a graph of launches,
// or one round of a persistent launch (round_of).
struct BRound {
    int p_first, do_entry, n_mid, do_exit;
    const void *endf;  // scaled form: end factors of this launch length
};

__device__ __forceinline__ BRound launch_round(const TbbParams &P)
{
    return BRound{P.p_first, P.do_entry, P.n_mid, P.do_exit, P.endf};
}

// Round k of a persistent launch of P.steps steps, P.depth per round: the
// same cut into launches as the host's graph of launches (steps n0 = k depth
// onwards; the entry conversion in round 0, the exit in the last).
__device__ __forceinline__ BRound round_of(const TbbParams &P, long long k)
{
    const long long n0 = k * P.depth;
    const long long L = (P.steps - n0 < P.depth) ? P.steps - n0 : P.depth;
    const bool last = k == P.rounds - 1;
    return BRound{(int)(n0 & 1), k == 0 ? 1 : 0, (int)(last ? L - 1 : L), last ? 1 : 0, last ? P.endf_last : P.endf};
}

// Entry, block steps and exit of one tile, normalised form.
template <bool EDGE, typename Real, int K, int NW, bool WT>
__device__ __forceinline__ void run_batch(Real (&v)[K], const TbbParams &P, const BRound &rd,
                                          const BatchDesc &bd, Exch<Real, NW, WT> &x, Span sp)
{
    Real L = 0, R = 0;
    if (rd.do_entry) {
        const StageC<Real> c{(Real)bd.r, (Real)bd.omr, (Real)0, (Real)bd.f_l, (Real)bd.f_r};
        if (((1 - rd.p_first) & 1) == 1) {
            exchange(v, L, R, x);
            stage<1, kEntry, EDGE>(v, L, R, sp, c);
        } else {
            stage<0, kEntry, EDGE>(v, L, R, sp, c);
        }
    }
    const StageC<Real> cm{(Real)bd.d, (Real)0, (Real)bd.kappa, (Real)bd.f_l, (Real)bd.f_r};
    int m = 0;
    if (rd.n_mid > 0 && (rd.p_first & 1)) {
        exchange(v, L, R, x);
        stage<1, kMidN, EDGE>(v, L, R, sp, cm);
        m = 1;
    }
    for (; m + 1 < rd.n_mid; m += 2) {
        stage<0, kMidN, EDGE>(v, L, R, sp, cm);
        exchange(v, L, R, x);
        stage<1, kMidN, EDGE>(v, L, R, sp, cm);
    }
    if (m < rd.n_mid)
        stage<0, kMidN, EDGE>(v, L, R, sp, cm);
    if (rd.do_exit) {
        const StageC<Real> c{(Real)bd.x1, (Real)bd.x2, (Real)bd.xs, (Real)0, (Real)0};
        if (((rd.p_first + rd.n_mid) & 1) == 1) {
            exchange(v, L, R, x);
            stage<1, kExit, EDGE>(v, L, R, sp, c);
        } else {
            stage<0, kExit, EDGE>(v, L, R, sp, c);
        }
    }
}


// Boundary fix-ups of one thread in the batched scaled form, set once per
// tile.  A problem starts on a row boundary and its walls are shifted out,
// so a thread's row is a whole interior run, the problem's first row, its
// last row (followed by padding), or padding of no problem.  Hence at most
// two of its points are singletons (register 0 under grouping 1 in a first
// row, register jhi - 1 whose partner jhi lies past the end).  The padding
// registers (from `keep` on) run the update like the others: no point of a
// problem reads them (both singletons replace the value computed from their
// outside partner), and the write-back leaves padding as the tile loaded it.
struct BatchFix {
    int keep;       // registers keep .. K-1 are padding (K: none)
    int tail;       // jhi - 1: the last point of the problem in this row (-1: none)
    bool head;      // register 0 is the problem's first point
};

template <int K>
__device__ __forceinline__ BatchFix batch_fix(int pid, Span sp)
{
    BatchFix f;
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

// One scaled block step x <- x + g x_partner on a warp that holds problem
// boundaries: every lane runs the one-FMA update, then the lanes that need
// it turn their singletons into x <- kap_s x (a switch on the runtime
// register index of the tail).
#define GE_TBB_SINGLE(J) \
    case J:              \
        if constexpr ((J) < K) nv[J] = kap * v[J]; \
        break;
template <int Q, typename Real, int K>
__device__ __forceinline__ void batch_mid_fixed(Real (&v)[K], Real L, Real R, const BatchFix &f, Real g, Real kap)
{
    Real nv[K];
#pragma unroll
    for (int j = 0; j < K; ++j)
        nv[j] = fma(g, pval<Q>(v, j, L, R), v[j]);
    if (Q == 1 && f.head && f.keep > 0)
        nv[0] = kap * v[0];
    // the last point's partner under grouping Q is tail + 1 when (tail + Q) is even
    if (f.tail >= 0 && ((f.tail + Q) & 1) == 0) {
        switch (f.tail) {
            GE_TBB_SINGLE(0) GE_TBB_SINGLE(1) GE_TBB_SINGLE(2) GE_TBB_SINGLE(3) GE_TBB_SINGLE(4) GE_TBB_SINGLE(5)
            GE_TBB_SINGLE(6) GE_TBB_SINGLE(7) GE_TBB_SINGLE(8) GE_TBB_SINGLE(9) GE_TBB_SINGLE(10) GE_TBB_SINGLE(11)
            GE_TBB_SINGLE(12) GE_TBB_SINGLE(13) GE_TBB_SINGLE(14) GE_TBB_SINGLE(15) GE_TBB_SINGLE(16) GE_TBB_SINGLE(17)
            GE_TBB_SINGLE(18) GE_TBB_SINGLE(19) GE_TBB_SINGLE(20) GE_TBB_SINGLE(21) GE_TBB_SINGLE(22) GE_TBB_SINGLE(23)
            GE_TBB_SINGLE(24) GE_TBB_SINGLE(25) GE_TBB_SINGLE(26) GE_TBB_SINGLE(27) GE_TBB_SINGLE(28) GE_TBB_SINGLE(29)
            GE_TBB_SINGLE(30) GE_TBB_SINGLE(31)
        default:
            break;
        }
    }
#pragma unroll
    for (int j = 0; j < K; ++j)
        v[j] = nv[j];
}
#undef GE_TBB_SINGLE

// One scaled block step: the fast stage inside a problem, the fixed-up one
// on warps that hold boundaries.
template <int Q, bool EDGE, typename Real, int K>
__device__ __forceinline__ void batch_mid(Real (&v)[K], Real L, Real R, Span sp, const BatchFix &f,
                                          const StageC<Real> &cm, const EmuG &eg)
{
    if constexpr (EDGE) {
        batch_mid_fixed<Q>(v, L, R, f, cm.a, cm.s);
    } else if constexpr (sizeof(Real) == 8 && GE_EMU_F64 > 0 && GE_EMU_F64 < K) {
        // FP64 interior warps: GE_EMU_F64 of each thread's updates on the
        // integer pipes (the FP64 unit's bits; the warp falls back if any lane
        // cannot, or if the problem's g is not a normal number)
        stage_mid_hybrid<Q, GE_EMU_F64>(v, L, R, cm.a, eg, emu_g_usable(eg));
    } else {
        stage<Q, kMid, false>(v, L, R, sp, cm);
    }
}

// Compensated block step on a warp that holds problem boundaries (the
// normalised form keeps the walls, so wall terms stay): the interior deltas
// d (x_p - x) on every register, then the thread's (at most two) boundary
// points fixed: a singleton takes (kappa - 1)(x + lo), then the wall terms
// fl at the problem's first point and fr at its last, in the order of the
// checked step; then the Kahan sums.  A problem's points get exactly the
// checked step's deltas; padding registers take garbage and are never
// written back.
#define GE_TBB_COMP_TAIL(J)                                                 \
    case J:                                                                 \
        if constexpr ((J) < K) {                                            \
            if (single)                                                     \
                t[J] = __fmul_rn(km1, v[J] + lo[J]);                        \
            if ((J) == 0 && f.head)                                         \
                t[J] += fl;                                                 \
            t[J] += fr;                                                     \
        }                                                                   \
        break;
template <int Q, int K, int NW, bool WT>
__device__ __forceinline__ void comp_batch_fixed(float (&v)[K], float (&lo)[K], float d, float km1, float fl,
                                                 float fr, Exch<float, NW, WT> &x, const BatchFix &f)
{
    float L = 0.0f, R = 0.0f;
    if (Q == 1)
        exchange(v, L, R, x);
    float t[K];
    if (Q == 0) {
#pragma unroll
        for (int j = 0; j < K; j += 2) {
            const float a = __fmul_rn(d, v[j + 1] - v[j]);
            t[j] = a;
            t[j + 1] = -a;
        }
    } else {
        t[0] = __fmul_rn(d, L - v[0]);
        t[K - 1] = __fmul_rn(d, R - v[K - 1]);
#pragma unroll
        for (int j = 1; j + 1 < K; j += 2) {
            const float a = __fmul_rn(d, v[j + 1] - v[j]);
            t[j] = a;
            t[j + 1] = -a;
        }
    }
    // register 0 is the first point: a singleton under grouping 1 (its
    // partner -1 is outside); a one-point problem is the tail too
    if (Q == 1 && f.head)
        t[0] = __fmul_rn(km1, v[0] + lo[0]);
    if (f.tail >= 0) {
        const bool single = ((f.tail + Q) & 1) == 0;  // partner tail + 1 is outside
        switch (f.tail) {
            GE_TBB_COMP_TAIL(0) GE_TBB_COMP_TAIL(1) GE_TBB_COMP_TAIL(2) GE_TBB_COMP_TAIL(3)
            GE_TBB_COMP_TAIL(4) GE_TBB_COMP_TAIL(5) GE_TBB_COMP_TAIL(6) GE_TBB_COMP_TAIL(7)
            GE_TBB_COMP_TAIL(8) GE_TBB_COMP_TAIL(9) GE_TBB_COMP_TAIL(10) GE_TBB_COMP_TAIL(11)
            GE_TBB_COMP_TAIL(12) GE_TBB_COMP_TAIL(13) GE_TBB_COMP_TAIL(14) GE_TBB_COMP_TAIL(15)
            GE_TBB_COMP_TAIL(16) GE_TBB_COMP_TAIL(17) GE_TBB_COMP_TAIL(18) GE_TBB_COMP_TAIL(19)
            GE_TBB_COMP_TAIL(20) GE_TBB_COMP_TAIL(21) GE_TBB_COMP_TAIL(22) GE_TBB_COMP_TAIL(23)
            GE_TBB_COMP_TAIL(24) GE_TBB_COMP_TAIL(25) GE_TBB_COMP_TAIL(26) GE_TBB_COMP_TAIL(27)
            GE_TBB_COMP_TAIL(28) GE_TBB_COMP_TAIL(29) GE_TBB_COMP_TAIL(30) GE_TBB_COMP_TAIL(31)
        default:
            break;
        }
    }
    if (f.head && f.tail != 0)
        t[0] += fl;
#pragma unroll
    for (int j = 0; j < K; ++j)
        kahan_add(v[j], lo[j], t[j]);
}
#undef GE_TBB_COMP_TAIL

template <int Q, bool EDGE, int K, int NW, bool WT>
__device__ __forceinline__ void comp_batch_step(float (&v)[K], float (&lo)[K], const TbParams &dummy, float d,
                                                float km1, float fl, float fr, Exch<float, NW, WT> &x, Span sp,
                                                const BatchFix &f)
{
    if constexpr (EDGE)
        comp_batch_fixed<Q>(v, lo, d, km1, fl, fr, x, f);
    else
        mid_comp<Q, false>(v, lo, dummy, d, km1, fl, fr, x, sp);
}

template <bool EDGE, int K, int NW, bool WT>
__device__ __forceinline__ void run_batch_comp(float (&v)[K], const TbbParams &P, const BatchDesc &bd, int pid,
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
    if constexpr (!EDGE && K % 4 == 0) {
        // interior warps: the same steps on register pairs (the same bits)
        comp_steps_pairs(v, P.p_first, P.n_mid, (float)bd.d, x);
    } else {
    float lo[K];
#pragma unroll
    for (int j = 0; j < K; ++j)
        lo[j] = 0.0f;
    const float d = (float)bd.d, km1 = (float)(bd.kappa - 1.0);
    const float fl = (float)bd.f_l, fr = (float)bd.f_r;
    TbParams dummy{};
    dummy.n = 0;
    const BatchFix fx = batch_fix<K>(pid, sp);
    int m = 0;
    if (P.n_mid > 0 && (P.p_first & 1)) {
        comp_batch_step<1, EDGE>(v, lo, dummy, d, km1, fl, fr, x, sp, fx);
        m = 1;
    }
    for (; m + 1 < P.n_mid; m += 2) {
        comp_batch_step<0, EDGE>(v, lo, dummy, d, km1, fl, fr, x, sp, fx);
        comp_batch_step<1, EDGE>(v, lo, dummy, d, km1, fl, fr, x, sp, fx);
    }
    if (m < P.n_mid)
        comp_batch_step<0, EDGE>(v, lo, dummy, d, km1, fl, fr, x, sp, fx);
#pragma unroll
    for (int j = 0; j < K; ++j)
        v[j] += lo[j];
    }
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
// Only points inside the problem are written back: padding keeps its values.
template <bool EDGE, typename Real, int K, int NW, bool WT>
__device__ __forceinline__ void run_batch_scaled(Real (&v)[K], const TbbParams &P, const BRound &rd, const BatchDesc &bd,
                                                 int pid, long long g0, Exch<Real, NW, WT> &x, Span sp)
{
    Real L = 0, R = 0;
    const Real ua = (Real)bd.ustar_a, ub = (Real)bd.ustar_b;
    // grid position j + 1 of register 0: one 64-bit conversion (the FP64 pipe)
    // per thread, the registers' positions by exact small additions
    const Real p1 = (Real)(g0 + 1);
    if (rd.do_entry) {
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (!EDGE || (j >= sp.jlo && j < sp.jhi))
                v[j] -= ua + ub * (p1 + (Real)j);
        const StageC<Real> c{(Real)bd.r, (Real)bd.omr, (Real)0, (Real)0, (Real)0};
        if (((1 - rd.p_first) & 1) == 1) {
            exchange(v, L, R, x);
            stage<1, kEntry, EDGE>(v, L, R, sp, c);
        } else {
            stage<0, kEntry, EDGE>(v, L, R, sp, c);
        }
    }
    const StageC<Real> cm{(Real)bd.g, (Real)0, (Real)bd.kap_s, (Real)0, (Real)0};
    const BatchFix fx = batch_fix<K>(pid, sp);
    // an interior (non-edge) warp holds rows of one problem only: lane 0's g
    // is the warp's (the edge path does not use it)
    const EmuG eg = emu_g(__shfl_sync(0xffffffffu, bd.g, 0));
    if constexpr (!EDGE && sizeof(Real) == 4 && K % 4 == 0) {
        // interior FP32 warps: the same steps and rescalings on register
        // pairs (packed FMAs; the same bits)
        constexpr int H = K / 2;
        uint64_t pr[H];
        to_pairs(v, pr);
        const uint64_t g2 = f2((float)cm.a, (float)cm.a);
        int m = 0, q = 0;
        while (m < rd.n_mid) {
            const int cnt = (rd.n_mid - m < P.R) ? rd.n_mid - m : P.R;
            int i = 0;
            if (((rd.p_first + m) & 1) == 1) {
                exchange_ends(f2_split(pr[0]).x, f2_split(pr[H - 1]).y, L, R, x);
                pair_mid<1>(pr, L, R, g2);
                i = 1;
            }
            for (; i + 1 < cnt; i += 2) {
                pair_mid<0>(pr, L, R, g2);
                exchange_ends(f2_split(pr[0]).x, f2_split(pr[H - 1]).y, L, R, x);
                pair_mid<1>(pr, L, R, g2);
            }
            if (i < cnt)
                pair_mid<0>(pr, L, R, g2);
            m += cnt;
            if (cnt == P.R) {
                const int e = pid >= 0 ? P.exps[(long long)pid * P.Q + q] : 0;
                const float sc = pow2neg<float>(e);
                const uint64_t s2 = f2(sc, sc);
#pragma unroll
                for (int j = 0; j < H; ++j)
                    pr[j] = f2_mul(pr[j], s2);
            }
            ++q;
        }
        from_pairs(pr, v);
    } else {
    int m = 0, q = 0;
    while (m < rd.n_mid) {
        const int cnt = (rd.n_mid - m < P.R) ? rd.n_mid - m : P.R;
        int i = 0;
        if (((rd.p_first + m) & 1) == 1) {
            exchange(v, L, R, x);
            batch_mid<1, EDGE>(v, L, R, sp, fx, cm, eg);
            i = 1;
        }
        for (; i + 1 < cnt; i += 2) {
            batch_mid<0, EDGE>(v, L, R, sp, fx, cm, eg);
            exchange(v, L, R, x);
            batch_mid<1, EDGE>(v, L, R, sp, fx, cm, eg);
        }
        if (i < cnt)
            batch_mid<0, EDGE>(v, L, R, sp, fx, cm, eg);
        m += cnt;
        if (cnt == P.R) {
            // every lane takes part (the FP64 form decides warp-wide); a lane
            // of no problem scales nothing
            const int e = pid >= 0 ? P.exps[(long long)pid * P.Q + q] : 0;
            scale_pow2<!EDGE>(v, e, pid >= 0 ? sp.jlo : 0, pid >= 0 ? sp.jhi : 0);
        }
        ++q;
    }
    }
    if (pid >= 0) {
        Real fh, fl;
        if constexpr (sizeof(Real) == 4) {
            const float2 f = reinterpret_cast<const float2 *>(rd.endf)[pid];
            fh = f.x, fl = f.y;
        } else {
            fh = reinterpret_cast<const double *>(rd.endf)[pid];
            fl = 0;
        }
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (!EDGE || (j >= sp.jlo && j < sp.jhi))
                v[j] = fma(v[j], fh, v[j] * fl);
    }
    if (rd.do_exit) {
        const StageC<Real> c{(Real)bd.x1, (Real)bd.x2, (Real)bd.xs, (Real)0, (Real)0};
        if (((rd.p_first + rd.n_mid) & 1) == 1) {
            exchange(v, L, R, x);
            stage<1, kExit, EDGE>(v, L, R, sp, c);
        } else {
            stage<0, kExit, EDGE>(v, L, R, sp, c);
        }
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (!EDGE || (j >= sp.jlo && j < sp.jhi))
                v[j] += ua + ub * (p1 + (Real)j);
    }
}

// Batched kernel for FP64 and compensated FP32: CTA rows (thread t holds
// tile row t; warp edges exchange through shared memory).  TR: rows per tile
// (= threads), a geometry the plan's autotuner picks (256: 2 CTAs per SM,
// 128: 4).  Plain FP32 runs the warp-specialised warp-window kernel below.
template <typename Real, bool COMP, int TR>
__global__ void __launch_bounds__(TR, TR == 256 ? 2 : 4)
    tbb_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ TbbParams P)
{
    constexpr bool WT = false;
    constexpr int NT = TR;
    constexpr int K = kRowBytes / (int)sizeof(Real);
    constexpr int NW = NT / 32;
    constexpr int CH = kRowBytes / 16;
    constexpr uint32_t kTileBytes = TR * kRowBytes;

    extern __shared__ unsigned char smem_raw[];
    unsigned char *tiles = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    __shared__ __align__(8) uint64_t mbar[3];  // two tile buffers, and one nothing arrives on
    __shared__ Real slot[2][NW][2];

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int hr = P.H / K, ur = P.U / K;
    const int my_row = t;  // CTA rows: thread t holds tile row t
    Exch<Real, NW, WT> x{slot, 0, lane, warp};

    if (t == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        mbar_init(&mbar[2], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // tiles come from the launch's dynamic queue in order (tiles with checked
    // warps are everywhere in a batch): thread 0 takes the next one while the
    // current tile is computed
    __shared__ long long s_next;
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

        Real v[K];
        {
            const unsigned char *rp = cur + my_row * kRowBytes;
#pragma unroll
            for (int c = 0; c < CH; ++c)
                chunk_to_regs<K>(rp + ((c ^ (my_row & 7)) << 4), v, c);
        }
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
            const BRound rd = launch_round(P);
            if (P.scaled) {
                if (edge_warp)
                    run_batch_scaled<true>(v, P, rd, bd, pid, g0, x, sp);
                else
                    run_batch_scaled<false>(v, P, rd, bd, pid, g0, x, sp);
            } else if (edge_warp) {
                run_batch<true>(v, P, rd, bd, x, sp);
            } else {
                run_batch<false>(v, P, rd, bd, x, sp);
            }
        } else {
            if (edge_warp)
                run_batch_comp<true>(v, P, bd, pid, x, sp);
            else
                run_batch_comp<false>(v, P, bd, pid, x, sp);
        }

        {
            unsigned char *rp = cur + my_row * kRowBytes;
            if (!edge_thr) {
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    regs_to_chunk<K>(rp + ((c ^ (my_row & 7)) << 4), v, c);
            } else {
                // only the points of the thread's problem: padding and rows of
                // no problem keep the values the tile loaded
                constexpr int PER = 16 / (int)sizeof(Real);
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    Real *q = reinterpret_cast<Real *>(rp + ((c ^ (my_row & 7)) << 4));
#pragma unroll
                    for (int i = 0; i < PER; ++i) {
                        const int j = c * PER + i;
                        if (pid >= 0 && j >= sp.jlo && j < sp.jhi)
                            q[i] = v[j];
                    }
                }
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
        tile = next_tile;
    }
}

// Plain FP32 batches, warp-specialised: one producer warp takes tiles from
// the launch's queue and loads them by TMA into two shared buffers; eight
// consumer warps each advance their window of the tile (warp windows carry
// their own halo, so the steps need no CTA barrier) and write their output
// rows out through their own staging rows.  The warps meet only at the
// buffers: `full` (the tile landed) and `empty` (all eight consumers have
// read it), so a warp that holds problem boundaries and runs longer holds
// back the reuse of a buffer, a tile later, not the other warps' next tile.
// (With one CTA barrier per tile the FP32 batch spent most stalls there.)
// TR: rows per tile, a geometry the plan's autotuner picks (256: eight
// consumer warps, 2 CTAs per SM; 128: four, 4 CTAs per SM).
constexpr int kWsStageBytes = 32 * kRowBytes;      // staging rows of one consumer warp
template <int TR>
struct Ws {
    static constexpr int kConsumers = TR / 32;     // consumer warps
    static constexpr int kThreads = TR + 32;       // plus the producer warp
    static constexpr int kMinBlocks = TR == 256 ? 2 : 4;
    // the persistent kernel's round bookkeeping needs more registers: with
    // 128-row tiles it runs 3 CTAs per SM (at 4 it spilled and ran slower)
    static constexpr int kMinBlocksPersist = TR == 256 ? 2 : 3;
    static int smem_bytes() { return 2 * TR * kRowBytes + kConsumers * kWsStageBytes + 1024; }
};

// Acquire load of a device-wide counter (another CTA's release publishes it).
__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// PERSIST: the whole solve in one launch.  Work items are (round k, tile i),
// k = 0 .. P.rounds - 1, claimed in order from the launch's queue (so every
// item of round k is claimed before any of round k + 1).  Round k reads
// buffer k & 1 (tensor map tmap[k & 1]) and writes P.outs[k & 1]; the
// producer loads item (k, i) only once tiles i - 1, i, i + 1 of round k - 1
// are done.  Completion: the consumer warps arrive on the shared barrier
// stored[b] after their stores of the item in buffer b; the producer lane
// (otherwise idle) waits for it, fences at GPU scope (the consumers' stores,
// seen through the barrier, are ordered before it) and adds NW to
// P.done[tile], so round k of tile i is done at done[i] >= (k + 1) NW.  The
// producer posts what it owes whenever it can, and always before it blocks
// on a dependency, so no wait of it is on its own CTA.  The dependency order
// also keeps every write after the reads of the buffer it overwrites (round
// k + 1 writes buffer k & 1, which round k read).  CTAs take items only once
// running, so the smallest unfinished item always has its inputs: no wait
// is circular.  Every wait is bounded; a timeout is recorded in P.err, which
// every dependency wait also watches, and the producer then hands its
// consumers the end marker.
template <int TR, bool PERSIST>
__global__ void __launch_bounds__(Ws<TR>::kThreads, PERSIST ? Ws<TR>::kMinBlocksPersist : Ws<TR>::kMinBlocks)
    tbb_ws_kernel(const __grid_constant__ CUtensorMap tmap0, const __grid_constant__ CUtensorMap tmap1,
                  const __grid_constant__ TbbParams P)
{
    using Real = float;
    constexpr bool WT = true;
    constexpr int K = kRowBytes / (int)sizeof(Real);
    constexpr int NW = Ws<TR>::kConsumers;
    constexpr int CH = kRowBytes / 16;
    constexpr uint32_t kTileBytes = TR * kRowBytes;

    extern __shared__ unsigned char smem_raw[];
    unsigned char *tiles = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
    unsigned char *stage_all = tiles + 2 * kTileBytes;
    __shared__ __align__(8) uint64_t full[2], empty[2], stored[4], never;
    __shared__ long long tile_of[2];
    __shared__ Real slot[2][NW][2];  // unused with warp windows (Exch needs the type)

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int hr = P.H / K, ur = P.U / K;
    const long long limit = P.stall > 0 ? P.stall : kWaitLimitCycles;
    const long long items = PERSIST ? (long long)P.rounds * P.n_tiles : P.n_tiles;

    if (t == 0) {
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
        mbar_init(&empty[0], NW);
        mbar_init(&empty[1], NW);
        for (int i = 0; i < 4; ++i)
            mbar_init(&stored[i], NW);
        mbar_init(&never, 1);
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == NW) {
        // producer: lane 0 issues, the other lanes leave
        if (lane != 0)
            return;
        long long issued[2] = {-1, -1};  // iteration of the last copy into each buffer
        // persistent launch: items handed out but not yet published (their
        // iterations sig .. it - 1, tiles in sig_tile by iteration mod 4)
        long long sig = 0;
        int sig_tile[4] = {0, 0, 0, 0};
        // publish iteration j: its consumers' stores (seen through
        // stored[j & 3]) and then the tile's count, released at GPU scope
        auto publish = [&](long long j, bool block) -> bool {
            const int bj = (int)(j & 3);
            const uint32_t ph = (uint32_t)((j >> 2) & 1);
            if (block ? !mbar_wait_backoff(&stored[bj], ph, kWaitLimitCycles) : !mbar_try_wait(&stored[bj], ph))
                return false;
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
            atomicAdd(P.done + sig_tile[bj], NW);
            return true;
        };
        bool failed = false;
        for (long long it = 0;; ++it) {
            const int b = (int)(it & 1);
            if (PERSIST) {
                // iteration it - 4 (the last one on stored[it & 3]) is
                // published before iteration it is handed out: that barrier
                // then never runs two phases ahead of what the producer has
                // seen (the consumers are two items behind at most, so this
                // hardly ever waits)
                bool okp = true;
                while (okp && sig <= it - 4) {
                    okp = publish(sig, true);
                    sig += okp ? 1 : 0;
                }
                if (!okp) {
                    atomicExch(P.err, kDevTimeout);
                    tile_of[b] = -1;
                    mbar_arrive(&full[b]);
                    if (issued[b ^ 1] == it - 1)
                        mbar_wait_bounded(&full[b ^ 1], (uint32_t)(((it - 1) >> 1) & 1), kWaitLimitCycles);
                    return;
                }
                while (sig < it && publish(sig, false))
                    ++sig;
            }
            if (it >= 2 && !mbar_wait_backoff(&empty[b], (uint32_t)(((it - 2) >> 1) & 1), limit)) {
                atomicExch(P.err, kDevTimeout);
                // let this CTA's own copies in flight land before it leaves
                for (int q = 0; q < 2; ++q)
                    if (issued[q] >= 0)
                        mbar_wait_bounded(&full[q], (uint32_t)((issued[q] >> 1) & 1), kWaitLimitCycles);
                return;
            }
            long long q;
            if (PERSIST)
                q = atomicAdd(P.tile_ctr, 1);  // only running CTAs hold items
            else
                q = it == 0 ? (long long)blockIdx.x : (long long)gridDim.x + atomicAdd(P.tile_ctr, 1);
            const long long k = PERSIST ? q / P.n_tiles : 0;
            const long long tile = q - k * P.n_tiles;
            bool ok = q < items;
            if (ok && PERSIST && k > 0) {
                // inputs of (k, tile): tiles tile - 1 .. tile + 1 of round k - 1
                const int need = (int)(k * NW);
                const long long jlo = tile > 0 ? tile - 1 : 0;
                const long long jhi = tile + 1 < P.n_tiles ? tile + 1 : P.n_tiles - 1;
                bool ready = true;
                for (long long j = jlo; j <= jhi; ++j)
                    ready = ready && ld_acquire(P.done + j) >= need;
                if (!ready) {
                    // before blocking: publish everything this CTA owes
                    while (ok && sig < it) {
                        ok = publish(sig, true);
                        sig += ok ? 1 : 0;
                    }
                    const long long t0 = clock64();
                    for (long long j = jlo; ok && j <= jhi; ++j) {
                        while (ld_acquire(P.done + j) < need) {
                            if (*(volatile int *)P.err != 0 || clock64() - t0 > limit) {
                                ok = false;
                                break;
                            }
                            __nanosleep(64);
                        }
                    }
                    if (!ok) {
                        atomicExch(P.err, kDevTimeout);
                        failed = true;
                    }
                }
                // the generic-proxy stores of those tiles, seen by this
                // thread, before its TMA (async proxy) reads them
                asm volatile("fence.proxy.async.global;" ::: "memory");
            }
            if (!ok) {
                tile_of[b] = -1;  // no more items: the consumers leave
                mbar_arrive(&full[b]);
                // the copy of the previous item may still be landing (the one
                // before it was read before empty[b] completed)
                if (issued[b ^ 1] == it - 1)
                    mbar_wait_bounded(&full[b ^ 1], (uint32_t)(((it - 1) >> 1) & 1), kWaitLimitCycles);
                // what this CTA still owes (its consumers finish their items)
                while (PERSIST && !failed && sig < it && publish(sig, true))
                    ++sig;
                return;
            }
            tile_of[b] = q;
            if (PERSIST)
                sig_tile[it & 3] = (int)tile;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&full[b], kTileBytes);
            tma_load_rows(tiles + b * kTileBytes, (k & 1) ? &tmap1 : &tmap0, &full[b], (int)(tile * ur - hr));
            issued[b] = it;
        }
    }

    // consumers: warp w owns the window of rows w (32 - 2 hr) .. + 31
    const int my_row = warp * (32 - 2 * hr) + lane;
    const bool writes = lane >= hr && lane < 32 - hr;
    const int out_rows = 32 - 2 * hr;      // this warp's output rows
    const int row_local = lane - hr;       // this lane's output row in the staging rows
    unsigned char *stage = stage_all + warp * kWsStageBytes;
    Exch<Real, NW, WT> x{slot, 0, lane, warp};
    for (long long it = 0;; ++it) {
        const int b = (int)(it & 1);
        if (!tile_wait(full, &never, b, it, P.stall)) {
            if (lane == 0)
                atomicExch(P.err, kDevTimeout);
            return;
        }
        const long long q = tile_of[b];
        if (q < 0)
            return;
        // round and tile (both fit 32 bits: tiles < 2^31, rounds <= steps)
        const int k = PERSIST ? (int)(q / P.n_tiles) : 0;
        const int tile = (int)(q - (long long)k * P.n_tiles);
        const BRound rd = PERSIST ? round_of(P, k) : launch_round(P);
        const unsigned char *cur = tiles + b * kTileBytes;
        Real v[K];
        {
            const unsigned char *rp = cur + my_row * kRowBytes;
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const unsigned char *src = rp + ((c ^ (my_row & 7)) << 4);
                chunk_to_regs<K>(src, v, c);
                // the loaded row, so that padding goes back unchanged
                if (writes)
                    *reinterpret_cast<uint4 *>(stage + row_local * kRowBytes + ((c ^ (row_local & 7)) << 4)) =
                        *reinterpret_cast<const uint4 *>(src);
            }
        }
        __syncwarp();
        if (lane == 0)
            mbar_arrive(&empty[b]);  // this warp is done with the buffer

        const long long grow = (long long)tile * ur - hr + my_row;
        const int pid = (grow >= 0 && grow < P.n_rows) ? __ldg(P.row_pid + grow) : -1;
        BatchDesc bd{};
        Span sp{K + 1, K + 1};
        if (pid >= 0) {
            bd = P.desc[pid];
            sp = make_span<K>(grow * K - bd.off, bd.n);
        }
        const bool edge_thr = !(sp.jlo <= -1 && sp.jhi >= K + 1);
        const bool edge_warp = __any_sync(0xffffffffu, edge_thr);
        const long long g0 = pid >= 0 ? grow * K - bd.off : 0;
        if (P.scaled) {
            if (edge_warp)
                run_batch_scaled<true>(v, P, rd, bd, pid, g0, x, sp);
            else
                run_batch_scaled<false>(v, P, rd, bd, pid, g0, x, sp);
        } else if (edge_warp) {
            run_batch<true>(v, P, rd, bd, x, sp);
        } else {
            run_batch<false>(v, P, rd, bd, x, sp);
        }

        if (writes) {
            unsigned char *rp = stage + row_local * kRowBytes;
            if (!edge_thr) {
#pragma unroll
                for (int c = 0; c < CH; ++c)
                    regs_to_chunk<K>(rp + ((c ^ (row_local & 7)) << 4), v, c);
            } else {
                // only the points of the thread's problem
#pragma unroll
                for (int c = 0; c < CH; ++c) {
                    Real *qp = reinterpret_cast<Real *>(rp + ((c ^ (row_local & 7)) << 4));
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int j = c * 4 + i;
                        if (pid >= 0 && j >= sp.jlo && j < sp.jhi)
                            qp[i] = v[j];
                    }
                }
            }
        }
        __syncwarp();
        {
            const long long grow0 = (long long)tile * ur + (long long)warp * out_rows;
            unsigned char *out = static_cast<unsigned char *>(PERSIST ? P.outs[k & 1] : P.out);
            for (int ch = lane; ch < out_rows * CH; ch += 32) {
                const int lr = ch / CH, c = ch % CH;
                const long long gr = grow0 + lr;
                if (gr < P.n_rows && warp * out_rows + lr < ur)
                    *reinterpret_cast<uint4 *>(out + gr * kRowBytes + c * 16) =
                        *reinterpret_cast<const uint4 *>(stage + lr * kRowBytes + ((c ^ (lr & 7)) << 4));
            }
        }
        __syncwarp();
        if (PERSIST && lane == 0)
            mbar_arrive(&stored[it & 3]);  // this warp's stores of the item (the producer publishes)
    }
}

constexpr int rows_smem_bytes(int tr) { return 2 * tr * kRowBytes + 1024; }

template <typename Real, bool COMP, int TR>
cudaError_t launch_batch_one(const void *tmap, const TbbParams &p, int grid, cudaStream_t s)
{
    const CUtensorMap *m = static_cast<const CUtensorMap *>(tmap);
    tbb_kernel<Real, COMP, TR><<<grid, TR, rows_smem_bytes(TR), s>>>(*m, p);
    return cudaGetLastError();
}

template <typename Real, bool COMP, int TR>
cudaError_t batch_attr_and_occupancy(int *blocks)
{
    cudaError_t e = cudaFuncSetAttribute(tbb_kernel<Real, COMP, TR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, rows_smem_bytes(TR));
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, tbb_kernel<Real, COMP, TR>, TR,
                                                         rows_smem_bytes(TR));
}

template <int TR>
cudaError_t ws_attr_and_occupancy(int *blocks)
{
    cudaError_t e = cudaFuncSetAttribute(tbb_ws_kernel<TR, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Ws<TR>::smem_bytes());
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, tbb_ws_kernel<TR, false>, Ws<TR>::kThreads,
                                                         Ws<TR>::smem_bytes());
}

template <int TR>
cudaError_t ws_persist_occupancy(int *blocks)
{
    cudaError_t e = cudaFuncSetAttribute(tbb_ws_kernel<TR, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         Ws<TR>::smem_bytes());
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, tbb_ws_kernel<TR, true>, Ws<TR>::kThreads,
                                                         Ws<TR>::smem_bytes());
}

template <int TR>
cudaError_t launch_ws(const void *tmap, const void *tmap_other, const TbbParams &p, int grid, cudaStream_t s)
{
    const CUtensorMap *m0 = static_cast<const CUtensorMap *>(tmap);
    const CUtensorMap *m1 = static_cast<const CUtensorMap *>(tmap_other ? tmap_other : tmap);
    if (p.rounds > 1)
        tbb_ws_kernel<TR, true><<<grid, Ws<TR>::kThreads, Ws<TR>::smem_bytes(), s>>>(*m0, *m1, p);
    else
        tbb_ws_kernel<TR, false><<<grid, Ws<TR>::kThreads, Ws<TR>::smem_bytes(), s>>>(*m0, *m1, p);
    return cudaGetLastError();
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

// 1 + g as a double-double, g the coefficient the kernel holds: FP64
// (mode 0), rounded to FP32 (1), the double-float pair (2).
__device__ __forceinline__ void growth_dev(const BatchDesc &d, int mode, double &gh, double &gl)
{
    const double g = mode == 1 ? (double)__double2float_rn(d.g)
                               : (mode == 2 ? __dadd_rn((double)d.dfc[0][0], (double)d.dfc[0][1]) : d.g);
    gh = __dadd_rn(1.0, g);
    gl = __dadd_rn(__dsub_rn(1.0, gh), g);  // exact: 1 + g == gh + gl
}

// exps[b][q]: after block q of R steps (scale starting at 1) the scale is
// brought back into [1, 2) by 2^-exps[b][q].
__global__ void batch_exps_kernel(const BatchDesc *__restrict__ desc, int np, int R, int Q, int mode,
                                  short *__restrict__ exps)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= np)
        return;
    double gh, gl, sh = 1.0, sl = 0.0;
    growth_dev(desc[b], mode, gh, gl);
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
// float2 (hi, lo) on the FP32 and double-float paths, double on the FP64 path.
__global__ void batch_endf_kernel(const BatchDesc *__restrict__ desc, const short *__restrict__ exps, int np, int R,
                                  int Q, int n_mid, int mode, void *endf)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= np)
        return;
    double gh, gl, sh = 1.0, sl = 0.0;
    growth_dev(desc[b], mode, gh, gl);
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
    if (mode != 0) {
        const float hi = __double2float_rn(inv);
        reinterpret_cast<float2 *>(endf)[b] = make_float2(hi, __double2float_rn(__dsub_rn(inv, (double)hi)));
    } else {
        reinterpret_cast<double *>(endf)[b] = inv;
    }
}

// status[b] = GE_ENONFINITE (5) when a value of problem b is NaN or Inf
// (status zeroed by the caller); one thread per 128-byte row.
template <typename Real>
__global__ void batch_check_kernel(const Real *__restrict__ u, const int *__restrict__ row_pid,
                                   const BatchDesc *__restrict__ desc, long long n_rows, int *__restrict__ status)
{
    constexpr int K = kRowBytes / (int)sizeof(Real);
    for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < n_rows;
         row += (long long)gridDim.x * blockDim.x) {
        const int pid = row_pid[row];
        if (pid < 0)
            continue;
        const long long lo = desc[pid].off, hi = lo + desc[pid].n;
        bool bad = false;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const long long e = row * K + j;
            if (e >= lo && e < hi && !isfinite(u[e]))
                bad = true;
        }
        if (bad)
            atomicExch(&status[pid], 5);
    }
}

}  // namespace

cudaError_t batch_check(int prec, const void *u, const int *row_pid, const BatchDesc *desc, long long n_rows,
                        int *status, cudaStream_t s)
{
    long long blocks = (n_rows + 255) / 256;
    if (blocks > 4096)
        blocks = 4096;
    if (prec == 0)
        batch_check_kernel<double><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const double *>(u), row_pid, desc,
                                                                    n_rows, status);
    else
        batch_check_kernel<float><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const float *>(u), row_pid, desc,
                                                                   n_rows, status);
    return cudaGetLastError();
}

cudaError_t batch_exps(const BatchDesc *desc, int n_problems, int R, int Q, int mode, short *exps, cudaStream_t s)
{
    batch_exps_kernel<<<(n_problems + 127) / 128, 128, 0, s>>>(desc, n_problems, R, Q, mode, exps);
    return cudaGetLastError();
}

cudaError_t batch_endf(const BatchDesc *desc, const short *exps, int n_problems, int R, int Q, int n_mid, int mode,
                       void *endf, cudaStream_t s)
{
    batch_endf_kernel<<<(n_problems + 127) / 128, 128, 0, s>>>(desc, exps, n_problems, R, Q, n_mid, mode, endf);
    return cudaGetLastError();
}

bool tbb_geometry(int prec, int tile_rows, int reach, int *H, int *U)
{
    const int K = kRowBytes / (prec == 0 ? 8 : 4);
    const int ht = (reach + K - 1) / K;
    const bool wt = prec == 1;  // plain FP32: tbb_ws_kernel's warp windows
    if (tile_rows != 128 && tile_rows != 256)
        return false;
    *H = ht * K;
    if (wt) {
        if (2 * ht >= 32)
            return false;
        *U = (tile_rows / 32) * (32 - 2 * ht) * K;
        return true;
    }
    *U = tile_rows * K - 2 * *H;
    return *U > 0;
}

int tbb_max_depth(int prec, int tile_rows)
{
    int H, U, d = kMaxTableSteps;
    while (d > 1 && !tbb_geometry(prec, tile_rows, d + 2, &H, &U))
        --d;
    return d;
}

cudaError_t tbb_occupancy(int prec, int tile_rows, int *blocks)
{
    if (prec == 1)
        return tile_rows == 128 ? ws_attr_and_occupancy<128>(blocks) : ws_attr_and_occupancy<256>(blocks);
    if (prec == 0)
        return tile_rows == 128 ? batch_attr_and_occupancy<double, false, 128>(blocks)
                                : batch_attr_and_occupancy<double, false, 256>(blocks);
    return tile_rows == 128 ? batch_attr_and_occupancy<float, true, 128>(blocks)
                            : batch_attr_and_occupancy<float, true, 256>(blocks);
}

cudaError_t tbb_persist_occupancy(int tile_rows, int *blocks)
{
    return tile_rows == 128 ? ws_persist_occupancy<128>(blocks) : ws_persist_occupancy<256>(blocks);
}

cudaError_t launch_tbb(int prec, int tile_rows, const void *tmap, const TbbParams &p, int grid, cudaStream_t s,
                       const void *tmap_other)
{
    if (prec == 1)
        return tile_rows == 128 ? launch_ws<128>(tmap, tmap_other, p, grid, s)
                                : launch_ws<256>(tmap, tmap_other, p, grid, s);
    if (p.rounds > 1)
        return cudaErrorInvalidValue;  // one launch per round for the other kernels
    if (prec == 0)
        return tile_rows == 128 ? launch_batch_one<double, false, 128>(tmap, p, grid, s)
                                : launch_batch_one<double, false, 256>(tmap, p, grid, s);
    return tile_rows == 128 ? launch_batch_one<float, true, 128>(tmap, p, grid, s)
                            : launch_batch_one<float, true, 256>(tmap, p, grid, s);
}

}  // namespace ge
