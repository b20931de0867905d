// ge_internal.h -- parameter blocks and launcher prototypes shared by the C ABI
// (ge_api.cpp, host compiler) and the kernel translation units (*.cu, nvcc).
// Plain C++: no device code, no CUDA headers beyond the runtime API.
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime_api.h>
#include <nvtx3/nvToolsExt.h>

namespace ge {

// Bytes of one shared-memory / tensor-map row; a thread of the tiled kernels
// owns exactly one row: 32 floats or 16 doubles.
constexpr int kRowBytes = 128;
// Rows of 128 bytes in one tile of the tiled kernels (8192 floats or 4096
// doubles), the box of their 2D TMA load.
constexpr int kTileRows = 256;

// NVTX range around a library call (visible in Nsight timelines; a no-op
// when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Headroom (in powers of two) of the scaled forms' data between rescalings:
// data magnitudes up to about 2^(largest exponent - headroom) are safe.
#ifndef GE_F32_HEADROOM
#define GE_F32_HEADROOM 64.0
#endif
constexpr double kF64Headroom = 256.0;

// Built-in steps per launch of the tiled kernels (FP64, FP32 and compensated
// FP32, double-float), measured best on N = 2^24, r = 2.
constexpr int kDefaultDepthF64 = 48;
constexpr int kDefaultDepthF32 = 128;
constexpr int kDefaultDepthDf = 96;

// Device error codes written to the context's error word.
enum DevErr : int { kDevOk = 0, kDevTimeout = 1 };

// Limit of a tile load wait in the tiled kernels: about 2 s of SM clock.
constexpr long long kWaitLimitCycles = 4000000000LL;

// Coefficients of the literal step (Eqs. (cc)/(dd), (aa)/(bb)), FP64 on the
// host; the FP32 kernels round them once.
struct CanonCoef {
    double c1, c2, c3, c4;  // (r+r^2, 1-r^2, r-r^2, r^2) / (1+2r)
    double s0, s1;          // r/(1+r), (1-r)/(1+r)
    double beta_l, beta_r;
};

// Most exact power-of-two rescalings one tiled launch may apply.
constexpr int kMaxRescale = 64;
// Most block steps one tiled launch may take.
constexpr int kMaxTableSteps = 512;

// One launch of the tiled right-hand-side kernel (GE_KERNEL_TEMPORAL and
// GE_KERNEL_ONESTEP).  See ge_tb.cu for the stage definitions.
//
// Scale bookkeeping (plain and FP64 kernels): the carried right-hand side is
// held as W = sigma * w.  Each block step multiplies sigma by (1 + 2r); every
// `rescale_every` block steps of a ge_step_n call the data and sigma are
// multiplied by the exact power of two 2^-rs_exp[k] (k-th rescaling of this
// launch).  The host runs the same double-precision sigma recurrence as the
// kernel's wall threads, so it knows sigma at the end of every launch: the
// next launch starts from it (`sigma_in`) and the exit coefficients carry
// 1/sigma.  Only warps that hold a wall point evaluate sigma in the kernel.
struct TbParams {
    void *out;            // destination buffer (element 0 = interior point 0)
    int *err;             // device error word
    long long n;          // interior points
    long long n_rows;     // 128-byte rows in each buffer (n_rows * K >= n)
    long long n_tiles;    // tiles of U output elements
    int U;                // output elements per tile (multiple of K)
    int H;                // halo elements per side (multiple of K, >= reach)
    long long stall;      // diagnostic: > 0 makes every tile wait poll a barrier nothing
                          // arrives on for this many cycles (the timeout path runs)
    int p_first;          // parity of the first step of this launch
    int do_entry;         // convert u -> w at the start
    int n_mid;            // block steps w_n -> w_{n+1} in this launch
    int do_exit;          // convert w -> u at the end
    int rescale_every;    // block steps between rescalings (0: never)
    int rescale_phase;    // block steps until the first rescaling of this launch
    double sigma_in;      // scale of the incoming right-hand side
    double onepg;         // 1 + 2r
    double g;             // 2r  (scaled block: (x, y) -> (x + 2r y, 2r x + y))
    double r, omr;        // r, 1 - r  (entry: w = (1-r) u + r u_partner)
    double kappa;         // singleton block factor: scaled (1+2r)(1-r)/(1+r);
                          // compensated kernel: (1-r)/(1+r)
    double d;             // compensated kernel: 2r/(1+2r)
    double f_l, f_r;      // wall terms r*beta_l, r*beta_r (unscaled)
    double x1, x2, xs;    // exit: (1+r)/(1+2r), r/(1+2r), 1/(1+r), each / sigma_end
    short rs_exp[kMaxRescale];  // exponents of this launch's rescalings
    // double-float kernel (ge_tb_df.cu) only
    int df_in;            // the source holds doubles (split on load), else (hi, lo) float pairs
    int df_out;           // write doubles, else (hi, lo) float pairs
    int df_gl;            // the pair of g = 2r has a nonzero low part
    const int *df_code;   // prescale exponent word written by df_prescale
    int *tile_ctr;        // dynamic tile queue: zero at the launch's start; CTA b takes
                          // queue position b first, then gridDim.x + atomicAdd(tile_ctr, 1)
    int emu;              // FP64: part of the interior updates on the integer pipes (1) or
                          // every update on the FP64 unit (0); the same bits either way
    int *tile_ctr_next;   // the next launch's queue word, zeroed by this launch (CTA 0);
                          // the launches of a stream alternate between two words, so no
                          // memset runs between them
    float dfc[7][2];      // (hi, lo) of g, kappa, r, 1 - r, x1, x2, xs
};

// Prescale exponent word of the double-float kernel: for the smallest e with
// |x| < 2^e over the data and the walls, code = e + kDfCodeBias (e >= -1073,
// subnormals included); 0 when every value is zero.
constexpr int kDfCodeBias = 2048;
// Prescale code of one value on the host; 0 for zero.
inline int df_code_host(double x)
{
    if (x == 0.0)
        return 0;
    int e = 0;
    std::frexp(x, &e);  // |x| = m 2^e with 0.5 <= m < 1: the smallest e with |x| < 2^e
    return e + kDfCodeBias;
}
// Zero the word, then raise it to the data's code and walls_code.
cudaError_t df_prescale(const void *u, long long n, int walls_code, int *code, cudaStream_t s);
bool tb_df_geometry(int reach, int *H, int *U);
cudaError_t tb_df_occupancy(int *blocks_per_sm);
cudaError_t launch_tb_df(const void *tmap, const TbParams &p, int grid, cudaStream_t s);

// One problem of a batch (device table, one entry per problem).  The batch
// kernel uses the normalised block map x <- x + d (x_p - x), so every value
// here is a plain per-problem constant (no scale bookkeeping).
struct BatchDesc {
    long long off;        // element offset of the problem in the packed buffer (row aligned)
    long long n;          // interior points
    double r, omr;        // entry: w = (1-r) u + r u_partner
    double d;             // 2r/(1+2r)
    double kappa;         // singleton block factor (1-r)/(1+r)
    double f_l, f_r;      // wall terms r*beta_l, r*beta_r
    double x1, x2, xs;    // exit: (1+r)/(1+2r), r/(1+2r), 1/(1+r)
    // scaled form (FP64 and plain FP32): the state minus the linear wall
    // profile u*_j = ustar_a + ustar_b (j + 1), an exact fixed point of the
    // step, so the shifted problem has zero walls
    double g;             // 2r
    double kap_s;         // singleton factor (1 + g)(1-r)/(1+r)
    double ustar_a, ustar_b;
    // double-float kernel (FP64 plans): (hi, lo) pairs of g = 2r, the
    // singleton factor (1 + g_hi + g_lo)(1-r)/(1+r), r, 1 - r, x1, x2, xs,
    // and the prescale code of the wall values (see kDfCodeBias)
    float dfc[7][2];
    int walls_code;
};

// One launch of the batched tiled kernel over the packed buffer.
struct TbbParams {
    void *out;
    int *err;
    const int *row_pid;        // problem id of every 128-byte row (-1: padding)
    const BatchDesc *desc;     // per-problem constants
    long long n_rows, n_tiles;
    long long stall;           // diagnostic, as in TbParams
    int *tile_ctr;             // dynamic tile queue, as in TbParams (zeroed before the launch)
    int U, H;
    int p_first, do_entry, n_mid, do_exit;
    // scaled form (scaled != 0): after every R block steps the data of
    // problem b are multiplied by 2^-exps[b * Q + q]; at the launch end by
    // endf[b] (FP32: float2 hi + lo, FP64: double), which brings them back to
    // the normalised state
    int scaled, R, Q;
    const short *exps;
    const void *endf;
    // double-float kernel only: the source holds doubles (converted on load),
    // the launch writes doubles, per-problem prescale codes
    int df_in, df_out;
    const int *df_codes;
    // persistent launch (rounds > 1; plain FP32 kernel): the whole solve of
    // `steps` steps as rounds of `depth` steps in one launch.  Round k reads
    // the buffer of the launch's tensor map k & 1 and writes outs[k & 1];
    // done[n_tiles] (zeroed first) counts the consumer warps that finished
    // each tile; endf is the end-factor slot of the full rounds, endf_last
    // that of the last one.  rounds <= 1: one launch (out, endf, and the
    // per-launch fields above).
    int rounds, depth;
    long long steps;
    void *outs[2];
    int *done;
    const void *endf_last;
};

// Host (hi, lo) float pair of a double, hi = fl32(x), lo = fl32(x - hi).
inline void df_split_host(double x, float *pair)
{
    pair[0] = (float)x;
    pair[1] = (float)(x - (double)pair[0]);
}

// Per-problem non-finite scan of a packed buffer (status zeroed first).
cudaError_t batch_check(int prec, const void *u, const int *row_pid, const BatchDesc *desc, long long n_rows,
                        int *status, cudaStream_t s);

// Rescale exponents of the batched scaled form (one row of Q per problem) and
// the end factor of a launch with n_mid block steps (kernels in ge_tbb.cu).
// mode: the coefficient the kernel holds for g = 2r: 0 FP64 (end factor
// double), 1 FP32, 2 the double-float pair (end factors float2 hi, lo).
cudaError_t batch_exps(const BatchDesc *desc, int n_problems, int R, int Q, int mode, short *exps, cudaStream_t s);
cudaError_t batch_endf(const BatchDesc *desc, const short *exps, int n_problems, int R, int Q, int n_mid, int mode,
                       void *endf, cudaStream_t s);

// Host-side scale bookkeeping of the scaled block map x <- x + g x_partner
// (tiled kernels).  That map multiplies the symmetric part of every pair by
// exactly 1 + g, with g the coefficient the kernel holds: 2r, rounded to FP32
// on the FP32 path.  The host mirrors the product of those factors as a
// double-double so that no systematic scale error builds up over many steps.
inline void scaled_growth(double r, bool f32, double *hi, double *lo)
{
    const double g = f32 ? (double)(float)(2.0 * r) : 2.0 * r;
    *hi = 1.0 + g;
    *lo = (1.0 - *hi) + g;  // exact: 1 + g == hi + lo
}

// (h, l) <- (h, l) * (bh, bl) in double-double arithmetic.
inline void dd_mul(double &h, double &l, double bh, double bl)
{
    const double p = h * bh;
    const double e = std::fma(h, bh, -p);
    const double t = e + (h * bl + l * bh);
    h = p + t;
    l = t - (h - p);
}

// x / (h + l) to double precision.
inline double dd_div(double x, double h, double l)
{
    const double q = x / h;
    return q - q * (l / h);
}

// Launchers (return the cudaError_t of the launch).
cudaError_t launch_canon_f64(const double *in, double *out, long long n, int parity,
                             const CanonCoef &c, cudaStream_t s);
cudaError_t launch_canon_f32(const float *in, float *out, long long n, int parity,
                             const CanonCoef &c, cudaStream_t s);
// General sub-domain width k (ge_sweep.cu), one step.
cudaError_t launch_sweep_f64(const double *in, double *out, long long n, int parity, long long k,
                             const CanonCoef &c, cudaStream_t s);
cudaError_t launch_sweep_f32(const float *in, float *out, long long n, int parity, long long k,
                             const CanonCoef &c, cudaStream_t s);
// Up to `steps` width-k steps in one launch (tile in shared memory);
// *done = steps taken, 0 when the width does not fit (use the one-step launch).
cudaError_t launch_sweep_tb_f64(const double *in, double *out, long long n, int parity, long long k, int steps,
                                const CanonCoef &c, int *done, cudaStream_t s);
cudaError_t launch_sweep_tb_f32(const float *in, float *out, long long n, int parity, long long k, int steps,
                                const CanonCoef &c, int *done, cudaStream_t s);

// prec: 0 = FP64, 1 = FP32, 2 = FP32 compensated.  tmap: 128-byte-aligned
// CUtensorMap (opaque here) describing the source buffer.
cudaError_t launch_tb(int prec, const void *tmap, const TbParams &p, int grid, cudaStream_t s);
// A launch of exactly one block step and nothing else (no entry, exit;
// plain FP32): the streaming kernel, from buffer `in` to `out`.
cudaError_t launch_tb_stream(int prec, const void *in, void *out, const TbParams &p, cudaStream_t s);
// tile_rows: 256 or 128 (the tile geometry of the plan; the tensor map's box
// must have as many rows).
cudaError_t launch_tbb(int prec, int tile_rows, const void *tmap, const TbbParams &p, int grid, cudaStream_t s,
                       const void *tmap_other = nullptr);
// Batched double-float kernel (ge_tbb_df.cu) for FP64 plans; its per-call
// prescale: codes[b] = max(desc[b].walls_code, code of the problem's values).
cudaError_t launch_tbb_df(const void *tmap, const TbbParams &p, int grid, cudaStream_t s);
cudaError_t tbb_df_occupancy(int *blocks_per_sm);
cudaError_t batch_df_prescale(const double *u, const int *row_pid, const BatchDesc *desc, long long n_rows,
                              int n_problems, int *codes, cudaStream_t s);
cudaError_t tbb_occupancy(int prec, int tile_rows, int *blocks_per_sm);
// Co-resident CTAs per SM of the persistent plain FP32 kernel.
cudaError_t tbb_persist_occupancy(int tile_rows, int *blocks_per_sm);
bool tbb_geometry(int prec, int tile_rows, int reach, int *H, int *U);
// Largest steps per launch whose reach (steps + 2 stages) fits the batched
// kernel's tile for this precision.
int tbb_max_depth(int prec, int tile_rows);
// Largest co-resident CTAs per SM for the tiled kernel of this precision.
cudaError_t tb_occupancy(int prec, int *blocks_per_sm);
int tb_smem_bytes();
// Tile geometry of a launch whose stages reach `reach` points: halo H and
// output elements U per tile.  False if the reach does not fit a tile.
bool tb_geometry(int prec, int reach, int *H, int *U);

// Host-side planning of tiled solves (ge_tb_plan.cpp), shared by the context
// API and ge_solve_noalloc.
//
// Launch-independent fields of the tiled right-hand-side kernel for mesh
// ratio r and wall values beta_l, beta_r (prec: 0 FP64, 1 FP32, 2 FP32
// compensated); *growth_lo receives the low part of the scaled map's growth
// factor (onepg + growth_lo == 1 + g exactly).
void tb_fill_base(double r, double beta_l, double beta_r, int prec, TbParams *p, double *growth_lo);
// A depth clamped to what one launch's rescaling and step tables hold.
int tb_clamp_depth(const TbParams &base, int depth);
// Where a tiled solve runs: two state buffers of n_rows 128-byte rows with a
// tensor map each, the device error word and the tile-queue word.
struct TbTarget {
    const void *tmap[2];  // 64-byte aligned CUtensorMap of each buffer (opaque here)
    void *buf[2];
    long long n, n_rows;
    int *err;
    int *tile_ctr;        // two tile-queue words (alternating launches)
    long long grid_cap;   // SMs x co-resident CTAs per SM
};
// Issue the launches of `steps` steps from global step `step0`, `depth` steps
// per launch (df: the double-float kernel; its prescale is the caller's).
// *cur names the buffer holding the state and is updated.  The host mirrors
// the kernel's scale recurrence (see TbParams): sigma starts at 1 after the
// entry conversion, is multiplied by (1+2r) per block step and by 2^-e at
// each rescaling, where e brings it back into [1, 2).  Returns
// cudaErrorInvalidValue when the depth does not fit a tile, else the first
// launch error.
cudaError_t tb_run(const TbTarget &t, const TbParams &base, double growth_lo, bool df, int prec, int *cur,
                   long long step0, long long steps, int depth, cudaStream_t s);

// Record the calling thread's last-failure text (read by ge_last_error()).
void set_last_error(const char *msg);

}  // namespace ge
