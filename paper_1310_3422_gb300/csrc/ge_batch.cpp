// ge_batch.cpp -- batched solves: many independent problems of uneven size and
// mesh ratio, packed back to back in one device buffer, advanced together by
// the batched tiled kernel (ge_tb.cu, tbb_kernel).  Host code only; built with
// -ffp-contract=off like the rest of the C ABI.
#include "ge.h"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime_api.h>

#include <cmath>
#include <cstdio>
#include <mutex>
#include <new>
#include <vector>

#include "ge_internal.h"

namespace {

ge_status bfail(ge_status st, const char *msg)
{
    ge::set_last_error(msg);
    return st;
}

ge_status bcuda(cudaError_t e, const char *what)
{
    char buf[400];
    std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    ge::set_last_error(buf);
    return e == cudaErrorMemoryAllocation ? GE_ENOMEM : GE_ECUDA;
}

PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

constexpr int kBatchDefaultDepthF64 = 48;
constexpr int kBatchDefaultDepthF32 = 64;

}  // namespace

struct ge_batch {
    CUtensorMap tmap[2];      // box of 256 rows, one per working buffer
    CUtensorMap tmap128[2];   // box of 128 rows (the 128-row tile geometry)
    ge_precision prec = GE_F32;
    cudaStream_t stream = nullptr;
    int n_problems = 0;
    int64_t total = 0;       // elements of the caller's packed buffer
    int64_t n_rows = 0;      // 128-byte rows of the working buffers
    void *buf[2] = {nullptr, nullptr};
    int *row_pid = nullptr;
    ge::BatchDesc *desc = nullptr;
    int *err = nullptr;
    int depth = 0;
    int num_sms = 0, blocks_per_sm = 0;
    // tile geometry of the launches (ge_batch_set_geometry, ge_batch_tune):
    // rows per tile (256 or 128) and co-resident CTAs per SM (0: as many as fit)
    int tile_rows = 256, ctas_per_sm = 0;
    int blocks_per_sm_128 = 0;
    // one persistent launch per run (plain FP32 plans; ge_batch_set_persistent)
    bool persistent = false;
    int *done = nullptr;     // per-tile completion counters of a persistent launch (n_rows ints)
    // scaled form (FP64, plain FP32): rescale exponents [n_problems][Q] and
    // end-factor slots, one per launch length n_mid met so far
    short *exps = nullptr;
    void *endf = nullptr;
    int R = 0, Q = 0;
    long long stall = 0;  // diagnostic (ge_batch_debug_stall)
    std::vector<int> slot_nmid;
    std::vector<char> slot_ready;
    // double-float kernel (FP64 plans, ge_batch_set_kernel)
    bool df = false;
    double r_max = 0.0;
    int *df_codes = nullptr;  // per-problem prescale codes of the current call
    int df_blocks_per_sm = 0;
};

namespace {

void release_batch(ge_batch *b)
{
    if (!b)
        return;
    for (int i = 0; i < 2; ++i)
        if (b->buf[i])
            cudaFree(b->buf[i]);
    if (b->row_pid)
        cudaFree(b->row_pid);
    if (b->desc)
        cudaFree(b->desc);
    if (b->err)
        cudaFree(b->err);
    if (b->exps)
        cudaFree(b->exps);
    if (b->endf)
        cudaFree(b->endf);
    if (b->df_codes)
        cudaFree(b->df_codes);
    if (b->done)
        cudaFree(b->done);
    delete b;
}

int prec_index(ge_precision p) { return p == GE_F64 ? 0 : (p == GE_F32 ? 1 : 2); }

constexpr int kEndfSlots = 64;

// End-factor slot of launches with n_mid block steps, computed on the plan's
// stream the first time (a kernel, so stream capture records it).  A slot
// filled inside a capture is not marked ready: the next direct run fills it
// again, since the captured graph may never be launched.  -1 when all slots
// are taken (that launch then uses the normalised form).
// Coefficient mode of the scaled form's tables (see ge::batch_exps).
int scale_mode(const ge_batch *b) { return b->df ? 2 : (b->prec == GE_F32 ? 1 : 0); }

int endf_slot(ge_batch *b, int n_mid, cudaError_t *err, std::vector<int> *filled)
{
    size_t i = 0;
    while (i < b->slot_nmid.size() && b->slot_nmid[i] != n_mid)
        ++i;
    if (i == b->slot_nmid.size()) {
        if ((int)i >= kEndfSlots)
            return -1;
        b->slot_nmid.push_back(n_mid);
        b->slot_ready.push_back(0);
    }
    // filled: slots this call has already enqueued (inside a capture a slot is
    // never marked ready, and one computation per call and slot suffices)
    bool enqueued = false;
    for (int f : *filled)
        enqueued = enqueued || f == (int)i;
    if (!b->slot_ready[i] && !enqueued) {
        filled->push_back((int)i);
        void *dst = static_cast<char *>(b->endf) + i * (size_t)b->n_problems * 8;
        *err = ge::batch_endf(b->desc, b->exps, b->n_problems, b->R, b->Q, n_mid, scale_mode(b), dst, b->stream);
        if (*err != cudaSuccess)
            return -1;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(b->stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone)
            b->slot_ready[i] = 1;
    }
    return (int)i;
}

// Largest co-resident CTAs per SM of the plan's kernel at a tile geometry.
int max_ctas(const ge_batch *b, int tile_rows)
{
    if (b->df)
        return b->df_blocks_per_sm;
    return tile_rows == 128 ? b->blocks_per_sm_128 : b->blocks_per_sm;
}

// Enqueue `steps` steps on the working buffers (state in buf[0] on entry)
// at the given depth and tile geometry (ctas 0: as many per SM as fit);
// returns the index of the buffer holding the result.
ge_status batch_steps(ge_batch *b, int64_t steps, int depth, int tile_rows, int ctas, int *result_buf)
{
    const int pidx = prec_index(b->prec);
    if (b->df)
        tile_rows = 256;  // the double-float kernel has the 256-row tile only
    const int cmax = max_ctas(b, tile_rows);
    if (ctas < 1 || ctas > cmax)
        ctas = cmax;
    int cur = 0;
    int64_t n0 = 0;
    std::vector<int> filled;  // end-factor slots enqueued by this call
    const int dmax = ge::tbb_max_depth(pidx, tile_rows);
    if (depth > dmax)
        depth = dmax;
    if (b->df) {
        // the call's prescale: per problem, the power of two just above its
        // largest |u| and wall value
        cudaError_t e = ge::batch_df_prescale(static_cast<const double *>(b->buf[0]), b->row_pid, b->desc,
                                              b->n_rows, b->n_problems, b->df_codes, b->stream);
        if (e != cudaSuccess)
            return bcuda(e, "ge_batch: double-float prescale");
    }
    if (b->persistent && pidx == 1 && !b->df && b->exps && b->done && steps > depth) {
        // the whole run as one persistent launch: rounds of `depth` steps
        // (the plan's scaled FP32 form; every round's reach fits the tile)
        const int64_t rounds = (steps + depth - 1) / depth;
        const int64_t L_last = steps - (rounds - 1) * depth;
        cudaError_t se = cudaSuccess;
        const int slot_mid = endf_slot(b, depth, &se, &filled);
        const int slot_last = se == cudaSuccess ? endf_slot(b, (int)(L_last - 1), &se, &filled) : -1;
        if (se != cudaSuccess)
            return bcuda(se, "ge_batch: end factors");
        ge::TbbParams p{};
        if (slot_mid >= 0 && slot_last >= 0 && ge::tbb_geometry(pidx, tile_rows, depth + 1, &p.H, &p.U)) {
            p.n_rows = b->n_rows;
            p.n_tiles = (b->n_rows * (ge::kRowBytes / 4) + p.U - 1) / p.U;
            p.row_pid = b->row_pid;
            p.desc = b->desc;
            p.err = b->err;
            p.stall = b->stall;
            p.scaled = 1;
            p.R = b->R;
            p.Q = b->Q;
            p.exps = b->exps;
            p.endf = static_cast<const char *>(b->endf) + (size_t)slot_mid * b->n_problems * 8;
            p.endf_last = static_cast<const char *>(b->endf) + (size_t)slot_last * b->n_problems * 8;
            p.rounds = (int)rounds;
            p.depth = depth;
            p.steps = steps;
            p.outs[0] = b->buf[1];  // round k reads buffer k & 1 and writes the other
            p.outs[1] = b->buf[0];
            p.done = b->done;
            p.tile_ctr = b->err + 48;
            // every CTA co-resident: at most what fits of the persistent kernel
            int pmax = 0;
            cudaError_t oe = ge::tbb_persist_occupancy(tile_rows, &pmax);
            if (oe != cudaSuccess || pmax < 1)
                return bcuda(oe == cudaSuccess ? cudaErrorInvalidConfiguration : oe, "ge_batch: persistent occupancy");
            long long grid = (long long)b->num_sms * (ctas < pmax ? ctas : pmax);
            if (grid > p.n_tiles)
                grid = p.n_tiles;
            cudaError_t e = cudaMemsetAsync(p.tile_ctr, 0, sizeof(int), b->stream);
            if (e == cudaSuccess)
                e = cudaMemsetAsync(b->done, 0, sizeof(int) * (size_t)p.n_tiles, b->stream);
            if (e == cudaSuccess)
                e = ge::launch_tbb(pidx, tile_rows, tile_rows == 128 ? &b->tmap128[0] : &b->tmap[0], p, (int)grid,
                                   b->stream, tile_rows == 128 ? &b->tmap128[1] : &b->tmap[1]);
            if (e != cudaSuccess)
                return bcuda(e, "ge_batch: persistent kernel launch");
            *result_buf = (int)(rounds & 1);
            return GE_OK;
        }
    }
    while (n0 < steps) {
        const int64_t L = (steps - n0 < depth) ? steps - n0 : depth;
        ge::TbbParams p{};
        const bool last = (n0 + L == steps);
        p.do_entry = (n0 == 0) ? 1 : 0;
        p.n_mid = (int)(last ? L - 1 : L);
        p.do_exit = last ? 1 : 0;
        p.p_first = (int)(n0 & 1);
        const int reach = p.do_entry + p.n_mid + p.do_exit;
        if (!ge::tbb_geometry(pidx, tile_rows, reach, &p.H, &p.U))
            return bfail(GE_EINVAL, "ge_batch: depth does not fit a tile");
        p.n_rows = b->n_rows;
        p.n_tiles = (b->n_rows * (ge::kRowBytes / (b->prec == GE_F64 ? 8 : 4)) + p.U - 1) / p.U;
        p.row_pid = b->row_pid;
        p.desc = b->desc;
        p.err = b->err;
        p.stall = b->stall;
        if (b->exps) {
            cudaError_t se = cudaSuccess;
            const int slot = endf_slot(b, p.n_mid, &se, &filled);
            if (se != cudaSuccess)
                return bcuda(se, "ge_batch: end factors");
            if (slot >= 0) {
                p.scaled = 1;
                p.R = b->R;
                p.Q = b->Q;
                p.exps = b->exps;
                p.endf = static_cast<const char *>(b->endf) + (size_t)slot * b->n_problems * 8;
            }
        }
        if (b->df && !p.scaled)
            return bfail(GE_EINVAL, "ge_batch: the double-float kernel needs an end-factor slot (at most 64 "
                                    "launch lengths per plan)");
        p.df_in = n0 == 0 ? 1 : 0;
        p.df_out = last ? 1 : 0;
        p.df_codes = b->df_codes;
        p.out = b->buf[cur ^ 1];
        p.tile_ctr = b->err + 48;  // the launch's tile queue, zeroed first
        long long grid = (long long)b->num_sms * ctas;
        if (grid > p.n_tiles)
            grid = p.n_tiles;
        cudaError_t e = cudaMemsetAsync(p.tile_ctr, 0, sizeof(int), b->stream);
        if (e == cudaSuccess)
            e = b->df ? ge::launch_tbb_df(&b->tmap[cur], p, (int)grid, b->stream)
                      : ge::launch_tbb(pidx, tile_rows, tile_rows == 128 ? &b->tmap128[cur] : &b->tmap[cur], p,
                                       (int)grid, b->stream);
        if (e != cudaSuccess)
            return bcuda(e, "ge_batch: kernel launch");
        cur ^= 1;
        n0 += L;
    }
    *result_buf = cur;
    return GE_OK;
}

}  // namespace

extern "C" {

ge_status ge_batch_create(ge_batch **out, int32_t n_problems, const int64_t *n, const double *r,
                          const double *beta_l, const double *beta_r, const int64_t *offsets, int64_t total,
                          ge_precision prec, void *stream)
{
    if (!out)
        return bfail(GE_EINVAL, "ge_batch_create: out is NULL");
    *out = nullptr;
    if (n_problems < 1 || !n || !r || !beta_l || !beta_r || !offsets || total < 1)
        return bfail(GE_EINVAL, "ge_batch_create: need n_problems >= 1, total >= 1 and non-NULL host arrays");
    if (prec != GE_F64 && prec != GE_F32 && prec != GE_F32_COMP)
        return bfail(GE_EINVAL, "ge_batch_create: unknown precision");
    const int K = ge::kRowBytes / (prec == GE_F64 ? 8 : 4);
    const int64_t n_rows = (total + K - 1) / K;
    if (n_rows >= (1LL << 31) - 2 * ge::kTileRows)
        return bfail(GE_EINVAL, "ge_batch_create: total is too large");
    std::vector<int> row_pid((size_t)n_rows, -1);
    std::vector<ge::BatchDesc> desc((size_t)n_problems);
    double r_max = 0.0;
    for (int32_t i = 0; i < n_problems; ++i) {
        const double ri = r[i];
        if (n[i] < 1 || offsets[i] < 0 || offsets[i] % K != 0 || offsets[i] + n[i] > total)
            return bfail(GE_EINVAL,
                         "ge_batch_create: each problem needs n >= 1, an offset that is a multiple of "
                         "128 bytes, and to lie inside the buffer");
        if (!(ri > 0.0) || !std::isfinite(ri) || !std::isfinite(beta_l[i]) || !std::isfinite(beta_r[i]))
            return bfail(GE_EINVAL, "ge_batch_create: need finite r > 0 and finite wall values");
        const int64_t r0 = offsets[i] / K, r1 = (offsets[i] + n[i] + K - 1) / K;
        for (int64_t row = r0; row < r1; ++row) {
            if (row_pid[(size_t)row] != -1)
                return bfail(GE_EINVAL, "ge_batch_create: problems share a 128-byte row (overlap)");
            row_pid[(size_t)row] = i;
        }
        const double det = 1.0 + 2.0 * ri;
        ge::BatchDesc &d = desc[(size_t)i];
        d.off = offsets[i];
        d.n = n[i];
        d.r = ri;
        d.omr = 1.0 - ri;
        d.d = 2.0 * ri / det;
        d.kappa = (1.0 - ri) / (1.0 + ri);
        d.f_l = ri * beta_l[i];
        d.f_r = ri * beta_r[i];
        d.x1 = (1.0 + ri) / det;
        d.x2 = ri / det;
        d.xs = 1.0 / (1.0 + ri);
        const double g_used = (prec == GE_F32) ? (double)(float)(2.0 * ri) : 2.0 * ri;
        d.g = 2.0 * ri;
        d.kap_s = (1.0 + g_used) * (1.0 - ri) / (1.0 + ri);
        d.ustar_a = beta_l[i];
        d.ustar_b = (beta_r[i] - beta_l[i]) / (double)(n[i] + 1);
        // double-float pairs: the scaled map's growth is 1 + (g_hi + g_lo)
        ge::df_split_host(2.0 * ri, d.dfc[0]);
        const double g_df = (double)d.dfc[0][0] + (double)d.dfc[0][1];
        ge::df_split_host((1.0 + g_df) * ((1.0 - ri) / (1.0 + ri)), d.dfc[1]);
        ge::df_split_host(ri, d.dfc[2]);
        ge::df_split_host(1.0 - ri, d.dfc[3]);
        ge::df_split_host(d.x1, d.dfc[4]);
        ge::df_split_host(d.x2, d.dfc[5]);
        ge::df_split_host(d.xs, d.dfc[6]);
        const int wl = ge::df_code_host(beta_l[i]), wr = ge::df_code_host(beta_r[i]);
        d.walls_code = wl > wr ? wl : wr;
        r_max = ri > r_max ? ri : r_max;
    }
    ge_batch *b = new (std::nothrow) ge_batch();
    if (!b)
        return bfail(GE_ENOMEM, "ge_batch_create: host allocation failed");
    b->r_max = r_max;
    b->prec = prec;
    b->stream = static_cast<cudaStream_t>(stream);
    b->n_problems = n_problems;
    b->total = total;
    b->n_rows = n_rows;
    b->depth = prec == GE_F64 ? kBatchDefaultDepthF64 : kBatchDefaultDepthF32;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t bytes = (size_t)n_rows * ge::kRowBytes;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        e = cudaMalloc(&b->buf[i], bytes);
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&b->row_pid), row_pid.size() * sizeof(int));
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&b->desc), desc.size() * sizeof(ge::BatchDesc));
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&b->err), 256);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->row_pid, row_pid.data(), row_pid.size() * sizeof(int), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->desc, desc.data(), desc.size() * sizeof(ge::BatchDesc), cudaMemcpyHostToDevice,
                            b->stream);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i)
        e = cudaMemsetAsync(b->buf[i], 0, bytes, b->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b->err, 0, 256, b->stream);
    if (e == cudaSuccess && prec != GE_F32_COMP) {
        // scaled form: rescale every R block steps, R chosen so the scale
        // stays below 2^headroom (as for one problem: inputs up to about
        // 2^(max exponent - headroom) are safe)
        const double headroom = prec == GE_F64 ? 256.0 : GE_F32_HEADROOM;
        const int R = (int)std::floor(headroom / std::log2(1.0 + 2.0 * r_max));
        b->R = R < 1 ? 1 : (R > ge::kMaxTableSteps ? ge::kMaxTableSteps : R);
        b->Q = (ge::kMaxTableSteps + b->R - 1) / b->R;
        e = cudaMalloc(reinterpret_cast<void **>(&b->exps), (size_t)n_problems * b->Q * sizeof(short));
        if (e == cudaSuccess)
            e = cudaMalloc(&b->endf, (size_t)kEndfSlots * n_problems * 8);
        if (e == cudaSuccess)
            e = ge::batch_exps(b->desc, n_problems, b->R, b->Q, scale_mode(b), b->exps, b->stream);
    }
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess)
        e = ge::tbb_occupancy(prec_index(prec), 256, &b->blocks_per_sm);
    if (e == cudaSuccess)
        e = ge::tbb_occupancy(prec_index(prec), 128, &b->blocks_per_sm_128);
    if (e != cudaSuccess || b->blocks_per_sm < 1 || b->blocks_per_sm_128 < 1) {
        release_batch(b);
        return bcuda(e == cudaSuccess ? cudaErrorInvalidConfiguration : e, "ge_batch_create");
    }
    auto enc = encoder();
    if (!enc) {
        release_batch(b);
        return bfail(GE_ECUDA, "ge_batch_create: cuTensorMapEncodeTiled is not available");
    }
    for (int i = 0; i < 4; ++i) {
        cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)n_rows};
        cuuint64_t strides[1] = {(cuuint64_t)ge::kRowBytes};
        cuuint32_t box[2] = {(cuuint32_t)K, (cuuint32_t)(i < 2 ? 256 : 128)};
        cuuint32_t estr[2] = {1, 1};
        CUresult cr = enc(i < 2 ? &b->tmap[i] : &b->tmap128[i - 2],
                          prec == GE_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                          2, b->buf[i & 1], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) {
            release_batch(b);
            return bfail(GE_ECUDA, "ge_batch_create: cuTensorMapEncodeTiled failed");
        }
    }
    *out = b;
    return GE_OK;
}

ge_status ge_batch_set_kernel(ge_batch *b, ge_kernel kernel)
{
    if (!b)
        return bfail(GE_EINVAL, "ge_batch_set_kernel: plan is NULL");
    const bool df = kernel == GE_KERNEL_TEMPORAL_DF;
    if (!df && kernel != GE_KERNEL_AUTO && kernel != GE_KERNEL_TEMPORAL)
        return bfail(GE_EINVAL, "ge_batch_set_kernel: batches run GE_KERNEL_TEMPORAL or GE_KERNEL_TEMPORAL_DF");
    if (df && b->prec != GE_F64)
        return bfail(GE_EINVAL, "ge_batch_set_kernel: the double-float kernel needs a GE_F64 plan");
    if (df && b->r_max > 1048576.0)
        return bfail(GE_EINVAL, "ge_batch_set_kernel: the double-float kernel takes r <= 2^20");
    if (df == b->df)
        return GE_OK;
    // launches in flight still read the scaled form's tables
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess && df && !b->df_codes)
        e = cudaMalloc(reinterpret_cast<void **>(&b->df_codes), (size_t)b->n_problems * sizeof(int));
    if (e == cudaSuccess && df && b->df_blocks_per_sm < 1)
        e = ge::tbb_df_occupancy(&b->df_blocks_per_sm);
    if (e != cudaSuccess)
        return bcuda(e, "ge_batch_set_kernel");
    // the scaled form's rescalings and end factors for the new arithmetic:
    // FP32 headroom for the double-float pairs, the FP64 one otherwise
    const double headroom = df ? GE_F32_HEADROOM : 256.0;
    int R = (int)std::floor(headroom / std::log2(1.0 + 2.0 * b->r_max));
    R = R < 1 ? 1 : (R > ge::kMaxTableSteps ? ge::kMaxTableSteps : R);
    const int Q = (ge::kMaxTableSteps + R - 1) / R;
    if (Q > b->Q) {
        cudaFree(b->exps);
        b->exps = nullptr;
        e = cudaMalloc(reinterpret_cast<void **>(&b->exps), (size_t)b->n_problems * Q * sizeof(short));
        if (e != cudaSuccess)
            return bcuda(e, "ge_batch_set_kernel: rescale table");
    }
    b->df = df;
    if (df)
        b->tile_rows = 256;  // the double-float kernel has the 256-row tile only
    b->R = R;
    b->Q = Q;
    b->slot_nmid.clear();
    b->slot_ready.clear();
    e = ge::batch_exps(b->desc, b->n_problems, b->R, b->Q, scale_mode(b), b->exps, b->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? GE_OK : bcuda(e, "ge_batch_set_kernel: rescale exponents");
}

ge_status ge_batch_set_depth(ge_batch *b, int32_t depth)
{
    if (!b || depth < 0 || depth > ge::kMaxTableSteps)
        return bfail(GE_EINVAL, "ge_batch_set_depth: NULL plan or depth outside 0..512");
    b->depth = depth ? depth : (b->prec == GE_F64 ? kBatchDefaultDepthF64 : kBatchDefaultDepthF32);
    return GE_OK;
}

ge_status ge_batch_get_depth(const ge_batch *b, int32_t *depth)
{
    if (!b || !depth)
        return bfail(GE_EINVAL, "ge_batch_get_depth: NULL argument");
    *depth = b->depth;
    return GE_OK;
}

ge_status ge_batch_run(ge_batch *b, void *u_dev, int64_t steps)
{
    ge::NvtxRange nvtx("ge_batch_run");
    if (!b || !u_dev || steps < 0)
        return bfail(GE_EINVAL, "ge_batch_run: NULL argument or steps < 0");
    if (steps == 0)
        return GE_OK;
    const size_t bytes = (size_t)b->total * (b->prec == GE_F64 ? 8 : 4);
    cudaError_t e = cudaMemcpyAsync(b->buf[0], u_dev, bytes, cudaMemcpyDeviceToDevice, b->stream);
    if (e != cudaSuccess)
        return bcuda(e, "ge_batch_run: copy in");
    int res = 0;
    ge_status st = batch_steps(b, steps, b->depth, b->tile_rows, b->ctas_per_sm, &res);
    if (st != GE_OK)
        return st;
    e = cudaMemcpyAsync(u_dev, b->buf[res], bytes, cudaMemcpyDeviceToDevice, b->stream);
    return e == cudaSuccess ? GE_OK : bcuda(e, "ge_batch_run: copy out");
}

ge_status ge_batch_set_geometry(ge_batch *b, int32_t tile_rows, int32_t ctas_per_sm)
{
    if (!b)
        return bfail(GE_EINVAL, "ge_batch_set_geometry: plan is NULL");
    if (tile_rows == 0)
        tile_rows = 256;
    if (tile_rows != 256 && tile_rows != 128)
        return bfail(GE_EINVAL, "ge_batch_set_geometry: tile_rows must be 0, 128 or 256");
    if (b->df && tile_rows != 256)
        return bfail(GE_EINVAL, "ge_batch_set_geometry: the double-float kernel has 256-row tiles only");
    if (ctas_per_sm < 0 || ctas_per_sm > max_ctas(b, tile_rows))
        return bfail(GE_EINVAL, "ge_batch_set_geometry: ctas_per_sm beyond what fits on an SM");
    b->tile_rows = tile_rows;
    b->ctas_per_sm = ctas_per_sm;
    return GE_OK;
}

ge_status ge_batch_get_geometry(const ge_batch *b, int32_t *tile_rows, int32_t *ctas_per_sm)
{
    if (!b || !tile_rows || !ctas_per_sm)
        return bfail(GE_EINVAL, "ge_batch_get_geometry: NULL argument");
    const int tr = b->df ? 256 : b->tile_rows;
    const int cmax = max_ctas(b, tr);
    *tile_rows = tr;
    *ctas_per_sm = (b->ctas_per_sm < 1 || b->ctas_per_sm > cmax) ? cmax : b->ctas_per_sm;
    return GE_OK;
}

ge_status ge_batch_set_persistent(ge_batch *b, int32_t on)
{
    if (!b || (on != 0 && on != 1))
        return bfail(GE_EINVAL, "ge_batch_set_persistent: NULL plan or value not 0/1");
    if (on && !b->done) {
        cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&b->done), sizeof(int) * (size_t)(b->n_rows + 1));
        if (e != cudaSuccess)
            return bcuda(e, "ge_batch_set_persistent");
    }
    b->persistent = on != 0;
    return GE_OK;
}

ge_status ge_batch_get_persistent(const ge_batch *b, int32_t *on)
{
    if (!b || !on)
        return bfail(GE_EINVAL, "ge_batch_get_persistent: NULL argument");
    *on = b->persistent ? 1 : 0;
    return GE_OK;
}

ge_status ge_batch_tune(ge_batch *b, const void *u_dev, int64_t steps, int32_t *best_depth)
{
    ge::NvtxRange nvtx("ge_batch_tune");
    if (!b || !u_dev || steps < 1)
        return bfail(GE_EINVAL, "ge_batch_tune: NULL argument or steps < 1");
    static const int cand[] = {16, 32, 48, 64, 96, 128, 192, 256};
    const size_t bytes = (size_t)b->total * (b->prec == GE_F64 ? 8 : 4);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    // time one configuration on `steps` steps of the caller's data: one
    // untimed run (first use of this launch shape), then a timed one
    auto timed = [&](int d, int tr, int ctas, float *ms) -> ge_status {
        int res = 0;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            e = cudaMemcpyAsync(b->buf[0], u_dev, bytes, cudaMemcpyDeviceToDevice, b->stream);
            if (e == cudaSuccess && rep == 1)
                e = cudaEventRecord(e0, b->stream);
            if (e != cudaSuccess)
                break;
            ge_status st = batch_steps(b, steps, d, tr, ctas, &res);
            if (st != GE_OK)
                return st;
            if (rep == 1)
                e = cudaEventRecord(e1, b->stream);
        }
        if (e == cudaSuccess)
            e = cudaEventSynchronize(e1);
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(ms, e0, e1);
        return GE_OK;
    };
    // coordinate search: the depth at the plan's geometry, then the geometry
    // (rows per tile x CTAs per SM) at that depth, then the depth again
    double best = 1e300;
    int best_d = b->depth, best_tr = b->df ? 256 : b->tile_rows;
    int best_c = max_ctas(b, best_tr);
    if (b->ctas_per_sm >= 1 && b->ctas_per_sm < best_c)
        best_c = b->ctas_per_sm;
    ge_status st = GE_OK;
    for (int pass = 0; pass < 3 && st == GE_OK && e == cudaSuccess; ++pass) {
        if (pass == 1) {
            const int tr0 = best_tr, c0 = best_c;
            for (int tr : {256, 128}) {
                if (b->df && tr != 256)
                    continue;
                for (int c = 1; c <= max_ctas(b, tr) && st == GE_OK && e == cudaSuccess; ++c) {
                    if (tr == tr0 && c == c0)
                        continue;
                    float ms = 0.0f;
                    st = timed(best_d, tr, c, &ms);
                    if (st == GE_OK && e == cudaSuccess && ms < best) {
                        best = ms;
                        best_tr = tr;
                        best_c = c;
                    }
                }
            }
        } else {
            for (int d : cand) {
                if (pass == 2 && d == best_d)
                    continue;
                float ms = 0.0f;
                st = timed(d, best_tr, best_c, &ms);
                if (st != GE_OK || e != cudaSuccess)
                    break;
                if (ms < best) {
                    best = ms;
                    best_d = d;
                }
            }
        }
    }
    // finally, for a plain FP32 plan: the run as one persistent launch
    // against one launch per `depth` steps, at the chosen depth and geometry
    bool best_persist = false;
    if (st == GE_OK && e == cudaSuccess && b->prec == GE_F32 && !b->df && b->exps && steps > best_d) {
        const bool was = b->persistent;
        st = ge_batch_set_persistent(b, 1);
        float ms = 0.0f;
        if (st == GE_OK)
            st = timed(best_d, best_tr, best_c, &ms);
        if (st == GE_OK && e == cudaSuccess && ms < best)
            best_persist = true;
        b->persistent = was;
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    if (st != GE_OK)
        return st;
    if (e != cudaSuccess)
        return bcuda(e, "ge_batch_tune");
    b->depth = best_d;
    b->tile_rows = best_tr;
    b->ctas_per_sm = best_c;
    b->persistent = best_persist;
    if (best_depth)
        *best_depth = best_d;
    return GE_OK;
}

ge_status ge_batch_sync(ge_batch *b)
{
    if (!b)
        return bfail(GE_EINVAL, "ge_batch_sync: NULL plan");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess)
        return bcuda(e, "ge_batch_sync");
    int word = 0;
    e = cudaMemcpy(&word, b->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return bcuda(e, "ge_batch_sync: reading the device error word");
    if (word != ge::kDevOk) {
        // reported once: the next run starts from the caller's buffer again
        e = cudaMemset(b->err, 0, sizeof(int));
        if (e != cudaSuccess)
            return bcuda(e, "ge_batch_sync: clearing the device error word");
    }
    if (word == ge::kDevTimeout)
        return bfail(GE_ETIMEOUT, "ge_batch: a tile load did not complete within the wait limit");
    return GE_OK;
}

ge_status ge_batch_check(ge_batch *b, const void *u_dev, int32_t *status_dev)
{
    if (!b || !u_dev || !status_dev)
        return bfail(GE_EINVAL, "ge_batch_check: NULL argument");
    static_assert(sizeof(int32_t) == sizeof(int), "status words are int");
    cudaError_t e = cudaMemsetAsync(status_dev, 0, sizeof(int32_t) * (size_t)b->n_problems, b->stream);
    if (e == cudaSuccess) {
        // rows of the caller's buffer only (the plan's rows cover total rounded up)
        const int K = ge::kRowBytes / (b->prec == GE_F64 ? 8 : 4);
        const long long rows = (b->total + K - 1) / K;
        // the last row may reach past `total`: problems end inside it, and the
        // kernel reads only elements inside a problem
        e = ge::batch_check(b->prec == GE_F64 ? 0 : 1, u_dev, b->row_pid, b->desc, rows,
                            reinterpret_cast<int *>(status_dev), b->stream);
    }
    return e == cudaSuccess ? GE_OK : bcuda(e, "ge_batch_check");
}

ge_status ge_batch_debug_stall(ge_batch *b, int64_t cycles)
{
    if (!b || cycles < 0)
        return bfail(GE_EINVAL, "ge_batch_debug_stall: NULL plan or cycles < 0");
    b->stall = (long long)cycles;
    return GE_OK;
}

void ge_batch_destroy(ge_batch *b)
{
    if (!b)
        return;
    cudaStreamSynchronize(b->stream);
    release_batch(b);
}

ge_status ge_solve_batch(int32_t n_problems, const int64_t *n, const double *r, const double *beta_l,
                         const double *beta_r, const int64_t *offsets, int64_t total, void *u_dev,
                         int32_t *status_dev, int64_t steps, ge_precision prec, void *stream)
{
    ge_batch *b = nullptr;
    ge_status st = ge_batch_create(&b, n_problems, n, r, beta_l, beta_r, offsets, total, prec, stream);
    if (st != GE_OK)
        return st;
    st = ge_batch_run(b, u_dev, steps);
    if (st == GE_OK && status_dev)
        st = ge_batch_check(b, u_dev, status_dev);
    if (st == GE_OK)
        st = ge_batch_sync(b);
    ge_batch_destroy(b);
    return st;
}

}  // extern "C"
