// ge_sno.cpp -- the spectral neural operator (learned surrogate of K GE steps):
// parameters, forward, backward and Adam, orchestrating the kernels of
// ge_sno_kernels.cu.  Host code only.
//
// Architecture (1D Fourier neural operator on the n interior points):
//   features (u0, x, r, beta_l + (beta_r - beta_l) x)  -> lift (4 -> C)
//   L layers: v <- act( iDFT_M( R_m * DFT_M(v) ) + v W + b ),  act = GELU except
//             after the last layer; DFT_M keeps the M lowest modes, R_m is a
//             complex C x C matrix per mode
//   projection C -> H (GELU) -> 1, added to u0 (residual output).
// Activations are channel-last [batch * n, C]: BF16 in the plain mode (the
// GEMMs round their operands to BF16 anyway), FP32 in split mode.  The FP32
// master parameters are rounded to BF16 at the start of every forward pass
// (the network has BF16 weights; Adam updates the masters with the gradient
// of the rounded network).  Every GEMM accumulates in FP32; split mode adds
// the BF16 residuals of FP32 operands (~FP32 products).
//
// Parameter vector (FP32, this order): W0 [4][C], b0 [C]; per layer: Rr
// [M][C][C] (out, in), Ri [M][C][C], W [C][C] (in, out), b [C]; Q1 [C][H],
// q1 [H], Q2 [H], q2 [1].
#include "ge_sno.h"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime_api.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "ge_internal.h"
#include "ge_sno_internal.h"

namespace {

ge_status sfail(ge_status st, const char *msg)
{
    ge::set_last_error(msg);
    return st;
}

ge_status scuda(cudaError_t e, const char *what)
{
    char buf[400];
    std::snprintf(buf, sizeof(buf), "%s: %s", what, cudaGetErrorString(e));
    ge::set_last_error(buf);
    return e == cudaErrorMemoryAllocation ? GE_ENOMEM : GE_ECUDA;
}

struct LayerOff {
    long long rr, ri, w, b;
};

}  // namespace

struct ge_sno {
    int n = 0, C = 0, M = 0, L = 0, H = 0, max_batch = 0;
    bool split = false;
    cudaStream_t stream = nullptr;
    long long n_params = 0;
    long long off_w0 = 0, off_b0 = 0, off_q1 = 0, off_qb1 = 0, off_q2 = 0, off_qb2 = 0;
    std::vector<LayerOff> lay;
    float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
    float *pw = nullptr;               // params rounded to BF16 (the weights the network uses), FP32
    void *pw16 = nullptr;              // the same as BF16 (plain mode)
    long long adam_t = 0;
    float *F = nullptr, *G = nullptr;  // [2M][n] and [n][2M]
    void *F16 = nullptr, *G16 = nullptr;  // the same rounded to BF16 (plain mode)
    float *wspec = nullptr;            // [L][M][2C][2C] (BF16 in the plain mode)
    float *dwspec = nullptr;           // [M][2C][2C]
    // activations (max_batch)
    float *feat = nullptr;             // [B n][4] FP32, or [B n][8] BF16 in the plain mode
    std::vector<float *> v;            // L + 1 buffers [B n][C]
    std::vector<float *> pre;          // L buffers [B n][C]
    std::vector<float *> vh;           // L buffers [B][2M][C]
    float *y = nullptr;                // [B][2M][C] scratch (mixing output / its gradient)
    float *hpre = nullptr, *h = nullptr;  // [B n][H]
    float *out = nullptr, *dout = nullptr, *loss = nullptr;  // [B n], [B n], [B]
    float *dA = nullptr, *dB = nullptr;   // [B n][max(C, H)] gradient scratch
    float *dvh = nullptr;                 // [B][2M][C]
    // tensor-core inference path (ge_sno_tc.cu; plain mode, C = 64, 2M = 32,
    // H = 128, n a multiple of 128): transposed B operands and tensor maps
    bool tc = true;                       // use it where the shape allows
    bool tc_ready = false;                // tensor maps encoded
    int num_sms = 0;
    void *wt = nullptr;                   // [L][C out][C in] BF16
    void *q1t = nullptr;                  // [H][C] BF16
    void *wst = nullptr;                  // [L][M][2C out][2C in] BF16 (K-major spectral weights)
    // the weight-derived operands above (and the rounded weights pw, pw16)
    // no longer match the parameters: set when the parameters change
    bool tc_stale = true;
    int *err = nullptr;                   // device error word of the tensor-core kernels
    CUtensorMap tm_g, tm_y, tm_wt, tm_q1t, tm_f, tm_wst;
    std::vector<CUtensorMap> tm_v;        // one per activation buffer v[0..L]
    std::vector<CUtensorMap> tm_vs;       // store maps of v[1..L] (index l: v[l + 1])
    std::vector<CUtensorMap> tm_vh;       // one per spectrum buffer vh[0..L-1]
    std::vector<void *> allocs;
};

namespace {

ge::GemmArgs gemm(const void *A, long long lda_i, long long lda_k, const void *B, long long ldb_k, long long ldb_j,
                  void *C, long long ldc, int M, int N, int K)
{
    ge::GemmArgs g{};
    g.A = A;
    g.B = B;
    g.C = C;
    g.M = M;
    g.N = N;
    g.K = K;
    g.lda_i = lda_i;
    g.lda_k = lda_k;
    g.ldb_k = ldb_k;
    g.ldb_j = ldb_j;
    g.ldc = ldc;
    g.alpha = 1.0f;
    g.beta = 0.0f;
    g.ksplit = 1;
    return g;
}

#define SNO_TRY(expr)                                    \
    do {                                                 \
        cudaError_t e_ = (expr);                         \
        if (e_ != cudaSuccess)                           \
            return scuda(e_, "ge_sno: " #expr);          \
    } while (0)

// Storage of the plain mode: BF16 activations, weights and DFT bases (the
// GEMMs round their operands to BF16 anyway, so the forward values are the
// same); split mode keeps FP32 everywhere.
bool bf16_mode(const ge_sno *s) { return !s->split; }

// Element `off` of a buffer in the mode's storage type.
const void *at(const void *base, long long off, bool bf)
{
    return static_cast<const char *>(base) + off * (bf ? 2 : 4);
}

void *at(void *base, long long off, bool bf) { return static_cast<char *>(base) + off * (bf ? 2 : 4); }

// The weights as the GEMMs read them: BF16 copy or FP32 rounded values.
const void *weight(const ge_sno *s, long long off)
{
    return bf16_mode(s) ? at(s->pw16, off, true) : static_cast<const void *>(s->pw + off);
}

// Activation in/out format of a GEMM: BF16 in the plain mode.
ge::GemmArgs &act_fmt(ge::GemmArgs &g, bool bf)
{
    g.in_bf16 = bf ? 1 : 0;
    g.out_bf16 = bf ? 1 : 0;
    g.dg_bf16 = bf ? 1 : 0;
    return g;
}

// Weight gradient of a pointwise layer: dW[in][out] = X^T dY over R rows
// (X rows ldx apart; split-K with atomics, FP32), db = column sums of dY.
ge_status weight_grad(ge_sno *s, const void *X, int in, int ldx, const void *dY, int out, long long R, float *dW,
                      float *db)
{
    const bool bf = bf16_mode(s);
    SNO_TRY(cudaMemsetAsync(dW, 0, sizeof(float) * in * out, s->stream));
    ge::GemmArgs g = gemm(X, 1, ldx, dY, out, 1, dW, out, in, out, (int)R);
    act_fmt(g, bf).out_bf16 = 0;
    long long ks = R / 1024;
    g.ksplit = (int)(ks < 1 ? 1 : (ks > 512 ? 512 : ks));
    SNO_TRY(ge::sno_gemm(g, 1, s->split, s->stream));
    if (db)
        SNO_TRY(ge::sno_colsum(dY, db, R, out, bf ? 1 : 0, s->stream));
    return GE_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 2D BF16 tensor map over [rows][cols] (row pitch cols * 2 bytes) with a
// box of box_cols x box_rows and the swizzle matching box_cols * 2 bytes.
bool bf16_map(CUtensorMap *m, void *base, long long rows, int cols, int box_cols, int box_rows)
{
    auto enc = tmap_encoder();
    if (!enc)
        return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    const CUtensorMapSwizzle sw = box_cols * 2 == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The tensor-core inference path applies: plain mode and the shape its
// kernels are built for.
bool tc_shape(const ge_sno *s)
{
    return s->C == 64 && 2 * s->M == 32 && s->H == 128 && s->n % 128 == 0;
}
bool tc_active(const ge_sno *s) { return s->tc && !s->split && tc_shape(s) && s->tc_ready; }

// Inference with the tensor-core kernels for the truncated DFT, the fused
// layers and the projection (the mode mixing keeps the mma.sync GEMM).
ge_status forward_tc(ge_sno *s, int B, const float *u0, const float *r, const float *bl, const float *br,
                     float *out);

// Forward pass for B problems into out ([B n], FP32).  keep: also store the
// pre-activations the backward pass needs (training).
ge_status forward(ge_sno *s, int B, const float *u0, const float *r, const float *bl, const float *br, float *out,
                  bool keep)
{
    const int n = s->n, C = s->C, M = s->M, H = s->H;
    const long long R = (long long)B * n;
    cudaStream_t st = s->stream;
    const bool bf = bf16_mode(s);
    const float *P = s->pw;  // FP32 rounded weights: biases and the spectral matrices' source
    const void *F = bf ? s->F16 : static_cast<const void *>(s->F);
    const void *G = bf ? s->G16 : static_cast<const void *>(s->G);
    if (!keep && tc_active(s))
        return forward_tc(s, B, u0, r, bl, br, out);
    SNO_TRY(ge::sno_round_bf16(s->params, s->pw, bf ? s->pw16 : nullptr, s->n_params, st));
    // lift (K = 4: no GEMM); the features themselves only for the backward pass
    if (keep)
        SNO_TRY(ge::sno_features(u0, r, bl, br, s->feat, B, n, bf ? 1 : 0, st));
    SNO_TRY(ge::sno_lift(u0, r, bl, br, weight(s, s->off_w0), P + s->off_b0, s->v[0], B, n, C, bf ? 1 : 0, st));
    ge::GemmArgs g;
    for (int l = 0; l < s->L; ++l) {
        const LayerOff &o = s->lay[l];
        void *ws = at(s->wspec, (long long)l * M * 4 * C * C, bf);
        SNO_TRY(ge::sno_spec_assemble(P + o.rr, P + o.ri, ws, M, C, bf ? 1 : 0, st));
        // truncated DFT along the grid: vh[b] = F [2M x n] * v[b] [n x C]
        g = gemm(F, n, 1, s->v[l], C, 1, s->vh[l], C, 2 * M, C, n);
        g.sA = 0;
        g.sB = (long long)n * C;
        g.sC = 2LL * M * C;
        SNO_TRY(ge::sno_gemm(act_fmt(g, bf), B, s->split, st));
        // per-mode complex mixing: y[:, m] [B x 2C] = vh[:, m] [B x 2C] * Wspec_m [2C x 2C]
        g = gemm(s->vh[l], 2LL * M * C, 1, ws, 2 * C, 1, s->y, 2LL * M * C, B, 2 * C, 2 * C);
        g.sA = 2 * C;
        g.sB = 4LL * C * C;
        g.sC = 2 * C;
        SNO_TRY(ge::sno_gemm(act_fmt(g, bf), M, s->split, st));
        // back to the grid and the pointwise path in one pass:
        // pre[b] = G [n x 2M] y[b] [2M x C] + v[b] W + b, next v = GELU(pre)
        // (the last layer has no activation: next v = pre)
        const bool last = l == s->L - 1;
        g = gemm(G, 2 * M, 1, s->y, C, 1, last ? s->v[l + 1] : (keep ? s->pre[l] : nullptr), C, n, C, 2 * M);
        g.sA = 0;
        g.sB = 2LL * M * C;
        g.sC = (long long)n * C;
        g.A2 = s->v[l];
        g.lda2_i = C;
        g.lda2_k = 1;
        g.sA2 = (long long)n * C;
        g.B2 = weight(s, o.w);
        g.ldb2_k = C;
        g.ldb2_j = 1;
        g.K2 = C;
        g.bias = P + o.b;
        if (!last) {
            g.act = s->v[l + 1];
            g.sAct = (long long)n * C;
        }
        SNO_TRY(ge::sno_gemm(act_fmt(g, bf), B, s->split, st));
    }
    // projection; the residual output (FP32) predicts the change of u over the jump
    if (!keep) {
        // inference: h never leaves the chip: the first projection's epilogue
        // writes per-row partial sums of GELU(.)_j Q2[j] (one per 32 hidden
        // columns, into the gradient scratch dA), summed in a fixed order
        // into out = u0 + q2 + sum
        const int slots = (H + 31) / 32;
        g = gemm(s->v[s->L], C, 1, weight(s, s->off_q1), H, 1, nullptr, H, (int)R, H, C);
        g.bias = P + s->off_qb1;
        g.dot_w = P + s->off_q2;
        g.dot_out = s->dA;
        g.dot_slots = slots;
        SNO_TRY(ge::sno_gemm(act_fmt(g, bf), 1, s->split, st));
        SNO_TRY(ge::sno_dot_finish(u0, P + s->off_qb2, s->dA, slots, out, R, st));
        return GE_OK;
    }
    g = gemm(s->v[s->L], C, 1, weight(s, s->off_q1), H, 1, s->hpre, H, (int)R, H, C);
    g.bias = P + s->off_qb1;
    g.act = s->h;
    SNO_TRY(ge::sno_gemm(act_fmt(g, bf), 1, s->split, st));
    g = gemm(s->h, H, 1, weight(s, s->off_q2), 1, 1, out, 1, (int)R, 1, H);
    g.bias = P + s->off_qb2;
    g.C0 = u0;
    g.beta = 1.0f;
    act_fmt(g, bf).out_bf16 = 0;
    SNO_TRY(ge::sno_gemm(g, 1, s->split, st));
    return GE_OK;
}

ge_status forward_tc(ge_sno *s, int B, const float *u0, const float *r, const float *bl, const float *br,
                     float *out)
{
    const int n = s->n, C = s->C, M = s->M, H = s->H;
    const long long R = (long long)B * n;
    cudaStream_t st = s->stream;
    const float *P = s->pw;
    if (s->tc_stale) {
        // operands derived from the weights, once per parameter change: the
        // rounded weights, the K-major copies W^T (per layer) and Q1^T, and
        // the K-major spectral weights Wspec_m^T
        SNO_TRY(ge::sno_round_bf16(s->params, s->pw, s->pw16, s->n_params, st));
        for (int l = 0; l < s->L; ++l)
            SNO_TRY(ge::sno_transpose_rows(at(s->pw16, s->lay[l].w, true), at(s->wt, (long long)l * C * C, true), 1,
                                           C, C, st));
        SNO_TRY(ge::sno_transpose_rows(at(s->pw16, s->off_q1, true), s->q1t, 1, C, H, st));
        for (int l = 0; l < s->L; ++l)
            SNO_TRY(ge::sno_spec_assemble(P + s->lay[l].rr, P + s->lay[l].ri,
                                          at(s->wst, (long long)l * M * 4 * C * C, true), M, C, 1, st, true));
        s->tc_stale = false;
    }
    SNO_TRY(ge::sno_lift(u0, r, bl, br, weight(s, s->off_w0), P + s->off_b0, s->v[0], B, n, C, 1, st));
    ge::SnoTcArgs a{};
    a.n_tiles = R / 128;
    a.tiles_per_problem = n / 128;
    a.err = s->err;
    a.limit = ge::kWaitLimitCycles;
    for (int l = 0; l < s->L; ++l) {
        const LayerOff &o = s->lay[l];
        // truncated DFT: vh[b] = F v[b]
        a.out = s->vh[l];
        SNO_TRY(ge::sno_tc_dft(&s->tm_f, &s->tm_v[l], a, s->num_sms, st));
        // per-mode complex mixing: y[b, m] = vh[b, m] Wspec_m
        const ge::SnoTcMixArgs x{B, l * M * 2 * C, 2LL * M * C, s->y, s->err, ge::kWaitLimitCycles};
        SNO_TRY(ge::sno_tc_mix(&s->tm_vh[l], &s->tm_wst, x, M, st));
        a.b2_row = l * C;
        a.gelu = l < s->L - 1 ? 1 : 0;
        a.bias = P + o.b;
        a.out = s->v[l + 1];
        const ge::SnoTcMaps m{&s->tm_g, &s->tm_y, &s->tm_v[l], &s->tm_wt, &s->tm_vs[l]};
        SNO_TRY(ge::sno_tc_layer(m, a, s->num_sms, st));
    }
    a.b2_row = 0;
    a.gelu = 1;
    a.bias = P + s->off_qb1;
    a.q2w = P + s->off_q2;
    a.q2b = P + s->off_qb2;
    a.u0 = u0;
    a.out = out;
    const ge::SnoTcMaps m{nullptr, nullptr, &s->tm_v[s->L], &s->tm_q1t, nullptr};
    SNO_TRY(ge::sno_tc_projection(m, a, s->num_sms, st));
    return GE_OK;
}

// Backward from s->dout ([B n]) into s->grads.
ge_status backward(ge_sno *s, int B)
{
    const int n = s->n, C = s->C, M = s->M, H = s->H;
    const long long R = (long long)B * n;
    cudaStream_t st = s->stream;
    const bool bf = bf16_mode(s);
    const void *F = bf ? s->F16 : static_cast<const void *>(s->F);
    const void *G = bf ? s->G16 : static_cast<const void *>(s->G);
    const int ldf = bf ? 8 : 4;
    float *Gd = s->grads;
    ge_status rc;
    // projection: out = h Q2 + q2
    if ((rc = weight_grad(s, s->h, H, H, s->dout, 1, R, Gd + s->off_q2, Gd + s->off_qb2)) != GE_OK)
        return rc;
    // dhpre = (dout Q2^T) * GELU'(hpre)
    ge::GemmArgs g = gemm(s->dout, 1, 1, weight(s, s->off_q2), 1, 1, s->dA, H, (int)R, H, 1);
    g.dgelu_pre = s->hpre;
    SNO_TRY(ge::sno_gemm(act_fmt(g, bf), 1, s->split, st));
    if ((rc = weight_grad(s, s->v[s->L], C, C, s->dA, H, R, Gd + s->off_q1, Gd + s->off_qb1)) != GE_OK)
        return rc;
    g = gemm(s->dA, H, 1, weight(s, s->off_q1), 1, H, s->dB, C, (int)R, C, H);  // dv_L = dhpre Q1^T
    SNO_TRY(ge::sno_gemm(act_fmt(g, bf), 1, s->split, st));
    // dv holds the gradient of the current layer's pre-activation: the last
    // layer has no activation, and every lower one's GELU' is applied in the
    // epilogue of the GEMM that makes its gradient.
    void *dv = s->dB, *dnext = s->dA;
    for (int l = s->L - 1; l >= 0; --l) {
        const LayerOff &o = s->lay[l];
        const void *ws = at(s->wspec, (long long)l * M * 4 * C * C, bf);
        const void *dpre = dv;
        // pointwise path weights
        if ((rc = weight_grad(s, s->v[l], C, C, dpre, C, R, Gd + o.w, Gd + o.b)) != GE_OK)
            return rc;
        // spectral path: dy[b] = G^T dpre[b]
        g = gemm(G, 1, 2 * M, dpre, C, 1, s->y, C, 2 * M, C, n);
        g.sA = 0;
        g.sB = (long long)n * C;
        g.sC = 2LL * M * C;
        SNO_TRY(ge::sno_gemm(act_fmt(g, bf), B, s->split, st));
        // dWspec_m = vh[:, m]^T dy[:, m]  (FP32)
        g = gemm(s->vh[l], 1, 2LL * M * C, s->y, 2LL * M * C, 1, s->dwspec, 2 * C, 2 * C, 2 * C, B);
        g.sA = 2 * C;
        g.sB = 2 * C;
        g.sC = 4LL * C * C;
        act_fmt(g, bf).out_bf16 = 0;
        SNO_TRY(ge::sno_gemm(g, M, s->split, st));
        SNO_TRY(ge::sno_spec_reduce(s->dwspec, Gd + o.rr, Gd + o.ri, M, C, st));
        // dvh[:, m] = dy[:, m] Wspec_m^T
        g = gemm(s->y, 2LL * M * C, 1, ws, 1, 2 * C, s->dvh, 2LL * M * C, B, 2 * C, 2 * C);
        g.sA = 2 * C;
        g.sB = 4LL * C * C;
        g.sC = 2 * C;
        SNO_TRY(ge::sno_gemm(act_fmt(g, bf), M, s->split, st));
        // gradient of v_l, both paths in one pass: dpre[b] W^T + F^T dvh[b],
        // times GELU'(pre_{l-1}) when v_l is an activation
        g = gemm(dpre, C, 1, weight(s, o.w), 1, C, dnext, C, n, C, C);
        g.sA = (long long)n * C;
        g.sB = 0;
        g.sC = (long long)n * C;
        g.A2 = F;
        g.lda2_i = 1;
        g.lda2_k = n;
        g.sA2 = 0;
        g.B2 = s->dvh;
        g.ldb2_k = C;
        g.ldb2_j = 1;
        g.sB2 = 2LL * M * C;
        g.K2 = 2 * M;
        if (l > 0) {
            g.dgelu_pre = s->pre[l - 1];
            g.sDg = (long long)n * C;
        }
        SNO_TRY(ge::sno_gemm(act_fmt(g, bf), B, s->split, st));
        void *t = dv;
        dv = dnext;
        dnext = t;
    }
    // lift
    return weight_grad(s, s->feat, 4, ldf, dv, C, R, Gd + s->off_w0, Gd + s->off_b0);
}

// Bits of the BF16 value nearest to a finite float (ties to even).
uint16_t bf16_bits(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, sizeof(u));
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

void release_sno(ge_sno *s)
{
    if (!s)
        return;
    for (void *p : s->allocs)
        cudaFree(p);
    delete s;
}

// splitmix64 + Box-Muller, for the initial weights
struct Rng {
    unsigned long long x;
    double next()
    {
        unsigned long long z = (x += 0x9E3779B97F4A7C15ULL);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        z = z ^ (z >> 31);
        return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    }
    double uniform(double a) { return (2.0 * next() - 1.0) * a; }
};

}  // namespace

extern "C" {

ge_status ge_sno_create(ge_sno **out, int32_t n, int32_t width, int32_t modes, int32_t layers, int32_t hidden,
                        int32_t max_batch, uint64_t seed, void *stream)
{
    if (!out)
        return sfail(GE_EINVAL, "ge_sno_create: out is NULL");
    *out = nullptr;
    if (n < 4 || width < 1 || modes < 1 || 2 * modes > n || layers < 1 || hidden < 1 || max_batch < 1)
        return sfail(GE_EINVAL, "ge_sno_create: need n >= 4, 1 <= modes <= n/2, width, layers, hidden, max_batch >= 1");
    ge_sno *s = new (std::nothrow) ge_sno();
    if (!s)
        return sfail(GE_ENOMEM, "ge_sno_create: host allocation failed");
    s->n = n;
    s->C = width;
    s->M = modes;
    s->L = layers;
    s->H = hidden;
    s->max_batch = max_batch;
    s->stream = static_cast<cudaStream_t>(stream);
    const long long C = width, M = modes, H = hidden;
    long long off = 0;
    s->off_w0 = off;
    off += 4 * C;
    s->off_b0 = off;
    off += C;
    for (int l = 0; l < layers; ++l) {
        LayerOff o;
        o.rr = off;
        off += M * C * C;
        o.ri = off;
        off += M * C * C;
        o.w = off;
        off += C * C;
        o.b = off;
        off += C;
        s->lay.push_back(o);
    }
    s->off_q1 = off;
    off += C * H;
    s->off_qb1 = off;
    off += H;
    s->off_q2 = off;
    off += H;
    s->off_qb2 = off;
    off += 1;
    s->n_params = off;

    const long long R = (long long)max_batch * n;
    auto alloc = [&](float **p, long long count) -> cudaError_t {
        cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), sizeof(float) * (count > 0 ? count : 1));
        if (e == cudaSuccess)
            s->allocs.push_back(*p);
        return e;
    };
    auto alloc_bytes = [&](void **p, long long bytes) -> cudaError_t {
        cudaError_t e = cudaMalloc(p, (size_t)(bytes > 16 ? bytes : 16));
        if (e == cudaSuccess)
            s->allocs.push_back(*p);
        return e;
    };
    cudaError_t e = cudaSuccess;
    e = e ? e : alloc(&s->params, off);
    e = e ? e : alloc_bytes(&s->pw16, 2 * off);
    e = e ? e : alloc_bytes(&s->F16, 2 * 2 * M * n);
    e = e ? e : alloc_bytes(&s->G16, 2 * 2 * M * n);
    e = e ? e : alloc(&s->grads, off);
    e = e ? e : alloc(&s->pw, off);
    e = e ? e : alloc(&s->adam_m, off);
    e = e ? e : alloc(&s->adam_v, off);
    e = e ? e : alloc(&s->F, 2 * M * n);
    e = e ? e : alloc(&s->G, 2 * M * n);
    e = e ? e : alloc(&s->wspec, layers * M * 4 * C * C);
    e = e ? e : alloc(&s->dwspec, M * 4 * C * C);
    e = e ? e : alloc(&s->feat, R * 4);
    s->v.assign(layers + 1, nullptr);
    s->pre.assign(layers, nullptr);
    s->vh.assign(layers, nullptr);
    for (int l = 0; l <= layers && e == cudaSuccess; ++l)
        e = alloc(&s->v[l], R * C);
    for (int l = 0; l < layers && e == cudaSuccess; ++l)
        e = alloc(&s->pre[l], R * C);
    for (int l = 0; l < layers && e == cudaSuccess; ++l)
        e = alloc(&s->vh[l], (long long)max_batch * 2 * M * C);
    e = e ? e : alloc(&s->y, (long long)max_batch * 2 * M * C);
    e = e ? e : alloc(&s->dvh, (long long)max_batch * 2 * M * C);
    e = e ? e : alloc(&s->hpre, R * H);
    e = e ? e : alloc(&s->h, R * H);
    e = e ? e : alloc(&s->out, R);
    e = e ? e : alloc(&s->dout, R);
    e = e ? e : alloc(&s->loss, max_batch);
    e = e ? e : alloc(&s->dA, R * (C > H ? C : H));
    e = e ? e : alloc(&s->dB, R * (C > H ? C : H));
    e = e ? e : alloc_bytes(&s->wt, 2LL * layers * C * C);
    e = e ? e : alloc_bytes(&s->q1t, 2LL * H * C);
    e = e ? e : alloc_bytes(&s->wst, 2LL * layers * M * 4 * C * C);
    e = e ? e : alloc_bytes(reinterpret_cast<void **>(&s->err), 256);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(s->err, 0, 256, s->stream);
    int dev = 0;
    if (e == cudaSuccess)
        e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        release_sno(s);
        return scuda(e, "ge_sno_create: device allocation");
    }
    if (tc_shape(s)) {
        // tensor maps of the tensor-core path (BF16 views of the buffers)
        bool ok = bf16_map(&s->tm_g, s->G16, n, 2 * modes, 2 * modes, 128) &&
                  bf16_map(&s->tm_f, s->F16, 2 * modes, n, 64, 2 * modes) &&
                  bf16_map(&s->tm_y, s->y, (long long)max_batch * 2 * modes, width, width, 2 * modes) &&
                  bf16_map(&s->tm_wt, s->wt, (long long)layers * C, width, width, 64) &&
                  bf16_map(&s->tm_q1t, s->q1t, hidden, width, width, 128);
        ok = ok && bf16_map(&s->tm_wst, s->wst, (long long)layers * modes * 2 * width, 2 * width, 64, 128);
        s->tm_v.resize(layers + 1);
        for (int l = 0; l <= layers && ok; ++l)
            ok = bf16_map(&s->tm_v[l], s->v[l], R, width, width, 128);
        s->tm_vs.resize(layers);
        for (int l = 0; l < layers && ok; ++l)
            ok = bf16_map(&s->tm_vs[l], s->v[l + 1], R, width, 32, 32);
        s->tm_vh.resize(layers);
        for (int l = 0; l < layers && ok; ++l)
            ok = bf16_map(&s->tm_vh[l], s->vh[l], max_batch, 2 * modes * width, 64, 128);
        s->tc_ready = ok;
    }
    // DFT bases: F[2m][j] = cos(2 pi m j / n), F[2m+1][j] = -sin(...);
    // G[j][2m] = w_m cos(...), G[j][2m+1] = -w_m sin(...), w_0 = 1/n, w_m = 2/n
    std::vector<float> F(2 * M * n), Gm(2 * M * n);
    const double two_pi = 6.283185307179586476925286766559;
    for (long long m = 0; m < M; ++m)
        for (long long j = 0; j < n; ++j) {
            const double th = two_pi * (double)((m * j) % n) / (double)n;
            const double w = (m == 0 ? 1.0 : 2.0) / (double)n;
            F[(2 * m) * n + j] = (float)std::cos(th);
            F[(2 * m + 1) * n + j] = (float)(-std::sin(th));
            Gm[j * 2 * M + 2 * m] = (float)(w * std::cos(th));
            Gm[j * 2 * M + 2 * m + 1] = (float)(-w * std::sin(th));
        }
    // initial parameters (seeded)
    std::vector<float> p((size_t)off, 0.0f);
    Rng rng{seed * 0x2545F4914F6CDD1DULL + 12345};
    for (long long i = 0; i < 4 * C; ++i)
        p[s->off_w0 + i] = (float)rng.uniform(1.0 / std::sqrt(4.0));
    for (int l = 0; l < layers; ++l) {
        const double a = 1.0 / (double)(C * C);
        for (long long i = 0; i < M * C * C; ++i) {
            p[s->lay[l].rr + i] = (float)(a * rng.next());
            p[s->lay[l].ri + i] = (float)(a * rng.next());
        }
        for (long long i = 0; i < C * C; ++i)
            p[s->lay[l].w + i] = (float)rng.uniform(1.0 / std::sqrt((double)C));
    }
    for (long long i = 0; i < C * H; ++i)
        p[s->off_q1 + i] = (float)rng.uniform(1.0 / std::sqrt((double)C));
    for (long long i = 0; i < H; ++i)
        p[s->off_q2 + i] = (float)rng.uniform(1.0 / std::sqrt((double)H));
    std::vector<uint16_t> F16(F.size()), G16(Gm.size());
    for (size_t i = 0; i < F.size(); ++i) {
        F16[i] = bf16_bits(F[i]);
        G16[i] = bf16_bits(Gm[i]);
    }
    e = cudaMemcpyAsync(s->F, F.data(), sizeof(float) * F.size(), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->G, Gm.data(), sizeof(float) * Gm.size(), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->F16, F16.data(), 2 * F16.size(), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->G16, G16.data(), 2 * G16.size(), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->params, p.data(), sizeof(float) * p.size(), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(s->adam_m, 0, sizeof(float) * off, s->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(s->adam_v, 0, sizeof(float) * off, s->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        release_sno(s);
        return scuda(e, "ge_sno_create: initialisation");
    }
    *out = s;
    return GE_OK;
}

ge_status ge_sno_num_params(const ge_sno *s, int64_t *count)
{
    if (!s || !count)
        return sfail(GE_EINVAL, "ge_sno_num_params: NULL argument");
    *count = s->n_params;
    return GE_OK;
}

ge_status ge_sno_get_params(ge_sno *s, float *dst_dev)
{
    if (!s || !dst_dev)
        return sfail(GE_EINVAL, "ge_sno_get_params: NULL argument");
    cudaError_t e = cudaMemcpyAsync(dst_dev, s->params, sizeof(float) * s->n_params, cudaMemcpyDeviceToDevice, s->stream);
    return e == cudaSuccess ? GE_OK : scuda(e, "ge_sno_get_params");
}

ge_status ge_sno_set_params(ge_sno *s, const float *src_dev)
{
    if (!s || !src_dev)
        return sfail(GE_EINVAL, "ge_sno_set_params: NULL argument");
    s->tc_stale = true;
    cudaError_t e = cudaMemcpyAsync(s->params, src_dev, sizeof(float) * s->n_params, cudaMemcpyDeviceToDevice, s->stream);
    return e == cudaSuccess ? GE_OK : scuda(e, "ge_sno_set_params");
}

ge_status ge_sno_set_precision(ge_sno *s, int32_t split)
{
    if (!s || (split != 0 && split != 1))
        return sfail(GE_EINVAL, "ge_sno_set_precision: NULL model or mode not 0/1");
    s->split = split != 0;
    return GE_OK;
}

ge_status ge_sno_set_tensor_cores(ge_sno *s, int32_t on)
{
    if (!s || (on != 0 && on != 1))
        return sfail(GE_EINVAL, "ge_sno_set_tensor_cores: NULL model or value not 0/1");
    s->tc = on != 0;
    return GE_OK;
}

ge_status ge_sno_get_tensor_cores(const ge_sno *s, int32_t *active)
{
    if (!s || !active)
        return sfail(GE_EINVAL, "ge_sno_get_tensor_cores: NULL argument");
    *active = tc_active(s) ? 1 : 0;
    return GE_OK;
}

ge_status ge_sno_sync(ge_sno *s)
{
    if (!s)
        return sfail(GE_EINVAL, "ge_sno_sync: NULL model");
    int word = 0;
    cudaError_t e = cudaMemcpyAsync(&word, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess)
        return scuda(e, "ge_sno_sync");
    if (word == ge::kDevTimeout) {
        cudaMemsetAsync(s->err, 0, sizeof(int), s->stream);
        return sfail(GE_ETIMEOUT, "ge_sno: a tensor-core kernel's wait did not complete within the limit");
    }
    return GE_OK;
}

ge_status ge_sno_forward(ge_sno *s, int32_t batch, const float *u0, const float *r, const float *bl, const float *br,
                         float *pred)
{
    ge::NvtxRange nvtx("ge_sno_forward");
    if (!s || !u0 || !r || !bl || !br || !pred || batch < 1 || batch > s->max_batch)
        return sfail(GE_EINVAL, "ge_sno_forward: NULL argument or batch outside 1..max_batch");
    return forward(s, batch, u0, r, bl, br, pred, false);
}

ge_status ge_sno_rows_nonfinite(ge_sno *s, const float *u, int64_t rows, int32_t *flags)
{
    if (!s || !u || !flags || rows < 0)
        return sfail(GE_EINVAL, "ge_sno_rows_nonfinite: NULL argument or rows < 0");
    static_assert(sizeof(int32_t) == sizeof(int), "int32 flags");
    cudaError_t e = ge::sno_rows_nonfinite(u, rows, s->n, reinterpret_cast<int *>(flags), s->stream);
    return e == cudaSuccess ? GE_OK : scuda(e, "ge_sno_rows_nonfinite");
}

ge_status ge_sno_rows_gather(ge_sno *s, const float *src, int64_t src_rows, const int64_t *idx, int64_t count,
                             float *dst)
{
    if (!s || !src || !idx || !dst || src_rows < 0 || count < 0)
        return sfail(GE_EINVAL, "ge_sno_rows_gather: NULL argument or negative count");
    static_assert(sizeof(int64_t) == sizeof(long long), "int64 indices");
    cudaError_t e = ge::sno_rows_move(src, dst, reinterpret_cast<const long long *>(idx), count, s->n, src_rows,
                                      false, s->stream);
    return e == cudaSuccess ? GE_OK : scuda(e, "ge_sno_rows_gather");
}

ge_status ge_sno_rows_scatter(ge_sno *s, float *dst, int64_t dst_rows, const int64_t *idx, const float *src,
                              int64_t count)
{
    if (!s || !src || !idx || !dst || dst_rows < 0 || count < 0)
        return sfail(GE_EINVAL, "ge_sno_rows_scatter: NULL argument or negative count");
    cudaError_t e = ge::sno_rows_move(src, dst, reinterpret_cast<const long long *>(idx), count, s->n, dst_rows,
                                      true, s->stream);
    return e == cudaSuccess ? GE_OK : scuda(e, "ge_sno_rows_scatter");
}

ge_status ge_sno_rows_rel_err(ge_sno *s, const float *a, int64_t a_rows, const int64_t *idx, const float *ref,
                              int64_t count, float *err)
{
    if (!s || !a || !idx || !ref || !err || a_rows < 0 || count < 0)
        return sfail(GE_EINVAL, "ge_sno_rows_rel_err: NULL argument or negative count");
    cudaError_t e = ge::sno_rows_rel_err(a, a_rows, reinterpret_cast<const long long *>(idx), ref, count, s->n, err,
                                         s->stream);
    return e == cudaSuccess ? GE_OK : scuda(e, "ge_sno_rows_rel_err");
}

ge_status ge_sno_loss_grad(ge_sno *s, int32_t batch, const float *u0, const float *r, const float *bl,
                           const float *br, const float *target, float *loss_dev, float *grads_dev)
{
    ge::NvtxRange nvtx("ge_sno_loss_grad");
    if (!s || !u0 || !r || !bl || !br || !target || batch < 1 || batch > s->max_batch)
        return sfail(GE_EINVAL, "ge_sno_loss_grad: NULL argument or batch outside 1..max_batch");
    ge_status st = forward(s, batch, u0, r, bl, br, s->out, true);
    if (st != GE_OK)
        return st;
    cudaError_t e = ge::sno_rel_l2(s->out, target, s->dout, s->loss, s->n, batch, bf16_mode(s) ? 1 : 0, s->stream);
    if (e != cudaSuccess)
        return scuda(e, "ge_sno_loss_grad: loss");
    st = backward(s, batch);
    if (st != GE_OK)
        return st;
    if (loss_dev)
        e = cudaMemcpyAsync(loss_dev, s->loss, sizeof(float) * batch, cudaMemcpyDeviceToDevice, s->stream);
    if (e == cudaSuccess && grads_dev)
        e = cudaMemcpyAsync(grads_dev, s->grads, sizeof(float) * s->n_params, cudaMemcpyDeviceToDevice, s->stream);
    return e == cudaSuccess ? GE_OK : scuda(e, "ge_sno_loss_grad: copy out");
}

ge_status ge_sno_adam_step(ge_sno *s, float lr)
{
    if (!s || !(lr >= 0.0f))
        return sfail(GE_EINVAL, "ge_sno_adam_step: NULL model or bad learning rate");
    s->adam_t += 1;
    s->tc_stale = true;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - (float)std::pow(b1, (double)s->adam_t), c2 = 1.0f - (float)std::pow(b2, (double)s->adam_t);
    cudaError_t e = ge::sno_adam(s->params, s->grads, s->adam_m, s->adam_v, s->n_params, lr, b1, b2, 1e-8f, c1, c2,
                                 s->stream);
    return e == cudaSuccess ? GE_OK : scuda(e, "ge_sno_adam_step");
}

ge_status ge_sno_train_step(ge_sno *s, int32_t batch, const float *u0, const float *r, const float *bl,
                            const float *br, const float *target, float lr, float *loss_dev)
{
    ge_status st = ge_sno_loss_grad(s, batch, u0, r, bl, br, target, loss_dev, nullptr);
    return st == GE_OK ? ge_sno_adam_step(s, lr) : st;
}

void ge_sno_destroy(ge_sno *s)
{
    if (!s)
        return;
    cudaStreamSynchronize(s->stream);
    release_sno(s);
}

}  // extern "C"
