// ge_sno_internal.h -- launch interface of the spectral-neural-operator kernels
// (ge_sno_kernels.cu) used by the model code (ge_sno.cpp).
#pragma once

#include <cuda_runtime_api.h>

namespace ge {

// C[b] = alpha * (op(A[b]) op(B[b]) + op(A2[b]) op(B2[b])) + beta * C0[b]
// + bias[j] for b < batch.  Element (i, k) of A is A[i * lda_i + k * lda_k],
// element (k, j) of B is B[k * ldb_k + j * ldb_j] (any strides express a
// transpose); the optional second product (A2, B2, K2 terms, its own
// strides) extends the K range, so two GEMMs into one output share one pass.
// C is row-major with leading dimension ldc.  C0 may alias C (read before
// write, same element).  Epilogue, in this order: dgelu_pre set -> the value
// is multiplied by GELU'(dgelu_pre[off]) (backward through an activation);
// C set -> the value is stored to C; act set -> GELU(value) is stored to act
// (same layout as C, batch stride sAct).  With ksplit > 1 the K range of
// the first product is cut into ksplit slices whose partial products are
// added into C with atomics (C must be zeroed first; no second product, C0,
// bias or epilogue).
//
// Element formats: A, B, A2, B2 are FP32, or all BF16 when in_bf16 (then no
// split mode); C and act are FP32, or BF16 when out_bf16 (not with ksplit);
// dgelu_pre is BF16 when dg_bf16; C0 and bias are always FP32.
struct GemmArgs {
    const void *A;
    const void *B;
    void *C;
    const float *C0;
    const float *bias;
    int M, N, K;
    long long lda_i, lda_k, ldb_k, ldb_j, ldc;
    long long sA, sB, sC, sC0;
    float alpha, beta;
    int ksplit;
    const void *A2;
    const void *B2;
    int K2;
    long long lda2_i, lda2_k, ldb2_k, ldb2_j, sA2, sB2;
    const void *dgelu_pre;
    long long sDg;
    void *act;
    long long sAct;
    int in_bf16, out_bf16, dg_bf16;
    // dot_w set (FP32, N entries): instead of storing, each output row i
    // writes its partial sums of GELU(value_ij) dot_w[j], one per 32-column
    // group of the tile columns, to dot_out[i * dot_slots + group] (no
    // atomics, so the result is deterministic); dot_slots >= ceil(N / 32).
    // No C, act or ksplit with it.
    const float *dot_w;
    float *dot_out;
    int dot_slots;
    // set by sno_gemm: vector staging allowed for A, B, A2, B2 (float4 for
    // FP32, 16-byte cp.async chunks of 8 elements for BF16); paired epilogue
    int vec[4];
    int pairs;
};

cudaError_t sno_gemm(const GemmArgs &g, int batch, bool split, cudaStream_t s);

// Tensor-core (tcgen05) inference GEMMs of ge_sno_tc.cu, over 128-row tiles
// of the activation rows (rows = batch * n, n a multiple of 128, C = 64
// channels, 2M = 32 spectral rows, H = 128 hidden columns).  Tensor maps
// (CUtensorMap, 64-byte aligned, opaque here), all BF16:
//   layer:      a1 = G [n][2M] (box 32 x 128, 64-byte swizzle), b1 = y
//               [batch * 2M][C] (box 64 x 32, 128-byte swizzle; read
//               MN-major), a2 = v [rows][C] (box 64 x 128, 128-byte swizzle),
//               b2 = W^T of all layers [L * C][C] (box 64 x 64, 128-byte
//               swizzle);
//   projection: a2 = v as above, b2 = Q1^T [H][C] (box 64 x 128).
struct SnoTcMaps {
    const void *a1, *b1, *a2, *b2;
    const void *out;  // layer: store map of the next activation [rows][C] (box 32 x 32, 64-byte swizzle)
};
struct SnoTcArgs {
    long long n_tiles;      // rows / 128
    int tiles_per_problem;  // n / 128
    int b2_row;             // first row of this call's B2 block (layer * C; 0 for Q1^T)
    int gelu;               // layer: GELU after the bias (not after the last layer)
    const float *bias;      // layer: b [C]; projection: q1 [H]
    const float *q2w;       // projection: Q2 [H]
    const float *q2b;       // projection: q2 [1]
    const float *u0;        // projection: u0 [rows]
    void *out;              // layer: next activation, BF16 [rows][C]; projection: FP32 [rows]
    int *err;               // device error word (GE_ETIMEOUT on a wait that gave up)
    long long limit;        // wait limit in SM cycles
};
cudaError_t sno_tc_layer(const SnoTcMaps &m, const SnoTcArgs &a, int sms, cudaStream_t s);
cudaError_t sno_tc_projection(const SnoTcMaps &m, const SnoTcArgs &a, int sms, cudaStream_t s);
// Truncated DFT vh[b] = F v[b] on the tensor cores (2M = 32, C = 64; map_f:
// F [2M][n] BF16, box 64 x 32, 128-byte swizzle; map_v: the activation map of
// the layer kernel); writes a.out = vh, BF16 [batch][2M][C].
cudaError_t sno_tc_dft(const void *map_f, const void *map_v, const SnoTcArgs &a, int sms, cudaStream_t s);
// Mode mixing y[b, m] = vh[b, m] Wspec_m on the tensor cores (2C = 128):
// map_vh over vh [batch rows][2M * 2C] (box 64 x 128, 128-byte swizzle),
// map_wst over the K-major spectral weights Wspec_m^T of all layers
// [L * M * 2C][2C] (box 64 x 128); grid = (ceil(batch / 128), modes).
struct SnoTcMixArgs {
    int batch;           // problems (rows of vh and y)
    int b_row0;          // first row of this layer's block of map_wst (l * M * 2C)
    long long row_elems; // elements of one problem's spectrum (2M * C)
    void *y;             // out: BF16 [batch][row_elems]
    int *err;            // device error word
    long long limit;     // wait limit in SM cycles
};
cudaError_t sno_tc_mix(const void *map_vh, const void *map_wst, const SnoTcMixArgs &a, int modes, cudaStream_t s);
// yt[b][c][k] = y[b][k][c] for BF16 [batch][k_rows][c_cols] blocks (the
// K-major copies W^T and Q1^T).
cudaError_t sno_transpose_rows(const void *y, void *yt, long long batch, int k_rows, int c_cols, cudaStream_t s);
cudaError_t sno_features(const float *u0, const float *r, const float *bl, const float *br, void *f, int batch,
                         int n, int bf16, cudaStream_t s);
cudaError_t sno_spec_assemble(const float *rr, const float *ri, void *w, int modes, int c, int bf16, cudaStream_t s,
                              bool k_major = false);
cudaError_t sno_spec_reduce(const float *dw, float *drr, float *dri, int modes, int c, cudaStream_t s);
cudaError_t sno_colsum(const void *x, float *out, long long rows, int cols, int bf16, cudaStream_t s);
cudaError_t sno_rel_l2(const float *pred, const float *target, void *dpred, float *loss, int n, int batch, int bf16,
                       cudaStream_t s);
cudaError_t sno_adam(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                     float eps, float c1, float c2, cudaStream_t s);
cudaError_t sno_round_bf16(const float *x, float *y, void *y16, long long n, cudaStream_t s);
// v0[b n + j][c] = b0[c] + sum_k feature_k(b, j) W0[k][c] (features as in
// sno_features, rounded to BF16 when bf16); W0 BF16 or FP32 as v0.
cudaError_t sno_lift(const float *u0, const float *r, const float *bl, const float *br, const void *w0,
                     const float *b0, void *v0, int batch, int n, int c, int bf16, cudaStream_t s);
// out[i] = u0[i] + q2[0] + sum_k part[i * slots + k], summed in a fixed order
// Fallback arbiter helpers on rows of n FP32 values (row indices outside
// [0, rows) are skipped; rel_err gives NaN for them).
cudaError_t sno_rows_nonfinite(const float *u, long long rows, int n, int *flags, cudaStream_t s);
cudaError_t sno_rows_move(const float *src, float *dst, const long long *idx, long long count, int n, long long rows,
                          bool scatter, cudaStream_t s);
cudaError_t sno_rows_rel_err(const float *a, long long a_rows, const long long *idx, const float *ref, long long count,
                             int n, float *err, cudaStream_t s);
cudaError_t sno_dot_finish(const float *u0, const float *q2, const float *part, int slots, float *out, long long n,
                           cudaStream_t s);

}  // namespace ge
