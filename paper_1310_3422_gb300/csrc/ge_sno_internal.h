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
struct GemmArgs {
    const float *A;
    const float *B;
    float *C;
    const float *C0;
    const float *bias;
    int M, N, K;
    long long lda_i, lda_k, ldb_k, ldb_j, ldc;
    long long sA, sB, sC, sC0;
    float alpha, beta;
    int ksplit;
    const float *A2;
    const float *B2;
    int K2;
    long long lda2_i, lda2_k, ldb2_k, ldb2_j, sA2, sB2;
    const float *dgelu_pre;
    long long sDg;
    float *act;
    long long sAct;
    // set by sno_gemm: float4 staging allowed for A, B, A2, B2; float2
    // epilogue accesses allowed
    int vec[4];
    int pairs;
};

cudaError_t sno_gemm(const GemmArgs &g, int batch, bool split, cudaStream_t s);
cudaError_t sno_features(const float *u0, const float *r, const float *bl, const float *br, float *f, int batch,
                         int n, cudaStream_t s);
cudaError_t sno_spec_assemble(const float *rr, const float *ri, float *w, int modes, int c, cudaStream_t s);
cudaError_t sno_spec_reduce(const float *dw, float *drr, float *dri, int modes, int c, cudaStream_t s);
cudaError_t sno_colsum(const float *x, float *out, long long rows, int cols, cudaStream_t s);
cudaError_t sno_rel_l2(const float *pred, const float *target, float *dpred, float *loss, int n, int batch,
                       cudaStream_t s);
cudaError_t sno_adam(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                     float eps, float c1, float c2, cudaStream_t s);
cudaError_t sno_round_bf16(const float *x, float *y, long long n, cudaStream_t s);

}  // namespace ge
