// ge_sno_internal.h -- launch interface of the spectral-neural-operator kernels
// (ge_sno_kernels.cu) used by the model code (ge_sno.cpp).
#pragma once

#include <cuda_runtime_api.h>

namespace ge {

// C[b] = alpha * op(A[b]) op(B[b]) + beta * C0[b] + bias[j] for b < batch.
// Element (i, k) of A is A[i * lda_i + k * lda_k], element (k, j) of B is
// B[k * ldb_k + j * ldb_j] (any strides express a transpose); C is row-major
// with leading dimension ldc.  C0 may alias C (read before write, same
// element).  With ksplit > 1 the K range is cut into ksplit slices whose
// partial products are added into C with atomics (C must be zeroed first;
// C0 and bias are not applied).
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
};

cudaError_t sno_gemm(const GemmArgs &g, int batch, bool split, cudaStream_t s);
cudaError_t sno_gelu_fwd(const float *pre, float *act, long long n, cudaStream_t s);
cudaError_t sno_gelu_bwd(const float *pre, const float *dact, float *dpre, long long n, cudaStream_t s);
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
cudaError_t sno_add(float *y, const float *x, long long n, cudaStream_t s);

}  // namespace ge
