// ge_canon.cu -- GE_KERNEL_CANONICAL: one launch per GE time step, evaluated
// literally (arXiv:1310.3422 Sec. 2, Eqs. (aa), (bb), (cc), (dd), sub-domain
// width 1).
//
// Every point is one thread.  Its role follows from the parity p of the
// global step counter: with partner = i+1 if (i+p) is even else i-1, a point
// whose partner lies inside [0, n) is a member of the 2-point group
// (min, max); otherwise it is a singleton at a wall.  Group members use the
// closed forms (cc) (left) and (dd) (right) with prefactor 1/(1+2r); a left
// singleton uses Saul'yev A with beta_l as the new-level neighbour, a right
// singleton Saul'yev B with beta_r.  Old-level values outside the grid are
// the wall values.
//
// Rounding: each sum of products is a chain of fused multiply-adds in the
// order the equation prints its terms (first product rounded on its own), so
// the FP64 instantiation is bit-identical to any serial FP64 evaluation in
// that order.  The kernel is bound by the FP64 pipe (4 DP operations per
// point) and serves as the reference-accuracy path.
#include "ge_internal.h"

namespace ge {
namespace {

template <typename Real>
__device__ __forceinline__ Real mul_rn(Real a, Real b);
template <>
__device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }
template <>
__device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }

template <typename Real>
__device__ __forceinline__ Real fma_rn(Real a, Real b, Real c);
template <>
__device__ __forceinline__ double fma_rn<double>(double a, double b, double c) { return __fma_rn(a, b, c); }
template <>
__device__ __forceinline__ float fma_rn<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }

template <typename Real>
struct Coef {
    Real c1, c2, c3, c4, s0, s1, bl, br;
};

template <typename Real>
__global__ void __launch_bounds__(256) canon_kernel(const Real *__restrict__ in, Real *__restrict__ out,
                                                    long long n, int parity, Coef<Real> k)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const long long partner = (((i + parity) & 1) == 0) ? i + 1 : i - 1;
        Real res;
        if (partner == i + 1 && partner < n) {
            // left member of group (i, i+1): Eq. (cc)
            const Real a = (i == 0) ? k.bl : in[i - 1];
            const Real b = in[i];
            const Real c = in[i + 1];
            const Real d = (i + 2 == n) ? k.br : in[i + 2];
            res = fma_rn(k.c4, d, fma_rn(k.c3, c, fma_rn(k.c2, b, mul_rn(k.c1, a))));
        } else if (partner == i - 1 && partner >= 0) {
            // right member of group (i-1, i): Eq. (dd)
            const long long lo = i - 1;
            const Real a = (lo == 0) ? k.bl : in[lo - 1];
            const Real b = in[lo];
            const Real c = in[i];
            const Real d = (i + 1 == n) ? k.br : in[i + 1];
            res = fma_rn(k.c1, d, fma_rn(k.c2, c, fma_rn(k.c3, b, mul_rn(k.c4, a))));
        } else if (partner < 0) {
            // left singleton: Saul'yev A, Eq. (aa), new-level neighbour = beta_l
            const Real far = (n == 1) ? k.br : in[1];
            res = fma_rn(k.s0, far, fma_rn(k.s1, in[0], mul_rn(k.s0, k.bl)));
        } else {
            // right singleton: Saul'yev B, Eq. (bb), new-level neighbour = beta_r
            const Real far = (n == 1) ? k.bl : in[n - 2];
            res = fma_rn(k.s0, far, fma_rn(k.s1, in[n - 1], mul_rn(k.s0, k.br)));
        }
        out[i] = res;
    }
}

template <typename Real>
cudaError_t launch(const Real *in, Real *out, long long n, int parity, const CanonCoef &c,
                   cudaStream_t s)
{
    Coef<Real> k;
    k.c1 = (Real)c.c1;
    k.c2 = (Real)c.c2;
    k.c3 = (Real)c.c3;
    k.c4 = (Real)c.c4;
    k.s0 = (Real)c.s0;
    k.s1 = (Real)c.s1;
    k.bl = (Real)c.beta_l;
    k.br = (Real)c.beta_r;
    const int threads = 256;
    long long blocks = (n + threads - 1) / threads;
    if (blocks > (1LL << 20))
        blocks = 1LL << 20;  // grid-stride loop covers the rest
    canon_kernel<Real><<<(unsigned)blocks, threads, 0, s>>>(in, out, n, parity, k);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_canon_f64(const double *in, double *out, long long n, int parity,
                             const CanonCoef &c, cudaStream_t s)
{
    return launch<double>(in, out, n, parity, c, s);
}

cudaError_t launch_canon_f32(const float *in, float *out, long long n, int parity,
                             const CanonCoef &c, cudaStream_t s)
{
    return launch<float>(in, out, n, parity, c, s);
}

}  // namespace ge
