// ge_canon.cu -- GE_KERNEL_CANONICAL: one launch per GE time step, evaluated
// literally (arXiv:1310.3422 Sec. 2, Eqs. (aa), (bb), (cc), (dd), sub-domain
// width 1).
//
// The role of a point follows from the parity p of the global step counter:
// with partner = i+1 if (i+p) is even else i-1, a point whose partner lies
// inside [0, n) is a member of the 2-point group (min, max); otherwise it is
// a singleton at a wall.  One thread evaluates one group (or singleton).
// Group members use the closed forms (cc) (left) and (dd) (right) with
// prefactor 1/(1+2r); a left singleton uses Saul'yev A with beta_l as the
// new-level neighbour, a right singleton Saul'yev B with beta_r.  Old-level
// values outside the grid are the wall values.
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

// One thread per unit of the step's grouping: unit u holds the points
// s = 2u - parity and s + 1.  Both inside: the group (s, s+1), Eqs. (cc)
// and (dd) from the shared old values a = u_{s-1}, b, c, d = u_{s+2} (the
// wall values beyond the grid); s = -1: point 0 alone (Saul'yev A); s + 1 = n:
// point n - 1 alone (Saul'yev B).  Only the two wall units branch, so a warp
// runs one FMA chain per group member (one thread per point had neighbouring
// lanes on the two different chains of (cc) and (dd)).
template <typename Real>
__global__ void __launch_bounds__(256) canon_kernel(const Real *__restrict__ in, Real *__restrict__ out,
                                                    long long n, int parity, Coef<Real> k)
{
    const long long units = (n + parity + 1) / 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += stride) {
        const long long s = 2 * u - parity;
        if (s >= 0 && s + 1 < n) {
            const Real a = (s == 0) ? k.bl : in[s - 1];
            const Real b = in[s];
            const Real c = in[s + 1];
            const Real d = (s + 2 == n) ? k.br : in[s + 2];
            // Eq. (cc), left member, terms in printed order
            out[s] = fma_rn(k.c4, d, fma_rn(k.c3, c, fma_rn(k.c2, b, mul_rn(k.c1, a))));
            // Eq. (dd), right member
            out[s + 1] = fma_rn(k.c1, d, fma_rn(k.c2, c, fma_rn(k.c3, b, mul_rn(k.c4, a))));
        } else if (s < 0) {
            // left singleton: Saul'yev A, Eq. (aa), new-level neighbour = beta_l
            const Real far = (n == 1) ? k.br : in[1];
            out[0] = fma_rn(k.s0, far, fma_rn(k.s1, in[0], mul_rn(k.s0, k.bl)));
        } else {
            // right singleton: Saul'yev B, Eq. (bb), new-level neighbour = beta_r
            const Real far = (n == 1) ? k.bl : in[n - 2];
            out[n - 1] = fma_rn(k.s0, far, fma_rn(k.s1, in[n - 1], mul_rn(k.s0, k.br)));
        }
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
    const long long units = (n + parity + 1) / 2;
    long long blocks = (units + threads - 1) / threads;
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
