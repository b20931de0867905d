// ge_sweep.cu -- the GE step with general sub-domain width k (arXiv:1310.3422
// Sec. 2: odd sub-domains [x_{2ik}, x_{2ik+k-1}], even sub-domains
// [x_{2ik+k}, x_{2(i+1)k-1}], Saul'yev A / B alternating between them and
// between the two steps of each pair, Eqs. (cc)/(dd) at the confluences).
//
// Paper node j (array index j-1, walls at j = 0 and n+1) lies in sub-domain
// s = floor(j/k).  At parity p it uses Saul'yev A (new-level neighbour on the
// left) when s + p is even, else Saul'yev B.  Where a B sub-domain meets the
// A sub-domain to its right, their two wall nodes form a coupled pair solved
// by Eqs. (cc)/(dd); from that pair the A run is swept to the right and the
// B run to the left.  One thread owns one such confluence unit (a B
// sub-domain followed by an A sub-domain, 2k nodes), the paper's own thread
// mapping ("sub-domain couples", Sec. 3): the sweeps are sequential
// recurrences.  A unit at the left wall has only its A part (swept from the
// wall value beta_l), one at the right wall only its B part (from beta_r).
//
// Every sum of products is a chain of fused multiply-adds in the order the
// equation prints its terms, so the FP64 result is bit-identical to a serial
// FP64 evaluation in that order.  k = 1 gives the 2-point group step.
#include "ge_internal.h"

namespace ge {
namespace {

template <typename Real>
struct SweepCoef {
    Real c1, c2, c3, c4, s0, s1, bl, br;
};

__device__ __forceinline__ double f_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float f_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double f_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float f_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

template <typename Real>
__global__ void __launch_bounds__(256) sweep_kernel(const Real *__restrict__ in, Real *__restrict__ out,
                                                    long long n, int parity, long long k, long long n_units,
                                                    SweepCoef<Real> c)
{
    // old value of paper node j (walls outside 1..n)
    auto old = [&](long long j) -> Real { return j == 0 ? c.bl : (j == n + 1 ? c.br : in[j - 1]); };
    // Saul'yev A / B at node j from its new-level neighbour `nb` and its
    // old-level far neighbour: (r nb + (1-r) u_j + r far) / (1+r)
    auto saulyev = [&](Real nb, long long j, long long far) -> Real {
        return f_fma(c.s0, old(far), f_fma(c.s1, in[j - 1], f_mul(c.s0, nb)));
    };
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n_units; u += stride) {
        const long long bA = 2 * u + parity;       // the unit's A sub-domain
        const long long a_lo = bA * k < 1 ? 1 : bA * k;
        const long long a_hi = bA * k + k - 1 > n ? n : bA * k + k - 1;
        const long long b_lo = (bA - 1) * k < 1 ? 1 : (bA - 1) * k;
        const long long b_hi = bA * k - 1 > n ? n : bA * k - 1;
        const bool has_a = a_lo <= a_hi, has_b = b_lo <= b_hi;
        if (has_a && has_b) {
            // confluence pair (j, j+1): B at j, A at j+1 -- Eqs. (cc), (dd)
            const long long j = bA * k - 1;
            const Real a = old(j - 1), b = old(j), cc = old(j + 1), d = old(j + 2);
            const Real y = f_fma(c.c4, d, f_fma(c.c3, cc, f_fma(c.c2, b, f_mul(c.c1, a))));
            const Real z = f_fma(c.c1, d, f_fma(c.c2, cc, f_fma(c.c3, b, f_mul(c.c4, a))));
            out[j - 1] = y;
            out[j] = z;
            Real prev = z;
            for (long long m = j + 2; m <= a_hi; ++m) {  // A run to the right
                prev = saulyev(prev, m, m + 1);
                out[m - 1] = prev;
            }
            prev = y;
            for (long long m = j - 1; m >= b_lo; --m) {  // B run to the left
                prev = saulyev(prev, m, m - 1);
                out[m - 1] = prev;
            }
        } else if (has_a) {  // left wall: A run from beta_l
            Real prev = c.bl;
            for (long long m = a_lo; m <= a_hi; ++m) {
                prev = saulyev(prev, m, m + 1);
                out[m - 1] = prev;
            }
        } else if (has_b) {  // right wall: B run from beta_r
            Real prev = c.br;
            for (long long m = b_hi; m >= b_lo; --m) {
                prev = saulyev(prev, m, m - 1);
                out[m - 1] = prev;
            }
        }
    }
}

// The same step with the CTA's units staged in shared memory: blockDim.x
// consecutive units (2k nodes each) are loaded with coalesced reads, every
// thread runs its unit's recurrences on its own padded shared-memory row
// (pitch 2k + 1 elements, odd, so the threads' rows fall in different
// banks), and the results leave with coalesced writes.  A thread reads the
// two old values just outside its unit (owned by its neighbours) before the
// barrier that precedes any update, so the in-place update is race free.
// Same arithmetic, in the same order, as sweep_kernel.
template <typename Real>
__global__ void __launch_bounds__(256) sweep_smem_kernel(const Real *__restrict__ in, Real *__restrict__ out,
                                                         long long n, int parity, int k, long long n_units,
                                                         SweepCoef<Real> c)
{
    extern __shared__ unsigned char sweep_smem[];
    Real *sm = reinterpret_cast<Real *>(sweep_smem);
    const int T = blockDim.x, t = threadIdx.x;
    const int w = 2 * k, pitch = 2 * k + 1;
    for (long long U0 = (long long)blockIdx.x * T; U0 < n_units; U0 += (long long)gridDim.x * T) {
        const long long base = (2 * U0 + parity - 1) * (long long)k;  // first node of unit U0
        const int units = (int)((n_units - U0) < T ? (n_units - U0) : T);
        const int span = units * w;
        for (int e = t; e < span; e += T) {
            const long long j = base + e;
            if (j >= 1 && j <= n)
                sm[(e / w) * pitch + e % w] = in[j - 1];
        }
        __syncthreads();
        const long long u = U0 + t;
        const long long ub = base + (long long)t * w;  // first node of this unit
        Real *row = sm + t * pitch;
        Real left = (Real)0, right = (Real)0;  // old values of nodes ub - 1 and ub + w
        if (t < units) {
            const long long jl = ub - 1, jr = ub + w;
            left = jl <= 0 ? c.bl : (jl > n ? c.br : (t > 0 ? sm[(t - 1) * pitch + w - 1] : in[jl - 1]));
            right = jr <= 0 ? c.bl : (jr > n ? c.br : (t + 1 < units ? sm[(t + 1) * pitch] : in[jr - 1]));
        }
        __syncthreads();
        if (t < units) {
            auto old = [&](long long j) -> Real {
                if (j == 0)
                    return c.bl;
                if (j == n + 1)
                    return c.br;
                if (j < ub)
                    return left;
                if (j >= ub + w)
                    return right;
                return row[j - ub];
            };
            auto saulyev = [&](Real nb, long long j, long long far) -> Real {
                return f_fma(c.s0, old(far), f_fma(c.s1, row[j - ub], f_mul(c.s0, nb)));
            };
            const long long bA = 2 * u + parity;
            const long long a_lo = bA * k < 1 ? 1 : bA * k;
            const long long a_hi = bA * k + k - 1 > n ? n : bA * k + k - 1;
            const long long b_lo = (bA - 1) * k < 1 ? 1 : (bA - 1) * k;
            const long long b_hi = bA * k - 1 > n ? n : bA * k - 1;
            const bool has_a = a_lo <= a_hi, has_b = b_lo <= b_hi;
            if (has_a && has_b) {
                const long long j = bA * k - 1;
                const Real a = old(j - 1), b = old(j), cc = old(j + 1), d = old(j + 2);
                const Real y = f_fma(c.c4, d, f_fma(c.c3, cc, f_fma(c.c2, b, f_mul(c.c1, a))));
                const Real z = f_fma(c.c1, d, f_fma(c.c2, cc, f_fma(c.c3, b, f_mul(c.c4, a))));
                Real prev = z;
                // A run to the right: reads old values at m and m + 1 before m is overwritten
                for (long long m = j + 2; m <= a_hi; ++m) {
                    const Real nv = saulyev(prev, m, m + 1);
                    row[m - ub] = nv;
                    prev = nv;
                }
                prev = y;
                for (long long m = j - 1; m >= b_lo; --m) {  // B run to the left
                    const Real nv = saulyev(prev, m, m - 1);
                    row[m - ub] = nv;
                    prev = nv;
                }
                row[j - ub] = y;
                row[j + 1 - ub] = z;
            } else if (has_a) {
                Real prev = c.bl;
                for (long long m = a_lo; m <= a_hi; ++m) {
                    const Real nv = saulyev(prev, m, m + 1);
                    row[m - ub] = nv;
                    prev = nv;
                }
            } else if (has_b) {
                Real prev = c.br;
                for (long long m = b_hi; m >= b_lo; --m) {
                    const Real nv = saulyev(prev, m, m - 1);
                    row[m - ub] = nv;
                    prev = nv;
                }
            }
        }
        __syncthreads();
        for (int e = t; e < span; e += T) {
            const long long j = base + e;
            if (j >= 1 && j <= n)
                out[j - 1] = sm[(e / w) * pitch + e % w];
        }
        __syncthreads();
    }
}

// D steps per launch on a tile kept in shared memory.  A tile covers NU
// units of the first step's grouping (nodes [T0, T0 + 2k NU)); nodes are
// stored with one pad slot after every 2k, so the threads' units (2k nodes,
// shifted by k on alternate steps) fall in different banks.  One step
// changes a unit from the old values of the unit and one node on each side,
// so the valid part of the tile shrinks by at most 2k + 1 nodes per side per
// step: the tile writes back its inner NU - 2 HU units, HU = D + 1 +
// ceil(D / 2k).  Each step every thread reads the two old values just
// outside its unit, the CTA synchronises, and the unit is updated in place
// with the arithmetic of sweep_smem_kernel, in the same order.
template <typename Real>
__global__ void __launch_bounds__(256) sweep_tb_kernel(const Real *__restrict__ in, Real *__restrict__ out, long long n,
                                                       int parity, int k, int steps, int NU, int HU,
                                                       long long n_tiles, SweepCoef<Real> c)
{
    extern __shared__ unsigned char sweep_smem[];
    Real *sm = reinterpret_cast<Real *>(sweep_smem);
    const int t = threadIdx.x;
    const int w = 2 * k;
    const int span = NU * w;  // tile nodes
    const long long out_units = NU - 2 * HU;
    for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        // first node of the tile: unit (tile * out_units - HU) of the first step's grouping
        const long long T0 = ((long long)(parity - 1) + 2 * (tile * out_units - HU)) * k;
        for (int e = t; e < span; e += blockDim.x) {
            const long long j = T0 + e;
            if (j >= 1 && j <= n)
                sm[e + e / w] = in[j - 1];
        }
        __syncthreads();
        for (int st = 0; st < steps; ++st) {
            // this step's units start at local node e0 = off + w * i (off = 0 on
            // the first step's grouping, k on the other); the partial ones at
            // the tile's ends are skipped
            const int off = (st & 1) ? k : 0;
            const int nu = (st & 1) ? NU - 1 : NU;
            const bool active = t < nu;
            const int e0 = off + w * t;
            const long long ub = T0 + e0;  // first node of this thread's unit
            const int base = e0 + e0 / w;
            const int split = w - (e0 % w);  // nodes of the unit before the next pad slot
            auto addr = [&](long long jj) -> int {
                const int i = (int)(jj - ub);
                return base + i + (i >= split ? 1 : 0);
            };
            Real left = (Real)0, right = (Real)0;  // old values of nodes ub - 1 and ub + w
            if (active) {
                const long long jl = ub - 1, jr = ub + w;
                if (e0 >= 1 && jl >= 1 && jl <= n)
                    left = sm[(e0 - 1) + (e0 - 1) / w];
                if (e0 + w < span && jr >= 1 && jr <= n)
                    right = sm[(e0 + w) + (e0 + w) / w];
            }
            __syncthreads();
            if (active) {
                auto old = [&](long long j) -> Real {
                    if (j == 0)
                        return c.bl;
                    if (j == n + 1)
                        return c.br;
                    if (j < ub)
                        return left;
                    if (j >= ub + w)
                        return right;
                    return sm[addr(j)];
                };
                auto saulyev = [&](Real nb, long long j, long long far) -> Real {
                    return f_fma(c.s0, old(far), f_fma(c.s1, sm[addr(j)], f_mul(c.s0, nb)));
                };
                const long long bA = ub / k + 1;  // the unit's A sub-domain
                const long long a_lo = bA * k < 1 ? 1 : bA * k;
                const long long a_hi = bA * k + k - 1 > n ? n : bA * k + k - 1;
                const long long b_lo = (bA - 1) * k < 1 ? 1 : (bA - 1) * k;
                const long long b_hi = bA * k - 1 > n ? n : bA * k - 1;
                const bool has_a = a_lo <= a_hi, has_b = b_lo <= b_hi;
                if (has_a && has_b) {
                    const long long j = bA * k - 1;
                    const Real a = old(j - 1), b = old(j), cc = old(j + 1), d = old(j + 2);
                    const Real y = f_fma(c.c4, d, f_fma(c.c3, cc, f_fma(c.c2, b, f_mul(c.c1, a))));
                    const Real z = f_fma(c.c1, d, f_fma(c.c2, cc, f_fma(c.c3, b, f_mul(c.c4, a))));
                    Real prev = z;
                    for (long long m = j + 2; m <= a_hi; ++m) {  // A run to the right
                        const Real nv = saulyev(prev, m, m + 1);
                        sm[addr(m)] = nv;
                        prev = nv;
                    }
                    prev = y;
                    for (long long m = j - 1; m >= b_lo; --m) {  // B run to the left
                        const Real nv = saulyev(prev, m, m - 1);
                        sm[addr(m)] = nv;
                        prev = nv;
                    }
                    sm[addr(j)] = y;
                    sm[addr(j + 1)] = z;
                } else if (has_a) {
                    Real prev = c.bl;
                    for (long long m = a_lo; m <= a_hi; ++m) {
                        const Real nv = saulyev(prev, m, m + 1);
                        sm[addr(m)] = nv;
                        prev = nv;
                    }
                } else if (has_b) {
                    Real prev = c.br;
                    for (long long m = b_hi; m >= b_lo; --m) {
                        const Real nv = saulyev(prev, m, m - 1);
                        sm[addr(m)] = nv;
                        prev = nv;
                    }
                }
            }
            __syncthreads();
        }
        // write back the tile's inner units
        const int o_lo = HU * w, o_hi = (NU - HU) * w;
        for (int e = o_lo + t; e < o_hi; e += blockDim.x) {
            const long long j = T0 + e;
            if (j >= 1 && j <= n)
                out[j - 1] = sm[e + e / w];
        }
        __syncthreads();
    }
}

template <typename Real>
cudaError_t launch_sweep_t(const Real *in, Real *out, long long n, int parity, long long k, const CanonCoef &cf,
                           cudaStream_t s)
{
    SweepCoef<Real> c{(Real)cf.c1, (Real)cf.c2, (Real)cf.c3, (Real)cf.c4,
                      (Real)cf.s0, (Real)cf.s1, (Real)cf.beta_l, (Real)cf.beta_r};
    // units u = 0.. cover sub-domains up to floor(n / k)
    const long long last_block = n / k;
    const long long n_units = (last_block + 1 - parity) / 2 + 1;
    // staged in shared memory when 32 or more units fit a CTA's 227 KB
    const long long per_unit = (2 * k + 1) * (long long)sizeof(Real);
    const long long max_smem = 227 * 1024;
    int threads = 256;
    while (threads > 32 && threads * per_unit > max_smem)
        threads -= 32;
    if (threads * per_unit <= max_smem) {
        const int smem = (int)(threads * per_unit);
        cudaError_t e = cudaFuncSetAttribute(sweep_smem_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess)
            return e;
        long long blocks = (n_units + threads - 1) / threads;
        if (blocks > (1LL << 20))
            blocks = 1LL << 20;
        sweep_smem_kernel<Real><<<(unsigned)blocks, threads, smem, s>>>(in, out, n, parity, (int)k, n_units, c);
        return cudaGetLastError();
    }
    threads = 256;
    long long blocks = (n_units + threads - 1) / threads;
    if (blocks > (1LL << 20))
        blocks = 1LL << 20;
    sweep_kernel<Real><<<(unsigned)blocks, threads, 0, s>>>(in, out, n, parity, k, n_units, c);
    return cudaGetLastError();
}

// Up to `steps` steps in one launch of sweep_tb_kernel; *done receives the
// steps taken.  0 when the width leaves too few units per tile (the caller
// then runs one step with launch_sweep_t).
template <typename Real>
cudaError_t launch_sweep_tb_t(const Real *in, Real *out, long long n, int parity, long long k, int steps,
                              const CanonCoef &cf, int *done, cudaStream_t s)
{
    *done = 0;
    if (k < 2 || steps < 1)
        return cudaSuccess;
    SweepCoef<Real> c{(Real)cf.c1, (Real)cf.c2, (Real)cf.c3, (Real)cf.c4,
                      (Real)cf.s0, (Real)cf.s1, (Real)cf.beta_l, (Real)cf.beta_r};
    const long long w = 2 * k;
    const long long max_smem = 227 * 1024;
    long long NU = max_smem / ((w + 1) * (long long)sizeof(Real));
    if (NU > 256)
        NU = 256;
    // steps per launch: the halo HU = D + 1 + ceil(D / 2k) units per side
    // leaves at least half of the tile's units as output
    int D = steps;
    auto halo = [&](int d) { return (long long)d + 1 + (d + w - 1) / w; };
    while (D > 1 && NU - 2 * halo(D) < NU / 2)
        --D;
    if (NU < 64 || NU - 2 * halo(D) < 1)
        return cudaSuccess;
    const int HU = (int)halo(D);
    const long long out_units = NU - 2 * HU;
    // tiles cover nodes from (parity - 1) k up to n
    const long long first = (long long)(parity - 1) * k;
    const long long n_tiles = (n + 1 - first + out_units * w - 1) / (out_units * w);
    const int smem = (int)(NU * (w + 1) * (long long)sizeof(Real));
    cudaError_t e = cudaFuncSetAttribute(sweep_tb_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess)
        return e;
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_tb_kernel<Real>, 256, smem);
    if (e != cudaSuccess)
        return e;
    long long grid = (long long)sms * (per_sm > 0 ? per_sm : 1);
    if (grid > n_tiles)
        grid = n_tiles;
    sweep_tb_kernel<Real><<<(unsigned)grid, 256, smem, s>>>(in, out, n, parity, (int)k, D, (int)NU, HU, n_tiles, c);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        *done = D;
    return e;
}

}  // namespace

cudaError_t launch_sweep_tb_f64(const double *in, double *out, long long n, int parity, long long k, int steps,
                                const CanonCoef &c, int *done, cudaStream_t s)
{
    return launch_sweep_tb_t<double>(in, out, n, parity, k, steps, c, done, s);
}

cudaError_t launch_sweep_tb_f32(const float *in, float *out, long long n, int parity, long long k, int steps,
                                const CanonCoef &c, int *done, cudaStream_t s)
{
    return launch_sweep_tb_t<float>(in, out, n, parity, k, steps, c, done, s);
}

cudaError_t launch_sweep_f64(const double *in, double *out, long long n, int parity, long long k,
                             const CanonCoef &c, cudaStream_t s)
{
    return launch_sweep_t<double>(in, out, n, parity, k, c, s);
}

cudaError_t launch_sweep_f32(const float *in, float *out, long long n, int parity, long long k,
                             const CanonCoef &c, cudaStream_t s)
{
    return launch_sweep_t<float>(in, out, n, parity, k, c, s);
}

}  // namespace ge
