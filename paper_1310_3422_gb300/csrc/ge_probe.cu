// ge_probe.cu -- register-only fused multiply-add throughput probe (FP64 and
// FP32), the measured ALU ceiling that the tiled kernels' roofline is read
// against.  The paper has no counterpart.
//
// Every thread runs `chains` (4, 8, 16 or 32) independent multiply-add chains
// x <- x * a + b for `iters` iterations, entirely in registers (no memory
// traffic in the loop), and stores its chain sum once at the end so that
// nothing is eliminated.  With a <= 1 and b small the values stay finite and
// normal.  The caller times the launch (CUDA events on the same stream) and
// may sweep the CTAs per SM and the chains per thread for the best rate; the
// multiply-adds done are blocks * kThreads * chains * iters.
#include <cuda_runtime.h>

#include <cstdint>

#include "ge.h"
#include "ge_dfma_emu.cuh"
#include "ge_internal.h"

namespace {

constexpr int kThreads = 256;

template <typename Real, int kChains>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(long long iters, Real a, Real b, Real *sink)
{
    Real x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        x[c] = (Real)(threadIdx.x + c) * (Real)1e-3;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c)
            x[c] = fma(x[c], a, b);
    }
    Real s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        s += x[c];
    sink[(size_t)blockIdx.x * kThreads + threadIdx.x] = s;
}

template <typename Real>
void launch_probe(int chains, int blocks, long long iters, Real a, Real b, Real *sink, cudaStream_t s)
{
    switch (chains) {
    case 4: fma_probe_kernel<Real, 4><<<blocks, kThreads, 0, s>>>(iters, a, b, sink); break;
    case 8: fma_probe_kernel<Real, 8><<<blocks, kThreads, 0, s>>>(iters, a, b, sink); break;
    case 16: fma_probe_kernel<Real, 16><<<blocks, kThreads, 0, s>>>(iters, a, b, sink); break;
    default: fma_probe_kernel<Real, 32><<<blocks, kThreads, 0, s>>>(iters, a, b, sink); break;
    }
}

// The integer-pipe FMA against the FP64 unit's on every input: counts[0] =
// inputs where a fast path reported ok but gave other bits than the FP64
// unit's fma (must stay 0), counts[1] = inputs the general fast path took,
// counts[2] = inputs the addition-only fast path took (same-sign inputs).
__global__ void emu_check_kernel(double g, const double *__restrict__ p, const double *__restrict__ x, long long n,
                                 unsigned long long *counts)
{
    const ge::EmuG eg = ge::emu_g(g);
    const bool usable = ge::emu_g_usable(eg);
    unsigned long long bad = 0, fast = 0, fast_add = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double want = __fma_rn(g, p[i], x[i]);
        bool ok;
        const double e = ge::emu_fma(eg, p[i], x[i], ok);
        if (ok && usable) {
            ++fast;
            bad += __double_as_longlong(e) != __double_as_longlong(want);
        }
        const unsigned same = ((unsigned)__double2hiint(p[i]) ^ (unsigned)__double2hiint(x[i]) ^
                               ((unsigned)eg.s << 31)) >> 31;
        if (same == 0u) {
            const double e2 = ge::emu_fma_add(eg, p[i], x[i], ok);
            if (ok && usable) {
                ++fast_add;
                bad += __double_as_longlong(e2) != __double_as_longlong(want);
            }
        }
    }
    atomicAdd(counts, bad);
    atomicAdd(counts + 1, fast);
    atomicAdd(counts + 2, fast_add);
}

}  // namespace

extern "C" ge_status ge_emu_fma_check(double g, const double *p_dev, const double *x_dev, int64_t n,
                                      uint64_t *counts_dev, void *stream)
{
    if (!p_dev || !x_dev || !counts_dev || n < 0) {
        ge::set_last_error("ge_emu_fma_check: NULL buffer or n < 0");
        return GE_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(counts_dev, 0, 3 * sizeof(uint64_t), s);
    if (e == cudaSuccess && n > 0) {
        const long long blocks = (n + kThreads - 1) / kThreads;
        emu_check_kernel<<<(int)(blocks < 4096 ? blocks : 4096), kThreads, 0, s>>>(
            g, p_dev, x_dev, n, reinterpret_cast<unsigned long long *>(counts_dev));
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        ge::set_last_error(cudaGetErrorString(e));
        return GE_ECUDA;
    }
    return GE_OK;
}

extern "C" ge_status ge_probe_fma(int32_t prec, int32_t blocks, int32_t chains, int64_t iters, void *sink_dev,
                                  void *stream)
{
    if ((prec != GE_F64 && prec != GE_F32) || blocks < 1 || iters < 1 || !sink_dev ||
        (chains != 4 && chains != 8 && chains != 16 && chains != 32)) {
        ge::set_last_error("ge_probe_fma: need prec GE_F64 or GE_F32, blocks >= 1, chains 4, 8, 16 or 32, "
                           "iters >= 1, a sink");
        return GE_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (prec == GE_F64)
        launch_probe<double>(chains, blocks, iters, 0.999999, 1e-7, static_cast<double *>(sink_dev), s);
    else
        launch_probe<float>(chains, blocks, iters, 0.9999f, 1e-5f, static_cast<float *>(sink_dev), s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        ge::set_last_error(cudaGetErrorString(e));
        return GE_ECUDA;
    }
    return GE_OK;
}
