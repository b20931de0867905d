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

}  // namespace

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
