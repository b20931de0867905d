// ge_noalloc.cu -- ge_solve_noalloc: the tiled GE solve for callers that may
// not allocate device memory.
//
// Who needs it: code that runs where the process's device memory belongs to
// someone else -- a plug-in inside a host application or inference server
// that hands out all device memory through its own pool, a real-time loop
// that must not take cudaMalloc's implicit device synchronisation, or a
// sandbox that forbids driver allocations after start-up.  Such callers
// provide their input and output buffers and get the solve without any
// cudaMalloc, cudaFree or other allocating call.
//
// The working buffers the tiled kernel needs (two ping-pong states padded
// to whole 128-byte rows, and the device error word) live in one file-scope
// static device array of fixed size (16 MiB + 256 bytes).  Once created on a
// device it stays there until the process exits.
//
// Set-up: the first call on a device, with that device current, looks the
// array's device address up with cudaGetSymbolAddress (host code cannot use
// the array's name as a device address) and remembers it for that device.
// With CUDA's default lazy module loading, that first call is also where the
// driver loads this file's module and the tiled kernel's module on the
// device and creates the array in device memory: those are driver
// allocations, with the synchronisation they imply.  So a caller that must
// not allocate later makes one warm-up call at start-up, on each device and
// for each precision it will use, with steps >= 1 (or runs the process with
// CUDA_MODULE_LOADING=EAGER, which loads every module when the context is
// created).  Make that first call before any stream capture.  After it,
// calls allocate nothing.
//
// Sharing: every call on a device uses the same array, which keeps the last
// call's contents.  A call clears what must start at zero (the error word
// and the padding after the last point) and overwrites the rest.  Two calls
// whose GPU work overlaps (different streams, or different host threads on
// one device) race on the array; callers must serialise them.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime_api.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "ge.h"
#include "ge_internal.h"

namespace {

constexpr long long kNoAllocMaxPoints = 1LL << 20;
constexpr size_t kNoAllocBufBytes = (size_t)kNoAllocMaxPoints * sizeof(double);  // whole rows
constexpr size_t kNoAllocErrOffset = 2 * kNoAllocBufBytes;
constexpr size_t kNoAllocBytes = kNoAllocErrOffset + 256;
static_assert(kNoAllocBufBytes % ge::kRowBytes == 0, "buffers must hold whole rows");

}  // namespace

// The shared working memory of ge_solve_noalloc (two state buffers + the
// device error word).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

// Failures are reported through ge_last_error(), like every other entry point.
ge_status nfail(ge_status st, const char *fmt, ...)
{
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    ge::set_last_error(msg);
    return st;
}

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
ge_status scratch_address(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return nfail(GE_ECUDA, "ge_solve_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices)
        return nfail(GE_EINVAL, "ge_solve_noalloc: device %d beyond the supported %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr)
            return nfail(GE_ECUDA, "ge_solve_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_ptr[dev];
    return GE_OK;
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

}  // namespace

extern "C" ge_status ge_solve_noalloc(int64_t n, double r, double beta_l, double beta_r, ge_precision prec,
                                      int32_t depth, int64_t steps, const void *u0_dev, void *u_out_dev,
                                      void *stream)
{
    if (n < 1 || n > kNoAllocMaxPoints)
        return nfail(GE_EINVAL, "ge_solve_noalloc: n = %lld outside 1..%lld (the fixed working-memory limit)",
                     (long long)n, kNoAllocMaxPoints);
    if (!(r > 0.0) || !std::isfinite(r) || !std::isfinite(beta_l) || !std::isfinite(beta_r))
        return nfail(GE_EINVAL, "ge_solve_noalloc: need a finite r > 0 and finite wall values");
    if (prec != GE_F64 && prec != GE_F32 && prec != GE_F32_COMP)
        return nfail(GE_EINVAL, "ge_solve_noalloc: unknown precision %d", (int)prec);
    if (depth < 0 || depth > 1023 || steps < 0)
        return nfail(GE_EINVAL, "ge_solve_noalloc: depth %d or steps %lld out of range", (int)depth,
                     (long long)steps);
    if (!u0_dev || !u_out_dev)
        return nfail(GE_EINVAL, "ge_solve_noalloc: NULL buffer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t esz = prec == GE_F64 ? sizeof(double) : sizeof(float);
    const int K = ge::kRowBytes / (int)esz;
    const long long n_rows = (n + K - 1) / K;

    unsigned char *base = nullptr;
    ge_status st = scratch_address(&base);
    if (st != GE_OK)
        return st;
    unsigned char *buf[2] = {base, base + kNoAllocBufBytes};
    int *err = reinterpret_cast<int *>(base + kNoAllocErrOffset);

    // zero what must start at zero: the error word and both buffers' padding
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
    const size_t used = (size_t)n * esz, rows_bytes = (size_t)n_rows * ge::kRowBytes;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b)
        if (rows_bytes > used)
            e = cudaMemsetAsync(buf[b] + used, 0, rows_bytes - used, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(buf[0], u0_dev, used, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess)
        return nfail(GE_ECUDA, "ge_solve_noalloc: preparing the working memory: %s", cudaGetErrorString(e));
    int cur = 0;

    if (steps > 0) {
        auto enc = encoder();
        if (!enc)
            return nfail(GE_ECUDA, "ge_solve_noalloc: cuTensorMapEncodeTiled is not available");
        alignas(64) CUtensorMap tmap[2];
        for (int b = 0; b < 2; ++b) {
            cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)n_rows};
            cuuint64_t strides[1] = {(cuuint64_t)ge::kRowBytes};
            cuuint32_t box[2] = {(cuuint32_t)K, (cuuint32_t)ge::kTileRows};
            cuuint32_t estr[2] = {1, 1};
            CUresult cr = enc(&tmap[b], prec == GE_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                              2, buf[b], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (cr != CUDA_SUCCESS)
                return nfail(GE_ECUDA, "ge_solve_noalloc: cuTensorMapEncodeTiled failed (%d)", (int)cr);
        }
        // coefficients of the tiled kernel (right-hand-side form, Sec. 2) and
        // its launches, planned by the same code as the context API's
        const int pidx = prec == GE_F64 ? 0 : (prec == GE_F32 ? 1 : 2);
        ge::TbParams base_p{};
        double growth_lo = 0.0;
        ge::tb_fill_base(r, beta_l, beta_r, pidx, &base_p, &growth_lo);
        const int d = depth > 0 ? depth : (prec == GE_F64 ? ge::kDefaultDepthF64 : ge::kDefaultDepthF32);
        int bps = 0, sms = 0, dev = 0;
        e = ge::tb_occupancy(pidx, &bps);
        if (e == cudaSuccess)
            e = cudaGetDevice(&dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || bps < 1)
            return nfail(GE_ECUDA, "ge_solve_noalloc: occupancy query failed");
        ge::TbTarget t{};
        t.tmap[0] = &tmap[0];
        t.tmap[1] = &tmap[1];
        t.buf[0] = buf[0];
        t.buf[1] = buf[1];
        t.n = n;
        t.n_rows = n_rows;
        t.err = err;
        t.tile_ctr = err + 48;  // the launches' two tile-queue words (48, 49)
        t.grid_cap = (long long)sms * bps;
        e = ge::tb_run(t, base_p, growth_lo, false, pidx, &cur, 0, steps, d, s);
        if (e == cudaErrorInvalidValue)
            return nfail(GE_EINVAL, "ge_solve_noalloc: depth %d does not fit a tile", d);
        if (e != cudaSuccess)
            return nfail(GE_ECUDA, "ge_solve_noalloc: launch: %s", cudaGetErrorString(e));
    }
    // the result and the error word travel on the caller's stream; one
    // synchronisation of that stream ends the call
    int word = 0;
    e = cudaMemcpyAsync(u_out_dev, buf[cur], used, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&word, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return nfail(GE_ECUDA, "ge_solve_noalloc: %s", cudaGetErrorString(e));
    if (word == ge::kDevTimeout)
        return nfail(GE_ETIMEOUT, "ge_solve_noalloc: a tile load did not complete within the wait limit");
    return GE_OK;
}
