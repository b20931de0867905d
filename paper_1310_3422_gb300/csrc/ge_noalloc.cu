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
// static device array of fixed size.  Every GPU that loads this library
// holds it (16 MiB + 256 bytes) until the process exits.
//
// Set-up: the first call on a device, with that device current, looks the
// array's device address up with cudaGetSymbolAddress (host code cannot use
// the array's name as a device address) and remembers it for that device.
// Make that first call before any stream capture.
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
        // coefficients of the tiled kernel (right-hand-side form, Sec. 2)
        const double det = 1.0 + 2.0 * r;
        ge::TbParams base_p{};
        base_p.g = 2.0 * r;
        double onepg_lo = 0.0;
        ge::scaled_growth(r, prec == GE_F32, &base_p.onepg, &onepg_lo);
        base_p.r = r;
        base_p.omr = 1.0 - r;
        base_p.d = 2.0 * r / det;
        base_p.f_l = r * beta_l;
        base_p.f_r = r * beta_r;
        const double x1 = (1.0 + r) / det, x2 = r / det, xs = 1.0 / (1.0 + r);
        int every = 0;
        if (prec == GE_F32_COMP) {
            base_p.kappa = (1.0 - r) / (1.0 + r);
        } else {
            base_p.kappa = det * (1.0 - r) / (1.0 + r);
            const double headroom = prec == GE_F64 ? 256.0 : 64.0;
            every = (int)std::floor(headroom / std::log2(1.0 + 2.0 * r));
            if (every < 1)
                every = 1;
        }
        base_p.rescale_every = every;
        base_p.stall = 0;
        int d = depth > 0 ? depth : (prec == GE_F64 ? 48 : 128);
        if (every > 0 && d > (ge::kMaxRescale - 1) * every)
            d = (ge::kMaxRescale - 1) * every;
        if (d > ge::kMaxTableSteps)
            d = ge::kMaxTableSteps;
        const int pidx = prec == GE_F64 ? 0 : (prec == GE_F32 ? 1 : 2);
        int bps = 0, sms = 0, dev = 0;
        e = ge::tb_occupancy(pidx, &bps);
        if (e == cudaSuccess)
            e = cudaGetDevice(&dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || bps < 1)
            return nfail(GE_ECUDA, "ge_solve_noalloc: occupancy query failed");

        double sigma = 1.0, sigma_lo = 0.0;  // double-double scale
        int until = every;
        long long n0 = 0;
        while (n0 < steps) {
            const long long L = (steps - n0 < d) ? steps - n0 : d;
            ge::TbParams p = base_p;
            const bool last = (n0 + L == steps);
            p.do_entry = (n0 == 0) ? 1 : 0;
            p.n_mid = (int)(last ? L - 1 : L);
            p.do_exit = last ? 1 : 0;
            p.p_first = (int)(n0 & 1);
            p.sigma_in = sigma;
            p.rescale_phase = until;
            if (every > 0) {
                int ev = 0;
                for (int m = 0; m < p.n_mid; ++m) {
                    ge::dd_mul(sigma, sigma_lo, p.onepg, onepg_lo);
                    if (--until == 0) {
                        until = every;
                        int e2 = 0;
                        std::frexp(sigma, &e2);
                        p.rs_exp[ev++] = (short)(e2 - 1);
                        sigma = std::ldexp(sigma, -(e2 - 1));
                        sigma_lo = std::ldexp(sigma_lo, -(e2 - 1));
                    }
                }
            }
            p.x1 = ge::dd_div(x1, sigma, sigma_lo);
            p.x2 = ge::dd_div(x2, sigma, sigma_lo);
            p.xs = ge::dd_div(xs, sigma, sigma_lo);
            const int reach = p.do_entry + p.n_mid + p.do_exit;
            if (!ge::tb_geometry(pidx, reach, &p.H, &p.U))
                return nfail(GE_EINVAL, "ge_solve_noalloc: depth %d does not fit a tile", d);
            p.n = n;
            p.n_rows = n_rows;
            p.n_tiles = (n + p.U - 1) / p.U;
            p.out = buf[cur ^ 1];
            p.err = err;
            p.tile_ctr = err + 48;  // the launch's tile queue, zeroed first
            long long grid = (long long)sms * bps;
            if (grid > p.n_tiles)
                grid = p.n_tiles;
            e = cudaMemsetAsync(p.tile_ctr, 0, sizeof(int), s);
            if (e == cudaSuccess)
                e = ge::launch_tb(pidx, &tmap[cur], p, (int)grid, s);
            if (e != cudaSuccess)
                return nfail(GE_ECUDA, "ge_solve_noalloc: launch: %s", cudaGetErrorString(e));
            cur ^= 1;
            n0 += L;
        }
    }
    e = cudaMemcpyAsync(u_out_dev, buf[cur], used, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return nfail(GE_ECUDA, "ge_solve_noalloc: %s", cudaGetErrorString(e));
    int word = 0;
    e = cudaMemcpy(&word, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return nfail(GE_ECUDA, "ge_solve_noalloc: reading the error word: %s", cudaGetErrorString(e));
    if (word == ge::kDevTimeout)
        return nfail(GE_ETIMEOUT, "ge_solve_noalloc: a tile load did not complete within the wait limit");
    return GE_OK;
}
