// spde_precond_noalloc: the block-diagonal preconditioner (spde_precond)
// for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code whose device memory is owned by
// another allocator (a framework's caching pool or a fixed arena that must
// account for every byte), and latency-critical loops where cudaMalloc /
// cudaFree would implicitly synchronise the device.  This entry point keeps
// the V-cycle's coarse-level scratch in a fixed array compiled into the
// library instead of allocating it.
//
// The array is file-scope device memory: every GPU that loads this library
// holds it (kNoallocScratchBytes) until the process exits.  Host code cannot
// use the array's name as a device address, so the first call on each device
// looks the address up with cudaGetSymbolAddress (with that device current)
// and caches it; make that first call before any stream capture.  All calls
// share the array: calls that overlap on the GPU (different streams, or
// threads) race on it.  Nothing in it needs clearing between calls, because
// each call writes every scratch element it reads.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/spde.h"
#include "internal.h"

namespace {

constexpr size_t kNoallocScratchBytes = 16u << 20;  // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// the message is what spde_last_error() returns on this thread
spde_status noalloc_fail(spde_status s, const char* fmt, ...) {
    char buf[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    spde::set_last_error(buf);
    return s;
}

}  // namespace

extern "C" spde_status spde_precond_noalloc(int n, double h, double kappa, int nsamples, int prec,
                                            const spde_opts* opts, const void* r, void* z, void* stream) {
    using namespace spde;
    const bool pow2 = n > 0 && (n & (n - 1)) == 0;
    if (!pow2 || n < 4 || n > 1024 || nsamples < 0 || nsamples > 65535 || !(h > 0.0) || !(kappa > 0.0) ||
        !std::isfinite(kappa))
        return noalloc_fail(SPDE_EINVAL, "bad size or parameters");
    if (prec != SPDE_PREC_FP64 && prec != SPDE_PREC_MIXED) return noalloc_fail(SPDE_EINVAL, "bad precision");
    if (nsamples == 0) return SPDE_OK;
    if (!r || !z) return noalloc_fail(SPDE_EINVAL, "null buffer");
    const size_t need = prec == SPDE_PREC_FP64 ? mg_scratch_elems<double>(n, nsamples) * sizeof(double)
                                               : mg_scratch_elems<float>(n, nsamples) * sizeof(float);
    if (need > kNoallocScratchBytes)
        return noalloc_fail(SPDE_EINVAL,
                            "needs %zu bytes of V-cycle scratch for n=%d, %d samples; the static scratch holds "
                            "%zu bytes (use fewer samples per call, or spde_precond)",
                            need, n, nsamples, kNoallocScratchBytes);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return noalloc_fail(SPDE_ECUDA, "no usable current device");
    }
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> g(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return noalloc_fail(SPDE_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                                    cudaGetErrorString(e));
            }
            g_noalloc_ptr[dev] = p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    spde_opts o;
    spde_opts_init(&o);
    if (opts) o = *opts;
    const double kh2 = (kappa * h) * (kappa * h);
    const int64_t n3 = (int64_t)n * n * n, N4 = 4 * n3;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    MGPlan plan;
    mg_plan_init(plan, n, kh2, o.schur_c, o.omega);
    int nb;
    if (prec == SPDE_PREC_FP64) {
        mg_plan_bind<double>(plan, nsamples, static_cast<double*>(scratch));
        const double* rr = static_cast<const double*>(r);
        double* zz = static_cast<double*>(z);
        launch_precond_u<double>(N4, (int)n3, nsamples, rr, zz, o.flux_diag, nullptr, nullptr, st);
        nb = launch_vcycle<double>(plan, nsamples, rr + 3 * n3, N4, zz + 3 * n3, N4, nullptr, nullptr, 0, st);
    } else {
        mg_plan_bind<float>(plan, nsamples, static_cast<float*>(scratch));
        const float* rr = static_cast<const float*>(r);
        float* zz = static_cast<float*>(z);
        launch_precond_u<float>(N4, (int)n3, nsamples, rr, zz, o.flux_diag, nullptr, nullptr, st);
        nb = launch_vcycle<float>(plan, nsamples, rr + 3 * n3, N4, zz + 3 * n3, N4, nullptr, nullptr, 0, st);
    }
    const cudaError_t e = cudaGetLastError();
    if (nb < 0 || e != cudaSuccess)
        return noalloc_fail(SPDE_ECUDA, "launch failed: %s", cudaGetErrorString(e));
    return SPDE_OK;
}
