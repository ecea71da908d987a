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
// use the array's name as a device address, so the first call in each CUDA
// context looks the address up with cudaGetSymbolAddress (with that device
// current) and caches it under the context's unique id (a context created
// after cudaDeviceReset, or a non-primary one, gets its own lookup); make
// that first call before any stream capture.  All calls share the array:
// calls that overlap on the GPU (different streams, or threads) race on it.
// Nothing in it needs clearing between calls, because each call writes
// every scratch element it reads; the fault word of the sweeps (also static)
// is cleared at the start of every call.
#include <cuda.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/spde.h"
#include "internal.h"

namespace {

constexpr size_t kNoallocScratchBytes = 16u << 20;  // 16 MiB
constexpr int kMaxCached = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];
// the V-cycle sweeps' fault word of these calls (raised when a bounded wait gives up)
static __device__ __align__(16) int g_noalloc_fault;

std::mutex g_noalloc_mu;
struct Cached {
    unsigned long long ctx_id;
    void* scratch;
    int* fault;
};
Cached g_cache[kMaxCached];
int g_ncache = 0;

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

// unique id of the current CUDA context (driver entry points fetched at run time,
// so the library does not link against libcuda)
bool current_context_id(unsigned long long* id) {
    typedef CUresult (*CtxGetCurrent)(CUcontext*);
    typedef CUresult (*CtxGetId)(CUcontext, unsigned long long*);
    static CtxGetCurrent get_cur = nullptr;
    static CtxGetId get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<CtxGetCurrent>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetId>(p);
        cudaGetLastError();
        looked = true;
    }
    if (!get_cur || !get_id) return false;
    CUcontext c = nullptr;
    if (get_cur(&c) != CUDA_SUCCESS || !c) return false;
    return get_id(c, id) == CUDA_SUCCESS;
}

}  // namespace

namespace spde {
// reads (and then clears) the fault word of the allocation-free preconditioner calls on
// the current device; synchronises st
cudaError_t noalloc_take_fault(int* raised, cudaStream_t st) {
    *raised = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(raised, g_noalloc_fault, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && *raised) {
        static const int zero = 0;
        e = cudaMemcpyToSymbolAsync(g_noalloc_fault, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    return e;
}
}  // namespace spde

extern "C" spde_status spde_precond_noalloc(int n, double h, double kappa, int nsamples, int prec,
                                            const spde_opts* opts, const void* r, void* z, void* stream) {
    using namespace spde;
    const bool pow2 = n > 0 && (n & (n - 1)) == 0;
    // the grid limit of every other entry point (at most 2^29 cells: 32-bit block offsets)
    if (!pow2 || n < 4 || n > 512 || nsamples < 0 || nsamples > 65535 || !(h > 0.0) || !(kappa > 0.0) ||
        !std::isfinite(kappa))
        return noalloc_fail(SPDE_EINVAL, "bad size or parameters (n a power of two in [4, 512])");
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
    unsigned long long cid = 0;
    if (!current_context_id(&cid)) {
        cudaGetLastError();
        return noalloc_fail(SPDE_ECUDA, "no current CUDA context");
    }
    void* scratch = nullptr;
    int* fault = nullptr;
    {
        std::lock_guard<std::mutex> g(g_noalloc_mu);
        for (int i = 0; i < g_ncache; ++i)
            if (g_cache[i].ctx_id == cid) {
                scratch = g_cache[i].scratch;
                fault = g_cache[i].fault;
            }
        if (!scratch) {
            void* p = nullptr;
            void* f = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e == cudaSuccess) e = cudaGetSymbolAddress(&f, g_noalloc_fault);
            if (e != cudaSuccess || !p || !f) {
                cudaGetLastError();
                return noalloc_fail(SPDE_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                                    cudaGetErrorString(e));
            }
            scratch = p;
            fault = static_cast<int*>(f);
            if (g_ncache < kMaxCached) g_cache[g_ncache++] = Cached{cid, p, fault};
        }
    }
    spde_opts o;
    spde_opts_init(&o);
    if (opts) o = *opts;
    const double kh2 = (kappa * h) * (kappa * h);
    const int64_t n3 = (int64_t)n * n * n, N4 = 4 * n3;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // a timeout of an earlier call is reported once (spde_precond_status) and must not
    // make this call skip its sweeps
    if (mg_fault_clear(fault, st) != cudaSuccess) {
        const cudaError_t e = cudaGetLastError();
        return noalloc_fail(SPDE_ECUDA, "clearing the fault word failed: %s", cudaGetErrorString(e));
    }
    MGPlan plan;
    mg_plan_init(plan, n, kh2, o.schur_c, o.omega);
    plan.fault = fault;
    plan.sz_pref = o.sweep_planes;
    plan.coarse_fp16 = o.coarse_fp16 != 0;
    plan.sweep_rows = o.sweep_rows != 0;
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
