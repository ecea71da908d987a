// C ABI of the sampler: contexts, embedding grids, meshes and the sampling
// driver (noise -> FP64 iterative refinement around batched MINRES ->
// projection + exp).  Every numerical step runs in this library's kernels.
#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/spde.h"
#include "internal.h"
#include "prof.h"

using namespace spde;

namespace spde {
thread_local Profiler* t_prof = nullptr;
void set_last_error(const char* msg);
const char* const kProfNames[PK_NCLASS] = {"noise",   "sumsq",  "residual64", "minres_A",  "alpha",
                                           "minres_B", "mg_down", "mg_coarse",  "mg_up",     "givens",
                                           "minres_D", "add_correction", "transpose_theta", "project_exp", "flux_from_theta", "schur_apply", "cg_update", "other"};
}  // namespace spde

namespace {

thread_local std::string g_err;

spde_status fail(spde_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
spde_status fail(spde_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

#define CUDA_TRY(x)                                                                                   \
    do {                                                                                              \
        cudaError_t e_ = (x);                                                                         \
        if (e_ != cudaSuccess) {                                                                      \
            cudaGetLastError(); /* clear a non-sticky error so later calls do not report it */        \
            return fail(e_ == cudaErrorMemoryAllocation ? SPDE_ENOMEM : SPDE_ECUDA, "%s: %s (%s:%d)", \
                        #x, cudaGetErrorString(e_), __FILE__, __LINE__);                              \
        }                                                                                             \
    } while (0)

#define STATUS_TRY(x)                       \
    do {                                    \
        spde_status s_ = (x);               \
        if (s_ != SPDE_OK) return s_;       \
    } while (0)

// g of Sec. 4 for nu = 1/2, d = 3, times sigma:
// (4 pi)^{3/4} kappa^{1/2} sqrt(Gamma(2) / Gamma(1/2)) sigma = sqrt(8 pi kappa) sigma
double g_half(double kappa, double sigma) { return sigma * std::sqrt(8.0 * M_PI * kappa); }

// Reduction the FP32 inner solve of a column aims for in one refinement step:
// opts.inner_tol (its precision floor), loosened to what the column still needs,
// 0.1 tol / rel, when that is larger (the last step of a solve to 1e-8 need not
// reach 1e-5).  A function of the column's own residual only, so a column's
// iterates do not depend on the other columns of its batch.
double inner_tol_for(const spde_opts& o, double rel) {
    return std::max(o.inner_tol, 0.1 * o.tol / std::max(rel, 1e-300));
}

// MINRES iterations between two host checks of the active columns at most
constexpr int kMaxChunk = 64;

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Cells of one grid at most: the kernels index a sample's four blocks with
// 32-bit offsets up to 4 x cells, which must stay below 2^31.
constexpr int64_t kMaxGridCells = int64_t(1) << 29;

template <typename T>
spde_status dev_alloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) return SPDE_OK;
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(SPDE_ENOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
    }
    return SPDE_OK;
}

template <typename T>
void dev_free(T*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}

// Solver workspace for S columns of one grid size and inner precision.
struct Workspace {
    Grid3 g;
    int S = 0, inner64 = -1;
    double* x64 = nullptr;   // [S][4n^3] refinement iterate (scaled unknowns)
    double* F = nullptr;     // [S][n^3] cell block of the scaled RHS
    void* vec[7] = {};       // inner vectors: d, wA, wB ([S][n^3], cell block only), r1, r2, yA, yB
    double* tri = nullptr;   // Thomas factors of the flux mass matrix T (2n - 2)
    float* tri32 = nullptr;  // the same in FP32 (Schur-complement operator)
    CgCol* cg = nullptr;     // Schur-complement CG state [S]
    void* mg = nullptr;      // V-cycle scratch
    double* partA = nullptr; // partial sums [S][kMaxPartials]: y.Ay of Lanczos pass A, then r1.y of pass B
    double* partB = nullptr;
    double* partC = nullptr;
    double* partR = nullptr;
    double* colv = nullptr;  // [2S] per-column reductions
    double* coltol = nullptr;  // [S] per-column tolerance of the FP32 inner solve
    double* h_tol = nullptr;   // pinned [S]
    MinresCol* st = nullptr;
    int* nact = nullptr;
    int* fault = nullptr;    // fault word of this workspace's V-cycle sweeps
    // graph-driven solves: device control block, the columns to correct, the
    // executable graphs captured for this workspace, and the event that marks the
    // end of the last call enqueued on it (calls on other streams wait for it)
    RefineCtl* ctl = nullptr;
    int* mask = nullptr;
    cudaEvent_t done = nullptr;
    // the options the solves on this workspace run with (the context's, with the level's
    // tuning applied; set by every call before it solves)
    spde_opts o{};
    struct Graph {
        int S, t64, warm, count;
        const void* fields;
        double kh2;
        cudaGraphExec_t exec;
    };
    std::vector<Graph> graphs;

    // wait until the last call enqueued on this workspace has finished
    void quiesce() {
        if (done) cudaEventSynchronize(done);
        cudaGetLastError();
    }
    void drop_graphs() {
        for (auto& gr : graphs) cudaGraphExecDestroy(gr.exec);
        graphs.clear();
    }
    int* h_nact = nullptr;   // pinned
    double* h_col = nullptr; // pinned [2S]
    MinresCol* h_st = nullptr;
    float* thetaT = nullptr; // [n^3][S]

    void release() {
        quiesce();
        drop_graphs();
        if (done) cudaEventDestroy(done);
        done = nullptr;
        dev_free(ctl);
        dev_free(mask);
        dev_free(x64);
        dev_free(F);
        for (auto& v : vec) {
            if (v) cudaFree(v);
            v = nullptr;
        }
        if (mg) cudaFree(mg);
        mg = nullptr;
        dev_free(partA);
        dev_free(partB);
        dev_free(partC);
        dev_free(partR);
        dev_free(colv);
        dev_free(coltol);
        dev_free(st);
        dev_free(nact);
        dev_free(fault);
        dev_free(thetaT);
        dev_free(tri);
        dev_free(tri32);
        dev_free(cg);
        if (h_nact) cudaFreeHost(h_nact);
        if (h_col) cudaFreeHost(h_col);
        if (h_st) cudaFreeHost(h_st);
        if (h_tol) cudaFreeHost(h_tol);
        h_tol = nullptr;
        h_nact = nullptr;
        h_col = nullptr;
        h_st = nullptr;
        g = Grid3();
        S = 0;
        inner64 = -1;
    }
};

int64_t workspace_bytes(const Grid3& g, int S, bool inner64) {
    const int64_t n3 = g.cells(), N4 = 4 * n3;
    const int64_t w = inner64 ? 8 : 4;
    int64_t b = (int64_t)S * (8 * N4 + 8 * n3 + 4 * w * N4 + 3 * w * n3 + 4 * n3);
    b += (int64_t)(inner64 ? mg_scratch_elems<double>(g, S) * 8 : mg_scratch_elems<float>(g, S) * 4);
    b += 4LL * S * kMaxPartials * 8 + 2LL * S * 8 + (int64_t)S * sizeof(MinresCol);
    return b;
}

struct Mesh {
    int64_t nverts = 0, ntets = 0, nnz = 0, ncols_used = 0;
    double* xyz = nullptr;
    int32_t* tets = nullptr;
    double* vol = nullptr;
    int64_t* rowptr = nullptr;
    int32_t* col = nullptr;
    double* g = nullptr;
    float* pi = nullptr;
    void release() {
        dev_free(xyz);
        dev_free(tets);
        dev_free(vol);
        dev_free(rowptr);
        dev_free(col);
        dev_free(g);
        dev_free(pi);
        nverts = ntets = nnz = 0;
    }
};

// Cell-wise kappa(x), sigma(x) of a level (spde_level_set_fields), as the
// coefficients the kernels use.
struct Fields {
    bool set = false;
    double* kh2_64 = nullptr;  // (kappa_c h)^2
    float* kh2_32 = nullptr;
    double* gh = nullptr;      // -g_c h, the per-cell factor of the scaled right-hand side
    double kh2_mean = 0.0;     // mean (kappa_c h)^2 (the refinement's scalar fallback)
    // per-cell multigrid diagonals of every level: D = 2^l (a 4^l + c k), a the children's
    // mean of (kappa h)^2, so the V-cycle follows kappa(x) on every level
    double* D64[16] = {};
    float* D32[16] = {};
    void release() {
        dev_free(kh2_64);
        dev_free(kh2_32);
        dev_free(gh);
        for (int l = 0; l < 16; ++l) {
            dev_free(D64[l]);
            dev_free(D32[l]);
        }
        set = false;
        kh2_mean = 0.0;
    }
};

struct Level {
    bool defined = false;
    Grid3 g;
    double h = 0.0;
    double lo[3] = {0, 0, 0};
    Mesh mesh;
    Workspace ws;
    Fields fields;
    bool tuned = false;  // spde_autotune / spde_level_set_tuning picked this level's schedule
    spde_tuning tune{};
};

// the options a level's solves run with: the context's, with the level's tuning
spde_opts level_opts(const spde_opts& base, const Level& L) {
    spde_opts o = base;
    if (L.tuned) {
        o.omega = L.tune.omega;
        o.inner_tol = L.tune.inner_tol;
        o.flux_diag = L.tune.flux_diag;
        o.sweep_planes = L.tune.sweep_planes;
    }
    return o;
}

}  // namespace

namespace {
struct Server;
}

struct spde_ctx {
    spde_opts opts;
    Profiler prof;
    std::mutex mu;
    Level lev[16];
    spde_stats stats;
    void* out_tmp = nullptr;
    size_t out_tmp_bytes = 0;
    Server* srv = nullptr;  // serving engine, started by the first spde_submit
    // graph-driven (asynchronous) calls: capture streams, the device record of their
    // solves' outcome (read by spde_wait / spde_get_stats), and whether it holds
    // results the host has not read yet
    cudaStream_t cap[3] = {nullptr, nullptr, nullptr};
    CallAcc* d_acc = nullptr;
    CallAcc* h_acc = nullptr;  // pinned
    bool acc_pending = false;
    int deferred = SPDE_OK;    // worst outcome of graph-driven calls not yet returned by spde_wait
};

namespace {

spde_status ensure_workspace(Workspace& ws, const Grid3& g, int S, bool inner64) {
    if (ws.g == g && ws.S >= S && ws.inner64 == (int)inner64) return SPDE_OK;
    ws.release();
    const size_t n3 = (size_t)g.cells(), N4 = 4 * n3;
    const size_t w = inner64 ? 8 : 4;
    STATUS_TRY(dev_alloc(&ws.x64, (size_t)S * N4));
    STATUS_TRY(dev_alloc(&ws.F, (size_t)S * n3));
    for (int iv = 0; iv < 7; ++iv) {
        void*& v = ws.vec[iv];
        cudaError_t e = cudaMalloc(&v, (size_t)S * (iv < 3 ? n3 : N4) * w);
        if (e != cudaSuccess) {
            v = nullptr;
            cudaGetLastError();
            ws.release();
            return fail(SPDE_ENOMEM, "workspace allocation failed (%d columns of %d x %d x %d)", S, g.nx, g.ny, g.nz);
        }
    }
    const size_t mgb = inner64 ? mg_scratch_elems<double>(g, S) * 8 : mg_scratch_elems<float>(g, S) * 4;
    if (mgb) {
        cudaError_t e = cudaMalloc(&ws.mg, mgb);
        if (e != cudaSuccess) {
            ws.mg = nullptr;
            cudaGetLastError();
            ws.release();
            return fail(SPDE_ENOMEM, "multigrid scratch allocation failed");
        }
    }
    STATUS_TRY(dev_alloc(&ws.partA, (size_t)S * kMaxPartials));
    STATUS_TRY(dev_alloc(&ws.partB, (size_t)S * kMaxPartials));
    STATUS_TRY(dev_alloc(&ws.partC, (size_t)S * kMaxPartials));
    STATUS_TRY(dev_alloc(&ws.partR, (size_t)S * kMaxPartials));
    STATUS_TRY(dev_alloc(&ws.colv, (size_t)2 * S));
    STATUS_TRY(dev_alloc(&ws.coltol, (size_t)S));
    STATUS_TRY(dev_alloc(&ws.st, (size_t)S));
    STATUS_TRY(dev_alloc(&ws.cg, (size_t)S));
    // per MINRES iteration of a chunk: [2q] columns still active after it, [2q+1] columns it left an update pending
    STATUS_TRY(dev_alloc(&ws.nact, 2 * kMaxChunk));
    STATUS_TRY(dev_alloc(&ws.fault, 1));
    STATUS_TRY(dev_alloc(&ws.ctl, 1));
    STATUS_TRY(dev_alloc(&ws.mask, (size_t)S));
    if (cudaEventCreateWithFlags(&ws.done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        ws.done = nullptr;
        ws.release();
        return fail(SPDE_ECUDA, "event creation failed");
    }
    if (cudaMemset(ws.fault, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        ws.release();
        return fail(SPDE_ECUDA, "clearing the fault word failed");
    }
    STATUS_TRY(dev_alloc(&ws.thetaT, (size_t)S * n3));
    {
        // Thomas factors of tridiag(1/6, 2/3, 1/6) on the n-1 interior faces of a line of the
        // longest extent n (the factors of a shorter line are the first ones of the same table)
        const int n = g.maxn();
        std::vector<double> tri(2 * (size_t)n - 2);
        double cprev = 0.0;
        for (int f = 0; f < n - 1; ++f) {
            const double piv = 2.0 / 3.0 - (f ? cprev / 6.0 : 0.0);
            tri[f] = (1.0 / 6.0) / piv;
            tri[(n - 1) + f] = 1.0 / piv;
            cprev = tri[f];
        }
        STATUS_TRY(dev_alloc(&ws.tri, tri.size()));
        STATUS_TRY(dev_alloc(&ws.tri32, tri.size()));
        std::vector<float> tri32(tri.begin(), tri.end());
        if (cudaMemcpy(ws.tri32, tri32.data(), tri32.size() * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(ws.tri, tri.data(), tri.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            ws.release();
            return fail(SPDE_ECUDA, "upload of line-solve factors failed");
        }
    }
    if (cudaMallocHost(&ws.h_nact, 2 * kMaxChunk * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&ws.h_col, 2 * S * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&ws.h_st, S * sizeof(MinresCol)) != cudaSuccess ||
        cudaMallocHost(&ws.h_tol, S * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        ws.release();
        return fail(SPDE_ENOMEM, "pinned host allocation failed");
    }
    ws.g = g;
    ws.S = S;
    ws.inner64 = inner64 ? 1 : 0;
    return SPDE_OK;
}

// Batched MINRES on the scaled mixed system for the columns flagged in
// st[].active; right-hand sides in r2 (inner type T), solution in d.
// One kappa per column (serving lanes): (kappa h)^2 per column in FP64 and in the
// inner type, and the per-column sweep coefficients of every tiled level.
struct ColKappa {
    const double* kh2_64 = nullptr;
    const void* kh2_t = nullptr;
    const void* qtab[16] = {};
};

template <typename T>
spde_status minres_batch(const spde_opts& o, const Grid3& g, double kh2, int S, Workspace& ws, double inner_tol,
                         int* iters_out, cudaStream_t st, const T* kh2c = nullptr, T* const* Dlev = nullptr,
                         const double* col_tol = nullptr, const ColKappa* ck = nullptr) {
    const T* kh2s = ck ? static_cast<const T*>(ck->kh2_t) : nullptr;
    const int64_t n3 = g.cells(), N4 = 4 * n3;
    T* d = static_cast<T*>(ws.vec[0]);
    T* w1 = static_cast<T*>(ws.vec[1]);
    T* w2 = static_cast<T*>(ws.vec[2]);
    T* r1 = static_cast<T*>(ws.vec[3]);
    T* r2 = static_cast<T*>(ws.vec[4]);
    T* ycur = static_cast<T*>(ws.vec[5]);
    T* ynext = static_cast<T*>(ws.vec[6]);
    MGPlan plan;
    if (!mg_plan_init(plan, g, kh2, o.schur_c, o.omega)) return fail(SPDE_EINVAL, "grid shape not supported by the V-cycle");
    mg_plan_bind<T>(plan, S, static_cast<T*>(ws.mg));
    plan.fault = ws.fault;
    plan.sz_pref = o.sweep_planes;
    plan.coarse_fp16 = o.coarse_fp16 != 0;
    plan.sweep_rows = o.sweep_rows != 0;
    if (Dlev)
        for (int l = 0; l < plan.nlev && l < 16; ++l) plan.D[l] = Dlev[l];
    if (ck) {
        plan.kh2col = ck->kh2_64;
        for (int l = 0; l < 16; ++l) plan.qtab[l] = ck->qtab[l];
    }
    const int act_stride = (int)(sizeof(MinresCol) / sizeof(int));
    const int* act = &ws.st[0].active;
    const double w = (double)sizeof(T);
    const double n3d = (double)n3;
    // y = P^{-1} r2, beta1
    plan.prof_cols = (double)S;
    prof_begin(PK_OTHER, st);
    const int nB0 = launch_precond_u<T>(N4, (int)n3, S, r2, ycur, o.flux_diag, ws.partB, ws.st, st);
    prof_end(st, (double)S * 6.0 * n3d * w);
    const int nC0 = launch_vcycle<T>(plan, S, r2 + 3 * n3, N4, ycur + 3 * n3, N4, ws.partC, act, act_stride, st);
    if (nC0 < 0) return fail(SPDE_ECUDA, "V-cycle launch configuration failed");
    CUDA_TRY(cudaMemsetAsync(ws.nact, 0, sizeof(int), st));
    prof_begin(PK_OTHER, st);
    CUDA_TRY(launch_minres_init(S, ws.partB, nB0, ws.partC, nC0, inner_tol, ws.st, ws.nact, st, col_tol));
    prof_end(st, (double)S * (nB0 + nC0) * 8.0);
    CUDA_TRY(cudaMemcpyAsync(ws.h_nact, ws.nact, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    int it = 0;
    int nactive = *ws.h_nact;
    bool pending = false;  // a w/x update of the last iteration waits for the next pass
    int last_itn = 0;
    int last_upd = 0;  // columns whose last update waits for the next pass
    T* yprev = nullptr;
    while (nactive > 0 && it < o.max_iter) {
        const int chunk = std::min(std::min(o.check_every, o.max_iter - it), kMaxChunk);
        // the profiler's byte counts are recorded per column and scaled after the chunk's
        // synchronisation by the columns each iteration really processed
        CUDA_TRY(cudaMemsetAsync(ws.nact, 0, 2 * chunk * sizeof(int), st));
        plan.prof_cols = 1.0;
        size_t rec[kMaxChunk + 1];
        double a_bytes[kMaxChunk], d_bytes[kMaxChunk];
        for (int q = 0; q < chunk; ++q) {
            const int itn = it + q + 1;  // 1-based iteration of the columns that started together
            rec[q] = t_prof ? t_prof->mark() : 0;
            // A(itn) fused with the pending w/x update D(itn - 1) (cell block only)
            prof_begin(PK_MINRES_A, st);
            const int nA = launch_minres_A<T>(g, kh2, S, ycur, r2, o.flux_diag, ws.partA, ws.st,
                                              pending ? yprev : nullptr, w1, w2, d, st, kh2c, kh2s);
            a_bytes[q] = (4.0 + (kh2c ? 1.0 : 0.0)) * n3d * w;
            d_bytes[q] = pending ? (itn - 1 >= 3 ? 6.0 : (itn - 1 == 2 ? 5.0 : 3.0)) * n3d * w : 0.0;
            prof_end(st, 0.0);
            if (pending) std::swap(w1, w2);
            prof_begin(PK_ALPHA, st);
            CUDA_TRY(launch_alpha(S, ws.partA, nA, ws.st, st));
            prof_end(st, nA * 8.0);
            // pass B: partA (consumed by the alpha step) now takes its partial sums of r1.y
            prof_begin(PK_MINRES_B, st);
            const int nB = launch_minres_B<T>(g, kh2, S, ycur, r2, o.flux_diag, r1, ws.partB, ws.partA, ws.st, st,
                                              kh2c, kh2s);
            prof_end(st, ((itn >= 2 ? 13.0 : 9.0) + (kh2c ? 1.0 : 0.0)) * n3d * w);
            const int nC = launch_vcycle<T>(plan, S, r1 + 3 * n3, N4, ynext + 3 * n3, N4, ws.partC, act, act_stride, st);
            prof_begin(PK_GIVENS, st);
            CUDA_TRY(launch_givens(S, ws.partB, nB, ws.partC, nC, ws.partA, ws.st, ws.nact + 2 * q, st, o.max_iter));
            prof_end(st, (2 * nB + nC) * 8.0);
            pending = true;
            last_itn = itn;
            yprev = ycur;
            std::swap(r1, r2);
            std::swap(ycur, ynext);
        }
        rec[chunk] = t_prof ? t_prof->mark() : 0;
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaMemcpyAsync(ws.h_nact, ws.nact, 2 * chunk * sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        if (t_prof) {
            for (int q = 0; q < chunk; ++q) {
                const double on = q == 0 ? (double)nactive : (double)ws.h_nact[2 * (q - 1)];
                const double upd = q == 0 ? (double)last_upd : (double)ws.h_nact[2 * (q - 1) + 1];
                t_prof->scale(rec[q], rec[q + 1], on);
                t_prof->set_bytes(rec[q], a_bytes[q] * on + d_bytes[q] * upd);
            }
            t_prof->flush();
        }
        it += chunk;
        nactive = ws.h_nact[2 * (chunk - 1)];
        last_upd = ws.h_nact[2 * (chunk - 1) + 1];
    }
    if (pending) {
        prof_begin(PK_MINRES_D, st);
        CUDA_TRY(launch_minres_D<T>(n3, S, yprev, w1, w2, d, ws.st, st));
        prof_end(st, (double)last_upd * (last_itn >= 3 ? 6.0 : (last_itn == 2 ? 5.0 : 3.0)) * n3d * w);
        std::swap(w1, w2);
    }
    *iters_out = it;
    return SPDE_OK;
}

// Schur-complement CG for the columns flagged in cg[].active: S d = -r_theta,
// r_theta the cell block of the mixed residual in ws.vec[4] (inner type T);
// d in ws.vec[0] ([S][n^3]).
template <typename T>
spde_status cg_batch(const spde_opts& o, const Grid3& g, double kh2, int S, Workspace& ws, double inner_tol,
                     int* iters_out, cudaStream_t st) {
    if (!g.cube()) return fail(SPDE_EINVAL, "the Schur-complement CG solver needs a cubic grid");
    const int n = g.nx;
    const int64_t n3 = g.cells();
    T* x = static_cast<T*>(ws.vec[0]);
    T* r = static_cast<T*>(ws.vec[1]);
    T* p = static_cast<T*>(ws.vec[2]);
    T* q = static_cast<T*>(ws.vec[3]);  // [S][n^3] view of a larger buffer
    T* z = static_cast<T*>(ws.vec[5]);
    const T* mixed_r = static_cast<const T*>(ws.vec[4]);
    const T* tri = std::is_same<T, float>::value ? reinterpret_cast<const T*>(ws.tri32) : reinterpret_cast<const T*>(ws.tri);
    MGPlan plan;
    mg_plan_init(plan, g, kh2, o.schur_c, o.omega);
    mg_plan_bind<T>(plan, S, static_cast<T*>(ws.mg));
    plan.fault = ws.fault;
    plan.sz_pref = o.sweep_planes;
    plan.coarse_fp16 = o.coarse_fp16 != 0;
    plan.sweep_rows = o.sweep_rows != 0;
    plan.prof_cols = (double)S;
    const int act_stride = (int)(sizeof(CgCol) / sizeof(int));
    const int* act = &ws.cg[0].active;
    const double w = (double)sizeof(T), n3d = (double)n3;
    prof_begin(PK_OTHER, st);
    const int nrr0 = launch_cg_rhs<T>(n3, S, mixed_r, r, ws.partB, ws.cg, st);
    prof_end(st, (double)S * 2.0 * n3d * w);
    const int nrz0 = launch_vcycle<T>(plan, S, r, n3, z, n3, ws.partC, act, act_stride, st);
    if (nrz0 < 0) return fail(SPDE_ECUDA, "V-cycle launch configuration failed");
    CUDA_TRY(cudaMemsetAsync(ws.nact, 0, sizeof(int), st));
    CUDA_TRY(launch_cg_init(S, ws.partC, nrz0, ws.partB, nrr0, inner_tol, ws.cg, ws.nact, st));
    CUDA_TRY(launch_cg_p<T>(n3, S, p, z, ws.cg, st));
    CUDA_TRY(cudaMemcpyAsync(ws.h_nact, ws.nact, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    int it = 0;
    int nactive = *ws.h_nact;
    while (nactive > 0 && it < o.max_iter) {
        const int chunk = std::min(o.check_every, o.max_iter - it);
        const double cols = (double)nactive;
        plan.prof_cols = cols;
        for (int k = 0; k < chunk; ++k) {
            prof_begin(PK_SCHUR_APPLY, st);
            const int nq = launch_schur_apply<T>(n, kh2, S, p, q, tri, static_cast<T*>(ws.vec[6]), ws.partA, ws.cg, st);
            prof_end(st, cols * 8.0 * n3d * w);  // axis passes: read p, write q; read p, q, write q (x2)
            if (nq < 0) return fail(SPDE_ECUDA, "Schur operator launch configuration failed");
            prof_begin(PK_ALPHA, st);
            CUDA_TRY(launch_cg_alpha(S, ws.partA, nq, ws.cg, st));
            prof_end(st, cols * nq * 8.0);
            prof_begin(PK_CG_UPDATE, st);
            const int nrr = launch_cg_xr<T>(n3, S, x, r, p, q, ws.partB, ws.cg, st);
            prof_end(st, cols * 6.0 * n3d * w);
            const int nrz = launch_vcycle<T>(plan, S, r, n3, z, n3, ws.partC, act, act_stride, st);
            if (k == chunk - 1) CUDA_TRY(cudaMemsetAsync(ws.nact, 0, sizeof(int), st));
            prof_begin(PK_GIVENS, st);
            CUDA_TRY(launch_cg_beta(S, ws.partB, nrr, ws.partC, nrz, ws.cg, (k == chunk - 1) ? ws.nact : nullptr, st,
                                    o.max_iter));
            prof_end(st, cols * (nrr + nrz) * 8.0);
            prof_begin(PK_CG_UPDATE, st);
            CUDA_TRY(launch_cg_p<T>(n3, S, p, z, ws.cg, st));
            prof_end(st, cols * 3.0 * n3d * w);
        }
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaMemcpyAsync(ws.h_nact, ws.nact, sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        if (t_prof) t_prof->flush();
        it += chunk;
        nactive = *ws.h_nact;
    }
    *iters_out = it;
    return SPDE_OK;
}

// a V-cycle sweep that gave up waiting for a plane copy leaves the columns of
// that solve invalid: report it (and reset the workspace's fault word for later calls)
static spde_status fault_status(int fault, int* dev_fault, cudaStream_t st) {
    if (!fault) return SPDE_OK;
    CUDA_TRY(mg_fault_clear(dev_fault, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return fail(SPDE_ETIMEOUT, "a multigrid sweep gave up waiting for a plane copy; this solve's results are invalid");
}

// Solve (D A D) x = [0; F] for S columns: FP64 iterative refinement around an
// inner MINRES of element type T.  F, x64 in ws; returns the max relative
// residual in *maxrel.
template <typename T>
spde_status refine_solve(spde_ctx* ctx, const Grid3& g, double kh2, int S, Workspace& ws, double* maxrel,
                         int* outer_out, int* inner_out, cudaStream_t st, bool warm = false,
                         const Fields* fl = nullptr) {
    const spde_opts& o = ws.o;
    const int64_t n3 = g.cells(), N4 = 4 * n3;
    // ||F||^2 per column
    prof_begin(PK_SUMSQ, st);
    int nb = launch_sumsq(n3, S, ws.F, n3, ws.partR, st);
    prof_end(st, (double)S * 8.0 * (double)n3);
    prof_begin(PK_OTHER, st);
    CUDA_TRY(launch_reduce(S, ws.partR, nb, ws.colv + S, st));
    prof_end(st, (double)S * nb * 8.0);
    // cold start: x = 0; warm start: the caller filled the cell block of x (flux recomputed below)
    if (!warm) CUDA_TRY(cudaMemsetAsync(ws.x64, 0, (size_t)S * N4 * sizeof(double), st));
    std::vector<int> mask(S, 1);
    int* d_mask = reinterpret_cast<int*>(ws.colv);  // reuse first S doubles' storage after use
    int outer = 0, inner_total = 0;
    double worst = 0.0;
    T* r2 = static_cast<T*>(ws.vec[4]);
    for (;;) {
        // r = [0; F] - A x (FP64) -> r2 (inner type); ||r||^2
        float* r32 = std::is_same<T, float>::value ? reinterpret_cast<float*>(r2) : nullptr;
        double* r64 = std::is_same<T, double>::value ? reinterpret_cast<double*>(r2) : nullptr;
        if (outer > 0 || warm) {
            // flux rows exact for the current cell field: u = -T^{-1} D1^T theta
            prof_begin(PK_FLUX, st);
            CUDA_TRY(launch_flux_from_theta(g, S, ws.x64, N4, ws.tri, st));
            prof_end(st, (double)S * 96.0 * (double)n3);
        }
        // x = 0 in the first step of a cold start: the residual is F, read without x
        const int xzero = (outer == 0 && !warm) ? 1 : 0;
        prof_begin(PK_RESIDUAL, st);
        nb = launch_residual64(g, kh2, S, ws.F, n3, ws.x64, r32, r64, ws.partR, nullptr, st, fl ? fl->kh2_64 : nullptr,
                               nullptr, xzero);
        prof_end(st, (double)S * (xzero ? 8.0 + 4.0 * sizeof(T) : 40.0 + 4.0 * sizeof(T) + (fl ? 8.0 : 0.0)) *
                         (double)n3);
        CUDA_TRY(cudaGetLastError());
        prof_begin(PK_OTHER, st);
        CUDA_TRY(launch_reduce(S, ws.partR, nb, ws.colv, st));
        prof_end(st, (double)S * nb * 8.0);
        CUDA_TRY(cudaMemcpyAsync(ws.h_col, ws.colv, 2 * S * sizeof(double), cudaMemcpyDeviceToHost, st));
        int fault = 0;
        CUDA_TRY(mg_fault_read(ws.fault, &fault, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        STATUS_TRY(fault_status(fault, ws.fault, st));
        int nact = 0;
        worst = 0.0;
        for (int s = 0; s < S; ++s) {
            const double fn = ws.h_col[S + s];
            const double rel = fn > 0.0 ? std::sqrt(ws.h_col[s] / fn) : 0.0;
            worst = std::max(worst, rel);
            mask[s] = (rel > o.tol) ? 1 : 0;
            nact += mask[s];
            ws.h_tol[s] = inner_tol_for(o, rel);
        }
        if (nact == 0 || outer >= o.max_outer) break;
        CUDA_TRY(cudaMemcpyAsync(d_mask, mask.data(), S * sizeof(int), cudaMemcpyHostToDevice, st));
        prof_begin(PK_OTHER, st);
        if (o.solver == SPDE_SOLVER_SCHUR_CG) CUDA_TRY(launch_cg_set_active(S, d_mask, ws.cg, st));
        else CUDA_TRY(launch_set_active(S, d_mask, ws.st, st));
        prof_end(st, (double)S * 4.0);
        // the inner solve only needs to reduce this step's residual by inner_tol (FP32) or
        // to reach the overall tolerance (FP64 inner)
        double itol = o.inner_tol;
        if (std::is_same<T, double>::value) itol = std::max(0.1 * o.tol / std::max(worst, 1e-300), 1e-15);
        int its = 0;
        if (o.solver == SPDE_SOLVER_SCHUR_CG) STATUS_TRY(cg_batch<T>(o, g, kh2, S, ws, itol, &its, st));
        else {
            const T* kh2c = nullptr;
            T* const* Dlev = nullptr;
            if (fl) {
                if constexpr (sizeof(T) == 4) {
                    kh2c = fl->kh2_32;
                    Dlev = fl->D32;
                } else {
                    kh2c = fl->kh2_64;
                    Dlev = fl->D64;
                }
            }
            const double* col_tol = nullptr;
            if (std::is_same<T, float>::value) {  // FP32 inner: each column's own reduction
                CUDA_TRY(cudaMemcpyAsync(ws.coltol, ws.h_tol, S * sizeof(double), cudaMemcpyHostToDevice, st));
                col_tol = ws.coltol;
            }
            STATUS_TRY(minres_batch<T>(o, g, kh2, S, ws, itol, &its, st, kh2c, Dlev, col_tol));
        }
        inner_total += its;
        prof_begin(PK_ADD_CORR, st);
        if (o.solver == SPDE_SOLVER_SCHUR_CG)
            CUDA_TRY(launch_cg_add<T>(n3, S, ws.x64, static_cast<const T*>(ws.vec[0]), ws.cg, st));
        else
            CUDA_TRY(launch_add_theta<T>(n3, S, ws.x64, static_cast<const T*>(ws.vec[0]), ws.st, st));
        prof_end(st, (double)nact * (16.0 + sizeof(T)) * (double)n3);
        ++outer;
    }
    *maxrel = worst;
    *outer_out = outer;
    *inner_out = inner_total;
    if (worst > o.tol) return fail(SPDE_ENOCONV, "refinement stopped at relative residual %.3e > tol %.3e", worst, o.tol);
    return SPDE_OK;
}

// ---------------------------------------------------------------------------
// Graph-driven refinement (the asynchronous path).
//
// One solve of S columns is captured once per (workspace, S, precision, warm
// start, fields, kappa) into a CUDA graph of the shape
//     ||F||^2;  x = 0;  init
//     while (go) {                         outer: refinement steps
//         flux from theta; FP64 residual; check -> go, columns, inner tolerances
//         y = P^{-1} r; MINRES start; iteration 1
//         while (more) { iteration; iteration; count -> more }   inner
//         final w/x update; theta += d
//     }
//     record the outcome
// whose conditions are set on the device by the control kernels (krylov.cu).
// It launches exactly the kernels of the synchronous path in the same order
// with the same arguments; the only difference is that iterations after every
// column has retired (at most one per loop body, where the host checks every
// check_every iterations) run as no-ops on retired columns.  Two iterations
// per loop body keep the ping-pong buffers in the same places at every test of
// the condition, so the captured pointers stay valid.
// ---------------------------------------------------------------------------
struct CaptureGuard {  // ends captures still open when a capture step fails
    cudaStream_t st[3] = {nullptr, nullptr, nullptr};
    ~CaptureGuard() {
        for (int i = 2; i >= 0; --i)
            if (st[i]) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(st[i], &g);
                if (g && i == 0) cudaGraphDestroy(g);
            }
        cudaGetLastError();
    }
};

// adds a while node at the capture point of `st` (which then depends on it) and
// returns its body graph
spde_status add_while(cudaStream_t st, cudaGraphConditionalHandle h, cudaGraph_t* body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    CUDA_TRY(cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd));
    if (cs != cudaStreamCaptureStatusActive) return fail(SPDE_ECUDA, "stream capture is not active");
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    CUDA_TRY(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
    *body = p.conditional.phGraph_out[0];
    CUDA_TRY(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return SPDE_OK;
}

spde_status ensure_capture_streams(spde_ctx* ctx) {
    for (auto& c : ctx->cap)
        if (!c) CUDA_TRY(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
    if (!ctx->d_acc) {
        STATUS_TRY(dev_alloc(&ctx->d_acc, 1));
        if (cudaMallocHost(&ctx->h_acc, sizeof(CallAcc)) != cudaSuccess) {
            cudaGetLastError();
            ctx->h_acc = nullptr;
            return fail(SPDE_ENOMEM, "pinned host allocation failed");
        }
    }
    return SPDE_OK;
}

template <typename T>
spde_status capture_refine(spde_ctx* ctx, const Grid3& g, double kh2, int S, Workspace& ws, bool warm,
                           const Fields* fl, bool count, cudaGraph_t* out) {
    const spde_opts& o = ws.o;
    const int64_t n3 = g.cells(), N4 = 4 * n3;
    const bool t64 = std::is_same<T, double>::value;
    cudaStream_t c0 = ctx->cap[0], c1 = ctx->cap[1], c2 = ctx->cap[2];
    const T* kh2c = nullptr;
    T* const* Dlev = nullptr;
    if (fl) {
        if constexpr (sizeof(T) == 4) {
            kh2c = fl->kh2_32;
            Dlev = fl->D32;
        } else {
            kh2c = fl->kh2_64;
            Dlev = fl->D64;
        }
    }
    MGPlan plan;
    if (!mg_plan_init(plan, g, kh2, o.schur_c, o.omega)) return fail(SPDE_EINVAL, "grid shape not supported by the V-cycle");
    mg_plan_bind<T>(plan, S, static_cast<T*>(ws.mg));
    plan.fault = ws.fault;
    plan.sz_pref = o.sweep_planes;
    plan.coarse_fp16 = o.coarse_fp16 != 0;
    plan.sweep_rows = o.sweep_rows != 0;
    if (Dlev)
        for (int l = 0; l < plan.nlev && l < 16; ++l) plan.D[l] = Dlev[l];
    const int act_stride = (int)(sizeof(MinresCol) / sizeof(int));
    const int* act = &ws.st[0].active;
    T* d = static_cast<T*>(ws.vec[0]);
    T* w1 = static_cast<T*>(ws.vec[1]);
    T* w2 = static_cast<T*>(ws.vec[2]);
    T* r1 = static_cast<T*>(ws.vec[3]);
    T* r2 = static_cast<T*>(ws.vec[4]);
    T* ycur = static_cast<T*>(ws.vec[5]);
    T* ynext = static_cast<T*>(ws.vec[6]);
    RefineCtl* ctl = ws.ctl;

    cudaGraph_t graph = nullptr;
    CUDA_TRY(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle h_outer, h_inner;
    if (cudaGraphConditionalHandleCreate(&h_outer, graph, 0, 0) != cudaSuccess) {
        cudaGraphDestroy(graph);
        CUDA_TRY(cudaGetLastError());
        return fail(SPDE_ECUDA, "conditional handle creation failed");
    }
    CaptureGuard guard;
    CUDA_TRY(cudaStreamBeginCaptureToGraph(c0, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    guard.st[0] = c0;
    // ||F||^2 per column, x = 0 (cold start), control block
    int nb = launch_sumsq(n3, S, ws.F, n3, ws.partR, c0);
    CUDA_TRY(launch_reduce(S, ws.partR, nb, ws.colv + S, c0));
    if (!warm) CUDA_TRY(cudaMemsetAsync(ws.x64, 0, (size_t)S * N4 * sizeof(double), c0));
    CUDA_TRY(launch_refine_init(ctl, ws.fault, h_outer, c0));
    cudaGraph_t outer_body = nullptr;
    STATUS_TRY(add_while(c0, h_outer, &outer_body));
    CUDA_TRY(cudaGraphConditionalHandleCreate(&h_inner, outer_body, 0, 0));
    CUDA_TRY(cudaStreamBeginCaptureToGraph(c1, outer_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    guard.st[1] = c1;
    {
        // one refinement step: residual, decisions, inner MINRES, correction
        CUDA_TRY(launch_flux_from_theta(g, S, ws.x64, N4, ws.tri, c1, warm ? nullptr : &ctl->outer));
        float* r32 = t64 ? nullptr : reinterpret_cast<float*>(r2);
        double* r64 = t64 ? reinterpret_cast<double*>(r2) : nullptr;
        nb = launch_residual64(g, kh2, S, ws.F, n3, ws.x64, r32, r64, ws.partR, nullptr, c1, fl ? fl->kh2_64 : nullptr,
                               nullptr, 0, warm ? nullptr : &ctl->outer);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(launch_reduce(S, ws.partR, nb, ws.colv, c1));
        CUDA_TRY(launch_refine_check(S, ws.colv, o.tol, o.inner_tol, t64 ? 1 : 0, o.max_outer, ws.fault, ws.mask,
                                     ws.coltol, ctl, h_outer, c1));
        CUDA_TRY(launch_set_active(S, ws.mask, ws.st, c1));
        const int nB0 = launch_precond_u<T>(N4, (int)n3, S, r2, ycur, o.flux_diag, ws.partB, ws.st, c1);
        const int nC0 = launch_vcycle<T>(plan, S, r2 + 3 * n3, N4, ycur + 3 * n3, N4, ws.partC, act, act_stride, c1);
        if (nC0 < 0) return fail(SPDE_ECUDA, "V-cycle launch configuration failed");
        CUDA_TRY(launch_minres_init(S, ws.partB, nB0, ws.partC, nC0, o.inner_tol, ws.st, ctl->cnt + 4, c1, ws.coltol));
        bool pending = false;
        T* yprev = nullptr;
        auto iteration = [&](cudaStream_t s, int slot) -> spde_status {
            const int nA = launch_minres_A<T>(g, kh2, S, ycur, r2, o.flux_diag, ws.partA, ws.st,
                                              pending ? yprev : nullptr, w1, w2, d, s, kh2c);
            if (pending) std::swap(w1, w2);
            CUDA_TRY(launch_alpha(S, ws.partA, nA, ws.st, s));
            // partA, consumed by the alpha step, takes pass B's partial sums of r1.y
            const int nB = launch_minres_B<T>(g, kh2, S, ycur, r2, o.flux_diag, r1, ws.partB, ws.partA, ws.st, s, kh2c);
            const int nC = launch_vcycle<T>(plan, S, r1 + 3 * n3, N4, ynext + 3 * n3, N4, ws.partC, act, act_stride, s);
            if (nC < 0) return fail(SPDE_ECUDA, "V-cycle launch configuration failed");
            CUDA_TRY(launch_givens(S, ws.partB, nB, ws.partC, nC, ws.partA, ws.st, ctl->cnt + 2 * slot, s, o.max_iter));
            pending = true;
            yprev = ycur;
            std::swap(r1, r2);
            std::swap(ycur, ynext);
            return SPDE_OK;
        };
        STATUS_TRY(iteration(c1, 0));
        CUDA_TRY(launch_loop_ctl(ctl, 0, 1, o.max_iter, h_inner, c1));
        cudaGraph_t inner_body = nullptr;
        STATUS_TRY(add_while(c1, h_inner, &inner_body));
        CUDA_TRY(cudaStreamBeginCaptureToGraph(c2, inner_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        guard.st[2] = c2;
        STATUS_TRY(iteration(c2, 0));
        STATUS_TRY(iteration(c2, 1));
        CUDA_TRY(launch_loop_ctl(ctl, 1, 2, o.max_iter, h_inner, c2));
        guard.st[2] = nullptr;
        cudaGraph_t tmp = nullptr;
        CUDA_TRY(cudaStreamEndCapture(c2, &tmp));
        // the pending update of the last iteration, then the correction of theta
        CUDA_TRY(launch_minres_D<T>(n3, S, yprev, w1, w2, d, ws.st, c1));
        CUDA_TRY(launch_add_theta<T>(n3, S, ws.x64, d, ws.st, c1));
    }
    guard.st[1] = nullptr;
    {
        cudaGraph_t tmp = nullptr;
        CUDA_TRY(cudaStreamEndCapture(c1, &tmp));
    }
    CUDA_TRY(launch_refine_finish(ctl, ctx->d_acc, count ? 1 : 0, c0));
    guard.st[0] = nullptr;
    CUDA_TRY(cudaStreamEndCapture(c0, &graph));
    *out = graph;
    return SPDE_OK;
}

// the executable graph of this solve shape, captured on first use
template <typename T>
spde_status refine_graph(spde_ctx* ctx, const Grid3& g, double kh2, int S, Workspace& ws, bool warm, const Fields* fl,
                         bool count, cudaGraphExec_t* exec) {
    const int t64 = std::is_same<T, double>::value ? 1 : 0;
    for (auto& gr : ws.graphs)
        if (gr.S == S && gr.t64 == t64 && gr.warm == (int)warm && gr.count == (int)count &&
            gr.fields == (const void*)fl && gr.kh2 == kh2) {
            *exec = gr.exec;
            return SPDE_OK;
        }
    STATUS_TRY(ensure_capture_streams(ctx));
    CUDA_TRY(mg_prepare());  // one-time attributes are set outside the capture
    CUDA_TRY(flux_prepare());
    Profiler* saved = t_prof;  // nothing is timed inside a capture
    t_prof = nullptr;
    cudaGraph_t graph = nullptr;
    const spde_status s = capture_refine<T>(ctx, g, kh2, S, ws, warm, fl, count, &graph);
    t_prof = saved;
    STATUS_TRY(s);
    cudaGraphExec_t ex = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&ex, graph, 0);
    cudaGraphDestroy(graph);
    CUDA_TRY(e);
    if (ws.graphs.size() >= 8) {  // a few shapes per workspace (kappa changes re-capture)
        cudaGraphExecDestroy(ws.graphs.front().exec);
        ws.graphs.erase(ws.graphs.begin());
    }
    ws.graphs.push_back(Workspace::Graph{S, t64, (int)warm, (int)count, (const void*)fl, kh2, ex});
    *exec = ex;
    return SPDE_OK;
}

// enqueue the graph-driven solve of S columns (F, x64 in ws) on st; the outcome
// goes to the context's device record
template <typename T>
spde_status refine_solve_async(spde_ctx* ctx, const Grid3& g, double kh2, int S, Workspace& ws, cudaStream_t st,
                               bool warm = false, const Fields* fl = nullptr, bool count = true) {
    cudaGraphExec_t ex = nullptr;
    STATUS_TRY(refine_graph<T>(ctx, g, kh2, S, ws, warm, fl, count, &ex));
    CUDA_TRY(cudaGraphLaunch(ex, st));
    return SPDE_OK;
}

// start of a graph-driven call on st: its outcome record is fresh unless earlier
// calls' outcomes are still unread; `ws` waits for the last call that used it
spde_status async_call_begin(spde_ctx* ctx, cudaStream_t st) {
    STATUS_TRY(ensure_capture_streams(ctx));
    if (!ctx->acc_pending) {
        CUDA_TRY(cudaMemsetAsync(ctx->d_acc, 0, sizeof(CallAcc), st));
        ctx->acc_pending = true;
        ctx->stats.outer_iters = 0;
        ctx->stats.inner_iters = 0;
        ctx->stats.max_rel_residual = 0.0;
    }
    return SPDE_OK;
}

// wait for every call enqueued on the context and fold the graph-driven solves'
// outcome into ctx->stats and ctx->deferred; with take, return the deferred
// outcome (SPDE_OK, ENOCONV or ETIMEOUT) and clear it
spde_status drain_calls(spde_ctx* ctx, bool take) {
    for (auto& L : ctx->lev) L.ws.quiesce();
    if (ctx->acc_pending) {
        CUDA_TRY(cudaMemcpy(ctx->h_acc, ctx->d_acc, sizeof(CallAcc), cudaMemcpyDeviceToHost));
        ctx->acc_pending = false;
        const CallAcc& a = *ctx->h_acc;
        double worst = 0.0;
        std::memcpy(&worst, &a.worst_bits, sizeof worst);
        ctx->stats.outer_iters = std::max(ctx->stats.outer_iters, a.outer);
        ctx->stats.inner_iters = std::max(ctx->stats.inner_iters, a.inner);
        ctx->stats.max_rel_residual = std::max(ctx->stats.max_rel_residual, worst);
        ctx->deferred = std::max(ctx->deferred, a.status);
    }
    if (!take) return SPDE_OK;
    const int d = ctx->deferred;
    ctx->deferred = SPDE_OK;
    if (d == SPDE_ETIMEOUT)
        return fail(SPDE_ETIMEOUT, "a multigrid sweep gave up waiting for a plane copy; those results are invalid");
    if (d == SPDE_ENOCONV)
        return fail(SPDE_ENOCONV, "tolerance not reached: relative residual %.3e", ctx->stats.max_rel_residual);
    return SPDE_OK;
}

spde_status check_level(spde_ctx* ctx, int level) {
    if (!ctx) return fail(SPDE_EINVAL, "null context");
    if (level < 0 || level >= 16 || !ctx->lev[level].defined) return fail(SPDE_EINVAL, "level %d is not defined", level);
    return SPDE_OK;
}

spde_status check_params(double kappa, double sigma) {
    if (!(kappa > 0.0) || !std::isfinite(kappa)) return fail(SPDE_EINVAL, "kappa must be finite and > 0");
    if (!(sigma > 0.0) || !std::isfinite(sigma)) return fail(SPDE_EINVAL, "sigma must be finite and > 0");
    return SPDE_OK;
}

// columns per batch that fit in free memory (mixed path)
int batch_capacity(const Grid3& g, int S, bool inner64) {
    size_t freeb = 0, totb = 0;
    if (cudaMemGetInfo(&freeb, &totb) != cudaSuccess) {
        cudaGetLastError();
        return S;
    }
    int cap = S;
    while (cap > 1 && workspace_bytes(g, cap, inner64) > (int64_t)(0.85 * (double)freeb)) cap = (cap + 1) / 2;
    return cap;
}

// Draw `S` samples starting at `first` into ws.x64 (scaled solution).
// With fl (a level with fields), kappa and sigma are ignored: the right-hand side
// is -g_c h xi_c cell by cell and the operator takes (kappa_c h)^2 per cell.
spde_status solve_samples(spde_ctx* ctx, Level& L, int S, double kappa, double sigma, uint64_t seed, uint64_t first,
                          cudaStream_t st, const Fields* fl = nullptr, bool graph = false) {
    const int64_t n3 = L.g.cells();
    const double kh2 = fl ? fl->kh2_mean : (kappa * L.h) * (kappa * L.h);
    // scaled RHS cell block: h^{-1/2} (-g h^{3/2} xi) = -g h xi
    prof_begin(PK_NOISE, st);
    CUDA_TRY(launch_noise(n3, S, seed, first, fl ? 1.0 : -g_half(kappa, sigma) * L.h, L.ws.F, n3, st));
    if (fl) CUDA_TRY(launch_scale_cells(n3, S, L.ws.F, n3, fl->gh, st));
    prof_end(st, (double)S * (fl ? 24.0 : 8.0) * (double)n3);
    if (graph) {
        if (L.ws.inner64 == 1) return refine_solve_async<double>(ctx, L.g, kh2, S, L.ws, st, false, fl);
        return refine_solve_async<float>(ctx, L.g, kh2, S, L.ws, st, false, fl);
    }
    double rel = 0.0;
    int outer = 0, inner = 0;
    spde_status s;
    if (L.ws.inner64 == 1) s = refine_solve<double>(ctx, L.g, kh2, S, L.ws, &rel, &outer, &inner, st, false, fl);
    else s = refine_solve<float>(ctx, L.g, kh2, S, L.ws, &rel, &outer, &inner, st, false, fl);
    ctx->stats.outer_iters = std::max(ctx->stats.outer_iters, outer);
    ctx->stats.inner_iters = std::max(ctx->stats.inner_iters, inner);
    ctx->stats.max_rel_residual = std::max(ctx->stats.max_rel_residual, rel);
    return s;
}

spde_status write_output(Level& L, int S, int out_kind, void* out_dev, cudaStream_t st) {
    const int64_t n3 = L.g.cells(), N4 = 4 * n3;
    const int kind = out_kind & 15;
    const int out64 = (out_kind & SPDE_OUT_F64) ? 1 : 0;
    const double unscale = 1.0 / std::sqrt(L.h);  // theta = h^{-1/2} scaled theta
    if (kind == SPDE_OUT_GRID_GAUSSIAN) {
        CUDA_TRY(launch_grid_out(n3, S, L.ws.x64 + 3 * n3, N4, unscale, out64, out_dev, st));
        return SPDE_OK;
    }
    if (!L.mesh.rowptr) return fail(SPDE_EINVAL, "no mesh attached to this level");
    prof_begin(PK_TRANSPOSE, st);
    CUDA_TRY(launch_transpose_theta(n3, S, L.ws.x64 + 3 * n3, N4, unscale, L.ws.thetaT, st));
    prof_end(st, (double)S * 12.0 * (double)n3);
    prof_begin(PK_PROJECT, st);
    CUDA_TRY(launch_project(L.mesh.ntets, S, L.mesh.rowptr, L.mesh.col, L.mesh.pi, L.ws.thetaT,
                            kind == SPDE_OUT_LOGNORMAL ? 0 : 1, out64, out_dev, st));
    // CSR once, the covered cells' rows of thetaT once, the output once
    prof_end(st, 8.0 * (double)(L.mesh.ntets + 1) + 8.0 * (double)L.mesh.nnz +
                     4.0 * (double)S * (double)L.mesh.ncols_used + (out64 ? 8.0 : 4.0) * (double)S * L.mesh.ntets);
    return SPDE_OK;
}

size_t out_elem_count(const Level& L, int S, int out_kind) {
    const int kind = out_kind & 15;
    const size_t per = kind == SPDE_OUT_GRID_GAUSSIAN ? (size_t)L.g.cells() : (size_t)L.mesh.ntets;
    return per * (size_t)S;
}

// makes the context's profiler visible to the launch wrappers for one call
struct ProfScope {
    explicit ProfScope(Profiler& p) { t_prof = &p; }
    ~ProfScope() { t_prof = nullptr; }
};

// device address of pinned host memory of the current device (mapped: unified addressing),
// or null when the pointer is not such memory
void* mapped_host_pointer(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    int dev = -1;
    if (a.type != cudaMemoryTypeHost || !a.devicePointer || cudaGetDevice(&dev) != cudaSuccess || a.device != dev)
        return nullptr;
    return a.devicePointer;
}

bool is_host_pointer(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

}  // namespace

namespace {

// ============================================================================
// Serving: continuous batching of sample requests.
//
// One lane per level: its own stream, worker thread and workspace of `cap`
// columns.  Every column carries its own kappa (the operator's (kappa h)^2 and
// the V-cycle's level coefficients per column), so requests for different
// kappa and sigma share a batch.  A lane works in rounds; a round is one
// refinement step of every occupied column (residual -> retire converged
// columns into their requests' outputs -> one batched inner MINRES solve ->
// correction).  Free columns take the next queued samples at every round
// boundary, so requests that arrive while others run join the batch without
// waiting for it to drain, and lanes of different levels overlap on the
// device.  Each column follows exactly the per-column sequence of
// spde_sample (the per-column coefficients are computed by the same host code
// as spde_sample's single ones), so a sample's result does not depend on the
// mix it ran in.
// ============================================================================
double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ServeReq {
    int64_t id = 0;
    int level = 0, nsamples = 0, out_kind = 0;
    double kappa = 0.0, sigma = 0.0;
    uint64_t seed = 0, first = 0;
    void* out = nullptr;
    int admitted = 0, finished = 0, dropped = 0;
    bool cancelled = false, done = false;
    spde_status status = SPDE_OK;
    double t_submit = 0.0, t_done = 0.0;
};
using ReqPtr = std::shared_ptr<ServeReq>;

struct Lane {
    struct Slot {
        ReqPtr req;
        int j = -1;          // sample index within the request
        int outer = 0;       // refinement steps done
        bool used = false;
        bool fresh = false;  // admitted this round
        double fnorm2 = 0.0;
    };
    Server* srv = nullptr;
    int level = 0;
    int cap = 0;
    int64_t bytes = 0;
    cudaStream_t st = nullptr;
    Workspace ws;
    std::deque<ReqPtr> queue;  // requests with samples not yet admitted (guarded by Server::mu)
    std::vector<Slot> slots;
    uint64_t *d_seed = nullptr, *d_sample = nullptr, *h_seed = nullptr, *h_sample = nullptr;
    double *d_scale = nullptr, *h_scale = nullptr;
    int *d_mask = nullptr, *h_mask = nullptr, *d_cols = nullptr, *h_cols = nullptr;
    int *d_fresh = nullptr, *h_fresh = nullptr;  // separate buffer: its copy may still be pending
    // each column's own kappa: (kappa h)^2 in FP64 and FP32, and the V-cycle sweep coefficients
    // of the tiled levels ([level][column][21], FP32)
    double *d_kh2 = nullptr, *h_kh2 = nullptr;
    float *d_kh2f = nullptr, *h_kh2f = nullptr;
    float *d_qtab = nullptr, *h_qtab = nullptr;
    int ntiled = 0;
    void **d_outs = nullptr, **h_outs = nullptr;
    std::thread th;
    std::condition_variable cv;
    bool stop = false;
    bool dead = false;
};

struct Server {
    spde_ctx* ctx = nullptr;
    std::mutex mu;
    std::map<int64_t, ReqPtr> reqs;
    std::deque<ReqPtr> pending;  // waiting for a lane (memory budget)
    std::map<std::pair<int, double>, std::unique_ptr<Lane>> lanes;
    std::vector<std::unique_ptr<Lane>> graveyard;  // exited lanes, joined outside their thread
    int64_t next_id = 1;
    int64_t used_bytes = 0;
};

int64_t lane_param_bytes(int cap) { return (int64_t)cap * ((8 + 8 + 8 + 4 + 4 + 4 + 8 + 8 + 4) * 2 + 16 * 21 * 4 * 2); }

void lane_free(Lane* L) {
    L->ws.release();
    dev_free(L->d_seed);
    dev_free(L->d_sample);
    dev_free(L->d_scale);
    dev_free(L->d_mask);
    dev_free(L->d_fresh);
    dev_free(L->d_cols);
    dev_free(L->d_kh2);
    dev_free(L->d_kh2f);
    dev_free(L->d_qtab);
    if (L->h_kh2) cudaFreeHost(L->h_kh2);
    if (L->h_kh2f) cudaFreeHost(L->h_kh2f);
    if (L->h_qtab) cudaFreeHost(L->h_qtab);
    L->h_kh2 = nullptr;
    L->h_kh2f = nullptr;
    L->h_qtab = nullptr;
    if (L->d_outs) cudaFree(L->d_outs);
    L->d_outs = nullptr;
    if (L->h_seed) cudaFreeHost(L->h_seed);
    if (L->h_sample) cudaFreeHost(L->h_sample);
    if (L->h_scale) cudaFreeHost(L->h_scale);
    if (L->h_mask) cudaFreeHost(L->h_mask);
    if (L->h_fresh) cudaFreeHost(L->h_fresh);
    if (L->h_cols) cudaFreeHost(L->h_cols);
    if (L->h_outs) cudaFreeHost(L->h_outs);
    L->h_seed = L->h_sample = nullptr;
    L->h_scale = nullptr;
    L->h_mask = L->h_cols = L->h_fresh = nullptr;
    L->h_outs = nullptr;
    if (L->st) cudaStreamDestroy(L->st);
    L->st = nullptr;
    cudaGetLastError();
}

spde_status lane_alloc(Lane* L, const Grid3& g) {
    const int cap = L->cap;
    if (cudaStreamCreateWithFlags(&L->st, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return fail(SPDE_ECUDA, "stream creation failed");
    }
    STATUS_TRY(ensure_workspace(L->ws, g, cap, false));
    STATUS_TRY(dev_alloc(&L->d_seed, cap));
    STATUS_TRY(dev_alloc(&L->d_sample, cap));
    STATUS_TRY(dev_alloc(&L->d_scale, cap));
    STATUS_TRY(dev_alloc(&L->d_mask, cap));
    STATUS_TRY(dev_alloc(&L->d_fresh, cap));
    STATUS_TRY(dev_alloc(&L->d_cols, cap));
    {
        MGPlan p;
        mg_plan_init(p, g, 0.0, 1.0, 0.8);
        L->ntiled = p.lc;
    }
    STATUS_TRY(dev_alloc(&L->d_kh2, cap));
    STATUS_TRY(dev_alloc(&L->d_kh2f, cap));
    STATUS_TRY(dev_alloc(&L->d_qtab, (size_t)std::max(L->ntiled, 1) * cap * 21));
    if (cudaMallocHost(&L->h_kh2, cap * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&L->h_kh2f, cap * sizeof(float)) != cudaSuccess ||
        cudaMallocHost(&L->h_qtab, (size_t)std::max(L->ntiled, 1) * cap * 21 * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SPDE_ENOMEM, "lane parameter allocation failed");
    }
    if (cudaMalloc(&L->d_outs, cap * sizeof(void*)) != cudaSuccess ||
        cudaMallocHost(&L->h_seed, cap * sizeof(uint64_t)) != cudaSuccess ||
        cudaMallocHost(&L->h_sample, cap * sizeof(uint64_t)) != cudaSuccess ||
        cudaMallocHost(&L->h_scale, cap * sizeof(double)) != cudaSuccess ||
        cudaMallocHost(&L->h_mask, cap * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&L->h_fresh, cap * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&L->h_cols, cap * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&L->h_outs, cap * sizeof(void*)) != cudaSuccess) {
        cudaGetLastError();
        return fail(SPDE_ENOMEM, "lane parameter allocation failed");
    }
    L->slots.assign(cap, Lane::Slot());
    return SPDE_OK;
}

// One refinement step of every occupied column (no lock held).
spde_status lane_round(Lane* L, std::vector<int>& finished) {
    spde_ctx* ctx = L->srv->ctx;
    Level& LV = ctx->lev[L->level];
    L->ws.o = level_opts(ctx->opts, LV);
    const spde_opts& o = L->ws.o;
    const Grid3 g = LV.g;
    const int S = L->cap;
    const int64_t n3 = g.cells(), N4 = 4 * n3;
    Workspace& ws = L->ws;
    cudaStream_t st = L->st;
    finished.clear();
    // every column carries its own kappa: (kappa h)^2 and the sweep coefficients of the
    // tiled levels, computed exactly as spde_sample computes them for one kappa
    double kh2 = 1.0;  // the scalar arguments (the per-column values take precedence)
    {
        MGPlan base;
        mg_plan_init(base, g, 1.0, o.schur_c, o.omega);
        for (int c = 0; c < S; ++c) {
            const Lane::Slot& sl = L->slots[c];
            const double k2 = sl.used ? (sl.req->kappa * LV.h) * (sl.req->kappa * LV.h) : 1.0;
            if (sl.used) kh2 = k2;
            L->h_kh2[c] = k2;
            L->h_kh2f[c] = (float)k2;
            for (int l = 0; l < L->ntiled; ++l) mg_coef_row<float>(base, l, k2, L->h_qtab + ((size_t)l * S + c) * 21);
        }
        CUDA_TRY(cudaMemcpyAsync(L->d_kh2, L->h_kh2, S * sizeof(double), cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(L->d_kh2f, L->h_kh2f, S * sizeof(float), cudaMemcpyHostToDevice, st));
        if (L->ntiled)
            CUDA_TRY(cudaMemcpyAsync(L->d_qtab, L->h_qtab, (size_t)L->ntiled * S * 21 * sizeof(float),
                                     cudaMemcpyHostToDevice, st));
    }
    ColKappa ck;
    ck.kh2_64 = L->d_kh2;
    ck.kh2_t = L->d_kh2f;
    for (int l = 0; l < L->ntiled; ++l) ck.qtab[l] = L->d_qtab + (size_t)l * S * 21;
    // fresh columns: noise, zero iterate, ||F||^2
    bool any_fresh = false, any_old = false;
    for (int c = 0; c < S; ++c) {
        const Lane::Slot& sl = L->slots[c];
        L->h_fresh[c] = (sl.used && sl.fresh) ? 1 : 0;
        if (sl.used && sl.fresh) {
            any_fresh = true;
            L->h_seed[c] = sl.req->seed;
            L->h_sample[c] = sl.req->first + (uint64_t)sl.j;
            L->h_scale[c] = -g_half(sl.req->kappa, sl.req->sigma) * LV.h;
        } else {
            L->h_seed[c] = 0;
            L->h_sample[c] = 0;
            L->h_scale[c] = 0.0;
        }
        if (sl.used && !sl.fresh) any_old = true;
    }
    if (any_fresh) {
        CUDA_TRY(cudaMemcpyAsync(L->d_seed, L->h_seed, S * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(L->d_sample, L->h_sample, S * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(L->d_scale, L->h_scale, S * sizeof(double), cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(L->d_fresh, L->h_fresh, S * sizeof(int), cudaMemcpyHostToDevice, st));
        CUDA_TRY(launch_noise_cols(n3, S, L->d_seed, L->d_sample, L->d_scale, L->d_fresh, ws.F, n3, st));
        for (int c = 0; c < S; ++c)
            if (L->h_fresh[c]) CUDA_TRY(cudaMemsetAsync(ws.x64 + (int64_t)c * N4, 0, N4 * sizeof(double), st));
        const int nb = launch_sumsq(n3, S, ws.F, n3, ws.partR, st);
        CUDA_TRY(launch_reduce(S, ws.partR, nb, ws.colv + S, st));
    }
    // residual of every occupied column (flux rows exact from theta first)
    for (int c = 0; c < S; ++c) L->h_mask[c] = L->slots[c].used ? 1 : 0;
    CUDA_TRY(cudaMemcpyAsync(L->d_mask, L->h_mask, S * sizeof(int), cudaMemcpyHostToDevice, st));
    if (any_old) CUDA_TRY(launch_flux_from_theta(g, S, ws.x64, N4, ws.tri, st));
    const int nbr = launch_residual64(g, kh2, S, ws.F, n3, ws.x64, static_cast<float*>(ws.vec[4]), nullptr, ws.partR,
                                      L->d_mask, st, nullptr, L->d_kh2);
    CUDA_TRY(launch_reduce(S, ws.partR, nbr, ws.colv, st));
    CUDA_TRY(cudaMemcpyAsync(ws.h_col, ws.colv, 2 * S * sizeof(double), cudaMemcpyDeviceToHost, st));
    int fault = 0;
    CUDA_TRY(mg_fault_read(ws.fault, &fault, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    STATUS_TRY(fault_status(fault, ws.fault, st));
    std::vector<int> going;
    for (int c = 0; c < S; ++c) {
        Lane::Slot& sl = L->slots[c];
        if (!sl.used) continue;
        if (sl.fresh) sl.fnorm2 = ws.h_col[S + c];
        sl.fresh = false;
        const double rel = sl.fnorm2 > 0.0 ? std::sqrt(ws.h_col[c] / sl.fnorm2) : 0.0;
        ws.h_tol[c] = inner_tol_for(o, rel);
        if (rel <= o.tol || sl.outer >= o.max_outer || sl.req->cancelled) {
            if (rel > o.tol && !sl.req->cancelled) sl.req->status = SPDE_ENOCONV;
            finished.push_back(c);
        } else {
            going.push_back(c);
        }
    }
    // retire: write each finished column into its request's output
    const double unscale = 1.0 / std::sqrt(LV.h);
    for (int pass = 0; pass < 2; ++pass) {  // pass 0: float outputs, pass 1: double outputs
        int R = 0;
        int kind_any = -1;
        for (int c : finished) {
            const Lane::Slot& sl = L->slots[c];
            if (sl.req->cancelled) continue;
            const int kind = sl.req->out_kind & 15;
            const int out64 = (sl.req->out_kind & SPDE_OUT_F64) ? 1 : 0;
            if (out64 != pass) continue;
            const size_t esz = out64 ? 8 : 4;
            if (kind == SPDE_OUT_GRID_GAUSSIAN) {
                void* dst = static_cast<char*>(sl.req->out) + (size_t)sl.j * n3 * esz;
                CUDA_TRY(launch_grid_out(n3, 1, ws.x64 + (int64_t)c * N4 + 3 * n3, N4, unscale, out64, dst, st));
            } else {
                // tet outputs are grouped by kind below
                (void)kind_any;
            }
        }
        for (int kind = 0; kind < 2; ++kind) {
            R = 0;
            for (int c : finished) {
                const Lane::Slot& sl = L->slots[c];
                if (sl.req->cancelled) continue;
                const int out64 = (sl.req->out_kind & SPDE_OUT_F64) ? 1 : 0;
                if (out64 != pass || (sl.req->out_kind & 15) != kind) continue;
                const size_t esz = out64 ? 8 : 4;
                L->h_cols[R] = c;
                L->h_outs[R] = static_cast<char*>(sl.req->out) + (size_t)sl.j * (size_t)LV.mesh.ntets * esz;
                ++R;
            }
            if (R == 0) continue;
            CUDA_TRY(cudaMemcpyAsync(L->d_cols, L->h_cols, R * sizeof(int), cudaMemcpyHostToDevice, st));
            CUDA_TRY(cudaMemcpyAsync(L->d_outs, L->h_outs, R * sizeof(void*), cudaMemcpyHostToDevice, st));
            CUDA_TRY(launch_transpose_cols(n3, R, L->d_cols, ws.x64 + 3 * n3, N4, unscale, ws.thetaT, st));
            CUDA_TRY(launch_project_ptrs(LV.mesh.ntets, R, LV.mesh.rowptr, LV.mesh.col, LV.mesh.pi, ws.thetaT,
                                         kind == SPDE_OUT_LOGNORMAL ? 0 : 1, pass, L->d_outs, st));
            CUDA_TRY(cudaStreamSynchronize(st));  // host arrays are reused by the next group
        }
    }
    // one inner MINRES solve for the columns still going, then the correction
    if (!going.empty()) {
        for (int c = 0; c < S; ++c) L->h_mask[c] = 0;
        for (int c : going) L->h_mask[c] = 1;
        CUDA_TRY(cudaMemcpyAsync(L->d_mask, L->h_mask, S * sizeof(int), cudaMemcpyHostToDevice, st));
        CUDA_TRY(launch_set_active(S, L->d_mask, ws.st, st));
        int its = 0;
        CUDA_TRY(cudaMemcpyAsync(ws.coltol, ws.h_tol, S * sizeof(double), cudaMemcpyHostToDevice, st));
        STATUS_TRY(minres_batch<float>(o, g, kh2, S, ws, o.inner_tol, &its, st, nullptr, nullptr, ws.coltol, &ck));
        CUDA_TRY(launch_add_theta<float>(n3, S, ws.x64, static_cast<const float*>(ws.vec[0]), ws.st, st));
        for (int c : going) L->slots[c].outer += 1;
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    return SPDE_OK;
}

void server_dispatch(Server* srv);  // lock held

void lane_main(Lane* L) {
    Server* srv = L->srv;
    cudaSetDevice(srv->ctx->opts.device);
    std::vector<int> finished;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            auto any_used = [&] {
                for (auto& sl : L->slots)
                    if (sl.used) return true;
                return false;
            };
            if (!any_used() && L->queue.empty()) {
                L->cv.wait_for(lk, std::chrono::milliseconds(200),
                               [&] { return L->stop || !L->queue.empty(); });
                if (!any_used() && L->queue.empty()) {
                    // idle: give the memory back, let waiting requests use it
                    L->dead = true;
                    break;
                }
            }
            if (L->stop && !any_used()) break;
            // admit queued samples into free columns
            for (auto& sl : L->slots) {
                if (sl.used) continue;
                while (!L->queue.empty() && (L->queue.front()->cancelled ||
                                             L->queue.front()->admitted >= L->queue.front()->nsamples))
                    L->queue.pop_front();
                if (L->queue.empty()) break;
                ReqPtr r = L->queue.front();
                sl.req = r;
                sl.j = r->admitted++;
                sl.outer = 0;
                sl.used = true;
                sl.fresh = true;
                sl.fnorm2 = 0.0;
            }
        }
        const spde_status s = lane_round(L, finished);
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            const double t = now_s();
            auto close_req = [&](const ReqPtr& r) {
                if (!r->done && r->finished + r->dropped >= r->nsamples) {
                    r->done = true;
                    r->t_done = t;
                }
            };
            if (s != SPDE_OK) {
                // a CUDA or allocation failure ends every request in this lane
                for (auto& sl : L->slots)
                    if (sl.used) {
                        sl.req->status = s;
                        sl.req->dropped += 1;
                        close_req(sl.req);
                        sl.used = false;
                        sl.req.reset();
                    }
                for (auto& r : L->queue) {
                    r->status = s;
                    r->dropped += r->nsamples - r->admitted;
                    r->admitted = r->nsamples;
                    close_req(r);
                }
                L->queue.clear();
                continue;
            }
            for (int c : finished) {
                Lane::Slot& sl = L->slots[c];
                if (sl.req->cancelled) sl.req->dropped += 1;
                else sl.req->finished += 1;
                close_req(sl.req);
                sl.used = false;
                sl.req.reset();
            }
            for (auto& r : L->queue)
                if (r->cancelled && r->admitted < r->nsamples) {
                    r->dropped += r->nsamples - r->admitted;
                    r->admitted = r->nsamples;
                    close_req(r);
                }
        }
    }
    lane_free(L);
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->used_bytes -= L->bytes;
    L->dead = true;
    auto it = srv->lanes.find({L->level, 0.0});
    if (it != srv->lanes.end() && it->second.get() == L) {
        srv->graveyard.push_back(std::move(it->second));
        srv->lanes.erase(it);
    }
    server_dispatch(srv);
}

// route pending requests to lanes, creating lanes within the memory budget (lock held)
void server_dispatch(Server* srv) {
    spde_ctx* ctx = srv->ctx;
    const spde_opts& o = ctx->opts;
    std::deque<ReqPtr> still;
    while (!srv->pending.empty()) {
        ReqPtr r = srv->pending.front();
        srv->pending.pop_front();
        if (r->cancelled) {
            r->dropped = r->nsamples - r->finished;
            r->admitted = r->nsamples;
            if (!r->done) {
                r->done = true;
                r->t_done = now_s();
            }
            continue;
        }
        auto key = std::make_pair(r->level, 0.0);  // one lane per level: columns carry their own kappa
        auto it = srv->lanes.find(key);
        if (it != srv->lanes.end() && !it->second->dead) {
            it->second->queue.push_back(r);
            it->second->cv.notify_one();
            continue;
        }
        if (it != srv->lanes.end()) {  // exiting lane: its thread releases its memory
            srv->graveyard.push_back(std::move(it->second));
            srv->lanes.erase(it);
        }
        const Grid3 g = ctx->lev[r->level].g;
        const int64_t per_col = workspace_bytes(g, 1, false);
        int cap = std::max(1, std::min(o.serve_max_batch, (int)(o.serve_budget_bytes / 4 / std::max<int64_t>(per_col, 1))));
        while (cap > 1 && srv->used_bytes + workspace_bytes(g, cap, false) + lane_param_bytes(cap) > o.serve_budget_bytes)
            cap /= 2;
        const int64_t need = workspace_bytes(g, cap, false) + lane_param_bytes(cap);
        if (srv->used_bytes + need > o.serve_budget_bytes) {
            still.push_back(r);  // wait for a lane to free memory
            continue;
        }
        std::unique_ptr<Lane> L(new Lane());
        L->srv = srv;
        L->level = r->level;
        L->cap = cap;
        L->bytes = need;
        cudaSetDevice(ctx->opts.device);
        const spde_status s = lane_alloc(L.get(), g);
        if (s != SPDE_OK) {
            lane_free(L.get());
            still.push_back(r);
            if (srv->lanes.empty()) {  // nothing can free memory: fail the request
                still.pop_back();
                r->status = s;
                r->dropped = r->nsamples;
                r->admitted = r->nsamples;
                r->done = true;
                r->t_done = now_s();
            }
            continue;
        }
        srv->used_bytes += need;
        L->queue.push_back(r);
        Lane* raw = L.get();
        srv->lanes[key] = std::move(L);
        raw->th = std::thread(lane_main, raw);
    }
    srv->pending = std::move(still);
}

void server_reap(Server* srv) {  // join exited lanes (lock not held)
    std::vector<std::unique_ptr<Lane>> g;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        g.swap(srv->graveyard);
    }
    for (auto& L : g)
        if (L->th.joinable()) L->th.join();
}

void server_stop(Server* srv) {
    std::vector<Lane*> ls;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        for (auto& r : srv->pending) r->cancelled = true;
        srv->pending.clear();
        for (auto& kv : srv->lanes) {
            for (auto& r : kv.second->queue) r->cancelled = true;
            kv.second->stop = true;
            kv.second->cv.notify_all();
            ls.push_back(kv.second.get());
        }
    }
    for (;;) {  // lanes move themselves to the graveyard when they exit
        server_reap(srv);
        std::lock_guard<std::mutex> lk(srv->mu);
        if (srv->lanes.empty()) break;
        for (auto& kv : srv->lanes) kv.second->cv.notify_all();
        std::this_thread::sleep_for(std::chrono::milliseconds(1));
    }
    server_reap(srv);
}

bool serving_busy(spde_ctx* ctx) {
    Server* srv = ctx->srv;
    if (!srv) return false;
    std::lock_guard<std::mutex> lk(srv->mu);
    return !srv->lanes.empty() || !srv->pending.empty() || !srv->reqs.empty();
}

}  // namespace

namespace spde {
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace spde

// ============================================================================
extern "C" {

spde_status spde_opts_init(spde_opts* o) {
    if (!o) return fail(SPDE_EINVAL, "null opts");
    o->precision = SPDE_PREC_MIXED;
    o->tol = 1e-10;
    o->inner_tol = 1e-5;
    o->max_outer = 8;
    o->max_iter = 400;
    o->omega = 0.8;
    o->schur_c = 1.0;
    o->flux_diag = 1.5;
    o->check_every = 8;
    o->device = 0;
    o->use_graphs = 1;
    o->serve_budget_bytes = (int64_t)120 << 30;
    o->serve_max_batch = 64;
    o->solver = SPDE_SOLVER_MINRES;
    o->sweep_planes = 0;
    o->coarse_fp16 = 0;
    o->sweep_rows = 1;
    return SPDE_OK;
}

spde_status spde_grid_create(spde_ctx** ctx, const spde_opts* opts) {
    if (!ctx) return fail(SPDE_EINVAL, "null ctx pointer");
    *ctx = nullptr;
    spde_opts o;
    spde_opts_init(&o);
    if (opts) o = *opts;
    if (o.precision != SPDE_PREC_MIXED && o.precision != SPDE_PREC_FP64) return fail(SPDE_EINVAL, "bad precision");
    if (o.solver != SPDE_SOLVER_MINRES && o.solver != SPDE_SOLVER_SCHUR_CG) return fail(SPDE_EINVAL, "bad solver");
    if (!(o.tol > 0.0) || !(o.inner_tol > 0.0) || o.max_outer < 1 || o.max_iter < 1 || o.check_every < 1)
        return fail(SPDE_EINVAL, "bad tolerance or iteration limits");
    if (!(o.omega > 0.0 && o.omega < 1.0)) return fail(SPDE_EINVAL, "omega must lie in (0, 1)");
    if (!(o.schur_c > 0.0) || !(o.flux_diag > 0.0)) return fail(SPDE_EINVAL, "preconditioner weights must be > 0");
    if (o.serve_budget_bytes <= 0 || o.serve_max_batch < 1 || o.serve_max_batch > 65535)
        return fail(SPDE_EINVAL, "bad serving budget or batch size");
    if (o.sweep_planes != 0 && o.sweep_planes != 8 && o.sweep_planes != 16 && o.sweep_planes != 32 &&
        o.sweep_planes != 64)
        return fail(SPDE_EINVAL, "sweep_planes must be 0, 8, 16, 32 or 64");
    int ndev = 0;
    CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (o.device < 0 || o.device >= ndev) return fail(SPDE_EINVAL, "device %d not present", o.device);
    CUDA_TRY(cudaSetDevice(o.device));
    spde_ctx* c = new spde_ctx();
    c->opts = o;
    std::memset(&c->stats, 0, sizeof c->stats);
    *ctx = c;
    return SPDE_OK;
}

namespace {
// a level of nx x ny x nz cells on the box lo .. hi (equal spacing on every axis)
spde_status level_add_impl(spde_ctx* ctx, int level, const int n[3], const double lo[3], const double hi[3]) {
    if (!ctx || !lo || !hi) return fail(SPDE_EINVAL, "null argument");
    if (level < 0 || level >= 16) return fail(SPDE_EINVAL, "level must lie in [0, 16)");
    for (int a = 0; a < 3; ++a)
        if (!is_pow2(n[a]) || n[a] < 4 || n[a] > 1024)
            return fail(SPDE_EINVAL, "cells per axis must be powers of two in [4, 1024]");
    if ((int64_t)n[0] * n[1] * n[2] > kMaxGridCells)
        return fail(SPDE_EINVAL, "at most 2^29 cells per grid (a cube of at most 512^3)");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(lo[a]) || !std::isfinite(hi[a]) || !(hi[a] > lo[a]))
            return fail(SPDE_EINVAL, "box must have hi > lo on every axis");
    const double h = (hi[0] - lo[0]) / n[0];
    for (int a = 1; a < 3; ++a)
        if (std::fabs((hi[a] - lo[a]) / n[a] - h) > 1e-12 * h) return fail(SPDE_EINVAL, "cells must be cubes");
    const Grid3 gr = make_grid(n[0], n[1], n[2]);
    if (!mg_grid_supported(gr))
        return fail(SPDE_EINVAL,
                    "grid %d x %d x %d not supported: the first level whose extents are not multiples of 32 x 16 x 8 "
                    "must have at most 4096 cells",
                    n[0], n[1], n[2]);
    std::lock_guard<std::mutex> g(ctx->mu);
    if (serving_busy(ctx)) return fail(SPDE_EBUSY, "requests are in flight; grids cannot change");
    CUDA_TRY(cudaSetDevice(ctx->opts.device));
    Level& L = ctx->lev[level];
    L.ws.release();  // waits for calls still using the level
    L.mesh.release();
    L.fields.release();
    L.defined = true;
    L.g = gr;
    L.h = h;
    for (int a = 0; a < 3; ++a) L.lo[a] = lo[a];
    return SPDE_OK;
}
}  // namespace

spde_status spde_level_add(spde_ctx* ctx, int level, int n, const double lo[3], const double hi[3]) {
    if (!is_pow2(n) || n < 4 || n > 512) return fail(SPDE_EINVAL, "n must be a power of two in [4, 512]");
    if (lo && hi) {
        const double ext = hi[0] - lo[0];
        for (int a = 0; a < 3; ++a)
            if (std::isfinite(lo[a]) && std::isfinite(hi[a]) && hi[a] > lo[a] &&
                std::fabs((hi[a] - lo[a]) - ext) > 1e-12 * ext)
                return fail(SPDE_EINVAL, "cells must be cubes (spde_level_add_box takes a box of n[0] x n[1] x n[2] cells)");
    }
    const int nn[3] = {n, n, n};
    return level_add_impl(ctx, level, nn, lo, hi);
}

spde_status spde_level_add_box(spde_ctx* ctx, int level, const int n[3], const double lo[3], const double hi[3]) {
    if (!n) return fail(SPDE_EINVAL, "null argument");
    return level_add_impl(ctx, level, n, lo, hi);
}

spde_status spde_mesh_attach(spde_ctx* ctx, int level, int64_t nverts, const double* xyz, int64_t ntets,
                             const int32_t* tets) {
    STATUS_TRY(check_level(ctx, level));
    if (nverts < 4 || ntets < 1 || !xyz || !tets) return fail(SPDE_EINVAL, "empty mesh");
    if (ntets > (int64_t)1 << 31) return fail(SPDE_EINVAL, "too many tets");
    std::lock_guard<std::mutex> g(ctx->mu);
    if (serving_busy(ctx)) return fail(SPDE_EBUSY, "requests are in flight; meshes cannot change");
    CUDA_TRY(cudaSetDevice(ctx->opts.device));
    Level& L = ctx->lev[level];
    L.ws.quiesce();  // a call still projecting onto the old mesh
    L.mesh.release();
    Mesh& m = L.mesh;
    cudaStream_t st = nullptr;
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    STATUS_TRY(dev_alloc(&m.xyz, (size_t)nverts * 3));
    STATUS_TRY(dev_alloc(&m.tets, (size_t)ntets * 4));
    STATUS_TRY(dev_alloc(&m.vol, (size_t)ntets));
    CUDA_TRY(cudaMemcpy(m.xyz, xyz, (size_t)nverts * 3 * sizeof(double), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(m.tets, tets, (size_t)ntets * 4 * sizeof(int32_t), cudaMemcpyHostToDevice));
    ClipResult res;
    CUDA_TRY(cudaEventRecord(e0, st));
    const int gn[3] = {L.g.nx, L.g.ny, L.g.nz};
    cudaError_t e = build_coupling(gn, L.h, L.lo, nverts, m.xyz, ntets, m.tets, m.vol, &m.rowptr, &m.col, &m.g,
                                   &m.pi, &res, st);
    CUDA_TRY(cudaEventRecord(e1, st));
    CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        m.release();
        return fail(e == cudaErrorMemoryAllocation ? SPDE_ENOMEM : SPDE_ECUDA, "coupling build failed: %s",
                    cudaGetErrorString(e));
    }
    if (res.bad_tet >= 0) {
        static const char* why[4] = {"", "degenerate or invalid tet", "tet outside the embedding box",
                                     "coupling row does not sum to the tet volume"};
        const int t = res.bad_tet, k = res.bad_kind;
        m.release();
        return fail(SPDE_EMESH, "mesh rejected: tet %d: %s", t, why[k & 3]);
    }
    m.nverts = nverts;
    m.ntets = ntets;
    m.nnz = res.nnz;
    {
        int64_t used = 0;
        CUDA_TRY(count_used_columns(res.nnz, m.col, L.g.cells(), &used, st));
        m.ncols_used = used;
    }
    ctx->stats.setup_ms = ms;
    ctx->stats.nnz = res.nnz;
    return SPDE_OK;
}

namespace {
spde_status sample_impl(spde_ctx* ctx, int level, int nsamples, double kappa, double sigma, bool use_fields,
                        uint64_t seed, uint64_t first_sample, int out_kind, void* out, void* stream);
}

spde_status spde_sample(spde_ctx* ctx, int level, int nsamples, double kappa, double sigma, uint64_t seed,
                        uint64_t first_sample, int out_kind, void* out, void* stream) {
    STATUS_TRY(check_level(ctx, level));
    STATUS_TRY(check_params(kappa, sigma));
    return sample_impl(ctx, level, nsamples, kappa, sigma, false, seed, first_sample, out_kind, out, stream);
}

spde_status spde_level_set_fields(spde_ctx* ctx, int level, const double* kappa_cells, const double* sigma_cells) {
    STATUS_TRY(check_level(ctx, level));
    if ((kappa_cells == nullptr) != (sigma_cells == nullptr))
        return fail(SPDE_EINVAL, "give both kappa and sigma, or neither (to clear the fields)");
    std::lock_guard<std::mutex> g(ctx->mu);
    if (serving_busy(ctx)) return fail(SPDE_EBUSY, "requests are in flight; fields cannot change");
    CUDA_TRY(cudaSetDevice(ctx->opts.device));
    Level& L = ctx->lev[level];
    L.ws.quiesce();
    L.ws.drop_graphs();  // captured graphs hold the old fields' addresses
    L.fields.release();
    if (!kappa_cells) return SPDE_OK;
    const int64_t n3 = L.g.cells();
    double sum = 0.0;
    for (int64_t e = 0; e < n3; ++e) {
        const double k = kappa_cells[e], sg = sigma_cells[e];
        if (!(k > 0.0) || !std::isfinite(k)) return fail(SPDE_EINVAL, "kappa must be finite and > 0 (cell %lld)", (long long)e);
        if (!(sg > 0.0) || !std::isfinite(sg)) return fail(SPDE_EINVAL, "sigma must be finite and > 0 (cell %lld)", (long long)e);
        sum += (k * L.h) * (k * L.h);
    }
    Fields& f = L.fields;
    double* dk = nullptr;
    double* ds = nullptr;
    spde_status st = dev_alloc(&f.kh2_64, (size_t)n3);
    if (st == SPDE_OK) st = dev_alloc(&f.kh2_32, (size_t)n3);
    if (st == SPDE_OK) st = dev_alloc(&f.gh, (size_t)n3);
    if (st == SPDE_OK) st = dev_alloc(&dk, (size_t)n3);
    if (st == SPDE_OK) st = dev_alloc(&ds, (size_t)n3);
    cudaError_t e = cudaSuccess;
    if (st == SPDE_OK) e = cudaMemcpy(dk, kappa_cells, (size_t)n3 * sizeof(double), cudaMemcpyHostToDevice);
    if (st == SPDE_OK && e == cudaSuccess)
        e = cudaMemcpy(ds, sigma_cells, (size_t)n3 * sizeof(double), cudaMemcpyHostToDevice);
    if (st == SPDE_OK && e == cudaSuccess) e = launch_field_coefs(n3, L.h, dk, ds, f.kh2_64, f.kh2_32, f.gh, 0);
    // multigrid diagonals, level by level: a_0 = (kappa_c h)^2, a_l = mean of the children
    double* a_prev = f.kh2_64;
    double* a_tmp[2] = {dk, ds};  // the device copies of kappa and sigma are free now: reuse them
    MGPlan hier;
    mg_plan_init(hier, L.g, 0.0, ctx->opts.schur_c, ctx->opts.omega);
    for (int l = 0; l < hier.nlev && st == SPDE_OK && e == cudaSuccess; ++l) {
        const size_t m = (size_t)hier.g[l].cells();
        st = dev_alloc(&f.D64[l], m);
        if (st == SPDE_OK) st = dev_alloc(&f.D32[l], m);
        if (st != SPDE_OK) break;
        double* a_l = a_prev;
        if (l > 0) {
            a_l = a_tmp[l & 1];
            e = launch_restrict_mean(hier.g[l - 1], a_prev, a_l, 0);
        }
        if (e == cudaSuccess)
            e = launch_level_diag(hier.g[l], hier.ls[l], hier.lq[l], ctx->opts.schur_c, a_l, f.D64[l], f.D32[l], 0);
        a_prev = a_l;
        if (e == cudaSuccess) e = cudaDeviceSynchronize();  // a_tmp alternates: finish before reuse
    }
    if (st == SPDE_OK && e == cudaSuccess) e = cudaDeviceSynchronize();
    dev_free(dk);
    dev_free(ds);
    if (st != SPDE_OK || e != cudaSuccess) {
        f.release();
        if (st != SPDE_OK) return st;
        CUDA_TRY(e);
    }
    f.kh2_mean = sum / (double)n3;
    f.set = true;
    return SPDE_OK;
}

spde_status spde_sample_fields(spde_ctx* ctx, int level, int nsamples, uint64_t seed, uint64_t first_sample,
                               int out_kind, void* out, void* stream) {
    STATUS_TRY(check_level(ctx, level));
    if (!ctx->lev[level].fields.set) return fail(SPDE_EINVAL, "level %d has no fields (spde_level_set_fields)", level);
    if (ctx->opts.solver != SPDE_SOLVER_MINRES) return fail(SPDE_EINVAL, "fields need the MINRES solver");
    return sample_impl(ctx, level, nsamples, 0.0, 0.0, true, seed, first_sample, out_kind, out, stream);
}

namespace {
// calls take the graph-driven path unless per-kernel timing is on (events cannot be
// recorded inside a graph's loops), graphs are switched off, or the inner solver is CG
bool graph_path(const spde_ctx* ctx) {
    return ctx->opts.use_graphs != 0 && !ctx->prof.on && ctx->opts.solver == SPDE_SOLVER_MINRES;
}

spde_status sample_impl(spde_ctx* ctx, int level, int nsamples, double kappa, double sigma, bool use_fields,
                        uint64_t seed, uint64_t first_sample, int out_kind, void* out, void* stream) {
    if (nsamples < 0) return fail(SPDE_EINVAL, "nsamples < 0");
    const int kind = out_kind & 15;
    if (kind > SPDE_OUT_GRID_GAUSSIAN || (out_kind & ~(15 | SPDE_OUT_F64))) return fail(SPDE_EINVAL, "bad out_kind");
    if (nsamples == 0) return SPDE_OK;
    if (!out) return fail(SPDE_EINVAL, "null output");
    std::lock_guard<std::mutex> g(ctx->mu);
    CUDA_TRY(cudaSetDevice(ctx->opts.device));
    ProfScope ps(ctx->prof);
    Level& L = ctx->lev[level];
    if (kind != SPDE_OUT_GRID_GAUSSIAN && !L.mesh.rowptr) return fail(SPDE_EINVAL, "no mesh attached to level %d", level);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool plain = ctx->opts.precision == SPDE_PREC_FP64;
    const bool graph = graph_path(ctx);
    const size_t esz = (out_kind & SPDE_OUT_F64) ? 8 : 4;
    const bool host_out = is_host_pointer(out);
    // pinned host memory of this device is written by the output kernels directly (over the
    // chip-to-chip link), with no staging buffer and copy; other host memory is staged and copied
    void* const host_mapped = host_out ? mapped_host_pointer(out) : nullptr;
    if (graph) {
        STATUS_TRY(async_call_begin(ctx, st));
    } else {
        ctx->stats.outer_iters = 0;
        ctx->stats.inner_iters = 0;
        ctx->stats.max_rel_residual = 0.0;
    }
    // plain path: one sample per solve; mixed path: batches that fit in memory
    int cap = 1;
    if (!plain) {
        if (L.ws.g == L.g && L.ws.S >= nsamples && L.ws.inner64 == 0) cap = nsamples;
        else {
            L.ws.release();
            cap = batch_capacity(L.g, nsamples, false);
        }
    }
    spde_status worst = SPDE_OK;
    for (int s0 = 0; s0 < nsamples; s0 += cap) {
        const int S = std::min(cap, nsamples - s0);
        STATUS_TRY(ensure_workspace(L.ws, L.g, plain ? 1 : std::min(cap, nsamples), plain));
        L.ws.o = level_opts(ctx->opts, L);
        if (graph) CUDA_TRY(cudaStreamWaitEvent(st, L.ws.done, 0));  // a call on another stream may still use it
        spde_status s = solve_samples(ctx, L, S, kappa, sigma, seed, first_sample + (uint64_t)s0, st,
                                      use_fields ? &L.fields : nullptr, graph);
        if (s != SPDE_OK && s != SPDE_ENOCONV) return s;
        if (s == SPDE_ENOCONV) worst = s;
        const size_t per = out_elem_count(L, 1, out_kind);
        void* dst = static_cast<char*>(out) + (size_t)s0 * per * esz;
        if (host_mapped) {
            STATUS_TRY(write_output(L, S, out_kind, static_cast<char*>(host_mapped) + (size_t)s0 * per * esz, st));
        } else if (host_out) {
            const size_t need = (size_t)S * per * esz;
            if (ctx->out_tmp_bytes < need) {
                if (ctx->out_tmp) {
                    CUDA_TRY(cudaStreamSynchronize(st));
                    cudaFree(ctx->out_tmp);
                }
                ctx->out_tmp = nullptr;
                ctx->out_tmp_bytes = 0;
                CUDA_TRY(cudaMalloc(&ctx->out_tmp, need));
                ctx->out_tmp_bytes = need;
            }
            STATUS_TRY(write_output(L, S, out_kind, ctx->out_tmp, st));
            CUDA_TRY(cudaMemcpyAsync(dst, ctx->out_tmp, need, cudaMemcpyDeviceToHost, st));
        } else {
            STATUS_TRY(write_output(L, S, out_kind, dst, st));
        }
        if (graph) CUDA_TRY(cudaEventRecord(L.ws.done, st));
    }
    if (graph && !host_out) return SPDE_OK;  // asynchronous: the outcome comes with spde_wait
    CUDA_TRY(cudaStreamSynchronize(st));
    if (graph) return drain_calls(ctx, true);  // host memory written: report the outcome now
    ctx->prof.flush();
    if (worst != SPDE_OK)
        return fail(worst, "tolerance not reached: relative residual %.3e", ctx->stats.max_rel_residual);
    return SPDE_OK;
}
}  // namespace

spde_status spde_submit(spde_ctx* ctx, int level, int nsamples, double kappa, double sigma, uint64_t seed,
                        uint64_t first_sample, int out_kind, void* out, int64_t* request) {
    STATUS_TRY(check_level(ctx, level));
    STATUS_TRY(check_params(kappa, sigma));
    if (!request) return fail(SPDE_EINVAL, "null request pointer");
    *request = 0;
    if (nsamples < 1) return fail(SPDE_EINVAL, "nsamples must be >= 1");
    const int kind = out_kind & 15;
    if (kind > SPDE_OUT_GRID_GAUSSIAN || (out_kind & ~(15 | SPDE_OUT_F64))) return fail(SPDE_EINVAL, "bad out_kind");
    if (!out) return fail(SPDE_EINVAL, "null output");
    if (ctx->opts.precision != SPDE_PREC_MIXED) return fail(SPDE_EINVAL, "serving runs the mixed-precision path");
    if (is_host_pointer(out)) return fail(SPDE_EINVAL, "serving writes device buffers only");
    if (kind != SPDE_OUT_GRID_GAUSSIAN && !ctx->lev[level].mesh.rowptr)
        return fail(SPDE_EINVAL, "no mesh attached to level %d", level);
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        if (!ctx->srv) {
            ctx->srv = new Server();
            ctx->srv->ctx = ctx;
        }
    }
    Server* srv = ctx->srv;
    server_reap(srv);
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->reqs.size() >= 100000) return fail(SPDE_EBUSY, "request table full");
    ReqPtr r = std::make_shared<ServeReq>();
    r->id = srv->next_id++;
    r->level = level;
    r->nsamples = nsamples;
    r->kappa = kappa;
    r->sigma = sigma;
    r->seed = seed;
    r->first = first_sample;
    r->out_kind = out_kind;
    r->out = out;
    r->t_submit = now_s();
    srv->reqs[r->id] = r;
    srv->pending.push_back(r);
    server_dispatch(srv);
    *request = r->id;
    return SPDE_OK;
}

spde_status spde_poll(spde_ctx* ctx, int64_t request, int* done, double* latency_ms, int* result) {
    if (!ctx || !done) return fail(SPDE_EINVAL, "null argument");
    Server* srv = ctx->srv;
    if (!srv) return fail(SPDE_EINVAL, "unknown request %lld", (long long)request);
    server_reap(srv);
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(request);
    if (it == srv->reqs.end()) return fail(SPDE_EINVAL, "unknown request %lld", (long long)request);
    const ReqPtr& r = it->second;
    *done = r->done ? 1 : 0;
    if (latency_ms) *latency_ms = r->done ? 1000.0 * (r->t_done - r->t_submit) : 1000.0 * (now_s() - r->t_submit);
    if (result) *result = r->done ? (r->cancelled ? SPDE_ECANCELED : r->status) : SPDE_OK;
    if (r->done) srv->reqs.erase(it);  // a finished request is reported once
    return SPDE_OK;
}

spde_status spde_cancel(spde_ctx* ctx, int64_t request) {
    if (!ctx) return fail(SPDE_EINVAL, "null context");
    Server* srv = ctx->srv;
    if (!srv) return fail(SPDE_EINVAL, "unknown request %lld", (long long)request);
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->reqs.find(request);
    if (it == srv->reqs.end()) return fail(SPDE_EINVAL, "unknown request %lld", (long long)request);
    it->second->cancelled = true;
    server_dispatch(srv);  // drops it if it still waits for a lane
    for (auto& kv : srv->lanes) kv.second->cv.notify_one();
    return SPDE_OK;
}

spde_status spde_sample_coupled(spde_ctx* ctx, int fine_level, int coarse_level, int nsamples, double kappa,
                                double sigma, uint64_t seed, uint64_t first_sample, int out_kind, void* out_fine,
                                void* out_coarse, void* stream) {
    STATUS_TRY(check_level(ctx, fine_level));
    STATUS_TRY(check_level(ctx, coarse_level));
    STATUS_TRY(check_params(kappa, sigma));
    if (nsamples < 0) return fail(SPDE_EINVAL, "nsamples < 0");
    const int kind = out_kind & 15;
    if (kind > SPDE_OUT_GRID_GAUSSIAN || (out_kind & ~(15 | SPDE_OUT_F64))) return fail(SPDE_EINVAL, "bad out_kind");
    if (nsamples == 0) return SPDE_OK;
    if (!out_fine || !out_coarse) return fail(SPDE_EINVAL, "null output");
    if (is_host_pointer(out_fine) || is_host_pointer(out_coarse)) return fail(SPDE_EINVAL, "device outputs only");
    std::lock_guard<std::mutex> g(ctx->mu);
    CUDA_TRY(cudaSetDevice(ctx->opts.device));
    Level& F = ctx->lev[fine_level];
    Level& C = ctx->lev[coarse_level];
    if (F.g.nx != 2 * C.g.nx || F.g.ny != 2 * C.g.ny || F.g.nz != 2 * C.g.nz || std::fabs(F.h * 2 - C.h) > 1e-12 * C.h)
        return fail(SPDE_EINVAL, "coarse grid must be the fine grid coarsened once (half the cells per axis, same box)");
    for (int a = 0; a < 3; ++a)
        if (std::fabs(F.lo[a] - C.lo[a]) > 1e-12 * C.h) return fail(SPDE_EINVAL, "levels must share the box");
    if (kind != SPDE_OUT_GRID_GAUSSIAN && (!F.mesh.rowptr || !C.mesh.rowptr))
        return fail(SPDE_EINVAL, "both levels need a mesh for tet outputs");
    ProfScope ps(ctx->prof);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool plain = ctx->opts.precision == SPDE_PREC_FP64;
    const bool graph = graph_path(ctx);
    const size_t esz = (out_kind & SPDE_OUT_F64) ? 8 : 4;
    if (graph) {
        STATUS_TRY(async_call_begin(ctx, st));
    } else {
        ctx->stats.outer_iters = 0;
        ctx->stats.inner_iters = 0;
        ctx->stats.max_rel_residual = 0.0;
    }
    int cap = 1;
    if (!plain) {
        const int64_t per = workspace_bytes(F.g, 1, false) + workspace_bytes(C.g, 1, false);
        size_t freeb = 0, totb = 0;
        if (!(F.ws.g == F.g) || F.ws.S < nsamples || !(C.ws.g == C.g) || C.ws.S < nsamples || F.ws.inner64 != 0 ||
            C.ws.inner64 != 0) {
            F.ws.release();
            C.ws.release();
            if (cudaMemGetInfo(&freeb, &totb) != cudaSuccess) cudaGetLastError();
            cap = std::max(1, std::min(nsamples, (int)((0.85 * (double)freeb) / (double)std::max<int64_t>(per, 1))));
        } else {
            cap = nsamples;
        }
    }
    const int64_t nf3 = F.g.cells(), nc3 = C.g.cells();
    spde_status worst = SPDE_OK;
    for (int s0 = 0; s0 < nsamples; s0 += cap) {
        const int S = std::min(cap, nsamples - s0);
        STATUS_TRY(ensure_workspace(F.ws, F.g, plain ? 1 : std::min(cap, nsamples), plain));
        STATUS_TRY(ensure_workspace(C.ws, C.g, plain ? 1 : std::min(cap, nsamples), plain));
        F.ws.o = level_opts(ctx->opts, F);
        C.ws.o = level_opts(ctx->opts, C);
        if (graph) {
            CUDA_TRY(cudaStreamWaitEvent(st, F.ws.done, 0));
            CUDA_TRY(cudaStreamWaitEvent(st, C.ws.done, 0));
        }
        // fine noise, then its restriction (Sec. 6.2: the same xi drives both levels)
        CUDA_TRY(launch_noise(nf3, S, seed, first_sample + (uint64_t)s0, -g_half(kappa, sigma) * F.h, F.ws.F, nf3, st));
        CUDA_TRY(launch_restrict_rhs(C.g, S, F.ws.F, nf3, C.ws.F, nc3, st));
        double rel = 0.0;
        int outer = 0, inner = 0;
        const double khc = (kappa * C.h) * (kappa * C.h), khf = (kappa * F.h) * (kappa * F.h);
        if (graph) {
            if (plain) STATUS_TRY(refine_solve_async<double>(ctx, C.g, khc, S, C.ws, st, false, nullptr, false));
            else STATUS_TRY(refine_solve_async<float>(ctx, C.g, khc, S, C.ws, st, false, nullptr, false));
            CUDA_TRY(launch_inject_theta(C.g, S, C.ws.x64, 4 * nc3, F.ws.x64, 4 * nf3, st));
            if (plain) STATUS_TRY(refine_solve_async<double>(ctx, F.g, khf, S, F.ws, st, true));
            else STATUS_TRY(refine_solve_async<float>(ctx, F.g, khf, S, F.ws, st, true));
            const size_t perf = out_elem_count(F, 1, out_kind), perc = out_elem_count(C, 1, out_kind);
            STATUS_TRY(write_output(F, S, out_kind, static_cast<char*>(out_fine) + (size_t)s0 * perf * esz, st));
            STATUS_TRY(write_output(C, S, out_kind, static_cast<char*>(out_coarse) + (size_t)s0 * perc * esz, st));
            CUDA_TRY(cudaEventRecord(F.ws.done, st));
            CUDA_TRY(cudaEventRecord(C.ws.done, st));
            continue;
        }
        spde_status sc = plain ? refine_solve<double>(ctx, C.g, khc, S, C.ws, &rel, &outer, &inner, st)
                               : refine_solve<float>(ctx, C.g, khc, S, C.ws, &rel, &outer, &inner, st);
        if (sc != SPDE_OK && sc != SPDE_ENOCONV) return sc;
        if (sc == SPDE_ENOCONV) worst = sc;
        ctx->stats.max_rel_residual = std::max(ctx->stats.max_rel_residual, rel);
        // fine solve started from the coarse field (Sec. 6.2, coarse solution as initial guess)
        CUDA_TRY(launch_inject_theta(C.g, S, C.ws.x64, 4 * nc3, F.ws.x64, 4 * nf3, st));
        spde_status sf = plain ? refine_solve<double>(ctx, F.g, khf, S, F.ws, &rel, &outer, &inner, st, true)
                               : refine_solve<float>(ctx, F.g, khf, S, F.ws, &rel, &outer, &inner, st, true);
        if (sf != SPDE_OK && sf != SPDE_ENOCONV) return sf;
        if (sf == SPDE_ENOCONV) worst = sf;
        ctx->stats.outer_iters = std::max(ctx->stats.outer_iters, outer);
        ctx->stats.inner_iters = std::max(ctx->stats.inner_iters, inner);
        ctx->stats.max_rel_residual = std::max(ctx->stats.max_rel_residual, rel);
        const size_t perf = out_elem_count(F, 1, out_kind), perc = out_elem_count(C, 1, out_kind);
        STATUS_TRY(write_output(F, S, out_kind, static_cast<char*>(out_fine) + (size_t)s0 * perf * esz, st));
        STATUS_TRY(write_output(C, S, out_kind, static_cast<char*>(out_coarse) + (size_t)s0 * perc * esz, st));
    }
    if (graph) return SPDE_OK;  // asynchronous: the outcome comes with spde_wait
    CUDA_TRY(cudaStreamSynchronize(st));
    ctx->prof.flush();
    if (worst != SPDE_OK) return fail(worst, "tolerance not reached: %.3e", ctx->stats.max_rel_residual);
    return SPDE_OK;
}

spde_status spde_query_footprint(spde_ctx* ctx, int level, int nsamples, int64_t* bytes) {
    STATUS_TRY(check_level(ctx, level));
    if (!bytes || nsamples < 0) return fail(SPDE_EINVAL, "bad argument");
    const Level& L = ctx->lev[level];
    const bool plain = ctx->opts.precision == SPDE_PREC_FP64;
    *bytes = workspace_bytes(L.g, plain ? 1 : nsamples, plain);
    return SPDE_OK;
}

spde_status spde_get_stats(spde_ctx* ctx, spde_stats* stats) {
    if (!ctx || !stats) return fail(SPDE_EINVAL, "null argument");
    std::lock_guard<std::mutex> g(ctx->mu);
    CUDA_TRY(cudaSetDevice(ctx->opts.device));
    STATUS_TRY(drain_calls(ctx, false));
    *stats = ctx->stats;
    return SPDE_OK;
}

namespace {
spde_status check_tuning(const spde_tuning& t) {
    if (!(t.omega > 0.0 && t.omega < 1.0) || !(t.inner_tol > 0.0 && t.inner_tol < 1.0) || !(t.flux_diag > 0.0) ||
        (t.sweep_planes != 0 && t.sweep_planes != 8 && t.sweep_planes != 16 && t.sweep_planes != 32 &&
         t.sweep_planes != 64))
        return fail(SPDE_EINVAL, "bad tuning (omega, inner_tol in (0, 1), flux_diag > 0, sweep_planes 0/8/16/32/64)");
    return SPDE_OK;
}

// put `t` (or nothing) on the level: later solves capture new graphs
spde_status set_tuning_locked(spde_ctx* ctx, Level& L, const spde_tuning* t) {
    L.ws.quiesce();
    L.ws.drop_graphs();
    L.tuned = t != nullptr;
    if (t) L.tune = *t;
    return SPDE_OK;
}
}  // namespace

spde_status spde_level_set_tuning(spde_ctx* ctx, int level, const spde_tuning* tuning) {
    STATUS_TRY(check_level(ctx, level));
    if (tuning) STATUS_TRY(check_tuning(*tuning));
    std::lock_guard<std::mutex> g(ctx->mu);
    if (serving_busy(ctx)) return fail(SPDE_EBUSY, "requests are in flight; the schedule cannot change");
    CUDA_TRY(cudaSetDevice(ctx->opts.device));
    return set_tuning_locked(ctx, ctx->lev[level], tuning);
}

spde_status spde_autotune(spde_ctx* ctx, int level, int nsamples, double kappa, double sigma, spde_tuning* best) {
    STATUS_TRY(check_level(ctx, level));
    STATUS_TRY(check_params(kappa, sigma));
    if (!best || nsamples < 1) return fail(SPDE_EINVAL, "bad argument");
    if (serving_busy(ctx)) return fail(SPDE_EBUSY, "requests are in flight");
    Level& L = ctx->lev[level];
    CUDA_TRY(cudaSetDevice(ctx->opts.device));
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        STATUS_TRY(drain_calls(ctx, true));
    }
    void* out = nullptr;
    CUDA_TRY(cudaMalloc(&out, (size_t)nsamples * (size_t)L.g.cells() * sizeof(float)));
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        cudaFree(out);
        if (st) cudaStreamDestroy(st);
        return fail(SPDE_ECUDA, "autotune set-up failed: %s", cudaGetErrorString(ce));
    }
    const bool had = L.tuned;
    const spde_tuning old = L.tune;
    uint64_t first = 0;
    // device time of one call with schedule t (infinite when it fails or misses the tolerance)
    auto measure = [&](const spde_tuning& t, double* ms) -> spde_status {
        {
            std::lock_guard<std::mutex> g(ctx->mu);
            STATUS_TRY(set_tuning_locked(ctx, L, &t));
        }
        *ms = INFINITY;
        for (int rep = 0; rep < 2; ++rep) {  // warm-up (graph capture), then the timed call
            CUDA_TRY(cudaEventRecord(e0, st));
            spde_status s = sample_impl(ctx, level, nsamples, kappa, sigma, false, 0x5eedULL, first,
                                        SPDE_OUT_GRID_GAUSSIAN, out, st);
            first += (uint64_t)nsamples;
            CUDA_TRY(cudaEventRecord(e1, st));
            CUDA_TRY(cudaEventSynchronize(e1));
            if (s == SPDE_OK) s = spde_wait(ctx);
            if (s == SPDE_ENOCONV || s == SPDE_ETIMEOUT) return SPDE_OK;  // not a usable schedule
            STATUS_TRY(s);
        }
        float f = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&f, e0, e1));
        *ms = f;
        return SPDE_OK;
    };
    const spde_opts base = level_opts(ctx->opts, L);
    spde_tuning cur{};
    cur.omega = base.omega;
    cur.inner_tol = base.inner_tol;
    cur.flux_diag = base.flux_diag;
    cur.sweep_planes = base.sweep_planes;
    double cur_ms = INFINITY;
    int evaluated = 0;
    spde_status s = measure(cur, &cur_ms);
    ++evaluated;
    const double default_ms = cur_ms;
    const double omegas[] = {0.7, 0.8, 0.9};
    const double itols[] = {1e-4, 1e-5, 1e-6};
    const double fds[] = {1.25, 1.5, 2.0};
    const int planes[] = {0, 8, 16, 32, 64};
    for (int pass = 0; pass < 2 && s == SPDE_OK; ++pass) {
        for (int knob = 0; knob < 4 && s == SPDE_OK; ++knob) {
            const int nc = knob == 3 ? 5 : 3;
            for (int c = 0; c < nc && s == SPDE_OK; ++c) {
                spde_tuning t = cur;
                if (knob == 0) t.omega = omegas[c];
                else if (knob == 1) t.inner_tol = itols[c];
                else if (knob == 2) t.flux_diag = fds[c];
                else t.sweep_planes = planes[c];
                if (t.omega == cur.omega && t.inner_tol == cur.inner_tol && t.flux_diag == cur.flux_diag &&
                    t.sweep_planes == cur.sweep_planes)
                    continue;
                double ms = INFINITY;
                s = measure(t, &ms);
                ++evaluated;
                if (s == SPDE_OK && ms < 0.99 * cur_ms) {
                    cur = t;
                    cur_ms = ms;
                }
            }
        }
    }
    cudaFree(out);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        if (s != SPDE_OK || !std::isfinite(cur_ms)) {
            set_tuning_locked(ctx, L, had ? &old : nullptr);
            if (s != SPDE_OK) return s;
            return fail(SPDE_ENOCONV, "no schedule reached the tolerance");
        }
        cur.ms_per_call = cur_ms;
        cur.default_ms = default_ms;
        cur.evaluated = evaluated;
        set_tuning_locked(ctx, L, &cur);
    }
    *best = cur;
    return SPDE_OK;
}

spde_status spde_wait(spde_ctx* ctx) {
    if (!ctx) return fail(SPDE_EINVAL, "null context");
    std::lock_guard<std::mutex> g(ctx->mu);
    CUDA_TRY(cudaSetDevice(ctx->opts.device));
    return drain_calls(ctx, true);
}

spde_status spde_mesh_info(spde_ctx* ctx, int level, int64_t* ntets, int64_t* nnz) {
    STATUS_TRY(check_level(ctx, level));
    const Mesh& m = ctx->lev[level].mesh;
    if (ntets) *ntets = m.ntets;
    if (nnz) *nnz = m.nnz;
    return SPDE_OK;
}

spde_status spde_mesh_copy_csr(spde_ctx* ctx, int level, int64_t* row_ptr, int32_t* col, double* gval, double* vol) {
    STATUS_TRY(check_level(ctx, level));
    std::lock_guard<std::mutex> g(ctx->mu);
    CUDA_TRY(cudaSetDevice(ctx->opts.device));
    const Mesh& m = ctx->lev[level].mesh;
    if (!m.rowptr) return fail(SPDE_EINVAL, "no mesh attached to level %d", level);
    if (row_ptr) CUDA_TRY(cudaMemcpy(row_ptr, m.rowptr, (m.ntets + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    if (col) CUDA_TRY(cudaMemcpy(col, m.col, m.nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (gval) CUDA_TRY(cudaMemcpy(gval, m.g, m.nnz * sizeof(double), cudaMemcpyDeviceToHost));
    if (vol) CUDA_TRY(cudaMemcpy(vol, m.vol, m.ntets * sizeof(double), cudaMemcpyDeviceToHost));
    return SPDE_OK;
}

spde_status spde_profile_enable(spde_ctx* ctx, int enable) {
    if (!ctx) return fail(SPDE_EINVAL, "null context");
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->prof.reset();
    ctx->prof.on = enable != 0;
    return SPDE_OK;
}

spde_status spde_profile_read(spde_ctx* ctx, int k, const char** name, int64_t* launches, double* ms, double* bytes) {
    if (!ctx) return fail(SPDE_EINVAL, "null context");
    if (k < 0 || k >= PK_NCLASS) return fail(SPDE_EINVAL, "kernel class out of range");
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->prof.flush();
    if (name) *name = kProfNames[k];
    if (launches) *launches = ctx->prof.launches[k];
    if (ms) *ms = ctx->prof.ms[k];
    if (bytes) *bytes = ctx->prof.bytes[k];
    return SPDE_OK;
}

const char* spde_last_error(void) { return g_err.c_str(); }

spde_status spde_destroy(spde_ctx* ctx) {
    if (!ctx) return SPDE_OK;
    if (ctx->srv) {
        server_stop(ctx->srv);
        delete ctx->srv;
        ctx->srv = nullptr;
    }
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        cudaSetDevice(ctx->opts.device);
        for (auto& L : ctx->lev) {
            L.ws.release();
            L.mesh.release();
            L.fields.release();
        }
        if (ctx->out_tmp) cudaFree(ctx->out_tmp);
        for (auto& c : ctx->cap)
            if (c) cudaStreamDestroy(c);
        dev_free(ctx->d_acc);
        if (ctx->h_acc) cudaFreeHost(ctx->h_acc);
    }
    delete ctx;
    return SPDE_OK;
}

// ---------------------------------------------------------------------------
// step-level entry points
// ---------------------------------------------------------------------------
spde_status spde_noise(int64_t ncells, int nsamples, uint64_t seed, uint64_t first_sample, double scale, double* out,
                       void* stream) {
    if (ncells < 0 || nsamples < 0) return fail(SPDE_EINVAL, "negative size");
    if (nsamples > 65535) return fail(SPDE_EINVAL, "at most 65535 samples per call");
    if (ncells == 0 || nsamples == 0) return SPDE_OK;
    if (!out) return fail(SPDE_EINVAL, "null output");
    CUDA_TRY(launch_noise(ncells, nsamples, seed, first_sample, scale, out, ncells, static_cast<cudaStream_t>(stream)));
    return SPDE_OK;
}

spde_status spde_noise_words(int64_t npairs, uint64_t seed, uint64_t sample, uint32_t* out, void* stream) {
    if (npairs < 0) return fail(SPDE_EINVAL, "negative size");
    if (npairs == 0) return SPDE_OK;
    if (!out) return fail(SPDE_EINVAL, "null output");
    CUDA_TRY(launch_noise_words(npairs, seed, sample, out, static_cast<cudaStream_t>(stream)));
    return SPDE_OK;
}

namespace {
bool grid_dims_ok(const int n[3]) {
    if (!n) return false;
    for (int a = 0; a < 3; ++a)
        if (!is_pow2(n[a]) || n[a] < 4 || n[a] > 1024) return false;
    return (int64_t)n[0] * n[1] * n[2] <= kMaxGridCells;
}
}  // namespace

spde_status spde_apply(int n, double h, double kappa, int nsamples, int prec, const void* x, void* y, void* stream) {
    const int nn[3] = {n, n, n};
    return spde_apply_box(nn, h, kappa, nsamples, prec, x, y, stream);
}

spde_status spde_apply_box(const int n[3], double h, double kappa, int nsamples, int prec, const void* x, void* y,
                           void* stream) {
    if (!grid_dims_ok(n) || nsamples < 0 || !(h > 0.0) || !std::isfinite(kappa) || kappa < 0.0)
        return fail(SPDE_EINVAL, "bad size or parameters");
    const Grid3 gr = make_grid(n[0], n[1], n[2]);
    if (nsamples > 65535) return fail(SPDE_EINVAL, "at most 65535 samples per call");
    if (nsamples == 0) return SPDE_OK;
    if (!x || !y) return fail(SPDE_EINVAL, "null buffer");
    const double kh2 = (kappa * h) * (kappa * h);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (prec == SPDE_PREC_FP64)
        CUDA_TRY(launch_apply<double>(gr, kh2, nsamples, static_cast<const double*>(x), static_cast<double*>(y), st));
    else if (prec == SPDE_PREC_MIXED)
        CUDA_TRY(launch_apply<float>(gr, kh2, nsamples, static_cast<const float*>(x), static_cast<float*>(y), st));
    else
        return fail(SPDE_EINVAL, "bad precision");
    return SPDE_OK;
}

namespace {
struct PrecondScratch {
    Grid3 g;
    int S = 0, prec = -1;
    void* mg = nullptr;
    double* part = nullptr;
};
std::mutex g_pc_mu;
PrecondScratch g_pc;
int* g_pc_fault = nullptr;  // fault word of the step-level preconditioner calls (kept until exit)
}  // namespace

spde_status spde_precond(int n, double h, double kappa, int nsamples, int prec, const spde_opts* opts, const void* r,
                         void* z, void* stream) {
    const int nn[3] = {n, n, n};
    return spde_precond_box(nn, h, kappa, nsamples, prec, opts, r, z, stream);
}

spde_status spde_precond_box(const int n[3], double h, double kappa, int nsamples, int prec, const spde_opts* opts,
                             const void* r, void* z, void* stream) {
    if (!grid_dims_ok(n) || nsamples < 0 || !(h > 0.0) || !(kappa > 0.0) || !std::isfinite(kappa))
        return fail(SPDE_EINVAL, "bad size or parameters");
    const Grid3 gr = make_grid(n[0], n[1], n[2]);
    if (!mg_grid_supported(gr)) return fail(SPDE_EINVAL, "grid shape not supported by the V-cycle");
    if (nsamples > 65535) return fail(SPDE_EINVAL, "at most 65535 samples per call");
    if (prec != SPDE_PREC_FP64 && prec != SPDE_PREC_MIXED) return fail(SPDE_EINVAL, "bad precision");
    if (nsamples == 0) return SPDE_OK;
    if (!r || !z) return fail(SPDE_EINVAL, "null buffer");
    spde_opts o;
    spde_opts_init(&o);
    if (opts) o = *opts;
    std::lock_guard<std::mutex> g(g_pc_mu);
    if (!(g_pc.g == gr) || g_pc.S < nsamples || g_pc.prec != prec) {
        if (g_pc.mg) cudaFree(g_pc.mg);
        dev_free(g_pc.part);
        g_pc = PrecondScratch();
        const size_t b = prec == SPDE_PREC_FP64 ? mg_scratch_elems<double>(gr, nsamples) * 8
                                                 : mg_scratch_elems<float>(gr, nsamples) * 4;
        if (b) CUDA_TRY(cudaMalloc(&g_pc.mg, b));
        STATUS_TRY(dev_alloc(&g_pc.part, (size_t)nsamples * kMaxPartials));
        g_pc.g = gr;
        g_pc.S = nsamples;
        g_pc.prec = prec;
    }
    if (!g_pc_fault) STATUS_TRY(dev_alloc(&g_pc_fault, 1));
    const double kh2 = (kappa * h) * (kappa * h);
    const int64_t n3 = gr.cells(), N4 = 4 * n3;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // each call starts with a clear fault word: a timeout is reported once, by
    // spde_precond_status, and does not make later calls skip their sweeps
    CUDA_TRY(mg_fault_clear(g_pc_fault, st));
    MGPlan plan;
    mg_plan_init(plan, gr, kh2, o.schur_c, o.omega);
    plan.fault = g_pc_fault;
    plan.sz_pref = o.sweep_planes;
    plan.coarse_fp16 = o.coarse_fp16 != 0;
    plan.sweep_rows = o.sweep_rows != 0;
    if (prec == SPDE_PREC_FP64) {
        mg_plan_bind<double>(plan, nsamples, static_cast<double*>(g_pc.mg));
        const double* rr = static_cast<const double*>(r);
        double* zz = static_cast<double*>(z);
        launch_precond_u<double>(N4, (int)n3, nsamples, rr, zz, o.flux_diag, nullptr, nullptr, st);
        if (launch_vcycle<double>(plan, nsamples, rr + 3 * n3, N4, zz + 3 * n3, N4, nullptr, nullptr, 0, st) < 0)
            return fail(SPDE_ECUDA, "V-cycle launch configuration failed");
    } else {
        mg_plan_bind<float>(plan, nsamples, static_cast<float*>(g_pc.mg));
        const float* rr = static_cast<const float*>(r);
        float* zz = static_cast<float*>(z);
        launch_precond_u<float>(N4, (int)n3, nsamples, rr, zz, o.flux_diag, nullptr, nullptr, st);
        if (launch_vcycle<float>(plan, nsamples, rr + 3 * n3, N4, zz + 3 * n3, N4, nullptr, nullptr, 0, st) < 0)
            return fail(SPDE_ECUDA, "V-cycle launch configuration failed");
    }
    CUDA_TRY(cudaGetLastError());
    return SPDE_OK;
}

spde_status spde_precond_status(void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int a = 0, b = 0;
    {
        std::lock_guard<std::mutex> g(g_pc_mu);
        if (g_pc_fault) {
            CUDA_TRY(mg_fault_read(g_pc_fault, &a, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            if (a) CUDA_TRY(mg_fault_clear(g_pc_fault, st));
        }
    }
    CUDA_TRY(noalloc_take_fault(&b, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (a || b)
        return fail(SPDE_ETIMEOUT, "a V-cycle sweep of the last %s call gave up waiting for a plane copy; the field "
                    "block of its z is unspecified", a ? "spde_precond / spde_precond_box" : "spde_precond_noalloc");
    return SPDE_OK;
}

spde_status spde_check_wait_limit(int device, double* waited_ms) {
    if (!waited_ms) return fail(SPDE_EINVAL, "null argument");
    *waited_ms = 0.0;
    CUDA_TRY(cudaSetDevice(device));
    // the probe raises a fault word of its own: solves running meanwhile on other
    // streams or contexts keep theirs clear
    unsigned long long* d = nullptr;
    CUDA_TRY(cudaMalloc(&d, 2 * sizeof(unsigned long long)));
    int* dfault = reinterpret_cast<int*>(d + 1);
    unsigned long long ns = 0;
    int fault = 0;
    cudaStream_t st = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = mg_fault_clear(dfault, st);
    if (e == cudaSuccess) e = mg_wait_probe(d, dfault, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ns, d, sizeof(ns), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = mg_fault_read(dfault, &fault, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (st) cudaStreamDestroy(st);
    cudaFree(d);
    CUDA_TRY(e);
    *waited_ms = 1e-6 * (double)ns;
    if (!fault) return fail(SPDE_ECUDA, "the probe's wait did not give up (fault word not raised)");
    return SPDE_OK;
}

spde_status spde_schur_apply(int n, double h, double kappa, int nsamples, int prec, const void* x, void* y,
                             void* stream) {
    if (!is_pow2(n) || n < 4 || n > 1024 || nsamples < 0 || !(h > 0.0) || !std::isfinite(kappa) || kappa < 0.0)
        return fail(SPDE_EINVAL, "bad size or parameters");
    if (nsamples > 65535) return fail(SPDE_EINVAL, "at most 65535 samples per call");
    if (prec != SPDE_PREC_FP64 && prec != SPDE_PREC_MIXED) return fail(SPDE_EINVAL, "bad precision");
    if (nsamples == 0) return SPDE_OK;
    if (!x || !y) return fail(SPDE_EINVAL, "null buffer");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const double kh2 = (kappa * h) * (kappa * h);
    std::vector<double> tri(2 * (size_t)n - 2);
    double cprev = 0.0;
    for (int f = 0; f < n - 1; ++f) {
        const double piv = 2.0 / 3.0 - (f ? cprev / 6.0 : 0.0);
        tri[f] = (1.0 / 6.0) / piv;
        tri[(n - 1) + f] = 1.0 / piv;
        cprev = tri[f];
    }
    void* dtri = nullptr;
    void* scratch = nullptr;
    const size_t esz = prec == SPDE_PREC_FP64 ? 8 : 4;
    const size_t tb = tri.size() * esz;
    CUDA_TRY(cudaMalloc(&dtri, tb));
    if (cudaMalloc(&scratch, (size_t)nsamples * n * n * n * esz) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(dtri);
        return fail(SPDE_ENOMEM, "scratch allocation failed");
    }
    cudaError_t e;
    int nb;
    if (prec == SPDE_PREC_FP64) {
        e = cudaMemcpy(dtri, tri.data(), tb, cudaMemcpyHostToDevice);
        nb = launch_schur_apply<double>(n, kh2, nsamples, static_cast<const double*>(x), static_cast<double*>(y),
                                        static_cast<const double*>(dtri), static_cast<double*>(scratch), nullptr,
                                        nullptr, st);
    } else {
        std::vector<float> t32(tri.begin(), tri.end());
        e = cudaMemcpy(dtri, t32.data(), tb, cudaMemcpyHostToDevice);
        nb = launch_schur_apply<float>(n, kh2, nsamples, static_cast<const float*>(x), static_cast<float*>(y),
                                       static_cast<const float*>(dtri), static_cast<float*>(scratch), nullptr,
                                       nullptr, st);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dtri);
    cudaFree(scratch);
    CUDA_TRY(e);
    if (nb < 0) return fail(SPDE_ECUDA, "launch configuration failed");
    return SPDE_OK;
}

spde_status spde_solve(spde_ctx* ctx, int level, int nsamples, double kappa, const double* rhs, double* x,
                       void* stream) {
    STATUS_TRY(check_level(ctx, level));
    STATUS_TRY(check_params(kappa, 1.0));
    if (nsamples < 0) return fail(SPDE_EINVAL, "nsamples < 0");
    if (nsamples == 0) return SPDE_OK;
    if (!rhs || !x) return fail(SPDE_EINVAL, "null buffer");
    std::lock_guard<std::mutex> g(ctx->mu);
    CUDA_TRY(cudaSetDevice(ctx->opts.device));
    Level& L = ctx->lev[level];
    L.ws.quiesce();  // an asynchronous call may still use the workspace
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool plain = ctx->opts.precision == SPDE_PREC_FP64;
    const Grid3 gr = L.g;
    const int64_t n3 = gr.cells(), N4 = 4 * n3;
    const double kh2 = (kappa * L.h) * (kappa * L.h);
    int cap = 1;
    if (!plain) {
        if (L.ws.g == gr && L.ws.S >= nsamples && L.ws.inner64 == 0) cap = nsamples;
        else {
            L.ws.release();
            cap = batch_capacity(gr, nsamples, false);
        }
    }
    ctx->stats.outer_iters = 0;
    ctx->stats.inner_iters = 0;
    ctx->stats.max_rel_residual = 0.0;
    spde_status worst = SPDE_OK;
    for (int s0 = 0; s0 < nsamples; s0 += cap) {
        const int S = std::min(cap, nsamples - s0);
        STATUS_TRY(ensure_workspace(L.ws, gr, plain ? 1 : std::min(cap, nsamples), plain));
        L.ws.o = level_opts(ctx->opts, L);
        CUDA_TRY(cudaMemcpyAsync(L.ws.F, rhs + (size_t)s0 * n3, (size_t)S * n3 * sizeof(double),
                                 cudaMemcpyDeviceToDevice, st));
        double rel = 0.0;
        int outer = 0, inner = 0;
        spde_status s = plain ? refine_solve<double>(ctx, gr, kh2, S, L.ws, &rel, &outer, &inner, st)
                              : refine_solve<float>(ctx, gr, kh2, S, L.ws, &rel, &outer, &inner, st);
        if (s != SPDE_OK && s != SPDE_ENOCONV) return s;
        if (s == SPDE_ENOCONV) worst = s;
        ctx->stats.outer_iters = std::max(ctx->stats.outer_iters, outer);
        ctx->stats.inner_iters = std::max(ctx->stats.inner_iters, inner);
        ctx->stats.max_rel_residual = std::max(ctx->stats.max_rel_residual, rel);
        CUDA_TRY(cudaMemcpyAsync(x + (size_t)s0 * N4, L.ws.x64, (size_t)S * N4 * sizeof(double),
                                 cudaMemcpyDeviceToDevice, st));
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    if (worst != SPDE_OK) return fail(worst, "tolerance not reached: %.3e", ctx->stats.max_rel_residual);
    return SPDE_OK;
}

spde_status spde_project(spde_ctx* ctx, int level, int nsamples, const double* theta, int out_kind, void* out,
                         void* stream) {
    STATUS_TRY(check_level(ctx, level));
    const int kind = out_kind & 15;
    if (kind > SPDE_OUT_GAUSSIAN || (out_kind & ~(15 | SPDE_OUT_F64))) return fail(SPDE_EINVAL, "bad out_kind");
    if (nsamples < 0) return fail(SPDE_EINVAL, "nsamples < 0");
    if (nsamples == 0) return SPDE_OK;
    if (!theta || !out) return fail(SPDE_EINVAL, "null buffer");
    std::lock_guard<std::mutex> g(ctx->mu);
    CUDA_TRY(cudaSetDevice(ctx->opts.device));
    Level& L = ctx->lev[level];
    if (!L.mesh.rowptr) return fail(SPDE_EINVAL, "no mesh attached to level %d", level);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n3 = L.g.cells();
    float* tT = nullptr;
    STATUS_TRY(dev_alloc(&tT, (size_t)nsamples * n3));
    cudaError_t e = launch_transpose_theta(n3, nsamples, theta, n3, 1.0, tT, st);
    if (e == cudaSuccess)
        e = launch_project(L.mesh.ntets, nsamples, L.mesh.rowptr, L.mesh.col, L.mesh.pi, tT,
                           kind == SPDE_OUT_LOGNORMAL ? 0 : 1, (out_kind & SPDE_OUT_F64) ? 1 : 0, out, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(tT);
    CUDA_TRY(e);
    return SPDE_OK;
}

}  // extern "C"
