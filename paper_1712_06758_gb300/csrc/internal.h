// Internal host-side declarations: kernel launchers and solver structures.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace spde {

constexpr int kReduceBlock = 256;
constexpr int kMaxPartials = 4096;   // per column, per partial-sum array

// Cells per axis of a uniform embedding grid (equal spacing h on all axes),
// each a power of two; cell (i, j, k) has flat index c = i + nx (j + ny k).
struct Grid3 {
    int nx = 0, ny = 0, nz = 0;
    int lx = 0, ly = 0, lz = 0;  // log2 of each extent
    __host__ __device__ int64_t cells() const { return (int64_t)nx * ny * nz; }
    __host__ __device__ int ext(int axis) const { return axis == 0 ? nx : (axis == 1 ? ny : nz); }
    __host__ __device__ int maxn() const { return nx > ny ? (nx > nz ? nx : nz) : (ny > nz ? ny : nz); }
    __host__ __device__ bool cube() const { return nx == ny && ny == nz; }
    // the next coarser grid of the multigrid hierarchy: every extent above 1 halves
    __host__ __device__ Grid3 coarser() const {
        Grid3 c;
        c.nx = nx > 1 ? nx >> 1 : 1;
        c.ny = ny > 1 ? ny >> 1 : 1;
        c.nz = nz > 1 ? nz >> 1 : 1;
        c.lx = lx > 0 ? lx - 1 : 0;
        c.ly = ly > 0 ? ly - 1 : 0;
        c.lz = lz > 0 ? lz - 1 : 0;
        return c;
    }
    __host__ __device__ bool operator==(const Grid3& o) const { return nx == o.nx && ny == o.ny && nz == o.nz; }
};

inline int log2_exact(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

inline Grid3 make_grid(int nx, int ny, int nz) {
    Grid3 g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.lx = log2_exact(nx);
    g.ly = log2_exact(ny);
    g.lz = log2_exact(nz);
    return g;
}
inline Grid3 make_grid(int n) { return make_grid(n, n, n); }

// Per-column MINRES state (Paige-Saunders recurrences), kept in FP64.
struct MinresCol {
    double beta, oldb, alpha, dbar, epsln, oldeps, phibar, cs, sn, gamma, delta, phi, beta1;
    double tol;      // stop when phibar <= tol * beta1
    double ry;       // r2.yprev of the last pass B: beta times the v.r1 term of the next alpha
    // coefficients of the pending w/x update (saved by the Givens step)
    double d_oldb, d_oldeps, d_delta, d_gamma, d_phi;
    // the per-column factors the vector passes use, computed once by the scalar
    // steps (FP64, and rounded to FP32 for the FP32 passes) so that no thread of
    // a vector pass divides in FP64
    double kd[8];
    float kf[8];
    int active;      // column still iterating
    int upd;         // a w/x update is pending (consumed by the next fused pass or the final D)
    int iters;
    int d_iter;      // iteration number of the pending update
};

// indices of MinresCol::kd / kf
enum {
    KC_IB = 0,    // 1 / beta            (Lanczos pass)
    KC_COEF = 1,  // beta / oldb, 0 in the first iteration
    KC_F = 2,     // alpha / beta        (pass B)
    KC_IV = 3,    // 1 / d_oldb          (w/x update)
    KC_OE = 4,    // d_oldeps
    KC_DE = 5,    // d_delta
    KC_IG = 6,    // 1 / d_gamma
    KC_PH = 7     // d_phi
};

template <typename T>
__host__ __device__ __forceinline__ T col_coef(const MinresCol& c, int k) {
    if constexpr (sizeof(T) == 4) return c.kf[k];
    else return c.kd[k];
}

// Per-column state of the Schur-complement CG (FP64 scalars).
struct CgCol {
    double rz, rr0, alpha, beta, tol2;
    int active;  // column still iterating
    int iters;
    int pad0, pad1;
};

// Device state of one refinement solve driven by a captured graph (no host
// round trip): the control kernels of krylov.cu make the decisions the host
// loop of the synchronous path makes, from the same FP64 numbers.
struct RefineCtl {
    int outer;    // corrections applied so far
    int inner;    // inner-solver loop iterations executed in this solve (all steps)
    int it;       // loop iterations of the current inner solve
    int status;   // 0, 4 (tolerance not reached) or 5 (a sweep timed out) once stopped
    int cnt[6];   // column counters of the Givens / CG steps of one loop body
    double worst; // largest relative residual at the last check
};

// Outcome of the graph-driven solves of the calls since the host last read it
// (solves on different streams update it with atomics; worst_bits holds the bits
// of a non-negative double, whose integer order is its numeric order).
struct CallAcc {
    int outer, inner, status, nsolve;
    unsigned long long worst_bits;
};

// Multigrid plan of one grid size for a batch of S columns.
struct MGPlan {
    Grid3 g[16];        // grids of the levels: g[l + 1] = g[l].coarser(), g[nlev - 1] has one cell
    double ls[16] = {}; // level factors: A_l = ls (kh2 lq I + c L_l); 2^l and 4^l while all axes halve
    double lq[16] = {};
    int nlev = 0;       // levels 0..nlev-1
    int lc = 0;         // first level handled by the one-CTA coarse kernel (<= 4096 cells)
    double kh2 = 0.0;   // (kappa h)^2 on level 0
    double c = 1.0;     // Schur weight
    double omega = 0.8; // Jacobi weight
    double prof_cols = 0.0; // columns assumed active, for the profiler's byte counts (0: all)
    // scratch (element type of the plan) for levels 1..lc: rhs b_l and result e_l,
    // each [S][cells of level l]
    void* b[16] = {};
    void* e[16] = {};
    // per-cell diagonal s (a_c + c k_c) of every level (element type of the plan), for
    // cell-wise kappa; null: one coefficient for the whole level
    const void* D[16] = {};
    // fault word of the solve (device int): a sweep whose bounded wait gives up raises it,
    // and later sweeps of the same solve skip their work until the owner clears it
    int* fault = nullptr;
    // z planes per CTA of the tiled sweeps: 8, 16 or 32 where the level's z extent
    // allows, 0 = chosen per level for occupancy
    int sz_pref = 0;
    // FP16 storage of the levels the one-CTA coarse kernel holds (FP32 path)
    bool coarse_fp16 = false;
    // FP32 sweeps of levels 32, 64 or 128 cells wide (constant kappa or one per column) on
    // whole-row tiles (k_mg_down_rows / k_mg_up_rows); 0: the 32 x 16 tiles everywhere
    bool sweep_rows = true;
    // one kappa per column (serving lanes): kh2col [S] (kappa h)^2 of level 0 (FP64), and
    // per tiled level l a table qtab[l] [S][21] (element type of the plan) of the
    // kappa-dependent sweep coefficients (mg_coef_row); null: plan.kh2 for every column
    const double* kh2col = nullptr;
    const void* qtab[16] = {};
};

// the kappa-dependent sweep coefficients of tiled level l for (kappa h)^2 = kh2 (the
// rest of the plan as given): omega / D(k), omega s c / D(k), (1/omega - 1) D(k), k = 0..6
template <typename T>
void mg_coef_row(const MGPlan& plan, int l, double kh2, T out[21]);

// ---- noise.cu
cudaError_t launch_noise(int64_t ncells, int S, uint64_t seed, uint64_t first, double scale,
                         double* out, int64_t col_stride, cudaStream_t st);

cudaError_t launch_noise_words(int64_t npairs, uint64_t seed, uint64_t sample, uint32_t* out, cudaStream_t st);

cudaError_t launch_noise_cols(int64_t ncells, int S, const uint64_t* seed, const uint64_t* sample, const double* scale,
                              const int* mask, double* out, int64_t col_stride, cudaStream_t st);

// ---- stencil.cu (element type T = float or double)
template <typename T>
cudaError_t launch_apply(const Grid3& g, double kh2, int S, const T* x, T* y, cudaStream_t st);
// r = [0; F] - A x (FP64), written to r32 (float, may be null) and r64 (double, may be
// null); partial sums of r.r per column into part [S][nblk]; returns nblk
// kh2c: (kappa h)^2 per cell (fields), kh2s: per column (serving lanes), else kh2
int launch_residual64(const Grid3& g, double kh2, int S, const double* F, int64_t F_stride, const double* x,
                      float* r32, double* r64, double* part, const int* active, cudaStream_t st,
                      const double* kh2c = nullptr, const double* kh2s = nullptr, int xzero = 0,
                      const int* zgate = nullptr);
// one-time kernel attributes of the flux line solves (done before any stream capture)
cudaError_t flux_prepare();
// the multigrid diagonal of a level with cell-wise (kappa h)^2: a_c = mean of the children's a
// (a_0 = (kappa_c h)^2; gf is the finer grid), D = s (a_c q + c k_c) with k_c the cell's
// existing neighbours and s, q the level's factors (2^l, 4^l on a cube)
cudaError_t launch_restrict_mean(const Grid3& gf, const double* af, double* ac, cudaStream_t st);
cudaError_t launch_level_diag(const Grid3& g, double s, double q, double c, const double* a, double* D64, float* D32,
                              cudaStream_t st);
// F[s][e] *= c[e] (per-cell noise factor of a level with fields)
cudaError_t launch_scale_cells(int64_t n3, int S, double* F, int64_t stride, const double* c, cudaStream_t st);
// (kappa h)^2 (FP64, FP32) and -g h per cell from cell-wise kappa, sigma (device arrays)
cudaError_t launch_field_coefs(int64_t n3, double h, const double* kappa, const double* sigma, double* kh2_64,
                               float* kh2_32, double* gh, cudaStream_t st);
// x += d (double += float) on active columns
cudaError_t launch_add_correction(int64_t nelem, int S, double* x, const float* d, const int* active,
                                  cudaStream_t st);
// u = -T^{-1} D1^T theta into the flux blocks of x ([S][4 cells], FP64), line by line;
// tri: Thomas factors of the longest extent tn (2 tn - 2 doubles, see k_flux_lines);
// gate (device, optional): the kernels do nothing while *gate == 0
cudaError_t launch_flux_from_theta(const Grid3& g, int S, double* x, int64_t col_stride, const double* tri,
                                   cudaStream_t st, const int* gate = nullptr);
// x cell block += d ([S][n^3]) for columns whose inner solve ran
template <typename T>
cudaError_t launch_add_theta(int64_t n3, int S, double* x, const T* d, const MinresCol* st_, cudaStream_t st);
// two-level coupling: F_c = (1/sqrt 2) sum over children of F_f; theta~_f = theta~_c(parent) / sqrt 2
// (gc: the coarse grid; the fine grid is twice it along every axis)
cudaError_t launch_restrict_rhs(const Grid3& gc, int S, const double* Ff, int64_t f_stride, double* Fc,
                                int64_t c_stride, cudaStream_t st);
cudaError_t launch_inject_theta(const Grid3& gc, int S, const double* xc, int64_t c_stride, double* xf,
                                int64_t f_stride, cudaStream_t st);
// partial sums of a.a over columns of a strided array; returns nblk
int launch_sumsq(int64_t nelem, int S, const double* a, int64_t stride, double* part, cudaStream_t st);
// out[s] = sum_b part[s][b] (fixed order)
cudaError_t launch_reduce(int S, const double* part, int nblk, double* out, cudaStream_t st);

// ---- krylov.cu
// A(k+1) fused with the pending D(k) when yprev != null (see krylov.cu): partA gets
// the partial sums of y.(A y).  The preconditioned Lanczos vector is fd * u on the
// flux blocks and y's cell block.
template <typename T>
int launch_minres_A(const Grid3& g, double kh2, int S, const T* y, const T* u, double fd, double* partA,
                    MinresCol* st_, const T* yprev, T* w1, const T* w2, T* xd, cudaStream_t st,
                    const T* kh2c = nullptr, const T* kh2s = nullptr);
// r1 = (A y) / beta - (beta / oldb) r1 - (alpha / beta) r2 in place, with the flux part
// of the next beta^2 in partB (the flux block of the next preconditioned vector is
// fd * r1 and is not stored) and r1.y in partE (the same block count)
template <typename T>
int launch_minres_B(const Grid3& g, double kh2, int S, const T* y, const T* r2, double fd, T* r1, double* partB,
                    double* partE, MinresCol* st_, cudaStream_t st, const T* kh2c = nullptr,
                    const T* kh2s = nullptr);
template <typename T>
int launch_precond_u(int64_t N4, int n3, int S, const T* r, T* y, double fd, double* part,
                     const MinresCol* st_, cudaStream_t st);
cudaError_t launch_alpha(int S, const double* partA, int nA, MinresCol* st_, cudaStream_t st);
// nactive (optional, two ints): [0] += columns still active after this step,
// [1] += columns whose w/x update this step left pending
// max_iter: a column stops after this many iterations (the iteration cap of the solve)
// partE: pass B's partial sums of r1.y (nB blocks), kept for the next alpha
cudaError_t launch_givens(int S, const double* partB, int nB, const double* partC, int nC, const double* partE,
                          MinresCol* st_, int* nactive, cudaStream_t st, int max_iter = 1 << 30);
// control kernels of the graph-driven refinement (one thread block each)
cudaError_t launch_refine_init(RefineCtl* ctl, int* fault, unsigned long long h_outer, cudaStream_t st);
// residual check of every column (colv: [S] |r|^2, then [S] |F|^2): mask, inner tolerances,
// stop decision (-> h_outer), and the step count
cudaError_t launch_refine_check(int S, const double* colv, double tol, double inner_tol, int fp64_inner,
                                int max_outer, const int* fault, int* mask, double* coltol, RefineCtl* ctl,
                                unsigned long long h_outer, cudaStream_t st);
// end of a loop body: iterations += add, continue while columns counted in slot remain and
// the iteration cap is not reached (-> h_loop); clears the counters
cudaError_t launch_loop_ctl(RefineCtl* ctl, int slot, int add, int max_iter, unsigned long long h_loop,
                            cudaStream_t st);
// count_iters = 0: record the solve's residual and status only (the coarse solve of a coupled pair)
cudaError_t launch_refine_finish(const RefineCtl* ctl, CallAcc* acc, int count_iters, cudaStream_t st);
// col_tol (device [S], optional): each column's own stopping tolerance instead of tol
cudaError_t launch_minres_init(int S, const double* partB, int nB, const double* partC, int nC,
                               double tol, MinresCol* st_, int* nactive, cudaStream_t st,
                               const double* col_tol = nullptr);
// cell-block update: w1, w2, x are [S][n^3]; ycur is [S][4 n^3]
template <typename T>
cudaError_t launch_minres_D(int64_t n3, int S, const T* ycur, T* w1, const T* w2, T* x,
                            const MinresCol* st_, cudaStream_t st);
template <typename T>
cudaError_t launch_add_correction_st(int64_t N4, int S, double* x, const T* d, const MinresCol* st_, cudaStream_t st);
cudaError_t launch_set_active(int S, const int* mask, MinresCol* st_, cudaStream_t st);
// column activity flags used by the V-cycle and elementwise kernels
cudaError_t launch_active_flags(int S, const MinresCol* st_, int* flags, cudaStream_t st);

// ---- mg.cu
// the fault word of a solve's V-cycle sweeps (a device int; 1: a wait for a plane copy
// gave up): mg_fault_read enqueues a copy into *host on st (valid once st has
// synchronised), mg_fault_clear enqueues its reset on st
cudaError_t mg_fault_read(const int* fault, int* host, cudaStream_t st);
// launches the bounded-wait self-check (one CTA whose wait must give up and raise *fault);
// its wait time goes to *elapsed_ns_dev
cudaError_t mg_wait_probe(unsigned long long* elapsed_ns_dev, int* fault, cudaStream_t st);
cudaError_t mg_fault_clear(int* fault, cudaStream_t st);
// one-time kernel attributes and driver entry points of the V-cycle (done before any stream capture)
cudaError_t mg_prepare();
template <typename T>
int launch_vcycle(const MGPlan& plan, int S, const T* b, int64_t b_stride, T* y, int64_t y_stride,
                  double* dot_part, const int* active, int act_stride, cudaStream_t st);
template <typename T>
size_t mg_scratch_elems(int n, int S);
template <typename T>
size_t mg_scratch_elems(const Grid3& g, int S);
// false when the hierarchy does not fit the kernels (more than 4096 cells on the
// first level whose extents are not multiples of the 32 x 16 x 8 tile)
bool mg_plan_init(MGPlan& plan, const Grid3& g, double kh2, double c, double omega);
void mg_plan_init(MGPlan& plan, int n, double kh2, double c, double omega);
bool mg_grid_supported(const Grid3& g);
template <typename T>
void mg_plan_bind(MGPlan& plan, int S, T* scratch);

// ---- schur.cu (Schur-complement CG on the cell unknowns)
template <typename T>
int launch_schur_apply(int n, double kh2, int S, const T* x, T* y, const T* tri, T* scratch, double* dot_part,
                       const CgCol* st, cudaStream_t stream);
template <typename T>
int launch_cg_xr(int64_t n3, int S, T* x, T* r, const T* p, const T* q, double* part, const CgCol* st, cudaStream_t s);
template <typename T>
cudaError_t launch_cg_p(int64_t n3, int S, T* p, const T* z, const CgCol* st, cudaStream_t s);
template <typename T>
int launch_cg_rhs(int64_t n3, int S, const T* mixed_r, T* r, double* part, const CgCol* st, cudaStream_t s);
template <typename T>
cudaError_t launch_cg_add(int64_t n3, int S, double* x, const T* d, const CgCol* st, cudaStream_t s);
cudaError_t launch_cg_alpha(int S, const double* part, int nb, CgCol* st, cudaStream_t s);
cudaError_t launch_cg_beta(int S, const double* prr, int nrr, const double* prz, int nrz, CgCol* st, int* nactive,
                           cudaStream_t s, int max_iter = 1 << 30);
cudaError_t launch_cg_init(int S, const double* prz, int nrz, const double* prr, int nrr, double tol, CgCol* st,
                           int* nactive, cudaStream_t s);
cudaError_t launch_cg_set_active(int S, const int* mask, CgCol* st, cudaStream_t s);

// ---- clip.cu
struct ClipResult {
    int64_t nnz;
    int bad_tet;      // first offending tet or -1
    int bad_kind;     // 0 none, 1 degenerate, 2 outside box, 3 row sum mismatch
};
// Build CSR (row_ptr, col, G, Pi) for a mesh already on the device.  Allocates the CSR
// arrays with cudaMalloc (ownership passes to the caller).  Synchronises st.
cudaError_t build_coupling(const int n[3], double h, const double lo[3], int64_t nverts, const double* d_xyz,
                           int64_t ntets, const int32_t* d_tets, double* d_vol, int64_t** d_rowptr,
                           int32_t** d_col, double** d_g, float** d_pi, ClipResult* res,
                           cudaStream_t st);

// ---- project.cu
// theta^T[c][s] = float(scale * x[s][x_off + c]) for s < S (x column stride x_stride)
cudaError_t launch_transpose_theta(int64_t ncell, int S, const double* x, int64_t x_stride, double scale,
                                   float* thetaT, cudaStream_t st);
// out[s][t] = map(sum_j pi[j] thetaT[col[j]][s]); kind 0 exp, 1 identity; f64 output if out64
cudaError_t launch_project(int64_t ntets, int S, const int64_t* rowptr, const int32_t* col,
                           const float* pi, const float* thetaT, int kind, int out64, void* out,
                           cudaStream_t st);
cudaError_t launch_transpose_cols(int64_t ncell, int R, const int* cols, const double* x, int64_t x_stride,
                                  double scale, float* thetaT, cudaStream_t st);
cudaError_t launch_project_ptrs(int64_t ntets, int R, const int64_t* rowptr, const int32_t* col, const float* pi,
                                const float* thetaT, int kind, int out64, void* const* outs, cudaStream_t st);
// number of distinct column indices of a CSR matrix (cells touched by the projection)
cudaError_t count_used_columns(int64_t nnz, const int32_t* col, int64_t ncell, int64_t* used, cudaStream_t st);
// grid output: out[s][c] = scale * x[s][x_off + c]
cudaError_t launch_grid_out(int64_t ncell, int S, const double* x, int64_t x_stride, double scale,
                            int out64, void* out, cudaStream_t st);

// set the message spde_last_error() returns on the calling thread
void set_last_error(const char* msg);

// noalloc.cu: reads and clears the fault word of the allocation-free preconditioner calls
// on the current device (*raised = 1 when one of their sweeps gave up); synchronises st
cudaError_t noalloc_take_fault(int* raised, cudaStream_t st);

}  // namespace spde
