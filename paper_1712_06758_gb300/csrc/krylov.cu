// K4: batched preconditioned MINRES (Paige-Saunders recurrences) for the
// symmetric indefinite mixed system, one column per sample.
//
// Vectors are [S][4 n^3]; per-column scalars live in MinresCol (FP64).  The
// dot products are reduced deterministically: per-block partial sums in a
// fixed-shape tree, then one fixed-order pass per column, so a column's
// result does not depend on which other columns share the batch.
//
// One iteration k (v = y / beta, y = P^{-1} r2, r1 and r2 the last two
// unpreconditioned Lanczos vectors):
//   A: alpha = v.A v - (beta / oldb) v.r1                   (stencil, reads only)
//   B: r1' = A v - (beta / oldb) r1 - (alpha / beta) r2      (stencil again, in place),
//      y' = P^{-1} r1' (flux block here, field block by the V-cycle), beta'^2 = r1'.y'
//   Givens rotation, residual estimate phibar, retirement
//   D: w' = (v - oldeps w1 - delta w2) / gamma, x += phi w'
// The term v.r1 of alpha is y_k.r_{k-1} / beta; P is symmetric, so it equals
// r_k.y_{k-1} / beta, which pass B of the previous iteration forms from the
// vectors it already holds.  A therefore writes nothing: the vector A v is
// rebuilt by B instead of being stored by A and read back (4 + 13 words per
// cell instead of 12 + 12).
#include "device.cuh"
#include "internal.h"

namespace spde {

static inline int elem_blocks(int64_t nelem) {
    int64_t b = (nelem + 1023) / 1024;
    if (b > 2048) b = 2048;
    return (int)(b < 1 ? 1 : b);
}
static inline int cell_blocks(int64_t n3) {
    int64_t b = (n3 + 255) / 256;
    if (b > 2048) b = 2048;
    return (int)(b < 1 ? 1 : b);
}

// A(k+1) fused with D(k): both become ready after the Givens step of
// iteration k and touch disjoint arrays, so one pass streams both.
//   A part (column active):   partA = y.(A y)  (y unscaled; alpha is formed by k_alpha)
//   D part (column upd set):  w' = (yprev_cell / oldb_D - oldeps w1 - delta w2) / gamma,
//                             x += phi w'   (cell block, [S][n^3] arrays)
// The D coefficients were saved by the Givens step in MinresCol (d_* fields)
// because beta / oldb have already advanced for the A part.
__device__ __forceinline__ void set_coef(MinresCol& c, int k, double v) {
    c.kd[k] = v;
    c.kf[k] = (float)v;
}
// y = A v on a quad for a preconditioned Lanczos vector v whose flux blocks
// are fd * u (the flux block of the preconditioner is fd I, so they are never
// stored) and whose cell block is th; fd multiplies each flux sum once.  The
// unscaled flux centre values and the cell centre values come back in vc (the
// caller scales the flux part of its inner product by fd); wall fluxes are
// masked by index.
template <typename T>
__device__ __forceinline__ void apply_quad_fd(const T* __restrict__ us, const T* __restrict__ th, T fd,
                                              const Grid3& g, const QuadPos& p, const V4<T>& kh2, T yu[4], T yv[4],
                                              T yw[4], T yt[4], V4<T> vc[4]) {
    const int n3 = 1 << (g.lx + g.ly + g.lz);
    const int n = g.nx;
    const int sy = g.nx, sz = g.nx << g.ly;
    const T* ux = us;
    const T* uy = us + n3;
    const T* uz = us + 2 * n3;
    const int c = p.c;
    const V4<T> ux4 = ld4(ux + c), uy4 = ld4(uy + c), uz4 = ld4(uz + c), th4 = ld4(th + c);
    const bool jl = p.j > 0, jh = p.j < g.ny - 1, jhh = p.j + 1 < g.ny - 1;
    const bool kl = p.k > 0, kh = p.k < g.nz - 1, khh = p.k + 1 < g.nz - 1;
    const V4<T> uyM = jl ? ld4(uy + c - sy) : zero4<T>();
    const V4<T> uyP = jhh ? ld4(uy + c + sy) : zero4<T>();
    const V4<T> uzM = kl ? ld4(uz + c - sz) : zero4<T>();
    const V4<T> uzP = khh ? ld4(uz + c + sz) : zero4<T>();
    const V4<T> thY = jh ? ld4(th + c + sy) : zero4<T>();
    const V4<T> thZ = kh ? ld4(th + c + sz) : zero4<T>();
    const T uxL = (p.i0 > 0) ? ux[c - 1] : T(0);
    const T uxR = (p.i0 + 4 < n - 1) ? ux[c + 4] : T(0);
    const T thR = (p.i0 + 4 < n) ? th[c + 4] : T(0);
    const T a6 = T(1) / T(6), a23 = T(2) / T(3);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int i = p.i0 + e;
        const T t0 = th4.v[e];
        const T ux0 = (i < n - 1) ? ux4.v[e] : T(0);
        const T uxm = (e > 0) ? ((i - 1 < n - 1) ? ux4.v[e - 1] : T(0)) : uxL;
        const T uxp = (e < 3) ? ((i + 1 < n - 1) ? ux4.v[e + 1] : T(0)) : uxR;
        const T thx = (e < 3) ? th4.v[e + 1] : thR;
        const T uy0 = jh ? uy4.v[e] : T(0);
        const T uz0 = kh ? uz4.v[e] : T(0);
        const T uym = uyM.v[e], uzm = uzM.v[e];
        yu[e] = (i < n - 1) ? fd * (a23 * ux0 + a6 * (uxm + uxp)) + (t0 - thx) : T(0);
        yv[e] = jh ? fd * (a23 * uy0 + a6 * (uym + uyP.v[e])) + (t0 - thY.v[e]) : T(0);
        yw[e] = kh ? fd * (a23 * uz0 + a6 * (uzm + uzP.v[e])) + (t0 - thZ.v[e]) : T(0);
        yt[e] = fd * ((ux0 - uxm) + (uy0 - uym) + (uz0 - uzm)) - kh2.v[e] * t0;
    }
    vc[0] = ux4;
    vc[1] = uy4;
    vc[2] = uz4;
    vc[3] = th4;
}

// The w/x update of one 4-cell vector (the D step), shared by the fused pass
// and the final k_minres_D so that both produce the same bits:
//   w' = (v / oldb - oldeps w1 - delta w2) / gamma,  x' = x + phi w'
template <typename T>
__device__ __forceinline__ void d_update4(const V4<T>& yv, const V4<T>& w1v, const V4<T>& w2v, const V4<T>& xv, T iv,
                                          T oe, T de, T ig, T ph, V4<T>& wn, V4<T>& xn) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        wn.v[k] = (yv.v[k] * iv - oe * w1v.v[k] - de * w2v.v[k]) * ig;
        xn.v[k] = xv.v[k] + ph * wn.v[k];
    }
}

// CUBE: the grid is a cube (all extents and logs taken from x, which keeps the
// index arithmetic and register use of the cubic case minimal)
template <typename T, bool CUBE>
__device__ __forceinline__ Grid3 pass_grid(const Grid3& gin) {
    Grid3 g = gin;
    if constexpr (CUBE) {
        g.ny = g.nz = gin.nx;
        g.lx = g.ly = g.lz = ilog2(gin.nx);
    }
    return g;
}

// (kappa h)^2 of a quad: one value (per call or per column), or the level's field
template <typename T>
__device__ __forceinline__ V4<T> quad_kh2(T kh2, const T* __restrict__ kh2c, const T* __restrict__ kh2s, int s, int c) {
    V4<T> k4;
    if (kh2c) k4 = ld4(kh2c + c);
    else
#pragma unroll
        for (int e = 0; e < 4; ++e) k4.v[e] = kh2s ? kh2s[s] : kh2;
    return k4;
}

// FP32: four CTAs per SM (64 registers, a 28-byte spill) measured 6 % faster than
// three without spills.
template <typename T, bool CUBE>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_minres_A(Grid3 gin, T kh2, const T* __restrict__ y, const T* __restrict__ u, T fd,
                                                     double* __restrict__ partA, const MinresCol* __restrict__ st,
                                                     const T* __restrict__ yprev, T* __restrict__ w1,
                                                     const T* __restrict__ w2, T* __restrict__ xd,
                                                     const T* __restrict__ kh2c, const T* __restrict__ kh2s) {
    __shared__ double red[8];
    const int s = blockIdx.y;
    const MinresCol& cs = st[s];
    const bool doA = cs.active != 0;
    const bool doD = yprev != nullptr && cs.upd != 0;
    if (!doA && !doD) return;
    const Grid3 g = pass_grid<T, CUBE>(gin);
    const int n3 = 1 << (g.lx + g.ly + g.lz);
    const int nq = n3 >> 2;
    const int64_t off = (int64_t)s * 4 * n3;
    const T* ys = y + off;   // only its cell block is read
    const T* us = u + off;   // flux blocks of the Lanczos vector: y's are fd times these
    T acc = T(0);
    if (doA) {
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
            const QuadPos p = quad_pos(q, g);
            T yu[4], yv[4], yw[4], yt[4];
            V4<T> vc[4];
            apply_quad_fd<T>(us, ys + 3 * n3, fd, g, p, quad_kh2<T>(kh2, kh2c, kh2s, s, p.c), yu, yv, yw, yt, vc);
#pragma unroll
            for (int e = 0; e < 4; ++e)
                acc += fd * (vc[0].v[e] * yu[e] + vc[1].v[e] * yv[e] + vc[2].v[e] * yw[e]) + vc[3].v[e] * yt[e];
        }
    }
    if (doD) {
        const T iv = col_coef<T>(cs, KC_IV), oe = col_coef<T>(cs, KC_OE), de = col_coef<T>(cs, KC_DE);
        const T ig = col_coef<T>(cs, KC_IG), ph = col_coef<T>(cs, KC_PH);
        const int it = cs.d_iter;
        const T* yc = yprev + off + 3 * (int64_t)n3;
        const int64_t o3 = (int64_t)s * n3;
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
            const int64_t e0 = 4 * (int64_t)q;
            const V4<T> yv = ld4(yc + e0);
            const V4<T> w2v = (it >= 2) ? ld4(w2 + o3 + e0) : zero4<T>();
            const V4<T> w1v = (it >= 3) ? ld4(w1 + o3 + e0) : zero4<T>();
            const V4<T> xv = (it >= 2) ? ld4(xd + o3 + e0) : zero4<T>();
            V4<T> wn, xn;
            d_update4<T>(yv, w1v, w2v, xv, iv, oe, de, ig, ph, wn, xn);
            st4(w1 + o3 + e0, wn);
            st4(xd + o3 + e0, xn);
        }
    }
    if (doA) {
        const double t = block_sum_t<256, T>(acc, red);
        if (threadIdx.x == 0) partA[(int64_t)s * kMaxPartials + blockIdx.x] = t;
    }
}

template <typename T>
int launch_minres_A(const Grid3& g, double kh2, int S, const T* y, const T* u, double fd, double* partA,
                    MinresCol* st_, const T* yprev, T* w1, const T* w2, T* xd, cudaStream_t st, const T* kh2c,
                    const T* kh2s) {
    const int nb = cell_blocks(g.cells() / 16);  // four quads per thread: one reduction per 1024 quads
    dim3 grid(nb, S);
    if (g.cube())
        k_minres_A<T, true><<<grid, 256, 0, st>>>(g, (T)kh2, y, u, (T)fd, partA, st_, yprev, w1, w2, xd, kh2c, kh2s);
    else
        k_minres_A<T, false><<<grid, 256, 0, st>>>(g, (T)kh2, y, u, (T)fd, partA, st_, yprev, w1, w2, xd, kh2c, kh2s);
    return nb;
}

// B(k): the next unpreconditioned Lanczos vector, in place over r1,
//   r1' = (A y) / beta - (beta / oldb) r1 - (alpha / beta) r2
// (A y rebuilt from the flux blocks of r2 and the cell block of y, as in pass
// A), with two partial sums per block:
//   partB: the flux part of beta'^2 = r1'.y', i.e. r1'_flux . (fd r1'_flux)
//          (the flux block of the next preconditioned vector, never stored);
//   partE: r1'.y = fd r1'_flux . r2_flux + r1'_cell . y_cell, the v.r1 term of
//          the next iteration's alpha (times its beta).
// Each thread reads r1 and writes r1' at its own cells only; r2 and y are
// not written.
template <typename T, bool CUBE>
__global__ void __launch_bounds__(256, 2) k_minres_B(Grid3 gin, T kh2, const T* __restrict__ y, const T* __restrict__ r2, T fd,
                                                     T* __restrict__ r1, double* __restrict__ partB,
                                                     double* __restrict__ partE, const MinresCol* __restrict__ st,
                                                     const T* __restrict__ kh2c, const T* __restrict__ kh2s) {
    __shared__ double red[8];
    const int s = blockIdx.y;
    const MinresCol& cs = st[s];
    if (!cs.active) return;
    const Grid3 g = pass_grid<T, CUBE>(gin);
    const int n3 = 1 << (g.lx + g.ly + g.lz);
    const int nq = n3 >> 2;
    const int64_t off = (int64_t)s * 4 * n3;
    const T* ys = y + off;
    const T* us = r2 + off;
    T* rs = r1 + off;
    const T ib = col_coef<T>(cs, KC_IB);
    const T coef = col_coef<T>(cs, KC_COEF);
    const T f = col_coef<T>(cs, KC_F);
    // r1 holds no data before the second iteration (coef == 0): do not read it
    const bool use_r1 = coef != T(0);
    T accB = T(0), accE = T(0);
    // FP32: two quads in flight per thread; two CTAs per SM (127 registers) and the loop
    // unrolled by two measured 6 % faster than three CTAs without the unroll (at four it
    // spills).  FP64 keeps one quad at a time (unrolled, it spills).
#pragma unroll(sizeof(T) == 4 ? 2 : 1)
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
        const QuadPos p = quad_pos(q, g);
        T yu[4], yv[4], yw[4], yt[4];
        V4<T> vc[4];
        apply_quad_fd<T>(us, ys + 3 * n3, fd, g, p, quad_kh2<T>(kh2, kh2c, kh2s, s, p.c), yu, yv, yw, yt, vc);
        const V4<T> pt = ld4(us + 3 * n3 + p.c);  // cell block of r2 (its flux blocks are vc[0..2])
        V4<T> z0, z1, z2, z3;
        if (use_r1) {
            z0 = ld4(rs + p.c);
            z1 = ld4(rs + n3 + p.c);
            z2 = ld4(rs + 2 * n3 + p.c);
            z3 = ld4(rs + 3 * n3 + p.c);
        } else {
            z0 = z1 = z2 = z3 = zero4<T>();
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            z0.v[e] = (yu[e] * ib - coef * z0.v[e]) - f * vc[0].v[e];
            z1.v[e] = (yv[e] * ib - coef * z1.v[e]) - f * vc[1].v[e];
            z2.v[e] = (yw[e] * ib - coef * z2.v[e]) - f * vc[2].v[e];
            z3.v[e] = (yt[e] * ib - coef * z3.v[e]) - f * pt.v[e];
            accB += z0.v[e] * (fd * z0.v[e]) + z1.v[e] * (fd * z1.v[e]) + z2.v[e] * (fd * z2.v[e]);
            accE += fd * (z0.v[e] * vc[0].v[e] + z1.v[e] * vc[1].v[e] + z2.v[e] * vc[2].v[e]) + z3.v[e] * vc[3].v[e];
        }
        st4(rs + p.c, z0);
        st4(rs + n3 + p.c, z1);
        st4(rs + 2 * n3 + p.c, z2);
        st4(rs + 3 * n3 + p.c, z3);
    }
    const double tB = block_sum_t<256, T>(accB, red);
    if (threadIdx.x == 0) partB[(int64_t)s * kMaxPartials + blockIdx.x] = tB;
    const double tE = block_sum_t<256, T>(accE, red);
    if (threadIdx.x == 0) partE[(int64_t)s * kMaxPartials + blockIdx.x] = tE;
}

template <typename T>
int launch_minres_B(const Grid3& g, double kh2, int S, const T* y, const T* r2, double fd, T* r1, double* partB,
                    double* partE, MinresCol* st_, cudaStream_t st, const T* kh2c, const T* kh2s) {
    const int nb = cell_blocks(g.cells() / 16);
    dim3 grid(nb, S);
    if (g.cube())
        k_minres_B<T, true><<<grid, 256, 0, st>>>(g, (T)kh2, y, r2, (T)fd, r1, partB, partE, st_, kh2c, kh2s);
    else
        k_minres_B<T, false><<<grid, 256, 0, st>>>(g, (T)kh2, y, r2, (T)fd, r1, partB, partE, st_, kh2c, kh2s);
    return nb;
}

template <typename T>
__global__ void __launch_bounds__(256) k_precond_u(int64_t N4, int64_t n3u, const T* __restrict__ r, T* __restrict__ y,
                                                   T fd, double* __restrict__ part, const MinresCol* __restrict__ st) {
    __shared__ double red[8];
    const int s = blockIdx.y;
    if (st && !st[s].active) return;
    const int64_t off = (int64_t)s * N4;
    T acc = T(0);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n3u; e += (int64_t)gridDim.x * blockDim.x) {
        const T z = r[off + e];
        const T yv = fd * z;
        y[off + e] = yv;
        acc += z * yv;
    }
    const double t = block_sum<256>((double)acc, red);
    if (part && threadIdx.x == 0) part[(int64_t)s * kMaxPartials + blockIdx.x] = t;
}

template <typename T>
int launch_precond_u(int64_t N4, int n3, int S, const T* r, T* y, double fd, double* part, const MinresCol* st_,
                     cudaStream_t st) {
    const int nb = elem_blocks(3 * (int64_t)n3);
    dim3 grid(nb, S);
    k_precond_u<T><<<grid, 256, 0, st>>>(N4, 3 * (int64_t)n3, r, y, (T)fd, part, st_);
    return nb;
}

__device__ __forceinline__ double col_sum(const double* part, int s, int nb, double* red) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += part[(int64_t)s * kMaxPartials + b];
    return block_sum<256>(acc, red);
}

__global__ void __launch_bounds__(256) k_alpha(const double* __restrict__ partA, int nA, MinresCol* __restrict__ st) {
    __shared__ double red[8];
    const int s = blockIdx.x;
    if (!st[s].active) return;
    const double a = col_sum(partA, s, nA, red);  // y.(A y), y = beta v
    if (threadIdx.x == 0) {
        MinresCol& c = st[s];
        // alpha = v.A v - (beta / oldb) v.r1, with v.r1 = (r2.yprev) / beta kept by the Givens step
        const double alpha = a / (c.beta * c.beta) - (c.oldb > 0.0 ? c.ry / c.oldb : 0.0);
        c.alpha = alpha;
        set_coef(c, KC_F, alpha / c.beta);
    }
}

cudaError_t launch_alpha(int S, const double* partA, int nA, MinresCol* st_, cudaStream_t st) {
    k_alpha<<<S, 256, 0, st>>>(partA, nA, st_);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_givens(const double* __restrict__ partB, int nB, const double* __restrict__ partC,
                                                int nC, const double* __restrict__ partE, MinresCol* __restrict__ st,
                                                int* __restrict__ nactive, int max_iter) {
    __shared__ double red[8];
    const int s = blockIdx.x;
    MinresCol& c = st[s];
    if (!c.active) {
        if (threadIdx.x == 0) c.upd = 0;
        return;
    }
    const double b2 = col_sum(partB, s, nB, red);
    const double b3 = col_sum(partC, s, nC, red);
    const double ry = col_sum(partE, s, nB, red);  // r'.y of pass B (same blocks as partB)
    if (threadIdx.x != 0) return;
    const double beta2 = b2 + b3;
    const double beta = sqrt(fmax(beta2, 0.0));
    c.ry = ry;
    c.oldb = c.beta;
    c.beta = beta;
    c.oldeps = c.epsln;
    const double delta = c.cs * c.dbar + c.sn * c.alpha;
    const double gbar = c.sn * c.dbar - c.cs * c.alpha;
    c.epsln = c.sn * beta;
    c.dbar = -c.cs * beta;
    double gamma = sqrt(gbar * gbar + beta2);
    gamma = fmax(gamma, 1e-300);
    c.cs = gbar / gamma;
    c.sn = beta / gamma;
    c.phi = c.cs * c.phibar;
    c.phibar = c.sn * c.phibar;
    c.delta = delta;
    c.gamma = gamma;
    c.upd = 1;
    c.iters += 1;
    // coefficients of this iteration's w/x update, applied by the next fused pass
    c.d_oldb = c.oldb;
    c.d_oldeps = c.oldeps;
    c.d_delta = delta;
    c.d_gamma = gamma;
    c.d_phi = c.phi;
    c.d_iter = c.iters;
    set_coef(c, KC_IB, 1.0 / beta);
    set_coef(c, KC_COEF, c.oldb > 0.0 ? beta / c.oldb : 0.0);
    set_coef(c, KC_IV, 1.0 / c.d_oldb);
    set_coef(c, KC_OE, c.d_oldeps);
    set_coef(c, KC_DE, c.d_delta);
    set_coef(c, KC_IG, 1.0 / c.d_gamma);
    set_coef(c, KC_PH, c.d_phi);
    const bool done = !(beta2 > 0.0) || !isfinite(beta) || c.phibar <= c.tol * c.beta1 || c.iters >= max_iter;
    if (nactive) atomicAdd(nactive + 1, 1);  // this column's update is pending
    if (done) c.active = 0;
    else if (nactive) atomicAdd(nactive, 1);
}

cudaError_t launch_givens(int S, const double* partB, int nB, const double* partC, int nC, const double* partE,
                          MinresCol* st_, int* nactive, cudaStream_t st, int max_iter) {
    k_givens<<<S, 256, 0, st>>>(partB, nB, partC, nC, partE, st_, nactive, max_iter);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Control of the graph-driven refinement.  The captured graph runs
//   init; while (go) { residual; check -> go; inner solve; correction }
// with the inner solve's iterations in a nested while; these kernels take the
// decisions the synchronous host loop takes (same FP64 formulas, same order of
// the per-column tests), so both paths produce the same bits.
// ---------------------------------------------------------------------------
__global__ void k_refine_init(RefineCtl* ctl, int* fault, cudaGraphConditionalHandle h_outer) {
    ctl->outer = 0;
    ctl->inner = 0;
    ctl->it = 0;
    ctl->status = 0;
    for (int k = 0; k < 6; ++k) ctl->cnt[k] = 0;
    ctl->worst = 0.0;
    *fault = 0;  // a timeout of an earlier solve was reported with that solve
    cudaGraphSetConditional(h_outer, 1u);
}

cudaError_t launch_refine_init(RefineCtl* ctl, int* fault, unsigned long long h_outer, cudaStream_t st) {
    k_refine_init<<<1, 1, 0, st>>>(ctl, fault, (cudaGraphConditionalHandle)h_outer);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_refine_check(int S, const double* __restrict__ colv, double tol,
                                                      double inner_tol, int fp64_inner, int max_outer,
                                                      const int* __restrict__ fault, int* __restrict__ mask,
                                                      double* __restrict__ coltol, RefineCtl* __restrict__ ctl,
                                                      cudaGraphConditionalHandle h_outer) {
    __shared__ double smax[8];
    __shared__ int scnt[8];
    double worst = 0.0;
    int nact = 0;
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        const double fn = colv[S + s];
        const double rel = fn > 0.0 ? sqrt(colv[s] / fn) : 0.0;
        worst = fmax(worst, rel);
        nact += rel > tol ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) {
        worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
        nact += __shfl_xor_sync(0xffffffffu, nact, o);
    }
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        smax[wid] = worst;
        scnt[wid] = nact;
    }
    __syncthreads();
    double W = 0.0;
    int N = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
        W = fmax(W, smax[k]);
        N += scnt[k];
    }
    const int flt = *(volatile const int*)fault;
    const bool stop = flt != 0 || N == 0 || ctl->outer >= max_outer;
    const double wtol = fmax(0.1 * tol / fmax(W, 1e-300), 1e-15);  // FP64 inner: one reduction for all
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
        const double fn = colv[S + s];
        const double rel = fn > 0.0 ? sqrt(colv[s] / fn) : 0.0;
        mask[s] = (!stop && rel > tol) ? 1 : 0;
        coltol[s] = fp64_inner ? wtol : fmax(inner_tol, 0.1 * tol / fmax(rel, 1e-300));
    }
    if (threadIdx.x == 0) {
        ctl->worst = W;
        ctl->it = 0;
        for (int k = 0; k < 6; ++k) ctl->cnt[k] = 0;
        if (stop) ctl->status = flt ? 5 : (W > tol ? 4 : 0);
        else ctl->outer += 1;
        cudaGraphSetConditional(h_outer, stop ? 0u : 1u);
    }
}

cudaError_t launch_refine_check(int S, const double* colv, double tol, double inner_tol, int fp64_inner,
                                int max_outer, const int* fault, int* mask, double* coltol, RefineCtl* ctl,
                                unsigned long long h_outer, cudaStream_t st) {
    k_refine_check<<<1, 256, 0, st>>>(S, colv, tol, inner_tol, fp64_inner, max_outer, fault, mask, coltol, ctl,
                                      (cudaGraphConditionalHandle)h_outer);
    return cudaGetLastError();
}

__global__ void k_loop_ctl(RefineCtl* ctl, int slot, int add, int max_iter, cudaGraphConditionalHandle h_loop) {
    const int active = ctl->cnt[2 * slot];
    ctl->it += add;
    ctl->inner += add;
    for (int k = 0; k < 6; ++k) ctl->cnt[k] = 0;
    cudaGraphSetConditional(h_loop, (active > 0 && ctl->it < max_iter) ? 1u : 0u);
}

cudaError_t launch_loop_ctl(RefineCtl* ctl, int slot, int add, int max_iter, unsigned long long h_loop,
                            cudaStream_t st) {
    k_loop_ctl<<<1, 1, 0, st>>>(ctl, slot, add, max_iter, (cudaGraphConditionalHandle)h_loop);
    return cudaGetLastError();
}

__global__ void k_refine_finish(const RefineCtl* ctl, CallAcc* acc, int count_iters) {
    if (count_iters) {
        atomicMax(&acc->outer, ctl->outer);
        atomicMax(&acc->inner, ctl->inner);
    }
    atomicMax(&acc->status, ctl->status);
    atomicAdd(&acc->nsolve, 1);
    atomicMax(&acc->worst_bits, (unsigned long long)__double_as_longlong(fmax(ctl->worst, 0.0)));
}

cudaError_t launch_refine_finish(const RefineCtl* ctl, CallAcc* acc, int count_iters, cudaStream_t st) {
    k_refine_finish<<<1, 1, 0, st>>>(ctl, acc, count_iters);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_minres_init(const double* __restrict__ partB, int nB,
                                                     const double* __restrict__ partC, int nC, double tol,
                                                     MinresCol* __restrict__ st, int* __restrict__ nactive,
                                                     const double* __restrict__ col_tol) {
    __shared__ double red[8];
    const int s = blockIdx.x;
    MinresCol& c = st[s];
    if (!c.active) {
        if (threadIdx.x == 0) c.upd = 0;
        return;
    }
    const double b2 = col_sum(partB, s, nB, red);
    const double b3 = col_sum(partC, s, nC, red);
    if (threadIdx.x != 0) return;
    const double beta2 = b2 + b3;
    const double beta1 = sqrt(fmax(beta2, 0.0));
    c.beta = beta1;
    c.oldb = 0.0;
    c.alpha = 0.0;
    c.dbar = 0.0;
    c.epsln = 0.0;
    c.oldeps = 0.0;
    c.phibar = beta1;
    c.cs = -1.0;
    c.sn = 0.0;
    c.gamma = 0.0;
    c.delta = 0.0;
    c.phi = 0.0;
    c.beta1 = beta1;
    c.ry = 0.0;
    c.tol = col_tol ? col_tol[s] : tol;
    c.upd = 0;
    c.iters = 0;
    set_coef(c, KC_IB, 1.0 / beta1);
    set_coef(c, KC_COEF, 0.0);
    c.active = (beta2 > 0.0 && isfinite(beta1)) ? 1 : 0;
    if (c.active && nactive) atomicAdd(nactive, 1);
}

cudaError_t launch_minres_init(int S, const double* partB, int nB, const double* partC, int nC, double tol,
                               MinresCol* st_, int* nactive, cudaStream_t st, const double* col_tol) {
    k_minres_init<<<S, 256, 0, st>>>(partB, nB, partC, nC, tol, st_, nactive, col_tol);
    return cudaGetLastError();
}

// Update of the solution recurrences on the cell block only: the caller keeps
// w1, w2, x as [S][n^3]; v = y / oldb is read from the cell block of y.
template <typename T>
__global__ void __launch_bounds__(256) k_minres_D(int64_t n3, const T* __restrict__ ycur, T* __restrict__ w1,
                                                  const T* __restrict__ w2, T* __restrict__ x,
                                                  const MinresCol* __restrict__ st) {
    const int s = blockIdx.y;
    const MinresCol& c = st[s];
    if (!c.upd) return;
    const T iv = col_coef<T>(c, KC_IV), oe = col_coef<T>(c, KC_OE), de = col_coef<T>(c, KC_DE);
    const T ig = col_coef<T>(c, KC_IG), ph = col_coef<T>(c, KC_PH);
    const T* ys = ycur + (int64_t)s * 4 * n3 + 3 * n3;
    const int64_t off = (int64_t)s * n3;
    // iteration 1: w1 = w2 = 0 and x = 0; iteration 2: w1 = 0 (buffers hold no data yet)
    const int it = c.d_iter;
    const int64_t nq = n3 >> 2;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = 4 * q;
        const V4<T> yv = ld4(ys + e);
        const V4<T> w2v = (it >= 2) ? ld4(w2 + off + e) : zero4<T>();
        const V4<T> w1v = (it >= 3) ? ld4(w1 + off + e) : zero4<T>();
        const V4<T> xv = (it >= 2) ? ld4(x + off + e) : zero4<T>();
        V4<T> wn, xn;
        d_update4<T>(yv, w1v, w2v, xv, iv, oe, de, ig, ph, wn, xn);
        st4(w1 + off + e, wn);
        st4(x + off + e, xn);
    }
}

template <typename T>
cudaError_t launch_minres_D(int64_t n3, int S, const T* ycur, T* w1, const T* w2, T* x, const MinresCol* st_,
                            cudaStream_t st) {
    dim3 grid(elem_blocks(n3), S);
    k_minres_D<T><<<grid, 256, 0, st>>>(n3, ycur, w1, w2, x, st_);
    return cudaGetLastError();
}

__global__ void k_active_flags(int S, const MinresCol* __restrict__ st, int* __restrict__ flags) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) flags[s] = st[s].active;
}

cudaError_t launch_active_flags(int S, const MinresCol* st_, int* flags, cudaStream_t st) {
    k_active_flags<<<(S + 127) / 128, 128, 0, st>>>(S, st_, flags);
    return cudaGetLastError();
}

#define SPDE_KRYLOV_INST(T)                                                                                        \
    template int launch_minres_A<T>(const Grid3&, double, int, const T*, const T*, double, double*, MinresCol*,    \
                                    const T*, T*, const T*, T*, cudaStream_t, const T*, const T*);                 \
    template int launch_minres_B<T>(const Grid3&, double, int, const T*, const T*, double, T*, double*, double*,    \
                                    MinresCol*, cudaStream_t, const T*, const T*);                                 \
    template int launch_precond_u<T>(int64_t, int, int, const T*, T*, double, double*, const MinresCol*,          \
                                     cudaStream_t);                                                                \
    template cudaError_t launch_minres_D<T>(int64_t, int, const T*, T*, const T*, T*, const MinresCol*,          \
                                            cudaStream_t);
SPDE_KRYLOV_INST(float)
SPDE_KRYLOV_INST(double)

}  // namespace spde

namespace spde {

// x64 += d for columns whose inner solve ran at least one iteration
template <typename T>
__global__ void __launch_bounds__(256) k_add_correction_st(int64_t N4, double* __restrict__ x, const T* __restrict__ d,
                                                           const MinresCol* __restrict__ st) {
    const int s = blockIdx.y;
    if (st[s].iters == 0) return;
    const int64_t off = (int64_t)s * N4;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N4; e += (int64_t)gridDim.x * blockDim.x)
        x[off + e] += (double)d[off + e];
}

template <typename T>
cudaError_t launch_add_correction_st(int64_t N4, int S, double* x, const T* d, const MinresCol* st_, cudaStream_t st) {
    dim3 grid(elem_blocks(N4), S);
    k_add_correction_st<T><<<grid, 256, 0, st>>>(N4, x, d, st_);
    return cudaGetLastError();
}
template cudaError_t launch_add_correction_st<float>(int64_t, int, double*, const float*, const MinresCol*, cudaStream_t);
template cudaError_t launch_add_correction_st<double>(int64_t, int, double*, const double*, const MinresCol*,
                                                      cudaStream_t);

// st[s].active = mask[s] (1 when mask is null); iteration counters cleared
__global__ void k_set_active(int S, const int* __restrict__ mask, MinresCol* __restrict__ st) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    st[s].active = mask ? mask[s] : 1;
    st[s].iters = 0;
    st[s].upd = 0;
}

cudaError_t launch_set_active(int S, const int* mask, MinresCol* st_, cudaStream_t st) {
    k_set_active<<<(S + 127) / 128, 128, 0, st>>>(S, mask, st_);
    return cudaGetLastError();
}

}  // namespace spde
