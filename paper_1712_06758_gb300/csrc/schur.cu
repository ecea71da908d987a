// Schur-complement variant of the field solve: preconditioned CG on the
// cell unknowns only, with the identical solution theta.
//
// Eliminating the fluxes from the scaled mixed system (first block row
// T u + D1^T theta = 0) gives S theta = -F with
//     S = (kappa h)^2 I + D1 T^{-1} D1^T           (symmetric positive definite)
// (Sec. 4.2: S = kappa^2 W + B M^{-1} B^T in scaled form).  S is applied
// matrix-free, one axis at a time: along every grid line the face values
// g = D1^T x are formed, T u = g is solved exactly by Thomas elimination
// (T = tridiag(1/6, 2/3, 1/6) on the n-1 interior faces), and the line's
// divergence D1 u is accumulated into the output.  Lines along x are
// contiguous rows: a CTA stages a tile of rows in shared memory (coalesced)
// and one warp walks them.  Lines along y and z are walked by one thread each,
// consecutive threads on consecutive x, so every step is one coalesced row of
// the grid; the forward elimination keeps its values in a scratch array that
// the backward substitution reads back (it stays in L2 while the lines are in
// flight), and the unrolled walks keep several independent loads in flight.
// The preconditioner is the same V-cycle as the MINRES field block.
#include "device.cuh"
#include "internal.h"

namespace spde {

constexpr int kRowThreads = 128;  // x-axis CTA
constexpr int kRowTileMax = 32;   // rows per x-axis CTA (one warp solves them)
constexpr int kLineThreads = 256; // y/z-axis CTA: one line per thread
constexpr size_t kSchurSmemMax = 200 * 1024;

template <typename T>
static int row_tile(int n) {
    int R = kRowTileMax;
    while (R > 1 && ((int64_t)R > (int64_t)n * n || 2 * (size_t)R * (n + 1) * sizeof(T) > kSchurSmemMax)) R >>= 1;
    return R;
}

// y = (kappa h)^2 x + the x-axis term, for the R rows (j, k) of one tile
template <typename T>
__global__ void __launch_bounds__(kRowThreads) k_schur_x(int n, int R, T kh2, const T* __restrict__ x, T* __restrict__ y,
                                                         const T* __restrict__ tri, const CgCol* __restrict__ st) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int s = blockIdx.y;
    if (st && !st[s].active) return;
    const int P = n + 1;                     // padded row: no bank conflicts along the walk
    T* sx = reinterpret_cast<T*>(smem_raw);  // [R][n + 1]: x
    T* su = sx + R * P;                      // [R][n + 1]: face values
    const int64_t n3 = (int64_t)n * n * n;
    const int64_t start = (int64_t)s * n3 + (int64_t)blockIdx.x * R * n;  // R contiguous rows
    const int t = threadIdx.x;
    for (int idx = t; idx < R * n; idx += kRowThreads) {
        const int l = idx / n, e = idx - l * n;
        sx[l * P + e] = x[start + idx];
    }
    __syncthreads();
    if (t < R) {
        // T u = D1^T x along the row, (D1^T x)_f = x_f - x_{f+1}; Thomas elimination
        const T* xl = sx + t * P;
        T* ul = su + t * P;
        const T* cp = tri;
        const T* inv = tri + (n - 1);
        const T a = T(1) / T(6);
        T prev = T(0);
        for (int f = 0; f < n - 1; ++f) {
            const T dp = ((xl[f] - xl[f + 1]) - a * prev) * inv[f];
            ul[f] = dp;
            prev = dp;
        }
        T un = prev;  // u_{n-2}
        for (int f = n - 3; f >= 0; --f) {
            const T uf = ul[f] - cp[f] * un;
            ul[f] = uf;
            un = uf;
        }
        ul[n - 1] = T(0);  // wall face
    }
    __syncthreads();
    for (int idx = t; idx < R * n; idx += kRowThreads) {  // cell e gains u_e - u_{e-1}
        const int l = idx / n, e = idx - l * n;
        const T* ul = su + l * P;
        y[start + idx] = kh2 * sx[l * P + e] + (ul[e] - (e > 0 ? ul[e - 1] : T(0)));
    }
}

// y += the term of axis AXIS (1: y, 2: z); with DOT, partial sums of x.y (y final)
template <typename T, int AXIS, bool DOT>
__global__ void __launch_bounds__(kLineThreads) k_schur_line(int n, int logn, const T* __restrict__ x, T* __restrict__ y,
                                                             T* __restrict__ scratch, const T* __restrict__ tri,
                                                             double* __restrict__ dot_part,
                                                             const CgCol* __restrict__ st) {
    __shared__ double red[kLineThreads / 32];
    const int s = blockIdx.y;
    if (st && !st[s].active) return;
    const int L = blockIdx.x * kLineThreads + threadIdx.x;  // line: x index i fastest
    const int nlines = 1 << (2 * logn);
    T acc = T(0);
    if (L < nlines) {
        const int i = L & (n - 1), o = L >> logn;
        const int64_t base = (AXIS == 1) ? i + ((int64_t)o << (2 * logn)) : i + ((int64_t)o << logn);
        const int64_t stride = (AXIS == 1) ? n : (int64_t)n * n;
        const int64_t off = (int64_t)s * ((int64_t)n * n * n) + base;
        const T* xs = x + off;
        T* ys = y + off;
        T* gs = scratch + off;
        const T* cp = tri;
        const T* inv = tri + (n - 1);
        const T a = T(1) / T(6);
        T prev = T(0), xc = xs[0];
#pragma unroll 8
        for (int f = 0; f < n - 1; ++f) {
            const T xn = xs[(int64_t)(f + 1) * stride];
            const T dp = ((xc - xn) - a * prev) * inv[f];
            gs[(int64_t)f * stride] = dp;
            prev = dp;
            xc = xn;
        }
        // backward substitution; cell c gains u_c - u_{c-1} (u_{-1} = u_{n-1} = 0)
        T un = prev;  // u_{n-2}
        {
            const int64_t gc = (int64_t)(n - 1) * stride;
            const T v = ys[gc] - un;
            ys[gc] = v;
            if (DOT) acc += xs[gc] * v;
        }
#pragma unroll 8
        for (int f = n - 3; f >= 0; --f) {
            const T uf = gs[(int64_t)f * stride] - cp[f] * un;
            const int64_t gc = (int64_t)(f + 1) * stride;
            const T v = ys[gc] + (un - uf);
            ys[gc] = v;
            if (DOT) acc += xs[gc] * v;
            un = uf;
        }
        {
            const T v = ys[0] + un;  // cell 0: u_0
            ys[0] = v;
            if (DOT) acc += xs[0] * v;
        }
    }
    if (DOT) {
        const double tsum = block_sum_t<kLineThreads, T>(acc, red);
        if (threadIdx.x == 0) dot_part[(int64_t)s * kMaxPartials + blockIdx.x] = tsum;
    }
}

template <typename T>
static cudaError_t schur_attrs() {
    static const cudaError_t e =
        cudaFuncSetAttribute(k_schur_x<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSchurSmemMax);
    return e;
}

// y = S x for S columns (scratch: [S][n^3] of the element type); partial sums of x.y per column
// into dot_part (blocks per column returned, or -1)
template <typename T>
int launch_schur_apply(int n, double kh2, int S, const T* x, T* y, const T* tri, T* scratch, double* dot_part,
                       const CgCol* st, cudaStream_t stream) {
    if (schur_attrs<T>() != cudaSuccess) return -1;
    const int logn = 31 - __builtin_clz(n);
    const int R = row_tile<T>(n);
    const size_t smem = 2 * (size_t)R * (n + 1) * sizeof(T);
    k_schur_x<T><<<dim3(n * n / R, S), kRowThreads, smem, stream>>>(n, R, (T)kh2, x, y, tri, st);
    const int nb = (n * n + kLineThreads - 1) / kLineThreads;
    dim3 grid(nb, S);
    k_schur_line<T, 1, false><<<grid, kLineThreads, 0, stream>>>(n, logn, x, y, scratch, tri, nullptr, st);
    if (dot_part)
        k_schur_line<T, 2, true><<<grid, kLineThreads, 0, stream>>>(n, logn, x, y, scratch, tri, dot_part, st);
    else
        k_schur_line<T, 2, false><<<grid, kLineThreads, 0, stream>>>(n, logn, x, y, scratch, tri, nullptr, st);
    return nb;
}

// ---------------------------------------------------------------------------
// CG vector updates and per-column scalars
// ---------------------------------------------------------------------------
// x += alpha p; r -= alpha q; partial r.r
template <typename T>
__global__ void __launch_bounds__(256) k_cg_xr(int64_t n3, T* __restrict__ x, T* __restrict__ r,
                                               const T* __restrict__ p, const T* __restrict__ q,
                                               double* __restrict__ part, const CgCol* __restrict__ st) {
    __shared__ double red[8];
    const int s = blockIdx.y;
    const CgCol& c = st[s];
    if (!c.active) return;
    const T al = (T)c.alpha;
    const int64_t off = (int64_t)s * n3;
    T acc = T(0);
    for (int64_t e = 4 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x); e < n3; e += 4 * (int64_t)gridDim.x * blockDim.x) {
        V4<T> xv = (c.iters > 0) ? ld4(x + off + e) : zero4<T>();
        V4<T> rv = ld4(r + off + e);
        const V4<T> pv = ld4(p + off + e), qv = ld4(q + off + e);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            xv.v[k] += al * pv.v[k];
            rv.v[k] -= al * qv.v[k];
            acc += rv.v[k] * rv.v[k];
        }
        st4(x + off + e, xv);
        st4(r + off + e, rv);
    }
    const double t = block_sum<256>((double)acc, red);
    if (threadIdx.x == 0) part[(int64_t)s * kMaxPartials + blockIdx.x] = t;
}

// p = z + beta p (beta = 0 starts the recurrence)
template <typename T>
__global__ void __launch_bounds__(256) k_cg_p(int64_t n3, T* __restrict__ p, const T* __restrict__ z,
                                              const CgCol* __restrict__ st) {
    const int s = blockIdx.y;
    const CgCol& c = st[s];
    if (!c.active) return;
    const T be = (T)c.beta;
    const bool first = c.iters == 0;
    const int64_t off = (int64_t)s * n3;
    for (int64_t e = 4 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x); e < n3; e += 4 * (int64_t)gridDim.x * blockDim.x) {
        const V4<T> zv = ld4(z + off + e);
        V4<T> pv = first ? zero4<T>() : ld4(p + off + e);
#pragma unroll
        for (int k = 0; k < 4; ++k) pv.v[k] = zv.v[k] + be * pv.v[k];
        st4(p + off + e, pv);
    }
}

__device__ __forceinline__ double cg_col_sum(const double* part, int s, int nb, double* red) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) acc += part[(int64_t)s * kMaxPartials + b];
    return block_sum<256>(acc, red);
}

// after q = S p: alpha = rz / p.q
__global__ void __launch_bounds__(256) k_cg_alpha(const double* __restrict__ part, int nb, CgCol* __restrict__ st) {
    __shared__ double red[8];
    const int s = blockIdx.x;
    CgCol& c = st[s];
    if (!c.active) return;
    const double pq = cg_col_sum(part, s, nb, red);
    if (threadIdx.x == 0) {
        c.alpha = (pq > 0.0 && isfinite(pq)) ? c.rz / pq : 0.0;
        if (!(pq > 0.0) || !isfinite(pq)) c.active = 0;  // breakdown: stop this column
    }
}

// after r update and z = M^{-1} r: convergence on ||r||, beta = rz_new / rz
__global__ void __launch_bounds__(256) k_cg_beta(const double* __restrict__ part_rr, int nrr,
                                                 const double* __restrict__ part_rz, int nrz, CgCol* __restrict__ st,
                                                 int* __restrict__ nactive, int max_iter) {
    __shared__ double red[8];
    const int s = blockIdx.x;
    CgCol& c = st[s];
    if (!c.active) return;
    const double rr = cg_col_sum(part_rr, s, nrr, red);
    const double rz = cg_col_sum(part_rz, s, nrz, red);
    if (threadIdx.x != 0) return;
    c.iters += 1;
    c.beta = (c.rz > 0.0) ? rz / c.rz : 0.0;
    c.rz = rz;
    const bool done = !(rr > c.tol2 * c.rr0) || !(rz > 0.0) || !isfinite(rz) || c.iters >= max_iter;
    if (done) c.active = 0;
    else if (nactive) atomicAdd(nactive, 1);
}

// start: r = b given, z = M^{-1} r; rz, rr0 from partial sums
__global__ void __launch_bounds__(256) k_cg_init(const double* __restrict__ part_rz, int nrz,
                                                 const double* __restrict__ part_rr, int nrr, double tol,
                                                 CgCol* __restrict__ st, int* __restrict__ nactive) {
    __shared__ double red[8];
    const int s = blockIdx.x;
    CgCol& c = st[s];
    if (!c.active) return;
    const double rz = cg_col_sum(part_rz, s, nrz, red);
    const double rr = cg_col_sum(part_rr, s, nrr, red);
    if (threadIdx.x != 0) return;
    c.rz = rz;
    c.rr0 = rr;
    c.tol2 = tol * tol;
    c.alpha = 0.0;
    c.beta = 0.0;
    c.iters = 0;
    c.active = (rr > 0.0 && rz > 0.0 && isfinite(rz)) ? 1 : 0;
    if (c.active && nactive) atomicAdd(nactive, 1);
}

// r = -(cell block of the mixed residual), partial r.r
template <typename T>
__global__ void __launch_bounds__(256) k_cg_rhs(int64_t n3, const T* __restrict__ mixed_r, T* __restrict__ r,
                                                double* __restrict__ part, const CgCol* __restrict__ st) {
    __shared__ double red[8];
    const int s = blockIdx.y;
    if (!st[s].active) return;
    const T* src = mixed_r + (int64_t)s * 4 * n3 + 3 * n3;
    T* dst = r + (int64_t)s * n3;
    T acc = T(0);
    for (int64_t e = 4 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x); e < n3; e += 4 * (int64_t)gridDim.x * blockDim.x) {
        V4<T> v = ld4(src + e);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v.v[k] = -v.v[k];
            acc += v.v[k] * v.v[k];
        }
        st4(dst + e, v);
    }
    const double t = block_sum<256>((double)acc, red);
    if (threadIdx.x == 0) part[(int64_t)s * kMaxPartials + blockIdx.x] = t;
}

__global__ void k_cg_set_active(int S, const int* __restrict__ mask, CgCol* __restrict__ st) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < S) {
        st[s].active = mask ? mask[s] : 1;
        st[s].iters = 0;
    }
}

static inline int cg_blocks(int64_t n3) {
    int64_t b = (n3 / 4 + 255) / 256;
    if (b > 2048) b = 2048;
    return (int)(b < 1 ? 1 : b);
}

template <typename T>
int launch_cg_xr(int64_t n3, int S, T* x, T* r, const T* p, const T* q, double* part, const CgCol* st, cudaStream_t s) {
    const int nb = cg_blocks(n3);
    k_cg_xr<T><<<dim3(nb, S), 256, 0, s>>>(n3, x, r, p, q, part, st);
    return nb;
}
template <typename T>
cudaError_t launch_cg_p(int64_t n3, int S, T* p, const T* z, const CgCol* st, cudaStream_t s) {
    k_cg_p<T><<<dim3(cg_blocks(n3), S), 256, 0, s>>>(n3, p, z, st);
    return cudaGetLastError();
}
template <typename T>
int launch_cg_rhs(int64_t n3, int S, const T* mixed_r, T* r, double* part, const CgCol* st, cudaStream_t s) {
    const int nb = cg_blocks(n3);
    k_cg_rhs<T><<<dim3(nb, S), 256, 0, s>>>(n3, mixed_r, r, part, st);
    return nb;
}
cudaError_t launch_cg_alpha(int S, const double* part, int nb, CgCol* st, cudaStream_t s) {
    k_cg_alpha<<<S, 256, 0, s>>>(part, nb, st);
    return cudaGetLastError();
}
cudaError_t launch_cg_beta(int S, const double* prr, int nrr, const double* prz, int nrz, CgCol* st, int* nactive,
                           cudaStream_t s, int max_iter) {
    k_cg_beta<<<S, 256, 0, s>>>(prr, nrr, prz, nrz, st, nactive, max_iter);
    return cudaGetLastError();
}
cudaError_t launch_cg_init(int S, const double* prz, int nrz, const double* prr, int nrr, double tol, CgCol* st,
                           int* nactive, cudaStream_t s) {
    k_cg_init<<<S, 256, 0, s>>>(prz, nrz, prr, nrr, tol, st, nactive);
    return cudaGetLastError();
}
// x_theta += d (d: [S][n^3]) for columns whose CG ran
template <typename T>
__global__ void __launch_bounds__(256) k_cg_add(int64_t n3, double* __restrict__ x, const T* __restrict__ d,
                                                const CgCol* __restrict__ st) {
    const int s = blockIdx.y;
    if (st[s].iters == 0) return;
    double* xs = x + (int64_t)s * 4 * n3 + 3 * n3;
    const T* ds = d + (int64_t)s * n3;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n3; e += (int64_t)gridDim.x * blockDim.x)
        xs[e] += (double)ds[e];
}

template <typename T>
cudaError_t launch_cg_add(int64_t n3, int S, double* x, const T* d, const CgCol* st, cudaStream_t s) {
    int64_t b = (n3 + 1023) / 1024;
    if (b > 2048) b = 2048;
    k_cg_add<T><<<dim3((unsigned)(b < 1 ? 1 : b), S), 256, 0, s>>>(n3, x, d, st);
    return cudaGetLastError();
}

cudaError_t launch_cg_set_active(int S, const int* mask, CgCol* st, cudaStream_t s) {
    k_cg_set_active<<<(S + 127) / 128, 128, 0, s>>>(S, mask, st);
    return cudaGetLastError();
}

#define SPDE_SCHUR_INST(T)                                                                                          \
    template int launch_schur_apply<T>(int, double, int, const T*, T*, const T*, T*, double*, const CgCol*,             \
                                       cudaStream_t);                                                               \
    template int launch_cg_xr<T>(int64_t, int, T*, T*, const T*, const T*, double*, const CgCol*, cudaStream_t);   \
    template cudaError_t launch_cg_p<T>(int64_t, int, T*, const T*, const CgCol*, cudaStream_t);                   \
    template int launch_cg_rhs<T>(int64_t, int, const T*, T*, double*, const CgCol*, cudaStream_t);                \
    template cudaError_t launch_cg_add<T>(int64_t, int, double*, const T*, const CgCol*, cudaStream_t);
SPDE_SCHUR_INST(float)
SPDE_SCHUR_INST(double)

}  // namespace spde
