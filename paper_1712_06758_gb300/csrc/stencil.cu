// K2 / K5: the scaled mixed operator (Eq. linsys_blocks) and the FP64
// refinement residual.
//
// Layout of one sample: [ux | uy | uz | theta], each nx ny nz long,
// c = i + nx (j + ny k).  ux[c] is the flux through the +x face of cell c;
// entries on the wall (i = nx-1 for ux, j = ny-1 for uy, k = nz-1 for uz) are
// the essential zeros
// u.n = 0 and are never read as unknowns.  Scaled operator:
//   y_ux = 1/6 ux[i-1] + 2/3 ux[i] + 1/6 ux[i+1] + th[i] - th[i+1]
//   y_th = sum_axes (u[c] - u[c - e]) - (kappa h)^2 th[c]
#include "device.cuh"
#include "internal.h"

namespace spde {

static inline int stencil_blocks(int64_t n3) {
    int64_t b = (n3 + 255) / 256;
    if (b > 2048) b = 2048;
    return (int)(b < 1 ? 1 : b);
}

template <typename T>
__global__ void __launch_bounds__(256) k_apply(Grid3 g, T kh2, const T* __restrict__ x, T* __restrict__ y) {
    const int n3 = 1 << (g.lx + g.ly + g.lz);
    const int64_t off = (int64_t)blockIdx.y * 4 * n3;
    const T* xs = x + off;
    T* ys = y + off;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < (n3 >> 2); q += gridDim.x * blockDim.x) {
        const QuadPos p = quad_pos(q, g);
        V4<T> a, b, c, d;
        apply_quad<T, T>(xs, g, p, kh2, a.v, b.v, c.v, d.v);
        st4(ys + p.c, a);
        st4(ys + n3 + p.c, b);
        st4(ys + 2 * n3 + p.c, c);
        st4(ys + 3 * n3 + p.c, d);
    }
}

template <typename T>
cudaError_t launch_apply(const Grid3& g, double kh2, int S, const T* x, T* y, cudaStream_t st) {
    dim3 grid(stencil_blocks(g.cells() / 4), S);
    k_apply<T><<<grid, 256, 0, st>>>(g, (T)kh2, x, y);
    return cudaGetLastError();
}
template cudaError_t launch_apply<float>(const Grid3&, double, int, const float*, float*, cudaStream_t);
template cudaError_t launch_apply<double>(const Grid3&, double, int, const double*, double*, cudaStream_t);

// the residual of one quad: flux rows zero, cell row d, as float and/or double
__device__ __forceinline__ void residual_store(float* __restrict__ r32, double* __restrict__ r64, int64_t off, int n3,
                                               int c, const V4<double>& d) {
    if (r32) {
        float* o = r32 + off;
        const V4<float> z = zero4<float>();
        V4<float> fd;
#pragma unroll
        for (int e = 0; e < 4; ++e) fd.v[e] = (float)d.v[e];
        st4(o + c, z);
        st4(o + n3 + c, z);
        st4(o + 2 * n3 + c, z);
        st4(o + 3 * n3 + c, fd);
    }
    if (r64) {
        double* o = r64 + off;
        const V4<double> z = zero4<double>();
        st4(o + c, z);
        st4(o + n3 + c, z);
        st4(o + 2 * n3 + c, z);
        st4(o + 3 * n3 + c, d);
    }
}

// r = [0; F] - A x in FP64; optional float and double copies; partial r.r.
// Every caller forms the flux of x exactly from its cell field first
// (u = -T^{-1} D1^T theta by FP64 line solves, or x = 0), so the flux rows of
// r vanish up to the rounding of those solves: they are written as zeros and
// only the cell row  F - (D1 u - (kappa h)^2 theta)  is formed (the FP64
// arithmetic, the rate-limiting unit here, drops to a third).
// x is known to be zero (the first step of a cold start) when xzero is set or
// *zgate is 0: the cell row is then F itself, taken without reading x (the same
// bits: every term of A x is +0).
__global__ void __launch_bounds__(256) k_residual64(Grid3 g, double kh2, const double* __restrict__ F, int64_t F_stride,
                                                    const double* __restrict__ x, float* __restrict__ r32,
                                                    double* __restrict__ r64, double* __restrict__ part,
                                                    const int* __restrict__ active, const double* __restrict__ kh2c,
                                                    const double* __restrict__ kh2s, int xzero,
                                                    const int* __restrict__ zgate) {
    __shared__ double red[8];
    const int s = blockIdx.y;
    if (active && !active[s]) return;
    const bool zero = xzero || (zgate && *zgate == 0);
    const double kh2v = kh2s ? kh2s[s] : kh2;  // one (kappa h)^2 per column (serving lanes) or per call
    const int n3 = 1 << (g.lx + g.ly + g.lz);
    const int64_t off = (int64_t)s * 4 * n3;
    const double* xs = x + off;
    const double* ux = xs;
    const double* uy = xs + n3;
    const double* uz = xs + 2 * n3;
    const double* th = xs + 3 * n3;
    const double* Fs = F + (int64_t)s * F_stride;
    const int sy = g.nx, sz = g.nx << g.ly;
    double acc = 0.0;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < (n3 >> 2); q += gridDim.x * blockDim.x) {
        const QuadPos p = quad_pos(q, g);
        const int c = p.c;
        if (zero) {
            const V4<double> d = ld4(Fs + c);
#pragma unroll
            for (int e = 0; e < 4; ++e) acc += d.v[e] * d.v[e];
            residual_store(r32, r64, off, n3, c, d);
            continue;
        }
        const bool jl = p.j > 0, jh = p.j < g.ny - 1;
        const bool kl = p.k > 0, kh = p.k < g.nz - 1;
        const V4<double> ux4 = ld4(ux + c), uy4 = ld4(uy + c), uz4 = ld4(uz + c), th4 = ld4(th + c);
        const V4<double> uyM = jl ? ld4(uy + c - sy) : zero4<double>();
        const V4<double> uzM = kl ? ld4(uz + c - sz) : zero4<double>();
        const double uxL = (p.i0 > 0) ? ux[c - 1] : 0.0;
        const V4<double> f = ld4(Fs + c);
        V4<double> k4;  // (kappa h)^2 per cell: one value, or the level's field
        if (kh2c) k4 = ld4(kh2c + c);
        else
#pragma unroll
            for (int e = 0; e < 4; ++e) k4.v[e] = kh2v;
        V4<double> d;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i = p.i0 + e;
            const double ux0 = (i < g.nx - 1) ? ux4.v[e] : 0.0;
            const double uxm = (e > 0) ? ux4.v[e - 1] : uxL;
            const double uy0 = jh ? uy4.v[e] : 0.0;
            const double uz0 = kh ? uz4.v[e] : 0.0;
            const double yt = (ux0 - uxm) + (uy0 - uyM.v[e]) + (uz0 - uzM.v[e]) - k4.v[e] * th4.v[e];
            d.v[e] = f.v[e] - yt;
            acc += d.v[e] * d.v[e];
        }
        residual_store(r32, r64, off, n3, c, d);
    }
    const double t = block_sum<256>(acc, red);
    if (threadIdx.x == 0) part[(int64_t)s * kMaxPartials + blockIdx.x] = t;
}

int launch_residual64(const Grid3& g, double kh2, int S, const double* F, int64_t F_stride, const double* x,
                      float* r32, double* r64, double* part, const int* active, cudaStream_t st, const double* kh2c,
                      const double* kh2s, int xzero, const int* zgate) {
    const int nb = stencil_blocks(g.cells() / 4);
    dim3 grid(nb, S);
    k_residual64<<<grid, 256, 0, st>>>(g, kh2, F, F_stride, x, r32, r64, part, active, kh2c, kh2s, xzero, zgate);
    return nb;
}

// a_c = mean of the children of coarse cell c: the fine grid gf, the coarse grid
// gf.coarser() (2 children along every axis that is coarsened, 1 along an axis
// of extent 1)
__global__ void __launch_bounds__(256) k_restrict_mean(Grid3 gf, const double* __restrict__ af, double* __restrict__ ac) {
    const Grid3 gc = gf.coarser();
    const int64_t n3 = gc.cells();
    const int dx = gf.nx > 1 ? 2 : 1, dy = gf.ny > 1 ? 2 : 1, dz = gf.nz > 1 ? 2 : 1;
    const double inv = 1.0 / (double)(dx * dy * dz);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n3; e += (int64_t)gridDim.x * blockDim.x) {
        const int I = (int)(e & (gc.nx - 1)), J = (int)((e >> gc.lx) & (gc.ny - 1)), K = (int)(e >> (gc.lx + gc.ly));
        double sum = 0.0;
        for (int dk = 0; dk < dz; ++dk)
            for (int dj = 0; dj < dy; ++dj)
                for (int di = 0; di < dx; ++di)
                    sum += af[(dx * I + di) + (int64_t)gf.nx * ((dy * J + dj) + (int64_t)gf.ny * (dz * K + dk))];
        ac[e] = inv * sum;
    }
}

cudaError_t launch_restrict_mean(const Grid3& gf, const double* af, double* ac, cudaStream_t st) {
    const int64_t nc3 = gf.coarser().cells();
    int64_t b = (nc3 + 255) / 256;
    if (b > 4096) b = 4096;
    k_restrict_mean<<<(unsigned)(b < 1 ? 1 : b), 256, 0, st>>>(gf, af, ac);
    return cudaGetLastError();
}

// D = s (a q + c k) per cell of a level (s, q: the level's Laplacian weight and
// mass-to-Laplacian factor, 2^l and 4^l on a cube), FP64 and FP32
__global__ void __launch_bounds__(256) k_level_diag(Grid3 g, double s, double q, double c, const double* __restrict__ a,
                                                    double* __restrict__ D64, float* __restrict__ D32) {
    const int64_t n3 = g.cells();
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n3; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e & (g.nx - 1)), j = (int)((e >> g.lx) & (g.ny - 1)), k = (int)(e >> (g.lx + g.ly));
        const int kc = nb_count1(i, g.nx) + nb_count1(j, g.ny) + nb_count1(k, g.nz);
        const double d = s * (a[e] * q + c * kc);
        D64[e] = d;
        D32[e] = (float)d;
    }
}

cudaError_t launch_level_diag(const Grid3& g, double s, double q, double c, const double* a, double* D64, float* D32,
                              cudaStream_t st) {
    const int64_t n3 = g.cells();
    int64_t b = (n3 + 255) / 256;
    if (b > 4096) b = 4096;
    k_level_diag<<<(unsigned)(b < 1 ? 1 : b), 256, 0, st>>>(g, s, q, c, a, D64, D32);
    return cudaGetLastError();
}

// F[s][e] *= c[e]: the per-cell noise factor -g(x) h of a level with fields
__global__ void __launch_bounds__(256) k_scale_cells(int64_t n3, double* __restrict__ F, int64_t stride,
                                                     const double* __restrict__ c) {
    double* Fs = F + (int64_t)blockIdx.y * stride;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n3; e += (int64_t)gridDim.x * blockDim.x)
        Fs[e] *= c[e];
}

cudaError_t launch_scale_cells(int64_t n3, int S, double* F, int64_t stride, const double* c, cudaStream_t st) {
    int64_t b = (n3 + 1023) / 1024;
    if (b > 4096) b = 4096;
    dim3 grid((unsigned)(b < 1 ? 1 : b), S);
    k_scale_cells<<<grid, 256, 0, st>>>(n3, F, stride, c);
    return cudaGetLastError();
}

// per-cell coefficients of a level with fields: (kappa h)^2 in FP64 and FP32, and
// the noise factor -g h with g = sigma sqrt(8 pi kappa) (the nu = 1/2, d = 3 normaliser)
__global__ void __launch_bounds__(256) k_field_coefs(int64_t n3, double h, const double* __restrict__ kappa,
                                                     const double* __restrict__ sigma, double* __restrict__ kh2_64,
                                                     float* __restrict__ kh2_32, double* __restrict__ gh) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n3; e += (int64_t)gridDim.x * blockDim.x) {
        const double kh = kappa[e] * h;
        kh2_64[e] = kh * kh;
        kh2_32[e] = (float)(kh * kh);
        gh[e] = -sigma[e] * sqrt(8.0 * 3.14159265358979323846 * kappa[e]) * h;
    }
}

cudaError_t launch_field_coefs(int64_t n3, double h, const double* kappa, const double* sigma, double* kh2_64,
                               float* kh2_32, double* gh, cudaStream_t st) {
    int64_t b = (n3 + 1023) / 1024;
    if (b > 4096) b = 4096;
    k_field_coefs<<<(unsigned)(b < 1 ? 1 : b), 256, 0, st>>>(n3, h, kappa, sigma, kh2_64, kh2_32, gh);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_add_correction(int64_t nelem, double* __restrict__ x,
                                                        const float* __restrict__ d, const int* __restrict__ active) {
    const int s = blockIdx.y;
    if (active && !active[s]) return;
    const int64_t off = (int64_t)s * nelem;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nelem; e += (int64_t)gridDim.x * blockDim.x)
        x[off + e] += (double)d[off + e];
}

cudaError_t launch_add_correction(int64_t nelem, int S, double* x, const float* d, const int* active,
                                  cudaStream_t st) {
    int64_t b = (nelem + 255) / 256;
    if (b > 4096) b = 4096;
    dim3 grid((unsigned)b, S);
    k_add_correction<<<grid, 256, 0, st>>>(nelem, x, d, active);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_sumsq(int64_t nelem, const double* __restrict__ a, int64_t stride,
                                               double* __restrict__ part) {
    __shared__ double red[8];
    const int s = blockIdx.y;
    const double* as = a + (int64_t)s * stride;
    double acc = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nelem; e += (int64_t)gridDim.x * blockDim.x)
        acc += as[e] * as[e];
    const double t = block_sum<256>(acc, red);
    if (threadIdx.x == 0) part[(int64_t)s * kMaxPartials + blockIdx.x] = t;
}

int launch_sumsq(int64_t nelem, int S, const double* a, int64_t stride, double* part, cudaStream_t st) {
    int64_t b = (nelem + 255) / 256;
    if (b > 2048) b = 2048;
    if (b < 1) b = 1;
    dim3 grid((unsigned)b, S);
    k_sumsq<<<grid, 256, 0, st>>>(nelem, a, stride, part);
    return (int)b;
}

__global__ void __launch_bounds__(256) k_reduce(const double* __restrict__ part, int nblk, double* __restrict__ out) {
    __shared__ double red[8];
    const int s = blockIdx.x;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += part[(int64_t)s * kMaxPartials + b];
    const double t = block_sum<256>(acc, red);
    if (threadIdx.x == 0) out[s] = t;
}

cudaError_t launch_reduce(int S, const double* part, int nblk, double* out, cudaStream_t st) {
    k_reduce<<<S, 256, 0, st>>>(part, nblk, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exact flux of a cell field: u = -T^{-1} D1^T theta, i.e. the first block row
// of the scaled system (T u + D1^T theta = 0) solved line by line.  T is
// tridiag(1/6, 2/3, 1/6) on the m-1 interior faces of a line of m cells; the
// wall face (index m-1 in the line) stays 0.  Thomas elimination with the
// factors c'_f (super-diagonal after elimination) and 1 / pivot_f, which
// depend only on f, not on the line's length: tri[0 .. tn-2] = c'_f and
// tri[tn-1 .. 2tn-3] = 1 / pivot_f for the longest extent tn, computed on the
// host, serve every axis.  One thread per line; consecutive threads take
// neighbouring lines.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_flux_lines(Grid3 g, int tn, int axis, const double* __restrict__ x,
                                                    double* __restrict__ xu, int64_t col_stride,
                                                    const double* __restrict__ tri, const int* __restrict__ gate) {
    if (gate && *gate == 0) return;
    const int L = blockIdx.x * blockDim.x + threadIdx.x;
    const int n3 = 1 << (g.lx + g.ly + g.lz);
    const int m = g.ext(axis);
    if (L >= (n3 >> (axis == 0 ? g.lx : (axis == 1 ? g.ly : g.lz)))) return;
    const int64_t off = (int64_t)blockIdx.y * col_stride;
    const double* th = x + off + 3 * (int64_t)n3;
    double* u = xu + off + (int64_t)axis * n3;
    int base, stride;
    if (axis == 0) {  // lines along x, indexed by (j, k)
        base = L << g.lx;
        stride = 1;
    } else if (axis == 1) {  // along y, indexed by (i, k)
        base = (L & (g.nx - 1)) + ((L >> g.lx) << (g.lx + g.ly));
        stride = g.nx;
    } else {  // along z, indexed by (i, j)
        base = L;
        stride = g.nx << g.ly;
    }
    const double* cp = tri;
    const double* inv = tri + (tn - 1);
    const double a = 1.0 / 6.0;
    // forward elimination of T u = -(theta_f - theta_{f+1}) = theta_{f+1} - theta_f
    double prev = 0.0, tcur = th[base];
    for (int f = 0; f < m - 1; ++f) {
        const double tnext = th[base + (f + 1) * stride];
        const double dp = ((tnext - tcur) - a * prev) * inv[f];
        u[base + f * stride] = dp;
        prev = dp;
        tcur = tnext;
    }
    u[base + (m - 1) * stride] = 0.0;
    // back substitution
    double xn = prev;
    for (int f = m - 3; f >= 0; --f) {
        const double xf = u[base + f * stride] - cp[f] * xn;
        u[base + f * stride] = xf;
        xn = xf;
    }
}

// Lines along x are contiguous rows: a CTA stages row_lines consecutive rows
// of theta in shared memory (coalesced), each thread solves one row in place
// there, and the tile goes back to the ux block coalesced.
constexpr int kRowTileElems = 8192;  // doubles of one staged tile (64 KB)
static inline int row_lines(const Grid3& g) {
    const int n = g.nx;
    const int rows = 1 << (g.ly + g.lz);
    const int lr = n >= kRowTileElems / 32 ? kRowTileElems / n : 32;
    return lr < rows ? lr : rows;  // a 4 x 4 x 4 grid has only 16 rows
}

__global__ void __launch_bounds__(128) k_flux_rows(Grid3 g, int tn, int lines_per_cta, const double* __restrict__ x,
                                                   double* __restrict__ xu, int64_t col_stride,
                                                   const double* __restrict__ tri, const int* __restrict__ gate) {
    extern __shared__ double srow[];  // lines_per_cta rows of nx + 1 (padded against bank conflicts)
    if (gate && *gate == 0) return;
    const int n = g.nx, logn = g.lx;
    const int64_t off = (int64_t)blockIdx.y * col_stride;
    const int n3 = 1 << (g.lx + g.ly + g.lz);
    const int64_t row0 = (int64_t)blockIdx.x * lines_per_cta;  // first (j, k) row of the tile
    const double* th = x + off + 3 * (int64_t)n3 + (row0 << logn);
    double* u = xu + off + (row0 << logn);
    const int tile = lines_per_cta << logn;
    for (int e = threadIdx.x; e < tile; e += blockDim.x) srow[(e >> logn) * (n + 1) + (e & (n - 1))] = th[e];
    __syncthreads();
    const double* cp = tri;
    const double* inv = tri + (tn - 1);
    const double a = 1.0 / 6.0;
    for (int L = threadIdx.x; L < lines_per_cta; L += blockDim.x) {
        double* r = srow + L * (n + 1);
        // forward elimination of T u = theta_{f+1} - theta_f, in place (theta_f is dead once dp_f exists)
        double prev = 0.0, tcur = r[0];
        for (int f = 0; f < n - 1; ++f) {
            const double tnext = r[f + 1];
            const double dp = ((tnext - tcur) - a * prev) * inv[f];
            r[f] = dp;
            prev = dp;
            tcur = tnext;
        }
        r[n - 1] = 0.0;  // wall flux
        double xn = prev;
        for (int f = n - 3; f >= 0; --f) {
            const double xf = r[f] - cp[f] * xn;
            r[f] = xf;
            xn = xf;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < tile; e += blockDim.x) u[e] = srow[(e >> logn) * (n + 1) + (e & (n - 1))];
}

static cudaError_t flux_rows_attr() {
    static const cudaError_t e = cudaFuncSetAttribute(k_flux_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (kRowTileElems + 64) * (int)sizeof(double));
    return e;
}

cudaError_t flux_prepare() { return flux_rows_attr(); }

cudaError_t launch_flux_from_theta(const Grid3& g, int S, double* x, int64_t col_stride, const double* tri,
                                   cudaStream_t st, const int* gate) {
    const int tn = g.maxn();
    const int rows = 1 << (g.ly + g.lz);
    const int lr = row_lines(g);
    const cudaError_t ea = flux_rows_attr();
    if (ea != cudaSuccess) return ea;
    dim3 grow(rows / lr, S);
    k_flux_rows<<<grow, 128, (size_t)lr * (g.nx + 1) * sizeof(double), st>>>(g, tn, lr, x, x, col_stride, tri, gate);
    for (int axis = 1; axis < 3; ++axis) {
        const int lines = (int)(g.cells() / g.ext(axis));
        dim3 grid((lines + 255) / 256, S);
        k_flux_lines<<<grid, 256, 0, st>>>(g, tn, axis, x, x, col_stride, tri, gate);
    }
    return cudaGetLastError();
}

// x_theta += d (d holds only the cell block, n^3 per column)
template <typename T>
__global__ void __launch_bounds__(256) k_add_theta(int64_t n3, double* __restrict__ x, const T* __restrict__ d,
                                                   const MinresCol* __restrict__ st) {
    const int s = blockIdx.y;
    if (st[s].iters == 0) return;
    double* xs = x + (int64_t)s * 4 * n3 + 3 * n3;
    const T* ds = d + (int64_t)s * n3;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n3; e += (int64_t)gridDim.x * blockDim.x)
        xs[e] += (double)ds[e];
}

template <typename T>
cudaError_t launch_add_theta(int64_t n3, int S, double* x, const T* d, const MinresCol* st_, cudaStream_t st) {
    int64_t b = (n3 + 1023) / 1024;
    if (b > 2048) b = 2048;
    dim3 grid((unsigned)(b < 1 ? 1 : b), S);
    k_add_theta<T><<<grid, 256, 0, st>>>(n3, x, d, st_);
    return cudaGetLastError();
}
template cudaError_t launch_add_theta<float>(int64_t, int, double*, const float*, const MinresCol*, cudaStream_t);
template cudaError_t launch_add_theta<double>(int64_t, int, double*, const double*, const MinresCol*, cudaStream_t);

// ---------------------------------------------------------------------------
// Two-level coupling (Sec. 6.2): the coarse white-noise right-hand side is the
// fine one summed over the 8 children of each coarse cell (P^T f; with
// f = W^{1/2} xi this has exactly the coarse covariance W_c).  In the scaled
// system (cell rows scaled by h^{-1/2}) that is F_c = (1/sqrt 2) sum F_f.
// ---------------------------------------------------------------------------
__global__ void k_restrict_rhs(Grid3 gc, const double* __restrict__ Ff, int64_t f_stride, double* __restrict__ Fc,
                               int64_t c_stride) {
    const int s = blockIdx.y;
    const int nfx = 2 * gc.nx, nfy = 2 * gc.ny;  // the fine grid is twice the coarse one along every axis
    const int64_t nc3 = gc.cells();
    const double* fs = Ff + (int64_t)s * f_stride;
    double* cs = Fc + (int64_t)s * c_stride;
    const double w = 0.70710678118654752440;  // 1 / sqrt(2)
    for (int64_t C = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; C < nc3; C += (int64_t)gridDim.x * blockDim.x) {
        const int I = (int)(C & (gc.nx - 1)), J = (int)((C >> gc.lx) & (gc.ny - 1)), K = (int)(C >> (gc.lx + gc.ly));
        double acc = 0.0;
        for (int dk = 0; dk < 2; ++dk)
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di)
                    acc += fs[(2 * I + di) + (int64_t)nfx * ((2 * J + dj) + (int64_t)nfy * (2 * K + dk))];
        cs[C] = w * acc;
    }
}

cudaError_t launch_restrict_rhs(const Grid3& gc, int S, const double* Ff, int64_t f_stride, double* Fc,
                                int64_t c_stride, cudaStream_t st) {
    const int64_t nc3 = gc.cells();
    int64_t b = (nc3 + 255) / 256;
    if (b > 4096) b = 4096;
    dim3 grid((unsigned)(b < 1 ? 1 : b), S);
    k_restrict_rhs<<<grid, 256, 0, st>>>(gc, Ff, f_stride, Fc, c_stride);
    return cudaGetLastError();
}

// Fine initial cell field = coarse field injected (piecewise-constant P of
// Sec. 6.1): physical theta_f = theta_c(parent), i.e. scaled
// theta~_f = theta~_c / sqrt 2 (cell scaling h^{1/2}, H = 2h).  Writes the
// cell block of xf (stride 4 x the fine cells); the flux blocks are recomputed later.
__global__ void k_inject_theta(Grid3 gc, const double* __restrict__ xc, int64_t c_stride, double* __restrict__ xf,
                               int64_t f_stride) {
    const int s = blockIdx.y;
    const int64_t nc3 = gc.cells(), nf3 = 8 * nc3;
    const int lfx = gc.lx + 1, lfy = gc.ly + 1;
    const double* tc = xc + (int64_t)s * c_stride + 3 * nc3;
    double* tf = xf + (int64_t)s * f_stride + 3 * nf3;
    const double w = 0.70710678118654752440;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nf3; c += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(c & ((1 << lfx) - 1)), j = (int)((c >> lfx) & ((1 << lfy) - 1)), k = (int)(c >> (lfx + lfy));
        tf[c] = w * tc[(i >> 1) + (int64_t)gc.nx * ((j >> 1) + (int64_t)gc.ny * (k >> 1))];
    }
}

cudaError_t launch_inject_theta(const Grid3& gc, int S, const double* xc, int64_t c_stride, double* xf,
                                int64_t f_stride, cudaStream_t st) {
    const int64_t nf3 = 8 * gc.cells();
    int64_t b = (nf3 + 255) / 256;
    if (b > 4096) b = 4096;
    dim3 grid((unsigned)b, S);
    k_inject_theta<<<grid, 256, 0, st>>>(gc, xc, c_stride, xf, f_stride);
    return cudaGetLastError();
}

}  // namespace spde
