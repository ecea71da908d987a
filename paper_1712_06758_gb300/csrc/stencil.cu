// K2 / K5: the scaled mixed operator (Eq. linsys_blocks) and the FP64
// refinement residual.
//
// Layout of one sample: [ux | uy | uz | theta], each n^3, c = i + n (j + n k).
// ux[c] is the flux through the +x face of cell c; entries on the wall
// (i = n-1 for ux, j = n-1 for uy, k = n-1 for uz) are the essential zeros
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
__global__ void __launch_bounds__(256) k_apply(int n, T kh2, const T* __restrict__ x, T* __restrict__ y) {
    const int64_t n3 = (int64_t)n * n * n;
    const int64_t off = (int64_t)blockIdx.y * 4 * n3;
    const T* xs = x + off;
    T* ys = y + off;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n3; c += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(c % n), j = (int)((c / n) % n), k = (int)(c / ((int64_t)n * n));
        const Cell4<T> r = apply_cell<T, T>(xs, n3, n, i, j, k, c, kh2);
        ys[c] = r.ux;
        ys[n3 + c] = r.uy;
        ys[2 * n3 + c] = r.uz;
        ys[3 * n3 + c] = r.th;
    }
}

template <typename T>
cudaError_t launch_apply(int n, double kh2, int S, const T* x, T* y, cudaStream_t st) {
    const int64_t n3 = (int64_t)n * n * n;
    dim3 grid(stencil_blocks(n3), S);
    k_apply<T><<<grid, 256, 0, st>>>(n, (T)kh2, x, y);
    return cudaGetLastError();
}
template cudaError_t launch_apply<float>(int, double, int, const float*, float*, cudaStream_t);
template cudaError_t launch_apply<double>(int, double, int, const double*, double*, cudaStream_t);

// r = [0; F] - A x in FP64; optional float and double copies; partial r.r
__global__ void __launch_bounds__(256) k_residual64(int n, double kh2, const double* __restrict__ F, int64_t F_stride,
                                                    const double* __restrict__ x, float* __restrict__ r32,
                                                    double* __restrict__ r64, double* __restrict__ part,
                                                    const int* __restrict__ active) {
    __shared__ double red[8];
    const int s = blockIdx.y;
    if (active && !active[s]) return;
    const int64_t n3 = (int64_t)n * n * n;
    const int64_t off = (int64_t)s * 4 * n3;
    const double* xs = x + off;
    const double* Fs = F + (int64_t)s * F_stride;
    double acc = 0.0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n3; c += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(c % n), j = (int)((c / n) % n), k = (int)(c / ((int64_t)n * n));
        const Cell4<double> a = apply_cell<double, double>(xs, n3, n, i, j, k, c, kh2);
        const double ru = -a.ux, rv = -a.uy, rw = -a.uz, rt = Fs[c] - a.th;
        acc += ru * ru + rv * rv + rw * rw + rt * rt;
        if (r32) {
            float* o = r32 + off;
            o[c] = (float)ru;
            o[n3 + c] = (float)rv;
            o[2 * n3 + c] = (float)rw;
            o[3 * n3 + c] = (float)rt;
        }
        if (r64) {
            double* o = r64 + off;
            o[c] = ru;
            o[n3 + c] = rv;
            o[2 * n3 + c] = rw;
            o[3 * n3 + c] = rt;
        }
    }
    const double t = block_sum<256>(acc, red);
    if (threadIdx.x == 0) part[(int64_t)s * kMaxPartials + blockIdx.x] = t;
}

int launch_residual64(int n, double kh2, int S, const double* F, int64_t F_stride, const double* x, float* r32,
                      double* r64, double* part, const int* active, cudaStream_t st) {
    const int64_t n3 = (int64_t)n * n * n;
    const int nb = stencil_blocks(n3);
    dim3 grid(nb, S);
    k_residual64<<<grid, 256, 0, st>>>(n, kh2, F, F_stride, x, r32, r64, part, active);
    return nb;
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

}  // namespace spde
