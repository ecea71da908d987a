// K1: white noise f = W^{1/2} xi (Sec. 4.2).  One thread per cell pair.
//
// xi ~ N(0, I) from Philox4x32-10 (key = seed, counter = (pair, tag 0,
// sample)) through 53-bit uniforms and the Box-Muller transform in FP64.
#include "device.cuh"
#include "internal.h"

namespace spde {

__global__ void __launch_bounds__(256) k_noise(int64_t ncells, int64_t npairs, uint32_t k0, uint32_t k1,
                                               uint64_t first, double scale, double* __restrict__ out,
                                               int64_t col_stride) {
    const int s = blockIdx.y;
    const uint64_t sample = first + (uint64_t)s;
    double* o = out + (int64_t)s * col_stride;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const U4 w = philox4x32_10(U4{(uint32_t)p, 0u, (uint32_t)sample, (uint32_t)(sample >> 32)}, k0, k1);
        const uint64_t a = ((((uint64_t)w.x) << 32) | w.y) >> 11;
        const uint64_t b = ((((uint64_t)w.z) << 32) | w.w) >> 11;
        const double u1 = ((double)a + 1.0) * 0x1.0p-53;  // (0, 1]
        const double u2 = (double)b * 0x1.0p-53;          // [0, 1)
        const double r = sqrt(-2.0 * log(u1));
        double sv, cv;
        sincospi(2.0 * u2, &sv, &cv);
        const int64_t c = 2 * p;
        o[c] = scale * r * cv;
        if (c + 1 < ncells) o[c + 1] = scale * r * sv;
    }
}

__global__ void __launch_bounds__(256) k_noise_words(int64_t npairs, uint32_t k0, uint32_t k1, uint64_t sample,
                                                     uint32_t* __restrict__ out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npairs; p += (int64_t)gridDim.x * blockDim.x) {
        const U4 w = philox4x32_10(U4{(uint32_t)p, 0u, (uint32_t)sample, (uint32_t)(sample >> 32)}, k0, k1);
        out[4 * p] = w.x;
        out[4 * p + 1] = w.y;
        out[4 * p + 2] = w.z;
        out[4 * p + 3] = w.w;
    }
}

cudaError_t launch_noise_words(int64_t npairs, uint64_t seed, uint64_t sample, uint32_t* out, cudaStream_t st) {
    int64_t blocks = (npairs + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) return cudaSuccess;
    k_noise_words<<<(unsigned)blocks, 256, 0, st>>>(npairs, (uint32_t)seed, (uint32_t)(seed >> 32), sample, out);
    return cudaGetLastError();
}

cudaError_t launch_noise(int64_t ncells, int S, uint64_t seed, uint64_t first, double scale, double* out,
                         int64_t col_stride, cudaStream_t st) {
    if (ncells <= 0 || S <= 0) return cudaSuccess;
    const int64_t npairs = (ncells + 1) / 2;
    int64_t blocks = (npairs + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    dim3 grid((unsigned)blocks, (unsigned)S);
    k_noise<<<grid, 256, 0, st>>>(ncells, npairs, (uint32_t)seed, (uint32_t)(seed >> 32), first, scale, out,
                                  col_stride);
    return cudaGetLastError();
}

// Per-column parameters (serving: every slot of a batch has its own request):
// column s draws sample[s] under key seed[s], scaled by scale[s]; columns with
// mask[s] == 0 are left untouched.
__global__ void __launch_bounds__(256) k_noise_cols(int64_t ncells, int64_t npairs, const uint64_t* __restrict__ seed,
                                                    const uint64_t* __restrict__ sample, const double* __restrict__ scale,
                                                    const int* __restrict__ mask, double* __restrict__ out,
                                                    int64_t col_stride) {
    const int s = blockIdx.y;
    if (!mask[s]) return;
    const uint64_t sd = seed[s], sm = sample[s];
    const uint32_t k0 = (uint32_t)sd, k1 = (uint32_t)(sd >> 32);
    const double sc = scale[s];
    double* o = out + (int64_t)s * col_stride;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npairs; p += (int64_t)gridDim.x * blockDim.x) {
        const U4 w = philox4x32_10(U4{(uint32_t)p, 0u, (uint32_t)sm, (uint32_t)(sm >> 32)}, k0, k1);
        const uint64_t a = ((((uint64_t)w.x) << 32) | w.y) >> 11;
        const uint64_t b = ((((uint64_t)w.z) << 32) | w.w) >> 11;
        const double u1 = ((double)a + 1.0) * 0x1.0p-53;
        const double u2 = (double)b * 0x1.0p-53;
        const double r = sqrt(-2.0 * log(u1));
        double sv, cv;
        sincospi(2.0 * u2, &sv, &cv);
        const int64_t c = 2 * p;
        o[c] = sc * r * cv;
        if (c + 1 < ncells) o[c + 1] = sc * r * sv;
    }
}

cudaError_t launch_noise_cols(int64_t ncells, int S, const uint64_t* seed, const uint64_t* sample, const double* scale,
                              const int* mask, double* out, int64_t col_stride, cudaStream_t st) {
    if (ncells <= 0 || S <= 0) return cudaSuccess;
    const int64_t npairs = (ncells + 1) / 2;
    int64_t blocks = (npairs + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    dim3 grid((unsigned)blocks, (unsigned)S);
    k_noise_cols<<<grid, 256, 0, st>>>(ncells, npairs, seed, sample, scale, mask, out, col_stride);
    return cudaGetLastError();
}

}  // namespace spde
