// Device helpers shared by the sampler's kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace spde {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 4 x 32-bit counter, 2 x 32-bit key,
// ten rounds; each round multiplies counter words 0 and 2 by two fixed odd
// constants, swaps in the high halves xor-ed with words 1/3 and the key, and
// the key advances by a Weyl step between rounds.
// ---------------------------------------------------------------------------
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
    const uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    const uint32_t kWeylA = 0x9E3779B9u, kWeylB = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hiA = __umulhi(kMulA, c.x), loA = kMulA * c.x;
        const uint32_t hiB = __umulhi(kMulB, c.z), loB = kMulB * c.z;
        c = U4{hiB ^ c.y ^ k0, loB, hiA ^ c.w ^ k1, loA};
        k0 += kWeylA;
        k1 += kWeylB;
    }
    return c;
}

// ---------------------------------------------------------------------------
// Deterministic block reduction of a double (fixed shape: warp shuffles then
// one pass over the warp sums).  All threads must call it; the result is
// valid in thread 0.
// ---------------------------------------------------------------------------
template <int BLOCK>
__device__ __forceinline__ double block_sum(double v, double* smem /* >= BLOCK/32 */) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (threadIdx.x < BLOCK / 32) ? smem[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    return s;
}

// number of existing neighbours of cell i along one axis of length n
__device__ __forceinline__ int nb_count1(int i, int n) { return (i > 0) + (i < n - 1); }

// ---------------------------------------------------------------------------
// The scaled mixed operator at one cell (Eq. linsys_blocks after the symmetric
// scaling by h^{-3/2} on fluxes and h^{-1/2} on cells).  xs points at the
// sample's ux block; the four blocks are n^3 apart.  Wall fluxes (i = n-1
// for ux, ...) are essential zeros and are never read.
// ---------------------------------------------------------------------------
template <typename S>
struct Cell4 {
    S ux, uy, uz, th;
};

template <typename T, typename S>
__device__ __forceinline__ Cell4<S> apply_cell(const T* __restrict__ xs, int64_t n3, int n, int i, int j, int k,
                                               int64_t c, S kh2) {
    const T* ux = xs;
    const T* uy = xs + n3;
    const T* uz = xs + 2 * n3;
    const T* th = xs + 3 * n3;
    const int64_t sy = n, sz = (int64_t)n * n;
    const S zero = S(0);
    const S t0 = (S)th[c];
    const S ux0 = (i < n - 1) ? (S)ux[c] : zero;
    const S uy0 = (j < n - 1) ? (S)uy[c] : zero;
    const S uz0 = (k < n - 1) ? (S)uz[c] : zero;
    const S uxm = (i > 0) ? (S)ux[c - 1] : zero;
    const S uym = (j > 0) ? (S)uy[c - sy] : zero;
    const S uzm = (k > 0) ? (S)uz[c - sz] : zero;
    const S a6 = S(1) / S(6), a23 = S(2) / S(3);
    Cell4<S> y;
    y.ux = (i < n - 1) ? a23 * ux0 + a6 * (uxm + ((i + 1 < n - 1) ? (S)ux[c + 1] : zero)) + (t0 - (S)th[c + 1]) : zero;
    y.uy = (j < n - 1) ? a23 * uy0 + a6 * (uym + ((j + 1 < n - 1) ? (S)uy[c + sy] : zero)) + (t0 - (S)th[c + sy])
                       : zero;
    y.uz = (k < n - 1) ? a23 * uz0 + a6 * (uzm + ((k + 1 < n - 1) ? (S)uz[c + sz] : zero)) + (t0 - (S)th[c + sz])
                       : zero;
    y.th = (ux0 - uxm) + (uy0 - uym) + (uz0 - uzm) - kh2 * t0;
    return y;
}

}  // namespace spde
