// Device helpers shared by the sampler's kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

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
// valid in the block's first thread (linear id 0).
// ---------------------------------------------------------------------------
template <int BLOCK>
__device__ __forceinline__ double block_sum(double v, double* smem /* >= BLOCK/32 */) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int lane = tid & 31, warp = tid >> 5;
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (tid < 32) {
        s = (tid < BLOCK / 32) ? smem[tid] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    __syncthreads();
    return s;
}

// Block sum of per-thread partials of the element type: FP32 partials are
// summed in FP32 within a warp (fixed shuffle tree) and the warps' sums in
// FP64; FP64 partials go through block_sum.  Deterministic for a fixed block.
template <int BLOCK, typename T>
__device__ __forceinline__ double block_sum_t(T v, double* smem /* >= BLOCK/32 */) {
    if constexpr (sizeof(T) == 8) {
        return block_sum<BLOCK>((double)v, smem);
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
        const int lane = tid & 31, warp = tid >> 5;
        if (lane == 0) smem[warp] = (double)v;
        __syncthreads();
        double s = 0.0;
        if (tid < 32) {
            s = (tid < BLOCK / 32) ? smem[tid] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        }
        __syncthreads();
        return s;
    }
}

// number of existing neighbours of cell i along one axis of length n
__device__ __forceinline__ int nb_count1(int i, int n) { return (i > 0) + (i < n - 1); }

// ---------------------------------------------------------------------------
// Four consecutive cells along x (i0 .. i0+3, i0 a multiple of 4) of the
// scaled mixed operator (Eq. linsys_blocks after the symmetric scaling by
// h^{-3/2} on fluxes and h^{-1/2} on cells), with 32-bit indices (extents are
// powers of two and a grid has at most 2^30 cells).  Center values come in as
// 16-byte vector loads; the x-neighbours outside the quad as two scalars.
// Wall fluxes (i = nx-1 for ux, j = ny-1 for uy, k = nz-1 for uz) are
// essential zeros, masked by index and never read.
// ---------------------------------------------------------------------------
template <typename T>
struct V4 {
    T v[4];
};

template <typename T>
__device__ __forceinline__ V4<T> ld4(const T* p) {
    V4<T> r;
    if constexpr (sizeof(T) == 4) {
        const float4 f = *reinterpret_cast<const float4*>(p);
        r.v[0] = f.x;
        r.v[1] = f.y;
        r.v[2] = f.z;
        r.v[3] = f.w;
    } else {
        const double2 a = reinterpret_cast<const double2*>(p)[0];
        const double2 b = reinterpret_cast<const double2*>(p)[1];
        r.v[0] = a.x;
        r.v[1] = a.y;
        r.v[2] = b.x;
        r.v[3] = b.y;
    }
    return r;
}

template <typename T>
__device__ __forceinline__ void st4(T* p, const V4<T>& r) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
    } else {
        reinterpret_cast<double2*>(p)[0] = make_double2(r.v[0], r.v[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(r.v[2], r.v[3]);
    }
}

template <typename T>
__device__ __forceinline__ V4<T> zero4() {
    V4<T> r;
#pragma unroll
    for (int e = 0; e < 4; ++e) r.v[e] = T(0);
    return r;
}

// quad index q of a grid (nx >= 4) -> (i0, j, k), c = i0 + nx (j + ny k)
struct QuadPos {
    int i0, j, k, c;
};
__device__ __forceinline__ QuadPos quad_pos(int q, const Grid3& g) {
    const int lq = g.lx - 2;  // quads per row = nx / 4
    QuadPos p;
    p.i0 = (q & ((1 << lq) - 1)) << 2;
    p.j = (q >> lq) & (g.ny - 1);
    p.k = q >> (lq + g.ly);
    p.c = p.i0 + ((p.j + (p.k << g.ly)) << g.lx);
    return p;
}

// y = A x on the quad; xs points at the sample's ux block (blocks nx ny nz apart)
template <typename T, typename S>
__device__ __forceinline__ void apply_quad(const T* __restrict__ xs, const Grid3& g, const QuadPos& p, S kh2,
                                           S yu[4], S yv[4], S yw[4], S yt[4]) {
    const int n3 = 1 << (g.lx + g.ly + g.lz);
    const int n = g.nx;
    const int sy = g.nx, sz = g.nx << g.ly;
    const T* ux = xs;
    const T* uy = xs + n3;
    const T* uz = xs + 2 * n3;
    const T* th = xs + 3 * n3;
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
    const S uxL = (p.i0 > 0) ? (S)ux[c - 1] : S(0);
    const S uxR = (p.i0 + 4 < n - 1) ? (S)ux[c + 4] : S(0);
    const S thR = (p.i0 + 4 < n) ? (S)th[c + 4] : S(0);
    const S a6 = S(1) / S(6), a23 = S(2) / S(3);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int i = p.i0 + e;
        const S t0 = (S)th4.v[e];
        const S ux0 = (i < n - 1) ? (S)ux4.v[e] : S(0);
        const S uxm = (e > 0) ? ((i - 1 < n - 1) ? (S)ux4.v[e - 1] : S(0)) : uxL;
        const S uxp = (e < 3) ? ((i + 1 < n - 1) ? (S)ux4.v[e + 1] : S(0)) : uxR;
        const S thx = (e < 3) ? (S)th4.v[e + 1] : thR;
        const S uy0 = jh ? (S)uy4.v[e] : S(0);
        const S uz0 = kh ? (S)uz4.v[e] : S(0);
        const S uym = (S)uyM.v[e], uzm = (S)uzM.v[e];
        yu[e] = (i < n - 1) ? a23 * ux0 + a6 * (uxm + uxp) + (t0 - thx) : S(0);
        yv[e] = jh ? a23 * uy0 + a6 * (uym + (S)uyP.v[e]) + (t0 - (S)thY.v[e]) : S(0);
        yw[e] = kh ? a23 * uz0 + a6 * (uzm + (S)uzP.v[e]) + (t0 - (S)thZ.v[e]) : S(0);
        yt[e] = (ux0 - uxm) + (uy0 - uym) + (uz0 - uzm) - kh2 * t0;
    }
}

__device__ __forceinline__ int ilog2(int n) { return 31 - __clz(n); }

}  // namespace spde
