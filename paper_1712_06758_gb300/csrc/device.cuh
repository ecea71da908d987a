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

// ---------------------------------------------------------------------------
// Four consecutive cells along x (i0 .. i0+3, i0 a multiple of 4) of the
// scaled mixed operator, with 32-bit indices (n a power of two <= 1024, so
// c < 2^30).  Center values come in as 16-byte vector loads; the x-neighbours
// outside the quad as two scalars.  Wall fluxes are masked by index.
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

// quad index q of an n^3 grid -> (i0, j, k), c = i0 + n (j + n k)
struct QuadPos {
    int i0, j, k, c;
};
__device__ __forceinline__ QuadPos quad_pos(int q, int logn) {
    const int lq = logn - 2;  // quads per row = n / 4
    QuadPos p;
    p.i0 = (q & ((1 << lq) - 1)) << 2;
    p.j = (q >> lq) & ((1 << logn) - 1);
    p.k = q >> (lq + logn);
    p.c = p.i0 + ((p.j + (p.k << logn)) << logn);
    return p;
}

// y = A x on the quad; xs points at the sample's ux block (blocks n^3 apart)
template <typename T, typename S>
__device__ __forceinline__ void apply_quad(const T* __restrict__ xs, int n, int logn, const QuadPos& p, S kh2,
                                           S yu[4], S yv[4], S yw[4], S yt[4]) {
    const int n3 = 1 << (3 * logn);
    const int sy = n, sz = n << logn;
    const T* ux = xs;
    const T* uy = xs + n3;
    const T* uz = xs + 2 * n3;
    const T* th = xs + 3 * n3;
    const int c = p.c;
    const V4<T> ux4 = ld4(ux + c), uy4 = ld4(uy + c), uz4 = ld4(uz + c), th4 = ld4(th + c);
    const bool jl = p.j > 0, jh = p.j < n - 1, jhh = p.j + 1 < n - 1;
    const bool kl = p.k > 0, kh = p.k < n - 1, khh = p.k + 1 < n - 1;
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
