// K7: L2 projection onto the tet mesh fused with the output map (Eq.
// proj_op: theta_h = W_h^{-1} G theta_bar = Pi theta_bar; lognormal
// k = exp(theta_h) after the projection, workflow figure of Sec. 6).
//
// Pi is CSR with rows = tets.  The grid fields of a batch are first
// transposed to thetaT[cell][sample] (FP32) so one CSR entry feeds all
// samples from one contiguous row; a warp computes one tet for 64 samples
// and a shared-memory tile turns the result into coalesced rows of
// out[sample][tet].
#include "device.cuh"
#include "internal.h"

namespace spde {

__global__ void k_transpose_theta(int64_t ncell, int S, const double* __restrict__ x, int64_t x_stride, double scale,
                                  float* __restrict__ thetaT) {
    __shared__ float tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32;
    const int s0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int s = s0 + r;
        const int64_t c = c0 + threadIdx.x;
        tile[r][threadIdx.x] = (s < S && c < ncell) ? (float)(scale * x[(int64_t)s * x_stride + c]) : 0.0f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t c = c0 + r;
        const int s = s0 + threadIdx.x;
        if (c < ncell && s < S) thetaT[c * S + s] = tile[threadIdx.x][r];
    }
}

cudaError_t launch_transpose_theta(int64_t ncell, int S, const double* x, int64_t x_stride, double scale,
                                   float* thetaT, cudaStream_t st) {
    dim3 grid((unsigned)((ncell + 31) / 32), (unsigned)((S + 31) / 32));
    k_transpose_theta<<<grid, dim3(32, 8), 0, st>>>(ncell, S, x, x_stride, scale, thetaT);
    return cudaGetLastError();
}

template <typename O>
__device__ __forceinline__ O out_map(float acc, int kind) {
    if (sizeof(O) == 8) return (O)(kind == 0 ? exp((double)acc) : (double)acc);
    return (O)(kind == 0 ? expf(acc) : acc);
}

// A CTA of 8 warps projects 32 tets, 4 per warp, for a chunk of up to 64
// samples: lane l holds samples 2l, 2l+1 of the chunk, so one pass over a
// tet's CSR row reads whole 256-byte rows of thetaT (one float2 per lane).
// The lanes first load up to 32 of the row's (pi, col) pairs together and
// hand them round by shuffles, so the row's thetaT gathers are independent
// and can be in flight at once; the sum still runs over the row in CSR
// order (the same fmaf sequence as the other projection kernels).  A
// shared-memory tile turns the 32 x 64 results into coalesced rows of
// out[sample][tet].
constexpr int kProjTets = 32, kProjChunk = 64;

template <typename O, int VEC>
__global__ void __launch_bounds__(256) k_project_rows(int64_t ntets, int S, const int64_t* __restrict__ rowptr,
                                                      const int32_t* __restrict__ col, const float* __restrict__ pi,
                                                      const float* __restrict__ thetaT, int kind, O* __restrict__ out) {
    __shared__ float tile[kProjChunk][kProjTets + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t t0 = (int64_t)blockIdx.x * kProjTets;
    for (int s0 = 0; s0 < S; s0 += kProjChunk) {
        const int sl = s0 + VEC * lane;  // this lane's first sample
        const bool on0 = sl < S, on1 = VEC == 2 && sl + 1 < S;
        for (int rr = 0; rr < 4; ++rr) {
            const int r = warp * 4 + rr;
            const int64_t t = t0 + r;
            float acc0 = 0.0f, acc1 = 0.0f, acc2 = 0.0f;  // acc2: the second sample of a VEC = 1 lane
            if (t < ntets) {
                const int64_t a = rowptr[t], b = rowptr[t + 1];
                for (int64_t base = a; base < b; base += 32) {
                    const int m = (b - base) < 32 ? (int)(b - base) : 32;
                    float wl = 0.0f;
                    int cl = 0;
                    if (lane < m) {
                        wl = pi[base + lane];
                        cl = col[base + lane];
                    }
#pragma unroll 8
                    for (int k = 0; k < m; ++k) {
                        const float w = __shfl_sync(0xffffffffu, wl, k);
                        const int64_t c = __shfl_sync(0xffffffffu, cl, k);
                        const float* row = thetaT + c * S;
                        if constexpr (VEC == 2) {
                            if (on1) {
                                const float2 v = *reinterpret_cast<const float2*>(row + sl);
                                acc0 = fmaf(w, v.x, acc0);
                                acc1 = fmaf(w, v.y, acc1);
                            } else if (on0) {
                                acc0 = fmaf(w, row[sl], acc0);
                            }
                        } else {
                            if (on0) acc0 = fmaf(w, row[sl], acc0);
                            if (sl + 32 < S && s0 + 32 + lane < S) acc2 = fmaf(w, row[s0 + 32 + lane], acc2);
                        }
                    }
                }
            }
            if constexpr (VEC == 2) {
                tile[2 * lane][r] = acc0;
                tile[2 * lane + 1][r] = acc1;
            } else {
                tile[lane][r] = acc0;
                tile[32 + lane][r] = acc2;
            }
        }
        __syncthreads();
        // rows out[s][t0 .. t0 + 31]
        for (int q = warp; q < kProjChunk; q += 8) {
            const int ss = s0 + q;
            const int64_t t = t0 + lane;
            if (ss < S && t < ntets) out[(int64_t)ss * ntets + t] = out_map<O>(tile[q][lane], kind);
        }
        __syncthreads();
    }
}

// S a multiple of 4: a half-warp per tet, a float4 of samples per lane (16 lanes
// cover a 64-sample chunk of a thetaT row), so one warp instruction gathers the
// rows of two tets.  Each half loads up to 16 of its row's (pi, col) pairs at
// once and hands them round by width-16 shuffles; the sum runs over the row in
// CSR order, as in the other projection kernels.
template <typename O>
__global__ void __launch_bounds__(256) k_project_quad(int64_t ntets, int S, const int64_t* __restrict__ rowptr,
                                                      const int32_t* __restrict__ col, const float* __restrict__ pi,
                                                      const float* __restrict__ thetaT, int kind, O* __restrict__ out) {
    __shared__ float tile[kProjChunk][kProjTets + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int half = lane >> 4, hl = lane & 15;
    const int64_t t0 = (int64_t)blockIdx.x * kProjTets;
    const int S4 = S >> 2;
    const float4* T4 = reinterpret_cast<const float4*>(thetaT);
    for (int s0 = 0; s0 < S; s0 += kProjChunk) {
        const int q = (s0 >> 2) + hl;  // this lane's float4 of the row
        const bool on = q < S4;
        for (int rr = 0; rr < 2; ++rr) {
            const int r = warp * 4 + rr * 2 + half;
            const int64_t t = t0 + r;
            int64_t a = 0, b = 0;
            if (t < ntets) {
                a = rowptr[t];
                b = rowptr[t + 1];
            }
            float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            for (int64_t base = a;; base += 16) {
                const int64_t left = b - base;
                const int mh = left <= 0 ? 0 : (left < 16 ? (int)left : 16);
                const int mo = __shfl_xor_sync(0xffffffffu, mh, 16);
                if (mh == 0 && mo == 0) break;  // both rows done (warp-uniform)
                float wl = 0.0f;
                int cl = 0;
                if (hl < mh) {
                    wl = pi[base + hl];
                    cl = col[base + hl];
                }
                const int mm = mh > mo ? mh : mo;
#pragma unroll 4
                for (int k = 0; k < mm; ++k) {
                    const float w = __shfl_sync(0xffffffffu, wl, k, 16);
                    const int c = __shfl_sync(0xffffffffu, cl, k, 16);
                    if (k < mh && on) {
                        const float4 v = T4[(int64_t)c * S4 + q];
                        acc.x = fmaf(w, v.x, acc.x);
                        acc.y = fmaf(w, v.y, acc.y);
                        acc.z = fmaf(w, v.z, acc.z);
                        acc.w = fmaf(w, v.w, acc.w);
                    }
                }
            }
            tile[4 * hl][r] = acc.x;
            tile[4 * hl + 1][r] = acc.y;
            tile[4 * hl + 2][r] = acc.z;
            tile[4 * hl + 3][r] = acc.w;
        }
        __syncthreads();
        for (int qq = warp; qq < kProjChunk; qq += 8) {
            const int ss = s0 + qq;
            const int64_t t = t0 + lane;
            if (ss < S && t < ntets) out[(int64_t)ss * ntets + t] = out_map<O>(tile[qq][lane], kind);
        }
        __syncthreads();
    }
}

// thread per tet, loop over the few samples
template <typename O>
__global__ void __launch_bounds__(256) k_project_thread(int64_t ntets, int S, const int64_t* __restrict__ rowptr,
                                                        const int32_t* __restrict__ col, const float* __restrict__ pi,
                                                        const float* __restrict__ thetaT, int kind, O* __restrict__ out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ntets) return;
    const int64_t a = rowptr[t], b = rowptr[t + 1];
    for (int s = 0; s < S; ++s) {
        float acc = 0.0f;
        for (int64_t j = a; j < b; ++j) acc = fmaf(pi[j], thetaT[(int64_t)col[j] * S + s], acc);
        out[(int64_t)s * ntets + t] = out_map<O>(acc, kind);
    }
}

cudaError_t launch_project(int64_t ntets, int S, const int64_t* rowptr, const int32_t* col, const float* pi,
                           const float* thetaT, int kind, int out64, void* out, cudaStream_t st) {
    if (S >= 8) {
        const unsigned nb = (unsigned)((ntets + kProjTets - 1) / kProjTets);
        // float4 / float2 gathers need rows of thetaT on 16 / 8 bytes (S a multiple of 4 / 2)
        if (S % 4 == 0) {
            if (out64) k_project_quad<double><<<nb, 256, 0, st>>>(ntets, S, rowptr, col, pi, thetaT, kind, (double*)out);
            else k_project_quad<float><<<nb, 256, 0, st>>>(ntets, S, rowptr, col, pi, thetaT, kind, (float*)out);
        } else if (S % 2 == 0) {
            if (out64) k_project_rows<double, 2><<<nb, 256, 0, st>>>(ntets, S, rowptr, col, pi, thetaT, kind, (double*)out);
            else k_project_rows<float, 2><<<nb, 256, 0, st>>>(ntets, S, rowptr, col, pi, thetaT, kind, (float*)out);
        } else {
            if (out64) k_project_rows<double, 1><<<nb, 256, 0, st>>>(ntets, S, rowptr, col, pi, thetaT, kind, (double*)out);
            else k_project_rows<float, 1><<<nb, 256, 0, st>>>(ntets, S, rowptr, col, pi, thetaT, kind, (float*)out);
        }
    } else {
        const unsigned nb = (unsigned)((ntets + 255) / 256);
        if (out64)
            k_project_thread<double><<<nb, 256, 0, st>>>(ntets, S, rowptr, col, pi, thetaT, kind, (double*)out);
        else
            k_project_thread<float><<<nb, 256, 0, st>>>(ntets, S, rowptr, col, pi, thetaT, kind, (float*)out);
    }
    return cudaGetLastError();
}

template <typename O>
__global__ void k_grid_out(int64_t ncell, const double* __restrict__ x, int64_t x_stride, double scale,
                           O* __restrict__ out) {
    const int s = blockIdx.y;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x)
        out[(int64_t)s * ncell + c] = (O)(scale * x[(int64_t)s * x_stride + c]);
}

cudaError_t launch_grid_out(int64_t ncell, int S, const double* x, int64_t x_stride, double scale, int out64,
                            void* out, cudaStream_t st) {
    int64_t b = (ncell + 255) / 256;
    if (b > 4096) b = 4096;
    dim3 grid((unsigned)b, S);
    if (out64) k_grid_out<double><<<grid, 256, 0, st>>>(ncell, x, x_stride, scale, (double*)out);
    else k_grid_out<float><<<grid, 256, 0, st>>>(ncell, x, x_stride, scale, (float*)out);
    return cudaGetLastError();
}

// thetaT[c][r] = float(scale * x[cols[r] * x_stride + c]) for the listed columns
__global__ void k_transpose_cols(int64_t ncell, int R, const int* __restrict__ cols, const double* __restrict__ x,
                                 int64_t x_stride, double scale, float* __restrict__ thetaT) {
    __shared__ float tile[32][33];
    const int64_t c0 = (int64_t)blockIdx.x * 32;
    const int r0 = blockIdx.y * 32;
    for (int rr = threadIdx.y; rr < 32; rr += blockDim.y) {
        const int r = r0 + rr;
        const int64_t c = c0 + threadIdx.x;
        tile[rr][threadIdx.x] = (r < R && c < ncell) ? (float)(scale * x[(int64_t)cols[r] * x_stride + c]) : 0.0f;
    }
    __syncthreads();
    for (int rr = threadIdx.y; rr < 32; rr += blockDim.y) {
        const int64_t c = c0 + rr;
        const int r = r0 + threadIdx.x;
        if (c < ncell && r < R) thetaT[c * R + r] = tile[threadIdx.x][rr];
    }
}

cudaError_t launch_transpose_cols(int64_t ncell, int R, const int* cols, const double* x, int64_t x_stride,
                                  double scale, float* thetaT, cudaStream_t st) {
    dim3 grid((unsigned)((ncell + 31) / 32), (unsigned)((R + 31) / 32));
    k_transpose_cols<<<grid, dim3(32, 8), 0, st>>>(ncell, R, cols, x, x_stride, scale, thetaT);
    return cudaGetLastError();
}

// projection with one output pointer per column (same FP32 fmaf order as k_project_*)
template <typename O>
__global__ void __launch_bounds__(256) k_project_ptrs(int64_t ntets, int R, const int64_t* __restrict__ rowptr,
                                                      const int32_t* __restrict__ col, const float* __restrict__ pi,
                                                      const float* __restrict__ thetaT, int kind,
                                                      O* const* __restrict__ outs) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ntets) return;
    const int64_t a = rowptr[t], b = rowptr[t + 1];
    for (int r = 0; r < R; ++r) {
        float acc = 0.0f;
        for (int64_t j = a; j < b; ++j) acc = fmaf(pi[j], thetaT[(int64_t)col[j] * R + r], acc);
        outs[r][t] = out_map<O>(acc, kind);
    }
}

cudaError_t launch_project_ptrs(int64_t ntets, int R, const int64_t* rowptr, const int32_t* col, const float* pi,
                                const float* thetaT, int kind, int out64, void* const* outs, cudaStream_t st) {
    const unsigned nb = (unsigned)((ntets + 255) / 256);
    if (out64)
        k_project_ptrs<double><<<nb, 256, 0, st>>>(ntets, R, rowptr, col, pi, thetaT, kind, (double* const*)outs);
    else
        k_project_ptrs<float><<<nb, 256, 0, st>>>(ntets, R, rowptr, col, pi, thetaT, kind, (float* const*)outs);
    return cudaGetLastError();
}

__global__ void k_mark_cols(int64_t nnz, const int32_t* __restrict__ col, unsigned char* __restrict__ flag) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nnz; j += (int64_t)gridDim.x * blockDim.x)
        flag[col[j]] = 1;
}

__global__ void k_count_flags(int64_t n, const unsigned char* __restrict__ flag, unsigned long long* __restrict__ cnt) {
    unsigned long long c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += flag[i];
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

cudaError_t count_used_columns(int64_t nnz, const int32_t* col, int64_t ncell, int64_t* used, cudaStream_t st) {
    unsigned char* flag = nullptr;
    unsigned long long* cnt = nullptr;
    unsigned long long h = 0;
    cudaError_t e = cudaMalloc(&flag, (size_t)ncell);
    if (e == cudaSuccess) e = cudaMalloc(&cnt, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, (size_t)ncell, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess && nnz > 0) {
        k_mark_cols<<<1024, 256, 0, st>>>(nnz, col, flag);
        k_count_flags<<<1024, 256, 0, st>>>(ncell, flag, cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(flag);
    cudaFree(cnt);
    *used = (int64_t)h;
    return e;
}

}  // namespace spde
