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

// S a multiple of 4: a group of 4 lanes per tet, 16 samples per lane (float4 i of the
// lane is the chunk's float4 gl + 4 i, so the group's four lanes read 64 contiguous bytes
// of a thetaT row per instruction); a warp works on 8 consecutive tets and no warp waits
// for another.  The entries of a row are loaded 16 at a time by the group's lanes
// together and handed round by width-4 shuffles, so the gathers of a block wait for one
// load latency.  The sum runs over the row in CSR order with the same fmaf sequence as
// the other projection kernels, so all of them give the same bits.  The results go
// straight from registers to out[sample][tet]: one store instruction writes, for each of
// four samples, the warp's 8 consecutive tets (one full 32-byte sector each).
constexpr int kGrpWarps = 4, kGrpTets = 8 * kGrpWarps;

__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <typename O>
__global__ void __launch_bounds__(32 * kGrpWarps) k_project_grp(int64_t ntets, int S, const int64_t* __restrict__ rowptr,
                                                                const int32_t* __restrict__ col, const float* __restrict__ pi,
                                                                const float* __restrict__ thetaT, int kind,
                                                                O* __restrict__ out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane >> 2, gl = lane & 3;
    const int64_t t = (int64_t)blockIdx.x * kGrpTets + warp * 8 + grp;
    const int S4 = S >> 2;
    const float4* T4 = reinterpret_cast<const float4*>(thetaT);
    int64_t a = 0, b = 0;
    if (t < ntets) {
        a = rowptr[t];
        b = rowptr[t + 1];
    }
    const int nblk = warp_max((int)((b - a + 15) >> 4));  // every group runs the warp's count
    for (int s0 = 0; s0 < S; s0 += kProjChunk) {
        const int q0 = (s0 >> 2) + gl;  // float4 i of this lane: q0 + 4 i
        bool on[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) on[i] = q0 + 4 * i < S4;
        float4 acc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        for (int blk = 0; blk < nblk; ++blk) {
            const int64_t base = a + 16 * (int64_t)blk;
            const int64_t left = b - base;
            const int len = left <= 0 ? 0 : (left < 16 ? (int)left : 16);
            float wl[4];
            int cl[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int k = gl + 4 * m;
                wl[m] = k < len ? pi[base + k] : 0.0f;
                cl[m] = k < len ? col[base + k] : 0;
            }
            const int lw = warp_max(len);
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                if (4 * m >= lw) break;
#pragma unroll
                for (int kk = 0; kk < 4; kk += 2) {  // two entries per step: independent gathers
                    const int k = 4 * m + kk;
                    const float w0 = __shfl_sync(0xffffffffu, wl[m], kk, 4);
                    const int c0 = __shfl_sync(0xffffffffu, cl[m], kk, 4);
                    const float w1 = __shfl_sync(0xffffffffu, wl[m], kk + 1, 4);
                    const int c1 = __shfl_sync(0xffffffffu, cl[m], kk + 1, 4);
                    const bool h0 = k < len, h1 = k + 1 < len;
                    const float4* row0 = T4 + (int64_t)c0 * S4;
                    const float4* row1 = T4 + (int64_t)c1 * S4;
                    float4 v0[4], v1[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (h0 && on[i]) v0[i] = row0[q0 + 4 * i];
                        if (h1 && on[i]) v1[i] = row1[q0 + 4 * i];
                    }
                    if (h0) {
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            if (on[i]) {
                                acc[i].x = fmaf(w0, v0[i].x, acc[i].x);
                                acc[i].y = fmaf(w0, v0[i].y, acc[i].y);
                                acc[i].z = fmaf(w0, v0[i].z, acc[i].z);
                                acc[i].w = fmaf(w0, v0[i].w, acc[i].w);
                            }
                    }
                    if (h1) {
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            if (on[i]) {
                                acc[i].x = fmaf(w1, v1[i].x, acc[i].x);
                                acc[i].y = fmaf(w1, v1[i].y, acc[i].y);
                                acc[i].z = fmaf(w1, v1[i].z, acc[i].z);
                                acc[i].w = fmaf(w1, v1[i].w, acc[i].w);
                            }
                    }
                }
            }
        }
        if (t < ntets) {
            // sample s0 + 4 (q0 - s0/4 + 4 i) + e = s0 + 4 (gl + 4 i) + e
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (on[i]) {
                    O* o = out + (int64_t)(s0 + 4 * (gl + 4 * i)) * ntets + t;
                    o[0] = out_map<O>(acc[i].x, kind);
                    o[ntets] = out_map<O>(acc[i].y, kind);
                    o[2 * ntets] = out_map<O>(acc[i].z, kind);
                    o[3 * ntets] = out_map<O>(acc[i].w, kind);
                }
        }
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
            const unsigned ng = (unsigned)((ntets + kGrpTets - 1) / kGrpTets);
            if (out64)
                k_project_grp<double><<<ng, 32 * kGrpWarps, 0, st>>>(ntets, S, rowptr, col, pi, thetaT, kind,
                                                                     (double*)out);
            else
                k_project_grp<float><<<ng, 32 * kGrpWarps, 0, st>>>(ntets, S, rowptr, col, pi, thetaT, kind,
                                                                    (float*)out);
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
