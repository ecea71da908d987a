// K6: one-time tet / hex clipping that assembles the coupling matrix of the
// L2 projection (Sec. 5.1-5.2).  For P0 spaces on both meshes the entry
// G[tau][c] = int_{tau cap c} 1 dx is the volume of the intersection, which
// is computed exactly in FP64 (no quadrature needed).
//
// Volume by the divergence theorem: the boundary of the convex polytope
// tau cap c consists of (a) the tet's faces clipped to the cell and (b) the
// cell's faces clipped to the tet.  With every face polygon oriented
// outward, 6 V = sum over faces, over fan triangles (v0, vi, vi+1), of
// v0 . (vi x vi+1).  Coordinates are cell-local and scaled by 1/h; tet
// vertex coordinates within EPS of a cell plane (0 or 1) are first moved
// onto it, and all sign tests are then exact, so parts (a) and (b) agree on
// every shared boundary (a face on a cell plane gets an exactly
// axis-aligned normal and exactly zero distances).  A tet face lying on a
// cell plane with the same outward direction is left to (b), so a shared
// face is counted once.
//
// Build: per tet, candidate cells from its bounding box -> exclusive scan ->
// volumes of all candidates -> scan of the nonzero counts -> CSR.
#include <cstdio>
#include <vector>

#include "device.cuh"
#include "internal.h"

namespace spde {

struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 operator-(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ D3 operator+(D3 a, D3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ D3 operator*(double s, D3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot3(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 cross3(D3 a, D3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double comp(D3 a, int ax) { return ax == 0 ? a.x : (ax == 1 ? a.y : a.z); }
__device__ __forceinline__ void set_comp(D3& a, int ax, double v) {
    if (ax == 0) a.x = v;
    else if (ax == 1) a.y = v;
    else a.z = v;
}

constexpr int kPolyMax = 12;
constexpr double kSnap = 1e-12;  // cell units: vertex coordinates this close to 0 or 1 are moved onto the plane

// fan sum of v0 . (vi x vi+1) over a polygon
__device__ __forceinline__ double fan6(const D3* p, int m) {
    double s = 0.0;
    for (int i = 1; i + 1 < m; ++i) s += dot3(p[0], cross3(p[i], p[i + 1]));
    return s;
}

// clip polygon in[0..m) by {x : x_ax * sgn <= bound * sgn} (axis-aligned)
__device__ int clip_axis(const D3* in, int m, D3* out, int ax, double bound, double sgn) {
    int k = 0;
    for (int i = 0; i < m; ++i) {
        const D3 a = in[i], b = in[(i + 1) % m];
        const double da = (comp(a, ax) - bound) * sgn, db = (comp(b, ax) - bound) * sgn;
        if (da <= 0.0 && k < kPolyMax) out[k++] = a;
        if ((da < 0.0 && db > 0.0) || (da > 0.0 && db < 0.0)) {
            D3 x = a + (da / (da - db)) * (b - a);
            set_comp(x, ax, bound);
            if (k < kPolyMax) out[k++] = x;
        }
    }
    return k;
}

// clip polygon by {x : n.(x - o) <= 0} (unit n, o a point of the plane).  The
// distance is taken from a point of the plane, not as n.x - n.o: for a plane
// nearly parallel to the polygon (a thin tet's side face over a cell face) the
// second form cancels two numbers of size 1 down to ~1e-5 and moves the cut
// points by ~1e-11, which the other half of the surface does not see.
__device__ int clip_plane(const D3* in, int m, D3* out, D3 n, D3 o) {
    int k = 0;
    for (int i = 0; i < m; ++i) {
        const D3 a = in[i], b = in[(i + 1) % m];
        const double da = dot3(n, a - o), db = dot3(n, b - o);
        if (da <= 0.0 && k < kPolyMax) out[k++] = a;
        if ((da < 0.0 && db > 0.0) || (da > 0.0 && db < 0.0)) {
            if (k < kPolyMax) out[k++] = a + (da / (da - db)) * (b - a);
        }
    }
    return k;
}

// volume of tet p (positively oriented, cell-local scaled coordinates) inside [0,1]^3
__device__ double tet_unit_cube_volume(const D3 p[4]) {
    // outward faces of a positively oriented tet
    const int F[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
    D3 bufA[kPolyMax], bufB[kPolyMax];
    double v6 = 0.0;
    D3 nrm[4];
    D3 anc[4];  // a vertex of each face: the origin of its distances
    for (int f = 0; f < 4; ++f) {
        const D3 a = p[F[f][0]], b = p[F[f][1]], c = p[F[f][2]];
        D3 nv = cross3(b - a, c - a);
        const double len = sqrt(dot3(nv, nv));
        nv = (1.0 / len) * nv;
        nrm[f] = nv;
        anc[f] = a;
        // (a) tet face clipped to the cell, unless it lies on a cell plane with
        // the same outward direction (then (b) supplies that face)
        bool skip = false;
        for (int ax = 0; ax < 3 && !skip; ++ax) {
            const double na = comp(nv, ax);
            const double ca = comp(a, ax), cb = comp(b, ax), cc = comp(c, ax);
            if (na > 0.5 && ca == 1.0 && cb == 1.0 && cc == 1.0) skip = true;
            if (na < -0.5 && ca == 0.0 && cb == 0.0 && cc == 0.0) skip = true;
        }
        if (skip) continue;
        bufA[0] = a;
        bufA[1] = b;
        bufA[2] = c;
        int m = 3;
        m = clip_axis(bufA, m, bufB, 0, 0.0, -1.0);
        m = clip_axis(bufB, m, bufA, 0, 1.0, 1.0);
        m = clip_axis(bufA, m, bufB, 1, 0.0, -1.0);
        m = clip_axis(bufB, m, bufA, 1, 1.0, 1.0);
        m = clip_axis(bufA, m, bufB, 2, 0.0, -1.0);
        m = clip_axis(bufB, m, bufA, 2, 1.0, 1.0);
        if (m >= 3) v6 += fan6(bufA, m);
    }
    // (b) cell faces clipped to the tet
    for (int ax = 0; ax < 3; ++ax) {
        const int bx = (ax + 1) % 3, cx = (ax + 2) % 3;
        for (int side = 0; side < 2; ++side) {
            // corners in (b, c) coordinates, counter-clockwise seen from outside
            const double lo_seq[4][2] = {{0, 0}, {0, 1}, {1, 1}, {1, 0}};
            const double hi_seq[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
            for (int q = 0; q < 4; ++q) {
                D3 v{0, 0, 0};
                set_comp(v, ax, (double)side);
                set_comp(v, bx, side ? hi_seq[q][0] : lo_seq[q][0]);
                set_comp(v, cx, side ? hi_seq[q][1] : lo_seq[q][1]);
                bufA[q] = v;
            }
            int m = 4;
            m = clip_plane(bufA, m, bufB, nrm[0], anc[0]);
            m = clip_plane(bufB, m, bufA, nrm[1], anc[1]);
            m = clip_plane(bufA, m, bufB, nrm[2], anc[2]);
            m = clip_plane(bufB, m, bufA, nrm[3], anc[3]);
            if (m >= 3) v6 += fan6(bufA, m);
        }
    }
    return v6 / 6.0;
}

struct ClipGrid {
    int n[3];  // cells per axis
    double h;
    double lo[3];
};

__device__ __forceinline__ void load_tet(const double* xyz, const int32_t* tets, int64_t t, D3 p[4]) {
    for (int v = 0; v < 4; ++v) {
        const int64_t id = tets[4 * t + v];
        p[v] = D3{xyz[3 * id], xyz[3 * id + 1], xyz[3 * id + 2]};
    }
}

__device__ __forceinline__ void note_bad(unsigned long long* bad, int64_t t, int kind) {
    atomicMin(bad, ((unsigned long long)t << 2) | (unsigned long long)kind);
}

// pass 1: orientation, volume, coverage, candidate count
__global__ void k_tet_prep(ClipGrid g, int64_t nverts, const double* __restrict__ xyz, int64_t ntets,
                           int32_t* __restrict__ tets, double* __restrict__ vol, int64_t* __restrict__ cand,
                           int* __restrict__ range, unsigned long long* __restrict__ bad) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ntets) return;
    for (int v = 0; v < 4; ++v) {
        const int32_t id = tets[4 * t + v];
        if (id < 0 || id >= nverts) {
            note_bad(bad, t, 1);
            cand[t] = 0;
            vol[t] = 0.0;
            return;
        }
    }
    D3 p[4];
    load_tet(xyz, tets, t, p);
    const double det = dot3(cross3(p[1] - p[0], p[2] - p[0]), p[3] - p[0]);
    if (det < 0.0) {  // fix orientation on the device copy
        const int32_t tmp = tets[4 * t + 2];
        tets[4 * t + 2] = tets[4 * t + 3];
        tets[4 * t + 3] = tmp;
    }
    const double v = fabs(det) / 6.0;
    vol[t] = v;
    if (!(v > 1e-9 * g.h * g.h * g.h)) {
        note_bad(bad, t, 1);
        cand[t] = 0;
        return;
    }
    int lo_i[3], hi_i[3];
    bool outside = false;
    for (int ax = 0; ax < 3; ++ax) {
        double mn = comp(p[0], ax), mx = mn;
        for (int q = 1; q < 4; ++q) {
            mn = fmin(mn, comp(p[q], ax));
            mx = fmax(mx, comp(p[q], ax));
        }
        const double a = (mn - g.lo[ax]) / g.h, b = (mx - g.lo[ax]) / g.h;
        const double tol = 1e-9;
        if (a < -tol || b > g.n[ax] + tol) outside = true;
        int ia = (int)floor(a), ib = (int)floor(b);
        ia = min(max(ia, 0), g.n[ax] - 1);
        ib = min(max(ib, 0), g.n[ax] - 1);
        lo_i[ax] = ia;
        hi_i[ax] = ib;
    }
    if (outside) {
        note_bad(bad, t, 2);
        cand[t] = 0;
        return;
    }
    for (int ax = 0; ax < 3; ++ax) {
        range[6 * t + 2 * ax] = lo_i[ax];
        range[6 * t + 2 * ax + 1] = hi_i[ax];
    }
    cand[t] = (int64_t)(hi_i[0] - lo_i[0] + 1) * (hi_i[1] - lo_i[1] + 1) * (hi_i[2] - lo_i[2] + 1);
}

// pass 2: volumes of every candidate cell
__global__ void k_tet_clip(ClipGrid g, const double* __restrict__ xyz, int64_t ntets, const int32_t* __restrict__ tets,
                           const int* __restrict__ range, const int64_t* __restrict__ cand_off,
                           const int64_t* __restrict__ cand, double* __restrict__ cvol, int32_t* __restrict__ ccell,
                           int64_t* __restrict__ nz) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ntets) return;
    if (cand[t] == 0) {
        nz[t] = 0;
        return;
    }
    D3 p[4];
    load_tet(xyz, tets, t, p);
    const int* r = range + 6 * t;
    int64_t o = cand_off[t];
    int64_t cnt = 0;
    const double ih = 1.0 / g.h;
    for (int k = r[4]; k <= r[5]; ++k)
        for (int j = r[2]; j <= r[3]; ++j)
            for (int i = r[0]; i <= r[1]; ++i) {
                const D3 c0{g.lo[0] + i * g.h, g.lo[1] + j * g.h, g.lo[2] + k * g.h};
                D3 q[4];
                for (int v = 0; v < 4; ++v) {
                    q[v] = ih * (p[v] - c0);
                    for (int ax = 0; ax < 3; ++ax) {
                        const double x = comp(q[v], ax);
                        if (fabs(x) <= kSnap) set_comp(q[v], ax, 0.0);
                        else if (fabs(x - 1.0) <= kSnap) set_comp(q[v], ax, 1.0);
                    }
                }
                double v = tet_unit_cube_volume(q);
                if (!(v > 1e-14)) v = 0.0;
                else ++cnt;
                cvol[o] = v * g.h * g.h * g.h;
                ccell[o] = (int32_t)(i + (int64_t)g.n[0] * (j + (int64_t)g.n[1] * k));
                ++o;
            }
    nz[t] = cnt;
}

// pass 3: compact to CSR; check row sums
__global__ void k_tet_compact(int64_t ntets, const int64_t* __restrict__ cand_off, const int64_t* __restrict__ cand,
                              const double* __restrict__ cvol, const int32_t* __restrict__ ccell,
                              const int64_t* __restrict__ rowptr, const double* __restrict__ vol,
                              int32_t* __restrict__ col, double* __restrict__ gval, float* __restrict__ pi,
                              double h3, unsigned long long* __restrict__ bad) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ntets) return;
    int64_t o = rowptr[t];
    double sum = 0.0;
    const double iv = 1.0 / vol[t];
    for (int64_t q = cand_off[t]; q < cand_off[t] + cand[t]; ++q) {
        const double v = cvol[q];
        if (v > 0.0) {
            col[o] = ccell[q];
            gval[o] = v;
            pi[o] = (float)(v * iv);
            sum += v;
            ++o;
        }
    }
    // coverage: the pieces must add up to the tet.  The fan sums of a piece carry
    // rounding at the scale of the cell (terms of size h^3 that cancel down to a
    // sliver's volume), so the bound has an absolute part of 1e-12 h^3 besides
    // the relative one; a tet reaching out of the box misses far more.
    if (cand[t] > 0 && !(fabs(sum - vol[t]) <= 1e-10 * vol[t] + 1e-12 * h3)) note_bad(bad, t, 3);
}

// ---- exclusive scan of int64 (three phases, no inter-block waiting) -------
constexpr int kScanBlock = 1024;

__global__ void k_scan_local(int64_t n, const int64_t* __restrict__ in, int64_t* __restrict__ out,
                             int64_t* __restrict__ block_tot) {
    __shared__ int64_t sh[kScanBlock];
    const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    const int64_t v = (i < n) ? in[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < kScanBlock; o <<= 1) {
        const int64_t add = (threadIdx.x >= o) ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += add;
        __syncthreads();
    }
    if (i < n) out[i] = sh[threadIdx.x] - v;  // exclusive
    if (threadIdx.x == kScanBlock - 1) block_tot[blockIdx.x] = sh[threadIdx.x];
}

__global__ void k_scan_totals(int64_t nb, int64_t* __restrict__ tot, int64_t* __restrict__ grand) {
    // one block: exclusive scan of the block totals in chunks with a carry
    __shared__ int64_t sh[kScanBlock];
    int64_t carry = 0;
    for (int64_t base = 0; base < nb; base += kScanBlock) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = (i < nb) ? tot[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < kScanBlock; o <<= 1) {
            const int64_t add = (threadIdx.x >= o) ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < nb) tot[i] = carry + sh[threadIdx.x] - v;
        const int64_t chunk = sh[kScanBlock - 1];
        __syncthreads();
        carry += chunk;
    }
    if (threadIdx.x == 0) *grand = carry;
}

__global__ void k_scan_add(int64_t n, int64_t* __restrict__ out, const int64_t* __restrict__ tot) {
    const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    if (i < n) out[i] += tot[blockIdx.x];
}

// exclusive scan of in[0..n) into out[0..n), out[n] = total; returns total via host
static cudaError_t exclusive_scan(int64_t n, const int64_t* in, int64_t* out, int64_t* tmp, int64_t* h_total,
                                  cudaStream_t st) {
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    k_scan_local<<<(unsigned)nb, kScanBlock, 0, st>>>(n, in, out, tmp);
    k_scan_totals<<<1, kScanBlock, 0, st>>>(nb, tmp, out + n);
    k_scan_add<<<(unsigned)nb, kScanBlock, 0, st>>>(n, out, tmp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(h_total, out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(st);
}

#define CK(x)                                    \
    do {                                         \
        cudaError_t e_ = (x);                    \
        if (e_ != cudaSuccess) {                 \
            err = e_;                            \
            cudaGetLastError();                  \
            goto done;                           \
        }                                        \
    } while (0)

cudaError_t build_coupling(const int n[3], double h, const double lo[3], int64_t nverts, const double* d_xyz, int64_t ntets,
                           const int32_t* d_tets_in, double* d_vol, int64_t** d_rowptr, int32_t** d_col, double** d_g,
                           float** d_pi, ClipResult* res, cudaStream_t st) {
    cudaError_t err = cudaSuccess;
    ClipGrid g{{n[0], n[1], n[2]}, h, {lo[0], lo[1], lo[2]}};
    int32_t* tets = const_cast<int32_t*>(d_tets_in);
    int64_t *cand = nullptr, *cand_off = nullptr, *nz = nullptr, *tmp = nullptr, *rowptr = nullptr;
    int* range = nullptr;
    double* cvol = nullptr;
    int32_t* ccell = nullptr;
    int32_t* col = nullptr;
    double* gv = nullptr;
    float* pv = nullptr;
    unsigned long long* bad = nullptr;
    unsigned long long h_bad = ~0ull;
    int64_t ncand = 0, nnz = 0;
    const int64_t nb = (ntets + kScanBlock - 1) / kScanBlock;
    const unsigned tb = (unsigned)((ntets + 255) / 256);
    *d_rowptr = nullptr;
    *d_col = nullptr;
    *d_g = nullptr;
    *d_pi = nullptr;
    res->nnz = 0;
    res->bad_tet = -1;
    res->bad_kind = 0;
    CK(cudaMalloc(&cand, ntets * sizeof(int64_t)));
    CK(cudaMalloc(&cand_off, (ntets + 1) * sizeof(int64_t)));
    CK(cudaMalloc(&nz, ntets * sizeof(int64_t)));
    CK(cudaMalloc(&tmp, (nb + 1) * sizeof(int64_t)));
    CK(cudaMalloc(&range, ntets * 6 * sizeof(int)));
    CK(cudaMalloc(&bad, sizeof(unsigned long long)));
    CK(cudaMemcpyAsync(bad, &h_bad, sizeof(h_bad), cudaMemcpyHostToDevice, st));
    k_tet_prep<<<tb, 256, 0, st>>>(g, nverts, d_xyz, ntets, tets, d_vol, cand, range, bad);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&h_bad, bad, sizeof(h_bad), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h_bad != ~0ull) {
        res->bad_tet = (int)(h_bad >> 2);
        res->bad_kind = (int)(h_bad & 3);
        goto done;
    }
    CK(exclusive_scan(ntets, cand, cand_off, tmp, &ncand, st));
    CK(cudaMalloc(&cvol, (ncand + 1) * sizeof(double)));
    CK(cudaMalloc(&ccell, (ncand + 1) * sizeof(int32_t)));
    k_tet_clip<<<(unsigned)((ntets + 127) / 128), 128, 0, st>>>(g, d_xyz, ntets, tets, range, cand_off, cand, cvol, ccell, nz);
    CK(cudaGetLastError());
    CK(cudaMalloc(&rowptr, (ntets + 1) * sizeof(int64_t)));
    CK(exclusive_scan(ntets, nz, rowptr, tmp, &nnz, st));
    CK(cudaMalloc(&col, (nnz + 1) * sizeof(int32_t)));
    CK(cudaMalloc(&gv, (nnz + 1) * sizeof(double)));
    CK(cudaMalloc(&pv, (nnz + 1) * sizeof(float)));
    k_tet_compact<<<tb, 256, 0, st>>>(ntets, cand_off, cand, cvol, ccell, rowptr, d_vol, col, gv, pv, h * h * h,
                                       bad);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&h_bad, bad, sizeof(h_bad), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h_bad != ~0ull) {
        res->bad_tet = (int)(h_bad >> 2);
        res->bad_kind = (int)(h_bad & 3);
    }
    res->nnz = nnz;
    *d_rowptr = rowptr;
    *d_col = col;
    *d_g = gv;
    *d_pi = pv;
    rowptr = nullptr;
    col = nullptr;
    gv = nullptr;
    pv = nullptr;
done:
    cudaFree(cand);
    cudaFree(cand_off);
    cudaFree(nz);
    cudaFree(tmp);
    cudaFree(range);
    cudaFree(bad);
    cudaFree(cvol);
    cudaFree(ccell);
    cudaFree(rowptr);
    cudaFree(col);
    cudaFree(gv);
    cudaFree(pv);
    return err;
}

}  // namespace spde
