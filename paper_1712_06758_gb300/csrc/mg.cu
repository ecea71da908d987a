// K3: field block of the MINRES preconditioner -- one symmetric geometric
// multigrid V-cycle for the cell-centred 7-point Schur approximation
//     A_0 = (kappa h)^2 I + c L          (L: Neumann graph Laplacian)
// on the nested embedding grids of Sec. 6.1.
//
// Level l has n_l = n >> l cells per axis and operator
//     A_l = 2^l ((kappa h)^2 4^l I + c L_l),   D_l = diag(A_l),
// transfers P = tensor product of the 1-D cell-centred linear prolongation
//     fine 2I <- 3/4 e_I + 1/4 e_{I-1},  fine 2I+1 <- 3/4 e_I + 1/4 e_{I+1}
// (indices clamped at the walls: reflection for the no-flux boundary) and
// R = P^T.  Each level: x = omega D^{-1} b (one Jacobi sweep from zero),
// coarse correction with r = b - A x, then one more Jacobi sweep; the
// one-cell level is solved exactly.  Same sweep before and after makes the
// operator symmetric; with 0 < omega < 1 it is positive definite, as MINRES
// needs.
//
// Kernels: levels with n_l >= 32 use shared-memory tiles (a down sweep that
// smooths, forms the residual and restricts in one pass; an up sweep that
// prolongs, corrects and post-smooths in one pass).  All levels with
// n_l <= 16 run inside one CTA per sample in shared memory.
#include "device.cuh"
#include "internal.h"
#include "prof.h"

namespace spde {

// tile of the fine level handled by one CTA in the down/up sweeps
constexpr int TFX = 32, TFY = 8, TFZ = 8;
constexpr int TCX = TFX / 2, TCY = TFY / 2, TCZ = TFZ / 2;
constexpr int kTileThreads = 256;
constexpr int kCoarseThreads = 512;
constexpr int kMaxTilesPerCol = 2048;

template <typename T>
struct LevelCoef {
    T s;         // 2^l
    T a;         // (kappa h)^2 4^l
    T c;         // Schur weight
    T omega;
    T invD[7];   // 1 / (s (a + c k)) for k neighbours
    T D[7];      // s (a + c k)
};

template <typename T>
static LevelCoef<T> level_coef(const MGPlan& p, int l) {
    LevelCoef<T> q;
    const double s = (double)(1 << l);
    const double a = p.kh2 * (double)(1ll << (2 * l));
    q.s = (T)s;
    q.a = (T)a;
    q.c = (T)p.c;
    q.omega = (T)p.omega;
    for (int k = 0; k <= 6; ++k) {
        q.invD[k] = (T)(1.0 / (s * (a + p.c * k)));
        q.D[k] = (T)(s * (a + p.c * k));
    }
    return q;
}

__device__ __forceinline__ float restrict_w(int a, int I, int nc) {
    switch (a) {
        case 0: return I > 0 ? 0.25f : 0.0f;
        case 1: return I == 0 ? 1.0f : 0.75f;
        case 2: return I == nc - 1 ? 1.0f : 0.75f;
        default: return I < nc - 1 ? 0.25f : 0.0f;
    }
}

// ---------------------------------------------------------------------------
// Down sweep at level l: b (fine, n_f^3) -> bc = R (b - A omega D^{-1} b).
// With x0 = omega D^{-1} b the residual is
//     r(f) = (1/omega - 1) D(f) x0(f) + s c sum_{neighbours g} x0(g),
// so one shared array of x0 on the tile + halo 2 (zero outside the box,
// which makes the sum run over existing neighbours only) gives r on the
// tile + halo 1, from which the 4^3-point restriction gathers.
// Thread block (32, 8): x along threadIdx.x, y along threadIdx.y, loops in z.
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool in_box(int x, int y, int z, int n) {
    return (unsigned)x < (unsigned)n && (unsigned)y < (unsigned)n && (unsigned)z < (unsigned)n;
}

template <typename T>
__device__ __forceinline__ void load_coef(const LevelCoef<T>& q, T* s_invD, T* s_D) {
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if (tid < 7) {
        s_invD[tid] = q.invD[tid];
        s_D[tid] = q.D[tid];
    }
}

// Streaming sweeps: a CTA owns a fine (x, y) tile of SX x SY cells and marches
// along z through SZ fine planes, keeping a few planes in shared-memory rings.
// Fine planes are fetched as 16-byte vectors starting 4 cells left of the tile
// (tiles and grids are multiples of 32, so a vector lies wholly inside or
// wholly outside the box), one plane ahead into registers, so the loads of
// plane f+2 are in flight while plane f is computed.
constexpr int SX = 32, SY = 16, SZ = 32;
constexpr int PW = SX + 8;               // plane row width in shared memory (x from fx0 - 4)
constexpr int XH = SY + 4;               // x0 rows, halo 2 (down sweep)
constexpr int RW = SX + 2, RH = SY + 2;  // residual plane, halo 1
constexpr int BH = SY + 2;               // b / x rows, halo 1 (up sweep)
constexpr int CW = SX / 2 + 2, CH = SY / 2 + 2;  // coarse plane with halo 1 (up sweep)
constexpr int kDownSSmem = 3 * PW * XH + 4 * RW * RH;
constexpr int kUpSSmem = 3 * PW * BH + 3 * PW * BH + 3 * CW * CH;
constexpr int kQ = PW / 4;               // float4 per plane row

__device__ __forceinline__ int ring3(int f) { return (f + 3) % 3; }  // f >= -3
__device__ __forceinline__ int ring4(int f) { return (f + 4) & 3; }  // f >= -4

template <typename T>
struct PlaneRegs {
    V4<T> v[2];
};

// fetch rows y0 .. y0+rows-1 of plane f (x from x0, PW wide) as vectors; zero outside the box
template <typename T>
__device__ __forceinline__ void fetch_plane(PlaneRegs<T>& r, const T* bs, int nf, int64_t plane, int f, int x0,
                                            int y0, int rows, int tid) {
    const bool zin = (unsigned)f < (unsigned)nf;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int idx = tid + u * kTileThreads;
        r.v[u] = zero4<T>();
        if (idx < kQ * rows && zin) {
            const int ly = idx / kQ, q4 = idx - ly * kQ;
            const int gx = x0 + 4 * q4, gy = y0 + ly;
            if ((unsigned)gx < (unsigned)nf && (unsigned)gy < (unsigned)nf)
                r.v[u] = ld4(bs + gx + (int64_t)nf * gy + plane * f);
        }
    }
}

// ---------------------------------------------------------------------------
// Down sweep at level l: bc = R (b - A omega D^{-1} b).  With x0 = omega D^{-1} b
//     r(f) = (1/omega - 1) D(f) x0(f) + s c sum_{neighbours g} x0(g)
// (x0 = 0 outside the box, so the sum runs over existing neighbours).
// Per fine plane: store the x0 plane f+1, fetch plane f+2, form r on plane
// f, and after every second plane restrict one coarse plane from the four r
// planes 2Z-1 .. 2Z+2.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kTileThreads) k_mg_down(int nf, LevelCoef<T> q, const T* __restrict__ b,
                                                          int64_t b_stride, T* __restrict__ bc, int64_t bc_stride,
                                                          const int* __restrict__ active, int act_stride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T s_invD[8], s_D[8];
    T* X = reinterpret_cast<T*>(smem_raw);  // 3 x0 planes, PW x XH
    T* R = X + 3 * PW * XH;                  // 4 residual planes, RW x RH
    const int col = blockIdx.y;
    if (active && !active[(int64_t)col * act_stride]) return;
    load_coef(q, s_invD, s_D);
    const int tid = threadIdx.x + 32 * threadIdx.y;
    const int nc = nf >> 1;
    const int ntx = nf / SX, nty = nf / SY, ntz = nf / SZ;
    const int ntiles = ntx * nty * ntz;
    const int64_t plane = (int64_t)nf * nf;
    const T* bs = b + (int64_t)col * b_stride;
    T* bcs = bc + (int64_t)col * bc_stride;
    const T rc = (T(1) / q.omega - T(1));
    const T sc = q.s * q.c;
    const T om = q.omega;
    __syncthreads();
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tX = tile % ntx, tY = (tile / ntx) % nty, tZ = tile / (ntx * nty);
        const int fx0 = tX * SX, fy0 = tY * SY, fz0 = tZ * SZ;
        const int cx0 = fx0 >> 1, cy0 = fy0 >> 1;
        // x0 = omega D^{-1} b into ring slot of plane f
        auto commit = [&](const PlaneRegs<T>& r, int f) {
            T* dst = X + ring3(f) * (PW * XH);
            const bool zin = (unsigned)f < (unsigned)nf;
            const int kz = zin ? nb_count1(f, nf) : 0;
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int idx = tid + u * kTileThreads;
                if (idx < kQ * XH) {
                    const int ly = idx / kQ, q4 = idx - ly * kQ;
                    const int gy = fy0 - 2 + ly;
                    const int ky = ((unsigned)gy < (unsigned)nf) ? nb_count1(gy, nf) : 0;
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int gx = fx0 - 4 + 4 * q4 + e;
                        const int kx = ((unsigned)gx < (unsigned)nf) ? nb_count1(gx, nf) : 0;
                        dst[4 * q4 + e + PW * ly] = om * r.v[u].v[e] * s_invD[kx + ky + kz];
                    }
                }
            }
        };
        PlaneRegs<T> pr;
        fetch_plane(pr, bs, nf, plane, fz0 - 2, fx0 - 4, fy0 - 2, XH, tid);
        commit(pr, fz0 - 2);
        fetch_plane(pr, bs, nf, plane, fz0 - 1, fx0 - 4, fy0 - 2, XH, tid);
        commit(pr, fz0 - 1);
        fetch_plane(pr, bs, nf, plane, fz0, fx0 - 4, fy0 - 2, XH, tid);
        for (int f = fz0 - 1; f <= fz0 + SZ; ++f) {
            commit(pr, f + 1);
            if (f + 2 <= fz0 + SZ + 1) fetch_plane(pr, bs, nf, plane, f + 2, fx0 - 4, fy0 - 2, XH, tid);
            __syncthreads();
            {
                const T* Xm = X + ring3(f - 1) * (PW * XH);
                const T* Xc = X + ring3(f) * (PW * XH);
                const T* Xp = X + ring3(f + 1) * (PW * XH);
                T* Rd = R + ring4(f) * (RW * RH);
                const bool zin = (unsigned)f < (unsigned)nf;
                const int kz = zin ? nb_count1(f, nf) : 0;
                for (int idx = tid; idx < RW * RH; idx += kTileThreads) {
                    const int ly = idx / RW, lx = idx - ly * RW;
                    const int gx = fx0 - 1 + lx, gy = fy0 - 1 + ly;
                    T r = T(0);
                    if (zin && (unsigned)gx < (unsigned)nf && (unsigned)gy < (unsigned)nf) {
                        const int xi = (lx + 3) + PW * (ly + 1);
                        const T nbs = (Xc[xi - 1] + Xc[xi + 1]) + (Xc[xi - PW] + Xc[xi + PW]) + (Xm[xi] + Xp[xi]);
                        r = rc * s_D[nb_count1(gx, nf) + nb_count1(gy, nf) + kz] * Xc[xi] + sc * nbs;
                    }
                    Rd[idx] = r;
                }
            }
            __syncthreads();
            if (f >= fz0 + 2 && ((f - fz0) & 1) == 0 && tid < (SX / 2) * (SY / 2)) {
                const int Z = (f - 2) >> 1;
                const int li = tid & (SX / 2 - 1), lj = tid / (SX / 2);
                const int I = cx0 + li, J = cy0 + lj;
                T wx[4], wy[4], wz[4];
#pragma unroll
                for (int a3 = 0; a3 < 4; ++a3) {
                    wx[a3] = (T)restrict_w(a3, I, nc);
                    wy[a3] = (T)restrict_w(a3, J, nc);
                    wz[a3] = (T)restrict_w(a3, Z, nc);
                }
                T acc = T(0);
#pragma unroll
                for (int c3 = 0; c3 < 4; ++c3) {
                    const T* Rp = R + ring4(2 * Z - 1 + c3) * (RW * RH);
                    T accy = T(0);
#pragma unroll
                    for (int b3 = 0; b3 < 4; ++b3) {
                        const T* row = Rp + 2 * li + RW * (2 * lj + b3);
                        accy += wy[b3] * (wx[0] * row[0] + wx[1] * row[1] + wx[2] * row[2] + wx[3] * row[3]);
                    }
                    acc += wz[c3] * accy;
                }
                bcs[I + (int64_t)nc * (J + (int64_t)nc * Z)] = acc;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Up sweep at level l: x = omega D^{-1} b + P ec ; y = x + omega D^{-1} (b - A x),
// optional partial sums of b.y (the MINRES beta^2 contribution).  Per fine
// plane g: store b(g) and (for even g) coarse plane g/2 + 1, fetch the next
// ones, form x(g) on the tile + halo 1, then y(g - 1) from x planes g-2 .. g.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kTileThreads) k_mg_up(int nf, LevelCoef<T> q, const T* __restrict__ b,
                                                        int64_t b_stride, const T* __restrict__ ec,
                                                        int64_t ec_stride, T* __restrict__ y, int64_t y_stride,
                                                        double* __restrict__ dot_part,
                                                        const int* __restrict__ active, int act_stride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[kTileThreads / 32];
    __shared__ T s_invD[8], s_D[8];
    T* B = reinterpret_cast<T*>(smem_raw);  // 3 b planes, PW x BH
    T* Xr = B + 3 * PW * BH;                 // 3 x planes, PW x BH
    T* C = Xr + 3 * PW * BH;                 // 3 coarse planes, CW x CH
    const int col = blockIdx.y;
    if (active && !active[(int64_t)col * act_stride]) return;
    load_coef(q, s_invD, s_D);
    const int tid = threadIdx.x + 32 * threadIdx.y;
    const int nc = nf >> 1;
    const int ntx = nf / SX, nty = nf / SY, ntz = nf / SZ;
    const int ntiles = ntx * nty * ntz;
    const int64_t plane = (int64_t)nf * nf, cplane = (int64_t)nc * nc;
    const T* bs = b + (int64_t)col * b_stride;
    const T* es = ec + (int64_t)col * ec_stride;
    T* ys = y + (int64_t)col * y_stride;
    const T om = q.omega;
    const T w0 = T(0.75), w1 = T(0.25);
    double dacc = 0.0;
    __syncthreads();
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tX = tile % ntx, tY = (tile / ntx) % nty, tZ = tile / (ntx * nty);
        const int fx0 = tX * SX, fy0 = tY * SY, fz0 = tZ * SZ;
        const int cx0 = fx0 >> 1, cy0 = fy0 >> 1;
        // coarse plane Z (clamped indices: wall reflection), one value per thread
        auto fetch_c = [&](int Z) -> T {
            T v = T(0);
            if (tid < CW * CH) {
                const int ly = tid / CW, lx = tid - ly * CW;
                const int gx = min(max(cx0 - 1 + lx, 0), nc - 1), gy = min(max(cy0 - 1 + ly, 0), nc - 1);
                v = es[gx + (int64_t)nc * gy + cplane * min(max(Z, 0), nc - 1)];
            }
            return v;
        };
        auto commit_c = [&](T v, int Z) {
            if (tid < CW * CH) C[ring3(Z) * (CW * CH) + tid] = v;
        };
        auto commit_b = [&](const PlaneRegs<T>& r, int g) {
            T* dst = B + ring3(g) * (PW * BH);
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int idx = tid + u * kTileThreads;
                if (idx < kQ * BH) st4(dst + 4 * idx, r.v[u]);
            }
        };
        auto make_x = [&](int g) {
            const T* Bg = B + ring3(g) * (PW * BH);
            T* Xg = Xr + ring3(g) * (PW * BH);
            const bool zin = (unsigned)g < (unsigned)nf;
            const int Iz = g >> 1;
            const T* Cz0 = C + ring3(Iz) * (CW * CH);
            const T* Cz1 = C + ring3((g & 1) ? Iz + 1 : Iz - 1) * (CW * CH);
            const int kz = zin ? nb_count1(g, nf) : 0;
            for (int idx = tid; idx < RW * BH; idx += kTileThreads) {
                const int ly = idx / RW, lx = idx - ly * RW;
                const int gx = fx0 - 1 + lx, gy = fy0 - 1 + ly;
                const int xi = (lx + 3) + PW * ly;
                T v = T(0);
                if (zin && (unsigned)gx < (unsigned)nf && (unsigned)gy < (unsigned)nf) {
                    const int Ix = gx >> 1, Iy = gy >> 1;
                    const int px0 = Ix - (cx0 - 1);
                    const int px1 = min(max((gx & 1) ? Ix + 1 : Ix - 1, 0), nc - 1) - (cx0 - 1);
                    const int py0 = Iy - (cy0 - 1);
                    const int py1 = min(max((gy & 1) ? Iy + 1 : Iy - 1, 0), nc - 1) - (cy0 - 1);
                    const T a00 = w0 * Cz0[px0 + CW * py0] + w1 * Cz0[px1 + CW * py0];
                    const T a10 = w0 * Cz0[px0 + CW * py1] + w1 * Cz0[px1 + CW * py1];
                    const T a01 = w0 * Cz1[px0 + CW * py0] + w1 * Cz1[px1 + CW * py0];
                    const T a11 = w0 * Cz1[px0 + CW * py1] + w1 * Cz1[px1 + CW * py1];
                    const T pe = w0 * (w0 * a00 + w1 * a10) + w1 * (w0 * a01 + w1 * a11);
                    v = om * Bg[xi] * s_invD[nb_count1(gx, nf) + nb_count1(gy, nf) + kz] + pe;
                }
                Xg[xi] = v;
            }
        };
        const int cz0 = fz0 >> 1;
        PlaneRegs<T> pb;
        commit_c(fetch_c(cz0 - 1), cz0 - 1);
        commit_c(fetch_c(cz0), cz0);
        fetch_plane(pb, bs, nf, plane, fz0 - 1, fx0 - 4, fy0 - 1, BH, tid);
        commit_b(pb, fz0 - 1);
        __syncthreads();
        make_x(fz0 - 1);
        fetch_plane(pb, bs, nf, plane, fz0, fx0 - 4, fy0 - 1, BH, tid);
        T pc = fetch_c(cz0 + 1);
        for (int g = fz0; g <= fz0 + SZ; ++g) {
            if ((g & 1) == 0) commit_c(pc, (g >> 1) + 1);
            commit_b(pb, g);
            if (g + 1 <= fz0 + SZ) {
                fetch_plane(pb, bs, nf, plane, g + 1, fx0 - 4, fy0 - 1, BH, tid);
                if (((g + 1) & 1) == 0) pc = fetch_c(((g + 1) >> 1) + 1);
            }
            __syncthreads();
            make_x(g);
            __syncthreads();
            const int f = g - 1;  // output plane
            if (f >= fz0 && tid < SX * SY / 4) {
                const T* Xm = Xr + ring3(f - 1) * (PW * BH);
                const T* Xc = Xr + ring3(f) * (PW * BH);
                const T* Xp = Xr + ring3(f + 1) * (PW * BH);
                const T* Bc = B + ring3(f) * (PW * BH);
                const int kz = nb_count1(f, nf);
                const int oy = tid / (SX / 4), ox0 = 4 * (tid - oy * (SX / 4));
                const int gy = fy0 + oy;
                const int ky = nb_count1(gy, nf);
                V4<T> out;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int gx = fx0 + ox0 + e;
                    const int xi = (ox0 + e + 4) + PW * (oy + 1);
                    const T x0 = Xc[xi];
                    const T nbs = (Xc[xi - 1] + Xc[xi + 1]) + (Xc[xi - PW] + Xc[xi + PW]) + (Xm[xi] + Xp[xi]);
                    const int k0 = nb_count1(gx, nf) + ky + kz;
                    const T bv = Bc[xi];
                    const T yv = x0 + om * s_invD[k0] * (bv - q.s * (q.a * x0 + q.c * ((T)k0 * x0 - nbs)));
                    out.v[e] = yv;
                    dacc += (double)(bv * yv);
                }
                st4(ys + (fx0 + ox0) + (int64_t)nf * gy + plane * f, out);
            }
        }
        __syncthreads();
    }
    if (dot_part) {
        const double tsum = block_sum<kTileThreads>(dacc, red);
        if (tid == 0) dot_part[(int64_t)col * kMaxPartials + blockIdx.x] = tsum;
    }
}

// ---------------------------------------------------------------------------
// All levels n_l <= 16 in one CTA per sample (shared memory).
// ---------------------------------------------------------------------------
struct CoarseDesc {
    int lc;        // first (absolute) level handled here
    int nlev;      // total number of levels (n_{nlev-1} = 1)
    int n0;        // n_lc
    double kh2, c, omega;
};

template <typename T>
__device__ __forceinline__ T cz_invD(const CoarseDesc& d, int l, int k) {
    const T s = (T)(1 << l);
    const T a = (T)(d.kh2 * (double)(1ll << (2 * l)));
    return T(1) / (s * (a + (T)d.c * (T)k));
}

template <typename T>
__device__ __forceinline__ T cz_Ax(const CoarseDesc& d, int l, const T* x, int n, int i, int j, int k) {
    const int f = i + n * (j + n * k);
    const T x0 = x[f];
    T lap = T(0);
    if (i > 0) lap += x0 - x[f - 1];
    if (i < n - 1) lap += x0 - x[f + 1];
    if (j > 0) lap += x0 - x[f - n];
    if (j < n - 1) lap += x0 - x[f + n];
    if (k > 0) lap += x0 - x[f - n * n];
    if (k < n - 1) lap += x0 - x[f + n * n];
    const T s = (T)(1 << l);
    const T a = (T)(d.kh2 * (double)(1ll << (2 * l)));
    return s * (a * x0 + (T)d.c * lap);
}

template <typename T>
__global__ void __launch_bounds__(kCoarseThreads) k_mg_coarse(CoarseDesc d, const T* __restrict__ bin, int64_t b_stride,
                                                              T* __restrict__ eout, int64_t e_stride,
                                                              double* __restrict__ dot_part,
                                                              const int* __restrict__ active, int act_stride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[kCoarseThreads / 32];
    T* sm = reinterpret_cast<T*>(smem_raw);
    const int col = blockIdx.x;
    if (active && !active[(int64_t)col * act_stride]) return;
    // layout: b_l and x_l for l = lc .. nlev-1, then a temp of n0^3
    int offb[16], offx[16], nn[16];
    int o = 0;
    for (int l = d.lc; l < d.nlev; ++l) {
        const int n = d.n0 >> (l - d.lc);
        nn[l] = n;
        offb[l] = o;
        o += n * n * n;
        offx[l] = o;
        o += n * n * n;
    }
    T* tmp = sm + o;
    const T* bs = bin + (int64_t)col * b_stride;
    T* es = eout + (int64_t)col * e_stride;
    {
        const int n = d.n0, n3 = n * n * n;
        for (int f = threadIdx.x; f < n3; f += blockDim.x) sm[offb[d.lc] + f] = bs[f];
    }
    __syncthreads();
    const T om = (T)d.omega;
    // down
    for (int l = d.lc; l < d.nlev - 1; ++l) {
        const int n = nn[l], n3 = n * n * n, nc = n >> 1;
        T* b = sm + offb[l];
        T* x = sm + offx[l];
        for (int f = threadIdx.x; f < n3; f += blockDim.x) {
            const int i = f % n, j = (f / n) % n, k = f / (n * n);
            x[f] = om * b[f] * cz_invD<T>(d, l, nb_count1(i, n) + nb_count1(j, n) + nb_count1(k, n));
        }
        __syncthreads();
        for (int f = threadIdx.x; f < n3; f += blockDim.x) {
            const int i = f % n, j = (f / n) % n, k = f / (n * n);
            tmp[f] = b[f] - cz_Ax<T>(d, l, x, n, i, j, k);
        }
        __syncthreads();
        T* bc = sm + offb[l + 1];
        for (int C = threadIdx.x; C < nc * nc * nc; C += blockDim.x) {
            const int I = C % nc, J = (C / nc) % nc, K = C / (nc * nc);
            T acc = T(0);
            for (int c3 = 0; c3 < 4; ++c3) {
                const int fk = 2 * K - 1 + c3;
                const T wz = (T)restrict_w(c3, K, nc);
                if (wz == T(0)) continue;
                for (int b3 = 0; b3 < 4; ++b3) {
                    const int fj = 2 * J - 1 + b3;
                    const T wy = (T)restrict_w(b3, J, nc) * wz;
                    if (wy == T(0)) continue;
                    for (int a3 = 0; a3 < 4; ++a3) {
                        const int fi = 2 * I - 1 + a3;
                        const T w = (T)restrict_w(a3, I, nc) * wy;
                        if (w == T(0)) continue;
                        acc += w * tmp[fi + n * (fj + n * fk)];
                    }
                }
            }
            bc[C] = acc;
        }
        __syncthreads();
    }
    // bottom: one cell, exact
    {
        const int l = d.nlev - 1;
        if (threadIdx.x == 0) sm[offx[l]] = sm[offb[l]] * cz_invD<T>(d, l, 0);
        __syncthreads();
    }
    // up
    for (int l = d.nlev - 2; l >= d.lc; --l) {
        const int n = nn[l], n3 = n * n * n, nc = n >> 1;
        const T* b = sm + offb[l];
        T* x = sm + offx[l];
        const T* e = sm + offx[l + 1];
        for (int f = threadIdx.x; f < n3; f += blockDim.x) {
            const int i = f % n, j = (f / n) % n, k = f / (n * n);
            const int Ix = i >> 1, Iy = j >> 1, Iz = k >> 1;
            const int Ox = min(max((i & 1) ? Ix + 1 : Ix - 1, 0), nc - 1);
            const int Oy = min(max((j & 1) ? Iy + 1 : Iy - 1, 0), nc - 1);
            const int Oz = min(max((k & 1) ? Iz + 1 : Iz - 1, 0), nc - 1);
            const int px[2] = {Ix, Ox}, py[2] = {Iy, Oy}, pz[2] = {Iz, Oz};
            const T w[2] = {T(0.75), T(0.25)};
            T pe = T(0);
            for (int c3 = 0; c3 < 2; ++c3)
                for (int b3 = 0; b3 < 2; ++b3)
                    for (int a3 = 0; a3 < 2; ++a3) pe += w[a3] * w[b3] * w[c3] * e[px[a3] + nc * (py[b3] + nc * pz[c3])];
            tmp[f] = x[f] + pe;
        }
        __syncthreads();
        for (int f = threadIdx.x; f < n3; f += blockDim.x) {
            const int i = f % n, j = (f / n) % n, k = f / (n * n);
            const T iD = cz_invD<T>(d, l, nb_count1(i, n) + nb_count1(j, n) + nb_count1(k, n));
            x[f] = tmp[f] + om * iD * (b[f] - cz_Ax<T>(d, l, tmp, n, i, j, k));
        }
        __syncthreads();
    }
    // write out (and b.e partial when this is the whole V-cycle)
    double dacc = 0.0;
    {
        const int n = d.n0, n3 = n * n * n;
        const T* x = sm + offx[d.lc];
        const T* b = sm + offb[d.lc];
        for (int f = threadIdx.x; f < n3; f += blockDim.x) {
            es[f] = x[f];
            dacc += (double)(b[f] * x[f]);
        }
    }
    if (dot_part) {
        const double tsum = block_sum<kCoarseThreads>(dacc, red);
        if (threadIdx.x == 0) dot_part[(int64_t)col * kMaxPartials] = tsum;
    }
}

static int coarse_smem_elems(int n0, int lc, int nlev) {
    int o = 0;
    for (int l = lc; l < nlev; ++l) {
        const int n = n0 >> (l - lc);
        o += 2 * n * n * n;
    }
    return o + n0 * n0 * n0;
}

void mg_plan_init(MGPlan& plan, int n, double kh2, double c, double omega) {
    plan.n = n;
    plan.kh2 = kh2;
    plan.c = c;
    plan.omega = omega;
    int nlev = 1;
    while ((n >> (nlev - 1)) > 1) ++nlev;
    plan.nlev = nlev;
    int lc = 0;
    while ((n >> lc) > 16) ++lc;
    plan.lc = lc;
}

template <typename T>
size_t mg_scratch_elems(int n, int S) {
    MGPlan p;
    mg_plan_init(p, n, 0.0, 1.0, 0.8);
    size_t tot = 0;
    for (int l = 1; l <= p.lc; ++l) {
        const size_t nl = (size_t)(n >> l);
        tot += 2 * nl * nl * nl;
    }
    return tot * (size_t)S;
}

template <typename T>
void mg_plan_bind(MGPlan& plan, int S, T* scratch) {
    size_t o = 0;
    for (int l = 1; l <= plan.lc; ++l) {
        const size_t nl = (size_t)(plan.n >> l);
        plan.b[l] = scratch + o;
        o += nl * nl * nl * (size_t)S;
        plan.e[l] = scratch + o;
        o += nl * nl * nl * (size_t)S;
    }
}

template <typename T>
static cudaError_t mg_attrs() {
    static bool done = false;  // set once per instantiation and process
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_mg_coarse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         coarse_smem_elems(16, 0, 5) * (int)sizeof(T));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mg_down<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kDownSSmem * (int)sizeof(T));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mg_up<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kUpSSmem * (int)sizeof(T));
    if (e == cudaSuccess) done = true;
    return e;
}

template <typename T>
int launch_vcycle(const MGPlan& plan, int S, const T* b, int64_t b_stride, T* y, int64_t y_stride, double* dot_part,
                  const int* active, int act_stride, cudaStream_t st) {
    const double prof_cols = plan.prof_cols > 0 ? plan.prof_cols : (double)S;
    if (mg_attrs<T>() != cudaSuccess) return -1;
    const int n = plan.n;
    CoarseDesc d;
    d.lc = plan.lc;
    d.nlev = plan.nlev;
    d.n0 = n >> plan.lc;
    d.kh2 = plan.kh2;
    d.c = plan.c;
    d.omega = plan.omega;
    const size_t csm = (size_t)coarse_smem_elems(d.n0, d.lc, d.nlev) * sizeof(T);
    const double w = (double)sizeof(T);
    const double n0c = (double)d.n0 * d.n0 * d.n0;
    if (plan.lc == 0) {
        prof_begin(PK_MG_COARSE, st);
        k_mg_coarse<T><<<S, kCoarseThreads, csm, st>>>(d, b, b_stride, y, y_stride, dot_part, active, act_stride);
        prof_end(st, prof_cols * 2.0 * n0c * w);
        return 1;
    }
    // down sweeps
    const T* in = b;
    int64_t in_stride = b_stride;
    for (int l = 0; l < plan.lc; ++l) {
        const int nf = n >> l, nc = nf >> 1;
        const int ntiles = (nf / SX) * (nf / SY) * (nf / SZ);
        dim3 grid(ntiles < kMaxTilesPerCol ? ntiles : kMaxTilesPerCol, S);
        T* out = static_cast<T*>(plan.b[l + 1]);
        prof_begin(PK_MG_DOWN, st);
        k_mg_down<T><<<grid, dim3(32, 8), kDownSSmem * sizeof(T), st>>>(nf, level_coef<T>(plan, l), in, in_stride, out,
                                                    (int64_t)nc * nc * nc, active, act_stride);
        prof_end(st, prof_cols * (1.0 + 0.125) * (double)nf * nf * nf * w);
        in = out;
        in_stride = (int64_t)nc * nc * nc;
    }
    {
        const int64_t s3 = (int64_t)d.n0 * d.n0 * d.n0;
        prof_begin(PK_MG_COARSE, st);
        k_mg_coarse<T><<<S, kCoarseThreads, csm, st>>>(d, static_cast<const T*>(plan.b[plan.lc]), s3,
                                                       static_cast<T*>(plan.e[plan.lc]), s3, nullptr, active,
                                                       act_stride);
        prof_end(st, prof_cols * 2.0 * n0c * w);
    }
    int nblk0 = 1;
    for (int l = plan.lc - 1; l >= 0; --l) {
        const int nf = n >> l, nc = nf >> 1;
        const int ntiles = (nf / SX) * (nf / SY) * (nf / SZ);
        const int nb = ntiles < kMaxTilesPerCol ? ntiles : kMaxTilesPerCol;
        dim3 grid(nb, S);
        const T* bl = (l == 0) ? b : static_cast<const T*>(plan.b[l]);
        const int64_t bls = (l == 0) ? b_stride : (int64_t)nf * nf * nf;
        T* yl = (l == 0) ? y : static_cast<T*>(plan.e[l]);
        const int64_t yls = (l == 0) ? y_stride : (int64_t)nf * nf * nf;
        prof_begin(PK_MG_UP, st);
        k_mg_up<T><<<grid, dim3(32, 8), kUpSSmem * sizeof(T), st>>>(nf, level_coef<T>(plan, l), bl, bls,
                                                  static_cast<const T*>(plan.e[l + 1]), (int64_t)nc * nc * nc, yl,
                                                  yls, (l == 0) ? dot_part : nullptr, active, act_stride);
        prof_end(st, prof_cols * (2.0 + 0.125) * (double)nf * nf * nf * w);
        if (l == 0) nblk0 = nb;
    }
    return nblk0;
}

#define SPDE_MG_INST(T)                                                                                            \
    template int launch_vcycle<T>(const MGPlan&, int, const T*, int64_t, T*, int64_t, double*, const int*, int,   \
                                  cudaStream_t);                                                                   \
    template size_t mg_scratch_elems<T>(int, int);                                                                 \
    template void mg_plan_bind<T>(MGPlan&, int, T*);
SPDE_MG_INST(float)
SPDE_MG_INST(double)

}  // namespace spde
