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
constexpr int SX = 32, SY = 16;  // the z extent per CTA (8, 16 or 32 planes) is chosen per launch
constexpr int PW = SX + 8;               // plane row width in shared memory (x from fx0 - 4)
constexpr int XH = SY + 4;               // x0 rows, halo 2 (down sweep)
constexpr int RW = SX + 2, RH = SY + 2;  // residual plane, halo 1
constexpr int BH = SY + 2;               // b / x rows, halo 1 (up sweep)
constexpr int CW = SX / 2 + 2, CH = SY / 2 + 2;  // coarse plane with halo 1 (up sweep)
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
// Per fine plane f: store the x0 plane f+1, fetch plane f+2, form r on plane
// f and restrict it in x and y at once (Rxy, 16 x 8 values); every second
// plane one coarse plane is the 4-tap z combination of four Rxy planes.
// Each thread's plane positions (offsets, neighbour counts, box tests) are
// fixed for a tile and computed once before the z-march.
// ---------------------------------------------------------------------------
constexpr int kRS = (RW * RH + kTileThreads - 1) / kTileThreads;  // r positions per thread (3)
constexpr int RXY = (SX / 2) * (SY / 2);                            // restricted plane (128)
constexpr int kDownS2Smem = 3 * PW * XH + RW * RH + 4 * RXY;

template <typename T>
__global__ void __launch_bounds__(kTileThreads, 4) k_mg_down(int nf, int SZ, LevelCoef<T> q, const T* __restrict__ b,
                                                             int64_t b_stride, T* __restrict__ bc, int64_t bc_stride,
                                                             const int* __restrict__ active, int act_stride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ T s_invD[8], s_D[8];
    T* const Xbase = reinterpret_cast<T*>(smem_raw);  // 3 x0 planes, PW x XH
    T* const Rp = Xbase + 3 * PW * XH;                 // residual plane, RW x RH
    T* const Rxy = Rp + RW * RH;                       // 4 x-y restricted planes
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
        // --- per-tile slot data
        // commit: one 4-wide row segment per thread (tid < kQ * XH)
        int c_off = -1, c_k[4] = {0, 0, 0, 0};
        if (tid < kQ * XH) {
            const int ly = tid / kQ, q4 = tid - ly * kQ;
            const int gy = fy0 - 2 + ly;
            const int ky = ((unsigned)gy < (unsigned)nf) ? nb_count1(gy, nf) : 0;
            c_off = 4 * q4 + PW * ly;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int gx = fx0 - 4 + 4 * q4 + e;
                c_k[e] = ky + (((unsigned)gx < (unsigned)nf) ? nb_count1(gx, nf) : 0);
            }
        }
        // residual positions: X offset and kx + ky, or -1 when outside the box in x/y
        int r_xi[kRS], r_k[kRS];
#pragma unroll
        for (int u = 0; u < kRS; ++u) {
            const int idx = tid + u * kTileThreads;
            r_xi[u] = 0;
            r_k[u] = -2;  // -2: no position; -1: outside the box
            if (idx < RW * RH) {
                const int ly = idx / RW, lx = idx - ly * RW;
                const int gx = fx0 - 1 + lx, gy = fy0 - 1 + ly;
                r_xi[u] = (lx + 3) + PW * (ly + 1);
                r_k[u] = ((unsigned)gx < (unsigned)nf && (unsigned)gy < (unsigned)nf)
                             ? nb_count1(gx, nf) + nb_count1(gy, nf)
                             : -1;
            }
        }
        // x-y restriction of one coarse (I, J) per thread (tid < RXY)
        T wx[4], wy[4];
        int rb = 0;
        {
            const int li = tid & (SX / 2 - 1), lj = (tid / (SX / 2)) & (SY / 2 - 1);
            const int I = cx0 + li, J = cy0 + lj;
#pragma unroll
            for (int a3 = 0; a3 < 4; ++a3) {
                wx[a3] = (T)restrict_w(a3, I, nc);
                wy[a3] = (T)restrict_w(a3, J, nc);
            }
            rb = 2 * li + RW * (2 * lj);
        }
        T* Xm = Xbase;
        T* Xc = Xbase + PW * XH;
        T* Xp = Xbase + 2 * PW * XH;
        auto commit = [&](const PlaneRegs<T>& r, T* dst, int f) {
            const int kz = ((unsigned)f < (unsigned)nf) ? nb_count1(f, nf) : 0;
            if (c_off >= 0) {
                V4<T> v;
#pragma unroll
                for (int e = 0; e < 4; ++e) v.v[e] = om * r.v[0].v[e] * s_invD[c_k[e] + kz];
                st4(dst + c_off, v);
            }
        };
        PlaneRegs<T> pr;
        fetch_plane(pr, bs, nf, plane, fz0 - 2, fx0 - 4, fy0 - 2, XH, tid);
        commit(pr, Xm, fz0 - 2);
        fetch_plane(pr, bs, nf, plane, fz0 - 1, fx0 - 4, fy0 - 2, XH, tid);
        commit(pr, Xc, fz0 - 1);
        fetch_plane(pr, bs, nf, plane, fz0, fx0 - 4, fy0 - 2, XH, tid);
        for (int f = fz0 - 1; f <= fz0 + SZ; ++f) {
            commit(pr, Xp, f + 1);
            if (f + 2 <= fz0 + SZ + 1) fetch_plane(pr, bs, nf, plane, f + 2, fx0 - 4, fy0 - 2, XH, tid);
            __syncthreads();
            {
                const bool zin = (unsigned)f < (unsigned)nf;
                const int kz = zin ? nb_count1(f, nf) : 0;
#pragma unroll
                for (int u = 0; u < kRS; ++u) {
                    if (r_k[u] == -2) continue;
                    T r = T(0);
                    if (zin && r_k[u] >= 0) {
                        const int xi = r_xi[u];
                        const T nbs = (Xc[xi - 1] + Xc[xi + 1]) + (Xc[xi - PW] + Xc[xi + PW]) + (Xm[xi] + Xp[xi]);
                        r = rc * s_D[r_k[u] + kz] * Xc[xi] + sc * nbs;
                    }
                    Rp[tid + u * kTileThreads] = r;
                }
            }
            __syncthreads();
            if (tid < RXY) {
                T acc = T(0);
#pragma unroll
                for (int b3 = 0; b3 < 4; ++b3) {
                    const T* row = Rp + rb + RW * b3;
                    acc += wy[b3] * (wx[0] * row[0] + wx[1] * row[1] + wx[2] * row[2] + wx[3] * row[3]);
                }
                Rxy[ring4(f) * RXY + tid] = acc;
                if (f >= fz0 + 2 && ((f - fz0) & 1) == 0) {
                    // coarse plane Z = f/2 - 1 from the x-y restricted planes 2Z-1 .. 2Z+2 = f-3 .. f
                    const int Z = (f - 2) >> 1;
                    T z = T(0);
#pragma unroll
                    for (int c3 = 0; c3 < 4; ++c3)
                        z += (T)restrict_w(c3, Z, nc) * ((c3 == 3) ? acc : Rxy[ring4(f - 3 + c3) * RXY + tid]);
                    const int li = tid & (SX / 2 - 1), lj = tid / (SX / 2);
                    bcs[(cx0 + li) + (int64_t)nc * ((cy0 + lj) + (int64_t)nc * Z)] = z;
                }
            }
            T* t = Xm;
            Xm = Xc;
            Xc = Xp;
            Xp = t;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Up sweep at level l: x = omega D^{-1} b + P ec ; y = x + omega D^{-1} (b - A x),
// optional partial sums of b.y (the MINRES beta^2 contribution).  Per fine
// plane g: store b(g) and (for even g) coarse plane g/2 + 1, fetch the next
// ones, form x(g) on the tile + halo 1, then y(g - 1) from x planes g-2 .. g.
// Per-thread positions, neighbour counts and prolongation offsets are fixed
// for a tile and computed once before the z-march.
// ---------------------------------------------------------------------------
constexpr int kXS = (RW * BH + kTileThreads - 1) / kTileThreads;  // x positions per thread (3)

template <typename T>
__global__ void __launch_bounds__(kTileThreads, 3) k_mg_up(int nf, int SZ, LevelCoef<T> q, const T* __restrict__ b,
                                                           int64_t b_stride, const T* __restrict__ ec,
                                                           int64_t ec_stride, T* __restrict__ y, int64_t y_stride,
                                                           double* __restrict__ dot_part,
                                                           const int* __restrict__ active, int act_stride) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[kTileThreads / 32];
    __shared__ T s_invD[8], s_D[8];
    T* const Bbase = reinterpret_cast<T*>(smem_raw);  // 3 b planes, PW x BH
    T* const Xbase = Bbase + 3 * PW * BH;              // 3 x planes, PW x BH
    T* const Cbase = Xbase + 3 * PW * BH;              // 3 coarse planes, CW x CH
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
    T dacc = T(0);  // per-thread partial of b.y in the element type; FP64 across threads
    __syncthreads();
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tX = tile % ntx, tY = (tile / ntx) % nty, tZ = tile / (ntx * nty);
        const int fx0 = tX * SX, fy0 = tY * SY, fz0 = tZ * SZ;
        const int cx0 = fx0 >> 1, cy0 = fy0 >> 1;
        const int cz0 = fz0 >> 1;
        // --- per-tile slot data
        int c_src = -1;  // coarse plane element of this thread (clamped x, y), or -1
        if (tid < CW * CH) {
            const int ly = tid / CW, lx = tid - ly * CW;
            const int gx = min(max(cx0 - 1 + lx, 0), nc - 1), gy = min(max(cy0 - 1 + ly, 0), nc - 1);
            c_src = gx + nc * gy;
        }
        int x_xi[kXS], x_k[kXS], x_c00[kXS], x_c10[kXS], x_c01[kXS], x_c11[kXS];
#pragma unroll
        for (int u = 0; u < kXS; ++u) {
            const int idx = tid + u * kTileThreads;
            x_xi[u] = 0;
            x_k[u] = -2;
            x_c00[u] = x_c10[u] = x_c01[u] = x_c11[u] = 0;
            if (idx < RW * BH) {
                const int ly = idx / RW, lx = idx - ly * RW;
                const int gx = fx0 - 1 + lx, gy = fy0 - 1 + ly;
                x_xi[u] = (lx + 3) + PW * ly;
                if ((unsigned)gx < (unsigned)nf && (unsigned)gy < (unsigned)nf) {
                    x_k[u] = nb_count1(gx, nf) + nb_count1(gy, nf);
                    const int Ix = gx >> 1, Iy = gy >> 1;
                    const int px0 = Ix - (cx0 - 1);
                    const int px1 = min(max((gx & 1) ? Ix + 1 : Ix - 1, 0), nc - 1) - (cx0 - 1);
                    const int py0 = Iy - (cy0 - 1);
                    const int py1 = min(max((gy & 1) ? Iy + 1 : Iy - 1, 0), nc - 1) - (cy0 - 1);
                    x_c00[u] = px0 + CW * py0;
                    x_c10[u] = px1 + CW * py0;
                    x_c01[u] = px0 + CW * py1;
                    x_c11[u] = px1 + CW * py1;
                } else {
                    x_k[u] = -1;
                }
            }
        }
        // output: 4 consecutive cells per thread (tid < SX * SY / 4)
        const int oy = tid / (SX / 4), ox0 = 4 * (tid - oy * (SX / 4));
        const bool has_out = tid < SX * SY / 4;
        const int o_xi = (ox0 + 4) + PW * (oy + 1);
        int o_k[4];
        {
            const int ky = has_out ? nb_count1(fy0 + oy, nf) : 0;
#pragma unroll
            for (int e = 0; e < 4; ++e) o_k[e] = ky + (has_out ? nb_count1(fx0 + ox0 + e, nf) : 0);
        }
        T* Bm = Bbase;  // b planes g-2, g-1, g (rotating)
        T* Bc = Bbase + PW * BH;
        T* Bp = Bbase + 2 * PW * BH;
        T* Xm = Xbase;  // x planes g-2, g-1, g (rotating)
        T* Xc = Xbase + PW * BH;
        T* Xp = Xbase + 2 * PW * BH;
        T* Cm = Cbase;  // coarse planes Z-1, Z, Z+1 with Z = g >> 1 (rotating at even g)
        T* Cc = Cbase + CW * CH;
        T* Cp = Cbase + 2 * CW * CH;
        auto fetch_c = [&](int Z) -> T {
            return (c_src >= 0) ? es[c_src + cplane * min(max(Z, 0), nc - 1)] : T(0);
        };
        auto commit_b = [&](const PlaneRegs<T>& r, T* dst) {
            if (tid < kQ * BH) st4(dst + 4 * tid, r.v[0]);
        };
        auto make_x = [&](int g, const T* Bg, T* Xg, const T* C0, const T* C1) {
            const bool zin = (unsigned)g < (unsigned)nf;
            const int kz = zin ? nb_count1(g, nf) : 0;
#pragma unroll
            for (int u = 0; u < kXS; ++u) {
                if (x_k[u] == -2) continue;
                T v = T(0);
                if (zin && x_k[u] >= 0) {
                    const T a00 = w0 * C0[x_c00[u]] + w1 * C0[x_c10[u]];
                    const T a10 = w0 * C0[x_c01[u]] + w1 * C0[x_c11[u]];
                    const T a01 = w0 * C1[x_c00[u]] + w1 * C1[x_c10[u]];
                    const T a11 = w0 * C1[x_c01[u]] + w1 * C1[x_c11[u]];
                    const T pe = w0 * (w0 * a00 + w1 * a10) + w1 * (w0 * a01 + w1 * a11);
                    v = om * Bg[x_xi[u]] * s_invD[x_k[u] + kz] + pe;
                }
                Xg[x_xi[u]] = v;
            }
        };
        PlaneRegs<T> pb;
        // prologue: coarse planes cz0-1 (Cc role for g = fz0-1 -> Iz = cz0-1) and cz0
        if (c_src >= 0) {
            Cc[tid] = fetch_c(cz0 - 1);
            Cp[tid] = fetch_c(cz0);
        }
        fetch_plane(pb, bs, nf, plane, fz0 - 1, fx0 - 4, fy0 - 1, BH, tid);
        commit_b(pb, Bp);
        __syncthreads();
        make_x(fz0 - 1, Bp, Xp, Cc, Cp);  // odd g: planes Iz and Iz + 1
        fetch_plane(pb, bs, nf, plane, fz0, fx0 - 4, fy0 - 1, BH, tid);
        T pc = fetch_c(cz0 + 1);
        for (int g = fz0; g <= fz0 + SZ; ++g) {
            // rotate roles: plane g goes to the freed slot
            {
                T* t = Bm;
                Bm = Bc;
                Bc = Bp;
                Bp = t;
                t = Xm;
                Xm = Xc;
                Xc = Xp;
                Xp = t;
            }
            if ((g & 1) == 0) {  // Z = g/2: coarse roles become (Z-1, Z, Z+1)
                T* t = Cm;
                Cm = Cc;
                Cc = Cp;
                Cp = t;
                if (c_src >= 0) Cp[tid] = pc;
            }
            commit_b(pb, Bp);
            if (g + 1 <= fz0 + SZ) {
                fetch_plane(pb, bs, nf, plane, g + 1, fx0 - 4, fy0 - 1, BH, tid);
                if (((g + 1) & 1) == 0) pc = fetch_c(((g + 1) >> 1) + 1);
            }
            __syncthreads();
            if ((g & 1) == 0) make_x(g, Bp, Xp, Cc, Cm);  // even g: planes Iz and Iz - 1
            else make_x(g, Bp, Xp, Cc, Cp);               // odd g: planes Iz and Iz + 1
            __syncthreads();
            const int f = g - 1;  // output plane: x planes f-1, f, f+1 = Xm, Xc, Xp; b(f) = Bc
            if (f >= fz0 && has_out) {
                const int kz = nb_count1(f, nf);
                V4<T> out;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int xi = o_xi + e;
                    const T x0 = Xc[xi];
                    const T nbs = (Xc[xi - 1] + Xc[xi + 1]) + (Xc[xi - PW] + Xc[xi + PW]) + (Xm[xi] + Xp[xi]);
                    const int k0 = o_k[e] + kz;
                    const T bv = Bc[xi];
                    const T yv = x0 + om * s_invD[k0] * (bv - q.s * (q.a * x0 + q.c * ((T)k0 * x0 - nbs)));
                    out.v[e] = yv;
                    dacc += bv * yv;
                }
                st4(ys + (fx0 + ox0) + (int64_t)nf * (fy0 + oy) + plane * f, out);
            }
        }
        __syncthreads();
    }
    if (dot_part) {
        const double tsum = block_sum<kTileThreads>((double)dacc, red);
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

// z planes per CTA for the level sweeps: the longest march (fewest halo planes)
// that still gives at least four CTAs per SM of a 152-SM GPU
static int pick_sz(int nf, int S) {
    const int base = (nf / SX) * (nf / SY);
    for (int sz = 32; sz > 8; sz >>= 1)
        if (nf % sz == 0 && (int64_t)base * (nf / sz) * S >= 4 * 152) return sz;
    return 8;
}

template <typename T>
static cudaError_t mg_set_attrs() {
    cudaError_t e = cudaFuncSetAttribute(k_mg_coarse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         coarse_smem_elems(16, 0, 5) * (int)sizeof(T));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mg_down<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kDownS2Smem * (int)sizeof(T));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mg_up<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kUpSSmem * (int)sizeof(T));
    return e;
}

// once per instantiation and process (thread-safe static initialisation)
template <typename T>
static cudaError_t mg_attrs() {
    static const cudaError_t e = mg_set_attrs<T>();
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
        const int sz = pick_sz(nf, S);
        const int ntiles = (nf / SX) * (nf / SY) * (nf / sz);
        dim3 grid(ntiles < kMaxTilesPerCol ? ntiles : kMaxTilesPerCol, S);
        T* out = static_cast<T*>(plan.b[l + 1]);
        prof_begin(PK_MG_DOWN, st);
        k_mg_down<T><<<grid, dim3(32, 8), kDownS2Smem * sizeof(T), st>>>(nf, sz, level_coef<T>(plan, l), in, in_stride, out,
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
        const int sz = pick_sz(nf, S);
        const int ntiles = (nf / SX) * (nf / SY) * (nf / sz);
        const int nb = ntiles < kMaxTilesPerCol ? ntiles : kMaxTilesPerCol;
        dim3 grid(nb, S);
        const T* bl = (l == 0) ? b : static_cast<const T*>(plan.b[l]);
        const int64_t bls = (l == 0) ? b_stride : (int64_t)nf * nf * nf;
        T* yl = (l == 0) ? y : static_cast<T*>(plan.e[l]);
        const int64_t yls = (l == 0) ? y_stride : (int64_t)nf * nf * nf;
        prof_begin(PK_MG_UP, st);
        k_mg_up<T><<<grid, dim3(32, 8), kUpSSmem * sizeof(T), st>>>(nf, sz, level_coef<T>(plan, l), bl, bls,
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
