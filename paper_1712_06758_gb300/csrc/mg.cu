// K3: field block of the MINRES preconditioner -- one symmetric geometric
// multigrid V-cycle for the cell-centred 7-point Schur approximation
//     A_0 = (kappa h)^2 I + c L          (L: Neumann graph Laplacian)
// on the nested embedding grids of Sec. 6.1.
//
// Level l + 1 halves every extent of level l that is above 1 (on a cube of n
// cells per axis: n_l = n >> l).  Level operator
//     A_l = s_l ((kappa h)^2 q_l I + c L_l),   D_l = diag(A_l),
// with q_l = 4^l and s_l the product over the coarsenings above it of
// (children per coarse cell) / 4, i.e. s_l = 2^l while all three axes halve
// (the rediscretised operator); an axis of extent 1 has no neighbours, so one
// weight serves every axis.  Transfers P = tensor product of the 1-D
// cell-centred linear prolongation
//     fine 2I <- 3/4 e_I + 1/4 e_{I-1},  fine 2I+1 <- 3/4 e_I + 1/4 e_{I+1}
// (indices clamped at the walls: reflection for the no-flux boundary; the
// identity along an axis that is not coarsened) and R = P^T.  Each level:
// x = omega D^{-1} b (one Jacobi sweep from zero), coarse correction with
// r = b - A x, then one more Jacobi sweep; the one-cell level is solved
// exactly.  Same sweep before and after makes the operator symmetric; with
// 0 < omega < 1 it is positive definite, as MINRES needs.
//
// Kernels: levels whose extents are multiples of the tile (32 x 16 x 8) use
// shared-memory tiles (a down sweep that smooths, forms the residual and
// restricts in one pass; an up sweep that prolongs, corrects and post-smooths
// in one pass).  The remaining levels (at most 4096 cells) run inside one CTA
// per sample in shared memory.
#include <cuda.h>  // CUtensorMap and its enums (the encoder is fetched from the driver at run time)

#include <cuda_fp16.h>

#include <type_traits>

#include "device.cuh"
#include "internal.h"
#include "prof.h"

namespace spde {

constexpr int kTileThreads = 256;
constexpr int kCoarseThreads = 1024;  // one CTA per column: 1024 threads measured 9 % faster than 512
constexpr int kMaxTilesPerCol = 2048;

template <typename T>
struct LevelCoef {
    T s;         // 2^l
    T c;         // Schur weight
    T omega;
    T oi[7];     // omega / D(k), D(k) = s (a + c k), a = (kappa h)^2 4^l, k existing neighbours
    T ois[7];    // omega s c / D(k)
    T rcD[7];    // (1/omega - 1) D(k)
};

template <typename T>
static LevelCoef<T> level_coef(const MGPlan& p, int l) {
    LevelCoef<T> q;
    const double s = p.ls[l];
    const double a = p.kh2 * p.lq[l];
    q.s = (T)s;
    q.c = (T)p.c;
    q.omega = (T)p.omega;
    for (int k = 0; k <= 6; ++k) {
        const double D = s * (a + p.c * k);
        q.oi[k] = (T)(p.omega / D);
        q.ois[k] = (T)(p.omega * s * p.c / D);
        q.rcD[k] = (T)((1.0 / p.omega - 1.0) * D);
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

__device__ __forceinline__ bool in_range(int i, int n) { return (unsigned)i < (unsigned)n; }

template <typename T>
struct V2 {
    T v[2];
};

template <typename T>
__device__ __forceinline__ V2<T> ld2(const T* p) {
    V2<T> r;
    if constexpr (sizeof(T) == 4) {
        const float2 f = *reinterpret_cast<const float2*>(p);
        r.v[0] = f.x;
        r.v[1] = f.y;
    } else {
        const double2 f = *reinterpret_cast<const double2*>(p);
        r.v[0] = f.x;
        r.v[1] = f.y;
    }
    return r;
}

// Sums of products with the rounding spelled out (which product is fused is otherwise the
// compiler's choice), so that sweeps that tile the grid differently give the same bits.
template <typename T>
__device__ __forceinline__ T mad2(T a, T b, T c, T d) {  // a b + c d
    return fma(a, b, c * d);
}
template <typename T>
__device__ __forceinline__ T mad4(const T w[4], T a, T b, T c, T d) {  // w0 a + w1 b + w2 c + w3 d
    return fma(w[3], d, fma(w[2], c, fma(w[1], b, w[0] * a)));
}
// prolongation weights 3/4 (own coarse cell) and 1/4 (its neighbour) along one axis, then two
template <typename T>
__device__ __forceinline__ T blend2(T own, T nb) {
    return mad2(T(0.75), own, T(0.25), nb);
}
template <typename T>
__device__ __forceinline__ T blend4(T a, T c, T b, T d) {  // a, b: own z plane; c, d: its neighbour
    return mad2(T(0.75), blend2(a, c), T(0.25), blend2(b, d));
}

template <typename T>
__device__ __forceinline__ void st2(T* p, T a, T b) {
    if constexpr (sizeof(T) == 4) *reinterpret_cast<float2*>(p) = make_float2(a, b);
    else *reinterpret_cast<double2*>(p) = make_double2(a, b);
}

// Streaming sweeps: a CTA owns a fine (x, y) tile of SX x SY cells and marches
// along z through SZ fine planes, keeping a few planes in shared-memory rings
// (tiles and grids are multiples of 32, so a 4-cell vector of a plane row lies
// wholly inside or wholly outside the box).  All per-cell work runs on 4-cell x
// segments: the x neighbours of a segment are its own lanes plus one value on
// each side, the y and z neighbours are vectors of the adjacent rows and
// planes.  The marches are software-pipelined: each step works on three planes
// at different stages, on different warps, with one barrier per step.
constexpr int SX = 32, SY = 16;  // the z extent per CTA (8, 16 or 32 planes) is chosen per launch
constexpr int PW = SX + 8;       // plane row width in shared memory (x from fx0 - 4)
constexpr int kQ = PW / 4;       // 4-cell segments per plane row
constexpr int XH = SY + 4;       // down sweep: x0 rows, y from fy0 - 2
constexpr int RH = SY + 2;       // down sweep: residual rows, y from fy0 - 1
constexpr int BH = SY + 2;       // up sweep: b and x rows, y from fy0 - 1
constexpr int RXY = (SX / 2) * (SY / 2);          // x-y restricted plane (128)
constexpr int CW = SX / 2 + 6, CH = SY / 2 + 2;   // up sweep: coarse plane, x from cx0 - 3, y from cy0 - 1
constexpr int kDownSmem = 4 * PW * XH + 2 * PW * RH + 4 * RXY;
constexpr int kUpSmem = 4 * PW * BH + 4 * CW * CH;

__device__ __forceinline__ int ring4(int f) { return (f + 4) & 3; }  // f >= -4

// neighbour counts of the 4 cells of a segment in x and y, packed 3 bits each
__device__ __forceinline__ int kxy_of(int packed, int e) { return (packed >> (3 * e)) & 7; }

// ---------------------------------------------------------------------------
// Fine planes arrive by TMA: a 4-D tiled tensor map over [S][n][n][n] with a
// box of PW x rows x 1 x 1 elements (x from fx0 - 4, which keeps the start on a
// 16-byte boundary); coordinates outside the grid read as zero, which is the
// "zero outside the box" the sweeps need.  One thread issues the copies into a
// ring of plane slots, each completing on its own mbarrier.  Every wait is
// bounded (about one second on the global timer); a wait that gives up sets
// the CTA's abort flag and the fault word of the solve that launched the
// sweep (a device int the caller owns, one per workspace), later waits and
// later sweeps of that solve return at once and the host reports
// SPDE_ETIMEOUT.  Other solves, with their own words, are not affected.
// ---------------------------------------------------------------------------
constexpr int kRing = 4;  // plane slots of the TMA ring (both sweeps): the z-march is unrolled by 4
template <int K>
using IC = std::integral_constant<int, K>;
constexpr int kProducer = kTileThreads - 32;  // issues the plane copies: lane 0 of the last warp, which has no
                                              // segment work in the residual and prolongation phases
constexpr unsigned long long kWaitLimitNs = 1000000000ull;

template <typename T>
__host__ __device__ constexpr int slot_elems(int rows) {  // a plane slot, rounded up to 128 bytes
    return ((PW * rows * (int)sizeof(T) + 127) / 128) * 128 / (int)sizeof(T);
}
template <typename T>
__host__ __device__ constexpr int down_smem_bytes() {
    return 128 + (int)sizeof(T) * (kRing * slot_elems<T>(XH) + kDownSmem);
}
template <typename T>
__host__ __device__ constexpr int up_smem_bytes() {
    return 128 + (int)sizeof(T) * (kRing * slot_elems<T>(BH) + kUpSmem);
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait for the phase of the given parity; false when it gave up
__device__ __noinline__ bool mbar_wait_slow(uint64_t* bar, uint32_t parity) {
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (global_ns() - t0 > kWaitLimitNs) return false;
    }
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    return mbar_try(bar, parity) || mbar_wait_slow(bar, parity);
}

__device__ __forceinline__ void tma_plane(void* dst, const CUtensorMap* map, uint64_t* bar, uint32_t bytes, int x,
                                          int y, int z, int w) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_addr(bar))
        : "memory");
}

// The ring of one CTA.  Within a tile, tile plane j lives in slot j mod NS; the
// tile's planes are all issued and consumed before the next tile starts.  Every
// thread tracks, per slot, the parity of the next completion it waits for; the
// producer also tracks the slots whose copy it has not yet seen complete.
template <typename T, int NS>
struct PlaneRing {
    T* slots;
    int slot;            // elements per slot
    uint64_t* bars;
    volatile int* abort;
    int* fault;          // the solve's fault word
    uint32_t bytes;
    uint32_t ph = 0;     // bit s: parity of slot s's next completion
    uint32_t pend = 0;   // producer: bit s set while a copy into slot s is unobserved

    __device__ __forceinline__ T* at(int s) const { return slots + s * slot; }
    // producer thread only; false once the CTA has given up
    __device__ __forceinline__ bool issue(int s, const CUtensorMap* map, int x, int y, int z, int w) {
        if (*abort) return false;
        tma_plane(at(s), map, bars + s, bytes, x, y, z, w);
        pend |= 1u << s;
        return true;
    }
    __device__ __forceinline__ const T* take(int s) {
        const uint32_t par = (ph >> s) & 1u;
        ph ^= 1u << s;
        if (!*abort) {
            if (mbar_wait(bars + s, par)) pend &= ~(1u << s);
            else {
                *abort = 1;
                atomicExch(fault, 1);
            }
        }
        return at(s);
    }
    // producer thread, after an abort: bounded wait for copies still in flight (their
    // slots were taken without waiting, so each awaits the phase before the current one)
    __device__ void drain() {
        for (int s = 0; s < NS; ++s)
            if ((pend >> s) & 1u) mbar_wait(bars + s, ((ph >> s) & 1u) ^ 1u);
        pend = 0;
    }
};

template <typename T, int NS>
__device__ __forceinline__ PlaneRing<T, NS> ring_setup(unsigned char* raw, int rows, uint64_t* bars,
                                                       volatile int* abort, int* fault, int tid) {
    PlaneRing<T, NS> r;
    r.fault = fault;
    const uint32_t a = smem_addr(raw);
    r.slots = reinterpret_cast<T*>(raw + ((128 - (a & 127)) & 127));
    r.slot = slot_elems<T>(rows);
    r.bars = bars;
    r.abort = abort;
    r.bytes = (uint32_t)(PW * rows * sizeof(T));
    if (tid == kProducer) {
        for (int i = 0; i < NS; ++i) mbar_init(bars + i);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    return r;
}

// ---------------------------------------------------------------------------
// Down sweep at level l: bc = R (b - A omega D^{-1} b).  With x0 = omega D^{-1} b
//     r(f) = (1/omega - 1) D(f) x0(f) + s c sum_{neighbours g} x0(g)
// (x0 = 0 outside the box, so the sum runs over existing neighbours).
// Step t (fine plane f = fz0 - 1 + t): warps 0-6 store the x0 plane f+2 (tile +
// halo 2) from its b plane, warps 0-5 form r on plane f (tile + halo 1) from
// x0 planes f-1 .. f+1, and warps 6-7 restrict r(f-1) in x and y at once (Rxy,
// 16 x 8 values, two coarse x per thread); every second step one coarse plane
// is the 4-tap z combination of four Rxy planes (each thread reads back only
// its own Rxy entries).  x0 planes live in 4 slots, r planes in 2, Rxy in 4:
// with tiles starting on multiples of 4 planes, the z-march unrolled by 4 has
// every slot index fixed at compile time.
// ---------------------------------------------------------------------------
constexpr int kRestrictBase = kTileThreads - RXY / 2;  // the restriction threads: the last two warps

template <typename T, bool PC>  // PC: per-cell diagonal (cell-wise kappa) in Dg
__global__ void __launch_bounds__(kTileThreads, sizeof(T) == 4 ? 4 : 2)
    k_mg_down(const __grid_constant__ CUtensorMap bmap, Grid3 gf, int SZ, LevelCoef<T> q, T* __restrict__ bc,
              int64_t bc_stride, const int* __restrict__ active, int act_stride, const T* __restrict__ Dg,
              int* __restrict__ fault, const T* __restrict__ qtab) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ T s_oi[8], s_rcD[8];
    __shared__ uint64_t s_bar[kRing];
    __shared__ int s_abort;
    const int col = blockIdx.y;
    if (active && !active[(int64_t)col * act_stride]) return;
    if (*(volatile int*)fault) return;  // an earlier sweep of this solve gave up: the host reports it, skip the work
    const int tid = threadIdx.x + 32 * threadIdx.y;
    PlaneRing<T, kRing> ring = ring_setup<T, kRing>(smem_raw, XH, s_bar, &s_abort, fault, tid);
    T* const Xbase = ring.slots + kRing * ring.slot;  // 4 x0 plane slots, PW x XH
    T* const Rbase = Xbase + 4 * PW * XH;             // 2 residual plane slots, PW x RH
    T* const Rxy = Rbase + 2 * PW * RH;               // 4 ring planes of the x-y restricted residual
    if (qtab) {  // this column's own kappa (serving lanes)
        if (tid < 7) {
            s_oi[tid] = qtab[(int64_t)col * 21 + tid];
            s_rcD[tid] = qtab[(int64_t)col * 21 + 14 + tid];
        }
    } else {
#pragma unroll
        for (int k = 0; k < 7; ++k)  // constant indices: the parameter struct stays in the constant bank
            if (tid == k) {
                s_oi[k] = q.oi[k];
                s_rcD[k] = q.rcD[k];
            }
    }
    const int nfx = gf.nx, nfy = gf.ny, nfz = gf.nz;  // all three halve (tiled levels)
    const int ncx = nfx >> 1, ncy = nfy >> 1, ncz = nfz >> 1;
    const int64_t fplane = (int64_t)nfx * nfy;
    const int ntx = nfx / SX, nty = nfy / SY, ntz = nfz / SZ;
    const int ntiles = ntx * nty * ntz;
    T* bcs = bc + (int64_t)col * bc_stride;
    const T sc = q.s * q.c;
    const int nplanes = SZ + 4;  // fine planes fz0 - 2 .. fz0 + SZ + 1 per tile
    __syncthreads();
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tX = tile % ntx, tY = (tile / ntx) % nty, tZ = tile / (ntx * nty);
        const int fx0 = tX * SX, fy0 = tY * SY, fz0 = tZ * SZ;
        const int cx0 = fx0 >> 1, cy0 = fy0 >> 1;
        int issued = 0;  // producer: planes of this tile requested so far
        auto issue_upto = [&](int jmax) {
            for (; issued < nplanes && issued <= jmax; ++issued)
                if (!ring.issue(issued & (kRing - 1), &bmap, fx0 - 4, fy0 - 2, fz0 - 2 + issued, col)) break;
        };
        if (tid == kProducer) issue_upto(kRing - 1);
        // --- per-tile slot data
        // x0 commit: one segment of the x0 plane (tid < kQ * XH); interior-plane factors cached
        const bool has_c = tid < kQ * XH;
        int c_off = 0, c_k = 0, c_g = -1;  // c_g: plane offset of the segment in the grid, -1 off the box
        T cI[4];
        {
            const int ly = tid / kQ, q4 = tid - ly * kQ;
            const int gy = fy0 - 2 + ly, gx0 = fx0 - 4 + 4 * q4;
            const bool in = has_c && in_range(gy, nfy) && in_range(gx0, nfx);
            c_off = 4 * q4 + PW * ly;
            if (in) c_g = gx0 + nfx * gy;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = in ? nb_count1(gy, nfy) + nb_count1(gx0 + e, nfx) : 0;
                c_k |= k << (3 * e);
                cI[e] = s_oi[k + 2];
            }
        }
        // residual: one segment of the residual plane (tid < kQ * RH)
        const bool has_r = tid < kQ * RH;
        int r_off = 0, r_k = 0, r_g = 0;
        bool r_in = false;
        T rI[4];
        {
            const int ly = tid / kQ, q4 = tid - ly * kQ;
            const int gy = fy0 - 1 + ly, gx0 = fx0 - 4 + 4 * q4;
            r_in = has_r && in_range(gy, nfy) && in_range(gx0, nfx);
            r_off = 4 * q4 + PW * ly;
            r_g = r_in ? gx0 + nfx * gy : 0;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = r_in ? nb_count1(gy, nfy) + nb_count1(gx0 + e, nfx) : 0;
                r_k |= k << (3 * e);
                rI[e] = s_rcD[k + 2];
            }
        }
        // restriction: coarse x pair (cx0 + 2 qm, + 1) of coarse row cy0 + qj
        const int qt = tid - kRestrictBase;
        const bool has_q = qt >= 0;
        const int qm = qt & 7, qj = (qt >> 3) & 7;
        T wa[4], wb[4], wy[4];
#pragma unroll
        for (int a3 = 0; a3 < 4; ++a3) {
            wa[a3] = (T)restrict_w(a3, cx0 + 2 * qm, ncx);
            wb[a3] = (T)restrict_w(a3, cx0 + 2 * qm + 1, ncx);
            wy[a3] = (T)restrict_w(a3, cy0 + qj, ncy);
        }
        const int q_off = 4 * qm + 3 + PW * (2 * qj);  // residual of fine (2I - 1, 2J - 1), I = cx0 + 2 qm
        T* const Rxq = Rxy + 2 * (qt & (RXY / 2 - 1));
        // x0 plane f = fz0 - 2 + j from tile plane j (ring slot JS = j mod 4; x0 slot (j + 2) mod 4)
        auto commit = [&](auto js, int f) {
            constexpr int JS = decltype(js)::value;
            const T* raw = ring.take(JS);
            if (has_c) {
                const bool wall = (f == 0 || f == nfz - 1);  // b = 0 off the box, any factor will do
                const V4<T> bv = ld4(raw + c_off);
                V4<T> v;
                if constexpr (PC) {  // per-cell diagonal (cell-wise kappa); b = 0 off the box
                    V4<T> dd;
#pragma unroll
                    for (int e = 0; e < 4; ++e) dd.v[e] = T(1);
                    if (c_g >= 0 && in_range(f, nfz)) dd = ld4(Dg + c_g + fplane * f);
#pragma unroll
                    for (int e = 0; e < 4; ++e) v.v[e] = q.omega * bv.v[e] / dd.v[e];
                } else if (!wall) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) v.v[e] = bv.v[e] * cI[e];
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) v.v[e] = bv.v[e] * s_oi[kxy_of(c_k, e) + 1];
                }
                st4(Xbase + ((JS + 2) & 3) * (PW * XH) + c_off, v);
            }
        };
        // step t: commit plane f + 2 (tile plane t + 3), residual of f, restriction of f - 1
        auto step = [&](auto kc, int t) {
            constexpr int K = decltype(kc)::value;  // t mod 4
            const int f = fz0 - 1 + t;
            if (t <= SZ) commit(IC<(K + 3) & 3>{}, f + 2);
            if (has_r && t <= SZ + 1) {
                V4<T> r = zero4<T>();
                if (r_in && in_range(f, nfz)) {
                    const bool wall = (f == 0 || f == nfz - 1);
                    const int xo = r_off + PW;  // x0 rows start one row above the residual rows
                    const T* Xc = Xbase + ((K + 3) & 3) * (PW * XH);
                    const T* Xm = Xbase + ((K + 2) & 3) * (PW * XH);
                    const T* Xp = Xbase + (K & 3) * (PW * XH);
                    const V4<T> c = ld4(Xc + xo), u = ld4(Xc + xo - PW), d = ld4(Xc + xo + PW);
                    const V4<T> m = ld4(Xm + xo), p = ld4(Xp + xo);
                    const T xl = Xc[xo - 1], xr = Xc[xo + 4];
                    T nbs[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const T left = (e == 0) ? xl : c.v[e - 1];
                        const T right = (e == 3) ? xr : c.v[e + 1];
                        nbs[e] = (left + right) + (u.v[e] + d.v[e]) + (m.v[e] + p.v[e]);
                    }
                    if constexpr (PC) {
                        const V4<T> dd = ld4(Dg + r_g + fplane * f);
                        const T rc = T(1) / q.omega - T(1);
#pragma unroll
                        for (int e = 0; e < 4; ++e) r.v[e] = rc * dd.v[e] * c.v[e] + sc * nbs[e];
                    } else if (!wall) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) r.v[e] = mad2(rI[e], c.v[e], sc, nbs[e]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e) r.v[e] = mad2(s_rcD[kxy_of(r_k, e) + 1], c.v[e], sc, nbs[e]);
                    }
                }
                st4(Rbase + ((K + 1) & 1) * (PW * RH) + r_off, r);
            }
            if (has_q && t >= 1) {
                const int fr = f - 1;  // plane restricted in this step
                T acc0 = T(0), acc1 = T(0);
                const T* Rp = Rbase + (K & 1) * (PW * RH);
#pragma unroll
                for (int b3 = 0; b3 < 4; ++b3) {
                    const T* row = Rp + q_off + PW * b3;
                    const T a0 = row[0], a5 = row[5];
                    const V4<T> v = ld4(row + 1);
                    const T p0 = mad4(wa, a0, v.v[0], v.v[1], v.v[2]);
                    const T p1 = mad4(wb, v.v[1], v.v[2], v.v[3], a5);
                    acc0 += wy[b3] * p0;
                    acc1 += wy[b3] * p1;
                }
                st2(Rxq + ((K + 2) & 3) * RXY, acc0, acc1);
                if ((K & 1) == 0 && t >= 4) {
                    // coarse plane Z = fr/2 - 1 from the x-y restricted planes 2Z-1 .. 2Z+2 = fr-3 .. fr
                    const int Z = (fr - 2) >> 1;
                    const T w3 = (T)restrict_w(3, Z, ncz);
                    T z0 = w3 * acc0, z1 = w3 * acc1;
#pragma unroll
                    for (int c3 = 0; c3 < 3; ++c3) {
                        const V2<T> v = ld2(Rxq + ((K + 3 + c3) & 3) * RXY);
                        const T w = (T)restrict_w(c3, Z, ncz);
                        z0 += w * v.v[0];
                        z1 += w * v.v[1];
                    }
                    st2(bcs + (cx0 + 2 * qm) + (int64_t)ncx * ((cy0 + qj) + (int64_t)ncy * Z), z0, z1);
                }
            }
            __syncthreads();
            // tile planes up to t + 3 are consumed: their slots are free
            if (tid == kProducer) issue_upto(t + 3 + kRing);
        };
        commit(IC<0>{}, fz0 - 2);
        commit(IC<1>{}, fz0 - 1);
        commit(IC<2>{}, fz0);
        __syncthreads();
        if (tid == kProducer) issue_upto(2 + kRing);  // tile planes 0 .. 2 are consumed
        const int nsteps = SZ + 3;  // f = fz0 - 1 .. fz0 + SZ + 1
        for (int t0 = 0; t0 < nsteps; t0 += 4) {
            step(IC<0>{}, t0);
            if (t0 + 1 < nsteps) step(IC<1>{}, t0 + 1);
            if (t0 + 2 < nsteps) step(IC<2>{}, t0 + 2);
            if (t0 + 3 < nsteps) step(IC<3>{}, t0 + 3);
        }
        if (tid == kProducer && s_abort) ring.drain();
    }
}

// ---------------------------------------------------------------------------
// Up sweep at level l: x = omega D^{-1} b + P ec ; y = x + omega D^{-1} (b - A x)
//     = (1 - omega) x + omega D^{-1} b + omega s c D^{-1} sum_{neighbours} x,
// optional partial sums of b.y (the MINRES beta^2 contribution).  Step t
// (g = fz0 + t): warps 0-5 form x(g+1) on the tile + halo 1 from b(g+1) and two
// coarse planes, warps 4-7 form y(g-1) from x planes g-2 .. g and b(g-1).  The
// prolongation of a 4-cell segment blends two coarse planes (z), two coarse
// rows (y) and then the four coarse x values the segment touches.  Coarse
// planes are stored with clamped x and y indices, which is the wall reflection
// of P; coarse plane Z lives in slot Z mod 4, x planes in 4 slots (fixed at
// compile time in the z-march unrolled by 4).
// ---------------------------------------------------------------------------
constexpr int kOutBase = kTileThreads - SX * SY / 4;  // the output threads: the last four warps

template <typename T, bool PC>  // PC: per-cell diagonal (cell-wise kappa) in Dg
__global__ void __launch_bounds__(kTileThreads, sizeof(T) == 4 ? 3 : 2)
    k_mg_up(const __grid_constant__ CUtensorMap bmap, Grid3 gf, int SZ, LevelCoef<T> q, const T* __restrict__ ec,
            int64_t ec_stride, T* __restrict__ y, int64_t y_stride, double* __restrict__ dot_part,
            const int* __restrict__ active, int act_stride, const T* __restrict__ Dg, int* __restrict__ fault,
            const T* __restrict__ qtab) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[kTileThreads / 32];
    __shared__ T s_oi[8], s_ois[8];
    __shared__ uint64_t s_bar[kRing];
    __shared__ int s_abort;
    const int col = blockIdx.y;
    if (active && !active[(int64_t)col * act_stride]) return;
    if (*(volatile int*)fault) return;
    const int tid = threadIdx.x + 32 * threadIdx.y;
    PlaneRing<T, kRing> ring = ring_setup<T, kRing>(smem_raw, BH, s_bar, &s_abort, fault, tid);
    T* const Xbase = ring.slots + kRing * ring.slot;  // 4 x plane slots, PW x BH
    T* const Cbase = Xbase + 4 * PW * BH;             // 4 coarse plane slots, CW x CH
    auto Cs = [&](int Z) { return Cbase + ((Z + 4) & 3) * (CW * CH); };  // Z >= -4
    if (qtab) {  // this column's own kappa (serving lanes)
        if (tid < 7) {
            s_oi[tid] = qtab[(int64_t)col * 21 + tid];
            s_ois[tid] = qtab[(int64_t)col * 21 + 7 + tid];
        }
    } else {
#pragma unroll
        for (int k = 0; k < 7; ++k)
            if (tid == k) {
                s_oi[k] = q.oi[k];
                s_ois[k] = q.ois[k];
            }
    }
    const int nfx = gf.nx, nfy = gf.ny, nfz = gf.nz;  // all three halve (tiled levels)
    const int ncx = nfx >> 1, ncy = nfy >> 1, ncz = nfz >> 1;
    const int ntx = nfx / SX, nty = nfy / SY, ntz = nfz / SZ;
    const int ntiles = ntx * nty * ntz;
    const int64_t plane = (int64_t)nfx * nfy, cplane = (int64_t)ncx * ncy;
    const T* es = ec + (int64_t)col * ec_stride;
    T* ys = y + (int64_t)col * y_stride;
    const T om1 = T(1) - q.omega;
    const int nplanes = SZ + 2;  // b planes fz0 - 1 .. fz0 + SZ per tile
    T dacc = T(0);  // per-thread partial of b.y in the element type; FP64 across warps
    __syncthreads();
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tX = tile % ntx, tY = (tile / ntx) % nty, tZ = tile / (ntx * nty);
        const int fx0 = tX * SX, fy0 = tY * SY, fz0 = tZ * SZ;
        const int cx0 = fx0 >> 1, cy0 = fy0 >> 1;
        const int cz0 = fz0 >> 1;
        int issued = 0;
        auto issue_upto = [&](int jmax) {
            for (; issued < nplanes && issued <= jmax; ++issued)
                if (!ring.issue(issued & (kRing - 1), &bmap, fx0 - 4, fy0 - 1, fz0 - 1 + issued, col)) break;
        };
        if (tid == kProducer) issue_upto(kRing - 1);
        // --- per-tile slot data
        int c_src = -1;  // coarse plane element of this thread (clamped x, y), or -1
        if (tid < CW * CH) {
            const int ly = tid / CW, lx = tid - ly * CW;
            const int gx = min(max(cx0 - 3 + lx, 0), ncx - 1), gy = min(max(cy0 - 1 + ly, 0), ncy - 1);
            c_src = gx + ncx * gy;
        }
        // prolongation: one segment of the x plane (tid < kQ * BH)
        const bool has_x = tid < kQ * BH;
        int x_off = 0, x_k = 0, p_r0 = 0, p_r1 = 0, x_g = 0;
        bool x_in = false;
        T xI[4];
        {
            const int ly = tid / kQ, q4 = tid - ly * kQ;
            const int gy = fy0 - 1 + ly, gx0 = fx0 - 4 + 4 * q4;
            x_in = has_x && in_range(gy, nfy) && in_range(gx0, nfx);
            x_off = 4 * q4 + PW * ly;
            x_g = x_in ? gx0 + nfx * gy : 0;
            if (x_in) {
                // coarse rows (gy >> 1) and its other neighbour; coarse x gx0/2 - 1 .. gx0/2 + 2
                p_r0 = ((gy >> 1) - (cy0 - 1)) * CW + 2 * q4;
                p_r1 = p_r0 + ((gy & 1) ? CW : -CW);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int k = x_in ? nb_count1(gy, nfy) + nb_count1(gx0 + e, nfx) : 0;
                x_k |= k << (3 * e);
                xI[e] = s_oi[k + 2];
            }
        }
        // output: one segment of the tile
        const int ot = tid - kOutBase;
        const bool has_out = ot >= 0;
        const int oy = (ot & (SX * SY / 4 - 1)) / (SX / 4), ox0 = 4 * (ot & (SX / 4 - 1));
        const int o_xi = (ox0 + 4) + PW * (oy + 1);
        int o_k = 0;
        T oI[4], sI[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = has_out ? nb_count1(fy0 + oy, nfy) + nb_count1(fx0 + ox0 + e, nfx) : 0;
            o_k |= k << (3 * e);
            oI[e] = s_oi[k + 2];
            sI[e] = s_ois[k + 2];
        }
        auto fetch_c = [&](int Z) -> T {
            return (c_src >= 0) ? es[c_src + cplane * min(max(Z, 0), ncz - 1)] : T(0);
        };
        // x(g) on the tile + halo 1 from b(g) = tile plane j = g - fz0 + 1 (ring slot JS = j mod 4,
        // x slot (j + 3) mod 4) and the coarse planes Iz = g >> 1 (weight 3/4) and its z neighbour
        // (Iz - 1 for even g, Iz + 1 for odd g)
        auto make_x = [&](auto js, int g) {
            constexpr int JS = decltype(js)::value;
            const T* Bg = ring.take(JS);
            if (!has_x) return;
            V4<T> v = zero4<T>();
            if (x_in && in_range(g, nfz)) {
                const bool wall = (g == 0 || g == nfz - 1);
                const int Iz = g >> 1;
                const T* C0 = Cs(Iz);
                const T* C1 = Cs((g & 1) ? Iz + 1 : Iz - 1);
                const V2<T> a0 = ld2(C0 + p_r0), a1 = ld2(C0 + p_r0 + 2);
                const V2<T> b0 = ld2(C0 + p_r1), b1 = ld2(C0 + p_r1 + 2);
                const V2<T> c0 = ld2(C1 + p_r0), c1 = ld2(C1 + p_r0 + 2);
                const V2<T> d0 = ld2(C1 + p_r1), d1 = ld2(C1 + p_r1 + 2);
                const T ar[4] = {a0.v[0], a0.v[1], a1.v[0], a1.v[1]};
                const T br[4] = {b0.v[0], b0.v[1], b1.v[0], b1.v[1]};
                const T cr[4] = {c0.v[0], c0.v[1], c1.v[0], c1.v[1]};
                const T dr[4] = {d0.v[0], d0.v[1], d1.v[0], d1.v[1]};
                T cy[4];
#pragma unroll
                for (int p = 0; p < 4; ++p)
                    cy[p] = blend4(ar[p], cr[p], br[p], dr[p]);
                const T pe[4] = {blend2(cy[1], cy[0]), blend2(cy[1], cy[2]), blend2(cy[2], cy[1]), blend2(cy[2], cy[3])};
                const V4<T> bb = ld4(Bg + x_off);
                if constexpr (PC) {  // per-cell diagonal (cell-wise kappa)
                    const V4<T> dd = ld4(Dg + x_g + plane * g);
#pragma unroll
                    for (int e = 0; e < 4; ++e) v.v[e] = q.omega * bb.v[e] / dd.v[e] + pe[e];
                } else if (!wall) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) v.v[e] = xI[e] * bb.v[e] + pe[e];
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) v.v[e] = s_oi[kxy_of(x_k, e) + 1] * bb.v[e] + pe[e];
                }
            }
            st4(Xbase + ((JS + 3) & 3) * (PW * BH) + x_off, v);
        };
        T pc = T(0);
        // step t (g = fz0 + t): x(g + 1) from tile plane t + 2, y(g - 1) from tile plane t
        auto step = [&](auto kc, int t) {
            constexpr int K = decltype(kc)::value;  // t mod 4
            const int g = fz0 + t;
            const int gn = g + 1;  // x plane formed in this step
            if (gn <= fz0 + SZ) {
                if ((K & 1) == 1) {  // gn even
                    // coarse plane gn/2 + 1 (slot of gn/2 - 3, no longer read) for x(gn + 1) onwards
                    if (c_src >= 0) Cs((gn >> 1) + 1)[tid] = pc;
                    if (gn + 2 <= fz0 + SZ) pc = fetch_c((gn >> 1) + 2);
                }
                make_x(IC<(K + 2) & 3>{}, gn);
            }
            const int f = g - 1;  // output plane: x planes f-1, f, f+1 and b(f) (tile plane t)
            if (t >= 1 && has_out) {
                const bool wall = (f == 0 || f == nfz - 1);
                const T* Xc = Xbase + ((K + 3) & 3) * (PW * BH);
                const T* Xm = Xbase + ((K + 2) & 3) * (PW * BH);
                const T* Xp = Xbase + (K & 3) * (PW * BH);
                const T* Bf = ring.at(K & 3);
                const V4<T> c = ld4(Xc + o_xi), u = ld4(Xc + o_xi - PW), d = ld4(Xc + o_xi + PW);
                const V4<T> m = ld4(Xm + o_xi), p = ld4(Xp + o_xi), bb = ld4(Bf + o_xi);
                const T xl = Xc[o_xi - 1], xr = Xc[o_xi + 4];
                T nbs[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const T left = (e == 0) ? xl : c.v[e - 1];
                    const T right = (e == 3) ? xr : c.v[e + 1];
                    nbs[e] = (left + right) + (u.v[e] + d.v[e]) + (m.v[e] + p.v[e]);
                }
                V4<T> out;
                if constexpr (PC) {  // y = (1 - omega) x + omega D^{-1} (b + s c sum x)
                    const V4<T> dd = ld4(Dg + (fx0 + ox0) + (int64_t)nfx * (fy0 + oy) + plane * f);
                    const T sc = q.s * q.c;
#pragma unroll
                    for (int e = 0; e < 4; ++e) out.v[e] = om1 * c.v[e] + q.omega * (bb.v[e] + sc * nbs[e]) / dd.v[e];
                } else if (!wall) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) out.v[e] = fma(sI[e], nbs[e], fma(oI[e], bb.v[e], om1 * c.v[e]));
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int kw = kxy_of(o_k, e) + 1;
                        out.v[e] = fma(s_ois[kw], nbs[e], fma(s_oi[kw], bb.v[e], om1 * c.v[e]));
                    }
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) dacc += bb.v[e] * out.v[e];
                st4(ys + (fx0 + ox0) + (int64_t)nfx * (fy0 + oy) + plane * f, out);
            }
            __syncthreads();
            // tile planes up to t are consumed: their slots are free
            if (tid == kProducer) issue_upto(t + kRing);
        };
        // prologue: coarse planes cz0-1 .. cz0+1, then x(fz0 - 1) and x(fz0)
        if (c_src >= 0) {
            Cs(cz0 - 1)[tid] = fetch_c(cz0 - 1);
            Cs(cz0)[tid] = fetch_c(cz0);
            Cs(cz0 + 1)[tid] = fetch_c(cz0 + 1);
        }
        pc = fetch_c(cz0 + 2);  // stored while x(fz0 + 2) is formed, first used by x(fz0 + 3)
        __syncthreads();
        make_x(IC<0>{}, fz0 - 1);
        make_x(IC<1>{}, fz0);
        __syncthreads();
        if (tid == kProducer) issue_upto(kRing);  // tile plane 0 (b(fz0 - 1)) is consumed
        const int nsteps = SZ + 1;  // g = fz0 .. fz0 + SZ
        for (int t0 = 0; t0 < nsteps; t0 += 4) {
            step(IC<0>{}, t0);
            if (t0 + 1 < nsteps) step(IC<1>{}, t0 + 1);
            if (t0 + 2 < nsteps) step(IC<2>{}, t0 + 2);
            if (t0 + 3 < nsteps) step(IC<3>{}, t0 + 3);
        }
        if (tid == kProducer && s_abort) ring.drain();
    }
    if (dot_part) {
        const double tsum = block_sum_t<kTileThreads, T>(dacc, red);
        if (tid == 0) dot_part[(int64_t)col * kMaxPartials + blockIdx.x] = tsum;
    }
}


// ---------------------------------------------------------------------------
// Row-tile sweeps (FP32, grids whose x extent is 32, 64 or 128 cells).  A CTA
// owns whole x rows: a tile is nx x TY cells in (x, y), marched along z.  A
// thread owns one 4-cell x segment of one row for the whole march, so
//   - the x neighbours of a segment come from the adjacent lanes by shuffles
//     (a row is Q = nx / 4 consecutive lanes; the row ends are the walls),
//   - its z neighbours (planes f - 1, f, f + 1) stay in a register ring,
//   - only the y neighbours (other rows, other warps) go through shared memory,
// and there is no halo in x.  The down sweep restricts in x inside the warp,
// in y through one shared-memory pass and in z in registers.
// ---------------------------------------------------------------------------
template <int NX, int TY_>
struct RowShape {
    static constexpr int TY = TY_;       // rows per tile
    static constexpr int Q = NX / 4;     // segments (lanes) per row
    static constexpr int RPW = 32 / Q;   // rows per warp
    static constexpr int R = TY + 4;     // rows of a plane slot: y from fy0 - 2
    static constexpr int NW = R / RPW;   // warps
    static constexpr int NT = 32 * NW;   // threads
    static constexpr int PLANE = NX * R; // floats per plane slot
    static constexpr int RXR = TY + 2;   // residual rows (y from fy0 - 1)
    static constexpr int CXN = NX / 2;   // coarse x per row
    static constexpr int NITEMS = (TY / 2) * (NX / 4);  // y-restriction items: coarse row x coarse x pair
};

template <int NX, int TY>
__host__ __device__ constexpr int down_rows_smem_bytes() {
    using Sh = RowShape<NX, TY>;
    return 128 + (int)sizeof(float) * ((kRing + 4) * Sh::PLANE + 2 * Sh::RXR * Sh::CXN);
}

// TMA ring of plane slots of `elems` floats each (copies of `bytes`), producer = thread 0
template <int NS>
__device__ __forceinline__ PlaneRing<float, NS> ring_setup_rows(unsigned char* raw, int elems, uint32_t bytes,
                                                                uint64_t* bars, volatile int* abort, int* fault,
                                                                int tid) {
    PlaneRing<float, NS> r;
    r.fault = fault;
    const uint32_t a = smem_addr(raw);
    r.slots = reinterpret_cast<float*>(raw + ((128 - (a & 127)) & 127));
    r.slot = elems;
    r.bars = bars;
    r.abort = abort;
    r.bytes = bytes;
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) mbar_init(bars + i);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    return r;
}

template <int NX, int TY>
__global__ void __launch_bounds__(RowShape<NX, TY>::NT, RowShape<NX, TY>::NT <= 384 ? 2 : 1)
    k_mg_down_rows(const __grid_constant__ CUtensorMap bmap, Grid3 gf, int SZ, LevelCoef<float> q,
                   float* __restrict__ bc, int64_t bc_stride, const int* __restrict__ active, int act_stride,
                   int* __restrict__ fault, const float* __restrict__ qtab) {
    using Sh = RowShape<NX, TY>;
    constexpr int Q = Sh::Q, RPW = Sh::RPW, R = Sh::R, PLANE = Sh::PLANE, CXN = Sh::CXN;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ float s_oi[8], s_rcD[8];
    __shared__ uint64_t s_bar[kRing];
    __shared__ int s_abort;
    const int col = blockIdx.y;
    if (active && !active[(int64_t)col * act_stride]) return;
    if (*(volatile int*)fault) return;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int qq = lane % Q;                  // segment: fine x 4 qq .. 4 qq + 3
    const int ly = warp * RPW + lane / Q;     // slot row: fine y = fy0 - 2 + ly
    PlaneRing<float, kRing> ring =
        ring_setup_rows<kRing>(smem_raw, PLANE, (uint32_t)(PLANE * sizeof(float)), s_bar, &s_abort, fault, tid);
    float* const Xs = ring.slots + kRing * PLANE;  // 4 x0 plane slots
    float* const RX = Xs + 4 * PLANE;              // 2 buffers of x-restricted residual rows
    if (qtab) {
        if (tid < 7) {
            s_oi[tid] = qtab[(int64_t)col * 21 + tid];
            s_rcD[tid] = qtab[(int64_t)col * 21 + 14 + tid];
        }
    } else {
#pragma unroll
        for (int k = 0; k < 7; ++k)
            if (tid == k) {
                s_oi[k] = q.oi[k];
                s_rcD[k] = q.rcD[k];
            }
    }
    const int nfy = gf.ny, nfz = gf.nz;
    const int ncx = NX >> 1, ncy = nfy >> 1, ncz = nfz >> 1;
    const int nty = nfy / TY, ntz = nfz / SZ;
    const int ntiles = nty * ntz;
    float* bcs = bc + (int64_t)col * bc_stride;
    const float sc = q.s * q.c;
    const int nplanes = SZ + 4;  // fine planes fz0 - 2 .. fz0 + SZ + 1 per tile
    // x-restriction weights of this segment's two coarse x (taps fine 2I - 1 .. 2I + 2)
    float wa[4], wb[4];
#pragma unroll
    for (int a3 = 0; a3 < 4; ++a3) {
        wa[a3] = restrict_w(a3, 2 * qq, ncx);
        wb[a3] = restrict_w(a3, 2 * qq + 1, ncx);
    }
    // y-restriction item of this thread: coarse row J, coarse x pair P (whole warps: spreading
    // the items over every warp measured slower, as every warp then runs the item code)
    const bool has_item = tid < Sh::NITEMS;
    const int iJ = tid / (NX / 4), iP = tid % (NX / 4);
    __syncthreads();
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tY = tile % nty, tZ = tile / nty;
        const int fy0 = tY * TY, fz0 = tZ * SZ;
        const int cy0 = fy0 >> 1;
        int issued = 0;  // producer: planes of this tile requested so far
        auto issue_upto = [&](int jmax) {
            for (; issued < nplanes && issued <= jmax; ++issued)
                if (!ring.issue(issued & (kRing - 1), &bmap, 0, fy0 - 2, fz0 - 2 + issued, col)) break;
        };
        if (tid == 0) issue_upto(kRing - 1);
        const int gy = fy0 - 2 + ly;
        const bool yin = in_range(gy, nfy);
        const bool has_r = ly >= 1 && ly <= R - 2;  // residual rows: y from fy0 - 1 to fy0 + TY
        int kxy = 0;  // x-y neighbour counts of the segment's cells, 3 bits each
        float cI[4], rI[4];  // x0 and residual factors of the segment's cells on interior planes
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = yin ? nb_count1(gy, nfy) + nb_count1(4 * qq + e, NX) : 0;
            kxy |= k << (3 * e);
            cI[e] = s_oi[k + 2];
            rI[e] = s_rcD[k + 2];
        }
        float wy[4];
#pragma unroll
        for (int a3 = 0; a3 < 4; ++a3) wy[a3] = restrict_w(a3, cy0 + iJ, ncy);
        V4<float> X0[4];  // x0 of this segment, tile plane j in X0[j & 3]
        V2<float> Rv[4];  // this item's x-y restricted residual, fine plane fr in Rv[fr mod 4]
        // x0 plane f = fz0 - 2 + j from tile plane j (TMA slot j mod 4): registers and x0 slot j mod 4
        auto commit = [&](auto js, int f) {
            constexpr int JS = decltype(js)::value;
            const float* raw = ring.take(JS);
            const V4<float> bv = ld4(raw + ly * NX + 4 * qq);
            V4<float> v;
            if (f != 0 && f != nfz - 1) {
#pragma unroll
                for (int e = 0; e < 4; ++e) v.v[e] = bv.v[e] * cI[e];
            } else {  // the z walls (b = 0 off the box, any factor will do)
#pragma unroll
                for (int e = 0; e < 4; ++e) v.v[e] = bv.v[e] * s_oi[kxy_of(kxy, e) + 1];
            }
            X0[JS] = v;
            st4(Xs + JS * PLANE + ly * NX + 4 * qq, v);
        };
        // step t: commit f + 2 (tile plane t + 3), residual and x-restriction of f (plane t + 1),
        // y- and z-restriction of f - 1 (from the previous step's rows)
        auto step = [&](auto kc, int t) {
            constexpr int K = decltype(kc)::value;  // t mod 4
            const int f = fz0 - 1 + t;
            if (t <= SZ) commit(IC<(K + 3) & 3>{}, f + 2);
            if (t <= SZ + 1) {
                const V4<float> c = X0[(K + 1) & 3], m = X0[K & 3], p = X0[(K + 2) & 3];
                const float xl0 = __shfl_up_sync(0xffffffffu, c.v[3], 1, Q);
                const float xr0 = __shfl_down_sync(0xffffffffu, c.v[0], 1, Q);
                const float xl = qq > 0 ? xl0 : 0.0f, xr = qq < Q - 1 ? xr0 : 0.0f;
                V4<float> r = zero4<float>();
                if (has_r && yin && in_range(f, nfz)) {
                    const float* Xf = Xs + ((K + 1) & 3) * PLANE + 4 * qq;
                    const V4<float> u = ld4(Xf + (ly - 1) * NX), d = ld4(Xf + (ly + 1) * NX);
                    float nbs[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float left = (e == 0) ? xl : c.v[e - 1];
                        const float right = (e == 3) ? xr : c.v[e + 1];
                        nbs[e] = (left + right) + (u.v[e] + d.v[e]) + (m.v[e] + p.v[e]);
                    }
                    if (f != 0 && f != nfz - 1) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) r.v[e] = mad2(rI[e], c.v[e], sc, nbs[e]);
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e) r.v[e] = mad2(s_rcD[kxy_of(kxy, e) + 1], c.v[e], sc, nbs[e]);
                    }
                }
                const float rl0 = __shfl_up_sync(0xffffffffu, r.v[3], 1, Q);
                const float rr0 = __shfl_down_sync(0xffffffffu, r.v[0], 1, Q);
                const float rl = qq > 0 ? rl0 : 0.0f, rr = qq < Q - 1 ? rr0 : 0.0f;
                if (has_r) {
                    const float x0v = mad4(wa, rl, r.v[0], r.v[1], r.v[2]);
                    const float x1v = mad4(wb, r.v[1], r.v[2], r.v[3], rr);
                    st2(RX + (K & 1) * (Sh::RXR * CXN) + (ly - 1) * CXN + 2 * qq, x0v, x1v);
                }
            }
            if (t >= 1 && has_item) {
                // fine plane fr = f - 1: rows 2J - 1 .. 2J + 2 of the previous step's buffer;
                // the x-y restricted value of plane fr goes to register slot fr mod 4
                const float* Rb = RX + ((K + 1) & 1) * (Sh::RXR * CXN) + 2 * iP;
                float v0 = 0.f, v1 = 0.f;
#pragma unroll
                for (int a3 = 0; a3 < 4; ++a3) {
                    const V2<float> rv = ld2(Rb + (2 * iJ + a3) * CXN);
                    v0 += wy[a3] * rv.v[0];
                    v1 += wy[a3] * rv.v[1];
                }
                Rv[(K + 2) & 3].v[0] = v0;
                Rv[(K + 2) & 3].v[1] = v1;
                if ((K & 1) == 0 && t >= 4) {
                    // coarse plane Z = fr/2 - 1 from the x-y restricted planes 2Z-1 .. 2Z+2 = fr-3 .. fr
                    const int Z = (f - 3) >> 1;
                    const float w3 = restrict_w(3, Z, ncz);
                    float z0 = w3 * v0, z1 = w3 * v1;
#pragma unroll
                    for (int c3 = 0; c3 < 3; ++c3) {
                        const float w = restrict_w(c3, Z, ncz);
                        z0 += w * Rv[(K + 3 + c3) & 3].v[0];
                        z1 += w * Rv[(K + 3 + c3) & 3].v[1];
                    }
                    st2(bcs + 2 * iP + (int64_t)ncx * ((cy0 + iJ) + (int64_t)ncy * Z), z0, z1);
                }
            }
            __syncthreads();
            // tile planes up to t + 3 are consumed: their slots are free
            if (tid == 0) issue_upto(t + 3 + kRing);
        };
        commit(IC<0>{}, fz0 - 2);
        commit(IC<1>{}, fz0 - 1);
        commit(IC<2>{}, fz0);
        __syncthreads();
        if (tid == 0) issue_upto(2 + kRing);  // tile planes 0 .. 2 are consumed
        const int nsteps = SZ + 3;  // f = fz0 - 1 .. fz0 + SZ + 1
        for (int t0 = 0; t0 < nsteps; t0 += 4) {
            step(IC<0>{}, t0);
            if (t0 + 1 < nsteps) step(IC<1>{}, t0 + 1);
            if (t0 + 2 < nsteps) step(IC<2>{}, t0 + 2);
            if (t0 + 3 < nsteps) step(IC<3>{}, t0 + 3);
        }
        if (tid == 0 && s_abort) ring.drain();
    }
}


// Up sweep on row tiles: the same x and y as k_mg_up, cell by cell.  Thread
// rows as in the down sweep (fine y from fy0 - 2); rows fy0 - 1 .. fy0 + TY
// form x, rows fy0 .. fy0 + TY - 1 form y.  The prolongation of a segment
// needs the coarse x 2 qq - 1 .. 2 qq + 2: the thread blends its own pair
// (2 qq, 2 qq + 1) in y and z and takes the outer two from its row neighbours
// by shuffles (clamped at the x walls, the reflection of P).  Each thread
// stages one element of every coarse plane (coarse rows cy0 - 1 .. cy0 + TY/2,
// clamped, all coarse x): there are exactly as many as threads.
template <int NX, int TY>
__host__ __device__ constexpr int up_rows_smem_bytes() {
    using Sh = RowShape<NX, TY>;
    return 128 + (int)sizeof(float) * (2 * kRing * Sh::PLANE + 4 * Sh::NT);
}

template <int NX, int TY>
__global__ void __launch_bounds__(RowShape<NX, TY>::NT, RowShape<NX, TY>::NT <= 384 ? 2 : 1)
    k_mg_up_rows(const __grid_constant__ CUtensorMap bmap, Grid3 gf, int SZ, LevelCoef<float> q,
                 const float* __restrict__ ec, int64_t ec_stride, float* __restrict__ y, int64_t y_stride,
                 double* __restrict__ dot_part, const int* __restrict__ active, int act_stride,
                 int* __restrict__ fault, const float* __restrict__ qtab) {
    using Sh = RowShape<NX, TY>;
    constexpr int Q = Sh::Q, RPW = Sh::RPW, R = Sh::R, PLANE = Sh::PLANE, CXN = Sh::CXN, NT = Sh::NT;
    static_assert((TY / 2 + 2) * CXN == NT, "one coarse element per thread");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[NT / 32];
    __shared__ float s_oi[8], s_ois[8];
    __shared__ uint64_t s_bar[kRing];
    __shared__ int s_abort;
    const int col = blockIdx.y;
    if (active && !active[(int64_t)col * act_stride]) return;
    if (*(volatile int*)fault) return;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int qq = lane % Q;
    const int ly = warp * RPW + lane / Q;  // fine y = fy0 - 2 + ly
    PlaneRing<float, kRing> ring =
        ring_setup_rows<kRing>(smem_raw, PLANE, (uint32_t)(PLANE * sizeof(float)), s_bar, &s_abort, fault, tid);
    float* const Xs = ring.slots + kRing * PLANE;  // 4 x plane slots
    float* const Cbase = Xs + 4 * PLANE;           // 4 coarse plane slots, NT elements each
    auto Cs = [&](int Z) { return Cbase + ((Z + 4) & 3) * NT; };  // Z >= -4
    if (qtab) {
        if (tid < 7) {
            s_oi[tid] = qtab[(int64_t)col * 21 + tid];
            s_ois[tid] = qtab[(int64_t)col * 21 + 7 + tid];
        }
    } else {
#pragma unroll
        for (int k = 0; k < 7; ++k)
            if (tid == k) {
                s_oi[k] = q.oi[k];
                s_ois[k] = q.ois[k];
            }
    }
    const int nfy = gf.ny, nfz = gf.nz;
    const int ncx = NX >> 1, ncy = nfy >> 1, ncz = nfz >> 1;
    const int nty = nfy / TY, ntz = nfz / SZ;
    const int ntiles = nty * ntz;
    const int64_t plane = (int64_t)NX * nfy, cplane = (int64_t)ncx * ncy;
    const float* es = ec + (int64_t)col * ec_stride;
    float* ys = y + (int64_t)col * y_stride;
    const float om1 = 1.0f - q.omega;
    const int nplanes = SZ + 2;  // b planes fz0 - 1 .. fz0 + SZ per tile
    float dacc = 0.0f;
    __syncthreads();
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int tY = tile % nty, tZ = tile / nty;
        const int fy0 = tY * TY, fz0 = tZ * SZ;
        const int cy0 = fy0 >> 1, cz0 = fz0 >> 1;
        int issued = 0;
        auto issue_upto = [&](int jmax) {
            for (; issued < nplanes && issued <= jmax; ++issued)
                if (!ring.issue(issued & (kRing - 1), &bmap, 0, fy0 - 2, fz0 - 1 + issued, col)) break;
        };
        if (tid == 0) issue_upto(kRing - 1);
        // this thread's coarse element: coarse row cy0 - 1 + tid / CXN (clamped), coarse x tid % CXN
        const int c_src = (tid % CXN) + ncx * min(max(cy0 - 1 + tid / CXN, 0), ncy - 1);
        auto fetch_c = [&](int Z) -> float { return es[c_src + cplane * min(max(Z, 0), ncz - 1)]; };
        const int gy = fy0 - 2 + ly;
        const bool yin = in_range(gy, nfy);
        const bool x_row = yin && ly >= 1 && ly <= R - 2;   // forms x
        const bool o_row = ly >= 2 && ly <= R - 3;          // forms y (always inside the grid)
        // coarse rows of the prolongation: gy >> 1 and its other neighbour, in slot rows from cy0 - 1
        const int p_r0 = x_row ? ((gy >> 1) - (cy0 - 1)) * CXN + 2 * qq : 0;
        const int p_r1 = x_row ? p_r0 + ((gy & 1) ? CXN : -CXN) : 0;
        int kxy = 0;
        float xI[4], sI[4];  // interior-plane factors (x and y both take omega D^-1 = oi)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = yin ? nb_count1(gy, nfy) + nb_count1(4 * qq + e, NX) : 0;
            kxy |= k << (3 * e);
            xI[e] = s_oi[k + 2];
            sI[e] = s_ois[k + 2];
        }
        V4<float> X[4];  // x of this segment, tile plane j (x(fz0 - 1 + j)) in X[j & 3]
        // x(g) from b(g) = tile plane j = g - fz0 + 1 and the coarse planes g >> 1 (weight 3/4) and
        // its z neighbour (Iz - 1 for even g, Iz + 1 for odd g)
        auto make_x = [&](auto js, int g) {
            constexpr int JS = decltype(js)::value;
            const float* Bg = ring.take(JS);
            const bool act = x_row && in_range(g, nfz);
            float cyA = 0.0f, cyB = 0.0f;  // y-z blend of coarse x 2 qq and 2 qq + 1
            if (act) {
                const int Iz = g >> 1;
                const float* C0 = Cs(Iz);
                const float* C1 = Cs((g & 1) ? Iz + 1 : Iz - 1);
                const V2<float> a = ld2(C0 + p_r0), b = ld2(C0 + p_r1);
                const V2<float> c = ld2(C1 + p_r0), d = ld2(C1 + p_r1);
                cyA = blend4(a.v[0], c.v[0], b.v[0], d.v[0]);
                cyB = blend4(a.v[1], c.v[1], b.v[1], d.v[1]);
            }
            const float l0 = __shfl_up_sync(0xffffffffu, cyB, 1, Q);
            const float r0 = __shfl_down_sync(0xffffffffu, cyA, 1, Q);
            const float cyL = qq > 0 ? l0 : cyA, cyR = qq < Q - 1 ? r0 : cyB;
            V4<float> v = zero4<float>();
            if (act) {
                const float pe[4] = {blend2(cyA, cyL), blend2(cyA, cyB), blend2(cyB, cyA), blend2(cyB, cyR)};
                const V4<float> bb = ld4(Bg + ly * NX + 4 * qq);
                if (g != 0 && g != nfz - 1) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) v.v[e] = xI[e] * bb.v[e] + pe[e];
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) v.v[e] = s_oi[kxy_of(kxy, e) + 1] * bb.v[e] + pe[e];
                }
            }
            X[JS] = v;
            st4(Xs + JS * PLANE + ly * NX + 4 * qq, v);
        };
        float pc = 0.0f;
        // step t (g = fz0 + t): x(g + 1) from tile plane t + 2, y(g - 1) from tile plane t
        auto step = [&](auto kc, int t) {
            constexpr int K = decltype(kc)::value;  // t mod 4
            const int g = fz0 + t;
            const int gn = g + 1;
            if (gn <= fz0 + SZ) {
                if ((K & 1) == 1) {  // gn even: coarse plane gn/2 + 1 (slot of gn/2 - 3, no longer read)
                    Cs((gn >> 1) + 1)[tid] = pc;
                    if (gn + 2 <= fz0 + SZ) pc = fetch_c((gn >> 1) + 2);
                }
                make_x(IC<(K + 2) & 3>{}, gn);
            }
            if (t >= 1) {
                const int f = g - 1;  // x planes f - 1, f, f + 1 and b(f) (tile plane t)
                const V4<float> c = X[K & 3], m = X[(K + 3) & 3], p = X[(K + 1) & 3];
                const float xl0 = __shfl_up_sync(0xffffffffu, c.v[3], 1, Q);
                const float xr0 = __shfl_down_sync(0xffffffffu, c.v[0], 1, Q);
                const float xl = qq > 0 ? xl0 : 0.0f, xr = qq < Q - 1 ? xr0 : 0.0f;
                if (o_row) {
                    const float* Xf = Xs + (K & 3) * PLANE + 4 * qq;
                    const V4<float> u = ld4(Xf + (ly - 1) * NX), d = ld4(Xf + (ly + 1) * NX);
                    const V4<float> bb = ld4(ring.at(K & 3) + ly * NX + 4 * qq);
                    float nbs[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float left = (e == 0) ? xl : c.v[e - 1];
                        const float right = (e == 3) ? xr : c.v[e + 1];
                        nbs[e] = (left + right) + (u.v[e] + d.v[e]) + (m.v[e] + p.v[e]);
                    }
                    V4<float> out;
                    if (f != 0 && f != nfz - 1) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) out.v[e] = fma(sI[e], nbs[e], fma(xI[e], bb.v[e], om1 * c.v[e]));
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int kw = kxy_of(kxy, e) + 1;
                            out.v[e] = fma(s_ois[kw], nbs[e], fma(s_oi[kw], bb.v[e], om1 * c.v[e]));
                        }
                    }
#pragma unroll
                    for (int e = 0; e < 4; ++e) dacc += bb.v[e] * out.v[e];
                    st4(ys + 4 * qq + (int64_t)NX * gy + plane * f, out);
                }
            }
            __syncthreads();
            // tile planes up to t are consumed: their slots are free
            if (tid == 0) issue_upto(t + kRing);
        };
        // prologue: coarse planes cz0 - 1 .. cz0 + 1, then x(fz0 - 1) and x(fz0)
        Cs(cz0 - 1)[tid] = fetch_c(cz0 - 1);
        Cs(cz0)[tid] = fetch_c(cz0);
        Cs(cz0 + 1)[tid] = fetch_c(cz0 + 1);
        pc = fetch_c(cz0 + 2);  // stored while x(fz0 + 2) is formed, first used by x(fz0 + 3)
        __syncthreads();
        make_x(IC<0>{}, fz0 - 1);
        make_x(IC<1>{}, fz0);
        __syncthreads();
        if (tid == 0) issue_upto(kRing);  // tile plane 0 (b(fz0 - 1)) is consumed
        const int nsteps = SZ + 1;  // g = fz0 .. fz0 + SZ
        for (int t0 = 0; t0 < nsteps; t0 += 4) {
            step(IC<0>{}, t0);
            if (t0 + 1 < nsteps) step(IC<1>{}, t0 + 1);
            if (t0 + 2 < nsteps) step(IC<2>{}, t0 + 2);
            if (t0 + 3 < nsteps) step(IC<3>{}, t0 + 3);
        }
        if (tid == 0 && s_abort) ring.drain();
    }
    if (dot_part) {
        const double tsum = block_sum_t<NT, float>(dacc, red);
        if (tid == 0) dot_part[(int64_t)col * kMaxPartials + blockIdx.x] = tsum;
    }
}

// ---------------------------------------------------------------------------
// The levels from lc down (at most 4096 cells on level lc) in one CTA per
// sample (shared memory).  Extents may differ per axis; an axis that has
// reached extent 1 is no longer coarsened (its transfers are the identity).
// ---------------------------------------------------------------------------
struct CoarseDesc {
    int lc;        // first (absolute) level handled here
    int nlev;      // total number of levels (the last one has one cell)
    Grid3 g[16];   // grids of the levels (absolute index)
    double kh2, c, omega;
    double ls[16], lq[16];  // level factors s_l, q_l
    const void* D[16];  // per-cell diagonals of the levels (cell-wise kappa), or null
    const double* kh2col;  // (kappa h)^2 of level 0 per column (serving lanes), or null: kh2
};

// storage of the one-CTA levels: the compute type, or FP16 (values scaled into range)
template <typename T, typename SM>
__device__ __forceinline__ T cz_ld(const SM* p, int i) {
    if constexpr (std::is_same<SM, __half>::value) return (T)__half2float(p[i]);
    else return p[i];
}
template <typename T, typename SM>
__device__ __forceinline__ void cz_st(SM* p, int i, T v) {
    if constexpr (std::is_same<SM, __half>::value) p[i] = __float2half_rn((float)v);
    else p[i] = v;
}

template <typename T>
__device__ __forceinline__ T cz_invD(const CoarseDesc& d, int l, int k, double kh2) {
    const T s = (T)d.ls[l];
    const T a = (T)(kh2 * d.lq[l]);
    return T(1) / (s * (a + (T)d.c * (T)k));
}

// 1 / diagonal of cell f (neighbour count kc) on level l
template <typename T>
__device__ __forceinline__ T cz_invDf(const CoarseDesc& d, int l, int kc, int f, double kh2) {
    if (d.D[l]) return T(1) / static_cast<const T*>(d.D[l])[f];
    return cz_invD<T>(d, l, kc, kh2);
}

template <typename T, typename SM>
__device__ __forceinline__ T cz_Ax(const CoarseDesc& d, int l, const SM* x, const Grid3& g, int i, int j, int k,
                                   double kh2) {
    const int sy = g.nx, sz = g.nx * g.ny;
    const int f = i + g.nx * (j + g.ny * k);
    const T x0 = cz_ld<T>(x, f);
    if (d.D[l]) {  // per-cell diagonal: D x0 - s c (sum of existing neighbours)
        T nb = T(0);
        if (i > 0) nb += cz_ld<T>(x, f - 1);
        if (i < g.nx - 1) nb += cz_ld<T>(x, f + 1);
        if (j > 0) nb += cz_ld<T>(x, f - sy);
        if (j < g.ny - 1) nb += cz_ld<T>(x, f + sy);
        if (k > 0) nb += cz_ld<T>(x, f - sz);
        if (k < g.nz - 1) nb += cz_ld<T>(x, f + sz);
        return static_cast<const T*>(d.D[l])[f] * x0 - (T)d.ls[l] * (T)d.c * nb;
    }
    T lap = T(0);
    if (i > 0) lap += x0 - cz_ld<T>(x, f - 1);
    if (i < g.nx - 1) lap += x0 - cz_ld<T>(x, f + 1);
    if (j > 0) lap += x0 - cz_ld<T>(x, f - sy);
    if (j < g.ny - 1) lap += x0 - cz_ld<T>(x, f + sy);
    if (k > 0) lap += x0 - cz_ld<T>(x, f - sz);
    if (k < g.nz - 1) lap += x0 - cz_ld<T>(x, f + sz);
    const T s = (T)d.ls[l];
    const T a = (T)(kh2 * d.lq[l]);
    return s * (a * x0 + (T)d.c * lap);
}

// the taps of the 1-D restriction onto coarse index I along one axis: fine
// indices f0 .. f0 + nt - 1 with weights w (zero outside the grid)
__device__ __forceinline__ int restrict_taps(bool coarsened, int I, int nc, int& f0, float w[4]) {
    if (!coarsened) {
        f0 = I;
        w[0] = 1.0f;
        return 1;
    }
    f0 = 2 * I - 1;
#pragma unroll
    for (int a = 0; a < 4; ++a) w[a] = restrict_w(a, I, nc);
    return 4;
}

// the two taps of the 1-D prolongation onto fine index i along one axis
__device__ __forceinline__ void prolong_taps(bool coarsened, int i, int nc, int p[2], float w[2]) {
    if (!coarsened) {
        p[0] = p[1] = i;
        w[0] = 1.0f;
        w[1] = 0.0f;
        return;
    }
    const int I = i >> 1;
    p[0] = I;
    p[1] = min(max((i & 1) ? I + 1 : I - 1, 0), nc - 1);
    w[0] = 0.75f;
    w[1] = 0.25f;
}

template <typename T, typename SM>
__global__ void __launch_bounds__(kCoarseThreads) k_mg_coarse(CoarseDesc d, const T* __restrict__ bin, int64_t b_stride,
                                                              T* __restrict__ eout, int64_t e_stride,
                                                              double* __restrict__ dot_part,
                                                              const int* __restrict__ active, int act_stride) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double red[kCoarseThreads / 32];
    SM* sm = reinterpret_cast<SM*>(smem_raw);
    __shared__ T s_scale;
    const int col = blockIdx.x;
    if (active && !active[(int64_t)col * act_stride]) return;
    const double kh2 = d.kh2col ? d.kh2col[col] : d.kh2;
    // layout: b_l and x_l for l = lc .. nlev-1, then a temp of level lc's size
    int offb[16], offx[16];
    int o = 0;
    for (int l = d.lc; l < d.nlev; ++l) {
        const int nl = (int)d.g[l].cells();
        offb[l] = o;
        o += nl;
        offx[l] = o;
        o += nl;
    }
    SM* tmp = sm + o;
    const T* bs = bin + (int64_t)col * b_stride;
    T* es = eout + (int64_t)col * e_stride;
    // FP16 storage: the column is scaled by 1 / max |b| (the V-cycle is linear), so every
    // stored value lies within FP16 range; the result is scaled back on the way out
    T scale = T(1);
    if constexpr (std::is_same<SM, __half>::value) {
        const int n3 = (int)d.g[d.lc].cells();
        float mx = 0.0f;
        for (int f = threadIdx.x; f < n3; f += blockDim.x) mx = fmaxf(mx, fabsf((float)bs[f]));
        for (int of = 16; of > 0; of >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, of));
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m = 0.0f;
            for (int w = 0; w < kCoarseThreads / 32; ++w) m = fmaxf(m, (float)red[w]);
            s_scale = m > 0.0f ? (T)m : T(1);
        }
        __syncthreads();
        scale = s_scale;
    }
    {
        const int n3 = (int)d.g[d.lc].cells();
        const T inv = T(1) / scale;
        for (int f = threadIdx.x; f < n3; f += blockDim.x) cz_st<T>(sm, offb[d.lc] + f, bs[f] * inv);
    }
    __syncthreads();
    const T om = (T)d.omega;
    // down
    for (int l = d.lc; l < d.nlev - 1; ++l) {
        const Grid3 g = d.g[l], gc = d.g[l + 1];
        const int n3 = (int)g.cells();
        SM* b = sm + offb[l];
        SM* x = sm + offx[l];
        for (int f = threadIdx.x; f < n3; f += blockDim.x) {
            const int i = f % g.nx, j = (f / g.nx) % g.ny, k = f / (g.nx * g.ny);
            cz_st<T>(x, f, om * cz_ld<T>(b, f) *
                                cz_invDf<T>(d, l, nb_count1(i, g.nx) + nb_count1(j, g.ny) + nb_count1(k, g.nz), f, kh2));
        }
        __syncthreads();
        for (int f = threadIdx.x; f < n3; f += blockDim.x) {
            const int i = f % g.nx, j = (f / g.nx) % g.ny, k = f / (g.nx * g.ny);
            cz_st<T>(tmp, f, cz_ld<T>(b, f) - cz_Ax<T>(d, l, x, g, i, j, k, kh2));
        }
        __syncthreads();
        SM* bc = sm + offb[l + 1];
        const int nc3 = (int)gc.cells();
        for (int C = threadIdx.x; C < nc3; C += blockDim.x) {
            const int I = C % gc.nx, J = (C / gc.nx) % gc.ny, K = C / (gc.nx * gc.ny);
            int fi0, fj0, fk0;
            float wxs[4], wys[4], wzs[4];
            const int ni = restrict_taps(g.nx > 1, I, gc.nx, fi0, wxs);
            const int nj = restrict_taps(g.ny > 1, J, gc.ny, fj0, wys);
            const int nk = restrict_taps(g.nz > 1, K, gc.nz, fk0, wzs);
            T acc = T(0);
            for (int c3 = 0; c3 < nk; ++c3) {
                const int fk = fk0 + c3;
                const T wz = (T)wzs[c3];
                if (wz == T(0)) continue;
                for (int b3 = 0; b3 < nj; ++b3) {
                    const int fj = fj0 + b3;
                    const T wy = (T)wys[b3] * wz;
                    if (wy == T(0)) continue;
                    for (int a3 = 0; a3 < ni; ++a3) {
                        const int fi = fi0 + a3;
                        const T w = (T)wxs[a3] * wy;
                        if (w == T(0)) continue;
                        acc += w * cz_ld<T>(tmp, fi + g.nx * (fj + g.ny * fk));
                    }
                }
            }
            cz_st<T>(bc, C, acc);
        }
        __syncthreads();
    }
    // bottom: one cell, exact
    {
        const int l = d.nlev - 1;
        if (threadIdx.x == 0) cz_st<T>(sm, offx[l], cz_ld<T>(sm, offb[l]) * cz_invDf<T>(d, l, 0, 0, kh2));
        __syncthreads();
    }
    // up
    for (int l = d.nlev - 2; l >= d.lc; --l) {
        const Grid3 g = d.g[l], gc = d.g[l + 1];
        const int n3 = (int)g.cells();
        const SM* b = sm + offb[l];
        SM* x = sm + offx[l];
        const SM* e = sm + offx[l + 1];
        for (int f = threadIdx.x; f < n3; f += blockDim.x) {
            const int i = f % g.nx, j = (f / g.nx) % g.ny, k = f / (g.nx * g.ny);
            int px[2], py[2], pz[2];
            float wx[2], wy[2], wz[2];
            prolong_taps(g.nx > 1, i, gc.nx, px, wx);
            prolong_taps(g.ny > 1, j, gc.ny, py, wy);
            prolong_taps(g.nz > 1, k, gc.nz, pz, wz);
            T pe = T(0);
            for (int c3 = 0; c3 < 2; ++c3)
                for (int b3 = 0; b3 < 2; ++b3)
                    for (int a3 = 0; a3 < 2; ++a3)
                        pe += (T)wx[a3] * (T)wy[b3] * (T)wz[c3] *
                              cz_ld<T>(e, px[a3] + gc.nx * (py[b3] + gc.ny * pz[c3]));
            cz_st<T>(tmp, f, cz_ld<T>(x, f) + pe);
        }
        __syncthreads();
        for (int f = threadIdx.x; f < n3; f += blockDim.x) {
            const int i = f % g.nx, j = (f / g.nx) % g.ny, k = f / (g.nx * g.ny);
            const T iD = cz_invDf<T>(d, l, nb_count1(i, g.nx) + nb_count1(j, g.ny) + nb_count1(k, g.nz), f, kh2);
            cz_st<T>(x, f, cz_ld<T>(tmp, f) + om * iD * (cz_ld<T>(b, f) - cz_Ax<T>(d, l, tmp, g, i, j, k, kh2)));
        }
        __syncthreads();
    }
    // write out (and b.e partial when this is the whole V-cycle)
    double dacc = 0.0;
    {
        const int n3 = (int)d.g[d.lc].cells();
        const SM* x = sm + offx[d.lc];
        for (int f = threadIdx.x; f < n3; f += blockDim.x) {
            const T xv = cz_ld<T>(x, f) * scale;
            es[f] = xv;
            dacc += (double)(bs[f] * xv);
        }
    }
    if (dot_part) {
        const double tsum = block_sum<kCoarseThreads>(dacc, red);
        if (threadIdx.x == 0) dot_part[(int64_t)col * kMaxPartials] = tsum;
    }
}

constexpr int kCoarseMaxCells = 4096;  // cells of the finest level the one-CTA kernel takes

static int coarse_smem_elems(const MGPlan& p) {
    int o = 0;
    for (int l = p.lc; l < p.nlev; ++l) o += 2 * (int)p.g[l].cells();
    return o + (int)p.g[p.lc].cells();
}
// bound over every plan: the levels below one of <= 4096 cells hold at most
// as many cells again in total (each has at most half the cells of the one above)
constexpr int kCoarseSmemElemsMax = 2 * (2 * kCoarseMaxCells) + kCoarseMaxCells;

static bool tiled_level(const Grid3& g) { return g.nx % SX == 0 && g.ny % SY == 0 && g.nz % 8 == 0; }

bool mg_plan_init(MGPlan& plan, const Grid3& g, double kh2, double c, double omega) {
    plan.kh2 = kh2;
    plan.c = c;
    plan.omega = omega;
    plan.g[0] = g;
    plan.ls[0] = 1.0;
    plan.lq[0] = 1.0;
    int nlev = 1;
    while (plan.g[nlev - 1].cells() > 1 && nlev < 16) {
        const Grid3& f = plan.g[nlev - 1];
        const int children = (f.nx > 1 ? 2 : 1) * (f.ny > 1 ? 2 : 1) * (f.nz > 1 ? 2 : 1);
        plan.g[nlev] = f.coarser();
        plan.ls[nlev] = plan.ls[nlev - 1] * children / 4.0;
        plan.lq[nlev] = plan.lq[nlev - 1] * 4.0;
        ++nlev;
    }
    plan.nlev = nlev;
    int lc = 0;
    while (lc < nlev - 1 && tiled_level(plan.g[lc])) ++lc;
    plan.lc = lc;
    return plan.g[nlev - 1].cells() == 1 && plan.g[lc].cells() <= kCoarseMaxCells;
}

bool mg_grid_supported(const Grid3& g) {
    MGPlan p;
    return mg_plan_init(p, g, 0.0, 1.0, 0.8);
}

void mg_plan_init(MGPlan& plan, int n, double kh2, double c, double omega) {
    mg_plan_init(plan, make_grid(n), kh2, c, omega);
}

template <typename T>
size_t mg_scratch_elems(const Grid3& g, int S) {
    MGPlan p;
    mg_plan_init(p, g, 0.0, 1.0, 0.8);
    size_t tot = 0;
    for (int l = 1; l <= p.lc; ++l) tot += 2 * (size_t)p.g[l].cells();
    return tot * (size_t)S;
}

template <typename T>
size_t mg_scratch_elems(int n, int S) {
    return mg_scratch_elems<T>(make_grid(n), S);
}

template <typename T>
void mg_plan_bind(MGPlan& plan, int S, T* scratch) {
    size_t o = 0;
    for (int l = 1; l <= plan.lc; ++l) {
        const size_t nl = (size_t)plan.g[l].cells();
        plan.b[l] = scratch + o;
        o += nl * (size_t)S;
        plan.e[l] = scratch + o;
        o += nl * (size_t)S;
    }
}

// z planes per CTA for the level sweeps: the longest march (fewest halo planes)
// that still gives at least four CTAs per SM of a 152-SM GPU.  The choice
// partitions the b.y partial sums of the up sweep, so it must not depend on
// how many columns share a batch: the FP32 path decides it for a batch of 64
// whatever the batch (a column gives the same bits alone, in a bigger batch or
// in a serving lane); the FP64 path, which runs one column at a time, for its S.
static int pick_sz(const Grid3& g, int S, int pref) {
    if ((pref == 8 || pref == 16 || pref == 32) && g.nz % pref == 0) return pref;
    const int base = (g.nx / SX) * (g.ny / SY);
    for (int sz = 32; sz > 8; sz >>= 1)
        if (g.nz % sz == 0 && (int64_t)base * (g.nz / sz) * S >= 4 * 152) return sz;
    return 8;
}

template <int NX, int TY>
static cudaError_t rows_attrs() {
    cudaError_t e = cudaFuncSetAttribute(k_mg_down_rows<NX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         down_rows_smem_bytes<NX, TY>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mg_up_rows<NX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 up_rows_smem_bytes<NX, TY>());
    return e;
}

template <typename T>
static cudaError_t mg_set_attrs() {
    cudaError_t e = cudaFuncSetAttribute(k_mg_coarse<T, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kCoarseSmemElemsMax * (int)sizeof(T));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mg_coarse<T, __half>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kCoarseSmemElemsMax * (int)sizeof(__half));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mg_down<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, down_smem_bytes<T>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mg_down<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, down_smem_bytes<T>());
    if constexpr (sizeof(T) == 4) {
        if (e == cudaSuccess) e = rows_attrs<128, 16>();
        if (e == cudaSuccess) e = rows_attrs<64, 16>();
        if (e == cudaSuccess) e = rows_attrs<32, 32>();
    }
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mg_up<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, up_smem_bytes<T>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mg_up<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, up_smem_bytes<T>());
    return e;
}

// cuTensorMapEncodeTiled from the driver (no link against libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (EncodeTiledFn) nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// tensor map of S stacked grids (column stride col_stride elements), box boxw x rows x 1 x 1
template <typename T>
static bool plane_map(CUtensorMap* m, const T* base, const Grid3& g, int S, int64_t col_stride, int rows,
                      int boxw = PW) {
    const EncodeTiledFn fn = encode_tiled();
    const size_t es = sizeof(T);
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15) || ((col_stride * es) & 15) || ((g.nx * es) & 15))
        return false;
    const cuuint64_t dims[4] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz, (cuuint64_t)S};
    const cuuint64_t strides[3] = {(cuuint64_t)g.nx * es, (cuuint64_t)g.nx * g.ny * es, (cuuint64_t)col_stride * es};
    const cuuint32_t box[4] = {(cuuint32_t)boxw, (cuuint32_t)rows, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(m, es == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
              const_cast<T*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Self-check of the bounded wait: one CTA waits on an mbarrier that is set up
// for one arrival which never comes, so phase 0 never completes; every thread
// must give up after the limit, raise the given fault word and return.
__global__ void k_wait_probe(unsigned long long* elapsed_ns, int* fault) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const unsigned long long t0 = global_ns();
    if (!mbar_wait(&bar, 0)) atomicExch(fault, 1);
    __syncthreads();
    if (threadIdx.x == 0) *elapsed_ns = global_ns() - t0;
}

cudaError_t mg_wait_probe(unsigned long long* elapsed_ns_dev, int* fault, cudaStream_t st) {
    k_wait_probe<<<1, 32, 0, st>>>(elapsed_ns_dev, fault);
    return cudaGetLastError();
}

cudaError_t mg_fault_read(const int* fault, int* host, cudaStream_t st) {
    return cudaMemcpyAsync(host, fault, sizeof(int), cudaMemcpyDeviceToHost, st);
}

cudaError_t mg_fault_clear(int* fault, cudaStream_t st) { return cudaMemsetAsync(fault, 0, sizeof(int), st); }

// once per instantiation and process (thread-safe static initialisation)
template <typename T>
static cudaError_t mg_attrs() {
    static const cudaError_t e = mg_set_attrs<T>();
    return e;
}

template <typename T>
void mg_coef_row(const MGPlan& plan, int l, double kh2, T out[21]) {
    MGPlan p = plan;
    p.kh2 = kh2;
    const LevelCoef<T> q = level_coef<T>(p, l);
    for (int k = 0; k < 7; ++k) {
        out[k] = q.oi[k];
        out[7 + k] = q.ois[k];
        out[14 + k] = q.rcD[k];
    }
}
template void mg_coef_row<float>(const MGPlan&, int, double, float*);
template void mg_coef_row<double>(const MGPlan&, int, double, double*);

cudaError_t mg_prepare() {
    cudaError_t e = mg_attrs<float>();
    if (e == cudaSuccess) e = mg_attrs<double>();
    if (e == cudaSuccess && !encode_tiled()) e = cudaErrorNotSupported;
    return e;
}

// z extent per row tile: the longest that still gives every SM a few CTAs (64 planes,
// which halve the halo planes of 32, only where that leaves four waves of CTAs)
static int pick_sz_rows(const Grid3& g, int ty, int S, int pref) {
    if ((pref == 8 || pref == 16 || pref == 32 || pref == 64) && g.nz % pref == 0) return pref;
    if (g.nz % 64 == 0 && (int64_t)(g.ny / ty) * (g.nz / 64) * S >= 4 * 152) return 64;
    for (int c = 32; c > 8; c >>= 1)
        if (g.nz % c == 0 && (int64_t)(g.ny / ty) * (g.nz / c) * S >= 2 * 152) return c;
    return 8;
}

// Row-tile down sweep of one level, FP32 with the level's constant diagonal: returns
// false (nothing launched) when the level's shape does not fit the row tiles.
template <int NX, int TY>
static bool down_rows_nx(const MGPlan& plan, int l, int S, const float* in, int64_t in_stride, float* out,
                         int64_t nc3, const int* active, int act_stride, cudaStream_t st) {
    using Sh = RowShape<NX, TY>;
    const Grid3& gf = plan.g[l];
    if (gf.ny % Sh::TY || gf.nz % 8) return false;
    const int sz = pick_sz_rows(gf, Sh::TY, S, plan.sz_pref);
    const int ntiles = (gf.ny / Sh::TY) * (gf.nz / sz);
    CUtensorMap map;
    if (!plane_map<float>(&map, in, gf, S, in_stride, Sh::R, NX)) return false;
    dim3 grid(ntiles < kMaxTilesPerCol ? ntiles : kMaxTilesPerCol, S);
    k_mg_down_rows<NX, TY><<<grid, Sh::NT, down_rows_smem_bytes<NX, TY>(), st>>>(
        map, gf, sz, level_coef<float>(plan, l), out, nc3, active, act_stride, plan.fault,
        static_cast<const float*>(plan.qtab[l]));
    return true;
}

// Row-tile up sweep of one level: returns the CTAs per column (the partials of b.y), or 0
// (nothing launched) when the level's shape does not fit the row tiles.  The tiling depends
// on the level's shape only, so each column's partial sums do not depend on the batch.
template <int NX, int TY>
static int up_rows_nx(const MGPlan& plan, int l, const float* b, int64_t b_stride, const float* ec, int64_t ec_stride,
                      float* y, int64_t y_stride, double* dot_part, int S, const int* active, int act_stride,
                      cudaStream_t st) {
    using Sh = RowShape<NX, TY>;
    const Grid3& gf = plan.g[l];
    if (gf.ny % Sh::TY || gf.nz % 8) return 0;
    const int sz = pick_sz_rows(gf, Sh::TY, 64, plan.sz_pref);
    const int ntiles = (gf.ny / Sh::TY) * (gf.nz / sz);
    const int nb = ntiles < kMaxTilesPerCol ? ntiles : kMaxTilesPerCol;
    CUtensorMap map;
    if (!plane_map<float>(&map, b, gf, S, b_stride, Sh::R, NX)) return 0;
    k_mg_up_rows<NX, TY><<<dim3(nb, S), Sh::NT, up_rows_smem_bytes<NX, TY>(), st>>>(
        map, gf, sz, level_coef<float>(plan, l), ec, ec_stride, y, y_stride, dot_part, active, act_stride,
        plan.fault, static_cast<const float*>(plan.qtab[l]));
    return nb;
}

template <typename T>
static int up_rows(const MGPlan& plan, int l, const T* b, int64_t b_stride, const T* ec, int64_t ec_stride, T* y,
                   int64_t y_stride, double* dot_part, int S, const int* active, int act_stride, cudaStream_t st) {
    if constexpr (sizeof(T) != 4) return 0;
    else {
        if (!plan.sweep_rows || plan.D[l]) return 0;
        // rows per tile: 16 (32 on 32-wide levels, where a warp holds four rows); 8-row tiles
        // (two CTAs per SM) measured slower on every level
#define SPDE_UP_ROWS(NX, TY) \
    up_rows_nx<NX, TY>(plan, l, b, b_stride, ec, ec_stride, y, y_stride, dot_part, S, active, act_stride, st)
        switch (plan.g[l].nx) {
            case 128: return SPDE_UP_ROWS(128, 16);
            case 64: return SPDE_UP_ROWS(64, 16);
            case 32: return SPDE_UP_ROWS(32, 32);
            default: return 0;
        }
#undef SPDE_UP_ROWS
    }
}

template <typename T>
static bool down_rows(const MGPlan& plan, int l, int S, const T* in, int64_t in_stride, T* out, int64_t nc3,
                      const int* active, int act_stride, cudaStream_t st) {
    if constexpr (sizeof(T) != 4) return false;
    else {
        if (!plan.sweep_rows || plan.D[l]) return false;
#define SPDE_DOWN_ROWS(NX, TY) down_rows_nx<NX, TY>(plan, l, S, in, in_stride, out, nc3, active, act_stride, st)
        switch (plan.g[l].nx) {
            case 128: return SPDE_DOWN_ROWS(128, 16);
            case 64: return SPDE_DOWN_ROWS(64, 16);
            case 32: return SPDE_DOWN_ROWS(32, 32);
            default: return false;
        }
#undef SPDE_DOWN_ROWS
    }
}

template <typename T>
int launch_vcycle(const MGPlan& plan, int S, const T* b, int64_t b_stride, T* y, int64_t y_stride, double* dot_part,
                  const int* active, int act_stride, cudaStream_t st) {
    const double prof_cols = plan.prof_cols > 0 ? plan.prof_cols : (double)S;
    if (mg_attrs<T>() != cudaSuccess) return -1;
    if (plan.lc > 0 && !plan.fault) return -1;  // the sweeps need the solve's fault word
    CoarseDesc d;
    d.lc = plan.lc;
    d.nlev = plan.nlev;
    d.kh2 = plan.kh2;
    d.kh2col = plan.kh2col;
    d.c = plan.c;
    d.omega = plan.omega;
    for (int l = 0; l < 16; ++l) {
        d.g[l] = plan.g[l];
        d.ls[l] = plan.ls[l];
        d.lq[l] = plan.lq[l];
        d.D[l] = plan.D[l];
    }
    // FP16 storage of the one-CTA levels (FP32 path only, when asked for)
    const bool half = plan.coarse_fp16 && sizeof(T) == 4;
    const size_t csm = (size_t)coarse_smem_elems(plan) * (half ? sizeof(__half) : sizeof(T));
    const double w = (double)sizeof(T);
    const int64_t s3 = plan.g[plan.lc].cells();
    if (plan.lc == 0) {
        prof_begin(PK_MG_COARSE, st);
        if (half)
            k_mg_coarse<T, __half><<<S, kCoarseThreads, csm, st>>>(d, b, b_stride, y, y_stride, dot_part, active,
                                                                   act_stride);
        else
            k_mg_coarse<T, T><<<S, kCoarseThreads, csm, st>>>(d, b, b_stride, y, y_stride, dot_part, active, act_stride);
        prof_end(st, prof_cols * 2.0 * (double)s3 * w);
        return 1;
    }
    // down sweeps
    const T* in = b;
    int64_t in_stride = b_stride;
    for (int l = 0; l < plan.lc; ++l) {
        const Grid3& gf = plan.g[l];
        const int64_t nc3 = plan.g[l + 1].cells();
        const int sz = pick_sz(gf, sizeof(T) == 4 ? 64 : S, plan.sz_pref);
        const int ntiles = (gf.nx / SX) * (gf.ny / SY) * (gf.nz / sz);
        dim3 grid(ntiles < kMaxTilesPerCol ? ntiles : kMaxTilesPerCol, S);
        T* out = static_cast<T*>(plan.b[l + 1]);
        prof_begin(PK_MG_DOWN, st);
        if (down_rows<T>(plan, l, S, in, in_stride, out, nc3, active, act_stride, st)) {
            prof_end(st, prof_cols * (1.0 + 0.125) * (double)gf.cells() * w);
            in = out;
            in_stride = nc3;
            continue;
        }
        CUtensorMap map;
        if (!plane_map<T>(&map, in, gf, S, in_stride, XH)) return -1;
        const T* Dl = static_cast<const T*>(plan.D[l]);
        const T* qt = static_cast<const T*>(plan.qtab[l]);
        if (Dl)
            k_mg_down<T, true><<<grid, dim3(32, 8), down_smem_bytes<T>(), st>>>(
                map, gf, sz, level_coef<T>(plan, l), out, nc3, active, act_stride, Dl, plan.fault, qt);
        else
            k_mg_down<T, false><<<grid, dim3(32, 8), down_smem_bytes<T>(), st>>>(
                map, gf, sz, level_coef<T>(plan, l), out, nc3, active, act_stride, nullptr, plan.fault, qt);
        prof_end(st, prof_cols * (1.0 + 0.125) * (double)gf.cells() * w);
        in = out;
        in_stride = nc3;
    }
    {
        prof_begin(PK_MG_COARSE, st);
        if (half)
            k_mg_coarse<T, __half><<<S, kCoarseThreads, csm, st>>>(d, static_cast<const T*>(plan.b[plan.lc]), s3,
                                                                   static_cast<T*>(plan.e[plan.lc]), s3, nullptr, active,
                                                                   act_stride);
        else
            k_mg_coarse<T, T><<<S, kCoarseThreads, csm, st>>>(d, static_cast<const T*>(plan.b[plan.lc]), s3,
                                                              static_cast<T*>(plan.e[plan.lc]), s3, nullptr, active,
                                                              act_stride);
        prof_end(st, prof_cols * 2.0 * (double)s3 * w);
    }
    int nblk0 = 1;
    for (int l = plan.lc - 1; l >= 0; --l) {
        const Grid3& gf = plan.g[l];
        const int64_t nf3 = gf.cells(), nc3 = plan.g[l + 1].cells();
        const int sz = pick_sz(gf, sizeof(T) == 4 ? 64 : S, plan.sz_pref);
        const int ntiles = (gf.nx / SX) * (gf.ny / SY) * (gf.nz / sz);
        const int nb = ntiles < kMaxTilesPerCol ? ntiles : kMaxTilesPerCol;
        dim3 grid(nb, S);
        const T* bl = (l == 0) ? b : static_cast<const T*>(plan.b[l]);
        const int64_t bls = (l == 0) ? b_stride : nf3;
        T* yl = (l == 0) ? y : static_cast<T*>(plan.e[l]);
        const int64_t yls = (l == 0) ? y_stride : nf3;
        prof_begin(PK_MG_UP, st);
        const int nbr = up_rows<T>(plan, l, bl, bls, static_cast<const T*>(plan.e[l + 1]), nc3, yl, yls,
                                   (l == 0) ? dot_part : nullptr, S, active, act_stride, st);
        if (nbr > 0) {
            prof_end(st, prof_cols * (2.0 + 0.125) * (double)nf3 * w);
            if (l == 0) nblk0 = nbr;
            continue;
        }
        CUtensorMap map;
        if (!plane_map<T>(&map, bl, gf, S, bls, BH)) return -1;
        const T* Dl = static_cast<const T*>(plan.D[l]);
        const T* qt = static_cast<const T*>(plan.qtab[l]);
        if (Dl)
            k_mg_up<T, true><<<grid, dim3(32, 8), up_smem_bytes<T>(), st>>>(
                map, gf, sz, level_coef<T>(plan, l), static_cast<const T*>(plan.e[l + 1]), nc3, yl, yls,
                (l == 0) ? dot_part : nullptr, active, act_stride, Dl, plan.fault, qt);
        else
            k_mg_up<T, false><<<grid, dim3(32, 8), up_smem_bytes<T>(), st>>>(
                map, gf, sz, level_coef<T>(plan, l), static_cast<const T*>(plan.e[l + 1]), nc3, yl, yls,
                (l == 0) ? dot_part : nullptr, active, act_stride, nullptr, plan.fault, qt);
        prof_end(st, prof_cols * (2.0 + 0.125) * (double)nf3 * w);
        if (l == 0) nblk0 = nb;
    }
    return nblk0;
}

#define SPDE_MG_INST(T)                                                                                            \
    template int launch_vcycle<T>(const MGPlan&, int, const T*, int64_t, T*, int64_t, double*, const int*, int,   \
                                  cudaStream_t);                                                                   \
    template size_t mg_scratch_elems<T>(int, int);                                                                 \
    template size_t mg_scratch_elems<T>(const Grid3&, int);                                                        \
    template void mg_plan_bind<T>(MGPlan&, int, T*);
SPDE_MG_INST(float)
SPDE_MG_INST(double)

}  // namespace spde
