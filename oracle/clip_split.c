/*
 * Tet / grid-cell intersection volumes in plain C (oracle; test and
 * baseline infrastructure, never linked into the library).
 *
 * Sec. 5.1: with piecewise-constant spaces on both meshes the coupling entry
 * G[tau][c] is the volume of tau cap c.  Same method as the oracle's exact
 * rational statement (clip.tet_box_volume_exact), in FP64: the cell box is
 * the intersection of six half-spaces {s (x_a - b) <= 0}; cutting a tet by
 * one leaves nothing, the whole tet, a corner tet (one vertex inside), a
 * prism (three inside) or a wedge (two inside), prisms and wedges split
 * into three tets; the volume is the sum of |det| / 6 over the pieces.
 * Coordinates are taken relative to the cell corner in units of h.
 *
 * oracle_clip_candidates fills one slot per candidate cell of every tet
 * (the cells of its bounding-box range, x fastest, then y, then z, starting
 * at cand_off[t]): the cell index and the intersection volume (0 for cells
 * the tet misses).  Tets are processed in parallel when built with OpenMP.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
    double p[4][3];
} tet_t;

typedef struct {
    tet_t* t;
    int n, cap;
} tet_list;

static int push(tet_list* L, const double* a, const double* b, const double* c, const double* d) {
    if (L->n == L->cap) {
        int nc = L->cap ? 2 * L->cap : 64;
        tet_t* nt = (tet_t*)realloc(L->t, (size_t)nc * sizeof(tet_t));
        if (!nt) return -1;
        L->t = nt;
        L->cap = nc;
    }
    tet_t* o = &L->t[L->n++];
    for (int k = 0; k < 3; ++k) {
        o->p[0][k] = a[k];
        o->p[1][k] = b[k];
        o->p[2][k] = c[k];
        o->p[3][k] = d[k];
    }
    return 0;
}

/* the point of edge a-b where coordinate ax equals bound (da, db: signed distances) */
static void meet(const double* a, const double* b, double da, double db, int ax, double bound, double* q) {
    const double s = da / (da - db);
    for (int k = 0; k < 3; ++k) q[k] = a[k] + s * (b[k] - a[k]);
    q[ax] = bound;
}

/* keep the parts of the tets of `in` with sign * (x[ax] - bound) <= 0 */
static int cut(const tet_list* in, tet_list* out, int ax, double bound, double sign) {
    out->n = 0;
    for (int i = 0; i < in->n; ++i) {
        const tet_t* t = &in->t[i];
        double d[4];
        int ins[4], outs[4], ni = 0, no = 0, strict = 0;
        for (int v = 0; v < 4; ++v) {
            d[v] = sign * (t->p[v][ax] - bound);
            if (d[v] > 0.0) outs[no++] = v;
            else {
                ins[ni++] = v;
                if (d[v] < 0.0) strict = 1;
            }
        }
        if (no == 0) {
            if (push(out, t->p[0], t->p[1], t->p[2], t->p[3])) return -1;
            continue;
        }
        if (!strict) continue; /* what is left lies in the plane */
        if (ni == 1) {
            const int v = ins[0];
            double q[3][3];
            for (int k = 0; k < 3; ++k) meet(t->p[v], t->p[outs[k]], d[v], d[outs[k]], ax, bound, q[k]);
            if (push(out, t->p[v], q[0], q[1], q[2])) return -1;
        } else if (ni == 3) {
            const int o = outs[0];
            double q[3][3];
            for (int k = 0; k < 3; ++k) meet(t->p[ins[k]], t->p[o], d[ins[k]], d[o], ax, bound, q[k]);
            const double *v1 = t->p[ins[0]], *v2 = t->p[ins[1]], *v3 = t->p[ins[2]];
            /* prism v1 v2 v3 / q0 q1 q2 */
            if (push(out, v1, v2, v3, q[0]) || push(out, v2, v3, q[0], q[1]) || push(out, v3, q[0], q[1], q[2]))
                return -1;
        } else {
            const double *v1 = t->p[ins[0]], *v2 = t->p[ins[1]];
            double p11[3], p12[3], p21[3], p22[3];
            meet(v1, t->p[outs[0]], d[ins[0]], d[outs[0]], ax, bound, p11);
            meet(v1, t->p[outs[1]], d[ins[0]], d[outs[1]], ax, bound, p12);
            meet(v2, t->p[outs[0]], d[ins[1]], d[outs[0]], ax, bound, p21);
            meet(v2, t->p[outs[1]], d[ins[1]], d[outs[1]], ax, bound, p22);
            /* wedge: triangle v1 p11 p12 above triangle v2 p21 p22 */
            if (push(out, v1, p11, p12, v2) || push(out, p11, p12, v2, p21) || push(out, p12, v2, p21, p22))
                return -1;
        }
    }
    return 0;
}

static double det6(const tet_t* t) {
    double u[3], v[3], w[3];
    for (int k = 0; k < 3; ++k) {
        u[k] = t->p[1][k] - t->p[0][k];
        v[k] = t->p[2][k] - t->p[0][k];
        w[k] = t->p[3][k] - t->p[0][k];
    }
    return u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) + u[2] * (v[0] * w[1] - v[1] * w[0]);
}

/* volume of tet q (cell-local coordinates, units of h) inside [0,1]^3; -1 on allocation failure */
static double unit_cell_volume(const double q[4][3], tet_list* A, tet_list* B) {
    A->n = 0;
    if (push(A, q[0], q[1], q[2], q[3])) return -1.0;
    for (int ax = 0; ax < 3; ++ax) {
        if (cut(A, B, ax, 0.0, -1.0)) return -1.0;
        if (cut(B, A, ax, 1.0, 1.0)) return -1.0;
        if (A->n == 0) return 0.0;
    }
    double v = 0.0;
    for (int i = 0; i < A->n; ++i) v += fabs(det6(&A->t[i]));
    return v / 6.0;
}

int oracle_clip_candidates(int64_t ntets, const double* xyz, const int32_t* tets, const int32_t* n, const double* lo,
                           double h, const int64_t* cand_off, int32_t* ccell, double* cvol) {
    int failed = 0;
#pragma omp parallel
    {
        tet_list A = {0, 0, 0}, B = {0, 0, 0};
#pragma omp for schedule(dynamic, 256)
        for (int64_t t = 0; t < ntets; ++t) {
            double p[4][3];
            for (int v = 0; v < 4; ++v)
                for (int k = 0; k < 3; ++k) p[v][k] = xyz[3 * (int64_t)tets[4 * t + v] + k];
            int a[3], b[3];
            for (int k = 0; k < 3; ++k) {
                double mn = p[0][k], mx = p[0][k];
                for (int v = 1; v < 4; ++v) {
                    mn = fmin(mn, p[v][k]);
                    mx = fmax(mx, p[v][k]);
                }
                a[k] = (int)floor((mn - lo[k]) / h);
                b[k] = (int)floor((mx - lo[k]) / h);
                if (a[k] < 0) a[k] = 0;
                if (a[k] > n[k] - 1) a[k] = n[k] - 1;
                if (b[k] < 0) b[k] = 0;
                if (b[k] > n[k] - 1) b[k] = n[k] - 1;
            }
            int64_t o = cand_off[t];
            for (int k = a[2]; k <= b[2]; ++k)
                for (int j = a[1]; j <= b[1]; ++j)
                    for (int i = a[0]; i <= b[0]; ++i) {
                        const double c0[3] = {lo[0] + i * h, lo[1] + j * h, lo[2] + k * h};
                        double q[4][3];
                        for (int v = 0; v < 4; ++v)
                            for (int m = 0; m < 3; ++m) q[v][m] = (p[v][m] - c0[m]) / h;
                        const double vol = unit_cell_volume(q, &A, &B);
                        if (vol < 0.0) failed = 1;
                        ccell[o] = (int32_t)(i + (int64_t)n[0] * (j + (int64_t)n[1] * k));
                        cvol[o] = vol > 0.0 ? vol * h * h * h : 0.0;
                        ++o;
                    }
        }
        free(A.t);
        free(B.t);
    }
    return failed ? -1 : 0;
}
