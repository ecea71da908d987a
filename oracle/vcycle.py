"""Plain restatement of the multigrid preconditioner operator (oracle).

Test infrastructure (oracle): never imported by the library.

The sampler preconditions MINRES on the mixed system (Sec. 4.2,
Eq. linsys) with a block-diagonal operator whose field block approximates
the inverse of the Schur complement S = kappa^2 W + B M^{-1} B^T by one
symmetric multigrid V-cycle on the cell-centred 7-point operator
    A_0 = kappa^2 h^2 I + c L          (scaled by the cell size, L = D D^T),
with the geometric hierarchy of nested embedding grids of Sec. 6.1.  This
module states that V-cycle operator as the library defines it:

  level l + 1 halves every extent of level l that is above 1 (on a cube of
  n cells per axis, n_l = n / 2^l) and level l has the operator
      A_l = s_l (kappa^2 h^2 q_l I + c L_l)     (Neumann graph Laplacian L_l),
      q_l = 4^l,  s_{l+1} = s_l (children per coarse cell) / 4,
  so s_l = 2^l while all three extents halve;
  transfers: P = tensor product of the 1-D cell-centred linear prolongation
      fine 2I   <- 3/4 e_I + 1/4 e_{I-1},   fine 2I+1 <- 3/4 e_I + 1/4 e_{I+1}
      (e_{-1} := e_0, e_{n_c} := e_{n_c - 1}: reflection at the no-flux wall)
      along every coarsened axis and the identity along an axis of extent 1,
      restriction R = P^T;
  one damped-Jacobi sweep before and after the coarse correction
      (x <- x + omega D_l^{-1} (b - A_l x), starting from x = 0);
  the one-cell level is solved exactly.
The resulting operator is symmetric positive definite for 0 < omega < 1.

The paper prints no value for this operator (it uses BoomerAMG on a
hybridised system; this V-cycle is the sampler's own design), so it is
pinned against an independent dense statement (Kronecker products of the
1-D transfers, explicit matrices) and against its algebraic properties:
symmetry, positive definiteness, convergence, exactness of the one-cell
level, reproduction of linear functions by the prolongation.
"""
import numpy as np


def laplacian(x):
    """Neumann 7-point graph Laplacian on an [z, y, x] array (any extents)."""
    out = np.zeros_like(x)
    for ax in range(3):
        a = [slice(None)] * 3
        b = [slice(None)] * 3
        a[ax] = slice(0, -1)
        b[ax] = slice(1, None)
        d = x[tuple(a)] - x[tuple(b)]
        out[tuple(a)] += d
        out[tuple(b)] -= d
    return out


def _shape(n):
    """[z, y, x] extents from one n (a cube) or a [z, y, x] triple."""
    if np.ndim(n) == 0:
        return (int(n),) * 3
    return tuple(int(v) for v in n)


def neighbour_count(n):
    """Existing neighbours of every cell of an [z, y, x] grid (n: one extent or three)."""
    shape = _shape(n)
    c = np.full(shape, 6.0)
    for ax in range(3):
        s = [slice(None)] * 3
        s[ax] = 0
        c[tuple(s)] -= 1.0
        s[ax] = shape[ax] - 1
        c[tuple(s)] -= 1.0
    return c


def coarser(shape):
    return tuple(v // 2 if v > 1 else 1 for v in shape)


def prolong_matrix_1d(nc):
    """[2 nc, nc] cell-centred linear prolongation with wall reflection."""
    p = np.zeros((2 * nc, nc))
    for i in range(2 * nc):
        big = i // 2
        other = big - 1 if i % 2 == 0 else big + 1
        other = min(max(other, 0), nc - 1)
        p[i, big] += 0.75
        p[i, other] += 0.25
    return p


def _along(mat, x, ax):
    return np.moveaxis(np.tensordot(mat, x, axes=([1], [ax])), 0, ax)


def prolong(e, fine_shape=None):
    """P e onto fine_shape (default: twice e's extents); axes whose extent does not change
    are not coarsened (identity)."""
    fine_shape = tuple(2 * v for v in e.shape) if fine_shape is None else tuple(fine_shape)
    for ax in range(3):
        if fine_shape[ax] != e.shape[ax]:
            e = _along(prolong_matrix_1d(e.shape[ax]), e, ax)
    return e


def restrict(r):
    """R r = P^T r onto the next coarser grid (every extent above 1 halves)."""
    for ax in range(3):
        if r.shape[ax] > 1:
            r = _along(prolong_matrix_1d(r.shape[ax] // 2).T, r, ax)
    return r


class VCycle:
    """n: cells per axis of a cube, or the [z, y, x] extents of a box."""

    def __init__(self, n, kh2, c=1.0, omega=0.8):
        self.shape = _shape(n)
        self.n = self.shape[0] if len(set(self.shape)) == 1 else None
        self.kh2, self.c, self.omega = float(kh2), float(c), float(omega)
        # level grids and factors s_l, q_l
        self.shapes, self.s, self.q = [self.shape], [1.0], [1.0]
        while np.prod(self.shapes[-1]) > 1:
            sh = self.shapes[-1]
            children = int(np.prod([2 if v > 1 else 1 for v in sh]))
            self.shapes.append(coarser(sh))
            self.s.append(self.s[-1] * children / 4.0)
            self.q.append(self.q[-1] * 4.0)

    def op(self, lvl, x):
        return self.s[lvl] * (self.kh2 * self.q[lvl] * x + self.c * laplacian(x))

    def diag(self, lvl, n=None):
        shape = self.shapes[lvl] if n is None else _shape(n)
        return self.s[lvl] * (self.kh2 * self.q[lvl] + self.c * neighbour_count(shape))

    def apply(self, b, lvl=0):
        """x = V b for an array b of level lvl's [z, y, x] extents."""
        d = self.diag(lvl, b.shape)
        if b.size == 1:
            return b / d
        x = self.omega * b / d
        r = b - self.op(lvl, x)
        x = x + prolong(self.apply(restrict(r), lvl + 1), b.shape)
        return x + self.omega * (b - self.op(lvl, x)) / d

    # ---- dense statement, for checking the recursive one -----------------
    def dense_operator(self, lvl, n=None):
        shape = self.shapes[lvl] if n is None else _shape(n)
        m = int(np.prod(shape))
        eye = np.eye(m)
        return np.stack([self.op(lvl, eye[i].reshape(shape)).ravel() for i in range(m)], axis=1)

    def dense(self, lvl=0, n=None):
        shape = self.shapes[lvl] if n is None else _shape(n)
        a = self.dense_operator(lvl, shape)
        m = int(np.prod(shape))
        if m == 1:
            return np.linalg.inv(a)
        s = np.diag(self.omega / self.diag(lvl, shape).ravel())
        cs = coarser(shape)
        # flat index i + nx (j + ny k): x fastest, so P = P_z (x) P_y (x) P_x
        pz, py, px = (prolong_matrix_1d(cs[ax]) if shape[ax] > 1 else np.eye(1) for ax in range(3))
        p = np.kron(np.kron(pz, py), px)
        k = p @ self.dense(lvl + 1, cs) @ p.T
        eye = np.eye(m)
        return (eye - s @ a) @ (s + k @ (eye - a @ s)) + s
