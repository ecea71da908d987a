"""Plain restatement of the multigrid preconditioner operator (oracle).

Test infrastructure (oracle): never imported by the library.

The sampler preconditions MINRES on the mixed system (Sec. 4.2,
Eq. linsys) with a block-diagonal operator whose field block approximates
the inverse of the Schur complement S = kappa^2 W + B M^{-1} B^T by one
symmetric multigrid V-cycle on the cell-centred 7-point operator
    A_0 = kappa^2 h^2 I + c L          (scaled by the cell size, L = D D^T),
with the geometric hierarchy of nested embedding grids of Sec. 6.1.  This
module states that V-cycle operator as the library defines it:

  level l has n_l = n / 2^l cells per axis and operator
      A_l = 2^l (kappa^2 h^2 4^l I + c L_l)     (Neumann graph Laplacian L_l),
  transfers: P = tensor product of the 1-D cell-centred linear prolongation
      fine 2I   <- 3/4 e_I + 1/4 e_{I-1},   fine 2I+1 <- 3/4 e_I + 1/4 e_{I+1}
      (e_{-1} := e_0, e_{n_c} := e_{n_c - 1}: reflection at the no-flux wall),
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
    """Neumann 7-point graph Laplacian on an [z, y, x] cube array."""
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


def neighbour_count(n):
    c = np.full((n, n, n), 6.0)
    for ax in range(3):
        s = [slice(None)] * 3
        s[ax] = 0
        c[tuple(s)] -= 1.0
        s[ax] = n - 1
        c[tuple(s)] -= 1.0
    return c


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


def prolong(e):
    p = prolong_matrix_1d(e.shape[0])
    for ax in range(3):
        e = _along(p, e, ax)
    return e


def restrict(r):
    p = prolong_matrix_1d(r.shape[0] // 2)
    for ax in range(3):
        r = _along(p.T, r, ax)
    return r


class VCycle:
    def __init__(self, n, kh2, c=1.0, omega=0.8):
        self.n, self.kh2, self.c, self.omega = int(n), float(kh2), float(c), float(omega)

    def op(self, lvl, x):
        return 2.0 ** lvl * (self.kh2 * 4.0 ** lvl * x + self.c * laplacian(x))

    def diag(self, lvl, n):
        return 2.0 ** lvl * (self.kh2 * 4.0 ** lvl + self.c * neighbour_count(n))

    def apply(self, b, lvl=0):
        """x = V b for an [n_l]^3 array b at level lvl."""
        n = b.shape[0]
        d = self.diag(lvl, n)
        if n == 1:
            return b / d
        x = self.omega * b / d
        r = b - self.op(lvl, x)
        x = x + prolong(self.apply(restrict(r), lvl + 1))
        return x + self.omega * (b - self.op(lvl, x)) / d

    # ---- dense statement, for checking the recursive one -----------------
    def dense_operator(self, lvl, n):
        eye = np.eye(n ** 3)
        return np.stack([self.op(lvl, eye[i].reshape(n, n, n)).ravel() for i in range(n ** 3)], axis=1)

    def dense(self, lvl=0, n=None):
        n = self.n if n is None else n
        a = self.dense_operator(lvl, n)
        if n == 1:
            return np.linalg.inv(a)
        s = np.diag(self.omega / self.diag(lvl, n).ravel())
        p1 = prolong_matrix_1d(n // 2)
        # flat index i + n (j + n k): x fastest, so P = P_z (x) P_y (x) P_x
        p = np.kron(np.kron(p1, p1), p1)
        k = p @ self.dense(lvl + 1, n // 2) @ p.T
        eye = np.eye(n ** 3)
        return (eye - s @ a) @ (s + k @ (eye - a @ s)) + s
