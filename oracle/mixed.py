"""Mixed RT0 x P0 discretisation of the reaction-diffusion SPDE (oracle).

Test infrastructure (oracle): never imported by the library.

Sec. 4, Eq. (SPDE): (kappa^2 - Laplace) theta = g W on the embedding box,
homogeneous Neumann (no-flux) boundary.  Mixed weak form, Eq.
(reac_diff_weak): find u in RT0, theta in P0 with
    m(u, v) + b(v, theta) = 0,
    b(u, q) - kappa^2 w(theta, q) = -g F^W(q),   u.n = 0 on the box boundary,
with m the L2 inner product of fluxes, w that of cell values and b(u, q) =
(div u, q).  The linear system is Eq. (linsys)/(linsys_blocks):
    [[M, B^T], [B, -kappa^2 W]] [u; theta] = [0; -g f],  f = W^{1/2} xi.
Eliminating u gives S theta = g f with S = kappa^2 W + B M^{-1} B^T, so
theta ~ N(0, g^2 S^{-1} W S^{-1}) (the covariance stated after
Eq. (linsys_blocks), with the g^2 factor written out).

The normaliser g follows Sec. 4: g = (4 pi)^{d/4} kappa^nu
sqrt(Gamma(nu + d/2) / Gamma(nu)), times sigma for marginal variance sigma^2;
at nu = 1/2, d = 3 this is g^2 = 8 pi kappa sigma^2.

Grid: nx x ny x nz cubes of edge h on the box lo + [0, nx h] x [0, ny h] x
[0, nz h] (n^3 for a cube; Sec. 7.2 embeds its domain in a non-cubic box).
Unknown ordering of this module (its own; unrelated to any device layout):
  x-faces (i = 1..nx-1, j, k)  id = (i-1) + (nx-1) (j + ny k)
  y-faces (i, j = 1..ny-1, k)  id = Nx + i + nx ((j-1) + (ny-1) k)
  z-faces (i, j, k = 1..nz-1)  id = Nx + Ny + i + nx (j + ny (k-1))
  cells   (i, j, k)            id = Nu + i + nx (j + ny k)
RT0 degree of freedom = the normal component u.e_axis on the face (the
paper fixes no scaling; theta does not depend on it).  Boundary faces carry
the essential condition u.n = 0 and are eliminated.

Space-dependent parameters (Sec. 1 states that the method, unlike circulant
embedding, admits correlation and marginal-variance functions that vary in
space; the paper gives no formula).  Reading taken here: kappa and sigma are
constant per cell of the embedding grid.  Then the reaction block is
diag(kappa_c^2) W and the noise of cell c carries the normaliser of Sec. 4
evaluated with that cell's kappa_c, sigma_c.  Every routine below that takes
`kappa` / `sigma` accepts either a number or an array of the cell values
(cell order i + nx (j + ny k)).
"""
import math

import numpy as np
import scipy.fft
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def g_normaliser(kappa, sigma=1.0, nu=0.5, d=3):
    """g of Sec. 4 times sigma: sigma (4 pi)^{d/4} kappa^nu sqrt(G(nu+d/2)/G(nu))."""
    return sigma * (4.0 * math.pi) ** (d / 4.0) * kappa ** nu * math.sqrt(
        math.gamma(nu + d / 2.0) / math.gamma(nu))


# --- local RT0 basis on the reference cube [0,1]^3 --------------------------
# local faces: 0 x-left, 1 x-right, 2 y-left, 3 y-right, 4 z-left, 5 z-right;
# each basis function is the lowest-order RT field whose normal component is
# 1 on its face and 0 on the other five, oriented along +axis.
def _local_basis(a, xi):
    axis, side = divmod(a, 2)
    v = np.zeros(xi.shape[:-1] + (3,))
    t = xi[..., axis]
    v[..., axis] = t if side == 1 else 1.0 - t
    return v


def _local_matrices():
    """6x6 reference mass and 6 reference divergence integrals.

    Mass by the tensor 2-point Gauss rule (exact for the quadratic
    integrands); divergence by the divergence of each (linear) basis field,
    evaluated by a centred difference, which is exact for linear fields.
    """
    gp = np.array([0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0)])
    pts = np.array([[x, y, z] for z in gp for y in gp for x in gp])
    wts = np.full(len(pts), 1.0 / 8.0)
    vals = [_local_basis(a, pts) for a in range(6)]
    mass = np.array([[np.sum(wts * np.einsum("pi,pi->p", vals[a], vals[b]))
                      for b in range(6)] for a in range(6)])
    div = np.zeros(6)
    eps = 0.125
    centre = np.array([[0.5, 0.5, 0.5]])
    for a in range(6):
        s = 0.0
        for ax in range(3):
            e = np.zeros(3)
            e[ax] = eps
            s += (_local_basis(a, centre + e)[0, ax] - _local_basis(a, centre - e)[0, ax]) / (2 * eps)
        div[a] = s  # constant over the cell; integral over the unit cube
    return mass, div


def _dims(n):
    """(nx, ny, nz) from one n (a cube) or three extents."""
    if np.ndim(n) == 0:
        return (int(n),) * 3
    return tuple(int(v) for v in n)


class MixedSystem:
    """Assembled [[M, B^T], [B, -kappa^2 W]] on a grid of spacing h: n is the
    number of cells per axis of a cube, or the extents (nx, ny, nz) of a box."""

    def __init__(self, n, h=None, lo=0.0):
        nx, ny, nz = self.dims = _dims(n)
        self.n = nx if nx == ny == nz else None
        self.h = h = (1.0 / nx) if h is None else float(h)
        self.lo = lo
        self.Nx = (nx - 1) * ny * nz
        self.Ny = nx * (ny - 1) * nz
        self.Nz = nx * ny * (nz - 1)
        self.Nu = self.Nx + self.Ny + self.Nz
        self.Nt = nx * ny * nz
        mass_ref, div_ref = _local_matrices()
        # physical cell: phi(x) = phi_ref((x - x0)/h), so
        #   int phi_a.phi_b = h^3 mass_ref,  int div phi_a = h^3 (1/h) div_ref
        mloc = h ** 3 * mass_ref
        bloc = h ** 2 * div_ref
        i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
        i, j, k = i.ravel(), j.ravel(), k.ravel()
        cell = i + nx * (j + ny * k)
        ext = (nx, ny, nz)
        gids = np.full((len(cell), 6), -1, dtype=np.int64)
        for a in range(6):
            axis, side = divmod(a, 2)
            fi = [i.copy(), j.copy(), k.copy()]
            fi[axis] = fi[axis] + side  # face position along axis, 0..n_axis
            pos = fi[axis]
            inner = (pos >= 1) & (pos <= ext[axis] - 1)
            if axis == 0:
                gid = (fi[0] - 1) + (nx - 1) * (fi[1] + ny * fi[2])
            elif axis == 1:
                gid = self.Nx + fi[0] + nx * ((fi[1] - 1) + (ny - 1) * fi[2])
            else:
                gid = self.Nx + self.Ny + fi[0] + nx * (fi[1] + ny * (fi[2] - 1))
            gids[:, a] = np.where(inner, gid, -1)
        rows, cols, vals = [], [], []
        for a in range(6):
            for b in range(6):
                if mloc[a, b] == 0.0:
                    continue
                ok = (gids[:, a] >= 0) & (gids[:, b] >= 0)
                rows.append(gids[ok, a])
                cols.append(gids[ok, b])
                vals.append(np.full(ok.sum(), mloc[a, b]))
        self.M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                               shape=(self.Nu, self.Nu))
        br, bc, bv = [], [], []
        for a in range(6):
            ok = gids[:, a] >= 0
            br.append(cell[ok])
            bc.append(gids[ok, a])
            bv.append(np.full(ok.sum(), bloc[a]))
        self.B = sp.csr_matrix((np.concatenate(bv), (np.concatenate(br), np.concatenate(bc))),
                               shape=(self.Nt, self.Nu))
        self.W = sp.identity(self.Nt, format="csr") * h ** 3

    def matrix(self, kappa):
        k2 = np.broadcast_to(np.asarray(kappa, dtype=np.float64) ** 2, (self.Nt,))
        return sp.bmat([[self.M, self.B.T], [self.B, -(sp.diags(k2) @ self.W)]], format="csc")

    def apply(self, kappa, u, theta):
        """y = A [u; theta] with the assembled blocks."""
        yu = self.M @ u + self.B.T @ theta
        yt = self.B @ u - np.asarray(kappa, dtype=np.float64) ** 2 * (self.W @ theta)
        return yu, yt

    def rhs(self, kappa, sigma, xi):
        """F = [0; -g f], f = W^{1/2} xi (Sec. 4.2); g per cell for cell-wise kappa, sigma."""
        f = np.sqrt(self.W.diagonal()) * xi
        g = g_normaliser(np.asarray(kappa, dtype=np.float64), np.asarray(sigma, dtype=np.float64))
        return np.concatenate([np.zeros(self.Nu), -g * f])

    def solve_sparse(self, kappa, sigma, xi):
        """Sparse direct (SuperLU) solve of the full saddle-point system."""
        lu = spla.splu(self.matrix(kappa))
        sol = lu.solve(self.rhs(kappa, sigma, xi))
        return sol[:self.Nu], sol[self.Nu:]

    def solve_dense(self, kappa, sigma, xi):
        sol = np.linalg.solve(self.matrix(kappa).toarray(), self.rhs(kappa, sigma, xi))
        return sol[:self.Nu], sol[self.Nu:]


# --- closed form on the uniform box --------------------------------------
# Per axis (n_d cells along axis d) the divergence maps DST-I face modes to
# DCT-II cell modes with factor 2 h^2 sin(pi k / 2 n_d), and the 1-D RT0 mass
# matrix (tridiagonal h^3 (1/6, 2/3, 1/6)) is diagonal on DST-I modes with
# eigenvalue h^3 (2 + cos(pi k / n_d)) / 3.  Hence S = kappa^2 W + B M^{-1} B^T
# is diagonalised by the orthonormal 3-D DCT-II with eigenvalues
#   Lambda(k) = kappa^2 h^3 + h sum_d 12 sin^2(pi k_d / 2 n_d) / (2 + cos(pi k_d / n_d)).
def schur_eigenvalues(n, h, kappa):
    """Lambda on the [z, y, x] mode grid; n: one extent (a cube) or (nx, ny, nz)."""
    nx, ny, nz = _dims(n)

    def lam1(m):
        k = np.arange(m)
        return 12.0 * np.sin(np.pi * k / (2 * m)) ** 2 / (2.0 + np.cos(np.pi * k / m))

    return kappa ** 2 * h ** 3 + h * (lam1(nz)[:, None, None] + lam1(ny)[None, :, None] + lam1(nx)[None, None, :])


def solve_dct(n, kappa, sigma, xi, h=None):
    """theta = g S^{-1} W^{1/2} xi by the DCT-II diagonalisation.

    n: cells per axis of a cube, or (nx, ny, nz); xi is a flat array of the
    cell values (x fastest) or [S, cells].
    """
    nx, ny, nz = _dims(n)
    h = (1.0 / nx) if h is None else h
    lam = schur_eigenvalues((nx, ny, nz), h, kappa)
    xi = np.asarray(xi, dtype=np.float64)
    batch = xi.reshape(-1, nz, ny, nx)  # [S, z, y, x]
    f = h ** 1.5 * batch
    th = scipy.fft.idctn(scipy.fft.dctn(f, type=2, norm="ortho", axes=(1, 2, 3), workers=-1) / lam,
                         type=2, norm="ortho", axes=(1, 2, 3), workers=-1)
    return (g_normaliser(kappa, sigma) * th).reshape(xi.shape)


def _dct_matrix(n):
    k = np.arange(n)[:, None]
    i = np.arange(n)[None, :]
    c = np.sqrt(2.0 / n) * np.cos(np.pi * k * (2 * i + 1) / (2 * n))
    c[0] /= np.sqrt(2.0)
    return c


def variance_exact(n, kappa, sigma, h=None):
    """Exact discrete variance of every cell: diag(g^2 S^{-1} W S^{-1}).

    n: cells per axis of a cube, or (nx, ny, nz).  Returned as an [z, y, x] array.
    """
    nx, ny, nz = _dims(n)
    h = (1.0 / nx) if h is None else h
    lam = schur_eigenvalues((nx, ny, nz), h, kappa)  # [kz, ky, kx]
    a = 1.0 / lam ** 2
    # var[z, y, x] = sum_k C_z[kz, z]^2 C_y[ky, y]^2 C_x[kx, x]^2 a[kz, ky, kx]
    v = np.einsum("abc,az->zbc", a, _dct_matrix(nz) ** 2)
    v = np.einsum("zbc,by->zyc", v, _dct_matrix(ny) ** 2)
    v = np.einsum("zyc,cx->zyx", v, _dct_matrix(nx) ** 2)
    return g_normaliser(kappa, sigma) ** 2 * h ** 3 * v


def covariance_column(n, kappa, sigma, cell, h=None):
    """Column g^2 h^3 C^T Lambda^{-2} C e_cell of the exact covariance, flat (n: one extent or three)."""
    nx, ny, nz = _dims(n)
    h = (1.0 / nx) if h is None else h
    lam = schur_eigenvalues((nx, ny, nz), h, kappa)
    e = np.zeros(nx * ny * nz)
    e[cell] = 1.0
    e = e.reshape(nz, ny, nx)
    col = scipy.fft.idctn(scipy.fft.dctn(e, type=2, norm="ortho") / lam ** 2, type=2, norm="ortho")
    return g_normaliser(kappa, sigma) ** 2 * h ** 3 * col.ravel()


def neumann_image_variance(x, kappa, sigma, box=1.0, nimg=3):
    """Continuum variance sigma^2 sum_images exp(-kappa |x - x_img|) in a box.

    Neumann reflection at every face of [0, box]^3; the Green's function of
    (kappa^2 - Laplace) is exp(-kappa r) / (4 pi r), whose self-convolution
    normalised by g gives the exponential covariance (Sec. 4, nu = 1/2).
    """
    x = np.asarray(x, dtype=np.float64)
    tot = 0.0
    rng = range(-nimg, nimg + 1)
    for a in rng:
        for b in rng:
            for c in rng:
                img = []
                for d, m in zip(range(3), (a, b, c)):
                    # image of coordinate x_d under m reflections
                    if m % 2 == 0:
                        img.append(x[d] + m * box)
                    else:
                        img.append(-x[d] + (m + 1) * box)
                r = math.dist(x, img)
                tot += math.exp(-kappa * r)
    return sigma ** 2 * tot


def restrict_noise(xi_f, n_f):
    """Coarse normals of a coupled two-level sample (Sec. 6.2).

    The coarse right-hand side is P^T applied to the fine one, f_c = P^T
    W_f^{1/2} xi_f with P the piecewise-constant prolongation (each coarse
    cell's value copied to its 8 children).  Written as f_c = W_c^{1/2} xi_c,
    xi_c = W_c^{-1/2} P^T W_f^{1/2} xi_f.  Input/output flat, x fastest.
    """
    nx, ny, nz = _dims(n_f)  # one extent (a cube) or the fine box's (nx, ny, nz), all even
    h_f = 1.0
    h_c = 2.0 * h_f
    f = (h_f ** 1.5) * np.asarray(xi_f, dtype=np.float64).reshape(nz, ny, nx)
    fc = f.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).sum(axis=(1, 3, 5))
    return (fc / h_c ** 1.5).ravel()


def restriction_matrix(n_f):
    """Dense P^T (coarse x fine) of the piecewise-constant prolongation."""
    n_c = n_f // 2
    r = np.zeros((n_c ** 3, n_f ** 3))
    for k in range(n_f):
        for j in range(n_f):
            for i in range(n_f):
                r[(i // 2) + n_c * ((j // 2) + n_c * (k // 2)), i + n_f * (j + n_f * k)] = 1.0
    return r
