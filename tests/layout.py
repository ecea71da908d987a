"""Host-side mapping between the library's layout and the oracle's.

Library (scaled, one sample): [ux | uy | uz | theta], each nx ny nz long with
c = i + nx (j + ny k); ux[c] is the +x face of cell c, wall entries zero;
scaled unknowns u~ = h^{3/2} u, theta~ = h^{1/2} theta.
Oracle (unscaled): interior x-faces, y-faces, z-faces, then cells, in the
order documented in oracle.mixed.  `n` is one extent (a cube) or (nx, ny, nz).
"""
import numpy as np


def dims(n):
    if np.ndim(n) == 0:
        return (int(n),) * 3
    return tuple(int(v) for v in n)


def face_maps(n):
    """Index arrays: library position of each oracle x/y/z face."""
    nx, ny, nz = dims(n)
    # oracle x-face (ix = 1..nx-1, j, k), id (ix-1) + (nx-1)(j + ny k) -> library cell (ix-1, j, k)
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx - 1), indexing="ij")
    fx = (ii + nx * (jj + ny * kk)).ravel()
    # oracle y-face (i, jy = 1..ny-1, k), id i + nx((jy-1) + (ny-1) k) -> library cell (i, jy-1, k)
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny - 1), np.arange(nx), indexing="ij")
    fy = (ii + nx * (jj + ny * kk)).ravel()
    # oracle z-face (i, j, kz = 1..nz-1), id i + nx(j + ny (kz-1)) -> library cell (i, j, kz-1)
    kk, jj, ii = np.meshgrid(np.arange(nz - 1), np.arange(ny), np.arange(nx), indexing="ij")
    fz = (ii + nx * (jj + ny * kk)).ravel()
    return fx, fy, fz


def lib_to_oracle(v, n, h):
    """Scaled library vector [4 cells] -> unscaled oracle (u, theta)."""
    n3 = int(np.prod(dims(n)))
    fx, fy, fz = face_maps(n)
    u = np.concatenate([v[fx], v[n3 + fy], v[2 * n3 + fz]]) * h ** -1.5
    th = v[3 * n3:] * h ** -0.5
    return u, th


def oracle_to_lib(u, th, n, h):
    """Unscaled oracle (u, theta) -> scaled library vector [4 cells]."""
    n3 = int(np.prod(dims(n)))
    fx, fy, fz = face_maps(n)
    a, b = len(fx), len(fx) + len(fy)
    v = np.zeros(4 * n3)
    v[fx] = u[:a] * h ** 1.5
    v[n3 + fy] = u[a:b] * h ** 1.5
    v[2 * n3 + fz] = u[b:] * h ** 1.5
    v[3 * n3:] = th * h ** 0.5
    return v


def wall_mask(n):
    """True at library positions that are wall fluxes (held at zero)."""
    nx, ny, nz = dims(n)
    n3 = nx * ny * nz
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    m = np.zeros(4 * n3, dtype=bool)
    m[:n3] = (ii == nx - 1).ravel()
    m[n3:2 * n3] = (jj == ny - 1).ravel()
    m[2 * n3:3 * n3] = (kk == nz - 1).ravel()
    return m


def oracle_eq_to_lib(yu, yt, n, h):
    """Equation-space oracle vector (e.g. A x) -> scaled library layout (D y)."""
    return oracle_to_lib(yu * h ** -3.0, yt * h ** -1.0, n, h)
