"""Host-side mapping between the library's layout and the oracle's.

Library (scaled, one sample): [ux | uy | uz | theta], each n^3 with
c = i + n (j + n k); ux[c] is the +x face of cell c, wall entries zero;
scaled unknowns u~ = h^{3/2} u, theta~ = h^{1/2} theta.
Oracle (unscaled): interior x-faces, y-faces, z-faces, then cells, in the
order documented in oracle.mixed.
"""
import numpy as np


def face_maps(n):
    """Index arrays: library position of each oracle x/y/z face."""
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    # oracle x-face (ix = 1..n-1, j, k): id (ix-1) + (n-1)(j + n k) -> library cell (ix-1, j, k)
    fx = []
    for kk in range(n):
        for jj in range(n):
            for ix in range(1, n):
                fx.append((ix - 1) + n * (jj + n * kk))
    fy = []
    for kk in range(n):
        for jy in range(1, n):
            for ii in range(n):
                fy.append(ii + n * ((jy - 1) + n * kk))
    fz = []
    for kz in range(1, n):
        for jj in range(n):
            for ii in range(n):
                fz.append(ii + n * (jj + n * (kz - 1)))
    return np.array(fx), np.array(fy), np.array(fz)


def lib_to_oracle(v, n, h):
    """Scaled library vector [4 n^3] -> unscaled oracle (u, theta)."""
    n3 = n ** 3
    fx, fy, fz = face_maps(n)
    u = np.concatenate([v[fx], v[n3 + fy], v[2 * n3 + fz]]) * h ** -1.5
    th = v[3 * n3:] * h ** -0.5
    return u, th


def oracle_to_lib(u, th, n, h):
    """Unscaled oracle (u, theta) -> scaled library vector [4 n^3]."""
    n3 = n ** 3
    fx, fy, fz = face_maps(n)
    nx = len(fx)
    v = np.zeros(4 * n3)
    v[fx] = u[:nx] * h ** 1.5
    v[n3 + fy] = u[nx:2 * nx] * h ** 1.5
    v[2 * n3 + fz] = u[2 * nx:] * h ** 1.5
    v[3 * n3:] = th * h ** 0.5
    return v


def wall_mask(n):
    """True at library positions that are wall fluxes (held at zero)."""
    n3 = n ** 3
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    # flat c = i + n (j + n k): build with (k, j, i) ordering
    kk, jj, ii = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    m = np.zeros(4 * n3, dtype=bool)
    m[:n3] = (ii == n - 1).ravel()
    m[n3:2 * n3] = (jj == n - 1).ravel()
    m[2 * n3:3 * n3] = (kk == n - 1).ravel()
    return m


def oracle_eq_to_lib(yu, yt, n, h):
    """Equation-space oracle vector (e.g. A x) -> scaled library layout (D y)."""
    return oracle_to_lib(yu * h ** -3.0, yt * h ** -1.0, n, h)
