"""L2 projection onto the tet mesh and the lognormal map (oracle).

Test infrastructure (oracle): never imported by the library.

Eq. (proj_op): s = W_h^{-1} G theta_bar = Pi_h theta_bar, with W_h the
diagonal P0 mass matrix of the tet mesh (the tet volumes) and G the
intersection-volume coupling (Sec. 5.1, read with the indices the other way
round where the printed formula swaps tau and tau_bar).  The lognormal
coefficient is k = exp(theta), applied after the projection (workflow figure
of Sec. 6).
"""
import numpy as np
import scipy.sparse as sp

from .clip import tet_volume


def project_rows(xyz, tets, grows, theta_bar):
    """theta_h for the tets in grows (dict tet -> {cell: volume}).

    theta_bar: [S, ncells] or [ncells].  Returns {tet: value(s)}.
    """
    theta_bar = np.asarray(theta_bar, dtype=np.float64)
    out = {}
    for t, row in grows.items():
        vol = tet_volume(xyz[tets[t]])
        cells = np.fromiter(row.keys(), dtype=np.int64)
        g = np.fromiter(row.values(), dtype=np.float64)
        out[t] = (theta_bar[..., cells] @ g) / vol
    return out


def lognormal(theta_h):
    return np.exp(theta_h)


def tet_volumes(xyz, tets):
    """|tau| of every tet (vectorised determinant)."""
    p = np.asarray(xyz, dtype=np.float64)[np.asarray(tets)]
    return np.abs(np.einsum("ij,ij->i", np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), p[:, 3] - p[:, 0])) / 6.0


def projection_matrix(rowptr, col, g, vol, ncells):
    """Pi = W_h^{-1} G as a SciPy CSR matrix [ntets, ncells] (Eq. proj_op)."""
    vals = np.asarray(g, dtype=np.float64) / np.repeat(np.asarray(vol, dtype=np.float64), np.diff(rowptr))
    return sp.csr_matrix((vals, col, rowptr), shape=(len(rowptr) - 1, ncells))


def project_csr(pi, theta_bar):
    """theta_h = Pi theta_bar for theta_bar [ncells] or [S, ncells] (one sparse product)."""
    theta_bar = np.asarray(theta_bar, dtype=np.float64)
    return (pi @ theta_bar.T).T
