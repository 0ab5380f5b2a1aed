"""Structure analysis of a configuration (Sec. III C-D) -- TEST INFRASTRUCTURE ONLY.

The paper identifies each charge's neighbours by the Voronoi tessellation, counts them (the
coordination number z_i, whose distribution P(z) it reports) and computes the local sixfold
bond-orientational order of Eq. (psi6),
    psi6_i = (1/z_i) sum_{j in N(i)} exp(6 i theta_ij),
theta_ij the angle of the bond i -> j against the x axis, with the averages <|psi6|> and
|<psi6>|.  Two charges are Voronoi neighbours when their cells share an edge, i.e. when they are
joined by an edge of the Delaunay triangulation (the dual graph); the triangulation comes from
scipy.spatial.Delaunay (Qhull), used here as a library step.  exp(6 i theta) is evaluated as the
sixth power of the unit bond vector written as a complex number, without trigonometric calls.

Only tests and the benchmark's checks use this module; the GPU library never imports it.
"""

from __future__ import annotations

import numpy as np


def neighbours(pos) -> list[np.ndarray]:
    """Voronoi neighbours of every charge (ascending indices), from the Delaunay edges."""
    from scipy.spatial import Delaunay

    p = np.asarray(pos, dtype=np.float64)
    n = p.shape[0]
    if n < 2:
        return [np.zeros(0, dtype=np.int64) for _ in range(n)]
    if n == 2:
        return [np.array([1]), np.array([0])]
    tri = Delaunay(p)
    sets = [set() for _ in range(n)]
    for a, b, c in tri.simplices:
        for u, v in ((a, b), (b, c), (c, a)):
            sets[u].add(v)
            sets[v].add(u)
    return [np.array(sorted(s), dtype=np.int64) for s in sets]


def order(pos, nbrs=None):
    """(z, psi6): coordination numbers and the complex local order parameter of Eq. (psi6)."""
    p = np.asarray(pos, dtype=np.float64)
    nbrs = neighbours(p) if nbrs is None else nbrs
    z = np.array([len(v) for v in nbrs], dtype=np.int64)
    psi = np.zeros(len(p), dtype=np.complex128)
    for i, v in enumerate(nbrs):
        if len(v) == 0:
            continue
        d = (p[v, 0] - p[i, 0]) + 1j * (p[v, 1] - p[i, 1])
        u = d / np.abs(d)
        psi[i] = (u ** 6).mean()
    return z, psi


def summary(z, psi, z_max: int = 15) -> dict:
    """P(z) for z = 0..z_max (the last bin holds z >= z_max), <|psi6|> and |<psi6>|."""
    zc = np.minimum(np.asarray(z), z_max)
    hist = np.bincount(zc, minlength=z_max + 1) / max(len(zc), 1)
    return {"P_z": hist, "mean_abs_psi6": float(np.abs(psi).mean()) if len(psi) else 0.0,
            "abs_mean_psi6": float(np.abs(psi.mean())) if len(psi) else 0.0}
