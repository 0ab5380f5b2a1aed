"""Seeded synthetic inputs for charges in the unit disk.

This module is shared by the CUDA path's tests/bench and by the CPU oracle's
tests.  It holds only workload construction (random draws, lattice geometry,
nearest-charge selection); none of the method's arithmetic (no energies,
gradients, projections or optimiser steps) lives here.

Workload shapes follow the Thomson-problem-in-a-disk setting of the paper
(Sec. II A: N unit charges in a disk of radius R = 1; the continuum density of
the ground state is the arcsine measure rho(r) ~ 1/sqrt(1 - r^2), Sec. I).

Every generator takes an explicit integer seed and uses numpy's PCG64, so the
same call returns the same bytes on every machine with this numpy.
"""

from __future__ import annotations

import math

import numpy as np

__all__ = [
    "arcsine_disk",
    "jitter_inside",
    "lattice_disk",
    "ngon",
    "subdomains",
    "instances",
    "arcsine_spacing",
    "min_pair_distance",
    "to_csr",
    "zorder",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def arcsine_disk(n: int, seed: int) -> np.ndarray:
    """N charges drawn from the arcsine density of the unit disk.

    The radial CDF of rho(r) ~ 1/sqrt(1 - r^2) over the disk is
    F(r) = 1 - sqrt(1 - r^2); inverting F at u ~ U(0,1) gives
    r = sqrt(1 - (1 - u)^2).  Angles are uniform on [0, 2 pi).
    Returns a C-contiguous (n, 2) float64 array of (x, y).
    """
    g = _rng(seed)
    u = g.random(n)
    th = g.random(n) * (2.0 * math.pi)
    r = np.sqrt(1.0 - (1.0 - u) ** 2)
    pos = np.empty((n, 2), dtype=np.float64)
    pos[:, 0] = r * np.cos(th)
    pos[:, 1] = r * np.sin(th)
    return pos


def arcsine_spacing(n: int, r: np.ndarray | float) -> np.ndarray | float:
    """Local triangular-lattice spacing of N charges with the arcsine density.

    The normalised density is N / (2 pi sqrt(1 - r^2)) per unit area; a
    triangular lattice of spacing h has one charge per (sqrt(3)/2) h^2.
    """
    r = np.asarray(r, dtype=np.float64)
    rho = n / (2.0 * math.pi * np.sqrt(np.maximum(1.0 - r * r, 1e-300)))
    return np.sqrt(2.0 / (math.sqrt(3.0) * rho))


def jitter_inside(pos: np.ndarray, sigma: np.ndarray | float, seed: int,
                  max_tries: int = 64) -> np.ndarray:
    """Add N(0, sigma^2) noise per coordinate, redrawing any charge that leaves the disk.

    A charge whose jittered position has |r| > 1 gets a fresh draw (up to
    max_tries); if every draw leaves the disk it keeps its original position.
    No projection is applied, so every output charge satisfies |r| <= 1 exactly.
    """
    g = _rng(seed)
    pos = np.array(pos, dtype=np.float64, copy=True)
    n = pos.shape[0]
    sig = np.broadcast_to(np.asarray(sigma, dtype=np.float64), (n,))
    out = pos.copy()
    todo = np.arange(n)
    for _ in range(max_tries):
        if todo.size == 0:
            break
        trial = pos[todo] + g.standard_normal((todo.size, 2)) * sig[todo, None]
        ok = (trial[:, 0] ** 2 + trial[:, 1] ** 2) <= 1.0
        out[todo[ok]] = trial[ok]
        todo = todo[~ok]
    return np.ascontiguousarray(out)


def ngon(n: int, phase: float = 0.0, radius: float = 1.0) -> np.ndarray:
    """Regular n-gon on the circle of the given radius (angles 2 pi k / n + phase)."""
    k = np.arange(n, dtype=np.float64)
    th = 2.0 * math.pi * k / n + phase
    return np.ascontiguousarray(np.stack([radius * np.cos(th), radius * np.sin(th)], axis=1))


def _triangular_points(h: float) -> np.ndarray:
    """Triangular lattice of spacing h centred at the origin, points with |p| < 1."""
    dy = h * math.sqrt(3.0) / 2.0
    rows = int(math.ceil(1.0 / dy)) + 1
    cols = int(math.ceil(1.0 / h)) + 2
    j = np.arange(-rows, rows + 1)
    i = np.arange(-cols, cols + 1)
    jj, ii = np.meshgrid(j, i, indexing="ij")
    x = (ii + 0.5 * (jj & 1)) * h
    y = jj * dy
    pts = np.stack([x.ravel(), y.ravel()], axis=1)
    r2 = pts[:, 0] ** 2 + pts[:, 1] ** 2
    return pts[r2 < 1.0]


def lattice_disk(n: int, seed: int, jitter_frac: float = 0.005) -> np.ndarray:
    """Triangular lattice background shaped like the arcsine density.

    1. Lattice with uniform-area spacing h0 = sqrt(2 pi / (sqrt(3) n)), shrunk
       in 0.1 % steps until at least n points lie strictly inside the unit disk;
       the n points of smallest radius are kept.
    2. Radial map r -> sqrt(1 - (1 - r^2)^2), which carries the uniform-area
       radial CDF r^2 onto the arcsine CDF 1 - sqrt(1 - r^2), so the local
       spacing follows rho^(-1/2).
    3. Gaussian jitter of jitter_frac x the local arcsine spacing per
       coordinate (charges that would leave the disk are redrawn).
    """
    h = math.sqrt(2.0 * math.pi / (math.sqrt(3.0) * n))
    while True:
        pts = _triangular_points(h)
        if pts.shape[0] >= n:
            break
        h *= 0.999
    r2 = pts[:, 0] ** 2 + pts[:, 1] ** 2
    order = np.argsort(r2, kind="stable")[:n]
    pts = pts[order]
    r = np.sqrt(pts[:, 0] ** 2 + pts[:, 1] ** 2)
    rm = np.sqrt(1.0 - (1.0 - r * r) ** 2)
    scale = np.where(r > 0.0, rm / np.where(r > 0.0, r, 1.0), 0.0)
    pts = pts * scale[:, None]
    if jitter_frac > 0.0:
        sig = jitter_frac * arcsine_spacing(n, rm)
        pts = jitter_inside(pts, sig, seed)
    return np.ascontiguousarray(pts)


def subdomains(pos: np.ndarray, n_sub: int, m_lo: int, m_hi: int, seed: int,
               frac_at_charge: float = 0.8) -> list[np.ndarray]:
    """Circular subdomains: the m nearest charges to a centre, m ~ U{m_lo..m_hi}.

    With probability frac_at_charge the centre sits on a charge picked
    uniformly at random (a stand-in for the defect charges that the adaptive
    cycle picks from local energies, Sec. II C step 3); otherwise the centre is
    uniform over the disk.  Returns one strictly ascending int32 index array per
    subdomain.  Subdomains may overlap.
    """
    from scipy.spatial import cKDTree

    g = _rng(seed)
    n = pos.shape[0]
    tree = cKDTree(pos)
    out = []
    for _ in range(n_sub):
        m = int(g.integers(m_lo, m_hi + 1))
        m = min(m, n)
        if g.random() < frac_at_charge:
            c = pos[int(g.integers(0, n))]
        else:
            rr = math.sqrt(g.random())
            th = g.random() * 2.0 * math.pi
            c = np.array([rr * math.cos(th), rr * math.sin(th)])
        _, idx = tree.query(c, k=m)
        idx = np.atleast_1d(idx)
        out.append(np.sort(idx).astype(np.int32))
    return out


def disjoint_subdomains(pos: np.ndarray, n_sub: int, m_lo: int, m_hi: int, seed: int, fill: float = 0.9,
                        frac_at_charge: float = 0.8) -> list[np.ndarray]:
    """Pairwise disjoint subdomains with the size mix of subdomains(): m ~ U{m_lo..m_hi} scaled by
    fill * N / sum(m) (so together they hold about fill * N charges), centres drawn as in
    subdomains(), and subdomain s taking the m_s nearest charges to its centre that no earlier
    subdomain holds.  Returns one strictly ascending int32 index array per subdomain."""
    from scipy.spatial import cKDTree

    g = _rng(seed)
    n = pos.shape[0]
    m = g.integers(m_lo, m_hi + 1, size=n_sub).astype(np.float64)
    m = np.maximum(1, np.floor(m * fill * n / m.sum())).astype(np.int64)
    tree = cKDTree(pos)
    free = np.ones(n, dtype=bool)
    out = []
    for k in range(n_sub):
        if g.random() < frac_at_charge:
            c = pos[int(g.integers(0, n))]
        else:
            rr = math.sqrt(g.random())
            th = g.random() * 2.0 * math.pi
            c = np.array([rr * math.cos(th), rr * math.sin(th)])
        want = int(min(m[k], free.sum()))
        q = want
        while True:
            _, idx = tree.query(c, k=min(n, q))
            idx = np.atleast_1d(idx)
            idx = idx[free[idx]]
            if idx.size >= want or q >= n:
                break
            q = min(n, 2 * q + 16)
        idx = idx[:want]
        free[idx] = False
        out.append(np.sort(idx).astype(np.int32))
    return out


def to_csr(sets: list[np.ndarray]) -> tuple[np.ndarray, np.ndarray]:
    """Concatenate index sets into (idx int32, offsets int64[len+1])."""
    offsets = np.zeros(len(sets) + 1, dtype=np.int64)
    for k, s in enumerate(sets):
        offsets[k + 1] = offsets[k] + len(s)
    idx = np.concatenate(sets).astype(np.int32) if sets else np.zeros(0, np.int32)
    return np.ascontiguousarray(idx), offsets


def instances(n_inst: int, n_lo: int, n_hi: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Independent instances, N_k ~ U{n_lo..n_hi} (seed), each an arcsine init with seed + 1 + k.

    Returns concatenated positions (sum N_k, 2) and int64 world offsets [n_inst+1].
    """
    g = _rng(seed)
    sizes = g.integers(n_lo, n_hi + 1, size=n_inst)
    offs = np.zeros(n_inst + 1, dtype=np.int64)
    offs[1:] = np.cumsum(sizes)
    pos = np.concatenate([arcsine_disk(int(s), seed + 1 + k) for k, s in enumerate(sizes)])
    return np.ascontiguousarray(pos), offs


def min_pair_distance(pos: np.ndarray) -> float:
    """Smallest distance between two distinct charges (kd-tree nearest neighbour)."""
    from scipy.spatial import cKDTree

    if pos.shape[0] < 2:
        return math.inf
    d, _ = cKDTree(pos).query(pos, k=2)
    return float(d[:, 1].min())


def zorder(pos: np.ndarray, bits: int = 16) -> np.ndarray:
    """Permutation that lists the charges along a Hilbert curve through their cells.

    The charges are identical, so relabelling them changes nothing physical; a
    configuration stored in this order keeps nearby charges at nearby indices
    (the Hilbert curve, unlike the Z curve, never jumps across the square).
    Coordinates in [-1, 1] are quantised to 2^bits cells per axis; the curve
    index of a cell follows the usual quadrant-by-quadrant construction (take the
    quadrant, add its offset, rotate/reflect the remaining bits into it).  Ties
    keep index order (stable sort).
    """
    q = np.clip(((np.asarray(pos, dtype=np.float64) + 1.0) * 0.5 * (1 << bits)).astype(np.int64), 0,
                (1 << bits) - 1)
    x, y = q[:, 0].copy(), q[:, 1].copy()
    side = 1 << bits
    d = np.zeros(q.shape[0], dtype=np.int64)
    s = side >> 1
    while s > 0:
        rx = ((x & s) > 0).astype(np.int64)
        ry = ((y & s) > 0).astype(np.int64)
        d += s * s * ((3 * rx) ^ ry)
        flip = (ry == 0) & (rx == 1)
        x = np.where(flip, side - 1 - x, x)
        y = np.where(flip, side - 1 - y, y)
        swap = ry == 0
        x, y = np.where(swap, y, x), np.where(swap, x, y)
        s >>= 1
    return np.argsort(d, kind="stable")
