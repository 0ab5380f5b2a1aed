"""GPU parity of the structure analysis (Sec. III C-D): Voronoi neighbours, coordination numbers
and psi6 of Eq. (psi6) against the oracle (the Delaunay edges of scipy's Qhull triangulation).

Neighbour sets are integer results and must match exactly; the inputs are seeded configurations
without cocircular quadruples (where the Voronoi diagram itself is not unique).  psi6 is a mean of
sixth powers of unit vectors in float64: 1e-13 absolute.
"""

from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import oracle
import synth
from oracle import structure as S
import paper_2609_24722_b300 as tc

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def check(pos, max_nbr=24):
    nb = S.neighbours(pos)
    zo, po = S.order(pos, nb)
    z, psi, summ, nbr = tc.voronoi_order(T(pos), max_nbr)
    tc.sync_status()
    z, psi, nbr = z.cpu().numpy(), psi.cpu().numpy(), nbr.cpu().numpy()
    np.testing.assert_array_equal(z, zo)
    for i in range(len(pos)):
        np.testing.assert_array_equal(nbr[i, :z[i]], nb[i])
        assert np.all(nbr[i, z[i]:] == -1)
    np.testing.assert_allclose(psi, po, rtol=0, atol=1e-13)
    so = S.summary(zo, po)
    np.testing.assert_allclose(summ["P_z"], so["P_z"], rtol=0, atol=1e-15)
    assert abs(summ["mean_abs_psi6"] - so["mean_abs_psi6"]) <= 1e-13
    assert abs(summ["abs_mean_psi6"] - so["abs_mean_psi6"]) <= 1e-13
    return z, psi, summ


@pytest.mark.parametrize("kind,n,seed", [("arcsine", 3000, 1), ("lattice", 2500, 2), ("arcsine", 257, 3),
                                         ("lattice", 700, 4)])
def test_voronoi_order_matches_oracle(kind, n, seed):
    pos = synth.arcsine_disk(n, seed) if kind == "arcsine" else synth.lattice_disk(n, seed, 0.05)
    check(pos)


def test_voronoi_order_split_configuration():
    """Boundary charges on the unit circle (the border-interior split) and a Hilbert-ordered layout."""
    n = 6000
    pos = synth.arcsine_disk(n, 7)
    pos = np.ascontiguousarray(pos[synth.zorder(pos)])
    p, _ = oracle.border_split(pos, oracle.boundary_count(n), 1 - 1 / (2 * math.sqrt(n)))
    check(p)


def test_voronoi_order_small_and_polygons():
    for k in [6, 7]:
        ang = 2 * math.pi * np.arange(k) / k + 0.05
        ring = 0.8 * np.stack([np.cos(ang), np.sin(ang)], 1)
        z, psi, _ = check(np.vstack([[0.0, 0.0], ring]))
        assert z[0] == k
    # three charges: a triangle, everyone neighbours everyone; two charges; one charge
    check(np.array([[0.1, 0.2], [-0.3, 0.0], [0.2, -0.4]]))
    check(np.array([[0.1, 0.2], [-0.3, 0.0]]))
    z, psi, summ, _ = tc.voronoi_order(T(np.array([[0.1, 0.2]])), 4)
    tc.sync_status()
    assert int(z[0]) == 0 and complex(psi[0]) == 0


def test_voronoi_coincident_charges_raise():
    pos = np.array([[0.1, 0.2], [0.1, 0.2], [0.5, 0.0], [-0.4, -0.1]])
    with pytest.raises(tc.TCError):
        tc.voronoi_order(T(pos))
        tc.sync_status()


def test_voronoi_order_full_size():
    """N = 100 000 after the border-interior split: the coordination numbers and psi6 of every charge."""
    n = 100_000
    pos = synth.lattice_disk(n, 0)
    pos = np.ascontiguousarray(pos[synth.zorder(pos)])
    p, _ = oracle.border_split(pos, oracle.boundary_count(n), 1 - 1 / (2 * math.sqrt(n)))
    z, psi, summ = check(p, max_nbr=16)
    # a jittered triangular lattice, radially compressed toward the wall: mostly sixfold
    assert summ["P_z"][6] > 0.8 and 0.5 < summ["mean_abs_psi6"] < 1.0
