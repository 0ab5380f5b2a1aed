"""GPU parity of the float32 difference-form energy change (tc_subdomain_delta_energy_mixed).

The kernel reports, per subdomain, an error bound 2^-15 sum |u|_a (1/|d| + 1/|d'|)/|d'| that must hold against
the exact energy change.  Against the float64 oracle the comparison allows the bound plus the
oracle's own rounding (1e-13 E_sub); against a 40-digit brute force (small cases) it allows the
bound alone.
"""

from __future__ import annotations

import mpmath as mp
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2609_24722_b300 as tc

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def exact_delta(pos, sub, new):
    """40-digit sum of the pair differences of moving charges `sub` to `new`."""
    mp.mp.dps = 40
    inA = np.zeros(len(pos), bool)
    inA[sub] = True
    P = [(mp.mpf(float(x)), mp.mpf(float(y))) for x, y in pos]
    Nw = [(mp.mpf(float(x)), mp.mpf(float(y))) for x, y in new]
    tot = mp.mpf(0)
    for a, i in enumerate(sub):
        for j in range(len(pos)):
            if inA[j]:
                continue
            tot += 1 / mp.sqrt((Nw[a][0] - P[j][0]) ** 2 + (Nw[a][1] - P[j][1]) ** 2) \
                - 1 / mp.sqrt((P[i][0] - P[j][0]) ** 2 + (P[i][1] - P[j][1]) ** 2)
        for b in range(a + 1, len(sub)):
            k = sub[b]
            tot += 1 / mp.sqrt((Nw[a][0] - Nw[b][0]) ** 2 + (Nw[a][1] - Nw[b][1]) ** 2) \
                - 1 / mp.sqrt((P[i][0] - P[k][0]) ** 2 + (P[i][1] - P[k][1]) ** 2)
    return tot


@pytest.mark.parametrize("n,scale", [(3000, 2e-3), (3001, 1e-5), (5000, 3e-8)])
def test_delta_mixed_within_bound_of_oracle(n, scale):
    pos = synth.lattice_disk(n, 4)
    subs = synth.subdomains(pos, 7, 20, 700, 5)
    idx, off = synth.to_csr(subs)
    rng = np.random.default_rng(9)
    new = oracle.project(pos[idx] + rng.normal(0, scale, (idx.size, 2)))
    d, b = tc.subdomain_delta_energy_mixed(T(pos), T(idx), T(off), T(new))
    tc.sync_status()
    d, b = d.cpu().numpy(), b.cpu().numpy()
    for s in range(len(subs)):
        ref = oracle.delta_energy(pos, subs[s], new[off[s]:off[s + 1]])
        _, _, esub = oracle.subdomain_grad(pos, subs[s], pos[subs[s]])
        assert b[s] > 0
        assert abs(d[s] - ref) <= b[s] + 1e-13 * esub, (s, d[s], ref, b[s])


def test_delta_mixed_small_moves_against_exact():
    """For tiny moves the difference form stays within its bound of the exact change, where float64
    pair differences already lose digits to cancellation."""
    n = 160
    pos = synth.arcsine_disk(n, 12)
    subs = [np.array([3, 40, 77, 78, 120], dtype=np.int32), np.array([5, 6, 7, 8, 9, 150], dtype=np.int32)]
    idx, off = synth.to_csr(subs)
    rng = np.random.default_rng(3)
    new = oracle.project(pos[idx] + rng.normal(0, 1e-11, (idx.size, 2)))
    d, b = tc.subdomain_delta_energy_mixed(T(pos), T(idx), T(off), T(new))
    d64 = tc.subdomain_delta_energy(T(pos), T(idx), T(off), T(new))
    tc.sync_status()
    d, b, d64 = d.cpu().numpy(), b.cpu().numpy(), d64.cpu().numpy()
    err32, err64 = 0.0, 0.0
    for s in range(2):
        ex = float(exact_delta(pos, subs[s], new[off[s]:off[s + 1]]))
        assert abs(d[s] - ex) <= b[s], (s, d[s], ex, b[s])
        assert abs(d[s] - ex) <= 1e-3 * abs(ex)
        err32 += abs(d[s] - ex)
        err64 += abs(d64[s] - ex)
    # the float64 direct form loses more to cancellation than the float32 difference form
    assert err32 <= err64


def test_delta_mixed_edge_cases():
    pos = synth.arcsine_disk(600, 2)
    # empty subdomain, a subdomain holding every charge, a single charge
    subs = [np.zeros(0, dtype=np.int32), np.arange(600, dtype=np.int32), np.array([17], dtype=np.int32)]
    idx, off = synth.to_csr(subs)
    rng = np.random.default_rng(1)
    new = oracle.project(pos[idx] + rng.normal(0, 1e-3, (idx.size, 2)))
    d, b = tc.subdomain_delta_energy_mixed(T(pos), T(idx), T(off), T(new))
    tc.sync_status()
    d, b = d.cpu().numpy(), b.cpu().numpy()
    assert d[0] == 0.0 and b[0] == 0.0
    e0 = oracle.energy(pos)
    for s in [1, 2]:
        ref = oracle.delta_energy(pos, subs[s], new[off[s]:off[s + 1]])
        assert abs(d[s] - ref) <= b[s] + 1e-13 * e0
    # zero subdomains
    z = torch.zeros(1, dtype=torch.int64, device=DEV)
    d0, b0 = tc.subdomain_delta_energy_mixed(T(pos), torch.zeros(0, dtype=torch.int32, device=DEV), z,
                                             torch.zeros((0, 2), dtype=torch.float64, device=DEV))
    assert d0.numel() == 0
    # a move onto another charge (dyadic coordinates: the float32 separation is exactly zero)
    grid = np.array([[0.25, 0.5], [-0.125, 0.375], [0.5, -0.25], [0.0, 0.0]])
    bad = grid[[1]]
    with pytest.raises(tc.TCError):
        tc.subdomain_delta_energy_mixed(T(grid), T(np.array([0], dtype=np.int32)), T(np.array([0, 1])), T(bad))
        tc.sync_status()
    # landing 1e-6 from another charge: finite, and the bound covers the error or exceeds the result
    near = grid[[1]] + np.array([[1e-6, 0.0]])
    d1, b1 = tc.subdomain_delta_energy_mixed(T(grid), T(np.array([0], dtype=np.int32)), T(np.array([0, 1])),
                                             T(near))
    tc.sync_status()
    ref = oracle.delta_energy(grid, np.array([0]), near)
    assert abs(d1.item() - ref) <= b1.item() or b1.item() > abs(ref)


def test_delta_mixed_full_size_sampled():
    """N = 100 000 lattice background, three subdomains of 200..400 charges: within bound of the oracle."""
    n = 100_000
    pos = synth.lattice_disk(n, 0)
    pos = np.ascontiguousarray(pos[synth.zorder(pos)])
    subs = synth.subdomains(pos, 3, 200, 400, 2)
    idx, off = synth.to_csr(subs)
    rng = np.random.default_rng(4)
    new = oracle.project(pos[idx] + rng.normal(0, 1e-5, (idx.size, 2)))
    d, b = tc.subdomain_delta_energy_mixed(T(pos), T(idx), T(off), T(new))
    tc.sync_status()
    d, b = d.cpu().numpy(), b.cpu().numpy()
    for s in range(3):
        ref = oracle.delta_energy(pos, subs[s], new[off[s]:off[s + 1]])
        _, _, esub = oracle.subdomain_grad(pos, subs[s], pos[subs[s]])
        assert abs(d[s] - ref) <= b[s] + 1e-13 * esub
