"""GPU parity of the float64-grade float32 pass (TC_F64X) against the float64 oracle.

TC_F64X forms every pair term in double-float arithmetic on the float32 pipes from a three-part
float32 split of the positions; it is held to the float64 tolerances: energy |dE|/E <= 1e-13,
gradient ||dg||/||g|| <= 1e-12 and |dg_i| <= 1e-12 G_i (G_i = sum_j 1/r_ij^2), local energies
|de_i| <= 1e-13 e_i.
"""

from __future__ import annotations

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


def gross(pos):
    out = np.empty(len(pos))
    for i in range(len(pos)):
        d = pos - pos[i]
        r2 = (d ** 2).sum(1)
        r2[i] = np.inf
        out[i] = (1.0 / r2).sum()
    return out


@pytest.mark.parametrize("n,kind", [(2, "a"), (3, "a"), (255, "a"), (257, "l"), (513, "a"), (1000, "l"),
                                    (2048, "a"), (3001, "l")])
def test_f64x_energy_grad_local_vs_oracle(n, kind):
    pos = synth.arcsine_disk(n, n) if kind == "a" else synth.lattice_disk(n, n, 0.05)
    p = T(pos)
    g, E = tc.grad(p, "fp64x", with_energy=True)
    E2, e = tc.local_energy(p, "fp64x")
    tc.sync_status()
    Eo, eo = oracle.energy(pos, local=True)
    go = oracle.grad(pos)
    G = gross(pos)
    assert abs(E.item() - Eo) <= 1e-13 * Eo
    assert abs(E2.item() - Eo) <= 1e-13 * Eo
    np.testing.assert_array_less(np.abs(e.cpu().numpy() - eo), 1e-13 * eo + 1e-300)
    gg = g.cpu().numpy()
    assert np.linalg.norm(gg - go) <= 1e-12 * np.linalg.norm(go)
    assert np.all(np.abs(gg - go) <= 1e-12 * G[:, None])


def test_f64x_relaxed_configuration_and_close_pairs():
    """A relaxed configuration (small gradient, close neighbours): the hardest case for the relative
    gradient test, since ||g|| is far below the gross force."""
    n = 1500
    pos = synth.arcsine_disk(n, 5)
    x, _, _ = oracle.lbfgs(pos, memory=8, max_iter=300, step0=1e-4, maxstep=0.01)
    p = T(x)
    g, E = tc.grad(p, "fp64x", with_energy=True)
    tc.sync_status()
    go, Eo = oracle.grad(x), oracle.energy(x)
    G = gross(x)
    assert abs(E.item() - Eo) <= 1e-13 * Eo
    assert np.all(np.abs(g.cpu().numpy() - go) <= 1e-12 * G[:, None])


def test_f64x_full_size_sampled_rows():
    n = 100_000
    pos = synth.arcsine_disk(n, 0)
    pos = np.ascontiguousarray(pos[synth.zorder(pos)])
    p = T(pos)
    g, E = tc.grad(p, "fp64x", with_energy=True)
    g64, E64 = tc.grad(p, "fp64", with_energy=True)
    tc.sync_status()
    assert abs(E.item() - E64.item()) <= 1e-13 * E64.item()
    rows = np.random.default_rng(3).choice(n, 40, replace=False).astype(np.int32)
    go, _ = oracle.rows_grad(pos, rows)
    gg = g.cpu().numpy()[rows]
    for k, i in enumerate(rows):
        d = pos - pos[i]
        r2 = (d ** 2).sum(1)
        r2[i] = np.inf
        Gi = (1.0 / r2).sum()
        assert np.all(np.abs(gg[k] - go[k]) <= 1e-12 * Gi)


def test_f64x_lbfgs_instances_match_oracle():
    """float64-grade float32 L-BFGS steps follow the oracle's float64 iteration."""
    sizes = [60, 150, 333]
    pos = np.concatenate([synth.arcsine_disk(m, 40 + m) for m in sizes])
    world = np.array([[0, 60], [60, 210], [210, 543]], dtype=np.int64)
    p = T(pos.copy())
    iters = 25
    r = tc.relax_subdomains(p, world=T(world), precision="fp64x", optimizer="lbfgs", n_steps=iters, memory=8,
                            step0=1e-4, maxstep=0.02, accept=False, want_energy=True)
    tc.sync_status()
    x = p.cpu().numpy()
    for k, (b, e) in enumerate(world):
        xo, it, rms = oracle.lbfgs(pos[b:e], memory=8, max_iter=iters, gtol=0.0, step0=1e-4, maxstep=0.02)
        assert np.abs(x[b:e] - xo).max() <= 1e-9
        assert abs(r.energy[k].item() - oracle.energy(xo)) <= 1e-12 * oracle.energy(xo)


def test_f64x_bb_subdomains_and_polish():
    """Subdomain BB steps in fp64x follow the oracle; a mixed run polished in fp64x ends stationary."""
    n = 2500
    pos = synth.lattice_disk(n, 7, 0.05)
    subs = synth.subdomains(pos, 5, 30, 200, 8)
    idx, off = synth.to_csr(subs)
    eta = 1e-4 / n
    p = T(pos.copy())
    r = tc.relax_subdomains(p, T(idx), T(off), precision="fp64x", optimizer="bb", n_steps=15, step0=eta,
                            alpha_min=0.0, alpha_max=10 * eta, accept=True)
    tc.sync_status()
    new = np.concatenate([oracle.subdomain_bb(pos, s, eta, 0.0, 10 * eta, 15) for s in subs])
    po, do, ao = oracle.accept_sequential(pos, idx, off, new)
    np.testing.assert_array_equal(r.status.cpu().numpy(), ao)
    np.testing.assert_allclose(p.cpu().numpy(), po, rtol=0, atol=1e-11)
    # polish in fp64x
    sizes = [5, 8, 60]
    pos2 = np.concatenate([synth.arcsine_disk(m, 7 + m) for m in sizes])
    world = np.array([[0, 5], [5, 13], [13, 73]], dtype=np.int64)
    q = T(pos2.copy())
    r2 = tc.relax_subdomains(q, world=T(world), precision="mixed", optimizer="lbfgs", n_steps=300, memory=8,
                             step0=1e-3, maxstep=0.05, gtol=1e-4, polish_steps=800, polish_gtol=1e-11,
                             accept=False, polish_precision="fp64x")
    tc.sync_status()
    assert np.all(r2.rms.cpu().numpy() < 1e-11)
