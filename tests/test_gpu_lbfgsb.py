"""GPU parity of L-BFGS-B on the (t, u) box (optimizer "lbfgsb_tu"; Sec. II C step 4, Sec. II D).

The oracle's tco_lbfgsb runs the same iteration (generalized Cauchy point, subspace step,
capped step, optional Armijo halving) in float64.  The GPU keeps the small matrices by ring slot
and sums in a different order, and CUDA's sin, cos, asin and atan2 may differ from the host's in
the last place.  On short trajectories that pass many breakpoints, the charges match to 1e-9.
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
HALF_PI = 1.5707963267948966


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


@pytest.mark.parametrize("line_search,memory", [(0, 8), (8, 8), (0, 3)])
def test_lbfgsb_instances_match_oracle(line_search, memory):
    sizes = [60, 150, 333]
    pos = np.concatenate([synth.arcsine_disk(m, 50 + m) for m in sizes])
    world = np.array([[0, 60], [60, 210], [210, 543]], dtype=np.int64)
    p = T(pos.copy())
    iters = 30
    r = tc.relax_subdomains(p, world=T(world), precision="fp64", optimizer="lbfgsb_tu", n_steps=iters,
                            memory=memory, step0=1e-4, maxstep=0.02, accept=False, want_energy=True,
                            line_search=line_search)
    tc.sync_status()
    x = p.cpu().numpy()
    breaks = 0
    for k, (b, e) in enumerate(world):
        xo, it, rms, nb = oracle.lbfgsb(pos[b:e], memory=memory, max_iter=iters, step0=1e-4, maxstep=0.02,
                                        line_search=line_search)
        breaks += nb
        assert np.abs(x[b:e] - xo).max() <= 1e-9
        eg = oracle.energy(x[b:e])
        assert abs(r.energy[k].item() - eg) <= 1e-12 * eg
        assert abs(r.rms[k].item() - rms) <= 1e-6 * rms
        assert r.steps[k].item() == iters
    assert breaks >= 20  # the Cauchy searches passed breakpoints


def test_lbfgsb_pinned_boundary_matches_oracle():
    """Pinned charges on (cos u, sin u), the others r = sigma sin^2 t with t boxed."""
    n = 300
    pos = synth.arcsine_disk(n, 17)
    p0, f = oracle.border_split(pos, oracle.boundary_count(n), 0.97)
    p = T(p0.copy())
    iters = 40
    r = tc.relax_subdomains(p, world=T(np.array([[0, n]], dtype=np.int64)), flags=T(f), precision="fp64",
                            optimizer="lbfgsb_tu", n_steps=iters, memory=8, step0=1e-4, maxstep=0.02, radius=0.97,
                            accept=False)
    tc.sync_status()
    x = p.cpu().numpy()
    xo, _, rms, nb = oracle.lbfgsb(p0, memory=8, max_iter=iters, step0=1e-4, maxstep=0.02, radius=0.97, flags=f)
    assert nb >= 1
    assert np.abs(x - xo).max() <= 1e-9
    assert abs(r.rms[0].item() - rms) <= 1e-6 * rms
    rr = np.hypot(x[:, 0], x[:, 1])
    assert np.all(np.abs(rr[f == 1] - 1.0) <= 4.5e-16)
    assert np.all(rr[f == 0] <= 0.97 * (1 + 1e-15))


def test_lbfgsb_subdomain_of_every_charge_is_the_instance():
    """A subdomain holding every charge of its world follows the instance trajectory."""
    n = 200
    pos = synth.arcsine_disk(n, 23)
    world = T(np.array([[0, n]], dtype=np.int64))
    kw = dict(precision="fp64", optimizer="lbfgsb_tu", n_steps=25, memory=5, step0=1e-4, maxstep=0.02,
              accept=False, want_energy=True)
    p1 = T(pos.copy())
    r1 = tc.relax_subdomains(p1, world=world, **kw)
    tc.sync_status()
    p2 = T(pos.copy())
    idx = T(np.arange(n, dtype=np.int32))
    off = T(np.array([0, n], dtype=np.int64))
    r2 = tc.relax_subdomains(p2, idx=idx, offsets=off, world=world, **kw)
    tc.sync_status()
    # accept = False leaves pos unchanged in subdomain mode: compare energies and RMS
    assert abs(r1.energy[0].item() - r2.energy[0].item()) <= 1e-12 * r1.energy[0].item()
    assert abs(r1.rms[0].item() - r2.rms[0].item()) <= 1e-9 * r1.rms[0].item()


def test_lbfgsb_mixed_with_polish_keeps_the_box():
    """A mixed-precision L-BFGS-B run polished in float64, with the line search: constraints hold
    and the energy drops."""
    n = 400
    pos = synth.arcsine_disk(n, 31)
    p0, f = oracle.border_split(pos, oracle.boundary_count(n), 0.96)
    p = T(p0.copy())
    r = tc.relax_subdomains(p, world=T(np.array([[0, n]], dtype=np.int64)), flags=T(f), precision="mixed",
                            optimizer="lbfgsb_tu", n_steps=150, memory=8, step0=1e-4, maxstep=0.02, radius=0.96,
                            gtol=1e-3, polish_steps=100, accept=False, want_energy=True, line_search=10)
    tc.sync_status()
    x = p.cpu().numpy()
    rr = np.hypot(x[:, 0], x[:, 1])
    assert np.all(np.abs(rr[f == 1] - 1.0) <= 4.5e-16)
    assert np.all(rr[f == 0] <= 0.96 * (1 + 1e-15))
    eg = oracle.energy(x)
    assert eg < oracle.energy(p0)
    assert abs(r.energy[0].item() - eg) <= 1e-12 * eg


def test_lbfgsb_rejects_more_than_eight_pairs():
    pos = T(synth.arcsine_disk(100, 1))
    world = T(np.array([[0, 100]], dtype=np.int64))
    with pytest.raises(tc.TCError):
        tc.relax_subdomains(pos, world=world, precision="fp64", optimizer="lbfgsb_tu", n_steps=2, memory=9,
                            step0=1e-4, maxstep=0.02, accept=False)


def test_lbfgsb_large_instance_matches_oracle():
    """An instance of 17 000 charges (more than the grid-wide L-BFGS path's threshold): one CTA
    steps it, on the same iteration as the oracle."""
    n = 17000
    pos = synth.arcsine_disk(n, 81)
    pos = np.ascontiguousarray(pos[synth.zorder(pos)])
    p = T(pos.copy())
    iters = 4
    r = tc.relax_subdomains(p, world=T(np.array([[0, n]], dtype=np.int64)), precision="fp64",
                            optimizer="lbfgsb_tu", n_steps=iters, memory=4, step0=1e-5, maxstep=0.01, accept=False)
    tc.sync_status()
    xo, _, rms, nb = oracle.lbfgsb(pos, memory=4, max_iter=iters, step0=1e-5, maxstep=0.01)
    assert nb >= 1
    assert np.abs(p.cpu().numpy() - xo).max() <= 1e-9
    assert abs(r.rms[0].item() - rms) <= 1e-6 * rms


def test_lbfgsb_degenerate_instances_match_oracle():
    """Instances of 1, 2 and 5 charges, and one whose charges are all pinned to the circle."""
    sizes = [1, 2, 5, 9]
    pos = np.concatenate([synth.arcsine_disk(m, 70 + m) for m in sizes])
    off = np.concatenate([[0], np.cumsum(sizes)])
    world = np.stack([off[:-1], off[1:]], 1).astype(np.int64)
    flags = np.zeros(len(pos), dtype=np.uint8)
    flags[off[3]:off[4]] = 1
    p0 = pos.copy()
    r0 = np.hypot(p0[:, 0], p0[:, 1])
    p0[flags == 1] /= r0[flags == 1, None]
    p = T(p0.copy())
    iters = 20
    tc.relax_subdomains(p, world=T(world), flags=T(flags), precision="fp64", optimizer="lbfgsb_tu", n_steps=iters,
                        memory=4, step0=1e-3, maxstep=0.05, accept=False)
    tc.sync_status()
    x = p.cpu().numpy()
    for k in range(len(sizes)):
        b, e = off[k], off[k + 1]
        xo, _, _, _ = oracle.lbfgsb(p0[b:e], memory=4, max_iter=iters, step0=1e-3, maxstep=0.05, flags=flags[b:e])
        assert np.abs(x[b:e] - xo).max() <= 1e-9
    rr = np.hypot(x[:, 0], x[:, 1])
    assert np.all(np.abs(rr[flags == 1] - 1.0) <= 4.5e-16)
    # a lone charge feels no force: it moves only by the rounding of x -> (t, u) -> x
    np.testing.assert_allclose(x[0], p0[0], rtol=0, atol=4e-16)
