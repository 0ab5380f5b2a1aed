"""GPU parity: libtc's CUDA kernels against the CPU oracle on the same seeded inputs.

Tolerances (float64 form): energy |dE|/E <= 1e-13; gradient normwise
||dg||/||g|| <= 1e-12 and per component |dg_i| <= 1e-12 G_i with
G_i = sum_j 1/r_ij^2.  Mixed form: gradient relative RMS <= 1e-5.
"""

from __future__ import annotations

import math

import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2609_24722_b300 as tc
from paper_2609_24722_b300 import _lib as L

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a), device=DEV)


def gross_rows(pos, rows=None):
    rows = np.arange(pos.shape[0]) if rows is None else rows
    out = np.empty(len(rows))
    for k, i in enumerate(rows):
        d = pos - pos[i]
        r2 = (d ** 2).sum(1)
        r2[i] = np.inf
        out[k] = (1.0 / r2).sum()
    return out


def check_grad(g, ref, G, tol=1e-12):
    assert np.linalg.norm(g - ref) <= tol * np.linalg.norm(ref)
    assert np.all(np.abs(g - ref) <= tol * G[:, None])


SIZES = [2, 3, 7, 33, 255, 256, 257, 511, 512, 513, 1000, 1537, 2048, 3001]


@pytest.mark.parametrize("n", SIZES)
def test_fp64_energy_grad_local_vs_oracle(n):
    pos = synth.arcsine_disk(n, 100 + n)
    p = T(pos)
    g, e = tc.grad(p, "fp64", with_energy=True)
    e2, loc = tc.local_energy(p, "fp64")
    tc.sync_status()
    eo, loco = oracle.energy(pos, local=True)
    go = oracle.grad(pos)
    assert abs(e.item() - eo) <= 1e-13 * eo
    assert abs(e2.item() - eo) <= 1e-13 * eo
    np.testing.assert_allclose(loc.cpu().numpy(), loco, rtol=1e-13, atol=0)
    check_grad(g.cpu().numpy(), go, gross_rows(pos))


@pytest.mark.parametrize("n", [2, 257, 1000, 3001])
def test_mixed_energy_grad_vs_oracle(n):
    pos = synth.arcsine_disk(n, 200 + n)
    p = T(pos)
    g, e = tc.grad(p, "mixed", with_energy=True)
    tc.sync_status()
    eo = oracle.energy(pos)
    go = oracle.grad(pos)
    gg = g.cpu().numpy()
    assert np.linalg.norm(gg - go) <= 1e-5 * np.linalg.norm(go)
    assert abs(e.item() - eo) <= 1e-6 * eo


def test_mixed_forward_backward_config_20000():
    """N = 20000 arcsine init + 1e-3 jitter: mixed and float64 gradients against the oracle."""
    n = 20000
    pos = synth.jitter_inside(synth.arcsine_disk(n, 1), 1e-3, 11)
    p = T(pos)
    go = oracle.grad(pos)
    eo = oracle.energy(pos)
    gm, em = tc.grad(p, "mixed", with_energy=True)
    gd, ed = tc.grad(p, "fp64", with_energy=True)
    tc.sync_status()
    gm, gd = gm.cpu().numpy(), gd.cpu().numpy()
    assert np.linalg.norm(gm - go) <= 1e-5 * np.linalg.norm(go)
    assert abs(ed.item() - eo) <= 1e-13 * eo
    rows = np.arange(0, n, 97)
    check_grad(gd[rows], go[rows], gross_rows(pos, rows))
    assert np.linalg.norm(gd - go) <= 1e-12 * np.linalg.norm(go)


@pytest.mark.parametrize("n,seed", [(20000, 1), (60000, 2)])
def test_mixed_sorted_input_uses_far_tiles_within_tolerance(n, seed):
    """Charges in Hilbert order: most tiles take the hi-only far path; accuracy must hold."""
    pos = synth.arcsine_disk(n, seed)
    pos = np.ascontiguousarray(pos[synth.zorder(pos)])
    p = T(pos)
    gm, em = tc.grad(p, "mixed", with_energy=True)
    tc.sync_status()
    rows = np.random.default_rng(seed).choice(n, 400, replace=False).astype(np.int32)
    rows = np.concatenate([rows, np.argsort(-np.linalg.norm(pos, axis=1))[:100].astype(np.int32)])
    go, eo_rows = oracle.rows_grad(pos, rows)
    g = gm.cpu().numpy()[rows]
    assert np.linalg.norm(g - go) <= 1e-5 * np.linalg.norm(go)
    _, loc = tc.local_energy(p, "mixed")
    np.testing.assert_allclose(loc.cpu().numpy()[rows], 0.5 * eo_rows, rtol=1e-6)


def test_every_mixed_launch_shape_gives_identical_results():
    """Launch shapes only change the CTA size, register blocking and the number of persistent CTAs,
    never a sum's order: the ranges of units (several per CTA here, taken from a queue) do not depend
    on the shape."""
    lib = L.lib()
    n = 30000
    pos = synth.lattice_disk(n, 3)
    pos = np.ascontiguousarray(pos[synth.zorder(pos)])
    subs = synth.subdomains(pos, 24, 300, 3000, 4)
    idx, off = synth.to_csr(subs)
    eta = 1e-4 / n
    old = lib.tc_get_pass_config(1)
    outs = []
    try:
        for cfg in range(lib.tc_pass_config_count(1)):
            assert lib.tc_set_pass_config(1, cfg) == 0
            p = T(pos)
            g, e = tc.grad(p, "mixed", with_energy=True)
            q = T(pos.copy())
            tc.relax_subdomains(q, T(idx), T(off), precision="mixed", optimizer="bb", n_steps=5, step0=eta,
                                alpha_min=0.0, alpha_max=10 * eta, accept=True)
            tc.sync_status()
            outs.append((g.cpu().numpy(), e.item(), q.cpu().numpy()))
    finally:
        lib.tc_set_pass_config(1, old)
    assert lib.tc_set_pass_config(1, 99) == 1
    for o in outs[1:]:
        np.testing.assert_array_equal(o[0], outs[0][0])
        assert o[1] == outs[0][1]
        np.testing.assert_array_equal(o[2], outs[0][2])
    rows = np.random.default_rng(4).choice(n, 400, replace=False)
    go, _ = oracle.rows_grad(pos, rows)
    assert np.linalg.norm(outs[0][0][rows] - go) <= 1e-5 * np.linalg.norm(go)


@pytest.mark.parametrize("n", [3, 10, 100, 1000])
def test_ngon_on_gpu(n):
    import mpmath as mp
    mp.mp.dps = 30
    ref = float(mp.mpf(n) / 2 * mp.fsum(1 / (2 * mp.sin(mp.pi * k / n)) for k in range(1, n)))
    e = tc.energy(T(synth.ngon(n, 0.1)), "fp64").item()
    tc.sync_status()
    assert abs(e - ref) <= 1e-13 * ref


def test_edge_cases_and_device_errors():
    z = torch.zeros((0, 2), dtype=torch.float64, device=DEV)
    assert tc.energy(z).item() == 0.0
    one = T(np.array([[0.3, -0.2]]))
    assert tc.energy(one).item() == 0.0
    assert torch.all(tc.grad(one) == 0)
    tc.sync_status()
    same = T(np.array([[0.1, 0.2], [0.1, 0.2], [0.5, 0.0]]))
    for prec in ("fp64", "mixed"):
        tc.grad(same, prec)
        with pytest.raises(tc.TCError) as ei:
            tc.sync_status()
        assert ei.value.code == 3
    out = T(np.array([[1.5, 0.0], [0.0, 0.0]]))
    tc.energy(out)
    with pytest.raises(tc.TCError) as ei:
        tc.sync_status()
    assert ei.value.code == 4
    # misaligned position pointer is rejected on the host
    buf = torch.zeros(2 * 10 + 1, dtype=torch.float64, device=DEV)
    mis = buf[1:].view(10, 2)
    e = torch.empty((), dtype=torch.float64, device=DEV)
    assert L.lib().tc_energy(mis.data_ptr(), 10, 0, e.data_ptr(), None, None) == 1


def test_determinism():
    pos = T(synth.arcsine_disk(5000, 3))
    for prec in ("fp64", "mixed"):
        a = tc.grad(pos, prec, with_energy=True)
        b = tc.grad(pos, prec, with_energy=True)
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_project_bitwise_vs_oracle():
    rng = np.random.default_rng(0)
    pts = rng.uniform(-1.4, 1.4, (5000, 2))
    flags = (rng.random(5000) < 0.2).astype(np.uint8)
    for radius, fl in [(1.0, None), (0.97, flags)]:
        p = T(pts.copy())
        tc.project_disk(p, radius, None if fl is None else T(fl))
        np.testing.assert_array_equal(p.cpu().numpy(), oracle.project(pts, radius, fl))


def test_subdomain_delta_energy_vs_oracle():
    n = 3000
    pos = synth.lattice_disk(n, 4)
    subs = synth.subdomains(pos, 6, 20, 300, 5)
    idx, off = synth.to_csr(subs)
    rng = np.random.default_rng(9)
    new = oracle.project(pos[idx] + rng.normal(0, 2e-3, (idx.size, 2)))
    d = tc.subdomain_delta_energy(T(pos), T(idx), T(off), T(new))
    tc.sync_status()
    d = d.cpu().numpy()
    e0 = oracle.energy(pos)
    for s in range(len(subs)):
        ref = oracle.delta_energy(pos, subs[s], new[off[s]:off[s + 1]])
        _, _, esub = oracle.subdomain_grad(pos, subs[s], pos[subs[s]])
        assert abs(d[s] - ref) <= 1e-12 * esub, (s, d[s], ref)
    # at this size the difference of totals is still accurate to ~1e-10 relative of E
    p1 = pos.copy()
    p1[subs[0]] = new[off[0]:off[1]]
    assert abs(d[0] - (oracle.energy(p1) - e0)) <= 1e-10 * e0


def test_gd_instance_matches_oracle_trajectory():
    """Config C1: N = 1000 arcsine init, 500 steps of projected GD with step 1e-4/N; positions and the
    energy every 20 steps follow the oracle (energy to 1e-11 relative)."""
    n = 1000
    pos = synth.arcsine_disk(n, 0)
    eta = 1e-4 / n
    p = T(pos.copy())
    world = T(np.array([[0, n]], dtype=np.int64))
    xo = pos.copy()
    for chunk in range(25):
        r = tc.relax_subdomains(p, world=world, precision="fp64", optimizer="gd", n_steps=20, step0=eta,
                                accept=False)
        tc.sync_status()
        xo, tr = oracle.pgd(xo, eta, 20)
        x = p.cpu().numpy()
        assert np.abs(x - xo).max() <= 1e-12
        e = tc.energy(p).item()
        assert abs(e - tr[-1]) <= 1e-11 * tr[-1]
        assert int(r.steps[0]) == 20 and int(r.status[0]) == 1


@pytest.mark.parametrize("n,m_lo,m_hi", [(2500, 30, 200), (6000, 100, 700)], ids=["n2500", "n6000"])
def test_bb_subdomains_and_sequential_accept_vs_oracle(n, m_lo, m_hi):
    """Float64 BB relaxation of overlapping subdomains and the sequential accept against the oracle.
    At n = 6000 the subdomains (296-610 charges) end in partial row blocks of 20-426 rows, which the
    float64 passes run on fewer whole warps, and each accept pass leaves 26-27 slots per row (one
    range per unit), which are summed over every SM before the accept kernel reads them."""
    pos = synth.lattice_disk(n, 7, 0.05)
    subs = synth.subdomains(pos, 5, m_lo, m_hi, 8)
    idx, off = synth.to_csr(subs)
    eta = 1e-4 / n
    steps = 15
    p = T(pos.copy())
    r = tc.relax_subdomains(p, T(idx), T(off), precision="fp64", optimizer="bb", n_steps=steps, step0=eta,
                            alpha_min=0.0, alpha_max=10 * eta, accept=True, want_energy=True)
    tc.sync_status()
    new = np.concatenate([oracle.subdomain_bb(pos, s, eta, 0.0, 10 * eta, steps) for s in subs])
    po, do, ao = oracle.accept_sequential(pos, idx, off, new)
    st = r.status.cpu().numpy()
    np.testing.assert_array_equal(st, ao)
    d = r.delta_e.cpu().numpy()
    for s in range(len(subs)):
        if ao[s] != 2:
            _, _, esub = oracle.subdomain_grad(pos, subs[s], pos[subs[s]])
            assert abs(d[s] - do[s]) <= 1e-11 * esub
    np.testing.assert_allclose(p.cpu().numpy(), po, rtol=0, atol=1e-11)
    es = r.energy.cpu().numpy()
    for s in range(len(subs)):
        _, _, eref = oracle.subdomain_grad(pos, subs[s], new[off[s]:off[s + 1]])
        assert abs(es[s] - eref) <= 1e-12 * eref


def test_lbfgs_instances_fp64_match_oracle():
    sizes = [60, 150, 333]
    pos = np.concatenate([synth.arcsine_disk(m, 40 + m) for m in sizes])
    world = np.array([[0, 60], [60, 210], [210, 543]], dtype=np.int64)
    p = T(pos.copy())
    iters = 25
    r = tc.relax_subdomains(p, world=T(world), precision="fp64", optimizer="lbfgs", n_steps=iters, memory=8,
                            step0=1e-4, maxstep=0.02, accept=False, want_energy=True)
    tc.sync_status()
    x = p.cpu().numpy()
    for k, (b, e) in enumerate(world):
        xo, it, rms = oracle.lbfgs(pos[b:e], memory=8, max_iter=iters, gtol=0.0, step0=1e-4, maxstep=0.02)
        assert np.abs(x[b:e] - xo).max() <= 1e-9
        assert abs(r.energy[k].item() - oracle.energy(xo)) <= 1e-12 * oracle.energy(xo)


def test_lbfgs_instances_across_row_blocks_match_oracle():
    """Instances that straddle the 512-row blocks take their float64 passes with each unordered pair
    once (row blocks against their later tiles, source sums rotated along the lanes): the L-BFGS
    iterates and the float64 energies must still follow the oracle."""
    sizes = [511, 512, 513, 1100, 1600]
    pos = np.concatenate([synth.arcsine_disk(m, 300 + m) for m in sizes])
    off = np.concatenate([[0], np.cumsum(sizes)])
    world = np.stack([off[:-1], off[1:]], 1).astype(np.int64)
    p = T(pos.copy())
    iters = 8
    r = tc.relax_subdomains(p, world=T(world), precision="fp64", optimizer="lbfgs", n_steps=iters, memory=8,
                            step0=1e-5, maxstep=0.01, accept=False, want_energy=True)
    tc.sync_status()
    x = p.cpu().numpy()
    for k in range(len(sizes)):
        b, e = off[k], off[k + 1]
        xo, it, rms = oracle.lbfgs(pos[b:e], memory=8, max_iter=iters, gtol=0.0, step0=1e-5, maxstep=0.01)
        assert np.abs(x[b:e] - xo).max() <= 1e-9
        assert abs(r.energy[k].item() - oracle.energy(xo)) <= 1e-12 * oracle.energy(xo)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_queued_passes_are_deterministic(prec):
    """The mixed and the symmetric float64 passes take their unit ranges from a queue, so which CTA
    computes which range changes from run to run; the sums do not."""
    n = 30000
    pos = synth.arcsine_disk(n, 8)
    pos = np.ascontiguousarray(pos[synth.zorder(pos)])
    p = T(pos)
    runs = []
    for _ in range(3):
        g, e = tc.grad(p, prec, with_energy=True)
        _, loc = tc.local_energy(p, prec)
        tc.sync_status()
        runs.append((g.cpu().numpy(), e.item(), loc.cpu().numpy()))
    for g, e, loc in runs[1:]:
        np.testing.assert_array_equal(g, runs[0][0])
        assert e == runs[0][1]
        np.testing.assert_array_equal(loc, runs[0][2])


def test_lbfgs_many_instances_queued_update_matches_oracle():
    """More instances than resident update CTAs: persistent CTAs take the instances, largest first,
    from a queue.  Every instance must still take every step and follow the oracle's iteration."""
    rng = np.random.default_rng(5)
    sizes = rng.integers(8, 81, 700)
    parts = [synth.arcsine_disk(int(m), 1000 + k) for k, m in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)])
    world = np.stack([off[:-1], off[1:]], 1).astype(np.int64)
    pos = np.concatenate(parts)
    iters = 12
    for rep in range(2):  # the second call reuses the queue counter the first left at zero
        p = T(pos.copy())
        r = tc.relax_subdomains(p, world=T(world), precision="fp64", optimizer="lbfgs", n_steps=iters, memory=8,
                                step0=1e-4, maxstep=0.02, accept=False, want_energy=True)
        tc.sync_status()
        assert (r.steps.cpu().numpy() == iters).all()
        x = p.cpu().numpy()
        for k in sorted({0, 699, int(np.argmax(sizes)), int(np.argmin(sizes)), 350}):
            b, e = off[k], off[k + 1]
            xo, it, rms = oracle.lbfgs(pos[b:e], memory=8, max_iter=iters, gtol=0.0, step0=1e-4, maxstep=0.02)
            assert np.abs(x[b:e] - xo).max() <= 1e-9
            assert abs(r.energy[k].item() - oracle.energy(xo)) <= 1e-12 * oracle.energy(xo)


def test_lbfgs_large_instance_grid_update_matches_oracle():
    """An instance above 16384 charges takes the grid-wide L-BFGS update; it must follow the oracle."""
    n = 17000
    pos = synth.arcsine_disk(n, 77)
    pos = np.ascontiguousarray(pos[synth.zorder(pos)])
    p = T(pos.copy())
    world = T(np.array([[0, n]], dtype=np.int64))
    iters = 3
    r = tc.relax_subdomains(p, world=world, precision="fp64", optimizer="lbfgs", n_steps=iters, memory=8,
                            step0=1e-6, maxstep=0.002, accept=False)
    tc.sync_status()
    xo, it, rms = oracle.lbfgs(pos, memory=8, max_iter=iters, gtol=0.0, step0=1e-6, maxstep=0.002)
    assert int(r.steps[0]) == iters
    assert np.abs(p.cpu().numpy() - xo).max() <= 1e-9
    assert abs(r.rms[0].item() - rms) <= 1e-6 * rms


def test_lbfgs_mixed_then_fp64_polish_converges():
    """Mixed bulk steps then float64 polish end at a float64-stationary configuration.

    The 60-charge instance needs about 530 float64 L-BFGS iterations from its start to reach
    RMS 1e-11 in the oracle, so the polish cap leaves room for that."""
    sizes = [5, 8, 60]
    pos = np.concatenate([synth.arcsine_disk(m, 7 + m) for m in sizes])
    world = np.array([[0, 5], [5, 13], [13, 73]], dtype=np.int64)
    p = T(pos.copy())
    r = tc.relax_subdomains(p, world=T(world), precision="mixed", optimizer="lbfgs", n_steps=300, memory=8,
                            step0=1e-3, maxstep=0.05, gtol=1e-4, polish_steps=800, polish_gtol=1e-11,
                            accept=False, want_energy=True)
    tc.sync_status()
    assert np.all(r.rms.cpu().numpy() < 1e-11)
    x = p.cpu().numpy()
    for k, (b, e) in enumerate(world):
        xo = x[b:e]
        eo = oracle.energy(xo)
        assert abs(r.energy[k].item() - eo) <= 1e-13 * eo
        assert eo < oracle.energy(pos[b:e])
        # stationary by the oracle's own float64 gradient: tangential force on wall
        # charges and the full force inside vanish to rounding
        _, rms_c, mx = oracle.projected_grad(xo, oracle.grad(xo))
        assert mx <= 1e-8 * np.abs(oracle.grad(xo)).max()
    # the smallest instance ends on the ring, its lowest state
    ring = oracle.energy(synth.ngon(5))
    assert abs(oracle.energy(x[0:5]) - ring) <= 1e-12 * ring


def test_mixed_subdomain_relaxation_lowers_energy():
    n = 20000
    pos = synth.lattice_disk(n, 3)
    subs = synth.subdomains(pos, 12, 200, 800, 2)
    idx, off = synth.to_csr(subs)
    p = T(pos.copy())
    eta = 1e-4 / n
    r = tc.relax_subdomains(p, T(idx), T(off), precision="mixed", optimizer="bb", n_steps=50, step0=eta,
                            alpha_min=0.0, alpha_max=10 * eta, accept=True)
    tc.sync_status()
    st = r.status.cpu().numpy()
    d = r.delta_e.cpu().numpy()
    assert np.all(d[st == 1] < 0) and np.all(d[st == 0] >= 0)
    assert (st == 1).sum() >= 1
    x = p.cpu().numpy()
    e0, e1 = oracle.energy(pos), oracle.energy(x)
    assert abs((e1 - e0) - d[st == 1].sum()) <= 1e-11 * e0
    # every accepted move is exactly the recorded float64 change: check one against the oracle
    s = int(np.flatnonzero(st == 1)[0])
    # (the accepted subdomain's new positions are in x)
    assert oracle.delta_energy(pos, subs[s], x[subs[s]]) < 0


def test_profiled_relaxation_with_accept():
    """profile=True records launch timings; results match the unprofiled call bit for bit."""
    n = 6000
    pos = synth.lattice_disk(n, 5)
    subs = synth.subdomains(pos, 8, 100, 600, 6)
    idx, off = synth.to_csr(subs)
    eta = 1e-4 / n
    outs = []
    for prof in (False, True):
        p = T(pos.copy())
        r = tc.relax_subdomains(p, T(idx), T(off), precision="mixed", optimizer="bb", n_steps=12, step0=eta,
                                alpha_min=0.0, alpha_max=10 * eta, accept=True, profile=prof)
        tc.sync_status()
        outs.append((p.cpu().numpy(), r.delta_e.cpu().numpy(), r.status.cpu().numpy()))
    for a, b in zip(outs[0], outs[1]):
        np.testing.assert_array_equal(a, b)
    pr = tc.relax_last_profile()
    assert pr["n_pass"] == 12 and pr["pass_ms"] > 0 and pr["accept_ms"] > 0
    assert pr["pass_pairs"] == sum(len(s) * (n - 1) for s in subs)
    assert pr["launches"] >= 2 * 12 + 2 * len(subs)


def test_autograd_function_and_gradcheck():
    pos = synth.arcsine_disk(64, 5) * 0.9
    p = T(pos).requires_grad_(True)
    e = tc.coulomb_energy(p, "fp64")
    e.backward()
    np.testing.assert_allclose(p.grad.cpu().numpy(), oracle.grad(pos), rtol=1e-12, atol=1e-12)
    assert abs(e.item() - oracle.energy(pos)) <= 1e-13 * e.item()
    q = T(pos).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x: tc.coulomb_energy(x, "fp64"), (q,), eps=1e-6, atol=1e-5, rtol=1e-6)


def test_sampled_rows_at_full_size():
    """N = 100 000: sampled gradient rows of the launch the benchmark times, against the oracle."""
    n = 100000
    pos = synth.arcsine_disk(n, 0)
    p = T(pos)
    rows = np.random.default_rng(0).choice(n, 24, replace=False).astype(np.int32)
    go, eo_rows = oracle.rows_grad(pos, rows)
    gm = tc.grad(p, "mixed").cpu().numpy()[rows]
    gd, ed = tc.grad(p, "fp64", with_energy=True)
    _, loc = tc.local_energy(p, "fp64")
    tc.sync_status()
    gd = gd.cpu().numpy()[rows]
    assert np.linalg.norm(gm - go) <= 1e-5 * np.linalg.norm(go)
    check_grad(gd, go, gross_rows(pos, rows))
    np.testing.assert_allclose(loc.cpu().numpy()[rows], 0.5 * eo_rows, rtol=1e-13)
    # Euler's identity for the degree -1 energy holds for the full float64 result
    gfull = tc.grad(p, "fp64").cpu().numpy()
    assert abs((pos * gfull).sum() + ed.item()) <= 1e-11 * ed.item()


@pytest.mark.parametrize("n", [2000, 17000])
def test_lbfgs_tolerance_stop_then_polish_equals_one_run(n):
    """A float64 L-BFGS phase that stops on its tolerance, then a float64 polish that keeps the
    history, takes the same steps as one uninterrupted run of as many steps (the converged point's
    gradient is recomputed, its pair fails the curvature test, and the direction is the same).
    n = 17000 takes the grid-wide update of large problems."""
    pos = synth.arcsine_disk(n, 91)
    pos = np.ascontiguousarray(pos[synth.zorder(pos)])
    world = T(np.array([[0, n]], dtype=np.int64))
    kw = dict(precision="fp64", optimizer="lbfgs", memory=8, step0=1e-5, maxstep=0.01, accept=False)
    p = T(pos.copy())
    r = tc.relax_subdomains(p, world=world, n_steps=30, **kw)
    tc.sync_status()
    gtol = 1.0001 * r.rms[0].item()
    pa = T(pos.copy())
    ra = tc.relax_subdomains(pa, world=world, n_steps=300, gtol=gtol, polish_steps=12, polish_gtol=0.0, **kw)
    tc.sync_status()
    k = int(ra.steps[0])
    assert 12 < k <= 30 + 12  # the first phase stopped on its tolerance
    pb = T(pos.copy())
    tc.relax_subdomains(pb, world=world, n_steps=k, **kw)
    tc.sync_status()
    np.testing.assert_array_equal(pa.cpu().numpy(), pb.cpu().numpy())


def test_repeated_calls_reuse_the_step_graph_with_new_arguments():
    """The executable step-loop graph is kept across calls and updated in place for a call of the
    same shape: a call on configuration A, then B, then A again (and a call of another shape in
    between) gives A's result bit for bit, equal to the directly launched (profiled) loop."""
    n = 5000
    kw = dict(world=T(np.array([[0, 2000], [2000, n]], dtype=np.int64)), precision="mixed", optimizer="lbfgs",
              n_steps=70, memory=8, step0=1e-5, maxstep=0.01, accept=False)
    a = synth.arcsine_disk(n, 61)
    b = synth.arcsine_disk(n, 62)
    outs = []
    for pos, extra in ((a, {}), (b, {}), (synth.arcsine_disk(3000, 63), {"world": T(np.array([[0, 3000]]))}),
                       (a, {}), (a, {"profile": True})):
        p = T(pos.copy())
        tc.relax_subdomains(p, **{**kw, **extra})
        tc.sync_status()
        outs.append(p.cpu().numpy())
    np.testing.assert_array_equal(outs[3], outs[0])
    np.testing.assert_array_equal(outs[4], outs[0])
    assert not np.array_equal(outs[1], outs[0])
