"""GPU parity of the subdomain gradient (Sec. II D objective) against the oracle, row by row.

tc_subdomain_grad runs the pair pass that every relaxation step runs (rows of the active set A
against the snapshot with A masked out, plus A's own rows at their moved positions), once, in
the launch configuration of the relaxation.  Each sampled subdomain's rows are compared with
oracle.subdomain_grad of the same snapshot and active positions:
  float64 and fp64x: gradient normwise ||dg||/||g|| <= 1e-12 and per component |dg_k| <= 1e-12 G_k
    (G_k = sum_j 1/r_kj^2 over every other charge), e_k and E_sub to 1e-13 relative;
  mixed (float32 pair terms): gradient relative RMS <= 1e-5 per subdomain, e_k to 1e-6.
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


def gross(pos, idx, act):
    """G_k = sum over every other charge of 1/r^2, with A's charges at act."""
    cur = pos.copy()
    cur[idx] = act
    out = np.empty(len(idx))
    for k, i in enumerate(idx):
        d = cur - cur[i]
        r2 = (d ** 2).sum(1)
        r2[i] = np.inf
        out[k] = (1.0 / r2).sum()
    return out


def moved(pos, idx, scale, seed):
    """Active positions a small random move away from the snapshot, inside the disk."""
    rng = np.random.default_rng(seed)
    return oracle.project(pos[idx] + rng.normal(0.0, scale, (len(idx), 2)))


def check_rows(prec, g, e, es, go, eo, eso, G):
    if prec == "mixed":
        assert np.linalg.norm(g - go) <= 1e-5 * np.linalg.norm(go)
        np.testing.assert_allclose(e, eo, rtol=1e-6, atol=0)
        assert abs(es - eso) <= 1e-6 * eso
    else:
        assert np.linalg.norm(g - go) <= 1e-12 * np.linalg.norm(go)
        assert np.all(np.abs(g - go) <= 1e-12 * G[:, None])
        np.testing.assert_allclose(e, eo, rtol=1e-13, atol=0)
        assert abs(es - eso) <= 1e-13 * eso


def run_all(pos, idx, off, act, prec):
    g, e, es = tc.subdomain_grad(T(pos), T(idx), T(off), None if act is None else T(act), prec)
    tc.sync_status()
    return g.cpu().numpy(), e.cpu().numpy(), es.cpu().numpy()


@pytest.fixture(scope="module")
def c3():
    """The timed workload's shape: N = 1e5 lattice background in Hilbert order, 256 subdomains of
    m ~ U{200..5000} nearest charges, active charges moved by ~1e-4 (the masked snapshot and the
    own rows then differ).  Sampled: the smallest subdomain (one partial row block), the largest,
    the one reaching furthest out (wall charges), and one whose last row block is under half full.
    The oracle's rows of the sampled subdomains are computed once for all precisions."""
    n = 100_000
    pos = synth.lattice_disk(n, 0)
    pos = np.ascontiguousarray(pos[synth.zorder(pos)])
    subs = synth.subdomains(pos, 256, 200, 5000, 2)
    idx, off = synth.to_csr(subs)
    act = moved(pos, idx, 1e-4, 5)
    sizes = np.diff(off)
    radii = np.array([np.linalg.norm(pos[s], axis=1).max() for s in subs])
    pick = [int(np.argmin(sizes)), int(np.argmax(sizes)), int(np.argmax(radii))]
    pick.append(next(s for s in range(len(subs)) if 256 < sizes[s] and sizes[s] % 512 < 256 and s not in pick))
    ref = {}
    for s in pick:
        a, b = off[s], off[s + 1]
        go, eo, eso = oracle.subdomain_grad(pos, subs[s], act[a:b])
        ref[s] = (go, eo, eso, gross(pos, subs[s], act[a:b]))
    return pos, idx, off, act, pick, ref


@pytest.mark.parametrize("prec", ["mixed", "fp64", "fp64x"])
def test_c3_shape_sampled_subdomains_vs_oracle(c3, prec):
    pos, idx, off, act, pick, ref = c3
    g, e, es = run_all(pos, idx, off, act, prec)
    assert np.diff(off)[pick[0]] < 512  # the smallest subdomain is one partial row block
    for s in pick:
        a, b = off[s], off[s + 1]
        go, eo, eso, G = ref[s]
        check_rows(prec, g[a:b], e[a:b], es[s], go, eo, eso, G)


@pytest.mark.parametrize("prec", ["mixed", "fp64", "fp64x"])
def test_unordered_arcsine_input_all_rows_vs_oracle(prec):
    """Arcsine random charges in generation order: every tile of a subdomain's rows is a near tile."""
    n = 20000
    pos = synth.jitter_inside(synth.arcsine_disk(n, 1), 1e-3, 11)
    subs = synth.subdomains(pos, 8, 100, 1500, 3)
    idx, off = synth.to_csr(subs)
    act = moved(pos, idx, 2e-4, 6)
    g, e, es = run_all(pos, idx, off, act, prec)
    for s in range(len(subs)):
        a, b = off[s], off[s + 1]
        go, eo, eso = oracle.subdomain_grad(pos, subs[s], act[a:b])
        G = gross(pos, subs[s], act[a:b]) if prec != "mixed" else None
        check_rows(prec, g[a:b], e[a:b], es[s], go, eo, eso, G)


@pytest.mark.parametrize("prec", ["mixed", "fp64", "fp64x"])
def test_ragged_and_degenerate_subdomains(prec):
    """Sizes around the 512-row block and 256-source tile (255, 256, 257, 511, 512, 513), one charge,
    an empty subdomain, and a subdomain of every charge (no fixed charges at all)."""
    n = 3001
    pos = synth.arcsine_disk(n, 21)
    rng = np.random.default_rng(4)
    sizes = [255, 256, 257, 511, 512, 513, 1, 0, n]
    subs = [np.sort(rng.choice(n, m, replace=False)).astype(np.int32) for m in sizes]
    idx, off = synth.to_csr(subs)
    act = moved(pos, idx, 3e-4, 7)
    g, e, es = run_all(pos, idx, off, act, prec)
    for s, m in enumerate(sizes):
        a, b = off[s], off[s + 1]
        if m == 0:
            assert es[s] == 0.0
            continue
        go, eo, eso = oracle.subdomain_grad(pos, subs[s], act[a:b])
        G = gross(pos, subs[s], act[a:b]) if prec != "mixed" else None
        check_rows(prec, g[a:b], e[a:b], es[s], go, eo, eso, G)
    # the whole configuration as one subdomain is the all-pairs gradient of the moved charges
    whole = pos.copy()
    whole[subs[-1]] = act[off[-2]:]
    gall, eall = tc.grad(T(whole), prec, with_energy=True)
    tc.sync_status()
    tol = 1e-5 if prec == "mixed" else 1e-12
    ga = gall.cpu().numpy()
    assert np.linalg.norm(g[off[-2]:] - ga) <= tol * np.linalg.norm(ga)


def test_default_act_is_the_snapshot_and_drives_the_relaxation_step():
    """act = NULL evaluates at the snapshot; and one projected GD step of tc_relax_subdomains (the
    same pass, launched by the relaxation) moves each interior charge of an accepted subdomain by
    -step0 times the gradient this call returns."""
    n = 9000
    pos = synth.lattice_disk(n, 3)
    pos = np.ascontiguousarray(pos[synth.zorder(pos)])
    subs, seen = [], set()
    for s in synth.subdomains(pos, 12, 100, 900, 4):
        if not seen.intersection(s.tolist()):
            subs.append(s)
            seen.update(s.tolist())
    idx, off = synth.to_csr(subs)
    g0, _, _ = run_all(pos, idx, off, None, "mixed")
    g1, _, _ = run_all(pos, idx, off, pos[idx], "mixed")
    np.testing.assert_array_equal(g0, g1)
    go = np.concatenate([oracle.subdomain_grad(pos, s, pos[s])[0] for s in subs])
    assert np.linalg.norm(g0 - go) <= 1e-5 * np.linalg.norm(go)
    eta = 1e-4 / n
    p = T(pos.copy())
    r = tc.relax_subdomains(p, T(idx), T(off), precision="mixed", optimizer="gd", n_steps=1, step0=eta,
                            accept=True)
    tc.sync_status()
    st = r.status.cpu().numpy()
    assert np.all(st == 1)  # disjoint subdomains, one small downhill step each
    x1 = p.cpu().numpy()[idx]
    inner = np.linalg.norm(x1, axis=1) < 0.999
    rec = (pos[idx][inner] - x1[inner]) / eta
    assert np.linalg.norm(rec - g0[inner]) <= 1e-9 * np.linalg.norm(g0[inner])


def test_subdomain_energy_gradcheck_config_20000():
    """E_sub of a 64-charge subset of the N = 20000 jittered arcsine input through the autograd
    Function: backward equals the oracle's gradient, and torch.autograd.gradcheck (central
    differences, eps = 1e-6) passes.  Rounding in E_sub (~2e6) limits the difference quotient to
    about 1e-16 * 2e6 / 1e-6 = 2e-4 plus the pass's own summation error, hence atol = 1e-2 on
    gradient entries of size ~1e5."""
    n = 20000
    pos = synth.jitter_inside(synth.arcsine_disk(n, 1), 1e-3, 11)
    sub = synth.subdomains(pos, 1, 64, 64, 9)[0]
    p, ix = T(pos), T(sub)
    act = T(pos[sub]).requires_grad_(True)
    es = tc.subdomain_energy(act, p, ix, "fp64")
    es.backward()
    go, _, eso = oracle.subdomain_grad(pos, sub, pos[sub])
    assert abs(es.item() - eso) <= 1e-13 * eso
    ga = act.grad.cpu().numpy()
    assert np.linalg.norm(ga - go) <= 1e-12 * np.linalg.norm(go)
    q = T(pos[sub]).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda a: tc.subdomain_energy(a, p, ix, "fp64"), (q,), eps=1e-6, atol=1e-2,
                                    rtol=1e-6)
    # the mixed forward/backward of the same subset, against the oracle
    am = T(pos[sub]).requires_grad_(True)
    em = tc.subdomain_energy(am, p, ix, "mixed")
    em.backward()
    assert abs(em.item() - eso) <= 1e-6 * eso
    assert np.linalg.norm(am.grad.cpu().numpy() - go) <= 1e-5 * np.linalg.norm(go)


def test_coulomb_energy_mixed_forward_backward_config_20000():
    """The whole-configuration autograd Function in the mixed form at N = 20000 (jittered arcsine):
    E to 1e-6 and dE/dr to relative RMS 1e-5 against the oracle; float64 to 1e-13 / 1e-12."""
    n = 20000
    pos = synth.jitter_inside(synth.arcsine_disk(n, 1), 1e-3, 11)
    go, eo = oracle.grad(pos), oracle.energy(pos)
    for prec, te, tg in (("mixed", 1e-6, 1e-5), ("fp64", 1e-13, 1e-12)):
        p = T(pos).requires_grad_(True)
        e = tc.coulomb_energy(p, prec)
        (2.0 * e).backward()
        tc.sync_status()
        assert abs(e.item() - eo) <= te * eo
        g = p.grad.cpu().numpy() / 2.0
        assert np.linalg.norm(g - go) <= tg * np.linalg.norm(go)
