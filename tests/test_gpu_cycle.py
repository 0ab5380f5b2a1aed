"""GPU parity of the adaptive cycle (Sec. II C): defect statistics, centres, nearest-m zones and
the batched cycle driver against the CPU oracle on the same seeded inputs.

Zones are integer results: they must match the oracle exactly.  The only floating-point inputs to
those decisions that the two sides may round differently are mu and sigma_e (summation order) and
the trigonometric centre (CUDA's and the host's sin/cos may differ in the last place); each test
first checks on the oracle's side that no decision lies within that rounding of its threshold,
so an exact comparison is meaningful.
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


def margin_ok(pos, e, u, off, idx, cen, st, kappa, wall_tol=1e-9):
    """No defect decision within 1e-12 of the threshold, no zone boundary within 1e-12 relative."""
    thr = st[0] + kappa * st[1]
    if np.any(np.abs(e - thr) <= 1e-12 * abs(thr)):
        return False
    for s in range(len(off) - 1):
        z = idx[off[s]:off[s + 1]]
        if 0 < len(z) < len(pos):
            d2 = ((pos - cen[s]) ** 2).sum(1)
            inside, outside = d2[z].max(), np.delete(d2, z).min()
            if outside - inside <= 1e-12 * max(outside, 1e-300) and outside != inside:
                return False
    return True


def select_both(pos, e, u, **kw):
    idx_o, off_o, cen_o, st_o = oracle.zone_select(pos, e, u, **kw)
    idx, off, cen, st = tc.select_subdomains(T(pos), T(e), T(u), **kw)
    torch.cuda.synchronize()
    return (idx_o, off_o, cen_o, st_o), (idx.cpu().numpy(), off.cpu().numpy(), cen.cpu().numpy(), st.cpu().numpy())


@pytest.mark.parametrize("n,seed", [(700, 1), (2000, 2), (5003, 3)])
def test_select_matches_oracle(n, seed):
    pos = synth.lattice_disk(n, seed, 0.05)
    _, e = oracle.energy(pos, local=True)
    u = np.random.default_rng(seed).random((37, 3))
    kw = dict(m_min=17, m_max=min(n - 1, 900), period=9, phase=4)
    (io, oo, co, so), (ig, og, cg, sg) = select_both(pos, e, u, **kw)
    assert margin_ok(pos, e, u, oo, io, co, so, -1.0)
    np.testing.assert_array_equal(og, oo)
    np.testing.assert_array_equal(ig, io)
    assert sg[2] == so[2]
    assert abs(sg[0] - so[0]) <= 1e-15 * so[0] and abs(sg[1] - so[1]) <= 1e-12 * so[1]
    np.testing.assert_allclose(cg, co, rtol=0, atol=4e-16)


def test_select_edge_cases():
    """m = 0, m >= n, one charge, exact ties broken by index, all-defect and no-defect draws."""
    g = np.arange(-6, 7) / 8.0
    grid = np.array([(x, y) for x in g for y in g if x * x + y * y <= 0.75])
    grid = grid[np.random.default_rng(2).permutation(len(grid))]
    n = len(grid)
    e = np.zeros(n)
    u = np.array([[0.5, 0.0, 0.3], [0.2, 0.0, 0.9]])
    for m in [0, 1, 5, 6, 9, 13, 20, 21, n - 1, n, n + 5]:
        (io, oo, co, so), (ig, og, cg, sg) = select_both(grid, e, u, m_min=m, m_max=m, period=1, kappa=1.0)
        np.testing.assert_array_equal(og, oo)
        np.testing.assert_array_equal(ig, io)
    # a single charge
    one = np.array([[0.1, -0.2]])
    (io, oo, _, _), (ig, og, _, _) = select_both(one, np.array([0.0]), u, m_min=0, m_max=3, period=2)
    np.testing.assert_array_equal(og, oo)
    np.testing.assert_array_equal(ig, io)
    # every centre a defect charge, then none
    pos = synth.arcsine_disk(900, 4)
    _, e = oracle.energy(pos, local=True)
    uu = np.random.default_rng(9).random((25, 3))
    for pd in [1.0, 0.0]:
        (io, oo, co, so), (ig, og, cg, sg) = select_both(pos, e, uu, m_min=10, m_max=200, period=5, p_defect=pd)
        np.testing.assert_array_equal(ig, io)
        np.testing.assert_allclose(cg, co, rtol=0, atol=4e-16)
    # zero subdomains
    idx, off, cen, st = tc.select_subdomains(T(pos), T(e), torch.zeros((0, 3), dtype=torch.float64, device=DEV),
                                             m_min=1, m_max=2, period=1)
    assert off.cpu().tolist() == [0]


def test_select_at_full_size_sampled():
    """N = 100 000 lattice background, 64 zones of 200..5000: the zones equal the oracle's."""
    n = 100_000
    pos = synth.lattice_disk(n, 0)
    pos = np.ascontiguousarray(pos[synth.zorder(pos)])
    p = T(pos)
    _, e = tc.local_energy(p, "fp64")
    e_np = e.cpu().numpy()
    u = np.random.default_rng(12).random((64, 3))
    kw = dict(m_min=200, m_max=5000, period=16, phase=0)
    idx, off, cen, st = tc.select_subdomains(p, e, T(u), **kw)
    torch.cuda.synchronize()
    io, oo, co, so = oracle.zone_select(pos, e_np, u, **kw)
    assert margin_ok(pos, e_np, u, oo, io, co, so, -1.0)
    np.testing.assert_array_equal(off.cpu().numpy(), oo)
    np.testing.assert_array_equal(idx.cpu().numpy(), io)


@pytest.mark.parametrize("batch", [1, 3, 8])
def test_cycle_fp64_matches_oracle(batch):
    """float64 local energies and float64 BB relaxation: the cycle follows the oracle's cycle."""
    n = 1500
    pos = synth.lattice_disk(n, 21, 0.05)
    u = np.random.default_rng(22).random((8, 3))
    eta = 1e-4 / n
    kw = dict(m_min=20, m_max=200, period=4)
    po, trace_o, do, ao = oracle.cycle(pos, u, batch=batch, step0=eta, alpha_min=0.0, alpha_max=10 * eta, steps=10,
                                       **kw)
    p = T(pos.copy())
    r, trace = tc.cycle(p, T(u), batch=batch, local_precision="fp64", precision="fp64", optimizer="bb", n_steps=10,
                        step0=eta, alpha_min=0.0, alpha_max=10 * eta, **kw)
    tc.sync_status()
    np.testing.assert_array_equal(r.status.cpu().numpy(), ao)
    np.testing.assert_allclose(p.cpu().numpy(), po, rtol=0, atol=1e-11)
    np.testing.assert_allclose(trace.cpu().numpy(), trace_o, rtol=1e-13)
    d = r.delta_e.cpu().numpy()
    m = ao != 2
    np.testing.assert_allclose(d[m], do[m], rtol=1e-9, atol=1e-9)


def test_cycle_mixed_lowers_energy_and_books_it():
    """Mixed local energies and mixed relaxation at N = 20 000: every batch lowers E by its accepted dE."""
    n = 20_000
    pos = synth.lattice_disk(n, 5)
    pos = np.ascontiguousarray(pos[synth.zorder(pos)])
    p = T(pos.copy())
    u = np.random.default_rng(31).random((24, 3))
    eta = 1e-4 / n
    r, trace = tc.cycle(p, T(u), batch=8, m_min=100, m_max=1500, period=12, local_precision="fp64",
                        precision="mixed", optimizer="bb", n_steps=40, step0=eta, alpha_min=0.0, alpha_max=10 * eta)
    tc.sync_status()
    tr = trace.cpu().numpy()
    st = r.status.cpu().numpy()
    d = r.delta_e.cpu().numpy()
    assert np.all(np.diff(tr) <= 0) and (st == 1).sum() >= 1
    for b in range(3):
        sl = slice(8 * b, 8 * b + 8)
        assert abs((tr[b + 1] - tr[b]) - d[sl][st[sl] == 1].sum()) <= 1e-12 * tr[b]
    assert abs(tr[-1] - oracle.energy(p.cpu().numpy())) <= 1e-13 * tr[-1]


# ------------------------------------------------ border-interior split (Sec. II B) ---

@pytest.mark.parametrize("n,seed", [(1, 0), (7, 1), (2000, 2), (100_000, 3)])
def test_border_split_matches_oracle(n, seed):
    pos = synth.arcsine_disk(n, seed)
    nb = oracle.boundary_count(n)
    sigma = 1 - 1 / (2 * np.sqrt(n))
    po, fo = oracle.border_split(pos, nb, sigma)
    p = T(pos.copy())
    f = tc.border_split(p, nb, sigma)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(f.cpu().numpy(), fo)
    np.testing.assert_array_equal(p.cpu().numpy(), po)


def test_border_split_defaults_and_ties():
    g = np.array([[1, 0], [0, 1], [-1, 0], [0, -1], [0.5, 0], [0, 0.25]], dtype=float) * 0.75
    po, fo = oracle.border_split(g, 2, 0.9)
    p = T(g.copy())
    f = tc.border_split(p, 2, 0.9)
    torch.cuda.synchronize()
    assert f.cpu().tolist() == fo.tolist() == [0, 0, 1, 1, 0, 0]
    np.testing.assert_array_equal(p.cpu().numpy(), po)
    pos = synth.arcsine_disk(5000, 6)
    p = T(pos.copy())
    f = tc.border_split(p)
    torch.cuda.synchronize()
    assert int(f.sum()) == oracle.boundary_count(5000)
    for nb in [0, 5000]:
        q = T(pos.copy())
        assert int(tc.border_split(q, nb, 0.99).sum()) == nb


def test_select_with_flags_matches_oracle():
    n = 3000
    pos = synth.arcsine_disk(n, 15)
    _, f = oracle.border_split(pos, oracle.boundary_count(n), 1.0)  # flags only; positions as drawn
    _, e = oracle.energy(pos, local=True)
    u = np.random.default_rng(16).random((30, 3))
    kw = dict(m_min=10, m_max=400, period=7, p_defect=0.9)
    io, oo, co, so = oracle.zone_select(pos, e, u, flags=f, **kw)
    idx, off, cen, st = tc.select_subdomains(T(pos), T(e), T(u), flags=T(f), **kw)
    torch.cuda.synchronize()
    assert margin_ok(pos, e, u, oo, io, co, so, -1.0)
    assert st.cpu().numpy()[2] == so[2]
    np.testing.assert_array_equal(off.cpu().numpy(), oo)
    np.testing.assert_array_equal(idx.cpu().numpy(), io)


@pytest.mark.parametrize("batch", [2, 5])
def test_cycle_pinned_sigma_ramp_fp64_matches_oracle(batch):
    n = 1500
    pos = synth.arcsine_disk(n, 13)
    s0 = 1 - 1 / (2 * np.sqrt(n))
    p0, f = oracle.border_split(pos, oracle.boundary_count(n), s0)
    u = np.random.default_rng(14).random((10, 3))
    eta = 1e-4 / n
    kw = dict(m_min=20, m_max=150, period=4)
    po, trace_o, do, ao = oracle.cycle(p0, u, batch=batch, step0=eta, alpha_min=0.0, alpha_max=10 * eta, steps=8,
                                       sigma0=s0, sigma1=1.0, flags=f, **kw)
    p = T(p0.copy())
    r, trace = tc.cycle(p, T(u), T(f), batch=batch, local_precision="fp64", precision="fp64", optimizer="bb",
                        n_steps=8, step0=eta, alpha_min=0.0, alpha_max=10 * eta, sigma0=s0, sigma1=1.0, **kw)
    tc.sync_status()
    np.testing.assert_array_equal(r.status.cpu().numpy(), ao)
    np.testing.assert_allclose(p.cpu().numpy(), po, rtol=0, atol=1e-11)
    np.testing.assert_allclose(trace.cpu().numpy(), trace_o, rtol=1e-13)
    x = p.cpu().numpy()
    rr = np.hypot(x[:, 0], x[:, 1])
    assert np.all(np.abs(rr[f == 1] - 1.0) <= 4.5e-16)


@pytest.mark.parametrize("batch,line_search", [(3, 0), (4, 4)])
def test_cycle_lbfgsb_zones_fp64_matches_oracle(batch, line_search):
    """The paper's cycle with its optimiser: L-BFGS-B on (t, u) per zone (Sec. II C step 4, Sec. II D)
    after the border-interior split, float64 throughout; accept decisions equal, charges to 1e-9."""
    n = 1500
    pos = synth.arcsine_disk(n, 13)
    s0 = 1 - 1 / (2 * np.sqrt(n))
    p0, f = oracle.border_split(pos, oracle.boundary_count(n), s0)
    u = np.random.default_rng(15).random((12, 3))
    kw = dict(m_min=20, m_max=150, period=4)
    po, trace_o, do, ao = oracle.cycle(p0, u, batch=batch, step0=1e-4, alpha_min=0.0, alpha_max=0.0, steps=12,
                                       sigma0=s0, sigma1=1.0, flags=f, optimizer="lbfgsb_tu", memory=6,
                                       maxstep=0.02, line_search=line_search, **kw)
    p = T(p0.copy())
    r, trace = tc.cycle(p, T(u), T(f), batch=batch, local_precision="fp64", precision="fp64",
                        optimizer="lbfgsb_tu", n_steps=12, memory=6, step0=1e-4, maxstep=0.02,
                        line_search=line_search, sigma0=s0, sigma1=1.0, **kw)
    tc.sync_status()
    np.testing.assert_array_equal(r.status.cpu().numpy(), ao)
    assert (ao == 1).sum() >= 3
    np.testing.assert_allclose(p.cpu().numpy(), po, rtol=0, atol=1e-9)
    # charges within 1e-9 move E by at most sum_i |g_i| 1e-9, a few 1e-10 of E here; the last
    # trace entry is E of the GPU's own final configuration, to float64 summation accuracy
    np.testing.assert_allclose(trace.cpu().numpy(), trace_o, rtol=1e-9)
    eg = oracle.energy(p.cpu().numpy())
    assert abs(trace[-1].item() - eg) <= 1e-13 * eg
    d = r.delta_e.cpu().numpy()
    np.testing.assert_allclose(d[ao == 1], do[ao == 1], rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("optimizer", ["bb", "lbfgsb_tu"])
def test_disjoint_cycle_fp64_matches_oracle(optimizer):
    """Disjoint batches (the longest prefix of pairwise disjoint zones among the next `batch`
    subdomains): the same batches, zones, accept decisions, positions and energy trace as the oracle,
    no zone skipped.  The GPU call takes sigma0 <= 0 as Eq. sigma; the oracle is given the value."""
    n = 1500
    pos = synth.arcsine_disk(n, 17)
    s0 = 1 - 1 / (2 * np.sqrt(n))
    p0, f = oracle.border_split(pos, oracle.boundary_count(n), s0)
    n_sub = 14
    u = np.random.default_rng(18).random((n_sub, 3))
    eta = 1e-4 / n
    kw = dict(m_min=20, m_max=200, period=5)
    opt = dict(memory=6, maxstep=0.02, step0=1e-4) if optimizer == "lbfgsb_tu" else dict(step0=eta)
    po, trace_o, do, ao = oracle.cycle(p0, u, batch=5, alpha_min=0.0, alpha_max=10 * eta, steps=8, sigma0=s0,
                                       sigma1=1.0, flags=f, disjoint=True, optimizer=optimizer, **opt, **kw)
    assert len(trace_o) - 1 > -(-n_sub // 5)  # some batch was cut short by an overlap
    p = T(p0.copy())
    r, trace = tc.cycle(p, T(u), T(f), batch=5, local_precision="fp64", precision="fp64", optimizer=optimizer,
                        n_steps=8, alpha_min=0.0, alpha_max=10 * eta, sigma0=0.0, sigma1=1.0, disjoint=True,
                        **opt, **kw)
    tc.sync_status()
    st = r.status.cpu().numpy()
    np.testing.assert_array_equal(st, ao)
    assert np.all(st != 2)
    # later batches start from positions moved by earlier ones, so float64 rounding differences
    # (fused multiply-adds on the GPU, none in the oracle) carry through: ~1e-10 after 14 zones,
    # which moves E (~1.8e6, wall forces ~1e5) by ~5e-6, i.e. ~3e-12 relative
    np.testing.assert_allclose(p.cpu().numpy(), po, rtol=0, atol=1e-9)
    tr = trace.cpu().numpy()
    assert tr.shape == trace_o.shape
    np.testing.assert_allclose(tr, trace_o, rtol=1e-11)


def test_border_split_default_sigma_is_eq_sigma():
    """sigma left out: the interior radius of Eq. sigma, 1 - 1/(2 sqrt(N)) (Sec. II B)."""
    n = 4000
    pos = synth.arcsine_disk(n, 19)
    po, fo = oracle.border_split(pos, oracle.boundary_count(n), 1 - 1 / (2 * np.sqrt(n)))
    p = T(pos.copy())
    f = tc.border_split(p)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(f.cpu().numpy(), fo)
    np.testing.assert_array_equal(p.cpu().numpy(), po)
