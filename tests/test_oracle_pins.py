"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties an oracle function to something other than itself: a closed
form, an extended-precision brute force, an exact invariant, a derivative
relation between two different oracle functions, a known minimum, or a number
the paper prints.  A dropped term, a wrong sign, a swapped index or a
transposed operand in tests/../oracle/tco.c fails at least one of them.
"""

from __future__ import annotations

import math
import os

import mpmath as mp
import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.txt")


def golden() -> dict:
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if "=" in line:
                k, v = line.split("=", 1)
                out[k.strip()] = float(v)
    return out


def gross(pos):
    """G_i = sum_{j != i} 1/r_ij^2, the scale of the gradient row before cancellation."""
    d = pos[:, None, :] - pos[None, :, :]
    r2 = (d ** 2).sum(-1)
    np.fill_diagonal(r2, np.inf)
    return (1.0 / r2).sum(1)


def cubic(pos):
    """C_i = sum_{j != i} 2/r_ij^3: how much row i's gradient moves per unit position error."""
    d = pos[:, None, :] - pos[None, :, :]
    r = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(r, np.inf)
    return (2.0 / r ** 3).sum(1)


# ------------------------------------------------------------ closed forms ---

def ngon_energy_mp(n):
    """Regular n-gon on the unit circle: E = (n/2) sum_{k=1}^{n-1} 1/(2 sin(pi k/n)) (chord lengths)."""
    mp.mp.dps = 40
    return mp.mpf(n) / 2 * mp.fsum(1 / (2 * mp.sin(mp.pi * k / n)) for k in range(1, n))


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 10, 100, 1000])
def test_ngon_closed_form(n):
    pos = synth.ngon(n, phase=0.37)
    e = oracle.energy(pos)
    ref = float(ngon_energy_mp(n))
    assert abs(e - ref) <= 4e-16 * ref * max(1.0, math.log2(n))
    g = oracle.grad(pos)
    u = pos / np.linalg.norm(pos, axis=1)[:, None]
    gr = (g * u).sum(1)
    gt = g - gr[:, None] * u
    G = gross(pos)
    # symmetry: no tangential force, equal inward radial gradient (outward force) on all charges;
    # the vertices' own rounding (~1 ulp of cos, sin, each) moves a row by up to ~1e-15 C_i
    tol = 1e-13 * G + 2e-15 * cubic(pos)
    assert np.all(np.linalg.norm(gt, axis=1) <= tol)
    assert np.all(gr < 0)
    assert np.ptp(gr) <= 2 * tol.max()


def test_small_hand_cases():
    e2 = oracle.energy(np.array([[1.0, 0.0], [-1.0, 0.0]]))
    assert e2 == 0.5
    g2 = oracle.grad(np.array([[1.0, 0.0], [-1.0, 0.0]]))
    # dE/dr_1 = -(r_1 - r_2)/|r_1 - r_2|^3 = -(2,0)/8: points inward; the force -g points outward
    np.testing.assert_array_equal(g2, [[-0.25, 0.0], [0.25, 0.0]])
    tri = synth.ngon(3)
    assert abs(oracle.energy(tri) - math.sqrt(3.0)) <= 2e-16 * math.sqrt(3.0)
    assert oracle.energy(np.zeros((0, 2))) == 0.0
    assert oracle.energy(np.array([[0.3, 0.1]])) == 0.0
    np.testing.assert_array_equal(oracle.grad(np.array([[0.3, 0.1]])), [[0.0, 0.0]])


def brute_mp(pos):
    mp.mp.dps = 40
    n = pos.shape[0]
    P = [(mp.mpf(float(x)), mp.mpf(float(y))) for x, y in pos]
    E = mp.mpf(0)
    g = [[mp.mpf(0), mp.mpf(0)] for _ in range(n)]
    le = [mp.mpf(0) for _ in range(n)]
    for i in range(n):
        for j in range(n):
            if i == j:
                continue
            dx, dy = P[i][0] - P[j][0], P[i][1] - P[j][1]
            r = mp.sqrt(dx * dx + dy * dy)
            if i < j:
                E += 1 / r
            le[i] += 1 / (2 * r)
            g[i][0] -= dx / r ** 3
            g[i][1] -= dy / r ** 3
    return E, np.array([[float(a), float(b)] for a, b in g]), np.array([float(v) for v in le])


@pytest.mark.parametrize("n,seed", [(3, 0), (7, 1), (12, 2), (20, 3)])
def test_brute_force_extended_precision(n, seed):
    pos = synth.arcsine_disk(n, seed)
    E, g, le = brute_mp(pos)
    e, loc = oracle.energy(pos, local=True)
    assert abs(e - float(E)) <= 2e-16 * float(E)
    np.testing.assert_allclose(loc, le, rtol=4e-16, atol=0)
    G = gross(pos)
    go = oracle.grad(pos)
    assert np.all(np.abs(go - g) <= 4e-16 * G[:, None])
    rows = np.array([n - 1, 0, n // 2], dtype=np.int32)
    gr, er = oracle.rows_grad(pos, rows)
    np.testing.assert_array_equal(gr, go[rows])
    np.testing.assert_allclose(er, 2 * le[rows], rtol=4e-16)


# ------------------------------------------------------------- invariants ---

def test_invariances_and_identities():
    n = 300
    pos = synth.arcsine_disk(n, 5)
    e, loc = oracle.energy(pos, local=True)
    g = oracle.grad(pos)
    G = gross(pos)
    th = 1.234
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    pr = pos @ R.T
    assert abs(oracle.energy(pr) - e) <= 1e-14 * e
    gr = oracle.grad(pr)
    assert np.all(np.linalg.norm(gr - g @ R.T, axis=1) <= 1e-13 * G)
    refl = pos * np.array([1.0, -1.0])
    assert abs(oracle.energy(refl) - e) <= 1e-14 * e
    np.testing.assert_allclose(oracle.grad(refl), g * np.array([1.0, -1.0]), atol=1e-13 * G.max(), rtol=0)
    perm = np.random.default_rng(0).permutation(n)
    assert abs(oracle.energy(pos[perm]) - e) <= 1e-14 * e
    assert np.all(np.abs(oracle.grad(pos[perm]) - g[perm]) <= 1e-13 * G[perm, None])
    # Newton's third law: the gradient rows sum to zero
    assert np.all(np.abs(g.sum(0)) <= 1e-13 * G.sum())
    # Euler's theorem for the degree -1 homogeneous E: sum_i r_i . g_i = -E
    assert abs((pos * g).sum() + e) <= 1e-12 * e
    # local energies add up to the total (Sec. II C step 1)
    assert abs(loc.sum() - e) <= 1e-14 * e


def test_scaling_law_degree_minus_one():
    pos = synth.arcsine_disk(200, 9) * 0.5
    e = oracle.energy(pos)
    assert abs(oracle.energy(pos * 0.5) - 2.0 * e) <= 1e-14 * e


# ------------------------------------------------- derivative relations ---

def test_gradient_matches_central_differences_of_delta_energy():
    """dE/dx_i from tco_grad equals the central difference of the pairwise dE (a different function)."""
    n = 2000
    pos = synth.arcsine_disk(n, 11)
    g = oracle.grad(pos)
    rng = np.random.default_rng(1)
    h = 1e-6
    for i in rng.choice(n, 6, replace=False):
        for c in range(2):
            plus = pos[i].copy()
            minus = pos[i].copy()
            plus[c] += h
            minus[c] -= h
            if np.linalg.norm(plus) > 1 or np.linalg.norm(minus) > 1:
                continue
            dp = oracle.delta_energy(pos, [i], plus[None])
            dm = oracle.delta_energy(pos, [i], minus[None])
            fd = (dp - dm) / (2 * h)
            # truncation h^2/6 |d3E| plus rounding eps |e_i| / h
            d = np.linalg.norm(pos - pos[i], axis=1)
            d[i] = np.inf
            tol = h * h * (6.0 / d ** 4).sum() + 1e-16 * (1.0 / d).sum() / h * 4
            assert abs(fd - g[i, c]) <= tol + 1e-9 * abs(g[i, c])


def test_subdomain_objective_definition_and_gradient():
    n = 400
    pos = synth.arcsine_disk(n, 3)
    idx = np.array(sorted(np.random.default_rng(2).choice(n, 40, replace=False)), dtype=np.int32)
    act = pos[idx].copy()
    g, e, esub = oracle.subdomain_grad(pos, idx, act)
    # E = E_sub + E(F alone): the subdomain objective is E minus the constant F-F energy
    F = np.setdiff1d(np.arange(n), idx)
    etot = oracle.energy(pos)
    assert abs(esub + oracle.energy(pos[F]) - etot) <= 1e-13 * etot
    # with A at the snapshot, the subdomain gradient rows equal the full gradient rows
    gf = oracle.grad(pos)
    np.testing.assert_allclose(g, gf[idx], rtol=0, atol=1e-13 * np.abs(gf).max())
    # move A, then: E_sub(new) - E_sub(old) == pairwise dE, and the gradient at the moved
    # configuration matches central differences of E_sub
    rng = np.random.default_rng(4)
    act2 = act + rng.normal(0, 1e-3, act.shape)
    act2 = oracle.project(act2)
    g2, _, esub2 = oracle.subdomain_grad(pos, idx, act2)
    de = oracle.delta_energy(pos, idx, act2)
    assert abs((esub2 - esub) - de) <= 1e-11 * esub
    h = 1e-6
    for k in [0, 7, 39]:
        for c in range(2):
            ap = act2.copy()
            am = act2.copy()
            ap[k, c] += h
            am[k, c] -= h
            dp = oracle.delta_energy(pos, idx, ap)
            dm = oracle.delta_energy(pos, idx, am)
            fd = (dp - dm) / (2 * h)
            assert abs(fd - g2[k, c]) <= 1e-5 * (1 + abs(g2[k, c]))


def test_delta_energy_against_extended_precision():
    n = 25
    pos = synth.arcsine_disk(n, 21)
    idx = np.array([2, 5, 6, 11, 24], dtype=np.int32)
    new = pos[idx] * 0.97 + 0.01
    E0, _, _ = brute_mp(pos)
    p1 = pos.copy()
    p1[idx] = new
    E1, _, _ = brute_mp(p1)
    de = oracle.delta_energy(pos, idx, new)
    assert abs(de - float(E1 - E0)) <= 1e-15 * float(E0)


def test_delta_energy_difference_of_totals_small_n():
    n = 1500
    pos = synth.arcsine_disk(n, 8)
    idx = np.arange(100, 400, 3, dtype=np.int32)
    new = oracle.project(pos[idx] + np.random.default_rng(6).normal(0, 2e-3, (idx.size, 2)))
    p1 = pos.copy()
    p1[idx] = new
    e0, e1 = oracle.energy(pos), oracle.energy(p1)
    de = oracle.delta_energy(pos, idx, new)
    assert abs(de - (e1 - e0)) <= 1e-13 * e0


# ----------------------------------------------------------- constraint ---

def test_project():
    rng = np.random.default_rng(3)
    pts = rng.uniform(-1.5, 1.5, (500, 2))
    out = oracle.project(pts, radius=0.9)
    r_in = np.linalg.norm(pts, axis=1)
    inside = r_in <= 0.9
    np.testing.assert_array_equal(out[inside], pts[inside])
    r_out = np.linalg.norm(out[~inside], axis=1)
    assert np.all(np.abs(r_out - 0.9) <= 4e-16)
    cross = pts[~inside, 0] * out[~inside, 1] - pts[~inside, 1] * out[~inside, 0]
    assert np.all(np.abs(cross) <= 1e-15 * r_in[~inside])
    assert np.all((pts[~inside] * out[~inside]).sum(1) > 0)
    flags = np.zeros(500, np.uint8)
    flags[::3] = 1
    outp = oracle.project(pts, radius=0.9, flags=flags)
    assert np.all(np.abs(np.linalg.norm(outp[::3], axis=1) - 1.0) <= 4e-16)


def test_projected_grad():
    pos = synth.ngon(12)
    g = oracle.grad(pos)
    pg, rms, mx = oracle.projected_grad(pos, g)
    # on the circle the outward force is blocked; the n-gon is stationary
    assert mx <= 1e-12 * np.abs(g).max()
    inner = pos * 0.5
    g2 = oracle.grad(inner)
    pg2, _, _ = oracle.projected_grad(inner, g2)
    np.testing.assert_array_equal(pg2, g2)


# --------------------------------------------------------------- descent ---

def test_pgd_step_and_descent():
    n = 300
    pos = synth.arcsine_disk(n, 13)
    eta = 1e-4 / n
    x1, tr = oracle.pgd(pos, eta, 1)
    manual = oracle.project(pos - eta * oracle.grad(pos))
    np.testing.assert_array_equal(x1, manual)
    _, tr = oracle.pgd(pos, eta, 30)
    assert np.all(np.diff(tr) < 0)
    # the regular polygon on the wall is a fixed point of projected descent
    ng = synth.ngon(9)
    x, _ = oracle.pgd(ng, 1e-3, 5)
    np.testing.assert_allclose(x, ng, atol=1e-15)


def test_subdomain_bb_reduces_energy_and_fixed_step_is_pgd():
    n = 600
    pos = synth.arcsine_disk(n, 17)
    idx = np.arange(0, n, 7, dtype=np.int32)
    eta = 1e-4 / n
    # alpha_min = alpha_max = step0 turns BB off: plain projected descent on E_sub
    x = oracle.subdomain_bb(pos, idx, eta, eta, eta, 3)
    a = pos[idx].copy()
    for _ in range(3):
        g, _, _ = oracle.subdomain_grad(pos, idx, a)
        a = oracle.project(a - eta * g)
    np.testing.assert_allclose(x, a, rtol=0, atol=1e-15)
    xb = oracle.subdomain_bb(pos, idx, eta, 0.0, 10 * eta, 40)
    assert oracle.delta_energy(pos, idx, xb) < oracle.delta_energy(pos, idx, x) < 0


def test_accept_sequential():
    n = 800
    pos = synth.lattice_disk(n, 1, 0.05)
    subs = [np.arange(0, 60, dtype=np.int32), np.arange(50, 120, dtype=np.int32),
            np.arange(200, 260, dtype=np.int32)]
    idx, off = synth.to_csr(subs)
    eta = 1e-4 / n
    new = np.concatenate([oracle.subdomain_bb(pos, s, eta, 0.0, 10 * eta, 20) for s in subs])
    new[off[2]:off[3]] = pos[subs[2]] + 0.01  # an uphill move
    new[off[2]:off[3]] = oracle.project(new[off[2]:off[3]])
    p1, d, acc = oracle.accept_sequential(pos, idx, off, new)
    assert acc[0] == 1 and d[0] < 0
    assert acc[1] == 2  # shares charges 50..59 with an accepted subdomain
    assert acc[2] == 0 and d[2] > 0
    e0, e1 = oracle.energy(pos), oracle.energy(p1)
    assert abs((e1 - e0) - d[0]) <= 1e-12 * e0
    np.testing.assert_array_equal(p1[subs[0]], new[:60])
    np.testing.assert_array_equal(p1[subs[2]], pos[subs[2]])


@pytest.mark.parametrize("n", [3, 4, 5, 8])
def test_lbfgs_reaches_ring_minimum(n):
    """For these small N the lowest-energy state of charges in a disk is the ring (regular N-gon)."""
    x, it, rms = oracle.lbfgs(synth.arcsine_disk(n, 2), max_iter=500, gtol=1e-12, step0=1e-3, maxstep=0.05)
    assert rms < 1e-12
    ref = float(ngon_energy_mp(n))
    assert abs(oracle.energy(x) - ref) <= 1e-14 * ref
    assert np.all(np.abs(np.linalg.norm(x, axis=1) - 1.0) <= 1e-12)


def test_lbfgs_relaxed_energy_against_asymptotic_expansion():
    """Relaxed minima at N = 100, 150 lie just above the fit of Eq. (asym) with the paper's coefficients."""
    gd = golden()
    for n, seed in [(100, 12), (150, 4)]:
        x, it, rms = oracle.lbfgs(synth.arcsine_disk(n, seed), max_iter=2000, gtol=1e-9, step0=1e-5,
                                  maxstep=0.03)
        assert rms < 1e-9
        e = oracle.energy(x)
        easym = math.pi / 4 * n ** 2 + gd["k2"] * n ** 1.5 + gd["k3"] * n + gd["k4"] * n ** 0.5 + gd["k5"]
        assert easym < e < easym * 1.006
        # stationarity in Cartesian form: tangential force on wall charges, full force inside
        pg, rms_c, mx = oracle.projected_grad(x, oracle.grad(x))
        assert mx < 1e-6


# ------------------------------------------------------ paper's numbers ---

def test_paper_numbers_recomputed():
    gd = golden()
    n = 1e5
    easym = math.pi / 4 * n ** 2 + gd["k2"] * n ** 1.5 + gd["k3"] * n + gd["k4"] * n ** 0.5 + gd["k5"]
    assert abs(easym - gd["E_asym_1e5"]) <= 1e-12 * easym
    dev = abs(gd["E_min_1e5"] - easym) / easym
    assert abs(dev - gd["deviation_1e5"]) <= 5e-4 * gd["deviation_1e5"]
    nb = gd["Nb_a"] * n ** (2 / 3) + gd["Nb_b"] * n ** (1 / 3) + gd["Nb_c"]
    assert round(nb) == gd["N_b_best"]


def test_arcsine_energy_trend():
    """E/N^2 -> pi/4 (Sec. I): arcsine-random charges have E[1/|X-Y|] = pi/2, so E ~ (pi/4) N(N-1)."""
    n = 1500
    vals = [oracle.energy(synth.arcsine_disk(n, s)) / (n * (n - 1) / 2) for s in range(6)]
    m = float(np.mean(vals))
    se = float(np.std(vals, ddof=1)) / math.sqrt(len(vals))
    assert abs(m - math.pi / 2) <= 4 * se + 2e-3


def test_error_statuses():
    with pytest.raises(oracle.OracleError) as e:
        oracle.energy(np.array([[0.2, 0.1], [0.2, 0.1]]))
    assert e.value.code == 3
    with pytest.raises(oracle.OracleError) as e:
        oracle.grad(np.array([[1.2, 0.0], [0.0, 0.0]]))
    assert e.value.code == 4
    with pytest.raises(oracle.OracleError) as e:
        oracle.delta_energy(synth.arcsine_disk(10, 0), [3, 3], np.zeros((2, 2)))
    assert e.value.code == 1


def test_openmp_build_is_bit_identical():
    """The OpenMP build only splits independent rows over threads: results equal the plain build."""
    pos = synth.arcsine_disk(3000, 5)
    rows = np.arange(0, 3000, 3, dtype=np.int32)
    g1, e1 = oracle.rows_grad(pos, rows)
    g2, e2 = oracle.rows_grad(pos, rows, openmp=True)
    assert oracle.threads() == 1 and oracle.threads(True) >= 1
    assert np.array_equal(g1, g2) and np.array_equal(e1, e2)
    with pytest.raises(oracle.OracleError):
        oracle.rows_grad(pos, np.array([0, 3000], dtype=np.int32), openmp=True)


# ---------------------------------------------------------------- the cycle (Sec. II C) ---

def test_zone_size_triangle_wave():
    """m = m_min at q = 0 mod P, m_max at q = P/2, linear in between, symmetric, capped at n."""
    assert [oracle.zone_size(q, 50, 200, 4, 10 ** 6) for q in range(9)] == [50, 125, 200, 125, 50, 125, 200, 125, 50]
    assert [oracle.zone_size(q, 50, 200, 5, 10 ** 6) for q in range(5)] == [50, 110, 170, 170, 110]
    assert {oracle.zone_size(q, 7, 900, 1, 10 ** 6) for q in range(10)} == {7}
    assert oracle.zone_size(2, 50, 200, 4, 120) == 120


def _zones(pos, e, u, **kw):
    idx, off, cen, st = oracle.zone_select(pos, e, u, **kw)
    return [idx[off[s]:off[s + 1]] for s in range(len(off) - 1)], off, cen, st


def test_zone_select_statistics_defects_and_nearest_sets():
    """mu and sigma_e equal numpy's mean and population std; the defect count follows the rule;
    each zone holds exactly m charges, ascending, and none outside it is nearer to the centre."""
    n = 1500
    pos = synth.lattice_disk(n, 11, 0.05)
    _, e = oracle.energy(pos, local=True)
    u = np.random.default_rng(4).random((12, 3))
    zones, off, cen, st = _zones(pos, e, u, m_min=30, m_max=300, period=6, phase=2)
    assert abs(st[0] - e.mean()) <= 1e-15 * e.mean()
    assert abs(st[1] - e.std()) <= 1e-12 * e.std()
    r = np.hypot(pos[:, 0], pos[:, 1])
    thr = e.mean() - e.std()
    n_def = int(np.sum((e > thr) & (r < 1 - 1e-9)))
    assert st[2] == n_def and 0 < n_def < n
    for s, z in enumerate(zones):
        assert len(z) == oracle.zone_size(2 + s, 30, 300, 6, n)
        assert np.all(np.diff(z) > 0)
        d2 = ((pos - cen[s]) ** 2).sum(1)
        out = np.setdiff1d(np.arange(n), z)
        assert d2[z].max() <= d2[out].min()
        assert np.hypot(*cen[s]) <= 1.0


def test_zone_centres_follow_the_mix():
    """p_defect = 1: every centre is a defect charge (the zone's nearest, at distance 0);
    p_defect = 0: centres are area-uniform in the disk (|c|^2 ~ U(0,1), angle ~ U(0, 2 pi))."""
    from scipy import stats as ss

    n = 800
    pos = synth.arcsine_disk(n, 3)
    _, e = oracle.energy(pos, local=True)
    u = np.random.default_rng(5).random((40, 3))
    zones, _, cen, st = _zones(pos, e, u, m_min=5, m_max=5, period=1, p_defect=1.0)
    r = np.hypot(pos[:, 0], pos[:, 1])
    defects = np.flatnonzero((e > st[0] - st[1]) & (r < 1 - 1e-9))
    for s in range(40):
        k = np.flatnonzero((pos == cen[s]).all(1))
        assert len(k) == 1 and k[0] in defects and k[0] in zones[s]
        # floor(u1 |D|) picks the defect
        assert k[0] == defects[int(u[s, 1] * len(defects))]
    u = np.random.default_rng(6).random((3000, 3))
    _, _, cen, _ = _zones(pos, e, u, m_min=0, m_max=0, period=1, p_defect=0.0)
    rr = (cen ** 2).sum(1)
    assert ss.kstest(rr, "uniform").pvalue > 1e-3
    th = np.mod(np.arctan2(cen[:, 1], cen[:, 0]), 2 * np.pi) / (2 * np.pi)
    assert ss.kstest(th, "uniform").pvalue > 1e-3


def test_zone_ties_break_by_index():
    """Charges on a dyadic grid have exact, equal distances to the centre (0, 0): the zone takes the
    ring members with the smallest indices, and m >= n takes every charge."""
    g = np.arange(-6, 7) / 8.0
    pos = np.array([(x, y) for x in g for y in g if x * x + y * y <= 0.75])
    rng = np.random.default_rng(2)
    pos = pos[rng.permutation(len(pos))]
    n = len(pos)
    e = np.zeros(n)  # flat energies: no defects, so the centre is the uniform draw
    u = np.array([[0.5, 0.0, 0.3]])  # u1 = 0: the centre is the origin
    d2 = (pos ** 2).sum(1)
    for m in [1, 5, 6, 9, 13, 20, 21, n, n + 5]:
        zones, _, cen, st = _zones(pos, e, u, m_min=m, m_max=m, period=1, kappa=1.0)
        assert st[2] == 0 and np.all(cen[0] == 0)
        z = zones[0]
        mm = min(m, n)
        assert len(z) == mm
        if mm < n:
            cut = np.sort(d2)[mm - 1]
            below = np.flatnonzero(d2 < cut)
            ties = np.flatnonzero(d2 == cut)[: mm - len(below)]
            assert np.array_equal(z, np.sort(np.concatenate([below, ties])))


def test_cycle_energy_bookkeeping():
    """Over a cycle the energy falls by exactly the accepted pairwise changes: E_(b+1) - E_b equals
    the sum of dE_s over the batch's accepted subdomains; rejected and skipped ones change nothing;
    batch = 1 never skips."""
    n = 1200
    pos = synth.lattice_disk(n, 9, 0.05)
    u = np.random.default_rng(8).random((9, 3))
    eta = 1e-4 / n
    for batch in [4, 1]:
        p, trace, d, acc = oracle.cycle(pos, u, m_min=20, m_max=160, period=4, batch=batch, step0=eta,
                                        alpha_min=0.0, alpha_max=10 * eta, steps=8)
        nb = -(-9 // batch)
        assert len(trace) == nb + 1 and np.all(np.diff(trace) <= 0)
        assert abs(trace[-1] - oracle.energy(p)) <= 1e-15 * trace[-1]
        for b in range(nb):
            sl = slice(b * batch, min(9, (b + 1) * batch))
            dsum = d[sl][acc[sl] == 1].sum()
            assert abs((trace[b + 1] - trace[b]) - dsum) <= 1e-12 * trace[b]
        assert np.all(d[acc == 1] < 0) and np.all(d[acc == 0] >= 0)
        assert (acc == 1).sum() >= 1
        if batch == 1:
            assert not np.any(acc == 2)


# ------------------------------------------------ border-interior split (Sec. II B) ---

def test_boundary_count_is_the_papers():
    """Eq. Nb at N = 1e5 gives the paper's N_b (Table I); small N clamp at 0; N_b grows with N."""
    gd = golden()
    assert oracle.boundary_count(100_000) == gd["N_b_best"]
    assert oracle.boundary_count(0) == 0 and oracle.boundary_count(1) == 0
    seq = [oracle.boundary_count(n) for n in range(1, 5000)]
    assert all(a <= b <= a + 2 for a, b in zip(seq, seq[1:]))
    assert all(0 <= b <= n for n, b in zip(range(1, 5000), seq))


def test_sigma_ramp_endpoints_and_linearity():
    s0 = 1 - 1 / (2 * math.sqrt(1e5))  # Eq. sigma
    assert oracle.sigma_ramp(s0, 1.0, 0, 9) == s0 and oracle.sigma_ramp(s0, 1.0, 8, 9) == 1.0
    assert oracle.sigma_ramp(s0, 1.0, 0, 1) == 1.0
    mid = oracle.sigma_ramp(s0, 1.0, 4, 9)
    assert abs(mid - (s0 + 1.0) / 2) <= 1e-16


def test_border_split_pins_the_outermost():
    """The n_b charges of largest |r| (ties: larger index first) end on the unit circle with flags set;
    the others end inside sigma, unchanged where they already were."""
    n = 2000
    pos = synth.arcsine_disk(n, 8)
    nb = oracle.boundary_count(n)
    sigma = 1 - 1 / (2 * math.sqrt(n))
    p, f = oracle.border_split(pos, nb, sigma)
    r0 = np.hypot(pos[:, 0], pos[:, 1])
    assert f.sum() == nb
    assert r0[f == 1].min() >= r0[f == 0].max()
    r1 = np.hypot(p[:, 0], p[:, 1])
    assert np.all(np.abs(r1[f == 1] - 1.0) <= 4.5e-16)
    assert np.all(r1[f == 0] <= sigma * (1 + 4.5e-16))
    keep = (f == 0) & (r0 <= sigma)
    assert np.array_equal(p[keep], pos[keep])
    # direction preserved
    cross = pos[:, 0] * p[:, 1] - pos[:, 1] * p[:, 0]
    assert np.all(np.abs(cross) <= 1e-15)
    # exact ties on a dyadic ring: the larger indices become boundary charges
    g = np.array([[1, 0], [0, 1], [-1, 0], [0, -1], [0.5, 0], [0, 0.25]], dtype=float) * 0.75
    _, f2 = oracle.border_split(g, 2, 0.9)
    assert f2.tolist() == [0, 0, 1, 1, 0, 0]


def test_cycle_with_pinned_boundary_and_sigma_ramp():
    """With the split and a sigma ramp, the cycle keeps its bookkeeping, pinned charges stay on the unit
    circle and never become centres' defects, and free charges stay within the final sigma."""
    n = 1500
    pos = synth.arcsine_disk(n, 13)
    nb = oracle.boundary_count(n)
    s0 = 1 - 1 / (2 * math.sqrt(n))
    p0, f = oracle.border_split(pos, nb, s0)
    u = np.random.default_rng(14).random((9, 3))
    eta = 1e-4 / n
    # pinned charges are never defects: on the unprojected input they are not excluded by radius
    _, e = oracle.energy(pos, local=True)
    _, _, cen, st = oracle.zone_select(pos, e, u, m_min=20, m_max=150, period=4, flags=f, p_defect=1.0)
    _, _, _, st_nf = oracle.zone_select(pos, e, u, m_min=20, m_max=150, period=4, p_defect=1.0)
    thr = st[0] - st[1]
    r0 = np.hypot(pos[:, 0], pos[:, 1])
    assert st_nf[2] - st[2] == np.sum((e > thr) & (f == 1) & (r0 < 1 - 1e-9)) > 0
    for c in cen:
        k = np.flatnonzero((pos == c).all(1))
        assert len(k) == 1 and f[k[0]] == 0
    p, trace, d, acc = oracle.cycle(p0, u, m_min=20, m_max=150, period=4, batch=3, step0=eta, alpha_min=0.0,
                                    alpha_max=10 * eta, steps=8, sigma0=s0, sigma1=1.0, flags=f)
    assert np.all(np.diff(trace) <= 0)
    for b in range(3):
        sl = slice(3 * b, 3 * b + 3)
        assert abs((trace[b + 1] - trace[b]) - d[sl][acc[sl] == 1].sum()) <= 1e-12 * trace[b]
    r = np.hypot(p[:, 0], p[:, 1])
    assert np.all(np.abs(r[f == 1] - 1.0) <= 4.5e-16)
    assert np.all(r[f == 0] <= 1.0 + 1e-15)
    assert (acc == 1).sum() >= 1


# ------------------------------------------------ structure analysis (Sec. III C-D) ---

def _tri_lattice(k, h=0.05, angle=0.0):
    pts = []
    for a in range(-k, k + 1):
        for b in range(-k, k + 1):
            x, y = h * (a + 0.5 * b), h * (b * math.sqrt(3) / 2)
            pts.append((x, y))
    p = np.array(pts)
    c, s = math.cos(angle), math.sin(angle)
    return p @ np.array([[c, s], [-s, c]])


def test_structure_triangular_lattice():
    """Interior sites of a triangular lattice have six neighbours and |psi6| = 1; rotating the lattice
    by alpha turns psi6 into exp(6 i alpha)."""
    from oracle import structure as S

    # a small in-plane jitter breaks the lattice's cocircular degeneracy without changing neighbours
    rng = np.random.default_rng(3)
    for alpha in [0.0, 0.1, 0.37]:
        p = _tri_lattice(6, angle=alpha)
        p = p + rng.normal(0, 1e-9, p.shape)
        z, psi = S.order(p)
        inner = np.hypot(p[:, 0], p[:, 1]) < 0.15
        assert np.all(z[inner] == 6)
        assert np.allclose(np.abs(psi[inner]), 1.0, atol=1e-6)
        assert np.allclose(psi[inner], np.exp(6j * alpha), atol=1e-6)


def test_structure_polygon_centres_and_euler():
    """A charge at the centre of a regular k-gon has k neighbours and psi6 = (1/k) sum exp(6 i 2 pi m/k)
    (1 for k = 6, 0 for k = 7); every triangulation has sum z = 2 (3N - 3 - h), h the hull size."""
    from oracle import structure as S

    for k, want in [(6, 1.0 + 0j), (7, 0j), (12, 0j)]:
        ang = 2 * math.pi * np.arange(k) / k + 0.05
        ring = 0.8 * np.stack([np.cos(ang), np.sin(ang)], 1)
        p = np.vstack([[0.0, 0.0], ring])
        z, psi = S.order(p)
        assert z[0] == k
        ref = np.exp(6j * 2 * math.pi * np.arange(k) / k).mean() * np.exp(6j * 0.05)
        assert abs(psi[0] - ref) <= 1e-12 and abs(abs(psi[0]) - abs(want)) <= 1e-12
    # ring of h charges on the circle + random interior: the hull is exactly the ring
    h = 40
    ang = 2 * math.pi * (np.arange(h) + 0.3) / h
    ring = np.stack([np.cos(ang), np.sin(ang)], 1)
    inner = synth.arcsine_disk(300, 4) * 0.9
    p = np.vstack([ring, inner])
    z, _ = S.order(p)
    assert z.sum() == 2 * (3 * len(p) - 3 - h)
    nb = S.neighbours(p)
    assert all(i in nb[j] for i in range(len(p)) for j in nb[i])  # symmetric


def test_lbfgs_line_search_is_monotone_and_converges():
    """With the Armijo line search every iteration lowers the energy (checked by rerunning the
    deterministic iteration for 1..25 steps), and the N = 8 ring relaxes to a float64-stationary point."""
    pos = synth.arcsine_disk(120, 21)
    es = []
    for k in range(1, 26):
        x, it, _ = oracle.lbfgs(pos, max_iter=k, step0=1e-3, maxstep=0.05, line_search=10)
        assert it == k
        es.append(oracle.energy(x))
    assert all(b <= a for a, b in zip(es, es[1:]))
    x, it, rms = oracle.lbfgs(synth.arcsine_disk(8, 2), max_iter=2000, gtol=1e-10, step0=1e-3, maxstep=0.05,
                              line_search=10)
    assert rms < 1e-10
    _, rms_c, _ = oracle.projected_grad(x, oracle.grad(x))
    assert rms_c < 1e-9


@pytest.mark.parametrize("n,expect", [(3, math.sqrt(3)), (4, 1 + 2 * math.sqrt(2)), (5, 6.881909602355867)])
def test_lbfgs_tu_reaches_ring_minima(n, expect):
    """L-BFGS on the paper's (t, u) variables (Sec. II D) relaxes small N to the regular polygon on the
    circle, the same minimum the smooth-map iteration finds, and ends float64-stationary."""
    pos = synth.arcsine_disk(n, 3)
    x, it, rms = oracle.lbfgs(pos, max_iter=3000, gtol=1e-10, step0=1e-3, maxstep=0.05, tu=True)
    assert rms < 1e-10
    assert abs(oracle.energy(x) - expect) <= 1e-12 * expect
    _, rms_c, _ = oracle.projected_grad(x, oracle.grad(x))
    assert rms_c < 1e-8
    x2, _, _ = oracle.lbfgs(pos, max_iter=3000, gtol=1e-10, step0=1e-3, maxstep=0.05)
    assert abs(oracle.energy(x2) - oracle.energy(x)) <= 1e-12 * expect


def test_lbfgs_tu_with_pinned_boundary():
    """Pinned charges move along the unit circle as (cos u, sin u); the others stay inside sigma."""
    n = 80
    pos = synth.arcsine_disk(n, 9)
    p0, f = oracle.border_split(pos, 12, 0.95)
    x, it, rms = oracle.lbfgs(p0, max_iter=300, step0=1e-3, maxstep=0.05, radius=0.95, flags=f, tu=True)
    r = np.hypot(x[:, 0], x[:, 1])
    assert np.all(np.abs(r[f == 1] - 1.0) <= 4.5e-16)
    assert np.all(r[f == 0] <= 0.95 * (1 + 1e-15))
    assert oracle.energy(x) < oracle.energy(p0)


# ------------------------------------------------------------------ L-BFGS-B ---
# The pieces of L-BFGS-B (Byrd, Lu, Nocedal & Zhu 1995; Sec. II C step 4) are pinned against dense
# linear algebra: the BFGS matrix by its rank-two recursion, the Cauchy point by scanning the
# projected path, the subspace step by a dense reduced Newton solve.

def _bfgs_pairs(nv, h, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((nv, nv))
    hess = a @ a.T + nv * np.eye(nv)
    s = rng.standard_normal((h, nv))
    return s, s @ hess.T  # y = H s: every pair has s.y > 0


def _bfgs_dense(s_rows, y_rows, theta):
    b = theta * np.eye(s_rows.shape[1] if s_rows.ndim == 2 else 0)
    for s, y in zip(s_rows, y_rows):
        bs = b @ s
        b = b - np.outer(bs, bs) / (s @ bs) + np.outer(y, y) / (y @ s)
    return b


@pytest.mark.parametrize("h", [1, 2, 3, 5])
def test_lbfgsb_compact_form_is_the_bfgs_recursion(h):
    """theta I - W M W^T equals h rank-two BFGS updates of theta I applied oldest first."""
    s, y = _bfgs_pairs(9, h, 10 + h)
    theta = 3.7
    m = oracle.lbfgsb_middle(s, y, theta)
    w = np.hstack([y.T, theta * s.T])
    b = theta * np.eye(9) - w @ m @ w.T
    ref = _bfgs_dense(s, y, theta)
    assert np.abs(b - ref).max() <= 1e-11 * np.abs(ref).max()


def _box_case(seed, theta=0.05):
    """Variables 0-5 boxed in [0, 1], 6-9 free, 10 fixed; two stored pairs."""
    rng = np.random.default_rng(seed)
    nv = 11
    lo = np.r_[np.zeros(6), np.full(4, -np.inf), 0.3]
    hi = np.r_[np.ones(6), np.full(4, np.inf), 0.3]
    x = np.r_[rng.uniform(0.05, 0.95, 6), rng.standard_normal(4), 0.3]
    g = rng.standard_normal(nv)
    g[:6] *= 12.0  # steep enough that the projected path meets several bounds
    g[10] = 0.7  # a fixed variable's gradient must not move it
    s, y = _bfgs_pairs(nv, 2, seed)
    return x, g, lo, hi, s, y, theta


def _model(x, g, b, v):
    dv = v - x
    return g @ dv + 0.5 * dv @ b @ dv


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_lbfgsb_cauchy_point_is_first_minimum_along_projected_path(seed):
    """The generalized Cauchy point is the first local minimiser of the quadratic model along
    P(x - t g), found here by scanning t on a fine grid and refining with a bounded Brent search."""
    from scipy.optimize import minimize_scalar

    x, g, lo, hi, s, y, theta = _box_case(seed)
    m = oracle.lbfgsb_middle(s, y, theta)
    xc, c, nb = oracle.lbfgsb_cauchy(x, g, lo, hi, s, y, theta, m)
    b = _bfgs_dense(s, y, theta)
    path = lambda t: np.clip(x - t * g, lo, hi)
    f = lambda t: _model(x, g, b, path(t))
    ts = np.linspace(0.0, 40.0, 400001)
    vals = np.array([f(t) for t in ts])
    k = next(k for k in range(1, len(ts) - 1) if vals[k] <= vals[k - 1] and vals[k] <= vals[k + 1])
    r = minimize_scalar(f, bounds=(ts[k - 1], ts[k + 1]), method="bounded", options={"xatol": 1e-12})
    np.testing.assert_allclose(xc, path(r.x), rtol=0, atol=1e-7)
    assert xc[10] == 0.3 and np.all(xc >= lo) and np.all(xc <= hi)
    w = np.hstack([y.T, theta * s.T])
    np.testing.assert_allclose(c, w.T @ (xc - x), rtol=0, atol=1e-10 * np.abs(w).max())
    assert nb >= 3  # each case passes several breakpoints


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5])
def test_lbfgsb_subspace_step_is_reduced_newton_then_backtracked(seed):
    """From the Cauchy point, the free variables take the Newton step of the model restricted to
    them (dense solve with the BFGS matrix), shortened so that every variable stays in its box."""
    x, g, lo, hi, s, y, theta = _box_case(seed, theta=0.8)
    m = oracle.lbfgsb_middle(s, y, theta)
    xc, c, _ = oracle.lbfgsb_cauchy(x, g, lo, hi, s, y, theta, m)
    xbar = oracle.lbfgsb_subspace(x, g, lo, hi, s, y, theta, m, xc, c)
    b = _bfgs_dense(s, y, theta)
    free = (lo < xc) & (xc < hi)
    rc = g + b @ (xc - x)
    du = -np.linalg.solve(b[np.ix_(free, free)], rc[free])
    a = 1.0
    for v, l_, h_, dv in zip(xc[free], lo[free], hi[free], du):
        if dv > 0 and np.isfinite(h_):
            a = min(a, (h_ - v) / dv)
        if dv < 0 and np.isfinite(l_):
            a = min(a, (l_ - v) / dv)
    ref = xc.copy()
    ref[free] = xc[free] + a * du
    np.testing.assert_allclose(xbar, ref, rtol=0, atol=1e-10)
    assert np.all(xbar >= lo) and np.all(xbar <= hi)


def test_lbfgsb_subspace_cases_include_a_shortened_step():
    shortened = 0
    for seed in range(1, 6):
        x, g, lo, hi, s, y, theta = _box_case(seed, theta=0.8)
        m = oracle.lbfgsb_middle(s, y, theta)
        xc, c, _ = oracle.lbfgsb_cauchy(x, g, lo, hi, s, y, theta, m)
        xbar = oracle.lbfgsb_subspace(x, g, lo, hi, s, y, theta, m, xc, c)
        b = _bfgs_dense(s, y, theta)
        free = (lo < xc) & (xc < hi)
        du = -np.linalg.solve(b[np.ix_(free, free)], (g + b @ (xc - x))[free])
        shortened += not np.allclose(xbar[free], xc[free] + du, rtol=0, atol=1e-12)
    assert shortened >= 1


@pytest.mark.parametrize("h", [0, 1, 4])
def test_lbfgsb_without_bounds_is_the_quasi_newton_step(h):
    """With no finite bound, Cauchy point plus subspace step is x - B^{-1} g."""
    nv = 10
    rng = np.random.default_rng(50 + h)
    x, g = rng.standard_normal(nv), rng.standard_normal(nv)
    lo, hi = np.full(nv, -np.inf), np.full(nv, np.inf)
    s, y = _bfgs_pairs(nv, max(h, 1), 60 + h)
    s, y = s[:h], y[:h]
    theta = 1.3
    m = oracle.lbfgsb_middle(s, y, theta) if h else np.zeros((0, 0))
    xc, c, nb = oracle.lbfgsb_cauchy(x, g, lo, hi, s, y, theta, m)
    xbar = oracle.lbfgsb_subspace(x, g, lo, hi, s, y, theta, m, xc, c)
    b = _bfgs_dense(s, y, theta) if h else theta * np.eye(nv)
    assert nb == 0
    np.testing.assert_allclose(xbar, x - np.linalg.solve(b, g), rtol=0, atol=1e-12 * max(1.0, np.abs(g).max()))


@pytest.mark.parametrize("n,expect", [(3, math.sqrt(3)), (4, 1 + 2 * math.sqrt(2)), (5, 6.881909602355867)])
def test_lbfgsb_reaches_ring_minima(n, expect):
    """L-BFGS-B on (t, u) relaxes small N to the regular polygon on the circle (the closed-form
    ring energies) and ends with a vanishing projected gradient."""
    pos = synth.arcsine_disk(n, 3)
    x, it, rms, _ = oracle.lbfgsb(pos, max_iter=3000, gtol=1e-10, step0=1e-3, maxstep=0.05)
    assert rms < 1e-10
    assert abs(oracle.energy(x) - expect) <= 1e-12 * expect
    _, rms_c, _ = oracle.projected_grad(x, oracle.grad(x))
    assert rms_c < 1e-8


def test_lbfgsb_pinned_boundary_and_armijo_descent():
    """Pinned charges stay on the unit circle, the others inside sigma; with the line search every
    accepted step lowers the energy, so a run of k + 1 iterations ends below a run of k."""
    n = 80
    pos = synth.arcsine_disk(n, 9)
    p0, f = oracle.border_split(pos, 12, 0.95)
    energies = []
    for k in [0, 5, 10, 20, 40]:
        x, it, rms, _ = oracle.lbfgsb(p0, max_iter=k, step0=1e-3, maxstep=0.05, radius=0.95, flags=f,
                                      line_search=20)
        r = np.hypot(x[:, 0], x[:, 1])
        assert np.all(np.abs(r[f == 1] - 1.0) <= 4.5e-16)
        assert np.all(r[f == 0] <= 0.95 * (1 + 1e-15))
        energies.append(oracle.energy(x))
    assert all(b < a for a, b in zip(energies, energies[1:]))


def test_subdomain_lbfgsb_of_every_charge_is_the_instance():
    """A subdomain holding every charge (E_sub gradient, pairwise energy change against the
    snapshot) runs the same iteration as the whole-configuration L-BFGS-B."""
    pos = synth.arcsine_disk(90, 4)
    a = oracle.subdomain_lbfgsb(pos, np.arange(90), memory=6, steps=40, step0=1e-3, maxstep=0.05, line_search=5)
    b, _, _, _ = oracle.lbfgsb(pos, memory=6, max_iter=40, step0=1e-3, maxstep=0.05, line_search=5)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)


@pytest.mark.parametrize("case", ["ring_two", "ring_three", "wall"])
def test_subdomain_lbfgsb_single_charge_reaches_the_constrained_minimum(case):
    """One moving charge against fixed ones: L-BFGS-B on (t, u) ends at the minimiser of its own
    energy sum_j 1/|x - s_j| over |x| <= sigma that scipy's SLSQP finds in Cartesian coordinates from
    the same start (interior minima, and one on the wall |x| = sigma, where t = pi/2 is active)."""
    from scipy.optimize import minimize

    ang = 2 * np.pi * np.arange(12) / 12
    ring = np.stack([np.cos(ang), np.sin(ang)], 1)
    bg, start = {
        "ring_two": (np.vstack([ring, [[0.0, 0.45], [0.0, -0.45]]]), [0.5, 0.12]),
        "ring_three": (np.vstack([ring, [[0.0, 0.45], [0.0, -0.45], [-0.5, 0.0]]]), [0.45, 0.1]),
        "wall": (np.array([[0.1, 0.05], [0.05, -0.1], [-0.1, 0.02], [0.3, 0.25]]), [0.5, 0.3]),
    }[case]
    snap = np.vstack([bg, [start]])
    k = snap.shape[0] - 1
    act = oracle.subdomain_lbfgsb(snap, [k], memory=5, steps=300, step0=1e-3, maxstep=0.05, radius=0.9)[0]
    energy = lambda x: sum(1.0 / math.hypot(x[0] - s[0], x[1] - s[1]) for s in bg)
    ref = minimize(energy, np.array(start), method="SLSQP", constraints=[{"type": "ineq", "fun": lambda x: 0.81 - x @ x}],
                   options={"ftol": 1e-16, "maxiter": 1000}).x
    np.testing.assert_allclose(act, ref, rtol=0, atol=1e-7)
    if case == "wall":
        assert abs(math.hypot(*act) - 0.9) <= 1e-15


def test_cycle_with_lbfgsb_zones_keeps_its_bookkeeping():
    """The cycle with L-BFGS-B per zone: E_{b+1} - E_b is the sum of batch b's accepted energy changes,
    the energy never rises, pinned charges stay on the circle and free ones inside the final sigma."""
    n = 1200
    pos = synth.arcsine_disk(n, 21)
    s0 = 1 - 1 / (2 * math.sqrt(n))
    p0, f = oracle.border_split(pos, oracle.boundary_count(n), s0)
    u = np.random.default_rng(22).random((9, 3))
    p, trace, d, acc = oracle.cycle(p0, u, m_min=20, m_max=150, period=4, batch=3, step0=1e-4, alpha_min=0.0,
                                    alpha_max=0.0, steps=12, sigma0=s0, sigma1=1.0, flags=f, optimizer="lbfgsb_tu",
                                    memory=6, maxstep=0.02, line_search=4)
    assert np.all(np.diff(trace) <= 0)
    for b in range(3):
        sl = slice(3 * b, 3 * b + 3)
        assert abs((trace[b + 1] - trace[b]) - d[sl][acc[sl] == 1].sum()) <= 1e-12 * trace[b]
    r = np.hypot(p[:, 0], p[:, 1])
    assert np.all(np.abs(r[f == 1] - 1.0) <= 4.5e-16)
    assert np.all(r[f == 0] <= 1.0 + 1e-15)
    assert (acc == 1).sum() >= 3


@pytest.mark.parametrize("opt", ["lbfgsb_tu", "bb"])
def test_cycle_is_its_steps_in_order(opt):
    """With one zone per batch, the cycle is: local energies, the zone of batch b at sigma_b, the zone
    optimiser (L-BFGS-B or projected BB) against the rest, the float64 accept; rebuilt here from
    those oracle pieces."""
    n = 400
    eta = 1e-4 / n
    pos = synth.arcsine_disk(n, 31)
    s0 = 1 - 1 / (2 * math.sqrt(n))
    p0, f = oracle.border_split(pos, oracle.boundary_count(n), s0)
    u = np.random.default_rng(32).random((5, 3))
    kw = dict(m_min=10, m_max=60, period=4)
    step0 = 1e-4 if opt == "lbfgsb_tu" else eta
    p, trace, d, acc = oracle.cycle(p0, u, batch=1, step0=step0, alpha_min=0.0, alpha_max=10 * eta, steps=6,
                                    sigma0=s0, sigma1=1.0, flags=f, optimizer=opt, memory=5,
                                    maxstep=0.02, line_search=3, **kw)
    q = p0.copy()
    for b in range(5):
        radius = oracle.sigma_ramp(s0, 1.0, b, 5)
        e_tot, e_loc = oracle.energy(q, local=True)
        assert trace[b] == e_tot
        idx, off, _, _ = oracle.zone_select(q, e_loc, u[b:b + 1], phase=b, radius=radius, flags=f, **kw)
        if opt == "lbfgsb_tu":
            act = oracle.subdomain_lbfgsb(q, idx, memory=5, steps=6, step0=step0, maxstep=0.02, radius=radius,
                                          flags=f, line_search=3)
        else:
            act = oracle.subdomain_bb(q, idx, step0, 0.0, 10 * eta, 6, radius=radius, flags=f)
        q, db, ab = oracle.accept_sequential(q, idx, off, act)
        assert db[0] == d[b] and ab[0] == acc[b]
    np.testing.assert_array_equal(p, q)
    assert trace[5] == oracle.energy(q)
    assert (acc == 1).sum() >= 3  # the zones really move


def _tu_to_x(z, sigma, f):
    t, u = z[:, 0], z[:, 1]
    r = np.where(f == 1, 1.0, sigma * np.sin(t) ** 2)
    ang = np.where(f == 1, z[:, 0], u)
    return np.stack([r * np.cos(ang), r * np.sin(ang)], 1)


def _smooth_to_x(z, sigma, f):
    rho = np.hypot(z[:, 0], z[:, 1])
    scale = np.where(f == 1, 1.0 / rho, sigma * np.sin(rho) / rho)
    return z * scale[:, None]


@pytest.mark.parametrize("tu", [False, True])
def test_first_lbfgs_step_follows_the_maps_gradient(tu):
    """Without history the first L-BFGS step is z - step0 dE/dz.  dE/dz is taken here by central
    differences of E(x(z)) over the map's own variables (Sec. II D's r = sigma sin^2 t, u; pinned
    charges on (cos u, sin u); or the smooth map x = sigma sin|z| z/|z|), so every term of the chain
    rule is checked, pinned charges included."""
    n, sigma = 30, 0.9
    pos = synth.arcsine_disk(n, 41)
    p0, f = oracle.border_split(pos, 6, sigma)
    r = np.hypot(p0[:, 0], p0[:, 1])
    if tu:
        z0 = np.stack([np.where(f == 1, np.arctan2(p0[:, 1], p0[:, 0]), np.arcsin(np.sqrt(np.minimum(r / sigma, 1)))),
                       np.where(f == 1, 0.0, np.arctan2(p0[:, 1], p0[:, 0]))], 1)
        to_x = _tu_to_x
    else:
        k = np.where(f == 1, 1.0, np.arcsin(np.minimum(r / sigma, 1)) / r)
        z0 = p0 * k[:, None]
        to_x = _smooth_to_x
    h = 1e-6
    gz = np.zeros_like(z0)
    for i in range(n):
        for c in range(2):
            if tu and f[i] == 1 and c == 1:
                continue  # the unused second variable of a pinned charge
            zp, zm = z0.copy(), z0.copy()
            zp[i, c] += h
            zm[i, c] -= h
            gz[i, c] = (oracle.energy(to_x(zp, sigma, f)) - oracle.energy(to_x(zm, sigma, f))) / (2 * h)
    step0 = 1e-6
    x1, _, _ = oracle.lbfgs(p0, memory=4, max_iter=1, step0=step0, maxstep=10.0, radius=sigma, flags=f, tu=tu)
    expect = to_x(z0 - step0 * gz, sigma, f)
    moved = np.abs(x1 - p0).max()
    assert moved > 1e-6
    assert np.abs(x1 - expect).max() <= 1e-5 * moved


def test_lbfgsb_reports_the_projected_gradient_rms():
    """L-BFGS-B's stop measure at the start point: RMS over charges of P(v - g) - v on the box
    t in [0, pi/2] (pinned charges: u free, second variable fixed), g by central differences of
    E(x(t, u)).  The gradients are large, so for most charges t - g_t falls outside the box and the
    projection decides the measure."""
    n, sigma = 40, 0.9
    pos = synth.arcsine_disk(n, 43)
    p0, f = oracle.border_split(pos, 7, sigma)
    r = np.hypot(p0[:, 0], p0[:, 1])
    ang = np.arctan2(p0[:, 1], p0[:, 0])
    z0 = np.stack([np.where(f == 1, ang, np.arcsin(np.sqrt(np.minimum(r / sigma, 1)))), np.where(f == 1, 0.0, ang)], 1)
    h = 1e-6
    g = np.zeros_like(z0)
    for i in range(n):
        for c in range(2 if f[i] == 0 else 1):
            zp, zm = z0.copy(), z0.copy()
            zp[i, c] += h
            zm[i, c] -= h
            g[i, c] = (oracle.energy(_tu_to_x(zp, sigma, f)) - oracle.energy(_tu_to_x(zm, sigma, f))) / (2 * h)
    lo = np.where(f[:, None] == 1, [-np.inf, 0.0], [0.0, -np.inf])
    hi = np.where(f[:, None] == 1, [np.inf, 0.0], [math.pi / 2, np.inf])
    pg = np.clip(z0 - g, lo, hi) - z0
    expect = math.sqrt((pg ** 2).sum() / n)
    assert (np.abs(np.clip(z0 - g, lo, hi) - (z0 - g)) > 1.0).any(1).sum() >= 10  # the box acts
    _, it, rms, _ = oracle.lbfgsb(p0, max_iter=0, radius=sigma, flags=f)
    assert it == 0
    assert abs(rms - expect) <= 1e-6 * expect


def _dense_inverse_bfgs(pairs, gamma, L):
    """H (L x L) after the BFGS inverse updates H <- V^T H V + rho s s^T (V = I - rho y s^T) of
    gamma I, oldest pair first (Nocedal & Wright, Eq. 6.17 and Sec. 7.2)."""
    H = gamma * np.eye(L)
    for s_, y_ in pairs:
        rho = 1.0 / (s_ @ y_)
        V = np.eye(L) - rho * np.outer(y_, s_)
        H = V.T @ H @ V + rho * np.outer(s_, s_)
    return H


LBFGS_PATHS = [
    # (n, seed, memory, iterations, step0, maxstep, tu, pinned, radius): 25-30 iterations with memory
    # 3-4 wrap the pair ring many times; the first and last cases skip pairs (s.y <= 1e-12 |s||y|)
    (10, 0, 3, 25, 1e-3, 0.3, False, 0, 1.0),
    (10, 5, 3, 25, 1e-3, 0.3, True, 0, 1.0),
    (10, 3, 3, 25, 1e-3, 0.3, False, 0, 1.0),
    (14, 8, 4, 30, 1e-3, 0.2, False, 4, 0.95),
    (14, 8, 4, 30, 1e-3, 0.2, True, 4, 0.95),
]


@pytest.mark.parametrize("n,seed,memory,iters,step0,maxstep,tu,pinned,radius", LBFGS_PATHS)
def test_lbfgs_direction_is_the_dense_inverse_bfgs_product(n, seed, memory, iters, step0, maxstep, tu, pinned,
                                                          radius):
    """The L-BFGS iteration (two-loop recursion with a ring of `memory` pairs) against the matrix it
    stands for: at every iterate the direction equals -H g, H built densely from gamma I by the
    BFGS inverse updates of the last `memory` kept pairs (gamma = s.y / y.y of the newest pair,
    step0 without pairs); the step scale is min(1, maxstep / max_i |d_i|); z moves by alpha d; a
    pair enters the ring iff s.y > 1e-12 |s||y|.  The pairs and gradients come from the recorded
    path, the chain rule of dE/dz being pinned on its own by the central-difference tests above.
    Gamma from the oldest pair, the loops walked in the wrong order or rho of the wrong slot each
    change the direction by O(1) on these paths."""
    x0 = synth.arcsine_disk(n, seed)
    flags = None
    if pinned:
        flags = np.zeros(n, np.uint8)
        flags[np.argsort(-np.linalg.norm(x0, axis=1))[:pinned]] = 1
        x0 = oracle.project(x0, radius, flags)
    xt, Z, Gz, D, A = oracle.lbfgs_trace(x0, memory=memory, max_iter=iters, step0=step0, maxstep=maxstep, tu=tu,
                                         flags=flags, radius=radius)
    assert len(A) == iters
    # recording the path changes nothing: the untraced iteration ends at the same positions
    xl, _, _ = oracle.lbfgs(x0, memory=memory, max_iter=iters, step0=step0, maxstep=maxstep, tu=tu, flags=flags,
                            radius=radius)
    np.testing.assert_array_equal(xt, xl)
    hist, skipped, wrapped = [], 0, 0
    for k in range(iters):
        g = Gz[k]
        gamma = (hist[-1][0] @ hist[-1][1]) / (hist[-1][1] @ hist[-1][1]) if hist else step0
        d = -_dense_inverse_bfgs(hist, gamma, g.size) @ g
        assert g @ d < 0  # every kept pair has s.y > 0, so H is positive definite
        assert np.linalg.norm(d - D[k]) <= 1e-9 * np.linalg.norm(d), k
        dmax = np.sqrt(d[0::2] ** 2 + d[1::2] ** 2).max()
        alpha = maxstep / dmax if dmax > maxstep else 1.0
        assert abs(A[k] - alpha) <= 1e-9 * alpha
        s_, y_ = Z[k + 1] - Z[k], Gz[k + 1] - Gz[k]
        assert np.abs(s_ - A[k] * D[k]).max() <= 1e-13 * (1.0 + np.abs(Z[k]).max())
        if s_ @ y_ > 1e-12 * np.linalg.norm(s_) * np.linalg.norm(y_):
            wrapped += len(hist) == memory
            hist = (hist + [(s_, y_)])[-memory:]
        else:
            skipped += 1
    assert wrapped >= 5  # the ring was full and overwrote its oldest pair several times
    if (seed, tu) in ((0, False), (5, True), (3, False)):
        assert skipped >= 1


def test_disjoint_cycle_is_its_steps_in_order():
    """The disjoint batch rule, rebuilt from the oracle's pieces: at each batch start the local
    energies, the zones of the next `batch` subdomains at sigma(b0) = s0 + (1 - s0) b0 / (n_sub - 1),
    their longest prefix of pairwise disjoint zones (set intersections here), each prefix zone
    relaxed against the batch-start configuration, the float64 accept in order.  No zone is skipped,
    every subdomain is optimised, and at least one batch is cut short by an overlap."""
    n = 600
    eta = 1e-4 / n
    pos = synth.arcsine_disk(n, 41)
    s0 = 1 - 1 / (2 * math.sqrt(n))
    p0, f = oracle.border_split(pos, oracle.boundary_count(n), s0)
    n_sub, cap = 12, 4
    u = np.random.default_rng(42).random((n_sub, 3))
    kw = dict(m_min=15, m_max=90, period=5)
    p, trace, d, acc = oracle.cycle(p0, u, batch=cap, step0=eta, alpha_min=0.0, alpha_max=10 * eta, steps=5,
                                    sigma0=s0, sigma1=1.0, flags=f, disjoint=True, **kw)
    q = p0.copy()
    b0, b, cut = 0, 0, 0
    while b0 < n_sub:
        k = min(cap, n_sub - b0)
        radius = s0 + (1.0 - s0) * b0 / (n_sub - 1)
        e_tot, e_loc = oracle.energy(q, local=True)
        assert trace[b] == e_tot
        idx, off, _, _ = oracle.zone_select(q, e_loc, u[b0:b0 + k], phase=b0, radius=radius, flags=f, **kw)
        zones = [set(idx[off[s]:off[s + 1]].tolist()) for s in range(k)]
        kk = 1
        while kk < k and all(not (zones[kk] & zones[j]) for j in range(kk)):
            kk += 1
        cut += kk < k
        act = np.concatenate([oracle.subdomain_bb(q, idx[off[s]:off[s + 1]], eta, 0.0, 10 * eta, 5, radius=radius,
                                                  flags=f) for s in range(kk)])
        q, db, ab = oracle.accept_sequential(q, idx[:off[kk]], off[:kk + 1], act)
        np.testing.assert_array_equal(db, d[b0:b0 + kk])
        np.testing.assert_array_equal(ab, acc[b0:b0 + kk])
        b0 += kk
        b += 1
    np.testing.assert_array_equal(p, q)
    assert len(trace) == b + 1 and trace[b] == oracle.energy(q)
    assert cut >= 1 and np.all(acc != 2) and (acc == 1).sum() >= 6


def test_disjoint_cycle_with_batch_one_is_the_plain_cycle():
    """batch = 1 is the paper's one-zone-at-a-time cycle in both forms (the ramp in b0 / (n_sub - 1)
    equals the ramp in b / (n_batches - 1) there)."""
    n = 300
    eta = 1e-4 / n
    pos = synth.arcsine_disk(n, 43)
    u = np.random.default_rng(44).random((6, 3))
    kw = dict(m_min=10, m_max=50, period=3, batch=1, step0=eta, alpha_min=0.0, alpha_max=10 * eta, steps=4,
              sigma0=0.97, sigma1=1.0)
    a = oracle.cycle(oracle.project(pos, 0.97), u, **kw)
    b = oracle.cycle(oracle.project(pos, 0.97), u, disjoint=True, **kw)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
