"""Seeded synthetic inputs: shape, determinism and distribution checks."""

import math

import numpy as np
from scipy import stats

import synth


def test_arcsine_radii_follow_the_arcsine_cdf():
    pos = synth.arcsine_disk(20000, 0)
    r = np.linalg.norm(pos, axis=1)
    assert r.max() <= 1.0
    # radial CDF of rho ~ 1/sqrt(1 - r^2) over the disk: F(r) = 1 - sqrt(1 - r^2)
    d, p = stats.kstest(r, lambda x: 1.0 - np.sqrt(1.0 - np.clip(x, 0, 1) ** 2))
    assert p > 1e-3
    th = np.arctan2(pos[:, 1], pos[:, 0])
    assert stats.kstest((th + math.pi) / (2 * math.pi), "uniform").pvalue > 1e-3


def test_determinism():
    np.testing.assert_array_equal(synth.arcsine_disk(1000, 3), synth.arcsine_disk(1000, 3))
    assert not np.array_equal(synth.arcsine_disk(1000, 3), synth.arcsine_disk(1000, 4))
    a = synth.lattice_disk(5000, 2)
    np.testing.assert_array_equal(a, synth.lattice_disk(5000, 2))


def test_lattice_background():
    n = 20000
    pos = synth.lattice_disk(n, 0)
    assert pos.shape == (n, 2)
    assert np.linalg.norm(pos, axis=1).max() <= 1.0
    assert synth.min_pair_distance(pos) > 0.0
    r = np.linalg.norm(pos, axis=1)
    # the radial map carries the lattice onto the arcsine CDF (up to lattice discreteness)
    d, _ = stats.kstest(r, lambda x: 1.0 - np.sqrt(1.0 - np.clip(x, 0, 1) ** 2))
    assert d < 0.01


def test_jitter_stays_inside_and_keeps_shape():
    pos = synth.ngon(64)
    out = synth.jitter_inside(pos, 1e-3, 5)
    assert np.linalg.norm(out, axis=1).max() <= 1.0
    assert np.abs(out - pos).max() < 1e-2


def test_subdomains_and_csr():
    pos = synth.lattice_disk(10000, 1)
    subs = synth.subdomains(pos, 20, 200, 500, 2)
    for s in subs:
        assert 200 <= s.size <= 500
        assert np.all(np.diff(s) > 0) and s[0] >= 0 and s[-1] < 10000
    idx, off = synth.to_csr(subs)
    assert off[0] == 0 and off[-1] == idx.size and idx.dtype == np.int32


def test_instances():
    pos, off = synth.instances(16, 100, 500, 3)
    sizes = np.diff(off)
    assert sizes.min() >= 100 and sizes.max() <= 500
    assert pos.shape == (off[-1], 2)
    np.testing.assert_array_equal(pos[off[2]:off[3]], synth.arcsine_disk(int(sizes[2]), 3 + 1 + 2))


def test_zorder_is_a_spatially_local_permutation():
    pos = synth.arcsine_disk(50000, 4)
    o = synth.zorder(pos)
    assert np.array_equal(np.sort(o), np.arange(pos.shape[0]))
    p = pos[o]
    # consecutive charges in Z-order are far closer than consecutive charges in random order
    step_z = np.linalg.norm(np.diff(p, axis=0), axis=1).mean()
    step_r = np.linalg.norm(np.diff(pos, axis=0), axis=1).mean()
    assert step_z < 0.05 * step_r
    # blocks of 512 consecutive charges are compact
    ext = max(np.ptp(p[k:k + 512], axis=0).max() for k in range(0, 50000 - 512, 512))
    assert ext < 0.6


def test_disjoint_subdomains_are_disjoint_and_fill_the_share():
    pos = synth.lattice_disk(20000, 1)
    subs = synth.disjoint_subdomains(pos, 64, 200, 5000, 3)
    allidx = np.concatenate(subs)
    assert len(np.unique(allidx)) == allidx.size
    assert 0.85 * 20000 <= allidx.size <= 0.9 * 20000
    for s in subs:
        assert s.dtype == np.int32 and np.all(np.diff(s) > 0)
    # the first subdomain is the nearest-charge ball around its centre (nothing was taken before it)
    first = subs[0]
    c = pos[first].mean(0)
    r_in = np.linalg.norm(pos[first] - c, axis=1).max()
    others = np.setdiff1d(np.arange(20000), first)
    assert np.linalg.norm(pos[others] - c, axis=1).min() > 0.5 * r_in
