"""Checkpoint and resume of the adaptive cycle (paper_2609_24722_b300/checkpoint.py).

Host logic on the CPU with a stand-in for the cycle call (deterministic, records its arguments);
the GPU test runs the real cycle.  A run interrupted after any call and resumed from its checkpoint
must end bit for bit where the uninterrupted run ends."""

from __future__ import annotations

import os
from dataclasses import dataclass

import numpy as np
import pytest
import torch

from paper_2609_24722_b300 import checkpoint as ck


@dataclass
class _R:
    delta_e: torch.Tensor
    energy: torch.Tensor
    rms: torch.Tensor
    steps: torch.Tensor
    status: torch.Tensor


class FakeCycle:
    """Moves every charge by a function of the call's uniforms and records the call arguments."""

    def __init__(self):
        self.calls = []

    def __call__(self, pos, uniforms, flags, *, phase, ramp_first, ramp_total, **kw):
        self.calls.append((phase, ramp_first, ramp_total, uniforms.shape[0]))
        k = uniforms.shape[0]
        e0 = float((pos ** 2).sum())
        pos.mul_(0.999).add_(1e-3 * uniforms.sum() * torch.ones_like(pos) / pos.shape[0])
        e1 = float((pos ** 2).sum())
        r = _R(uniforms[:, 0].double() - 0.5, uniforms[:, 1].double(), uniforms[:, 2].double(),
               torch.full((k,), 7, dtype=torch.int32), (uniforms[:, 0] > 0.5).int())
        return r, torch.tensor([e0, e1], dtype=torch.float64)


def _inputs(n=50, n_sub=11, seed=0):
    g = np.random.default_rng(seed)
    return torch.tensor(g.uniform(-0.5, 0.5, (n, 2))), torch.tensor(g.random((n_sub, 3)))


def test_interrupt_and_resume_equal_the_uninterrupted_run(tmp_path):
    kw = dict(batch=2, m_min=3, m_max=9, period=4, phase=5)
    pos0, u = _inputs()
    pa = pos0.clone()
    fa = FakeCycle()
    ra, ta, da = ck.run_cycle(pa, u, None, chunk=4, path=str(tmp_path / "a.npz"), cycle_fn=fa, **kw)
    assert da == 11
    assert fa.calls == [(5, 0, 11, 4), (9, 4, 11, 4), (13, 8, 11, 3)]
    assert len(ta) == 3 + 1  # one energy before each call and after the last
    pb = pos0.clone()
    path = str(tmp_path / "b.npz")
    _, _, db = ck.run_cycle(pb, u, None, chunk=4, path=path, stop_after=1, cycle_fn=FakeCycle(), **kw)
    assert db == 4 and os.path.exists(path)
    pb.fill_(123.0)  # whatever the process holds is replaced by the checkpoint on resume
    fb = FakeCycle()
    rb, tb, db = ck.run_cycle(pb, u, None, chunk=4, path=path, cycle_fn=fb, **kw)
    assert db == 11 and fb.calls == [(9, 4, 11, 4), (13, 8, 11, 3)]
    assert torch.equal(pa, pb)
    np.testing.assert_array_equal(ta, tb)
    for f in ck._FIELDS:
        np.testing.assert_array_equal(ra[f], rb[f])


def test_resume_refuses_another_run(tmp_path):
    kw = dict(batch=2, m_min=3, m_max=9, period=4)
    pos0, u = _inputs()
    path = str(tmp_path / "c.npz")
    ck.run_cycle(pos0.clone(), u, None, chunk=4, path=path, stop_after=1, cycle_fn=FakeCycle(), **kw)
    with pytest.raises(ValueError):
        ck.run_cycle(pos0.clone(), u + 0.0 * u + 1e-9, None, chunk=4, path=path, cycle_fn=FakeCycle(), **kw)
    with pytest.raises(ValueError):
        ck.run_cycle(pos0.clone(), u, None, chunk=4, path=path, cycle_fn=FakeCycle(), **{**kw, "m_max": 10})
    with pytest.raises(ValueError):
        ck.run_cycle(pos0.clone(), u, None, chunk=3, path=str(tmp_path / "d.npz"), cycle_fn=FakeCycle(), **kw)


@pytest.mark.gpu
@pytest.mark.parametrize("disjoint", [False, True])
def test_gpu_cycle_interrupted_and_resumed_is_bitwise_the_same(tmp_path, disjoint):
    import synth
    import paper_2609_24722_b300 as tc

    n = 3000
    dev = "cuda:0"
    pos = synth.arcsine_disk(n, 71)
    p0 = torch.tensor(pos, device=dev)
    f0 = tc.border_split(p0)
    u = torch.tensor(np.random.default_rng(72).random((12, 3)), device=dev)
    kw = dict(batch=2, m_min=30, m_max=300, period=5, local_precision="fp64", precision="mixed",
              optimizer="lbfgsb_tu", n_steps=10, memory=6, step0=1e-4, maxstep=0.01, sigma0=0.0, sigma1=1.0,
              disjoint=disjoint)
    pa, fa = p0.clone(), f0.clone()
    ra, ta, _ = ck.run_cycle(pa, u, fa, chunk=4, path=str(tmp_path / "a.npz"), **kw)
    pb, fb = p0.clone(), f0.clone()
    path = str(tmp_path / "b.npz")
    ck.run_cycle(pb, u, fb, chunk=4, path=path, stop_after=2, **kw)
    pb2, fb2 = torch.zeros_like(p0), torch.zeros_like(f0)
    rb, tb, db = ck.run_cycle(pb2, u, fb2, chunk=4, path=path, **kw)
    tc.sync_status()
    assert db == 12
    assert torch.equal(pa, pb2) and torch.equal(fa, fb2)
    np.testing.assert_array_equal(ta, tb)
    for f in ck._FIELDS:
        np.testing.assert_array_equal(ra[f], rb[f])
    assert (ra["status"] == 1).sum() >= 3
