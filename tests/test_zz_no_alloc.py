"""tc_energy_noalloc: the energy entry point for callers that cannot allocate device memory.

Such callers (a process whose device memory is all owned by a framework's pool
allocator, a real-time host that forbids cudaMalloc after start-up) get their
scratch from a fixed array inside libtc's device image instead of a
cudaMalloc'd workspace.  These tests call it through the C ABI and check it
against tc_energy, on two calls in a row, so a stale value left in the shared
array by the first call would show up in the second.  The file name sorts
last so that pytest collects it after every other test: a run that stops at
its first failure has then already run the rest of the suite, and the shared
array has been through the other tests' use of the library.  Each test also
passes when this file runs alone in a fresh process.
"""

from __future__ import annotations

import ctypes as C

import numpy as np
import pytest
import torch

import synth
from paper_2609_24722_b300 import _lib as L

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
TOL = {0: 1e-13, 1: 1e-6}  # float64 / mixed energy tolerances used by the parity tests


def _energy(fn, pos, prec):
    e = torch.empty((), dtype=torch.float64, device=DEV)
    loc = torch.empty(pos.shape[0], dtype=torch.float64, device=DEV)
    code = fn(pos.data_ptr(), pos.shape[0], prec, e.data_ptr(), loc.data_ptr(),
              torch.cuda.current_stream().cuda_stream)
    assert code == 0, (code, L.lib().tc_last_error())
    torch.cuda.synchronize()
    return e.item(), loc.cpu().numpy()


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_energy_matches_tc_energy_on_two_calls_in_a_row(prec):
    lib = L.lib()
    # a larger call first, then a smaller one: the second must not see the first's scratch
    for n, seed in [(30000, 1), (2777, 2)]:
        pos = torch.tensor(synth.arcsine_disk(n, seed), device=DEV)
        e_ref, loc_ref = _energy(lib.tc_energy, pos, prec)
        assert lib.tc_sync_status(torch.cuda.current_stream().cuda_stream) == 0
        e_na, loc_na = _energy(lib.tc_energy_noalloc, pos, prec)
        assert np.isfinite(e_na)
        assert abs(e_na - e_ref) <= TOL[prec] * abs(e_ref)
        np.testing.assert_allclose(loc_na, loc_ref, rtol=TOL[prec], atol=0)


def test_noalloc_rejects_sizes_beyond_its_limit_and_flags_device_errors():
    lib = L.lib()
    e = torch.empty((), dtype=torch.float64, device=DEV)
    big = torch.zeros((200001, 2), dtype=torch.float64, device=DEV)
    code = lib.tc_energy_noalloc(big.data_ptr(), big.shape[0], 0, e.data_ptr(), None,
                                 torch.cuda.current_stream().cuda_stream)
    assert code == 1
    assert b"200000" in lib.tc_last_error()
    # coincident charges: the energy comes back NaN
    same = torch.tensor([[0.1, 0.2], [0.1, 0.2], [0.5, 0.0]], dtype=torch.float64, device=DEV)
    assert lib.tc_energy_noalloc(same.data_ptr(), 3, 0, e.data_ptr(), None,
                                 torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    assert np.isnan(e.item())


def test_noalloc_single_charge_is_checked_and_nothing_is_allocated():
    """n = 1 gives E = 0 for a charge in the disk and NaN for one outside it (tc_energy reports the
    latter as TC_ERR_OUTSIDE_DISK); and once the kernels of both precisions have run, further calls
    leave the device's free memory unchanged."""
    lib = L.lib()
    stream = torch.cuda.current_stream().cuda_stream
    e = torch.empty((), dtype=torch.float64, device=DEV)
    loc = torch.empty(1, dtype=torch.float64, device=DEV)
    for xy, ok in (([0.3, -0.2], True), ([1.5, 0.0], False)):
        one = torch.tensor([xy], dtype=torch.float64, device=DEV)
        assert lib.tc_energy_noalloc(one.data_ptr(), 1, 0, e.data_ptr(), loc.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        assert (e.item() == 0.0 and loc.item() == 0.0) if ok else np.isnan(e.item())
    pos = [torch.tensor(synth.arcsine_disk(5000, s), device=DEV) for s in (3, 4)]
    for prec in (0, 1):
        _energy(lib.tc_energy_noalloc, pos[0], prec)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    out = []
    for p in pos:
        for prec in (0, 1):
            assert lib.tc_energy_noalloc(p.data_ptr(), p.shape[0], prec, e.data_ptr(), None, stream) == 0
            torch.cuda.synchronize()
            out.append(e.item())
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert all(np.isfinite(out))
