"""The C-ABI library builds for sm_103a, loads without a GPU and exports every declared entry point."""

import ctypes as C

import pytest

from paper_2609_24722_b300 import _lib as L
from paper_2609_24722_b300 import build as B


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def test_exports_every_declared_function(lib):
    names = L.declared_functions()
    assert {"tc_energy", "tc_grad", "tc_subdomain_delta_energy", "tc_relax_subdomains",
            "tc_project_disk"} <= set(names)
    for name in names:
        assert hasattr(lib, name), name


def test_struct_layouts_match_header(lib):
    # tc_relax_params: 4 int32, 6 double, 2 int32, 1 double, 4 int32 -> 96 bytes
    assert C.sizeof(L.RelaxParams) == 96 and L.RelaxParams.polish_precision.offset == 88
    assert L.RelaxParams.line_search.offset == 92
    assert L.RelaxParams.step0.offset == 16 and L.RelaxParams.polish_steps.offset == 64
    assert L.RelaxParams.want_energy.offset == 80
    assert L.RESULT_BYTES == 32
    assert C.sizeof(L.RelaxProfile) == 56
    # tc_zone_params: 4 double, 4 int32; tc_cycle_params: zone, relax, 2 int32
    assert C.sizeof(L.ZoneParams) == 48 and L.ZoneParams.m_min.offset == 32
    assert C.sizeof(L.CycleParams) == 184 and L.CycleParams.relax.offset == 48 and L.CycleParams.batch.offset == 144
    assert L.CycleParams.disjoint.offset == 168 and L.CycleParams.ramp_total.offset == 176
    assert L.CycleParams.sigma0.offset == 152


def test_status_strings(lib):
    for code in range(8):
        s = lib.tc_status_string(code)
        assert isinstance(s, bytes) and len(s) > 0
    assert lib.tc_status_string(0) == b"ok"


def test_argument_errors_are_synchronous_without_touching_a_device(lib):
    # invalid arguments are rejected on the host before any CUDA call
    assert lib.tc_energy(None, 10, 0, None, None, None) == 1
    assert lib.tc_grad(None, 10, 0, None, None, None) == 1
    assert lib.tc_project_disk(None, 10, 1.0, None, None) == 1
    assert lib.tc_project_disk(None, 0, -1.0, None, None) == 1
    prm = L.RelaxParams(precision=7)
    assert lib.tc_relax_subdomains(None, 10, None, None, 1, None, None, C.byref(prm), None, None) == 1
    z = L.ZoneParams(kappa=-1.0, p_defect=0.8, radius=1.0, wall_tol=1e-9, m_min=5, m_max=3, period=4)
    assert lib.tc_select_subdomains(None, 10, None, None, C.byref(z), 1, None, None, None, None, None, None) == 1
    cp = L.CycleParams(zone=z, batch=0)
    assert lib.tc_cycle(None, 10, None, C.byref(cp), 1, None, None, None, None) == 1
    z.m_max = 7
    cp = L.CycleParams(zone=z, batch=1, sigma0=0.5, sigma1=0.4)  # sigma must not fall
    assert lib.tc_cycle(None, 10, None, C.byref(cp), 1, None, None, None, None) == 1
    assert lib.tc_border_split(None, 10, 11, 0.9, None, None) == 1  # n_b > n
    # L-BFGS-B keeps at most 8 pairs; an optimizer past the last is rejected
    ok = dict(precision=0, n_steps=1, memory=8, step0=1e-3, maxstep=0.01, radius=1.0)
    prm = L.RelaxParams(optimizer=L.TC_OPT_LBFGSB_TU, **{**ok, "memory": 9})
    assert lib.tc_relax_subdomains(None, 10, None, None, 1, None, None, C.byref(prm), None, None) == 1
    prm = L.RelaxParams(optimizer=L.TC_OPT_LBFGSB_TU + 1, **ok)
    assert lib.tc_relax_subdomains(None, 10, None, None, 1, None, None, C.byref(prm), None, None) == 1


def test_enum_values_match_header():
    """Every enumerator that the binding names has the header's value."""
    import os
    import re

    hdr = open(os.path.join(os.path.dirname(L.__file__), "..", "include", "tc.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    values = {}
    for body in re.findall(r"typedef enum\s*\{(.*?)\}", hdr, flags=re.S):
        for name, val in re.findall(r"(TC_[A-Z0-9_]+)\s*=\s*(\d+)", body):
            values[name] = int(val)
    named = {k: getattr(L, k) for k in dir(L) if k.startswith("TC_") and isinstance(getattr(L, k), int)}
    assert {"TC_OPT_LBFGSB_TU", "TC_F64X", "TC_MIXED"} <= set(named)
    for k, v in named.items():
        assert k in values and values[k] == v, k


def test_boundary_count_host_only_matches_oracle(lib):
    """Eq. Nb on the host: the library's N_b equals the oracle's for every n up to 3000 and at 1e5."""
    import oracle

    for n in list(range(0, 3001)) + [12345, 100000, 10 ** 7]:
        assert lib.tc_boundary_count(n) == oracle.boundary_count(n)
    assert lib.tc_boundary_count(100000) == 6099


def test_zone_offsets_host_only_matches_oracle(lib):
    """tc_zone_offsets is host logic: the zone-size schedule equals the oracle's on every position."""
    import oracle

    for (m_min, m_max, period, phase, n) in [(50, 200, 4, 0, 1000), (200, 5000, 7, 3, 100000), (0, 9, 1, 5, 20),
                                             (10, 400, 10, 0, 300), (3, 3, 2, 1, 2)]:
        z = L.ZoneParams(kappa=-1.0, p_defect=0.8, radius=1.0, wall_tol=1e-9, m_min=m_min, m_max=m_max,
                         period=period, phase=phase)
        ns = 23
        off = (C.c_int64 * (ns + 1))()
        assert lib.tc_zone_offsets(C.byref(z), n, ns, C.cast(off, C.c_void_p)) == 0
        sizes = [off[s + 1] - off[s] for s in range(ns)]
        assert off[0] == 0
        assert sizes == [oracle.zone_size(phase + s, m_min, m_max, period, n) for s in range(ns)]
    bad = L.ZoneParams(kappa=-1.0, p_defect=1.5, radius=1.0, wall_tol=0.0, m_min=1, m_max=2, period=1)
    off = (C.c_int64 * 2)()
    assert lib.tc_zone_offsets(C.byref(bad), 10, 1, C.cast(off, C.c_void_p)) == 1


def test_stream_k_owner_formula():
    """owner(u) = ceil(G (u+1) / W) - 1 is the CTA whose range [floor(W k/G), floor(W (k+1)/G)) holds u."""
    for W in [1, 2, 7, 100, 391, 1000, 76636]:
        for G in [1, 2, 3, 148, 296, 592, 1184]:
            if G > W:
                continue
            b = [(W * k) // G for k in range(G + 1)]
            k = 0
            for u in range(0, W, max(1, W // 997)):
                while not (b[k] <= u < b[k + 1]):
                    k += 1 if b[k + 1] <= u else -1
                assert (G * (u + 1) + W - 1) // W - 1 == k
