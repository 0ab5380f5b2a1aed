"""ctypes binding of libtc.so (argument marshalling only).

The shared library is built in-tree by paper_2609_24722_b300/build.py.  There
is no fallback: if libtc.so is missing or fails to load, every call raises.
"""

from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtc.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "tc.h")

TC_OK = 0
TC_FP64 = 0
TC_MIXED = 1
TC_F64X = 2
TC_OPT_GD, TC_OPT_BB, TC_OPT_LBFGS, TC_OPT_LBFGS_TU, TC_OPT_LBFGSB_TU = 0, 1, 2, 3, 4
STATUS_NAMES = {0: "TC_OK", 1: "TC_ERR_INVALID_ARG", 2: "TC_ERR_CUDA", 3: "TC_ERR_NONFINITE",
                4: "TC_ERR_OUTSIDE_DISK", 5: "TC_ERR_TIMEOUT", 6: "TC_ERR_NOT_CONVERGED", 7: "TC_ERR_NO_MEMORY"}


class TCError(RuntimeError):
    """A libtc call returned a non-zero tc_status."""

    def __init__(self, code: int, what: str):
        msg = _lib().tc_status_string(code).decode() if _LIB is not None else STATUS_NAMES.get(code, str(code))
        detail = ""
        if code == 2 and _LIB is not None:
            detail = " -- " + _lib().tc_last_error().decode()
        super().__init__(f"{what}: {STATUS_NAMES.get(code, code)} ({msg}){detail}")
        self.code = code


class RelaxParams(C.Structure):
    """tc_relax_params of include/tc.h."""

    _fields_ = [
        ("precision", C.c_int32),
        ("optimizer", C.c_int32),
        ("n_steps", C.c_int32),
        ("memory", C.c_int32),
        ("step0", C.c_double),
        ("alpha_min", C.c_double),
        ("alpha_max", C.c_double),
        ("maxstep", C.c_double),
        ("gtol", C.c_double),
        ("radius", C.c_double),
        ("polish_steps", C.c_int32),
        ("accept", C.c_int32),
        ("polish_gtol", C.c_double),
        ("want_energy", C.c_int32),
        ("profile", C.c_int32),
        ("polish_precision", C.c_int32),
        ("line_search", C.c_int32),
    ]


class RelaxProfile(C.Structure):
    """tc_relax_profile of include/tc.h."""

    _fields_ = [
        ("pass_ms", C.c_double),
        ("update_ms", C.c_double),
        ("relax_ms", C.c_double),
        ("accept_ms", C.c_double),
        ("setup_ms", C.c_double),
        ("n_pass", C.c_int32),
        ("launches", C.c_int32),
        ("pass_pairs", C.c_int64),
    ]


class ZoneParams(C.Structure):
    """tc_zone_params of include/tc.h."""

    _fields_ = [
        ("kappa", C.c_double),
        ("p_defect", C.c_double),
        ("radius", C.c_double),
        ("wall_tol", C.c_double),
        ("m_min", C.c_int32),
        ("m_max", C.c_int32),
        ("period", C.c_int32),
        ("phase", C.c_int32),
    ]


class CycleParams(C.Structure):
    """tc_cycle_params of include/tc.h."""

    _fields_ = [
        ("zone", ZoneParams),
        ("relax", RelaxParams),
        ("batch", C.c_int32),
        ("local_precision", C.c_int32),
        ("sigma0", C.c_double),
        ("sigma1", C.c_double),
        ("disjoint", C.c_int32),
        ("ramp_first", C.c_int32),
        ("ramp_total", C.c_int32),
    ]


RESULT_BYTES = 32  # sizeof(tc_subdomain_result): 3 double + 2 int32

_LIB = None


def _lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libtc.so is not built ({LIB_PATH}); run paper_2609_24722_b300/build.py")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        sigs = {
            "tc_energy": ([vp, i64, i32, vp, vp, vp], C.c_int),
            "tc_grad": ([vp, i64, i32, vp, vp, vp], C.c_int),
            "tc_energy_noalloc": ([vp, i64, i32, vp, vp, vp], C.c_int),
            "tc_subdomain_delta_energy": ([vp, i64, vp, vp, i32, vp, vp, vp], C.c_int),
            "tc_subdomain_delta_energy_mixed": ([vp, i64, vp, vp, i32, vp, vp, vp, vp], C.c_int),
            "tc_subdomain_grad": ([vp, i64, vp, vp, i32, vp, i32, vp, vp, vp, vp], C.c_int),
            "tc_relax_subdomains": ([vp, i64, vp, vp, i32, vp, vp, C.POINTER(RelaxParams), vp, vp], C.c_int),
            "tc_project_disk": ([vp, i64, d, vp, vp], C.c_int),
            "tc_status_string": ([C.c_int], C.c_char_p),
            "tc_last_error": ([], C.c_char_p),
            "tc_pass_config_count": ([i32], C.c_int32),
            "tc_set_pass_config": ([i32, i32], C.c_int),
            "tc_get_pass_config": ([i32], C.c_int32),
            "tc_sync_status": ([vp], C.c_int),
            "tc_shutdown": ([], None),
            "tc_probe_pipes": ([vp, vp], C.c_int),
            "tc_relax_last_profile": ([C.POINTER(RelaxProfile)], C.c_int),
            "tc_zone_offsets": ([C.POINTER(ZoneParams), i64, i32, vp], C.c_int),
            "tc_select_subdomains": ([vp, i64, vp, vp, C.POINTER(ZoneParams), i32, vp, vp, vp, vp, vp, vp],
                                     C.c_int),
            "tc_cycle": ([vp, i64, vp, C.POINTER(CycleParams), i32, vp, vp, vp, vp], C.c_int),
            "tc_boundary_count": ([i64], i64),
            "tc_voronoi_order": ([vp, i64, vp, vp, vp, i32, vp, vp], C.c_int),
            "tc_border_split": ([vp, i64, i64, d, vp, vp], C.c_int),
        }
        for name, (args, res) in sigs.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _LIB = L
    return _LIB


def lib() -> C.CDLL:
    return _lib()


def check(code: int, what: str) -> None:
    if code != TC_OK:
        raise TCError(code, what)


def declared_functions() -> list[str]:
    """Names of the functions include/tc.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tc_[a-z0-9_]+)\s*\(", text)))
