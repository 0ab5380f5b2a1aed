"""CPU oracle for the charges-in-a-disk hot path (TEST INFRASTRUCTURE ONLY).

Thin ctypes wrapper over oracle/tco.c, a plain single-thread FP64 program with
Neumaier-compensated sums.  Only tests, the smoke check and the benchmark's
CPU-baseline arm use it; the GPU library never imports, links or calls it, and
it shares nothing with the GPU library.

Paper passages followed (Lavrov & Nikonov, Thomson problem in a disk):
  energy          Eq. (hamiltonian) with the hard wall of Eq. (potential)
  grad            its analytic Cartesian gradient (Sec. II C step 4: analytic gradients)
  local energy    Sec. II C step 1
  subdomain_grad  the subdomain objective E_sub of Sec. II D
  delta_energy    E_sub(new) - E_sub(old), summed as pair differences
  project         the hard wall as a projection; pinned boundary charges of Sec. II B
  lbfgs / bb / pgd  projected descent on E (the paper's local optimiser is
                  L-BFGS-B, Sec. II C step 4; see the function docs for the
                  variant written here)
  border_split    the border-interior split of Sec. II B (Eq. Nb, radius sigma)
  zone_select     steps 1-3 of the optimisation cycle of Sec. II C (defect
                  threshold, centre choice) and the zone of step 4
  cycle           the optimisation cycle of Sec. II C, in batches
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_ERR = {1: "invalid argument", 3: "non-finite (coincident charges or NaN)",
        4: "charge outside the disk", 7: "out of memory"}


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what}: {_ERR.get(code, code)} (status {code})")
        self.code = code


_libs: dict = {}


def lib(openmp: bool = False) -> C.CDLL:
    """The plain single-thread build, or (openmp=True) the same source built with OpenMP."""
    if openmp not in _libs:
        path = _build.build(openmp=openmp)
        L = C.CDLL(path)
        d, i64, vp = C.c_double, C.c_int64, C.c_void_p
        sig = {
            "tco_energy": [vp, i64, vp, vp],
            "tco_grad": [vp, i64, vp],
            "tco_rows_grad": [vp, i64, vp, i64, vp, vp],
            "tco_subdomain_grad": [vp, i64, vp, i64, vp, vp, vp, vp],
            "tco_delta_energy": [vp, i64, vp, i64, vp, vp],
            "tco_project": [vp, i64, d, vp],
            "tco_projected_grad": [vp, vp, i64, d, vp, vp, vp, vp],
            "tco_pgd": [vp, i64, d, i64, d, vp, vp],
            "tco_subdomain_bb": [vp, i64, vp, i64, d, d, d, i64, d, vp, vp],
            "tco_accept_sequential": [vp, i64, vp, vp, i64, vp, vp, vp],
            "tco_lbfgs": [vp, i64, i64, i64, d, d, d, d, vp, vp, vp],
            "tco_lbfgs_ls": [vp, i64, i64, i64, d, d, d, d, vp, i64, i64, vp, vp],
            "tco_lbfgs_trace": [vp, i64, i64, i64, d, d, d, d, vp, i64, i64, vp, vp, vp, vp, vp, vp],
            "tco_lbfgsb": [vp, i64, i64, i64, d, d, d, d, vp, i64, vp, vp, vp],
            "tco_lbfgsb_middle": [i64, vp, vp, i64, d, vp],
            "tco_lbfgsb_cauchy": [i64, vp, vp, vp, vp, i64, vp, vp, d, vp, vp, vp, vp],
            "tco_lbfgsb_subspace": [i64, vp, vp, vp, vp, i64, vp, vp, d, vp, vp, vp, vp],
            "tco_threads": [],
            "tco_zone_select": [vp, i64, vp, vp, d, d, d, d, i64, i64, i64, i64, i64, vp, vp, vp, vp, vp],
            "tco_cycle": [vp, i64, vp, d, d, d, d, d, i64, i64, i64, i64, i64, vp, d, d, d, i64, vp, vp, vp],
            "tco_cycle_opt": [vp, i64, vp, d, d, d, d, d, i64, i64, i64, i64, i64, vp, i64, d, d, d, i64, d, i64, i64,
                              vp, vp, vp],
            "tco_subdomain_lbfgsb": [vp, i64, vp, i64, i64, i64, d, d, d, vp, i64, vp],
            "tco_cycle_run": [vp, i64, vp, d, d, d, d, d, i64, i64, i64, i64, i64, i64, vp, i64, d, d, d, i64, d, i64,
                              i64, vp, vp, vp, vp],
            "tco_border_split": [vp, i64, i64, d, vp],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.tco_zone_size.argtypes = [i64, i64, i64, i64, i64]
        L.tco_zone_size.restype = i64
        L.tco_boundary_count.argtypes = [i64]
        L.tco_boundary_count.restype = i64
        L.tco_sigma_ramp.argtypes = [d, d, i64, i64]
        L.tco_sigma_ramp.restype = d
        _libs[openmp] = L
    return _libs[openmp]


def threads(openmp: bool = False) -> int:
    """Host threads tco_rows_grad runs on in the plain (1) or OpenMP build."""
    return int(lib(openmp).tco_threads())


def _pos(pos) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(pos, dtype=np.float64))
    if a.ndim != 2 or a.shape[1] != 2:
        raise ValueError("positions must have shape (n, 2)")
    return a


def _p(a):
    return None if a is None else a.ctypes.data


def _check(code: int, what: str) -> None:
    if code != 0:
        raise OracleError(code, what)


def energy(pos, local: bool = False):
    """E = sum_{i<j} 1/r_ij; with local=True also e_i = 1/2 sum_{j != i} 1/r_ij."""
    p = _pos(pos)
    e = np.zeros(1)
    le = np.zeros(p.shape[0]) if local else None
    _check(lib().tco_energy(_p(p), p.shape[0], _p(e), _p(le)), "energy")
    return (float(e[0]), le) if local else float(e[0])


def grad(pos) -> np.ndarray:
    """g_i = dE/dr_i = sum_{j != i} -(r_i - r_j)/r_ij^3, shape (n, 2)."""
    p = _pos(pos)
    g = np.zeros_like(p)
    _check(lib().tco_grad(_p(p), p.shape[0], _p(g)), "grad")
    return g


def rows_grad(pos, rows, openmp: bool = False):
    """Gradient rows (and sum_{j != i} 1/r_ij) of the charges `rows` against all n.

    openmp=True runs the rows on all host threads (same arithmetic per row)."""
    p = _pos(pos)
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int32))
    g = np.zeros((r.size, 2))
    e = np.zeros(r.size)
    _check(lib(openmp).tco_rows_grad(_p(p), p.shape[0], _p(r), r.size, _p(g), _p(e)), "rows_grad")
    return g, e


def subdomain_grad(snap, idx, act):
    """Gradient, local energies e_k and E_sub of the subdomain objective (Sec. II D)."""
    s = _pos(snap)
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.int32))
    a = _pos(act)
    g = np.zeros_like(a)
    e = np.zeros(ix.size)
    es = np.zeros(1)
    _check(lib().tco_subdomain_grad(_p(s), s.shape[0], _p(ix), ix.size, _p(a), _p(g), _p(e), _p(es)),
           "subdomain_grad")
    return g, e, float(es[0])


def delta_energy(pos, idx, new_act) -> float:
    """Energy change of moving charges idx to new_act, summed as pair differences."""
    p = _pos(pos)
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.int32))
    na = _pos(new_act)
    d = np.zeros(1)
    _check(lib().tco_delta_energy(_p(p), p.shape[0], _p(ix), ix.size, _p(na), _p(d)), "delta_energy")
    return float(d[0])


def project(pos, radius: float = 1.0, flags=None) -> np.ndarray:
    """Hard-wall projection r <- r min(1, radius/|r|); pinned charges to the unit circle."""
    p = _pos(pos).copy()
    f = None if flags is None else np.ascontiguousarray(np.asarray(flags, dtype=np.uint8))
    _check(lib().tco_project(_p(p), p.shape[0], float(radius), _p(f)), "project")
    return p


def projected_grad(pos, g, radius: float = 1.0, flags=None):
    """Gradient with wall-blocked components removed; returns (pg, rms, max)."""
    p = _pos(pos)
    gg = _pos(g)
    f = None if flags is None else np.ascontiguousarray(np.asarray(flags, dtype=np.uint8))
    pg = np.zeros_like(p)
    rms = np.zeros(1)
    mx = np.zeros(1)
    _check(lib().tco_projected_grad(_p(p), _p(gg), p.shape[0], float(radius), _p(f), _p(pg), _p(rms), _p(mx)),
           "projected_grad")
    return pg, float(rms[0]), float(mx[0])


def pgd(pos, eta: float, steps: int, radius: float = 1.0, flags=None):
    """Projected gradient descent x <- P(x - eta g); returns (x, energy trace[steps+1])."""
    p = _pos(pos).copy()
    f = None if flags is None else np.ascontiguousarray(np.asarray(flags, dtype=np.uint8))
    tr = np.zeros(steps + 1)
    _check(lib().tco_pgd(_p(p), p.shape[0], float(eta), int(steps), float(radius), _p(f), _p(tr)), "pgd")
    return p, tr


def _flags(flags):
    return None if flags is None else np.ascontiguousarray(np.asarray(flags, dtype=np.uint8))


def subdomain_bb(snap, idx, step0: float, alpha_min: float, alpha_max: float, steps: int,
                 radius: float = 1.0, flags=None) -> np.ndarray:
    """Projected BB gradient descent of one subdomain against the snapshot; returns x (m, 2).

    flags (n, nullable): pinned charges, projected to the unit circle."""
    s = _pos(snap)
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.int32))
    f = _flags(flags)
    out = np.zeros((ix.size, 2))
    _check(lib().tco_subdomain_bb(_p(s), s.shape[0], _p(ix), ix.size, float(step0), float(alpha_min),
                                  float(alpha_max), int(steps), float(radius), _p(f), _p(out)), "subdomain_bb")
    return out


def accept_sequential(pos, idx, offsets, new_act):
    """Sequential FP64 accept/reject; returns (new pos, delta[n_sub], accepted[n_sub] in {0,1,2})."""
    p = _pos(pos).copy()
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.int32))
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
    na = _pos(new_act)
    ns = off.size - 1
    d = np.zeros(ns)
    acc = np.zeros(ns, dtype=np.uint8)
    _check(lib().tco_accept_sequential(_p(p), p.shape[0], _p(ix), _p(off), ns, _p(na), _p(d), _p(acc)),
           "accept_sequential")
    return p, d, acc


def lbfgs(pos, memory: int = 8, max_iter: int = 1000, gtol: float = 0.0, step0: float = 1e-4,
          maxstep: float = 1e-2, radius: float = 1.0, flags=None, line_search: int = 0, tu: bool = False):
    """L-BFGS on the wall map (tu=True: on the paper's (t, u) variables) with a max-displacement cap
    and, for line_search > 0, an Armijo backtracking line search of at most that many halvings;
    returns (x, iterations, final RMS of dE/d(variables))."""
    p = _pos(pos).copy()
    f = None if flags is None else np.ascontiguousarray(np.asarray(flags, dtype=np.uint8))
    it = np.zeros(1, dtype=np.int64)
    rms = np.zeros(1)
    _check(lib().tco_lbfgs_ls(_p(p), p.shape[0], int(memory), int(max_iter), float(gtol), float(step0),
                              float(maxstep), float(radius), _p(f), int(line_search), int(bool(tu)), _p(it),
                              _p(rms)), "lbfgs")
    return p, int(it[0]), float(rms[0])


def lbfgs_trace(pos, memory: int = 8, max_iter: int = 10, gtol: float = 0.0, step0: float = 1e-4,
                maxstep: float = 1e-2, radius: float = 1.0, flags=None, line_search: int = 0, tu: bool = False):
    """The lbfgs iteration with its path: returns (x, z (k+1, 2n), dE/dz (k+1, 2n), directions (k, 2n),
    step scales (k,)) for the k iterations taken (the step scale is the one before any halving)."""
    p = _pos(pos).copy()
    f = None if flags is None else np.ascontiguousarray(np.asarray(flags, dtype=np.uint8))
    L = 2 * p.shape[0]
    ztr = np.zeros((max_iter + 1, max(L, 1)))
    gtr = np.zeros((max_iter + 1, max(L, 1)))
    dtr = np.zeros((max(max_iter, 1), max(L, 1)))
    atr = np.zeros(max(max_iter, 1))
    it = np.zeros(1, dtype=np.int64)
    rms = np.zeros(1)
    _check(lib().tco_lbfgs_trace(_p(p), p.shape[0], int(memory), int(max_iter), float(gtol), float(step0),
                                 float(maxstep), float(radius), _p(f), int(line_search), int(bool(tu)), _p(it),
                                 _p(rms), _p(ztr), _p(gtr), _p(dtr), _p(atr)), "lbfgs_trace")
    k = int(it[0])
    return p, ztr[:k + 1, :L], gtr[:k + 1, :L], dtr[:k, :L], atr[:k]


def lbfgsb(pos, memory: int = 8, max_iter: int = 1000, gtol: float = 0.0, step0: float = 1e-4,
           maxstep: float = 1e-2, radius: float = 1.0, flags=None, line_search: int = 0):
    """L-BFGS-B on the (t, u) variables with the box t in [0, pi/2]; returns (x, iterations, final
    projected-gradient RMS, breakpoints passed by the Cauchy searches)."""
    p = _pos(pos).copy()
    f = None if flags is None else np.ascontiguousarray(np.asarray(flags, dtype=np.uint8))
    it = np.zeros(1, dtype=np.int64)
    nb = np.zeros(1, dtype=np.int64)
    rms = np.zeros(1)
    _check(lib().tco_lbfgsb(_p(p), p.shape[0], int(memory), int(max_iter), float(gtol), float(step0),
                            float(maxstep), float(radius), _p(f), int(line_search), _p(it), _p(rms), _p(nb)),
           "lbfgsb")
    return p, int(it[0]), float(rms[0]), int(nb[0])


def _vecs(*arrs):
    return [np.ascontiguousarray(np.asarray(a, dtype=np.float64)) for a in arrs]


def subdomain_lbfgsb(snap, idx, memory: int = 8, steps: int = 100, step0: float = 1e-4, maxstep: float = 1e-2,
                     radius: float = 1.0, flags=None, line_search: int = 0):
    """L-BFGS-B on (t, u) of the charges idx against the others held at snap; returns their positions."""
    s = _pos(snap)
    ix = np.ascontiguousarray(np.asarray(idx, dtype=np.int32))
    f = _flags(flags)
    act = np.zeros((ix.size, 2))
    _check(lib().tco_subdomain_lbfgsb(_p(s), s.shape[0], _p(ix), ix.size, int(memory), int(steps), float(step0),
                                      float(maxstep), float(radius), _p(f), int(line_search), _p(act)),
           "subdomain_lbfgsb")
    return act


def lbfgsb_middle(S, Y, theta: float):
    """M = K^{-1} of the compact representation B = theta I - W M W^T (rows of S, Y: pairs, oldest first)."""
    S, Y = _vecs(S, Y)
    h, nv = S.shape
    M = np.zeros((2 * h, 2 * h))
    _check(lib().tco_lbfgsb_middle(h, _p(S), _p(Y), nv, float(theta), _p(M)), "lbfgsb_middle")
    return M


def lbfgsb_cauchy(x, g, lo, hi, S, Y, theta: float, M):
    """Generalized Cauchy point: returns (xc, c = W^T (xc - x), breakpoints passed)."""
    x, g, lo, hi, S, Y, M = _vecs(x, g, lo, hi, S, Y, M)
    h = S.shape[0] if S.ndim == 2 else 0
    xc = np.zeros_like(x)
    c = np.zeros(max(2 * h, 1))
    nb = np.zeros(1, dtype=np.int64)
    _check(lib().tco_lbfgsb_cauchy(x.size, _p(x), _p(g), _p(lo), _p(hi), h, _p(S), _p(Y), float(theta), _p(M),
                                   _p(xc), _p(c), _p(nb)), "lbfgsb_cauchy")
    return xc, c[:2 * h], int(nb[0])


def lbfgsb_subspace(x, g, lo, hi, S, Y, theta: float, M, xc, c):
    """Subspace minimisation from the Cauchy point xc: returns xbar."""
    x, g, lo, hi, S, Y, M, xc = _vecs(x, g, lo, hi, S, Y, M, xc)
    c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(-1))
    h = S.shape[0] if S.ndim == 2 else 0
    xbar = np.zeros_like(x)
    _check(lib().tco_lbfgsb_subspace(x.size, _p(x), _p(g), _p(lo), _p(hi), h, _p(S), _p(Y), float(theta), _p(M),
                                     _p(xc), _p(c if c.size else np.zeros(1)), _p(xbar)), "lbfgsb_subspace")
    return xbar


def zone_size(q: int, m_min: int, m_max: int, period: int, n: int) -> int:
    """Active-set size at schedule position q (triangle wave between m_min and m_max)."""
    return int(lib().tco_zone_size(int(q), int(m_min), int(m_max), int(period), int(n)))


def zone_select(pos, local_e, uniforms, m_min: int, m_max: int, period: int, phase: int = 0,
                kappa: float = -1.0, p_defect: float = 0.8, radius: float = 1.0, wall_tol: float = 1e-9,
                flags=None):
    """Defects, centres and nearest-m zones of Sec. II C; returns (idx, offsets, centres, stats).

    uniforms: (n_sub, 3) in [0, 1); stats = (mu, sigma_e, number of defects)."""
    p = _pos(pos)
    n = p.shape[0]
    e = np.ascontiguousarray(np.asarray(local_e, dtype=np.float64))
    u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64).reshape(-1, 3))
    ns = u.shape[0]
    cap = sum(zone_size(phase + s, m_min, m_max, period, n) for s in range(ns))
    idx = np.zeros(max(cap, 1), dtype=np.int32)
    off = np.zeros(ns + 1, dtype=np.int64)
    cen = np.zeros((ns, 2))
    stats = np.zeros(3)
    f = _flags(flags)
    _check(lib().tco_zone_select(_p(p), n, _p(e), _p(f), float(kappa), float(p_defect), float(radius),
                                 float(wall_tol),
                                 int(m_min), int(m_max), int(period), int(phase), ns, _p(u), _p(idx), _p(off),
                                 _p(cen), _p(stats)), "zone_select")
    return idx[:cap], off, cen, stats


def cycle(pos, uniforms, m_min: int, m_max: int, period: int, batch: int, step0: float, alpha_min: float,
          alpha_max: float, steps: int, kappa: float = -1.0, p_defect: float = 0.8, sigma0: float = 1.0,
          sigma1: float = 1.0, wall_tol: float = 1e-9, flags=None, optimizer: str = "bb", memory: int = 8,
          maxstep: float = 1e-3, line_search: int = 0, disjoint: bool = False):
    """One optimisation cycle (Sec. II C) in batches; returns (pos, trace, delta, accepted).

    sigma0 -> sigma1: interior radius ramp over the batches; flags: pinned boundary charges;
    optimizer "bb" (projected BB) or "lbfgsb_tu" (L-BFGS-B on (t, u) per zone).  disjoint=True: a batch
    is the longest prefix of pairwise disjoint zones among the next `batch` subdomains (the rest are
    selected again for the next batch); the trace then has one entry per batch run, plus one."""
    p = _pos(pos).copy()
    f = _flags(flags)
    u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64).reshape(-1, 3))
    ns = u.shape[0]
    trace = np.zeros(ns + 1)
    d = np.zeros(max(ns, 1))
    acc = np.zeros(max(ns, 1), dtype=np.uint8)
    nb = np.zeros(1, dtype=np.int64)
    opt = {"bb": 0, "lbfgsb_tu": 1}[optimizer]
    _check(lib().tco_cycle_run(_p(p), p.shape[0], _p(f), float(kappa), float(p_defect), float(sigma0),
                               float(sigma1), float(wall_tol), int(m_min), int(m_max), int(period), ns, int(batch),
                               int(bool(disjoint)), _p(u), opt, float(step0), float(alpha_min), float(alpha_max),
                               int(memory), float(maxstep), int(line_search), int(steps), _p(trace), _p(d), _p(acc),
                               _p(nb)), "cycle")
    return p, trace[:int(nb[0]) + 1], d[:ns], acc[:ns]


def boundary_count(n: int) -> int:
    """Eq. Nb: N_b = round(2.84328 N^(2/3) - 0.530196 N^(1/3) - 2.32866), within [0, n]."""
    return int(lib().tco_boundary_count(int(n)))


def sigma_ramp(sigma0: float, sigma1: float, b: int, n_batches: int) -> float:
    """Interior radius of batch b (linear ramp from sigma0 to sigma1)."""
    return float(lib().tco_sigma_ramp(float(sigma0), float(sigma1), int(b), int(n_batches)))


def border_split(pos, n_b: int, sigma: float):
    """Sec. II B split: the n_b outermost charges (by (|r|^2, i)) pinned to the unit circle, the rest
    confined to radius sigma; returns (pos, flags)."""
    p = _pos(pos).copy()
    f = np.zeros(p.shape[0], dtype=np.uint8)
    _check(lib().tco_border_split(_p(p), p.shape[0], int(n_b), float(sigma), _p(f)), "border_split")
    return p, f


def library_path() -> str:
    return os.path.abspath(lib()._name)
