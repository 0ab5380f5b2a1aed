"""Coulomb charges in the unit disk on one B300: Python binding of libtc.

Thin wrappers over the C ABI in include/tc.h.  Tensors are CUDA float64
(positions (n, 2)), int32 index sets and int64 offsets; every step of the
computation runs in libtc's CUDA kernels on the current torch stream.  There is
no CPU path: on a machine without a GPU or without libtc.so every call raises.

    energy(pos)            E = sum_{i<j} 1/r_ij            (Eq. hamiltonian)
    grad(pos)              dE/dr                            (its analytic gradient)
    local_energy(pos)      e_i = 1/2 sum_{j != i} 1/r_ij    (Sec. II C step 1)
    project_disk(pos)      hard wall of Eq. (potential) as a projection
    subdomain_delta_energy pairwise E_sub(new) - E_sub(old) (Sec. II D)
    subdomain_grad         dE_sub/da, e_k and E_sub of many subdomains (Sec. II D)
    relax_subdomains       batched local relaxation of subdomains / instances
    coulomb_energy         torch.autograd.Function: energy forward, gradient backward
    subdomain_energy       the same for E_sub of one subdomain as a function of its charges
"""

from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import _lib as L
from ._lib import TCError, RelaxParams

__all__ = [
    "energy", "grad", "local_energy", "project_disk", "subdomain_delta_energy", "relax_subdomains",
    "coulomb_energy", "CoulombEnergy", "sync_status", "probe_pipes", "relax_last_profile", "TCError", "RelaxParams",
    "library_path", "zone_params", "zone_offsets", "select_subdomains", "cycle", "subdomain_delta_energy_mixed",
    "boundary_count", "border_split", "voronoi_order", "subdomain_grad", "subdomain_energy", "SubdomainEnergy",
]

_PREC = {"fp64": L.TC_FP64, "mixed": L.TC_MIXED, "fp64x": L.TC_F64X}
_OPT = {"gd": L.TC_OPT_GD, "bb": L.TC_OPT_BB, "lbfgs": L.TC_OPT_LBFGS, "lbfgs_tu": L.TC_OPT_LBFGS_TU,
        "lbfgsb_tu": L.TC_OPT_LBFGSB_TU}


def library_path() -> str:
    return L.LIB_PATH


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _p(t) -> int | None:
    return None if t is None else t.data_ptr()


def _pos(t: torch.Tensor, name: str = "pos") -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if t.dim() != 2 or t.shape[1] != 2 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous (n, 2) tensor")
    return t


def _prec(p) -> int:
    if isinstance(p, int):
        return p
    return _PREC[p]


def sync_status() -> None:
    """Wait for the current stream and raise if a kernel recorded a device error."""
    L.check(L.lib().tc_sync_status(_stream()), "device status")


def energy(pos: torch.Tensor, precision="fp64") -> torch.Tensor:
    """Total energy E (0-d CUDA float64 tensor)."""
    _pos(pos)
    out = torch.empty((), dtype=torch.float64, device=pos.device)
    L.check(L.lib().tc_energy(_p(pos), pos.shape[0], _prec(precision), _p(out), None, _stream()), "tc_energy")
    return out


def local_energy(pos: torch.Tensor, precision="fp64") -> tuple[torch.Tensor, torch.Tensor]:
    """(E, e) with e_i = 1/2 sum_{j != i} 1/r_ij."""
    _pos(pos)
    out = torch.empty((), dtype=torch.float64, device=pos.device)
    e = torch.empty(pos.shape[0], dtype=torch.float64, device=pos.device)
    L.check(L.lib().tc_energy(_p(pos), pos.shape[0], _prec(precision), _p(out), _p(e), _stream()), "tc_energy")
    return out, e


def grad(pos: torch.Tensor, precision="fp64", with_energy: bool = False):
    """dE/dr (n, 2); with with_energy=True also E from the same pass."""
    _pos(pos)
    g = torch.empty_like(pos)
    e = torch.empty((), dtype=torch.float64, device=pos.device) if with_energy else None
    L.check(L.lib().tc_grad(_p(pos), pos.shape[0], _prec(precision), _p(g), _p(e), _stream()), "tc_grad")
    return (g, e) if with_energy else g


def project_disk(pos: torch.Tensor, radius: float = 1.0, flags: torch.Tensor | None = None) -> torch.Tensor:
    """In place: r <- r min(1, radius/|r|); charges with flags != 0 go to the unit circle."""
    _pos(pos)
    if flags is not None and (flags.dtype != torch.uint8 or not flags.is_cuda or flags.numel() != pos.shape[0]):
        raise TypeError("flags must be a CUDA uint8 tensor with one entry per charge")
    L.check(L.lib().tc_project_disk(_p(pos), pos.shape[0], float(radius), _p(flags), _stream()), "tc_project_disk")
    return pos


def _csr(idx, offsets):
    if idx.dtype != torch.int32 or not idx.is_cuda or not idx.is_contiguous():
        raise TypeError("idx must be a contiguous CUDA int32 tensor")
    if offsets.dtype != torch.int64 or not offsets.is_cuda or not offsets.is_contiguous():
        raise TypeError("offsets must be a contiguous CUDA int64 tensor")


def subdomain_delta_energy(pos, idx, offsets, new_active) -> torch.Tensor:
    """Pairwise float64 energy change of moving each subdomain's charges to new_active."""
    _pos(pos)
    _csr(idx, offsets)
    _pos(new_active, "new_active")
    n_sub = offsets.numel() - 1
    out = torch.empty(max(n_sub, 0), dtype=torch.float64, device=pos.device)
    L.check(L.lib().tc_subdomain_delta_energy(_p(pos), pos.shape[0], _p(idx), _p(offsets), n_sub,
                                              _p(new_active), _p(out), _stream()), "tc_subdomain_delta_energy")
    return out


def subdomain_delta_energy_mixed(pos, idx, offsets, new_active) -> tuple[torch.Tensor, torch.Tensor]:
    """Difference-form float32 energy change of each subdomain and its error bound (delta, bound)."""
    _pos(pos)
    _csr(idx, offsets)
    _pos(new_active, "new_active")
    n_sub = offsets.numel() - 1
    out = torch.empty(max(n_sub, 0), dtype=torch.float64, device=pos.device)
    bound = torch.empty(max(n_sub, 0), dtype=torch.float64, device=pos.device)
    L.check(L.lib().tc_subdomain_delta_energy_mixed(_p(pos), pos.shape[0], _p(idx), _p(offsets), n_sub,
                                                    _p(new_active), _p(out), _p(bound), _stream()),
            "tc_subdomain_delta_energy_mixed")
    return out, bound


def subdomain_grad(pos, idx, offsets, act=None, precision="fp64"):
    """Gradient rows dE_sub/da (M, 2), local energies e_k (M,) and E_sub per subdomain (n_sub,) of the
    subdomain objective (Sec. II D): the charges idx at act (default: their positions in pos) against
    every other charge at pos."""
    _pos(pos)
    _csr(idx, offsets)
    if act is not None:
        _pos(act, "act")
        if act.shape[0] != idx.numel():
            raise ValueError("act must hold one position per active index")
    n_sub = offsets.numel() - 1
    m = idx.numel()
    g = torch.empty((m, 2), dtype=torch.float64, device=pos.device)
    e = torch.empty(m, dtype=torch.float64, device=pos.device)
    es = torch.empty(max(n_sub, 0), dtype=torch.float64, device=pos.device)
    L.check(L.lib().tc_subdomain_grad(_p(pos), pos.shape[0], _p(idx), _p(offsets), n_sub, _p(act), _prec(precision),
                                      _p(g), _p(e), _p(es), _stream()), "tc_subdomain_grad")
    return g, e, es


@dataclass
class RelaxResult:
    delta_e: torch.Tensor   # float64 pairwise energy change (NaN when not computed)
    energy: torch.Tensor    # float64 final E_sub / E (NaN when not requested)
    rms: torch.Tensor       # final RMS stationarity
    steps: torch.Tensor     # int32 steps taken
    status: torch.Tensor    # int32: 0 rejected, 1 accepted/written, 2 skipped


def relax_subdomains(pos, idx=None, offsets=None, world=None, flags=None, *, precision="mixed", optimizer="bb",
                     n_steps=200, memory=8, step0=1e-9, alpha_min=0.0, alpha_max=1e-8, maxstep=1e-3, gtol=0.0,
                     radius=1.0, polish_steps=0, polish_gtol=0.0, accept=True, want_energy=False,
                     profile=False, polish_precision="fp64", line_search=0) -> RelaxResult:
    """Relax subdomains (idx/offsets given) or independent instances (idx None, world given)."""
    _pos(pos)
    if idx is not None:
        _csr(idx, offsets)
        n_sub = offsets.numel() - 1
    else:
        if world is None:
            raise ValueError("instance mode needs world ranges")
        n_sub = world.shape[0]
    if world is not None and (world.dtype != torch.int64 or not world.is_cuda or not world.is_contiguous()):
        raise TypeError("world must be a contiguous CUDA int64 tensor of shape (n_sub, 2)")
    prm = _relax_params(precision, optimizer, n_steps, memory, step0, alpha_min, alpha_max, maxstep, gtol, radius,
                        polish_steps, polish_gtol, accept, want_energy, profile, polish_precision, line_search)
    raw = torch.empty((max(n_sub, 1), 4), dtype=torch.float64, device=pos.device)
    L.check(L.lib().tc_relax_subdomains(_p(pos), pos.shape[0], _p(idx), _p(offsets), n_sub, _p(world), _p(flags),
                                        C.byref(prm), _p(raw), _stream()), "tc_relax_subdomains")
    return _results(raw, n_sub)


def _relax_params(precision, optimizer, n_steps, memory, step0, alpha_min, alpha_max, maxstep, gtol, radius,
                  polish_steps, polish_gtol, accept, want_energy, profile, polish_precision="fp64",
                  line_search=0) -> RelaxParams:
    return RelaxParams(precision=_prec(precision), optimizer=_OPT[optimizer] if isinstance(optimizer, str) else optimizer,
                       n_steps=int(n_steps), memory=int(memory), step0=float(step0), alpha_min=float(alpha_min),
                       alpha_max=float(alpha_max), maxstep=float(maxstep), gtol=float(gtol), radius=float(radius),
                       polish_steps=int(polish_steps), accept=int(bool(accept)), polish_gtol=float(polish_gtol),
                       want_energy=int(bool(want_energy)), profile=int(bool(profile)),
                       polish_precision=_prec(polish_precision), line_search=int(line_search))


def _results(raw: torch.Tensor, n_sub: int) -> RelaxResult:
    raw = raw[:n_sub]
    # the two int32 fields share the fourth 8-byte column of each 32-byte record
    ints = raw.view(torch.int32).view(n_sub, 8)[:, 6:8]
    return RelaxResult(raw[:, 0], raw[:, 1], raw[:, 2], ints[:, 0].clone(), ints[:, 1].clone())


def zone_params(m_min: int, m_max: int, period: int, phase: int = 0, kappa: float = -1.0, p_defect: float = 0.8,
                radius: float = 1.0, wall_tol: float = 1e-9) -> L.ZoneParams:
    """tc_zone_params: defect threshold mu + kappa sigma_e, centre mix, zone-size triangle wave."""
    return L.ZoneParams(kappa=float(kappa), p_defect=float(p_defect), radius=float(radius), wall_tol=float(wall_tol),
                        m_min=int(m_min), m_max=int(m_max), period=int(period), phase=int(phase))


def zone_offsets(n: int, n_sub: int, **zone) -> list[int]:
    """Host CSR offsets of n_sub zones (no GPU work)."""
    prm = zone_params(**zone)
    off = (C.c_int64 * (n_sub + 1))()
    L.check(L.lib().tc_zone_offsets(C.byref(prm), int(n), int(n_sub), C.cast(off, C.c_void_p)), "tc_zone_offsets")
    return list(off)


def _vec(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA {dtype} tensor")
    return t


def select_subdomains(pos, local_e, uniforms, flags=None, **zone):
    """Defect threshold, centres and nearest-m zones (Sec. II C steps 2-4).

    uniforms: (n_sub, 3) CUDA float64 in [0, 1).  Returns (idx int32, offsets int64,
    centres (n_sub, 2), stats (mu, sigma_e, number of defects))."""
    _pos(pos)
    _vec(local_e, torch.float64, "local_e")
    _vec(uniforms, torch.float64, "uniforms")
    n_sub = uniforms.numel() // 3
    off_h = zone_offsets(pos.shape[0], n_sub, **zone)
    prm = zone_params(**zone)
    idx = torch.empty(max(off_h[-1], 1), dtype=torch.int32, device=pos.device)
    offsets = torch.empty(n_sub + 1, dtype=torch.int64, device=pos.device)
    centres = torch.empty((max(n_sub, 1), 2), dtype=torch.float64, device=pos.device)
    stats = torch.empty(3, dtype=torch.float64, device=pos.device)
    if flags is not None:
        _vec(flags, torch.uint8, "flags")
    L.check(L.lib().tc_select_subdomains(_p(pos), pos.shape[0], _p(local_e), _p(flags), C.byref(prm), n_sub,
                                         _p(uniforms), _p(idx), _p(offsets), _p(centres), _p(stats), _stream()),
            "tc_select_subdomains")
    return idx[:off_h[-1]], offsets, centres[:n_sub], stats


def cycle(pos, uniforms, flags=None, *, batch: int, m_min: int, m_max: int, period: int, phase: int = 0,
          kappa: float = -1.0, p_defect: float = 0.8, wall_tol: float = 1e-9, sigma0: float = 1.0, sigma1: float = 1.0,
          local_precision="mixed", precision="mixed", optimizer="bb", n_steps=200, memory=8, step0=1e-9,
          alpha_min=0.0, alpha_max=1e-8, maxstep=1e-3, gtol=0.0, polish_steps=0, polish_gtol=0.0,
          want_energy=False, profile=False, line_search=0, disjoint=False, ramp_first=0, ramp_total=0):
    """One optimisation cycle (Sec. II C) of uniforms.shape[0] subdomains in batches, in place on pos.

    flags (uint8, nullable): pinned boundary charges; sigma0 -> sigma1: interior radius ramp (sigma0 <= 0:
    Eq. sigma).  disjoint=True: each batch is the longest prefix of pairwise disjoint zones among the next
    `batch` subdomains.  ramp_first / ramp_total: this call is subdomains ramp_first .. of a cycle of
    ramp_total (the sigma ramp spans the whole cycle; 0 = this call alone).  Returns (RelaxResult per
    subdomain, energy trace: E before each batch and after the last)."""
    _pos(pos)
    _vec(uniforms, torch.float64, "uniforms")
    if flags is not None:
        _vec(flags, torch.uint8, "flags")
    n_sub = uniforms.numel() // 3
    prm = L.CycleParams()
    prm.zone = zone_params(m_min, m_max, period, phase, kappa, p_defect, 1.0, wall_tol)
    prm.relax = _relax_params(precision, optimizer, n_steps, memory, step0, alpha_min, alpha_max, maxstep, gtol,
                              1.0, polish_steps, polish_gtol, True, want_energy, profile, line_search=line_search)
    prm.batch = int(batch)
    prm.local_precision = _prec(local_precision)
    prm.sigma0 = float(sigma0)
    prm.sigma1 = float(sigma1)
    prm.disjoint = int(bool(disjoint))
    prm.ramp_first = int(ramp_first)
    prm.ramp_total = int(ramp_total)
    n_batches = (n_sub if disjoint else -(-n_sub // max(int(batch), 1))) if n_sub else 0
    raw = torch.empty((max(n_sub, 1), 4), dtype=torch.float64, device=pos.device)
    trace = torch.full((n_batches + 1,), float("nan"), dtype=torch.float64, device=pos.device)
    L.check(L.lib().tc_cycle(_p(pos), pos.shape[0], _p(flags), C.byref(prm), n_sub, _p(uniforms), _p(raw),
                             _p(trace), _stream()), "tc_cycle")
    if disjoint:
        trace = trace[~torch.isnan(trace)]
    return _results(raw, n_sub), trace


def boundary_count(n: int) -> int:
    """Eq. Nb: the number of boundary charges for n charges."""
    return int(L.lib().tc_boundary_count(int(n)))


def border_split(pos, n_b: int | None = None, sigma: float | None = None) -> torch.Tensor:
    """Sec. II B split in place: the n_b outermost charges pinned to the unit circle, the rest confined
    to sigma.  Defaults: n_b from Eq. Nb, sigma from Eq. sigma (libtc takes sigma <= 0 as Eq. sigma).
    Returns the uint8 flags."""
    _pos(pos)
    n = pos.shape[0]
    n_b = boundary_count(n) if n_b is None else int(n_b)
    sigma = 0.0 if sigma is None else float(sigma)
    flags = torch.empty(n, dtype=torch.uint8, device=pos.device)
    L.check(L.lib().tc_border_split(_p(pos), n, n_b, sigma, _p(flags), _stream()), "tc_border_split")
    return flags


def relax_last_profile() -> dict:
    """Launch timings of this thread's last relax_subdomains(..., profile=True) call."""
    prof = L.RelaxProfile()
    L.check(L.lib().tc_relax_last_profile(C.byref(prof)), "tc_relax_last_profile")
    return {f: getattr(prof, f) for f, _ in L.RelaxProfile._fields_}


def probe_pipes() -> dict:
    """Measured FFMA lane-ops/s, DFMA ops/s and MUFU.RSQ ops/s of the current device."""
    rates = (C.c_double * 4)()
    L.check(L.lib().tc_probe_pipes(C.cast(rates, C.c_void_p), _stream()), "tc_probe_pipes")
    return {"ffma_per_s": rates[0], "dfma_per_s": rates[1], "mufu_per_s": rates[2], "pairmix_per_s": rates[3]}


class CoulombEnergy(torch.autograd.Function):
    """E(pos) forward; backward recomputes dE/dr with tc_grad (no N x N storage)."""

    @staticmethod
    def forward(ctx, pos, precision="fp64"):
        ctx.save_for_backward(pos)
        ctx.precision = precision
        return energy(pos.contiguous(), precision)

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, gout):
        (pos,) = ctx.saved_tensors
        g = grad(pos.contiguous(), ctx.precision)
        return gout * g, None


def coulomb_energy(pos: torch.Tensor, precision="fp64") -> torch.Tensor:
    return CoulombEnergy.apply(pos, precision)


class SubdomainEnergy(torch.autograd.Function):
    """E_sub(act) of one subdomain (Sec. II D): the charges idx at act against the others held at pos.

    Forward and backward are one tc_subdomain_grad call each (the backward recomputes the pair terms;
    nothing m x N is stored).  Only act is differentiable."""

    @staticmethod
    def forward(ctx, act, pos, idx, precision="fp64"):
        offsets = torch.tensor([0, idx.numel()], dtype=torch.int64, device=pos.device)
        ctx.save_for_backward(act, pos, idx, offsets)
        ctx.precision = precision
        _, _, es = subdomain_grad(pos, idx, offsets, act.detach().contiguous(), precision)
        return es[0]

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, gout):
        act, pos, idx, offsets = ctx.saved_tensors
        g, _, _ = subdomain_grad(pos, idx, offsets, act.detach().contiguous(), ctx.precision)
        return gout * g, None, None, None


def subdomain_energy(act: torch.Tensor, pos: torch.Tensor, idx: torch.Tensor, precision="fp64") -> torch.Tensor:
    return SubdomainEnergy.apply(act, pos, idx, precision)


def voronoi_order(pos, max_nbr: int = 0):
    """Voronoi coordination numbers and psi6 (Sec. III C-D, Eq. psi6).

    Returns (z int32 (n,), psi6 complex128 (n,), summary dict, neighbours (n, max_nbr) int32 or None)."""
    _pos(pos)
    n = pos.shape[0]
    z = torch.empty(n, dtype=torch.int32, device=pos.device)
    psi = torch.empty((n, 2), dtype=torch.float64, device=pos.device)
    nbr = torch.empty((n, max_nbr), dtype=torch.int32, device=pos.device) if max_nbr > 0 else None
    summ = torch.empty(18, dtype=torch.float64, device=pos.device)
    L.check(L.lib().tc_voronoi_order(_p(pos), n, _p(z), _p(psi), _p(nbr), int(max_nbr), _p(summ), _stream()),
            "tc_voronoi_order")
    sm = summ.cpu()
    summary = {"mean_abs_psi6": float(sm[0]), "abs_mean_psi6": float(sm[1]), "P_z": sm[2:].numpy()}
    return z, torch.view_as_complex(psi), summary, nbr
