"""Checkpoint and resume of a long adaptive cycle (Sec. II C).

The paper's cycle of T = 1000 subdomain optimisations ran for about 31 hours on a CPU; a run that
long needs to survive interruption.  run_cycle() runs a cycle as a sequence of tc_cycle calls of
`chunk` subdomains each (the sigma ramp and the zone-size schedule span the whole cycle, so the
calls take the radii and sizes of one long cycle) and, after every call, writes the state to
`path` (an .npz written to a temporary name and renamed, so a crash leaves the previous checkpoint
intact): the positions, the flags, the number of subdomains done (the position in the uniform
draws), the energy trace and the per-subdomain results so far, plus the run's parameters and a
SHA-256 of the uniforms, which a resume checks.  A run resumed from any of its checkpoints ends
bit for bit where the same run without the interruption ends: the kernels are deterministic and
the state between calls is exactly what is saved.  Checkpoints fall on call boundaries, which are
batch boundaries; with disjoint batches a batch never spans two calls.

No L-BFGS history is saved: each subdomain's optimisation starts and ends inside one call.
"""

from __future__ import annotations

import hashlib
import json
import os

import numpy as np
import torch

from . import cycle as _cycle

_FIELDS = ("delta_e", "energy", "rms", "steps", "status")


def _params_key(n: int, n_sub: int, chunk: int, kw: dict) -> str:
    return json.dumps({"n": n, "n_sub": n_sub, "chunk": chunk,
                       **{k: (float(v) if isinstance(v, float) else v) for k, v in sorted(kw.items())}},
                      sort_keys=True)


def _digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def save_state(path: str, state: dict) -> None:
    """Write a checkpoint atomically (temporary file, then rename)."""
    tmp = path + ".tmp.npz"
    np.savez(tmp, **state)
    os.replace(tmp, path)


def load_state(path: str) -> dict:
    with np.load(path, allow_pickle=False) as z:
        return {k: z[k] for k in z.files}


def run_cycle(pos: torch.Tensor, uniforms: torch.Tensor, flags: torch.Tensor | None = None, *, chunk: int,
              path: str | None = None, resume: bool = True, stop_after: int | None = None, cycle_fn=None,
              **cycle_kw):
    """Run the cycle of uniforms.shape[0] subdomains on pos (in place) in calls of `chunk` subdomains,
    checkpointing to `path` after each call.

    resume=True and an existing checkpoint at `path`: continue from it (its parameters and uniforms
    must match; pos and flags are overwritten with the saved ones).  stop_after: return after this
    many calls of this invocation (an interruption, for tests and for time-limited jobs).  cycle_fn:
    the cycle call (default: paper_2609_24722_b300.cycle).  With fixed batches, chunk must be a
    multiple of `batch`.  Returns (results dict of numpy arrays over the subdomains done, energy
    trace, subdomains done)."""
    cycle_fn = _cycle if cycle_fn is None else cycle_fn
    n, n_sub = pos.shape[0], uniforms.shape[0]
    if chunk < 1 or (not cycle_kw.get("disjoint", False) and chunk % int(cycle_kw["batch"]) != 0):
        raise ValueError("chunk must be >= 1 and, with fixed batches, a multiple of batch")
    phase0 = int(cycle_kw.pop("phase", 0))
    key = _params_key(n, n_sub, chunk, {**cycle_kw, "phase": phase0})
    u_digest = _digest(uniforms.detach().cpu().numpy())
    done = 0
    res = {f: np.full(n_sub, np.nan) if f in ("delta_e", "energy", "rms") else np.zeros(n_sub, np.int32)
           for f in _FIELDS}
    trace: list[float] = []
    if path and resume and os.path.exists(path):
        st = load_state(path)
        if str(st["params"]) != key or str(st["uniforms_sha256"]) != u_digest:
            raise ValueError(f"checkpoint {path} belongs to another run (parameters or uniforms differ)")
        done = int(st["done"])
        trace = st["trace"].tolist()
        for f in _FIELDS:
            res[f] = st[f].copy()
        pos.copy_(torch.as_tensor(st["pos"], device=pos.device))
        if flags is not None:
            flags.copy_(torch.as_tensor(st["flags"], device=flags.device))
    calls = 0
    while done < n_sub and (stop_after is None or calls < stop_after):
        k = min(chunk, n_sub - done)
        r, tr = cycle_fn(pos, uniforms[done:done + k], flags, phase=phase0 + done, ramp_first=done,
                         ramp_total=n_sub, **cycle_kw)
        tr = tr.detach().cpu().numpy().tolist()
        trace = tr if not trace else trace + tr[1:]  # a call's first entry is the previous call's last
        for f in _FIELDS:
            res[f][done:done + k] = getattr(r, f).detach().cpu().numpy()
        done += k
        calls += 1
        if path:
            save_state(path, {"pos": pos.detach().cpu().numpy(),
                              "flags": (flags.detach().cpu().numpy() if flags is not None else np.zeros(0, np.uint8)),
                              "done": np.int64(done), "trace": np.asarray(trace, dtype=np.float64),
                              "params": np.str_(key), "uniforms_sha256": np.str_(u_digest),
                              **{f: res[f] for f in _FIELDS}})
    return {f: res[f][:done] for f in _FIELDS}, np.asarray(trace), done
