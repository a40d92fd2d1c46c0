"""Autotuning of the fused Chebyshev sweep and the JSON cache that aao_create reads.

The library times the candidates itself (aao_autotune: whole preconditioner applies, CUDA events
on the handle's stream); this module only runs it for a grid and records the winner in the cache
file, one entry per (device, dim, n, ell, precision, p):

    {"version": 1, "entries": [{"device": "...", "dim": 2, "n": [1024, 1024, 1], "ell": 10,
      "prec": "mixed", "p": 40, "kernel": "stream", "S": 4, "H": 88, "D": 3, "NW": 8,
      "us_per_apply": 612.0}]}

aao_set_tune_cache(path) (or the environment variable AAO_TUNE_CACHE) makes every later
aao_create in the process apply the matching entry.
"""
from __future__ import annotations

import json
import os
import tempfile
from typing import Dict, List, Optional

from . import binding

KEY_FIELDS = ("device", "dim", "n", "ell", "prec", "p")


def load(path: str) -> Dict:
    if not os.path.exists(path):
        return {"version": 1, "entries": []}
    with open(path) as f:
        d = json.load(f)
    if not isinstance(d, dict) or not isinstance(d.get("entries"), list):
        raise ValueError("%s is not a tune cache (no 'entries' list)" % path)
    return d


def save_entry(path: str, entry: Dict) -> None:
    """Insert or replace the entry with the same key, writing the file atomically."""
    d = load(path)
    key = tuple(json.dumps(entry.get(k)) for k in KEY_FIELDS)
    d["entries"] = [e for e in d["entries"] if tuple(json.dumps(e.get(k)) for k in KEY_FIELDS) != key]
    d["entries"].append(entry)
    folder = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(prefix=".tune_", dir=folder)
    with os.fdopen(fd, "w") as f:
        json.dump(d, f, indent=1)
    os.replace(tmp, path)


def make_entry(device: str, dim: int, n, ell: int, prec: int, p: int, best: Dict) -> Dict:
    return {"device": device, "dim": int(dim), "n": [int(v) for v in (list(n) + [1, 1, 1])[:3]],
            "ell": int(ell), "prec": "mixed" if prec == binding.AAO_MIXED else "fp64", "p": int(p),
            "kernel": best["kernel"], "S": int(best["S"]), "H": int(best["H"]), "D": int(best["D"]),
            "NW": int(best["NW"]), "us_per_apply": float(best["us_per_apply"])}


def tune_solver(solver, device: str, dim: int, n, ell: int, prec: int, p: int, reps: int = 3,
                path: Optional[str] = None):
    """Autotune an existing solver handle; record the winner in ``path`` if given.

    Returns (entry, candidates)."""
    best, cands = solver.autotune(reps)
    entry = make_entry(device, dim, n, ell, prec, p, best)
    if path:
        save_entry(path, entry)
    return entry, cands


def tune_grid(dim: int, n, kx, ky, kz, ell: int, alpha: float, p: int, path: Optional[str] = None,
              prec: int = binding.AAO_MIXED, reps: int = 3, stream=None):
    """Create a one-vector-Krylov handle for the grid, autotune it and record the result."""
    import torch
    device = torch.cuda.get_device_name()
    s = binding.Solver(dim, n, kx, ky, kz, ell, alpha, prec=prec, inner_its=p, restart=1, stream=stream)
    try:
        return tune_solver(s, device, dim, n, ell, prec, p, reps, path)
    finally:
        s.close()
