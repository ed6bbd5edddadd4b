"""Checkpoint and resume of a continuation state (the setting of Sec. 4, numerical
parameter continuation): the field strength mu, the order parameter psi on the
mesh, the mesh's description, optionally the learned warm start's parameters and
the points accepted so far.

Layout of a state directory (all binaries little-endian, no header):
    meta.json       {"format": 1, "dim", "N", "edge", "bhat", "mu", "n",
                     "psi": "psi.bin", "params": "ws_params.bin" | null,
                     "points": [...]}
    psi.bin         n complex values, FP64 (re, im interleaved), node order
    ws_params.bin   the warm-start parameters, FP32 (when saved)

Resuming restarts the continuation from (psi, mu) on a mesh made from the saved
description: the tangent of the first new step is computed afresh
(Jc = -dGL/dmu), as at any start.
"""
from __future__ import annotations

import json
import os

import numpy as np

FORMAT = 1


def _host(a, dtype):
    try:
        import torch

        if isinstance(a, torch.Tensor):
            a = a.detach().cpu().numpy()
    except ImportError:
        pass
    return np.ascontiguousarray(np.asarray(a), dtype=np.dtype(dtype).newbyteorder("<"))


def save_state(path: str, *, dim: int, N: int, mu: float, psi, edge: float = 1.0, bhat=(0.0, 0.0, 1.0),
               ws_params=None, points=None) -> None:
    """Writes the state to directory `path` (created if missing).  psi: n complex
    values (numpy or torch, any device), node order; ws_params: the warm start's
    flat parameter vector or None; points: a list of point dicts or None."""
    os.makedirs(path, exist_ok=True)
    p = _host(psi, np.complex128).ravel()
    n = int(N) ** int(dim)
    if p.size != n:
        raise ValueError(f"psi has {p.size} values, the mesh {n} nodes")
    p.tofile(os.path.join(path, "psi.bin"))
    params_name = None
    if ws_params is not None:
        params_name = "ws_params.bin"
        _host(ws_params, np.float32).ravel().tofile(os.path.join(path, params_name))
    meta = {"format": FORMAT, "dim": int(dim), "N": int(N), "edge": float(edge),
            "bhat": [float(v) for v in bhat], "mu": float(mu), "n": n, "psi": "psi.bin",
            "params": params_name, "points": list(points) if points is not None else []}
    with open(os.path.join(path, "meta.json"), "w") as f:
        json.dump(meta, f, indent=1)


def load_state(path: str) -> dict:
    """Reads a state written by save_state: the metadata dict with "psi" (numpy
    complex128, n values) and "params" (numpy float32 or None) replaced by the
    arrays."""
    with open(os.path.join(path, "meta.json")) as f:
        meta = json.load(f)
    if meta.get("format") != FORMAT:
        raise ValueError(f"unknown state format {meta.get('format')}")
    psi = np.fromfile(os.path.join(path, meta["psi"]), dtype="<c16")
    if psi.size != meta["n"]:
        raise ValueError(f"psi.bin holds {psi.size} values, meta.json says {meta['n']}")
    meta["psi"] = psi.astype(np.complex128)
    if meta.get("params"):
        meta["params"] = np.fromfile(os.path.join(path, meta["params"]), dtype="<f4").astype(np.float32)
    else:
        meta["params"] = None
    return meta
