"""Kernel-shape autotuner for ctqw_propagate_taylor.

The library compiles several CTA / cluster shapes of its fused kernels and,
besides them, the row-wavefront kernel, the tiled kernel at several
temporal-blocking depths and the per-term path.  Which one is
fastest depends on N, K, the number of realizations and the GPU.  The tuner
times every candidate the handle supports on a scratch copy of the state for
a few steps (CUDA events on the caller's stream, after one untimed warm-up),
keeps the fastest, and caches the choice in a JSON file keyed by the
lattice shape, type, order, realization count and device.

The order K itself comes from the truncation bound (ctqw_autotune_order, or
K = 0 in ctqw_propagate_taylor).
"""
from __future__ import annotations

import json
import os
from typing import Dict, Iterable, List, Optional, Tuple

import torch

from . import ctqw

# candidate flag words: full-row shapes 0..2, banded shapes 4..6, the row
# wavefront, the tiled kernel at depths 4, 2, 8, and the per-term path
CANDIDATES: Tuple[int, ...] = (
    ctqw.FUSED_SHAPE(0), ctqw.FUSED_SHAPE(1), ctqw.FUSED_SHAPE(2),
    ctqw.FUSED_SHAPE(4), ctqw.FUSED_SHAPE(5), ctqw.FUSED_SHAPE(6),
    ctqw.FLAG_WAVEFRONT, ctqw.FLAG_TILED(0), ctqw.FLAG_TILED(1), ctqw.FLAG_TILED(2),
    ctqw.FLAG_TILED(3), ctqw.FLAG_TILED(4), ctqw.FLAG_TILED(5), ctqw.FLAG_TILED(6),
    ctqw.FLAG_PLAIN,
)

DEFAULT_CACHE = os.environ.get(
    "CTQW_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "ctqw_autotune.json"))


def cache_key(h: ctqw.Hamiltonian, dtype: int, K: int) -> str:
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    sizes = ",".join(str(n) for n in h.group_sizes)
    return (f"m{h.m}|N{sizes}|R{h.R}|p{int(h.periodic)}|dtype{dtype}|K{K}|"
            f"{props.name}|sm{props.multi_processor_count}")


def _load(path: str) -> Dict[str, dict]:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, table: Dict[str, dict]) -> None:
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_candidates(h: ctqw.Hamiltonian, psi: torch.Tensor, dtype: int, dt: float, K: int,
                    steps: int = 4, candidates: Iterable[int] = CANDIDATES) -> List[Tuple[int, float]]:
    """(flags, ms per step) of every candidate the handle supports.

    psi is not modified: each candidate runs on a scratch copy.
    """
    stream = torch.cuda.current_stream()
    out = []
    scratch = torch.empty_like(psi)
    for flags in candidates:
        try:
            ws = h.workspace(dtype, ctqw.TAYLOR, flags, psi.device)
        except ctqw.CtqwError:
            continue
        try:
            scratch.copy_(psi)
            ctqw.ctqw_propagate_taylor(h, scratch, dtype, dt, K, 1, 0, None, None, None, flags, ws)
        except ctqw.CtqwError as e:
            # a shape not compiled for this size, or a path this handle cannot take
            if e.status in (ctqw.CTQW_EUNSUPPORTED, ctqw.CTQW_EINVAL):
                continue
            raise
        scratch.copy_(psi)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctqw.ctqw_propagate_taylor(h, scratch, dtype, dt, K, steps, 0, None, None, None, flags, ws)
        e1.record(stream)
        e1.synchronize()
        ctqw.ctqw_check_status(h)
        out.append((flags, e0.elapsed_time(e1) / steps))
    return out


def tuned_flags(h: ctqw.Hamiltonian, psi: torch.Tensor, dtype: int, dt: float, K: int,
                steps: int = 4, cache_path: Optional[str] = DEFAULT_CACHE,
                candidates: Iterable[int] = CANDIDATES) -> int:
    """Flag word of the fastest supported candidate (from the cache when known)."""
    key = cache_key(h, dtype, K)
    table = _load(cache_path) if cache_path else {}
    if key in table:
        return int(table[key]["flags"])
    timings = time_candidates(h, psi, dtype, dt, K, steps, candidates)
    if not timings:
        raise RuntimeError("autotune: no candidate supports this handle")
    best, best_ms = min(timings, key=lambda t: t[1])
    if cache_path:
        table = _load(cache_path)
        table[key] = {"flags": best, "ms_per_step": best_ms,
                      "timings": {str(f): ms for f, ms in timings}}
        _store(cache_path, table)
    return best


def tune(h: ctqw.Hamiltonian, psi: torch.Tensor, dtype: int, dt: float, n_steps: int,
         K_min: int = 1, K_max: int = 30, steps: int = 4, cache_path: Optional[str] = DEFAULT_CACHE,
         candidates: Iterable[int] = CANDIDATES) -> Tuple[int, int]:
    """(K, flags) for a propagation of n_steps steps of dt on this handle.

    K is the smallest order in K_min..K_max whose summed truncation bound
    stays within a tenth of the type's tolerance (ctqw_autotune_order; a
    larger K only costs time), then flags the fastest kernel shape for that
    K: for a ragged batch the tiled kernels at every compiled depth and
    region, and the per-term path.
    """
    K = ctqw.ctqw_autotune_order(h, dtype, dt, n_steps, K_min, K_max)
    return K, tuned_flags(h, psi, dtype, dt, K, steps, cache_path, candidates)
