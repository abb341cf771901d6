"""Bank sharding across GPUs (one process per GPU).

SVD banks are independent (Section II.C.3: banks are only stacked for
batching), so the multi-GPU path partitions banks across ranks and needs no
collective on the data path: every rank receives the same strain blocks and
filters its own banks.  Only the per-window trigger lists are gathered, on
the host, and merged in (window, detector, bank, template) order; the
loudest trigger of each (window, detector) across all banks is one small
reduction over at most one record per bank.
"""
from __future__ import annotations

from typing import Iterable, List, Sequence

import numpy as np


def bank_cost(slices, n_templates: int, f0: int = 2048) -> float:
    """Per detector-second FLOP of one bank: FIR 2 L N r plus reconstruction
    2 (2M) L r over its slices (the dominant terms of the filtering path)."""
    total = 0.0
    for s in slices:
        L, N = s.bases.shape
        total += 2.0 * L * N * s.rate + 4.0 * n_templates * L * s.rate
    return total


def assign_banks(costs: Sequence[float], world: int) -> List[List[int]]:
    """Longest-processing-time-first assignment: banks in decreasing cost,
    each to the currently least-loaded rank (ties to the lower rank)."""
    load = [0.0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for b in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(b)
        load[r] += costs[b]
    for lst in out:
        lst.sort()
    return out


def merge_triggers(parts: Iterable[np.ndarray]) -> np.ndarray:
    """Concatenate per-rank trigger arrays and order them by window,
    detector, bank, template (the single-GPU order)."""
    parts = [p for p in parts if p is not None and len(p)]
    if not parts:
        return np.zeros(0, dtype=_dtype())
    m = np.concatenate(parts)
    order = np.lexsort((m["tmpl"], m["bank"], m["detector"], m["window"]))
    return m[order]


def loudest_per_window(triggers: np.ndarray) -> np.ndarray:
    """The loudest trigger of each (window, detector) over all banks
    (lowest bank, then template, on ties)."""
    if len(triggers) == 0:
        return triggers
    key = np.lexsort((triggers["tmpl"], triggers["bank"], -triggers["snr"], triggers["detector"], triggers["window"]))
    t = triggers[key]
    first = np.ones(len(t), dtype=bool)
    first[1:] = (t["window"][1:] != t["window"][:-1]) | (t["detector"][1:] != t["detector"][:-1])
    return t[first]


def gather_triggers(local: np.ndarray, group=None) -> np.ndarray:
    """All ranks' triggers merged, returned on every rank (torch.distributed
    object all-gather; host memory only)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, local, group=group)
    return merge_triggers(parts)


def _dtype():
    from .lloid import TRIGGER_DTYPE
    return TRIGGER_DTYPE
