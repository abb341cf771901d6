"""Streaming serve loop over one context: continuous batching of banks.

A *request* is a bank to filter.  Requests wait in FIFO order until
``lloid_load_bank`` accepts them under the context's HBM budget (it answers
LLOID_EBUDGET when memory is short); once admitted, a bank's work shares
every launch with the banks already running, so requests that arrive while
others are on the GPU overlap with them.  Finishing a request unloads its
bank and frees room for the next pending one.  Blocks of strain arrive from
all detectors at a fixed pace; the loop pushes each block as it arrives and
pulls the triggers of the windows it completes, recording the latency from
the block's arrival to its triggers on the host.

A bank admitted while the stream runs is exact from its second push on: the
detector streams it reads are always kept, but its own per-level history
starts empty.
"""
from __future__ import annotations

import collections
import time
from typing import Callable, Dict, List, Optional

import numpy as np

from .lloid import TRIGGER_DTYPE, Context, LloidError


class Server:
    def __init__(self, ctx: Context, block: int, f0: int = 2048):
        self.ctx = ctx
        self.block = block
        self.f0 = f0
        self.pending: collections.deque = collections.deque()
        self.running: Dict[int, object] = {}      # bank id -> request tag
        self.pos = 0
        self.latency_ms: List[float] = []
        self.admitted_at: Dict[object, int] = {}

    def submit(self, slices, tag=None):
        """Queue a bank (list of slices) for filtering."""
        self.pending.append((slices, tag))

    def finish(self, bank_id: int):
        """Unload a running bank (its request is done)."""
        self.ctx.unload_bank(bank_id)
        self.running.pop(bank_id, None)

    def admit(self) -> List[int]:
        """Load pending banks in FIFO order while the budget allows."""
        new = []
        while self.pending:
            slices, tag = self.pending[0]
            try:
                bid = self.ctx.load_bank(slices)
            except LloidError as e:
                if e.name == "LLOID_EBUDGET":
                    break
                raise
            self.pending.popleft()
            self.running[bid] = tag
            self.admitted_at[tag] = self.pos
            new.append(bid)
        return new

    def step(self, blocks: np.ndarray) -> np.ndarray:
        """Admit what fits, push one block for every detector, return the
        triggers of the windows the block completes."""
        self.admit()
        n = blocks.shape[-1]
        W = self.ctx.window
        w0 = self.pos // W
        self.ctx.push_all(self.pos, blocks)
        self.pos += n
        w1 = self.pos // W
        if w1 > w0:
            return self.ctx.pull(w0, n_windows=w1 - w0)
        return np.zeros(0, dtype=TRIGGER_DTYPE)

    def run_paced(self, source: Callable[[int], np.ndarray], n_blocks: int, pace: float = 1.0,
                  on_triggers: Optional[Callable] = None):
        """Feed n_blocks blocks at `pace` times real time; block k arrives at
        start + k * block_seconds / pace.  Latency = time its triggers are on
        the host - its arrival time."""
        dt = self.block / self.f0 / pace
        start = time.perf_counter() + dt
        for k in range(n_blocks):
            arrival = start + k * dt
            now = time.perf_counter()
            if now < arrival:
                time.sleep(arrival - now)
            trig = self.step(source(k))
            self.latency_ms.append(1000.0 * (time.perf_counter() - arrival))
            if on_triggers is not None:
                on_triggers(k, trig)

    def latency_summary(self) -> dict:
        if not self.latency_ms:
            return {}
        a = np.sort(np.asarray(self.latency_ms))
        q = lambda p: float(a[min(len(a) - 1, int(np.ceil(p * len(a))) - 1)])
        return {"p50": q(0.50), "p99": q(0.99), "p99.9": q(0.999), "max": float(a[-1]), "n": int(len(a))}
