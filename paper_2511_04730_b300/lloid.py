"""Python binding of the LLOID C ABI (argument marshalling only).

Every step of the hot path runs in the CUDA library; this module converts
arguments (numpy arrays, torch tensors, streams) to the plain pointers and
sizes of ``include/lloid.h`` and raises ``LloidError`` on a non-OK status.
"""
from __future__ import annotations

import ctypes
from typing import Iterable, Optional

import numpy as np

from . import _lib

TRIGGER_DTYPE = np.dtype([
    ("detector", np.int32), ("bank", np.int32), ("tmpl", np.int32), ("is_bank_max", np.int32),
    ("window", np.int64), ("sample", np.int64), ("snr", np.float32), ("phase", np.float32),
    ("re", np.float32), ("im", np.float32), ("xi2", np.float32), ("pad", np.int32),
])
assert TRIGGER_DTYPE.itemsize == ctypes.sizeof(_lib.LloidTrigger)
EVENT_DTYPE = np.dtype([
    ("window", np.int64), ("bank", np.int32), ("tmpl", np.int32), ("n_ifo", np.int32), ("ifo_mask", np.uint32),
    ("net_snr", np.float32), ("ref_detector", np.int32), ("ref_sample", np.int64),
])
assert EVENT_DTYPE.itemsize == ctypes.sizeof(_lib.LloidEvent)


class LloidError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_lib.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status
        self.name = _lib.STATUS_NAMES.get(status, str(status))


def default_config() -> _lib.LloidConfig:
    lib = _lib.load()
    cfg = _lib.LloidConfig()
    lib.lloid_config_default(ctypes.byref(cfg))
    return cfg


def _bank_desc(slices: Iterable, autocorr=None):
    """lloid_bank_desc of a bank (and the arrays it points to, to keep alive)."""
    slices = list(slices)
    keep = []
    arr = (_lib.LloidSlice * len(slices))()
    n_rows = None
    for i, s in enumerate(slices):
        b = np.ascontiguousarray(s.bases, dtype=np.float64)
        c = np.ascontiguousarray(s.coeffs, dtype=np.float64)
        keep += [b, c]
        if n_rows is None:
            n_rows = c.shape[0]
        arr[i].rate, arr[i].n_taps, arr[i].j_start = int(s.rate), int(b.shape[1]), int(s.j_start)
        arr[i].n_basis = int(b.shape[0])
        arr[i].bases = b.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        arr[i].coeffs = c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        if c.shape != (n_rows, b.shape[0]):
            raise ValueError("coeffs must be [2M, L] with one 2M for the bank")
    keep.append(arr)
    desc = _lib.LloidBankDesc(n_rows // 2, len(slices), arr)
    if autocorr is not None:
        ac = np.asarray(autocorr, dtype=np.complex128)
        if ac.ndim != 2 or ac.shape[0] != n_rows // 2 or ac.shape[1] % 2 != 1:
            raise ValueError("autocorr must be [M, 2d + 1] complex")
        acf = np.ascontiguousarray(ac.view(np.float64).reshape(ac.shape[0], ac.shape[1], 2))
        keep.append(acf)
        desc.ac_half = (ac.shape[1] - 1) // 2
        desc.autocorr = acf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return desc, keep, n_rows


def autotune(banks, n: int, reps: int = 4, n_detectors: int = 1, precision: str = "bf16_split",
             max_block: Optional[int] = None, max_history: Optional[int] = None, device: int = 0,
             f0: int = 2048, window: int = 2048) -> dict:
    """lloid_autotune: time the candidate forms and basis-filter occupancies on
    scratch contexts with these banks and pushes of n samples; returns the
    chosen setting (pass it as Context(tuning=...)) with every candidate's
    device time per push."""
    lib = _lib.load()
    cfg = default_config()
    cfg.f0, cfg.n_detectors, cfg.window_samples = f0, n_detectors, window
    cfg.precision = _lib.PRECISIONS[precision]
    cfg.max_block = n if max_block is None else max_block
    if max_history is not None:
        cfg.max_history = max_history
    cfg.device = device
    descs = (_lib.LloidBankDesc * len(banks))()
    keep = []
    for i, b in enumerate(banks):
        d, k, _ = _bank_desc(b)
        descs[i] = d
        keep.append(k)
    out = _lib.LloidTuning()
    st = lib.lloid_autotune(ctypes.byref(cfg), ctypes.cast(descs, ctypes.c_void_p), len(banks), n, reps,
                            ctypes.byref(out))
    if st != 0:
        raise LloidError(st, "lloid_autotune failed")
    names = {0: "by ratio", 2: "all ladder", 4: "all f0"}
    cands = [{"form": names.get(out.cand_flags[i], "?"), "form_ratio": out.cand_ratio[i],
              "fir_ctas": out.cand_ctas[i], "ms_per_push": out.ms[i]} for i in range(out.n_tried)]
    return {"form_ratio": out.form_ratio, "flags_form": out.flags_form, "fir_ctas": out.fir_ctas,
            "best": out.best, "candidates": cands}


class Context:
    """One LLOID streaming context on one GPU (``lloid_create``)."""

    def __init__(self, n_detectors: int = 1, precision: str = "fp32", max_block: int = 16384,
                 max_history: Optional[int] = None, window: int = 2048, threshold: float = 4.0,
                 device: int = 0, stream=None, hbm_budget: int = 0, f0: int = 2048, min_rate: int = 32,
                 n_down: int = 32, n_up: int = 8, stage_timing: bool = False, coinc_window: Optional[int] = None,
                 form: Optional[str] = None, fill_gaps: bool = False, overlap: int = 0,
                 tuning: Optional[dict] = None):
        self._lib = _lib.load()
        cfg = default_config()
        cfg.f0, cfg.n_detectors, cfg.n_down, cfg.n_up = f0, n_detectors, n_down, n_up
        cfg.window_samples, cfg.snr_threshold = window, threshold
        cfg.window_overlap = overlap
        cfg.precision = _lib.PRECISIONS[precision]
        cfg.max_block = max_block
        if max_history is not None:
            cfg.max_history = max_history
        cfg.min_rate, cfg.device, cfg.hbm_budget_bytes = min_rate, device, hbm_budget
        if coinc_window is not None:
            cfg.coinc_window = coinc_window
        cfg.cuda_stream = None if stream is None else ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        if form not in _lib.FORM_FLAGS:
            raise ValueError(f"form must be one of {sorted(k for k in _lib.FORM_FLAGS if k)} or None")
        cfg.flags = ((_lib.FLAG_STAGE_TIMING if stage_timing else 0) | _lib.FORM_FLAGS[form] |
                     (_lib.FLAG_FILL_GAPS if fill_gaps else 0))
        if tuning is not None:          # the result of autotune()
            if form is None:
                cfg.flags |= tuning["flags_form"]
            cfg.form_ratio, cfg.fir_ctas = tuning["form_ratio"], tuning["fir_ctas"]
        self.cfg = cfg
        self.precision = precision
        self.n_detectors = n_detectors
        self.window = window
        h = ctypes.c_void_p()
        st = self._lib.lloid_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != 0:
            raise LloidError(st, "lloid_create failed (bad configuration or device error)")
        self._h = h
        self.banks = {}
        self.stream_ptr = int(self._lib.lloid_stream(h) or 0)
        self._ext_stream = None

    # -- helpers --------------------------------------------------------------
    def _check(self, st: int):
        if st != 0:
            msg = self._lib.lloid_last_error(self._h).decode()
            raise LloidError(st, msg)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lloid_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- banks ----------------------------------------------------------------
    def load_bank(self, slices: Iterable, autocorr=None) -> int:
        """Load an SVD bank given as objects with rate, j_start, bases [L, N]
        and coeffs [2M, L] (float64); optional autocorr [M, 2d + 1] complex
        (R_i(t), t = -d .. d) enables the Eq. 10 statistic for its triggers.
        Returns the bank id."""
        desc, keep, n_rows = _bank_desc(slices, autocorr)
        bid = ctypes.c_int32()
        self._check(self._lib.lloid_load_bank(self._h, ctypes.byref(desc), ctypes.byref(bid)))
        self.banks[bid.value] = n_rows // 2
        return bid.value

    def bank_form(self, bank_id: int) -> str:
        """Form a bank runs in on the split path: "ladder" or "f0" (lloid_bank_form)."""
        f = int(self._lib.lloid_bank_form(self._h, bank_id))
        if f < 0:
            self._check(-1)
        return "f0" if f == 1 else "ladder"

    def inject_fault(self, kind: str, count: int = 1):
        """lloid_inject_fault: "alloc", "drop_block", "delay" (microseconds) or
        "wait_expiry" (microseconds)."""
        self._check(self._lib.lloid_inject_fault(self._h, _lib.FAULTS[kind], int(count)))

    def clear_error(self):
        """lloid_clear_error: forget an expired device wait."""
        self._check(self._lib.lloid_clear_error(self._h))

    def unload_bank(self, bank_id: int):
        self._check(self._lib.lloid_unload_bank(self._h, bank_id))
        self.banks.pop(bank_id, None)

    # -- streaming ------------------------------------------------------------
    @staticmethod
    def _ptr(block):
        """(pointer, n, is_device) for a float32 numpy array or torch tensor."""
        if isinstance(block, np.ndarray):
            if block.dtype != np.float32 or not block.flags.c_contiguous:
                raise ValueError("host blocks must be C-contiguous float32")
            return block.ctypes.data, block.shape[-1], 0
        import torch
        if not isinstance(block, torch.Tensor) or block.dtype != torch.float32 or not block.is_contiguous():
            raise ValueError("blocks must be contiguous float32 numpy arrays or torch tensors")
        return block.data_ptr(), block.shape[-1], 1 if block.is_cuda else 0

    def _after_torch(self):
        """Order the library stream after torch's current stream (device inputs/outputs)."""
        import torch
        if self._ext_stream is None:
            self._ext_stream = torch.cuda.ExternalStream(self.stream_ptr, device=f"cuda:{self.cfg.device}")
        cur = torch.cuda.current_stream(self.cfg.device)
        if cur.cuda_stream != self.stream_ptr:
            self._ext_stream.wait_stream(cur)

    def _torch_after(self):
        """Order torch's current stream after the library's reads of a device
        block, so the caching allocator cannot hand the block's memory to new
        work before the library has consumed it."""
        import torch
        cur = torch.cuda.current_stream(self.cfg.device)
        if cur.cuda_stream != self.stream_ptr:
            cur.wait_stream(self._ext_stream)

    def push(self, det: int, t0: int, block):
        p, n, dev = self._ptr(block)
        if dev:
            self._after_torch()
        self._check(self._lib.lloid_push_strain(self._h, det, t0, ctypes.c_void_p(p), n, dev))
        if dev:
            self._torch_after()

    def push_all(self, t0: int, blocks):
        p, n, dev = self._ptr(blocks)
        if dev:
            self._after_torch()
        self._check(self._lib.lloid_push_strain_all(self._h, t0, ctypes.c_void_p(p), n, dev))
        if dev:
            self._torch_after()

    def pull(self, window: int, timeout_ms: int = -1, n_windows: int = 1) -> np.ndarray:
        """Triggers of windows window .. window + n_windows - 1 as a numpy
        structured array (TRIGGER_DTYPE)."""
        n_out = ctypes.c_int64()
        if getattr(self, "_pull_buf", None) is None:
            self._pull_buf = np.empty(1 << 14, dtype=TRIGGER_DTYPE)
        while True:
            out = self._pull_buf
            st = self._lib.lloid_pull_triggers_range(self._h, window, n_windows,
                                                     out.ctypes.data_as(ctypes.POINTER(_lib.LloidTrigger)),
                                                     out.size, ctypes.byref(n_out), timeout_ms)
            if st == -8:   # ERANGE: grow the reusable buffer and retry
                self._pull_buf = np.empty(int(n_out.value) * 2, dtype=TRIGGER_DTYPE)
                continue
            self._check(st)
            return out[: n_out.value].copy()

    def pull_submit(self, window: int, n_windows: int = 1) -> int:
        """Start a pull of windows window .. window + n_windows - 1 behind the
        pushes already enqueued; returns a ticket for pull_collect."""
        t = ctypes.c_int32()
        self._check(self._lib.lloid_pull_submit(self._h, window, n_windows, ctypes.byref(t)))
        return int(t.value)

    def pull_collect(self, ticket: int, timeout_ms: int = -1) -> np.ndarray:
        """Triggers of a submitted pull (TRIGGER_DTYPE), once its copy has landed."""
        n_out = ctypes.c_int64()
        st = self._lib.lloid_pull_collect(self._h, ticket, None, 0, ctypes.byref(n_out), timeout_ms)
        if st == 0:
            return np.zeros(0, dtype=TRIGGER_DTYPE)
        if st != -8:
            self._check(st)
        out = np.empty(int(n_out.value), dtype=TRIGGER_DTYPE)
        self._check(self._lib.lloid_pull_collect(self._h, ticket, out.ctypes.data_as(ctypes.POINTER(_lib.LloidTrigger)),
                                                 out.size, ctypes.byref(n_out), timeout_ms))
        return out[: n_out.value]

    def set_background_bins(self, snr_edges, xi2_edges):
        """Start background collection (Section II.D.5) on these ascending edges."""
        se = np.ascontiguousarray(snr_edges, dtype=np.float32)
        xe = np.ascontiguousarray(xi2_edges, dtype=np.float32)
        self._bg_shape = (self.n_detectors, se.size - 1, xe.size - 1)
        self._check(self._lib.lloid_set_background_bins(
            self._h, se.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), se.size - 1,
            xe.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), xe.size - 1))

    def background(self, bank: int) -> np.ndarray:
        """Counts [n_detectors, n_snr, n_xi2] of a bank's single-detector triggers."""
        out = np.zeros(self._bg_shape, dtype=np.uint32)
        self._check(self._lib.lloid_get_background(self._h, bank, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                                   out.size))
        return out

    def pull_events(self, window: int, n_windows: int = 1, timeout_ms: int = -1) -> np.ndarray:
        """Coincident events (at most one per bank and window) of windows
        window .. window + n_windows - 1 as a numpy structured array (EVENT_DTYPE)."""
        n_out = ctypes.c_int64()
        cap = 256
        while True:
            out = np.empty(cap, dtype=EVENT_DTYPE)
            st = self._lib.lloid_pull_events(self._h, window, n_windows,
                                             out.ctypes.data_as(ctypes.POINTER(_lib.LloidEvent)), cap,
                                             ctypes.byref(n_out), timeout_ms)
            if st == -8:
                cap = int(n_out.value)
                continue
            self._check(st)
            return out[: n_out.value].copy()

    def snr_block(self, det: int, bank: int):
        """SNR rows [2M, n] of the last push of ``det`` for ``bank`` (torch, on device)."""
        import torch
        M = self.banks[bank]
        n = ctypes.c_int64()
        t0 = ctypes.c_int64()
        cap = ctypes.c_int64(0)
        # ask for the size first
        st = self._lib.lloid_snr_block(self._h, det, bank, None, 0, ctypes.byref(t0), ctypes.byref(n))
        if st not in (0, -8):
            self._check(st)
        out = torch.empty((2 * M, int(n.value)), dtype=torch.float32, device=f"cuda:{self.cfg.device}")
        self._after_torch()
        self._check(self._lib.lloid_snr_block(self._h, det, bank, ctypes.c_void_p(out.data_ptr()), out.numel(),
                                              ctypes.byref(t0), ctypes.byref(n)))
        return out, int(t0.value)

    def save_state(self) -> bytes:
        """Checkpoint of the streaming state (lloid_save_state)."""
        n = ctypes.c_size_t(0)
        self._check(self._lib.lloid_save_state(self._h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._check(self._lib.lloid_save_state(self._h, buf, ctypes.byref(n)))
        return buf.raw[: n.value]

    def restore_state(self, blob: bytes):
        """Resume from save_state() output (same configuration and banks)."""
        self._check(self._lib.lloid_restore_state(self._h, blob, len(blob)))

    def synchronize(self):
        self._check(self._lib.lloid_synchronize(self._h))

    def launch_count(self) -> int:
        return int(self._lib.lloid_launch_count(self._h))

    def bytes_in_use(self):
        """(state bytes, bank bytes) held on the device."""
        a, b = ctypes.c_size_t(), ctypes.c_size_t()
        self._check(self._lib.lloid_bytes_in_use(self._h, ctypes.byref(a), ctypes.byref(b)))
        return int(a.value), int(b.value)

    def stage_times(self, reset: bool = False) -> dict:
        """{stage: (milliseconds, launches)} since the last reset (needs stage_timing=True)."""
        ms = (ctypes.c_double * _lib.N_STAGES)()
        ln = (ctypes.c_int64 * _lib.N_STAGES)()
        self._check(self._lib.lloid_stage_times(self._h, ms, ln, 1 if reset else 0))
        return {name: (ms[i], int(ln[i])) for i, name in enumerate(_lib.STAGE_NAMES)}


def triggers_from_snr_noalloc(z, t0: int, window: int = 2048, threshold: float = 4.0, detector: int = 0,
                              bank: int = 0, out=None, n_out=None, stream=None):
    """Allocation-free trigger extraction for an SNR block already on the GPU.

    For callers that must not allocate device memory while they run: the
    library call itself uses only its compiled-in scratch.  ``z`` is a
    contiguous float32 CUDA tensor [2M, n]; ``out`` (uint8 CUDA tensor of
    cap * 48 bytes) and ``n_out`` (int64 CUDA tensor of one element) are
    preallocated by the caller, or allocated here for convenience.  Returns
    the triggers as a numpy structured array (this read-back synchronises)."""
    import torch
    lib = _lib.load()
    if not isinstance(z, torch.Tensor) or not z.is_cuda or z.dtype != torch.float32 or not z.is_contiguous() \
            or z.dim() != 2 or z.shape[0] % 2:
        raise ValueError("z must be a contiguous float32 CUDA tensor [2M, n]")
    n_rows, n = z.shape
    for name, t, dt in (("out", out, torch.uint8), ("n_out", n_out, torch.int64)):
        if t is not None and (not isinstance(t, torch.Tensor) or t.device != z.device or t.dtype != dt
                              or not t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous {dt} tensor on {z.device}")
    if out is None:
        out = torch.empty((n_rows // 2) * (n // window) * TRIGGER_DTYPE.itemsize, dtype=torch.uint8, device=z.device)
    if n_out is None:
        n_out = torch.zeros(1, dtype=torch.int64, device=z.device)
    cap = out.numel() // TRIGGER_DTYPE.itemsize
    s = torch.cuda.current_stream(z.device) if stream is None else stream
    st = lib.lloid_triggers_from_snr_noalloc(ctypes.c_void_p(z.data_ptr()), n_rows // 2, n, t0, window, threshold,
                                             detector, bank, ctypes.c_void_p(out.data_ptr()), cap,
                                             ctypes.c_void_p(n_out.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    if st != 0:
        raise LloidError(st, "lloid_triggers_from_snr_noalloc failed")
    k = int(n_out.item())
    return np.frombuffer(out[: min(k, cap) * TRIGGER_DTYPE.itemsize].cpu().numpy().tobytes(), dtype=TRIGGER_DTYPE)


class Whitener:
    """PSD estimation and whitening (Section II.B.2) on the GPU
    (``lloid_whitener_create``); output feeds ``Context.push``."""

    def __init__(self, rate_in: int = 16384, rate_out: int = 2048, n_fft: Optional[int] = None,
                 z_pad: Optional[int] = None, n_med: int = 7, n_avg: int = 64, n_detectors: int = 1,
                 max_push: Optional[int] = None, device: int = 0):
        self._lib = _lib.load()
        cfg = _lib.LloidWhitenerConfig()
        self._lib.lloid_whitener_config_default(ctypes.byref(cfg))
        cfg.rate_in, cfg.rate_out = rate_in, rate_out
        cfg.n_fft = 4 * rate_in if n_fft is None else n_fft
        cfg.z_pad = rate_in if z_pad is None else z_pad
        cfg.n_med, cfg.n_avg, cfg.n_detectors, cfg.device = n_med, n_avg, n_detectors, device
        cfg.max_push = 16 * rate_in if max_push is None else max_push
        self.hop = cfg.n_fft // 2 - cfg.z_pad
        self.ratio = rate_in // rate_out
        self.n_bins = cfg.n_fft // self.ratio // 2 + 1
        h = ctypes.c_void_p()
        st = self._lib.lloid_whitener_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != 0:
            raise LloidError(st, "lloid_whitener_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lloid_whitener_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def whiten(self, det: int, block: np.ndarray) -> np.ndarray:
        """Append input samples (a multiple of the hop); return the final output samples."""
        x = np.ascontiguousarray(block, dtype=np.float32)
        out = np.empty(x.size // self.ratio + 1, dtype=np.float32)
        n_out = ctypes.c_int64()
        st = self._lib.lloid_whiten(self._h, det, x.ctypes.data_as(ctypes.c_void_p), x.size, 0,
                                    out.ctypes.data_as(ctypes.c_void_p), out.size, ctypes.byref(n_out), 0)
        if st != 0:
            raise LloidError(st, "lloid_whiten")
        return out[: n_out.value].copy()

    def psd(self, det: int = 0) -> np.ndarray:
        out = np.empty(self.n_bins, dtype=np.float32)
        st = self._lib.lloid_whitener_psd(self._h, det, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), out.size)
        if st != 0:
            raise LloidError(st, "lloid_whitener_psd")
        return out
