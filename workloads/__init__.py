"""Seeded synthetic workloads for the LLOID hot path.

This module is the one piece of code shared by the FP64 oracle (``oracle/``)
and the CUDA product path (``paper_2511_04730_b300``).  It only *generates
inputs*: Newtonian chirp templates, the time-slice plan of a bank, white
Gaussian strain and injections.  It holds none of the filtering arithmetic of
the method (no SVD, no resampling, no correlation, no reconstruction, no
trigger finding); each side implements those on its own.

Conventions
-----------
* ``f0`` is the full sample rate (2048 Hz in every workload).
* A template is indexed by ``j`` = samples *before merger* at the full rate,
  ``tau = j / f0`` seconds.  Row ``2i`` of a bank is the cosine part
  ``h_c`` of template ``i`` and row ``2i+1`` its sine part ``h_s`` (the paper
  filters the real and imaginary parts of each complex template as two real
  filters, Section II.C, matched-filter definition Eq. 1).
* Data are already whitened (unit-variance white noise), so the whitened
  template is the template itself.

Input recipe (stands in for the paper's O3 mock-data challenge strain and O4
template bank, which are not available):
* chirps: leading-order (Newtonian) inspiral, ``f(tau)``, ``phi(tau)``,
  amplitude ``tau^-1/4``, support from the ISCO frequency (capped at
  ``0.4 f0``) down to 30 Hz, Tukey(0.1) taper over the support, ``h_c`` and
  ``h_s`` each normalised to unit L2 norm in FP64;
* slice boundaries on a fixed ladder of seconds before merger; each slice's
  rate is the smallest power of two ``r`` (within ``[r_min, f0]``) whose
  ``0.4 r`` bounds the highest template frequency in the slice (the paper
  samples each slice at the Nyquist rate of its highest frequency content,
  Section II.C.1); the slice nearest merger always runs at ``f0``;
* strain: i.i.d. N(0, 1) float32 at ``f0`` from numpy PCG64;
* injections: ``A (cos phi0 h_c + sin phi0 h_s)`` of a bank template ending at
  a seeded sample, which a matched filter recovers as ``|z| = A``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

F0 = 2048
T_SUN = 4.925491e-6          # G M_sun / c^3 in seconds
F_LOW = 30.0                 # lower frequency of every template (Hz)
ISCO_NUM = 4397.0            # f_ISCO ~ 4397 Hz / (M_total / M_sun)
TUKEY_ALPHA = 0.1
DEFAULT_BOUNDARIES_S = (0.0, 0.25, 0.5, 1.0, 2.0, 4.0, 8.0, 16.0, 32.0, 64.0, 128.0)
N_DOWN_DESIGN, N_UP_DESIGN = 32, 8    # filter half-lengths the slice plan must leave room for


# ----------------------------------------------------------------------------
# Newtonian chirp physics (leading-order post-Newtonian inspiral)
# ----------------------------------------------------------------------------

def tau_of_f(f, mchirp):
    """Time before merger (s) at GW frequency f (Hz), leading order."""
    m = T_SUN * mchirp
    return (5.0 / 256.0) * m ** (-5.0 / 3.0) * (math.pi * np.asarray(f, dtype=np.float64)) ** (-8.0 / 3.0)


def f_of_tau(tau, mchirp):
    """GW frequency (Hz) at time before merger tau (s), leading order."""
    m = T_SUN * mchirp
    tau = np.asarray(tau, dtype=np.float64)
    return (1.0 / math.pi) * (5.0 / (256.0 * tau)) ** 0.375 * m ** (-0.625)


def phase_of_tau(tau, mchirp):
    """Orbital-phase-derived GW phase at time before merger tau (s)."""
    m = T_SUN * mchirp
    return -2.0 * (5.0 * m) ** (-0.625) * np.asarray(tau, dtype=np.float64) ** 0.625


def f_end(mchirp, f0=F0):
    """Upper frequency: ISCO of an equal-mass binary, capped at 0.4 f0."""
    m_total = 2.0 ** 1.2 * mchirp
    return min(ISCO_NUM / m_total, 0.4 * f0)


def _tukey(n_support, pos, alpha=TUKEY_ALPHA):
    """Tukey window of length n_support evaluated at integer positions pos."""
    pos = np.asarray(pos, dtype=np.float64)
    if n_support <= 1:
        return np.ones_like(pos)
    x = pos / (n_support - 1)
    w = np.ones_like(x)
    edge = alpha / 2.0
    lo = x < edge
    hi = x > 1.0 - edge
    w[lo] = 0.5 * (1.0 + np.cos(math.pi * (2.0 * x[lo] / alpha - 1.0)))
    w[hi] = 0.5 * (1.0 + np.cos(math.pi * (2.0 * x[hi] / alpha - 2.0 / alpha + 1.0)))
    return w


@dataclasses.dataclass
class ChirpBank:
    """A set of M Newtonian chirp templates (2M real rows), evaluated lazily.

    ``rows(j)`` returns the FP64 samples of every row at the full-rate
    before-merger indices ``j`` so that long templates never have to be held at
    the full rate.
    """

    mchirp: np.ndarray            # [M] chirp masses (M_sun)
    n_samples: int                # bank length in full-rate samples
    f0: int = F0
    j_lo: np.ndarray = None       # [M] first support sample (nearest merger)
    j_hi: np.ndarray = None       # [M] one past the last support sample
    norm_c: np.ndarray = None     # [M] L2 norms before normalisation
    norm_s: np.ndarray = None

    def __post_init__(self):
        self.mchirp = np.asarray(self.mchirp, dtype=np.float64)
        M = self.mchirp.size
        self.j_lo = np.empty(M, dtype=np.int64)
        self.j_hi = np.empty(M, dtype=np.int64)
        for i, mc in enumerate(self.mchirp):
            t_end = float(tau_of_f(f_end(mc, self.f0), mc))
            t_low = float(tau_of_f(F_LOW, mc))
            self.j_lo[i] = int(math.ceil(t_end * self.f0))
            self.j_hi[i] = min(int(math.floor(t_low * self.f0)) + 1, self.n_samples)
            if self.j_hi[i] <= self.j_lo[i] + 1:
                raise ValueError(f"template {i} (Mc={mc}) has empty support")
        # Unit-normalise h_c and h_s separately (FP64) over each support.
        self.norm_c = np.empty(M)
        self.norm_s = np.empty(M)
        for i in range(M):
            hc, hs = self._one(i, np.arange(self.j_lo[i], self.j_hi[i]))
            self.norm_c[i] = math.sqrt(float(np.einsum("i,i->", hc, hc)))
            self.norm_s[i] = math.sqrt(float(np.einsum("i,i->", hs, hs)))

    @property
    def n_templates(self) -> int:
        return int(self.mchirp.size)

    @property
    def n_rows(self) -> int:
        return 2 * self.n_templates

    def _one(self, i: int, jj: np.ndarray) -> tuple:
        """Unnormalised (h_c, h_s) of template i at samples jj, all inside its support."""
        t = jj / float(self.f0)
        amp = t ** -0.25
        ph = phase_of_tau(t, self.mchirp[i])
        win = _tukey(int(self.j_hi[i] - self.j_lo[i]), jj - self.j_lo[i])
        g = amp * win
        return g * np.cos(ph), g * np.sin(ph)

    def _raw(self, j, which=None):
        """Unnormalised rows [2M', len(j)] at before-merger samples j.  When j
        is an arithmetic progression (every use here) each template is only
        evaluated on the part of j inside its support."""
        j = np.asarray(j, dtype=np.int64)
        idx = range(self.mchirp.size) if which is None else list(which)
        out = np.zeros((2 * len(idx), j.size), dtype=np.float64)
        step = int(j[1] - j[0]) if j.size > 1 else 1
        regular = j.size > 1 and step > 0 and np.all(np.diff(j) == step)
        for o, i in enumerate(idx):
            lo, hi = int(self.j_lo[i]), int(self.j_hi[i])
            if regular:
                m0 = max(0, -(-(lo - int(j[0])) // step))
                m1 = min(j.size, -(-(hi - int(j[0])) // step))
                if m1 <= m0:
                    continue
                hc, hs = self._one(i, j[m0:m1])
                out[2 * o, m0:m1] = hc
                out[2 * o + 1, m0:m1] = hs
            else:
                sel = (j >= lo) & (j < hi)
                if not np.any(sel):
                    continue
                hc, hs = self._one(i, j[sel])
                out[2 * o, sel] = hc
                out[2 * o + 1, sel] = hs
        return out

    def rows(self, j, which=None) -> np.ndarray:
        """FP64 samples [2M, len(j)] of the unit-norm rows at before-merger
        indices j (only templates ``which``, in that order, if given)."""
        r = self._raw(j, which)
        idx = np.arange(self.mchirp.size) if which is None else np.asarray(list(which))
        r[0::2] /= self.norm_c[idx, None]
        r[1::2] /= self.norm_s[idx, None]
        return r

    def full(self) -> np.ndarray:
        """All rows at the full rate, [2M, n_samples] (small banks only)."""
        return self.rows(np.arange(self.n_samples))

    def max_freq_in(self, j_start: int, j_stop: int) -> float:
        """Highest GW frequency any template reaches in [j_start, j_stop)."""
        best = 0.0
        for i, mc in enumerate(self.mchirp):
            a = max(j_start, int(self.j_lo[i]))
            b = min(j_stop, int(self.j_hi[i]))
            if b <= a:
                continue
            best = max(best, float(f_of_tau(a / float(self.f0), mc)))
        return best


# ----------------------------------------------------------------------------
# Slice plan
# ----------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class SlicePlan:
    """Time slices of a bank: slice s spans before-merger full-rate samples
    [j_start[s], j_start[s] + n_taps[s] * (f0 // rate[s])) and is sampled at
    rate[s]; ``n_taps[s]`` is its length at that rate."""

    rate: tuple
    j_start: tuple
    n_taps: tuple

    @property
    def n_slices(self) -> int:
        return len(self.rate)


def plan_slices(bank: ChirpBank, boundaries_s: Sequence[float] = DEFAULT_BOUNDARIES_S,
                r_min: int = 128, fixed_rates: Optional[Sequence[int]] = None) -> SlicePlan:
    """Cut the bank into time slices and pick each slice's power-of-two rate.

    Slices whose templates are all zero are dropped.  With ``fixed_rates`` the
    rates are taken as given (the 64-template workload fixes them).
    """
    f0 = bank.f0
    edges = [int(round(b * f0)) for b in boundaries_s]
    edges = [e for e in edges if e < bank.n_samples] + [bank.n_samples]
    rates, starts, taps = [], [], []
    for s in range(len(edges) - 1):
        a, b = edges[s], edges[s + 1]
        if b <= a:
            continue
        live = np.any((bank.j_lo < b) & (bank.j_hi > a))
        if not live:
            continue
        if fixed_rates is not None:
            r = int(fixed_rates[s])
        elif s == 0:
            r = f0
        else:
            fmax = bank.max_freq_in(a, b)
            r = r_min
            while r < f0 and 0.4 * r < fmax:
                r *= 2
            # pre-synchronisation (Eq. 9) needs the slice to start at least
            # D (N_down + sum of the ladder's N_up terms) < D (N_down + 2 N_up)
            # samples before merger: raise the rate until it does
            while r < f0 and a < (f0 // r) * (N_DOWN_DESIGN + 2 * N_UP_DESIGN):
                r *= 2
        D = f0 // r
        if a % D or (b - a) % D:
            raise ValueError("slice edges must be multiples of the decimation factor")
        rates.append(r)
        starts.append(a)
        taps.append((b - a) // D)
    return SlicePlan(tuple(rates), tuple(starts), tuple(taps))


# ----------------------------------------------------------------------------
# Strain and injections
# ----------------------------------------------------------------------------

def white_noise(n: int, seed: int) -> np.ndarray:
    """Unit-variance white Gaussian strain, float32, PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(n, dtype=np.float32)


@dataclasses.dataclass
class Injection:
    tmpl: int          # template index within the bank
    end_sample: int    # full-rate sample of the merger (template j = 0)
    snr: float         # amplitude A
    phase: float       # phi0


def draw_injections(n_inj: int, n_templates: int, n_data: int, tmpl_len: int,
                    snr_range, seed: int, f0: int = F0) -> List[Injection]:
    """Seeded injections: template uniform, end sample uniform in
    [tmpl_len + f0, n_data - f0), SNR uniform in snr_range, phase uniform."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = tmpl_len + f0, n_data - f0
    if n_inj == 0:
        return []
    if hi <= lo:
        raise ValueError("data too short for injections")
    out = []
    for _ in range(n_inj):
        out.append(Injection(int(rng.integers(0, n_templates)), int(rng.integers(lo, hi)),
                             float(rng.uniform(*snr_range)), float(rng.uniform(0.0, 2.0 * math.pi))))
    return out


def add_injection(strain: np.ndarray, bank: ChirpBank, inj: Injection) -> None:
    """strain[end - j] += A (cos phi0 h_c[j] + sin phi0 h_s[j]) in place."""
    i = inj.tmpl
    j = np.arange(int(bank.j_lo[i]), int(bank.j_hi[i]))
    j = j[inj.end_sample - j >= 0]
    j = j[inj.end_sample - j < strain.size]
    r = bank.rows(j, [i])
    sig = inj.snr * (math.cos(inj.phase) * r[0] + math.sin(inj.phase) * r[1])
    np.add.at(strain, inj.end_sample - j, sig.astype(strain.dtype))


# ----------------------------------------------------------------------------
# The paper-shaped workloads
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    banks: List[ChirpBank]
    plans: List[SlicePlan]
    n_det: int
    n_seconds: int
    injections: List[List[Injection]]   # per detector (bank index, injection)
    inj_bank: List[List[int]]
    f0: int = F0
    seed_base: int = 100

    @property
    def n_templates(self) -> int:
        return sum(b.n_templates for b in self.banks)

    def strain(self, det: int, n: Optional[int] = None) -> np.ndarray:
        """Seeded strain of one detector (noise + that detector's injections)."""
        n_total = self.n_seconds * self.f0
        d = white_noise(n_total, self.seed_base + det)
        for b, inj in zip(self.inj_bank[det], self.injections[det]):
            add_injection(d, self.banks[b], inj)
        return d if n is None else d[:n]


def _make_bank(args):
    mc, n_samples, f0 = args
    return ChirpBank(mc, n_samples, f0)


def _contiguous_banks(mchirp_sorted, sizes, n_seconds_fn, f0, workers: int = 1):
    jobs = []
    a = 0
    for sz in sizes:
        mc = mchirp_sorted[a:a + sz]
        a += sz
        jobs.append((mc, n_seconds_fn(mc) * f0, f0))
    if workers <= 1 or len(jobs) < 2:
        return [_make_bank(j) for j in jobs]
    import multiprocessing as mp
    import os
    saved = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS")}
    os.environ.update(OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1")   # one thread per worker
    try:
        with mp.get_context("spawn").Pool(workers) as pool:  # spawn: safe next to a CUDA context
            return pool.map(_make_bank, jobs, chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def make_workload(name: str, n_det: Optional[int] = None, n_seconds: Optional[int] = None,
                  n_templates: Optional[int] = None, n_banks: Optional[int] = None,
                  n_inj: Optional[int] = None, workers: int = 1,
                  bank_indices: Optional[Sequence[int]] = None) -> Workload:
    """Build one of the paper-shaped synthetic workloads by name.

    * ``tiny``   : 8 templates, Mc in [5, 15], 4 s, two slices; 16 s, 1 detector.
    * ``bank64`` : 64 templates, Mc U[5, 15], 8 s, slices [0, 1) s at 2048 Hz and
      [1, 8) s at 256 Hz; 64 s, 1 detector, one injection at SNR 12.
    * ``bank1000``: 1000 templates, Mc log-U[1, 20], durations clip(tau(30 Hz), 8, 64)
      s, slices 2048/1024/512/256/128 Hz; 1024 s, 2 detectors, 20 injections at
      SNR U[6, 20].
    * ``banks20``: 10,000 templates (Mc log-U[1, 20]) sorted by Mc and split into
      20 contiguous banks of 200-800 templates; 4096 s, 2 detectors, 100
      injections at SNR U[5, 25].
    * ``banks500``: 500 banks of U{100..1000} templates (Mc log-U[1, 50],
      durations clip(tau(30 Hz), 2, 128) s); 1024 s, 3 detectors.
    Any size argument overrides the default (used for bounded samples);
    ``workers`` > 1 builds multi-bank workloads in a process pool.
    ``bank_indices`` keeps only those banks of a multi-bank workload (the same
    banks, with the same templates, as in the full set), so that a few real
    banks of the 500-bank set can be used without building the other ones.
    """
    f0 = F0
    if name == "tiny":
        rng = np.random.Generator(np.random.PCG64(7))
        M = n_templates or 8
        bank = ChirpBank(np.sort(rng.uniform(8.0, 15.0, M)), 4 * f0, f0)
        plan = plan_slices(bank, (0.0, 1.0, 4.0), fixed_rates=(2048, 256))
        nd, ns = n_det or 1, n_seconds or 16
        inj = [[Injection(M // 2, 10 * f0 + 17, 12.0, 0.7)] if ns >= 12 else [] for _ in range(nd)]
        return Workload(name, [bank], [plan], nd, ns, inj, [[0] * len(x) for x in inj])
    if name == "bank64":
        rng = np.random.Generator(np.random.PCG64(1))
        M = n_templates or 64
        bank = ChirpBank(np.sort(rng.uniform(5.0, 15.0, M)), 8 * f0, f0)
        plan = plan_slices(bank, (0.0, 1.0, 8.0), fixed_rates=(2048, 256))
        nd, ns = n_det or 1, n_seconds or 64
        injs, ib = [], []
        for det in range(nd):
            x = draw_injections(n_inj if n_inj is not None else 1, M, ns * f0, bank.n_samples,
                                (12.0, 12.0), 200 + det)
            injs.append(x)
            ib.append([0] * len(x))
        return Workload(name, [bank], [plan], nd, ns, injs, ib)
    if name == "bank1000":
        rng = np.random.Generator(np.random.PCG64(1))
        M = n_templates or 1000
        mc = np.sort(np.exp(rng.uniform(math.log(1.0), math.log(20.0), M)))
        dur = int(np.clip(math.ceil(float(tau_of_f(F_LOW, mc.min()))), 8, 64))
        dur = 1 << int(math.ceil(math.log2(dur)))
        bank = ChirpBank(mc, dur * f0, f0)
        plan = plan_slices(bank, DEFAULT_BOUNDARIES_S, r_min=128)
        nd, ns = n_det or 2, n_seconds or 1024
        injs, ib = [], []
        k = 20 if n_inj is None else n_inj
        for det in range(nd):
            x = draw_injections(k, M, ns * f0, bank.n_samples, (6.0, 20.0), 200 + det)
            injs.append(x)
            ib.append([0] * len(x))
        return Workload(name, [bank], [plan], nd, ns, injs, ib)
    if name in ("banks20", "banks500"):
        if name == "banks20":
            total, nb, lo_mc, hi_mc, dmin, dmax, rmin = 10000, 20, 1.0, 20.0, 8, 64, 128
            nd_def, ns_def, inj_def, snr = 2, 4096, 100, (5.0, 25.0)
            size_lo, size_hi = 200, 800
        else:
            total, nb, lo_mc, hi_mc, dmin, dmax, rmin = None, 500, 1.0, 50.0, 2, 128, 32
            nd_def, ns_def, inj_def, snr = 3, 1024, 17, (6.0, 20.0)
            size_lo, size_hi = 100, 1000
        nb = n_banks or nb
        rng = np.random.Generator(np.random.PCG64(1))
        sizes = rng.integers(size_lo, size_hi + 1, nb).astype(np.float64)
        if total is not None:
            sizes = np.maximum(1, np.round(sizes * (n_templates or total) / sizes.sum())).astype(np.int64)
        else:
            sizes = sizes.astype(np.int64)
            if n_templates is not None:
                sizes = np.maximum(1, np.round(sizes * n_templates / sizes.sum())).astype(np.int64)
        mc = np.sort(np.exp(rng.uniform(math.log(lo_mc), math.log(hi_mc), int(sizes.sum()))))

        def dur_fn(m):
            d = int(np.clip(math.ceil(float(tau_of_f(F_LOW, m.min()))), dmin, dmax))
            return 1 << int(math.ceil(math.log2(d)))

        if bank_indices is not None:
            starts = np.concatenate([[0], np.cumsum(sizes)])
            keep = [int(i) for i in bank_indices]
            mc = np.concatenate([mc[starts[i]:starts[i + 1]] for i in keep])
            sizes = sizes[keep]
        banks = _contiguous_banks(mc, sizes, dur_fn, f0, workers)
        plans = [plan_slices(b, DEFAULT_BOUNDARIES_S, r_min=rmin) for b in banks]
        nd, ns = n_det or nd_def, n_seconds or ns_def
        injs, ib = [], []
        k = inj_def if n_inj is None else n_inj
        for det in range(nd):
            rr = np.random.Generator(np.random.PCG64(300 + det))
            x, bi = [], []
            for t in range(k):
                b = int(rr.integers(0, len(banks)))
                one = draw_injections(1, banks[b].n_templates, ns * f0,
                                      max(bb.n_samples for bb in banks), snr, 200 + 1000 * det + t)
                x += one
                bi.append(b)
            injs.append(x)
            ib.append(bi)
        return Workload(name, banks, plans, nd, ns, injs, ib)
    raise KeyError(name)
