"""FP64 CPU oracle of the LLOID hot path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA path; the only common dependency is the seeded input generator
``workloads`` (templates, slice plans, noise, injections).

What it computes (every array is float64, every step written out plainly):

(A) ``brute_force_snr``  -- the matched filter of Eq. 1 in discrete form,
    z_i[k] = sum_j hbar_i[j] d[k - j], hbar_i = h_c + i h_s, d[k < 0] = 0.
(B) ``lloid_snr``        -- the LLOID approximation of (A), step by step in the
    paper's order (Section II.C):
      1. downsample the strain to each slice rate with the sinc-windowed-sinc
         kernel of Eq. 4 (c = f N_down);
      2. filter each slice with its SVD basis (Eq. 5), reading the segment
         picked by pre-synchronisation (Eq. 9);
      3. reconstruct each slice's SNR through sigma * v (Eq. 6);
      4. from the lowest rate up, upsample with the polyphase form of
         Eq. 7-8 (c = f N_up) and add the next rate's slices (Eq. 9 recursion).
(C) ``triggers``         -- per window and template, the max of |z| above the
    threshold, its time and phase, and the per-bank maximum (Section II.D.1).
(D) ``svd_bank``         -- per-slice SVD of the real/imaginary-stacked
    templates keeping 99.99 % of the slice energy (Eq. 3).
(F) ``coincident_events`` -- coincidence across detectors and clustering per
    bank (Sections II.D.3-4): per (bank, window, template) the loudest
    detector's trigger is the reference and every other detector's trigger
    within the coincidence window joins it; with two or more detectors it is
    an event of network SNR sqrt(sum rho^2); per (bank, window) only the
    event of highest network SNR is kept.
(H) ``Whitener``         -- PSD estimation and whitening of Section II.B.2:
    blocks of N input samples (an N - 2Z Hann-windowed segment between Z
    zeros) advancing by N/2 - Z, FFT, downsampling by keeping the bins below
    the output Nyquist, per-bin median of the last n_med instantaneous PSDs,
    running geometric mean, x e^gamma, whitening, inverse FFT at the output
    rate, Tukey window, overlap-add; output lags the input by N/2.
(G) ``background_counts`` -- the per-(bank, detector) background histogram
    of Section II.D.5: SNR and xi2 of the single-detector triggers (those not
    in their template's coincidence) binned on given edges, only while two
    or more detectors operate.
(E) ``autocorrelation`` and ``xi2`` -- the signal-consistency statistic of
    Eq. 10 (Section II.D.2) for each trigger:
      xi2 = sum_{t=-d}^{d} |z[k+t] - z[k] R(t)|^2 / sum_{t=-d}^{d} (2 - 2 |R(t)|^2),
    R the template's complex autocorrelation with R(0) = 1.

Readings of points the paper leaves open:
* discrete unit-variance form of Eq. 1 (no factor 2): E|z|^2 = 2 in white
  noise and an injection at amplitude A gives |z| = A;
* downsampling is zero-phase (centred) with unit DC gain, w = g / sum(g), and
  the decimated stream is scaled by sqrt(D) so it keeps unit variance; the
  slice matrix carries the other sqrt(D): A^s[row][m] = sqrt(D) h[J_s + D m];
* Eq. 5 is written in before-merger indexing:
  Y^s_l[q] = sum_m u^s_l[m] d_s[q - J_s / D_s - m];
* Eq. 8 is read as centred for every phase, Up[p] = sum_t z_phi[t]
  x[floor(p / F) + N_up - t] (the printed causal form differs by the N_up
  delay that pre-synchronisation absorbs); the upsampling kernel is not
  renormalised (g[c] = 1 makes it interpolating);
* the ladder is the bank's distinct slice rates plus f0;
* triggers: windows [max(0, wW - overlap), (w + 1) W), "exceeds" is strict,
  ties go to the earliest sample, the bank maximum to the lowest template;
* coincidence: one window (samples) for every detector pair, inclusive
  (|k_a - k_b| <= delta); the reference is the loudest detector (lowest index
  on ties); a coincidence needs two or more detectors; clustering keeps the
  highest network SNR per (bank, window), lowest template on ties; windows do
  not overlap, so triggers in different windows never coincide;
* background: a trigger is single unless it is a member of its template's
  coincidence (two or more detectors within the window of the loudest);
  bins are given as ascending float32 edges e_0 < ... < e_n, a value x goes to
  the number of edges e_1 .. e_{n-1} that are <= x (so the first and last bins
  take everything outside the edges); the comparisons are made in float32,
  as on the GPU;
* whitening: periodic Hann of length L = N - 2Z (hop L/2 windows sum to one);
  instantaneous PSD |X_k|^2 / sum w^2; the median of the last n_med (n_med
  odd; while fewer exist, of the largest odd number of the newest ones)
  divided by kappa_k = exp(E[log median of k unit exponentials] + gamma) is a
  geometric-mean estimate of the bin's exponential distribution (E[log] of it
  equals that of a single sample, log mean - gamma);
  running geometric mean log G <- log G + (log g - log G) / min(i, n_avg) over
  the i-th estimate (n_avg = 64: the paper does not give it); PSD = G e^gamma;
  Y_k = X_k / sqrt(PSD_k) sqrt(N_out / N) / N_out for k <= N_out / 2 (the
  Nyquist bin's real part), inverse real FFT of size N_out, Tukey window with
  cosine tapers of Z_out samples at each end; a block whose segment holds a
  non-finite sample adds nothing and does not update the PSD; output sample
  j corresponds to input sample j rate_in / rate_out - Z;
* Eq. 10: R(t) = sum_j hbar[j] conj(hbar[j - t]) / sum_j |hbar[j]|^2 (the
  complex template's autocorrelation, so that a noise-free signal gives
  z[k + t] = z[k] R(t) and white noise gives E xi2 = 1 under the E|z|^2 = 2
  normalisation the denominator 2 - 2|R|^2 implies); the sums run over the
  full autocorrelation length 2 d + 1 centred on the peak, and z before the
  start of the stream is 0.

Parity status: (A), Eq. 4, Eq. 7-8, the reconstruction, the trigger rules and
Eq. 10 are pinned by closed forms, special cases, invariants and brute force
in ``tests/test_oracle_pins.py``.  (B) as an approximation of (A) has no exact
pin in the paper: it is held to 1 % relative SNR at injections (parity
unpinned beyond that tolerance).
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import List, Sequence

import numpy as np

N_DOWN = 32      # half-length of the downsampling kernel at the target rate (Section II.C.2)
N_UP = 8         # half-length of the upsampling kernel (Section II.C.2)
SNR_THRESHOLD = 4.0   # trigger threshold on |z| (Section II.D.1)


# ----------------------------------------------------------------------------
# Eq. 4: sinc-windowed sinc kernel
# ----------------------------------------------------------------------------

def sinc_kernel(f: int, c: int) -> np.ndarray:
    """g[k], k = 0..2c: sinc of zero spacing f times a sinc window of half
    length c, with g[c] = 1 (Eq. 4)."""
    g = np.empty(2 * c + 1, dtype=np.float64)
    for k in range(2 * c + 1):
        if k == c:
            g[k] = 1.0
        else:
            a = math.pi * (k - c) / f
            b = math.pi * (k - c) / c
            g[k] = (math.sin(a) / a) * (math.sin(b) / b)
    return g


# ----------------------------------------------------------------------------
# A stream is an array plus the index of its first sample.
# ----------------------------------------------------------------------------

@dataclass
class Stream:
    """Samples x[..., i] of index start + i (the last axis is time)."""
    x: np.ndarray
    start: int

    @property
    def stop(self) -> int:
        return self.start + self.x.shape[-1]

    def window(self, lo: int, hi: int) -> np.ndarray:
        """Samples lo..hi-1, zero outside the stored range."""
        out = np.zeros(self.x.shape[:-1] + (hi - lo,), dtype=np.float64)
        a, b = max(lo, self.start), min(hi, self.stop)
        if b > a:
            out[..., a - lo:b - lo] = self.x[..., a - self.start:b - self.start]
        return out


# ----------------------------------------------------------------------------
# (A) brute force, Eq. 1
# ----------------------------------------------------------------------------

def brute_force_snr(d: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """z_row[k] = sum_{j=0}^{N-1} rows[row][j] d[k - j] for k in [0, len(d)),
    with d[k < 0] = 0.  ``rows`` is [2M, N] in before-merger order.  Returns the
    real rows [2M, len(d)]; z_i = out[2i] + 1j out[2i+1]."""
    d = np.asarray(d, dtype=np.float64)
    T = d.size
    out = np.empty((rows.shape[0], T))
    for r in range(rows.shape[0]):
        out[r] = np.convolve(d, rows[r])[:T]
    return out


def brute_force_snr_fft(d: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """Same as ``brute_force_snr`` through zero-padded FFTs (independent route)."""
    d = np.asarray(d, dtype=np.float64)
    T, N = d.size, rows.shape[1]
    n = 1 << int(math.ceil(math.log2(T + N)))
    D = np.fft.rfft(d, n)
    H = np.fft.rfft(rows, n, axis=1)
    return np.fft.irfft(H * D[None, :], n, axis=1)[:, :T]


# ----------------------------------------------------------------------------
# (D) SVD bank, Eq. 3
# ----------------------------------------------------------------------------

@dataclass
class OracleSlice:
    rate: int
    j_start: int
    bases: np.ndarray     # [L, N] orthonormal u_l
    coeffs: np.ndarray    # [2M, L] = v_il sigma_l


def slice_matrix(bank, rate: int, j_start: int, n_taps: int) -> np.ndarray:
    """A^s[row][m] = sqrt(D) h_row[J_s + D m], m < N_s (the slice, decimated)."""
    D = bank.f0 // rate
    j = j_start + D * np.arange(n_taps)
    return math.sqrt(D) * bank.rows(j)


def svd_bank(bank, plan, energy: float = 0.9999, full_rank: bool = False) -> List[OracleSlice]:
    """Per slice: A = U S V^T, keep the leading L bases holding ``energy`` of
    sum S^2 (all of them with ``full_rank``); bases u_l = V^T[l], coefficients
    v_il sigma_l = U[i, l] S[l] (Eq. 3)."""
    out = []
    for r, J, N in zip(plan.rate, plan.j_start, plan.n_taps):
        A = slice_matrix(bank, r, J, N)
        U, S, Vt = np.linalg.svd(A, full_matrices=False)
        if full_rank:
            L = S.size
        else:
            cum = np.cumsum(S ** 2)
            L = int(np.searchsorted(cum, energy * cum[-1]) + 1)
            L = min(L, S.size)
        out.append(OracleSlice(r, J, Vt[:L].copy(), U[:, :L] * S[None, :L]))
    return out


def identity_bank(bank, plan) -> List[OracleSlice]:
    """No compression: the bases are the slice rows themselves and the
    coefficients the identity (the multirate path without SVD)."""
    out = []
    for r, J, N in zip(plan.rate, plan.j_start, plan.n_taps):
        A = slice_matrix(bank, r, J, N)
        out.append(OracleSlice(r, J, A.copy(), np.eye(A.shape[0])))
    return out


# ----------------------------------------------------------------------------
# (B) LLOID, Eq. 4-9
# ----------------------------------------------------------------------------

def downsample(d: Stream, D: int, q_lo: int, q_hi: int, n_down: int = N_DOWN) -> Stream:
    """d_s[q] = sqrt(D) sum_{k=0}^{2c} w[k] d[D q + c - k], w = g / sum(g),
    g from Eq. 4 with f = D and c = D N_down, for q in [q_lo, q_hi)."""
    if D == 1:
        return Stream(d.window(q_lo, q_hi), q_lo)
    c = D * n_down
    g = sinc_kernel(D, c)
    w = g / g.sum()
    lo = D * q_lo + c - 2 * c
    hi = D * (q_hi - 1) + c + 1
    seg = d.window(lo, hi)                  # seg[i] = d[lo + i]
    conv = np.convolve(seg, w)              # conv[i] = sum_k w[k] seg[i - k]
    q = np.arange(q_lo, q_hi)
    return Stream(math.sqrt(D) * conv[D * q + c - lo], q_lo)


def polyphase_upsample(x: Stream, F: int, n_up: int = N_UP) -> Stream:
    """Eq. 7-8 (centred reading): the kernel g (Eq. 4, f = F, c = F N_up) is
    split into F sub-kernels z_j[k] = g[k F + j], k = 0..2c/F, and output p
    takes Up[p] = sum_k z_{p mod F}[k] x[floor(p / F) + N_up - k]."""
    if F == 1:
        return Stream(x.x.copy(), x.start)
    c = F * n_up
    g = sinc_kernel(F, c)
    K = 2 * c // F
    sub = np.zeros((F, K + 1))
    for j in range(F):
        for k in range(K + 1):
            if k * F + j <= 2 * c:
                sub[j, k] = g[k * F + j]
    p = np.arange(F * x.start, F * x.stop)
    out = np.zeros(x.x.shape[:-1] + (p.size,))
    base = p // F + n_up
    phase = p % F
    b0 = int(base.min())
    for k in range(K + 1):
        xs = x.window(b0 - k, int(base.max()) - k + 1)     # xs[..., i] = x[b0 - k + i]
        out += sub[phase, k] * xs[..., base - b0]
    return Stream(out, F * x.start)


def zero_stuff_upsample(x: Stream, F: int, n_up: int = N_UP) -> Stream:
    """Textbook interpolation: insert F-1 zeros between samples and convolve
    with g centred on c, Up[p] = sum_k x[k] g[p - F k + c] (used as a pin)."""
    if F == 1:
        return Stream(x.x.copy(), x.start)
    c = F * n_up
    g = sinc_kernel(F, c)
    n = F * x.x.size
    stuffed = np.zeros(n)
    stuffed[::F] = x.x
    full = np.convolve(stuffed, g)           # full[i] = sum_m stuffed[m] g[i - m]
    return Stream(full[c:c + n], F * x.start)   # 1-D input only


def ladder_rates(slices: Sequence[OracleSlice], f0: int) -> List[int]:
    """Distinct slice rates plus f0, ascending."""
    return sorted(set(s.rate for s in slices) | {f0})


def presync_ok(slices: Sequence[OracleSlice], f0: int, n_down: int = N_DOWN, n_up: int = N_UP) -> bool:
    """Pre-synchronisation without added latency (Section II.C.3, Eq. 9):
    J_s / f0 >= N_down / f_s + sum over ladder rates f_s <= f < f0 of N_up / f."""
    lad = ladder_rates(slices, f0)
    for s in slices:
        if s.rate == f0:
            if s.j_start < 0:
                return False
            continue
        need = n_down * (f0 // s.rate) + sum(n_up * (f0 // f) for f in lad if s.rate <= f < f0)
        if s.j_start < need:
            return False
    return True


def lloid_snr(d: np.ndarray, slices: Sequence[OracleSlice], f0: int, n_down: int = N_DOWN,
              n_up: int = N_UP, pad: int = 8192) -> np.ndarray:
    """LLOID SNR rows [2M, len(d)] for strain d starting at sample 0 with zero
    history (d[k < 0] = 0).  Every stream is evaluated on a range padded by
    ``pad`` full-rate samples on both sides so that truncation never reaches
    the returned samples."""
    d = np.asarray(d, dtype=np.float64)
    T = d.size
    lad = ladder_rates(slices, f0)
    grid = f0 // lad[0]
    Tg = -(-T // grid) * grid           # whole samples at every rate; the zeros
    full = Stream(np.concatenate([d, np.zeros(Tg - T)]), 0)   # appended lie in the future
    pad = -(-pad // grid) * grid
    n_rows = slices[0].coeffs.shape[0]
    # Per-rate sums S_r of the reconstructed slices (Eq. 5-6), on [lo_r, hi_r).
    S = {}
    for r in lad:
        D = f0 // r
        S[r] = Stream(np.zeros((n_rows, (Tg + 2 * pad) // D)), -pad // D)
    for s in slices:
        D = f0 // s.rate
        off = s.j_start // D                      # pre-synchronisation offset (Eq. 9)
        L, N = s.bases.shape
        qa, qb = S[s.rate].start, S[s.rate].start + S[s.rate].x.shape[1]
        ds = downsample(full, D, qa - off - N + 1, qb - off, n_down)
        # Eq. 5: Y_l[q] = sum_m u_l[m] d_s[q - off - m]
        Y = np.empty((L, qb - qa))
        for l in range(L):
            conv = np.convolve(ds.x, s.bases[l])   # conv[i] = sum_m u[m] ds.x[i - m]
            # ds.x[i] is d_s[ds.start + i]; want index q - off  ->  i = q - off - ds.start
            i = np.arange(qa, qb) - off - ds.start
            Y[l] = conv[i]
        # Eq. 6: reconstruction through sigma * v
        S[s.rate].x += s.coeffs @ Y
    # Eq. 9 recursion, lowest rate upward, with Eq. 7-8 upsampling.
    acc = None
    for r_lo, r_hi in zip([None] + lad[:-1], lad):
        if acc is None:
            acc = Stream(S[r_hi].x.copy(), S[r_hi].start)
            continue
        F = r_hi // r_lo
        up = polyphase_upsample(acc, F, n_up)
        tgt = S[r_hi]
        acc = Stream(tgt.x + up.window(tgt.start, tgt.stop), tgt.start)
    return acc.x[:, -acc.start:-acc.start + T]


# ----------------------------------------------------------------------------
# (C) triggers, Section II.D.1
# ----------------------------------------------------------------------------

@dataclass
class Trigger:
    detector: int
    bank: int
    tmpl: int
    window: int
    sample: int
    snr: float
    phase: float
    re: float
    im: float
    is_bank_max: bool


def triggers(z_rows: np.ndarray, window: int, overlap: int = 0, threshold: float = SNR_THRESHOLD,
             detector: int = 0, bank: int = 0, n_windows=None, t_offset: int = 0) -> List[Trigger]:
    """For every complete window w, [max(0, wW - overlap), (w + 1) W), and
    template i: k* = the first argmax of |z_i|^2; a trigger if |z_i[k*]| >
    threshold.  The trigger of the template with the largest |z|^2 in the
    bank (lowest template index on ties) is flagged ``is_bank_max``."""
    re, im = z_rows[0::2], z_rows[1::2]
    p = re * re + im * im
    T = z_rows.shape[1]
    nw = T // window if n_windows is None else n_windows
    out = []
    for w in range(nw):
        a = max(0, w * window - overlap) - t_offset
        b = (w + 1) * window - t_offset
        if a < 0 or b > T:
            continue
        seg = p[:, a:b]
        k = np.argmax(seg, axis=1)
        best = seg[np.arange(seg.shape[0]), k]
        top = int(np.argmax(best))
        for i in range(seg.shape[0]):
            if math.sqrt(best[i]) > threshold:
                kk = a + int(k[i])
                out.append(Trigger(detector, bank, i, w, kk + t_offset, math.sqrt(best[i]),
                                   math.atan2(im[i, kk], re[i, kk]), re[i, kk], im[i, kk], i == top))
    return out


# ----------------------------------------------------------------------------
# (E) signal-based consistency, Eq. 10 (Section II.D.2)
# ----------------------------------------------------------------------------

def autocorrelation(h_c: np.ndarray, h_s: np.ndarray, half: int) -> np.ndarray:
    """R(t) for t = -half .. half (index t + half): the complex template
    hbar = h_c + i h_s correlated with itself,
    R(t) = sum_j hbar[j] conj(hbar[j - t]) / sum_j |hbar[j]|^2, hbar = 0
    outside its samples; R(0) = 1."""
    h = np.asarray(h_c, dtype=np.float64) + 1j * np.asarray(h_s, dtype=np.float64)
    n = h.size
    norm = float(np.sum(np.abs(h) ** 2))
    out = np.empty(2 * half + 1, dtype=np.complex128)
    for t in range(-half, half + 1):
        # pairs (j, j - t) with both inside [0, n)
        lo, hi = max(0, t), min(n, n + t)
        out[t + half] = np.sum(h[lo:hi] * np.conj(h[lo - t:hi - t])) / norm if hi > lo else 0.0
    return out


def xi2(z: np.ndarray, k: int, R: np.ndarray) -> float:
    """Eq. 10 at a peak: z is one template's complex SNR series (index =
    sample), k the peak sample, R its autocorrelation for t = -d .. d.  Samples
    before the start of the series are 0; the series must reach k + d."""
    half = (R.size - 1) // 2
    if k + half >= z.size:
        raise ValueError("the series does not reach k + d")
    num = 0.0
    for t in range(-half, half + 1):
        zt = z[k + t] if k + t >= 0 else 0.0
        num += abs(zt - z[k] * R[t + half]) ** 2
    den = float(np.sum(2.0 - 2.0 * np.abs(R) ** 2))
    return num / den


# ----------------------------------------------------------------------------
# (F) coincidence and clustering, Sections II.D.3-4
# ----------------------------------------------------------------------------

@dataclass
class Event:
    window: int
    bank: int
    tmpl: int
    n_ifo: int
    ifo_mask: int
    net_snr: float
    ref_detector: int
    ref_sample: int


def coincident_events(trigs: Sequence[Trigger], delta: int) -> List[Event]:
    """Events of a trigger list (any detectors, banks, windows)."""
    by_key = {}
    for t in trigs:
        by_key.setdefault((t.bank, t.window, t.tmpl), {})[t.detector] = t
    best = {}
    for (bank, w, i), per_det in by_key.items():
        dets = sorted(per_det)
        ref = dets[0]
        for d in dets[1:]:
            if per_det[d].snr > per_det[ref].snr:
                ref = d
        k0 = per_det[ref].sample
        members = [d for d in dets if abs(per_det[d].sample - k0) <= delta]
        if len(members) < 2:
            continue
        net = math.sqrt(sum(per_det[d].snr ** 2 for d in members))
        ev = Event(w, bank, i, len(members), sum(1 << d for d in members), net, ref, k0)
        cur = best.get((bank, w))
        if cur is None or net > cur.net_snr or (net == cur.net_snr and i < cur.tmpl):
            best[(bank, w)] = ev
    return [best[k] for k in sorted(best)]


# ----------------------------------------------------------------------------
# (G) background collection, Section II.D.5
# ----------------------------------------------------------------------------

def _bin(x: float, edges: np.ndarray) -> int:
    x32 = np.float32(x)
    b = 0
    for e in edges[1:-1]:
        if np.float32(e) <= x32:
            b += 1
    return b


def background_counts(trigs: Sequence[Trigger], xi2_of, n_det: int, delta: int, snr_edges: np.ndarray,
                      xi2_edges: np.ndarray) -> dict:
    """{(bank, detector): counts [n_snr, n_xi2]} over the single-detector
    triggers; xi2_of(trigger) gives its xi2."""
    out = {}
    if n_det < 2:
        return out
    by_key = {}
    for t in trigs:
        by_key.setdefault((t.bank, t.window, t.tmpl), {})[t.detector] = t
    for (bank, w, i), per_det in by_key.items():
        dets = sorted(per_det)
        ref = dets[0]
        for d in dets[1:]:
            if per_det[d].snr > per_det[ref].snr:
                ref = d
        k0 = per_det[ref].sample
        members = [d for d in dets if abs(per_det[d].sample - k0) <= delta]
        coincident = set(members) if len(members) >= 2 else set()
        for d in dets:
            if d in coincident:
                continue
            h = out.setdefault((bank, d), np.zeros((len(snr_edges) - 1, len(xi2_edges) - 1), dtype=np.int64))
            h[_bin(per_det[d].snr, snr_edges), _bin(xi2_of(per_det[d]), xi2_edges)] += 1
    return out


# ----------------------------------------------------------------------------
# (H) PSD estimation and whitening, Section II.B.2
# ----------------------------------------------------------------------------

def median_log_factor(k: int) -> float:
    """kappa_k = exp(E[log M] + gamma) for M the median of k (odd) independent
    unit exponentials.  M has density c (1 - e^-x)^m e^-(m+1)x, m = (k-1)/2,
    c = k!/(m!)^2; expanding (1 - e^-x)^m and using
    int_0^inf log(x) e^-ax dx = -(gamma + log a)/a:
    E[log M] = -c sum_j C(m, j) (-1)^j (gamma + log(m+1+j)) / (m+1+j)."""
    m = (k - 1) // 2
    c = math.factorial(k) / math.factorial(m) ** 2
    e = 0.0
    for j in range(m + 1):
        a = m + 1 + j
        e -= c * math.comb(m, j) * (-1) ** j * (np.euler_gamma + math.log(a)) / a
    return math.exp(e + np.euler_gamma)


def hann_periodic(L: int) -> np.ndarray:
    n = np.arange(L)
    return np.sin(np.pi * n / L) ** 2


def tukey(n: int, taper: int) -> np.ndarray:
    """Flat 1 with cosine tapers of `taper` samples at each end."""
    w = np.ones(n)
    if taper > 0:
        t = np.arange(taper)
        ramp = 0.5 * (1.0 - np.cos(np.pi * (t + 0.5) / taper))
        w[:taper] = ramp
        w[n - taper:] = ramp[::-1]
    return w


class Whitener:
    """One detector's whitening stream (FP64)."""

    def __init__(self, rate_in: int, rate_out: int, n_fft: int, z_pad: int, n_med: int = 7, n_avg: int = 64):
        self.r_in, self.r_out, self.N, self.Z = rate_in, rate_out, n_fft, z_pad
        self.n_med, self.n_avg = n_med, n_avg
        self.L = n_fft - 2 * z_pad
        self.hop = n_fft // 2 - z_pad
        self.N_out = n_fft * rate_out // rate_in
        self.Z_out = z_pad * rate_out // rate_in
        self.hop_out = self.hop * rate_out // rate_in
        self.w = hann_periodic(self.L)
        self.W2 = float(np.sum(self.w ** 2))
        self.T = tukey(self.N_out, self.Z_out)
        self.buf = np.zeros(0)
        self.hist = []               # recent instantaneous PSDs (n_med)
        self.logG = None
        self.n_est = 0
        self.acc = np.zeros(self.N_out)

    def psd(self) -> np.ndarray:
        return np.exp(self.logG) * math.exp(np.euler_gamma)

    def _update_psd(self, p_inst: np.ndarray) -> None:
        self.hist = (self.hist + [p_inst])[-self.n_med:]
        k = len(self.hist) if len(self.hist) % 2 else len(self.hist) - 1
        med = np.median(np.stack(self.hist[-k:]), axis=0)
        g = med / median_log_factor(k)
        self.n_est += 1
        if self.logG is None:
            self.logG = np.log(g)
        else:
            self.logG = self.logG + (np.log(g) - self.logG) / min(self.n_est, self.n_avg)

    def push(self, x: np.ndarray) -> np.ndarray:
        """Append input samples (a multiple of the hop); return the output
        samples that became final."""
        self.buf = np.concatenate([self.buf, np.asarray(x, dtype=np.float64)])
        out = []
        while self.buf.size >= self.L:
            seg = self.buf[:self.L]
            self.buf = self.buf[self.hop:]
            b = np.zeros(self.N)
            b[self.Z:self.Z + self.L] = self.w * seg
            k_out = self.N_out // 2
            y = np.zeros(self.N_out)
            if np.all(np.isfinite(seg)):
                X = np.fft.rfft(b)[:k_out + 1]
                self._update_psd(np.abs(X) ** 2 / self.W2)
                Y = X / np.sqrt(self.psd()) * math.sqrt(self.N_out / self.N) / self.N_out
                y = np.fft.irfft(Y * self.N_out, n=self.N_out)   # numpy's irfft divides by N_out
            self.acc += self.T * y
            out.append(self.acc[:self.hop_out].copy())
            self.acc = np.concatenate([self.acc[self.hop_out:], np.zeros(self.hop_out)])
        return np.concatenate(out) if out else np.zeros(0)
