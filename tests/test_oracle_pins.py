"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed
forms of Eq. 4, the textbook definition behind Eq. 7-8, a brute-force loop
that is the definition of Eq. 1, two independent routes (direct sum and FFT),
special cases where LLOID must reduce to the matched filter exactly, and
invariants (linearity, shift equivariance on the multirate grid, causality
under pre-synchronisation).  They are chosen so that a dropped term, a wrong
sign or offset, a transposed operand or a missing sqrt(D) fails one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import lloid_oracle as O

F0 = 2048


# --------------------------------------------------------------------------
# constants the paper prints
# --------------------------------------------------------------------------

def test_paper_constants(golden_dir):
    g = json.load(open(os.path.join(golden_dir, "paper_constants.json")))
    assert O.N_DOWN == g["n_down"]["value"]
    assert O.N_UP == g["n_up"]["value"]
    assert O.SNR_THRESHOLD == g["snr_threshold"]["value"]
    # Eq. 7: each polyphase sub-kernel has 2c/f + 1 = 2 N_up + 1 taps
    assert 2 * O.N_UP + 1 == g["upsample_subkernel_len"]["value"]


# --------------------------------------------------------------------------
# Eq. 4 closed form
# --------------------------------------------------------------------------

@pytest.mark.parametrize("f,n_half", [(2, 32), (4, 32), (8, 32), (16, 32), (2, 8), (8, 8), (64, 8)])
def test_sinc_kernel_closed_form(f, n_half):
    c = f * n_half
    g = O.sinc_kernel(f, c)
    assert g.size == 2 * c + 1
    assert g[c] == 1.0
    # zeros of the sinc at every multiple of f away from the centre
    for n in range(1, c // f + 1):
        assert abs(g[c + n * f]) < 1e-15 and abs(g[c - n * f]) < 1e-15
    # zero-phase (symmetric) and the sinc window vanishes at both ends
    assert np.allclose(g, g[::-1], atol=0, rtol=0)
    assert abs(g[0]) < 1e-15 and abs(g[-1]) < 1e-15
    # one sample off a zero the kernel is the product of two sincs
    k = c + 1
    a, b = math.pi / f, math.pi / c
    assert g[k] == pytest.approx(math.sin(a) / a * math.sin(b) / b, rel=1e-14)
    # DC gain of a sinc with zero spacing f is f
    assert g.sum() == pytest.approx(f, rel=2e-2)


# --------------------------------------------------------------------------
# Eq. 7-8 against zero-stuffing + convolution (textbook interpolation)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("F", [2, 4, 8, 16])
def test_polyphase_equals_zero_stuff(F):
    rng = np.random.default_rng(F)
    x = O.Stream(rng.standard_normal(300), 0)
    a = O.polyphase_upsample(x, F)
    b = O.zero_stuff_upsample(x, F)
    assert a.start == b.start == 0
    assert np.max(np.abs(a.x - b.x)) < 1e-13
    # interpolating: every F-th output is the input sample itself
    assert np.max(np.abs(a.x[::F] - x.x)) < 1e-14


def test_polyphase_2d_rows_match_1d():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((3, 50))
    a = O.polyphase_upsample(O.Stream(X, -5), 4)
    for r in range(3):
        b = O.polyphase_upsample(O.Stream(X[r], -5), 4)
        assert a.start == b.start == -20
        assert np.max(np.abs(a.x[r] - b.x)) == 0.0


# --------------------------------------------------------------------------
# (A) brute force: the definition written as loops, and the FFT route
# --------------------------------------------------------------------------

def test_brute_force_is_the_definition():
    rng = np.random.default_rng(11)
    T, N = 40, 7
    d = rng.standard_normal(T)
    rows = rng.standard_normal((4, N))
    z = O.brute_force_snr(d, rows)
    for r in range(4):
        for k in range(T):
            s = 0.0
            for j in range(N):
                if k - j >= 0:
                    s += rows[r, j] * d[k - j]
            assert abs(z[r, k] - s) < 1e-12


def test_brute_force_direct_equals_fft():
    w = W.make_workload("tiny", n_seconds=6)
    rows = w.banks[0].full()
    d = w.strain(0).astype(np.float64)
    a = O.brute_force_snr(d, rows)
    b = O.brute_force_snr_fft(d, rows)
    assert np.max(np.abs(a - b)) < 1e-12


# --------------------------------------------------------------------------
# Injections and noise statistics (Eq. 1 normalisation)
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def bank64():
    w = W.make_workload("bank64", n_seconds=16)
    return w.banks[0], w.plans[0]


@pytest.mark.parametrize("phase", [0.0, 1.1])
def test_injection_recovers_amplitude(bank64, phase):
    bank, plan = bank64
    T = 16 * F0
    A, i, k0 = 12.0, 5, 12 * F0 + 3
    d = np.zeros(T)
    rows = bank.full()
    for j in range(rows.shape[1]):
        d[k0 - j] += A * (math.cos(phase) * rows[2 * i, j] + math.sin(phase) * rows[2 * i + 1, j])
    za = O.brute_force_snr_fft(d, rows)
    cs = float(rows[2 * i] @ rows[2 * i + 1])          # <h_c, h_s>
    assert za[2 * i, k0] == pytest.approx(A * (math.cos(phase) + math.sin(phase) * cs), abs=1e-10)
    assert za[2 * i + 1, k0] == pytest.approx(A * (math.cos(phase) * cs + math.sin(phase)), abs=1e-10)
    # LLOID recovers the same SNR to 1 % (the paper's <1 % agreement level)
    zb = O.lloid_snr(d, O.svd_bank(bank, plan), F0)
    snr_b = abs(zb[2 * i, k0] + 1j * zb[2 * i + 1, k0])
    assert abs(snr_b - A) < 0.01 * A
    assert abs(math.atan2(zb[2 * i + 1, k0], zb[2 * i, k0]) - phase) < 0.01


def test_noise_expectation_two():
    """E|z|^2 = ||h_c||^2 + ||h_s||^2 = 2 for unit white noise (Eq. 1)."""
    w = W.make_workload("tiny", n_seconds=40)
    rows = w.banks[0].full()
    d = W.white_noise(40 * F0, 12345).astype(np.float64)
    za = O.brute_force_snr_fft(d, rows)[:, 4 * F0:]
    p = za[0::2] ** 2 + za[1::2] ** 2
    # batch means over 2 s batches (longer than any template) for the error bar
    nb = p.shape[1] // (2 * F0)
    means = p[:, :nb * 2 * F0].reshape(p.shape[0], nb, 2 * F0).mean(axis=(0, 2))
    m, se = means.mean(), means.std(ddof=1) / math.sqrt(nb)
    assert abs(m - 2.0) < 5 * se
    zb = O.lloid_snr(d, O.svd_bank(w.banks[0], w.plans[0]), F0)[:, 4 * F0:]
    pb = zb[0::2] ** 2 + zb[1::2] ** 2
    assert abs(pb.mean() / p.mean() - 1.0) < 0.02


def test_downsampled_noise_has_unit_variance():
    d = O.Stream(W.white_noise(64 * F0, 4).astype(np.float64), 0)
    for D in (2, 8, 16):
        ds = O.downsample(d, D, 64, 64 * F0 // D - 64)
        assert abs(ds.x.var() - 1.0) < 0.03


def test_sinusoid_down_then_up():
    """An in-band sinusoid survives downsampling + upsampling with no delay."""
    f0 = F0
    t = np.arange(16 * f0)
    for D in (2, 8, 16):
        r = f0 // D
        x = np.cos(2 * math.pi * 0.3 * r * t / f0 + 0.4)
        ds = O.downsample(O.Stream(x, 0), D, 0, x.size // D)
        up = O.polyphase_upsample(O.Stream(ds.x / math.sqrt(D), 0), D)
        mid = slice(4 * f0, 12 * f0)
        err = np.max(np.abs(up.x[mid] - x[mid]))
        assert err < 2e-3, (D, err)


# --------------------------------------------------------------------------
# Special cases where LLOID must equal the matched filter
# --------------------------------------------------------------------------

def test_full_rank_single_rate_equals_brute_force():
    """One slice at f0, D = 1, full-rank SVD: (B) == (A)."""
    w = W.make_workload("tiny", n_seconds=8)
    bank = w.banks[0]
    plan = W.SlicePlan((F0,), (0,), (bank.n_samples,))
    sl = O.svd_bank(bank, plan, full_rank=True)
    d = w.strain(0).astype(np.float64)
    zb = O.lloid_snr(d, sl, F0)
    za = O.brute_force_snr_fft(d, bank.full())
    assert np.max(np.abs(za - zb)) < 1e-10


def test_full_rank_multirate_equals_no_svd(bank64):
    """Full-rank SVD reproduces the per-template multirate path (no SVD)."""
    bank, plan = bank64
    d = W.white_noise(8 * F0, 77).astype(np.float64)
    zs = O.lloid_snr(d, O.svd_bank(bank, plan, full_rank=True), F0)
    zi = O.lloid_snr(d, O.identity_bank(bank, plan), F0)
    assert np.max(np.abs(zs - zi)) < 1e-10


def test_svd_bank_energy_and_orthonormality(bank64):
    bank, plan = bank64
    for s, (r, J, N) in zip(O.svd_bank(bank, plan), zip(plan.rate, plan.j_start, plan.n_taps)):
        A = O.slice_matrix(bank, r, J, N)
        L = s.bases.shape[0]
        assert np.max(np.abs(s.bases @ s.bases.T - np.eye(L))) < 1e-12
        Sv = np.linalg.svd(A, compute_uv=False)
        tot = np.sum(Sv ** 2)
        assert np.sum(Sv[:L] ** 2) >= 0.9999 * tot
        assert np.sum(Sv[:L - 1] ** 2) < 0.9999 * tot
        resid = A - s.coeffs @ s.bases
        assert np.sum(resid ** 2) == pytest.approx(np.sum(Sv[L:] ** 2), rel=1e-6, abs=1e-20)


# --------------------------------------------------------------------------
# Invariants of (B)
# --------------------------------------------------------------------------

def test_linearity(bank64):
    bank, plan = bank64
    sl = O.svd_bank(bank, plan)
    d1 = W.white_noise(6 * F0, 1).astype(np.float64)
    d2 = W.white_noise(6 * F0, 2).astype(np.float64)
    z = O.lloid_snr(2.5 * d1 - 0.75 * d2, sl, F0)
    z12 = 2.5 * O.lloid_snr(d1, sl, F0) - 0.75 * O.lloid_snr(d2, sl, F0)
    assert np.max(np.abs(z - z12)) < 1e-11


def test_shift_equivariance_on_grid(bank64):
    bank, plan = bank64
    sl = O.svd_bank(bank, plan)
    d = W.white_noise(6 * F0, 9).astype(np.float64)
    Dmax = F0 // min(plan.rate)
    for delta in (Dmax, 5 * Dmax):
        z = O.lloid_snr(d, sl, F0)
        zs = O.lloid_snr(np.concatenate([np.zeros(delta), d]), sl, F0)
        assert np.max(np.abs(zs[:, delta:] - z)) < 1e-11
    # off the multirate grid the output is only approximately shifted
    zs = O.lloid_snr(np.concatenate([np.zeros(3), d]), sl, F0)
    assert np.max(np.abs(zs[:, 3:] - z)) > 1e-6


def test_presync_makes_output_causal(bank64):
    """With pre-synchronisation (Eq. 9) z[k] depends on d[<= k] only."""
    bank, plan = bank64
    sl = O.svd_bank(bank, plan)
    assert O.presync_ok(sl, F0)
    d = W.white_noise(6 * F0, 21).astype(np.float64)
    cut = 4 * F0 + 37
    d2 = d.copy()
    d2[cut:] = W.white_noise(d.size - cut, 22)
    z1 = O.lloid_snr(d, sl, F0)
    z2 = O.lloid_snr(d2, sl, F0)
    assert np.max(np.abs(z1[:, :cut] - z2[:, :cut])) < 1e-12
    assert np.max(np.abs(z1[:, cut:] - z2[:, cut:])) > 1e-3


def test_presync_condition_values(bank64):
    bank, plan = bank64
    sl = O.svd_bank(bank, plan)
    # 256 Hz slice: N_down / 256 + N_up / 256 seconds = 320 samples <= J = 2048
    moved = [sl[0], O.OracleSlice(256, 320, sl[1].bases, sl[1].coeffs)]
    assert O.presync_ok(moved, F0)
    moved = [sl[0], O.OracleSlice(256, 312, sl[1].bases, sl[1].coeffs)]
    assert not O.presync_ok(moved, F0)


# --------------------------------------------------------------------------
# (C) trigger rules on hand-built SNR series
# --------------------------------------------------------------------------

def test_triggers_hand_built():
    W_ = 8
    T = 3 * W_
    z = np.zeros((6, T))                       # 3 templates
    # template 0: |z| = 5 at k=2 and a tie at k=6 -> earliest (k=2); window 0
    z[0, 2] = 5.0
    z[1, 6] = 5.0
    # template 1: |z| = 4 exactly at k=3 (not > 4), 4.5 in window 1 at k=12
    z[2, 3] = 4.0
    z[3, 12] = 4.5
    # template 2: |z| = 6 in window 0 at k=7 (phase 90 deg), 4.5 in window 1 at k=9
    z[5, 7] = 6.0
    z[4, 9] = -4.5
    tr = O.triggers(z, W_, threshold=4.0)
    got = [(t.window, t.tmpl, t.sample, round(t.snr, 12), round(t.phase, 12), t.is_bank_max) for t in tr]
    want = [
        (0, 0, 2, 5.0, 0.0, False),
        (0, 2, 7, 6.0, round(math.pi / 2, 12), True),
        (1, 1, 12, 4.5, round(math.pi / 2, 12), True),     # ties with template 2: lowest index
        (1, 2, 9, 4.5, round(math.pi, 12), False),
    ]
    assert got == want
    # overlap: window 1 = [W - 2, 2W) also sees k = 6, 7
    tr = O.triggers(z, W_, overlap=2, threshold=4.0)
    w1 = [(t.tmpl, t.sample) for t in tr if t.window == 1]
    assert w1 == [(0, 6), (1, 12), (2, 7)]


# --------------------------------------------------------------------------
# Eq. 10: autocorrelation and the signal-consistency statistic
# --------------------------------------------------------------------------

def test_autocorrelation_against_library_correlate(bank64):
    """R(0) = 1, R(-t) = conj R(t), and R equals numpy's full correlation of
    the complex template normalised at lag 0 (an independent route)."""
    rows = bank64[0].full()
    for i in (0, 33, 63):
        h = rows[2 * i] + 1j * rows[2 * i + 1]
        R = O.autocorrelation(rows[2 * i], rows[2 * i + 1], 175)
        assert abs(R[175] - 1.0) < 1e-14
        assert np.max(np.abs(R[::-1] - np.conj(R))) < 1e-14
        c = np.correlate(h, h, mode="full")          # c[n - 1 + t] = sum_j h[j + t] conj(h[j])
        n = h.size
        ref = c[n - 1 - 175:n + 175] / c[n - 1]
        assert np.max(np.abs(R - ref)) < 1e-12


@pytest.mark.parametrize("i,amp,phase", [(0, 12.0, 0.3), (40, 20.0, 2.0)])
def test_xi2_noise_free_signal_is_consistent(bank64, i, amp, phase):
    """A noise-free injection of the template itself gives z[k + t] = z[k] R(t)
    up to the template's tiny non-analytic part: xi2 ~ 0; the same data seen
    through another template gives a large xi2."""
    b = bank64[0]
    rows = b.full()
    T = 32 * F0
    d = np.zeros(T)
    W.add_injection(d, b, W.Injection(i, 20 * F0, amp, phase))
    z = O.brute_force_snr(d, rows[2 * i:2 * i + 2])
    zc = z[0] + 1j * z[1]
    k = int(np.argmax(np.abs(zc)))
    assert k == 20 * F0
    assert O.xi2(zc, k, O.autocorrelation(rows[2 * i], rows[2 * i + 1], 350)) < 1e-6
    j = (i + 7) % 64
    zj = O.brute_force_snr(d, rows[2 * j:2 * j + 2])
    zj = zj[0] + 1j * zj[1]
    kj = int(np.argmax(np.abs(zj)))
    assert O.xi2(zj, kj, O.autocorrelation(rows[2 * j], rows[2 * j + 1], 350)) > 0.5


def test_xi2_white_noise_mean_is_one(bank64):
    """In white noise E|z(t) - z(0) R(t)|^2 = 2 - 2|R(t)|^2 at any sample, so
    the mean of xi2 over many positions is 1 (within 4 standard errors)."""
    b = bank64[0]
    rows = b.full()
    rng = np.random.default_rng(5)
    T = 32 * F0
    d = rng.standard_normal(T)
    i = 10
    z = O.brute_force_snr(d, rows[2 * i:2 * i + 2])
    zc = z[0] + 1j * z[1]
    R = O.autocorrelation(rows[2 * i], rows[2 * i + 1], 350)
    v = np.array([O.xi2(zc, int(k), R) for k in rng.integers(9000, T - 400, 400)])
    assert abs(v.mean() - 1.0) < 4 * v.std() / np.sqrt(v.size)
    # doubling the data quadruples xi2 (numerator quadratic in z, denominator fixed)
    k = 12345
    assert abs(O.xi2(2 * zc, k, R) - 4 * O.xi2(zc, k, R)) < 1e-12 * O.xi2(zc, k, R) + 1e-15


# --------------------------------------------------------------------------
# Coincidence and clustering (Sections II.D.3-4) on hand-built trigger lists
# --------------------------------------------------------------------------

def _t(det, tmpl, w, k, snr, bank=0):
    return O.Trigger(det, bank, tmpl, w, k, snr, 0.0, snr, 0.0, False)


def test_coincidence_hand_built():
    D = 66
    trigs = [
        # window 0, template 3: H (det 0) and L (det 1) exactly D apart -> coincident
        _t(0, 3, 0, 1000, 6.0), _t(1, 3, 0, 1000 + D, 8.0),
        # template 4: D + 1 apart -> not coincident, no event
        _t(0, 4, 0, 500, 9.0), _t(1, 4, 0, 500 + D + 1, 9.5),
        # template 5: three detectors, V (det 2) too far from the loudest (det 2 is the loudest!)
        _t(0, 5, 0, 300, 5.0), _t(1, 5, 0, 310, 5.5), _t(2, 5, 0, 300 + 200, 7.0),
        # window 1: only single-detector triggers -> no event
        _t(0, 3, 1, 2100, 12.0),
        # bank 1, window 0: two events, equal network SNR -> lowest template wins
        _t(0, 7, 0, 100, 3.0, bank=1), _t(1, 7, 0, 101, 4.0, bank=1),
        _t(0, 2, 0, 900, 4.0, bank=1), _t(1, 2, 0, 899, 3.0, bank=1),
    ]
    ev = O.coincident_events(trigs, D)
    assert [(e.bank, e.window) for e in ev] == [(0, 0), (1, 0)]
    e0, e1 = ev
    # bank 0: template 3 (sqrt(36 + 64) = 10) beats template 5, whose loudest detector (V) has
    # no partner within D (H and L are 200 / 190 samples away), so template 5 has no event
    assert (e0.tmpl, e0.n_ifo, e0.ifo_mask, e0.ref_detector, e0.ref_sample) == (3, 2, 0b11, 1, 1000 + D)
    assert abs(e0.net_snr - 10.0) < 1e-12
    assert (e1.tmpl, e1.net_snr, e1.ifo_mask) == (2, 5.0, 0b11)


def test_coincidence_of_a_loud_reference_with_three_detectors():
    trigs = [_t(0, 1, 2, 4500, 6.0), _t(1, 1, 2, 4530, 9.0), _t(2, 1, 2, 4470, 2.0)]
    (e,) = O.coincident_events(trigs, 66)
    # all within 66 of the loudest (det 1 at 4530): 4500 (30), 4470 (60)
    assert (e.n_ifo, e.ifo_mask, e.ref_detector) == (3, 0b111, 1)
    assert abs(e.net_snr - math.sqrt(36 + 81 + 4)) < 1e-12


# --------------------------------------------------------------------------
# Background collection (Section II.D.5) on a hand-built trigger list
# --------------------------------------------------------------------------

def test_background_counts_hand_built():
    snr_e = np.array([4.0, 6.0, 10.0, 100.0], dtype=np.float32)
    xi2_e = np.array([0.1, 1.0, 10.0], dtype=np.float32)
    trigs = [
        _t(0, 3, 0, 1000, 6.0), _t(1, 3, 0, 1030, 8.0),        # coincident pair: not background
        _t(0, 4, 0, 500, 5.0), _t(1, 4, 0, 900, 11.0),          # too far apart: both single
        _t(2, 4, 0, 880, 200.0),                                # joins det 1?  no: det 2 is the loudest,
                                                                # det 1 (20 away) joins it, det 0 stays single
        _t(0, 5, 1, 2100, 4.5),                                 # alone in its template: single
    ]
    xi2 = {(0, 3): 0.5, (1, 3): 0.5, (0, 4): 0.05, (1, 4): 2.0, (2, 4): 50.0, (0, 5): 1.0}
    h = O.background_counts(trigs, lambda t: xi2[(t.detector, t.tmpl)], 3, 66, snr_e, xi2_e)
    assert sorted(h) == [(0, 0)]
    expect = np.zeros((3, 2), dtype=np.int64)
    expect[0, 0] += 1        # det 0, template 4: snr 5 -> bin 0, xi2 0.05 -> bin 0 (below the first edge)
    expect[0, 1] += 1        # det 0, template 5: snr 4.5 -> bin 0, xi2 1.0 -> bin 1 (an edge counts upward)
    assert np.array_equal(h[(0, 0)], expect)
    assert O.background_counts(trigs, lambda t: 1.0, 1, 66, snr_e, xi2_e) == {}
    # edges decide in float32: a value equal to an edge goes to the upper bin
    assert O._bin(6.0, snr_e) == 1 and O._bin(np.nextafter(np.float32(6.0), np.float32(0)), snr_e) == 0
    assert O._bin(1e9, snr_e) == 2 and O._bin(-5.0, snr_e) == 0


# --------------------------------------------------------------------------
# PSD estimation and whitening (Section II.B.2)
# --------------------------------------------------------------------------

def test_median_log_factor_closed_form_against_quadrature():
    from scipy import integrate
    assert abs(O.median_log_factor(1) - 1.0) < 1e-15          # E[log X] = -gamma for one exponential
    assert abs(O.median_log_factor(3) - 9.0 / 8.0) < 1e-14    # exp(2 log 3 - 3 log 2)
    for k in (5, 7, 9):
        m = (k - 1) // 2
        c = math.factorial(k) / math.factorial(m) ** 2
        f = lambda x: math.log(x) * c * (-math.expm1(-x)) ** m * math.exp(-(m + 1) * x)
        e = integrate.quad(f, 0.0, 1.0, limit=200)[0] + integrate.quad(f, 1.0, math.inf, limit=200)[0]
        assert abs(O.median_log_factor(k) - math.exp(e + np.euler_gamma)) < 1e-9


def test_hann_windows_sum_to_one_and_tukey_shape():
    w = O.hann_periodic(512)
    assert np.max(np.abs(w[:256] + w[256:] - 1.0)) < 1e-15
    t = O.tukey(100, 10)
    assert np.all(t[10:90] == 1.0) and np.array_equal(t[:10], t[90:][::-1])
    assert np.all(np.diff(t[:10]) > 0) and 0 < t[0] < t[9] < 1
    # raised-cosine taper: t[i] + t[9 - i] = 1 (mirror symmetry about the half point)
    assert np.max(np.abs(t[:10] + t[:10][::-1] - 1.0)) < 1e-15


def _whiten(x, wh, hop):
    return np.concatenate([wh.push(x[i:i + hop]) for i in range(0, x.size, hop)])


def test_whitening_white_and_coloured_noise():
    """After the PSD settles: unit variance for white noise of any level, and
    coloured noise comes out white (no correlation at small lags)."""
    from scipy.signal import lfilter
    fi, fo = 4096, 512
    rng = np.random.default_rng(2)
    x = 3.0 * rng.standard_normal(120 * fi)
    y = _whiten(x, O.Whitener(fi, fo, 4 * fi, fi), 2 * fi - fi)[30 * fo:]
    assert abs(y.var() - 1.0) < 0.05
    xc = lfilter([1.0, 0.9], [1.0, -0.5], rng.standard_normal(120 * fi))
    yc = _whiten(xc, O.Whitener(fi, fo, 4 * fi, fi), fi)[30 * fo:]
    assert abs(yc.var() - 1.0) < 0.05
    for lag in (1, 2, 3):
        assert abs(np.corrcoef(yc[:-lag], yc[lag:])[0, 1]) < 0.03
    # the raw input was strongly correlated
    assert np.corrcoef(xc[:-1], xc[1:])[0, 1] > 0.5


def test_whitening_latency_and_alignment():
    """Output sample j is input sample j rate_in / rate_out - Z: an impulse in
    white noise (PSD settled) comes out at (t0 + Z) rate_out / rate_in, and the
    output reaches it N/2 input samples after the input did."""
    fi, fo = 4096, 512
    N, Z = 4 * fi, fi
    rng = np.random.default_rng(3)
    x = 0.01 * rng.standard_normal(40 * fi)
    t0 = 30 * fi + 800
    x[t0] += 50.0
    wh = O.Whitener(fi, fo, N, Z)
    hop = N // 2 - Z
    outs, got_at = [], None
    for i in range(0, x.size, hop):
        o = wh.push(x[i:i + hop])
        outs.append(o)
        if got_at is None and sum(v.size for v in outs) > (t0 + Z) * fo // fi:
            got_at = i + hop
    y = np.concatenate(outs)
    assert int(np.argmax(np.abs(y))) == (t0 + Z) * fo // fi
    assert got_at - t0 <= N // 2 + hop


def test_whitening_skips_blocks_with_gaps():
    fi, fo = 4096, 512
    rng = np.random.default_rng(4)
    x = rng.standard_normal(30 * fi)
    x[20 * fi + 5] = np.nan
    wh = O.Whitener(fi, fo, 4 * fi, fi)
    y = _whiten(x, wh, fi)
    assert np.all(np.isfinite(y))
    # the two blocks whose 2 s segments hold the gap add nothing and estimate nothing
    assert wh.n_est == (30 * fi - (4 * fi - 2 * fi)) // fi + 1 - 2
