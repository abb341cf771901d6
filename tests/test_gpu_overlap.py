"""Trigger windows that overlap (Section II.D.1): window w covers
[max(0, wW - overlap), (w + 1) W).  Triggers against the oracle's rule with
the same overlap, for the ladder form (the 64-template bank) and the f0 form
(a 986-template bank of the 500-bank set), with a signal just before a window
start; and a coincidence that only forms because the windows overlap: the
same signal peaks 40 samples apart in two detectors, on either side of a
window start."""
import numpy as np
import pytest

import workloads as W
from oracle import lloid_oracle as O
from tests.gpu_helpers import F0, TOL, compare_triggers

pytestmark = pytest.mark.gpu
OV = 66                     # (0.0273 + 0.005) s x 2048 Hz


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_04730_b300 as P
    from paper_2511_04730_b300 import build
    build.build()
    return P


def _sub(sl, templates):
    rows = np.stack([2 * templates, 2 * templates + 1], axis=1).reshape(-1)
    return [O.OracleSlice(s.rate, s.j_start, s.bases, s.coeffs[rows]) for s in sl]


@pytest.fixture(scope="module")
def cases():
    out = {}
    w = W.make_workload("bank64", n_seconds=24, n_inj=0)
    d = w.strain(0).astype(np.float64)
    W.add_injection(d, w.banks[0], W.Injection(30, 9 * F0 - 20, 10.0, 0.5))   # peak 20 samples before window 9
    sel = np.arange(64)
    out["ladder"] = (w.banks[0], w.plans[0], d, sel, O.lloid_snr(d, O.svd_bank(w.banks[0], w.plans[0]), F0))
    w = W.make_workload("banks500", bank_indices=(394,), n_seconds=16, n_det=1, n_inj=0)
    d = w.strain(0).astype(np.float64)
    W.add_injection(d, w.banks[0], W.Injection(500, 7 * F0 - 33, 10.0, 1.5))
    sel = np.unique(np.r_[np.arange(0, 986, 29), 500, 985])
    out["f0"] = (w.banks[0], w.plans[0], d, sel, O.lloid_snr(d, _sub(O.svd_bank(w.banks[0], w.plans[0]), sel), F0))
    return out


@pytest.mark.parametrize("precision,form", [("fp32", "ladder"), ("fp16_split", "ladder"), ("bf16_split", "ladder"),
                                            ("fp16_split", "f0"), ("bf16_split", "f0")])
def test_overlapping_windows_against_the_oracle(P, cases, precision, form):
    bank, plan, d, sel, zo = cases[form]
    with P.Context(n_detectors=1, precision=precision, max_block=8192, max_history=8 * F0, overlap=OV,
                   form=None if precision == "fp32" else form) as ctx:
        bid = ctx.load_bank(P.build_svd_bank(bank, plan))
        if precision != "fp32":
            assert ctx.bank_form(bid) == form
        trig = []
        for t in range(0, d.size, 8192):
            ctx.push(0, t, np.ascontiguousarray(d[t:t + 8192], dtype=np.float32))
            trig.append(ctx.pull(t // F0, n_windows=8192 // F0))
    trig = np.concatenate(trig)
    g = trig[np.isin(trig["tmpl"], sel)].copy()
    g["tmpl"] = np.searchsorted(sel, g["tmpl"])
    otr = O.triggers(zo, F0, overlap=OV)
    assert compare_triggers(g, otr, zo, TOL[precision], F0, overlap=OV) == []
    early = [t for t in otr if t.sample < t.window * F0]   # maxima inside the overlap
    assert len(early) > 0
    assert any(int(r["sample"]) < int(r["window"]) * F0 for r in trig)


def test_coincidence_across_a_window_start(P):
    """The same signal peaks 40 samples apart in two detectors, on either side of
    the start of window 8.  Without overlap each window sees one detector's peak
    and only the other's fading edge; with the overlap, window 8 holds both peaks.
    The GPU's events of windows 7 and 8 equal the FP64 oracle's (its triggers
    with the same overlap, then its coincidence rule), and the overlap raises the
    event's network SNR."""
    w = W.make_workload("bank64", n_seconds=16, n_det=2, n_inj=0)
    bank = w.banks[0]
    strains = [w.strain(k).astype(np.float64) for k in range(2)]
    k0 = 8 * F0
    W.add_injection(strains[0], bank, W.Injection(20, k0 - 20, 14.0, 0.3))
    W.add_injection(strains[1], bank, W.Injection(20, k0 + 20, 14.0, 0.9))
    sb = P.build_svd_bank(bank, w.plans[0])
    sl = O.svd_bank(bank, w.plans[0])
    zo = [O.lloid_snr(s, sl, F0) for s in strains]
    best = {}
    for ov in (0, OV):
        with P.Context(n_detectors=2, precision="fp32", max_block=4096, max_history=8 * F0, overlap=ov) as ctx:
            ctx.load_bank(sb)
            got = []
            for t in range(0, 16 * F0, 4096):
                ctx.push_all(t, np.ascontiguousarray(np.stack([s[t:t + 4096] for s in strains]), dtype=np.float32))
                got.append(ctx.pull_events(t // F0, n_windows=2))
            ev = np.concatenate(got)
        otr = [t for d in range(2) for t in O.triggers(zo[d], F0, overlap=ov, detector=d)]
        ref = {e.window: e for e in O.coincident_events(otr, 66) if e.window in (7, 8)}
        g = {int(e["window"]): e for e in ev if int(e["window"]) in (7, 8)}
        assert set(g) == set(ref)
        for win, o in ref.items():
            e = g[win]
            assert (int(e["tmpl"]), int(e["ifo_mask"]), int(e["ref_detector"]), int(e["ref_sample"])) == \
                   (o.tmpl, o.ifo_mask, o.ref_detector, o.ref_sample)
            assert abs(float(e["net_snr"]) - o.net_snr) < 2e-3
        best[ov] = max(o.net_snr for o in ref.values())
    assert best[OV] > best[0] + 0.5
