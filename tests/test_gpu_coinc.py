"""Coincidence across detectors and per-bank clustering on the GPU
(Sections II.D.3-4).  The GPU forms events from its own triggers; the oracle's
rules applied to those same triggers must give exactly the same events (the
logic is integer and comparison work: bit-exact apart from the float network
SNR).  End to end, a coincident injection in three detectors is the event of
its window with all three detectors, as in the oracle run on FP64 SNR."""
import numpy as np
import pytest

import workloads as W
from oracle import lloid_oracle as O
from tests.gpu_helpers import F0

pytestmark = pytest.mark.gpu
DELTA = 66


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_04730_b300 as P
    from paper_2511_04730_b300 import build
    build.build()
    return P


@pytest.fixture(scope="module")
def case():
    w = W.make_workload("bank64", n_seconds=48, n_det=3, n_inj=0)
    b = w.banks[0]
    strains = [w.strain(d).astype(np.float64) for d in range(3)]
    k0 = 30 * F0 + 500
    for d, (dk, snr) in enumerate([(0, 12.0), (20, 9.0), (-40, 7.0)]):
        W.add_injection(strains[d], b, W.Injection(20, k0 + dk, snr, 0.4 + d))
    return w, np.stack(strains), k0


def _as_oracle(trig):
    return [O.Trigger(int(r["detector"]), int(r["bank"]), int(r["tmpl"]), int(r["window"]), int(r["sample"]),
                      float(r["snr"]), float(r["phase"]), float(r["re"]), float(r["im"]), bool(r["is_bank_max"]))
            for r in trig]


@pytest.mark.parametrize("precision", ["fp32", "fp16_split"])
def test_events_follow_the_rules_on_the_gpu_triggers(P, case, precision):
    w, strains, k0 = case
    sb = P.build_svd_bank(w.banks[0], w.plans[0])
    B = 4096
    trig, ev = [], []
    # threshold 3 so that noise triggers coincide in most windows (many events to compare)
    with P.Context(n_detectors=3, precision=precision, max_block=B, max_history=64 * F0,
                   coinc_window=DELTA, threshold=3.0) as ctx:
        ctx.load_bank(sb)
        for t in range(0, strains.shape[1], B):
            ctx.push_all(t, np.ascontiguousarray(strains[:, t:t + B], dtype=np.float32))
            w0, w1 = t // F0, (t + B) // F0
            trig.append(ctx.pull(w0, n_windows=w1 - w0))
            ev.append(ctx.pull_events(w0, n_windows=w1 - w0))
    trig, ev = np.concatenate(trig), np.concatenate(ev)
    ref = O.coincident_events(_as_oracle(trig), DELTA)
    assert len(ev) == len(ref) and len(ref) > 30
    for g, o in zip(ev, ref):
        assert (int(g["window"]), int(g["bank"]), int(g["tmpl"]), int(g["n_ifo"]), int(g["ifo_mask"]),
                int(g["ref_detector"]), int(g["ref_sample"])) == \
               (o.window, o.bank, o.tmpl, o.n_ifo, o.ifo_mask, o.ref_detector, o.ref_sample)
        assert abs(float(g["net_snr"]) - o.net_snr) <= 1e-5 * o.net_snr
    inj = ev[ev["window"] == 30]
    assert len(inj) == 1
    assert (int(inj["tmpl"][0]), int(inj["ifo_mask"][0]), int(inj["ref_detector"][0])) == (20, 0b111, 0)
    # the same event from the FP64 oracle end to end (paper threshold 4 there)
    sl = O.svd_bank(w.banks[0], w.plans[0])
    otr = []
    for d in range(3):
        z = O.lloid_snr(strains[d, :32 * F0], sl, F0)
        otr += [t for t in O.triggers(z, F0, detector=d) if t.window == 30]
    (oe,) = [e for e in O.coincident_events(otr, DELTA) if e.window == 30]
    assert (oe.tmpl, oe.ifo_mask, oe.ref_detector) == (20, 0b111, 0)
    assert abs(float(inj["net_snr"][0]) - oe.net_snr) < 1e-2


def test_events_need_two_detectors(P, case):
    w, strains, _ = case
    sb = P.build_svd_bank(w.banks[0], w.plans[0])
    with P.Context(n_detectors=1, precision="fp32", max_block=4096, max_history=64 * F0) as ctx:
        ctx.load_bank(sb)
        for t in range(0, 8 * F0, 4096):
            ctx.push(0, t, np.ascontiguousarray(strains[0, t:t + 4096], dtype=np.float32))
        assert len(ctx.pull_events(0, n_windows=8)) == 0
        with pytest.raises(P.LloidError) as e:
            ctx.pull_events(8)
        assert e.value.name == "LLOID_ENOTREADY"


def test_background_counts_match_the_rules(P, case):
    """Background histogram (Section II.D.5) of a three-detector stream with
    xi2: the GPU's counts equal the oracle's rules applied to the GPU's own
    triggers (exact integers; bins decided on the same float32 values)."""
    from paper_2511_04730_b300.svdbank import template_autocorrelation
    w, strains, _ = case
    sb = P.build_svd_bank(w.banks[0], w.plans[0])
    R = template_autocorrelation(w.banks[0], 175)
    snr_e = np.geomspace(3.0, 100.0, 9).astype(np.float32)
    xi2_e = np.geomspace(0.05, 50.0, 7).astype(np.float32)
    B = 4096
    trig = []
    with P.Context(n_detectors=3, precision="fp16_split", max_block=B, max_history=64 * F0,
                   coinc_window=DELTA, threshold=3.0) as ctx:
        bid = ctx.load_bank(sb, autocorr=R)
        ctx.set_background_bins(snr_e, xi2_e)
        nw = 0
        for t in range(0, strains.shape[1], B):
            ctx.push_all(t, np.ascontiguousarray(strains[:, t:t + B], dtype=np.float32))
            ready = (t + B - 175) // F0
            if ready > nw:
                trig.append(ctx.pull(nw, n_windows=ready - nw))
                nw = ready
        counts = ctx.background(bid)
    trig = np.concatenate(trig)
    xi2 = {(int(r["detector"]), int(r["tmpl"]), int(r["window"])): float(r["xi2"]) for r in trig}
    ref = O.background_counts(_as_oracle(trig), lambda t: xi2[(t.detector, t.tmpl, t.window)], 3, DELTA,
                              snr_e, xi2_e)
    assert counts.sum() > 100
    for d in range(3):
        assert np.array_equal(counts[d].astype(np.int64), ref.get((bid, d), np.zeros_like(counts[d], dtype=np.int64)))
