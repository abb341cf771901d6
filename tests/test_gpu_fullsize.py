"""GPU path vs the FP64 oracle on the shapes the full-size workloads use.

* Four real banks of the 500-bank configuration (885 to 1000 templates, so
  seven or eight 128-template tiles each; ladders 128-256-512-2048,
  128-256-2048, 256-2048 and f0 alone), two detectors, in one context:
  every tile offset of the reconstruction, the finalisation chunks of 64
  templates, the coincidence chunks of 256 templates, and the bank maximum
  across all of them.  The oracle evaluates a spread of templates (every
  tile's first and last rows and every 23rd template between them): it is
  linear in the coefficient rows, so feeding it the selected rows of each
  slice gives exactly those templates' SNR.
* Banks with fixed slice rates whose ladders take every upsampling factor
  F = 2 ... 64 and whose lowest slices run at 32 and 64 Hz (downsampling by
  D = 32 and 64), including a 300-template bank that crosses tiles on the
  shifted-window path of F = 32 and 64.

Tolerances (max |delta z|, complex): 1e-3 FP32, 5e-3 split precision."""
import numpy as np
import pytest

import workloads as W
from oracle import lloid_oracle as O
from tests.gpu_helpers import F0, TOL, compare_triggers

pytestmark = pytest.mark.gpu
PRECISIONS = ["fp32", "fp16_split", "bf16_split"]
# the split paths in both forms of a bank (per-rate ladder; everything brought up to f0 first)
CASES = [("fp32", None)] + [(p, f) for p in PRECISIONS[1:] for f in ("ladder", "f0")]
CONFIG4_BANKS = (168, 373, 394, 466)
DELTA = 66


@pytest.fixture(scope="module")
def lloid():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_04730_b300 as P
    from paper_2511_04730_b300 import build
    build.build()
    return P


def _spread(M):
    """Templates the oracle evaluates: each 128-tile's first and last rows and
    every 23rd template, plus the bank's last template."""
    sel = set(range(0, M, 23)) | {M - 1}
    for t in range(0, M, 128):
        sel |= {t, min(M - 1, t + 127)}
    return np.array(sorted(sel))


def _rows_of(templates):
    return np.stack([2 * templates, 2 * templates + 1], axis=1).reshape(-1)


def _oracle_subset(slices, templates, d):
    """The oracle's SNR rows of the given templates (their coefficient rows only)."""
    rows = _rows_of(templates)
    sub = [O.OracleSlice(s.rate, s.j_start, s.bases, s.coeffs[rows]) for s in slices]
    return O.lloid_snr(d.astype(np.float64), sub, F0)


def _stream(ctx, bids, strains, block, n_det):
    """Push every detector together; keep each bank's SNR rows and every trigger and event."""
    T = strains.shape[1]
    z = {(b, det): [] for b in bids for det in range(n_det)}
    trig, ev = [], []
    for t in range(0, T, block):
        ctx.push_all(t, np.ascontiguousarray(strains[:, t:t + block], dtype=np.float32))
        for b in bids:
            for det in range(n_det):
                zb, t0 = ctx.snr_block(det, b)
                assert t0 == t
                z[(b, det)].append(zb.cpu().numpy())
        w0, w1 = t // F0, (t + block) // F0
        trig.append(ctx.pull(w0, n_windows=w1 - w0))
        if n_det > 1:
            ev.append(ctx.pull_events(w0, n_windows=w1 - w0))
    z = {k: np.concatenate(v, axis=1) for k, v in z.items()}
    return z, np.concatenate(trig), (np.concatenate(ev) if ev else None)


def _max_dz(z_rows, zo):
    d = (z_rows[0::2] - zo[0::2]) ** 2 + (z_rows[1::2] - zo[1::2]) ** 2
    return float(np.sqrt(d.max()))


# ---------------------------------------------------------------------------
# real banks of the 500-bank configuration
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def c4():
    n_det, secs = 2, 16
    w = W.make_workload("banks500", bank_indices=CONFIG4_BANKS, n_seconds=secs, n_det=n_det, n_inj=0)
    strains = np.stack([w.strain(d).astype(np.float64) for d in range(n_det)])
    # a coincident injection into template 700 (sixth tile) of the 885-template bank
    for d, (dk, snr) in enumerate([(0, 15.0), (30, 11.0)]):
        W.add_injection(strains[d], w.banks[0], W.Injection(700, 12 * F0 + 333 + dk, snr, 1.1 + d))
    sel, zo = [], {}
    for k, (bank, plan) in enumerate(zip(w.banks, w.plans)):
        s = _spread(bank.n_templates)
        if k == 0:
            s = np.union1d(s, [700])
        sel.append(s)
        sl = O.svd_bank(bank, plan)
        for d in range(n_det):
            zo[(k, d)] = _oracle_subset(sl, s, strains[d])
    return w, strains, sel, zo


@pytest.mark.parametrize("precision,form", CASES)
def test_config4_banks_snr_and_triggers(lloid, c4, precision, form):
    w, strains, sel, zo = c4
    n_det = strains.shape[0]
    assert [b.n_templates for b in w.banks] == [885, 1000, 986, 1000]
    assert sorted({F0 // r for p in w.plans for r in p.rate}) == [1, 4, 8, 16]
    # threshold 3: most template-windows trigger, so the chunked finalisation and coincidence see
    # dense lists (the oracle's triggers below use the same threshold)
    with lloid.Context(n_detectors=n_det, precision=precision, max_block=16384, max_history=16 * F0,
                       coinc_window=DELTA, threshold=3.0, form=form) as ctx:
        bids = [ctx.load_bank(lloid.build_svd_bank(b, p)) for b, p in zip(w.banks, w.plans)]
        if form:
            assert [ctx.bank_form(b) for b in bids] == [form] * 4
        z, trig, ev = _stream(ctx, bids, strains, 16384, n_det)
    worst = 0.0
    for k, b in enumerate(bids):
        rows = _rows_of(sel[k])
        for d in range(n_det):
            err = _max_dz(z[(b, d)][rows], zo[(k, d)])
            worst = max(worst, err)
            print(f"{precision} {form} bank {k} (M={w.banks[k].n_templates}) det {d}: max|dz| = {err:.3e}")
            assert err <= TOL[precision]
            # triggers of the evaluated templates vs the oracle's, per bank and detector
            g = trig[(trig["bank"] == b) & (trig["detector"] == d) & np.isin(trig["tmpl"], sel[k])].copy()
            g["tmpl"] = np.searchsorted(sel[k], g["tmpl"])
            otr = O.triggers(zo[(k, d)], F0, threshold=3.0)
            assert compare_triggers(g, otr, zo[(k, d)], TOL[precision], F0, threshold=3.0) == []
    print(f"{precision} {form}: worst max|dz| over the four banks = {worst:.3e}")
    # bank maximum: one per (detector, bank, window), and it is the loudest of the bank's triggers
    n_max = 0
    for (d, b, win) in {(int(r["detector"]), int(r["bank"]), int(r["window"])) for r in trig}:
        rows = trig[(trig["detector"] == d) & (trig["bank"] == b) & (trig["window"] == win)]
        assert rows["is_bank_max"].sum() == 1
        assert rows[rows["is_bank_max"] == 1][0]["snr"] >= rows["snr"].max() - TOL[precision]
        n_max += 1
    assert n_max > n_det * len(bids) * (strains.shape[1] // F0) // 2
    # coincidence and clustering over chunks of 256 templates: the oracle's rules on the GPU's triggers
    as_or = [O.Trigger(int(r["detector"]), int(r["bank"]), int(r["tmpl"]), int(r["window"]), int(r["sample"]),
                       float(r["snr"]), float(r["phase"]), float(r["re"]), float(r["im"]), bool(r["is_bank_max"]))
             for r in trig]
    ref = sorted(O.coincident_events(as_or, DELTA), key=lambda e: (e.window, e.bank))
    ev = np.sort(ev, order=["window", "bank"])
    assert len(ev) == len(ref) and len(ref) >= 3
    assert max(int(e["tmpl"]) for e in ev) >= 256
    for g, o in zip(ev, ref):
        assert (int(g["window"]), int(g["bank"]), int(g["tmpl"]), int(g["n_ifo"]), int(g["ifo_mask"]),
                int(g["ref_detector"]), int(g["ref_sample"])) == \
               (o.window, o.bank, o.tmpl, o.n_ifo, o.ifo_mask, o.ref_detector, o.ref_sample)
        assert abs(float(g["net_snr"]) - o.net_snr) <= 1e-5 * o.net_snr
    # the injection: an event of both detectors in its window (its template's neighbours are
    # nearly degenerate with it, so the loudest template need not be 700 itself)
    inj = ev[(ev["window"] == 12) & (ev["bank"] == bids[0])]
    assert len(inj) == 1 and int(inj["ifo_mask"][0]) == 0b11 and float(inj["net_snr"][0]) > 15.0


# ---------------------------------------------------------------------------
# every ladder factor, 32 and 64 Hz slices
# ---------------------------------------------------------------------------
# (templates, slice boundaries in seconds, fixed rates): each bank's ladder is
# its distinct rates plus f0
ZOO = [
    (12, (0.0, 1.5, 8.0), (2048, 32)),                                        # F = 64, D = 64
    (12, (0.0, 1.0, 8.0), (2048, 64)),                                        # F = 32, D = 32
    (12, (0.0, 1.0, 8.0), (2048, 128)),                                       # F = 16
    (300, (0.0, 0.5, 2.0, 8.0), (2048, 512, 32)),                             # F = 16 then 4, three tiles
    (300, (0.0, 1.0, 8.0), (2048, 64)),                                       # F = 32, three tiles
    (6, (0.0, 0.25, 0.5, 1.0, 1.5, 2.0, 3.0, 8.0), (2048, 1024, 512, 256, 128, 64, 32)),    # F = 2 x 6
]
# the small banks have at most 96 bases, so they can run in the f0 form; the 300-template
# banks (more than 96 bases) stay in the ladder form whatever the context asks


@pytest.fixture(scope="module")
def zoo():
    rng = np.random.Generator(np.random.PCG64(11))
    banks, plans = [], []
    for M, edges, rates in ZOO:
        bank = W.ChirpBank(np.sort(rng.uniform(3.0, 6.0, M)), 8 * F0, F0)
        plan = W.plan_slices(bank, edges, fixed_rates=rates)
        assert tuple(plan.rate) == rates
        banks.append(bank)
        plans.append(plan)
    d = W.white_noise(20 * F0, 77).astype(np.float64)
    W.add_injection(d, banks[3], W.Injection(250, 14 * F0 + 99, 13.0, 0.3))
    zo, sel = [], []
    for bank, plan in zip(banks, plans):
        s = _spread(bank.n_templates) if bank.n_templates > 128 else np.arange(bank.n_templates)
        sel.append(s)
        zo.append(_oracle_subset(O.svd_bank(bank, plan), s, d))
    return banks, plans, d, sel, zo


@pytest.mark.parametrize("precision,form", CASES)
def test_every_ladder_factor(lloid, zoo, precision, form):
    banks, plans, d, sel, zo = zoo
    with lloid.Context(n_detectors=1, precision=precision, max_block=8192, max_history=8 * F0, form=form) as ctx:
        bids = [ctx.load_bank(lloid.build_svd_bank(b, p)) for b, p in zip(banks, plans)]
        forms = [ctx.bank_form(b) for b in bids]
        z, trig, _ = _stream(ctx, bids, d[None, :], 8192, 1)
    if form == "f0":
        assert [f for k, f in enumerate(forms) if banks[k].n_templates < 100] == ["f0"] * 4
    for k, b in enumerate(bids):
        err = _max_dz(z[(b, 0)][_rows_of(sel[k])], zo[k])
        print(f"{precision} {form}->{forms[k]} ladder {ZOO[k][2]} (M={banks[k].n_templates}): max|dz| = {err:.3e}")
        assert err <= TOL[precision]
        g = trig[(trig["bank"] == b) & np.isin(trig["tmpl"], sel[k])].copy()
        g["tmpl"] = np.searchsorted(sel[k], g["tmpl"])
        assert compare_triggers(g, O.triggers(zo[k], F0), zo[k], TOL[precision], F0) == []
