"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Sizes: the 64-template bank (two slices, 2048 and 256 Hz) over 64 s spans
many FIR, upsample and reconstruction tiles; the 1000-template bank checks
the full five-rate ladder on sampled segments.  Tolerances (max |delta z|,
complex): 1e-3 for the FP32 path, 5e-3 for the split-precision tensor-core
paths."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import lloid_oracle as O
from tests.gpu_helpers import F0, TOL, compare_triggers, max_abs_complex, stream_snr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lloid():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_04730_b300 as P
    from paper_2511_04730_b300 import build
    build.build()
    return P


@pytest.fixture(scope="module")
def bank64_case():
    w = W.make_workload("bank64")
    bank, plan = w.banks[0], w.plans[0]
    d = w.strain(0)
    z_or = O.lloid_snr(d.astype(np.float64), O.svd_bank(bank, plan), F0)
    return w, bank, plan, d, z_or


def _ctx(P, precision, **kw):
    return P.Context(n_detectors=kw.pop("n_detectors", 1), precision=precision,
                     max_block=kw.pop("max_block", 16384), max_history=kw.pop("max_history", 64 * F0), **kw)


# the split paths in both forms of a bank (per-rate ladder; basis outputs brought up to f0 first)
FORMS = [("fp32", None)] + [(p, f) for p in ("fp16_split", "bf16_split") for f in ("ladder", "f0")]


@pytest.mark.parametrize("precision,form", FORMS)
def test_snr_parity_bank64(lloid, bank64_case, precision, form):
    w, bank, plan, d, z_or = bank64_case
    sb = lloid.build_svd_bank(bank, plan)
    with _ctx(lloid, precision, form=form) as ctx:
        bid = ctx.load_bank(sb)
        form = f"{form}->{ctx.bank_form(bid)}"
        z = stream_snr(ctx, bid, d, 8192)
    err = max_abs_complex(z, z_or)
    print(f"{precision} {form}: max|dz| = {err:.3e}")
    assert err <= TOL[precision]
    # the injection is recovered at its sample
    inj = w.injections[0][0]
    i, k = inj.tmpl, inj.end_sample
    assert abs(abs(complex(z[2 * i, k], z[2 * i + 1, k])) - abs(complex(z_or[2 * i, k], z_or[2 * i + 1, k]))) < TOL[precision]


@pytest.mark.parametrize("precision", ["fp32", "fp16_split", "bf16_split"])
def test_trigger_parity_bank64(lloid, bank64_case, precision):
    w, bank, plan, d, z_or = bank64_case
    sb = lloid.build_svd_bank(bank, plan)
    with _ctx(lloid, precision) as ctx:
        bid = ctx.load_bank(sb)
        got = []
        for t in range(0, d.size, 4096):
            ctx.push(0, t, d[t:t + 4096].copy())
            got += [ctx.pull(win) for win in range(t // F0, (t + 4096) // F0)]
        trig = np.concatenate(got)
    otr = O.triggers(z_or, F0)
    assert len(trig) > 0
    problems = compare_triggers(trig, otr, z_or, TOL[precision], F0)
    assert problems == []
    # bank maximum: one per window, on the loudest template
    for win in range(d.size // F0):
        rows = trig[trig["window"] == win]
        if len(rows):
            assert rows["is_bank_max"].sum() == 1
            top = rows[rows["is_bank_max"] == 1][0]
            assert top["snr"] >= rows["snr"].max() - TOL[precision]
    # phase = atan2(im, re)
    assert np.allclose(trig["phase"], np.arctan2(trig["im"], trig["re"]), atol=1e-5)


@pytest.mark.parametrize("precision", ["fp32", "fp16_split"])
def test_streaming_block_sizes_identical(lloid, bank64_case, precision):
    """The SNR does not depend on how the stream is cut into blocks."""
    w, bank, plan, d, _ = bank64_case
    sb = lloid.build_svd_bank(bank, plan)
    d = d[: 24 * F0]
    outs = []
    for block in (16384, 384, 1152, 2048):
        with _ctx(lloid, precision) as ctx:
            bid = ctx.load_bank(sb)
            outs.append(stream_snr(ctx, bid, d, block))
    for z in outs[1:]:
        assert np.array_equal(z, outs[0])


@pytest.mark.parametrize("precision,form", FORMS)
@pytest.mark.parametrize("which", [0, 1])
def test_single_slice_banks(lloid, bank64_case, precision, form, which):
    """One slice at a time: slice 0 alone (f0, no ladder: FIR + top level) and
    slice 1 alone (256 Hz: the SNR comes only through the Eq. 7-8 ladder)."""
    w, bank, plan, d, _ = bank64_case
    sb = lloid.build_svd_bank(bank, plan)
    sl = O.svd_bank(bank, plan)
    d = d[: 16 * F0]
    z_or = O.lloid_snr(d.astype(np.float64), [sl[which]], F0)
    with _ctx(lloid, precision, form=form) as ctx:
        bid = ctx.load_bank([sb[which]])
        z = stream_snr(ctx, bid, d, 4096)
    err = max_abs_complex(z, z_or)
    print(f"{precision} {form} slice {which}: max|dz| = {err:.3e}")
    assert err <= TOL[precision]


def test_push_all_equals_single_detector_pushes(lloid, bank64_case):
    w, bank, plan, d, _ = bank64_case
    sb = lloid.build_svd_bank(bank, plan)
    d2 = W.white_noise(d.size, 901)
    n = 8 * F0
    with _ctx(lloid, "fp32", n_detectors=2) as a, _ctx(lloid, "fp32", n_detectors=2) as b:
        ia, ib = a.load_bank(sb), b.load_bank(sb)
        for t in range(0, n, 2048):
            a.push_all(t, np.stack([d[t:t + 2048], d2[t:t + 2048]]).astype(np.float32))
            b.push(0, t, d[t:t + 2048].copy())
            b.push(1, t, d2[t:t + 2048].copy())
        for det in (0, 1):
            za, _ = a.snr_block(det, ia)
            zb, _ = b.snr_block(det, ib)
            assert np.array_equal(za.cpu().numpy(), zb.cpu().numpy())
        ta = np.concatenate([a.pull(x) for x in range(n // F0)])
        tb = np.concatenate([b.pull(x) for x in range(n // F0)])
        assert np.array_equal(ta, tb)


def test_device_pointer_push(lloid, bank64_case):
    import torch
    w, bank, plan, d, _ = bank64_case
    sb = lloid.build_svd_bank(bank, plan)
    with _ctx(lloid, "fp32") as a, _ctx(lloid, "fp32") as b:
        ia, ib = a.load_bank(sb), b.load_bank(sb)
        for t in range(0, 4 * F0, 2048):
            a.push(0, t, d[t:t + 2048].copy())
            b.push(0, t, torch.from_numpy(d[t:t + 2048].copy()).cuda())
        za, _ = a.snr_block(0, ia)
        zb, _ = b.snr_block(0, ib)
        assert torch.equal(za, zb)


@pytest.fixture(scope="module")
def ladder_case():
    w = W.make_workload("bank1000", n_templates=96, n_seconds=96, n_det=1, n_inj=2)
    bank, plan = w.banks[0], w.plans[0]
    d = w.strain(0)
    # oracle on [a - H, a + S): H = one full template plus the ladder halos, a
    # multiple of the lowest rate's decimation so the grid is preserved
    sl = O.svd_bank(bank, plan)
    H, S = 66 * F0, 2 * F0
    segs = {a: O.lloid_snr(d[a - H:a + S].astype(np.float64), sl, F0)[:, H:] for a in (66 * F0, 90 * F0)}
    return bank, plan, d, segs, S


@pytest.mark.parametrize("precision,form", FORMS)
def test_multirate_ladder_bank1000_segments(lloid, ladder_case, precision, form):
    """Five-rate bank (2048/1024/512/256/128 Hz, 64 s templates): sampled
    segments of the stream against the oracle run on the segment's history."""
    bank, plan, d, segs, S = ladder_case
    assert sorted(set(plan.rate)) == [128, 256, 512, 1024, 2048]
    sb = lloid.build_svd_bank(bank, plan)
    with _ctx(lloid, precision, max_history=64 * F0, form=form) as ctx:
        bid = ctx.load_bank(sb)
        z = stream_snr(ctx, bid, d, 16384)
    for a, zo in segs.items():
        err = max_abs_complex(z[:, a:a + S], zo)
        print(f"{precision} {form} segment {a}: max|dz| = {err:.3e}")
        assert err <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp32", "fp16_split", "bf16_split"])
def test_triggers_across_finalize_chunks(lloid, ladder_case, precision):
    """96 templates: window maxima are finalised in chunks of 64 templates and
    the bank maximum is found across the chunks.  Triggers of the windows of
    the oracle's segments (absolute windows and samples) against the oracle's."""
    bank, plan, d, segs, S = ladder_case
    sb = lloid.build_svd_bank(bank, plan)
    end = max(segs) + S
    got = []
    with _ctx(lloid, precision, max_history=64 * F0) as ctx:
        ctx.load_bank(sb)
        for t in range(0, end, 16384):
            ctx.push(0, t, np.ascontiguousarray(d[t:t + 16384], dtype=np.float32))
            got += [ctx.pull(win) for win in range(t // F0, (t + 16384) // F0)]
    trig = np.concatenate(got)
    n_checked = 0
    for a, zo in segs.items():
        w0, w1 = a // F0, (a + S) // F0
        g = trig[(trig["window"] >= w0) & (trig["window"] < w1)]
        otr = O.triggers(zo, F0, n_windows=w1, t_offset=a)
        assert compare_triggers(g, otr, zo, TOL[precision], F0, t_offset=a) == []
        for w in range(w0, w1):
            rows = g[g["window"] == w]
            if len(rows):
                n_checked += 1
                assert rows["is_bank_max"].sum() == 1
                top = rows[rows["is_bank_max"] == 1][0]
                assert top["snr"] >= rows["snr"].max() - TOL[precision]
    assert n_checked > 0


def test_error_codes(lloid, bank64_case):
    w, bank, plan, d, _ = bank64_case
    sb = lloid.build_svd_bank(bank, plan)
    with _ctx(lloid, "fp32") as ctx:
        bid = ctx.load_bank(sb)
        with pytest.raises(lloid.LloidError) as e:
            ctx.push(0, 128, d[:2048].copy())          # stream starts at 0
        assert e.value.name == "LLOID_EGAP"
        with pytest.raises(lloid.LloidError) as e:
            ctx.push(0, 0, d[:100].copy())             # not a multiple of 128
        assert e.value.name == "LLOID_EINVAL"
        ctx.push(0, 0, d[:2048].copy())
        with pytest.raises(lloid.LloidError) as e:
            ctx.pull(1)                                 # window 1 not pushed yet
        assert e.value.name == "LLOID_ENOTREADY"
        ctx.pull(0)
        # pre-synchronisation violated: a 256 Hz slice needs J >= 8 (N_down + N_up) = 320
        bad = [lloid.SliceArrays(256, 312, sb[1].bases, sb[1].coeffs, 1.0)]
        ok = [lloid.SliceArrays(256, 320, sb[1].bases, sb[1].coeffs, 1.0)]
        ctx.load_bank(ok)
        with pytest.raises(lloid.LloidError) as e:
            ctx.load_bank(bad)
        assert e.value.name == "LLOID_EINVAL" and "pre-synchronisation" in str(e.value)
    with _ctx(lloid, "fp32", hbm_budget=64 << 20) as ctx:
        with pytest.raises(lloid.LloidError) as e:
            for _ in range(64):
                ctx.load_bank(sb)
        assert e.value.name == "LLOID_EBUDGET"
