"""Several banks in one context (the batched path) and serving isolation.

Three banks cut from the same chirp family with different chirp-mass ranges
have different lengths (64, 32, 8 s), slice plans and ladders (5, 4 and 3
rates; upsampling factors 2 and 8).  All of them run in the same launches;
each bank's SNR must match the FP64 oracle, and must be identical to the SNR
the bank produces when it is loaded alone (a result does not depend on what
else is being filtered)."""
import numpy as np
import pytest

import workloads as W
from oracle import lloid_oracle as O
from tests.gpu_helpers import F0, TOL, max_abs_complex

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
def case():
    w = W.make_workload("banks20", n_templates=240, n_banks=3, n_seconds=96, n_det=1, n_inj=3)
    d = w.strain(0)
    H, S = 66 * F0, 2 * F0
    segs = []
    for bank, plan in zip(w.banks, w.plans):
        sl = O.svd_bank(bank, plan)
        segs.append({a: O.lloid_snr(d[a - H:a + S].astype(np.float64), sl, F0)[:, H:] for a in (66 * F0, 90 * F0)})
    return w, d, segs, S


def _stream(ctx, bids, d, block):
    zs = {b: [] for b in bids}
    trig = []
    for t in range(0, d.size, block):
        ctx.push(0, t, np.ascontiguousarray(d[t:t + block]))
        for b in bids:
            z, t0 = ctx.snr_block(0, b)
            zs[b].append(z.cpu().numpy())
        trig.append(ctx.pull(t // F0, n_windows=block // F0))
    return {b: np.concatenate(v, axis=1) for b, v in zs.items()}, np.concatenate(trig)


@pytest.mark.parametrize("precision", ["fp32", "fp16_split", "bf16_split"])
def test_three_banks_in_one_context(lloid, case, precision):
    w, d, segs, S = case
    with lloid.Context(n_detectors=1, precision=precision, max_block=16384, max_history=64 * F0) as ctx:
        bids = [ctx.load_bank(lloid.build_svd_bank(b, p)) for b, p in zip(w.banks, w.plans)]
        zs, trig = _stream(ctx, bids, d, 16384)
    for k, b in enumerate(bids):
        for a, zo in segs[k].items():
            err = max_abs_complex(zs[b][:, a:a + S], zo)
            print(f"{precision} bank {k} segment {a}: max|dz| = {err:.3e}")
            assert err <= TOL[precision]
    # every window has exactly one bank maximum per (detector, bank) that triggered
    for win in np.unique(trig["window"]):
        for b in bids:
            rows = trig[(trig["window"] == win) & (trig["bank"] == b)]
            if len(rows):
                assert rows["is_bank_max"].sum() == 1


@pytest.mark.parametrize("precision", ["fp32", "fp16_split"])
def test_bank_alone_equals_bank_in_the_mix(lloid, case, precision):
    w, d, segs, S = case
    d = d[: 24 * F0]
    banks = [lloid.build_svd_bank(b, p) for b, p in zip(w.banks, w.plans)]
    with lloid.Context(n_detectors=1, precision=precision, max_block=8192, max_history=64 * F0) as mix:
        mids = [mix.load_bank(sb) for sb in banks]
        z_mix, t_mix = _stream(mix, mids, d, 8192)
    for k, sb in enumerate(banks):
        with lloid.Context(n_detectors=1, precision=precision, max_block=8192, max_history=64 * F0) as alone:
            aid = alone.load_bank(sb)
            z_alone, t_alone = _stream(alone, [aid], d, 8192)
        assert np.array_equal(z_alone[aid], z_mix[mids[k]])
        tm = t_mix[t_mix["bank"] == mids[k]]
        for f in ("window", "tmpl", "sample", "snr", "phase", "is_bank_max"):
            assert np.array_equal(tm[f], t_alone[f]), f
