"""Serving: admission by HBM budget and continuous batching.

A bank admitted while the stream runs must give, from its second push on,
exactly the triggers it gives when it runs from the start (banks of 200
templates, two template tiles, in both forms of the split path); a bank that
does not fit the budget waits until a running bank finishes."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
F0 = 2048


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
def case(P):
    w = W.make_workload("banks20", n_templates=600, n_banks=3, n_seconds=24, n_det=2, n_inj=0)
    banks = [P.build_svd_bank(b, p) for b, p in zip(w.banks, w.plans)]
    strain = np.stack([w.strain(d) for d in range(2)]).astype(np.float32)
    return banks, strain


def _ctx(P, **kw):
    kw.setdefault("precision", "fp16_split")
    return P.Context(n_detectors=2, max_block=F0, max_history=64 * F0, **kw)


@pytest.mark.parametrize("precision,form", [("fp16_split", "ladder"), ("bf16_split", "f0"), ("fp32", None)])
def test_midstream_admission_matches_from_start(P, case, precision, form):
    from paper_2511_04730_b300.serving import Server
    banks, strain = case
    assert min(len(b[0].coeffs) // 2 for b in banks) > 128       # coefficient rows: re and im per template
    n_blocks = strain.shape[1] // F0
    blk = lambda k: np.ascontiguousarray(strain[:, k * F0:(k + 1) * F0])
    with _ctx(P, precision=precision, form=form) as a, _ctx(P, precision=precision, form=form) as b:
        sa, sb = Server(a, F0), Server(b, F0)
        for i, bank in enumerate(banks):
            sa.submit(bank, tag=i)
        sb.submit(banks[0], tag=0)
        sb.submit(banks[1], tag=1)
        ta, tb = [], []
        for k in range(n_blocks):
            if k == 6:
                sb.submit(banks[2], tag=2)          # arrives while the others run
            ta.append(sa.step(blk(k)))
            tb.append(sb.step(blk(k)))
        ta, tb = np.concatenate(ta), np.concatenate(tb)
    assert sb.admitted_at[2] == 6 * F0
    bank2_a = ta[(ta["bank"] == 2) & (ta["window"] >= 7)]
    bank2_b = tb[(tb["bank"] == 2) & (tb["window"] >= 7)]
    assert len(bank2_a) > 0
    for f in ("detector", "window", "tmpl", "sample", "snr", "phase", "is_bank_max"):
        assert np.array_equal(bank2_a[f], bank2_b[f]), f
    # the other banks are unaffected by the admission
    for bank_id in (0, 1):
        ra, rb = ta[ta["bank"] == bank_id], tb[tb["bank"] == bank_id]
        assert np.array_equal(ra["snr"], rb["snr"]) and np.array_equal(ra["sample"], rb["sample"])


def test_budget_admission_waits_for_memory(P, case):
    from paper_2511_04730_b300.serving import Server
    banks, strain = case
    with _ctx(P) as probe:
        state0, _ = probe.bytes_in_use()
        sizes = []
        for bank in banks:
            before = probe.bytes_in_use()[1]
            probe.load_bank(bank)
            sizes.append(probe.bytes_in_use()[1] - before)
        state = probe.bytes_in_use()[0]
    # room for banks 0 and 1, not for bank 2 as well
    budget = state + sizes[0] + sizes[1] + sizes[2] // 2
    assert sizes[2] <= sizes[0]
    with _ctx(P, hbm_budget=budget) as ctx:
        srv = Server(ctx, F0)
        for i, bank in enumerate(banks):
            srv.submit(bank, tag=i)
        srv.step(np.ascontiguousarray(strain[:, :F0]))
        assert sorted(srv.running.values()) == [0, 1] and len(srv.pending) == 1
        bank0 = [b for b, t in srv.running.items() if t == 0][0]
        srv.finish(bank0)                          # request 0 done: memory frees
        srv.step(np.ascontiguousarray(strain[:, F0:2 * F0]))
        assert sorted(srv.running.values()) == [1, 2] and not srv.pending


def test_paced_latency_is_reported(P, case):
    from paper_2511_04730_b300.serving import Server
    banks, strain = case
    with P.Context(n_detectors=2, precision="fp16_split", max_block=512, max_history=64 * F0) as ctx:
        srv = Server(ctx, 512)
        for i, bank in enumerate(banks):
            srv.submit(bank, tag=i)
        srv.run_paced(lambda k: np.ascontiguousarray(strain[:, k * 512:(k + 1) * 512]), n_blocks=40, pace=10.0)
        lat = srv.latency_summary()
    assert lat["n"] == 40 and 0 < lat["p50"] <= lat["p99"] <= lat["max"]
    print("latency ms", lat)
