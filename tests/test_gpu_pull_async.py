"""Submitted pulls (lloid_pull_submit / lloid_pull_collect).

A pull submitted after a push and collected after the next push returns the
same list, entry for entry, as a blocking pull taken right after the push:
later pushes and pulls do not change it.  Lists longer than the part copied at
submit time (the first pull of a slot copies none) are completed from the
slot's device list.  The ticket limit and bad tickets are errors.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
F0 = 2048
B = 4 * F0


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
    w = W.make_workload("banks20", n_templates=600, n_banks=3, n_seconds=128, n_det=2, n_inj=2)
    banks = [P.build_svd_bank(b, p) for b, p in zip(w.banks, w.plans)]
    d = np.stack([w.strain(k) for k in range(2)]).astype(np.float32)
    return banks, d, max(b.n_samples for b in w.banks)


def _ctx(P, hist):
    # a low threshold: hundreds of triggers per window, more than a first pull copies
    return P.Context(n_detectors=2, precision="bf16_split", max_block=B, max_history=hist, threshold=2.5)


def test_submitted_pulls_equal_blocking_pulls(P, case):
    banks, d, hist = case
    n_blk = d.shape[1] // B
    with _ctx(P, hist) as ref:
        for b in banks:
            ref.load_bank(b)
        want = []
        for k in range(n_blk):
            ref.push_all(k * B, np.ascontiguousarray(d[:, k * B:(k + 1) * B]))
            want.append(ref.pull(k * B // F0, n_windows=B // F0))
    assert max(len(x) for x in want) > 256
    with _ctx(P, hist) as ctx:
        for b in banks:
            ctx.load_bank(b)
        got, tickets = [], []
        for k in range(n_blk):
            ctx.push_all(k * B, np.ascontiguousarray(d[:, k * B:(k + 1) * B]))
            tickets.append(ctx.pull_submit(k * B // F0, n_windows=B // F0))
            if len(tickets) == 3:                       # two pushes and two compactions later
                got.append(ctx.pull_collect(tickets.pop(0)))
        got += [ctx.pull_collect(t) for t in tickets]
    assert len(got) == len(want)
    for g, x in zip(got, want):
        assert g.dtype == x.dtype and np.array_equal(g, x)


def test_ticket_limit_and_bad_tickets(P, case):
    banks, d, hist = case
    with _ctx(P, hist) as ctx:
        ctx.load_bank(banks[0])
        ctx.push_all(0, np.ascontiguousarray(d[:, :B]))
        ts = [ctx.pull_submit(0) for _ in range(8)]
        assert sorted(ts) == list(range(8))
        with pytest.raises(P.LloidError) as e:
            ctx.pull_submit(0)
        assert e.value.name == "LLOID_EINVAL"
        first = ctx.pull_collect(ts[0])
        for t in ts[1:]:
            assert np.array_equal(ctx.pull_collect(t), first)
        with pytest.raises(P.LloidError) as e:
            ctx.pull_collect(ts[0])                      # already collected
        assert e.value.name == "LLOID_EINVAL"
        with pytest.raises(P.LloidError) as e:
            ctx.pull_submit(B // F0)                     # not pushed yet
        assert e.value.name == "LLOID_ENOTREADY"
