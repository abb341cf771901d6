"""Failure handling on the GPU, in the forms that fault, trap or hang nothing.

* An expired device wait: one bounded wait on a barrier that nothing
  completes (the wait every pipeline stage uses) runs out after 2 ms; pulls
  and synchronize report LLOID_ETIMEOUT with its code until the error is
  cleared, and the context then carries on exactly as one that never saw it.
* A slow device (a bounded delay on the stream): a pull with timeout 0
  returns LLOID_ETIMEOUT, the same pull without a limit returns the triggers.
* A failed device allocation while loading a bank keeps nothing; the next
  load succeeds.
* A dropped block leaves a gap: the next push is LLOID_EGAP, or, with gap
  filling, the missing samples are zeros, exactly as if zeros had been pushed.
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
    w = W.make_workload("bank64", n_seconds=24)
    return P.build_svd_bank(w.banks[0], w.plans[0]), w.strain(0)


def _ctx(P, **kw):
    return P.Context(n_detectors=1, precision="fp16_split", max_block=B, max_history=8 * F0, **kw)


def _run(ctx, d, blocks):
    out = []
    for k in blocks:
        ctx.push(0, k * B, np.ascontiguousarray(d[k * B:(k + 1) * B]))
        out.append(ctx.pull(k * B // F0, n_windows=B // F0))
    return np.concatenate(out)


def test_expired_wait_is_reported_and_cleared(P, case):
    sb, d = case
    with _ctx(P) as ref:
        ref.load_bank(sb)
        want = _run(ref, d, range(6))
    with _ctx(P) as ctx:
        ctx.load_bank(sb)
        got = [_run(ctx, d, range(3))]
        ctx.inject_fault("wait_expiry", 2000)
        with pytest.raises(P.LloidError) as e:
            ctx.synchronize()
        assert e.value.name == "LLOID_ETIMEOUT" and "code 90" in str(e.value)
        with pytest.raises(P.LloidError) as e:
            ctx.pull(2 * B // F0)
        assert e.value.name == "LLOID_ETIMEOUT"
        ctx.clear_error()
        ctx.synchronize()
        got.append(_run(ctx, d, range(3, 6)))
    assert np.array_equal(np.concatenate(got), want)


def test_pull_times_out_on_a_slow_device_then_succeeds(P, case):
    sb, d = case
    with _ctx(P) as ref:
        ref.load_bank(sb)
        want = _run(ref, d, range(2))
    with _ctx(P) as ctx:
        ctx.load_bank(sb)
        first = _run(ctx, d, range(1))
        ctx.inject_fault("delay", 300000)              # 0.3 s on the stream before the next push
        ctx.push(0, B, np.ascontiguousarray(d[B:2 * B]))
        with pytest.raises(P.LloidError) as e:
            ctx.pull(B // F0, timeout_ms=0, n_windows=B // F0)
        assert e.value.name == "LLOID_ETIMEOUT"
        second = ctx.pull(B // F0, n_windows=B // F0)
    assert np.array_equal(np.concatenate([first, second]), want)


def test_failed_allocation_keeps_nothing(P, case):
    sb, d = case
    with _ctx(P) as ctx:
        before = ctx.bytes_in_use()
        ctx.inject_fault("alloc", 1)
        with pytest.raises(P.LloidError) as e:
            ctx.load_bank(sb)
        assert e.value.name == "LLOID_ENOMEM"
        assert ctx.bytes_in_use() == before
        bid = ctx.load_bank(sb)
        assert ctx.bytes_in_use()[1] > before[1]
        with _ctx(P) as ref:
            ref.load_bank(sb)
            assert np.array_equal(_run(ctx, d, range(2)), _run(ref, d, range(2)))
        assert bid == 0 or bid == 1


def test_dropped_block_gap_and_zero_fill(P, case):
    sb, d = case
    with _ctx(P) as ctx:
        ctx.load_bank(sb)
        _run(ctx, d, range(1))
        ctx.inject_fault("drop_block", 1)
        ctx.push(0, B, np.ascontiguousarray(d[B:2 * B]))          # lost
        with pytest.raises(P.LloidError) as e:
            ctx.push(0, 2 * B, np.ascontiguousarray(d[2 * B:3 * B]))
        assert e.value.name == "LLOID_EGAP"
    dz = d.copy()
    dz[B:2 * B] = 0.0
    with _ctx(P, fill_gaps=True) as ctx, _ctx(P) as ref:
        bid, rid = ctx.load_bank(sb), ref.load_bank(sb)
        got, want = [_run(ctx, d, range(1))], [_run(ref, dz, range(1))]
        ctx.inject_fault("drop_block", 1)
        ctx.push(0, B, np.ascontiguousarray(d[B:2 * B]))          # lost: filled by zeros below
        ref.push(0, B, np.ascontiguousarray(dz[B:2 * B]))
        ctx.push(0, 2 * B, np.ascontiguousarray(d[2 * B:3 * B]))  # the gap [B, 2B) becomes zeros
        ref.push(0, 2 * B, np.ascontiguousarray(dz[2 * B:3 * B]))
        za, _ = ctx.snr_block(0, bid)
        zb, _ = ref.snr_block(0, rid)
        assert np.array_equal(za.cpu().numpy(), zb.cpu().numpy())
        got.append(ctx.pull(B // F0, n_windows=2 * B // F0))
        want.append(ref.pull(B // F0, n_windows=2 * B // F0))
    assert np.array_equal(np.concatenate(got), np.concatenate(want))
