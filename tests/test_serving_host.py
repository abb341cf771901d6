"""The serving loop's host logic on the CPU, over a stand-in context that
records the calls and refuses banks past a memory budget the way
lloid_load_bank does (LLOID_EBUDGET): FIFO admission, admission resumed when a
finished bank frees room, the windows each block completes, paced arrival
times and the latency percentiles (nearest rank)."""
import numpy as np
import pytest

from paper_2511_04730_b300.lloid import TRIGGER_DTYPE, LloidError
from paper_2511_04730_b300.serving import Server

W = 2048


class FakeCtx:
    def __init__(self, budget):
        self.window = W
        self.budget = budget            # bank "sizes" that fit at once
        self.loaded = {}
        self.next_id = 0
        self.pushes, self.pulls = [], []

    def load_bank(self, slices):
        size = slices["size"]
        if sum(self.loaded.values()) + size > self.budget:
            raise LloidError(-3, "over budget")
        bid = self.next_id
        self.next_id += 1
        self.loaded[bid] = size
        return bid

    def unload_bank(self, bid):
        del self.loaded[bid]

    def push_all(self, t0, blocks):
        self.pushes.append((t0, blocks.shape[-1]))

    def pull(self, w0, n_windows=1):
        self.pulls.append((w0, n_windows))
        out = np.zeros(n_windows, dtype=TRIGGER_DTYPE)
        out["window"] = np.arange(w0, w0 + n_windows)
        return out


def test_fifo_admission_under_the_budget():
    ctx = FakeCtx(budget=10)
    srv = Server(ctx, block=W)
    for i, size in enumerate([4, 5, 3, 2]):
        srv.submit({"size": size}, tag=i)
    srv.step(np.zeros((2, W), np.float32))
    assert sorted(srv.running.values()) == [0, 1]          # 4 + 5 fit; 3 more would not: FIFO stops there
    assert [t for _, t in srv.pending] == [2, 3]           # the smaller bank behind it waits its turn
    srv.finish(next(b for b, t in srv.running.items() if t == 0))
    srv.step(np.zeros((2, W), np.float32))
    assert sorted(srv.running.values()) == [1, 2, 3]       # 5 + 3 + 2 = 10 fits once the 4 has left
    assert not srv.pending
    assert srv.admitted_at == {0: 0, 1: 0, 2: W, 3: W}     # stream position at admission


def test_other_load_errors_are_raised():
    class Broken(FakeCtx):
        def load_bank(self, slices):
            raise LloidError(-1, "bad bank")
    srv = Server(Broken(budget=10), block=W)
    srv.submit({"size": 1})
    with pytest.raises(LloidError) as e:
        srv.step(np.zeros((1, W), np.float32))
    assert e.value.name == "LLOID_EINVAL"


@pytest.mark.parametrize("block", [W // 4, W, 3 * W])
def test_each_block_pulls_the_windows_it_completes(block):
    ctx = FakeCtx(budget=1)
    srv = Server(ctx, block=block)
    got = []
    for _ in range(12):
        got.append(srv.step(np.zeros((3, block), np.float32)))
    assert [p for p, _ in ctx.pushes] == [k * block for k in range(12)]
    windows = np.concatenate([g["window"] for g in got])
    assert np.array_equal(windows, np.arange(12 * block // W))   # every window once, in order
    for (w0, n), k in zip(ctx.pulls, [k for k in range(12) if (k + 1) * block // W > k * block // W]):
        assert w0 == k * block // W and n == (k + 1) * block // W - w0


def test_latency_percentiles_are_nearest_rank():
    srv = Server(FakeCtx(1), block=W)
    assert srv.latency_summary() == {}
    srv.latency_ms = list(np.random.default_rng(0).permutation(np.arange(1.0, 1001.0)))
    q = srv.latency_summary()
    assert (q["p50"], q["p99"], q["p99.9"], q["max"], q["n"]) == (500.0, 990.0, 999.0, 1000.0, 1000)


def test_paced_run_records_one_latency_per_block():
    ctx = FakeCtx(budget=1)
    srv = Server(ctx, block=W // 4)
    seen = []
    srv.run_paced(lambda k: np.zeros((2, W // 4), np.float32), 40, pace=1e6, on_triggers=lambda k, t: seen.append(k))
    assert len(srv.latency_ms) == 40 and seen == list(range(40))
    assert all(x >= 0.0 for x in srv.latency_ms)
    assert len(ctx.pulls) == 10                            # a window every fourth block
