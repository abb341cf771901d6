"""The allocation-free trigger entry point agrees with the streaming path.

lloid_triggers_from_snr_noalloc serves callers that cannot allocate device
memory while they run (a real-time strain callback that must not block in
cudaMalloc, or a framework that owns the GPU's memory pool): it extracts the
triggers of an SNR block the caller holds, with scratch compiled into the
library.  Here it is called through the C ABI on two consecutive blocks and
must reproduce lloid_pull_triggers for the same windows.

This file is collected last on purpose, and it sets up everything it needs,
so it passes alone in a fresh process or after the other tests.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

F0 = 2048
TOL = 5e-3          # the split-precision tolerance of the parity tests


def test_noalloc_matches_pull_triggers_on_two_blocks():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_04730_b300 as P
    from paper_2511_04730_b300 import build
    from paper_2511_04730_b300.lloid import triggers_from_snr_noalloc
    build.build()
    w = W.make_workload("bank64", n_seconds=24)
    bank, plan = w.banks[0], w.plans[0]
    d = w.strain(0)
    block = 4 * F0
    calls = 0
    with P.Context(n_detectors=1, precision="fp16_split", max_block=block, max_history=64 * F0) as ctx:
        bid = ctx.load_bank(P.build_svd_bank(bank, plan))
        for t in range(0, d.size, block):
            ctx.push(0, t, d[t:t + block].copy())
            if t < d.size - 2 * block:
                continue
            z, t0 = ctx.snr_block(0, bid)                      # [2M, block] on the device
            ref = ctx.pull(t0 // F0, n_windows=block // F0)    # the existing entry point
            got = triggers_from_snr_noalloc(z, t0, window=F0, threshold=4.0, detector=0, bank=bid)
            calls += 1
            zz = z.cpu().numpy()
            p = np.sqrt(zz[0::2] ** 2 + zz[1::2] ** 2)
            rk = {(int(r["window"]), int(r["tmpl"])): r for r in ref}
            gk = {(int(r["window"]), int(r["tmpl"])): r for r in got}
            for key in set(rk) ^ set(gk):                      # only threshold near-ties may differ
                win, i = key
                seg = p[i, win * F0 - t0:(win + 1) * F0 - t0]
                assert abs(seg.max() - 4.0) < TOL, key
            for key in set(rk) & set(gk):
                a, b = rk[key], gk[key]
                assert abs(float(a["snr"]) - float(b["snr"])) < TOL
                if a["sample"] != b["sample"]:                 # a near-tie: both maxima valid
                    assert abs(p[key[1], int(b["sample"]) - t0] - float(a["snr"])) < TOL
                assert a["detector"] == b["detector"] and a["bank"] == b["bank"]
            assert ref["is_bank_max"].sum() == got["is_bank_max"].sum()
            assert len(got) > 0
    assert calls == 2


def test_noalloc_rejects_blocks_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import ctypes
    from paper_2511_04730_b300 import _lib
    lib = _lib.load()
    n_out = ctypes.c_int64()
    # 300 templates x 1024 windows > 262144 template-window pairs
    st = lib.lloid_triggers_from_snr_noalloc(ctypes.c_void_p(16), 300, 1024 * F0, 0, F0, 4.0, 0, 0,
                                             ctypes.c_void_p(16), 1, ctypes.c_void_p(16), None)
    assert _lib.STATUS_NAMES[st] == "LLOID_ERANGE"


def _reference_triggers(zz, t0, window, threshold):
    """The trigger rule in float32 on the host: per window and template the first
    maximum of |z|^2, a trigger above the threshold."""
    re, im = zz[0::2], zz[1::2]
    p = re * re + im * im
    M, n = p.shape
    out = {}
    for wl in range(n // window):
        seg = p[:, wl * window:(wl + 1) * window]
        k = np.argmax(seg, axis=1)
        for i in range(M):
            if np.sqrt(seg[i, k[i]]) > threshold:
                out[(t0 // window + wl, i)] = (t0 + wl * window + int(k[i]), float(np.sqrt(seg[i, k[i]])))
    return out, p


def test_noalloc_many_chunks_and_a_short_output():
    """More pairs than one compaction chunk (64 templates x 32 windows = 2048 pairs,
    chunks of 1024) are compacted in (window, template) order, and an output shorter
    than the trigger list gets its first records with n_out counting them all."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_04730_b300 import build
    from paper_2511_04730_b300.lloid import TRIGGER_DTYPE, triggers_from_snr_noalloc
    build.build()
    M, n_win, t0 = 64, 32, 5 * F0
    g = torch.Generator(device="cpu").manual_seed(5)
    z = (1.6 * torch.randn((2 * M, n_win * F0), generator=g)).to("cuda")
    got = triggers_from_snr_noalloc(z, t0, window=F0, threshold=4.0, detector=1, bank=3)
    ref, p = _reference_triggers(z.cpu().numpy(), t0, F0, 4.0)
    keys = [(int(r["window"]), int(r["tmpl"])) for r in got]
    assert keys == sorted(keys)                                 # (window, template) order
    assert len(got) > 1024 // 4 and set(keys) == set(ref)       # near-threshold ties are improbable here
    for r in got:
        i = int(r["tmpl"])
        k, snr = ref[(int(r["window"]), i)]
        assert abs(float(r["snr"]) - snr) <= 1e-5 * snr
        if int(r["sample"]) != k:                               # |z|^2 rounded differently: a 1-ulp tie
            assert p[i, int(r["sample"]) - t0] >= p[i, k - t0] * (1 - 1e-6)
        assert int(r["detector"]) == 1 and int(r["bank"]) == 3
    for w in range(t0 // F0, t0 // F0 + n_win):
        rows = got[got["window"] == w]
        if len(rows):
            assert rows["is_bank_max"].sum() == 1
            assert float(rows[rows["is_bank_max"] == 1][0]["snr"]) == float(rows["snr"].max())
    # a short output: the first cap records, and the full count in n_out
    cap = 5
    out = torch.zeros(cap * TRIGGER_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int64, device="cuda")
    head = triggers_from_snr_noalloc(z, t0, window=F0, threshold=4.0, detector=1, bank=3, out=out, n_out=n_out)
    assert int(n_out.item()) == len(got)
    assert len(head) == cap and head.tobytes() == got[:cap].tobytes()
    with pytest.raises(ValueError):
        triggers_from_snr_noalloc(z[:, ::2], t0)                # not contiguous
