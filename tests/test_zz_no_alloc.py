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
