"""Checkpoint/resume: a context restored from a checkpoint continues the
stream exactly as the saved context does (SNR rows and triggers identical),
including a window that was half-filled when the checkpoint was taken."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
F0 = 2048
BLOCK = 1536                     # does not divide the 1 s window: checkpoints land mid-window


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_04730_b300 as P
    from paper_2511_04730_b300 import build
    build.build()
    return P


@pytest.mark.parametrize("precision", ["fp32", "fp16_split"])
def test_resume_is_exact(P, precision):
    w = W.make_workload("banks20", n_templates=120, n_banks=2, n_seconds=24, n_det=2, n_inj=0)
    banks = [P.build_svd_bank(b, p) for b, p in zip(w.banks, w.plans)]
    strain = np.stack([w.strain(d) for d in range(2)]).astype(np.float32)
    mk = lambda: P.Context(n_detectors=2, precision=precision, max_block=BLOCK, max_history=64 * F0)

    def run(ctx, k0, k1):
        z, trig = [], []
        for k in range(k0, k1):
            t = k * BLOCK
            ctx.push_all(t, np.ascontiguousarray(strain[:, t:t + BLOCK]))
            z.append(np.concatenate([ctx.snr_block(d, b)[0].cpu().numpy() for d in range(2) for b in ctx.banks]))
            w0, w1 = t // F0, (t + BLOCK) // F0
            if w1 > w0:
                trig.append(ctx.pull(w0, n_windows=w1 - w0))
        return np.concatenate(z, axis=1), np.concatenate(trig)

    with mk() as a:
        for sb in banks:
            a.load_bank(sb)
        run(a, 0, 9)                                   # 13824 samples: window 6 half done
        blob = a.save_state()
        za, ta = run(a, 9, 24)
    with mk() as b:
        for sb in banks:
            b.load_bank(sb)
        b.restore_state(blob)
        zb, tb = run(b, 9, 24)
    assert np.array_equal(za, zb)
    assert np.array_equal(ta, tb)
    assert len(ta) > 0 and ta["window"].min() == 6


def test_mismatched_context_is_rejected(P):
    w = W.make_workload("banks20", n_templates=120, n_banks=2, n_seconds=8, n_det=1, n_inj=0)
    banks = [P.build_svd_bank(b, p) for b, p in zip(w.banks, w.plans)]
    with P.Context(n_detectors=1, precision="fp32", max_block=2048, max_history=64 * F0) as a:
        a.load_bank(banks[0])
        blob = a.save_state()
    with P.Context(n_detectors=1, precision="fp32", max_block=2048, max_history=64 * F0) as b:
        b.load_bank(banks[1])
        with pytest.raises(P.LloidError) as e:
            b.restore_state(blob)
        assert e.value.name == "LLOID_EINVAL"
