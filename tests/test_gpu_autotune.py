"""The autotuner of the batched path (lloid_autotune): it times seven
candidate settings (every bank in the ladder form; the cost-model choice at
form ratios 1, 0.5 and 2; every bank that can in the f0 form; then one and two
basis-filter CTAs per SM) on scratch contexts, and its choice, applied to a
streaming context, gives the same SNR as the default setting within the
split-precision tolerance."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_helpers import F0, TOL

pytestmark = pytest.mark.gpu


def test_autotune_times_candidates_and_its_choice_streams():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2511_04730_b300 as P
    from paper_2511_04730_b300 import build
    build.build()
    w = W.make_workload("banks500", bank_indices=(168, 373, 394, 466, 47), n_seconds=16, n_det=2, n_inj=0)
    banks = [P.build_svd_bank(b, p) for b, p in zip(w.banks, w.plans)]
    hist = max(b.n_samples for b in w.banks)
    tun = P.autotune(banks, 8192, reps=2, n_detectors=2, precision="bf16_split", max_history=hist)
    assert len(tun["candidates"]) == 7 and 0 <= tun["best"] < 7
    assert all(c["ms_per_push"] > 0 for c in tun["candidates"])
    best = tun["candidates"][tun["best"]]
    assert best["ms_per_push"] == min(c["ms_per_push"] for c in tun["candidates"])
    print("autotune:", tun)
    d = np.stack([w.strain(k) for k in range(2)]).astype(np.float32)
    z = {}
    for name, kw in (("default", {}), ("tuned", {"tuning": tun})):
        with P.Context(n_detectors=2, precision="bf16_split", max_block=8192, max_history=hist, **kw) as ctx:
            ids = [ctx.load_bank(b) for b in banks]
            forms = [ctx.bank_form(i) for i in ids]
            if name == "tuned" and best["form"] == "all ladder":
                assert forms == ["ladder"] * len(ids)
            for t in range(0, d.shape[1], 8192):
                ctx.push_all(t, np.ascontiguousarray(d[:, t:t + 8192]))
            z[name] = [ctx.snr_block(1, i)[0].cpu().numpy() for i in ids]
    for a, b in zip(z["default"], z["tuned"]):
        dz = np.sqrt((a[0::2] - b[0::2]) ** 2 + (a[1::2] - b[1::2]) ** 2).max()
        assert dz <= TOL["bf16_split"]
