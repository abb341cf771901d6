"""Shared helpers of the GPU parity tests (drive the C ABI, compare with the oracle)."""
import math

import numpy as np

F0 = 2048
TOL = {"fp32": 1e-3, "fp16_split": 5e-3, "bf16_split": 5e-3}


def stream_snr(ctx, bank_id, strain, block, det=0):
    """Push ``strain`` in blocks through detector ``det`` and return the SNR
    rows [2M, T] read back after every push with lloid_snr_block."""
    T = strain.size
    M = ctx.banks[bank_id]
    z = np.empty((2 * M, T), dtype=np.float32)
    t = 0
    while t < T:
        n = min(block, T - t)
        ctx.push(det, t, np.ascontiguousarray(strain[t:t + n], dtype=np.float32))
        zb, t0 = ctx.snr_block(det, bank_id)
        assert t0 == t
        z[:, t:t + n] = zb.cpu().numpy()
        t += n
    return z


def max_abs_complex(za, zb):
    """max |za_i - zb_i| over templates and samples (complex difference)."""
    d = (za[0::2] - zb[0::2]) ** 2 + (za[1::2] - zb[1::2]) ** 2
    return float(np.sqrt(d.max()))


def compare_triggers(gpu, oracle_trigs, z_oracle, tol, window, threshold=4.0, t_offset=0, overlap=0):
    """Check GPU triggers against the oracle's.

    Unique parts are compared exactly: the set of (window, template) pairs
    whose oracle window maximum is clear of the threshold by more than tol, and
    their sample whenever the oracle's runner-up in that window is more than
    tol below its maximum.  Elsewhere the GPU's choice must be a valid one: its
    sample's oracle |z| is within tol of the oracle maximum."""
    re, im = z_oracle[0::2], z_oracle[1::2]
    p = np.sqrt(re * re + im * im)
    o = {(t.window, t.tmpl): t for t in oracle_trigs}
    g = {(int(r["window"]), int(r["tmpl"])): r for r in gpu}
    problems = []
    for key in set(o) | set(g):
        w, i = key
        a = max(0, w * window - overlap) - t_offset
        b = (w + 1) * window - t_offset
        seg = p[i, a:b]
        best = float(seg.max())
        if key in o and key not in g:
            if best > threshold + tol:
                problems.append(("missing", key, best))
            continue
        if key in g and key not in o:
            if best < threshold - tol:
                problems.append(("extra", key, best))
            continue
        gk = int(g[key]["sample"]) - t_offset
        if gk != o[key].sample - t_offset:
            if p[i, gk] < best - tol:
                problems.append(("sample", key, gk, o[key].sample, float(p[i, gk]), best))
        if abs(float(g[key]["snr"]) - o[key].snr) > tol:
            problems.append(("snr", key, float(g[key]["snr"]), o[key].snr))
    return problems


def oracle_bank_z(oracle, bank, plan, strain):
    sl = oracle.svd_bank(bank, plan)
    return oracle.lloid_snr(strain.astype(np.float64), sl, F0), sl
