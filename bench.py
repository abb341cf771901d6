#!/usr/bin/env python
"""Throughput of the LLOID hot path on B300: template-seconds filtered per second.

Workload (default: the 500-bank configuration): 500 SVD banks of U{100..1000}
Newtonian chirp templates (about 280k templates, chirp mass log-uniform in
[1, 50] Msun, durations 2-128 s, each bank cut into time slices at 128-2048 Hz
and SVD-compressed to 99.99 % of each slice's energy), 3 detectors x 1024 s of
seeded unit white noise at 2048 Hz (synthetic stand-in for the paper's
mock-data-challenge strain), BF16 split precision.  ``--workload bank1000`` and
``--workload banks20`` select the 1000-template bank and the 20-bank precision
configuration.

A step pushes one block (--block-seconds, default 8 s) of strain for every
detector through every stage (ingest, downsample, basis FIR, upsample,
reconstruction + window maxima, finalisation) and pulls the triggers of the
windows the block completes.  The stream continues across steps, cycling
through the record.  L2 is flushed (256 MB write) between steps, outside the
timed intervals, which are CUDA-event pairs on the library's stream around
each step.

Output: one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead (bounded samples of the same workload).  The ``cpu_baseline``
leg times the oracle on a bounded sample of the workload and keeps its SNR,
against which the GPU path's error distribution per precision is reported.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

F0 = 2048
METRIC = "template-seconds filtered/s at max |dSNR|<=5e-3 vs FP32 path; p50/p99 block latency"
UNIT = "template-s/s"
# bounded oracle samples of each workload: banks (indices into the workload's banks), the
# first templates of each, seconds of one detector's strain from the stream start
ORACLE_SAMPLE = {"banks500": ((25, 125, 225, 325, 425), 48, 20),
                 "banks20": ((2, 9, 16), 48, 20),
                 "bank1000": ((0,), 64, 68)}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", default="lloid", choices=["lloid", "reference"])
    p.add_argument("--precision", default="bf16_split", choices=["fp32", "fp16_split", "bf16_split"])
    p.add_argument("--block-seconds", type=int, default=8)
    p.add_argument("--templates", type=int, default=1000)
    p.add_argument("--seconds", type=int, default=1024)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--whiten-seconds", type=int, default=256,
                   help="seconds of 16384 Hz strain per detector for the whitening measurement (0: skip it)")
    p.add_argument("--xi2-half", type=int, default=None,
                   help="Eq. 10 autocorrelation half-length d for the xi2 measurement (0: skip it; "
                        "default 350 for the one-bank workload, 0 otherwise)")
    p.add_argument("--no-fp32-compare", action="store_true")
    p.add_argument("--latency-steps", type=int, default=32)
    p.add_argument("--workload", default="banks500", choices=["bank1000", "banks20", "banks500"])
    p.add_argument("--banks", type=int, default=None, help="use the first N banks of a multi-bank workload")
    p.add_argument("--detectors", type=int, default=None)
    p.add_argument("--serve", action="store_true", help="paced serving loop with latency percentiles")
    p.add_argument("--serve-block", type=int, default=2048)
    p.add_argument("--pace", type=float, default=1.0)
    p.add_argument("--serve-seconds", type=int, default=60)
    p.add_argument("--serve-blocks", type=int, default=None, help="blocks to stream (overrides --serve-seconds)")
    p.add_argument("--no-serve-summary", action="store_true",
                   help="skip the short 10x-pace serving run of the default bench line")
    p.add_argument("--form", default=None, choices=["ladder", "f0"],
                   help="force every bank into one form of the split path (default: per-bank choice)")
    p.add_argument("--no-autotune", action="store_true",
                   help="skip the autotuner (default: tune the form ratio and FIR occupancy on a bank sample)")
    p.add_argument("--autotune-banks", type=int, default=100, help="banks of the sample the autotuner times")
    return p.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (weak scaling: every rank filters its own replica)
# ---------------------------------------------------------------------------
def dist_init(args):
    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "lloid" else "gloo"
        dist.init_process_group(backend=backend)
        return dist.get_rank(), dist.get_world_size(), dist
    return 0, 1, None


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
_NVML_SAMPLER = r"""
import ctypes, sys, time
out = open(sys.argv[2], "w", buffering=1)
try:
    nv = ctypes.CDLL("libnvidia-ml.so.1")
    if nv.nvmlInit_v2() != 0:
        raise RuntimeError("nvmlInit failed")
    want = sys.argv[3].replace("-", "").lower()
    n = ctypes.c_uint(0)
    nv.nvmlDeviceGetCount_v2(ctypes.byref(n))
    h = None
    for i in range(n.value):                       # the device whose UUID matches, else the index
        c = ctypes.c_void_p()
        nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(i), ctypes.byref(c))
        buf = ctypes.create_string_buffer(96)
        nv.nvmlDeviceGetUUID(c, buf, ctypes.c_uint(96))
        if want and want in buf.value.decode().replace("-", "").lower():
            h = c
    if h is None:
        h = ctypes.c_void_p()
        nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(int(sys.argv[1])), ctypes.byref(h))
    reasons_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
        nv.nvmlDeviceGetCurrentClocksThrottleReasons
    sm, mx, r = ctypes.c_uint(0), ctypes.c_uint(0), ctypes.c_ulonglong(0)
    nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))          # 1 = SM clock domain
    while True:
        nv.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(sm))
        reasons_fn(h, ctypes.byref(r))
        out.write(f"{time.time():.6f} {sm.value} {mx.value} {r.value}\n")
        time.sleep(0.002)
except Exception as e:
    out.write("# " + repr(e).replace("\n", " ") + "\n")
"""


class ClockSampler:
    """SM clock and clock-event reasons sampled every ~2 ms by a separate
    process (NVML), started before the timed region and trimmed to it."""
    REASONS = {"hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40,
               "sw_power_cap": 0x4}

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None
        self.error = None
        try:
            import torch
            self.uuid = str(torch.cuda.get_device_properties(device).uuid)
        except Exception:
            self.uuid = ""

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".txt")
            os.close(fd)
            self.proc = subprocess.Popen([sys.executable, "-c", _NVML_SAMPLER, str(self.device), self.path,
                                          self.uuid],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            deadline = time.time() + 20
            while time.time() < deadline and self.proc.poll() is None and os.path.getsize(self.path) == 0:
                time.sleep(0.01)
        except Exception as e:
            self.error = repr(e)
            self.proc = None

    def begin(self):
        self.t0 = time.time()

    def end(self):
        self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return {"error": self.error or "sampler not started"}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            if line.startswith("#"):
                self.error = line[1:].strip()
            f = line.split()
            if len(f) == 4 and not line.startswith("#"):
                rows.append((float(f[0]), float(f[1]), float(f[2]), int(f[3])))
        os.unlink(self.path)
        if not rows:
            return {"error": self.error or "no samples"}
        t0, t1 = self.t0 or rows[0][0], self.t1 or rows[-1][0]
        inside = [r for r in rows if t0 <= r[0] <= t1]
        if len(inside) < 3:      # a region shorter than a few samples: the samples nearest to it
            inside = sorted(rows, key=lambda r: abs(r[0] - 0.5 * (t0 + t1)))[:3]
        reasons = sorted(n for n, bit in self.REASONS.items() if any(r[3] & bit for r in inside))
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "samples": len(inside), "region_ms": round(1000 * (t1 - t0), 2), "source": "nvml",
                "reasons": reasons}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
WORKLOADS = {
    "bank1000": ("1000 Newtonian chirp templates (Mc log-U[1,20] Msun, 64 s, 9 slices 2048/1024/512/256/128 Hz, "
                 "SVD 99.99%), 2 detectors x 1024 s white noise + 20 injections/detector, 1 s trigger windows"),
    "banks20": ("10,000 Newtonian chirp templates (Mc log-U[1,20] Msun) in 20 contiguous-Mc SVD banks of 200-800, "
                "durations 8-64 s, 2 detectors x 4096 s white noise + 100 injections"),
    "banks500": ("500 SVD banks of U{100..1000} templates (~280k, Mc log-U[1,50] Msun, durations 2-128 s, 1-10 slices, "
                 "128-2048 Hz, SVD 99.99%), 3 detectors x 1024 s white noise + 17 injections/detector, "
                 "1 s trigger windows"),
}


def _svd_job(args):
    from paper_2511_04730_b300 import build_svd_bank
    bank, plan = args
    return build_svd_bank(bank, plan)


def make_inputs(args, rank):
    import numpy as np
    import workloads as W
    workers = max(1, min(16, os.cpu_count() or 1))
    if args.workload == "bank1000":
        w = W.make_workload("bank1000", n_templates=args.templates, n_seconds=args.seconds, n_det=args.detectors)
    else:
        secs = args.seconds if args.seconds != 1024 or args.workload == "banks500" else None
        w = W.make_workload(args.workload, n_seconds=secs, n_banks=args.banks, n_det=args.detectors,
                            workers=workers)
    w.seed_base = 100 + 10 * rank
    strain = np.stack([w.strain(d) for d in range(w.n_det)]).astype(np.float32)
    return w, strain


def build_banks(w):
    """SVD banks of every bank of the workload (a spawn pool for many banks)."""
    from paper_2511_04730_b300 import build_svd_bank
    if len(w.banks) < 4:
        return [build_svd_bank(b, p) for b, p in zip(w.banks, w.plans)]
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS")}
    os.environ.update(OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1")
    try:
        with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
            return pool.map(_svd_job, list(zip(w.banks, w.plans)), chunksize=1)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


def algorithmic_work(slices, M, f0=F0, n_up=8):
    """Per detector-second per bank (the hot-path accounting of Eq. 5-8):
    FIR 2 L N r, reconstruction 2 (2M) L r, ladder 2 (2M) 2 N_up r (F-1)/F
    for each stage into rate r, window maxima 2M f0 compares."""
    fir = sum(2.0 * s.n_basis * s.n_taps * s.rate for s in slices)
    rec_by = {}
    for s in slices:
        rec_by[s.rate] = rec_by.get(s.rate, 0.0) + 2.0 * (2 * M) * s.n_basis * s.rate
    lad = sorted(set(s.rate for s in slices) | {f0})
    up_by = {hi: 2.0 * (2 * M) * 2 * n_up * hi * (hi // lo - 1) / (hi // lo) for lo, hi in zip(lad[:-1], lad[1:])}
    cmp_ = 2.0 * M * f0
    return {"fir": fir, "recon": sum(rec_by.values()), "ladder": sum(up_by.values()), "max": cmp_,
            "below_f0": sum(v for r, v in rec_by.items() if r < f0) + sum(v for r, v in up_by.items() if r < f0),
            "at_f0": rec_by.get(f0, 0.0) + up_by.get(f0, 0.0) + cmp_}


def yhat_flops(slices, f0=F0, n_up=8):
    """Multiply-adds (x2) per detector-second that k_yhat executes for a bank in the f0 form:
    every basis of a slice below f0 through its composed upsampler (the Eq. 7-8 stages of the
    bank's ladder from the slice's rate up, c = F N_up each), ceil(length / D) taps per output
    sample, columns in chunks of 4; slices at f0 are copied."""
    lad = sorted(set(s.rate for s in slices) | {f0})
    total = 0.0
    for s in slices:
        if s.rate == f0:
            continue
        length = 1
        chain = [r for r in lad if r >= s.rate]
        for lo, hi in zip(chain[:-1], chain[1:]):
            F = hi // lo
            length = F * (length - 1) + 2 * F * n_up + 1
        D = f0 // s.rate
        total += 2.0 * (-(-s.n_basis // 4) * 4) * f0 * (-(-length // D))
    return total


# DRAM read + write bytes per launch of each stage's kernel, from the ncu captures
# summarised in profiles/; valid only while the kernel sources hash to the prefix they
# were taken with.
TRAFFIC_SOURCES = ("kernels_f0.cuh", "kernels_tc.cuh", "kernels_tc2.cuh", "lloid_common.cuh")
TRAFFIC_SHA = "3039a125aadd606d"
TRAFFIC_PROFILE = ("profiles/dram_banks500_bf16split.md (one pass, all f0-possible banks in the f0 form); per launch of "
                   "the stage's main kernel: k_f0_top for recon, k_yhat for upsample, k_fir_tc for fir (the few ladder "
                   "levels in the same stages are not included)")
TRAFFIC_KERNEL = {"recon": "k_f0_top", "upsample": "k_yhat", "fir": "k_fir_tc"}
TRAFFIC = {("banks500", "bf16_split", 8, 3): {"recon": 3.379e9 + 0.201e9, "upsample": 8.333e9 + 3.261e9,
                                               "fir": 1.020e9 + 2.412e9}}


def kernel_sources_sha():
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2511_04730_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload, precision, block_seconds, n_det, stage, subset=False):
    """The recorded bytes per launch of the stage's main kernel, or None: for the whole
    workload only (subset: a --banks sample of it) and while the kernel sources are the
    ones the figures were taken from."""
    if subset or not TRAFFIC_SHA or kernel_sources_sha() != TRAFFIC_SHA:
        return None
    return TRAFFIC.get((workload, precision, block_seconds, n_det), {}).get(stage)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0}, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle leg (cpu_baseline, the error distribution against it, and --impl reference)
# ---------------------------------------------------------------------------
def oracle_sample_workload(workload):
    """The bounded sample of a workload the oracle runs on: a few of its banks,
    one detector, the first seconds of the stream (no injections)."""
    import workloads as W
    banks, M_sub, secs = ORACLE_SAMPLE[workload]
    if workload == "bank1000":
        w = W.make_workload("bank1000", n_templates=M_sub, n_seconds=secs, n_det=1, n_inj=0)
    else:
        w = W.make_workload(workload, bank_indices=banks, n_seconds=secs, n_det=1, n_inj=0)
    return w, M_sub, secs


def oracle_run(w, k, M_sub, d):
    """The FP64 oracle's LLOID SNR and triggers of bank k's first M_sub templates
    on strain d (its coefficient rows only: the oracle is linear in them).
    Returns (z [2 M_sub, T], triggers, seconds, cpu seconds)."""
    import numpy as np
    from oracle import lloid_oracle as O
    sl = O.svd_bank(w.banks[k], w.plans[k])
    sub = [O.OracleSlice(s.rate, s.j_start, s.bases, s.coeffs[: 2 * M_sub]) for s in sl]
    t, c = time.perf_counter(), time.process_time()
    z = O.lloid_snr(d.astype(np.float64), sub, F0)
    trig = O.triggers(z, F0)
    return z, trig, time.perf_counter() - t, time.process_time() - c


def oracle_leg(workload):
    """cpu_baseline: the oracle as it stands, timed on this host's cores over the
    bounded sample; its SNR and triggers are kept for the precision report."""
    w, M_sub, secs = oracle_sample_workload(workload)
    d = w.strain(0)
    out, wall, cpu = [], 0.0, 0.0
    for k in range(len(w.banks)):
        z, trig, dt, dc = oracle_run(w, k, M_sub, d)
        out.append((k, z, trig))
        wall += dt
        cpu += dc
    units = M_sub * secs * len(w.banks)
    banks = ORACLE_SAMPLE[workload][0]
    desc = (f"{len(w.banks)} banks ({', '.join(map(str, banks))}) of the workload, the first {M_sub} templates of "
            f"each, 1 detector x {secs} s (oracle FP64 numpy LLOID + triggers)")
    cpu_line = {"value": units / wall, "unit": UNIT, "cores": max(1.0, round(cpu / wall, 1)), "kind": "oracle",
                "sample": desc, "seconds": round(wall, 2)}
    return cpu_line, (w, M_sub, d, out)


def run_reference(args, rank, world, dist):
    """The base contract's reference arm: the oracle, timed on host cores; each step
    is one bank of the bounded sample (the banks in turn)."""
    if rank != 0:
        return
    w, M_sub, secs = oracle_sample_workload(args.workload)
    d = w.strain(0)
    nb = len(w.banks)
    for i in range(args.warmup):
        oracle_run(w, i % nb, M_sub, d)
    vals, cpus = [], []
    t0 = time.perf_counter()
    for i in range(args.steps):
        _, _, dt, dc = oracle_run(w, i % nb, M_sub, d)
        vals.append(dt)
        cpus.append(dc)
    wall = time.perf_counter() - t0
    value = M_sub * secs * args.steps / sum(vals)
    sample = (f"each step: the first {M_sub} templates of one of {nb} banks of the workload (in turn) x "
              f"1 detector x {secs} s (oracle FP64 numpy LLOID + triggers)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload], "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": max(1.0, round(sum(cpus) / sum(vals), 1)),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def precision_report(P, sample, forms=("ladder", "f0"), dev=0):
    """The GPU path's SNR on the oracle's sample, per precision (and per form of the
    split paths), against the oracle's FP64 SNR: quantiles of |dz| over every
    (template, sample) and the agreement of the triggers (same window, template and
    sample as the oracle's; otherwise the GPU's sample within the tolerance of the
    oracle's window maximum)."""
    import numpy as np
    from paper_2511_04730_b300 import build_svd_bank
    w, M_sub, d, out = sample
    T = d.size
    sb = [build_svd_bank(b, p) for b, p in zip(w.banks, w.plans)]
    rep = {}
    tol = {"fp32": 1e-3, "fp16_split": 5e-3, "bf16_split": 5e-3}
    cases = [("fp32", None)] + [(p, f) for p in ("fp16_split", "bf16_split") for f in forms]
    for prec, form in cases:
        dz_all, n_trig, n_same, n_valid, n_wrong, n_missing, n_extra = [], 0, 0, 0, 0, 0, 0
        with P.Context(n_detectors=1, precision=prec, max_block=8192, max_history=max(b.n_samples for b in w.banks),
                       device=dev, form=form) as ctx:
            ids = [ctx.load_bank(x) for x in sb]
            zs = {i: [] for i in ids}
            trig = []
            for t in range(0, T - T % 8192, 8192):
                ctx.push(0, t, np.ascontiguousarray(d[t:t + 8192], dtype=np.float32))
                for i in ids:
                    zs[i].append(ctx.snr_block(0, i)[0][: 2 * M_sub].cpu().numpy())
                trig.append(ctx.pull(t // F0, n_windows=8192 // F0))
            trig = np.concatenate(trig)
        for (k, zo, otr), i in zip(out, ids):
            z = np.concatenate(zs[i], axis=1)
            n = z.shape[1]
            dz = np.sqrt((z[0::2] - zo[0::2, :n]) ** 2 + (z[1::2] - zo[1::2, :n]) ** 2)
            dz_all.append(dz.ravel())
            p = np.sqrt(zo[0::2, :n] ** 2 + zo[1::2, :n] ** 2)
            g = {(int(r["window"]), int(r["tmpl"])): r for r in trig[(trig["bank"] == i) & (trig["tmpl"] < M_sub)]}
            for o in otr:
                if (o.window + 1) * F0 > n:
                    continue
                n_trig += 1
                r = g.pop((o.window, o.tmpl), None)
                if r is None:
                    n_missing += o.snr > 4.0 + tol[prec]          # else: within the tolerance of the threshold
                    continue
                if int(r["sample"]) == o.sample:
                    n_same += 1
                elif p[o.tmpl, int(r["sample"])] >= o.snr - tol[prec]:
                    n_valid += 1
                else:
                    n_wrong += 1
            for (win, tm), r in g.items():
                if (win + 1) * F0 <= n:
                    n_extra += p[tm, win * F0:(win + 1) * F0].max() < 4.0 - tol[prec]
        a = np.concatenate(dz_all)
        key = prec if form is None else f"{prec}/{form}"
        rep[key] = {"max": float(a.max()), "p99": float(np.quantile(a, 0.99)), "p50": float(np.median(a)),
                    "n": int(a.size), "triggers": n_trig, "same_sample": n_same, "other_valid_sample": n_valid,
                    "wrong_sample": n_wrong, "missing": int(n_missing), "extra": int(n_extra)}
    return {"vs": "FP64 oracle on the cpu_baseline sample", "tolerance": tol, "dz": rep}


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def run_lloid(args, rank, world, dist):
    import numpy as np
    import torch
    import paper_2511_04730_b300 as P
    from paper_2511_04730_b300 import build

    build.build()
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    if args.xi2_half is None:
        args.xi2_half = 350 if args.workload == "bank1000" else 0
    w, strain = make_inputs(args, rank)
    all_banks = build_banks(w)
    if len(all_banks) > 1 and world > 1:            # shard the bank set: LPT on per-bank work
        from paper_2511_04730_b300 import sharding
        costs = [sharding.bank_cost(sb_, b.n_templates) for sb_, b in zip(all_banks, w.banks)]
        mine = sharding.assign_banks(costs, world)[rank]
    else:
        mine = list(range(len(all_banks)))
    banks_sb = [all_banks[i] for i in mine]
    M_list = [w.banks[i].n_templates for i in mine]
    M = sum(M_list)
    n_det = w.n_det
    max_hist = max(b.n_samples for b in w.banks)
    B = args.block_seconds * F0
    T = strain.shape[1]
    assert T % B == 0
    n_blk = T // B
    # blocks laid out [block][detector][sample] so that every step's input is contiguous
    blocks = np.ascontiguousarray(strain.reshape(n_det, n_blk, B).transpose(1, 0, 2))
    d_blocks = torch.from_numpy(blocks).to(f"cuda:{dev}")
    h_blocks = torch.from_numpy(blocks).pin_memory()

    # the autotuner: candidate forms and FIR occupancies timed on a sample of the banks
    tuning, tune_info = None, None
    if args.precision != "fp32" and not args.no_autotune and args.form is None:
        stride = max(1, len(banks_sb) // max(1, args.autotune_banks))
        sample = banks_sb[::stride]
        t_tune = time.perf_counter()
        tuning = P.autotune(sample, B, reps=3, n_detectors=n_det, precision=args.precision,
                            max_history=max_hist, device=dev)
        c_def = next(c for c in tuning["candidates"] if c["form"] == "by ratio" and c["form_ratio"] == 1.0)
        tune_info = {"sample_banks": len(sample), "seconds": round(time.perf_counter() - t_tune, 1),
                     "chosen": tuning["candidates"][tuning["best"]], "candidates": tuning["candidates"],
                     "gain_over_default": c_def["ms_per_push"] / tuning["candidates"][tuning["best"]]["ms_per_push"]}

    def make_ctx(precision, timing, form=args.form, max_block=B):
        return P.Context(n_detectors=n_det, precision=precision, max_block=max_block, max_history=max_hist,
                         device=dev, stage_timing=timing, form=form,
                         tuning=tuning if precision == args.precision else None)

    def load_all(ctx, which=None):
        return [ctx.load_bank(banks_sb[i]) for i in (range(len(banks_sb)) if which is None else which)]

    def serve_measure(block, pace, n_serve):
        """The streaming loop (serving.Server) over the bank set: every bank is submitted,
        admitted under the HBM budget, the FIR history filled at full speed, then n_serve
        blocks of `block` samples from every detector arrive at `pace` times real time.
        Latency: block arrival -> the triggers of the windows it completes on the host."""
        from paper_2511_04730_b300.serving import Server
        ctx = P.Context(n_detectors=n_det, precision=args.precision, max_block=block, max_history=max_hist,
                        device=dev, form=args.form)
        srv = Server(ctx, block)
        for i, x in enumerate(banks_sb):
            srv.submit(x, tag=i)
        nb = T // block
        blocks_s = np.ascontiguousarray(strain.reshape(n_det, nb, block).transpose(1, 0, 2))
        src = lambda k: blocks_s[k % nb]
        warm = max_hist // block + 4
        for k in range(warm):                          # admit every bank and fill the history
            srv.step(src(k))
        srv.latency_ms.clear()
        t0 = time.perf_counter()
        srv.run_paced(lambda k: src(warm + k), n_serve, pace=pace)
        wall = time.perf_counter() - t0
        ctx.close()
        return {"block_seconds": block / F0, "pace": pace, "blocks": n_serve, "latency_ms": srv.latency_summary(),
                "seconds_streamed": n_serve * block / F0, "wall_s": round(wall, 2),
                "template_s_per_s": M * n_det * n_serve * block / F0 / wall,
                "data": f"the workload's {T // F0} s of strain per detector, cycled"}

    if args.serve:
        res = serve_measure(args.serve_block, args.pace, args.serve_blocks or args.serve_seconds * F0 // args.serve_block)
        if rank == 0:
            print(json.dumps({
                "mode": "serve", "metric": "per-block latency (block arrival -> its windows' triggers on the host)",
                **res, "n_templates": M, "n_banks": len(banks_sb), "n_detectors": n_det, "precision": args.precision,
                "workload": WORKLOADS[args.workload]}), flush=True)
        return

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")

    def run_steps(ctx, k_steps, pos, host=False, lat=None, lag=0, pipelined=False):
        """k_steps timed steps; returns (ms per step list, pos, launches, h2d, d2h).
        lag = 1: pull the windows that became ready (xi2 needs d samples of the
        next block), i.e. the previous block's last window and this block's others.
        pipelined: each step's pull is submitted behind its push and collected two
        pushes later (the host reads a block's triggers while the GPU filters the next
        two, so a host stall shorter than a step does not idle the GPU); the K steps
        are timed as one region and every pull is collected in it."""
        ext = torch.cuda.ExternalStream(ctx.stream_ptr, device=f"cuda:{dev}")
        ms, h2d, d2h = [], 0, 0
        l0 = ctx.launch_count()
        with torch.cuda.stream(ext):
            if pipelined:
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                tickets = []
                a.record(ext)
                for _ in range(k_steps):
                    flush.fill_(pos & 0xFF)                   # L2 flush, inside the region
                    k = (pos // B) % n_blk
                    if host:
                        blk = h_blocks[k].numpy()
                        ctx.push_all(pos, blk)
                        h2d += blk.nbytes
                    else:
                        ctx.push_all(pos, d_blocks[k])
                    w_lo = max(0, pos // F0 - lag)
                    tickets.append(ctx.pull_submit(w_lo, n_windows=(pos + B) // F0 - lag - w_lo))
                    if len(tickets) > 2:
                        d2h += 8 + ctx.pull_collect(tickets.pop(0)).nbytes
                    pos += B
                for t in tickets:
                    d2h += 8 + ctx.pull_collect(t).nbytes
                b.record(ext)
                b.synchronize()
                ms = [a.elapsed_time(b) / k_steps] * k_steps
                return ms, pos, ctx.launch_count() - l0, h2d, d2h
            for _ in range(k_steps):
                flush.fill_(pos & 0xFF)                       # L2 flush, outside the events
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                k = (pos // B) % n_blk
                a.record(ext)
                t_host = time.perf_counter()
                if host:
                    blk = h_blocks[k].numpy()                 # pinned host memory
                    ctx.push_all(pos, blk)
                    h2d += blk.nbytes
                else:
                    ctx.push_all(pos, d_blocks[k])
                w_lo = max(0, pos // F0 - lag)
                tr = ctx.pull(w_lo, n_windows=(pos + B) // F0 - lag - w_lo)   # the windows this block completes
                d2h += 8 + tr.nbytes
                b.record(ext)
                b.synchronize()
                if lat is not None:
                    lat.append(1000 * (time.perf_counter() - t_host))
                ms.append(a.elapsed_time(b))
                pos += B
        return ms, pos, ctx.launch_count() - l0, h2d, d2h

    # ---- throughput: K steps without per-stage events, clocks sampled during them
    ctx = make_ctx(args.precision, timing=False)
    ids = load_all(ctx)
    forms = {}
    form_of = []
    for i in ids:
        f = ctx.bank_form(i)
        form_of.append(f)
        forms[f] = forms.get(f, 0) + 1
    pos = 0
    _, pos, _, _, _ = run_steps(ctx, args.warmup, pos, pipelined=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(dev)
    sampler.start()
    sampler.begin()
    ms, pos, launches, _, _ = run_steps(ctx, args.steps, pos, pipelined=True)
    torch.cuda.synchronize()
    sampler.end()
    clocks = sampler.stop()
    ctx.close()

    # ---- stage breakdown and roofline: the same K steps again, with CUDA events around every stage
    ctx = make_ctx(args.precision, timing=True)
    load_all(ctx)
    pos = 0
    _, pos, _, _, _ = run_steps(ctx, args.warmup, pos)
    ctx.stage_times(reset=True)
    torch.cuda.synchronize()
    ms_t, pos, _, _, _ = run_steps(ctx, args.steps, pos)
    torch.cuda.synchronize()
    stages = ctx.stage_times(reset=True)
    ctx.close()

    # ---- end to end: host blocks in, triggers out, through the public API
    e2e = None
    if not args.no_e2e:
        ctx = make_ctx(args.precision, False)
        load_all(ctx)
        pos = 0
        _, pos, _, _, _ = run_steps(ctx, args.warmup, pos, host=True, pipelined=True)
        ms_e, pos, _, h2d, d2h = run_steps(ctx, args.steps, pos, host=True, pipelined=True)
        ctx.close()
        e2e = {"value": M * args.block_seconds * n_det * args.steps / (sum(ms_e) / 1000.0), "unit": UNIT,
               "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps,
               "ms_per_step": statistics.mean(ms_e)}

    # ---- the plain FP32 path (reference precision) on the same blocks, a few steps
    paths = {args.precision: M * args.block_seconds * n_det * args.steps / (sum(ms) / 1000.0)}
    if args.precision != "fp32" and not args.no_fp32_compare:
        k32 = min(args.steps, 3)
        ctx = make_ctx("fp32", timing=False)
        load_all(ctx)
        pos = 0
        _, pos, _, _, _ = run_steps(ctx, 1, pos, pipelined=True)
        ms32, pos, _, _, _ = run_steps(ctx, k32, pos, pipelined=True)
        ctx.close()
        paths["fp32"] = M * args.block_seconds * n_det * k32 / (sum(ms32) / 1000.0)
        paths["fp32_steps"] = k32

    # ---- accuracy against the FP32 path on a sample of banks (every SNR sample of every
    # template of those banks, over the last pushes after a full template history)
    max_dsnr = None
    if args.precision != "fp32" and not args.no_fp32_compare:
        stride = max(1, len(banks_sb) // 24)
        chk = list(range(0, len(banks_sb), stride))
        a, b = make_ctx(args.precision, False), make_ctx("fp32", False)
        ia, ib = load_all(a, chk), load_all(b, chk)
        hist = max(w.banks[mine[i]].n_samples for i in chk)
        max_dsnr = 0.0
        n_push = (hist + 2 * B - 1) // B + 2
        for k in range(n_push):
            blk = d_blocks[k % n_blk]
            a.push_all(k * B, blk)
            b.push_all(k * B, blk)
            if k >= n_push - 2:
                for det in range(n_det):
                    for x, y, j in zip(ia, ib, chk):
                        za, _ = a.snr_block(det, x)
                        zb, _ = b.snr_block(det, y)
                        dz = torch.sqrt(((za - zb) ** 2).view(M_list[j], 2, -1).sum(1)).max().item()
                        max_dsnr = max(max_dsnr, dz)
        a.close()
        b.close()
        max_dsnr = {"value": max_dsnr, "banks": len(chk), "templates": sum(M_list[j] for j in chk),
                    "samples_per_template": 2 * B, "detectors": n_det}

    # ---- per-block latency at 1 s blocks (block arrival on the host -> its window's triggers on the host)
    lat = []
    if args.latency_steps:
        ctx = make_ctx(args.precision, False, max_block=F0)
        load_all(ctx)
        pos = 0
        h_sec = torch.from_numpy(np.ascontiguousarray(
            strain.reshape(n_det, T // F0, F0).transpose(1, 0, 2))).pin_memory()
        warm = 8
        for k in range(warm + args.latency_steps):
            blk = h_sec[(pos // F0) % (T // F0)].numpy()
            t0 = time.perf_counter()
            ctx.push_all(pos, blk)
            ctx.pull(pos // F0)
            if k >= warm:
                lat.append(1000 * (time.perf_counter() - t0))
            pos += F0
        ctx.close()

    # ---- Eq. 10 (a NEXT row): the same steps with autocorrelations loaded for every bank
    xi2 = None
    if args.xi2_half > 0:
        from paper_2511_04730_b300.svdbank import template_autocorrelation
        t_ac = time.perf_counter()
        acs = [template_autocorrelation(w.banks[i], args.xi2_half) for i in mine]
        t_ac = time.perf_counter() - t_ac
        ctx = make_ctx(args.precision, timing=True)
        for x, ac in zip(banks_sb, acs):
            ctx.load_bank(x, autocorr=ac)
        pos = 0
        _, pos, _, _, _ = run_steps(ctx, args.warmup, pos, lag=1, pipelined=True)
        ctx.stage_times(reset=True)
        torch.cuda.synchronize()
        ms_x, pos, _, _, d2h_x = run_steps(ctx, args.steps, pos, lag=1, pipelined=True)
        st_x = ctx.stage_times(reset=True)
        ctx.close()
        units_x = M * args.block_seconds * n_det
        xi2 = {"value": units_x * args.steps / (sum(ms_x) / 1000.0), "unit": UNIT,
               "ms_per_step": statistics.mean(ms_x), "autocorr_samples": 2 * args.xi2_half + 1,
               "finalize_plus_xi2_ms_per_step": round(st_x["finalize"][0] / args.steps, 4),
               "recon_ms_per_step": round(st_x["recon"][0] / args.steps, 4),
               "d2h_bytes_per_step": d2h_x // args.steps, "autocorr_build_s": round(t_ac, 1)}

    # ---- PSD estimation and whitening (a NEXT row): 16384 Hz -> 2048 Hz, N = 4 s, Z = 1 s, 16 s pushes
    whiten = None
    if args.whiten_seconds > 0 and rank == 0:
        fi, push = 16384, 16 * 16384
        wx = np.random.default_rng(9).standard_normal((n_det, args.whiten_seconds * fi)).astype(np.float32)
        dwx = torch.from_numpy(wx).to(f"cuda:{dev}")
        wout = torch.empty(push // 8 + 1, dtype=torch.float32, device=f"cuda:{dev}")
        torch.cuda.synchronize()                 # the whitener works on its own stream
        with P.Whitener(fi, F0, n_detectors=n_det, max_push=push) as wg:
            lib = wg._lib
            import ctypes
            n_out = ctypes.c_int64()

            def wpass(lo, hi):
                for i in range(lo, hi, push):
                    for det in range(n_det):
                        st = lib.lloid_whiten(wg._h, det, ctypes.c_void_p(dwx[det, i:i + push].data_ptr()), push, 1,
                                              ctypes.c_void_p(wout.data_ptr()), wout.numel(), ctypes.byref(n_out), 1)
                        assert st == 0, st
            half = (args.whiten_seconds // 2) * fi // push * push
            wpass(0, half)                       # warm-up: plans, PSD settles
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            wpass(half, wx.shape[1] // push * push)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            secs = (wx.shape[1] // push * push - half) / fi * n_det
        whiten = {"value": secs / dt, "unit": "detector-seconds whitened/s", "input_rate": fi, "output_rate": F0,
                  "n_fft_s": 4, "z_s": 1, "push_s": 16, "seconds": secs}

    # ---- the oracle leg (rank 0): cpu_baseline, and the error distribution of every precision against it
    cpu, precision = None, None
    if rank == 0 and not args.no_cpu_baseline:
        cpu, sample = oracle_leg(args.workload)
        precision = precision_report(P, sample, dev=dev)

    units = M * args.block_seconds * n_det
    my_time = sum(ms) / 1000.0
    if dist is not None:
        t = torch.tensor([my_time], device=f"cuda:{dev}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        my_time = float(t.item())
    if len(all_banks) == 1:                        # replicas: every rank filters its own copy
        value = units * args.steps * world / my_time
    else:                                          # shards of one bank set
        value = w.n_templates * args.block_seconds * n_det * args.steps / my_time

    # ---- per-stage algorithmic work by form, roofline of the dominant stage
    works = [algorithmic_work(x, m) for x, m in zip(banks_sb, M_list)]
    det_s = args.block_seconds * n_det
    tc = args.precision != "fp32"
    wk = {"fir": 0.0, "upsample": 0.0, "recon": 0.0, "f0_executed": 0.0, "yhat_executed": 0.0}
    products = 3 if args.precision == "bf16_split" else 2
    for wo, f, x, m in zip(works, form_of, banks_sb, M_list):
        wk["fir"] += wo["fir"]
        if not tc:
            wk["upsample"] += wo["ladder"]
            wk["recon"] += wo["recon"] + wo["max"]
        elif f == "f0":            # Eq. 6-8 of the bank, all in the f0 kernel
            wk["recon"] += wo["recon"] + wo["ladder"] + wo["max"]
            k_all = sum(s.n_basis for s in x)
            # tensor work the f0 kernel executes: re and im of C Yhat at f0 over the padded bases and
            # template tiles, one MMA per hi/lo product
            wk["f0_executed"] += 2 * 2.0 * (-(-m // 128) * 128) * (-(-k_all // 16) * 16) * F0 * products
            wk["yhat_executed"] += yhat_flops(x)
        else:
            wk["upsample"] += wo["below_f0"]
            wk["recon"] += wo["at_f0"]
    pk, pk_kind = peaks()
    alu_peak = 148 * 128 * 2 * pk.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    alu_note = "FP32 FFMA: 148 SMs x 128 lanes x 2 flop x max SM clock"
    tc_peak = pk["bf16_tflops"]
    tc_note = (f"{pk_kind} dense bf16 burst (the kernels run inside a {statistics.mean(ms):.1f} ms step"
               + ("; fp16 nominal rate equal" if args.precision == "fp16_split" else "") + ")")
    yhat_stage = tc and forms.get("f0", 0) > 0
    if tc:
        rec_name = ("k_level_tc (f0 level + window maxima)" if forms.get("f0", 0) == 0 else
                    "k_f0_top (f0 form: upsampling + reconstruction + window maxima)" if forms.get("ladder", 0) == 0
                    else "k_f0_top (f0-form banks) + k_level_tc (f0 level of ladder-form banks)")
        # the upsample stage holds k_yhat (the f0 form's Eq. 7-8, FP32 multiply-adds, counted as
        # executed: the paper's order does this work on 2M rows, the f0 form on the K bases) and
        # the ladder levels below f0 of the ladder-form banks
        up = (("k_yhat (f0 form, executed FP32 work)" + (" + k_level_tc (ladder levels below f0)"
                                                           if forms.get("ladder", 0) else ""),
               "alu", alu_peak, alu_note, wk["yhat_executed"] + wk["upsample"], "TFLOP/s") if yhat_stage else
              ("k_level_tc (levels below f0)", "tensor", tc_peak, tc_note, wk["upsample"], "TFLOP/s"))
        kinds = {"fir": ("k_fir_tc", "tensor", tc_peak, tc_note, wk["fir"], "TFLOP/s"),
                 "upsample": up,
                 "recon": (rec_name, "tensor", tc_peak, tc_note, wk["recon"], "TFLOP/s")}
    else:
        kinds = {"fir": ("k_fir_f32", "alu", alu_peak, alu_note, wk["fir"], "TFLOP/s"),
                 "upsample": ("k_upsample", "alu", alu_peak, alu_note, wk["upsample"], "TFLOP/s"),
                 "recon": ("k_recon_f32", "alu", alu_peak, alu_note, wk["recon"], "TFLOP/s")}
    per_stage = {}
    for st_name in ("fir", "upsample", "recon"):
        tot_ms, n_l = stages[st_name]
        if n_l == 0:
            continue
        kname, bound, peak, note, work, unit = kinds[st_name]
        lps = n_l / args.steps
        launch_ms = tot_ms / n_l
        scale = 1e9 if unit == "GB/s" else 1e12
        achieved = (work * det_s / lps) / (launch_ms / 1000.0) / scale
        per_stage[st_name] = {"kernel": kname, "bound": bound, "launch_ms": launch_ms, "launches_per_step": lps,
                              "achieved": achieved, "unit": unit, "peak": peak, "frac": achieved / peak,
                              "peak_source": note, "algorithmic_per_launch": work * det_s / lps}
        t_meas = measured_traffic(args.workload, args.precision, args.block_seconds, n_det, st_name,
                                  subset=args.banks is not None)
        if t_meas:
            per_stage[st_name]["traffic"] = {"bytes_per_launch": t_meas, "kernel": TRAFFIC_KERNEL[st_name]}
        if st_name == "recon" and wk["f0_executed"] > 0:   # context: what the tensor pipe actually runs
            per_stage[st_name]["f0_kernel_executed_tflop_per_step"] = wk["f0_executed"] * det_s / 1e12
    dom = max(per_stage, key=lambda k: stages[k][0])
    d = per_stage[dom]
    traffic = measured_traffic(args.workload, args.precision, args.block_seconds, n_det, dom,
                               subset=args.banks is not None)
    roofline = {"kernel": d["kernel"], "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"],
                "unit": d["unit"], "frac": d["frac"], "traffic": traffic, "peak_source": d["peak_source"],
                "traffic_source": (f"ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, {TRAFFIC_PROFILE}"
                                   if traffic else None),
                "algorithmic_per_launch": d["algorithmic_per_launch"], "launch_ms": d["launch_ms"]}
    stage_ms = {k: round(v[0] / args.steps, 4) for k, v in stages.items()}

    # a short run of the streaming loop at 10x real time (the full serving measurement is --serve)
    serving = None
    if rank == 0 and world == 1 and not args.no_serve_summary:
        serving = {"0.25s_blocks_10x": serve_measure(F0 // 4, 10.0, 800),
                   "1s_blocks_10x": serve_measure(F0, 10.0, 200)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(ms), "higher_is_better": True,
            "scaling": "weak" if len(all_banks) == 1 else "strong", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp16_split": "f16", "bf16_split": "bf16"}[args.precision],
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "n_templates": M, "n_banks": len(banks_sb),
                       "n_detectors": n_det, "block_seconds": args.block_seconds, "precision": args.precision,
                       "l2": "flushed between steps (256 MB write on the stream, inside the timed region)",
                       "pulls": "each step's triggers submitted behind its push, collected two pushes later",
                       "bases_total": sum(s.n_basis for x in banks_sb for s in x), "bank_forms": forms,
                       "parallelism": (f"replicas x{world}" if len(all_banks) == 1 else f"bank shards x{world}")},
            "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "roofline": roofline, "cpu_baseline": cpu,
            "max_dsnr_vs_fp32": max_dsnr,
            "precision": precision,
            "latency_ms_1s_blocks": ({"p50": statistics.median(lat),
                                      "p99": sorted(lat)[min(len(lat) - 1, int(0.99 * len(lat)))],
                                      "n": len(lat)} if lat else None),
            "stage_ms_per_step": stage_ms,
            "ms_per_step_with_stage_events": statistics.mean(ms_t),
            "kernels": per_stage,
            "serving": serving,
            "autotune": tune_info,
            "xi2": xi2,
            "whiten": whiten,
            "paths": paths,
        }
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, dist = dist_init(args)
    if args.impl == "reference":
        run_reference(args, rank, world, dist)
    else:
        run_lloid(args, rank, world, dist)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
