#!/usr/bin/env python
"""Throughput of the LLOID hot path on B300: template-seconds filtered per second.

Workload (the 1000-template configuration): 1000 Newtonian chirp templates,
chirp mass log-uniform in [1, 20] Msun, 64 s long, cut into 9 time slices at
2048/1024/512/256/128 Hz and SVD-compressed to 99.99 % of each slice's
energy; 2 detectors x 1024 s of seeded unit white noise at 2048 Hz with 20
injections per detector at SNR U[6, 20] (synthetic stand-in for the paper's
mock-data-challenge strain).

A step pushes one block (--block-seconds, default 8 s) of strain for every
detector through every stage (ingest, downsample, basis FIR, upsample,
reconstruction + window maxima, finalisation) and pulls the triggers of the
windows the block completes.  The stream continues across steps, cycling
through the 1024 s record.  L2 is flushed (256 MB write) between steps,
outside the timed intervals, which are CUDA-event pairs on the library's
stream around each step.

Output: one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead (bounded samples of the same workload).
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
REF_M = 8                    # templates per reference-arm step (a bounded oracle sample)
REF_SECONDS = 24             # seconds of strain per reference-arm step (~0.4 s of oracle work)
METRIC = "template-seconds filtered/s at max |dSNR|<=5e-3 vs FP32 path; p50/p99 block latency"
UNIT = "template-s/s"
WORKLOAD = ("1000 Newtonian chirp templates (Mc log-U[1,20] Msun, 64 s, 9 slices 2048/1024/512/256/128 Hz, "
            "SVD 99.99%), 2 detectors x 1024 s white noise + 20 injections/detector, 1 s trigger windows")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", default="lloid", choices=["lloid", "reference"])
    p.add_argument("--precision", default="fp16_split", choices=["fp32", "fp16_split", "bf16_split"])
    p.add_argument("--block-seconds", type=int, default=8)
    p.add_argument("--templates", type=int, default=1000)
    p.add_argument("--seconds", type=int, default=1024)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--whiten-seconds", type=int, default=64,
                   help="seconds of 16384 Hz strain per detector for the whitening measurement (0: skip it)")
    p.add_argument("--xi2-half", type=int, default=350,
                   help="Eq. 10 autocorrelation half-length d for the xi2 measurement (0: skip it)")
    p.add_argument("--no-fp32-compare", action="store_true")
    p.add_argument("--latency-steps", type=int, default=32)
    p.add_argument("--workload", default="bank1000", choices=["bank1000", "banks20", "banks500"])
    p.add_argument("--banks", type=int, default=None, help="use the first N banks of a multi-bank workload")
    p.add_argument("--detectors", type=int, default=None)
    p.add_argument("--serve", action="store_true", help="paced serving loop with latency percentiles")
    p.add_argument("--serve-block", type=int, default=2048)
    p.add_argument("--pace", type=float, default=1.0)
    p.add_argument("--serve-seconds", type=int, default=60)
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
    "bank1000": WORKLOAD,
    "banks20": ("10,000 Newtonian chirp templates (Mc log-U[1,20] Msun) in 20 contiguous-Mc SVD banks of 200-800, "
                "durations 8-64 s, 2 detectors x 4096 s white noise + 100 injections"),
    "banks500": ("500 SVD banks of U{100..1000} templates (~280k, Mc log-U[1,50] Msun, durations 2-128 s, 1-10 slices, "
                 "32-2048 Hz), 3 detectors x 1024 s white noise"),
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


# DRAM read + write bytes per launch of each stage's kernel, from the ncu
# capture summarised in profiles/k_level_tc_k_fir_tc_bank1000.md; valid only
# while the tensor-core kernel sources hash to the prefix it was taken with.
TRAFFIC_SOURCES = ("kernels_tc.cuh", "kernels_tc2.cuh", "lloid_common.cuh")
TRAFFIC_SHA = "822f4761ed7fedee"
TRAFFIC = {("bank1000", "fp16_split", 8, 2): {"upsample": 76.5e6, "recon": 156.9e6, "fir": 118.7e6}}


def measured_traffic(workload, precision, block_seconds, n_det, stage):
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_2511_04730_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != TRAFFIC_SHA:
        return None
    return TRAFFIC.get((workload, precision, block_seconds, n_det), {}).get(stage)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0}, "fallback"


# ---------------------------------------------------------------------------
# CPU oracle leg (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
def oracle_sample(M=64, seconds=68, seed_det=0):
    """Time the FP64 oracle's LLOID on a bounded sample: the first M templates'
    worth of the 1000-template family (same Mc range, same slicing rule), one
    detector, `seconds` of data from the start of the stream."""
    import numpy as np
    import workloads as W
    from oracle import lloid_oracle as O
    w = W.make_workload("bank1000", n_templates=M, n_seconds=seconds, n_det=1, n_inj=0)
    sl = O.svd_bank(w.banks[0], w.plans[0])
    d = w.strain(seed_det).astype(np.float64)
    t, c = time.perf_counter(), time.process_time()
    z = O.lloid_snr(d, sl, F0)
    O.triggers(z, F0)
    dt, dc = time.perf_counter() - t, time.process_time() - c
    cores = max(1, round(dc / dt, 1))          # threads actually busy (CPU time / wall time)
    return M * seconds / dt, dt, f"{M} templates of the 1000-template family x 1 detector x {seconds} s " \
                                 f"(oracle FP64 numpy LLOID + triggers)", cores


def run_reference(args, rank, world, dist):
    """The base contract's reference arm: the oracle, timed on host cores."""
    if rank != 0:
        return
    vals = []
    cores = []
    secs = REF_SECONDS
    for _ in range(args.warmup):
        oracle_sample(M=REF_M, seconds=secs)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, dt, sample, c = oracle_sample(M=REF_M, seconds=secs)
        vals.append(dt)
        cores.append(c)
    wall = time.perf_counter() - t0
    value = REF_M * secs * args.steps / sum(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": max(cores), "kind": "oracle",
                             "sample": "each step: " + sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
    sb = banks_sb[0]
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

    def make_ctx(precision, timing):
        return P.Context(n_detectors=n_det, precision=precision, max_block=B, max_history=max_hist,
                         device=dev, stage_timing=timing)

    def load_all(ctx):
        return [ctx.load_bank(x) for x in banks_sb]

    if args.serve:
        from paper_2511_04730_b300.serving import Server
        SB = args.serve_block
        ctx = P.Context(n_detectors=n_det, precision=args.precision, max_block=SB, max_history=max_hist, device=dev)
        srv = Server(ctx, SB)
        for i, x in enumerate(banks_sb):
            srv.submit(x, tag=i)
        nb = T // SB
        blocks_s = np.ascontiguousarray(strain.reshape(n_det, nb, SB).transpose(1, 0, 2))
        src = lambda k: blocks_s[k % nb]
        warm = max_hist // SB + 4
        for k in range(warm):                          # admit every bank and fill the history
            srv.step(src(k))
        srv.latency_ms.clear()
        n_serve = args.serve_seconds * F0 // SB
        t0 = time.perf_counter()
        srv.run_paced(lambda k: src(warm + k), n_serve, pace=args.pace)
        wall = time.perf_counter() - t0
        ctx.close()
        if rank == 0:
            lat = srv.latency_summary()
            print(json.dumps({
                "mode": "serve", "metric": "per-block latency (block arrival -> its windows' triggers on the host)",
                "latency_ms": lat, "block_seconds": SB / F0, "pace": args.pace, "seconds_streamed": n_serve * SB / F0,
                "wall_s": wall, "template_s_per_s": M * n_det * n_serve * SB / F0 / wall,
                "n_templates": M, "n_banks": len(banks_sb), "n_detectors": n_det, "precision": args.precision,
                "workload": WORKLOADS[args.workload]}), flush=True)
        return

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")

    def run_steps(ctx, k_steps, pos, host=False, lat=None, lag=0):
        """k_steps timed steps; returns (ms per step list, pos, launches, h2d, d2h).
        lag = 1: pull the windows that became ready (xi2 needs d samples of the
        next block), i.e. the previous block's last window and this block's others."""
        ext = torch.cuda.ExternalStream(ctx.stream_ptr, device=f"cuda:{dev}")
        ms, h2d, d2h = [], 0, 0
        l0 = ctx.launch_count()
        with torch.cuda.stream(ext):
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

    result = {}
    per_ctx = {}
    precisions = [args.precision] + ([] if args.no_fp32_compare or args.precision == "fp32" else ["fp32"])
    clocks = None
    for prec in precisions:
        # throughput: K steps without per-stage events
        ctx = make_ctx(prec, timing=False)
        load_all(ctx)
        pos = 0
        _, pos, _, _, _ = run_steps(ctx, args.warmup, pos)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        sampler = ClockSampler(dev) if prec == args.precision else None
        if sampler:
            sampler.start()
            sampler.begin()
        ms, pos, launches, _, _ = run_steps(ctx, args.steps, pos)
        torch.cuda.synchronize()
        if sampler:
            sampler.end()
            clocks = sampler.stop()
        ctx.close()
        per_ctx[prec] = {"ms": ms, "launches": launches}
        if prec != args.precision:
            continue
        # stage breakdown and roofline: the same K steps again, with CUDA events around every stage
        ctx = make_ctx(prec, timing=True)
        load_all(ctx)
        pos = 0
        _, pos, _, _, _ = run_steps(ctx, args.warmup, pos)
        ctx.stage_times(reset=True)
        torch.cuda.synchronize()
        ms_t, pos, _, _, _ = run_steps(ctx, args.steps, pos)
        torch.cuda.synchronize()
        per_ctx[prec]["stages"] = ctx.stage_times(reset=True)
        per_ctx[prec]["ms_timed_stages"] = ms_t
        ctx.close()

    # Eq. 10 (a NEXT row): the same steps with autocorrelations loaded for every bank
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
        _, pos, _, _, _ = run_steps(ctx, args.warmup, pos, lag=1)
        ctx.stage_times(reset=True)
        torch.cuda.synchronize()
        ms_x, pos, _, _, d2h_x = run_steps(ctx, args.steps, pos, lag=1)
        st_x = ctx.stage_times(reset=True)
        ctx.close()
        units_x = M * args.block_seconds * n_det
        xi2 = {"value": units_x * args.steps / (sum(ms_x) / 1000.0), "unit": UNIT,
               "ms_per_step": statistics.mean(ms_x), "autocorr_samples": 2 * args.xi2_half + 1,
               "finalize_plus_xi2_ms_per_step": round(st_x["finalize"][0] / args.steps, 4),
               "recon_ms_per_step": round(st_x["recon"][0] / args.steps, 4),
               "d2h_bytes_per_step": d2h_x // args.steps, "autocorr_build_s": round(t_ac, 1)}

    # PSD estimation and whitening (a NEXT row): 16384 Hz -> 2048 Hz, N = 4 s, Z = 1 s, 16 s pushes
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

    # accuracy of the measured path against the FP32 path (same stream, same blocks)
    max_dsnr = None
    if args.precision != "fp32" and not args.no_fp32_compare:
        a, b = make_ctx(args.precision, False), make_ctx("fp32", False)
        ia, ib = load_all(a), load_all(b)
        max_dsnr = 0.0
        n_chk = min(8, len(ia))                       # compare the first banks (all of them for one bank)
        for k in range((max_hist + 8 * F0) // B):
            blk = d_blocks[k % n_blk]
            a.push_all(k * B, blk)
            b.push_all(k * B, blk)
            if (k + 1) * B >= max_hist:
                for det in range(n_det):
                    for j in range(n_chk):
                        za, _ = a.snr_block(det, ia[j])
                        zb, _ = b.snr_block(det, ib[j])
                        dz = torch.sqrt(((za - zb) ** 2).view(M_list[j], 2, -1).sum(1)).max().item()
                        max_dsnr = max(max_dsnr, dz)
        a.close()
        b.close()

    # end to end: host blocks in, triggers out, through the public API
    e2e = None
    if not args.no_e2e:
        ctx = make_ctx(args.precision, False)
        load_all(ctx)
        pos = 0
        _, pos, _, _, _ = run_steps(ctx, args.warmup, pos, host=True)
        ms_e, pos, _, h2d, d2h = run_steps(ctx, args.steps, pos, host=True)
        ctx.close()
        e2e = {"value": M * args.block_seconds * n_det * args.steps / (sum(ms_e) / 1000.0), "unit": UNIT,
               "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps}

    # per-block latency at 1 s blocks (block arrival on the host -> its window's triggers on the host)
    lat = []
    if args.latency_steps:
        ctx = P.Context(n_detectors=n_det, precision=args.precision, max_block=F0, max_history=max_hist, device=dev)
        load_all(ctx)
        pos = 0
        h_sec = torch.from_numpy(np.ascontiguousarray(
            strain.reshape(n_det, T // F0, F0).transpose(1, 0, 2))).pin_memory()
        warm = max_hist // F0 + 8
        for k in range(warm + args.latency_steps):
            blk = h_sec[(pos // F0) % (T // F0)].numpy()
            t0 = time.perf_counter()
            ctx.push_all(pos, blk)
            ctx.pull(pos // F0)
            if k >= warm:
                lat.append(1000 * (time.perf_counter() - t0))
            pos += F0
        ctx.close()

    main = per_ctx[args.precision]
    ms = main["ms"]
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

    # roofline of the dominant kernel (stage with the largest device time)
    stages = main["stages"]
    dom = max(("fir", "upsample", "recon"), key=lambda k: stages[k][0])
    dur_ms = stages[dom][0] / max(1, stages[dom][1])
    works = [algorithmic_work(x, m) for x, m in zip(banks_sb, M_list)]
    work = {k: sum(wk[k] for wk in works) for k in works[0]}
    det_s = args.block_seconds * n_det
    pk, pk_kind = peaks()
    alu_peak = 148 * 128 * 2 * pk.get("sm_max_mhz", 2032.0) * 1e6 / 1e12
    tc = args.precision != "fp32"
    alu_note = "FP32 FFMA: 148 SMs x 128 lanes x 2 flop x max SM clock"
    tc_peak, tc_note = pk["bf16_tflops_sustained"], f"{pk_kind} dense bf16 sustained (fp16 nominal rate equal)"
    if tc:   # stage -> (kernel, bound, peak, peak note, algorithmic flop per detector-second)
        kinds = {"fir": ("k_fir_tc", "tensor", tc_peak, tc_note, work["fir"]),
                 "upsample": ("k_level_tc (levels below f0)", "tensor", tc_peak, tc_note, work["below_f0"]),
                 "recon": ("k_level_tc (f0 level + window maxima)", "tensor", tc_peak, tc_note, work["at_f0"])}
    else:
        kinds = {"fir": ("k_fir_f32", "alu", alu_peak, alu_note, work["fir"]),
                 "upsample": ("k_upsample", "alu", alu_peak, alu_note, work["ladder"]),
                 "recon": ("k_recon_f32", "alu", alu_peak, alu_note, work["recon"] + work["max"])}
    kname, bound, peak, peak_note, per_dets = kinds[dom]
    launches_dom = max(1.0, stages[dom][1] / args.steps)
    alg = per_dets * det_s / launches_dom          # one launch's share of the stage's work
    achieved = alg / (dur_ms / 1000.0) / 1e12
    traffic = measured_traffic(args.workload, args.precision, args.block_seconds, n_det, dom)
    roofline = {"kernel": kname, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": peak_note,
                "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, "
                                   "profiles/k_level_tc_k_fir_tc_bank1000.md") if traffic else None,
                "algorithmic_flop_per_launch": alg, "launch_ms": dur_ms}
    per_stage = {}
    for st_name in ("fir", "upsample", "recon"):
        ms_l = stages[st_name][0] / max(1, stages[st_name][1])
        k = kinds[st_name]
        lps = stages[st_name][1] / args.steps
        per_stage[st_name] = {"kernel": k[0], "launch_ms": ms_l, "launches_per_step": lps,
                              "algorithmic_tflops": (k[4] * det_s / max(lps, 1.0)) / (ms_l / 1000.0) / 1e12
                              if ms_l > 0 else None}
    recon_info = per_stage
    stage_ms = {k: round(v[0] / args.steps, 4) for k, v in stages.items()}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, dt, sample, cores = oracle_sample()
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample, "seconds": dt}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": statistics.mean(ms), "higher_is_better": True,
            "scaling": "weak" if len(all_banks) == 1 else "strong", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp16_split": "f16", "bf16_split": "bf16"}[args.precision],
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "n_templates": M, "n_banks": len(banks_sb),
                       "n_detectors": n_det, "block_seconds": args.block_seconds, "precision": args.precision,
                       "l2": "flushed between steps (256 MB write, outside the timed events)",
                       "bases_total": sum(s.n_basis for x in banks_sb for s in x),
                       "parallelism": (f"replicas x{world}" if len(all_banks) == 1 else f"bank shards x{world}")},
            "e2e": e2e, "gpu_launches": main["launches"], "clocks": clocks,
            "roofline": roofline, "cpu_baseline": cpu,
            "max_dsnr_vs_fp32": max_dsnr,
            "latency_ms_1s_blocks": ({"p50": statistics.median(lat),
                                      "p99": sorted(lat)[min(len(lat) - 1, int(0.99 * len(lat)))],
                                      "n": len(lat)} if lat else None),
            "stage_ms_per_step": stage_ms,
            "xi2": xi2,
            "whiten": whiten,
            "ms_per_step_with_stage_events": statistics.mean(main["ms_timed_stages"]),
            "kernels": recon_info,
            "paths": {p: units * args.steps / (sum(v["ms"]) / 1000.0) for p, v in per_ctx.items()},
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
