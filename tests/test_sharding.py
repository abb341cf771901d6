"""Multi-rank bank sharding on CPU: two gloo ranks each filter their LPT share
of the banks with the FP64 oracle and gather the triggers; the merged list
equals the single-process list.  No GPU is involved: the data path has no
collective, only this host-side merge."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import workloads as W
from oracle import lloid_oracle as O
from paper_2511_04730_b300 import sharding
from paper_2511_04730_b300.lloid import TRIGGER_DTYPE

F0 = 2048


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case():
    return W.make_workload("banks20", n_templates=36, n_banks=3, n_seconds=16, n_det=1, n_inj=0)


def _triggers_of(w, bank_ids, d):
    out = []
    for b in bank_ids:
        bank, plan = w.banks[b], w.plans[b]
        z = O.lloid_snr(d, O.svd_bank(bank, plan), F0)
        for t in O.triggers(z, F0, bank=b):
            rec = np.zeros(1, dtype=TRIGGER_DTYPE)
            rec["detector"], rec["bank"], rec["tmpl"], rec["is_bank_max"] = t.detector, t.bank, t.tmpl, t.is_bank_max
            rec["window"], rec["sample"], rec["snr"] = t.window, t.sample, t.snr
            rec["phase"], rec["re"], rec["im"] = t.phase, t.re, t.im
            out.append(rec)
    return np.concatenate(out) if out else np.zeros(0, dtype=TRIGGER_DTYPE)


def _rank_main(rank, world, port, result_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = _case()
    d = w.strain(0).astype(np.float64)
    costs = [sharding.bank_cost(O.svd_bank(b, p), b.n_templates) for b, p in zip(w.banks, w.plans)]
    mine = sharding.assign_banks(costs, world)[rank]
    merged = sharding.gather_triggers(_triggers_of(w, mine, d))
    if rank == 0:
        np.save(result_path, merged)
    dist.barrier()
    dist.destroy_process_group()


def test_lpt_assignment():
    assert sharding.assign_banks([5, 3, 3, 2, 1], 2) == [[0, 3], [1, 2, 4]]
    assert sharding.assign_banks([1, 1, 1], 3) == [[0], [1], [2]]
    parts = sharding.assign_banks(list(np.random.default_rng(0).uniform(1, 10, 50)), 4)
    assert sorted(sum(parts, [])) == list(range(50))


def test_two_gloo_ranks_match_one_process(tmp_path):
    w = _case()
    d = w.strain(0).astype(np.float64)
    ref = sharding.merge_triggers([_triggers_of(w, range(len(w.banks)), d)])
    out = str(tmp_path / "merged.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    merged = np.load(out)
    assert len(ref) > 0
    assert np.array_equal(merged, ref)
    loud = sharding.loudest_per_window(merged)
    for win in np.unique(merged["window"]):
        rows = merged[merged["window"] == win]
        assert loud[loud["window"] == win]["snr"][0] == rows["snr"].max()
