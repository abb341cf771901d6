"""Properties of the seeded workload generator: unit-norm rows, slice plans
on the decimation grid that satisfy pre-synchronisation (Eq. 9) for every
bank family, and reproducible strain."""
import numpy as np

import workloads as W
from oracle import lloid_oracle as O


def _check_plans(w):
    for bank, plan in zip(w.banks, w.plans):
        sl = [O.OracleSlice(r, J, np.zeros((1, N)), np.zeros((2 * bank.n_templates, 1)))
              for r, J, N in zip(plan.rate, plan.j_start, plan.n_taps)]
        assert O.presync_ok(sl, w.f0)
        assert plan.rate[0] == w.f0 and plan.j_start[0] == 0
        for r, J, N in zip(plan.rate, plan.j_start, plan.n_taps):
            assert J % (w.f0 // r) == 0


def test_plans_satisfy_presync():
    _check_plans(W.make_workload("bank64", n_seconds=8, n_inj=0))
    _check_plans(W.make_workload("bank1000", n_templates=50, n_seconds=8, n_det=1, n_inj=0))
    _check_plans(W.make_workload("banks20", n_templates=400, n_banks=8, n_seconds=8, n_det=1, n_inj=0))
    _check_plans(W.make_workload("banks500", n_templates=3000, n_banks=40, n_seconds=8, n_det=1, n_inj=0))


def test_rows_unit_norm_and_strain_reproducible():
    w = W.make_workload("tiny", n_seconds=8)
    rows = w.banks[0].full()
    assert np.allclose(np.linalg.norm(rows, axis=1), 1.0, atol=1e-12)
    assert np.array_equal(w.strain(0), W.make_workload("tiny", n_seconds=8).strain(0))


def test_bank_indices_pick_the_same_banks():
    """A few banks of a multi-bank workload, built alone, are the banks of the full set."""
    full = W.make_workload("banks20", n_templates=400, n_banks=8, n_seconds=8, n_det=1, n_inj=0)
    part = W.make_workload("banks20", n_templates=400, n_banks=8, n_seconds=8, n_det=1, n_inj=0, bank_indices=(5, 2))
    for b, k in zip(part.banks, (5, 2)):
        assert np.array_equal(b.mchirp, full.banks[k].mchirp)
        assert b.n_samples == full.banks[k].n_samples
    assert part.plans == [full.plans[5], full.plans[2]]
