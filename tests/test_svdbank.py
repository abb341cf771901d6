"""The product's offline SVD bank construction (Eq. 3) and its Eq. 10
autocorrelation, on the CPU.  The factorisation goes through a Gram matrix and
an eigendecomposition.  These tests pin it to what an SVD fixes: orthonormal
bases, a residual equal to the discarded singular values (Eckart-Young), the
smallest basis count that holds the requested energy, and both Gram branches.
The autocorrelation is checked against its definition, summed directly."""
import math

import numpy as np
import pytest

import workloads as W
from paper_2511_04730_b300.svdbank import build_svd_bank, factor_slice, template_autocorrelation


def _low_rank(rows, taps, rank, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((rows, rank)) @ np.diag(np.geomspace(1.0, 1e-4, rank)) @ rng.standard_normal((rank, taps))
    return a + 1e-9 * rng.standard_normal((rows, taps))


@pytest.mark.parametrize("rows,taps", [(40, 300), (300, 40)])     # both Gram branches
@pytest.mark.parametrize("energy", [0.99, 0.9999])
def test_factor_slice_is_the_truncated_svd(rows, taps, energy):
    A = _low_rank(rows, taps, 24, rows + taps)
    bases, coeffs, kept = factor_slice(A, energy)
    L = bases.shape[0]
    assert bases.shape == (L, taps) and coeffs.shape == (rows, L)
    assert np.allclose(bases @ bases.T, np.eye(L), atol=1e-10)
    s = np.linalg.svd(A, compute_uv=False)
    cum = np.cumsum(s ** 2) / np.sum(s ** 2)
    assert L == int(np.searchsorted(cum, energy) + 1)          # the smallest count reaching the energy
    assert kept == pytest.approx(cum[L - 1], rel=1e-10)
    resid = np.linalg.norm(A - coeffs @ bases) ** 2
    assert resid == pytest.approx(np.sum(s[L:] ** 2), rel=1e-6, abs=1e-12 * np.sum(s ** 2))


def test_factor_slice_caps_and_degenerate_cases():
    A = _low_rank(30, 200, 20, 3)
    b, c, _ = factor_slice(A, 0.999999, max_basis=5)
    assert b.shape[0] == 5 and c.shape == (30, 5)
    s = np.linalg.svd(A, compute_uv=False)
    assert np.linalg.norm(A - c @ b) ** 2 == pytest.approx(np.sum(s[5:] ** 2), rel=1e-6)
    b, c, kept = factor_slice(np.zeros((6, 50)))
    assert b.shape == (0, 50) and c.shape == (6, 0) and kept == 1.0
    # rank one: one basis reproduces it exactly
    u = np.arange(1.0, 9.0)[:, None] * np.linspace(-1.0, 1.0, 64)[None, :]
    b, c, kept = factor_slice(u, 0.9999)
    assert b.shape[0] == 1 and np.allclose(c @ b, u, atol=1e-12) and kept == pytest.approx(1.0)


def test_bank_slices_reproduce_the_templates():
    """Every slice of a real bank: coeffs x bases gives back the sqrt(D)-scaled
    template samples of the slice to within the discarded energy."""
    w = W.make_workload("bank64", n_seconds=8, n_inj=0)
    bank, plan = w.banks[0], w.plans[0]
    sl = build_svd_bank(bank, plan, energy=0.9999)
    assert [s.rate for s in sl] == [int(r) for r in plan.rate]
    for s, N in zip(sl, plan.n_taps):
        D = bank.f0 // s.rate
        A = math.sqrt(D) * bank.rows(s.j_start + D * np.arange(N))
        err = np.linalg.norm(A - s.coeffs @ s.bases) ** 2
        assert err <= (1.0 - s.energy_kept) * np.linalg.norm(A) ** 2 * (1 + 1e-8) + 1e-20
        assert s.energy_kept >= 0.9999


def test_autocorrelation_matches_its_definition():
    w = W.make_workload("tiny", n_seconds=8, n_inj=0)
    bank = w.banks[0]
    half = 12
    R = template_autocorrelation(bank, half, chunk=3)
    full = bank.full()                                   # [2M, n] rows re / im
    h = full[0::2] + 1j * full[1::2]
    n = h.shape[1]
    for i in range(h.shape[0]):
        norm = np.sum(np.abs(h[i]) ** 2)
        for t in range(-half, half + 1):
            j = np.arange(max(0, t), min(n, n + t))    # h[j] and h[j - t] both defined
            want = np.sum(h[i, j] * np.conj(h[i, j - t])) / norm
            assert abs(R[i, t + half] - want) < 1e-12
        assert R[i, half] == pytest.approx(1.0)
        assert np.allclose(R[i, ::-1], np.conj(R[i]), atol=1e-12)   # R(-t) = conj R(t)
