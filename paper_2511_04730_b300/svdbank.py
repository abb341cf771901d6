"""Offline SVD bank construction (Eq. 3), the producer of ``load_bank`` inputs.

For each time slice of a template group the real/imaginary-stacked slice
matrix A^s[row][m] = sqrt(D_s) h_row[J_s + D_s m] (m < N_s, the slice sampled
at its own rate, with the sqrt(D) that pairs with the unit-variance
downsampled strain) is factored as A = V Sigma U^T; the leading L_s basis
rows u_l and the coefficients v_il sigma_l are kept, L_s being the smallest
count holding the requested fraction of the slice energy (99.99 % by default).

The factorisation goes through the Gram matrix of the smaller side in FP64
(eigendecomposition), which gives the same retained subspace as a direct SVD
and is several times cheaper for the wide slice matrices of long templates.
This is offline, host-side work; nothing of it runs per strain block.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np


@dataclasses.dataclass
class SliceArrays:
    rate: int
    j_start: int
    bases: np.ndarray      # [L, N] float64, orthonormal rows
    coeffs: np.ndarray     # [2M, L] float64, row 2i real / 2i+1 imaginary
    energy_kept: float     # retained fraction of sum sigma^2

    @property
    def n_basis(self) -> int:
        return int(self.bases.shape[0])

    @property
    def n_taps(self) -> int:
        return int(self.bases.shape[1])


def factor_slice(A: np.ndarray, energy: float = 0.9999, max_basis: Optional[int] = None):
    """Leading factors of A (rows x taps): returns (bases [L, taps], coeffs [rows, L], kept)."""
    rows, taps = A.shape
    if rows <= taps:
        G = A @ A.T                         # rows x rows
        lam, V = np.linalg.eigh(G)
        order = np.argsort(lam)[::-1]
        lam, V = np.clip(lam[order], 0.0, None), V[:, order]
    else:
        G = A.T @ A                         # taps x taps
        lam, U = np.linalg.eigh(G)
        order = np.argsort(lam)[::-1]
        lam, U = np.clip(lam[order], 0.0, None), U[:, order]
    total = float(lam.sum())
    if total <= 0.0:
        return np.zeros((0, taps)), np.zeros((rows, 0)), 1.0
    cum = np.cumsum(lam)
    L = int(np.searchsorted(cum, energy * total) + 1)
    L = min(L, int(np.count_nonzero(lam > 0)))
    if max_basis is not None:
        L = min(L, max_basis)
    sig = np.sqrt(lam[:L])
    if rows <= taps:
        V = V[:, :L]
        bases = (A.T @ V / sig[None, :]).T          # u_l = A^T v_l / sigma_l
        coeffs = V * sig[None, :]
    else:
        U = U[:, :L]
        bases = U.T
        coeffs = A @ U                               # v_l sigma_l = A u_l
    # re-orthonormalise the bases (Gram route loses a little orthogonality)
    Q, R = np.linalg.qr(bases.T)
    bases = Q.T
    coeffs = coeffs @ R.T
    return bases, coeffs, float(cum[L - 1] / total)


def build_svd_bank(bank, plan, energy: float = 0.9999, max_basis: Optional[int] = None) -> List[SliceArrays]:
    """SVD bank of a ``workloads.ChirpBank`` cut by a ``workloads.SlicePlan``."""
    out = []
    for rate, J, N in zip(plan.rate, plan.j_start, plan.n_taps):
        D = bank.f0 // rate
        j = J + D * np.arange(N)
        A = math.sqrt(D) * bank.rows(j)
        bases, coeffs, kept = factor_slice(A, energy, max_basis)
        if bases.shape[0] == 0:
            continue
        out.append(SliceArrays(int(rate), int(J), np.ascontiguousarray(bases), np.ascontiguousarray(coeffs), kept))
    return out


def template_autocorrelation(bank, half: int, chunk: int = 16) -> np.ndarray:
    """R_i(t), t = -half .. half, of every template of a ``workloads.ChirpBank``
    (Eq. 10): the complex template hbar = h_c + i h_s correlated with itself
    through FFTs, R(t) = sum_j hbar[j] conj(hbar[j - t]) / sum_j |hbar[j]|^2.
    Returns [M, 2 half + 1] complex128."""
    M = bank.mchirp.size
    out = np.empty((M, 2 * half + 1), dtype=np.complex128)
    for a in range(0, M, chunk):
        idx = list(range(a, min(M, a + chunk)))
        lo = int(min(bank.j_lo[i] for i in idx))
        hi = int(max(bank.j_hi[i] for i in idx))
        r = bank.rows(np.arange(lo, hi), idx)
        h = r[0::2] + 1j * r[1::2]
        n = 1 << int(math.ceil(math.log2(2 * h.shape[1] + 1)))
        H = np.fft.fft(h, n, axis=1)
        c = np.fft.ifft(H * np.conj(H), axis=1)           # c[t] = sum_j h[j + t] conj(h[j])
        lags = np.arange(-half, half + 1)
        out[a:a + len(idx)] = c[:, lags % n] / c[:, :1].real
    return out
