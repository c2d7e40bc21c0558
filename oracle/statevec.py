"""State-vector level of the paper (Sec. 2), complex128.

Test infrastructure only (see the package docstring).

The one-qubit amplitude update of Sec. 2,
    b[i_1..i_k..i_n] = u[i_k, 0] a[i_1..0..i_n] + u[i_k, 1] a[i_1..1..i_n],
and its k-qubit generalisation are written out with explicit index groups:
every amplitude index is split into the bits of the targets (the local index
sum_j bit(targets[j]) << j) and the remaining bits; each group of 2^k
amplitudes sharing the remaining bits is multiplied by U.

Pins: `apply_gate` equals the product with the brute-force 2^n x 2^n
operator of `full_operator` (n <= 6); the index groups partition 0..2^n-1
(n <= 12); ideal Grover and QFT circuits reproduce their closed forms.
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np


@lru_cache(maxsize=48)
def group_indices(n: int, targets: tuple) -> np.ndarray:
    """(2^(n-k), 2^k) array: row = the non-target bits, column = local index."""
    k = len(targets)
    if len(set(targets)) != k or any(t < 0 or t >= n for t in targets):
        raise ValueError("invalid targets")
    others = [q for q in range(n) if q not in targets]
    r = np.arange(1 << (n - k), dtype=np.int64)
    base = np.zeros_like(r)
    for pos, q in enumerate(others):
        base |= ((r >> pos) & 1) << q
    c = np.arange(1 << k, dtype=np.int64)
    offs = np.zeros_like(c)
    for j, t in enumerate(targets):
        offs |= ((c >> j) & 1) << t
    idx = base[:, None] | offs[None, :]
    idx.setflags(write=False)
    return idx


def apply_gate(psi: np.ndarray, n: int, targets, U: np.ndarray) -> np.ndarray:
    """New amplitudes after the k-qubit gate U on `targets` (Sec. 2).

    `psi` may carry extra trailing axes (columns of a factor, or of rho):
    the gate acts along axis 0.
    """
    idx = group_indices(n, tuple(int(t) for t in targets))
    out = np.array(psi, dtype=np.complex128, copy=True)
    groups = out[idx]                      # (2^(n-k), 2^k, ...)
    out[idx] = np.einsum("ab,gb...->ga...", U, groups)
    return out


def full_operator(n: int, targets, U: np.ndarray) -> np.ndarray:
    """Brute-force 2^n x 2^n matrix of U on `targets` (identity elsewhere)."""
    N = 1 << n
    tmask = 0
    for t in targets:
        tmask |= 1 << t

    def local(i):
        return sum(((i >> t) & 1) << j for j, t in enumerate(targets))

    M = np.zeros((N, N), dtype=np.complex128)
    for row in range(N):
        for col in range(N):
            if (row & ~tmask) == (col & ~tmask):
                M[row, col] = U[local(row), local(col)]
    return M


def basis_state(n: int, x: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[x] = 1.0
    return psi


def phase_flip(psi: np.ndarray, index: int) -> np.ndarray:
    """I - 2|index><index| (Grover's oracle and, globally rephased, diffusion)."""
    out = np.array(psi, dtype=np.complex128, copy=True)
    out[index] *= -1.0
    return out


def fidelity(phi: np.ndarray, psi: np.ndarray) -> float:
    """|<phi|psi>|^2."""
    return float(abs(np.vdot(phi, psi)) ** 2)
