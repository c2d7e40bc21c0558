"""Density-matrix level of the paper (Sec. 3), complex128.

Test infrastructure only (see the package docstring).

`apply_channel` computes Eq. 3, rho <- sum_i E_i rho E_i^dagger, as matrix
algebra on the 2^n x 2^n rho (left product along the rows, right product as
the conjugate transpose of a left product).  `vectorise` / `apply_superop`
restate Sec. 3's reduction to the vector case: with vec index i * 2^n + j,
vec(E rho E^dagger) = (E (x) E*) vec(rho), i.e. a 2k-qubit gate on the column
bits t and the row bits t + n of a 2n-qubit vector.  (The text prints
"U (x) U"; the complex conjugate on the second factor is required for
U rho U^dagger and is the reading taken here.)

Pins: `apply_channel` equals the product with brute-force full operators
(n <= 5); the vectorised form equals `apply_channel`; trace, Hermiticity and
positivity are preserved; the xi-averaged channel equals the Gauss-Hermite
average of the Monte Carlo gate.
"""
from __future__ import annotations

import numpy as np

from . import statevec


def pure(psi: np.ndarray) -> np.ndarray:
    return np.outer(psi, psi.conj())


def left(n: int, targets, E: np.ndarray, rho: np.ndarray) -> np.ndarray:
    """E rho (E acting on the row index)."""
    return statevec.apply_gate(rho, n, targets, E)


def apply_channel(rho: np.ndarray, n: int, targets, kraus) -> np.ndarray:
    """Eq. 3: sum_i E_i rho E_i^dagger."""
    out = np.zeros_like(rho, dtype=np.complex128)
    for E in kraus:
        er = left(n, targets, E, rho)                   # E rho
        out += left(n, targets, E, er.conj().T).conj().T  # (E (E rho)^dag)^dag
    return out


def apply_unitary(rho: np.ndarray, n: int, targets, U: np.ndarray) -> np.ndarray:
    return apply_channel(rho, n, targets, [U])


def phase_flip(rho: np.ndarray, index: int) -> np.ndarray:
    """F rho F with F = I - 2|index><index|."""
    out = np.array(rho, dtype=np.complex128, copy=True)
    out[index, :] *= -1.0
    out[:, index] *= -1.0
    return out


def fidelity(phi: np.ndarray, rho: np.ndarray) -> float:
    """<phi|rho|phi>."""
    return float(np.real(np.vdot(phi, rho @ phi)))


def trace(rho: np.ndarray) -> float:
    return float(np.real(np.trace(rho)))


# ------------------------------------------------------- vectorised (Sec. 3)

def vectorise(rho: np.ndarray) -> np.ndarray:
    """vec(rho)[i * 2^n + j] = rho[i, j]."""
    return np.asarray(rho, dtype=np.complex128).reshape(-1).copy()


def unvectorise(v: np.ndarray, n: int) -> np.ndarray:
    return v.reshape(1 << n, 1 << n)


def superoperator(kraus) -> np.ndarray:
    """sum_i E_i (x) conj(E_i) with the row (E_i) factor on the high bits."""
    return sum(np.kron(E, E.conj()) for E in kraus)


def superop_targets(n: int, targets) -> tuple:
    """Column bits t, then row bits t + n, as the local index of the superop."""
    return tuple(int(t) for t in targets) + tuple(int(t) + n for t in targets)


def apply_superop(v: np.ndarray, n: int, targets, kraus) -> np.ndarray:
    return statevec.apply_gate(v, 2 * n, superop_targets(n, targets), superoperator(kraus))
