"""Gate matrices, Kraus sets and the paper's closed forms, in complex128.

Test infrastructure only (see the package docstring).

k-qubit matrices use the local index sum_j bit(targets[j]) << j, so for two
qubits the matrix of "A on targets[0], B on targets[1]" is kron(B, A).

Pins (tests/test_oracle_pins.py): completeness sum E^dagger E = I (Eq. 3);
each Kraus set equals the Gauss-Hermite average over xi of the noisy gate it
replaces (Eqs. 6 and 9); the rank-1 Grover formula (Eq. 10) is reproduced
exactly by the independent fixed-rank simulator; the QFT estimates (Eqs. 11,
15) are compared with the exact density matrix as the sanity checks they are.
"""
from __future__ import annotations

import math

import numpy as np

SQRT_HALF = 1.0 / math.sqrt(2.0)

#: The rotation generator of Eq. 1: V_noise(a) = cos(a) I + sin(a) J.
J = np.array([[0.0, 1.0], [-1.0, 0.0]], dtype=np.complex128)


def hadamard() -> np.ndarray:
    """Eq. 4."""
    return np.array([[1.0, 1.0], [1.0, -1.0]], dtype=np.complex128) * SQRT_HALF


def v_noise(angle: float) -> np.ndarray:
    """Eq. 1 with angle = e * xi."""
    c, s = math.cos(angle), math.sin(angle)
    return np.array([[c, s], [-s, c]], dtype=np.complex128)


def controlled_phase(theta: float) -> np.ndarray:
    """Eq. 2: diag(1, 1, 1, e^{-i theta})."""
    return np.diag([1.0, 1.0, 1.0, np.exp(-1j * theta)]).astype(np.complex128)


def phase_noise(angle: float, k: int) -> np.ndarray:
    """Eq. 8 generalised to k qubits: identity except e^{-i angle} on |1..1>."""
    d = np.ones(1 << k, dtype=np.complex128)
    d[-1] = np.exp(-1j * angle)
    return np.diag(d)


def rotation_noise(xis, e: float) -> np.ndarray:
    """Independent V_noise(e xi_j) on each target j (local-index order)."""
    m = np.ones((1, 1), dtype=np.complex128)
    for xi in xis:  # targets[0] first: it is the least significant local bit
        m = np.kron(v_noise(e * xi), m)
    return m


def noisy_unitary(U: np.ndarray, noise: str, e: float, xi_a: float, xi_b: float) -> np.ndarray:
    """One Monte Carlo sample of a noisy gate.

    rotation: U * (V(e xi) on every target), Eq. 5 (V acts first);
              targets[0] takes xi_a, targets[1] takes xi_b.
    phase   : U * U_R(e xi_a), Eqs. 7-8.
    """
    k = int(round(math.log2(U.shape[0])))
    if noise == "rotation":
        xis = [xi_a, xi_b][:k]
        if k > 2:
            raise ValueError("rotation noise is defined for 1- and 2-qubit gates")
        return U @ rotation_noise(xis, e)
    if noise == "phase":
        return U @ phase_noise(e * xi_a, k)
    raise ValueError(noise)


def hadamard_noise_weights(e: float):
    """lambda_1, lambda_2 of Eq. 6: (1 +- exp(-2 e^2)) / 2."""
    q = math.exp(-2.0 * e * e)
    return 0.5 * (1.0 + q), 0.5 * (1.0 - q)


def rotation_kraus(U: np.ndarray, e: float):
    """Kraus set of U * V_noise averaged over xi (Eqs. 5-6).

    One qubit: {sqrt(l1) U, sqrt(l2) U J}.  Two qubits (independent noise on
    each target): the tensor products of the one-qubit sets, ordered with the
    targets[0] operator varying fastest.
    """
    k = int(round(math.log2(U.shape[0])))
    l1, l2 = hadamard_noise_weights(e)
    one = [math.sqrt(l1) * np.eye(2, dtype=np.complex128), math.sqrt(l2) * J]
    if k == 1:
        return [U @ a for a in one]
    if k == 2:
        return [U @ np.kron(b, a) for b in one for a in one]
    raise ValueError("rotation noise is defined for 1- and 2-qubit gates")


def phase_kraus(U: np.ndarray, e: float):
    """Kraus set of U * U_R averaged over xi (Eqs. 7-9), P = exp(-e^2)."""
    k = int(round(math.log2(U.shape[0])))
    P = math.exp(-e * e)
    d1 = np.ones(1 << k, dtype=np.complex128)
    d1[-1] = math.sqrt(P)
    d2 = np.zeros(1 << k, dtype=np.complex128)
    d2[-1] = math.sqrt(1.0 - P)
    return [U @ np.diag(d1), U @ np.diag(d2)]


def rotated_phase_kraus(U: np.ndarray, e: float):
    """The rotated Kraus pair of the controlled phase (Eqs. 12-14):
    B_1 = (E_1 + f E_2) / sqrt(1 + f^2), B_2 = (-f E_1 + E_2) / sqrt(1 + f^2)
    with {E_1, E_2} of Eq. 9 and f of Eq. 13 -- the same channel, its first
    operator along the leading singular vector of the matrix psi of Eq. 12."""
    E1, E2 = phase_kraus(U, e)
    f = rotated_cp_f(e)
    s = 1.0 / math.sqrt(1.0 + f * f)
    return [s * (E1 + f * E2), s * (-f * E1 + E2)]


def branch_operator(U: np.ndarray, noise: str, e: float, rotated: bool = False) -> np.ndarray:
    """The first (dominant) Kraus operator of a noisy gate: sqrt(lambda_1) U for
    rotation noise (Eq. 6), U diag(1,..,1,sqrt P) for phase noise (Eq. 9), or
    the rotated B_1 of Eq. 14 -- the single branch kept by the rank-1 estimates
    behind Eqs. 11 and 15."""
    if noise == "phase":
        return (rotated_phase_kraus(U, e) if rotated else phase_kraus(U, e))[0]
    return kraus_set(U, noise, e)[0]


def kraus_set(U: np.ndarray, noise: str, e: float):
    if noise == "rotation":
        return rotation_kraus(U, e)
    if noise == "phase":
        return phase_kraus(U, e)
    raise ValueError(noise)


# ---------------------------------------------------------------- closed forms

def grover_ideal_success(n: int, k: int) -> float:
    """Ideal success probability sin^2((2k+1) asin(2^{-n/2}))."""
    return math.sin((2 * k + 1) * math.asin(2.0 ** (-n / 2.0))) ** 2


def grover_rank1_success(n: int, k: int, e: float) -> float:
    """Eq. 10: p_noise(k) = lambda_1^(n + 2nk) p_ideal(k)."""
    l1, _ = hadamard_noise_weights(e)
    return l1 ** (n + 2 * n * k) * grover_ideal_success(n, k)


def qft_estimate_eq11(n: int, e: float) -> float:
    """Eq. 11: P_H^n P_R^{n(n-1)/8}, P_H = lambda_1, P_R = exp(-e^2)."""
    ph, _ = hadamard_noise_weights(e)
    return ph ** n * math.exp(-e * e) ** (n * (n - 1) / 8.0)


def rotated_cp_f(e: float) -> float:
    """f of Eqs. 13-14: (sqrt(1+3P) - P - 1) / sqrt(P(1-P))."""
    P = math.exp(-e * e)
    return (math.sqrt(1.0 + 3.0 * P) - P - 1.0) / math.sqrt(P * (1.0 - P))


def qft_estimate_eq15(n: int, e: float) -> float:
    """Eq. 15: P_H^n P~_R^{n(n-1)/8}, P~_R = (sqrt P + f sqrt(1-P))^2 / (1+f^2)^4."""
    ph, _ = hadamard_noise_weights(e)
    P = math.exp(-e * e)
    f = rotated_cp_f(e)
    pr = (math.sqrt(P) + f * math.sqrt(1.0 - P)) ** 2 / (1.0 + f * f) ** 4
    return ph ** n * pr ** (n * (n - 1) / 8.0)
