"""Choi-Jamiolkowski relative states of noisy circuits (Sec. 4, Eqs. 16-17).

Test infrastructure only (see the package docstring).

An n-qubit circuit acts on the first subsystem (qubits 0..n-1) of 2n qubits
prepared in the maximally entangled state of Eq. 16,
    |Omega> = 2^{-n/2} sum_i |i>_sys |i>_ref   (amplitude index i + (i << n)),
and the relative state of Eq. 17 is the 2n-qubit density matrix
rho_E = (E (x) I)(|Omega><Omega|).  The accuracy of the circuit as a whole is
the fidelity <Psi|rho_E|Psi> with the ideal relative state
|Psi> = (U (x) I)|Omega>.

The runners repeat those of circuits.py on 2n qubits with every gate on
qubits 0..n-1 and the same gate ids (so the same noise draws).  Phase flips
(the Grover oracle and diffusion) are not part of this level: a flip of one
system index is not a flip of one 2n-qubit amplitude, and the paper's
relative states are shown for the QFT.

Pins (tests/test_oracle_pins.py): the relative state has trace 1 and
reference marginal I / 2^n (the channel preserves the trace); for a single
channel {E_i} with ideal U the fidelity is sum_i |tr(U^dagger E_i)|^2 / 4^n
(a single noisy Hadamard: lambda_1 of Eq. 6); noiseless circuits give 1; the
exact relative state is the mean over Monte Carlo trajectories.
"""
from __future__ import annotations

import numpy as np

from . import circuits, density, gates, philox, statevec


def maximally_entangled(n: int) -> np.ndarray:
    """|Omega> of Eq. 16 on 2n qubits (system = low n bits)."""
    psi = np.zeros(1 << (2 * n), dtype=np.complex128)
    i = np.arange(1 << n)
    psi[i + (i << n)] = 2.0 ** (-n / 2)
    return psi


def _check(ops):
    for op in ops:
        if op.kind == "FLIP":
            raise ValueError("phase flips are not defined on relative states here")


def relative_trajectory(n: int, ops, e: float, seed: int, traj: int, noisy: bool = True) -> np.ndarray:
    """One Monte Carlo trajectory of (U_xi (x) I)|Omega> (gate ids as in circuits.py)."""
    _check(ops)
    psi = maximally_entangled(n)
    for g, op in enumerate(ops):
        U = circuits.op_unitary(op)
        if noisy and op.noisy:
            xa, xb = philox.normal_pair(seed, traj, g)
            U = gates.noisy_unitary(U, circuits.op_noise(op), e, xa, xb)
        psi = statevec.apply_gate(psi, 2 * n, circuits.op_targets(op), U)
    return psi


def ideal_relative(n: int, ops) -> np.ndarray:
    """|Psi> = (U (x) I)|Omega>."""
    return relative_trajectory(n, ops, 0.0, 0, 0, noisy=False)


def relative_state(n: int, ops, e: float) -> np.ndarray:
    """rho_E of Eq. 17 with every noisy gate replaced by its Kraus set (Eqs. 6, 9)."""
    _check(ops)
    rho = density.pure(maximally_entangled(n))
    for op in ops:
        U = circuits.op_unitary(op)
        if op.noisy:
            rho = density.apply_channel(rho, 2 * n, circuits.op_targets(op), gates.kraus_set(U, circuits.op_noise(op), e))
        else:
            rho = density.apply_unitary(rho, 2 * n, circuits.op_targets(op), U)
    return rho


def reference_marginal(rho: np.ndarray, n: int) -> np.ndarray:
    """Partial trace of a 2n-qubit density matrix over the system (low n bits)."""
    d = 1 << n
    r = rho.reshape(d, d, d, d)          # [ref_row, sys_row, ref_col, sys_col]
    return np.einsum("aibi->ab", r)


def channel_fidelity(kraus, U: np.ndarray) -> float:
    """<Psi|rho_E|Psi> of one channel {E_i} with ideal U: sum_i |tr(U^dagger E_i)|^2 / d^2."""
    d = U.shape[0]
    return float(sum(abs(np.trace(U.conj().T @ E)) ** 2 for E in kraus) / (d * d))
