"""Amplitude and phase relaxation (T1, T2) and the correction codes of Sec. 4.

Test infrastructure only (see the package docstring).

Sec. 4 names the two relaxation processes of its relative-state package (T1
amplitude, T2 phase) without giving their Kraus forms; the textbook forms
are taken here.  Over a time t a qubit relaxing with T1 and T2 undergoes
amplitude damping with gamma = 1 - exp(-t/T1) followed by pure dephasing that
brings the total decay of the coherences to exp(-t/T2):

    K0 = diag(1, c),  K1 = [[0, sqrt(gamma)], [0, 0]],
    K2 = diag(0, sqrt(exp(-t/T1) - c^2)),   c = exp(-t/T2),

physical for T2 <= 2 T1.  Populations relax as rho_11 -> exp(-t/T1) rho_11
(the lost weight moves to rho_00) and coherences as rho_01 -> c rho_01.

A phase error of probability p is the channel {sqrt(1-p) I, sqrt(p) Z}; it
scales coherences by 1 - 2p, i.e. it is the phase relaxation above with
T1 = infinity and exp(-t/T2) = 1 - 2p, which is Eq. 19.

Circuits (Sec. 4.1, 4.2; Fig. 5 is not reproduced in the text, so the
textbook circuits are taken): a step list of ("U", targets, matrix) and
("K", targets, [E_i]) entries, run on the density matrix of one data qubit,
its code qubits and one reference qubit (the last).  The reference and the
data qubit start in the maximally entangled state of Eq. 16, so the fidelity
with the ideal output is the relative-state fidelity of the logical channel
(Eq. 17).  After decoding the syndrome qubits are reset to |0> (the channel
{|0><0|, |0><1|}), which leaves the data-reference state as it is and makes
the ideal output pure.

  * three-qubit phase code: CNOT(0,1) CNOT(0,2), H on 0..2; errors; H on
    0..2, CNOT(0,1) CNOT(0,2), Toffoli(1,2 -> 0).
  * Shor's nine-qubit code: CNOT(0,3) CNOT(0,6), H on 0,3,6, then CNOT(b,b+1)
    CNOT(b,b+2) for b = 0,3,6; errors; the inner decoders (CNOTs and
    Toffoli(b+1,b+2 -> b)), H on 0,3,6, CNOT(0,3) CNOT(0,6), Toffoli(3,6 -> 0).

Pins (tests/test_oracle_relaxation.py): the relaxation set is complete and
gives the closed-form populations and coherences; two relaxations of t1 and
t2 compose to one of t1 + t2; Eq. 19's phase relaxation equals the phase
error channel; the three-qubit code's relative-state fidelity is
1 - 3p^2 + 2p^3 and the minimum over pure inputs of sqrt(<psi|rho|psi>) is
Eq. 18; Shor's code under phase errors follows the same law with the
block error probability p_b = (1 - (1-2p)^3) / 2 (a block carries a phase
error when an odd number of its three qubits do); p = 0 gives 1.
"""
from __future__ import annotations

import math

import numpy as np

from . import density, statevec

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
H = np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)


def cnot() -> np.ndarray:
    """CNOT on targets (control, target): local index bit 0 = control."""
    U = np.eye(4, dtype=np.complex128)
    U[[1, 3]] = U[[3, 1]]
    return U


def toffoli() -> np.ndarray:
    """Toffoli on targets (control, control, target): flips bit 2 when bits 0, 1 are set."""
    U = np.eye(8, dtype=np.complex128)
    U[[3, 7]] = U[[7, 3]]
    return U


def relaxation_kraus(t: float, T1: float, T2: float):
    """Amplitude damping (T1) then pure dephasing, total coherence decay exp(-t/T2)."""
    if not (t >= 0 and T1 > 0 and T2 > 0):
        raise ValueError("need t >= 0, T1 > 0, T2 > 0")
    if T2 > 2 * T1:
        raise ValueError("T2 > 2 T1 is not a channel")
    keep = math.exp(-t / T1)            # T1 = inf gives keep = 1 (no damping)
    c = math.exp(-t / T2)
    gamma = 1.0 - keep
    K0 = np.array([[1, 0], [0, c]], dtype=np.complex128)
    K1 = np.array([[0, math.sqrt(gamma)], [0, 0]], dtype=np.complex128)
    K2 = np.array([[0, 0], [0, math.sqrt(max(keep - c * c, 0.0))]], dtype=np.complex128)
    return [K0, K1, K2]


def phase_error_kraus(p: float):
    """Phase error of probability p on one qubit."""
    return [math.sqrt(1.0 - p) * I2, math.sqrt(p) * Z]


def t2_from_p(t: float, p: float) -> float:
    """Eq. 19: the T2 whose phase relaxation over t equals a phase error of probability p."""
    return -t / math.log(1.0 - 2.0 * p)


def reset_kraus():
    """Reset of a qubit to |0>."""
    return [np.array([[1, 0], [0, 0]], dtype=np.complex128),
            np.array([[0, 1], [0, 0]], dtype=np.complex128)]


def run_steps(n: int, steps, rho: np.ndarray) -> np.ndarray:
    for kind, targets, m in steps:
        if kind == "U":
            rho = density.apply_unitary(rho, n, targets, m)
        else:
            rho = density.apply_channel(rho, n, targets, m)
    return rho


def _bell_prep(data: int, ref: int):
    return [("U", (data,), H), ("U", (data, ref), cnot())]


def phase_code_encoder():
    return [("U", (0, 1), cnot()), ("U", (0, 2), cnot())] + [("U", (q,), H) for q in range(3)]


def phase_code_decoder():
    return ([("U", (q,), H) for q in range(3)]
            + [("U", (0, 1), cnot()), ("U", (0, 2), cnot()), ("U", (1, 2, 0), toffoli())])


def shor_encoder():
    s = [("U", (0, 3), cnot()), ("U", (0, 6), cnot())] + [("U", (q,), H) for q in (0, 3, 6)]
    for b in (0, 3, 6):
        s += [("U", (b, b + 1), cnot()), ("U", (b, b + 2), cnot())]
    return s


def shor_decoder():
    s = []
    for b in (0, 3, 6):
        s += [("U", (b, b + 1), cnot()), ("U", (b, b + 2), cnot()), ("U", (b + 1, b + 2, b), toffoli())]
    s += [("U", (q,), H) for q in (0, 3, 6)]
    s += [("U", (0, 3), cnot()), ("U", (0, 6), cnot()), ("U", (3, 6, 0), toffoli())]
    return s


CODES = {"phase3": 3, "shor9": 9}      # code qubits


def _encoder(code: str):
    return phase_code_encoder() if code == "phase3" else shor_encoder()


def _decoder(code: str):
    return phase_code_decoder() if code == "phase3" else shor_decoder()


def code_steps(code: str, errors, logical=None):
    """Steps of one protected use of the data qubit.

    errors(q) -> Kraus set acting on code qubit q between encoding and
    decoding.  `logical` is an optional list of steps applied after encoding
    (a logical gate, e.g. `logical_z`).
    """
    nq = CODES[code]
    s = _encoder(code) + list(logical or [])
    s += [("K", (q,), errors(q)) for q in range(nq)]
    s += _decoder(code)
    s += [("K", (q,), reset_kraus()) for q in range(1, nq)]
    return s


def logical_z(code: str):
    """Logical Z of both codes: X on every code qubit (the code words are
    |+..+> +- |-..-> patterns on which X^{(x) 3} acts as the block sign)."""
    return [("U", (q,), X) for q in range(CODES[code])]


def code_relative_fidelity(code: str, errors, logical=None, ideal_logical=None) -> float:
    """<Psi|rho|Psi> of the logical channel's relative state (data 0, reference last)."""
    nq = CODES[code]
    n = nq + 1
    prep = _bell_prep(0, nq)
    rho = density.pure(statevec.basis_state(n, 0))
    rho = run_steps(n, prep + code_steps(code, errors, logical), rho)
    psi = statevec.basis_state(n, 0)
    for kind, targets, m in prep + list(ideal_logical or []):
        psi = statevec.apply_gate(psi, n, targets, m)
    return density.fidelity(psi, rho)


def uncoded_relative_fidelity(channel, gate=None) -> float:
    """Same quantity for one unprotected qubit (data 0, reference 1)."""
    rho = density.pure(statevec.basis_state(2, 0))
    steps = _bell_prep(0, 1) + ([("U", (0,), gate)] if gate is not None else []) + [("K", (0,), channel)]
    rho = run_steps(2, steps, rho)
    psi = statevec.basis_state(2, 0)
    for kind, targets, m in _bell_prep(0, 1) + ([("U", (0,), gate)] if gate is not None else []):
        psi = statevec.apply_gate(psi, 2, targets, m)
    return density.fidelity(psi, rho)


def phase_code_output(p: float, psi_in: np.ndarray) -> np.ndarray:
    """Data-qubit density matrix after the three-qubit code for a pure input."""
    n = 3
    psi = np.zeros(8, dtype=np.complex128)
    psi[0], psi[1] = psi_in[0], psi_in[1]
    rho = run_steps(n, code_steps("phase3", lambda q: phase_error_kraus(p)), density.pure(psi))
    r = rho.reshape(4, 2, 4, 2)           # [ancillas, data, ancillas, data]
    return np.einsum("aiaj->ij", r)


def qft_relaxation_fidelity(m: int, t: float, T1: float, T2: float, ops) -> float:
    """Relative-state fidelity of an m-qubit circuit whose gates are ideal and
    after each of which every system qubit relaxes for t (Fig. 9's setting).

    `ops` are (targets, matrix) pairs on system qubits 0..m-1; references are
    qubits m..2m-1 (Eq. 16 layout i + (i << m)).
    """
    n = 2 * m
    omega = np.zeros(1 << n, dtype=np.complex128)
    i = np.arange(1 << m)
    omega[i + (i << m)] = 2.0 ** (-m / 2)
    rho = density.pure(omega)
    psi = omega.copy()
    K = relaxation_kraus(t, T1, T2)
    for targets, U in ops:
        rho = density.apply_unitary(rho, n, targets, U)
        psi = statevec.apply_gate(psi, n, targets, U)
        for q in range(m):
            rho = density.apply_channel(rho, n, (q,), K)
    return density.fidelity(psi, rho)

