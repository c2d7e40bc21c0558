"""Relative states of protected and relaxing circuits (Sec. 4.1-4.3) on the GPU.

Everything here marshals arguments: the gates, channels and fidelities run in
the CUDA library (qs_apply_gate, qs_apply_kraus, qs_apply_relaxation,
qs_fidelity_stored).

Layout of a code experiment: data qubit 0, code qubits 1..nq-1, reference
qubit nq.  The data qubit and the reference start in the maximally entangled
state of Eq. 16 (H on 0, CNOT 0 -> nq), so the fidelity with the ideal output
is the relative-state fidelity (Eq. 17) of the logical one-qubit channel.
The circuits are the textbook ones (Fig. 5 is not reproduced in the text):

  * "phase3", the three-qubit phase code (Sec. 4.1): encode CNOT(0,1)
    CNOT(0,2), H on 0..2; errors; decode H on 0..2, CNOT(0,1) CNOT(0,2),
    Toffoli(1,2 -> 0);
  * "shor9", Shor's code (Sec. 4.2): CNOT(0,3) CNOT(0,6), H on 0,3,6, then
    CNOT(b,b+1) CNOT(b,b+2) for b = 0,3,6; errors; the inner decoders with
    Toffoli(b+1,b+2 -> b), H on 0,3,6, CNOT(0,3) CNOT(0,6), Toffoli(3,6 -> 0).

After decoding the syndrome qubits are reset to |0> ({|0><0|, |0><1|}), which
leaves the data-reference state unchanged and makes the ideal output pure.
Errors act on every code qubit between encoding and decoding: a phase error
of probability p ({sqrt(1-p) I, sqrt(p) Z}) or T1/T2 relaxation over t.
The logical Z of both codes is X on every code qubit.
"""
from __future__ import annotations

import math

import numpy as np

from . import circuits, qs

X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
H = circuits.hadamard()
CNOT = np.eye(4, dtype=np.complex128)[[0, 3, 2, 1]]          # targets (control, target)
TOFFOLI = np.eye(8, dtype=np.complex128)[[0, 1, 2, 7, 4, 5, 6, 3]]   # (control, control, target)
RESET = [np.array([[1, 0], [0, 0]], dtype=np.complex128), np.array([[0, 1], [0, 0]], dtype=np.complex128)]

CODE_QUBITS = {"phase3": 3, "shor9": 9}


def phase_error(p: float):
    return [math.sqrt(1.0 - p) * np.eye(2, dtype=np.complex128), math.sqrt(p) * Z]


def _encoder(code: str):
    if code == "phase3":
        return [((0, 1), CNOT), ((0, 2), CNOT), ((0,), H), ((1,), H), ((2,), H)]
    s = [((0, 3), CNOT), ((0, 6), CNOT), ((0,), H), ((3,), H), ((6,), H)]
    for b in (0, 3, 6):
        s += [((b, b + 1), CNOT), ((b, b + 2), CNOT)]
    return s


def _decoder(code: str):
    if code == "phase3":
        return [((0,), H), ((1,), H), ((2,), H), ((0, 1), CNOT), ((0, 2), CNOT), ((1, 2, 0), TOFFOLI)]
    s = []
    for b in (0, 3, 6):
        s += [((b, b + 1), CNOT), ((b, b + 2), CNOT), ((b + 1, b + 2, b), TOFFOLI)]
    s += [((0,), H), ((3,), H), ((6,), H), ((0, 3), CNOT), ((0, 6), CNOT), ((3, 6, 0), TOFFOLI)]
    return s


def _apply_errors(h, qubits, error):
    kind = error[0]
    if kind == "phase":
        ks = phase_error(error[1])
        for q in qubits:
            qs.qs_apply_kraus(h, (q,), ks)
    elif kind == "relax":
        t, T1, T2 = error[1:]
        qs.qs_apply_relaxation(h, list(qubits), t, T1, T2)
    elif kind != "none":
        raise ValueError(f"unknown error kind {kind!r}")


def code_relative_fidelity(code: str, error, logical_z: bool = False, dtype: int = qs.QS_C128,
                           mode: int = qs.QS_DENSITY, rank: int = 0) -> float:
    """<Psi|rho|Psi> of the logical channel's relative state.

    error: ("phase", p), ("relax", t, T1, T2) or ("none",).  With logical_z
    the logical Z (X on every code qubit) follows the encoder and the ideal
    output is Z on the data qubit.
    """
    nq = CODE_QUBITS[code]
    n = nq + 1
    prep = [((0,), H), ((0, nq), CNOT)]
    h = qs.qs_create(n, rank=rank, mode=mode, dtype=dtype)
    ref = qs.qs_create(n, mode=qs.QS_STATEVEC, dtype=dtype)
    try:
        qs.qs_set_basis_state(h, 0)
        steps = prep + _encoder(code) + ([((q,), X) for q in range(nq)] if logical_z else [])
        for t, U in steps:
            qs.qs_apply_gate(h, t, U)
        _apply_errors(h, range(nq), error)
        for t, U in _decoder(code):
            qs.qs_apply_gate(h, t, U)
        for q in range(1, nq):
            qs.qs_apply_kraus(h, (q,), RESET)
        qs.qs_set_basis_state(ref, 0)
        for t, U in prep + ([((0,), Z)] if logical_z else []):
            qs.qs_apply_gate(ref, t, U)
        qs.qs_set_reference_from(h, ref, 0)
        return float(qs.qs_fidelity_stored(h)[0])
    finally:
        qs.qs_destroy(ref)
        qs.qs_destroy(h)


def uncoded_relative_fidelity(error, gate=None, dtype: int = qs.QS_C128) -> float:
    """Same quantity for one unprotected qubit (data 0, reference 1)."""
    h = qs.qs_create(2, mode=qs.QS_DENSITY, dtype=dtype)
    ref = qs.qs_create(2, mode=qs.QS_STATEVEC, dtype=dtype)
    try:
        steps = [((0,), H), ((0, 1), CNOT)] + ([((0,), gate)] if gate is not None else [])
        for hh in (h, ref):
            qs.qs_set_basis_state(hh, 0)
            for t, U in steps:
                qs.qs_apply_gate(hh, t, U)
        _apply_errors(h, (0,), error)
        qs.qs_set_reference_from(h, ref, 0)
        return float(qs.qs_fidelity_stored(h)[0])
    finally:
        qs.qs_destroy(ref)
        qs.qs_destroy(h)


def circuit_relaxation_fidelity(m: int, gates, t: float, T1: float, T2: float, dtype: int = qs.QS_C128,
                                mode: int = qs.QS_DENSITY, rank: int = 0) -> float:
    """Relative-state fidelity of an m-qubit circuit of ideal gates after each
    of which every system qubit relaxes for t (Sec. 4.3, Fig. 9's setting).

    gates: (targets, U) pairs on qubits 0..m-1; the references are qubits
    m..2m-1 (Eq. 16 layout i + (i << m)).
    """
    n = 2 * m
    h = qs.qs_create(n, rank=rank, mode=mode, dtype=dtype)
    ref = qs.qs_create(n, mode=qs.QS_STATEVEC, dtype=dtype)
    try:
        qs.qs_set_maximally_entangled(h)
        qs.qs_set_maximally_entangled(ref)
        sysq = list(range(m))
        for targets, U in gates:
            qs.qs_apply_gate(h, targets, U)
            qs.qs_apply_gate(ref, targets, U)
            qs.qs_apply_relaxation(h, sysq, t, T1, T2)
        qs.qs_set_reference_from(h, ref, 0)
        return float(qs.qs_fidelity_stored(h)[0])
    finally:
        qs.qs_destroy(ref)
        qs.qs_destroy(h)


def qft_gates(m: int):
    """The QFT of the paper's circuits (no final swaps) as (targets, U) pairs."""
    out = []
    for j in range(m - 1, -1, -1):
        out.append(((j,), H))
        for k in range(j - 1, -1, -1):
            out.append(((k, j), circuits.controlled_phase(math.pi / float(1 << (j - k)))))
    return out
