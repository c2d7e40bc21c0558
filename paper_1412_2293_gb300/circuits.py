"""Product-side circuit helpers: gate descriptors -> qs_gate structs and runs.

The matrices are the paper's: the Hadamard of Eq. 4 (noisy: rotation noise of
Eq. 1 acting first, Eq. 5) and the controlled phase shift of Eq. 2 (noisy:
theta -> theta + e xi, Eqs. 7-8).  Everything here only marshals arguments;
the simulation runs in the CUDA library.
"""
from __future__ import annotations

import math
from typing import List

import numpy as np

from . import qs
from .inputs import Op

_H = np.array([[1.0, 1.0], [1.0, -1.0]], dtype=np.complex128) / math.sqrt(2.0)


def hadamard() -> np.ndarray:
    return _H.copy()


def controlled_phase(theta: float) -> np.ndarray:
    return np.diag([1.0, 1.0, 1.0, np.exp(-1j * theta)]).astype(np.complex128)


def op_gate(op: Op, per_member_flip: bool = False):
    """qs_gate for one descriptor."""
    if op.kind == "H":
        return qs.make_gate((op.qubits[0],), _H, noisy=op.noisy, noise=qs.QS_NOISE_ROTATION)
    if op.kind == "CP":
        j, k = op.qubits
        return qs.make_gate((k, j), controlled_phase(op.theta), noisy=op.noisy, noise=qs.QS_NOISE_PHASE)
    if op.kind == "FLIP":
        if per_member_flip and op.index != 0:
            return qs.make_gate(kind=qs.QS_FLIP_PER_MEMBER)
        return qs.make_gate(kind=qs.QS_GATE_FLIP, index=op.index)
    raise ValueError(op.kind)


def to_gates(ops: List[Op], per_member_flip: bool = False):
    return [op_gate(o, per_member_flip) for o in ops]


def apply_ops(h, ops: List[Op], e: float, seed: int, gate_id0: int = 0):
    """Issue a circuit gate by gate through the single-gate entry points.

    Gate g of the list draws its noise with gate id gate_id0 + g."""
    for g, op in enumerate(ops):
        if op.kind == "FLIP":
            qs.qs_apply_phase_flip(h, op.index)
            continue
        if op.kind == "H":
            targets, U, noise = (op.qubits[0],), _H, qs.QS_NOISE_ROTATION
        else:
            j, k = op.qubits
            targets, U, noise = (k, j), controlled_phase(op.theta), qs.QS_NOISE_PHASE
        if op.noisy:
            qs.qs_apply_noisy_gate(h, targets, U, noise, e, seed, gate_id0 + g)
        else:
            qs.qs_apply_gate(h, targets, U)


def apply_branch_ops(h, ops: List[Op], e: float, rotated: bool = False):
    """Issue a circuit with every noisy gate replaced by its first Kraus branch
    (direct, Eq. 9, or rotated, Eqs. 12-14): the rank-1 estimates of Sec. 3.2."""
    for op in ops:
        if op.kind == "FLIP":
            qs.qs_apply_phase_flip(h, op.index)
            continue
        if op.kind == "H":
            targets, U, noise = (op.qubits[0],), _H, qs.QS_NOISE_ROTATION
        else:
            j, k = op.qubits
            targets, U, noise = (k, j), controlled_phase(op.theta), qs.QS_NOISE_PHASE
        if op.noisy:
            qs.qs_apply_branch_gate(h, targets, U, noise, e, rotated)
        else:
            qs.qs_apply_gate(h, targets, U)


def ideal_reference(n: int, ops: List[Op], x0: int, dtype: int, stream=None):
    """A batch-1 handle holding the noiseless circuit output (the fidelity reference)."""
    h = qs.qs_create(n, 1, 0, qs.QS_STATEVEC, dtype, stream)
    try:
        qs.qs_set_basis_state(h, x0)
        ideal = [Op(o.kind, o.qubits, o.theta, o.index, False) for o in ops]
        p = qs.qs_plan_create(h, to_gates(ideal))
        try:
            qs.qs_plan_run(p, 0.0, 0, 0, h)
        finally:
            qs.qs_plan_destroy(p)
        qs.qs_synchronize(h)
    except Exception:
        qs.qs_destroy(h)
        raise
    return h
