"""Circuit runners: gate descriptors through each representation of the paper.

Test infrastructure only (see the package docstring).

A circuit is a list of ``paper_1412_2293_gb300.inputs.Op`` descriptors; gate
ids are positions in that list (flips included) and key the noise draw of the
Monte Carlo method (Sec. 2): trajectory b at gate g uses
``philox.normal_pair(seed, b, g)``.

  * ``run_trajectory``  one Monte Carlo trajectory (Sec. 2, Eqs. 1-2):
    noisy H = H V(e xi_a) (Eq. 5, V first); noisy CP = U_theta U_R(e xi_a)
    (Eqs. 7-8).
  * ``run_density``     the exact density matrix with every noisy gate replaced
    by its xi-averaged Kraus set (Sec. 3.1, Eqs. 6 and 9).
  * ``run_fixed_rank``  the same channels on a rank-r factor (Sec. 3.2).
  * ``ideal_state``     the noiseless circuit (reference of the fidelity).
"""
from __future__ import annotations

import numpy as np

from . import density, fixed_rank, gates, philox, statevec


def op_unitary(op) -> np.ndarray:
    if op.kind == "H":
        return gates.hadamard()
    if op.kind == "CP":
        return gates.controlled_phase(op.theta)
    raise ValueError(op.kind)


def op_targets(op):
    if op.kind == "CP":
        return (op.qubits[1], op.qubits[0])   # (k, j): the matrix is symmetric
    return tuple(op.qubits)


def op_noise(op) -> str:
    return "phase" if op.kind == "CP" else "rotation"


def run_trajectory(n, ops, x0, e, seed, traj, noisy=True) -> np.ndarray:
    psi = statevec.basis_state(n, x0)
    for g, op in enumerate(ops):
        if op.kind == "FLIP":
            psi = statevec.phase_flip(psi, op.index)
            continue
        U = op_unitary(op)
        if noisy and op.noisy:
            xa, xb = philox.normal_pair(seed, traj, g)
            U = gates.noisy_unitary(U, op_noise(op), e, xa, xb)
        psi = statevec.apply_gate(psi, n, op_targets(op), U)
    return psi


def ideal_state(n, ops, x0) -> np.ndarray:
    return run_trajectory(n, ops, x0, 0.0, 0, 0, noisy=False)


def trajectory_fidelities(n, ops, x0, e, seed, trajs, ref=None):
    """|<ideal|psi_b>|^2 for each trajectory b in `trajs`."""
    if ref is None:
        ref = ideal_state(n, ops, x0)
    return np.array([statevec.fidelity(ref, run_trajectory(n, ops, x0, e, seed, b)) for b in trajs])


def run_density(n, ops, x0, e) -> np.ndarray:
    rho = density.pure(statevec.basis_state(n, x0))
    for op in ops:
        if op.kind == "FLIP":
            rho = density.phase_flip(rho, op.index)
            continue
        U = op_unitary(op)
        if op.noisy:
            rho = density.apply_channel(rho, n, op_targets(op), gates.kraus_set(U, op_noise(op), e))
        else:
            rho = density.apply_unitary(rho, n, op_targets(op), U)
    return rho


def run_fixed_rank(n, ops, x0, e, r, normalize=False, trace_log=None) -> np.ndarray:
    L = fixed_rank.initial_factor(n, x0)
    for op in ops:
        if op.kind == "FLIP":
            L = fixed_rank.phase_flip(L, op.index)
            continue
        U = op_unitary(op)
        if op.noisy:
            kr = gates.kraus_set(U, op_noise(op), e)
            L, lam = fixed_rank.truncate(fixed_rank.apply_kraus(L, n, op_targets(op), kr), r, normalize)
            if trace_log is not None:
                trace_log.append(float(np.sum(lam[:L.shape[1]])))
        else:
            L = fixed_rank.apply_unitary(L, n, op_targets(op), U)
    return L


def run_branch(n, ops, x0, e, rotated=False) -> np.ndarray:
    """Rank-1 by branch selection: every noisy gate replaced by its first Kraus
    operator (direct, Eq. 9, or rotated, Eq. 14); the state is not renormalised,
    so |<ideal|psi>|^2 is the rank-1 estimate of the fidelity (Sec. 3.2, Fig. 4)."""
    psi = statevec.basis_state(n, x0)
    for op in ops:
        if op.kind == "FLIP":
            psi = statevec.phase_flip(psi, op.index)
            continue
        U = op_unitary(op)
        if op.noisy:
            U = gates.branch_operator(U, op_noise(op), e, rotated)
        psi = statevec.apply_gate(psi, n, op_targets(op), U)
    return psi
