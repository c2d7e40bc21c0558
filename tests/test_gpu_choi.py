"""Choi-Jamiolkowski relative states (Sec. 4, Eqs. 16-17) through the C ABI,
against the oracle: density matrix, Monte Carlo trajectories (single-gate and
fused-pass paths from a non-basis start) and the fixed-rank factor."""
import math

import numpy as np
import pytest

from oracle import choi as ochoi
from paper_1412_2293_gb300 import circuits as pcirc
from paper_1412_2293_gb300 import inputs, qs

pytestmark = pytest.mark.gpu
SEED = inputs.DEFAULT_SEED


@pytest.fixture(scope="module", autouse=True)
def library():
    from paper_1412_2293_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return qs.lib()


def test_entangled_start_in_every_mode():
    m = 3
    om = ochoi.maximally_entangled(m)
    h = qs.qs_create(2 * m, 2, 0, qs.QS_STATEVEC, qs.QS_C128)
    qs.qs_set_maximally_entangled(h)
    np.testing.assert_allclose(qs.qs_get_state(h).reshape(2, -1), np.stack([om, om]), atol=1e-15)
    qs.qs_destroy(h)
    h = qs.qs_create(2 * m, 1, 0, qs.QS_DENSITY, qs.QS_C128)
    qs.qs_set_maximally_entangled(h)
    np.testing.assert_allclose(qs.qs_get_state(h), np.outer(om, om.conj()).ravel(), atol=1e-15)
    qs.qs_destroy(h)
    h = qs.qs_create(2 * m, 1, 4, qs.QS_FIXED_RANK, qs.QS_C128)
    qs.qs_set_maximally_entangled(h)
    assert qs.qs_get_rank(h) == 1
    np.testing.assert_allclose(qs.qs_get_state(h).reshape(4, -1)[0], om, atol=1e-15)
    qs.qs_destroy(h)
    h = qs.qs_create(5, 1, 0, qs.QS_STATEVEC, qs.QS_C128)
    with pytest.raises(qs.QSError) as ei:
        qs.qs_set_maximally_entangled(h)
    assert ei.value.status == qs.QS_ERR_INVALID_ARG
    qs.qs_destroy(h)


def test_relative_state_density_matches_oracle():
    m, e = 3, 0.05
    ops = inputs.qft_circuit(m)
    h = qs.qs_create(2 * m, 1, 0, qs.QS_DENSITY, qs.QS_C128)
    qs.qs_set_maximally_entangled(h)
    pcirc.apply_ops(h, ops, e, SEED)
    got = qs.qs_get_state(h)
    psi = ochoi.ideal_relative(m, ops)
    f = qs.qs_fidelity(h, psi)[0]
    tr = qs.qs_trace(h)[0]
    qs.qs_destroy(h)
    rho = ochoi.relative_state(m, ops, e)
    np.testing.assert_allclose(got, rho.ravel(), atol=1e-12)
    want = np.real(np.vdot(psi, rho @ psi))
    assert abs(f - want) <= 1e-12
    assert abs(tr - 1.0) <= 1e-12


@pytest.mark.parametrize("m,dtype,tol", [(3, qs.QS_C128, 1e-12), (5, qs.QS_C64, 1e-5)])
def test_relative_trajectories_match_oracle(m, dtype, tol):
    """m = 5: 10 qubits, the circuit runs as a fused pass from the entangled start."""
    e, batch = 0.05, 4
    ops = inputs.qft_circuit(m)
    h = qs.qs_create(2 * m, batch, 0, qs.QS_STATEVEC, dtype)
    qs.qs_set_maximally_entangled(h)
    p = qs.qs_plan_create(h, pcirc.to_gates(ops))
    qs.qs_plan_run(p, e, SEED, 0, h)
    qs.qs_plan_destroy(p)
    got = qs.qs_get_state(h).reshape(batch, -1)
    qs.qs_destroy(h)
    for b in range(batch):
        np.testing.assert_allclose(got[b], ochoi.relative_trajectory(m, ops, e, SEED, b), atol=tol)


def test_monte_carlo_relative_fidelity_mean_equals_density():
    m, e, T = 3, 0.2, 256
    ops = inputs.qft_circuit(m)
    psi = ochoi.ideal_relative(m, ops)
    h = qs.qs_create(2 * m, T, 0, qs.QS_STATEVEC, qs.QS_C128)
    qs.qs_set_maximally_entangled(h)
    pcirc.apply_ops(h, ops, e, SEED)
    f = qs.qs_fidelity(h, psi)
    qs.qs_destroy(h)
    hd = qs.qs_create(2 * m, 1, 0, qs.QS_DENSITY, qs.QS_C128)
    qs.qs_set_maximally_entangled(hd)
    pcirc.apply_ops(hd, ops, e, SEED)
    exact = qs.qs_fidelity(hd, psi)[0]
    qs.qs_destroy(hd)
    assert abs(f.mean() - exact) < 4 * f.std() / math.sqrt(T) + 1e-12


def test_fixed_rank_relative_state_at_full_rank_is_exact():
    m, e = 2, 0.1                                        # 4 qubits: full rank 16
    ops = inputs.qft_circuit(m)
    h = qs.qs_create(2 * m, 1, 16, qs.QS_FIXED_RANK, qs.QS_C128)
    qs.qs_set_maximally_entangled(h)
    pcirc.apply_ops(h, ops, e, SEED)
    r = qs.qs_get_rank(h)
    L = qs.qs_get_state(h).reshape(16, -1)[:r].T
    qs.qs_destroy(h)
    np.testing.assert_allclose(L @ L.conj().T, ochoi.relative_state(m, ops, e), atol=1e-12)


# ---------------------------------------------------------------- rank-1 by branch selection (Eqs. 12-15)
from oracle import circuits as ocirc  # noqa: E402
from oracle import gates as ogates  # noqa: E402


@pytest.mark.parametrize("n", [6, 9])
@pytest.mark.parametrize("rotated", [False, True])
def test_branch_rank1_matches_oracle(n, rotated):
    e, x0 = 0.05, 11
    ops = inputs.qft_circuit(n)
    ideal = ocirc.ideal_state(n, ops, x0)
    for mode, rank in ((qs.QS_STATEVEC, 0), (qs.QS_FIXED_RANK, 1)):
        h = qs.qs_create(n, 1, rank, mode, qs.QS_C128)
        qs.qs_set_basis_state(h, x0)
        pcirc.apply_branch_ops(h, ops, e, rotated)
        f = qs.qs_fidelity(h, ideal)[0]
        got = qs.qs_get_state(h)[: 1 << n]
        qs.qs_destroy(h)
        want = ocirc.run_branch(n, ops, x0, e, rotated)
        np.testing.assert_allclose(got, want, atol=1e-12)
        fw = abs(np.vdot(ideal, want)) ** 2
        assert abs(f - fw) <= 1e-12 * fw


def test_branch_rank1_grover_is_eq10_and_rotation_improves_qft():
    e, n = 0.01, 10
    k, w = inputs.grover_iterations(n), inputs.draw_marked(n, SEED)
    h = qs.qs_create(n, 1, 0, qs.QS_STATEVEC, qs.QS_C128)
    pcirc.apply_branch_ops(h, inputs.grover_circuit(n, k, w), e)
    p = qs.qs_fidelity(h, None, w)[0]
    qs.qs_destroy(h)
    want = ogates.grover_rank1_success(n, k, e)
    assert abs(p - want) <= 1e-12 * want
    ops = inputs.qft_circuit(n)
    ideal = ocirc.ideal_state(n, ops, 3)
    fs = []
    for rotated in (False, True):
        h = qs.qs_create(n, 1, 0, qs.QS_STATEVEC, qs.QS_C128)
        qs.qs_set_basis_state(h, 3)
        pcirc.apply_branch_ops(h, ops, 0.05, rotated)
        fs.append(qs.qs_fidelity(h, ideal)[0])
        qs.qs_destroy(h)
    assert fs[1] > fs[0]                                   # the rotated branch keeps more of the state
