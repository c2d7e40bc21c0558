"""T1/T2 relaxation, three-qubit and Shor codes, and density-matrix gates on
three and four qubits (Sec. 4.1-4.3) through the C ABI, against the oracle
and the closed forms it is pinned to (Eq. 18)."""
import math

import numpy as np
import pytest

from oracle import density as odens
from oracle import gates as ogates
from oracle import relaxation as orx
from paper_1412_2293_gb300 import codes, qs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def library():
    from paper_1412_2293_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return qs.lib()


def rand_density(rng, n, rank=4):
    A = rng.normal(size=(1 << n, rank)) + 1j * rng.normal(size=(1 << n, rank))
    rho = A @ A.conj().T
    return rho / np.trace(rho)


def rand_unitary(rng, d):
    q, r = np.linalg.qr(rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d)))
    return q * (np.diag(r) / np.abs(np.diag(r)))


def oracle_relax(rho, n, qubits, t, T1, T2):
    K = orx.relaxation_kraus(t, T1, T2)
    for q in qubits:
        rho = odens.apply_channel(rho, n, (q,), K)
    return rho


TOL = {qs.QS_C128: 1e-13, qs.QS_C64: 2e-6}


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
@pytest.mark.parametrize("n,qubits", [(5, [2]), (5, [0, 4]), (5, [4, 1, 3]), (5, [0, 1, 2, 3, 4]), (10, [0, 9, 5])])
@pytest.mark.parametrize("times", [(0.7, 3.0, 2.0), (1.0, math.inf, 0.8), (0.5, 1.0, 2.0)])
def test_density_relaxation_parity(dtype, n, qubits, times):
    rng = np.random.default_rng(n * 7 + len(qubits))
    rho = rand_density(rng, n)
    h = qs.qs_create(n, 1, 0, qs.QS_DENSITY, dtype)
    try:
        qs.qs_set_state(h, rho.ravel())
        qs.qs_apply_relaxation(h, qubits, *times)
        got = qs.qs_get_state(h).reshape(1 << n, 1 << n)
    finally:
        qs.qs_destroy(h)
    want = oracle_relax(rho, n, qubits, *times)
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= TOL[dtype] * scale


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_density_relaxation_full_size_closed_form(dtype):
    # |Omega><Omega| on 14 qubits (the bench's size for this kernel), every
    # qubit relaxed: trace stays 1 and each (system, reference) Bell pair
    # keeps <Phi|(R (x) R)(|Phi><Phi|)|Phi> = (1 + gamma^2 + keep^2 + 2 c^2) / 4
    n, m = 14, 7
    t, T1, T2 = 0.3, 3.0, 2.0
    keep, c = math.exp(-t / T1), math.exp(-t / T2)
    gamma = 1.0 - keep
    want = ((1.0 + gamma ** 2 + keep ** 2 + 2.0 * c * c) / 4.0) ** m
    h = qs.qs_create(n, 1, 0, qs.QS_DENSITY, dtype)
    ref = qs.qs_create(n, 1, 0, qs.QS_STATEVEC, dtype)
    try:
        qs.qs_set_maximally_entangled(h)
        qs.qs_set_maximally_entangled(ref)
        qs.qs_apply_relaxation(h, list(range(n)), t, T1, T2)
        qs.qs_set_reference_from(h, ref, 0)
        f = float(qs.qs_fidelity_stored(h)[0])
        tr = float(qs.qs_trace(h)[0])
    finally:
        qs.qs_destroy(ref)
        qs.qs_destroy(h)
    tol = 1e-12 if dtype == qs.QS_C128 else 2e-5
    assert abs(tr - 1.0) < tol
    assert abs(f - want) < tol


def test_fixed_rank_relaxation_parity():
    n = 4
    rng = np.random.default_rng(3)
    U = rand_unitary(rng, 16)
    h = qs.qs_create(n, 1, 9, qs.QS_FIXED_RANK, qs.QS_C128)
    try:
        qs.qs_set_basis_state(h, 0)
        qs.qs_apply_gate(h, (0, 1, 2, 3), U)
        qs.qs_apply_relaxation(h, [1, 3], 0.8, 2.0, 1.5)
        cols = qs.qs_get_rank(h)
        L = qs.qs_get_state(h).reshape(-1, 1 << n)[:cols]
    finally:
        qs.qs_destroy(h)
    got = L.T @ L.conj()
    psi = U[:, 0]
    want = oracle_relax(np.outer(psi, psi.conj()), n, [1, 3], 0.8, 2.0, 1.5)
    assert cols == 9
    assert np.abs(got - want).max() < 1e-13


def test_fixed_rank_relaxation_omits_zero_operators():
    # pure dephasing (T1 = inf): two Kraus operators per qubit, rank 2^3 (with
    # the zero amplitude-damping operator kept it would be 27 > 16)
    h = qs.qs_create(3, 1, 16, qs.QS_FIXED_RANK, qs.QS_C128)
    try:
        qs.qs_set_basis_state(h, 0)
        for q in range(3):
            qs.qs_apply_gate(h, (q,), ogates.hadamard())
        qs.qs_apply_relaxation(h, [0, 1, 2], 1.0, math.inf, 2.0)
        assert qs.qs_get_rank(h) == 8
    finally:
        qs.qs_destroy(h)


@pytest.mark.parametrize("k", [3, 4])
@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_density_gates_on_three_and_four_qubits(k, dtype):
    n = 6
    rng = np.random.default_rng(10 + k)
    rho = rand_density(rng, n)
    U = rand_unitary(rng, 1 << k)
    targets = (5, 0, 3, 2)[:k]
    h = qs.qs_create(n, 1, 0, qs.QS_DENSITY, dtype)
    try:
        qs.qs_set_state(h, rho.ravel())
        qs.qs_apply_gate(h, targets, U)
        qs.qs_apply_gate(h, (1, 4, 2)[:3], orx.toffoli())
        got = qs.qs_get_state(h).reshape(1 << n, 1 << n)
    finally:
        qs.qs_destroy(h)
    want = odens.apply_unitary(odens.apply_unitary(rho, n, targets, U), n, (1, 4, 2), orx.toffoli())
    assert np.abs(got - want).max() < TOL[dtype] * 10 * np.abs(want).max()


@pytest.mark.parametrize("p", [0.0, 0.03, 0.2, 0.5])
@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_three_qubit_code_eq18(p, dtype):
    f = codes.code_relative_fidelity("phase3", ("phase", p), dtype=dtype)
    want = 1.0 - 3.0 * p * p + 2.0 * p ** 3          # Eq. 18 squared
    assert abs(f - want) < (1e-13 if dtype == qs.QS_C128 else 2e-6)
    assert abs(math.sqrt(f) - orx_fmin(p)) < (1e-12 if dtype == qs.QS_C128 else 2e-6)


def orx_fmin(p):
    return math.sqrt(1.0 - 3.0 * p * p + 2.0 * p ** 3)


def test_three_qubit_code_phase_relaxation_eq19():
    # the phase error as phase relaxation with T2 from Eq. 19
    p, t = 0.1, 1.0
    f = codes.code_relative_fidelity("phase3", ("relax", t, math.inf, orx.t2_from_p(t, p)))
    assert abs(f - (1.0 - 3.0 * p * p + 2.0 * p ** 3)) < 1e-13


@pytest.mark.parametrize("logical_z", [False, True])
def test_three_qubit_code_t1_t2_parity(logical_z):
    # Fig. 8's setting: T1 = 3, T2 = 2 over one time unit
    f = codes.code_relative_fidelity("phase3", ("relax", 1.0, 3.0, 2.0), logical_z=logical_z)
    want = orx.code_relative_fidelity("phase3", lambda q: orx.relaxation_kraus(1.0, 3.0, 2.0),
                                      logical=orx.logical_z("phase3") if logical_z else None,
                                      ideal_logical=[("U", (0,), orx.Z)] if logical_z else None)
    assert abs(f - want) < 1e-13


def test_three_qubit_code_fixed_rank():
    p = 0.07
    f = codes.code_relative_fidelity("phase3", ("phase", p), mode=qs.QS_FIXED_RANK, rank=16)
    assert abs(f - (1.0 - 3.0 * p * p + 2.0 * p ** 3)) < 1e-12


@pytest.mark.parametrize("p", [0.01, 0.1])
def test_shor_code_phase_errors_closed_form(p):
    f = codes.code_relative_fidelity("shor9", ("phase", p))
    pb = (1.0 - (1.0 - 2.0 * p) ** 3) / 2.0
    assert abs(f - (1.0 - 3.0 * pb * pb + 2.0 * pb ** 3)) < 1e-12


def test_shor_code_t1_t2_parity():
    f = codes.code_relative_fidelity("shor9", ("relax", 1.0, 3.0, 2.0), logical_z=True)
    want = orx.code_relative_fidelity("shor9", lambda q: orx.relaxation_kraus(1.0, 3.0, 2.0),
                                      logical=orx.logical_z("shor9"), ideal_logical=[("U", (0,), orx.Z)])
    assert abs(f - want) < 1e-12


def test_uncoded_qubit():
    assert abs(codes.uncoded_relative_fidelity(("phase", 0.2)) - 0.8) < 1e-14
    f = codes.uncoded_relative_fidelity(("relax", 1.0, 3.0, 2.0), gate=orx.Z)
    want = orx.uncoded_relative_fidelity(orx.relaxation_kraus(1.0, 3.0, 2.0), gate=orx.Z)
    assert abs(f - want) < 1e-14


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
@pytest.mark.parametrize("T1,T2", [(3.0, 2.0), (20.0, 5.0), (math.inf, 10.0)])
def test_qft_relaxation_parity(dtype, T1, T2):
    m, t = 3, 0.1
    f = codes.circuit_relaxation_fidelity(m, codes.qft_gates(m), t, T1, T2, dtype=dtype)
    ops = []
    for j in range(m - 1, -1, -1):
        ops.append(((j,), ogates.hadamard()))
        for k in range(j - 1, -1, -1):
            ops.append(((k, j), ogates.controlled_phase(math.pi / float(1 << (j - k)))))
    want = orx.qft_relaxation_fidelity(m, t, T1, T2, ops)
    assert abs(f - want) < (1e-12 if dtype == qs.QS_C128 else 2e-5)


def test_relaxation_errors():
    h = qs.qs_create(3, 1, 0, qs.QS_DENSITY, qs.QS_C128)
    sv = qs.qs_create(3, 1, 0, qs.QS_STATEVEC, qs.QS_C128)
    try:
        for args in [([0], 1.0, 1.0, 2.5), ([0], -1.0, 1.0, 1.0), ([0, 0], 1.0, 3.0, 2.0), ([3], 1.0, 3.0, 2.0),
                     ([0], 1.0, 0.0, 1.0), ([0], math.nan, 3.0, 2.0)]:
            with pytest.raises(qs.QSError) as e:
                qs.qs_apply_relaxation(h, *args)
            assert e.value.status == qs.QS_ERR_INVALID_ARG
        with pytest.raises(qs.QSError) as e:
            qs.qs_apply_relaxation(sv, [0], 1.0, 3.0, 2.0)
        assert e.value.status == qs.QS_ERR_NOT_SUPPORTED
        qs.qs_apply_relaxation(h, [], 1.0, 3.0, 2.0)          # nothing to do
    finally:
        qs.qs_destroy(sv)
        qs.qs_destroy(h)
