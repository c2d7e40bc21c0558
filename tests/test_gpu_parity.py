"""Parity of the CUDA path (through the C ABI) with the oracle, on the GPU.

Tolerances: complex128 results within 1e-12 (amplitudes absolute, fidelities
relative), complex64 within 1e-5; Philox words bit-exact; the Gaussian draws
within a few ulp (libm against CUDA's FP64 log/sincos).
"""
import math

import numpy as np
import pytest

from oracle import circuits as ocirc
from oracle import density as odm
from oracle import fixed_rank as ofr
from oracle import gates as ogates
from oracle import philox as ophilox
from oracle import statevec as osv
from paper_1412_2293_gb300 import circuits as pcirc
from paper_1412_2293_gb300 import inputs, qs
from tests.tolerances import assert_amplitudes_close

pytestmark = pytest.mark.gpu

SEED = inputs.DEFAULT_SEED
TOL = {qs.QS_C128: 1e-12, qs.QS_C64: 1e-5}
DTYPES = [qs.QS_C128, qs.QS_C64]


@pytest.fixture(scope="module", autouse=True)
def library():
    from paper_1412_2293_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return qs.lib()


class Handle:
    def __init__(self, *a, **k):
        self.h = qs.qs_create(*a, **k)

    def __enter__(self):
        return self.h

    def __exit__(self, *exc):
        qs.qs_destroy(self.h)


def rand_unitary(rng, d):
    z = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def rand_states(rng, n, batch):
    v = rng.normal(size=(batch, 1 << n)) + 1j * rng.normal(size=(batch, 1 << n))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


# ----------------------------------------------------------------- noise draw

@pytest.mark.parametrize("seed", [SEED, 0, 2**63 + 12345])
@pytest.mark.parametrize("gate_id", [0, 7, 2**32 + 5])
def test_philox_words_bit_exact_and_normals(seed, gate_id):
    traj0, count = 3, 1024
    words, normals = qs.qs_debug_noise(seed, traj0, gate_id, count)
    for i in range(0, count, 37):
        assert tuple(int(w) for w in words[i]) == ophilox.noise_words(seed, traj0 + i, gate_id)
    xa, xb = ophilox.normal_pairs_array(seed, np.arange(traj0, traj0 + count), gate_id)
    np.testing.assert_allclose(normals[:, 0], xa, rtol=4e-15, atol=4e-15)
    np.testing.assert_allclose(normals[:, 1], xb, rtol=4e-15, atol=4e-15)


# ----------------------------------------------------------------- single gates

@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("targets", [(0,), (6,), (3,), (1, 5), (6, 0), (2, 4, 0), (0, 1, 2, 3), (6, 3, 1, 5)])
def test_ideal_gate_matches_oracle(dtype, targets):
    rng = np.random.default_rng(len(targets) * 10 + targets[0])
    n, batch = 7, 3
    psi = rand_states(rng, n, batch)
    U = rand_unitary(rng, 1 << len(targets))
    with Handle(n, batch, 0, qs.QS_STATEVEC, dtype) as h:
        qs.qs_set_state(h, psi.reshape(-1))
        qs.qs_apply_gate(h, targets, U)
        got = qs.qs_get_state(h).reshape(batch, -1)
    for b in range(batch):
        assert_amplitudes_close(got[b], osv.apply_gate(psi[b], n, targets, U), dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_diagonal_gate_path_matches_oracle(dtype):
    rng = np.random.default_rng(5)
    n, batch = 8, 2
    psi = rand_states(rng, n, batch)
    U = np.diag(np.exp(1j * rng.uniform(0, 6, size=4)))
    U[0, 0] = 1.0
    with Handle(n, batch, 0, qs.QS_STATEVEC, dtype) as h:
        qs.qs_set_state(h, psi.reshape(-1))
        qs.qs_apply_gate(h, (5, 2), U)
        qs.qs_apply_phase_flip(h, 77)
        got = qs.qs_get_state(h).reshape(batch, -1)
    for b in range(batch):
        want = osv.phase_flip(osv.apply_gate(psi[b], n, (5, 2), U), 77)
        assert_amplitudes_close(got[b], want, dtype)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("case", ["H_rot", "U1_rot", "U1_phase", "CP_phase", "U2_rot", "U2_phase"])
def test_noisy_gate_matches_oracle(dtype, case):
    rng = np.random.default_rng(abs(hash(case)) % 1000)
    n, batch, e, gid, off = 6, 5, 0.07, 1234, 7
    psi = rand_states(rng, n, batch)
    if case == "H_rot":
        targets, U, noise = (4,), ogates.hadamard(), "rotation"
    elif case == "U1_rot":
        targets, U, noise = (0,), rand_unitary(rng, 2), "rotation"
    elif case == "U1_phase":
        targets, U, noise = (2,), rand_unitary(rng, 2), "phase"
    elif case == "CP_phase":
        targets, U, noise = (1, 5), ogates.controlled_phase(0.3), "phase"
    elif case == "U2_rot":
        targets, U, noise = (3, 0), rand_unitary(rng, 4), "rotation"
    else:
        targets, U, noise = (5, 1), rand_unitary(rng, 4), "phase"
    qn = qs.QS_NOISE_ROTATION if noise == "rotation" else qs.QS_NOISE_PHASE
    with Handle(n, batch, 0, qs.QS_STATEVEC, dtype) as h:
        qs.qs_set_state(h, psi.reshape(-1))
        qs.qs_set_trajectory_offset(h, off)
        qs.qs_apply_noisy_gate(h, targets, U, qn, e, SEED, gid)
        got = qs.qs_get_state(h).reshape(batch, -1)
    for b in range(batch):
        xa, xb = ophilox.normal_pair(SEED, off + b, gid)
        Ub = ogates.noisy_unitary(U, noise, e, xa, xb)
        assert_amplitudes_close(got[b], osv.apply_gate(psi[b], n, targets, Ub), dtype)


# ----------------------------------------------------------------- circuits

def oracle_traj(n, ops, x0, e, b):
    return ocirc.run_trajectory(n, ops, x0, e, SEED, b)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("circ,n", [("qft", 10), ("qft", 12), ("qft", 13), ("qft", 15), ("grover", 10),
                                    ("grover", 11), ("grover", 13)])
def test_plan_trajectories_match_oracle(dtype, circ, n):
    batch, e = 3, 0.05
    if circ == "qft":
        ops, x0 = inputs.qft_circuit(n), inputs.draw_basis_input(n, SEED)
    else:
        ops, x0 = inputs.grover_circuit(n, 2, inputs.draw_marked(n, SEED)), 0
    with Handle(n, batch, 0, qs.QS_STATEVEC, dtype) as h:
        qs.qs_set_basis_state(h, x0)
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        passes, _ = qs.qs_plan_info(p)
        qs.qs_plan_run(p, e, SEED, 0, h)
        qs.qs_plan_destroy(p)
        got = qs.qs_get_state(h).reshape(batch, -1)
    if circ == "qft" and n >= 13:
        assert passes == 2            # one high-window and one low-window pass
    for b in range(batch):
        assert_amplitudes_close(got[b], oracle_traj(n, ops, x0, e, b), dtype)


@pytest.mark.parametrize("dtype", DTYPES)
def test_gate_by_gate_equals_plan(dtype):
    n, batch, e = 12, 4, 0.02
    ops, x0 = inputs.qft_circuit(n), 1234
    with Handle(n, batch, 0, qs.QS_STATEVEC, dtype) as h1, Handle(n, batch, 0, qs.QS_STATEVEC, dtype) as h2:
        qs.qs_set_basis_state(h1, x0)
        qs.qs_set_basis_state(h2, x0)
        pcirc.apply_ops(h1, ops, e, SEED)
        p = qs.qs_plan_create(h2, pcirc.to_gates(ops))
        qs.qs_plan_run(p, e, SEED, 0, h2)
        a = qs.qs_get_state(h1)
        b = qs.qs_get_state(h2)
        assert_amplitudes_close(a, b, dtype)
        # a second run (graph replay) from the same start gives the same state
        qs.qs_set_basis_state(h2, x0)
        qs.qs_plan_run(p, e, SEED, 0, h2)
        np.testing.assert_allclose(qs.qs_get_state(h2), b, atol=0)
        qs.qs_plan_destroy(p)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [11, 14])
def test_fused_fidelity_and_per_member_starts_match_oracle(dtype, n):
    """The first pass creates per-member basis starts; the last pass reduces the fidelity."""
    batch, e = 5, 0.03
    ops = inputs.qft_circuit(n)
    xs = [(37 * b + 5) % (1 << n) for b in range(batch)]
    ideal0 = ocirc.ideal_state(n, ops, xs[0])
    with Handle(n, batch, 0, qs.QS_STATEVEC, dtype) as h:
        ref = np.asarray(ideal0)
        qs.qs_set_reference(h, ref)
        qs.qs_set_basis_states(h, xs)
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        f_fused = qs.qs_plan_run_fidelity(p, e, SEED, 0, h)
        got = qs.qs_get_state(h).reshape(batch, -1)
        f_sep = qs.qs_fidelity_stored(h)
        # run again from the same starts: replays the captured graph
        qs.qs_set_basis_states(h, xs)
        f_again = qs.qs_plan_run_fidelity(p, e, SEED, 0, h)
        qs.qs_plan_destroy(p)
    np.testing.assert_allclose(f_fused, f_sep, rtol=TOL[dtype], atol=TOL[dtype])
    np.testing.assert_allclose(f_again, f_fused, rtol=0, atol=0)
    for b in range(batch):
        want = oracle_traj(n, ops, xs[b], e, b)
        assert_amplitudes_close(got[b], want, dtype)
        assert abs(f_fused[b] - osv.fidelity(ideal0, want)) <= TOL[dtype] * 10


def test_lazy_start_state_is_written_before_other_consumers():
    n = 10
    with Handle(n, 2, 0, qs.QS_STATEVEC, qs.QS_C128) as h:
        qs.qs_set_basis_state(h, 7)
        st = qs.qs_get_state(h).reshape(2, -1)
        assert st[:, 7].tolist() == [1, 1] and np.count_nonzero(st) == 2
        qs.qs_set_basis_states(h, [3, 9])
        qs.qs_apply_gate(h, (0,), ogates.hadamard())
        st = qs.qs_get_state(h).reshape(2, -1)
        np.testing.assert_allclose(st[0], osv.apply_gate(osv.basis_state(n, 3), n, (0,), ogates.hadamard()), atol=1e-15)
        np.testing.assert_allclose(st[1], osv.apply_gate(osv.basis_state(n, 9), n, (0,), ogates.hadamard()), atol=1e-15)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n,seed", [(10, 1), (13, 2), (14, 3), (16, 4)])
def test_random_circuits_through_the_planner_match_oracle(dtype, n, seed):
    """Random noisy H / controlled phases / flips: windows, segments and the
    commutation checks of the planner against the plain gate-by-gate oracle."""
    rng = np.random.default_rng(seed)
    ops = []
    for _ in range(120):
        r = rng.random()
        if r < 0.45:
            ops.append(inputs.Op("H", (int(rng.integers(n)),), noisy=bool(rng.random() < 0.8)))
        elif r < 0.93:
            j, k = rng.choice(n, size=2, replace=False)
            ops.append(inputs.Op("CP", (int(j), int(k)), theta=float(rng.uniform(0, 6)), noisy=bool(rng.random() < 0.8)))
        else:
            ops.append(inputs.Op("FLIP", index=int(rng.integers(1 << n))))
    batch, e, x0 = 3, 0.07, int(rng.integers(1 << n))
    with Handle(n, batch, 0, qs.QS_STATEVEC, dtype) as h:
        qs.qs_set_basis_state(h, x0)
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        qs.qs_plan_run(p, e, SEED, 11, h)
        qs.qs_plan_destroy(p)
        got = qs.qs_get_state(h).reshape(batch, -1)
    for b in range(batch):
        psi = osv.basis_state(n, x0)
        for g, op in enumerate(ops):
            if op.kind == "FLIP":
                psi = osv.phase_flip(psi, op.index)
                continue
            U = ocirc.op_unitary(op)
            if op.noisy:
                xa, xb = ophilox.normal_pair(SEED, b, 11 + g)
                U = ogates.noisy_unitary(U, ocirc.op_noise(op), e, xa, xb)
            psi = osv.apply_gate(psi, n, ocirc.op_targets(op), U)
        assert_amplitudes_close(got[b], psi, dtype, k=4.0)


def _ry(theta):
    c, s_ = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -s_], [s_, c]], dtype=np.complex128)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("case", ["bit_flips", "noisy_flips", "near_pi", "strong_noise_h"])
def test_real_gates_with_small_pivots_match_oracle(dtype, case):
    """Real one-qubit gates whose M00 is small or zero (a bit flip, a rotation
    by nearly pi, rotation noise large enough to turn a Hadamard into one)
    through the fused passes, against the gate-by-gate oracle: the factored
    form must pivot instead of dividing by the small entry."""
    rng = np.random.default_rng({"bit_flips": 21, "noisy_flips": 22, "near_pi": 23, "strong_noise_h": 24}[case])
    n, batch = 13, 3
    X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    e = {"bit_flips": 0.03, "noisy_flips": 0.05, "near_pi": 0.03, "strong_noise_h": 0.25}[case]
    gates = []
    for _ in range(80):
        r = rng.random()
        q = int(rng.integers(n))
        if r < 0.35:
            gates.append(qs.make_gate((q,), ogates.hadamard(), noisy=True))
        elif r < 0.55:
            j, k = rng.choice(n, size=2, replace=False)
            gates.append(qs.make_gate((int(j), int(k)), ogates.controlled_phase(float(rng.uniform(0, 6))),
                                      noisy=True, noise=qs.QS_NOISE_PHASE))
        elif case == "bit_flips":
            gates.append(qs.make_gate((q,), X))
        elif case == "noisy_flips":
            gates.append(qs.make_gate((q,), X, noisy=True))
        elif case == "near_pi":
            gates.append(qs.make_gate((q,), _ry(math.pi - 1e-3 * (1 + rng.random()))))
        else:
            gates.append(qs.make_gate((q,), ogates.hadamard(), noisy=True))
    x0 = int(rng.integers(1 << n))
    with Handle(n, batch, 0, qs.QS_STATEVEC, dtype) as h:
        qs.qs_set_basis_state(h, x0)
        p = qs.qs_plan_create(h, gates)
        passes, _ = qs.qs_plan_info(p, h)
        qs.qs_plan_run(p, e, SEED, 7, h)
        qs.qs_plan_destroy(p)
        got = qs.qs_get_state(h).reshape(batch, -1)
    assert passes < len(gates)                                  # the gates ran fused
    for b in range(batch):
        psi = osv.basis_state(n, x0)
        for g, gate in enumerate(gates):
            d = 1 << gate.k
            U = np.array(gate.U[:2 * d * d]).view(np.complex128).reshape(d, d)
            if gate.noisy:
                xa, xb = ophilox.normal_pair(SEED, b, 7 + g)
                U = ogates.noisy_unitary(U, "phase" if gate.noise == qs.QS_NOISE_PHASE else "rotation", e, xa, xb)
            psi = osv.apply_gate(psi, n, tuple(gate.targets[:gate.k]), U)
        assert_amplitudes_close(got[b], psi, dtype, k=4.0, err_msg=f"{case} member {b}")


def test_plan_with_unfusable_gates_matches_oracle():
    rng = np.random.default_rng(9)
    n, batch, e = 11, 2, 0.03
    U2 = rand_unitary(rng, 4)
    gates = [qs.make_gate((q,), ogates.hadamard(), noisy=True) for q in range(n)]
    gates.append(qs.make_gate((3, 9), U2))                     # dense 2-qubit: single step
    gates += [qs.make_gate((q,), ogates.hadamard(), noisy=True) for q in (0, 10, 5)]
    gates.append(qs.make_gate((10, 2), ogates.controlled_phase(0.4), noisy=True, noise=qs.QS_NOISE_PHASE))
    with Handle(n, batch, 0, qs.QS_STATEVEC, qs.QS_C128) as h:
        p = qs.qs_plan_create(h, gates)
        qs.qs_plan_run(p, e, SEED, 100, h)
        qs.qs_plan_destroy(p)
        got = qs.qs_get_state(h).reshape(batch, -1)
    for b in range(batch):
        psi = osv.basis_state(n, 0)
        for g, gate in enumerate(gates):
            d = 1 << gate.k
            U = np.array(gate.U[:2 * d * d]).view(np.complex128).reshape(d, d)
            t = tuple(gate.targets[:gate.k])
            if gate.noisy:
                xa, xb = ophilox.normal_pair(SEED, b, 100 + g)
                U = ogates.noisy_unitary(U, "phase" if gate.noise == qs.QS_NOISE_PHASE else "rotation", e, xa, xb)
            psi = osv.apply_gate(psi, n, t, U)
        np.testing.assert_allclose(got[b], psi, atol=1e-12)


def test_qft_full_size_sampled_trajectories():
    """The benchmark shape: n = 20, 1024 complex64 trajectories, fused plan."""
    n, T, e = 20, 1024, 0.01
    ops, x0 = inputs.qft_circuit(n), inputs.draw_basis_input(n, SEED)
    with Handle(n, T, 0, qs.QS_STATEVEC, qs.QS_C64) as h:
        ref = pcirc.ideal_reference(n, ops, x0, qs.QS_C64)
        try:
            qs.qs_set_reference_from(h, ref, 0)
        finally:
            qs.qs_destroy(ref)
        qs.qs_set_basis_state(h, x0)
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        qs.qs_plan_run(p, e, SEED, 0, h)
        f = qs.qs_fidelity_stored(h)
        norms = qs.qs_trace(h)
        sampled = (0, 513, T - 1)
        states = {b: qs.qs_get_state_range(h, b << n, 1 << n) for b in sampled}
        qs.qs_plan_destroy(p)
    np.testing.assert_allclose(norms, 1.0, atol=1e-5)
    ideal = ocirc.ideal_state(n, ops, x0)
    for b in sampled:
        psi = oracle_traj(n, ops, x0, e, b)
        # every amplitude of the trajectory, element by element
        assert_amplitudes_close(states[b], psi, qs.QS_C64, err_msg=f"trajectory {b}")
        want = osv.fidelity(ideal, psi)
        assert abs(f[b] - want) < 1e-5, (b, f[b], want)
    # distribution sanity against Eq. 11 (lower estimate) and 1
    assert np.all(f <= 1 + 1e-5)
    assert f.mean() > ogates.qft_estimate_eq11(n, e) - 0.01


# ----------------------------------------------------------------- density matrix

@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("circ", ["qft", "grover"])
def test_density_circuit_matches_oracle(dtype, circ):
    n, e = 4, 0.05
    ops = inputs.qft_circuit(n) if circ == "qft" else inputs.grover_circuit(n, 3, 11)
    x0 = 9 if circ == "qft" else 0
    with Handle(n, 1, 0, qs.QS_DENSITY, dtype) as h:
        qs.qs_set_basis_state(h, x0)
        pcirc.apply_ops(h, ops, e, SEED)
        got = qs.qs_get_state(h).reshape(1 << n, 1 << n)
        ideal = ocirc.ideal_state(n, ops, x0)
        f = qs.qs_fidelity(h, ideal)[0]
        tr = qs.qs_trace(h)[0]
    rho = ocirc.run_density(n, ops, x0, e)
    np.testing.assert_allclose(got, rho, atol=TOL[dtype])
    assert abs(f - odm.fidelity(ideal, rho)) <= TOL[dtype] * max(1.0, f)
    assert abs(tr - 1.0) <= TOL[dtype]


def test_density_custom_kraus_matches_oracle():
    rng = np.random.default_rng(12)
    n = 3
    # a random CPTP map from an isometry (4 operators of size 4x4)
    V = np.linalg.qr(rng.normal(size=(16, 4)) + 1j * rng.normal(size=(16, 4)))[0]
    ks = [V[4 * i:4 * i + 4, :] for i in range(4)]
    rho0 = np.zeros((8, 8), complex)
    rho0[5, 5] = 1
    rho0 = odm.apply_unitary(rho0, n, (0,), ogates.hadamard())
    with Handle(n, 1, 0, qs.QS_DENSITY, qs.QS_C128) as h:
        qs.qs_set_state(h, rho0.reshape(-1))
        qs.qs_apply_kraus(h, (2, 0), ks)
        got = qs.qs_get_state(h).reshape(8, 8)
    np.testing.assert_allclose(got, odm.apply_channel(rho0, n, (2, 0), ks), atol=1e-12)


# ----------------------------------------------------------------- fixed rank

@pytest.mark.parametrize("n,e", [(5, 0.05), (6, 0.01), (8, 0.02)])
def test_rank1_grover_reproduces_eq10(n, e):
    k = inputs.grover_iterations(n)
    w = inputs.draw_marked(n, SEED)
    ops = inputs.grover_circuit(n, k, w)
    with Handle(n, 1, 1, qs.QS_FIXED_RANK, qs.QS_C128) as h:
        pcirc.apply_ops(h, ops, e, SEED)
        p = qs.qs_fidelity(h, None, w)[0]
    want = ogates.grover_rank1_success(n, k, e)
    assert abs(p - want) <= 1e-12 * want
    with Handle(n, 1, 1, qs.QS_FIXED_RANK, qs.QS_C128) as h:
        qs.qs_set_normalize(h, 1)
        pcirc.apply_ops(h, ops, e, SEED)
        p = qs.qs_fidelity(h, None, w)[0]
    assert abs(p - ogates.grover_ideal_success(n, k)) <= 1e-12


@pytest.mark.parametrize("circ,n,r,normalize", [("grover", 5, 2, 0), ("grover", 5, 4, 0), ("grover", 6, 3, 1),
                                                ("qft", 5, 2, 0), ("qft", 5, 4, 1), ("qft", 4, 16, 0)])
def test_fixed_rank_matches_oracle(circ, n, r, normalize):
    e = 0.05
    if circ == "qft":
        ops, x0 = inputs.qft_circuit(n), 5
    else:
        ops, x0 = inputs.grover_circuit(n, inputs.grover_iterations(n), 6), 0
    ideal = ocirc.ideal_state(n, ops, x0)
    with Handle(n, 1, r, qs.QS_FIXED_RANK, qs.QS_C128) as h:
        qs.qs_set_normalize(h, normalize)
        qs.qs_set_basis_state(h, x0)
        pcirc.apply_ops(h, ops, e, SEED)
        f = qs.qs_fidelity(h, ideal)[0]
        tr = qs.qs_trace(h)[0]
        m = qs.qs_get_rank(h)
        L = qs.qs_get_state(h).reshape(r, 1 << n)[:m].T
    Lo = ocirc.run_fixed_rank(n, ops, x0, e, r, normalize=bool(normalize))
    assert m == Lo.shape[1]
    np.testing.assert_allclose(L @ L.conj().T, Lo @ Lo.conj().T, atol=1e-12)
    fo = ofr.fidelity(ideal, Lo)
    assert abs(f - fo) <= 1e-12 * max(fo, 1e-300)
    assert abs(tr - ofr.trace(Lo)) <= 1e-12
    if r >= (1 << n):
        rho = ocirc.run_density(n, ops, x0, e)
        np.testing.assert_allclose(L @ L.conj().T, rho, atol=1e-12)


@pytest.mark.parametrize("r", [2, 4, 8])
def test_fixed_rank_grover_n16_prefix_matches_oracle(r):
    """The configuration of the fixed-rank workload (Grover, n = 16, e = 0.01,
    Sec. 3.2) over its first 304 channels (the start and nine iterations):
    at 2^16 rows the Gram reduction sums more partial blocks per thread than
    any smaller test reaches.  Fidelity, trace and L L^dagger on sampled rows
    against the oracle on the same prefix."""
    n, e = 16, 0.01
    w = inputs.draw_marked(n, SEED)
    ops = inputs.grover_circuit(n, inputs.grover_iterations(n), w)
    prefix = ops[:16 + 9 * (2 * n + 2)]
    assert sum(1 for o in prefix if o.noisy) == 304
    ideal = ocirc.ideal_state(n, prefix, 0)
    with Handle(n, 1, r, qs.QS_FIXED_RANK, qs.QS_C128) as h:
        qs.qs_set_basis_state(h, 0)
        pcirc.apply_ops(h, prefix, e, SEED)
        f = qs.qs_fidelity(h, ideal)[0]
        tr = qs.qs_trace(h)[0]
        m = qs.qs_get_rank(h)
        L = qs.qs_get_state(h).reshape(r, 1 << n)[:m].T
    Lo = ocirc.run_fixed_rank(n, prefix, 0, e, r)
    assert m == Lo.shape[1]
    fo, to = ofr.fidelity(ideal, Lo), ofr.trace(Lo)
    assert abs(f - fo) <= 1e-12 * fo, (f, fo)
    assert abs(tr - to) <= 1e-12 * to, (tr, to)
    rows = np.sort(np.random.default_rng(r).choice(1 << n, size=96, replace=False))
    rows = np.union1d(rows, [0, w, (1 << n) - 1])
    got, want = L[rows] @ L[rows].conj().T, Lo[rows] @ Lo[rows].conj().T
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("circ", ["grover", "qft"])
def test_batched_fixed_rank_members_equal_separate_runs_and_oracle(circ):
    """Members of uneven rank and noise in one FIXED_RANK handle (one launch
    per kernel for all of them, Sec. 3.2 per member): each member equals the
    same job run alone, bit for bit, and the oracle."""
    n = 9
    ranks = [1, 2, 4, 8, 3]
    es = [0.01, 0.03, 0.0, 0.05, 0.02]
    B = len(ranks)
    if circ == "qft":
        ops, x0 = inputs.qft_circuit(n), 5
    else:
        ops, x0 = inputs.grover_circuit(n, 3, 77), 0
    gates_ops = ops
    ideal = ocirc.ideal_state(n, ops, x0)
    with Handle(n, B, max(ranks), qs.QS_FIXED_RANK, qs.QS_C128) as h:
        qs.qs_set_member_ranks(h, ranks)
        qs.qs_set_member_noise(h, es, [SEED] * B, list(range(B)))
        qs.qs_set_basis_state(h, x0)
        pcirc.apply_ops(h, gates_ops, 0.5, SEED)            # the call's e is overridden per member
        f = qs.qs_fidelity(h, ideal)
        tr = qs.qs_trace(h)
        cols = qs.qs_get_member_columns(h)
        st = qs.qs_get_state(h).reshape(B, max(ranks), 1 << n)
    for b in range(B):
        with Handle(n, 1, ranks[b], qs.QS_FIXED_RANK, qs.QS_C128) as h1:
            qs.qs_set_basis_state(h1, x0)
            pcirc.apply_ops(h1, gates_ops, es[b], SEED)
            f1 = qs.qs_fidelity(h1, ideal)[0]
            m1 = qs.qs_get_rank(h1)
            L1 = qs.qs_get_state(h1).reshape(ranks[b], 1 << n)
        assert cols[b] == m1
        assert f[b] == f1, (b, f[b], f1)                      # bit-identical to the job alone
        np.testing.assert_array_equal(st[b, :m1], L1[:m1])
        assert not np.any(st[b, m1:])                          # dead columns stay zero
        Lo = ocirc.run_fixed_rank(n, ops, x0, es[b], ranks[b])
        fo = ofr.fidelity(ideal, Lo)
        assert abs(f[b] - fo) <= 1e-12 * fo, (b, f[b], fo)
        assert abs(tr[b] - ofr.trace(Lo)) <= 1e-12
        L = st[b, :m1].T
        np.testing.assert_allclose(L @ L.conj().T, Lo @ Lo.conj().T, atol=1e-12)


@pytest.mark.parametrize("circ,batch", [("grover", 1), ("qft", 1), ("grover", 4), ("qft", 3)])
def test_fixed_rank_plan_equals_gate_by_gate(circ, batch):
    """A FIXED_RANK plan (every gate on every member, the circuit replayed as
    one CUDA graph, Kraus sets built on the device from e) equals the same
    gates issued one by one, bit for bit, twice in a row; the members' column
    counts on the host follow."""
    n, e = 9, 0.03
    ranks = [8, 2, 5, 1][:batch]
    if circ == "qft":
        ops, x0 = inputs.qft_circuit(n), 6
    else:
        ops, x0 = inputs.grover_circuit(n, 3, 101), 0
    es = [0.03, 0.01, 0.0, 0.05][:batch]
    ideal = ocirc.ideal_state(n, ops, x0)
    results = []
    for use_plan in (False, True):
        with Handle(n, batch, max(ranks), qs.QS_FIXED_RANK, qs.QS_C128) as h:
            qs.qs_set_member_ranks(h, ranks)
            if batch > 1:
                qs.qs_set_member_noise(h, es, [SEED] * batch, list(range(batch)))
            p = qs.qs_plan_create(h, pcirc.to_gates(ops)) if use_plan else None
            runs = []
            for _ in range(2):
                qs.qs_set_basis_state(h, x0)
                if use_plan:
                    qs.qs_plan_run(p, e, SEED, 0, h)
                else:
                    pcirc.apply_ops(h, ops, e, SEED)
                runs.append((qs.qs_fidelity(h, ideal), qs.qs_get_state(h), qs.qs_get_member_columns(h)))
            if p is not None:
                qs.qs_plan_destroy(p)
        results.append(runs)
    for (fa, sa, ca), (fb, sb, cb) in zip(results[0], results[1]):
        np.testing.assert_array_equal(fa, fb)
        np.testing.assert_array_equal(sa, sb)
        np.testing.assert_array_equal(ca, cb)
    # and the plan against the oracle
    f = results[1][1][0]
    for b in range(batch):
        Lo = ocirc.run_fixed_rank(n, ops, x0, es[b] if batch > 1 else e, ranks[b])
        fo = ofr.fidelity(ideal, Lo)
        assert abs(f[b] - fo) <= 1e-12 * fo, (b, f[b], fo)


def test_explicit_truncation_matches_oracle():
    rng = np.random.default_rng(2)
    n, r = 6, 6
    L0 = rng.normal(size=(1 << n, r)) + 1j * rng.normal(size=(1 << n, r))
    with Handle(n, 1, r, qs.QS_FIXED_RANK, qs.QS_C128) as h:
        qs.qs_set_state(h, L0.T.reshape(-1))
        qs.qs_set_rank_columns(h, r)
        qs.qs_truncate_rank(h, 3, 0)
        assert qs.qs_get_rank(h) == 3
        L = qs.qs_get_state(h).reshape(r, 1 << n)[:3].T
        rest = qs.qs_get_state(h).reshape(r, 1 << n)[3:]
    Lo, _ = ofr.truncate(L0, 3)
    np.testing.assert_allclose(L @ L.conj().T, Lo @ Lo.conj().T, atol=1e-11)
    assert np.all(rest == 0)


# ----------------------------------------------------------------- batching, errors

def test_member_noise_equals_separate_runs():
    n, e_list = 11, [0.01, 0.03, 0.0, 0.05]
    seeds = [11, 22, 33, 44]
    trajs = [5, 0, 9, 2]
    ops = inputs.qft_circuit(n)
    gates = pcirc.to_gates(ops)
    with Handle(n, 4, 0, qs.QS_STATEVEC, qs.QS_C128) as h:
        qs.qs_set_member_noise(h, e_list, seeds, trajs)
        qs.qs_set_basis_state(h, 3)
        p = qs.qs_plan_create(h, gates)
        qs.qs_plan_run(p, 0.5, 999, 0, h)        # call values are overridden per member
        qs.qs_plan_destroy(p)
        mixed = qs.qs_get_state(h).reshape(4, -1)
    for b in range(4):
        with Handle(n, 1, 0, qs.QS_STATEVEC, qs.QS_C128) as h1:
            qs.qs_set_trajectory_offset(h1, trajs[b])
            qs.qs_set_basis_state(h1, 3)
            p = qs.qs_plan_create(h1, gates)
            qs.qs_plan_run(p, e_list[b], seeds[b], 0, h1)
            qs.qs_plan_destroy(p)
            alone = qs.qs_get_state(h1)
        np.testing.assert_allclose(mixed[b], alone, atol=1e-13)


@pytest.mark.parametrize("dtype", DTYPES)
def test_clearing_member_noise_restores_the_call_arguments(dtype):
    """Per-member noise overrides a run's e and seed until it is cleared; after
    qs_set_member_noise(h, NULL, ...) the next run draws with the call's own e."""
    n, batch = 12, 3
    ops = inputs.qft_circuit(n)
    x0 = inputs.draw_basis_input(n, SEED)
    with Handle(n, batch, 0, qs.QS_STATEVEC, dtype) as h:
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        qs.qs_set_member_noise(h, [0.2] * batch, [SEED] * batch, list(range(batch)))
        qs.qs_set_basis_state(h, x0)
        qs.qs_plan_run(p, 0.001, SEED, 0, h)               # the members' e = 0.2 wins
        noisy = qs.qs_get_state(h).reshape(batch, -1)
        qs.qs_set_member_noise(h)                           # cleared
        qs.qs_set_basis_state(h, x0)
        qs.qs_plan_run(p, 0.001, SEED, 0, h)               # the call's e again
        quiet = qs.qs_get_state(h).reshape(batch, -1)
        qs.qs_plan_destroy(p)
    for b in range(batch):
        assert_amplitudes_close(noisy[b], ocirc.run_trajectory(n, ops, x0, 0.2, SEED, b), dtype)
        assert_amplitudes_close(quiet[b], ocirc.run_trajectory(n, ops, x0, 0.001, SEED, b), dtype)


def test_invalid_arguments_are_rejected():
    with Handle(5, 2, 0, qs.QS_STATEVEC, qs.QS_C128) as h:
        for bad in [lambda: qs.qs_apply_gate(h, (5,), np.eye(2)),
                    lambda: qs.qs_apply_gate(h, (1, 1), np.eye(4)),
                    lambda: qs.qs_apply_phase_flip(h, 32),
                    lambda: qs.qs_set_basis_state(h, 1 << 5),
                    lambda: qs.qs_apply_noisy_gate(h, (0,), np.eye(2), 0, -1.0, 1, 1),
                    lambda: qs.qs_apply_noisy_gate(h, (0, 1, 2), np.eye(8), 0, 0.1, 1, 1)]:
            with pytest.raises(qs.QSError) as ei:
                bad()
            assert ei.value.status == qs.QS_ERR_INVALID_ARG
        with pytest.raises(qs.QSError) as ei:
            qs.qs_apply_kraus(h, (0,), [np.eye(2)])
        assert ei.value.status == qs.QS_ERR_NOT_SUPPORTED
    with Handle(3, 1, 0, qs.QS_DENSITY, qs.QS_C128) as h:
        with pytest.raises(qs.QSError) as ei:
            qs.qs_apply_kraus(h, (0,), [np.eye(2), np.eye(2)])      # not trace preserving
        assert ei.value.status == qs.QS_ERR_INVALID_ARG
    with pytest.raises(qs.QSError):
        qs.qs_create(0, 1, 0, qs.QS_STATEVEC, qs.QS_C64)
    with pytest.raises(qs.QSError):
        qs.qs_create(4, 2, 0, qs.QS_DENSITY, qs.QS_C64)


def test_smallest_sizes():
    # one qubit, one member; ragged sizes below one tile
    with Handle(1, 1, 0, qs.QS_STATEVEC, qs.QS_C128) as h:
        qs.qs_apply_gate(h, (0,), ogates.hadamard())
        np.testing.assert_allclose(qs.qs_get_state(h), [2 ** -0.5, 2 ** -0.5], atol=1e-15)
        assert abs(qs.qs_fidelity(h, None, 1)[0] - 0.5) < 1e-15
    with Handle(3, 7, 0, qs.QS_STATEVEC, qs.QS_C64) as h:
        qs.qs_apply_gate(h, (2,), ogates.hadamard())
        np.testing.assert_allclose(qs.qs_trace(h), 1.0, atol=1e-6)


@pytest.mark.parametrize("circ,n,batch", [("qft", 18, 32), ("grover", 16, 64)])
def test_every_kernel_configuration_gives_the_same_result(circ, n, batch):
    """Each pass configuration (tile buffers, warps, blocks per SM) at sizes
    where every warp or block streams several tiles, with a created start
    state and the fused fidelity; sampled members against the oracle."""
    e = 0.02
    if circ == "qft":
        ops, xs = inputs.qft_circuit(n), [(97 * b + 11) % (1 << n) for b in range(batch)]
    else:
        ops, xs = inputs.grover_circuit(n, 3, 12345 % (1 << n)), [0] * batch
    ideal0 = ocirc.ideal_state(n, ops, xs[0])
    results = {}
    with Handle(n, batch, 0, qs.QS_STATEVEC, qs.QS_C64) as h:
        qs.qs_set_reference(h, np.asarray(ideal0))
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        nl, nh = qs.qs_plan_configs(p, h)
        assert (nl, nh) == (3, 3)
        for lc in range(nl):
            for hc in range(nh):
                qs.qs_plan_set_config(p, lc, hc, h)
                assert qs.qs_plan_get_config(p, h) == (lc, hc)
                qs.qs_set_basis_states(h, xs)
                f = qs.qs_plan_run_fidelity(p, e, SEED, 0, h)
                results[(lc, hc)] = (f, qs.qs_get_state(h).reshape(batch, -1))
        with pytest.raises(qs.QSError):
            qs.qs_plan_set_config(p, 3, 0, h)
        with pytest.raises(qs.QSError):
            qs.qs_plan_set_config(p, 0, 3, h)
        qs.qs_plan_destroy(p)
    f0, s0 = results[(0, 0)]
    for key, (f, st) in results.items():
        np.testing.assert_allclose(st, s0, atol=1e-6, err_msg=str(key))
        np.testing.assert_allclose(f, f0, atol=1e-6, err_msg=str(key))
    for b in (0, batch - 1):
        want = oracle_traj(n, ops, xs[b], e, b)
        assert_amplitudes_close(s0[b], want, qs.QS_C64)
        assert abs(f0[b] - osv.fidelity(ideal0, want)) <= 1e-5


def test_autotune_picks_a_configuration_and_results_stay_correct():
    n, batch, e = 16, 32, 0.01
    ops = inputs.qft_circuit(n)
    with Handle(n, batch, 0, qs.QS_STATEVEC, qs.QS_C64) as h:
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        qs.qs_set_basis_state(h, 3)
        lo, hi = qs.qs_plan_autotune(p, 2, e, SEED, h)
        assert lo > 0 and hi > 0
        cfg = qs.qs_plan_get_config(p, h)
        assert 0 <= cfg[0] < 3 and 0 <= cfg[1] < 3
        qs.qs_set_basis_state(h, 3)
        qs.qs_plan_run(p, e, SEED, 0, h)
        got = qs.qs_get_state(h).reshape(batch, -1)
        qs.qs_plan_destroy(p)
    assert_amplitudes_close(got[1], oracle_traj(n, ops, 3, e, 1), qs.QS_C64)
    with Handle(n, 2, 0, qs.QS_STATEVEC, qs.QS_C128) as h:
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        assert qs.qs_plan_configs(p, h) == (1, 1)
        qs.qs_plan_autotune(p, 1, e, SEED, h)
        assert qs.qs_plan_get_config(p, h) == (0, 0)
        qs.qs_plan_destroy(p)


@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_density_hermitian_sweeps_match_oracle(dtype):
    # a Hermitian start (basis state): channels on qubits >= 5 and the
    # diagonal blocks run on the upper tiles and mirror them (several tiles
    # per dimension at n = 9); against the oracle and a non-Hermitian start
    # that takes the full sweeps (the same state plus an antihermitian part
    # that every operation here maps linearly)
    n, e, x0 = 9, 0.05, 300
    ops = inputs.qft_circuit(n)
    tol = 1e-12 if dtype == qs.QS_C128 else 1e-5 * 2.0 ** (-n)    # entries are of order 2^-n
    with Handle(n, 1, 0, qs.QS_DENSITY, dtype) as h:
        qs.qs_set_basis_state(h, x0)
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        qs.qs_plan_run(p, e, SEED, 0, h)
        qs.qs_plan_destroy(p)
        got = qs.qs_get_state(h).reshape(1 << n, 1 << n)
    rho = ocirc.run_density(n, ops, x0, e)
    assert np.abs(got - rho).max() < tol
    assert np.abs(got - got.conj().T).max() < tol * 1e-2     # Hermitian (to rounding of the full sweeps)
    # the full sweeps on a matrix that is not Hermitian: linear in the input
    rng = np.random.default_rng(8)
    A = (rng.normal(size=(1 << n, 1 << n)) + 1j * rng.normal(size=(1 << n, 1 << n))) / (1 << n)
    start = osv.basis_state(n, x0)
    start = np.outer(start, start.conj()) + A
    with Handle(n, 1, 0, qs.QS_DENSITY, dtype) as h:
        qs.qs_set_state(h, start.ravel())
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        qs.qs_plan_run(p, e, SEED, 0, h)
        qs.qs_plan_destroy(p)
        got2 = qs.qs_get_state(h).reshape(1 << n, 1 << n)
    want2 = start
    for op in ops:
        U = ocirc.op_unitary(op)
        kr = ogates.kraus_set(U, ocirc.op_noise(op), e) if op.noisy else [U]
        want2 = odm.apply_channel(want2, n, ocirc.op_targets(op), kr)
    assert np.abs(got2 - want2).max() < tol * 10


def test_plan_timing_with_single_steps():
    # a density plan (channels as single steps, diagonal blocks) timed per
    # launch: kinds and counts match the plan, the state is unchanged by timing
    n, e = 7, 0.05
    ops = inputs.qft_circuit(n)
    states = []
    for timing in (False, True):
        with Handle(n, 1, 0, qs.QS_DENSITY, qs.QS_C128) as h:
            qs.qs_set_basis_state(h, 3)
            p = qs.qs_plan_create(h, pcirc.to_gates(ops))
            qs.qs_plan_set_timing(p, timing, h)
            qs.qs_plan_run(p, e, SEED, 0, h)
            if timing:
                ms, kinds = qs.qs_plan_last_times(p, h=h)
                _, launches = qs.qs_plan_info(p, h)
                assert len(ms) == launches and all(m >= 0 for m in ms)
                assert kinds.count("single_gate") == n and kinds.count("dm_diag_block") == n - 1
            qs.qs_plan_destroy(p)
            states.append(qs.qs_get_state(h))
    np.testing.assert_array_equal(states[0], states[1])


@pytest.mark.parametrize("circ,n", [("qft", 6), ("qft", 7), ("grover", 5)])
@pytest.mark.parametrize("dtype", [qs.QS_C128, qs.QS_C64])
def test_density_plan_with_diagonal_blocks_matches_oracle(circ, n, dtype):
    """Plans on density matrices run each run of diagonal channels (noisy
    controlled phases, flips) as one sweep; the result equals the oracle and
    the gate-by-gate channels."""
    e = 0.05
    if circ == "qft":
        ops, x0 = inputs.qft_circuit(n), 5
    else:
        ops, x0 = inputs.grover_circuit(n, 2, 6), 0
    with Handle(n, 1, 0, qs.QS_DENSITY, dtype) as h:
        qs.qs_set_basis_state(h, x0)
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        qs.qs_plan_run(p, e, SEED, 0, h)
        planned = qs.qs_get_state(h)
        # the same plan again from the start: the blocks are reusable
        qs.qs_set_basis_state(h, x0)
        qs.qs_plan_run(p, e, SEED, 0, h)
        again = qs.qs_get_state(h)
        qs.qs_plan_destroy(p)
    with Handle(n, 1, 0, qs.QS_DENSITY, dtype) as h:
        qs.qs_set_basis_state(h, x0)
        pcirc.apply_ops(h, ops, e, SEED)
        single = qs.qs_get_state(h)
    rho = ocirc.run_density(n, ops, x0, e)
    tol = 1e-12 if dtype == qs.QS_C128 else 1e-6      # complex64: FP32 channels and diagonal blocks
    np.testing.assert_allclose(planned, rho.ravel(), atol=tol)
    np.testing.assert_allclose(planned, single, atol=tol / 10)
    np.testing.assert_array_equal(again, planned)
