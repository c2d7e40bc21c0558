"""Dense k-qubit blocks, k = 3..5 (the k-qubit update of Sec. 2), through the
C ABI against the oracle: the complex64 tensor-core path (tcgen05, split tf32
operands) and the CUDA-core sweeps, on batches of members, density matrices,
ragged and exact-fit tile counts, and the overlap of a full-size batch."""
import numpy as np
import pytest

from oracle import density as odens
from oracle import statevec
from paper_1412_2293_gb300 import qs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def library():
    from paper_1412_2293_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return qs.lib()


def rand_unitary(rng, d):
    q, r = np.linalg.qr(rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d)))
    return q * (np.diag(r) / np.abs(np.diag(r)))


def rand_states(rng, members, n):
    v = rng.normal(size=(members, 1 << n)) + 1j * rng.normal(size=(members, 1 << n))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def run(n, members, targets, U, psi, dtype, tensor=True):
    h = qs.qs_create(n, members, 0, qs.QS_STATEVEC, dtype)
    try:
        qs.qs_set_tensor_cores(h, tensor)
        qs.qs_set_state(h, psi.ravel())
        qs.qs_apply_gate(h, targets, U)
        return qs.qs_get_state(h).reshape(members, -1)
    finally:
        qs.qs_destroy(h)


def bound(U, psi):
    # FP32 error scale of one output amplitude: sum_j |U_ij| |psi_j|
    return np.abs(U).sum(axis=1).max() * np.abs(psi).max()


CASES = [
    (10, 3, (9, 2, 5), 3),            # scattered targets, three members, one tile each
    (12, 5, (0, 1, 2, 3, 4), 2),      # the low bits: a group is 32 consecutive amplitudes
    (12, 5, (11, 3, 7, 0, 5), 1),     # scattered, top bit included
    (13, 4, (4, 5, 6, 7), 5),         # contiguous middle range, odd member count
    (14, 5, (13, 12, 11, 10, 9), 2),  # the high bits: groups far apart
    (8, 3, (0, 7, 3), 1),             # n - k < 7: the CUDA-core sweep
]


@pytest.mark.parametrize("n,k,targets,members", CASES)
@pytest.mark.parametrize("tensor", [True, False])
def test_dense_block_c64(n, k, targets, members, tensor):
    rng = np.random.default_rng(n * 31 + k)
    U = rand_unitary(rng, 1 << k)
    psi = rand_states(rng, members, n)
    got = run(n, members, targets, U, psi, qs.QS_C64, tensor)
    want = np.stack([statevec.apply_gate(p, n, targets, U) for p in psi])
    assert np.abs(got - want).max() < 4e-6 * bound(U, psi)


@pytest.mark.parametrize("k,targets", [(3, (1, 6, 4)), (4, (0, 9, 2, 5)), (5, (10, 0, 4, 7, 2))])
def test_dense_block_c128(k, targets):
    n, members = 11, 2
    rng = np.random.default_rng(70 + k)
    U = rand_unitary(rng, 1 << k)
    psi = rand_states(rng, members, n)
    got = run(n, members, targets, U, psi, qs.QS_C128)
    want = np.stack([statevec.apply_gate(p, n, targets, U) for p in psi])
    assert np.abs(got - want).max() < 1e-14


def test_tensor_and_cuda_core_paths_agree():
    n, members, targets = 13, 4, (2, 8, 5, 11, 0)
    rng = np.random.default_rng(5)
    U = rand_unitary(rng, 32)
    psi = rand_states(rng, members, n)
    a = run(n, members, targets, U, psi, qs.QS_C64, True)
    b = run(n, members, targets, U, psi, qs.QS_C64, False)
    assert np.abs(a - b).max() < 8e-6 * bound(U, psi)
    # different arithmetic (split tf32 products vs FP32 multiply-adds): not bit-identical
    assert np.abs(a - b).max() > 0


@pytest.mark.parametrize("k,targets", [(3, (4, 17, 9)), (4, (0, 12, 19, 6)), (5, (2, 7, 11, 15, 18))])
def test_many_tiles_per_block(k, targets):
    # 8 members of 2^20 amplitudes: thousands of tiles, so every persistent
    # block streams many of them (the next tile's loads overlap the current
    # one); element by element against the oracle
    n, members = 20, 8
    rng = np.random.default_rng(90 + k)
    U = rand_unitary(rng, 1 << k)
    psi = rand_states(rng, members, n)
    got = run(n, members, targets, U, psi, qs.QS_C64)
    want = np.stack([statevec.apply_gate(p, n, targets, U) for p in psi])
    assert np.abs(got - want).max() < 4e-6 * bound(U, psi)


def test_real_and_permutation_blocks():
    # a Toffoli and a real orthogonal block: exact up to the split's rounding
    n, members = 12, 2
    rng = np.random.default_rng(6)
    T = np.eye(8, dtype=np.complex128)[[0, 1, 2, 7, 4, 5, 6, 3]]
    psi = rand_states(rng, members, n)
    got = run(n, members, (3, 9, 0), T, psi, qs.QS_C64)
    want = np.stack([statevec.apply_gate(p, n, (3, 9, 0), T) for p in psi])
    assert np.abs(got - want).max() < 4e-6 * bound(T, psi)
    O, _ = np.linalg.qr(rng.normal(size=(16, 16)))
    got = run(n, members, (6, 1, 10, 4), O.astype(np.complex128), psi, qs.QS_C64)
    want = np.stack([statevec.apply_gate(p, n, (6, 1, 10, 4), O) for p in psi])
    assert np.abs(got - want).max() < 4e-6 * bound(O, psi)


@pytest.mark.parametrize("k,targets", [(3, (5, 1, 8)), (5, (0, 2, 4, 6, 8))])
def test_density_dense_block_c64(k, targets):
    # rho <- U rho U^dagger on a 9-qubit density matrix: two tensor-core sweeps of the 18-qubit vector
    n = 9
    rng = np.random.default_rng(80 + k)
    A = rng.normal(size=(1 << n, 3)) + 1j * rng.normal(size=(1 << n, 3))
    rho = A @ A.conj().T
    rho /= np.trace(rho)
    U = rand_unitary(rng, 1 << k)
    h = qs.qs_create(n, 1, 0, qs.QS_DENSITY, qs.QS_C64)
    try:
        qs.qs_set_state(h, rho.ravel())
        qs.qs_apply_gate(h, targets, U)
        got = qs.qs_get_state(h).reshape(1 << n, 1 << n)
        tr = float(qs.qs_trace(h)[0])
    finally:
        qs.qs_destroy(h)
    want = odens.apply_unitary(rho, n, targets, U)
    assert np.abs(got - want).max() < 1e-5 * np.abs(want).max() * 8
    assert abs(tr - 1.0) < 1e-5


def test_full_size_batch_overlap():
    # the bench's configuration: n = 20, 1024 complex64 members (8 GiB), k = 5.
    # Start: a product of seeded one-qubit states (built on the device by
    # one-qubit gates); after the block every member's overlap with a fixed
    # vector close to the ideal output must match the host's value.
    n, members, targets = 20, 1024, (3, 9, 14, 17, 19)
    rng = np.random.default_rng(11)
    U = rand_unitary(rng, 32)
    V = [rand_unitary(rng, 2) for _ in range(n)]
    psi0 = np.ones(1, dtype=np.complex128)
    for q in range(n):
        psi0 = np.kron(V[q][:, 0], psi0)
    ideal = statevec.apply_gate(psi0, n, targets, U)
    ref = ideal + 0.3 * rand_states(rng, 1, n)[0]
    ref /= np.linalg.norm(ref)
    want = abs(np.vdot(ref, ideal)) ** 2
    h = qs.qs_create(n, members, 0, qs.QS_STATEVEC, qs.QS_C64)
    try:
        qs.qs_set_basis_state(h, 0)
        for q in range(n):
            qs.qs_apply_gate(h, (q,), V[q])
        qs.qs_apply_gate(h, targets, U)
        f = qs.qs_fidelity(h, ref)
    finally:
        qs.qs_destroy(h)
    assert f.shape == (members,)
    assert np.abs(f - want).max() < 2e-5
    assert f.max() - f.min() < 1e-6          # every member took the same path


def test_k6_rejected():
    h = qs.qs_create(10, 1, 0, qs.QS_STATEVEC, qs.QS_C64)
    try:
        with pytest.raises(qs.QSError) as e:
            qs.qs_apply_gate(h, (0, 1, 2, 3, 4, 5), np.eye(64))
        assert e.value.status == qs.QS_ERR_INVALID_ARG
    finally:
        qs.qs_destroy(h)
