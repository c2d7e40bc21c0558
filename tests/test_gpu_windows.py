"""Fused passes over states of more than 20 qubits, where a window lies below
the top ten qubits: random circuits against the oracle, the QFT against its
closed form (three passes at n = 24 and 28) and the planned noisy QFT
against the gate-by-gate calls."""
import math

import numpy as np
import pytest

from oracle import circuits as ocirc
from oracle import gates as ogates
from oracle import philox as ophilox
from oracle import statevec as osv
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


def qft_closed_form(n, x):
    """QFT of |x> without the final swaps, phases e^{-i theta}:
    amplitude at bitrev(y) = 2^{-n/2} exp(-2 pi i x y / 2^n)."""
    y = np.arange(1 << n, dtype=np.int64)
    rev = np.zeros_like(y)
    for b in range(n):
        rev |= ((y >> b) & 1) << (n - 1 - b)
    out = np.empty(1 << n, dtype=np.complex128)
    out[rev] = 2.0 ** (-n / 2) * np.exp(-2j * np.pi * ((x * y) % (1 << n)) / float(1 << n))
    return out


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("seed", [3, 4])
def test_random_circuit_n21_matches_oracle(dtype, seed):
    n = 21
    rng = np.random.default_rng(seed)
    ops = []
    for _ in range(70):
        r = rng.random()
        if r < 0.5:
            ops.append(inputs.Op("H", (int(rng.integers(n)),), noisy=bool(rng.random() < 0.8)))
        elif r < 0.95:
            j, k = rng.choice(n, size=2, replace=False)
            ops.append(inputs.Op("CP", (int(j), int(k)), theta=float(rng.uniform(0, 6)), noisy=bool(rng.random() < 0.8)))
        else:
            ops.append(inputs.Op("FLIP", index=int(rng.integers(1 << n))))
    batch, e, x0 = 2, 0.05, int(rng.integers(1 << n))
    h = qs.qs_create(n, batch, 0, qs.QS_STATEVEC, dtype)
    try:
        qs.qs_set_basis_state(h, x0)
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        qs.qs_plan_run(p, e, SEED, 5, h)
        qs.qs_plan_destroy(p)
        got = qs.qs_get_state(h).reshape(batch, -1)
    finally:
        qs.qs_destroy(h)
    tol = 1e-12 if dtype == qs.QS_C128 else 2e-5
    for b in range(batch):
        psi = osv.basis_state(n, x0)
        for g, op in enumerate(ops):
            if op.kind == "FLIP":
                psi = osv.phase_flip(psi, op.index)
                continue
            U = ocirc.op_unitary(op)
            if op.noisy:
                xa, xb = ophilox.normal_pair(SEED, b, 5 + g)
                U = ogates.noisy_unitary(U, ocirc.op_noise(op), e, xa, xb)
            psi = osv.apply_gate(psi, n, ocirc.op_targets(op), U)
        assert np.abs(got[b] - psi).max() < tol * max(np.abs(psi).max(), 1e-300) * 50


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_qft_n24_three_passes_closed_form(dtype):
    n, x, batch = 24, 0xA5C3F1, 2
    h = qs.qs_create(n, batch, 0, qs.QS_STATEVEC, dtype)
    try:
        p = qs.qs_plan_create(h, pcirc.to_gates(inputs.qft_circuit(n, noisy=False)))
        passes, _ = qs.qs_plan_info(p, h)
        assert passes == 3
        qs.qs_set_basis_state(h, x)
        qs.qs_plan_run(p, 0.0, SEED, 0, h)
        qs.qs_plan_destroy(p)
        got = qs.qs_get_state(h).reshape(batch, -1)
    finally:
        qs.qs_destroy(h)
    want = qft_closed_form(n, x)
    tol = 1e-13 if dtype == qs.QS_C128 else 2e-5
    for b in range(batch):
        assert np.abs(got[b] - want).max() < tol * 2.0 ** (-n / 2)


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_noisy_qft_n23_plan_equals_gate_by_gate(dtype):
    n, batch, e, x = 23, 3, 0.03, 0x5A5A5A
    ops = inputs.qft_circuit(n)
    a = qs.qs_create(n, batch, 0, qs.QS_STATEVEC, dtype)
    b = qs.qs_create(n, batch, 0, qs.QS_STATEVEC, dtype)
    try:
        qs.qs_set_basis_state(a, x)
        p = qs.qs_plan_create(a, pcirc.to_gates(ops))
        passes, _ = qs.qs_plan_info(p, a)
        assert passes == 3
        qs.qs_plan_run(p, e, SEED, 0, a)
        qs.qs_plan_destroy(p)
        qs.qs_set_basis_state(b, x)
        pcirc.apply_ops(b, ops, e, SEED)
        ga = qs.qs_get_state(a).reshape(batch, -1)
        gb = qs.qs_get_state(b).reshape(batch, -1)
    finally:
        qs.qs_destroy(b)
        qs.qs_destroy(a)
    tol = 1e-12 if dtype == qs.QS_C128 else 2e-5
    assert np.abs(ga - gb).max() < tol * np.abs(gb).max() * 10


def test_qft_n28_three_passes():
    # 2 GiB per member: windows [18, 28), [8, 18) and [0, 10)
    n, x, batch = 28, 0x9E3779B, 2
    h = qs.qs_create(n, batch, 0, qs.QS_STATEVEC, qs.QS_C64)
    try:
        p = qs.qs_plan_create(h, pcirc.to_gates(inputs.qft_circuit(n, noisy=False)))
        passes, _ = qs.qs_plan_info(p, h)
        assert passes == 3
        qs.qs_set_basis_state(h, x)
        qs.qs_plan_run(p, 0.0, SEED, 0, h)
        qs.qs_plan_destroy(p)
        want = qft_closed_form(n, x)
        for y in (0, 12345, (1 << n) - 3):
            f = qs.qs_fidelity(h, None, y)
            assert np.abs(f * 2.0 ** n - 1.0).max() < 1e-4
        ref = want + 0.0
        f = qs.qs_fidelity(h, ref)
        assert np.abs(f - 1.0).max() < 1e-4
    finally:
        qs.qs_destroy(h)


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_out_terms_spanning_both_halves_of_the_out_factor_index(dtype):
    # n = 18: the first dense gate, H(8), puts the first pass on the window
    # [0, 10); its out-factor index holds qubits 10..17, split into 10..15 and
    # 16..17.  The controlled phases at the start act before any gate the pass
    # skips, so it takes those outside the window as out terms: CP(12, 17),
    # CP(10, 16), CP(15, 16) have one qubit in each half, CP(10, 11) and
    # CP(16, 17) lie in one half, CP(3, 16) and CP(5, 14) attach to a window
    # bit.  Later passes take the rest.
    n, batch, e = 18, 2, 0.05
    ops = [inputs.Op("CP", (2, 7), theta=0.7, noisy=True), inputs.Op("CP", (12, 17), theta=1.9, noisy=True),
           inputs.Op("CP", (10, 16), theta=2.6, noisy=False), inputs.Op("CP", (15, 16), theta=0.4, noisy=True),
           inputs.Op("CP", (10, 11), theta=1.1, noisy=True), inputs.Op("CP", (16, 17), theta=2.2, noisy=True),
           inputs.Op("CP", (3, 16), theta=0.8, noisy=True), inputs.Op("CP", (5, 14), theta=1.4, noisy=True)]
    ops += [inputs.Op("H", (q,), noisy=True) for q in range(8, n)]
    ops += [inputs.Op("CP", (9, 15), theta=0.9, noisy=True), inputs.Op("CP", (6, 13), theta=1.3, noisy=True)]
    ops += [inputs.Op("H", (q,), noisy=True) for q in range(0, 10)]
    ops += [inputs.Op("CP", (2, 5), theta=0.5, noisy=True), inputs.Op("CP", (4, 12), theta=1.7, noisy=True)]
    x0 = 0b101101110010111011
    h = qs.qs_create(n, batch, 0, qs.QS_STATEVEC, dtype)
    try:
        qs.qs_set_basis_state(h, x0)
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        qs.qs_plan_run(p, e, SEED, 9, h)
        qs.qs_plan_destroy(p)
        got = qs.qs_get_state(h).reshape(batch, -1)
    finally:
        qs.qs_destroy(h)
    tol = 1e-12 if dtype == qs.QS_C128 else 2e-5
    for b in range(batch):
        psi = osv.basis_state(n, x0)
        for g, op in enumerate(ops):
            U = ocirc.op_unitary(op)
            if op.noisy:
                xa, xb = ophilox.normal_pair(SEED, b, 9 + g)
                U = ogates.noisy_unitary(U, ocirc.op_noise(op), e, xa, xb)
            psi = osv.apply_gate(psi, n, ocirc.op_targets(op), U)
        assert np.abs(got[b] - psi).max() < tol * np.abs(psi).max() * 10
