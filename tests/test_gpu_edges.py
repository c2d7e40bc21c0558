"""Edge cases through the C ABI: allocations beyond HBM fail cleanly and leave
the device usable; states past 2^32 amplitudes (64-bit indexing) in the
fused passes and the density sweeps, against closed forms; empty gate lists
and empty qubit lists."""
import math

import numpy as np
import pytest

from paper_1412_2293_gb300 import circuits as pcirc
from paper_1412_2293_gb300 import inputs, qs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def library():
    from paper_1412_2293_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return qs.lib()


def test_allocation_beyond_hbm_fails_cleanly():
    # 2^36 complex64 amplitudes = 512 GiB, more than the device holds
    with pytest.raises(qs.QSError) as e:
        qs.qs_create(36, 1, 0, qs.QS_STATEVEC, qs.QS_C64)
    assert e.value.status == qs.QS_ERR_OUT_OF_MEMORY
    with pytest.raises(qs.QSError) as e:
        qs.qs_create(18, 1, 0, qs.QS_DENSITY, qs.QS_C128)       # 4^18 x 16 B = 1 TiB
    assert e.value.status == qs.QS_ERR_OUT_OF_MEMORY
    # the device is still usable
    h = qs.qs_create(4, 1, 0, qs.QS_STATEVEC, qs.QS_C128)
    try:
        qs.qs_apply_gate(h, (0,), pcirc.hadamard())
        assert abs(qs.qs_trace(h)[0] - 1.0) < 1e-15
    finally:
        qs.qs_destroy(h)


def test_qft_on_2_pow_33_amplitudes():
    # 64 GiB complex64: member-local offsets beyond 32 bits in every fused
    # pass (the high windows' 64-bit kernel).  The noiseless QFT of a basis
    # state has |amplitude|^2 = 2^-33 everywhere; the norm stays 1.
    n, x = 33, 0x1F0F0F0F1
    h = qs.qs_create(n, 1, 0, qs.QS_STATEVEC, qs.QS_C64)
    try:
        ops = inputs.qft_circuit(n, noisy=False)
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        passes, _ = qs.qs_plan_info(p, h)
        assert passes == 4                    # windows [23, 33), [13, 23), [3, 13), [0, 10)
        qs.qs_set_basis_state(h, x)
        qs.qs_plan_run(p, 0.0, 1, 0, h)
        qs.qs_plan_destroy(p)
        for y in (0, 1, (1 << 32) + 5, (1 << n) - 1):
            f = qs.qs_fidelity(h, None, y)[0]
            assert abs(f * 2 ** n - 1.0) < 1e-4
        assert abs(qs.qs_trace(h)[0] - 1.0) < 1e-4
        # the inverse circuit (reversed order, conjugate phases) must bring
        # every phase back: the state returns to |x>
        inv = [inputs.Op(o.kind, o.qubits, -o.theta, o.index, False) for o in reversed(ops)]
        p = qs.qs_plan_create(h, pcirc.to_gates(inv))
        qs.qs_plan_run(p, 0.0, 1, 0, h)
        qs.qs_plan_destroy(p)
        assert abs(qs.qs_fidelity(h, None, x)[0] - 1.0) < 1e-4
    finally:
        qs.qs_destroy(h)


def test_density_relaxation_on_2_pow_32_entries():
    # 16-qubit complex128 density matrix (4^16 entries, 64 GiB): amplitude
    # damping of |x><x| leaves <0|rho|0> = gamma^popcount(x) and trace 1
    n, x = 16, 0b1011001110001101
    t, T1, T2 = 0.4, 2.0, 1.0
    gamma = 1.0 - math.exp(-t / T1)
    h = qs.qs_create(n, 1, 0, qs.QS_DENSITY, qs.QS_C128)
    try:
        qs.qs_set_basis_state(h, x)
        qs.qs_apply_relaxation(h, list(range(n)), t, T1, T2)
        f0 = qs.qs_fidelity(h, None, 0)[0]
        fx = qs.qs_fidelity(h, None, x)[0]
        tr = qs.qs_trace(h)[0]
    finally:
        qs.qs_destroy(h)
    k = bin(x).count("1")
    assert abs(f0 - gamma ** k) < 1e-12 * max(gamma ** k, 1e-300) + 1e-300
    assert abs(fx - (1.0 - gamma) ** k) < 1e-12
    assert abs(tr - 1.0) < 1e-12


def test_empty_gate_list_and_empty_qubit_list():
    n, batch = 12, 4
    h = qs.qs_create(n, batch, 0, qs.QS_STATEVEC, qs.QS_C64)
    try:
        qs.qs_set_basis_states(h, [3, 5, 7, 9])
        p = qs.qs_plan_create(h, [])
        qs.qs_plan_run(p, 0.01, 1, 0, h)
        qs.qs_plan_destroy(p)
        for b, xb in enumerate([3, 5, 7, 9]):
            assert qs.qs_fidelity(h, None, xb)[b] == 1.0
    finally:
        qs.qs_destroy(h)
    d = qs.qs_create(3, 1, 0, qs.QS_DENSITY, qs.QS_C128)
    try:
        qs.qs_set_basis_state(d, 6)
        qs.qs_apply_relaxation(d, [], 1.0, 3.0, 2.0)
        assert qs.qs_fidelity(d, None, 6)[0] == 1.0
    finally:
        qs.qs_destroy(d)
