"""Failure detection on the GPU without a fault (GPU).

A fused pass waits for each tile copy with a bounded number of polls.  The
handle's wait limit set to 0 makes every such wait give up at once -- a copy
that cannot land in the time it is given.  The pass must then let its copies
in flight land, record the failure in the device status word and return; the
run reports QS_ERR_TIMEOUT, and with the default limit back the same handle
and plan run the circuit correctly (checked against the oracle).
"""
import numpy as np
import pytest

from oracle import circuits as ocirc
from oracle import statevec as osv
from paper_1412_2293_gb300 import circuits as pcirc
from paper_1412_2293_gb300 import inputs, qs
from tests.tolerances import assert_amplitudes_close

pytestmark = pytest.mark.gpu

SEED = inputs.DEFAULT_SEED


@pytest.fixture(scope="module", autouse=True)
def library():
    from paper_1412_2293_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return qs.lib()


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_tile_copy_wait_gives_up_and_the_handle_stays_usable(dtype):
    n, batch, e = 14, 4, 0.05
    ops = inputs.qft_circuit(n)
    x0 = inputs.draw_basis_input(n, SEED)
    h = qs.qs_create(n, batch, 0, qs.QS_STATEVEC, dtype)
    try:
        ref = pcirc.ideal_reference(n, ops, x0, dtype)
        try:
            qs.qs_set_reference_from(h, ref, 0)
        finally:
            qs.qs_destroy(ref)
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        try:
            qs.qs_set_basis_state(h, x0)
            qs.qs_plan_run(p, e, SEED, 0, h)               # start synthesised: no copy waits
            qs.qs_set_wait_limit(h, 0)                     # every tile-copy wait gives up at once
            with pytest.raises(qs.QSError) as ei:
                qs.qs_plan_run_fidelity(p, e, SEED, 0, h)  # reads the state: its first wait gives up
            assert ei.value.status == qs.QS_ERR_TIMEOUT
            qs.qs_set_wait_limit(h, -1)
            qs.qs_set_basis_state(h, x0)
            f = qs.qs_plan_run_fidelity(p, e, SEED, 0, h)
            got = qs.qs_get_state(h).reshape(batch, -1)
            # once reported, the status is clear
            f2 = qs.qs_fidelity_stored(h)
        finally:
            qs.qs_plan_destroy(p)
    finally:
        qs.qs_destroy(h)
    ideal = ocirc.ideal_state(n, ops, x0)
    tol = 1e-12 if dtype == qs.QS_C128 else 1e-5
    for b in (0, batch - 1):
        want = ocirc.run_trajectory(n, ops, x0, e, SEED, b)
        assert_amplitudes_close(got[b], want, dtype)
        assert abs(f[b] - osv.fidelity(ideal, want)) <= tol
    np.testing.assert_allclose(f2, f, rtol=0, atol=tol)


def test_wait_limit_rejects_values_beyond_32_bits():
    h = qs.qs_create(10, 1, 0, qs.QS_STATEVEC, qs.QS_C64)
    try:
        with pytest.raises(qs.QSError) as ei:
            qs.qs_set_wait_limit(h, 1 << 32)
        assert ei.value.status == qs.QS_ERR_INVALID_ARG
        qs.qs_set_wait_limit(h, -5)                         # any negative value: the default
    finally:
        qs.qs_destroy(h)
