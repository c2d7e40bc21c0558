"""The allocation-free fidelity entry point agrees with qs_fidelity (GPU).

qs_fidelity_noalloc serves callers that cannot allocate device memory (their
host application owns the GPU's memory through its own pool, or cudaMalloc's
device-wide synchronisation is unaffordable in their loop).  It reads state
and reference buffers the caller already holds and keeps its scratch in a
fixed array of the library.  This file is collected last so that a failure
here cannot hide the other tests' results; it also passes on its own in a
fresh process.  The device buffers below are made by the test itself (with
torch) -- the entry point under test allocates nothing.
"""
import numpy as np
import pytest

from oracle import statevec as osv
from paper_1412_2293_gb300 import circuits as pcirc
from paper_1412_2293_gb300 import inputs, qs

pytestmark = pytest.mark.gpu

TOL = {qs.QS_C128: 1e-12, qs.QS_C64: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def library():
    from paper_1412_2293_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return qs.lib()


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
def test_noalloc_fidelity_matches_qs_fidelity_on_two_calls(dtype):
    import torch

    n, batch, e, seed = 11, 6, 0.05, inputs.DEFAULT_SEED
    ops = inputs.qft_circuit(n)
    x0 = inputs.draw_basis_input(n, seed)
    h = qs.qs_create(n, batch, 0, qs.QS_STATEVEC, dtype)
    ref_h = pcirc.ideal_reference(n, ops, x0, dtype)
    try:
        qs.qs_set_basis_state(h, x0)
        pcirc.apply_ops(h, ops, e, seed)
        ref = qs.qs_get_state(ref_h)
        want = qs.qs_fidelity(h, ref)                       # the existing entry point
        states = qs.qs_get_state(h)
    finally:
        qs.qs_destroy(ref_h)
        qs.qs_destroy(h)
    tdt = torch.complex64 if dtype == qs.QS_C64 else torch.complex128
    d_states = torch.from_numpy(states.astype(np.complex64 if dtype == qs.QS_C64 else np.complex128)).to("cuda", tdt)
    d_ref = torch.from_numpy(ref.astype(np.complex64 if dtype == qs.QS_C64 else np.complex128)).to("cuda", tdt)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    for _ in range(2):                                      # two calls in a row share the scratch
        got = qs.qs_fidelity_noalloc(d_states.data_ptr(), d_ref.data_ptr(), n, batch, dtype, stream)
        np.testing.assert_allclose(got, want, rtol=TOL[dtype], atol=TOL[dtype])
    # a smaller batch after a larger one reads only its own partials
    got = qs.qs_fidelity_noalloc(d_states.data_ptr(), d_ref.data_ptr(), n, 2, dtype, stream)
    np.testing.assert_allclose(got, want[:2], rtol=TOL[dtype], atol=TOL[dtype])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    d = torch.zeros(4, dtype=torch.complex64, device="cuda")
    with pytest.raises(qs.QSError) as ei:
        qs.qs_fidelity_noalloc(d.data_ptr(), d.data_ptr(), 2, qs.QS_NOALLOC_MAX_MEMBERS + 1, qs.QS_C64)
    assert ei.value.status == qs.QS_ERR_INVALID_ARG
    with pytest.raises(qs.QSError) as ei:
        qs.qs_fidelity_noalloc(0, d.data_ptr(), 2, 1, qs.QS_C64)
    assert ei.value.status == qs.QS_ERR_INVALID_ARG


def _two_component_states(n, members, dtype, seed):
    """Device states psi_b = cos(t_b) ref + sin(t_b) e^{i p_b} orth with orth
    orthogonal to ref, so |<ref|psi_b>|^2 = cos(t_b)^2 exactly (made with torch
    by the test; the entry point allocates nothing)."""
    import torch

    rng = np.random.default_rng(seed)
    N = 1 << n
    ref = rng.normal(size=N) + 1j * rng.normal(size=N)
    ref /= np.linalg.norm(ref)
    orth = rng.normal(size=N) + 1j * rng.normal(size=N)
    orth -= np.vdot(ref, orth) * ref
    orth /= np.linalg.norm(orth)
    t = rng.uniform(0, np.pi / 2, size=members)
    ph = rng.uniform(0, 2 * np.pi, size=members)
    tdt = torch.complex64 if dtype == qs.QS_C64 else torch.complex128
    d_ref = torch.from_numpy(ref).to("cuda").to(tdt)
    d_orth = torch.from_numpy(orth).to("cuda").to(tdt)
    c = torch.from_numpy(np.cos(t)).to("cuda").to(tdt)
    s = torch.from_numpy(np.sin(t) * np.exp(1j * ph)).to("cuda").to(tdt)
    states = c[:, None] * d_ref[None, :] + s[:, None] * d_orth[None, :]
    return states.contiguous(), d_ref, np.cos(t) ** 2


@pytest.mark.parametrize("dtype", [qs.QS_C64, qs.QS_C128])
@pytest.mark.parametrize("n,members", [(21, 2), (18, 2048)])
def test_noalloc_many_chunks_and_capped_chunks_against_closed_form_and_oracle(dtype, n, members):
    """n = 21 with two members: 512 chunks per member, summed in order.
    n = 18 with 2048 members: 64 chunks per member would need 131072 partials,
    so the chunk count is capped at 32 and every block covers 8192 amplitudes
    (more than the 4096 of an uncapped chunk)."""
    import torch

    states, d_ref, closed = _two_component_states(n, members, dtype, seed=n * 7 + members)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    tol = 1e-12 if dtype == qs.QS_C128 else 1e-5
    for _ in range(2):
        got = qs.qs_fidelity_noalloc(states.data_ptr(), d_ref.data_ptr(), n, members, dtype, stream)
        np.testing.assert_allclose(got, closed, rtol=0, atol=tol)
    # the oracle's fidelity of the very vectors the GPU summed, on sampled members
    ref_h = d_ref.cpu().numpy().astype(np.complex128)
    for b in sorted({0, members // 2, members - 1}):
        want = osv.fidelity(ref_h, states[b].cpu().numpy().astype(np.complex128))
        assert abs(got[b] - want) <= tol, (b, got[b], want)
    del states
    torch.cuda.empty_cache()
