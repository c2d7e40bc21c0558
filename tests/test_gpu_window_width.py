"""Window width m of the fused passes (10, 11, 12): every width against the
oracle on random circuits (windows low and high, three register stages,
flips, per-member flips, controlled phases inside and across the window), the
noisy QFT with created starts and the fused fidelity, the QFT at n = 24 in two
passes, the autotuner's choice, and the rejected widths."""
import numpy as np
import pytest

from oracle import circuits as ocirc
from oracle import gates as ogates
from oracle import philox as ophilox
from oracle import statevec as osv
from paper_1412_2293_gb300 import circuits as pcirc
from paper_1412_2293_gb300 import inputs, qs
from tests.tolerances import assert_amplitudes_close

pytestmark = pytest.mark.gpu
SEED = inputs.DEFAULT_SEED
WIDTHS = (10, 11, 12)


@pytest.fixture(scope="module", autouse=True)
def library():
    from paper_1412_2293_gb300 import build
    build.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return qs.lib()


class Handle:
    def __init__(self, *a):
        self.h = qs.qs_create(*a)

    def __enter__(self):
        return self.h

    def __exit__(self, *exc):
        qs.qs_destroy(self.h)


def random_ops(rng, n, count):
    ops = []
    for _ in range(count):
        r = rng.random()
        if r < 0.45:
            ops.append(inputs.Op("H", (int(rng.integers(n)),), noisy=bool(rng.random() < 0.8)))
        elif r < 0.92:
            j, k = rng.choice(n, size=2, replace=False)
            ops.append(inputs.Op("CP", (int(j), int(k)), theta=float(rng.uniform(0, 6)), noisy=bool(rng.random() < 0.8)))
        elif r < 0.94:
            ops.append(inputs.Op("FLIP", index=0))
        else:
            ops.append(inputs.Op("FLIP", index=int(rng.integers(1 << n))))
    return ops


def oracle_run(n, ops, x0, e, b, gate_id0, marked=None):
    """Gate by gate; in a per-member run (marked given) a flip at a nonzero
    index flips the member's marked index instead (circuits.to_gates with
    per_member_flip)."""
    psi = osv.basis_state(n, x0)
    for g, op in enumerate(ops):
        if op.kind == "FLIP":
            psi = osv.phase_flip(psi, marked if marked is not None and op.index != 0 else op.index)
            continue
        U = ocirc.op_unitary(op)
        if op.noisy:
            xa, xb = ophilox.normal_pair(SEED, b, gate_id0 + g)
            U = ogates.noisy_unitary(U, ocirc.op_noise(op), e, xa, xb)
        psi = osv.apply_gate(psi, n, ocirc.op_targets(op), U)
    return psi


@pytest.mark.parametrize("m", WIDTHS)
@pytest.mark.parametrize("n,seed", [(12, 1), (13, 2), (16, 3), (21, 4)])
def test_random_circuits_each_width_match_oracle(m, n, seed):
    rng = np.random.default_rng(100 * seed + m)
    ops = random_ops(rng, n, 90 if n < 21 else 60)
    batch, e, x0 = 2, 0.06, int(rng.integers(1 << n))
    with Handle(n, batch, 0, qs.QS_STATEVEC, qs.QS_C64) as h:
        qs.qs_set_basis_state(h, x0)
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        qs.qs_plan_set_window(p, m, h)
        assert qs.qs_plan_get_window(p, h) == m
        qs.qs_plan_run(p, e, SEED, 7, h)
        qs.qs_plan_destroy(p)
        got = qs.qs_get_state(h).reshape(batch, -1)
    for b in range(batch):
        assert_amplitudes_close(got[b], oracle_run(n, ops, x0, e, b, 7), qs.QS_C64, k=4.0, err_msg=f"member {b}")


@pytest.mark.parametrize("m", (11, 12))
def test_per_member_flips_and_grover_each_width(m):
    """Grover with each member's own marked item (per-member flips in every
    register stage) and random circuits with per-member flips."""
    n, batch, e = 14, 4, 0.03
    marked = [(2654435761 * (b + 1)) % (1 << n) for b in range(batch)]
    ops = inputs.grover_circuit(n, 2, 1)
    rng = np.random.default_rng(m)
    ops2 = random_ops(rng, n, 80)
    for circuit in (ops, ops2):
        with Handle(n, batch, 0, qs.QS_STATEVEC, qs.QS_C64) as h:
            # the members' own keys equal the call's: trajectory b, seed SEED, e
            qs.qs_set_member_noise(h, e=[e] * batch, seed=[SEED] * batch, traj=list(range(batch)), marked=marked)
            qs.qs_set_basis_state(h, 0)
            p = qs.qs_plan_create(h, pcirc.to_gates(circuit, per_member_flip=True))
            qs.qs_plan_set_window(p, m, h)
            qs.qs_plan_run(p, e, SEED, 0, h)
            qs.qs_plan_destroy(p)
            got = qs.qs_get_state(h).reshape(batch, -1)
        for b in range(batch):
            want = oracle_run(n, circuit, 0, e, b, 0, marked=marked[b])
            assert_amplitudes_close(got[b], want, qs.QS_C64, k=4.0, err_msg=f"member {b}")


@pytest.mark.parametrize("n", [15, 17])
def test_noisy_qft_widths_agree_with_created_starts_and_fused_fidelity(n):
    """Per-member basis starts created by the first pass and the fidelity
    reduced by the last, for each width: states against the oracle and the
    fidelities against each other and the oracle's."""
    batch, e = 6, 0.03
    ops = inputs.qft_circuit(n)
    xs = [(131 * b + 17) % (1 << n) for b in range(batch)]
    ideal0 = ocirc.ideal_state(n, ops, xs[0])
    wants = [ocirc.run_trajectory(n, ops, xs[b], e, SEED, b) for b in range(batch)]
    fids = {}
    with Handle(n, batch, 0, qs.QS_STATEVEC, qs.QS_C64) as h:
        qs.qs_set_reference(h, np.asarray(ideal0))
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        for m in WIDTHS:
            qs.qs_plan_set_window(p, m, h)
            passes, _ = qs.qs_plan_info(p)
            assert passes == (1 if n <= m else 2)
            qs.qs_set_basis_states(h, xs)
            f = qs.qs_plan_run_fidelity(p, e, SEED, 0, h)
            got = qs.qs_get_state(h).reshape(batch, -1)
            for b in range(batch):
                assert_amplitudes_close(got[b], wants[b], qs.QS_C64, err_msg=f"m={m} member {b}")
                assert abs(f[b] - osv.fidelity(ideal0, wants[b])) <= 1e-5
            # graph replay gives the same numbers
            qs.qs_set_basis_states(h, xs)
            np.testing.assert_array_equal(qs.qs_plan_run_fidelity(p, e, SEED, 0, h), f)
            fids[m] = f
        qs.qs_plan_destroy(p)
    for m in WIDTHS:
        np.testing.assert_allclose(fids[m], fids[10], rtol=0, atol=2e-6)


def test_qft_n24_two_passes_with_twelve_qubit_windows():
    """The QFT of a basis state at n = 24 against its closed form: m = 12
    takes two passes where m = 10 takes three."""
    n, x0 = 24, 0x9E3779 & ((1 << 24) - 1)
    ops = inputs.qft_circuit(n)
    y = np.arange(1 << n, dtype=np.int64)
    rev = np.zeros_like(y)
    for b in range(n):
        rev |= ((y >> b) & 1) << (n - 1 - b)
    want = np.empty(1 << n, dtype=np.complex128)
    want[rev] = 2.0 ** (-n / 2) * np.exp(-2j * np.pi * ((x0 * y) % (1 << n)) / float(1 << n))
    with Handle(n, 1, 0, qs.QS_STATEVEC, qs.QS_C64) as h:
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        assert qs.qs_plan_info(p)[0] == 3
        qs.qs_plan_set_window(p, 12, h)
        assert qs.qs_plan_info(p)[0] == 2
        qs.qs_set_basis_state(h, x0)
        qs.qs_plan_run(p, 0.0, SEED, 0, h)
        got = qs.qs_get_state(h)
        qs.qs_plan_destroy(p)
    assert_amplitudes_close(got, want, qs.QS_C64, k=2.0)


def test_autotune_chooses_a_width_and_results_stay_correct():
    n, batch, e = 17, 16, 0.02
    ops = inputs.qft_circuit(n)
    with Handle(n, batch, 0, qs.QS_STATEVEC, qs.QS_C64) as h:
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        qs.qs_plan_set_timing(p, True, h)
        lo, hi = qs.qs_plan_autotune(p, 2, e, SEED, h)
        m = qs.qs_plan_get_window(p, h)
        assert m in WIDTHS and lo > 0 and hi > 0
        nl, nh = qs.qs_plan_configs(p, h)
        cfg = qs.qs_plan_get_config(p, h)
        assert 0 <= cfg[0] < nl and 0 <= cfg[1] < nh
        qs.qs_set_basis_state(h, 5)
        qs.qs_plan_run(p, e, SEED, 0, h)
        # timing slots follow the re-planned passes
        ms, kinds = qs.qs_plan_last_times(p, h=h)
        assert len(ms) == 2 * qs.qs_plan_info(p)[0]
        got = qs.qs_get_state(h).reshape(batch, -1)
        qs.qs_plan_destroy(p)
    for b in (0, batch - 1):
        assert_amplitudes_close(got[b], ocirc.run_trajectory(n, ops, 5, e, SEED, b), qs.QS_C64)


def test_rejected_widths_leave_the_plan_usable():
    n = 13
    ops = inputs.qft_circuit(n)
    with Handle(n, 2, 0, qs.QS_STATEVEC, qs.QS_C128) as h:
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        with pytest.raises(qs.QSError):
            qs.qs_plan_set_window(p, 11, h)                  # complex128: m = 10 only
        qs.qs_plan_set_window(p, 10, h)
        qs.qs_plan_autotune(p, 1, 0.01, SEED, h)
        assert qs.qs_plan_get_window(p, h) == 10
        qs.qs_set_basis_state(h, 3)
        qs.qs_plan_run(p, 0.01, SEED, 0, h)
        got = qs.qs_get_state(h).reshape(2, -1)
        qs.qs_plan_destroy(p)
    assert_amplitudes_close(got[1], ocirc.run_trajectory(n, ops, 3, 0.01, SEED, 1), qs.QS_C128)
    with Handle(n, 2, 0, qs.QS_STATEVEC, qs.QS_C64) as h:
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        for bad in (9, 13, 0):
            with pytest.raises(qs.QSError):
                qs.qs_plan_set_window(p, bad, h)
        assert qs.qs_plan_get_window(p, h) == 10
        qs.qs_plan_destroy(p)
    with Handle(11, 2, 0, qs.QS_STATEVEC, qs.QS_C64) as h:
        # n < m: no pass fits; the gates run one by one and stay correct
        p = qs.qs_plan_create(h, pcirc.to_gates(inputs.qft_circuit(11)))
        qs.qs_plan_set_window(p, 12, h)
        assert qs.qs_plan_info(p)[0] == len(inputs.qft_circuit(11))
        qs.qs_set_basis_state(h, 9)
        qs.qs_plan_run(p, 0.02, SEED, 0, h)
        got = qs.qs_get_state(h).reshape(2, -1)
        qs.qs_plan_destroy(p)
    assert_amplitudes_close(got[0], ocirc.run_trajectory(11, inputs.qft_circuit(11), 9, 0.02, SEED, 0), qs.QS_C64)


@pytest.mark.parametrize("m", (11, 12))
def test_full_window_programs_match_oracle(m):
    """n = 22: for m = 11 both passes are full windows (compiled programs);
    for m = 12 the high pass is.  Sampled members against the oracle, all
    members' fused fidelities against m = 10."""
    n, batch, e = 22, 3, 0.02
    ops = inputs.qft_circuit(n)
    xs = [(977 * b + 3) % (1 << n) for b in range(batch)]
    ideal0 = ocirc.ideal_state(n, ops, xs[0])
    fids = {}
    with Handle(n, batch, 0, qs.QS_STATEVEC, qs.QS_C64) as h:
        qs.qs_set_reference(h, np.asarray(ideal0))
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        for w in (10, m):
            qs.qs_plan_set_window(p, w, h)
            assert qs.qs_plan_info(p)[0] == (3 if w == 10 else 2)
            qs.qs_set_basis_states(h, xs)
            fids[w] = qs.qs_plan_run_fidelity(p, e, SEED, 0, h)
        got = qs.qs_get_state(h).reshape(batch, -1)
        qs.qs_plan_destroy(p)
    np.testing.assert_allclose(fids[m], fids[10], rtol=0, atol=2e-6)
    want = ocirc.run_trajectory(n, ops, xs[batch - 1], e, SEED, batch - 1)
    assert_amplitudes_close(got[batch - 1], want, qs.QS_C64)


def test_autotune_times_runs_from_the_pending_start_and_keeps_it():
    """With a basis start set before autotuning, every profiled run creates it
    in its first pass; afterwards the start is still pending, so the next run
    begins from it."""
    n, batch, e, x0 = 15, 8, 0.02, 12345
    ops = inputs.qft_circuit(n)
    ideal = ocirc.ideal_state(n, ops, x0)
    with Handle(n, batch, 0, qs.QS_STATEVEC, qs.QS_C64) as h:
        qs.qs_set_reference(h, np.asarray(ideal))
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        qs.qs_set_basis_state(h, x0)
        qs.qs_plan_autotune(p, 1, e, SEED, h)
        f = qs.qs_plan_run_fidelity(p, e, SEED, 0, h)         # no new start: the pending one
        got = qs.qs_get_state(h).reshape(batch, -1)
        qs.qs_plan_destroy(p)
    want = ocirc.run_trajectory(n, ops, x0, e, SEED, batch - 1)
    assert_amplitudes_close(got[batch - 1], want, qs.QS_C64)
    assert abs(f[batch - 1] - osv.fidelity(ideal, want)) <= 1e-5
