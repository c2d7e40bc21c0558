"""Planted mistakes in the oracle must be caught by its pins (CPU only).

Each test patches one plausible mistake into the oracle (a transposed
operand, a dropped conjugate, swapped weights, a wrong sign, a reversed
sort) and checks that the corresponding independent pin now fails.
"""
import math

import numpy as np

from oracle import circuits, density, fixed_rank, gates, statevec
from paper_1412_2293_gb300 import inputs


def _rand(rng, d):
    return rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))


def test_transposed_gate_is_caught_by_brute_force_pin(monkeypatch):
    rng = np.random.default_rng(0)
    n, targets = 4, (2, 0)
    U = _rand(rng, 4)
    psi = rng.normal(size=16) + 0j
    want = statevec.full_operator(n, targets, U) @ psi
    orig = statevec.apply_gate
    monkeypatch.setattr(statevec, "apply_gate", lambda p, n_, t, M: orig(p, n_, t, M.T))
    assert np.abs(statevec.apply_gate(psi, n, targets, U) - want).max() > 1e-3


def test_swapped_targets_are_caught_by_brute_force_pin():
    rng = np.random.default_rng(1)
    U = _rand(rng, 4)
    psi = rng.normal(size=32) + 0j
    want = statevec.full_operator(5, (1, 3), U) @ psi
    assert np.abs(statevec.apply_gate(psi, 5, (3, 1), U) - want).max() > 1e-3


def test_dropped_conjugate_is_caught_by_vectorisation_pin(monkeypatch):
    rng = np.random.default_rng(2)
    n = 2
    q, _ = np.linalg.qr(_rand(rng, 2))
    ks = gates.rotation_kraus(q, 0.3)
    A = rng.normal(size=(4, 2)) + 1j * rng.normal(size=(4, 2))
    rho = A @ A.conj().T
    want = density.apply_channel(rho, n, (1,), ks)
    monkeypatch.setattr(density, "superoperator", lambda kr: sum(np.kron(E, E) for E in kr))
    got = density.unvectorise(density.apply_superop(density.vectorise(rho), n, (1,), ks), n)
    assert np.abs(got - want).max() > 1e-3


def test_swapped_kraus_weights_are_caught_by_gauss_hermite_pin(monkeypatch):
    from tests.test_oracle_pins import gauss_hermite_channel
    e = 0.3
    rho = np.array([[0.7, 0.2 - 0.1j], [0.2 + 0.1j, 0.3]])
    want = gauss_hermite_channel(rho, gates.hadamard(), "rotation", e, 1)
    monkeypatch.setattr(gates, "hadamard_noise_weights",
                        lambda e_: tuple(reversed((0.5 * (1 + math.exp(-2 * e_ * e_)),
                                                   0.5 * (1 - math.exp(-2 * e_ * e_))))))
    got = sum(E @ rho @ E.conj().T for E in gates.rotation_kraus(gates.hadamard(), e))
    assert np.abs(got - want).max() > 1e-3


def test_wrong_phase_damping_is_caught_by_gauss_hermite_pin(monkeypatch):
    from tests.test_oracle_pins import gauss_hermite_channel
    e = 0.4
    rho = np.full((4, 4), 0.25, dtype=complex)
    U = gates.controlled_phase(0.9)
    want = gauss_hermite_channel(rho, U, "phase", e, 2)
    # P = exp(-e^2/2) instead of exp(-e^2)
    def bad(U_, e_):
        P = math.exp(-e_ * e_ / 2)
        return [U_ @ np.diag([1, 1, 1, math.sqrt(P)]), U_ @ np.diag([0, 0, 0, math.sqrt(1 - P)])]
    monkeypatch.setattr(gates, "phase_kraus", bad)
    got = sum(E @ rho @ E.conj().T for E in gates.kraus_set(U, "phase", e))
    assert np.abs(got - want).max() > 1e-3


def test_wrong_cp_sign_is_caught_by_qft_closed_form(monkeypatch):
    n, x = 3, 5
    N = 1 << n
    phi = np.zeros(N, dtype=complex)
    for y in range(N):
        phi[int(format(y, f"0{n}b")[::-1], 2)] = np.exp(-2j * np.pi * x * y / N) / math.sqrt(N)
    monkeypatch.setattr(gates, "controlled_phase",
                        lambda th: np.diag([1, 1, 1, np.exp(1j * th)]).astype(complex))
    psi = circuits.ideal_state(n, inputs.qft_circuit(n, noisy=False), x)
    assert np.abs(psi - phi).max() > 1e-3


def test_keeping_the_smallest_eigenvalues_is_caught_by_eckart_young(monkeypatch):
    rng = np.random.default_rng(3)
    Lp = rng.normal(size=(16, 4)) + 1j * rng.normal(size=(16, 4))
    rho = Lp @ Lp.conj().T
    lam, U = np.linalg.eigh(rho)
    best = (U[:, -1:] * lam[-1:]) @ U[:, -1:].conj().T
    eigh = np.linalg.eigh
    monkeypatch.setattr(np.linalg, "eigh", lambda G: (lambda lv: (-lv[0], lv[1]))(eigh(G)))
    L, _ = fixed_rank.truncate(Lp, 1)
    assert np.abs(L @ L.conj().T - best).max() > 1e-3


def test_rank1_formula_pin_detects_an_extra_noisy_gate():
    # Eq. 10's exponent n + 2nk counts the noisy Hadamards: one more noisy
    # gate changes the rank-1 result by a factor lambda_1.
    n, e = 4, 0.05
    k = inputs.grover_iterations(n)
    ops = inputs.grover_circuit(n, k, 3) + [inputs.Op("H", (0,), noisy=True), inputs.Op("H", (0,), noisy=False)]
    L = circuits.run_fixed_rank(n, ops, 0, e, 1)
    p = fixed_rank.fidelity(statevec.basis_state(n, 3), L)
    assert abs(p - gates.grover_rank1_success(n, k, e)) > 1e-4


def test_mutation_relative_state_on_the_reference_half_is_caught(monkeypatch):
    """Gates applied to the reference qubits instead of the system: the single-channel pin
    still holds by symmetry, but the noiseless-circuit pin does not."""
    import numpy as np

    from oracle import choi, statevec
    orig = statevec.apply_gate

    def shifted(psi, n2, targets, U):
        return orig(psi, n2, tuple(t + n2 // 2 for t in targets), U)

    n = 3
    ops = [inputs.Op(o.kind, o.qubits, o.theta, o.index, False) for o in inputs.qft_circuit(n)]
    psi = choi.ideal_relative(n, ops)
    monkeypatch.setattr(choi.statevec, "apply_gate", shifted)
    rho = choi.relative_state(n, ops, 0.0)
    monkeypatch.undo()
    # the ideal vector applies U to the system, the mutated state to the reference: not equal
    assert abs(np.real(np.vdot(psi, rho @ psi)) - 1.0) > 1e-3


def test_mutation_unnormalised_entangled_state_is_caught(monkeypatch):
    import numpy as np

    from oracle import choi
    orig = choi.maximally_entangled
    monkeypatch.setattr(choi, "maximally_entangled", lambda n: orig(n) * 2.0 ** (n / 2))
    rho = choi.relative_state(2, inputs.qft_circuit(2), 0.1)
    assert abs(np.trace(rho) - 1.0) > 1e-3


def _kat_fails(monkeypatch, **patch):
    from oracle import philox
    from tests.test_oracle_pins import philox_kat_vectors
    for k, v in patch.items():
        monkeypatch.setattr(philox, k, v)
    return any(philox.philox4x32_10(c, k_) != w for c, k_, w in philox_kat_vectors())


def test_swapped_philox_multipliers_are_caught_by_known_answers(monkeypatch):
    from oracle import philox
    assert _kat_fails(monkeypatch, PHILOX_M0=philox.PHILOX_M1, PHILOX_M1=philox.PHILOX_M0)


def test_swapped_weyl_increments_are_caught_by_known_answers(monkeypatch):
    from oracle import philox
    assert _kat_fails(monkeypatch, PHILOX_W0=philox.PHILOX_W1, PHILOX_W1=philox.PHILOX_W0)


def test_wrong_round_count_is_caught_by_known_answers(monkeypatch):
    assert _kat_fails(monkeypatch, PHILOX_ROUNDS=7)


def test_swapped_product_halves_are_caught_by_known_answers(monkeypatch):
    # a round that takes lo(M c) where hi(M c) belongs (and vice versa)
    from oracle import philox
    M = philox.MASK32

    def bad(counter, key):
        c0, c1, c2, c3 = (int(x) & M for x in counter)
        k0, k1 = (int(x) & M for x in key)
        for rnd in range(10):
            if rnd:
                k0 = (k0 + philox.PHILOX_W0) & M
                k1 = (k1 + philox.PHILOX_W1) & M
            p0, p1 = philox.PHILOX_M0 * c0, philox.PHILOX_M1 * c2
            c0, c1, c2, c3 = ((p1 & M) ^ c1 ^ k0, p1 >> 32, (p0 & M) ^ c3 ^ k1, p0 >> 32)
        return c0, c1, c2, c3

    from tests.test_oracle_pins import philox_kat_vectors
    assert any(bad(c, k) != w for c, k, w in philox_kat_vectors())
