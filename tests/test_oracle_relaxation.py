"""Pins of the relaxation channels and correction codes (Sec. 4; CPU only).

The oracle's T1/T2 channel is checked against the closed-form relaxation of
populations and coherences and the semigroup law; Eq. 19 against the phase
error channel; the three-qubit phase code against Eq. 18 (both as the
relative-state fidelity 1 - 3p^2 + 2p^3 and as the minimum over pure inputs
of sqrt(<psi|rho|psi>)); Shor's code against the same law at the block error
probability; and the relaxation of a whole register against the product of
single-qubit channel fidelities.  Planted mistakes (a dropped Toffoli, a
reversed CNOT, swapped relaxation weights) must fail these pins.
"""
import math

import numpy as np
import pytest

from oracle import density, relaxation as rx, statevec


def rand_density(rng, n, rank=3):
    A = rng.normal(size=(1 << n, rank)) + 1j * rng.normal(size=(1 << n, rank))
    rho = A @ A.conj().T
    return rho / np.trace(rho)


def eq18_fmin(p):
    """Eq. 18, Sec. 4.1: minimum fidelity of the three-qubit phase code."""
    return math.sqrt(1.0 - 3.0 * p * p + 2.0 * p ** 3)


def block_error(p):
    """Odd number of phase errors among three qubits: 3p(1-p)^2 + p^3."""
    return (1.0 - (1.0 - 2.0 * p) ** 3) / 2.0


CASES = [(0.7, 3.0, 2.0), (1.0, 3.0, 6.0), (0.25, math.inf, 1.5), (2.0, 1.0, 0.4), (0.0, 2.0, 1.0)]


@pytest.mark.parametrize("t,T1,T2", CASES)
def test_relaxation_closed_form(t, T1, T2):
    K = rx.relaxation_kraus(t, T1, T2)
    assert np.abs(sum(E.conj().T @ E for E in K) - np.eye(2)).max() < 1e-14
    rng = np.random.default_rng(0)
    rho = rand_density(rng, 1, rank=2)
    out = density.apply_channel(rho, 1, (0,), K)
    keep, c = math.exp(-t / T1), math.exp(-t / T2)
    assert abs(out[1, 1] - keep * rho[1, 1]) < 1e-14
    assert abs(out[0, 0] - (rho[0, 0] + (1 - keep) * rho[1, 1])) < 1e-14
    assert abs(out[0, 1] - c * rho[0, 1]) < 1e-14
    assert abs(out[1, 0] - c * rho[1, 0]) < 1e-14


def test_relaxation_semigroup():
    rng = np.random.default_rng(1)
    rho = rand_density(rng, 3)
    a = density.apply_channel(rho, 3, (1,), rx.relaxation_kraus(0.4, 2.5, 1.7))
    a = density.apply_channel(a, 3, (1,), rx.relaxation_kraus(0.9, 2.5, 1.7))
    b = density.apply_channel(rho, 3, (1,), rx.relaxation_kraus(1.3, 2.5, 1.7))
    assert np.abs(a - b).max() < 1e-14


def test_relaxation_rejects_unphysical():
    with pytest.raises(ValueError):
        rx.relaxation_kraus(1.0, 1.0, 2.5)
    with pytest.raises(ValueError):
        rx.relaxation_kraus(-1.0, 1.0, 1.0)


@pytest.mark.parametrize("p", [0.02, 0.2, 0.45])
def test_eq19_phase_relaxation_is_the_phase_error(p):
    t = 1.3
    rng = np.random.default_rng(2)
    rho = rand_density(rng, 2)
    a = density.apply_channel(rho, 2, (0,), rx.relaxation_kraus(t, math.inf, rx.t2_from_p(t, p)))
    b = density.apply_channel(rho, 2, (0,), rx.phase_error_kraus(p))
    assert np.abs(a - b).max() < 1e-14


@pytest.mark.parametrize("p", [0.0, 0.01, 0.1, 0.3, 0.5])
def test_eq18_three_qubit_code_relative_fidelity(p):
    f = rx.code_relative_fidelity("phase3", lambda q: rx.phase_error_kraus(p))
    assert abs(f - eq18_fmin(p) ** 2) < 1e-13


@pytest.mark.parametrize("p", [0.05, 0.25])
def test_eq18_is_the_minimum_over_pure_inputs(p):
    fs = []
    for theta in np.linspace(0.0, math.pi, 9):
        for phi in np.linspace(0.0, 2 * math.pi, 8, endpoint=False):
            psi = np.array([math.cos(theta / 2), np.exp(1j * phi) * math.sin(theta / 2)])
            out = rx.phase_code_output(p, psi)
            fs.append(math.sqrt(max(np.real(np.vdot(psi, out @ psi)), 0.0)))
    assert min(fs) >= eq18_fmin(p) - 1e-13
    assert abs(min(fs) - eq18_fmin(p)) < 1e-13       # reached at |0> (theta = 0)
    assert abs(max(fs) - 1.0) < 1e-13                # |+> is untouched


def test_three_qubit_code_beats_one_qubit_below_one_half():
    for p in (0.05, 0.2, 0.4):
        coded = rx.code_relative_fidelity("phase3", lambda q: rx.phase_error_kraus(p))
        bare = rx.uncoded_relative_fidelity(rx.phase_error_kraus(p))
        assert abs(bare - (1.0 - p)) < 1e-14
        assert coded > bare


@pytest.mark.parametrize("p", [0.02, 0.15])
def test_shor_code_phase_errors(p):
    f = rx.code_relative_fidelity("shor9", lambda q: rx.phase_error_kraus(p))
    pb = block_error(p)
    assert abs(f - (1.0 - 3.0 * pb * pb + 2.0 * pb ** 3)) < 1e-12


@pytest.mark.parametrize("code", ["phase3", "shor9"])
def test_logical_z_without_errors_is_ideal(code):
    f = rx.code_relative_fidelity(code, lambda q: [np.eye(2)], logical=rx.logical_z(code),
                                  ideal_logical=[("U", (0,), rx.Z)])
    assert abs(f - 1.0) < 1e-12
    if code == "phase3":
        # and it is not the identity: against the ideal without Z the overlap vanishes
        g = rx.code_relative_fidelity(code, lambda q: [np.eye(2)], logical=rx.logical_z(code))
        assert abs(g) < 1e-12


def test_logical_z_commutes_with_the_phase_code_law():
    p = 0.12
    f = rx.code_relative_fidelity("phase3", lambda q: rx.phase_error_kraus(p), logical=rx.logical_z("phase3"),
                                  ideal_logical=[("U", (0,), rx.Z)])
    assert abs(f - eq18_fmin(p) ** 2) < 1e-13


def test_register_relaxation_is_a_product_of_qubit_fidelities():
    # one identity gate then every qubit relaxes: Choi fidelity of each qubit
    # is sum_i |tr K_i|^2 / 4 = (1 + 2c + exp(-t/T1)) / 4
    t, T1, T2, m = 0.6, 3.0, 2.0, 3
    f = rx.qft_relaxation_fidelity(m, t, T1, T2, [((0,), np.eye(2))])
    per = (1.0 + 2.0 * math.exp(-t / T2) + math.exp(-t / T1)) / 4.0
    assert abs(f - per ** m) < 1e-13
    assert abs(rx.qft_relaxation_fidelity(m, 1.0, math.inf, math.inf, [((0, 1), rx.cnot())]) - 1.0) < 1e-13


def test_gate_matrices_are_the_textbook_permutations():
    # brute force on basis states: CNOT (c, t) and Toffoli (c1, c2, t)
    for x in range(8):
        psi = statevec.basis_state(3, x)
        out = statevec.apply_gate(psi, 3, (2, 0), rx.cnot())
        want = x ^ 1 if x & 4 else x
        assert abs(out[want] - 1.0) < 1e-15
        out = statevec.apply_gate(psi, 3, (0, 2, 1), rx.toffoli())
        want = x ^ 2 if (x & 1) and (x & 4) else x
        assert abs(out[want] - 1.0) < 1e-15


# ----------------------------------------------------------- planted mistakes

def test_mutation_dropped_toffoli_is_caught(monkeypatch):
    p = 0.1
    orig = rx.phase_code_decoder
    monkeypatch.setattr(rx, "phase_code_decoder", lambda: orig()[:-1])
    f = rx.code_relative_fidelity("phase3", lambda q: rx.phase_error_kraus(p))
    assert abs(f - eq18_fmin(p) ** 2) > 1e-3


def test_mutation_reversed_cnot_is_caught(monkeypatch):
    p = 0.1
    orig = rx.phase_code_encoder
    monkeypatch.setattr(rx, "phase_code_encoder",
                        lambda: [("U", (1, 0), rx.cnot())] + orig()[1:])
    f = rx.code_relative_fidelity("phase3", lambda q: rx.phase_error_kraus(p))
    assert abs(f - eq18_fmin(p) ** 2) > 1e-3


def test_mutation_swapped_relaxation_rates_is_caught(monkeypatch):
    orig = rx.relaxation_kraus
    monkeypatch.setattr(rx, "relaxation_kraus", lambda t, T1, T2: orig(t, T2 * 2.0, T1 / 2.0) if T1 / 2.0 <= 2 * T2 * 2.0 else orig(t, T1, T2))
    rho = rand_density(np.random.default_rng(3), 1, rank=2)
    out = density.apply_channel(rho, 1, (0,), rx.relaxation_kraus(0.7, 3.0, 2.0))
    assert abs(out[1, 1] - math.exp(-0.7 / 3.0) * rho[1, 1]) > 1e-3


# ------------------------------------------- the product's circuit definitions

def test_product_code_circuits_follow_eq18_and_the_shor_law():
    # paper_1412_2293_gb300/codes.py defines its own gate matrices, encoders and
    # decoders for the GPU runs; run through the oracle's density functions
    # here, they must give the same closed forms (CPU only)
    from paper_1412_2293_gb300 import codes

    def run(code, p):
        nq = codes.CODE_QUBITS[code]
        n = nq + 1
        rho = density.pure(statevec.basis_state(n, 0))
        prep = [((0,), codes.H), ((0, nq), codes.CNOT)]
        for t, U in prep + codes._encoder(code):
            rho = density.apply_unitary(rho, n, t, U)
        for q in range(nq):
            rho = density.apply_channel(rho, n, (q,), codes.phase_error(p))
        for t, U in codes._decoder(code):
            rho = density.apply_unitary(rho, n, t, U)
        for q in range(1, nq):
            rho = density.apply_channel(rho, n, (q,), codes.RESET)
        psi = statevec.basis_state(n, 0)
        for t, U in prep:
            psi = statevec.apply_gate(psi, n, t, U)
        return density.fidelity(psi, rho)

    p = 0.13
    assert abs(run("phase3", p) - eq18_fmin(p) ** 2) < 1e-13
    pb = block_error(p)
    assert abs(run("shor9", p) - (1.0 - 3.0 * pb * pb + 2.0 * pb ** 3)) < 1e-12
