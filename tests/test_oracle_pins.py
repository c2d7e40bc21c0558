"""Pins of the oracle to things other than itself (CPU only).

Each test checks an oracle function against what the paper or the
mathematics fixes: brute-force operators, closed forms (ideal Grover, QFT of
basis states, Eq. 10), Gauss-Hermite averages of the Monte Carlo gates
(Eqs. 6, 9), invariants (trace, Hermiticity, positivity), limiting cases
(e = 0, r = 1, r = full rank) and statistics (Philox, Monte Carlo mean).
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import circuits, density, fixed_rank, gates, philox, statevec
from paper_1412_2293_gb300 import inputs


def rand_matrix(rng, d):
    return rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))


def rand_unitary(rng, d):
    q, r = np.linalg.qr(rand_matrix(rng, d))
    return q * (np.diag(r) / np.abs(np.diag(r)))


def rand_state(rng, n):
    v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
    return v / np.linalg.norm(v)


def rand_density(rng, n, rank=3):
    A = rng.normal(size=(1 << n, rank)) + 1j * rng.normal(size=(1 << n, rank))
    rho = A @ A.conj().T
    return rho / np.trace(rho)


# ---------------------------------------------------------------- Sec. 2 update

@pytest.mark.parametrize("n,targets", [(1, (0,)), (3, (1,)), (4, (3, 0)), (5, (2, 4)), (6, (5, 1, 3)), (6, (0, 1, 2))])
def test_apply_gate_matches_brute_force_operator(n, targets):
    rng = np.random.default_rng(n * 100 + len(targets))
    U = rand_matrix(rng, 1 << len(targets))
    psi = rand_state(rng, n)
    want = statevec.full_operator(n, targets, U) @ psi
    got = statevec.apply_gate(psi, n, targets, U)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


def test_one_qubit_update_is_the_papers_formula():
    # b[..i_k..] = u[i_k,0] a[..0..] + u[i_k,1] a[..1..] written per index.
    rng = np.random.default_rng(7)
    n, t = 5, 2
    U = rand_matrix(rng, 2)
    a = rand_state(rng, n)
    b = np.zeros_like(a)
    for i in range(1 << n):
        ik = (i >> t) & 1
        i0 = i & ~(1 << t)
        b[i] = U[ik, 0] * a[i0] + U[ik, 1] * a[i0 | (1 << t)]
    np.testing.assert_allclose(statevec.apply_gate(a, n, (t,), U), b, atol=1e-14)


@pytest.mark.parametrize("n,targets", [(8, (0,)), (10, (9, 3)), (12, (5, 11, 0)), (12, (1, 2, 3, 4))])
def test_index_groups_partition_all_amplitudes(n, targets):
    idx = statevec.group_indices(n, targets)
    assert idx.shape == (1 << (n - len(targets)), 1 << len(targets))
    assert np.array_equal(np.sort(idx.ravel()), np.arange(1 << n))
    for j, t in enumerate(targets):   # column c carries bit j of c at qubit t
        cols = np.arange(1 << len(targets))
        assert np.all(((idx >> t) & 1) == ((cols >> j) & 1)[None, :])


def test_invalid_targets_rejected():
    with pytest.raises(ValueError):
        statevec.group_indices(4, (1, 1))
    with pytest.raises(ValueError):
        statevec.group_indices(4, (4,))


# ---------------------------------------------------------------- ideal circuits

@pytest.mark.parametrize("n", [2, 3, 4, 6, 8, 10])
def test_ideal_grover_closed_form(n):
    w = inputs.draw_marked(n, 11)
    for k in sorted({1, 2, inputs.grover_iterations(n)}):
        psi = circuits.ideal_state(n, inputs.grover_circuit(n, k, w, noisy=False), 0)
        p = abs(psi[w]) ** 2
        want = math.sin((2 * k + 1) * math.asin(2.0 ** (-n / 2))) ** 2
        assert abs(p - want) <= 1e-12 * want
        assert abs(np.linalg.norm(psi) - 1) < 1e-13


def test_grover_iteration_counts():
    # floor(pi/4 sqrt(2^n)) for the sizes of the workloads
    assert [inputs.grover_iterations(n) for n in (10, 12, 16)] == [25, 50, 201]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_ideal_qft_of_basis_states_closed_form(n):
    # Without final swaps and with the e^{-i theta} of Eq. 2 the output of |x>
    # is phi[bitrev(y)] = 2^{-n/2} exp(-2 pi i x y / 2^n).
    N = 1 << n
    ops = inputs.qft_circuit(n, noisy=False)
    for x in range(N) if n <= 4 else (0, 1, N - 1, 37 % N):
        psi = circuits.ideal_state(n, ops, x)
        phi = np.zeros(N, dtype=complex)
        for y in range(N):
            rev = int(format(y, f"0{n}b")[::-1], 2)
            phi[rev] = np.exp(-2j * np.pi * x * y / N) / math.sqrt(N)
        np.testing.assert_allclose(psi, phi, atol=1e-13)


# ---------------------------------------------------------------- noise model

def test_noise_off_reduces_every_mode_to_the_ideal_circuit():
    n = 4
    for ops in (inputs.qft_circuit(n), inputs.grover_circuit(n, 2, 9)):
        x = 5 if inputs.circuit_name(ops) == "qft" else 0
        ideal = circuits.ideal_state(n, ops, x)
        psi = circuits.run_trajectory(n, ops, x, 0.0, 123, 4)
        np.testing.assert_allclose(psi, ideal, atol=1e-13)
        rho = circuits.run_density(n, ops, x, 0.0)
        np.testing.assert_allclose(rho, np.outer(ideal, ideal.conj()), atol=1e-13)
        L = circuits.run_fixed_rank(n, ops, x, 0.0, 1)
        assert abs(fixed_rank.fidelity(ideal, L) - 1) < 1e-12


@pytest.mark.parametrize("e", [0.0, 0.01, 0.3, 1.0])
def test_kraus_sets_are_complete(e):
    rng = np.random.default_rng(3)
    for U, noise in [(gates.hadamard(), "rotation"), (gates.controlled_phase(0.7), "phase"),
                     (rand_unitary(rng, 2), "rotation"), (rand_unitary(rng, 4), "rotation"),
                     (rand_unitary(rng, 2), "phase"), (rand_unitary(rng, 4), "phase")]:
        ks = gates.kraus_set(U, noise, e)
        S = sum(E.conj().T @ E for E in ks)
        np.testing.assert_allclose(S, np.eye(U.shape[0]), atol=1e-14)


def gauss_hermite_channel(rho, U, noise, e, k, order=80):
    """E_xi[U_xi rho U_xi^dagger] by probabilists' Gauss-Hermite quadrature."""
    x, w = np.polynomial.hermite_e.hermegauss(order)
    w = w / w.sum()
    out = np.zeros_like(rho)
    if noise == "rotation" and k == 2:
        for xa, wa in zip(x, w):
            for xb, wb in zip(x, w):
                V = gates.noisy_unitary(U, noise, e, xa, xb)
                out += wa * wb * V @ rho @ V.conj().T
        return out
    for xa, wa in zip(x, w):
        V = gates.noisy_unitary(U, noise, e, xa, 0.0)
        out += wa * V @ rho @ V.conj().T
    return out


@pytest.mark.parametrize("e", [0.01, 0.2, 0.7])
def test_kraus_sets_equal_xi_average_of_the_noisy_gates(e):
    # Eqs. 6 and 9 are the xi-averages of Eqs. 5 and 7.
    rng = np.random.default_rng(11)
    cases = [(gates.hadamard(), "rotation", 1), (rand_unitary(rng, 2), "rotation", 1),
             (rand_unitary(rng, 4), "rotation", 2), (gates.controlled_phase(1.1), "phase", 2),
             (rand_unitary(rng, 2), "phase", 1)]
    for U, noise, k in cases:
        rho = rand_density(rng, k, rank=2)
        want = gauss_hermite_channel(rho, U, noise, e, k)
        got = sum(E @ rho @ E.conj().T for E in gates.kraus_set(U, noise, e))
        np.testing.assert_allclose(got, want, atol=1e-13)


def test_hadamard_kraus_matches_printed_form():
    # Eq. 6 prints E1 = sqrt(l1) I, E2 = sqrt(l2) [[0,1],[-1,0]] for the noise
    # part; the Kraus set of H V_noise is H times those.
    e = 0.05
    l1, l2 = gates.hadamard_noise_weights(e)
    assert abs(l1 - 0.5 * (1 + math.exp(-2 * e * e))) < 1e-16
    ks = gates.rotation_kraus(np.eye(2, dtype=complex), e)
    np.testing.assert_allclose(ks[0], math.sqrt(l1) * np.eye(2))
    np.testing.assert_allclose(ks[1], math.sqrt(l2) * np.array([[0, 1], [-1, 0]]))


def test_phase_kraus_matches_printed_form():
    e = 0.2
    P = math.exp(-e * e)
    ks = gates.phase_kraus(np.eye(4, dtype=complex), e)
    np.testing.assert_allclose(ks[0], np.diag([1, 1, 1, math.sqrt(P)]))
    np.testing.assert_allclose(ks[1], np.diag([0, 0, 0, math.sqrt(1 - P)]))


# ---------------------------------------------------------------- density matrix

@pytest.mark.parametrize("n,targets", [(3, (1,)), (4, (0, 3)), (3, (2, 0))])
def test_channel_matches_brute_force_operators(n, targets):
    rng = np.random.default_rng(5 + n)
    U = rand_unitary(rng, 1 << len(targets))
    ks = gates.rotation_kraus(U, 0.3) if len(targets) <= 2 else None
    rho = rand_density(rng, n)
    want = sum(statevec.full_operator(n, targets, E) @ rho @ statevec.full_operator(n, targets, E).conj().T
               for E in ks)
    np.testing.assert_allclose(density.apply_channel(rho, n, targets, ks), want, atol=1e-13)


@pytest.mark.parametrize("n,targets", [(2, (0,)), (3, (2,)), (3, (0, 2)), (4, (3, 1))])
def test_vectorised_form_equals_channel(n, targets):
    # Sec. 3: U rho U^dag  <->  (U (x) U*) vec(rho)
    rng = np.random.default_rng(17 + n)
    U = rand_unitary(rng, 1 << len(targets))
    ks = gates.phase_kraus(U, 0.4)
    rho = rand_density(rng, n)
    want = density.apply_channel(rho, n, targets, ks)
    got = density.unvectorise(density.apply_superop(density.vectorise(rho), n, targets, ks), n)
    np.testing.assert_allclose(got, want, atol=1e-13)


@pytest.mark.parametrize("circ", ["qft", "grover"])
def test_density_stays_a_density_matrix(circ):
    n, e = 4, 0.2
    ops = inputs.qft_circuit(n) if circ == "qft" else inputs.grover_circuit(n, 3, 6)
    rho = circuits.run_density(n, ops, 3 if circ == "qft" else 0, e)
    assert abs(np.trace(rho) - 1) < 1e-13
    np.testing.assert_allclose(rho, rho.conj().T, atol=1e-14)
    assert np.linalg.eigvalsh(rho).min() > -1e-13


@pytest.mark.parametrize("circ,n,e", [("grover", 4, 0.05), ("qft", 4, 0.1)])
def test_monte_carlo_mean_matches_exact_density(circ, n, e):
    ops = inputs.grover_circuit(n, 3, 11) if circ == "grover" else inputs.qft_circuit(n)
    x = 0 if circ == "grover" else 9
    ideal = circuits.ideal_state(n, ops, x)
    exact = density.fidelity(ideal, circuits.run_density(n, ops, x, e))
    T = 1500
    f = circuits.trajectory_fidelities(n, ops, x, e, 2024, range(T), ref=ideal)
    sigma = f.std(ddof=1) / math.sqrt(T)
    assert abs(f.mean() - exact) < 4 * sigma + 1e-12, (f.mean(), exact, sigma)


# ---------------------------------------------------------------- fixed rank

@pytest.mark.parametrize("n,e", [(3, 0.01), (4, 0.05), (5, 0.1), (6, 0.01), (7, 0.03)])
def test_rank1_unnormalised_grover_is_eq10(n, e):
    k = inputs.grover_iterations(n)
    w = inputs.draw_marked(n, 5)
    L = circuits.run_fixed_rank(n, inputs.grover_circuit(n, k, w), 0, e, 1)
    p = fixed_rank.fidelity(statevec.basis_state(n, w), L)
    want = gates.grover_rank1_success(n, k, e)
    assert abs(p - want) <= 1e-12 * want


@pytest.mark.parametrize("n,e", [(3, 0.05), (5, 0.02)])
def test_rank1_normalised_grover_is_ideal(n, e):
    k = inputs.grover_iterations(n)
    w = inputs.draw_marked(n, 8)
    L = circuits.run_fixed_rank(n, inputs.grover_circuit(n, k, w), 0, e, 1, normalize=True)
    p = fixed_rank.fidelity(statevec.basis_state(n, w), L)
    assert abs(p - gates.grover_ideal_success(n, k)) < 1e-12


@pytest.mark.parametrize("circ", ["qft", "grover"])
def test_full_rank_equals_exact_density(circ):
    n, e = 3, 0.1
    ops = inputs.qft_circuit(n) if circ == "qft" else inputs.grover_circuit(n, 2, 5)
    x = 6 if circ == "qft" else 0
    rho = circuits.run_density(n, ops, x, e)
    L = circuits.run_fixed_rank(n, ops, x, e, 1 << n)
    np.testing.assert_allclose(L @ L.conj().T, rho, atol=1e-13)


def test_rank_r_approaches_exact_density():
    n, e = 4, 0.05
    w = 11
    ops = inputs.grover_circuit(n, inputs.grover_iterations(n), w)
    ideal = circuits.ideal_state(n, ops, 0)
    exact = density.fidelity(ideal, circuits.run_density(n, ops, 0, e))
    errs = []
    for r in (1, 2, 4, 8, 16):
        L = circuits.run_fixed_rank(n, ops, 0, e, r)
        errs.append(abs(fixed_rank.fidelity(ideal, L) - exact))
    assert errs[-1] < 1e-12
    assert all(b <= a + 1e-12 for a, b in zip(errs, errs[1:]))


def test_truncation_is_the_best_rank_r_approximation():
    rng = np.random.default_rng(21)
    Lp = rng.normal(size=(32, 6)) + 1j * rng.normal(size=(32, 6))
    rho = Lp @ Lp.conj().T
    lam, U = np.linalg.eigh(rho)
    for r in (1, 2, 3, 5):
        L, _ = fixed_rank.truncate(Lp, r)
        best = (U[:, -r:] * lam[-r:]) @ U[:, -r:].conj().T   # Eckart-Young
        np.testing.assert_allclose(L @ L.conj().T, best, atol=1e-11)


def test_tie_rule_is_independent_of_the_basis_inside_a_tie():
    # A Gram spectrum with an exact 3-fold tie straddling the cutoff r = 2.
    rng = np.random.default_rng(4)
    Q = rand_unitary(rng, 16)[:, :5]
    Lp = (Q * np.sqrt([3.0, 1.0, 1.0, 1.0, 0.2])) @ rand_unitary(rng, 5)
    lam, V = np.linalg.eigh(Lp.conj().T @ Lp)
    V = V[:, ::-1]
    S = V[:, 1:4]                                   # the tied eigenspace
    B1 = fixed_rank.canonical_basis(S)
    B2 = fixed_rank.canonical_basis(S @ rand_unitary(rng, 3))
    np.testing.assert_allclose(B1, B2, atol=1e-12)  # basis-independent
    np.testing.assert_allclose(B1.conj().T @ B1, np.eye(3), atol=1e-13)
    np.testing.assert_allclose(B1 @ B1.conj().T, S @ S.conj().T, atol=1e-13)
    # per-column phases of L' (eigenvector phases of the previous step) do
    # not change which part of the tie is kept
    L0, _ = fixed_rank.truncate(Lp, 2)
    L1, _ = fixed_rank.truncate(Lp * np.exp(1j * np.arange(5))[None, :], 2)
    np.testing.assert_allclose(L1 @ L1.conj().T, L0 @ L0.conj().T, atol=1e-12)
    # the kept part is a rank-2 piece of the spectrum {3, 1}
    ev = np.linalg.eigvalsh(L0 @ L0.conj().T)[::-1]
    np.testing.assert_allclose(ev[:3], [3.0, 1.0, 0.0], atol=1e-12)


def test_clusters_group_ties():
    lam = np.array([4.0, 2.0, 2.0 - 1e-12, 2.0 - 3e-11, 1.0, 0.5, 0.5])
    assert fixed_rank.clusters(lam) == [(0, 1), (1, 4), (4, 5), (5, 7)]


# ---------------------------------------------------------------- QFT estimates

@pytest.mark.parametrize("n,e", [(3, 0.01), (4, 0.05), (5, 0.02), (6, 0.01)])
def test_qft_exact_fidelity_against_eq11_and_eq15(n, e):
    x = inputs.draw_basis_input(n, 3)
    ops = inputs.qft_circuit(n)
    ideal = circuits.ideal_state(n, ops, x)
    exact = density.fidelity(ideal, circuits.run_density(n, ops, x, e))
    assert exact >= gates.qft_estimate_eq11(n, e) - 1e-12
    # Eqs. 11 and 15 are geometric-mean estimates that ignore the input state:
    # Eq. 11 held as a lower bound in every case tried; Eq. 15 can overshoot
    # for some inputs, so it is only required to sit within the infidelity.
    eq11, eq15 = gates.qft_estimate_eq11(n, e), gates.qft_estimate_eq15(n, e)
    assert abs(exact - eq15) < 1 - eq11


def test_eq15_reduces_to_eq11_without_rotation():
    # with f = 0 the rotated pair (Eq. 14) is the original one (Eq. 9)
    e = 0.05
    ph, _ = gates.hadamard_noise_weights(e)
    P = math.exp(-e * e)
    assert abs(gates.qft_estimate_eq11(5, e) - ph ** 5 * P ** (5 * 4 / 8)) < 1e-15
    assert gates.qft_estimate_eq15(5, e) > gates.qft_estimate_eq11(5, e)


# ---------------------------------------------------------------- Philox

GOLDEN = __import__("os").path.join(__import__("os").path.dirname(__file__), "golden")


def philox_kat_vectors():
    """Known-answer vectors of Philox4x32-10 (tests/golden/philox4x32_10_kat.txt):
    (counter[4], key[2], output[4]) as Python ints, from the generator's
    publication (Salmon et al., SC'11, and its Random123 distribution)."""
    out = []
    with open(__import__("os").path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            out.append((tuple(w[0:4]), tuple(w[4:6]), tuple(w[6:10])))
    return out


def test_philox_matches_published_known_answers():
    kats = philox_kat_vectors()
    assert len(kats) == 3
    for ctr, key, want in kats:
        assert philox.philox4x32_10(ctr, key) == want


def test_philox_array_matches_published_known_answers():
    kats = philox_kat_vectors()
    cols = [np.array([k[0][i] for k in kats], dtype=np.uint64) for i in range(4)]
    k0 = np.array([k[1][0] for k in kats], dtype=np.uint64)
    k1 = np.array([k[1][1] for k in kats], dtype=np.uint64)
    got = philox.philox4x32_10_array(*cols, k0, k1)
    for i, (_, _, want) in enumerate(kats):
        assert tuple(int(g[i]) for g in got) == want


def test_noise_words_map_seed_traj_gate_onto_key_and_counter():
    # counter = (traj lo, traj hi, gate lo, gate hi), key = (seed lo, seed hi):
    # the third published vector, addressed through the noise draw
    ctr, key, want = philox_kat_vectors()[2]
    traj = ctr[0] | (ctr[1] << 32)
    gate = ctr[2] | (ctr[3] << 32)
    seed = key[0] | (key[1] << 32)
    assert philox.noise_words(seed, traj, gate) == want


def test_philox_vector_and_scalar_agree():
    trajs = np.array([0, 1, 2**32 - 1, 2**32 + 5, 12345678901])
    gids = np.array([0, 7, 2**32 + 1, 3, 99])
    xa, xb = philox.normal_pairs_array(0x14122293, trajs, gids)
    for i in range(len(trajs)):
        a, b = philox.normal_pair(0x14122293, int(trajs[i]), int(gids[i]))
        assert xa[i] == a and xb[i] == b


def test_philox_words_are_uniform_bits():
    N = 20000
    t = np.arange(N, dtype=np.uint64)
    w = philox.philox4x32_10_array(t, t * np.uint64(3), np.uint64(9), np.uint64(0), np.uint64(1), np.uint64(2))
    bits = np.stack([(np.stack(w) >> np.uint64(b)) & np.uint64(1) for b in range(32)]).astype(float)
    p = bits.mean(axis=-1)          # (32 bits, 4 words)
    assert np.all(np.abs(p - 0.5) < 5 * 0.5 / math.sqrt(N))
    # neighbouring counters give unrelated words
    c = np.corrcoef(w[0][:-1].astype(float), w[0][1:].astype(float))[0, 1]
    assert abs(c) < 5 / math.sqrt(N)


def test_philox_normals_are_standard_normal():
    N = 100000
    xa, xb = philox.normal_pairs_array(0x14122293, np.arange(N) % 1000, np.arange(N) // 1000)
    for x in (xa, xb):
        assert abs(x.mean()) < 5 / math.sqrt(N)
        assert abs(x.var() - 1) < 5 * math.sqrt(2 / N)
        assert abs(stats.kurtosis(x)) < 5 * math.sqrt(24 / N)
        assert stats.kstest(x, "norm").pvalue > 1e-4
    assert abs(np.corrcoef(xa, xb)[0, 1]) < 5 / math.sqrt(N)


def test_philox_differs_across_seed_traj_gate():
    a = philox.noise_words(1, 2, 3)
    assert a != philox.noise_words(2, 2, 3)
    assert a != philox.noise_words(1, 3, 3)
    assert a != philox.noise_words(1, 2, 4)
    assert a != philox.noise_words(1, 2 + (1 << 32), 3)
    assert a != philox.noise_words(1, 2, 3 + (1 << 32))


# ---------------------------------------------------------------- relative states (Sec. 4)
from oracle import choi as ochoi  # noqa: E402


def test_maximally_entangled_state():
    om = ochoi.maximally_entangled(2)
    assert abs(np.vdot(om, om) - 1.0) < 1e-15
    nz = np.flatnonzero(np.abs(om) > 0)
    np.testing.assert_array_equal(nz, [0, 5, 10, 15])           # |i>|i>, index i + 4 i
    np.testing.assert_allclose(om[nz], 0.5)


@pytest.mark.parametrize("e", [0.05, 0.2])
def test_relative_state_is_trace_one_with_maximally_mixed_reference(e):
    n = 3
    ops = inputs.qft_circuit(n)
    rho = ochoi.relative_state(n, ops, e)
    assert abs(np.trace(rho) - 1.0) < 1e-13
    np.testing.assert_allclose(rho, rho.conj().T, atol=1e-14)
    assert np.linalg.eigvalsh(rho).min() > -1e-13
    np.testing.assert_allclose(ochoi.reference_marginal(rho, n), np.eye(1 << n) / (1 << n), atol=1e-14)


@pytest.mark.parametrize("e", [0.01, 0.1, 0.3])
def test_relative_state_fidelity_of_single_channels(e):
    # one noisy Hadamard: sum_i |tr(H^dag E_i)|^2 / 4 = lambda_1 (tr J = 0), Eq. 6
    H = gates.hadamard()
    lam1, _ = gates.hadamard_noise_weights(e)
    assert abs(ochoi.channel_fidelity(gates.rotation_kraus(H, e), H) - lam1) < 1e-15
    op = inputs.Op("H", (0,), 0.0, 0, True)
    rho = ochoi.relative_state(1, [op], e)
    psi = ochoi.ideal_relative(1, [op])
    assert abs(np.real(np.vdot(psi, rho @ psi)) - lam1) < 1e-14
    # one noisy controlled phase: |3 + sqrt P|^2 / 16 + (1 - P) / 16, Eq. 9
    P = math.exp(-e * e)
    theta = 0.7
    U = gates.controlled_phase(theta)
    want = ((3.0 + math.sqrt(P)) ** 2 + (1.0 - P)) / 16.0
    assert abs(ochoi.channel_fidelity(gates.phase_kraus(U, e), U) - want) < 1e-15
    op = inputs.Op("CP", (1, 0), theta, 0, True)
    rho = ochoi.relative_state(2, [op], e)
    psi = ochoi.ideal_relative(2, [op])
    assert abs(np.real(np.vdot(psi, rho @ psi)) - want) < 1e-14


def test_noiseless_relative_state_has_fidelity_one():
    n = 3
    ops = [inputs.Op(o.kind, o.qubits, o.theta, o.index, False) for o in inputs.qft_circuit(n)]
    rho = ochoi.relative_state(n, ops, 0.1)
    psi = ochoi.ideal_relative(n, ops)
    assert abs(np.real(np.vdot(psi, rho @ psi)) - 1.0) < 1e-13


def test_relative_state_is_the_monte_carlo_mean():
    n, e, T = 2, 0.3, 400
    ops = inputs.qft_circuit(n)
    psi = ochoi.ideal_relative(n, ops)
    rho = ochoi.relative_state(n, ops, e)
    exact = np.real(np.vdot(psi, rho @ psi))
    f = np.array([abs(np.vdot(psi, ochoi.relative_trajectory(n, ops, e, 99, b))) ** 2 for b in range(T)])
    assert abs(f.mean() - exact) < 4 * f.std() / math.sqrt(T) + 1e-12


def test_relative_states_reject_phase_flips():
    with pytest.raises(ValueError):
        ochoi.relative_state(2, inputs.grover_circuit(2, 1, 3), 0.1)


# ---------------------------------------------------------------- rotated Kraus pair (Eqs. 12-15)
@pytest.mark.parametrize("e", [0.01, 0.1, 0.5])
def test_rotated_pair_follows_the_svd_of_eq12(e):
    P = math.exp(-e * e)
    a, b = math.sqrt(P), math.sqrt(1.0 - P)
    psi = np.array([[1, 1, 1, a], [0, 0, 0, b]], dtype=float)
    Uv, sv, _ = np.linalg.svd(psi)
    # squared singular values 2 +- sqrt(1 + 3P) (the printed S repeats sqrt(lambda_1))
    np.testing.assert_allclose(np.sort(sv ** 2), [2 - math.sqrt(1 + 3 * P), 2 + math.sqrt(1 + 3 * P)], atol=1e-13)
    f = gates.rotated_cp_f(e)
    u0 = Uv[:, 0] * np.sign(Uv[0, 0])
    np.testing.assert_allclose(u0, np.array([1.0, f]) / math.sqrt(1 + f * f), atol=1e-13)   # Eq. 13, first column
    U = gates.controlled_phase(0.9)
    B = gates.rotated_phase_kraus(U, e)
    s = 1 / math.sqrt(1 + f * f)
    np.testing.assert_allclose(np.diag(U.conj().T @ B[0]), s * np.array([1, 1, 1, a + f * b]), atol=1e-15)     # Eq. 14a
    np.testing.assert_allclose(np.diag(U.conj().T @ B[1]), s * np.array([-f, -f, -f, -f * a + b]), atol=1e-15)  # Eq. 14b
    # the same channel as Eq. 9
    np.testing.assert_allclose(sum(E.conj().T @ E for E in B), np.eye(4), atol=1e-14)
    np.testing.assert_allclose(density.superoperator(B), density.superoperator(gates.phase_kraus(U, e)), atol=1e-14)


def test_branch_rank1_closed_forms():
    e, n = 0.05, 6
    # Grover: only Hadamards are noisy, each branch sqrt(lambda_1) H: Eq. 10
    k = 2
    w = 13
    ops = inputs.grover_circuit(n, k, w)
    psi = circuits.run_branch(n, ops, 0, e)
    lam1, _ = gates.hadamard_noise_weights(e)
    assert abs(abs(psi[w]) ** 2 - lam1 ** (n + 2 * n * k) * gates.grover_ideal_success(n, k)) < 1e-13
    # one controlled phase on |+>|+>: |sum_x d_x / 4|^2 with the branch's diagonal d
    P = math.exp(-e * e)
    f = gates.rotated_cp_f(e)
    plus2 = np.full(4, 0.5, dtype=np.complex128)
    U = gates.controlled_phase(0.3)
    for rotated, d in ((False, [1, 1, 1, math.sqrt(P)]),
                       (True, np.array([1, 1, 1, math.sqrt(P) + f * math.sqrt(1 - P)]) / math.sqrt(1 + f * f))):
        out = statevec.apply_gate(plus2, 2, (0, 1), gates.branch_operator(U, "phase", e, rotated))
        ideal = statevec.apply_gate(plus2, 2, (0, 1), U)
        assert abs(abs(np.vdot(ideal, out)) ** 2 - abs(sum(d) / 4) ** 2) < 1e-15
