"""Seeded synthetic workloads shared by the CUDA path, the oracle and the benchmark.

This module holds no simulation arithmetic.  It only describes circuits as
lists of gate descriptors (kind, qubits, angle parameter) and draws the
seeded inputs the workloads need: the Grover marked item, the basis input of
the QFT, and the job stream of the serving workload.  Both the product path
and the oracle turn the descriptors into matrices on their own.

Workload shapes follow the paper's experiments:
  * Grover's search with noisy Hadamard gates (Sec. 2, Fig. 1; Sec. 3.2,
    Fig. 2; Sec. 3.3, Eq. 10): H on every qubit, then k iterations of
    oracle, H on every qubit, diffusion, H on every qubit.  That gives
    n + 2nk noisy Hadamards, the exponent of Eq. 10.
  * The quantum Fourier transform (Sec. 3.3, Eqs. 11 and 15; Fig. 4): for
    j = n-1 down to 0, H on qubit j, then the controlled phase shift of
    Eq. 2 on (j, k) with angle pi / 2^(j-k) for k = j-1 down to 0.  No
    final swaps.  That gives n Hadamards and n(n-1)/2 controlled phases.
Qubit t is bit t of the amplitude index (qubit 0 is the least significant).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

DEFAULT_SEED = 0x14122293

# Sub-stream tags for numpy's seeded generator; each input gets its own.
_TAG_MARKED = 1
_TAG_BASIS = 2
_TAG_JOBS = 3


@dataclass(frozen=True)
class Op:
    """One gate of a circuit.

    kind   "H"    Hadamard (Eq. 4) on qubits[0]; with noisy=True the Monte
                  Carlo rotation noise of Eq. 1 acts first (Eq. 5).
           "CP"   controlled phase shift (Eq. 2) on qubits (j, k) with angle
                  theta; with noisy=True the angle is perturbed (Eqs. 7-8).
           "FLIP" negation of the single amplitude at `index` (Grover oracle
                  and diffusion as diagonal phase flips); never noisy.
    """

    kind: str
    qubits: Tuple[int, ...] = ()
    theta: float = 0.0
    index: int = 0
    noisy: bool = False


def grover_iterations(n: int) -> int:
    """Iteration count k >= 0 that maximises the ideal success probability.

    The ideal amplitude of the marked item after k iterations is
    sin((2k+1) * asin(2^(-n/2))); the best k is the integer nearest to
    pi / (4 asin(2^(-n/2))) - 1/2 (checked against its neighbours).
    """
    a = math.asin(2.0 ** (-n / 2.0))
    k0 = max(0, int(round(math.pi / (4.0 * a) - 0.5)))
    best = max(
        (k for k in (k0 - 1, k0, k0 + 1) if k >= 0),
        key=lambda k: math.sin((2 * k + 1) * a) ** 2,
    )
    return best


def grover_circuit(n: int, iterations: int, marked: int, noisy: bool = True) -> List[Op]:
    """Grover's search as gate descriptors (noisy Hadamards, noiseless flips)."""
    if not 0 <= marked < (1 << n):
        raise ValueError("marked item out of range")
    layer = [Op("H", (q,), noisy=noisy) for q in range(n)]
    ops: List[Op] = list(layer)
    for _ in range(iterations):
        ops.append(Op("FLIP", index=marked))      # oracle I - 2|w><w|
        ops.extend(layer)
        ops.append(Op("FLIP", index=0))           # diffusion, global -1 dropped
        ops.extend(layer)
    return ops


def qft_circuit(n: int, noisy: bool = True) -> List[Op]:
    """QFT without final swaps, controlled phases with the paper's e^{-i theta}."""
    ops: List[Op] = []
    for j in range(n - 1, -1, -1):
        ops.append(Op("H", (j,), noisy=noisy))
        for k in range(j - 1, -1, -1):
            ops.append(Op("CP", (j, k), theta=math.pi / float(1 << (j - k)), noisy=noisy))
    return ops


def _rng(seed: int, tag: int, *extra: int) -> np.random.Generator:
    return np.random.default_rng([seed & 0xFFFFFFFFFFFFFFFF, tag, *extra])


def draw_marked(n: int, seed: int = DEFAULT_SEED) -> int:
    """Marked item w of Grover's search, uniform over the 2^n basis states."""
    return int(_rng(seed, _TAG_MARKED, n).integers(0, 1 << n))


def draw_basis_input(n: int, seed: int = DEFAULT_SEED) -> int:
    """Random computational-basis input x of the QFT workloads."""
    return int(_rng(seed, _TAG_BASIS, n).integers(0, 1 << n))


def circuit_name(ops: List[Op]) -> str:
    kinds = {o.kind for o in ops}
    return "qft" if "CP" in kinds else "grover"


@dataclass
class Workload:
    """A named benchmark workload: circuit, sizes and noise level."""

    name: str
    n: int
    circuit: str            # "grover" | "qft"
    mode: str               # "statevec" | "density" | "fixed_rank"
    dtype: str              # "c64" | "c128"
    e: float
    trajectories: int = 1
    rank: int = 0
    seed: int = DEFAULT_SEED
    extra: dict = field(default_factory=dict)

    def ops(self, noisy: bool = True) -> List[Op]:
        if self.circuit == "grover":
            k = self.extra.get("iterations", grover_iterations(self.n))
            return grover_circuit(self.n, k, draw_marked(self.n, self.seed), noisy)
        return qft_circuit(self.n, noisy)

    def initial_basis(self) -> int:
        return 0 if self.circuit == "grover" else draw_basis_input(self.n, self.seed)


# The five workload shapes: plain noisy Grover (one trajectory at a time),
# batched noisy QFT, fixed-rank Grover, exact density-matrix QFT, serving.
WORKLOADS = {
    "mc_grover_n10_c128": Workload("mc_grover_n10_c128", 10, "grover", "statevec", "c128", 0.01, trajectories=100),
    "mc_qft_n20_c64": Workload("mc_qft_n20_c64", 20, "qft", "statevec", "c64", 0.01, trajectories=1024),
    # same circuit with 128 trajectories (1 GiB state): the profiling size
    "mc_qft_n20_c64_t128": Workload("mc_qft_n20_c64_t128", 20, "qft", "statevec", "c64", 0.01, trajectories=128),
    "mc_qft_n20_c64_e1e-3": Workload("mc_qft_n20_c64_e1e-3", 20, "qft", "statevec", "c64", 0.001, trajectories=1024),
    "mc_qft_n20_c128": Workload("mc_qft_n20_c128", 20, "qft", "statevec", "c128", 0.01, trajectories=1024),
    "rank_grover_n16": Workload("rank_grover_n16", 16, "grover", "fixed_rank", "c128", 0.01, rank=8),
    "dm_qft_n14": Workload("dm_qft_n14", 14, "qft", "density", "c128", 0.01),
    # smaller cases of the same two shapes (profiling, quick runs)
    "rank_grover_n12": Workload("rank_grover_n12", 12, "grover", "fixed_rank", "c128", 0.01, rank=8),
    "dm_qft_n10": Workload("dm_qft_n10", 10, "qft", "density", "c128", 0.01),
}


@dataclass(frozen=True)
class Job:
    """One request of the serving workload."""

    job_id: int
    arrival_s: float
    circuit: str
    n: int
    mode: str               # "statevec" (Monte Carlo) or "fixed_rank"
    trajectories: int
    rank: int
    e: float
    seed: int
    iterations: int         # Grover iteration count (capped); 0 for QFT


def draw_job_stream(
    num_jobs: int,
    rate_per_s: float,
    seed: int = DEFAULT_SEED,
    n_range: Tuple[int, int] = (12, 28),
    log2_traj_range: Tuple[int, int] = (6, 12),
    max_rank: int = 8,
    e_range: Tuple[float, float] = (1e-4, 1e-2),
    grover_iteration_cap: int = 16,
) -> List[Job]:
    """Poisson arrivals of mixed fidelity-estimation jobs.

    Half the jobs are Grover, half QFT; half are Monte Carlo (2^U{6..12}
    trajectories, complex64) and half fixed rank (r ~ U{1..max_rank},
    complex128); n ~ U{n_range}; e log-uniform in e_range.  Grover jobs
    run min(k_opt, grover_iteration_cap) iterations.
    """
    rng = _rng(seed, _TAG_JOBS, num_jobs)
    t = 0.0
    jobs = []
    for i in range(num_jobs):
        t += float(rng.exponential(1.0 / rate_per_s))
        circuit = "grover" if rng.random() < 0.5 else "qft"
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        mc = rng.random() < 0.5
        traj = 1 << int(rng.integers(log2_traj_range[0], log2_traj_range[1] + 1)) if mc else 1
        rank = 0 if mc else int(rng.integers(1, max_rank + 1))
        e = float(math.exp(rng.uniform(math.log(e_range[0]), math.log(e_range[1]))))
        js = int(rng.integers(0, 2**63))
        iters = min(grover_iterations(n), grover_iteration_cap) if circuit == "grover" else 0
        jobs.append(Job(i, t, circuit, n, "statevec" if mc else "fixed_rank", traj, rank, e, js, iters))
    return jobs


def job_ops(job: Job) -> List[Op]:
    if job.circuit == "grover":
        return grover_circuit(job.n, job.iterations, draw_marked(job.n, job.seed))
    return qft_circuit(job.n)


def job_initial_basis(job: Job) -> int:
    return 0 if job.circuit == "grover" else draw_basis_input(job.n, job.seed)
