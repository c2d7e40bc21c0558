"""Continuous-batching server for fidelity-estimation jobs.

A job asks for the fidelity of a noisy circuit (Grover or QFT, n qubits,
noise level e) with its ideal output, either as a Monte Carlo estimate over
T trajectories (Sec. 2: complex64, one fidelity per trajectory) or through
the fixed-rank density matrix (Sec. 3.2: complex128, rank r).

* Admission: jobs wait until their device memory fits an HBM budget
  (cudaMemGetInfo at start minus a reserve, or a given byte count).  With a
  per-request limit on estimated device time (`limit_s`), a Monte Carlo job
  above it runs the largest power-of-two number of trajectories (at least
  MIN_TRAJECTORIES) that fits, and says so in its result; a fixed-rank job
  above it is refused with the estimate as the reason.
* Batching: Monte Carlo trajectories of every pending job with the same
  shape (circuit, n, Grover iteration count) are packed into one launch of
  one plan; a batch member carries its own job's noise level, key, trajectory
  counter, basis input and marked item (qs_set_member_noise /
  qs_set_basis_states), so a trajectory gives the same result alone and in
  any mix.  Jobs larger than the per-launch member limit run in waves.
* Overlap: several worker threads, each with its own CUDA stream, run units
  concurrently; new arrivals are admitted as soon as memory and a worker
  free up (continuous batching at launch granularity).
* Each job records its arrival and completion time; `run_stream` reports
  circuits/s and p50/p99 latency.

The scheduling logic (`Scheduler`) holds no GPU calls and is tested on the
CPU with a fake executor; `GpuExecutor` does the CUDA work through the C ABI.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import threading
import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

import numpy as np

from . import inputs

C64_BYTES = 8
C128_BYTES = 16


# ------------------------------------------------------------------ work units
@dataclass
class Slice:
    job_id: int
    first: int              # first trajectory counter of this slice
    count: int


@dataclass
class Unit:
    """One launch of work: a Monte Carlo round or a whole fixed-rank job."""

    kind: str                         # "mc" | "rank"
    key: Tuple
    slices: List[Slice]
    members: int                      # launch batch (MC: a power of two >= sum of counts)
    bytes: int                        # device memory of the launch's own buffers
    uid: int = 0

    @property
    def cache_key(self) -> Tuple:
        return self.key + (self.members,)


@dataclass
class JobState:
    job: inputs.Job                   # as served (trajectories possibly reduced by the limit)
    arrival: float
    next_traj: int = 0                # MC: first trajectory not yet scheduled
    done_traj: int = 0
    fidelities: Optional[np.ndarray] = None
    finish: Optional[float] = None
    ref_bytes: int = 0                # MC: the ideal reference, held from first launch to completion
    ref_charged: bool = False
    requested: int = 0                # trajectories the request asked for
    progress: float = 0.0             # when the job last had a unit issued (its arrival before)


def mc_key(job: inputs.Job) -> Tuple:
    return ("mc", job.circuit, job.n, job.iterations)


def rank_key(job: inputs.Job) -> Tuple:
    return ("rank", job.circuit, job.n, job.iterations)


RANK_MAX = 8                          # rank bound of a batched fixed-rank handle
RANK_MEMBERS = 16                     # most fixed-rank jobs in one launch


def member_bytes(n: int) -> int:
    """Device bytes of one complex64 trajectory (upper bound): its amplitudes,
    reduction partials (1/64 of the state), the out-of-window factors of the
    fused passes (11 complex per 1024 amplitudes) and at most 512 KiB of
    per-member gate parameters and phase tables."""
    return (1 << n) * C64_BYTES + (1 << n) // 64 + (11 * C64_BYTES << max(n - 10, 0)) + (1 << 19)


def rank_bytes(n: int, r: int = RANK_MAX) -> int:
    """Device bytes of one member of a batched fixed-rank launch (rank bound
    r): factor, work buffer of min(32, 8 r) columns, Gram partials and other
    scratch, and the job's reference."""
    N = 1 << n
    return (r + min(32, 8 * r)) * N * C128_BYTES + N * 256 + N * C128_BYTES


# Device-time model of a request (seconds).  Monte Carlo: the fused passes
# read and write every trajectory's state once per pass at an effective
# MC_BYTES_PER_S (complex64); a pass holds the gates of one window, so the
# QFT takes ceil(n / 10) passes and Grover's search that many per layer of
# Hadamards (1 + 2 x iterations layers, the flips between them end a pass).
# Fixed rank: per channel and amplitude, RANK_S_PER_AMP + r RANK_S_PER_AMP_R
# + r^2 RANK_S_PER_AMP_R2 seconds (expansion and projection grow with r, the
# FP64 Gram matrix with (K r)^2; complex128; fitted to the QFT at n = 20..24,
# r = 1, 2, 4, 8).  Estimates for admission only; a job's latency is measured.
MC_BYTES_PER_S = 4.0e12
RANK_S_PER_AMP = 0.052e-9
RANK_S_PER_AMP_R = 0.018e-9
RANK_S_PER_AMP_R2 = 0.030e-9
MIN_TRAJECTORIES = 64


def job_gate_counts(job: inputs.Job) -> Tuple[int, int]:
    """(gates, noisy gates) of a job's circuit."""
    n = job.n
    if job.circuit == "grover":
        return n + job.iterations * (2 + 2 * n), n + 2 * n * job.iterations
    return n + n * (n - 1) // 2, n + n * (n - 1) // 2


def estimate_passes(job: inputs.Job) -> int:
    per_layer = -(-job.n // 10)
    return per_layer * (1 + 2 * job.iterations) if job.circuit == "grover" else per_layer


def estimate_seconds(job: inputs.Job, trajectories: Optional[int] = None) -> float:
    if job.mode == "fixed_rank":
        r = job.rank
        return job_gate_counts(job)[1] * float(1 << job.n) * (RANK_S_PER_AMP + r * RANK_S_PER_AMP_R +
                                                              r * r * RANK_S_PER_AMP_R2)
    t = job.trajectories if trajectories is None else trajectories
    return t * float(1 << job.n) * C64_BYTES * 2 * estimate_passes(job) / MC_BYTES_PER_S


def bucket_for(members: int, lo: int, hi: int) -> int:
    b = lo
    while b < members:
        b *= 2
    return min(max(b, lo), hi)


def largest_bucket(limit: int, hi: int) -> int:
    """Largest power of two <= min(limit, hi), or 0."""
    limit = min(limit, hi)
    if limit < 1:
        return 0
    return 1 << (int(limit).bit_length() - 1)


class Scheduler:
    """Admission and batching decisions (no device calls).

    Launch batches are powers of two between `min_bucket` and `max_members`
    so that launches of one shape reuse cached handles and plans."""

    def __init__(self, budget_bytes: int, max_members: int = 4096, min_bucket: int = 16,
                 starve_s: float = 2.0, limit_s: Optional[float] = None, share: float = 0.5):
        if max_members & (max_members - 1) or min_bucket & (min_bucket - 1) or min_bucket > max_members:
            raise ValueError("min_bucket and max_members must be powers of two, min_bucket <= max_members")
        self.budget = int(budget_bytes)
        self.limit_s = limit_s                # per-request limit on estimated device seconds, or None
        self.refused: Dict[int, str] = {}     # job id -> reason
        self.reduced: Dict[int, Tuple[int, int]] = {}   # job id -> (requested, served) trajectories
        self.max_members = max_members
        self.min_bucket = min_bucket
        self.starve_s = starve_s              # after this wait the oldest job stops backfilling
        self.share = share                    # most of the budget one shape holds while others wait
        self.key_used: Dict[Tuple, int] = collections.defaultdict(int)
        self.used = 0
        self.jobs: Dict[int, JobState] = {}
        self.order: List[int] = []            # job ids in arrival order with work left
        self.in_flight: Dict[int, Unit] = {}
        self.finished: List[int] = []
        self._uid = 0
        self.peak_used = 0
        self.max_in_flight = 0

    # -- bookkeeping -------------------------------------------------------
    def min_bytes(self, job: inputs.Job) -> int:
        """Device memory of the smallest unit a job can run in."""
        if job.mode == "fixed_rank":
            return rank_bytes(job.n)
        return member_bytes(job.n) * self.min_bucket + (1 << job.n) * C64_BYTES

    def admit(self, job: inputs.Job) -> Tuple[Optional[inputs.Job], str]:
        """The job as it will run under the per-request limit, or (None, reason)."""
        if self.limit_s is None:
            return job, ""
        est = estimate_seconds(job)
        if est <= self.limit_s:
            return job, ""
        if job.mode == "statevec":
            t = job.trajectories
            while t > MIN_TRAJECTORIES and estimate_seconds(job, t) > self.limit_s:
                t //= 2
            if estimate_seconds(job, t) <= self.limit_s:
                return dataclasses.replace(job, trajectories=t), ""
        return None, f"estimated {est:.1f} s of device time, limit {self.limit_s:.1f} s"

    def submit(self, job: inputs.Job, now: float) -> bool:
        """Queue a job; False when the per-request limit refuses it."""
        if job.mode not in ("statevec", "fixed_rank") or job.trajectories < 1:
            raise ValueError(f"job {job.job_id}: unsupported mode {job.mode!r}")
        if job.job_id in self.jobs or job.job_id in self.refused:
            raise ValueError(f"job {job.job_id} submitted twice")
        if self.min_bytes(job) > self.budget:
            raise MemoryError(f"job {job.job_id} needs {self.min_bytes(job)} bytes, more than the budget {self.budget}")
        requested = job.trajectories
        served, reason = self.admit(job)
        if served is None:
            self.refused[job.job_id] = reason
            return False
        job = served
        if job.trajectories != requested:
            self.reduced[job.job_id] = (requested, job.trajectories)
        st = JobState(job, now, requested=requested, progress=now)
        if job.mode == "statevec":
            st.fidelities = np.full(job.trajectories, np.nan)
            st.ref_bytes = (1 << job.n) * C64_BYTES
        self.jobs[job.job_id] = st
        self.order.append(job.job_id)
        return True

    def pending(self) -> int:
        return len(self.order)

    def busy(self) -> bool:
        return bool(self.order) or bool(self.in_flight)

    # -- decisions ---------------------------------------------------------
    def next_unit(self, now: float = 0.0) -> Optional[Unit]:
        """The next unit that fits the budget, oldest job first, or None.

        While other jobs wait, a shape that already has a unit in flight, or a
        job past its first wave, holds at most `share` of the budget, so a job
        that runs in many waves leaves room for later arrivals.
        Younger jobs backfill memory the oldest cannot use yet, until the
        oldest has made no progress (no unit issued) for `starve_s` seconds:
        then nothing new starts before it."""
        free = self.budget - self.used
        others = len(self.order) > 1
        for pos, jid in enumerate(list(self.order)):
            st = self.jobs[jid]
            job = st.job
            key = rank_key(job) if job.mode == "fixed_rank" else mc_key(job)
            # while others wait, a shape with a unit in flight, or the later waves
            # of a job, take at most `share` of the budget
            capped = others and (self.key_used[key] > 0 or st.next_traj > 0)
            avail = min(free, int(self.share * self.budget) - self.key_used[key]) if capped else free
            if job.mode == "fixed_rank":
                made = self._rank_unit(key, avail)
                if made is not None:
                    return self._issue(made, [], now)
            else:
                made = self._mc_unit(key, avail)
                if made is not None:
                    return self._issue(*made, now)
            if pos == 0 and now - st.progress > self.starve_s:
                return None
        return None

    def _rank_unit(self, key, free):
        """Pack pending fixed-rank jobs of one shape (ranks up to RANK_MAX, own
        e, start, marked item) into one launch of a batched handle."""
        per = rank_bytes(key[2])
        fit = largest_bucket(free // per, RANK_MEMBERS)
        if fit < 1:
            return None
        slices = []
        for jid in self.order:
            st = self.jobs[jid]
            if st.job.mode == "fixed_rank" and rank_key(st.job) == key:
                slices.append(Slice(jid, 0, 1))
                if len(slices) >= fit:
                    break
        if not slices:
            return None
        for sl in slices:
            self.order.remove(sl.job_id)
        members = bucket_for(len(slices), 1, RANK_MEMBERS)
        return Unit("rank", key, slices, members, members * per)

    def _mc_unit(self, key, free):
        """Pack pending trajectories of every job of one shape into one launch."""
        per = member_bytes(key[2])
        slices, total, refs, charge = [], 0, 0, []
        for jid in self.order:
            st = self.jobs[jid]
            if st.job.mode != "statevec" or mc_key(st.job) != key:
                continue
            left = st.job.trajectories - st.next_traj
            if left <= 0:
                continue
            ref = 0 if st.ref_charged or jid in charge else st.ref_bytes
            fit = largest_bucket((free - refs - ref) // per, self.max_members)
            if fit < self.min_bucket or fit <= total:
                break
            take = min(left, fit - total)
            slices.append(Slice(jid, st.next_traj, take))
            total += take
            refs += ref
            if ref:
                charge.append(jid)
            if total >= self.max_members:
                break
        if not slices:
            return None
        members = bucket_for(total, self.min_bucket, self.max_members)
        for sl in slices:
            st = self.jobs[sl.job_id]
            st.next_traj += sl.count
            if st.next_traj >= st.job.trajectories:
                self.order.remove(sl.job_id)
        return Unit("mc", key, slices, members, members * per), charge

    def _issue(self, unit: Unit, charge: List[int], now: float = 0.0) -> Unit:
        self._uid += 1
        unit.uid = self._uid
        self.used += unit.bytes
        self.key_used[unit.key] += unit.bytes
        for sl in unit.slices:
            self.jobs[sl.job_id].progress = now
        for jid in charge:
            st = self.jobs[jid]
            st.ref_charged = True
            self.used += st.ref_bytes
        if self.used > self.budget:
            raise AssertionError("scheduler exceeded its memory budget")
        self.peak_used = max(self.peak_used, self.used)
        self.in_flight[unit.uid] = unit
        self.max_in_flight = max(self.max_in_flight, len(self.in_flight))
        return unit

    def complete(self, unit: Unit, results: List[np.ndarray], now: float) -> List[int]:
        """Record a finished unit; returns the ids of jobs that are now complete."""
        self.in_flight.pop(unit.uid)
        self.used -= unit.bytes
        self.key_used[unit.key] -= unit.bytes
        done = []
        for sl, res in zip(unit.slices, results):
            st = self.jobs[sl.job_id]
            if unit.kind == "rank":
                st.fidelities = np.asarray(res, dtype=np.float64).reshape(-1)
                st.done_traj = 1
                st.finish = now
                done.append(sl.job_id)
                continue
            st.fidelities[sl.first:sl.first + sl.count] = res
            st.done_traj += sl.count
            if st.done_traj >= st.job.trajectories:
                st.finish = now
                if st.ref_charged:
                    self.used -= st.ref_bytes
                done.append(sl.job_id)
        self.finished.extend(done)
        return done


def choose_window(qs, p, h, n: int) -> int:
    """Window width of a Monte Carlo plan: 11 or 12 qubits when that leaves two
    passes where 10 needs more (the QFT at n = 21..24), else 10.

    A Monte Carlo plan runs from basis starts, so its first pass only writes
    the state; with two passes the wider window's only reading pass is the low
    one, which keeps its speed.  A plan with more passes (Grover's search, or
    n > 24) would read the state through wide high windows, whose single
    128 KiB tile per SM leaves the load exposed, so it stays at 10."""
    passes10 = qs.qs_plan_info(p, h)[0]
    if passes10 <= 2:
        return 10
    for m in (11, 12):
        if n < m:
            break
        qs.qs_plan_set_window(p, m, h)
        if qs.qs_plan_info(p, h)[0] == 2:
            return m
    qs.qs_plan_set_window(p, 10, h)
    return 10


# ------------------------------------------------------------------ GPU executor
class GpuExecutor:
    """Runs units through the C ABI; one CUDA stream per worker thread.

    Idle handles (with their plans) stay in a cache of at most `cache_bytes`
    so that launches of a recurring shape skip allocation and planning; the
    server keeps that many bytes out of its scheduling budget."""

    def __init__(self, workers: int = 4, cache_bytes: int = 4 << 30):
        import torch

        from . import build, qs
        build.build()
        self.qs = qs
        self.workers = workers
        self.streams = [torch.cuda.Stream() for _ in range(workers)]
        self.ref_streams = [torch.cuda.Stream() for _ in range(workers)]
        self.refs: Dict[int, object] = {}          # job id -> reference handle
        self.lock = threading.Lock()
        self.cache_bytes = cache_bytes
        self.idle: "collections.OrderedDict[Tuple, List]" = collections.OrderedDict()   # key -> [(h, p, bytes)]
        self.idle_bytes = 0

    # -- handle cache ------------------------------------------------------
    def _checkout(self, key):
        with self.lock:
            lst = self.idle.get(key)
            if not lst:
                return None
            ent = lst.pop()
            if not lst:
                del self.idle[key]
            self.idle_bytes -= ent[2]
            return ent

    def _checkin(self, key, ent):
        drop = []
        with self.lock:
            while self.idle and self.idle_bytes + ent[2] > self.cache_bytes:
                k0, lst = next(iter(self.idle.items()))
                old = lst.pop(0)
                if not lst:
                    del self.idle[k0]
                self.idle_bytes -= old[2]
                drop.append(old)
            if self.idle_bytes + ent[2] <= self.cache_bytes:
                self.idle.setdefault(key, []).append(ent)
                self.idle.move_to_end(key)
                self.idle_bytes += ent[2]
            else:
                drop.append(ent)
        for h, p, _ in drop:
            self._free(h, p)

    def _free(self, h, p):
        if p is not None:
            self.qs.qs_plan_destroy(p)
        self.qs.qs_destroy(h)

    def close(self):
        with self.lock:
            ents = [e for lst in self.idle.values() for e in lst]
            self.idle.clear()
            self.idle_bytes = 0
            refs = list(self.refs.values())
            self.refs.clear()
        for h, p, _ in ents:
            self._free(h, p)
        for h in refs:
            self.qs.qs_destroy(h)

    # -- references --------------------------------------------------------
    def release_job(self, job_id: int) -> None:
        with self.lock:
            h = self.refs.pop(job_id, None)
        if h is not None:
            self.qs.qs_destroy(h)

    def _reference(self, w: int, job: inputs.Job, dtype: int):
        """Ideal output of a job (batch-1 handle on worker w's reference stream, synchronised)."""
        from . import circuits as pc
        with self.lock:
            h = self.refs.get(job.job_id)
        if h is not None:
            return h
        h = pc.ideal_reference(job.n, inputs.job_ops(job), inputs.job_initial_basis(job), dtype,
                               self.ref_streams[w])
        with self.lock:
            if job.job_id in self.refs:          # built concurrently by another worker
                other, h = h, self.refs[job.job_id]
            else:
                self.refs[job.job_id] = h
                other = None
        if other is not None:
            self.qs.qs_destroy(other)
        return h

    # -- units -------------------------------------------------------------
    def run(self, w: int, unit: Unit, jobs: Dict[int, JobState]) -> List[np.ndarray]:
        if unit.kind == "rank":
            return self._run_rank(w, unit, jobs)
        return self._run_mc(w, unit, jobs)

    def _run_rank(self, w, unit, jobs):
        """The fixed-rank jobs of a unit as members of one batched handle: each
        with its own rank, e, start state and marked item, the circuit run as
        one replayed plan, each fidelity against the job's own reference."""
        qs = self.qs
        from . import circuits as pc
        _, circuit, n, iters = unit.key
        ent = self._checkout(unit.cache_key)
        if ent is None:
            ops = inputs.grover_circuit(n, iters, 1) if circuit == "grover" else inputs.qft_circuit(n)
            h = qs.qs_create(n, unit.members, RANK_MAX, qs.QS_FIXED_RANK, qs.QS_C128, self.streams[w])
            try:
                p = qs.qs_plan_create(h, pc.to_gates(ops, per_member_flip=True))
            except BaseException:
                qs.qs_destroy(h)
                raise
            ent = (h, p, unit.bytes)
        h, p, _ = ent
        try:
            B = unit.members
            ranks = np.ones(B, dtype=np.int32)
            e = np.zeros(B)
            basis = np.zeros(B, dtype=np.uint64)
            marked = np.zeros(B, dtype=np.uint64)
            for m, sl in enumerate(unit.slices):
                job = jobs[sl.job_id].job
                ranks[m], e[m] = job.rank, job.e
                basis[m] = inputs.job_initial_basis(job)
                if circuit == "grover":
                    marked[m] = inputs.draw_marked(job.n, job.seed)
            # padding members (rank 1) repeat the last job; their results are dropped
            m = len(unit.slices)
            if m < B:
                e[m:], basis[m:], marked[m:] = e[m - 1], basis[m - 1], marked[m - 1]
            qs.qs_set_member_ranks(h, ranks)
            qs.qs_set_member_noise(h, e, np.zeros(B, dtype=np.uint64), np.zeros(B, dtype=np.uint64), marked)
            qs.qs_set_basis_states(h, basis)
            qs.qs_plan_run(p, 0.0, 0, 0, h)
            out = []
            for m, sl in enumerate(unit.slices):
                ref = self._reference(w, jobs[sl.job_id].job, qs.QS_C128)
                out.append(qs.qs_fidelity_ref(h, ref, m, 1))
        except BaseException:
            self._free(h, p)
            raise
        self._checkin(unit.cache_key, ent)
        return out

    def _run_mc(self, w, unit, jobs):
        qs = self.qs
        from . import circuits as pc
        _, circuit, n, iters = unit.key
        ent = self._checkout(unit.cache_key)
        if ent is None:
            # the oracle's phase flip runs per member, so one plan serves every marked item
            ops = inputs.grover_circuit(n, iters, 1) if circuit == "grover" else inputs.qft_circuit(n)
            h = qs.qs_create(n, unit.members, 0, qs.QS_STATEVEC, qs.QS_C64, self.streams[w])
            try:
                p = qs.qs_plan_create(h, pc.to_gates(ops, per_member_flip=True))
                choose_window(qs, p, h, n)
            except BaseException:
                qs.qs_destroy(h)
                raise
            ent = (h, p, unit.bytes)
        h, p, _ = ent
        try:
            B = unit.members
            e = np.zeros(B)
            seed = np.zeros(B, dtype=np.uint64)
            traj = np.zeros(B, dtype=np.uint64)
            basis = np.zeros(B, dtype=np.uint64)
            marked = np.zeros(B, dtype=np.uint64)
            m, spans = 0, []
            for sl in unit.slices:
                job = jobs[sl.job_id].job
                e[m:m + sl.count] = job.e
                seed[m:m + sl.count] = job.seed
                traj[m:m + sl.count] = np.arange(sl.first, sl.first + sl.count, dtype=np.uint64)
                basis[m:m + sl.count] = inputs.job_initial_basis(job)
                if circuit == "grover":
                    marked[m:m + sl.count] = inputs.draw_marked(job.n, job.seed)
                spans.append((m, sl.count))
                m += sl.count
            # padding members rerun the last trajectory; their results are dropped
            if m < B:
                e[m:], seed[m:], traj[m:], basis[m:], marked[m:] = e[m - 1], seed[m - 1], traj[m - 1], basis[m - 1], marked[m - 1]
            qs.qs_set_member_noise(h, e, seed, traj, marked)
            qs.qs_set_basis_states(h, basis)
            qs.qs_plan_run(p, 0.0, 0, 0, h)
            out = []
            for sl, (first, count) in zip(unit.slices, spans):
                ref = self._reference(w, jobs[sl.job_id].job, qs.QS_C64)
                out.append(qs.qs_fidelity_ref(h, ref, first, count))
        except BaseException:
            self._free(h, p)
            raise
        self._checkin(unit.cache_key, ent)
        return out


# ------------------------------------------------------------------ the server
@dataclass
class JobResult:
    job_id: int
    fidelities: np.ndarray
    arrival: float
    finish: float

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


class Server:
    """Request loop: admission, batching and overlapped execution of jobs."""

    def __init__(self, executor=None, workers: int = 4, budget_bytes: Optional[int] = None,
                 reserve_bytes: int = 8 << 30, max_members: int = 4096, min_bucket: int = 16,
                 limit_s: Optional[float] = None):
        if executor is None:
            executor = GpuExecutor(workers)
        if budget_bytes is None:
            import torch
            free, _ = torch.cuda.mem_get_info()
            budget_bytes = max(free - reserve_bytes - getattr(executor, "cache_bytes", 0), 1 << 28)
        self.ex = executor
        self.sched = Scheduler(budget_bytes, max_members, min_bucket, limit_s=limit_s)
        self.lock = threading.Condition()
        self.t0 = time.perf_counter()
        self.results: Dict[int, JobResult] = {}
        self.errors: List[BaseException] = []
        self.free_workers = list(range(executor.workers))
        self.max_rank_jobs = 0                    # most fixed-rank jobs in one launch so far
        self.stop = False
        self.threads: List[threading.Thread] = []
        self.dispatcher = threading.Thread(target=self._dispatch, daemon=True)
        self.dispatcher.start()

    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, job: inputs.Job) -> bool:
        """Queue a job; False when the per-request limit refuses it."""
        with self.lock:
            ok = self.sched.submit(job, self.now())
            self.lock.notify_all()
        return ok

    def _dispatch(self):
        while True:
            with self.lock:
                while not self.stop and not (self.free_workers and self.sched.pending()):
                    self.lock.wait(0.05)
                if self.stop:
                    return
                try:
                    unit = self.sched.next_unit(self.now())
                except BaseException as exc:               # a job that can never fit
                    self.errors.append(exc)
                    self.stop = True
                    self.lock.notify_all()
                    return
                if unit is None:
                    self.lock.wait(0.01)
                    continue
                if unit.kind == "rank":
                    self.max_rank_jobs = max(self.max_rank_jobs, len(unit.slices))
                w = self.free_workers.pop()
                th = threading.Thread(target=self._work, args=(w, unit), daemon=True)
                self.threads.append(th)
                th.start()

    def _work(self, w: int, unit: Unit):
        try:
            res = self.ex.run(w, unit, self.sched.jobs)
            err = None
        except BaseException as exc:
            res, err = None, exc
        done = []
        with self.lock:
            if err is not None:
                self.errors.append(err)
                self.stop = True
            else:
                done = self.sched.complete(unit, res, self.now())
                for jid in done:
                    st = self.sched.jobs[jid]
                    self.results[jid] = JobResult(jid, st.fidelities, st.arrival, st.finish)
        for jid in done:                          # frees device memory: outside the lock
            self.ex.release_job(jid)
        with self.lock:
            self.free_workers.append(w)
            self.lock.notify_all()

    def drain(self, timeout: float = 600.0) -> Dict[int, JobResult]:
        end = time.perf_counter() + timeout
        with self.lock:
            while self.sched.busy() and not self.stop:
                left = end - time.perf_counter()
                if left <= 0:
                    raise TimeoutError("server did not finish its jobs in time")
                self.lock.wait(min(left, 0.05))
        if self.errors:
            raise self.errors[0]
        return dict(self.results)

    def close(self):
        with self.lock:
            self.stop = True
            self.lock.notify_all()
        self.dispatcher.join(timeout=5)
        for th in self.threads:
            th.join(timeout=60)
        self.ex.close()


def run_stream(jobs: List[inputs.Job], server: Server, time_scale: float = 1.0, timeout: float = 600.0):
    """Submit jobs at their (scaled) arrival times; return results and statistics."""
    t_start = server.now()
    for job in sorted(jobs, key=lambda j: j.arrival_s):
        delay = t_start + job.arrival_s * time_scale - server.now()
        if delay > 0:
            time.sleep(delay)
        server.submit(job)
    results = server.drain(timeout)
    lat = np.array([r.latency for r in results.values()]) if results else np.zeros(1)
    span = (max(r.finish for r in results.values()) - t_start) if results else 0.0
    circuits = sum(len(r.fidelities) for r in results.values())
    stats = {"jobs": len(results), "circuits": int(circuits), "span_s": span,
             "circuits_per_s": circuits / span if span > 0 else math.inf,
             "jobs_per_s": len(results) / span if span > 0 else math.inf,
             "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
             "peak_budget_used": server.sched.peak_used, "budget": server.sched.budget,
             "refused": dict(server.sched.refused), "reduced": dict(server.sched.reduced)}
    return results, stats
