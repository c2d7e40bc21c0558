"""Scheduler and request loop of the continuous-batching server, on the CPU.

A fake executor stands in for the GPU: it sleeps for a time that grows with
the launch and returns a value that names the job and trajectory, so every
result can be traced back to the work that made it."""
import threading
import time

import numpy as np
import pytest

from paper_1412_2293_gb300 import inputs
from paper_1412_2293_gb300.server import (Scheduler, Server, Unit, bucket_for, largest_bucket,
                                          member_bytes, rank_bytes, run_stream)


def job(i, n=12, traj=64, circuit="qft", mode="statevec", rank=0, arrival=0.0, iters=0):
    return inputs.Job(i, arrival, circuit, n, mode, traj if mode == "statevec" else 1, rank,
                      1e-3, 1000 + i, iters)


def value(job_id, t):
    return job_id + t * 1e-6


class FakeExecutor:
    def __init__(self, workers=3, sec_per_member=2e-6):
        self.workers = workers
        self.sec = sec_per_member
        self.lock = threading.Lock()
        self.running = 0
        self.max_running = 0
        self.units = []
        self.released = []

    def run(self, w, unit, jobs):
        with self.lock:
            self.running += 1
            self.max_running = max(self.max_running, self.running)
            self.units.append(unit)
        time.sleep(0.002 + self.sec * unit.members)
        out = []
        for sl in unit.slices:
            if unit.kind == "rank":
                out.append(np.array([value(sl.job_id, 0)]))
            else:
                out.append(np.array([value(sl.job_id, t) for t in range(sl.first, sl.first + sl.count)]))
        with self.lock:
            self.running -= 1
        return out

    def release_job(self, job_id):
        self.released.append(job_id)

    def close(self):
        pass


def test_buckets():
    assert bucket_for(1, 16, 4096) == 16
    assert bucket_for(17, 16, 4096) == 32
    assert bucket_for(5000, 16, 4096) == 4096
    assert largest_bucket(1000, 4096) == 512
    assert largest_bucket(0, 4096) == 0
    assert largest_bucket(10 ** 9, 4096) == 4096


def test_same_shape_jobs_share_one_launch():
    s = Scheduler(1 << 40)
    s.submit(job(0, traj=64), 0.0)
    s.submit(job(1, traj=32), 0.0)
    s.submit(job(2, n=13, traj=64), 0.0)          # another shape
    u = s.next_unit()
    assert u.kind == "mc" and u.key == ("mc", "qft", 12, 0)
    assert [(x.job_id, x.first, x.count) for x in u.slices] == [(0, 0, 64), (1, 0, 32)]
    assert u.members == 128
    u2 = s.next_unit()
    assert [(x.job_id, x.count) for x in u2.slices] == [(2, 64)]
    assert s.next_unit() is None


def test_large_job_runs_in_waves_and_budget_holds():
    n = 16
    per = member_bytes(n)
    ref = (1 << n) * 8
    budget = 300 * per + ref
    s = Scheduler(budget, max_members=4096)
    s.submit(job(0, n=n, traj=1000), 0.0)
    units = []
    while True:
        u = s.next_unit()
        if u is None:
            break
        units.append(u)
    # the reference is held for the job's lifetime; the other 300 members' room
    # takes the largest power-of-two launches that fit
    assert [u.members for u in units] == [256, 32]
    assert s.used <= budget
    covered = []
    for u in units:
        s.complete(u, [np.zeros(u.slices[0].count)], 1.0)
        covered.append((u.slices[0].first, u.slices[0].count))
    while s.busy():
        u = s.next_unit()
        assert u is not None and s.used <= budget
        covered.append((u.slices[0].first, u.slices[0].count))
        s.complete(u, [np.zeros(u.slices[0].count)], 2.0)
    starts = [c[0] for c in covered]
    assert starts == sorted(starts) and sum(c[1] for c in covered) == 1000
    assert s.used == 0 and s.finished == [0]


def test_job_that_can_never_fit_is_refused():
    s = Scheduler(1 << 20)
    with pytest.raises(MemoryError):
        s.submit(job(0, n=20, traj=64), 0.0)
    with pytest.raises(MemoryError):
        s.submit(job(1, n=16, mode="fixed_rank", rank=4), 0.0)
    with pytest.raises(ValueError):
        s.submit(inputs.Job(2, 0.0, "qft", 10, "density", 1, 0, 1e-3, 1, 0), 0.0)


def test_backfill_stops_when_the_oldest_job_starves():
    n = 14
    big = rank_bytes(18, 8)
    # one 16-member launch with its reference beside the rank job, less a byte
    s = Scheduler(big + 16 * member_bytes(n) + (1 << n) * 8 - 1, starve_s=1.0)
    s.submit(job(0, n=14, traj=16), 0.0)
    u0 = s.next_unit(0.0)                         # occupies memory
    s.submit(job(1, n=18, mode="fixed_rank", rank=8), 0.0)
    s.submit(job(2, n=14, traj=16), 0.0)
    assert s.next_unit(0.5).slices[0].job_id == 2  # backfill while job 1 is young
    s.submit(job(3, n=14, traj=16), 0.6)
    assert s.next_unit(1.5) is None               # job 1 waited too long: no backfill
    s.complete(u0, [np.zeros(16)], 1.6)
    assert s.next_unit(1.6) is None               # still not enough room for job 1
    for uid in list(s.in_flight):
        s.complete(s.in_flight[uid], [np.zeros(16)], 1.7)
    u = s.next_unit(1.7)
    assert u.kind == "rank" and u.slices[0].job_id == 1


def test_server_runs_a_job_stream_with_overlap():
    jobs = inputs.draw_job_stream(60, rate_per_s=2000.0, seed=7, n_range=(10, 14), log2_traj_range=(4, 10),
                                  max_rank=4)
    ex = FakeExecutor(workers=3)
    budget = 64 << 20
    srv = Server(ex, budget_bytes=budget, max_members=256)
    try:
        results, stats = run_stream(jobs, srv, time_scale=1.0, timeout=60)
    finally:
        srv.close()
    assert stats["jobs"] == len(jobs)
    for j in jobs:
        r = results[j.job_id]
        expect = np.array([value(j.job_id, t) for t in range(j.trajectories)])
        np.testing.assert_array_equal(r.fidelities, expect)     # every trajectory exactly once, in place
        assert r.finish >= r.arrival
    assert sorted(ex.released) == sorted(j.job_id for j in jobs)
    assert ex.max_running >= 2                                   # work overlaps
    assert srv.sched.peak_used <= budget and srv.sched.used == 0
    # launches mixed jobs of one shape
    assert any(len(u.slices) > 1 for u in ex.units)
    assert all(u.members & (u.members - 1) == 0 for u in ex.units if u.kind == "mc")
    assert stats["latency_p99_s"] >= stats["latency_p50_s"] > 0


def test_executor_error_surfaces():
    class Broken(FakeExecutor):
        def run(self, w, unit, jobs):
            raise RuntimeError("device call failed")

    srv = Server(Broken(workers=2), budget_bytes=1 << 30)
    try:
        srv.submit(job(0))
        with pytest.raises(RuntimeError, match="device call failed"):
            srv.drain(timeout=10)
    finally:
        srv.close()


def test_member_bytes_cover_state_partials_and_out_factors():
    from paper_1412_2293_gb300.server import member_bytes
    for n in (12, 20, 28):
        state = 8 << n
        # amplitudes, fused-fidelity partials (1/64) and 11 complex64 out factors per 1024 amplitudes
        assert member_bytes(n) >= state + (1 << n) // 64 + 88 * (1 << (n - 10))


def test_fixed_rank_jobs_of_one_shape_share_a_launch():
    n = 12
    s = Scheduler(1 << 34)
    k = inputs.grover_iterations(n)
    for i in range(5):
        s.submit(job(i, n=n, circuit="grover", mode="fixed_rank", rank=1 + i, iters=k), 0.0)
    s.submit(job(5, n=n, circuit="qft", mode="fixed_rank", rank=3), 0.0)
    u = s.next_unit(0.0)
    assert u.kind == "rank" and [sl.job_id for sl in u.slices] == [0, 1, 2, 3, 4]
    assert u.members == 8 and u.bytes == 8 * rank_bytes(n)
    u2 = s.next_unit(0.0)
    assert u2.kind == "rank" and [sl.job_id for sl in u2.slices] == [5] and u2.members == 1
    assert s.next_unit(0.0) is None
    s.complete(u, [np.zeros(1)] * 5, 1.0)
    s.complete(u2, [np.zeros(1)], 1.0)
    assert sorted(s.finished) == [0, 1, 2, 3, 4, 5] and s.used == 0


def test_per_request_limit_reduces_monte_carlo_jobs_and_refuses_fixed_rank():
    """A Monte Carlo job over the limit runs the largest power-of-two number of
    trajectories that fits it (at least 64); a fixed-rank job over it is
    refused; jobs under it are untouched."""
    from paper_1412_2293_gb300.server import MIN_TRAJECTORIES, estimate_seconds
    limit = 2.0
    s = Scheduler(1 << 50, max_members=4096, limit_s=limit)
    small = job(0, n=12, traj=256)
    big = job(1, n=26, traj=4096)
    huge = job(2, n=28, traj=4096, circuit="grover", iters=16)
    rank_big = job(3, n=26, mode="fixed_rank", rank=8)
    rank_small = job(4, n=14, mode="fixed_rank", rank=2)
    assert estimate_seconds(small) < limit < estimate_seconds(big)
    assert s.submit(small, 0.0) and s.submit(big, 0.0) and s.submit(rank_small, 0.0)
    served = s.jobs[1].job.trajectories
    assert served < 4096 and served & (served - 1) == 0 and served >= MIN_TRAJECTORIES
    assert estimate_seconds(big, served) <= limit < estimate_seconds(big, 2 * served)
    assert s.reduced == {1: (4096, served)} and s.jobs[1].requested == 4096
    assert len(s.jobs[1].fidelities) == served and s.jobs[0].job.trajectories == 256
    # even 64 trajectories of the capped Grover search at n = 28 exceed the limit
    assert estimate_seconds(huge, MIN_TRAJECTORIES) > limit
    assert not s.submit(huge, 0.0) and 2 in s.refused
    assert not s.submit(rank_big, 0.0) and "limit" in s.refused[3]
    assert sorted(s.jobs) == [0, 1, 4] and s.pending() == 3
    with pytest.raises(ValueError):
        s.submit(rank_big, 0.0)                                  # a refused id cannot come back


def test_server_reports_refused_and_reduced_jobs():
    jobs = [job(0, n=12, traj=64), job(1, n=26, traj=4096, arrival=0.001),
            job(2, n=26, mode="fixed_rank", rank=8, arrival=0.002)]
    ex = FakeExecutor(workers=2, sec_per_member=1e-7)
    srv = Server(ex, budget_bytes=1 << 50, max_members=4096, limit_s=2.0)
    try:
        results, stats = run_stream(jobs, srv, time_scale=1.0, timeout=60)
    finally:
        srv.close()
    assert sorted(results) == [0, 1] and list(stats["refused"]) == [2]
    req, served = stats["reduced"][1]
    assert req == 4096 and len(results[1].fidelities) == served < 4096
    np.testing.assert_array_equal(results[1].fidelities, [value(1, t) for t in range(served)])


def test_a_job_in_many_waves_leaves_room_for_later_arrivals():
    """A job whose trajectories fill the budget several times over runs in
    waves; once other jobs wait, its later waves take at most half the
    budget, so a small job arriving after it starts before it is done."""
    per = member_bytes(16)
    s = Scheduler(64 * per + (1 << 16) * 8 * 4, max_members=64, min_bucket=16, starve_s=100.0)
    s.submit(job(0, n=16, traj=1024), 0.0)
    u0 = s.next_unit(0.0)
    assert u0.members == 64                          # the first wave takes what is free
    s.submit(job(1, n=12, traj=64), 0.1)
    assert s.next_unit(0.1) is None                  # no room yet
    s.complete(u0, [np.zeros(64)], 0.2)
    u2 = s.next_unit(0.2)
    assert [sl.job_id for sl in u2.slices] == [0] and u2.members == 32
    u3 = s.next_unit(0.2)
    assert [sl.job_id for sl in u3.slices] == [1]    # the small job runs beside the big one
    assert s.jobs[0].next_traj < 1024 and s.used <= s.budget


def test_window_choice_takes_a_wider_window_only_for_two_passes():
    """choose_window: 11 or 12 qubits when that leaves two passes (a write-only
    first pass and the last) where 10 needs more; otherwise back to 10."""
    from paper_1412_2293_gb300.server import choose_window

    class FakeQs:
        def __init__(self, passes):
            self.passes, self.m, self.calls = passes, 10, []

        def qs_plan_info(self, p, h=None):
            return self.passes[self.m], 0

        def qs_plan_set_window(self, p, m, h=None):
            self.calls.append(m)
            self.m = m

    cases = [(22, {10: 3, 11: 2, 12: 2}, 11), (24, {10: 3, 11: 3, 12: 2}, 12), (20, {10: 2, 11: 2, 12: 2}, 10),
             (21, {10: 99, 11: 66, 12: 66}, 10), (11, {10: 3, 11: 2}, 11), (10, {10: 4}, 10)]
    for n, passes, want in cases:
        q = FakeQs(passes)
        assert choose_window(q, None, None, n) == want, (n, passes)
        assert q.m == want                                   # the plan is left at the width returned
