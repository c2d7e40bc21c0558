"""Continuous-batching server on the GPU: each job's result is the same alone
and in the mix, and matches the oracle on sampled trajectories."""
import numpy as np
import pytest

from oracle import circuits as ocirc
from oracle import fixed_rank as ofr
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


def test_fidelity_ref_matches_stored_reference():
    n, B = 10, 6
    ops = inputs.qft_circuit(n)
    ref = pcirc.ideal_reference(n, ops, 5, qs.QS_C128)
    h = qs.qs_create(n, B, 0, qs.QS_STATEVEC, qs.QS_C128)
    try:
        qs.qs_set_basis_state(h, 5)
        p = qs.qs_plan_create(h, pcirc.to_gates(ops))
        qs.qs_plan_run(p, 0.02, 77, 0, h)
        qs.qs_plan_destroy(p)
        got = qs.qs_fidelity_ref(h, ref, 2, 3)
        qs.qs_set_reference_from(h, ref, 0)
        want = qs.qs_fidelity_stored(h)[2:5]
        np.testing.assert_array_equal(got, want)
        for bad in [lambda: qs.qs_fidelity_ref(h, ref, 4, 3), lambda: qs.qs_fidelity_ref(h, ref, -1, 1),
                    lambda: qs.qs_fidelity_ref(h, ref, 0, 0)]:
            with pytest.raises(qs.QSError) as ei:
                bad()
            assert ei.value.status == qs.QS_ERR_INVALID_ARG
        other = qs.qs_create(n + 1, 1, 0, qs.QS_STATEVEC, qs.QS_C128)
        try:
            with pytest.raises(qs.QSError) as ei:
                qs.qs_fidelity_ref(h, other, 0, 1)
            assert ei.value.status == qs.QS_ERR_INVALID_ARG
        finally:
            qs.qs_destroy(other)
    finally:
        qs.qs_destroy(h)
        qs.qs_destroy(ref)


def mixed_jobs():
    k10 = min(inputs.grover_iterations(10), 4)
    J = inputs.Job
    return [
        J(0, 0.000, "qft", 10, "statevec", 48, 0, 1e-2, 101, 0),
        J(1, 0.001, "qft", 10, "statevec", 100, 0, 3e-3, 102, 0),
        J(2, 0.001, "grover", 10, "statevec", 40, 0, 5e-3, 103, k10),
        J(3, 0.002, "grover", 10, "statevec", 20, 0, 2e-2, 104, k10),
        J(4, 0.002, "qft", 12, "statevec", 300, 0, 1e-3, 105, 0),
        J(5, 0.003, "grover", 8, "fixed_rank", 1, 3, 2e-2, 106, inputs.grover_iterations(8)),
        J(6, 0.003, "qft", 9, "fixed_rank", 1, 4, 3e-2, 107, 0),
        J(7, 0.004, "qft", 11, "statevec", 16, 0, 1e-2, 108, 0),
        # more fixed-rank jobs of the same two shapes (own rank, e, start, marked item)
        J(8, 0.004, "grover", 8, "fixed_rank", 1, 1, 5e-3, 109, inputs.grover_iterations(8)),
        J(9, 0.004, "grover", 8, "fixed_rank", 1, 8, 1e-2, 110, inputs.grover_iterations(8)),
        J(10, 0.004, "qft", 9, "fixed_rank", 1, 2, 1e-3, 111, 0),
    ]


def test_server_results_same_alone_and_in_the_mix():
    from paper_1412_2293_gb300.server import GpuExecutor, JobState, Server, Slice, Unit, bucket_for, member_bytes, \
        rank_bytes, run_stream
    jobs = mixed_jobs()
    srv = Server(GpuExecutor(workers=3, cache_bytes=1 << 30), budget_bytes=2 << 30, max_members=128)
    try:
        results, stats = run_stream(jobs, srv, time_scale=1.0, timeout=600)
        max_run = srv.sched.max_in_flight
        units = srv.sched._uid
        batched_rank = srv.max_rank_jobs
    finally:
        srv.close()
    assert stats["jobs"] == len(jobs)
    assert units > 4 and max_run >= 2
    assert batched_rank >= 2                                      # fixed-rank jobs shared a launch

    # each job alone, in a launch of its own
    ex = GpuExecutor(workers=1, cache_bytes=0)
    try:
        for j in jobs:
            states = {j.job_id: JobState(j, 0.0)}
            if j.mode == "fixed_rank":
                u = Unit("rank", ("rank", j.circuit, j.n, j.iterations), [Slice(j.job_id, 0, 1)], 1, rank_bytes(j.n))
            else:
                B = bucket_for(j.trajectories, 16, 1 << 12)
                u = Unit("mc", ("mc", j.circuit, j.n, j.iterations), [Slice(j.job_id, 0, j.trajectories)], B,
                         B * member_bytes(j.n))
            alone = ex.run(0, u, states)[0]
            ex.release_job(j.job_id)
            np.testing.assert_array_equal(results[j.job_id].fidelities, alone, err_msg=f"job {j.job_id}")
    finally:
        ex.close()

    # sampled trajectories and the fixed-rank jobs against the oracle
    for j in jobs:
        ops, x0 = inputs.job_ops(j), inputs.job_initial_basis(j)
        got = results[j.job_id].fidelities
        if j.mode == "statevec":
            trajs = [0, j.trajectories // 2, j.trajectories - 1]
            want = ocirc.trajectory_fidelities(j.n, ops, x0, j.e, j.seed, trajs)
            np.testing.assert_allclose(got[trajs], want, atol=1e-5, err_msg=f"job {j.job_id}")
        else:
            L = ocirc.run_fixed_rank(j.n, ops, x0, j.e, j.rank)
            want = ofr.fidelity(ocirc.ideal_state(j.n, ops, x0), L)
            assert abs(got[0] - want) <= 1e-12 * want, (j.job_id, got[0], want)
