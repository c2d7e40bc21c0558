#!/usr/bin/env python
"""Benchmark of the noisy-circuit hot path on GB300.

Workload (default): batched Monte Carlo noisy QFT, n = 20 qubits, 1024
complex64 trajectories with FP32 arithmetic, e = 0.01 (noisy Hadamards with
the rotation noise of Eq. 1, noisy controlled phases theta -> theta + e xi),
random basis input from the seed.  One step = run the 210-gate circuit from
the basis input on every trajectory (fused passes in one CUDA graph: the first
pass creates the input in registers, the last also reduces the fidelity with
the ideal output) and read the 1024 fidelities back to the host.

Metric: amplitude-gate updates/s = trajectories * 2^n * gates / time.
Prints one JSON line (rank 0).  --impl reference times the oracle (the plain
complex128 CPU simulator) on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "amplitude-gate updates/s"
UNIT = "updates/s"


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, which):
        if which == 0:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [l for t, l in self.lines if self.t0 is not None and self.t0 - 0.1 <= t <= (self.t1 or t) + 0.1]
        if not rows:
            rows = [l for _, l in self.lines]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [x.strip() for x in r.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def plan_source_hash():
    h = hashlib.sha256()
    for f in ("pass.cuh", "philox.cuh"):
        with open(os.path.join(ROOT, "paper_1412_2293_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kind):
    """DRAM bytes per launch from the committed ncu summary, if the kernel is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        with open(path) as f:
            t = json.load(f)
    except Exception:
        return None
    if t.get("source_hash") != plan_source_hash():
        return None
    v = t.get("kernels", {}).get(kind)
    return None if v is None else float(v)


def workload_setup(name):
    from paper_1412_2293_gb300 import inputs
    W = inputs.WORKLOADS[name]
    ops = W.ops()
    x0 = W.initial_basis()
    return W, ops, x0


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_1412_2293_gb300 import build as qbuild
    from paper_1412_2293_gb300 import circuits as pcirc
    from paper_1412_2293_gb300 import qs, shard

    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    torch.cuda.set_device(local_rank)
    qbuild.build()
    W, ops, x0 = workload_setup(args.workload)
    n, T, e, seed = W.n, W.trajectories, W.e, W.seed
    dtype = qs.QS_C64 if W.dtype == "c64" else qs.QS_C128
    esize = 8 if dtype == qs.QS_C64 else 16
    stream = torch.cuda.Stream()
    traj0, _ = shard.trajectory_range(rank, T)          # weak scaling: each rank its own trajectories
    h = qs.qs_create(n, T, 0, qs.QS_STATEVEC, dtype, stream)
    ref = pcirc.ideal_reference(n, ops, x0, dtype, stream)
    qs.qs_set_reference_from(h, ref, 0)
    qs.qs_destroy(ref)
    qs.qs_set_trajectory_offset(h, traj0)
    p = qs.qs_plan_create(h, pcirc.to_gates(ops))
    # window width and kernel configuration of the passes: given, or the fastest on this
    # plan (eager runs, untimed)
    if args.kernel_config:
        lo, hi = (int(x) for x in args.kernel_config.split(","))
        qs.qs_plan_set_window(p, args.window, h)
        qs.qs_plan_set_config(p, lo, hi, h)
        tune_ms = (-1.0, -1.0)
    else:
        qs.qs_set_basis_state(h, x0)                     # timed as the steps run: start created by the first pass
        tune_ms = qs.qs_plan_autotune(p, 2, e, seed, h)
    kernel_cfg = qs.qs_plan_get_config(p, h)
    window = qs.qs_plan_get_window(p, h)
    passes, launches = qs.qs_plan_info(p, h)
    qs.qs_plan_set_timing(p, True, h)
    updates_per_step = T * (1 << n) * len(ops)

    def step():
        qs.qs_set_basis_state(h, x0)                     # created by the first pass
        return qs.qs_plan_run_fidelity(p, e, seed, 0, h)  # fidelity reduced by the last pass

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        fid = step()
    # timed region: device time with CUDA events on the library's stream
    kern = {}
    sampler = ClockSampler(local_rank) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.mark(0)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    order_kinds = []
    for _ in range(args.steps):
        fid = step()
        ms, kinds = qs.qs_plan_last_times(p, h=h)
        order_kinds = [k for k in kinds if k.startswith("pass")]
        for m, k in zip(ms, kinds):
            kern.setdefault(k, []).append(m)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    if sampler:
        sampler.mark(1)
    elapsed_ms = shard.max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
    ms_per_step = elapsed_ms / args.steps
    value = shard.job_throughput(updates_per_step, world, ms_per_step / 1e3)
    clocks = sampler.stop() if sampler else None

    # end to end through the C ABI with host buffers: every step uploads the
    # members' inputs (basis state, noise key, trajectory counter, e) from host
    # memory and reads the fidelities back.
    xs = np.full(T, x0, dtype=np.uint64)
    e_arr = np.full(T, e, dtype=np.float64)
    s_arr = np.full(T, seed, dtype=np.uint64)
    t_arr = np.arange(traj0, traj0 + T, dtype=np.uint64)

    def step_e2e():
        qs.qs_set_member_noise(h, e_arr, s_arr, t_arr)
        qs.qs_set_basis_states(h, xs)
        return qs.qs_plan_run_fidelity(p, e, seed, 0, h)

    qs.qs_plan_set_timing(p, False, h)
    for _ in range(max(1, args.warmup)):
        fid_e2e = step_e2e()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        fid_e2e = step_e2e()
    torch.cuda.synchronize()
    t_e2e = shard.max_over_ranks((time.perf_counter() - t0) / args.steps, dist, "cuda")
    e2e_value = shard.job_throughput(updates_per_step, world, t_e2e)
    assert np.allclose(fid_e2e, fid, atol=1e-6), "end-to-end run disagrees with the device-resident run"
    # per-member inputs override later runs' arguments: clear them before h is reused
    qs.qs_set_member_noise(h)

    # roofline of the dominant kernel (the fused pass with the most time).
    # Algorithmic bytes: every pass reads and writes the state once, except the
    # first, which creates the basis start in registers and only writes.
    peaks, peak_src = measured_peaks()
    state_bytes = T * (1 << n) * esize
    first_kind = order_kinds[0] if order_kinds else None
    dom = max((k for k in kern if k.startswith("pass")), key=lambda k: sum(kern[k]))
    per_launch = {k: statistics.mean(v) for k, v in kern.items()}
    bytes_per_pass = state_bytes if dom == first_kind else 2 * state_bytes
    avg_ms = statistics.mean(kern[dom])
    achieved = bytes_per_pass / (avg_ms / 1e3) / 1e9
    traffic = ncu_traffic(dom)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
                "kernel": "k_pass_high" if dom == "pass_high" else "k_pass_low",
                "algorithmic_bytes_per_launch": bytes_per_pass, "avg_launch_ms": round(avg_ms, 4),
                "peak_source": f"{peak_src} hbm_gbs (copy bandwidth)",
                "launch_ms_by_kind": {k: round(v, 4) for k, v in per_launch.items()}}

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if dtype == qs.QS_C64 else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "circuit": W.circuit, "n": n, "trajectories_per_gpu": T,
                   "gates": len(ops), "e": e, "noise": "rotation (H), phase (CP), Philox on device",
                   "passes_per_step": passes, "parallelism": f"trajectories sharded over {world} GPU(s)",
                   "kernel_config": {"window": window, "low": kernel_cfg[0], "high": kernel_cfg[1],
                                     "autotune_ms": [round(x, 4) for x in tune_ms]},
                   "circuits_per_s": T * world / (ms_per_step / 1e3),
                   "state_bytes": T * (1 << n) * esize,
                   "l2": "inputs larger than L2 (state of every step is %d MiB)" % (T * (1 << n) * esize >> 20),
                   "fidelity_mean": float(np.mean(fid)), "fidelity_min": float(np.min(fid))},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(xs.nbytes + e_arr.nbytes + s_arr.nbytes + t_arr.nbytes),
                "d2h_bytes_per_step": int(fid.nbytes), "ms_per_step": t_e2e * 1e3},
        "gpu_launches": args.steps * (launches + 1),
        "roofline": roofline,
    }
    if not args.no_extras and world == 1:
        # the other rows are measured on the single-GPU run only
        result["rows"] = extra_rows(h, n, T, esize, stream, peaks)
    qs.qs_plan_destroy(p)
    qs.qs_destroy(h)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(W, ops, x0, fid[0])
    if dist is not None:
        dist.destroy_process_group()
    return result


def _oracle_trajectory(args):
    """One oracle trajectory (a worker of the all-core baseline)."""
    n, ops, x0, e, seed, traj = args
    from oracle import circuits as ocirc
    return ocirc.run_trajectory(n, ops, x0, e, seed, traj)


def cpu_baseline(W, ops, x0, gpu_fid0):
    """The oracle as it stands, on the host: whole trajectories of the workload,
    one per host core in parallel (trajectories are independent), and one on a
    single thread.

    Trajectory 0 was also run on the GPU in complex64; the difference of the
    two fidelities is the error of the GPU result against the FP64 oracle."""
    import multiprocessing as mp

    from oracle import circuits as ocirc
    from oracle import statevec as osv
    t0 = time.perf_counter()
    psi = ocirc.run_trajectory(W.n, ops, x0, W.e, W.seed, 0)
    dt1 = time.perf_counter() - t0
    f0 = osv.fidelity(ocirc.ideal_state(W.n, ops, x0), psi)
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_trajectory, [(W.n, [], x0, W.e, W.seed, 0)] * cores)   # workers up
        t0 = time.perf_counter()
        pool.map(_oracle_trajectory, [(W.n, ops, x0, W.e, W.seed, b) for b in range(cores)])
        dtn = time.perf_counter() - t0
    upd = (1 << W.n) * len(ops)
    return {"value": upd * cores / dtn, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} of {W.trajectories} trajectories of {W.name}, one per core (complex128 NumPy, "
                      f"spawned processes), {dtn:.1f} s",
            "single_thread_value": upd / dt1, "single_thread_s": round(dt1, 2),
            "fidelity_oracle": f0, "fidelity_gpu": float(gpu_fid0), "fidelity_abs_error": abs(f0 - float(gpu_fid0))}


def extra_rows(h, n, T, esize, stream, peaks):
    """Bounded measurements of the other hot-path rows (a few seconds each)."""
    import numpy as np
    import torch

    from paper_1412_2293_gb300 import circuits as pcirc
    from paper_1412_2293_gb300 import inputs, qs

    out = {}
    ev = lambda: torch.cuda.Event(enable_timing=True)

    # a1: single-gate pair sweep over the whole batched state (one HBM read + write per gate)
    Hm = pcirc.hadamard()
    for t in (0, 7, 19):
        qs.qs_apply_gate(h, (t,), Hm)
    e0, e1 = ev(), ev()
    torch.cuda.synchronize()
    e0.record(stream)
    targets = [0, 3, 7, 12, 19, 5, 16, 9]
    for t in targets:
        qs.qs_apply_gate(h, (t,), Hm)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / len(targets)
    gbs = 2 * T * (1 << n) * esize / (ms / 1e3) / 1e9
    out["a1_pair_sweep"] = {"kernel": "k_apply_1q", "state_bytes": T * (1 << n) * esize, "ms_per_gate": round(ms, 4),
                            "achieved_GBps": round(gbs, 1), "frac_of_measured_hbm": round(gbs / peaks["hbm_gbs"], 4),
                            "targets": targets}

    # f1: dense k-qubit blocks (k = 3..5) over the whole batch, complex64: the tcgen05 path
    # (split-tf32 GEMM) against the CUDA-core sweep; the state (8 GiB) is larger than L2
    rng = np.random.default_rng(inputs.DEFAULT_SEED)
    f1 = {}
    tf32_peak = peaks["bf16_tflops"] * 1.1 / 2.25          # nominal tf32 / bf16 dense ratio
    for k, targets in ((3, (2, 9, 15)), (4, (1, 6, 12, 18)), (5, (3, 9, 14, 17, 19))):
        d = 1 << k
        U, _ = np.linalg.qr(rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d)))
        row = {}
        for tc in (True, False):
            qs.qs_set_tensor_cores(h, tc)
            qs.qs_apply_gate(h, targets, U)
            e0, e1 = ev(), ev()
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(3):
                qs.qs_apply_gate(h, targets, U)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 3
            gbs = 2 * T * (1 << n) * esize / (ms / 1e3) / 1e9
            row["tensor_cores" if tc else "cuda_cores"] = {
                "ms": round(ms, 3), "achieved_GBps": round(gbs, 1),
                "frac_of_measured_hbm": round(gbs / peaks["hbm_gbs"], 4)}
        flops = 3 * 8 * d * T * (1 << n)      # three tf32 products of (groups x 2d) by (2d x 2d)
        tcr = row["tensor_cores"]
        tcr["tf32_TFLOPs"] = round(flops / (tcr["ms"] / 1e3) / 1e12, 1)
        tcr["frac_of_tf32_peak"] = round(tcr["tf32_TFLOPs"] / tf32_peak, 4)
        row["targets"] = targets
        f1[f"k{k}"] = row
    qs.qs_set_tensor_cores(h, True)
    out["f1_dense_blocks"] = {"kernel": "k_dense_tc", "state_bytes": T * (1 << n) * esize, "members": T, "qubits": n,
                              "tf32_peak_TFLOPs": round(tf32_peak, 1),
                              "tf32_peak_basis": "measured bf16 dense x 1.1/2.25 (nominal tf32/bf16)", **f1}

    # plain FP64 one trajectory per launch sequence vs batched complex64 (Grover n = 10)
    W1 = inputs.WORKLOADS["mc_grover_n10_c128"]
    ops1, x1 = W1.ops(), W1.initial_basis()
    marked = inputs.draw_marked(W1.n, W1.seed)
    hp = qs.qs_create(W1.n, 1, 0, qs.QS_STATEVEC, qs.QS_C128, stream)
    plain_f = []
    reps = 3
    t0 = time.perf_counter()
    for b in range(reps):
        qs.qs_set_trajectory_offset(hp, b)
        qs.qs_set_basis_state(hp, x1)
        pcirc.apply_ops(hp, ops1, W1.e, W1.seed)
        plain_f.append(float(qs.qs_fidelity(hp, None, marked)[0]))
    dt_plain = (time.perf_counter() - t0) / reps
    qs.qs_destroy(hp)
    hb = qs.qs_create(W1.n, 1024, 0, qs.QS_STATEVEC, qs.QS_C64, stream)
    pb = qs.qs_plan_create(hb, pcirc.to_gates(ops1))
    qs.qs_set_basis_state(hb, x1)
    qs.qs_plan_run(pb, W1.e, W1.seed, 0, hb)
    qs.qs_synchronize(hb)
    t0 = time.perf_counter()
    for _ in range(reps):
        qs.qs_set_basis_state(hb, x1)
        qs.qs_plan_run(pb, W1.e, W1.seed, 0, hb)
        fb = qs.qs_fidelity(hb, None, marked)
    dt_batch = (time.perf_counter() - t0) / reps
    passes, _ = qs.qs_plan_info(pb, hb)
    qs.qs_plan_destroy(pb)
    qs.qs_destroy(hb)
    err = max(abs(fb[b] - plain_f[b]) for b in range(reps))
    # Fig. 1's quantity: the distribution of 1 - p over the trajectories, and Eq. 10's
    # rank-1 value lambda_1^(n + 2nk) sin^2((2k+1) asin 2^(-n/2)) beside its mean
    k1 = W1.extra.get("iterations", inputs.grover_iterations(W1.n))
    lam1 = (1.0 + math.exp(-2.0 * W1.e * W1.e)) / 2.0
    eq10 = lam1 ** (W1.n + 2 * W1.n * k1) * math.sin((2 * k1 + 1) * math.asin(2.0 ** (-W1.n / 2.0))) ** 2
    fbn = np.asarray(fb)
    out["plain_vs_batched_grover_n10"] = {
        "plain_c128_gate_by_gate_circuits_per_s": round(1.0 / dt_plain, 2),
        "batched_c64_fused_circuits_per_s": round(1024 / dt_batch, 1),
        "speedup": round((1024 / dt_batch) * dt_plain, 1), "fused_passes": passes,
        "success_prob_max_abs_diff_c64_vs_c128": err, "gates": len(ops1), "iterations": k1,
        "success_prob_mean": float(fbn.mean()), "success_prob_stderr": float(fbn.std() / math.sqrt(len(fbn))),
        "one_minus_p_p5_p50_p95": [float(x) for x in np.percentile(1.0 - fbn, [5, 50, 95])],
        "eq10": eq10}

    # a6: exact density matrix of the noisy QFT, n = 14 (2^28 entries): complex128 (FP64 pipe
    # bound on this GPU) and complex64 (HBM bound), the fidelity of each with the ideal output
    W4 = inputs.WORKLOADS["dm_qft_n14"]
    ops4, x4 = W4.ops(), W4.initial_basis()
    a6 = {}
    for dt, name in ((qs.QS_C128, "c128"), (qs.QS_C64, "c64")):
        hd = qs.qs_create(W4.n, 1, 0, qs.QS_DENSITY, dt, stream)
        hi4 = pcirc.ideal_reference(W4.n, ops4, x4, dt, stream)
        qs.qs_set_basis_state(hd, x4)
        pcirc.apply_ops(hd, ops4[:3], W4.e, W4.seed)
        qs.qs_synchronize(hd)
        qs.qs_set_basis_state(hd, x4)
        # the circuit as a plan: runs of diagonal channels (the controlled phases after each
        # Hadamard) become one sweep each
        pd4 = qs.qs_plan_create(hd, pcirc.to_gates(ops4))
        e0, e1 = ev(), ev()
        torch.cuda.synchronize()
        e0.record(stream)
        qs.qs_plan_run(pd4, W4.e, W4.seed, 0, hd)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_dm = e0.elapsed_time(e1)
        _, dm_launches = qs.qs_plan_info(pd4, hd)
        qs.qs_plan_destroy(pd4)
        qs.qs_set_reference_from(hd, hi4, 0)
        a6[name] = {"ms_per_circuit": round(ms_dm, 2), "launches": dm_launches,
                    "trace": float(qs.qs_trace(hd)[0]), "fidelity": float(qs.qs_fidelity_stored(hd)[0]),
                    "updates_per_s": (1 << (2 * W4.n)) * len(ops4) / (ms_dm / 1e3)}
        qs.qs_destroy(hi4)
        qs.qs_destroy(hd)
    out["a6_density_qft_n14"] = {"channels": len(ops4), "entries": 1 << (2 * W4.n), **a6,
                                 "fidelity_c64_minus_c128": a6["c64"]["fidelity"] - a6["c128"]["fidelity"]}

    # a7: fixed-rank Grover n = 16 as a plan (the circuit replayed as one CUDA graph): the
    # first 208 channels timed per rank r = 1, 2, 4, 8 (one job), the same with 8 jobs of
    # ranks 1..8 batched in one handle (a9: rank columns of uneven sizes in one launch), and
    # the whole circuit at r = 1 against Eq. 10: F = lambda1^(n + 2nk) p_ideal
    W3 = inputs.WORKLOADS["rank_grover_n16"]
    ops3 = W3.ops()
    sub = ops3[:16 + 6 * 34]
    noisy = sum(1 for o in sub if o.noisy)
    total_noisy = sum(1 for o in ops3 if o.noisy)

    def rank_plan_ms(ops_, B, ranks):
        hr = qs.qs_create(W3.n, B, max(ranks), qs.QS_FIXED_RANK, qs.QS_C128, stream)
        qs.qs_set_member_ranks(hr, ranks)
        pr = qs.qs_plan_create(hr, pcirc.to_gates(ops_))
        for _ in range(2):                               # the second run replays the captured graph
            qs.qs_set_basis_state(hr, 0)
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record(stream)
            qs.qs_plan_run(pr, W3.e, W3.seed, 0, hr)
            e1.record(stream)
            torch.cuda.synchronize()
        qs.qs_plan_destroy(pr)
        return e0.elapsed_time(e1), hr

    sweep = {}
    for r in (1, 2, 4, 8):
        ms_r, hr = rank_plan_ms(sub, 1, [r])
        qs.qs_destroy(hr)
        sweep[f"r{r}_ms_per_channel"] = round(ms_r / noisy, 4)
    ranks8 = [1, 2, 3, 4, 5, 6, 7, 8]
    ms_b, hr = rank_plan_ms(sub, 8, ranks8)
    qs.qs_destroy(hr)
    sweep["batched_8_jobs_r1_to_8"] = {"ms_per_channel": round(ms_b / noisy, 4),
                                      "ms_per_job_channel": round(ms_b / noisy / 8, 4)}
    ms_full, hr = rank_plan_ms(ops3, 1, [1])
    marked3 = inputs.draw_marked(W3.n, W3.seed)
    k3 = inputs.grover_iterations(W3.n)
    p_r1 = float(qs.qs_fidelity(hr, None, marked3)[0])
    qs.qs_destroy(hr)
    lam1 = (1.0 + math.exp(-2.0 * W3.e ** 2)) / 2.0
    p_eq10 = lam1 ** (W3.n + 2 * W3.n * k3) * math.sin((2 * k3 + 1) * math.asin(2.0 ** (-W3.n / 2))) ** 2
    sweep.update({"channels_timed": noisy, "circuit_channels": total_noisy,
                  "r1_whole_circuit_s": round(ms_full / 1e3, 4), "r1_success_probability": p_r1, "eq10": p_eq10,
                  "r1_rel_diff_from_eq10": abs(p_r1 - p_eq10) / p_eq10,
                  "note": "plan runs (expansion, FP64 Gram, eigensolver, projection per channel, one CUDA graph)"})
    out["a7_fixed_rank_grover_n16"] = sweep

    # a6 vs a7: exact density matrix and fixed rank r = 1..8 on the QFT n = 14, |F_r - F_exact|
    href = pcirc.ideal_reference(W4.n, ops4, x4, qs.QS_C128, stream)
    phi = qs.qs_get_state(href)
    qs.qs_destroy(href)
    hd = qs.qs_create(W4.n, 1, 0, qs.QS_DENSITY, qs.QS_C128, stream)
    qs.qs_set_basis_state(hd, x4)
    pcirc.apply_ops(hd, ops4, W4.e, W4.seed)
    f_exact = float(qs.qs_fidelity(hd, phi)[0])
    qs.qs_destroy(hd)
    cmp = {"f_exact": f_exact}
    for r in (1, 2, 4, 8):
        hr = qs.qs_create(W4.n, 1, r, qs.QS_FIXED_RANK, qs.QS_C128, stream)
        qs.qs_set_basis_state(hr, x4)
        e0, e1 = ev(), ev()
        e0.record(stream)
        pcirc.apply_ops(hr, ops4, W4.e, W4.seed)
        e1.record(stream)
        f_r = float(qs.qs_fidelity(hr, phi)[0])
        cmp[f"r{r}"] = {"f": f_r, "abs_diff": abs(f_r - f_exact), "ms_per_circuit": round(e0.elapsed_time(e1), 2)}
        qs.qs_destroy(hr)
    out["dm_vs_fixed_rank_qft_n14"] = cmp

    # a9: window width m of the passes.  The noisy QFT at n = 20 (this run's 1024
    # trajectories) and n = 24 (64 trajectories, 8 GiB): each width with its default
    # kernel configuration, passes per step and the HBM floor of those passes, then the
    # width and configurations the autotuner picks on a fresh plan
    Wq = inputs.WORKLOADS["mc_qft_n20_c64"]
    a9 = {}
    for nq, Tq in ((Wq.n, T), (24, 64)):
        opsq = inputs.qft_circuit(nq)
        xq = inputs.draw_basis_input(nq, Wq.seed)
        hq = qs.qs_create(nq, Tq, 0, qs.QS_STATEVEC, qs.QS_C64, stream)
        refq = pcirc.ideal_reference(nq, opsq, xq, qs.QS_C64, stream)
        qs.qs_set_reference_from(hq, refq, 0)
        qs.qs_destroy(refq)
        sb = Tq * (1 << nq) * 8
        row = {"trajectories": Tq, "state_bytes": sb}
        fm = {}
        for m in (10, 11, 12):
            pq = qs.qs_plan_create(hq, pcirc.to_gates(opsq))
            qs.qs_plan_set_window(pq, m, hq)
            npass, _ = qs.qs_plan_info(pq, hq)
            for _ in range(2):
                qs.qs_set_basis_state(hq, xq)
                qs.qs_plan_run_fidelity(pq, Wq.e, Wq.seed, 0, hq)
            e0, e1 = ev(), ev()
            reps = 5
            e0.record(stream)
            for _ in range(reps):
                qs.qs_set_basis_state(hq, xq)
                fq = qs.qs_plan_run_fidelity(pq, Wq.e, Wq.seed, 0, hq)
            e1.record(stream)
            torch.cuda.synchronize()
            msq = e0.elapsed_time(e1) / reps
            qs.qs_plan_destroy(pq)
            fm[m] = np.asarray(fq)
            floor = (2 * npass - 1) * sb / (peaks["hbm_gbs"] * 1e9) * 1e3    # the first pass only writes
            row[f"m{m}"] = {"passes": npass, "ms_per_step": round(msq, 3), "hbm_floor_ms": round(floor, 3),
                            "frac_of_floor": round(floor / msq, 4), "fidelity_mean": float(fm[m].mean())}
        row["fidelity_max_abs_diff_vs_m10"] = max(float(np.abs(fm[m] - fm[10]).max()) for m in (11, 12))
        pq = qs.qs_plan_create(hq, pcirc.to_gates(opsq))
        qs.qs_set_basis_state(hq, xq)
        tl, th = qs.qs_plan_autotune(pq, 2, Wq.e, Wq.seed, hq)
        row["autotuned"] = {"window": qs.qs_plan_get_window(pq, hq), "config": list(qs.qs_plan_get_config(pq, hq)),
                            "pass_ms": [round(tl, 4), round(th, 4)]}
        qs.qs_plan_destroy(pq)
        qs.qs_destroy(hq)
        a9[f"qft_n{nq}"] = row
    out["a9_window_width"] = a9

    # a3 at the other precision and noise level of the bench circuit: complex128 on the
    # same 1024 trajectories (16 GiB), compared member by member with the complex64 run,
    # and complex64 at e = 0.001; each on a fresh handle (no per-member inputs left over)
    Wq = inputs.WORKLOADS["mc_qft_n20_c64"]
    opsq, xq = Wq.ops(), Wq.initial_basis()
    fids = {}
    for label, dtype_, Tq, eq in (("mc_qft_n20_c64_e1e-2", qs.QS_C64, T, Wq.e),
                                  ("mc_qft_n20_c128", qs.QS_C128, T, Wq.e),
                                  ("mc_qft_n20_c64_e1e-3", qs.QS_C64, T, 0.001)):
        hq = qs.qs_create(Wq.n, Tq, 0, qs.QS_STATEVEC, dtype_, stream)
        refq = pcirc.ideal_reference(Wq.n, opsq, xq, dtype_, stream)
        qs.qs_set_reference_from(hq, refq, 0)
        qs.qs_destroy(refq)
        pq = qs.qs_plan_create(hq, pcirc.to_gates(opsq))
        qs.qs_set_basis_state(hq, xq)
        qs.qs_plan_autotune(pq, 1, eq, Wq.seed, hq)
        for _ in range(2):
            qs.qs_set_basis_state(hq, xq)
            fq = qs.qs_plan_run_fidelity(pq, eq, Wq.seed, 0, hq)
        e0, e1 = ev(), ev()
        e0.record(stream)
        reps = 5
        for _ in range(reps):
            qs.qs_set_basis_state(hq, xq)
            fq = qs.qs_plan_run_fidelity(pq, eq, Wq.seed, 0, hq)
        e1.record(stream)
        torch.cuda.synchronize()
        msq = e0.elapsed_time(e1) / reps
        qs.qs_plan_destroy(pq)
        qs.qs_destroy(hq)
        fids[label] = np.asarray(fq)
        # Eq. 11, P_H^n P_R^{n(n-1)/8} with P_H = (1 + exp(-2 e^2)) / 2 and
        # P_R = exp(-e^2), a geometric-mean estimate a little below the mean
        est = (0.5 * (1.0 + math.exp(-2.0 * eq * eq))) ** Wq.n * math.exp(-eq * eq) ** (Wq.n * (Wq.n - 1) / 8.0)
        assert est - 1e-3 < float(np.mean(fq)) <= 1.0, (label, float(np.mean(fq)), est)
        out[label] = {"ms_per_step": round(msq, 3), "trajectories": Tq, "e": eq,
                      "updates_per_s": Tq * (1 << Wq.n) * len(opsq) / (msq / 1e3),
                      "fidelity_mean": float(np.mean(fq)), "eq11_estimate": est}
    d = np.abs(fids["mc_qft_n20_c64_e1e-2"] - fids["mc_qft_n20_c128"])
    out["mc_qft_n20_c128"]["c64_vs_c128_fidelity_abs_diff"] = {"max": float(d.max()), "mean": float(d.mean())}
    out["mc_qft_n20_c128"]["c64_vs_c128_circuits_per_s_ratio"] = round(
        out["mc_qft_n20_c128"]["ms_per_step"] / out["mc_qft_n20_c64_e1e-2"]["ms_per_step"], 3)

    # f3: Choi-Jamiolkowski relative state of the noisy QFT on 7 system qubits (Sec. 4): the
    # exact relative state (density matrix of 14 qubits, 4 GiB) and 1024 Monte Carlo
    # trajectories of the 14-qubit entangled start through the fused passes
    m7, e7 = 7, 0.01
    ops7 = inputs.qft_circuit(m7)
    hi7 = qs.qs_create(2 * m7, 1, 0, qs.QS_STATEVEC, qs.QS_C128, stream)
    qs.qs_set_maximally_entangled(hi7)
    p7 = qs.qs_plan_create(hi7, pcirc.to_gates([inputs.Op(o.kind, o.qubits, o.theta, o.index, False) for o in ops7]))
    qs.qs_plan_run(p7, 0.0, 0, 0, hi7)
    qs.qs_plan_destroy(p7)
    psi7 = qs.qs_get_state(hi7)
    hd7 = qs.qs_create(2 * m7, 1, 0, qs.QS_DENSITY, qs.QS_C128, stream)
    qs.qs_set_maximally_entangled(hd7)
    e0, e1 = ev(), ev()
    e0.record(stream)
    pcirc.apply_ops(hd7, ops7, e7, inputs.DEFAULT_SEED)
    e1.record(stream)
    f_dm7 = float(qs.qs_fidelity(hd7, psi7)[0])
    ms_dm7 = e0.elapsed_time(e1)
    qs.qs_destroy(hd7)
    T7 = 1024
    hm7 = qs.qs_create(2 * m7, T7, 0, qs.QS_STATEVEC, qs.QS_C64, stream)
    pm7 = qs.qs_plan_create(hm7, pcirc.to_gates(ops7))
    qs.qs_set_maximally_entangled(hm7)
    qs.qs_plan_run(pm7, e7, inputs.DEFAULT_SEED, 0, hm7)
    qs.qs_set_maximally_entangled(hm7)
    e0, e1 = ev(), ev()
    e0.record(stream)
    qs.qs_plan_run(pm7, e7, inputs.DEFAULT_SEED, 0, hm7)
    e1.record(stream)
    f_mc7 = qs.qs_fidelity(hm7, psi7)
    ms_mc7 = e0.elapsed_time(e1)
    qs.qs_plan_destroy(pm7)
    qs.qs_destroy(hm7)
    qs.qs_destroy(hi7)
    out["f3_relative_state_qft_m7"] = {
        "system_qubits": m7, "e": e7, "fidelity_exact": f_dm7, "density_ms": round(ms_dm7, 2),
        "fidelity_mc_mean": float(np.mean(f_mc7)), "fidelity_mc_stderr": float(np.std(f_mc7) / math.sqrt(T7)),
        "mc_trajectories": T7, "mc_ms": round(ms_mc7, 3),
        "mc_minus_exact_in_stderr": float((np.mean(f_mc7) - f_dm7) / max(np.std(f_mc7) / math.sqrt(T7), 1e-300))}

    # f2: the rank-1 estimates of Fig. 4 for the noisy QFT, n = 12, e = 0.01: exact fidelity
    # (density matrix), rank 1 by the direct and the rotated (Eqs. 12-14) branch, and the closed
    # forms Eq. 11 (P_H^n P^(n(n-1)/8)) and Eq. 15 (P_H^n P~_R^(n(n-1)/8))
    n12, e12, x12 = 12, 0.01, 5
    ops12 = inputs.qft_circuit(n12)
    hi12 = pcirc.ideal_reference(n12, ops12, x12, qs.QS_C128, stream)
    phi12 = qs.qs_get_state(hi12)
    qs.qs_destroy(hi12)
    hd12 = qs.qs_create(n12, 1, 0, qs.QS_DENSITY, qs.QS_C128, stream)
    qs.qs_set_basis_state(hd12, x12)
    pcirc.apply_ops(hd12, ops12, e12, inputs.DEFAULT_SEED)
    f_exact12 = float(qs.qs_fidelity(hd12, phi12)[0])
    qs.qs_destroy(hd12)
    branch = {}
    for rotated in (False, True):
        hb = qs.qs_create(n12, 1, 0, qs.QS_STATEVEC, qs.QS_C128, stream)
        qs.qs_set_basis_state(hb, x12)
        pcirc.apply_branch_ops(hb, ops12, e12, rotated)
        branch["improved" if rotated else "direct"] = float(qs.qs_fidelity(hb, phi12)[0])
        qs.qs_destroy(hb)
    P12 = math.exp(-e12 * e12)
    PH = (1.0 + math.exp(-2.0 * e12 * e12)) / 2.0
    f12 = (math.sqrt(1.0 + 3.0 * P12) - P12 - 1.0) / math.sqrt(P12 * (1.0 - P12))
    PR = (math.sqrt(P12) + f12 * math.sqrt(1.0 - P12)) ** 2 / (1.0 + f12 * f12) ** 4
    ncp = n12 * (n12 - 1) / 8.0
    out["f2_rank1_estimates_qft_n12"] = {
        "e": e12, "fidelity_exact": f_exact12, "rank1_direct": branch["direct"], "rank1_improved": branch["improved"],
        "eq11": PH ** n12 * P12 ** ncp, "eq15": PH ** n12 * PR ** ncp}

    # f4: T1/T2 relaxation of every qubit of a 14-qubit complex64 density matrix (2^28 entries,
    # 2.1 GB, larger than L2; two qubits per sweep, one read and one write of rho each), then the
    # relative-state fidelities of Sec. 4.1-4.3 through the same calls
    from paper_1412_2293_gb300 import codes
    n14, relax = 14, (0.01, 3.0, 2.0)
    hr = qs.qs_create(n14, 1, 0, qs.QS_DENSITY, qs.QS_C64, stream)
    qs.qs_set_maximally_entangled(hr)
    allq = list(range(n14))
    qs.qs_apply_relaxation(hr, allq, *relax)
    reps = 3
    e0, e1 = ev(), ev()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        qs.qs_apply_relaxation(hr, allq, *relax)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_relax = e0.elapsed_time(e1) / reps
    tr_relax = float(qs.qs_trace(hr)[0])
    qs.qs_destroy(hr)
    sweeps = (n14 + 1) // 2
    sweep_bytes = 2 * (1 << (2 * n14)) * 8
    gbs = sweep_bytes * sweeps / (ms_relax / 1e3) / 1e9
    t0 = time.perf_counter()
    p_grid = [0.01, 0.05, 0.1, 0.2, 0.3]
    phase3 = [codes.code_relative_fidelity("phase3", ("phase", p)) for p in p_grid]
    shor9 = [codes.code_relative_fidelity("shor9", ("phase", p)) for p in p_grid[:3]]
    fig8 = {"uncoded": codes.uncoded_relative_fidelity(("relax", 1.0, 3.0, 2.0), gate=np.diag([1.0, -1.0])),
            "phase3": codes.code_relative_fidelity("phase3", ("relax", 1.0, 3.0, 2.0), logical_z=True),
            "shor9": codes.code_relative_fidelity("shor9", ("relax", 1.0, 3.0, 2.0), logical_z=True)}
    ms_codes = (time.perf_counter() - t0) * 1e3
    t0 = time.perf_counter()
    g5 = codes.qft_gates(5)
    fig9 = {f"T1={T1:g},T2={T2:g}": codes.circuit_relaxation_fidelity(5, g5, 0.1, T1, T2)
            for T1 in (1.0, 5.0, 20.0) for T2 in (1.0, 2.0, 10.0) if T2 <= 2 * T1}
    ms_fig9 = (time.perf_counter() - t0) * 1e3
    out["f4_relaxation_and_codes"] = {
        "kernel": "k_dm_relax", "qubits": n14, "dtype": "c64", "t_T1_T2": relax, "sweeps_per_call": sweeps,
        "bytes_per_sweep": sweep_bytes, "ms_all_qubits": round(ms_relax, 3),
        "achieved_GBps": round(gbs, 1), "frac_of_measured_hbm": round(gbs / peaks["hbm_gbs"], 4),
        "trace_after": tr_relax,
        "phase3_p": p_grid, "phase3_fidelity": phase3,
        "eq18_fmin_squared": [1.0 - 3.0 * p * p + 2.0 * p ** 3 for p in p_grid],
        "shor9_fidelity": shor9, "codes_ms": round(ms_codes, 1),
        "fig8_logical_z_T1_3_T2_2": fig8, "fig9_qft5_t0.1": fig9, "fig9_ms": round(ms_fig9, 1)}

    # the largest single-GPU state vector: one noisy QFT trajectory on 34 qubits (128 GiB
    # complex64, four fused passes); its fidelity |<QFT x|psi>|^2 is read as the overlap with |x>
    # after the ideal inverse circuit
    n34, x34, e34 = 34, 0x2B7E15162, 0.01
    ops34 = inputs.qft_circuit(n34)
    h34 = qs.qs_create(n34, 1, 0, qs.QS_STATEVEC, qs.QS_C64, stream)
    try:
        p34 = qs.qs_plan_create(h34, pcirc.to_gates(ops34))
        inv34 = qs.qs_plan_create(h34, pcirc.to_gates(
            [inputs.Op(o.kind, o.qubits, -o.theta, o.index, False) for o in reversed(ops34)]))
        passes34, _ = qs.qs_plan_info(p34, h34)
        qs.qs_set_basis_state(h34, x34)
        e0, e1 = ev(), ev()
        torch.cuda.synchronize()
        e0.record(stream)
        qs.qs_plan_run(p34, e34, inputs.DEFAULT_SEED, 0, h34)
        e1.record(stream)
        torch.cuda.synchronize()
        ms34 = e0.elapsed_time(e1)
        qs.qs_plan_run(inv34, 0.0, 0, 0, h34)
        f34 = float(qs.qs_fidelity(h34, None, x34)[0])
        qs.qs_plan_destroy(inv34)
        qs.qs_plan_destroy(p34)
    finally:
        qs.qs_destroy(h34)
    out["mc_qft_n34_one_trajectory"] = {
        "qubits": n34, "state_GiB": 2 ** 34 * 8 / 2 ** 30, "gates": len(ops34), "passes": passes34, "e": e34,
        "ms_per_circuit": round(ms34, 1), "updates_per_s": (1 << n34) * len(ops34) / (ms34 / 1e3),
        "pass_GBps": round(passes34 * 2 * (1 << n34) * 8 / (ms34 / 1e3) / 1e9, 1), "fidelity": f34}

    out["a11_serving_full_range"] = serving_full_range_row()
    out["a11_serving"] = serving_row()
    cap = out["a11_serving"]["jobs_per_s"]
    out["a11_serving_rate_sweep"] = {f"{m}x_capacity": serving_row(num_jobs=60, rate_per_s=m * cap, seed_offset=1)
                                     for m in (0.5, 1.0, 2.0)}
    return out


def serving_row(num_jobs=100, rate_per_s=200.0, workers=4, seed_offset=0):
    """Continuous batching of a mixed stream of fidelity-estimation jobs.

    Poisson arrivals of Grover and QFT jobs, half Monte Carlo (2^6..2^10
    complex64 trajectories) and half fixed rank (r <= 8, complex128), n from 12
    to 20, e log-uniform in [1e-4, 1e-2].  Wall-clock throughput and latency
    from arrival to the job's last fidelity on the host."""
    from paper_1412_2293_gb300 import inputs
    from paper_1412_2293_gb300.server import GpuExecutor, Server, run_stream
    jobs = inputs.draw_job_stream(num_jobs, rate_per_s, seed=inputs.DEFAULT_SEED + seed_offset, n_range=(12, 20),
                                  log2_traj_range=(6, 10), max_rank=8)
    srv = Server(GpuExecutor(workers=workers), max_members=1024)
    try:
        _, stats = run_stream(jobs, srv, time_scale=1.0, timeout=600)
        units, max_run = srv.sched._uid, srv.sched.max_in_flight
    finally:
        srv.close()
    mc = [j for j in jobs if j.mode == "statevec"]
    return {"jobs": stats["jobs"], "mc_jobs": len(mc), "fixed_rank_jobs": len(jobs) - len(mc),
            "circuits": stats["circuits"], "arrival_rate_per_s": rate_per_s, "workers": workers,
            "launch_units": units, "max_units_in_flight": max_run,
            "span_s": round(stats["span_s"], 3), "circuits_per_s": round(stats["circuits_per_s"], 1),
            "jobs_per_s": round(stats["jobs_per_s"], 2), "latency_p50_s": round(stats["latency_p50_s"], 4),
            "latency_p99_s": round(stats["latency_p99_s"], 4),
            "stream": "n 12..20, MC 2^6..2^10 trajectories c64, fixed rank r 1..8 c128, Grover iterations capped at 16"}


def serving_full_range_row(num_jobs=24, rate_per_s=4.0, workers=4, limit_s=10.0):
    """The serving workload over its whole size range: n 12..28, Monte Carlo
    2^6..2^12 complex64 trajectories or fixed rank r 1..8 (complex128), Grover
    iterations capped at 16, Poisson arrivals; bounded by the job count.
    States up to 2 GiB per trajectory run in waves under the HBM budget.  A
    request whose estimated device time exceeds limit_s runs the largest
    power-of-two trajectory count that fits (Monte Carlo) or is refused (fixed
    rank); both are listed."""
    import numpy as np

    from paper_1412_2293_gb300 import inputs
    from paper_1412_2293_gb300.server import GpuExecutor, Server, estimate_seconds, run_stream
    jobs = inputs.draw_job_stream(num_jobs, rate_per_s, seed=inputs.DEFAULT_SEED + 2, n_range=(12, 28),
                                  log2_traj_range=(6, 12), max_rank=8)
    srv = Server(GpuExecutor(workers=workers), max_members=1024, limit_s=limit_s)
    try:
        res, stats = run_stream(jobs, srv, time_scale=1.0, timeout=900)
        budget, units = srv.sched.budget, srv.sched._uid
    finally:
        srv.close()
    byid = {j.job_id: j for j in jobs}
    shape = lambda j: (f"{j.circuit} n={j.n} " + (f"T={j.trajectories}" if j.mode == "statevec" else f"rank {j.rank}"))
    served = [byid[i] for i in res]
    lat = {m: [res[j.job_id].latency for j in served if j.mode == m] for m in ("statevec", "fixed_rank")}
    pct = lambda v, q: round(float(np.percentile(v, q)), 3) if v else None
    return {"stream": "n 12..28, MC 2^6..2^12 trajectories c64, fixed rank r 1..8 c128, Grover iterations "
                      "capped at 16, e log-uniform [1e-4, 1e-2]",
            "jobs_submitted": len(jobs), "jobs_served": stats["jobs"], "circuits": stats["circuits"],
            "span_s": round(stats["span_s"], 3), "circuits_per_s": round(stats["circuits_per_s"], 1),
            "jobs_per_s": round(stats["jobs_per_s"], 3),
            "latency_p50_s": round(stats["latency_p50_s"], 3), "latency_p99_s": round(stats["latency_p99_s"], 3),
            "mc_latency_p50_p99_s": [pct(lat["statevec"], 50), pct(lat["statevec"], 99)],
            "fixed_rank_latency_p50_p99_s": [pct(lat["fixed_rank"], 50), pct(lat["fixed_rank"], 99)],
            "served_n_range": [min(j.n for j in served), max(j.n for j in served)] if served else None,
            "served_trajectories_max": max((len(res[j.job_id].fidelities) for j in served if j.mode == "statevec"),
                                           default=0),
            "limit_s": limit_s,
            "reduced": {shape(byid[i]): {"served_trajectories": t, "estimate_s": round(estimate_seconds(byid[i]), 1)}
                        for i, (_, t) in stats["reduced"].items()},
            "refused": {shape(byid[i]): why for i, why in stats["refused"].items()},
            "launch_units": units, "hbm_budget_GiB": round(budget / 2 ** 30, 1),
            "peak_budget_used_GiB": round(stats["peak_budget_used"] / 2 ** 30, 1),
            "per_job": {f"{j.job_id}: {shape(j)}": {
                "latency_s": round(res[j.job_id].latency, 3), "estimate_s": round(estimate_seconds(j), 2),
                "served_trajectories": len(res[j.job_id].fidelities) if j.mode == "statevec" else None,
                "mean_fidelity": float(np.mean(res[j.job_id].fidelities))} for j in served}}


# ------------------------------------------------------------------ density / fixed rank


def run_channels(args, rank, world, local_rank):
    """Exact density matrix or fixed-rank workload: one step = the whole circuit
    (every noisy gate replaced by its xi-averaged Kraus channel) + the fidelity."""
    import numpy as np
    import torch

    from paper_1412_2293_gb300 import build as qbuild
    from paper_1412_2293_gb300 import circuits as pcirc
    from paper_1412_2293_gb300 import qs

    torch.cuda.set_device(local_rank)
    qbuild.build()
    W, ops, x0 = workload_setup(args.workload)
    n = W.n
    mode = qs.QS_DENSITY if W.mode == "density" else qs.QS_FIXED_RANK
    stream = torch.cuda.Stream()
    h = qs.qs_create(n, 1, W.rank, mode, qs.QS_C128, stream)
    ref = pcirc.ideal_reference(n, ops, x0, qs.QS_C128, stream)
    qs.qs_set_reference_from(h, ref, 0)
    qs.qs_destroy(ref)
    channels = sum(1 for o in ops if o.noisy)
    entries = (1 << (2 * n)) if mode == qs.QS_DENSITY else (1 << n) * W.rank
    updates_per_step = entries * len(ops)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    per_kind = {}
    plan = None
    # the circuit as a plan: density -- noisy H channels as single sweeps, each run of
    # diagonal channels as one sweep, timed per launch with events inside the captured
    # graph; fixed rank -- every gate on the device, the circuit replayed as one graph
    plan = qs.qs_plan_create(h, pcirc.to_gates(ops))
    if mode == qs.QS_DENSITY:
        qs.qs_plan_set_timing(plan, True, h)
    _, plan_kernels = qs.qs_plan_info(plan, h)

    def step(timed):
        qs.qs_set_basis_state(h, x0)
        if plan is not None:
            qs.qs_plan_run(plan, W.e, W.seed, 0, h)
            if timed and mode == qs.QS_DENSITY:
                for m, k in zip(*qs.qs_plan_last_times(plan, h=h)):
                    per_kind.setdefault("H_channel" if k == "single_gate" else k, []).append(m)
            return qs.qs_fidelity_stored(h)
        for g, op in enumerate(ops):
            if timed:
                a, b = ev(), ev()
                a.record(stream)
            pcirc.apply_ops(h, [op], W.e, W.seed, gate_id0=g)
            if timed:
                b.record(stream)
                kind = "flip" if op.kind == "FLIP" else (op.kind + ("_channel" if op.noisy else "_gate"))
                per_kind.setdefault(kind, []).append((a, b))
        return qs.qs_fidelity_stored(h)

    for _ in range(args.warmup):
        f = step(False)
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record(stream)
    for _ in range(args.steps):
        f = step(True)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    kinds = {k: statistics.mean(x if isinstance(x, float) else x[0].elapsed_time(x[1]) for x in v)
             for k, v in per_kind.items()}
    if plan is not None:
        qs.qs_plan_destroy(plan)
    if mode == qs.QS_DENSITY:
        # the kind of launch with the most time: the superoperator of a noisy H (a real 4x4
        # matrix l1 H (x) H + l2 HJ (x) HJ: 4 real-by-complex multiply-adds, 16 flop per entry)
        # or a run of diagonal channels (the factor u(x) conj(u(y)) sqrt(P)^k and its product
        # with the entry: two complex multiplications and a real scale, 14 flop per entry).
        # rho is Hermitian, so the algorithmic work is that of the entries on or above the
        # diagonal: half of it (the sweeps on qubits below 5 still do all of it)
        totals = {k: len(per_kind[k]) * kinds[k] for k in kinds}
        dom = max(totals, key=totals.get)
        flop = (1 << (2 * n)) * (14 if dom == "dm_diag_block" else 16) // 2
        bytes_ = 3 * (1 << (2 * n)) * 16 // 2
    else:
        # the whole step: every channel's Gram matrix (M(M+1)/2 pairs of columns) and
        # projection (M x keep) over 2^n rows, M = 2 m_prev and keep = min(r, M), the
        # column count doubling from 1 up to r; FP64 multiply-adds, 2 flop each for the
        # real factor of Grover (real arithmetic), 8 for a complex one
        dom = "fixed_rank_step"
        real = W.circuit == "grover"
        cols, fma = 1, 0
        for op in ops:
            if not op.noisy:
                continue
            M = 2 * cols
            keep = min(W.rank, M)
            fma += (1 << n) * (M * (M + 1) // 2 + M * keep)
            cols = keep
        flop = fma * (2 if real else 8)
        bytes_ = 3 * (1 << n) * W.rank * 16 * channels
        kinds = {"fixed_rank_step": ms}
    avg = kinds.get(dom, ms)
    achieved = flop / (avg / 1e3) / 1e12
    fp64_peak, _ = qs.qs_measure_peaks()
    out = {"metric": METRIC, "value": updates_per_step / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "mode": W.mode, "circuit": W.circuit, "n": n, "rank": W.rank,
                      "channels": channels, "gates": len(ops), "e": W.e, "circuits_per_s": 1e3 / ms,
                      "fidelity": float(f[0]), "trace": float(qs.qs_trace(h)[0])},
           # density: per step the plan's kernels, the start state, the fidelity's two reductions
           "gpu_launches": args.steps * (plan_kernels + 3) if plan is not None else None,
           "roofline": {"bound": "alu", "achieved": round(achieved, 4), "peak": round(fp64_peak, 4), "unit": "TFLOP/s",
                        "frac": round(achieved / fp64_peak, 4), "traffic": None,
                        "kernel": {"H_channel": "noisy-H channel (all its launches)",
                                   "dm_diag_block": "k_dm_diag_block (runs of diagonal channels)",
                                   "fixed_rank_step": "the whole circuit (expansion, Gram, eigensolver, "
                                                      "projection per channel)"}.get(dom, dom),
                        "avg_launch_ms": round(avg, 4),
                        "algorithmic_flop_per_launch": flop, "algorithmic_bytes_per_launch": bytes_,
                        "peak_source": "FP64 FMA rate measured live (qs_measure_peaks)",
                        "launch_ms_by_kind": {k: round(v, 4) for k, v in kinds.items()}}}
    qs.qs_destroy(h)
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_channels(W, ops, x0, updates_per_step)
    return out


def cpu_baseline_channels(W, ops, x0, updates_per_step, budget_s=15.0):
    """The oracle on one host thread for the density / fixed-rank workloads.

    Fixed rank: the circuit's gates in order at full size until the time
    budget is spent, extrapolated over the whole gate list.  Density: the
    complex128 matrix of the full size (4^n entries) is too slow for the
    oracle, so the same circuit family's gates run at 12 qubits in order, and
    the time per entry and gate is scaled to 4^n entries."""
    import numpy as np

    from oracle import circuits as ocirc
    from oracle import density as oden
    from oracle import fixed_rank as ofr
    from oracle import gates as ogates
    from oracle import statevec as osv
    from paper_1412_2293_gb300 import inputs

    def step_op(state, op, n, density):
        if op.kind == "FLIP":
            return oden.phase_flip(state, op.index) if density else ofr.phase_flip(state, op.index)
        U = ocirc.op_unitary(op)
        t = ocirc.op_targets(op)
        if op.noisy:
            kr = ogates.kraus_set(U, ocirc.op_noise(op), W.e)
            if density:
                return oden.apply_channel(state, n, t, kr)
            return ofr.truncate(ofr.apply_kraus(state, n, t, kr), W.rank)[0]
        return oden.apply_unitary(state, n, t, U) if density else ofr.apply_unitary(state, n, t, U)

    density = W.mode == "density"
    n_s = min(W.n, 12) if density else W.n
    ops_s = ops if n_s == W.n else (inputs.qft_circuit(n_s) if W.circuit == "qft" else
                                   inputs.grover_circuit(n_s, inputs.grover_iterations(n_s), 0))
    state = oden.pure(osv.basis_state(n_s, x0 % (1 << n_s))) if density else ofr.initial_factor(n_s, x0)
    t0 = time.perf_counter()
    count = 0
    for op in ops_s:
        state = step_op(state, op, n_s, density)
        count += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    entries_s = (1 << (2 * n_s)) if density else (1 << n_s) * W.rank
    per_update = dt / (count * entries_s)
    value = 1.0 / per_update
    if density and n_s != W.n:
        sample = (f"first {count} of {len(ops_s)} gates of the {W.circuit} circuit on {n_s} qubits "
                  f"(4^{n_s} entries, complex128 NumPy, one thread, {dt:.1f} s); time per entry and gate "
                  f"scaled to the 4^{W.n}-entry workload (extrapolated)")
    else:
        sample = (f"first {count} of {len(ops_s)} gates at full size (n = {W.n}, r = {W.rank}; complex128 "
                  f"NumPy, one thread, {dt:.1f} s), extrapolated over the circuit")
    return {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
            "circuit_s_extrapolated": updates_per_step / value}


# ------------------------------------------------------------------ single-kernel runs
MICRO = {
    # name: (what, qubits, members or None, k, targets)
    "dense_k5": ("dense", 20, 128, 5, (3, 9, 14, 17, 19)),
    "dense_k3": ("dense", 20, 128, 3, (2, 9, 15)),
    "relax_dm_n13": ("relax", 13, None, 0, ()),
    "dm_qft_n12": ("dmplan", 12, None, 0, ()),
}


def run_micro(args):
    """One kernel on its own, for a profiler: --warmup + --steps launches of a
    complex64 dense block (1 GiB batch) or of the density-matrix relaxation
    (13 qubits, 512 MiB), or runs of the noisy QFT plan on a 12-qubit
    complex128 density matrix (256 MiB: Hermitian channel sweeps and diagonal
    blocks); prints the mean time of the timed launches (runs)."""
    import numpy as np
    import torch

    from paper_1412_2293_gb300 import build, inputs, qs
    build.build()
    what, n, members, k, targets = MICRO[args.micro]
    stream = torch.cuda.current_stream()
    if what == "dense":
        h = qs.qs_create(n, members, 0, qs.QS_STATEVEC, qs.QS_C64, stream)
        qs.qs_set_basis_state(h, 0)
        qs.qs_apply_gate(h, (0,), np.array([[1, 1], [1, -1]]) / np.sqrt(2.0))
        rng = np.random.default_rng(inputs.DEFAULT_SEED)
        U, _ = np.linalg.qr(rng.normal(size=(1 << k, 1 << k)) + 1j * rng.normal(size=(1 << k, 1 << k)))
        launch = lambda: qs.qs_apply_gate(h, targets, U)
        nbytes = 2 * members * (1 << n) * 8
    elif what == "relax":
        h = qs.qs_create(n, 1, 0, qs.QS_DENSITY, qs.QS_C64, stream)
        qs.qs_set_basis_state(h, 0)
        launch = lambda: qs.qs_apply_relaxation(h, [0, 7], 0.05, 3.0, 2.0)
        nbytes = 2 * (1 << (2 * n)) * 8
    else:
        from paper_1412_2293_gb300 import circuits as pcirc
        h = qs.qs_create(n, 1, 0, qs.QS_DENSITY, qs.QS_C128, stream)
        plan = qs.qs_plan_create(h, pcirc.to_gates(inputs.qft_circuit(n)))
        _, nl = qs.qs_plan_info(plan, h)

        def launch():
            qs.qs_set_basis_state(h, 5)
            qs.qs_plan_run(plan, 0.01, inputs.DEFAULT_SEED, 0, h)
        nbytes = nl * 2 * (1 << (2 * n)) * 16
    for _ in range(args.warmup):
        launch()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        launch()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    qs.qs_destroy(h)
    return {"micro": args.micro, "ms_per_launch": round(ms, 4), "GBps": round(nbytes / (ms / 1e3) / 1e9, 1),
            "launches": args.warmup + args.steps}


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    """The oracle on the host cores, each step a slice of one trajectory's gates."""
    import numpy as np

    from oracle import circuits as ocirc
    from oracle import gates as ogates
    from oracle import philox as ophilox
    from oracle import statevec as osv

    if rank != 0:
        return None
    W, ops, x0 = workload_setup(args.workload)
    n = W.n
    slice_gates = 21
    psi = osv.basis_state(n, x0)
    pos = 0

    def step():
        nonlocal psi, pos
        for _ in range(slice_gates):
            g = pos % len(ops)
            if g == 0:
                psi = osv.basis_state(n, x0)
            op = ops[g]
            if op.kind == "FLIP":
                psi = osv.phase_flip(psi, op.index)
            else:
                U = ocirc.op_unitary(op)
                if op.noisy:
                    xa, xb = ophilox.normal_pair(W.seed, 0, g)
                    U = ogates.noisy_unitary(U, ocirc.op_noise(op), W.e, xa, xb)
                psi = osv.apply_gate(psi, n, ocirc.op_targets(op), U)
            pos += 1

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = (1 << n) * slice_gates / dt
    sample = f"{slice_gates} consecutive gates of one trajectory of {W.name} per step (oracle, complex128 NumPy)"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "circuit": W.circuit, "n": n, "gates": len(ops), "e": W.e},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="mc_qft_n20_c64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the bounded measurements of the other rows")
    ap.add_argument("--kernel-config", default=None,
                    help="low,high pass configuration indices (qs_plan_set_config) instead of autotuning")
    ap.add_argument("--window", type=int, default=10,
                    help="window width of the passes with --kernel-config (qs_plan_set_window)")
    ap.add_argument("--micro", choices=sorted(MICRO), default=None,
                    help="time one kernel on its own (for a profiler) instead of the bench step")
    args = ap.parse_args()
    if args.micro:
        print(json.dumps(run_micro(args)), flush=True)
        return
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local_rank = env_rank()
    from paper_1412_2293_gb300 import inputs
    mode = inputs.WORKLOADS[args.workload].mode
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif mode != "statevec":
        out = run_channels(args, rank, world, local_rank) if rank == 0 else None
    else:
        out = run_ours(args, rank, world, local_rank)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
