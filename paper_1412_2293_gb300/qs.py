"""Thin ctypes binding of the C ABI in include/qs.h (argument marshalling only).

Every function has the name of the C entry point it calls and raises
``QSError`` on a non-OK status.  All computation happens in the CUDA library;
if the library is not built, or no CUDA device is present, calls fail loudly --
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libqsim.so")

QS_OK, QS_ERR_INVALID_ARG, QS_ERR_OUT_OF_MEMORY, QS_ERR_CUDA, QS_ERR_NOT_SUPPORTED, QS_ERR_TIMEOUT = range(6)
QS_STATEVEC, QS_DENSITY, QS_FIXED_RANK = range(3)
QS_C64, QS_C128 = range(2)
QS_NOISE_ROTATION, QS_NOISE_PHASE = range(2)
QS_GATE_DENSE, QS_GATE_FLIP, QS_FLIP_PER_MEMBER = range(3)

STATUS_NAMES = {0: "QS_OK", 1: "QS_ERR_INVALID_ARG", 2: "QS_ERR_OUT_OF_MEMORY", 3: "QS_ERR_CUDA",
                4: "QS_ERR_NOT_SUPPORTED", 5: "QS_ERR_TIMEOUT"}


class QSError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class qs_gate(ct.Structure):
    _fields_ = [("kind", ct.c_int), ("k", ct.c_int), ("targets", ct.c_int * 2), ("noisy", ct.c_int),
                ("noise", ct.c_int), ("index", ct.c_uint64), ("U", ct.c_double * 32)]


_lib = None
_P = ct.c_void_p
_D = ct.POINTER(ct.c_double)
_U64 = ct.POINTER(ct.c_uint64)
_I = ct.POINTER(ct.c_int)

_SIGS = {
    "qs_version": ([], ct.c_char_p),
    "qs_create": ([ct.c_int, ct.c_int, ct.c_int, ct.c_int, ct.c_int, _P, ct.POINTER(_P)], ct.c_int),
    "qs_destroy": ([_P], ct.c_int),
    "qs_last_error": ([_P], ct.c_char_p),
    "qs_synchronize": ([_P], ct.c_int),
    "qs_info": ([_P, _I, _I, _I, _I, _I, _I], ct.c_int),
    "qs_set_basis_state": ([_P, ct.c_uint64], ct.c_int),
    "qs_set_basis_states": ([_P, _U64], ct.c_int),
    "qs_set_maximally_entangled": ([_P], ct.c_int),
    "qs_apply_gate": ([_P, _I, ct.c_int, _D], ct.c_int),
    "qs_apply_phase_flip": ([_P, ct.c_uint64], ct.c_int),
    "qs_apply_noisy_gate": ([_P, _I, ct.c_int, _D, ct.c_int, ct.c_double, ct.c_uint64, ct.c_uint64], ct.c_int),
    "qs_apply_branch_gate": ([_P, _I, ct.c_int, _D, ct.c_int, ct.c_double, ct.c_int], ct.c_int),
    "qs_apply_kraus": ([_P, _I, ct.c_int, _D, ct.c_int], ct.c_int),
    "qs_apply_relaxation": ([_P, _I, ct.c_int, ct.c_double, ct.c_double, ct.c_double], ct.c_int),
    "qs_truncate_rank": ([_P, ct.c_int, ct.c_int], ct.c_int),
    "qs_set_normalize": ([_P, ct.c_int], ct.c_int),
    "qs_set_tensor_cores": ([_P, ct.c_int], ct.c_int),
    "qs_get_rank": ([_P, _I], ct.c_int),
    "qs_fidelity": ([_P, _D, ct.c_uint64, _D], ct.c_int),
    "qs_set_reference": ([_P, _D], ct.c_int),
    "qs_set_reference_from": ([_P, _P, ct.c_int], ct.c_int),
    "qs_fidelity_stored": ([_P, _D], ct.c_int),
    "qs_trace": ([_P, _D], ct.c_int),
    "qs_fidelity_ref": ([_P, _P, ct.c_int, ct.c_int, _D], ct.c_int),
    "qs_state_size": ([_P, ct.POINTER(ct.c_size_t)], ct.c_int),
    "qs_get_state": ([_P, _D, ct.c_size_t], ct.c_int),
    "qs_set_state": ([_P, _D, ct.c_size_t], ct.c_int),
    "qs_get_state_range": ([_P, ct.c_size_t, ct.c_size_t, _D], ct.c_int),
    "qs_set_rank_columns": ([_P, ct.c_int], ct.c_int),
    "qs_set_trajectory_offset": ([_P, ct.c_uint64], ct.c_int),
    "qs_set_wait_limit": ([_P, ct.c_int64], ct.c_int),
    "qs_set_member_ranks": ([_P, _I], ct.c_int),
    "qs_get_member_columns": ([_P, _I], ct.c_int),
    "qs_set_member_noise": ([_P, _D, _U64, _U64, _U64], ct.c_int),
    "qs_plan_create": ([_P, ct.POINTER(qs_gate), ct.c_int, ct.POINTER(_P)], ct.c_int),
    "qs_plan_run": ([_P, ct.c_double, ct.c_uint64, ct.c_uint64], ct.c_int),
    "qs_plan_run_fidelity": ([_P, ct.c_double, ct.c_uint64, ct.c_uint64, _D], ct.c_int),
    "qs_plan_info": ([_P, _I, _I], ct.c_int),
    "qs_plan_profile": ([_P, ct.c_int, ct.c_double, ct.c_uint64, ct.c_uint64, _D, _I, ct.c_int, _I], ct.c_int),
    "qs_plan_destroy": ([_P], ct.c_int),
    "qs_plan_set_timing": ([_P, ct.c_int], ct.c_int),
    "qs_plan_last_times": ([_P, _D, _I, ct.c_int, _I], ct.c_int),
    "qs_plan_configs": ([_P, _I, _I], ct.c_int),
    "qs_plan_set_config": ([_P, ct.c_int, ct.c_int], ct.c_int),
    "qs_plan_get_config": ([_P, _I, _I], ct.c_int),
    "qs_plan_autotune": ([_P, ct.c_int, ct.c_double, ct.c_uint64, _D], ct.c_int),
    "qs_plan_set_window": ([_P, ct.c_int], ct.c_int),
    "qs_plan_get_window": ([_P, _I], ct.c_int),
    "qs_fidelity_noalloc": ([_P, _P, ct.c_int, ct.c_int, ct.c_int, _P, _D], ct.c_int),
    "qs_measure_peaks": ([_D, _D], ct.c_int),
    "qs_debug_noise": ([ct.c_uint64, ct.c_uint64, ct.c_uint64, ct.c_int, ct.POINTER(ct.c_uint32), _D], ct.c_int),
}


def lib():
    """Load the CUDA library (built in-tree by ``paper_1412_2293_gb300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built ({LIB_PATH}); run paper_1412_2293_gb300.build.build()")
        L = ct.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _check(status, h=None):
    if status != QS_OK:
        msg = lib().qs_last_error(h).decode() if h else ""
        raise QSError(status, msg)


def _dptr(a):
    return a.ctypes.data_as(_D)


def _cplx_interleaved(M):
    M = np.ascontiguousarray(np.asarray(M, dtype=np.complex128))
    return np.ascontiguousarray(M.view(np.float64).reshape(-1))


def _targets(t):
    arr = (ct.c_int * len(t))(*[int(x) for x in t])
    return arr


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ct.c_void_p(stream.cuda_stream)
    return ct.c_void_p(int(stream))


def qs_version():
    return lib().qs_version().decode()


def qs_create(n, batch=1, rank=0, mode=QS_STATEVEC, dtype=QS_C64, stream=None):
    h = _P()
    _check(lib().qs_create(int(n), int(batch), int(rank), int(mode), int(dtype), _stream_ptr(stream), ct.byref(h)))
    return h


def qs_destroy(h):
    _check(lib().qs_destroy(h))


def qs_last_error(h):
    return lib().qs_last_error(h).decode()


def qs_synchronize(h):
    _check(lib().qs_synchronize(h), h)


def qs_set_basis_state(h, x):
    _check(lib().qs_set_basis_state(h, int(x)), h)


def qs_set_basis_states(h, xs):
    a = np.ascontiguousarray(np.asarray(xs, dtype=np.uint64))
    _check(lib().qs_set_basis_states(h, a.ctypes.data_as(_U64)), h)


def qs_set_maximally_entangled(h):
    _check(lib().qs_set_maximally_entangled(h), h)


def qs_apply_gate(h, targets, U):
    u = _cplx_interleaved(U)
    _check(lib().qs_apply_gate(h, _targets(targets), len(targets), _dptr(u)), h)


def qs_apply_phase_flip(h, index):
    _check(lib().qs_apply_phase_flip(h, int(index)), h)


def qs_apply_noisy_gate(h, targets, U, noise, e, seed, gate_id):
    u = _cplx_interleaved(U)
    _check(lib().qs_apply_noisy_gate(h, _targets(targets), len(targets), _dptr(u), int(noise), float(e),
                                     int(seed), int(gate_id)), h)


def qs_apply_branch_gate(h, targets, U, noise, e, rotated=False):
    u = _cplx_interleaved(U)
    _check(lib().qs_apply_branch_gate(h, _targets(targets), len(targets), _dptr(u), int(noise), float(e),
                                      1 if rotated else 0), h)


def qs_apply_kraus(h, targets, kraus):
    e = np.concatenate([_cplx_interleaved(E) for E in kraus])
    _check(lib().qs_apply_kraus(h, _targets(targets), len(targets), _dptr(e), len(kraus)), h)


def qs_apply_relaxation(h, qubits, t, T1, T2):
    """T1/T2 relaxation over t of every qubit in `qubits` (T1, T2 may be math.inf)."""
    _check(lib().qs_apply_relaxation(h, _targets(qubits), len(qubits), float(t), float(T1), float(T2)), h)


def qs_truncate_rank(h, r, normalize=0):
    _check(lib().qs_truncate_rank(h, int(r), int(normalize)), h)


def qs_set_tensor_cores(h, on=True):
    _check(lib().qs_set_tensor_cores(h, 1 if on else 0), h)


def qs_set_normalize(h, normalize):
    _check(lib().qs_set_normalize(h, int(normalize)), h)


def qs_get_rank(h):
    r = ct.c_int()
    _check(lib().qs_get_rank(h, ct.byref(r)), h)
    return r.value


def qs_info(h):
    """dict(n, batch, rank, mode, dtype, results) of a handle."""
    v = [ct.c_int() for _ in range(6)]
    _check(lib().qs_info(h, *[ct.byref(x) for x in v]), h)
    return dict(zip(("n", "batch", "rank", "mode", "dtype", "results"), (x.value for x in v)))


def _results(h):
    return qs_info(h)["results"]


def qs_fidelity(h, ref=None, ref_basis=0):
    out = np.zeros(_results(h), dtype=np.float64)
    if ref is None:
        _check(lib().qs_fidelity(h, None, int(ref_basis), _dptr(out)), h)
    else:
        r = _cplx_interleaved(ref)
        _check(lib().qs_fidelity(h, _dptr(r), 0, _dptr(out)), h)
    return out


def qs_set_reference(h, ref):
    r = _cplx_interleaved(ref)
    _check(lib().qs_set_reference(h, _dptr(r)), h)


def qs_set_reference_from(h, src, b=0):
    _check(lib().qs_set_reference_from(h, src, int(b)), h)


def qs_fidelity_stored(h):
    out = np.zeros(_results(h), dtype=np.float64)
    _check(lib().qs_fidelity_stored(h, _dptr(out)), h)
    return out


def qs_fidelity_ref(h, ref, first, count):
    out = np.zeros(int(count), dtype=np.float64)
    _check(lib().qs_fidelity_ref(h, ref, int(first), int(count), _dptr(out)), h)
    return out


def qs_trace(h):
    out = np.zeros(_results(h), dtype=np.float64)
    _check(lib().qs_trace(h, _dptr(out)), h)
    return out


def qs_state_size(h):
    n = ct.c_size_t()
    _check(lib().qs_state_size(h, ct.byref(n)), h)
    return n.value


def qs_get_state(h):
    n = qs_state_size(h)
    out = np.zeros(2 * n, dtype=np.float64)
    _check(lib().qs_get_state(h, _dptr(out), n), h)
    return out.view(np.complex128)


def qs_get_state_range(h, first, count):
    """Elements [first, first + count) of the state as complex128."""
    out = np.zeros(2 * int(count), dtype=np.float64)
    _check(lib().qs_get_state_range(h, int(first), int(count), _dptr(out)), h)
    return out.view(np.complex128)


def qs_set_state(h, state):
    s = _cplx_interleaved(state)
    _check(lib().qs_set_state(h, _dptr(s), len(s) // 2), h)


def qs_set_rank_columns(h, m):
    _check(lib().qs_set_rank_columns(h, int(m)), h)


def qs_set_member_ranks(h, ranks):
    r = np.ascontiguousarray(np.asarray(ranks, dtype=np.int32))
    _check(lib().qs_set_member_ranks(h, r.ctypes.data_as(_I)), h)


def qs_get_member_columns(h):
    out = np.zeros(qs_info(h)["batch"], dtype=np.int32)
    _check(lib().qs_get_member_columns(h, out.ctypes.data_as(_I)), h)
    return out


def qs_set_wait_limit(h, polls):
    _check(lib().qs_set_wait_limit(h, int(polls)), h)


def qs_set_trajectory_offset(h, offset):
    _check(lib().qs_set_trajectory_offset(h, int(offset)), h)


def qs_set_member_noise(h, e=None, seed=None, traj=None, marked=None):
    def u64(x):
        return None if x is None else np.ascontiguousarray(np.asarray(x, dtype=np.uint64))
    ea = None if e is None else np.ascontiguousarray(np.asarray(e, dtype=np.float64))
    sa, ta, ma = u64(seed), u64(traj), u64(marked)
    _check(lib().qs_set_member_noise(
        h, None if ea is None else _dptr(ea), None if sa is None else sa.ctypes.data_as(_U64),
        None if ta is None else ta.ctypes.data_as(_U64), None if ma is None else ma.ctypes.data_as(_U64)), h)


def make_gate(targets=(), U=None, noisy=False, noise=QS_NOISE_ROTATION, kind=QS_GATE_DENSE, index=0):
    g = qs_gate()
    g.kind = int(kind)
    g.index = int(index)
    g.noisy = int(bool(noisy))
    g.noise = int(noise)
    if kind == QS_GATE_DENSE:
        g.k = len(targets)
        for j, t in enumerate(targets):
            g.targets[j] = int(t)
        u = _cplx_interleaved(U)
        for i, v in enumerate(u):
            g.U[i] = float(v)
    return g


def qs_plan_create(h, gates):
    arr = (qs_gate * len(gates))(*gates)
    p = _P()
    _check(lib().qs_plan_create(h, arr, len(gates), ct.byref(p)), h)
    return p


def qs_plan_run(p, e, seed, gate_id0=0, h=None):
    _check(lib().qs_plan_run(p, float(e), int(seed), int(gate_id0)), h)


def qs_plan_run_fidelity(p, e, seed, gate_id0, h):
    """Run the plan and return the members' fidelities with the stored reference."""
    out = np.zeros(_results(h), dtype=np.float64)
    _check(lib().qs_plan_run_fidelity(p, float(e), int(seed), int(gate_id0), _dptr(out)), h)
    return out


def qs_plan_info(p, h=None):
    a, b = ct.c_int(), ct.c_int()
    _check(lib().qs_plan_info(p, ct.byref(a), ct.byref(b)), h)
    return a.value, b.value


PROFILE_KINDS = {0: "precompute", 1: "pass_low", 2: "pass_high", 3: "single_gate", 4: "dm_diag_block"}


def qs_plan_profile(p, reps, e, seed, gate_id0=0, cap=4096, h=None):
    """Mean CUDA-event duration (ms) of each launch of one plan run, with its kind."""
    ms = np.zeros(cap, dtype=np.float64)
    kinds = np.zeros(cap, dtype=np.int32)
    count = ct.c_int()
    _check(lib().qs_plan_profile(p, int(reps), float(e), int(seed), int(gate_id0), _dptr(ms),
                                 kinds.ctypes.data_as(_I), cap, ct.byref(count)), h)
    c = min(count.value, cap)
    return ms[:c].copy(), [PROFILE_KINDS[int(k)] for k in kinds[:c]]


def qs_plan_configs(p, h=None):
    a, b = ct.c_int(), ct.c_int()
    _check(lib().qs_plan_configs(p, ct.byref(a), ct.byref(b)), h)
    return a.value, b.value


def qs_plan_set_config(p, low_cfg, high_cfg, h=None):
    _check(lib().qs_plan_set_config(p, int(low_cfg), int(high_cfg)), h)


def qs_plan_get_config(p, h=None):
    a, b = ct.c_int(), ct.c_int()
    _check(lib().qs_plan_get_config(p, ct.byref(a), ct.byref(b)), h)
    return a.value, b.value


def qs_plan_set_window(p, m, h=None):
    _check(lib().qs_plan_set_window(p, int(m)), h)


def qs_plan_get_window(p, h=None):
    m = ct.c_int()
    _check(lib().qs_plan_get_window(p, ct.byref(m)), h)
    return m.value


def qs_plan_autotune(p, reps=3, e=0.0, seed=0, h=None):
    """Time every window width and kernel configuration, keep the fastest;
    returns (low ms, high ms) of the configurations kept."""
    best = np.zeros(2, dtype=np.float64)
    _check(lib().qs_plan_autotune(p, int(reps), float(e), int(seed), _dptr(best)), h)
    return float(best[0]), float(best[1])


def qs_plan_set_timing(p, on=True, h=None):
    _check(lib().qs_plan_set_timing(p, int(bool(on))), h)


def qs_plan_last_times(p, cap=4096, h=None):
    """Durations (ms) and kinds of each launch of the most recent timed plan run."""
    ms = np.zeros(cap, dtype=np.float64)
    kinds = np.zeros(cap, dtype=np.int32)
    count = ct.c_int()
    _check(lib().qs_plan_last_times(p, _dptr(ms), kinds.ctypes.data_as(_I), cap, ct.byref(count)), h)
    c = min(count.value, cap)
    return ms[:c].copy(), [PROFILE_KINDS[int(k)] for k in kinds[:c]]


def qs_plan_destroy(p):
    _check(lib().qs_plan_destroy(p))


QS_NOALLOC_MAX_MEMBERS = 65535


def qs_fidelity_noalloc(states_ptr, ref_ptr, n, members, dtype, stream=None):
    """|<ref|states_b>|^2 for caller-held device buffers, with no device allocation.

    For callers that cannot allocate device memory (their host application
    owns the GPU's memory, or cudaMalloc's synchronisation is unaffordable):
    `states_ptr` / `ref_ptr` are device addresses (e.g. a tensor's
    ``data_ptr()``) in the STATEVEC layout of `dtype`.  Calls on one device
    share a fixed scratch array, so calls that overlap on the GPU race.
    """
    out = np.zeros(int(members), dtype=np.float64)
    _check(lib().qs_fidelity_noalloc(ct.c_void_p(int(states_ptr)), ct.c_void_p(int(ref_ptr)), int(n),
                                     int(members), int(dtype), _stream_ptr(stream), _dptr(out)))
    return out


def qs_measure_peaks():
    """(fp64_tflops, fp32_tflops) measured on the current device."""
    a, b = ct.c_double(), ct.c_double()
    _check(lib().qs_measure_peaks(ct.byref(a), ct.byref(b)))
    return a.value, b.value


def qs_debug_noise(seed, traj, gate_id, count):
    words = np.zeros(4 * count, dtype=np.uint32)
    normals = np.zeros(2 * count, dtype=np.float64)
    _check(lib().qs_debug_noise(int(seed), int(traj), int(gate_id), int(count),
                                words.ctypes.data_as(ct.POINTER(ct.c_uint32)), _dptr(normals)))
    return words.reshape(count, 4), normals.reshape(count, 2)
