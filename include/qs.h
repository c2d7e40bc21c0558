/*
 * qs.h -- C ABI of the GB300 noisy-circuit simulator hot path.
 *
 * The operations are those of Bogdanov et al., "Numerical and analytical
 * research of the impact of decoherence on quantum circuits"
 * (arXiv:1412.2293):
 *   - the amplitude update of Sec. 2 (one qubit: b[..i_k..] =
 *     u[i_k,0] a[..0..] + u[i_k,1] a[..1..]; k qubits likewise);
 *   - Monte Carlo noisy gates, Sec. 2, Eqs. 1-2 (rotation V_noise(e xi) acting
 *     before the gate, Eq. 5; controlled-phase angle theta -> theta + e xi,
 *     Eqs. 7-8), xi ~ N(0,1) drawn on the device;
 *   - the density matrix and quantum operations, Sec. 3, Eq. 3, in the
 *     vectorised form (U (x) U*) vec(rho) of Sec. 3;
 *   - the fixed-rank approximation of Sec. 3.2 (factor L, rho = L L^dagger,
 *     Gram-matrix eigendecomposition, truncation to rank r);
 *   - fidelity and trace reductions (Figs. 1-4, Eq. 10);
 *   - rank-1 estimates by branch selection (Eqs. 11-15), Choi-Jamiolkowski
 *     relative states (Sec. 4, Eqs. 16-17) and amplitude / phase relaxation
 *     (T1, T2; Sec. 4.1-4.3, Eqs. 18-19);
 *   - dense k-qubit blocks, k <= 5 (complex64 on the tcgen05 tensor cores).
 *
 * Conventions (all entry points):
 *   - Qubit t is bit t of the amplitude index (qubit 0 least significant).
 *   - A k-qubit matrix is 2^k x 2^k, row-major, complex numbers interleaved
 *     (re, im) as doubles; its local index is sum_j bit(targets[j]) << j.
 *   - Host arrays passed in are owned by the caller and are read (copied)
 *     before the call returns; output arrays are written before it returns.
 *   - Work is issued on the CUDA stream given to qs_create, in call order.
 *     Calls that return results (qs_fidelity, qs_trace, qs_get_state, ...)
 *     synchronise that stream; the others return once the work is enqueued.
 *   - Every entry point returns a qs_status; no C++ exception crosses the
 *     ABI.  qs_last_error(h) gives a human-readable detail string.
 *   - A handle is not thread-safe: one host thread at a time per handle.
 *   - The library never falls back to the CPU: without a usable CUDA device
 *     qs_create fails with QS_ERR_CUDA.
 */
#ifndef QS_H
#define QS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qs_ctx* qs_handle;
typedef struct qs_plan_s* qs_plan;

typedef enum {
  QS_OK = 0,
  QS_ERR_INVALID_ARG = 1,    /* bad size, target, pointer or Kraus set     */
  QS_ERR_OUT_OF_MEMORY = 2,  /* device allocation or memory budget refused */
  QS_ERR_CUDA = 3,           /* a CUDA runtime call or kernel failed        */
  QS_ERR_NOT_SUPPORTED = 4,  /* operation undefined for the handle's mode   */
  QS_ERR_TIMEOUT = 5         /* a bounded device wait gave up               */
} qs_status;

typedef enum {
  QS_STATEVEC = 0,   /* `batch` independent state vectors (Monte Carlo, Sec. 2) */
  QS_DENSITY = 1,    /* exact vectorised density matrix (Sec. 3)               */
  QS_FIXED_RANK = 2  /* rank-r factor of the density matrix (Sec. 3.2)         */
} qs_mode;

typedef enum { QS_C64 = 0, QS_C128 = 1 } qs_dtype;

typedef enum {
  QS_NOISE_ROTATION = 0, /* Eq. 1: U V_noise(e xi) on each target (V first, Eq. 5) */
  QS_NOISE_PHASE = 1     /* Eqs. 7-8: U diag(1,..,1, e^{-i e xi})                 */
} qs_noise;

/* ------------------------------------------------------------------ handles */

/* Create a simulator on the current CUDA device.
 *   n       qubits, 1 <= n; memory: STATEVEC batch * 2^n, DENSITY 4^n,
 *           FIXED_RANK batch * (rank + min(32, 8 rank)) * 2^n complex
 *           elements (plus small scratch).
 *   batch   STATEVEC: number of trajectories (>= 1).  FIXED_RANK: number of
 *           independent factors (members, >= 1) that every call advances
 *           together -- each with its own truncation rank
 *           (qs_set_member_ranks), column count and, for noisy gates, noise
 *           level (qs_set_member_noise); one launch of each kernel serves
 *           all of them.  DENSITY: must be 1.
 *   rank    FIXED_RANK: truncation rank r >= 1 (the largest of the members');
 *           other modes: ignored (0).
 *   dtype   QS_C64 (complex float, FP32 arithmetic) or QS_C128 (FP64).
 *           Reductions (fidelity, trace, Gram matrix, eigensolver) always
 *           accumulate in FP64.
 *   cuda_stream  a cudaStream_t (may be NULL = legacy default stream).
 * The state starts as |0...0> in every batch member.  Device memory is
 * owned by the handle and released by qs_destroy.
 * Errors: INVALID_ARG (sizes), OUT_OF_MEMORY, CUDA (no device). */
qs_status qs_create(int n, int batch, int rank, qs_mode mode, qs_dtype dtype,
                    void* cuda_stream, qs_handle* out);
qs_status qs_destroy(qs_handle h);
const char* qs_last_error(qs_handle h);
qs_status qs_synchronize(qs_handle h);

/* Shape of a handle (any pointer may be NULL).  *results = number of doubles
 * qs_fidelity / qs_trace write (batch for STATEVEC and FIXED_RANK, 1 for
 * DENSITY). */
qs_status qs_info(qs_handle h, int* n, int* batch, int* rank, int* mode, int* dtype, int* results);

/* Every batch member (trajectory / density matrix / factor) <- |x><x|.
 * FIXED_RANK: every member's factor becomes one column.  Errors: INVALID_ARG
 * if x >= 2^n. */
qs_status qs_set_basis_state(qs_handle h, uint64_t x);

/* Per-member basis states: xs[b] for b < batch (STATEVEC; FIXED_RANK: each
 * member's factor becomes the one column |xs[b]>). */
qs_status qs_set_basis_states(qs_handle h, const uint64_t* xs);

/* Choi-Jamiolkowski relative states (Sec. 4): the maximally entangled state
 * of Eq. 16 on the handle's n = 2m qubits, 2^{-m/2} sum_i |i>_sys |i>_ref,
 * system = qubits 0..m-1 (amplitude index i + (i << m)).  STATEVEC: every
 * member; DENSITY: |Omega><Omega|; FIXED_RANK: one column.  A circuit on
 * qubits 0..m-1 then yields the relative state of Eq. 17; its fidelity with
 * the ideal relative state (a STATEVEC handle given the same start and the
 * noiseless circuit) measures the circuit as a whole.  n odd ->
 * QS_ERR_INVALID_ARG. */
qs_status qs_set_maximally_entangled(qs_handle h);

/* ------------------------------------------------------------------- gates */

/* Ideal k-qubit gate U (k = 1..5) on `targets` (distinct, < n) -- Sec. 2.
 * DENSITY: rho <- U rho U^dagger via (U (x) U*) on bits (t, t + n), Sec. 3;
 *   one 2k-qubit sweep for k <= 2, two k-qubit sweeps (U on the row bits
 *   t + n, U* on the column bits t) for k = 3..5.
 * FIXED_RANK: L <- U L (no truncation).
 * A dense (non-diagonal) U with k >= 3 on a complex64 state of at least k + 7
 * qubits (per member; for DENSITY the 2n-qubit vector) runs on the tcgen05
 * tensor cores as one GEMM over all groups and members: operands split into
 * tf32 hi + lo parts, hi*hi + lo*hi + hi*lo accumulated in FP32 (relative
 * error about 1e-6 of sum |U_ij||psi_j|); see qs_set_tensor_cores.
 * Errors: INVALID_ARG for bad targets / k / NULL pointers. */
qs_status qs_apply_gate(qs_handle h, const int* targets, int k, const double* U);

/* I - 2|index><index| on every member (Grover oracle; the diffusion with its
 * global phase dropped is the flip of index 0).  Errors: INVALID_ARG. */
qs_status qs_apply_phase_flip(qs_handle h, uint64_t index);

/* Noisy gate, k = 1 or 2 (Sec. 2, Eqs. 1, 2, 5, 7, 8).
 * STATEVEC: member b applies U * N_b with N_b from xi drawn by Philox4x32-10
 *   (key = seed, counter = (traj_b, gate_id)); traj_b = offset + b (see
 *   qs_set_trajectory_offset) unless per-slot noise is set.  Rotation noise
 *   uses xi_a on targets[0] and xi_b on targets[1]; phase noise uses xi_a.
 * DENSITY / FIXED_RANK: the xi-averaged channel (Eqs. 6, 9): rotation ->
 *   {sqrt(l1) U, sqrt(l2) U J} per target (l1,2 = (1 +- exp(-2e^2))/2),
 *   phase -> {U diag(1,..,sqrt P), U diag(0,..,sqrt(1-P))}, P = exp(-e^2);
 *   FIXED_RANK truncates every member to its rank afterwards (Sec. 3.2);
 *   with per-member noise set, member b's channel uses its own e[b].
 * Errors: INVALID_ARG (k, targets, e < 0). */
qs_status qs_apply_noisy_gate(qs_handle h, const int* targets, int k, const double* U,
                              qs_noise noise, double e, uint64_t seed, uint64_t gate_id);

/* Rank-1 estimate by branch selection (Sec. 3.2, the estimates behind Eqs. 11
 * and 15, Fig. 4): the noisy gate replaced by the first operator of its
 * xi-averaged Kraus set -- sqrt(lambda_1) U (rotation noise, Eq. 6),
 * U diag(1,..,1,sqrt P) (phase noise, Eq. 9), or with rotated = 1 for phase
 * noise the rotated B_1 = (E_1 + f E_2) / sqrt(1 + f^2) of Eqs. 12-14.  The
 * state is not renormalised: after a circuit, |<ideal|psi>|^2 is the rank-1
 * estimate of the fidelity.  Applied to every member (STATEVEC), column
 * (FIXED_RANK) or as B rho B^dagger (DENSITY).  Arguments and errors as
 * qs_apply_noisy_gate. */
qs_status qs_apply_branch_gate(qs_handle h, const int* targets, int k, const double* U, qs_noise noise,
                               double e, int rotated);

/* Quantum operation sum_i E_i rho E_i^dagger (Eq. 3) with num_ops Kraus
 * operators E (num_ops consecutive 2^k x 2^k matrices), k = 1..2.
 * The set must satisfy sum_i E_i^dagger E_i = I within 1e-12 (else
 * INVALID_ARG).  DENSITY: superoperator sum_i E_i (x) E_i* on bits (t, t+n).
 * A DENSITY handle tracks whether its matrix is exactly Hermitian (after
 * qs_create, qs_set_basis_state, qs_set_maximally_entangled, and qs_set_state
 * of an exactly Hermitian matrix); while it is, one-qubit channels with a real
 * superoperator on qubits t >= 5 (every noisy Hadamard, qs_apply_noisy_gate)
 * and the diagonal blocks of plans compute only the entries on or above the
 * diagonal and write the ones below as their conjugates.
 * FIXED_RANK: L' = [E_1 L | ... | E_K L], then truncation to the handle's
 * rank when num_ops > 1.  STATEVEC: NOT_SUPPORTED. */
qs_status qs_apply_kraus(qs_handle h, const int* targets, int k, const double* E, int num_ops);

/* Amplitude (T1) and phase (T2) relaxation over time t of each of the
 * `count` distinct qubits in `qubits` (Sec. 4 names both processes; the
 * channel is the textbook one: amplitude damping with gamma = 1 - exp(-t/T1),
 * then dephasing to a total coherence factor c = exp(-t/T2)):
 *   rho_00 += gamma rho_11,  rho_11 *= exp(-t/T1),  rho_01, rho_10 *= c.
 * T1 or T2 = +infinity turns that process off; a phase error of probability p
 * is T1 = inf with exp(-t/T2) = 1 - 2p (Eq. 19).
 * DENSITY: in place, two qubits per sweep of rho (each entry read and written
 *   once per sweep); coefficients in the handle's precision.
 * FIXED_RANK: per qubit the Kraus set diag(1, c), sqrt(gamma)|0><1|,
 *   diag(0, sqrt(exp(-t/T1) - c^2)) (zero operators omitted) as
 *   qs_apply_kraus, i.e. expansion and truncation to the handle's rank.
 * STATEVEC: NOT_SUPPORTED.
 * Errors: INVALID_ARG for count < 0, a qubit out of range or repeated,
 * t < 0 or not finite, T1 <= 0, T2 <= 0, or T2 > 2 T1 (not a channel). */
qs_status qs_apply_relaxation(qs_handle h, const int* qubits, int count, double t, double T1, double T2);

/* on = 0 sends complex64 dense blocks with k >= 3 to the CUDA-core sweep
 * (FP32 complex multiply-adds) instead of the tensor cores; on = 1 (the
 * default) restores the tensor-core path.  Errors: INVALID_ARG for NULL. */
qs_status qs_set_tensor_cores(qs_handle h, int on);

/* FIXED_RANK: truncate every member's factor to rank r (<= handle rank) by
 * the Gram-matrix eigendecomposition (Sec. 3.2).  normalize = 0 keeps the trace
 * sum of the kept eigenvalues; 1 rescales to unit trace.  Eigenvalues within
 * 1e-10 * Lambda_1 form one cluster whose basis is made canonical by
 * Gram-Schmidt of the projected Gram-space axes.  Other modes: NOT_SUPPORTED. */
qs_status qs_truncate_rank(qs_handle h, int r, int normalize);

/* FIXED_RANK: normalisation used by the automatic truncations (default 0). */
qs_status qs_set_normalize(qs_handle h, int normalize);

/* FIXED_RANK: current number of factor columns (<= rank; the largest over
 * the members). */
qs_status qs_get_rank(qs_handle h, int* out);

/* FIXED_RANK: truncation rank of each member, ranks[b] in 1..rank for b <
 * batch (default: the handle's rank), so members of uneven rank share one
 * handle and one launch per kernel.  Errors: INVALID_ARG for a rank out of
 * range, NOT_SUPPORTED for other modes. */
qs_status qs_set_member_ranks(qs_handle h, const int* ranks);

/* FIXED_RANK: live columns of each member's factor, out[batch]. */
qs_status qs_get_member_columns(qs_handle h, int* out);

/* ------------------------------------------------------------ reductions */

/* Fidelity with a pure reference phi, per member, FP64 accumulation:
 *   STATEVEC |<phi|psi_b>|^2 (out[batch]); DENSITY <phi|rho|phi> (out[1]);
 *   FIXED_RANK sum_c |<phi|L_c>|^2 (out[1]).
 * phi = `ref` (2^n interleaved complex doubles, host) if ref != NULL, else
 * the basis state |ref_basis>.  FIXED_RANK writes one value per member
 * (out[batch]).  Synchronises.  Errors: INVALID_ARG. */
qs_status qs_fidelity(qs_handle h, const double* ref, uint64_t ref_basis, double* out);

/* Store a reference phi on the device once (2^n complex doubles, host), for
 * qs_fidelity_stored.  Or copy member `b` of a STATEVEC handle `src` with the
 * same n (device to device). */
qs_status qs_set_reference(qs_handle h, const double* ref);
qs_status qs_set_reference_from(qs_handle h, qs_handle src, int b);
qs_status qs_fidelity_stored(qs_handle h, double* out);

/* STATEVEC: |<ref_0|psi_b>|^2 for members b = first .. first+count-1, with
 * ref_0 = member 0 of the STATEVEC handle `ref` (same n and dtype; read in
 * place on the device, after `ref`'s stream is synchronised); FIXED_RANK:
 * sum_c |<ref_0|L_{b,c}>|^2 over member b's columns.  out[count].
 * Lets members of one batch (different jobs) use different references. */
qs_status qs_fidelity_ref(qs_handle h, qs_handle ref, int first, int count, double* out);

/* Trace: STATEVEC squared norm per member (out[batch]); DENSITY tr(rho);
 * FIXED_RANK sum_c ||L_c||^2 per member (out[batch]).  Synchronises. */
qs_status qs_trace(qs_handle h, double* out);

/* ------------------------------------------------------- state transfer */

/* Number of complex elements of the state: STATEVEC batch * 2^n,
 * DENSITY 4^n (vec index i * 2^n + j for rho[i][j]), FIXED_RANK
 * batch * rank * 2^n (column-major: column c of member b at offset
 * (b rank + c) 2^n; a member's columns past its live count are 0). */
qs_status qs_state_size(qs_handle h, size_t* out);
/* Copy the state to / from host memory as interleaved complex doubles
 * (count = qs_state_size).  Synchronises.  qs_set_state on a DENSITY handle
 * checks whether the matrix is exactly Hermitian (rho[j][i] == conj rho[i][j]
 * bit for bit); only then do the Hermitian sweeps (see qs_apply_kraus) run. */
qs_status qs_get_state(qs_handle h, double* host, size_t count);
qs_status qs_set_state(qs_handle h, const double* host, size_t count);
/* Copy elements [first, first + count) of the state to host memory as
 * interleaved complex doubles (for STATEVEC, member b is the range
 * [b 2^n, (b + 1) 2^n)), without copying the rest.  Synchronises.
 * Errors: INVALID_ARG if the range exceeds qs_state_size or host is NULL. */
qs_status qs_get_state_range(qs_handle h, size_t first, size_t count, double* host);

/* FIXED_RANK: set every member's number of live columns after qs_set_state. */
qs_status qs_set_rank_columns(qs_handle h, int m);

/* Failure detection: every tile-copy wait of the fused passes polls its
 * mbarrier at most `polls` times (default 2^22, restored by polls < 0;
 * 0 gives up at once).  A pass whose wait gives up lets the copies it has in
 * flight land (bounded by the default), records the failure in a device
 * status word and returns; the next call that reads results (qs_fidelity,
 * qs_plan_run_fidelity, ...) returns QS_ERR_TIMEOUT once, clears the word, and
 * the handle stays usable.  Errors: INVALID_ARG for polls >= 2^32. */
qs_status qs_set_wait_limit(qs_handle h, int64_t polls);

/* --------------------------------------------------- Monte Carlo counters */

/* STATEVEC: member b uses trajectory counter offset + b (default 0), so a
 * run split across processes draws the same noise as one run. */
qs_status qs_set_trajectory_offset(qs_handle h, uint64_t offset);

/* STATEVEC: per-member noise (continuous batching of different jobs in one
 * handle).  e[b], seed[b], traj[b] override the call arguments and the
 * offset for member b; marked[b] (may be NULL) replaces the index of plan
 * flips marked QS_FLIP_PER_MEMBER.  FIXED_RANK: e[b] sets member b's
 * averaged channel in qs_apply_noisy_gate (seed and traj are required but
 * unused) and marked[b] the index of member b's QS_FLIP_PER_MEMBER flips.
 * Pass all NULL to clear. */
qs_status qs_set_member_noise(qs_handle h, const double* e, const uint64_t* seed,
                              const uint64_t* traj, const uint64_t* marked);

/* ----------------------------------------------------------------- plans */

/* A circuit applied as a whole: the planner groups the gates into fused
 * passes (runs of gates on a window of qubits applied in one read and one
 * write of the state; diagonal gates folded in), and the run is replayed
 * from a captured CUDA graph.  Noisy gates draw with gate_id = gate_id0 +
 * position in the list, so a plan run equals the same gates issued one by
 * one through qs_apply_noisy_gate / qs_apply_gate / qs_apply_phase_flip. */
typedef enum {
  QS_GATE_DENSE = 0,       /* matrix U on targets[0..k-1]                  */
  QS_GATE_FLIP = 1,        /* I - 2|index><index|                          */
  QS_FLIP_PER_MEMBER = 2   /* flip of marked[b] (qs_set_member_noise)      */
} qs_gate_kind;

typedef struct {
  int kind;            /* qs_gate_kind                                   */
  int k;               /* 1 or 2 for QS_GATE_DENSE                       */
  int targets[2];
  int noisy;           /* 0 = ideal; 1 = noisy with `noise`              */
  int noise;           /* qs_noise                                       */
  uint64_t index;      /* QS_GATE_FLIP                                   */
  double U[32];        /* 2^k x 2^k interleaved complex                  */
} qs_gate;

/* Build a plan for `h` (the plan keeps a reference to h; destroy it first).
 * STATEVEC handles with n >= 10 get fused passes over windows of ten qubits:
 * qubits 0..9, and c..c+9 (c >= 3 complex64, c >= 2 complex128) chosen per run
 * of gates, the top ten first; gates no window can hold, and other shapes,
 * run gate by gate with the same kernels as the single-gate calls.
 * FIXED_RANK handles: every gate on every member (noisy gates as their
 * averaged channels with expansion and truncation, Sec. 3.2), the launch
 * shapes fixed when the plan is made and the column counts kept on the
 * device, so the whole circuit replays as one CUDA graph; needs K * rank <=
 * 32 for every noisy gate (NOT_SUPPORTED otherwise).
 * Errors: INVALID_ARG for a malformed gate (nothing is built). */
qs_status qs_plan_create(qs_handle h, const qs_gate* gates, int num_gates, qs_plan* out);
/* Run the plan once on the handle's stream with noise level e and key seed
 * (per-member values from qs_set_member_noise take precedence). */
qs_status qs_plan_run(qs_plan p, double e, uint64_t seed, uint64_t gate_id0);
/* Run the plan and return the fidelity of every member with the stored
 * reference (qs_set_reference / qs_set_reference_from) in out[batch]: when
 * the plan ends with a fused pass, that pass also reduces <phi|psi_b> (FP64
 * across blocks) instead of a separate read of the state.  A start state set
 * by qs_set_basis_state(s) is created by the first fused pass instead of being
 * written to memory first.  STATEVEC only.  Synchronises. */
qs_status qs_plan_run_fidelity(qs_plan p, double e, uint64_t seed, uint64_t gate_id0, double* out);

/* Number of passes over the state one run makes, and kernels it launches. */
qs_status qs_plan_info(qs_plan p, int* passes, int* launches);
qs_status qs_plan_destroy(qs_plan p);

/* Time each kernel of one plan run with CUDA events on the handle's stream
 * (eager launches, `reps` runs averaged; the state is modified as by
 * qs_plan_run; a basis start set by qs_set_basis_state(s) and not yet used is
 * created by the first pass of every profiled run, as plan runs do, and is
 * used up afterwards).  ms[i] = mean duration of launch i of a run, kinds[i] =
 * 0 noise/parameter precompute, 1 low-window pass, 2 high-window pass,
 * 3 single-gate step (all kernels of the step together), 4 density-matrix
 * run of diagonal channels (one sweep); at most `cap`
 * entries, *count = launches per run.  Synchronises. */
qs_status qs_plan_profile(qs_plan p, int reps, double e, uint64_t seed, uint64_t gate_id0,
                          double* ms, int* kinds, int cap, int* count);

/* Per-launch timing of plan runs: with on = 1 every later qs_plan_run also
 * records CUDA events around each kernel launch it makes (inside the graph);
 * qs_plan_last_times then gives the durations of the most recent run (it
 * waits for that run), kinds as for qs_plan_profile. */
qs_status qs_plan_set_timing(qs_plan p, int on);
qs_status qs_plan_last_times(qs_plan p, double* ms, int* kinds, int cap, int* count);

/* Window width m of the fused passes (no counterpart in the paper, which
 * updates the state one gate at a time, Sec. 2: a pass applies the run of
 * gates acting on m qubits to each tile of 2^m amplitudes with one read and
 * one write of the state).  m = 10 for a new plan; 11 and 12 need a STATEVEC
 * complex64 handle with n <= 32 (NOT_SUPPORTED otherwise; INVALID_ARG for
 * another m).  A wider window takes more gates per pass, so fewer passes over
 * the state (the QFT at n = 24: two passes for m = 12, three for m = 10).
 * Setting m re-plans the passes (waits for the handle's stream, drops the
 * captured graphs and resets the kernel configuration to the new width's
 * default); results agree with every m up to rounding.  On failure (device
 * memory) the plan runs nothing until a later call succeeds. */
qs_status qs_plan_set_window(qs_plan p, int m);
qs_status qs_plan_get_window(qs_plan p, int* m);

/* Kernel configuration of the fused passes (no counterpart in the paper: the
 * tiling of the update, Sec. 2, is the implementation's).  For m = 10 and
 * each window geometry (low: qubits 0..9, high: the 10 highest) a
 * configuration index in [0, count): complex64 has three low and three high
 * -- low 0: 12 warps, two
 * tile buffers per warp; low 1: 16 warps, one buffer; low 2: 12 warps, one
 * buffer; high 0: one block of
 * 8 warps per SM, two buffers; high 1: two such blocks per SM, one buffer;
 * high 2: four blocks of 4 warps per SM (4-column tiles), one buffer --
 * complex128 one of each.  m = 11 and 12 have one of each: low 12 warps in
 * groups of 2^(m-10) warps per tile, one buffer per group; high one block
 * of 16 warps per SM, one buffer, tiles of 8 (m = 11) or 4 (m = 12) columns.
 * A new plan starts with low 2 / high 1 (complex64), 0 / 0 (complex128).
 * Results do not depend on the configuration.  qs_plan_configs returns the
 * counts; qs_plan_set_config rejects an index out of range with
 * QS_ERR_INVALID_ARG; qs_plan_get_config returns the current choice. */
qs_status qs_plan_configs(qs_plan p, int* low_count, int* high_count);
qs_status qs_plan_set_config(qs_plan p, int low_cfg, int high_cfg);
qs_status qs_plan_get_config(qs_plan p, int* low_cfg, int* high_cfg);
/* Autotune: for every window width the handle allows (10, 11 and 12 for a
 * STATEVEC complex64 handle with m <= n <= 32, else the current one), time
 * every configuration on this plan (qs_plan_profile with `reps` runs each,
 * noise e and key seed); keep the width whose run is fastest with its
 * fastest configuration per geometry, and write those configurations' mean
 * pass times in ms to best_ms[0] (low) and best_ms[1] (high) (-1 where the
 * plan has no pass of that geometry; best_ms may be NULL).
 * qs_plan_get_window then reports the width chosen.  The runs overwrite the
 * state; a basis start set before the call (qs_set_basis_state(s)) is
 * created by the first pass of every profiled run, so the passes are timed
 * as the plan's runs from that start will execute them, and it is still the
 * pending start afterwards.  Synchronises. */
qs_status qs_plan_autotune(qs_plan p, int reps, double e, uint64_t seed, double* best_ms);

/* ------------------------------------------------------------ utilities */

/* The Philox4x32-10 words and normals the device draws for (seed, traj,
 * gate_id), count consecutive trajectories starting at traj (for checking
 * the device stream against an independent implementation).
 * words: 4 * count uint32; normals: 2 * count doubles (xi_a, xi_b). */
qs_status qs_debug_noise(uint64_t seed, uint64_t traj, uint64_t gate_id, int count,
                         uint32_t* words, double* normals);

/* Allocation-free fidelity.  The paper has no counterpart: this is a
 * deployment variant of qs_fidelity for callers that cannot allocate device
 * memory -- a host application or framework that owns the GPU's memory
 * through its own pool and forbids other allocators, or a latency-critical
 * loop that cannot afford cudaMalloc's device-wide synchronisation.
 *   states  device pointer, `members` consecutive state vectors of 2^n
 *           complex elements of `dtype` (the STATEVEC layout), caller-owned.
 *   ref     device pointer, 2^n complex elements of `dtype`, caller-owned.
 *   out     host pointer, `members` doubles: |<ref|states_b>|^2; every FP32
 *           (complex64) partial sums at most 16 products before it joins an
 *           FP64 sum, and blocks are added in FP64, as in qs_fidelity.
 *   cuda_stream  the stream the work is issued on (NULL = legacy stream);
 *           the call synchronises it before returning.
 * The call allocates nothing: its scratch is a fixed array of
 * 2 * QS_NOALLOC_MAX_PARTIALS + QS_NOALLOC_MAX_MEMBERS doubles (1.5 MiB) that
 * every GPU loading this library holds until the process exits.  The first
 * call on a device looks up that array's device address (cudaGetSymbolAddress
 * with the device current) and keeps it; make that first call before any
 * stream capture.  The kept address belongs to the device's primary context:
 * do not call this entry point after a cudaDeviceReset or from a context of
 * the caller's own.
 * All calls on a device share the array: calls whose work overlaps on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller.  Errors: INVALID_ARG for NULL pointers, n outside 1..40, members < 1
 * or members > QS_NOALLOC_MAX_MEMBERS (the scratch limit); CUDA on a failed
 * launch or copy. */
#define QS_NOALLOC_MAX_MEMBERS 65535
#define QS_NOALLOC_MAX_PARTIALS 65536
qs_status qs_fidelity_noalloc(const void* states, const void* ref, int n, int members, qs_dtype dtype,
                              void* cuda_stream, double* out);

/* Measured FP64 and FP32 multiply-add rates of the current device (TFLOP/s),
 * from dependent FMA chains on every SM (the denominators of the rooflines of
 * arithmetic-bound kernels).  Synchronises the device. */
qs_status qs_measure_peaks(double* fp64_tflops, double* fp32_tflops);

/* Library version string. */
const char* qs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* QS_H */
