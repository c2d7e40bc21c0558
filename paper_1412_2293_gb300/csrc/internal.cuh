// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "qs.h"

namespace qs {

// ------------------------------------------------------------ complex types
template <typename R> struct CT;
template <> struct CT<float> { using C = float2; };
template <> struct CT<double> { using C = double2; };
template <typename R> using cplx = typename CT<R>::C;

template <typename R> __host__ __device__ __forceinline__ cplx<R> mk(R re, R im) {
  cplx<R> c; c.x = re; c.y = im; return c;
}
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
  C c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) {
  C c; c.x = a.x + b.x; c.y = a.y + b.y; return c;
}
// a + m * b
template <typename C> __host__ __device__ __forceinline__ C cfma(C m, C b, C a) {
  C c; c.x = a.x + m.x * b.x - m.y * b.y; c.y = a.y + m.x * b.y + m.y * b.x; return c;
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }

// ----------------------------------------------------------- small structs
constexpr int kMaxK = 5;                 // dense gates up to 5 qubits (32 x 32)
constexpr int kMaxGramDim = 32;          // K * m of a fixed-rank channel
constexpr int kMaxRank = 16;             // largest truncation rank

// Targets of a k-qubit operation: original order (local-index bits) and the
// ascending positions used to enumerate the untouched bits.
struct Targets {
  int k;
  int t[kMaxK];
  int sorted[kMaxK];
  uint64_t off[1 << kMaxK];              // index offset of each local index
};

// Where member b of a batch takes its noise: arrays override scalars.
struct NoiseSrc {
  const double* e;                       // may be null
  const uint64_t* seed;                  // may be null
  const uint64_t* traj;                  // may be null
  double e0;
  uint64_t seed0;
  uint64_t traj0;                        // member b draws traj0 + b
};

// Column counts of the members of a FIXED_RANK handle (device arrays of
// `batch` ints): live columns m_b, truncation rank r_b, columns M_b of the
// channel in progress, columns kept by its truncation.
struct RankCounts {
  int* cols;
  int* rank;
  int* M;
  int* keep;
};

// A noisy gate whose xi-averaged Kraus set (Eqs. 6, 9) the fixed-rank
// expansion builds on the device for each member from its noise level e_b:
// e_member[b] if set, else *e_run if set, else e_value.
struct KrausGate {
  double U[32];                          // 2^k x 2^k interleaved complex
  int k;                                 // 1 or 2
  int noise;                             // qs_noise
  double e_value;
  const double* e_member;
  const double* e_run;
};

// ------------------------------------------------------------- error state
struct Status {
  qs_status code = QS_OK;
  std::string msg;
};

}  // namespace qs

// The opaque handle of the C ABI.
struct qs_ctx {
  int n = 0;
  int batch = 1;
  int rank = 0;
  qs_mode mode = QS_STATEVEC;
  qs_dtype dtype = QS_C64;
  cudaStream_t stream = nullptr;
  int device = 0;
  size_t esize = 8;                      // bytes per complex element

  void* state = nullptr;                 // STATEVEC batch*2^n, DENSITY 4^n, FIXED_RANK rank*2^n
  size_t state_elems = 0;

  // FIXED_RANK: `batch` members, member b's factor in columns [b rank, (b+1)
  // rank) of the state and its L' in columns [b mcap, (b+1) mcap) of `work`;
  // column counts per member on the device (rc) and mirrored on the host
  // (m_cols, m_rank; `cols` = the largest live count)
  void* work = nullptr;
  size_t work_elems = 0;
  int mcap = 0;
  int cols = 1;
  int normalize = 0;
  qs::RankCounts rc{};
  double* rsmall = nullptr;              // per member: Gram, eigenvectors, eigenvalues, scale, Kraus sets
  std::vector<int> m_cols, m_rank;
  // FIXED_RANK: every entry of L has a zero imaginary part (real start, real
  // gates and Kraus operators so far); the channel kernels then use real
  // arithmetic (the same results, a quarter of the FP64 work)
  bool real_factor = false;

  // scratch (device)
  double* partials = nullptr;            // reduction partials
  size_t partials_cap = 0;               // doubles
  void* mats = nullptr;                  // per-member gate matrices
  size_t mats_cap = 0;                   // bytes
  double* small = nullptr;               // Gram matrix, eigenvectors, results
  size_t small_cap = 0;                  // doubles
  int* dstatus = nullptr;                // device status words
  double* hpinned = nullptr;             // pinned host staging for results
  size_t hpinned_cap = 0;

  // per-member noise (continuous batching)
  uint64_t traj_offset = 0;
  double* m_e = nullptr;
  uint64_t* m_seed = nullptr;
  uint64_t* m_traj = nullptr;
  uint64_t* m_marked = nullptr;
  bool member_noise = false;
  bool member_marked = false;
  double m_e_max = 0.0;                  // largest per-member e (host copy)
  int64_t wait_polls = -1;               // fused passes' tile-copy wait limit (-1: the default)

  // stored fidelity reference (2^n complex in the handle's dtype)
  void* ref = nullptr;
  bool has_ref = false;
  bool tensor_cores = true;              // complex64 dense blocks with k >= 3 on tcgen05
  bool hermitian = true;                 // DENSITY: the stored matrix is exactly Hermitian

  // STATEVEC start state not yet written: 1 = every member |pending_x>,
  // 2 = member b |m_basis[b]>.  Written by the first consumer (a fused first
  // pass creates it in registers instead of reading memory).
  int pending = 0;
  uint64_t pending_x = 0;
  uint64_t* m_basis = nullptr;

  std::string err;
};

namespace qs {

// ------------------------------------------------------------ launch glue
// Every function below enqueues on `s` and returns cudaGetLastError().

size_t elem_size(qs_dtype d);

cudaError_t launch_set_entangled(qs_ctx* h, void* psi, int members, int dm);
cudaError_t launch_set_basis(qs_ctx* h, void* psi, int n, int members, uint64_t x,
                             const uint64_t* xs_dev);
cudaError_t launch_noise_mats(qs_ctx* h, void* mats, int members, int k, const double* U,
                              int noise, int diag_only, const NoiseSrc& src, uint64_t gate_id);
cudaError_t launch_apply_1q(qs_ctx* h, void* psi, int n, int members, int t,
                            const double* U, const void* mats_dev);
cudaError_t launch_apply_kq(qs_ctx* h, void* psi, int n, int members, const Targets& tg,
                            const void* mat_dev, bool per_member, bool real = false);
cudaError_t launch_apply_diag(qs_ctx* h, void* psi, int n, int members, const Targets& tg,
                              const void* diag_dev, bool per_member, uint32_t active_mask);
cudaError_t launch_phase_flip(qs_ctx* h, void* psi, int n, int members, uint64_t index,
                              const uint64_t* per_member);
cudaError_t launch_dm_flip(qs_ctx* h, void* rho, int n, uint64_t index);
// Dense k-qubit block (k = 3..5) on complex64 members with tcgen05 tensor
// cores (3xTF32 split, FP32 accumulation); U_dev = D x D interleaved floats.
// cudaErrorNotSupported unless dense_tc_applicable(n, k) and the handle is complex64.
bool dense_tc_applicable(int n, int k);
cudaError_t launch_dense_tc(qs_ctx* h, void* psi, int n, int members, const int* targets, int k,
                            const float* U_dev);
// T1/T2 relaxation of `count` qubits of a density matrix, two per sweep
// (gamma = 1 - exp(-t/T1), keep = exp(-t/T1), c = exp(-t/T2)).
cudaError_t launch_dm_relax(qs_ctx* h, void* rho, int n, const int* qubits, int count, double gamma,
                            double keep, double c);
// A one-qubit channel with a real superoperator S (local index bit 0 = column
// bit t, bit 1 = row bit t + n) on a Hermitian density matrix (n >= 6): only
// the 2 x 2 groups on or above the diagonal are read and multiplied; tiles
// above the diagonal also write their conjugate transposes through shared
// memory.  S_dev: 16 values of the handle's precision with stride 2.
cudaError_t launch_dm_superop1_herm(qs_ctx* h, void* rho, int n, int t, const void* S_dev);

// reductions (results land in h->small, as doubles)
// reductions over `members` state vectors of 2^n; with group > 1 the values
// of each run of `group` consecutive members are added (a fixed-rank
// member's columns): out[members / group]
cudaError_t launch_dot(qs_ctx* h, const void* psi, const void* ref, int n, int members,
                       int group, double* out_dev);
cudaError_t launch_norm(qs_ctx* h, const void* psi, int n, int members, int group,
                        double* out_dev);
cudaError_t launch_basis_prob(qs_ctx* h, const void* psi, int n, int members, uint64_t x,
                              int group, double* out_dev);
cudaError_t launch_dm_trace(qs_ctx* h, const void* rho, int n, double* out_dev);
cudaError_t launch_dm_expect(qs_ctx* h, const void* rho, const void* ref, int n, double* out_dev);
cudaError_t launch_convert_ref(qs_ctx* h, const double* src_dev, void* dst, size_t count);

// fixed rank, every member of the handle (counts in h->rc): expansion of the
// factors into L' with K Kraus operators (member b's at E + b e_stride,
// e_stride = 0: shared), FP64 Gram matrices, eigensolver and truncation (to
// the members' ranks, or to trunc_r > 0), projection back into the factors.
// max_* are the largest counts over the members (launch sizes).
cudaError_t launch_kraus_expand(qs_ctx* h, const Targets& tg, bool real, const double* E_dev, int K, int e_stride,
                                int max_cols);
// the same with the Kraus set of a noisy gate built on the device per member
cudaError_t launch_kraus_expand_gate(qs_ctx* h, const Targets& tg, bool real, const KrausGate& g, int max_cols);
// Kraus operators of a noisy gate's averaged channel (2 for k = 1 or phase
// noise, 4 for k = 2 rotation noise)
inline int kraus_count(int k, int noise) { return noise == QS_NOISE_ROTATION && k == 2 ? 4 : 2; }
cudaError_t launch_gram(qs_ctx* h, bool real, int max_M);
cudaError_t launch_eig_truncate(qs_ctx* h, int trunc_r, int normalize);
cudaError_t launch_project(qs_ctx* h, bool real, int K, int max_keep);
int gram_rows_per_block(int n);
// one-time kernel attributes of the fixed-rank kernels (outside any capture)
cudaError_t rank_kernel_attributes();
size_t gram_partials_doubles(int n, int members);

// debug noise
cudaError_t launch_debug_noise(uint64_t seed, uint64_t traj, uint64_t gate_id, int count,
                               uint32_t* words_dev, double* normals_dev, cudaStream_t s);

// layout of a fixed-rank member's FP64 block in h->rsmall (doubles, stride
// kRankStride), and of the results in h->small
constexpr size_t kSmallG = 0;          // Gram matrix, 2 * 32 * 32
constexpr size_t kSmallW = 2048;       // eigenvectors, 2 * 32 * 16
constexpr size_t kSmallLam = 3072;     // eigenvalues, 32
constexpr size_t kSmallScale = 3104;   // 1
constexpr size_t kSmallE = 3200;       // Kraus operators, <= 2 * 8 * 16
constexpr int kRankStride = 3456;
constexpr size_t kSmallOutIndex = 4096;  // results, batch doubles

// Write a pending basis start state into memory (no-op when none is pending).
qs_status materialize_basis(qs_ctx* h);
// Copy `count` results from the small block to the host and check the
// device status words (eigensolver, timed-out waits).  Synchronises.
qs_status read_results(qs_ctx* h, double* out, int count);

// helpers
cudaError_t measure_fma_rates(double* fp64_tflops, double* fp32_tflops);
int num_sms();
NoiseSrc noise_src(qs_ctx* h, double e, uint64_t seed);
Targets make_targets(int n, const int* targets, int k);

}  // namespace qs
