// C ABI of the simulator (include/qs.h): argument checks, device memory,
// and the dispatch of each call to the kernels of the handle's mode.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

using qs::Targets;
using cd = std::complex<double>;

namespace {

using qs::kSmallG;
using qs::kSmallW;
using qs::kSmallLam;
using qs::kSmallScale;
using qs::kSmallE;
constexpr size_t kSmallOut = qs::kSmallOutIndex;
constexpr int kMaxKraus = 8;

qs_status fail(qs_handle h, qs_status code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

qs_status cuda_fail(qs_handle h, cudaError_t e, const char* where) {
  return fail(h, QS_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define QS_CUDA(h, call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

bool valid_targets(const qs_ctx* h, const int* t, int k, std::string* why) {
  if (!t) { *why = "targets is NULL"; return false; }
  for (int j = 0; j < k; ++j) {
    if (t[j] < 0 || t[j] >= h->n) { *why = "target out of range"; return false; }
    for (int i = 0; i < j; ++i)
      if (t[i] == t[j]) { *why = "duplicate target"; return false; }
  }
  return true;
}

std::vector<cd> to_cplx(const double* U, int d) {
  std::vector<cd> m((size_t)d * d);
  for (int i = 0; i < d * d; ++i) m[i] = cd(U[2 * i], U[2 * i + 1]);
  return m;
}

std::vector<double> to_interleaved(const std::vector<cd>& m) {
  std::vector<double> v(2 * m.size());
  for (size_t i = 0; i < m.size(); ++i) { v[2 * i] = m[i].real(); v[2 * i + 1] = m[i].imag(); }
  return v;
}

bool is_diagonal(const std::vector<cd>& m, int d) {
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c)
      if (r != c && m[r * d + c] != cd(0.0, 0.0)) return false;
  return true;
}

std::vector<cd> matmul(const std::vector<cd>& a, const std::vector<cd>& b, int d) {
  std::vector<cd> c((size_t)d * d, cd(0.0, 0.0));
  for (int i = 0; i < d; ++i)
    for (int k = 0; k < d; ++k)
      for (int j = 0; j < d; ++j) c[i * d + j] += a[i * d + k] * b[k * d + j];
  return c;
}

// xi-averaged Kraus sets (Eqs. 6 and 9); k = 1 or 2.
std::vector<std::vector<cd>> averaged_kraus(const std::vector<cd>& U, int k, int noise, double e) {
  const int d = 1 << k;
  std::vector<std::vector<cd>> out;
  if (noise == QS_NOISE_ROTATION) {
    const double q = std::exp(-2.0 * e * e);
    const double l1 = 0.5 * (1.0 + q), l2 = 0.5 * (1.0 - q);
    // one-qubit noise operators A_0 = sqrt(l1) I, A_1 = sqrt(l2) J, J = [[0,1],[-1,0]]
    auto one = [&](int which, int r, int c) -> double {
      if (which == 0) return r == c ? std::sqrt(l1) : 0.0;
      if (r == 0 && c == 1) return std::sqrt(l2);
      if (r == 1 && c == 0) return -std::sqrt(l2);
      return 0.0;
    };
    const int nops = k == 1 ? 2 : 4;
    for (int op = 0; op < nops; ++op) {
      const int wa = op & 1, wb = (op >> 1) & 1;       // targets[0] varies fastest
      std::vector<cd> N((size_t)d * d, cd(0.0, 0.0));
      for (int r = 0; r < d; ++r)
        for (int c = 0; c < d; ++c) {
          double v = one(wa, r & 1, c & 1);
          if (k == 2) v *= one(wb, (r >> 1) & 1, (c >> 1) & 1);
          N[r * d + c] = v;
        }
      out.push_back(matmul(U, N, d));
    }
  } else {
    const double P = std::exp(-e * e);
    std::vector<cd> d1((size_t)d * d, cd(0.0, 0.0)), d2((size_t)d * d, cd(0.0, 0.0));
    for (int i = 0; i < d; ++i) d1[i * d + i] = 1.0;
    d1[(d - 1) * d + (d - 1)] = std::sqrt(P);
    d2[(d - 1) * d + (d - 1)] = std::sqrt(1.0 - P);
    out.push_back(matmul(U, d1, d));
    out.push_back(matmul(U, d2, d));
  }
  return out;
}

bool kraus_complete(const std::vector<std::vector<cd>>& ks, int d, double tol) {
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c) {
      cd s(0.0, 0.0);
      for (const auto& E : ks)
        for (int m = 0; m < d; ++m) s += std::conj(E[m * d + r]) * E[m * d + c];
      if (std::abs(s - (r == c ? cd(1.0, 0.0) : cd(0.0, 0.0))) > tol) return false;
    }
  return true;
}

// superoperator sum_i E_i (x) conj(E_i): row factor on the high local bits
std::vector<cd> superop(const std::vector<std::vector<cd>>& ks, int d) {
  const int D = d * d;
  std::vector<cd> S((size_t)D * D, cd(0.0, 0.0));
  for (const auto& E : ks)
    for (int ro = 0; ro < d; ++ro)
      for (int co = 0; co < d; ++co)
        for (int ri = 0; ri < d; ++ri)
          for (int ci = 0; ci < d; ++ci)
            S[(size_t)(ro * d + co) * D + (ri * d + ci)] += E[ro * d + ri] * std::conj(E[co * d + ci]);
  return S;
}

template <typename R>
std::vector<R> to_real_array(const std::vector<cd>& m) {
  std::vector<R> v(2 * m.size());
  for (size_t i = 0; i < m.size(); ++i) { v[2 * i] = (R)m[i].real(); v[2 * i + 1] = (R)m[i].imag(); }
  return v;
}

// Upload a uniform matrix (or diagonal) in the handle's precision into h->mats.
qs_status upload_mat(qs_handle h, const std::vector<cd>& m) {
  const size_t bytes = m.size() * 2 * (h->esize / 2);
  if (bytes > h->mats_cap) return fail(h, QS_ERR_INVALID_ARG, "matrix too large");
  if (h->dtype == QS_C64) {
    auto v = to_real_array<float>(m);
    QS_CUDA(h, cudaMemcpyAsync(h->mats, v.data(), bytes, cudaMemcpyHostToDevice, h->stream));
  } else {
    auto v = to_real_array<double>(m);
    QS_CUDA(h, cudaMemcpyAsync(h->mats, v.data(), bytes, cudaMemcpyHostToDevice, h->stream));
  }
  return QS_OK;
}

// Apply a uniform matrix U (dimension d = 2^k) on `targets` of every member.
qs_status apply_uniform(qs_handle h, void* psi, int n, int members, const int* targets, int k,
                        const std::vector<cd>& U) {
  const int d = 1 << k;
  const Targets tg = qs::make_targets(n, targets, k);
  if (is_diagonal(U, d)) {
    uint32_t mask = 0;
    std::vector<cd> diag(d);
    for (int l = 0; l < d; ++l) {
      diag[l] = U[l * d + l];
      if (diag[l] != cd(1.0, 0.0)) mask |= 1u << l;
    }
    if (!mask) return QS_OK;
    qs_status st = upload_mat(h, diag);
    if (st != QS_OK) return st;
    QS_CUDA(h, qs::launch_apply_diag(h, psi, n, members, tg, h->mats, false, mask));
    return QS_OK;
  }
  if (k == 1) {
    const auto v = to_interleaved(U);
    QS_CUDA(h, qs::launch_apply_1q(h, psi, n, members, targets[0], v.data(), nullptr));
    return QS_OK;
  }
  qs_status st = upload_mat(h, U);
  if (st != QS_OK) return st;
  if (k >= 3 && h->dtype == QS_C64 && h->tensor_cores && qs::dense_tc_applicable(n, k)) {
    QS_CUDA(h, qs::launch_dense_tc(h, psi, n, members, targets, k, static_cast<const float*>(h->mats)));
    return QS_OK;
  }
  bool real = true;
  for (const auto& v : U) if (v.imag() != 0.0) real = false;
  QS_CUDA(h, qs::launch_apply_kq(h, psi, n, members, tg, h->mats, false, real));
  return QS_OK;
}

// DENSITY: superoperator of a Kraus set on bits (t, t + n).
bool all_real(const std::vector<cd>& m);

qs_status dm_apply_channel(qs_handle h, const int* targets, int k, const std::vector<std::vector<cd>>& ks) {
  if (k == 1 && h->hermitian && h->n >= 6) {
    // a real, non-diagonal superoperator (every noisy Hadamard) on a Hermitian
    // rho: the groups on and above the diagonal only, mirrored below
    const auto S = superop(ks, 2);
    if (all_real(S) && !is_diagonal(S, 4)) {
      const qs_status st = upload_mat(h, S);
      if (st != QS_OK) return st;
      QS_CUDA(h, qs::launch_dm_superop1_herm(h, h->state, h->n, targets[0], h->mats));
      return QS_OK;
    }
  }
  int t2[2 * qs::kMaxK];
  for (int j = 0; j < k; ++j) { t2[j] = targets[j]; t2[k + j] = targets[j] + h->n; }
  return apply_uniform(h, h->state, 2 * h->n, 1, t2, 2 * k, superop(ks, 1 << k));
}

bool all_real(const std::vector<cd>& m) {
  for (const auto& v : m) if (v.imag() != 0.0) return false;
  return true;
}

// FIXED_RANK: columns the unitary kernels sweep -- the live ones of a single
// member, or every column of every member (dead columns are zero and stay so)
int rank_swept(qs_handle h) { return h->batch == 1 ? h->cols : h->batch * h->rank; }

// host mirror of the members' column counts -> device (small synchronous copies)
qs_status rank_upload_counts(qs_handle h) {
  QS_CUDA(h, cudaMemcpyAsync(h->rc.cols, h->m_cols.data(), h->batch * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  QS_CUDA(h, cudaMemcpyAsync(h->rc.rank, h->m_rank.data(), h->batch * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  h->cols = *std::max_element(h->m_cols.begin(), h->m_cols.end());
  return QS_OK;
}

// Gram matrices, eigensolver, truncation and projection of every member's L'
// (M_b columns on the device); keep_b = min(r_b, M_b) (r_b = trunc_r when > 0)
// mirrored on the host.  K: Kraus operators of the channel (L' = K m_b columns).
qs_status rank_truncate_work(qs_handle h, int K, int trunc_r, int normalize) {
  int max_M = 0, max_keep = 0;
  for (int b = 0; b < h->batch; ++b) {
    const int M = K * h->m_cols[b];
    const int keep = std::min(trunc_r > 0 ? trunc_r : h->m_rank[b], M);
    max_M = std::max(max_M, M);
    max_keep = std::max(max_keep, keep);
    h->m_cols[b] = keep;
  }
  QS_CUDA(h, qs::launch_gram(h, h->real_factor, max_M));
  QS_CUDA(h, qs::launch_eig_truncate(h, trunc_r, normalize));
  QS_CUDA(h, qs::launch_project(h, h->real_factor, K, max_keep));
  h->cols = *std::max_element(h->m_cols.begin(), h->m_cols.end());
  return QS_OK;
}

// FIXED_RANK: L'_b = [E_1 L_b | ..], then truncation when K > 1.  ks: one
// Kraus set for every member, or (per_member) `batch` sets of K operators.
qs_status rank_apply_kraus(qs_handle h, const int* targets, int k, const std::vector<std::vector<cd>>& ks,
                           int per_member = 0) {
  const int d = 1 << k;
  const int K = per_member ? (int)ks.size() / h->batch : (int)ks.size();
  for (const auto& E : ks) if (!all_real(E)) h->real_factor = false;
  if (K == 1 && !per_member) return apply_uniform(h, h->state, h->n, rank_swept(h), targets, k, ks[0]);
  int max_cols = 0;
  for (int b = 0; b < h->batch; ++b) {
    if (K * h->m_cols[b] > std::min(qs::kMaxGramDim, h->mcap))
      return fail(h, QS_ERR_NOT_SUPPORTED, "Kraus count times rank exceeds the Gram-matrix limit of 32");
    max_cols = std::max(max_cols, h->m_cols[b]);
  }
  std::vector<double> e;
  for (const auto& E : ks) { auto v = to_interleaved(E); e.insert(e.end(), v.begin(), v.end()); }
  const size_t set_bytes = (size_t)K * d * d * 2 * sizeof(double);
  double* Edev = h->rsmall + qs::kSmallE;
  if (per_member) {
    QS_CUDA(h, cudaMemcpy2DAsync(Edev, qs::kRankStride * sizeof(double), e.data(), set_bytes, set_bytes, h->batch,
                                 cudaMemcpyHostToDevice, h->stream));
  } else {
    QS_CUDA(h, cudaMemcpyAsync(Edev, e.data(), set_bytes, cudaMemcpyHostToDevice, h->stream));
  }
  const Targets tg = qs::make_targets(h->n, targets, k);
  QS_CUDA(h, qs::launch_kraus_expand(h, tg, h->real_factor, Edev, K, per_member ? qs::kRankStride : 0, max_cols));
  return rank_truncate_work(h, K, 0, h->normalize);
}

// FIXED_RANK: the averaged channel of a noisy gate on every member, then
// truncation
qs_status rank_channel_gate(qs_handle h, const int* targets, const qs::KrausGate& g) {
  const int K = qs::kraus_count(g.k, g.noise);
  bool real = true;
  for (int i = 1; i < 2 * (1 << g.k) * (1 << g.k); i += 2) real &= g.U[i] == 0.0;
  if (!real) h->real_factor = false;
  int max_cols = 0;
  for (int b = 0; b < h->batch; ++b) {
    if (K * h->m_cols[b] > std::min(qs::kMaxGramDim, h->mcap))
      return fail(h, QS_ERR_NOT_SUPPORTED, "Kraus count times rank exceeds the Gram-matrix limit of 32");
    max_cols = std::max(max_cols, h->m_cols[b]);
  }
  const Targets tg = qs::make_targets(h->n, targets, g.k);
  QS_CUDA(h, qs::launch_kraus_expand_gate(h, tg, h->real_factor, g, max_cols));
  return rank_truncate_work(h, K, 0, h->normalize);
}

// FIXED_RANK: column c = 0 of every member <- |x> (or Eq. 16's state), the rest 0
qs_status rank_set_start(qs_handle h, int entangled, uint64_t x, const uint64_t* xs = nullptr) {
  const size_t N = 1ull << h->n;
  QS_CUDA(h, cudaMemsetAsync(h->state, 0, h->state_elems * h->esize, h->stream));
  for (int b = 0; b < h->batch; ++b) {
    void* col0 = (char*)h->state + (size_t)b * h->rank * N * h->esize;
    if (entangled) QS_CUDA(h, qs::launch_set_entangled(h, col0, 1, 0));
    else QS_CUDA(h, qs::launch_set_basis(h, col0, h->n, 1, xs ? xs[b] : x, nullptr));
  }
  std::fill(h->m_cols.begin(), h->m_cols.end(), 1);
  h->real_factor = true;
  return rank_upload_counts(h);
}

qs_status read_out(qs_handle h, double* out, int count) { return qs::read_results(h, out, count); }

}  // namespace

namespace qs {
qs_status read_results(qs_ctx* h, double* out, int count) {
  QS_CUDA(h, cudaMemcpyAsync(out, h->small + kSmallOut, count * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  QS_CUDA(h, cudaStreamSynchronize(h->stream));
  int status[4] = {0, 0, 0, 0};
  QS_CUDA(h, cudaMemcpy(status, h->dstatus, sizeof(status), cudaMemcpyDeviceToHost));
  if (status[2] != 0 || status[3] != 0) {
    // reported once: the words are cleared so the handle's next run starts clean
    QS_CUDA(h, cudaMemset(h->dstatus + 2, 0, 2 * sizeof(int)));
    return fail(h, QS_ERR_TIMEOUT, status[2] != 0 ? "a fused pass timed out waiting for a tile copy"
                                                  : "a tensor-core block timed out waiting for its MMAs");
  }
  if (h->mode == QS_FIXED_RANK && status[1] != 0)
    return fail(h, QS_ERR_CUDA, status[1] == 1 ? "eigensolver did not converge" : "tie-cluster basis incomplete");
  return QS_OK;
}

qs_status materialize_basis(qs_ctx* h) {
  if (!h->pending) return QS_OK;
  const uint64_t* xs = h->pending == 2 ? h->m_basis : nullptr;
  QS_CUDA(h, launch_set_basis(h, h->state, h->n, h->batch, h->pending_x, xs));
  h->pending = 0;
  return QS_OK;
}

NoiseSrc noise_src(qs_ctx* h, double e, uint64_t seed) {
  NoiseSrc s{};
  s.e0 = e;
  s.seed0 = seed;
  s.traj0 = h->traj_offset;
  if (h->member_noise) { s.e = h->m_e; s.seed = h->m_seed; s.traj = h->m_traj; }
  return s;
}
}  // namespace qs

extern "C" {

const char* qs_version(void) { return "paper_1412_2293_gb300 0.1 (sm_103a)"; }

qs_status qs_create(int n, int batch, int rank, qs_mode mode, qs_dtype dtype, void* cuda_stream,
                    qs_handle* out) {
  if (!out) return QS_ERR_INVALID_ARG;
  *out = nullptr;
  if (n < 1 || n > 40) return QS_ERR_INVALID_ARG;
  if (mode != QS_STATEVEC && mode != QS_DENSITY && mode != QS_FIXED_RANK) return QS_ERR_INVALID_ARG;
  if (dtype != QS_C64 && dtype != QS_C128) return QS_ERR_INVALID_ARG;
  if (mode == QS_STATEVEC && batch < 1) return QS_ERR_INVALID_ARG;
  if (mode == QS_DENSITY && batch != 1) return QS_ERR_INVALID_ARG;
  if (mode == QS_FIXED_RANK && batch < 1) return QS_ERR_INVALID_ARG;
  if (mode == QS_FIXED_RANK && (rank < 1 || rank > qs::kMaxRank)) return QS_ERR_INVALID_ARG;
  if (mode == QS_DENSITY && 2 * n > 40) return QS_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) { cudaGetLastError(); return QS_ERR_CUDA; }

  qs_ctx* h = new (std::nothrow) qs_ctx();
  if (!h) return QS_ERR_OUT_OF_MEMORY;
  h->n = n;
  h->batch = batch;
  h->rank = mode == QS_FIXED_RANK ? rank : 0;
  h->mode = mode;
  h->dtype = dtype;
  h->stream = (cudaStream_t)cuda_stream;
  h->esize = qs::elem_size(dtype);
  cudaGetDevice(&h->device);

  const uint64_t N = 1ull << n;
  size_t members = mode == QS_STATEVEC ? (size_t)batch : 1;
  if (mode == QS_STATEVEC) h->state_elems = (size_t)batch * N;
  else if (mode == QS_DENSITY) h->state_elems = N * N;
  else h->state_elems = (size_t)batch * rank * N;

  auto bail = [&](qs_status st) { qs_destroy(h); return st; };
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  if (h->state_elems * h->esize > free_b) return bail(QS_ERR_OUT_OF_MEMORY);
  if (cudaMalloc(&h->state, h->state_elems * h->esize) != cudaSuccess) { cudaGetLastError(); return bail(QS_ERR_OUT_OF_MEMORY); }
  if (mode == QS_FIXED_RANK) {
    // L' of a member: at most kMaxKraus operators times its rank, and the Gram limit
    h->mcap = std::min(qs::kMaxGramDim, kMaxKraus * rank);
    h->work_elems = (size_t)batch * h->mcap * N;
    if (h->work_elems * h->esize > free_b - h->state_elems * h->esize) return bail(QS_ERR_OUT_OF_MEMORY);
    if (cudaMalloc(&h->work, h->work_elems * h->esize) != cudaSuccess) { cudaGetLastError(); return bail(QS_ERR_OUT_OF_MEMORY); }
    members = (size_t)batch * std::max(h->mcap, rank);
    if (cudaMalloc((void**)&h->rsmall, (size_t)batch * qs::kRankStride * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return bail(QS_ERR_OUT_OF_MEMORY); }
    int* counts = nullptr;
    if (cudaMalloc((void**)&counts, 4 * (size_t)batch * sizeof(int)) != cudaSuccess) { cudaGetLastError(); return bail(QS_ERR_OUT_OF_MEMORY); }
    h->rc = qs::RankCounts{counts, counts + batch, counts + 2 * batch, counts + 3 * batch};
    h->m_cols.assign(batch, 1);
    h->m_rank.assign(batch, rank);
    if (qs::rank_kernel_attributes() != cudaSuccess) return bail(QS_ERR_CUDA);
  }
  // scratch sized for every reduction of this shape, so that runs never allocate
  const uint64_t chunks = (N + 4095) / 4096;
  size_t partials = 2 * chunks * members;
  if (mode == QS_DENSITY) partials = std::max<size_t>(partials, 2 * N);
  if (mode == QS_FIXED_RANK) partials = std::max<size_t>(partials, qs::gram_partials_doubles(n, batch));
  h->partials_cap = partials;
  if (cudaMalloc((void**)&h->partials, partials * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return bail(QS_ERR_OUT_OF_MEMORY); }
  h->mats_cap = std::max<size_t>((size_t)batch * 2 * 16, 2 * 1024) * (h->esize / 2);
  if (cudaMalloc(&h->mats, h->mats_cap) != cudaSuccess) { cudaGetLastError(); return bail(QS_ERR_OUT_OF_MEMORY); }
  h->small_cap = kSmallOut + std::max<size_t>((size_t)batch, 64);
  if (cudaMalloc((void**)&h->small, h->small_cap * sizeof(double)) != cudaSuccess) { cudaGetLastError(); return bail(QS_ERR_OUT_OF_MEMORY); }
  if (cudaMalloc((void**)&h->dstatus, 4 * sizeof(int)) != cudaSuccess) { cudaGetLastError(); return bail(QS_ERR_OUT_OF_MEMORY); }
  if (cudaMemsetAsync(h->dstatus, 0, 4 * sizeof(int), h->stream) != cudaSuccess) return bail(QS_ERR_CUDA);
  h->cols = 1;
  cudaError_t e = cudaSuccess;
  if (mode == QS_STATEVEC) { h->pending = 1; h->pending_x = 0; }
  else if (mode == QS_DENSITY) e = qs::launch_set_basis(h, h->state, n, 1, 0, nullptr);
  else if (rank_set_start(h, 0, 0) != QS_OK) return bail(QS_ERR_CUDA);
  if (e != cudaSuccess) return bail(QS_ERR_CUDA);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bail(QS_ERR_CUDA);
  *out = h;
  return QS_OK;
}

qs_status qs_destroy(qs_handle h) {
  if (!h) return QS_ERR_INVALID_ARG;
  cudaStreamSynchronize(h->stream);
  void* ptrs[] = {h->state, h->work, h->partials, h->mats, h->small, h->dstatus, h->m_e,
                  h->m_seed, h->m_traj, h->m_marked, h->ref, h->m_basis, h->rsmall, h->rc.cols};
  for (void* p : ptrs) if (p) cudaFree(p);
  if (h->hpinned) cudaFreeHost(h->hpinned);
  delete h;
  return QS_OK;
}

const char* qs_last_error(qs_handle h) { return h ? h->err.c_str() : "null handle"; }

qs_status qs_info(qs_handle h, int* n, int* batch, int* rank, int* mode, int* dtype, int* results) {
  if (!h) return QS_ERR_INVALID_ARG;
  if (n) *n = h->n;
  if (batch) *batch = h->batch;
  if (rank) *rank = h->rank;
  if (mode) *mode = (int)h->mode;
  if (dtype) *dtype = (int)h->dtype;
  if (results) *results = h->mode == QS_DENSITY ? 1 : h->batch;
  return QS_OK;
}

qs_status qs_synchronize(qs_handle h) {
  if (!h) return QS_ERR_INVALID_ARG;
  QS_CUDA(h, cudaStreamSynchronize(h->stream));
  return QS_OK;
}

qs_status qs_set_basis_state(qs_handle h, uint64_t x) {
  if (!h) return QS_ERR_INVALID_ARG;
  if (x >= (1ull << h->n)) return fail(h, QS_ERR_INVALID_ARG, "basis index out of range");
  if (h->mode == QS_STATEVEC) {
    h->pending = 1;                       // written by its first consumer
    h->pending_x = x;
  } else if (h->mode == QS_DENSITY) {
    const uint64_t N = 1ull << h->n;
    QS_CUDA(h, qs::launch_set_basis(h, h->state, 2 * h->n, 1, x * N + x, nullptr));
    h->hermitian = true;
  } else {
    return rank_set_start(h, 0, x);
  }
  return QS_OK;
}

qs_status qs_set_maximally_entangled(qs_handle h) {
  if (!h) return QS_ERR_INVALID_ARG;
  if (h->n % 2) return fail(h, QS_ERR_INVALID_ARG, "the maximally entangled state needs an even qubit count");
  h->pending = 0;
  if (h->mode == QS_STATEVEC) {
    QS_CUDA(h, qs::launch_set_entangled(h, h->state, h->batch, 0));
  } else if (h->mode == QS_DENSITY) {
    QS_CUDA(h, qs::launch_set_entangled(h, h->state, 1, 1));
    h->hermitian = true;
  } else {
    return rank_set_start(h, 1, 0);
  }
  return QS_OK;
}

qs_status qs_set_basis_states(qs_handle h, const uint64_t* xs) {
  if (!h || !xs) return QS_ERR_INVALID_ARG;
  if (h->mode == QS_DENSITY) return fail(h, QS_ERR_NOT_SUPPORTED, "per-member basis states need STATEVEC or FIXED_RANK");
  for (int b = 0; b < h->batch; ++b)
    if (xs[b] >= (1ull << h->n)) return fail(h, QS_ERR_INVALID_ARG, "basis index out of range");
  if (h->mode == QS_FIXED_RANK) return rank_set_start(h, 0, 0, xs);
  if (!h->m_basis) QS_CUDA(h, cudaMalloc((void**)&h->m_basis, h->batch * sizeof(uint64_t)));
  // an earlier run may still read m_basis
  QS_CUDA(h, cudaStreamSynchronize(h->stream));
  QS_CUDA(h, cudaMemcpy(h->m_basis, xs, h->batch * sizeof(uint64_t), cudaMemcpyHostToDevice));
  h->pending = 2;                         // written by its first consumer
  return QS_OK;
}

qs_status qs_apply_gate(qs_handle h, const int* targets, int k, const double* U) {
  if (!h) return QS_ERR_INVALID_ARG;
  { const qs_status st = qs::materialize_basis(h); if (st != QS_OK) return st; }
  if (k < 1 || k > qs::kMaxK) return fail(h, QS_ERR_INVALID_ARG, "k must be 1..5");
  if (!U) return fail(h, QS_ERR_INVALID_ARG, "U is NULL");
  std::string why;
  if (!valid_targets(h, targets, k, &why)) return fail(h, QS_ERR_INVALID_ARG, why);
  const auto M = to_cplx(U, 1 << k);
  if (h->mode == QS_STATEVEC) return apply_uniform(h, h->state, h->n, h->batch, targets, k, M);
  if (h->mode == QS_FIXED_RANK) {
    if (!all_real(M)) h->real_factor = false;
    return apply_uniform(h, h->state, h->n, rank_swept(h), targets, k, M);
  }
  if (k <= 2) return dm_apply_channel(h, targets, k, {M});
  // k = 3, 4: U on the row bits t + n and conj(U) on the column bits t, two
  // sweeps of k-qubit gates on the 2n-qubit vector (a 2k-qubit superoperator
  // would exceed the dense-gate limit)
  int rows[qs::kMaxK];
  for (int j = 0; j < k; ++j) rows[j] = targets[j] + h->n;
  std::vector<cd> Mc(M.size());
  for (size_t i = 0; i < M.size(); ++i) Mc[i] = std::conj(M[i]);
  const qs_status st = apply_uniform(h, h->state, 2 * h->n, 1, rows, k, M);
  if (st != QS_OK) return st;
  return apply_uniform(h, h->state, 2 * h->n, 1, targets, k, Mc);
}

qs_status qs_apply_phase_flip(qs_handle h, uint64_t index) {
  if (!h) return QS_ERR_INVALID_ARG;
  { const qs_status st = qs::materialize_basis(h); if (st != QS_OK) return st; }
  if (index >= (1ull << h->n)) return fail(h, QS_ERR_INVALID_ARG, "index out of range");
  if (h->mode == QS_STATEVEC) { QS_CUDA(h, qs::launch_phase_flip(h, h->state, h->n, h->batch, index, nullptr)); }
  else if (h->mode == QS_FIXED_RANK) { QS_CUDA(h, qs::launch_phase_flip(h, h->state, h->n, rank_swept(h), index, nullptr)); }
  else { QS_CUDA(h, qs::launch_dm_flip(h, h->state, h->n, index)); }
  return QS_OK;
}

qs_status qs_apply_branch_gate(qs_handle h, const int* targets, int k, const double* U, qs_noise noise,
                               double e, int rotated) {
  if (!h) return QS_ERR_INVALID_ARG;
  { const qs_status st = qs::materialize_basis(h); if (st != QS_OK) return st; }
  if (k < 1 || k > 2) return fail(h, QS_ERR_INVALID_ARG, "noisy gates are defined for k = 1, 2");
  if (!U) return fail(h, QS_ERR_INVALID_ARG, "U is NULL");
  if (!(e >= 0.0) || !std::isfinite(e)) return fail(h, QS_ERR_INVALID_ARG, "e must be finite and >= 0");
  if (noise != QS_NOISE_ROTATION && noise != QS_NOISE_PHASE) return fail(h, QS_ERR_INVALID_ARG, "bad noise kind");
  std::string why;
  if (!valid_targets(h, targets, k, &why)) return fail(h, QS_ERR_INVALID_ARG, why);
  const int d = 1 << k;
  const auto ks = averaged_kraus(to_cplx(U, d), k, noise, e);
  std::vector<cd> B = ks[0];
  const double P = std::exp(-e * e);
  if (rotated && noise == QS_NOISE_PHASE && P < 1.0) {
    // Eqs. 12-14: B_1 = (E_1 + f E_2) / sqrt(1 + f^2), f = (sqrt(1 + 3P) - P - 1) / sqrt(P (1 - P))
    const double f = (std::sqrt(1.0 + 3.0 * P) - P - 1.0) / std::sqrt(P * (1.0 - P));
    const double sc = 1.0 / std::sqrt(1.0 + f * f);
    for (size_t i = 0; i < B.size(); ++i) B[i] = sc * (ks[0][i] + f * ks[1][i]);
  }
  if (h->mode == QS_DENSITY) return dm_apply_channel(h, targets, k, {B});
  if (h->mode == QS_FIXED_RANK) {
    if (!all_real(B)) h->real_factor = false;
    return apply_uniform(h, h->state, h->n, rank_swept(h), targets, k, B);
  }
  return apply_uniform(h, h->state, h->n, h->batch, targets, k, B);
}

qs_status qs_apply_noisy_gate(qs_handle h, const int* targets, int k, const double* U, qs_noise noise,
                              double e, uint64_t seed, uint64_t gate_id) {
  if (!h) return QS_ERR_INVALID_ARG;
  { const qs_status st = qs::materialize_basis(h); if (st != QS_OK) return st; }
  if (k < 1 || k > 2) return fail(h, QS_ERR_INVALID_ARG, "noisy gates are defined for k = 1, 2");
  if (!U) return fail(h, QS_ERR_INVALID_ARG, "U is NULL");
  if (!(e >= 0.0) || !std::isfinite(e)) return fail(h, QS_ERR_INVALID_ARG, "e must be finite and >= 0");
  if (noise != QS_NOISE_ROTATION && noise != QS_NOISE_PHASE) return fail(h, QS_ERR_INVALID_ARG, "bad noise kind");
  std::string why;
  if (!valid_targets(h, targets, k, &why)) return fail(h, QS_ERR_INVALID_ARG, why);
  const int d = 1 << k;
  const auto M = to_cplx(U, d);
  if (h->mode == QS_STATEVEC) {
    const qs::NoiseSrc src = qs::noise_src(h, e, seed);
    const Targets tg = qs::make_targets(h->n, targets, k);
    const bool diag = noise == QS_NOISE_PHASE && is_diagonal(M, d);
    QS_CUDA(h, qs::launch_noise_mats(h, h->mats, h->batch, k, U, noise, diag ? 1 : 0, src, gate_id));
    if (diag) {
      uint32_t mask = 1u << (d - 1);
      for (int l = 0; l < d - 1; ++l) if (M[l * d + l] != cd(1.0, 0.0)) mask |= 1u << l;
      QS_CUDA(h, qs::launch_apply_diag(h, h->state, h->n, h->batch, tg, h->mats, true, mask));
    } else if (k == 1) {
      QS_CUDA(h, qs::launch_apply_1q(h, h->state, h->n, h->batch, targets[0], nullptr, h->mats));
    } else {
      QS_CUDA(h, qs::launch_apply_kq(h, h->state, h->n, h->batch, tg, h->mats, true));
    }
    return QS_OK;
  }
  if (h->mode == QS_FIXED_RANK) {
    // the averaged channel, its Kraus set built on the device from e (or from
    // each member's own e, qs_set_member_noise)
    qs::KrausGate g{};
    for (int i = 0; i < 2 * d * d; ++i) g.U[i] = U[i];
    g.k = k;
    g.noise = noise;
    g.e_value = e;
    g.e_member = h->member_noise ? h->m_e : nullptr;
    return rank_channel_gate(h, targets, g);
  }
  const auto ks = averaged_kraus(M, k, noise, e);
  if (h->mode == QS_DENSITY) return dm_apply_channel(h, targets, k, ks);
  return rank_apply_kraus(h, targets, k, ks);
}

qs_status qs_apply_kraus(qs_handle h, const int* targets, int k, const double* E, int num_ops) {
  if (!h) return QS_ERR_INVALID_ARG;
  if (h->mode == QS_STATEVEC) return fail(h, QS_ERR_NOT_SUPPORTED, "Kraus channels need DENSITY or FIXED_RANK");
  if (k < 1 || k > 2) return fail(h, QS_ERR_INVALID_ARG, "Kraus operators are limited to k = 1, 2");
  if (!E || num_ops < 1 || num_ops > kMaxKraus) return fail(h, QS_ERR_INVALID_ARG, "need 1..8 Kraus operators");
  std::string why;
  if (!valid_targets(h, targets, k, &why)) return fail(h, QS_ERR_INVALID_ARG, why);
  const int d = 1 << k;
  std::vector<std::vector<cd>> ks;
  for (int i = 0; i < num_ops; ++i) ks.push_back(to_cplx(E + (size_t)i * 2 * d * d, d));
  if (!kraus_complete(ks, d, 1e-12)) return fail(h, QS_ERR_INVALID_ARG, "sum E^dagger E != I (tolerance 1e-12)");
  if (h->mode == QS_DENSITY) return dm_apply_channel(h, targets, k, ks);
  return rank_apply_kraus(h, targets, k, ks);
}

qs_status qs_apply_relaxation(qs_handle h, const int* qubits, int count, double t, double T1, double T2) {
  if (!h) return QS_ERR_INVALID_ARG;
  if (h->mode == QS_STATEVEC) return fail(h, QS_ERR_NOT_SUPPORTED, "relaxation needs DENSITY or FIXED_RANK");
  if (count < 0 || (count > 0 && !qubits)) return fail(h, QS_ERR_INVALID_ARG, "bad qubit list");
  for (int j = 0; j < count; ++j) {
    if (qubits[j] < 0 || qubits[j] >= h->n) return fail(h, QS_ERR_INVALID_ARG, "qubit out of range");
    for (int i = 0; i < j; ++i)
      if (qubits[i] == qubits[j]) return fail(h, QS_ERR_INVALID_ARG, "duplicate qubit");
  }
  if (!(t >= 0.0) || !std::isfinite(t)) return fail(h, QS_ERR_INVALID_ARG, "t must be finite and >= 0");
  if (!(T1 > 0.0) || !(T2 > 0.0)) return fail(h, QS_ERR_INVALID_ARG, "T1 and T2 must be > 0 (inf allowed)");
  if (T2 > 2.0 * T1) return fail(h, QS_ERR_INVALID_ARG, "T2 > 2 T1 is not a channel");
  { const qs_status st = qs::materialize_basis(h); if (st != QS_OK) return st; }
  const double keep = std::exp(-t / T1), c = std::exp(-t / T2), gamma = 1.0 - keep;
  if (count == 0 || (gamma == 0.0 && c == 1.0)) return QS_OK;
  if (h->mode == QS_DENSITY) {
    QS_CUDA(h, qs::launch_dm_relax(h, h->state, h->n, qubits, count, gamma, keep, c));
    return QS_OK;
  }
  // FIXED_RANK: the Kraus set diag(1, c), sqrt(gamma) |0><1|, diag(0, sqrt(keep - c^2)),
  // zero operators left out, one expansion and truncation per qubit
  std::vector<std::vector<cd>> ks;
  ks.push_back({cd(1, 0), cd(0, 0), cd(0, 0), cd(c, 0)});
  if (gamma > 0.0) ks.push_back({cd(0, 0), cd(std::sqrt(gamma), 0), cd(0, 0), cd(0, 0)});
  const double d2 = keep - c * c;
  if (d2 > 0.0) ks.push_back({cd(0, 0), cd(0, 0), cd(0, 0), cd(std::sqrt(d2), 0)});
  for (int j = 0; j < count; ++j) {
    const qs_status st = rank_apply_kraus(h, qubits + j, 1, ks);
    if (st != QS_OK) return st;
  }
  return QS_OK;
}

qs_status qs_truncate_rank(qs_handle h, int r, int normalize) {
  if (!h) return QS_ERR_INVALID_ARG;
  if (h->mode != QS_FIXED_RANK) return fail(h, QS_ERR_NOT_SUPPORTED, "truncation needs FIXED_RANK");
  if (r < 1 || r > h->rank) return fail(h, QS_ERR_INVALID_ARG, "r must be 1..rank");
  // copy every member's L into its work columns (M_b = m_b), then truncate
  // from there back into L
  const size_t col_bytes = (1ull << h->n) * h->esize;
  QS_CUDA(h, cudaMemcpy2DAsync(h->work, (size_t)h->mcap * col_bytes, h->state, (size_t)h->rank * col_bytes,
                               (size_t)h->rank * col_bytes, h->batch, cudaMemcpyDeviceToDevice, h->stream));
  QS_CUDA(h, cudaMemcpyAsync(h->rc.M, h->m_cols.data(), h->batch * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  return rank_truncate_work(h, 1, r, normalize);
}

qs_status qs_set_tensor_cores(qs_handle h, int on) {
  if (!h) return QS_ERR_INVALID_ARG;
  h->tensor_cores = on != 0;
  return QS_OK;
}

qs_status qs_set_normalize(qs_handle h, int normalize) {
  if (!h) return QS_ERR_INVALID_ARG;
  h->normalize = normalize ? 1 : 0;
  return QS_OK;
}

qs_status qs_get_rank(qs_handle h, int* out) {
  if (!h || !out) return QS_ERR_INVALID_ARG;
  *out = h->mode == QS_FIXED_RANK ? h->cols : 1;
  return QS_OK;
}

static qs_status upload_ref(qs_handle h, const double* ref, void* dst) {
  const size_t N = 1ull << h->n;
  double* tmp = nullptr;
  QS_CUDA(h, cudaMallocAsync((void**)&tmp, N * 2 * sizeof(double), h->stream));
  QS_CUDA(h, cudaMemcpyAsync(tmp, ref, N * 2 * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  QS_CUDA(h, qs::launch_convert_ref(h, tmp, dst, N));
  QS_CUDA(h, cudaFreeAsync(tmp, h->stream));
  return QS_OK;
}

static qs_status fidelity_dev(qs_handle h, const void* phi_dev, double* out) {
  double* o = h->small + kSmallOut;
  if (h->mode == QS_STATEVEC) {
    QS_CUDA(h, qs::launch_dot(h, h->state, phi_dev, h->n, h->batch, 1, o));
    return read_out(h, out, h->batch);
  }
  if (h->mode == QS_FIXED_RANK) {
    const int cols = rank_swept(h);
    QS_CUDA(h, qs::launch_dot(h, h->state, phi_dev, h->n, cols, cols / h->batch, o));
    return read_out(h, out, h->batch);
  }
  QS_CUDA(h, qs::launch_dm_expect(h, h->state, phi_dev, h->n, o));
  return read_out(h, out, 1);
}

qs_status qs_fidelity(qs_handle h, const double* ref, uint64_t ref_basis, double* out) {
  if (!h || !out) return QS_ERR_INVALID_ARG;
  { const qs_status st = qs::materialize_basis(h); if (st != QS_OK) return st; }
  const uint64_t N = 1ull << h->n;
  double* o = h->small + kSmallOut;
  if (!ref) {
    if (ref_basis >= N) return fail(h, QS_ERR_INVALID_ARG, "basis index out of range");
    if (h->mode == QS_STATEVEC) {
      QS_CUDA(h, qs::launch_basis_prob(h, h->state, h->n, h->batch, ref_basis, 1, o));
      return read_out(h, out, h->batch);
    }
    if (h->mode == QS_FIXED_RANK) {
      const int cols = rank_swept(h);
      QS_CUDA(h, qs::launch_basis_prob(h, h->state, h->n, cols, ref_basis, cols / h->batch, o));
      return read_out(h, out, h->batch);
    }
    // rho[x][x]
    double v[2] = {0.0, 0.0};
    if (h->dtype == QS_C128) {
      QS_CUDA(h, cudaMemcpyAsync(v, (const char*)h->state + (ref_basis * N + ref_basis) * 16, 16,
                                 cudaMemcpyDeviceToHost, h->stream));
      QS_CUDA(h, cudaStreamSynchronize(h->stream));
    } else {
      float f[2];
      QS_CUDA(h, cudaMemcpyAsync(f, (const char*)h->state + (ref_basis * N + ref_basis) * 8, 8,
                                 cudaMemcpyDeviceToHost, h->stream));
      QS_CUDA(h, cudaStreamSynchronize(h->stream));
      v[0] = f[0];
    }
    out[0] = v[0];
    return QS_OK;
  }
  void* tmp = nullptr;
  QS_CUDA(h, cudaMallocAsync(&tmp, N * h->esize, h->stream));
  qs_status st = upload_ref(h, ref, tmp);
  if (st != QS_OK) { cudaFreeAsync(tmp, h->stream); return st; }
  st = fidelity_dev(h, tmp, out);
  cudaFreeAsync(tmp, h->stream);
  return st;
}

qs_status qs_set_reference(qs_handle h, const double* ref) {
  if (!h || !ref) return QS_ERR_INVALID_ARG;
  if (!h->ref) QS_CUDA(h, cudaMalloc(&h->ref, (1ull << h->n) * h->esize));
  qs_status st = upload_ref(h, ref, h->ref);
  if (st == QS_OK) h->has_ref = true;
  return st;
}

qs_status qs_set_reference_from(qs_handle h, qs_handle src, int b) {
  if (!h || !src) return QS_ERR_INVALID_ARG;
  { const qs_status st = qs::materialize_basis(src); if (st != QS_OK) return fail(h, st, src->err); }
  if (src->mode != QS_STATEVEC || src->n != h->n || src->dtype != h->dtype || b < 0 || b >= src->batch)
    return fail(h, QS_ERR_INVALID_ARG, "reference must be a member of a STATEVEC handle with the same n and dtype");
  if (!h->ref) QS_CUDA(h, cudaMalloc(&h->ref, (1ull << h->n) * h->esize));
  QS_CUDA(h, cudaStreamSynchronize(src->stream));
  QS_CUDA(h, cudaMemcpyAsync(h->ref, (const char*)src->state + ((size_t)b << h->n) * h->esize,
                             (1ull << h->n) * h->esize, cudaMemcpyDeviceToDevice, h->stream));
  h->has_ref = true;
  return QS_OK;
}

qs_status qs_fidelity_stored(qs_handle h, double* out) {
  if (!h || !out) return QS_ERR_INVALID_ARG;
  { const qs_status st = qs::materialize_basis(h); if (st != QS_OK) return st; }
  if (!h->has_ref) return fail(h, QS_ERR_INVALID_ARG, "no stored reference");
  return fidelity_dev(h, h->ref, out);
}

qs_status qs_fidelity_ref(qs_handle h, qs_handle ref, int first, int count, double* out) {
  if (!h || !ref || !out) return QS_ERR_INVALID_ARG;
  if (h->mode == QS_DENSITY || ref->mode != QS_STATEVEC || ref->n != h->n || ref->dtype != h->dtype)
    return fail(h, QS_ERR_INVALID_ARG, "reference must be a STATEVEC handle with the same n and dtype");
  if (first < 0 || count < 1 || first + count > h->batch) return fail(h, QS_ERR_INVALID_ARG, "member range out of bounds");
  { const qs_status st = qs::materialize_basis(h); if (st != QS_OK) return st; }
  { const qs_status st = qs::materialize_basis(ref); if (st != QS_OK) return fail(h, st, ref->err); }
  QS_CUDA(h, cudaStreamSynchronize(ref->stream));
  // FIXED_RANK: member b's columns, summed (sum_c |<ref|L_{b,c}>|^2)
  const size_t cols = h->mode == QS_FIXED_RANK ? (size_t)h->rank : 1;
  const char* psi = (const char*)h->state + (((size_t)first * cols) << h->n) * h->esize;
  QS_CUDA(h, qs::launch_dot(h, psi, ref->state, h->n, (int)(count * cols), (int)cols, h->small + kSmallOut));
  return read_out(h, out, count);
}

qs_status qs_trace(qs_handle h, double* out) {
  if (!h || !out) return QS_ERR_INVALID_ARG;
  { const qs_status st = qs::materialize_basis(h); if (st != QS_OK) return st; }
  double* o = h->small + kSmallOut;
  if (h->mode == QS_STATEVEC) {
    QS_CUDA(h, qs::launch_norm(h, h->state, h->n, h->batch, 1, o));
    return read_out(h, out, h->batch);
  }
  if (h->mode == QS_FIXED_RANK) {
    const int cols = rank_swept(h);
    QS_CUDA(h, qs::launch_norm(h, h->state, h->n, cols, cols / h->batch, o));
    return read_out(h, out, h->batch);
  }
  QS_CUDA(h, qs::launch_dm_trace(h, h->state, h->n, o));
  return read_out(h, out, 1);
}

qs_status qs_state_size(qs_handle h, size_t* out) {
  if (!h || !out) return QS_ERR_INVALID_ARG;
  *out = h->state_elems;
  return QS_OK;
}

qs_status qs_get_state(qs_handle h, double* host, size_t count) {
  if (!h || !host) return QS_ERR_INVALID_ARG;
  { const qs_status st = qs::materialize_basis(h); if (st != QS_OK) return st; }
  if (count != h->state_elems) return fail(h, QS_ERR_INVALID_ARG, "count must equal qs_state_size");
  QS_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->dtype == QS_C128) {
    QS_CUDA(h, cudaMemcpy(host, h->state, count * 16, cudaMemcpyDeviceToHost));
  } else {
    std::vector<float> f(2 * count);
    QS_CUDA(h, cudaMemcpy(f.data(), h->state, count * 8, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < 2 * count; ++i) host[i] = f[i];
  }
  return QS_OK;
}

qs_status qs_get_state_range(qs_handle h, size_t first, size_t count, double* host) {
  if (!h || (!host && count)) return QS_ERR_INVALID_ARG;
  { const qs_status st = qs::materialize_basis(h); if (st != QS_OK) return st; }
  if (first > h->state_elems || count > h->state_elems - first)
    return fail(h, QS_ERR_INVALID_ARG, "range beyond qs_state_size");
  if (!count) return QS_OK;
  QS_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->dtype == QS_C128) {
    QS_CUDA(h, cudaMemcpy(host, static_cast<const double2*>(h->state) + first, count * 16, cudaMemcpyDeviceToHost));
  } else {
    std::vector<float> f(2 * count);
    QS_CUDA(h, cudaMemcpy(f.data(), static_cast<const float2*>(h->state) + first, count * 8, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < 2 * count; ++i) host[i] = f[i];
  }
  return QS_OK;
}

qs_status qs_set_state(qs_handle h, const double* host, size_t count) {
  if (!h || !host) return QS_ERR_INVALID_ARG;
  if (count != h->state_elems) return fail(h, QS_ERR_INVALID_ARG, "count must equal qs_state_size");
  QS_CUDA(h, cudaStreamSynchronize(h->stream));
  h->pending = 0;
  if (h->mode == QS_FIXED_RANK) {
    bool real = true;
    for (size_t i = 0; i < count && real; ++i) real = host[2 * i + 1] == 0.0;
    h->real_factor = real;
  }
  if (h->mode == QS_DENSITY) {
    // the Hermitian sweeps read only the upper triangle: only for an exactly Hermitian matrix
    const uint64_t N = 1ull << h->n;
    bool herm = true;
    for (uint64_t i = 0; i < N && herm; ++i)
      for (uint64_t j = i; j < N && herm; ++j) {
        const double* a = host + 2 * (i * N + j);
        const double* b = host + 2 * (j * N + i);
        herm = a[0] == b[0] && a[1] == -b[1];
      }
    h->hermitian = herm;
  }
  if (h->dtype == QS_C128) {
    QS_CUDA(h, cudaMemcpy(h->state, host, count * 16, cudaMemcpyHostToDevice));
  } else {
    std::vector<float> f(2 * count);
    for (size_t i = 0; i < 2 * count; ++i) f[i] = (float)host[i];
    QS_CUDA(h, cudaMemcpy(h->state, f.data(), count * 8, cudaMemcpyHostToDevice));
  }
  return QS_OK;
}

qs_status qs_set_rank_columns(qs_handle h, int m) {
  if (!h) return QS_ERR_INVALID_ARG;
  if (h->mode != QS_FIXED_RANK) return fail(h, QS_ERR_NOT_SUPPORTED, "needs FIXED_RANK");
  if (m < 1 || m > h->rank) return fail(h, QS_ERR_INVALID_ARG, "m must be 1..rank");
  std::fill(h->m_cols.begin(), h->m_cols.end(), m);
  return rank_upload_counts(h);
}

qs_status qs_set_member_ranks(qs_handle h, const int* ranks) {
  if (!h || !ranks) return QS_ERR_INVALID_ARG;
  if (h->mode != QS_FIXED_RANK) return fail(h, QS_ERR_NOT_SUPPORTED, "needs FIXED_RANK");
  for (int b = 0; b < h->batch; ++b)
    if (ranks[b] < 1 || ranks[b] > h->rank) return fail(h, QS_ERR_INVALID_ARG, "member ranks must be 1..rank");
  h->m_rank.assign(ranks, ranks + h->batch);
  return rank_upload_counts(h);
}

qs_status qs_get_member_columns(qs_handle h, int* out) {
  if (!h || !out) return QS_ERR_INVALID_ARG;
  if (h->mode != QS_FIXED_RANK) return fail(h, QS_ERR_NOT_SUPPORTED, "needs FIXED_RANK");
  std::copy(h->m_cols.begin(), h->m_cols.end(), out);
  return QS_OK;
}

qs_status qs_set_wait_limit(qs_handle h, int64_t polls) {
  if (!h) return QS_ERR_INVALID_ARG;
  if (polls > 0xffffffffll) return fail(h, QS_ERR_INVALID_ARG, "wait limit above 2^32 - 1 polls");
  h->wait_polls = polls < 0 ? -1 : polls;
  return QS_OK;
}

qs_status qs_set_trajectory_offset(qs_handle h, uint64_t offset) {
  if (!h) return QS_ERR_INVALID_ARG;
  h->traj_offset = offset;
  return QS_OK;
}

qs_status qs_set_member_noise(qs_handle h, const double* e, const uint64_t* seed, const uint64_t* traj,
                              const uint64_t* marked) {
  if (!h) return QS_ERR_INVALID_ARG;
  if (h->mode == QS_DENSITY) return fail(h, QS_ERR_NOT_SUPPORTED, "per-member noise needs STATEVEC or FIXED_RANK");
  if (!e && !seed && !traj && !marked) { h->member_noise = false; h->member_marked = false; return QS_OK; }
  if (!e || !seed || !traj) return fail(h, QS_ERR_INVALID_ARG, "e, seed and traj must all be given");
  double e_max = 0.0;
  for (int b = 0; b < h->batch; ++b) {
    if (!(e[b] >= 0.0) || !std::isfinite(e[b])) return fail(h, QS_ERR_INVALID_ARG, "e must be finite and >= 0");
    e_max = std::max(e_max, e[b]);
  }
  const size_t B = h->batch;
  if (!h->m_e) QS_CUDA(h, cudaMalloc((void**)&h->m_e, B * sizeof(double)));
  if (!h->m_seed) QS_CUDA(h, cudaMalloc((void**)&h->m_seed, B * sizeof(uint64_t)));
  if (!h->m_traj) QS_CUDA(h, cudaMalloc((void**)&h->m_traj, B * sizeof(uint64_t)));
  QS_CUDA(h, cudaMemcpyAsync(h->m_e, e, B * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  QS_CUDA(h, cudaMemcpyAsync(h->m_seed, seed, B * sizeof(uint64_t), cudaMemcpyHostToDevice, h->stream));
  QS_CUDA(h, cudaMemcpyAsync(h->m_traj, traj, B * sizeof(uint64_t), cudaMemcpyHostToDevice, h->stream));
  h->member_noise = true;
  h->m_e_max = e_max;
  if (marked) {
    for (int b = 0; b < h->batch; ++b)
      if (marked[b] >= (1ull << h->n)) return fail(h, QS_ERR_INVALID_ARG, "marked index out of range");
    // FIXED_RANK: one index per column (a member's columns share its index)
    const size_t per = h->mode == QS_FIXED_RANK ? (size_t)h->rank : 1;
    std::vector<uint64_t> cols(B * per);
    for (size_t i = 0; i < cols.size(); ++i) cols[i] = marked[i / per];
    if (!h->m_marked) QS_CUDA(h, cudaMalloc((void**)&h->m_marked, cols.size() * sizeof(uint64_t)));
    QS_CUDA(h, cudaMemcpyAsync(h->m_marked, cols.data(), cols.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, h->stream));
    h->member_marked = true;
  } else {
    h->member_marked = false;
  }
  // the host arrays are consumed by the time the stream reaches the copies
  QS_CUDA(h, cudaStreamSynchronize(h->stream));
  return QS_OK;
}

qs_status qs_measure_peaks(double* fp64_tflops, double* fp32_tflops) {
  if (!fp64_tflops || !fp32_tflops) return QS_ERR_INVALID_ARG;
  return qs::measure_fma_rates(fp64_tflops, fp32_tflops) == cudaSuccess ? QS_OK : QS_ERR_CUDA;
}

qs_status qs_debug_noise(uint64_t seed, uint64_t traj, uint64_t gate_id, int count, uint32_t* words,
                         double* normals) {
  if (count < 1 || !words || !normals) return QS_ERR_INVALID_ARG;
  uint32_t* dw = nullptr;
  double* dn = nullptr;
  if (cudaMalloc((void**)&dw, (size_t)count * 4 * sizeof(uint32_t)) != cudaSuccess) return QS_ERR_OUT_OF_MEMORY;
  if (cudaMalloc((void**)&dn, (size_t)count * 2 * sizeof(double)) != cudaSuccess) { cudaFree(dw); return QS_ERR_OUT_OF_MEMORY; }
  cudaError_t e = qs::launch_debug_noise(seed, traj, gate_id, count, dw, dn, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(words, dw, (size_t)count * 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(normals, dn, (size_t)count * 2 * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(dw);
  cudaFree(dn);
  return e == cudaSuccess ? QS_OK : QS_ERR_CUDA;
}

}  // extern "C"
