// Fixed-rank approximation of the density matrix (Sec. 3.2).
//
// rho = L L^dagger with L a 2^n x m factor stored column-major (column c is a
// state vector at offset c * 2^n).  A channel with Kraus operators E_1..E_K
// (Eq. 3) produces L' = [E_1 L | ... | E_K L] (M = K m columns); the best
// rank-r approximation of L' L'^dagger is L' W_r, where W_r holds the r
// leading eigenvectors of the M x M Gram matrix G = L'^dagger L'.
//
// Kernels: Kraus expansion (L -> L'), Gram matrix in FP64 (block partials
// plus a fixed-order sum), a one-block parallel cyclic Jacobi eigensolver in
// FP64 with the canonical basis rule for tied eigenvalues, and the
// projection L <- scale * L' W_r.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace qs {

namespace {

constexpr int kExpBlock = 256;
constexpr int kGramRows = 64;            // rows of L' per Gram block
constexpr int kJacobiSweeps = 40;        // bound on the eigensolver's sweeps
constexpr double kTieTol = 1e-10;        // cluster: within 1e-10 * Lambda_1
constexpr double kGsAccept = 1e-3;       // residual norm to accept a projection
constexpr double kGsFallback = 1e-8;

__device__ __forceinline__ uint64_t insert0(uint64_t v, int s) {
  return ((v >> s) << (s + 1)) | (v & ((1ull << s) - 1));
}

// Lp[a*m + c] = E_a L[c]; one thread per (group, column).
template <typename R, int K_Q>
__global__ void __launch_bounds__(kExpBlock) k_kraus_expand(const cplx<R>* __restrict__ L,
                                                            cplx<R>* __restrict__ Lp, int n, int m,
                                                            Targets tg, const double* __restrict__ E,
                                                            int K) {
  using C = cplx<R>;
  constexpr int D = 1 << K_Q;
  __shared__ C sE[8 * D * D];
  for (int i = threadIdx.x; i < K * D * D; i += blockDim.x) sE[i] = mk<R>((R)E[2 * i], (R)E[2 * i + 1]);
  __syncthreads();
  const uint64_t N = 1ull << n;
  const uint64_t groups = N >> K_Q;
  const uint64_t total = groups * (uint64_t)m;
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total;
       w += (uint64_t)gridDim.x * blockDim.x) {
    const int c = (int)(w / groups);
    const uint64_t g = w - (uint64_t)c * groups;
    uint64_t base = g;
#pragma unroll
    for (int j = 0; j < K_Q; ++j) base = insert0(base, tg.sorted[j]);
    C v[D];
#pragma unroll
    for (int l = 0; l < D; ++l) v[l] = L[(uint64_t)c * N + base + tg.off[l]];
    for (int a = 0; a < K; ++a) {
      C* out = Lp + (uint64_t)(a * m + c) * N + base;
#pragma unroll
      for (int r = 0; r < D; ++r) {
        C acc = mk<R>(R(0), R(0));
#pragma unroll
        for (int q = 0; q < D; ++q) acc = cfma(sE[(a * D + r) * D + q], v[q], acc);
        out[tg.off[r]] = acc;
      }
    }
  }
}

// Gram partials: block b sums rows [b*kGramRows, (b+1)*kGramRows) for every
// (p <= q); partial layout [block][p][q] complex.
template <typename R>
__global__ void __launch_bounds__(256) k_gram_partials(const cplx<R>* __restrict__ Lp, int n, int M,
                                                       double* __restrict__ partials) {
  __shared__ double2 tile[kMaxGramDim][kGramRows + 1];
  const uint64_t N = 1ull << n;
  const uint64_t r0 = (uint64_t)blockIdx.x * kGramRows;
  for (int i = threadIdx.x; i < M * kGramRows; i += blockDim.x) {
    const int p = i / kGramRows, x = i % kGramRows;
    const uint64_t row = r0 + x;
    double2 v = make_double2(0.0, 0.0);
    if (row < N) { const cplx<R> a = Lp[(uint64_t)p * N + row]; v = make_double2(a.x, a.y); }
    tile[p][x] = v;
  }
  __syncthreads();
  const int pairs = M * M;
  double* out = partials + (size_t)blockIdx.x * 2 * M * M;
  for (int idx = threadIdx.x; idx < pairs; idx += blockDim.x) {
    const int p = idx / M, q = idx % M;
    if (q < p) continue;
    double re = 0.0, im = 0.0;
    for (int x = 0; x < kGramRows; ++x) {
      const double2 a = tile[p][x], b = tile[q][x];
      re += a.x * b.x + a.y * b.y;       // conj(a) * b
      im += a.x * b.y - a.y * b.x;
    }
    out[2 * (p * M + q)] = re;
    out[2 * (p * M + q) + 1] = im;
  }
}

// G[p][q] = sum over blocks (fixed order); lower triangle by conjugation.
__global__ void k_gram_reduce(const double* __restrict__ partials, int blocks, int M, double* G) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * M) return;
  const int p = idx / M, q = idx % M;
  if (q < p) return;
  double re = 0.0, im = 0.0;
  for (int b = 0; b < blocks; ++b) {
    re += partials[(size_t)b * 2 * M * M + 2 * (p * M + q)];
    im += partials[(size_t)b * 2 * M * M + 2 * (p * M + q) + 1];
  }
  G[2 * (p * M + q)] = re;
  G[2 * (p * M + q) + 1] = im;
  G[2 * (q * M + p)] = re;
  G[2 * (q * M + p) + 1] = p == q ? 0.0 : -im;
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 zscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// One block: eigendecomposition of the Hermitian G (M x M) by parallel cyclic
// Jacobi (round-robin pairing, M/2 disjoint rotations per step), eigenvalues
// sorted descending, clusters of ties given a canonical basis, then
// W = first r canonical eigenvectors (M x keep), keep = min(r, M), and
// lam[0..M) sorted descending; out_scale = 1/sqrt(sum lam[:keep]) or 1.
__global__ void __launch_bounds__(512) k_eig_truncate(const double* __restrict__ Gin, int M, int r,
                                                      int normalize, double* __restrict__ W,
                                                      double* __restrict__ lam_out, int* keep_out,
                                                      double* scale_out, int* status) {
  __shared__ double2 A[kMaxGramDim][kMaxGramDim + 1];
  __shared__ double2 V[kMaxGramDim][kMaxGramDim + 1];
  __shared__ double2 rot[kMaxGramDim / 2][4];          // R[p][p], R[p][q], R[q][p], R[q][q]
  __shared__ int pp[kMaxGramDim / 2], qq[kMaxGramDim / 2];
  __shared__ int order[kMaxGramDim + 1];
  __shared__ double lam[kMaxGramDim];
  __shared__ double off_norm, tot_norm;
  // canonical vectors (columns) reuse A's storage once the eigenvalues are read
  auto& basis = A;
  __shared__ double2 vtmp[kMaxGramDim];
  __shared__ double vnorm;
  __shared__ int nbasis;

  const int tid = threadIdx.x;
  const int Mp = M + (M & 1);                           // even number of players
  for (int i = tid; i < M * M; i += blockDim.x) {
    const int p = i / M, q = i % M;
    A[p][q] = make_double2(Gin[2 * i], Gin[2 * i + 1]);
    V[p][q] = make_double2(p == q ? 1.0 : 0.0, 0.0);
  }
  if (tid == 0) {
    for (int i = 0; i < Mp; ++i) order[i] = i;
  }
  __syncthreads();

  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    if (tid == 0) {
      double off = 0.0, tot = 0.0;
      for (int p = 0; p < M; ++p)
        for (int q = 0; q < M; ++q) {
          const double v = A[p][q].x * A[p][q].x + A[p][q].y * A[p][q].y;
          tot += v;
          if (p != q) off += v;
        }
      off_norm = off;
      tot_norm = tot;
    }
    __syncthreads();
    if (off_norm <= 1e-32 * tot_norm || off_norm == 0.0) break;
    for (int step = 0; step < Mp - 1; ++step) {
      // pairs of this step from the round-robin arrangement
      if (tid < Mp / 2) {
        int p = order[tid], q = order[Mp - 1 - tid];
        if (p > q) { const int t = p; p = q; q = t; }
        pp[tid] = p;
        qq[tid] = q;
        double2 R00 = make_double2(1.0, 0.0), R01 = make_double2(0.0, 0.0);
        double2 R10 = make_double2(0.0, 0.0), R11 = make_double2(1.0, 0.0);
        if (q < M) {
          const double2 apq = A[p][q];
          const double mag = sqrt(apq.x * apq.x + apq.y * apq.y);
          const double app = A[p][p].x, aqq = A[q][q].x;
          if (mag > 1e-300) {
            // phase e^{-i phi} on q makes the (p, q) entry real, then a real rotation
            const double2 ph = make_double2(apq.x / mag, -apq.y / mag);    // e^{-i phi}
            const double theta = (aqq - app) / (2.0 * mag);
            const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
            const double c = 1.0 / sqrt(1.0 + t * t), s = t * c;
            R00 = make_double2(c, 0.0);
            R01 = make_double2(s, 0.0);
            R10 = zscale(ph, -s);
            R11 = zscale(ph, c);
          }
        }
        rot[tid][0] = R00; rot[tid][1] = R01; rot[tid][2] = R10; rot[tid][3] = R11;
      }
      __syncthreads();
      const int npairs = Mp / 2;
      // A <- A R (columns p, q), V <- V R
      for (int i = tid; i < npairs * M; i += blockDim.x) {
        const int j = i / M, k = i % M;
        const int p = pp[j], q = qq[j];
        if (q >= M) continue;
        const double2 R00 = rot[j][0], R01 = rot[j][1], R10 = rot[j][2], R11 = rot[j][3];
        const double2 akp = A[k][p], akq = A[k][q];
        A[k][p] = zadd(zmul(akp, R00), zmul(akq, R10));
        A[k][q] = zadd(zmul(akp, R01), zmul(akq, R11));
        const double2 vkp = V[k][p], vkq = V[k][q];
        V[k][p] = zadd(zmul(vkp, R00), zmul(vkq, R10));
        V[k][q] = zadd(zmul(vkp, R01), zmul(vkq, R11));
      }
      __syncthreads();
      // A <- R^dagger A (rows p, q)
      for (int i = tid; i < npairs * M; i += blockDim.x) {
        const int j = i / M, k = i % M;
        const int p = pp[j], q = qq[j];
        if (q >= M) continue;
        const double2 R00 = rot[j][0], R01 = rot[j][1], R10 = rot[j][2], R11 = rot[j][3];
        const double2 apk = A[p][k], aqk = A[q][k];
        A[p][k] = zadd(zmul(zconj(R00), apk), zmul(zconj(R10), aqk));
        A[q][k] = zadd(zmul(zconj(R01), apk), zmul(zconj(R11), aqk));
      }
      __syncthreads();
      if (tid == 0) {                                   // rotate all but order[0]
        const int last = order[Mp - 1];
        for (int i = Mp - 1; i > 1; --i) order[i] = order[i - 1];
        order[1] = last;
      }
      __syncthreads();
    }
    if (sweep == kJacobiSweeps - 1 && tid == 0) status[0] = 1;   // not converged
  }

  // sort eigenvalues descending (selection sort, ties keep index order)
  if (tid == 0) {
    for (int i = 0; i < M; ++i) { order[i] = i; lam[i] = A[i][i].x; }
    for (int i = 0; i < M; ++i) {
      int best = i;
      for (int j = i + 1; j < M; ++j)
        if (lam[order[j]] > lam[order[best]]) best = j;
      const int t = order[i]; order[i] = order[best]; order[best] = t;
    }
    nbasis = 0;
  }
  __syncthreads();   // A is free from here on (basis aliases it)
  const int keep = r < M ? r : M;
  const double lam1 = lam[order[0]] > 0.0 ? lam[order[0]] : 0.0;

  // clusters (anchor = first member) and their canonical bases, until keep
  int i0 = 0;
  while (i0 < keep) {
    int i1 = i0 + 1;
    while (i1 < M && lam[order[i0]] - lam[order[i1]] <= kTieTol * lam1) ++i1;
    const int s = i1 - i0;
    const int first = nbasis;
    // P = S S^dagger; GS of P e_j, j = 0..M-1, thresholds kGsAccept then kGsFallback
    for (int pass = 0; pass < 2 && nbasis - first < s; ++pass) {
      const double thr = pass == 0 ? kGsAccept : kGsFallback;
      for (int j = 0; j < M && nbasis - first < s; ++j) {
        // v = P e_j = sum_c S[:, c] conj(S[j, c])
        for (int k = tid; k < M; k += blockDim.x) {
          double2 acc = make_double2(0.0, 0.0);
          for (int c = 0; c < s; ++c) {
            const int col = order[i0 + c];
            acc = zadd(acc, zmul(V[k][col], zconj(V[j][col])));
          }
          vtmp[k] = acc;
        }
        __syncthreads();
        for (int rep = 0; rep < 2; ++rep) {
          for (int u = first; u < nbasis; ++u) {
            // v -= basis_u * <basis_u, v>
            if (tid == 0) {
              double2 d = make_double2(0.0, 0.0);
              for (int k = 0; k < M; ++k) d = zadd(d, zmul(zconj(basis[k][u]), vtmp[k]));
              rot[0][0] = d;
            }
            __syncthreads();
            const double2 d = rot[0][0];
            for (int k = tid; k < M; k += blockDim.x) vtmp[k] = zsub(vtmp[k], zmul(basis[k][u], d));
            __syncthreads();
          }
        }
        if (tid == 0) {
          double nv = 0.0;
          for (int k = 0; k < M; ++k) nv += vtmp[k].x * vtmp[k].x + vtmp[k].y * vtmp[k].y;
          vnorm = sqrt(nv);
        }
        __syncthreads();
        if (vnorm > thr) {
          const double inv = 1.0 / vnorm;
          for (int k = tid; k < M; k += blockDim.x) basis[k][nbasis] = zscale(vtmp[k], inv);
          __syncthreads();
          if (tid == 0) nbasis = nbasis + 1;
        }
        __syncthreads();
      }
    }
    if (nbasis - first < s && tid == 0) status[0] = 2;           // incomplete cluster
    __syncthreads();
    i0 = i1;
  }

  // outputs
  for (int i = tid; i < M * keep; i += blockDim.x) {
    const int p = i / keep, c = i % keep;
    const double2 v = c < nbasis ? basis[p][c] : make_double2(0.0, 0.0);
    W[2 * (p * keep + c)] = v.x;
    W[2 * (p * keep + c) + 1] = v.y;
  }
  if (tid == 0) {
    double kept = 0.0;
    for (int i = 0; i < M; ++i) lam_out[i] = lam[order[i]];
    for (int i = 0; i < keep; ++i) kept += lam[order[i]];
    keep_out[0] = keep;
    scale_out[0] = normalize ? 1.0 / sqrt(kept) : 1.0;
  }
}

// L[c'] = scale * sum_p Lp[p] W[p][c'] for c' < keep; one thread per row.
template <typename R>
__global__ void __launch_bounds__(256) k_project(const cplx<R>* __restrict__ Lp, cplx<R>* __restrict__ L,
                                                 int n, int M, const double* __restrict__ W,
                                                 const int* __restrict__ keep_p,
                                                 const double* __restrict__ scale_p) {
  __shared__ double2 sW[kMaxGramDim * kMaxRank];
  const int keep = keep_p[0];
  const double scale = scale_p[0];
  for (int i = threadIdx.x; i < M * keep; i += blockDim.x)
    sW[i] = make_double2(W[2 * i] * scale, W[2 * i + 1] * scale);
  __syncthreads();
  const uint64_t N = 1ull << n;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N;
       x += (uint64_t)gridDim.x * blockDim.x) {
    double2 acc[kMaxRank];
#pragma unroll
    for (int c = 0; c < kMaxRank; ++c) acc[c] = make_double2(0.0, 0.0);
    for (int p = 0; p < M; ++p) {
      const cplx<R> a = Lp[(uint64_t)p * N + x];
      const double2 ad = make_double2(a.x, a.y);
#pragma unroll
      for (int c = 0; c < kMaxRank; ++c)
        if (c < keep) acc[c] = zadd(acc[c], zmul(ad, sW[p * keep + c]));
    }
#pragma unroll
    for (int c = 0; c < kMaxRank; ++c)
      if (c < keep) L[(uint64_t)c * N + x] = mk<R>((R)acc[c].x, (R)acc[c].y);
  }
}

template <typename R>
cudaError_t expand_dispatch(qs_ctx* h, const void* L, void* Lp, int n, int m, const Targets& tg,
                            const void* E, int K) {
  const uint64_t work = ((1ull << n) >> tg.k) * (uint64_t)m;
  uint64_t blocks = (work + kExpBlock - 1) / kExpBlock;
  const uint64_t cap = (uint64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  auto* l = static_cast<const cplx<R>*>(L);
  auto* lp = static_cast<cplx<R>*>(Lp);
  if (tg.k == 1)
    k_kraus_expand<R, 1><<<(int)blocks, kExpBlock, 0, h->stream>>>(l, lp, n, m, tg, (const double*)E, K);
  else if (tg.k == 2)
    k_kraus_expand<R, 2><<<(int)blocks, kExpBlock, 0, h->stream>>>(l, lp, n, m, tg, (const double*)E, K);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_kraus_expand(qs_ctx* h, const void* L, void* Lp, int n, int m, const Targets& tg,
                                const void* E, int K) {
  if (h->dtype == QS_C64) return expand_dispatch<float>(h, L, Lp, n, m, tg, E, K);
  return expand_dispatch<double>(h, L, Lp, n, m, tg, E, K);
}

cudaError_t launch_gram(qs_ctx* h, const void* Lp, int n, int M, double* G) {
  const uint64_t N = 1ull << n;
  const int blocks = (int)((N + kGramRows - 1) / kGramRows);
  const size_t need = (size_t)blocks * 2 * M * M;
  if (h->partials_cap < need) {
    if (h->partials) cudaFreeAsync(h->partials, h->stream);
    h->partials = nullptr;
    h->partials_cap = 0;
    if (cudaMallocAsync((void**)&h->partials, need * sizeof(double), h->stream) != cudaSuccess)
      return cudaErrorMemoryAllocation;
    h->partials_cap = need;
  }
  if (h->dtype == QS_C64)
    k_gram_partials<float><<<blocks, 256, 0, h->stream>>>((const float2*)Lp, n, M, h->partials);
  else
    k_gram_partials<double><<<blocks, 256, 0, h->stream>>>((const double2*)Lp, n, M, h->partials);
  k_gram_reduce<<<(M * M + 255) / 256, 256, 0, h->stream>>>(h->partials, blocks, M, G);
  return cudaGetLastError();
}

cudaError_t launch_eig_truncate(qs_ctx* h, const double* G, int M, int r, int normalize, double* W,
                                double* lam, double* scale, int* keep, int* status) {
  k_eig_truncate<<<1, 512, 0, h->stream>>>(G, M, r, normalize, W, lam, keep, scale, status);
  return cudaGetLastError();
}

cudaError_t launch_project(qs_ctx* h, const void* Lp, void* L, int n, int M, const double* W,
                           const double* scale, const int* keep) {
  const uint64_t N = 1ull << n;
  uint64_t blocks = (N + 255) / 256;
  const uint64_t cap = (uint64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  if (h->dtype == QS_C64)
    k_project<float><<<(int)blocks, 256, 0, h->stream>>>((const float2*)Lp, (float2*)L, n, M, W, keep, scale);
  else
    k_project<double><<<(int)blocks, 256, 0, h->stream>>>((const double2*)Lp, (double2*)L, n, M, W, keep, scale);
  return cudaGetLastError();
}

}  // namespace qs
