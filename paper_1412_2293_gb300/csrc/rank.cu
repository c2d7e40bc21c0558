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

#include <type_traits>

#include "internal.cuh"

namespace qs {

namespace {

constexpr int kExpBlock = 256;
constexpr int kGramRows = 64;            // rows of L' per Gram block
constexpr int kJacobiSweeps = 40;        // bound on the eigensolver's sweeps
constexpr double kTieTol = 1e-10;        // cluster: within 1e-10 * Lambda_1
constexpr double kGsAccept = 1e-3;       // residual norm to accept a projection
constexpr double kGsFallback = 1e-8;
constexpr double kRotTol = 4e-16;        // rotate while |a_pq| > kRotTol * max|a_ii|

__device__ __forceinline__ uint64_t insert0(uint64_t v, int s) {
  return ((v >> s) << (s + 1)) | (v & ((1ull << s) - 1));
}

// Lp[a*m + c] = E_a L[c]; one thread per (group, column).  REAL: L and the
// E_a are real (imaginary parts zero), real arithmetic.
template <typename R, int K_Q, bool REAL>
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
    if constexpr (REAL) {
      R v[D];
#pragma unroll
      for (int l = 0; l < D; ++l) v[l] = L[(uint64_t)c * N + base + tg.off[l]].x;
      for (int a = 0; a < K; ++a) {
        C* out = Lp + (uint64_t)(a * m + c) * N + base;
#pragma unroll
        for (int r = 0; r < D; ++r) {
          R acc = R(0);
#pragma unroll
          for (int q = 0; q < D; ++q) acc = fma(sE[(a * D + r) * D + q].x, v[q], acc);
          out[tg.off[r]] = mk<R>(acc, R(0));
        }
      }
    } else {
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
}

// Gram partials: block b sums rows [b*kGramRows, (b+1)*kGramRows) for every
// (p <= q), one thread per entry of the upper triangle; partial layout
// [block][p][q] complex.  REAL: real arithmetic (imaginary parts are zero).
template <typename R, bool REAL>
__global__ void __launch_bounds__(256) k_gram_partials(const cplx<R>* __restrict__ Lp, int n, int M,
                                                       double* __restrict__ partials) {
  using T = typename std::conditional<REAL, double, double2>::type;
  __shared__ T tile[kMaxGramDim][kGramRows + 1];
  const uint64_t N = 1ull << n;
  const uint64_t r0 = (uint64_t)blockIdx.x * kGramRows;
  for (int i = threadIdx.x; i < M * kGramRows; i += blockDim.x) {
    const int p = i / kGramRows, x = i % kGramRows;
    const uint64_t row = r0 + x;
    const cplx<R> a = row < N ? Lp[(uint64_t)p * N + row] : mk<R>(R(0), R(0));
    if constexpr (REAL) tile[p][x] = a.x;
    else tile[p][x] = make_double2(a.x, a.y);
  }
  __syncthreads();
  double* out = partials + (size_t)blockIdx.x * 2 * M * M;
  const int tri = M * (M + 1) / 2;
  for (int idx = threadIdx.x; idx < tri; idx += blockDim.x) {
    // idx -> (p, q), p <= q, row-major over the upper triangle
    int p = 0, rem = idx;
    while (rem >= M - p) { rem -= M - p; ++p; }
    const int q = p + rem;
    double re = 0.0, im = 0.0;
    if constexpr (REAL) {
      double re2 = 0.0;
      for (int x = 0; x < kGramRows; x += 2) {
        re = fma(tile[p][x], tile[q][x], re);
        re2 = fma(tile[p][x + 1], tile[q][x + 1], re2);
      }
      re += re2;
    } else {
      for (int x = 0; x < kGramRows; ++x) {
        const double2 a = tile[p][x], b = tile[q][x];
        re += a.x * b.x + a.y * b.y;       // conj(a) * b
        im += a.x * b.y - a.y * b.x;
      }
    }
    out[2 * (p * M + q)] = re;
    out[2 * (p * M + q) + 1] = im;
  }
}

// G[p][q] = sum over the partial blocks (fixed-order tree); one block per
// entry, lower triangle by conjugation.
__global__ void __launch_bounds__(256) k_gram_reduce(const double* __restrict__ partials, int blocks, int M, double* G) {
  const int p = blockIdx.x / M, q = blockIdx.x % M;
  if (q < p) return;
  __shared__ double sre[256], sim[256];
  double re = 0.0, im = 0.0;
  for (int b = threadIdx.x; b < blocks; b += blockDim.x) {
    re += partials[(size_t)b * 2 * M * M + 2 * (p * M + q)];
    im += partials[(size_t)b * 2 * M * M + 2 * (p * M + q) + 1];
  }
  sre[threadIdx.x] = re;
  sim[threadIdx.x] = im;
  __syncthreads();
  for (int o = 128; o; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sre[threadIdx.x] += sre[threadIdx.x + o];
      sim[threadIdx.x] += sim[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    G[2 * (p * M + q)] = sre[0];
    G[2 * (p * M + q) + 1] = p == q ? 0.0 : sim[0];
    G[2 * (q * M + p)] = sre[0];
    G[2 * (q * M + p) + 1] = p == q ? 0.0 : -sim[0];
  }
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// Scalar helpers for the real (double) and complex (double2) Jacobi variants.
__device__ __forceinline__ double tmul(double a, double b) { return a * b; }
__device__ __forceinline__ double2 tmul(double2 a, double2 b) { return zmul(a, b); }
__device__ __forceinline__ double tadd(double a, double b) { return a + b; }
__device__ __forceinline__ double2 tadd(double2 a, double2 b) { return zadd(a, b); }
__device__ __forceinline__ double tconj(double a) { return a; }
__device__ __forceinline__ double2 tconj(double2 a) { return zconj(a); }
__device__ __forceinline__ double tre(double a) { return a; }
__device__ __forceinline__ double tre(double2 a) { return a.x; }
__device__ __forceinline__ double tabs2(double a) { return a * a; }
__device__ __forceinline__ double tabs2(double2 a) { return a.x * a.x + a.y * a.y; }
template <typename T> __device__ __forceinline__ T tscal(double v);
template <> __device__ __forceinline__ double tscal<double>(double v) { return v; }
template <> __device__ __forceinline__ double2 tscal<double2>(double v) { return make_double2(v, 0.0); }
__device__ __forceinline__ double tscale(double a, double v) { return a * v; }
__device__ __forceinline__ double2 tscale(double2 a, double v) { return make_double2(a.x * v, a.y * v); }
__device__ __forceinline__ double tphase(double a, double inv) { return a * inv; }                     // sign
__device__ __forceinline__ double2 tphase(double2 a, double inv) { return make_double2(a.x * inv, -a.y * inv); }  // e^{-i arg}
__device__ __forceinline__ double trsqrt(double a) { return rsqrt(a); }


constexpr int kJP = kMaxGramDim + 1;                    // pitch of the Jacobi arrays

// Parallel cyclic Jacobi on the Hermitian (or real symmetric) A (M x M,
// pitch kJP), accumulating V (V <- V R, from any unitary start).  Each step
// applies Mp/2 disjoint rotations from the round-robin schedule: pair 0 =
// (Mp-1, s), pair i = ((s+i) mod (Mp-1), (s-i) mod (Mp-1)).  A rotation
// zeroes a_pq: a phase makes a_pq real, then the classical angle; the tangent
// is found in FP32 (any tangent gives an exactly unitary rotation, the next
// sweep removes what is left), cos and sin from one rsqrt.  The update
// A <- R^dagger A R is done per 2x2 block of the upper triangle and mirrored;
// a step in which no pair rotates skips it.  Sweeps stop when no |a_pq|
// exceeds tol * max|a_ii|.  T is double / double2 (FP64) or float / float2
// (the FP32 pre-pass).  Returns false if the sweep bound was reached.
template <typename T>
__device__ bool jacobi(T* A, T* V, int M, double tol) {
  using RT = decltype(tre(T{}));
  __shared__ T rot[kMaxGramDim / 2][4];
  __shared__ int pp[kMaxGramDim / 2], qq[kMaxGramDim / 2];
  __shared__ RT thr2;
  const int tid = threadIdx.x;
  const int Mp = M + (M & 1);
  const int nb = Mp / 2;
  const int nblk = nb * (nb + 1) / 2;
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    if (tid == 0) {
      RT dmax = 0;
      for (int p = 0; p < M; ++p) dmax = fmax(dmax, fabs(tre(A[p * kJP + p])));
      thr2 = ((RT)tol * dmax) * ((RT)tol * dmax);
    }
    __syncthreads();
    int did = 0;
    for (int st = 0; st < Mp - 1; ++st) {
      int sd = 0;
      if (tid < nb) {
        int p, q;
        if (tid == 0) { p = st; q = Mp - 1; }
        else { p = (st + tid) % (Mp - 1); q = (st - tid + Mp - 1) % (Mp - 1); }
        if (p > q) { const int t = p; p = q; q = t; }
        pp[tid] = p;
        qq[tid] = q;
        T R00 = tscal<T>(1.0), R01 = tscal<T>(0.0), R10 = tscal<T>(0.0), R11 = tscal<T>(1.0);
        if (q < M) {
          const T apq = A[p * kJP + q];
          const RT a2 = tabs2(apq);
          if (a2 > thr2 && a2 > (RT)0) {
            sd = 1;
            const RT inv = trsqrt(a2);
            const T ph = tphase(apq, inv);
            const RT theta = (tre(A[q * kJP + q]) - tre(A[p * kJP + p])) * (RT)0.5 * inv;
            const float th = (float)theta;
            const float tf = copysignf(1.0f, th) / (fabsf(th) + sqrtf(1.0f + th * th));
            const RT t = (RT)tf;
            const RT c = trsqrt((RT)1 + t * t), sn = t * c;
            R00 = tscal<T>(c);
            R01 = tscal<T>(sn);
            R10 = tscale(ph, -sn);
            R11 = tscale(ph, c);
          }
        }
        rot[tid][0] = R00; rot[tid][1] = R01; rot[tid][2] = R10; rot[tid][3] = R11;
      }
      if (!__syncthreads_or(sd)) continue;               // nothing rotates in this step
      did = 1;
      for (int w = tid; w < nblk + M * nb; w += blockDim.x) {
        if (w < nblk) {
          // block (i, j), i <= j: Y = R_i^dagger X R_j
          int i = 0, rem = w;
          while (rem >= nb - i) { rem -= nb - i; ++i; }
          const int j = i + rem;
          const int r0 = pp[i], r1 = qq[i], c0 = pp[j], c1 = qq[j];
          const bool vr1 = r1 < M, vc1 = c1 < M;
          const T z = tscal<T>(0.0);
          const T x00 = A[r0 * kJP + c0];
          const T x01 = vc1 ? A[r0 * kJP + c1] : z;
          const T x10 = vr1 ? A[r1 * kJP + c0] : z;
          const T x11 = (vr1 && vc1) ? A[r1 * kJP + c1] : z;
          const T a00 = rot[j][0], a01 = rot[j][1], a10 = rot[j][2], a11 = rot[j][3];
          const T t00 = tadd(tmul(x00, a00), tmul(x01, a10)), t01 = tadd(tmul(x00, a01), tmul(x01, a11));
          const T t10 = tadd(tmul(x10, a00), tmul(x11, a10)), t11 = tadd(tmul(x10, a01), tmul(x11, a11));
          const T b00 = tconj(rot[i][0]), b01 = tconj(rot[i][2]), b10 = tconj(rot[i][1]), b11 = tconj(rot[i][3]);
          const T y00 = tadd(tmul(b00, t00), tmul(b01, t10)), y01 = tadd(tmul(b00, t01), tmul(b01, t11));
          const T y10 = tadd(tmul(b10, t00), tmul(b11, t10)), y11 = tadd(tmul(b10, t01), tmul(b11, t11));
          A[r0 * kJP + c0] = y00;
          if (vc1) A[r0 * kJP + c1] = y01;
          if (vr1) A[r1 * kJP + c0] = y10;
          if (vr1 && vc1) A[r1 * kJP + c1] = y11;
          if (i != j) {                                  // Hermitian mirror
            A[c0 * kJP + r0] = tconj(y00);
            if (vc1) A[c1 * kJP + r0] = tconj(y01);
            if (vr1) A[c0 * kJP + r1] = tconj(y10);
            if (vr1 && vc1) A[c1 * kJP + r1] = tconj(y11);
          }
        } else {
          // V <- V R for row k and pair j
          const int v = w - nblk;
          const int k = v / nb, j = v % nb;
          const int p = pp[j], q = qq[j];
          if (q < M) {
            const T vp = V[k * kJP + p], vq = V[k * kJP + q];
            V[k * kJP + p] = tadd(tmul(vp, rot[j][0]), tmul(vq, rot[j][2]));
            V[k * kJP + q] = tadd(tmul(vp, rot[j][1]), tmul(vq, rot[j][3]));
          }
        }
      }
      __syncthreads();
    }
    if (!__syncthreads_or(did)) return true;             // no rotation in the whole sweep
  }
  return false;
}

// After the eigensolver: eigenvalues (diagonal of A) sorted descending
// (ties keep index order), clusters of ties given a canonical basis, and the
// outputs W = first keep canonical eigenvectors (M x keep, complex layout),
// lam_out (sorted), keep and the scale.  T is double (real G: real
// eigenvectors, real arithmetic) or double2.  Candidate j of a cluster with
// eigenvectors S is P e_j, P = S S^dagger, minus its components along the
// cluster's accepted vectors q_t; as the q_t lie in range(P),
// <q_t, P e_j> = conj(q_t[j]) and |P e_j - ...|^2 = P_jj - sum_t |q_t[j]|^2,
// so the projections need no dot products.  An accepted vector is
// normalised by its computed norm.  The cluster stage runs in one warp
// (lane = row).
template <typename T>
__device__ void eig_finish(T* A, T* V, int M, int r, int normalize, double* __restrict__ W,
                           double* __restrict__ lam_out, int* keep_out, double* scale_out, int* status) {
  __shared__ int order[kMaxGramDim + 1];
  __shared__ double lam[kMaxGramDim];
  __shared__ int nbasis;
  T* basis = A;                                         // canonical vectors (columns), pitch kJP
  const int tid = threadIdx.x;
  for (int i = tid; i < M; i += blockDim.x) lam[i] = tre(A[i * kJP + i]);
  __syncthreads();
  if (tid == 0) {
    for (int i = 0; i < M; ++i) order[i] = i;
    for (int i = 0; i < M; ++i) {
      int best = i;
      for (int j = i + 1; j < M; ++j)
        if (lam[order[j]] > lam[order[best]]) best = j;
      const int t = order[i]; order[i] = order[best]; order[best] = t;
    }
  }
  __syncthreads();   // A is free from here on (basis aliases it)
  const int keep = r < M ? r : M;
  const double lam1 = lam[order[0]] > 0.0 ? lam[order[0]] : 0.0;
  if (tid < 32) {
    const int lane = tid;
    int found = 0;
    int i0 = 0;
    while (i0 < keep) {
      int i1 = i0 + 1;
      while (i1 < M && lam[order[i0]] - lam[order[i1]] <= kTieTol * lam1) ++i1;
      const int s = i1 - i0;
      const int first = found;
      // P = S S^dagger; GS of P e_j, j = 0..M-1, thresholds kGsAccept then kGsFallback
      for (int pass = 0; pass < 2 && found - first < s; ++pass) {
        const double thr = pass == 0 ? kGsAccept : kGsFallback;
        for (int j = 0; j < M && found - first < s; ++j) {
          T v = tscal<T>(0.0);
          double n2 = 0.0;                               // P_jj, then the residual's norm^2
          for (int c = 0; c < s; ++c) {
            const int col = order[i0 + c];
            const T sj = V[j * kJP + col];
            if (lane < M) v = tadd(v, tmul(V[lane * kJP + col], tconj(sj)));
            n2 += tabs2(sj);
          }
          for (int t = first; t < found; ++t) {
            const T qj = basis[j * kJP + t];
            if (lane < M) v = tadd(v, tscale(tmul(basis[lane * kJP + t], tconj(qj)), -1.0));
            n2 -= tabs2(qj);
          }
          if (n2 > thr * thr) {
            double nv = lane < M ? tabs2(v) : 0.0;
            for (int o = 16; o; o >>= 1) nv += __shfl_xor_sync(0xffffffffu, nv, o);
            if (lane < M) basis[lane * kJP + found] = tscale(v, rsqrt(nv));
            ++found;
            __syncwarp();
          }
        }
      }
      if (found - first < s && lane == 0) status[0] = 2;           // incomplete cluster
      i0 = i1;
    }
    if (lane == 0) nbasis = found;
  }
  __syncthreads();
  // outputs
  for (int i = tid; i < M * keep; i += blockDim.x) {
    const int p = i / keep, c = i % keep;
    const T v = c < nbasis ? basis[p * kJP + c] : tscal<T>(0.0);
    if constexpr (sizeof(T) == 16) {
      W[2 * (p * keep + c)] = v.x;
      W[2 * (p * keep + c) + 1] = v.y;
    } else {
      W[2 * (p * keep + c)] = v;
      W[2 * (p * keep + c) + 1] = 0.0;
    }
  }
  if (tid == 0) {
    double kept = 0.0;
    for (int i = 0; i < M; ++i) lam_out[i] = lam[order[i]];
    for (int i = 0; i < keep; ++i) kept += lam[order[i]];
    keep_out[0] = keep;
    scale_out[0] = normalize ? 1.0 / sqrt(kept) : 1.0;
  }
}

// One block: eigendecomposition of the Hermitian G (M x M) by parallel cyclic
// Jacobi (real arithmetic when G is real), then eig_finish.
__global__ void __launch_bounds__(512) k_eig_truncate(const double* __restrict__ Gin, int M, int r,
                                                      int normalize, double* __restrict__ W,
                                                      double* __restrict__ lam_out, int* keep_out,
                                                      double* scale_out, int* status) {
  __shared__ double2 A[kMaxGramDim][kJP];
  __shared__ double2 V[kMaxGramDim][kJP];
  const int tid = threadIdx.x;
  int cplx = 0;
  for (int i = tid; i < M * M; i += blockDim.x) cplx |= Gin[2 * i + 1] != 0.0;
  cplx = __syncthreads_or(cplx);
  if (cplx) {
    for (int i = tid; i < M * M; i += blockDim.x) {
      const int p = i / M, q = i % M;
      A[p][q] = make_double2(Gin[2 * i], Gin[2 * i + 1]);
      V[p][q] = make_double2(p == q ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    if (!jacobi<double2>(&A[0][0], &V[0][0], M, kRotTol) && tid == 0) status[0] = 1;
    __syncthreads();
    eig_finish<double2>(&A[0][0], &V[0][0], M, r, normalize, W, lam_out, keep_out, scale_out, status);
  } else {
    double* Ar = reinterpret_cast<double*>(&A[0][0]);
    double* Vr = reinterpret_cast<double*>(&V[0][0]);
    for (int i = tid; i < M * M; i += blockDim.x) {
      const int p = i / M, q = i % M;
      Ar[p * kJP + q] = Gin[2 * i];
      Vr[p * kJP + q] = p == q ? 1.0 : 0.0;
    }
    __syncthreads();
    if (!jacobi<double>(Ar, Vr, M, kRotTol) && tid == 0) status[0] = 1;
    __syncthreads();
    eig_finish<double>(Ar, Vr, M, r, normalize, W, lam_out, keep_out, scale_out, status);
  }
}

// L[c] = scale * sum_p Lp[p] W[p][c] for c < keep; one thread per row, all
// kept columns (each element of L' is read once).  REAL: L' and W are real.
template <typename R, bool REAL>
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
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (uint64_t)gridDim.x * blockDim.x) {
    if constexpr (REAL) {
      double acc[kMaxRank];
#pragma unroll
      for (int c = 0; c < kMaxRank; ++c) acc[c] = 0.0;
      for (int p = 0; p < M; ++p) {
        const double a = Lp[(uint64_t)p * N + x].x;
#pragma unroll
        for (int c = 0; c < kMaxRank; ++c)
          if (c < keep) acc[c] = fma(a, sW[p * keep + c].x, acc[c]);
      }
#pragma unroll
      for (int c = 0; c < kMaxRank; ++c)
        if (c < keep) L[(uint64_t)c * N + x] = mk<R>((R)acc[c], R(0));
    } else {
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
}

template <typename R>
cudaError_t expand_dispatch(qs_ctx* h, const void* L, void* Lp, int n, int m, const Targets& tg, bool real,
                            const void* E, int K) {
  const uint64_t work = ((1ull << n) >> tg.k) * (uint64_t)m;
  uint64_t blocks = (work + kExpBlock - 1) / kExpBlock;
  const uint64_t cap = (uint64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  auto* l = static_cast<const cplx<R>*>(L);
  auto* lp = static_cast<cplx<R>*>(Lp);
  const double* e = (const double*)E;
  if (tg.k == 1 && real) k_kraus_expand<R, 1, true><<<(int)blocks, kExpBlock, 0, h->stream>>>(l, lp, n, m, tg, e, K);
  else if (tg.k == 1) k_kraus_expand<R, 1, false><<<(int)blocks, kExpBlock, 0, h->stream>>>(l, lp, n, m, tg, e, K);
  else if (tg.k == 2 && real) k_kraus_expand<R, 2, true><<<(int)blocks, kExpBlock, 0, h->stream>>>(l, lp, n, m, tg, e, K);
  else if (tg.k == 2) k_kraus_expand<R, 2, false><<<(int)blocks, kExpBlock, 0, h->stream>>>(l, lp, n, m, tg, e, K);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_kraus_expand(qs_ctx* h, const void* L, void* Lp, int n, int m, const Targets& tg, bool real,
                                const void* E, int K) {
  if (h->dtype == QS_C64) return expand_dispatch<float>(h, L, Lp, n, m, tg, real, E, K);
  return expand_dispatch<double>(h, L, Lp, n, m, tg, real, E, K);
}

cudaError_t launch_gram(qs_ctx* h, const void* Lp, int n, int M, bool real, double* G) {
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
  if (h->dtype == QS_C64 && real)
    k_gram_partials<float, true><<<blocks, 256, 0, h->stream>>>((const float2*)Lp, n, M, h->partials);
  else if (h->dtype == QS_C64)
    k_gram_partials<float, false><<<blocks, 256, 0, h->stream>>>((const float2*)Lp, n, M, h->partials);
  else if (real)
    k_gram_partials<double, true><<<blocks, 256, 0, h->stream>>>((const double2*)Lp, n, M, h->partials);
  else
    k_gram_partials<double, false><<<blocks, 256, 0, h->stream>>>((const double2*)Lp, n, M, h->partials);
  k_gram_reduce<<<M * M, 256, 0, h->stream>>>(h->partials, blocks, M, G);
  return cudaGetLastError();
}

cudaError_t launch_eig_truncate(qs_ctx* h, const double* G, int M, int r, int normalize, double* W,
                                double* lam, double* scale, int* keep, int* status) {
  k_eig_truncate<<<1, 512, 0, h->stream>>>(G, M, r, normalize, W, lam, keep, scale, status);
  return cudaGetLastError();
}

cudaError_t launch_project(qs_ctx* h, const void* Lp, void* L, int n, int M, bool real, const double* W,
                           const double* scale, const int* keep) {
  const uint64_t N = 1ull << n;
  uint64_t blocks = (N + 255) / 256;
  const uint64_t cap = (uint64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  if (h->dtype == QS_C64 && real)
    k_project<float, true><<<(int)blocks, 256, 0, h->stream>>>((const float2*)Lp, (float2*)L, n, M, W, keep, scale);
  else if (h->dtype == QS_C64)
    k_project<float, false><<<(int)blocks, 256, 0, h->stream>>>((const float2*)Lp, (float2*)L, n, M, W, keep, scale);
  else if (real)
    k_project<double, true><<<(int)blocks, 256, 0, h->stream>>>((const double2*)Lp, (double2*)L, n, M, W, keep, scale);
  else
    k_project<double, false><<<(int)blocks, 256, 0, h->stream>>>((const double2*)Lp, (double2*)L, n, M, W, keep, scale);
  return cudaGetLastError();
}

}  // namespace qs
