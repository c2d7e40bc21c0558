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

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "internal.cuh"

namespace qs {

namespace {

constexpr int kExpBlock = 256;
constexpr int kGramRows = 64;            // rows of L' per shared-memory tile of the Gram kernel
constexpr int kGramTarget = 512;         // about this many row blocks per member (fixed by n)
constexpr int kTriMax = kMaxGramDim * (kMaxGramDim + 1) / 2;
constexpr int kJacobiSweeps = 40;        // bound on the eigensolver's sweeps
constexpr double kTieTol = 1e-10;        // cluster: within 1e-10 * Lambda_1
constexpr double kGsAccept = 1e-3;       // residual norm to accept a projection
constexpr double kGsFallback = 1e-8;
constexpr double kRotTol = 4e-16;        // rotate while |a_pq| > kRotTol * max|a_ii|
constexpr int kJacobiSweeps32 = 12;      // bound on the FP32 pre-pass
constexpr double kRotTol32 = 1e-6;       // FP32 pre-pass: rotate while |a_pq| > this * max|a_ii|

__device__ __forceinline__ uint64_t insert0(uint64_t v, int s) {
  return ((v >> s) << (s + 1)) | (v & ((1ull << s) - 1));
}

// Lp_b[a m_b + c] = E_a L_b[c] for member b = blockIdx.y; one thread per
// (group, column).  The member's Kraus operators are E + b e_stride (e_stride
// = 0: one set for every member).  Block (0, b) records M_b = K m_b.  REAL: L
// and the E_a are real (imaginary parts zero), real arithmetic.
// Entry (row, col) of operator `op` of the xi-averaged Kraus set of a noisy
// gate U (Eqs. 5-6 and 8-9) at noise level e: rotation noise -> U N with N
// the tensor product over the targets (target 0 the low local bit) of
// sqrt(l1) I or sqrt(l2) J, J = [[0, 1], [-1, 0]], l1,2 = (1 +- e^{-2e^2})/2;
// phase noise -> U diag(1, .., 1, sqrt P) and U diag(0, .., 0, sqrt(1 - P)),
// P = e^{-e^2}.
__device__ double2 kraus_entry(const KrausGate& g, double e, int op, int row, int col) {
  const int D = 1 << g.k;
  double nre[4];                                         // column `col` of N (real)
  if (g.noise == QS_NOISE_ROTATION) {
    const double q = exp(-2.0 * e * e);
    const double s1 = sqrt(0.5 * (1.0 + q)), s2 = sqrt(0.5 * (1.0 - q));
    for (int x = 0; x < D; ++x) {
      double v = 1.0;
      for (int j = 0; j < g.k; ++j) {
        const int w = (op >> j) & 1, rb = (x >> j) & 1, cb = (col >> j) & 1;
        v *= w == 0 ? (rb == cb ? s1 : 0.0) : (rb == 0 && cb == 1 ? s2 : (rb == 1 && cb == 0 ? -s2 : 0.0));
      }
      nre[x] = v;
    }
  } else {
    const double P = exp(-e * e);
    for (int x = 0; x < D; ++x) nre[x] = 0.0;
    if (op == 0) nre[col] = col == D - 1 ? sqrt(P) : 1.0;
    else if (col == D - 1) nre[col] = sqrt(1.0 - P);
  }
  double re = 0.0, im = 0.0;                             // (U N)[row][col]
  for (int x = 0; x < D; ++x) {
    re += g.U[2 * (row * D + x)] * nre[x];
    im += g.U[2 * (row * D + x) + 1] * nre[x];
  }
  return make_double2(re, im);
}

template <typename R, int K_Q, bool REAL, bool DIAG = false>
__global__ void __launch_bounds__(kExpBlock) k_kraus_expand(const cplx<R>* __restrict__ L,
                                                            cplx<R>* __restrict__ Lp, int n, int rcap, int mcap,
                                                            Targets tg, const double* __restrict__ E, int K,
                                                            int e_stride, RankCounts rc, const KrausGate g) {
  using C = cplx<R>;
  constexpr int D = 1 << K_Q;
  __shared__ C sE[8 * D * D];
  const int b = blockIdx.y;
  if (g.k > 0) {
    // the member's averaged Kraus set, built here from its noise level
    const double e = g.e_member ? g.e_member[b] : (g.e_run ? *g.e_run : g.e_value);
    for (int i = threadIdx.x; i < K * D * D; i += blockDim.x) {
      const double2 v = kraus_entry(g, e, i / (D * D), (i / D) % D, i % D);
      sE[i] = mk<R>((R)v.x, (R)v.y);
    }
  } else {
    const double* Eb = E + (size_t)b * e_stride;
    for (int i = threadIdx.x; i < K * D * D; i += blockDim.x) sE[i] = mk<R>((R)Eb[2 * i], (R)Eb[2 * i + 1]);
  }
  const int m = rc.cols[b];
  if (blockIdx.x == 0 && threadIdx.x == 0) rc.M[b] = K * m;
  __syncthreads();
  const uint64_t N = 1ull << n;
  const uint64_t groups = N >> K_Q;
  const uint64_t total = groups * (uint64_t)m;
  const C* Lb = L + (uint64_t)b * rcap * N;
  C* Lpb = Lp + (uint64_t)b * mcap * N;
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
      for (int l = 0; l < D; ++l) v[l] = Lb[(uint64_t)c * N + base + tg.off[l]].x;
      for (int a = 0; a < K; ++a) {
        C* out = Lpb + (uint64_t)(a * m + c) * N + base;
#pragma unroll
        for (int r = 0; r < D; ++r) {
          R acc = R(0);
          if constexpr (DIAG) {
            acc = sE[(a * D + r) * D + r].x * v[r];
          } else {
#pragma unroll
            for (int q = 0; q < D; ++q) acc = fma(sE[(a * D + r) * D + q].x, v[q], acc);
          }
          out[tg.off[r]] = mk<R>(acc, R(0));
        }
      }
    } else {
      C v[D];
#pragma unroll
      for (int l = 0; l < D; ++l) v[l] = Lb[(uint64_t)c * N + base + tg.off[l]];
      for (int a = 0; a < K; ++a) {
        C* out = Lpb + (uint64_t)(a * m + c) * N + base;
#pragma unroll
        for (int r = 0; r < D; ++r) {
          C acc = mk<R>(R(0), R(0));
          if constexpr (DIAG) {
            acc = cmul(sE[(a * D + r) * D + r], v[r]);
          } else {
#pragma unroll
            for (int q = 0; q < D; ++q) acc = cfma(sE[(a * D + r) * D + q], v[q], acc);
          }
          out[tg.off[r]] = acc;
        }
      }
    }
  }
}

// (p, q), p <= q, of entry idx of the upper triangle of an M x M matrix,
// row-major
__device__ __forceinline__ void tri_pq(int idx, int M, int* p, int* q) {
  int pp = 0, rem = idx;
  while (rem >= M - pp) { rem -= M - pp; ++pp; }
  *p = pp;
  *q = pp + rem;
}

// Gram partials of member b = blockIdx.y: block x sums rows
// [x rows_per_block, (x + 1) rows_per_block) of L'_b, in tiles of kGramRows
// rows through shared memory, for every entry (p <= q) of the upper triangle
// (each entry a fixed-order FP64 sum).  Blocks of 16 tiles of rows or more
// (n >= 19) run kGramThreads threads, smaller ones half as many (their
// channels are latency-bound, and fewer warps meet at each barrier).  A thread
// owns entries idx, idx + blockDim, ...; when the block is large and the
// triangle has at most blockDim / 2 entries (M <= 21 at 512 threads) its rows
// are split instead among G = min(blockDim / tri, kGramRows) groups of
// threads (group g takes the tile rows x = g mod G), so nearly every thread
// works and the FP64 units of all four schedulers are busy, and the groups'
// sums are added in group order at the end.  Partial layout
// [member][block][kTriMax] complex.  The row split and the block size depend
// only on n, so a member's result does not depend on the batch.
constexpr int kGramThreads = 512;

template <typename R, bool REAL>
__global__ void __launch_bounds__(kGramThreads) k_gram_partials(const cplx<R>* __restrict__ Lp, int n, int mcap,
                                                                int rows_per_block, RankCounts rc,
                                                                double* __restrict__ partials) {
  using T = typename std::conditional<REAL, double, double2>::type;
  // threads: kGramThreads where rows are split (blocks of 16 tiles or more), else half
  constexpr int kOwn = (kTriMax + kGramThreads / 2 - 1) / (kGramThreads / 2);
  const int nt = (int)blockDim.x;
  __shared__ T tile[kMaxGramDim][kGramRows + 1];
  __shared__ double2 gsum[kGramThreads];
  const int b = blockIdx.y;
  const int M = rc.M[b];
  const int tri = M * (M + 1) / 2;
  // row groups per entry (at most one per row of a tile); only where a block
  // has rows enough to keep them busy (from n = 19 on), the small factors'
  // channels being latency-bound
  const int G = tri <= nt / 2 && rows_per_block >= 16 * kGramRows ? min(nt / tri, kGramRows) : 1;
  const int g = G > 1 ? (int)threadIdx.x / tri : 0;    // this thread's group (G: idle)
  const uint64_t N = 1ull << n;
  const cplx<R>* Lpb = Lp + (uint64_t)b * mcap * N;
  int ep[kOwn], eq[kOwn];
  double re[kOwn], im[kOwn], re2[kOwn];
#pragma unroll
  for (int j = 0; j < kOwn; ++j) {
    const int idx = G > 1 ? (j == 0 ? (int)threadIdx.x % tri : tri) : (int)threadIdx.x + nt * j;
    ep[j] = eq[j] = 0;
    if (idx < tri && g < G) tri_pq(idx, M, &ep[j], &eq[j]);
    re[j] = im[j] = re2[j] = 0.0;
  }
  const uint64_t r0 = (uint64_t)blockIdx.x * rows_per_block;
  for (int s = 0; s < rows_per_block; s += kGramRows) {
    __syncthreads();
    for (int i = threadIdx.x; i < M * kGramRows; i += blockDim.x) {
      const int p = i / kGramRows, x = i % kGramRows;
      const uint64_t row = r0 + s + x;
      const cplx<R> a = row < N ? Lpb[(uint64_t)p * N + row] : mk<R>(R(0), R(0));
      if constexpr (REAL) tile[p][x] = a.x;
      else tile[p][x] = make_double2(a.x, a.y);
    }
    __syncthreads();
    if (G > 1) {
      if (g >= G) continue;
      const int p = ep[0], q = eq[0];
      if constexpr (REAL) {
        int k = 0;
        for (int x = g; x < kGramRows; x += G, ++k) {
          if (k & 1) re2[0] = fma(tile[p][x], tile[q][x], re2[0]);
          else re[0] = fma(tile[p][x], tile[q][x], re[0]);
        }
      } else {
        for (int x = g; x < kGramRows; x += G) {
          const double2 a = tile[p][x], c = tile[q][x];
          re[0] = fma(a.x, c.x, fma(a.y, c.y, re[0]));   // conj(a) * c, four FMAs
          im[0] = fma(a.x, c.y, fma(-a.y, c.x, im[0]));
        }
      }
      continue;
    }
#pragma unroll
    for (int j = 0; j < kOwn; ++j) {
      if ((int)threadIdx.x + nt * j >= tri) continue;
      const int p = ep[j], q = eq[j];
      if constexpr (REAL) {
        for (int x = 0; x < kGramRows; x += 2) {
          re[j] = fma(tile[p][x], tile[q][x], re[j]);
          re2[j] = fma(tile[p][x + 1], tile[q][x + 1], re2[j]);
        }
      } else {
        for (int x = 0; x < kGramRows; ++x) {
          const double2 a = tile[p][x], c = tile[q][x];
          re[j] = fma(a.x, c.x, fma(a.y, c.y, re[j]));   // conj(a) * c, four FMAs
          im[j] = fma(a.x, c.y, fma(-a.y, c.x, im[j]));
        }
      }
    }
  }
  double* out = partials + ((size_t)b * gridDim.x + blockIdx.x) * 2 * kTriMax;
  if (G > 1) {
    // the groups' sums of each entry, added in group order
    if (g < G) gsum[threadIdx.x] = make_double2(re[0] + re2[0], im[0]);
    __syncthreads();
    if ((int)threadIdx.x < tri) {
      double sr = 0.0, si = 0.0;
      for (int k = 0; k < G; ++k) {
        sr += gsum[k * tri + threadIdx.x].x;
        si += gsum[k * tri + threadIdx.x].y;
      }
      out[2 * threadIdx.x] = sr;
      out[2 * threadIdx.x + 1] = si;
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < kOwn; ++j) {
    const int idx = (int)threadIdx.x + nt * j;
    if (idx >= tri) continue;
    out[2 * idx] = re[j] + re2[j];
    out[2 * idx + 1] = im[j];
  }
}

// G_b[p][q] = the sum over member b's partial blocks (fixed-order tree), one
// block per entry of the upper triangle (grid.x) and member (grid.y); the
// lower triangle by conjugation.
__global__ void __launch_bounds__(256) k_gram_reduce(const double* __restrict__ partials, int blocks,
                                                     RankCounts rc, double* __restrict__ small, int sstride) {
  const int b = blockIdx.y, idx = blockIdx.x;
  const int M = rc.M[b];
  if (idx >= M * (M + 1) / 2) return;                    // the whole block
  int p, q;
  tri_pq(idx, M, &p, &q);
  __shared__ double sre[256], sim[256];
  double re = 0.0, im = 0.0;
  const double* part = partials + (size_t)b * blocks * 2 * kTriMax;
  for (int k = threadIdx.x; k < blocks; k += blockDim.x) {
    re += part[(size_t)k * 2 * kTriMax + 2 * idx];
    im += part[(size_t)k * 2 * kTriMax + 2 * idx + 1];
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
    double* G = small + (size_t)b * sstride + kSmallG;
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
__device__ __forceinline__ double trsqrt(double a) { return rsqrt(a); }
// the same for the FP32 pre-pass (float / float2)
__device__ __forceinline__ float tmul(float a, float b) { return a * b; }
__device__ __forceinline__ float2 tmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ float tadd(float a, float b) { return a + b; }
__device__ __forceinline__ float2 tadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float tconj(float a) { return a; }
__device__ __forceinline__ float2 tconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float tre(float a) { return a; }
__device__ __forceinline__ float tre(float2 a) { return a.x; }
__device__ __forceinline__ float tabs2(float a) { return a * a; }
__device__ __forceinline__ float tabs2(float2 a) { return a.x * a.x + a.y * a.y; }
template <> __device__ __forceinline__ float tscal<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ float2 tscal<float2>(double v) { return make_float2((float)v, 0.f); }
__device__ __forceinline__ float tscale(float a, float v) { return a * v; }
__device__ __forceinline__ float2 tscale(float2 a, float v) { return make_float2(a.x * v, a.y * v); }
__device__ __forceinline__ float trsqrt(float a) { return rsqrtf(a); }
// e^{-i arg a} for a != 0: the sign of a real a, conj(a) / |a| for a complex
// one (FP64 unit modulus: an FP32 reciprocal square root refined by two
// Newton steps in FP64)
__device__ __forceinline__ double unit_phase(double a) { return a < 0.0 ? -1.0 : 1.0; }
__device__ __forceinline__ double2 unit_phase(double2 a) {
  const double a2 = a.x * a.x + a.y * a.y;
  double y = (double)rsqrtf((float)a2);
  y = y * fma(-0.5 * a2 * y, y, 1.5);
  y = y * fma(-0.5 * a2 * y, y, 1.5);
  return make_double2(a.x * y, -a.y * y);
}
__device__ __forceinline__ float unit_phase(float a) { return a < 0.f ? -1.f : 1.f; }
__device__ __forceinline__ float2 unit_phase(float2 a) {
  const float inv = rsqrtf(a.x * a.x + a.y * a.y);
  return make_float2(a.x * inv, -a.y * inv);
}

// conversions between the FP64 and FP32 forms
__device__ __forceinline__ float to32f(float a) { return a; }
__device__ __forceinline__ float2 to32f(float2 a) { return a; }
__device__ __forceinline__ float to32f(double a) { return (float)a; }
__device__ __forceinline__ float2 to32f(double2 a) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ float to32(double a) { return (float)a; }
__device__ __forceinline__ float2 to32(double2 a) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double to64(float a) { return a; }
__device__ __forceinline__ double2 to64(float2 a) { return make_double2(a.x, a.y); }


constexpr int kJP = kMaxGramDim + 1;                    // pitch of the Jacobi arrays

// Parallel cyclic Jacobi on the Hermitian (or real symmetric) A (M x M,
// pitch kJP), accumulating V (V <- V R, from any unitary start).  Each step
// applies Mp/2 disjoint rotations from the round-robin schedule: pair 0 =
// (Mp-1, s), pair i = ((s+i) mod (Mp-1), (s-i) mod (Mp-1)).  A pair rotates
// while |a_pq| > tol * max|a_ii| (decided in FP32: the test needs no more);
// the rotation zeroes a_pq: a phase makes a_pq real, then the classical angle
// with the tangent found in FP32 (any tangent gives an exactly unitary
// rotation, the next sweep removes what is left), cos and sin from one rsqrt.
// The update A <- R^dagger A R and V <- V R touches only the rotating
// pairs' rows and columns; a step in which no pair rotates skips it.  Sweeps
// stop when no pair rotates.  T is double / double2 (FP64) or float / float2 (the
// FP32 pre-pass).  Returns false if the sweep bound was reached.
template <typename T>
__device__ bool jacobi(T* A, T* V, int M, double tol, int max_sweeps = kJacobiSweeps) {
  using RT = decltype(tre(T{}));
  __shared__ T rot[kMaxGramDim / 2][4];
  __shared__ int pp[kMaxGramDim / 2], qq[kMaxGramDim / 2], rotates[kMaxGramDim / 2];
  __shared__ float thr;
  const int tid = threadIdx.x;
  const int Mp = M + (M & 1);
  const int nb = Mp / 2;

  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid < 32) {
      float dmax = 0.f;
      for (int p = tid; p < M; p += 32) dmax = fmaxf(dmax, fabsf((float)tre(A[p * kJP + p])));
      for (int o = 16; o; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      if (tid == 0) thr = (float)tol * dmax;
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
          const float af = sqrtf(tabs2(to32f(apq)));
          if (af > thr && af > 0.f) {
            sd = 1;
            // the angle only has to be close (FP32); cos, sin and the phase
            // must make R exactly unitary (in R's precision)
            const float th = (float)(tre(A[q * kJP + q]) - tre(A[p * kJP + p])) * 0.5f / af;
            const float tf = copysignf(1.0f, th) / (fabsf(th) + sqrtf(1.0f + th * th));
            const RT t = (RT)tf;
            const RT c = trsqrt(fma(t, t, (RT)1)), sn = t * c;
            const T ph = unit_phase(apq);
            R00 = tscal<T>(c);
            R01 = tscal<T>(sn);
            R10 = tscale(ph, -sn);
            R11 = tscale(ph, c);
          }
        }
        rot[tid][0] = R00; rot[tid][1] = R01; rot[tid][2] = R10; rot[tid][3] = R11;
        rotates[tid] = sd;
      }
      if (!__syncthreads_or(sd)) continue;               // nothing rotates in this step
      did = 1;
      // A <- R^dagger (A R) and V <- V R for the step's disjoint rotations, in
      // full-lane passes: first the columns p, q of A and of V (item = pair j,
      // row k; a warp covers two pairs), then the rows p, q of A.  Pairs that
      // do not rotate are skipped.
      for (int w = tid; w < 2 * nb * M; w += blockDim.x) {
        const int which = w / (nb * M), jk = w % (nb * M);
        const int j = jk / M, k = jk % M;
        if (!rotates[j]) continue;
        T* X = which ? V : A;
        const int p = pp[j], q = qq[j];
        const T a = X[k * kJP + p], c = X[k * kJP + q];
        X[k * kJP + p] = tadd(tmul(a, rot[j][0]), tmul(c, rot[j][2]));
        X[k * kJP + q] = tadd(tmul(a, rot[j][1]), tmul(c, rot[j][3]));
      }
      __syncthreads();
      for (int w = tid; w < nb * M; w += blockDim.x) {
        const int j = w / M, k = w % M;
        if (!rotates[j]) continue;
        const int p = pp[j], q = qq[j];
        const T a = A[p * kJP + k], c = A[q * kJP + k];
        A[p * kJP + k] = tadd(tmul(tconj(rot[j][0]), a), tmul(tconj(rot[j][2]), c));
        A[q * kJP + k] = tadd(tmul(tconj(rot[j][1]), a), tmul(tconj(rot[j][3]), c));
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
  // descending, ties in index order: position of i = how many come before it
  for (int i = tid; i < M; i += blockDim.x) {
    int pos = 0;
    for (int j = 0; j < M; ++j) pos += lam[j] > lam[i] || (lam[j] == lam[i] && j < i);
    order[pos] = i;
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
      if (s == 1) {
        // one eigenvector v: the first candidate is P e_j = v conj(v_j) for the
        // first j with |v_j| > kGsAccept -- the loop below, without its search
        const int col = order[i0];
        const T vl = lane < M ? V[lane * kJP + col] : tscal<T>(0.0);
        const unsigned ok = __ballot_sync(0xffffffffu, lane < M && tabs2(vl) > kGsAccept * kGsAccept);
        if (ok) {
          const int j = __ffs(ok) - 1;
          const T sj = V[j * kJP + col];
          const T v = tmul(vl, tconj(sj));
          double nv = lane < M ? tabs2(v) : 0.0;
          for (int o = 16; o; o >>= 1) nv += __shfl_xor_sync(0xffffffffu, nv, o);
          if (lane < M) basis[lane * kJP + found] = tscale(v, rsqrt(nv));
          ++found;
          __syncwarp();
          i0 = i1;
          continue;
        }
      }
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

template <typename T> __device__ __forceinline__ T gload(const double* G, int M, int r, int c);
template <> __device__ __forceinline__ double gload<double>(const double* G, int M, int r, int c) {
  return G[2 * (r * M + c)];
}
template <> __device__ __forceinline__ double2 gload<double2>(const double* G, int M, int r, int c) {
  return make_double2(G[2 * (r * M + c)], G[2 * (r * M + c) + 1]);
}

extern __shared__ double2 eig_sm[];                       // three M x kJP matrices of double2

// Eigendecomposition of one member's Gram matrix G (Hermitian, M x M), then
// eig_finish.  A warp-wide FP64 instruction occupies a scheduler's FP64 unit
// for about 64 clocks on this GPU, so a Jacobi sweep is several times
// cheaper in FP32.  The sweeps therefore run first in FP32 (to 1e-6 of the
// largest eigenvalue); their eigenvectors Q are made orthonormal in FP64 by
// two Newton-Schulz steps Q <- Q (3 I - Q^dagger Q) / 2 (the error squares:
// 1e-7 -> 1e-14 -> 1e-28), A = Q^dagger G Q is formed in FP64, and the FP64
// Jacobi finishes from there, accumulating onto Q: its first sweeps rotate
// pairs whose off-diagonal the FP32 sweeps left at about 1e-7 of the
// largest eigenvalue, the later ones only the few pairs still above
// 4e-16 of it.  The result is an FP64 eigendecomposition of G.
template <typename T, typename T32>
__device__ void eig_member(const double* __restrict__ Gin, int M, int r, int normalize, double* __restrict__ W,
                           double* __restrict__ lam, int* keep, double* scale, int* status) {
  T* A = reinterpret_cast<T*>(eig_sm);
  T* V = reinterpret_cast<T*>(eig_sm + kMaxGramDim * kJP);
  T* X = reinterpret_cast<T*>(eig_sm + 2 * kMaxGramDim * kJP);
  T32* A32 = reinterpret_cast<T32*>(X);                   // the FP32 pass lives in X's space
  T32* V32 = A32 + kMaxGramDim * kJP;
  const int tid = threadIdx.x, MM = M * M;
  for (int i = tid; i < MM; i += blockDim.x) {
    const int p = i / M, q = i % M;
    A32[p * kJP + q] = to32(gload<T>(Gin, M, p, q));
    V32[p * kJP + q] = tscal<T32>(p == q ? 1.0 : 0.0);
  }
  __syncthreads();
  jacobi<T32>(A32, V32, M, kRotTol32, kJacobiSweeps32);  // not converging here only costs FP64 sweeps
  __syncthreads();
  for (int i = tid; i < MM; i += blockDim.x) V[(i / M) * kJP + i % M] = to64(V32[(i / M) * kJP + i % M]);
  __syncthreads();
  for (int it = 0; it < 2; ++it) {
    for (int i = tid; i < MM; i += blockDim.x) {          // X = Q^dagger Q
      const int rr = i / M, c = i % M;
      T acc = tscal<T>(0.0);
      for (int k = 0; k < M; ++k) acc = tadd(acc, tmul(tconj(V[k * kJP + rr]), V[k * kJP + c]));
      X[rr * kJP + c] = acc;
    }
    __syncthreads();
    for (int i = tid; i < MM; i += blockDim.x) {          // A = Q (3 I - X) / 2
      const int rr = i / M, c = i % M;
      T acc = tscale(V[rr * kJP + c], 1.5);
      for (int k = 0; k < M; ++k) acc = tadd(acc, tscale(tmul(V[rr * kJP + k], X[k * kJP + c]), -0.5));
      A[rr * kJP + c] = acc;
    }
    __syncthreads();
    for (int i = tid; i < MM; i += blockDim.x) V[(i / M) * kJP + i % M] = A[(i / M) * kJP + i % M];
    __syncthreads();
  }
  for (int i = tid; i < MM; i += blockDim.x) {            // X = G Q
    const int rr = i / M, c = i % M;
    T acc = tscal<T>(0.0);
    for (int k = 0; k < M; ++k) acc = tadd(acc, tmul(gload<T>(Gin, M, rr, k), V[k * kJP + c]));
    X[rr * kJP + c] = acc;
  }
  __syncthreads();
  for (int i = tid; i < MM; i += blockDim.x) {            // A = Q^dagger X, upper triangle, mirrored
    const int rr = i / M, c = i % M;
    if (rr > c) continue;
    T acc = tscal<T>(0.0);
    for (int k = 0; k < M; ++k) acc = tadd(acc, tmul(tconj(V[k * kJP + rr]), X[k * kJP + c]));
    if (rr == c) acc = tscal<T>(tre(acc));
    A[rr * kJP + c] = acc;
    A[c * kJP + rr] = tconj(acc);
  }
  __syncthreads();
  if (!jacobi<T>(A, V, M, kRotTol) && tid == 0) status[0] = 1;
  __syncthreads();
  eig_finish<T>(A, V, M, r, normalize, W, lam, keep, scale, status);
}

// One block per member: eigendecomposition of G_b (M_b x M_b; real
// arithmetic when G_b is real), truncation to r_b (or to trunc_r > 0 for an
// explicit truncation), keep_b recorded.
__global__ void __launch_bounds__(256) k_eig_truncate(double* __restrict__ small, int sstride, RankCounts rc,
                                                      int trunc_r, int normalize, int* status) {
  const int b = blockIdx.x;
  const int M = rc.M[b];
  const int r = trunc_r > 0 ? trunc_r : rc.rank[b];
  double* base = small + (size_t)b * sstride;
  const double* Gin = base + kSmallG;
  int cplx = 0;
  for (int i = threadIdx.x; i < M * M; i += blockDim.x) cplx |= Gin[2 * i + 1] != 0.0;
  cplx = __syncthreads_or(cplx);
  if (cplx)
    eig_member<double2, float2>(Gin, M, r, normalize, base + kSmallW, base + kSmallLam, rc.keep + b,
                                base + kSmallScale, status);
  else
    eig_member<double, float>(Gin, M, r, normalize, base + kSmallW, base + kSmallLam, rc.keep + b,
                              base + kSmallScale, status);
}

// L_b[c] = scale_b sum_p L'_b[p] W_b[p][c] for c < keep_b, columns keep_b..
// m_b - 1 cleared, then m_b = keep_b; one thread per row and member
// (grid.y), all kept columns (each element of L' is read once).  KMAX is a
// power of two >= every keep_b.  REAL: L' and W are real.
template <typename R, bool REAL, int KMAX>
__global__ void __launch_bounds__(256) k_project(const cplx<R>* __restrict__ Lp, cplx<R>* __restrict__ L, int n,
                                                 int mcap, int rcap, int K, const double* __restrict__ small,
                                                 int sstride, RankCounts rc) {
  __shared__ double2 sW[kMaxGramDim * KMAX];
  const int b = blockIdx.y;
  const int M = rc.M[b], keep = rc.keep[b];
  const int old_cols = M / K;
  const double* base = small + (size_t)b * sstride;
  const double scale = base[kSmallScale];
  const double* W = base + kSmallW;
  for (int i = threadIdx.x; i < M * KMAX; i += blockDim.x) {
    const int p = i / KMAX, c = i % KMAX;
    sW[i] = c < keep ? make_double2(W[2 * (p * keep + c)] * scale, W[2 * (p * keep + c) + 1] * scale)
                     : make_double2(0.0, 0.0);
  }
  __syncthreads();
  if (blockIdx.x == 0 && threadIdx.x == 0) rc.cols[b] = keep;
  const uint64_t N = 1ull << n;
  const cplx<R>* Lpb = Lp + (uint64_t)b * mcap * N;
  cplx<R>* Lb = L + (uint64_t)b * rcap * N;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (uint64_t)gridDim.x * blockDim.x) {
    if constexpr (REAL) {
      double acc[KMAX];
#pragma unroll
      for (int c = 0; c < KMAX; ++c) acc[c] = 0.0;
      for (int p = 0; p < M; ++p) {
        const double a = Lpb[(uint64_t)p * N + x].x;
#pragma unroll
        for (int c = 0; c < KMAX; ++c)
          if (c < keep) acc[c] = fma(a, sW[p * KMAX + c].x, acc[c]);   // keep: the same across the block
      }
#pragma unroll
      for (int c = 0; c < KMAX; ++c)
        if (c < keep) Lb[(uint64_t)c * N + x] = mk<R>((R)acc[c], R(0));
    } else {
      double2 acc[KMAX];
#pragma unroll
      for (int c = 0; c < KMAX; ++c) acc[c] = make_double2(0.0, 0.0);
      for (int p = 0; p < M; ++p) {
        const cplx<R> a = Lpb[(uint64_t)p * N + x];
        const double ax = a.x, ay = a.y;
#pragma unroll
        for (int c = 0; c < KMAX; ++c) {
          if (c >= keep) continue;                         // keep: the same across the block
          const double2 w = sW[p * KMAX + c];              // a * w, four FMAs
          acc[c].x = fma(ax, w.x, fma(-ay, w.y, acc[c].x));
          acc[c].y = fma(ax, w.y, fma(ay, w.x, acc[c].y));
        }
      }
#pragma unroll
      for (int c = 0; c < KMAX; ++c)
        if (c < keep) Lb[(uint64_t)c * N + x] = mk<R>((R)acc[c].x, (R)acc[c].y);
    }
    for (int c = keep; c < old_cols; ++c) Lb[(uint64_t)c * N + x] = mk<R>(R(0), R(0));
  }
}

// Blocks of a grid-stride kernel over `rows` rows per member: about four
// 256-thread blocks per SM in all, at least one per member.
unsigned rows_blocks(uint64_t rows, int members) {
  const uint64_t want = ((uint64_t)num_sms() * 4 + members - 1) / members;
  const uint64_t most = (rows + 255) / 256;
  return (unsigned)std::max<uint64_t>(1, std::min(want, most));
}

template <typename R>
cudaError_t expand_dispatch(qs_ctx* h, const Targets& tg, bool real, const double* E, int K, int e_stride,
                            int max_cols, const KrausGate& g) {
  const uint64_t work = ((1ull << h->n) >> tg.k) * (uint64_t)max_cols;
  const dim3 grid(rows_blocks(work, h->batch), h->batch);
  auto* l = static_cast<const cplx<R>*>(h->state);
  auto* lp = static_cast<cplx<R>*>(h->work);
  const int n = h->n, rcap = h->rank, mcap = h->mcap;
  // a diagonal gate with phase noise has diagonal Kraus operators: one product per output
  bool diag = g.k == 2 && g.noise == QS_NOISE_PHASE;
  for (int r = 0; diag && r < 4; ++r)
    for (int c = 0; c < 4; ++c)
      if (r != c && (g.U[2 * (r * 4 + c)] != 0.0 || g.U[2 * (r * 4 + c) + 1] != 0.0)) diag = false;
  if (diag && real) k_kraus_expand<R, 2, true, true><<<grid, kExpBlock, 0, h->stream>>>(l, lp, n, rcap, mcap, tg, E, K, e_stride, h->rc, g);
  else if (diag) k_kraus_expand<R, 2, false, true><<<grid, kExpBlock, 0, h->stream>>>(l, lp, n, rcap, mcap, tg, E, K, e_stride, h->rc, g);
  else if (tg.k == 1 && real) k_kraus_expand<R, 1, true><<<grid, kExpBlock, 0, h->stream>>>(l, lp, n, rcap, mcap, tg, E, K, e_stride, h->rc, g);
  else if (tg.k == 1) k_kraus_expand<R, 1, false><<<grid, kExpBlock, 0, h->stream>>>(l, lp, n, rcap, mcap, tg, E, K, e_stride, h->rc, g);
  else if (tg.k == 2 && real) k_kraus_expand<R, 2, true><<<grid, kExpBlock, 0, h->stream>>>(l, lp, n, rcap, mcap, tg, E, K, e_stride, h->rc, g);
  else if (tg.k == 2) k_kraus_expand<R, 2, false><<<grid, kExpBlock, 0, h->stream>>>(l, lp, n, rcap, mcap, tg, E, K, e_stride, h->rc, g);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <typename R, bool REAL, int KMAX>
void project_launch(qs_ctx* h, int K) {
  const dim3 grid(rows_blocks(1ull << h->n, h->batch), h->batch);
  k_project<R, REAL, KMAX><<<grid, 256, 0, h->stream>>>(static_cast<const cplx<R>*>(h->work),
                                                        static_cast<cplx<R>*>(h->state), h->n, h->mcap, h->rank, K,
                                                        h->rsmall, kRankStride, h->rc);
}

template <typename R, bool REAL>
void project_kmax(qs_ctx* h, int K, int max_keep) {
  if (max_keep <= 1) project_launch<R, REAL, 1>(h, K);
  else if (max_keep <= 2) project_launch<R, REAL, 2>(h, K);
  else if (max_keep <= 4) project_launch<R, REAL, 4>(h, K);
  else if (max_keep <= 8) project_launch<R, REAL, 8>(h, K);
  else project_launch<R, REAL, 16>(h, K);
}

}  // namespace

int gram_rows_per_block(int n) {
  const uint64_t N = 1ull << n;
  const uint64_t per = (N + (uint64_t)kGramRows * kGramTarget - 1) / ((uint64_t)kGramRows * kGramTarget);
  return (int)(per * kGramRows);
}

size_t gram_partials_doubles(int n, int members) {
  const uint64_t N = 1ull << n;
  const uint64_t blocks = (N + gram_rows_per_block(n) - 1) / gram_rows_per_block(n);
  return (size_t)members * blocks * 2 * kTriMax;
}

cudaError_t launch_kraus_expand(qs_ctx* h, const Targets& tg, bool real, const double* E, int K, int e_stride,
                                int max_cols) {
  KrausGate none{};
  if (h->dtype == QS_C64) return expand_dispatch<float>(h, tg, real, E, K, e_stride, max_cols, none);
  return expand_dispatch<double>(h, tg, real, E, K, e_stride, max_cols, none);
}

cudaError_t launch_kraus_expand_gate(qs_ctx* h, const Targets& tg, bool real, const KrausGate& g, int max_cols) {
  const int K = kraus_count(g.k, g.noise);
  if (h->dtype == QS_C64) return expand_dispatch<float>(h, tg, real, nullptr, K, 0, max_cols, g);
  return expand_dispatch<double>(h, tg, real, nullptr, K, 0, max_cols, g);
}

cudaError_t launch_gram(qs_ctx* h, bool real, int max_M) {
  const uint64_t N = 1ull << h->n;
  const int rows = gram_rows_per_block(h->n);
  const int blocks = (int)((N + rows - 1) / rows);
  const dim3 grid(blocks, h->batch);
  const int nt = rows >= 16 * kGramRows ? kGramThreads : kGramThreads / 2;   // see k_gram_partials
  if (h->dtype == QS_C64 && real)
    k_gram_partials<float, true><<<grid, nt, 0, h->stream>>>((const float2*)h->work, h->n, h->mcap, rows, h->rc, h->partials);
  else if (h->dtype == QS_C64)
    k_gram_partials<float, false><<<grid, nt, 0, h->stream>>>((const float2*)h->work, h->n, h->mcap, rows, h->rc, h->partials);
  else if (real)
    k_gram_partials<double, true><<<grid, nt, 0, h->stream>>>((const double2*)h->work, h->n, h->mcap, rows, h->rc, h->partials);
  else
    k_gram_partials<double, false><<<grid, nt, 0, h->stream>>>((const double2*)h->work, h->n, h->mcap, rows, h->rc, h->partials);
  k_gram_reduce<<<dim3(max_M * (max_M + 1) / 2, h->batch), 256, 0, h->stream>>>(h->partials, blocks, h->rc, h->rsmall, kRankStride);
  return cudaGetLastError();
}

namespace {
constexpr int kEigSmem = 3 * kMaxGramDim * kJP * (int)sizeof(double2);
}

cudaError_t rank_kernel_attributes() {
  static std::atomic<bool> attr{false};
  if (attr.load()) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(k_eig_truncate, cudaFuncAttributeMaxDynamicSharedMemorySize, kEigSmem);
  if (e == cudaSuccess) attr.store(true);
  return e;
}

cudaError_t launch_eig_truncate(qs_ctx* h, int trunc_r, int normalize) {
  const cudaError_t e = rank_kernel_attributes();
  if (e != cudaSuccess) return e;
  k_eig_truncate<<<h->batch, 256, kEigSmem, h->stream>>>(h->rsmall, kRankStride, h->rc, trunc_r, normalize, h->dstatus + 1);
  return cudaGetLastError();
}

cudaError_t launch_project(qs_ctx* h, bool real, int K, int max_keep) {
  if (h->dtype == QS_C64 && real) project_kmax<float, true>(h, K, max_keep);
  else if (h->dtype == QS_C64) project_kmax<float, false>(h, K, max_keep);
  else if (real) project_kmax<double, true>(h, K, max_keep);
  else project_kmax<double, false>(h, K, max_keep);
  return cudaGetLastError();
}

}  // namespace qs
