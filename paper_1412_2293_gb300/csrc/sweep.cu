// Amplitude sweeps: one HBM read and write of the state per gate.
//
// The update is the one of Sec. 2: for a one-qubit gate on qubit t every
// pair (a[i0], a[i0 | 2^t]) with bit t of i0 clear is replaced by U times the
// pair; a k-qubit gate does the same on groups of 2^k amplitudes.  A batch of
// members (Monte Carlo trajectories, or factor columns) is one long array;
// the member of a pair is its index >> n, which gives per-member noisy
// matrices (Eqs. 1-2) without any extra indexing.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "internal.cuh"
#include "philox.cuh"

namespace qs {

namespace {

constexpr int kBlock = 256;

inline int grid_for(uint64_t work, int per_thread = 1) {
  const uint64_t threads = (work + per_thread - 1) / per_thread;
  uint64_t blocks = (threads + kBlock - 1) / kBlock;
  const uint64_t cap = (uint64_t)num_sms() * 16;   // enough resident blocks; grid-stride beyond
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  return (int)blocks;
}

// insert a zero bit at position s
__device__ __forceinline__ uint64_t insert0(uint64_t v, int s) {
  const uint64_t low = v & ((1ull << s) - 1);
  return ((v >> s) << (s + 1)) | low;
}

// Maximally entangled state of Eq. 16 on 2m qubits (system = low m bits):
// amplitude 2^{-m/2} at i + (i << m), i < 2^m, for every member; or, dm,
// the density matrix |Omega><Omega| on vec indices x * 2^(2m) + y.
template <typename R>
__global__ void k_set_entangled(cplx<R>* psi, int m, int members, int dm) {
  const uint64_t D = 1ull << m;
  const int n = 2 * m;
  const uint64_t total = dm ? D * D : D * (uint64_t)members;
  const R amp = dm ? (R)ldexp(1.0, -m) : (R)sqrt(ldexp(1.0, -m));
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t a = w / D, i = w % D;
    if (dm) {
      const uint64_t x = a + (a << m), y = i + (i << m);
      psi[(x << n) + y] = mk<R>(amp, R(0));
    } else {
      psi[(a << n) + i + (i << m)] = mk<R>(amp, R(0));
    }
  }
}

template <typename R>
__global__ void k_set_basis(cplx<R>* psi, int n, int members, uint64_t x, const uint64_t* xs) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < members) {
    const uint64_t xi = xs ? xs[b] : x;
    psi[((uint64_t)b << n) + xi] = mk<R>(R(1), R(0));
  }
}

// One matrix per member: the ideal U (FP64, interleaved) times the noise of
// that member (Eqs. 1, 2, 5, 7, 8), rounded to R.  diag_only writes only the
// 2^k diagonal entries (a diagonal U under phase noise stays diagonal).
struct DMat { double v[2 * 16]; };

template <typename R>
__global__ void k_noise_mats(R* out, int members, int k, DMat U, int noise, int diag_only,
                             NoiseSrc src, uint64_t gate_id) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= members) return;
  const double e = src.e ? src.e[b] : src.e0;
  const uint64_t seed = src.seed ? src.seed[b] : src.seed0;
  const uint64_t traj = src.traj ? src.traj[b] : src.traj0 + (uint64_t)b;
  const double2 xi = noise_normals(seed, traj, gate_id);
  const int d = 1 << k;
  if (noise == QS_NOISE_ROTATION) {
    // V(a) = [[cos a, sin a], [-sin a, cos a]] on each target; targets[0] is
    // the low local bit.  Real matrix NV[r][c] = prod_j V_j[r_j][c_j].
    double ca, sa, cb = 1.0, sb = 0.0;
    sincos(e * xi.x, &sa, &ca);
    if (k == 2) sincos(e * xi.y, &sb, &cb);
    const double Va[2][2] = {{ca, sa}, {-sa, ca}};
    const double Vb[2][2] = {{cb, sb}, {-sb, cb}};
    R* o = out + (size_t)b * 2 * d * d;
    for (int r = 0; r < d; ++r) {
      for (int c = 0; c < d; ++c) {
        double re = 0.0, im = 0.0;
        for (int m = 0; m < d; ++m) {
          double nv = Va[m & 1][c & 1];
          if (k == 2) nv *= Vb[(m >> 1) & 1][(c >> 1) & 1];
          re += U.v[2 * (r * d + m)] * nv;
          im += U.v[2 * (r * d + m) + 1] * nv;
        }
        o[2 * (r * d + c)] = (R)re;
        o[2 * (r * d + c) + 1] = (R)im;
      }
    }
  } else {
    // U * diag(1, .., 1, e^{-i e xi_a})
    double s, c;
    sincos(e * xi.x, &s, &c);
    const double pr = c, pi = -s;
    if (diag_only) {
      R* o = out + (size_t)b * 2 * d;
      for (int r = 0; r < d; ++r) {
        double re = U.v[2 * (r * d + r)], im = U.v[2 * (r * d + r) + 1];
        if (r == d - 1) {
          const double t = re * pr - im * pi;
          im = re * pi + im * pr;
          re = t;
        }
        o[2 * r] = (R)re;
        o[2 * r + 1] = (R)im;
      }
    } else {
      R* o = out + (size_t)b * 2 * d * d;
      for (int r = 0; r < d; ++r) {
        for (int cc = 0; cc < d; ++cc) {
          double re = U.v[2 * (r * d + cc)], im = U.v[2 * (r * d + cc) + 1];
          if (cc == d - 1) {
            const double t = re * pr - im * pi;
            im = re * pi + im * pr;
            re = t;
          }
          o[2 * (r * d + cc)] = (R)re;
          o[2 * (r * d + cc) + 1] = (R)im;
        }
      }
    }
  }
}

template <typename R> struct Mat2 { cplx<R> m00, m01, m10, m11; };

template <typename R>
__device__ __forceinline__ Mat2<R> load_mat2(const R* p) {
  Mat2<R> m;
  m.m00 = mk<R>(p[0], p[1]); m.m01 = mk<R>(p[2], p[3]);
  m.m10 = mk<R>(p[4], p[5]); m.m11 = mk<R>(p[6], p[7]);
  return m;
}

// Pair sweep (Sec. 2): npairs = members * 2^(n-1).  Member of pair p is
// p >> (n-1); its matrix is mats[member] when PER_MEMBER.
template <typename R, bool PER_MEMBER>
__global__ void __launch_bounds__(kBlock) k_apply_1q(cplx<R>* __restrict__ psi, int n, int t,
                                                     uint64_t npairs, Mat2<R> mu,
                                                     const R* __restrict__ mats) {
  using C = cplx<R>;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t bit = 1ull << t;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += stride) {
    const uint64_t i0 = insert0(p, t);
    const uint64_t i1 = i0 | bit;
    Mat2<R> m = mu;
    if (PER_MEMBER) m = load_mat2<R>(mats + (p >> (n - 1)) * 8);
    const C a0 = psi[i0], a1 = psi[i1];
    psi[i0] = cfma(m.m01, a1, cmul(m.m00, a0));
    psi[i1] = cfma(m.m11, a1, cmul(m.m10, a0));
  }
}

// Dense k-qubit gate (k <= 5) on groups of 2^k amplitudes.  REAL: the
// (uniform) matrix has no imaginary part, so each entry costs two multiply-adds.
template <typename R, int K, bool REAL>
__global__ void __launch_bounds__(kBlock) k_apply_kq(cplx<R>* __restrict__ psi, int n,
                                                     uint64_t ngroups, Targets tg,
                                                     const R* __restrict__ mat, int per_member) {
  using C = cplx<R>;
  constexpr int D = 1 << K;
  __shared__ C sm[D * D];
  __shared__ R smr[REAL ? D * D : 1];
  if (!per_member) {
    for (int i = threadIdx.x; i < D * D; i += blockDim.x) {
      if (REAL) smr[i] = mat[2 * i];
      else sm[i] = mk<R>(mat[2 * i], mat[2 * i + 1]);
    }
    __syncthreads();
  }
  if (REAL && !per_member) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += stride) {
      uint64_t base = g;
#pragma unroll
      for (int j = 0; j < K; ++j) base = insert0(base, tg.sorted[j]);
      C a[D];
#pragma unroll
      for (int l = 0; l < D; ++l) a[l] = psi[base + tg.off[l]];
#pragma unroll
      for (int r = 0; r < D; ++r) {
        R re = 0, im = 0;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const R m = smr[r * D + c];
          re += m * a[c].x;
          im += m * a[c].y;
        }
        psi[base + tg.off[r]] = mk<R>(re, im);
      }
    }
    return;
  }
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += stride) {
    uint64_t base = g;
#pragma unroll
    for (int j = 0; j < K; ++j) base = insert0(base, tg.sorted[j]);
    C a[D];
#pragma unroll
    for (int l = 0; l < D; ++l) a[l] = psi[base + tg.off[l]];
    const R* mp = per_member ? mat + (g >> (n - K)) * 2 * D * D : nullptr;
#pragma unroll
    for (int r = 0; r < D; ++r) {
      C acc = mk<R>(R(0), R(0));
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const C m = per_member ? mk<R>(mp[2 * (r * D + c)], mp[2 * (r * D + c) + 1]) : sm[r * D + c];
        acc = cfma(m, a[c], acc);
      }
      psi[base + tg.off[r]] = acc;
    }
  }
}

// Diagonal k-qubit gate: amplitude with local index l is multiplied by d[l];
// only the local indices in active_mask are touched (d[l] = 1 elsewhere).
template <typename R, int K>
__global__ void __launch_bounds__(kBlock) k_apply_diag(cplx<R>* __restrict__ psi, int n,
                                                       uint64_t ngroups, Targets tg,
                                                       const R* __restrict__ diag, int per_member,
                                                       uint32_t active_mask) {
  using C = cplx<R>;
  constexpr int D = 1 << K;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += stride) {
    uint64_t base = g;
#pragma unroll
    for (int j = 0; j < K; ++j) base = insert0(base, tg.sorted[j]);
    const R* dp = per_member ? diag + (g >> (n - K)) * 2 * D : diag;
#pragma unroll
    for (int l = 0; l < D; ++l) {
      if (active_mask & (1u << l)) {
        const uint64_t i = base + tg.off[l];
        psi[i] = cmul(mk<R>(dp[2 * l], dp[2 * l + 1]), psi[i]);
      }
    }
  }
}

template <typename R>
__global__ void k_phase_flip(cplx<R>* psi, int n, int members, uint64_t index, const uint64_t* per) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < members) {
    const uint64_t i = ((uint64_t)b << n) + (per ? per[b] : index);
    cplx<R> v = psi[i];
    v.x = -v.x; v.y = -v.y;
    psi[i] = v;
  }
}

// rho <- F rho F, F = I - 2|w><w|, on vec index i * 2^n + j: negate row w
// and column w (the (w, w) entry twice, i.e. unchanged).
template <typename R>
__global__ void k_dm_flip(cplx<R>* rho, int n, uint64_t w) {
  const uint64_t N = 1ull << n;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (uint64_t)gridDim.x * blockDim.x) {
    if (j == w) continue;
    cplx<R>* a = rho + w * N + j;
    cplx<R>* c = rho + j * N + w;
    a->x = -a->x; a->y = -a->y;
    c->x = -c->x; c->y = -c->y;
  }
}

// T1/T2 relaxation (amplitude damping with gamma = 1 - keep, then dephasing
// to a total coherence factor c) of M qubits at once on a density matrix,
// vec index x * 2^n + y.  For one qubit q and every (x, y) with bit q clear in
// both, the four entries of the (x_q, y_q) block become
//   (0,0) += gamma * (1,1),   (1,1) *= keep,   (0,1), (1,0) *= c.
// A thread owns the 4^M entries that share the other bits (local index bit
// 2m = y-bit of qubit m, bit 2m + 1 = its x-bit) and applies the M channels
// in registers, so M qubits cost one read and one write of rho.
struct RelaxSet {
  int pos[4];      // the 2M vec-bit positions, ascending (insertion order)
  int bit[4];      // local bit j -> vec bit position (y-bit q, x-bit q + n)
};

template <typename R, int M>
__global__ void __launch_bounds__(256) k_dm_relax(cplx<R>* rho, int n, RelaxSet rs, R gamma, R keep, R c) {
  constexpr int L = 1 << (2 * M);
  const uint64_t bases = 1ull << (2 * n - 2 * M);
  uint64_t off[L];
#pragma unroll
  for (int j = 0; j < L; ++j) {
    uint64_t o = 0;
#pragma unroll
    for (int b = 0; b < 2 * M; ++b) o |= (uint64_t)((j >> b) & 1) << rs.bit[b];
    off[j] = o;
  }
  for (uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < bases; w += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t base = w;
#pragma unroll
    for (int b = 0; b < 2 * M; ++b) base = insert0(base, rs.pos[b]);
    cplx<R> a[L];
#pragma unroll
    for (int j = 0; j < L; ++j) a[j] = rho[base + off[j]];
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const int yb = 1 << (2 * m), xb = 2 << (2 * m);
#pragma unroll
      for (int j = 0; j < L; ++j) {
        if (j & (yb | xb)) continue;
        const cplx<R> d = a[j | yb | xb];
        a[j].x = fma(gamma, d.x, a[j].x);
        a[j].y = fma(gamma, d.y, a[j].y);
        a[j | yb | xb] = mk<R>(keep * d.x, keep * d.y);
        a[j | yb] = mk<R>(c * a[j | yb].x, c * a[j | yb].y);
        a[j | xb] = mk<R>(c * a[j | xb].x, c * a[j | xb].y);
      }
    }
#pragma unroll
    for (int j = 0; j < L; ++j) rho[base + off[j]] = a[j];
  }
}

// One-qubit channel with a real superoperator on a Hermitian rho, qubit t >=
// 5.  Groups (the 2 x 2 blocks of rows x0, x0 | T and columns y0, y0 | T, T =
// 2^t) are indexed with bit t removed from x0 and y0 and tiled 32 x 32; since
// t >= 5 a tile's 32 group columns are 32 consecutive matrix columns.  A tile
// on the diagonal is computed in full; a tile above it is computed and also
// written, conjugated and transposed, over the tile below it (which is never
// read): half the reads and half the arithmetic, every access coalesced.
template <typename R>
__global__ void __launch_bounds__(256) k_dm_superop1_herm(cplx<R>* __restrict__ rho, int n, int t,
                                                          const R* __restrict__ S2) {
  __shared__ cplx<R> tile[32][33];
  R S[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) S[i] = S2[2 * i];
  const uint64_t N = 1ull << n, T = 1ull << t;
  const uint64_t TT = (N >> 1) / 32;                     // tiles per dimension
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (uint64_t b = blockIdx.x; b < TT * TT; b += gridDim.x) {
    const uint64_t bx = b / TT, by = b % TT;
    if (bx > by) continue;
    cplx<R> o[4][4];                                     // [row k][quad entry q]
    uint64_t x0s[4];
    const uint64_t y0 = insert0(by * 32 + tx, t);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint64_t x0 = insert0(bx * 32 + ty + 8 * k, t);
      x0s[k] = x0;
      const uint64_t p[4] = {x0 * N + y0, x0 * N + (y0 | T), (x0 | T) * N + y0, (x0 | T) * N + (y0 | T)};
      cplx<R> a[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) a[j] = rho[p[j]];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        R re = 0, im = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) { re = fma(S[4 * q + j], a[j].x, re); im = fma(S[4 * q + j], a[j].y, im); }
        o[k][q] = mk<R>(re, im);
        rho[p[q]] = o[k][q];
      }
    }
    if (bx == by) continue;                              // uniform across the block
    // the mirrored groups: entry q of group (x0, y0) goes to the transposed position
    const uint64_t mx0 = insert0(bx * 32 + tx, t);       // column of the mirrored write
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      __syncthreads();
#pragma unroll
      for (int k = 0; k < 4; ++k) tile[tx][ty + 8 * k] = cconj(o[k][q]);
      __syncthreads();
      // q = 0: (x0, y0) -> (y0, x0); 1: (x0, y0|T) -> (y0|T, x0); 2: (x0|T, y0) -> (y0, x0|T);
      // 3: (x0|T, y0|T) -> (y0|T, x0|T)
      const uint64_t ro = (q & 1) ? T : 0, co = (q & 2) ? T : 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint64_t my0 = insert0(by * 32 + ty + 8 * k, t);
        rho[(my0 | ro) * N + (mx0 | co)] = tile[ty + 8 * k][tx];
      }
    }
    __syncthreads();
  }
}

// The same for qubits t < 5: a raw 32 x 32 tile of rho holds whole groups
// (both partners of every row and column are inside it), so it is loaded into
// shared memory, each of its 256 groups is transformed by one thread, and the
// tile is written back and, above the diagonal, also conjugated and
// transposed over the tile below it.
template <typename R>
__global__ void __launch_bounds__(256) k_dm_superop1_herm_low(cplx<R>* __restrict__ rho, int n, int t,
                                                              const R* __restrict__ S2) {
  __shared__ cplx<R> tile[32][33];
  R S[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) S[i] = S2[2 * i];
  const uint64_t N = 1ull << n;
  const uint64_t TT = N / 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int T = 1 << t;
  // this thread's group in the tile: rows r0, r0 | T, columns c0, c0 | T
  const int gid = threadIdx.x;                           // 256 groups = 16 x 16
  const int r0 = (int)insert0((uint64_t)(gid >> 4), t), c0 = (int)insert0((uint64_t)(gid & 15), t);
  for (uint64_t b = blockIdx.x; b < TT * TT; b += gridDim.x) {
    const uint64_t bx = b / TT, by = b % TT;
    if (bx > by) continue;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) tile[ty + 8 * k][tx] = rho[(bx * 32 + ty + 8 * k) * N + by * 32 + tx];
    __syncthreads();
    {
      cplx<R> a[4] = {tile[r0][c0], tile[r0][c0 | T], tile[r0 | T][c0], tile[r0 | T][c0 | T]};
      cplx<R> o[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        R re = 0, im = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) { re = fma(S[4 * q + j], a[j].x, re); im = fma(S[4 * q + j], a[j].y, im); }
        o[q] = mk<R>(re, im);
      }
      tile[r0][c0] = o[0];
      tile[r0][c0 | T] = o[1];
      tile[r0 | T][c0] = o[2];
      tile[r0 | T][c0 | T] = o[3];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) rho[(bx * 32 + ty + 8 * k) * N + by * 32 + tx] = tile[ty + 8 * k][tx];
    if (bx != by) {
#pragma unroll
      for (int k = 0; k < 4; ++k) rho[(by * 32 + ty + 8 * k) * N + bx * 32 + tx] = cconj(tile[tx][ty + 8 * k]);
    }
  }
}

__global__ void k_debug_noise(uint64_t seed, uint64_t traj, uint64_t gate_id, int count,
                              uint32_t* words, double* normals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) {
    const Words4 w = noise_words(seed, traj + (uint64_t)i, gate_id);
    for (int j = 0; j < 4; ++j) words[4 * i + j] = w.w[j];
    const double2 xi = noise_normals(seed, traj + (uint64_t)i, gate_id);
    normals[2 * i] = xi.x;
    normals[2 * i + 1] = xi.y;
  }
}

template <typename R, bool REAL>
cudaError_t apply_kq_dispatch(qs_ctx* h, void* psi, int n, int members, const Targets& tg,
                              const void* mat, bool per_member) {
  const uint64_t ng = (uint64_t)members << (n - tg.k);
  const int g = grid_for(ng);
  auto* p = static_cast<cplx<R>*>(psi);
  const R* m = static_cast<const R*>(mat);
  switch (tg.k) {
    case 1: k_apply_kq<R, 1, REAL><<<g, kBlock, 0, h->stream>>>(p, n, ng, tg, m, per_member); break;
    case 2: k_apply_kq<R, 2, REAL><<<g, kBlock, 0, h->stream>>>(p, n, ng, tg, m, per_member); break;
    case 3: k_apply_kq<R, 3, REAL><<<g, kBlock, 0, h->stream>>>(p, n, ng, tg, m, per_member); break;
    case 4: k_apply_kq<R, 4, REAL><<<g, kBlock, 0, h->stream>>>(p, n, ng, tg, m, per_member); break;
    case 5: k_apply_kq<R, 5, REAL><<<g, kBlock, 0, h->stream>>>(p, n, ng, tg, m, per_member); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t apply_diag_dispatch(qs_ctx* h, void* psi, int n, int members, const Targets& tg,
                                const void* diag, bool per_member, uint32_t mask) {
  const uint64_t ng = (uint64_t)members << (n - tg.k);
  const int g = grid_for(ng);
  auto* p = static_cast<cplx<R>*>(psi);
  const R* d = static_cast<const R*>(diag);
  switch (tg.k) {
    case 1: k_apply_diag<R, 1><<<g, kBlock, 0, h->stream>>>(p, n, ng, tg, d, per_member, mask); break;
    case 2: k_apply_diag<R, 2><<<g, kBlock, 0, h->stream>>>(p, n, ng, tg, d, per_member, mask); break;
    case 3: k_apply_diag<R, 3><<<g, kBlock, 0, h->stream>>>(p, n, ng, tg, d, per_member, mask); break;
    case 4: k_apply_diag<R, 4><<<g, kBlock, 0, h->stream>>>(p, n, ng, tg, d, per_member, mask); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Dependent multiply-add chains (8 per thread) to measure the arithmetic rate.
template <typename T>
__global__ void k_fma_chain(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (T)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = x[i] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

cudaError_t measure_fma_rates(double* fp64_tflops, double* fp32_tflops) {
  const int grid = num_sms() * 8, block = 256;
  double* d = nullptr;
  cudaError_t e = cudaMalloc((void**)&d, (size_t)grid * block * sizeof(double));
  if (e != cudaSuccess) return e;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best64 = 0.0, best32 = 0.0;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    const int it64 = 2048, it32 = 65536;
    float ms = 0.f;
    cudaEventRecord(e0);
    k_fma_chain<double><<<grid, block>>>(d, it64, 0.999999, 1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    best64 = std::max(best64, 2.0 * 8 * it64 * (double)grid * block / (ms * 1e-3) / 1e12);
    cudaEventRecord(e0);
    k_fma_chain<float><<<grid, block>>>((float*)d, it32, 0.999999f, 1e-7f);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    best32 = std::max(best32, 2.0 * 8 * it32 * (double)grid * block / (ms * 1e-3) / 1e12);
    e = cudaGetLastError();
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d);
  *fp64_tflops = best64;
  *fp32_tflops = best32;
  return e;
}

size_t elem_size(qs_dtype d) { return d == QS_C64 ? 8 : 16; }

int num_sms() {
  static std::atomic<int> cached{0};
  int sms = cached.load();
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    cached.store(sms);
  }
  return sms;
}

Targets make_targets(int n, const int* targets, int k) {
  (void)n;
  Targets tg{};
  tg.k = k;
  for (int j = 0; j < k; ++j) { tg.t[j] = targets[j]; tg.sorted[j] = targets[j]; }
  for (int a = 0; a < k; ++a)
    for (int b = a + 1; b < k; ++b)
      if (tg.sorted[b] < tg.sorted[a]) { const int x = tg.sorted[a]; tg.sorted[a] = tg.sorted[b]; tg.sorted[b] = x; }
  for (int l = 0; l < (1 << k); ++l) {
    uint64_t o = 0;
    for (int j = 0; j < k; ++j) if ((l >> j) & 1) o |= 1ull << targets[j];
    tg.off[l] = o;
  }
  return tg;
}

cudaError_t launch_set_basis(qs_ctx* h, void* psi, int n, int members, uint64_t x, const uint64_t* xs) {
  cudaError_t e = cudaMemsetAsync(psi, 0, ((size_t)members << n) * h->esize, h->stream);
  if (e != cudaSuccess) return e;
  const int g = (members + kBlock - 1) / kBlock;
  if (h->dtype == QS_C64) k_set_basis<float><<<g, kBlock, 0, h->stream>>>((float2*)psi, n, members, x, xs);
  else k_set_basis<double><<<g, kBlock, 0, h->stream>>>((double2*)psi, n, members, x, xs);
  return cudaGetLastError();
}

cudaError_t launch_set_entangled(qs_ctx* h, void* psi, int members, int dm) {
  const int m = h->n / 2;
  const size_t elems = dm ? (size_t)1 << (2 * h->n) : ((size_t)members << h->n);
  cudaError_t e = cudaMemsetAsync(psi, 0, elems * h->esize, h->stream);
  if (e != cudaSuccess) return e;
  const uint64_t total = dm ? (1ull << (2 * m)) : ((uint64_t)members << m);
  uint64_t g = (total + kBlock - 1) / kBlock;
  if (g > (uint64_t)num_sms() * 16) g = (uint64_t)num_sms() * 16;
  if (h->dtype == QS_C64) k_set_entangled<float><<<(int)g, kBlock, 0, h->stream>>>((float2*)psi, m, members, dm);
  else k_set_entangled<double><<<(int)g, kBlock, 0, h->stream>>>((double2*)psi, m, members, dm);
  return cudaGetLastError();
}

cudaError_t launch_noise_mats(qs_ctx* h, void* mats, int members, int k, const double* U, int noise,
                              int diag_only, const NoiseSrc& src, uint64_t gate_id) {
  DMat m{};
  const int d = 1 << k;
  for (int i = 0; i < 2 * d * d; ++i) m.v[i] = U[i];
  const int g = (members + 127) / 128;
  if (h->dtype == QS_C64)
    k_noise_mats<float><<<g, 128, 0, h->stream>>>((float*)mats, members, k, m, noise, diag_only, src, gate_id);
  else
    k_noise_mats<double><<<g, 128, 0, h->stream>>>((double*)mats, members, k, m, noise, diag_only, src, gate_id);
  return cudaGetLastError();
}

cudaError_t launch_apply_1q(qs_ctx* h, void* psi, int n, int members, int t, const double* U,
                            const void* mats) {
  const uint64_t np = (uint64_t)members << (n - 1);
  const int g = grid_for(np);
  if (h->dtype == QS_C64) {
    Mat2<float> mu{};
    if (U) {
      mu.m00 = make_float2((float)U[0], (float)U[1]); mu.m01 = make_float2((float)U[2], (float)U[3]);
      mu.m10 = make_float2((float)U[4], (float)U[5]); mu.m11 = make_float2((float)U[6], (float)U[7]);
      k_apply_1q<float, false><<<g, kBlock, 0, h->stream>>>((float2*)psi, n, t, np, mu, nullptr);
    } else {
      k_apply_1q<float, true><<<g, kBlock, 0, h->stream>>>((float2*)psi, n, t, np, mu, (const float*)mats);
    }
  } else {
    Mat2<double> mu{};
    if (U) {
      mu.m00 = make_double2(U[0], U[1]); mu.m01 = make_double2(U[2], U[3]);
      mu.m10 = make_double2(U[4], U[5]); mu.m11 = make_double2(U[6], U[7]);
      k_apply_1q<double, false><<<g, kBlock, 0, h->stream>>>((double2*)psi, n, t, np, mu, nullptr);
    } else {
      k_apply_1q<double, true><<<g, kBlock, 0, h->stream>>>((double2*)psi, n, t, np, mu, (const double*)mats);
    }
  }
  return cudaGetLastError();
}

cudaError_t launch_apply_kq(qs_ctx* h, void* psi, int n, int members, const Targets& tg,
                            const void* mat, bool per_member, bool real) {
  if (real && !per_member) {
    if (h->dtype == QS_C64) return apply_kq_dispatch<float, true>(h, psi, n, members, tg, mat, false);
    return apply_kq_dispatch<double, true>(h, psi, n, members, tg, mat, false);
  }
  if (h->dtype == QS_C64) return apply_kq_dispatch<float, false>(h, psi, n, members, tg, mat, per_member);
  return apply_kq_dispatch<double, false>(h, psi, n, members, tg, mat, per_member);
}

cudaError_t launch_apply_diag(qs_ctx* h, void* psi, int n, int members, const Targets& tg,
                              const void* diag, bool per_member, uint32_t mask) {
  if (h->dtype == QS_C64) return apply_diag_dispatch<float>(h, psi, n, members, tg, diag, per_member, mask);
  return apply_diag_dispatch<double>(h, psi, n, members, tg, diag, per_member, mask);
}

cudaError_t launch_phase_flip(qs_ctx* h, void* psi, int n, int members, uint64_t index,
                              const uint64_t* per) {
  const int g = (members + kBlock - 1) / kBlock;
  if (h->dtype == QS_C64) k_phase_flip<float><<<g, kBlock, 0, h->stream>>>((float2*)psi, n, members, index, per);
  else k_phase_flip<double><<<g, kBlock, 0, h->stream>>>((double2*)psi, n, members, index, per);
  return cudaGetLastError();
}

cudaError_t launch_dm_superop1_herm(qs_ctx* h, void* rho, int n, int t, const void* S_dev) {
  const uint64_t tt = t < 5 ? 1 : (1ull << (n - 1)) / 32;
  uint64_t blocks = tt * tt;
  const uint64_t cap = (uint64_t)num_sms() * 8;
  if (blocks > cap) blocks = cap;
  if (t < 5) {
    uint64_t lb = (1ull << (2 * n - 10));
    if (lb > cap) lb = cap;
    if (h->dtype == QS_C64)
      k_dm_superop1_herm_low<float><<<(unsigned)lb, 256, 0, h->stream>>>((float2*)rho, n, t, (const float*)S_dev);
    else
      k_dm_superop1_herm_low<double><<<(unsigned)lb, 256, 0, h->stream>>>((double2*)rho, n, t, (const double*)S_dev);
    return cudaGetLastError();
  }
  if (h->dtype == QS_C64)
    k_dm_superop1_herm<float><<<(unsigned)blocks, 256, 0, h->stream>>>((float2*)rho, n, t, (const float*)S_dev);
  else
    k_dm_superop1_herm<double><<<(unsigned)blocks, 256, 0, h->stream>>>((double2*)rho, n, t, (const double*)S_dev);
  return cudaGetLastError();
}

cudaError_t launch_dm_relax(qs_ctx* h, void* rho, int n, const int* qubits, int count, double gamma,
                            double keep, double c) {
  for (int i = 0; i < count; i += 2) {
    const int M = std::min(2, count - i);
    RelaxSet rs{};
    for (int m = 0; m < M; ++m) { rs.bit[2 * m] = qubits[i + m]; rs.bit[2 * m + 1] = qubits[i + m] + n; }
    for (int b = 0; b < 2 * M; ++b) rs.pos[b] = rs.bit[b];
    std::sort(rs.pos, rs.pos + 2 * M);
    const int g = grid_for(1ull << (2 * n - 2 * M));
    if (h->dtype == QS_C64) {
      auto* p = (float2*)rho;
      if (M == 2) k_dm_relax<float, 2><<<g, kBlock, 0, h->stream>>>(p, n, rs, (float)gamma, (float)keep, (float)c);
      else k_dm_relax<float, 1><<<g, kBlock, 0, h->stream>>>(p, n, rs, (float)gamma, (float)keep, (float)c);
    } else {
      auto* p = (double2*)rho;
      if (M == 2) k_dm_relax<double, 2><<<g, kBlock, 0, h->stream>>>(p, n, rs, gamma, keep, c);
      else k_dm_relax<double, 1><<<g, kBlock, 0, h->stream>>>(p, n, rs, gamma, keep, c);
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_dm_flip(qs_ctx* h, void* rho, int n, uint64_t w) {
  const int g = grid_for(1ull << n);
  if (h->dtype == QS_C64) k_dm_flip<float><<<g, kBlock, 0, h->stream>>>((float2*)rho, n, w);
  else k_dm_flip<double><<<g, kBlock, 0, h->stream>>>((double2*)rho, n, w);
  return cudaGetLastError();
}

cudaError_t launch_debug_noise(uint64_t seed, uint64_t traj, uint64_t gate_id, int count,
                               uint32_t* words, double* normals, cudaStream_t s) {
  k_debug_noise<<<(count + 127) / 128, 128, 0, s>>>(seed, traj, gate_id, count, words, normals);
  return cudaGetLastError();
}

}  // namespace qs
