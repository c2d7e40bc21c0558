// Circuit plans: fused window passes over the state, replayed as CUDA graphs.
//
// A pass applies every gate of a run whose dense targets lie in a window of
// m qubits (m = 10 by default; 11 or 12 for complex64 plans, chosen by
// qs_plan_set_window or the autotuner) with one read and one write of the
// state (the amplitude update of
// Sec. 2 done on a tile in registers and shared memory instead of once per
// gate in HBM).  Each thread holds 32 amplitudes of a tile that differ in 5
// "register" bits of the window; a one-qubit gate on a register bit is a
// butterfly over the thread's registers; an exchange through shared memory
// changes which 5 window bits are in registers (two register stages for
// m = 10, three above).
//
// Diagonal two-qubit gates with the form diag(1, 1, 1, x) -- the controlled
// phase shift of Eq. 2 and its Monte Carlo version theta -> theta + e xi
// (Eqs. 7-8) -- are folded in without touching memory:
//   * both qubits in the window: applied right where they occur, attached to
//     the qubit with the higher local index a (a register bit at that point);
//     consecutive ones attached to the same a form one table
//     T[x & (2^a - 1)] of products of their factors;
//   * one or no qubit in the window ("out" terms): they commute with every
//     dense gate of the pass except ones on their window qubit, so the
//     planner forbids those and the pass applies all of them at its end.
// Grover's oracle and diffusion are single-amplitude flips.
//
// Geometry LOW: window = qubits 0..m-1, 2^(m-10) warps per 2^m consecutive
// amplitudes.  Geometry HIGH: the m qubits c..c+m-1, c >= COLB (the top m,
// or a window lower down for larger states); a block handles 2^COLB
// consecutive "columns" (qubits 0..COLB-1) of 2^m window combinations, so
// every global access moves 2^COLB consecutive elements.
//
// Noise of a run: a precompute kernel draws xi for every noisy gate of a pass
// and every member (Philox, same counters as the single-gate calls), builds
// the members' matrices, phase tables and out factors, and the pass kernel
// reads them from a per-member parameter block.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "internal.cuh"
#include "pass.cuh"
#include "philox.cuh"

using cd = std::complex<double>;

namespace qs {
namespace fused {

// per-pass limits (precompute shared memory <= 24 KB, bounded parameter block)
constexpr size_t kMaxContribs = 1024;
constexpr size_t kMaxDwin = 64;
constexpr size_t kMaxTableEntries = 8192;
constexpr size_t kMaxOut = 1024;
constexpr size_t kMaxOps = kMaxPassOps;

// ---------------------------------------------------------------- precompute
enum : int { PD_DENSE = 0, PD_OUT = 1, PD_DWIN = 2 };

struct DGate {            // a gate as the precompute kernel sees it
  double U[32];
  int k;
  int noisy;
  int noise;
  int pad;
  uint64_t gate_pos;      // position in the circuit (gate id offset)
};

struct Producer {
  int kind;
  int gate;               // DENSE / OUT: gate index
  int j;                  // DWIN: attach bit, table of 2^j entries; DENSE: window bit
  int sh;                 // DWIN: 0, or the table split into 2^sh + 2^(j-sh) entries (bits below sh, then the rest)
  int tq;                 // DWIN: 0, or the entry for x stored at (x mod 2^tq) 2^(j-tq) + x / 2^tq (high passes)
  int real;               // DENSE: real matrix, stored as its shears (r0, r0, s1, s1)
  int contrib_start, contrib_count;
  uint32_t off;
  int toff;               // DWIN: offset of its parts in the precompute's FP64 table scratch
};

struct OutStarts { int v[kMaxWin + 2]; };   // out terms of attach a: [v[a], v[a + 1]); a = m: none

struct Contrib {          // DWIN contribution: partner local bit m, gate
  int m;
  int gate;
};

struct RunParams {        // values of one run (written before each launch)
  double e;
  uint64_t seed;
  uint64_t gate_id0;
  uint64_t traj0;
  uint64_t basis;         // basis state of every member when the run starts from one
};

__device__ __forceinline__ void member_noise(const NoiseSrc& src, const RunParams* rp, int b, double* e,
                                             uint64_t* seed, uint64_t* traj) {
  *e = src.e ? src.e[b] : rp->e;
  *seed = src.seed ? src.seed[b] : rp->seed;
  *traj = src.traj ? src.traj[b] : rp->traj0 + (uint64_t)b;
}

// sin and cos of the noise angle e xi_a of one gate and member: FP64 for
// complex128; FP32 for complex64, whose amplitudes the angle only enters in
// FP32 (the normals then come from noise_normals_f32)
template <typename R>
__device__ __forceinline__ void noise_sincos(double e, uint64_t seed, uint64_t traj, uint64_t gid, double* s, double* c) {
  if constexpr (sizeof(R) == 4) {
    const float2 xi = noise_normals_f32(seed, traj, gid);
    float sf, cf;
    sincosf((float)e * xi.x, &sf, &cf);
    *s = sf;
    *c = cf;
  } else {
    const double2 xi = noise_normals(seed, traj, gid);
    sincos(e * xi.x, s, c);
  }
}

// factor of the |1..1> entry of a diag(1,..,1,x) gate for one member
template <typename R>
__device__ __forceinline__ double2 diag_factor(const DGate& g, double e, uint64_t seed, uint64_t traj,
                                               uint64_t gid) {
  const int d = 1 << g.k;
  double re = g.U[2 * ((d - 1) * d + (d - 1))], im = g.U[2 * ((d - 1) * d + (d - 1)) + 1];
  if (g.noisy && g.noise == QS_NOISE_PHASE) {
    double s, c;
    noise_sincos<R>(e, seed, traj, gid, &s, &c);
    const double t = re * c + im * s;                   // x * e^{-i e xi}
    im = im * c - re * s;
    re = t;
  }
  return make_double2(re, im);
}

// Member's noisy 2x2 matrix of a one-qubit gate (interleaved complex, row-major).
template <typename R>
__device__ __forceinline__ void noisy_matrix(const DGate& g, double e, uint64_t seed, uint64_t traj, uint64_t gid,
                                             double (&m)[8]) {
  for (int q = 0; q < 8; ++q) m[q] = g.U[q];
  if (!g.noisy) return;
  double s, c;
  noise_sincos<R>(e, seed, traj, gid, &s, &c);
  if (g.noise == QS_NOISE_ROTATION) {
    // U * [[c, s], [-s, c]]
    for (int r = 0; r < 2; ++r) {
      const double u0r = g.U[4 * r], u0i = g.U[4 * r + 1], u1r = g.U[4 * r + 2], u1i = g.U[4 * r + 3];
      m[4 * r] = u0r * c - u1r * s;
      m[4 * r + 1] = u0i * c - u1i * s;
      m[4 * r + 2] = u0r * s + u1r * c;
      m[4 * r + 3] = u0i * s + u1i * c;
    }
  } else {
    // U * diag(1, e^{-i e xi})
    for (int r = 0; r < 2; ++r) {
      const double ur = g.U[4 * r + 2], ui = g.U[4 * r + 3];
      m[4 * r + 2] = ur * c + ui * s;
      m[4 * r + 3] = ui * c - ur * s;
    }
  }
}

// Smallest pivot magnitude of a factored real gate: a smaller (or zero) pivot
// is replaced by this value, an error of at most this much in one matrix
// entry, far below the precision of R (intermediate values stay in range).
template <typename R> __device__ __forceinline__ double min_pivot() { return sizeof(R) == 4 ? 0x1p-30 : 0x1p-300; }

constexpr int kSmallBits = 5;        // table levels the precompute runs for all parts together

// Members' parameters of one pass, one block of 128 threads per member: the
// noisy matrices of the dense gates in their factored forms, the phase
// tables, the out factors.  The producer list holds the dense gates, then the
// tables, then the out terms (the order build_pass writes).  Every draw and
// product is independent of the others except two chains: the dense gates of
// one window bit (the diagonal carried from gate to gate) and the doubling of
// one table; warp 0 runs the first (one lane per window bit), warps 1-3 the
// second (whole tables per warp), with no block barrier between them.
template <typename R>
__global__ void __launch_bounds__(128) k_precompute(R* __restrict__ params, int stride, const DGate* __restrict__ gates,
                                                    const Producer* __restrict__ prods, int num_prods,
                                                    const Contrib* __restrict__ contribs, int num_contribs,
                                                    int num_dwin, int num_dense, int tab_entries, int diag_off,
                                                    NoiseSrc src, const RunParams* rp, int stable, int m) {
  // shared: [num_contribs] factors, [num_dwin][kMaxWin] partner factors,
  // [tab_entries] FP64 table scratch (a table's parts from its toff), the
  // dense matrices ([num_dense][4] complex), then a copy of the dense and
  // table producers and the contributions' partner bits
  extern __shared__ double2 pre_sm[];
  double2* cf = pre_sm;
  double2* fm = cf + num_contribs;
  double2* tab = fm + (size_t)num_dwin * kMaxWin;
  double2* dmat = tab + tab_entries;
  Producer* sp = reinterpret_cast<Producer*>(dmat + 4 * (size_t)num_dense);
  const int nsp = num_dense + num_dwin;
  unsigned char* cbit = reinterpret_cast<unsigned char*>(sp + nsp);
  const int b = blockIdx.x, tid = threadIdx.x;
  double e;
  uint64_t seed, traj;
  member_noise(src, rp, b, &e, &seed, &traj);
  R* out = params + (uint64_t)b * stride;

  // per-part bookkeeping of the tables (2b): order by size, bits, scratch,
  // first partner factor, output offset; parts with more than q bits (q <=
  // kSmallBits) and all parts
  __shared__ int perm[2 * kMaxDwin], sbits[2 * kMaxDwin], stoff[2 * kMaxDwin], sfb[2 * kMaxDwin];
  __shared__ uint32_t sout[2 * kMaxDwin];
  __shared__ int nact[kSmallBits + 2];
  if (tid < kSmallBits + 2) nact[tid] = 0;
  auto w_base = [](int w) { return w * kMaxWin; };

  // (1) every draw, one item per thread: the noisy 2x2 matrices of the dense
  // gates (FP64, [slot][4] complex; a real gate as (M00, M01), (M10, M11)),
  // the factors of the table contributions, the out factors (straight to
  // the parameters); and the copy of the producers
  for (int i = tid; i < nsp; i += blockDim.x) sp[i] = prods[i];
  const int num_out = num_prods - nsp;
  for (int k = tid; k < num_dense + num_contribs + num_out; k += blockDim.x) {
    if (k < num_dense) {
      const Producer p = prods[k];
      const DGate& g = gates[p.gate];
      double mm[8];
      noisy_matrix<R>(g, e, seed, traj, rp->gate_id0 + g.gate_pos, mm);
      double2* slot = dmat + p.contrib_start * 4;
      if (p.real) {
        slot[0] = make_double2(mm[0], mm[2]);
        slot[1] = make_double2(mm[4], mm[6]);
      } else {
        for (int q = 0; q < 4; ++q) slot[q] = make_double2(mm[2 * q], mm[2 * q + 1]);
      }
    } else if (k < num_dense + num_contribs) {
      const int i = k - num_dense;
      const Contrib c = contribs[i];
      const DGate& g = gates[c.gate];
      cf[i] = diag_factor<R>(g, e, seed, traj, rp->gate_id0 + g.gate_pos);
      cbit[i] = (unsigned char)c.m;
    } else {
      const Producer p = prods[nsp + k - num_dense - num_contribs];   // an out term
      const DGate& g = gates[p.gate];
      const double2 f = diag_factor<R>(g, e, seed, traj, rp->gate_id0 + g.gate_pos);
      out[p.off] = (R)f.x;
      out[p.off + 1] = (R)f.y;
    }
  }
  __syncthreads();

  if (tid < 32) {
    // (2a) dense gates: lane J walks window bit J's gates in circuit order.
    // The diagonal diag(pa, pd) = pa diag(1, rho) left by the previous real
    // gate on the bit is carried into the next one: pa joins the overall
    // scale and a real gate M becomes M' = M diag(1, rho) = [[a, b], [c, d]],
    // factored as diag(d0, d1) [[1, w], [0, 1]] [[1, 0], [q, 1]] [[1, p], [0, 1]]
    // (the kernel: x0 += p x1, x1 += q x0, x0 += w x1), and diag(d0, d1) is
    // carried on.  Pivot on a = M'00 (w = 0: d0 = a, p = b / a, d1 = det'/a,
    // q = c / d1) while |a| >= |column 0| / 4; otherwise (stable runs only) on
    // c (q = 1: d1 = c, p = d / c - 1, d0 = det'/c, w = a c / det' - 1), where
    // no factor exceeds about 4 for an orthogonal M.  Runs that are not stable
    // always take the first form (the host checks that the pivot stays large).
    // A complex gate absorbs the carried diagonal.  What is left at the end
    // goes to the diag block.  The lanes step through their own gates side by
    // side (each finds its next gate, then all factor at once).
    __shared__ double pivot_a[kMaxWin];
    const int J = tid;
    if (J < m) {
      double pa = 1.0, rho = 1.0;
      int i = 0;
      for (;;) {
        while (i < num_dense && sp[i].j != J) ++i;
        if (i >= num_dense) break;
        const Producer& p = sp[i++];
        const double2* slot = dmat + p.contrib_start * 4;
        if (p.real) {
          const double mp = min_pivot<R>();
          auto clamp = [mp](double x) { return fabs(x) < mp ? (x < 0.0 ? -mp : mp) : x; };
          const double a = slot[0].x, bb = slot[0].y * rho, c = slot[1].x, d = slot[1].y * rho;
          const double det = a * d - bb * c;
          double fp, fq, fw, d0, d1;
          if (!stable || fabs(a) >= 0.25 * sqrt(a * a + c * c)) {
            d0 = clamp(a);
            d1 = clamp(det / d0);
            fp = bb / d0;
            fq = c / d1;
            fw = 0.0;
          } else {
            d1 = clamp(c);
            const double dt = clamp(det);
            fp = d / d1 - 1.0;
            d0 = dt / d1;
            fq = 1.0;
            fw = a * d1 / dt - 1.0;
          }
          out[p.off] = (R)fp;                           // (p, p, q, q, w, w)
          out[p.off + 1] = (R)fp;
          out[p.off + 2] = (R)fq;
          out[p.off + 3] = (R)fq;
          out[p.off + 4] = (R)fw;
          out[p.off + 5] = (R)fw;
          pa *= d0;
          rho = d1 / d0;
        } else {
          const double pd = rho * pa;
          for (int q = 0; q < 4; ++q) {
            const double2 v = slot[q];
            const double sc = (q & 1) ? pd : pa;        // column 0 by pa, column 1 by pd
            out[p.off + 2 * q] = (R)(v.x * sc);
            out[p.off + 2 * q + 1] = (R)(v.y * sc);
          }
          pa = 1.0;
          rho = 1.0;
        }
      }
      pivot_a[J] = pa;
      if (diag_off >= 0) out[diag_off + J] = (R)rho;
    }
    __syncwarp();
    if (diag_off >= 0 && tid == 0) {
      double sc = 1.0;
      for (int q = 0; q < m; ++q) sc *= pivot_a[q];
      out[diag_off + m] = (R)sc;
    }
  } else {
    // (2b) partner factors f[q] of each table (the product of its
    // contributions with partner bit q, in list order), one (table, q) per
    // thread of warps 1-3; a single contribution is taken as it is (the
    // product 1 f is f exactly), so the usual case needs no FP64 product
    for (int k = tid - 32; k < num_dwin * m; k += blockDim.x - 32) {
      const int w = k / m, q = k % m;
      const Producer& p = sp[num_dense + w];
      double2 acc = make_double2(1.0, 0.0);
      bool first = true;
      for (int c = p.contrib_start; c < p.contrib_start + p.contrib_count; ++c)
        if (cbit[c] == q) {
          const double2 f = cf[c];
          acc = first ? f : make_double2(acc.x * f.x - acc.y * f.y, acc.x * f.y + acc.y * f.x);
          first = false;
        }
      fm[w * kMaxWin + q] = acc;
    }
    // tables T[x] = prod_{q in x} f[q] over the bits of a part (a table is
    // one part over bits [0, j) or two, [0, sh) then [sh, j)), by doubling in
    // FP64: T[x + 2^q] = T[x] f[q] for x < 2^q, one complex product per
    // entry.  Level q of one part has 2^q items, so the first kSmallBits
    // levels of a part alone would issue FP64 instructions with few lanes
    // busy: those levels run for all parts together (the parts sorted by
    // size, a level's items spread over warps 1-3), and each larger part
    // then finishes its levels in one warp.  Written in R.
    const int u = tid - 32, lane = tid & 31, wq = (tid >> 5) - 1;
    auto slot_bits = [&](int sl) {
      const Producer& p = sp[num_dense + (sl >> 1)];
      if (p.sh > 0) return (sl & 1) ? p.j - p.sh : p.sh;
      return (sl & 1) ? -1 : p.j;
    };
    const int nslot = 2 * num_dwin;
    for (int sl = u; sl < nslot; sl += blockDim.x - 32) {
      const int bits = slot_bits(sl);
      if (bits < 0) continue;
      const Producer& p = sp[num_dense + (sl >> 1)];
      const int part = sl & 1;
      int rank = 0;                                     // by bits descending, then slot
      for (int v = 0; v < nslot; ++v) {
        const int bv = slot_bits(v);
        rank += bv > bits || (bv == bits && v < sl);
      }
      perm[rank] = sl;
      sbits[sl] = bits;
      stoff[sl] = p.toff + (part ? 1 << p.sh : 0);
      sfb[sl] = w_base(sl >> 1) + (part ? p.sh : 0);
      sout[sl] = p.off + (part ? ((2u << p.sh) + 3u) & ~3u : 0u);
      tab[stoff[sl]] = make_double2(1.0, 0.0);
      for (int q = 0; q <= kSmallBits; ++q)
        if (bits > q) atomicAdd(&nact[q], 1);
      atomicAdd(&nact[kSmallBits + 1], 1);
    }
    asm volatile("bar.sync 1, 96;" ::: "memory");       // warps 1-3 only
    for (int q = 0; q < kSmallBits; ++q) {
      const int items = nact[q] << q;
      for (int k = u; k < items; k += blockDim.x - 32) {
        const int sl = perm[k >> q], x = k & ((1 << q) - 1);
        double2* t = tab + stoff[sl];
        const double2 f = fm[sfb[sl] + q];
        const double2 v = t[x];
        t[x + (1 << q)] = make_double2(v.x * f.x - v.y * f.y, v.x * f.y + v.y * f.x);
      }
      asm volatile("bar.sync 1, 96;" ::: "memory");
    }
    auto write_part = [&](int sl) {
      const int bits = sbits[sl];
      const double2* t = tab + stoff[sl];
      const int tq = sp[num_dense + (sl >> 1)].tq;
      const uint32_t o = sout[sl];
      for (int x = lane; x < (1 << bits); x += 32) {
        const int at = tq > 0 ? ((x & ((1 << tq) - 1)) << (bits - tq)) | (x >> tq) : x;
        out[o + 2 * at] = (R)t[x].x;
        out[o + 2 * at + 1] = (R)t[x].y;
      }
    };
    // larger parts: the remaining levels and the write, round robin over the warps
    const int nbig = nact[kSmallBits], nall = nact[kSmallBits + 1];
    for (int i = wq; i < nbig; i += 3) {
      const int sl = perm[i];
      double2* t = tab + stoff[sl];
      for (int q = kSmallBits; q < sbits[sl]; ++q) {
        const double2 f = fm[sfb[sl] + q];
        const int half = 1 << q;
        for (int x = lane; x < half; x += 32) {
          const double2 v = t[x];
          t[x + half] = make_double2(v.x * f.x - v.y * f.y, v.x * f.y + v.y * f.x);
        }
        __syncwarp();
      }
      write_part(sl);
    }
    for (int i = nbig + wq; i < nall; i += 3) write_part(perm[i]);
  }
}

// Out factors of every tile of a pass: for member b and each value o of the
// out-of-window bits (those below the window, then those above it), entry
// (o, a) = the product of the out terms attached to window bit a (a = m:
// attached to none) whose out-of-window bits are all set in o, times the
// deferred real diagonal of bit a (the overall scale for a = m).  The pass
// kernels read the m + 1 entries of their tile directly.
//
// The product factors over o = y 2^L + x (x: the low L = kOutLoBits bits): a
// term whose bits all lie in x's part (in y's) depends on x (on y) alone, so
// an entry is Tlo[a][x] Thi[a][y] times the terms whose bits lie in both (none
// for two-qubit gates with one qubit in the window).  A block takes a run of
// y (entries [y 2^L (m + 1), (y + 1) 2^L (m + 1)) each), builds Tlo over every
// x (the diagonal of a folded in) and Thi over its y, and each thread keeps
// one column c = x (m + 1) + a of the run's rows: one product per entry,
// the warps' stores contiguous.
constexpr int kOutLoBits = 6;        // bits of o in Tlo
constexpr int kOutEntries = 16384;   // out-factor entries per block (at least one row of y)

// rows of y per block (the Thi entries per attach a block needs)
inline int out_table_rows(int obits, int m) {
  const int L = obits < kOutLoBits ? obits : kOutLoBits;
  const int row = (m + 1) << L;
  const int rows = kOutEntries / row > 1 ? kOutEntries / row : 1;
  const int all = 1 << (obits - L);
  return rows < all ? rows : all;
}

template <typename R>
__global__ void __launch_bounds__(256) k_out_table(cplx<R>* __restrict__ tab, const R* __restrict__ params, int stride,
                                                   const OutTerm* __restrict__ outs, OutStarts starts, int diag_off,
                                                   int obits, int wstart, uint32_t chunks, int m, int rows) {
  // shared: the member's terms (masks, factors, classes), Tlo[m + 1][2^L], Thi[m + 1][rows]
  extern __shared__ unsigned char ot_sm[];
  const int nterms = starts.v[m + 1];
  const int A = m + 1;
  const int L = obits < kOutLoBits ? obits : kOutLoBits;
  const int nx = 1 << L;
  uint64_t* masks = reinterpret_cast<uint64_t*>(ot_sm);
  cplx<R>* fac = reinterpret_cast<cplx<R>*>(masks + ((nterms + 1) & ~1));   // 16-byte aligned
  cplx<R>* tlo = fac + nterms;
  cplx<R>* thi = tlo + A * nx;
  unsigned char* cls = reinterpret_cast<unsigned char*>(thi + A * rows);
  const uint64_t b = blockIdx.x / chunks;
  const R* P = params + b * (uint64_t)stride;
  // member-local out-of-window bits of o: the wstart bits below the window,
  // then the bits above it
  auto expand = [&](uint64_t o) { return ((o >> wstart) << (wstart + m)) | (o & ((1ull << wstart) - 1)); };
  const uint64_t lo_bits = expand((1ull << L) - 1);
  __shared__ int sv[kMaxWin + 2];                      // term ranges by attach
  if ((int)threadIdx.x < m + 2) sv[threadIdx.x] = starts.v[threadIdx.x];
  int straddle = 0;
  for (int k = threadIdx.x; k < nterms; k += blockDim.x) {
    const OutTerm t = outs[k];
    masks[k] = t.cmask;
    fac[k] = mk<R>(P[t.off], P[t.off + 1]);
    const int c = (t.cmask & ~lo_bits) == 0 ? 0 : ((t.cmask & lo_bits) == 0 ? 1 : 2);
    cls[k] = (unsigned char)c;
    straddle |= c == 2;
  }
  straddle = __syncthreads_or(straddle);
  // the block's rows of y
  const uint64_t y0 = (uint64_t)(blockIdx.x % chunks) * rows;
  const uint64_t ycount = 1ull << (obits - L);
  const int ny = (int)(y0 + rows < ycount ? rows : ycount - y0);
  auto term_product = [&](int a, int want, uint64_t fixed, R re, R im) {
    for (int k = sv[a]; k < sv[a + 1]; ++k) {
      if (cls[k] == want && (fixed & masks[k]) == masks[k]) {
        const cplx<R> f = fac[k];
        const R nr = re * f.x - im * f.y;
        im = re * f.y + im * f.x;
        re = nr;
      }
    }
    return mk<R>(re, im);
  };
  for (int k = threadIdx.x; k < A * (nx + ny); k += blockDim.x) {
    const int a = k % A, u = k / A;
    if (u < nx) {
      const R d = diag_off >= 0 ? P[diag_off + a] : R(1);
      tlo[a * nx + u] = term_product(a, 0, expand((uint64_t)u), d, R(0));
    } else {
      const int yy = u - nx;
      thi[a * rows + yy] = term_product(a, 1, expand((y0 + yy) << L), R(1), R(0));
    }
  }
  __syncthreads();
  const int row = A * nx;
  cplx<R>* dst = tab + (b << obits) * A + y0 * row;
  for (int c = threadIdx.x; c < row; c += blockDim.x) {
    const int x = c / A, a = c % A;
    const cplx<R> t = tlo[a * nx + x];
    for (int yy = 0; yy < ny; ++yy) {
      const cplx<R> h = thi[a * rows + yy];
      cplx<R> v = mk<R>(t.x * h.x - t.y * h.y, t.x * h.y + t.y * h.x);
      if (straddle) v = term_product(a, 2, expand(((y0 + yy) << L) | (uint64_t)x), v.x, v.y);
      dst[(uint64_t)yy * row + c] = v;
    }
  }
}

// A run of diagonal channels on the exact density matrix (Sec. 3): noiseless
// diagonal gates and phase flips (rho -> D rho D^dagger) and noisy diagonal
// gates with the phase-noise Kraus pair of Eq. 9.  Each multiplies rho[x][y]
// by d(x) conj(d(y)), and a noisy one also by sqrt(P) when exactly one of x, y
// has all its targets set (the pair gives 1 when both or neither have), so the
// run multiplies rho[x][y] by u(x) conj(u(y)) qpow[popcount(mask(x) ^ mask(y))]
// with u = the product of the diagonals and bit c of mask(x) = "x has all
// targets of noisy gate c set".  vec index x 2^n + y.
// Tables and arithmetic in the state's precision (complex64: FP32 throughout).
// Bit 31 of mask(x) marks an index whose factor is exactly 1 with no noisy
// gate active: pairs of such indices are skipped by an integer test.
template <typename R> struct QPow { R v[33]; };
constexpr uint32_t kDmTrivial = 1u << 31;

template <typename R>
__global__ void __launch_bounds__(256) k_dm_diag_block(cplx<R>* __restrict__ rho, int n, const cplx<R>* __restrict__ u,
                                                       const uint32_t* __restrict__ mask, QPow<R> qp) {
  const uint64_t N = 1ull << n;
  const uint64_t total = N * N;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t x = v >> n, y = v & (N - 1);
    const uint32_t mx = mask[x], my = mask[y];
    if (mx & my & kDmTrivial) continue;
    const cplx<R> ux = u[x], uy = u[y];
    const R d = qp.v[__popc((mx ^ my) & ~kDmTrivial)];
    const R fr = (ux.x * uy.x + ux.y * uy.y) * d, fi = (ux.y * uy.x - ux.x * uy.y) * d;
    const cplx<R> r = rho[v];
    rho[v] = mk<R>(r.x * fr - r.y * fi, r.x * fi + r.y * fr);
  }
}

}  // namespace fused
}  // namespace qs

// ======================================================================= host
using namespace qs;
using namespace qs::fused;

namespace {

struct PGate {
  qs_gate g;
  std::vector<cd> U;
  bool dense1 = false;    // fusable one-qubit gate
  bool cp = false;        // fusable diag(1, .., 1, x) two-qubit gate
  bool flip = false;
  bool diag = false;      // any diagonal gate (for commutation)
  uint64_t qmask = 0;     // qubits touched (all for flips)
};

struct PassPlan {
  bool high = false;
  int colb = 3;
  int m = kWin;                   // window width
  int win[kMaxWin];
  int start_stage = 0;
  std::vector<FOp> ops;
  std::vector<OutTerm> outs;      // sorted by attach
  int out_start[kMaxWin + 2];     // terms of attach a: [out_start[a], out_start[a + 1]); a = m: none
  std::vector<Producer> prods;
  std::vector<Contrib> contribs;
  int num_dwin = 0;
  int num_dense = 0;
  int diag_off = -1;              // deferred diagonals of the factored real gates
  int tab_entries = 0;            // FP64 scratch entries of the tables in the precompute
  int stride = 0;                 // R units per member
  std::vector<int> other;
  int tile_shift = 0;             // log2(tiles per member)
  std::vector<Seg> segs;          // the ops in canonical segments (what the kernels run)
  int prog = 0;                   // compile-time program of the pass kernel (0: interpreted)
  std::vector<Flip> flips;
  CUtensorMap tmap;               // HIGH: [members * 2^(n-c) rows][2^c columns] (c = win[0]), boxes of 2^colb columns
  CUtensorMap tmap4;              // HIGH complex64, m = 10: the same with boxes of 4 columns (configuration 2)
  // device copies
  FOp* d_ops = nullptr;
  OutTerm* d_outs = nullptr;
  Producer* d_prods = nullptr;
  Contrib* d_contribs = nullptr;
  void* d_params = nullptr;
  void* d_alpha = nullptr;        // per member and out-of-window tile value: m + 1 out factors
};

struct Step {
  int kind;               // 0 = fused pass, 1 = single gate, 2 = density-matrix diagonal block,
                          // 5 = the gates of a fixed-rank plan (RankOp list)
  int pass = -1;
  int gate = -1;          // single gate, or the diagonal block's index
};

// One gate of a fixed-rank plan, applied to every member with launch shapes
// fixed when the plan is made (the members' column counts stay on the device).
struct RankOp {
  int kind;               // 0 flip, 1 one-qubit unitary, 2 diagonal, 3 two-qubit dense, 4 noisy channel
  int gate;
  size_t mat_off = 0;     // kinds 2, 3: offset (elements of the handle's precision) in d_rank_mats
  uint32_t mask = 0;      // kind 2: local indices whose factor is not 1
  bool real = true;       // the gate keeps a real factor real
};

struct DmBlock {          // density matrix: a run of diagonal channels (k_dm_diag_block)
  double2* d_u = nullptr;         // complex128 handles
  float2* d_uf = nullptr;         // complex64 handles
  uint32_t* d_mask = nullptr;
  int noisy = 0;
};

}  // namespace

struct qs_plan_s {
  qs_ctx* h = nullptr;
  std::vector<PGate> gates;
  std::vector<PassPlan> passes;
  std::vector<Step> steps;
  DGate* d_gates = nullptr;
  RunParams* d_run = nullptr;
  RunParams* h_run = nullptr;     // pinned
  // captured graphs, one per run variant: start (0 loaded, 1 one basis state,
  // 2 per-member basis states) x fused fidelity (0, 1)
  // (x 2: real gates in the two-shear form, or pivoted with a third shear)
  static constexpr int kVariants = 12;
  cudaGraphExec_t exec[kVariants] = {};
  bool graph_member_noise[kVariants] = {};
  bool graph_member_marked[kVariants] = {};
  bool graph_timing[kVariants] = {};
  int64_t graph_wait_polls[kVariants] = {};
  int stable = 0;                 // the running variant: 1 = pivoted real gates
  double* d_fid = nullptr;        // fused-fidelity partials [member][tile] complex
  void* d_params = nullptr;       // per-member gate parameters of the running pass (shared by the passes)
  void* d_alpha = nullptr;        // out factors of the running pass (shared by the passes)
  std::vector<DmBlock> dm_blocks;
  std::vector<RankOp> rank_ops;   // FIXED_RANK plans
  void* d_rank_mats = nullptr;
  int rank_variant = 0;           // the running variant: real start, per-member noise, normalisation
  int rank_kmax = 0;              // the largest member rank: the projection's column bound
  int graph_kmax[kVariants] = {};
  int colb = 3;
  int m = kWin;                   // window width of the fused passes
  int low_cfg = 0;                // kernel configuration of each window geometry (see launch_pass_kernel)
  int high_cfg = 0;
  int launches = 0;               // timing slots of a run (precompute, pass, single step)
  int kernels = 0;                // kernels one run launches
  bool timing = false;
  std::vector<cudaEvent_t> events;     // launches + 1 when timing
  std::vector<int> event_kinds;
  std::string err;
};

namespace {

// Largest |xi| the noise draw can produce: Box-Muller of a uniform no
// smaller than 2^-54 gives sqrt(-2 ln 2^-54) = 8.65.
constexpr double kXiMax = 8.7;

// True when every member is certain to keep the two-shear form of every real
// one-qubit gate of the plan: |M00| >= |column 0| / 4 for M = U V_noise(theta),
// |theta| <= e_max kXiMax (rotation noise acting first), bounded from U alone:
// |M00| >= |U00| cos(theta) - |U01| sin(theta) and |column 0| <= |U|_F.
bool two_shear_safe(const std::vector<struct PGate>& gates, double e_max);

qs_status pfail(qs_plan p, qs_status st, const std::string& m) {
  if (p && p->h) p->h->err = m;
  if (p) p->err = m;
  return st;
}

bool is_diag(const std::vector<cd>& U, int d) {
  for (int r = 0; r < d; ++r)
    for (int c = 0; c < d; ++c)
      if (r != c && U[r * d + c] != cd(0, 0)) return false;
  return true;
}

PGate classify(const qs_gate& g, int n) {
  PGate p;
  p.g = g;
  if (g.kind == QS_GATE_FLIP || g.kind == QS_FLIP_PER_MEMBER) {
    p.flip = true;
    p.diag = true;
    p.qmask = n >= 64 ? ~0ull : ((1ull << n) - 1);
    return p;
  }
  const int d = 1 << g.k;
  p.U.resize(d * d);
  for (int i = 0; i < d * d; ++i) p.U[i] = cd(g.U[2 * i], g.U[2 * i + 1]);
  for (int j = 0; j < g.k; ++j) p.qmask |= 1ull << g.targets[j];
  const bool diag = is_diag(p.U, d);
  p.diag = diag && (!g.noisy || g.noise == QS_NOISE_PHASE);
  if (g.k == 1) p.dense1 = true;
  if (g.k == 2 && diag && (!g.noisy || g.noise == QS_NOISE_PHASE) && p.U[0] == cd(1, 0) &&
      p.U[5] == cd(1, 0) && p.U[10] == cd(1, 0))
    p.cp = true;
  return p;
}

bool commute(const PGate& a, const PGate& b) {
  if (a.diag && b.diag) return true;
  return (a.qmask & b.qmask) == 0;
}

// Register stage for window bit j of a window of m bits: the current stage
// when its register bits hold j, else A (the top five), B (bits 0..4) or C
// (bits 5..9, m > 10) -- the one that holds j.
int stage_for(int j, int m, int cur) {
  if (cur >= 0 && j >= stage_base(m, cur) && j < stage_base(m, cur) + kRegBits) return cur;
  if (j >= m - kRegBits) return 0;
  return j < kRegBits ? 1 : 2;
}

bool two_shear_safe(const std::vector<PGate>& gates, double e_max) {
  for (const PGate& g : gates) {
    if (!g.dense1) continue;
    bool real = true;
    for (const auto& v : g.U) if (v.imag() != 0.0) real = false;
    if (!real || (g.g.noisy && g.g.noise == QS_NOISE_PHASE)) continue;   // complex path: no pivot
    const double th = g.g.noisy ? e_max * kXiMax : 0.0;
    if (th >= 1.5) return false;
    const double u00 = std::abs(g.U[0]), u01 = std::abs(g.U[1]);
    const double fro = std::sqrt(std::norm(g.U[0]) + std::norm(g.U[1]) + std::norm(g.U[2]) + std::norm(g.U[3]));
    if (u00 * std::cos(th) - u01 * std::sin(th) < 0.25 * fro) return false;
  }
  return true;
}

// Greedy pass builder starting at remaining[0]; returns absorbed flags.
// Start c of a high window [c, c + m) for a run whose first dense gate is on
// qubit q >= m: of the candidates n - m (the top), q - m + 1 (the run goes
// down) and q (it goes up), the one holding most of the run's next one-qubit
// gates; -1 when none is allowed (c >= colb, and the tensor map's row
// coordinate, members x 2^(n-c), within 31 bits).
int choose_window(const std::vector<PGate>& G, const std::vector<int>& rem, int n, int colb, uint64_t batch, int q,
                  int m) {
  int best = -1, best_count = -1;
  const int cand[3] = {n - m, q - (m - 1), q};
  for (int c : cand) {
    c = std::min(std::max(c, colb), n - m);
    if (c < colb || q < c || q >= c + m) continue;
    if (n - c >= 31 || (batch << (n - c)) >= (1ull << 31)) continue;
    int count = 0;
    for (size_t i = 0; i < rem.size() && i < 256; ++i) {
      const PGate& g = G[rem[i]];
      if (!g.dense1 && !g.cp && !g.flip) break;
      if (g.dense1 && g.g.targets[0] >= c && g.g.targets[0] < c + m) ++count;
    }
    if (count > best_count) { best = c; best_count = count; }
  }
  return best;
}

bool build_pass(const std::vector<PGate>& G, const std::vector<int>& rem, int n, int colb, uint64_t batch,
                size_t op_budget, int m, PassPlan* P, std::vector<char>* absorbed) {
  P->colb = colb;
  P->m = m;
  // window from the first fusable dense gate (lookahead)
  int q = -1;
  for (size_t i = 0; i < rem.size() && i < 64; ++i) {
    const PGate& g = G[rem[i]];
    if (!g.dense1 && !g.cp && !g.flip) break;
    if (g.dense1) { q = g.g.targets[0]; break; }
  }
  P->high = false;
  int c0 = 0;
  if (q >= m) {
    if (n < m + colb) return false;                  // a high tile needs 2^colb columns
    c0 = choose_window(G, rem, n, colb, batch, q, m);
    if (c0 < 0) return false;
    P->high = true;
  }
  for (int l = 0; l < m; ++l) P->win[l] = c0 + l;
  int loc[64];
  for (int i = 0; i < 64; ++i) loc[i] = -1;
  for (int l = 0; l < m; ++l) loc[P->win[l]] = l;

  std::vector<int> skipped;
  uint64_t locked = 0;                                  // window local bits with out terms
  int stage = -1;
  int dense_count = 0;
  struct Dw { int j; std::vector<Contrib> cs; int sh; int tq; };
  std::vector<Dw> dwins;                                // indexed by producer order
  std::vector<std::pair<int, int>> out_gates;           // (attach, gate) in order
  std::vector<uint64_t> out_masks;
  P->ops.clear();
  // an exchange op names the stage it goes to (j); a low pass starts in stage A
  auto need_stage = [&](int j) {
    const int st = stage_for(j, m, stage);
    if (stage == -1) {
      stage = st;
      P->start_stage = P->high ? st : 0;
      if (!P->high && st != 0) { FOp x{}; x.type = OP_EXCH; x.j = (uint8_t)st; P->ops.push_back(x); }
    } else if (stage != st) {
      FOp x{}; x.type = OP_EXCH; x.j = (uint8_t)st; P->ops.push_back(x); stage = st;
    }
  };
  size_t ncontrib = 0, table_entries = 0;
  for (size_t i = 0; i < rem.size(); ++i) {
    const PGate& g = G[rem[i]];
    if (!g.dense1 && !g.cp && !g.flip) break;           // a gate the pass cannot hold ends the scan
    // bounds of one pass: precompute shared memory and the per-member block
    // (a new table has at most 2^(m-1) entries: the total stays within kMaxTableEntries)
    if (ncontrib >= kMaxContribs || dwins.size() >= kMaxDwin ||
        table_entries + (1u << (m - 1)) > kMaxTableEntries ||
        out_gates.size() >= kMaxOut || P->ops.size() + 2 > op_budget)
      break;
    bool ok = true;
    for (int s : skipped) if (!commute(G[s], g)) { ok = false; break; }
    bool can = false;
    if (ok) {
      if (g.dense1) {
        const int l = loc[g.g.targets[0]];
        can = l >= 0 && !((locked >> l) & 1);
      } else {
        can = true;                                     // diagonal gates always fit
      }
    }
    if (!can) {
      skipped.push_back(rem[i]);
      if (skipped.size() > 96) break;
      continue;
    }
    (*absorbed)[i] = 1;
    if (g.dense1) {
      const int l = loc[g.g.targets[0]];
      need_stage(l);
      FOp x{};
      x.type = OP_DENSE;
      x.j = (uint8_t)l;
      bool real = true;
      for (const auto& v : g.U) if (v.imag() != 0.0) real = false;
      if (g.g.noisy && g.g.noise == QS_NOISE_PHASE) real = false;
      x.real = real ? 1 : 0;
      Producer pr{};
      pr.kind = PD_DENSE;
      pr.gate = rem[i];
      pr.j = l;
      pr.real = x.real;
      pr.contrib_start = dense_count;                   // DENSE: slot of its matrix in the precompute
      x.off = (uint32_t)P->prods.size();                // patched to an offset below
      P->prods.push_back(pr);
      P->ops.push_back(x);
      ++dense_count;
    } else if (g.flip) {
      FOp x{};
      x.type = g.g.kind == QS_GATE_FLIP ? OP_FLIP : OP_FLIPM;
      x.index = g.g.index;
      P->ops.push_back(x);
    } else {
      const int p0 = g.g.targets[0], p1 = g.g.targets[1];
      const int l0 = loc[p0], l1 = loc[p1];
      if (l0 >= 0 && l1 >= 0) {
        const int a = std::max(l0, l1), partner = std::min(l0, l1);
        need_stage(a);
        if (!P->ops.empty() && P->ops.back().type == OP_DWIN && P->ops.back().j == a) {
          dwins[P->ops.back().off].cs.push_back(Contrib{partner, rem[i]});
        } else {
          FOp x{};
          x.type = OP_DWIN;
          x.j = (uint8_t)a;
          x.off = (uint32_t)dwins.size();
          // windows above 10 qubits keep the table as its factors over the
          // thread's bits and the register bits of the stage
          const int sh = m > kWin ? stage_base(m, stage) : 0;
          // a high pass keeps a whole table register-index fastest: a lane's
          // factors for neighbouring register values are adjacent
          const int tq = (P->high && sh == 0) ? stage_base(m, stage) : 0;
          dwins.push_back(Dw{a, {Contrib{partner, rem[i]}}, sh, tq});
          P->ops.push_back(x);
          table_entries += sh > 0 ? (1u << sh) + (1u << (a - sh)) : 1u << a;
        }
        ++ncontrib;
      } else {
        int a = -1;
        uint64_t cm = 0;
        if (l0 >= 0) { a = l0; cm = 1ull << p1; }
        else if (l1 >= 0) { a = l1; cm = 1ull << p0; }
        else { cm = (1ull << p0) | (1ull << p1); }
        if (a >= 0) locked |= 1ull << a;
        out_gates.push_back({a, rem[i]});
        out_masks.push_back(cm);
      }
    }
  }
  if (dense_count == 0 && out_gates.empty() && dwins.empty()) {
    // only flips (or nothing): not worth a pass unless something was absorbed
    bool any = false;
    for (char c : *absorbed) any |= c != 0;
    if (!any) return false;
  }
  if (stage == -1) { stage = 0; P->start_stage = 0; }

  // parameter layout: dense matrices, tables, out factors
  std::vector<Producer> prods;
  uint32_t off = 0;
  bool any_real = false;
  for (auto& x : P->ops) {
    if (x.type == OP_DENSE) {
      Producer pr = P->prods[x.off];
      pr.off = off;
      x.off = off;
      off += 8;                                         // (p, p, q, q, w, w, -, -) or the complex 2x2
      any_real |= pr.real != 0;
      prods.push_back(pr);
    }
  }
  P->num_dense = dense_count;
  P->diag_off = -1;
  if (any_real) {                                       // ratios of the m window bits + scale
    P->diag_off = (int)off;
    off += (uint32_t)((m + 1 + 3) & ~3);
  }
  P->contribs.clear();
  P->num_dwin = 0;
  P->tab_entries = 0;
  for (auto& x : P->ops) {
    if (x.type == OP_DWIN) {
      Dw& d = dwins[x.off];
      Producer pr{};
      pr.kind = PD_DWIN;
      pr.j = d.j;
      pr.sh = d.sh;
      pr.tq = d.tq;
      pr.toff = P->tab_entries;
      P->tab_entries += d.sh > 0 ? (1 << d.sh) + (1 << (d.j - d.sh)) : 1 << d.j;
      pr.contrib_start = (int)P->contribs.size();
      pr.contrib_count = (int)d.cs.size();
      for (auto& c : d.cs) P->contribs.push_back(c);
      pr.off = off;
      x.off = off;
      // parts rounded to 4 R units: every part starts 16-byte aligned (pair loads)
      auto part = [](int bits) { return ((2u << bits) + 3u) & ~3u; };
      off += d.sh > 0 ? part(d.sh) + part(d.j - d.sh) : part(d.j);
      prods.push_back(pr);
      ++P->num_dwin;
    }
  }
  // out terms sorted by attach (a = -1 last)
  std::vector<int> order(out_gates.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const int ax = out_gates[x].first < 0 ? m : out_gates[x].first;
    const int ay = out_gates[y].first < 0 ? m : out_gates[y].first;
    return ax < ay;
  });
  P->outs.clear();
  for (int i = 0; i < kMaxWin + 2; ++i) P->out_start[i] = 0;
  int cnt[kMaxWin + 1] = {0};
  for (int idx : order) {
    const int a = out_gates[idx].first;
    OutTerm t{};
    t.a = a;
    t.off = off;
    t.cmask = out_masks[idx];
    Producer pr{};
    pr.kind = PD_OUT;
    pr.gate = out_gates[idx].second;
    pr.off = off;
    off += 2;
    prods.push_back(pr);
    P->outs.push_back(t);
    cnt[a < 0 ? m : a]++;
  }
  int acc = 0;
  for (int a = 0; a <= m; ++a) { P->out_start[a] = acc; acc += cnt[a]; }
  P->out_start[m + 1] = acc;
  P->prods = prods;
  P->stride = (int)((off + 3) & ~3u);
  P->other.clear();
  if (P->high) {
    for (int b = P->colb; b < n; ++b) if (loc[b] < 0) P->other.push_back(b);
    P->tile_shift = n - m - P->colb;
  } else {
    P->tile_shift = n - m;
  }
  return true;
}

// Group a pass's ops into segments (see Seg).  Returns false when they do
// not fit the kernel-parameter limits.
bool segment_pass(PassPlan* P) {
  // partner masks of the phase tables, in op order
  std::vector<uint32_t> partners;
  for (const Producer& pr : P->prods) {
    if (pr.kind != PD_DWIN) continue;
    uint32_t m = 0;
    for (int c = pr.contrib_start; c < pr.contrib_start + pr.contrib_count; ++c) m |= 1u << P->contribs[c].m;
    partners.push_back(m);
  }
  struct Item { int type; int j; uint32_t partners; const FOp* op; };
  std::vector<Item> cur;
  int cur_stage = 0;
  bool open = false;
  P->segs.clear();
  P->flips.clear();
  auto order_ok = [&](const std::vector<Item>& items, bool desc) {
    auto pos = [&](const Item& it) {
      const int rj = it.j - stage_base(P->m, cur_stage);
      const int idx = desc ? 4 - rj : rj;
      return 2 * idx + (it.type == OP_DWIN ? 1 : 0);
    };
    for (size_t x = 0; x < items.size(); ++x)
      for (size_t y = x + 1; y < items.size(); ++y) {
        const Item& a = items[x];
        const Item& b = items[y];
        bool commute = true;
        if (a.type == OP_DENSE && b.type == OP_DENSE) commute = a.j != b.j;
        else if (a.type == OP_DENSE && b.type == OP_DWIN) commute = a.j != b.j && !((b.partners >> a.j) & 1);
        else if (a.type == OP_DWIN && b.type == OP_DENSE) commute = a.j != b.j && !((a.partners >> b.j) & 1);
        if (!commute && pos(a) >= pos(b)) return false;
      }
    return true;
  };
  std::vector<FOp> pending_flips;
  auto close = [&]() {
    if (!open) return;
    Seg sg{};
    sg.stage = (uint8_t)cur_stage;
    sg.desc = order_ok(cur, true) ? 1 : 0;
    for (const Item& it : cur) {
      const int rj = it.j - stage_base(P->m, cur_stage);
      if (it.type == OP_DENSE) {
        sg.dense |= 1u << rj;
        sg.doff[rj] = it.op->off;
        if (it.op->real) sg.real |= 1u << rj;
      } else {
        sg.dwin |= 1u << rj;
        sg.woff[rj] = it.op->off;
      }
    }
    sg.flip0 = (uint16_t)P->flips.size();
    sg.nflip = (uint8_t)pending_flips.size();
    for (const FOp& f : pending_flips) {
      Flip fl{};
      fl.index = f.index;
      fl.per_member = f.type == OP_FLIPM ? 1 : 0;
      P->flips.push_back(fl);
    }
    P->segs.push_back(sg);
    cur.clear();
    pending_flips.clear();
    open = false;
  };
  int stage = P->high ? P->start_stage : 0;
  size_t dw = 0;
  for (const FOp& op : P->ops) {
    if (op.type == OP_EXCH) { close(); stage = op.j; continue; }
    if (op.type == OP_FLIP || op.type == OP_FLIPM) {
      if (!open) { open = true; cur_stage = stage; }
      pending_flips.push_back(op);
      close();                                          // nothing dense may follow a flip in a segment
      continue;
    }
    Item it{op.type, op.j, op.type == OP_DWIN ? partners[dw++] : 0u, &op};
    bool fits = open && cur_stage == stage;
    if (fits)
      for (const Item& x : cur)
        if (x.type == it.type && x.j == it.j) fits = false;          // one of each per register bit
    if (fits) {
      std::vector<Item> trial = cur;
      trial.push_back(it);
      fits = order_ok(trial, true) || order_ok(trial, false);
    }
    if (!fits) { close(); open = true; cur_stage = stage; }
    cur.push_back(it);
  }
  close();
  return P->segs.size() <= (size_t)kMaxSegs && P->flips.size() <= (size_t)kMaxFlips;
}

// The compiled program a pass can run (see prog_layers), or 0.  Only the
// shapes compiled into the pass kernels qualify: real one-qubit gates on all
// ten window bits, stage A then stage B, descending, with the phase tables of
// the noisy QFT (every bit of stage A, bits 1..4 of stage B).
constexpr int kLayerPrograms[] = {prog_layers(0x1f, 0x1e)};

// Windows of 11 and 12 qubits: the full-window program (wide_full_prog),
// segments A, C, B (a low pass may lack A: it starts in A all the same).
int choose_wide_prog(const PassPlan& P) {
  const int want = wide_full_prog(P.m);
  if (!want || !P.flips.empty() || P.segs.empty() || P.segs.size() > 3) return 0;
  const int first = 3 - (int)P.segs.size();            // stages A, C, B from index first
  if (first != 0 && (P.high || first != 1)) return 0;
  static const int order[3] = {0, 2, 1};
  int prog = kProgWide;
  for (size_t i = 0; i < P.segs.size(); ++i) {
    const Seg& g = P.segs[i];
    const int k = first + (int)i;
    if (g.stage != order[k] || !g.desc || g.nflip || g.real != g.dense) return 0;
    prog |= ((int)g.dense << (10 * k)) | ((int)g.dwin << (10 * k + 5));
  }
  return prog == want ? prog : 0;
}

int choose_prog(const PassPlan& P) {
  if (P.m != kWin) return choose_wide_prog(P);
  if (P.segs.size() != 2 || !P.flips.empty() || (P.high && P.start_stage != 0)) return 0;
  const Seg& a = P.segs[0];
  const Seg& b = P.segs[1];
  if (a.stage != 0 || b.stage != 1 || !a.desc || !b.desc || a.nflip || b.nflip) return 0;
  if (a.dense != 0x1f || b.dense != 0x1f || a.real != 0x1f || b.real != 0x1f) return 0;
  const int prog = prog_layers(a.dwin, b.dwin);
  for (int q : kLayerPrograms)
    if (q == prog) return prog;
  return 0;
}

template <typename T>
qs_status upload(qs_plan p, T** dst, const std::vector<T>& v) {
  if (v.empty()) { *dst = nullptr; return QS_OK; }
  if (cudaMalloc((void**)dst, v.size() * sizeof(T)) != cudaSuccess) return pfail(p, QS_ERR_OUT_OF_MEMORY, "plan upload");
  if (cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess)
    return pfail(p, QS_ERR_CUDA, "plan upload copy");
  return QS_OK;
}

// Kernel configurations of the two window geometries.  complex64:
//   low  0: 12 warps, two tile buffers per warp (registers <= 170)
//   low  1: 16 warps, one buffer per warp, next copy issued after the tile's
//           last shared read (registers <= 128)
//   low  2: 12 warps, one buffer per warp (registers <= 170)
//   high 0: one block of 8 warps per SM, two tile buffers
//   high 1: two blocks per SM, one buffer each (registers <= 128)
//   high 2: four blocks of 4 warps per SM (tiles of 4 columns), one buffer each
// complex128: low 4 warps / two buffers, high 4 columns / two buffers.
// Wider windows: see launch_pass_wide.
constexpr int kLowCfgsF = 3, kHighCfgsF = 3, kLowCfgsD = 1, kHighCfgsD = 1;
template <typename R> constexpr int high_colb() { return sizeof(R) == 4 ? 3 : 2; }
int num_low_cfgs(size_t esize, int m) { return m != kWin ? 1 : (esize == 8 ? kLowCfgsF : kLowCfgsD); }
int num_high_cfgs(size_t esize, int m) { return m != kWin ? 1 : (esize == 8 ? kHighCfgsF : kHighCfgsD); }

// Tensor map of the state as [batch * 1024 rows][2^(n-10) columns] of 8-byte
// elements (a complex128 amplitude is two of them), boxes of 2^colb amplitudes
// x 256 rows.
qs_status make_tmap(qs_plan p, PassPlan* P, int colb, CUtensorMap* map) {
  static std::atomic<PFN_cuTensorMapEncodeTiled_v12000> encode_fn{nullptr};
  PFN_cuTensorMapEncodeTiled_v12000 encode = encode_fn.load();
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return pfail(p, QS_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    encode_fn.store(encode);
  }
  qs_ctx* h = p->h;
  const uint64_t per = h->esize / 8;                     // 8-byte elements per amplitude
  // rows: (member, bits above the window, window bits); columns: the bits below the window
  const int c = P->win[0];
  cuuint64_t dims[2] = {(cuuint64_t)(1ull << c) * per, (cuuint64_t)h->batch << (h->n - c)};
  cuuint64_t strides[1] = {dims[0] * 8};
  cuuint32_t box[2] = {(cuuint32_t)((1u << colb) * per), 256};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, h->state, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return pfail(p, QS_ERR_CUDA, "tensor map encode failed");
  return QS_OK;
}

// columns per high-window tile of the configuration launched (0 for the low window)
int launch_colb(qs_plan p, const PassPlan& P) {
  if (!P.high) return 0;
  if (P.m != kWin) return wide_colb(P.m);
  return p->h->esize == 8 && p->high_cfg == 2 ? 2 : P.colb;
}
int launch_tile_shift(qs_plan p, const PassPlan& P) { return p->h->n - P.m - launch_colb(p, P); }
// fused-fidelity partials per member: one per tile, and per warp of a tile in
// the low window (2^(m-10) warps)
int fid_slots(qs_plan p, const PassPlan& P) {
  return (1 << launch_tile_shift(p, P)) * (P.high ? 1 : 1 << (P.m - kWin));
}

PassArgs pass_args(qs_plan p, const PassPlan& P, int synth, int fid) {
  qs_ctx* h = p->h;
  PassArgs A{};
  A.n = h->n;
  A.m = P.m;
  A.start_stage = P.start_stage;
  for (int l = 0; l < P.m; ++l) A.win[l] = P.win[l];
  A.nseg = (int)P.segs.size();
  for (int i = 0; i < A.nseg; ++i) A.segs[i] = P.segs[i];
  for (size_t i = 0; i < P.flips.size(); ++i) A.flips[i] = P.flips[i];
  A.alpha_tab = P.d_alpha;
  A.param_stride = P.stride;
  A.params = P.d_params;
  A.marked = h->m_marked;
  const uint64_t total = (uint64_t)h->batch << h->n;
  A.tile_shift = launch_tile_shift(p, P);
  A.tiles = total >> (P.m + launch_colb(p, P));
  A.status = h->dstatus + 2;
  A.synth = synth ? 1 : 0;
  A.basis = synth == 2 ? h->m_basis : nullptr;
  A.basis0 = &p->d_run->basis;
  A.fid = fid;
  A.ref = h->ref;
  A.fid_partials = p->d_fid;
  A.diag_off = P.diag_off;
  A.stable = p->stable;
  A.spin_limit = h->wait_polls < 0 ? kSpinLimit : (uint32_t)h->wait_polls;
  return A;
}

// Shared memory of k_precompute: contribution factors, partner factors, table
// scratch and dense matrices (FP64 complex), the dense and table producers,
// the contributions' partner bits.
size_t precompute_smem(size_t contribs, size_t dwin, size_t tab_entries, size_t dense) {
  return (contribs + dwin * kMaxWin + tab_entries + 4 * dense) * sizeof(double2) + (dense + dwin) * sizeof(Producer) +
         contribs;
}

// Members' noise draws, matrices, phase tables and out factors of one pass.
template <typename R>
cudaError_t launch_precompute(qs_plan p, const PassPlan& P, cudaStream_t s) {
  qs_ctx* h = p->h;
  NoiseSrc src{};
  if (h->member_noise) { src.e = h->m_e; src.seed = h->m_seed; src.traj = h->m_traj; }
  const size_t pre_smem = precompute_smem(P.contribs.size(), P.num_dwin, P.tab_entries, P.num_dense);
  k_precompute<R><<<h->batch, 128, pre_smem, s>>>((R*)P.d_params, P.stride, p->d_gates, P.d_prods,
                                                   (int)P.prods.size(), P.d_contribs, (int)P.contribs.size(),
                                                   P.num_dwin, P.num_dense, P.tab_entries, P.diag_off, src,
                                                   p->d_run, p->stable, P.m);
  if (P.d_alpha) {
    OutStarts st{};
    for (int i = 0; i < kMaxWin + 2; ++i) st.v[i] = P.out_start[i];
    const int obits = h->n - P.m;
    const int nterms = P.out_start[P.m + 1];
    const int L = obits < kOutLoBits ? obits : kOutLoBits;
    const int rows = out_table_rows(obits, P.m);
    const uint32_t chunks = (uint32_t)(((1ull << (obits - L)) + rows - 1) / rows);
    const size_t sm = (size_t)((nterms + 1) & ~1) * sizeof(uint64_t) +
                      ((size_t)nterms + (size_t)(P.m + 1) * ((1u << L) + rows)) * sizeof(cplx<R>) + nterms;
    k_out_table<R><<<(unsigned)(chunks * (uint64_t)h->batch), 256, sm, s>>>(
        (cplx<R>*)P.d_alpha, (const R*)P.d_params, P.stride, P.d_outs, st, P.diag_off, obits, P.win[0], chunks, P.m,
        rows);
  }
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pass_kernel(qs_plan p, const PassPlan& P, cudaStream_t s, int synth, int fid) {
  using C = cplx<R>;
  qs_ctx* h = p->h;
  const PassArgs A = pass_args(p, P, synth, fid);
  const int prog = p->stable ? 0 : P.prog;               // the compiled programs take two shears
  const int sms = num_sms();
  auto grid = [&](uint64_t units, int per_sm) {
    const uint64_t cap = (uint64_t)sms * per_sm;
    return (int)(units < cap ? units : cap);
  };
  C* psi = (C*)h->state;
  constexpr int kQft = prog_layers(0x1f, 0x1e);
  if constexpr (sizeof(R) == 4) {
    // wider windows (n <= 32, checked when the width is set)
    if (P.m != kWin) return launch_pass_wide(psi, P.tmap, A, P.high, P.m, prog, sms, s);
  }
  if (!P.high) {
    if constexpr (sizeof(R) == 4) {
      if (prog == kQft && p->low_cfg == 1)
        k_pass_low<R, 16, 1, kQft><<<grid((A.tiles + 15) / 16, 1), 16 * 32, low_smem<R, 16, 1>(), s>>>(psi, A);
      else if (prog == kQft && p->low_cfg == 2)
        k_pass_low<R, 12, 1, kQft><<<grid((A.tiles + 11) / 12, 1), 12 * 32, low_smem<R, 12, 1>(), s>>>(psi, A);
      else if (p->low_cfg == 1)
        k_pass_low<R, 16, 1><<<grid((A.tiles + 15) / 16, 1), 16 * 32, low_smem<R, 16, 1>(), s>>>(psi, A);
      else if (p->low_cfg == 2)
        k_pass_low<R, 12, 1><<<grid((A.tiles + 11) / 12, 1), 12 * 32, low_smem<R, 12, 1>(), s>>>(psi, A);
      else
        k_pass_low<R, 12, 2><<<grid((A.tiles + 11) / 12, 1), 12 * 32, low_smem<R, 12, 2>(), s>>>(psi, A);
    } else {
      k_pass_low<R, 4, 2><<<grid((A.tiles + 3) / 4, 1), 4 * 32, low_smem<R, 4, 2>(), s>>>(psi, A);
    }
  } else {
    constexpr int CB = high_colb<R>();
    if (A.n > 32) {                // 64-bit member-local offsets; one configuration
      k_pass_high<R, CB, 2, true><<<grid(A.tiles, 1), HighShape<CB>::THREADS, high_smem<R, CB, 2>(), s>>>(psi, P.tmap, A);
      return cudaGetLastError();
    }
    if constexpr (sizeof(R) == 4) {
      if (p->high_cfg == 1) {
        if (prog == kQft)
          k_pass_high<R, CB, 1, false, kQft><<<grid(A.tiles, 2), HighShape<CB>::THREADS, high_smem<R, CB, 1>(), s>>>(psi, P.tmap, A);
        else
          k_pass_high<R, CB, 1><<<grid(A.tiles, 2), HighShape<CB>::THREADS, high_smem<R, CB, 1>(), s>>>(psi, P.tmap, A);
        return cudaGetLastError();
      }
      if (p->high_cfg == 2) {
        if (prog == kQft)
          k_pass_high<R, 2, 1, false, kQft><<<grid(A.tiles, 4), HighShape<2>::THREADS, high_smem<R, 2, 1>(), s>>>(psi, P.tmap4, A);
        else
          k_pass_high<R, 2, 1><<<grid(A.tiles, 4), HighShape<2>::THREADS, high_smem<R, 2, 1>(), s>>>(psi, P.tmap4, A);
        return cudaGetLastError();
      }
    }
    k_pass_high<R, CB, 2><<<grid(A.tiles, 1), HighShape<CB>::THREADS, high_smem<R, CB, 2>(), s>>>(psi, P.tmap, A);
  }
  return cudaGetLastError();
}

// fused fidelity: out[b] = |sum over the last pass's tiles of member b|^2.
// One warp per member: lane l adds slots l, l + 32, ... in order, then the
// lanes' sums meet in a fixed shuffle tree (FP64 throughout, the same order
// on every run).
__global__ void __launch_bounds__(256) k_fid_finalize(const double* __restrict__ partials, int members, int tiles,
                                                      double* __restrict__ out) {
  const int b = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= members) return;                            // uniform per warp
  const double* pm = partials + 2 * (uint64_t)b * tiles;
  double re = 0.0, im = 0.0;
  for (int t = lane; t < tiles; t += 32) {
    re += pm[2 * t];
    im += pm[2 * t + 1];
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) out[b] = re * re + im * im;
}

cudaError_t set_smem_attrs(size_t esize) {
  static std::atomic<bool> done[2] = {false, false};
  const int which = esize == 8 ? 0 : 1;
  if (done[which]) return cudaSuccess;
  const size_t pre_max = precompute_smem(kMaxContribs, kMaxDwin, kMaxTableEntries, kMaxOps);
  cudaError_t e = esize == 8
      ? cudaFuncSetAttribute(k_precompute<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pre_max)
      : cudaFuncSetAttribute(k_precompute<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pre_max);
  if (e != cudaSuccess) return e;
  if (esize == 8) {
    e = set_pass_attrs(k_pass_low<float, 12, 2>, low_smem<float, 12, 2>(), 1);
    if (e == cudaSuccess) e = set_pass_attrs(k_pass_low<float, 16, 1>, low_smem<float, 16, 1>(), 1);
    if (e == cudaSuccess) e = set_pass_attrs(k_pass_low<float, 12, 1>, low_smem<float, 12, 1>(), 1);
    if (e == cudaSuccess) e = set_pass_attrs(k_pass_high<float, 3, 2>, high_smem<float, 3, 2>(), 1);
    if (e == cudaSuccess) e = set_pass_attrs(k_pass_high<float, 3, 1>, high_smem<float, 3, 1>(), 2);
    if (e == cudaSuccess) e = set_pass_attrs(k_pass_high<float, 2, 1>, high_smem<float, 2, 1>(), 4);
    if (e == cudaSuccess) e = set_pass_attrs(k_pass_high<float, 3, 2, true>, high_smem<float, 3, 2>(), 1);
    constexpr int kQft = prog_layers(0x1f, 0x1e);
    if (e == cudaSuccess) e = set_pass_attrs(k_pass_low<float, 16, 1, kQft>, low_smem<float, 16, 1>(), 1);
    if (e == cudaSuccess) e = set_pass_attrs(k_pass_low<float, 12, 1, kQft>, low_smem<float, 12, 1>(), 1);
    if (e == cudaSuccess) e = set_pass_attrs(k_pass_high<float, 3, 1, false, kQft>, high_smem<float, 3, 1>(), 2);
    if (e == cudaSuccess) e = set_pass_attrs(k_pass_high<float, 2, 1, false, kQft>, high_smem<float, 2, 1>(), 4);
    if (e == cudaSuccess) e = set_wide_attrs();
  } else {
    e = set_pass_attrs(k_pass_low<double, 4, 2>, low_smem<double, 4, 2>(), 1);
    if (e == cudaSuccess) e = set_pass_attrs(k_pass_high<double, 2, 2>, high_smem<double, 2, 2>(), 1);
    if (e == cudaSuccess) e = set_pass_attrs(k_pass_high<double, 2, 2, true>, high_smem<double, 2, 2>(), 1);
  }
  if (e == cudaSuccess) done[which] = true;
  return e;
}

// The same on a Hermitian rho (n >= 5): tiles of 32 x 32 entries; a tile on
// the diagonal is computed in full, a tile above it is computed and also
// written, conjugated and transposed, over the tile below it (the factor of
// (y, x) is the conjugate of that of (x, y)), through shared memory so every
// access is coalesced: half the reads and half the arithmetic.
// A thread keeps one column y and takes rows x = 8 k + warp, so a row is the
// same across a warp.  The factor u(x) conj(u(y)) q^popcount(m(x) ^ m(y)) is
// formed only as far as the row and column need: a trivial row (u = 1, no
// noisy gate) takes the column's own factor conj(u(y)) q^popcount(m(y)),
// computed once per tile; a non-trivial row over columns that are all
// trivial takes u(x) q^popcount(m(x)); only pairs where both are non-trivial
// pay the full product.  Pairs of trivial rows and columns are skipped.
template <typename R>
__global__ void __launch_bounds__(256) k_dm_diag_block_herm(cplx<R>* __restrict__ rho, int n,
                                                            const cplx<R>* __restrict__ u,
                                                            const uint32_t* __restrict__ mask, QPow<R> qp) {
  __shared__ cplx<R> tile[32][33];
  __shared__ R qv[33];
  if (threadIdx.x < 33) qv[threadIdx.x] = qp.v[threadIdx.x];
  __syncthreads();
  const uint64_t N = 1ull << n;
  const uint64_t TT = N / 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (uint64_t b = blockIdx.x; b < TT * TT; b += gridDim.x) {
    const uint64_t bx = b / TT, by = b % TT;
    if (bx > by) continue;
    const uint64_t y = by * 32 + tx;
    const uint32_t my = mask[y];
    const cplx<R> uy = u[y];
    const uint32_t myb = my & ~kDmTrivial;
    const bool ytriv = (my & kDmTrivial) != 0;
    const bool cols_trivial = __all_sync(0xffffffffu, ytriv);
    const R dy = qv[__popc(myb)];
    const cplx<R> colf = mk<R>(uy.x * dy, -uy.y * dy);  // factor of a trivial row
    cplx<R> o[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint64_t x = bx * 32 + ty + 8 * k;
      const uint32_t mx = mask[x];                      // the same across the warp
      const cplx<R> r = rho[x * N + y];
      o[k] = r;
      cplx<R> f;
      if (mx & kDmTrivial) {
        if (ytriv) continue;
        f = colf;
      } else {
        const cplx<R> ux = u[x];
        if (cols_trivial) {
          const R dx = qv[__popc(mx)];
          f = mk<R>(ux.x * dx, ux.y * dx);
        } else {
          const R d = qv[__popc(mx ^ myb)];
          f = mk<R>((ux.x * uy.x + ux.y * uy.y) * d, (ux.y * uy.x - ux.x * uy.y) * d);
        }
      }
      o[k] = mk<R>(r.x * f.x - r.y * f.y, r.x * f.y + r.y * f.x);
      rho[x * N + y] = o[k];
    }
    if (bx == by) continue;                              // uniform across the block
#pragma unroll
    for (int k = 0; k < 4; ++k) tile[tx][ty + 8 * k] = cconj(o[k]);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) rho[(by * 32 + ty + 8 * k) * N + bx * 32 + tx] = tile[ty + 8 * k][tx];
    __syncthreads();
  }
}

qs_status run_single(qs_plan p, const PGate& g, const RunParams& rp, int pos);

// a density-matrix diagonal block with noise level rp.e: qpow[k] = sqrt(P)^k, P = exp(-e^2)
qs_status run_dm_block(qs_plan p, const DmBlock& b, const RunParams& rp) {
  qs_ctx* h = p->h;
  QPow<double> qp{};
  const double q = std::sqrt(std::exp(-rp.e * rp.e));
  qp.v[0] = 1.0;
  for (int i = 1; i <= 32; ++i) qp.v[i] = qp.v[i - 1] * q;
  const uint64_t total = 1ull << (2 * h->n);
  uint64_t blocks = (total + 255) / 256;
  const uint64_t cap = (uint64_t)num_sms() * 16;
  if (blocks > cap) blocks = cap;
  const bool herm = h->hermitian && h->n >= 5;
  const uint64_t tiles = herm ? (1ull << (2 * h->n - 10)) : 0;
  const unsigned hblocks = (unsigned)std::min<uint64_t>(tiles, (uint64_t)num_sms() * 8);
  if (h->dtype == QS_C64) {
    QPow<float> qf{};
    for (int i = 0; i <= 32; ++i) qf.v[i] = (float)qp.v[i];
    if (herm)
      k_dm_diag_block_herm<float><<<hblocks, 256, 0, h->stream>>>((float2*)h->state, h->n, b.d_uf, b.d_mask, qf);
    else
      k_dm_diag_block<float><<<(int)blocks, 256, 0, h->stream>>>((float2*)h->state, h->n, b.d_uf, b.d_mask, qf);
  } else {
    if (herm)
      k_dm_diag_block_herm<double><<<hblocks, 256, 0, h->stream>>>((double2*)h->state, h->n, b.d_u, b.d_mask, qp);
    else
      k_dm_diag_block<double><<<(int)blocks, 256, 0, h->stream>>>((double2*)h->state, h->n, b.d_u, b.d_mask, qp);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? QS_OK : pfail(p, QS_ERR_CUDA, cudaGetErrorString(e));
}

qs_status run_rank_ops(qs_plan p);

qs_status run_step(qs_plan p, const Step& st, const RunParams& rp) {
  if (st.kind == 2) return run_dm_block(p, p->dm_blocks[st.gate], rp);
  if (st.kind == 5) return run_rank_ops(p);
  return run_single(p, p->gates[st.gate], rp, st.gate);
}

// The gates of a fixed-rank plan on every member (enqueued on h->stream, so
// they can be captured): unitaries on all columns (dead ones are zero),
// noisy gates as the averaged channel built on the device from the run's e
// (or the members' own), expansion, Gram matrices, eigensolver, projection.
qs_status run_rank_ops(qs_plan p) {
  qs_ctx* h = p->h;
  const int members = h->batch * h->rank;
  bool real = (p->rank_variant >> 2) & 1;
  const bool member_e = (p->rank_variant >> 1) & 1;
  const int normalize = p->rank_variant & 1;
  const size_t esz = h->esize / 2;
  cudaError_t e = cudaSuccess;
  for (const RankOp& op : p->rank_ops) {
    const qs_gate& g = p->gates[op.gate].g;
    if (!op.real) real = false;
    if (op.kind == 0) {
      // QS_FLIP_PER_MEMBER: every column's own index (its member's marked item)
      e = launch_phase_flip(h, h->state, h->n, members, g.index, g.kind == QS_FLIP_PER_MEMBER ? h->m_marked : nullptr);
    } else if (op.kind == 1) {
      e = launch_apply_1q(h, h->state, h->n, members, g.targets[0], g.U, nullptr);
    } else {
      const Targets tg = make_targets(h->n, g.targets, g.k);
      const void* mat = static_cast<const char*>(p->d_rank_mats) + op.mat_off * esz;
      if (op.kind == 2) {
        e = launch_apply_diag(h, h->state, h->n, members, tg, mat, false, op.mask);
      } else if (op.kind == 3) {
        e = launch_apply_kq(h, h->state, h->n, members, tg, mat, false, op.real);
      } else {
        KrausGate kg{};
        for (int i = 0; i < 32; ++i) kg.U[i] = g.U[i];
        kg.k = g.k;
        kg.noise = g.noise;
        kg.e_member = member_e ? h->m_e : nullptr;
        kg.e_run = &p->d_run->e;
        const int K = kraus_count(g.k, g.noise);
        e = launch_kraus_expand_gate(h, tg, real, kg, h->rank);
        if (e == cudaSuccess) e = launch_gram(h, real, std::min(kMaxGramDim, K * h->rank));
        if (e == cudaSuccess) e = launch_eig_truncate(h, 0, normalize);
        if (e == cudaSuccess) e = launch_project(h, real, K, p->rank_kmax);
      }
    }
    if (e != cudaSuccess) return pfail(p, QS_ERR_CUDA, std::string("fixed-rank plan: ") + cudaGetErrorString(e));
  }
  return QS_OK;
}

// Host mirror of a fixed-rank run: column counts (keep = min(r_b, K m_b) per
// channel) and whether the factor is still real.
void advance_rank_mirror(qs_plan p) {
  qs_ctx* h = p->h;
  for (const RankOp& op : p->rank_ops) {
    if (!op.real) h->real_factor = false;
    if (op.kind != 4) continue;
    const qs_gate& g = p->gates[op.gate].g;
    const int K = kraus_count(g.k, g.noise);
    for (int b = 0; b < h->batch; ++b) h->m_cols[b] = std::min(h->m_rank[b], K * h->m_cols[b]);
  }
  h->cols = *std::max_element(h->m_cols.begin(), h->m_cols.end());
}

qs_status run_single(qs_plan p, const PGate& g, const RunParams& rp, int pos) {
  qs_ctx* h = p->h;
  if (g.g.kind == QS_GATE_FLIP) return qs_apply_phase_flip(h, g.g.index);
  if (g.g.kind == QS_FLIP_PER_MEMBER) {
    cudaError_t e = launch_phase_flip(h, h->state, h->n, h->batch, 0, h->m_marked);
    return e == cudaSuccess ? QS_OK : pfail(p, QS_ERR_CUDA, cudaGetErrorString(e));
  }
  if (g.g.noisy)
    return qs_apply_noisy_gate(h, g.g.targets, g.g.k, g.g.U, (qs_noise)g.g.noise, rp.e, rp.seed,
                               rp.gate_id0 + (uint64_t)pos);
  return qs_apply_gate(h, g.g.targets, g.g.k, g.g.U);
}

// Enqueue one run.  synth: the first pass creates the start state (1: one
// basis state, 2: per-member basis states); fid: the last pass also reduces
// the fidelity with the stored reference into h->small (kSmallOut).
qs_status enqueue_run(qs_plan p, cudaStream_t s, int synth, int fid) {
  qs_ctx* h = p->h;
  cudaStream_t saved = h->stream;
  h->stream = s;
  size_t ev = 0;
  cudaStreamCaptureStatus capturing = cudaStreamCaptureStatusNone;
  if (p->timing) cudaStreamIsCapturing(s, &capturing);
  auto mark = [&](int kind) {
    if (!p->timing) return;
    // under stream capture an external record becomes an event-record node;
    // eager runs (plans with single-gate steps) record plainly
    if (capturing == cudaStreamCaptureStatusActive)
      cudaEventRecordWithFlags(p->events[ev], s, cudaEventRecordExternal);
    else
      cudaEventRecord(p->events[ev], s);
    if (ev > 0) p->event_kinds[ev - 1] = kind;
    ++ev;
  };
  mark(-1);
  const bool f32 = h->dtype == QS_C64;
  for (size_t i = 0; i < p->steps.size(); ++i) {
    const Step& st = p->steps[i];
    if (st.kind == 0) {
      const PassPlan& P = p->passes[st.pass];
      const int sy = i == 0 ? synth : 0;
      const int fd = (i + 1 == p->steps.size()) ? fid : 0;
      cudaError_t e = f32 ? launch_precompute<float>(p, P, s) : launch_precompute<double>(p, P, s);
      mark(0);
      if (e == cudaSuccess) e = f32 ? launch_pass_kernel<float>(p, P, s, sy, fd) : launch_pass_kernel<double>(p, P, s, sy, fd);
      mark(P.high ? 2 : 1);
      if (e == cudaSuccess && fd) {
        k_fid_finalize<<<(h->batch + 7) / 8, 256, 0, s>>>(p->d_fid, h->batch, fid_slots(p, P), h->small + kSmallOutIndex);
        e = cudaGetLastError();
      }
      if (e != cudaSuccess) { h->stream = saved; return pfail(p, QS_ERR_CUDA, std::string("fused pass: ") + cudaGetErrorString(e)); }
    } else {
      qs_status r = run_step(p, st, *p->h_run);
      mark(st.kind == 2 ? 4 : 3);
      if (r != QS_OK) { h->stream = saved; return r; }
    }
  }
  h->stream = saved;
  return QS_OK;
}

bool fusable_start(qs_plan p) { return !p->steps.empty() && p->steps[0].kind == 0; }
bool fusable_end(qs_plan p) { return !p->steps.empty() && p->steps.back().kind == 0; }

// One run of the plan (graph replay when every step is a fused pass).
qs_status run_plan(qs_plan p, double e, uint64_t seed, uint64_t gate_id0, int want_fid) {
  qs_ctx* h = p->h;
  if (!(e >= 0.0) || !std::isfinite(e)) return pfail(p, QS_ERR_INVALID_ARG, "e must be finite and >= 0");
  for (const PGate& g : p->gates)
    if (g.g.kind == QS_FLIP_PER_MEMBER && !h->member_marked)
      return pfail(p, QS_ERR_INVALID_ARG, "per-member flips need marked indices (qs_set_member_noise)");
  // a pending basis start is synthesised by the first pass when there is one
  int synth = 0;
  if (h->pending) {
    if (fusable_start(p)) {
      synth = h->pending;
    } else {
      qs_status st = materialize_basis(h);
      if (st != QS_OK) return st;
    }
  }
  const int fid = want_fid && fusable_end(p) ? 1 : 0;
  // the pinned run block may still be read by an earlier launch of the graph
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return pfail(p, QS_ERR_CUDA, "stream sync");
  p->stable = two_shear_safe(p->gates, h->member_noise ? h->m_e_max : e) ? 0 : 1;
  if (h->mode == QS_FIXED_RANK) {
    p->rank_variant = (h->real_factor ? 4 : 0) | (h->member_noise ? 2 : 0) | (h->normalize ? 1 : 0);
    p->rank_kmax = *std::max_element(h->m_rank.begin(), h->m_rank.end());
  }
  p->h_run->e = e;
  p->h_run->seed = seed;
  p->h_run->gate_id0 = gate_id0;
  p->h_run->traj0 = h->traj_offset;
  p->h_run->basis = h->pending_x;
  // the run owns the start state from here on: later steps (single gates)
  // must not write the basis state again
  if (synth) h->pending = 0;
  // fused passes and fixed-rank plans replay as graphs; other single steps run eagerly
  const bool has_single = std::any_of(p->steps.begin(), p->steps.end(),
                                      [](const Step& s) { return s.kind != 0 && s.kind != 5; });
  qs_status st = QS_OK;
  if (has_single) {
    if (cudaMemcpyAsync(p->d_run, p->h_run, sizeof(RunParams), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
      return pfail(p, QS_ERR_CUDA, "run params copy");
    st = enqueue_run(p, h->stream, synth, fid);
  } else {
    const int v = h->mode == QS_FIXED_RANK ? p->rank_variant : p->stable * 6 + synth * 2 + fid;
    if (p->exec[v] && (p->graph_member_noise[v] != h->member_noise || p->graph_member_marked[v] != h->member_marked ||
                       p->graph_timing[v] != p->timing || p->graph_wait_polls[v] != h->wait_polls ||
                       p->graph_kmax[v] != p->rank_kmax)) {
      cudaGraphExecDestroy(p->exec[v]);
      p->exec[v] = nullptr;
    }
    if (!p->exec[v]) {
      cudaStream_t cs;
      if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return pfail(p, QS_ERR_CUDA, "capture stream");
      cudaGraph_t graph;
      cudaError_t e1 = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e1 == cudaSuccess) e1 = cudaMemcpyAsync(p->d_run, p->h_run, sizeof(RunParams), cudaMemcpyHostToDevice, cs);
      qs_status cst = e1 == cudaSuccess ? enqueue_run(p, cs, synth, fid) : QS_ERR_CUDA;
      cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
      cudaStreamDestroy(cs);
      if (cst != QS_OK) return cst;
      if (e1 != cudaSuccess || e2 != cudaSuccess) return pfail(p, QS_ERR_CUDA, "graph capture");
      cudaError_t e3 = cudaGraphInstantiate(&p->exec[v], graph, 0);
      cudaGraphDestroy(graph);
      if (e3 != cudaSuccess) { p->exec[v] = nullptr; return pfail(p, QS_ERR_CUDA, "graph instantiate"); }
      p->graph_member_noise[v] = h->member_noise;
      p->graph_member_marked[v] = h->member_marked;
      p->graph_timing[v] = p->timing;
      p->graph_wait_polls[v] = h->wait_polls;
      p->graph_kmax[v] = p->rank_kmax;
    }
    if (cudaGraphLaunch(p->exec[v], h->stream) != cudaSuccess) return pfail(p, QS_ERR_CUDA, "graph launch");
  }
  if (st == QS_OK && h->mode == QS_FIXED_RANK) advance_rank_mirror(p);
  return st;
}

// Fused passes of a state-vector plan (window width p->m) for the gates in
// rem, in order; a gate no pass can hold becomes a single step.
void plan_passes(qs_plan p, std::vector<int> rem) {
  qs_ctx* h = p->h;
  const bool fuse = h->mode == QS_STATEVEC && h->n >= p->m;
  while (!rem.empty()) {
    if (fuse) {
      PassPlan P;
      std::vector<char> absorbed(rem.size(), 0);
      bool built = false;
      for (size_t budget = kMaxOps; budget >= 4 && !built; budget /= 2) {
        P = PassPlan();
        std::fill(absorbed.begin(), absorbed.end(), 0);
        // a high window starts at or above the columns of a tile
        const int colb = p->m == kWin ? p->colb : wide_colb(p->m);
        if (!build_pass(p->gates, rem, h->n, colb, (uint64_t)h->batch, budget, p->m, &P, &absorbed)) break;
        built = segment_pass(&P);
        if (built) P.prog = choose_prog(P);
      }
      if (built) {
        bool any = false;
        for (char c : absorbed) any |= c != 0;
        if (any) {
          p->passes.push_back(P);
          p->steps.push_back(Step{0, (int)p->passes.size() - 1, -1});
          std::vector<int> next;
          for (size_t i = 0; i < rem.size(); ++i) if (!absorbed[i]) next.push_back(rem[i]);
          rem.swap(next);
          continue;
        }
      }
    }
    p->steps.push_back(Step{1, -1, rem[0]});
    rem.erase(rem.begin());
  }
}

// Device copies of the passes' op lists, their tensor maps, and the buffers
// every pass shares: one parameter block and one out-factor table (a pass's
// precompute runs on the same stream right before the pass itself) and the
// fused-fidelity partials.
qs_status alloc_passes(qs_plan p) {
  qs_ctx* h = p->h;
  qs_status st = QS_OK;
  size_t params_bytes = 16, alpha_bytes = 0;
  for (auto& P : p->passes) {
    if (st != QS_OK) break;
    st = upload(p, &P.d_ops, P.ops);
    if (st == QS_OK) st = upload(p, &P.d_outs, P.outs);
    if (st == QS_OK) st = upload(p, &P.d_prods, P.prods);
    if (st == QS_OK) st = upload(p, &P.d_contribs, P.contribs);
    if (st == QS_OK) {
      params_bytes = std::max(params_bytes, (size_t)P.stride * h->batch * (h->esize / 2));
      // out factors of every tile: members x 2^(n-m) tile values x (m + 1) complex
      if (P.out_start[P.m + 1] > 0)
        alpha_bytes = std::max(alpha_bytes, (((size_t)h->batch * (P.m + 1)) << (h->n - P.m)) * h->esize);
    }
    if (st == QS_OK && P.high) st = make_tmap(p, &P, P.colb, &P.tmap);
    if (st == QS_OK && P.high && h->esize == 8 && P.m == kWin) st = make_tmap(p, &P, 2, &P.tmap4);
  }
  // the most fidelity partials any configuration writes: 2^(n-10) per member
  const size_t fid_slots_max = (size_t)1 << (h->n - kWin);
  if (st == QS_OK && !p->passes.empty()) {
    if (cudaMalloc(&p->d_params, params_bytes) != cudaSuccess) st = pfail(p, QS_ERR_OUT_OF_MEMORY, "plan params");
    if (st == QS_OK && alpha_bytes && cudaMalloc(&p->d_alpha, alpha_bytes) != cudaSuccess)
      st = pfail(p, QS_ERR_OUT_OF_MEMORY, "plan out factors");
    for (auto& P : p->passes) {
      P.d_params = p->d_params;
      P.d_alpha = P.out_start[P.m + 1] > 0 ? p->d_alpha : nullptr;
    }
  }
  if (st == QS_OK && !p->passes.empty() &&
      cudaMalloc((void**)&p->d_fid, 2 * fid_slots_max * h->batch * sizeof(double)) != cudaSuccess)
    st = pfail(p, QS_ERR_OUT_OF_MEMORY, "fidelity partials");
  return st;
}

void free_passes(qs_plan p) {
  for (auto& P : p->passes) {
    void* ptrs[] = {P.d_ops, P.d_outs, P.d_prods, P.d_contribs};
    for (void* x : ptrs) if (x) cudaFree(x);
  }
  p->passes.clear();
  if (p->d_params) cudaFree(p->d_params);
  if (p->d_alpha) cudaFree(p->d_alpha);
  if (p->d_fid) cudaFree(p->d_fid);
  p->d_params = p->d_alpha = nullptr;
  p->d_fid = nullptr;
}

// timing slots (precompute + pass, or one single step) and kernels of one run
// (the out-factor table is timed with the precompute)
void count_launches(qs_plan p) {
  p->launches = 0;
  for (const Step& s : p->steps) p->launches += s.kind == 0 ? 2 : 1;
  p->kernels = p->launches;
  for (const Step& s : p->steps)
    if (s.kind == 0 && p->passes[s.pass].d_alpha) ++p->kernels;
}

}  // namespace

extern "C" {

qs_status qs_plan_create(qs_handle h, const qs_gate* gates, int num_gates, qs_plan* out) {
  if (!h || !out || (num_gates > 0 && !gates) || num_gates < 0) return QS_ERR_INVALID_ARG;
  *out = nullptr;
  qs_plan p = new (std::nothrow) qs_plan_s();
  if (!p) return QS_ERR_OUT_OF_MEMORY;
  p->h = h;
  for (int i = 0; i < num_gates; ++i) {
    const qs_gate& g = gates[i];
    if (g.kind == QS_GATE_FLIP) {
      if (g.index >= (1ull << h->n)) { delete p; h->err = "flip index out of range"; return QS_ERR_INVALID_ARG; }
    } else if (g.kind == QS_FLIP_PER_MEMBER) {
      if (h->mode == QS_DENSITY) { delete p; h->err = "per-member flips need STATEVEC or FIXED_RANK"; return QS_ERR_NOT_SUPPORTED; }
    } else if (g.kind == QS_GATE_DENSE) {
      if (g.k < 1 || g.k > 2) { delete p; h->err = "plan gates must have k = 1 or 2"; return QS_ERR_INVALID_ARG; }
      for (int j = 0; j < g.k; ++j) {
        if (g.targets[j] < 0 || g.targets[j] >= h->n) { delete p; h->err = "target out of range"; return QS_ERR_INVALID_ARG; }
        for (int q = 0; q < j; ++q)
          if (g.targets[q] == g.targets[j]) { delete p; h->err = "duplicate target"; return QS_ERR_INVALID_ARG; }
      }
      if (g.noisy && g.noise != QS_NOISE_ROTATION && g.noise != QS_NOISE_PHASE) { delete p; h->err = "bad noise kind"; return QS_ERR_INVALID_ARG; }
    } else {
      delete p;
      h->err = "bad gate kind";
      return QS_ERR_INVALID_ARG;
    }
    p->gates.push_back(classify(g, h->n));
  }
  p->colb = h->dtype == QS_C64 ? 3 : 2;
  // default configurations: the fastest measured on the noisy QFT, n = 20
  // (12 warps with one buffer; two high-window blocks per SM)
  if (h->dtype == QS_C64) { p->low_cfg = 2; p->high_cfg = 1; }
  // fused passes use 32-bit member-local offsets
  std::vector<int> rem;
  for (int i = 0; i < num_gates; ++i) rem.push_back(i);
  std::vector<std::vector<int>> dm_groups;
  std::vector<double> rank_mats;                         // matrices of kinds 2, 3 (doubles, interleaved)
  if (h->mode == QS_FIXED_RANK) {
    // every gate on every member with launch shapes fixed here; the whole
    // circuit replays as one graph
    for (int i : rem) {
      const PGate& g = p->gates[i];
      RankOp op{};
      op.gate = i;
      if (g.g.kind == QS_GATE_FLIP || g.g.kind == QS_FLIP_PER_MEMBER) {
        op.kind = 0;
      } else {
        const int d = 1 << g.g.k;
        for (const auto& v : g.U) if (v.imag() != 0.0) op.real = false;
        if (g.g.noisy) {
          op.kind = 4;
          if (kraus_count(g.g.k, g.g.noise) * h->rank > kMaxGramDim) {
            delete p;
            h->err = "Kraus count times rank exceeds the Gram-matrix limit of 32";
            return QS_ERR_NOT_SUPPORTED;
          }
        } else if (g.g.k == 1 && !is_diag(g.U, 2)) {
          op.kind = 1;
        } else if (is_diag(g.U, d)) {
          op.kind = 2;
          op.mat_off = rank_mats.size() / 2;
          for (int l = 0; l < d; ++l) {
            const cd f = g.U[(size_t)l * d + l];
            rank_mats.push_back(f.real());
            rank_mats.push_back(f.imag());
            if (f != cd(1.0, 0.0)) op.mask |= 1u << l;
          }
          if (!op.mask) continue;                         // the identity
        } else {
          op.kind = 3;
          op.mat_off = rank_mats.size() / 2;
          for (const auto& v : g.U) { rank_mats.push_back(v.real()); rank_mats.push_back(v.imag()); }
        }
      }
      p->rank_ops.push_back(op);
    }
    p->steps.push_back(Step{5, -1, -1});
    rem.clear();
  }
  if (h->mode == QS_DENSITY) {
    // runs of diagonal channels become one sweep each (k_dm_diag_block)
    auto dm_diag = [&](const PGate& g) {
      if (g.g.kind == QS_GATE_FLIP) return true;
      if (g.g.kind != QS_GATE_DENSE || !g.diag) return false;
      return !g.g.noisy || g.g.noise == QS_NOISE_PHASE;
    };
    std::vector<int> cur;
    int noisy = 0;
    auto close = [&]() {
      if (cur.empty()) return;
      dm_groups.push_back(cur);
      p->steps.push_back(Step{2, -1, (int)dm_groups.size() - 1});
      cur.clear();
      noisy = 0;
    };
    for (int i : rem) {
      const PGate& g = p->gates[i];
      if (dm_diag(g)) {
        if (g.g.kind == QS_GATE_DENSE && g.g.noisy && noisy == 31) close();   // bit 31 of the masks: see kDmTrivial
        cur.push_back(i);
        if (g.g.kind == QS_GATE_DENSE && g.g.noisy) ++noisy;
      } else {
        close();
        p->steps.push_back(Step{1, -1, i});
      }
    }
    close();
    rem.clear();
  }
  plan_passes(p, rem);
  std::vector<DGate> dg(p->gates.size());
  for (size_t i = 0; i < p->gates.size(); ++i) {
    const qs_gate& g = p->gates[i].g;
    DGate x{};
    for (int q = 0; q < 32; ++q) x.U[q] = g.U[q];
    x.k = g.k;
    x.noisy = g.noisy;
    x.noise = g.noise;
    x.gate_pos = i;
    dg[i] = x;
  }
  qs_status st = upload(p, &p->d_gates, dg);
  for (const auto& grp : dm_groups) {
    if (st != QS_OK) break;
    const uint64_t N = 1ull << h->n;
    std::vector<double2> u(N, make_double2(1.0, 0.0));
    std::vector<uint32_t> mask(N, 0u);
    int c = 0;
    for (int gi : grp) {
      const PGate& g = p->gates[gi];
      if (g.g.kind == QS_GATE_FLIP) {
        if (g.g.index < N) u[g.g.index] = make_double2(-u[g.g.index].x, -u[g.g.index].y);
        continue;
      }
      const int k = g.g.k, d = 1 << k;
      for (uint64_t x = 0; x < N; ++x) {
        int l = 0;
        for (int j = 0; j < k; ++j) l |= (int)((x >> g.g.targets[j]) & 1) << j;
        const cd f = g.U[(size_t)l * d + l];
        const double2 a = u[x];
        u[x] = make_double2(a.x * f.real() - a.y * f.imag(), a.x * f.imag() + a.y * f.real());
        if (g.g.noisy && l == d - 1) mask[x] |= 1u << c;
      }
      if (g.g.noisy) ++c;
    }
    for (uint64_t x = 0; x < N; ++x)
      if (mask[x] == 0 && u[x].x == 1.0 && u[x].y == 0.0) mask[x] = kDmTrivial;
    DmBlock b;
    b.noisy = c;
    if (h->dtype == QS_C64) {
      std::vector<float2> uf(u.size());
      for (size_t i = 0; i < u.size(); ++i) uf[i] = make_float2((float)u[i].x, (float)u[i].y);
      st = upload(p, &b.d_uf, uf);
    } else {
      st = upload(p, &b.d_u, u);
    }
    if (st == QS_OK) st = upload(p, &b.d_mask, mask);
    p->dm_blocks.push_back(b);
  }
  if (st == QS_OK && !rank_mats.empty()) {
    if (h->dtype == QS_C64) {
      std::vector<float> f(rank_mats.begin(), rank_mats.end());
      st = upload(p, reinterpret_cast<float**>(&p->d_rank_mats), f);
    } else {
      st = upload(p, reinterpret_cast<double**>(&p->d_rank_mats), rank_mats);
    }
  }
  if (st == QS_OK) st = alloc_passes(p);
  if (st == QS_OK && cudaMalloc((void**)&p->d_run, sizeof(RunParams)) != cudaSuccess) st = pfail(p, QS_ERR_OUT_OF_MEMORY, "run params");
  if (st == QS_OK && cudaMallocHost((void**)&p->h_run, sizeof(RunParams)) != cudaSuccess) st = pfail(p, QS_ERR_OUT_OF_MEMORY, "run params");
  if (st == QS_OK && set_smem_attrs(h->esize) != cudaSuccess) st = pfail(p, QS_ERR_CUDA, "shared memory attribute");
  if (st != QS_OK) { qs_plan_destroy(p); return st; }
  count_launches(p);
  if (!p->rank_ops.empty()) {
    p->kernels -= 1;
    for (const RankOp& op : p->rank_ops) p->kernels += op.kind == 4 ? 5 : 1;   // channel: expand, Gram x 2, eig, project
    if (rank_kernel_attributes() != cudaSuccess) { qs_plan_destroy(p); return QS_ERR_CUDA; }
  }
  *out = p;
  return QS_OK;
}

qs_status qs_plan_run(qs_plan p, double e, uint64_t seed, uint64_t gate_id0) {
  if (!p) return QS_ERR_INVALID_ARG;
  return run_plan(p, e, seed, gate_id0, 0);
}

qs_status qs_plan_run_fidelity(qs_plan p, double e, uint64_t seed, uint64_t gate_id0, double* out) {
  if (!p || !out) return QS_ERR_INVALID_ARG;
  qs_ctx* h = p->h;
  if (h->mode != QS_STATEVEC) return pfail(p, QS_ERR_NOT_SUPPORTED, "fused fidelity needs STATEVEC");
  if (!h->has_ref) return pfail(p, QS_ERR_INVALID_ARG, "no stored reference (qs_set_reference)");
  qs_status st = run_plan(p, e, seed, gate_id0, 1);
  if (st != QS_OK) return st;
  if (!fusable_end(p)) return qs_fidelity_stored(h, out);
  return read_results(h, out, h->batch);
}

qs_status qs_plan_profile(qs_plan p, int reps, double e, uint64_t seed, uint64_t gate_id0, double* ms,
                          int* kinds, int cap, int* count) {
  if (!p || reps < 1 || !ms || !kinds || !count) return QS_ERR_INVALID_ARG;
  qs_ctx* h = p->h;
  // a pending basis start is created by the first pass of every profiled run,
  // as plan runs do (the runs overwrite the state, so each recreates it)
  int synth = 0;
  if (h->pending) {
    if (fusable_start(p)) {
      synth = h->pending;
    } else {
      qs_status st = materialize_basis(h);
      if (st != QS_OK) return st;
    }
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return pfail(p, QS_ERR_CUDA, "stream sync");
  p->stable = two_shear_safe(p->gates, h->member_noise ? h->m_e_max : e) ? 0 : 1;
  if (h->mode == QS_FIXED_RANK) {
    p->rank_variant = (h->real_factor ? 4 : 0) | (h->member_noise ? 2 : 0) | (h->normalize ? 1 : 0);
    p->rank_kmax = *std::max_element(h->m_rank.begin(), h->m_rank.end());
  }
  p->h_run->e = e;
  p->h_run->seed = seed;
  p->h_run->gate_id0 = gate_id0;
  p->h_run->traj0 = h->traj_offset;
  p->h_run->basis = h->pending_x;
  if (cudaMemcpyAsync(p->d_run, p->h_run, sizeof(RunParams), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
    return pfail(p, QS_ERR_CUDA, "run params copy");
  int nl = 0;
  for (const Step& st : p->steps) nl += st.kind == 0 ? 2 : 1;
  std::vector<cudaEvent_t> ev((size_t)nl * reps + 1);
  for (auto& x : ev) if (cudaEventCreate(&x) != cudaSuccess) return pfail(p, QS_ERR_CUDA, "event create");
  std::vector<int> kind(nl);
  size_t k = 0;
  qs_status result = QS_OK;
  cudaEventRecord(ev[k++], h->stream);
  for (int r = 0; r < reps && result == QS_OK; ++r) {
    int li = 0;
    for (const Step& st : p->steps) {
      if (st.kind == 0) {
        const PassPlan& P = p->passes[st.pass];
        const bool f32 = h->dtype == QS_C64;
        const int sy = li == 0 ? synth : 0;
        cudaError_t x = f32 ? launch_precompute<float>(p, P, h->stream) : launch_precompute<double>(p, P, h->stream);
        cudaEventRecord(ev[k++], h->stream);
        kind[li++] = 0;
        if (x == cudaSuccess) x = f32 ? launch_pass_kernel<float>(p, P, h->stream, sy, 0) : launch_pass_kernel<double>(p, P, h->stream, sy, 0);
        cudaEventRecord(ev[k++], h->stream);
        kind[li++] = P.high ? 2 : 1;
        if (x != cudaSuccess) { result = pfail(p, QS_ERR_CUDA, cudaGetErrorString(x)); break; }
      } else {
        result = run_step(p, st, *p->h_run);
        cudaEventRecord(ev[k++], h->stream);
        kind[li++] = st.kind == 2 ? 4 : 3;
        if (result != QS_OK) break;
      }
    }
  }
  if (cudaEventSynchronize(ev[k - 1]) != cudaSuccess && result == QS_OK) result = pfail(p, QS_ERR_CUDA, "profile sync");
  if (synth) h->pending = 0;                           // the runs own the state now
  if (result == QS_OK) {
    for (int i = 0; i < nl && i < cap; ++i) {
      double acc = 0.0;
      for (int r = 0; r < reps; ++r) {
        float t = 0.f;
        const size_t a = (size_t)r * nl + i;
        cudaEventElapsedTime(&t, ev[a], ev[a + 1]);
        acc += t;
      }
      ms[i] = acc / reps;
      kinds[i] = kind[i];
    }
    *count = nl;
  }
  for (auto& x : ev) cudaEventDestroy(x);
  return result;
}

namespace {
void drop_graphs(qs_plan p) {
  for (auto& x : p->exec)
    if (x) { cudaGraphExecDestroy(x); x = nullptr; }
}
}  // namespace

qs_status qs_plan_configs(qs_plan p, int* low_count, int* high_count) {
  if (!p || !low_count || !high_count) return QS_ERR_INVALID_ARG;
  *low_count = num_low_cfgs(p->h->esize, p->m);
  *high_count = num_high_cfgs(p->h->esize, p->m);
  return QS_OK;
}

qs_status qs_plan_set_config(qs_plan p, int low_cfg, int high_cfg) {
  if (!p) return QS_ERR_INVALID_ARG;
  if (low_cfg < 0 || low_cfg >= num_low_cfgs(p->h->esize, p->m) || high_cfg < 0 ||
      high_cfg >= num_high_cfgs(p->h->esize, p->m))
    return pfail(p, QS_ERR_INVALID_ARG, "kernel configuration out of range");
  if (low_cfg != p->low_cfg || high_cfg != p->high_cfg) {
    // graphs hold the old kernels; wait for runs that may still use them
    if (cudaStreamSynchronize(p->h->stream) != cudaSuccess) return pfail(p, QS_ERR_CUDA, "stream sync");
    drop_graphs(p);
    p->low_cfg = low_cfg;
    p->high_cfg = high_cfg;
  }
  return QS_OK;
}

qs_status qs_plan_get_config(qs_plan p, int* low_cfg, int* high_cfg) {
  if (!p || !low_cfg || !high_cfg) return QS_ERR_INVALID_ARG;
  *low_cfg = p->low_cfg;
  *high_cfg = p->high_cfg;
  return QS_OK;
}

qs_status qs_plan_set_window(qs_plan p, int m) {
  if (!p) return QS_ERR_INVALID_ARG;
  qs_ctx* h = p->h;
  if (m != 10 && m != 11 && m != 12) return pfail(p, QS_ERR_INVALID_ARG, "window width must be 10, 11 or 12");
  if (m == p->m) return QS_OK;
  if (h->mode != QS_STATEVEC || h->dtype != QS_C64)
    return pfail(p, QS_ERR_NOT_SUPPORTED, "windows of 11 or 12 qubits need a STATEVEC complex64 handle");
  if (m != kWin && h->n > 32) return pfail(p, QS_ERR_NOT_SUPPORTED, "windows of 11 or 12 qubits need n <= 32");
  // graphs and a run in flight hold the old passes' buffers
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return pfail(p, QS_ERR_CUDA, "stream sync");
  drop_graphs(p);
  free_passes(p);
  p->steps.clear();
  p->m = m;
  if (m == kWin) { p->low_cfg = 2; p->high_cfg = 1; }   // the defaults of qs_plan_create
  else { p->low_cfg = 0; p->high_cfg = 0; }
  std::vector<int> rem(p->gates.size());
  for (size_t i = 0; i < rem.size(); ++i) rem[i] = (int)i;
  plan_passes(p, rem);
  qs_status st = alloc_passes(p);
  if (st != QS_OK) {
    // leave a plan that runs nothing rather than one with missing buffers
    free_passes(p);
    p->steps.clear();
    count_launches(p);
    return st;
  }
  count_launches(p);
  if (!p->events.empty()) {
    // timing slots follow the new steps
    for (auto& ev : p->events) cudaEventDestroy(ev);
    p->events.clear();
    p->event_kinds.clear();
    if (p->timing) {
      p->timing = false;
      st = qs_plan_set_timing(p, 1);
    }
  }
  return st;
}

qs_status qs_plan_get_window(qs_plan p, int* m) {
  if (!p || !m) return QS_ERR_INVALID_ARG;
  *m = p->m;
  return QS_OK;
}

namespace {
// Best low and high configurations of the plan's current window width: the
// time of the low and high passes of one run under each, averaged over reps
// profiled runs; total = the whole run under the chosen pair.
qs_status tune_configs(qs_plan p, int reps, double e, uint64_t seed, int* bl, int* bh, double* low_best,
                       double* high_best, double* total) {
  const int nl = num_low_cfgs(p->h->esize, p->m), nh = num_high_cfgs(p->h->esize, p->m);
  const int ncfg = std::max(nl, nh);
  std::vector<double> low_ms(ncfg, -1.0), high_ms(ncfg, -1.0), other_ms(ncfg, 0.0);
  std::vector<double> ms((size_t)std::max(p->launches, 1));
  std::vector<int> kinds(ms.size());
  for (int c = 0; c < ncfg; ++c) {
    qs_status st = qs_plan_set_config(p, std::min(c, nl - 1), std::min(c, nh - 1));
    if (st != QS_OK) return st;
    int count = 0;
    const int pend = p->h->pending;
    const uint64_t pend_x = p->h->pending_x;
    // one untimed run first: a kernel's first launch also loads its module
    st = qs_plan_profile(p, 1, e, seed, 0, ms.data(), kinds.data(), (int)ms.size(), &count);
    if (st != QS_OK) return st;
    p->h->pending = pend;                              // each profile starts from the pending start
    p->h->pending_x = pend_x;
    st = qs_plan_profile(p, reps, e, seed, 0, ms.data(), kinds.data(), (int)ms.size(), &count);
    p->h->pending = pend;
    p->h->pending_x = pend_x;
    if (st != QS_OK) return st;
    double lo = 0.0, hi = 0.0, other = 0.0;
    bool has_lo = false, has_hi = false;
    for (int i = 0; i < count && i < (int)ms.size(); ++i) {
      if (kinds[i] == 1) { lo += ms[i]; has_lo = true; }
      else if (kinds[i] == 2) { hi += ms[i]; has_hi = true; }
      else other += ms[i];
    }
    if (has_lo && c < nl) low_ms[c] = lo;
    if (has_hi && c < nh) high_ms[c] = hi;
    other_ms[c] = other;
  }
  auto best = [](const std::vector<double>& v, int n) {
    int b = 0;
    for (int c = 1; c < n; ++c)
      if (v[c] >= 0.0 && (v[b] < 0.0 || v[c] < v[b])) b = c;
    return b;
  };
  *bl = best(low_ms, nl);
  *bh = best(high_ms, nh);
  *low_best = low_ms[*bl];
  *high_best = high_ms[*bh];
  // precompute and single steps do not depend on the configuration: their
  // time averaged over the configurations profiled
  double other = 0.0;
  for (int c = 0; c < ncfg; ++c) other += other_ms[c];
  *total = std::max(0.0, *low_best) + std::max(0.0, *high_best) + other / ncfg;
  return QS_OK;
}
}  // namespace

qs_status qs_plan_autotune(qs_plan p, int reps, double e, uint64_t seed, double* best_ms) {
  if (!p || reps < 1) return QS_ERR_INVALID_ARG;
  qs_ctx* h = p->h;
  // a pending basis start is created by every profiled run and is still
  // pending afterwards (see qs_plan_profile)
  const int pend = h->pending;
  const uint64_t pend_x = h->pending_x;
  struct Restore {
    qs_ctx* h; int pend; uint64_t x;
    ~Restore() { if (pend) { h->pending = pend; h->pending_x = x; } }
  } restore{h, pend, pend_x};
  // window widths to try: 10, and 11 and 12 where the handle allows them
  std::vector<int> widths = {p->m};
  if (h->mode == QS_STATEVEC && h->dtype == QS_C64 && h->n <= 32)
    for (int m = kWin; m <= kMaxWin; ++m)
      if (m != p->m && h->n >= m) widths.push_back(m);
  int best_m = p->m, best_l = 0, best_h = 0;
  double best_total = -1.0, best_lo = -1.0, best_hi = -1.0;
  for (int m : widths) {
    qs_status st = qs_plan_set_window(p, m);
    if (st != QS_OK) return st;
    int bl = 0, bh = 0;
    double lo = 0.0, hi = 0.0, total = 0.0;
    st = tune_configs(p, reps, e, seed, &bl, &bh, &lo, &hi, &total);
    if (st != QS_OK) return st;
    if (best_total < 0.0 || total < best_total) {
      best_total = total;
      best_m = m;
      best_l = bl;
      best_h = bh;
      best_lo = lo;
      best_hi = hi;
    }
  }
  qs_status st = qs_plan_set_window(p, best_m);
  if (st != QS_OK) return st;
  if (best_ms) { best_ms[0] = best_lo; best_ms[1] = best_hi; }
  return qs_plan_set_config(p, best_l, best_h);
}

qs_status qs_plan_set_timing(qs_plan p, int on) {
  if (!p) return QS_ERR_INVALID_ARG;
  if (on && p->events.empty()) {
    p->events.resize((size_t)p->launches + 1);
    p->event_kinds.assign((size_t)p->launches, 0);
    for (auto& e : p->events)
      if (cudaEventCreate(&e) != cudaSuccess) return pfail(p, QS_ERR_CUDA, "event create");
  }
  p->timing = on != 0;
  return QS_OK;
}

qs_status qs_plan_last_times(qs_plan p, double* ms, int* kinds, int cap, int* count) {
  if (!p || !ms || !kinds || !count) return QS_ERR_INVALID_ARG;
  if (!p->timing || p->events.empty()) return pfail(p, QS_ERR_INVALID_ARG, "timing is off");
  if (cudaEventSynchronize(p->events.back()) != cudaSuccess) return pfail(p, QS_ERR_CUDA, "event sync");
  const int nl = p->launches;
  for (int i = 0; i < nl && i < cap; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p->events[i], p->events[i + 1]) != cudaSuccess) return pfail(p, QS_ERR_CUDA, "elapsed");
    ms[i] = t;
    kinds[i] = p->event_kinds[i];
  }
  *count = nl;
  return QS_OK;
}

qs_status qs_plan_info(qs_plan p, int* passes, int* launches) {
  if (!p) return QS_ERR_INVALID_ARG;
  if (passes) *passes = (int)p->steps.size();
  if (launches) *launches = p->kernels;
  return QS_OK;
}

qs_status qs_plan_destroy(qs_plan p) {
  if (!p) return QS_ERR_INVALID_ARG;
  if (p->h) cudaStreamSynchronize(p->h->stream);
  for (auto& x : p->exec) if (x) cudaGraphExecDestroy(x);
  free_passes(p);
  if (p->d_gates) cudaFree(p->d_gates);
  for (auto& b : p->dm_blocks) {
    if (b.d_u) cudaFree(b.d_u);
    if (b.d_uf) cudaFree(b.d_uf);
    if (b.d_mask) cudaFree(b.d_mask);
  }
  if (p->d_run) cudaFree(p->d_run);
  if (p->h_run) cudaFreeHost(p->h_run);
  if (p->d_rank_mats) cudaFree(p->d_rank_mats);
  for (auto& e : p->events) cudaEventDestroy(e);
  delete p;
  return QS_OK;
}

}  // extern "C"
