// Fused window passes (device side).  See plan.cu for the planner.
//
// A pass applies a run of gates whose dense targets lie in a window of M
// qubits (M = 10, 11 or 12) to every tile of the state in one HBM read and
// one HBM write (the amplitude update of Sec. 2, with the memory dependence
// the paper describes kept inside a tile).  Each thread holds 32 amplitudes
// that differ in 5 "register" bits of the window: a one-qubit gate on a
// register bit is a butterfly over registers; an exchange through shared
// memory changes which 5 window bits are in registers.  The register bits of
// a stage are 5 consecutive window bits: stage 0 (A) the top five, stage 1
// (B) bits 0..4 and, for M > 10, stage 2 (C) bits 5..9; the other M - 5 bits
// index the thread (32 lanes x 2^(M-10) warps of a tile).
//
// Tiles stream through shared memory: while a block computes tile i, the copy
// engine fills the other buffer with tile i+1 (a 1D bulk copy per tile for
// the low window, a 2D tensor-map copy per block for the high window),
// completion tracked by mbarriers.  Every wait is bounded: on timeout the
// kernel records an error in a device status word, waits (bounded) for
// copies it still has in flight, and returns.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include <cstdint>

#include "internal.cuh"

namespace qs {
namespace fused {

constexpr int kWin = 10;                   // the default window width M
constexpr int kMaxWin = 12;                // the widest window (complex64)
constexpr int kRegBits = 5;
constexpr int kAmps = 32;
constexpr int kMaxOther = 48;
constexpr uint32_t kSpinLimit = 1u << 22;
constexpr int kStatusTimeout = 0x51;       // value written to the status word on a timed-out wait
constexpr int kMaxPassOps = 256;           // ops of one pass before segmentation
constexpr int kMaxSegs = 48;               // segments of one pass (kernel parameters)
constexpr int kMaxFlips = 64;

enum : uint8_t { OP_DENSE = 0, OP_DWIN = 1, OP_FLIP = 2, OP_FLIPM = 3, OP_EXCH = 4 };

// One planner op (host side; the kernels see segments).
struct FOp {
  uint8_t type;
  uint8_t j;          // local window bit (DENSE, DWIN)
  uint8_t real;       // DENSE: matrix is real
  uint8_t pad;
  uint32_t off;       // parameter offset (R units) in the member block
  uint64_t index;     // FLIP: member-local amplitude index
};

// A segment: gates of one register stage applied in a canonical order --
// for each register bit rj, descending (desc = 1) or ascending, the dense
// gate on rj (if in `dense`) then the phase table attached to rj (if in
// `dwin`) -- followed by `nflip` flips.  The planner only forms a segment
// when that order keeps every pair of non-commuting gates in circuit order.
struct Seg {
  uint8_t stage;      // 0 = A (registers = window bits M-5..M-1), 1 = B (0..4), 2 = C (5..9)
  uint8_t dense;
  uint8_t dwin;
  uint8_t real;
  uint8_t desc;
  uint8_t nflip;
  uint16_t flip0;
  uint32_t doff[kRegBits];
  uint32_t woff[kRegBits];
};

struct Flip {
  uint64_t index;     // member-local amplitude index
  uint32_t per_member;  // 1: the member's marked index instead
  uint32_t pad;
};

struct OutTerm {
  int32_t a;          // attach local bit, or -1
  uint32_t off;       // parameter offset of the factor
  uint64_t cmask;     // member-local out-of-window bits that must be set
};

struct PassArgs {
  int n;
  int start_stage;            // 0 = A, 1 = B
  int m;                      // window width M (the kernel's template argument)
  int win[kMaxWin];
  int nseg;
  Seg segs[kMaxSegs];         // the program (constant bank: uniform, cached)
  Flip flips[kMaxFlips];
  // out factors per member and out-of-window tile value o (2^(n-M) of them):
  // M + 1 complex, entry a = the product of the out terms attached to window
  // bit a (M: none) whose out-of-window bits are set in o, times the deferred
  // diagonal of bit a (M: the overall scale); null when the pass has none
  const void* alpha_tab;
  int param_stride;           // R units per member
  const void* params;
  const uint64_t* marked;     // per-member flip index
  uint64_t tiles;
  int tile_shift;             // log2(tiles per member)
  int* status;                // device status word
  // first pass of a run started from basis states: synthesise, do not load
  int synth;
  const uint64_t* basis;      // per-member basis index, or null: basis0
  const uint64_t* basis0;     // device word
  // last pass of a run with a fused fidelity: partials of <ref|psi>
  int fid;
  const void* ref;            // 2^n reference amplitudes
  double* fid_partials;       // [member][tile in member] complex
  // real one-qubit gates run with their diagonal factored out (see
  // butterfly_fact); the factors left at the end of the pass are applied
  // there: per member, diag_off (R units) holds ratio_j = d_j / a_j for each
  // window bit j and the overall scale prod_j a_j; -1 when the pass has none
  int diag_off;
  // 1: the real gates carry a third shear (see dense_real_reg); only the
  // interpreted kernels (PROG = 0) run with it
  int stable;
  // polls of a tile-copy wait before the pass gives up (kSpinLimit unless the
  // handle sets another); the clean-up waits of a pass that gave up always
  // take kSpinLimit
  uint32_t spin_limit;
};

// First window bit held in registers in stage S of a window of M bits.
__host__ __device__ constexpr int stage_base(int m, int s) { return s == 0 ? m - kRegBits : (s == 1 ? 0 : 5); }

// Where register r of thread t (the thread's M - 5 window bits, in
// increasing order of the bits they stand for) sits in a tile of 2^M
// amplitudes in stage S: tile_base + r tile_step, in the plain layout (as
// copied from memory) and in the padded exchange layout, which puts one pad
// slot after every 32 amplitudes, x -> x + x / 32.  Both layouts keep the
// accesses of a warp free of bank conflicts in every stage: its lanes hold
// consecutive amplitudes (stages A, C) or amplitudes 32 apart that the
// padding moves to consecutive banks (stage B).
template <int M, int S>
__device__ __forceinline__ int tile_base(int t) {
  if constexpr (S == 0) return t;
  else if constexpr (S == 1) return t << 5;
  else return (t & 31) | ((t >> 5) << 10);
}
template <int M, int S> __device__ __forceinline__ constexpr int tile_step() {
  return S == 0 ? 1 << (M - 5) : (S == 1 ? 1 : 32);
}
template <int M, int S>
__device__ __forceinline__ int pad_base(int t) {
  if constexpr (S == 0) return t + (t >> 5);
  else if constexpr (S == 1) return 33 * t;
  else return (t & 31) + 1056 * (t >> 5);
}
template <int M, int S> __device__ __forceinline__ constexpr int pad_step() {
  return S == 0 ? (1 << (M - 5)) + (1 << (M - 10)) : (S == 1 ? 1 : 33);
}
// the window bit that thread bit k stands for in stage S
template <int M, int S> __device__ __forceinline__ constexpr int thread_bit(int k) {
  return S == 0 ? k : (S == 1 ? k + 5 : (k < 5 ? k : k + 5));
}

// Run f with the stage as a compile-time constant (stage 2 exists for M > 10).
template <int M, typename F>
__device__ __forceinline__ void with_stage(int stage, F&& f) {
  if (stage == 0) {
    f(std::integral_constant<int, 0>{});
  } else if (M == kWin || stage == 1) {
    f(std::integral_constant<int, 1>{});
  } else {
    if constexpr (M > kWin) f(std::integral_constant<int, 2>{});
  }
}

// Barrier over the 32 G threads of one tile (G = 1: the warp).  Named
// barrier id + 1 (id 0 is __syncthreads).
template <int G>
__device__ __forceinline__ void group_sync(int id) {
  if constexpr (G == 1) __syncwarp();
  else asm volatile("bar.sync %0, %1;" ::"r"(id + 1), "r"(G * 32) : "memory");
}
// True on every thread of the group when it is true on any of them.
template <int G>
__device__ __forceinline__ bool group_any(int id, bool v) {
  if constexpr (G == 1) {
    return __any_sync(0xffffffffu, v);
  } else {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, %2, %3, q;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(r) : "r"((uint32_t)v), "r"(id + 1), "r"(G * 32) : "memory");
    return r != 0;
  }
}

// ---------------------------------------------------------------- async copies
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Bounded wait for the phase with the given parity: at most `limit` polls;
// false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit = kSpinLimit) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done) : "r"(a), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 1D bulk copy global -> shared, completion on `bar` (bytes % 16 == 0, both 16-B aligned)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
// 2D tensor-map copy of one box to shared memory
__device__ __forceinline__ void tma_g2s_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// bring a 128-byte line into L1 ahead of its use
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

__device__ __forceinline__ void report_timeout(int* status) {
  if (status) atomicExch(status, kStatusTimeout);
}

// ---------------------------------------------------------------- arithmetic
// One complex parameter (8- or 16-byte aligned): a single vector load.
template <typename R>
__device__ __forceinline__ cplx<R> ld_c(const R* p) { return __ldg(reinterpret_cast<const cplx<R>*>(p)); }

__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Complex products of the passes.  complex64 runs them on the packed
// two-lane FP32 pipe: f a = f.x (a.x, a.y) + f.y (-a.y, a.x) is one packed
// multiply and one packed FMA whose operands are the amplitude with its
// halves swapped and the factor's halves broadcast or negated -- operand
// forms the packed instructions take directly, so a complex product is two
// instructions and its result stays a register pair for the packed shears
// (four scalar instructions, and moves into pairs, otherwise).
template <typename R>
__device__ __forceinline__ cplx<R> pmul(cplx<R> f, cplx<R> a) {
  if constexpr (sizeof(R) == 4) {
    const float2 t = mul2(a, make_float2(f.x, f.x));
    return fma2(make_float2(a.y, a.x), make_float2(-f.y, f.y), t);
  } else {
    return cmul(f, a);
  }
}
// c + m b
template <typename R>
__device__ __forceinline__ cplx<R> pfma(cplx<R> m, cplx<R> b, cplx<R> c) {
  if constexpr (sizeof(R) == 4) {
    const float2 t = fma2(b, make_float2(m.x, m.x), c);
    return fma2(make_float2(b.y, b.x), make_float2(-m.y, m.y), t);
  } else {
    return cfma(m, b, c);
  }
}
// acc += conj(f) a
template <typename R>
__device__ __forceinline__ cplx<R> pdot(cplx<R> acc, cplx<R> f, cplx<R> a) {
  if constexpr (sizeof(R) == 4) {
    acc = fma2(a, make_float2(f.x, f.x), acc);
    return fma2(make_float2(a.y, a.x), make_float2(f.y, -f.y), acc);
  } else {
    acc.x += f.x * a.x + f.y * a.y;
    acc.y += f.x * a.y - f.y * a.x;
    return acc;
  }
}

// A real 2x2 gate [[a, b], [c, d]] written as two shears and a diagonal,
// diag(a, det / a) [[1, 0], [s1, 1]] [[1, r0], [0, 1]], r0 = b / a,
// s1 = c a / det: x0 += r0 x1, then x1 += s1 x0, each one FMA per component
// (packed two-lane for complex64) that updates its register in place.  The
// diagonal commutes with every diagonal operation of the pass; the
// precompute folds it into the next gate on the same qubit or leaves it for
// the end of the pass (PassArgs::diag_off).
template <typename R>
__device__ __forceinline__ void butterfly_fact(cplx<R>& x0, cplx<R>& x1, R r0, R s1) {
  x0.x = fma(r0, x1.x, x0.x);
  x0.y = fma(r0, x1.y, x0.y);
  x1.x = fma(s1, x0.x, x1.x);
  x1.y = fma(s1, x0.y, x1.y);
}

template <typename R, int RJ>
__device__ __forceinline__ void dense_real_reg(cplx<R> (&a)[kAmps], const R* m);
template <typename R, int RJ>
__device__ __forceinline__ void third_shear_reg(cplx<R> (&a)[kAmps], const R* m);

template <typename R, int RJ>
__device__ __forceinline__ void dense_reg(cplx<R> (&a)[kAmps], const R* m, bool real, bool stable) {
  if (real) {
    dense_real_reg<R, RJ>(a, m);
    if (stable) third_shear_reg<R, RJ>(a, m);
  } else {
    const cplx<R> u00 = ld_c(m), u01 = ld_c(m + 2), u10 = ld_c(m + 4), u11 = ld_c(m + 6);
#pragma unroll
    for (int r = 0; r < kAmps; ++r) {
      if (r & (1 << RJ)) continue;
      const cplx<R> x0 = a[r], x1 = a[r | (1 << RJ)];
      a[r] = pfma<R>(u01, x1, pmul<R>(u00, x0));
      a[r | (1 << RJ)] = pfma<R>(u11, x1, pmul<R>(u10, x0));
    }
  }
}

template <typename R, int RJ>
__device__ __forceinline__ void dense_real_reg(cplx<R> (&a)[kAmps], const R* m) {
  {
    // stored as (r0, r0, s1, s1): the broadcast pairs of the packed FMA come
    // straight from one 16-byte load (complex64)
    if constexpr (sizeof(R) == 4) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(m));
      const float2 p0 = make_float2(q.x, q.y), p1 = make_float2(q.z, q.w);
#pragma unroll
      for (int r = 0; r < kAmps; ++r) {
        if (r & (1 << RJ)) continue;
        a[r] = fma2(p0, a[r | (1 << RJ)], a[r]);
        a[r | (1 << RJ)] = fma2(p1, a[r], a[r | (1 << RJ)]);
      }
    } else {
      const R r0 = __ldg(m), s1 = __ldg(m + 2);
#pragma unroll
      for (int r = 0; r < kAmps; ++r) {
        if (r & (1 << RJ)) continue;
        butterfly_fact<R>(a[r], a[r | (1 << RJ)], r0, s1);
      }
    }
  }
}

// The third shear x0 += w x1 of the pivoted form of a real gate (stored as
// (w, w) after the first two; w = 0 for members whose gate takes the
// two-shear form).  A gate whose M00 is small against its first column (a
// bit flip, a rotation near pi) is factored as diag(d0, d1) [[1, w], [0, 1]]
// [[1, 0], [1, 1]] [[1, p], [0, 1]] with the pivot on M10, so no factor is
// large.
template <typename R, int RJ>
__device__ __forceinline__ void third_shear_reg(cplx<R> (&a)[kAmps], const R* m) {
  if constexpr (sizeof(R) == 4) {
    const float2 w = __ldg(reinterpret_cast<const float2*>(m + 4));
#pragma unroll
    for (int r = 0; r < kAmps; ++r) {
      if (r & (1 << RJ)) continue;
      a[r] = fma2(w, a[r | (1 << RJ)], a[r]);
    }
  } else {
    const R w = __ldg(m + 4);
#pragma unroll
    for (int r = 0; r < kAmps; ++r) {
      if (r & (1 << RJ)) continue;
      a[r].x = fma(w, a[r | (1 << RJ)].x, a[r].x);
      a[r].y = fma(w, a[r | (1 << RJ)].y, a[r].y);
    }
  }
}

// Multiply registers with bit RJ set by T[idx], the phase table of window
// bit SH + RJ over the bits below it: idx = tbits (the thread's window bits
// below SH) | (register bits below RJ) << SH.  SPLIT (windows above 10
// qubits): the table is stored as its two factors, 2^SH entries over the
// thread's bits then 2^RJ over the register bits (the product over a set of
// bits splits that way), so a tile reads a few hundred entries per table
// instead of up to 2^11, and the register part is the same for every lane.
// TRANS (high window): the entry (tbits, q) is stored at tbits 2^RJ + q, the
// register index fastest.  Where a thread's factors for q and q + 1 sit side
// by side (register-bit index fastest: SH = 0, SPLIT or TRANS) complex64
// reads them with one 16-byte load, half the loads of the table.
template <typename R, int RJ, int SH, bool SPLIT = false, bool TRANS = false>
__device__ __forceinline__ void dwin_reg(cplx<R> (&a)[kAmps], const R* T, int tbits) {
  constexpr int Q = 1 << RJ;
  constexpr bool kSplit = SPLIT && SH > 0;
  constexpr bool kTrans = TRANS && !kSplit && SH > 0;
  constexpr bool kPair = sizeof(R) == 4 && Q >= 2 && (SH == 0 || kSplit || kTrans);
  cplx<R> flo = mk<R>(R(1), R(0));
  if constexpr (kSplit) flo = ld_c(T + 2 * tbits);
  // the factors over q of this thread: one row of the table
  const R* row = kSplit ? T + 2 * (1 << SH) : (kTrans ? T + 2 * (tbits << RJ) : T);
  auto apply = [&](int q, cplx<R> f) {
#pragma unroll
    for (int hi = 0; hi < kAmps / (2 * Q); ++hi) {
      const int r = q | Q | (hi << (RJ + 1));
      a[r] = pmul<R>(f, a[r]);
    }
  };
  if constexpr (kPair) {
#pragma unroll
    for (int q = 0; q < Q; q += 2) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(row + 2 * q));
      cplx<R> f0 = mk<R>(v.x, v.y), f1 = mk<R>(v.z, v.w);
      if constexpr (kSplit) {
        f0 = q == 0 ? flo : pmul<R>(f0, flo);
        f1 = pmul<R>(f1, flo);
      }
      apply(q, f0);
      apply(q + 1, f1);
    }
  } else {
    // factor q multiplies the registers with bit RJ set and low bits q; each
    // factor is consumed right after its load (few live registers)
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      cplx<R> f;
      if constexpr (kSplit) {
        f = q == 0 ? flo : pmul<R>(ld_c(row + 2 * q), flo);
      } else if constexpr (kTrans) {
        f = ld_c(row + 2 * q);
      } else {
        const int idx = SH ? (tbits + (q << SH)) : q;
        f = ld_c(T + 2 * idx);
      }
      apply(q, f);
    }
  }
}

template <typename R>
__device__ __forceinline__ void flip_reg(cplx<R> (&a)[kAmps], bool match, int rw) {
#pragma unroll
  for (int r = 0; r < kAmps; ++r)
    if (match && r == rw) { a[r].x = -a[r].x; a[r].y = -a[r].y; }
}

// a[rho] *= c * prod_{r in rho} alpha[r]: a 16-entry table over register bits
// 0..3 by doubling, applied to the lower half, then scaled by alpha[4] for
// the upper half (the table never holds more than 16 factors).
template <typename R>
__device__ __forceinline__ void apply_reg_product(cplx<R> (&a)[kAmps], cplx<R> c, const cplx<R> (&al)[kRegBits]) {
  cplx<R> t[16];
  t[0] = c;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < (1 << r); ++q) t[q | (1 << r)] = pmul<R>(al[r], t[q]);
#pragma unroll
  for (int r = 0; r < 16; ++r) a[r] = pmul<R>(t[r], a[r]);
#pragma unroll
  for (int r = 0; r < 16; ++r) a[r + 16] = pmul<R>(pmul<R>(al[4], t[r]), a[r + 16]);
}

// a[rho] *= c * prod_{r in rho} t[r] for real factors (the deferred diagonals
// of the pass's real gates), by the same doubling over register bits 0..3
template <typename R>
__device__ __forceinline__ void apply_real_product(cplx<R> (&a)[kAmps], R c, const R (&t5)[kRegBits]) {
  R t[16];
  t[0] = c;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < (1 << r); ++q) t[q | (1 << r)] = t[q] * t5[r];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const R lo = t[r], hi = t[r] * t5[4];
    if constexpr (sizeof(R) == 4) {
      a[r] = mul2(make_float2(lo, lo), a[r]);
      a[r + 16] = mul2(make_float2(hi, hi), a[r + 16]);
    } else {
      a[r] = mk<R>(lo * a[r].x, lo * a[r].y);
      a[r + 16] = mk<R>(hi * a[r + 16].x, hi * a[r + 16].y);
    }
  }
}

// sum_r conj(ref_r) a_r over a thread's 32 registers, in four interleaved
// FP32 partials (chains of 8 instead of one of 32), added pairwise at the end
template <typename R, typename F>
__device__ __forceinline__ cplx<R> reg_dot(const cplx<R> (&a)[kAmps], F&& ref_at) {
  cplx<R> acc[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) acc[k] = mk<R>(R(0), R(0));
#pragma unroll
  for (int r = 0; r < kAmps; ++r) acc[r & 3] = pdot<R>(acc[r & 3], ref_at(r), a[r]);
  return mk<R>((acc[0].x + acc[1].x) + (acc[2].x + acc[3].x), (acc[0].y + acc[1].y) + (acc[2].y + acc[3].y));
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- segments
template <typename R, int J, int SH, bool SPLIT, bool TRANS>
__device__ __forceinline__ void seg_step(cplx<R> (&a)[kAmps], const Seg& sg, const R* P, int tbits, bool stable) {
  if ((sg.dense >> J) & 1) dense_reg<R, J>(a, P + sg.doff[J], (sg.real >> J) & 1, stable);
  if ((sg.dwin >> J) & 1) dwin_reg<R, J, SH, SPLIT, TRANS>(a, P + sg.woff[J], tbits);
}

template <typename R, int SH, bool SPLIT = false, bool TRANS = false>
__device__ __forceinline__ void run_seg(cplx<R> (&a)[kAmps], const Seg& sg, const R* P, int tbits, bool stable) {
  if (sg.desc) {
    seg_step<R, 4, SH, SPLIT, TRANS>(a, sg, P, tbits, stable);
    seg_step<R, 3, SH, SPLIT, TRANS>(a, sg, P, tbits, stable);
    seg_step<R, 2, SH, SPLIT, TRANS>(a, sg, P, tbits, stable);
    seg_step<R, 1, SH, SPLIT, TRANS>(a, sg, P, tbits, stable);
    seg_step<R, 0, SH, SPLIT, TRANS>(a, sg, P, tbits, stable);
  } else {
    seg_step<R, 0, SH, SPLIT, TRANS>(a, sg, P, tbits, stable);
    seg_step<R, 1, SH, SPLIT, TRANS>(a, sg, P, tbits, stable);
    seg_step<R, 2, SH, SPLIT, TRANS>(a, sg, P, tbits, stable);
    seg_step<R, 3, SH, SPLIT, TRANS>(a, sg, P, tbits, stable);
    seg_step<R, 4, SH, SPLIT, TRANS>(a, sg, P, tbits, stable);
  }
}

// Compile-time programs.  The common pass -- a layer of real one-qubit gates
// on every register bit of stage A, descending, each followed by its phase
// table where the program has one, then the same on stage B -- runs as
// straight-line code: no per-step branches or segment-table lookups, so the
// compiler schedules the table loads of a step ahead of the work before it.
// PROG = 0: the segment list is interpreted (any program).  Otherwise, for
// M = 10, bit 10 is set, bits 0..4 hold the phase-table mask of stage A and
// bits 5..9 that of stage B; the planner picks it only for a program of
// exactly that shape (two descending segments A then B, all five gates real,
// no flips).  For M > 10 (prog_wide) bit 30 is set and the program is three
// descending segments A, C, B, each with its mask of real gates and of phase
// tables (5 bits each).
constexpr int kProgLayers = 1 << 10;
constexpr int prog_layers(int dwin_a, int dwin_b) { return kProgLayers | dwin_a | (dwin_b << 5); }
constexpr int kProgWide = 1 << 30;
constexpr int prog_wide(int dense_a, int dwin_a, int dense_c, int dwin_c, int dense_b, int dwin_b) {
  return kProgWide | dense_a | (dwin_a << 5) | (dense_c << 10) | (dwin_c << 15) | (dense_b << 20) | (dwin_b << 25);
}
__host__ __device__ constexpr int prog_field(int prog, int k) { return (prog >> (5 * k)) & 31; }

template <typename R, int SH, int D, int W, int J, bool SPLIT, bool TRANS>
__device__ __forceinline__ void layer_step(cplx<R> (&a)[kAmps], const Seg& sg, const R* P, int tbits) {
  if constexpr (((D >> J) & 1) != 0) dense_real_reg<R, J>(a, P + sg.doff[J]);
  if constexpr (((W >> J) & 1) != 0) dwin_reg<R, J, SH, SPLIT, TRANS>(a, P + sg.woff[J], tbits);
}

template <typename R, int SH, int W, int D = 31, bool SPLIT = false, bool TRANS = false>
__device__ __forceinline__ void run_layer(cplx<R> (&a)[kAmps], const Seg& sg, const R* P, int tbits) {
  layer_step<R, SH, D, W, 4, SPLIT, TRANS>(a, sg, P, tbits);
  layer_step<R, SH, D, W, 3, SPLIT, TRANS>(a, sg, P, tbits);
  layer_step<R, SH, D, W, 2, SPLIT, TRANS>(a, sg, P, tbits);
  layer_step<R, SH, D, W, 1, SPLIT, TRANS>(a, sg, P, tbits);
  layer_step<R, SH, D, W, 0, SPLIT, TRANS>(a, sg, P, tbits);
}

// ---------------------------------------------------------------- LOW pass
// Window = qubits 0..M-1.  A tile is 2^M consecutive amplitudes, handled by a
// group of G = 2^(M-10) warps (one warp for M = 10).  A block owns a
// contiguous range of tiles and its groups take them in turn, so at any time
// they work on neighbouring tiles of one member and share its parameters in
// L1.  Tiles stream through one or two shared-memory buffers per group,
// filled by one bulk copy each.  Register exchanges happen in place in the
// current buffer, in the padded layout (pad_base); stores are coalesced from
// stage A or C, whose lanes hold consecutive amplitudes.
template <int WARPS, int NBUF, int M = kWin> struct LowShape {
  static constexpr int G = 1 << (M - kWin);            // warps per tile
  static constexpr int GROUPS = WARPS / G;
  static constexpr int TILE = 1 << M;
  static constexpr int BUF = TILE + TILE / 32;         // a tile in the padded exchange layout
  static constexpr int PER_GROUP = NBUF * BUF;         // tile buffers
  static constexpr int THREADS = WARPS * 32;
};

// Shared-memory reads of a tile after its first one: one per register
// exchange of the program (and, for the low window, the exchange back to the
// store layout when the program ends in stage B).  With a single tile buffer
// the next tile's copy may start once the last of them is done.
__device__ __forceinline__ int exchange_count(const PassArgs& A, int stage, bool back_to_a) {
  int n = 0;
  for (int si = 0; si < A.nseg; ++si)
    if (A.segs[si].stage != stage) { ++n; stage = A.segs[si].stage; }
  if (back_to_a && stage == 1) ++n;
  return n;
}

template <typename R, int WARPS, int NBUF, int PROG = 0, int M = kWin>
__global__ void __launch_bounds__(WARPS * 32, 1) k_pass_low(cplx<R>* __restrict__ psi, const __grid_constant__ PassArgs A) {
  static_assert(NBUF == 1 || NBUF == 2, "one or two tile buffers");
  static_assert(PROG == 0 || (M == kWin) == ((PROG & kProgWide) == 0), "program kind matches the width");
  using C = cplx<R>;
  using S = LowShape<WARPS, NBUF, M>;
  constexpr int G = S::G;
  static_assert(WARPS % G == 0, "whole groups");
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[S::GROUPS][2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp / G, wig = warp % G;             // group, warp within the group
  const int t = lane + 32 * wig;                        // the thread's window bits 0..M-6 of its tile
  const bool leader = lane == 0 && wig == 0;
  C* wbase = reinterpret_cast<C*>(smem_raw) + (size_t)grp * S::PER_GROUP;
  const uint64_t nmask = (1ull << A.n) - 1;
  const R* params = static_cast<const R*>(A.params);
  const uint32_t tile_bytes = (uint32_t)S::TILE * (uint32_t)sizeof(C);
  const uint64_t per = (A.tiles + gridDim.x - 1) / gridDim.x;
  const uint64_t bfirst = (uint64_t)blockIdx.x * per;
  const uint64_t last = bfirst + per < A.tiles ? bfirst + per : A.tiles;
  const uint64_t first = bfirst + grp;

  if (leader) {
    mbar_init(&bars[grp][0], 1);
    mbar_init(&bars[grp][1], 1);
    mbar_fence_init();
  }
  group_sync<G>(grp);
  if (!A.synth && leader && first < last) {
    mbar_expect_tx(&bars[grp][0], tile_bytes);
    bulk_g2s(wbase, psi + (first << M), tile_bytes, &bars[grp][0]);
  }
  int in_flight = (!A.synth && first < last) ? 1 : 0;
  const int nx = NBUF == 1 ? exchange_count(A, 0, true) : 0;
  uint32_t it = 0;
  for (uint64_t ti = first; ti < last; ti += S::GROUPS, ++it) {
    const int cur = NBUF == 2 ? (int)(it & 1) : 0;
    const uint32_t parity = NBUF == 2 ? ((it >> 1) & 1) : (it & 1);
    C* cbuf = wbase + cur * S::BUF;
    const uint64_t tn = ti + S::GROUPS;                 // this group's next tile
    if (NBUF == 2 && !A.synth && leader && tn < last) {
      fence_proxy_async();
      mbar_expect_tx(&bars[grp][cur ^ 1], tile_bytes);
      bulk_g2s(wbase + (cur ^ 1) * S::BUF, psi + (tn << M), tile_bytes, &bars[grp][cur ^ 1]);
      ++in_flight;
    }
    // single buffer: start the next tile's copy once this tile's last shared read is done
    int reads_left = nx;
    auto release = [&]() {
      if constexpr (NBUF == 1) {
        if (--reads_left == 0 && !A.synth) {
          fence_proxy_async();
          group_sync<G>(grp);
          if (leader && tn < last) {
            mbar_expect_tx(&bars[grp][0], tile_bytes);
            bulk_g2s(wbase, psi + (tn << M), tile_bytes, &bars[grp][0]);
            ++in_flight;
          }
        }
      }
    };
    const uint64_t base = ti << M;
    const uint64_t member = base >> A.n;
    const uint64_t mloc = base & nmask;
    const R* P = params + member * (uint64_t)A.param_stride;
    const uint64_t aidx = ((member << (A.n - M)) | (mloc >> M)) * (M + 1);   // this tile's out factors
    // read at the end of the tile: into L1 now
    if (A.alpha_tab && wig == 0 && lane < 2) prefetch_l1(static_cast<const C*>(A.alpha_tab) + aidx + lane * 8);
    C a[kAmps];
    if (A.synth) {
      // the one amplitude equal to 1: register x >> (M-5) & 31 of thread x & (2^(M-5) - 1)
      const uint64_t x = A.basis ? A.basis[member] : A.basis0[0];
#pragma unroll
      for (int r = 0; r < kAmps; ++r) a[r] = mk<R>(R(0), R(0));
      if ((x & ~(uint64_t)(S::TILE - 1)) == mloc && (int)(x & ((1u << (M - 5)) - 1)) == t) {
        const int hr = (int)((x >> (M - 5)) & 31);
#pragma unroll
        for (int r = 0; r < kAmps; ++r)
          if (r == hr) a[r].x = R(1);
      }
    } else {
      // the group gives up together (a thread that saw the copy land follows
      // one that did not), after its copies in flight have landed: the
      // block's shared memory must outlive them
      if (group_any<G>(grp, !mbar_wait(&bars[grp][cur], parity, A.spin_limit))) {
        report_timeout(A.status);
        if (leader) {
          mbar_wait(&bars[grp][cur], parity);
          if (NBUF == 2 && in_flight > 1) mbar_wait(&bars[grp][cur ^ 1], ((it + 1) >> 1) & 1);
        }
        group_sync<G>(grp);
        return;
      }
      if (leader) --in_flight;
      {
        const int tb = tile_base<M, 0>(t);
        constexpr int ts = tile_step<M, 0>();
#pragma unroll
        for (int r = 0; r < kAmps; ++r) a[r] = cbuf[tb + r * ts];
      }
      if constexpr (NBUF == 1) { ++reads_left; release(); }   // counts the first read
    }
    int stage = 0;
    // register exchange between two stages, in place in the tile buffer
    auto exchange = [&](int from, int to) {
      group_sync<G>(grp);
      with_stage<M>(from, [&](auto F) {
        constexpr int SF = decltype(F)::value;
        const int pb = pad_base<M, SF>(t);
#pragma unroll
        for (int r = 0; r < kAmps; ++r) cbuf[pb + r * pad_step<M, SF>()] = a[r];
      });
      group_sync<G>(grp);
      with_stage<M>(to, [&](auto T) {
        constexpr int ST = decltype(T)::value;
        const int pb = pad_base<M, ST>(t);
#pragma unroll
        for (int r = 0; r < kAmps; ++r) a[r] = cbuf[pb + r * pad_step<M, ST>()];
      });
    };
    if constexpr (PROG != 0 && M == kWin) {
      run_layer<R, M - kRegBits, PROG & 31>(a, A.segs[0], P, t);
      exchange(0, 1);
      stage = 1;
      release();
      run_layer<R, 0, (PROG >> 5) & 31>(a, A.segs[1], P, 0);
    } else if constexpr (PROG != 0) {
      // segments A (when the program has gates there), C, B
      int si = 0;
      if constexpr (prog_field(PROG, 0) | prog_field(PROG, 1))
        run_layer<R, M - kRegBits, prog_field(PROG, 1), prog_field(PROG, 0), true>(a, A.segs[si++], P, t);
      exchange(0, 2);
      release();
      run_layer<R, 5, prog_field(PROG, 3), prog_field(PROG, 2), true>(a, A.segs[si++], P, lane);
      exchange(2, 1);
      stage = 1;
      release();
      run_layer<R, 0, prog_field(PROG, 5), prog_field(PROG, 4), true>(a, A.segs[si], P, 0);
    }
    for (int si = 0; si < (PROG != 0 ? 0 : A.nseg); ++si) {
      const Seg& sg = A.segs[si];
      if (sg.stage != stage) {
        exchange(stage, sg.stage);
        stage = sg.stage;
        release();
      }
      with_stage<M>(stage, [&](auto SC) {
        constexpr int SS = decltype(SC)::value;
        constexpr int SH = stage_base(M, SS);
        run_seg<R, SH, (M > kWin)>(a, sg, P, SS == 0 ? t : (SS == 2 ? lane : 0), A.stable != 0);
        const uint64_t fixed = mloc | (uint64_t)tile_base<M, SS>(t);
        constexpr uint64_t regmask = 31ull << SH;
        for (int f = 0; f < sg.nflip; ++f) {
          const Flip fl = A.flips[sg.flip0 + f];
          const uint64_t w = fl.per_member ? A.marked[member] : fl.index;
          flip_reg<R>(a, (w & ~regmask) == fixed, (int)((w >> SH) & 31));
        }
      });
    }
    // out factors or deferred diagonals: entry B + r for register r, and the
    // product of the entries of the thread's set window bits times entry M
    if (A.alpha_tab) {
      const R* al_g = reinterpret_cast<const R*>(static_cast<const C*>(A.alpha_tab) + aidx);
      with_stage<M>(stage, [&](auto SC) {
        constexpr int SS = decltype(SC)::value;
        constexpr int B = stage_base(M, SS);
        C al[kRegBits];
        C c = ld_c(al_g + 2 * M);
#pragma unroll
        for (int r = 0; r < kRegBits; ++r) al[r] = ld_c(al_g + 2 * (B + r));
#pragma unroll
        for (int k = 0; k < M - kRegBits; ++k)
          if ((t >> k) & 1) c = pmul<R>(ld_c(al_g + 2 * thread_bit<M, SS>(k)), c);
        apply_reg_product<R>(a, c, al);
      });
    } else if (A.diag_off >= 0) {
      const R* dg = P + A.diag_off;
      with_stage<M>(stage, [&](auto SC) {
        constexpr int SS = decltype(SC)::value;
        constexpr int B = stage_base(M, SS);
        R t5[kRegBits];
        R c = __ldg(dg + M);
#pragma unroll
        for (int r = 0; r < kRegBits; ++r) t5[r] = __ldg(dg + B + r);
#pragma unroll
        for (int k = 0; k < M - kRegBits; ++k)
          if ((t >> k) & 1) c *= __ldg(dg + thread_bit<M, SS>(k));
        apply_real_product<R>(a, c, t5);
      });
    }
    if (stage == 1) {
      exchange(1, 0);
      stage = 0;
      release();
    }
    // stage A or C: lanes hold consecutive amplitudes
    with_stage<M>(stage, [&](auto SC) {
      constexpr int SS = decltype(SC)::value;
      if constexpr (SS != 1) {
        const int tb = tile_base<M, SS>(t);
        constexpr int ts = tile_step<M, SS>();
        if (A.fid) {
          const C* ref = static_cast<const C*>(A.ref) + mloc + tb;
          const C acc = reg_dot<R>(a, [&](int r) { return __ldcg(ref + r * ts); });
          const double sre = warp_sum_d((double)acc.x), sim = warp_sum_d((double)acc.y);
          if (lane == 0) {
            const uint64_t slot = (member * (1ull << A.tile_shift) + (mloc >> M)) * G + wig;
            A.fid_partials[2 * slot] = sre;
            A.fid_partials[2 * slot + 1] = sim;
          }
        }
        C* out = psi + base + tb;
#pragma unroll
        for (int r = 0; r < kAmps; ++r) out[r * ts] = a[r];
      }
    });
    group_sync<G>(grp);
  }
}

// ---------------------------------------------------------------- HIGH pass
// Window = the M qubits c..c+M-1, c >= COLB.  A block streams a contiguous
// range of tiles of 2^COLB consecutive "columns" (qubits 0..COLB-1) x 2^M
// window rows, each loaded as boxes of 256 rows of a 2D tensor map
// [members * 2^(n-c) rows][2^c columns].  A thread's lanes hold the columns
// and 5 - COLB of its M - 5 window bits, its warp the rest.  The window bits
// are contiguous, so register r of stage S sits at offset
// r << (c + stage_base(S)).  The copy lands in the plain layout [x][col]; the
// in-place exchanges use the padded layout of the rows (pad_base).
template <int COLB, int M = kWin> struct HighShape {
  static constexpr int COLS = 1 << COLB;
  static constexpr int LW = kRegBits - COLB;            // lane bits that are window bits
  static constexpr int WARPS = 1 << (COLB + M - kWin);  // warp bits = the thread's other window bits
  static constexpr int THREADS = WARPS * 32;
  static constexpr int TILE = COLS << M;                // amplitudes of a tile
  static constexpr int BUF = COLS * ((1 << M) + (1 << (M - 5)));   // a tile in the padded exchange layout
  static constexpr int BOXES = (1 << M) / 256;          // tensor-map boxes of 256 rows
};

template <typename R, int COLB, int NBUF, bool WIDE = false, int PROG = 0, int M = kWin>
__global__ void __launch_bounds__(HighShape<COLB, M>::THREADS, NBUF == 1 ? 16 / HighShape<COLB, M>::WARPS : 1)
    k_pass_high(cplx<R>* __restrict__ psi, const __grid_constant__ CUtensorMap tmap, const __grid_constant__ PassArgs A) {
  static_assert(NBUF == 1 || NBUF == 2, "one or two tile buffers");
  static_assert(PROG == 0 || (M == kWin) == ((PROG & kProgWide) == 0), "program kind matches the width");
  using C = cplx<R>;
  using S = HighShape<COLB, M>;
  // member-local amplitude offsets: 32-bit up to 32 qubits, 64-bit (WIDE) above
  using Off = typename std::conditional<WIDE, uint64_t, uint32_t>::type;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ double fid_red[2][S::WARPS];
  C* smbase = reinterpret_cast<C*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int col = lane & (S::COLS - 1);
  const int tw = (lane >> COLB) | (warp << S::LW);      // the thread's M - 5 window bits
  const R* params = static_cast<const R*>(A.params);
  const uint32_t tile_bytes = (uint32_t)(S::TILE * sizeof(C));
  const int elem_cols = (int)(sizeof(C) / 8);          // 8-byte tensor elements per amplitude
  const int c0 = A.win[0];
  const uint64_t per = (A.tiles + gridDim.x - 1) / gridDim.x;
  const uint64_t first = (uint64_t)blockIdx.x * per;
  const uint64_t last = first + per < A.tiles ? first + per : A.tiles;
  // a tile index within a member splits into the column block among the
  // bits below the window (cshift bits) and the value of the bits above it
  const int cshift = c0 - COLB;
  const uint64_t cmask = (1ull << cshift) - 1;

  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](uint64_t t, int which) {
    const uint64_t member = t >> A.tile_shift;
    const uint64_t tl = t & ((1ull << A.tile_shift) - 1);
    mbar_expect_tx(&bars[which], tile_bytes);
    const int x = (int)((tl & cmask) * S::COLS) * elem_cols;
    const uint64_t row0 = ((member << (A.tile_shift - cshift)) | (tl >> cshift)) << M;
    C* dst = smbase + which * S::BUF;
#pragma unroll
    for (int b = 0; b < S::BOXES; ++b)
      tma_g2s_2d(dst + b * 256 * S::COLS, &tmap, x, (int)(row0 + b * 256), &bars[which]);
  };
  if (!A.synth && threadIdx.x == 0 && first < last) issue(first, 0);
  int in_flight = (!A.synth && first < last) ? 1 : 0;
  const int nx = NBUF == 1 ? exchange_count(A, A.start_stage, false) : 0;
  uint32_t it = 0;
  for (uint64_t t = first; t < last; ++t, ++it) {
    const int cur = NBUF == 2 ? (int)(it & 1) : 0;
    const uint32_t parity = NBUF == 2 ? ((it >> 1) & 1) : (it & 1);
    if (NBUF == 2 && !A.synth && threadIdx.x == 0 && t + 1 < last) {
      fence_proxy_async();
      issue(t + 1, cur ^ 1);
      ++in_flight;
    }
    // single buffer: start the next tile's copy once this tile's last shared read is done
    int reads_left = nx;
    auto release = [&]() {
      if constexpr (NBUF == 1) {
        if (--reads_left == 0 && !A.synth) {
          fence_proxy_async();
          __syncthreads();
          if (threadIdx.x == 0 && t + 1 < last) {
            issue(t + 1, 0);
            ++in_flight;
          }
        }
      }
    };
    const uint64_t member = t >> A.tile_shift;
    const uint64_t tl = t & ((1ull << A.tile_shift) - 1);
    // member-local offset of the tile (bits outside the window and the
    // columns), and the same bits packed below each other (the out-factor
    // table's index: bits below the window, then the bits above it)
    const Off tbits = (Off)(((tl >> cshift) << (c0 + M)) | ((tl & cmask) << COLB));
    const Off obits = (Off)(((tl >> cshift) << c0) | ((tl & cmask) << COLB));
    const R* P = params + member * (uint64_t)A.param_stride;
    C* sm = smbase + cur * S::BUF;
    // this tile's out factors (read at the end of the tile): into L1 now
    if (A.alpha_tab) {
      const char* at = reinterpret_cast<const char*>(static_cast<const C*>(A.alpha_tab) +
                                                     ((member << (A.n - M)) | obits) * (M + 1));
      constexpr int kLines = (int)((S::COLS * (M + 1) * sizeof(C)) / 128) + 2;
      if ((int)threadIdx.x < kLines) prefetch_l1(at + threadIdx.x * 128);
    }
    C a[kAmps];
    int stage = A.start_stage;
    if (A.synth) {
      // the one amplitude equal to 1: register (x >> sh) & 31 of the thread
      // whose other bits match (one thread of the member's whole state)
      const uint64_t x = A.basis ? A.basis[member] : A.basis0[0];
#pragma unroll
      for (int r = 0; r < kAmps; ++r) a[r] = mk<R>(R(0), R(0));
      with_stage<M>(stage, [&](auto SC) {
        constexpr int SS = decltype(SC)::value;
        const int sh = c0 + stage_base(M, SS);
        const Off fixed = tbits | (Off)col | ((Off)tile_base<M, SS>(tw) << c0);
        if ((x & ~(31ull << sh)) == (uint64_t)fixed) {
          const int hr = (int)((x >> sh) & 31);
#pragma unroll
          for (int r = 0; r < kAmps; ++r)
            if (r == hr) a[r].x = R(1);
        }
      });
    } else {
      // the block gives up together, after its copies in flight have landed
      if (__syncthreads_or(!mbar_wait(&bars[cur], parity, A.spin_limit))) {
        report_timeout(A.status);
        if (threadIdx.x == 0) {
          mbar_wait(&bars[cur], parity);
          if (NBUF == 2 && in_flight > 1) mbar_wait(&bars[cur ^ 1], ((it + 1) >> 1) & 1);
        }
        return;
      }
      if (threadIdx.x == 0) --in_flight;
      // the copy lands in the plain layout [x][col]
      with_stage<M>(stage, [&](auto SC) {
        constexpr int SS = decltype(SC)::value;
        const int tb = tile_base<M, SS>(tw) * S::COLS + col;
        constexpr int ts = tile_step<M, SS>() * S::COLS;
#pragma unroll
        for (int r = 0; r < kAmps; ++r) a[r] = sm[tb + r * ts];
      });
      if constexpr (NBUF == 1) { ++reads_left; release(); }   // counts the first read
    }
    // register exchange between two stages, in place in the tile buffer
    auto exchange = [&](int from, int to) {
      __syncthreads();
      with_stage<M>(from, [&](auto F) {
        constexpr int SF = decltype(F)::value;
        const int pb = pad_base<M, SF>(tw) * S::COLS + col;
#pragma unroll
        for (int r = 0; r < kAmps; ++r) sm[pb + r * (pad_step<M, SF>() * S::COLS)] = a[r];
      });
      __syncthreads();
      with_stage<M>(to, [&](auto T) {
        constexpr int ST = decltype(T)::value;
        const int pb = pad_base<M, ST>(tw) * S::COLS + col;
#pragma unroll
        for (int r = 0; r < kAmps; ++r) a[r] = sm[pb + r * (pad_step<M, ST>() * S::COLS)];
      });
    };
    if constexpr (PROG != 0 && M == kWin) {   // the planner guarantees start stage A
      run_layer<R, M - kRegBits, PROG & 31, 31, false, true>(a, A.segs[0], P, tw);
      exchange(0, 1);
      stage = 1;
      release();
      run_layer<R, 0, (PROG >> 5) & 31>(a, A.segs[1], P, 0);
    } else if constexpr (PROG != 0) {         // segments A, C, B; start stage A
      run_layer<R, M - kRegBits, prog_field(PROG, 1), prog_field(PROG, 0), true>(a, A.segs[0], P, tw);
      exchange(0, 2);
      release();
      run_layer<R, 5, prog_field(PROG, 3), prog_field(PROG, 2), true>(a, A.segs[1], P, tw & 31);
      exchange(2, 1);
      stage = 1;
      release();
      run_layer<R, 0, prog_field(PROG, 5), prog_field(PROG, 4), true>(a, A.segs[2], P, 0);
    }
    for (int si = 0; si < (PROG != 0 ? 0 : A.nseg); ++si) {
      const Seg& sg = A.segs[si];
      if (sg.stage != stage) {
        exchange(stage, sg.stage);
        stage = sg.stage;
        release();
      }
      with_stage<M>(stage, [&](auto SC) {
        constexpr int SS = decltype(SC)::value;
        constexpr int SH = stage_base(M, SS);
        run_seg<R, SH, (M > kWin), true>(a, sg, P, SS == 0 ? tw : (SS == 2 ? (tw & 31) : 0), A.stable != 0);
        const int sh = c0 + SH;
        const uint64_t regmask = 31ull << sh;
        const Off fixed = tbits | (Off)col | ((Off)tile_base<M, SS>(tw) << c0);
        for (int f = 0; f < sg.nflip; ++f) {
          const Flip fl = A.flips[sg.flip0 + f];
          const uint64_t w = fl.per_member ? A.marked[member] : fl.index;
          flip_reg<R>(a, (w & ~regmask) == fixed, (int)((w >> sh) & 31));
        }
      });
    }
    // out factors or deferred diagonals (as in the low pass)
    if (A.alpha_tab) {
      const R* al_c = reinterpret_cast<const R*>(static_cast<const C*>(A.alpha_tab) +
                                                 ((member << (A.n - M)) | obits | (Off)col) * (M + 1));
      with_stage<M>(stage, [&](auto SC) {
        constexpr int SS = decltype(SC)::value;
        constexpr int B = stage_base(M, SS);
        C c = ld_c(al_c + 2 * M);
        C al[kRegBits];
#pragma unroll
        for (int r = 0; r < kRegBits; ++r) al[r] = ld_c(al_c + 2 * (B + r));
#pragma unroll
        for (int k = 0; k < M - kRegBits; ++k)
          if ((tw >> k) & 1) c = pmul<R>(ld_c(al_c + 2 * thread_bit<M, SS>(k)), c);
        apply_reg_product<R>(a, c, al);
      });
    } else if (A.diag_off >= 0) {
      const R* dg = P + A.diag_off;
      with_stage<M>(stage, [&](auto SC) {
        constexpr int SS = decltype(SC)::value;
        constexpr int B = stage_base(M, SS);
        R t5[kRegBits];
        R c = __ldg(dg + M);
#pragma unroll
        for (int r = 0; r < kRegBits; ++r) t5[r] = __ldg(dg + B + r);
#pragma unroll
        for (int k = 0; k < M - kRegBits; ++k)
          if ((tw >> k) & 1) c *= __ldg(dg + thread_bit<M, SS>(k));
        apply_real_product<R>(a, c, t5);
      });
    }
    with_stage<M>(stage, [&](auto SC) {
      constexpr int SS = decltype(SC)::value;
      const int sh = c0 + stage_base(M, SS);
      const Off fixed = tbits + (Off)col + ((Off)tile_base<M, SS>(tw) << c0);
      if (A.fid) {
        const C* ref = static_cast<const C*>(A.ref) + fixed;
        const C acc = reg_dot<R>(a, [&](int r) { return __ldcg(ref + ((Off)r << sh)); });
        const double sre = warp_sum_d((double)acc.x), sim = warp_sum_d((double)acc.y);
        if (lane == 0) { fid_red[0][warp] = sre; fid_red[1][warp] = sim; }
        __syncthreads();
        if (threadIdx.x == 0) {
          double tr = 0.0, tim = 0.0;
          for (int w = 0; w < S::WARPS; ++w) { tr += fid_red[0][w]; tim += fid_red[1][w]; }
          const uint64_t slot = member * (1ull << A.tile_shift) + tl;
          A.fid_partials[2 * slot] = tr;
          A.fid_partials[2 * slot + 1] = tim;
        }
      }
      // register r goes to fixed + r 2^sh: a running 32-bit offset (64-bit for
      // WIDE) from the member's base instead of a shift and a 64-bit add each
      C* out = psi + (member << A.n);
      Off o = fixed;
      const Off step = (Off)1 << sh;
#pragma unroll
      for (int r = 0; r < kAmps; ++r, o += step) out[o] = a[r];
    });
    __syncthreads();
  }
}

// ---------------------------------------------------------------- host side
template <typename R, int W, int NB, int M = kWin>
size_t low_smem() {
  using S = LowShape<W, NB, M>;
  return (size_t)S::GROUPS * S::PER_GROUP * sizeof(cplx<R>);
}
template <typename R, int CB, int NB, int M = kWin>
size_t high_smem() {
  return NB * (size_t)HighShape<CB, M>::BUF * sizeof(cplx<R>);
}

// Dynamic shared memory of a pass kernel, and a carveout preference just
// large enough for `blocks` resident blocks per SM, so the rest of the
// unified L1 caches the members' parameters and phase tables.
template <typename K>
cudaError_t set_pass_attrs(K kernel, size_t dyn, int blocks) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  constexpr size_t kSmemPerSM = 228 * 1024, kReservedPerBlock = 1024, kStatic = 1024;
  const size_t need = (size_t)blocks * (dyn + kStatic + kReservedPerBlock);
  const int pct = (int)std::min<size_t>(100, (need * 100 + kSmemPerSM - 1) / kSmemPerSM);
  return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

// Windows of 11 and 12 qubits (complex64, pass_wide.cu).  Columns of a high
// tile: 8 for m = 11, 4 for m = 12 (tiles of 128 KB whose rows fill whole
// 32-byte sectors).
constexpr int wide_colb(int m) { return 14 - m; }
// The compiled program of a pass that applies a real gate, then the phase
// table over the bits below it, on every bit of the window, top down (the
// noisy QFT on m qubits of a larger state), or 0 for other widths.
constexpr int wide_full_prog(int m) {
  return m == 11 ? prog_wide(0x1f, 0x1f, 0x01, 0x01, 0x1f, 0x1e)
                 : (m == 12 ? prog_wide(0x1f, 0x1f, 0x03, 0x03, 0x1f, 0x1e) : 0);
}
cudaError_t launch_pass_wide(cplx<float>* psi, const CUtensorMap& tmap, const PassArgs& A, bool high, int m, int prog,
                             int sms, cudaStream_t s);
cudaError_t set_wide_attrs();

}  // namespace fused
}  // namespace qs
