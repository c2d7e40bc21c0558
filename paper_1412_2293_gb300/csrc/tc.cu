// Dense k-qubit blocks (k = 3..5) on complex64 states with the fifth-generation
// tensor cores (tcgen05, accumulators in tensor memory).
//
// The update is the one of Sec. 2 for a k-qubit gate: every group of 2^k
// amplitudes that share the non-target bits is multiplied by U.  Across a
// batch (trajectories, or factor columns) and across the groups this is one
// dense contraction, so it runs as a GEMM:
//
//   tile  = 128 groups (the 7 lowest non-target bits) x 2^k target values,
//   A     = the tile as a real matrix, row m = group, column 2j + c = part c
//           (re, im) of the amplitude with local index j       (128 x 2D),
//   B     = the real form of U: row 2i + c', column 2j + c holds
//           Re U_ij, -Im U_ij (c' = 0) and Im U_ij, Re U_ij (c' = 1)  (2D x 2D),
//   D     = A B^T: row m holds the new amplitudes of group m, interleaved,
//
// with D = 2^k.  The MMA is kind::tf32 with FP32 accumulation; FP32 accuracy
// comes from splitting both operands, x = hi + lo with hi the top 19 bits
// (the part a tf32 operand keeps), and accumulating hi*hi + lo*hi + hi*lo
// (the dropped lo*lo term is below 2^-20 of |x||u|).
//
// One CTA = 4 warps; thread t owns group m = t of every tile: it loads the
// tile's row m from HBM (lanes read consecutive groups), splits it into the
// hi/lo operand tiles in shared memory, thread 0 issues the MMAs, and after
// their commit every warp reads its 32 TMEM lanes (rows) back and stores the
// row to HBM.  Persistent CTAs stride over the tiles; a CTA issues its next
// tile's loads into a second register set before writing the current tile
// (k <= 4) or right after the MMAs (k = 5), so they overlap the MMAs and the
// epilogue.  Every wait on the MMA
// commit is bounded: on expiry the kernel records the fact in status and
// leaves after freeing its tensor memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "internal.cuh"

namespace qs {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTcRows = 128;            // groups per tile (MMA M)
constexpr int kTcFree = 7;              // non-target bits inside a tile
constexpr uint32_t kSpinLimit = 1u << 24;

struct TcArgs {
  float2* psi;
  uint64_t tiles;                       // members * 2^(n - k - 7)
  uint32_t off_j[32];                   // index offset of local index j (targets in caller order)
  int pos[12];                          // ascending positions of the tile's k + 7 bits
  int free_pos[kTcFree];                // the 7 free bits, ascending (group index m)
  const float* U;                       // D x D interleaved complex, row-major
  int* status;                          // status[0] = 1 on an MMA wait that expired
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t insert0(uint64_t v, int s) {
  const uint64_t low = v & ((1ull << s) - 1);
  return ((v >> s) << (s + 1)) | low;
}

// Byte offset of element (row, col) in a K-major operand without swizzle:
// 8-row x 16-byte core matrices, the row direction fastest (SBO = 128 B),
// the K direction every rows/8 core matrices (LBO = rows * 16 B).
__device__ __forceinline__ uint32_t op_byte(int row, int col, int rows) {
  return (uint32_t)(row * 16 + (col >> 2) * rows * 16 + (col & 3) * 4);
}

// Shared-memory matrix descriptor (tcgen05): start, LBO, SBO in 16-byte
// units, descriptor version 1 (bits 46-47), no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32
// (bits 7-9, 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
      :: "r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(mbar) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x NC consecutive 32-bit columns of tensor memory -> NC registers per thread.
template <int NC>
__device__ __forceinline__ void tmem_load(uint32_t taddr, float* v);

#define QS_R4(i) "=f"(v[i]), "=f"(v[i + 1]), "=f"(v[i + 2]), "=f"(v[i + 3])
template <>
__device__ __forceinline__ void tmem_load<16>(uint32_t taddr, float* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : QS_R4(0), QS_R4(4), QS_R4(8), QS_R4(12) : "r"(taddr));
}
template <>
__device__ __forceinline__ void tmem_load<32>(uint32_t taddr, float* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : QS_R4(0), QS_R4(4), QS_R4(8), QS_R4(12), QS_R4(16), QS_R4(20), QS_R4(24), QS_R4(28) : "r"(taddr));
}
#undef QS_R4

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

template <int K>
__global__ void __launch_bounds__(kTcThreads) k_dense_tc(TcArgs args) {
  constexpr int D = 1 << K;             // amplitudes per group
  constexpr int KD = 2 * D;             // MMA K (real columns) and N (real rows of B)
  constexpr int kCols = KD < 32 ? 32 : KD;   // tensor-memory columns (power of two >= 32)
  constexpr uint32_t kABytes = kTcRows * KD * 4;
  constexpr uint32_t kBBytes = KD * KD * 4;
  constexpr uint32_t kIdesc = tf32_idesc(kTcRows, KD);

  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* a_hi = smem;
  unsigned char* a_lo = smem + kABytes;
  unsigned char* b_hi = smem + 2 * kABytes;
  unsigned char* b_lo = smem + 2 * kABytes + kBBytes;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;

  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(&tmem_base)), "r"((uint32_t)kCols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // the real form of U, split into hi and lo operand tiles
  for (int e = tid; e < KD * KD; e += kTcThreads) {
    const int row = e / KD, col = e % KD;          // row 2i + c', column 2j + c
    const int i = row >> 1, cp = row & 1, j = col >> 1, c = col & 1;
    const float ur = args.U[2 * (i * D + j)], ui = args.U[2 * (i * D + j) + 1];
    const float f = cp == 0 ? (c == 0 ? ur : -ui) : (c == 0 ? ui : ur);
    const float hi = tf32_hi(f);
    const uint32_t b = op_byte(row, col, KD);
    *reinterpret_cast<float*>(b_hi + b) = hi;
    *reinterpret_cast<float*>(b_lo + b) = f - hi;
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t mbar_a = smem_u32(&mbar);

  // offset of this thread's group inside a tile
  uint64_t off_m = 0;
#pragma unroll
  for (int b = 0; b < kTcFree; ++b) off_m |= (uint64_t)((tid >> b) & 1) << args.free_pos[b];

  auto tile_base = [&](uint64_t t) {
#pragma unroll
    for (int b = 0; b < K + kTcFree; ++b) t = insert0(t, args.pos[b]);
    return t | off_m;
  };
  uint32_t phase = 0;
  bool ok = true;
  uint64_t t = blockIdx.x;
  uint64_t base = tile_base(t);
  // two register sets in turn (k <= 4): while one tile is written, multiplied
  // and stored, the next tile's loads land in the other
  float2 xa[D], xb[D];
  if (t < args.tiles) {
    const float2* p = args.psi + base;
#pragma unroll
    for (int j = 0; j < D; ++j) xa[j] = p[args.off_j[j]];
  }
  auto process = [&](float2 (&x)[D], float2 (&xn)[D]) -> bool {
    if (t >= args.tiles) return false;
    const uint64_t tn = t + gridDim.x;
    const uint64_t base_n = tile_base(tn);
    auto prefetch = [&]() {
      if (tn < args.tiles) {
        const float2* p = args.psi + base_n;
#pragma unroll
        for (int j = 0; j < D; ++j) xn[j] = p[args.off_j[j]];
      }
    };
    // k <= 4: the next loads go out before this tile's operand writes; k = 5
    // (twice the registers per set) issues them after the MMAs
    if constexpr (K <= 4) prefetch();
    // row m = tid of A: columns 2j .. 2j + 3 for j even are one 16-byte chunk
#pragma unroll
    for (int j = 0; j < D; j += 2) {
      const float4 v = make_float4(x[j].x, x[j].y, x[j + 1].x, x[j + 1].y);
      const float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
      const uint32_t b = op_byte(tid, 2 * j, kTcRows);
      *reinterpret_cast<float4*>(a_hi + b) = h;
      *reinterpret_cast<float4*>(a_lo + b) = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      fence_after();
      const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
      constexpr uint32_t lbo_a = kTcRows * 16, lbo_b = KD * 16;
      uint32_t acc = 0;
#pragma unroll
      for (int s = 0; s < KD / 8; ++s) {          // K = 8 per instruction: two core matrices along K
        const uint64_t dah = smem_desc(ah + 2 * s * lbo_a, lbo_a, 128);
        const uint64_t dal = smem_desc(al + 2 * s * lbo_a, lbo_a, 128);
        const uint64_t dbh = smem_desc(bh + 2 * s * lbo_b, lbo_b, 128);
        const uint64_t dbl = smem_desc(bl + 2 * s * lbo_b, lbo_b, 128);
        mma_tf32(tmem, dah, dbh, kIdesc, acc);
        acc = 1;
        mma_tf32(tmem, dal, dbh, kIdesc, 1);
        mma_tf32(tmem, dah, dbl, kIdesc, 1);
      }
      mma_commit(mbar_a);
    }
    if constexpr (K > 4) prefetch();
    const bool got = mbar_wait(mbar_a, phase);
    if (__syncthreads_or(!got)) { ok = false; return false; }   // every thread leaves together
    phase ^= 1;
    fence_after();
    // read back and store in chunks of at most 32 columns (16 amplitudes)
    constexpr int kChunk = KD < 32 ? KD : 32;
    float2* q = args.psi + base;
#pragma unroll
    for (int c0 = 0; c0 < KD; c0 += kChunk) {
      float d[kChunk];
      tmem_load<kChunk>(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, d);
      tmem_wait_ld();
#pragma unroll
      for (int i = 0; i < kChunk / 2; ++i) q[args.off_j[c0 / 2 + i]] = make_float2(d[2 * i], d[2 * i + 1]);
    }
    fence_before();
    __syncthreads();
    t = tn;
    base = base_n;
    return true;
  };
  // k = 5 keeps one set: its late prefetch reuses the registers of the tile
  // just written to shared memory
  float2 (&xs)[D] = K <= 4 ? xb : xa;
  while (process(xa, xs) && process(xs, xa)) {
  }
  if (!ok) {
    if (tid == 0) atomicExch(args.status, 1);
    mbar_wait(mbar_a, phase);              // let an MMA still in flight finish (bounded)
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"((uint32_t)kCols) : "memory");
  }
}

template <int K>
constexpr size_t tc_smem_bytes() {
  return (size_t)2 * kTcRows * (2 << K) * 4 + (size_t)2 * (2 << K) * (2 << K) * 4;
}

template <int K>
cudaError_t launch_k(const TcArgs& a, cudaStream_t s) {
  static std::atomic<int> grid_cache{0};
  const size_t smem = tc_smem_bytes<K>();
  int grid = grid_cache.load();
  if (grid == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_dense_tc<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_dense_tc<K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    // resident CTAs per SM from the kernel's own needs (shared memory with the
    // per-block reserve, registers at warp granularity of 256, threads, and
    // tensor-memory columns so that no CTA waits in tcgen05.alloc)
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, k_dense_tc<K>);
    if (e != cudaSuccess) return e;
    int dev = 0, smem_sm = 0, reserve = 0, regs_sm = 0, threads_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserve, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + reserve);
    const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;
    const int by_regs = regs_sm / (warp_regs * (kTcThreads / 32));
    const int by_threads = threads_sm / kTcThreads;
    constexpr int cols = (2 << K) < 32 ? 32 : (2 << K);
    const int per_sm = std::max(1, std::min({by_smem, by_regs, by_threads, 512 / cols}));
    grid = per_sm * num_sms();
    grid_cache.store(grid);
  }
  const uint64_t g = std::min<uint64_t>((uint64_t)grid, a.tiles);
  k_dense_tc<K><<<(unsigned)g, kTcThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool dense_tc_applicable(int n, int k) { return k >= 3 && k <= 5 && n - k >= kTcFree && n <= 32; }

cudaError_t launch_dense_tc(qs_ctx* h, void* psi, int n, int members, const int* targets, int k,
                            const float* U_dev) {
  if (!dense_tc_applicable(n, k) || h->dtype != QS_C64 || members < 1) return cudaErrorNotSupported;
  TcArgs a{};
  a.psi = static_cast<float2*>(psi);
  a.tiles = (uint64_t)members << (n - k - kTcFree);
  a.U = U_dev;
  a.status = h->dstatus + 3;
  uint32_t tmask = 0;
  for (int i = 0; i < k; ++i) tmask |= 1u << targets[i];
  for (int j = 0; j < (1 << k); ++j) {
    uint32_t o = 0;
    for (int i = 0; i < k; ++i) o |= (uint32_t)((j >> i) & 1) << targets[i];
    a.off_j[j] = o;
  }
  int nf = 0;
  for (int b = 0; b < n && nf < kTcFree; ++b)
    if (!(tmask >> b & 1)) a.free_pos[nf++] = b;
  int np = 0;
  for (int b = 0; b < n; ++b)
    if ((tmask >> b & 1) || (nf > 0 && b <= a.free_pos[kTcFree - 1] && !(tmask >> b & 1))) a.pos[np++] = b;
  if (np != k + kTcFree) return cudaErrorInvalidValue;
  switch (k) {
    case 3: return launch_k<3>(a, h->stream);
    case 4: return launch_k<4>(a, h->stream);
    default: return launch_k<5>(a, h->stream);
  }
}

}  // namespace qs
