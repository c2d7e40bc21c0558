// Fidelity of a batch of state vectors without any device allocation.
//
// Some callers cannot allocate device memory: a host application or
// framework that owns the GPU's memory through its own pool and forbids other
// allocators, or a latency-critical loop that cannot afford cudaMalloc's
// device-wide synchronisation and unpredictable cost.  This entry point
// computes the same |<phi|psi_b>|^2 as qs_fidelity, on state and reference
// buffers the caller already holds, with its scratch in a fixed array that
// every GPU loading this library keeps for the life of the process.
//
// The scratch is one file-scope __device__ array.  Its host-side name is only
// a stand-in, so host code never passes it to a kernel: the first call on a
// device looks up the array's device address with cudaGetSymbolAddress (with
// that device current) and caches it; later calls on that device reuse it.
// The cached address belongs to the device's primary context as it was at
// that first call: a caller that resets the device (cudaDeviceReset) or runs
// in a context of its own must not use this entry point afterwards.  All
// calls on a device share the array and it keeps the last call's contents;
// each call overwrites every partial it reads, so nothing needs clearing, but
// two calls whose work overlaps on the GPU (different streams, or different
// host threads) race on the array.
//
// Precision: each thread sums at most kNaTerms products in the state's
// precision, then adds that partial to an FP64 sum; blocks and chunks are
// added in FP64 in a fixed order, so the rounding of a complex64 fidelity
// does not grow with the number of amplitudes a block covers.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.cuh"

namespace {

constexpr int kNaBlock = 256;
constexpr int kNaTerms = 16;             // products per FP32 partial before it joins the FP64 sum
constexpr int kNaMaxDevices = 64;

// partials: 2 doubles per (member, chunk); results: 1 double per member
static __device__ __align__(256) double g_noalloc_scratch[2 * QS_NOALLOC_MAX_PARTIALS + QS_NOALLOC_MAX_MEMBERS];


__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partials[b][c] = sum over chunk c of member b of conj(ref_i) psi_i
template <typename R>
__global__ void __launch_bounds__(kNaBlock) k_na_dot(const qs::cplx<R>* __restrict__ psi,
                                                     const qs::cplx<R>* __restrict__ ref, int n, int chunks,
                                                     uint64_t chunk, double* __restrict__ partials) {
  __shared__ double sre[kNaBlock / 32], sim[kNaBlock / 32];
  const int c = blockIdx.x, b = blockIdx.y;
  const uint64_t N = 1ull << n;
  const uint64_t beg = (uint64_t)c * chunk;
  const uint64_t end = beg + chunk < N ? beg + chunk : N;
  const qs::cplx<R>* p = psi + (uint64_t)b * N;
  double dre = 0.0, dim = 0.0;
  for (uint64_t x = beg + threadIdx.x; x < end;) {
    R re = 0, im = 0;
    for (int k = 0; k < kNaTerms && x < end; ++k, x += blockDim.x) {
      const qs::cplx<R> a = p[x], r = ref[x];
      re += r.x * a.x + r.y * a.y;
      im += r.x * a.y - r.y * a.x;
    }
    dre += (double)re;
    dim += (double)im;
  }
  dre = na_warp_sum(dre);
  dim = na_warp_sum(dim);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sre[w] = dre; sim[w] = dim; }
  __syncthreads();
  if (w == 0) {
    dre = l < kNaBlock / 32 ? sre[l] : 0.0;
    dim = l < kNaBlock / 32 ? sim[l] : 0.0;
    dre = na_warp_sum(dre);
    dim = na_warp_sum(dim);
    if (l == 0) {
      partials[2 * ((uint64_t)b * chunks + c)] = dre;
      partials[2 * ((uint64_t)b * chunks + c) + 1] = dim;
    }
  }
}

// results[b] = |sum_c partials[b][c]|^2, partials added in a fixed order
__global__ void k_na_finalize(const double* __restrict__ partials, int members, int chunks,
                              double* __restrict__ results) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= members) return;
  double re = 0.0, im = 0.0;
  for (int c = 0; c < chunks; ++c) {
    re += partials[2 * ((uint64_t)b * chunks + c)];
    im += partials[2 * ((uint64_t)b * chunks + c) + 1];
  }
  results[b] = re * re + im * im;
}

std::mutex g_na_mutex;
double* g_na_ptr[kNaMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set up once).
cudaError_t na_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" qs_status qs_fidelity_noalloc(const void* states, const void* ref, int n, int members,
                                         qs_dtype dtype, void* cuda_stream, double* out) {
  if (!states || !ref || !out) return QS_ERR_INVALID_ARG;
  if (n < 1 || n > 40 || members < 1) return QS_ERR_INVALID_ARG;
  if (dtype != QS_C64 && dtype != QS_C128) return QS_ERR_INVALID_ARG;
  if (members > QS_NOALLOC_MAX_MEMBERS) return QS_ERR_INVALID_ARG;   // beyond the fixed scratch
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double* scratch = nullptr;
  if (na_scratch(&scratch) != cudaSuccess) { cudaGetLastError(); return QS_ERR_CUDA; }
  double* partials = scratch;
  double* results = scratch + 2 * QS_NOALLOC_MAX_PARTIALS;
  // chunks per member: enough blocks to fill the GPU, within the scratch
  const uint64_t N = 1ull << n;
  uint64_t chunks = (N + 4095) / 4096;
  const uint64_t cap = QS_NOALLOC_MAX_PARTIALS / (uint64_t)members;
  if (chunks > cap) chunks = cap;
  if (chunks < 1) chunks = 1;
  const uint64_t chunk = (N + chunks - 1) / chunks;
  dim3 grid((unsigned)chunks, (unsigned)members);
  if (dtype == QS_C64)
    k_na_dot<float><<<grid, kNaBlock, 0, s>>>((const float2*)states, (const float2*)ref, n, (int)chunks, chunk, partials);
  else
    k_na_dot<double><<<grid, kNaBlock, 0, s>>>((const double2*)states, (const double2*)ref, n, (int)chunks, chunk, partials);
  k_na_finalize<<<(members + 255) / 256, 256, 0, s>>>(partials, members, (int)chunks, results);
  if (cudaGetLastError() != cudaSuccess) return QS_ERR_CUDA;
  if (cudaMemcpyAsync(out, results, (size_t)members * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return QS_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return QS_ERR_CUDA;
  return QS_OK;
}
