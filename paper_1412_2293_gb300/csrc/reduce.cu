// Fidelity and trace reductions (Figs. 1-4, Eq. 10).
//
// Each member's sum is split into fixed chunks; a block reduces one chunk
// and writes an FP64 partial; a second kernel adds the partials of a member
// in a fixed order, so results are deterministic run to run.  Inside a
// thread, a complex64 state accumulates its (short) run of products in FP32
// -- each product of two FP32 numbers is formed in FP32 as the amplitudes
// are -- and everything from the warp level up is FP64.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.cuh"

namespace qs {

namespace {

constexpr int kRBlock = 256;
constexpr int kChunk = 4096;            // amplitudes per block

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of (a, b); result valid in thread 0.
__device__ __forceinline__ double2 block_sum2(double a, double b) {
  __shared__ double sa[32], sb[32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sa[w] = a; sb[w] = b; }
  __syncthreads();
  double2 r = make_double2(0.0, 0.0);
  if (w == 0) {
    const int nw = blockDim.x >> 5;
    a = l < nw ? sa[l] : 0.0;
    b = l < nw ? sb[l] : 0.0;
    r.x = warp_sum(a);
    r.y = warp_sum(b);
  }
  __syncthreads();
  return r;
}

// partial[member][chunk] = sum over the chunk of conj(ref_i) psi_i
template <typename R>
__global__ void __launch_bounds__(kRBlock) k_dot_partials(const cplx<R>* __restrict__ psi,
                                                          const cplx<R>* __restrict__ ref, int n,
                                                          int chunks, int chunk, double* partials) {
  const int c = blockIdx.x, b = blockIdx.y;
  const uint64_t N = 1ull << n;
  const uint64_t beg = (uint64_t)c * chunk;
  const cplx<R>* p = psi + (uint64_t)b * N;
  R re = 0, im = 0;
  for (int i = threadIdx.x; i < chunk; i += blockDim.x) {
    const uint64_t x = beg + i;
    if (x < N) {
      const cplx<R> a = p[x], r = ref[x];
      re += r.x * a.x + r.y * a.y;
      im += r.x * a.y - r.y * a.x;
    }
  }
  const double2 s = block_sum2((double)re, (double)im);
  if (threadIdx.x == 0) {
    partials[2 * ((uint64_t)b * chunks + c)] = s.x;
    partials[2 * ((uint64_t)b * chunks + c) + 1] = s.y;
  }
}

// partial[member][chunk] = sum |psi_i|^2 (stored in the .x slot)
template <typename R>
__global__ void __launch_bounds__(kRBlock) k_norm_partials(const cplx<R>* __restrict__ psi, int n,
                                                           int chunks, int chunk, double* partials) {
  const int c = blockIdx.x, b = blockIdx.y;
  const uint64_t N = 1ull << n;
  const uint64_t beg = (uint64_t)c * chunk;
  const cplx<R>* p = psi + (uint64_t)b * N;
  R s = 0;
  for (int i = threadIdx.x; i < chunk; i += blockDim.x) {
    const uint64_t x = beg + i;
    if (x < N) { const cplx<R> a = p[x]; s += a.x * a.x + a.y * a.y; }
  }
  const double2 t = block_sum2((double)s, 0.0);
  if (threadIdx.x == 0) {
    partials[2 * ((uint64_t)b * chunks + c)] = t.x;
    partials[2 * ((uint64_t)b * chunks + c) + 1] = 0.0;
  }
}

// v_b = |sum_c partial|^2 (mode 0) or sum_c partial.x (mode 1); out[g] =
// v_{g group} + ... + v_{g group + group - 1} in order (group = 1: out[b] =
// v_b).  One warp per output: lane l adds chunks l, l + 32, ... in order, the
// lanes meet in a fixed shuffle tree (the same order on every call).
__global__ void __launch_bounds__(256) k_finalize(const double* partials, int members, int chunks, int mode, int group,
                                                  double* out) {
  const int outs = members / group;
  const int lane = threadIdx.x & 31;
  const int warps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int g = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); g < outs; g += warps) {
    double s = 0.0;
    for (int b = g * group; b < (g + 1) * group; ++b) {
      const double* pb = partials + 2 * (uint64_t)b * chunks;
      double re = 0.0, im = 0.0;
      for (int c = lane; c < chunks; c += 32) {
        re += pb[2 * c];
        im += pb[2 * c + 1];
      }
      re = warp_sum(re);
      im = warp_sum(im);
      s += mode == 0 ? re * re + im * im : re;
    }
    if (lane == 0) out[g] = s;
  }
}

// warps of the finalize launch for `outs` outputs (eight per block)
inline unsigned finalize_blocks(int outs) { return (unsigned)std::max(1, std::min((outs + 7) / 8, 4096)); }

template <typename R>
__global__ void k_basis_prob(const cplx<R>* psi, int n, int members, uint64_t x, int group, double* out) {
  const int outs = members / group;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < outs; g += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = g * group; b < (g + 1) * group; ++b) {
      const cplx<R> a = psi[((uint64_t)b << n) + x];
      s += (double)a.x * a.x + (double)a.y * a.y;
    }
    out[g] = s;
  }
}

// tr(rho): sum_i Re rho[i][i] at vec index i * (2^n + 1)
template <typename R>
__global__ void __launch_bounds__(kRBlock) k_dm_trace_partials(const cplx<R>* rho, int n, int chunks,
                                                               int chunk, double* partials) {
  const uint64_t N = 1ull << n;
  const uint64_t beg = (uint64_t)blockIdx.x * chunk;
  double s = 0.0;
  for (int i = threadIdx.x; i < chunk; i += blockDim.x) {
    const uint64_t x = beg + i;
    if (x < N) s += (double)rho[x * (N + 1)].x;
  }
  const double2 t = block_sum2(s, 0.0);
  if (threadIdx.x == 0) { partials[2 * blockIdx.x] = t.x; partials[2 * blockIdx.x + 1] = 0.0; }
}

// <phi|rho|phi> = sum_i conj(phi_i) sum_j rho[i][j] phi_j, one block per row
template <typename R>
__global__ void __launch_bounds__(kRBlock) k_dm_expect_rows(const cplx<R>* __restrict__ rho,
                                                            const cplx<R>* __restrict__ phi, int n,
                                                            double* partials) {
  const uint64_t N = 1ull << n;
  const uint64_t i = blockIdx.x;
  const cplx<R>* row = rho + i * N;
  double re = 0.0, im = 0.0;
  for (uint64_t j = threadIdx.x; j < N; j += blockDim.x) {
    const cplx<R> a = row[j], f = phi[j];
    re += (double)a.x * f.x - (double)a.y * f.y;
    im += (double)a.x * f.y + (double)a.y * f.x;
  }
  const double2 v = block_sum2(re, im);
  if (threadIdx.x == 0) {
    const cplx<R> f = phi[i];
    partials[2 * i] = (double)f.x * v.x + (double)f.y * v.y;         // Re(conj(f) v)
    partials[2 * i + 1] = (double)f.x * v.y - (double)f.y * v.x;
  }
}

template <typename R>
__global__ void k_convert_ref(const double* src, cplx<R>* dst, size_t count) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = mk<R>((R)src[2 * i], (R)src[2 * i + 1]);
}

bool ensure_partials(qs_ctx* h, size_t doubles) {
  if (h->partials_cap >= doubles) return true;
  if (h->partials) cudaFreeAsync(h->partials, h->stream);
  h->partials = nullptr;
  h->partials_cap = 0;
  if (cudaMallocAsync((void**)&h->partials, doubles * sizeof(double), h->stream) != cudaSuccess) return false;
  h->partials_cap = doubles;
  return true;
}

int chunk_count(int n) {
  const uint64_t N = 1ull << n;
  return (int)((N + kChunk - 1) / kChunk);
}

}  // namespace

cudaError_t launch_dot(qs_ctx* h, const void* psi, const void* ref, int n, int members,
                       int group, double* out) {
  const int chunks = chunk_count(n);
  if (!ensure_partials(h, (size_t)2 * chunks * members)) return cudaErrorMemoryAllocation;
  dim3 grid(chunks, members);
  if (h->dtype == QS_C64)
    k_dot_partials<float><<<grid, kRBlock, 0, h->stream>>>((const float2*)psi, (const float2*)ref, n, chunks, kChunk, h->partials);
  else
    k_dot_partials<double><<<grid, kRBlock, 0, h->stream>>>((const double2*)psi, (const double2*)ref, n, chunks, kChunk, h->partials);
  k_finalize<<<finalize_blocks(members / group), 256, 0, h->stream>>>(h->partials, members, chunks, 0, group, out);
  return cudaGetLastError();
}

cudaError_t launch_norm(qs_ctx* h, const void* psi, int n, int members, int group, double* out) {
  const int chunks = chunk_count(n);
  if (!ensure_partials(h, (size_t)2 * chunks * members)) return cudaErrorMemoryAllocation;
  dim3 grid(chunks, members);
  if (h->dtype == QS_C64)
    k_norm_partials<float><<<grid, kRBlock, 0, h->stream>>>((const float2*)psi, n, chunks, kChunk, h->partials);
  else
    k_norm_partials<double><<<grid, kRBlock, 0, h->stream>>>((const double2*)psi, n, chunks, kChunk, h->partials);
  k_finalize<<<finalize_blocks(members / group), 256, 0, h->stream>>>(h->partials, members, chunks, 1, group, out);
  return cudaGetLastError();
}

cudaError_t launch_basis_prob(qs_ctx* h, const void* psi, int n, int members, uint64_t x,
                              int group, double* out) {
  const unsigned g = (unsigned)((members / group + 255) / 256);
  if (h->dtype == QS_C64)
    k_basis_prob<float><<<g, 256, 0, h->stream>>>((const float2*)psi, n, members, x, group, out);
  else
    k_basis_prob<double><<<g, 256, 0, h->stream>>>((const double2*)psi, n, members, x, group, out);
  return cudaGetLastError();
}

cudaError_t launch_dm_trace(qs_ctx* h, const void* rho, int n, double* out) {
  const int chunks = chunk_count(n);
  if (!ensure_partials(h, (size_t)2 * chunks)) return cudaErrorMemoryAllocation;
  if (h->dtype == QS_C64)
    k_dm_trace_partials<float><<<chunks, kRBlock, 0, h->stream>>>((const float2*)rho, n, chunks, kChunk, h->partials);
  else
    k_dm_trace_partials<double><<<chunks, kRBlock, 0, h->stream>>>((const double2*)rho, n, chunks, kChunk, h->partials);
  k_finalize<<<1, 32, 0, h->stream>>>(h->partials, 1, chunks, 1, 1, out);
  return cudaGetLastError();
}

cudaError_t launch_dm_expect(qs_ctx* h, const void* rho, const void* phi, int n, double* out) {
  const uint64_t N = 1ull << n;
  if (!ensure_partials(h, (size_t)2 * N)) return cudaErrorMemoryAllocation;
  if (h->dtype == QS_C64)
    k_dm_expect_rows<float><<<(unsigned)N, kRBlock, 0, h->stream>>>((const float2*)rho, (const float2*)phi, n, h->partials);
  else
    k_dm_expect_rows<double><<<(unsigned)N, kRBlock, 0, h->stream>>>((const double2*)rho, (const double2*)phi, n, h->partials);
  // sum of N row partials: treat them as one member with N chunks, real part
  k_finalize<<<1, 32, 0, h->stream>>>(h->partials, 1, (int)N, 1, 1, out);
  return cudaGetLastError();
}

cudaError_t launch_convert_ref(qs_ctx* h, const double* src, void* dst, size_t count) {
  const int g = (int)std::min<size_t>((count + 255) / 256, (size_t)num_sms() * 16);
  if (h->dtype == QS_C64) k_convert_ref<float><<<g, 256, 0, h->stream>>>(src, (float2*)dst, count);
  else k_convert_ref<double><<<g, 256, 0, h->stream>>>(src, (double2*)dst, count);
  return cudaGetLastError();
}

}  // namespace qs
