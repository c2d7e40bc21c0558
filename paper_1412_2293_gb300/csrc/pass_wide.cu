// Fused passes with windows of 11 and 12 qubits (complex64): the kernels of
// pass.cuh instantiated for M = 11, 12, in a translation unit of their own so
// the library's units compile in parallel.  One configuration per geometry:
//   low  12 warps, groups of 2^(m-10) warps per tile, one buffer per group;
//   high one block of 16 warps per SM, one buffer: tiles of 2^(14-m) columns
//        x 2^m rows (128 KB), so every row fills whole 32-byte sectors.
// The compiled program of the full window (wide_full_prog) has its own
// instantiation; any other pass runs the interpreted segment list.
#include "pass.cuh"

namespace qs {
namespace fused {

namespace {
constexpr int kWarps = 12;

template <int M>
cudaError_t launch_m(cplx<float>* psi, const CUtensorMap& tmap, const PassArgs& A, bool high, bool full, int sms,
                     cudaStream_t s) {
  using L = LowShape<kWarps, 1, M>;
  constexpr int CB = wide_colb(M);
  using H = HighShape<CB, M>;
  constexpr int FULL = wide_full_prog(M);
  if (!high) {
    const uint64_t blocks = (A.tiles + L::GROUPS - 1) / L::GROUPS;
    const int grid = (int)(blocks < (uint64_t)sms ? blocks : (uint64_t)sms);
    if (full)
      k_pass_low<float, kWarps, 1, FULL, M><<<grid, L::THREADS, low_smem<float, kWarps, 1, M>(), s>>>(psi, A);
    else
      k_pass_low<float, kWarps, 1, 0, M><<<grid, L::THREADS, low_smem<float, kWarps, 1, M>(), s>>>(psi, A);
  } else {
    const int grid = (int)(A.tiles < (uint64_t)sms ? A.tiles : (uint64_t)sms);
    if (full)
      k_pass_high<float, CB, 1, false, FULL, M><<<grid, H::THREADS, high_smem<float, CB, 1, M>(), s>>>(psi, tmap, A);
    else
      k_pass_high<float, CB, 1, false, 0, M><<<grid, H::THREADS, high_smem<float, CB, 1, M>(), s>>>(psi, tmap, A);
  }
  return cudaGetLastError();
}

template <int M>
cudaError_t attrs_m() {
  constexpr int CB = wide_colb(M);
  constexpr int FULL = wide_full_prog(M);
  cudaError_t e = set_pass_attrs(k_pass_low<float, kWarps, 1, 0, M>, low_smem<float, kWarps, 1, M>(), 1);
  if (e == cudaSuccess) e = set_pass_attrs(k_pass_low<float, kWarps, 1, FULL, M>, low_smem<float, kWarps, 1, M>(), 1);
  if (e == cudaSuccess) e = set_pass_attrs(k_pass_high<float, CB, 1, false, 0, M>, high_smem<float, CB, 1, M>(), 1);
  if (e == cudaSuccess) e = set_pass_attrs(k_pass_high<float, CB, 1, false, FULL, M>, high_smem<float, CB, 1, M>(), 1);
  return e;
}
}  // namespace

cudaError_t launch_pass_wide(cplx<float>* psi, const CUtensorMap& tmap, const PassArgs& A, bool high, int m, int prog,
                             int sms, cudaStream_t s) {
  if (m == 11) return launch_m<11>(psi, tmap, A, high, prog == wide_full_prog(11), sms, s);
  if (m == 12) return launch_m<12>(psi, tmap, A, high, prog == wide_full_prog(12), sms, s);
  return cudaErrorInvalidValue;
}

cudaError_t set_wide_attrs() {
  cudaError_t e = attrs_m<11>();
  if (e == cudaSuccess) e = attrs_m<12>();
  return e;
}

}  // namespace fused
}  // namespace qs
