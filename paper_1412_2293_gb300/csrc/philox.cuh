// Counter-based noise draw of the Monte Carlo method (Sec. 2, Eq. 1).
//
// Philox4x32 with 10 rounds, as defined by Salmon, Moraes, Dror and Shaw,
// "Parallel random numbers: as easy as 1, 2, 3" (SC'11).  The noise of
// trajectory `traj` at gate `gate_id` under key `seed` is
//   words  = Philox4x32_10(counter = (traj lo, traj hi, gate lo, gate hi),
//                          key = (seed lo, seed hi))
//   u1, u2 = ((64-bit word pair >> 11) + 0.5) * 2^-53   (open interval)
//   xi_a   = sqrt(-2 ln u1) cos(2 pi u2),  xi_b = sqrt(-2 ln u1) sin(2 pi u2)
// (Box-Muller).  The integer words are exact; the normals use the CUDA FP64
// log / sincos.
#pragma once

#include <cstdint>

namespace qs {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

struct Words4 { uint32_t w[4]; };

__device__ __forceinline__ Words4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += kPhiloxW0; k1 += kPhiloxW1; }
    const uint32_t hi0 = __umulhi(kPhiloxM0, c0), lo0 = kPhiloxM0 * c0;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c2), lo1 = kPhiloxM1 * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  Words4 out;
  out.w[0] = c0; out.w[1] = c1; out.w[2] = c2; out.w[3] = c3;
  return out;
}

__device__ __forceinline__ Words4 noise_words(uint64_t seed, uint64_t traj, uint64_t gate_id) {
  return philox4x32_10((uint32_t)traj, (uint32_t)(traj >> 32), (uint32_t)gate_id,
                       (uint32_t)(gate_id >> 32), (uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ __forceinline__ double open_uniform53(uint32_t hi, uint32_t lo) {
  const uint64_t v = ((((uint64_t)hi) << 32) | lo) >> 11;
  return ((double)v + 0.5) * 0x1.0p-53;
}

// (xi_a, xi_b)
__device__ __forceinline__ double2 noise_normals(uint64_t seed, uint64_t traj, uint64_t gate_id) {
  const Words4 w = noise_words(seed, traj, gate_id);
  const double u1 = open_uniform53(w.w[0], w.w[1]);
  const double u2 = open_uniform53(w.w[2], w.w[3]);
  const double r = sqrt(-2.0 * log(u1));
  // same double argument as the host definition: (2 pi) * u2
  double s, c;
  sincos(2.0 * 3.141592653589793 * u2, &s, &c);
  return make_double2(r * c, r * s);
}

// The same draw with the logarithm, square root and cosine/sine evaluated in
// FP32 (for complex64 simulation, where the noise angle only enters FP32
// arithmetic): the words and uniforms are as above; the normals agree with
// the FP64 ones to a few FP32 ulp.
__device__ __forceinline__ float2 noise_normals_f32(uint64_t seed, uint64_t traj, uint64_t gate_id) {
  const Words4 w = noise_words(seed, traj, gate_id);
  const float u1 = (float)open_uniform53(w.w[0], w.w[1]);
  const float u2 = (float)open_uniform53(w.w[2], w.w[3]);
  const float r = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);                         // sin, cos of 2 pi u2
  return make_float2(r * c, r * s);
}

}  // namespace qs
