// transforms_f64.cuh -- normal and exponential transforms evaluated in FP64.
//
// The transforms are defined on the exact rational uniform u = z / M,
// M = m1 + 1, z in [1, m1]:
//   Box-Muller (Sec. 3.1, Algorithm 1): R = sqrt(-2 ln u1), Theta = 2 pi u2,
//     X = R cos Theta, Y = R sin Theta, on consecutive draws (u1, u2) of one
//     stream;
//   exponential (Sec. 3.2): E = -ln(u) / rate.
// Two exact integer reductions keep relative accuracy where the result is
// small: ln u uses log1p(-(M - z)/M) above u = 1/2, and the angle is reduced
// in integers, 4z = q M + r, Theta = (pi/2) q + (pi/2) r / M, with the octant
// reflection r -> M - r so that sin/cos see an argument in [0, pi/4].
#pragma once
#include <stdint.h>

#include "mrg32k3a_core.cuh"

namespace mrg {

constexpr double NORM = 1.0 / 4294967088.0;  // RN64(1/(m1+1)), folded exactly by the compiler

__device__ __forceinline__ double ln_u_f64(uint32_t z) {
  if (z > 2147483544u) {                      // 2z > M
    uint32_t c = (uint32_t)(MNORM - z);       // exact complement, < M/2
    return log1p(-(double)c * NORM);
  }
  return log((double)z * NORM);
}

// sin and cos of 2 pi z / M.
__device__ __forceinline__ void sincos_turn_f64(uint32_t z, double& s, double& c) {
  uint64_t t = 4ull * z;
  uint32_t q = (uint32_t)(t >= MNORM) + (uint32_t)(t >= 2 * MNORM) + (uint32_t)(t >= 3 * MNORM);
  uint32_t r = (uint32_t)(t - (uint64_t)q * MNORM);  // in [0, M)
  bool refl = 2ull * r > MNORM;
  uint32_t rr = refl ? (uint32_t)(MNORM - r) : r;    // <= M/2
  double sp, cp;
  sincospi((double)rr * (0.5 * NORM), &sp, &cp);      // phi = (pi/2) rr / M
  if (refl) { double t2 = sp; sp = cp; cp = t2; }
  switch (q) {
    case 0: s = sp;  c = cp;  break;
    case 1: s = cp;  c = -sp; break;
    case 2: s = -sp; c = -cp; break;
    default: s = -cp; c = sp; break;
  }
}

__device__ __forceinline__ void box_muller_f64(uint32_t z1, uint32_t z2, double& x, double& y) {
  double R = sqrt(-2.0 * ln_u_f64(z1));
  double s, c;
  sincos_turn_f64(z2, s, c);
  x = R * c;
  y = R * s;
}

__device__ __forceinline__ double exponential_f64(uint32_t z, double inv_rate) {
  return -ln_u_f64(z) * inv_rate;
}

}  // namespace mrg
