// ozaki_round.cuh -- the exact fixed-point result of an Ozaki-sliced product
// rounded once to fp64, for device code and for the host check
// (tests/host_harness).
//
// The product kernels sum the digit products of each level exactly and
// combine the eight levels as T = sum_l acc_l 128^(7-l) = th 2^28 + tl (two
// int64 halves).  With |acc_l| <= (l + 1) 2^19 (l + 1 digit pairs, 128 terms,
// digits of magnitude <= 64), |T| < 2^68.03.  The entry is T 2^E rounded to
// nearest-even:
//   * Th = floor(T / 64) fits an int64 (|Th| < 2^63) and Tl = T mod 64;
//   * when |Th| < 2^56, T itself fits an int64 and one int64 -> fp64
//     conversion (round to nearest) rounds it;
//   * otherwise Th | (Tl != 0) is T / 64 rounded to odd on the integers,
//     with at least 57 significant bits; rounding that to 53 bits gives the
//     round-to-nearest of T / 64 (rounding to odd with two or more extra
//     bits, then to nearest: Boldo and Melquiond, IEEE Trans. Computers 57,
//     2008), and the factor 64 is exact;
//   * the power of two 2^E is applied to the exponent field; results below
//     fp64's normal range are flushed to +0.
#pragma once
#include <stdint.h>
#include <string.h>

namespace mrg {
namespace grf {

__host__ __device__ __forceinline__ double ozaki_i64_to_f64_rn(int64_t x) {
#ifdef __CUDA_ARCH__
  return __ll2double_rn((long long)x);
#else
  return (double)x;   // round to nearest in the default floating-point mode
#endif
}

__host__ __device__ __forceinline__ uint64_t ozaki_f64_bits(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t b;
  memcpy(&b, &d, 8);
  return b;
#endif
}

__host__ __device__ __forceinline__ double ozaki_f64_of_bits(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, 8);
  return d;
#endif
}

// (th 2^28 + tl) 2^E rounded to nearest-even fp64 (|th 2^28 + tl| < 2^68.03,
// |tl| < 2^62); below the normal range +0.
__host__ __device__ __forceinline__ double ozaki_round(int64_t th, int64_t tl, int E) {
  const int64_t Th = (int64_t)((uint64_t)th << 22) + (tl >> 6);   // floor(T / 64)
  const int64_t Tl = tl & 63;
  const bool small = Th >= -(INT64_C(1) << 56) && Th < (INT64_C(1) << 56);
  const int64_t X = small ? (int64_t)((uint64_t)Th << 6) + Tl : (Th | (int64_t)(Tl != 0));
  const int sc = small ? E : E + 6;
  const uint64_t b = ozaki_f64_bits(ozaki_i64_to_f64_rn(X));
  if ((b << 1) == 0) return 0.0;
  const int ex = (int)((b >> 52) & 0x7FF) + sc;
  if (ex <= 0) return 0.0;
  if (ex >= 0x7FF) return ozaki_f64_of_bits((b & 0x8000000000000000ull) | 0x7FF0000000000000ull);
  return ozaki_f64_of_bits(b + ((uint64_t)(int64_t)sc << 52));
}

}  // namespace grf
}  // namespace mrg
