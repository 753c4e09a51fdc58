// mrg31k3p_core.cuh -- device arithmetic of MRG31k3p (L'Ecuyer and Touzin
// 2000), the base generator of the paper's package (Sec. 2: "MRG31k3p").
//
//   x1[n] = (2^22 x1[n-2] + (2^7 + 1) x1[n-3]) mod m1,  m1 = 2^31 - 1
//   x2[n] = (2^15 x2[n-1] + (2^15 + 1) x2[n-3]) mod m2,  m2 = 2^31 - 21069
//   z[n]  = (x1[n] - x2[n]) mod m1, 0 mapped to m1: an integer in [1, m1]
//           (Sec. 2.2: "an integer between 1 and 2147483647")
//   u     = z / 2^31 (the product with 1/(m1 + 1) = 2^-31 is exact in fp64)
//
// Streams are 2^134 steps apart (Sec. 2.1).  State words are newest first, as
// for MRG32k3a (the Sec. 2.1 printout).  All arithmetic is 32/64-bit integer;
// reductions fold the high part with 2^31 = 1 (mod m1) and
// 2^31 = 21069 (mod m2).
#pragma once
#include <stdint.h>

#include "mrg32k3a_core.cuh"

namespace mrg {
namespace g31 {

constexpr uint32_t M1 = 2147483647u;  // 2^31 - 1
constexpr uint32_t M2 = 2147462579u;  // 2^31 - 21069
constexpr uint32_t C2 = 21069u;       // 2^31 mod m2
constexpr uint32_t MASK31 = 0x7FFFFFFFu;
constexpr int JUMP_BITS = 198;        // A^(2^i), i < 198
constexpr int STREAM_LOG2 = 134;

// t < 2^64 -> t mod m1.
MRG_HD uint32_t red1(uint64_t t) {
  t = (t & MASK31) + (t >> 31);                 // < 2^31 + 2^33
  t = (t & MASK31) + (t >> 31);                 // < 2^31 + 4
  const uint32_t r = (uint32_t)t;
  return r >= M1 ? r - M1 : r;
}

// t < 2^64 -> t mod m2.
MRG_HD uint32_t red2(uint64_t t) {
  t = (t & MASK31) + (t >> 31) * C2;            // < 2^31 + 2^33 * 21069 < 2^48
  t = (t & MASK31) + (t >> 31) * C2;            // < 2^31 + 2^17 * 21069 < 2^33
  t = (t & MASK31) + (t >> 31) * C2;            // < 2^31 + 4 * 21069 = m2 + 5 * 21069
  const uint32_t r = (uint32_t)t;
  return r >= M2 ? r - M2 : r;
}

// One step on canonical words; returns z in [1, m1].
MRG_HD uint32_t step(State& s) {
  // component 1: 2^22 x1[n-2] + 129 x1[n-3] < 2^53 + 2^39
  const uint64_t p = ((uint64_t)s.a1 << 22) + (uint64_t)s.a2 * 129u;
  uint32_t t = (uint32_t)(p & MASK31) + (uint32_t)(p >> 31);   // < 2^31 + 2^23
  t = (t & MASK31) + (t >> 31);                                // <= 2^31 - 1 + 1
  const uint32_t x1 = t >= M1 ? t - M1 : t;
  // component 2: 2^15 x2[n-1] + 32769 x2[n-3] < 2^47
  const uint64_t q = ((uint64_t)s.b0 << 15) + (uint64_t)s.b2 * 32769u;
  const uint64_t u = (q & MASK31) + (q >> 31) * C2;            // < 2^31 + 2^16 * 21069 < 2^32
  const uint32_t v = (uint32_t)(u & MASK31) + (uint32_t)(u >> 31) * C2;  // < 2^31 + 21069
  const uint32_t x2 = v >= M2 ? v - M2 : v;
  s.a2 = s.a1; s.a1 = s.a0; s.a0 = x1;
  s.b2 = s.b1; s.b1 = s.b0; s.b0 = x2;
  // x1 - x2 mod m1 with 0 -> m1: |x1 - x2| < m1 and m2 < m1
  return x1 > x2 ? x1 - x2 : x1 - x2 + M1;
}

// x <- A x mod m for one component (canonical words, entries < 2^31).
template <int COMP>
MRG_HD void matvec(const uint32_t* __restrict__ A, uint32_t& x0, uint32_t& x1, uint32_t& x2) {
  const uint64_t y0 = (uint64_t)A[0] * x0 + (uint64_t)A[1] * x1 + (uint64_t)A[2] * x2;  // < 3 * 2^62
  const uint64_t y1 = (uint64_t)A[3] * x0 + (uint64_t)A[4] * x1 + (uint64_t)A[5] * x2;
  const uint64_t y2 = (uint64_t)A[6] * x0 + (uint64_t)A[7] * x1 + (uint64_t)A[8] * x2;
  if (COMP == 0) { x0 = red1(y0); x1 = red1(y1); x2 = red1(y2); }
  else           { x0 = red2(y0); x1 = red2(y1); x2 = red2(y2); }
}

// fp64 bits of u = z / 2^31 (exact): with s = clz(z) >= 1 and zn = z << s in
// [2^31, 2^32), u = (zn / 2^31) 2^-s: biased exponent 1023 - s and the 53-bit
// significand zn << 21 (its leading one lands in the exponent field).
MRG_HD uint64_t uniform_bits64(uint32_t z) {
  const uint32_t s = clz32(z);
  const uint32_t zn = z << s;
  return ((uint64_t)(1022u - s) << 52) + ((uint64_t)zn << 21);
}

// fp32 bits of RN32(z / 2^31): the 24 leading bits of zn, rounded to nearest
// even on the 8 dropped bits; a carry out of the significand steps the
// exponent (biased 127 - s).
MRG_HD uint32_t uniform_bits32(uint32_t z) {
  const uint32_t s = clz32(z);
  const uint32_t zn = z << s;
  const uint64_t t = (uint64_t)zn + 0x7Fu + ((zn >> 8) & 1u);
  return ((126u - s) << 23) + (uint32_t)(t >> 8);
}

}  // namespace g31
}  // namespace mrg
