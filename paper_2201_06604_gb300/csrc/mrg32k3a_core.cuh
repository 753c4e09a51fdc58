// mrg32k3a_core.cuh -- device arithmetic of the MRG32k3a hot path (sm_103a).
//
// The generator (the combined MRG of L'Ecuyer 1999, named in Sec. 1 and 2 as
// the generator of RngStreams): two order-3 components
//   x1[n] = (1403580 x1[n-2] -  810728 x1[n-3]) mod m1,  m1 = 2^32 - 209
//   x2[n] = ( 527612 x2[n-1] - 1370589 x2[n-3]) mod m2,  m2 = 2^32 - 22853
// and the output z[n] = (x1[n] - x2[n]) mod m1, with 0 mapped to m1, so that
// z lies in [1, m1] (the paper's generator maps its output the same way,
// Sec. 2.2).  Streams are 2^127 steps apart and substreams 2^76 (Sec. 2.1:
// a new stream jumps ahead by Z from the previous one).
//
// Everything here is exact 32/64-bit integer arithmetic: products are
// 32x32->64 (one IMAD.WIDE), and reductions fold the high word with
// 2^32 = 209 (mod m1) and 2^32 = 22853 (mod m2).  No FP64 instruction is on
// the recurrence or on the uniform transforms: GB300's FP64 pipe is a small
// fraction of its integer throughput.
//
// State words are kept newest first, the order of the paper's stream printout
// (Sec. 2.1): (x1[n-1], x1[n-2], x1[n-3], x2[n-1], x2[n-2], x2[n-3]).
#pragma once
#include <stdint.h>

#define MRG_HD __host__ __device__ __forceinline__

namespace mrg {

constexpr uint32_t M1 = 4294967087u;     // 2^32 - 209
constexpr uint32_t M2 = 4294944443u;     // 2^32 - 22853
constexpr uint32_t C1 = 209u;            // 2^32 mod m1
constexpr uint32_t C2 = 22853u;          // 2^32 mod m2
constexpr uint32_t A12 = 1403580u;       // x1 coefficient of x1[n-2]
constexpr uint32_t A13N = 810728u;       // minus the coefficient of x1[n-3]
constexpr uint32_t A21 = 527612u;        // x2 coefficient of x2[n-1]
constexpr uint32_t A23N = 1370589u;      // minus the coefficient of x2[n-3]
constexpr uint64_t MNORM = 4294967088ull; // m1 + 1

// norm = RN64(1/(m1+1)) = (2^52 + NORM_DELTA) * 2^-84.  The host checks this
// against 1.0/(m1+1) at library load.
constexpr uint64_t NORM_DELTA = 218103819ull;

// Jump tables: A_c^(2^i) mod m_c for i in [0, JUMP_BITS), row-major 3x3.
// Bits 0..127 cover any offset inside a stream, 127+j the j-th bit of a
// stream index (the period ~2^191 holds 2^64 streams).
constexpr int JUMP_BITS = 191;
constexpr int STREAM_LOG2 = 127;
constexpr int SUBSTREAM_LOG2 = 76;

struct State {
  uint32_t a0, a1, a2;  // x1[n-1], x1[n-2], x1[n-3]
  uint32_t b0, b1, b2;  // x2[n-1], x2[n-2], x2[n-3]
};

MRG_HD uint32_t clz32(uint32_t x) {
#ifdef __CUDA_ARCH__
  return __clz(x);
#else
  return x ? __builtin_clz(x) : 32;
#endif
}

// ---------------------------------------------------------------------------
// Modular reductions
// ---------------------------------------------------------------------------

// t < 2^54  ->  t mod m1.
MRG_HD uint32_t red1(uint64_t t) {
  uint32_t hi = (uint32_t)(t >> 32), lo = (uint32_t)t;      // hi < 2^22
  uint64_t r = (uint64_t)hi * C1 + lo;                       // < 2^33
  uint32_t rh = (uint32_t)(r >> 32), rl = (uint32_t)r;       // rh in {0,1}
  uint32_t r2 = rl + rh * C1;                                // no wrap: rh=1 -> rl < 2^30
  return r2 >= M1 ? r2 - M1 : r2;                            // r2 < 2^32 < 2 m1
}

// t < 2^54  ->  t mod m2.
MRG_HD uint32_t red2(uint64_t t) {
  uint32_t hi = (uint32_t)(t >> 32), lo = (uint32_t)t;      // hi < 2^22
  uint64_t r = (uint64_t)hi * C2 + lo;                       // < 2^37
  uint32_t rh = (uint32_t)(r >> 32), rl = (uint32_t)r;       // rh <= 23
  uint64_t r2 = (uint64_t)rh * C2 + rl;                      // < 2^32 + 2^20
  uint32_t r2h = (uint32_t)(r2 >> 32), r2l = (uint32_t)r2;   // r2h in {0,1}
  uint32_t r3 = r2l + r2h * C2;                              // no wrap: r2h=1 -> r2l < 2^20
  return r3 >= M2 ? r3 - M2 : r3;                            // r3 < 2^32 < 2 m2
}

// ---------------------------------------------------------------------------
// One step of the recurrence; returns z in [1, m1].
// ---------------------------------------------------------------------------
MRG_HD uint32_t step(State& s) {
  // x1[n] = A12 x1[n-2] + A13N (m1 - x1[n-3])  (mod m1); both terms < 2^53
  uint32_t p1 = red1((uint64_t)A12 * s.a1 + (uint64_t)A13N * (M1 - s.a2));
  // x2[n] = A21 x2[n-1] + A23N (m2 - x2[n-3])  (mod m2); sum < 2^54
  uint32_t p2 = red2((uint64_t)A21 * s.b0 + (uint64_t)A23N * (M2 - s.b2));
  s.a2 = s.a1; s.a1 = s.a0; s.a0 = p1;
  s.b2 = s.b1; s.b1 = s.b0; s.b0 = p2;
  return p1 > p2 ? p1 - p2 : p1 - p2 + M1;   // p2 < m2 < m1: result in [1, m1]
}

// ---------------------------------------------------------------------------
// Jump-ahead: x <- A^(2^i) x per component, tables in constant memory.
// ---------------------------------------------------------------------------

// (a * x) folded once: congruent to a*x mod m, < 2^48.
template <uint32_t C>
MRG_HD uint64_t mulfold(uint32_t a, uint32_t x) {
  uint64_t p = (uint64_t)a * x;
  return (uint64_t)(uint32_t)(p >> 32) * C + (uint32_t)p;
}

template <int COMP>
MRG_HD void matvec(const uint32_t* __restrict__ A, uint32_t& x0,
                                       uint32_t& x1, uint32_t& x2) {
  constexpr uint32_t C = COMP == 0 ? C1 : C2;
  uint64_t y0 = mulfold<C>(A[0], x0) + mulfold<C>(A[1], x1) + mulfold<C>(A[2], x2);
  uint64_t y1 = mulfold<C>(A[3], x0) + mulfold<C>(A[4], x1) + mulfold<C>(A[5], x2);
  uint64_t y2 = mulfold<C>(A[6], x0) + mulfold<C>(A[7], x1) + mulfold<C>(A[8], x2);
  if (COMP == 0) { x0 = red1(y0); x1 = red1(y1); x2 = red1(y2); }
  else           { x0 = red2(y0); x1 = red2(y1); x2 = red2(y2); }
}

// ---------------------------------------------------------------------------
// fp64 uniform u = RN64(z * norm), built exactly in integers.
//
// With s = clz(z), zn = z << s in [2^31, 2^32):  z * norm = P * 2^(-84-s),
// P = zn * (2^52 + NORM_DELTA) = zn * 2^52 + zn * NORM_DELTA  in [2^83, 2^85).
// The 53 leading bits of P rounded to nearest-even give the significand;
// adding it (hidden bit included) to (biased exponent - 1) << 52 lets a
// rounding carry step the exponent.  Bit-identical to the IEEE product
// (double)z * norm, which an FP64 DMUL would compute.
// ---------------------------------------------------------------------------
MRG_HD uint64_t uniform_bits64(uint32_t z) {
  uint32_t s = clz32(z);
  uint32_t zn = z << s;
  uint64_t t = (uint64_t)zn * (uint32_t)NORM_DELTA;     // < 2^60
  uint32_t lo = (uint32_t)t;
  uint64_t H = ((uint64_t)zn << 20) + (t >> 32);        // P >> 32, in [2^51, 2^53)
  bool big = (H >> 52) != 0;                            // P >= 2^84
  uint64_t S = big ? H : ((H << 1) | (lo >> 31));       // 53-bit significand
  uint32_t R = big ? lo : (lo << 1);                    // discarded bits, left-aligned
  uint32_t eb = (big ? 1023u : 1022u) - s;              // biased exponent
  uint32_t up = (R > 0x80000000u) | ((R == 0x80000000u) & (uint32_t)S);
  return ((uint64_t)(eb - 1) << 52) + S + up;
}

// fp32 uniform = RN32(the fp64 uniform) (the paper computes the product in
// double and stores it to a float array, Sec. 2.2 Listing 1).  Values are
// normal in both formats (>= 2^-32), so rounding the 53-bit significand to 24
// bits with nearest-even and re-biasing the exponent is exact.
MRG_HD uint32_t f32_bits_from_f64(uint64_t d) {
  uint32_t hi = (uint32_t)(d >> 32), lo = (uint32_t)d;
  uint32_t e = (hi >> 20) - 1023u + 127u;               // rebias
  uint32_t m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);     // top 23 fraction bits
  uint32_t rest = lo & 0x1FFFFFFFu;                     // 29 discarded bits
  uint32_t up = (rest > 0x10000000u) | ((rest == 0x10000000u) & m);
  return ((e << 23) | m) + up;                          // carry steps the exponent
}

}  // namespace mrg
