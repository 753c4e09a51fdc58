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
// Modular reductions for the jump-ahead (canonical states, words < m)
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
// The recurrence in offset form.
//
// Inside the generation loops a state word is kept as x~1 = x1 + 209 and
// x~2 = x2 + 22853 (both still < 2^32).  With that offset:
//   * m - x[n-3] is the 32-bit negation of x~[n-3];
//   * the constant parts of the offsets fold into one 64-bit addend K;
//   * after folding the high word with 2^32 = c (mod m), the value v
//     satisfies v = x[n] + c (mod m) and v >= c, and the reduced offset word
//     is x~[n] = low32(v) + c * high32(v): the carry word replaces the usual
//     compare-and-subtract, so the step is multiply-adds (IMAD pipe) plus
//     two negations instead of compare/select chains (ALU pipe).
// ---------------------------------------------------------------------------

constexpr uint64_t K1 = 4001619076ull;  // (209 - 1403580*209) mod m1, >= 209
constexpr uint64_t K2 = 827339146ull;   // (22853 - 527612*22853) mod m2, >= 22853

struct TState {
  uint32_t a0, a1, a2;  // x1 + 209, newest first
  uint32_t b0, b1, b2;  // x2 + 22853, newest first
};

MRG_HD TState to_offset(const State& s) {
  return TState{s.a0 + C1, s.a1 + C1, s.a2 + C1, s.b0 + C2, s.b1 + C2, s.b2 + C2};
}

MRG_HD State from_offset(const TState& t) {
  return State{t.a0 - C1, t.a1 - C1, t.a2 - C1, t.b0 - C2, t.b1 - C2, t.b2 - C2};
}

// One step; returns z in [1, m1].
MRG_HD uint32_t step(TState& s) {
  // component 1: t = 1403580 x1[n-2] + 810728 (m1 - x1[n-3]) + 209  (mod m1)
  uint64_t t = (uint64_t)A13N * (0u - s.a2) + K1;           // < 2^52 + 2^32
  t += (uint64_t)A12 * s.a1;                                 // < 2^54
  uint64_t v = (uint64_t)(uint32_t)(t >> 32) * C1 + (uint32_t)t;      // < 2^33, >= 209
  uint32_t p1 = (uint32_t)v + C1 * (uint32_t)(v >> 32);                // x1[n] + 209
  // component 2: t2 = 527612 x2[n-1] + 1370589 (m2 - x2[n-3]) + 22853  (mod m2)
  uint64_t t2 = (uint64_t)A23N * (0u - s.b2) + K2;          // < 2^53 + 2^33
  t2 += (uint64_t)A21 * s.b0;                                // < 2^54
  uint64_t v2 = (uint64_t)(uint32_t)(t2 >> 32) * C2 + (uint32_t)t2;   // < 2^37
  uint64_t w2 = (uint64_t)(uint32_t)(v2 >> 32) * C2 + (uint32_t)v2;   // < 2^32 + 2^20, >= 22853
  uint32_t p2 = (uint32_t)w2 + C2 * (uint32_t)(w2 >> 32);              // x2[n] + 22853
  s.a2 = s.a1; s.a1 = s.a0; s.a0 = p1;
  s.b2 = s.b1; s.b1 = s.b0; s.b0 = p2;
  // z = x1 - x2 (mod m1) in [1, m1].  With D = x1[n] - x2[n] = p1 - p2 + 22644,
  // H = p1 + (2^32 - p2) + 22643 = D - 1 + 2^32 carries exactly when D >= 1;
  // then z = D = low32(H) + 1, otherwise z = D + m1 = low32(H) - 208.
  uint64_t H = (uint64_t)p1 + (uint32_t)(0u - p2) + 22643u;
  return (uint32_t)H + C1 * (uint32_t)(H >> 32) - 208u;
}

// ---------------------------------------------------------------------------
// Jump-ahead: x <- A^(2^i) x per component (canonical words).
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
// norm = (2^52 + DELTA) 2^-84.  With s = clz(z) and zn = z << s in
// [2^31, 2^32):  z * norm = (zn + e) 2^(-32-s),  e = zn * DELTA / 2^52 < 256.
//   * zn < ZN_BIG (= m1 + 1, i.e. zn + e < 2^32): the 53-bit significand is
//     S = zn 2^21 + RN(t / 2^31), t = zn * DELTA, and the biased exponent
//     1022 - s.  The remainder t mod 2^31 equals 2^30 only for zn = 3 2^30,
//     where the kept part is even, so round-half-down is exactly
//     round-to-nearest-even: RN(t / 2^31) = (t + 2^30 - 1) >> 31.
//   * zn >= ZN_BIG (rare): S = zn 2^20 + RN(t / 2^32), exponent 1023 - s;
//     t mod 2^32 never equals 2^31 there, so no tie.
// bits = ((biased exponent - 1) << 52) + S: a rounding carry out of S steps
// the exponent.  The exponent goes in as the high word of the 64-bit addend,
// so the common path is clz, shift and two multiply-adds.
// ---------------------------------------------------------------------------

constexpr uint32_t ZN_BIG = 4294967088u;

MRG_HD uint64_t uniform_bits64(uint32_t z) {
  uint32_t s = clz32(z);
  uint32_t zn = z << s;
  uint64_t t = (uint64_t)zn * (uint32_t)NORM_DELTA + 0x3FFFFFFFull;   // < 2^60
  uint32_t r = (uint32_t)(t >> 31);                                    // RN(t/2^31), < 2^29 + 1
  uint32_t E = (1021u - s) << 20;
  if (zn >= ZN_BIG) {                                                  // rare
    r = (uint32_t)((t + 0x40000001ull) >> 32);                         // RN(zn*DELTA / 2^32)
    return (uint64_t)zn * (1u << 20) + (((uint64_t)(E + (1u << 20)) << 32) | r);
  }
  return (uint64_t)zn * (1u << 21) + (((uint64_t)E << 32) | r);
}

// fp32 uniform = RN32(the fp64 uniform) (the paper computes the product in
// double and stores it to a float array, Sec. 2.2 Listing 1).  Values are
// normal in both formats (>= 2^-32): bits >> 29 is the rebiased-by-896
// float with a truncated significand; adding 2^28 - 1 + (kept LSB) before
// the shift rounds to nearest-even, a carry stepping the exponent.
MRG_HD uint32_t f32_bits_from_f64(uint64_t d) {
  uint64_t odd = (d >> 29) & 1u;
  return (uint32_t)((d + 0x0FFFFFFFull + odd) >> 29) - (896u << 23);
}

// The same fp32 uniform straight from z, without forming the double.  With
// zn, s and the significand S = zn 2^21 + RN(zn DELTA / 2^31) of the fp64
// uniform above, the float keeps S rounded at bit 29.  Rounding half up
// there is nearest-even for every z (the fp64 significands with a remainder
// of exactly 2^28 all have an odd kept part), and both roundings nest into
// one floor:
//   floor((S + 2^28) / 2^29) = floor((zn 2^52 + zn DELTA + 2^59 + 2^30 - 1) / 2^60)
//                            = floor((zn + h) / 2^8),   h = floor(t / 2^52),
// with t = zn DELTA + 2^59 + 2^30 - 1 < 2^61 (one wide multiply-add).  The
// float is ((125 - s) << 23) + that 24-bit significand, whose carry into
// 2^24 steps the exponent.  When zn + h passes 2^32 the value rounds up to
// 2^-s exactly (significand 2^24) -- for zn >= ZN_BIG, where the double
// itself lies in the next binade, the float is 2^-s too.  Checked against
// RN32 of the IEEE product for every z on the host.
MRG_HD uint32_t uniform_bits32(uint32_t z) {
  const uint32_t s = clz32(z);
  const uint32_t zn = z << s;
  const uint64_t t = (uint64_t)zn * (uint32_t)NORM_DELTA + ((1ull << 59) + (1ull << 30) - 1);
  const uint32_t sum = zn + (uint32_t)(t >> 52);
  const uint32_t m = sum < zn ? (1u << 24) : (sum >> 8);
  return ((125u - s) << 23) + m;
}

// ---------------------------------------------------------------------------
// Device fast paths: the same arithmetic written as PTX so that ptxas keeps
// the multiply-adds on the IMAD pipe and the fold carries as predicated adds
// (the portable versions above are the specification; the host harness and
// the GPU tests check that both agree bit for bit).
// ---------------------------------------------------------------------------
// NEG_ALU: the two negations 2^32 - x of a step written as subtractions from
// zero instead of multiply-adds by 2^32 - 1 (the form the step used first).
// The per-draw instruction and pipe counts of the two forms barely differ
// (ncu), but ptxas schedules the surrounding code differently, and the
// times do differ: per 2^30 outputs the subtraction form took the fp32
// uniforms 1.544 -> 1.503 ms and the fp32 exponentials 2.243 -> 2.216, the
// fp64 uniforms about 1 % less, the fp64 exponentials 3.65 -> 3.59, and the
// fp32 normals 2.972 -> 3.010 and the fused consumer 13.85 -> 13.89 (2^32
// draws), so each caller chooses.
template <bool NEG_ALU = false>
__device__ __forceinline__ uint32_t step_fast(TState& s, uint64_t k1, uint64_t k2) {
#ifndef __CUDA_ARCH__
  return step(s);  // host compilation pass only; never executed on the host
#else
  uint32_t p1, p2, z, na2, nb2;
  if constexpr (NEG_ALU) {
    asm("sub.u32 %0, 0, %1;" : "=r"(na2) : "r"(s.a2));
    asm("sub.u32 %0, 0, %1;" : "=r"(nb2) : "r"(s.b2));
  } else {
    asm("mad.lo.u32 %0, %1, 0xFFFFFFFF, 0;" : "=r"(na2) : "r"(s.a2));
    asm("mad.lo.u32 %0, %1, 0xFFFFFFFF, 0;" : "=r"(nb2) : "r"(s.b2));
  }
  // component 1: t = 810728 (2^32 - a2) + K1 + 1403580 a1 ; one fold, carry adds 209
  asm("{\n\t.reg .u32 lo, hi, vl;\n\t.reg .u64 t;\n\t.reg .pred c;\n\t"
      "mad.wide.u32 t, %1, 810728, %3;\n\t"
      "mad.wide.u32 t, %2, 1403580, t;\n\t"
      "mov.b64 {lo, hi}, t;\n\t"
      "mad.lo.u32 vl, hi, 209, lo;\n\t"
      "setp.lt.u32 c, vl, lo;\n\t"
      "@c add.u32 vl, vl, 209;\n\t"
      "mov.u32 %0, vl;\n\t}"
      : "=r"(p1) : "r"(na2), "r"(s.a1), "l"(k1));
  // component 2: t = 1370589 (2^32 - b2) + K2 + 527612 b0 ; two folds
  asm("{\n\t.reg .u32 lo, hi, vl, vh, wl;\n\t.reg .u64 t, v;\n\t.reg .pred c;\n\t"
      "mad.wide.u32 t, %1, 1370589, %3;\n\t"
      "mad.wide.u32 t, %2, 527612, t;\n\t"
      "mov.b64 {lo, hi}, t;\n\t"
      "mad.wide.u32 v, hi, 22853, t;\n\t"       // hi*22853 + lo + hi*2^32
      "mov.b64 {vl, vh}, v;\n\t"
      "sub.u32 vh, vh, hi;\n\t"                  // drop hi*2^32
      "mad.lo.u32 wl, vh, 22853, vl;\n\t"
      "setp.lt.u32 c, wl, vl;\n\t"
      "@c add.u32 wl, wl, 22853;\n\t"
      "mov.u32 %0, wl;\n\t}"
      : "=r"(p2) : "r"(nb2), "r"(s.b0), "l"(k2));
  s.a2 = s.a1; s.a1 = s.a0; s.a0 = p1;
  s.b2 = s.b1; s.b1 = s.b0; s.b0 = p2;
  // z: h = p1 + (22643 - p2) carries exactly when D >= 1, i.e. when h < p1;
  // z = h + 209 c - 208 (the carry as a predicated add keeps it off the
  // IMAD pipe, which the step's wide products already fill)
  asm("{\n\t.reg .u32 q, h;\n\t.reg .pred c;\n\t"
      "sub.u32 q, 22643, %2;\n\t"
      "add.u32 h, %1, q;\n\t"
      "setp.lt.u32 c, h, %1;\n\t"
      "@c add.u32 h, h, 209;\n\t"
      "sub.u32 %0, h, 208;\n\t}"
      : "=r"(z) : "r"(p1), "r"(p2));
  return z;
#endif
}

__device__ __forceinline__ uint64_t uniform_bits64_fast(uint32_t z) {
#ifndef __CUDA_ARCH__
  return uniform_bits64(z);  // host compilation pass only
#else
  uint32_t zn, s, r, E, lo, hi;
  asm("bfind.shiftamt.u32 %0, %1;" : "=r"(s) : "r"(z));
  zn = z << s;
  uint64_t t;
  asm("mad.wide.u32 %0, %1, 218103819, 0x3FFFFFFF;" : "=l"(t) : "r"(zn));
  asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(t));
  asm("shf.r.clamp.b32 %0, %1, %2, 31;" : "=r"(r) : "r"(lo), "r"(hi));
  asm("mad.lo.u32 %0, %1, 0xFFF00000, 0x3FD00000;" : "=r"(E) : "r"(s));   // (1021 - s) << 20
  uint64_t a, b;
  if (__builtin_expect(zn >= ZN_BIG, 0)) {
    r = (uint32_t)((t + 0x40000001ull) >> 32);
    asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "r"(r), "r"(E + (1u << 20)));
    asm("mad.wide.u32 %0, %1, 1048576, %2;" : "=l"(b) : "r"(zn), "l"(a));
    return b;
  }
  asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "r"(r), "r"(E));
  asm("mad.wide.u32 %0, %1, 2097152, %2;" : "=l"(b) : "r"(zn), "l"(a));
  return b;
#endif
}

}  // namespace mrg
