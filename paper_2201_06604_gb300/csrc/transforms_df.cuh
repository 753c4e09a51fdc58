// transforms_df.cuh -- normal and exponential transforms in double-float
// arithmetic (pairs of fp32 values, ~46 significant bits) on the FP32 pipe.
//
// GB300 executes FP64 at a small fraction of its FP32 rate, so the
// transforms are evaluated as unevaluated sums hi + lo of two floats with
// error-free products (FMA) and sums; every add and multiply of the
// error-free transformations uses the __f*_rn intrinsics so that the compiler
// never contracts or reassociates them.
//
// Definitions (on the exact rational uniform u = z / M, M = m1 + 1):
//   Box-Muller (Sec. 3.1, Algorithm 1): R = sqrt(-2 ln u1), Theta = 2 pi u2,
//     X = R cos Theta, Y = R sin Theta;
//   exponential (Sec. 3.2): E = -ln(u) / rate.
//
// ln u (relative error ~2^-46 outside the top bucket; inside it, where
// ln u is ln(1 + r) itself, the Taylor terms from r^3 on (up to 2^-17.6 |r|)
// are summed in fp32, which bounds it at ~2^-40 -- 1.3e-12 relative, measured):
//   z = zn 2^-s with zn in [2^31, 2^32); bucket k = the 7 bits after the
//   leading one; C_k = the bucket centre 2^31 + (2k+1) 2^23, except the top
//   bucket whose centre is M itself.  With d = zn - C_k (exact, |d| < 2^24)
//   and r = d / C_k (|r| <= 2^-8):
//     ln u = ln(C_k / (M 2^s)) + ln(1 + r),
//   the first term from a table over all 32 shifts s and 128 buckets k (a
//   float pair each), ln(1 + r) by its Taylor series to r^6.  For z >= 2^31
//   in the top bucket the table term is exactly zero, so ln u = ln(1 + r)
//   keeps its relative accuracy as u -> 1.
// sin / cos of 2 pi z / M (absolute error ~2^-47, relative near zeros):
//   exact integer reduction z = q D + w, D = M / 4, w in [0, D); reflection
//   w -> D - w above D/2 (swapping sin and cos); bucket j = (w + 2^22) >> 23
//   with table angle a_j = (pi/2) j 2^23 / D and residual
//   delta = (pi/2)(w - j 2^23) / D, |delta| <= 0.0062; sin/cos(delta) by
//   Taylor series and the angle-addition formulas.  Bucket 0 has a_0 = 0
//   (sin 0 = 0, cos 0 = 1 exactly), so small angles keep their relative
//   accuracy and an exact zero of sin or cos comes out as exactly zero.
#pragma once
#include <stdint.h>

#include "mrg32k3a_core.cuh"

namespace mrg {

struct df {
  float hi, lo;
};

// Table layout (float4 units), built on the host (host_jump.cpp) and
// copied to shared memory by every block that transforms (42.1 KB):
//   [0, 64)      log: 128 float pairs (1/C_k).hi, (1/C_k).lo (pair k)
//   [64, 584)    trig: sin(a_j).hi, sin(a_j).lo, cos(a_j).hi, cos(a_j).lo,
//                eight copies of each entry side by side (entry j, copy c
//                at 64 + 8 j + c).  A 16-byte load serves a quarter warp
//                (8 lanes, 32 banks) per shared-memory wavefront; lane l
//                reads copy l mod 8, which sits in banks 4c .. 4c + 3 for
//                every j, so the lane-divergent lookup never conflicts (one
//                copy cost ~2.6 wavefronts per quarter warp).
//   [584, 2632)  4096 float pairs: ln(C_k / (M 2^s)).hi, .lo at pair
//                128 s + k (one load replaces -s ln 2 and its error-free sum)
constexpr int TAB_LOG = 0;
constexpr int TAB_TRIG = 64;
constexpr int TRIG_COPIES = 8;
constexpr int TAB_LS = TAB_TRIG + 65 * TRIG_COPIES;
constexpr int TAB_ENTRIES = TAB_LS + 2048;

// 1 / C_k as a float pair.
__device__ __forceinline__ float2 log_inv_ck(const float4* __restrict__ tab, uint32_t k) {
  return reinterpret_cast<const float2*>(tab + TAB_LOG)[k];
}

// ln(C_k / (M 2^s)) as a float pair.
__device__ __forceinline__ float2 log_ck_shift(const float4* __restrict__ tab, uint32_t s, uint32_t k) {
  return reinterpret_cast<const float2*>(tab + TAB_LS)[(s << 7) | k];
}

// sin(a_j) and cos(a_j) as float pairs, from this lane's copy.
__device__ __forceinline__ float4 trig_entry(const float4* __restrict__ tab, uint32_t j) {
  return tab[TAB_TRIG + j * TRIG_COPIES + (threadIdx.x & (TRIG_COPIES - 1))];
}

// The modulus M of the uniform u = z / M that the transforms take, with the
// constants of its reductions.  The tables of each M come from the host
// (transform_table / transform_table_m32) and are passed in `tab`.
struct UM32k3a {                                  // M = m1 + 1 of MRG32k3a
  static constexpr uint32_t TOP_CK = 4294967088u; // centre of the top log bucket: M
  static constexpr uint32_t D = 1073741772u;      // M / 4
  static constexpr uint32_t QFIX = 52u;           // 2^30 - D
  static constexpr float PID_HI = 0x1.921fb6p-30f;  // RN32(pi / (2 D))
  static constexpr float PID_LO = 0x1.15f92cp-55f;  // RN32(pi / (2 D) - PID_HI)
};
struct UM2p32 {                                   // M = 2^32 (MRG31k3p: z' = 2 z)
  static constexpr uint32_t TOP_CK = 0u;          // M mod 2^32: zn - M as a signed word
  static constexpr uint32_t D = 1073741824u;      // 2^30
  static constexpr uint32_t QFIX = 0u;
  static constexpr float PID_HI = 0x1.921fb6p-30f;  // RN32(pi / 2^31)
  static constexpr float PID_LO = -0x1.777a5cp-55f; // RN32(pi / 2^31 - PID_HI)
};

__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  return df{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  return df{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ df df_mul(df x, df y) {
  float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ df df_mul_f(df x, float f) {
  float p = __fmul_rn(x.hi, f);
  float e = __fmaf_rn(x.hi, f, -p);
  e = __fmaf_rn(x.lo, f, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ df df_neg(df x) { return df{-x.hi, -x.lo}; }

// x + y when |x.hi| >= |y.hi| or x.hi = 0 (the order is known): the
// error-free sum of the leading parts needs no magnitude test.
__device__ __forceinline__ df df_add_ordered(df x, df y) {
  const df s = fast_two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

// x * y for a df x and a small df y as (leading product, exact) + (the rest,
// in fp32): the cross terms are below 2^-24 of the product, so their own
// rounding stays below 2^-48 of it.
__device__ __forceinline__ df df_mul_split(df x, df y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return df{p, e};  // not renormalised: p + e with |e| << |p|
}

// Small exact integer (|v| < 2^22) to float without the conversion unit.
__device__ __forceinline__ float small_int_to_float(int32_t v) {
  return __fsub_rn(__int_as_float(0x4B400000 + v), 12582912.0f);
}

// ln(z / M) for z in [1, M - 1].
template <class UM>
__device__ __forceinline__ df ln_u_df_m(uint32_t z, const float4* __restrict__ tab) {
  uint32_t s;
  asm("bfind.shiftamt.u32 %0, %1;" : "=r"(s) : "r"(z));
  const uint32_t zn = z << s;
  const uint32_t k = (zn >> 24) & 127u;
  const uint32_t ck = k == 127u ? UM::TOP_CK : 0x80800000u + (k << 24);
  const int32_t d = (int32_t)(zn - ck);                 // |d| < 2^24: exact in fp32
  const float2 T = log_inv_ck(tab, k);
  // r = d / C_k as the exact leading product plus the rest (not
  // renormalised: every use below takes both parts)
  const float dfl = (float)d;
  const float rp = __fmul_rn(T.x, dfl);
  const df r{rp, __fmaf_rn(T.y, dfl, __fmaf_rn(T.x, dfl, -rp))};
  // ln(1 + r) = r - r^2/2 + r^3 (1/3 - r/4 + r^2/5 - r^3/6)
  const float rh = r.hi;
  const float p2 = __fmul_rn(rh, rh);
  const float e2 = __fmaf_rn(2.0f * rh, r.lo, __fmaf_rn(rh, rh, -p2));   // r^2 = p2 + e2
  float poly = __fmaf_rn(rh, -1.0f / 6.0f, 0.2f);
  poly = __fmaf_rn(rh, poly, -0.25f);
  poly = __fmaf_rn(rh, poly, 1.0f / 3.0f);
  const float c3 = __fmul_rn(__fmul_rn(p2, rh), poly);
  // |r| < 2^-7, so |r| >= r^2 / 2: the order of the sum is known
  df l1p = df_add_ordered(r, df{-0.5f * p2, __fmaf_rn(-0.5f, e2, c3)});
  // ln(C_k / (M 2^s)) + ln(1 + r): |ln(C_k / (M 2^s))| >= ln 2 when s > 0,
  // and |ln(C_k / M)| >= |ln(1 + r)| outside the top bucket (where the table
  // term is exactly 0), so the order of the sum is known.
  const float2 L = log_ck_shift(tab, s, k);
  return df_add_ordered(df{L.x, L.y}, l1p);
}

// ln(z / M) to ~2^-34 relative, for fp32 outputs (whose 2-ulp budget is
// 2^-23): the same reduction and error-free leading parts as ln_u_df_m --
// the product r = d / C_k kept with its rounding error (which alone would
// be a whole fp32 ulp of the result near u = 1 - 2^-8), and the three terms
// added largest first -- but the Taylor tail and the low parts in plain
// fp32, renormalised once at the end.
template <class UM>
__device__ __forceinline__ df ln_u_lite_raw_m(uint32_t z, const float4* __restrict__ tab) {
  uint32_t s;
  asm("bfind.shiftamt.u32 %0, %1;" : "=r"(s) : "r"(z));
  const uint32_t zn = z << s;
  const uint32_t k = (zn >> 24) & 127u;
  const uint32_t ck = k == 127u ? UM::TOP_CK : 0x80800000u + (k << 24);
  const float df_ = (float)(int32_t)(zn - ck);          // |d| < 2^24: exact
  const float2 T = log_inv_ck(tab, k);
  const float rh = __fmul_rn(T.x, df_);
  const float re = __fmaf_rn(T.y, df_, __fmaf_rn(T.x, df_, -rh));   // r = rh + re
  // ln(1 + r) - r = r^2 (-1/2 + r (1/3 + r (-1/4 + r (1/5 - r / 6))))
  float poly = __fmaf_rn(rh, -1.0f / 6.0f, 0.2f);
  poly = __fmaf_rn(rh, poly, -0.25f);
  poly = __fmaf_rn(rh, poly, 1.0f / 3.0f);
  poly = __fmaf_rn(rh, poly, -0.5f);
  // re + the tail r^2 poly, rounded once (an FMA: the packed evaluation's
  // compiler would fuse a separate product into the add anyway)
  const float rt = __fmaf_rn(__fmul_rn(rh, rh), poly, re);
  const float2 L = log_ck_shift(tab, s, k);
  const df u = fast_two_sum(L.x, rh);        // |ln(C_k / (M 2^s))| >= |r|, or both 0
  const float lo = __fadd_rn(u.lo, __fadd_rn(L.y, rt));
  return df{u.hi, lo};  // not renormalised: in the top bucket |lo| reaches 2^-9 |hi|
}

// The same, renormalised (the square root's single correction step needs
// |lo| <= ulp(hi)).
template <class UM>
__device__ __forceinline__ df ln_u_lite_m(uint32_t z, const float4* __restrict__ tab) {
  const df l = ln_u_lite_raw_m<UM>(z, tab);
  return fast_two_sum(l.hi, l.lo);
}

// sqrt of a positive df (relative error ~2^-46) as r0 + c, not renormalised
// (|c| is about 2^-23 r0 at most).
__device__ __forceinline__ df df_sqrt_raw(df x) {
  float y = rsqrtf(x.hi);
  y = __fmul_rn(y, __fmaf_rn(-0.5f * x.hi, __fmul_rn(y, y), 1.5f));   // one Newton step
  const float r0 = __fmul_rn(x.hi, y);
  const float e = __fadd_rn(__fmaf_rn(-r0, r0, x.hi), x.lo);           // x - r0^2
  return df{r0, __fmul_rn(__fmul_rn(e, y), 0.5f)};
}

// RN32 of a * b for a df a and b (unnormalised pairs allowed): the cross
// terms in fp32, the leading product and the sum rounded once by the FMA
// (the dropped a.lo b.lo and the cross terms' rounding are ~2^-46 of it).
__device__ __forceinline__ float df_mul_to_f32(df a, float b_hi, float b_lo) {
  return __fmaf_rn(a.hi, b_hi, __fmaf_rn(a.hi, b_lo, __fmul_rn(a.lo, b_hi)));
}

// The exact reduction of the angle 2 pi z / M, z in [1, M - 1]: quadrant q
// (z = q D + w, w in [0, D)), reflection w -> D - w above D / 2, table
// bucket j and the bucket residual dwf (an exact float in [-2^22, 2^22)).
// (The residual as an integer dw, |dw| <= 2^22; turn_reduce converts it.)
template <class UM>
__device__ __forceinline__ void turn_reduce_int(uint32_t z, uint32_t& q, bool& refl, uint32_t& j,
                                                int32_t& dw) {
  constexpr uint32_t D = UM::D;  // M / 4
  q = z >> 30;
  uint32_t w = (z & 0x3FFFFFFFu) + UM::QFIX * q;  // z - q D  (q D = q 2^30 - QFIX q)
  if (w >= D) { w -= D; ++q; }                     // z = q D + w, w in [0, D)
  refl = 2u * w > D;
  const uint32_t wr = refl ? D - w : w;       // [0, D/2]
  j = (wr + 0x400000u) >> 23;                 // 0..64
  dw = (int32_t)(wr - (j << 23));
}

template <class UM>
__device__ __forceinline__ void turn_reduce(uint32_t z, uint32_t& q, bool& refl, uint32_t& j,
                                            float& dwf) {
  int32_t dw;
  turn_reduce_int<UM>(z, q, refl, j, dw);
  dwf = small_int_to_float(dw);
}

// |sin| and |cos| of 2 pi z / M for z in [1, M - 1], with their signs as
// the sign-bit masks sgn_s, sgn_c of the quadrant (0 or 0x80000000).
template <class UM>
__device__ __forceinline__ void sincos_turn_df_m(uint32_t z, const float4* __restrict__ tab, df& sn,
                                                 df& cs, uint32_t& sgn_s, uint32_t& sgn_c) {
  uint32_t q, j;
  bool refl;
  float dwf;
  turn_reduce<UM>(z, q, refl, j, dwf);
  const df delta = df_mul_f(df{UM::PID_HI, UM::PID_LO}, dwf);
  const float dh = delta.hi;
  const float d2 = __fmul_rn(dh, dh);
  // sin(delta) = delta + delta^3 (-1/6 + delta^2 / 120), the cubic term
  // added to delta.lo in the same rounding as its last product (one FMA)
  const float sd_lo = __fmaf_rn(__fmul_rn(dh, d2), __fmaf_rn(d2, 1.0f / 120.0f, -1.0f / 6.0f), delta.lo);
  const df sd = fast_two_sum(dh, sd_lo);
  // cos(delta) - 1 = -delta^2/2 + delta^4 (1/24 - delta^2 / 720)
  const float e2 = __fmaf_rn(2.0f * dh, delta.lo, __fmaf_rn(dh, dh, -d2));
  const float cc = __fmul_rn(__fmul_rn(d2, d2), __fmaf_rn(d2, -1.0f / 720.0f, 1.0f / 24.0f));
  const df cm1 = fast_two_sum(-0.5f * d2, __fmaf_rn(-0.5f, e2, cc));
  const float4 T = trig_entry(tab, j);
  const df sj{T.x, T.y}, cj{T.z, T.w};
  // sin(a + d) = sj + cj sin d + sj (cos d - 1);  cos(a + d) = cj - sj sin d + cj (cos d - 1).
  // |sin d| <= 0.0062 and |cos d - 1| <= 2e-5, so each product is formed as
  // its exact leading part plus fp32 cross terms, the leading parts are
  // added largest first (the table value dominates, or is 0 for j = 0 where
  // the result is the product itself), and the small remainders are summed
  // in fp32: the error stays near 1e-15 against the 1.5e-13 an fp64 output
  // of R cos(theta) allows.
  const df ps = df_mul_split(cj, sd), pc = df_mul_split(sj, cm1);
  const df qs = df_mul_split(sj, sd), qc = df_mul_split(cj, cm1);
  df sp, cp;
  // (left unnormalised, |lo| <~ 1.5 ulp(hi): their one use, df_mul by R,
  // renormalises its product)
  {
    const df u1 = fast_two_sum(sj.hi, ps.hi);
    const df u2 = fast_two_sum(u1.hi, pc.hi);
    sp = df{u2.hi, __fadd_rn(__fadd_rn(u1.lo, u2.lo), __fadd_rn(sj.lo, __fadd_rn(ps.lo, pc.lo)))};
  }
  {
    const df u1 = fast_two_sum(cj.hi, -qs.hi);
    const df u2 = fast_two_sum(u1.hi, qc.hi);
    cp = df{u2.hi, __fadd_rn(__fadd_rn(u1.lo, u2.lo), __fadd_rn(cj.lo, __fsub_rn(qc.lo, qs.lo)))};
  }
  // angle = (pi/2) q + phi, phi = reflected or not; sp, cp >= 0
  const bool swap = refl ^ (q & 1u);
  sn = swap ? cp : sp;
  cs = swap ? sp : cp;
  sgn_s = (q >> 1) << 31;                    // quadrants 2, 3
  sgn_c = ((q ^ (q >> 1)) & 1u) << 31;       // quadrants 1, 2
}

// Conversion of a df to IEEE double bits, in integers (|error| <= 1 ulp of
// the double).  Requires |hi| normal or zero and |lo| <= ulp(hi).
//   * hi as a double: its exponent-and-significand bits moved up 29 places,
//     the exponent rebiased by 1023 - 127 = 896 (one wide multiply-add);
//   * lo in units of the double's last place at hi's binade, 2^(e - 179),
//     rounded to an integer with the sign of lo relative to hi, added to the
//     magnitude bits -- a carry or borrow moves the exponent;
//   * when hi is a power of two and lo is negative the sum lies in the binade
//     below, whose last place is half as large: lo counts twice there.
__device__ __forceinline__ uint64_t df_to_f64_bits(df v) {
  const uint32_t hb = __float_as_uint(v.hi);
  const uint32_t ah = hb & 0x7FFFFFFFu;
  if (ah == 0) return (uint64_t)(hb & 0x80000000u) << 32;   // +-0
  uint64_t mag;
  asm("mad.wide.u32 %0, %1, 536870912, 0x3800000000000000;" : "=l"(mag) : "r"(ah));  // ah 2^29 + 896 2^52
  const uint32_t eh = ah >> 23;                              // biased fp32 exponent of hi
  int32_t li;
  if (__builtin_expect(eh >= 52, 1)) {                       // 2^(179 - eh) is a float
    const float scale = __uint_as_float(((306u - eh) << 23) ^ (hb & 0x80000000u));
    li = __float2int_rn(__fmul_rn(v.lo, scale));
  } else {                                                   // |hi| < 2^-75: scale in two steps
    const float s1 = __uint_as_float((127u + 64u) << 23);    // 2^64
    const float s2 = __uint_as_float(((242u - eh) << 23) ^ (hb & 0x80000000u));  // 2^(115 - eh)
    li = __float2int_rn(__fmul_rn(__fmul_rn(v.lo, s1), s2));
  }
  if (li < 0 && (ah & 0x7FFFFFu) == 0) li *= 2;
  mag += (uint64_t)(int64_t)li;
  return mag | ((uint64_t)(hb & 0x80000000u) << 32);
}

// The same for a df with hi >= 0 (or -0) and hi = 0 or |hi| >= 2^-75, given
// the sign to set as a sign-bit mask -- the magnitudes of Box-Muller
// outputs: a nonzero normal is at least R_min sin(2 pi / M) ~ 2e-5 * 1.5e-9
// = 3e-14.  A zero takes the sign too (as R times a negated zero does).
__device__ __forceinline__ uint64_t df_abs_to_f64_bits(df v, uint32_t sgn) {
  const uint32_t ah = __float_as_uint(v.hi) & 0x7FFFFFFFu;
  const uint64_t sb = (uint64_t)sgn << 32;
  if (ah == 0) return sb;
  uint64_t mag;
  asm("mad.wide.u32 %0, %1, 536870912, 0x3800000000000000;" : "=l"(mag) : "r"(ah));  // ah 2^29 + 896 2^52
  const float scale = __uint_as_float((306u - (ah >> 23)) << 23);                // 2^(179 - eh)
  int32_t li = __float2int_rn(__fmul_rn(v.lo, scale));
  if (li < 0 && (ah & 0x7FFFFFu) == 0) li *= 2;
  return (mag + (uint64_t)(int64_t)li) | sb;
}

__device__ __forceinline__ float df_to_f32(df v) { return __fadd_rn(v.hi, v.lo); }

// Box-Muller on one pair for fp64 outputs: R |cos| and R |sin| in
// double-float, converted to double bits with the quadrant's signs.
template <class UM>
__device__ __forceinline__ void box_muller_f64_m(uint32_t z1, uint32_t z2,
                                                 const float4* __restrict__ tab, uint64_t& x,
                                                 uint64_t& y) {
  const df l = ln_u_df_m<UM>(z1, tab);
  const df R = df_sqrt_raw(df{-2.0f * l.hi, -2.0f * l.lo});   // df_mul renormalises
  df sn, cs;
  uint32_t sgn_s, sgn_c;
  sincos_turn_df_m<UM>(z2, tab, sn, cs, sgn_s, sgn_c);
  x = df_abs_to_f64_bits(df_mul(R, cs), sgn_c);
  y = df_abs_to_f64_bits(df_mul(R, sn), sgn_s);
}

// sin and cos of 2 pi z / M for fp32 outputs, to ~2^-40 relative: the same
// reduction, table and Taylor terms as sincos_turn_df_m, but one exact
// leading product per function (sin(a + d) = sj + cj sin d + sj (cos d - 1):
// cj.hi d.hi exact, added to sj.hi error-free; the other terms, each below
// 2^-7 of the result, summed in fp32) and cos d - 1 in plain fp32 (it
// enters at most ~2e-5 of the result).  Returned without their signs, which
// come back as the sign-bit masks sgn_s, sgn_c of quadrant q.
//   error: sin in bucket 0 is the residual itself; elsewhere |sin| >= 0.006
//   and the fp32 terms contribute ~2^-38 absolute; |cos| >= 0.7.
template <class UM>
__device__ __forceinline__ void sincos_turn_lite_m(uint32_t z, const float4* __restrict__ tab,
                                                   df& sn, df& cs, uint32_t& sgn_s,
                                                   uint32_t& sgn_c) {
  uint32_t q, j;
  bool refl;
  float dwf;
  turn_reduce<UM>(z, q, refl, j, dwf);
  // delta = (pi / (2D)) dwf as dh + dl (dh exact leading product)
  const float dh = __fmul_rn(UM::PID_HI, dwf);
  const float dl = __fmaf_rn(UM::PID_LO, dwf, __fmaf_rn(UM::PID_HI, dwf, -dh));
  const float d2 = __fmul_rn(dh, dh);
  // sin d = dh + sdl,  sdl = dl + d^3 (-1/6 + d^2 / 120)
  const float sdl = __fmaf_rn(__fmul_rn(dh, d2), __fmaf_rn(d2, 1.0f / 120.0f, -1.0f / 6.0f), dl);
  // cos d - 1 = d^2 (-1/2 + d^2 (1/24 - d^2 / 720))
  const float cm1 = __fmul_rn(d2, __fmaf_rn(d2, __fmaf_rn(d2, -1.0f / 720.0f, 1.0f / 24.0f), -0.5f));
  const float4 T = trig_entry(tab, j);
  df sp, cp;
  {  // sj + cj sin d + sj (cos d - 1); |sj.hi| >= |cj.hi dh| or sj = 0
    const float p = __fmul_rn(T.z, dh);
    float a = __fadd_rn(T.y, __fmaf_rn(T.z, dh, -p));
    a = __fmaf_rn(T.x, cm1, a);
    a = __fmaf_rn(T.z, sdl, a);
    a = __fmaf_rn(T.w, dh, a);
    const df u = fast_two_sum(T.x, p);
    sp = df{u.hi, __fadd_rn(u.lo, a)};
  }
  {  // cj - sj sin d + cj (cos d - 1); |cj.hi| >= 0.7 > |sj.hi dh|
    const float p = __fmul_rn(T.x, dh);
    float a = __fsub_rn(T.w, __fmaf_rn(T.x, dh, -p));
    a = __fmaf_rn(T.z, cm1, a);
    a = __fmaf_rn(-T.x, sdl, a);
    a = __fmaf_rn(-T.y, dh, a);
    const df u = fast_two_sum(T.z, -p);
    cp = df{u.hi, __fadd_rn(u.lo, a)};
  }
  const bool swap = refl ^ (q & 1u);
  sn = swap ? cp : sp;
  cs = swap ? sp : cp;
  sgn_s = (q >> 1) << 31;                    // quadrants 2, 3
  sgn_c = ((q ^ (q >> 1)) & 1u) << 31;       // quadrants 1, 2
}

// Box-Muller for fp32 outputs: R from the ~2^-34 log, sin and cos from the
// lite reduction, each output rounded once (df_mul_to_f32) and then signed.
// Accuracy ~2^-33 relative before the final rounding.
template <class UM>
__device__ __forceinline__ void box_muller_f32_m(uint32_t z1, uint32_t z2,
                                                 const float4* __restrict__ tab, float& x,
                                                 float& y) {
  const df l = ln_u_lite_m<UM>(z1, tab);
  const df R = df_sqrt_raw(df{-2.0f * l.hi, -2.0f * l.lo});
  df sn, cs;
  uint32_t sgn_s, sgn_c;
  sincos_turn_lite_m<UM>(z2, tab, sn, cs, sgn_s, sgn_c);
  x = __uint_as_float(__float_as_uint(df_mul_to_f32(R, cs.hi, cs.lo)) ^ sgn_c);
  y = __uint_as_float(__float_as_uint(df_mul_to_f32(R, sn.hi, sn.lo)) ^ sgn_s);
}

// X + Y of one Box-Muller pair, R (cos + sin), as an unrounded float pair
// for sums whose tolerance is relative to the sum of |X| and |Y| (~2^-30):
// the ~2^-34 log and the lite sin/cos (absolute error ~2^-38), signed,
// added error-free, times R with the exact leading product.  Absolute
// error <= ~2^-34 per pair (R <= 6.7), whether or not cos and sin cancel.
// box_muller_sum_lite_rest_m is the part after R, given R (the fused
// consumer computes R of two pairs at once); box_muller_sum_lite_m the whole.
template <class UM>
__device__ __forceinline__ df box_muller_sum_lite_rest_m(df R, uint32_t z2,
                                                         const float4* __restrict__ tab) {
  df sn, cs;
  uint32_t sgn_s, sgn_c;
  sincos_turn_lite_m<UM>(z2, tab, sn, cs, sgn_s, sgn_c);
  const float ch = __uint_as_float(__float_as_uint(cs.hi) ^ sgn_c);
  const float cl = __uint_as_float(__float_as_uint(cs.lo) ^ sgn_c);
  const float sh = __uint_as_float(__float_as_uint(sn.hi) ^ sgn_s);
  const float sl = __uint_as_float(__float_as_uint(sn.lo) ^ sgn_s);
  const df t = two_sum(ch, sh);
  const float tl = __fadd_rn(t.lo, __fadd_rn(cl, sl));
  return df_mul_split(R, df{t.hi, tl});
}

template <class UM>
__device__ __forceinline__ df box_muller_sum_lite_m(uint32_t z1, uint32_t z2,
                                                    const float4* __restrict__ tab) {
  const df l = ln_u_lite_m<UM>(z1, tab);
  return box_muller_sum_lite_rest_m<UM>(df_sqrt_raw(df{-2.0f * l.hi, -2.0f * l.lo}), z2, tab);
}

// -ln(u) / rate for fp32 outputs: the ~2^-34 log times -1/rate (a float
// pair), rounded once.
template <class UM>
__device__ __forceinline__ float exp_f32_m(uint32_t z, const float4* __restrict__ tab, float ir_hi,
                                           float ir_lo) {
  const df l = ln_u_lite_raw_m<UM>(z, tab);
  return df_mul_to_f32(df{ir_hi, ir_lo}, l.hi, l.lo);
}

// The transforms of MRG32k3a's uniforms u = z / (m1 + 1).
__device__ __forceinline__ df ln_u_df(uint32_t z, const float4* __restrict__ tab) {
  return ln_u_df_m<UM32k3a>(z, tab);
}
__device__ __forceinline__ void box_muller_f64(uint32_t z1, uint32_t z2, const float4* __restrict__ tab,
                                               uint64_t& x, uint64_t& y) {
  box_muller_f64_m<UM32k3a>(z1, z2, tab, x, y);
}
__device__ __forceinline__ df ln_u_lite(uint32_t z, const float4* __restrict__ tab) {
  return ln_u_lite_m<UM32k3a>(z, tab);
}
__device__ __forceinline__ void box_muller_f32(uint32_t z1, uint32_t z2, const float4* __restrict__ tab,
                                               float& x, float& y) {
  box_muller_f32_m<UM32k3a>(z1, z2, tab, x, y);
}
__device__ __forceinline__ float exp_f32(uint32_t z, const float4* __restrict__ tab, float ir_hi,
                                         float ir_lo) {
  return exp_f32_m<UM32k3a>(z, tab, ir_hi, ir_lo);
}

}  // namespace mrg
