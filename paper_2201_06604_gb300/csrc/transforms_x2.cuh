// transforms_x2.cuh -- the double-float transforms of two draws (Box-Muller:
// two pairs) at once with packed fp32x2 instructions (add/sub/mul/fma
// .rn.f32x2: two IEEE fp32 operations in one instruction): fp64 normals,
// the radius R of fp32 normals, fp32 and fp64 exponentials.
//
// The transform kernels are bound by instruction issue, not by the FP32
// pipes (about half busy): a packed instruction carries two fp32 operations
// through one issue slot.  Every function below performs, element by
// element, the fp32 operations of its scalar counterpart in
// transforms_df.cuh with the same operands and the same rounding, so the
// outputs are bit-identical to the scalar path's (which rows too narrowly
// aligned for 16-byte stores, the last draws of a transform, an odd last
// pair of the fused consumer and the matrix-layout kernel take; generate,
// batched and served requests use the packed forms); only the integer
// parts (reductions, table indices, the conversion to double bits) and the
// MUFU reciprocal square root stay per element.
//
// Two rules keep that identity:
//   * A scalar FMA negates an operand for free; a packed one cannot.  So
//     where the scalar code forms an error-free product p = RN(a b),
//     e = fma(a, b, -p), this code forms np = RN(a (-b)) = -p from an
//     operand already at hand in negated form and carries np onward: IEEE
//     defines x - y as x + (-y), so RN(s - np) is RN(s + p) bit for bit, and
//     a fast-two-sum given -b returns its low part negated (a sign of zero
//     aside, which no output sees).
//   * The compiler fuses a packed product whose only use is a packed add or
//     subtract into an FMA even under .rn, which would round once where the
//     scalar code rounds twice.  No inexact product here has an add or
//     subtract as its only use (the scalar code adds the one such term,
//     the cubic term of sin(delta), with an FMA in both forms).
#pragma once
#include <stdint.h>

#include "transforms_df.cuh"

namespace mrg {

typedef unsigned long long f2;   // low word: element a, high word: element b

__device__ __forceinline__ f2 pk(float a, float b) {
  f2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk(f2 v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 bc(float a) { return pk(a, a); }
__device__ __forceinline__ f2 add2(f2 x, f2 y) {
  f2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
  return r;
}
__device__ __forceinline__ f2 sub2(f2 x, f2 y) {
  f2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
  return r;
}
__device__ __forceinline__ f2 mul2(f2 x, f2 y) {
  f2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
  return r;
}
__device__ __forceinline__ f2 fma2(f2 x, f2 y, f2 z) {
  f2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(x), "l"(y), "l"(z));
  return r;
}
// -x, exactly (a product with -1: one instruction, where flipping both sign
// bits takes two integer ones)
__device__ __forceinline__ f2 neg2(f2 x) { return mul2(x, bc(-1.0f)); }
// per element: a where the mask's word is all ones, else b
__device__ __forceinline__ f2 sel2(f2 m, f2 a, f2 b) { return (a & m) | (b & ~m); }
__device__ __forceinline__ f2 mask2(bool a, bool b) {
  return (a ? 0xFFFFFFFFull : 0ull) | (b ? 0xFFFFFFFF00000000ull : 0ull);
}

struct df2 {
  f2 hi, lo;
};

__device__ __forceinline__ df2 fast_two_sum2(f2 a, f2 b) {   // |a| >= |b| per element
  const f2 s = add2(a, b);
  return df2{s, sub2(b, sub2(s, a))};
}

// fast_two_sum(a, b) given nb = -b: the sum, and the low part negated.
__device__ __forceinline__ df2 fast_two_sum_nb2(f2 a, f2 nb) {
  const f2 s = sub2(a, nb);
  return df2{s, add2(nb, sub2(s, a))};
}

__device__ __forceinline__ df2 df_add_ordered2(df2 x, df2 y) {
  const df2 s = fast_two_sum2(x.hi, y.hi);
  return fast_two_sum2(s.hi, add2(s.lo, add2(x.lo, y.lo)));
}

// ln(z / M) of two draws (ln_u_df_m on each).
template <class UM>
__device__ __forceinline__ df2 ln_u_df_m2(uint32_t za, uint32_t zb, const float4* __restrict__ tab) {
  uint32_t sa, sb;
  asm("bfind.shiftamt.u32 %0, %1;" : "=r"(sa) : "r"(za));
  asm("bfind.shiftamt.u32 %0, %1;" : "=r"(sb) : "r"(zb));
  const uint32_t zna = za << sa, znb = zb << sb;
  const uint32_t ka = (zna >> 24) & 127u, kb = (znb >> 24) & 127u;
  const uint32_t cka = ka == 127u ? UM::TOP_CK : 0x80800000u + (ka << 24);
  const uint32_t ckb = kb == 127u ? UM::TOP_CK : 0x80800000u + (kb << 24);
  const float2 Ta = log_inv_ck(tab, ka), Tb = log_inv_ck(tab, kb);
  const f2 dfl = pk((float)(int32_t)(zna - cka), (float)(int32_t)(znb - ckb));
  const f2 Tx = pk(Ta.x, Tb.x), Ty = pk(Ta.y, Tb.y);
  // r = d / C_k = rh + rl, not renormalised
  const f2 rh = mul2(Tx, dfl);
  const f2 nrh = neg2(rh);
  const f2 rl = fma2(Ty, dfl, fma2(Tx, dfl, nrh));
  // r^2 = p2 + e2, carried as np2 = -p2 (p2 rh = np2 nrh exactly)
  const f2 np2 = mul2(rh, nrh);
  const f2 e2 = fma2(mul2(bc(2.0f), rh), rl, fma2(rh, rh, np2));
  f2 poly = fma2(rh, bc(-1.0f / 6.0f), bc(0.2f));
  poly = fma2(rh, poly, bc(-0.25f));
  poly = fma2(rh, poly, bc(1.0f / 3.0f));
  const f2 c3 = mul2(mul2(np2, nrh), poly);
  const df2 l1p = df_add_ordered2(df2{rh, rl}, df2{mul2(bc(0.5f), np2), fma2(bc(-0.5f), e2, c3)});
  const float2 La = log_ck_shift(tab, sa, ka), Lb = log_ck_shift(tab, sb, kb);
  return df_add_ordered2(df2{pk(La.x, Lb.x), pk(La.y, Lb.y)}, l1p);
}

// R = sqrt(-2 l) of two logarithms (df_sqrt_raw on -2 l), with -R.hi.
__device__ __forceinline__ df2 df_sqrt_m2l2(df2 l, f2& nRh) {
  const f2 xh = mul2(bc(-2.0f), l.hi), xl = mul2(bc(-2.0f), l.lo);
  float xa, xb;
  upk(xh, xa, xb);
  f2 y = pk(rsqrtf(xa), rsqrtf(xb));
  y = mul2(y, fma2(l.hi, mul2(y, y), bc(1.5f)));   // -x.hi / 2 is l.hi exactly
  const f2 r0 = mul2(xh, y);
  nRh = neg2(r0);
  const f2 e = add2(fma2(nRh, r0, xh), xl);
  return df2{r0, mul2(mul2(e, y), bc(0.5f))};
}

// x y for x given with nxh = -x.hi (df_mul).
__device__ __forceinline__ df2 df_mul_nx2(df2 x, f2 nxh, df2 y) {
  const f2 np = mul2(nxh, y.hi);
  f2 e = fma2(x.hi, y.hi, np);
  e = fma2(x.hi, y.lo, e);
  e = fma2(x.lo, y.hi, e);
  const f2 s = sub2(e, np);
  return df2{s, sub2(e, add2(s, np))};
}

// The leading product of x y negated, and the rest, for y given with
// nyh = -y.hi (df_mul_split: {-p, e}).
__device__ __forceinline__ df2 df_mul_split_ny2(df2 x, df2 y, f2 nyh) {
  const f2 np = mul2(x.hi, nyh);
  f2 e = fma2(x.hi, y.hi, np);
  e = fma2(x.hi, y.lo, e);
  e = fma2(x.lo, y.hi, e);
  return df2{np, e};
}

// |sin| and |cos| of 2 pi z / M for two draws, with the quadrants' sign
// masks (sincos_turn_df_m on each).
template <class UM>
__device__ __forceinline__ void sincos_turn_df_m2(uint32_t za, uint32_t zb,
                                                  const float4* __restrict__ tab, df2& sn, df2& cs,
                                                  uint32_t& sgn_sa, uint32_t& sgn_ca,
                                                  uint32_t& sgn_sb, uint32_t& sgn_cb) {
  uint32_t qa, ja, qb, jb;
  bool refla, reflb;
  int32_t dwa, dwb;
  turn_reduce_int<UM>(za, qa, refla, ja, dwa);
  turn_reduce_int<UM>(zb, qb, reflb, jb, dwb);
  const f2 dwf = sub2(pk(__int_as_float(0x4B400000 + dwa), __int_as_float(0x4B400000 + dwb)),
                      bc(12582912.0f));                      // small_int_to_float
  // delta = (PID_HI, PID_LO) dwf, its leading product carried negated
  const f2 ndp = mul2(bc(-UM::PID_HI), dwf);
  f2 de = fma2(bc(UM::PID_HI), dwf, ndp);
  de = fma2(bc(UM::PID_LO), dwf, de);
  const f2 dh = sub2(de, ndp);
  const f2 dl = sub2(de, add2(dh, ndp));
  const f2 d2 = mul2(dh, dh);
  const f2 sd_lo = fma2(mul2(dh, d2), fma2(d2, bc(1.0f / 120.0f), bc(-1.0f / 6.0f)), dl);
  const df2 sd = fast_two_sum2(dh, sd_lo);
  const f2 e2 = fma2(mul2(bc(2.0f), dh), dl, fma2(dh, dh, neg2(d2)));
  const f2 cc = mul2(mul2(d2, d2), fma2(d2, bc(-1.0f / 720.0f), bc(1.0f / 24.0f)));
  const df2 cm1 = fast_two_sum2(mul2(bc(-0.5f), d2), fma2(bc(-0.5f), e2, cc));
  const f2 nsdh = neg2(sd.hi), ncm1h = neg2(cm1.hi);
  const float4 Ta = trig_entry(tab, ja), Tb = trig_entry(tab, jb);
  const df2 sj{pk(Ta.x, Tb.x), pk(Ta.y, Tb.y)}, cj{pk(Ta.z, Tb.z), pk(Ta.w, Tb.w)};
  const df2 ps = df_mul_split_ny2(cj, sd, nsdh), pc = df_mul_split_ny2(sj, cm1, ncm1h);
  const df2 qs = df_mul_split_ny2(sj, sd, nsdh), qc = df_mul_split_ny2(cj, cm1, ncm1h);
  df2 sp, cp;
  {   // sj + ps + pc, the low parts of both sums negated
    const df2 u1 = fast_two_sum_nb2(sj.hi, ps.hi);
    const df2 u2 = fast_two_sum_nb2(u1.hi, pc.hi);
    sp = df2{u2.hi, sub2(add2(sj.lo, add2(ps.lo, pc.lo)), add2(u1.lo, u2.lo))};
  }
  {   // cj - qs + qc, the second sum's low part negated
    const df2 u1 = fast_two_sum2(cj.hi, qs.hi);
    const df2 u2 = fast_two_sum_nb2(u1.hi, qc.hi);
    cp = df2{u2.hi, add2(sub2(u1.lo, u2.lo), add2(cj.lo, sub2(qc.lo, qs.lo)))};
  }
  const f2 swap = mask2(refla ^ (bool)(qa & 1u), reflb ^ (bool)(qb & 1u));
  sn = df2{sel2(swap, cp.hi, sp.hi), sel2(swap, cp.lo, sp.lo)};
  cs = df2{sel2(swap, sp.hi, cp.hi), sel2(swap, sp.lo, cp.lo)};
  sgn_sa = (qa >> 1) << 31;
  sgn_ca = ((qa ^ (qa >> 1)) & 1u) << 31;
  sgn_sb = (qb >> 1) << 31;
  sgn_cb = ((qb ^ (qb >> 1)) & 1u) << 31;
}

// Two Box-Muller pairs (z1a, z2a) and (z1b, z2b) to fp64 bits, identical to
// box_muller_f64_m on each pair.
template <class UM>
__device__ __forceinline__ void box_muller_f64_x2(uint32_t z1a, uint32_t z2a, uint32_t z1b,
                                                  uint32_t z2b, const float4* __restrict__ tab,
                                                  uint64_t& xa, uint64_t& ya, uint64_t& xb,
                                                  uint64_t& yb) {
  const df2 l = ln_u_df_m2<UM>(z1a, z1b, tab);
  f2 nRh;
  const df2 R = df_sqrt_m2l2(l, nRh);
  df2 sn, cs;
  uint32_t ssa, sca, ssb, scb;
  sincos_turn_df_m2<UM>(z2a, z2b, tab, sn, cs, ssa, sca, ssb, scb);
  const df2 X = df_mul_nx2(R, nRh, cs), Y = df_mul_nx2(R, nRh, sn);
  float xha, xhb, xla, xlb, yha, yhb, yla, ylb;
  upk(X.hi, xha, xhb);
  upk(X.lo, xla, xlb);
  upk(Y.hi, yha, yhb);
  upk(Y.lo, yla, ylb);
  xa = df_abs_to_f64_bits(df{xha, xla}, sca);
  ya = df_abs_to_f64_bits(df{yha, yla}, ssa);
  xb = df_abs_to_f64_bits(df{xhb, xlb}, scb);
  yb = df_abs_to_f64_bits(df{yhb, ylb}, ssb);
}

// ---- fp32 outputs ------------------------------------------------------------

// ln(z / M) of two draws to ~2^-34 relative, not renormalised
// (ln_u_lite_raw_m on each).
template <class UM>
__device__ __forceinline__ df2 ln_u_lite_raw_m2(uint32_t za, uint32_t zb,
                                                const float4* __restrict__ tab) {
  uint32_t sa, sb;
  asm("bfind.shiftamt.u32 %0, %1;" : "=r"(sa) : "r"(za));
  asm("bfind.shiftamt.u32 %0, %1;" : "=r"(sb) : "r"(zb));
  const uint32_t zna = za << sa, znb = zb << sb;
  const uint32_t ka = (zna >> 24) & 127u, kb = (znb >> 24) & 127u;
  const uint32_t cka = ka == 127u ? UM::TOP_CK : 0x80800000u + (ka << 24);
  const uint32_t ckb = kb == 127u ? UM::TOP_CK : 0x80800000u + (kb << 24);
  const float2 Ta = log_inv_ck(tab, ka), Tb = log_inv_ck(tab, kb);
  const f2 dfl = pk((float)(int32_t)(zna - cka), (float)(int32_t)(znb - ckb));
  const f2 Tx = pk(Ta.x, Tb.x), Ty = pk(Ta.y, Tb.y);
  const f2 rh = mul2(Tx, dfl);
  const f2 re = fma2(Ty, dfl, fma2(Tx, dfl, neg2(rh)));    // r = rh + re
  f2 poly = fma2(rh, bc(-1.0f / 6.0f), bc(0.2f));
  poly = fma2(rh, poly, bc(-0.25f));
  poly = fma2(rh, poly, bc(1.0f / 3.0f));
  poly = fma2(rh, poly, bc(-0.5f));
  const f2 rt = fma2(mul2(rh, rh), poly, re);
  const float2 La = log_ck_shift(tab, sa, ka), Lb = log_ck_shift(tab, sb, kb);
  const df2 u = fast_two_sum2(pk(La.x, Lb.x), rh);
  return df2{u.hi, add2(u.lo, add2(pk(La.y, Lb.y), rt))};
}

// RN32 of a b for two df a and b (df_mul_to_f32 on each).
__device__ __forceinline__ f2 df_mul_to_f32_2(df2 a, df2 b) {
  return fma2(a.hi, b.hi, fma2(a.hi, b.lo, mul2(a.lo, b.hi)));
}

__device__ __forceinline__ float with_sign(float v, uint32_t sgn) {
  return __uint_as_float(__float_as_uint(v) ^ sgn);
}

// Two Box-Muller pairs (z1a, z2a) and (z1b, z2b) to fp32, identical to
// box_muller_f32_m on each pair.  Only R = sqrt(-2 ln u1) is packed; sin and
// cos stay one pair at a time.  A packed instruction occupies both FP32
// sub-pipes, and the heavy one also runs the recurrence's IMADs and the
// moves that pair operands: with sin/cos packed too, that pipe became the
// limit (measured per 2^30 outputs: all packed 3.17 ms, sin/cos only 3.18,
// none 3.10-3.13, the log and square root only 2.99).
template <class UM>
__device__ __forceinline__ void box_muller_f32_x2(uint32_t z1a, uint32_t z2a, uint32_t z1b,
                                                  uint32_t z2b, const float4* __restrict__ tab,
                                                  float& xa, float& ya, float& xb, float& yb) {
  const df2 lr = ln_u_lite_raw_m2<UM>(z1a, z1b, tab);
  const df2 l = fast_two_sum2(lr.hi, lr.lo);                 // ln_u_lite_m
  f2 nRh;
  const df2 R = df_sqrt_m2l2(l, nRh);
  float rha, rhb, rla, rlb;
  upk(R.hi, rha, rhb);
  upk(R.lo, rla, rlb);
  df sn, cs;
  uint32_t ss, sc;
  sincos_turn_lite_m<UM>(z2a, tab, sn, cs, ss, sc);
  xa = with_sign(df_mul_to_f32(df{rha, rla}, cs.hi, cs.lo), sc);
  ya = with_sign(df_mul_to_f32(df{rha, rla}, sn.hi, sn.lo), ss);
  sincos_turn_lite_m<UM>(z2b, tab, sn, cs, ss, sc);
  xb = with_sign(df_mul_to_f32(df{rhb, rlb}, cs.hi, cs.lo), sc);
  yb = with_sign(df_mul_to_f32(df{rhb, rlb}, sn.hi, sn.lo), ss);
}

// X + Y of two Box-Muller pairs as float pairs (box_muller_sum_lite_m on
// each), with R of both packed as for the fp32 normals.
template <class UM>
__device__ __forceinline__ void box_muller_sum_lite_x2(uint32_t z1a, uint32_t z2a, uint32_t z1b,
                                                       uint32_t z2b, const float4* __restrict__ tab,
                                                       df& va, df& vb) {
  const df2 lr = ln_u_lite_raw_m2<UM>(z1a, z1b, tab);
  const df2 l = fast_two_sum2(lr.hi, lr.lo);
  f2 nRh;
  const df2 R = df_sqrt_m2l2(l, nRh);
  float rha, rhb, rla, rlb;
  upk(R.hi, rha, rhb);
  upk(R.lo, rla, rlb);
  va = box_muller_sum_lite_rest_m<UM>(df{rha, rla}, z2a, tab);
  vb = box_muller_sum_lite_rest_m<UM>(df{rhb, rlb}, z2b, tab);
}

// -ln(u) / rate of two draws to fp64 bits, identical to
// df_to_f64_bits(df_mul(ln_u_df_m(z), {ir_hi, ir_lo})) on each: the log of
// both draws packed, the product by -1/rate packed (df_mul_nx2 is df_mul
// given the negated leading part of its first operand), the conversion to
// double bits per element.
template <class UM>
__device__ __forceinline__ void exp_f64_x2(uint32_t za, uint32_t zb, const float4* __restrict__ tab,
                                           float ir_hi, float ir_lo, uint64_t& ea, uint64_t& eb) {
  const df2 l = ln_u_df_m2<UM>(za, zb, tab);
  const df2 p = df_mul_nx2(l, neg2(l.hi), df2{bc(ir_hi), bc(ir_lo)});
  float ha, hb, la, lb;
  upk(p.hi, ha, hb);
  upk(p.lo, la, lb);
  ea = df_to_f64_bits(df{ha, la});
  eb = df_to_f64_bits(df{hb, lb});
}

// -ln(u) / rate of two draws to fp32, identical to exp_f32_m on each.
template <class UM>
__device__ __forceinline__ void exp_f32_x2(uint32_t za, uint32_t zb, const float4* __restrict__ tab,
                                           float ir_hi, float ir_lo, float& ea, float& eb) {
  const df2 l = ln_u_lite_raw_m2<UM>(za, zb, tab);
  upk(df_mul_to_f32_2(df2{bc(ir_hi), bc(ir_lo)}, l), ea, eb);
}

}  // namespace mrg
