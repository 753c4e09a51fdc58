// host_jump.cpp -- host-side jump-ahead math of libmrg32k3a.
//
// Builds the tables A_c^(2^i) mod m_c (i < JUMP_BITS) that the kernels read
// from constant memory, and evaluates the small jumps the host needs itself
// (the stream creator's next seed, Sec. 2.1: after n streams the creator has
// advanced n * 2^127 steps).  Companion matrices act on newest-first states:
// (x[n], x[n-1], x[n-2]) = A (x[n-1], x[n-2], x[n-3]).
#include "host_jump.h"

#include <cmath>
#include <cstring>

namespace mrg {
namespace host {

namespace {

typedef unsigned __int128 u128;

const uint64_t kMod[2] = {4294967087ull, 4294944443ull};

// Companion matrices: component 1 has coefficients (0, 1403580, -810728) on
// (x[n-1], x[n-2], x[n-3]); component 2 has (527612, 0, -1370589).
void companion(int c, uint64_t A[9]) {
  const uint64_t m = kMod[c];
  const uint64_t row0[2][3] = {{0, 1403580ull, m - 810728ull},
                               {527612ull, 0, m - 1370589ull}};
  for (int j = 0; j < 3; ++j) A[j] = row0[c][j];
  A[3] = 1; A[4] = 0; A[5] = 0;
  A[6] = 0; A[7] = 1; A[8] = 0;
}

void mat_mul(const uint64_t X[9], const uint64_t Y[9], uint64_t m, uint64_t out[9]) {
  uint64_t t[9];
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) {
      u128 acc = 0;
      for (int k = 0; k < 3; ++k) acc += (u128)X[3 * r + k] * Y[3 * k + q];
      t[3 * r + q] = (uint64_t)(acc % m);
    }
  std::memcpy(out, t, sizeof t);
}

void mat_vec(const uint64_t A[9], uint64_t x[3], uint64_t m) {
  uint64_t y[3];
  for (int r = 0; r < 3; ++r) {
    u128 acc = 0;
    for (int k = 0; k < 3; ++k) acc += (u128)A[3 * r + k] * x[k];
    y[r] = (uint64_t)(acc % m);
  }
  std::memcpy(x, y, sizeof y);
}

struct Tables {
  uint64_t pow2[2][kJumpBits][9];
  Tables() {
    for (int c = 0; c < 2; ++c) {
      companion(c, pow2[c][0]);
      for (int i = 1; i < kJumpBits; ++i) mat_mul(pow2[c][i - 1], pow2[c][i - 1], kMod[c], pow2[c][i]);
    }
  }
};

const Tables& tables() {
  static const Tables t;
  return t;
}

}  // namespace

void jump_table_u32(uint32_t out[2][kJumpBits][9]) {
  const Tables& t = tables();
  for (int c = 0; c < 2; ++c)
    for (int i = 0; i < kJumpBits; ++i)
      for (int k = 0; k < 9; ++k) out[c][i][k] = (uint32_t)t.pow2[c][i][k];
}

bool state_valid(const uint32_t s[6]) {
  for (int k = 0; k < 3; ++k)
    if (s[k] >= kMod[0] || s[3 + k] >= kMod[1]) return false;
  if ((s[0] | s[1] | s[2]) == 0) return false;
  if ((s[3] | s[4] | s[5]) == 0) return false;
  return true;
}

void jump_pow2_multiple(uint32_t s[6], uint64_t e, int base) {
  const Tables& t = tables();
  uint64_t x[2][3] = {{s[0], s[1], s[2]}, {s[3], s[4], s[5]}};
  for (int j = 0; j < 64 && (e >> j); ++j)
    if ((e >> j) & 1)
      for (int c = 0; c < 2; ++c) mat_vec(t.pow2[c][base + j], x[c], kMod[c]);
  for (int k = 0; k < 3; ++k) {
    s[k] = (uint32_t)x[0][k];
    s[3 + k] = (uint32_t)x[1][k];
  }
}

bool norm_constant_ok(uint64_t delta) {
  // The kernels build RN64(z / (m1 + 1)) from the significand 2^52 + delta
  // and exponent -32 of norm = RN64(1 / (m1 + 1)); check both here.
  double norm = 1.0 / 4294967088.0;
  uint64_t bits;
  std::memcpy(&bits, &norm, sizeof bits);
  uint64_t sig = (bits & ((1ull << 52) - 1)) | (1ull << 52);
  int exp = (int)((bits >> 52) & 0x7FF) - 1023;
  return exp == -32 && sig == (1ull << 52) + delta;
}

namespace {
void split(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

// Tables for uniforms u = z / M (z < M <= 2^32), quarter turn D = M / 4.
void transform_table_for(double M, double D, float out[kTransformEntries][4]) {
  // log buckets: centre C_k of the zn-range [2^31 + k 2^24, 2^31 + (k+1) 2^24),
  // the top bucket centred at M so that ln(C_127 / M) = 0 exactly.
  float* inv = &out[0][0];
  for (int k = 0; k < 128; ++k) {
    const double C = k == 127 ? M : 2147483648.0 + (2.0 * k + 1.0) * 8388608.0;
    split(1.0 / C, inv[2 * k], inv[2 * k + 1]);
  }
  // trig buckets: a_j = (pi/2) j 2^23 / D (a_0 = 0 exactly), each entry in
  // kTransformTrigCopies identical copies side by side
  for (int j = 0; j < 65; ++j) {
    const double a = (M_PI / 2) * ((j * 8388608.0) / D);
    for (int c = 0; c < kTransformTrigCopies; ++c) {
      float* e = out[64 + kTransformTrigCopies * j + c];
      split(std::sin(a), e[0], e[1]);
      split(std::cos(a), e[2], e[3]);
    }
  }
  // ln(C_k / (M 2^s)) = ln(C_k / M) - s ln 2 for every shift s and bucket k,
  // as float pairs after the trig entries (pair 128 s + k); one fused
  // multiply-add (explicit, so that no compiler contracts it differently on
  // another host)
  float* ls = &out[64 + 65 * kTransformTrigCopies][0];
  for (int sh = 0; sh < 32; ++sh)
    for (int k = 0; k < 128; ++k) {
      const double C = k == 127 ? M : 2147483648.0 + (2.0 * k + 1.0) * 8388608.0;
      const double v = std::fma(-(double)sh, 0.6931471805599453094, std::log1p((C - M) / M));
      split(v, ls[2 * (sh * 128 + k)], ls[2 * (sh * 128 + k) + 1]);
    }
}
}  // namespace

void transform_table(float out[kTransformEntries][4]) {
  transform_table_for(4294967088.0, 1073741772.0, out);   // M = m1 + 1, D = M / 4
}

void transform_table_m32(float out[kTransformEntries][4]) {
  transform_table_for(4294967296.0, 1073741824.0, out);   // M = 2^32, D = 2^30
}

// ---------------------------------------------------------------------------
// MRG31k3p: x1[n] = (2^22 x1[n-2] + (2^7 + 1) x1[n-3]) mod m1,
//           x2[n] = (2^15 x2[n-1] + (2^15 + 1) x2[n-3]) mod m2.
// ---------------------------------------------------------------------------
namespace g31 {
namespace {

const uint64_t kMod31[2] = {2147483647ull, 2147462579ull};

void companion31(int c, uint64_t A[9]) {
  const uint64_t row0[2][3] = {{0, 1ull << 22, (1ull << 7) + 1}, {1ull << 15, 0, (1ull << 15) + 1}};
  for (int j = 0; j < 3; ++j) A[j] = row0[c][j];
  A[3] = 1; A[4] = 0; A[5] = 0;
  A[6] = 0; A[7] = 1; A[8] = 0;
}

struct Tables31 {
  uint64_t pow2[2][kJumpBits][9];
  Tables31() {
    for (int c = 0; c < 2; ++c) {
      companion31(c, pow2[c][0]);
      for (int i = 1; i < kJumpBits; ++i)
        mat_mul(pow2[c][i - 1], pow2[c][i - 1], kMod31[c], pow2[c][i]);
    }
  }
};

const Tables31& tables31() {
  static const Tables31 t;
  return t;
}

}  // namespace

void jump_table_u32(uint32_t out[2][kJumpBits][9]) {
  const Tables31& t = tables31();
  for (int c = 0; c < 2; ++c)
    for (int i = 0; i < kJumpBits; ++i)
      for (int k = 0; k < 9; ++k) out[c][i][k] = (uint32_t)t.pow2[c][i][k];
}

bool state_valid(const uint32_t s[6]) {
  for (int k = 0; k < 3; ++k)
    if (s[k] >= kMod31[0] || s[3 + k] >= kMod31[1]) return false;
  if ((s[0] | s[1] | s[2]) == 0) return false;
  if ((s[3] | s[4] | s[5]) == 0) return false;
  return true;
}

void jump_pow2_multiple(uint32_t s[6], uint64_t e, int base) {
  const Tables31& t = tables31();
  uint64_t x[2][3] = {{s[0], s[1], s[2]}, {s[3], s[4], s[5]}};
  for (int j = 0; j < 64 && (e >> j); ++j)
    if ((e >> j) & 1)
      for (int c = 0; c < 2; ++c) mat_vec(t.pow2[c][base + j], x[c], kMod31[c]);
  for (int k = 0; k < 3; ++k) {
    s[k] = (uint32_t)x[0][k];
    s[3 + k] = (uint32_t)x[1][k];
  }
}

}  // namespace g31

}  // namespace host
}  // namespace mrg
