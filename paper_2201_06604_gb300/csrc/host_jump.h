// host_jump.h -- host-side jump-ahead helpers of libmrg32k3a (internal).
#pragma once
#include <stdint.h>

namespace mrg {
namespace host {

constexpr int kJumpBits = 191;  // A^(2^i), i < 191: offsets < 2^128, stream index < 2^64

// A_c^(2^i) mod m_c as uint32 (row-major 3x3), c = 0 (m1) and 1 (m2).
void jump_table_u32(uint32_t out[2][kJumpBits][9]);

// x1 words < m1, x2 words < m2, neither triple all zero.
bool state_valid(const uint32_t s[6]);

// s <- A^(e * 2^base) s, for 0 <= base and base + 63 < kJumpBits.
void jump_pow2_multiple(uint32_t s[6], uint64_t e, int base);

// True when RN64(1/(m1+1)) has exponent -32 and significand 2^52 + delta.
bool norm_constant_ok(uint64_t delta);

// Tables of the double-float transforms (layout in transforms_df.cuh), in
// units of four floats:
// entries [0, 64): 1/C_k for the 128 log buckets, as float pairs;
// entries [64, 584): sin and cos of the bucket angles a_j, eight copies of
// each of the 65 entries side by side;
// entries [584, 2632): ln(C_k / (M 2^s)) for every shift s < 32 and bucket
// k, as 4096 float pairs.
constexpr int kTransformTrigCopies = 8;
constexpr int kTransformEntries = 64 + 65 * kTransformTrigCopies + 2048;
void transform_table(float out[kTransformEntries][4]);

// The same tables for uniforms u = z' / 2^32 (M = 2^32, quarter turn D = 2^30):
// the transforms of MRG31k3p, whose u = z / 2^31 is fed as z' = 2 z.
void transform_table_m32(float out[kTransformEntries][4]);

// MRG31k3p (L'Ecuyer and Touzin 2000), the paper's own generator (Sec. 2):
// m1 = 2^31 - 1, m2 = 2^31 - 21069; streams 2^134 apart (Sec. 2.1).
namespace g31 {
constexpr int kJumpBits = 198;  // A^(2^i), i < 198: offsets < 2^134, stream index < 2^64
constexpr int kStreamLog2 = 134;
void jump_table_u32(uint32_t out[2][kJumpBits][9]);
bool state_valid(const uint32_t s[6]);
void jump_pow2_multiple(uint32_t s[6], uint64_t e, int base);
}  // namespace g31

}  // namespace host
}  // namespace mrg
