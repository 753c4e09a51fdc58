// grf_kernels.cuh -- Gaussian random fields by direct matrix decomposition
// (Sec. 5, Algorithm 2) on GB300: Matern covariance matrices (step 1), their
// LDL^T factorisation (step 2) and U = L D^(1/2) Z (step 4; Z comes from the
// generator's normals, step 3).
//
// The factorisation is a right-looking blocked LDL^T with 128-column panels:
//   1. the 128 x 128 diagonal block is factored (and its unit lower factor
//      inverted) by one CTA per matrix in double-float arithmetic;
//   2. the panel below it, L_ik = A_ik L_kk^-T D_k^-1, and
//   3. the trailing update A_ij -= L_ik D_k L_jk^T
// are fp64 matrix products with K = 128, computed on the tensor cores by an
// error-free splitting of each fp64 operand into S bf16 slices (the Ozaki
// scheme: Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix
// multiplication by using fast routines of matrix multiplication and its
// applications", Numer. Algorithms 59 (2012)), here in its fixed-point form:
//   * every operand row i is scaled by 2^-e_i so that its entries lie in
//     (-1/2, 1/2), rounded to a 7S-bit fixed-point integer X and cut into S
//     balanced base-128 digits s_0 .. s_(S-1) (|s_p| <= 64, exact in bf16):
//     a_ik ~ 2^e_i sum_p s_p 2^(-7(p+1)), error <= 2^(e_i - 7S - 1);
//   * the digit products of one level l = p + q (p, q < S, l < S) are summed
//     by tcgen05.mma into one fp32 TMEM accumulator; every product is an
//     integer below 2^12 in magnitude, a level holds at most 8 x 128 of them,
//     so each level sum is an exact integer of magnitude <= 2^22;
//   * the S level sums are combined exactly in 128-bit integers (two
//     64-bit words), T = sum_l acc_l 128^(S-1-l) (|T| < 2^69), and the
//     product is T 2^(e_i + f_j - 7(S+1)), rounded once to fp64.
// Levels l >= S are dropped: with S = 8 their weight is below 2^-63 of the
// leading term, under the 2^-57 truncation of the operands themselves.
#pragma once
#include <stdint.h>

#include <type_traits>

#include "matern.cuh"
#include "ozaki_round.cuh"
#include "tc_sm100.cuh"
#include "transforms_df.cuh"

namespace mrg {
namespace grf {

constexpr int NB = 128;        // panel width (the K extent of every product)
constexpr int BM = 128;        // output tile rows (MMA M)
constexpr int BN = 64;         // output tile columns (MMA N)
constexpr int RB_A = 128;      // rows per block of an A-role operand image
constexpr int RB_B = 64;       // rows per block of a B-role operand image
constexpr uint32_t SLICE_A = RB_A * NB * 2;  // bytes of one bf16 slice of an A block (32 KB)
constexpr uint32_t SLICE_B = RB_B * NB * 2;  // (16 KB)
constexpr uint64_t WAIT_NS = 2000000000ull;  // bound of every device wait (2 s)

// Error flags a kernel records (bitwise or) in the caller's status word.
constexpr int ERR_TIMEOUT = 1;

// 32-byte global accesses of four doubles (address 32-byte aligned).
__device__ __forceinline__ void ld_v4f64(const double* p, double* v) {
  asm volatile("ld.global.v4.f64 {%0, %1, %2, %3}, [%4];"
               : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
               : "l"(p));
}
__device__ __forceinline__ void st_v4f64(double* p, const double* v) {
  asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(v[0]), "d"(v[1]),
               "d"(v[2]), "d"(v[3])
               : "memory");
}

// ---------------------------------------------------------------------------
// Step 1: Matern covariance (Sec. 5).  Sigma_ij = var * corr(x), x =
// sqrt(8 kappa) |d_ij| / phi, d_ij = diag(1, omega) R(theta) (x_i - x_j).
// ---------------------------------------------------------------------------

struct MaternParams {
  double kappa, var, norm;       // norm = 2^(1-kappa) / Gamma(kappa)
  double scale;                  // sqrt(8 kappa) / phi
  double c, s, omega;            // cos theta, sin theta, anisotropy ratio
};

__device__ __forceinline__ double matern_cov_at(const MaternParams& p, double dx, double dy) {
  const double u = p.c * dx - p.s * dy;
  const double v = p.omega * (p.s * dx + p.c * dy);
  const double x = p.scale * sqrt(u * u + v * v);
  return p.var * matern_corr(x, p.kappa, p.norm);
}

// Raster of nrow x ncol square cells (row-major point order, point k at
// column k mod ncol, row k div ncol): the covariance depends only on the
// offset (dr, dc) between two cells, so it is evaluated once per offset,
// dr in (-nrow, nrow), dc in (-ncol, ncol), table[(dr + nrow - 1) (2 ncol - 1)
// + dc + ncol - 1].  The offsets (dr, dc) and (-dr, -dc) have the same
// covariance and mirror indices o and per - 1 - o around the centre
// c = (per - 1) / 2 (per is odd), so one thread per (matrix, o >= c)
// evaluates it once and writes both entries (the evaluation is bound by the
// FP64 pipe).
__global__ void __launch_bounds__(256) matern_offsets_kernel(const MaternParams* __restrict__ prm,
                                                             uint32_t batch, uint32_t nrow,
                                                             uint32_t ncol, double cell,
                                                             double* __restrict__ table) {
  const uint64_t per = (uint64_t)(2 * nrow - 1) * (2 * ncol - 1);
  const uint64_t half = per / 2 + 1;                 // o = c .. per - 1
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= half * batch) return;
  const uint32_t b = (uint32_t)(t / half);
  const uint64_t o = per / 2 + (t - (uint64_t)b * half);
  const int dr = (int)(o / (2 * ncol - 1)) - (int)(nrow - 1);
  const int dc = (int)(o % (2 * ncol - 1)) - (int)(ncol - 1);
  const double v = matern_cov_at(prm[b], dc * cell, dr * cell);
  table[(uint64_t)b * per + o] = v;
  table[(uint64_t)b * per + (per - 1 - o)] = v;
}

// Fills the n x n matrices (n = nrow ncol, leading dimension ld) from the
// offset tables.  A block item is a run of 1024 columns of one row of one
// matrix (its matrix, row and run derived once per block, by a grid-stride
// loop over the items); each thread takes four consecutive columns, walking
// their (row, column) cells by increments, and writes them with one 32-byte
// store when `vec` (cov, ld and the matrix stride allow it) or one by one.
// 32-bit index arithmetic inside a row: n <= 2^20.
__global__ void __launch_bounds__(256) matern_fill_kernel(const double* __restrict__ table,
                                                          uint32_t batch, uint32_t nrow,
                                                          uint32_t ncol, double* __restrict__ cov,
                                                          uint64_t ld, uint64_t mstride, int vec) {
  const uint32_t n = nrow * ncol;
  const uint32_t bpr = (n + 1023) / 1024;            // items per row
  const uint64_t items = (uint64_t)batch * n * bpr;
  const uint32_t tw = 2 * ncol - 1;                  // table row width
  const uint64_t per_t = (uint64_t)(2 * nrow - 1) * tw;
  for (uint64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const uint32_t b = (uint32_t)(it / ((uint64_t)n * bpr));
    const uint64_t rem = it - (uint64_t)b * n * bpr;
    const uint32_t i = (uint32_t)(rem / bpr);
    const uint32_t x = (uint32_t)(rem - (uint64_t)i * bpr);
    const uint32_t j0 = x * 1024 + 4 * threadIdx.x;
    if (j0 >= n) continue;
    const uint32_t ri = i / ncol, ci = i - (i / ncol) * ncol;
    uint32_t rj = j0 / ncol, cj = j0 - (j0 / ncol) * ncol;
    // entry (dr, dc) at (dr + nrow - 1) tw + dc + ncol - 1, dr = ri - rj, dc = ci - cj
    const double* tb = table + (uint64_t)b * per_t + (uint64_t)(ri + nrow - 1) * tw + (ci + ncol - 1);
    double v[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      v[e] = j0 + e < n ? tb[-(int64_t)rj * tw - (int64_t)cj] : 0.0;
      if (++cj == ncol) {
        cj = 0;
        ++rj;
      }
    }
    double* row = cov + (uint64_t)b * mstride + (uint64_t)i * ld + j0;
    if (vec && j0 + 4 <= n) {
      st_v4f64(row, v);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (j0 + e < n) row[e] = v[e];
    }
  }
}

// Arbitrary points (n x 2, x then y, device): one entry per thread.
__global__ void __launch_bounds__(256) matern_points_kernel(const MaternParams* __restrict__ prm,
                                                            uint32_t batch, const double* __restrict__ xy,
                                                            uint64_t n, double* __restrict__ cov,
                                                            uint64_t ld, uint64_t mstride) {
  const uint64_t per = n * n;
  const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < per * batch; t += step) {
    const uint32_t b = (uint32_t)(t / per);
    const uint64_t rem = t - (uint64_t)b * per;
    const uint64_t i = rem / n, j = rem - i * n;
    const double dx = xy[2 * i] - xy[2 * j], dy = xy[2 * i + 1] - xy[2 * j + 1];
    cov[(uint64_t)b * mstride + i * ld + j] = i == j ? prm[b].var : matern_cov_at(prm[b], dx, dy);
  }
}

// ---------------------------------------------------------------------------
// Operand slicing.  An operand of the products is a set of rows with a K
// extent of 128 (zero beyond the panel's width), stored as an image of
// blocks of RB rows; block b holds S slices of RB x 128 bf16 each, in the
// shared-memory layout the MMA reads (tc_sm100.cuh), so that a block's slice
// is one contiguous bulk copy.  exps[row] = e_row.
// ---------------------------------------------------------------------------

// Biased exponent field of an fp64 value (0 for zero and subnormals).
__device__ __forceinline__ int biased_exp(double v) {
  return (int)((__double_as_longlong(v) >> 52) & 0x7FF);
}

// round(v 2^-e 2^(7S)) as an integer, for |v| < 2^(e-1); subnormals give 0.
template <int S>
__device__ __forceinline__ int64_t fixed_point(double v, int e) {
  const uint64_t bits = (uint64_t)__double_as_longlong(v);
  const int eb = (int)((bits >> 52) & 0x7FF);
  if (eb == 0) return 0;
  const uint64_t m = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  // v = m 2^(eb - 1075); X = m 2^(eb - 1075 + 7S - e) = m >> sh
  const int sh = 1075 - eb - 7 * S + e;
  int64_t x;
  if (sh <= 0) x = (int64_t)(m << (-sh));          // sh >= -2 (|v| < 2^(e-1), S <= 8)
  else if (sh >= 60) x = 0;
  else x = (int64_t)((m + (1ull << (sh - 1))) >> sh);
  return (bits >> 63) ? -x : x;
}

// bf16 bits of a small integer d (|d| <= 64: exact).
__device__ __forceinline__ uint32_t bf16_of_small_int(int d) {
  return __float_as_uint(__int_as_float(0x4B400000 + d) - 12582912.0f) >> 16;
}

// One row of an operand, four consecutive K elements per lane (k = 4 lane ..
// 4 lane + 3, zero beyond the panel), sliced by one warp: the row exponent
// (warp maximum), then S digits per element written into the image block
// `blk` (RB rows) at row rr.  A-role blocks hold the S slices one after the
// other, each an RB-row operand; B-role blocks (`stacked`) hold them as one
// operand of S RB rows, slice p's row r at row p RB + r, so that one MMA can
// take several consecutive slices as the rows of a wider N.  All 32 lanes
// must call it.
template <int S>
__device__ __forceinline__ void slice_row(const double v[4], uint8_t* __restrict__ blk, int RB,
                                          int rr, int32_t* __restrict__ exp_out, bool stacked) {
  const int lane = threadIdx.x & 31;
  int emax = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) emax = max(emax, biased_exp(v[i]));
  emax = __reduce_max_sync(0xffffffffu, emax);
  // |v| < 2^(emax - 1022) = 2^(e - 1): entries of the scaled row lie in (-1/2, 1/2)
  const int e = emax == 0 ? 0 : emax - 1023 + 2;
  uint32_t dig[S][2];
  int64_t x[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) x[i] = emax == 0 ? 0 : fixed_point<S>(v[i], e);
  uint32_t d16[S][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t X = x[i];
#pragma unroll
    for (int p = S - 1; p >= 1; --p) {
      const int d = (int)((X + 64) & 127) - 64;   // balanced digit in [-64, 63]
      d16[p][i] = bf16_of_small_int(d);
      X = (X - d) >> 7;
    }
    d16[0][i] = bf16_of_small_int((int)X);        // |X| <= 64
  }
#pragma unroll
  for (int p = 0; p < S; ++p) {
    dig[p][0] = d16[p][0] | (d16[p][1] << 16);
    dig[p][1] = d16[p][2] | (d16[p][3] << 16);
  }
  // stacked: row p RB + rr of an S RB-row operand (its 8-row groups advance
  // 1024 bytes, so slice p starts RB 128 bytes after slice p - 1 in each
  // 64-element K half); else row rr of slice p's own RB-row operand
  const uint32_t off = stacked ? tc::sw128_offset((uint32_t)(S * RB), (uint32_t)rr, (uint32_t)(4 * lane))
                               : tc::sw128_offset((uint32_t)RB, (uint32_t)rr, (uint32_t)(4 * lane));
  const size_t pstride = stacked ? (size_t)RB * 128 : (size_t)RB * NB * 2;
#pragma unroll
  for (int p = 0; p < S; ++p)
    *reinterpret_cast<uint2*>(blk + (size_t)p * pstride + off) = make_uint2(dig[p][0], dig[p][1]);
  if (lane == 0) *exp_out = e;
}

// Slices rows [0, rows_pad) of a panel: row r is a[(r) * lda + k] for k < kb
// (zero for r >= rows or k >= kb).  When img_a is set, into img_a (A role,
// 128-row blocks) as is; when img_b is set, into img_b (B role, 64-row
// blocks), multiplied by colscale[k] if that is set (W = L D).  One warp per
// row.
struct SliceArgs {
  const double* a;
  uint64_t lda, a_mstride;
  uint32_t rows, rows_pad, kb;
  uint8_t* img_a;
  int32_t* exp_a;
  uint64_t img_a_mstride, exp_a_mstride;
  uint8_t* img_b;
  int32_t* exp_b;
  uint64_t img_b_mstride, exp_b_mstride;
  const double* colscale;
  uint64_t colscale_mstride;
};

template <int S>
__global__ void __launch_bounds__(256) slice_kernel(SliceArgs g) {
  const uint32_t b = blockIdx.y;
  const uint32_t r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (r >= g.rows_pad) return;  // whole warps leave together
  const int lane = threadIdx.x & 31;
  const double* row = g.a + b * g.a_mstride + (uint64_t)r * g.lda;
  double v[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t k = 4 * lane + i;
    v[i] = (r < g.rows && k < g.kb) ? row[k] : 0.0;
  }
  if (g.img_a)
    slice_row<S>(v, g.img_a + b * g.img_a_mstride + (uint64_t)(r / RB_A) * S * SLICE_A, RB_A,
                 (int)(r % RB_A), g.exp_a + b * g.exp_a_mstride + r, false);
  if (g.img_b) {
    if (g.colscale) {
      const double* cs = g.colscale + b * g.colscale_mstride;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint32_t k = 4 * lane + i;
        v[i] = k < g.kb ? v[i] * cs[k] : 0.0;
      }
    }
    slice_row<S>(v, g.img_b + b * g.img_b_mstride + (uint64_t)(r / RB_B) * S * SLICE_B, RB_B,
                 (int)(r % RB_B), g.exp_b + b * g.exp_b_mstride + r, true);
  }
}

// ---------------------------------------------------------------------------
// The products on the tensor cores, on 128 x 64 output tiles: the B block's
// S slices stay in shared memory while the A block's slices stream through a
// ring of NST stages; A slice p meets B slices q = 0 .. S-1-p in TMEM
// accumulator p + q (64 columns each, S x 64 <= 512); the accumulators are
// combined exactly and the result written (PANEL: C = product) or subtracted
// (TRAIL: C -= product) in fp64.
// ---------------------------------------------------------------------------

struct GemmArgs {
  const uint8_t* img_a;    // A-role image: block ti = rows [128 ti, 128 ti + 128) of the output
  const int32_t* exp_a;
  const uint8_t* img_b;    // B-role image: block tj = columns [64 tj, 64 tj + 64)
  const int32_t* exp_b;
  uint64_t img_a_mstride, exp_a_mstride, img_b_mstride, exp_b_mstride;
  double* c;               // output element (r, col) at c + b c_mstride + r ldc + col
  uint64_t ldc, c_mstride;
  uint32_t m, n;           // output rows and columns
  uint32_t tiles_n;        // rectangle tile sets: column tiles per row of tiles
  int tile_set;            // TRAIL: TILES_LOWER, TILES_NEXT (tj < 2) or TILES_REST (tj >= 2)
  uint32_t tiles_total;    // tiles of the set per matrix
  uint32_t batch;          // matrices
  uint32_t per_cta;        // consecutive items (tiles) each CTA processes
  int vec32;               // c and ldc * 8 are multiples of 32 bytes (vector row access)
  int* status;
};

// Tile sets of a trailing update: all lower tiles, the two tile columns of
// the next panel (a rectangle: tiles_n = 2), or the lower tiles right of it.
constexpr int TILES_LOWER = 0, TILES_NEXT = 1, TILES_REST = 2;

template <int S>
struct GemmSmem {
  static constexpr int NST = 3;                                   // A-slice ring stages
  static constexpr uint32_t B_BYTES = (uint32_t)S * SLICE_B;
  static constexpr uint32_t A_OFF = B_BYTES;
  static constexpr uint32_t BAR_OFF = A_OFF + NST * SLICE_A;
  // mbarriers: full_b, full_a[NST], empty_a[NST], level[S], tmem_free; then
  // the TMEM base address and the abort flag
  static constexpr uint32_t TOTAL = BAR_OFF + 256 + 1024;         // + alignment slack
};

// Tile (ti, tj) of the lower-triangular tile set of an m x m output with
// 128 x 64 tiles: row of tiles ti holds tiles tj < min(2 ti + 2, tiles_n).
__device__ __forceinline__ void lower_tile(uint32_t x, uint32_t& ti, uint32_t& tj) {
  uint32_t t = (uint32_t)((sqrtf(4.0f * (float)x + 1.0f) - 1.0f) * 0.5f);
  while ((uint64_t)(t + 1) * (t + 2) <= x) ++t;
  while ((uint64_t)t * (t + 1) > x) --t;
  ti = t;
  tj = x - t * (t + 1);
}

// Warps 0-15 drain TMEM (warp w reads lanes 32 (w mod 4) .. 32 (w mod 4) + 31,
// as tcgen05.ld requires); warp 16 allocates TMEM and its lane 0 issues the
// copies and the MMAs.  (The runtime charges a block's registers in groups of
// four warps, so 17 warps leave 96 registers per thread, as measured.)
constexpr int EPI_WARPS = 16;
constexpr int PRODUCER_WARP = EPI_WARPS;
constexpr int GEMM_THREADS = (EPI_WARPS + 1) * 32;
constexpr int EPI_COLS = BN * 4 / EPI_WARPS;   // columns per epilogue thread (16)

// The tile (ti, tj) of item x of the tile set (identical for every thread),
// column by column: consecutive items share their column of tiles and so
// their B block, which a CTA then loads once for its whole run of them.
__device__ __forceinline__ void tile_of(const GemmArgs& g, bool trail, uint32_t x, uint32_t& ti,
                                        uint32_t& tj) {
  const uint32_t rows = (g.m + BM - 1) / BM;   // tile rows of the output
  if (trail && g.tile_set == TILES_REST) {
    // lower tiles right of the next panel: column tj >= 2 holds the tile rows
    // ti >= tj / 2 (64 tj < 128 (ti + 1)), rows - tj / 2 of them; columns
    // 2 m and 2 m + 1 hold rows - m each, so (m - 1)(2 rows - m) items
    // precede column 2 m: solve for m, then place x in the pair
    const float bq = 2.0f * (float)rows + 1.0f;
    const float disc = fmaxf(bq * bq - 4.0f * (2.0f * (float)rows + (float)x), 0.0f);
    uint32_t m = max((uint32_t)((bq - sqrtf(disc)) * 0.5f), 1u);
    auto before = [rows](uint32_t mm) { return (mm - 1) * (2 * rows - mm); };
    while (m + 1 <= rows && before(m + 1) <= x) ++m;
    while (m > 1 && before(m) > x) --m;
    const uint32_t y = x - before(m);
    if (y < rows - m) {
      tj = 2 * m;
      ti = m + y;
    } else {
      tj = 2 * m + 1;
      ti = m + y - (rows - m);
    }
  } else if (trail && g.tile_set == TILES_LOWER) {
    lower_tile(x, ti, tj);
  } else {   // a rectangle of tiles_n columns of tiles (the panel; the next panel of a trailing update)
    ti = x % rows;
    tj = x / rows;
  }
}

// One CTA takes `per_cta` consecutive items of the flat set (matrix-major:
// item = b * tiles + x).  Warp 16 produces: its lane 0 streams the A block's
// slices through a ring of NST stages without a break between tiles (the
// next tile's first slices load while this tile's last ones multiply),
// reloads the B block only when the tile column changes, and issues for A
// slice p the MMAs with B slices q = 0 .. S-1-p into TMEM accumulator p + q.
// Level l (accumulator l) is final once slices 0 .. l are multiplied: after
// each slice (in kSliceOrder) a commit on level[l] marks every level that
// became final there; the 16 epilogue warps read and fold each level while
// the remaining slices multiply, release TMEM
// after the last level (tmem_free), and round and store the tile while the
// next tile's MMAs run.  The MMA issue is fully unrolled over precomputed
// descriptors.  Every wait is bounded; after a timeout the producer keeps
// committing (empty) level barriers so that no warp waits out more bounds.
// The order in which a tile's A slices are multiplied: long and short ones
// alternate (slice p takes S - p products), so that two consecutive slices
// always outlast the copy of the next one into the ring.  Slice 0 comes
// first: its MMAs initialise every level.  kLevelsDone(i): the levels that
// are final once the first i + 1 slices of the order are done (level l
// needs slices 0 .. l), as a bit mask of the levels newly final there.
__host__ __device__ constexpr int kSliceOrder(int i) {
  return (i & 1) ? 7 - (i >> 1) : (i >> 1);   // 0, 7, 1, 6, 2, 5, 3, 4
}
__host__ __device__ constexpr uint32_t kLevelsDone(int i) {
  return i == 7 ? 0xF0u : (i & 1) ? 0u : 1u << (i >> 1);
}

template <int S, bool TRAIL>
__global__ void __launch_bounds__(GEMM_THREADS, 1) ozaki_gemm_kernel(GemmArgs g) {
  using SM = GemmSmem<S>;
  constexpr int NST = SM::NST;
  static_assert(S == 8 && NST == 3, "the unrolled MMA schedule below is written for 8 slices");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  uint8_t* sB = smem;
  uint8_t* sA = smem + SM::A_OFF;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::BAR_OFF);
  uint64_t* full_b = bar;                     // [1]
  uint64_t* full_a = bar + 1;                 // [NST]
  uint64_t* empty_a = bar + 1 + NST;          // [NST]
  uint64_t* level = bar + 1 + 2 * NST;        // [S]
  uint64_t* tmem_free = level + S;            // [1], EPI_WARPS arrivals per tile
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tmem_free + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_free + 2);

  const uint64_t total = (uint64_t)g.tiles_total * g.batch;
  const uint64_t it0 = (uint64_t)blockIdx.x * g.per_cta;
  if (it0 >= total) return;                  // uniform over the CTA, before any allocation
  const uint32_t nit = (uint32_t)(total - it0 < g.per_cta ? total - it0 : g.per_cta);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    tc::mbar_init(full_b, 1);
    for (int i = 0; i < NST; ++i) {
      tc::mbar_init(&full_a[i], 1);
      tc::mbar_init(&empty_a[i], 1);
    }
    for (int l = 0; l < S; ++l) tc::mbar_init(&level[l], 1);
    tc::mbar_init(tmem_free, EPI_WARPS);
    *abort_flag = 0;
    tc::fence_barrier_init();
  }
  if (warp == PRODUCER_WARP) tc::tmem_alloc(tslot, 512);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tslot;

  // item -> matrix, tile and operand blocks
  auto item = [&](uint32_t k, uint32_t& b, uint32_t& ti, uint32_t& tj) {
    const uint64_t it = it0 + k;
    b = (uint32_t)(it / g.tiles_total);
    tile_of(g, TRAIL, (uint32_t)(it - (uint64_t)b * g.tiles_total), ti, tj);
  };
  auto a_block = [&](uint32_t k) {
    uint32_t b, ti, tj;
    item(k, b, ti, tj);
    return g.img_a + b * g.img_a_mstride + (uint64_t)ti * S * SLICE_A;
  };

  if (warp == PRODUCER_WARP) {
    if (lane == 0) {
      bool ok = true;
      const uint64_t ad0 = tc::sw128_desc(tc::smem_u32(sA));
      const uint64_t bd0 = tc::sw128_desc(tc::smem_u32(sB));
      const uint32_t dhi = (uint32_t)(ad0 >> 32);   // equal for both operands
      const uint32_t alo0 = (uint32_t)ad0, blo0 = (uint32_t)bd0;
      // the first tile's B block and A slices 0 .. NST-1
      uint32_t b, ti, tj;
      item(0, b, ti, tj);
      uint32_t cur_b = b, cur_tj = tj, bloads = 1;
      tc::mbar_arrive_expect_tx(full_b, SM::B_BYTES);
      tc::bulk_g2s(sB, g.img_b + b * g.img_b_mstride + (uint64_t)tj * S * SLICE_B, SM::B_BYTES,
                   full_b);
      const uint8_t* gA0 = a_block(0);
#pragma unroll
      for (int i = 0; i < NST; ++i) {
        tc::mbar_arrive_expect_tx(&full_a[i], SLICE_A);
        tc::bulk_g2s(sA + i * SLICE_A, gA0 + (size_t)kSliceOrder(i) * SLICE_A, SLICE_A, &full_a[i]);
      }
      const uint8_t* gA_nxt = nit > 1 ? a_block(1) : gA0;
      for (uint32_t k = 0; k < nit; ++k) {
        item(k, b, ti, tj);
        const uint8_t* gA_cur = k == 0 ? gA0 : gA_nxt;
        if (k > 0) gA_nxt = k + 1 < nit ? a_block(k + 1) : gA_cur;
        if (k > 0 && (b != cur_b || tj != cur_tj)) {
          // a new tile column: its B block replaces the old one once every
          // MMA of the previous tile (the last to read it) has completed
          if (ok) ok = tc::mbar_wait(&level[S - 1], (k - 1) & 1, WAIT_NS);
          if (ok) {
            tc::mbar_arrive_expect_tx(full_b, SM::B_BYTES);
            tc::bulk_g2s(sB, g.img_b + b * g.img_b_mstride + (uint64_t)tj * S * SLICE_B,
                         SM::B_BYTES, full_b);
            ++bloads;
          }
          cur_b = b;
          cur_tj = tj;
        }
        // the previous tile's accumulators have all been read
        if (k > 0 && ok) ok = tc::mbar_wait(tmem_free, (k - 1) & 1, WAIT_NS);
        if (ok) ok = tc::mbar_wait(full_b, (bloads - 1) & 1, WAIT_NS);
        if (ok) tc::tc_fence_after();
#pragma unroll
        for (int i = 0; i < S; ++i) {
          const int p = kSliceOrder(i);              // the A slice of this position
          const uint32_t gp = k * S + (uint32_t)i;   // position over the CTA's run
          const int st = (int)(gp % NST);
          if (ok) ok = tc::mbar_wait(&full_a[st], (gp / NST) & 1, WAIT_NS);
          if (ok) {
            tc::tc_fence_after();
            // descriptor start addresses advance in 16-byte units
            const uint32_t alo = alo0 + (uint32_t)((st * SLICE_A) >> 4);
            // the S - p products of slice p as MMAs over up to four consecutive
            // B slices each (rows 64 q0 .. of the stacked B block, N = 64 c):
            // their accumulators, levels p + q0 .. p + q0 + c - 1, are
            // adjacent TMEM columns
#pragma unroll
            for (int q0 = 0; q0 < S - p; q0 += 4) {
              const int c = S - p - q0 < 4 ? S - p - q0 : 4;
              const uint32_t idesc = tc::idesc_bf16_f32(BM, (uint32_t)(BN * c));
              const uint32_t blo = blo0 + (uint32_t)((q0 * RB_B * 128) >> 4);
              const uint32_t d = tmem + (uint32_t)(p + q0) * BN;
#pragma unroll
              for (int kk = 0; kk < NB / 16; ++kk)
                tc::mma_bf16_lo(d, alo + (uint32_t)(((kk >> 2) * (RB_A * 128) + (kk & 3) * 32) >> 4),
                                blo + (uint32_t)(((kk >> 2) * (S * RB_B * 128) + (kk & 3) * 32) >> 4),
                                dhi, idesc, (p > 0 || kk > 0) ? 1u : 0u);
            }
          }
          tc::mma_commit(&empty_a[st]);   // stage st is free once these MMAs are done
#pragma unroll
          for (int l = 0; l < S; ++l)      // and these levels are final
            if (kLevelsDone(i) & (1u << l)) tc::mma_commit(&level[l]);
          // refill the stage of position gp - 1 with position gp - 1 + NST
          // (this tile's or the next tile's) once the MMAs of gp - 1 are done
          if (gp >= 1) {
            const uint32_t gr = gp - 1 + NST;
            if (gr / S < nit) {
              const int sr = (int)((gp - 1) % NST);
              if (ok) ok = tc::mbar_wait(&empty_a[sr], ((gp - 1) / NST) & 1, WAIT_NS);
              if (ok) {
                tc::mbar_arrive_expect_tx(&full_a[sr], SLICE_A);
                const uint8_t* src = (gr / S == k ? gA_cur : gA_nxt) +
                                     (size_t)kSliceOrder((int)(gr % S)) * SLICE_A;
                tc::bulk_g2s(sA + sr * SLICE_A, src, SLICE_A, &full_a[sr]);
              }
            }
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(g.status, ERR_TIMEOUT);
      }
    }
    __syncwarp();
  } else {
    const int quarter = warp & 3, part = warp >> 2;
    const uint32_t r = (uint32_t)(quarter * 32 + lane);
    const uint32_t tlane = tmem + ((uint32_t)(quarter * 32) << 16);
    const uint32_t c0 = (uint32_t)part * EPI_COLS;   // this thread's first column inside the tile
    for (uint32_t k = 0; k < nit; ++k) {
      uint32_t b, ti, tj;
      item(k, b, ti, tj);
      const uint32_t row = ti * BM + r, cbeg = tj * BN + c0;
      const bool row_ok = row < g.m;
      const int ea = row_ok ? g.exp_a[b * g.exp_a_mstride + row] : 0;
      if (TRAIL && row_ok && cbeg < g.n) {   // the old C values, read at the end of the tile
        const double* cp = g.c + b * g.c_mstride + (uint64_t)row * g.ldc + cbeg;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(cp));
        if (cbeg + EPI_COLS - 1 < g.n)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(cp + EPI_COLS - 1));
      }
      // Level l as the integer bits(acc_l + 1.5 2^23) - 0x4B400000 (exact:
      // |acc_l| <= 2^22), folded as the levels become final:
      // T = sum_l acc_l 128^(7-l) = t_hi 2^28 + t_lo with
      //   t_hi = (acc_0 128 + acc_1) 2^14 + acc_2 128 + acc_3   (< 2^44)
      //   t_lo = (acc_4 128 + acc_5) 2^14 + acc_6 128 + acc_7
      // (each pair in 32-bit wrapping arithmetic: it fits in 30 bits)
      constexpr uint32_t M129 = 0x4B400000u * 129u;   // the offsets of a pair (mod 2^32)
      uint32_t u[EPI_COLS];
      int32_t pa[EPI_COLS];
      int64_t th[EPI_COLS], tl[EPI_COLS];
      bool ok = true;
#pragma unroll
      for (int l = 0; l < S; ++l) {
        if (ok) ok = tc::mbar_wait(&level[l], k & 1, WAIT_NS);
        ok = __all_sync(0xffffffffu, ok);
        tc::tc_fence_after();
        float acc[EPI_COLS];
        tc::tmem_ld8(tlane + (uint32_t)l * BN + c0, acc);
        tc::tmem_ld8(tlane + (uint32_t)l * BN + c0 + 8, acc + 8);
        tc::tmem_ld_wait();
#pragma unroll
        for (int c = 0; c < EPI_COLS; ++c) {
          const uint32_t v = __float_as_uint(acc[c] + 12582912.0f);
          if ((l & 1) == 0) {
            u[c] = v;
          } else {
            const int32_t pr = (int32_t)(u[c] * 128u + v - M129);
            if (l == 1 || l == 5) pa[c] = pr;
            else if (l == 3) th[c] = (int64_t)pa[c] * 16384 + pr;
            else tl[c] = (int64_t)pa[c] * 16384 + pr;
          }
        }
      }
      // every level read: the next tile's MMAs may overwrite the columns
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(tmem_free);
      if (!ok) {
        if (lane == 0) {
          *abort_flag = 1;
          atomicOr(g.status, ERR_TIMEOUT);
        }
        continue;
      }
      if (!row_ok) continue;
      // T 2^(e_row + e_col - 7 (S + 1)), rounded once, written (panel) or
      // subtracted from the old value (trailing update)
      double* crow = g.c + b * g.c_mstride + (uint64_t)row * g.ldc;
      const int32_t* eb = g.exp_b + b * g.exp_b_mstride;
      const int ebase = ea - 7 * (S + 1);
      const bool vec = g.vec32 != 0 && cbeg + EPI_COLS <= g.n;
#pragma unroll
      for (int kc = 0; kc < EPI_COLS; kc += 8) {
        double v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int c = kc + e;
          const uint32_t col = cbeg + (uint32_t)c;
          v[e] = ozaki_round(th[c], tl[c], ebase + (col < g.n ? eb[col] : 0));
        }
        const uint32_t colc = cbeg + (uint32_t)kc;
        if (vec) {
          if (TRAIL) {
            double cv[8];
            ld_v4f64(crow + colc, cv);
            ld_v4f64(crow + colc + 4, cv + 4);
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = cv[e] - v[e];
          }
          st_v4f64(crow + colc, v);
          st_v4f64(crow + colc + 4, v + 4);
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const uint32_t col = colc + e;
            if (col < g.n) crow[col] = TRAIL ? crow[col] - v[e] : v[e];
          }
        }
      }
    }
  }
  // every MMA has completed (the epilogue waited for the last level of every
  // tile) and every TMEM load has been waited for
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == PRODUCER_WARP) tc::tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------
// Diagonal block: LDL^T of a kb x kb block (kb <= 128) by one CTA of
// DIAG_THREADS per matrix (ldl_diag_kernel), then the inverse X of its unit
// lower factor by columns on many CTAs (ldl_inverse_kernel), in
// double-float arithmetic (fp32 pairs; GB300's FP64 rate is a small fraction
// of its FP32 rate) on the block scaled by a power of two (its largest
// diagonal entry brought near 1, so that fp32's exponent range holds it).
// Writes L (strict lower part of the block, unit diagonal implied), D (on the
// block's diagonal and into d[]), and the panel product's B operand, row n
// of B = row n of X divided by d_n (so that L_ik = A_ik B^T), which
// slice_kernel then cuts into digit planes.
// ---------------------------------------------------------------------------

constexpr int DG = NB + 1;   // row pitch of the shared block, in float pairs (odd: fewer bank conflicts)

struct DiagArgs {
  double* a;
  uint64_t lda, a_mstride;
  double* d;
  uint64_t d_mstride;
  uint32_t k0, kb;
  uint8_t* img_x;
  int32_t* exp_x;
  uint64_t img_x_mstride, exp_x_mstride;
  int* info;               // per matrix: 0, or 1 + the first non-positive pivot's index
};

// x 2^-sc as a double-float, in integers (no FP64 instruction): hi = x
// rounded to fp32 at bit 29 of the significand, lo = the remainder (up to 29
// bits, rounded to fp32).  Requires x 2^-sc zero or within fp32's normal range.
__device__ __forceinline__ df df_of_scaled(double x, int sc) {
  const uint64_t bits = (uint64_t)__double_as_longlong(x);
  const int e = (int)((bits >> 52) & 0x7FF);
  if (e == 0) return df{0.0f, 0.0f};
  const uint32_t sgn = (uint32_t)(bits >> 32) & 0x80000000u;
  const uint64_t m = bits & 0xFFFFFFFFFFFFFull;
  const uint64_t mh = (m + 0x0FFFFFFFull + ((m >> 29) & 1)) >> 29;   // 23 bits (+ a carry)
  const int ef = e - sc - 1023 + 127;                                 // biased fp32 exponent
  if (ef <= 0) return df{0.0f, 0.0f};                                 // below 2^-126: flushed
  if (ef >= 255) return df{__uint_as_float(sgn | 0x7F800000u), 0.0f};  // beyond fp32: inf
  const float hi = __uint_as_float(sgn | (((uint32_t)ef << 23) + (uint32_t)mh));
  const int64_t r = (int64_t)m - (int64_t)(mh << 29);                 // |r| <= 2^28
  // lo = r 2^(e - sc - 1023 - 52); its scale as a float while that is normal
  if (ef <= 52) return df{hi, 0.0f};
  const float lo = __fmul_rn(__ll2float_rn(sgn ? -r : r), __uint_as_float((uint32_t)(ef - 52) << 23));
  return df{hi, lo};
}

// A normalised double-float times 2^sc as a double (integer conversion of
// the pair, then the exponent moved; zero stays zero).
__device__ __forceinline__ double f64_of_scaled(df v, int sc) {
  uint64_t bits = df_to_f64_bits(v);
  if ((bits & 0x7FFFFFFFFFFFFFFFull) != 0) bits += (uint64_t)(int64_t)sc << 52;
  return __longlong_as_double((long long)bits);
}

// a - b c in double-float
__device__ __forceinline__ df df_fnms(df a, df b, df c) {
  const float p = __fmul_rn(b.hi, c.hi);
  float e = __fmaf_rn(b.hi, c.hi, -p);
  e = __fmaf_rn(b.hi, c.lo, e);
  e = __fmaf_rn(b.lo, c.hi, e);
  const df s = two_sum(a.hi, -p);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(a.lo, e)));
}

// 1 / d in double-float: approximate fp32 reciprocal and one Newton step whose residual
// 1 - d r0 is formed exactly (the product's error by FMA; 1 - p is exact).
__device__ __forceinline__ df df_recip(df d) {
  float r0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(d.hi));   // the Newton step below corrects it
  const float p = __fmul_rn(d.hi, r0);
  const float pe = __fmaf_rn(d.hi, r0, -p);
  const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, p), pe), __fmul_rn(d.lo, r0));
  return fast_two_sum(r0, __fmul_rn(r0, e));
}

constexpr int NPAIR = NB * (NB - 1) / 2;   // pairs (i, l), 1 <= l <= i < 128



// Shared-memory storage of a double-float, 8-byte aligned so that a pair
// moves in one access.
struct __align__(8) dfs {
  float hi, lo;
};
__device__ __forceinline__ df ld_df(const dfs& x) {
  const float2 v = *reinterpret_cast<const float2*>(&x);
  return df{v.x, v.y};
}
__device__ __forceinline__ void st_df(dfs& x, df v) {
  *reinterpret_cast<float2*>(&x) = make_float2(v.hi, v.lo);
}

// The lower triangle (strict: below the diagonal only) of a kb x kb fp64
// block times 2^-sc into a shared double-float array of row pitch DG.
template <int NTH>
__device__ __forceinline__ void load_lower_df(const double* __restrict__ A, uint64_t lda, int kb,
                                              int sc, dfs* dst, bool strict) {
  // warp w takes rows w, w + NW, .., w + (RW - 1) NW, then the next RW;
  // its lanes run along the row (coalesced loads, no index division); a
  // batch's loads (4 RW per lane, kb <= 128) are all in flight before the
  // first conversion
  constexpr int NW = NTH / 32;
  constexpr int RW = NW >= 32 ? 4 : 8;      // rows per batch (registers allow 8 in small blocks)
  const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
  for (int i0 = warp; i0 < kb; i0 += RW * NW) {
    double v[RW][4];
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      const int i = i0 + r * NW;
      const int len = i < kb ? (strict ? i : i + 1) : 0;
      const double* row = A + (uint64_t)i * lda;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = u * 32 + lane;
        v[r][u] = j < len ? row[j] : 0.0;
      }
    }
#pragma unroll
    for (int r = 0; r < RW; ++r) {
      const int i = i0 + r * NW;
      const int len = i < kb ? (strict ? i : i + 1) : 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = u * 32 + lane;
        if (j < len) st_df(dst[i * DG + j], df_of_scaled(v[r][u], sc));
      }
    }
  }
}

// Right-looking LDL^T of the diagonal block, one CTA per matrix: after
// column j of L is known (step j), every thread takes its share of the
// trailing update a_il -= l_ij w_l (j < l <= i < kb, w = column j before
// scaling), from a table of (i, l) pairs ordered by column l descending, so
// that the pairs of step j are a prefix of it: every lane works on every
// step.  DIAG_P steps form a pass, which costs two barriers.  Double-float
// arithmetic on the FP32 pipes (GB300's FP64 pipe retires 1.6 DFMA per
// cycle per SM, against 128 FP32 FMAs).
constexpr int DIAG_THREADS = 1024;
constexpr int DIAG_P = 4;   // pivots per pass of the diagonal block's LDL^T (measured: 3: 88 us, 4: 82, 6: 97; 5 spills)

// P pivots j .. j + P - 1 of the diagonal block's LDL^T in one pass, with
// the operations of one pivot at a time in the same order (so the same
// bits): every thread factors the P x P pivot block itself (pivot c: d_c,
// its column of L below it inside the block, the block's trailing pairs);
// the rows below the block (one thread each) take column c of L and update
// their later pivot columns for c = 0 .. P-1; after one barrier every
// trailing pair (columns >= j + P) receives the P updates.  s_w, s_l:
// [P][NB], the columns before and after scaling.  Returns after the
// trailing barrier.
template <int P>
__device__ __forceinline__ void diag_pass(dfs* __restrict__ sm, dfs* __restrict__ s_w,
                                          dfs* __restrict__ s_l, dfs* __restrict__ s_d,
                                          const uint16_t* __restrict__ s_pair, int* s_bad, int kb,
                                          int j, int tid) {
  constexpr int NT = DIAG_THREADS;
  static_assert(NT >= NB, "one thread per row below the pivot block");
  // only thread 0 and the threads with a row below the block need the
  // pivot block (a prefix of the threads: whole warps drop out)
  const bool active = tid == 0 || j + P + tid < kb;
  df Bk[P][P];                       // the pivot block, lower part
  df rc[P], Wb[P][P], Lb[P][P];
  if (active) {
#pragma unroll
    for (int r = 0; r < P; ++r)
#pragma unroll
      for (int c = 0; c <= r; ++c) Bk[r][c] = ld_df(sm[(j + r) * DG + j + c]);
    int bad = 0;
#pragma unroll
    for (int c = 0; c < P; ++c) {
      const bool pos = Bk[c][c].hi > 0x1p-100f;
      if (!pos && !bad) bad = 1 + c;
      rc[c] = pos ? df_recip(Bk[c][c]) : df{0.0f, 0.0f};
#pragma unroll
      for (int r = c + 1; r < P; ++r) {
        Wb[r][c] = Bk[r][c];
        Lb[r][c] = df_mul(Bk[r][c], rc[c]);
      }
#pragma unroll
      for (int k = c + 1; k < P; ++k)
#pragma unroll
        for (int r = k; r < P; ++r) Bk[r][k] = df_fnms(Bk[r][k], Lb[r][c], Wb[k][c]);
    }
    if (tid == 0) {
#pragma unroll
      for (int c = 0; c < P; ++c) st_df(s_d[j + c], Bk[c][c]);
      if (bad && !*s_bad) *s_bad = j + bad;
    }
    const int i = j + P + tid;
    if (i < kb) {
      df x[P];
#pragma unroll
      for (int c = 0; c < P; ++c) x[c] = ld_df(sm[i * DG + j + c]);
#pragma unroll
      for (int c = 0; c < P; ++c) {
        const df w = x[c];
        const df l = df_mul(w, rc[c]);
        st_df(s_w[c * NB + i], w);
        st_df(s_l[c * NB + i], l);
        st_df(sm[i * DG + j + c], l);
#pragma unroll
        for (int k = c + 1; k < P; ++k) x[k] = df_fnms(x[k], l, Wb[k][c]);
      }
    }
  }
  __syncthreads();
  // the block's own L entries replace its inputs now that every thread has
  // read them (the trailing pairs below start at column j + P)
  if (tid == 0) {
#pragma unroll
    for (int c = 0; c < P; ++c)
#pragma unroll
      for (int r = c + 1; r < P; ++r) st_df(sm[(j + r) * DG + j + c], Lb[r][c]);
  }
  // two elements per thread and trip, loaded before either is computed
  const int np = (kb - P - j) * (kb - P + 1 - j) / 2;   // trailing pairs, columns >= j + P
  for (int t = tid; t < np; t += 2 * NT) {
    const int tb = t + NT;
    const int pa = s_pair[t], pb = tb < np ? s_pair[tb] : pa;   // pb = pa: computed, not stored
    const int ia = pa >> 8, la = pa & 255, ib = pb >> 8, lb = pb & 255;
    df ya = ld_df(sm[ia * DG + la]), yb = ld_df(sm[ib * DG + lb]);
#pragma unroll
    for (int c = 0; c < P; ++c) {
      ya = df_fnms(ya, ld_df(s_l[c * NB + ia]), ld_df(s_w[c * NB + la]));
      yb = df_fnms(yb, ld_df(s_l[c * NB + ib]), ld_df(s_w[c * NB + lb]));
    }
    st_df(sm[ia * DG + la], ya);
    if (tb < np) st_df(sm[ib * DG + lb], yb);
  }
  __syncthreads();
}

template <int S>
__global__ void __launch_bounds__(DIAG_THREADS, 1) ldl_diag_kernel(DiagArgs g) {
  extern __shared__ dfs sm[];              // [NB][DG]: the block, L below the diagonal
  __shared__ dfs s_w[DIAG_P * NB];         // the pass's pivot columns before scaling
  __shared__ dfs s_l[DIAG_P * NB];         // and of L
  __shared__ dfs s_d[NB];                  // the pivots (scaled block)
  __shared__ uint16_t s_pair[NPAIR];       // (i << 8) | l
  __shared__ int s_scale, s_bad;
  const uint32_t b = blockIdx.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int NT = DIAG_THREADS;
  const int kb = (int)g.kb;
  double* A = g.a + b * g.a_mstride + (uint64_t)g.k0 * g.lda + g.k0;
  if (warp == 0) {
    int em = 0;
    for (int j = lane; j < kb; j += 32) em = max(em, biased_exp(A[(uint64_t)j * g.lda + j]));
    em = __reduce_max_sync(0xffffffffu, em);
    if (lane == 0) {
      s_scale = em == 0 ? 0 : em - 1023;
      s_bad = 0;
    }
  }
  // pair table: column l (1 <= l < kb) holds rows l .. kb-1 at offset
  // (kb-1-l)(kb-l)/2
  for (int l = tid + 1; l < kb; l += NT) {
    const int off = (kb - 1 - l) * (kb - l) / 2;
    for (int i = l; i < kb; ++i) s_pair[off + i - l] = (uint16_t)((i << 8) | l);
  }
  __syncthreads();
  const int sc = s_scale;
  load_lower_df<NT>(A, g.lda, kb, sc, sm, false);
  __syncthreads();
  // DIAG_P pivots per pass, then single ones for the last kb mod DIAG_P
  int j = 0;
  for (; j + DIAG_P <= kb; j += DIAG_P) diag_pass<DIAG_P>(sm, s_w, s_l, s_d, s_pair, &s_bad, kb, j, tid);
  for (; j < kb; ++j) diag_pass<1>(sm, s_w, s_l, s_d, s_pair, &s_bad, kb, j, tid);
  // outputs: L (strict lower part) and D into the matrix, one row per warp
  // at a time with the lanes along it (the lower triangle only, no index
  // division), and D into d[]
  for (int i = warp; i < kb; i += NT / 32) {
    double* row = A + (uint64_t)i * g.lda;
    for (int j = lane; j <= i; j += 32)
      row[j] = j < i ? f64_of_scaled(ld_df(sm[i * DG + j]), 0) : f64_of_scaled(ld_df(s_d[i]), sc);
  }
  for (int j = tid; j < kb; j += NT) g.d[b * g.d_mstride + g.k0 + j] = f64_of_scaled(ld_df(s_d[j]), sc);
  if (tid == 0 && s_bad) atomicCAS(&g.info[b], 0, (int)g.k0 + s_bad);
}

// The panel product's B operand from the diagonal block's factor:
// B[n][k] = X[n][k] / d_n with X = L_kk^-1 (unit lower), so that
// L_ik = A_ik L_kk^-T D^-1 = A_ik B^T.  The columns of X are independent
// solutions of L x = e_c: one warp per column, by forward substitution in
// outer-product order (x = e_c; for m = c, c+1, ..: x_i -= L[i][m] x_m for
// i > m -- backward stable per column), lanes over the rows, double-float
// arithmetic, L from the matrix (fp64, written by ldl_diag_kernel).  Grid:
// (columns / INV_COLS, matrices), INV_COLS warps per CTA.  Writes B (fp64, 128 x 128,
// zero outside kb x kb) to bx.
constexpr int INV_COLS = 8;   // columns (warps) per CTA (measured: 4 per CTA, one per SM sub-partition, was slower)

__global__ void __launch_bounds__(INV_COLS * 32) ldl_inverse_kernel(const double* __restrict__ a,
                                                                    uint64_t lda, uint64_t a_mstride,
                                                                    uint32_t k0, uint32_t kb,
                                                                    const double* __restrict__ d,
                                                                    uint64_t d_mstride,
                                                                    double* __restrict__ bx,
                                                                    uint64_t bx_mstride) {
  extern __shared__ dfs sLf[];             // [NB][DG]: L of the diagonal block (strict lower part)
  const uint32_t b = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double* A = a + b * a_mstride + (uint64_t)k0 * lda + k0;
  load_lower_df<INV_COLS * 32>(A, lda, (int)kb, 0, sLf, true);
  __syncthreads();
  const int c = blockIdx.x * INV_COLS + warp;
  double* B = bx + b * bx_mstride;
  if (c >= NB) return;
  if (c >= (int)kb) {                       // padding column: zero
    for (int n = lane; n < NB; n += 32) B[n * NB + c] = 0.0;
    return;
  }
  // x_i for i = lane + 32 t, t = 0..3
  df x[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) x[t] = lane + 32 * t == c ? df{1.0f, 0.0f} : df{0.0f, 0.0f};
  // Step m: x_i -= L_im x_m for i > m.  Only x_{m+1} gates the next step, so
  // it is updated first and broadcast at once, and the other rows' updates
  // (rows i > m + 1 only) fill the shuffle's latency; rows i <= m are
  // final.  The same operations as plain row order, so the same bits.
  df xm{1.0f, 0.0f};                        // x_c
  const int last = (int)kb - 1;
  auto step = [&](auto tcv, int m) {
    constexpr int tc = decltype(tcv)::value;       // x_{m+1} is x[tc] of lane (m + 1) mod 32
    const int ic = lane + 32 * tc;
    if (ic > m && ic < (int)kb) x[tc] = df_fnms(x[tc], ld_df(sLf[ic * DG + m]), xm);
    const int l1 = (m + 1) & 31;
    const df xn{__shfl_sync(0xffffffffu, x[tc].hi, l1), __shfl_sync(0xffffffffu, x[tc].lo, l1)};
#pragma unroll
    for (int t = tc + 1; t < 4; ++t) {
      const int i = lane + 32 * t;
      if (i < (int)kb) x[t] = df_fnms(x[t], ld_df(sLf[i * DG + m]), xm);
    }
    xm = xn;
  };
  // the segments of m in which x_{m+1} sits in x[0], x[1], x[2], x[3]
  for (int m = c; m < min(last, 31); ++m) step(std::integral_constant<int, 0>{}, m);
  for (int m = max(c, 31); m < min(last, 63); ++m) step(std::integral_constant<int, 1>{}, m);
  for (int m = max(c, 63); m < min(last, 95); ++m) step(std::integral_constant<int, 2>{}, m);
  for (int m = max(c, 95); m < last; ++m) step(std::integral_constant<int, 3>{}, m);
  // B[n][c] = x_n / d_n (x_n = 0 above the diagonal, n < c)
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int n = lane + 32 * t;
    double v = 0.0;
    if (n < (int)kb && n >= c) v = f64_of_scaled(x[t], 0) / d[b * d_mstride + k0 + n];
    B[n * NB + c] = v;
  }
}

// ---------------------------------------------------------------------------
// Equilibration by powers of two (exact): the products above are accurate to
// ~2^-55 of their operand rows' largest entries, so a matrix whose diagonal
// spans many orders of magnitude is factored as S A S with S = diag(2^-e_i),
// e_i = floor(log2(a_ii) / 2), and its factors scaled back:
// L_ij = L'_ij 2^(e_i - e_j), D_i = D'_i 2^(2 e_i).  A matrix whose e_i are
// all equal (a stationary covariance: every a_ii = sigma^2) is left alone.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) equil_exps_kernel(const double* __restrict__ a, uint64_t lda,
                                                         uint64_t a_mstride, uint64_t n,
                                                         int32_t* __restrict__ e,
                                                         uint64_t e_mstride, int* nonuniform) {
  const uint32_t b = blockIdx.y;
  const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double* A = a + b * a_mstride;
  auto half_exp = [](double v) {
    const int eb = biased_exp(v);
    return eb == 0 ? 0 : (eb - 1023) >> 1;   // floor((eb - 1023) / 2)
  };
  const int ei = half_exp(A[i * lda + i]);
  e[b * e_mstride + i] = ei;
  if (ei != half_exp(A[0])) atomicOr(&nonuniform[b], 1);
}

// dir > 0: a_ij <- a_ij 2^(-e_i - e_j) on the lower triangle; dir < 0: the
// factor back, L_ij <- L_ij 2^(e_i - e_j) (j < i), D_i <- D_i 2^(2 e_i) on
// the diagonal and in d.  No-op for a matrix whose exponents are uniform.
__global__ void __launch_bounds__(256) equil_apply_kernel(double* __restrict__ a, uint64_t lda,
                                                          uint64_t a_mstride, uint64_t n,
                                                          const int32_t* __restrict__ e,
                                                          uint64_t e_mstride,
                                                          const int* __restrict__ nonuniform,
                                                          double* __restrict__ d, int dir) {
  const uint32_t b = blockIdx.y;
  if (!nonuniform[b]) return;
  const int32_t* eb = e + b * e_mstride;
  double* A = a + b * a_mstride;
  const uint64_t total = n * (n + 1) / 2;
  const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += step) {
    // t -> (i, j), j <= i, row-major over the lower triangle
    uint64_t i = (uint64_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (i * (i + 1) / 2 > t) --i;
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    const uint64_t j = t - i * (i + 1) / 2;
    double& v = A[i * lda + j];
    if (dir > 0) {
      v = scalbn(v, -eb[i] - eb[j]);
    } else if (j < i) {
      v = scalbn(v, eb[i] - eb[j]);
    } else {
      v = scalbn(v, 2 * eb[i]);
      d[b * n + i] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Step 4: U = L D^(1/2) Z for nsim columns of standard normals per matrix.
// z and u are [batch][nsim][n] (one simulation contiguous); y = D^(1/2) z is
// formed first, then one warp per row i accumulates sum_{j <= i} L_ij y_j
// for every simulation (L_ii = 1) in fp64, four partial sums per lane and
// simulation.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) scale_sqrt_d_kernel(const double* __restrict__ d,
                                                           uint64_t d_mstride,
                                                           const double* __restrict__ z,
                                                           double* __restrict__ y, uint64_t n,
                                                           uint32_t nsim, uint32_t batch) {
  const uint64_t per = (uint64_t)nsim * n;
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * batch) return;
  const uint32_t b = (uint32_t)(t / per);
  const uint64_t j = (t - (uint64_t)b * per) % n;
  y[t] = sqrt(d[b * d_mstride + j]) * z[t];
}

// SP simulations per pass of a row; four independent accumulators per
// simulation and lane, so that four loads of the row (and their y) are in
// flight and four FMA chains interleave (the FP64 pipe, 1.6 DFMA per cycle
// per SM, allows ~0.25 ms for four 5580 x 5580 factors and two simulations;
// one chain per lane left the kernel waiting on its loads at 1.1 ms).
template <int SP>
__global__ void __launch_bounds__(256) lower_times_y_kernel(const double* __restrict__ l,
                                                            uint64_t ldl, uint64_t l_mstride,
                                                            const double* __restrict__ y,
                                                            double* __restrict__ u, uint64_t n,
                                                            uint32_t nsim, uint32_t batch) {
  constexpr int U = 4;
  const uint64_t row = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const uint32_t b = blockIdx.y;
  if (row >= n) return;
  const double* lr = l + b * l_mstride + row * ldl;
  const double* yb = y + (uint64_t)b * nsim * n;
  double* ub = u + (uint64_t)b * nsim * n;
  const uint64_t len = row + 1;                 // L_row,row = 1 (unit diagonal)
  for (uint32_t s0 = 0; s0 < nsim; s0 += SP) {
    double acc[SP][U];
#pragma unroll
    for (int s = 0; s < SP; ++s)
#pragma unroll
      for (int k = 0; k < U; ++k) acc[s][k] = 0.0;
    uint64_t j0 = 0;
    for (; j0 + 32 * U <= len; j0 += 32 * U) {
      double lv[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const uint64_t j = j0 + 32 * k + lane;
        lv[k] = j == row ? 1.0 : lr[j];
      }
#pragma unroll
      for (int s = 0; s < SP; ++s)
        if (s0 + s < nsim) {
          const double* ys = yb + (uint64_t)(s0 + s) * n + j0 + lane;
#pragma unroll
          for (int k = 0; k < U; ++k) acc[s][k] = fma(lv[k], ys[32 * k], acc[s][k]);
        }
    }
    for (uint64_t j = j0 + lane; j < len; j += 32) {
      const double lij = j == row ? 1.0 : lr[j];
#pragma unroll
      for (int s = 0; s < SP; ++s)
        if (s0 + s < nsim) acc[s][0] = fma(lij, yb[(uint64_t)(s0 + s) * n + j], acc[s][0]);
    }
#pragma unroll
    for (int s = 0; s < SP; ++s) {
      double v = (acc[s][0] + acc[s][1]) + (acc[s][2] + acc[s][3]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0 && s0 + s < nsim) ub[(uint64_t)(s0 + s) * n + row] = v;
    }
  }
}

}  // namespace grf
}  // namespace mrg
