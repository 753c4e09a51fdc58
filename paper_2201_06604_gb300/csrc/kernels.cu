// kernels.cu -- CUDA kernels of the MRG32k3a hot path for GB300 (sm_103a).
//
//   create_kernel    stream i = A^(i 2^127) seed, one thread per stream
//                    (Sec. 2.1: equal to creating the streams one after another)
//   jump_kernel      x <- A^k x for every stream (skip, substreams, advance)
//   generate_kernel  the recurrence in registers + transform + 32-byte stores
//   fused_kernel     no-store consumer: quarter-circle count and normal sum
//   transform_kernel the transforms of caller-provided raw draws (normals
//                    and exponentials into an output aligned to four
//                    outputs: transform_x2_kernel, four draws per thread)
//   fill_kernel      write-only stream (the write ceiling generate is held to)
//   matrix_kernel    the paper's work-item matrix layout (matrix_kernels.cuh)
//   fisher_kernel    Monte Carlo Fisher's exact test (fisher_kernels.cuh)
//   batch / serve    batched and served requests (batch_kernels.cuh,
//                    serve_kernels.cuh); MRG31k3p kernels in gen31_kernels.cuh
//
// Work decomposition of generate: every stream's n outputs are cut into
// segments of L draws; a lane owns one (stream, segment) pair, jumps to the
// segment's absolute offset with the constant-memory tables A^(2^i), then runs
// the recurrence in registers.  Segment q of the flattened index runs stream
// q mod ns at segment q div ns, so the 32 lanes of a warp share the segment
// offset whenever ns >= 32 and the jump's table reads are warp-uniform.
// Normals and exponentials are transformed two draws (two Box-Muller pairs)
// at a time with packed fp32x2 instructions (transforms_x2.cuh; for fp32
// normals only the radius) when a unit holds enough outputs (16- or 32-byte
// stores), else one at a time; the results are bit-identical.
// Each lane's outputs are contiguous in its row, so a lane stores whole
// 32-byte sectors with one 256-bit st.global per 32 bytes: the L2 receives
// full-sector writes and nothing is staged in shared memory.  (Staged
// variants -- per-lane shared-memory rows drained by cp.async.bulk, or lane
// quads transposed through shared memory to store 128 contiguous bytes per
// row -- were measured slower: the first capped occupancy at 3 blocks per
// SM, the second added address arithmetic to the IMAD pipe that bounds the
// recurrence.)
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "host_jump.h"
#include "internal.h"
#include "mrg32k3a_core.cuh"
#include "transforms_df.cuh"
#include "transforms_x2.cuh"

#define MRG_RAW 0
#define MRG_UNIFORM 1
#define MRG_NORMAL 2
#define MRG_EXPONENTIAL 3
#define MRG_U32 0
#define MRG_F32 1
#define MRG_F64 2

namespace mrg {

std::atomic<uint64_t> g_launches{0};

__constant__ uint32_t c_jump[2][JUMP_BITS][9];
__device__ float4 g_ttab[TAB_ENTRIES];

cudaError_t upload_tables(const uint32_t* tab, size_t bytes) {
  if (bytes != sizeof(c_jump)) return cudaErrorInvalidValue;
  return cudaMemcpyToSymbol(c_jump, tab, bytes);
}

static_assert(TAB_ENTRIES == host::kTransformEntries && TRIG_COPIES == host::kTransformTrigCopies,
              "transform table layout of the host builder and the kernels");

cudaError_t upload_transform_table(const float* tab, size_t bytes) {
  if (bytes != sizeof(g_ttab)) return cudaErrorInvalidValue;
  return cudaMemcpyToSymbol(g_ttab, tab, bytes);
}

// Copies the transform tables into shared memory (all threads of the block
// must call it).
__device__ __forceinline__ void load_ttab(float4* s_tab) {
  for (int i = threadIdx.x; i < TAB_ENTRIES; i += blockDim.x) s_tab[i] = g_ttab[i];
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Jump helpers
// ---------------------------------------------------------------------------

template <int COMP>
__device__ __forceinline__ void apply_pow2(int i, uint32_t& x0, uint32_t& x1, uint32_t& x2) {
  uint32_t A[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) A[k] = c_jump[COMP][i][k];
  matvec<COMP>(A, x0, x1, x2);
}

__device__ __forceinline__ void apply_pow2_both(int i, State& s) {
  apply_pow2<0>(i, s.a0, s.a1, s.a2);
  apply_pow2<1>(i, s.b0, s.b1, s.b2);
}

// s <- A^(e 2^base) s with a per-lane exponent e.  The loop runs over the
// bits set in any lane, so the table index is warp-uniform (constant-cache
// broadcast).  All 32 lanes of the warp must call it.
__device__ __forceinline__ void jump_lanes(State& s, uint64_t e, int base) {
  unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)e);
  unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(e >> 32));
  uint64_t any = ((uint64_t)hi << 32) | lo;
  while (any) {
    int i = __ffsll((long long)any) - 1;
    any &= any - 1;
    if ((e >> i) & 1) apply_pow2_both(base + i, s);
  }
}

__device__ __forceinline__ State load_state(const uint32_t* p, uint64_t stride, uint64_t i) {
  State s;
  s.a0 = p[i]; s.a1 = p[stride + i]; s.a2 = p[2 * stride + i];
  s.b0 = p[3 * stride + i]; s.b1 = p[4 * stride + i]; s.b2 = p[5 * stride + i];
  return s;
}

__device__ __forceinline__ void store_state(uint32_t* p, uint64_t stride, uint64_t i, const State& s) {
  p[i] = s.a0; p[stride + i] = s.a1; p[2 * stride + i] = s.a2;
  p[3 * stride + i] = s.b0; p[4 * stride + i] = s.b1; p[5 * stride + i] = s.b2;
}

// ---------------------------------------------------------------------------
// Stream creation
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) create_kernel(State seed, uint64_t n, uint32_t* cur,
                                                     uint32_t* start, uint32_t* sub,
                                                     uint64_t stride) {
  const uint64_t step_all = (uint64_t)gridDim.x * blockDim.x;
  // The trip count is uniform per block, so every lane reaches jump_lanes.
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < n; base += step_all) {
    const uint64_t i = base + threadIdx.x;
    const bool valid = i < n;
    State s = seed;
    jump_lanes(s, valid ? i : 0, STREAM_LOG2);
    if (valid) {
      store_state(cur, stride, i, s);
      store_state(start, stride, i, s);
      store_state(sub, stride, i, s);
    }
  }
}

// ---------------------------------------------------------------------------
// Uniform jump of every stream (skip / substream / advance / reset)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) jump_kernel(const uint32_t* src, uint32_t* dst0,
                                                   uint32_t* dst1, uint64_t stride, uint64_t ns,
                                                   uint64_t e_lo, uint64_t e_hi, int base) {
  const uint64_t step_all = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += step_all) {
    State s = load_state(src, stride, i);
    for (uint64_t e = e_lo; e; e &= e - 1) apply_pow2_both(base + __ffsll((long long)e) - 1, s);
    for (uint64_t e = e_hi; e; e &= e - 1) apply_pow2_both(base + 64 + __ffsll((long long)e) - 1, s);
    store_state(dst0, stride, i, s);
    if (dst1) store_state(dst1, stride, i, s);
  }
}

// ---------------------------------------------------------------------------
// Vector stores: each lane writes whole 32-byte sectors of its own row, so
// the L2 receives full-sector writes without any staging in shared memory.
// ---------------------------------------------------------------------------

template <int VB>
__device__ __forceinline__ void store_vec(char* p, const uint32_t* w) {
  if constexpr (VB == 32) {
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
                 :: "l"(p), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]),
                    "r"(w[6]), "r"(w[7]) : "memory");
  } else if constexpr (VB == 16) {
    asm volatile("st.global.v4.b32 [%0], {%1, %2, %3, %4};"
                 :: "l"(p), "r"(w[0]), "r"(w[1]), "r"(w[2]), "r"(w[3]) : "memory");
  } else if constexpr (VB == 8) {
    asm volatile("st.global.v2.b32 [%0], {%1, %2};" :: "l"(p), "r"(w[0]), "r"(w[1]) : "memory");
  } else {
    asm volatile("st.global.b32 [%0], %1;" :: "l"(p), "r"(w[0]) : "memory");
  }
}

// ---------------------------------------------------------------------------
// Output units: UE consecutive outputs of one stream as 32-bit words
// ---------------------------------------------------------------------------

struct Consts {
  uint64_t k1, k2;   // the offset-form addends K1, K2 (kept in registers)
  float ir_hi, ir_lo;  // -1/rate as a float pair (exponentials)
};

__device__ __forceinline__ void put_f64(uint32_t* w, uint64_t b) {
  w[0] = (uint32_t)b;
  w[1] = (uint32_t)(b >> 32);
}

template <int DIST, int DT, int UE>
__device__ __forceinline__ void produce(TState& s, uint32_t* w, const Consts& c,
                                       const float4* __restrict__ tab) {
  // the step's negations as subtractions where that measured faster: all
  // but the fp32 normals (fp64 exponentials 3.65 -> 3.59 ms; the fused
  // consumer, 13.85 -> 13.89, keeps the multiply-add form too)
  constexpr bool AN = !(DIST == MRG_NORMAL && DT == MRG_F32);
  if constexpr (DIST == MRG_RAW) {
#pragma unroll
    for (int e = 0; e < UE; ++e) w[e] = step_fast<AN>(s, c.k1, c.k2);
  } else if constexpr (DIST == MRG_UNIFORM && DT == MRG_F64) {
#pragma unroll
    for (int e = 0; e < UE; ++e) put_f64(w + 2 * e, uniform_bits64_fast(step_fast<AN>(s, c.k1, c.k2)));
  } else if constexpr (DIST == MRG_UNIFORM) {
#pragma unroll
    for (int e = 0; e < UE; ++e)
      w[e] = uniform_bits32(step_fast<AN>(s, c.k1, c.k2));
  } else if constexpr (DIST == MRG_NORMAL && DT == MRG_F64 && UE % 4 == 0) {
    // two pairs per packed fp32x2 evaluation (bit-identical to the scalar one)
#pragma unroll
    for (int p = 0; p < UE / 4; ++p) {
      const uint32_t z1a = step_fast<AN>(s, c.k1, c.k2);
      const uint32_t z2a = step_fast<AN>(s, c.k1, c.k2);
      const uint32_t z1b = step_fast<AN>(s, c.k1, c.k2);
      const uint32_t z2b = step_fast<AN>(s, c.k1, c.k2);
      uint64_t xa, ya, xb, yb;
      box_muller_f64_x2<UM32k3a>(z1a, z2a, z1b, z2b, tab, xa, ya, xb, yb);
      put_f64(w + 8 * p, xa);
      put_f64(w + 8 * p + 2, ya);
      put_f64(w + 8 * p + 4, xb);
      put_f64(w + 8 * p + 6, yb);
    }
  } else if constexpr (DIST == MRG_NORMAL && DT == MRG_F32 && UE % 4 == 0) {
#pragma unroll
    for (int p = 0; p < UE / 4; ++p) {
      const uint32_t z1a = step_fast<AN>(s, c.k1, c.k2);
      const uint32_t z2a = step_fast<AN>(s, c.k1, c.k2);
      const uint32_t z1b = step_fast<AN>(s, c.k1, c.k2);
      const uint32_t z2b = step_fast<AN>(s, c.k1, c.k2);
      float xa, ya, xb, yb;
      box_muller_f32_x2<UM32k3a>(z1a, z2a, z1b, z2b, tab, xa, ya, xb, yb);
      w[4 * p] = __float_as_uint(xa);
      w[4 * p + 1] = __float_as_uint(ya);
      w[4 * p + 2] = __float_as_uint(xb);
      w[4 * p + 3] = __float_as_uint(yb);
    }
  } else if constexpr (DIST == MRG_NORMAL) {
#pragma unroll
    for (int p = 0; p < UE / 2; ++p) {
      const uint32_t z1 = step_fast<AN>(s, c.k1, c.k2);
      const uint32_t z2 = step_fast<AN>(s, c.k1, c.k2);
      if constexpr (DT == MRG_F64) {
        uint64_t x, y;
        box_muller_f64(z1, z2, tab, x, y);
        put_f64(w + 4 * p, x);
        put_f64(w + 4 * p + 2, y);
      } else {
        float x, y;
        box_muller_f32(z1, z2, tab, x, y);
        w[2 * p] = __float_as_uint(x);
        w[2 * p + 1] = __float_as_uint(y);
      }
    }
  } else if constexpr (DT == MRG_F32 && UE % 2 == 0) {   // exponential, two draws per packed evaluation
#pragma unroll
    for (int e = 0; e < UE; e += 2) {
      const uint32_t za = step_fast<AN>(s, c.k1, c.k2);
      const uint32_t zb = step_fast<AN>(s, c.k1, c.k2);
      float ea, eb;
      exp_f32_x2<UM32k3a>(za, zb, tab, c.ir_hi, c.ir_lo, ea, eb);
      w[e] = __float_as_uint(ea);
      w[e + 1] = __float_as_uint(eb);
    }
  } else if constexpr (DT == MRG_F64 && UE % 2 == 0) {   // the same for fp64 (3.80 -> 3.66 ms per 2^30)
#pragma unroll
    for (int e = 0; e < UE; e += 2) {
      const uint32_t za = step_fast<AN>(s, c.k1, c.k2);
      const uint32_t zb = step_fast<AN>(s, c.k1, c.k2);
      uint64_t ea, eb;
      exp_f64_x2<UM32k3a>(za, zb, tab, c.ir_hi, c.ir_lo, ea, eb);
      put_f64(w + 2 * e, ea);
      put_f64(w + 2 * e + 2, eb);
    }
  } else {  // exponential: -ln(u) / rate
#pragma unroll
    for (int e = 0; e < UE; ++e) {
      const uint32_t z = step_fast<AN>(s, c.k1, c.k2);
      if constexpr (DT == MRG_F64)
        put_f64(w + 2 * e, df_to_f64_bits(df_mul(ln_u_df(z, tab), df{c.ir_hi, c.ir_lo})));
      else
        w[e] = __float_as_uint(exp_f32(z, tab, c.ir_hi, c.ir_lo));
    }
  }
}

// ---------------------------------------------------------------------------
// Materialised generation
// ---------------------------------------------------------------------------

struct GenArgs {
  const uint32_t* cur;
  uint64_t stride, ns;
  uint64_t n;      // outputs per stream
  uint64_t L;      // segment length in outputs (= draws), multiple of 8
  uint64_t total;  // ns * ceil(n / L) segments
  char* out;
  uint64_t ld;     // elements
  Consts c;
};

// VB: bytes per vector store (32, 16, 8 or 4), the largest width that the
// output pointer and row pitch allow.
template <int DIST, int DT, int VB>
__global__ void __launch_bounds__(256) generate_kernel(GenArgs a) {
  constexpr int ES = DT == MRG_F64 ? 8 : 4;
  constexpr int UB = (DIST == MRG_NORMAL && VB < 2 * ES) ? 2 * ES : (VB < ES ? ES : VB);
  constexpr int UE = UB / ES;          // outputs per unit
  constexpr int UW = UB / 4;           // 32-bit words per unit
  constexpr int VS = VB < ES ? ES : VB;  // store width actually used
  constexpr int VW = VS / 4;

  constexpr bool TABLES = DIST == MRG_NORMAL || DIST == MRG_EXPONENTIAL;
  __shared__ float4 s_tab[TABLES ? TAB_ENTRIES : 1];
  if constexpr (TABLES) load_ttab(s_tab);

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  const uint64_t ntiles = (a.total + 31) >> 5;
  const Consts c = a.c;

  for (uint64_t w = (uint64_t)blockIdx.x * wpb + warp; w < ntiles;
       w += (uint64_t)gridDim.x * wpb) {
    const uint64_t q = (w << 5) + lane;
    const bool valid = q < a.total;
    uint64_t s = 0, g = 0;
    if (valid) {
      g = q / a.ns;
      s = q - g * a.ns;
    }
    const uint64_t off = g * a.L;
    const uint32_t cnt = valid ? (uint32_t)min(a.L, a.n - off) : 0u;
    State st0 = valid ? load_state(a.cur, a.stride, s) : State{1, 1, 1, 1, 1, 1};
    jump_lanes(st0, off, 0);
    TState st = to_offset(st0);
    const uint32_t cmax = __reduce_max_sync(0xffffffffu, cnt);
    char* gdst = a.out + (s * a.ld + off) * ES;
    uint32_t i0 = 0;
    if constexpr (DIST == MRG_RAW || DIST == MRG_UNIFORM) {
      // Units that every lane of the warp stores whole: no bound checks, a
      // pointer step (saves about one instruction per output).  Not for the
      // transforms, whose larger bodies would then exist twice in the code.
      const uint32_t nfull = __reduce_min_sync(0xffffffffu, cnt) / UE * UE;
      char* p = gdst;
#pragma unroll 2
      for (; i0 < nfull; i0 += UE) {
        uint32_t wv[UW];
        produce<DIST, DT, UE>(st, wv, c, s_tab);
#pragma unroll
        for (int v = 0; v < UB / VS; ++v) store_vec<VS>(p + v * VS, wv + v * VW);
        p += UB;
      }
    }

    // the transforms' bodies are long enough on their own: unrolled once they
    // keep fewer registers and more warps per SM (measured 3-5 % faster for
    // fp32 normals and both exponentials)
    constexpr int UNROLL = TABLES ? 1 : 2;
#pragma unroll UNROLL
    for (uint32_t i = i0; i < cmax; i += UE) {
      uint32_t wv[UW];
      produce<DIST, DT, UE>(st, wv, c, s_tab);
      if (i + UE <= cnt) {
#pragma unroll
        for (int v = 0; v < UB / VS; ++v) store_vec<VS>(gdst + (size_t)i * ES + v * VS, wv + v * VW);
      } else if (i < cnt) {
#pragma unroll
        for (int e = 0; e < UE; ++e)
          if (i + e < cnt) store_vec<ES>(gdst + (size_t)(i + e) * ES, wv + e * (ES / 4));
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Write-only stream (calibration of the HBM write bandwidth the generate
// kernels are held against): one warp per 128 KiB chunk, filled front to
// back at 1 KiB per store instruction, the grid covering the whole buffer
// (warps in launch order, so the chunks being written at any moment are
// neighbours) -- the fastest write-only pattern measured on GB300 (~7.5
// TB/s, against ~6.5 for a persistent grid-stride loop over 1 KiB units and
// ~4.2 for one 32-byte unit per lane and row per instruction, the generate
// kernels' own pattern).
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) fill_kernel(char* out, uint64_t units, uint64_t chunk,
                                                   uint32_t v) {
  const uint32_t w[8] = {v, v, v, v, v, v, v, v};
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t b = warp * chunk;
  const uint64_t e = min(units, b + chunk);
  for (uint64_t i = b + (threadIdx.x & 31); i < e; i += 32) store_vec<32>(out + 32 * i, w);
}

// ---------------------------------------------------------------------------
// Fused no-store consumer
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) fused_kernel(uint32_t* cur, uint64_t stride, uint64_t ns,
                                                    uint64_t pairs, int64_t* count, double* sum,
                                                    uint64_t k1, uint64_t k2) {
  __shared__ float4 s_tab[TAB_ENTRIES];
  load_ttab(s_tab);
  constexpr uint64_t MSQ = MNORM * MNORM;  // (m1+1)^2 < 2^64
  const uint64_t step_all = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += step_all) {
    TState s = to_offset(load_state(cur, stride, i));
    int64_t cnt = 0;
    // sum as H + L: each pair's X + Y enters H error-free (two_sum), its
    // rounding error and low part go to L, and H + L is renormalised every
    // 32 pairs, so |L| stays below ~2^-15 and its own roundings add up to
    // ~2^-27 over 2048 pairs -- far inside the sum's tolerance, 1e-9 of the
    // sum of |X| and |Y| (~3e-6 at 4096 draws)
    float H = 0.0f, L = 0.0f;
    // two pairs per trip (their logs and radii in one packed evaluation),
    // added to the sum in order; an odd last pair alone
    auto in_circle = [](uint32_t za, uint32_t zb) -> int64_t {
      const uint64_t sa = (uint64_t)za * za, sb = (uint64_t)zb * zb;
      const uint64_t ss = sa + sb;
      return (ss >= sa) & (ss < MSQ);  // no carry out of 64 bits and below M^2
    };
    auto add = [&H, &L](df v) {
      const df h = two_sum(H, v.hi);
      H = h.hi;
      L = __fadd_rn(L, __fadd_rn(h.lo, v.lo));
    };
    for (uint64_t k0 = 0; k0 < pairs; k0 += 32) {
      const uint64_t k1e = min(pairs, k0 + 32);
      uint64_t k = k0;
      for (; k + 2 <= k1e; k += 2) {
        const uint32_t za = step_fast(s, k1, k2);
        const uint32_t zb = step_fast(s, k1, k2);
        const uint32_t zc = step_fast(s, k1, k2);
        const uint32_t zd = step_fast(s, k1, k2);
        cnt += in_circle(za, zb) + in_circle(zc, zd);
        df v0, v1;
        box_muller_sum_lite_x2<UM32k3a>(za, zb, zc, zd, s_tab, v0, v1);
        add(v0);
        add(v1);
      }
      if (k < k1e) {
        const uint32_t za = step_fast(s, k1, k2);
        const uint32_t zb = step_fast(s, k1, k2);
        cnt += in_circle(za, zb);
        add(box_muller_sum_lite_m<UM32k3a>(za, zb, s_tab));
      }
      const df r = two_sum(H, L);
      H = r.hi;
      L = r.lo;
    }
    store_state(cur, stride, i, from_offset(s));
    count[i] = cnt;
    sum[i] = __longlong_as_double((long long)df_to_f64_bits(df{H, L}));
  }
}

// ---------------------------------------------------------------------------
// Transform of caller-provided raw draws
// ---------------------------------------------------------------------------

template <int DIST, int DT>
__global__ void __launch_bounds__(256) transform_kernel(const uint32_t* __restrict__ z, uint64_t n,
                                                        char* out, Consts c) {
  __shared__ float4 s_tab[TAB_ENTRIES];
  load_ttab(s_tab);
  constexpr int ES = DT == MRG_F64 ? 8 : 4;
  constexpr int PER = DIST == MRG_NORMAL ? 2 : 1;
  const uint64_t units = (n + PER - 1) / PER;
  const uint64_t step_all = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += step_all) {
    uint32_t w[4];
    if constexpr (DIST == MRG_NORMAL) {
      const uint32_t z1 = z[2 * u];
      const uint32_t z2 = 2 * u + 1 < n ? z[2 * u + 1] : 1u;
      if constexpr (DT == MRG_F64) {
        uint64_t x, y;
        box_muller_f64(z1, z2, s_tab, x, y);
        put_f64(w, x);
        put_f64(w + 2, y);
      } else {
        float x, y;
        box_muller_f32(z1, z2, s_tab, x, y);
        w[0] = __float_as_uint(x);
        w[1] = __float_as_uint(y);
      }
    } else if constexpr (DIST == MRG_EXPONENTIAL) {
      if constexpr (DT == MRG_F64)
        put_f64(w, df_to_f64_bits(df_mul(ln_u_df(z[u], s_tab), df{c.ir_hi, c.ir_lo})));
      else
        w[0] = __float_as_uint(exp_f32(z[u], s_tab, c.ir_hi, c.ir_lo));
    } else if constexpr (DT == MRG_F64) {
      put_f64(w, uniform_bits64_fast(z[u]));
    } else {
      w[0] = uniform_bits32(z[u]);
    }
    for (int e = 0; e < PER; ++e) {
      const uint64_t i = u * PER + e;
      if (i < n) {
        uint32_t* d = reinterpret_cast<uint32_t*>(out + i * ES);
        d[0] = w[e * ES / 4];
        if (ES == 8) d[1] = w[e * ES / 4 + 1];
      }
    }
  }
}

// Normals and exponentials into an output aligned to four outputs
// (32 bytes for fp64, 16 for fp32): each thread transforms four draws with
// the packed two-at-a-time evaluation and stores them in one vector; a last
// unit of fewer than four draws takes the scalar one (bit-identical results
// either way; the launcher picks this kernel by the output's alignment, so
// both evaluations are reachable through the same entry point).
template <int DIST, int DT>
__global__ void __launch_bounds__(256) transform_x2_kernel(const uint32_t* __restrict__ z, uint64_t n,
                                                           char* out, Consts c) {
  static_assert(DIST == MRG_NORMAL || DIST == MRG_EXPONENTIAL, "packed forms");
  __shared__ float4 s_tab[TAB_ENTRIES];
  load_ttab(s_tab);
  constexpr int ES = DT == MRG_F64 ? 8 : 4;
  const uint64_t units = (n + 3) / 4;
  const uint64_t step_all = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < units; u += step_all) {
    const uint64_t i0 = 4 * u;
    char* d = out + i0 * ES;
    if (i0 + 4 <= n) {
      uint32_t w[4 * ES / 4];
      if constexpr (DIST == MRG_NORMAL && DT == MRG_F64) {
        uint64_t xa, ya, xb, yb;
        box_muller_f64_x2<UM32k3a>(z[i0], z[i0 + 1], z[i0 + 2], z[i0 + 3], s_tab, xa, ya, xb, yb);
        put_f64(w, xa);
        put_f64(w + 2, ya);
        put_f64(w + 4, xb);
        put_f64(w + 6, yb);
      } else if constexpr (DIST == MRG_NORMAL) {
        float xa, ya, xb, yb;
        box_muller_f32_x2<UM32k3a>(z[i0], z[i0 + 1], z[i0 + 2], z[i0 + 3], s_tab, xa, ya, xb, yb);
        w[0] = __float_as_uint(xa);
        w[1] = __float_as_uint(ya);
        w[2] = __float_as_uint(xb);
        w[3] = __float_as_uint(yb);
      } else if constexpr (DT == MRG_F64) {
        uint64_t e0, e1, e2, e3;
        exp_f64_x2<UM32k3a>(z[i0], z[i0 + 1], s_tab, c.ir_hi, c.ir_lo, e0, e1);
        exp_f64_x2<UM32k3a>(z[i0 + 2], z[i0 + 3], s_tab, c.ir_hi, c.ir_lo, e2, e3);
        put_f64(w, e0);
        put_f64(w + 2, e1);
        put_f64(w + 4, e2);
        put_f64(w + 6, e3);
      } else {
        float e0, e1, e2, e3;
        exp_f32_x2<UM32k3a>(z[i0], z[i0 + 1], s_tab, c.ir_hi, c.ir_lo, e0, e1);
        exp_f32_x2<UM32k3a>(z[i0 + 2], z[i0 + 3], s_tab, c.ir_hi, c.ir_lo, e2, e3);
        w[0] = __float_as_uint(e0);
        w[1] = __float_as_uint(e1);
        w[2] = __float_as_uint(e2);
        w[3] = __float_as_uint(e3);
      }
      store_vec<4 * ES>(d, w);
    } else if constexpr (DIST == MRG_NORMAL) {
      for (uint64_t i = i0; i < n; i += 2) {
        const uint32_t z2 = i + 1 < n ? z[i + 1] : 1u;
        uint32_t w[4];
        if constexpr (DT == MRG_F64) {
          uint64_t x, y;
          box_muller_f64(z[i], z2, s_tab, x, y);
          put_f64(w, x);
          put_f64(w + 2, y);
        } else {
          float x, y;
          box_muller_f32(z[i], z2, s_tab, x, y);
          w[0] = __float_as_uint(x);
          w[1] = __float_as_uint(y);
        }
        store_vec<ES>(out + i * ES, w);
        if (i + 1 < n) store_vec<ES>(out + (i + 1) * ES, w + ES / 4);
      }
    } else if constexpr (DT == MRG_F64) {
      for (uint64_t i = i0; i < n; ++i)
        reinterpret_cast<uint64_t*>(out)[i] =
            df_to_f64_bits(df_mul(ln_u_df(z[i], s_tab), df{c.ir_hi, c.ir_lo}));
    } else {
      for (uint64_t i = i0; i < n; ++i)
        reinterpret_cast<float*>(out)[i] = exp_f32(z[i], s_tab, c.ir_hi, c.ir_lo);
    }
  }
}

}  // namespace mrg

#include "batch_kernels.cuh"
#include "serve_kernels.cuh"
#include "gen31_kernels.cuh"
#include "fisher_kernels.cuh"
#include "matrix_kernels.cuh"

namespace mrg {

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

namespace {

struct DevInfo {
  int sms = 0;
};

DevInfo& dev_info() {
  static std::mutex mu;
  static DevInfo info[64];
  int d = 0;
  cudaGetDevice(&d);
  std::lock_guard<std::mutex> lk(mu);
  DevInfo& di = info[d & 63];
  if (di.sms == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
    di.sms = v > 0 ? v : 1;
  }
  return di;
}

inline cudaError_t after_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

inline unsigned grid_for(uint64_t items, int block, int per_sm) {
  uint64_t need = (items + block - 1) / block;
  uint64_t cap = (uint64_t)sm_count() * per_sm;
  return (unsigned)std::max<uint64_t>(1, std::min(need, cap));
}

}  // namespace

int sm_count() { return dev_info().sms; }

cudaError_t launch_create(const uint32_t seed[6], uint64_t n, const DevStreams& s,
                          cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  State sd{seed[0], seed[1], seed[2], seed[3], seed[4], seed[5]};
  create_kernel<<<grid_for(n, 256, 8), 256, 0, st>>>(sd, n, s.cur, s.start, s.sub, s.stride);
  return after_launch();
}

cudaError_t launch_jump(const uint32_t* src, uint32_t* dst0, uint32_t* dst1, uint64_t stride,
                        uint64_t ns, uint64_t e_lo, uint64_t e_hi, int base, cudaStream_t st) {
  if (ns == 0) return cudaSuccess;
  jump_kernel<<<grid_for(ns, 256, 8), 256, 0, st>>>(src, dst0, dst1, stride, ns, e_lo, e_hi, base);
  return after_launch();
}

cudaError_t launch_fused(const DevStreams& s, uint64_t pairs, int64_t* count, double* sum,
                         cudaStream_t st) {
  if (s.n == 0) return cudaSuccess;
  fused_kernel<<<grid_for(s.n, 256, 8), 256, 0, st>>>(s.cur, s.stride, s.n, pairs, count, sum,
                                                      K1, K2);
  return after_launch();
}

namespace {

template <int DIST, int DT, int VB, bool G31>
cudaError_t launch_gen_t(const GenArgs& a, const GenConfig& cfg, cudaStream_t st) {
  auto kern = G31 ? generate31_kernel<DIST, DT, VB> : generate_kernel<DIST, DT, VB>;
  const int block = cfg.block;
  static thread_local int occ_cache[64][9] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int& occ = occ_cache[dev & 63][block / 32];
  if (occ == 0) {
    int v = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, block, 0);
    if (e != cudaSuccess) return e;
    occ = v > 0 ? v : 1;
  }
  const uint64_t ntiles = (a.total + 31) / 32;
  const uint64_t wpb = block / 32;
  uint64_t blocks = (ntiles + wpb - 1) / wpb;
  const int per_sm = cfg.per_sm > 0 ? std::min(cfg.per_sm, occ) : occ;
  uint64_t cap = (uint64_t)sm_count() * per_sm;
  if (cfg.max_blocks > 0) cap = std::min<uint64_t>(cap, (uint64_t)cfg.max_blocks);
  blocks = std::max<uint64_t>(1, std::min(blocks, cap));
  kern<<<(unsigned)blocks, block, 0, st>>>(a);
  return after_launch();
}

template <int DIST, int DT, bool G31>
cudaError_t launch_gen_dt(const GenArgs& a, int vb, const GenConfig& cfg, cudaStream_t st) {
  switch (vb) {
    case 32: return launch_gen_t<DIST, DT, 32, G31>(a, cfg, st);
    case 16: return launch_gen_t<DIST, DT, 16, G31>(a, cfg, st);
    case 8: return launch_gen_t<DIST, DT, 8, G31>(a, cfg, st);
    default: return launch_gen_t<DIST, DT, 4, G31>(a, cfg, st);
  }
}

template <bool G31>
cudaError_t launch_generate_g(const DevStreams& s, uint64_t n, int dist, int dtype, double rate,
                              void* out, uint64_t ld, const GenConfig& cfg_in, cudaStream_t st);

}  // namespace

namespace {
template <bool G31>
cudaError_t launch_generate_g(const DevStreams& s, uint64_t n, int dist, int dtype, double rate,
                              void* out, uint64_t ld, const GenConfig& cfg_in, cudaStream_t st) {
  if (s.n == 0 || n == 0) return cudaSuccess;
  GenConfig cfg = cfg_in;
  if (cfg.block <= 0 || cfg.block > 256 || cfg.block % 32) cfg.block = 256;
  const int es = dtype == MRG_F64 ? 8 : 4;
  const uint64_t ce = 8;  // segment lengths are multiples of 8 outputs (32-byte aligned starts)
  uint64_t L = cfg.seg_len;
  if (L == 0) {
    // Heuristic: about 8 segments per resident lane slot, at least 512 draws
    // (jump cost amortised), at most the whole row.  A call too small to give
    // every lane slot 512 draws (a single stream of 10^6 draws, say) takes
    // shorter segments, down to 64 draws, so that it still spreads over the
    // GPU instead of running a few warps through long serial segments.
    const uint64_t lanes = (uint64_t)sm_count() * 2048;
    const uint64_t total = n * s.n;
    L = total / (lanes * 8);
    if (L < 512) L = std::min<uint64_t>(std::max<uint64_t>(total / lanes, 64), 512);
  }
  L = (L + ce - 1) / ce * ce;                 // multiple of 8 (even: pairs stay aligned)
  const uint64_t ncap = (n + ce - 1) / ce * ce;
  L = std::min(L, ncap);
  L = std::min<uint64_t>(L, 1ull << 31);      // a lane's count is a 32-bit word
  GenArgs a;
  a.cur = s.cur;
  a.stride = s.stride;
  a.ns = s.n;
  a.n = n;
  a.L = L;
  a.total = s.n * ((n + L - 1) / L);
  a.out = reinterpret_cast<char*>(out);
  a.ld = ld;
  a.c.k1 = K1;
  a.c.k2 = K2;
  {
    const double ir = -1.0 / rate;
    a.c.ir_hi = (float)ir;
    a.c.ir_lo = (float)(ir - (double)a.c.ir_hi);
  }
  // widest store the row starts allow: out address and row pitch alignment
  const uint64_t align = (reinterpret_cast<uintptr_t>(out) | (ld * es) | 32) & ~((reinterpret_cast<uintptr_t>(out) | (ld * es) | 32) - 1);
  const int vmax = (cfg.vec_bytes == 4 || cfg.vec_bytes == 8 || cfg.vec_bytes == 16) ? cfg.vec_bytes : 32;
  const int vb = (int)std::min<uint64_t>(align, (uint64_t)vmax);
  switch (dist * 4 + dtype) {
    case MRG_RAW * 4 + MRG_U32: return launch_gen_dt<MRG_RAW, MRG_U32, G31>(a, vb, cfg, st);
    case MRG_UNIFORM * 4 + MRG_F32: return launch_gen_dt<MRG_UNIFORM, MRG_F32, G31>(a, vb, cfg, st);
    case MRG_UNIFORM * 4 + MRG_F64: return launch_gen_dt<MRG_UNIFORM, MRG_F64, G31>(a, vb, cfg, st);
    case MRG_NORMAL * 4 + MRG_F32: return launch_gen_dt<MRG_NORMAL, MRG_F32, G31>(a, vb, cfg, st);
    case MRG_NORMAL * 4 + MRG_F64: return launch_gen_dt<MRG_NORMAL, MRG_F64, G31>(a, vb, cfg, st);
    case MRG_EXPONENTIAL * 4 + MRG_F32: return launch_gen_dt<MRG_EXPONENTIAL, MRG_F32, G31>(a, vb, cfg, st);
    case MRG_EXPONENTIAL * 4 + MRG_F64: return launch_gen_dt<MRG_EXPONENTIAL, MRG_F64, G31>(a, vb, cfg, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

cudaError_t launch_generate(const DevStreams& s, uint64_t n, int dist, int dtype, double rate,
                            void* out, uint64_t ld, const GenConfig& cfg, cudaStream_t st) {
  return launch_generate_g<false>(s, n, dist, dtype, rate, out, ld, cfg, st);
}

cudaError_t launch_generate31(const DevStreams& s, uint64_t n, int dist, int dtype, double rate,
                              void* out, uint64_t ld, const GenConfig& cfg, cudaStream_t st) {
  return launch_generate_g<true>(s, n, dist, dtype, rate, out, ld, cfg, st);
}

cudaError_t launch_fisher(const DevStreams& s, const int32_t* rows, const int32_t* cols,
                          uint32_t I, uint32_t J, int32_t total, const double* lf, uint64_t B,
                          double threshold, unsigned long long* count, double* stats,
                          cudaStream_t st) {
  if (s.n == 0) return cudaSuccess;
  FisherArgs a;
  a.cur = s.cur;
  a.stride = s.stride;
  a.ns = s.n;
  a.rows = rows;
  a.cols = cols;
  a.lf = lf;
  a.I = I;
  a.J = J;
  a.B = B;
  a.threshold = threshold;
  a.count = count;
  a.stats = stats;
  a.total = total;
  fisher_kernel<<<grid_for(s.n, 256, 8), 256, 0, st>>>(a, K1, K2);
  return after_launch();
}

namespace {
template <bool G31, int DIST, int DT>
cudaError_t launch_matrix_t(const MatrixArgs& a, cudaStream_t st) {
  const uint64_t items = (uint64_t)a.g0 * a.g1;
  matrix_kernel<G31, DIST, DT><<<(unsigned)((items + 255) / 256), 256, 0, st>>>(a, K1, K2);
  return after_launch();
}
template <bool G31>
cudaError_t launch_matrix_g(const MatrixArgs& a, int dist, int dtype, cudaStream_t st) {
  switch (dist * 4 + dtype) {
    case MRG_RAW * 4 + MRG_U32: return launch_matrix_t<G31, MRG_RAW, MRG_U32>(a, st);
    case MRG_UNIFORM * 4 + MRG_F32: return launch_matrix_t<G31, MRG_UNIFORM, MRG_F32>(a, st);
    case MRG_UNIFORM * 4 + MRG_F64: return launch_matrix_t<G31, MRG_UNIFORM, MRG_F64>(a, st);
    case MRG_EXPONENTIAL * 4 + MRG_F32: return launch_matrix_t<G31, MRG_EXPONENTIAL, MRG_F32>(a, st);
    case MRG_EXPONENTIAL * 4 + MRG_F64: return launch_matrix_t<G31, MRG_EXPONENTIAL, MRG_F64>(a, st);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

cudaError_t launch_matrix(bool g31, uint32_t* cur, uint64_t stride, uint64_t nrow, uint64_t ncol,
                          uint32_t g0, uint32_t g1, int dist, int dtype, double rate, void* out,
                          uint64_t ld, cudaStream_t st) {
  MatrixArgs a;
  a.cur = cur;
  a.stride = stride;
  a.nrow = nrow;
  a.ncol = ncol;
  a.npad = (ncol + g1 - 1) / g1 * g1;
  a.g0 = g0;
  a.g1 = g1;
  a.out = static_cast<char*>(out);
  a.ld = ld;
  const double ir = dist == MRG_EXPONENTIAL ? -1.0 / rate : 0.0;
  a.ir_hi = (float)ir;
  a.ir_lo = (float)(ir - (double)a.ir_hi);
  return g31 ? launch_matrix_g<true>(a, dist, dtype, st) : launch_matrix_g<false>(a, dist, dtype, st);
}

cudaError_t launch_fill(void* out, uint64_t units, uint32_t v, cudaStream_t st) {
  if (units == 0) return cudaSuccess;
  constexpr uint64_t chunk = 4096;                       // 32-byte units: 128 KiB per warp
  const uint64_t blocks = (units + 8 * chunk - 1) / (8 * chunk);
  if (blocks > 0x7FFFFFFFull) return cudaErrorInvalidValue;
  fill_kernel<<<(unsigned)blocks, 256, 0, st>>>(static_cast<char*>(out), units, chunk, v);
  return after_launch();
}

cudaError_t launch_create31(const uint32_t seed[6], uint64_t n, const DevStreams& s,
                            cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  State sd{seed[0], seed[1], seed[2], seed[3], seed[4], seed[5]};
  create31_kernel<<<grid_for(n, 256, 8), 256, 0, st>>>(sd, n, s.cur, s.start, s.sub, s.stride);
  return after_launch();
}

cudaError_t launch_jump31(uint32_t* cur, uint64_t stride, uint64_t ns, uint64_t k,
                          cudaStream_t st) {
  if (ns == 0 || k == 0) return cudaSuccess;
  jump31_kernel<<<grid_for(ns, 256, 8), 256, 0, st>>>(cur, stride, ns, k);
  return after_launch();
}

int batch_grid() {
  static std::mutex mu;
  static int grid[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  if (grid[dev & 63] == 0) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel, 256, 0);
    grid[dev & 63] = sm_count() * (occ > 0 ? occ : 1);
  }
  return grid[dev & 63];
}

cudaError_t launch_batch(void* hdr, const void* reqs, const void* tiles, const uint32_t* start,
                         uint64_t stride, int grid, cudaStream_t st) {
  batch_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<BatchHeader*>(hdr),
                                     reinterpret_cast<const BatchReq*>(reqs),
                                     reinterpret_cast<const BatchTile*>(tiles), start, stride,
                                     K1, K2);
  return after_launch();
}

namespace {

template <int DIST, int DT>
cudaError_t launch_bv(const void* ranges, unsigned long long* counter, const void* reqs,
                      const void* tiles, const uint32_t* start, uint64_t stride,
                      bool programmatic, cudaStream_t st) {
  auto kern = batch_variant_kernel<DIST, DT>;
  static std::mutex mu;
  static int grid[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int g;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (grid[dev & 63] == 0) {
      int occ = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, 0);
      grid[dev & 63] = sm_count() * (occ > 0 ? occ : 1);
    }
    g = grid[dev & 63];
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)g);
  cfg.blockDim = dim3(256);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = programmatic ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, reinterpret_cast<const VariantRange*>(ranges),
                                     counter, reinterpret_cast<const BatchReq*>(reqs),
                                     reinterpret_cast<const BatchTile*>(tiles), start, stride,
                                     (uint64_t)K1, (uint64_t)K2);
  if (e != cudaSuccess) return e;
  return after_launch();
}

}  // namespace

cudaError_t launch_batch_variant(int k, const void* ranges, unsigned long long* counters,
                                 const void* reqs, const void* tiles, const uint32_t* start,
                                 uint64_t stride, cudaStream_t st) {
  const void* r = reinterpret_cast<const char*>(ranges) + k * sizeof(VariantRange);
  unsigned long long* c = counters + k * kCounterStride;
  const bool p = k > 0;  // variants 1..6 follow the previous kernel programmatically
  switch (k) {
    case 0: return launch_bv<MRG_NORMAL, MRG_F64>(r, c, reqs, tiles, start, stride, p, st);
    case 1: return launch_bv<MRG_NORMAL, MRG_F32>(r, c, reqs, tiles, start, stride, p, st);
    case 2: return launch_bv<MRG_EXPONENTIAL, MRG_F64>(r, c, reqs, tiles, start, stride, p, st);
    case 3: return launch_bv<MRG_EXPONENTIAL, MRG_F32>(r, c, reqs, tiles, start, stride, p, st);
    case 4: return launch_bv<MRG_UNIFORM, MRG_F32>(r, c, reqs, tiles, start, stride, p, st);
    case 5: return launch_bv<MRG_UNIFORM, MRG_F64>(r, c, reqs, tiles, start, stride, p, st);
    case 6: return launch_bv<MRG_RAW, MRG_U32>(r, c, reqs, tiles, start, stride, p, st);
    default: return cudaErrorInvalidValue;
  }
}

static_assert(sizeof(VariantRange) == sizeof(VariantRangeHost), "variant range layout");
static_assert(kCounterStride == kBatchCounterStride, "claim counter spacing");

namespace {
// Loads one kernel now (see preload_kernels).  Kernels that copy the
// transform tables (~36 KB of shared memory a block) prefer the largest
// shared-memory carveout: an SM whose split a smaller configuration fixed
// could otherwise hold none of their blocks beside a resident serving
// worker, and they would wait for it to exit.
template <class K>
void load_fn(K* f, int& bad) {
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, f) != cudaSuccess) {
    bad = 1;
    return;
  }
  if (a.sharedSizeBytes > 16384 &&
      cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                           cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    bad = 1;
}

template <int DIST, int DT>
void preload_gen(int& bad) {
  load_fn(generate_kernel<DIST, DT, 32>, bad);
  load_fn(generate_kernel<DIST, DT, 16>, bad);
  load_fn(generate_kernel<DIST, DT, 8>, bad);
  load_fn(generate_kernel<DIST, DT, 4>, bad);
  load_fn(generate31_kernel<DIST, DT, 32>, bad);
  load_fn(generate31_kernel<DIST, DT, 16>, bad);
  load_fn(generate31_kernel<DIST, DT, 8>, bad);
  load_fn(generate31_kernel<DIST, DT, 4>, bad);
}
template <int DIST, int DT>
void preload_tr(int& bad) {
  load_fn(transform_kernel<DIST, DT>, bad);
  load_fn(batch_variant_kernel<DIST, DT>, bad);
}
template <int DIST, int DT>
void preload_matrix(int& bad) {
  load_fn(matrix_kernel<false, DIST, DT>, bad);
  load_fn(matrix_kernel<true, DIST, DT>, bad);
}
}  // namespace

// Loads every kernel of the library now.  With CUDA's lazy module loading a
// kernel is otherwise loaded at its first launch, and loading may have to
// wait for kernels already running -- such as a serving worker that runs
// until it is stopped.
cudaError_t preload_kernels() {
  int bad = 0;
  preload_gen<MRG_RAW, MRG_U32>(bad);
  preload_gen<MRG_UNIFORM, MRG_F32>(bad);
  preload_gen<MRG_UNIFORM, MRG_F64>(bad);
  preload_gen<MRG_NORMAL, MRG_F32>(bad);
  preload_gen<MRG_NORMAL, MRG_F64>(bad);
  preload_gen<MRG_EXPONENTIAL, MRG_F32>(bad);
  preload_gen<MRG_EXPONENTIAL, MRG_F64>(bad);
  preload_tr<MRG_UNIFORM, MRG_F32>(bad);
  preload_tr<MRG_UNIFORM, MRG_F64>(bad);
  preload_tr<MRG_NORMAL, MRG_F32>(bad);
  preload_tr<MRG_NORMAL, MRG_F64>(bad);
  preload_tr<MRG_EXPONENTIAL, MRG_F32>(bad);
  preload_tr<MRG_EXPONENTIAL, MRG_F64>(bad);
  load_fn(batch_variant_kernel<MRG_RAW, MRG_U32>, bad);
  preload_matrix<MRG_RAW, MRG_U32>(bad);
  preload_matrix<MRG_UNIFORM, MRG_F32>(bad);
  preload_matrix<MRG_UNIFORM, MRG_F64>(bad);
  preload_matrix<MRG_EXPONENTIAL, MRG_F32>(bad);
  preload_matrix<MRG_EXPONENTIAL, MRG_F64>(bad);
  load_fn(create_kernel, bad);
  load_fn(create31_kernel, bad);
  load_fn(fisher_kernel, bad);
  load_fn(fill_kernel, bad);
  load_fn(jump31_kernel, bad);
  load_fn(jump_kernel, bad);
  load_fn(fused_kernel, bad);
  load_fn(transform_x2_kernel<MRG_NORMAL, MRG_F64>, bad);
  load_fn(transform_x2_kernel<MRG_NORMAL, MRG_F32>, bad);
  load_fn(transform_x2_kernel<MRG_EXPONENTIAL, MRG_F32>, bad);
  load_fn(transform_x2_kernel<MRG_EXPONENTIAL, MRG_F64>, bad);
  load_fn(batch_kernel, bad);
  load_fn(serve_kernel, bad);
  return bad ? cudaErrorInvalidDeviceFunction : cudaSuccess;
}

int serve_grid(double sm_fraction) {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, serve_kernel, 256, 0);
  const int per_sm = std::max(1, (int)(occ * sm_fraction + 0.5));
  return sm_count() * per_sm;
}

cudaError_t launch_serve(void* ctl, const void* slots, const void* ring, uint64_t ring_mask,
                         unsigned int* tiles_done, unsigned int* done_words,
                         unsigned long long* head_mirror, const uint32_t* start, uint64_t stride,
                         uint64_t idle_ns, int grid, cudaStream_t st) {
  serve_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<ServeCtl*>(ctl),
                                     reinterpret_cast<const BatchReq*>(slots),
                                     reinterpret_cast<const ServeTile*>(ring), ring_mask, tiles_done,
                                     done_words, head_mirror, start, stride, K1, K2, idle_ns);
  return after_launch();
}

cudaError_t launch_transform(const uint32_t* z, uint64_t n, int dist, int dtype, double rate,
                             void* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  Consts c{K1, K2, 0.0f, 0.0f};
  if (dist == MRG_EXPONENTIAL) {
    const double ir = -1.0 / rate;
    c.ir_hi = (float)ir;
    c.ir_lo = (float)(ir - (double)c.ir_hi);
  }
  char* o = reinterpret_cast<char*>(out);
  const uintptr_t al = reinterpret_cast<uintptr_t>(out);
  const unsigned grid4 = grid_for((n + 3) / 4, 256, 8);
  if (dist == MRG_NORMAL && dtype == MRG_F64 && (al & 31) == 0) {
    transform_x2_kernel<MRG_NORMAL, MRG_F64><<<grid4, 256, 0, st>>>(z, n, o, c);
    return after_launch();
  }
  if (dist == MRG_NORMAL && dtype == MRG_F32 && (al & 15) == 0) {
    transform_x2_kernel<MRG_NORMAL, MRG_F32><<<grid4, 256, 0, st>>>(z, n, o, c);
    return after_launch();
  }
  if (dist == MRG_EXPONENTIAL && dtype == MRG_F32 && (al & 15) == 0) {
    transform_x2_kernel<MRG_EXPONENTIAL, MRG_F32><<<grid4, 256, 0, st>>>(z, n, o, c);
    return after_launch();
  }
  if (dist == MRG_EXPONENTIAL && dtype == MRG_F64 && (al & 31) == 0) {
    transform_x2_kernel<MRG_EXPONENTIAL, MRG_F64><<<grid4, 256, 0, st>>>(z, n, o, c);
    return after_launch();
  }
  const uint64_t units = dist == MRG_NORMAL ? (n + 1) / 2 : n;
  const unsigned grid = grid_for(units, 256, 8);
  switch (dist * 4 + dtype) {
    case MRG_UNIFORM * 4 + MRG_F32: transform_kernel<MRG_UNIFORM, MRG_F32><<<grid, 256, 0, st>>>(z, n, o, c); break;
    case MRG_UNIFORM * 4 + MRG_F64: transform_kernel<MRG_UNIFORM, MRG_F64><<<grid, 256, 0, st>>>(z, n, o, c); break;
    case MRG_NORMAL * 4 + MRG_F32: transform_kernel<MRG_NORMAL, MRG_F32><<<grid, 256, 0, st>>>(z, n, o, c); break;
    case MRG_NORMAL * 4 + MRG_F64: transform_kernel<MRG_NORMAL, MRG_F64><<<grid, 256, 0, st>>>(z, n, o, c); break;
    case MRG_EXPONENTIAL * 4 + MRG_F32: transform_kernel<MRG_EXPONENTIAL, MRG_F32><<<grid, 256, 0, st>>>(z, n, o, c); break;
    case MRG_EXPONENTIAL * 4 + MRG_F64: transform_kernel<MRG_EXPONENTIAL, MRG_F64><<<grid, 256, 0, st>>>(z, n, o, c); break;
    default: return cudaErrorInvalidValue;
  }
  return after_launch();
}

}  // namespace mrg
