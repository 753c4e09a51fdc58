// gen31_kernels.cuh -- kernels of MRG31k3p, the paper's own generator
// (included by kernels.cu, which owns store_vec, load_state and Consts).
//
// The same decomposition as the MRG32k3a kernels: stream i starts
// i * 2^134 steps after the creator seed (Sec. 2.1, streams created one after
// another), and every lane of the generate kernel owns a contiguous segment
// of one stream's row, reached by an absolute jump, so the output does not
// depend on the launch shape.  The transforms take u = z / 2^31 as
// z' / 2^32 with z' = 2 z (the double-float code with M = 2^32).
#pragma once

#include "mrg31k3p_core.cuh"

namespace mrg {

__constant__ uint32_t c_jump31[2][g31::JUMP_BITS][9];
__device__ float4 g_ttab31[TAB_ENTRIES];

cudaError_t upload_tables31(const uint32_t* tab, size_t bytes) {
  if (bytes != sizeof(c_jump31)) return cudaErrorInvalidValue;
  return cudaMemcpyToSymbol(c_jump31, tab, bytes);
}

cudaError_t upload_transform_table31(const float* tab, size_t bytes) {
  if (bytes != sizeof(g_ttab31)) return cudaErrorInvalidValue;
  return cudaMemcpyToSymbol(g_ttab31, tab, bytes);
}

__device__ __forceinline__ void load_ttab31(float4* s_tab) {
  for (int i = threadIdx.x; i < TAB_ENTRIES; i += blockDim.x) s_tab[i] = g_ttab31[i];
  __syncthreads();
}

__device__ __forceinline__ void apply_pow2_31(int i, State& s) {
  uint32_t A[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) A[k] = c_jump31[0][i][k];
  g31::matvec<0>(A, s.a0, s.a1, s.a2);
#pragma unroll
  for (int k = 0; k < 9; ++k) A[k] = c_jump31[1][i][k];
  g31::matvec<1>(A, s.b0, s.b1, s.b2);
}

// s <- A^(e 2^base) s with a per-lane exponent e; the loop runs over the bits
// set in any lane, so table reads are warp-uniform.  All 32 lanes call it.
__device__ __forceinline__ void jump_lanes31(State& s, uint64_t e, int base) {
  unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)e);
  unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(e >> 32));
  uint64_t any = ((uint64_t)hi << 32) | lo;
  while (any) {
    int i = __ffsll((long long)any) - 1;
    any &= any - 1;
    if ((e >> i) & 1) apply_pow2_31(base + i, s);
  }
}

__global__ void __launch_bounds__(256) create31_kernel(State seed, uint64_t n, uint32_t* cur,
                                                       uint32_t* start, uint32_t* sub,
                                                       uint64_t stride) {
  const uint64_t step_all = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < n; base += step_all) {
    const uint64_t i = base + threadIdx.x;
    const bool valid = i < n;
    State s = seed;
    jump_lanes31(s, valid ? i : 0, g31::STREAM_LOG2);
    if (valid) {
      store_state(cur, stride, i, s);
      store_state(start, stride, i, s);
      store_state(sub, stride, i, s);
    }
  }
}

// cur <- A^k cur for every stream (k < 2^64; the advance after a generate
// call, or a skip).
__global__ void __launch_bounds__(256) jump31_kernel(uint32_t* cur, uint64_t stride, uint64_t ns,
                                                     uint64_t k) {
  const uint64_t step_all = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += step_all) {
    State s = load_state(cur, stride, i);
    for (uint64_t e = k; e; e &= e - 1) apply_pow2_31(__ffsll((long long)e) - 1, s);
    store_state(cur, stride, i, s);
  }
}

template <int DIST, int DT, int UE>
__device__ __forceinline__ void produce31(State& s, uint32_t* w, const Consts& c,
                                          const float4* __restrict__ tab) {
  if constexpr (DIST == MRG_RAW) {
#pragma unroll
    for (int e = 0; e < UE; ++e) w[e] = g31::step(s);
  } else if constexpr (DIST == MRG_UNIFORM && DT == MRG_F64) {
#pragma unroll
    for (int e = 0; e < UE; ++e) put_f64(w + 2 * e, g31::uniform_bits64(g31::step(s)));
  } else if constexpr (DIST == MRG_UNIFORM) {
#pragma unroll
    for (int e = 0; e < UE; ++e) w[e] = g31::uniform_bits32(g31::step(s));
  } else if constexpr (DIST == MRG_NORMAL && DT == MRG_F64 && UE % 4 == 0) {
    // two pairs per packed fp32x2 evaluation (bit-identical to the scalar one)
#pragma unroll
    for (int p = 0; p < UE / 4; ++p) {
      const uint32_t z1a = 2u * g31::step(s);
      const uint32_t z2a = 2u * g31::step(s);
      const uint32_t z1b = 2u * g31::step(s);
      const uint32_t z2b = 2u * g31::step(s);
      uint64_t xa, ya, xb, yb;
      box_muller_f64_x2<UM2p32>(z1a, z2a, z1b, z2b, tab, xa, ya, xb, yb);
      put_f64(w + 8 * p, xa);
      put_f64(w + 8 * p + 2, ya);
      put_f64(w + 8 * p + 4, xb);
      put_f64(w + 8 * p + 6, yb);
    }
  } else if constexpr (DIST == MRG_NORMAL && DT == MRG_F32 && UE % 4 == 0) {
#pragma unroll
    for (int p = 0; p < UE / 4; ++p) {
      const uint32_t z1a = 2u * g31::step(s);
      const uint32_t z2a = 2u * g31::step(s);
      const uint32_t z1b = 2u * g31::step(s);
      const uint32_t z2b = 2u * g31::step(s);
      float xa, ya, xb, yb;
      box_muller_f32_x2<UM2p32>(z1a, z2a, z1b, z2b, tab, xa, ya, xb, yb);
      w[4 * p] = __float_as_uint(xa);
      w[4 * p + 1] = __float_as_uint(ya);
      w[4 * p + 2] = __float_as_uint(xb);
      w[4 * p + 3] = __float_as_uint(yb);
    }
  } else if constexpr (DIST == MRG_NORMAL) {
#pragma unroll
    for (int p = 0; p < UE / 2; ++p) {
      const uint32_t z1 = g31::step(s);
      const uint32_t z2 = g31::step(s);
      if constexpr (DT == MRG_F64) {
        uint64_t x, y;
        box_muller_f64_m<UM2p32>(2u * z1, 2u * z2, tab, x, y);
        put_f64(w + 4 * p, x);
        put_f64(w + 4 * p + 2, y);
      } else {
        float x, y;
        box_muller_f32_m<UM2p32>(2u * z1, 2u * z2, tab, x, y);
        w[2 * p] = __float_as_uint(x);
        w[2 * p + 1] = __float_as_uint(y);
      }
    }
  } else if constexpr (DT == MRG_F64 && UE % 2 == 0) {   // exponential, two draws per packed evaluation
#pragma unroll
    for (int e = 0; e < UE; e += 2) {
      const uint32_t za = 2u * g31::step(s);
      const uint32_t zb = 2u * g31::step(s);
      uint64_t ea, eb;
      exp_f64_x2<UM2p32>(za, zb, tab, c.ir_hi, c.ir_lo, ea, eb);
      put_f64(w + 2 * e, ea);
      put_f64(w + 2 * e + 2, eb);
    }
  } else if constexpr (DT == MRG_F32 && UE % 2 == 0) {   // exponential, two draws per packed evaluation
#pragma unroll
    for (int e = 0; e < UE; e += 2) {
      const uint32_t za = 2u * g31::step(s);
      const uint32_t zb = 2u * g31::step(s);
      float ea, eb;
      exp_f32_x2<UM2p32>(za, zb, tab, c.ir_hi, c.ir_lo, ea, eb);
      w[e] = __float_as_uint(ea);
      w[e + 1] = __float_as_uint(eb);
    }
  } else {  // exponential: -ln(u) / rate
#pragma unroll
    for (int e = 0; e < UE; ++e) {
      const uint32_t z2 = 2u * g31::step(s);
      if constexpr (DT == MRG_F64)
        put_f64(w + 2 * e, df_to_f64_bits(df_mul(ln_u_df_m<UM2p32>(z2, tab), df{c.ir_hi, c.ir_lo})));
      else
        w[e] = __float_as_uint(exp_f32_m<UM2p32>(z2, tab, c.ir_hi, c.ir_lo));
    }
  }
}

// Materialised generation (same argument block and lane mapping as
// generate_kernel: segment q runs stream q mod ns at segment q div ns).
template <int DIST, int DT, int VB>
__global__ void __launch_bounds__(256) generate31_kernel(GenArgs a) {
  constexpr int ES = DT == MRG_F64 ? 8 : 4;
  constexpr int UB = (DIST == MRG_NORMAL && VB < 2 * ES) ? 2 * ES : (VB < ES ? ES : VB);
  constexpr int UE = UB / ES;
  constexpr int UW = UB / 4;
  constexpr int VS = VB < ES ? ES : VB;
  constexpr int VW = VS / 4;

  constexpr bool TABLES = DIST == MRG_NORMAL || DIST == MRG_EXPONENTIAL;
  __shared__ float4 s_tab[TABLES ? TAB_ENTRIES : 1];
  if constexpr (TABLES) load_ttab31(s_tab);

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
    State st = valid ? load_state(a.cur, a.stride, s) : State{1, 1, 1, 1, 1, 1};
    jump_lanes31(st, off, 0);
    const uint32_t cmax = __reduce_max_sync(0xffffffffu, cnt);
    char* gdst = a.out + (s * a.ld + off) * ES;

    constexpr int UNROLL = TABLES ? 1 : 2;  // as in generate_kernel
#pragma unroll UNROLL
    for (uint32_t i = 0; i < cmax; i += UE) {
      uint32_t wv[UW];
      produce31<DIST, DT, UE>(st, wv, c, s_tab);
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

}  // namespace mrg
