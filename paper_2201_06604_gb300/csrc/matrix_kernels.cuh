// matrix_kernels.cuh -- the paper's matrix layout (Sec. 2.2, runifGpu /
// rexpGpu with Nglobal), kept as a compatibility mode (included by
// kernels.cu).
//
// A G0 x G1 grid of work items fills an Nrow x Ncol row-major matrix: work
// item (i0, i1) owns stream i0 * G1 + i1 and visits rows i0, i0 + G0, ... and,
// within each row, columns i1, i1 + G1, ... of the matrix padded to Npad =
// ceil(Ncol / G1) * G1 columns, taking one draw per visited position and
// writing it only where the column is a real one.  This is the reading under
// which the paper's printed runifGpu vector and rexpGpu matrix are reproduced
// (a vector of n values is the n x 1 matrix).  Unlike mrg_generate, the
// output depends on the work-item grid; one thread runs one work item.
#pragma once

namespace mrg {

struct MatrixArgs {
  uint32_t* cur;
  uint64_t stride;
  uint64_t nrow, ncol, npad;
  uint32_t g0, g1;
  char* out;
  uint64_t ld;           // elements
  float ir_hi, ir_lo;    // -1/rate (exponentials)
};

template <bool G31, int DIST, int DT>
__global__ void __launch_bounds__(256) matrix_kernel(MatrixArgs a, uint64_t k1, uint64_t k2) {
  constexpr int ES = DT == MRG_F64 ? 8 : 4;
  __shared__ float4 s_tab[DIST == MRG_EXPONENTIAL ? TAB_ENTRIES : 1];
  if constexpr (DIST == MRG_EXPONENTIAL) {
    if constexpr (G31) load_ttab31(s_tab);
    else load_ttab(s_tab);
  }
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (uint64_t)a.g0 * a.g1) return;
  const uint32_t i0 = (uint32_t)(t / a.g1), i1 = (uint32_t)(t % a.g1);
  State st = load_state(a.cur, a.stride, t);
  TState ts = to_offset(st);
  for (uint64_t r = i0; r < a.nrow; r += a.g0) {
    for (uint64_t c = i1; c < a.npad; c += a.g1) {
      uint32_t z;
      if constexpr (G31) z = g31::step(st);
      else z = step_fast(ts, k1, k2);
      if (c >= a.ncol) continue;
      char* dst = a.out + (r * a.ld + c) * ES;
      if constexpr (DIST == MRG_RAW) {
        *reinterpret_cast<uint32_t*>(dst) = z;
      } else if constexpr (DIST == MRG_UNIFORM) {
        if constexpr (DT == MRG_F64)
          *reinterpret_cast<uint64_t*>(dst) = G31 ? g31::uniform_bits64(z) : uniform_bits64_fast(z);
        else
          *reinterpret_cast<uint32_t*>(dst) = G31 ? g31::uniform_bits32(z) : uniform_bits32(z);
      } else if constexpr (DT == MRG_F64) {
        const df l = G31 ? ln_u_df_m<UM2p32>(2u * z, s_tab) : ln_u_df(z, s_tab);
        *reinterpret_cast<uint64_t*>(dst) = df_to_f64_bits(df_mul(l, df{a.ir_hi, a.ir_lo}));
      } else {
        *reinterpret_cast<float*>(dst) = G31 ? exp_f32_m<UM2p32>(2u * z, s_tab, a.ir_hi, a.ir_lo)
                                             : exp_f32(z, s_tab, a.ir_hi, a.ir_lo);
      }
    }
  }
  if constexpr (G31) store_state(a.cur, a.stride, t, st);
  else store_state(a.cur, a.stride, t, from_offset(ts));
}

}  // namespace mrg
