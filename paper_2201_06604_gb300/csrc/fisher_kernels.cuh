// fisher_kernels.cuh -- Monte Carlo Fisher's exact test (Sec. 4) fused with
// the generator (included by kernels.cu).
//
// Replicate b runs on stream b mod ns and takes that stream's next
// (I-1)(J-1) fp64 uniforms; one thread owns one stream and runs its
// replicates in increasing b, so the streams advance exactly as if the draws
// had been generated and consumed one after another.  A replicate samples a
// table with the observed margins row by row, left to right (Patefield's
// method as the paper describes it): cell (i, j) is the number of marked
// items among the R units still to place in row i, drawn without replacement
// from the S units left in columns j..J-1 of rows i..I-1, of which K are in
// column j -- a hypergeometric variable, sampled by standard inversion of its
// CDF (the smallest x with u <= F(x)) with one uniform.  The statistic
// -sum log(n_ij!) is accumulated row by row, left to right, from a table of
// log-factorials; nothing but the count (and optionally the statistics)
// leaves the SM.
//
// The inversion works outwards from the mode (see hyper_inv): O(standard
// deviation) steps in double-float arithmetic, with an fp64 re-evaluation of
// the rare draws that fall within 2^-32 of a CDF step, so every decision is
// the one fp64 standard inversion takes (the precision of the paper's R
// code).
#pragma once

namespace mrg {

struct FisherArgs {
  uint32_t* cur;
  uint64_t stride, ns;
  const int32_t* rows;   // row sums, I
  const int32_t* cols;   // column sums, J
  const double* lf;      // log(k!), k = 0..n
  uint32_t I, J;
  uint64_t B;            // replicates
  double threshold;      // count statistics <= threshold
  unsigned long long* count;
  double* stats;         // per-replicate statistic, or null
  int32_t total;         // n
};

// log P(X = x) of the hypergeometric law below, evaluated in the order the
// exact path and its reference definition use.
__device__ __forceinline__ double hyper_logpmf(int32_t S, int32_t K, int32_t R, int32_t x,
                                               const double* __restrict__ lf) {
  return lf[K] - lf[x] - lf[K - x] + lf[S - K] - lf[R - x] - lf[S - K - R + x] -
         (lf[S] - lf[R] - lf[S - R]);
}

// Exact path: F accumulated in fp64 from the bottom of the support, one pmf
// term (one exp) per point -- the definition of standard inversion written
// out.  Used only when the fast path cannot tell the side of a CDF step.
__device__ __noinline__ int32_t hyper_inv_exact(int32_t S, int32_t K, int32_t R, double u,
                                                const double* __restrict__ lf) {
  const int32_t lo = max(0, R - (S - K));
  const int32_t hi = min(R, K);
  double F = 0.0;
  for (int32_t x = lo; x < hi; ++x) {
    F += exp(hyper_logpmf(S, K, R, x, lf));
    if (u <= F) return x;
  }
  return hi;
}

// a / b for exact floats a, b (integers below 2^24) as a double-float.
__device__ __forceinline__ df df_quot(float a, float b) {
  const float h = __fdiv_rn(a, b);
  const float r = __fmaf_rn(-h, b, a);     // exact remainder
  return df{h, __fdiv_rn(r, b)};
}

__device__ __forceinline__ double df_value(df v) { return (double)v.hi + (double)v.lo; }

// Smallest x with u <= F(x) for the number of marked items in R draws without
// replacement from S items of which K are marked (0 <= K, R <= S), S < 2^24.
//
// Fast path: P(m) at the mode from the log-factorial table (fp64, one exp);
// F(m) by summing the pmf down from m until the terms vanish against it;
// then a walk down (u <= F(m)) or up (u > F(m)), the pmf following its ratio
// recursion -- all in double-float arithmetic on the FP32 pipe (~2^-47
// relative per operation; GB300's FP64 pipe is a small fraction of its FP32
// rate).  The fast result is kept only if u lies more than 2^-32 from both
// CDF values that bracket it, far beyond the rounding of either evaluation;
// otherwise the exact fp64 path decides.  So the decision is the fp64 one.
__device__ __forceinline__ int32_t hyper_inv(int32_t S, int32_t K, int32_t R, double u,
                                             const double* __restrict__ lf) {
  const int32_t lo = max(0, R - (S - K));
  const int32_t hi = min(R, K);
  if (lo == hi) return lo;
  const int32_t SKR = S - K - R;
  int32_t m = (int32_t)(((int64_t)(R + 1) * (K + 1)) / (S + 2));
  m = min(max(m, lo), hi);
  const double pm64 = exp(hyper_logpmf(S, K, R, m, lf));
  const float pm_hi = (float)pm64;
  const df pm{pm_hi, (float)(pm64 - (double)pm_hi)};
  // P(x - 1) / P(x) = [x / (K - x + 1)] [(SKR + x) / (R - x + 1)]
  auto down = [&](int32_t x) {
    return df_mul(df_quot((float)x, (float)(K - x + 1)),
                  df_quot((float)(SKR + x), (float)(R - x + 1)));
  };
  // P(x + 1) / P(x) = [(K - x) / (x + 1)] [(R - x) / (SKR + x + 1)]
  auto up = [&](int32_t x) {
    return df_mul(df_quot((float)(K - x), (float)(x + 1)),
                  df_quot((float)(R - x), (float)(SKR + x + 1)));
  };
  df F = pm, q = pm;
  for (int32_t x = m; x > lo; --x) {
    q = df_mul(q, down(x));
    F = df_add(F, q);
    if (q.hi <= F.hi * 0x1p-60f) break;
  }
  int32_t x = m;
  df px = pm, Fx = F;
  if (df_value(F) >= u) {  // walk down while u <= F(x - 1) = F(x) - P(x)
    while (x > lo) {
      const df Fprev = df_add(Fx, df_neg(px));
      if (u > df_value(Fprev)) break;
      px = df_mul(px, down(x));
      Fx = Fprev;
      --x;
    }
  } else {                 // walk up while F(x) < u
    while (x < hi && df_value(Fx) < u) {
      px = df_mul(px, up(x));
      ++x;
      Fx = df_add(Fx, px);
    }
  }
  // bracket: F(x - 1) < u <= F(x); 0 below the support
  const double fx = df_value(Fx);
  const double fprev = x > lo ? df_value(df_add(Fx, df_neg(px))) : 0.0;
  constexpr double kGuard = 0x1p-32;
  if (fx - u >= kGuard && u - fprev >= kGuard) return x;
  return hyper_inv_exact(S, K, R, u, lf);
}

__global__ void __launch_bounds__(256) fisher_kernel(FisherArgs a, uint64_t k1, uint64_t k2) {
  __shared__ int32_t s_rows[kFisherMaxDim], s_cols[kFisherMaxDim];
  for (uint32_t t = threadIdx.x; t < a.I; t += blockDim.x) s_rows[t] = a.rows[t];
  for (uint32_t t = threadIdx.x; t < a.J; t += blockDim.x) s_cols[t] = a.cols[t];
  __syncthreads();
  const double* __restrict__ lf = a.lf;
  const uint32_t I = a.I, J = a.J;
  const uint64_t step_all = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t sidx = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; sidx < a.ns;
       sidx += step_all) {
    TState st = to_offset(load_state(a.cur, a.stride, sidx));
    unsigned long long cnt = 0;
    int32_t C[kFisherMaxDim];
    for (uint64_t b = sidx; b < a.B; b += a.ns) {
      for (uint32_t j = 0; j < J; ++j) C[j] = s_cols[j];
      int32_t rest = a.total;
      double T = 0.0;
      for (uint32_t i = 0; i + 1 < I; ++i) {
        int32_t R = s_rows[i];
        int32_t S = rest;
        for (uint32_t j = 0; j + 1 < J; ++j) {
          const double u = __longlong_as_double((long long)uniform_bits64_fast(step_fast(st, k1, k2)));
          const int32_t x = hyper_inv(S, C[j], R, u, lf);
          T -= lf[x];
          S -= C[j];
          C[j] -= x;
          R -= x;
        }
        T -= lf[R];
        C[J - 1] -= R;
        rest -= s_rows[i];
      }
      for (uint32_t j = 0; j < J; ++j) T -= lf[C[j]];
      if (a.stats) a.stats[b] = T;
      cnt += T <= a.threshold;
    }
    if (cnt) atomicAdd(a.count, cnt);
    store_state(a.cur, a.stride, sidx, from_offset(st));
  }
}

}  // namespace mrg
