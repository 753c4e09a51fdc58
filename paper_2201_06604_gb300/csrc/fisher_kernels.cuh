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

__device__ __forceinline__ double df_value(df v) { return (double)v.hi + (double)v.lo; }

// x * y for floats as an exact double-float (FMA error-free product).
__device__ __forceinline__ df two_prod(float x, float y) {
  const float p = __fmul_rn(x, y);
  return df{p, __fmaf_rn(x, y, -p)};
}

// (a1 a2) / (b1 b2) for exact floats (integers below 2^24) as a double-float:
// exact numerator and denominator products, one reciprocal, one correction
// step (relative error ~2^-45).
__device__ __forceinline__ df df_ratio(float a1, float a2, float b1, float b2) {
  const df num = two_prod(a1, a2), den = two_prod(b1, b2);
  const float rc = __frcp_rn(den.hi);
  const float q1 = __fmul_rn(num.hi, rc);
  // num - q1 den, exactly enough: q1 den as a double-float
  const df t = df_mul_f(den, q1);
  const df r = df_add(num, df_neg(t));
  return fast_two_sum(q1, __fmul_rn(r.hi, rc));
}

// exp(x) for x in [-80, 0] as a double-float (relative error ~2^-38): x = k ln 2
// + r in fp64, exp(r / 256) by its Taylor series to the fifth power, squared
// eight times, scaled by 2^k.
__device__ __forceinline__ df df_exp(double x) {
  const double k = rint(x * 1.4426950408889634);
  const double r = (x - k * 0.6931471805599453) - k * 2.3190468138462996e-17;  // |r| < 0.35
  const double rs = r * 0x1p-8;
  const float rh = (float)rs;
  const df t{rh, (float)(rs - (double)rh)};
  // 1 + t + t^2/2 + t^3/6 + t^4/24 + t^5/120, |t| < 0.0014
  df e = df_add(df{1.0f, 0.0f}, t);
  df tp = df_mul(t, t);
  e = df_add(e, df{tp.hi * 0.5f, tp.lo * 0.5f});
  const float tf = t.hi;
  const float tail = __fmul_rn(tp.hi, __fmul_rn(tf, __fmaf_rn(tf, __fmaf_rn(tf, 1.0f / 120.0f, 1.0f / 24.0f), 1.0f / 6.0f)));
  e = df_add(e, df{tail, 0.0f});
#pragma unroll
  for (int i = 0; i < 8; ++i) e = df_mul(e, e);
  const float sc = __int_as_float((127 + (int)k) << 23);   // 2^k, k in [-115, 0]
  return df{e.hi * sc, e.lo * sc};
}

// v <= u for a double-float v and a double u given as a double-float.
__device__ __forceinline__ bool df_le(df v, df u) { return v.hi < u.hi || (v.hi == u.hi && v.lo <= u.lo); }

// Smallest x with u <= F(x) for the number of marked items in R draws without
// replacement from S items of which K are marked (0 <= K, R <= S), S < 2^24.
//
// Fast path: log P(m) at the mode from the log-factorial table (fp64: the
// terms cancel down from ~S ln S), P(m) = exp of it, F(m) by summing the pmf
// down from m until the terms vanish against it, then a walk down
// (u <= F(m)) or up (u > F(m)), the pmf following its ratio recursion -- all
// but the log sum in double-float arithmetic on the FP32 pipe (GB300's FP64
// rate is a small fraction of its FP32 rate).  The fast result is kept only
// if u lies at least 2^-32 from both CDF values that bracket it -- far beyond
// the ~1e-11 error of either evaluation; otherwise the exact fp64 path
// decides.  So the decision is the fp64 one.
__device__ __forceinline__ int32_t hyper_inv(int32_t S, int32_t K, int32_t R, double u,
                                             const double* __restrict__ lf) {
  const int32_t lo = max(0, R - (S - K));
  const int32_t hi = min(R, K);
  if (lo == hi) return lo;
  const int32_t SKR = S - K - R;
  int32_t m = (int32_t)(((int64_t)(R + 1) * (K + 1)) / (S + 2));
  m = min(max(m, lo), hi);
  const df pm = df_exp(hyper_logpmf(S, K, R, m, lf));
  const float uh = (float)u;
  const df ud{uh, (float)(u - (double)uh)};
  // P(x - 1) / P(x) = x (SKR + x) / ((K - x + 1) (R - x + 1)); the four
  // integer factors are kept as floats (exact below 2^24) and stepped by one
  df F = pm, q = pm;
  {
    float a = (float)m, b = (float)(SKR + m), c = (float)(K - m + 1), d = (float)(R - m + 1);
    for (int32_t x = m; x > lo; --x) {
      q = df_mul(q, df_ratio(a, b, c, d));
      F = df_add(F, q);
      if (q.hi <= F.hi * 0x1p-60f) break;
      a -= 1.0f; b -= 1.0f; c += 1.0f; d += 1.0f;
    }
  }
  int32_t x = m;
  df px = pm, Fx = F;
  if (df_le(ud, F)) {      // walk down while u <= F(x - 1) = F(x) - P(x)
    float a = (float)m, b = (float)(SKR + m), c = (float)(K - m + 1), d = (float)(R - m + 1);
    while (x > lo) {
      const df Fprev = df_add(Fx, df_neg(px));
      if (!df_le(ud, Fprev)) break;
      px = df_mul(px, df_ratio(a, b, c, d));
      Fx = Fprev;
      --x;
      a -= 1.0f; b -= 1.0f; c += 1.0f; d += 1.0f;
    }
  } else {                 // walk up while F(x) < u:
    // P(x + 1) / P(x) = (K - x) (R - x) / ((x + 1) (SKR + x + 1))
    float a = (float)(K - m), b = (float)(R - m), c = (float)(m + 1), d = (float)(SKR + m + 1);
    while (x < hi && !df_le(ud, Fx)) {
      px = df_mul(px, df_ratio(a, b, c, d));
      ++x;
      Fx = df_add(Fx, px);
      a -= 1.0f; b -= 1.0f; c += 1.0f; d += 1.0f;
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
