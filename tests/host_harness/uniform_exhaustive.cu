// Host-side check of the kernels' integer arithmetic, compiled by nvcc for
// the CPU from the same header the kernels use (test infrastructure).
//   mode "uniform": for every z in [1, m1], uniform_bits64(z) equals the bits
//     of the IEEE product (double)z * RN64(1/(m1+1)), and f32_bits_from_f64
//     of it and uniform_bits32(z) (the fp32 uniform formed without the
//     double) equal the bits of (float) of that product.
//   mode "step" n seed: prints n outputs of mrg::step from a state.
//   mode "uniform31": for every z in [1, 2^31 - 1], g31::uniform_bits64(z) and
//     g31::uniform_bits32(z) equal the bits of (double)z * 2^-31 and of its
//     rounding to float (MRG31k3p).
//   mode "step31" n seed: prints n outputs of g31::step from a state.
//   mode "matern": prints e^x K_nu(x) and the Matern correlation of
//     matern.cuh on a grid of orders and arguments ("nu x kscaled corr").
//   mode "ozround": reads lines "th tl E" (decimal) and prints the bits of
//     ozaki_round(th, tl, E) as 16 hex digits, one a line (the rounding of the
//     GRF product kernels' exact level sum).
//   mode "tables": prints the double-float transform tables the library
//     uploads (host_jump.cpp, linked in), for M = m1 + 1 (table 0) and
//     M = 2^32 (table 1), one float4 entry a line as hex floats.
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "../../paper_2201_06604_gb300/csrc/mrg32k3a_core.cuh"
#include "../../paper_2201_06604_gb300/csrc/mrg31k3p_core.cuh"
#include "../../paper_2201_06604_gb300/csrc/host_jump.h"
#include "../../paper_2201_06604_gb300/csrc/matern.cuh"
#include "../../paper_2201_06604_gb300/csrc/ozaki_round.cuh"
#include <cmath>

static int check_uniform(unsigned lo, unsigned hi) {
  volatile double norm_v = 1.0 / 4294967088.0;
  const double norm = norm_v;
  long long bad = 0;
#pragma omp parallel for reduction(+ : bad) schedule(static, 1 << 16)
  for (long long zz = lo; zz <= (long long)hi; ++zz) {
    uint32_t z = (uint32_t)zz;
    double d = (double)z * norm;
    uint64_t want;
    std::memcpy(&want, &d, 8);
    float f = (float)d;
    uint32_t wantf;
    std::memcpy(&wantf, &f, 4);
    uint64_t got = mrg::uniform_bits64(z);
    if (got != want || mrg::f32_bits_from_f64(got) != wantf || mrg::uniform_bits32(z) != wantf) {
      if (bad < 5) std::printf("mismatch z=%u got=%016llx want=%016llx\n", z,
                               (unsigned long long)got, (unsigned long long)want);
      ++bad;
    }
  }
  std::printf("checked [%u, %u]: %lld mismatches\n", lo, hi, bad);
  return bad != 0;
}

static int check_uniform31() {
  long long bad = 0;
#pragma omp parallel for reduction(+ : bad) schedule(static, 1 << 16)
  for (long long zz = 1; zz < (1ll << 31); ++zz) {
    uint32_t z = (uint32_t)zz;
    double d = (double)z * 0x1p-31;
    float f = (float)d;
    uint64_t want;
    uint32_t wantf;
    std::memcpy(&want, &d, 8);
    std::memcpy(&wantf, &f, 4);
    if (mrg::g31::uniform_bits64(z) != want || mrg::g31::uniform_bits32(z) != wantf) {
      if (bad < 5) std::printf("mismatch z=%u\n", z);
      ++bad;
    }
  }
  std::printf("checked [1, 2^31 - 1]: %lld mismatches\n", bad);
  return bad != 0;
}

static float g_tab[mrg::host::kTransformEntries][4];

static int print_tables() {
  for (int t = 0; t < 2; ++t) {
    if (t == 0) mrg::host::transform_table(g_tab);
    else mrg::host::transform_table_m32(g_tab);
    for (int i = 0; i < mrg::host::kTransformEntries; ++i)
      std::printf("%d %d %a %a %a %a\n", t, i, (double)g_tab[i][0], (double)g_tab[i][1],
                  (double)g_tab[i][2], (double)g_tab[i][3]);
  }
  return 0;
}

static int print_matern() {
  const double nus[] = {0.0, 0.05, 0.5, 0.6, 1.25, 1.5, 2.15, 2.5, 3.0, 5.5, 10.0};
  for (double nu : nus) {
    const double norm = nu > 0 ? std::pow(2.0, 1.0 - nu) / std::tgamma(nu) : 0.0;
    for (int i = 0; i <= 400; ++i) {
      const double x = 1e-6 * std::pow(7e8, i / 400.0);       // 1e-6 .. 700, geometric
      std::printf("%.17g %.17g %.17g %.17g\n", nu, x, mrg::bessel_k_scaled(nu, x),
                  nu > 0 ? mrg::matern_corr(x, nu, norm) : 0.0);
    }
  }
  return 0;
}

static int ozround() {
  long long th, tl;
  int E;
  while (std::scanf("%lld %lld %d", &th, &tl, &E) == 3) {
    const double d = mrg::grf::ozaki_round(th, tl, E);
    uint64_t b;
    std::memcpy(&b, &d, 8);
    std::printf("%016llx\n", (unsigned long long)b);
  }
  return 0;
}

int main(int argc, char** argv) {
  if (argc >= 2 && !std::strcmp(argv[1], "tables")) return print_tables();
  if (argc >= 2 && !std::strcmp(argv[1], "ozround")) return ozround();
  if (argc >= 2 && !std::strcmp(argv[1], "matern")) return print_matern();
  if (argc >= 2 && !std::strcmp(argv[1], "uniform31")) return check_uniform31();
  if (argc >= 9 && !std::strcmp(argv[1], "step31")) {
    long n = std::atol(argv[2]);
    mrg::State c{(uint32_t)std::strtoul(argv[3], 0, 10), (uint32_t)std::strtoul(argv[4], 0, 10),
                 (uint32_t)std::strtoul(argv[5], 0, 10), (uint32_t)std::strtoul(argv[6], 0, 10),
                 (uint32_t)std::strtoul(argv[7], 0, 10), (uint32_t)std::strtoul(argv[8], 0, 10)};
    for (long i = 0; i < n; ++i) std::printf("%u\n", mrg::g31::step(c));
    std::printf("%u %u %u %u %u %u\n", c.a0, c.a1, c.a2, c.b0, c.b1, c.b2);
    return 0;
  }
  if (argc >= 2 && !std::strcmp(argv[1], "uniform")) {
    unsigned lo = argc > 2 ? (unsigned)std::strtoul(argv[2], 0, 10) : 1u;
    unsigned hi = argc > 3 ? (unsigned)std::strtoul(argv[3], 0, 10) : mrg::M1;
    return check_uniform(lo, hi);
  }
  if (argc >= 9 && !std::strcmp(argv[1], "step")) {
    long n = std::atol(argv[2]);
    mrg::State c{(uint32_t)std::strtoul(argv[3], 0, 10), (uint32_t)std::strtoul(argv[4], 0, 10),
                 (uint32_t)std::strtoul(argv[5], 0, 10), (uint32_t)std::strtoul(argv[6], 0, 10),
                 (uint32_t)std::strtoul(argv[7], 0, 10), (uint32_t)std::strtoul(argv[8], 0, 10)};
    mrg::TState s = mrg::to_offset(c);
    for (long i = 0; i < n; ++i) std::printf("%u\n", mrg::step(s));
    c = mrg::from_offset(s);
    std::printf("%u %u %u %u %u %u\n", c.a0, c.a1, c.a2, c.b0, c.b1, c.b2);
    return 0;
  }
  std::fprintf(stderr, "usage: uniform [lo hi] | step n s0..s5 | uniform31 | step31 n s0..s5 | tables | matern | ozround\n");
  return 2;
}
