// capi.cu -- extern "C" entry points of libmrg32k3a (declared in
// include/mrg32k3a.h).  Argument checking, per-device table upload, and the
// host-side creator arithmetic live here; every per-stream step runs in the
// kernels of kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mrg32k3a.h"
#include "host_jump.h"
#include "internal.h"
#include "mrg32k3a_core.cuh"

namespace {

thread_local std::string t_err;

int fail(int code, const char* msg) {
  t_err = msg;
  return code;
}

int fail_cuda(cudaError_t e, const char* where) {
  t_err = std::string(where) + ": " + cudaGetErrorName(e) + ": " + cudaGetErrorString(e);
  return MRG_ECUDA;
}

// Per-device one-time set-up: the jump tables go to constant memory.
int ensure_device() {
  static std::mutex mu;
  static bool ready[64] = {};
  static uint32_t tab[2][mrg::host::kJumpBits][9];
  static float ttab[mrg::host::kTransformEntries][4];
  static uint32_t tab31[2][mrg::host::g31::kJumpBits][9];
  static float ttab31[mrg::host::kTransformEntries][4];
  static bool tab_built = false;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_cuda(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(MRG_ECUDA, "device index out of range");
  std::lock_guard<std::mutex> lk(mu);
  if (ready[dev]) return MRG_OK;
  if (!tab_built) {
    if (!mrg::host::norm_constant_ok(mrg::NORM_DELTA))
      return fail(MRG_ECUDA, "RN64(1/(m1+1)) does not match the kernels' constant");
    mrg::host::jump_table_u32(tab);
    mrg::host::transform_table(ttab);
    mrg::host::g31::jump_table_u32(tab31);
    mrg::host::transform_table_m32(ttab31);
    tab_built = true;
  }
  e = mrg::upload_tables(&tab[0][0][0], sizeof(tab));
  if (e != cudaSuccess) return fail_cuda(e, "uploading jump tables");
  e = mrg::upload_transform_table(&ttab[0][0], sizeof(ttab));
  if (e != cudaSuccess) return fail_cuda(e, "uploading transform tables");
  e = mrg::upload_tables31(&tab31[0][0][0], sizeof(tab31));
  if (e == cudaSuccess) e = mrg::upload_transform_table31(&ttab31[0][0], sizeof(ttab31));
  if (e != cudaSuccess) return fail_cuda(e, "uploading MRG31k3p tables");
  e = mrg::preload_kernels();
  if (e != cudaSuccess) return fail_cuda(e, "loading the library's kernels");
  ready[dev] = true;
  return MRG_OK;
}

bool streams_ok(const mrg_streams* s) {
  return s && s->cur && s->start && s->sub && s->stride >= s->n;
}

mrg::DevStreams dev(const mrg_streams* s) {
  return mrg::DevStreams{s->cur, s->start, s->sub, s->n, s->stride};
}

inline cudaStream_t cs(void* p) { return reinterpret_cast<cudaStream_t>(p); }

// rows x leading dimension x element size stays addressable (< 2^62 bytes).
bool extent_ok(uint64_t rows, uint64_t ld, uint64_t es) {
  const unsigned __int128 bytes = (unsigned __int128)rows * ld * es;
  return bytes < ((unsigned __int128)1 << 62);
}

}  // namespace

namespace mrg {
int ensure_device_ready() { return ensure_device(); }
int set_error(int code, const char* msg) { return fail(code, msg); }
}  // namespace mrg

extern "C" {

const char* mrg_last_error(void) { return t_err.c_str(); }

uint64_t mrg_launch_count(void) { return mrg::g_launches.load(); }

const char* mrg_version(void) { return "libmrg32k3a 0.1 (sm_103a)"; }

int mrg_seed_check(const uint32_t seed[6]) {
  if (!seed) return fail(MRG_EINVAL, "seed is NULL");
  if (!mrg::host::state_valid(seed))
    return fail(MRG_EINVAL, "invalid seed: need x1 words < m1, x2 words < m2, no all-zero triple");
  return MRG_OK;
}

int mrg_creator_advance(const uint32_t seed[6], uint64_t n_streams, uint32_t out[6]) {
  int rc = mrg_seed_check(seed);
  if (rc) return rc;
  if (!out) return fail(MRG_EINVAL, "out is NULL");
  if (n_streams > (1ull << 63)) return fail(MRG_ERANGE, "too many streams");
  uint32_t t[6];
  std::memcpy(t, seed, sizeof t);
  mrg::host::jump_pow2_multiple(t, n_streams, mrg::STREAM_LOG2);
  std::memcpy(out, t, sizeof t);
  return MRG_OK;
}

int mrg_create_streams(const uint32_t seed[6], uint64_t n, const mrg_streams* s,
                       uint32_t next_seed[6], void* stream) {
  int rc = mrg_seed_check(seed);
  if (rc) return rc;
  if (n > (1ull << 63)) return fail(MRG_ERANGE, "too many streams");
  if (n > 0 && !streams_ok(s)) return fail(MRG_EINVAL, "bad stream set");
  if (n > 0 && n > s->n) return fail(MRG_EINVAL, "n exceeds the stream set");
  if (n > 0) {
    if ((rc = ensure_device())) return rc;
    cudaError_t e = mrg::launch_create(seed, n, dev(s), cs(stream));
    if (e != cudaSuccess) return fail_cuda(e, "create_kernel");
  }
  if (next_seed) {
    uint32_t t[6];
    std::memcpy(t, seed, sizeof t);
    mrg::host::jump_pow2_multiple(t, n, mrg::STREAM_LOG2);
    std::memcpy(next_seed, t, sizeof t);
  }
  return MRG_OK;
}

int mrg_generate(const mrg_streams* s, uint64_t n, int dist, int dtype, double rate, void* out,
                 uint64_t ld, void* stream) {
  if (!streams_ok(s)) return fail(MRG_EINVAL, "bad stream set");
  bool pair_ok = (dist == MRG_RAW && dtype == MRG_U32) ||
                 ((dist == MRG_UNIFORM || dist == MRG_NORMAL || dist == MRG_EXPONENTIAL) &&
                  (dtype == MRG_F32 || dtype == MRG_F64));
  if (!pair_ok) return fail(MRG_EINVAL, "unsupported dist/dtype combination");
  if (dist == MRG_EXPONENTIAL && !(rate >= 0x1p-64 && rate <= 0x1p64))
    return fail(MRG_EINVAL, "exponential rate must lie in [2^-64, 2^64]");
  if (n == 0 || s->n == 0) return MRG_OK;
  if (!out) return fail(MRG_EINVAL, "out is NULL");
  if (ld < n) return fail(MRG_EINVAL, "ld < n");
  if (reinterpret_cast<uintptr_t>(out) % (dtype == MRG_F64 ? 8 : 4))
    return fail(MRG_EINVAL, "out is not aligned to its element size");
  if (n > (1ull << 62) || !extent_ok(s->n, ld, dtype == MRG_F64 ? 8 : 4))
    return fail(MRG_ERANGE, "size too large");
  int rc = ensure_device();
  if (rc) return rc;
  const mrg::GenConfig cfg = mrg::generate_config_for(dist, dtype, s->n, n);
  cudaError_t e = mrg::launch_generate(dev(s), n, dist, dtype, rate, out, ld, cfg, cs(stream));
  if (e != cudaSuccess) return fail_cuda(e, "generate_kernel");
  const uint64_t consumed = dist == MRG_NORMAL ? n + (n & 1) : n;
  e = mrg::launch_jump(s->cur, s->cur, nullptr, s->stride, s->n, consumed, 0, 0, cs(stream));
  if (e != cudaSuccess) return fail_cuda(e, "jump_kernel (advance)");
  return MRG_OK;
}

// ---------------------------------------------------------------------------
// Monte Carlo Fisher's exact test (Sec. 4)
// ---------------------------------------------------------------------------

}  // extern "C"

namespace {

constexpr uint64_t kFisherHeader = 1024;  // count (8 B), rows, cols (4 B each, <= 64)

// log(k!) for k = 0..n on the host (lgamma).  The table is shared and grown
// by replacement: a caller keeps its own reference while it copies, so a
// concurrent call that needs a longer table never frees one in use.
std::shared_ptr<const std::vector<double>> host_logfact(uint64_t n) {
  static std::mutex mu;
  static std::shared_ptr<const std::vector<double>> table;
  std::lock_guard<std::mutex> lk(mu);
  if (!table || table->size() <= n) {
    auto grown = std::make_shared<std::vector<double>>(table ? *table : std::vector<double>{});
    for (uint64_t k = grown->size(); k <= n; ++k) grown->push_back(std::lgamma((double)k + 1.0));
    table = grown;
  }
  return table;
}


}  // namespace

extern "C" {

int mrg_generate_matrix(const mrg_streams* s, int generator, uint64_t nrow, uint64_t ncol,
                        uint32_t gsize0, uint32_t gsize1, int dist, int dtype, double rate,
                        void* out, uint64_t ld, void* stream) {
  if (!streams_ok(s)) return fail(MRG_EINVAL, "bad stream set");
  if (generator != MRG_GEN_MRG32K3A && generator != MRG_GEN_MRG31K3P)
    return fail(MRG_EINVAL, "unknown generator");
  if (dist == MRG_NORMAL)
    return fail(MRG_EINVAL, "normals are not generated in the matrix layout (the paper pairs "
                            "two work items' streams there); use mrg_generate");
  const bool pair_ok = (dist == MRG_RAW && dtype == MRG_U32) ||
                       ((dist == MRG_UNIFORM || dist == MRG_EXPONENTIAL) &&
                        (dtype == MRG_F32 || dtype == MRG_F64));
  if (!pair_ok) return fail(MRG_EINVAL, "unsupported dist/dtype combination");
  if (dist == MRG_EXPONENTIAL && !(rate >= 0x1p-64 && rate <= 0x1p64))
    return fail(MRG_EINVAL, "exponential rate must lie in [2^-64, 2^64]");
  if (gsize0 == 0 || gsize1 == 0) return fail(MRG_EINVAL, "empty work-item grid");
  if ((uint64_t)gsize0 * gsize1 > s->n) return fail(MRG_EINVAL, "fewer streams than work items");
  if ((uint64_t)gsize0 * gsize1 > (1ull << 31)) return fail(MRG_ERANGE, "work-item grid too large");
  if (nrow == 0 || ncol == 0) return MRG_OK;
  if (!out) return fail(MRG_EINVAL, "out is NULL");
  if (ld < ncol) return fail(MRG_EINVAL, "ld < ncol");
  if (reinterpret_cast<uintptr_t>(out) % (dtype == MRG_F64 ? 8 : 4))
    return fail(MRG_EINVAL, "out is not aligned to its element size");
  if (!extent_ok(nrow, ld, dtype == MRG_F64 ? 8 : 4)) return fail(MRG_ERANGE, "size too large");
  int rc = ensure_device();
  if (rc) return rc;
  cudaError_t e = mrg::launch_matrix(generator == MRG_GEN_MRG31K3P, s->cur, s->stride, nrow, ncol,
                                     gsize0, gsize1, dist, dtype, rate, out, ld, cs(stream));
  if (e != cudaSuccess) return fail_cuda(e, "matrix_kernel");
  return MRG_OK;
}

int mrg_fill_u32(void* out, uint64_t n_words, uint32_t value, void* stream) {
  if (n_words == 0) return MRG_OK;
  if (!out || reinterpret_cast<uintptr_t>(out) % 32 || n_words % 8)
    return fail(MRG_EINVAL, "out must be 32-byte aligned and n_words a multiple of 8");
  int rc = ensure_device();
  if (rc) return rc;
  cudaError_t e = mrg::launch_fill(out, n_words / 8, value, cs(stream));
  if (e != cudaSuccess) return fail_cuda(e, "fill_kernel");
  return MRG_OK;
}

uint64_t mrg_fisher_scratch_bytes(uint64_t n_total) {
  return kFisherHeader + 8 * (n_total + 1);
}

int mrg_fisher_sim(const mrg_streams* s, const int32_t* table, uint32_t I, uint32_t J,
                   uint64_t B, void* scratch, uint64_t scratch_bytes, double* stats,
                   uint64_t* count, double* threshold, double* p_value, void* stream) {
  if (!streams_ok(s) || s->n == 0) return fail(MRG_EINVAL, "bad stream set");
  if (!table || !count) return fail(MRG_EINVAL, "table/count is NULL");
  if (I < 2 || J < 2 || I > mrg::kFisherMaxDim || J > mrg::kFisherMaxDim)
    return fail(MRG_EINVAL, "table must be I x J with 2 <= I, J <= 64");
  int32_t rows[mrg::kFisherMaxDim] = {}, cols[mrg::kFisherMaxDim] = {};
  int64_t total = 0;
  for (uint32_t i = 0; i < I; ++i)
    for (uint32_t j = 0; j < J; ++j) {
      const int32_t v = table[(size_t)i * J + j];
      if (v < 0) return fail(MRG_EINVAL, "negative table entry");
      rows[i] += v;
      cols[j] += v;
      total += v;
      if (total >= (1 << 24)) return fail(MRG_ERANGE, "table total not below 2^24");
    }
  if (!scratch || reinterpret_cast<uintptr_t>(scratch) % 256 ||
      scratch_bytes < mrg_fisher_scratch_bytes((uint64_t)total))
    return fail(MRG_EINVAL, "scratch NULL, not 256-byte aligned or smaller than "
                            "mrg_fisher_scratch_bytes(total)");
  if (stats && reinterpret_cast<uintptr_t>(stats) % 8) return fail(MRG_EINVAL, "stats misaligned");
  int rc = ensure_device();
  if (rc) return rc;
  const std::shared_ptr<const std::vector<double>> lfp = host_logfact((uint64_t)total);
  const std::vector<double>& lf = *lfp;
  // the observed statistic, -sum log(n_ij!) row by row; "at or below" it is
  // taken with a relative allowance of 64 ulp, so that a table whose
  // statistic equals it mathematically counts whatever its rounding
  double tobs = 0.0;
  for (uint32_t i = 0; i < I; ++i)
    for (uint32_t j = 0; j < J; ++j) tobs -= lf[table[(size_t)i * J + j]];
  const double thr = tobs / (1.0 + 64.0 * DBL_EPSILON);
  if (threshold) *threshold = thr;
  char* sc = static_cast<char*>(scratch);
  unsigned long long* d_count = reinterpret_cast<unsigned long long*>(sc);
  int32_t* d_rows = reinterpret_cast<int32_t*>(sc + 256);
  int32_t* d_cols = reinterpret_cast<int32_t*>(sc + 512);
  double* d_lf = reinterpret_cast<double*>(sc + kFisherHeader);
  cudaStream_t st = cs(stream);
  cudaError_t e = cudaMemsetAsync(d_count, 0, 8, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_rows, rows, 4 * I, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_cols, cols, 4 * J, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_lf, lf.data(), 8 * ((uint64_t)total + 1), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail_cuda(e, "copying the Fisher tables");
  e = mrg::launch_fisher(dev(s), d_rows, d_cols, I, J, (int32_t)total, d_lf, B, thr, d_count,
                         stats, st);
  if (e != cudaSuccess) return fail_cuda(e, "fisher_kernel");
  unsigned long long h = 0;
  e = cudaMemcpyAsync(&h, d_count, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail_cuda(e, "reading the Fisher count");
  *count = h;
  // the simulated p-value of Sec. 4: the observed table counts as one of
  // B + 1 equally likely tables
  if (p_value) *p_value = (1.0 + (double)h) / ((double)B + 1.0);
  return MRG_OK;
}

// ---------------------------------------------------------------------------
// MRG31k3p, the paper's own generator
// ---------------------------------------------------------------------------

int mrg31k3p_seed_check(const uint32_t seed[6]) {
  if (!seed) return fail(MRG_EINVAL, "seed is NULL");
  if (!mrg::host::g31::state_valid(seed))
    return fail(MRG_EINVAL, "invalid MRG31k3p seed: need x1 words < 2^31 - 1, x2 words < "
                            "2^31 - 21069, no all-zero triple");
  return MRG_OK;
}

int mrg31k3p_creator_advance(const uint32_t seed[6], uint64_t n_streams, uint32_t out[6]) {
  int rc = mrg31k3p_seed_check(seed);
  if (rc) return rc;
  if (!out) return fail(MRG_EINVAL, "out is NULL");
  if (n_streams > (1ull << 63)) return fail(MRG_ERANGE, "too many streams");
  uint32_t t[6];
  std::memcpy(t, seed, sizeof t);
  mrg::host::g31::jump_pow2_multiple(t, n_streams, mrg::host::g31::kStreamLog2);
  std::memcpy(out, t, sizeof t);
  return MRG_OK;
}

int mrg31k3p_create_streams(const uint32_t seed[6], uint64_t n, const mrg_streams* s,
                            uint32_t next_seed[6], void* stream) {
  int rc = mrg31k3p_seed_check(seed);
  if (rc) return rc;
  if (n > (1ull << 63)) return fail(MRG_ERANGE, "too many streams");
  if (n > 0 && !streams_ok(s)) return fail(MRG_EINVAL, "bad stream set");
  if (n > 0 && n > s->n) return fail(MRG_EINVAL, "n exceeds the stream set");
  if (n > 0) {
    if ((rc = ensure_device())) return rc;
    cudaError_t e = mrg::launch_create31(seed, n, dev(s), cs(stream));
    if (e != cudaSuccess) return fail_cuda(e, "create31_kernel");
  }
  if (next_seed) {
    uint32_t t[6];
    std::memcpy(t, seed, sizeof t);
    mrg::host::g31::jump_pow2_multiple(t, n, mrg::host::g31::kStreamLog2);
    std::memcpy(next_seed, t, sizeof t);
  }
  return MRG_OK;
}

int mrg31k3p_generate(const mrg_streams* s, uint64_t n, int dist, int dtype, double rate,
                      void* out, uint64_t ld, void* stream) {
  if (!streams_ok(s)) return fail(MRG_EINVAL, "bad stream set");
  bool pair_ok = (dist == MRG_RAW && dtype == MRG_U32) ||
                 ((dist == MRG_UNIFORM || dist == MRG_NORMAL || dist == MRG_EXPONENTIAL) &&
                  (dtype == MRG_F32 || dtype == MRG_F64));
  if (!pair_ok) return fail(MRG_EINVAL, "unsupported dist/dtype combination");
  if (dist == MRG_EXPONENTIAL && !(rate >= 0x1p-64 && rate <= 0x1p64))
    return fail(MRG_EINVAL, "exponential rate must lie in [2^-64, 2^64]");
  if (n == 0 || s->n == 0) return MRG_OK;
  if (!out) return fail(MRG_EINVAL, "out is NULL");
  if (ld < n) return fail(MRG_EINVAL, "ld < n");
  if (reinterpret_cast<uintptr_t>(out) % (dtype == MRG_F64 ? 8 : 4))
    return fail(MRG_EINVAL, "out is not aligned to its element size");
  if (n > (1ull << 62) || !extent_ok(s->n, ld, dtype == MRG_F64 ? 8 : 4))
    return fail(MRG_ERANGE, "size too large");
  int rc = ensure_device();
  if (rc) return rc;
  cudaError_t e = mrg::launch_generate31(dev(s), n, dist, dtype, rate, out, ld, mrg::GenConfig{},
                                         cs(stream));
  if (e != cudaSuccess) return fail_cuda(e, "generate31_kernel");
  const uint64_t consumed = dist == MRG_NORMAL ? n + (n & 1) : n;
  e = mrg::launch_jump31(s->cur, s->stride, s->n, consumed, cs(stream));
  if (e != cudaSuccess) return fail_cuda(e, "jump31_kernel (advance)");
  return MRG_OK;
}

int mrg31k3p_skip(const mrg_streams* s, uint64_t k, void* stream) {
  if (!streams_ok(s)) return fail(MRG_EINVAL, "bad stream set");
  if (s->n == 0 || k == 0) return MRG_OK;
  int rc = ensure_device();
  if (rc) return rc;
  cudaError_t e = mrg::launch_jump31(s->cur, s->stride, s->n, k, cs(stream));
  if (e != cudaSuccess) return fail_cuda(e, "jump31_kernel (skip)");
  return MRG_OK;
}

int mrg_generate_host(const mrg_streams* s, uint64_t n, int dist, int dtype, double rate,
                      void* out_host, uint64_t ld, void* scratch, uint64_t scratch_bytes,
                      void* stream) {
  if (!streams_ok(s)) return fail(MRG_EINVAL, "bad stream set");
  if (n == 0 || s->n == 0) return MRG_OK;
  if (!out_host || !scratch) return fail(MRG_EINVAL, "out_host/scratch is NULL");
  if (ld < n) return fail(MRG_EINVAL, "ld < n");
  const uint64_t es = dtype == MRG_F64 ? 8 : 4;
  const uint64_t row = n * es;
  const uint64_t half = (scratch_bytes / 2) & ~(uint64_t)255;
  if (half < row) return fail(MRG_EINVAL, "scratch smaller than two stream rows");
  const uint64_t rows = half / row;
  int rc = ensure_device();
  if (rc) return rc;
  // per-device copy stream and ping-pong events
  static std::mutex mu;
  static cudaStream_t copy_st[64];
  static cudaEvent_t gen_ev[64][2], copy_ev[64][2];
  int devi = 0;
  cudaGetDevice(&devi);
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!copy_st[devi]) {
      cudaError_t e = cudaStreamCreateWithFlags(&copy_st[devi], cudaStreamNonBlocking);
      for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaEventCreateWithFlags(&gen_ev[devi][b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&copy_ev[devi][b], cudaEventDisableTiming);
      }
      if (e != cudaSuccess) return fail_cuda(e, "creating copy stream/events");
    }
  }
  cudaStream_t gs = cs(stream), ks = copy_st[devi];
  char* sc = reinterpret_cast<char*>(scratch);
  char* ho = reinterpret_cast<char*>(out_host);
  uint64_t c = 0;
  for (uint64_t r0 = 0; r0 < s->n; r0 += rows, ++c) {
    const int b = (int)(c & 1);
    const uint64_t m = std::min<uint64_t>(rows, s->n - r0);
    mrg_streams v{s->cur + r0, s->start + r0, s->sub + r0, m, s->stride};
    cudaError_t e = cudaSuccess;
    if (c >= 2) e = cudaStreamWaitEvent(gs, copy_ev[devi][b], 0);  // half b drained
    if (e != cudaSuccess) return fail_cuda(e, "cudaStreamWaitEvent");
    rc = mrg_generate(&v, n, dist, dtype, rate, sc + b * half, n, stream);
    if (rc) return rc;
    e = cudaEventRecord(gen_ev[devi][b], gs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ks, gen_ev[devi][b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(ho + r0 * ld * es, ld * es, sc + b * half, row, row, m,
                            cudaMemcpyDeviceToHost, ks);
    if (e == cudaSuccess) e = cudaEventRecord(copy_ev[devi][b], ks);
    if (e != cudaSuccess) return fail_cuda(e, "copy to host");
  }
  cudaError_t e = cudaStreamSynchronize(ks);
  if (e == cudaSuccess) e = cudaStreamSynchronize(gs);
  if (e != cudaSuccess) return fail_cuda(e, "cudaStreamSynchronize (generate_host)");
  return MRG_OK;
}

int mrg_transform(const uint32_t* z, uint64_t n, int dist, int dtype, double rate, void* out,
                  void* stream) {
  bool pair_ok = (dist == MRG_UNIFORM || dist == MRG_NORMAL || dist == MRG_EXPONENTIAL) &&
                 (dtype == MRG_F32 || dtype == MRG_F64);
  if (!pair_ok) return fail(MRG_EINVAL, "unsupported dist/dtype combination");
  if (dist == MRG_EXPONENTIAL && !(rate >= 0x1p-64 && rate <= 0x1p64))
    return fail(MRG_EINVAL, "exponential rate must lie in [2^-64, 2^64]");
  if (n == 0) return MRG_OK;
  if (!z || !out) return fail(MRG_EINVAL, "z/out is NULL");
  if (reinterpret_cast<uintptr_t>(out) % (dtype == MRG_F64 ? 8 : 4) ||
      reinterpret_cast<uintptr_t>(z) % 4)
    return fail(MRG_EINVAL, "misaligned pointer");
  int rc = ensure_device();
  if (rc) return rc;
  cudaError_t e = mrg::launch_transform(z, n, dist, dtype, rate, out, cs(stream));
  if (e != cudaSuccess) return fail_cuda(e, "transform_kernel");
  return MRG_OK;
}

int mrg_skip(const mrg_streams* s, uint64_t k_hi, uint64_t k_lo, void* stream) {
  if (!streams_ok(s)) return fail(MRG_EINVAL, "bad stream set");
  if (s->n == 0 || (k_hi == 0 && k_lo == 0)) return MRG_OK;
  int rc = ensure_device();
  if (rc) return rc;
  cudaError_t e = mrg::launch_jump(s->cur, s->cur, nullptr, s->stride, s->n, k_lo, k_hi, 0, cs(stream));
  if (e != cudaSuccess) return fail_cuda(e, "jump_kernel (skip)");
  return MRG_OK;
}

int mrg_substream_next(const mrg_streams* s, void* stream) {
  if (!streams_ok(s)) return fail(MRG_EINVAL, "bad stream set");
  if (s->n == 0) return MRG_OK;
  int rc = ensure_device();
  if (rc) return rc;
  cudaError_t e = mrg::launch_jump(s->sub, s->sub, s->cur, s->stride, s->n, 1, 0,
                                   mrg::SUBSTREAM_LOG2, cs(stream));
  if (e != cudaSuccess) return fail_cuda(e, "jump_kernel (substream)");
  return MRG_OK;
}

int mrg_reset_substream(const mrg_streams* s, void* stream) {
  if (!streams_ok(s)) return fail(MRG_EINVAL, "bad stream set");
  if (s->n == 0) return MRG_OK;
  int rc = ensure_device();
  if (rc) return rc;
  cudaError_t e = mrg::launch_jump(s->sub, s->cur, nullptr, s->stride, s->n, 0, 0, 0, cs(stream));
  if (e != cudaSuccess) return fail_cuda(e, "jump_kernel (reset substream)");
  return MRG_OK;
}

int mrg_reset_stream(const mrg_streams* s, void* stream) {
  if (!streams_ok(s)) return fail(MRG_EINVAL, "bad stream set");
  if (s->n == 0) return MRG_OK;
  int rc = ensure_device();
  if (rc) return rc;
  cudaError_t e = mrg::launch_jump(s->start, s->cur, s->sub, s->stride, s->n, 0, 0, 0, cs(stream));
  if (e != cudaSuccess) return fail_cuda(e, "jump_kernel (reset stream)");
  return MRG_OK;
}

int mrg_get_state(const mrg_streams* s, uint32_t* host, void* stream) {
  if (!streams_ok(s)) return fail(MRG_EINVAL, "bad stream set");
  if (s->n == 0) return MRG_OK;
  if (!host) return fail(MRG_EINVAL, "host buffer is NULL");
  const uint32_t* src[3] = {s->cur, s->start, s->sub};
  for (int a = 0; a < 3; ++a) {
    cudaError_t e = cudaMemcpy2DAsync(host + (size_t)a * 6 * s->n, s->n * 4, src[a], s->stride * 4,
                                      s->n * 4, 6, cudaMemcpyDeviceToHost, cs(stream));
    if (e != cudaSuccess) return fail_cuda(e, "cudaMemcpy2DAsync (get_state)");
  }
  cudaError_t e = cudaStreamSynchronize(cs(stream));
  if (e != cudaSuccess) return fail_cuda(e, "cudaStreamSynchronize (get_state)");
  return MRG_OK;
}

int mrg_set_state(const mrg_streams* s, const uint32_t* host, void* stream) {
  if (!streams_ok(s)) return fail(MRG_EINVAL, "bad stream set");
  if (s->n == 0) return MRG_OK;
  if (!host) return fail(MRG_EINVAL, "host buffer is NULL");
  const uint64_t n = s->n;
  for (int a = 0; a < 3; ++a)
    for (uint64_t i = 0; i < n; ++i) {
      uint32_t st[6];
      for (int k = 0; k < 6; ++k) st[k] = host[((size_t)a * 6 + k) * n + i];
      if (!mrg::host::state_valid(st)) {
        char buf[96];
        std::snprintf(buf, sizeof buf, "invalid state (array %d, stream %llu)", a,
                      (unsigned long long)i);
        return fail(MRG_EINVAL, buf);
      }
    }
  uint32_t* dst[3] = {s->cur, s->start, s->sub};
  for (int a = 0; a < 3; ++a) {
    cudaError_t e = cudaMemcpy2DAsync(dst[a], s->stride * 4, host + (size_t)a * 6 * n, n * 4, n * 4,
                                      6, cudaMemcpyHostToDevice, cs(stream));
    if (e != cudaSuccess) return fail_cuda(e, "cudaMemcpy2DAsync (set_state)");
  }
  cudaError_t e = cudaStreamSynchronize(cs(stream));
  if (e != cudaSuccess) return fail_cuda(e, "cudaStreamSynchronize (set_state)");
  return MRG_OK;
}

int mrg_fused_pi_normsum(const mrg_streams* s, uint64_t draws, int64_t* count, double* sum,
                         void* stream) {
  if (!streams_ok(s)) return fail(MRG_EINVAL, "bad stream set");
  if (s->n == 0) return MRG_OK;
  if (!count || !sum) return fail(MRG_EINVAL, "count/sum is NULL");
  int rc = ensure_device();
  if (rc) return rc;
  cudaError_t e = mrg::launch_fused(dev(s), (draws + 1) / 2, count, sum, cs(stream));
  if (e != cudaSuccess) return fail_cuda(e, "fused_kernel");
  return MRG_OK;
}

// ---------------------------------------------------------------------------
// Batched requests
// ---------------------------------------------------------------------------

}  // extern "C"

namespace mrg {

// One request of a batch (mrg_batch_run, mrg_batch_run_static): checks it
// against a stream set of ns streams and writes its device record under the
// tiling (seg_min, seg_max, target); *tiles receives its warp-tile count.
int prepare_request(const mrg_request& q, uint64_t ns, uint32_t seg_min, uint32_t seg_max,
                    uint64_t target, BatchReqHost* h, uint64_t* tiles) {
  const bool pair_ok = (q.dist == MRG_RAW && q.dtype == MRG_U32) ||
                       ((q.dist == MRG_UNIFORM || q.dist == MRG_NORMAL ||
                         q.dist == MRG_EXPONENTIAL) && (q.dtype == MRG_F32 || q.dtype == MRG_F64));
  if (!pair_ok) return fail(MRG_EINVAL, "request with unsupported dist/dtype");
  if (q.stream >= ns) return fail(MRG_EINVAL, "request stream index out of range");
  if (q.substream >= (1ull << 51)) return fail(MRG_ERANGE, "substream index >= 2^51");
  const uint64_t draws = q.dist == MRG_NORMAL ? q.n + (q.n & 1) : q.n;
  if (q.offset > (1ull << 62) || draws > (1ull << 62) || q.offset + draws > (1ull << 62))
    return fail(MRG_ERANGE, "offset + draws too large");
  if (q.n > 0 && (!q.out || reinterpret_cast<uintptr_t>(q.out) % 32))
    return fail(MRG_EINVAL, "request output NULL or not 32-byte aligned");
  if (q.dist == MRG_EXPONENTIAL && !(q.rate >= 0x1p-64 && q.rate <= 0x1p64))
    return fail(MRG_EINVAL, "exponential rate must lie in [2^-64, 2^64]");
  const uint32_t L = tiled_seg_len(q.n, seg_min, seg_max, target);
  const uint64_t nseg = (q.n + L - 1) / L;
  if (nseg > 0xFFFFFFFFull) return fail(MRG_ERANGE, "request has more than 2^32 segments");
  h->out = reinterpret_cast<uint64_t>(q.out);
  h->n = q.n;
  h->off = q.offset;
  h->sub = q.substream;
  h->stream = q.stream;
  h->dist = (uint32_t)q.dist;
  h->dtype = (uint32_t)q.dtype;
  const double ir = q.dist == MRG_EXPONENTIAL ? -1.0 / q.rate : 0.0;
  h->ir_hi = (float)ir;
  h->ir_lo = (float)(ir - (double)h->ir_hi);
  h->L = L;
  h->nseg = (uint32_t)nseg;
  *tiles = (nseg + 31) / 32;
  return MRG_OK;
}

}  // namespace mrg

// Host staging of one run's tables (pinned).  A batch object has two, used in
// turn, so that the tables of the next run are built while the GPU still
// copies or runs the previous one.
struct BatchStaging {
  mrg::VariantRangeHost* ranges = nullptr;  // kVariants tile ranges
  mrg::BatchReqHost* reqs = nullptr;
  mrg::BatchTileHost* tiles = nullptr;
  cudaEvent_t copied = nullptr;             // the copies out of this staging are done
  bool used = false;
};

struct mrg_batch {
  int device = 0;
  mrg_streams s{};
  uint32_t max_req = 0;
  uint64_t max_tiles = 0;
  uint64_t last_tiles = 0;
  void* d_ranges = nullptr;
  unsigned long long* d_counters = nullptr;
  void* d_reqs = nullptr;
  void* d_tiles = nullptr;
  BatchStaging stage[2];
  int next_stage = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;               // end of the last run's kernels
  bool ran = false;
  mrg_tiling tiling{8, 256, 32};
  std::vector<uint32_t> order;  // request order of the tile table (host scratch)
};

namespace {

void batch_free(mrg_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->done) cudaEventDestroy(b->done);
  cudaFree(b->d_ranges);
  cudaFree(b->d_counters);
  cudaFree(b->d_reqs);
  cudaFree(b->d_tiles);
  for (BatchStaging& st : b->stage) {
    if (st.copied) cudaEventDestroy(st.copied);
    cudaFreeHost(st.ranges);
    cudaFreeHost(st.reqs);
    cudaFreeHost(st.tiles);
  }
  delete b;
}

bool tiling_ok(const mrg_tiling& t) {
  return t.seg_min >= 8 && t.seg_min % 8 == 0 && t.seg_max % 8 == 0 && t.seg_min <= t.seg_max &&
         t.seg_max <= (1u << 20) && t.target_segments >= 1;
}

// Validates the requests and writes the request, tile and range tables of
// one run into staging S under tiling `t`; *ntiles receives the tile count.
int build_batch_tables(mrg_batch* b, BatchStaging& S, const mrg_request* reqs, uint32_t nreq,
                       const mrg_tiling& t, uint64_t* ntiles) {
  uint64_t nt = 0;
  for (uint32_t r = 0; r < nreq; ++r) {
    uint64_t tiles = 0;
    const int rc = mrg::prepare_request(reqs[r], b->s.n, t.seg_min, t.seg_max, t.target_segments,
                                        &S.reqs[r], &tiles);
    if (rc) return rc;
    nt += tiles;
    if (nt > b->max_tiles) return fail(MRG_ERANGE, "more tiles than the batch holds");
  }
  // Tile order: grouped by output variant (one persistent kernel per variant
  // runs its group), and within a variant by segment length, longest first,
  // so that the last tiles claimed are the shortest (a short tail).
  auto& order = b->order;
  order.resize(nreq);
  for (uint32_t r = 0; r < nreq; ++r) order[r] = r;
  auto rank = [&](uint32_t r) { return mrg::kVariantRank[S.reqs[r].dist * 4 + S.reqs[r].dtype]; };
  std::sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
    const int rx = rank(x), ry = rank(y);
    if (rx != ry) return rx < ry;
    if (S.reqs[x].L != S.reqs[y].L) return S.reqs[x].L > S.reqs[y].L;
    return x < y;
  });
  for (int v = 0; v < mrg::kVariants; ++v) S.ranges[v] = mrg::VariantRangeHost{0, 0};
  uint64_t k = 0;
  int v = 0;
  for (uint32_t r : order) {
    const int rv = rank(r);
    for (; v < rv; ++v) S.ranges[v + 1].begin = S.ranges[v + 1].end = k;
    const uint64_t tiles = ((uint64_t)S.reqs[r].nseg + 31) / 32;
    for (uint64_t j = 0; j < tiles; ++j) S.tiles[k++] = mrg::BatchTileHost{r, (uint32_t)(32 * j)};
    S.ranges[rv].end = k;
  }
  for (; v + 1 < mrg::kVariants; ++v) S.ranges[v + 1].begin = S.ranges[v + 1].end = k;
  *ntiles = nt;
  return MRG_OK;
}

// Tile count of the requests under tiling t (no table is written).
uint64_t count_tiles(const mrg_request* reqs, uint32_t nreq, const mrg_tiling& t) {
  uint64_t nt = 0;
  for (uint32_t r = 0; r < nreq; ++r) {
    const uint32_t L = mrg::tiled_seg_len(reqs[r].n, t.seg_min, t.seg_max, t.target_segments);
    nt += ((reqs[r].n + L - 1) / L + 31) / 32;
  }
  return nt;
}

}  // namespace

extern "C" {

int mrg_batch_create(const mrg_streams* s, uint32_t max_requests, uint64_t max_tiles,
                     mrg_batch** out, void* stream) {
  if (!out) return fail(MRG_EINVAL, "out is NULL");
  *out = nullptr;
  if (!streams_ok(s)) return fail(MRG_EINVAL, "bad stream set");
  if (max_requests == 0 || max_tiles == 0) return fail(MRG_EINVAL, "empty batch capacity");
  if (max_tiles > (1ull << 32)) return fail(MRG_ERANGE, "max_tiles too large");
  int rc = ensure_device();
  if (rc) return rc;
  mrg_batch* b = new mrg_batch;
  cudaGetDevice(&b->device);
  b->s = *s;
  b->max_req = max_requests;
  b->max_tiles = max_tiles;
  const size_t rb = sizeof(mrg::BatchReqHost) * max_requests;
  const size_t tb = sizeof(mrg::BatchTileHost) * max_tiles;
  const size_t hb = sizeof(mrg::VariantRangeHost) * mrg::kVariants;
  const size_t cb = sizeof(unsigned long long) * mrg::kBatchCounterStride * mrg::kVariants;
  cudaError_t e = cudaMalloc(&b->d_ranges, hb);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_counters, cb);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_reqs, rb);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_tiles, tb);
  for (BatchStaging& st : b->stage) {
    if (e == cudaSuccess) e = cudaMallocHost((void**)&st.ranges, hb);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&st.reqs, rb);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&st.tiles, tb);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st.copied, cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    batch_free(b);
    return fail_cuda(e, "allocating batch tables");
  }
  // Capture [claim counters = 0, one persistent kernel per variant] once.
  // Each run copies its tables into the device tables before launching it.
  cudaStream_t cap = nullptr;
  e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counters, 0, cb, cap);
  for (int v = 0; v < mrg::kVariants && e == cudaSuccess; ++v)
    e = mrg::launch_batch_variant(v, b->d_ranges, b->d_counters, b->d_reqs, b->d_tiles, s->start,
                                  s->stride, cap);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cap, &g);
  if (e == cudaSuccess) e = e2;
  b->graph = g;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (cap) cudaStreamDestroy(cap);
  (void)stream;
  if (e != cudaSuccess) {
    batch_free(b);
    return fail_cuda(e, "capturing the batch graph");
  }
  *out = b;
  return MRG_OK;
}

int mrg_batch_run(mrg_batch* b, const mrg_request* reqs, uint32_t nreq, void* stream) {
  if (!b) return fail(MRG_EINVAL, "batch is NULL");
  if (nreq > 0 && !reqs) return fail(MRG_EINVAL, "reqs is NULL");
  if (nreq > b->max_req) return fail(MRG_ERANGE, "more requests than the batch holds");
  BatchStaging& S = b->stage[b->next_stage];
  if (S.used) {  // the copies out of this staging (two runs ago) must be done
    cudaError_t e = cudaEventSynchronize(S.copied);
    if (e != cudaSuccess) return fail_cuda(e, "waiting for an earlier batch's table copies");
  }
  uint64_t nt = 0;
  int rc = build_batch_tables(b, S, reqs, nreq, b->tiling, &nt);
  if (rc) return rc;
  cudaStream_t st = cs(stream);
  cudaError_t e = cudaSuccess;
  // the device tables are shared by all runs: the previous run's kernels
  // must be done with them, whatever stream it ran on
  if (b->ran) e = cudaStreamWaitEvent(st, b->done, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_ranges, S.ranges, sizeof(mrg::VariantRangeHost) * mrg::kVariants,
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nreq)
    e = cudaMemcpyAsync(b->d_reqs, S.reqs, sizeof(mrg::BatchReqHost) * nreq, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nt)
    e = cudaMemcpyAsync(b->d_tiles, S.tiles, sizeof(mrg::BatchTileHost) * nt, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(S.copied, st);
  if (e != cudaSuccess) return fail_cuda(e, "copying the batch tables");
  S.used = true;
  b->next_stage ^= 1;
  b->last_tiles = nt;
  e = cudaGraphLaunch(b->exec, st);
  if (e == cudaSuccess) e = cudaEventRecord(b->done, st);
  if (e != cudaSuccess) return fail_cuda(e, "cudaGraphLaunch (batch)");
  mrg::g_launches.fetch_add(mrg::kVariants, std::memory_order_relaxed);
  b->ran = true;
  return MRG_OK;
}

int mrg_batch_set_tiling(mrg_batch* b, const mrg_tiling* t) {
  if (!b) return fail(MRG_EINVAL, "batch is NULL");
  const mrg_tiling d{8, 256, 32};
  if (t && !tiling_ok(*t)) return fail(MRG_EINVAL, "tiling outside its ranges");
  b->tiling = t ? *t : d;
  return MRG_OK;
}

int mrg_batch_get_tiling(const mrg_batch* b, mrg_tiling* t) {
  if (!b || !t) return fail(MRG_EINVAL, "NULL argument");
  *t = b->tiling;
  return MRG_OK;
}

int mrg_batch_tune(mrg_batch* b, const mrg_request* reqs, uint32_t nreq, uint32_t reps,
                   mrg_batch_tune_entry* results, uint32_t max_results, uint32_t* n_results,
                   mrg_tiling* best, void* stream) {
  if (n_results) *n_results = 0;
  if (!b) return fail(MRG_EINVAL, "batch is NULL");
  if (nreq == 0 || !reqs) return fail(MRG_EINVAL, "no requests to tune on");
  if (max_results && !results) return fail(MRG_EINVAL, "results is NULL");
  if (nreq > b->max_req) return fail(MRG_ERANGE, "more requests than the batch holds");
  if (reps == 0) reps = 3;
  if (reps > 100) reps = 100;
  std::vector<mrg_tiling> cand{b->tiling};
  for (uint32_t lo : {8u, 64u})
    for (uint32_t hi : {128u, 256u, 512u, 2048u})
      for (uint64_t tg : {32ull, 256ull, 2048ull}) {
        if (lo > hi) continue;
        const mrg_tiling t{lo, hi, tg};
        if (t.seg_min == b->tiling.seg_min && t.seg_max == b->tiling.seg_max &&
            t.target_segments == b->tiling.target_segments)
          continue;
        if (count_tiles(reqs, nreq, t) <= b->max_tiles) cand.push_back(t);
      }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return fail_cuda(e, "cudaEventCreate (batch tune)");
  }
  const mrg_tiling keep = b->tiling;
  float best_ms = 0.0f;
  size_t best_i = 0;
  uint32_t nr = 0;
  int rc = MRG_OK;
  for (size_t i = 0; i < cand.size() && rc == MRG_OK; ++i) {
    b->tiling = cand[i];
    float ms = 0.0f;
    rc = mrg_batch_run(b, reqs, nreq, stream);  // warm-up (and validation)
    const uint64_t tiles = b->last_tiles;
    if (rc == MRG_OK) {
      // replays reuse the device tables the warm-up copied (the graph zeroes
      // the claim counters itself)
      e = cudaEventRecord(e0, cs(stream));
      for (uint32_t r = 0; r < reps && e == cudaSuccess; ++r) {
        e = cudaGraphLaunch(b->exec, cs(stream));
        if (e == cudaSuccess) mrg::g_launches.fetch_add(mrg::kVariants, std::memory_order_relaxed);
      }
      if (e == cudaSuccess) e = cudaEventRecord(e1, cs(stream));
      if (e == cudaSuccess) e = cudaEventRecord(b->done, cs(stream));
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) rc = fail_cuda(e, "timing a tiling (batch tune)");
    }
    if (rc != MRG_OK) break;
    ms /= (float)reps;
    if (nr < max_results) results[nr++] = mrg_batch_tune_entry{cand[i], tiles, ms};
    if (i == 0 || ms < best_ms) {
      best_ms = ms;
      best_i = i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != MRG_OK) {
    b->tiling = keep;
    return rc;
  }
  b->tiling = cand[best_i];
  if (best) *best = cand[best_i];
  if (n_results) *n_results = nr;
  return MRG_OK;
}

uint64_t mrg_batch_last_tiles(const mrg_batch* b) { return b ? b->last_tiles : 0; }

int mrg_batch_destroy(mrg_batch* b) {
  if (!b) return MRG_OK;
  if (b->ran) cudaEventSynchronize(b->done);
  batch_free(b);
  return MRG_OK;
}

int mrg_batch_run_plain(const mrg_streams* s, const mrg_request* reqs, uint32_t nreq,
                        void* stream) {
  if (!streams_ok(s)) return fail(MRG_EINVAL, "bad stream set");
  if (nreq > 0 && !reqs) return fail(MRG_EINVAL, "reqs is NULL");
  for (uint32_t r = 0; r < nreq; ++r) {  // the batch's own checks, nothing launched yet
    mrg::BatchReqHost h;
    uint64_t tiles = 0;
    const int rc = mrg::prepare_request(reqs[r], s->n, 8, 2048, 32, &h, &tiles);
    if (rc) return rc;
  }
  int rc = ensure_device();
  if (rc) return rc;
  cudaStream_t st = cs(stream);
  for (uint32_t r = 0; r < nreq; ++r) {
    const mrg_request& q = reqs[r];
    if (q.n == 0) continue;
    // cur of the request's stream <- start * A^(substream 2^76 + offset)
    const unsigned __int128 e =
        ((unsigned __int128)q.substream << mrg::SUBSTREAM_LOG2) + (unsigned __int128)q.offset;
    cudaError_t ce = mrg::launch_jump(s->start + q.stream, s->cur + q.stream, nullptr, s->stride, 1,
                                      (uint64_t)e, (uint64_t)(e >> 64), 0, st);
    if (ce != cudaSuccess) return fail_cuda(ce, "jump_kernel (request position)");
    const mrg::DevStreams one{s->cur + q.stream, s->start + q.stream, s->sub + q.stream, 1,
                              s->stride};
    const mrg::GenConfig cfg = mrg::generate_config_for(q.dist, q.dtype, 1, q.n);
    ce = mrg::launch_generate(one, q.n, q.dist, q.dtype, q.rate, q.out, q.n, cfg, st);
    if (ce != cudaSuccess) return fail_cuda(ce, "generate_kernel (plain request)");
  }
  return MRG_OK;
}

}  // extern "C"
