// tune.cu -- autotuner of the generate kernel's launch shape.
//
// The launch shape of generate_kernel -- draws per lane segment, threads per
// block, the per-lane store width and the blocks per SM the grid is sized
// for -- changes only how the work is cut, never the output: every segment
// starts with a jump to its absolute offset.  The tuner times a set of
// candidate shapes with CUDA events on the caller's stream, keeps the fastest
// in a per-device table keyed by (distribution, output type, size class), and
// mrg_generate then launches with it.  The size class is the pair
// (bit length of n_streams * n, bit length of n), so a tuned shape is reused
// for calls of about the same size and shape.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/mrg32k3a.h"
#include "internal.h"

namespace mrg {
namespace {

int bitlen(uint64_t v) { return v ? 64 - __builtin_clzll(v) : 0; }

using Key = std::tuple<int, int, int, int, int>;  // device, dist, dtype, bitlen(ns*n), bitlen(n)

std::mutex g_mu;
std::map<Key, GenConfig> g_table;

Key key_for(int dev, int dist, int dtype, uint64_t ns, uint64_t n) {
  const unsigned __int128 tot = (unsigned __int128)ns * n;
  const uint64_t t = tot >> 64 ? ~0ull : (uint64_t)tot;
  return Key{dev, dist, dtype, bitlen(t), bitlen(n)};
}

GenConfig from_abi(const mrg_launch_config& c) {
  GenConfig g;
  g.seg_len = c.seg_len;
  g.block = c.block ? (int)c.block : 256;
  g.vec_bytes = c.vec_bytes ? (int)c.vec_bytes : 32;
  g.per_sm = (int)c.blocks_per_sm;
  return g;
}

mrg_launch_config to_abi(const GenConfig& g) {
  mrg_launch_config c{};
  c.seg_len = g.seg_len;
  c.block = (uint32_t)g.block;
  c.vec_bytes = (uint32_t)g.vec_bytes;
  c.blocks_per_sm = (uint32_t)g.per_sm;
  return c;
}

bool config_ok(const mrg_launch_config& c) {
  const bool block_ok = c.block == 0 || (c.block % 32 == 0 && c.block <= 256);
  const bool vec_ok = c.vec_bytes == 0 || c.vec_bytes == 4 || c.vec_bytes == 8 ||
                      c.vec_bytes == 16 || c.vec_bytes == 32;
  return block_ok && vec_ok && c.blocks_per_sm <= 64 && c.seg_len <= (1ull << 40);
}

}  // namespace

GenConfig generate_config_for(int dist, int dtype, uint64_t ns, uint64_t n) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_table.find(key_for(dev, dist, dtype, ns, n));
  return it == g_table.end() ? GenConfig{} : it->second;
}

}  // namespace mrg

namespace {

bool pair_ok(int dist, int dtype) {
  return (dist == MRG_RAW && dtype == MRG_U32) ||
         ((dist == MRG_UNIFORM || dist == MRG_NORMAL || dist == MRG_EXPONENTIAL) &&
          (dtype == MRG_F32 || dtype == MRG_F64));
}

// Arguments shared by mrg_generate_config and mrg_tune_generate.
int check_generate_args(const mrg_streams* s, uint64_t n, int dist, int dtype, double rate,
                        void* out, uint64_t ld) {
  if (!s || !s->cur || !s->start || !s->sub || s->stride < s->n)
    return mrg::set_error(MRG_EINVAL, "bad stream set");
  if (!pair_ok(dist, dtype)) return mrg::set_error(MRG_EINVAL, "unsupported dist/dtype combination");
  if (dist == MRG_EXPONENTIAL && !(rate >= 0x1p-64 && rate <= 0x1p64))
    return mrg::set_error(MRG_EINVAL, "exponential rate must lie in [2^-64, 2^64]");
  if (n == 0 || s->n == 0) return MRG_OK;
  if (!out) return mrg::set_error(MRG_EINVAL, "out is NULL");
  if (ld < n) return mrg::set_error(MRG_EINVAL, "ld < n");
  if (reinterpret_cast<uintptr_t>(out) % (dtype == MRG_F64 ? 8 : 4))
    return mrg::set_error(MRG_EINVAL, "out is not aligned to its element size");
  const unsigned __int128 bytes = (unsigned __int128)s->n * ld * (dtype == MRG_F64 ? 8 : 4);
  if (n > (1ull << 62) || bytes >= ((unsigned __int128)1 << 62))
    return mrg::set_error(MRG_ERANGE, "size too large");
  return MRG_OK;
}

mrg::DevStreams devs(const mrg_streams* s) {
  return mrg::DevStreams{s->cur, s->start, s->sub, s->n, s->stride};
}

int cuda_fail(cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorName(e) + ": " + cudaGetErrorString(e);
  return mrg::set_error(MRG_ECUDA, m.c_str());
}

}  // namespace

extern "C" {

int mrg_generate_config(const mrg_streams* s, uint64_t n, int dist, int dtype, double rate,
                        void* out, uint64_t ld, const mrg_launch_config* cfg, void* stream) {
  int rc = check_generate_args(s, n, dist, dtype, rate, out, ld);
  if (rc) return rc;
  if (!cfg || !mrg::config_ok(*cfg)) return mrg::set_error(MRG_EINVAL, "bad launch configuration");
  if (n == 0 || s->n == 0) return MRG_OK;
  if ((rc = mrg::ensure_device_ready())) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = mrg::launch_generate(devs(s), n, dist, dtype, rate, out, ld, mrg::from_abi(*cfg), st);
  if (e != cudaSuccess) return cuda_fail(e, "generate_kernel");
  const uint64_t consumed = dist == MRG_NORMAL ? n + (n & 1) : n;
  e = mrg::launch_jump(s->cur, s->cur, nullptr, s->stride, s->n, consumed, 0, 0, st);
  if (e != cudaSuccess) return cuda_fail(e, "jump_kernel (advance)");
  return MRG_OK;
}

int mrg_tune_generate(const mrg_streams* s, uint64_t n, int dist, int dtype, double rate,
                      void* out, uint64_t ld, uint32_t reps, mrg_tune_entry* results,
                      uint32_t max_results, uint32_t* n_results, mrg_launch_config* best,
                      void* stream) {
  if (n_results) *n_results = 0;
  int rc = check_generate_args(s, n, dist, dtype, rate, out, ld);
  if (rc) return rc;
  if (n == 0 || s->n == 0) return mrg::set_error(MRG_EINVAL, "nothing to tune (n or n_streams is 0)");
  if (max_results && !results) return mrg::set_error(MRG_EINVAL, "results is NULL");
  if ((rc = mrg::ensure_device_ready())) return rc;
  if (reps == 0) reps = 3;
  if (reps > 100) reps = 100;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

  // Candidates: the library default first (so the tuner never records a
  // shape slower than the untuned one), then segment lengths x block sizes x
  // store widths.  Segment lengths beyond the row collapse to one segment
  // per stream and are tried once.
  std::vector<mrg::GenConfig> cand;
  cand.push_back(mrg::GenConfig{});
  const uint64_t ncap = (n + 7) / 8 * 8;
  const uint64_t segs[] = {256, 512, 1024, 2048, 4096, 8192, 16384};
  const int blocks[] = {128, 256};
  const int vecs[] = {32, 16};
  bool whole_row_done = false;
  for (uint64_t L : segs) {
    const bool whole = L >= ncap;
    if (whole && whole_row_done) continue;
    whole_row_done |= whole;
    for (int b : blocks)
      for (int v : vecs) {
        mrg::GenConfig g;
        g.seg_len = std::min(L, ncap);
        g.block = b;
        g.vec_bytes = v;
        cand.push_back(g);
      }
  }

  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return cuda_fail(e, "cudaEventCreate (tune)");
  }
  const mrg::DevStreams d = devs(s);
  float best_ms = 0.0f;
  size_t best_i = 0;
  uint32_t nr = 0;
  for (size_t i = 0; i < cand.size() && e == cudaSuccess; ++i) {
    e = mrg::launch_generate(d, n, dist, dtype, rate, out, ld, cand[i], st);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (uint32_t r = 0; r < reps && e == cudaSuccess; ++r)
      e = mrg::launch_generate(d, n, dist, dtype, rate, out, ld, cand[i], st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) break;
    ms /= (float)reps;
    if (nr < max_results) results[nr++] = mrg_tune_entry{mrg::to_abi(cand[i]), ms};
    if (i == 0 || ms < best_ms) {
      best_ms = ms;
      best_i = i;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(e, "timing a candidate (tune)");
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> lk(mrg::g_mu);
    mrg::g_table[mrg::key_for(dev, dist, dtype, s->n, n)] = cand[best_i];
  }
  if (best) *best = mrg::to_abi(cand[best_i]);
  if (n_results) *n_results = nr;
  return MRG_OK;
}

int mrg_tune_lookup(int dist, int dtype, uint64_t n_streams, uint64_t n, mrg_launch_config* cfg) {
  if (!cfg) return mrg::set_error(MRG_EINVAL, "cfg is NULL");
  if (!pair_ok(dist, dtype)) return mrg::set_error(MRG_EINVAL, "unsupported dist/dtype combination");
  *cfg = mrg::to_abi(mrg::generate_config_for(dist, dtype, n_streams, n));
  return MRG_OK;
}

int mrg_tune_set(int dist, int dtype, uint64_t n_streams, uint64_t n, const mrg_launch_config* cfg) {
  if (!pair_ok(dist, dtype)) return mrg::set_error(MRG_EINVAL, "unsupported dist/dtype combination");
  if (cfg && !mrg::config_ok(*cfg)) return mrg::set_error(MRG_EINVAL, "bad launch configuration");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  std::lock_guard<std::mutex> lk(mrg::g_mu);
  const mrg::Key k = mrg::key_for(dev, dist, dtype, n_streams, n);
  if (cfg) mrg::g_table[k] = mrg::from_abi(*cfg);
  else mrg::g_table.erase(k);
  return MRG_OK;
}

void mrg_tune_clear(void) {
  std::lock_guard<std::mutex> lk(mrg::g_mu);
  mrg::g_table.clear();
}

}  // extern "C"
