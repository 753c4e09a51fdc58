// noalloc.cu -- batched generation for callers that cannot allocate device
// memory.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured (allocation is not a capturable operation), plug-ins hosted
// by an application that owns the whole device-memory budget through its own
// allocator, and latency-critical loops where cudaMalloc's implicit device
// synchronisation is not acceptable.  mrg_batch_run_static serves them: it
// runs the same persistent batch kernel as mrg_batch_run, but its request
// table, tile table and claim counter live in the fixed-size device array
// below, which every GPU that loads the library holds until the process
// exits.  Nothing in this file allocates memory, on the device or the host.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/mrg32k3a.h"
#include "internal.h"

namespace {

constexpr uint32_t kMaxRequests = 1024;   // requests per call
constexpr uint32_t kMaxTiles = 16384;     // tiles per call (a tile = <= 32 segments)
constexpr size_t kHeaderBytes = 256;      // claim counter + tile count, padded
constexpr size_t kReqBytes = sizeof(mrg::BatchReqHost) * kMaxRequests;
constexpr size_t kTileBytes = sizeof(mrg::BatchTileHost) * kMaxTiles;
constexpr size_t kScratchBytes = kHeaderBytes + kReqBytes + kTileBytes;  // 192.25 KiB

// The scratch.  In host code this name is only a host-side stand-in for the
// symbol; its device address comes from cudaGetSymbolAddress (set_up below).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Host staging of the tables, static so that building them allocates
// nothing; g_mu serialises its use.
struct Staging {
  mrg::BatchHeaderHost hdr;
  mrg::BatchReqHost reqs[kMaxRequests];
  mrg::BatchTileHost tiles[kMaxTiles];
};
Staging g_stage;
std::mutex g_mu;
unsigned char* g_dev_scratch[64] = {};  // device address of g_scratch, per device

// Per-device set-up, with that device current: the library's tables, and the
// device address of g_scratch.
int set_up(int dev) {
  if (g_dev_scratch[dev]) return MRG_OK;
  int rc = mrg::ensure_device_ready();
  if (rc) return rc;
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) return mrg::set_error(MRG_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
  g_dev_scratch[dev] = static_cast<unsigned char*>(p);
  return MRG_OK;
}

// Same segment length rule as mrg_batch_run (whole 32-byte units, ~n/32).
uint32_t seg_len(uint64_t draws) {
  uint64_t L = (draws + 31) / 32;
  L = (L + 7) / 8 * 8;
  if (L < 8) L = 8;
  if (L > 2048) L = 2048;
  return (uint32_t)L;
}

}  // namespace

extern "C" int mrg_batch_run_static(const mrg_streams* s, const mrg_request* reqs, uint32_t nreq,
                                    void* stream) {
  if (!s || !s->cur || !s->start || !s->sub || s->stride < s->n)
    return mrg::set_error(MRG_EINVAL, "bad stream set");
  if (nreq > 0 && !reqs) return mrg::set_error(MRG_EINVAL, "reqs is NULL");
  if (nreq > kMaxRequests)
    return mrg::set_error(MRG_ERANGE, "more than 1024 requests in one static-scratch call");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) return mrg::set_error(MRG_ECUDA, "cudaGetDevice failed");
  std::lock_guard<std::mutex> lk(g_mu);
  int rc = set_up(dev);
  if (rc) return rc;
  uint64_t nt = 0;
  for (uint32_t r = 0; r < nreq; ++r) {
    const mrg_request& q = reqs[r];
    const bool pair_ok = (q.dist == MRG_RAW && q.dtype == MRG_U32) ||
                         ((q.dist == MRG_UNIFORM || q.dist == MRG_NORMAL ||
                           q.dist == MRG_EXPONENTIAL) && (q.dtype == MRG_F32 || q.dtype == MRG_F64));
    if (!pair_ok) return mrg::set_error(MRG_EINVAL, "request with unsupported dist/dtype");
    if (q.stream >= s->n) return mrg::set_error(MRG_EINVAL, "request stream index out of range");
    if (q.substream >= (1ull << 51)) return mrg::set_error(MRG_ERANGE, "substream index >= 2^51");
    const uint64_t draws = q.dist == MRG_NORMAL ? q.n + (q.n & 1) : q.n;
    if (q.offset > (1ull << 62) || draws > (1ull << 62) || q.offset + draws > (1ull << 62))
      return mrg::set_error(MRG_ERANGE, "offset + draws too large");
    if (q.n > 0 && (!q.out || reinterpret_cast<uintptr_t>(q.out) % 32))
      return mrg::set_error(MRG_EINVAL, "request output NULL or not 32-byte aligned");
    if (q.dist == MRG_EXPONENTIAL && !(q.rate >= 0x1p-64 && q.rate <= 0x1p64))
      return mrg::set_error(MRG_EINVAL, "exponential rate must lie in [2^-64, 2^64]");
    mrg::BatchReqHost& h = g_stage.reqs[r];
    h.out = reinterpret_cast<uint64_t>(q.out);
    h.n = q.n;
    h.off = q.offset;
    h.sub = q.substream;
    h.stream = q.stream;
    h.dist = (uint32_t)q.dist;
    h.dtype = (uint32_t)q.dtype;
    const double ir = q.dist == MRG_EXPONENTIAL ? -1.0 / q.rate : 0.0;
    h.ir_hi = (float)ir;
    h.ir_lo = (float)(ir - (double)h.ir_hi);
    h.L = seg_len(q.n);
    h.nseg = (uint32_t)((q.n + h.L - 1) / h.L);
    const uint64_t tiles = (h.nseg + 31) / 32;
    if (nt + tiles > kMaxTiles)
      return mrg::set_error(MRG_ERANGE, "more than 16384 tiles in one static-scratch call");
    for (uint64_t k = 0; k < tiles; ++k) g_stage.tiles[nt + k] = mrg::BatchTileHost{r, (uint32_t)(32 * k)};
    nt += tiles;
  }
  if (nt == 0) return MRG_OK;
  // The claim counter must start at zero: the header is rewritten every call.
  g_stage.hdr.next_tile = 0;
  g_stage.hdr.ntiles = nt;
  unsigned char* d = g_dev_scratch[dev];
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // Pageable-source copies: each returns once g_stage has been read.
  e = cudaMemcpyAsync(d, &g_stage.hdr, sizeof(g_stage.hdr), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d + kHeaderBytes, g_stage.reqs, sizeof(mrg::BatchReqHost) * nreq,
                        cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d + kHeaderBytes + kReqBytes, g_stage.tiles, sizeof(mrg::BatchTileHost) * nt,
                        cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return mrg::set_error(MRG_ECUDA, cudaGetErrorString(e));
  e = mrg::launch_batch(d, d + kHeaderBytes, d + kHeaderBytes + kReqBytes, s->start, s->stride,
                        mrg::batch_grid(), st);
  if (e != cudaSuccess) return mrg::set_error(MRG_ECUDA, cudaGetErrorString(e));
  return MRG_OK;
}
