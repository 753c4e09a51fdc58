// noalloc.cu -- batched generation for callers that cannot allocate device
// memory.
//
// Some callers cannot call cudaMalloc: plug-ins hosted by an application that
// owns the whole device-memory budget through its own allocator (a cudaMalloc
// behind its back can fail or push the host application out of memory), and
// latency-critical loops where cudaMalloc's implicit device synchronisation
// is not acceptable.  mrg_batch_run_static serves them: it
// runs the same persistent batch kernel as mrg_batch_run, but its request
// table, tile table and claim counter live in the fixed-size device array
// below, which every GPU that loads the library holds until the process
// exits.  Nothing in this file allocates memory, on the device or the host.
#include <cuda_runtime.h>

#include <algorithm>
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
  uint32_t order[kMaxRequests];  // request order of the tile table
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

// Tiling of the static path: segments of ~n/32 draws, 8..2048, whole 32-byte units.
constexpr uint32_t kSegMin = 8, kSegMax = 2048;
constexpr uint64_t kTargetSegments = 32;

}  // namespace

extern "C" int mrg_batch_run_static(const mrg_streams* s, const mrg_request* reqs, uint32_t nreq,
                                    void* stream) {
  if (!s || !s->cur || !s->start || !s->sub || s->stride < s->n)
    return mrg::set_error(MRG_EINVAL, "bad stream set");
  if (nreq > 0 && !reqs) return mrg::set_error(MRG_EINVAL, "reqs is NULL");
  if (nreq > kMaxRequests)
    return mrg::set_error(MRG_ERANGE, "more than 1024 requests in one static-scratch call");
  std::lock_guard<std::mutex> lk(g_mu);
  int rc = MRG_OK;
  uint64_t nt = 0;
  for (uint32_t r = 0; r < nreq; ++r) {
    uint64_t tiles = 0;
    rc = mrg::prepare_request(reqs[r], s->n, kSegMin, kSegMax, kTargetSegments, &g_stage.reqs[r],
                              &tiles);
    if (rc) return rc;
    nt += tiles;
    if (nt > kMaxTiles)
      return mrg::set_error(MRG_ERANGE, "more than 16384 tiles in one static-scratch call");
  }
  // Tiles of the longest segments first, so that the last tiles claimed by
  // the persistent kernel are the shortest (a short tail); the sort works in
  // the static staging and allocates nothing.
  for (uint32_t r = 0; r < nreq; ++r) g_stage.order[r] = r;
  std::stable_sort(g_stage.order, g_stage.order + nreq, [](uint32_t x, uint32_t y) {
    return g_stage.reqs[x].L > g_stage.reqs[y].L;
  });
  uint64_t k = 0;
  for (uint32_t i = 0; i < nreq; ++i) {
    const uint32_t r = g_stage.order[i];
    const uint64_t tiles = ((uint64_t)g_stage.reqs[r].nseg + 31) / 32;
    for (uint64_t j = 0; j < tiles; ++j) g_stage.tiles[k++] = mrg::BatchTileHost{r, (uint32_t)(32 * j)};
  }
  if (nt == 0) return MRG_OK;
  // The requests are valid: only now is the device touched.
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) return mrg::set_error(MRG_ECUDA, "cudaGetDevice failed");
  rc = set_up(dev);
  if (rc) return rc;
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
