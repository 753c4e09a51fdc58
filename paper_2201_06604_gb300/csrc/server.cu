// server.cu -- serving engine: continuous batching of generation requests
// into one persistent worker kernel (serve_kernels.cuh).
//
// Admission is by slots and output memory: a request is admitted only if a
// slot is free and its output fits in the caller's device arena (first fit);
// otherwise submit returns MRG_EBUSY and the caller keeps it queued.
//
// Request descriptors and ring records live in device memory.  The host
// writes them into pinned staging arrays and copies them on its copy stream,
// followed, in the same stream, by the new ring tail; the worker's warps read
// the tail with an acquire load and the records with L1-bypassing loads.
// (Host-mapped records read by the warps directly over the C2C link took
// 0.1-0.4 ms per tile under load; device-memory reads take microseconds.)
// Each tail publication copies from its own staging word, so a copy still
// pending can never pick up a newer tail whose records are not copied yet.  The
// tiles of admitted requests go to the ring of the running worker in chunks
// of kChunk, round-robin over the requests in flight (pump), so a small
// request that arrives behind a large one waits for at most one chunk per
// request ahead of it instead of the large request's whole backlog; pump runs
// on every submit and poll.  Requests overlap on the device with those
// already in flight.  The client acknowledges a finished request with
// release, which returns its slot and output memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <deque>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <thread>
#include <unordered_map>
#include <vector>

#include <time.h>

#include "../../include/mrg32k3a.h"
#include "internal.h"

struct mrg_server {
  int device = 0;
  mrg_streams s{};
  char* arena = nullptr;
  uint64_t arena_bytes = 0;
  uint32_t max_slots = 0;
  uint64_t ring_tiles = 0;      // power of two
  uint64_t idle_ns = 0;
  int grid = 0;
  // pinned host staging of the device-resident descriptors and ring
  mrg::BatchReqHost* slots_h = nullptr;
  mrg::ServeTileHost* ring_h = nullptr;
  mrg::BatchReqHost* slots_d = nullptr;     // device memory
  mrg::ServeTileHost* ring_d = nullptr;     // device memory
  // host-mapped pinned memory written by the worker
  unsigned int* done_h = nullptr;
  unsigned int* done_d = nullptr;
  // staging words of published tails, one per publication (round robin), and
  // the event that marks each one's copy as done
  unsigned long long* tail_h = nullptr;
  cudaEvent_t tail_ev[256] = {};
  uint64_t publications = 0;
  unsigned long long* head_h = nullptr;    // mapped: claim counter mirror (written by the worker)
  unsigned long long* head_d = nullptr;
  unsigned int* stop_h = nullptr;
  // device memory
  mrg::ServeCtlHost* ctl_d = nullptr;
  unsigned int* tiles_done_d = nullptr;
  cudaStream_t worker = nullptr;
  cudaStream_t copier = nullptr;
  bool running = false;
  bool failed = false;
  // bookkeeping
  std::mutex mu;
  uint64_t tail = 0;
  uint64_t next_seq = 1;
  std::vector<uint32_t> free_slots;
  std::map<uint64_t, uint64_t> free_mem;   // offset -> size
  struct Inflight {
    uint32_t slot;
    uint32_t seq;
    uint64_t mem_off, mem_size;
    uint64_t ntiles, emitted;
    uint64_t ring_first;     // first ring position (valid once emitted > 0)
    bool done;
  };
  std::unordered_map<uint64_t, Inflight> inflight;  // id -> state
  std::multiset<uint64_t> ring_firsts;               // first ring positions of started, undone requests
  std::deque<uint64_t> start_queue;                  // admitted ids with no tile emitted yet (FIFO)
  std::deque<uint64_t> emit_queue;                   // started ids with tiles still to emit
  uint64_t reserved = 0;                             // tiles of started requests not yet emitted
  // feeder thread: keeps the ring's backlog topped up while tiles are pending
  std::thread feeder;
  std::atomic<bool> quit{false};
  mrg_tiling tiling{32, 128, 8192};
};

namespace {

constexpr uint64_t kAlign = 256;
constexpr unsigned kTailWords = 256;   // staging words of published tails (round robin)
constexpr uint64_t kChunk = 256;       // tiles of one request per round-robin turn
constexpr uint64_t kBacklog = 8192;    // published tiles not yet claimed, at most (about one
                                       // per resident warp of the whole GPU)

// Default tiling, for latency.  A request that arrives while others occupy
// the warps waits for about one tile's duration, which grows with the
// segment length, so segments are short: n / 8192 draws, at least 32 (the
// jump to a segment costs about as much as a few dozen draws), at most 128;
// a large request is then many tiles that keep every warp busy, fed into the
// ring a chunk at a time.  mrg_server_set_tiling changes it.
constexpr mrg_tiling kDefaultTiling{32, 128, 8192};

bool arena_alloc(mrg_server* sv, uint64_t size, uint64_t* off) {
  for (auto it = sv->free_mem.begin(); it != sv->free_mem.end(); ++it) {
    if (it->second >= size) {
      *off = it->first;
      const uint64_t rest = it->second - size;
      const uint64_t next = it->first + size;
      sv->free_mem.erase(it);
      if (rest) sv->free_mem[next] = rest;
      return true;
    }
  }
  return false;
}

void arena_free(mrg_server* sv, uint64_t off, uint64_t size) {
  auto it = sv->free_mem.emplace(off, size).first;
  auto nx = std::next(it);
  if (nx != sv->free_mem.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    sv->free_mem.erase(nx);
  }
  if (it != sv->free_mem.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      sv->free_mem.erase(it);
    }
  }
}

// Starts admitted requests in arrival order, appends chunks of their tiles to
// the ring round-robin while there is ring space, and publishes the new tail.
//
// A ring position is reused only once the request whose first tile lies at
// or before it has completed.  A request therefore starts only when the ring
// can hold all of its tiles together with every tile still to be emitted for
// the requests already started -- otherwise large requests emitted round-robin
// could fill the ring with their first chunks, none could emit its last tile,
// none would complete, and nothing could move (observed under saturation
// before this rule).  Started requests can always finish emitting, so the
// oldest completes and frees the ring behind it.
int pump(mrg_server* sv) {
  uint64_t ring_low = sv->ring_firsts.empty() ? sv->tail : *sv->ring_firsts.begin();
  while (!sv->start_queue.empty()) {
    const uint64_t id = sv->start_queue.front();
    auto& f = sv->inflight[id];
    if ((sv->tail - ring_low) + sv->reserved + f.ntiles > sv->ring_tiles) break;
    sv->start_queue.pop_front();
    sv->reserved += f.ntiles;
    f.ring_first = sv->tail;              // its first tile lands at or after this position
    sv->ring_firsts.insert(f.ring_first);
    sv->emit_queue.push_back(id);
    ring_low = *sv->ring_firsts.begin();
  }
  uint64_t space = sv->ring_tiles - (sv->tail - ring_low);
  const uint64_t claimed = *reinterpret_cast<volatile unsigned long long*>(sv->head_h);
  const uint64_t backlog = sv->tail > claimed ? sv->tail - claimed : 0;
  space = std::min<uint64_t>(space, backlog < kBacklog ? kBacklog - backlog : 0);
  const uint64_t tail0 = sv->tail;
  size_t turns = sv->emit_queue.size();
  while (space > 0 && turns-- > 0) {
    const uint64_t id = sv->emit_queue.front();
    sv->emit_queue.pop_front();
    auto& f = sv->inflight[id];
    const uint64_t k = std::min<uint64_t>(std::min<uint64_t>(kChunk, f.ntiles - f.emitted), space);
    for (uint64_t i = 0; i < k; ++i)
      sv->ring_h[(sv->tail + i) & (sv->ring_tiles - 1)] =
          mrg::ServeTileHost{f.slot, (uint32_t)(32 * (f.emitted + i)), (uint32_t)f.ntiles, f.seq};
    f.emitted += k;
    sv->tail += k;
    sv->reserved -= k;
    space -= k;
    if (f.emitted < f.ntiles) sv->emit_queue.push_back(id);
    if (turns == 0 && space > 0 && !sv->emit_queue.empty()) turns = sv->emit_queue.size();
  }
  if (sv->tail == tail0) return MRG_OK;
  // records [tail0, tail) to the device ring (two copies if they wrap), then
  // the tail, all on the copy stream (executed in this order)
  const uint64_t mask = sv->ring_tiles - 1;
  cudaError_t e = cudaSuccess;
  for (uint64_t p = tail0; p < sv->tail && e == cudaSuccess;) {
    const uint64_t i = p & mask;
    const uint64_t k = std::min<uint64_t>(sv->tail - p, sv->ring_tiles - i);
    e = cudaMemcpyAsync(sv->ring_d + i, sv->ring_h + i, k * sizeof(mrg::ServeTileHost),
                        cudaMemcpyHostToDevice, sv->copier);
    p += k;
  }
  const unsigned w = (unsigned)(sv->publications++ % kTailWords);
  if (e == cudaSuccess && sv->publications > kTailWords)
    e = cudaEventSynchronize(sv->tail_ev[w]);  // the copy that last used this word is done
  if (e == cudaSuccess) {
    sv->tail_h[w] = sv->tail;
    e = cudaMemcpyAsync(&sv->ctl_d->tail, sv->tail_h + w, sizeof(unsigned long long),
                        cudaMemcpyHostToDevice, sv->copier);
  }
  if (e == cudaSuccess) e = cudaEventRecord(sv->tail_ev[w], sv->copier);
  if (e != cudaSuccess) return mrg::set_error(MRG_ECUDA, cudaGetErrorString(e));
  return MRG_OK;
}

int launch_worker(mrg_server* sv) {
  mrg::ServeCtlHost c{};
  c.head = sv->tail;  // resume claiming at the first unpublished position
  c.tail = sv->tail;
  *sv->head_h = sv->tail;
  *sv->stop_h = 0;
  cudaError_t e = cudaMemcpyAsync(sv->ctl_d, &c, sizeof c, cudaMemcpyHostToDevice, sv->worker);
  if (e == cudaSuccess) e = cudaStreamSynchronize(sv->worker);
  if (e == cudaSuccess)
    e = mrg::launch_serve(sv->ctl_d, sv->slots_d, sv->ring_d, sv->ring_tiles - 1, sv->tiles_done_d,
                          sv->done_d, sv->head_d, sv->s.start, sv->s.stride, sv->idle_ns, sv->grid,
                          sv->worker);
  if (e != cudaSuccess) return mrg::set_error(MRG_ECUDA, cudaGetErrorString(e));
  sv->running = true;
  sv->failed = false;
  return MRG_OK;
}

// The worker stream finished while it should be running: the idle limit
// fired (no published work for idle_ns).  Every request still in flight is
// reported as failed.
int check_worker(mrg_server* sv) {
  if (!sv->running) return sv->failed ? MRG_ETIMEOUT : MRG_OK;
  cudaError_t q = cudaStreamQuery(sv->worker);
  if (q == cudaErrorNotReady) return MRG_OK;
  sv->running = false;
  if (q != cudaSuccess) {
    sv->failed = true;
    return mrg::set_error(MRG_ECUDA, cudaGetErrorString(q));
  }
  sv->failed = true;
  return mrg::set_error(MRG_ETIMEOUT, "serving worker reached its idle limit and exited");
}

void feeder_main(mrg_server* sv) {
  timespec ts{0, 2000};  // 2 us between rounds
  while (!sv->quit.load(std::memory_order_relaxed)) {
    bool pending;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      const bool work = !sv->emit_queue.empty() || !sv->start_queue.empty();
      if (sv->running && work) pump(sv);
      pending = !sv->emit_queue.empty() || !sv->start_queue.empty();
    }
    if (!pending) ts.tv_nsec = 20000;   // idle: 20 us
    else ts.tv_nsec = 2000;
    nanosleep(&ts, nullptr);
  }
}

void server_free(mrg_server* sv) {
  if (!sv) return;
  if (sv->feeder.joinable()) {
    sv->quit.store(true);
    sv->feeder.join();
  }
  if (sv->worker) cudaStreamDestroy(sv->worker);
  if (sv->copier) cudaStreamDestroy(sv->copier);
  for (cudaEvent_t ev : sv->tail_ev)
    if (ev) cudaEventDestroy(ev);
  cudaFree(sv->ctl_d);
  cudaFree(sv->slots_d);
  cudaFree(sv->ring_d);
  cudaFree(sv->tiles_done_d);
  cudaFreeHost(sv->slots_h);
  cudaFreeHost(sv->ring_h);
  cudaFreeHost(sv->done_h);
  cudaFreeHost(sv->tail_h);
  cudaFreeHost(sv->stop_h);
  cudaFreeHost(sv->head_h);
  delete sv;
}

}  // namespace

extern "C" {

int mrg_server_create(const mrg_streams* s, void* arena, uint64_t arena_bytes, uint32_t max_slots,
                      uint64_t ring_tiles, double idle_seconds, double sm_fraction,
                      mrg_server** out) {
  if (!out) return mrg::set_error(MRG_EINVAL, "out is NULL");
  *out = nullptr;
  if (!s || !s->start || s->stride < s->n || s->n == 0) return mrg::set_error(MRG_EINVAL, "bad stream set");
  if (!arena || arena_bytes < kAlign || reinterpret_cast<uintptr_t>(arena) % kAlign)
    return mrg::set_error(MRG_EINVAL, "arena NULL, too small or not 256-byte aligned");
  if (max_slots == 0 || ring_tiles < 2 || (ring_tiles & (ring_tiles - 1)))
    return mrg::set_error(MRG_EINVAL, "max_slots must be > 0 and ring_tiles a power of two");
  if (!(idle_seconds > 0.0 && idle_seconds <= 3600.0))
    return mrg::set_error(MRG_EINVAL, "idle_seconds must lie in (0, 3600]");
  if (!(sm_fraction > 0.0 && sm_fraction <= 1.0))
    return mrg::set_error(MRG_EINVAL, "sm_fraction must lie in (0, 1]");
  int rc = mrg::ensure_device_ready();
  if (rc) return rc;
  mrg_server* sv = new mrg_server;
  cudaGetDevice(&sv->device);
  sv->s = *s;
  sv->arena = static_cast<char*>(arena);
  sv->arena_bytes = arena_bytes / kAlign * kAlign;
  sv->max_slots = max_slots;
  sv->ring_tiles = ring_tiles;
  sv->idle_ns = (uint64_t)(idle_seconds * 1e9);
  sv->grid = mrg::serve_grid(sm_fraction);
  cudaError_t e = cudaHostAlloc((void**)&sv->slots_h, sizeof(mrg::BatchReqHost) * max_slots, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&sv->ring_h, sizeof(mrg::ServeTileHost) * ring_tiles, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaMalloc((void**)&sv->slots_d, sizeof(mrg::BatchReqHost) * max_slots);
  if (e == cudaSuccess) e = cudaMalloc((void**)&sv->ring_d, sizeof(mrg::ServeTileHost) * ring_tiles);
  for (unsigned k = 0; k < kTailWords && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&sv->tail_ev[k], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&sv->done_h, sizeof(unsigned int) * max_slots, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&sv->tail_h, sizeof(unsigned long long) * kTailWords, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&sv->stop_h, sizeof(unsigned int), cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&sv->head_h, sizeof(unsigned long long), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&sv->head_d, sv->head_h, 0);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&sv->done_d, sv->done_h, 0);
  if (e == cudaSuccess) e = cudaMalloc((void**)&sv->ctl_d, sizeof(mrg::ServeCtlHost));
  if (e == cudaSuccess) e = cudaMalloc((void**)&sv->tiles_done_d, sizeof(unsigned int) * max_slots);
  if (e == cudaSuccess) e = cudaMemset(sv->tiles_done_d, 0, sizeof(unsigned int) * max_slots);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->worker, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->copier, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    server_free(sv);
    return mrg::set_error(MRG_ECUDA, cudaGetErrorString(e));
  }
  std::memset(sv->done_h, 0, sizeof(unsigned int) * max_slots);
  for (uint32_t i = max_slots; i-- > 0;) sv->free_slots.push_back(i);
  sv->free_mem[0] = sv->arena_bytes;
  rc = launch_worker(sv);
  if (rc) {
    server_free(sv);
    return rc;
  }
  sv->feeder = std::thread(feeder_main, sv);
  *out = sv;
  return MRG_OK;
}

int mrg_server_submit(mrg_server* sv, const mrg_request* q, uint64_t* id, void** out) {
  if (!sv || !q || !id) return mrg::set_error(MRG_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  int rc = check_worker(sv);
  if (rc) return rc;
  const bool pair_ok = (q->dist == MRG_RAW && q->dtype == MRG_U32) ||
                       ((q->dist == MRG_UNIFORM || q->dist == MRG_NORMAL ||
                         q->dist == MRG_EXPONENTIAL) && (q->dtype == MRG_F32 || q->dtype == MRG_F64));
  if (!pair_ok) return mrg::set_error(MRG_EINVAL, "unsupported dist/dtype combination");
  if (q->stream >= sv->s.n) return mrg::set_error(MRG_EINVAL, "stream index out of range");
  if (q->n == 0) return mrg::set_error(MRG_EINVAL, "empty request");
  if (q->substream >= (1ull << 51)) return mrg::set_error(MRG_ERANGE, "substream index >= 2^51");
  const uint64_t draws = q->dist == MRG_NORMAL ? q->n + (q->n & 1) : q->n;
  if (q->offset > (1ull << 62) || draws > (1ull << 62) || q->offset + draws > (1ull << 62))
    return mrg::set_error(MRG_ERANGE, "offset + draws too large");
  if (q->dist == MRG_EXPONENTIAL && !(q->rate >= 0x1p-64 && q->rate <= 0x1p64))
    return mrg::set_error(MRG_EINVAL, "exponential rate must lie in [2^-64, 2^64]");
  const uint32_t L = mrg::tiled_seg_len(q->n, sv->tiling.seg_min, sv->tiling.seg_max,
                                        sv->tiling.target_segments);
  const uint64_t nseg = (q->n + L - 1) / L;
  const uint64_t ntiles = (nseg + 31) / 32;
  const uint64_t bytes = (q->n * (q->dtype == MRG_F64 ? 8 : 4) + kAlign - 1) / kAlign * kAlign;
  if (bytes > sv->arena_bytes || nseg > 0xFFFFFFFFull)
    return mrg::set_error(MRG_ERANGE, "request larger than the server's arena");
  if (ntiles > sv->ring_tiles)
    return mrg::set_error(MRG_ERANGE, "request has more tiles than the server's ring holds");
  // admission: a slot and output memory (tiles go to the ring in chunks)
  if (sv->free_slots.empty()) return mrg::set_error(MRG_EBUSY, "no free slot");
  uint64_t off = 0;
  if (!arena_alloc(sv, bytes, &off)) return mrg::set_error(MRG_EBUSY, "output arena full");
  const uint32_t slot = sv->free_slots.back();
  sv->free_slots.pop_back();
  const uint64_t seq64 = sv->next_seq++;
  uint32_t seq = (uint32_t)seq64;
  if (seq == 0) seq = 1;  // 0 marks "never completed"
  mrg::BatchReqHost& h = sv->slots_h[slot];
  h.out = reinterpret_cast<uint64_t>(sv->arena + off);
  h.n = q->n;
  h.off = q->offset;
  h.sub = q->substream;
  h.stream = q->stream;
  h.dist = (uint32_t)q->dist;
  h.dtype = (uint32_t)q->dtype;
  const double ir = q->dist == MRG_EXPONENTIAL ? -1.0 / q->rate : 0.0;
  h.ir_hi = (float)ir;
  h.ir_lo = (float)(ir - (double)h.ir_hi);
  h.L = L;
  h.nseg = (uint32_t)nseg;
  // the descriptor reaches the device before any ring record that names it
  // (same copy stream); its staging entry is rewritten only after the slot is
  // released, long after this copy
  cudaError_t e = cudaMemcpyAsync(sv->slots_d + slot, &h, sizeof h, cudaMemcpyHostToDevice, sv->copier);
  if (e != cudaSuccess) {
    sv->free_slots.push_back(slot);
    arena_free(sv, off, bytes);
    return mrg::set_error(MRG_ECUDA, cudaGetErrorString(e));
  }
  sv->inflight[seq64] = mrg_server::Inflight{slot, seq, off, bytes, ntiles, 0, 0, false};
  sv->start_queue.push_back(seq64);
  rc = pump(sv);
  if (rc) return rc;
  *id = seq64;
  if (out) *out = sv->arena + off;
  return MRG_OK;
}

int mrg_server_poll(mrg_server* sv, uint64_t* ids, uint32_t max_ids, uint32_t* count) {
  if (!sv || !count || (max_ids && !ids)) return mrg::set_error(MRG_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  *count = 0;
  for (auto& kv : sv->inflight) {
    auto& f = kv.second;
    if (f.done) continue;
    const unsigned int w = reinterpret_cast<volatile unsigned int*>(sv->done_h)[f.slot];
    if (w != f.seq) continue;
    f.done = true;
    sv->ring_firsts.erase(sv->ring_firsts.find(f.ring_first));
    if (*count < max_ids) ids[(*count)++] = kv.first;
  }
  std::atomic_thread_fence(std::memory_order_acquire);
  int rc = pump(sv);
  if (rc) return rc;
  return check_worker(sv);
}

int mrg_server_release(mrg_server* sv, uint64_t id) {
  if (!sv) return mrg::set_error(MRG_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->inflight.find(id);
  if (it == sv->inflight.end()) return mrg::set_error(MRG_EINVAL, "unknown request id");
  if (!it->second.done) return mrg::set_error(MRG_EBUSY, "request not finished");
  sv->free_slots.push_back(it->second.slot);
  arena_free(sv, it->second.mem_off, it->second.mem_size);
  sv->inflight.erase(it);
  return MRG_OK;
}

int mrg_server_set_tiling(mrg_server* sv, const mrg_tiling* t) {
  if (!sv) return mrg::set_error(MRG_EINVAL, "server is NULL");
  if (t && !(t->seg_min >= 8 && t->seg_min % 8 == 0 && t->seg_max % 8 == 0 &&
             t->seg_min <= t->seg_max && t->seg_max <= (1u << 20) && t->target_segments >= 1))
    return mrg::set_error(MRG_EINVAL, "tiling outside its ranges");
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->tiling = t ? *t : kDefaultTiling;
  return MRG_OK;
}

uint64_t mrg_server_inflight(mrg_server* sv) {
  if (!sv) return 0;
  std::lock_guard<std::mutex> lk(sv->mu);
  uint64_t k = 0;
  for (auto& kv : sv->inflight) k += kv.second.done ? 0 : 1;
  return k;
}

int mrg_server_restart(mrg_server* sv) {
  if (!sv) return mrg::set_error(MRG_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(sv->mu);
  check_worker(sv);
  if (sv->running) return MRG_OK;
  cudaError_t e = cudaStreamSynchronize(sv->worker);
  if (e == cudaSuccess) e = cudaStreamSynchronize(sv->copier);
  if (e != cudaSuccess) return mrg::set_error(MRG_ECUDA, cudaGetErrorString(e));
  // requests that were in flight when the worker stopped are dropped
  for (auto it = sv->inflight.begin(); it != sv->inflight.end();) {
    if (!it->second.done) {
      sv->free_slots.push_back(it->second.slot);
      arena_free(sv, it->second.mem_off, it->second.mem_size);
      it = sv->inflight.erase(it);
    } else {
      ++it;
    }
  }
  sv->ring_firsts.clear();
  sv->emit_queue.clear();
  sv->start_queue.clear();
  sv->reserved = 0;
  e = cudaMemset(sv->tiles_done_d, 0, sizeof(unsigned int) * sv->max_slots);
  if (e != cudaSuccess) return mrg::set_error(MRG_ECUDA, cudaGetErrorString(e));
  return launch_worker(sv);
}

int mrg_server_destroy(mrg_server* sv) {
  if (!sv) return MRG_OK;
  int rc = MRG_OK;
  {
    std::unique_lock<std::mutex> lk(sv->mu);
    // let the feeder publish every admitted tile first (bounded by the ring)
    for (int spin = 0;
         sv->running && (!sv->emit_queue.empty() || !sv->start_queue.empty()) && spin < 200000;
         ++spin) {
      lk.unlock();
      timespec ts{0, 10000};
      nanosleep(&ts, nullptr);
      lk.lock();
      check_worker(sv);
    }
    if (sv->running) {
      // stop only affects warps waiting for unpublished positions: every
      // published tile is still processed before the worker exits
      *sv->stop_h = 1;
      cudaError_t e = cudaMemcpyAsync(&sv->ctl_d->stop, sv->stop_h, sizeof(unsigned int),
                                      cudaMemcpyHostToDevice, sv->copier);
      if (e == cudaSuccess) e = cudaStreamSynchronize(sv->worker);
      if (e != cudaSuccess) rc = mrg::set_error(MRG_ECUDA, cudaGetErrorString(e));
      sv->running = false;
    }
    cudaStreamSynchronize(sv->copier);
  }
  server_free(sv);
  return rc;
}

}  // extern "C"
