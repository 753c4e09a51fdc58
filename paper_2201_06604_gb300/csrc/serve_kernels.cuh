// serve_kernels.cuh -- the persistent worker of the serving engine (included
// by kernels.cu).
//
// The host admits requests into slots (descriptor records in device memory),
// appends their tiles to a ring (also in device memory) in chunks,
// round-robin over the requests in flight, and publishes the new ring tail
// with one small copy that follows the record copies on the same stream.
// Records are read with volatile (L1-bypassing) loads, since a ring entry is
// rewritten by the copy engine on every lap of the ring.  Warps
// claim ring positions from a device counter; a warp whose position is not
// published yet waits for it with a bounded, backed-off poll of the
// device-side tail.  The warp that finishes the last tile of a request
// writes the request's sequence number into the slot's done word in
// host-mapped memory, which the host polls.  New requests thus join a kernel
// that is already running: their tiles interleave with those of earlier
// requests on the same SMs.
//
// Every wait is bounded: a warp gives up after `idle_ns` nanoseconds without
// a published tile (the worker then records status 2 and exits) and exits at
// once when the host sets `stop` while it is waiting.  The host only sets
// stop once every published tile has completed, so no published tile is ever
// abandoned.
#pragma once

namespace mrg {

// Each word on its own 128-byte line: the claim counter's atomics and the
// idle warps' polls of the tail do not contend for one L2 line.
struct ServeCtl {                                 // device memory
  alignas(128) unsigned long long head;           // claim counter (ring positions)
  alignas(128) unsigned long long tail;           // published ring positions (host copies)
  alignas(128) unsigned int stop;                 // host: exit when no published work is left
  alignas(128) unsigned int status;               // worker exit reason: 0 stop, 2 idle limit
};

struct ServeTile {                // 16 bytes, in the device-memory ring
  uint32_t slot;
  uint32_t g0;                    // first segment of the tile
  uint32_t ntiles;                // tiles of this request
  uint32_t seq;                   // low 32 bits of the request's sequence number
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned int ld_volatile_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void __launch_bounds__(256) serve_kernel(ServeCtl* ctl, const BatchReq* slots,
                                                    const ServeTile* ring, uint64_t ring_mask,
                                                    unsigned int* tiles_done,
                                                    unsigned int* done_words,
                                                    unsigned long long* head_mirror,
                                                    const uint32_t* start, uint64_t stride,
                                                    uint64_t k1, uint64_t k2, uint64_t idle_ns) {
  __shared__ float4 s_tab[TAB_ENTRIES];
  load_ttab(s_tab);
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long t = 0;
    int go = 1;
    if (lane == 0) {
      t = atomicAdd(&ctl->head, 1ull);
      // let the host see roughly how far the claims have got (it keeps the
      // published backlog short so that new requests are not queued behind it)
      if ((t & 31u) == 0)
        asm volatile("st.relaxed.sys.global.u64 [%0], %1;" :: "l"(head_mirror), "l"(t) : "memory");
      uint64_t since = global_ns();
      unsigned int backoff = 128;
      while (ld_acquire_u64(&ctl->tail) <= t) {   // position not published yet
        if (ld_volatile_u32(&ctl->stop)) { go = 0; break; }
        if (global_ns() - since > idle_ns) { atomicMax(&ctl->status, 2u); go = 0; break; }
        __nanosleep(backoff);                     // at most ~16 us between polls
        if (backoff < 16384) backoff <<= 1;
      }
    }
    t = __shfl_sync(0xffffffffu, t, 0);
    go = __shfl_sync(0xffffffffu, go, 0);
    if (!go) break;
    // The ring entry and the slot descriptor were written by the host before
    // the tail that covers them was published (acquire above).
    ServeTile T;
    {
      uint32_t a, b, c, d;
      asm volatile("ld.volatile.global.v4.u32 {%0, %1, %2, %3}, [%4];"
                   : "=r"(a), "=r"(b), "=r"(c), "=r"(d) : "l"(ring + (t & ring_mask)) : "memory");
      T.slot = a; T.g0 = b; T.ntiles = c; T.seq = d;
    }
    BatchReq R;
    {
      const volatile BatchReq* src = &slots[T.slot];
      R.out = src->out; R.n = src->n; R.off = src->off; R.sub = src->sub; R.stream = src->stream;
      R.dist = src->dist; R.dtype = src->dtype; R.ir_hi = src->ir_hi; R.ir_lo = src->ir_lo;
      R.L = src->L; R.nseg = src->nseg;
    }
    BatchTile bt{0u, T.g0};
    batch_tile(&R, &bt, 0, start, stride, k1, k2, s_tab);
    __syncwarp();
    if (lane == 0) {
      __threadfence();                 // this warp's outputs before its count
      const unsigned int k = atomicAdd(&tiles_done[T.slot], 1u) + 1u;
      if (k == T.ntiles) {
        tiles_done[T.slot] = 0u;       // the slot is reused only after the host sees completion
        __threadfence_system();        // cumulative: every tile counted above, system-wide
        asm volatile("st.release.sys.global.u32 [%0], %1;" :: "l"(done_words + T.slot), "r"(T.seq) : "memory");
      }
    }
  }
}

}  // namespace mrg
