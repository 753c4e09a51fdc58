// batch_kernels.cuh -- persistent kernel serving a table of uneven requests
// (included by kernels.cu, which owns the constant and global tables).
//
// A request r asks for n outputs of one distribution and output type from an
// absolute position of one stream: start_s + j 2^76 + off draws (substream j
// of stream s, Sec. 2.1), written to its own output array.  The host cuts
// every request into segments of L_r draws (L_r a multiple of 8) and groups
// up to 32 consecutive segments of one request into a tile; a persistent grid
// of warps claims tiles from a device counter, so short and long requests are
// load-balanced without per-request launches.  Every lane jumps to its
// segment's absolute position, so outputs do not depend on the batch, its
// order, the tiling or the launch shape.
#pragma once

namespace mrg {

struct BatchReq {      // 64 bytes, filled on the host
  uint64_t out;        // device address of the request's output
  uint64_t n;          // outputs
  uint64_t off;        // draws after the substream start
  uint64_t sub;        // substream index j (< 2^51)
  uint64_t stream;     // stream index into the stream set
  uint32_t dist, dtype;
  float ir_hi, ir_lo;  // -1/rate as a float pair (exponentials)
  uint32_t L;          // segment length, multiple of 8
  uint32_t nseg;       // ceil(n / L)
};

static_assert(sizeof(BatchReq) == 64, "request record layout");

struct BatchTile {     // 8 bytes
  uint32_t req;
  uint32_t g0;         // first segment of the tile (lanes take g0 .. g0 + 31)
};

struct BatchHeader {   // device-resident, rewritten before every launch
  unsigned long long next_tile;  // claim counter
  uint64_t ntiles;
};

// One lane's segment of one request, generated and stored with 32-byte stores.
template <int DIST, int DT>
__device__ __forceinline__ void batch_segment(TState& st, const BatchReq& R, uint32_t cnt,
                                              char* gdst, uint32_t cmax, const Consts& c,
                                              const float4* __restrict__ tab) {
  constexpr int ES = DT == MRG_F64 ? 8 : 4;
  constexpr int UE = 32 / ES;  // 32-byte units
#pragma unroll 1
  for (uint32_t i = 0; i < cmax; i += UE) {
    uint32_t wv[8];
    produce<DIST, DT, UE>(st, wv, c, tab);
    if (i + UE <= cnt) {
      store_vec<32>(gdst + (size_t)i * ES, wv);
    } else if (i < cnt) {
#pragma unroll
      for (int e = 0; e < UE; ++e)
        if (i + e < cnt) store_vec<ES>(gdst + (size_t)(i + e) * ES, wv + e * (ES / 4));
    }
  }
}

// One tile of request R of a known variant: segments g0 .. g0 + 31.  All 32
// lanes of the warp call it.
template <int DIST, int DT>
__device__ __forceinline__ void batch_tile_v(const BatchReq& R, uint32_t g0,
                                             const uint32_t* __restrict__ start, uint64_t stride,
                                             uint64_t k1, uint64_t k2,
                                             const float4* __restrict__ tab) {
  constexpr int ES = DT == MRG_F64 ? 8 : 4;
  const int lane = threadIdx.x & 31;
  const uint32_t g = g0 + lane;
  const bool valid = g < R.nseg;
  const uint64_t seg_off = (uint64_t)g * R.L;
  const uint32_t cnt = valid ? (uint32_t)min((uint64_t)R.L, R.n - seg_off) : 0u;
  const uint32_t cmax = __reduce_max_sync(0xffffffffu, cnt);
  State st0 = load_state(start, stride, R.stream);
  // substream: A^(j 2^76), warp-uniform
  for (uint64_t j = R.sub; j; j &= j - 1) apply_pow2_both(SUBSTREAM_LOG2 + __ffsll((long long)j) - 1, st0);
  // offset of this lane's segment (< 2^64), per lane
  jump_lanes(st0, R.off + (valid ? seg_off : 0), 0);
  TState st = to_offset(st0);
  const Consts c{k1, k2, R.ir_hi, R.ir_lo};
  char* gdst = reinterpret_cast<char*>(R.out) + seg_off * ES;
  batch_segment<DIST, DT>(st, R, cnt, gdst, cmax, c, tab);
}

// Processes tile t of any variant (dispatch on the request's variant).  All
// 32 lanes of the warp call it.
__device__ __forceinline__ void batch_tile(const BatchReq* __restrict__ reqs,
                                           const BatchTile* __restrict__ tiles, uint64_t t,
                                           const uint32_t* __restrict__ start, uint64_t stride,
                                           uint64_t k1, uint64_t k2,
                                           const float4* __restrict__ tab) {
  const BatchTile T = tiles[t];
  const BatchReq R = reqs[T.req];
  switch (R.dist * 4 + R.dtype) {
    case MRG_RAW * 4 + MRG_U32: batch_tile_v<MRG_RAW, MRG_U32>(R, T.g0, start, stride, k1, k2, tab); break;
    case MRG_UNIFORM * 4 + MRG_F32: batch_tile_v<MRG_UNIFORM, MRG_F32>(R, T.g0, start, stride, k1, k2, tab); break;
    case MRG_UNIFORM * 4 + MRG_F64: batch_tile_v<MRG_UNIFORM, MRG_F64>(R, T.g0, start, stride, k1, k2, tab); break;
    case MRG_NORMAL * 4 + MRG_F32: batch_tile_v<MRG_NORMAL, MRG_F32>(R, T.g0, start, stride, k1, k2, tab); break;
    case MRG_NORMAL * 4 + MRG_F64: batch_tile_v<MRG_NORMAL, MRG_F64>(R, T.g0, start, stride, k1, k2, tab); break;
    case MRG_EXPONENTIAL * 4 + MRG_F32: batch_tile_v<MRG_EXPONENTIAL, MRG_F32>(R, T.g0, start, stride, k1, k2, tab); break;
    default: batch_tile_v<MRG_EXPONENTIAL, MRG_F64>(R, T.g0, start, stride, k1, k2, tab); break;
  }
}

// Persistent worker over a table of mixed variants: warps claim tiles until
// the table is exhausted.
__global__ void __launch_bounds__(256) batch_kernel(BatchHeader* hdr, const BatchReq* reqs,
                                                    const BatchTile* tiles, const uint32_t* start,
                                                    uint64_t stride, uint64_t k1, uint64_t k2) {
  __shared__ float4 s_tab[TAB_ENTRIES];
  load_ttab(s_tab);
  const int lane = threadIdx.x & 31;
  const uint64_t ntiles = hdr->ntiles;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(&hdr->next_tile, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= ntiles) break;
    batch_tile(reqs, tiles, t, start, stride, k1, k2, s_tab);
  }
}

// Range of one variant in a variant-grouped tile table (device-resident,
// rewritten before every run).  Its claim counter lives apart, in a counter
// array that the batch graph zeroes at the start of every replay.
struct VariantRange {
  uint64_t begin, end;  // tiles [begin, end) of the table
};
constexpr int kCounterStride = 16;  // counters 128 bytes apart (one L2 line each)

// Persistent worker over the tiles of ONE variant (a range of a table grouped
// by variant).  A batch launches one of these per variant, each a
// programmatic dependent of the previous one: each kernel's code is one
// transform path, so warps sharing an SM sub-partition do not evict each
// other's instructions from its instruction cache, as the seven inlined paths
// of batch_kernel do when variants mix on one SM (measured: instruction-fetch
// stalls were the largest stall reason of the mixed kernel).
template <int DIST, int DT>
__global__ void __launch_bounds__(256) batch_variant_kernel(const VariantRange* rng,
                                                            unsigned long long* next,
                                                            const BatchReq* reqs,
                                                            const BatchTile* tiles,
                                                            const uint32_t* start, uint64_t stride,
                                                            uint64_t k1, uint64_t k2) {
  // The next variant's kernel is launched as a programmatic dependent: let it
  // be scheduled as soon as every block of this grid is resident, so that its
  // blocks take over SMs as this grid's blocks run out of tiles (the two
  // kernels touch disjoint outputs and neither reads what the other writes).
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  constexpr bool TABLES = DIST == MRG_NORMAL || DIST == MRG_EXPONENTIAL;
  __shared__ float4 s_tab[TABLES ? TAB_ENTRIES : 1];
  if constexpr (TABLES) load_ttab(s_tab);
  const int lane = threadIdx.x & 31;
  const uint64_t begin = rng->begin, end = rng->end;
  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = begin + atomicAdd(next, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= end) break;
    const BatchTile T = tiles[t];
    const BatchReq R = reqs[T.req];
    batch_tile_v<DIST, DT>(R, T.g0, start, stride, k1, k2, s_tab);
  }
}

}  // namespace mrg
