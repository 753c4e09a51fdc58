// kernels.cu -- CUDA kernels of the MRG32k3a hot path for GB300 (sm_103a).
//
//   create_kernel    stream i = A^(i 2^127) seed, one thread per stream
//                    (Sec. 2.1: equal to creating the streams one after another)
//   jump_kernel      x <- A^k x for every stream (skip, substreams, advance)
//   generate_kernel  the recurrence in registers + transform + staged store
//   fused_kernel     no-store consumer: quarter-circle count and normal sum
//
// Work decomposition of generate: every stream's n outputs are cut into
// segments of L draws; a lane owns one (stream, segment) pair, jumps to the
// segment's absolute offset with the constant-memory tables A^(2^i), then runs
// the recurrence in registers.  Segment q of the flattened index runs stream
// q mod ns at segment q div ns, so the 32 lanes of a warp share the segment
// offset whenever ns >= 32 and the jump's table reads are warp-uniform.
// Outputs go through a per-lane row of shared memory (CHUNK bytes, padded by
// 16 B so that the 8 lanes of a 128-bit store phase hit distinct banks) and
// leave with one cp.async.bulk (TMA bulk copy) per row chunk: each lane's
// destination is contiguous, so the copy engine writes whole 128-byte lines
// while the SM goes on with the next chunk's arithmetic.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "mrg32k3a_core.cuh"
#include "transforms_f64.cuh"

#define MRG_RAW 0
#define MRG_UNIFORM 1
#define MRG_NORMAL 2
#define MRG_EXPONENTIAL 3
#define MRG_U32 0
#define MRG_F32 1
#define MRG_F64 2

namespace mrg {

std::atomic<uint64_t> g_launches{0};

__constant__ uint32_t c_jump[2][JUMP_BITS][9];

cudaError_t upload_tables(const uint32_t* tab, size_t bytes) {
  if (bytes != sizeof(c_jump)) return cudaErrorInvalidValue;
  return cudaMemcpyToSymbol(c_jump, tab, bytes);
}

// ---------------------------------------------------------------------------
// Jump helpers
// ---------------------------------------------------------------------------

template <int COMP>
__device__ __forceinline__ void apply_pow2(int i, uint32_t& x0, uint32_t& x1, uint32_t& x2) {
  uint32_t A[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) A[k] = c_jump[COMP][i][k];
  matvec<COMP>(A, x0, x1, x2);
}

__device__ __forceinline__ void apply_pow2_both(int i, State& s) {
  apply_pow2<0>(i, s.a0, s.a1, s.a2);
  apply_pow2<1>(i, s.b0, s.b1, s.b2);
}

// s <- A^(e 2^base) s with a per-lane exponent e.  The loop runs over the
// bits set in any lane, so the table index is warp-uniform (constant-cache
// broadcast).  All 32 lanes of the warp must call it.
__device__ __forceinline__ void jump_lanes(State& s, uint64_t e, int base) {
  unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)e);
  unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(e >> 32));
  uint64_t any = ((uint64_t)hi << 32) | lo;
  while (any) {
    int i = __ffsll((long long)any) - 1;
    any &= any - 1;
    if ((e >> i) & 1) apply_pow2_both(base + i, s);
  }
}

__device__ __forceinline__ State load_state(const uint32_t* p, uint64_t stride, uint64_t i) {
  State s;
  s.a0 = p[i]; s.a1 = p[stride + i]; s.a2 = p[2 * stride + i];
  s.b0 = p[3 * stride + i]; s.b1 = p[4 * stride + i]; s.b2 = p[5 * stride + i];
  return s;
}

__device__ __forceinline__ void store_state(uint32_t* p, uint64_t stride, uint64_t i, const State& s) {
  p[i] = s.a0; p[stride + i] = s.a1; p[2 * stride + i] = s.a2;
  p[3 * stride + i] = s.b0; p[4 * stride + i] = s.b1; p[5 * stride + i] = s.b2;
}

// ---------------------------------------------------------------------------
// Stream creation
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) create_kernel(State seed, uint64_t n, uint32_t* cur,
                                                     uint32_t* start, uint32_t* sub,
                                                     uint64_t stride) {
  const uint64_t step_all = (uint64_t)gridDim.x * blockDim.x;
  // The trip count is uniform per block, so every lane reaches jump_lanes.
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < n; base += step_all) {
    const uint64_t i = base + threadIdx.x;
    const bool valid = i < n;
    State s = seed;
    jump_lanes(s, valid ? i : 0, STREAM_LOG2);
    if (valid) {
      store_state(cur, stride, i, s);
      store_state(start, stride, i, s);
      store_state(sub, stride, i, s);
    }
  }
}

// ---------------------------------------------------------------------------
// Uniform jump of every stream (skip / substream / advance / reset)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) jump_kernel(const uint32_t* src, uint32_t* dst0,
                                                   uint32_t* dst1, uint64_t stride, uint64_t ns,
                                                   uint64_t e_lo, uint64_t e_hi, int base) {
  const uint64_t step_all = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += step_all) {
    State s = load_state(src, stride, i);
    for (uint64_t e = e_lo; e; e &= e - 1) apply_pow2_both(base + __ffsll((long long)e) - 1, s);
    for (uint64_t e = e_hi; e; e &= e - 1) apply_pow2_both(base + 64 + __ffsll((long long)e) - 1, s);
    store_state(dst0, stride, i, s);
    if (dst1) store_state(dst1, stride, i, s);
  }
}

// ---------------------------------------------------------------------------
// TMA bulk-copy primitives (shared -> global), per thread
// ---------------------------------------------------------------------------

__device__ __forceinline__ void fence_proxy_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void bulk_s2g(void* gdst, uint32_t ssrc, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
               :: "l"(gdst), "r"(ssrc), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_commit() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_read0() {
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void bulk_wait_all() {
  asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Output pieces: 16 bytes of consecutive outputs of one stream
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint4 pack64(uint64_t a, uint64_t b) {
  return make_uint4((uint32_t)a, (uint32_t)(a >> 32), (uint32_t)b, (uint32_t)(b >> 32));
}

__device__ __forceinline__ uint4 pack_d(double a, double b) {
  return pack64((uint64_t)__double_as_longlong(a), (uint64_t)__double_as_longlong(b));
}

template <int DIST, int DT>
__device__ __forceinline__ uint4 piece(State& s, double inv_rate) {
  if constexpr (DIST == MRG_RAW) {
    uint32_t z0 = step(s), z1 = step(s), z2 = step(s), z3 = step(s);
    return make_uint4(z0, z1, z2, z3);
  } else if constexpr (DIST == MRG_UNIFORM && DT == MRG_F64) {
    uint64_t u0 = uniform_bits64(step(s));
    uint64_t u1 = uniform_bits64(step(s));
    return pack64(u0, u1);
  } else if constexpr (DIST == MRG_UNIFORM) {
    uint32_t v0 = f32_bits_from_f64(uniform_bits64(step(s)));
    uint32_t v1 = f32_bits_from_f64(uniform_bits64(step(s)));
    uint32_t v2 = f32_bits_from_f64(uniform_bits64(step(s)));
    uint32_t v3 = f32_bits_from_f64(uniform_bits64(step(s)));
    return make_uint4(v0, v1, v2, v3);
  } else if constexpr (DIST == MRG_NORMAL && DT == MRG_F64) {
    uint32_t z1 = step(s);
    uint32_t z2 = step(s);
    double x, y;
    box_muller_f64(z1, z2, x, y);
    return pack_d(x, y);
  } else if constexpr (DIST == MRG_NORMAL) {
    uint32_t z1 = step(s);
    uint32_t z2 = step(s);
    uint32_t z3 = step(s);
    uint32_t z4 = step(s);
    double x0, y0, x1, y1;
    box_muller_f64(z1, z2, x0, y0);
    box_muller_f64(z3, z4, x1, y1);
    return make_uint4(__float_as_uint(__double2float_rn(x0)), __float_as_uint(__double2float_rn(y0)),
                      __float_as_uint(__double2float_rn(x1)), __float_as_uint(__double2float_rn(y1)));
  } else if constexpr (DT == MRG_F64) {  // exponential
    double e0 = exponential_f64(step(s), inv_rate);
    double e1 = exponential_f64(step(s), inv_rate);
    return pack_d(e0, e1);
  } else {
    float e0 = __double2float_rn(exponential_f64(step(s), inv_rate));
    float e1 = __double2float_rn(exponential_f64(step(s), inv_rate));
    float e2 = __double2float_rn(exponential_f64(step(s), inv_rate));
    float e3 = __double2float_rn(exponential_f64(step(s), inv_rate));
    return make_uint4(__float_as_uint(e0), __float_as_uint(e1), __float_as_uint(e2),
                      __float_as_uint(e3));
  }
}

// ---------------------------------------------------------------------------
// Materialised generation
// ---------------------------------------------------------------------------

struct GenArgs {
  const uint32_t* cur;
  uint64_t stride, ns;
  uint64_t n;      // outputs per stream
  uint64_t L;      // segment length in outputs (= draws), multiple of the chunk
  uint64_t total;  // ns * ceil(n / L) segments
  char* out;
  uint64_t ld;     // elements
  double inv_rate;
};

template <int DIST, int DT, int CHUNK, bool BULK>
__global__ void __launch_bounds__(256) generate_kernel(GenArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int ES = DT == MRG_F64 ? 8 : 4;     // bytes per element
  constexpr int PIECES = CHUNK / 16;
  constexpr int CE = CHUNK / ES;                // elements per row chunk
  constexpr int PE = 16 / ES;                   // elements per piece
  constexpr int PITCH = CHUNK + 16;
  constexpr bool CHEAP = DIST == MRG_RAW || DIST == MRG_UNIFORM;

  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int wpb = blockDim.x >> 5;
  unsigned char* row = smem + (size_t)(warp * 32 + lane) * PITCH;
  const uint32_t row_s = (uint32_t)__cvta_generic_to_shared(row);
  const uint64_t ntiles = (a.total + 31) >> 5;

  for (uint64_t w = (uint64_t)blockIdx.x * wpb + warp; w < ntiles;
       w += (uint64_t)gridDim.x * wpb) {
    const uint64_t q = (w << 5) + lane;
    const bool valid = q < a.total;
    uint64_t s = 0, g = 0;
    if (valid) {
      g = q / a.ns;
      s = q - g * a.ns;
    }
    const uint64_t off = g * a.L;
    const uint32_t cnt = valid ? (uint32_t)min(a.L, a.n - off) : 0u;
    State st = valid ? load_state(a.cur, a.stride, s) : State{1, 1, 1, 1, 1, 1};
    jump_lanes(st, off, 0);
    const uint32_t cmax = __reduce_max_sync(0xffffffffu, cnt);
    char* gdst = a.out + (s * a.ld + off) * ES;

    for (uint32_t c0 = 0; c0 < cmax; c0 += CE) {
      if constexpr (BULK) {
        bulk_wait_read0();  // the previous chunk's copy has read this row
        if constexpr (CHEAP) {
#pragma unroll
          for (int p = 0; p < PIECES; ++p)
            *reinterpret_cast<uint4*>(row + p * 16) = piece<DIST, DT>(st, a.inv_rate);
        } else {
#pragma unroll 1
          for (int p = 0; p < PIECES; ++p)
            *reinterpret_cast<uint4*>(row + p * 16) = piece<DIST, DT>(st, a.inv_rate);
        }
        if (c0 < cnt) {
          const uint32_t m = min((uint32_t)CE, cnt - c0);
          const uint32_t bytes = m * ES;
          const uint32_t full = bytes & ~15u;
          if (full) {
            fence_proxy_async_shared();
            bulk_s2g(gdst + (size_t)c0 * ES, row_s, full);
            bulk_commit();
          }
          for (uint32_t b = full; b < bytes; b += 4)
            *reinterpret_cast<uint32_t*>(gdst + (size_t)c0 * ES + b) =
                *reinterpret_cast<const uint32_t*>(row + b);
        }
      } else {
#pragma unroll 1
        for (int p = 0; p < PIECES; ++p) {
          uint4 v = piece<DIST, DT>(st, a.inv_rate);
          const uint32_t e0 = c0 + p * PE;
          const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
          if constexpr (ES == 8) {
            if (e0 < cnt) {
              uint32_t* d = reinterpret_cast<uint32_t*>(gdst + (size_t)e0 * 8);
              d[0] = w4[0]; d[1] = w4[1];
            }
            if (e0 + 1 < cnt) {
              uint32_t* d = reinterpret_cast<uint32_t*>(gdst + (size_t)(e0 + 1) * 8);
              d[0] = w4[2]; d[1] = w4[3];
            }
          } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
              if (e0 + k < cnt) *reinterpret_cast<uint32_t*>(gdst + (size_t)(e0 + k) * 4) = w4[k];
          }
        }
      }
    }
  }
  if constexpr (BULK) bulk_wait_all();
}

// ---------------------------------------------------------------------------
// Fused no-store consumer
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) fused_kernel(uint32_t* cur, uint64_t stride, uint64_t ns,
                                                    uint64_t pairs, int64_t* count, double* sum) {
  constexpr uint64_t MSQ = MNORM * MNORM;  // (m1+1)^2 < 2^64
  const uint64_t step_all = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += step_all) {
    State s = load_state(cur, stride, i);
    int64_t cnt = 0;
    double acc = 0.0;
    for (uint64_t k = 0; k < pairs; ++k) {
      uint32_t za = step(s);
      uint32_t zb = step(s);
      uint64_t sa = (uint64_t)za * za, sb = (uint64_t)zb * zb;
      uint64_t ss = sa + sb;
      cnt += (ss >= sa) & (ss < MSQ);  // no carry out of 64 bits and below M^2
      double x, y;
      box_muller_f64(za, zb, x, y);
      acc += x;
      acc += y;
    }
    store_state(cur, stride, i, s);
    count[i] = cnt;
    sum[i] = acc;
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

namespace {

struct DevInfo {
  int sms = 0;
};

DevInfo& dev_info() {
  static std::mutex mu;
  static DevInfo info[64];
  int d = 0;
  cudaGetDevice(&d);
  std::lock_guard<std::mutex> lk(mu);
  DevInfo& di = info[d & 63];
  if (di.sms == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
    di.sms = v > 0 ? v : 1;
  }
  return di;
}

inline cudaError_t after_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

inline unsigned grid_for(uint64_t items, int block, int per_sm) {
  uint64_t need = (items + block - 1) / block;
  uint64_t cap = (uint64_t)sm_count() * per_sm;
  return (unsigned)std::max<uint64_t>(1, std::min(need, cap));
}

}  // namespace

int sm_count() { return dev_info().sms; }

cudaError_t launch_create(const uint32_t seed[6], uint64_t n, const DevStreams& s,
                          cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  State sd{seed[0], seed[1], seed[2], seed[3], seed[4], seed[5]};
  create_kernel<<<grid_for(n, 256, 8), 256, 0, st>>>(sd, n, s.cur, s.start, s.sub, s.stride);
  return after_launch();
}

cudaError_t launch_jump(const uint32_t* src, uint32_t* dst0, uint32_t* dst1, uint64_t stride,
                        uint64_t ns, uint64_t e_lo, uint64_t e_hi, int base, cudaStream_t st) {
  if (ns == 0) return cudaSuccess;
  jump_kernel<<<grid_for(ns, 256, 8), 256, 0, st>>>(src, dst0, dst1, stride, ns, e_lo, e_hi, base);
  return after_launch();
}

cudaError_t launch_fused(const DevStreams& s, uint64_t pairs, int64_t* count, double* sum,
                         cudaStream_t st) {
  if (s.n == 0) return cudaSuccess;
  fused_kernel<<<grid_for(s.n, 256, 8), 256, 0, st>>>(s.cur, s.stride, s.n, pairs, count, sum);
  return after_launch();
}

namespace {

template <int DIST, int DT, int CHUNK, bool BULK>
cudaError_t launch_gen_t(const GenArgs& a, const GenConfig& cfg, cudaStream_t st) {
  auto kern = generate_kernel<DIST, DT, CHUNK, BULK>;
  const int block = cfg.block;
  const size_t smem = BULK ? (size_t)block * (CHUNK + 16) : 0;
  static thread_local int occ_cache[64][2] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  int& occ = occ_cache[dev & 63][block == 256 ? 0 : 1];
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (occ == 0) {
    int v = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, block, smem);
    if (e != cudaSuccess) return e;
    occ = v > 0 ? v : 1;
  }
  const uint64_t ntiles = (a.total + 31) / 32;
  const uint64_t wpb = block / 32;
  uint64_t blocks = (ntiles + wpb - 1) / wpb;
  uint64_t cap = (uint64_t)sm_count() * occ;
  if (cfg.max_blocks > 0) cap = std::min<uint64_t>(cap, (uint64_t)cfg.max_blocks);
  blocks = std::max<uint64_t>(1, std::min(blocks, cap));
  kern<<<(unsigned)blocks, block, smem, st>>>(a);
  return after_launch();
}

template <int DIST, int DT>
cudaError_t launch_gen_dt(const GenArgs& a, bool bulk, const GenConfig& cfg, cudaStream_t st) {
  if (!bulk) return launch_gen_t<DIST, DT, 128, false>(a, cfg, st);
  if (cfg.chunk == 256) return launch_gen_t<DIST, DT, 256, true>(a, cfg, st);
  return launch_gen_t<DIST, DT, 128, true>(a, cfg, st);
}

}  // namespace

cudaError_t launch_generate(const DevStreams& s, uint64_t n, int dist, int dtype, double rate,
                            void* out, uint64_t ld, const GenConfig& cfg_in, cudaStream_t st) {
  if (s.n == 0 || n == 0) return cudaSuccess;
  GenConfig cfg = cfg_in;
  if (cfg.block <= 0 || cfg.block > 256 || cfg.block % 32) cfg.block = 256;
  if (cfg.chunk != 256) cfg.chunk = 128;
  const int es = dtype == MRG_F64 ? 8 : 4;
  const uint64_t ce = (uint64_t)cfg.chunk / es;
  uint64_t L = cfg.seg_len;
  if (L == 0) {
    // Heuristic: about 16 segments per resident lane slot, at least 4 chunks,
    // at most the whole row.
    const uint64_t lanes = (uint64_t)sm_count() * 2048;
    const uint64_t total = n * s.n;
    L = total / (lanes * 16);
    L = std::max<uint64_t>(L, 4 * ce);
  }
  L = (L + ce - 1) / ce * ce;                 // whole chunks (even: pairs stay aligned)
  const uint64_t ncap = (n + ce - 1) / ce * ce;
  L = std::min(L, ncap);
  GenArgs a;
  a.cur = s.cur;
  a.stride = s.stride;
  a.ns = s.n;
  a.n = n;
  a.L = L;
  a.total = s.n * ((n + L - 1) / L);
  a.out = reinterpret_cast<char*>(out);
  a.ld = ld;
  a.inv_rate = 1.0 / rate;
  const bool bulk = (reinterpret_cast<uintptr_t>(out) % 16 == 0) && ((ld * es) % 16 == 0);
  switch (dist * 4 + dtype) {
    case MRG_RAW * 4 + MRG_U32: return launch_gen_dt<MRG_RAW, MRG_U32>(a, bulk, cfg, st);
    case MRG_UNIFORM * 4 + MRG_F32: return launch_gen_dt<MRG_UNIFORM, MRG_F32>(a, bulk, cfg, st);
    case MRG_UNIFORM * 4 + MRG_F64: return launch_gen_dt<MRG_UNIFORM, MRG_F64>(a, bulk, cfg, st);
    case MRG_NORMAL * 4 + MRG_F32: return launch_gen_dt<MRG_NORMAL, MRG_F32>(a, bulk, cfg, st);
    case MRG_NORMAL * 4 + MRG_F64: return launch_gen_dt<MRG_NORMAL, MRG_F64>(a, bulk, cfg, st);
    case MRG_EXPONENTIAL * 4 + MRG_F32: return launch_gen_dt<MRG_EXPONENTIAL, MRG_F32>(a, bulk, cfg, st);
    case MRG_EXPONENTIAL * 4 + MRG_F64: return launch_gen_dt<MRG_EXPONENTIAL, MRG_F64>(a, bulk, cfg, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mrg
