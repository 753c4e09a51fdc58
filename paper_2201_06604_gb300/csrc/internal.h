// internal.h -- launchers shared by the C-ABI layer and the kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

struct mrg_request;  // include/mrg32k3a.h

namespace mrg {

struct DevStreams {
  uint32_t* cur;
  uint32_t* start;
  uint32_t* sub;
  uint64_t n;
  uint64_t stride;
};

// Launch shape of the generate kernel.  Outputs never depend on it: every
// segment starts with a jump to its absolute offset.
struct GenConfig {
  uint64_t seg_len = 0;   // draws per segment (rounded up to a multiple of 8); 0 = heuristic
  int block = 256;        // threads per block (multiple of 32, <= 256)
  int max_blocks = 0;     // 0 = fill every SM
  int vec_bytes = 32;     // widest per-lane store (32, 16, 8 or 4); alignment may lower it
  int per_sm = 0;         // resident blocks per SM the grid is sized for; 0 = occupancy maximum
};

// The launch configuration mrg_generate uses for (dist, dtype) on ns streams
// of n draws on the current device: a tuned one if the autotuner recorded
// one for that size class, else the defaults above (tune.cu).
GenConfig generate_config_for(int dist, int dtype, uint64_t ns, uint64_t n);

extern std::atomic<uint64_t> g_launches;

// Copies the jump tables into the current device's constant memory and the
// transform tables into its global memory.
cudaError_t upload_tables(const uint32_t* tab, size_t bytes);
cudaError_t upload_transform_table(const float* tab, size_t bytes);

cudaError_t launch_create(const uint32_t seed[6], uint64_t n, const DevStreams& s,
                          cudaStream_t st);

// dst0 (and dst1 if not null) <- A^(e * 2^base) src, e = e_hi * 2^64 + e_lo,
// for streams [0, ns).  Requires base + bitlen(e) <= JUMP_BITS.
cudaError_t launch_jump(const uint32_t* src, uint32_t* dst0, uint32_t* dst1, uint64_t stride,
                        uint64_t ns, uint64_t e_lo, uint64_t e_hi, int base, cudaStream_t st);

// Generates n values per stream into out (stream-major, leading dimension
// ld elements).  Does not advance the states.
cudaError_t launch_generate(const DevStreams& s, uint64_t n, int dist, int dtype, double rate,
                            void* out, uint64_t ld, const GenConfig& cfg, cudaStream_t st);

cudaError_t launch_fused(const DevStreams& s, uint64_t pairs, int64_t* count, double* sum,
                         cudaStream_t st);

// The paper's matrix layout (matrix_kernels.cuh): a g0 x g1 grid of work
// items, item t on stream t, fills an nrow x ncol row-major matrix (leading
// dimension ld); dist RAW / UNIFORM / EXPONENTIAL.
cudaError_t launch_matrix(bool g31, uint32_t* cur, uint64_t stride, uint64_t nrow, uint64_t ncol,
                          uint32_t g0, uint32_t g1, int dist, int dtype, double rate, void* out,
                          uint64_t ld, cudaStream_t st);

// out[0 .. 32 units) = the word v repeated (32-byte stores; out 32-byte aligned).
cudaError_t launch_fill(void* out, uint64_t units, uint32_t v, cudaStream_t st);

// Monte Carlo Fisher's exact test (fisher_kernels.cuh): B replicates on the
// streams of s (replicate b on stream b mod s.n); rows/cols/lf/count in
// device memory, *count accumulated (not reset), stats optional.
constexpr uint32_t kFisherMaxDim = 64;
cudaError_t launch_fisher(const DevStreams& s, const int32_t* rows, const int32_t* cols,
                          uint32_t I, uint32_t J, int32_t total, const double* lf, uint64_t B,
                          double threshold, unsigned long long* count, double* stats,
                          cudaStream_t st);

// MRG31k3p (gen31_kernels.cuh): tables, stream creation (2^134 apart), the
// advance cur <- A^k cur (k < 2^64) and materialised generation.
cudaError_t upload_tables31(const uint32_t* tab, size_t bytes);
cudaError_t upload_transform_table31(const float* tab, size_t bytes);
cudaError_t launch_create31(const uint32_t seed[6], uint64_t n, const DevStreams& s,
                            cudaStream_t st);
cudaError_t launch_jump31(uint32_t* cur, uint64_t stride, uint64_t ns, uint64_t k,
                          cudaStream_t st);
cudaError_t launch_generate31(const DevStreams& s, uint64_t n, int dist, int dtype, double rate,
                              void* out, uint64_t ld, const GenConfig& cfg, cudaStream_t st);

// Applies the output transform to caller-provided raw draws z[i] in [1, m1]
// (consecutive pairs for normals): out[i] as generate would write it.
cudaError_t launch_transform(const uint32_t* z, uint64_t n, int dist, int dtype, double rate,
                             void* out, cudaStream_t st);

// Number of SMs of the current device (cached per device).
int sm_count();

// Batched requests (batch_kernels.cuh).  Host-side mirrors of the device
// descriptors: 64-byte request and 8-byte tile records.
struct BatchReqHost {
  uint64_t out, n, off, sub, stream;
  uint32_t dist, dtype;
  float ir_hi, ir_lo;
  uint32_t L, nseg;
};
struct BatchTileHost {
  uint32_t req, g0;
};
struct BatchHeaderHost {
  unsigned long long next_tile;
  uint64_t ntiles;
};
static_assert(sizeof(BatchReqHost) == 64, "request record layout");
static_assert(sizeof(BatchTileHost) == 8, "tile record layout");

// Serving engine (serve_kernels.cuh): control block and ring record mirrors.
struct ServeCtlHost {
  alignas(128) unsigned long long head;
  alignas(128) unsigned long long tail;
  alignas(128) unsigned int stop;
  alignas(128) unsigned int status;
};
struct ServeTileHost {
  uint32_t slot, g0, ntiles, seq;
};
static_assert(sizeof(ServeTileHost) == 16, "ring record layout");
int serve_grid(double sm_fraction);
// Loads every kernel of the library on the current device (see kernels.cu).
cudaError_t preload_kernels();
cudaError_t launch_serve(void* ctl, const void* slots, const void* ring, uint64_t ring_mask,
                         unsigned int* tiles_done, unsigned int* done_words,
                         unsigned long long* head_mirror, const uint32_t* start, uint64_t stride,
                         uint64_t idle_ns, int grid, cudaStream_t st);

// Library set-up of the current device (jump and transform tables), and the
// calling thread's error text; both implemented in capi.cu.
int ensure_device_ready();
int set_error(int code, const char* msg);

// Segment length (draws per lane) of a request of `draws` draws under a
// tiling: ceil(draws / target) rounded up to whole 32-byte units (8 values),
// clamped to [seg_min, seg_max].
inline uint32_t tiled_seg_len(uint64_t draws, uint32_t seg_min, uint32_t seg_max,
                              uint64_t target) {
  uint64_t L = (draws + target - 1) / target;
  L = (L + 7) / 8 * 8;
  if (L < seg_min) L = seg_min;
  if (L > seg_max) L = seg_max;
  return (uint32_t)L;
}

// Checks one batched request against a stream set of ns streams and writes
// its device record under the tiling (seg_min, seg_max, target); *tiles
// receives its warp-tile count.  Returns MRG_OK or an MRG_E* code with the
// error text set (capi.cu).  Both batch entry points validate through it.
int prepare_request(const mrg_request& q, uint64_t ns, uint32_t seg_min, uint32_t seg_max,
                    uint64_t target, BatchReqHost* h, uint64_t* tiles);

// Range of one variant in a variant-grouped tile table (device mirror:
// VariantRange in batch_kernels.cuh), and the spacing of the per-variant
// claim counters (in 8-byte words).
struct VariantRangeHost {
  uint64_t begin, end;
};
static_assert(sizeof(VariantRangeHost) == 16, "variant range layout");
constexpr int kBatchCounterStride = 16;

// Output variants in the order the batch runner groups and launches them
// (by instruction count per output, costliest first):
//   0 normal f64, 1 normal f32, 2 exponential f64, 3 exponential f32,
//   4 uniform f32, 5 uniform f64, 6 raw u32.
constexpr int kVariants = 7;
// rank of dist * 4 + dtype in that order (9 = not a variant)
constexpr int kVariantRank[16] = {6, 9, 9, 9,  9, 4, 5, 9,  9, 1, 0, 9,  9, 3, 2, 9};

// One launch of the persistent kernel of variant k over its range of the
// tile table (ranges: kVariants records; counters: kVariants claim counters
// kBatchCounterStride words apart, zero before the launch).
cudaError_t launch_batch_variant(int k, const void* ranges, unsigned long long* counters,
                                 const void* reqs, const void* tiles, const uint32_t* start,
                                 uint64_t stride, cudaStream_t st);

// Persistent grid size of the batch kernel on the current device.
int batch_grid();
// One launch of the persistent batch kernel over the device tables.
cudaError_t launch_batch(void* hdr, const void* reqs, const void* tiles, const uint32_t* start,
                         uint64_t stride, int grid, cudaStream_t st);

}  // namespace mrg
