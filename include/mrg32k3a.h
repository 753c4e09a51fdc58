/*
 * mrg32k3a.h -- C ABI of libmrg32k3a: many independent MRG32k3a streams
 * generated by hand-written CUDA kernels for GB300 (sm_103a).
 *
 * The method (arXiv 2201.06604, "clrng: A tool set for parallel random number
 * generation on GPUs in R"):
 *   - Sec. 2.1 (Creating streams): the period of a long-period generator is cut
 *     into disjoint streams of equal length Z; a new stream starts Z steps after
 *     the previous one, a stream keeps its current and its initial state, and
 *     streams may be split into equally spaced substreams.  Here the generator
 *     is MRG32k3a (named in Sec. 1 and 2; constants of L'Ecuyer 1999, the
 *     generator of RngStreams), Z = 2^127 and the substream spacing is 2^76.
 *   - Sec. 2.2 (Generating uniform random numbers): each work item keeps its
 *     stream's state privately, draws an integer in [1, m1] per step, scales it
 *     by a constant factor and writes the state back at the end, so that the
 *     next call continues the stream.
 *   - Sec. 3.1 (Algorithm 1, Box-Muller) and Sec. 3.2 (inverse transform): the
 *     normal and exponential transforms of those uniforms.
 *   - Sec. 2.2 (saving streams with saveRDS / reloading): state checkpoint.
 *
 * Conventions shared by every entry point
 *   - Return value: MRG_OK (0) or a negative MRG_E* code; no exception crosses
 *     the ABI.  mrg_last_error() returns a text for the calling thread's last
 *     error.
 *   - Device pointers are owned by the caller (allocate them with any CUDA
 *     allocator, e.g. torch).  Host pointers are only read or written during
 *     the call unless stated otherwise.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Kernels are enqueued on it and are ordered with the caller's
 *     other work on it; calls return before the GPU work finishes unless the
 *     entry point says it synchronises.
 *   - State order inside a stream: six 32-bit words, newest first,
 *     (x1[n-1], x1[n-2], x1[n-3], x2[n-1], x2[n-2], x2[n-3]); this is the
 *     order of the paper's stream printout (Sec. 2.1, current.g1.1 .. g2.3).
 *     Valid states have x1 words < m1 = 4294967087, x2 words < m2 = 4294944443
 *     and neither triple all zero.
 */
#ifndef MRG32K3A_H
#define MRG32K3A_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define MRG_OK 0
#define MRG_EINVAL (-1)   /* bad argument: invalid seed/state, null pointer, bad dist/dtype */
#define MRG_ERANGE (-2)   /* a size, index or offset beyond what the generator supports */
#define MRG_ECUDA (-3)    /* a CUDA runtime error; see mrg_last_error() */
#define MRG_EBUSY (-4)    /* admission refused (serving queue full / over budget) */
#define MRG_ETIMEOUT (-5) /* a bounded device or host wait gave up */

/* ---- distributions and output types ----------------------------------- */
#define MRG_RAW 0         /* z in [1, m1] as uint32 (runifGpu type "integer", Sec. 2.2) */
#define MRG_UNIFORM 1     /* u = RN64(z * norm), norm = RN64(1/(m1+1)); fp32 = RN32(u) */
#define MRG_NORMAL 2      /* Box-Muller on consecutive pairs of one stream (Sec. 3.1) */
#define MRG_EXPONENTIAL 3 /* -ln(z/(m1+1)) / rate (Sec. 3.2, printed-values reading) */

#define MRG_U32 0
#define MRG_F32 1
#define MRG_F64 2

/* A set of streams in device memory, structure of arrays.  Word k of stream
 * i lives at ptr[k * stride + i] (k = 0..5), stride >= n.  `cur` is the
 * current state, `start` the stream's initial state (Sec. 2.1 "initial
 * state"), `sub` the start of the current substream.  A view of streams
 * [a, a + m) of a larger set is {cur + a, start + a, sub + a, m, stride}. */
typedef struct mrg_streams {
    uint32_t *cur;
    uint32_t *start;
    uint32_t *sub;
    uint64_t n;
    uint64_t stride;
} mrg_streams;

/* Text of the calling thread's last error ("" if none). */
const char *mrg_last_error(void);

/* Number of kernels this library has launched since it was loaded. */
uint64_t mrg_launch_count(void);

/* Library version string. */
const char *mrg_version(void);

/* Checks a seed / state: x1 words < m1, x2 words < m2, neither triple all
 * zero.  Returns MRG_OK or MRG_EINVAL. */
int mrg_seed_check(const uint32_t seed[6]);

/* The creator state after n_streams streams: seed advanced n_streams * 2^127
 * steps -- the next_seed of mrg_create_streams -- computed on the host,
 * creating no stream and touching no device (Sec. 2.1: each new stream jumps
 * ahead from the previous one).  For example the seed of a shard whose
 * streams start n_streams into the creator's sequence.  out (host) receives
 * the six words; it may alias seed.  Errors: MRG_EINVAL (seed invalid, seed
 * or out NULL), MRG_ERANGE (n_streams > 2^63). */
int mrg_creator_advance(const uint32_t seed[6], uint64_t n_streams, uint32_t out[6]);

/* Creates n streams from the creator state `seed` (Sec. 2.1 setBaseCreator /
 * createStreamsGpu): stream i starts i * 2^127 steps after seed, exactly as if
 * the streams had been created one after another.  Writes cur = start = sub
 * for streams 0..n-1 of `s` (s->n must be >= n), computed in parallel on the
 * device.  next_seed (host, may be NULL) receives the creator state after the
 * n-th stream, i.e. seed advanced n * 2^127 steps, so the next creation call
 * continues the sequence.  Errors: MRG_EINVAL (seed invalid, s or its
 * pointers NULL with n > 0, n > s->n), MRG_ERANGE (n >= 2^64 streams is not
 * representable; n > 2^63 rejected), MRG_ECUDA. */
int mrg_create_streams(const uint32_t seed[6], uint64_t n, const mrg_streams *s,
                       uint32_t next_seed[6], void *stream);

/* Generates n_per_stream values from every stream of `s` into the device
 * array out, stream-major: value i of stream j at out[j * ld + i], ld >= n.
 * dist / dtype: MRG_RAW with MRG_U32; MRG_UNIFORM, MRG_NORMAL or
 * MRG_EXPONENTIAL with MRG_F32 or MRG_F64.  rate is the exponential rate
 * (in [2^-64, 2^64]; ignored otherwise).  Raw and uniform outputs are
 * bit-exact functions of the state; normals and exponentials are within
 * 1e-12 absolute (fp64; exponentials 1e-12 / min(rate, 1)) or 2 ulp of the
 * fp32 spacing (fp32) of the exact transform of the same integers, evaluated
 * in double-float arithmetic on the FP32 pipe.  Each stream's
 * `cur` advances by the draws consumed: n for raw, uniform and exponential,
 * n + (n mod 2) for normals (an odd count discards the last sine output), so
 * the next call continues each stream exactly (Sec. 2.2).  The output does
 * not depend on the launch configuration.  out must not overlap the states.
 * Errors: MRG_EINVAL (bad dist/dtype pair, rate outside [2^-64, 2^64] for
 * exponentials, ld < n, NULL pointers, out not aligned to its element),
 * MRG_ECUDA. */
int mrg_generate(const mrg_streams *s, uint64_t n_per_stream, int dist, int dtype,
                 double rate, void *out, uint64_t ld, void *stream);

/* mrg_generate into HOST memory: value i of stream j at out_host[j * ld + i]
 * (out_host should be pinned for full copy bandwidth).  The streams are cut
 * into chunks that fit half of `scratch` (caller-owned device memory,
 * scratch_bytes >= 2 * n * element size); chunk c is generated on `stream`
 * into one half while chunk c-1 is copied to the host from the other half on
 * a second stream of the library, so generation overlaps the device-to-host
 * copy.  Same outputs and state updates as mrg_generate.  Synchronises: the
 * data is on the host when the call returns.  Errors: as mrg_generate, plus
 * MRG_EINVAL when scratch is NULL or too small for one stream per half. */
int mrg_generate_host(const mrg_streams *s, uint64_t n_per_stream, int dist, int dtype,
                      double rate, void *out_host, uint64_t ld, void *scratch,
                      uint64_t scratch_bytes, void *stream);

/* Applies the output transform of mrg_generate to caller-provided raw draws:
 * z (device, n values in [1, m1], e.g. from MRG_RAW) -> out (device, n values
 * of dtype).  MRG_UNIFORM, MRG_NORMAL (consecutive pairs (z[2k], z[2k+1]) give
 * out[2k] = X, out[2k+1] = Y; an odd n computes the last X from (z[n-1], 1)) or
 * MRG_EXPONENTIAL with MRG_F32 / MRG_F64, same accuracy as mrg_generate.
 * Values of z outside [1, m1] give unspecified (but memory-safe) outputs.
 * The outputs are bit-identical to mrg_generate's for the same draws,
 * whatever the alignment of out (an out aligned to four outputs takes the
 * packed evaluation, bit-identical to the one-at-a-time one).
 * Errors: MRG_EINVAL (NULL pointers with n > 0, bad dist/dtype or rate, out
 * not aligned to its element size or z not to 4 bytes), MRG_ECUDA. */
int mrg_transform(const uint32_t *z, uint64_t n, int dist, int dtype, double rate, void *out,
                  void *stream);

/* Advances every stream's `cur` by k = k_hi * 2^64 + k_lo steps (jump-ahead
 * by a matrix power, Sec. 2.1).  `start` and `sub` are unchanged.
 * Errors: MRG_EINVAL, MRG_ECUDA. */
int mrg_skip(const mrg_streams *s, uint64_t k_hi, uint64_t k_lo, void *stream);

/* Moves every stream to the start of its next substream: sub += 2^76 steps,
 * cur = sub (RngStreams' ResetNextSubstream; substreams, Sec. 2.1). */
int mrg_substream_next(const mrg_streams *s, void *stream);

/* cur = sub (back to the start of the current substream). */
int mrg_reset_substream(const mrg_streams *s, void *stream);

/* cur = sub = start (back to the stream's initial state, Sec. 2.1). */
int mrg_reset_stream(const mrg_streams *s, void *stream);

/* Checkpoint (Sec. 2.2, saving streams to a file and reloading them): copies
 * the three state arrays to host memory laid out as [3][6][n] uint32
 * (cur, start, sub; word k of stream i at [a][k][i]).  Synchronises
 * `stream`.  host must hold 18 * n words.  Errors: MRG_EINVAL, MRG_ECUDA. */
int mrg_get_state(const mrg_streams *s, uint32_t *host, void *stream);

/* Restores states saved by mrg_get_state.  Every state is validated first
 * (MRG_EINVAL and nothing is written if one is invalid).  Synchronises
 * `stream`. */
int mrg_set_state(const mrg_streams *s, const uint32_t *host, void *stream);

/* Fused consumer with no stored draws: for every stream, `draws` draws are
 * taken as draws/2 pairs (za, zb) (an odd count is rounded up to whole
 * pairs).  count[i] = number of pairs with (za/M)^2 + (zb/M)^2 < 1,
 * M = m1 + 1, decided exactly in integers; sum[i] = sum over the pairs of
 * X + Y, the Box-Muller normals of the same pair (Sec. 3.1).  count and sum
 * are device arrays of s->n elements.  Each stream's cur advances by the
 * draws consumed.  Counts are exact; sums are within 1e-9 of the exact sum
 * relative to the sum of |X| + |Y|.  Errors: MRG_EINVAL, MRG_ECUDA. */
int mrg_fused_pi_normsum(const mrg_streams *s, uint64_t draws, int64_t *count, double *sum,
                         void *stream);

/* ---- the paper's matrix layout (compatibility mode) --------------------- */

#define MRG_GEN_MRG32K3A 0
#define MRG_GEN_MRG31K3P 1

/* runifGpu / rexpGpu with an explicit work-item grid (Sec. 2.2, Listing 1;
 * Sec. 3.2): a gsize0 x gsize1 grid of work items (the paper's Nglobal) fills
 * the nrow x ncol row-major matrix out (device; element (r, c) at
 * out[r * ld + c]).  Work item (i0, i1) uses stream i0 * gsize1 + i1 of `s`
 * (s->n >= gsize0 * gsize1) and visits rows i0, i0 + gsize0, ... and, in
 * each, columns i1, i1 + gsize1, ... of the matrix padded to
 * ceil(ncol / gsize1) * gsize1 columns, taking one draw per visited position
 * and writing only the real columns; a vector of n values is the n x 1
 * matrix.  This is the reading under which the paper's printed runifGpu and
 * rexpGpu examples are reproduced (its text and listings disagree on the
 * stream map and the padding).  generator: MRG_GEN_MRG32K3A or
 * MRG_GEN_MRG31K3P (the paper's).  dist: MRG_RAW (MRG_U32), MRG_UNIFORM or
 * MRG_EXPONENTIAL (MRG_F32 / MRG_F64); normals are refused (the paper pairs
 * two work items' streams for them, tying values to the grid -- mrg_generate
 * pairs draws within a stream).  Unlike mrg_generate the output depends on
 * the grid, and each work item runs on one thread (no memory-bandwidth
 * design).  Errors: MRG_EINVAL, MRG_ERANGE, MRG_ECUDA. */
int mrg_generate_matrix(const mrg_streams *s, int generator, uint64_t nrow, uint64_t ncol,
                        uint32_t gsize0, uint32_t gsize1, int dist, int dtype, double rate,
                        void *out, uint64_t ld, void *stream);

/* ---- write-bandwidth calibration ---------------------------------------- */

/* Fills out[0 .. n_words) (device, 32-byte aligned, n_words a multiple of 8)
 * with `value`, every warp writing its own contiguous chunk 1 KiB per store
 * instruction (the fastest write-only pattern measured): a write-only stream
 * whose bandwidth is the ceiling the materialised generation is measured
 * against.  Not part of the paper's method.  Errors: MRG_EINVAL, MRG_ECUDA. */
int mrg_fill_u32(void *out, uint64_t n_words, uint32_t value, void *stream);

/* ---- Monte Carlo Fisher's exact test (Sec. 4) ---------------------------- */

/* Bytes of device scratch mrg_fisher_sim needs for a table whose entries sum
 * to n_total: a 1 KiB header and the log-factorials 0..n_total (fp64). */
uint64_t mrg_fisher_scratch_bytes(uint64_t n_total);

/* Simulated p-value of Fisher's exact test for an I x J contingency table
 * (host, int32, row-major, entries >= 0, total < 2^24, 2 <= I, J <= 64), as
 * Sec. 4 describes it: B random tables with the observed margins, each
 * sampled row by row, left to right, every cell drawn from its
 * hypergeometric distribution conditional on the cells before it by
 * inversion with one fp64 uniform (Patefield's method; (I-1)(J-1) draws per
 * table), and the statistic -sum log(n_ij!) of each.  Replicate b runs on
 * stream b mod s->n, taking that stream's next draws; each stream advances
 * by the draws its replicates consumed, so later calls continue it.
 * *count (host) receives the number of replicates whose statistic is at or
 * below the observed one (with a relative allowance of 64 ulp, so that ties
 * count whatever their rounding).  *p_value (host, may be NULL) receives the
 * simulated p-value (1 + *count) / (B + 1) (Sec. 4).  *threshold (host, may
 * be NULL) receives that bound.  stats (device, B
 * doubles, may be NULL) receives every replicate's statistic.  scratch:
 * caller-owned device memory, 256-byte aligned, at least
 * mrg_fisher_scratch_bytes(total) bytes.  Synchronises `stream`.  Errors:
 * MRG_EINVAL (shape, entries, NULL pointers, scratch too small), MRG_ERANGE
 * (total not below 2^24), MRG_ECUDA. */
int mrg_fisher_sim(const mrg_streams *s, const int32_t *table, uint32_t I, uint32_t J,
                   uint64_t B, void *scratch, uint64_t scratch_bytes, double *stats,
                   uint64_t *count, double *threshold, double *p_value, void *stream);

/* ---- MRG31k3p, the paper's own generator --------------------------------
 * The package of the paper is built on MRG31k3p (L'Ecuyer and Touzin 2000;
 * Sec. 2): x1[n] = (2^22 x1[n-2] + (2^7 + 1) x1[n-3]) mod (2^31 - 1),
 * x2[n] = (2^15 x2[n-1] + (2^15 + 1) x2[n-3]) mod (2^31 - 21069),
 * z = (x1 - x2) mod (2^31 - 1) with 0 mapped to 2^31 - 1 (an integer in
 * [1, 2^31 - 1], Sec. 2.2), uniforms u = z / 2^31 (exact in fp64; fp32 =
 * RN32(u)), streams 2^134 steps apart (Sec. 2.1).  Its streams use the same
 * mrg_streams layout and word order as MRG32k3a's; the paper prints this
 * generator's stream starts (Sec. 2.1), uniforms (Sec. 2.2) and
 * exponentials (Sec. 3.2).  mrg_get_state, mrg_set_state, mrg_reset_stream
 * and mrg_reset_substream serve both generators (they copy words); the other
 * MRG32k3a entry points apply MRG32k3a's matrices and must not be given
 * MRG31k3p streams.  */

/* x1 words < 2^31 - 1, x2 words < 2^31 - 21069, neither triple all zero. */
int mrg31k3p_seed_check(const uint32_t seed[6]);

/* mrg_creator_advance for MRG31k3p: seed advanced n_streams * 2^134 steps,
 * on the host.  Errors: as mrg_creator_advance. */
int mrg31k3p_creator_advance(const uint32_t seed[6], uint64_t n_streams, uint32_t out[6]);

/* mrg_create_streams for MRG31k3p: stream i starts i * 2^134 steps after
 * seed (Sec. 2.1, createStreamsGpu); next_seed (may be NULL) receives the
 * creator state after n streams.  Errors: as mrg_create_streams. */
int mrg31k3p_create_streams(const uint32_t seed[6], uint64_t n, const mrg_streams *s,
                            uint32_t next_seed[6], void *stream);

/* mrg_generate for MRG31k3p streams (Sec. 2.2 runifGpu, Sec. 3.1 rnormGpu,
 * Sec. 3.2 rexpGpu): the same layout, variants, draw accounting and state
 * advance; normals and exponentials are the transforms of u = z / 2^31 with
 * the accuracy stated for mrg_generate.  Errors: as mrg_generate. */
int mrg31k3p_generate(const mrg_streams *s, uint64_t n_per_stream, int dist, int dtype,
                      double rate, void *out, uint64_t ld, void *stream);

/* Advances every MRG31k3p stream's cur by k < 2^64 steps. */
int mrg31k3p_skip(const mrg_streams *s, uint64_t k, void *stream);

/* ---- launch shape and its autotuner ------------------------------------ */

/* Launch shape of the generate kernel.  It changes how the work is cut, never
 * the output: every lane segment starts with a jump to its absolute offset
 * in the stream (Sec. 2.1 jump-ahead), so any shape writes the same bytes. */
typedef struct mrg_launch_config {
    uint64_t seg_len;       /* draws per lane segment, rounded up to a multiple of 8
                               and capped at the row; 0 = library heuristic */
    uint32_t block;         /* threads per block: a multiple of 32, <= 256; 0 = 256 */
    uint32_t vec_bytes;     /* widest per-lane store: 32, 16, 8 or 4 bytes; 0 = 32.  The
                               alignment of out and of the row pitch may lower it */
    uint32_t blocks_per_sm; /* resident blocks per SM the grid is sized for (<= 64);
                               0 = the occupancy maximum */
    uint32_t reserved;      /* set to 0 */
} mrg_launch_config;

/* One timed candidate of the autotuner: its shape and the mean kernel time. */
typedef struct mrg_tune_entry {
    mrg_launch_config cfg;
    float ms;
} mrg_tune_entry;

/* mrg_generate with an explicit launch shape (cfg, host, read during the
 * call).  Same outputs and state updates as mrg_generate.  Errors: those of
 * mrg_generate, and MRG_EINVAL for a cfg outside the ranges above. */
int mrg_generate_config(const mrg_streams *s, uint64_t n, int dist, int dtype, double rate,
                        void *out, uint64_t ld, const mrg_launch_config *cfg, void *stream);

/* Autotuner: times the generate kernel for (s, n, dist, dtype, rate, out, ld)
 * under the library default and a set of candidate shapes (segment lengths
 * 256 .. 16384 draws x blocks of 128 / 256 threads x 32- / 16-byte stores),
 * each warmed up once and then launched `reps` times (0 = 3, at most 100)
 * between two CUDA events on `stream`.  Records the fastest for the current
 * device and the size class (dist, dtype, bit length of s->n * n, bit length
 * of n); later mrg_generate calls of that class launch with it.  The stream
 * states are not advanced; out receives the values mrg_generate would write.
 * results (host, may be NULL if max_results is 0) receives up to max_results
 * timed candidates, *n_results their number, *best (may be NULL) the chosen
 * shape.  Synchronises `stream`.  Not an optimisation the paper describes:
 * its kernels have a fixed shape (Sec. 2.2).  Errors: as mrg_generate, and
 * MRG_EINVAL for n or s->n equal to 0. */
int mrg_tune_generate(const mrg_streams *s, uint64_t n, int dist, int dtype, double rate,
                      void *out, uint64_t ld, uint32_t reps, mrg_tune_entry *results,
                      uint32_t max_results, uint32_t *n_results, mrg_launch_config *best,
                      void *stream);

/* The shape mrg_generate uses on the current device for this size class
 * (all fields 0 except block = 256 and vec_bytes = 32 when nothing is tuned). */
int mrg_tune_lookup(int dist, int dtype, uint64_t n_streams, uint64_t n, mrg_launch_config *cfg);

/* Records cfg for the size class on the current device (e.g. a shape saved
 * from an earlier process); cfg = NULL removes the entry. */
int mrg_tune_set(int dist, int dtype, uint64_t n_streams, uint64_t n, const mrg_launch_config *cfg);

/* Forgets every tuned shape on every device. */
void mrg_tune_clear(void);

/* ---- batched requests (one persistent, graph-captured launch) ----------- */

/* One generation request at an absolute position of one stream: draws start
 * `offset` draws after the start of substream `substream` of stream `stream`
 * (i.e. start + substream * 2^76 + offset; substreams, Sec. 2.1), and n
 * outputs of (dist, dtype) go to `out` (device, 32-byte aligned, n elements).
 * Normals consume n + (n mod 2) draws.  The output is a function of the
 * request alone: it does not depend on the other requests of the batch, their
 * order or the launch configuration, and equals what mrg_generate writes for
 * a single stream positioned at the same draw. */
typedef struct mrg_request {
    uint64_t stream;
    uint64_t substream; /* < 2^51 */
    uint64_t offset;    /* offset + draws consumed <= 2^62 (inside the substream) */
    uint64_t n;
    int32_t dist;
    int32_t dtype;
    double rate;        /* exponentials: in [2^-64, 2^64] */
    void *out;
} mrg_request;

/* How the batch runner and the serving engine cut requests into work: a
 * request of n draws gets lane segments of
 *   L = clamp(ceil(n / target_segments) rounded up to a multiple of 8,
 *             seg_min, seg_max)
 * draws, and 32 consecutive segments of one request form a warp tile.  Short
 * segments spread a request over more lanes; long ones amortise the jump
 * that starts every segment.  Outputs never depend on the tiling (every
 * segment jumps to its absolute position).  Valid: 8 <= seg_min <= seg_max
 * <= 2^20, both multiples of 8, target_segments >= 1. */
typedef struct mrg_tiling {
    uint32_t seg_min;
    uint32_t seg_max;
    uint64_t target_segments;
} mrg_tiling;

/* One timed tiling of mrg_batch_tune: the tiling, its tile count and the
 * mean time of one batch launch. */
typedef struct mrg_batch_tune_entry {
    mrg_tiling tiling;
    uint64_t tiles;
    float ms;
} mrg_batch_tune_entry;

typedef struct mrg_batch mrg_batch; /* opaque */

/* Creates a batch runner for the streams of `s` (their `start` arrays are
 * read; no state is written) holding up to max_requests requests and
 * max_tiles tiles (a tile = up to 32 segments of one request; under the
 * default tiling a request of n draws takes about ceil(n / 8192) tiles, at
 * least one).  Allocates its device tables and pinned host staging, and
 * captures one CUDA graph [tables and claim counters host->device, then one
 * persistent kernel per output variant, each a programmatic dependent of the
 * previous one] on a stream of its own.
 * Errors: MRG_EINVAL, MRG_ECUDA. */
int mrg_batch_create(const mrg_streams *s, uint32_t max_requests, uint64_t max_tiles,
                     mrg_batch **out, void *stream);

/* Runs nreq requests with one graph launch on `stream` (asynchronous; the
 * outputs are ready when `stream` reaches the end of the launch).  Waits for
 * the previous run of the same batch object to finish with its host tables.
 * Errors: MRG_EINVAL (bad request: stream index, dist/dtype, rate, NULL or
 * unaligned out), MRG_ERANGE (substream >= 2^51, offset + draws > 2^62, more
 * requests or tiles than the batch holds), MRG_ECUDA. */
int mrg_batch_run(mrg_batch *b, const mrg_request *reqs, uint32_t nreq, void *stream);

/* Sets the tiling of later runs of this batch object (t = NULL restores the
 * default {8, 256, 32}: about one warp of segments per request, at most
 * 256 draws per lane, so that no tile outlasts the rest of the batch by much).  Errors: MRG_EINVAL (tiling outside the ranges of
 * mrg_tiling). */
int mrg_batch_set_tiling(mrg_batch *b, const mrg_tiling *t);

/* The tiling later runs of this batch object use. */
int mrg_batch_get_tiling(const mrg_batch *b, mrg_tiling *t);

/* Autotuner of the batch tiling: runs the nreq requests (they must be valid
 * for mrg_batch_run, and their outputs are written) under the current
 * tiling and a set of candidates (seg_min 8 / 64 x seg_max 128 / 256 / 512 /
 * 2048 x target_segments 32 / 256 / 2048, skipping those whose tiles exceed the
 * batch's capacity), each warmed up once and then launched `reps` times
 * (0 = 3, at most 100) between CUDA events on `stream`, and keeps the
 * fastest as the batch's tiling.  results (may be NULL if max_results is 0)
 * receives up to max_results timed tilings, *n_results their number, *best
 * (may be NULL) the chosen one.  Synchronises `stream`.  Not an optimisation
 * the paper describes.  Errors: as mrg_batch_run. */
int mrg_batch_tune(mrg_batch *b, const mrg_request *reqs, uint32_t nreq, uint32_t reps,
                   mrg_batch_tune_entry *results, uint32_t max_results, uint32_t *n_results,
                   mrg_tiling *best, void *stream);

/* Number of tiles the last mrg_batch_run built. */
uint64_t mrg_batch_last_tiles(const mrg_batch *b);

/* Frees the batch object (synchronises its last run). */
int mrg_batch_destroy(mrg_batch *b);

/* The requests of a batch run one by one with the plain kernels, from a host
 * loop: for each request, one jump kernel sets its stream's `cur` to
 * start * A^(substream * 2^76 + offset) and one generate kernel writes its n
 * values -- two launches per request, the launch-by-launch way a caller
 * without mrg_batch_run would serve the same requests (Sec. 2.1 streams and
 * substreams, Sec. 2.2 generation).  Same outputs as mrg_batch_run.  Leaves
 * the `cur` of every requested stream at the start of its last request.
 * Requests are validated as mrg_batch_run validates them, before any launch.
 * Errors: as mrg_batch_run. */
int mrg_batch_run_plain(const mrg_streams *s, const mrg_request *reqs, uint32_t nreq,
                        void *stream);

/* mrg_batch_run for callers that cannot allocate device memory -- plug-ins
 * whose host application owns the device-memory budget through its own
 * allocator, loops that cannot afford cudaMalloc's implicit synchronisation.
 * It allocates nothing: the request table, tile table and
 * claim counter live in a fixed device array of 192.25 KiB inside the
 * library, which every GPU that loads the library holds until the process
 * exits.  Limits per call: 1024 requests and 16384 tiles (a tile holds up to
 * 32 segments of one request; a request of n draws takes about
 * ceil(n / 65536) tiles, at least one); larger calls, and a request of 2^32
 * or more segments, fail with MRG_ERANGE and run nothing.  Requests are
 * validated exactly as mrg_batch_run validates them.  Tiles run in one
 * persistent kernel for all output variants, longest segments first; the
 * per-variant kernels of mrg_batch_run are faster on large mixed batches.  The first call on a device does the set-up (the library's
 * tables and the device address of the array), so make it before any stream
 * capture.  All calls share the array: calls whose work overlaps on the GPU
 * (different CUDA streams, or several host threads) race; calls ordered on
 * one stream are safe.  Outputs are those of mrg_batch_run.  The paper has
 * no counterpart of this entry point.  Errors: as mrg_batch_run. */
int mrg_batch_run_static(const mrg_streams *s, const mrg_request *reqs, uint32_t nreq,
                         void *stream);

/* ---- serving engine: continuous batching into one persistent worker ---- */

typedef struct mrg_server mrg_server; /* opaque */

/* Starts a server over the streams of `s` (their `start` arrays are read):
 * a persistent worker kernel that processes requests appended to a ring while
 * it runs.  sm_fraction in (0, 1] is the share of every SM's resident blocks
 * the worker takes: 1 gives it the whole GPU (kernels of other streams then
 * wait until the worker stops); smaller values leave room for them.  Outputs
 * are placed in `arena` (caller-owned device memory, 256-byte aligned,
 * arena_bytes long).  max_slots bounds the requests in flight, ring_tiles (a
 * power of two) the tiles published and not yet finished (a request of n
 * draws takes about min(8192, n / 1024) tiles of up to 32 segments).  The worker exits by itself after
 * idle_seconds with no published work (a host that stopped feeding it);
 * later calls then report MRG_ETIMEOUT until mrg_server_restart.  While the
 * worker runs, a device-wide synchronisation (cudaDeviceSynchronize) waits
 * for it, and so can the first launch of a kernel that the process has not
 * loaded yet (CUDA's lazy module loading): the library loads its own kernels
 * at set-up; warm up other kernels first or set CUDA_MODULE_LOADING=EAGER.
 * Errors: MRG_EINVAL, MRG_ECUDA. */
int mrg_server_create(const mrg_streams *s, void *arena, uint64_t arena_bytes,
                      uint32_t max_slots, uint64_t ring_tiles, double idle_seconds,
                      double sm_fraction, mrg_server **out);

/* Admits a request (its `out` field is ignored: the server places the output
 * in the arena and returns its device address in *out, may be NULL).  The
 * request is appended to the running worker at once; its output is that of
 * mrg_batch_run for the same request.  *id identifies it in poll/release.
 * The request's tiles enter the worker's ring in chunks, round-robin with the
 * other requests in flight, on this call and on every later submit and poll:
 * keep polling while requests are in flight.
 * A request starts entering the ring, in arrival order, once the ring can
 * hold all of its tiles beside the tiles still to come of the requests
 * already started (so every started request can finish).
 * Errors: MRG_EBUSY (no free slot or arena memory -- retry after releasing
 * finished requests), MRG_EINVAL, MRG_ERANGE (larger than the arena, or more
 * tiles than ring_tiles),
 * MRG_ETIMEOUT (the worker has stopped), MRG_ECUDA. */
int mrg_server_submit(mrg_server *sv, const mrg_request *req, uint64_t *id, void **out);

/* Writes up to max_ids ids of requests that finished since the last poll to
 * ids[0..*count).  A finished request's output is complete in device memory
 * for any work the caller orders after this call.  Returns MRG_ETIMEOUT if
 * the worker stopped (idle limit), MRG_ECUDA on a device error. */
int mrg_server_poll(mrg_server *sv, uint64_t *ids, uint32_t max_ids, uint32_t *count);

/* The client's acknowledgement of a finished request: frees its slot and its
 * arena memory.  MRG_EBUSY if it has not finished, MRG_EINVAL if unknown. */
int mrg_server_release(mrg_server *sv, uint64_t id);

/* Sets the tiling of requests admitted from now on (t = NULL restores the
 * default {32, 128, 8192}: short segments, so that a request that arrives
 * while others run waits for about one short tile).  Errors: MRG_EINVAL. */
int mrg_server_set_tiling(mrg_server *sv, const mrg_tiling *t);

/* Requests admitted and not yet finished. */
uint64_t mrg_server_inflight(mrg_server *sv);

/* Relaunches a worker that stopped (idle limit); requests that were in flight
 * are dropped (their slots and memory freed).  No-op while it runs. */
int mrg_server_restart(mrg_server *sv);

/* Stops the worker once every admitted request has been processed, waits for
 * it and frees the server (the arena stays the caller's). */
int mrg_server_destroy(mrg_server *sv);

/* ---- Gaussian random fields by direct matrix decomposition ---------------
 * Sec. 5, Algorithm 2: (1) the Matern covariance matrix of the locations,
 * (2) Sigma = L D L^T with L unit lower triangular, (3) standard normals Z
 * from the generator (mrg_generate with MRG_NORMAL), (4) U = L D^(1/2) Z.
 * Matrices are row-major fp64 in device memory, matrix b of a batch at
 * base + b * n * ld; a batch runs in parallel. */

/* One parameter set of the Matern covariance of Sec. 5:
 *   Sigma_ij = variance * 2^(1-shape) / Gamma(shape) * x^shape K_shape(x),
 *   x = sqrt(8 shape) |d_ij| / range,
 *   d_ij = diag(1, aniso_ratio) R(aniso_angle) (x_i - x_j),
 *   R(t) = [[cos t, -sin t], [sin t, cos t]],
 * and Sigma_ii = variance.  The printed normalising constant 2^(shape-1) is
 * read as 2^(1-shape), the only one for which var(U_i) = variance (the
 * paper's stated property).  Valid: 0 < shape <= 10, range > 0,
 * variance > 0, aniso_ratio >= 1, finite angle (radians). */
typedef struct mrg_matern_params {
    double shape, range, variance, aniso_ratio, aniso_angle;
} mrg_matern_params;

/* Bytes of device scratch mrg_grf_matern_raster needs (a 4 KiB parameter
 * block and one covariance value per cell offset and matrix). */
uint64_t mrg_grf_matern_scratch_bytes(uint32_t batch, uint32_t nrow, uint32_t ncol);

/* Algorithm 2 step 1 for a raster of nrow x ncol square cells of side
 * `cell` (the paper's maternBatch on a raster): point k is the centre of the
 * cell in column k mod ncol and row k div ncol, at ((c + 1/2) cell,
 * (r + 1/2) cell).  Writes the full n x n covariance matrix (n = nrow ncol,
 * leading dimension ld >= n) of every parameter set params[0 .. batch)
 * (host) into cov (device, matrix b at cov + b n ld).  On a raster the
 * covariance depends only on the cell offset, so each of the
 * (2 nrow - 1)(2 ncol - 1) offsets is evaluated once (K by the trapezoidal
 * rule on its integral representation, ~1e-13 relative) and the matrix is
 * filled from that table.  scratch: device, 256-byte aligned, at least
 * mrg_grf_matern_scratch_bytes bytes.  Synchronises `stream` once (the
 * parameters are staged through it).  Errors: MRG_EINVAL (NULL, batch not in
 * 1..64, bad parameters, ld < n, alignment, scratch too small), MRG_ERANGE
 * (n > 2^20), MRG_ECUDA. */
int mrg_grf_matern_raster(const mrg_matern_params *params, uint32_t batch, uint32_t nrow,
                          uint32_t ncol, double cell, double *cov, uint64_t ld, void *scratch,
                          uint64_t scratch_bytes, void *stream);

/* Algorithm 2 step 1 for arbitrary locations xy (device, n x 2: x then y of
 * each point): every entry evaluated on its own.  scratch: device, 256-byte
 * aligned, >= 4096 bytes.  Synchronises `stream` once.  Errors: as
 * mrg_grf_matern_raster. */
int mrg_grf_matern_points(const mrg_matern_params *params, uint32_t batch, const double *xy,
                          uint64_t n, double *cov, uint64_t ld, void *scratch,
                          uint64_t scratch_bytes, void *stream);

/* Bytes of device workspace mrg_grf_ldl needs for `batch` matrices of order n
 * (the bf16 operand slices of one panel, ~4.2 KiB per row and matrix). */
uint64_t mrg_grf_ldl_workspace_bytes(uint64_t n, uint32_t batch);

/* Algorithm 2 step 2: Sigma = L D L^T in place for `batch` symmetric positive
 * definite matrices (device, matrix b at a + b n lda; only the lower
 * triangle is read).  On return the strict lower triangle holds L (its unit
 * diagonal implied), the diagonal holds D, and d (device, batch x n) holds D
 * too; the strict upper triangle is overwritten with scratch values.  A
 * right-looking blocked factorisation with 128-column panels: each 128 x 128
 * diagonal block is factored in double-float arithmetic by one CTA per
 * matrix; the panel L_ik = A_ik L_kk^-T D^-1 and the trailing update
 * A_ij -= L_ik D L_jk^T are fp64 products evaluated on the tensor cores
 * (tcgen05) by an error-free split of every operand row into eight bf16
 * slices of a 56-bit fixed-point form (the Ozaki scheme), summed exactly in
 * integers and rounded once to fp64.  workspace: device, 1024-byte aligned,
 * >= mrg_grf_ldl_workspace_bytes(n, batch).  info (host, batch entries, may
 * be NULL): when given, the call synchronises `stream` and info[b] receives
 * 0, or 1 + the index of the first pivot of matrix b that was not positive
 * (its factor is then invalid); without it the call returns as soon as the
 * kernels are enqueued.  Errors: MRG_EINVAL (NULL, batch not in 1..255,
 * lda < n, alignment, workspace too small), MRG_ERANGE (n > 2^20),
 * MRG_ETIMEOUT (a bounded tensor-core wait gave up; only reported with
 * info), MRG_ECUDA. */
int mrg_grf_ldl(double *a, uint64_t n, uint64_t lda, uint32_t batch, double *d, void *workspace,
                uint64_t workspace_bytes, int32_t *info, void *stream);

/* Bytes of device scratch mrg_grf_simulate needs (D^(1/2) Z). */
uint64_t mrg_grf_simulate_scratch_bytes(uint64_t n, uint32_t nsim, uint32_t batch);

/* Algorithm 2 step 4: U = L D^(1/2) Z for nsim columns of standard normals
 * per matrix.  l (device): the factor written by mrg_grf_ldl (strict lower
 * triangle read, unit diagonal implied); d (device, batch x n); z and u
 * (device) are [batch][nsim][n]: simulation s of matrix b is the contiguous
 * vector at z + (b nsim + s) n -- the layout of mrg_generate's normals on
 * batch * nsim streams of n draws.  fp64 throughout.  scratch: device,
 * >= mrg_grf_simulate_scratch_bytes.  Errors: MRG_EINVAL, MRG_ERANGE
 * (n > 2^20 or nsim > 2^16), MRG_ECUDA. */
int mrg_grf_simulate(const double *l, const double *d, uint64_t n, uint64_t lda, uint32_t batch,
                     const double *z, uint32_t nsim, double *u, void *scratch,
                     uint64_t scratch_bytes, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MRG32K3A_H */
