// grf.cu -- C-ABI entry points and launchers of the Gaussian-random-field
// path (Sec. 5, Algorithm 2): Matern covariance matrices, their batched
// LDL^T factorisation on the tensor cores, and U = L D^(1/2) Z.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/mrg32k3a.h"
#include "grf_kernels.cuh"
#include "internal.h"

namespace {

using namespace mrg::grf;

constexpr int kSlices = 8;             // bf16 slices per fp64 operand (56-bit fixed point)
constexpr uint32_t kMaxBatch = 64;     // matrices per call (parameters travel by value)

struct ParamBlock {
  MaternParams p[kMaxBatch];
};

uint64_t align_up(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

// Per-matrix workspace layout of the factorisation (bytes, 1024-aligned
// parts).  The operand images of the panel and trailing products exist twice:
// step k writes set k mod 2 while the bulk of step k - 1's trailing update
// still reads the other.
struct LdlLayout {
  uint64_t img_a[2], img_w[2], img_x, bx, exp_a[2], exp_w[2], exp_x, exp_eq, per_matrix, common;
  explicit LdlLayout(uint64_t n) {
    const uint64_t ta = (n + RB_A - 1) / RB_A;
    uint64_t o = 0;
    for (int q = 0; q < 2; ++q) {
      img_a[q] = o;
      o += ta * kSlices * SLICE_A;
      img_w[q] = o;
      o += 2 * ta * kSlices * SLICE_B;
    }
    img_x = o;
    o += 2 * kSlices * SLICE_B;
    bx = o;                      // the panel product's B operand in fp64, 128 x 128
    o += NB * NB * 8;
    for (int q = 0; q < 2; ++q) {
      exp_a[q] = o;
      o += align_up(ta * RB_A * 4, 1024);
      exp_w[q] = o;
      o += align_up(ta * RB_A * 4, 1024);
    }
    exp_x = o;
    exp_eq = exp_x + 1024;
    per_matrix = exp_eq + align_up(n * 4, 1024);
    common = 2048;   // status word, per-matrix info and equilibration flags (<= 255 matrices)
  }
  uint64_t bytes(uint32_t batch) const { return common + per_matrix * batch; }
};

// The factorisation's two streams on the current device, created once: a
// high-priority one for the critical chain (diagonal block, slicing, panel,
// the next panel's trailing tiles) and one for the bulk of each trailing
// update, with the events that order them.
struct LdlStreams {
  cudaStream_t chain = nullptr, bulk = nullptr;
  cudaEvent_t ops = nullptr, rest = nullptr, fork = nullptr, join = nullptr;
};

int ldl_streams(LdlStreams** out) {
  static std::mutex mu;
  static LdlStreams per_dev[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return mrg::set_error(MRG_ECUDA, "cudaGetDevice failed");
  std::lock_guard<std::mutex> lk(mu);
  LdlStreams& S = per_dev[dev];
  if (!S.chain) {
    int least = 0, greatest = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&S.chain, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&S.bulk, cudaStreamNonBlocking, least);
    for (cudaEvent_t* ev : {&S.ops, &S.rest, &S.fork, &S.join})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return mrg::set_error(MRG_ECUDA, "creating the factorisation's streams");
  }
  *out = &S;
  return MRG_OK;
}

int set_attrs_once() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return mrg::set_error(MRG_ECUDA, "cudaGetDevice failed");
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return MRG_OK;
  cudaError_t e = cudaFuncSetAttribute(ozaki_gemm_kernel<kSlices, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)GemmSmem<kSlices>::TOTAL);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(ozaki_gemm_kernel<kSlices, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)GemmSmem<kSlices>::TOTAL);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(ldl_diag_kernel<kSlices>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(NB * DG * sizeof(mrg::df)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(ldl_inverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(NB * DG * sizeof(mrg::df)));
  if (e != cudaSuccess) return mrg::set_error(MRG_ECUDA, cudaGetErrorString(e));
  done[dev] = true;
  return MRG_OK;
}

// Tiles per CTA of a product launch: enough for one wave over the SMs, at
// most `cap` (the bulk of a trailing update takes short chunks, so that the
// critical chain's kernels find SMs between them).
uint32_t chunk(uint64_t tiles, uint32_t batch, uint32_t cap) {
  const uint64_t items = tiles * batch;
  const uint64_t sms = (uint64_t)mrg::sm_count();
  return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(cap, (items + sms - 1) / sms));
}

dim3 grid_of(const GemmArgs& g) {
  const uint64_t items = (uint64_t)g.tiles_total * g.batch;
  return dim3((unsigned)((items + g.per_cta - 1) / g.per_cta));
}

int after(cudaError_t e, const char* what) {
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    return mrg::set_error(MRG_ECUDA, msg.c_str());
  }
  mrg::g_launches.fetch_add(1, std::memory_order_relaxed);
  return MRG_OK;
}

int params_block(const mrg_matern_params* params, uint32_t batch, ParamBlock* pb) {
  for (uint32_t b = 0; b < batch; ++b) {
    const mrg_matern_params& q = params[b];
    if (!(q.shape > 0.0 && q.shape <= 10.0) || !(q.range > 0.0) || !(q.variance > 0.0) ||
        !(q.aniso_ratio >= 1.0) || !std::isfinite(q.aniso_angle) || !std::isfinite(q.range) ||
        !std::isfinite(q.variance) || !std::isfinite(q.aniso_ratio))
      return mrg::set_error(MRG_EINVAL, "Matern parameters: need 0 < shape <= 10, range > 0, "
                                        "variance > 0, aniso_ratio >= 1, finite angle");
    MaternParams& p = pb->p[b];
    p.kappa = q.shape;
    p.var = q.variance;
    p.norm = std::exp2(1.0 - q.shape) / std::tgamma(q.shape);
    p.scale = std::sqrt(8.0 * q.shape) / q.range;
    p.c = std::cos(q.aniso_angle);
    p.s = std::sin(q.aniso_angle);
    p.omega = q.aniso_ratio;
  }
  return MRG_OK;
}

// Copies the parameter block to the head of the caller's scratch.
int upload_params(const ParamBlock& pb, uint32_t batch, void* scratch, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(scratch, &pb, sizeof(MaternParams) * batch,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // pb lives on the caller's stack
  if (e != cudaSuccess) return mrg::set_error(MRG_ECUDA, "copying the Matern parameters");
  return MRG_OK;
}

}  // namespace

extern "C" {

uint64_t mrg_grf_matern_scratch_bytes(uint32_t batch, uint32_t nrow, uint32_t ncol) {
  return 4096 + (uint64_t)batch * (2ull * nrow - 1) * (2ull * ncol - 1) * 8;
}

int mrg_grf_matern_raster(const mrg_matern_params* params, uint32_t batch, uint32_t nrow,
                          uint32_t ncol, double cell, double* cov, uint64_t ld, void* scratch,
                          uint64_t scratch_bytes, void* stream) {
  if (!params || !cov || !scratch) return mrg::set_error(MRG_EINVAL, "NULL argument");
  if (batch == 0 || batch > kMaxBatch) return mrg::set_error(MRG_EINVAL, "batch must be 1..64");
  if (nrow == 0 || ncol == 0) return mrg::set_error(MRG_EINVAL, "empty raster");
  const uint64_t n = (uint64_t)nrow * ncol;
  if (n > (1u << 20)) return mrg::set_error(MRG_ERANGE, "more than 2^20 cells");
  if (ld < n) return mrg::set_error(MRG_EINVAL, "ld < nrow * ncol");
  if (!(cell > 0.0) || !std::isfinite(cell)) return mrg::set_error(MRG_EINVAL, "cell must be > 0");
  if (reinterpret_cast<uintptr_t>(cov) % 8 || reinterpret_cast<uintptr_t>(scratch) % 256)
    return mrg::set_error(MRG_EINVAL, "cov not 8-byte or scratch not 256-byte aligned");
  if (scratch_bytes < mrg_grf_matern_scratch_bytes(batch, nrow, ncol))
    return mrg::set_error(MRG_EINVAL, "scratch smaller than mrg_grf_matern_scratch_bytes");
  ParamBlock pb;
  int rc = params_block(params, batch, &pb);
  if (rc) return rc;
  rc = mrg::ensure_device_ready();
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  rc = upload_params(pb, batch, scratch, st);
  if (rc) return rc;
  const MaternParams* dprm = static_cast<const MaternParams*>(scratch);
  double* table = reinterpret_cast<double*>(static_cast<char*>(scratch) + 4096);
  const uint64_t per_t = (2ull * nrow - 1) * (2ull * ncol - 1);
  const uint64_t nt = (per_t / 2 + 1) * batch;      // one thread per mirrored pair of offsets
  matern_offsets_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(dprm, batch, nrow, ncol, cell,
                                                                       table);
  rc = after(cudaSuccess, "matern_offsets_kernel");
  if (rc) return rc;
  const uint64_t items = (uint64_t)batch * n * ((n + 1023) / 1024);
  const int grid = (int)std::min<uint64_t>(items, (uint64_t)mrg::sm_count() * 32);
  const int vec = reinterpret_cast<uintptr_t>(cov) % 32 == 0 && ld % 4 == 0;
  matern_fill_kernel<<<grid, 256, 0, st>>>(table, batch, nrow, ncol, cov, ld, n * ld, vec);
  return after(cudaSuccess, "matern_fill_kernel");
}

int mrg_grf_matern_points(const mrg_matern_params* params, uint32_t batch, const double* xy,
                          uint64_t n, double* cov, uint64_t ld, void* scratch,
                          uint64_t scratch_bytes, void* stream) {
  if (!params || !xy || !cov || !scratch) return mrg::set_error(MRG_EINVAL, "NULL argument");
  if (batch == 0 || batch > kMaxBatch) return mrg::set_error(MRG_EINVAL, "batch must be 1..64");
  if (n == 0) return MRG_OK;
  if (n > (1u << 20)) return mrg::set_error(MRG_ERANGE, "more than 2^20 points");
  if (ld < n) return mrg::set_error(MRG_EINVAL, "ld < n");
  if (reinterpret_cast<uintptr_t>(cov) % 8 || reinterpret_cast<uintptr_t>(xy) % 8 ||
      reinterpret_cast<uintptr_t>(scratch) % 256 || scratch_bytes < 4096)
    return mrg::set_error(MRG_EINVAL, "misaligned pointer or scratch below 4096 bytes");
  ParamBlock pb;
  int rc = params_block(params, batch, &pb);
  if (rc) return rc;
  rc = mrg::ensure_device_ready();
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  rc = upload_params(pb, batch, scratch, st);
  if (rc) return rc;
  const int grid = mrg::sm_count() * 8;
  matern_points_kernel<<<grid, 256, 0, st>>>(static_cast<const MaternParams*>(scratch), batch, xy,
                                             n, cov, ld, n * ld);
  return after(cudaSuccess, "matern_points_kernel");
}

uint64_t mrg_grf_ldl_workspace_bytes(uint64_t n, uint32_t batch) {
  return LdlLayout(n).bytes(batch);
}

int mrg_grf_ldl(double* a, uint64_t n, uint64_t lda, uint32_t batch, double* d, void* workspace,
                uint64_t workspace_bytes, int32_t* info, void* stream) {
  if (!a || !d || !workspace) return mrg::set_error(MRG_EINVAL, "NULL argument");
  if (batch == 0 || batch > 255) return mrg::set_error(MRG_EINVAL, "batch must be 1..255");
  if (n == 0) return MRG_OK;
  if (n > (1u << 20)) return mrg::set_error(MRG_ERANGE, "n above 2^20");
  if (lda < n) return mrg::set_error(MRG_EINVAL, "lda < n");
  if (reinterpret_cast<uintptr_t>(a) % 8 || reinterpret_cast<uintptr_t>(d) % 8 ||
      reinterpret_cast<uintptr_t>(workspace) % 1024)
    return mrg::set_error(MRG_EINVAL, "a or d not 8-byte, or workspace not 1024-byte aligned");
  const LdlLayout L(n);
  if (workspace_bytes < L.bytes(batch))
    return mrg::set_error(MRG_EINVAL, "workspace smaller than mrg_grf_ldl_workspace_bytes");
  int rc = mrg::ensure_device_ready();
  if (rc) return rc;
  rc = set_attrs_once();
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  int* status = reinterpret_cast<int*>(ws);
  int* dinfo = status + 1;
  int* nonuniform = status + 256;
  LdlStreams* SS = nullptr;
  if ((rc = ldl_streams(&SS))) return rc;
  // the streams and events are shared by every call on this device: calls
  // are serialised on the host, so that no call records an event again
  // before another call's waits on it are enqueued
  static std::mutex call_mu;
  std::lock_guard<std::mutex> call_lk(call_mu);
  cudaStream_t hi = SS->chain, lo = SS->bulk;
  cudaError_t e = cudaEventRecord(SS->fork, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(hi, SS->fork, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(lo, SS->fork, 0);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws, 0, L.common, hi);
  if (e != cudaSuccess) return mrg::set_error(MRG_ECUDA, "starting the factorisation");
  char* base = ws + L.common;
  const uint64_t pm = L.per_matrix;
  const uint64_t a_ms = n * lda;
  int32_t* eq = reinterpret_cast<int32_t*>(base + L.exp_eq);
  const dim3 egrid((unsigned)((n + 255) / 256), batch);
  equil_exps_kernel<<<egrid, 256, 0, hi>>>(a, lda, a_ms, n, eq, pm / 4, nonuniform);
  if ((rc = after(cudaSuccess, "equil_exps_kernel"))) return rc;
  const dim3 agrid((unsigned)std::min<uint64_t>((n * (n + 1) / 2 + 255) / 256,
                                                (uint64_t)mrg::sm_count() * 16), batch);
  equil_apply_kernel<<<agrid, 256, 0, hi>>>(a, lda, a_ms, n, eq, pm / 4, nonuniform, d, 1);
  if ((rc = after(cudaSuccess, "equil_apply_kernel (scale)"))) return rc;
  const int vec32 = reinterpret_cast<uintptr_t>(a) % 32 == 0 && lda % 4 == 0;
  bool rest_pending = false;   // a bulk trailing update is in flight on `lo`
  int k = 0;
  for (uint64_t k0 = 0; k0 < n; k0 += NB, ++k) {
    const int q = k & 1;
    const uint32_t kb = (uint32_t)std::min<uint64_t>(NB, n - k0);
    const uint64_t t0 = k0 + kb, nt = n - t0;
    DiagArgs dg;
    dg.a = a;
    dg.lda = lda;
    dg.a_mstride = a_ms;
    dg.d = d;
    dg.d_mstride = n;
    dg.k0 = (uint32_t)k0;
    dg.kb = kb;
    dg.img_x = reinterpret_cast<uint8_t*>(base + L.img_x);
    dg.exp_x = reinterpret_cast<int32_t*>(base + L.exp_x);
    dg.img_x_mstride = pm;
    dg.exp_x_mstride = pm / 4;
    dg.info = dinfo;
    ldl_diag_kernel<kSlices><<<batch, DIAG_THREADS, NB * DG * sizeof(mrg::df), hi>>>(dg);
    if ((rc = after(cudaSuccess, "ldl_diag_kernel"))) return rc;
    if (nt == 0) break;
    // B = L_kk^-1 / d (by columns, many CTAs) and its B-role slices
    double* bx = reinterpret_cast<double*>(base + L.bx);
    ldl_inverse_kernel<<<dim3(NB / INV_COLS, batch), INV_COLS * 32, NB * DG * sizeof(mrg::df), hi>>>(
        a, lda, a_ms, (uint32_t)k0, kb, d, n, bx, pm / 8);
    if ((rc = after(cudaSuccess, "ldl_inverse_kernel"))) return rc;
    {
      SliceArgs sx;
      sx.a = bx;
      sx.lda = NB;
      sx.a_mstride = pm / 8;
      sx.rows = NB;
      sx.rows_pad = NB;
      sx.kb = NB;
      sx.img_a = nullptr;
      sx.exp_a = nullptr;
      sx.img_a_mstride = sx.exp_a_mstride = 0;
      sx.img_b = dg.img_x;
      sx.exp_b = dg.exp_x;
      sx.img_b_mstride = pm;
      sx.exp_b_mstride = pm / 4;
      sx.colscale = nullptr;
      sx.colscale_mstride = 0;
      slice_kernel<kSlices><<<dim3(NB / 8, batch), 256, 0, hi>>>(sx);
      if ((rc = after(cudaSuccess, "slice_kernel (panel B)"))) return rc;
    }
    const uint32_t rows_pad = (uint32_t)align_up(nt, RB_A);
    // panel operand: A_ik (rows t0.., columns k0.., kb wide)
    SliceArgs sa;
    sa.a = a + t0 * lda + k0;
    sa.lda = lda;
    sa.a_mstride = a_ms;
    sa.rows = (uint32_t)nt;
    sa.rows_pad = rows_pad;
    sa.kb = kb;
    sa.img_a = reinterpret_cast<uint8_t*>(base + L.img_a[q]);
    sa.exp_a = reinterpret_cast<int32_t*>(base + L.exp_a[q]);
    sa.img_a_mstride = pm;
    sa.exp_a_mstride = pm / 4;
    sa.img_b = nullptr;
    sa.exp_b = nullptr;
    sa.img_b_mstride = sa.exp_b_mstride = 0;
    sa.colscale = nullptr;
    sa.colscale_mstride = 0;
    const dim3 sgrid(rows_pad / 8, batch);
    slice_kernel<kSlices><<<sgrid, 256, 0, hi>>>(sa);
    if ((rc = after(cudaSuccess, "slice_kernel (panel)"))) return rc;
    // L_ik = A_ik X^T, written over A_ik
    GemmArgs gp;
    gp.img_a = sa.img_a;
    gp.exp_a = sa.exp_a;
    gp.img_b = dg.img_x;
    gp.exp_b = dg.exp_x;
    gp.img_a_mstride = pm;
    gp.exp_a_mstride = pm / 4;
    gp.img_b_mstride = pm;
    gp.exp_b_mstride = pm / 4;
    gp.c = a + t0 * lda + k0;
    gp.ldc = lda;
    gp.c_mstride = a_ms;
    gp.m = (uint32_t)nt;
    gp.n = kb;
    gp.tiles_n = (kb + BN - 1) / BN;
    gp.tile_set = TILES_LOWER;
    gp.vec32 = vec32;
    gp.status = status;
    gp.batch = batch;
    gp.tiles_total = (uint32_t)((nt + BM - 1) / BM * gp.tiles_n);
    gp.per_cta = chunk(gp.tiles_total, batch, 1 << 30);
    ozaki_gemm_kernel<kSlices, false><<<grid_of(gp), GEMM_THREADS, GemmSmem<kSlices>::TOTAL, hi>>>(gp);
    if ((rc = after(cudaSuccess, "ozaki_gemm_kernel (panel)"))) return rc;
    // trailing operands: L_ik (A role) and W = L_ik D_k (B role)
    sa.img_b = reinterpret_cast<uint8_t*>(base + L.img_w[q]);
    sa.exp_b = reinterpret_cast<int32_t*>(base + L.exp_w[q]);
    sa.img_b_mstride = pm;
    sa.exp_b_mstride = pm / 4;
    sa.colscale = d + k0;
    sa.colscale_mstride = n;
    slice_kernel<kSlices><<<sgrid, 256, 0, hi>>>(sa);
    if ((rc = after(cudaSuccess, "slice_kernel (trailing)"))) return rc;
    // The trailing update A_ij -= L_i W_j^T.  Its two tile columns of the
    // next panel are on the critical chain; they also update columns that
    // the previous step's bulk update writes, so they wait for it.  The
    // rest goes to the bulk stream and overlaps the next step's chain.
    GemmArgs gt = gp;
    gt.img_b = sa.img_b;
    gt.exp_b = sa.exp_b;
    gt.c = a + t0 * lda + t0;
    gt.n = (uint32_t)nt;
    const uint64_t T = (nt + BM - 1) / BM, Tc = (nt + BN - 1) / BN;
    if (rest_pending && (e = cudaStreamWaitEvent(hi, SS->rest, 0)) != cudaSuccess)
      return mrg::set_error(MRG_ECUDA, "ordering the trailing updates");
    gt.tile_set = TILES_NEXT;
    gt.tiles_n = (uint32_t)std::min<uint64_t>(2, Tc);
    gt.tiles_total = (uint32_t)(T * gt.tiles_n);
    gt.per_cta = chunk(gt.tiles_total, batch, 1 << 30);
    ozaki_gemm_kernel<kSlices, true><<<grid_of(gt), GEMM_THREADS, GemmSmem<kSlices>::TOTAL, hi>>>(gt);
    if ((rc = after(cudaSuccess, "ozaki_gemm_kernel (next panel)"))) return rc;
    rest_pending = false;
    if (Tc > 2) {
      if ((e = cudaEventRecord(SS->ops, hi)) != cudaSuccess ||
          (e = cudaStreamWaitEvent(lo, SS->ops, 0)) != cudaSuccess)
        return mrg::set_error(MRG_ECUDA, "handing the trailing update to the bulk stream");
      gt.tile_set = TILES_REST;
      gt.tiles_n = (uint32_t)Tc;
      gt.tiles_total = (uint32_t)((T - 2) * (T - 1) + (Tc - 2));
      gt.per_cta = chunk(gt.tiles_total, batch, 4);
      ozaki_gemm_kernel<kSlices, true><<<grid_of(gt), GEMM_THREADS, GemmSmem<kSlices>::TOTAL, lo>>>(gt);
      if ((rc = after(cudaSuccess, "ozaki_gemm_kernel (trailing)"))) return rc;
      if ((e = cudaEventRecord(SS->rest, lo)) != cudaSuccess)
        return mrg::set_error(MRG_ECUDA, "recording the trailing update");
      rest_pending = true;
    }
  }
  if (rest_pending && (e = cudaStreamWaitEvent(hi, SS->rest, 0)) != cudaSuccess)
    return mrg::set_error(MRG_ECUDA, "joining the trailing updates");
  equil_apply_kernel<<<agrid, 256, 0, hi>>>(a, lda, a_ms, n, eq, pm / 4, nonuniform, d, -1);
  if ((rc = after(cudaSuccess, "equil_apply_kernel (unscale)"))) return rc;
  // the caller's stream continues once both streams are done
  e = cudaEventRecord(SS->join, hi);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, SS->join, 0);
  if (e == cudaSuccess) e = cudaEventRecord(SS->join, lo);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, SS->join, 0);
  if (e != cudaSuccess) return mrg::set_error(MRG_ECUDA, "joining the factorisation's streams");
  if (info) {
    int32_t h[256];
    e = cudaMemcpyAsync(h, ws, 4 * (1 + batch), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return mrg::set_error(MRG_ECUDA, cudaGetErrorString(e));
    for (uint32_t b = 0; b < batch; ++b) info[b] = h[1 + b];
    if (h[0]) return mrg::set_error(MRG_ETIMEOUT, "a tensor-core wait gave up (2 s)");
  }
  return MRG_OK;
}

uint64_t mrg_grf_simulate_scratch_bytes(uint64_t n, uint32_t nsim, uint32_t batch) {
  return (uint64_t)batch * nsim * n * 8;
}

int mrg_grf_simulate(const double* l, const double* d, uint64_t n, uint64_t lda, uint32_t batch,
                     const double* z, uint32_t nsim, double* u, void* scratch,
                     uint64_t scratch_bytes, void* stream) {
  if (!l || !d || !z || !u || !scratch) return mrg::set_error(MRG_EINVAL, "NULL argument");
  if (batch == 0 || batch > 65535) return mrg::set_error(MRG_EINVAL, "batch must be 1..65535");
  if (n == 0 || nsim == 0) return MRG_OK;
  if (lda < n) return mrg::set_error(MRG_EINVAL, "lda < n");
  if (n > (1u << 20) || nsim > (1u << 16)) return mrg::set_error(MRG_ERANGE, "n or nsim too large");
  if ((reinterpret_cast<uintptr_t>(l) | reinterpret_cast<uintptr_t>(d) |
       reinterpret_cast<uintptr_t>(z) | reinterpret_cast<uintptr_t>(u) |
       reinterpret_cast<uintptr_t>(scratch)) % 8)
    return mrg::set_error(MRG_EINVAL, "pointers must be 8-byte aligned");
  if (scratch_bytes < mrg_grf_simulate_scratch_bytes(n, nsim, batch))
    return mrg::set_error(MRG_EINVAL, "scratch smaller than mrg_grf_simulate_scratch_bytes");
  int rc = mrg::ensure_device_ready();
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double* y = static_cast<double*>(scratch);
  const uint64_t tot = (uint64_t)batch * nsim * n;
  scale_sqrt_d_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(d, n, z, y, n, nsim, batch);
  if ((rc = after(cudaSuccess, "scale_sqrt_d_kernel"))) return rc;
  const dim3 grid((unsigned)((n + 7) / 8), batch);
  if (nsim <= 2)
    lower_times_y_kernel<2><<<grid, 256, 0, st>>>(l, lda, n * lda, y, u, n, nsim, batch);
  else if (nsim <= 4)
    lower_times_y_kernel<4><<<grid, 256, 0, st>>>(l, lda, n * lda, y, u, n, nsim, batch);
  else
    lower_times_y_kernel<8><<<grid, 256, 0, st>>>(l, lda, n * lda, y, u, n, nsim, batch);
  return after(cudaSuccess, "lower_times_y_kernel");
}

}  // extern "C"
