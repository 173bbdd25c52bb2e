// C ABI of the HPSCD GB300 library (declared in include/hpscd.h): argument
// checks, workspace, tensor-map encoding and the launch sequence of a solve.
#include <cudaTypedefs.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "ctx.h"

using namespace hpscd;

namespace {

struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Layout {
  size_t G = 0, Gt = 0, dvec = 0, partial = 0, e = 0, hacc = 0, npart = 0, gw = 0, ypart = 0, hist = 0,
         ctl = 0, sel = 0, order = 0, swp = 0, h0 = 0, y2 = 0;
  size_t xcopy = 0, ycopy = 0, acopy = 0, total = 0;
};

struct Plan {
  TallConfig cfg;
  GramPlan gp;
  GramTCPlan gtc;
  bool tc_ok = false;  // the tensor-core Gram applies to this shape
  int ldG = 0;
  int64_t ntiles = 0;
  int grid = 0;
  int e_smem = 0;  // the tall sweep keeps e in shared memory
  Layout L;
};

int esize(int dtype) { return dtype == HPSCD_F32 ? 4 : 2; }

int check_opts(const hpscd_opts* o) {
  if (!o) return HPSCD_ERR_INVALID_ARG;
  if (!(o->tol >= 0.0) || !isfinite(o->tol)) return HPSCD_ERR_INVALID_ARG;
  if (o->max_sweeps < 0 || o->max_sweeps > (int64_t)1 << 40) return HPSCD_ERR_INVALID_ARG;
  if (o->stop_rule < HPSCD_STOP_REL_RES || o->stop_rule > HPSCD_STOP_NONE) return HPSCD_ERR_INVALID_ARG;
  if (o->refresh_every < 0) return HPSCD_ERR_INVALID_ARG;
  if (o->debug_flags & ~(HPSCD_DEBUG_STALL_BARRIER | HPSCD_DEBUG_SIMT_GRAM | HPSCD_DEBUG_E_IN_HBM))
    return HPSCD_ERR_INVALID_ARG;
  for (int i = 0; i < 5; ++i)
    if (o->reserved[i] != 0) return HPSCD_ERR_INVALID_ARG;
  return HPSCD_OK;
}

int check_shape(int dtype, int layout, int64_t m, int64_t n, int64_t ld) {
  if (dtype != HPSCD_F32 && dtype != HPSCD_BF16 && dtype != HPSCD_F16) return HPSCD_ERR_INVALID_ARG;
  if (layout != HPSCD_COL_MAJOR && layout != HPSCD_ROW_MAJOR) return HPSCD_ERR_INVALID_ARG;
  if (m < 0 || n < 0) return HPSCD_ERR_INVALID_ARG;
  if (m > ((int64_t)1 << 31) - 1024 || n > ((int64_t)1 << 31) - 1024) return HPSCD_ERR_INVALID_ARG;
  const int64_t minld = layout == HPSCD_COL_MAJOR ? (m > 1 ? m : 1) : (n > 1 ? n : 1);
  if (ld < minld) return HPSCD_ERR_INVALID_ARG;
  return HPSCD_OK;
}

// Sizes the workspace of a solve.  Returns false for unsupported shapes.
int make_plan(const hpscd_ctx* ctx, int dtype, int layout, int64_t m, int64_t n, int64_t ld,
              const hpscd_opts* o, bool host_copies, Plan* P, int64_t order_entries = 0,
              int64_t swap_rounds = 0) {
  if (layout != HPSCD_COL_MAJOR) return HPSCD_ERR_UNSUPPORTED;
  if (n > 512) return HPSCD_ERR_UNSUPPORTED;
  if (!tall_config(dtype, (int)n, ctx->max_smem, &P->cfg)) return HPSCD_ERR_UNSUPPORTED;
  P->gp = gram_plan(m, P->cfg.npad, ctx->sms);
  P->tc_ok = gram_tc_plan(dtype, m, (int)n, ctx->sms, ctx->max_smem, &P->gtc);
  P->ldG = P->tc_ok && P->gtc.npad > P->gp.npad ? P->gtc.npad : P->gp.npad;
  P->ntiles = (m + P->cfg.rows - 1) / P->cfg.rows;
  int64_t grid = ctx->sms > 256 ? 256 : ctx->sms;  // the kernel's norm reduction covers 256 CTAs
  if (P->ntiles < grid) grid = P->ntiles;
  if (grid < 1) grid = 1;
  P->grid = (int)grid;
  // The residual of each CTA's row panels stays in shared memory when it fits
  // beside at least four TMA stages (the kernel's other buffers are fixed).
  P->e_smem = 0;
  if (!(o->debug_flags & HPSCD_DEBUG_E_IN_HBM) && m > 0) {
    const int64_t npan_max = (P->ntiles + P->grid - 1) / P->grid;
    const int64_t e_bytes = npan_max * P->cfg.rows * (int64_t)sizeof(float) + 16;
    int nst = P->cfg.nstages, smem = P->cfg.smem_bytes;
    while ((int64_t)smem + e_bytes > ctx->max_smem - 256 && nst > 4) {
      --nst;
      smem -= P->cfg.stage_bytes;
    }
    if ((int64_t)smem + e_bytes <= ctx->max_smem - 256) {
      P->cfg.nstages = nst;
      P->cfg.smem_bytes = smem + (int)e_bytes;
      P->e_smem = 1;
    }
  }
  Layout& L = P->L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes, 256);
    return at;
  };
  L.G = take((size_t)P->ldG * P->ldG * sizeof(float));
  L.Gt = take((size_t)P->ldG * P->ldG * sizeof(float));
  L.dvec = take((size_t)P->ldG * sizeof(float));
  L.partial = take(P->tc_ok && P->gtc.partial_bytes > P->gp.partial_bytes ? P->gtc.partial_bytes
                                                                          : P->gp.partial_bytes);
  L.e = take((size_t)(m > 0 ? m : 1) * sizeof(float));
  L.hacc = take((size_t)3 * P->cfg.npad * sizeof(double));
  L.npart = take((size_t)2 * P->grid * sizeof(double));
  L.gw = take((size_t)2 * P->cfg.npad * sizeof(float));
  L.ypart = take((size_t)P->grid * sizeof(double));
  L.hist = take((size_t)(o->max_sweeps + 1) * sizeof(double));
  L.ctl = take(sizeof(GridCtl));
  L.sel = take((size_t)(o->max_sweeps + 1) * sizeof(int64_t));
  L.order = take((size_t)(order_entries > 0 ? order_entries : 1) * sizeof(int32_t));
  L.swp = take((size_t)2 * (swap_rounds > 0 ? swap_rounds : 1) * sizeof(int64_t));
  L.h0 = take((size_t)P->ldG * sizeof(double));
  L.y2 = take(sizeof(double));
  if (host_copies) {
    L.xcopy = take((size_t)(n > 0 ? n : 1) * (size_t)ld * esize(dtype));
    L.ycopy = take((size_t)(m > 0 ? m : 1) * sizeof(float));
    L.acopy = take((size_t)(n > 0 ? n : 1) * sizeof(float));
  }
  L.total = off;
  return HPSCD_OK;
}

int ensure_ws(hpscd_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return HPSCD_OK;
  if (!ctx->ws_owned) return HPSCD_ERR_NO_MEMORY;
  if (ctx->ws) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_bytes = 0;
  }
  size_t want = bytes + bytes / 8;
  if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
    cudaGetLastError();
    ctx->ws = nullptr;
    return HPSCD_ERR_NO_MEMORY;
  }
  ctx->ws_bytes = want;
  return HPSCD_OK;
}

int encode_tall_map(hpscd_ctx* ctx, const void* X, int dtype, int64_t m, int64_t n, int64_t ld,
                    const TallConfig& cfg, CUtensorMap* map) {
  if (!ctx->encode) return 0;
  const int es = esize(dtype);
  if ((reinterpret_cast<uintptr_t>(X) & 15) != 0) return 0;
  if (((uint64_t)ld * es) % 16 != 0) return 0;
  if (m < 1 || n < 1) return 0;
  if ((uint64_t)ld * es >= ((uint64_t)1 << 40)) return 0;
  cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)n};
  cuuint64_t strides[1] = {(cuuint64_t)ld * es};
  cuuint32_t box[2] = {(cuuint32_t)cfg.rows, (cuuint32_t)cfg.box_cols};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = ctx->encode(map, x_tmap_type(dtype),
                           2, const_cast<void*>(X), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 1 : 0;
}

// 128-byte-swizzled map for the tensor-core Gram: boxes of one 128-byte K
// block (32 float32 / 64 bfloat16 rows) × 128 columns.
int encode_gram_map(hpscd_ctx* ctx, const void* X, int dtype, int64_t m, int64_t n, int64_t ld,
                    CUtensorMap* map) {
  if (!ctx->encode) return 0;
  const int es = esize(dtype);
  if ((reinterpret_cast<uintptr_t>(X) & 15) != 0 || ((uint64_t)ld * es) % 16 != 0) return 0;
  if (m < 1 || n < 1 || (uint64_t)ld * es >= ((uint64_t)1 << 40)) return 0;
  cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)n};
  cuuint64_t strides[1] = {(cuuint64_t)ld * es};
  cuuint32_t box[2] = {(cuuint32_t)(128 / es), 128};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = ctx->encode(map, x_tmap_type(dtype),
                           2, const_cast<void*>(X), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? 1 : 0;
}

// G = X^T X into G (ldG), by the tensor-core kernel when it applies, else the
// CUDA-core kernel.  `err` receives a device-side failure flag.
// When Gt is given, also G~ = D^{-1} G and d (fused into the tensor-core
// path's reduction; one extra kernel after the CUDA-core path).
// When y, h0 and y2 are given and the tensor-core kernel runs, it also forms
// h0 = X^T y and *y2 = ||y||^2 from the same read of X (*got_h0 = true).
int run_gram(hpscd_ctx* ctx, const void* X, int dtype, int64_t m, int64_t n, int64_t ld,
             const Plan& P, void* partial, float* G, int ldG, int* err, bool force_simt,
             int* launches, float* Gt = nullptr, float* dvec = nullptr, const float* y = nullptr,
             double* h0 = nullptr, double* y2 = nullptr, bool* got_h0 = nullptr) {
  CUtensorMap gmap;
  memset(&gmap, 0, sizeof(gmap));
  if (got_h0) *got_h0 = false;
  if (!force_simt && P.tc_ok && encode_gram_map(ctx, X, dtype, m, n, ld, &gmap)) {
    // y's K blocks by TMA: a 1-D map of y (rows past m read as zero), boxes of
    // one K block (32 rows for float32 X, 64 for bfloat16)
    CUtensorMap ymap;
    memset(&ymap, 0, sizeof(ymap));
    bool ytma = false;
    if (y && (reinterpret_cast<uintptr_t>(y) & 15) == 0 && m < ((int64_t)1 << 32)) {
      cuuint64_t dims[1] = {(cuuint64_t)m};
      cuuint64_t strides[1] = {0};
      cuuint32_t box[1] = {(cuuint32_t)(dtype == HPSCD_F32 ? 32 : 64)};
      cuuint32_t estr[1] = {1};
      ytma = ctx->encode(&ymap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 1, const_cast<float*>(y), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    if (launch_gram_tc(&gmap, dtype, m, P.gtc, static_cast<float*>(partial), err,
                       (uint64_t)(ctx->timeout_s * 1e9), G, ldG, ctx->stream, (int)n, Gt,
                       dvec, y, h0, y2, ytma ? &ymap : nullptr) != cudaSuccess) {
      cudaGetLastError();
      return HPSCD_ERR_CUDA;
    }
    if (got_h0) *got_h0 = y && h0 && y2;
    *launches = 4;  // the Gram kernel and its three reduce kernels
    return HPSCD_OK;
  }
  if (launch_gram(X, dtype, m, (int)n, ld, P.gp, static_cast<double*>(partial), G, ldG,
                  ctx->stream) != cudaSuccess ||
      (Gt && launch_scale_rows(G, ldG, (int)n, Gt, dvec, ctx->stream) != cudaSuccess)) {
    cudaGetLastError();
    return HPSCD_ERR_CUDA;
  }
  *launches = Gt ? 3 : 2;
  return HPSCD_OK;
}

// ---- wide systems: row-major X, m <= 4096 (the cluster sweep) ----
struct WideLayout {
  size_t Mb = 0, Nb = 0, e = 0, a64 = 0, dsw = 0, atmp = 0, ysq = 0, hist = 0, ctl = 0, r2 = 0, tsum = 0,
         rpart = 0, xcopy = 0, ycopy = 0, acopy = 0, total = 0;
};

int make_wide_plan(const hpscd_ctx* ctx, int dtype, int64_t m, int64_t n, int64_t ld,
                   const hpscd_opts* o, bool host_copies, WideConfig* cfg, WideLayout* L) {
  if (dtype != HPSCD_F32) return HPSCD_ERR_UNSUPPORTED;
  if (!wide_config(m, ctx->max_smem, cfg)) return HPSCD_ERR_UNSUPPORTED;
  const int64_t nblk = (n + cfg->W - 1) / cfg->W;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes, 256);
    return at;
  };
  L->Mb = take((size_t)nblk * cfg->W * cfg->W * sizeof(float));
  L->Nb = take((size_t)nblk * cfg->W * cfg->W * sizeof(float));
  L->e = take((size_t)m * sizeof(float));
  L->a64 = take((size_t)n * sizeof(double));
  L->dsw = take((size_t)n * sizeof(float));
  L->atmp = take((size_t)n * sizeof(float));
  L->ysq = take(sizeof(double));
  L->hist = take((size_t)(o->max_sweeps + 1) * sizeof(double));
  L->ctl = take(sizeof(GridCtl));
  L->r2 = take((size_t)m * sizeof(double));
  L->tsum = take(2 * sizeof(double));
  L->rpart = take((size_t)m * 32 * sizeof(double));
  if (host_copies) {
    L->xcopy = take((size_t)m * ld * sizeof(float));
    L->ycopy = take((size_t)m * sizeof(float));
    L->acopy = take((size_t)n * sizeof(float));
  }
  L->total = off;
  return HPSCD_OK;
}

int solve_wide(hpscd_ctx* ctx, const void* X, int64_t m, int64_t n, int64_t ld, const float* y,
               float* a, int a_is_guess, const hpscd_opts* o, double* hist, int64_t* sweeps_done,
               double* final_rel_res, const WideConfig& cfg, const WideLayout& L) {
  const bool aligned = ctx->encode && (reinterpret_cast<uintptr_t>(X) & 15) == 0 && (ld * 4) % 16 == 0;
  char* ws = static_cast<char*>(ctx->ws);
  GridCtl* ctl = reinterpret_cast<GridCtl*>(ws + L.ctl);
  cudaStream_t st = ctx->stream;
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)cfg.W, (cuuint32_t)cfg.rows_box};
  cuuint32_t estr[2] = {1, 1};
  const int use_tma =
      aligned && ctx->encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(X), dims,
                             strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  if (cudaMemsetAsync(ctl, 0, sizeof(GridCtl), st) != cudaSuccess) return HPSCD_ERR_CUDA;
  if (cudaEventRecord(ctx->ev[0], st) != cudaSuccess) return HPSCD_ERR_CUDA;
  WideParams p{};
  p.X = static_cast<const float*>(X);
  p.use_tma = use_tma;
  p.m = m;
  p.n = n;
  p.ld = ld;
  p.Mb = reinterpret_cast<float*>(ws + L.Mb);
  p.Nb = reinterpret_cast<float*>(ws + L.Nb);
  p.e = reinterpret_cast<float*>(ws + L.e);
  p.a64 = reinterpret_cast<double*>(ws + L.a64);
  p.dsw = reinterpret_cast<float*>(ws + L.dsw);
  p.a_out = a;
  p.ysq = reinterpret_cast<double*>(ws + L.ysq);
  p.hist = reinterpret_cast<double*>(ws + L.hist);
  p.ctl = ctl;
  p.tol = o->tol;
  p.max_sweeps = o->max_sweeps;
  p.stop_rule = o->stop_rule;
  p.timeout_ns = (uint64_t)(ctx->timeout_s * 1e9);
  p.rpart = reinterpret_cast<double*>(ws + L.rpart);
  p.trace = nullptr;
  p.trace_passes = 0;
  if (ctx->trace_passes > 0 && ctx->trace_dev) {
    if (cudaMemsetAsync(ctx->trace_dev, 0, (size_t)ctx->trace_passes * 6 * sizeof(unsigned long long),
                        st) != cudaSuccess)
      return HPSCD_ERR_CUDA;
    p.trace = ctx->trace_dev;
    p.trace_passes = ctx->trace_passes;
    ctx->trace_grid = 0;
  }
  if (launch_wide(static_cast<const float*>(X), m, n, ld, cfg, &map, p, y, a, a_is_guess,
                  reinterpret_cast<float*>(ws + L.atmp), st) != cudaSuccess) {
    cudaGetLastError();
    return HPSCD_ERR_CUDA;
  }
  // Under REL_RES the cluster kernel stops on the residual it updates; the stop
  // is then confirmed on e = y - X·a for the float32 a it returned (Dot2, all
  // SMs).  If that misses the tolerance the sweeps go on from the recomputed e.
  int64_t before = 0;  // sweeps made by earlier launches of this solve
  int64_t conf_at[8];
  double conf_val[8];
  int nconf = 0;
  int status = HPSCD_ERR_NOT_CONVERGED;
  GridCtl c{};
  double final_res = 0.0;
  double* tsum = reinterpret_cast<double*>(ws + L.tsum);
  for (;;) {
    if (cudaMemcpyAsync(ctx->ctl_host, ctl, sizeof(GridCtl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return HPSCD_ERR_CUDA;
    c = *ctx->ctl_host;
    const int64_t total = before + c.sweeps;
    final_res = c.final_res;
    status = c.status;
    if (c.err != DEV_OK || c.status != HPSCD_OK || o->stop_rule != HPSCD_STOP_REL_RES || nconf == 8) {
      c.sweeps = total;
      break;
    }
    if (launch_wide_confirm(static_cast<const float*>(X), m, n, ld, y, a, p.e, p.rpart,
                            reinterpret_cast<double*>(ws + L.r2), tsum, st) != cudaSuccess ||
        cudaMemcpyAsync(ctx->host_scratch, tsum, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(ctx->host_scratch + 1, p.ysq, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      return HPSCD_ERR_CUDA;
    }
    const double ynorm = sqrt(ctx->host_scratch[1]);
    const double rel = ynorm > 0.0 ? sqrt(ctx->host_scratch[0]) / ynorm : sqrt(ctx->host_scratch[0]);
    conf_at[nconf] = total;
    conf_val[nconf++] = rel;
    final_res = rel;
    c.sweeps = total;
    if (!isfinite(rel)) { status = HPSCD_ERR_NONFINITE; break; }
    if (rel <= o->tol) { status = HPSCD_OK; break; }
    if (total >= o->max_sweeps) { status = HPSCD_ERR_NOT_CONVERGED; break; }
    WideParams q = p;
    q.hist = p.hist + total;  // the continuation's sweep 0 is sweep `total` of the solve
    q.max_sweeps = o->max_sweeps - total;
    if (cudaMemsetAsync(ctl, 0, sizeof(GridCtl), st) != cudaSuccess ||
        launch_wide_continue(n, cfg, &map, q, reinterpret_cast<float*>(ws + L.atmp), st) != cudaSuccess) {
      cudaGetLastError();
      return HPSCD_ERR_CUDA;
    }
    before = total;
  }
  if (cudaEventRecord(ctx->ev[2], st) != cudaSuccess) return HPSCD_ERR_CUDA;
  if (cudaEventSynchronize(ctx->ev[2]) != cudaSuccess) return HPSCD_ERR_CUDA;
  if (hist && c.sweeps >= 0 && c.sweeps <= o->max_sweeps) {
    if (cudaMemcpy(hist, p.hist, (size_t)(c.sweeps + 1) * sizeof(double), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return HPSCD_ERR_CUDA;
    for (int k = 0; k < nconf; ++k)
      if (conf_at[k] <= c.sweeps) hist[conf_at[k]] = conf_val[k];  // the confirmed (true) values
  }
  if (sweeps_done) *sweeps_done = c.sweeps;
  if (final_rel_res) *final_rel_res = final_res;
  hpscd_timing t{};
  cudaEventElapsedTime(&t.sweep_ms, ctx->ev[0], ctx->ev[2]);
  t.passes = c.sweeps;
  t.x_bytes = m * n * 4;
  t.grid = cfg.csize;
  t.kernel_launches = 6 + 4 * nconf;
  ctx->last = t;
  if (c.err != DEV_OK) return HPSCD_ERR_TIMEOUT;
  return status;
}

// m == 0: nothing to sweep; y = 0, so every recorded residual is the absolute norm 0.
int solve_empty_rows(hpscd_ctx* ctx, int64_t n, float* a, int a_is_guess, const hpscd_opts* o,
                     double* hist, int64_t* sweeps_done, double* final_rel_res) {
  if (!a_is_guess && n > 0 && cudaMemsetAsync(a, 0, (size_t)n * sizeof(float), ctx->stream) != cudaSuccess)
    return HPSCD_ERR_CUDA;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return HPSCD_ERR_CUDA;
  int64_t s = 0;
  if (o->stop_rule == HPSCD_STOP_REL_CHANGE) s = o->max_sweeps > 0 ? 1 : 0;
  if (o->stop_rule == HPSCD_STOP_NONE) s = o->max_sweeps;
  if (hist)
    for (int64_t i = 0; i <= s; ++i) hist[i] = 0.0;
  if (sweeps_done) *sweeps_done = s;
  if (final_rel_res) *final_rel_res = 0.0;
  ctx->last = hpscd_timing{};
  if (o->stop_rule == HPSCD_STOP_REL_CHANGE && o->max_sweeps == 0) return HPSCD_ERR_NOT_CONVERGED;
  return HPSCD_OK;
}

// Result of an asynchronous solve, written after the sweep kernel has finished
// (every CTA's error report has landed in the control block by then).
__global__ void copy_result_kernel(const GridCtl* ctl, hpscd_sys_result* res) {
  res->sweeps = ctl->sweeps;
  res->rel_res = ctl->final_res;
  res->status = ctl->err != DEV_OK ? HPSCD_ERR_TIMEOUT : ctl->status;
  res->passes = (int32_t)ctl->passes;
}

// The variants of the sweep: Algorithm 1 (thr <= 1, select = 0), Algorithm 2
// (blocks of thr columns from one residual) and Algorithm 3 (select = 1: one
// greedily chosen column per pass; sel receives the choices, HOST int64[max_sweeps]).
int solve_device(hpscd_ctx* ctx, const void* X, int dtype, int layout, int64_t m, int64_t n,
                 int64_t ld, const float* y, float* a, int a_is_guess, const hpscd_opts* o,
                 double* hist, int64_t* sweeps_done, double* final_rel_res, const Plan& P,
                 int thr = 0, int select = 0, int64_t* sel = nullptr, const int* order = nullptr,
                 hpscd_sys_result* async_res = nullptr, double* hist_dev = nullptr,
                 int swap_rounds = 0, int64_t* swaps = nullptr) {
  if (m == 0) return solve_empty_rows(ctx, n, a, a_is_guess, o, hist, sweeps_done, final_rel_res);
  char* ws = static_cast<char*>(ctx->ws);
  const Layout& L = P.L;
  float* G = reinterpret_cast<float*>(ws + L.G);
  GridCtl* ctl = reinterpret_cast<GridCtl*>(ws + L.ctl);
  cudaStream_t st = ctx->stream;
  // an asynchronous call records its events in the ring and returns after the launches
  const bool async = async_res != nullptr;
  const int slot = (int)(ctx->ring_calls % hpscd_ctx::RING);
  cudaEvent_t* ev = async ? ctx->ring_ev[slot] : ctx->ev;

  if (cudaMemsetAsync(ctl, 0, sizeof(GridCtl), st) != cudaSuccess) return HPSCD_ERR_CUDA;
  if (cudaEventRecord(ev[0], st) != cudaSuccess) return HPSCD_ERR_CUDA;
  int gram_launches = 0;
  float* Gt = reinterpret_cast<float*>(ws + L.Gt);
  float* dvec = reinterpret_cast<float*>(ws + L.dvec);
  // a cold start takes X^T y and ||y||^2 from the set-up's read of X, so the
  // sweep kernel makes no pass of its own before the first sweep
  double* h0 = reinterpret_cast<double*>(ws + L.h0);
  double* y2 = reinterpret_cast<double*>(ws + L.y2);
  bool got_h0 = false;
  int rcg = run_gram(ctx, X, dtype, m, n, ld, P, ws + L.partial, G, P.ldG, &ctl->err,
                     (o->debug_flags & HPSCD_DEBUG_SIMT_GRAM) != 0, &gram_launches, Gt, dvec,
                     a_is_guess ? nullptr : y, h0, y2, &got_h0);
  if (rcg != HPSCD_OK) return rcg;
  if (cudaMemsetAsync(ws + L.hacc, 0, (size_t)3 * P.cfg.npad * sizeof(double), st) != cudaSuccess)
    return HPSCD_ERR_CUDA;
  if (cudaEventRecord(ev[1], st) != cudaSuccess) return HPSCD_ERR_CUDA;

  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  const int use_tma = encode_tall_map(ctx, X, dtype, m, n, ld, P.cfg, &map);

  TallParams p{};
  p.X = X;
  p.m = m;
  p.n = (int)n;
  p.ld = ld;
  p.y = y;
  p.e = reinterpret_cast<float*>(ws + L.e);
  p.a_out = a;
  p.a_in = a;
  p.warm = a_is_guess ? 1 : 0;
  p.Gt = Gt;
  p.dvec = dvec;
  p.ldG = P.ldG;
  p.hacc = reinterpret_cast<double*>(ws + L.hacc);
  p.npart = reinterpret_cast<double*>(ws + L.npart);
  p.gw = reinterpret_cast<float*>(ws + L.gw);
  p.ypart = reinterpret_cast<double*>(ws + L.ypart);
  p.hist = hist_dev ? hist_dev : reinterpret_cast<double*>(ws + L.hist);
  p.ctl = ctl;
  p.tol = o->tol;
  p.max_sweeps = o->max_sweeps;
  p.stop_rule = o->stop_rule;
  p.refresh_every = o->refresh_every;
  p.ntiles = P.ntiles;
  p.nstages = P.cfg.nstages;
  p.use_tma = use_tma;
  p.timeout_ns = (uint64_t)(ctx->timeout_s * 1e9);
  p.stall_barrier = (o->debug_flags & HPSCD_DEBUG_STALL_BARRIER) ? 1 : 0;
  p.thr = thr;
  p.select = select;
  p.sel_out = select ? reinterpret_cast<int64_t*>(ws + L.sel) : nullptr;
  p.swap_rounds = select ? swap_rounds : 0;
  p.swap_out = (select && swap_rounds > 0) ? reinterpret_cast<int64_t*>(ws + L.swp) : nullptr;
  if (p.swap_out && cudaMemsetAsync(p.swap_out, 0xff, (size_t)2 * swap_rounds * sizeof(int64_t), st) !=
                        cudaSuccess)
    return HPSCD_ERR_CUDA;
  p.order = order;
  p.h0 = got_h0 ? h0 : nullptr;
  p.y2 = got_h0 ? y2 : nullptr;
  p.confirm = select ? 0 : 1;
  p.e_smem = P.e_smem;
  p.trace = nullptr;
  p.trace_passes = 0;
  if (ctx->trace_passes > 0 && ctx->trace_dev) {
    const size_t words = (size_t)ctx->trace_passes * 6 + (size_t)P.grid;
    if (cudaMemsetAsync(ctx->trace_dev, 0, words * sizeof(unsigned long long), st) != cudaSuccess)
      return HPSCD_ERR_CUDA;
    p.trace = ctx->trace_dev;
    p.trace_passes = ctx->trace_passes;
    ctx->trace_grid = P.grid;
  }
  if (launch_tall_sweep(dtype, P.cfg, &map, p, P.grid, st) != cudaSuccess) {
    cudaGetLastError();
    return HPSCD_ERR_CUDA;
  }
  if (cudaEventRecord(ev[2], st) != cudaSuccess) return HPSCD_ERR_CUDA;
  if (async) {
    copy_result_kernel<<<1, 1, 0, st>>>(ctl, async_res);
    if (cudaGetLastError() != cudaSuccess) return HPSCD_ERR_CUDA;
    hpscd_timing& t = ctx->ring_info[slot];
    t = hpscd_timing{};
    t.passes = -1;
    t.x_bytes = m * n * esize(dtype);
    t.grid = P.grid;
    t.kernel_launches = gram_launches + 2;
    ++ctx->ring_calls;
    return HPSCD_OK;
  }
  if (cudaMemcpyAsync(ctx->ctl_host, ctl, sizeof(GridCtl), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return HPSCD_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return HPSCD_ERR_CUDA;
  const GridCtl c = *ctx->ctl_host;
  const int64_t last = o->max_sweeps + p.swap_rounds;  // passes a solve may make, less one
  if (hist && c.sweeps >= 0 && c.sweeps <= last) {
    if (cudaMemcpy(hist, p.hist, (size_t)(c.sweeps + 1) * sizeof(double), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return HPSCD_ERR_CUDA;
  }
  const int64_t nsel = c.sweeps < o->max_sweeps ? c.sweeps : o->max_sweeps;
  if (sel && select && nsel > 0 && c.sweeps <= last) {
    if (cudaMemcpy(sel, p.sel_out, (size_t)nsel * sizeof(int64_t), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return HPSCD_ERR_CUDA;
  }
  if (swaps && p.swap_out &&
      cudaMemcpy(swaps, p.swap_out, (size_t)2 * swap_rounds * sizeof(int64_t), cudaMemcpyDeviceToHost) !=
          cudaSuccess)
    return HPSCD_ERR_CUDA;
  if (sweeps_done) *sweeps_done = c.sweeps;
  if (final_rel_res) *final_rel_res = c.final_res;
  hpscd_timing t{};
  cudaEventElapsedTime(&t.setup_ms, ctx->ev[0], ctx->ev[1]);
  cudaEventElapsedTime(&t.sweep_ms, ctx->ev[1], ctx->ev[2]);
  t.passes = c.passes;
  t.x_bytes = m * n * esize(dtype);
  t.grid = P.grid;
  t.kernel_launches = gram_launches + 1;
  ctx->last = t;
  (void)layout;
  if (c.err != DEV_OK) return HPSCD_ERR_TIMEOUT;
  return c.status;
}


// ---- column-major X with n > 512: the panel sweep ----
struct PanelPlan {
  Plan full, last;  // Gram plans of a full panel and of the last (ragged) one
  int npanels = 0;
  int grid = 0;
  size_t G = 0, Gt = 0, dvec = 0, partial = 0, e = 0, a64 = 0, hacc = 0, npart = 0, ypart = 0,
         hist = 0, ctl = 0, total = 0;
};

void panel_gram_plan(const hpscd_ctx* ctx, int dtype, int64_t m, int nq, Plan* g) {
  g->gp = gram_plan(m, nq, ctx->sms);
  g->tc_ok = gram_tc_plan(dtype, m, nq, ctx->sms, ctx->max_smem, &g->gtc);
  g->ldG = PANEL_W;
}

int make_panel_plan(const hpscd_ctx* ctx, int dtype, int64_t m, int64_t n, const hpscd_opts* o,
                    PanelPlan* P) {
  if (n <= 512 || n > ((int64_t)1 << 30)) return HPSCD_ERR_UNSUPPORTED;
  P->npanels = (int)((n + PANEL_W - 1) / PANEL_W);
  const int nlast = (int)(n - (int64_t)(P->npanels - 1) * PANEL_W);
  panel_gram_plan(ctx, dtype, m, PANEL_W, &P->full);
  panel_gram_plan(ctx, dtype, m, nlast, &P->last);
  P->grid = ctx->sms;
  auto pbytes = [](const Plan& g) {
    return g.tc_ok && g.gtc.partial_bytes > g.gp.partial_bytes ? g.gtc.partial_bytes : g.gp.partial_bytes;
  };
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes, 256);
    return at;
  };
  const size_t pw2 = (size_t)PANEL_W * PANEL_W * sizeof(float);
  P->G = take(pw2);
  P->Gt = take(pw2 * P->npanels);
  P->dvec = take((size_t)P->npanels * PANEL_W * sizeof(float));
  P->partial = take(pbytes(P->full) > pbytes(P->last) ? pbytes(P->full) : pbytes(P->last));
  P->e = take((size_t)((m + 127) / 128 * 128) * sizeof(float));
  P->a64 = take((size_t)n * sizeof(double));
  P->hacc = take((size_t)3 * PANEL_W * sizeof(double));
  P->npart = take((size_t)2 * P->grid * sizeof(double));
  P->ypart = take((size_t)P->grid * sizeof(double));
  P->hist = take((size_t)(o->max_sweeps + 1) * sizeof(double));
  P->ctl = take(sizeof(GridCtl));
  P->total = off;
  return HPSCD_OK;
}

int solve_panel(hpscd_ctx* ctx, const void* X, int dtype, int64_t m, int64_t n, int64_t ld,
                const float* y, float* a, int a_is_guess, const hpscd_opts* o, double* hist,
                int64_t* sweeps_done, double* final_rel_res, const PanelPlan& P) {
  if (m == 0) return solve_empty_rows(ctx, n, a, a_is_guess, o, hist, sweeps_done, final_rel_res);
  char* ws = static_cast<char*>(ctx->ws);
  cudaStream_t st = ctx->stream;
  GridCtl* ctl = reinterpret_cast<GridCtl*>(ws + P.ctl);
  float* G = reinterpret_cast<float*>(ws + P.G);
  float* Gt = reinterpret_cast<float*>(ws + P.Gt);
  float* dvec = reinterpret_cast<float*>(ws + P.dvec);
  if (cudaMemsetAsync(ctl, 0, sizeof(GridCtl), st) != cudaSuccess) return HPSCD_ERR_CUDA;
  if (cudaEventRecord(ctx->ev[0], st) != cudaSuccess) return HPSCD_ERR_CUDA;
  // the panels' diagonal Gram blocks: G~ = D^{-1} G_QQ and d, panel by panel
  const int es = esize(dtype);
  int launches = 0;
  for (int q = 0; q < P.npanels; ++q) {
    const int64_t q0 = (int64_t)q * PANEL_W;
    const int nq = (int)(n - q0 < PANEL_W ? n - q0 : PANEL_W);
    const Plan& g = (q == P.npanels - 1) ? P.last : P.full;
    const void* Xq = static_cast<const char*>(X) + (size_t)q0 * (size_t)ld * es;
    int gl = 0;
    const int rcg = run_gram(ctx, Xq, dtype, m, nq, ld, g, ws + P.partial, G, PANEL_W, &ctl->err,
                             (o->debug_flags & HPSCD_DEBUG_SIMT_GRAM) != 0, &gl,
                             Gt + (size_t)q * PANEL_W * PANEL_W, dvec + q0);
    if (rcg != HPSCD_OK) return rcg;
    launches += gl;
  }
  // the substitution solves each 32-column diagonal block with its inverse
  if (launch_invert_panel_diag(Gt, P.npanels, st) != cudaSuccess) {
    cudaGetLastError();
    return HPSCD_ERR_CUDA;
  }
  ++launches;
  if (cudaMemsetAsync(ws + P.hacc, 0, (size_t)3 * PANEL_W * sizeof(double), st) != cudaSuccess)
    return HPSCD_ERR_CUDA;
  if (cudaEventRecord(ctx->ev[1], st) != cudaSuccess) return HPSCD_ERR_CUDA;
  PanelParams p{};
  p.X = X;
  p.m = m;
  p.n = (int)n;
  p.ld = ld;
  const uintptr_t vec_align = dtype == HPSCD_F32 ? 16 : 8;
  p.vec = ((reinterpret_cast<uintptr_t>(X) % vec_align) == 0 && ld % 4 == 0) ? 1 : 0;
  p.y = y;
  p.e = reinterpret_cast<float*>(ws + P.e);
  p.a_in = a;
  p.warm = a_is_guess ? 1 : 0;
  p.a_out = a;
  p.a64 = reinterpret_cast<double*>(ws + P.a64);
  p.Gt = Gt;
  p.dvec = dvec;
  p.npanels = P.npanels;
  p.hacc = reinterpret_cast<double*>(ws + P.hacc);
  p.npart = reinterpret_cast<double*>(ws + P.npart);
  p.ypart = reinterpret_cast<double*>(ws + P.ypart);
  p.hist = reinterpret_cast<double*>(ws + P.hist);
  p.ctl = ctl;
  p.tol = o->tol;
  p.max_sweeps = o->max_sweeps;
  p.stop_rule = o->stop_rule;
  p.refresh_every = o->refresh_every;
  p.timeout_ns = (uint64_t)(ctx->timeout_s * 1e9);
  p.stall_barrier = (o->debug_flags & HPSCD_DEBUG_STALL_BARRIER) ? 1 : 0;
  // TMA boxes of 128 rows x 64 KB of columns where X allows (16-byte base, ld·elem a
  // multiple of 16), as many stages (at most 4) as fit beside the rest
  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  p.use_tma = 0;
  p.nstages = 0;
  if (ctx->encode && (reinterpret_cast<uintptr_t>(X) & 15) == 0 && ((uint64_t)ld * es) % 16 == 0 &&
      (uint64_t)ld * es < ((uint64_t)1 << 40)) {
    int nst = 4;
    while (nst > 1 && panel_tma_smem(nst) + 8192 > ctx->max_smem) --nst;
    cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)ld * es};
    cuuint32_t box[2] = {128, (cuuint32_t)(PANEL_BOX_BYTES / (128 * es))};
    cuuint32_t estr[2] = {1, 1};
    if (nst >= 2 && ctx->encode(&map, x_tmap_type(dtype), 2, const_cast<void*>(X), dims, strides, box, estr,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
      p.use_tma = 1;
      p.nstages = nst;
    }
  }
  if (launch_panel_sweep(dtype, p, p.use_tma ? &map : nullptr, P.grid, st) != cudaSuccess) {
    cudaGetLastError();
    return HPSCD_ERR_CUDA;
  }
  if (cudaEventRecord(ctx->ev[2], st) != cudaSuccess) return HPSCD_ERR_CUDA;
  if (cudaMemcpyAsync(ctx->ctl_host, ctl, sizeof(GridCtl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return HPSCD_ERR_CUDA;
  const GridCtl c = *ctx->ctl_host;
  if (hist && c.sweeps >= 0 && c.sweeps <= o->max_sweeps &&
      cudaMemcpy(hist, p.hist, (size_t)(c.sweeps + 1) * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return HPSCD_ERR_CUDA;
  if (sweeps_done) *sweeps_done = c.sweeps;
  if (final_rel_res) *final_rel_res = c.final_res;
  hpscd_timing t{};
  cudaEventElapsedTime(&t.setup_ms, ctx->ev[0], ctx->ev[1]);
  cudaEventElapsedTime(&t.sweep_ms, ctx->ev[1], ctx->ev[2]);
  t.passes = c.passes;
  t.x_bytes = m * n * es;
  t.grid = P.grid;
  t.kernel_launches = launches + 1;
  ctx->last = t;
  if (c.err != DEV_OK) return HPSCD_ERR_TIMEOUT;
  return c.status;
}

// ---- routing: which sweep runs a solve, after which one-off relayout of X ----
//   column-major, n <= 512          the tall sweep
//   column-major, n > 512           the panel sweep
//   row-major, m <= 4096            the cluster sweep (16-bit X widened to float32 first)
//   row-major, m > 4096             transposed once to column-major, then as above
enum RouteKind { ROUTE_EMPTY, ROUTE_TALL, ROUTE_PANEL, ROUTE_WIDE };
enum Relayout { RL_NONE, RL_TRANSPOSE, RL_WIDEN };

struct Route {
  RouteKind kind = ROUTE_TALL;
  int relayout = RL_NONE;
  int dtype_k = HPSCD_F32;  // element type the sweep reads
  int64_t ld_k = 0;         // leading dimension the sweep reads
  Plan tall;
  PanelPlan panel;
  WideConfig wc{};
  WideLayout wl;
  size_t xk = 0;            // the relaid copy of X
  size_t xh = 0, yh = 0, ah = 0;  // host entry point: device copies of X, y and a
  size_t total = 0;
};

int make_route(const hpscd_ctx* ctx, int dtype, int layout, int64_t m, int64_t n, int64_t ld,
               const hpscd_opts* o, bool host_copies, Route* R) {
  int rc;
  R->dtype_k = dtype;
  R->ld_k = ld;
  int lay = layout;
  size_t inner = 0;
  if (m == 0) {
    R->kind = ROUTE_EMPTY;
  } else if (n == 0) {
    R->kind = ROUTE_TALL;
    R->ld_k = m;
    if ((rc = make_plan(ctx, dtype, HPSCD_COL_MAJOR, m, n, m, o, false, &R->tall))) return rc;
    inner = R->tall.L.total;
  } else {
    if (lay == HPSCD_ROW_MAJOR) {
      if (wide_config(m, ctx->max_smem, &R->wc)) {
        R->kind = ROUTE_WIDE;
        if (dtype != HPSCD_F32) {
          R->relayout = RL_WIDEN;
          R->dtype_k = HPSCD_F32;
          R->ld_k = (n + 3) / 4 * 4;  // float32 rows on 16-byte boundaries
        }
        if ((rc = make_wide_plan(ctx, R->dtype_k, m, n, R->ld_k, o, false, &R->wc, &R->wl))) return rc;
        inner = R->wl.total;
      } else {
        R->relayout = RL_TRANSPOSE;
        R->ld_k = (m + 31) / 32 * 32;  // columns on 128-byte boundaries (the sweeps' TMA boxes)
        lay = HPSCD_COL_MAJOR;
      }
    }
    if (lay == HPSCD_COL_MAJOR) {
      if (n <= 512) {
        R->kind = ROUTE_TALL;
        if ((rc = make_plan(ctx, dtype, HPSCD_COL_MAJOR, m, n, R->ld_k, o, false, &R->tall))) return rc;
        inner = R->tall.L.total;
      } else {
        R->kind = ROUTE_PANEL;
        if ((rc = make_panel_plan(ctx, dtype, m, n, o, &R->panel))) return rc;
        inner = R->panel.total;
      }
    }
  }
  size_t off = align_up(inner, 256);
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes, 256);
    return at;
  };
  if (R->relayout == RL_TRANSPOSE) R->xk = take((size_t)n * (size_t)R->ld_k * esize(dtype));
  if (R->relayout == RL_WIDEN) R->xk = take((size_t)m * (size_t)R->ld_k * sizeof(float));
  if (host_copies) {
    const size_t xe = layout == HPSCD_COL_MAJOR ? (size_t)(n > 0 ? n : 1) * (size_t)ld
                                                : (size_t)(m > 0 ? m : 1) * (size_t)ld;
    R->xh = take(xe * esize(dtype));
    R->yh = take((size_t)(m > 0 ? m : 1) * sizeof(float));
    R->ah = take((size_t)(n > 0 ? n : 1) * sizeof(float));
  }
  R->total = off;
  return HPSCD_OK;
}

// Runs a routed solve on device buffers (X as given by the caller, or its
// device copy for the host entry point); the workspace holds R.total bytes.
int run_route(hpscd_ctx* ctx, const Route& R, const void* X, int dtype, int64_t m, int64_t n,
              int64_t ld, const float* y, float* a, int a_is_guess, const hpscd_opts* o, double* hist,
              int64_t* sweeps_done, double* final_rel_res) {
  if (R.kind == ROUTE_EMPTY) return solve_empty_rows(ctx, n, a, a_is_guess, o, hist, sweeps_done, final_rel_res);
  char* ws = static_cast<char*>(ctx->ws);
  cudaStream_t st = ctx->stream;
  const void* Xk = X;
  float rl_ms = 0.f;
  if (R.relayout != RL_NONE) {
    Xk = ws + R.xk;
    if (cudaEventRecord(ctx->ev_rl[0], st) != cudaSuccess) return HPSCD_ERR_CUDA;
    const cudaError_t e =
        R.relayout == RL_TRANSPOSE
            ? launch_transpose_to_col(X, dtype, m, n, ld, ws + R.xk, R.ld_k, ctx->sms, st)
            : launch_widen_rows(X, dtype, m, n, ld, reinterpret_cast<float*>(ws + R.xk), R.ld_k, ctx->sms, st);
    if (e != cudaSuccess || cudaEventRecord(ctx->ev_rl[1], st) != cudaSuccess) {
      cudaGetLastError();
      return HPSCD_ERR_CUDA;
    }
  }
  int rc;
  if (R.kind == ROUTE_WIDE)
    rc = solve_wide(ctx, Xk, m, n, R.ld_k, y, a, a_is_guess, o, hist, sweeps_done, final_rel_res, R.wc, R.wl);
  else if (R.kind == ROUTE_PANEL)
    rc = solve_panel(ctx, Xk, R.dtype_k, m, n, R.ld_k, y, a, a_is_guess, o, hist, sweeps_done,
                     final_rel_res, R.panel);
  else
    rc = solve_device(ctx, Xk, R.dtype_k, HPSCD_COL_MAJOR, m, n, R.ld_k, y, a, a_is_guess, o, hist,
                      sweeps_done, final_rel_res, R.tall);
  if (R.relayout != RL_NONE && rc != HPSCD_ERR_CUDA &&
      cudaEventElapsedTime(&rl_ms, ctx->ev_rl[0], ctx->ev_rl[1]) == cudaSuccess) {
    // the relayout is part of the set-up (the cluster sweep times its set-up with its sweeps)
    if (R.kind == ROUTE_WIDE) ctx->last.sweep_ms += rl_ms;
    else ctx->last.setup_ms += rl_ms;
    ctx->last.kernel_launches += 1;
  }
  return rc;
}

}  // namespace

namespace {

void free_ctx(hpscd_ctx* ctx) {
  DeviceGuard g(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  if (ctx->ws && ctx->ws_owned) cudaFree(ctx->ws);
  for (int i = 0; i < 3; ++i)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  for (int i = 0; i < 2; ++i)
    if (ctx->ev_rl[i]) cudaEventDestroy(ctx->ev_rl[i]);
  for (int r = 0; r < hpscd_ctx::RING; ++r)
    for (int i = 0; i < 3; ++i)
      if (ctx->ring_ev[r][i]) cudaEventDestroy(ctx->ring_ev[r][i]);
  if (ctx->ctl_host) cudaFreeHost(ctx->ctl_host);
  if (ctx->host_scratch) cudaFreeHost(ctx->host_scratch);
  if (ctx->trace_dev) cudaFree(ctx->trace_dev);
  delete ctx;
}

}  // namespace

namespace hpscd {
void ctx_retain(hpscd_ctx* ctx) { ++ctx->children; }
void ctx_release(hpscd_ctx* ctx) {
  if (--ctx->children == 0 && ctx->closing) free_ctx(ctx);
}
}  // namespace hpscd

extern "C" {

int hpscd_create(hpscd_ctx** out, int device, void* stream) {
  if (!out) return HPSCD_ERR_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess) { cudaGetLastError(); return HPSCD_ERR_CUDA; }
  if (device < 0 || device >= count) return HPSCD_ERR_INVALID_ARG;
  DeviceGuard g(device);
  if (!g.ok) return HPSCD_ERR_CUDA;
  hpscd_ctx* c = new (std::nothrow) hpscd_ctx();
  if (!c) return HPSCD_ERR_NO_MEMORY;
  c->device = device;
  c->stream = static_cast<cudaStream_t>(stream);
  if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) !=
          cudaSuccess) {
    delete c;
    return HPSCD_ERR_CUDA;
  }
  for (int i = 0; i < 3; ++i)
    if (cudaEventCreate(&c->ev[i]) != cudaSuccess) { hpscd_destroy(c); return HPSCD_ERR_CUDA; }
  for (int i = 0; i < 2; ++i)
    if (cudaEventCreate(&c->ev_rl[i]) != cudaSuccess) { hpscd_destroy(c); return HPSCD_ERR_CUDA; }
  if (cudaMallocHost(reinterpret_cast<void**>(&c->ctl_host), sizeof(GridCtl)) != cudaSuccess) {
    c->ctl_host = nullptr;
    hpscd_destroy(c);
    return HPSCD_ERR_CUDA;
  }
  if (cudaMallocHost(reinterpret_cast<void**>(&c->host_scratch), 2 * sizeof(double)) != cudaSuccess) {
    c->host_scratch = nullptr;
    hpscd_destroy(c);
    return HPSCD_ERR_CUDA;
  }
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
          cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    c->encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  else
    cudaGetLastError();
  *out = c;
  return HPSCD_OK;
}

int hpscd_destroy(hpscd_ctx* ctx) {
  if (!ctx) return HPSCD_OK;
  if (ctx->children > 0) {  // freed by the last batch or network to go
    ctx->closing = true;
    return HPSCD_OK;
  }
  free_ctx(ctx);
  return HPSCD_OK;
}

int hpscd_set_stream(hpscd_ctx* ctx, void* stream) {
  if (!ctx) return HPSCD_ERR_INVALID_ARG;
  ctx->stream = static_cast<cudaStream_t>(stream);
  return HPSCD_OK;
}

int hpscd_set_timeout(hpscd_ctx* ctx, double seconds) {
  if (!ctx || !(seconds > 0.0) || seconds > 3600.0) return HPSCD_ERR_INVALID_ARG;
  ctx->timeout_s = seconds;
  return HPSCD_OK;
}

int hpscd_workspace_size(hpscd_ctx* ctx, int dtype, int layout, int64_t m, int64_t n,
                         const hpscd_opts* opts, size_t* bytes) {
  if (!ctx || !bytes) return HPSCD_ERR_INVALID_ARG;
  int rc = check_opts(opts);
  if (rc) return rc;
  const int64_t ld = layout == HPSCD_COL_MAJOR ? (m > 1 ? m : 1) : (n > 1 ? n : 1);
  if ((rc = check_shape(dtype, layout, m, n, ld))) return rc;
  Route R;
  if ((rc = make_route(ctx, dtype, layout, m, n, ld, opts, false, &R))) return rc;
  *bytes = R.total;
  return HPSCD_OK;
}

int hpscd_set_workspace(hpscd_ctx* ctx, void* ptr, size_t bytes) {
  if (!ctx) return HPSCD_ERR_INVALID_ARG;
  if (ptr && (reinterpret_cast<uintptr_t>(ptr) & 255) != 0) return HPSCD_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->ws && ctx->ws_owned) cudaFree(ctx->ws);
  ctx->ws = ptr;
  ctx->ws_bytes = ptr ? bytes : 0;
  ctx->ws_owned = (ptr == nullptr);
  return HPSCD_OK;
}

int hpscd_solve(hpscd_ctx* ctx, const void* X, int dtype, int layout, int64_t m, int64_t n,
                int64_t ld, const float* y, float* a, int a_is_guess, const hpscd_opts* opts,
                double* hist, int64_t* sweeps_done, double* final_rel_res) {
  if (!ctx) return HPSCD_ERR_INVALID_ARG;
  int rc = check_opts(opts);
  if (rc) return rc;
  if ((rc = check_shape(dtype, layout, m, n, ld))) return rc;
  if ((m > 0 && n > 0 && !X) || (m > 0 && !y) || (n > 0 && !a)) return HPSCD_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return HPSCD_ERR_CUDA;
  Route R;
  if ((rc = make_route(ctx, dtype, layout, m, n, ld, opts, false, &R))) return rc;
  if ((rc = ensure_ws(ctx, R.total))) return rc;
  return run_route(ctx, R, X, dtype, m, n, ld, y, a, a_is_guess, opts, hist, sweeps_done, final_rel_res);
}

int hpscd_solve_blocks(hpscd_ctx* ctx, const void* X, int dtype, int64_t m, int64_t n, int64_t ld,
                       const float* y, float* a, int a_is_guess, int64_t thr,
                       const hpscd_opts* opts, double* hist, int64_t* sweeps_done,
                       double* final_rel_res) {
  if (!ctx || thr < 1) return HPSCD_ERR_INVALID_ARG;
  int rc = check_opts(opts);
  if (rc) return rc;
  if ((rc = check_shape(dtype, HPSCD_COL_MAJOR, m, n, ld))) return rc;
  if ((m > 0 && n > 0 && !X) || (m > 0 && !y) || (n > 0 && !a)) return HPSCD_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return HPSCD_ERR_CUDA;
  Plan P;
  if ((rc = make_plan(ctx, dtype, HPSCD_COL_MAJOR, m, n, ld, opts, false, &P))) return rc;
  if ((rc = ensure_ws(ctx, P.L.total))) return rc;
  const int t = thr > n ? (int)(n > 0 ? n : 1) : (int)thr;
  return solve_device(ctx, X, dtype, HPSCD_COL_MAJOR, m, n, ld, y, a, a_is_guess, opts, hist,
                      sweeps_done, final_rel_res, P, t, 0, nullptr);
}

int hpscd_select(hpscd_ctx* ctx, const void* X, int dtype, int64_t m, int64_t n, int64_t ld,
                 const float* y, float* a, const hpscd_opts* opts, int64_t* sel, double* hist,
                 int64_t* steps_done, double* final_rel_res) {
  if (!ctx) return HPSCD_ERR_INVALID_ARG;
  int rc = check_opts(opts);
  if (rc) return rc;
  if ((rc = check_shape(dtype, HPSCD_COL_MAJOR, m, n, ld))) return rc;
  if (m < 1 || n < 1 || !X || !y || !a || (!sel && opts->max_sweeps > 0)) return HPSCD_ERR_INVALID_ARG;
  if (opts->refresh_every != 0) return HPSCD_ERR_UNSUPPORTED;
  DeviceGuard g(ctx->device);
  if (!g.ok) return HPSCD_ERR_CUDA;
  Plan P;
  if ((rc = make_plan(ctx, dtype, HPSCD_COL_MAJOR, m, n, ld, opts, false, &P))) return rc;
  if ((rc = ensure_ws(ctx, P.L.total))) return rc;
  return solve_device(ctx, X, dtype, HPSCD_COL_MAJOR, m, n, ld, y, a, 0, opts, hist, steps_done,
                      final_rel_res, P, 0, 1, sel);
}

int hpscd_select_swap(hpscd_ctx* ctx, const void* X, int dtype, int64_t m, int64_t n, int64_t ld,
                      const float* y, float* a, const hpscd_opts* opts, int64_t swap_rounds,
                      int64_t* sel, int64_t* swaps, double* hist, int64_t* steps_done,
                      double* final_rel_res) {
  if (!ctx) return HPSCD_ERR_INVALID_ARG;
  int rc = check_opts(opts);
  if (rc) return rc;
  if ((rc = check_shape(dtype, HPSCD_COL_MAJOR, m, n, ld))) return rc;
  if (m < 1 || n < 1 || !X || !y || !a || (!sel && opts->max_sweeps > 0) || swap_rounds < 0 ||
      swap_rounds > (1 << 20) || (!swaps && swap_rounds > 0))
    return HPSCD_ERR_INVALID_ARG;
  if (opts->refresh_every != 0) return HPSCD_ERR_UNSUPPORTED;
  DeviceGuard g(ctx->device);
  if (!g.ok) return HPSCD_ERR_CUDA;
  // the workspace holds the history of the selection steps and the swap steps
  hpscd_opts osz = *opts;
  osz.max_sweeps = opts->max_sweeps + swap_rounds;
  Plan P;
  if ((rc = make_plan(ctx, dtype, HPSCD_COL_MAJOR, m, n, ld, &osz, false, &P, 0, swap_rounds))) return rc;
  if ((rc = ensure_ws(ctx, P.L.total))) return rc;
  return solve_device(ctx, X, dtype, HPSCD_COL_MAJOR, m, n, ld, y, a, 0, opts, hist, steps_done,
                      final_rel_res, P, 0, 1, sel, nullptr, nullptr, nullptr, (int)swap_rounds, swaps);
}

int hpscd_solve_order(hpscd_ctx* ctx, const void* X, int dtype, int64_t m, int64_t n, int64_t ld,
                      const float* y, float* a, int a_is_guess, const int32_t* order,
                      const hpscd_opts* opts, double* hist, int64_t* sweeps_done,
                      double* final_rel_res) {
  if (!ctx) return HPSCD_ERR_INVALID_ARG;
  int rc = check_opts(opts);
  if (rc) return rc;
  if ((rc = check_shape(dtype, HPSCD_COL_MAJOR, m, n, ld))) return rc;
  if ((m > 0 && n > 0 && !X) || (m > 0 && !y) || (n > 0 && !a)) return HPSCD_ERR_INVALID_ARG;
  if (n > 0 && opts->max_sweeps > ((int64_t)1 << 28) / n) return HPSCD_ERR_UNSUPPORTED;
  const int64_t entries = opts->max_sweeps * n;
  if (entries > 0 && !order) return HPSCD_ERR_INVALID_ARG;
  for (int64_t k = 0; k < entries; ++k)
    if (order[k] < 0 || order[k] >= n) return HPSCD_ERR_INVALID_ARG;
  if (dtype != HPSCD_F32) return HPSCD_ERR_UNSUPPORTED;
  DeviceGuard g(ctx->device);
  if (!g.ok) return HPSCD_ERR_CUDA;
  Plan P;
  if ((rc = make_plan(ctx, dtype, HPSCD_COL_MAJOR, m, n, ld, opts, false, &P, entries))) return rc;
  if ((rc = ensure_ws(ctx, P.L.total))) return rc;
  int* order_dev = reinterpret_cast<int*>(static_cast<char*>(ctx->ws) + P.L.order);
  if (entries > 0 && cudaMemcpyAsync(order_dev, order, (size_t)entries * sizeof(int32_t),
                                     cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return HPSCD_ERR_CUDA;
  }
  return solve_device(ctx, X, dtype, HPSCD_COL_MAJOR, m, n, ld, y, a, a_is_guess, opts, hist,
                      sweeps_done, final_rel_res, P, 0, 0, nullptr, order_dev);
}

int hpscd_solve_async(hpscd_ctx* ctx, const void* X, int dtype, int64_t m, int64_t n, int64_t ld,
                      const float* y, float* a, int a_is_guess, const hpscd_opts* opts,
                      double* hist, hpscd_sys_result* res) {
  if (!ctx || !res) return HPSCD_ERR_INVALID_ARG;
  int rc = check_opts(opts);
  if (rc) return rc;
  if ((rc = check_shape(dtype, HPSCD_COL_MAJOR, m, n, ld))) return rc;
  if (m < 1 || n < 1 || !X || !y || !a) return HPSCD_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return HPSCD_ERR_CUDA;
  if (!ctx->ring_ev[0][0]) {
    for (int r = 0; r < hpscd_ctx::RING; ++r)
      for (int i = 0; i < 3; ++i)
        if (cudaEventCreate(&ctx->ring_ev[r][i]) != cudaSuccess) {
          cudaGetLastError();
          return HPSCD_ERR_CUDA;
        }
  }
  Plan P;
  if ((rc = make_plan(ctx, dtype, HPSCD_COL_MAJOR, m, n, ld, opts, false, &P))) return rc;
  if ((rc = ensure_ws(ctx, P.L.total))) return rc;
  return solve_device(ctx, X, dtype, HPSCD_COL_MAJOR, m, n, ld, y, a, a_is_guess, opts, nullptr,
                      nullptr, nullptr, P, 0, 0, nullptr, nullptr, res, hist);
}

int hpscd_async_timings(hpscd_ctx* ctx, int64_t count, hpscd_timing* out) {
  if (!ctx || !out || count < 1 || count > hpscd_ctx::RING || count > ctx->ring_calls)
    return HPSCD_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return HPSCD_ERR_CUDA;
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return HPSCD_ERR_CUDA;
  }
  for (int64_t k = 0; k < count; ++k) {
    const int slot = (int)((ctx->ring_calls - count + k) % hpscd_ctx::RING);
    out[k] = ctx->ring_info[slot];
    if (cudaEventElapsedTime(&out[k].setup_ms, ctx->ring_ev[slot][0], ctx->ring_ev[slot][1]) != cudaSuccess ||
        cudaEventElapsedTime(&out[k].sweep_ms, ctx->ring_ev[slot][1], ctx->ring_ev[slot][2]) != cudaSuccess) {
      cudaGetLastError();
      return HPSCD_ERR_CUDA;
    }
  }
  return HPSCD_OK;
}

int hpscd_solve_host(hpscd_ctx* ctx, const void* X, int dtype, int layout, int64_t m,
                     int64_t n, int64_t ld, const float* y, float* a, int a_is_guess,
                     const hpscd_opts* opts, double* hist, int64_t* sweeps_done,
                     double* final_rel_res) {
  if (!ctx) return HPSCD_ERR_INVALID_ARG;
  int rc = check_opts(opts);
  if (rc) return rc;
  if ((rc = check_shape(dtype, layout, m, n, ld))) return rc;
  if ((m > 0 && n > 0 && !X) || (m > 0 && !y) || (n > 0 && !a)) return HPSCD_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return HPSCD_ERR_CUDA;
  Route R;
  if ((rc = make_route(ctx, dtype, layout, m, n, ld, opts, true, &R))) return rc;
  if ((rc = ensure_ws(ctx, R.total))) return rc;
  char* ws = static_cast<char*>(ctx->ws);
  void* Xd = ws + R.xh;
  float* yd = reinterpret_cast<float*>(ws + R.yh);
  float* ad = reinterpret_cast<float*>(ws + R.ah);
  cudaStream_t st = ctx->stream;
  const size_t xbytes = (m > 0 && n > 0) ? (layout == HPSCD_COL_MAJOR ? (size_t)n * ld * esize(dtype)
                                                                       : (size_t)m * ld * esize(dtype))
                                         : 0;
  if (xbytes && cudaMemcpyAsync(Xd, X, xbytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return HPSCD_ERR_CUDA;
  if (m > 0 && cudaMemcpyAsync(yd, y, (size_t)m * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return HPSCD_ERR_CUDA;
  if (n > 0 && a_is_guess &&
      cudaMemcpyAsync(ad, a, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return HPSCD_ERR_CUDA;
  rc = run_route(ctx, R, Xd, dtype, m, n, ld, yd, ad, a_is_guess, opts, hist, sweeps_done, final_rel_res);
  if (rc == HPSCD_ERR_CUDA || rc == HPSCD_ERR_INVALID_ARG || rc == HPSCD_ERR_UNSUPPORTED) return rc;
  if (n > 0 && cudaMemcpyAsync(a, ad, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return HPSCD_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return HPSCD_ERR_CUDA;
  return rc;
}

int hpscd_set_trace(hpscd_ctx* ctx, int max_passes) {
  if (!ctx || max_passes < 0 || max_passes > 65536) return HPSCD_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (ctx->trace_dev) {
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->trace_dev);
    ctx->trace_dev = nullptr;
  }
  ctx->trace_passes = 0;
  if (max_passes == 0) return HPSCD_OK;
  const size_t words = (size_t)max_passes * 6 + 4096;
  if (cudaMalloc(&ctx->trace_dev, words * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    ctx->trace_dev = nullptr;
    return HPSCD_ERR_NO_MEMORY;
  }
  ctx->trace_passes = max_passes;
  return HPSCD_OK;
}

int hpscd_get_trace(hpscd_ctx* ctx, unsigned long long* out, int64_t words, int64_t* written) {
  if (!ctx || !out || words < 0) return HPSCD_ERR_INVALID_ARG;
  if (!ctx->trace_dev) { if (written) *written = 0; return HPSCD_OK; }
  DeviceGuard g(ctx->device);
  int64_t avail = (int64_t)ctx->trace_passes * 6 + ctx->trace_grid;
  if (words < avail) avail = words;
  if (cudaMemcpy(out, ctx->trace_dev, (size_t)avail * sizeof(unsigned long long),
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return HPSCD_ERR_CUDA;
  if (written) *written = avail;
  return HPSCD_OK;
}

int hpscd_gram(hpscd_ctx* ctx, const void* X, int dtype, int64_t m, int64_t n, int64_t ld,
               float* G, int64_t ldG, int flags) {
  if (!ctx) return HPSCD_ERR_INVALID_ARG;
  int rc = check_shape(dtype, HPSCD_COL_MAJOR, m, n, ld);
  if (rc) return rc;
  if (m < 1 || n < 1 || !X || !G || ldG < n || (flags & ~HPSCD_DEBUG_SIMT_GRAM))
    return HPSCD_ERR_INVALID_ARG;
  DeviceGuard g(ctx->device);
  if (!g.ok) return HPSCD_ERR_CUDA;
  hpscd_opts o{};
  o.max_sweeps = 0;
  Plan P;
  if ((rc = make_plan(ctx, dtype, HPSCD_COL_MAJOR, m, n, ld, &o, false, &P))) return rc;
  if ((rc = ensure_ws(ctx, P.L.total))) return rc;
  char* ws = static_cast<char*>(ctx->ws);
  float* Gw = reinterpret_cast<float*>(ws + P.L.G);
  GridCtl* ctl = reinterpret_cast<GridCtl*>(ws + P.L.ctl);
  cudaStream_t st = ctx->stream;
  if (cudaMemsetAsync(ctl, 0, sizeof(GridCtl), st) != cudaSuccess) return HPSCD_ERR_CUDA;
  if (cudaEventRecord(ctx->ev[0], st) != cudaSuccess) return HPSCD_ERR_CUDA;
  int launches = 0;
  rc = run_gram(ctx, X, dtype, m, n, ld, P, ws + P.L.partial, Gw, P.ldG, &ctl->err,
                (flags & HPSCD_DEBUG_SIMT_GRAM) != 0, &launches);
  if (rc) return rc;
  if (cudaEventRecord(ctx->ev[1], st) != cudaSuccess) return HPSCD_ERR_CUDA;
  if (cudaMemcpy2DAsync(G, (size_t)ldG * sizeof(float), Gw, (size_t)P.ldG * sizeof(float),
                        (size_t)n * sizeof(float), (size_t)n, cudaMemcpyDeviceToDevice, st) !=
      cudaSuccess)
    return HPSCD_ERR_CUDA;
  if (cudaMemcpyAsync(ctx->ctl_host, ctl, sizeof(GridCtl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return HPSCD_ERR_CUDA;
  hpscd_timing t{};
  cudaEventElapsedTime(&t.setup_ms, ctx->ev[0], ctx->ev[1]);
  t.x_bytes = m * n * esize(dtype);
  t.kernel_launches = launches;
  ctx->last = t;
  return ctx->ctl_host->err ? HPSCD_ERR_TIMEOUT : HPSCD_OK;
}

int hpscd_last_timing(hpscd_ctx* ctx, hpscd_timing* out) {
  if (!ctx || !out) return HPSCD_ERR_INVALID_ARG;
  *out = ctx->last;
  return HPSCD_OK;
}

const char* hpscd_status_string(int status) {
  switch (status) {
    case HPSCD_OK: return "ok";
    case HPSCD_ERR_INVALID_ARG: return "invalid argument";
    case HPSCD_ERR_NOT_CONVERGED: return "not converged within max_sweeps";
    case HPSCD_ERR_NONFINITE: return "non-finite residual";
    case HPSCD_ERR_TIMEOUT: return "device-side wait timed out";
    case HPSCD_ERR_CUDA: return "CUDA runtime error";
    case HPSCD_ERR_UNSUPPORTED: return "unsupported shape/layout/dtype";
    case HPSCD_ERR_NO_MEMORY: return "out of workspace memory";
    default: return "unknown status";
  }
}

}  // extern "C"
