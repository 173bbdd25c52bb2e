// hpscd_solve_noalloc: the tall solve with all of its device scratch in one
// file-scope __device__ array instead of cudaMalloc'd workspace.
//
// Who needs it: callers that must not allocate device memory at solve time.
// cudaMalloc/cudaFree can synchronize the device and stall unrelated streams
// (a latency problem for serving loops), and some callers run where another
// allocator already owns the device memory (a framework's caching allocator, a
// fixed per-process memory budget) or where allocation is simply not allowed.
// This entry point allocates nothing: it needs no context (creating one
// allocates events and pinned host memory), takes the caller's stream, and
// works in the array below, which every GPU that loads the library holds
// until the process exits.
#include <cudaTypedefs.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "kernels.h"

using namespace hpscd;

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(24) << 20;  // 24 MiB
constexpr int64_t NOALLOC_MAX_M = int64_t(1) << 20;
constexpr int64_t NOALLOC_MAX_N = 256;
constexpr int64_t NOALLOC_MAX_SWEEPS = 4096;
constexpr int NOALLOC_MAX_KSPLIT = 16;
constexpr int NOALLOC_MAX_DEVICES = 64;

// The shared scratch.  Host code must not pass its name to a kernel: on the
// host it is only a stand-in symbol; the device address comes from
// cudaGetSymbolAddress, once per device, in noalloc_setup().
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

struct NoallocDevice {
  bool ready = false;
  unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch on this device
  int sms = 0;
  int max_smem = 0;
};
NoallocDevice g_devices[NOALLOC_MAX_DEVICES];
std::mutex g_mutex;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
bool g_encode_tried = false;

// Once per device, with that device current.
int noalloc_setup(int dev, NoallocDevice** out) {
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return HPSCD_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  NoallocDevice& d = g_devices[dev];
  if (!d.ready) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return HPSCD_ERR_CUDA;
    }
    if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&d.max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess) {
      cudaGetLastError();
      return HPSCD_ERR_CUDA;
    }
    d.scratch = static_cast<unsigned char*>(ptr);
    d.ready = true;
  }
  if (!g_encode_tried) {
    g_encode_tried = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    else
      cudaGetLastError();
  }
  *out = &d;
  return HPSCD_OK;
}

inline size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// The kernels dereference X, y and a: each must be device (or managed) memory
// that device `dev` can address.  cudaPointerGetAttributes allocates nothing.
bool on_device(const void* ptr, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" int hpscd_solve_noalloc(void* stream, const void* X, int dtype, int64_t m, int64_t n,
                                   int64_t ld, const float* y, float* a, int a_is_guess,
                                   const hpscd_opts* o, double* hist, int64_t* sweeps_done,
                                   double* final_rel_res) {
  // ---- arguments ----
  if (!o || !(o->tol >= 0.0) || !isfinite(o->tol) || o->max_sweeps < 0 ||
      o->stop_rule < HPSCD_STOP_REL_RES || o->stop_rule > HPSCD_STOP_NONE ||
      o->refresh_every < 0 || o->debug_flags != 0)
    return HPSCD_ERR_INVALID_ARG;
  for (int i = 0; i < 5; ++i)
    if (o->reserved[i] != 0) return HPSCD_ERR_INVALID_ARG;
  if (dtype != HPSCD_F32 && dtype != HPSCD_BF16 && dtype != HPSCD_F16) return HPSCD_ERR_INVALID_ARG;
  if (m < 1 || n < 1 || ld < m || !X || !y || !a) return HPSCD_ERR_INVALID_ARG;
  if (m > NOALLOC_MAX_M || n > NOALLOC_MAX_N || o->max_sweeps > NOALLOC_MAX_SWEEPS)
    return HPSCD_ERR_UNSUPPORTED;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return HPSCD_ERR_CUDA; }
  if (!on_device(X, dev) || !on_device(y, dev) || !on_device(a, dev)) return HPSCD_ERR_INVALID_ARG;
  NoallocDevice* d = nullptr;
  int rc = noalloc_setup(dev, &d);
  if (rc != HPSCD_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);

  // ---- plan (same kernels and geometry as hpscd_solve, fewer Gram row splits) ----
  TallConfig cfg;
  if (!tall_config(dtype, (int)n, d->max_smem, &cfg)) return HPSCD_ERR_UNSUPPORTED;
  const GramPlan gp = gram_plan_capped(m, cfg.npad, d->sms, NOALLOC_MAX_KSPLIT);
  const int64_t ntiles = (m + cfg.rows - 1) / cfg.rows;
  int64_t grid64 = d->sms > 256 ? 256 : d->sms;
  if (ntiles < grid64) grid64 = ntiles;
  const int grid = (int)grid64;

  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t at = off; off = up256(off + bytes); return at; };
  const size_t oG = take((size_t)gp.npad * gp.npad * sizeof(float));
  const size_t oGt = take((size_t)gp.npad * gp.npad * sizeof(float));
  const size_t oD = take((size_t)gp.npad * sizeof(float));
  const size_t oPartial = take(gp.partial_bytes);
  const size_t oE = take((size_t)m * sizeof(float));
  const size_t oHacc = take((size_t)3 * cfg.npad * sizeof(double));
  const size_t oNpart = take((size_t)2 * grid * sizeof(double));
  const size_t oGw = take((size_t)2 * cfg.npad * sizeof(float));
  const size_t oYpart = take((size_t)grid * sizeof(double));
  const size_t oHist = take((size_t)(o->max_sweeps + 1) * sizeof(double));
  const size_t oCtl = take(sizeof(GridCtl));
  if (off > NOALLOC_SCRATCH_BYTES) return HPSCD_ERR_UNSUPPORTED;
  unsigned char* ws = d->scratch;
  float* G = reinterpret_cast<float*>(ws + oG);
  GridCtl* ctl = reinterpret_cast<GridCtl*>(ws + oCtl);

  // ---- the scratch keeps the previous call's contents: clear what must start at zero ----
  if (cudaMemsetAsync(ctl, 0, sizeof(GridCtl), st) != cudaSuccess ||
      cudaMemsetAsync(ws + oHacc, 0, (size_t)3 * cfg.npad * sizeof(double), st) != cudaSuccess)
    return HPSCD_ERR_CUDA;
  float* Gt = reinterpret_cast<float*>(ws + oGt);
  float* dvec = reinterpret_cast<float*>(ws + oD);
  if (launch_gram(X, dtype, m, (int)n, ld, gp, reinterpret_cast<double*>(ws + oPartial), G,
                  gp.npad, st) != cudaSuccess ||
      launch_scale_rows(G, gp.npad, (int)n, Gt, dvec, st) != cudaSuccess) {
    cudaGetLastError();
    return HPSCD_ERR_CUDA;
  }

  CUtensorMap map;
  memset(&map, 0, sizeof(map));
  int use_tma = 0;
  const int es = dtype == HPSCD_F32 ? 4 : 2;
  if (g_encode && (reinterpret_cast<uintptr_t>(X) & 15) == 0 && ((uint64_t)ld * es) % 16 == 0) {
    cuuint64_t dims[2] = {(cuuint64_t)m, (cuuint64_t)n};
    cuuint64_t strides[1] = {(cuuint64_t)ld * es};
    cuuint32_t box[2] = {(cuuint32_t)cfg.rows, (cuuint32_t)cfg.box_cols};
    cuuint32_t estr[2] = {1, 1};
    use_tma = g_encode(&map,
                       x_tmap_type(dtype),
                       2, const_cast<void*>(X), dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }

  TallParams p{};
  p.X = X;
  p.m = m;
  p.n = (int)n;
  p.ld = ld;
  p.y = y;
  p.e = reinterpret_cast<float*>(ws + oE);
  p.a_out = a;
  p.a_in = a;
  p.warm = a_is_guess ? 1 : 0;
  p.Gt = Gt;
  p.dvec = dvec;
  p.ldG = gp.npad;
  p.hacc = reinterpret_cast<double*>(ws + oHacc);
  p.npart = reinterpret_cast<double*>(ws + oNpart);
  p.gw = reinterpret_cast<float*>(ws + oGw);
  p.ypart = reinterpret_cast<double*>(ws + oYpart);
  p.hist = reinterpret_cast<double*>(ws + oHist);
  p.ctl = ctl;
  p.tol = o->tol;
  p.max_sweeps = o->max_sweeps;
  p.stop_rule = o->stop_rule;
  p.refresh_every = o->refresh_every;
  p.ntiles = ntiles;
  p.nstages = cfg.nstages;
  p.use_tma = use_tma;
  p.timeout_ns = 5000000000ull;
  p.stall_barrier = 0;
  p.trace = nullptr;
  p.trace_passes = 0;
  p.confirm = 1;  // REL_RES is confirmed on the true residual, as in hpscd_solve
  if (launch_tall_sweep(dtype, cfg, &map, p, grid, st) != cudaSuccess) {
    cudaGetLastError();
    return HPSCD_ERR_CUDA;
  }

  // ---- results (plain host memory; the copies are synchronous) ----
  GridCtl c;
  if (cudaMemcpyAsync(&c, ctl, sizeof(GridCtl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return HPSCD_ERR_CUDA;
  if (hist && c.sweeps >= 0 && c.sweeps <= o->max_sweeps) {
    if (cudaMemcpyAsync(hist, p.hist, (size_t)(c.sweeps + 1) * sizeof(double),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return HPSCD_ERR_CUDA;
  }
  if (sweeps_done) *sweeps_done = c.sweeps;
  if (final_rel_res) *final_rel_res = c.final_res;
  if (c.err != DEV_OK) return HPSCD_ERR_TIMEOUT;
  return c.status;
}
