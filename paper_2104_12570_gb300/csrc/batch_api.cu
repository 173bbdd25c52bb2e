// C ABI of the batched solve (declared in include/hpscd.h): descriptor
// checks, the queue order, the batch workspace, the CUDA graph of a launch
// and the autotuner over the number of CTAs per system.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "ctx.h"

using namespace hpscd;

struct hpscd_batch {
  hpscd_ctx* ctx = nullptr;
  int64_t count = 0;
  int K = 1, clusters = 0, smem = 0, ecap = 0;
  int64_t mmax = 0;
  hpscd_opts opts{};
  void* dev = nullptr;
  hpscd_sys* sys_d = nullptr;
  int* order_d = nullptr;
  int* queue_d = nullptr;
  hpscd_sys_result* res_d = nullptr;
  float* gpart = nullptr;
  float* gfinal = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool launched = false;
  BatchParams params{};
  std::vector<hpscd_sys> sys_host;   // descriptors as given
  int64_t* mn_d = nullptr;           // device int64 m[count], n[count]
  hpscd_mlp* mlp = nullptr;          // learned warm start (optional)
  const float* theta = nullptr;      // device float[count][16]
};

namespace {

constexpr int kMaxN = 256;

struct DevGuard {
  int prev = -1;
  bool ok = false;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
  }
  ~DevGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

inline size_t align256(size_t x) { return (x + 255) / 256 * 256; }

int check_batch_opts(const hpscd_opts* o) {
  if (!o) return HPSCD_ERR_INVALID_ARG;
  if (!(o->tol >= 0.0) || o->tol > 1e300) return HPSCD_ERR_INVALID_ARG;
  if (o->max_sweeps < 0 || o->max_sweeps > ((int64_t)1 << 40)) return HPSCD_ERR_INVALID_ARG;
  if (o->stop_rule < HPSCD_STOP_REL_RES || o->stop_rule > HPSCD_STOP_NONE) return HPSCD_ERR_INVALID_ARG;
  if (o->refresh_every < 0 || o->debug_flags != 0) return HPSCD_ERR_INVALID_ARG;
  for (int i = 0; i < 5; ++i)
    if (o->reserved[i]) return HPSCD_ERR_INVALID_ARG;
  if (o->refresh_every != 0) return HPSCD_ERR_UNSUPPORTED;
  return HPSCD_OK;
}

int check_systems(const hpscd_sys* sys, int64_t count, int64_t* mmax) {
  *mmax = 0;
  for (int64_t i = 0; i < count; ++i) {
    const hpscd_sys& s = sys[i];
    if (s.m < 0 || s.n < 0 || s.reserved != 0) return HPSCD_ERR_INVALID_ARG;
    if (s.n > kMaxN) return HPSCD_ERR_UNSUPPORTED;
    if (s.m > ((int64_t)1 << 30)) return HPSCD_ERR_UNSUPPORTED;
    if (s.ld < (s.m > 1 ? s.m : 1)) return HPSCD_ERR_INVALID_ARG;
    if ((s.m > 0 && s.n > 0 && !s.X) || (s.m > 0 && !s.y) || (s.n > 0 && !s.a))
      return HPSCD_ERR_INVALID_ARG;
    if (s.m > *mmax) *mmax = s.m;
  }
  return HPSCD_OK;
}

void release(hpscd_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->dev) cudaFree(b->dev);
  b->exec = nullptr;
  b->graph = nullptr;
  b->cap = nullptr;
  b->dev = nullptr;
}

// The launch sequence, captured once per configuration: reset the queue,
// [learned warm start: MLP forward + scatter into every system's a], run the
// persistent kernel.
int capture(hpscd_batch* b) {
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return HPSCD_ERR_CUDA;
  bool body = cudaMemsetAsync(b->queue_d, 0, sizeof(int), b->cap) == cudaSuccess;
  if (body && b->mlp && b->count > 0)
    body = mlp_enqueue_warm_start(b->mlp, b->cap, b->theta, b->mn_d, b->mn_d + b->count, b->sys_d,
                                  b->count) == HPSCD_OK;
  body = body && launch_batched(b->params, b->K, b->clusters, b->smem, b->cap) == cudaSuccess;
  const bool ended = cudaStreamEndCapture(b->cap, &b->graph) == cudaSuccess;
  if (!(body && ended && cudaGraphInstantiate(&b->exec, b->graph, 0) == cudaSuccess)) {
    cudaGetLastError();
    return HPSCD_ERR_CUDA;
  }
  return HPSCD_OK;
}

// Fit check and cluster count of a candidate number of CTAs per system.
bool candidate(const hpscd_ctx* ctx, int64_t mmax, int K, int* smem, int* clusters) {
  *smem = batched_smem_bytes(mmax, K);
  if (*smem > ctx->max_smem) return false;
  *clusters = batched_max_clusters(K, *smem, ctx->max_smem);
  return *clusters > 0;
}

int create(hpscd_ctx* ctx, const hpscd_sys* sys, int64_t count, const hpscd_opts* opts, int K,
           int panel, hpscd_batch** out) {
  int64_t mmax = 0;
  int rc = check_systems(sys, count, &mmax);
  if (rc) return rc;
  int smem = 0, clusters = 0;
  if (K == 0) {
    // default: one CTA per system while there are systems enough for every
    // SM; fewer systems than SMs get clusters so every SM has work
    K = 1;
    int s2, c2;
    while (K < 8 && count > 0 && count * K * 2 <= ctx->sms && candidate(ctx, mmax, K * 2, &s2, &c2)) K *= 2;
    if (!candidate(ctx, mmax, K, &smem, &clusters)) {
      for (K = 2; K <= 8 && !candidate(ctx, mmax, K, &smem, &clusters); K *= 2) {}
      if (K > 8) return HPSCD_ERR_UNSUPPORTED;
    }
  } else if (K != 1 && K != 2 && K != 4 && K != 8) {
    return HPSCD_ERR_INVALID_ARG;
  } else if (!candidate(ctx, mmax, K, &smem, &clusters)) {
    return HPSCD_ERR_UNSUPPORTED;
  }
  hpscd_batch* b = new (std::nothrow) hpscd_batch();
  if (!b) return HPSCD_ERR_NO_MEMORY;
  b->ctx = ctx;
  b->count = count;
  b->K = K;
  b->clusters = clusters;
  b->smem = smem;
  b->ecap = batched_ecap(mmax, K);
  b->mmax = mmax;
  b->opts = *opts;
  const int grid = clusters * K;
  const size_t n_sys = (size_t)(count > 0 ? count : 1);
  size_t off = 0;
  const size_t o_sys = off; off = align256(off + n_sys * sizeof(hpscd_sys));
  const size_t o_order = off; off = align256(off + n_sys * sizeof(int));
  const size_t o_queue = off; off = align256(off + sizeof(int));
  const size_t o_res = off; off = align256(off + n_sys * sizeof(hpscd_sys_result));
  const size_t o_gpart = off; off = align256(off + (size_t)grid * 256 * 256 * sizeof(float));
  const size_t o_gfinal = off; off = align256(off + (size_t)clusters * 256 * 256 * sizeof(float));
  const size_t o_mn = off; off = align256(off + 2 * n_sys * sizeof(int64_t));
  if (cudaMalloc(&b->dev, off) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return HPSCD_ERR_NO_MEMORY;
  }
  char* base = static_cast<char*>(b->dev);
  b->sys_d = reinterpret_cast<hpscd_sys*>(base + o_sys);
  b->order_d = reinterpret_cast<int*>(base + o_order);
  b->queue_d = reinterpret_cast<int*>(base + o_queue);
  b->res_d = reinterpret_cast<hpscd_sys_result*>(base + o_res);
  b->gpart = reinterpret_cast<float*>(base + o_gpart);
  b->gfinal = reinterpret_cast<float*>(base + o_gfinal);
  b->mn_d = reinterpret_cast<int64_t*>(base + o_mn);
  std::vector<int64_t> mn((size_t)2 * n_sys, 0);
  for (int64_t i = 0; i < count; ++i) { mn[(size_t)i] = sys[i].m; mn[(size_t)(count + i)] = sys[i].n; }

  // queue order: decreasing m·n (longest first), ties by index
  std::vector<int> order((size_t)count);
  for (int64_t i = 0; i < count; ++i) order[(size_t)i] = (int)i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return sys[x].m * sys[x].n > sys[y].m * sys[y].n;
  });
  cudaStream_t st = ctx->stream;
  if ((count > 0 && (cudaMemcpyAsync(b->sys_d, sys, (size_t)count * sizeof(hpscd_sys),
                                     cudaMemcpyHostToDevice, st) != cudaSuccess ||
                     cudaMemcpyAsync(b->order_d, order.data(), (size_t)count * sizeof(int),
                                     cudaMemcpyHostToDevice, st) != cudaSuccess)) ||
      cudaMemsetAsync(b->res_d, 0, n_sys * sizeof(hpscd_sys_result), st) != cudaSuccess ||
      cudaMemcpyAsync(b->mn_d, mn.data(), mn.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    release(b);
    delete b;
    return HPSCD_ERR_CUDA;
  }

  BatchParams p{};
  p.sys = b->sys_d;
  p.order = b->order_d;
  p.count = (int)count;
  p.queue = b->queue_d;
  p.res = b->res_d;
  p.gpart = b->gpart;
  p.gfinal = b->gfinal;
  p.ecap = b->ecap;
  p.panel = panel;
  p.tol = opts->tol;
  p.max_sweeps = opts->max_sweeps;
  p.stop_rule = opts->stop_rule;

  b->params = p;
  b->sys_host.assign(sys, sys + count);
  bool ok = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess &&
            capture(b) == HPSCD_OK;
  if (!ok) {
    cudaGetLastError();
    release(b);
    delete b;
    return HPSCD_ERR_CUDA;
  }
  ctx_retain(ctx);
  *out = b;
  return HPSCD_OK;
}

}  // namespace

extern "C" {

int hpscd_batch_create(hpscd_ctx* ctx, const hpscd_sys* sys, int64_t count, int dtype,
                       const hpscd_opts* opts, const hpscd_tuning* tuning, hpscd_batch** out) {
  if (!ctx || !out || count < 0 || count > (1 << 30) || (count > 0 && !sys)) return HPSCD_ERR_INVALID_ARG;
  *out = nullptr;
  if (dtype != HPSCD_F32 && dtype != HPSCD_BF16) return HPSCD_ERR_INVALID_ARG;
  if (dtype != HPSCD_F32) return HPSCD_ERR_UNSUPPORTED;
  int rc = check_batch_opts(opts);
  if (rc) return rc;
  int K = 0, panel = 0;
  if (tuning) {
    for (int i = 0; i < 6; ++i)
      if (tuning->reserved[i]) return HPSCD_ERR_INVALID_ARG;
    K = tuning->cluster;
    panel = tuning->panel;
    if (K < 0 || panel < 0 || panel > 2) return HPSCD_ERR_INVALID_ARG;
  }
  DevGuard g(ctx->device);
  if (!g.ok) return HPSCD_ERR_CUDA;
  return create(ctx, sys, count, opts, K, panel, out);
}

int hpscd_batch_launch(hpscd_batch* b) {
  if (!b) return HPSCD_ERR_INVALID_ARG;
  DevGuard g(b->ctx->device);
  if (!g.ok) return HPSCD_ERR_CUDA;
  cudaStream_t st = b->ctx->stream;
  if (cudaEventRecord(b->ctx->ev[1], st) != cudaSuccess || cudaGraphLaunch(b->exec, st) != cudaSuccess ||
      cudaEventRecord(b->ctx->ev[2], st) != cudaSuccess) {
    cudaGetLastError();
    return HPSCD_ERR_CUDA;
  }
  b->launched = true;
  return HPSCD_OK;
}

int hpscd_batch_results(hpscd_batch* b, hpscd_sys_result* out) {
  if (!b || (b->count > 0 && !out)) return HPSCD_ERR_INVALID_ARG;
  DevGuard g(b->ctx->device);
  if (!g.ok) return HPSCD_ERR_CUDA;
  if (cudaStreamSynchronize(b->ctx->stream) != cudaSuccess) { cudaGetLastError(); return HPSCD_ERR_CUDA; }
  if (b->count > 0 &&
      cudaMemcpy(out, b->res_d, (size_t)b->count * sizeof(hpscd_sys_result), cudaMemcpyDeviceToHost) !=
          cudaSuccess) {
    cudaGetLastError();
    return HPSCD_ERR_CUDA;
  }
  if (b->launched) {
    hpscd_timing t{};
    cudaEventElapsedTime(&t.sweep_ms, b->ctx->ev[1], b->ctx->ev[2]);
    int64_t passes = 0;
    for (int64_t i = 0; i < b->count; ++i) passes += out[i].passes;
    t.passes = passes;
    t.grid = b->clusters * b->K;
    t.kernel_launches = 1;
    b->ctx->last = t;
  }
  for (int64_t i = 0; i < b->count; ++i)
    if (out[i].status != HPSCD_OK) return out[i].status;
  return HPSCD_OK;
}

int hpscd_batch_set_warm_start(hpscd_batch* b, hpscd_mlp* mlp, const float* theta) {
  if (!b || (mlp && !theta && b->count > 0)) return HPSCD_ERR_INVALID_ARG;
  if (mlp && mlp_device(mlp) != b->ctx->device) return HPSCD_ERR_INVALID_ARG;
  DevGuard g(b->ctx->device);
  if (!g.ok) return HPSCD_ERR_CUDA;
  if (cudaStreamSynchronize(b->ctx->stream) != cudaSuccess) { cudaGetLastError(); return HPSCD_ERR_CUDA; }
  // the kernel starts every system from its a when a warm start is configured
  std::vector<hpscd_sys> d(b->sys_host);
  if (mlp)
    for (auto& s : d) s.a_is_guess = 1;
  if (b->count > 0 &&
      cudaMemcpy(b->sys_d, d.data(), d.size() * sizeof(hpscd_sys), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return HPSCD_ERR_CUDA;
  }
  if (mlp != b->mlp) {
    if (mlp) mlp_retain(mlp);
    if (b->mlp) mlp_release(b->mlp);
  }
  b->mlp = mlp;
  b->theta = mlp ? theta : nullptr;
  return capture(b);
}

int hpscd_batch_tuning(hpscd_batch* b, hpscd_tuning* out) {
  if (!b || !out) return HPSCD_ERR_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  out->cluster = b->K;
  out->panel = b->params.panel;
  return HPSCD_OK;
}

int hpscd_batch_destroy(hpscd_batch* b) {
  if (!b) return HPSCD_OK;
  hpscd_ctx* ctx = b->ctx;
  {
    DevGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    release(b);
    if (b->mlp) mlp_release(b->mlp);
    delete b;
  }
  ctx_release(ctx);
  return HPSCD_OK;
}

int hpscd_autotune_batch(hpscd_ctx* ctx, const hpscd_sys* sys, int64_t count, int dtype,
                         int64_t trial_sweeps, hpscd_tuning* out, double* ms_per_candidate) {
  if (!ctx || !out || count < 1 || count > (1 << 30) || !sys || trial_sweeps < 1 ||
      trial_sweeps > 1000)
    return HPSCD_ERR_INVALID_ARG;
  if (dtype != HPSCD_F32) return HPSCD_ERR_UNSUPPORTED;
  DevGuard g(ctx->device);
  if (!g.ok) return HPSCD_ERR_CUDA;
  std::vector<hpscd_sys> trial(sys, sys + count);
  for (auto& s : trial) { s.hist = nullptr; s.a_is_guess = 0; }
  hpscd_opts o{};
  o.tol = 0.0;
  o.max_sweeps = trial_sweeps;
  o.stop_rule = HPSCD_STOP_NONE;
  std::vector<hpscd_sys_result> res((size_t)count);
  // event time of a batch planned with (K, panel) and `sweeps` sweeps: the mean
  // of two launches after a warm-up; < 0 when the shape does not fit
  auto time_batch = [&](int K, int panel, int64_t sweeps, double* ms) -> int {
    hpscd_opts os = o;
    os.max_sweeps = sweeps;
    hpscd_batch* b = nullptr;
    int rc = create(ctx, trial.data(), count, &os, K, panel, &b);
    if (rc == HPSCD_ERR_UNSUPPORTED) { *ms = -1.0; return HPSCD_OK; }
    if (rc) return rc;
    float total = 0.f;
    for (int rep = 0; rep < 3 && rc == HPSCD_OK; ++rep) {
      rc = hpscd_batch_launch(b);
      if (rc == HPSCD_OK) rc = hpscd_batch_results(b, res.data());
      if (rep > 0) total += ctx->last.sweep_ms;
    }
    hpscd_batch_destroy(b);
    *ms = total / 2.0;
    return rc;
  };
  double best = -1.0;
  int bestK = 0, bestP = 0;
  const int Ks[4] = {1, 2, 4, 8};
  if (ms_per_candidate)
    for (int i = 0; i < 12; ++i) ms_per_candidate[i] = -1.0;
  for (int ci = 0; ci < 4; ++ci) {
    // the set-up (the Gram of every system) depends on the cluster size only
    double t0 = 0.0;
    int rc = time_batch(Ks[ci], 0, 0, &t0);
    if (rc) return rc;
    if (t0 < 0.0) continue;  // this cluster size does not fit
    for (int pi = 0; pi < 3; ++pi) {
      double tt = 0.0;
      if ((rc = time_batch(Ks[ci], pi, trial_sweeps, &tt))) return rc;
      if (tt < 0.0) continue;
      // candidates are compared on the sweeps alone (the set-up is paid once per
      // solve and does not depend on the panel)
      const double ms = tt - t0 > 0.0 ? tt - t0 : 0.0;
      if (ms_per_candidate) ms_per_candidate[3 * ci + pi] = ms;
      if (best < 0.0 || ms < best) { best = ms; bestK = Ks[ci]; bestP = pi; }
    }
  }
  if (bestK == 0) return HPSCD_ERR_UNSUPPORTED;
  memset(out, 0, sizeof(*out));
  out->cluster = bestK;
  out->panel = bestP;
  return HPSCD_OK;
}

}  // extern "C"
