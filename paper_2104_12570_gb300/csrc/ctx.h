// Library context (private to the C-ABI layer): device, stream, workspace,
// events and tracing state shared by every entry point of one hpscd_ctx.
#pragma once
#include <cudaTypedefs.h>

#include "kernels.h"

struct hpscd_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int sms = 0;
  int max_smem = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_owned = true;
  double timeout_s = 5.0;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_rl[2] = {nullptr, nullptr};  // around a set-up relayout of X
  hpscd::GridCtl* ctl_host = nullptr;  // pinned
  double* host_scratch = nullptr;      // pinned, 2 doubles (the wide path's confirmation)
  hpscd_timing last{};
  int trace_passes = 0;                  // 0: tracing off
  unsigned long long* trace_dev = nullptr;
  int trace_grid = 0;
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  // asynchronous solves: CUDA events of the most recent calls (set-up start,
  // sweep start, sweep end) in a ring, created on the first such call, and
  // what each call launched
  static constexpr int RING = 64;
  cudaEvent_t ring_ev[RING][3] = {};
  hpscd_timing ring_info[RING] = {};
  int64_t ring_calls = 0;
  // batches and networks made on this context: hpscd_destroy while any is
  // alive only marks the context closing; the last one to go frees it
  int children = 0;
  bool closing = false;
};

namespace hpscd {
void ctx_retain(hpscd_ctx* ctx);
void ctx_release(hpscd_ctx* ctx);  // frees a closing context with no children left
}  // namespace hpscd

// Learned warm start inside a batch's graph (mlp.cu): enqueue on `st` the MLP
// forward pass for systems [0, count) of `sys` (theta: device float[count][16];
// m, n: device int64[count]) and write each prediction into the system's a.
struct hpscd_mlp;
namespace hpscd {
int mlp_enqueue_warm_start(hpscd_mlp* p, cudaStream_t st, const float* theta, const int64_t* m,
                           const int64_t* n, const hpscd_sys* sys, int64_t count);
int mlp_device(const hpscd_mlp* p);
// A batch that starts from the network holds it: hpscd_mlp_destroy while a
// batch holds it is deferred until the last holder lets go.
void mlp_retain(hpscd_mlp* p);
void mlp_release(hpscd_mlp* p);
}  // namespace hpscd
