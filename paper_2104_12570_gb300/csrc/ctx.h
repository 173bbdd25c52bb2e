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
  hpscd::GridCtl* ctl_host = nullptr;  // pinned
  hpscd_timing last{};
  int trace_passes = 0;                  // 0: tracing off
  unsigned long long* trace_dev = nullptr;
  int trace_grid = 0;
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
};
