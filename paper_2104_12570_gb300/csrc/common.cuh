// Device helpers shared by the HPSCD kernels: PTX wrappers for mbarrier and
// TMA (cp.async.bulk.tensor), bounded waits, and a grid barrier for
// cooperatively launched persistent kernels.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hpscd.h"

namespace hpscd {

constexpr unsigned FULL_MASK = 0xffffffffu;

// Device-side error codes written to the control block (host maps them to hpscd_status).
enum DevErr : int { DEV_OK = 0, DEV_TIMEOUT_BARRIER = 1, DEV_TIMEOUT_COPY = 2 };

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of an mbarrier to complete; gives up after
// `timeout_ns` (returns false).  Never spins without bound.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (uint32_t it = 1; it < (1u << 30); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63) == 0 && global_timer_ns() - t0 > timeout_ns) return false;
  }
  return false;
}

// 2-D tiled TMA load of box {c0.., c1..} of `map` into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int32_t c0, int32_t c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const unsigned* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Control block of one persistent launch (device memory, zeroed by the host).
struct GridCtl {
  unsigned arrive;    // grid barrier arrival counter
  unsigned gen;       // grid barrier generation
  int err;            // first device-side error (DevErr)
  int status;         // hpscd_status of the solve
  long long sweeps;   // completed sweeps
  double final_res;   // hist[sweeps]
  long long passes;   // streaming passes made
};

// Grid-wide barrier for a cooperative launch.  Thread 0 of each CTA arrives;
// the last arrival resets the counter and bumps the generation.  Waits are
// bounded by `timeout_ns` and abandoned as soon as any CTA has recorded an
// error.  Returns false (in every thread of the CTA) on timeout or error.
// `expected` is normally gridDim.x; a value above it makes the wait run out
// (the timeout test).
__device__ __forceinline__ bool grid_barrier(GridCtl* ctl, unsigned expected, uint64_t timeout_ns) {
  __shared__ int s_fail;
  __syncthreads();
  if (threadIdx.x == 0) {
    int fail = 0;
    const unsigned g = ld_acquire_u32(&ctl->gen);
    __threadfence();
    const unsigned prev = atomicAdd(&ctl->arrive, 1u);
    if (prev == expected - 1) {
      atomicExch(&ctl->arrive, 0u);
      __threadfence();
      st_release_u32(&ctl->gen, g + 1);
    } else {
      const uint64_t t0 = global_timer_ns();
      for (uint32_t it = 0;; ++it) {
        if (ld_acquire_u32(&ctl->gen) != g) break;
        if ((it & 15) == 15) {
          if (*((volatile int*)&ctl->err) != DEV_OK) { fail = 1; break; }
          if (global_timer_ns() - t0 > timeout_ns || it > (1u << 30)) {
            atomicCAS(&ctl->err, DEV_OK, (int)DEV_TIMEOUT_BARRIER);
            fail = 1;
            break;
          }
          __nanosleep(32);
        }
      }
    }
    s_fail = fail;
  }
  __syncthreads();
  const bool ok = (s_fail == 0);
  __syncthreads();
  return ok;
}

// Named CTA barrier over the first `nthreads` threads (barrier id 1), for
// kernels where a producer warp does not take part in the compute barriers.
__device__ __forceinline__ void named_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}
__device__ __forceinline__ int named_sync_or(int nthreads, int pred) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.s32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.s32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(pred), "r"(nthreads)
      : "memory");
  return r;
}

// grid_barrier for kernels whose compute threads are the first `nthreads`
// of the CTA (named barrier 1 instead of __syncthreads).
__device__ __forceinline__ bool grid_barrier_named(GridCtl* ctl, unsigned expected,
                                                   uint64_t timeout_ns, int nthreads,
                                                   int* s_fail) {
  named_sync(nthreads);
  if (threadIdx.x == 0) {
    int fail = 0;
    const unsigned g = ld_acquire_u32(&ctl->gen);
    __threadfence();
    const unsigned prev = atomicAdd(&ctl->arrive, 1u);
    if (prev == expected - 1) {
      atomicExch(&ctl->arrive, 0u);
      __threadfence();
      st_release_u32(&ctl->gen, g + 1);
    } else {
      const uint64_t t0 = global_timer_ns();
      for (uint32_t it = 0;; ++it) {
        if (ld_acquire_u32(&ctl->gen) != g) break;
        if ((it & 15) == 15) {
          if (*((volatile int*)&ctl->err) != DEV_OK) { fail = 1; break; }
          if (global_timer_ns() - t0 > timeout_ns || it > (1u << 30)) {
            atomicCAS(&ctl->err, DEV_OK, (int)DEV_TIMEOUT_BARRIER);
            fail = 1;
            break;
          }
          __nanosleep(32);
        }
      }
    }
    *s_fail = fail;
  }
  named_sync(nthreads);
  const bool ok = (*((volatile int*)s_fail) == 0);
  named_sync(nthreads);
  return ok;
}

// ---- thread-block clusters: distributed shared memory and the cluster barrier ----
__device__ __forceinline__ uint32_t mapa_u32(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Every thread of every CTA of the cluster arrives (release) and waits (acquire).
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
__device__ __forceinline__ float ld_cluster_f32(uint32_t addr) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ double ld_cluster_f64(uint32_t addr) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ int ld_cluster_s32(uint32_t addr) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ float bf16_bits_to_float(uint16_t b) {
  return __uint_as_float(static_cast<uint32_t>(b) << 16);
}

}  // namespace hpscd
