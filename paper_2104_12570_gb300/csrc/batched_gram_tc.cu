// Tensor-core Gram set-up of a batch: G~ = D^{-1} G and d = diag(G) of every
// system (column-major float32, n <= 256) whose X the TMA can address (16-byte
// base, leading dimension a multiple of 4), one launch for the whole batch.
//
// A persistent CTA per SM pops systems from a queue (the batch's order,
// largest first) and accumulates G = X^T X of one system at a time in tensor
// memory: TMA brings 32-row K blocks of the system's columns (128-byte swizzle,
// through the system's own tensor map), the float32 tiles are split into tf32
// hi/lo, and tcgen05.mma accumulates hi·hi + hi·lo + lo·hi into the lower
// 128x128 tiles ((0,0) or (0,0),(1,0),(1,1)).  The diagonal <X_j, X_j> is
// summed on the CUDA cores from the same tiles (the tensor-core accumulation
// drifts on long sums of positive terms).  The epilogue divides each row by
// its denominator (the ⊘ step of Eq. da2 applied once to the couplings) and
// writes G~ (both triangles) and d into the system's slot, which the sweep
// kernel then reads instead of forming G itself.
// Warp roles and the full/ready/empty protocol are those of gram_tc.cu; the
// stage counters run on across systems, and a block barrier between systems
// keeps the next system's MMAs from overwriting tensor memory that the
// epilogue is still reading.  Every wait is bounded.
#include <string.h>

#include "kernels.h"
#include "tc_common.cuh"

namespace hpscd {

namespace {

using namespace tc;

constexpr int BG_THREADS = 192;  // producer, MMA issuer, 4 workers
constexpr int BG_WORKERS = 128;
constexpr int BG_WORK_WARP0 = 2;
constexpr int KROWS = 32;        // float32 rows per 128-byte K block

struct BatchGramParams {
  const hpscd_sys* sys;
  const int* order;
  int count;
  int* queue;
  const int64_t* gt_off;   // [count]: slot offset (floats), -1: not on this path
  float* gt;
  int* err;
  uint64_t timeout_ns;
  int nstages;
};

__global__ void __launch_bounds__(BG_THREADS, 1)
    batched_gram_tc_kernel(const CUtensorMap* __restrict__ maps, const BatchGramParams p) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int STAGE_RAW = 2 * ATOM_BYTES;      // two 128-column blocks
  constexpr int STAGE_BYTES = 2 * STAGE_RAW;     // raw (then hi) + lo
  const int nst = p.nstages;
  uint64_t* full = reinterpret_cast<uint64_t*>(base + (size_t)nst * STAGE_BYTES);
  uint64_t* ready = full + 8;
  uint64_t* empty = ready + 8;
  uint64_t* done = empty + 8;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* s_fail = reinterpret_cast<int*>(tmem_slot + 1);
  int* s_sys = s_fail + 1;
  float* dsm = reinterpret_cast<float*>(s_sys + 3);  // [256] denominators of the system

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&ready[s], BG_WORKERS / 32);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    *s_fail = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int* vfail = s_fail;
  auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 1;; ++it) {
      if (mbar_try_wait(bar, parity)) return true;
      if ((it & 63) == 0) {
        if (*vfail) return false;
        if (global_timer_ns() - t0 > p.timeout_ns) {
          *vfail = 1;
          atomicExch(p.err, 1);
          return false;
        }
      }
    }
  };

  const int wt = tid - BG_WORK_WARP0 * 32;
  const bool worker = warp >= BG_WORK_WARP0 && warp < BG_WORK_WARP0 + BG_WORKERS / 32;
  int64_t gk = 0;       // K blocks of earlier systems (the stage counters run on)
  uint32_t nsys = 0;    // systems done by this CTA (parity of `done`)
  int64_t pissued = 0;  // producer: K blocks whose copies were issued
  for (;;) {
    if (tid == 0) {
      const int q = atomicAdd(p.queue, 1);
      s_sys[0] = q < p.count ? p.order[q] : -1;
    }
    __syncthreads();
    const int sidx = s_sys[0];
    if (sidx < 0 || *vfail) break;
    const int64_t off = p.gt_off[sidx];
    if (off < 0) { __syncthreads(); continue; }
    const int64_t m = p.sys[sidx].m;
    const int n = (int)p.sys[sidx].n;
    const int nb = n > BLK ? 2 : 1;
    const int ntile = nb == 2 ? 3 : 1;
    const int64_t nkb = (m + KROWS - 1) / KROWS;
    const CUtensorMap* tm = maps + sidx;

    if (warp == 0) {
      // ---------------- producer ----------------
      if (lane == 0) {
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                         reinterpret_cast<uint64_t>(tm))
                     : "memory");
        for (int64_t kb = 0; kb < nkb; ++kb) {
          const int64_t u = gk + kb;
          const int s = (int)(u % nst);
          if (u >= nst && !wait(&empty[s], (uint32_t)(((u / nst) - 1) & 1))) break;
          unsigned char* dst = base + (size_t)s * STAGE_BYTES;
          mbar_arrive_expect_tx(&full[s], (uint32_t)(nb * ATOM_BYTES));
          for (int b = 0; b < nb; ++b)
            tma_load_2d(dst + b * ATOM_BYTES, tm, &full[s], (int32_t)(kb * KROWS), b * BLK);
          pissued = u + 1;
        }
      }
      __syncwarp();
    } else if (warp == 1) {
      // ---------------- MMA issuer ----------------
      if (lane == 0) {
        const uint32_t idesc = make_idesc(2u, BLK);
        for (int64_t kb = 0; kb < nkb; ++kb) {
          const int64_t u = gk + kb;
          const int s = (int)(u % nst);
          if (!wait(&ready[s], (uint32_t)((u / nst) & 1))) break;
          tc_fence_after();
          const uint32_t a_base = smem_u32(base + (size_t)s * STAGE_BYTES);
          for (int t = 0; t < ntile; ++t) {
            // tiles (0,0), (1,0), (1,1): slot of block I and of block J
            const int si = t == 0 ? 0 : 1, sj = t == 2 ? 1 : 0;
            const uint32_t d_tmem = tmem + (uint32_t)(BLK * t);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const uint32_t koff = k * 32;
              const uint64_t ah = make_sw128_desc(a_base + si * ATOM_BYTES + koff);
              const uint64_t bh = make_sw128_desc(a_base + sj * ATOM_BYTES + koff);
              const uint64_t al = make_sw128_desc(a_base + STAGE_RAW + si * ATOM_BYTES + koff);
              const uint64_t bl = make_sw128_desc(a_base + STAGE_RAW + sj * ATOM_BYTES + koff);
              mma_issue<true>(d_tmem, ah, bh, idesc, (kb > 0 || k > 0) ? 1u : 0u);
              mma_issue<true>(d_tmem, ah, bl, idesc, 1u);
              mma_issue<true>(d_tmem, al, bh, idesc, 1u);
            }
          }
          mma_commit(&empty[s]);
        }
        mma_commit(done);
      }
      __syncwarp();
    }

    // ---------------- workers: diagonal sums and the tf32 split ----------------
    constexpr int MAXQ = 16;  // 16-byte chunks per worker per stage (two blocks)
    double dsq64[MAXQ];
    bool ok = true;
    if (worker) {
      float dsq[MAXQ];
#pragma unroll
      for (int q = 0; q < MAXQ; ++q) { dsq[q] = 0.f; dsq64[q] = 0.0; }
      const int nq = 8 * nb;
      for (int64_t kb = 0; kb < nkb; ++kb) {
        const int64_t u = gk + kb;
        const int s = (int)(u % nst);
        int w = 1;
        if (lane == 0) w = wait(&full[s], (uint32_t)((u / nst) & 1)) ? 1 : 0;
        w = __shfl_sync(FULL_MASK, w, 0);
        __syncwarp();
        if (!w) { ok = false; break; }
        unsigned char* st = base + (size_t)s * STAGE_BYTES;
        uint4* raw4 = reinterpret_cast<uint4*>(st);
        uint4* lo4 = reinterpret_cast<uint4*>(st + STAGE_RAW);
#pragma unroll
        for (int q = 0; q < MAXQ; ++q) {
          if (q < nq) {
            const uint4 x = raw4[wt + BG_WORKERS * q];
            const float a0 = __uint_as_float(x.x), a1 = __uint_as_float(x.y);
            const float a2 = __uint_as_float(x.z), a3 = __uint_as_float(x.w);
            dsq[q] = fmaf(a0, a0, fmaf(a1, a1, fmaf(a2, a2, fmaf(a3, a3, dsq[q]))));
            uint4 h, l;
            h.x = x.x & 0xFFFFE000u; h.y = x.y & 0xFFFFE000u;
            h.z = x.z & 0xFFFFE000u; h.w = x.w & 0xFFFFE000u;
            l.x = __float_as_uint(a0 - __uint_as_float(h.x));
            l.y = __float_as_uint(a1 - __uint_as_float(h.y));
            l.z = __float_as_uint(a2 - __uint_as_float(h.z));
            l.w = __float_as_uint(a3 - __uint_as_float(h.w));
            raw4[wt + BG_WORKERS * q] = h;
            lo4[wt + BG_WORKERS * q] = l;
          }
        }
        if ((kb & 63) == 63) {
#pragma unroll
          for (int q = 0; q < MAXQ; ++q) { dsq64[q] += (double)dsq[q]; dsq[q] = 0.f; }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ready[s])) : "memory");
      }
#pragma unroll
      for (int q = 0; q < MAXQ; ++q) dsq64[q] += (double)dsq[q];
      if (ok) {
        int w = 1;
        if (lane == 0) w = wait(done, nsys & 1u) ? 1 : 0;
        w = __shfl_sync(FULL_MASK, w, 0);
        __syncwarp();
        ok = w != 0;
      }
      tc_fence_after();
      // denominators: the 8 workers 8a..8a+7 share column a + 16q
#pragma unroll
      for (int q = 0; q < MAXQ; ++q) {
        double v = dsq64[q];
        v += __shfl_xor_sync(FULL_MASK, v, 1);
        v += __shfl_xor_sync(FULL_MASK, v, 2);
        v += __shfl_xor_sync(FULL_MASK, v, 4);
        const int col = wt / 8 + 16 * q;
        if ((wt & 7) == 0 && q < nq) dsm[col] = col < n ? (float)v : 0.f;
      }
      named_sync(BG_WORKERS + 0 * 32);  // workers only: d of every column
      if (ok && !*vfail) {
        // G~ rows from tensor memory: worker warp w reads lane quarter w % 4
        const int ldg = 32 * ((n + 31) / 32);
        float* G = p.gt + off;
        const int quarter = warp & 3;
        for (int t = 0; t < ntile; ++t) {
          const int I = t == 0 ? 0 : 1, J = t == 2 ? 1 : 0;
          const int i = BLK * I + 32 * quarter + lane;
          const float di = i < n ? dsm[i] : 0.f;
          for (int c0 = 0; c0 < BLK; c0 += 32) {
            if (BLK * J + c0 >= ldg) break;
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + BLK * t + c0, v);
            if (i >= ldg) continue;
#pragma unroll
            for (int k = 0; k < 32; ++k) {
              const int j = BLK * J + c0 + k;
              if (j >= ldg) continue;
              float gij = 0.f;
              if (i < n && j < n && di > 0.f) gij = (i == j) ? 1.f : v[k] / di;
              G[(int64_t)i * ldg + j] = gij;
              if (I != J) {
                const float dj = j < n ? dsm[j] : 0.f;
                G[(int64_t)j * ldg + i] = (i < n && j < n && dj > 0.f) ? v[k] / dj : 0.f;
              }
            }
          }
        }
        // row ldg of the slot: d
        for (int c = wt; c < ldg; c += BG_WORKERS) G[(int64_t)ldg * ldg + c] = c < n ? dsm[c] : 0.f;
      }
    }
    gk += nkb;
    ++nsys;
    tc_fence_before();
    __syncthreads();  // tensor memory and the stages are free for the next system
    tc_fence_after();
  }
  // after a failure, the copies still in flight land before the CTA retires
  if (tid == 0 && *vfail) {
    for (int64_t u = pissued > nst ? pissued - nst : 0; u < pissued; ++u)
      for (uint32_t it = 0; !mbar_try_wait(&full[u % nst], (uint32_t)((u / nst) & 1)); ++it)
        if (it > (1u << 26)) break;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
}

}  // namespace

int batched_gram_tc_smem(int max_smem, int* nstages) {
  constexpr int STAGE_BYTES = 4 * ATOM_BYTES;
  int nst = (max_smem - 1024 - 2048) / STAGE_BYTES;
  if (nst > 4) nst = 4;
  if (nst < 2) return -1;
  *nstages = nst;
  const int smem = nst * STAGE_BYTES + 1024 + 2048;
  return smem;
}

cudaError_t launch_batched_gram_tc(const CUtensorMap* maps, const hpscd_sys* sys, const int* order,
                                   int count, int* queue, const int64_t* gt_off, float* gt, int* err,
                                   uint64_t timeout_ns, int grid, int smem, int nstages,
                                   cudaStream_t stream) {
  BatchGramParams p{};
  p.sys = sys;
  p.order = order;
  p.count = count;
  p.queue = queue;
  p.gt_off = gt_off;
  p.gt = gt;
  p.err = err;
  p.timeout_ns = timeout_ns;
  p.nstages = nstages;
  batched_gram_tc_kernel<<<grid, BG_THREADS, smem, stream>>>(maps, p);
  return cudaGetLastError();
}

cudaError_t batched_gram_tc_prepare(int max_smem) {
  return cudaFuncSetAttribute(batched_gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              max_smem);
}

}  // namespace hpscd
