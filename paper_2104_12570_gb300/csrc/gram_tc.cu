// Tensor-core set-up kernel: G = X^T X of a column-major X with tcgen05.
//
// The sweep needs <X_j, X_j> (the denominators of Eq. da2) and the lower
// triangle of G (Eq. ek1-ek applied inside a sweep).  G is a dense contraction
// over the m rows, the one part of the method that belongs on the tensor
// cores.  Each CTA takes a range of rows (K) and a group of at most four lower
// 128×128 tiles (I, J) of G, streams the 128-column blocks of X those tiles
// need (at most four; two for float32, whose split doubles a stage) through
// shared memory by TMA (128-byte swizzle: each column's K elements are the
// operand's contiguous K-major rows), and accumulates D_IJ = X_I^T X_J in
// tensor memory (128 columns per tile) with tcgen05.mma issued by one thread.
// bfloat16 or IEEE binary16 X: kind::f16 (exact products, float32
// accumulation).  float32 X: kind::tf32 on a two-term split
// x = hi + lo (hi = x with the low 13 mantissa bits dropped, which is what a
// tf32 operand reads of x, so the stage keeps x in place; lo = x - hi, exact,
// rounded to tf32), accumulating hi·hi + hi·lo + lo·hi, which leaves ~2^-21
// relative error per product, of either sign.  A group that holds the full
// square of a pair of diagonal column blocks takes two products instead of
// three: with the split stored as 2·lo (exact), D = H^T H + H^T (2L) and
// (D + D^T) / 2 = H^T H + H^T L + L^T H, the same three terms; the epilogue
// forms the symmetric part through shared memory.  The tensor-core
// accumulation loses accuracy on long sums of positive terms, so the diagonal <X_j, X_j> is summed on the CUDA cores from
// the same shared-memory tiles (float32, float64 across blocks).  Per-split
// float32 partials are summed in a fixed order by gram_tc_reduce_kernel into
// the symmetric G.  The same workers also form X^T y and ||y||^2 from those
// tiles (y read alongside), the dot products of the sweep's starting residual
// e = y of a cold start, so the sweep does not need a pass over X to form them.
#include <cuda_fp16.h>
#include <string.h>

#include "kernels.h"
#include "tc_common.cuh"

namespace hpscd {

namespace {

using namespace tc;

// Worker warps: two per SM sub-partition, so that the split's dependent
// arithmetic of one warp overlaps the other's (with one worker warp per
// sub-partition the split of a float32 stage took about as long as its MMAs).
#ifndef GRAM_WORKER_WARPS
#define GRAM_WORKER_WARPS 8
#endif
constexpr int GT_NWW = GRAM_WORKER_WARPS;
static_assert(GT_NWW == 4 || GT_NWW == 8, "4 or 8 worker warps");
constexpr int GT_THREADS = 64 + 32 * GT_NWW;  // producer, MMA issuer, workers
// Warp roles: warp 0 lane 0 feeds the stages by TMA; warp 1 lane 0 issues
// the MMAs; warps 2.. (the workers; worker warp w reads tensor-memory lane
// quarter w % 4) sum the squares of every column (the diagonal), split
// float32 tiles into tf32 hi/lo, and run the epilogue.  Per stage s and K block kb:
//   full[s]  : TMA bytes landed                 (producer -> workers, MMA for bf16)
//   ready[s] : the workers are done with the tile (workers -> MMA issuer)
//   empty[s] : the MMAs that read the tile completed (tcgen05.commit -> producer)
// so the split of block kb+1 and the copies of later blocks overlap the MMAs
// of block kb.  Every wait is bounded; a wait that gives up raises s_fail, which
// every role polls, and the CTA drains its copies and frees tensor memory.
constexpr int GT_WORK_WARP0 = 2;
constexpr int GT_WORKERS = 32 * GT_NWW;
constexpr int GT_CPS = 1024 / GT_WORKERS;  // 16-byte chunks of a worker per 128-column slot

// 1-D tiled TMA load of `box` elements of `map` from coordinate c0 (rows past
// the tensor's end read as zero), completing on `bar`.
__device__ __forceinline__ void tma_load_1d(void* dst, const CUtensorMap* map, uint64_t* bar, int32_t c0) {
  asm volatile(
      "cp.async.bulk.tensor.1d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2}], [%3];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(smem_u32(bar))
      : "memory");
}

constexpr int YSTAGE_BYTES = 256;  // one K block of y (64 floats at most)

// DT: the storage type of X (HPSCD_F32, HPSCD_BF16 or HPSCD_F16).
template <int DT>
__global__ void __launch_bounds__(GT_THREADS, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap ymap,
                   const GramTCParams p) {
  constexpr bool TF32 = DT == HPSCD_F32;
  constexpr int KB = TF32 ? 32 : 64;         // rows of X per 128-byte K block
  // operand format of the instruction descriptor: tf32 (kind::tf32), else
  // bf16 or f16 (kind::f16, A and B of the same type)
  constexpr uint32_t FMT = TF32 ? 2u : (DT == HPSCD_BF16 ? 1u : 0u);
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // this CTA's group and row split (the splits of group g are CTAs split_base[g]..)
  int g = 0;
  while (g + 1 < p.grp.ngroups && (int)blockIdx.x >= p.grp.split_base[g + 1]) ++g;
  const int split = (int)blockIdx.x - p.grp.split_base[g];
  const int nload = p.grp.nload[g];
  const int ntile = p.grp.ntile[g];
  const bool sym = TF32 && p.grp.sym[g] != 0;
  const int stage_raw = nload * ATOM_BYTES;
  const int stage_bytes = stage_raw * (TF32 ? 2 : 1);
  const int nst = p.nstages;
  // y's K block of each stage (by TMA with the X tiles when p.y_tma)
  float* ystage = reinterpret_cast<float*>(base + (size_t)nst * stage_bytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + (size_t)nst * stage_bytes + nst * YSTAGE_BYTES);
  uint64_t* ready = full + 8;
  uint64_t* empty = ready + 8;
  uint64_t* done = empty + 8;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* s_fail = reinterpret_cast<int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t r0 = (int64_t)split * p.grp.rows_per[g];
  const int64_t r1 = min(p.m, r0 + p.grp.rows_per[g]);
  const int64_t nkb = r1 > r0 ? (r1 - r0 + KB - 1) / KB : 0;

  if (tid == 0) {
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&ready[s], GT_WORKERS / 32);
      // float32: the split is done before the MMAs read the tile, so only the
      // MMA commit frees it; bfloat16: the workers read it alongside the MMAs
      mbar_init(&empty[s], TF32 ? 1 : 1 + GT_WORKERS / 32);
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
  auto fail_now = [&]() {
    *vfail = 1;
    atomicExch(p.err, 1);
  };
  auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (uint32_t it = 1;; ++it) {
      if (mbar_try_wait(bar, parity)) return true;
      if ((it & 63) == 0) {
        if (*vfail) return false;
        if (global_timer_ns() - t0 > p.timeout_ns) { fail_now(); return false; }
      }
    }
  };

  // ---------------- producer: warp 0, lane 0 ----------------
  if (warp == 0) {
    if (lane == 0) {
      int64_t kb = 0;
      for (; kb < nkb; ++kb) {
        const int s = (int)(kb % nst);
        if (kb >= nst && !wait(&empty[s], (uint32_t)(((kb / nst) - 1) & 1))) break;
        unsigned char* dst = base + (size_t)s * stage_bytes;
        mbar_arrive_expect_tx(&full[s], (uint32_t)stage_raw + (p.y_tma ? KB * 4u : 0u));
        for (int b = 0; b < nload; ++b)
          tma_load_2d(dst + b * ATOM_BYTES, &tmap, &full[s], (int32_t)(r0 + kb * KB),
                      p.grp.load_blk[g][b] * BLK);
        if (p.y_tma)
          tma_load_1d(reinterpret_cast<unsigned char*>(ystage) + s * YSTAGE_BYTES, &ymap, &full[s],
                      (int32_t)(r0 + kb * KB));
      }
      // the copies issued land before the CTA may retire
      for (int64_t k = kb - nst > 0 ? kb - nst : 0; k < kb; ++k) {
        const int s = (int)(k % nst);
        for (uint32_t it = 0; !mbar_try_wait(&full[s], (uint32_t)((k / nst) & 1)); ++it)
          if (it > (1u << 26)) break;
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer: warp 1, lane 0 ----------------
    if (lane == 0) {
      // Two tiles (I, J) and (I, J+1) whose J blocks sit next to each other in the
      // stage and whose accumulators are adjacent in tensor memory are one MMA of
      // N = 256 (the B operand spans both blocks): the shared A operand is read
      // once and a third fewer MMAs are issued.
      const uint32_t idesc128 = make_idesc(FMT, BLK), idesc256 = make_idesc(FMT, 2 * BLK);
      for (int64_t kb = 0; kb < nkb; ++kb) {
        const int s = (int)(kb % nst);
        const uint32_t par = (uint32_t)((kb / nst) & 1);
        if (TF32 ? !wait(&ready[s], par) : !wait(&full[s], par)) break;
        tc_fence_after();
        const uint32_t a_base = smem_u32(base + (size_t)s * stage_bytes);
        for (int t = 0; t < ntile; ++t) {
          const uint32_t d_tmem = tmem + (uint32_t)(BLK * t);
          const int si = p.grp.tile_si[g][t], sj = p.grp.tile_sj[g][t];
          const bool pair = t + 1 < ntile && p.grp.tile_si[g][t + 1] == si &&
                            p.grp.tile_sj[g][t + 1] == sj + 1;
          const uint32_t idesc = pair ? idesc256 : idesc128;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t koff = k * 32;
            const uint64_t ah = make_sw128_desc(a_base + si * ATOM_BYTES + koff);
            const uint64_t bh = make_sw128_desc(a_base + sj * ATOM_BYTES + koff);
            const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
            mma_issue<TF32>(d_tmem, ah, bh, idesc, acc);
            if constexpr (TF32) {
              const uint64_t bl = make_sw128_desc(a_base + stage_raw + sj * ATOM_BYTES + koff);
              mma_issue<TF32>(d_tmem, ah, bl, idesc, 1u);  // H^T L (H^T 2L in a full-square group)
              if (!sym) {
                const uint64_t al = make_sw128_desc(a_base + stage_raw + si * ATOM_BYTES + koff);
                mma_issue<TF32>(d_tmem, al, bh, idesc, 1u);
              }
            }
          }
          if (pair) ++t;
        }
        mma_commit(&empty[s]);
      }
      // every MMA issued completes on `done` (also after a failure, before TMEM is freed)
      mma_commit(done);
    }
    __syncwarp();
  }

  // ---------------- workers: warps 2..5 ----------------
  // <X_j, X_j> on the CUDA cores: worker w sums the squares of the 16-byte
  // chunks w + W·q of every stage (W workers), i.e. of column w/8 + (W/8)·(q %
  // GT_CPS) of slot q / GT_CPS (the swizzle only permutes chunks within a
  // column's 128 bytes); float32 per 64 K blocks, float64 across them.  The tensor-core accumulation drifts on long sums of
  // positive terms, so these replace its diagonal.
  // <X_j, y> (when p.y is given): the chunk a worker reads holds K rows
  // 4c..4c+3 (float32; 8c..8c+7 for bfloat16) of its column, c = the logical
  // chunk (w & 7) XOR (column & 7) of the 128-byte swizzle; the column index
  // w/8 + (W/8)·q' has (column & 7) = (w/8) & 7 for every q', so each worker
  // needs the same YR values of y per K block, loaded one block ahead.
  // Float64 accumulation: every 64 K blocks the 8 workers that share a column
  // (8 consecutive lanes) sum their float32 partials with shuffles, and lane j
  // of the 8 keeps the float64 totals of q = j, j+8, ...
  constexpr int MAXQ = 4 * GT_CPS;  // 16-byte chunks per worker per stage (nload <= 4)
  constexpr int YR = TF32 ? 4 : 8;  // rows of a 16-byte chunk
  const int wt = tid - GT_WORK_WARP0 * 32;
  const bool worker = warp >= GT_WORK_WARP0 && warp < GT_WORK_WARP0 + GT_WORKERS / 32;
  bool any_diag = false;
  for (int k = 0; k < nload; ++k) any_diag |= p.grp.diag_slot[g][k] != 0;
  const bool want_y = p.y != nullptr && (any_diag || g == 0);
  const int jl = lane & 7;
  double dsq64[MAXQ / 8], xy64[MAXQ / 8], y2_64 = 0.0;
#pragma unroll
  for (int k = 0; k < MAXQ / 8; ++k) { dsq64[k] = 0.0; xy64[k] = 0.0; }
  if (worker) {
    float dsq[MAXQ], xy[MAXQ], y2 = 0.f;
#pragma unroll
    for (int q = 0; q < MAXQ; ++q) { dsq[q] = 0.f; xy[q] = 0.f; }
    const int nq = GT_CPS * nload;
    const int yoff = YR * ((wt & 7) ^ ((wt >> 3) & 7));  // first K row of the worker's chunk
    float yv[YR], yn[YR];
    // without the TMA copy of y (y not 16-byte aligned): rows r0 + kb·KB + yoff..
    // from global memory, one K block ahead
    const bool yvec = (reinterpret_cast<uintptr_t>(p.y) & 15) == 0;
    const bool yglob = want_y && !p.y_tma;
    auto load_y = [&](int64_t kb, float (&dst)[YR]) {
      const int64_t row0 = r0 + kb * KB + yoff;
      if (!yglob) {
#pragma unroll
        for (int r = 0; r < YR; ++r) dst[r] = 0.f;
      } else if (kb < nkb && yvec && row0 + YR <= p.m) {
#pragma unroll
        for (int r = 0; r < YR; r += 4) {
          const float4 t = __ldg(reinterpret_cast<const float4*>(p.y + row0 + r));
          dst[r] = t.x; dst[r + 1] = t.y; dst[r + 2] = t.z; dst[r + 3] = t.w;
        }
      } else {
#pragma unroll
        for (int r = 0; r < YR; ++r)
          dst[r] = (want_y && kb < nkb && row0 + r < p.m) ? __ldg(p.y + row0 + r) : 0.f;
      }
    };
    load_y(0, yv);
    auto flush = [&]() {
#pragma unroll
      for (int q = 0; q < MAXQ; ++q) {
        if (q < nq) {
          float a = dsq[q], b = xy[q];
          a += __shfl_xor_sync(FULL_MASK, a, 1);
          b += __shfl_xor_sync(FULL_MASK, b, 1);
          a += __shfl_xor_sync(FULL_MASK, a, 2);
          b += __shfl_xor_sync(FULL_MASK, b, 2);
          a += __shfl_xor_sync(FULL_MASK, a, 4);
          b += __shfl_xor_sync(FULL_MASK, b, 4);
          if ((q & 7) == jl) { dsq64[q >> 3] += (double)a; xy64[q >> 3] += (double)b; }
        }
        dsq[q] = 0.f;
        xy[q] = 0.f;
      }
      y2_64 += (double)y2;
      y2 = 0.f;
    };
    for (int64_t kb = 0; kb < nkb; ++kb) {
      const int s = (int)(kb % nst);
      const uint32_t par = (uint32_t)((kb / nst) & 1);
      load_y(kb + 1, yn);  // the next block's rows, in flight while this one is worked on
      int ok = 1;
      if (lane == 0) ok = wait(&full[s], par) ? 1 : 0;
      ok = __shfl_sync(FULL_MASK, ok, 0);
      __syncwarp();
      if (!ok) break;
      unsigned char* st = base + (size_t)s * stage_bytes;
      uint4* raw4 = reinterpret_cast<uint4*>(st);
      uint4* lo4 = reinterpret_cast<uint4*>(st + stage_raw);
      if (want_y && p.y_tma) {
        const float4* ys = reinterpret_cast<const float4*>(
            reinterpret_cast<const unsigned char*>(ystage) + s * YSTAGE_BYTES) + yoff / 4;
#pragma unroll
        for (int r = 0; r < YR; r += 4) {
          const float4 t = ys[r / 4];
          yv[r] = t.x; yv[r + 1] = t.y; yv[r + 2] = t.z; yv[r + 3] = t.w;
        }
      }
#pragma unroll
      for (int r = 0; r < YR; ++r) y2 = fmaf(yv[r], yv[r], y2);
      // 16-bit X: only the slots of diagonal tiles carry sums that are kept
      // (float32 splits every slot)
#pragma unroll
      for (int q = 0; q < MAXQ; ++q) {
        if (q < nq && (TF32 || p.grp.diag_slot[g][q / GT_CPS])) {
          const uint4 x = raw4[wt + GT_WORKERS * q];
          if constexpr (TF32) {
            const float a0 = __uint_as_float(x.x), a1 = __uint_as_float(x.y);
            const float a2 = __uint_as_float(x.z), a3 = __uint_as_float(x.w);
            dsq[q] = fmaf(a0, a0, fmaf(a1, a1, fmaf(a2, a2, fmaf(a3, a3, dsq[q]))));
            xy[q] = fmaf(a0, yv[0], fmaf(a1, yv[1], fmaf(a2, yv[2], fmaf(a3, yv[3], xy[q]))));
            // split: a tf32 operand is x with its low 13 mantissa bits ignored,
            // so x itself stays in place as hi = x & ~0x1fff (no store); lo =
            // x - hi, exact in float32, rounded to tf32 into the second half
            // (2·lo in a full-square group: the scaling is exact)
            const float ls = sym ? 2.f : 1.f;
            uint4 l;
            l.x = __float_as_uint(ls * __uint_as_float(tf32_rna(a0 - __uint_as_float(x.x & 0xffffe000u))));
            l.y = __float_as_uint(ls * __uint_as_float(tf32_rna(a1 - __uint_as_float(x.y & 0xffffe000u))));
            l.z = __float_as_uint(ls * __uint_as_float(tf32_rna(a2 - __uint_as_float(x.z & 0xffffe000u))));
            l.w = __float_as_uint(ls * __uint_as_float(tf32_rna(a3 - __uint_as_float(x.w & 0xffffe000u))));
            lo4[wt + GT_WORKERS * q] = l;
          } else {
            const uint32_t w4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
              float lo16, hi16;  // rows 2h and 2h+1 of the chunk
              if constexpr (DT == HPSCD_BF16) {
                lo16 = __uint_as_float(w4[h] << 16);
                hi16 = __uint_as_float(w4[h] & 0xffff0000u);
              } else {
                lo16 = __half2float(__ushort_as_half((unsigned short)(w4[h] & 0xffffu)));
                hi16 = __half2float(__ushort_as_half((unsigned short)(w4[h] >> 16)));
              }
              dsq[q] = fmaf(lo16, lo16, fmaf(hi16, hi16, dsq[q]));
              xy[q] = fmaf(lo16, yv[2 * h], fmaf(hi16, yv[2 * h + 1], xy[q]));
            }
          }
        }
      }
      if ((kb & 63) == 63) flush();
      if constexpr (TF32) fence_proxy_async_smem();  // the split is visible to the MMAs
      __syncwarp();
      if (lane == 0) {
        if constexpr (TF32) mbar_arrive(&ready[s]);
        else mbar_arrive(&empty[s]);
      }
      if (yglob) {
#pragma unroll
        for (int r = 0; r < YR; ++r) yv[r] = yn[r];
      }
    }
    flush();
  }

  // ---------------- epilogue ----------------
  bool ok = true;
  if (worker) {
    int w = 1;
    if (lane == 0) w = wait(done, 0) ? 1 : 0;
    w = __shfl_sync(FULL_MASK, w, 0);
    __syncwarp();
    ok = w != 0;
  }
  tc_fence_after();
  const int fail = __syncthreads_or((!ok || *vfail) ? 1 : 0);
  if (!fail && worker) {
    // column totals: lane j of each 8-lane group holds q = 8h + j: slot
    // k = q / GT_CPS, column wt/8 + (W/8)·(q % GT_CPS) of the slot
#pragma unroll
    for (int h = 0; h < MAXQ / 8; ++h) {
      const int q = 8 * h + jl, k = q / GT_CPS;
      const int lcol = wt / 8 + (GT_WORKERS / 8) * (q % GT_CPS);  // column within slot k
      if (k < nload && p.grp.diag_slot[g][k]) {
        const size_t at = (size_t)split * p.npad + p.grp.load_blk[g][k] * BLK + lcol;
        p.dpart[at] = dsq64[h];
        if (p.y) p.hpart[at] = xy64[h];
      }
    }
    // ||y||^2 of the split: workers 0..7 of group 0 read every K row once
    if (p.y && g == 0 && wt < 8) {
      double v = y2_64;
      v += __shfl_xor_sync(0xffu, v, 1);
      v += __shfl_xor_sync(0xffu, v, 2);
      v += __shfl_xor_sync(0xffu, v, 4);
      if (wt == 0) p.y2part[split] = v;
    }
    // tensor memory: worker warp w reads lane quarter w % 4 (rows 32·(w%4)..+31);
    // the GT_NWW / 4 warps of a quarter take equal column ranges of each tile
    const int quarter = warp & 3;
    constexpr int CW = BLK / (GT_NWW / 4);
    const int cbeg = CW * ((warp - GT_WORK_WARP0) / 4);
    float* out = p.partial + (size_t)split * p.npad * p.npad;
    auto tile_row = [&](int t, int c0, float (&v)[32]) {
      if (nkb > 0) {
        tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + BLK * t + c0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
      }
    };
    if (sym) {
      // lower tile (I, J) = (D_IJ + D_JI^T) / 2: D_JI goes to shared memory (the
      // stages are idle now), row-major with a padded pitch, and is read back
      // transposed
      constexpr int SP = BLK + 4;
      float* S = reinterpret_cast<float*>(base);
      const int rr = 32 * quarter + lane;
      for (int t = 0; t < ntile; ++t) {
        const int I = p.grp.tile_i[g][t], J = p.grp.tile_j[g][t];
        if (I < J) continue;
        int tt = t;
        for (int u = 0; u < ntile; ++u)
          if (p.grp.tile_i[g][u] == J && p.grp.tile_j[g][u] == I) tt = u;
        for (int c0 = cbeg; c0 < cbeg + CW; c0 += 32) {
          float v[32];
          tile_row(tt, c0, v);
#pragma unroll
          for (int q = 0; q < 8; ++q)
            *reinterpret_cast<float4*>(S + rr * SP + c0 + 4 * q) =
                make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
        asm volatile("bar.sync 1, %0;" ::"n"(GT_WORKERS) : "memory");
        float* orow = out + (size_t)(BLK * I + rr) * p.npad + BLK * J;
        for (int c0 = cbeg; c0 < cbeg + CW; c0 += 32) {
          float v[32];
          tile_row(t, c0, v);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            float w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) w[e] = 0.5f * (v[4 * q + e] + S[(c0 + 4 * q + e) * SP + rr]);
            *reinterpret_cast<float4*>(orow + c0 + 4 * q) = make_float4(w[0], w[1], w[2], w[3]);
          }
        }
        asm volatile("bar.sync 1, %0;" ::"n"(GT_WORKERS) : "memory");
      }
    }
    for (int t = 0; t < (sym ? 0 : ntile); ++t) {
      const int row = BLK * p.grp.tile_i[g][t] + 32 * quarter + lane;
      float* orow = out + (size_t)row * p.npad + BLK * p.grp.tile_j[g][t];
      for (int c0 = cbeg; c0 < cbeg + CW; c0 += 32) {
        float v[32];
        tile_row(t, c0, v);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(orow + c0 + 4 * q) =
              make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
}

// Sum of the per-split partials in two stages (fixed order, so every run
// gives the same G):
//   stage 1: tmp[s][i][j..j+3] = sum over the splits of slice s of the lower
//            partials (float4 loads, independent across threads; one thread
//            per slice, row and 4 columns; a tile's splits are those of the
//            group that holds it), and slice s of d_i = sum_k dpart[k][i] (the
//            CUDA-core diagonal, float64) and, when asked, of (X^T y)_i and
//            ||y||^2, over the same slices of the splits;
//   stage 1b: d, X^T y and ||y||^2: the 16 slice sums added in order;
//   stage 2: G_ij = G_ji = sum_s tmp[s][i][j], G_ii = d_i; optionally
//            G~ = D^{-1} G in both triangles and d as float32.
constexpr int RED_SLICES = 16;
// dsl, hsl: [RED_SLICES][npad] slice sums of the diagonal and X^T y; ysl: [RED_SLICES]
__global__ void gram_tc_reduce1_kernel(const float* __restrict__ partial,
                                       const double* __restrict__ dpart, const GramTCGroups grp, int npad,
                                       float* __restrict__ tmp, double* __restrict__ dsl,
                                       const double* __restrict__ hpart, const double* __restrict__ y2part,
                                       double* __restrict__ hsl, double* __restrict__ ysl) {
  const int n4 = npad / 4;
  const int64_t total = (int64_t)RED_SLICES * npad * n4;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int j4 = (int)(idx % n4);
    const int i = (int)((idx / n4) % npad);
    const int sl = (int)(idx / ((int64_t)n4 * npad));
    if (4 * j4 > i) continue;
    const int ks = grp.tile_splits[i / BLK][(4 * j4) / BLK];
    const int k0 = ks * sl / RED_SLICES, k1 = ks * (sl + 1) / RED_SLICES;
    // float32 over a slice's few splits (the float64 pipe is a small fraction of
    // the float32 one on this part); the 16 slices are added in float64
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll 4
    for (int k = k0; k < k1; ++k) {
      const float4 v = *(reinterpret_cast<const float4*>(partial + ((size_t)k * npad + i) * npad) + j4);
      a0 += v.x; a1 += v.y; a2 += v.z; a3 += v.w;
    }
    *reinterpret_cast<float4*>(tmp + ((size_t)sl * npad + i) * npad + 4 * j4) = make_float4(a0, a1, a2, a3);
    if (j4 == 0) {
      // slice sl of the diagonal and X^T y of block i / BLK (from the group holding
      // tile (I, I)) and of ||y||^2 (from group 0, whose splits cover every row)
      const int kd = grp.tile_splits[i / BLK][i / BLK];
      const int d0 = kd * sl / RED_SLICES, d1 = kd * (sl + 1) / RED_SLICES;
      double dd = 0.0;
      for (int k = d0; k < d1; ++k) dd += dpart[(size_t)k * npad + i];
      dsl[(size_t)sl * npad + i] = dd;
      if (hsl) {
        double hh = 0.0;
        for (int k = d0; k < d1; ++k) hh += hpart[(size_t)k * npad + i];
        hsl[(size_t)sl * npad + i] = hh;
        if (i == 0) {
          const int ky = grp.nsplit[0];
          double yy = 0.0;
          for (int k = ky * sl / RED_SLICES; k < ky * (sl + 1) / RED_SLICES; ++k) yy += y2part[k];
          ysl[sl] = yy;
        }
      }
    }
  }
}

// d_i, (X^T y)_i and ||y||^2: the slice sums in slice order (one thread per row)
__global__ void gram_tc_reduce1b_kernel(const double* __restrict__ dsl, const double* __restrict__ hsl,
                                        const double* __restrict__ ysl, int npad, double* __restrict__ d64,
                                        double* __restrict__ h0, double* __restrict__ y2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  double dd = 0.0, hh = 0.0;
#pragma unroll
  for (int sl = 0; sl < RED_SLICES; ++sl) {
    dd += dsl[(size_t)sl * npad + i];
    if (h0) hh += hsl[(size_t)sl * npad + i];
  }
  d64[i] = dd;
  if (h0) {
    h0[i] = hh;
    if (i == 0) {
      double yy = 0.0;
      for (int sl = 0; sl < RED_SLICES; ++sl) yy += ysl[sl];
      *y2 = yy;
    }
  }
}

__global__ void gram_tc_reduce2_kernel(const float* __restrict__ tmp, const double* __restrict__ d64,
                                       int npad, int n, float* __restrict__ G, int ldG,
                                       float* __restrict__ Gt, float* __restrict__ dvec) {
  const int64_t total = (int64_t)npad * npad;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / npad), j = (int)(idx % npad);
    if (j > i) continue;
    float g;
    if (j == i) {
      g = (float)d64[i];
    } else {
      double sacc = 0.0;
#pragma unroll
      for (int sl = 0; sl < RED_SLICES; ++sl) sacc += tmp[((size_t)sl * npad + i) * npad + j];
      g = (float)sacc;
    }
    G[(int64_t)i * ldG + j] = g;
    G[(int64_t)j * ldG + i] = g;
    if (Gt) {
      const float di = (float)d64[i], dj = (float)d64[j];
      const bool live_i = i < n && di > 0.f, live_j = j < n && dj > 0.f;
      if (j == i) {
        Gt[(int64_t)i * ldG + i] = live_i ? 1.f : 0.f;
        if (dvec) dvec[i] = live_i ? di : 0.f;
      } else {
        Gt[(int64_t)i * ldG + j] = (live_i && j < n) ? g / di : 0.f;
        Gt[(int64_t)j * ldG + i] = (live_j && i < n) ? g / dj : 0.f;
      }
    }
  }
}

}  // namespace

// Adds tile (I, J) to group g, streaming blocks I and J into slots.
static void add_tile(GramTCGroups& G, int g, int I, int J) {
  auto slot = [&](int blk) {
    for (int s = 0; s < G.nload[g]; ++s)
      if (G.load_blk[g][s] == blk) return s;
    G.load_blk[g][G.nload[g]] = blk;
    G.diag_slot[g][G.nload[g]] = 0;
    return G.nload[g]++;
  };
  const int t = G.ntile[g]++;
  G.tile_i[g][t] = I;
  G.tile_j[g][t] = J;
  G.tile_si[g][t] = slot(I);
  G.tile_sj[g][t] = slot(J);
  if (I == J) G.diag_slot[g][G.tile_si[g][t]] = 1;
}

bool gram_tc_plan(int dtype, int64_t m, int n, int sms, int max_smem, GramTCPlan* gp) {
  if (m < 1 || n < 1 || n > 512) return false;
  const int nb = (n + BLK - 1) / BLK;
  gp->npad = nb * BLK;
  GramTCGroups& G = gp->grp;
  memset(&G, 0, sizeof(G));
  // Groups of lower tiles: at most 4 tiles (512 TMEM columns); bfloat16 streams
  // up to 4 column blocks per stage, float32 (whose hi/lo split doubles a
  // stage) at most 2.
  // float32: the diagonal block pairs (0, 1) and (2, 3) as full squares (both
  // (I, J) and (J, I): two products each, see the kernel; 1M x 256 set-up 0.429
  // -> 0.421 ms, 4M x 512 8.63 -> 8.46 ms); a lone diagonal block (n <= 128,
  // where the symmetrizing epilogue did not pay) and the other off-diagonal
  // tiles with three products
  static const int f32_groups[4][6][4][2] = {
      {{{0, 0}, {-1, -1}}},
      {{{0, 0}, {0, 1}, {1, 0}, {1, 1}}},
      {{{0, 0}, {0, 1}, {1, 0}, {1, 1}}, {{2, 0}, {2, 2}, {-1, -1}}, {{2, 1}, {-1, -1}}},
      {{{0, 0}, {0, 1}, {1, 0}, {1, 1}}, {{2, 2}, {2, 3}, {3, 2}, {3, 3}},
       {{2, 0}, {-1, -1}}, {{3, 0}, {-1, -1}}, {{2, 1}, {-1, -1}}, {{3, 1}, {-1, -1}}}};
  static const int f32_sym[4][6] = {{0}, {1}, {1, 0, 0}, {1, 1, 0, 0, 0, 0}};
  static const int bf16_groups[4][3][4][2] = {
      {{{0, 0}, {-1, -1}}},
      {{{0, 0}, {1, 0}, {1, 1}, {-1, -1}}},
      {{{2, 0}, {2, 1}, {2, 2}, {-1, -1}}, {{0, 0}, {1, 0}, {1, 1}, {-1, -1}}},
      {{{3, 0}, {3, 1}, {3, 2}, {3, 3}}, {{2, 0}, {2, 1}, {2, 2}, {-1, -1}},
       {{0, 0}, {1, 0}, {1, 1}, {-1, -1}}}};
  static const int f32_ngroups[4] = {1, 1, 3, 6}, bf16_ngroups[4] = {1, 1, 2, 3};
  const bool f32 = dtype == HPSCD_F32;
  const int ng = f32 ? f32_ngroups[nb - 1] : bf16_ngroups[nb - 1];
  for (int gi = 0; gi < ng; ++gi) {
    const int(*tiles)[2] = f32 ? f32_groups[nb - 1][gi] : bf16_groups[nb - 1][gi];
    const int g = G.ngroups++;
    for (int t = 0; t < 4 && tiles[t][0] >= 0; ++t) add_tile(G, g, tiles[t][0], tiles[t][1]);
    G.sym[g] = f32 ? f32_sym[nb - 1][gi] : 0;
  }
  int maxload = 0;
  for (int g = 0; g < G.ngroups; ++g) maxload = G.nload[g] > maxload ? G.nload[g] : maxload;
  gp->maxload = maxload;
  const int kb_rows = f32 ? 32 : 64;
  const int stage = maxload * ATOM_BYTES * (f32 ? 2 : 1);
  int nst = (max_smem - 2048) / (stage + YSTAGE_BYTES);
  if (nst > 6) nst = 6;
  if (nst < 2) return false;
  gp->nstages = nst;
  gp->smem_bytes = nst * stage + nst * YSTAGE_BYTES + 1024 + 256;
  // one CTA per SM: each CTA allocates all 512 tensor-memory columns
  if (gp->smem_bytes < max_smem / 2 + 4096) gp->smem_bytes = max_smem / 2 + 4096;
  // row splits per group in proportion to its work per K block: for float32 the
  // column blocks it streams (and splits into hi/lo), for 16-bit X its tiles
  // (measured on 4,000,000 x 512: float32 9.6 ms by blocks, 15.6 ms by tiles;
  // bfloat16 2.38 ms by tiles, 2.67 ms by blocks, 2.47 ms with equal splits);
  // at most one CTA per SM in all
  auto weight = [&](int g) { return f32 ? G.nload[g] : G.ntile[g]; };
  int wsum = 0;
  for (int g = 0; g < G.ngroups; ++g) wsum += weight(g);
  const int64_t maxsplit = (m + kb_rows - 1) / kb_rows;
  int total = 0, ksmax = 0;
  for (int g = 0; g < G.ngroups; ++g) {
    int64_t ns = (int64_t)sms * weight(g) / wsum;
    if (ns < 1) ns = 1;
    if (ns > maxsplit) ns = maxsplit;
    int64_t rps = (m + ns - 1) / ns;
    rps = (rps + kb_rows - 1) / kb_rows * kb_rows;
    ns = (m + rps - 1) / rps;
    G.nsplit[g] = (int)ns;
    G.rows_per[g] = rps;
    G.split_base[g] = total;
    total += (int)ns;
    if (ns > ksmax) ksmax = (int)ns;
    for (int t = 0; t < G.ntile[g]; ++t) G.tile_splits[G.tile_i[g][t]][G.tile_j[g][t]] = (int)ns;
  }
  gp->ksplit = ksmax;
  gp->nctas = total;
  gp->rows_per_split = G.rows_per[0];
  gp->partial_bytes = (size_t)gp->ksplit * gp->npad * gp->npad * sizeof(float) +
                      (size_t)gp->ksplit * gp->npad * sizeof(double) +
                      (size_t)RED_SLICES * gp->npad * gp->npad * sizeof(float) +
                      (size_t)gp->npad * sizeof(double) +
                      (size_t)gp->ksplit * gp->npad * sizeof(double) +  // X^T y partials
                      (size_t)gp->ksplit * sizeof(double) +             // ||y||^2 partials
                      (size_t)2 * RED_SLICES * gp->npad * sizeof(double) +  // slice sums of d, X^T y
                      (size_t)RED_SLICES * sizeof(double);              // and of ||y||^2
  return true;
}

cudaError_t launch_gram_tc(const CUtensorMap* tmap, int dtype, int64_t m, const GramTCPlan& gp,
                           float* partial, int* err, uint64_t timeout_ns, float* G, int ldG,
                           cudaStream_t stream, int n, float* Gt, float* dvec, const float* y,
                           double* h0, double* y2, const CUtensorMap* ymap) {
  GramTCParams p{};
  p.m = m;
  p.npad = gp.npad;
  p.grp = gp.grp;
  p.rows_per_split = gp.rows_per_split;
  p.partial = partial;
  p.dpart = reinterpret_cast<double*>(reinterpret_cast<char*>(partial) +
                                      (size_t)gp.ksplit * gp.npad * gp.npad * sizeof(float));
  p.err = err;
  p.timeout_ns = timeout_ns;
  p.nstages = gp.nstages;
  float* tmp = reinterpret_cast<float*>(reinterpret_cast<char*>(p.dpart) +
                                        (size_t)gp.ksplit * gp.npad * sizeof(double));
  double* d64 = reinterpret_cast<double*>(tmp + (size_t)RED_SLICES * gp.npad * gp.npad);
  const bool with_y = y && h0 && y2;
  p.y = with_y ? y : nullptr;
  p.y_tma = (with_y && ymap) ? 1 : 0;
  CUtensorMap ym;
  if (ymap) ym = *ymap;
  else memset(&ym, 0, sizeof(ym));
  p.hpart = d64 + gp.npad;
  p.y2part = p.hpart + (size_t)gp.ksplit * gp.npad;
  double* dsl = p.y2part + gp.ksplit;               // [RED_SLICES][npad]
  double* hsl = dsl + (size_t)RED_SLICES * gp.npad;  // [RED_SLICES][npad]
  double* ysl = hsl + (size_t)RED_SLICES * gp.npad;  // [RED_SLICES]
  dim3 grid(gp.nctas);
  cudaError_t e;
  auto kern = dtype == HPSCD_F32    ? gram_tc_kernel<HPSCD_F32>
              : dtype == HPSCD_BF16 ? gram_tc_kernel<HPSCD_BF16>
                                    : gram_tc_kernel<HPSCD_F16>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, gp.smem_bytes);
  if (e != cudaSuccess) return e;
  kern<<<grid, GT_THREADS, gp.smem_bytes, stream>>>(*tmap, ym, p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t t1 = (int64_t)RED_SLICES * gp.npad * (gp.npad / 4);
  gram_tc_reduce1_kernel<<<(unsigned)((t1 + 255) / 256), 256, 0, stream>>>(
      partial, p.dpart, gp.grp, gp.npad, tmp, dsl, p.hpart, p.y2part, with_y ? hsl : nullptr, ysl);
  gram_tc_reduce1b_kernel<<<(unsigned)((gp.npad + 127) / 128), 128, 0, stream>>>(
      dsl, with_y ? hsl : nullptr, ysl, gp.npad, d64, with_y ? h0 : nullptr, with_y ? y2 : nullptr);
  const int64_t t2 = (int64_t)gp.npad * gp.npad;
  gram_tc_reduce2_kernel<<<(unsigned)((t2 + 255) / 256), 256, 0, stream>>>(tmp, d64, gp.npad, n, G, ldG,
                                                                          Gt, dvec);
  return cudaGetLastError();
}

}  // namespace hpscd
