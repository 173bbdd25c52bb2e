// Column sweep of Algorithm 1 for wide systems (row-major X, m <= 4096,
// n >> m): the transposed path.
//
// In a wide system the residual e has only m entries while the sweep is a
// chain of n dependent column steps.  One thread-block cluster of WC CTAs
// walks that chain: CTA c owns rows [r0_c, r1_c) and keeps its slice of e in
// shared memory for the whole solve.  The columns are taken in the paper's
// order in blocks of W = 64.  TMA re-tiles row-major X on the fly: the box
// {64 columns, rows of this CTA} is the block's slab for this CTA.  Per block:
//   1. each CTA forms its partial <X_j, e> (j in the block) over its rows;
//   2. the partials are pushed to every CTA of the cluster through
//      distributed shared memory, with a release-arrive on the receiver's
//      mbarrier (bounded waits, no cluster-wide hardware barrier);
//   3. every CTA sums them in a fixed order and solves the block's chain
//      da_j = (<X_j, e> - sum_{l<j in block} G_jl da_l) / G_jj (Eq. da2 and
//      Eq. ek1-ek inside the block) as s = <X_., e> ⊘ d (the elementwise form
//      of the ⊘ step) followed by da_j = s_j - sum_{l<j} (G_jl / G_jj) da_l,
//      which keeps the division off the dependency chain; the set-up kernel
//      stores each block's Gram with its rows pre-divided by G_jj;
//   4. each CTA applies e <- e - X_block·da to its rows (Eq. ek1-ek) and CTA 0
//      adds da to a.
// After each sweep the cluster forms ||e|| (float64) and tests the stopping
// rule; the chain is latency-bound by construction (n dependent steps).
#include "kernels.h"

namespace hpscd {

namespace {

constexpr int WW = 64;        // columns per block
constexpr int WNT = 512;      // threads per CTA
constexpr int WNW = WNT / 32;

__device__ __forceinline__ void st_cluster_f64(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ void arrive_remote(uint32_t bar_cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(
                   bar_cluster_addr)
               : "memory");
}
__device__ __forceinline__ bool try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool wait_cluster_bounded(uint64_t* bar, uint32_t parity,
                                                     uint64_t timeout_ns) {
  if (try_wait_cluster(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (uint32_t it = 1; it < (1u << 30); ++it) {
    if (try_wait_cluster(bar, parity)) return true;
    if ((it & 63) == 0 && global_timer_ns() - t0 > timeout_ns) return false;
  }
  return false;
}

}  // namespace

// ---- set-up: the 64x64 Gram block of every column block, and d ----
// grid: one CTA per column block; rows streamed with plain loads.
__global__ void __launch_bounds__(256) wide_gram_blocks_kernel(const float* __restrict__ X,
                                                               int64_t m, int64_t n, int64_t ld,
                                                               float* __restrict__ Gb) {
  __shared__ float tile[32][WW + 1];
  const int64_t b = blockIdx.x;
  const int64_t c0 = b * WW;
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;  // 16x16 threads, 4x4 outputs each
  float acc[4][4];
  double acc64[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { acc[i][j] = 0.f; acc64[i][j] = 0.0; }
  int chunks = 0;
  for (int64_t r0 = 0; r0 < m; r0 += 32) {
    for (int idx = tid; idx < 32 * WW; idx += 256) {
      const int r = idx / WW, c = idx % WW;
      const int64_t row = r0 + r, col = c0 + c;
      tile[r][c] = (row < m && col < n) ? X[row * ld + col] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < 32; ++r) {
      float av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { av[i] = tile[r][ty * 4 + i]; bv[i] = tile[r][tx * 4 + i]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
    if (++chunks == 8) {
      chunks = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { acc64[i][j] += acc[i][j]; acc[i][j] = 0.f; }
    }
  }
  // store the block as  d_i on the diagonal and H_ik = G_ik / d_i below it
  // (the couplings pre-divided by the row's denominator; 0 for a zero column),
  // transposed: entry (i, k) at [k][i], so the chain's lanes (one row each)
  // read consecutive words of column k
  __shared__ float gs[WW][WW + 1];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) gs[ty * 4 + i][tx * 4 + j] = (float)(acc64[i][j] + acc[i][j]);
  __syncthreads();
  float* out = Gb + b * (WW * WW);
  for (int idx = tid; idx < WW * WW; idx += 256) {
    const int k = idx / WW, i = idx % WW;
    const float di = gs[i][i];
    float v;
    if (k == i) v = di;
    else if (k < i) v = di > 0.f ? gs[i][k] / di : 0.f;
    else v = 0.f;
    out[idx] = v;
  }
}

// ---- the true residual e = y - X·a of a row-major X (float64-grade) ----
// Stage 1: grid (rows / 8, WS slices of the columns); warp w of a CTA takes
// row blockIdx.x·8 + w over its column slice with Dot2 accumulation (Ogita,
// Rump, Oishi 2005) per lane, then sums the 32 lanes' (s + c) in float64:
// part[row][slice].  Stage 2: per row, the WS slices summed in a fixed order,
// e = y - sum (float32) and (y - sum)^2 in float64 before the rounding.
// Splitting each row over the grid keeps tens of thousands of warps reading X.
constexpr int WS = 32;

__global__ void __launch_bounds__(256) wide_dot2_rows_kernel(const float* __restrict__ X, int64_t m,
                                                             int64_t n, int64_t ld,
                                                             const float* __restrict__ a,
                                                             double* __restrict__ part) {
  const int64_t row = (int64_t)blockIdx.x * 8 + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  const int64_t j0 = n * blockIdx.y / WS, j1 = n * (blockIdx.y + 1) / WS;
  const float* xr = X + row * ld;
  float s = 0.f, c = 0.f;
  for (int64_t j = j0 + lane; j < j1; j += 32) {
    const float xv = __ldg(xr + j), av = __ldg(a + j);
    const float p = xv * av, pe = fmaf(xv, av, -p);
    const float t = s + p, z = t - s;
    c += ((s - (t - z)) + (p - z)) + pe;
    s = t;
  }
  double v = (double)s + (double)c;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL_MASK, v, off);
  if (lane == 0) part[row * WS + blockIdx.y] = v;
}

__global__ void wide_residual_rows_kernel(const double* __restrict__ part, int64_t m,
                                          const float* __restrict__ y, float* __restrict__ e,
                                          double* __restrict__ r2) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= m) return;
  double v = 0.0;
#pragma unroll 8
  for (int k = 0; k < WS; ++k) v += part[row * WS + k];
  const double ed = (double)y[row] - v;
  e[row] = (float)ed;
  if (r2) r2[row] = ed * ed;
}

// *out = sum of r2[0..m) in a fixed order (one CTA)
__global__ void wide_sum_kernel(const double* __restrict__ r2, int64_t m, double* __restrict__ out) {
  __shared__ double ws[32];
  double v = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) v += r2[i];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL_MASK, v, off);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x / 32] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += ws[w];
    *out = t;
  }
}

// ---- the cluster sweep ----
__global__ void __launch_bounds__(WNT, 1)
    wide_sweep_kernel(const __grid_constant__ CUtensorMap tmap, const WideParams p) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int WC = p.csize;
  const uint32_t me = cluster_ctarank();
  const int64_t m = p.m;
  const int64_t n = p.n;
  const int64_t r0 = m * me / WC, r1 = m * (me + 1) / WC;
  const int rows = (int)(r1 - r0);
  const int rows_box = p.rows_box;  // box height (>= rows of every CTA)
  const int nst = p.nstages;
  const int stage_bytes = rows_box * WW * 4;
  float* stages = reinterpret_cast<float*>(base);
  float* es = reinterpret_cast<float*>(base + (size_t)nst * stage_bytes);  // [rows_box, padded to 4]
  float* xbuf = es + ((rows_box + 3) & ~3);    // [2][16][WW] partial dots from each CTA
  float* red = xbuf + 2 * 16 * WW;             // [WNW][WW]
  float* gsum = red + WNW * WW;                // [WW]
  float* da_s = gsum + WW;                     // [WW]
  float* psum = da_s + WW;                     // [WW] this CTA's partial dots
  float* gblk = psum + WW;                     // [2][WW][WW] Gram blocks (double-buffered)
  double* nbuf = reinterpret_cast<double*>(gblk + 2 * WW * WW);  // [16] norm partials
  double* wsum = nbuf + 16;                    // [WNW]
  uint64_t* full = reinterpret_cast<uint64_t*>(wsum + WNW);
  uint64_t* xbar = full + 8;                   // [2] dots exchange, [2] norm exchange
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t nblk = (n + WW - 1) / WW;
  // optional trace (CTA 0, thread 0): for the first trace_passes blocks, the
  // global time after the copy wait, the dots, the exchange, the chain, the update
  uint64_t trace_k = 0;
  auto stamp = [&](int f) {
    if (p.trace && me == 0 && tid == 0 && trace_k < (uint64_t)p.trace_passes)
      p.trace[trace_k * 6 + f] = global_timer_ns();
  };

  if (tid == 0) {
    for (int s = 0; s < nst; ++s) mbar_init(&full[s], 1);
    for (int k = 0; k < 4; ++k) mbar_init(&xbar[k], WC);
    fence_mbar_init();
  }
  for (int r = tid; r < rows_box; r += WNT) es[r] = (r < rows) ? p.e[r0 + r] : 0.f;
  __syncthreads();
  cluster_sync_all();  // every CTA's barriers are initialised before anyone arrives remotely

  uint64_t issued = 0, waited = 0;
  auto issue = [&](uint64_t k) {
    const int s = (int)(k % nst);
    const int64_t b = (int64_t)(k % (uint64_t)nblk);
    mbar_arrive_expect_tx(&full[s], (uint32_t)stage_bytes);
    tma_load_2d(stages + (size_t)s * rows_box * WW, &tmap, &full[s], (int32_t)(b * WW),
                (int32_t)r0);
  };
  const bool tma = p.use_tma != 0;
  if (tid == 0 && tma)
    while (issued < (uint64_t)nst) issue(issued++);

  int err = DEV_OK;
  int status = HPSCD_ERR_NOT_CONVERGED;
  const double ynorm = sqrt(*p.ysq);
  double r_prev = 0.0;
  int64_t sweeps = 0;
  uint64_t kseq = 0;     // block sequence number (all sweeps)
  uint64_t xround = 0;   // exchange rounds (dots)
  uint64_t nround = 0;   // exchange rounds (norms)

  // the residual norm of the CTA's rows, exchanged to every CTA (fixed-order sum)
  auto cluster_norm = [&](double* out) -> bool {
    double v = 0.0;
    for (int r = tid; r < rows; r += WNT) v = fma((double)es[r], (double)es[r], v);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL_MASK, v, off);
    if (lane == 0) wsum[warp] = v;
    __syncthreads();
    const int q = (int)(nround & 1);
    if (tid < WC) {
      double tot = 0.0;
      for (int w = 0; w < WNW; ++w) tot += wsum[w];
      const uint32_t dst = mapa_u32(smem_u32(&nbuf[me]), (uint32_t)tid);
      st_cluster_f64(dst, tot);
      arrive_remote(mapa_u32(smem_u32(&xbar[2 + q]), (uint32_t)tid));
    }
    const bool ok = wait_cluster_bounded(&xbar[2 + q], (uint32_t)((nround / 2) & 1), p.timeout_ns);
    ++nround;
    double t = 0.0;
    for (int c = 0; c < WC; ++c) t += nbuf[c];
    *out = t;
    __syncthreads();  // nbuf is read before the next round overwrites it
    return __syncthreads_or(ok ? 0 : 1) == 0;
  };

  double enorm2 = 0.0;
  if (!cluster_norm(&enorm2)) err = DEV_TIMEOUT_BARRIER;
  double rel = ynorm > 0.0 ? sqrt(enorm2) / ynorm : sqrt(enorm2);
  if (me == 0 && tid == 0) p.hist[0] = rel;
  if (err == DEV_OK) {
    if (!isfinite(rel)) status = HPSCD_ERR_NONFINITE;
    else if (p.stop_rule == HPSCD_STOP_REL_RES && rel <= p.tol && !p.continuing) status = HPSCD_OK;
    else if (p.max_sweeps == 0) status = (p.stop_rule == HPSCD_STOP_NONE) ? HPSCD_OK : HPSCD_ERR_NOT_CONVERGED;
    else status = -1;  // keep sweeping
  }
  r_prev = rel;

  // Gram block of column block b -> gblk[b & 1], by cp.async (16 bytes per thread-step)
  // buffer (k & 1) holds the Gram of block k % nblk, k the block sequence number
  auto prefetch_gram = [&](uint64_t k) {
    const float* src = p.Gb + (int64_t)(k % (uint64_t)nblk) * (WW * WW);
    float* dst = gblk + (k & 1) * (WW * WW);
    for (int i = tid; i < WW * WW / 4; i += WNT)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst + 4 * i)),
                   "l"(src + 4 * i)
                   : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  prefetch_gram(0);

  for (int64_t sw = 1; status == -1 && err == DEV_OK; ++sw) {
    for (int64_t b = 0; b < nblk; ++b, ++kseq) {
      const int s = (int)(kseq % nst);
      prefetch_gram(kseq + 1);  // the next block's Gram, while this one is worked on
      float* st = stages + (size_t)s * rows_box * WW;
      bool ok = true;
      if (tma) {
        ok = mbar_wait_bounded(&full[s], (uint32_t)((kseq / nst) & 1), p.timeout_ns);
      } else {
        // plain loads (row stride not 16-byte aligned); the stage was released
        // by the barrier that ended the previous block
        const int64_t c0 = b * WW;
        for (int idx = tid; idx < rows * WW; idx += WNT) {
          const int r = idx / WW, c = idx % WW;
          st[idx] = (c0 + c < n) ? p.X[(r0 + r) * p.ld + c0 + c] : 0.f;
        }
        __syncthreads();
      }
      // 1. partial dots: warp w takes rows w, w+16, ...; lane the column pair 2·lane
      float p0 = 0.f, p1 = 0.f;
      if (ok) {
        for (int r = warp; r < rows; r += WNW) {
          const float2 xv = *reinterpret_cast<const float2*>(st + r * WW + 2 * lane);
          const float er = es[r];
          p0 = fmaf(xv.x, er, p0);
          p1 = fmaf(xv.y, er, p1);
        }
      }
      red[warp * WW + 2 * lane] = p0;
      red[warp * WW + 2 * lane + 1] = p1;
      stamp(0);
      if (__syncthreads_or(ok ? 0 : 1)) { err = DEV_TIMEOUT_COPY; break; }
      if (tma) ++waited;
      // 2. push this CTA's partials to every CTA of the cluster: thread t < WC
      //    stores the 64 sums into CTA t and then release-arrives on its barrier
      const int q = (int)(xround & 1);
      if (tid < WW) {
        float v = 0.f;
#pragma unroll
        for (int w = 0; w < WNW; ++w) v += red[w * WW + tid];
        psum[tid] = v;
      }
      __syncthreads();
      stamp(1);
      if (tid < WC) {
        const uint32_t dst = mapa_u32(smem_u32(&xbuf[(q * 16 + me) * WW]), (uint32_t)tid);
        const float4* src = reinterpret_cast<const float4*>(psum);
#pragma unroll
        for (int j4 = 0; j4 < WW / 4; ++j4) {
          const float4 v = src[j4];
          asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(dst + 16 * j4),
                       "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                       : "memory");
        }
        arrive_remote(mapa_u32(smem_u32(&xbar[q]), (uint32_t)tid));
      }
      ok = wait_cluster_bounded(&xbar[q], (uint32_t)((xround / 2) & 1), p.timeout_ns);
      ++xround;
      stamp(2);
      // 3. sum in a fixed order, then the block's chain in warp 0
      if (tid < WW) {
        float g = 0.f;
        for (int c = 0; c < WC; ++c) g += xbuf[(q * 16 + c) * WW + tid];
        gsum[tid] = g;
      }
      asm volatile("cp.async.wait_group 1;" ::: "memory");  // this block's Gram has landed
      if (__syncthreads_or(ok ? 0 : 1)) { err = DEV_TIMEOUT_BARRIER; break; }
      if (warp == 0) {
        const float* Gb = gblk + (kseq & 1) * (WW * WW);
        const int64_t c0 = b * WW;
        // the ⊘ step on the block's numerators (elementwise, off the chain),
        // then da_k = s_k - sum_{l<k} H_kl da_l with H = D^{-1}·(strict lower G):
        // lane owns block rows lane (slot 0) and lane + 32 (slot 1)
        // Gb holds the block transposed: entry (i, k) at Gb[k * WW + i]
        const float d_0 = (c0 + lane < n) ? Gb[lane * WW + lane] : 0.f;
        const float d_1 = (c0 + lane + 32 < n) ? Gb[(lane + 32) * WW + lane + 32] : 0.f;
        float s_0 = d_0 > 0.f ? gsum[lane] / d_0 : 0.f;
        float s_1 = d_1 > 0.f ? gsum[lane + 32] / d_1 : 0.f;
        float m_0 = 0.f, m_1 = 0.f;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const float h0 = Gb[k * WW + lane];
          const float h1 = Gb[k * WW + lane + 32];
          const float qk = __shfl_sync(FULL_MASK, s_0, k);
          if (lane == k) m_0 = qk;
          if (lane > k) s_0 = fmaf(-h0, qk, s_0);
          s_1 = fmaf(-h1, qk, s_1);
        }
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const float h1 = Gb[(32 + k) * WW + lane + 32];
          const float qk = __shfl_sync(FULL_MASK, s_1, k);
          if (lane == k) m_1 = qk;
          if (lane > k) s_1 = fmaf(-h1, qk, s_1);
        }
        da_s[lane] = m_0;
        da_s[lane + 32] = m_1;
      }
      __syncthreads();
      stamp(3);
      // 4. e <- e - X_block·da for this CTA's rows; a += da (CTA 0).  Four
      //    threads per row, 16 columns each, walked from a start that depends
      //    on the row and on the part (parts 0 and 2, 1 and 3 share banks), so
      //    the 32 lanes of a warp read 32 different banks at every step.
      // the bound is a multiple of 32: every lane of a warp takes the same trip
      // count, as the full-mask shuffles below require
      const int nt4 = ((4 * rows_box + 31) / 32) * 32;
      for (int t = tid; t < nt4; t += WNT) {
        const int r = t >> 2, part = t & 3;
        float acc0 = 0.f, acc1 = 0.f;
        if (r < rows) {
          const float* xr = st + r * WW + 16 * part;
          const float* dr = da_s + 16 * part;
          const int sh = r + 8 * (part >> 1);
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const int c0i = (j + sh) & 15, c1i = (j + 1 + sh) & 15;
            acc0 = fmaf(xr[c0i], dr[c0i], acc0);
            acc1 = fmaf(xr[c1i], dr[c1i], acc1);
          }
        }
        float acc = acc0 + acc1;
        acc += __shfl_xor_sync(FULL_MASK, acc, 1);
        acc += __shfl_xor_sync(FULL_MASK, acc, 2);
        if (part == 0 && r < rows) es[r] -= acc;
      }
      // this sweep's da of the block, store only (a is updated after the sweep)
      if (me == 0 && tid < WW && b * WW + tid < n) p.dsw[b * WW + tid] = da_s[tid];
      __syncthreads();  // the stage and da_s are free
      stamp(4);
      ++trace_k;
      if (tid == 0 && tma) {
        fence_proxy_async_smem();
        issue(issued++);
      }
    }
    if (err != DEV_OK) break;
    sweeps = sw;
    // a += this sweep's da: CTA 0's stores are made visible before the norm
    // exchange (a cluster-scope release), then every CTA adds a slice
    __threadfence();
    if (!cluster_norm(&enorm2)) { err = DEV_TIMEOUT_BARRIER; break; }
    for (int64_t j = (int64_t)me * WNT + tid; j < n; j += (int64_t)WC * WNT)
      p.a64[j] += (double)__ldcg(p.dsw + j);
    rel = ynorm > 0.0 ? sqrt(enorm2) / ynorm : sqrt(enorm2);
    if (me == 0 && tid == 0) p.hist[sw] = rel;
    if (!isfinite(rel)) status = HPSCD_ERR_NONFINITE;
    else if (p.stop_rule == HPSCD_STOP_REL_RES && rel <= p.tol) status = HPSCD_OK;
    else if (p.stop_rule == HPSCD_STOP_REL_CHANGE && (r_prev == 0.0 || fabs(r_prev - rel) < p.tol * r_prev)) status = HPSCD_OK;
    else if (sw == p.max_sweeps) status = (p.stop_rule == HPSCD_STOP_NONE) ? HPSCD_OK : HPSCD_ERR_NOT_CONVERGED;
    r_prev = rel;
  }

  // drain copies in flight; write e and the results
  asm volatile("cp.async.wait_all;" ::: "memory");
  if (tid == 0) {
    for (uint64_t k = waited; k < issued; ++k)
      if (!mbar_wait_bounded(&full[k % nst], (uint32_t)((k / nst) & 1), p.timeout_ns)) {
        if (err == DEV_OK) err = DEV_TIMEOUT_COPY;
        break;
      }
  }
  for (int r = tid; r < rows; r += WNT) p.e[r0 + r] = es[r];
  if (err != DEV_OK && tid == 0) atomicCAS(&p.ctl->err, DEV_OK, err);
  if (me == 0 && tid == 0) {
    p.ctl->status = (err != DEV_OK) ? HPSCD_ERR_TIMEOUT : (status == -1 ? HPSCD_ERR_NOT_CONVERGED : status);
    p.ctl->sweeps = sweeps;
    p.ctl->final_res = r_prev;
    p.ctl->passes = sweeps;
  }
  __syncthreads();
  // no CTA leaves while another may still write into its shared memory
  cluster_sync_all();
}

// ||y||^2 in float64, one CTA, fixed order (m <= 4096)
__global__ void wide_ynorm_kernel(const float* __restrict__ y, int64_t m, double* __restrict__ out) {
  __shared__ double ws[32];
  double v = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) v = fma((double)y[i], (double)y[i], v);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL_MASK, v, off);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x / 32] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += ws[w];
    *out = t;
  }
}

__global__ void wide_finish_kernel(const double* __restrict__ a64, float* __restrict__ a, int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    a[j] = (float)a64[j];
}

__global__ void wide_init_kernel(const float* __restrict__ a_in, int warm, double* __restrict__ a64,
                                 float* __restrict__ a_tmp, int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const float v = warm ? a_in[j] : 0.f;
    a64[j] = (double)v;
    a_tmp[j] = v;
  }
}

bool wide_config(int64_t m, int max_smem, WideConfig* cfg) {
  if (m < 1 || m > 4096) return false;
  int csize = 16;
  while (csize > 1 && (m + csize - 1) / csize < 8) csize /= 2;  // small m: fewer CTAs
  cfg->csize = csize;
  cfg->rows_box = (int)((m + csize - 1) / csize);
  if (cfg->rows_box > 256) return false;
  const int stage = cfg->rows_box * WW * 4;
  const int fixed = 1024 + ((cfg->rows_box + 3) & ~3) * 4 + 2 * 16 * WW * 4 + WNW * WW * 4 + 3 * WW * 4 +
                    2 * WW * WW * 4 + 16 * 8 + WNW * 8 + 16 * 8 + 256;
  int nst = (max_smem - fixed) / stage;
  if (nst > 8) nst = 8;
  if (nst < 2) return false;
  cfg->nstages = nst;
  cfg->smem_bytes = fixed + nst * stage;
  return true;
}

namespace {
cudaError_t launch_true_residual(const float* X, int64_t m, int64_t n, int64_t ld, const float* y,
                                 const float* a, float* e, double* part, double* r2,
                                 cudaStream_t stream) {
  wide_dot2_rows_kernel<<<dim3((unsigned)((m + 7) / 8), WS), 256, 0, stream>>>(X, m, n, ld, a, part);
  wide_residual_rows_kernel<<<(unsigned)((m + 255) / 256), 256, 0, stream>>>(part, m, y, e, r2);
  return cudaGetLastError();
}

cudaError_t launch_sweep_cluster(const WideConfig& cfg, const CUtensorMap* tmap, WideParams p,
                                 cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(wide_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       cfg.smem_bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(wide_sweep_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  p.csize = cfg.csize;
  p.rows_box = cfg.rows_box;
  p.nstages = cfg.nstages;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(cfg.csize);
  lc.blockDim = dim3(WNT);
  lc.dynamicSmemBytes = cfg.smem_bytes;
  lc.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cfg.csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  return cudaLaunchKernelEx(&lc, wide_sweep_kernel, *tmap, p);
}
}  // namespace

cudaError_t launch_wide(const float* X, int64_t m, int64_t n, int64_t ld, const WideConfig& cfg,
                        const CUtensorMap* tmap, WideParams p, const float* y, const float* a_in,
                        int warm, float* a_tmp, cudaStream_t stream) {
  const int64_t nblk = (n + WW - 1) / WW;
  wide_gram_blocks_kernel<<<(unsigned)nblk, 256, 0, stream>>>(X, m, n, ld, p.Gb);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  wide_init_kernel<<<256, 256, 0, stream>>>(a_in, warm, p.a64, a_tmp, n);
  wide_ynorm_kernel<<<1, 256, 0, stream>>>(y, m, p.ysq);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = launch_true_residual(X, m, n, ld, y, a_tmp, p.e, p.rpart, nullptr, stream)) != cudaSuccess)
    return e;
  p.continuing = 0;
  if ((e = launch_sweep_cluster(cfg, tmap, p, stream)) != cudaSuccess) return e;
  wide_finish_kernel<<<256, 256, 0, stream>>>(p.a64, p.a_out, n);
  return cudaGetLastError();
}

cudaError_t launch_wide_confirm(const float* X, int64_t m, int64_t n, int64_t ld, const float* y,
                                const float* a, float* e, double* part, double* r2, double* sum,
                                cudaStream_t stream) {
  cudaError_t err = launch_true_residual(X, m, n, ld, y, a, e, part, r2, stream);
  if (err != cudaSuccess) return err;
  wide_sum_kernel<<<1, 256, 0, stream>>>(r2, m, sum);
  return cudaGetLastError();
}

cudaError_t launch_wide_continue(int64_t n, const WideConfig& cfg, const CUtensorMap* tmap,
                                 WideParams p, float* a_tmp, cudaStream_t stream) {
  // a64 <- the float32 coefficients the residual p.e was recomputed for
  wide_init_kernel<<<256, 256, 0, stream>>>(p.a_out, 1, p.a64, a_tmp, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  p.continuing = 1;
  if ((e = launch_sweep_cluster(cfg, tmap, p, stream)) != cudaSuccess) return e;
  wide_finish_kernel<<<256, 256, 0, stream>>>(p.a64, p.a_out, n);
  return cudaGetLastError();
}

}  // namespace hpscd
