// Column sweep of Algorithm 1 for wide systems (row-major X, m <= 4096,
// n >> m): the transposed path.
//
// In a wide system the residual e has only m entries while the sweep is a
// chain of n dependent column steps.  One thread-block cluster of WC CTAs
// walks that chain: CTA c owns rows [r0_c, r1_c) and keeps its slice of e in
// shared memory for the whole solve.  The columns are taken in the paper's
// order in blocks of W (64, or 32 when a CTA owns more than 128 rows); TMA
// re-tiles row-major X on the fly: the box {W columns, rows of this CTA} is
// the block's slab for this CTA.
//
// The steps of block b (Eq. da2 and Eq. ek1-ek inside the block) are
//     da_j = (<X_j, e> - sum_{l<j in block} G_jl da_l) / G_jj,
// a forward substitution with the block's unit lower triangle.  The set-up
// writes it as a matrix: M_b = (I + D_b^{-1} L_b)^{-1} D_b^{-1} (L_b the strict
// lower triangle of G_bb = X_b^T X_b, D_b its diagonal; a zero column gives a
// zero row), so da_b = M_b·(X_b^T e_{b-1}), where e_{b-1} is the residual
// after block b-1.  Two blocks of lookahead take the exchange of the dot
// products off the chain: each CTA forms X_{b+2}^T e_b over its rows right
// after block b's update and pushes the partials to every CTA then; they are
// used two blocks later, corrected for the one block applied in between by
// Eq. ek1-ek: X_b^T e_{b-1} = X_b^T e_{b-2} - P_b·da_{b-1} with the coupling
// P_b = X_b^T X_{b-1}.  The set-up stores N_b = M_b·P_b, so the chain is
//     da_b = M_b·q_b - N_b·da_{b-1},   q_b = sum over the CTAs of X_b^T e_{b-2},
// two W×W products per block on the dependency chain (the paper's column
// order is kept; only the association of the sums differs).  One iteration
// of a CTA, for block b:
//   1. wait (bounded) for round b of the exchange, sum its WC partials in a
//      fixed order (every CTA holds identical values);
//   2. da_b = M_b·q_b - N_b·da_{b-1}  (8 threads per row; M_b and N_b are
//      staged in shared memory by two bulk copies one block ahead);
//   3. one pass over the CTA's rows: e_r -= X_b[r]·da_b, then the partial
//      X_{b+2}^T e over the new e_r (the two slabs are both in shared memory);
//   4. the partials summed over the CTA's warps and pushed into slot (b+2) % 4
//      of every CTA of the cluster by st.async (distributed shared memory; the
//      bytes complete on the receiver's mbarrier, which the receiver arms with
//      the round's byte count, so the sender does not wait).  A CTA can run at
//      most two blocks ahead of the slowest one (it waits for round b, which
//      every CTA pushes two blocks earlier), so four slots are never
//      overwritten unread; slot s is re-armed for round b+4 right after round
//      b is consumed, which every push of round b+4 follows.
// After the last block of a sweep the cluster forms ||e|| (float64) and tests
// the stopping rule.
#include "kernels.h"

namespace hpscd {

namespace {

constexpr int WNT = 512;      // threads per CTA
constexpr int WNW = WNT / 32;
constexpr int XSLOTS = 4;     // exchange slots of the dot products (lookahead 2 + slack)

__device__ __forceinline__ void st_cluster_f64(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ void arrive_remote(uint32_t bar_cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(
                   bar_cluster_addr)
               : "memory");
}
// Asynchronous store of 16 bytes into another CTA's shared memory; the bytes
// complete (complete_tx) on that CTA's mbarrier at `bar` (both cluster addresses).
__device__ __forceinline__ void st_async_v4(uint32_t addr, float4 v, uint32_t bar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
          addr),
      "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(bar)
      : "memory");
}
// 1-D bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global into this CTA's shared memory, completing on `bar`
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
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

// ---- set-up: M_b and N_b of every column block ----
// One CTA per block b: D = X_b^T [X_b | X_{b-1}] (W x 2W: G = X_b^T X_b and the
// coupling P = X_b^T X_{b-1} to the previous block, cyclically: block 0's is
// the last block, which precedes it in the next sweep) over all m rows.  X is
// staged through shared memory 32 rows at a time, double-buffered by cp.async
// (two CTAs per SM); 16 x 16 threads each hold W/16 rows x 2W/16 columns of D
// (thread tx: columns 4·tx.. of G's half and of P's half, W/32 groups of four
// each, so that eight consecutive threads read 128 contiguous bytes), float32
// products summed in float32 over 256 rows and those sums in float32.
// Then, in shared memory: d = diag(G), H = D^{-1}·strict_lower(G),
// T = (I + H)^{-1} (column k by forward substitution in thread k),
// M = T·D^{-1}, N = M·P; M and N are stored row-major [W][W].
template <int W>
__global__ void __launch_bounds__(256, 2) wide_setup_kernel(const float* __restrict__ X, int64_t m,
                                                            int64_t n, int64_t ld, int64_t nblk,
                                                            float* __restrict__ Mb,
                                                            float* __restrict__ Nb) {
  constexpr int W2 = 2 * W;
  constexpr int TR = W / 16;    // rows of D per thread
  constexpr int TC = W2 / 16;   // columns of D per thread
  constexpr int XP = W2 + 4;    // tile pitch (16-byte rows)
  constexpr int WP = W + 4;     // pitch of the W x W matrices
  constexpr int F4 = 32 * W2 / 4 / 256;  // float4 of a tile per thread
  extern __shared__ float wsm[];
  float* xs = wsm;              // [2][32][XP]: columns 0..W-1 block b, W..2W-1 block b-1
  float* Gs = xs + 2 * 32 * XP; // [W][WP]
  float* Ps = Gs + W * WP;      // [W][WP]
  float* Ts = Ps + W * WP;      // [W][WP] T, then M
  float* dsv = Ts + W * WP;     // [W]
  const int64_t b = blockIdx.x;
  const int64_t bp = (b + nblk - 1) % nblk;
  const int64_t c0 = b * W, cp0 = bp * W;
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  const bool vec = (reinterpret_cast<uintptr_t>(X) & 15) == 0 && (ld & 3) == 0;
  // float4 q of a tile: row (tid + 256 q) / (W2 / 4), columns 4·((tid + 256 q) % (W2 / 4));
  // 16-byte cp.async where the four columns exist and X is aligned, else plain loads
  auto fetch = [&](int64_t rbase, float* dst) {
#pragma unroll
    for (int q = 0; q < F4; ++q) {
      const int i = tid + 256 * q;
      const int r = i / (W2 / 4), c = 4 * (i % (W2 / 4));
      const int64_t row = rbase + r;
      const int64_t col = c < W ? c0 + c : cp0 + (c - W);
      const float* src = X + row * ld + col;
      float* d = dst + r * XP + c;
      if (row < m && vec && col + 3 < n) {
        cp_async16(d, src);
      } else {
        d[0] = (row < m && col < n) ? __ldg(src) : 0.f;
        d[1] = (row < m && col + 1 < n) ? __ldg(src + 1) : 0.f;
        d[2] = (row < m && col + 2 < n) ? __ldg(src + 2) : 0.f;
        d[3] = (row < m && col + 3 < n) ? __ldg(src + 3) : 0.f;
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  float acc[TR][TC], acc2[TR][TC];
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < TC; ++j) { acc[i][j] = 0.f; acc2[i][j] = 0.f; }
  fetch(0, xs);
  int tiles = 0;
  int buf = 0;
  for (int64_t r0 = 0; r0 < m; r0 += 32, buf ^= 1) {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();  // tile r0 landed in buffer buf; buffer buf ^ 1 is free
    if (r0 + 32 < m) fetch(r0 + 32, xs + (buf ^ 1) * 32 * XP);  // in flight while this tile is used
    const float* xt = xs + buf * 32 * XP;
#pragma unroll 4
    for (int r = 0; r < 32; ++r) {
      float av[TR], bv[TC];
#pragma unroll
      for (int i = 0; i < TR; i += 2) {
        const float2 t = *reinterpret_cast<const float2*>(xt + r * XP + ty * TR + i);
        av[i] = t.x; av[i + 1] = t.y;
      }
#pragma unroll
      for (int j = 0; j < TC; j += 4) {
        // group j / 4 of this thread's columns: 64·(j / 4) + 4·tx (W = 64), 32·(j / 4) + 4·tx (W = 32)
        const float4 t = *reinterpret_cast<const float4*>(xt + r * XP + (j / 4) * (W2 / (TC / 4)) + 4 * tx);
        bv[j] = t.x; bv[j + 1] = t.y; bv[j + 2] = t.z; bv[j + 3] = t.w;
      }
#pragma unroll
      for (int i = 0; i < TR; ++i)
#pragma unroll
        for (int j = 0; j < TC; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    if (++tiles == 8) {
      tiles = 0;
#pragma unroll
      for (int i = 0; i < TR; ++i)
#pragma unroll
        for (int j = 0; j < TC; ++j) { acc2[i][j] += acc[i][j]; acc[i][j] = 0.f; }
    }
  }
  // this thread's columns of D (see the loads): G for columns < W, P above
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < TC; ++j) {
      const int col = (j / 4) * (W2 / (TC / 4)) + 4 * tx + (j % 4);
      float* dst = col < W ? Gs : Ps;
      dst[(ty * TR + i) * WP + (col % W)] = acc2[i][j] + acc[i][j];
    }
  __syncthreads();
  if (tid < W) dsv[tid] = Gs[tid * WP + tid];
  __syncthreads();
  // H = D^{-1}·strict_lower(G) in place of G's lower triangle (a zero row for d_i = 0)
  for (int idx = tid; idx < W * W; idx += 256) {
    const int i = idx / W, l = idx % W;
    if (l < i) {
      const float di = dsv[i];
      Gs[i * WP + l] = di > 0.f ? Gs[i * WP + l] / di : 0.f;
    }
  }
  __syncthreads();
  // T = (I + H)^{-1}, column k in thread k, held in registers:
  // T_ik = delta_ik - sum_{l<i} H_il T_lk (T_lk = 0 for l < k)
  if (tid < W) {
    const int k = tid;
    float t[W];
#pragma unroll
    for (int i = 0; i < W; ++i) {
      float acc_t = 0.f;
#pragma unroll
      for (int l = 0; l < i; ++l) acc_t = fmaf(Gs[i * WP + l], t[l], acc_t);
      t[i] = i < k ? 0.f : (i == k ? 1.f : -acc_t);
    }
#pragma unroll
    for (int i = 0; i < W; ++i) Ts[i * WP + k] = t[i];
  }
  __syncthreads();
  // M = T·D^{-1} (in place; a zero column gives a zero column of M)
  for (int idx = tid; idx < W * W; idx += 256) {
    const int i = idx / W, j = idx % W;
    const float dj = dsv[j];
    Ts[i * WP + j] = dj > 0.f ? Ts[i * WP + j] / dj : 0.f;
  }
  __syncthreads();
  // N = M·P, four consecutive columns per thread and step
  float* Mo = Mb + b * (W * W);
  float* No = Nb + b * (W * W);
  for (int idx = tid; idx < W * W / 4; idx += 256) {
    const int i = idx / (W / 4), j = 4 * (idx % (W / 4));
    float4 a4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int l = 0; l <= i; ++l) {
      const float mil = Ts[i * WP + l];
      const float4 pv = *reinterpret_cast<const float4*>(Ps + l * WP + j);
      a4.x = fmaf(mil, pv.x, a4.x);
      a4.y = fmaf(mil, pv.y, a4.y);
      a4.z = fmaf(mil, pv.z, a4.z);
      a4.w = fmaf(mil, pv.w, a4.w);
    }
    *reinterpret_cast<float4*>(No + i * W + j) = a4;
    *reinterpret_cast<float4*>(Mo + i * W + j) = *reinterpret_cast<const float4*>(Ts + i * WP + j);
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
// Shared memory of a CTA (byte offsets from a 1024-aligned base).
struct WSmem {
  int stages, es, xbuf, red, mn, qs, da, dap, nbuf, wsum, bars, total;
};
__host__ __device__ inline WSmem wide_smem_plan(int W, int rows_box, int nst) {
  WSmem s;
  int off = 0;
  auto take = [&](int bytes) {
    const int at = off;
    off += (bytes + 127) / 128 * 128;
    return at;
  };
  s.stages = take(nst * rows_box * W * 4);
  s.es = take(rows_box * 4);
  s.xbuf = take(XSLOTS * 16 * W * 4);  // [slot][source CTA][W] partial dots
  s.red = take(WNW * W * 4);           // [warp][W]
  s.mn = take(2 * W * W * 4);          // [M, N][W][W] of the block (the next one's copied in after its use)
  s.qs = take(W * 4);
  s.da = take(W * 4);
  s.dap = take(W * 4);
  s.nbuf = take(16 * 8);
  s.wsum = take(WNW * 8);
  s.bars = take((8 + XSLOTS + 2 + 1) * 8);  // full[<= 8], dot slots, norm rounds, M/N
  s.total = off + 1024;                 // alignment slack
  return s;
}

template <int W>
__global__ void __launch_bounds__(WNT, 1)
    wide_sweep_kernel(const __grid_constant__ CUtensorMap tmap, const WideParams p) {
  constexpr int CPL = W / 32;  // columns per lane in the row pass (2 or 1)
  constexpr int CPT = W / 8;   // columns per thread in the chain (8 threads per row)
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
  const WSmem L = wide_smem_plan(W, rows_box, nst);
  float* stages = reinterpret_cast<float*>(base + L.stages);
  float* es = reinterpret_cast<float*>(base + L.es);
  float* xbuf = reinterpret_cast<float*>(base + L.xbuf);
  float* red = reinterpret_cast<float*>(base + L.red);
  float* mn = reinterpret_cast<float*>(base + L.mn);
  float* qs = reinterpret_cast<float*>(base + L.qs);
  float* da_s = reinterpret_cast<float*>(base + L.da);
  float* dap_s = reinterpret_cast<float*>(base + L.dap);
  double* nbuf = reinterpret_cast<double*>(base + L.nbuf);
  double* wsum = reinterpret_cast<double*>(base + L.wsum);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + L.bars);
  uint64_t* xbar = full + 8;       // [XSLOTS] dot exchange
  uint64_t* nbar = xbar + XSLOTS;  // [2] norm exchange
  uint64_t* mnbar = nbar + 2;      // M_b, N_b of the block landed (one phase per block)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t nblk = (n + W - 1) / W;
  // optional trace (CTA 0, thread 0): for the first trace_passes blocks, the
  // global time after the round's wait and sum, after the chain, after the
  // next block's copies are issued, after the slab wait, after the row pass,
  // after the push
  uint64_t trace_k = 0;
  auto stamp = [&](int f) {
    if (p.trace && me == 0 && tid == 0 && trace_k < (uint64_t)p.trace_passes)
      p.trace[trace_k * 6 + f] = global_timer_ns();
  };

  const uint32_t round_bytes = (uint32_t)(WC * W * 4);  // every CTA's W partials
  if (tid == 0) {
    for (int s = 0; s < nst; ++s) mbar_init(&full[s], 1);
    // one arrival (this CTA's, with the round's byte count) per round
    for (int k = 0; k < XSLOTS; ++k) {
      mbar_init(&xbar[k], 1);
      mbar_arrive_expect_tx(&xbar[k], round_bytes);
    }
    for (int k = 0; k < 2; ++k) mbar_init(&nbar[k], WC);
    mbar_init(mnbar, 1);
    fence_mbar_init();
  }
  for (int r = tid; r < rows_box; r += WNT) es[r] = (r < rows) ? p.e[r0 + r] : 0.f;
  for (int c = tid; c < W; c += WNT) dap_s[c] = 0.f;
  __syncthreads();
  cluster_sync_all();  // every CTA's barriers are initialised before anyone arrives remotely

  // stage ring: sequence number k (block k % nblk of the whole solve) in stage k % nst
  const bool tma = p.use_tma != 0;
  uint64_t issued = 0, waited = 0;
  auto issue = [&](uint64_t k) {
    const int s = (int)(k % nst);
    const int64_t b = (int64_t)(k % (uint64_t)nblk);
    mbar_arrive_expect_tx(&full[s], (uint32_t)(rows_box * W * 4));
    tma_load_2d(stages + (size_t)s * rows_box * W, &tmap, &full[s], (int32_t)(b * W), (int32_t)r0);
  };
  if (tid == 0 && tma)
    while (issued < (uint64_t)nst) issue(issued++);
  // the slab of sequence k in shared memory, waited for in sequence order by
  // every warp itself (lane 0 polls the copy's mbarrier); plain loads and a CTA
  // barrier when X is not TMA-aligned.  ok turns false when a wait gave up.
  auto slab = [&](uint64_t k, bool& ok) -> const float* {
    float* st = stages + (size_t)(k % nst) * rows_box * W;
    if (tma) {
      int w = 1;
      if (lane == 0) w = mbar_wait_bounded(&full[k % nst], (uint32_t)((k / nst) & 1), p.timeout_ns) ? 1 : 0;
      w = __shfl_sync(FULL_MASK, w, 0);
      __syncwarp();
      ++waited;
      if (!w) ok = false;
    } else {
      const int64_t c0 = (int64_t)(k % (uint64_t)nblk) * W;
      for (int idx = tid; idx < rows * W; idx += WNT) {
        const int r = idx / W, c = idx % W;
        st[idx] = (c0 + c < n) ? p.X[(r0 + r) * p.ld + c0 + c] : 0.f;
      }
      __syncthreads();
    }
    return st;
  };

  int err = DEV_OK;
  int status = HPSCD_ERR_NOT_CONVERGED;
  const double ynorm = sqrt(*p.ysq);
  double r_prev = 0.0;
  int64_t sweeps = 0;
  uint64_t nround = 0;  // norm exchange rounds
  uint64_t pushed = 0;  // dot exchange rounds pushed by this CTA (every CTA pushes the same)

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
      arrive_remote(mapa_u32(smem_u32(&nbar[q]), (uint32_t)tid));
    }
    const bool ok = wait_cluster_bounded(&nbar[q], (uint32_t)((nround / 2) & 1), p.timeout_ns);
    ++nround;
    double t = 0.0;
    for (int c = 0; c < WC; ++c) t += nbuf[c];
    *out = t;
    __syncthreads();  // nbuf is read before the next round overwrites it
    return __syncthreads_or(ok ? 0 : 1) == 0;
  };

  // this CTA's partials (the warp partials of the row pass, in red, complete
  // after a CTA barrier), pushed as round `round` into every CTA of the
  // cluster: thread j < W/4 of warp 0 sums float4 j over the warps and stores
  // it into every CTA by st.async (no barrier: red is next written after two)
  auto push_round = [&](uint64_t round) {
    constexpr int Q = W / 4;
    if (tid < Q) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int w = 0; w < WNW; ++w) {
        const float4 t = *reinterpret_cast<const float4*>(red + w * W + 4 * tid);
        v.x += t.x; v.y += t.y; v.z += t.z; v.w += t.w;
      }
      const int slot = (int)(round % XSLOTS);
      const uint32_t src = smem_u32(&xbuf[(slot * 16 + me) * W + 4 * tid]);
      const uint32_t bar = smem_u32(&xbar[slot]);
      for (int dstc = 0; dstc < WC; ++dstc)
        st_async_v4(mapa_u32(src, (uint32_t)dstc), v, mapa_u32(bar, (uint32_t)dstc));
    }
    ++pushed;
  };

  // dots only (no update): the prologue's rounds 0 and 1 against the initial e
  auto dots_only = [&](const float* st) {
    __syncthreads();  // the previous round's push has read red
    float pd[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) pd[c] = 0.f;
    for (int r = warp; r < rows; r += WNW) {
      const float er = es[r];
#pragma unroll
      for (int c = 0; c < CPL; ++c) pd[c] = fmaf(st[r * W + CPL * lane + c], er, pd[c]);
    }
#pragma unroll
    for (int c = 0; c < CPL; ++c) red[warp * W + CPL * lane + c] = pd[c];
    __syncthreads();
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

  // chain operands: thread (row ci = tid / 8, part cj = tid % 8) takes columns
  // [cj·CPT, (cj+1)·CPT) of row ci of M_b and N_b; both matrices of the next
  // block are copied into the buffer as soon as this block's products are done
  // (one buffer: the space goes to one more TMA stage)
  const int ci = tid / 8, cj = tid % 8;
  const bool chain_thread = tid < 8 * W;
  // M_b and N_b by two bulk copies issued by thread 0 (one instruction each,
  // not thousands of per-thread 16-byte copies in the memory pipe)
  uint64_t mn_issued = 0;  // M/N copies issued (thread 0)
  auto load_mn = [&](int64_t b, int buf) {
    (void)buf;
    if (tid == 0) {
      fence_proxy_async_smem();  // the buffer's last reads (the previous block's products) come first
      mbar_arrive_expect_tx(mnbar, (uint32_t)(2 * W * W * 4));
      bulk_g2s(mn, p.Mb + b * (W * W), (uint32_t)(W * W * 4), mnbar);
      bulk_g2s(mn + W * W, p.Nb + b * (W * W), (uint32_t)(W * W * 4), mnbar);
      ++mn_issued;
    }
  };

  if (status == -1 && err == DEV_OK) {
    // prologue: rounds 0 and 1, the dots of sequences 0 and 1 against the initial e
    bool ok = true;
    for (uint64_t k = 0; k < 2 && ok; ++k) {
      const float* st = slab(k, ok);
      if (__syncthreads_or(ok ? 0 : 1)) { ok = false; break; }  // the same decision in every warp
      dots_only(st);
      push_round(k);
    }
    if (!ok) err = DEV_TIMEOUT_COPY;
    load_mn(0, 0);
  }

  uint64_t kseq = 0;  // block sequence number (all sweeps)
  for (int64_t sw = 1; status == -1 && err == DEV_OK; ++sw) {
    for (int64_t b = 0; b < nblk; ++b, ++kseq) {
      // 1. round kseq: the partials of block b against e_{k-2}, summed in CTA
      //    order by the warps of threads < W, which wait for the round themselves
      const int slot = (int)(kseq % XSLOTS);
      int wok = 1;
      if (warp * 32 < W) {
        if (lane == 0) wok = wait_cluster_bounded(&xbar[slot], (uint32_t)((kseq / XSLOTS) & 1), p.timeout_ns) ? 1 : 0;
        wok = __shfl_sync(FULL_MASK, wok, 0);
        __syncwarp();
        if (wok && tid < W) {
          // loads issued together (WC <= 16), summed in CTA order
          float v[16];
#pragma unroll
          for (int c = 0; c < 16; ++c) v[c] = c < WC ? xbuf[(slot * 16 + c) * W + tid] : 0.f;
          float g = 0.f;
#pragma unroll
          for (int c = 0; c < 16; ++c) g += v[c];
          qs[tid] = g;
        }
      }
      // this block's M_b and N_b (phase kseq of mnbar)
      if (wok && !mbar_wait_bounded(mnbar, (uint32_t)(kseq & 1), p.timeout_ns)) wok = 0;
      if (__syncthreads_or(wok ? 0 : 1)) { err = DEV_TIMEOUT_BARRIER; break; }
      // the slot is free: arm it for round kseq + 4 (every push of that round follows)
      if (tid == 0) mbar_arrive_expect_tx(&xbar[slot], round_bytes);
      stamp(0);
      // 2. the block's steps: da_b = M_b q_b - N_b da_{b-1}
      const int cur = 0;  // one M/N buffer
      if (chain_thread) {
        const float* mrow = mn + (size_t)cur * 2 * W * W + ci * W + cj * CPT;
        const float* nrow = mrow + W * W;
        float acc = 0.f;
#pragma unroll
        for (int c = 0; c < CPT; c += 4) {
          const float4 mv = *reinterpret_cast<const float4*>(mrow + c);
          const float4 nv = *reinterpret_cast<const float4*>(nrow + c);
          const float* q = qs + cj * CPT + c;
          const float* d = dap_s + cj * CPT + c;
          acc = fmaf(mv.x, q[0], acc);
          acc = fmaf(mv.y, q[1], acc);
          acc = fmaf(mv.z, q[2], acc);
          acc = fmaf(mv.w, q[3], acc);
          acc = fmaf(-nv.x, d[0], acc);
          acc = fmaf(-nv.y, d[1], acc);
          acc = fmaf(-nv.z, d[2], acc);
          acc = fmaf(-nv.w, d[3], acc);
        }
        acc += __shfl_xor_sync(FULL_MASK, acc, 1);
        acc += __shfl_xor_sync(FULL_MASK, acc, 2);
        acc += __shfl_xor_sync(FULL_MASK, acc, 4);
        if (cj == 0) da_s[ci] = acc;
      }
      __syncthreads();
      stamp(1);
      load_mn(b + 1 < nblk ? b + 1 : 0, 0);  // the next block's into the buffer just used, landing before its products
      if (me == 0 && tid < W && b * W + tid < n) p.dsw[b * W + tid] = da_s[tid];
      if (tid < W) dap_s[tid] = da_s[tid];
      stamp(2);
      // 3. the row pass: e_r -= X_b[r]·da_b, then the partial X_{b+2}^T e
      bool ok = true;
      const float* sk = stages + (size_t)(kseq % nst) * rows_box * W;  // waited for two blocks ago
      const float* s2 = slab(kseq + 2, ok);  // a failed wait is acted on after the pass
      stamp(3);
      {
        float dl[CPL], pd[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) { dl[c] = da_s[CPL * lane + c]; pd[c] = 0.f; }
        for (int rb = warp; rb < rows; rb += 8 * WNW) {
          // up to 8 rows of this warp at once: independent shuffle reductions
          float u[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int r = rb + i * WNW;
            float v = 0.f;
            if (r < rows) {
              if constexpr (CPL == 2) {
                const float2 x2 = *reinterpret_cast<const float2*>(sk + r * W + 2 * lane);
                v = fmaf(x2.x, dl[0], x2.y * dl[CPL - 1]);
              } else {
                v = sk[r * W + lane] * dl[0];
              }
            }
            u[i] = v;
          }
#pragma unroll
          for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int i = 0; i < 8; ++i) u[i] += __shfl_xor_sync(FULL_MASK, u[i], off);
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int r = rb + i * WNW;
            if (r < rows) {
              const float er = es[r] - u[i];
              if constexpr (CPL == 2) {
                const float2 y2 = *reinterpret_cast<const float2*>(s2 + r * W + 2 * lane);
                pd[0] = fmaf(y2.x, er, pd[0]);
                pd[CPL - 1] = fmaf(y2.y, er, pd[CPL - 1]);
              } else {
                pd[0] = fmaf(s2[r * W + lane], er, pd[0]);
              }
              __syncwarp();
              if (lane == 0) es[r] = er;
            }
          }
        }
#pragma unroll
        for (int c = 0; c < CPL; ++c) red[warp * W + CPL * lane + c] = pd[c];
      }
      // e, red complete; slab kseq is free
      if (__syncthreads_or(ok ? 0 : 1)) { err = DEV_TIMEOUT_COPY; break; }
      stamp(4);
      if (tid == 0 && tma) {
        fence_proxy_async_smem();
        issue(issued++);  // sequence kseq + nst into the stage just released
      }
      // 4. push round kseq + 2
      push_round(kseq + 2);
      stamp(5);
      ++trace_k;
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
  // the M/N copy issued last lands before the CTA may retire
  if (tid == 0 && mn_issued > 0)
    mbar_wait_bounded(mnbar, (uint32_t)((mn_issued - 1) & 1), p.timeout_ns);
  if (tid == 0 && tma) {
    for (uint64_t k = waited; k < issued; ++k)
      if (!mbar_wait_bounded(&full[k % nst], (uint32_t)((k / nst) & 1), p.timeout_ns)) {
        if (err == DEV_OK) err = DEV_TIMEOUT_COPY;
        break;
      }
  }
  // the rounds pushed into this CTA but not consumed: their bytes land before
  // the CTA may exit (bounded; in an error exit some never complete)
  if (tid == 0 && err == DEV_OK)
    for (uint64_t r = kseq; r < pushed; ++r)
      if (!wait_cluster_bounded(&xbar[r % XSLOTS], (uint32_t)((r / XSLOTS) & 1), p.timeout_ns)) {
        err = DEV_TIMEOUT_BARRIER;
        break;
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

namespace {
int wide_setup_smem(int W) { return (2 * 32 * (2 * W + 4) + 3 * W * (W + 4) + W) * 4; }
}  // namespace

bool wide_config(int64_t m, int max_smem, WideConfig* cfg) {
  if (m < 1 || m > 4096) return false;
  int csize = 16;
  while (csize > 1 && (m + csize - 1) / csize < 8) csize /= 2;  // small m: fewer CTAs
  cfg->csize = csize;
  cfg->rows_box = (int)((m + csize - 1) / csize);
  if (cfg->rows_box > 256) return false;
  // slabs of blocks b, b+1, b+2 stay resident with at least one copy ahead
  cfg->W = cfg->rows_box <= 128 ? 64 : 32;
  int nst = 6;
  while (nst >= 4 && wide_smem_plan(cfg->W, cfg->rows_box, nst).total > max_smem) --nst;
  if (nst < 4) return false;
  cfg->nstages = nst;
  cfg->smem_bytes = wide_smem_plan(cfg->W, cfg->rows_box, nst).total;
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

template <int W>
cudaError_t launch_setup_w(const float* X, int64_t m, int64_t n, int64_t ld, float* Mb, float* Nb,
                           cudaStream_t stream) {
  const int64_t nblk = (n + W - 1) / W;
  const int smem = wide_setup_smem(W);
  cudaError_t e = cudaFuncSetAttribute(wide_setup_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  wide_setup_kernel<W><<<(unsigned)nblk, 256, smem, stream>>>(X, m, n, ld, nblk, Mb, Nb);
  return cudaGetLastError();
}

template <int W>
cudaError_t launch_cluster_w(const WideConfig& cfg, const CUtensorMap* tmap, const WideParams& p,
                             cudaStream_t stream) {
  auto kern = wide_sweep_kernel<W>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, cfg.smem_bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
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
  return cudaLaunchKernelEx(&lc, kern, *tmap, p);
}

cudaError_t launch_sweep_cluster(const WideConfig& cfg, const CUtensorMap* tmap, WideParams p,
                                 cudaStream_t stream) {
  p.csize = cfg.csize;
  p.rows_box = cfg.rows_box;
  p.nstages = cfg.nstages;
  return cfg.W == 64 ? launch_cluster_w<64>(cfg, tmap, p, stream)
                     : launch_cluster_w<32>(cfg, tmap, p, stream);
}
}  // namespace

cudaError_t launch_wide(const float* X, int64_t m, int64_t n, int64_t ld, const WideConfig& cfg,
                        const CUtensorMap* tmap, WideParams p, const float* y, const float* a_in,
                        int warm, float* a_tmp, cudaStream_t stream) {
  cudaError_t e = cfg.W == 64 ? launch_setup_w<64>(X, m, n, ld, p.Mb, p.Nb, stream)
                              : launch_setup_w<32>(X, m, n, ld, p.Mb, p.Nb, stream);
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
