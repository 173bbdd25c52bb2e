// Batched column sweep of Algorithm 1: thousands of independent, uneven
// column-major systems (m rows, n <= 256 columns each) swept to their
// stopping rule in ONE persistent launch.
//
// Work distribution.  The grid holds as many thread-block clusters of K CTAs
// as fit on the GPU at once (K = CTAs per system, picked by the autotuner).
// Each cluster pops the next system from an atomic queue (systems ordered by
// decreasing m·n, so the longest jobs start first) and solves it completely:
// CTA k of the cluster owns a contiguous slice of the system's rows and keeps
// that slice of the residual e in shared memory for the whole solve.
//
// Per system (the same restatement of a sweep as the tall kernel, Eq. ek1-ek
// and Eq. da2): with g = X^T e at the start of a sweep and G = X^T X,
//     da_j = (g_j - sum_{l<j} G_jl da_l) / G_jj,   j = 1..n in order,
// is exactly the sweep's n column steps.  Writing d = diag(G) and
// G~ = D^{-1} G (each row divided by its denominator, the ⊘ step of the
// paper applied once to the couplings), the sweep is
//     r   = g ⊘ d                       (elementwise, Eq. da2's division)
//     da_j = r_j - sum_{l<j} G~_jl da_l  (forward substitution, no division
//                                         on the dependency chain)
// followed by e <- e - X·da and a <- a + da.
//   set-up:  the cluster forms G (CUDA cores, X staged through shared memory,
//            each CTA over its rows; partials summed in rank order), d and G~;
//   pass p:  one read of X forms e_out = e_in - X·v (v = da_p; a warm start's
//            a_0 on pass 0) and h = X^T e_in, plus ||e_out||^2 in float64;
//            the CTAs of the cluster exchange their partial h and norms
//            through distributed shared memory (one cluster barrier) and sum
//            them in rank order, so every CTA holds bitwise identical values;
//            hist[p] = ||e_p|| / ||y||, the stopping test, then
//            r = h ⊘ d - G~·v (= (X^T e_p) ⊘ d) and the forward substitution.
// There are no spin waits: the only waits are CTA and cluster barriers, which
// every CTA of a cluster reaches in the same order (the stopping decision is
// taken on identical values in all of them).
#include "kernels.h"

namespace hpscd {

namespace {

constexpr int BNT = 512;            // threads per CTA
constexpr int BNW = BNT / 32;       // warps
constexpr int BMAXN = 256;          // columns of a batched system (max)
constexpr int BLDG = 256;           // leading dimension of the Gram slots
constexpr int GR = 32;              // rows per staged Gram panel
constexpr int GPITCH = GR + 1;      // padded pitch of a staged column (conflict-free reads)
constexpr int DIAGP = 32 * 31 / 2;  // strictly lower entries of a 32x32 block
constexpr int REDF = 8192;          // floats of one row-sum reduction buffer

// Shared-memory plan of one CTA (byte offsets from a 128-byte aligned base).
struct BSmem {
  int e, uni, hred, hpart, h64, rvec, da, dd, v, a64, diag, scal, total;
};

__host__ __device__ inline BSmem bsmem_plan(int ecap) {
  BSmem s;
  int off = 0;
  auto take = [&](int bytes) {
    const int at = off;
    off += (bytes + 127) / 128 * 128;
    return at;
  };
  s.e = take(ecap * 4);
  const int gstage = 2 * BMAXN * GPITCH * 4;  // Gram staging (double buffer)
  const int red = 2 * REDF * 4;               // row-sum reduction (double buffer)
  s.uni = take(gstage > red ? gstage : red);
  s.hred = take(BNW * BMAXN * 8);   // float64 row-group sums of h
  s.hpart = take(2 * BMAXN * 8);    // float64 CTA partials of h (exchanged in the cluster)
  s.h64 = take(BMAXN * 8);          // h of the pass, summed over the cluster
  s.rvec = take(BMAXN * 4);
  s.da = take(BMAXN * 4);
  s.dd = take(BMAXN * 4);
  s.v = take(BMAXN * 4);
  s.a64 = take(BMAXN * 8);
  s.diag = take((BMAXN / 32) * DIAGP * 4);
  s.scal = take(64 * 8);
  s.total = off + 128;  // alignment slack
  return s;
}

__device__ __forceinline__ int pow2floor(int x) {
  int p = 1;
  while (p * 2 <= x) p *= 2;
  return p;
}

// Block reduction of a double over all BNT threads (result in every thread).
__device__ __forceinline__ double block_sum_f64(double v, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(FULL_MASK, v, off);
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < BNW; ++w) s += scratch[w];  // fixed order
  return s;
}

// ---- set-up: partial Gram of this CTA's rows -------------------------------
// Lower 32x32 blocks (BI >= BJ) of X_rows^T X_rows, one block per warp and
// round; in a round with fewer than 16 blocks, S warps share a block and each
// takes every S-th staged panel (their partials are summed in slice order).
// Lane (i, j) of a warp (i = lane / 8, j = lane % 8) owns rows BI*32 + i*8..+7
// and columns BJ*32 + j*4..+3 of its block.  Result: Gp (lower blocks only,
// leading dimension BLDG).
__device__ void gram_partial(const float* __restrict__ X, int64_t ld, int64_t r0, int mloc, int n,
                             float* stage, float* Gp) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nb = (n + 31) / 32;
  const int NB = nb * (nb + 1) / 2;
  const int li = lane >> 3, lj = lane & 7;
  const int npanel = (mloc + GR - 1) / GR;
  for (int b0 = 0; b0 < NB; b0 += BNW) {
    const int q = min(BNW, NB - b0);
    const int S = q >= BNW ? 1 : pow2floor(BNW / q);
    const int myb = warp / S, slice = warp % S;
    const bool active = myb < q;
    int BI = 0, BJ = 0;
    if (active) {
      int t = b0 + myb;  // lower-triangular block index -> (BI, BJ), row-major over BI
      while (t > BI) { t -= BI + 1; ++BI; }
      BJ = t;
    }
    float acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    for (int pn = 0; pn < npanel; ++pn) {
      float* buf = stage + (pn & 1) * (BMAXN * GPITCH);
      const int rbase = pn * GR;
      // stage rows [rbase, rbase+GR) of every column (zero past mloc and n)
      for (int idx = tid; idx < nb * 32 * GR; idx += BNT) {
        const int c = idx / GR, r = idx % GR;
        float v = 0.f;
        if (c < n && rbase + r < mloc) v = __ldg(X + (int64_t)c * ld + r0 + rbase + r);
        buf[c * GPITCH + r] = v;
      }
      __syncthreads();
      if (active && (pn % S) == slice) {
        const float* pa = buf + (BI * 32 + li * 8) * GPITCH;
        const float* pb = buf + (BJ * 32 + lj * 4) * GPITCH;
#pragma unroll 4
        for (int r = 0; r < GR; ++r) {
          float av[8], bv[4];
#pragma unroll
          for (int a = 0; a < 8; ++a) av[a] = pa[a * GPITCH + r];
#pragma unroll
          for (int b = 0; b < 4; ++b) bv[b] = pb[b * GPITCH + r];
#pragma unroll
          for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
        }
      }
      // the next panel is staged into the other buffer; the one after it
      // overwrites this one only after the next barrier
    }
    __syncthreads();
    // slices of a block -> shared memory, summed in slice order by slice 0
    float* red = stage;  // [BNW][1024]
    if (S > 1) {
      if (active) {
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) red[warp * 1024 + (li * 8 + a) * 32 + lj * 4 + b] = acc[a][b];
      }
      __syncthreads();
      if (active && slice == 0) {
        for (int s = 1; s < S; ++s) {
#pragma unroll
          for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
              acc[a][b] += red[(warp + s) * 1024 + (li * 8 + a) * 32 + lj * 4 + b];
        }
      }
    }
    if (active && slice == 0) {
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        float4* dst = reinterpret_cast<float4*>(Gp + (int64_t)(BI * 32 + li * 8 + a) * BLDG + BJ * 32 + lj * 4);
        *dst = make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
      }
    }
    __syncthreads();
  }
}

// ---- one streaming pass over this CTA's rows --------------------------------
// CPW columns per warp; RPL = 16 / CPW row blocks of 128 rows per lane step,
// so every lane has 16 independent 16-byte loads in flight.  NWC warps split
// the columns, NWR = 16 / NWC warps split the rows of a panel.
template <int CPW>
__device__ void stream_pass(const float* __restrict__ X, int64_t ld, int64_t r0, int mloc, int n,
                            int nwc, int vec, float* e_s, const float* vsm, float* red,
                            double* hred, double& nrm_out) {
  constexpr int RPL = 16 / CPW;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nwr = BNW / nwc;
  const int wc = warp % nwc, wr = warp / nwc;
  const int ph = nwr * RPL * 128;
  float h[CPW];
#pragma unroll
  for (int j = 0; j < CPW; ++j) h[j] = 0.f;
  const float* vw = vsm + wc * CPW;  // v of this warp's columns (zero past n)
  double nrm = 0.0;
  int pi = 0;
  for (int pbase = 0; pbase < mloc; pbase += ph, ++pi) {
    float* rb_buf = red + (pi & 1) * REDF;
    float xv[RPL][CPW][4];
    float ein[RPL][4];
#pragma unroll
    for (int rb = 0; rb < RPL; ++rb) {
      const int lrow = pbase + (wr * RPL + rb) * 128 + 4 * lane;
#pragma unroll
      for (int q = 0; q < 4; ++q) ein[rb][q] = (lrow + q < mloc) ? e_s[lrow + q] : 0.f;
#pragma unroll
      for (int j = 0; j < CPW; ++j) {
        const int col = wc * CPW + j;
        const float* src = X + (int64_t)col * ld + r0 + lrow;
        if (col < n && vec && lrow + 3 < mloc) {
          const float4 t = __ldg(reinterpret_cast<const float4*>(src));
          xv[rb][j][0] = t.x; xv[rb][j][1] = t.y; xv[rb][j][2] = t.z; xv[rb][j][3] = t.w;
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            xv[rb][j][q] = (col < n && lrow + q < mloc) ? __ldg(src + q) : 0.f;
        }
      }
    }
#pragma unroll
    for (int rb = 0; rb < RPL; ++rb) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int j = 0; j < CPW; ++j) {
        const float vj = vw[j];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          h[j] = fmaf(xv[rb][j][q], ein[rb][q], h[j]);
          acc[q] = fmaf(xv[rb][j][q], vj, acc[q]);
        }
      }
      float* dst = rb_buf + wc * ph + (wr * RPL + rb) * 128 + 4 * lane;
      *reinterpret_cast<float4*>(dst) = make_float4(acc[0], acc[1], acc[2], acc[3]);
    }
    __syncthreads();
    for (int t = tid; t < ph; t += BNT) {
      const int lrow = pbase + t;
      if (lrow < mloc) {
        float s = 0.f;
        for (int w = 0; w < nwc; ++w) s += rb_buf[w * ph + t];
        const float e_new = e_s[lrow] - s;
        e_s[lrow] = e_new;
        nrm = fma((double)e_new, (double)e_new, nrm);
      }
    }
  }
  // lane partials of h -> one value per (row group, column), summed in float64
#pragma unroll
  for (int j = 0; j < CPW; ++j) {
    float sf = h[j];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sf += __shfl_xor_sync(FULL_MASK, sf, off);
    const double s = (double)sf;
    const int col = wc * CPW + j;
    if (lane == 0 && col < n) hred[wr * BMAXN + col] = s;
  }
  nrm_out = nrm;
}

// Loads that the compiler may not hoist out of the sweep loop: the confirmation
// step reads these descriptor fields only when it runs, so they do not stay
// live (in registers) across the streaming passes.
__device__ __forceinline__ const float* ld_volatile_ptr(const float* const* addr) {
  const float* v;
  asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(addr));
  return v;
}
__device__ __forceinline__ int ld_volatile_s32(const int32_t* addr) {
  int v;
  asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(addr));
  return v;
}

// The residual of the coefficients ahi (shared, float32) on this CTA's rows:
// e = y - X·ahi with Dot2 accumulation (Ogita, Rump, Oishi 2005), one thread
// per row; returns this thread's share of ||y - X·ahi||^2 in float64, taken
// before e is rounded to float32.
__device__ double true_residual_rows(const float* __restrict__ X, int64_t ld, int64_t r0, int mloc,
                                     int n, const float* __restrict__ y, const float* ahi,
                                     float* e_s) {
  double t2 = 0.0;
  for (int i = threadIdx.x; i < mloc; i += BNT) {
    float s = 0.f, c = 0.f;
    for (int j = 0; j < n; ++j) {
      const float xv = __ldg(X + (int64_t)j * ld + r0 + i), av = ahi[j];
      const float pr = xv * av, pe = fmaf(xv, av, -pr);
      const float t = s + pr, z = t - s;
      c += ((s - (t - z)) + (pr - z)) + pe;
      s = t;
    }
    const double ed = ((double)__ldg(y + r0 + i) - (double)s) - (double)c;
    e_s[i] = (float)ed;
    t2 = fma(ed, ed, t2);
  }
  return t2;
}

// Forward substitution da_j = r_j - sum_{l<j} G~_jl da_l in blocks of 32
// columns: warp 0 solves each diagonal block as a product with its inverse
// (staged in diag_s by invert_diag_blocks, once per system); every thread
// t >= 32 owns row t and applies each finished block to it.  r is overwritten.
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

// stage: shared scratch of BMAXN rows × SEGP floats, free between passes; each
// thread below the block copies its row's segment of the block there with
// cp.async before the walk (no registers held), so the copy overlaps the walk.
constexpr int SEGP = 36;  // row pitch of the staged segments (16-byte rows, conflict-free float4 reads)
static_assert(BMAXN * SEGP <= 2 * REDF, "the staged segments fit the pass scratch");
// diag_s holds, per 32-column block b, the strictly lower triangle L_b of the
// unit lower triangular diagonal block I + L_b of G~ (packed by rows); it is
// replaced in place by the strictly lower triangle of M_b = (I + L_b)^{-1}, so
// that the substitution of a block is a product with M_b.  Warp w takes blocks
// w, w + BNW, ...; lane j forms column j: M_ij = -sum_{k<i} L_ik M_kj, i > j.
__device__ void invert_diag_blocks(float* diag_s, int nb) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int b = warp; b < nb; b += BNW) {
    float* blk = diag_s + b * DIAGP;
    float mcol[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      const float* li = blk + (i * (i - 1)) / 2;
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < i; ++k) s = fmaf(li[k], mcol[k], s);  // mcol[k] = 0 for k < lane
      mcol[i] = i < lane ? 0.f : (i == lane ? 1.f : -s);
    }
    __syncwarp();
#pragma unroll
    for (int i = 1; i < 32; ++i)
      if (i > lane) blk[(i * (i - 1)) / 2 + lane] = mcol[i];
    __syncwarp();
  }
}

__device__ void forward_sub_scaled(const float* __restrict__ Gt, int n, float* r, float* da,
                                   const float* diag_s, float* stage) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nb = (n + 31) / 32;
  for (int b = 0; b < nb; ++b) {
    const int b0 = 32 * b;
    const bool mine = tid >= b0 + 32 && tid < n;
    if (mine) {
      const float* src = Gt + (int64_t)tid * BLDG + b0;
      float* dst = stage + tid * SEGP;
#pragma unroll
      for (int q = 0; q < 8; ++q) cp_async16(dst + 4 * q, src + 4 * q);
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    if (warp == 0) {
      const int i = b0 + lane;
      float seg[32];
      const float* dl = diag_s + b * DIAGP + (lane * (lane - 1)) / 2;
#pragma unroll
      for (int k = 0; k < 32; ++k) seg[k] = (k < lane) ? dl[k] : 0.f;
      // diag_s holds the strictly lower part of M_b = (I + L_b)^{-1}: the block's
      // da = M_b r, 32 independent shuffles
      const float ri = (i < n) ? r[i] : 0.f;
      float acc[4] = {ri, 0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < 32; ++k) acc[k & 3] = fmaf(seg[k], __shfl_sync(FULL_MASK, ri, k), acc[k & 3]);
      da[i] = (i < n) ? (acc[0] + acc[1]) + (acc[2] + acc[3]) : 0.f;
    }
    __syncthreads();
    if (mine) {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      const float4* g4 = reinterpret_cast<const float4*>(stage + tid * SEGP);
      float acc = 0.f;
#pragma unroll
      for (int k4 = 0; k4 < 8; ++k4) {
        const float4 g = g4[k4];
        acc = fmaf(g.x, da[b0 + 4 * k4], acc);
        acc = fmaf(g.y, da[b0 + 4 * k4 + 1], acc);
        acc = fmaf(g.z, da[b0 + 4 * k4 + 2], acc);
        acc = fmaf(g.w, da[b0 + 4 * k4 + 3], acc);
      }
      r[tid] -= acc;
    }
    __syncthreads();
  }
}

template <int K>
__global__ void __launch_bounds__(BNT, 1) batched_sweep_kernel(const BatchParams p) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const BSmem L = bsmem_plan(p.ecap);
  float* e_s = reinterpret_cast<float*>(base + L.e);
  float* uni = reinterpret_cast<float*>(base + L.uni);
  double* hred = reinterpret_cast<double*>(base + L.hred);
  double* hpart = reinterpret_cast<double*>(base + L.hpart);  // [2][BMAXN]
  double* h64 = reinterpret_cast<double*>(base + L.h64);
  float* rvec = reinterpret_cast<float*>(base + L.rvec);
  float* da_s = reinterpret_cast<float*>(base + L.da);
  float* dd_s = reinterpret_cast<float*>(base + L.dd);
  float* vsm = reinterpret_cast<float*>(base + L.v);
  double* a64_s = reinterpret_cast<double*>(base + L.a64);
  float* diag_s = reinterpret_cast<float*>(base + L.diag);
  double* scal = reinterpret_cast<double*>(base + L.scal);  // [0..15] block sums, [16..19] exchange
  int* sys_s = reinterpret_cast<int*>(scal + 60);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = (K > 1) ? cluster_ctarank() : 0u;
  const int cl = blockIdx.x / K;  // cluster index
  float* Gp = p.gpart + (size_t)blockIdx.x * BLDG * BLDG;
  float* Gt = p.gfinal + (size_t)cl * BLDG * BLDG;

  auto csync = [&]() {
    if constexpr (K > 1) {
      __threadfence();
      cluster_sync_all();
    } else {
      __syncthreads();
    }
  };

  for (;;) {
    if (rank == 0 && tid == 0) {
      const int q = atomicAdd(p.queue, 1);
      sys_s[0] = q < p.count ? p.order[q] : -1;
    }
    csync();
    int sidx;
    if constexpr (K > 1) sidx = ld_cluster_s32(mapa_u32(smem_u32(sys_s), 0));
    else sidx = sys_s[0];
    if (sidx < 0) break;
    const hpscd_sys sd = p.sys[sidx];
    const float* X = static_cast<const float*>(sd.X);
    const int64_t m = sd.m, ld = sd.ld;
    const int n = (int)sd.n;
    // rows of this CTA: slices of 128-row multiples, so 16-byte alignment holds
    const int64_t blocks128 = (m + 127) / 128;
    const int64_t r0 = (blocks128 * rank / K) * 128;
    const int64_t r1 = rank + 1 == K ? m : (blocks128 * (rank + 1) / K) * 128;
    const int64_t r1c = r1 < m ? r1 : m;
    const int mloc = r1c > r0 ? (int)(r1c - r0) : 0;
    const int vec = ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && (ld % 4 == 0);

    // ---- set-up: G, d and G~ = D^{-1} G ----
    gram_partial(X, ld, r0, mloc, n, uni, Gp);
    csync();
    // d = diag(G) (every CTA, rank order)
    for (int c = tid; c < BMAXN; c += BNT) {
      float s = 0.f;
      if (c < n) {
        for (int k = 0; k < K; ++k)
          s += __ldcg(p.gpart + ((size_t)(cl * K + k) * BLDG + c) * BLDG + c);
      }
      dd_s[c] = s;
    }
    __syncthreads();
    // rows [j0, j1) of G~ by this CTA: lower entries summed over the cluster's
    // partials, divided by the row's d; the mirrored entry by the column's d
    {
      const int j0 = (int)((int64_t)n * rank / K), j1 = (int)((int64_t)n * (rank + 1) / K);
      for (int j = j0 + warp; j < j1; j += BNW) {
        const float dj = dd_s[j];
        for (int l = lane; l <= j; l += 32) {
          float s = 0.f;
          for (int k = 0; k < K; ++k)
            s += __ldcg(p.gpart + ((size_t)(cl * K + k) * BLDG + j) * BLDG + l);
          const float dl = dd_s[l];
          if (l == j) {
            Gt[(size_t)j * BLDG + j] = dj > 0.f ? 1.f : 0.f;
          } else {
            Gt[(size_t)j * BLDG + l] = dj > 0.f ? s / dj : 0.f;
            Gt[(size_t)l * BLDG + j] = dl > 0.f ? s / dl : 0.f;
          }
        }
        // columns n..32·ceil(n/32)-1 of the row are read (times da = 0) by the substitution
        for (int l = n + lane; l < ((n + 31) / 32) * 32; l += 32) Gt[(size_t)j * BLDG + l] = 0.f;
      }
    }
    csync();
    // diagonal blocks of G~ (strictly lower, packed) into shared memory
    for (int idx = tid; idx < ((n + 31) / 32) * DIAGP; idx += BNT) {
      const int b = idx / DIAGP, qq = idx % DIAGP;
      int i = 1;
      while ((i * (i + 1)) / 2 <= qq) ++i;
      const int k = qq - (i * (i - 1)) / 2;
      const int row = 32 * b + i, col = 32 * b + k;
      diag_s[idx] = (row < n) ? __ldcg(Gt + (size_t)row * BLDG + col) : 0.f;
    }
    __syncthreads();
    invert_diag_blocks(diag_s, (n + 31) / 32);
    // residual slice e = y, coefficients, v
    double ysq = 0.0;
    for (int t = tid; t < p.ecap; t += BNT) {
      float v = 0.f;
      if (t < mloc) {
        v = __ldg(sd.y + r0 + t);
        ysq = fma((double)v, (double)v, ysq);
      }
      e_s[t] = v;
    }
    for (int c = tid; c < BMAXN; c += BNT) {
      const float a0 = (c < n && sd.a_is_guess) ? sd.a[c] : 0.f;
      a64_s[c] = (double)a0;
      vsm[c] = a0;
      da_s[c] = 0.f;
    }
    ysq = block_sum_f64(ysq, scal);
    __syncthreads();

    // column split of the streaming pass
    // columns per warp: the narrowest that covers n with the CTA's warps, or wider
    const int cpw0 = n <= 64 ? 4 : (n <= 128 ? 8 : 16);
    const int cpw = p.panel >= 2 ? 16 : (cpw0 << p.panel) > 16 ? 16 : (cpw0 << p.panel);
    int nwc = (n + cpw - 1) / cpw;
    nwc = nwc < 1 ? 1 : nwc;
    { int pw = 1; while (pw < nwc) pw *= 2; nwc = pw; }
    if (nwc > BNW) nwc = BNW;

    double ynorm = 0.0, r_prev = 0.0;
    int status = HPSCD_ERR_NOT_CONVERGED;
    int64_t pass = 0;
    int refills = 0;       // passes that only re-formed h from a recomputed e (no step, no test)
    int confirms = 0;      // true-residual passes made
    bool refill = false;   // this pass is such a refill
    for (pass = 0;; ++pass) {
      const int64_t sw = pass - refills;  // sweeps reflected in e
      double nrm = 0.0;
      if (cpw == 4) stream_pass<4>(X, ld, r0, mloc, n, nwc, vec, e_s, vsm, uni, hred, nrm);
      else if (cpw == 8) stream_pass<8>(X, ld, r0, mloc, n, nwc, vec, e_s, vsm, uni, hred, nrm);
      else stream_pass<16>(X, ld, r0, mloc, n, nwc, vec, e_s, vsm, uni, hred, nrm);
      nrm = block_sum_f64(nrm, scal);
      __syncthreads();
      const int buf = (int)(pass & 1);
      const int nwr = BNW / nwc;
      for (int c = tid; c < n; c += BNT) {
        double s = 0.0;
        for (int w = 0; w < nwr; ++w) s += hred[w * BMAXN + c];
        hpart[buf * BMAXN + c] = s;
      }
      if (tid == 0) {
        scal[16 + buf] = nrm;
        if (pass == 0) scal[18] = ysq;
      }
      // exchange: partial h and norms of every CTA of the cluster, rank order
      csync();
      double enorm2 = 0.0, ysum = 0.0;
      if constexpr (K > 1) {
        for (int k = 0; k < K; ++k) {
          enorm2 += ld_cluster_f64(mapa_u32(smem_u32(&scal[16 + buf]), (uint32_t)k));
          if (pass == 0) ysum += ld_cluster_f64(mapa_u32(smem_u32(&scal[18]), (uint32_t)k));
        }
        for (int c = tid; c < n; c += BNT) {
          double s = 0.0;
          for (int k = 0; k < K; ++k)
            s += ld_cluster_f64(mapa_u32(smem_u32(&hpart[buf * BMAXN + c]), (uint32_t)k));
          h64[c] = s;
        }
      } else {
        enorm2 = scal[16 + buf];
        ysum = scal[18];
        for (int c = tid; c < n; c += BNT) h64[c] = hpart[buf * BMAXN + c];
      }
      if (pass == 0) ynorm = sqrt(ysum);
      const double enorm = sqrt(enorm2);
      double rel = ynorm > 0.0 ? enorm / ynorm : enorm;
      bool stop = false;
      const bool tested = !refill;
      refill = false;
      if (tested) {
        if (rank == 0 && tid == 0 && sd.hist) sd.hist[sw] = rel;
        if (!isfinite(rel)) {
          status = HPSCD_ERR_NONFINITE; stop = true;
        } else if (p.stop_rule == HPSCD_STOP_REL_RES && rel <= p.tol) {
          if (pass == 0 && !ld_volatile_s32(&p.sys[sidx].a_is_guess)) {
            status = HPSCD_OK; stop = true;  // e = y exactly
          } else {
            // confirm on the true residual of the float32 coefficients to be
            // returned: e = y - X·fl32(a) on every CTA's rows, ||e|| over the cluster
            __syncthreads();
            for (int c = tid; c < BMAXN; c += BNT) {
              const float hi = (float)a64_s[c];
              a64_s[c] = (double)hi;
              vsm[c] = hi;
            }
            __syncthreads();
            double t2 = true_residual_rows(X, ld, r0, mloc, n, ld_volatile_ptr(&p.sys[sidx].y), vsm, e_s);
            t2 = block_sum_f64(t2, scal);
            ++confirms;
            if (tid == 0) scal[20] = t2;
            csync();
            double tot = 0.0;
            if constexpr (K > 1) {
              for (int k = 0; k < K; ++k) tot += ld_cluster_f64(mapa_u32(smem_u32(&scal[20]), (uint32_t)k));
            } else {
              tot = scal[20];
            }
            rel = ynorm > 0.0 ? sqrt(tot) / ynorm : sqrt(tot);
            if (rank == 0 && tid == 0 && sd.hist) sd.hist[sw] = rel;
            if (!isfinite(rel)) { status = HPSCD_ERR_NONFINITE; stop = true; }
            else if (rel <= p.tol) { status = HPSCD_OK; stop = true; }
            else if (sw == p.max_sweeps) { status = HPSCD_ERR_NOT_CONVERGED; stop = true; }
            else refill = true;  // the next pass forms h from the recomputed e, with v = 0
          }
        } else if (p.stop_rule == HPSCD_STOP_REL_CHANGE && sw >= 1 &&
                   (r_prev == 0.0 || fabs(r_prev - rel) < p.tol * r_prev)) {
          status = HPSCD_OK; stop = true;
        } else if (sw == p.max_sweeps) {
          status = (p.stop_rule == HPSCD_STOP_NONE) ? HPSCD_OK : HPSCD_ERR_NOT_CONVERGED;
          stop = true;
        }
        r_prev = rel;
      }
      if (stop) break;
      if (refill) {
        ++refills;
        for (int c = tid; c < BMAXN; c += BNT) { vsm[c] = 0.f; da_s[c] = 0.f; }
        __syncthreads();
        continue;
      }
      __syncthreads();  // h64 complete
      // r = h ⊘ d - G~·v, one thread per row: the row's float4 loads are
      // independent of one another, so they are in flight together (columns past
      // n read zeros of G~ and of v up to the next multiple of 4)
      for (int c = tid; c < n; c += BNT) {
        const float4* g4 = reinterpret_cast<const float4*>(Gt + (size_t)c * BLDG);
        const float4* v4 = reinterpret_cast<const float4*>(vsm);
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        const int nq = (n + 3) / 4;
#pragma unroll 8
        for (int q = 0; q < nq; ++q) {
          const float4 g = __ldcg(g4 + q);
          const float4 w = v4[q];
          a0 = fmaf(g.x, w.x, a0);
          a1 = fmaf(g.y, w.y, a1);
          a2 = fmaf(g.z, w.z, a2);
          a3 = fmaf(g.w, w.w, a3);
        }
        const float dc = dd_s[c];
        rvec[c] = (float)((dc > 0.f ? h64[c] / (double)dc : 0.0) - (double)((a0 + a1) + (a2 + a3)));
      }
      __syncthreads();
      forward_sub_scaled(Gt, n, rvec, da_s, diag_s, uni);  // uni is free between passes
      for (int c = tid; c < n; c += BNT) {
        a64_s[c] += (double)da_s[c];
        vsm[c] = da_s[c];
      }
      __syncthreads();
    }
    if (rank == 0) {
      for (int c = tid; c < n; c += BNT) sd.a[c] = (float)a64_s[c];
      if (tid == 0) {
        hpscd_sys_result rr;
        rr.sweeps = pass - refills;
        rr.rel_res = r_prev;
        rr.status = status;
        const int64_t np_ = pass + 1 + confirms;
        rr.passes = (int32_t)(np_ > 0x7fffffff ? 0x7fffffff : np_);
        p.res[sidx] = rr;
      }
    }
    // the next pop (rank 0) must not overwrite sys_s before every CTA read it,
    // and the partial-h buffers are reused by the next system
    csync();
  }
  if constexpr (K > 1) cluster_sync_all();  // no CTA exits while another may still read its shared memory
}

template <int K>
cudaError_t launch_k(const BatchParams& p, int grid, int smem, cudaStream_t stream) {
  // the shared-memory attribute was set by clusters_k (before any stream capture)
  auto kern = batched_sweep_kernel<K>;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(grid);
  lc.blockDim = dim3(BNT);
  lc.dynamicSmemBytes = smem;
  lc.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = K;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  return cudaLaunchKernelEx(&lc, kern, p);
}

// Clusters of K CTAs with `smem` bytes each that are resident at once.  The
// kernel's dynamic shared-memory limit is raised to the device maximum (not to
// `smem`), so graphs captured for other batches stay launchable.
template <int K>
int clusters_k(int smem, int max_smem) {
  auto kern = batched_sweep_kernel<K>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(K);
  lc.blockDim = dim3(BNT);
  lc.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = K;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  int nc = 0;
  if (cudaOccupancyMaxActiveClusters(&nc, kern, &lc) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nc;
}

}  // namespace

int batched_smem_bytes(int64_t mmax, int K) {
  const int64_t rows = (mmax + K - 1) / K + 128;  // a slice is a multiple of 128 rows, plus the tail
  const int ecap = (int)((rows + 127) / 128 * 128);
  return bsmem_plan(ecap).total;
}

int batched_ecap(int64_t mmax, int K) {
  const int64_t rows = (mmax + K - 1) / K + 128;
  return (int)((rows + 127) / 128 * 128);
}

int batched_max_clusters(int K, int smem, int max_smem) {
  switch (K) {
    case 1: return clusters_k<1>(smem, max_smem);
    case 2: return clusters_k<2>(smem, max_smem);
    case 4: return clusters_k<4>(smem, max_smem);
    case 8: return clusters_k<8>(smem, max_smem);
    default: return 0;
  }
}

cudaError_t launch_batched(const BatchParams& p, int K, int clusters, int smem, cudaStream_t stream) {
  const int grid = clusters * K;
  switch (K) {
    case 1: return launch_k<1>(p, grid, smem, stream);
    case 2: return launch_k<2>(p, grid, smem, stream);
    case 4: return launch_k<4>(p, grid, smem, stream);
    case 8: return launch_k<8>(p, grid, smem, stream);
    default: return cudaErrorInvalidConfiguration;
  }
}

}  // namespace hpscd
