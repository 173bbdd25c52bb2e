// Persistent column sweep of Algorithm 1 for tall and square systems
// (column-major X, n <= 512), one CTA per SM, cooperative launch.
//
// Algorithm 1 makes column j's step depend on the residual left by column
// j-1, through a reduction over all m rows.  Writing e_s for the residual at
// the start of sweep s and g = X^T e_s, Eq. ek1-ek gives, just before column
// j of sweep s,
//     <X_j, e> = g_j - sum_{l<j} <X_j, X_l> da_l,
// so the whole sweep's steps follow from g and the lower triangle of
// G = X^T X by forward substitution, in the paper's column order:
//     da_j = (g_j - sum_{l<j} G_jl da_l) / G_jj        (Eq. da2, the ⊘ step)
// and then e_{s+1} = e_s - X·da (the n rank-1 corrections of the sweep,
// Eq. ek1-ek) and a <- a + da.  In exact arithmetic this is Algorithm 1 step
// for step; it lets one streaming pass over X per sweep carry all of the
// sweep's dot products and rank-1 corrections:
//
//   pass p (one read of X):  e <- e - X·da_p   (or e <- y - X·a on a
//                            true-residual pass), then g <- X^T e and
//                            ||e||^2 (float64), tile by tile;
//   grid barrier;            every CTA sums the per-CTA partials of g and
//                            ||e||^2 in a fixed order (bitwise identical in
//                            every CTA), records hist[p] = ||e||/||y||, tests
//                            the stopping rule, and runs the forward
//                            substitution to get da_{p+1}.
//
// X streams through shared memory by TMA (cp.async.bulk.tensor, zero fill
// past m and n) in tiles of R rows × all columns, nstages deep; each warp owns
// CPW columns, each lane RPL consecutive rows.  Phase A forms per-warp row
// partials of X·v, a cross-warp reduction gives the new e of the tile; phase
// B accumulates the lane's partial X^T e in registers for the whole pass.
#include "kernels.h"

namespace hpscd {

namespace {

constexpr int NW = 16;
constexpr int NT = NW * 32;

template <typename T, int RPL>
struct RowLoad;
template <>
struct RowLoad<float, 1> {
  __device__ static void load(const float* p, float (&v)[1]) { v[0] = *p; }
};
template <>
struct RowLoad<float, 2> {
  __device__ static void load(const float* p, float (&v)[2]) {
    const float2 t = *reinterpret_cast<const float2*>(p);
    v[0] = t.x; v[1] = t.y;
  }
};
template <>
struct RowLoad<float, 4> {
  __device__ static void load(const float* p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
};
template <>
struct RowLoad<uint16_t, 2> {
  __device__ static void load(const uint16_t* p, float (&v)[2]) {
    const uint32_t t = *reinterpret_cast<const uint32_t*>(p);
    v[0] = __uint_as_float(t << 16);
    v[1] = __uint_as_float(t & 0xffff0000u);
  }
};
template <>
struct RowLoad<uint16_t, 4> {
  __device__ static void load(const uint16_t* p, float (&v)[4]) {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    v[0] = __uint_as_float(t.x << 16);
    v[1] = __uint_as_float(t.x & 0xffff0000u);
    v[2] = __uint_as_float(t.y << 16);
    v[3] = __uint_as_float(t.y & 0xffff0000u);
  }
};

template <typename T>
__device__ __forceinline__ T zero_elem();
template <>
__device__ __forceinline__ float zero_elem<float>() { return 0.f; }
template <>
__device__ __forceinline__ uint16_t zero_elem<uint16_t>() { return 0; }

// Forward substitution of one sweep (see the file comment):
//   da_j = (r_j - sum_{l<j} G_jl da_l) / d_j, j = 0..n-1, da_j = 0 when d_j = 0.
// Blocks of 32 columns: warp 0 solves the diagonal block with shuffles, then
// every thread applies the block's contribution to one later row.
// r (shared, in: g, overwritten), d and da are shared arrays of length npad.
__device__ void forward_substitution(const float* __restrict__ G, int ldG, int n, int npad,
                                     float* r, const float* d, float* da) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int c = n + tid; c < npad; c += NT) da[c] = 0.f;
  for (int b0 = 0; b0 < n; b0 += 32) {
    if (warp == 0) {
      const int i = b0 + lane;
      float gl[32];
      const float4* row = reinterpret_cast<const float4*>(G + (int64_t)i * ldG + b0);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 t = __ldg(row + q);
        gl[4 * q] = t.x; gl[4 * q + 1] = t.y; gl[4 * q + 2] = t.z; gl[4 * q + 3] = t.w;
      }
      // lanes past n (and past npad when npad < 32) hold zeros and write nothing
      float ri = (i < n) ? r[i] : 0.f;
      const float di = (i < n) ? d[i] : 0.f;
      float mine = 0.f;
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        float q = 0.f;
        if (lane == k) q = (di > 0.f) ? ri / di : 0.f;
        q = __shfl_sync(FULL_MASK, q, k);
        if (lane == k) mine = q;
        if (lane > k) ri = fmaf(-gl[k], q, ri);
      }
      if (i < npad) da[i] = mine;
    }
    __syncthreads();
    for (int i = b0 + 32 + tid; i < n; i += NT) {
      const float4* row = reinterpret_cast<const float4*>(G + (int64_t)i * ldG + b0);
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 t = __ldg(row + q);
        acc = fmaf(t.x, da[b0 + 4 * q], acc);
        acc = fmaf(t.y, da[b0 + 4 * q + 1], acc);
        acc = fmaf(t.z, da[b0 + 4 * q + 2], acc);
        acc = fmaf(t.w, da[b0 + 4 * q + 3], acc);
      }
      r[i] -= acc;
    }
    __syncthreads();
  }
}

// Error-free product and sum (Ogita, Rump, Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26(6), 2005): Dot2 keeps the running sum as an
// unevaluated float pair, giving float64-grade accuracy for the true-residual pass.
__device__ __forceinline__ void dot2_step(float x, float v, float& s, float& c) {
  const float p = x * v;
  const float pe = fmaf(x, v, -p);
  const float t = s + p;
  const float z = t - s;
  const float err = (s - (t - z)) + (p - z);
  s = t;
  c += err + pe;
}

template <typename T, int CPW, int RPL>
__global__ void __launch_bounds__(NT, 1)
    tall_sweep_kernel(const __grid_constant__ CUtensorMap tmap, const TallParams p) {
  constexpr int R = 32 * RPL;
  constexpr int NPAD = NW * CPW;
  constexpr int STAGE_ELEMS = R * NPAD;
  constexpr int BOXC = NPAD < 256 ? NPAD : 256;

  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  T* stages = reinterpret_cast<T*>(base);
  float* red_hi = reinterpret_cast<float*>(base + (size_t)p.nstages * STAGE_ELEMS * sizeof(T));
  float* red_lo = red_hi + NW * R;
  float* etile = red_lo + NW * R;
  float* rvec = etile + R;
  float* da_s = rvec + NPAD;
  float* dd_s = da_s + NPAD;
  double* a64_s = reinterpret_cast<double*>(dd_s + NPAD);
  double* scal = a64_s + NPAD;  // [0]: ||e||^2 total, [1]: ||y||^2 total, [2..33]: scratch
  uint64_t* mbar = reinterpret_cast<uint64_t*>(scal + 40);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grid = gridDim.x;
  const int64_t t0 = p.ntiles * blockIdx.x / grid;
  const int64_t t1 = p.ntiles * (blockIdx.x + 1) / grid;
  const int64_t nt = t1 - t0;
  const int nst = p.nstages;
  const bool tma = p.use_tma != 0;
  const int64_t m = p.m;
  const int n = p.n;

  if (tid == 0 && tma) {
    for (int s = 0; s < nst; ++s) mbar_init(&mbar[s], 1);
    fence_mbar_init();
  }
  for (int c = tid; c < NPAD; c += NT) {
    a64_s[c] = (c < n && p.warm) ? (double)p.a_in[c] : 0.0;
    dd_s[c] = (c < n) ? p.G[(int64_t)c * p.ldG + c] : 0.f;
  }
  __syncthreads();

  uint64_t issued = 0, consumed = 0, waited = 0;
  auto issue_next = [&]() {
    const uint64_t seq = issued++;
    const int s = (int)(seq % nst);
    const int64_t tile = t0 + (int64_t)(seq % (uint64_t)nt);
    T* dst = stages + (size_t)s * STAGE_ELEMS;
    mbar_arrive_expect_tx(&mbar[s], STAGE_ELEMS * sizeof(T));
#pragma unroll
    for (int cb = 0; cb < NPAD; cb += BOXC)
      tma_load_2d(dst + cb * R, &tmap, &mbar[s], (int32_t)(tile * R), cb);
  };
  if (tma && tid == 0)
    for (int s = 0; s < nst; ++s) issue_next();

  float v[CPW];
#pragma unroll
  for (int k = 0; k < CPW; ++k) v[k] = (float)a64_s[warp * CPW + k];
  float gacc[CPW];
#pragma unroll
  for (int k = 0; k < CPW; ++k) gacc[k] = 0.f;

  int err = DEV_OK;
  int status = HPSCD_ERR_NOT_CONVERGED;
  double r_prev = 0.0, ynorm = 0.0;
  int64_t pass = 0, sweeps = 0;

  for (pass = 0;; ++pass) {
    const int mode = (pass == 0) ? (p.warm ? MODE_REFRESH : MODE_COPY)
                                 : ((p.refresh_every > 0 && pass % p.refresh_every == 0)
                                        ? MODE_REFRESH
                                        : MODE_NORMAL);
    double nrm = 0.0, ysq = 0.0;
    for (int64_t it = 0; it < nt; ++it) {
      const int64_t tile = t0 + it;
      const uint64_t seq = consumed++;
      const int s = (int)(seq % nst);
      T* st = stages + (size_t)s * STAGE_ELEMS;
      const int64_t row = tile * R + tid;
      float e_old = 0.f, y_row = 0.f;
      if (tid < R && row < m) {
        if (mode == MODE_NORMAL) e_old = p.e[row];
        else y_row = p.y[row];
      }
      bool ok = true;
      if (tma) {
        ok = mbar_wait_bounded(&mbar[s], (uint32_t)((seq / nst) & 1), p.timeout_ns);
      } else {
        __syncthreads();
        const T* X = reinterpret_cast<const T*>(p.X);
        for (int idx = tid; idx < STAGE_ELEMS; idx += NT) {
          const int c = idx / R, r = idx % R;
          const int64_t gr = tile * R + r;
          st[idx] = (gr < m && c < n) ? X[(int64_t)c * p.ld + gr] : zero_elem<T>();
        }
        __syncthreads();
      }
      // phase A: per-warp partial of (X·v) for the tile's rows
      if (ok && mode != MODE_COPY) {
        float ph[RPL], pl[RPL];
#pragma unroll
        for (int r = 0; r < RPL; ++r) { ph[r] = 0.f; pl[r] = 0.f; }
#pragma unroll
        for (int k = 0; k < CPW; ++k) {
          float xv[RPL];
          RowLoad<T, RPL>::load(st + (warp * CPW + k) * R + lane * RPL, xv);
#pragma unroll
          for (int r = 0; r < RPL; ++r) {
            if (mode == MODE_NORMAL) ph[r] = fmaf(xv[r], v[k], ph[r]);
            else dot2_step(xv[r], v[k], ph[r], pl[r]);
          }
        }
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
          red_hi[warp * R + lane * RPL + r] = ph[r];
          red_lo[warp * R + lane * RPL + r] = pl[r];
        }
      }
      // S1: all warps are past phase B of the previous tile and phase A of this one
      const int fail = __syncthreads_or(ok ? 0 : 1);
      if (fail) { err = DEV_TIMEOUT_COPY; break; }
      ++waited;
      if (tma && tid == 0 && seq >= 1) {
        fence_proxy_async_smem();
        issue_next();  // refills the previous tile's stage
      }
      if (tid < R) {
        float e_new = 0.f;
        if (row < m) {
          if (mode == MODE_NORMAL) {
            float sacc = 0.f;
#pragma unroll
            for (int w = 0; w < NW; ++w) sacc += red_hi[w * R + tid];
            e_new = e_old - sacc;
          } else if (mode == MODE_COPY) {
            e_new = y_row;
          } else {
            double sacc = 0.0;
#pragma unroll
            for (int w = 0; w < NW; ++w)
              sacc += (double)red_hi[w * R + tid] + (double)red_lo[w * R + tid];
            e_new = (float)((double)y_row - sacc);
          }
          p.e[row] = e_new;
          nrm = fma((double)e_new, (double)e_new, nrm);
          if (pass == 0) ysq = fma((double)y_row, (double)y_row, ysq);
        }
        etile[tid] = e_new;
      }
      __syncthreads();  // S2
      // phase B: lane partials of X^T e
      float ev[RPL];
#pragma unroll
      for (int r = 0; r < RPL; ++r) ev[r] = etile[lane * RPL + r];
#pragma unroll
      for (int k = 0; k < CPW; ++k) {
        float xv[RPL];
        RowLoad<T, RPL>::load(st + (warp * CPW + k) * R + lane * RPL, xv);
#pragma unroll
        for (int r = 0; r < RPL; ++r) gacc[k] = fmaf(xv[r], ev[r], gacc[k]);
      }
    }
    if (err != DEV_OK) break;

    // publish this CTA's partials
    const int buf = (int)(pass & 1);
#pragma unroll
    for (int k = 0; k < CPW; ++k) {
      float sacc = gacc[k];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) sacc += __shfl_xor_sync(FULL_MASK, sacc, off);
      if (lane == 0) p.gpart[((size_t)buf * grid + blockIdx.x) * NPAD + warp * CPW + k] = sacc;
      gacc[k] = 0.f;
    }
    if (warp < R / 32) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        nrm += __shfl_xor_sync(FULL_MASK, nrm, off);
        ysq += __shfl_xor_sync(FULL_MASK, ysq, off);
      }
      if (lane == 0) { scal[2 + warp] = nrm; scal[2 + 16 + warp] = ysq; }
    }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < R / 32; ++w) { a += scal[2 + w]; b += scal[2 + 16 + w]; }
      p.npart[(size_t)buf * grid + blockIdx.x] = a;
      if (pass == 0) p.ypart[blockIdx.x] = b;
    }
    const unsigned expected = (unsigned)grid + ((p.stall_barrier && pass == 0) ? 1u : 0u);
    if (!grid_barrier(p.ctl, expected, p.timeout_ns)) { err = DEV_TIMEOUT_BARRIER; break; }

    // every CTA: g = sum of partials (fixed order), ||e||^2, ||y||^2
    for (int c = tid; c < NPAD; c += NT) {
      double sacc = 0.0;
      const float* gp = p.gpart + (size_t)buf * grid * NPAD + c;
#pragma unroll 8
      for (int b = 0; b < grid; ++b) sacc += (double)__ldcg(gp + (size_t)b * NPAD);
      rvec[c] = (float)sacc;
    }
    if (warp == 0) {
      double a = 0.0, b = 0.0;
      for (int blk = lane; blk < grid; blk += 32) {
        a += __ldcg(p.npart + (size_t)buf * grid + blk);
        if (pass == 0) b += __ldcg(p.ypart + blk);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(FULL_MASK, a, off);
        b += __shfl_xor_sync(FULL_MASK, b, off);
      }
      if (lane == 0) { scal[0] = a; scal[1] = b; }
    }
    __syncthreads();
    if (pass == 0) ynorm = sqrt(scal[1]);
    const double enorm = sqrt(scal[0]);
    const double rel = ynorm > 0.0 ? enorm / ynorm : enorm;
    if (blockIdx.x == 0 && tid == 0) p.hist[pass] = rel;
    sweeps = pass;
    bool stop = false;
    if (!isfinite(rel)) {
      status = HPSCD_ERR_NONFINITE; stop = true;
    } else if (p.stop_rule == HPSCD_STOP_REL_RES && rel <= p.tol) {
      status = HPSCD_OK; stop = true;
    } else if (p.stop_rule == HPSCD_STOP_REL_CHANGE && pass >= 1 &&
               (r_prev == 0.0 || fabs(r_prev - rel) < p.tol * r_prev)) {
      status = HPSCD_OK; stop = true;
    } else if (pass == p.max_sweeps) {
      status = (p.stop_rule == HPSCD_STOP_NONE) ? HPSCD_OK : HPSCD_ERR_NOT_CONVERGED;
      stop = true;
    }
    r_prev = rel;
    if (stop) break;

    forward_substitution(p.G, p.ldG, n, NPAD, rvec, dd_s, da_s);
    for (int c = tid; c < NPAD; c += NT) a64_s[c] += (double)da_s[c];
    __syncthreads();
    const int64_t nx = pass + 1;
    const bool next_refresh = p.refresh_every > 0 && nx % p.refresh_every == 0;
#pragma unroll
    for (int k = 0; k < CPW; ++k) {
      const int c = warp * CPW + k;
      v[k] = next_refresh ? (float)a64_s[c] : da_s[c];
    }
  }

  // drain copies still in flight before the CTA retires
  if (tma && tid == 0) {
    for (uint64_t seq = waited; seq < issued; ++seq)
      if (!mbar_wait_bounded(&mbar[seq % nst], (uint32_t)((seq / nst) & 1), p.timeout_ns)) {
        if (err == DEV_OK) err = DEV_TIMEOUT_COPY;
        break;
      }
  }
  __syncthreads();
  if (err != DEV_OK && tid == 0) atomicCAS(&p.ctl->err, DEV_OK, err);
  if (blockIdx.x == 0) {
    for (int c = tid; c < n; c += NT) p.a_out[c] = (float)a64_s[c];
    if (tid == 0) {
      p.ctl->status = (err != DEV_OK) ? HPSCD_ERR_TIMEOUT : status;
      p.ctl->sweeps = sweeps;
      p.ctl->final_res = r_prev;
      p.ctl->passes = pass + 1;
    }
  }
}

template <typename T, int CPW, int RPL>
cudaError_t launch_one(const TallConfig& cfg, const CUtensorMap* tmap, const TallParams& p,
                       int grid, cudaStream_t stream) {
  auto kern = tall_sweep_kernel<T, CPW, RPL>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       cfg.smem_bytes);
  if (e != cudaSuccess) return e;
  CUtensorMap map = *tmap;
  TallParams pp = p;
  void* args[] = {(void*)&map, (void*)&pp};
  return cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(NT), args,
                                     (size_t)cfg.smem_bytes, stream);
}

}  // namespace

// Tile geometry: CPW = columns per warp (power of two, 16·CPW >= n), RPL = rows
// per lane chosen so one stage (R × 16·CPW elements) stays near 64 KB.
bool tall_config(int dtype, int n, int max_smem, TallConfig* cfg) {
  if (n < 0 || n > 512) return false;
  int cpw = 1;
  while (NW * cpw < n) cpw *= 2;
  const int esz = (dtype == HPSCD_F32) ? 4 : 2;
  const int rowbytes = NW * cpw * esz;
  int rpl = rowbytes <= 256 ? 4 : (rowbytes <= 1024 ? 2 : 1);
  if (dtype == HPSCD_BF16 && rpl == 1) rpl = 2;
  cfg->cpw = cpw;
  cfg->rpl = rpl;
  cfg->npad = NW * cpw;
  cfg->rows = 32 * rpl;
  cfg->stage_bytes = cfg->rows * cfg->npad * esz;
  cfg->box_cols = cfg->npad < 256 ? cfg->npad : 256;
  cfg->threads = NT;
  const int fixed = 1024 /*align*/ + (2 * NW * cfg->rows + cfg->rows) * 4 + cfg->npad * (3 * 4 + 8) +
                    40 * 8 + 8 * 8;
  int nst = (max_smem - 256 - fixed) / cfg->stage_bytes;
  if (nst > 8) nst = 8;
  if (nst < 2) return false;
  cfg->nstages = nst;
  cfg->smem_bytes = fixed + nst * cfg->stage_bytes;
  return true;
}

cudaError_t launch_tall_sweep(int dtype, const TallConfig& cfg, const CUtensorMap* tmap,
                              const TallParams& p, int grid, cudaStream_t stream) {
#define HPSCD_TALL_CASE(T, C, R)                                        \
  if (cfg.cpw == C && cfg.rpl == R) return launch_one<T, C, R>(cfg, tmap, p, grid, stream);
  if (dtype == HPSCD_F32) {
    HPSCD_TALL_CASE(float, 1, 4)
    HPSCD_TALL_CASE(float, 2, 4)
    HPSCD_TALL_CASE(float, 4, 4)
    HPSCD_TALL_CASE(float, 8, 2)
    HPSCD_TALL_CASE(float, 16, 2)
    HPSCD_TALL_CASE(float, 32, 1)
  } else {
    HPSCD_TALL_CASE(uint16_t, 1, 4)
    HPSCD_TALL_CASE(uint16_t, 2, 4)
    HPSCD_TALL_CASE(uint16_t, 4, 4)
    HPSCD_TALL_CASE(uint16_t, 8, 4)
    HPSCD_TALL_CASE(uint16_t, 16, 2)
    HPSCD_TALL_CASE(uint16_t, 32, 2)
  }
#undef HPSCD_TALL_CASE
  return cudaErrorInvalidConfiguration;
}

}  // namespace hpscd
