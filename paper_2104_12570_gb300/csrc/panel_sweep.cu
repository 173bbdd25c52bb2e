// Persistent column sweep of Algorithm 1 for column-major X with more than
// 512 columns (any m): one CTA per SM, cooperative launch.
//
// The n columns are taken in panels of PW = 512 consecutive columns, panel by
// panel in the paper's column order.  Inside a panel Q the steps follow, as in
// the tall sweep, from the dot products against the residual e as it stands
// before the panel and the panel's diagonal block of G = X^T X (Eq. ek1-ek
// applied to the panel's own columns), by forward substitution on the
// pre-divided couplings G~ = D^{-1} G:
//     da_j = <X_j, e> / G_jj - sum_{l<j, l in Q} G~_jl da_l   (Eq. da2, j in Q).
// Across panels the residual itself carries the coupling: pass t applies the
// rank-1 corrections of the panel solved before it (e <- e - X_P·da_P, Eq.
// ek1-ek) and forms the next panel's dot products against that updated e,
// row segment by row segment (a segment's dots need only the segment's e), so
// the only couplings formed in set-up are the panels' diagonal Gram blocks
// (O(m·n·PW) work, not the O(m·n^2) of a full Gram) and every column is read
// twice per sweep: once for its dot products, once for its corrections.
//
// Every CTA owns a contiguous range of 128-row chunks and walks it in segments
// of SEG_CHUNKS chunks (plain loads) or box by box (TMA): first the corrections (a warp per chunk, each lane 4
// consecutive rows, the segment's updated e kept in shared memory and written
// back), then the dots (a warp per 32 columns of the next panel, float32 sums
// over the segment, float64 across segments and, by atomics, across CTAs).
// After a grid barrier every CTA reads the same float64 dot products, forms
// r = h ⊘ d and runs the panel's substitution itself (bitwise the same in
// every CTA), so the next pass needs no broadcast of da.
#include <cuda_fp16.h>
#include <string.h>

#include "kernels.h"

namespace hpscd {

namespace {

constexpr int PW = PANEL_W;       // columns per panel
constexpr int PNW = 16;           // warps per CTA
constexpr int PNT = PNW * 32;     // threads per CTA (one per column of a panel)
constexpr int SEG_CHUNKS = 32;    // 128-row chunks per row segment
constexpr int SEG_ROWS = SEG_CHUNKS * 128;

// what a pass does to the residual before the dot products
enum PassKind : int {
  PK_COPY_Y = 0,  // e = y (cold start)
  PK_APPLY = 1,   // e -= X_P·da_P (the panel solved before this pass)
  PK_TRUE = 2     // e = y - X·v over all n columns, compensated (Dot2)
};

// Four consecutive rows of one column, widened exactly to float32.
template <typename T>
struct Rows4;
template <>
struct Rows4<float> {
  __device__ static void vec(const float* p, float (&v)[4]) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  __device__ static float one(const float* p) { return __ldg(p); }
};
template <>
struct Rows4<uint16_t> {
  __device__ static void vec(const uint16_t* p, float (&v)[4]) {
    const uint2 t = __ldg(reinterpret_cast<const uint2*>(p));
    v[0] = __uint_as_float(t.x << 16);
    v[1] = __uint_as_float(t.x & 0xffff0000u);
    v[2] = __uint_as_float(t.y << 16);
    v[3] = __uint_as_float(t.y & 0xffff0000u);
  }
  __device__ static float one(const uint16_t* p) { return bf16_bits_to_float(__ldg(p)); }
};
template <>
struct Rows4<__half> {
  __device__ static void vec(const __half* p, float (&v)[4]) {
    const uint2 t = __ldg(reinterpret_cast<const uint2*>(p));
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&t.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&t.y));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  __device__ static float one(const __half* p) {
    return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short*>(p))));
  }
};

// Four consecutive rows of a column of a TMA box in shared memory (plain
// loads: __ldg is for global memory only), widened exactly to float32.
template <typename T>
struct BoxRows4;
template <>
struct BoxRows4<float> {
  __device__ static void load(const float* p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
};
template <>
struct BoxRows4<uint16_t> {
  __device__ static void load(const uint16_t* p, float (&v)[4]) {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    v[0] = __uint_as_float(t.x << 16);
    v[1] = __uint_as_float(t.x & 0xffff0000u);
    v[2] = __uint_as_float(t.y << 16);
    v[3] = __uint_as_float(t.y & 0xffff0000u);
  }
};
template <>
struct BoxRows4<__half> {
  __device__ static void load(const __half* p, float (&v)[4]) {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&t.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&t.y));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};

// Rows r0..r0+3 of column `col` (zero past m).  vec: X is aligned for vector loads.
template <typename T>
__device__ __forceinline__ void load_rows4(const T* __restrict__ X, int64_t ld, int64_t col, int64_t r0,
                                           int64_t m, bool vec, float (&v)[4]) {
  const T* p = X + col * ld + r0;
  if (vec && r0 + 4 <= m) {
    Rows4<T>::vec(p, v);
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = (r0 + i < m) ? Rows4<T>::one(p + i) : 0.f;
  }
}

// s + c += -x·v with the error-free transformations of Dot2 (TwoProduct by
// fma, TwoSum), so that s + c carries about twice float32's precision.
__device__ __forceinline__ void dot2_sub(float x, float v, float& s, float& c) {
  const float p = -x * v;
  const float pe = fmaf(-x, v, -p);
  const float t = s + p;
  const float bb = t - s;
  const float err = (s - (t - bb)) + (p - bb);
  s = t;
  c += err + pe;
}

// Forward substitution of one panel: on entry r_s[i] = h_i / d_i (i < nq); on
// exit da_s[i] = da_i (0 for nq <= i < PW).  Gq: the panel's G~ block, row-major
// with row stride PW, whose 32 x 32 diagonal blocks hold (below the diagonal)
// M_b = (I + L_b)^{-1} in place of L_b (invert_panel_diag_kernel, in the
// set-up).  Blocks of 32 steps: warp 0 solves a block as da_b = M_b r_b (lane l
// owns step 32b + l and keeps its row of M_b in registers: 32 independent
// shuffles), then every thread applies the block to its later row.
__device__ void panel_substitution(const float* __restrict__ Gq, int nq, float* r_s, float* da_s) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nb = (nq + 31) / 32;
  for (int b = 0; b < nb; ++b) {
    const int i0 = 32 * b;
    if (warp == 0) {
      const int i = i0 + lane;
      float g[32];
      if (i < nq) {
        const float4* row = reinterpret_cast<const float4*>(Gq + (size_t)i * PW + i0);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float4 t = __ldg(row + k);
          g[4 * k] = t.x; g[4 * k + 1] = t.y; g[4 * k + 2] = t.z; g[4 * k + 3] = t.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) g[k] = 0.f;
      }
      const float v = (i < nq) ? r_s[i] : 0.f;
      float acc[4] = {v, 0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const float dk = __shfl_sync(FULL_MASK, v, k);
        acc[k & 3] = fmaf(lane > k ? g[k] : 0.f, dk, acc[k & 3]);
      }
      da_s[i] = (i < nq) ? (acc[0] + acc[1]) + (acc[2] + acc[3]) : 0.f;
    }
    __syncthreads();
    const int i = tid;
    if (i >= i0 + 32 && i < nq) {
      const float4* row = reinterpret_cast<const float4*>(Gq + (size_t)i * PW + i0);
      float acc = r_s[i];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float4 t = __ldg(row + k);
        acc = fmaf(-t.x, da_s[i0 + 4 * k], acc);
        acc = fmaf(-t.y, da_s[i0 + 4 * k + 1], acc);
        acc = fmaf(-t.z, da_s[i0 + 4 * k + 2], acc);
        acc = fmaf(-t.w, da_s[i0 + 4 * k + 3], acc);
      }
      r_s[i] = acc;
    }
    __syncthreads();
  }
  for (int i = 32 * nb + tid; i < PW; i += PNT) da_s[i] = 0.f;
  __syncthreads();
}

// Set-up of the panel substitution: each 32 x 32 diagonal block I + L_b of a
// panel's G~ block (unit lower triangular below the diagonal) gets M_b =
// (I + L_b)^{-1} written over L_b, in place; the diagonal and the upper part
// stay.  One warp per block (blockIdx.x = panel · PW/32 + b); lane j forms
// column j: M_ij = -sum_{k<i} L_ik M_kj for i > j, reading L before any write.
__global__ void __launch_bounds__(32) invert_panel_diag_kernel(float* __restrict__ Gt) {
  const int lane = threadIdx.x;
  const int q = blockIdx.x / (PW / 32), b = blockIdx.x % (PW / 32);
  float* blk = Gt + (size_t)q * PW * PW + (size_t)(32 * b) * PW + 32 * b;
  float mcol[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < i; ++k) s = fmaf(blk[(size_t)i * PW + k], mcol[k], s);  // mcol[k] = 0 for k < lane
    mcol[i] = i < lane ? 0.f : (i == lane ? 1.f : -s);
  }
  __syncwarp();
#pragma unroll
  for (int i = 1; i < 32; ++i)
    if (i > lane) blk[(size_t)i * PW + lane] = mcol[i];
}

// Sum over the CTAs of one partial per CTA, in a fixed order (the same value
// in every CTA).  Called by all threads; the result is in every thread.
__device__ double sum_partials(const double* __restrict__ part, int count, double* red) {
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int i = threadIdx.x; i < count; i += 32) s += __ldcg(part + i);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(FULL_MASK, s, o);
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  const double v = red[0];
  __syncthreads();
  return v;
}

__device__ __forceinline__ double rel_of(double e2, double y2) {
  const double en = sqrt(e2), yn = sqrt(y2);
  return yn > 0.0 ? en / yn : en;
}

// TMA: X streams through shared memory by TMA in boxes of 128 rows x BC
// columns (32 KB) instead of plain loads.
template <typename T, bool TMA>
__global__ void __launch_bounds__(PNT, 1)
    panel_sweep_kernel(const __grid_constant__ CUtensorMap tmap, const PanelParams p) {
  __shared__ __align__(16) float e_sm[TMA ? 4 : SEG_ROWS];
  __shared__ __align__(16) float r_s[PW];
  __shared__ __align__(16) float da_s[PW];
  __shared__ double red[PNW];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* __restrict__ X = static_cast<const T*>(p.X);
  const int64_t m = p.m, ld = p.ld;
  const int n = p.n, npan = p.npanels;
  const bool vec = p.vec != 0;
  // the CTA's contiguous range of 128-row chunks
  const int64_t nchunks = (m + 127) / 128;
  const int64_t c_begin = nchunks * blockIdx.x / gridDim.x;
  const int64_t c_end = nchunks * (blockIdx.x + 1) / gridDim.x;
  const unsigned G = gridDim.x;
  const bool lead = blockIdx.x == 0;
  int err = DEV_OK;

  if (lead)
    for (int j = tid; j < n; j += PNT) p.a64[j] = p.warm ? (double)p.a_in[j] : 0.0;

  // One pass: the residual step of `kind`, then the dot products of panel qd
  // into hacc[hb]; the CTA's ||e||^2 (and, on the first pass, ||y||^2) partials.
  auto run_pass = [&](int kind, int qp, int qd, int hb, int nb, bool first) {
    const int p0 = qp * PW, np = min(PW, n - p0);
    const int d0 = qd * PW, nd = min(PW, n - d0);
    double e2 = 0.0, y2 = 0.0, acc64 = 0.0;
    const int dcol = 32 * warp;  // this warp's first column of the dot panel
    for (int64_t s0 = c_begin; s0 < c_end; s0 += SEG_CHUNKS) {
      const int nc = (int)min((int64_t)SEG_CHUNKS, c_end - s0);
      // residual step, a warp per chunk
      for (int c = warp; c < nc; c += PNW) {
        const int64_t r0 = (s0 + c) * 128 + 4 * lane;
        float ev[4];
        if (kind == PK_APPLY) {
          const float4 t = *reinterpret_cast<const float4*>(p.e + r0);
          // eight columns' loads in flight per step, two accumulator sets
          float a0[4] = {0.f, 0.f, 0.f, 0.f}, a1[4] = {0.f, 0.f, 0.f, 0.f};
          int j = 0;
          for (; j + 8 <= np; j += 8) {
            float x[8][4];
#pragma unroll
            for (int u = 0; u < 8; ++u) load_rows4<T>(X, ld, p0 + j + u, r0, m, vec, x[u]);
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
              const float v0 = da_s[j + u], v1 = da_s[j + u + 1];
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                a0[i] = fmaf(x[u][i], v0, a0[i]);
                a1[i] = fmaf(x[u + 1][i], v1, a1[i]);
              }
            }
          }
          for (; j < np; ++j) {
            float x0[4];
            load_rows4<T>(X, ld, p0 + j, r0, m, vec, x0);
#pragma unroll
            for (int i = 0; i < 4; ++i) a0[i] = fmaf(x0[i], da_s[j], a0[i]);
          }
          ev[0] = t.x - (a0[0] + a1[0]);
          ev[1] = t.y - (a0[1] + a1[1]);
          ev[2] = t.z - (a0[2] + a1[2]);
          ev[3] = t.w - (a0[3] + a1[3]);
        } else {
          float yv[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) yv[i] = (r0 + i < m) ? __ldg(p.y + r0 + i) : 0.f;
          if (first) {
#pragma unroll
            for (int i = 0; i < 4; ++i) y2 += (double)yv[i] * (double)yv[i];
          }
          if (kind == PK_COPY_Y) {
#pragma unroll
            for (int i = 0; i < 4; ++i) ev[i] = yv[i];
          } else {
            // e = y - X·v, v = hi + lo of the float64 coefficients (lo = 0 for the
            // float32 coefficients of a confirmation, or a warm start's guess)
            float s[4], cc[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { s[i] = yv[i]; cc[i] = 0.f; }
            // four columns' loads in flight per step
            for (int j0 = 0; j0 < n; j0 += 4) {
              float x[4][4], vh[4], vl[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int j = j0 + u;
                vh[u] = 0.f;
                vl[u] = 0.f;
                if (j < n) {
                  load_rows4<T>(X, ld, j, r0, m, vec, x[u]);
                  if (first) {
                    vh[u] = __ldg(p.a_in + j);
                  } else {
                    const double a = __ldcg(p.a64 + j);
                    vh[u] = (float)a;
                    vl[u] = (float)(a - (double)vh[u]);
                  }
                } else {
#pragma unroll
                  for (int i = 0; i < 4; ++i) x[u][i] = 0.f;
                }
              }
#pragma unroll
              for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                  dot2_sub(x[u][i], vh[u], s[i], cc[i]);
                  cc[i] = fmaf(-x[u][i], vl[u], cc[i]);
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) ev[i] = s[i] + cc[i];
          }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (r0 + i >= m) ev[i] = 0.f;
          e2 += (double)ev[i] * (double)ev[i];
        }
        *reinterpret_cast<float4*>(p.e + r0) = make_float4(ev[0], ev[1], ev[2], ev[3]);
        *reinterpret_cast<float4*>(e_sm + c * 128 + 4 * lane) = make_float4(ev[0], ev[1], ev[2], ev[3]);
      }
      __syncthreads();
      // dot products of the dot panel's columns dcol..dcol+31 over the segment
      if (dcol < nd) {
        float acc[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) acc[k] = 0.f;
        for (int c = 0; c < nc; ++c) {
          const int64_t r0 = (s0 + c) * 128 + 4 * lane;
          const float4 et = *reinterpret_cast<const float4*>(e_sm + c * 128 + 4 * lane);
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            if (dcol + k < nd) {
              float x[4];
              load_rows4<T>(X, ld, d0 + dcol + k, r0, m, vec, x);
              acc[k] = fmaf(x[0], et.x, fmaf(x[1], et.y, fmaf(x[2], et.z, fmaf(x[3], et.w, acc[k]))));
            }
          }
        }
        // lane k ends with the segment's sum for column dcol + k
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
          const bool upper = (lane & o) != 0;
#pragma unroll
          for (int k = 0; k < o; ++k) {
            const float send = upper ? acc[k] : acc[k + o];
            const float keep = upper ? acc[k + o] : acc[k];
            acc[k] = keep + __shfl_xor_sync(FULL_MASK, send, o);
          }
        }
        acc64 += (double)acc[0];
      }
      __syncthreads();
    }
    if (dcol + lane < nd && c_end > c_begin) atomicAdd(p.hacc + (size_t)hb * PW + dcol + lane, acc64);
    // the CTA's ||e||^2 and ||y||^2 partials
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      e2 += __shfl_xor_sync(FULL_MASK, e2, o);
      y2 += __shfl_xor_sync(FULL_MASK, y2, o);
    }
    if (lane == 0) red[warp] = e2;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < PNW; ++w) s += red[w];
      p.npart[(size_t)nb * G + blockIdx.x] = s;
    }
    __syncthreads();
    if (first) {
      if (lane == 0) red[warp] = y2;
      __syncthreads();
      if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < PNW; ++w) s += red[w];
        p.ypart[blockIdx.x] = s;
      }
      __syncthreads();
    }
  };

  // ---- the same pass streamed by TMA ----
  // Per 128-row chunk of the CTA: the apply boxes (the previous panel's columns,
  // or all columns for y - X·v), each warp its BC/16 columns and each lane 4
  // rows, keeping the lane's row partials (Dot2 pairs for y - X·v); a cross-warp
  // reduction gives the chunk's new e (threads 0..127, one row each); then the
  // dot boxes of the next panel against that e, each lane keeping its 32 column
  // partials over the chunks (float64 every 8 chunks).  Box s of a pass is
  // sequence qbase + s of the stage ring (stage and parity from it); the ring is
  // refilled after each box's CTA barrier and drains at the end of the pass.
  constexpr int BC = PANEL_BOX_BYTES / (128 * (int)sizeof(T));  // box columns: 128 (float32) or 256 (16-bit)
  constexpr int CWB = BC / 16;                          // columns of a box per warp
  constexpr int NBP = PW / BC;                          // boxes of a full panel
  constexpr int BOXB = 128 * BC * (int)sizeof(T);
  extern __shared__ unsigned char dyn_smem[];
  unsigned char* dbase = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dyn_smem) + 1023) & ~uintptr_t(1023));
  const int nst = p.nstages;
  T* stages = reinterpret_cast<T*>(dbase);
  float* red_h = reinterpret_cast<float*>(dbase + (size_t)nst * BOXB);  // [PNW][128]
  float* red_l = red_h + PNW * 128;                                     // [PNW][128]
  float* ech = red_l + PNW * 128;                                       // [128]
  uint64_t* full = reinterpret_cast<uint64_t*>(ech + 128);              // [nst]
  uint64_t qbase = 0, issued_g = 0, waited_g = 0;
  bool tma_fail = false;
  if (TMA && tid == 0) {
    for (int i = 0; i < nst; ++i) mbar_init(&full[i], 1);
    fence_mbar_init();
  }
  if (TMA) __syncthreads();
  auto run_pass_tma = [&](int kind, int qp, int qd, int hb, int nb, bool first) -> bool {
    const int p0 = qp * PW, np = min(PW, n - p0);
    const int d0 = qd * PW, nd = min(PW, n - d0);
    const int nA = kind == PK_APPLY ? (np + BC - 1) / BC : (kind == PK_TRUE ? (n + BC - 1) / BC : 0);
    const int a0c = kind == PK_APPLY ? p0 : 0;  // first column of the apply boxes
    const int nD = (nd + BC - 1) / BC;
    const int bpc = nA + nD;                    // boxes per chunk
    const int64_t nch = c_end - c_begin;
    const uint64_t total = (uint64_t)(nch > 0 ? nch : 0) * (uint64_t)bpc;
    auto issue = [&](uint64_t s) {  // box s of the pass (thread 0)
      const uint64_t gs = qbase + s;
      const int st = (int)(gs % nst);
      const int64_t ch = c_begin + (int64_t)(s / bpc);
      const int idx = (int)(s % bpc);
      const int col = idx < nA ? a0c + idx * BC : d0 + (idx - nA) * BC;
      mbar_arrive_expect_tx(&full[st], (uint32_t)BOXB);
      tma_load_2d(stages + (size_t)st * 128 * BC, &tmap, &full[st], (int32_t)(ch * 128), col);
    };
    if (tid == 0)
      for (uint64_t s = 0; s < total && s < (uint64_t)nst; ++s) { issue(s); ++issued_g; }
    // one box of the pass: wait for it (every thread), hand it to f, release it
    auto box = [&](uint64_t s, auto f) -> bool {
      const uint64_t gs = qbase + s;
      const int st = (int)(gs % nst);
      const bool ok = mbar_wait_bounded(&full[st], (uint32_t)((gs / nst) & 1), p.timeout_ns);
      ++waited_g;
      if (ok) f(stages + (size_t)st * 128 * BC);
      if (__syncthreads_or(ok ? 0 : 1)) return false;
      if (tid == 0 && s + nst < total) {
        fence_proxy_async_smem();
        issue(s + nst);
        ++issued_g;
      }
      return true;
    };
    double e2 = 0.0, y2 = 0.0, acc64 = 0.0;
    float gacc[NBP][CWB];
#pragma unroll
    for (int b = 0; b < NBP; ++b)
#pragma unroll
      for (int c = 0; c < CWB; ++c) gacc[b][c] = 0.f;
    int since_flush = 0;
    // lane l ends with the warp's total of accumulator l = b·CWB + c
    auto flush = [&]() {
      float v[32];
#pragma unroll
      for (int b = 0; b < NBP; ++b)
#pragma unroll
        for (int c = 0; c < CWB; ++c) { v[b * CWB + c] = gacc[b][c]; gacc[b][c] = 0.f; }
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < o; ++k) {
          const float send = upper ? v[k] : v[k + o];
          const float keep = upper ? v[k + o] : v[k];
          v[k] = keep + __shfl_xor_sync(FULL_MASK, send, o);
        }
      }
      acc64 += (double)v[0];
    };
    for (int64_t ci = 0; ci < nch; ++ci) {
      const int64_t ch = c_begin + ci;
      // the reducers' inputs of this chunk, loaded before its boxes are worked on
      const int64_t rrow = ch * 128 + tid;
      float e_in = 0.f, y_in = 0.f;
      if (tid < 128 && rrow < m) {
        if (kind == PK_APPLY) e_in = p.e[rrow];
        else y_in = __ldg(p.y + rrow);
      }
      float ph[4] = {0.f, 0.f, 0.f, 0.f}, pl[4] = {0.f, 0.f, 0.f, 0.f};
      for (int b = 0; b < nA; ++b) {
        const int colw = a0c + b * BC + warp * CWB;  // this warp's first column of the box
        const bool ok = box((uint64_t)ci * bpc + b, [&](const T* bx) {
#pragma unroll
          for (int c = 0; c < CWB; ++c) {
            const int j = colw + c;
            float x[4];
            BoxRows4<T>::load(bx + (warp * CWB + c) * 128 + 4 * lane, x);  // zero past m and n
            if (kind == PK_APPLY) {
              const float v = (j - p0 < np) ? da_s[j - p0] : 0.f;
#pragma unroll
              for (int r = 0; r < 4; ++r) ph[r] = fmaf(x[r], v, ph[r]);
            } else if (j < n) {
              float vh, vl;
              if (first) {
                vh = __ldg(p.a_in + j);
                vl = 0.f;
              } else {
                const double a = __ldcg(p.a64 + j);
                vh = (float)a;
                vl = (float)(a - (double)vh);
              }
              // ph, pl: the Dot2 pair (s, c) of sum x·v
#pragma unroll
              for (int r = 0; r < 4; ++r) {
                const float pr = x[r] * vh, pe = fmaf(x[r], vh, -pr);
                const float t = ph[r] + pr, bb = t - ph[r];
                pl[r] += ((ph[r] - (t - bb)) + (pr - bb)) + pe;
                ph[r] = t;
                pl[r] = fmaf(x[r], vl, pl[r]);
              }
            }
          }
        });
        if (!ok) return false;
      }
      // the chunk's new residual: one reducer thread per row
      *reinterpret_cast<float4*>(red_h + warp * 128 + 4 * lane) = make_float4(ph[0], ph[1], ph[2], ph[3]);
      *reinterpret_cast<float4*>(red_l + warp * 128 + 4 * lane) = make_float4(pl[0], pl[1], pl[2], pl[3]);
      __syncthreads();
      if (tid < 128) {
        const int64_t row = rrow;
        float en = 0.f;
        if (row < m) {
          double e64;
          if (kind == PK_APPLY) {
            float sacc = 0.f;
#pragma unroll
            for (int w = 0; w < PNW; ++w) sacc += red_h[w * 128 + tid];
            en = e_in - sacc;
            e64 = (double)en;
          } else if (kind == PK_COPY_Y) {
            en = y_in;
            e64 = (double)en;
          } else {
            double tot = 0.0;
#pragma unroll
            for (int w = 0; w < PNW; ++w) tot += (double)red_h[w * 128 + tid] + (double)red_l[w * 128 + tid];
            e64 = (double)y_in - tot;
            en = (float)e64;
          }
          p.e[row] = en;
          e2 = fma(e64, e64, e2);
          if (first) y2 = fma((double)y_in, (double)y_in, y2);
        }
        ech[tid] = en;
      }
      __syncthreads();
      const float4 ev = *reinterpret_cast<const float4*>(ech + 4 * lane);
#pragma unroll
      for (int b = 0; b < NBP; ++b) {
        if (b >= nD) break;
        const bool ok = box((uint64_t)ci * bpc + nA + b, [&](const T* bx) {
#pragma unroll
          for (int c = 0; c < CWB; ++c) {
            float x[4];
            BoxRows4<T>::load(bx + (warp * CWB + c) * 128 + 4 * lane, x);
            gacc[b][c] = fmaf(x[0], ev.x, fmaf(x[1], ev.y, fmaf(x[2], ev.z, fmaf(x[3], ev.w, gacc[b][c]))));
          }
        });
        if (!ok) return false;
      }
      if (++since_flush == 8) {
        flush();
        since_flush = 0;
      }
    }
    if (since_flush) flush();
    qbase += total;
    {
      const int b = lane / CWB, c = lane % CWB;
      const int col = b * BC + warp * CWB + c;  // within the dot panel
      if (col < nd && nch > 0) atomicAdd(p.hacc + (size_t)hb * PW + col, acc64);
    }
    // the CTA's ||e||^2 (and ||y||^2) partials: the reducer threads' sums
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      e2 += __shfl_xor_sync(FULL_MASK, e2, o);
      y2 += __shfl_xor_sync(FULL_MASK, y2, o);
    }
    if (lane == 0 && warp < 4) {
      red[warp] = e2;
      red[4 + warp] = y2;
    }
    __syncthreads();
    if (tid == 0) {
      p.npart[(size_t)nb * G + blockIdx.x] = red[0] + red[1] + red[2] + red[3];
      if (first) p.ypart[blockIdx.x] = red[4] + red[5] + red[6] + red[7];
    }
    __syncthreads();
    return true;
  };
  auto pass = [&](int kind, int qp, int qd, int hb, int nb, bool first) -> bool {
    if constexpr (TMA) {
      if (!run_pass_tma(kind, qp, qd, hb, nb, first)) {
        tma_fail = true;
        return false;
      }
      return true;
    } else {
      run_pass(kind, qp, qd, hb, nb, first);
      return true;
    }
  };

  // After a pass's barrier: r = h ⊘ d of the dot panel, hacc[hb] left for the
  // next-but-one pass zeroed by CTA 0.
  auto take_dots = [&](int qd, int hb) {
    const int d0 = qd * PW, nd = min(PW, n - d0);
    if (tid < PW) {
      float r = 0.f;
      if (tid < nd) {
        const float dj = p.dvec[d0 + tid];
        if (dj > 0.f) r = (float)(__ldcg(p.hacc + (size_t)hb * PW + tid) / (double)dj);
      }
      r_s[tid] = r;
    }
    if (lead && tid < PW) p.hacc[(size_t)((hb + 2) % 3) * PW + tid] = 0.0;
    __syncthreads();
  };

  auto solve_panel = [&](int q) {
    const int q0 = q * PW, nq = min(PW, n - q0);
    panel_substitution(p.Gt + (size_t)q * PW * PW, nq, r_s, da_s);
    if (lead && tid < nq) p.a64[q0 + tid] += (double)da_s[tid];
  };

  int64_t t = 0;         // passes made
  int64_t s = 0;         // sweeps completed
  int status = HPSCD_ERR_NOT_CONVERGED;
  double r_prev = 0.0, r = 0.0, y2 = 0.0;
  int nconf = 0;
  bool stall = p.stall_barrier != 0;
  auto sync_grid = [&]() -> bool {
    const unsigned expect = G + (stall ? 1u : 0u);
    stall = false;
    if (!grid_barrier(p.ctl, expect, p.timeout_ns)) {
      err = DEV_TIMEOUT_BARRIER;
      return false;
    }
    return true;
  };

  // pass 0: the initial residual (y, or y - X·a0 of a warm start) and the
  // first panel's dot products
  bool done = !pass(p.warm ? PK_TRUE : PK_COPY_Y, 0, 0, 0, 0, true);
  if (!done && !sync_grid()) done = true;
  if (!done) {
    take_dots(0, 0);
    y2 = sum_partials(p.ypart, G, red);
    r = rel_of(sum_partials(p.npart, G, red), y2);
    if (lead && tid == 0) p.hist[0] = r;
    if (!isfinite(r)) {
      status = HPSCD_ERR_NONFINITE;
      done = true;
    } else if (p.max_sweeps == 0) {
      status = (p.stop_rule == HPSCD_STOP_REL_CHANGE || (p.stop_rule == HPSCD_STOP_REL_RES && r > p.tol))
                   ? HPSCD_ERR_NOT_CONVERGED
                   : HPSCD_OK;
      done = true;
    } else if (p.stop_rule == HPSCD_STOP_REL_RES && r <= p.tol) {
      status = HPSCD_OK;  // e_0 is a true residual already
      done = true;
    }
    r_prev = r;
  }
  int q = 0;  // the panel whose dot products are in r_s
  if (!done) solve_panel(q);
  while (!done) {
    ++t;
    const int qn = (q + 1) % npan;
    const bool boundary = qn == 0;
    const bool refresh = boundary && p.refresh_every > 0 && ((s + 1) % p.refresh_every) == 0;
    if (refresh && !sync_grid()) break;  // the coefficients of the last panel are visible
    const int hb = (int)(t % 3), nb = (int)(t & 1);
    if (!pass(refresh ? PK_TRUE : PK_APPLY, q, qn, hb, nb, false)) break;
    if (!sync_grid()) break;
    take_dots(qn, hb);
    q = qn;
    if (boundary) {
      ++s;
      r = rel_of(sum_partials(p.npart + (size_t)nb * G, G, red), y2);
      if (lead && tid == 0) p.hist[s] = r;
      if (!isfinite(r)) {
        status = HPSCD_ERR_NONFINITE;
        break;
      }
      bool met = false;
      if (p.stop_rule == HPSCD_STOP_REL_RES) met = r <= p.tol;
      else if (p.stop_rule == HPSCD_STOP_REL_CHANGE) met = r_prev == 0.0 || fabs(r_prev - r) < p.tol * r_prev;
      const bool last = s >= p.max_sweeps;
      if ((met || last) && p.stop_rule != HPSCD_STOP_NONE && nconf < 8) {
        // the stop is taken on y - X·a of the float32 coefficients returned
        ++nconf;
        if (lead)
          for (int j = tid; j < n; j += PNT) p.a64[j] = (double)(float)p.a64[j];
        if (!sync_grid()) break;
        ++t;
        const int hb2 = (int)(t % 3), nb2 = (int)(t & 1);
        if (!pass(PK_TRUE, 0, 0, hb2, nb2, false)) break;
        if (!sync_grid()) break;
        take_dots(0, hb2);
        r = rel_of(sum_partials(p.npart + (size_t)nb2 * G, G, red), y2);
        if (lead && tid == 0) p.hist[s] = r;
        if (!isfinite(r)) {
          status = HPSCD_ERR_NONFINITE;
          break;
        }
        if (p.stop_rule == HPSCD_STOP_REL_RES) met = r <= p.tol;
      }
      if (met || last) {
        status = (met || p.stop_rule == HPSCD_STOP_NONE) ? HPSCD_OK : HPSCD_ERR_NOT_CONVERGED;
        break;
      }
      r_prev = r;
    }
    solve_panel(q);
  }
  if (tma_fail) err = DEV_TIMEOUT_COPY;
  // copies still in flight land before the CTA retires
  if (TMA && tid == 0)
    for (uint64_t g = waited_g; g < issued_g; ++g)
      if (!mbar_wait_bounded(&full[g % nst], (uint32_t)((g / nst) & 1), p.timeout_ns)) break;
  if (err != DEV_OK && tid == 0) atomicCAS(&p.ctl->err, DEV_OK, err);
  if (lead) {
    __syncthreads();
    for (int j = tid; j < n; j += PNT) p.a_out[j] = (float)p.a64[j];
    if (tid == 0) {
      p.ctl->status = status;
      p.ctl->sweeps = s;
      p.ctl->final_res = r;
      p.ctl->passes = t + 1;
    }
  }
}

}  // namespace

// Dynamic shared memory of the TMA instantiation with nst stages.
int panel_tma_smem(int nst) { return nst * PANEL_BOX_BYTES + 2 * PNW * 128 * 4 + 128 * 4 + 8 * 8 + 1024; }

cudaError_t launch_invert_panel_diag(float* Gt, int npanels, cudaStream_t stream) {
  if (npanels <= 0) return cudaSuccess;
  invert_panel_diag_kernel<<<npanels * (PW / 32), 32, 0, stream>>>(Gt);
  return cudaGetLastError();
}

cudaError_t launch_panel_sweep(int dtype, const PanelParams& p, const CUtensorMap* tmap, int grid,
                               cudaStream_t stream) {
  PanelParams pp = p;
  CUtensorMap map;
  if (tmap) map = *tmap;
  else memset(&map, 0, sizeof(map));
  void* args[] = {(void*)&map, (void*)&pp};
  const bool tma = p.use_tma != 0 && tmap != nullptr;
  const void* kern;
  if (tma)
    kern = dtype == HPSCD_F32    ? (const void*)panel_sweep_kernel<float, true>
           : dtype == HPSCD_BF16 ? (const void*)panel_sweep_kernel<uint16_t, true>
                                 : (const void*)panel_sweep_kernel<__half, true>;
  else
    kern = dtype == HPSCD_F32    ? (const void*)panel_sweep_kernel<float, false>
           : dtype == HPSCD_BF16 ? (const void*)panel_sweep_kernel<uint16_t, false>
                                 : (const void*)panel_sweep_kernel<__half, false>;
  const int smem = tma ? panel_tma_smem(p.nstages) : 0;
  if (tma) {
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
  }
  return cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(PNT), args, (size_t)smem, stream);
}

}  // namespace hpscd
