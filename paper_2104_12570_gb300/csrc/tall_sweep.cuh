#pragma once
// Persistent column sweep of Algorithm 1 for tall and square systems
// (column-major X, n <= 512), one CTA per SM, cooperative launch.
//
// Algorithm 1 makes column j's step depend on the residual left by column
// j-1, through a reduction over all m rows.  Writing e_s for the residual
// after sweep s and g_s = X^T e_s, Eq. ek1-ek gives, just before column j of
// sweep s+1,
//     <X_j, e> = g_{s,j} - sum_{l<j} <X_j, X_l> da_l,
// so the whole sweep's steps follow from g_s and the lower triangle of
// G = X^T X by forward substitution, in the paper's column order:
//     da_j = (g_{s,j} - sum_{l<j} G_jl da_l) / G_jj      (Eq. da2, the ⊘ step)
// followed by e_{s+1} = e_s - X·da (the sweep's n rank-1 corrections, Eq.
// ek1-ek) and a <- a + da.  In exact arithmetic this is Algorithm 1 step for
// step.  One streaming pass over X per sweep carries all of the sweep's dot
// products and rank-1 corrections:
//
//   pass p reads X once and, row panel by row panel, forms
//       e_out = e_in - X·v        (v = da_p; on a true-residual pass
//                                  e_out = y - X·a_p instead)
//       h     = X^T e_in          (against the residual the pass starts from)
//       ||e_out||^2 in float64;
//   the CTAs add their partials of h into one float64 vector (atomics) and
//   publish their ||e||^2 partials; grid barrier; every CTA reads the same h
//   and sums the norm partials in a fixed order (bitwise identical in every
//   CTA), records hist[p] = ||e_p|| / ||y||, tests the stopping rule, forms
//       r = h ⊘ d - G~·da_p       (= (X^T e_p) ⊘ d by Eq. ek1-ek; d = diag(G),
//                                  G~ = D^{-1} G, the ⊘ step applied once to
//                                  the couplings in set-up)
//   and runs the forward substitution da_j = r_j - sum_{l<j} G~_jl da_l for
//   da_{p+1}, which has no division on its dependency chain.
// Pass 0 starts from e_in = y (h = X^T y) with v = a_0 (or nothing).
//
// Taking the dots against e_in rather than e_out makes the two halves of a
// pass independent, so X streams through shared memory by TMA in chunks of
// 128 rows × C columns (512 contiguous bytes per column for float32; TMA
// zero-fills past m and n) with a full/empty mbarrier pair per stage and one
// CTA barrier per 128-row panel.  Each warp owns C/16 columns of every chunk
// and each lane 4 consecutive rows: the lane keeps its partial X^T e for its
// columns in registers for the whole pass, and its partial row sums of X·v
// for the panel, which a cross-warp reduction turns into the panel's e_out.
#include <cuda_fp16.h>

#include "kernels.h"

namespace hpscd {

namespace {

constexpr int NW = 16;          // warps
constexpr int NT = NW * 32;     // threads
constexpr int DIAG_PACK = 32 * 31 / 2;  // strictly lower entries of a 32x32 block

template <typename T>
__device__ __forceinline__ T zero_elem();
template <>
__device__ __forceinline__ float zero_elem<float>() { return 0.f; }
template <>
__device__ __forceinline__ uint16_t zero_elem<uint16_t>() { return 0; }
template <>
__device__ __forceinline__ __half zero_elem<__half>() { return __ushort_as_half((unsigned short)0); }

// Row segment of the couplings of one step to the 32 steps of a block, for a
// given column order: g[k] = row[oc[k]] (oc: the block's columns), 0 past lim.
__device__ __forceinline__ void gather_seg32(const float* __restrict__ row, const int* oc, int lim,
                                             float (&g)[32]) {
#pragma unroll
  for (int k = 0; k < 32; ++k) g[k] = (k < lim) ? __ldg(row + oc[k]) : 0.f;
}

__device__ __forceinline__ void load_seg32(const float* __restrict__ src, float (&g)[32]) {
  const float4* row = reinterpret_cast<const float4*>(src);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float4 t = __ldg(row + q);
    g[4 * q] = t.x; g[4 * q + 1] = t.y; g[4 * q + 2] = t.z; g[4 * q + 3] = t.w;
  }
}

// Forward substitution of one sweep (see the file comment):
//   da_j = r_j - sum_{l<j} G~_jl da_l, j = 0..n-1 (r = g ⊘ d; da_j = 0 when d_j = 0,
//   where row j of G~ is zero).
// Blocks of 32 columns.  Warp 0 walks each diagonal block with shuffles,
// reading the block's strictly lower triangle from shared memory (diag_s,
// packed, staged once per launch); thread t >= 32 owns row t and applies each
// finished block to it, loading its G~ segment for the next block right after
// using the current one, so the load overlaps the next block's walk.  r (in:
// g ⊘ d, overwritten) and da are shared arrays of length npad.
// With thr > 1 (Algorithm 2) the couplings of a row to the columns of its own
// block of thr columns are dropped: row t keeps columns l < (t / thr)·thr.
__device__ __forceinline__ void mask_seg32(float (&g)[32], int t, int b0, int thr) {
  if (thr <= 1) return;
  const int lim = (t / thr) * thr - b0;
#pragma unroll
  for (int k = 0; k < 32; ++k) g[k] = (k < lim) ? g[k] : 0.f;
}

__device__ __forceinline__ int ld_acquire_cta(const int* p) {
  int v;
  asm volatile("ld.acquire.cta.shared::cta.s32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_cta(int* p, int v) {
  asm volatile("st.release.cta.shared::cta.s32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}
// Lane 0 waits (bounded) until *flag >= want, then the warp proceeds together.
// Returns false when the wait gave up.
__device__ __forceinline__ bool warp_wait_flag(const int* flag, int want, uint64_t timeout_ns) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) {
    // the hand-offs of the substitution take well under a microsecond: spin
    // without the timer first, then bound the wait by the timeout
    uint32_t spin = 0;
    while (spin < 4096 && ld_acquire_cta(flag) < want) ++spin;
    if (spin == 4096) {
      const uint64_t t0 = global_timer_ns();
      for (uint32_t it = 0;; ++it) {
        if (ld_acquire_cta(flag) >= want) break;
        if ((it & 63) == 63 && global_timer_ns() - t0 > timeout_ns) { ok = 0; break; }
      }
    }
  }
  ok = __shfl_sync(FULL_MASK, ok, 0);
  __syncwarp();
  return ok != 0;
}

// Forward substitution of one sweep (see the file comment):
//   da_j = r_j - sum_{l<j} G~_jl da_l, j = 0..n-1 (r = g ⊘ d; da_j = 0 when d_j = 0,
//   where row j of G~ is zero).
// Dataflow over blocks of 32 columns, no CTA barrier between blocks: warp w
// owns rows 32w..32w+31.  Warp 0 solves block c as soon as warp c has applied
// blocks 0..c-1 to its rows (da_c = M_c r_c with the block's inverse
// M_c = (I + L_c)^{-1} in diag_s: 32 independent shuffles; formed once per
// launch, or every sweep for a given column order, whose blocks change with
// the order), then publishes da of the block; every warp w
// applies each published block b < w to its rows (its G~ segment of block b+1
// loaded while it waits) and, after block w-1, signals warp 0.  The critical
// path is one block's solve plus one hand-off per block.  With thr > 1
// (Algorithm 2) the couplings inside a block of thr columns are masked.
// flags: [0] blocks solved, [1 + w] warp w's rows ready; r (in: g ⊘ d) and da
// are shared arrays of length npad.  Returns false when a wait gave up.
// ORD: the unknowns are the steps of a given column order (o: step -> column,
// shared, -1 past n): step t couples to earlier step l through G~[o_t][o_l];
// diag_s then holds the gathered diagonal blocks of this sweep.
template <bool ORD>
__device__ bool forward_substitution(const float* __restrict__ Gt, int ldG, int n, int npad,
                                     float* r, float* da, const float* diag_s, int thr,
                                     int* flags, uint64_t timeout_ns, const int* o = nullptr) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int c = n + tid; c < npad; c += NT) da[c] = 0.f;
  if (tid <= NW) flags[tid] = 0;
  named_sync(NT);  // r (written by the caller) and the cleared flags are visible
  if (n <= 0) return true;
  const int nb = (n + 31) / 32;
  bool ok = true;
  if (warp == 0) {
    for (int b = 0; b < nb && ok; ++b) {
      const int i = 32 * b + lane;
      float seg[32];
      const float* dl = diag_s + b * DIAG_PACK + (lane * (lane - 1)) / 2;
#pragma unroll
      for (int k = 0; k < 32; ++k) seg[k] = (k < lane) ? dl[k] : 0.f;
      if (b > 0 && !warp_wait_flag(&flags[1 + b], 1, timeout_ns)) { ok = false; break; }
      float ri = (i < n) ? r[i] : 0.f;
      // diag_s: the strictly lower part of M_b = (I + L_b)^{-1}, so the block's
      // da = M_b r takes 32 independent shuffles instead of a dependent walk
      float acc[4] = {ri, 0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < 32; ++k) acc[k & 3] = fmaf(seg[k], __shfl_sync(FULL_MASK, ri, k), acc[k & 3]);
      ri = (acc[0] + acc[1]) + (acc[2] + acc[3]);
      if (i < npad) da[i] = (i < n) ? ri : 0.f;
      __syncwarp();
      if (lane == 0) st_release_cta(&flags[0], b + 1);
    }
  } else if (warp < nb) {
    const int t = tid;
    float rt = (t < n) ? r[t] : 0.f;
    float seg[32];
    const float* grow = Gt + (int64_t)(t < n ? (ORD ? o[t] : t) : 0) * ldG;
    if constexpr (ORD) {
      gather_seg32(grow, o, n, seg);
    } else {
      load_seg32(grow, seg);
      mask_seg32(seg, t, 0, thr);
    }
    for (int b = 0; b < warp; ++b) {
      if (!warp_wait_flag(&flags[0], b + 1, timeout_ns)) { ok = false; break; }
      const float4* dab = reinterpret_cast<const float4*>(da + 32 * b);
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
      for (int k = 0; k < 32; k += 4) {
        const float4 d4 = dab[k / 4];
        a0 = fmaf(seg[k], d4.x, a0);
        a1 = fmaf(seg[k + 1], d4.y, a1);
        a2 = fmaf(seg[k + 2], d4.z, a2);
        a3 = fmaf(seg[k + 3], d4.w, a3);
      }
      rt -= (a0 + a1) + (a2 + a3);
      if (b + 1 < warp) {
        if constexpr (ORD) {
          gather_seg32(grow, o + 32 * (b + 1), n - 32 * (b + 1), seg);
        } else {
          load_seg32(grow + 32 * (b + 1), seg);
          mask_seg32(seg, t, 32 * (b + 1), thr);
        }
      }
    }
    if (t < npad) r[t] = rt;
    __syncwarp();
    if (lane == 0) st_release_cta(&flags[1 + warp], 1);
  }
  return named_sync_or(NT, ok ? 0 : 1) == 0;  // da complete (or a wait gave up)
}

// diag_s holds, per 32-column block b, the strictly lower triangle L_b of the
// unit lower triangular diagonal block I + L_b of G~ (packed by rows).  Replaced
// in place by the strictly lower triangle of M_b = (I + L_b)^{-1}, again unit
// lower triangular, so the substitution of a block becomes a product with M_b
// (the same da in exact arithmetic).  Warp w takes blocks w, w + NW, ...; lane j
// forms column j: M_ij = -sum_{k<i} L_ik M_kj for i > j, in float32.
__device__ void invert_diag_blocks(float* diag_s, int nb) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int b = warp; b < nb; b += NW) {
    float* blk = diag_s + b * DIAG_PACK;
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

// Algorithm 3's step (Sec. 8): with r = (X^T e) ⊘ d (every column's da against
// the same residual), E_j = ||e - X_j da_j||^2 = ||e||^2 - r_j^2 d_j, so the
// column of least error is the one of largest r_j^2 d_j (ties: lowest j).  The
// step adds only that column: da = r_jhat at jhat, 0 elsewhere.  Returns jhat.
__device__ int select_step(int n, int npad, const float* r, const float* d, float* da,
                           float* fscr, int* iscr) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  float best = -1.f;
  int bj = 0x7fffffff;
  for (int c = tid; c < n; c += NT) {
    const float sc = d[c] > 0.f ? r[c] * r[c] * d[c] : 0.f;
    if (sc > best || (sc == best && c < bj)) { best = sc; bj = c; }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float ob = __shfl_xor_sync(FULL_MASK, best, off);
    const int oj = __shfl_xor_sync(FULL_MASK, bj, off);
    if (ob > best || (ob == best && oj < bj)) { best = ob; bj = oj; }
  }
  if (lane == 0) { fscr[warp] = best; iscr[warp] = bj; }
  named_sync(NT);
  best = fscr[0];
  bj = iscr[0];
  for (int w = 1; w < NW; ++w)
    if (fscr[w] > best || (fscr[w] == best && iscr[w] < bj)) { best = fscr[w]; bj = iscr[w]; }
  if (bj >= n) bj = 0;
  for (int c = tid; c < npad; c += NT) da[c] = (c == bj && n > 0) ? r[c] : 0.f;
  named_sync(NT);
  return bj;
}

// A swap step of the feature-removal loop (Sec. 8), after the selection steps:
// over the selected columns k (a_k != 0) and the others j (d_j > 0), the error
// after dropping k and refitting j on the residual without it is
//   E_kj = ||e||^2 + 2 a_k h_k + a_k^2 d_k - t^2 / d_j,  t = h_j + a_k G_jk,
// with h = X^T e = r·d and G_jk = G~_kj·d_k (row k of G~).  Thread j scores its
// column against every k; a block argmin (lowest k, then j, on ties) picks the
// pair.  When E < ||e||^2 the step's update is da_k = -a_k, da_j = t / d_j and
// the function returns k (and j through *jout); otherwise it returns -1.
// ks: shared int scratch of npad entries (the selected columns); fscr/iscr: as
// select_step (fscr holds doubles here, 2·NW of them).
__device__ int swap_step(int n, int npad, const float* r, const float* d, const double* a64,
                         const float* __restrict__ Gt, int ldG, double ee, float* da, int* ks,
                         double* fscr, int* iscr, int* jout) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    int c = 0;
    for (int k = 0; k < n; ++k)
      if (a64[k] != 0.0) ks[1 + c++] = k;
    ks[0] = c;
  }
  named_sync(NT);
  const int ns = ks[0];
  double best = 0.0;
  int bk = 0x7fffffff, bj = 0x7fffffff;
  for (int j = tid; j < n; j += NT) {
    const double dj = (double)d[j];
    if (a64[j] != 0.0 || !(dj > 0.0)) continue;
    const double hj = (double)r[j] * dj;
    for (int q = 0; q < ns; ++q) {
      const int k = ks[1 + q];
      const double ak = a64[k], dk = (double)d[k];
      const double hk = (double)r[k] * dk;
      const double t = hj + ak * ((double)__ldg(Gt + (int64_t)k * ldG + j) * dk);
      const double E = ee + 2.0 * ak * hk + ak * ak * dk - t * t / dj;
      if (bk == 0x7fffffff || E < best || (E == best && (k < bk || (k == bk && j < bj)))) {
        best = E; bk = k; bj = j;
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double ob = __shfl_xor_sync(FULL_MASK, best, off);
    const int ok = __shfl_xor_sync(FULL_MASK, bk, off);
    const int oj = __shfl_xor_sync(FULL_MASK, bj, off);
    if (ok != 0x7fffffff &&
        (bk == 0x7fffffff || ob < best || (ob == best && (ok < bk || (ok == bk && oj < bj))))) {
      best = ob; bk = ok; bj = oj;
    }
  }
  if (lane == 0) { fscr[warp] = best; iscr[warp] = bk; iscr[NW + warp] = bj; }
  named_sync(NT);
  best = fscr[0]; bk = iscr[0]; bj = iscr[NW];
  for (int w = 1; w < NW; ++w) {
    const int ok = iscr[w], oj = iscr[NW + w];
    if (ok != 0x7fffffff &&
        (bk == 0x7fffffff || fscr[w] < best || (fscr[w] == best && (ok < bk || (ok == bk && oj < bj))))) {
      best = fscr[w]; bk = ok; bj = oj;
    }
  }
  const bool take = bk != 0x7fffffff && best < ee;
  double delta = 0.0;
  if (take) {
    const double dk = (double)d[bk], dj = (double)d[bj];
    delta = ((double)r[bj] * dj + a64[bk] * ((double)__ldg(Gt + (int64_t)bk * ldG + bj) * dk)) / dj;
  }
  for (int c = tid; c < npad; c += NT)
    da[c] = !take ? 0.f : (c == bk ? (float)(-a64[bk]) : (c == bj ? (float)delta : 0.f));
  named_sync(NT);
  *jout = take ? bj : -1;
  return take ? bk : -1;
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

template <typename T>
struct Row4;
template <>
struct Row4<float> {
  __device__ static void load(const float* p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
};
template <>
struct Row4<uint16_t> {
  __device__ static void load(const uint16_t* p, float (&v)[4]) {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    v[0] = __uint_as_float(t.x << 16);
    v[1] = __uint_as_float(t.x & 0xffff0000u);
    v[2] = __uint_as_float(t.y << 16);
    v[3] = __uint_as_float(t.y & 0xffff0000u);
  }
};
template <>
struct Row4<__half> {
  __device__ static void load(const __half* p, float (&v)[4]) {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&t.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&t.y));
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

constexpr int PR = 128;  // rows per panel (and per chunk)
constexpr int TRACE_FIELDS = 6;

// Neumaier-compensated float32 accumulation: s + c carries the sum of the
// added terms to about twice float32 precision, without float64 arithmetic
// (float64 throughput is low on this part).
__device__ __forceinline__ void comp_add(float x, float& s, float& c) {
  const float t = s + x;
  c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
  s = t;
}

// One chunk's work for one warp: lane partials of X^T e_in for the warp's
// columns (phase B) and, unless the pass only copies y, the lane's partial row
// sums of X·v (phase A).  On a true-residual pass v = a_hi + a_lo (vsm / vreg
// hold a_hi = fl32(a), vlo holds a_lo = fl32(a - a_hi)): X·a_hi is summed as
// Dot2 pairs and X·a_lo, 2^-24 smaller, is added to the pair's low part.
template <int MODE, typename T, int CW, int CPW, bool VREG>
__device__ __forceinline__ void chunk_compute(const T* __restrict__ st, int warp, int lane,
                                              int ch, const float (&ein)[4],
                                              float (&gacc)[CPW], const float (&vreg)[VREG ? CPW : 1],
                                              const float* __restrict__ vsm,
                                              const float* __restrict__ vlo, float (&ph)[4],
                                              float (&pl)[4]) {
  constexpr int C = NW * CW;
#pragma unroll
  for (int jj = 0; jj < CW; ++jj) {
    const int j = ch * CW + jj;
    float xv[4];
    Row4<T>::load(st + (warp * CW + jj) * PR + 4 * lane, xv);
#pragma unroll
    for (int r = 0; r < 4; ++r) gacc[j] = fmaf(xv[r], ein[r], gacc[j]);
    if constexpr (MODE != MODE_COPY) {
      float vk;
      if constexpr (VREG) vk = vreg[j];
      else vk = vsm[ch * C + warp * CW + jj];
      float vl = 0.f;
      if constexpr (MODE == MODE_REFRESH) vl = vlo[ch * C + warp * CW + jj];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if constexpr (MODE == MODE_NORMAL) {
          ph[r] = fmaf(xv[r], vk, ph[r]);
        } else {
          dot2_step(xv[r], vk, ph[r], pl[r]);
          pl[r] = fmaf(xv[r], vl, pl[r]);
        }
      }
    }
  }
}

// KMODE 0: the sweep (Algorithm 1, or Algorithm 2 with thr); 1: a given column
// order per sweep (float32); 2: greedy selection (Algorithm 3) and its swap steps.
// Separate instantiations keep each mode's code out of the others.
template <typename T, int CW, int NCH, int KMODE>
__global__ void __launch_bounds__(NT, 1)
    tall_sweep_kernel(const __grid_constant__ CUtensorMap tmap, const TallParams p) {
  constexpr bool ORD = KMODE == 1;
  constexpr bool SEL = KMODE == 2;
  constexpr int C = NW * CW;          // columns per chunk
  constexpr int NPAD = C * NCH;       // padded column count
  constexpr int CPW = CW * NCH;       // columns per warp over a whole row
  constexpr int CHUNK_ELEMS = PR * C;
  constexpr bool V_IN_REGS = CPW <= 8;

  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nst = p.nstages;
  T* stages = reinterpret_cast<T*>(base);
  float* red_hi = reinterpret_cast<float*>(base + (size_t)nst * CHUNK_ELEMS * sizeof(T));
  float* red_lo = red_hi + 2 * NW * PR;  // [2][NW][PR] each
  float* rvec = red_lo + 2 * NW * PR;
  float* da_s = rvec + NPAD;
  float* dd_s = da_s + NPAD;
  float* vsm = dd_s + NPAD;
  float* vlo = vsm + NPAD;      // a_lo of a true-residual pass (0 otherwise)
  double* a64_s = reinterpret_cast<double*>(vlo + NPAD);
  double* scal = a64_s + NPAD;  // [0]: ||e||^2, [1]: ||y||^2, [2..33]: scratch
  uint64_t* full = reinterpret_cast<uint64_t*>(scal + 40);
  uint64_t* empty = full + 16;
  int* flags = reinterpret_cast<int*>(empty + 16);  // [1]: grid barrier result
  float* diag_s = reinterpret_cast<float*>(flags + 4);  // [max(1, NPAD/32)][DIAG_PACK]
  // with p.e_smem: e of the CTA's row panels, [panels of this CTA][PR]
  float* e_res = reinterpret_cast<float*>(
      (reinterpret_cast<uintptr_t>(diag_s + (NPAD >= 32 ? NPAD / 32 : 1) * DIAG_PACK) + 15) & ~uintptr_t(15));

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int grid = gridDim.x;
  const int64_t npanels = p.ntiles;
  const int64_t pn0 = npanels * blockIdx.x / grid;
  const int64_t pn1 = npanels * (blockIdx.x + 1) / grid;
  const int64_t npan = pn1 - pn0;
  const uint64_t nchunk = (uint64_t)npan * NCH;  // chunks per pass
  const bool tma = p.use_tma != 0;
  const int64_t m = p.m;
  const int n = p.n;

  if (tid == 0) {
    if (tma) {
      for (int s = 0; s < nst; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], NW); }
      fence_mbar_init();
    }
  }
  for (int c = tid; c < NPAD; c += NT) {
    a64_s[c] = (c < n && p.warm) ? (double)p.a_in[c] : 0.0;
    dd_s[c] = (c < n) ? p.dvec[c] : 0.f;
    da_s[c] = 0.f;
    vlo[c] = 0.f;
  }
  for (int idx = tid; idx < ((n + 31) / 32) * DIAG_PACK; idx += NT) {
    const int b = idx / DIAG_PACK, q = idx % DIAG_PACK;
    int i = 1;
    while ((i * (i + 1)) / 2 <= q) ++i;
    const int k = q - (i * (i - 1)) / 2;
    // Algorithm 2 drops the couplings inside a block of thr columns
    const bool keep = p.thr <= 1 || 32 * b + k < ((32 * b + i) / p.thr) * p.thr;
    diag_s[idx] = (32 * b + i < n && keep) ? p.Gt[(int64_t)(32 * b + i) * p.ldG + 32 * b + k] : 0.f;
  }
  __syncthreads();
  if constexpr (!SEL) {  // a given column order (ORD) regathers and inverts every sweep
    invert_diag_blocks(diag_s, (n + 31) / 32);
    __syncthreads();
  }

  // ---------------- TMA issue (thread 0) ----------------
  // chunk sequence q = pass·nchunk + panel·NCH + ch, periodic over passes;
  // stage q % nst.  The first nst chunks are issued up front; after the CTA
  // barrier that ends chunk q, thread 0 issues chunk q + nst into its stage.
  uint64_t issued = 0, waited = 0;
  auto issue_chunk = [&](uint64_t k) {
    const int s = (int)(k % nst);
    const uint64_t kp = k % nchunk;
    const int64_t panel = pn0 + (int64_t)(kp / NCH);
    const int ch = (int)(kp % NCH);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&full[s], CHUNK_ELEMS * sizeof(T));
    tma_load_2d(stages + (size_t)s * CHUNK_ELEMS, &tmap, &full[s], (int32_t)(panel * PR), ch * C);
  };
  if (tma && tid == 0 && nchunk > 0)
    while (issued < (uint64_t)nst) issue_chunk(issued++);

  // ---------------- compute warps ----------------
  for (int c = tid; c < NPAD; c += NT) vsm[c] = (float)a64_s[c];
  named_sync(NT);
  float v[V_IN_REGS ? CPW : 1];
  if constexpr (V_IN_REGS) {
#pragma unroll
    for (int j = 0; j < CPW; ++j) v[j] = vsm[(j / CW) * C + warp * CW + (j % CW)];
  }
  float gacc[CPW];
#pragma unroll
  for (int j = 0; j < CPW; ++j) gacc[j] = 0.f;

  int err = DEV_OK;
  int status = HPSCD_ERR_NOT_CONVERGED;
  double r_prev = 0.0, ynorm = 0.0;
  int64_t pass = 0, sweeps = 0;
  int64_t sw = 0;          // sweeps (or selection steps) reflected in the residual of a pass
  // what the next pass is: 0 a sweep, 1 a confirmation (no step), 2 the
  // predicted last sweep, whose pass forms the true residual
  int next_kind = 0;
  uint64_t qbase = 0;

  // optional trace: CTA 0 records, per pass, the global time at the start of
  // the pass, end of streaming, end of the grid barrier, end of the partial-sum
  // reduction, end of G·da and end of the forward substitution; every CTA
  // records the end of its streaming in pass 1 (load balance).
  unsigned long long* tr = (p.trace && blockIdx.x == 0 && tid == 0) ? p.trace : nullptr;
  auto stamp = [&](int64_t ps, int k) {
    if (tr && ps < p.trace_passes) tr[ps * TRACE_FIELDS + k] = global_timer_ns();
  };
  // A cold start whose X^T y and ||y||^2 the set-up formed (p.h0) makes pass 0
  // virtual: e_0 = y is not materialised and the first streamed pass reads y.
  // A confirmation pass (REL_RES with p.confirm) follows a pass whose tracked
  // residual met the tolerance: it recomputes e = y - X·a for the float32
  // coefficients that would be returned, and the rule is tested on that.
  for (pass = 0;; ++pass) {
    stamp(pass, 0);
    const bool conf = next_kind == 1;
    const bool fin = next_kind == 2;
    next_kind = 0;
    if (pass > 0 && !conf) ++sw;
    const bool virt = pass == 0 && p.h0 != nullptr && !p.warm;
    const int mode = (pass == 0) ? (p.warm ? MODE_REFRESH : MODE_COPY)
                     : (conf || fin || (p.refresh_every > 0 && sw % p.refresh_every == 0))
                         ? MODE_REFRESH
                         : MODE_NORMAL;
    // the residual the pass starts from (y until a pass has written e), at row
    // `row`, local index `li` among the CTA's rows
    // (e_rows: the shared-memory copy indexed by the row itself, a generic pointer)
    const bool from_y = pass == 0 || (pass == 1 && p.h0 && !p.warm);
    float* const e_rows = p.e_smem ? e_res - pn0 * PR : p.e;
    const float* __restrict__ ein_src = from_y ? p.y : e_rows;
    const int buf = (int)(pass & 1);
    const int hb = (int)(pass % 3);
    double nrm = 0.0, ysq = 0.0;
    bool ok = true;
    if (!virt) {
    float ein[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int64_t row = pn0 * PR + 4 * lane + r;
      ein[r] = (npan > 0 && row < m) ? ein_src[row] : 0.f;
    }
    for (int64_t pi = 0; pi < npan; ++pi) {
      const int64_t rbase = (pn0 + pi) * PR;
      // reducer inputs of this panel and residual rows of the next, loaded early
      const int rr = tid - (NT - PR);  // reducer rows are owned by the last PR/32 warps
      const int64_t rrow = rbase + rr;
      float red_ein = 0.f, red_y = 0.f;
      if (rr >= 0 && rrow < m) {
        if (mode != MODE_COPY) red_ein = ein_src[rrow];
        if (mode != MODE_NORMAL) red_y = p.y[rrow];
      }
      float ein_next[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int64_t row = rbase + PR + 4 * lane + r;
        ein_next[r] = (pi + 1 < npan && row < m) ? ein_src[row] : 0.f;
      }
      float ph[4] = {0.f, 0.f, 0.f, 0.f}, pl[4] = {0.f, 0.f, 0.f, 0.f};
      const int rb = (int)(pi & 1);
      bool fail = false;
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) {
        const uint64_t q = qbase + (uint64_t)pi * NCH + ch;
        const int s = (int)(q % nst);
        T* st = stages + (size_t)s * CHUNK_ELEMS;
        if (tma) {
          if (ok && !mbar_wait_bounded(&full[s], (uint32_t)((q / nst) & 1), p.timeout_ns)) ok = false;
        } else {
          const T* X = reinterpret_cast<const T*>(p.X);
          for (int idx = tid; idx < CHUNK_ELEMS; idx += NT) {
            const int c = idx / PR, r = idx % PR;
            const int64_t gr = rbase + r;
            const int gc = ch * C + c;
            st[idx] = (gr < m && gc < n) ? X[(int64_t)gc * p.ld + gr] : zero_elem<T>();
          }
          named_sync(NT);
        }
        if (ok) {
          if (mode == MODE_NORMAL)
            chunk_compute<MODE_NORMAL, T, CW, CPW, V_IN_REGS>(st, warp, lane, ch, ein, gacc, v, vsm, vlo, ph, pl);
          else if (mode == MODE_REFRESH)
            chunk_compute<MODE_REFRESH, T, CW, CPW, V_IN_REGS>(st, warp, lane, ch, ein, gacc, v, vsm, vlo, ph, pl);
          else
            chunk_compute<MODE_COPY, T, CW, CPW, V_IN_REGS>(st, warp, lane, ch, ein, gacc, v, vsm, vlo, ph, pl);
        }
        if (ch == NCH - 1) {
          // the panel's row sums go to the cross-warp reduction buffer
          float* rh = red_hi + (rb * NW + warp) * PR + 4 * lane;
          *reinterpret_cast<float4*>(rh) = make_float4(ph[0], ph[1], ph[2], ph[3]);
          if (mode == MODE_REFRESH) {
            float* rl = red_lo + (rb * NW + warp) * PR + 4 * lane;
            *reinterpret_cast<float4*>(rl) = make_float4(pl[0], pl[1], pl[2], pl[3]);
          }
        }
        // every warp is done with chunk q (and, after the last chunk, has written its row sums)
        if (named_sync_or(NT, ok ? 0 : 1)) { fail = true; break; }
        if (tma && tid == 0) {
          ++waited;
          issue_chunk(issued++);  // chunk q + nst into the stage just released
        }
      }
      if (fail) { err = DEV_TIMEOUT_COPY; break; }
      if (rr >= 0 && rrow < m) {
        float e_new;
        double e64 = 0.0;
        if (mode == MODE_NORMAL) {
          float sacc = 0.f;
#pragma unroll
          for (int w = 0; w < NW; ++w) sacc += red_hi[(rb * NW + w) * PR + rr];
          e_new = red_ein - sacc;
        } else if (mode == MODE_COPY) {
          e_new = red_y;
        } else {
          // sum of the 16 (hi, lo) warp pairs, compensated; y - sum in float64
          float sh = 0.f, sc = 0.f, sl = 0.f;
#pragma unroll
          for (int w = 0; w < NW; ++w) {
            comp_add(red_hi[(rb * NW + w) * PR + rr], sh, sc);
            sl += red_lo[(rb * NW + w) * PR + rr];
          }
          e64 = ((double)red_y - (double)sh) - ((double)sc + (double)sl);
          e_new = (float)e64;
        }
        e_rows[rrow] = e_new;
        // a true-residual pass takes the norm of y - X·a before e is rounded to float32
        if (mode != MODE_REFRESH) e64 = (double)e_new;
        nrm = fma(e64, e64, nrm);
        if (pass == 0) ysq = fma((double)red_y, (double)red_y, ysq);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) ein[r] = ein_next[r];
    }
    if (err != DEV_OK) break;
    qbase += nchunk;
    stamp(pass, 1);
    if (p.trace && pass == 1 && tid == 0)
      p.trace[(int64_t)p.trace_passes * TRACE_FIELDS + blockIdx.x] = global_timer_ns();

    // publish this CTA's partials: h into hacc[pass % 3] (float64 atomics),
    // G~·w rows into gw[pass % 2], ||e||^2 into npart[pass % 2]
    // this CTA's rows of G~·w (w = da_p, or a_0 on a warm pass 0), one warp per
    // row c = blockIdx.x + k·grid; the rows are spread over the CTAs and
    // published with the partials, so after the barrier r costs n loads
    if (pass > 0 || p.warm) {
      const float* w = (pass == 0) ? vsm : da_s;
      for (int c = blockIdx.x + warp * grid; c < n; c += NW * grid) {
        const float* grow = p.Gt + (int64_t)c * p.ldG;
        float acc = 0.f;
        for (int l = lane; l < n; l += 32) acc = fmaf(__ldg(grow + l), w[l], acc);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(FULL_MASK, acc, off);
        if (lane == 0) p.gw[(size_t)buf * NPAD + c] = acc;
      }
    }
#pragma unroll
    for (int j = 0; j < CPW; ++j) {
      float sacc = gacc[j];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) sacc += __shfl_xor_sync(FULL_MASK, sacc, off);
      const int c = (j / CW) * C + warp * CW + (j % CW);
      if (lane == 0 && c < n) atomicAdd(p.hacc + (size_t)hb * NPAD + c, (double)sacc);
      gacc[j] = 0.f;
    }
    if (warp >= NW - PR / 32) {
      const int rw = warp - (NW - PR / 32);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        nrm += __shfl_xor_sync(FULL_MASK, nrm, off);
        ysq += __shfl_xor_sync(FULL_MASK, ysq, off);
      }
      if (lane == 0) { scal[2 + rw] = nrm; scal[2 + 16 + rw] = ysq; }
    }
    named_sync(NT);
    if (tid == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < PR / 32; ++w) { a += scal[2 + w]; b += scal[2 + 16 + w]; }
      p.npart[(size_t)buf * grid + blockIdx.x] = a;
      if (pass == 0) p.ypart[blockIdx.x] = b;
    }
    // the test hook stalls the first grid barrier taken (pass 1 when pass 0 is virtual)
    const int64_t first_barrier = (p.h0 && !p.warm) ? 1 : 0;
    const unsigned expected = (unsigned)grid + ((p.stall_barrier && pass == first_barrier) ? 1u : 0u);
    if (!grid_barrier_named(p.ctl, expected, p.timeout_ns, NT, &flags[1])) {
      err = DEV_TIMEOUT_BARRIER;
      break;
    }
    stamp(pass, 2);

    // every CTA: r = h ⊘ d - G~·w from the accumulated h (the same values in
    // every CTA); CTA 0 clears the h buffer of pass + 2, which no CTA reads any
    // more (its readers passed this barrier) and none adds to before the next one
    if (blockIdx.x == 0)
      for (int c = tid; c < NPAD; c += NT) p.hacc[(size_t)((pass + 2) % 3) * NPAD + c] = 0.0;
    }  // !virt
    if (tid < NPAD) {
      float rv = 0.f;
      if (tid < n && dd_s[tid] > 0.f) {
        if (virt) {
          rv = (float)(__ldg(p.h0 + tid) / (double)dd_s[tid]);
        } else {
          const double hd = __ldcg(p.hacc + (size_t)hb * NPAD + tid);
          const double gwc = (pass > 0 || p.warm) ? (double)__ldcg(p.gw + (size_t)buf * NPAD + tid) : 0.0;
          rv = (float)(hd / (double)dd_s[tid] - gwc);
        }
      }
      rvec[tid] = rv;
    }
    if (warp == 0 && virt) {
      if (lane == 0) { const double y2 = __ldg(p.y2); scal[0] = y2; scal[1] = y2; }
    } else if (warp == 0) {
      // at most 8 CTAs per lane (grid <= 256); loads issued together
      double av[8], bv[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int blk = lane + 32 * k;
        av[k] = blk < grid ? __ldcg(p.npart + (size_t)buf * grid + blk) : 0.0;
        bv[k] = (pass == 0 && blk < grid) ? __ldcg(p.ypart + blk) : 0.0;
      }
      double a = 0.0, b = 0.0;
#pragma unroll
      for (int k = 0; k < 8; ++k) { a += av[k]; b += bv[k]; }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(FULL_MASK, a, off);
        b += __shfl_xor_sync(FULL_MASK, b, off);
      }
      if (lane == 0) { scal[0] = a; scal[1] = b; }
    }
    named_sync(NT);
    stamp(pass, 3);
    if (pass == 0) ynorm = sqrt(scal[1]);
    const double enorm = sqrt(scal[0]);
    const double rel = ynorm > 0.0 ? enorm / ynorm : enorm;
    if (blockIdx.x == 0 && tid == 0) p.hist[sw] = rel;  // a confirmation overwrites the tracked value
    sweeps = sw;
    // e_out is y - X·a for exactly the float32 coefficients a_out would get:
    // pass 0 (a = 0, or the float32 guess) and a confirmation pass
    const bool exact = pass == 0 || conf || fin;
    // after the selection steps of Algorithm 3, up to swap_rounds swap steps
    const bool swap_phase = SEL && p.swap_rounds > 0 && sw >= p.max_sweeps;
    bool stop = false;
    if (!isfinite(rel)) {
      status = HPSCD_ERR_NONFINITE; stop = true;
    } else if (!swap_phase && p.stop_rule == HPSCD_STOP_REL_RES && rel <= p.tol) {
      if (exact || !p.confirm) { status = HPSCD_OK; stop = true; }
      else next_kind = 1;
    } else if (!swap_phase && p.stop_rule == HPSCD_STOP_REL_CHANGE && sw >= 1 &&
               (r_prev == 0.0 || fabs(r_prev - rel) < p.tol * r_prev)) {
      status = HPSCD_OK; stop = true;
    }
    if (!stop && next_kind != 1 && sw == p.max_sweeps + (SEL ? p.swap_rounds : 0)) {
      status = (p.stop_rule == HPSCD_STOP_NONE || swap_phase) ? HPSCD_OK : HPSCD_ERR_NOT_CONVERGED;
      stop = true;
    }
    // When the residual's decay predicts that the next sweep ends at half the
    // tolerance or below, that sweep's pass forms y - X·a of the returned
    // coefficients itself (and the rule is tested on it), in place of a
    // separate confirmation pass after it.
    if (!stop && next_kind == 0 && p.confirm && p.stop_rule == HPSCD_STOP_REL_RES && sw >= 1 &&
        r_prev > 0.0 && rel * (rel / r_prev) <= 0.5 * p.tol)
      next_kind = 2;
    r_prev = rel;
    if (stop) break;
    if (next_kind == 1) {
      // the next pass recomputes e = y - X·a for a = fl32(a64), the coefficients
      // that would be returned, and applies no step (da = 0)
      for (int c = tid; c < NPAD; c += NT) {
        const float hi = (float)a64_s[c];
        a64_s[c] = (double)hi;
        vsm[c] = hi;
        vlo[c] = 0.f;
        da_s[c] = 0.f;
      }
      named_sync(NT);
      if constexpr (V_IN_REGS) {
#pragma unroll
        for (int j = 0; j < CPW; ++j) v[j] = vsm[(j / CW) * C + warp * CW + (j % CW)];
      }
      continue;
    }

    int removed = -1;  // a swap step's dropped column (its coefficient becomes exactly 0)
    if constexpr (SEL) {
    if (swap_phase) {
      // scratch: the row-sum buffers are free between passes
      int jin = -1;
      removed = swap_step(n, NPAD, rvec, dd_s, a64_s, p.Gt, p.ldG, scal[0], da_s,
                          reinterpret_cast<int*>(red_hi) + 4 * NW, reinterpret_cast<double*>(red_lo),
                          reinterpret_cast<int*>(red_hi), &jin);
      if (blockIdx.x == 0 && tid == 0 && p.swap_out) {
        p.swap_out[2 * (sw - p.max_sweeps)] = removed;
        p.swap_out[2 * (sw - p.max_sweeps) + 1] = jin;
      }
      if (removed < 0) {  // no exchange lowers the error: done
        status = HPSCD_OK;
        break;
      }
    } else {
      // scratch for the argmax: the row-sum buffer is free between passes
      const int jhat = select_step(n, NPAD, rvec, dd_s, da_s, red_hi, reinterpret_cast<int*>(red_lo));
      if (blockIdx.x == 0 && tid == 0 && p.sel_out) p.sel_out[sw] = jhat;
    }
    } else if constexpr (ORD) {
      // the steps of sweep pass + 1 take the columns order[pass·n + k]: gather
      // their r and the diagonal blocks of their couplings, substitute over the
      // steps, then sum the steps of each column in step order (identical in
      // every CTA).  Between passes the row-sum buffer holds the steps' da and
      // columns, vsm their r; the flags live in red_lo as in the plain sweep.
      float* dstep = red_hi;
      int* o_s = reinterpret_cast<int*>(red_hi + NPAD);
      float* rstep = vsm;
      const int* ord = p.order + (size_t)sw * n;
      for (int k = tid; k < NPAD; k += NT) o_s[k] = k < n ? __ldg(ord + k) : -1;
      named_sync(NT);
      for (int k = tid; k < NPAD; k += NT) rstep[k] = k < n ? rvec[o_s[k]] : 0.f;
      for (int idx = tid; idx < ((n + 31) / 32) * DIAG_PACK; idx += NT) {
        const int b = idx / DIAG_PACK, q = idx % DIAG_PACK;
        int i = 1;
        while ((i * (i + 1)) / 2 <= q) ++i;
        const int k = q - (i * (i - 1)) / 2;
        diag_s[idx] = (32 * b + i < n) ? __ldg(p.Gt + (int64_t)o_s[32 * b + i] * p.ldG + o_s[32 * b + k])
                                       : 0.f;
      }
      named_sync(NT);
      invert_diag_blocks(diag_s, (n + 31) / 32);
      if (!forward_substitution<true>(p.Gt, p.ldG, n, NPAD, rstep, dstep, diag_s, 1,
                                      reinterpret_cast<int*>(red_lo), p.timeout_ns, o_s)) {
        err = DEV_TIMEOUT_BARRIER;
        break;
      }
      for (int c = tid; c < NPAD; c += NT) {
        float acc = 0.f;
        if (c < n)
          for (int k = 0; k < n; ++k)
            if (o_s[k] == c) acc += dstep[k];
        da_s[c] = acc;
      }
      named_sync(NT);
    } else {
      // the row-sum buffers are free between passes: flags of the substitution
      if (!forward_substitution<false>(p.Gt, p.ldG, n, NPAD, rvec, da_s, diag_s, p.thr,
                                       reinterpret_cast<int*>(red_lo), p.timeout_ns)) {
        err = DEV_TIMEOUT_BARRIER;
        break;
      }
    }
    stamp(pass, 5);
    const int64_t nx = sw + 1;
    const bool next_refresh = p.refresh_every > 0 && nx % p.refresh_every == 0;
    for (int c = tid; c < NPAD; c += NT) {
      if constexpr (SEL) a64_s[c] = (c == removed) ? 0.0 : a64_s[c] + (double)da_s[c];
      else a64_s[c] += (double)da_s[c];
      // a refresh forms y - X·a from a itself: a = hi + lo, both float32; the
      // predicted last sweep forms it for the float32 coefficients returned
      const float hi = (float)a64_s[c];
      if (next_kind == 2) a64_s[c] = (double)hi;
      vsm[c] = (next_refresh || next_kind == 2) ? hi : da_s[c];
      vlo[c] = (next_refresh && next_kind != 2) ? (float)(a64_s[c] - (double)hi) : 0.f;
    }
    named_sync(NT);
    if constexpr (V_IN_REGS) {
#pragma unroll
      for (int j = 0; j < CPW; ++j) v[j] = vsm[(j / CW) * C + warp * CW + (j % CW)];
    }
  }

  // drain copies still in flight before the CTA retires
  if (tma && tid == 0) {
    for (uint64_t k = waited; k < issued; ++k)
      if (!mbar_wait_bounded(&full[k % nst], (uint32_t)((k / nst) & 1), p.timeout_ns)) {
        if (err == DEV_OK) err = DEV_TIMEOUT_COPY;
        break;
      }
  }
  named_sync(NT);
  if (err != DEV_OK && tid == 0) atomicCAS(&p.ctl->err, DEV_OK, err);
  if (blockIdx.x == 0) {
    for (int c = tid; c < n; c += NT) p.a_out[c] = (float)a64_s[c];
    if (tid == 0) {
      p.ctl->status = (err != DEV_OK) ? HPSCD_ERR_TIMEOUT : status;
      p.ctl->sweeps = sweeps;
      p.ctl->final_res = r_prev;
      p.ctl->passes = pass + 1 - ((p.h0 && !p.warm) ? 1 : 0);  // passes over X made
    }
  }
}

template <typename T, int CW, int NCH, int KMODE = 0>
cudaError_t launch_one(const TallConfig& cfg, const CUtensorMap* tmap, const TallParams& p,
                       int grid, cudaStream_t stream) {
  auto kern = tall_sweep_kernel<T, CW, NCH, KMODE>;
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

}  // namespace hpscd
