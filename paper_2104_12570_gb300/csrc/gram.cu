// Set-up kernels: the Gram matrix G = X^T X of a column-major X.
//
// Algorithm 1 divides by <X_j, X_j> in every column step (Eq. da2); X does not
// change, so those denominators are formed once, as the diagonal of G.  The
// off-diagonal lower triangle G_jl = <X_j, X_l> (l < j) lets the persistent
// sweep obtain <X_j, e> against the residual as it stands just before column
// j, from the sweep-start dot products: <X_j, e> = g_j - sum_{l<j} G_jl da_l
// (Eq. ek1-ek applied to the columns already updated in this sweep).
//
// Tiles of 64x64 outputs, split over rows; float32 products accumulated in
// float32 over 1024-row blocks, then in float64 across blocks and splits.
#include <cuda_fp16.h>

#include "kernels.h"

namespace hpscd {

namespace {

constexpr int GT = 64;     // output tile edge
constexpr int GKB = 32;    // rows per shared-memory chunk
constexpr int GFLUSH = 32; // chunks per float64 flush (1024 rows)

template <typename T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<uint16_t>(uint16_t v) { return bf16_bits_to_float(v); }
template <>
__device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }

// grid: (ntile, ksplit); block 256.  Tile t enumerates (I >= J) 64-column blocks.
template <typename T>
__global__ void __launch_bounds__(256) gram_partial_kernel(const T* __restrict__ X, int64_t m, int n,
                                                          int64_t ld, int64_t rows_per_split,
                                                          double* __restrict__ partial) {
  __shared__ float As[GKB][GT + 4];
  __shared__ float Bs[GKB][GT + 4];
  const int t = blockIdx.x;
  // decode t -> (I, J), I >= J, row-major over the lower triangle
  int I = 0;
  while ((I + 1) * (I + 2) / 2 <= t) ++I;
  const int J = t - I * (I + 1) / 2;
  const int64_t k0 = (int64_t)blockIdx.y * rows_per_split;
  const int64_t k1 = min(m, k0 + rows_per_split);
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;

  float acc[4][4];
  double acc64[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) { acc[i][j] = 0.f; acc64[i][j] = 0.0; }

  int chunk = 0;
  for (int64_t k = k0; k < k1; k += GKB) {
#pragma unroll
    for (int q = 0; q < (GKB * GT) / 256; ++q) {
      const int idx = tid + 256 * q;
      const int c = idx / GKB, r = idx % GKB;
      const int64_t row = k + r;
      const int ca = I * GT + c, cb = J * GT + c;
      float va = 0.f, vb = 0.f;
      if (row < k1) {
        if (ca < n) va = to_f<T>(X[(int64_t)ca * ld + row]);
        if (cb < n) vb = to_f<T>(X[(int64_t)cb * ld + row]);
      }
      As[r][c] = va;
      Bs[r][c] = vb;
    }
    __syncthreads();
#pragma unroll 8
    for (int r = 0; r < GKB; ++r) {
      const float4 a4 = *reinterpret_cast<const float4*>(&As[r][ty * 4]);
      const float4 b4 = *reinterpret_cast<const float4*>(&Bs[r][tx * 4]);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w};
      const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
    if (++chunk == GFLUSH) {
      chunk = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) { acc64[i][j] += (double)acc[i][j]; acc[i][j] = 0.f; }
    }
  }
  double* out = partial + ((size_t)blockIdx.y * gridDim.x + t) * (GT * GT);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) out[(ty * 4 + i) * GT + tx * 4 + j] = acc64[i][j] + (double)acc[i][j];
}

// G[i][j] = G[j][i] = sum over splits (fixed order) of the lower partial tiles.
__global__ void gram_reduce_kernel(const double* __restrict__ partial, int ntile, int ksplit,
                                   int npad, float* __restrict__ G, int ldG) {
  const int64_t total = (int64_t)npad * npad;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i0 = (int)(idx / npad), j0 = (int)(idx % npad);
    const int i = i0 >= j0 ? i0 : j0, j = i0 >= j0 ? j0 : i0;  // G is symmetric
    const int I = i / GT, J = j / GT;
    const int t = I * (I + 1) / 2 + J;
    const int off = (i % GT) * GT + (j % GT);
    double s = 0.0;
    for (int k = 0; k < ksplit; ++k) s += partial[((size_t)k * ntile + t) * (GT * GT) + off];
    G[(int64_t)i0 * ldG + j0] = (float)s;
  }
}

}  // namespace

GramPlan gram_plan(int64_t m, int npad, int sms) { return gram_plan_capped(m, npad, sms, 0); }

// As gram_plan, with at most max_ksplit row splits when max_ksplit > 0 (the
// partial tiles then take less memory).
GramPlan gram_plan_capped(int64_t m, int npad, int sms, int max_ksplit) {
  GramPlan gp;
  gp.npad = ((npad + GT - 1) / GT) * GT;
  const int nb = gp.npad / GT;
  gp.ntile = nb * (nb + 1) / 2;
  int64_t want = (int64_t)4 * sms / gp.ntile;
  if (want < 1) want = 1;
  int64_t maxsplit = (m + 1023) / 1024;
  if (maxsplit < 1) maxsplit = 1;
  if (max_ksplit > 0 && maxsplit > max_ksplit) maxsplit = max_ksplit;
  gp.ksplit = (int)(want < maxsplit ? want : maxsplit);
  int64_t rps = (m + gp.ksplit - 1) / gp.ksplit;
  rps = ((rps + GKB - 1) / GKB) * GKB;
  if (rps < GKB) rps = GKB;
  gp.rows_per_split = rps;
  gp.ksplit = (int)((m + rps - 1) / rps);
  if (gp.ksplit < 1) gp.ksplit = 1;
  gp.partial_bytes = (size_t)gp.ksplit * gp.ntile * GT * GT * sizeof(double);
  return gp;
}

cudaError_t launch_gram(const void* X, int dtype, int64_t m, int n, int64_t ld, const GramPlan& gp,
                        double* partial, float* G, int ldG, cudaStream_t stream) {
  dim3 grid(gp.ntile, gp.ksplit);
  if (dtype == HPSCD_F32)
    gram_partial_kernel<float><<<grid, 256, 0, stream>>>((const float*)X, m, n, ld,
                                                         gp.rows_per_split, partial);
  else if (dtype == HPSCD_BF16)
    gram_partial_kernel<uint16_t><<<grid, 256, 0, stream>>>((const uint16_t*)X, m, n, ld,
                                                            gp.rows_per_split, partial);
  else
    gram_partial_kernel<__half><<<grid, 256, 0, stream>>>((const __half*)X, m, n, ld,
                                                          gp.rows_per_split, partial);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const int64_t total = (int64_t)gp.npad * gp.npad;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  gram_reduce_kernel<<<blocks, 256, 0, stream>>>(partial, gp.ntile, gp.ksplit, gp.npad, G, ldG);
  return cudaGetLastError();
}

}  // namespace hpscd
