// Layout kernels of the set-up: a row-major X whose shape the cluster sweep
// does not take (m above its row limit) is transposed once into a column-major
// copy for the tall or panel sweep, and a 16-bit row-major X for the cluster
// sweep is widened once into float32.  Both copy element values exactly
// (the transpose moves bit patterns; the widening is exact).
#include <cuda_fp16.h>

#include "kernels.h"

namespace hpscd {

namespace {

constexpr int TT = 32;  // transpose tile edge

// out(col-major, ldo)[i + j·ldo] = X(row-major, ld)[i·ld + j] for i < m, j < n,
// through a shared-memory tile (both sides coalesced).  grid: (ceil(n/32), tiles of rows).
template <typename E>
__global__ void __launch_bounds__(256) transpose_kernel(const E* __restrict__ X, int64_t m, int64_t n,
                                                        int64_t ld, E* __restrict__ out, int64_t ldo,
                                                        int64_t row_tiles) {
  __shared__ E tile[TT][TT + 1];
  const int64_t j0 = (int64_t)blockIdx.x * TT;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of 32 per step
  for (int64_t bt = blockIdx.y; bt < row_tiles; bt += gridDim.y) {
    const int64_t i0 = bt * TT;
#pragma unroll
    for (int k = 0; k < TT; k += 8) {
      const int64_t i = i0 + ty + k, j = j0 + tx;
      if (i < m && j < n) tile[ty + k][tx] = X[i * ld + j];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TT; k += 8) {
      const int64_t j = j0 + ty + k, i = i0 + tx;
      if (i < m && j < n) out[j * ldo + i] = tile[tx][ty + k];
    }
    __syncthreads();
  }
}

template <typename T>
__device__ __forceinline__ float widen(T v);
template <>
__device__ __forceinline__ float widen<uint16_t>(uint16_t v) { return bf16_bits_to_float(v); }
template <>
__device__ __forceinline__ float widen<__half>(__half v) { return __half2float(v); }

// out[i·ldo + j] = float(X[i·ld + j]), row-major both.
template <typename T>
__global__ void __launch_bounds__(256) widen_rows_kernel(const T* __restrict__ X, int64_t m, int64_t n,
                                                         int64_t ld, float* __restrict__ out, int64_t ldo) {
  const int64_t total = m * n;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = k / n, j = k - i * n;
    out[i * ldo + j] = widen<T>(X[i * ld + j]);
  }
}

}  // namespace

cudaError_t launch_transpose_to_col(const void* X, int dtype, int64_t m, int64_t n, int64_t ld, void* out,
                                    int64_t ldo, int sms, cudaStream_t stream) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  const int64_t row_tiles = (m + TT - 1) / TT;
  const int64_t col_tiles = (n + TT - 1) / TT;
  if (col_tiles > 0x7fffffff) return cudaErrorInvalidValue;
  int64_t gy = (int64_t)sms * 8 / (col_tiles < 1 ? 1 : col_tiles);
  if (gy < 1) gy = 1;
  if (gy > row_tiles) gy = row_tiles;
  if (gy > 65535) gy = 65535;
  dim3 grid((unsigned)col_tiles, (unsigned)gy);
  if (dtype == HPSCD_F32)
    transpose_kernel<uint32_t><<<grid, 256, 0, stream>>>(static_cast<const uint32_t*>(X), m, n, ld,
                                                          static_cast<uint32_t*>(out), ldo, row_tiles);
  else
    transpose_kernel<uint16_t><<<grid, 256, 0, stream>>>(static_cast<const uint16_t*>(X), m, n, ld,
                                                          static_cast<uint16_t*>(out), ldo, row_tiles);
  return cudaGetLastError();
}

cudaError_t launch_widen_rows(const void* X, int dtype, int64_t m, int64_t n, int64_t ld, float* out,
                              int64_t ldo, int sms, cudaStream_t stream) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  const int blocks = sms * 8;
  if (dtype == HPSCD_BF16)
    widen_rows_kernel<uint16_t><<<blocks, 256, 0, stream>>>(static_cast<const uint16_t*>(X), m, n, ld, out,
                                                            ldo);
  else if (dtype == HPSCD_F16)
    widen_rows_kernel<__half><<<blocks, 256, 0, stream>>>(static_cast<const __half*>(X), m, n, ld, out, ldo);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace hpscd
