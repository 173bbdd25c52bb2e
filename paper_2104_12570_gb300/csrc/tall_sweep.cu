// Host side of the persistent tall sweep: chunk geometry, the coupling
// scaling kernel of the set-up, and the launch dispatch over the kernel's
// instantiations (float32 and bfloat16 here; IEEE binary16 in
// tall_sweep_f16.cu).  The kernel itself is in tall_sweep.cuh.
#include "tall_sweep.cuh"

namespace hpscd {

namespace {

// G~ = D^{-1} G (row i divided by G_ii; a zero row for G_ii <= 0), d = diag(G),
// columns n..ldG-1 of G~ zeroed.  One CTA per row.
__global__ void scale_rows_kernel(const float* __restrict__ G, int ldG, int n, float* __restrict__ Gt,
                                  float* __restrict__ d) {
  const int i = blockIdx.x;
  const float gi = G[(int64_t)i * ldG + i];
  const bool live = gi > 0.f;
  for (int j = threadIdx.x; j < ldG; j += blockDim.x) {
    float v = 0.f;
    if (live && j < n) v = (j == i) ? 1.f : G[(int64_t)i * ldG + j] / gi;
    Gt[(int64_t)i * ldG + j] = v;
  }
  if (threadIdx.x == 0) d[i] = live ? gi : 0.f;
}

}  // namespace

cudaError_t launch_scale_rows(const float* G, int ldG, int n, float* Gt, float* d, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  scale_rows_kernel<<<n, 256, 0, stream>>>(G, ldG, n, Gt, d);
  return cudaGetLastError();
}

// Chunk geometry: 128 rows × C columns, C = 16·CW with CW = 4 (float32) or 8
// (bfloat16) for wide enough n, so a chunk is 32 KB and each column segment
// 512 or 256 contiguous bytes; NCH chunks (a power of two) cover n.
bool tall_config(int dtype, int n, int max_smem, TallConfig* cfg) {
  if (n < 0 || n > 512) return false;
  const int esz = (dtype == HPSCD_F32) ? 4 : 2;
  const int cwmax = (dtype == HPSCD_F32) ? 4 : 8;
  int cw = 1;
  while (cw < cwmax && NW * cw < n) cw *= 2;
  const int c = NW * cw;
  int nch = 1;
  while (c * nch < n) nch *= 2;
  cfg->cpw = cw;      // columns per warp per chunk
  cfg->rpl = nch;     // chunks per panel
  cfg->npad = c * nch;
  cfg->rows = PR;
  cfg->stage_bytes = PR * c * esz;
  cfg->box_cols = c;
  cfg->threads = NT;
  const int nblk = cfg->npad >= 32 ? cfg->npad / 32 : 1;
  const int fixed = 1024 /*align*/ + 4 * NW * PR * 4 + cfg->npad * (5 * 4 + 8) + 40 * 8 +
                    32 * 8 + 16 + nblk * DIAG_PACK * 4;
  int nst = (max_smem - 256 - fixed) / cfg->stage_bytes;
  if (nst > 12) nst = 12;
  if (nst < 3) return false;
  cfg->nstages = nst;
  cfg->smem_bytes = fixed + nst * cfg->stage_bytes;
  return true;
}

cudaError_t launch_tall_sweep(int dtype, const TallConfig& cfg, const CUtensorMap* tmap,
                              const TallParams& p, int grid, cudaStream_t stream) {
#define HPSCD_TALL_CASE(T, W, N)                                        \
  if (cfg.cpw == W && cfg.rpl == N) return launch_one<T, W, N>(cfg, tmap, p, grid, stream);
#define HPSCD_TALL_ORD_CASE(W, N)                                       \
  if (cfg.cpw == W && cfg.rpl == N) return launch_one<float, W, N, 1>(cfg, tmap, p, grid, stream);
#define HPSCD_TALL_SEL_CASE(T, W, N)                                    \
  if (cfg.cpw == W && cfg.rpl == N) return launch_one<T, W, N, 2>(cfg, tmap, p, grid, stream);
  if (p.order) {  // the given-order variant: float32 only
    if (dtype != HPSCD_F32) return cudaErrorInvalidValue;
    HPSCD_TALL_ORD_CASE(1, 1)
    HPSCD_TALL_ORD_CASE(2, 1)
    HPSCD_TALL_ORD_CASE(4, 1)
    HPSCD_TALL_ORD_CASE(4, 2)
    HPSCD_TALL_ORD_CASE(4, 4)
    HPSCD_TALL_ORD_CASE(4, 8)
    return cudaErrorInvalidConfiguration;
  }
  if (dtype == HPSCD_F16) return launch_tall_sweep_f16(cfg, tmap, p, grid, stream);
  if (p.select) {  // selection and swap steps
    if (dtype == HPSCD_F32) {
      HPSCD_TALL_SEL_CASE(float, 1, 1)
      HPSCD_TALL_SEL_CASE(float, 2, 1)
      HPSCD_TALL_SEL_CASE(float, 4, 1)
      HPSCD_TALL_SEL_CASE(float, 4, 2)
      HPSCD_TALL_SEL_CASE(float, 4, 4)
      HPSCD_TALL_SEL_CASE(float, 4, 8)
    } else {
      HPSCD_TALL_SEL_CASE(uint16_t, 1, 1)
      HPSCD_TALL_SEL_CASE(uint16_t, 2, 1)
      HPSCD_TALL_SEL_CASE(uint16_t, 4, 1)
      HPSCD_TALL_SEL_CASE(uint16_t, 8, 1)
      HPSCD_TALL_SEL_CASE(uint16_t, 8, 2)
      HPSCD_TALL_SEL_CASE(uint16_t, 8, 4)
    }
    return cudaErrorInvalidConfiguration;
  }
  if (dtype == HPSCD_F32) {
    HPSCD_TALL_CASE(float, 1, 1)
    HPSCD_TALL_CASE(float, 2, 1)
    HPSCD_TALL_CASE(float, 4, 1)
    HPSCD_TALL_CASE(float, 4, 2)
    HPSCD_TALL_CASE(float, 4, 4)
    HPSCD_TALL_CASE(float, 4, 8)
  } else {
    HPSCD_TALL_CASE(uint16_t, 1, 1)
    HPSCD_TALL_CASE(uint16_t, 2, 1)
    HPSCD_TALL_CASE(uint16_t, 4, 1)
    HPSCD_TALL_CASE(uint16_t, 8, 1)
    HPSCD_TALL_CASE(uint16_t, 8, 2)
    HPSCD_TALL_CASE(uint16_t, 8, 4)
  }
#undef HPSCD_TALL_CASE
#undef HPSCD_TALL_ORD_CASE
#undef HPSCD_TALL_SEL_CASE
  return cudaErrorInvalidConfiguration;
}

}  // namespace hpscd
