// IEEE binary16 instantiations of the persistent tall sweep (the plain sweep
// and the selection / swap steps), compiled apart from the float32 and
// bfloat16 ones so that the library's translation units build in parallel.
// The kernel reads each 16-bit element and widens it exactly to float32;
// everything after the load is the float32 arithmetic of the other types.
#include "tall_sweep.cuh"

namespace hpscd {

cudaError_t launch_tall_sweep_f16(const TallConfig& cfg, const CUtensorMap* tmap, const TallParams& p,
                                  int grid, cudaStream_t stream) {
  if (p.order) return cudaErrorInvalidValue;  // the given-order variant is float32 only
#define HPSCD_F16_CASE(W, N, K) \
  if (cfg.cpw == W && cfg.rpl == N) return launch_one<__half, W, N, K>(cfg, tmap, p, grid, stream);
  if (p.select) {
    HPSCD_F16_CASE(1, 1, 2)
    HPSCD_F16_CASE(2, 1, 2)
    HPSCD_F16_CASE(4, 1, 2)
    HPSCD_F16_CASE(8, 1, 2)
    HPSCD_F16_CASE(8, 2, 2)
    HPSCD_F16_CASE(8, 4, 2)
    return cudaErrorInvalidConfiguration;
  }
  HPSCD_F16_CASE(1, 1, 0)
  HPSCD_F16_CASE(2, 1, 0)
  HPSCD_F16_CASE(4, 1, 0)
  HPSCD_F16_CASE(8, 1, 0)
  HPSCD_F16_CASE(8, 2, 0)
  HPSCD_F16_CASE(8, 4, 0)
#undef HPSCD_F16_CASE
  return cudaErrorInvalidConfiguration;
}

}  // namespace hpscd
