// Learned warm start: a 3-layer MLP  phi(theta, m, n) -> a  (width 256, ReLU),
// trained on solutions the sweep itself produces for a parametric family of
// systems, whose prediction seeds a solve ("or initial guess" of Algorithm 2;
// the paper's remark that similar systems are solved many times, Sec. 9).
//
// Arithmetic: bfloat16 weights and activations as matrix operands, float32
// accumulation (tensor memory), float32 master weights and Adam moments.
// Every matrix product of the forward and backward pass is one launch of
// mlp_gemm_kernel: D[M×N] = A[M×K] · B[N×K]^T with both operands K-major
// bfloat16, streamed by TMA (128-byte swizzle) and multiplied by tcgen05.mma
// (kind::f16, M = 128, N = 64 or 256) issued by one thread; the epilogue reads
// the accumulator with tcgen05.ld and fuses bias, ReLU / ReLU-mask and the
// stores (row-major and transposed bfloat16, or float32).  Activations are
// kept in both layouts so every backward product also has K-major operands:
//   Z1 = Phi W1^T, H1 = relu(Z1 + b1)     dW3 = dOut^T H2    dH2 = dOut W3
//   Z2 = H1 W2^T,  H2 = relu(Z2 + b2)     dZ2 = dH2 * [H2 > 0], dW2 = dZ2^T H1
//   Out = H2 W3^T + b3                   dZ1 = (dZ2 W2) * [H1 > 0], dW1 = dZ1^T Phi
// Loss: mean over the valid entries (j < n of each row) of (Out - a*)^2.
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "ctx.h"

namespace hpscd {

namespace {

constexpr int MT = 128;        // rows of a D tile (MMA M)
constexpr int KB = 64;         // K per stage (128 bytes of bfloat16)
constexpr int G_THREADS = 128;
constexpr int G_STAGES = 3;
constexpr int IN_F = 18, IN_P = 64, HID = 256, OUT_F = 256, THETA = 16;

__device__ __forceinline__ uint64_t sw128_desc(uint32_t smem_addr) {
  // K-major operand, 128-byte swizzle: start >> 4, leading offset 1 (unused),
  // stride offset 1024 B >> 4 between 8-row groups, version 1, layout SW128.
  uint64_t d = 0;
  d |= (uint64_t)((smem_addr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// kind::f16 instruction descriptor: D float32, A = B = bfloat16, K-major, M = 128, N.
__host__ __device__ constexpr uint32_t bf16_idesc(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(MT >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint16_t f2bf(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float bf2f(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

enum EpiMode : int {
  EPI_BIAS_RELU = 0,  // v = relu(acc + bias): bf16 out (row-major) and bf16 outT (transposed)
  EPI_BIAS_F32 = 1,   // v = acc + bias: float32 out
  EPI_F32 = 2,        // v = acc: float32 out
  EPI_MASK = 3        // v = acc * [mask > 0]: bf16 out (optional) and bf16 outT (optional)
};

struct GemmEpi {
  int mode;
  int M, N, K;            // M multiple of 128, N in {64, 256}, K multiple of 64
  const float* bias;      // [N]
  void* out;              // row-major [M][ldo] (bf16 or float32), may be null (EPI_MASK)
  int ldo;
  uint16_t* outT;         // transposed bf16 [N][ldt], may be null
  int ldt;
  const uint16_t* mask;   // bf16 [M][ldm] (EPI_MASK)
  int ldm;
  int* err;
  uint64_t timeout_ns;
};

// One CTA per 128-row tile of D; the whole N in tensor memory.
__global__ void __launch_bounds__(G_THREADS, 1)
    mlp_gemm_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
                    const GemmEpi e) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int N = e.N;
  const int a_bytes = MT * 128, b_bytes = N * 128;
  const int stage_bytes = a_bytes + b_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(base + (size_t)G_STAGES * stage_bytes);
  uint64_t* empty = full + G_STAGES;
  uint64_t* done = empty + G_STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row0 = blockIdx.x * MT;
  const int nk = e.K / KB;

  if (tid == 0) {
    for (int s = 0; s < G_STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
    mbar_init(done, 1);
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(N)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  int issued = 0;
  auto issue = [&](int kb) {
    const int s = kb % G_STAGES;
    unsigned char* dst = base + (size_t)s * stage_bytes;
    mbar_arrive_expect_tx(&full[s], (uint32_t)stage_bytes);
    tma_load_2d(dst, &ta, &full[s], kb * KB, row0);
    tma_load_2d(dst + a_bytes, &tb, &full[s], kb * KB, 0);
  };
  if (tid == 0)
    while (issued < G_STAGES && issued < nk) issue(issued++);

  bool ok = true;
  int consumed = 0;
  const uint32_t idesc = bf16_idesc(N);
  for (int kb = 0; kb < nk; ++kb) {
    const int s = kb % G_STAGES;
    if (tid == 0) {
      if (ok && !mbar_wait_bounded(&full[s], (uint32_t)((kb / G_STAGES) & 1), e.timeout_ns)) ok = false;
      if (ok) {
        tc_fence_after();
        const uint32_t a_base = smem_u32(base + (size_t)s * stage_bytes);
        const uint32_t b_base = a_base + a_bytes;
#pragma unroll
        for (int k = 0; k < KB / 16; ++k) {
          const uint64_t ad = sw128_desc(a_base + 32 * k);
          const uint64_t bd = sw128_desc(b_base + 32 * k);
          const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&empty[s]))
            : "memory");
        consumed = kb + 1;
        // refill this stage for K block kb + G_STAGES once its MMAs have read it
        if (issued < nk) {
          if (!mbar_wait_bounded(&empty[s], (uint32_t)((kb / G_STAGES) & 1), e.timeout_ns)) ok = false;
          else issue(issued++);
        }
      }
    }
  }
  if (tid == 0) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(done))
        : "memory");
  }
  __syncthreads();
  if (!mbar_wait_bounded(done, 0, e.timeout_ns)) ok = false;
  tc_fence_after();
  const int fail = __syncthreads_or((tid == 0 && !ok) ? 1 : 0) || !ok;
  if (!fail) {
    const int r = row0 + 32 * warp + lane;  // this thread's row of D
    for (int c0 = 0; c0 < N; c0 += 32) {
      float v[32];
      if (nk > 0) {
        tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + c0, v);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = 0.f;
      }
      if (e.mode == EPI_BIAS_RELU || e.mode == EPI_BIAS_F32) {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] += __ldg(e.bias + c0 + i);
      }
      if (e.mode == EPI_BIAS_RELU) {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = fmaxf(v[i], 0.f);
      }
      if (e.mode == EPI_MASK) {
        const uint16_t* mrow = e.mask + (size_t)r * e.ldm + c0;
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = bf2f(mrow[i]) > 0.f ? v[i] : 0.f;
      }
      if (e.mode == EPI_BIAS_F32 || e.mode == EPI_F32) {
        float* o = static_cast<float*>(e.out) + (size_t)r * e.ldo + c0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(o + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      } else {
        if (e.out) {
          uint16_t* o = static_cast<uint16_t*>(e.out) + (size_t)r * e.ldo + c0;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            uint4 w;
            w.x = (uint32_t)f2bf(v[8 * q]) | ((uint32_t)f2bf(v[8 * q + 1]) << 16);
            w.y = (uint32_t)f2bf(v[8 * q + 2]) | ((uint32_t)f2bf(v[8 * q + 3]) << 16);
            w.z = (uint32_t)f2bf(v[8 * q + 4]) | ((uint32_t)f2bf(v[8 * q + 5]) << 16);
            w.w = (uint32_t)f2bf(v[8 * q + 6]) | ((uint32_t)f2bf(v[8 * q + 7]) << 16);
            *reinterpret_cast<uint4*>(o + 8 * q) = w;
          }
        }
        if (e.outT) {
#pragma unroll
          for (int i = 0; i < 32; ++i) e.outT[(size_t)(c0 + i) * e.ldt + r] = f2bf(v[i]);
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(e.err, 1);
    for (int kb = consumed; kb < issued; ++kb)
      if (!mbar_wait_bounded(&full[kb % G_STAGES], (uint32_t)((kb / G_STAGES) & 1), e.timeout_ns)) break;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(N) : "memory");
}

// phi(theta, m, n) = [theta_1..16, n / 256, log(m) / log(16384)], zero-padded to
// 64 columns; rows >= B are zero.  Writes Phi [Bp][64] and Phi^T [64][Bp] (bf16).
__global__ void mlp_features_kernel(const float* __restrict__ theta, const int64_t* __restrict__ m,
                                    const int64_t* __restrict__ n, int B, int Bp, uint16_t* phi,
                                    uint16_t* phiT, int ldT) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Bp * IN_P) return;
  const int b = idx / IN_P, c = idx % IN_P;
  float v = 0.f;
  if (b < B) {
    if (c < THETA) v = theta[(size_t)b * THETA + c];
    else if (c == THETA) v = (float)n[b] / 256.f;
    else if (c == THETA + 1) v = (float)(log((double)(m[b] > 0 ? m[b] : 1)) / log(16384.0));
  }
  const uint16_t h = f2bf(v);
  phi[(size_t)b * IN_P + c] = h;
  if (phiT) phiT[(size_t)c * ldT + b] = h;
}

// dOut = 2 (Out - T) [j < n_b] / count (bf16, both layouts); loss partial sums.
__global__ void mlp_loss_grad_kernel(const float* __restrict__ out, const float* __restrict__ target,
                                     const int64_t* __restrict__ n, int B, int Bp, double inv_count,
                                     uint16_t* dout, uint16_t* doutT, int ldT, double* loss) {
  __shared__ double red[8];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (idx < Bp * OUT_F) {
    const int b = idx / OUT_F, j = idx % OUT_F;
    float g = 0.f;
    if (b < B && j < n[b]) {
      const float d = out[idx] - target[(size_t)b * OUT_F + j];
      l = (double)d * (double)d;
      g = (float)(2.0 * (double)d * inv_count);
    }
    const uint16_t h = f2bf(g);
    dout[idx] = h;
    doutT[(size_t)j * ldT + b] = h;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(FULL_MASK, l, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(loss, s * inv_count);
  }
}

// db[j] = sum_b G^T[j][b] (rows of a transposed bf16 gradient), one warp per j.
__global__ void mlp_rowsum_kernel(const uint16_t* __restrict__ gT, int ld, int B, int rows, float* db) {
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (j >= rows) return;
  float s = 0.f;
  for (int b = lane; b < B; b += 32) s += bf2f(gT[(size_t)j * ld + b]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(FULL_MASK, s, off);
  if (lane == 0) db[j] = s;
}

// Adam (Kingma & Ba 2015) on float32 masters; refreshes the bf16 copies
// (row-major w and, for square weights, the transpose wT).
__global__ void mlp_adam_kernel(float* w, const float* g, float* mo, float* vo, int count, int rows,
                                int cols, int valid_cols, float lr, float b1, float b2, float eps,
                                float c1, float c2, uint16_t* wb, uint16_t* wbT) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= count) return;
  const int c = cols > 0 ? idx % cols : 0;
  if (cols > 0 && c >= valid_cols) return;  // padded input columns stay zero
  const float gi = g[idx];
  const float m = b1 * mo[idx] + (1.f - b1) * gi;
  const float v = b2 * vo[idx] + (1.f - b2) * gi * gi;
  mo[idx] = m;
  vo[idx] = v;
  const float wn = w[idx] - lr * (m / c1) / (sqrtf(v / c2) + eps);
  w[idx] = wn;
  if (wb) {
    wb[idx] = f2bf(wn);
    if (wbT) wbT[(size_t)c * rows + idx / cols] = f2bf(wn);
  }
}

__global__ void mlp_cast_kernel(const float* w, int count, int rows, int cols, uint16_t* wb, uint16_t* wbT) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= count) return;
  wb[idx] = f2bf(w[idx]);
  if (wbT) wbT[(size_t)(idx % cols) * rows + idx / cols] = f2bf(w[idx]);
}

// a_b[j] = Out[b][j] for j < n_b, written into the systems' coefficient vectors.
__global__ void mlp_scatter_kernel(const float* __restrict__ out, const hpscd_sys* sys, int64_t b0,
                                   int B) {
  const int b = blockIdx.x;
  if (b >= B) return;
  const hpscd_sys s = sys[b0 + b];
  for (int j = threadIdx.x; j < s.n; j += blockDim.x) s.a[j] = out[(size_t)b * OUT_F + j];
}

}  // namespace

}  // namespace hpscd

using namespace hpscd;

struct hpscd_mlp {
  hpscd_ctx* ctx = nullptr;
  int users = 0;         // batches that start from this network
  bool closing = false;  // destroyed while held: freed by the last holder
  int bmax = 0;  // rows of the activation buffers (multiple of 128)
  void* dev = nullptr;
  // float32 masters, gradients, Adam moments: W1 [256][64], b1, W2 [256][256], b2, W3, b3
  float *w[6] = {}, *g[6] = {}, *mo[6] = {}, *vo[6] = {};
  uint16_t *w1b = nullptr, *w2b = nullptr, *w2t = nullptr, *w3b = nullptr, *w3t = nullptr;
  uint16_t *phi = nullptr, *phiT = nullptr, *h1 = nullptr, *h1T = nullptr, *h2 = nullptr, *h2T = nullptr;
  uint16_t *dout = nullptr, *doutT = nullptr, *dz2 = nullptr, *dz2T = nullptr, *dz1T = nullptr;
  float* out = nullptr;
  int64_t *mbuf = nullptr, *nbuf = nullptr;
  double* loss = nullptr;
  int* err = nullptr;
  int64_t step = 0;
  CUtensorMap m_phi, m_w1, m_h1, m_w2, m_h2, m_w3, m_dout, m_doutT, m_h2T, m_w3t, m_dz2, m_dz2T,
      m_h1T, m_w2t, m_dz1T, m_phiT;
};

namespace {

constexpr int kParamRows[6] = {HID, HID, HID, HID, OUT_F, OUT_F};
constexpr int kParamCols[6] = {IN_P, 0, HID, 0, HID, 0};
inline size_t param_count(int i) { return (size_t)kParamRows[i] * (kParamCols[i] ? kParamCols[i] : 1); }

inline size_t al256(size_t x) { return (x + 255) / 256 * 256; }

bool encode_bf16(const hpscd_ctx* ctx, CUtensorMap* map, const void* base, int rows, int cols,
                 int box_rows) {
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {(cuuint32_t)KB, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return ctx->encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

int gemm_smem(int N) { return G_STAGES * (MT * 128 + N * 128) + 1024 + 256; }

int launch_gemm(hpscd_mlp* p, cudaStream_t st, const CUtensorMap& A, const CUtensorMap& Bm, GemmEpi e) {
  e.err = p->err;
  e.timeout_ns = (uint64_t)(p->ctx->timeout_s * 1e9);
  const int smem = gemm_smem(e.N);
  mlp_gemm_kernel<<<e.M / MT, G_THREADS, smem, st>>>(A, Bm, e);
  return cudaGetLastError() == cudaSuccess ? HPSCD_OK : HPSCD_ERR_CUDA;
}

// Forward pass over Bp rows (multiple of 128): features -> H1 -> H2 -> Out.
// m, n: device int64[B].
int forward(hpscd_mlp* p, cudaStream_t st, const float* theta, const int64_t* m, const int64_t* n,
            int B, int Bp, bool need_T) {
  mlp_features_kernel<<<(Bp * IN_P + 255) / 256, 256, 0, st>>>(theta, m, n, B, Bp, p->phi,
                                                               need_T ? p->phiT : nullptr, p->bmax);
  if (cudaGetLastError() != cudaSuccess) return HPSCD_ERR_CUDA;
  GemmEpi e{};
  e.mode = EPI_BIAS_RELU; e.M = Bp; e.N = HID; e.K = IN_P; e.bias = p->w[1];
  e.out = p->h1; e.ldo = HID; e.outT = need_T ? p->h1T : nullptr; e.ldt = p->bmax;
  int rc = launch_gemm(p, st, p->m_phi, p->m_w1, e);
  if (rc) return rc;
  e = GemmEpi{};
  e.mode = EPI_BIAS_RELU; e.M = Bp; e.N = HID; e.K = HID; e.bias = p->w[3];
  e.out = p->h2; e.ldo = HID; e.outT = need_T ? p->h2T : nullptr; e.ldt = p->bmax;
  if ((rc = launch_gemm(p, st, p->m_h1, p->m_w2, e))) return rc;
  e = GemmEpi{};
  e.mode = EPI_BIAS_F32; e.M = Bp; e.N = OUT_F; e.K = HID; e.bias = p->w[5];
  e.out = p->out; e.ldo = OUT_F;
  return launch_gemm(p, st, p->m_h2, p->m_w3, e);
}

// Loss and gradients of the masked mean-squared error into p->g, p->loss.
int backward(hpscd_mlp* p, cudaStream_t st, const float* target, int B, int Bp, double inv_count) {
  if (cudaMemsetAsync(p->loss, 0, sizeof(double), st) != cudaSuccess) return HPSCD_ERR_CUDA;
  mlp_loss_grad_kernel<<<(Bp * OUT_F + 255) / 256, 256, 0, st>>>(p->out, target, p->nbuf, B, Bp,
                                                                  inv_count, p->dout, p->doutT, p->bmax,
                                                                  p->loss);
  if (cudaGetLastError() != cudaSuccess) return HPSCD_ERR_CUDA;
  GemmEpi e{};
  // dW3 = dOut^T H2
  e.mode = EPI_F32; e.M = OUT_F; e.N = HID; e.K = Bp; e.out = p->g[4]; e.ldo = HID;
  int rc = launch_gemm(p, st, p->m_doutT, p->m_h2T, e);
  if (rc) return rc;
  // dZ2 = (dOut W3) * [H2 > 0]
  e = GemmEpi{};
  e.mode = EPI_MASK; e.M = Bp; e.N = HID; e.K = OUT_F; e.mask = p->h2; e.ldm = HID;
  e.out = p->dz2; e.ldo = HID; e.outT = p->dz2T; e.ldt = p->bmax;
  if ((rc = launch_gemm(p, st, p->m_dout, p->m_w3t, e))) return rc;
  // dW2 = dZ2^T H1
  e = GemmEpi{};
  e.mode = EPI_F32; e.M = HID; e.N = HID; e.K = Bp; e.out = p->g[2]; e.ldo = HID;
  if ((rc = launch_gemm(p, st, p->m_dz2T, p->m_h1T, e))) return rc;
  // dZ1 = (dZ2 W2) * [H1 > 0] (transposed only)
  e = GemmEpi{};
  e.mode = EPI_MASK; e.M = Bp; e.N = HID; e.K = HID; e.mask = p->h1; e.ldm = HID;
  e.out = nullptr; e.outT = p->dz1T; e.ldt = p->bmax;
  if ((rc = launch_gemm(p, st, p->m_dz2, p->m_w2t, e))) return rc;
  // dW1 = dZ1^T Phi
  e = GemmEpi{};
  e.mode = EPI_F32; e.M = HID; e.N = IN_P; e.K = Bp; e.out = p->g[0]; e.ldo = IN_P;
  if ((rc = launch_gemm(p, st, p->m_dz1T, p->m_phiT, e))) return rc;
  // bias gradients: row sums of the transposed gradients
  mlp_rowsum_kernel<<<OUT_F / 8, 256, 0, st>>>(p->doutT, p->bmax, Bp, OUT_F, p->g[5]);
  mlp_rowsum_kernel<<<HID / 8, 256, 0, st>>>(p->dz2T, p->bmax, Bp, HID, p->g[3]);
  mlp_rowsum_kernel<<<HID / 8, 256, 0, st>>>(p->dz1T, p->bmax, Bp, HID, p->g[1]);
  return cudaGetLastError() == cudaSuccess ? HPSCD_OK : HPSCD_ERR_CUDA;
}

// Copies host m, n (int64[B]) to the device and returns 1 / sum_b min(n_b, 256).
int stage_shapes(hpscd_mlp* p, const int64_t* m, const int64_t* n, int B, double* inv_count) {
  double cnt = 0.0;
  for (int b = 0; b < B; ++b) {
    if (m[b] < 0 || n[b] < 0 || n[b] > OUT_F) return HPSCD_ERR_INVALID_ARG;
    cnt += (double)n[b];
  }
  if (inv_count) *inv_count = cnt > 0 ? 1.0 / cnt : 0.0;
  if (B > 0 && (cudaMemcpyAsync(p->mbuf, m, (size_t)B * 8, cudaMemcpyHostToDevice, p->ctx->stream) != cudaSuccess ||
                cudaMemcpyAsync(p->nbuf, n, (size_t)B * 8, cudaMemcpyHostToDevice, p->ctx->stream) != cudaSuccess))
    return HPSCD_ERR_CUDA;
  return HPSCD_OK;
}

int check_io(const hpscd_mlp* p, const void* theta, const void* m, const void* n, int64_t B) {
  if (!p || B < 0 || B > p->bmax) return HPSCD_ERR_INVALID_ARG;
  if (B > 0 && (!theta || !m || !n)) return HPSCD_ERR_INVALID_ARG;
  return HPSCD_OK;
}

struct DevSet {
  int prev = -1;
  bool ok = false;
  explicit DevSet(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = prev == dev || cudaSetDevice(dev) == cudaSuccess;
  }
  ~DevSet() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int finish(hpscd_mlp* p) {
  int err = 0;
  if (cudaMemcpyAsync(&err, p->err, sizeof(int), cudaMemcpyDeviceToHost, p->ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(p->ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return HPSCD_ERR_CUDA;
  }
  return err ? HPSCD_ERR_TIMEOUT : HPSCD_OK;
}

}  // namespace

namespace hpscd {

static void free_mlp(hpscd_mlp* p) {
  hpscd_ctx* ctx = p->ctx;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device) cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(p->dev);
  delete p;
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  ctx_release(ctx);
}

int mlp_device(const hpscd_mlp* p) { return p->ctx->device; }

void mlp_retain(hpscd_mlp* p) { ++p->users; }

void mlp_release(hpscd_mlp* p) {
  if (--p->users == 0 && p->closing) free_mlp(p);
}

int mlp_enqueue_warm_start(hpscd_mlp* p, cudaStream_t st, const float* theta, const int64_t* m,
                           const int64_t* n, const hpscd_sys* sys, int64_t count) {
  for (int64_t b0 = 0; b0 < count; b0 += p->bmax) {
    const int B = (int)(count - b0 < p->bmax ? count - b0 : p->bmax);
    const int Bp = (B + MT - 1) / MT * MT;
    int rc = forward(p, st, theta + b0 * THETA, m + b0, n + b0, B, Bp, false);
    if (rc) return rc;
    mlp_scatter_kernel<<<B, 256, 0, st>>>(p->out, sys, b0, B);
    if (cudaGetLastError() != cudaSuccess) return HPSCD_ERR_CUDA;
  }
  return HPSCD_OK;
}

}  // namespace hpscd

extern "C" {

int hpscd_mlp_create(hpscd_ctx* ctx, int64_t max_batch, hpscd_mlp** out) {
  if (!ctx || !out || max_batch < 1 || max_batch > (1 << 20)) return HPSCD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!ctx->encode) return HPSCD_ERR_UNSUPPORTED;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return HPSCD_ERR_CUDA;
  hpscd_mlp* p = new (std::nothrow) hpscd_mlp();
  if (!p) return HPSCD_ERR_NO_MEMORY;
  p->ctx = ctx;
  p->bmax = (int)((max_batch + MT - 1) / MT * MT);
  const size_t Bm = (size_t)p->bmax;
  size_t off = 0;
  size_t o_w[6], o_g[6], o_m[6], o_v[6];
  for (int i = 0; i < 6; ++i) {
    o_w[i] = off; off = al256(off + param_count(i) * 4);
    o_g[i] = off; off = al256(off + param_count(i) * 4);
    o_m[i] = off; off = al256(off + param_count(i) * 4);
    o_v[i] = off; off = al256(off + param_count(i) * 4);
  }
  auto take = [&](size_t bytes) { const size_t at = off; off = al256(off + bytes); return at; };
  const size_t o_w1b = take((size_t)HID * IN_P * 2), o_w2b = take((size_t)HID * HID * 2),
               o_w2t = take((size_t)HID * HID * 2), o_w3b = take((size_t)OUT_F * HID * 2),
               o_w3t = take((size_t)OUT_F * HID * 2);
  const size_t o_phi = take(Bm * IN_P * 2), o_phiT = take(Bm * IN_P * 2), o_h1 = take(Bm * HID * 2),
               o_h1T = take(Bm * HID * 2), o_h2 = take(Bm * HID * 2), o_h2T = take(Bm * HID * 2),
               o_dout = take(Bm * OUT_F * 2), o_doutT = take(Bm * OUT_F * 2), o_dz2 = take(Bm * HID * 2),
               o_dz2T = take(Bm * HID * 2), o_dz1T = take(Bm * HID * 2), o_out = take(Bm * OUT_F * 4),
               o_mb = take(Bm * 8), o_nb = take(Bm * 8), o_loss = take(8), o_err = take(8);
  if (cudaMalloc(&p->dev, off) != cudaSuccess) {
    cudaGetLastError();
    delete p;
    if (prev >= 0) cudaSetDevice(prev);
    return HPSCD_ERR_NO_MEMORY;
  }
  char* b = static_cast<char*>(p->dev);
  for (int i = 0; i < 6; ++i) {
    p->w[i] = reinterpret_cast<float*>(b + o_w[i]);
    p->g[i] = reinterpret_cast<float*>(b + o_g[i]);
    p->mo[i] = reinterpret_cast<float*>(b + o_m[i]);
    p->vo[i] = reinterpret_cast<float*>(b + o_v[i]);
  }
  auto u16 = [&](size_t o) { return reinterpret_cast<uint16_t*>(b + o); };
  p->w1b = u16(o_w1b); p->w2b = u16(o_w2b); p->w2t = u16(o_w2t); p->w3b = u16(o_w3b); p->w3t = u16(o_w3t);
  p->phi = u16(o_phi); p->phiT = u16(o_phiT); p->h1 = u16(o_h1); p->h1T = u16(o_h1T);
  p->h2 = u16(o_h2); p->h2T = u16(o_h2T); p->dout = u16(o_dout); p->doutT = u16(o_doutT);
  p->dz2 = u16(o_dz2); p->dz2T = u16(o_dz2T); p->dz1T = u16(o_dz1T);
  p->out = reinterpret_cast<float*>(b + o_out);
  p->mbuf = reinterpret_cast<int64_t*>(b + o_mb);
  p->nbuf = reinterpret_cast<int64_t*>(b + o_nb);
  p->loss = reinterpret_cast<double*>(b + o_loss);
  p->err = reinterpret_cast<int*>(b + o_err);
  const int bm = p->bmax;
  bool ok = cudaMemsetAsync(p->dev, 0, off, ctx->stream) == cudaSuccess &&
            cudaStreamSynchronize(ctx->stream) == cudaSuccess;
  // operand maps: A operands are read in 128-row boxes, B operands in N-row boxes
  ok = ok && encode_bf16(ctx, &p->m_phi, p->phi, bm, IN_P, MT) &&
       encode_bf16(ctx, &p->m_w1, p->w1b, HID, IN_P, HID) &&
       encode_bf16(ctx, &p->m_h1, p->h1, bm, HID, MT) &&
       encode_bf16(ctx, &p->m_w2, p->w2b, HID, HID, HID) &&
       encode_bf16(ctx, &p->m_h2, p->h2, bm, HID, MT) &&
       encode_bf16(ctx, &p->m_w3, p->w3b, OUT_F, HID, OUT_F) &&
       encode_bf16(ctx, &p->m_dout, p->dout, bm, OUT_F, MT) &&
       encode_bf16(ctx, &p->m_doutT, p->doutT, OUT_F, bm, MT) &&
       encode_bf16(ctx, &p->m_h2T, p->h2T, HID, bm, HID) &&
       encode_bf16(ctx, &p->m_w3t, p->w3t, HID, OUT_F, HID) &&
       encode_bf16(ctx, &p->m_dz2, p->dz2, bm, HID, MT) &&
       encode_bf16(ctx, &p->m_dz2T, p->dz2T, HID, bm, MT) &&
       encode_bf16(ctx, &p->m_h1T, p->h1T, HID, bm, HID) &&
       encode_bf16(ctx, &p->m_w2t, p->w2t, HID, HID, HID) &&
       encode_bf16(ctx, &p->m_dz1T, p->dz1T, HID, bm, MT) &&
       encode_bf16(ctx, &p->m_phiT, p->phiT, IN_P, bm, IN_P);
  ok = ok && cudaFuncSetAttribute(mlp_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  gemm_smem(256)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    cudaFree(p->dev);
    delete p;
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return HPSCD_ERR_CUDA;
  }
  if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  ctx_retain(ctx);
  *out = p;
  return HPSCD_OK;
}

int hpscd_mlp_destroy(hpscd_mlp* p) {
  if (!p) return HPSCD_OK;
  if (p->users > 0) {
    p->closing = true;
    return HPSCD_OK;
  }
  free_mlp(p);
  return HPSCD_OK;
}

// Host parameter vector: W1 [256][18], b1 [256], W2 [256][256], b2 [256],
// W3 [256][256], b3 [256] (row-major, float32).
int hpscd_mlp_set_params(hpscd_mlp* p, const float* host_params) {
  if (!p || !host_params) return HPSCD_ERR_INVALID_ARG;
  DevSet g(p->ctx->device);
  if (!g.ok) return HPSCD_ERR_CUDA;
  cudaStream_t st = p->ctx->stream;
  size_t off = 0;
  for (int i = 0; i < 6; ++i) {
    const size_t cnt = param_count(i);
    cudaError_t e;
    if (i == 0) {
      e = cudaMemsetAsync(p->w[0], 0, cnt * 4, st);
      if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(p->w[0], IN_P * 4, host_params, IN_F * 4, IN_F * 4, HID,
                              cudaMemcpyHostToDevice, st);
      off += (size_t)HID * IN_F;
    } else {
      e = cudaMemcpyAsync(p->w[i], host_params + off, cnt * 4, cudaMemcpyHostToDevice, st);
      off += cnt;
    }
    if (e != cudaSuccess || cudaMemsetAsync(p->mo[i], 0, cnt * 4, st) != cudaSuccess ||
        cudaMemsetAsync(p->vo[i], 0, cnt * 4, st) != cudaSuccess)
      return HPSCD_ERR_CUDA;
  }
  mlp_cast_kernel<<<(HID * IN_P + 255) / 256, 256, 0, st>>>(p->w[0], HID * IN_P, HID, IN_P, p->w1b, nullptr);
  mlp_cast_kernel<<<(HID * HID + 255) / 256, 256, 0, st>>>(p->w[2], HID * HID, HID, HID, p->w2b, p->w2t);
  mlp_cast_kernel<<<(OUT_F * HID + 255) / 256, 256, 0, st>>>(p->w[4], OUT_F * HID, OUT_F, HID, p->w3b, p->w3t);
  p->step = 0;
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return HPSCD_ERR_CUDA;
  return HPSCD_OK;
}

static int copy_params_out(hpscd_mlp* p, float* const src[6], float* host) {
  if (cudaStreamSynchronize(p->ctx->stream) != cudaSuccess) return HPSCD_ERR_CUDA;
  size_t off = 0;
  for (int i = 0; i < 6; ++i) {
    cudaError_t e;
    if (i == 0) {
      e = cudaMemcpy2D(host, IN_F * 4, src[0], IN_P * 4, IN_F * 4, HID, cudaMemcpyDeviceToHost);
      off += (size_t)HID * IN_F;
    } else {
      e = cudaMemcpy(host + off, src[i], param_count(i) * 4, cudaMemcpyDeviceToHost);
      off += param_count(i);
    }
    if (e != cudaSuccess) return HPSCD_ERR_CUDA;
  }
  return HPSCD_OK;
}

int hpscd_mlp_get_params(hpscd_mlp* p, float* host_params) {
  if (!p || !host_params) return HPSCD_ERR_INVALID_ARG;
  DevSet g(p->ctx->device);
  return g.ok ? copy_params_out(p, p->w, host_params) : HPSCD_ERR_CUDA;
}

int64_t hpscd_mlp_param_count(void) {
  return (int64_t)HID * IN_F + HID + (int64_t)HID * HID + HID + (int64_t)OUT_F * HID + OUT_F;
}

int hpscd_mlp_predict(hpscd_mlp* p, const float* theta, const int64_t* m, const int64_t* n,
                      int64_t B, float* out) {
  int rc = check_io(p, theta, m, n, B);
  if (rc) return rc;
  if (B > 0 && !out) return HPSCD_ERR_INVALID_ARG;
  DevSet g(p->ctx->device);
  if (!g.ok) return HPSCD_ERR_CUDA;
  if (B == 0) return HPSCD_OK;
  cudaStream_t st = p->ctx->stream;
  const int Bp = (int)((B + MT - 1) / MT * MT);
  if (cudaMemsetAsync(p->err, 0, sizeof(int), st) != cudaSuccess) return HPSCD_ERR_CUDA;
  if ((rc = stage_shapes(p, m, n, (int)B, nullptr))) return rc;
  if ((rc = forward(p, st, theta, p->mbuf, p->nbuf, (int)B, Bp, false))) return rc;
  if (cudaMemcpyAsync(out, p->out, (size_t)B * OUT_F * 4, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return HPSCD_ERR_CUDA;
  return finish(p);
}

static int loss_and_grads(hpscd_mlp* p, const float* theta, const int64_t* m, const int64_t* n,
                          const float* target, int64_t B, double* loss) {
  int rc = check_io(p, theta, m, n, B);
  if (rc) return rc;
  if (B < 1 || !target) return HPSCD_ERR_INVALID_ARG;
  cudaStream_t st = p->ctx->stream;
  const int Bp = (int)((B + MT - 1) / MT * MT);
  double inv_count = 0.0;
  if (cudaMemsetAsync(p->err, 0, sizeof(int), st) != cudaSuccess) return HPSCD_ERR_CUDA;
  if ((rc = stage_shapes(p, m, n, (int)B, &inv_count))) return rc;
  if ((rc = forward(p, st, theta, p->mbuf, p->nbuf, (int)B, Bp, true))) return rc;
  if ((rc = backward(p, st, target, (int)B, Bp, inv_count))) return rc;
  if (loss && cudaMemcpyAsync(loss, p->loss, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return HPSCD_ERR_CUDA;
  return HPSCD_OK;
}

int hpscd_mlp_gradients(hpscd_mlp* p, const float* theta, const int64_t* m, const int64_t* n,
                        const float* target, int64_t B, double* loss, float* host_grads) {
  if (!host_grads) return HPSCD_ERR_INVALID_ARG;
  DevSet g(p ? p->ctx->device : 0);
  if (!g.ok) return HPSCD_ERR_CUDA;
  int rc = loss_and_grads(p, theta, m, n, target, B, loss);
  if (rc) return rc;
  if ((rc = finish(p))) return rc;
  return copy_params_out(p, p->g, host_grads);
}

int hpscd_mlp_train_step(hpscd_mlp* p, const float* theta, const int64_t* m, const int64_t* n,
                         const float* target, int64_t B, float lr, float beta1, float beta2,
                         float eps, double* loss) {
  if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return HPSCD_ERR_INVALID_ARG;
  DevSet g(p ? p->ctx->device : 0);
  if (!g.ok) return HPSCD_ERR_CUDA;
  int rc = loss_and_grads(p, theta, m, n, target, B, loss);
  if (rc) return rc;
  p->step += 1;
  const float c1 = (float)(1.0 - pow((double)beta1, (double)p->step));
  const float c2 = (float)(1.0 - pow((double)beta2, (double)p->step));
  cudaStream_t st = p->ctx->stream;
  for (int i = 0; i < 6; ++i) {
    const int cnt = (int)param_count(i);
    uint16_t* wb = i == 0 ? p->w1b : (i == 2 ? p->w2b : (i == 4 ? p->w3b : nullptr));
    uint16_t* wbT = i == 2 ? p->w2t : (i == 4 ? p->w3t : nullptr);
    const int cols = kParamCols[i];
    mlp_adam_kernel<<<(cnt + 255) / 256, 256, 0, st>>>(p->w[i], p->g[i], p->mo[i], p->vo[i], cnt,
                                                      kParamRows[i], cols, i == 0 ? IN_F : cols, lr,
                                                      beta1, beta2, eps, c1, c2, wb, wbT);
  }
  if (cudaGetLastError() != cudaSuccess) return HPSCD_ERR_CUDA;
  return finish(p);
}

}  // extern "C"
