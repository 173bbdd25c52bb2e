// Internal launch interface between the C-ABI layer and the CUDA kernels.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace hpscd {

// Tensor-map element type of a stored X (TMA copies only its bytes; the type
// fixes the element size).
inline CUtensorMapDataType x_tmap_type(int dtype) {
  return dtype == HPSCD_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
         : dtype == HPSCD_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                               : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
}

// ---- Gram set-up: G = X^T X (lower triangle incl. diagonal), G_jj = <X_j, X_j> ----
struct GramPlan {
  int npad;         // padded column count (multiple of 64)
  int ntile;        // lower-triangular 64x64 tiles
  int ksplit;       // row splits
  int64_t rows_per_split;
  size_t partial_bytes;  // float64 partial tiles
};
GramPlan gram_plan(int64_t m, int npad, int sms);
GramPlan gram_plan_capped(int64_t m, int npad, int sms, int max_ksplit);  // <= max_ksplit splits
cudaError_t launch_gram(const void* X, int dtype, int64_t m, int n, int64_t ld, const GramPlan& gp,
                        double* partial, float* G, int ldG, cudaStream_t stream);

// ---- tensor-core Gram set-up (tcgen05), G = X^T X ----
// A group is a set of at most 4 lower 128×128 tiles (I, J) of G (one TMEM
// accumulator of 128 columns each) computed by one CTA from the column blocks
// it streams (slots of a stage, at most 4).
constexpr int GTC_MAX_GROUPS = 8;
struct GramTCGroups {
  int ngroups;
  int ntile[GTC_MAX_GROUPS];
  int tile_si[GTC_MAX_GROUPS][4];   // slot of block I of each tile
  int tile_sj[GTC_MAX_GROUPS][4];   // slot of block J
  int tile_i[GTC_MAX_GROUPS][4];    // block I (rows of G)
  int tile_j[GTC_MAX_GROUPS][4];    // block J (columns of G)
  int nload[GTC_MAX_GROUPS];
  int load_blk[GTC_MAX_GROUPS][4];  // column block streamed into each slot
  int diag_slot[GTC_MAX_GROUPS][4]; // 1 when the group holds tile (b, b) of the block in that slot
  // row splits: group g runs nsplit[g] CTAs (linear indices split_base[g]..), each over
  // rows_per[g] rows, in proportion to its work per K block
  int nsplit[GTC_MAX_GROUPS];
  int split_base[GTC_MAX_GROUPS];
  int64_t rows_per[GTC_MAX_GROUPS];
  int tile_splits[4][4];            // nsplit of the group that holds lower tile (I, J)
  // float32 only: 1 when the group holds the full square of its column blocks
  // (both (I, J) and (J, I)), accumulated with two products and symmetrized
  int sym[GTC_MAX_GROUPS];
};
struct GramTCPlan {
  int npad;                 // multiple of 128
  GramTCGroups grp;
  int maxload;
  int ksplit;               // the most row splits of a group (partial buffers per split)
  int nctas;                // CTAs of the launch (the splits of every group)
  int64_t rows_per_split;
  int nstages;
  int smem_bytes;
  size_t partial_bytes;     // float32 partials [ksplit][npad][npad] + float64 [ksplit][npad]
};
struct GramTCParams {
  int64_t m;
  int npad;
  GramTCGroups grp;
  int64_t rows_per_split;
  float* partial;
  double* dpart;   // [ksplit][npad] CUDA-core sums of squares (the diagonal)
  int* err;
  uint64_t timeout_ns;
  int nstages;
  const float* y;   // or null: also form X^T y and ||y||^2
  int y_tma;        // 1: y's K blocks arrive by TMA with the stages (y 16-byte aligned)
  double* hpart;    // [ksplit][npad] per-split X^T y (the diagonal tiles' workers)
  double* y2part;   // [ksplit] per-split ||y||^2
};
bool gram_tc_plan(int dtype, int64_t m, int n, int sms, int max_smem, GramTCPlan* gp);
// G = X^T X into G (ldG); when Gt is given, also G~ = D^{-1} G (ldG, rows and
// columns >= n zero) and d = diag(G) (float32, dvec).  When y, h0 and y2 are
// given, also h0 = X^T y (float64 [npad]) and *y2 = ||y||^2 (float64).
cudaError_t launch_gram_tc(const CUtensorMap* tmap, int dtype, int64_t m, const GramTCPlan& gp,
                           float* partial, int* err, uint64_t timeout_ns, float* G, int ldG,
                           cudaStream_t stream, int n, float* Gt, float* dvec,
                           const float* y = nullptr, double* h0 = nullptr, double* y2 = nullptr,
                           const CUtensorMap* ymap = nullptr);

// ---- persistent tall sweep (column-major X, n <= 512) ----
constexpr int MODE_COPY = 0, MODE_NORMAL = 1, MODE_REFRESH = 2;

struct TallParams {
  const void* X;
  int64_t m;
  int n;
  int64_t ld;
  const float* y;
  float* e;
  float* a_out;
  const float* a_in;
  int warm;
  const float* Gt;     // G~ = D^{-1} G: row j of G divided by G_jj (0 for a zero
                       // column), row-major, leading dimension ldG, columns n..ldG-1 zero
  const float* dvec;   // d = diag(G) [n]
  int ldG;
  double* hacc;        // [3][npad]: X^T e_in of a pass, accumulated over the CTAs
                       // (float64 atomics); zero-filled by the host
  double* npart;       // [2][grid]
  float* gw;           // [2][npad]: G~·w rows published by the CTAs
  double* ypart;   // [grid]
  double* hist;    // [max_sweeps + 1]
  GridCtl* ctl;
  double tol;
  int64_t max_sweeps;
  int stop_rule;
  int refresh_every;
  int64_t ntiles;  // 128-row panels
  int nstages;
  int use_tma;
  uint64_t timeout_ns;
  int stall_barrier;  // test hook: first barrier waits for one arrival too many
  int thr;            // > 1: Algorithm 2 — columns in blocks of thr take their steps from
                      // the same residual (no couplings inside a block); <= 1: Algorithm 1
  int select;         // 1: Algorithm 3 — each pass adds the one column with the largest
                      // <X_j,e>^2 / <X_j,X_j> (greedy selection) instead of a sweep
  int64_t* sel_out;   // Algorithm 3: column chosen after pass p, [max_sweeps]
  int swap_rounds;    // Algorithm 3 then at most this many swap steps (Sec. 8's removal loop)
  int64_t* swap_out;  // the (dropped, added) pair of each swap step, [swap_rounds][2]; -1: none
  const int* order;   // or null: step k of sweep s takes column order[(s-1)·n + k]
                      // ([max_sweeps][n], each in [0, n); the random-index variant)
  unsigned long long* trace;  // optional: per-pass phase timestamps (see hpscd_trace)
  int trace_passes;           // capacity of trace in passes
  const double* h0;   // or null: X^T y of a cold start from the set-up (float64 [npad]);
                      // pass 0 then reads nothing (e_0 = y, r_0 = h0 ⊘ d)
  const double* y2;   // ||y||^2 (float64), given with h0
  int confirm;        // 1: under REL_RES a tracked residual at the tolerance is confirmed
                      // by a pass that recomputes e = y - X·a of the returned a
  int e_smem;         // 1: the residual of the CTA's rows stays in shared memory (after the
                      // kernel's other buffers); 0: e lives in HBM (p.e)
};

struct TallConfig {
  int cpw;   // columns per warp per chunk (CW)
  int rpl;   // chunks per 128-row panel (NCH)
  int npad, rows, stage_bytes, box_cols, nstages, smem_bytes, threads;
};
bool tall_config(int dtype, int n, int max_smem, TallConfig* cfg);
// G~ = D^{-1} G and d = diag(G) from the Gram matrix G (n×n, ldG), columns n..ldG-1 of G~ zeroed.
cudaError_t launch_scale_rows(const float* G, int ldG, int n, float* Gt, float* d, cudaStream_t stream);
cudaError_t launch_tall_sweep(int dtype, const TallConfig& cfg, const CUtensorMap* tmap,
                              const TallParams& p, int grid, cudaStream_t stream);
// The IEEE binary16 instantiations (tall_sweep_f16.cu).
cudaError_t launch_tall_sweep_f16(const TallConfig& cfg, const CUtensorMap* tmap, const TallParams& p,
                                  int grid, cudaStream_t stream);

// ---- set-up relayouts (relayout.cu) ----
// out (column-major, leading dimension ldo) = X (row-major, ld), element bits copied.
cudaError_t launch_transpose_to_col(const void* X, int dtype, int64_t m, int64_t n, int64_t ld, void* out,
                                    int64_t ldo, int sms, cudaStream_t stream);
// out (row-major float32, ldo) = X (row-major bfloat16 or binary16, ld), widened exactly.
cudaError_t launch_widen_rows(const void* X, int dtype, int64_t m, int64_t n, int64_t ld, float* out,
                              int64_t ldo, int sms, cudaStream_t stream);

// ---- panel sweep (column-major X, n > 512): panels of PANEL_W columns ----
constexpr int PANEL_W = 512;
constexpr int PANEL_BOX_BYTES = 65536;  // TMA box of the panel sweep: 128 rows x 64 KB of columns
struct PanelParams {
  const void* X;         // column-major, leading dimension ld
  int64_t m;
  int n;
  int64_t ld;
  int vec;               // X and ld allow 16-byte (float32) / 8-byte (16-bit) row loads
  const float* y;
  float* e;              // [ceil(m/128)·128] residual (rows past m kept zero)
  const float* a_in;     // the initial guess when warm
  int warm;
  float* a_out;          // [n] float32 coefficients returned
  double* a64;           // [n] float64 coefficients
  const float* Gt;       // [npanels][PANEL_W][PANEL_W] G~ = D^{-1} G of each panel's diagonal block
  const float* dvec;     // [npanels·PANEL_W] d = diag(G)
  int npanels;
  double* hacc;          // [3][PANEL_W] a pass's dot products (float64 atomics); zeroed by the host
  double* npart;         // [2][grid] ||e||^2 partials
  double* ypart;         // [grid] ||y||^2 partials
  double* hist;          // [max_sweeps + 1]
  GridCtl* ctl;
  double tol;
  int64_t max_sweeps;
  int stop_rule;
  int refresh_every;
  uint64_t timeout_ns;
  int stall_barrier;     // test hook: the first grid barrier waits for one arrival too many
  int use_tma;           // 1: X streams by TMA (tensor map: dims {m, n}, boxes of 128 rows x
                         // PANEL_BOX_BYTES / (128·elem) columns), else plain loads
  int nstages;           // TMA stages (PANEL_BOX_BYTES each)
};
int panel_tma_smem(int nst);  // dynamic shared memory of the TMA kernel
// The panels' G~ blocks (npanels × PANEL_W²): each 32 × 32 diagonal block's
// strictly lower part replaced in place by that of its unit lower triangular inverse.
cudaError_t launch_invert_panel_diag(float* Gt, int npanels, cudaStream_t stream);
cudaError_t launch_panel_sweep(int dtype, const PanelParams& p, const CUtensorMap* tmap, int grid,
                               cudaStream_t stream);

// ---- wide sweep (row-major X, m <= 4096): one thread-block cluster ----
struct WideParams {
  const float* X;    // row-major X (plain-load path)
  int use_tma;
  int64_t m, n, ld;
  float* Mb;         // [nblk][W][W] M_b = (I + D^-1 L_b)^-1 D^-1 of each column block (set-up)
  float* Nb;         // [nblk][W][W] N_b = M_b·(X_b^T X_{b-1}), the coupling to the previous block
  float* e;          // [m] residual (in: initial; out: final)
  double* a64;       // [n] coefficients
  float* dsw;        // [n] da of the current sweep
  float* a_out;      // [n]
  double* ysq;       // ||y||^2 (device)
  double* hist;
  GridCtl* ctl;
  double tol;
  int64_t max_sweeps;
  int stop_rule;
  int csize, rows_box, nstages;
  uint64_t timeout_ns;
  unsigned long long* trace;  // optional: per-block phase stamps of the first blocks
  int trace_passes;
  int continuing;             // 1: a continuation after a failed confirmation (no stop at sweep 0)
  double* rpart;              // [m][32] per-row float64 partials of a true-residual pass
};
struct WideConfig {
  int csize, rows_box, nstages, smem_bytes;
  int W;  // columns per block: 64, or 32 when a CTA owns more than 128 rows
};
bool wide_config(int64_t m, int max_smem, WideConfig* cfg);
cudaError_t launch_wide(const float* X, int64_t m, int64_t n, int64_t ld, const WideConfig& cfg,
                        const CUtensorMap* tmap, WideParams p, const float* y, const float* a_in,
                        int warm, float* a_tmp, cudaStream_t stream);
// e = y - X·a (Dot2, float64-grade) for the float32 a, and *sum = ||y - X·a||^2 (float64)
cudaError_t launch_wide_confirm(const float* X, int64_t m, int64_t n, int64_t ld, const float* y,
                                const float* a, float* e, double* part, double* r2, double* sum,
                                cudaStream_t stream);
// sweeps on from the residual p.e of the coefficients p.a_out (after launch_wide_confirm)
cudaError_t launch_wide_continue(int64_t n, const WideConfig& cfg, const CUtensorMap* tmap,
                                 WideParams p, float* a_tmp, cudaStream_t stream);

// ---- batched sweep: many column-major systems, one persistent launch ----
struct BatchParams {
  const hpscd_sys* sys;     // device [count]
  const int* order;         // device [count]: queue order (decreasing m·n)
  int count;
  int* queue;               // device counter, zeroed before every launch
  hpscd_sys_result* res;    // device [count]
  float* gpart;             // [grid][256*256] partial Gram of each CTA
  float* gfinal;            // [clusters][256*256] G~ = D^{-1} G of each cluster's system
  int ecap;                 // residual rows held in shared memory per CTA
  int panel;                // columns per warp of a streaming pass: 0 narrowest, 1 twice, 2 sixteen
  double tol;
  int64_t max_sweeps;
  int stop_rule;
};
int batched_smem_bytes(int64_t mmax, int K);
int batched_ecap(int64_t mmax, int K);
int batched_max_clusters(int K, int smem, int max_smem);
cudaError_t launch_batched(const BatchParams& p, int K, int clusters, int smem, cudaStream_t stream);

}  // namespace hpscd
