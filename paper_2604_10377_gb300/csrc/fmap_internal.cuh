// Internal declarations shared by the functional-map CUDA sources.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/fmap.h"

namespace fmap {

constexpr int kMaxK = 304;
// per-pair partial sums of the training loss: one per 64 x 64 tile of C
constexpr int kMaxLossTiles = ((kMaxK + 63) / 64) * ((kMaxK + 63) / 64);
constexpr int kMaxD = 4096;

// Device copy of a shape descriptor plus the offsets the library assigns to it.
struct ShapeDev {
  int64_t n;
  int32_t k, d;
  const float* phi;
  int64_t ld_phi;
  const float* mass;
  const float* evals;
  const void* feat;
  int64_t ld_feat;
  void* dfeat;
  float* dfeat32;      // optional FP32 copy of dF before rounding (BF16 batches), row stride ld_feat
  int64_t a_off;       // float offset of A_s in the flat A buffer
  int32_t slot_beg;    // [slot_beg, slot_end): entries of slot_list holding dA contributions
  int32_t slot_end;
};

// Device copy of a pair descriptor plus workspace offsets.
// Row stride (floats) of the FP32 Gram matrix G in the workspace: k rounded up to a
// multiple of 4 (every row starts on a 16-byte boundary, for bulk copies into shared
// memory) with an odd number of 16-byte quads (rows read by consecutive threads as
// float4 then fall on distinct bank groups).
__host__ __device__ __forceinline__ int gram_ld(int k) {
  const int q = (k + 3) >> 2;
  return 4 * (q | 1);
}

// Packed, skewed lower storage of a row system (the row solves' shared-memory layout):
// row a holds columns 0 .. (a | 7), i.e. up to the end of its 8 x 8 diagonal block, in
// 8 (a / 8 + 1) + 4 floats, so a row's 8-column segment is two aligned float4 and
// consecutive rows of a block start on different banks. rowoff(a) is the offset of row
// a; rowoff(a) is a multiple of 4 for every a.
__host__ __device__ __forceinline__ int rowoff(int a) {
  const int q = a >> 3, s = a & 7;
  return 32 * q * (q + 2) + s * (8 * q + 12);
}

// The Gram region of a pair: G row-major (k rows of gram_ld(k) floats, then 8 floats of
// slack), then, from gram_packed_off(k) (a multiple of 32 floats), rows 0 .. k-1 of G
// in the packed layout above (rowoff(k) floats), which the row solves copy into shared
// memory with one bulk copy.
__host__ __device__ __forceinline__ int64_t gram_packed_off(int k) {
  return ((int64_t)k * gram_ld(k) + 8 + 31) / 32 * 32;
}
__host__ __device__ __forceinline__ int64_t gram_floats(int k) { return gram_packed_off(k) + rowoff(k); }

struct PairDev {
  int32_t x, y;
  int32_t k, d;
  float lam;
  int32_t hi_gram;     // 1: Gram matrix accumulated in FP64
  const float* mask;   // k x k or nullptr (use eigenvalues)
  const float* lam_rows;   // k_Y weights, one per row system (in place of lam), or nullptr
  float* dlam_rows;        // k_Y outputs dL/dlambda_i (with lam_rows), or nullptr
  int64_t c_off;       // float offset of C_p / dC_p in the flat k x k buffers
  int64_t g_off;       // float offset (workspace) of G = A_x A_x^T  (k x k, row stride gram_ld(k))
  int64_t r_off;       // float offset (workspace) of R = A_y A_x^T  (k x k)
  int64_t g64_off;     // float2 offset (workspace) of the double-float (hi, lo) Gram, or -1
  int64_t gam_off;     // float offset (workspace) of Gamma (k x k)
  int64_t w_off;       // float offset (workspace) of W = Gamma^T C + C^T Gamma (k x k)
  int64_t e_off;       // float offset (workspace) of E = C C^T - I (k x k)
  int64_t sx_off;      // float offset (workspace) of this pair's dA_x contribution (k x d)
  int64_t sy_off;      // float offset (workspace) of this pair's dA_y contribution (k x d)
  int64_t fac_off;     // float offset of saved factors (k packed triangles), or -1
};

struct BatchDev {
  const ShapeDev* shapes;
  const PairDev* pairs;
  const int64_t* slot_list;     // workspace float offsets of dA contributions, grouped per shape
  int32_t n_shapes, n_pairs;
  int32_t feat_bf16;
  int32_t ir_steps;       // refinement steps of the forward row solves
  int32_t ir_steps_adj;   // refinement steps of the adjoint row solves
};

__host__ __device__ inline int64_t tri(int64_t k) { return k * (k + 1) / 2; }

// Segment of the tensor-core projection: a vertex range of one feature group
// (fg M-tiles of 128 features starting at feature f0) of one shape.
struct TcItem {
  int32_t shape, f0, fg, npad;
  int32_t n0, nk;      // basis rows n0 .. n0+nk of A (npad = nk rounded up to 16)
  int64_t v0, v1;
  int64_t part_off;    // float offset (workspace) of the segment's partial, nk x (fg*128)
};

// Items [it_beg, it_end) hold the partials of basis rows n0 .. n0+nk and features
// f0 .. f0+dspan of one shape.
struct TcRedGroup {
  int32_t shape, f0, dspan, stride;
  int32_t n0, nk;
  int32_t it_beg, it_end;
};

struct TcProjParams {
  const ShapeDev* shapes;
  const CUtensorMap* fmaps;     // per shape: features, BF16 box 64 x 64 or FP32 box 32 x 32 (features x
                                //   vertices), 128-byte swizzle
  const CUtensorMap* phimaps;   // per shape: FP32 basis, box 32 basis x (64 or 32) vertices, 128-byte swizzle
  const CUtensorMap* massmaps;  // per shape: FP32 mass, 1-D box of 64 or 32
  const TcItem* items;          // segments, grouped by CTA
  const int32_t* cta_first;     // CTA c owns segments [cta_first[c], cta_first[c + 1])
  int32_t stages;
  uint32_t f_stage_bytes;
  uint32_t p_stage_bytes;
  uint32_t tmem_cols;
  float* ws;
  int* err;                   // workspace error word
};

// Work item of the tensor-core backward projection: a vertex chunk of one feature
// group (nf <= 128 features from f0) of one shape; kb = blocks of 32 basis functions.
struct TcBwdItem {
  int32_t shape, f0, nf, kb;
  int64_t v0, v1;
  int64_t img_off;     // float offset (workspace) of the group's dA^T image
};

struct TcBwdGroup {
  int32_t shape, f0, nf, kb;
  int64_t img_off;
};

struct TcBwdParams {
  const ShapeDev* shapes;
  const CUtensorMap* phimaps;  // per shape: FP32 Phi, box 32 x 64, 128-byte swizzle
  const CUtensorMap* dfmaps;   // per shape: dF (BF16 or FP32), box 16 x 32, no swizzle (TMA stores)
  const TcBwdItem* items;       // BF16: item j of CTA pair c is [2 j] for CTA 2c, [2 j + 1] for CTA 2c + 1;
                                //   FP32: one item per entry
  const int32_t* cta_first;     // BF16: CTA pair c owns items [cta_first[c], cta_first[c + 1]);
                                //   FP32: CTA c
  int32_t stages;
  uint32_t b_bytes_max;
  uint32_t tmem_cols;
  const float* ws;
  int* err;
};

cudaError_t project_bwd_tc_set_smem(int bytes);
cudaError_t launch_build_dat_image(const ShapeDev* shapes, const TcBwdGroup* groups, int n_groups, int max_elems,
                                   const float* d_a, float* ws, cudaStream_t st);
cudaError_t launch_project_bwd_tc(const TcBwdParams& p, int grid, int smem_bytes, cudaStream_t st);
cudaError_t project_bwd_tc32_set_smem(int bytes);
cudaError_t launch_build_dat_image32(const ShapeDev* shapes, const TcBwdGroup* groups, int n_groups, int max_elems,
                                     const float* d_a, float* ws, cudaStream_t st);
cudaError_t launch_project_bwd_tc32(const TcBwdParams& p, int grid, int smem_bytes, cudaStream_t st);

cudaError_t project_tc_set_smem(int bytes);
cudaError_t project_tc32_set_smem(int bytes);
cudaError_t launch_project_tc32(const TcProjParams& p, int grid, int smem_bytes, cudaStream_t st);
int project_tc_threads();
cudaError_t launch_project_tc(const TcProjParams& p, int grid, int smem_bytes, cudaStream_t st);
cudaError_t launch_project_tc_reduce(const ShapeDev* shapes, const TcItem* items, const TcRedGroup* groups,
                                     int n_groups, int64_t max_elems, float* a_out, const float* ws,
                                     cudaStream_t st);

// ---- launchers (each enqueues on `st`; return cudaError_t of the launch) ----
// with_r = false computes G only (the adjoint solves never read R)
cudaError_t launch_gram(const BatchDev& b, int max_k, const float* a, float* ws, cudaStream_t st,
                        bool with_r = true);

struct SolveGroup {
  int32_t first;     // index into the system list
  int32_t count;     // systems in this group
  int32_t kmax;      // largest k in the group
  int32_t threads;
  int32_t no_g_copy; // 1: no shared-memory copy of G for the refinement residual (the residual
                     // then reads G from L2); 0: the built-in rule, a copy for k <= 128
};

enum SolveMode { kSolveForward = 0, kSolveAdjoint = 1 };

cudaError_t launch_solve(const BatchDev& b, const SolveGroup& g, const int2* systems, int mode,
                         const float* rhs_flat, float* out_flat, float* saved_rw, int32_t* status,
                         float* ws, cudaStream_t st);
// The mask and lambda gradients (when d_mask / d_lambda are given, or a pair has per-row
// lambda outputs: row_grads) and, with simt, W and the dA contributions on the CUDA cores
// (FP32 FMA tiles)
cudaError_t launch_adjoint_gemms(const BatchDev& b, int max_k, int max_d, const float* a, const float* c,
                                 float* d_mask, float* d_lambda, bool row_grads, float* ws, bool simt,
                                 cudaStream_t st);

// One CTA of the tensor-core adjoint GEMMs: output rows r0 .. r0+127 and columns f0 .. f0+NT-1
// of W (kind 2), dA_y (kind 1) or dA_x (kind 0) of one pair.
struct AdjItem {
  int32_t pair, kind, r0, f0;
};
struct AdjTcPlan {
  std::vector<AdjItem> items;   // the first launch's n_first items (kinds 2, 1), then kind 0
  int n_first = 0;
  int stages = 0;               // shared-memory stages, 1 or 2 (0 on input: the built-in choice)
  int features = 0;             // output columns per CTA, 64, 128 or 256 (0 on input: built-in)
  bool fills_sms = false;       // at least two dA_x tiles of 128 columns per SM
};
// shapes[p] = (k_X, k_Y, d) of pair p; fills the work list, longest reduction first
void adjoint_tc_plan(const std::vector<int3>& shapes, int sms, AdjTcPlan& P);
cudaError_t launch_adjoint_tc(const BatchDev& b, const AdjItem* items, const AdjTcPlan& P, const float* a,
                              const float* c, float* ws, cudaStream_t st);
cudaError_t adjoint_tc_set_smem();
cudaError_t launch_gather_da(const BatchDev& b, int max_kd, float* d_a, const float* ws, cudaStream_t st);
cudaError_t launch_loss_orth(const BatchDev& b, int max_k, const float* c, const float* c_gt, float* loss,
                             float* d_c, float* ws, float* partial, cudaStream_t st);
cudaError_t launch_status_clear(int32_t* status, int n, cudaStream_t st);
cudaError_t solve_set_smem_limits();
int64_t chol_factor_floats(int k);   // saved factor size of one row system (padded packed rows)

}  // namespace fmap
