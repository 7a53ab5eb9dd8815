// The training loss on the tensor-core GEMM kernel of the adjoint (k_adjoint_tc.cu):
// E = C C^T - I and dL/dC = 4 E C + 2 (C - C_gt) as its item kinds 3 and 4, 128 columns
// per CTA, and L_p = ||E||^2 + ||C - C_gt||^2 from their per-tile partials.
#pragma once

#include <vector>

#include "fmap_internal.cuh"

namespace fmap {

constexpr int kLossNt = 128;   // output columns per CTA of the loss GEMMs

// shapes[p] = (k_X, k_Y, d) of pair p: the loss items of every pair (E tiles first)
void adjoint_tc_loss_plan(const std::vector<int3>& shapes, AdjTcPlan& P);
// c, c_gt, d_c: flat buffers (c offsets); loss: float[n_pairs] or nullptr; partial: the
// batch's kMaxLossTiles floats per pair in the workspace; ws: E at each pair's e_off
cudaError_t launch_loss_tc(const BatchDev& b, const AdjItem* items, const AdjTcPlan& P, const float* c,
                           const float* c_gt, float* loss, float* d_c, float* ws, float* partial, cudaStream_t st);

}  // namespace fmap
