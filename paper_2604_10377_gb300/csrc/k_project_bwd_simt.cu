// Backward projection on the CUDA cores (FP32 FMA) for FP32 features (chain rule of
// Eq. 1): dF_s = diag(M_s) Phi_s dA_s, written in FP32. BF16 features take the
// tensor-core kernel; the FP32 output here is compared with finite differences of the
// FP64 pipeline at 1e-4, which a single TF32 pass would not meet.
#include "fmap_internal.cuh"

namespace fmap {
namespace {

constexpr int kTile = 64;   // output tile edge
constexpr int kStage = 16;  // basis functions per shared-memory stage

// dF tile: 64 vertices x 64 features, 4 x 4 per thread, basis functions staged 16 at a time.
__global__ void __launch_bounds__(256) project_bwd_simt_kernel(BatchDev b, const BwdTile* tiles, const float* d_a) {
  __shared__ float sP[kTile][kStage + 1];
  __shared__ float sA[kStage][kTile + 4];
  const BwdTile t = tiles[blockIdx.x];
  const ShapeDev s = b.shapes[t.shape];
  if (s.dfeat == nullptr) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const float* da = d_a + s.a_off;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int kk0 = 0; kk0 < s.k; kk0 += kStage) {
    for (int e = tid; e < kTile * kStage; e += 256) {
      const int vv = e / kStage, c = e % kStage;
      const int64_t v = t.v0 + vv;
      const int kk = kk0 + c;
      sP[vv][c] = (v < s.n && kk < s.k) ? s.phi[v * s.ld_phi + kk] : 0.f;
    }
    for (int e = tid; e < kStage * kTile; e += 256) {
      const int c = e / kTile, ff = e % kTile;
      const int kk = kk0 + c, f = t.f0 + ff;
      sA[c][ff] = (kk < s.k && f < s.d) ? da[(int64_t)kk * s.d + f] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kStage; ++c) {
      float pa[4], ab[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) pa[i] = sP[ty * 4 + i][c];
#pragma unroll
      for (int j = 0; j < 4; ++j) ab[j] = sA[c][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(pa[i], ab[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t v = t.v0 + ty * 4 + i;
    if (v >= s.n) continue;
    const float m = s.mass[v];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int f = t.f0 + tx * 4 + j;
      if (f >= s.d) continue;
      const float val = acc[i][j] * m;
      const int64_t idx = v * s.ld_feat + f;
      if (b.feat_bf16)
        reinterpret_cast<__nv_bfloat16*>(s.dfeat)[idx] = __float2bfloat16_rn(val);
      else
        reinterpret_cast<float*>(s.dfeat)[idx] = val;
    }
  }
}

}  // namespace

cudaError_t launch_project_bwd_simt(const BatchDev& b, const BwdTile* tiles, int ntiles, const float* d_a,
                                    cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  project_bwd_simt_kernel<<<ntiles, 256, 0, st>>>(b, tiles, d_a);
  return cudaGetLastError();
}

}  // namespace fmap
