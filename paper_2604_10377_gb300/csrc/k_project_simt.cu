// Projection kernels on the CUDA cores (FP32 FMA): the first, plain path.
//
// Forward (Eq. 1): A_s = Phi_s^T diag(M_s) F_s, split over vertex chunks: every
// work item writes the partial sum of its chunk, and a second kernel adds the
// chunks of a shape in a fixed order (bitwise reproducible, no atomics).
// Backward (chain rule of Eq. 1): dF_s = diag(M_s) Phi_s dA_s.
#include "fmap_internal.cuh"

namespace fmap {
namespace {

constexpr int kTile = 64;   // output tile edge
constexpr int kStage = 16;  // vertices (forward) or basis functions (backward) per smem stage

__device__ __forceinline__ float load_feat(const void* f, int64_t idx, int bf16) {
  if (bf16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(f)[idx]);
  return reinterpret_cast<const float*>(f)[idx];
}

__global__ void __launch_bounds__(256) project_simt_kernel(BatchDev b, const ProjTile* tiles, float* ws) {
  __shared__ float sP[kStage][kTile + 4];
  __shared__ float sF[kStage][kTile + 4];
  const ProjTile t = tiles[blockIdx.x];
  const ShapeDev s = b.shapes[t.shape];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

  for (int64_t v0 = t.v0; v0 < t.v1; v0 += kStage) {
    for (int e = tid; e < kStage * kTile; e += 256) {
      const int vv = e / kTile, c = e % kTile;
      const int64_t v = v0 + vv;
      float p = 0.f, f = 0.f;
      if (v < t.v1) {
        const int kk = t.kk0 + c;
        if (kk < s.k) p = s.phi[v * s.ld_phi + kk] * s.mass[v];
        const int ff = t.f0 + c;
        if (ff < s.d) f = load_feat(s.feat, v * s.ld_feat + ff, b.feat_bf16);
      }
      sP[vv][c] = p;
      sF[vv][c] = f;
    }
    __syncthreads();
    // two-level summation: the stage's 16 products, then the running sum
    float st[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) st[i][j] = 0.f;
#pragma unroll
    for (int vv = 0; vv < kStage; ++vv) {
      float pa[4], fb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) pa[i] = sP[vv][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) fb[j] = sF[vv][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) st[i][j] = fmaf(pa[i], fb[j], st[i][j]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += st[i][j];
    __syncthreads();
  }
  float* part = ws + s.part_off + (int64_t)t.chunk * s.k * s.d;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int kk = t.kk0 + ty * 4 + i;
    if (kk >= s.k) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int f = t.f0 + tx * 4 + j;
      if (f < s.d) part[(int64_t)kk * s.d + f] = acc[i][j];
    }
  }
}

// A_s[e] = sum over chunks c (in order) of partial[c][e]
__global__ void project_reduce_kernel(BatchDev b, float* a_out, const float* ws) {
  const ShapeDev s = b.shapes[blockIdx.y];
  const int64_t kd = (int64_t)s.k * s.d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < kd; e += (int64_t)gridDim.x * blockDim.x) {
    const float* part = ws + s.part_off + e;
    float acc = 0.f;
    for (int c = 0; c < s.nchunk; ++c) acc += part[(int64_t)c * kd];
    a_out[s.a_off + e] = acc;
  }
}

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

cudaError_t launch_project_simt(const BatchDev& b, const ProjTile* tiles, int ntiles, float* ws, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  project_simt_kernel<<<ntiles, 256, 0, st>>>(b, tiles, ws);
  return cudaGetLastError();
}

cudaError_t launch_project_reduce(const BatchDev& b, int max_kd, float* a_out, const float* ws, cudaStream_t st) {
  if (b.n_shapes <= 0) return cudaSuccess;
  dim3 grid((max_kd + 255) / 256, b.n_shapes);
  project_reduce_kernel<<<grid, 256, 0, st>>>(b, a_out, ws);
  return cudaGetLastError();
}

cudaError_t launch_project_bwd_simt(const BatchDev& b, const BwdTile* tiles, int ntiles, const float* d_a,
                                    cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  project_bwd_simt_kernel<<<ntiles, 256, 0, st>>>(b, tiles, d_a);
  return cudaGetLastError();
}

}  // namespace fmap
