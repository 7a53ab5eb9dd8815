// Gram matrix and right-hand sides of the row systems (Eq. 4):
//   G = A_x A_x^T and R = A_y A_x^T, both k x k, per pair.
// For pairs flagged hi_gram (large k) G is accumulated in double-float
// arithmetic: every product is split exactly (fma) and summed with an
// error-free transformation, which keeps ~48 significant bits, as an FP64
// accumulation would, on the FP32 pipe (GB300's FP64 rate is a small fraction
// of its FP32 rate). The (hi, lo) pair is kept for the residual of iterative
// refinement, and hi + lo rounded to FP32 feeds the Cholesky factorisation.
#include "fmap_internal.cuh"

namespace fmap {
namespace {

constexpr int kT = 32;

// (hi, lo) += a * b with an exact product and an error-free sum.
__device__ __forceinline__ void df_fma(float& hi, float& lo, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float pe = fmaf(a, b, -p);
  const float s = __fadd_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(e, pe));
}

__device__ __forceinline__ void gram_tile_df(const float* X, int k, int d, int ti, int tj, float* out32,
                                             float2* outhl) {
  __shared__ float sX[kT][kT + 1];
  __shared__ float sY[kT][kT + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
  for (int f0 = 0; f0 < d; f0 += kT) {
    for (int e = threadIdx.x; e < kT * kT; e += 256) {
      const int r = e / kT, c = e % kT;
      const int xi = ti * kT + r, yj = tj * kT + r, f = f0 + c;
      sX[r][c] = (xi < k && f < d) ? X[(int64_t)xi * d + f] : 0.f;
      sY[r][c] = (yj < k && f < d) ? X[(int64_t)yj * d + f] : 0.f;
    }
    __syncthreads();
    for (int c = 0; c < kT; ++c) {
      const float yv = sY[tx][c];
#pragma unroll
      for (int r = 0; r < 4; ++r) df_fma(hi[r], lo[r], sX[ty + 8 * r][c], yv);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = ti * kT + ty + 8 * r, j = tj * kT + tx;
    if (i < k && j < k) {
      const float s = __fadd_rn(hi[r], lo[r]);
      const float e = __fsub_rn(lo[r], __fsub_rn(s, hi[r]));
      out32[(int64_t)i * k + j] = s;
      outhl[(int64_t)i * k + j] = make_float2(s, e);
    }
  }
}

template <typename Acc>
__device__ __forceinline__ void gram_tile(const float* X, const float* Y, int k, int d, int ti, int tj,
                                          float* out32, double* out64) {
  __shared__ float sX[kT][kT + 1];
  __shared__ float sY[kT][kT + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 warps
  Acc acc[4] = {Acc(0), Acc(0), Acc(0), Acc(0)};
  for (int f0 = 0; f0 < d; f0 += kT) {
    for (int e = threadIdx.x; e < kT * kT; e += 256) {
      const int r = e / kT, c = e % kT;
      const int xi = ti * kT + r, yj = tj * kT + r, f = f0 + c;
      sX[r][c] = (xi < k && f < d) ? X[(int64_t)xi * d + f] : 0.f;
      sY[r][c] = (yj < k && f < d) ? Y[(int64_t)yj * d + f] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int c = 0; c < kT; ++c) {
      const Acc yv = Acc(sY[tx][c]);
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[r] += Acc(sX[ty + 8 * r][c]) * yv;
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = ti * kT + ty + 8 * r, j = tj * kT + tx;
    if (i < k && j < k) {
      out32[(int64_t)i * k + j] = (float)acc[r];
      if (out64) out64[(int64_t)i * k + j] = (double)acc[r];
    }
  }
}

__global__ void __launch_bounds__(256) gram_kernel(BatchDev b, const float* a, float* ws) {
  const PairDev pd = b.pairs[blockIdx.z];
  const int k = pd.k, d = pd.d;
  const int nt = (k + kT - 1) / kT;
  if ((int)blockIdx.x >= nt * nt) return;
  const int ti = blockIdx.x / nt, tj = blockIdx.x % nt;
  const float* ax = a + b.shapes[pd.x].a_off;
  const float* ay = a + b.shapes[pd.y].a_off;
  if (blockIdx.y == 0) {
    if (pd.hi_gram)
      gram_tile_df(ax, k, d, ti, tj, ws + pd.g_off, reinterpret_cast<float2*>(ws) + pd.g64_off);
    else
      gram_tile<float>(ax, ax, k, d, ti, tj, ws + pd.g_off, nullptr);
  } else {
    gram_tile<float>(ay, ax, k, d, ti, tj, ws + pd.r_off, nullptr);
  }
}

}  // namespace

cudaError_t launch_gram(const BatchDev& b, int max_k, const float* a, float* ws, cudaStream_t st) {
  if (b.n_pairs <= 0) return cudaSuccess;
  const int nt = (max_k + kT - 1) / kT;
  dim3 grid(nt * nt, 2, b.n_pairs);
  gram_kernel<<<grid, 256, 0, st>>>(b, a, ws);
  return cudaGetLastError();
}

}  // namespace fmap
