// Gram matrix and right-hand sides of the row systems (Eq. 4):
//   G = A_x A_x^T and R = A_y A_x^T, both k x k, per pair.
// G is accumulated in FP64 for pairs flagged hi_gram (large k); the FP64 copy is
// kept for the residual of iterative refinement, and its FP32 rounding feeds the
// Cholesky factorisation.
#include "fmap_internal.cuh"

namespace fmap {
namespace {

constexpr int kT = 32;

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
    double* g64 = pd.g64_off >= 0 ? reinterpret_cast<double*>(ws) + pd.g64_off : nullptr;
    if (pd.hi_gram)
      gram_tile<double>(ax, ax, k, d, ti, tj, ws + pd.g_off, g64);
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
