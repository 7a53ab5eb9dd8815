// Gram matrix and right-hand sides of the row systems (Eq. 4):
//   G = A_x A_x^T (k_X x k_X) and R = A_y A_x^T (k_Y x k_X), per pair.
// 64 x 64 output tiles, 4 x 4 outputs per thread, the feature dimension staged
// through shared memory 16 columns at a time. G is symmetric: only its lower
// tiles are computed and each is written twice (transposed), and once more into a packed
// copy of the lower rows (each row up to the end of its 8 x 8 diagonal block) that the
// row solves load into shared memory with a single bulk copy.
// For pairs flagged hi_gram (large k) G is accumulated in double-float
// arithmetic: every product is split exactly (fma) and summed with an
// error-free transformation, which keeps ~48 significant bits, as an FP64
// accumulation would, on the FP32 pipe (GB300's FP64 rate is a small fraction
// of its FP32 rate). The (hi, lo) pair is kept for the residual of iterative
// refinement, and hi + lo rounded to FP32 feeds the Cholesky factorisation.
#include "fmap_internal.cuh"

namespace fmap {
namespace {

constexpr int kT = 64;
constexpr int kS = 16;

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

// out[i][j] = sum_f X[i0 + i][f] Y[j0 + j][f] for one 64 x 64 tile (X has kx rows, Y ky).
template <bool kDF>
__device__ __forceinline__ void gram_tile(const float* X, const float* Y, int kx, int ky, int d, int i0, int j0,
                                          float (&hi)[4][4], float (&lo)[4][4]) {
  __shared__ float sX[kS][kT + 4];
  __shared__ float sY[kS][kT + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { hi[a][b] = 0.f; lo[a][b] = 0.f; }
  // the next slab is loaded into registers while this one computes
  constexpr int kPer = kT * kS / 256;
  float rx[kPer], ry[kPer];
  auto fetch = [&](int f0) {
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int e = tid + 256 * u, r = e / kS, c = e % kS, f = f0 + c;
      rx[u] = (i0 + r < kx && f < d) ? X[(int64_t)(i0 + r) * d + f] : 0.f;
      ry[u] = (j0 + r < ky && f < d) ? Y[(int64_t)(j0 + r) * d + f] : 0.f;
    }
  };
  fetch(0);
  for (int f0 = 0; f0 < d; f0 += kS) {
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int e = tid + 256 * u, r = e / kS, c = e % kS;
      sX[c][r] = rx[u];
      sY[c][r] = ry[u];
    }
    __syncthreads();
    if (f0 + kS < d) fetch(f0 + kS);
#pragma unroll
    for (int c = 0; c < kS; ++c) {
      const float4 xa = *reinterpret_cast<const float4*>(&sX[c][ty * 4]);
      const float4 yb = *reinterpret_cast<const float4*>(&sY[c][tx * 4]);
      const float xv[4] = {xa.x, xa.y, xa.z, xa.w};
      const float yv[4] = {yb.x, yb.y, yb.z, yb.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if (kDF)
            df_fma(hi[a][b], lo[a][b], xv[a], yv[b]);
          else
            hi[a][b] = fmaf(xv[a], yv[b], hi[a][b]);
        }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) gram_kernel(BatchDev b, const float* a, float* ws) {
  const PairDev pd = b.pairs[blockIdx.z];
  const int k = pd.k, d = pd.d;
  const int nt = (k + kT - 1) / kT;
  const float* ax = a + b.shapes[pd.x].a_off;
  const float* ay = a + b.shapes[pd.y].a_off;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float hi[4][4], lo[4][4];
  if (blockIdx.y == 0) {
    // G: lower tiles only (ti >= tj), mirrored on store
    int t = blockIdx.x, ti = 0;
    while (t > ti) { t -= ti + 1; ++ti; }
    const int tj = t;
    if (ti >= nt) return;
    const int i0 = ti * kT, j0 = tj * kT;
    float* g = ws + pd.g_off;
    float* gp = g + gram_packed_off(k);   // the same values in the row solves' packed layout
    const int ldg = gram_ld(k);
    float2* ghl = pd.hi_gram ? reinterpret_cast<float2*>(ws) + pd.g64_off : nullptr;
    if (pd.hi_gram)
      gram_tile<true>(ax, ax, k, k, d, i0, j0, hi, lo);
    else
      gram_tile<false>(ax, ax, k, k, d, i0, j0, hi, lo);
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = i0 + ty * 4 + r, j = j0 + tx * 4 + c;
        if (i >= k || j >= k) continue;
        float v = hi[r][c], e = 0.f;
        if (ghl) {
          v = __fadd_rn(hi[r][c], lo[r][c]);
          e = __fsub_rn(lo[r][c], __fsub_rn(v, hi[r][c]));
        }
        g[(int64_t)i * ldg + j] = v;
        g[(int64_t)j * ldg + i] = v;
        if (j <= (i | 7)) gp[rowoff(i) + j] = v;
        if (i <= (j | 7)) gp[rowoff(j) + i] = v;
        if (ghl) {
          ghl[(int64_t)i * k + j] = make_float2(v, e);
          ghl[(int64_t)j * k + i] = make_float2(v, e);
        }
      }
  } else {
    // R = A_y A_x^T (ky x k): every tile
    const int ky = b.shapes[pd.y].k, nty = (ky + kT - 1) / kT;
    if ((int)blockIdx.x >= nty * nt) return;
    const int i0 = (blockIdx.x / nt) * kT, j0 = (blockIdx.x % nt) * kT;
    gram_tile<false>(ay, ax, ky, k, d, i0, j0, hi, lo);
    float* r = ws + pd.r_off;
#pragma unroll
    for (int rr = 0; rr < 4; ++rr)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = i0 + ty * 4 + rr, j = j0 + tx * 4 + c;
        if (i < ky && j < k) r[(int64_t)i * k + j] = hi[rr][c];
      }
  }
}

}  // namespace

cudaError_t launch_gram(const BatchDev& b, int max_k, const float* a, float* ws, cudaStream_t st, bool with_r) {
  if (b.n_pairs <= 0) return cudaSuccess;
  const int nt = (max_k + kT - 1) / kT;
  dim3 grid(nt * nt, with_r ? 2 : 1, b.n_pairs);
  gram_kernel<<<grid, 256, 0, st>>>(b, a, ws);
  return cudaGetLastError();
}

}  // namespace fmap
