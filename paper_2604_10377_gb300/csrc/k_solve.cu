// Row-wise regularised solve (Eq. 5-9) and its adjoint.
//
// One thread block per row system S_i = G + lambda diag(D_i): the packed lower
// triangle of S_i lives in shared memory, is factorised in place by a
// right-looking Cholesky in FP32, and the solve is followed by iterative
// refinement with the residual taken against G (FP64 G for hi_gram pairs).
// The same kernel solves the adjoint systems S_i gamma_i = dL/dc_i, reusing saved
// factors when the caller kept them.
#include <math.h>

#include "fmap_internal.cuh"

namespace fmap {
namespace {

__device__ __forceinline__ float mask_entry(const PairDev& pd, const float* evx, const float* evy, int i, int a) {
  if (pd.mask) return pd.mask[(int64_t)i * pd.k + a];
  const float t = evy[i] - evx[a];
  return t * t;
}

__device__ __forceinline__ void set_status(int32_t* status, int p, int32_t code) {
  if (status) atomicCAS(status + p, 0, code);
}

// In-place solve of L L^T x = v by warp 0 (v in shared memory, overwritten with x).
__device__ __forceinline__ void warp_chol_solve(const float* L, const float* dg, float* v, int k, int lane) {
  __syncwarp();
  for (int j = 0; j < k; ++j) {           // L y = v
    const float yj = v[j] / dg[j];
    __syncwarp();
    if (lane == 0) v[j] = yj;
    for (int a = j + 1 + lane; a < k; a += 32) v[a] = fmaf(-L[tri(a) + j], yj, v[a]);
    __syncwarp();
  }
  for (int j = k - 1; j >= 0; --j) {      // L^T x = y
    const float xj = v[j] / dg[j];
    __syncwarp();
    if (lane == 0) v[j] = xj;
    const float* row = L + tri(j);
    for (int a = lane; a < j; a += 32) v[a] = fmaf(-row[a], xj, v[a]);
    __syncwarp();
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) solve_kernel(BatchDev b, const int2* systems, int first, int count, int mode,
                                                  const float* rhs_flat, float* out_flat, float* saved,
                                                  int32_t* status, float* ws) {
  constexpr int NW = NT / 32;
  extern __shared__ float smem[];
  __shared__ int s_bad;
  if ((int)blockIdx.x >= count) return;
  const int2 sys = systems[first + blockIdx.x];
  const int p = sys.x, i = sys.y;
  const PairDev pd = b.pairs[p];
  const int k = pd.k;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* evx = b.shapes[pd.x].evals;
  const float* evy = b.shapes[pd.y].evals;
  float* L = smem;                                  // packed lower triangle, tri(k)
  float* dg = smem + ((tri(k) + 3) & ~3LL);         // sqrt pivots, k
  float* v = dg + k;                                // working vector, k
  float* xs = v + k;                                // solution, k
  float* rh = xs + k;                               // right-hand side, k
  const float* G = ws + pd.g_off;
  const float* rhs = (mode == kSolveForward) ? ws + pd.r_off + (int64_t)i * k : rhs_flat + pd.c_off + (int64_t)i * k;
  float* out = (mode == kSolveForward) ? out_flat + pd.c_off + (int64_t)i * k : ws + pd.gam_off + (int64_t)i * k;
  float* fac = (saved != nullptr && pd.fac_off >= 0) ? saved + pd.fac_off + (int64_t)i * tri(k) : nullptr;
  const float lam = pd.lam;

  if (tid == 0) {
    s_bad = 0;
    // a projection wait that timed out leaves its error in the workspace's first word
    if (i == 0 && reinterpret_cast<const int*>(ws)[0] != 0) set_status(status, p, FMAP_ERR_TIMEOUT);
  }
  for (int a = tid; a < k; a += NT) rh[a] = rhs[a];

  if (mode == kSolveAdjoint && fac != nullptr) {
    // factors saved by the forward solve (diagonal entries hold the sqrt pivots)
    for (int64_t e = tid; e < tri(k); e += NT) L[e] = fac[e];
    __syncthreads();
    for (int a = tid; a < k; a += NT) dg[a] = L[tri(a) + a];
    __syncthreads();
  } else {
    for (int a = warp; a < k; a += NW) {
      const float* grow = G + (int64_t)a * k;
      float* lrow = L + tri(a);
      for (int c = lane; c <= a; c += 32) lrow[c] = grow[c];
      if (lane == 0) lrow[a] = grow[a] + lam * mask_entry(pd, evx, evy, i, a);
    }
    __syncthreads();
    for (int j = 0; j < k; ++j) {
      const float piv = L[tri(j) + j];
      if (!(piv > 0.f) || !(piv < INFINITY)) {
        if (tid == 0) s_bad = j + 1;
        break;
      }
      const float dj = sqrtf(piv);
      const float inv = 1.f / dj;
      if (tid == 0) dg[j] = dj;
      for (int a = j + 1 + tid; a < k; a += NT) L[tri(a) + j] *= inv;
      __syncthreads();
      for (int a = j + 1 + warp; a < k; a += NW) {
        const float la = L[tri(a) + j];
        float* row = L + tri(a);
        for (int c = j + 1 + lane; c <= a; c += 32) row[c] = fmaf(-la, L[tri(c) + j], row[c]);
      }
      __syncthreads();
    }
    __syncthreads();
    if (s_bad) {
      if (tid == 0) set_status(status, p, FMAP_ERR_NOT_SPD | (i << 8));
      for (int a = tid; a < k; a += NT) out[a] = __int_as_float(0x7fc00000);
      return;
    }
    if (mode == kSolveForward && fac != nullptr) {
      for (int64_t e = tid; e < tri(k); e += NT) fac[e] = L[e];
      __syncthreads();
      for (int a = tid; a < k; a += NT) fac[tri(a) + a] = dg[a];
    }
  }

  // x = S^{-1} rhs
  for (int a = tid; a < k; a += NT) v[a] = rh[a];
  __syncthreads();
  if (warp == 0) warp_chol_solve(L, dg, v, k, lane);
  __syncthreads();
  for (int a = tid; a < k; a += NT) xs[a] = v[a];
  __syncthreads();

  // iterative refinement: x += S^{-1} (rhs - S x)
  const double* G64 = pd.g64_off >= 0 ? reinterpret_cast<const double*>(ws) + pd.g64_off : nullptr;
  for (int it = 0; it < b.ir_steps; ++it) {
    for (int a = warp; a < k; a += NW) {
      float r;
      if (G64) {
        const double* grow = G64 + (int64_t)a * k;
        double sum = 0.0;
        for (int c = lane; c < k; c += 32) sum += grow[c] * (double)xs[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        sum += (double)lam * (double)mask_entry(pd, evx, evy, i, a) * (double)xs[a];
        r = (float)((double)rh[a] - sum);
      } else {
        const float* grow = G + (int64_t)a * k;
        float sum = 0.f;
        for (int c = lane; c < k; c += 32) sum = fmaf(grow[c], xs[c], sum);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        sum = fmaf(lam * mask_entry(pd, evx, evy, i, a), xs[a], sum);
        r = rh[a] - sum;
      }
      if (lane == 0) v[a] = r;
    }
    __syncthreads();
    if (warp == 0) warp_chol_solve(L, dg, v, k, lane);
    __syncthreads();
    for (int a = tid; a < k; a += NT) xs[a] += v[a];
    __syncthreads();
  }

  bool finite = true;
  for (int a = tid; a < k; a += NT) {
    const float xv = xs[a];
    out[a] = xv;
    if (!isfinite(xv)) finite = false;
  }
  if (!finite) set_status(status, p, FMAP_ERR_NONFINITE | (i << 8));
}

template <int NT>
cudaError_t set_limit() {
  const int bytes = (int)((tri(kMaxK) + 4 + 4 * kMaxK) * sizeof(float));
  return cudaFuncSetAttribute(solve_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// ---------------------------------------------------------------- adjoint GEMMs
constexpr int kTile = 64;
constexpr int kStage = 16;

// W = Gamma^T C + C^T Gamma (k x k), and the mask gradient dD = -lambda Gamma o C.
__global__ void __launch_bounds__(256) adjoint_w_kernel(BatchDev b, const float* c_flat, float* d_mask, float* ws) {
  __shared__ float sG[kStage][kTile + 4];   // Gamma[m][a-tile]
  __shared__ float sC[kStage][kTile + 4];   // C[m][a-tile]
  __shared__ float sGb[kStage][kTile + 4];  // Gamma[m][b-tile]
  __shared__ float sCb[kStage][kTile + 4];  // C[m][b-tile]
  const PairDev pd = b.pairs[blockIdx.z];
  const int k = pd.k;
  const int nt = (k + kTile - 1) / kTile;
  if ((int)blockIdx.x >= nt * nt) return;
  const int a0 = (blockIdx.x / nt) * kTile, b0 = (blockIdx.x % nt) * kTile;
  const float* gam = ws + pd.gam_off;
  const float* cm = c_flat + pd.c_off;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4] = {};
  for (int m0 = 0; m0 < k; m0 += kStage) {
    for (int e = tid; e < kStage * kTile; e += 256) {
      const int mm = e / kTile, cc = e % kTile, m = m0 + mm;
      const bool okm = m < k;
      sG[mm][cc] = (okm && a0 + cc < k) ? gam[(int64_t)m * k + a0 + cc] : 0.f;
      sC[mm][cc] = (okm && a0 + cc < k) ? cm[(int64_t)m * k + a0 + cc] : 0.f;
      sGb[mm][cc] = (okm && b0 + cc < k) ? gam[(int64_t)m * k + b0 + cc] : 0.f;
      sCb[mm][cc] = (okm && b0 + cc < k) ? cm[(int64_t)m * k + b0 + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int mm = 0; mm < kStage; ++mm) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float ga = sG[mm][ty * 4 + i], ca = sC[mm][ty * 4 + i];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          acc[i][j] = fmaf(ga, sCb[mm][tx * 4 + j], fmaf(ca, sGb[mm][tx * 4 + j], acc[i][j]));
      }
    }
    __syncthreads();
  }
  float* w = ws + pd.w_off;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = a0 + ty * 4 + i;
    if (a >= k) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = b0 + tx * 4 + j;
      if (c >= k) continue;
      w[(int64_t)a * k + c] = acc[i][j];
      if (d_mask) d_mask[pd.c_off + (int64_t)a * k + c] = -pd.lam * gam[(int64_t)a * k + c] * cm[(int64_t)a * k + c];
    }
  }
}

// dlambda_p = -sum_ij D_ij Gamma_ij C_ij, fixed-order block reduction (one block per pair).
__global__ void __launch_bounds__(256) adjoint_dlambda_kernel(BatchDev b, const float* c_flat, float* d_lambda,
                                                              const float* ws) {
  __shared__ float red[256];
  const int p = blockIdx.x;
  const PairDev pd = b.pairs[p];
  const int k = pd.k;
  const float* gam = ws + pd.gam_off;
  const float* cm = c_flat + pd.c_off;
  const float* evx = b.shapes[pd.x].evals;
  const float* evy = b.shapes[pd.y].evals;
  float acc = 0.f;
  for (int e = threadIdx.x; e < k * k; e += 256) {
    const int i = e / k, j = e % k;
    acc = fmaf(mask_entry(pd, evx, evy, i, j) * gam[e], cm[e], acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) d_lambda[p] = -red[0];
}

// Per-pair contributions:
//   which 0: dA_x = Gamma^T A_y - W A_x   (into sx_off)
//   which 1: dA_y = Gamma A_x             (into sy_off)
__global__ void __launch_bounds__(256) adjoint_da_kernel(BatchDev b, const float* a_flat, float* ws) {
  __shared__ float sX[kTile][kStage + 1];   // left operand [a][m]
  __shared__ float sY[kStage][kTile + 4];   // right operand [m][f]
  __shared__ float sX2[kTile][kStage + 1];
  __shared__ float sY2[kStage][kTile + 4];
  const PairDev pd = b.pairs[blockIdx.z];
  const int k = pd.k, d = pd.d;
  const int ntf = (d + kTile - 1) / kTile, nta = (k + kTile - 1) / kTile;
  if ((int)blockIdx.x >= ntf * nta) return;
  const int a0 = (blockIdx.x / ntf) * kTile, f0 = (blockIdx.x % ntf) * kTile;
  const int which = blockIdx.y;
  const float* gam = ws + pd.gam_off;
  const float* w = ws + pd.w_off;
  const float* ax = a_flat + b.shapes[pd.x].a_off;
  const float* ay = a_flat + b.shapes[pd.y].a_off;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4] = {};
  for (int m0 = 0; m0 < k; m0 += kStage) {
    for (int e = tid; e < kTile * kStage; e += 256) {
      const int aa = e / kStage, mm = e % kStage;
      const int a = a0 + aa, m = m0 + mm;
      const bool ok = a < k && m < k;
      if (which == 0) {
        sX[aa][mm] = ok ? gam[(int64_t)m * k + a] : 0.f;     // Gamma^T[a][m]
        sX2[aa][mm] = ok ? -w[(int64_t)a * k + m] : 0.f;     // -W[a][m]
      } else {
        sX[aa][mm] = ok ? gam[(int64_t)a * k + m] : 0.f;     // Gamma[a][m]
      }
    }
    for (int e = tid; e < kStage * kTile; e += 256) {
      const int mm = e / kTile, ff = e % kTile;
      const int m = m0 + mm, f = f0 + ff;
      const bool ok = m < k && f < d;
      if (which == 0) {
        sY[mm][ff] = ok ? ay[(int64_t)m * d + f] : 0.f;
        sY2[mm][ff] = ok ? ax[(int64_t)m * d + f] : 0.f;
      } else {
        sY[mm][ff] = ok ? ax[(int64_t)m * d + f] : 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int mm = 0; mm < kStage; ++mm) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float xa = sX[ty * 4 + i][mm];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xa, sY[mm][tx * 4 + j], acc[i][j]);
      }
    }
    if (which == 0) {
#pragma unroll
      for (int mm = 0; mm < kStage; ++mm) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float xa = sX2[ty * 4 + i][mm];
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xa, sY2[mm][tx * 4 + j], acc[i][j]);
        }
      }
    }
    __syncthreads();
  }
  float* out = ws + (which == 0 ? pd.sx_off : pd.sy_off);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = a0 + ty * 4 + i;
    if (a >= k) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int f = f0 + tx * 4 + j;
      if (f < d) out[(int64_t)a * d + f] = acc[i][j];
    }
  }
}

// dA_s = sum of the shape's contributions, in pair order.
__global__ void gather_da_kernel(BatchDev b, float* d_a, const float* ws) {
  const ShapeDev s = b.shapes[blockIdx.y];
  const int64_t kd = (int64_t)s.k * s.d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < kd; e += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.f;
    for (int q = s.slot_beg; q < s.slot_end; ++q) acc += ws[b.slot_list[q] + e];
    d_a[s.a_off + e] = acc;
  }
}

// Loss ||C C^T - I||^2 + ||C - C_gt||^2 and dL/dC = 4 (C C^T - I) C + 2 (C - C_gt); one block per pair.
__global__ void __launch_bounds__(256) loss_orth_kernel(BatchDev b, const float* c_flat, const float* gt_flat,
                                                        float* loss, float* d_c, float* ws) {
  __shared__ float red[256];
  const int p = blockIdx.x;
  const PairDev pd = b.pairs[p];
  const int k = pd.k;
  const float* c = c_flat + pd.c_off;
  const float* gt = gt_flat + pd.c_off;
  float* e = ws + pd.e_off;
  float acc = 0.f;
  for (int idx = threadIdx.x; idx < k * k; idx += 256) {
    const int a = idx / k, bb = idx % k;
    const float* ca = c + (int64_t)a * k;
    const float* cb = c + (int64_t)bb * k;
    float s = 0.f;
    for (int l = 0; l < k; ++l) s = fmaf(ca[l], cb[l], s);
    if (a == bb) s -= 1.f;
    e[idx] = s;
    const float r = c[idx] - gt[idx];
    acc = fmaf(s, s, fmaf(r, r, acc));
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) loss[p] = red[0];
  if (d_c == nullptr) return;
  for (int idx = threadIdx.x; idx < k * k; idx += 256) {
    const int a = idx / k, bb = idx % k;
    const float* ea = e + (int64_t)a * k;
    float s = 0.f;
    for (int l = 0; l < k; ++l) s = fmaf(ea[l], c[(int64_t)l * k + bb], s);
    d_c[pd.c_off + idx] = 4.f * s + 2.f * (c[idx] - gt[idx]);
  }
}

__global__ void status_clear_kernel(int32_t* status, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) status[i] = 0;
}

}  // namespace

cudaError_t solve_set_smem_limits() {
  cudaError_t e;
  if ((e = set_limit<64>()) != cudaSuccess) return e;
  if ((e = set_limit<128>()) != cudaSuccess) return e;
  return set_limit<256>();
}

cudaError_t launch_solve(const BatchDev& b, const SolveGroup& g, const int2* systems, int mode, const float* rhs_flat,
                         float* out_flat, float* saved, int32_t* status, float* ws, cudaStream_t st) {
  if (g.count <= 0) return cudaSuccess;
  const size_t smem = (size_t)(((tri(g.kmax) + 3) & ~3LL) + 4 * g.kmax) * sizeof(float);
  switch (g.threads) {
    case 64:
      solve_kernel<64><<<g.count, 64, smem, st>>>(b, systems, g.first, g.count, mode, rhs_flat, out_flat, saved, status, ws);
      break;
    case 128:
      solve_kernel<128><<<g.count, 128, smem, st>>>(b, systems, g.first, g.count, mode, rhs_flat, out_flat, saved, status, ws);
      break;
    default:
      solve_kernel<256><<<g.count, 256, smem, st>>>(b, systems, g.first, g.count, mode, rhs_flat, out_flat, saved, status, ws);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_adjoint_gemms(const BatchDev& b, int max_k, int max_d, const float* a, const float* c,
                                 float* d_mask, float* d_lambda, float* ws, cudaStream_t st) {
  if (b.n_pairs <= 0) return cudaSuccess;
  const int ntk = (max_k + kTile - 1) / kTile, ntd = (max_d + kTile - 1) / kTile;
  adjoint_w_kernel<<<dim3(ntk * ntk, 1, b.n_pairs), 256, 0, st>>>(b, c, d_mask, ws);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (d_lambda) {
    adjoint_dlambda_kernel<<<b.n_pairs, 256, 0, st>>>(b, c, d_lambda, ws);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  adjoint_da_kernel<<<dim3(ntk * ntd, 2, b.n_pairs), 256, 0, st>>>(b, a, ws);
  return cudaGetLastError();
}

cudaError_t launch_gather_da(const BatchDev& b, int max_kd, float* d_a, const float* ws, cudaStream_t st) {
  if (b.n_shapes <= 0) return cudaSuccess;
  gather_da_kernel<<<dim3((max_kd + 255) / 256, b.n_shapes), 256, 0, st>>>(b, d_a, ws);
  return cudaGetLastError();
}

cudaError_t launch_loss_orth(const BatchDev& b, const float* c, const float* c_gt, float* loss, float* d_c, float* ws,
                             cudaStream_t st) {
  if (b.n_pairs <= 0) return cudaSuccess;
  loss_orth_kernel<<<b.n_pairs, 256, 0, st>>>(b, c, c_gt, loss, d_c, ws);
  return cudaGetLastError();
}

cudaError_t launch_status_clear(int32_t* status, int n, cudaStream_t st) {
  if (n <= 0 || status == nullptr) return cudaSuccess;
  status_clear_kernel<<<(n + 255) / 256, 256, 0, st>>>(status, n);
  return cudaGetLastError();
}

}  // namespace fmap
