// A pair's map C is k_Y x k_X: k_X = pd.k (shape x, row-system size, columns of C) and
// k_Y = the basis size of shape y (rows of C); the paper's maps are square.
//
// Adjoint of the row-wise solve (given Gamma from the adjoint row solves):
// W = Gamma^T C + C^T Gamma, dA_x = Gamma^T A_y - W A_x, dA_y = Gamma A_x,
// dD = -lambda Gamma o C, dlambda = -sum(D o Gamma o C); the per-shape gather of
// dA contributions; the training loss; the status clear.
#include <math.h>

#include "fmap_internal.cuh"

namespace fmap {
namespace {

__device__ __forceinline__ float mask_entry(const PairDev& pd, const float* evx, const float* evy, int i, int a) {
  if (pd.mask) return pd.mask[(int64_t)i * pd.k + a];
  const float t = evy[i] - evx[a];
  return t * t;
}

// ---------------------------------------------------------------- adjoint GEMMs
constexpr int kTile = 64;
constexpr int kStage = 16;
constexpr int kPer = kTile * kStage / 256;   // stage elements per thread and operand


// W = Gamma^T C + C^T Gamma (k_X x k_X; Gamma and C are k_Y x k_X).
__global__ void __launch_bounds__(256, 3) adjoint_w_kernel(BatchDev b, const float* c_flat, float* ws) {
  __shared__ __align__(16) float sG[kStage][kTile + 4];   // Gamma[m][a-tile]
  __shared__ __align__(16) float sC[kStage][kTile + 4];   // C[m][a-tile]
  __shared__ __align__(16) float sGb[kStage][kTile + 4];  // Gamma[m][b-tile]
  __shared__ __align__(16) float sCb[kStage][kTile + 4];  // C[m][b-tile]
  const PairDev pd = b.pairs[blockIdx.z];
  const int k = pd.k, ky = b.shapes[pd.y].k;   // Gamma, C: ky x k
  const int nt = (k + kTile - 1) / kTile;
  if ((int)blockIdx.x >= nt * nt) return;
  const int a0 = (blockIdx.x / nt) * kTile, b0 = (blockIdx.x % nt) * kTile;
  const float* gam = ws + pd.gam_off;
  const float* cm = c_flat + pd.c_off;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4] = {};
  // the next stage's operands are loaded into registers while this stage computes
  float rg[kPer], rc[kPer], rgb[kPer], rcb[kPer];
  auto fetch = [&](int m0) {
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int e = tid + 256 * u, mm = e / kTile, cc = e % kTile, m = m0 + mm;
      const bool okm = m < ky;
      rg[u] = (okm && a0 + cc < k) ? gam[(int64_t)m * k + a0 + cc] : 0.f;
      rc[u] = (okm && a0 + cc < k) ? cm[(int64_t)m * k + a0 + cc] : 0.f;
      rgb[u] = (okm && b0 + cc < k) ? gam[(int64_t)m * k + b0 + cc] : 0.f;
      rcb[u] = (okm && b0 + cc < k) ? cm[(int64_t)m * k + b0 + cc] : 0.f;
    }
  };
  fetch(0);
  for (int m0 = 0; m0 < ky; m0 += kStage) {
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int e = tid + 256 * u, mm = e / kTile, cc = e % kTile;
      sG[mm][cc] = rg[u];
      sC[mm][cc] = rc[u];
      sGb[mm][cc] = rgb[u];
      sCb[mm][cc] = rcb[u];
    }
    __syncthreads();
    if (m0 + kStage < ky) fetch(m0 + kStage);
#pragma unroll
    for (int mm = 0; mm < kStage; ++mm) {
      const float4 g4 = *reinterpret_cast<const float4*>(&sG[mm][ty * 4]);
      const float4 c4 = *reinterpret_cast<const float4*>(&sC[mm][ty * 4]);
      const float4 gb4 = *reinterpret_cast<const float4*>(&sGb[mm][tx * 4]);
      const float4 cb4 = *reinterpret_cast<const float4*>(&sCb[mm][tx * 4]);
      const float ga[4] = {g4.x, g4.y, g4.z, g4.w}, ca[4] = {c4.x, c4.y, c4.z, c4.w};
      const float gb[4] = {gb4.x, gb4.y, gb4.z, gb4.w}, cb[4] = {cb4.x, cb4.y, cb4.z, cb4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(ga[i], cb[j], fmaf(ca[i], gb[j], acc[i][j]));
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
    }
  }
}

// The mask gradient dD = -lambda_i Gamma o C (when d_mask is given; lambda_i = lambda
// without row weights), dlambda_p = -sum_ij D_ij Gamma_ij C_ij (when d_lambda is given;
// with row weights the sum of the per-row gradients) and, for pairs with row weights and an
// output for them, dlambda_i = -sum_j D_ij Gamma_ij C_ij (one warp per row, lanes in a fixed
// order); over the k_Y x k_X entries, fixed-order block reductions (one block per pair).
__global__ void __launch_bounds__(256) adjoint_dlambda_kernel(BatchDev b, const float* c_flat, float* d_mask,
                                                              float* d_lambda, const float* ws) {
  __shared__ float red[256];
  const int p = blockIdx.x;
  const PairDev pd = b.pairs[p];
  const int k = pd.k, ky = b.shapes[pd.y].k, n = ky * pd.k;   // the ky x k entries
  const float* gam = ws + pd.gam_off;
  const float* cm = c_flat + pd.c_off;
  const float* evx = b.shapes[pd.x].evals;
  const float* evy = b.shapes[pd.y].evals;
  if (d_mask)
    for (int e = threadIdx.x; e < n; e += 256) {
      const float lam = pd.lam_rows ? pd.lam_rows[e / k] : pd.lam;
      d_mask[pd.c_off + e] = -lam * gam[e] * cm[e];
    }
  if (pd.dlam_rows) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = warp; i < ky; i += 8) {
      float acc = 0.f;
      for (int j = lane; j < k; j += 32) {
        const int e = i * k + j;
        acc = fmaf(mask_entry(pd, evx, evy, i, j) * gam[e], cm[e], acc);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) pd.dlam_rows[i] = -acc;
    }
  }
  if (!d_lambda) return;
  float acc = 0.f;
  for (int e = threadIdx.x; e < n; e += 256) {
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

// Per-pair contributions (Gamma is k_Y x k_X, W k_X x k_X):
//   which 0: dA_x = Gamma^T A_y - W A_x   (k_X x d, into sx_off; the two products share
//            one loop over max(k_X, k_Y), each operand zero past its own length)
//   which 1: dA_y = Gamma A_x             (k_Y x d, into sy_off)
__global__ void __launch_bounds__(256) adjoint_da_kernel(BatchDev b, const float* a_flat, float* ws) {
  // both operands stored m-major in shared memory, so that a thread's 4 rows and 4
  // columns of one step are two float4 reads
  __shared__ __align__(16) float sX[kStage][kTile + 4];    // left operand [m][a]
  __shared__ __align__(16) float sY[kStage][kTile + 4];    // right operand [m][f]
  __shared__ __align__(16) float sX2[kStage][kTile + 4];
  __shared__ __align__(16) float sY2[kStage][kTile + 4];
  const PairDev pd = b.pairs[blockIdx.z];
  const int k = pd.k, ky = b.shapes[pd.y].k, d = pd.d;
  const int which = blockIdx.y;
  const int rows = which == 0 ? k : ky;                    // rows of the contribution
  const int mlen = which == 0 ? max(k, ky) : k;            // length of the reduction
  const int ntf = (d + kTile - 1) / kTile, nta = (rows + kTile - 1) / kTile;
  if ((int)blockIdx.x >= ntf * nta) return;
  const int a0 = (blockIdx.x / ntf) * kTile, f0 = (blockIdx.x % ntf) * kTile;
  const float* gam = ws + pd.gam_off;
  const float* w = ws + pd.w_off;
  const float* ax = a_flat + b.shapes[pd.x].a_off;
  const float* ay = a_flat + b.shapes[pd.y].a_off;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4] = {};
  // the next stage's operands are loaded into registers while this stage computes
  float r1[kPer], r2[kPer], r3[kPer], r4[kPer];
  auto fetch = [&](int m0) {
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int e = tid + 256 * u;
      {
        // Gamma^T[a][m] = Gamma[m][a]: consecutive threads take consecutive a (coalesced)
        const int aa = e % kTile, mm = e / kTile, a = a0 + aa, m = m0 + mm;
        r1[u] = (which == 0 && a < k && m < ky) ? gam[(int64_t)m * k + a] : 0.f;
      }
      {
        // which 0: -W[a][m] (a, m < k_X); which 1: Gamma[a][m] (a < k_Y, m < k_X)
        const int aa = e / kStage, mm = e % kStage, a = a0 + aa, m = m0 + mm;
        const bool ok = a < rows && m < k;
        r2[u] = !ok ? 0.f : (which == 0 ? -w[(int64_t)a * k + m] : gam[(int64_t)a * k + m]);
      }
      {
        // which 0: A_y[m] (m < k_Y) beside A_x[m] (m < k_X); which 1: A_x[m] (m < k_X)
        const int mm = e / kTile, ff = e % kTile, m = m0 + mm, f = f0 + ff;
        const bool okf = f < d;
        r3[u] = which == 0 ? ((okf && m < ky) ? ay[(int64_t)m * d + f] : 0.f)
                           : ((okf && m < k) ? ax[(int64_t)m * d + f] : 0.f);
        r4[u] = (which == 0 && okf && m < k) ? ax[(int64_t)m * d + f] : 0.f;
      }
    }
  };
  fetch(0);
  for (int m0 = 0; m0 < mlen; m0 += kStage) {
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int e = tid + 256 * u;
      if (which == 0) sX[e / kTile][e % kTile] = r1[u];
      if (which == 0)
        sX2[e % kStage][e / kStage] = r2[u];
      else
        sX[e % kStage][e / kStage] = r2[u];
      sY[e / kTile][e % kTile] = r3[u];
      if (which == 0) sY2[e / kTile][e % kTile] = r4[u];
    }
    __syncthreads();
    if (m0 + kStage < mlen) fetch(m0 + kStage);
#pragma unroll
    for (int mm = 0; mm < kStage; ++mm) {
      const float4 xa = *reinterpret_cast<const float4*>(&sX[mm][ty * 4]);
      const float4 yb = *reinterpret_cast<const float4*>(&sY[mm][tx * 4]);
      const float xv[4] = {xa.x, xa.y, xa.z, xa.w}, yv[4] = {yb.x, yb.y, yb.z, yb.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xv[i], yv[j], acc[i][j]);
    }
    if (which == 0) {
#pragma unroll
      for (int mm = 0; mm < kStage; ++mm) {
        const float4 xa = *reinterpret_cast<const float4*>(&sX2[mm][ty * 4]);
        const float4 yb = *reinterpret_cast<const float4*>(&sY2[mm][tx * 4]);
        const float xv[4] = {xa.x, xa.y, xa.z, xa.w}, yv[4] = {yb.x, yb.y, yb.z, yb.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xv[i], yv[j], acc[i][j]);
      }
    }
    __syncthreads();
  }
  float* out = ws + (which == 0 ? pd.sx_off : pd.sy_off);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = a0 + ty * 4 + i;
    if (a >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int f = f0 + tx * 4 + j;
      if (f < d) out[(int64_t)a * d + f] = acc[i][j];
    }
  }
}

// dA_s = sum of the shape's contributions, in pair order. Each thread sums four
// consecutive entries (one float4 per contribution when the shape's output is 16-byte
// aligned; the contribution slots always are).
__global__ void gather_da_kernel(BatchDev b, float* d_a, const float* ws) {
  const ShapeDev s = b.shapes[blockIdx.y];
  const int64_t kd = (int64_t)s.k * s.d;
  const int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (e0 >= kd) return;
  float* out = d_a + s.a_off;
  const bool vec = ((kd & 3) == 0) && ((reinterpret_cast<uintptr_t>(out) & 15) == 0);
  if (vec) {
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int q = s.slot_beg; q < s.slot_end; ++q) {
      const float4 u = *reinterpret_cast<const float4*>(ws + b.slot_list[q] + e0);
      acc.x += u.x; acc.y += u.y; acc.z += u.z; acc.w += u.w;
    }
    *reinterpret_cast<float4*>(out + e0) = acc;
  } else {
    for (int j = 0; j < 4 && e0 + j < kd; ++j) {
      float acc = 0.f;
      for (int q = s.slot_beg; q < s.slot_end; ++q) acc += ws[b.slot_list[q] + e0 + j];
      out[e0 + j] = acc;
    }
  }
}

// Training loss ||C C^T - I||^2 + ||C - C_gt||^2 and dL/dC = 4 (C C^T - I) C + 2 (C - C_gt),
// as two tiled passes over (64 x 64 output tile, pair):
//   pass 1: E = C C^T - I (into the workspace) and per-tile partial sums of the loss;
//   pass 2: dC = 4 E C + 2 (C - C_gt); tile 0 of each pair adds the partials in order.

__global__ void __launch_bounds__(256) loss_e_kernel(BatchDev b, const float* c_flat, const float* gt_flat,
                                                      float* ws, float* partial) {
  __shared__ __align__(16) float sX[kStage][kTile + 4];   // C^T[m][a] = C[a][m]
  __shared__ __align__(16) float sY[kStage][kTile + 4];   // C^T[m][b] = C[b][m]
  __shared__ float red[256];
  const int p = blockIdx.z;
  const PairDev pd = b.pairs[p];
  const int k = pd.k, ky = b.shapes[pd.y].k;   // C is ky x k, E = C C^T - I is ky x ky
  // tiles over ky rows and max(ky, k) columns: E where the column is < ky, the
  // ||C - C_gt||^2 term where it is < k
  const int nta = (ky + kTile - 1) / kTile, ntb = (max(ky, k) + kTile - 1) / kTile;
  if ((int)blockIdx.x >= nta * ntb) return;
  const int a0 = (blockIdx.x / ntb) * kTile, b0 = (blockIdx.x % ntb) * kTile;
  const float* c = c_flat + pd.c_off;
  const float* gt = gt_flat + pd.c_off;
  float* e = ws + pd.e_off;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4] = {};
  // the next stage's operands are loaded into registers while this stage computes
  float rx[kPer], ry[kPer];
  auto fetch = [&](int m0) {
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      // rows of C read in 16-element segments (consecutive threads, consecutive m)
      const int q = tid + 256 * u, r = q / kStage, mm = q % kStage;
      rx[u] = (a0 + r < ky && m0 + mm < k) ? c[(int64_t)(a0 + r) * k + m0 + mm] : 0.f;
      ry[u] = (b0 + r < ky && m0 + mm < k) ? c[(int64_t)(b0 + r) * k + m0 + mm] : 0.f;
    }
  };
  fetch(0);
  for (int m0 = 0; m0 < k; m0 += kStage) {
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int q = tid + 256 * u, r = q / kStage, mm = q % kStage;
      sX[mm][r] = rx[u];
      sY[mm][r] = ry[u];
    }
    __syncthreads();
    if (m0 + kStage < k) fetch(m0 + kStage);
#pragma unroll
    for (int mm = 0; mm < kStage; ++mm) {
      const float4 xa = *reinterpret_cast<const float4*>(&sX[mm][ty * 4]);
      const float4 yb = *reinterpret_cast<const float4*>(&sY[mm][tx * 4]);
      const float xv[4] = {xa.x, xa.y, xa.z, xa.w}, yv[4] = {yb.x, yb.y, yb.z, yb.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xv[i], yv[j], acc[i][j]);
    }
    __syncthreads();
  }
  float part = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = a0 + ty * 4 + i;
    if (a >= ky) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int bb = b0 + tx * 4 + j;
      if (bb < k) {
        const float r = c[(int64_t)a * k + bb] - gt[(int64_t)a * k + bb];
        part = fmaf(r, r, part);
      }
      if (bb < ky) {
        const float v = acc[i][j] - (a == bb ? 1.f : 0.f);
        e[(int64_t)a * ky + bb] = v;
        part = fmaf(v, v, part);
      }
    }
  }
  red[tid] = part;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (tid < st) red[tid] += red[tid + st];
    __syncthreads();
  }
  if (tid == 0) partial[(int64_t)p * kMaxLossTiles + blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(256) loss_grad_kernel(BatchDev b, const float* c_flat, const float* gt_flat,
                                                         float* loss, float* d_c, const float* ws,
                                                         const float* partial) {
  __shared__ __align__(16) float sX[kStage][kTile + 4];   // E^T[m][a] = E[a][m]
  __shared__ __align__(16) float sY[kStage][kTile + 4];   // C[m][b]
  const int p = blockIdx.z;
  const PairDev pd = b.pairs[p];
  const int k = pd.k, ky = b.shapes[pd.y].k;
  const int nta = (ky + kTile - 1) / kTile, ntb = (k + kTile - 1) / kTile;
  if (blockIdx.x == 0 && threadIdx.x == 0 && loss) {
    // the partial sums of loss_e's tiles, in tile order
    const int nte = nta * ((max(ky, k) + kTile - 1) / kTile);
    float total = 0.f;
    for (int t = 0; t < nte; ++t) total += partial[(int64_t)p * kMaxLossTiles + t];
    loss[p] = total;
  }
  if (d_c == nullptr) return;
  // dC = 4 E C + 2 (C - C_gt): ky x k tiles, reduction over ky
  if ((int)blockIdx.x >= nta * ntb) return;
  const int a0 = (blockIdx.x / ntb) * kTile, b0 = (blockIdx.x % ntb) * kTile;
  const float* c = c_flat + pd.c_off;
  const float* gt = gt_flat + pd.c_off;
  const float* e = ws + pd.e_off;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4] = {};
  // the next stage's operands are loaded into registers while this stage computes
  float rx[kPer], ry[kPer];
  auto fetch = [&](int m0) {
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int q = tid + 256 * u;
      {
        const int r = q / kStage, mm = q % kStage;
        rx[u] = (a0 + r < ky && m0 + mm < ky) ? e[(int64_t)(a0 + r) * ky + m0 + mm] : 0.f;
      }
      {
        const int mm = q / kTile, r = q % kTile;
        ry[u] = (b0 + r < k && m0 + mm < ky) ? c[(int64_t)(m0 + mm) * k + b0 + r] : 0.f;
      }
    }
  };
  fetch(0);
  for (int m0 = 0; m0 < ky; m0 += kStage) {
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int q = tid + 256 * u;
      sX[q % kStage][q / kStage] = rx[u];
      sY[q / kTile][q % kTile] = ry[u];
    }
    __syncthreads();
    if (m0 + kStage < ky) fetch(m0 + kStage);
#pragma unroll
    for (int mm = 0; mm < kStage; ++mm) {
      const float4 xa = *reinterpret_cast<const float4*>(&sX[mm][ty * 4]);
      const float4 yb = *reinterpret_cast<const float4*>(&sY[mm][tx * 4]);
      const float xv[4] = {xa.x, xa.y, xa.z, xa.w}, yv[4] = {yb.x, yb.y, yb.z, yb.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) acc[i][jj] = fmaf(xv[i], yv[jj], acc[i][jj]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = a0 + ty * 4 + i;
    if (a >= ky) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int bb = b0 + tx * 4 + j;
      if (bb >= k) continue;
      const int64_t idx = (int64_t)a * k + bb;
      d_c[pd.c_off + idx] = 4.f * acc[i][j] + 2.f * (c[idx] - gt[idx]);
    }
  }
}

__global__ void status_clear_kernel(int32_t* status, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) status[i] = 0;
}

}  // namespace

cudaError_t launch_adjoint_gemms(const BatchDev& b, int max_k, int max_d, const float* a, const float* c,
                                 float* d_mask, float* d_lambda, bool row_grads, float* ws, bool simt,
                                 cudaStream_t st) {
  if (b.n_pairs <= 0) return cudaSuccess;
  const int ntk = (max_k + kTile - 1) / kTile, ntd = (max_d + kTile - 1) / kTile;
  cudaError_t e;
  if (simt) {
    adjoint_w_kernel<<<dim3(ntk * ntk, 1, b.n_pairs), 256, 0, st>>>(b, c, ws);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (d_lambda || d_mask || row_grads) {
    adjoint_dlambda_kernel<<<b.n_pairs, 256, 0, st>>>(b, c, d_mask, d_lambda, ws);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (!simt) return cudaSuccess;
  adjoint_da_kernel<<<dim3(ntk * ntd, 2, b.n_pairs), 256, 0, st>>>(b, a, ws);
  return cudaGetLastError();
}

cudaError_t launch_gather_da(const BatchDev& b, int max_kd, float* d_a, const float* ws, cudaStream_t st) {
  if (b.n_shapes <= 0) return cudaSuccess;
  gather_da_kernel<<<dim3((max_kd + 1023) / 1024, b.n_shapes), 256, 0, st>>>(b, d_a, ws);
  return cudaGetLastError();
}

cudaError_t launch_loss_orth(const BatchDev& b, int max_k, const float* c, const float* c_gt, float* loss,
                             float* d_c, float* ws, float* partial, cudaStream_t st) {
  if (b.n_pairs <= 0) return cudaSuccess;
  const int nt = (max_k + kTile - 1) / kTile;
  loss_e_kernel<<<dim3(nt * nt, 1, b.n_pairs), 256, 0, st>>>(b, c, c_gt, ws, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  loss_grad_kernel<<<dim3(nt * nt, 1, b.n_pairs), 256, 0, st>>>(b, c, c_gt, loss, d_c, ws, partial);
  return cudaGetLastError();
}

cudaError_t launch_status_clear(int32_t* status, int n, cudaStream_t st) {
  if (n <= 0 || status == nullptr) return cudaSuccess;
  status_clear_kernel<<<(n + 255) / 256, 256, 0, st>>>(status, n);
  return cudaGetLastError();
}

}  // namespace fmap
