// Row-wise regularised solve (Eq. 5-9) and the adjoint row solves.
//
// One thread block per row system S_i = G + lambda diag(D_i) (row i of pair p).
// S_i is padded to kp = k rounded up to 8 (identity in the padding) and kept in
// shared memory as packed lower rows: row a holds 8 (a/8 + 1) + 4 floats, so a
// row's 8-column tile segment is two aligned float4 and consecutive rows fall on
// different banks. The factorisation is a blocked right-looking Cholesky in FP32
// with 8-column panels and one panel of lookahead:
//   TRSM     every thread solves one row of panel J below its diagonal block,
//            x = s L_JJ^-T, as a product with the stored inverse block;
//   (a)      every thread updates one row of the next column block J+1;
//   (b)      warp 0 factors the diagonal block J+1 in registers and stores its
//            inverse, while the other warps update the rest of the trailing matrix
//            in 8 x 8 register tiles, S_AB -= L_AJ L_BJ^T.
// Three block barriers per panel. Forward and back substitution are done by
// warp 0 with the inverse diagonal blocks (no dependency chain inside a block);
// then `ir_steps` steps of iterative refinement with the residual rhs - S x in
// FP32; for hi_gram pairs the residual takes G as the two FP32 halves (hi + lo)
// of its double-float accumulation.
#include <math.h>

#include "fmap_internal.cuh"

namespace fmap {
namespace {

// Offset of row a in the packed, skewed lower storage.
__host__ __device__ __forceinline__ int rowoff(int a) {
  const int q = a >> 3, s = a & 7;
  return 32 * q * (q + 2) + s * (8 * q + 12);
}

// Floats of one factor: the packed rows plus the Q inverse diagonal blocks.
__host__ __device__ __forceinline__ int factor_floats(int Q) { return 32 * Q * (Q + 2) + 64 * Q; }

__device__ __forceinline__ float mask_entry(const PairDev& pd, const float* evx, const float* evy, int i, int a) {
  if (pd.mask) return pd.mask[(int64_t)i * pd.k + a];
  const float t = evy[i] - evx[a];
  return t * t;
}

__device__ __forceinline__ void set_status(int32_t* status, int p, int32_t code) {
  if (status) atomicCAS(status + p, 0, code);
}

// Warp 0: factor the 8 x 8 diagonal block J in place (lane 0, registers) and store
// its inverse (lanes 0-7, one column each). Returns false on a bad pivot.
__device__ __forceinline__ bool diag_block(float* S, float* linv, int J, int lane) {
  const int r0 = 8 * J;
  bool bad = false;
  if (lane == 0) {
    float a[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) a[i][j] = S[rowoff(r0 + i) + r0 + j];
    float rinv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float piv = a[j][j];
      if (!(piv > 0.f) || !(piv < INFINITY)) bad = true;
      const float r = rsqrtf(piv);     // 1 / L_jj; iterative refinement absorbs its last-bit error
      a[j][j] = piv * r;
      rinv[j] = r;
#pragma unroll
      for (int i = j + 1; i < 8; ++i) a[i][j] *= r;
#pragma unroll
      for (int i = j + 1; i < 8; ++i)
#pragma unroll
        for (int m = j + 1; m <= i; ++m) a[i][m] = fmaf(-a[i][j], a[m][j], a[i][m]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j <= i; ++j) S[rowoff(r0 + i) + r0 + j] = a[i][j];
#pragma unroll
    for (int j = 0; j < 8; ++j) linv[J * 64 + j * 9] = rinv[j];   // diagonal of L_JJ^-1
  }
  bad = __shfl_sync(0xffffffffu, bad ? 1 : 0, 0) != 0;
  __syncwarp();
  if (lane < 8) {
    // column `lane` of L_JJ^-1: forward substitution on the unit vector
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float* row = S + rowoff(r0 + i) + r0;
      float t = (i == lane) ? 1.f : 0.f;
#pragma unroll
      for (int m = 0; m < i; ++m) t = fmaf(-row[m], x[m], t);
      x[i] = (i >= lane) ? t * linv[J * 64 + i * 9] : 0.f;
    }
    __syncwarp(0xffu);   // lanes 0-7: every diagonal entry is read before any column is stored
#pragma unroll
    for (int i = 0; i < 8; ++i) linv[J * 64 + i * 8 + lane] = x[i];
  }
  __syncwarp();
  return !bad;
}

// v <- L^{-1} v with every thread of the block (NT >= kp): thread t updates row
// r0 + 8 + t against y_J; warp 0 owns the next block's rows and applies its inverse
// diagonal block right after updating them. One barrier per 8-row block.
template <int NT>
__device__ __forceinline__ void block_fwd(const float* S, const float* linv, float* v, int Q, int tid, int lane,
                                          int warp) {
  const int kp = 8 * Q;
  if (warp == 0) {
    float y = 0.f;
    if (lane < 8)
#pragma unroll
      for (int j = 0; j < 8; ++j) y = fmaf(linv[lane * 8 + j], v[j], y);
    __syncwarp();
    if (lane < 8) v[lane] = y;
  }
  __syncthreads();
  for (int J = 0; J < Q; ++J) {
    const int r0 = 8 * J;
    const int a = r0 + 8 + tid;
    if (a < kp) {
      const float4* ra = reinterpret_cast<const float4*>(S + rowoff(a) + r0);
      const float4 l0 = ra[0], l1 = ra[1];
      const float4 y0 = *reinterpret_cast<const float4*>(v + r0);
      const float4 y1 = *reinterpret_cast<const float4*>(v + r0 + 4);
      float t = v[a];
      t = fmaf(-l0.x, y0.x, t); t = fmaf(-l0.y, y0.y, t); t = fmaf(-l0.z, y0.z, t); t = fmaf(-l0.w, y0.w, t);
      t = fmaf(-l1.x, y1.x, t); t = fmaf(-l1.y, y1.y, t); t = fmaf(-l1.z, y1.z, t); t = fmaf(-l1.w, y1.w, t);
      v[a] = t;
    }
    if (J + 1 < Q && warp == 0) {
      __syncwarp();
      float y = 0.f;
      if (lane < 8) {
        const float* li = linv + (J + 1) * 64 + lane * 8;
#pragma unroll
        for (int j = 0; j < 8; ++j) y = fmaf(li[j], v[r0 + 8 + j], y);
      }
      __syncwarp();
      if (lane < 8) v[r0 + 8 + lane] = y;
    }
    __syncthreads();
  }
}

// v <- L^{-T} v: thread t updates row t against x_J; the warp owning the previous
// block's rows applies that block's transposed inverse. One barrier per block.
template <int NT>
__device__ __forceinline__ void block_bwd(const float* S, const float* linv, float* v, int Q, int tid, int lane,
                                          int warp) {
  {
    const int r0 = 8 * (Q - 1);
    if (warp == (r0 >> 5)) {
      const int i = lane - (r0 & 31);
      float x = 0.f;
      if (i >= 0 && i < 8)
#pragma unroll
        for (int j = 0; j < 8; ++j) x = fmaf(linv[(Q - 1) * 64 + j * 8 + i], v[r0 + j], x);
      __syncwarp();
      if (i >= 0 && i < 8) v[r0 + i] = x;
    }
  }
  __syncthreads();
  for (int J = Q - 1; J >= 1; --J) {
    const int r0 = 8 * J;
    if (tid < r0) {
      float t = v[tid];
#pragma unroll
      for (int m = 0; m < 8; ++m) t = fmaf(-S[rowoff(r0 + m) + tid], v[r0 + m], t);
      v[tid] = t;
    }
    const int p0 = r0 - 8;                 // rows of block J - 1, owned by threads p0..p0+7
    if (warp == (p0 >> 5)) {
      __syncwarp();
      const int i = lane - (p0 & 31);
      float x = 0.f;
      if (i >= 0 && i < 8)
#pragma unroll
        for (int j = 0; j < 8; ++j) x = fmaf(linv[(J - 1) * 64 + j * 8 + i], v[p0 + j], x);
      __syncwarp();
      if (i >= 0 && i < 8) v[p0 + i] = x;
    }
    __syncthreads();
  }
}

template <int NT>
__global__ void __launch_bounds__(NT, (NT >= 256 ? 2 : (NT >= 128 ? 3 : 4)))
    chol_solve_kernel(BatchDev b, const int2* systems, int first, int count, int mode, const float* rhs_flat,
                      float* out_flat, float* saved, int32_t* status, float* ws) {
  constexpr int NW = NT / 32;
  extern __shared__ __align__(16) float smem[];
  __shared__ int s_bad;
  if ((int)blockIdx.x >= count) return;
  const int2 sys = systems[first + blockIdx.x];
  const int p = sys.x, i = sys.y;
  const PairDev pd = b.pairs[p];
  const int k = pd.k;
  const int Q = (k + 7) >> 3, kp = 8 * Q;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float* evx = b.shapes[pd.x].evals;
  const float* evy = b.shapes[pd.y].evals;
  const int ssz = rowoff(kp);
  float* S = smem;                 // packed skewed lower rows
  float* linv = S + ssz;           // inverse diagonal blocks, Q x 64
  float* pan = linv + 64 * Q;      // current panel, column-major: pan[c * kp + a]
  float* v = pan + 8 * kp;         // working vector
  float* xs = v + kp;              // solution
  float* rh = xs + kp;             // right-hand side
  const float* G = ws + pd.g_off;
  const float2* Ghl = pd.g64_off >= 0 ? reinterpret_cast<const float2*>(ws) + pd.g64_off : nullptr;
  const float* rhs = (mode == kSolveForward) ? ws + pd.r_off + (int64_t)i * k : rhs_flat + pd.c_off + (int64_t)i * k;
  float* out = (mode == kSolveForward) ? out_flat + pd.c_off + (int64_t)i * k : ws + pd.gam_off + (int64_t)i * k;
  const int fsz = factor_floats(Q);
  float* fac = (saved != nullptr && pd.fac_off >= 0) ? saved + pd.fac_off + (int64_t)i * fsz : nullptr;
  const float lam = pd.lam;

  if (tid == 0) {
    s_bad = 0;
    // a projection wait that timed out leaves its error in the workspace's first word
    if (i == 0 && reinterpret_cast<const int*>(ws)[0] != 0) set_status(status, p, FMAP_ERR_TIMEOUT);
  }
  for (int a = tid; a < kp; a += NT) rh[a] = a < k ? rhs[a] : 0.f;

  if (mode == kSolveAdjoint && fac != nullptr) {
    for (int e = tid; e < fsz / 4; e += NT) reinterpret_cast<float4*>(S)[e] = reinterpret_cast<const float4*>(fac)[e];
    __syncthreads();
  } else {
    // S = G + lambda diag(D_i), identity in the padding rows; one warp per row, four
    // rows' loads in flight before any store
    for (int a0 = warp; a0 < kp; a0 += 4 * NW) {
      float val[4][kMaxK / 32];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int a = a0 + u * NW;
        const float* grow = G + (int64_t)a * k;
#pragma unroll
        for (int q = 0; q < kMaxK / 32; ++q) {
          const int c = lane + 32 * q;
          val[u][q] = (a < k && c < a) ? grow[c] : 0.f;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int a = a0 + u * NW;
        if (a >= kp) break;
        float* row = S + rowoff(a);
        const int len = (a & ~7) + 8;
#pragma unroll
        for (int q = 0; q < kMaxK / 32; ++q) {
          const int c = lane + 32 * q;
          if (c < len) {
            float x = val[u][q];
            if (c == a) x = a < k ? G[(int64_t)a * k + a] + lam * mask_entry(pd, evx, evy, i, a) : 1.f;
            row[c] = x;
          }
        }
      }
    }
    for (int a = tid; a < kp; a += NT) v[a] = rh[a];   // right-hand side, reduced during the factorisation
    __syncthreads();
    if (warp == 0 && !diag_block(S, linv, 0, lane) && lane == 0) s_bad = 1;
    __syncthreads();
    for (int J = 0; J < Q && !s_bad; ++J) {
      const int r0 = 8 * J;
      const float* li = linv + J * 64;
      // forward substitution, bordered into the factorisation: y_J = L_JJ^-1 v_J
      if (warp == 0) {
        float y = 0.f;
        if (lane < 8)
#pragma unroll
          for (int j = 0; j < 8; ++j) y = fmaf(li[lane * 8 + j], v[r0 + j], y);
        __syncwarp();
        if (lane < 8) v[r0 + lane] = y;
      }
      // TRSM: rows below the diagonal block, x = s L_JJ^-T
      for (int a = r0 + 8 + tid; a < kp; a += NT) {
        float4* ra = reinterpret_cast<float4*>(S + rowoff(a) + r0);
        const float4 s0 = ra[0], s1 = ra[1];
        const float sv[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
        float x[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          float t = 0.f;
#pragma unroll
          for (int m = 0; m <= c; ++m) t = fmaf(sv[m], li[c * 8 + m], t);
          x[c] = t;
        }
        ra[0] = make_float4(x[0], x[1], x[2], x[3]);
        ra[1] = make_float4(x[4], x[5], x[6], x[7]);
#pragma unroll
        for (int c = 0; c < 8; ++c) pan[c * kp + a] = x[c];
      }
      __syncthreads();
      if (J + 1 == Q) break;
      // (a) the next column block, one row per thread; the row's right-hand side
      // takes the panel's contribution, v_a -= L_aJ y_J
      const int n0 = r0 + 8;
      for (int a = n0 + tid; a < kp; a += NT) {
        float4* ra = reinterpret_cast<float4*>(S + rowoff(a) + n0);
        const float4 u0 = ra[0], u1 = ra[1];
        float acc[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
        float va = v[a];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float la = pan[c * kp + a];
          va = fmaf(-la, v[r0 + c], va);
          const float4* pb = reinterpret_cast<const float4*>(pan + c * kp + n0);
          const float4 b0 = pb[0], b1 = pb[1];
          acc[0] = fmaf(-la, b0.x, acc[0]); acc[1] = fmaf(-la, b0.y, acc[1]);
          acc[2] = fmaf(-la, b0.z, acc[2]); acc[3] = fmaf(-la, b0.w, acc[3]);
          acc[4] = fmaf(-la, b1.x, acc[4]); acc[5] = fmaf(-la, b1.y, acc[5]);
          acc[6] = fmaf(-la, b1.z, acc[6]); acc[7] = fmaf(-la, b1.w, acc[7]);
        }
        ra[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
        ra[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
        v[a] = va;
      }
      __syncthreads();
      // (b) warp 0: next diagonal block; warps 1..: trailing tiles (A, B), J+2 <= B <= A < Q
      if (warp == 0) {
        if (!diag_block(S, linv, J + 1, lane) && lane == 0) s_bad = 1;
      } else {
        const int m = Q - J - 2;
        const int T = m * (m + 1) / 2;
        for (int t = tid - 32; t < T; t += NT - 32) {
          int ai = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
          while ((ai + 1) * (ai + 2) / 2 <= t) ++ai;
          while (ai * (ai + 1) / 2 > t) --ai;
          const int bi = t - ai * (ai + 1) / 2;
          const int A = 8 * (J + 2 + ai), B = 8 * (J + 2 + bi);
          float acc[8][8];
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const float4* sr = reinterpret_cast<const float4*>(S + rowoff(A + r) + B);
            const float4 u0 = sr[0], u1 = sr[1];
            acc[r][0] = u0.x; acc[r][1] = u0.y; acc[r][2] = u0.z; acc[r][3] = u0.w;
            acc[r][4] = u1.x; acc[r][5] = u1.y; acc[r][6] = u1.z; acc[r][7] = u1.w;
          }
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float4* pa = reinterpret_cast<const float4*>(pan + c * kp + A);
            const float4* pb = reinterpret_cast<const float4*>(pan + c * kp + B);
            const float4 a0 = pa[0], a1 = pa[1], b0 = pb[0], b1 = pb[1];
            const float la[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float lb[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
              for (int q = 0; q < 8; ++q) acc[r][q] = fmaf(-la[r], lb[q], acc[r][q]);
          }
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            float4* sr = reinterpret_cast<float4*>(S + rowoff(A + r) + B);
            sr[0] = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
            sr[1] = make_float4(acc[r][4], acc[r][5], acc[r][6], acc[r][7]);
          }
        }
      }
      __syncthreads();
    }
    if (s_bad) {
      if (tid == 0) set_status(status, p, FMAP_ERR_NOT_SPD | (i << 8));
      for (int a = tid; a < k; a += NT) out[a] = __int_as_float(0x7fc00000);
      return;
    }
    if (mode == kSolveForward && fac != nullptr)
      for (int e = tid; e < fsz / 4; e += NT) reinterpret_cast<float4*>(fac)[e] = reinterpret_cast<const float4*>(S)[e];
  }

  // x = S^{-1} rhs: the factorisation already applied L^{-1} to v; with loaded factors
  // the forward substitution runs here
  if (mode == kSolveAdjoint && fac != nullptr) {
    for (int a = tid; a < kp; a += NT) v[a] = rh[a];
    __syncthreads();
    block_fwd<NT>(S, linv, v, Q, tid, lane, warp);
  }
  block_bwd<NT>(S, linv, v, Q, tid, lane, warp);
  for (int a = tid; a < kp; a += NT) xs[a] = v[a];
  __syncthreads();

  // iterative refinement: x += S^{-1} (rhs - S x); four rows of G in flight per warp
  const int n_ir = mode == kSolveForward ? b.ir_steps : b.ir_steps_adj;
  for (int it = 0; it < n_ir; ++it) {
    for (int a0 = warp; a0 < kp; a0 += 4 * NW) {
      float sum[4] = {0.f, 0.f, 0.f, 0.f};
      if (Ghl) {
        float2 g[4][kMaxK / 32];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int a = a0 + u * NW;
#pragma unroll
          for (int q = 0; q < kMaxK / 32; ++q) {
            const int c = lane + 32 * q;
            g[u][q] = (a < k && c < k) ? Ghl[(int64_t)a * k + c] : make_float2(0.f, 0.f);
          }
        }
#pragma unroll
        for (int q = 0; q < kMaxK / 32; ++q) {
          const int c = lane + 32 * q;
          const float xv = c < k ? xs[c] : 0.f;
#pragma unroll
          for (int u = 0; u < 4; ++u) sum[u] = fmaf(g[u][q].y, xv, fmaf(g[u][q].x, xv, sum[u]));
        }
      } else {
        float g[4][kMaxK / 32];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int a = a0 + u * NW;
#pragma unroll
          for (int q = 0; q < kMaxK / 32; ++q) {
            const int c = lane + 32 * q;
            g[u][q] = (a < k && c < k) ? G[(int64_t)a * k + c] : 0.f;
          }
        }
#pragma unroll
        for (int q = 0; q < kMaxK / 32; ++q) {
          const int c = lane + 32 * q;
          const float xv = c < k ? xs[c] : 0.f;
#pragma unroll
          for (int u = 0; u < 4; ++u) sum[u] = fmaf(g[u][q], xv, sum[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum[u] += __shfl_xor_sync(0xffffffffu, sum[u], o);
        const int a = a0 + u * NW;
        if (lane == 0 && a < kp)
          v[a] = a < k ? rh[a] - fmaf(lam * mask_entry(pd, evx, evy, i, a), xs[a], sum[u]) : 0.f;
      }
    }
    __syncthreads();
    block_fwd<NT>(S, linv, v, Q, tid, lane, warp);
    block_bwd<NT>(S, linv, v, Q, tid, lane, warp);
    for (int a = tid; a < kp; a += NT) xs[a] += v[a];
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

size_t chol_smem_bytes(int kmax) {
  const int Q = (kmax + 7) / 8, kp = 8 * Q;
  return (size_t)(factor_floats(Q) + 8 * kp + 3 * kp) * sizeof(float);
}

template <int NT>
cudaError_t set_limit() {
  return cudaFuncSetAttribute(chol_solve_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)chol_smem_bytes(kMaxK));
}

}  // namespace

int64_t chol_factor_floats(int k) { return factor_floats((k + 7) / 8); }

cudaError_t solve_set_smem_limits() {
  cudaError_t e;
  if ((e = set_limit<64>()) != cudaSuccess) return e;
  if ((e = set_limit<128>()) != cudaSuccess) return e;
  return set_limit<256>();
}

cudaError_t launch_solve(const BatchDev& b, const SolveGroup& g, const int2* systems, int mode, const float* rhs_flat,
                         float* out_flat, float* saved, int32_t* status, float* ws, cudaStream_t st) {
  if (g.count <= 0) return cudaSuccess;
  const size_t smem = chol_smem_bytes(g.kmax);
  switch (g.threads) {
    case 64:
      chol_solve_kernel<64><<<g.count, 64, smem, st>>>(b, systems, g.first, g.count, mode, rhs_flat, out_flat, saved,
                                                       status, ws);
      break;
    case 128:
      chol_solve_kernel<128><<<g.count, 128, smem, st>>>(b, systems, g.first, g.count, mode, rhs_flat, out_flat,
                                                         saved, status, ws);
      break;
    default:
      chol_solve_kernel<256><<<g.count, 256, smem, st>>>(b, systems, g.first, g.count, mode, rhs_flat, out_flat,
                                                         saved, status, ws);
      break;
  }
  return cudaGetLastError();
}

}  // namespace fmap
