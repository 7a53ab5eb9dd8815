// Row-wise regularised solve (Eq. 5-9) and the adjoint row solves.
//
// One thread block per row system S_i = G + lambda diag(D_i) (row i of pair p).
// S_i is padded to kp = k rounded up to 8 (identity in the padding) and kept in
// shared memory as packed lower rows, row a padded to a multiple of 8 entries, so
// every 8 x 8 tile row segment is two aligned float4. The factorisation is a
// blocked right-looking Cholesky in FP32 with 8-column panels:
//   1. warp 0 factors the 8 x 8 diagonal block with shuffles;
//   2. every thread solves one row of the panel below it (L_aJ = S_aJ L_JJ^-T);
//   3. every thread updates 8 x 8 register tiles of the trailing matrix,
//      S_AB -= L_AJ L_BJ^T, reading the panel from a column-major buffer.
// Three block barriers per panel. Forward and back substitution are done by
// warp 0 in 8-row blocks; then `ir_steps` steps of iterative refinement with
// the residual rhs - S x accumulated in FP32, or in double-float (error-free
// products and sums, ~48 bits) from the (hi, lo) Gram for hi_gram pairs.
#include <math.h>

#include "fmap_internal.cuh"

namespace fmap {
namespace {

__host__ __device__ __forceinline__ int rowoff(int a) {
  const int q = a >> 3, s = a & 7;
  return 8 * (q + 1) * (4 * q + s);
}

__device__ __forceinline__ float mask_entry(const PairDev& pd, const float* evx, const float* evy, int i, int a) {
  if (pd.mask) return pd.mask[(int64_t)i * pd.k + a];
  const float t = evy[i] - evx[a];
  return t * t;
}

__device__ __forceinline__ void set_status(int32_t* status, int p, int32_t code) {
  if (status) atomicCAS(status + p, 0, code);
}

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

// Warp 0: in-place solve of L L^T v = v (L packed in S, kp = 8 Q).
__device__ __forceinline__ void warp_subst(const float* S, float* v, int Q, int lane) {
  for (int J = 0; J < Q; ++J) {                 // L y = v
    const int r0 = 8 * J;
    float yv = lane < 8 ? v[r0 + lane] : 0.f;
    const float* row = S + rowoff(r0 + (lane & 7));
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (lane == j) yv = yv / row[r0 + j];
      const float yj = __shfl_sync(0xffffffffu, yv, j);
      if (lane > j && lane < 8) yv = fmaf(-row[r0 + j], yj, yv);
    }
    __syncwarp();
    if (lane < 8) v[r0 + lane] = yv;
    __syncwarp();
    float y[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) y[m] = v[r0 + m];
    for (int a = r0 + 8 + lane; a < 8 * Q; a += 32) {
      const float4* ra = reinterpret_cast<const float4*>(S + rowoff(a) + r0);
      const float4 l0 = ra[0], l1 = ra[1];
      float t = v[a];
      t = fmaf(-l0.x, y[0], t); t = fmaf(-l0.y, y[1], t); t = fmaf(-l0.z, y[2], t); t = fmaf(-l0.w, y[3], t);
      t = fmaf(-l1.x, y[4], t); t = fmaf(-l1.y, y[5], t); t = fmaf(-l1.z, y[6], t); t = fmaf(-l1.w, y[7], t);
      v[a] = t;
    }
    __syncwarp();
  }
  for (int J = Q - 1; J >= 0; --J) {           // L^T x = y
    const int r0 = 8 * J;
    float xv = lane < 8 ? v[r0 + lane] : 0.f;
#pragma unroll
    for (int j = 7; j >= 0; --j) {
      const float* rj = S + rowoff(r0 + j);
      if (lane == j) xv = xv / rj[r0 + j];
      const float xj = __shfl_sync(0xffffffffu, xv, j);
      if (lane < j) xv = fmaf(-rj[r0 + lane], xj, xv);
    }
    __syncwarp();
    if (lane < 8) v[r0 + lane] = xv;
    __syncwarp();
    float x[8];
    const float* rr[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) { x[m] = v[r0 + m]; rr[m] = S + rowoff(r0 + m); }
    for (int a = lane; a < r0; a += 32) {
      float t = v[a];
#pragma unroll
      for (int m = 0; m < 8; ++m) t = fmaf(-rr[m][a], x[m], t);
      v[a] = t;
    }
    __syncwarp();
  }
}

template <int NT>
__global__ void __launch_bounds__(NT, (NT >= 256 ? 2 : (NT >= 128 ? 3 : 4))) chol_solve_kernel(BatchDev b, const int2* systems, int first, int count,
                                                       int mode, const float* rhs_flat, float* out_flat,
                                                       float* saved, int32_t* status, float* ws) {
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
  float* S = smem;                 // packed padded lower rows
  float* pan = S + ssz;            // panel, column-major: pan[c * kp + a]
  float* v = pan + 8 * kp;         // working vector
  float* xs = v + kp;              // solution
  float* rh = xs + kp;             // right-hand side
  const float* G = ws + pd.g_off;
  const float2* Ghl = pd.g64_off >= 0 ? reinterpret_cast<const float2*>(ws) + pd.g64_off : nullptr;
  const float* rhs = (mode == kSolveForward) ? ws + pd.r_off + (int64_t)i * k : rhs_flat + pd.c_off + (int64_t)i * k;
  float* out = (mode == kSolveForward) ? out_flat + pd.c_off + (int64_t)i * k : ws + pd.gam_off + (int64_t)i * k;
  float* fac = (saved != nullptr && pd.fac_off >= 0) ? saved + pd.fac_off + (int64_t)i * ssz : nullptr;
  const float lam = pd.lam;

  if (tid == 0) {
    s_bad = 0;
    // a projection wait that timed out leaves its error in the workspace's first word
    if (i == 0 && reinterpret_cast<const int*>(ws)[0] != 0) set_status(status, p, FMAP_ERR_TIMEOUT);
  }
  for (int a = tid; a < kp; a += NT) rh[a] = a < k ? rhs[a] : 0.f;

  if (mode == kSolveAdjoint && fac != nullptr) {
    for (int e = tid; e < ssz / 4; e += NT) reinterpret_cast<float4*>(S)[e] = reinterpret_cast<const float4*>(fac)[e];
    __syncthreads();
  } else {
    // S = G + lambda diag(D_i), identity in the padding rows
    for (int a = warp; a < kp; a += NW) {
      float* row = S + rowoff(a);
      const int len = (a & ~7) + 8;
      const float* grow = G + (int64_t)a * k;
      for (int c = lane; c < len; c += 32) {
        float val = 0.f;
        if (a < k) {
          if (c < a) val = grow[c];
          else if (c == a) val = grow[a] + lam * mask_entry(pd, evx, evy, i, a);
        } else if (c == a) {
          val = 1.f;
        }
        row[c] = val;
      }
    }
    __syncthreads();
    for (int J = 0; J < Q; ++J) {
      const int r0 = 8 * J;
      // 1. diagonal block
      if (warp == 0) {
        float x[8];
        const float* row = S + rowoff(r0 + (lane & 7)) + r0;
#pragma unroll
        for (int c = 0; c < 8; ++c) x[c] = lane < 8 ? row[c] : 0.f;
        bool bad = false;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float piv = __shfl_sync(0xffffffffu, x[j], j);
          if (!(piv > 0.f) || !(piv < INFINITY)) bad = true;
          const float d = sqrtf(piv);
          const float inv = 1.f / d;
          if (lane == j) x[j] = d;
          if (lane > j) x[j] *= inv;
#pragma unroll
          for (int c = j + 1; c < 8; ++c) {
            const float lc = __shfl_sync(0xffffffffu, x[j], c);
            if (lane >= c) x[c] = fmaf(-x[j], lc, x[c]);
          }
        }
        if (lane < 8) {
          float* wrow = S + rowoff(r0 + lane) + r0;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            wrow[c] = x[c];
            pan[c * kp + r0 + lane] = c <= lane ? x[c] : 0.f;
          }
        }
        if (lane == 0 && bad) s_bad = r0 + 1;
      }
      __syncthreads();
      if (s_bad) break;
      // 2. panel rows below the diagonal block: x L_JJ^T = s
      for (int a = r0 + 8 + tid; a < kp; a += NT) {
        float4* ra = reinterpret_cast<float4*>(S + rowoff(a) + r0);
        const float4 s0 = ra[0], s1 = ra[1];
        float s[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
        float x[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          float t = s[c];
#pragma unroll
          for (int m = 0; m < c; ++m) t = fmaf(-x[m], pan[m * kp + r0 + c], t);
          x[c] = t / pan[c * kp + r0 + c];
        }
        ra[0] = make_float4(x[0], x[1], x[2], x[3]);
        ra[1] = make_float4(x[4], x[5], x[6], x[7]);
#pragma unroll
        for (int c = 0; c < 8; ++c) pan[c * kp + a] = x[c];
      }
      __syncthreads();
      // 3. trailing update, 8 x 8 tiles (A, B) with J < B <= A < Q
      const int m = Q - J - 1;
      const int T = m * (m + 1) / 2;
      for (int t = tid; t < T; t += NT) {
        int ai = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
        while ((ai + 1) * (ai + 2) / 2 <= t) ++ai;
        while (ai * (ai + 1) / 2 > t) --ai;
        const int bi = t - ai * (ai + 1) / 2;
        const int A = 8 * (J + 1 + ai), B = 8 * (J + 1 + bi);
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
      __syncthreads();
    }
    if (s_bad) {
      // report the row system; the failing pivot lies in block (s_bad - 1) / 8
      if (tid == 0) set_status(status, p, FMAP_ERR_NOT_SPD | (i << 8));
      for (int a = tid; a < k; a += NT) out[a] = __int_as_float(0x7fc00000);
      return;
    }
    if (mode == kSolveForward && fac != nullptr)
      for (int e = tid; e < ssz / 4; e += NT) reinterpret_cast<float4*>(fac)[e] = reinterpret_cast<const float4*>(S)[e];
  }

  // x = S^{-1} rhs
  for (int a = tid; a < kp; a += NT) v[a] = rh[a];
  __syncthreads();
  if (warp == 0) warp_subst(S, v, Q, lane);
  __syncthreads();
  for (int a = tid; a < kp; a += NT) xs[a] = v[a];
  __syncthreads();

  // iterative refinement: x += S^{-1} (rhs - S x)
  for (int it = 0; it < b.ir_steps; ++it) {
    for (int a = warp; a < kp; a += NW) {
      float r = 0.f;
      if (a < k) {
        const float dterm = lam * mask_entry(pd, evx, evy, i, a);
        if (Ghl) {
          const float2* grow = Ghl + (int64_t)a * k;
          float hi = 0.f, lo = 0.f;
          for (int c = lane; c < k; c += 32) {
            const float2 g = grow[c];
            df_fma(hi, lo, g.x, xs[c]);
            lo = fmaf(g.y, xs[c], lo);
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
            const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
            const float s = __fadd_rn(hi, h2);
            const float bb = __fsub_rn(s, hi);
            const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(h2, bb));
            hi = s;
            lo = __fadd_rn(lo, __fadd_rn(l2, e));
          }
          // r = rhs - (hi + lo) - dterm * x_a, the large terms first
          const float dx = __fmul_rn(dterm, xs[a]);
          const float dxe = fmaf(dterm, xs[a], -dx);
          r = __fsub_rn(__fsub_rn(rh[a], hi), dx) - (lo + dxe);
        } else {
          const float* grow = G + (int64_t)a * k;
          float sum = 0.f;
          for (int c = lane; c < k; c += 32) sum = fmaf(grow[c], xs[c], sum);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
          r = rh[a] - fmaf(dterm, xs[a], sum);
        }
      }
      if (lane == 0) v[a] = r;
    }
    __syncthreads();
    if (warp == 0) warp_subst(S, v, Q, lane);
    __syncthreads();
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
  return (size_t)(rowoff(kp) + 8 * kp + 3 * kp) * sizeof(float);
}

template <int NT>
cudaError_t set_limit() {
  return cudaFuncSetAttribute(chol_solve_kernel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)chol_smem_bytes(kMaxK));
}

}  // namespace

int64_t chol_factor_floats(int k) {
  const int Q = (k + 7) / 8;
  return rowoff(8 * Q);
}

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
