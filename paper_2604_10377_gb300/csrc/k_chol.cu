// Row-wise regularised solve (Eq. 5-9) and the adjoint row solves.
//
// One thread block per row system S_i = G + lambda diag(D_i) (row i of pair p).
// S_i is padded to kp = k rounded up to 8 (identity in the padding) and kept in
// shared memory as packed lower rows (rowoff: row a holds 8 (a/8 + 1) + 4 floats, so a
// row's 8-column tile segment is two aligned float4 and consecutive rows fall on
// different banks). The Gram kernel leaves G in that layout too, so one bulk copy
// loads it; then lambda D_i is added to the diagonal. The factorisation is a blocked
// right-looking Cholesky in FP32 with 8-column panels and one panel of lookahead:
//   TRSM     every thread solves one row of panel J below its diagonal block,
//            x = s L_JJ^-T, as a product with the stored inverse block; one warp
//            applies L_JJ^-1 to the right-hand side (forward substitution bordered
//            into the factorisation);
//   (a)      every thread updates one row of the next column block J+1 and its
//            right-hand side entry;
//   (b)      warp 0 factors the diagonal block J+1 in registers and stores its
//            inverse, while the other warps update the rest of the trailing matrix
//            in 8x4 or 4x4 register tiles (whichever balances best),
//            S_AB -= L_AJ L_BJ^T, two columns per packed FP32x2 FMA (each lane of the
//            pair rounds like a scalar fmaf).
// (a) and (b) touch disjoint blocks, so a panel costs two block barriers. The back
// substitution and the refinement's triangular solves use every warp with the inverses
// of 16-row diagonal blocks (one barrier per 16 rows); `ir_steps` steps of iterative refinement
// take the residual rhs - S x in FP32, for hi_gram pairs with G as the two FP32
// halves (hi + lo) of its double-float accumulation.
#include <math.h>

#include "fmap_internal.cuh"
#include "tc_ptx.cuh"

namespace fmap {
namespace {

// Rounds of 128 columns that cover a row of G in the refinement residual.
constexpr int kResRounds = (kMaxK + 127) / 128;

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

// Warp 0: factor the 8 x 8 diagonal block J in place and store its inverse. Lanes
// 0-7 each factor the block in registers (the same arithmetic on every lane, loads
// broadcast), then lane c forms column c of L_JJ^-1 from its own registers. Returns
// false on a bad pivot.
__device__ __forceinline__ bool diag_block(float* S, float* linv, int J, int lane) {
  const int r0 = 8 * J;
  bool bad = false;
  if (lane < 8) {
    float a[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float4* rp = reinterpret_cast<const float4*>(S + rowoff(r0 + i) + r0);
      const float4 u0 = rp[0], u1 = rp[1];
      a[i][0] = u0.x; a[i][1] = u0.y; a[i][2] = u0.z; a[i][3] = u0.w;
      a[i][4] = u1.x; a[i][5] = u1.y; a[i][6] = u1.z; a[i][7] = u1.w;
    }
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
    // column `lane` of L_JJ^-1: forward substitution on the unit vector
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float t = (i == lane) ? 1.f : 0.f;
#pragma unroll
      for (int m = 0; m < i; ++m) t = fmaf(-a[i][m], x[m], t);
      x[i] = (i >= lane) ? t * rinv[i] : 0.f;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) linv[J * 64 + i * 8 + lane] = x[i];
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float4* rp = reinterpret_cast<float4*>(S + rowoff(r0 + i) + r0);
        rp[0] = make_float4(a[i][0], a[i][1], a[i][2], a[i][3]);
        rp[1] = make_float4(a[i][4], a[i][5], a[i][6], a[i][7]);
      }
    }
  }
  bad = __shfl_sync(0xffffffffu, bad ? 1 : 0, 0) != 0;
  __syncwarp();
  return !bad;
}

// Row index of entry t of a lower triangle enumerated row by row (t = a(a+1)/2 + b).
__device__ __forceinline__ void tri_decode(int t, int& a, int& b) {
  int ai = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while ((ai + 1) * (ai + 2) / 2 <= t) ++ai;
  while (ai * (ai + 1) / 2 > t) --ai;
  a = ai;
  b = t - ai * (ai + 1) / 2;
}

__device__ __forceinline__ uint64_t pk2(float x, float y) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ void upk2(uint64_t v, float& x, float& y) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v));
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// S[A.., B..] -= L[A.., J] L[B.., J]^T for one R x C tile (R, C in {4, 8}), with the
// panel's 8 columns read from `pan` (column-major, leading dimension kp). Pairs of
// columns are updated with packed FP32x2 FMAs.
template <int R, int C>
__device__ __forceinline__ void trail_tile(float* S, const float* pan, int kp, int A, int B) {
  uint64_t acc[R][C / 2];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const float4* sr = reinterpret_cast<const float4*>(S + rowoff(A + r) + B);
#pragma unroll
    for (int h = 0; h < C / 4; ++h) {
      const float4 u = sr[h];
      acc[r][2 * h] = pk2(u.x, u.y); acc[r][2 * h + 1] = pk2(u.z, u.w);
    }
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    float la[R];
    uint64_t lb[C / 2];
    const float4* pa = reinterpret_cast<const float4*>(pan + c * kp + A);
    const float4* pb = reinterpret_cast<const float4*>(pan + c * kp + B);
#pragma unroll
    for (int h = 0; h < R / 4; ++h) {
      const float4 u = pa[h];
      la[4 * h] = -u.x; la[4 * h + 1] = -u.y; la[4 * h + 2] = -u.z; la[4 * h + 3] = -u.w;
    }
#pragma unroll
    for (int h = 0; h < C / 4; ++h) {
      const float4 u = pb[h];
      lb[2 * h] = pk2(u.x, u.y); lb[2 * h + 1] = pk2(u.z, u.w);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint64_t l2 = pk2(la[r], la[r]);
#pragma unroll
      for (int q = 0; q < C / 2; ++q) acc[r][q] = fma2(l2, lb[q], acc[r][q]);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    float4* sr = reinterpret_cast<float4*>(S + rowoff(A + r) + B);
#pragma unroll
    for (int h = 0; h < C / 4; ++h) {
      float x0, x1, x2, x3;
      upk2(acc[r][2 * h], x0, x1); upk2(acc[r][2 * h + 1], x2, x3);
      sr[h] = make_float4(x0, x1, x2, x3);
    }
  }
}

// The triangular solves work on 16-row blocks p (rows 16p .. 16p+15; the last block has
// 8 rows when Q is odd). The inverse of a 16-row diagonal block is formed from the two
// 8x8 inverses A^-1, B^-1 and the block below the diagonal L21:
//   [A 0; L21 B]^-1 = [A^-1 0; M B^-1] with M = -B^-1 L21 A^-1,
// and M (64 floats per 16-row block) is computed once per factor: one thread per column j
// of a block forms T = L21 (column j of A^-1), then column j of M = -B^-1 T.
__device__ __forceinline__ void load8(const float* src, float (&d)[8]) {
  const float4 u0 = reinterpret_cast<const float4*>(src)[0], u1 = reinterpret_cast<const float4*>(src)[1];
  d[0] = u0.x; d[1] = u0.y; d[2] = u0.z; d[3] = u0.w;
  d[4] = u1.x; d[5] = u1.y; d[6] = u1.z; d[7] = u1.w;
}

__device__ __forceinline__ void pair_blocks_prepare(const float* S, const float* linv, float* mo, int Q, int tid,
                                                    int nt) {
  const int np = Q >> 1;   // 16-row blocks with two 8-row halves
  for (int e = tid; e < np * 8; e += nt) {
    const int p = e >> 3, j = e & 7;
    const float* Ai = linv + (2 * p) * 64;        // A^-1, row-major
    const float* Bi = linv + (2 * p + 1) * 64;    // B^-1
    float ac[8];
#pragma unroll
    for (int l = 0; l < 8; ++l) ac[l] = Ai[l * 8 + j];
    float T[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      // (L21 A^-1)[m][j]
      float l21[8];
      load8(S + rowoff(16 * p + 8 + m) + 16 * p, l21);
      float t = 0.f;
#pragma unroll
      for (int l = 0; l < 8; ++l) t = fmaf(l21[l], ac[l], t);
      T[m] = t;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float bi[8];
      load8(Bi + i * 8, bi);
      float acc = 0.f;
#pragma unroll
      for (int m = 0; m < 8; ++m) acc = fmaf(bi[m], T[m], acc);
      mo[p * 64 + i * 8 + j] = -acc;
    }
  }
}

// Lanes 0-15 of one warp: v[16p ..] <- (16-row diagonal block p)^-1 v[16p ..].
__device__ __forceinline__ void apply_inv_fwd(const float* linv, const float* mo, float* v, int p, int Q, int lane) {
  const int r0 = 16 * p;
  const bool two = 2 * p + 1 < Q;
  float y = 0.f;
  if (lane < 8) {
    float a[8], vt[8];
    load8(linv + (2 * p) * 64 + lane * 8, a);
    load8(v + r0, vt);
#pragma unroll
    for (int j = 0; j < 8; ++j) y = fmaf(a[j], vt[j], y);
  } else if (lane < 16 && two) {
    const int i = lane - 8;
    float mi[8], bi[8], vt[8], vb[8];
    load8(mo + p * 64 + i * 8, mi);
    load8(linv + (2 * p + 1) * 64 + i * 8, bi);
    load8(v + r0, vt);
    load8(v + r0 + 8, vb);
#pragma unroll
    for (int j = 0; j < 8; ++j) y = fmaf(mi[j], vt[j], fmaf(bi[j], vb[j], y));
  }
  __syncwarp();
  if (lane < (two ? 16 : 8)) v[r0 + lane] = y;
  __syncwarp();
}

// Lanes l0 .. l0+15 of one warp: v[16p ..] <- (16-row diagonal block p)^-T v[16p ..].
__device__ __forceinline__ void apply_inv_bwd(const float* linv, const float* mo, float* v, int p, int Q, int i) {
  const int r0 = 16 * p;
  const bool two = 2 * p + 1 < Q;
  float x = 0.f;
  if (i >= 0 && i < 8) {
    const float* Ai = linv + (2 * p) * 64;
    float vt[8];
    load8(v + r0, vt);
#pragma unroll
    for (int j = 0; j < 8; ++j) x = fmaf(Ai[j * 8 + i], vt[j], x);
    if (two) {
      const float* Mp = mo + p * 64;
      float vb[8];
      load8(v + r0 + 8, vb);
#pragma unroll
      for (int j = 0; j < 8; ++j) x = fmaf(Mp[j * 8 + i], vb[j], x);
    }
  } else if (i >= 8 && i < 16 && two) {
    const float* Bi = linv + (2 * p + 1) * 64;
    float vb[8];
    load8(v + r0 + 8, vb);
#pragma unroll
    for (int j = 0; j < 8; ++j) x = fmaf(Bi[j * 8 + (i - 8)], vb[j], x);
  }
  __syncwarp();
  if (i >= 0 && i < (two ? 16 : 8)) v[r0 + i] = x;
  __syncwarp();
}

// v <- L^{-1} v with every thread of the block (NT >= kp): thread t updates row
// r0 + 16 + t against the finished block; warp 0 owns the next block's rows and applies
// its inverse right after updating them. One block barrier per 16-row block.
template <int NT>
__device__ __forceinline__ void block_fwd(const float* S, const float* linv, const float* mo, float* v, int Q,
                                          int tid, int lane, int warp) {
  const int kp = 8 * Q, nb = (Q + 1) >> 1;
  if (warp == 0) apply_inv_fwd(linv, mo, v, 0, Q, lane);
  __syncthreads();
  for (int p = 0; p + 1 < nb; ++p) {
    const int r0 = 16 * p;
    const int a = r0 + 16 + tid;
    if (a < kp) {
      const float4* ra = reinterpret_cast<const float4*>(S + rowoff(a) + r0);
      const float4* ya = reinterpret_cast<const float4*>(v + r0);
      float t = v[a];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const float4 l = ra[h], y = ya[h];
        t = fmaf(-l.x, y.x, t); t = fmaf(-l.y, y.y, t); t = fmaf(-l.z, y.z, t); t = fmaf(-l.w, y.w, t);
      }
      v[a] = t;
    }
    if (warp == 0) {
      __syncwarp();
      apply_inv_fwd(linv, mo, v, p + 1, Q, lane);
    }
    __syncthreads();
  }
}

// v <- L^{-T} v: thread t updates row t against the finished block; the warp owning the
// previous block's rows applies that block's transposed inverse. One barrier per block.
template <int NT>
__device__ __forceinline__ void block_bwd(const float* S, const float* linv, const float* mo, float* v, int Q,
                                          int tid, int lane, int warp) {
  const int kp = 8 * Q, nb = (Q + 1) >> 1;
  {
    const int r0 = 16 * (nb - 1);
    if (warp == (r0 >> 5)) apply_inv_bwd(linv, mo, v, nb - 1, Q, lane - (r0 & 31));
  }
  __syncthreads();
  for (int p = nb - 1; p >= 1; --p) {
    const int r0 = 16 * p;
    const int w = (r0 + 16 <= kp) ? 16 : 8;
    if (tid < r0) {
      float t = v[tid];
      float vt[8];
      load8(v + r0, vt);
#pragma unroll
      for (int m = 0; m < 8; ++m) t = fmaf(-S[rowoff(r0 + m) + tid], vt[m], t);
      if (w == 16) {
        float vb[8];
        load8(v + r0 + 8, vb);
#pragma unroll
        for (int m = 0; m < 8; ++m) t = fmaf(-S[rowoff(r0 + 8 + m) + tid], vb[m], t);
      }
      v[tid] = t;
    }
    const int p0 = r0 - 16;                 // rows of block p - 1, owned by threads p0..p0+15
    if (warp == (p0 >> 5)) {
      __syncwarp();
      apply_inv_bwd(linv, mo, v, p - 1, Q, lane - (p0 & 31));
    }
    __syncthreads();
  }
}

template <int NT>
__global__ void __launch_bounds__(NT, (NT > 256 ? 1 : (NT >= 256 ? 2 : (NT >= 128 ? 4 : 8))))
    chol_solve_kernel(BatchDev b, const int2* systems, int first, int count, int mode, const float* rhs_flat,
                      float* out_flat, float* saved, int32_t* status, float* ws, int gs_ok) {
  constexpr int NW = NT / 32;
  extern __shared__ __align__(16) float smem[];
  __shared__ int s_bad;
  __shared__ __align__(8) uint64_t s_bar;   // bulk copies of the Gram rows
  __shared__ int s_abort;
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
  float* dg = rh + kp;             // lambda D_i (the diagonal shift of this row system)
  float* Gs = dg + kp;             // copy of G for the refinement residual (launches with gs_ok)
  const float* G = ws + pd.g_off;
  const int ldg = gram_ld(k);
  const float2* Ghl = pd.g64_off >= 0 ? reinterpret_cast<const float2*>(ws) + pd.g64_off : nullptr;
  const float* rhs = (mode == kSolveForward) ? ws + pd.r_off + (int64_t)i * k : rhs_flat + pd.c_off + (int64_t)i * k;
  float* out = (mode == kSolveForward) ? out_flat + pd.c_off + (int64_t)i * k : ws + pd.gam_off + (int64_t)i * k;
  const int fsz = factor_floats(Q);
  float* fac = (saved != nullptr && pd.fac_off >= 0) ? saved + pd.fac_off + (int64_t)i * fsz : nullptr;
  const float lam = pd.lam_rows ? pd.lam_rows[i] : pd.lam;   // row weight of this system
  const int n_ir = mode == kSolveForward ? b.ir_steps : b.ir_steps_adj;
  // small FP32-Gram systems keep G in shared memory for the refinement residual
  const bool use_gs = gs_ok != 0 && Ghl == nullptr && n_ir > 0;
  const uint32_t gs_bytes = use_gs ? (uint32_t)k * (uint32_t)ldg * 4u : 0u;

  if (tid == 0) {
    s_bad = 0;
    s_abort = 0;
    tc::mbar_init(&s_bar, 1);
    tc::fence_mbar_init();
    // a projection wait that timed out leaves its error in the workspace's first word
    if (i == 0 && reinterpret_cast<const int*>(ws)[0] != 0) set_status(status, p, FMAP_ERR_TIMEOUT);
  }
  for (int a = tid; a < kp; a += NT) {
    rh[a] = a < k ? rhs[a] : 0.f;
    dg[a] = a < k ? lam * mask_entry(pd, evx, evy, i, a) : 0.f;
  }

  if (mode == kSolveAdjoint && fac != nullptr) {
    // the saved factor (packed rows and inverse blocks) and, for refinement, G: bulk copies
    __syncthreads();   // barrier initialised
    if (tid == 0) {
      tc::mbar_arrive_expect_tx(&s_bar, (uint32_t)fsz * 4u + gs_bytes);
      tc::bulk_g2s(S, fac, (uint32_t)fsz * 4u, &s_bar);
      if (use_gs) tc::bulk_g2s(Gs, G, gs_bytes, &s_bar);
    }
    tc::mbar_wait(&s_bar, 0, &s_abort);
    __syncthreads();
    if (s_abort) {
      // a copy that never completed: report, give it a bounded time to land, leave (every
      // thread of the block takes this branch together)
      if (tid == 0) set_status(status, p, FMAP_ERR_TIMEOUT);
      const uint64_t t0 = tc::globaltimer();
      while (!tc::mbar_try_wait(&s_bar, 0) && tc::globaltimer() - t0 < tc::kWaitTimeoutNs) {}
      return;
    }
  } else {
    // S = G + lambda diag(D_i). The Gram kernel left rows 0 .. k-1 of G in this packed
    // layout (each row up to the end of its diagonal block; the entries above the
    // diagonal inside a diagonal block are never read): one bulk copy brings them in
    // (with G itself for the residual when it stays in shared memory). Padding rows are
    // identity rows, written meanwhile.
    __syncthreads();   // barrier initialised
    if (tid == 0) {
      const uint32_t s_bytes = (uint32_t)rowoff(k) * 4u;
      tc::mbar_arrive_expect_tx(&s_bar, s_bytes + gs_bytes);
      tc::bulk_g2s(S, G + gram_packed_off(k), s_bytes, &s_bar);
      if (use_gs) tc::bulk_g2s(Gs, G, gs_bytes, &s_bar);
    }
    for (int a = k + tid; a < kp; a += NT) {
      float* row = S + rowoff(a);
      for (int c = 0; c < (a & ~7) + 8; ++c) row[c] = (c == a) ? 1.f : 0.f;
    }
    tc::mbar_wait(&s_bar, 0, &s_abort);
    __syncthreads();   // every thread's copies are visible
    if (s_abort) {
      if (tid == 0) set_status(status, p, FMAP_ERR_TIMEOUT);
      const uint64_t t0 = tc::globaltimer();
      while (!tc::mbar_try_wait(&s_bar, 0) && tc::globaltimer() - t0 < tc::kWaitTimeoutNs) {}
      return;
    }
    for (int a = tid; a < k; a += NT) S[rowoff(a) + a] += dg[a];
    for (int a = tid; a < kp; a += NT) v[a] = rh[a];   // right-hand side, reduced during the factorisation
    __syncthreads();
    if (warp == 0 && !diag_block(S, linv, 0, lane) && lane == 0) s_bad = 1;
    __syncthreads();
    for (int J = 0; J < Q && !s_bad; ++J) {
      const int r0 = 8 * J;
      const float* li = linv + J * 64;
      // forward substitution, bordered into the factorisation: y_J = L_JJ^-1 v_J, on the
      // last warp when it has no panel rows (off the TRSM's critical path), else warp 0
      const int yw = (r0 + 8 + (NW - 1) * 32 >= kp) ? NW - 1 : 0;
      if (warp == yw) {
        float y = 0.f;
        if (lane < 8)
#pragma unroll
          for (int j = 0; j < 8; ++j) y = fmaf(li[lane * 8 + j], v[r0 + j], y);
        __syncwarp();
        if (lane < 8) v[r0 + lane] = y;
      }
      // TRSM: rows below the diagonal block, x = s L_JJ^-T. Thread t owns row r0 + 8 + t
      // (every launch has NT >= kp threads) here and in (a), which reuses x.
      const int ar = r0 + 8 + tid;
      float x[8];
      if (ar < kp) {
        float4* ra = reinterpret_cast<float4*>(S + rowoff(ar) + r0);
        const float4 s0 = ra[0], s1 = ra[1];
        const float sv[8] = {s0.x, s0.y, s0.z, s0.w, s1.x, s1.y, s1.z, s1.w};
        const float4* l4 = reinterpret_cast<const float4*>(li);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float4 q0 = l4[2 * c];
          float lr[8] = {q0.x, q0.y, q0.z, q0.w, 0.f, 0.f, 0.f, 0.f};
          if (c >= 4) {
            const float4 q1 = l4[2 * c + 1];
            lr[4] = q1.x; lr[5] = q1.y; lr[6] = q1.z; lr[7] = q1.w;
          }
          float t = 0.f;
#pragma unroll
          for (int m = 0; m <= c; ++m) t = fmaf(sv[m], lr[m], t);
          x[c] = t;
        }
        ra[0] = make_float4(x[0], x[1], x[2], x[3]);
        ra[1] = make_float4(x[4], x[5], x[6], x[7]);
#pragma unroll
        for (int c = 0; c < 8; ++c) pan[c * kp + ar] = x[c];
      }
      __syncthreads();
      if (J + 1 == Q) break;
      // (a) the next column block, one row per thread; the row's right-hand side
      // takes the panel's contribution, v_a -= L_aJ y_J
      const int n0 = r0 + 8;
      if (ar < kp) {
        float4* ra = reinterpret_cast<float4*>(S + rowoff(ar) + n0);
        const float4 u0 = ra[0], u1 = ra[1];
        float acc[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
        const float4 y0 = reinterpret_cast<const float4*>(v + r0)[0], y1 = reinterpret_cast<const float4*>(v + r0)[1];
        const float yv[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
        float va = v[ar];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float la = x[c];
          va = fmaf(-la, yv[c], va);
          const float4* pb = reinterpret_cast<const float4*>(pan + c * kp + n0);
          const float4 b0 = pb[0], b1 = pb[1];
          acc[0] = fmaf(-la, b0.x, acc[0]); acc[1] = fmaf(-la, b0.y, acc[1]);
          acc[2] = fmaf(-la, b0.z, acc[2]); acc[3] = fmaf(-la, b0.w, acc[3]);
          acc[4] = fmaf(-la, b1.x, acc[4]); acc[5] = fmaf(-la, b1.y, acc[5]);
          acc[6] = fmaf(-la, b1.z, acc[6]); acc[7] = fmaf(-la, b1.w, acc[7]);
        }
        ra[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
        ra[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
        v[ar] = va;
      }
      // (a) writes column block J+1 and (b)'s tiles touch only blocks J+2.. (both read the
      // panel), so no block barrier separates them: warp 0 updated the diagonal block's
      // rows itself (threads 0-7) and factors it right away
      __syncwarp();
      // (b) warp 0: next diagonal block; warps 1..: trailing tiles (A, B), J+2 <= B <= A < Q
      if (warp == 0) {
        if (!diag_block(S, linv, J + 1, lane) && lane == 0) s_bad = 1;
      } else {
        // trailing blocks (A, B), J+2 <= B <= A < Q, as 8x4 or 4x4 register tiles: the
        // size whose rounds over the NT - 32 threads cost the fewest instructions (8x8
        // tiles fit the registers only with a partly rolled panel loop and ran slower)
        const int m = Q - J - 2;
        const int nb = NT - 32, t0 = tid - 32, base = 8 * (J + 2);
        const int T84 = m * (m + 1), T44 = m * (2 * m + 1);
        const int c84 = (T84 + nb - 1) / nb * 296, c44 = (T44 + nb - 1) / nb * 152;
        if (c84 <= c44) {
          for (int t = t0; t < T84; t += nb) {
            int ai, bi;
            tri_decode(t >> 1, ai, bi);
            trail_tile<8, 4>(S, pan, kp, base + 8 * ai, base + 8 * bi + 4 * (t & 1));
          }
        } else {
          for (int t = t0; t < T44; t += nb) {
            int ai, bi;
            tri_decode(t, ai, bi);
            trail_tile<4, 4>(S, pan, kp, base + 4 * ai, base + 4 * bi);
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

  // inverses of the 16-row diagonal blocks (their off-diagonal parts, in the panel's space)
  float* mo = pan;
  pair_blocks_prepare(S, linv, mo, Q, tid, NT);
  __syncthreads();

  // x = S^{-1} rhs: the factorisation already applied L^{-1} to v; with loaded factors
  // the forward substitution runs here
  if (mode == kSolveAdjoint && fac != nullptr) {
    for (int a = tid; a < kp; a += NT) v[a] = rh[a];
    __syncthreads();
    block_fwd<NT>(S, linv, mo, v, Q, tid, lane, warp);
  }
  block_bwd<NT>(S, linv, mo, v, Q, tid, lane, warp);
  float* ycol = pan + 4 * kp;   // past the 16-row inverse blocks (mo holds at most 4 kp floats)
  for (int a = tid; a < kp; a += NT) {
    xs[a] = v[a];
    ycol[a] = 0.f;
  }
  __syncthreads();

  // iterative refinement: x += S^{-1} (rhs - S x). With G in shared memory every thread
  // forms one row's residual (float4 reads, four partial sums); otherwise the warps read
  // the lower triangle of G from global memory, four rows in flight per warp.
  const float* Gres = use_gs ? Gs : G;
  for (int it = 0; it < n_ir; ++it) {
    if (use_gs) {
      for (int a = tid; a < kp; a += NT) {
        float s4[4] = {0.f, 0.f, 0.f, 0.f};
        if (a < k) {
          const float4* gr = reinterpret_cast<const float4*>(Gs + (int64_t)a * ldg);
          const float4* xq = reinterpret_cast<const float4*>(xs);
          const int nq = k >> 2;   // full quads; the columns past k hold no G entries
          for (int q = 0; q < nq; ++q) {
            const float4 g4 = gr[q], x4 = xq[q];
            s4[0] = fmaf(g4.x, x4.x, s4[0]);
            s4[1] = fmaf(g4.y, x4.y, s4[1]);
            s4[2] = fmaf(g4.z, x4.z, s4[2]);
            s4[3] = fmaf(g4.w, x4.w, s4[3]);
          }
          for (int c = 4 * nq; c < k; ++c) s4[c & 3] = fmaf(Gs[(int64_t)a * ldg + c], xs[c], s4[c & 3]);
        }
        v[a] = a < k ? rh[a] - fmaf(dg[a], xs[a], (s4[0] + s4[1]) + (s4[2] + s4[3])) : 0.f;
      }
      __syncthreads();
      block_fwd<NT>(S, linv, mo, v, Q, tid, lane, warp);
      block_bwd<NT>(S, linv, mo, v, Q, tid, lane, warp);
      for (int a = tid; a < kp; a += NT) xs[a] += v[a];
      __syncthreads();
      continue;
    }
    // G is symmetric: only its lower triangle is read. Row a's entries c <= a give the row
    // part of (G x)_a (reduced across the warp into v[a]); each entry c < a also gives
    // G_ac x_a to (G x)_c, summed per lane over the warp's rows (column c = lane + 32 j in
    // colacc[j]) and added into ycol warp by warp in a fixed order (reproducible sums).
    float colacc[4 * kResRounds];
#pragma unroll
    for (int j = 0; j < 4 * kResRounds; ++j) colacc[j] = 0.f;
    for (int a0 = warp; a0 < kp; a0 += 4 * NW) {
      float sum[4] = {0.f, 0.f, 0.f, 0.f};
      float xa[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int a = a0 + u * NW;
        xa[u] = a < k ? xs[a] : 0.f;
      }
      const int amax = min(a0 + 3 * NW, k - 1);   // the longest row of the group
#pragma unroll
      for (int r = 0; r < kResRounds; ++r) {       // 128 columns (four per lane) per round
        const int c0 = 128 * r;
        if (c0 > amax) break;
        if (Ghl) {
          float2 g[4][4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int a = a0 + u * NW;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int c = c0 + lane + 32 * q;
              g[u][q] = (a < k && c <= a) ? Ghl[(int64_t)a * k + c] : make_float2(0.f, 0.f);
            }
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = c0 + lane + 32 * q;
            const float xv = c < k ? xs[c] : 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              sum[u] = fmaf(g[u][q].y, xv, fmaf(g[u][q].x, xv, sum[u]));
              const float xo = (c < a0 + u * NW) ? xa[u] : 0.f;   // off-diagonal entries only
              colacc[4 * r + q] = fmaf(g[u][q].y, xo, fmaf(g[u][q].x, xo, colacc[4 * r + q]));
            }
          }
        } else {
          float g[4][4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int a = a0 + u * NW;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int c = c0 + lane + 32 * q;
              g[u][q] = (a < k && c <= a) ? Gres[(int64_t)a * ldg + c] : 0.f;
            }
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int c = c0 + lane + 32 * q;
            const float xv = c < k ? xs[c] : 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              sum[u] = fmaf(g[u][q], xv, sum[u]);
              const float xo = (c < a0 + u * NW) ? xa[u] : 0.f;
              colacc[4 * r + q] = fmaf(g[u][q], xo, colacc[4 * r + q]);
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum[u] += __shfl_xor_sync(0xffffffffu, sum[u], o);
        const int a = a0 + u * NW;
        if (lane == 0 && a < kp) v[a] = sum[u];
      }
    }
    for (int w = 0; w < NW; ++w) {
      if (warp == w) {
#pragma unroll
        for (int j = 0; j < 4 * kResRounds; ++j) {
          const int c = 32 * j + lane;
          if (c < k) ycol[c] += colacc[j];
        }
      }
      __syncthreads();
    }
    for (int a = tid; a < kp; a += NT)
      v[a] = a < k ? rh[a] - fmaf(dg[a], xs[a], v[a] + ycol[a]) : 0.f;
    __syncthreads();
    block_fwd<NT>(S, linv, mo, v, Q, tid, lane, warp);
    block_bwd<NT>(S, linv, mo, v, Q, tid, lane, warp);
    for (int a = tid; a < kp; a += NT) {
      xs[a] += v[a];
      ycol[a] = 0.f;
    }
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

// Launches for k <= kGsMaxK reserve a copy of G (k x gram_ld(k) floats) after the vectors.
constexpr int kGsMaxK = 128;

size_t chol_smem_bytes(int kmax, bool g_copy = true) {
  const int Q = (kmax + 7) / 8, kp = 8 * Q;
  const int64_t gs = (g_copy && kmax <= kGsMaxK) ? (int64_t)kmax * gram_ld(kmax) : 0;
  return (size_t)(factor_floats(Q) + 8 * kp + 4 * kp + gs) * sizeof(float);
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
  if ((e = set_limit<256>()) != cudaSuccess) return e;
  if ((e = set_limit<320>()) != cudaSuccess) return e;
  return adjoint_tc_set_smem();
}

cudaError_t launch_solve(const BatchDev& b, const SolveGroup& g, const int2* systems, int mode, const float* rhs_flat,
                         float* out_flat, float* saved, int32_t* status, float* ws, cudaStream_t st) {
  if (g.count <= 0) return cudaSuccess;
  // one thread per row: the substitutions, the TRSM and the (a) update assume NT >= kp
  const int nt = (g.threads == 64 || g.threads == 128 || g.threads == 256) ? g.threads : 320;
  if (8 * ((g.kmax + 7) / 8) > nt) return cudaErrorInvalidValue;
  const bool g_copy = g.no_g_copy == 0 && g.kmax <= kGsMaxK;
  const size_t smem = chol_smem_bytes(g.kmax, g_copy);
  const int gs = g_copy ? 1 : 0;
  switch (g.threads) {
    case 64:
      chol_solve_kernel<64><<<g.count, 64, smem, st>>>(b, systems, g.first, g.count, mode, rhs_flat, out_flat, saved,
                                                       status, ws, gs);
      break;
    case 128:
      chol_solve_kernel<128><<<g.count, 128, smem, st>>>(b, systems, g.first, g.count, mode, rhs_flat, out_flat,
                                                         saved, status, ws, gs);
      break;
    case 256:
      chol_solve_kernel<256><<<g.count, 256, smem, st>>>(b, systems, g.first, g.count, mode, rhs_flat, out_flat,
                                                         saved, status, ws, gs);
      break;
    default:
      chol_solve_kernel<320><<<g.count, 320, smem, st>>>(b, systems, g.first, g.count, mode, rhs_flat, out_flat,
                                                         saved, status, ws, gs);
      break;
  }
  return cudaGetLastError();
}

}  // namespace fmap
