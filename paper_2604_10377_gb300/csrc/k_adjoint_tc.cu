// Adjoint GEMMs of the row-wise solve on the tensor cores (the adjoint of Eq. 5; Gamma
// from the adjoint row solves, C the map, both k_Y x k_X), per pair, as one GEMM each:
//   kind 2: W    = Gamma^T C + C^T Gamma = [Gamma^T | C^T] [C ; Gamma]      (k_X x k_X, w_off)
//   kind 1: dA_y = Gamma A_x                                                 (k_Y x d, sy_off)
//   kind 0: dA_x = Gamma^T A_y - W A_x = [Gamma^T | -W] [A_y ; A_x]         (k_X x d, sx_off)
// and the training loss L = ||C C^T - I||^2 + ||C - C_gt||^2 of the same pairs:
//   kind 3: E    = C C^T - I                                            (k_Y x k_Y, e_off)
//   kind 4: dL/dC = 4 E C + 2 (C - C_gt)                                (k_Y x k_X, into d_c)
// M = the output's rows in tiles of 128, N = its columns in tiles of NT (64, 128 or 256),
// K = the reduction (2 k_Y, k_X, k_Y + k_X or k_Y) in blocks of 32. Kinds 2 and 1 share the
// first launch, kind 0 (which reads W) is the second; the loss takes kind 3, then kind 4
// (which reads E), whose tiles also leave their part of ||E||^2 and ||C - C_gt||^2, summed
// per pair in a fixed order by a third launch. Each launch walks a host-built list of
// (pair, kind, row tile, column tile) items, longest reduction first.
//
// tcgen05.mma kind::tf32 in three passes on TF32 head / remainder splits (x = h + l with
// h = tf32(x), l = x - h exact): h_A h_B + l_A h_B + h_A l_B accumulated in FP32 in TMEM,
// the accuracy class of an FP32 accumulation (each product ~2^-21 relative). Every thread
// of the CTA loads its share of the next K-block into registers while the MMAs of the
// current one run, then writes it as K-major, 128-byte-swizzled head and remainder tiles
// (16-byte stores, conflict-free under the swizzle); thread 0 issues the MMAs and commits
// each shared-memory stage to its barrier. All waits are bounded; a wait that gives up sets
// the workspace's control word to FMAP_ERR_TIMEOUT.
#include "adjoint_tc.cuh"
#include "fmap_internal.cuh"
#include "tc_ptx.cuh"

namespace fmap {
namespace {

// Operands and outputs of the training-loss kinds (3, 4); unused by the adjoint kinds.
struct LossArgs {
  const float* c_gt;   // flat C_gt (c offsets)
  float* d_c;          // flat dL/dC
  float* partial;      // per pair kMaxLossTiles partial sums of the loss, one per output tile
};

constexpr int kAdjThreads = 256;
constexpr int kAdjRows = 128;                              // MMA M
constexpr uint32_t kAdjATile = kAdjRows * 128;             // 128 rows x 32 K of FP32

template <int NT>
struct AdjTile {
  static constexpr uint32_t kBTile = NT * 128;                          // NT feature rows x 32 K
  static constexpr uint32_t kStage = 2 * kAdjATile + 2 * kBTile;        // heads and remainders
  static constexpr int kPerB = NT * 32 / kAdjThreads;                   // B values per thread and block
};

// byte offset of the 16-byte chunk (row r, K indices 4c..4c+3) in a K-major tile of 128-byte
// rows with the 128-byte swizzle (the tile base is 1024-byte aligned)
__device__ __forceinline__ uint32_t swz_chunk(int r, int c) {
  return (uint32_t)r * 128u + ((uint32_t)((c ^ (r & 7)) << 4));
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, float a, float b, float c, float d) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}

__device__ __forceinline__ void st_shared_f32(uint32_t addr, float a) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(addr), "f"(a) : "memory");
}

// four consecutive K values of one row, as TF32 heads into one tile and remainders into the other
__device__ __forceinline__ void put_split4(uint32_t head, uint32_t rem, uint32_t off, const float* x) {
  float h[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) h[j] = tc::tf32_rna(x[j]);
  st_shared_v4(head + off, h[0], h[1], h[2], h[3]);
  st_shared_v4(rem + off, x[0] - h[0], x[1] - h[1], x[2] - h[2], x[3] - h[3]);
}

// NT output columns per CTA (64, 128 or 256: the MMA's N). STAGES shared-memory stages: with
// one, a CTA's conversion of block kb + 1 waits for the MMAs of kb and the other CTAs on the
// SM fill the gap; with two, a CTA converts block kb + 1 while the MMAs of kb run.
// LOSS: the instantiation of the loss kinds (3, 4); the adjoint's (0, 1, 2) leave it false.
// The launch bound asks for the CTAs per SM that the shared memory allows (one stage:
// 4 / 3 / 2 at 64 / 128 / 256 columns; two stages: 2 / 1 / 1).
template <int STAGES, int NT, bool LOSS>
__global__ void __launch_bounds__(kAdjThreads, STAGES == 1 ? (NT == 256 ? 2 : (NT == 128 ? 3 : 4)) : (NT == 64 ? 2 : 1))
    adjoint_tc_kernel(BatchDev b, const AdjItem* items,
                                                                 const float* a_flat, const float* c_flat,
                                                                 float* ws, LossArgs la) {
  using T = AdjTile<NT>;
  extern __shared__ uint8_t smem_raw[];
  const AdjItem it = items[blockIdx.x];
  const PairDev pd = b.pairs[it.pair];
  const int kind = it.kind;
  const int k = pd.k, ky = b.shapes[pd.y].k, d = pd.d;
  // output rows, output columns (and B rows), reduction length
  const int rows = (kind == 0 || kind == 2) ? k : ky;
  const int ncols = kind == 2 ? k : (kind == 3 ? ky : (kind == 4 ? k : d));
  const int kred = kind == 0 ? ky + k : (kind == 2 ? 2 * ky : (kind == 4 ? ky : k));
  const int r0 = it.r0, f0 = it.f0;
  const int nn = min(NT, ncols - f0), npad = (nn + 15) & ~15;
  const int nkb = (kred + 31) / 32;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* empty = reinterpret_cast<uint64_t*>(smem + STAGES * T::kStage);   // a stage's MMAs completed
  uint64_t* acc = empty + STAGES;                                             // every MMA completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* red = reinterpret_cast<float*>(tmem_slot + 2);                       // [8] loss partials
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) tc::mbar_init(&empty[s], 1);
    tc::mbar_init(acc, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, NT);
    tc::tmem_relinquish();
    tc::tc_fence_before();
  }
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const float* __restrict__ gam = ws + pd.gam_off;
  const float* __restrict__ cm = c_flat + pd.c_off;
  const float* __restrict__ ax = a_flat + b.shapes[pd.x].a_off;
  // A operand, kinds 0 and 2: [Gamma^T | S^T] read down columns (S = -W, read as -W^T since
  // W = Gamma^T C + C^T Gamma is symmetric, or S = C), a1 rows of Gamma then a2 rows of S.
  const float* __restrict__ sa2 = kind == 0 ? ws + pd.w_off : cm;
  const int a2 = kind == 0 ? k : ky;
  const float sgn2 = kind == 0 ? -1.f : 1.f;
  // A operand, kinds 1, 3, 4, read along rows a < k_Y: Gamma, C or E (row stride lda)
  const float* __restrict__ sar = kind == 1 ? gam : (kind == 3 ? cm : ws + pd.e_off);
  const int lda = kind == 4 ? ky : k;
  // B operand: b1 rows of sb1 then b2 rows of sb2, row stride ldb, columns f < ncols; kind 3
  // reads it along rows instead (B[j][m] = C[j][m])
  const float* __restrict__ sb1 = kind == 0 ? a_flat + b.shapes[pd.y].a_off : (kind == 1 ? ax : cm);
  const float* __restrict__ sb2 = kind == 0 ? ax : gam;
  const int b1 = kind == 1 ? k : ky, b2 = kind == 0 ? k : ((kind == 1 || kind == 4) ? 0 : ky);
  const int ldb = ncols;
  const uint32_t idesc = tc::idesc_tf32(kAdjRows, (uint32_t)npad);
  const uint32_t sbase = tc::smem_u32(smem);

  // A operand, kinds 0 and 2: thread tid owns row tid % 128 and the 16 K indices
  // 16 * (tid / 128) + j (a warp's loads of one j are 32 consecutive floats of a column).
  // Kinds 1, 3, 4 (read along rows): lane = K index, warp + 8 u = row.
  // B operand: thread tid owns column tid % NT and kPerB consecutive K indices; kind 3:
  // lane = K index, warp + 8 u = row, like the A operand of kind 1.
  const int ra = tid & (kAdjRows - 1), kq = 16 * (tid >> 7);
  const int fr = tid % NT, kqb = (tid / NT) * T::kPerB, f = f0 + fr;
  const bool b_row = fr < npad, b_in = f < ncols;
  float xa[16], xb[T::kPerB];
  auto fetch = [&](int kb) {
    if (!LOSS && (kind == 0 || kind == 2)) {
      const int a = r0 + ra;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int m = 32 * kb + kq + j;
        float x = 0.f;
        if (a < k) {
          if (m < ky) x = gam[(int64_t)m * k + a];
          else if (m < ky + a2) x = sgn2 * sa2[(int64_t)(m - ky) * k + a];
        }
        xa[j] = x;
      }
    } else {
      const int m = 32 * kb + lane;
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int a = r0 + warp + 8 * u;
        xa[u] = (a < ky && m < kred) ? sar[(int64_t)a * lda + m] : 0.f;
      }
    }
    if (LOSS && kind == 3) {
      const int m = 32 * kb + lane;
#pragma unroll
      for (int u = 0; u < T::kPerB; ++u) {
        const int jr = f0 + warp + 8 * u;
        xb[u] = (jr < ky && m < k) ? cm[(int64_t)jr * k + m] : 0.f;
      }
      return;
    }
#pragma unroll
    for (int j = 0; j < T::kPerB; ++j) {
      const int m = 32 * kb + kqb + j;
      float x = 0.f;
      if (b_in) {
        if (m < b1) x = sb1[(int64_t)m * ldb + f];
        else if (m < b1 + b2) x = sb2[(int64_t)(m - b1) * ldb + f];
      }
      xb[j] = x;
    }
  };

  fetch(0);
  for (int kb = 0; kb < nkb; ++kb) {
    const int s = kb % STAGES;
    const uint32_t ah = sbase + (uint32_t)s * T::kStage, al = ah + kAdjATile, bh = al + kAdjATile,
                   bl = bh + T::kBTile;
    // the stage's previous MMAs (block kb - STAGES) have read it
    if (kb >= STAGES) tc::mbar_wait(&empty[s], (uint32_t)(((kb - STAGES) / STAGES) & 1), abort_flag);
    if (!LOSS && (kind == 0 || kind == 2)) {
#pragma unroll
      for (int c = 0; c < 4; ++c) put_split4(ah, al, swz_chunk(ra, (kq >> 2) + c), xa + 4 * c);
    } else {
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        // one row's 32 K values per warp: 32 distinct banks
        const uint32_t off = swz_chunk(warp + 8 * u, lane >> 2) + (uint32_t)((lane & 3) << 2);
        const float h = tc::tf32_rna(xa[u]);
        st_shared_f32(ah + off, h);
        st_shared_f32(al + off, xa[u] - h);
      }
    }
    if (LOSS && kind == 3) {
#pragma unroll
      for (int u = 0; u < T::kPerB; ++u) {
        const uint32_t off = swz_chunk(warp + 8 * u, lane >> 2) + (uint32_t)((lane & 3) << 2);
        const float h = tc::tf32_rna(xb[u]);
        st_shared_f32(bh + off, h);
        st_shared_f32(bl + off, xb[u] - h);
      }
    } else if (b_row) {
#pragma unroll
      for (int c = 0; c < T::kPerB / 4; ++c) put_split4(bh, bl, swz_chunk(fr, (kqb >> 2) + c), xb + 4 * c);
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    if (kb + 1 < nkb) fetch(kb + 1);   // in flight during the MMAs below
    if (tid == 0 && !*abort_flag) {
      tc::tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint64_t adh = tc::smem_desc(ah + ks * 32, 16, 1024, tc::kLayoutSW128);
        const uint64_t adl = tc::smem_desc(al + ks * 32, 16, 1024, tc::kLayoutSW128);
        const uint64_t bdh = tc::smem_desc(bh + ks * 32, 16, 1024, tc::kLayoutSW128);
        const uint64_t bdl = tc::smem_desc(bl + ks * 32, 16, 1024, tc::kLayoutSW128);
        tc::mma_tf32(tmem, adh, bdh, idesc, (kb | ks) != 0 ? 1u : 0u);
        tc::mma_tf32(tmem, adl, bdh, idesc, 1u);
        tc::mma_tf32(tmem, adh, bdl, idesc, 1u);
      }
      tc::mma_commit(&empty[s]);
    }
  }
  if (tid == 0 && !*abort_flag) tc::mma_commit(acc);
  __syncthreads();   // the final commit is issued before anyone waits on it
  bool ok = !*abort_flag && tc::mbar_wait(acc, 0, abort_flag);
  ok = __all_sync(0xffffffffu, ok);   // the TMEM loads below are warp-collective
  tc::tc_fence_after();
  float part = 0.f;   // kinds 3, 4: this thread's share of the tile's loss terms
  if (ok) {
    // lanes of quadrant warp % 4 are output rows; warps w and w + 4 take column halves
    const int q = warp & 3, h = warp >> 2;
    const int row = r0 + 32 * q + lane;
    float* out = LOSS ? (kind == 3 ? ws + pd.e_off : la.d_c + pd.c_off)
                      : ws + (kind == 0 ? pd.sx_off : (kind == 1 ? pd.sy_off : pd.w_off));
    const float* gt = LOSS ? la.c_gt + pd.c_off : nullptr;
    // 16-byte stores where every row starts on a 16-byte boundary (the workspace offsets are
    // aligned; dL/dC sits at the pair's c offset, which need not be)
    const bool vec = (ncols & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0;
    for (int c0 = (NT / 2) * h; c0 < npad && c0 < (NT / 2) * (h + 1); c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
      if (row < rows) {
        const int col0 = f0 + c0;
        if (LOSS && kind == 3) {
          // E = C C^T - I, and ||E||^2
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            v[j] -= (col0 + j == row) ? 1.f : 0.f;
            if (col0 + j < ncols) part = fmaf(v[j], v[j], part);
          }
        } else if (LOSS) {
          // dL/dC = 4 E C + 2 (C - C_gt), and ||C - C_gt||^2
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            if (col0 + j < ncols) {
              const float r = cm[(int64_t)row * k + col0 + j] - gt[(int64_t)row * k + col0 + j];
              part = fmaf(r, r, part);
              v[j] = fmaf(4.f, v[j], 2.f * r);
            }
          }
        }
        float* o = out + (int64_t)row * ncols + col0;
        if (vec && col0 + 16 <= ncols) {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            reinterpret_cast<float4*>(o)[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (col0 + j < ncols) o[j] = v[j];
        }
      }
    }
  }
  if (LOSS) {
    // the tile's loss partial: warp sums, then the eight warps in order (reproducible)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    if (tid == 0) {
      float t = 0.f;
      for (int w = 0; w < kAdjThreads / 32; ++w) t += red[w];
      const int nrt = (ky + kAdjRows - 1) / kAdjRows;
      const int ne = nrt * ((ky + NT - 1) / NT);                 // E tiles of the pair
      const int slot = kind == 3 ? (r0 / kAdjRows) * ((ky + NT - 1) / NT) + f0 / NT
                                 : ne + (r0 / kAdjRows) * ((k + NT - 1) / NT) + f0 / NT;
      la.partial[(int64_t)it.pair * kMaxLossTiles + slot] = t;
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (*abort_flag) {
    // MMAs that never signalled: a bounded time for them, then report
    if (tid == 0) {
      const uint64_t t0 = tc::globaltimer();
      while (tc::globaltimer() - t0 < 2000000ull) {}
      atomicExch(reinterpret_cast<int*>(ws), (int)FMAP_ERR_TIMEOUT);
    }
    __syncthreads();
  }
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, NT);
  }
}

template <int STAGES, int NT>
constexpr size_t adj_smem() { return 1024 + (size_t)STAGES * AdjTile<NT>::kStage + 128; }

template <int STAGES, int NT, bool LOSS = false>
cudaError_t set_smem_one() {
  return cudaFuncSetAttribute(adjoint_tc_kernel<STAGES, NT, LOSS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)adj_smem<STAGES, NT>());
}

template <int STAGES, int NT, bool LOSS = false>
void launch_one(const BatchDev& b, const AdjItem* items, int n, const float* a, const float* c, float* ws,
                cudaStream_t st, LossArgs la = LossArgs{}) {
  if (n > 0)
    adjoint_tc_kernel<STAGES, NT, LOSS><<<n, kAdjThreads, adj_smem<STAGES, NT>(), st>>>(b, items, a, c, ws, la);
}

// loss[p] = the pair's tile partials of ||E||^2 (kind 3 tiles), then of ||C - C_gt||^2
// (kind 4 tiles), added in slot order
__global__ void loss_tc_sum_kernel(BatchDev b, const float* partial, float* loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= b.n_pairs) return;
  const PairDev pd = b.pairs[p];
  const int k = pd.k, ky = b.shapes[pd.y].k;
  const int nrt = (ky + kAdjRows - 1) / kAdjRows;
  const int n = nrt * ((ky + kLossNt - 1) / kLossNt) + nrt * ((k + kLossNt - 1) / kLossNt);
  float t = 0.f;
  for (int s = 0; s < n; ++s) t += partial[(int64_t)p * kMaxLossTiles + s];
  loss[p] = t;
}

template <int STAGES>
void launch_nt(int nt, const BatchDev& b, const AdjItem* items, int n, const float* a, const float* c, float* ws,
               cudaStream_t st) {
  if (nt == 64) launch_one<STAGES, 64>(b, items, n, a, c, ws, st);
  else if (nt == 128) launch_one<STAGES, 128>(b, items, n, a, c, ws, st);
  else launch_one<STAGES, 256>(b, items, n, a, c, ws, st);
}

}  // namespace

cudaError_t adjoint_tc_set_smem() {
  cudaError_t e;
  if ((e = set_smem_one<1, 64>()) != cudaSuccess) return e;
  if ((e = set_smem_one<1, 128>()) != cudaSuccess) return e;
  if ((e = set_smem_one<1, 256>()) != cudaSuccess) return e;
  if ((e = set_smem_one<2, 64>()) != cudaSuccess) return e;
  if ((e = set_smem_one<2, 128>()) != cudaSuccess) return e;
  if ((e = set_smem_one<2, 256>()) != cudaSuccess) return e;
  return set_smem_one<1, kLossNt, true>();
}

void adjoint_tc_plan(const std::vector<int3>& shapes, int sms, AdjTcPlan& P) {
  // shapes[p] = (k_X, k_Y, d) of pair p
  auto build = [&](int nt) {
    P.items.clear();
    std::vector<std::pair<int, AdjItem>> first, second;   // (K-blocks, item)
    for (int p = 0; p < (int)shapes.size(); ++p) {
      const int k = shapes[p].x, ky = shapes[p].y, d = shapes[p].z;
      const int rows[3] = {k, ky, k}, cols[3] = {d, d, k}, kred[3] = {ky + k, k, 2 * ky};
      for (int kind = 0; kind < 3; ++kind)
        for (int r0 = 0; r0 < rows[kind]; r0 += kAdjRows)
          for (int f0 = 0; f0 < cols[kind]; f0 += nt)
            (kind == 0 ? second : first).push_back({(kred[kind] + 31) / 32, AdjItem{p, kind, r0, f0}});
    }
    auto longest_first = [](const std::pair<int, AdjItem>& u, const std::pair<int, AdjItem>& v) {
      return u.first > v.first;
    };
    std::stable_sort(first.begin(), first.end(), longest_first);
    std::stable_sort(second.begin(), second.end(), longest_first);
    for (const auto& x : first) P.items.push_back(x.second);
    for (const auto& x : second) P.items.push_back(x.second);
    P.n_first = (int)first.size();
    return (int)second.size();
  };
  // enough dA_x tiles of 128 columns for two per SM: the tensor cores pay (below that the two
  // dependent launches are bound by one CTA's reduction loop and the FP32 FMA tiles are faster)
  P.fills_sms = build(128) >= 2 * sms;
  if (P.features == 0) P.features = P.fills_sms ? 128 : 64;
  build(P.features);
  // one stage: twice the CTAs per SM of two stages, which measured faster at every width
  if (P.stages == 0) P.stages = 1;
}

cudaError_t launch_adjoint_tc(const BatchDev& b, const AdjItem* items, const AdjTcPlan& P, const float* a,
                              const float* c, float* ws, cudaStream_t st) {
  if (P.items.empty()) return cudaSuccess;
  if (P.stages != 1 && P.stages != 2) return cudaErrorInvalidValue;
  if (P.features != 64 && P.features != 128 && P.features != 256) return cudaErrorInvalidValue;
  const int n_total = (int)P.items.size(), n2 = n_total - P.n_first;
  // W and dA_y, then dA_x (which reads W)
  if (P.stages == 1) launch_nt<1>(P.features, b, items, P.n_first, a, c, ws, st);
  else launch_nt<2>(P.features, b, items, P.n_first, a, c, ws, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (P.stages == 1) launch_nt<1>(P.features, b, items + P.n_first, n2, a, c, ws, st);
  else launch_nt<2>(P.features, b, items + P.n_first, n2, a, c, ws, st);
  return cudaGetLastError();
}

void adjoint_tc_loss_plan(const std::vector<int3>& shapes, AdjTcPlan& P) {
  // kind 3 tiles, then kind 4 tiles, each longest reduction first; 128 columns per CTA
  std::vector<std::pair<int, AdjItem>> e_items, g_items;
  for (int p = 0; p < (int)shapes.size(); ++p) {
    const int k = shapes[p].x, ky = shapes[p].y;
    for (int r0 = 0; r0 < ky; r0 += kAdjRows) {
      for (int f0 = 0; f0 < ky; f0 += kLossNt) e_items.push_back({(k + 31) / 32, AdjItem{p, 3, r0, f0}});
      for (int f0 = 0; f0 < k; f0 += kLossNt) g_items.push_back({(ky + 31) / 32, AdjItem{p, 4, r0, f0}});
    }
  }
  auto longest_first = [](const std::pair<int, AdjItem>& u, const std::pair<int, AdjItem>& v) {
    return u.first > v.first;
  };
  std::stable_sort(e_items.begin(), e_items.end(), longest_first);
  std::stable_sort(g_items.begin(), g_items.end(), longest_first);
  P.items.clear();
  for (const auto& x : e_items) P.items.push_back(x.second);
  for (const auto& x : g_items) P.items.push_back(x.second);
  P.n_first = (int)e_items.size();
  P.features = kLossNt;
  P.stages = 1;
}

cudaError_t launch_loss_tc(const BatchDev& b, const AdjItem* items, const AdjTcPlan& P, const float* c,
                           const float* c_gt, float* loss, float* d_c, float* ws, float* partial, cudaStream_t st) {
  if (P.items.empty()) return cudaSuccess;
  const LossArgs la{c_gt, d_c, partial};
  const int n2 = (int)P.items.size() - P.n_first;
  // E, then dL/dC (which reads E), then the loss sums
  launch_one<1, kLossNt, true>(b, items, P.n_first, nullptr, c, ws, st, la);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  launch_one<1, kLossNt, true>(b, items + P.n_first, n2, nullptr, c, ws, st, la);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (loss) {
    loss_tc_sum_kernel<<<(b.n_pairs + 127) / 128, 128, 0, st>>>(b, partial, loss);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace fmap
