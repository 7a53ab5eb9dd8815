// Adjoint GEMMs of the row-wise solve on the tensor cores (the adjoint of Eq. 5; Gamma
// from the adjoint row solves, C the map, both k_Y x k_X), per pair, as one GEMM each:
//   kind 2: W    = Gamma^T C + C^T Gamma = [Gamma^T | C^T] [C ; Gamma]      (k_X x k_X, w_off)
//   kind 1: dA_y = Gamma A_x                                                 (k_Y x d, sy_off)
//   kind 0: dA_x = Gamma^T A_y - W A_x = [Gamma^T | -W] [A_y ; A_x]         (k_X x d, sx_off)
// M = the output's rows in tiles of 128, N = its columns in tiles of NT (64, 128 or 256),
// K = the reduction (2 k_Y, k_X or k_Y + k_X) in blocks of 32. Kinds 2 and 1 share the first
// launch, kind 0 (which reads W) is the second; each launch walks a host-built list of
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
#include "fmap_internal.cuh"
#include "tc_ptx.cuh"

namespace fmap {
namespace {

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
template <int STAGES, int NT>
__global__ void __launch_bounds__(kAdjThreads) adjoint_tc_kernel(BatchDev b, const AdjItem* items,
                                                                 const float* a_flat, const float* c_flat,
                                                                 float* ws) {
  using T = AdjTile<NT>;
  extern __shared__ uint8_t smem_raw[];
  const AdjItem it = items[blockIdx.x];
  const PairDev pd = b.pairs[it.pair];
  const int kind = it.kind;
  const int k = pd.k, ky = b.shapes[pd.y].k, d = pd.d;
  const int rows = kind == 1 ? ky : k;                         // output rows
  const int ncols = kind == 2 ? k : d;                         // output columns (and B rows)
  const int kred = kind == 0 ? ky + k : (kind == 1 ? k : 2 * ky);
  const int r0 = it.r0, f0 = it.f0;
  const int nn = min(NT, ncols - f0), npad = (nn + 15) & ~15;
  const int nkb = (kred + 31) / 32;

  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* empty = reinterpret_cast<uint64_t*>(smem + STAGES * T::kStage);   // a stage's MMAs completed
  uint64_t* acc = empty + STAGES;                                             // every MMA completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
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
  // B operand: b1 rows of sb1 then b2 rows of sb2, row stride ldb, columns f < ncols.
  const float* __restrict__ sb1 = kind == 0 ? a_flat + b.shapes[pd.y].a_off : (kind == 1 ? ax : cm);
  const float* __restrict__ sb2 = kind == 0 ? ax : gam;
  const int b1 = kind == 1 ? k : ky, b2 = kind == 0 ? k : (kind == 1 ? 0 : ky);
  const int ldb = ncols;
  const uint32_t idesc = tc::idesc_tf32(kAdjRows, (uint32_t)npad);
  const uint32_t sbase = tc::smem_u32(smem);

  // A operand, kinds 0 and 2: thread tid owns row tid % 128 and the 16 K indices
  // 16 * (tid / 128) + j (a warp's loads of one j are 32 consecutive floats of a column).
  // Kind 1 (Gamma, read along rows): lane = K index, warp + 8 u = row.
  // B operand: thread tid owns column tid % NT and kPerB consecutive K indices.
  const int ra = tid & (kAdjRows - 1), kq = 16 * (tid >> 7);
  const int fr = tid % NT, kqb = (tid / NT) * T::kPerB, f = f0 + fr;
  const bool b_row = fr < npad, b_in = f < ncols;
  float xa[16], xb[T::kPerB];
  auto fetch = [&](int kb) {
    if (kind != 1) {
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
        xa[u] = (a < ky && m < k) ? gam[(int64_t)a * k + m] : 0.f;
      }
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
    if (kind != 1) {
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
    if (b_row) {
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
  if (ok) {
    // lanes of quadrant warp % 4 are output rows; warps w and w + 4 take column halves
    const int q = warp & 3, h = warp >> 2;
    const int row = r0 + 32 * q + lane;
    float* out = ws + (kind == 0 ? pd.sx_off : (kind == 1 ? pd.sy_off : pd.w_off));
    const bool vec = (ncols & 3) == 0;   // 16-byte aligned rows (every offset is)
    for (int c0 = (NT / 2) * h; c0 < npad && c0 < (NT / 2) * (h + 1); c0 += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
      if (row < rows) {
        float* o = out + (int64_t)row * ncols + f0 + c0;
        if (vec && f0 + c0 + 16 <= ncols) {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            reinterpret_cast<float4*>(o)[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (f0 + c0 + j < ncols) o[j] = v[j];
        }
      }
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
constexpr size_t adj_smem() { return 1024 + (size_t)STAGES * AdjTile<NT>::kStage + 64; }

template <int STAGES, int NT>
cudaError_t set_smem_one() {
  return cudaFuncSetAttribute(adjoint_tc_kernel<STAGES, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)adj_smem<STAGES, NT>());
}

template <int STAGES, int NT>
void launch_one(const BatchDev& b, const AdjItem* items, int n, const float* a, const float* c, float* ws,
                cudaStream_t st) {
  if (n > 0) adjoint_tc_kernel<STAGES, NT><<<n, kAdjThreads, adj_smem<STAGES, NT>(), st>>>(b, items, a, c, ws);
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
  return set_smem_one<2, 256>();
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

}  // namespace fmap
