// Spectral projection on the 5th-generation tensor cores (Eq. 1), BF16 features.
//
//   A_s^T (d x k) = F_s^T (d x n) . P_s (n x k),   P_s = diag(M_s) Phi_s
//
// One persistent CTA per SM walks its own contiguous range of the batch's
// (shape, feature group) vertex sequence (stream-K split into equal-cost
// ranges); a range is cut into segments at shape / group boundaries and every
// segment writes one partial A. Per 64-vertex stage:
//   warp 0      TMA-loads the F tile (MN-major, 128-byte swizzle), the Phi tile
//               (FP32, 32-column boxes, 128-byte swizzle) and the 64 masses;
//   warps 2-9   read Phi and M from shared memory, form P = M * Phi in FP32 and
//               split it into BF16 hi + lo (P = hi + lo to ~2^-17), written in place
//               over the Phi tile as K-major 128-byte-swizzled B tiles: the mass is
//               fused into the operand load;
//   warp 1      issues tcgen05.mma (M = 128 features, N = k rounded up to 16,
//               K = 16 vertices) for hi and lo into FP32 accumulators in TMEM.
// At the end of a segment warps 2-9 read the accumulators back (tcgen05.ld) and
// write the segment's partial A; a second kernel adds the partials of each shape
// in a fixed order. F is exact in BF16, so A carries only the ~2^-17 error of
// the hi/lo split and FP32 accumulation.
//
// Every mbarrier wait is bounded (tc::kWaitTimeoutNs); a wait that gives up
// raises a CTA-wide abort flag, every role stops, TMEM is freed, and the
// workspace error word is set to FMAP_ERR_TIMEOUT (reported per pair by the solve).
#include "fmap_internal.cuh"
#include "tc_ptx.cuh"

namespace fmap {
namespace {

constexpr int kConvWarps = 8;
constexpr int kThreads = 32 * (2 + kConvWarps);
constexpr int kStageV = 64;            // vertices per pipeline stage (= one 128-byte K row of bf16)
constexpr uint32_t kBoxBytes = 64 * 64 * 2;   // one TMA box: 64 vertices x 64 features bf16
constexpr uint32_t kPhiBoxBytes = 64 * 128;    // one TMA box: 64 vertices x 32 basis functions fp32

// (a, b) -> BF16 heads RN(a), RN(b) and remainders RN(a - head), RN(b - head), each pair
// packed low = a, high = b (one packed conversion per pair).
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

__global__ void __launch_bounds__(kThreads, 1) project_tc_kernel(TcProjParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = P.stages;
  uint8_t* sF = smem;
  uint8_t* sP = sF + (size_t)S * P.f_stage_bytes;       // Phi tile, converted in place into P hi / lo
  float* sM = reinterpret_cast<float*>(sP + (size_t)S * P.p_stage_bytes);   // 64 masses per stage
  uint64_t* bars = reinterpret_cast<uint64_t*>(sM + (size_t)S * kStageV);
  uint64_t* full_f = bars;
  uint64_t* full_p = bars + S;
  uint64_t* empty = bars + 2 * S;
  uint64_t* acc_full = bars + 3 * S;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full_f[s], 1);
      tc::mbar_init(&full_p[s], kConvWarps);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(acc_full, 1);
    tc::mbar_init(acc_empty, kConvWarps);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tmem_slot, P.tmem_cols);
    tc::tmem_relinquish();
    tc::tc_fence_before();
  }
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      uint32_t stage = 0, phase = 0;
      for (int it = P.cta_first[blockIdx.x]; it < P.cta_first[blockIdx.x + 1]; ++it) {
        const TcItem item = P.items[it];
        const CUtensorMap* fmap = P.fmaps + item.shape;
        const CUtensorMap* pmap = P.phimaps + item.shape;
        const CUtensorMap* mmap = P.massmaps + item.shape;
        tc::prefetch_tmap(fmap);
        tc::prefetch_tmap(pmap);
        tc::prefetch_tmap(mmap);
        const int nst = (int)((item.v1 - item.v0 + kStageV - 1) / kStageV);
        const int kb = (item.npad + 31) / 32;
        const uint32_t bytes = (uint32_t)item.fg * 2 * kBoxBytes + (uint32_t)kb * kPhiBoxBytes + kStageV * 4;
        for (int st = 0; st < nst; ++st) {
          if (!tc::mbar_wait(&empty[stage], phase ^ 1, abort_flag)) goto producer_done;
          tc::mbar_arrive_expect_tx(&full_f[stage], bytes);
          uint8_t* dst = sF + (size_t)stage * P.f_stage_bytes;
          uint8_t* pdst = sP + (size_t)stage * P.p_stage_bytes;
          const int y = (int)(item.v0 + (int64_t)st * kStageV);
          for (int m = 0; m < item.fg; ++m)
            for (int h = 0; h < 2; ++h)
              tc::tma_load_2d(dst + (m * 2 + h) * kBoxBytes, fmap, &full_f[stage], item.f0 + m * 128 + h * 64, y);
          for (int b = 0; b < kb; ++b)
            tc::tma_load_2d(pdst + b * kPhiBoxBytes, pmap, &full_f[stage], item.n0 + b * 32, y);
          tc::tma_load_1d(sM + (size_t)stage * kStageV, mmap, &full_f[stage], y);
          if (++stage == (uint32_t)S) { stage = 0; phase ^= 1; }
        }
      }
    producer_done:
      if (*abort_flag) {
        // let copies already in flight land before the CTA's shared memory goes away
        const uint64_t t0 = tc::globaltimer();
        while (tc::globaltimer() - t0 < 2000000ull) {}
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t stage = 0, phase = 0, acc_phase = 0;
      for (int it = P.cta_first[blockIdx.x]; it < P.cta_first[blockIdx.x + 1]; ++it) {
        const TcItem item = P.items[it];
        if (!tc::mbar_wait(acc_empty, acc_phase ^ 1, abort_flag)) break;
        tc::tc_fence_after();
        const uint32_t idesc = tc::idesc_bf16_f32(128, (uint32_t)item.npad, 1, 0);
        const int nst = (int)((item.v1 - item.v0 + kStageV - 1) / kStageV);
        bool ok = true;
        for (int st = 0; st < nst && ok; ++st) {
          ok = tc::mbar_wait(&full_f[stage], phase, abort_flag) && tc::mbar_wait(&full_p[stage], phase, abort_flag);
          if (!ok) break;
          tc::tc_fence_after();
          const uint32_t a_base = tc::smem_u32(sF + (size_t)stage * P.f_stage_bytes);
          const uint32_t ph = tc::smem_u32(sP + (size_t)stage * P.p_stage_bytes);
          const uint32_t pl = ph + (uint32_t)item.npad * 128u;
#pragma unroll
          for (int kk = 0; kk < kStageV / 16; ++kk) {
            const uint64_t bh = tc::smem_desc(ph + kk * 32, 16, 1024, tc::kLayoutSW128);
            const uint64_t bl = tc::smem_desc(pl + kk * 32, 16, 1024, tc::kLayoutSW128);
            for (int m = 0; m < item.fg; ++m) {
              const uint64_t ad = tc::smem_desc(a_base + m * 2 * kBoxBytes + kk * 2048, kBoxBytes, 1024,
                                                tc::kLayoutSW128);
              const uint32_t d = tmem_base + (uint32_t)(m * item.npad);
              tc::mma_bf16(d, ad, bh, idesc, (st | kk) != 0 ? 1u : 0u);
              tc::mma_bf16(d, ad, bl, idesc, 1u);
            }
          }
          tc::mma_commit(&empty[stage]);
          if (++stage == (uint32_t)S) { stage = 0; phase ^= 1; }
        }
        if (!ok) break;
        tc::mma_commit(acc_full);
        acc_phase ^= 1;
      }
    }
  } else {
    // ------------------------------------------------------------ converters + epilogue
    const int cw = warp - 2;
    const int qs = lane & 7, csub = lane >> 3;
    uint32_t stage = 0, phase = 0, acc_phase = 0;
    for (int it = P.cta_first[blockIdx.x]; it < P.cta_first[blockIdx.x + 1]; ++it) {
      const TcItem item = P.items[it];
      const ShapeDev s = P.shapes[item.shape];
      const int k = s.k;
      const int nst = (int)((item.v1 - item.v0 + kStageV - 1) / kStageV);
      const int kb = (item.npad + 31) / 32;
      for (int st = 0; st < nst; ++st) {
        if (!tc::mbar_wait(&full_f[stage], phase, abort_flag)) goto conv_done;
        uint8_t* tile = sP + (size_t)stage * P.p_stage_bytes;
        const float* mst = sM + (size_t)stage * kStageV;
        const int64_t vbase = item.v0 + (int64_t)st * kStageV;
        // read phase: unit (box b, row group c = 4 cg + csub, quad qs) = rows 8c..8c+7 x basis 32b+4qs..+3
        float4 x[2][8];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int wu = cw + kConvWarps * r;
          if (wu < 2 * kb) {
            const int b = wu >> 1, c = 4 * (wu & 1) + csub;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int vl = 8 * c + i;
              x[r][i] = *reinterpret_cast<const float4*>(tile + b * kPhiBoxBytes + vl * 128 + ((qs ^ (vl & 7)) << 4));
            }
          }
        }
        tc::named_barrier_sync(1, 32 * kConvWarps);
        // write phase: P hi at [0, npad*128), lo at [npad*128, 2*npad*128), K-major, 128-byte swizzle
        uint8_t* th = tile;
        uint8_t* tl = tile + (size_t)item.npad * 128;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int wu = cw + kConvWarps * r;
          if (wu < 2 * kb) {
            const int b = wu >> 1, c = 4 * (wu & 1) + csub;
            float mv[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) mv[i] = (vbase + 8 * c + i < item.v1) ? mst[8 * c + i] : 0.f;
            const int n0 = 32 * b + 4 * qs;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int n = n0 + j;
              if (n >= item.npad) continue;
              float pv[8];
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                const float4 q = x[r][i];
                const float xv = j == 0 ? q.x : (j == 1 ? q.y : (j == 2 ? q.z : q.w));
                pv[i] = xv * mv[i];
              }
              uint4 hv, lv;
              split_pair(pv[0], pv[1], hv.x, lv.x);
              split_pair(pv[2], pv[3], hv.y, lv.y);
              split_pair(pv[4], pv[5], hv.z, lv.z);
              split_pair(pv[6], pv[7], hv.w, lv.w);
              const uint32_t off = (uint32_t)n * 128u + ((uint32_t)(c ^ (n & 7)) << 4);
              *reinterpret_cast<uint4*>(th + off) = hv;
              *reinterpret_cast<uint4*>(tl + off) = lv;
            }
          }
        }
        (void)k;
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&full_p[stage]);
        if (++stage == (uint32_t)S) { stage = 0; phase ^= 1; }
      }
      // epilogue: accumulators -> this item's partial A (k x stride, row-major)
      if (!tc::mbar_wait(acc_full, acc_phase, abort_flag)) goto conv_done;
      tc::tc_fence_after();
      {
        const int quarter = warp & 3, half = cw >> 2;
        const int stride = item.fg * 128;
        float* part = P.ws + item.part_off;
        for (int m = 0; m < item.fg; ++m) {
          const int fl = m * 128 + quarter * 32 + lane;
          const bool fok = item.f0 + fl < s.d;
          for (int ch = half; ch < item.npad / 16; ch += 2) {
            float v[16];
            tc::tmem_ld16(tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(m * item.npad + ch * 16), v);
            if (fok) {
#pragma unroll
              for (int t = 0; t < 16; ++t) {
                const int n = ch * 16 + t;
                if (n < item.nk) part[(int64_t)n * stride + fl] = v[t];
              }
            }
          }
        }
      }
      tc::tc_fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(acc_empty);
      acc_phase ^= 1;
    }
  conv_done:;
  }

  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem_base, P.tmem_cols);
  if (threadIdx.x == 0 && *abort_flag) atomicExch(P.err, (int)FMAP_ERR_TIMEOUT);
}

// A_s[n0 + n][f0 + f] = sum over the group's items (in order) of partial[n][f].
__global__ void project_tc_reduce_kernel(const ShapeDev* shapes, const TcItem* items, const TcRedGroup* groups,
                                         float* a_out, const float* ws) {
  const TcRedGroup g = groups[blockIdx.y];
  const ShapeDev s = shapes[g.shape];
  // four consecutive features per thread (dspan, f0, d are multiples of 16 and the
  // partials are 256-byte aligned; float4 stores when the output buffer is 16-byte aligned)
  const int q4 = g.dspan >> 2, total = g.nk * q4;
  const bool vec = (reinterpret_cast<uintptr_t>(a_out) & 15) == 0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int n = e / q4, f = (e - n * q4) * 4;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int i = g.it_beg; i < g.it_end; ++i) {
      const float4 u = *reinterpret_cast<const float4*>(ws + items[i].part_off + (int64_t)n * g.stride + f);
      acc.x += u.x; acc.y += u.y; acc.z += u.z; acc.w += u.w;
    }
    float* o = a_out + s.a_off + (int64_t)(g.n0 + n) * s.d + g.f0 + f;
    if (vec) {
      *reinterpret_cast<float4*>(o) = acc;
    } else {
      o[0] = acc.x; o[1] = acc.y; o[2] = acc.z; o[3] = acc.w;
    }
  }
}

}  // namespace

cudaError_t project_tc_set_smem(int bytes) {
  return cudaFuncSetAttribute(project_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

int project_tc_threads() { return kThreads; }

cudaError_t launch_project_tc(const TcProjParams& p, int grid, int smem_bytes, cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  project_tc_kernel<<<grid, kThreads, smem_bytes, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_project_tc_reduce(const ShapeDev* shapes, const TcItem* items, const TcRedGroup* groups,
                                     int n_groups, int64_t max_elems, float* a_out, const float* ws,
                                     cudaStream_t st) {
  if (n_groups <= 0) return cudaSuccess;
  dim3 grid((unsigned)std::min<int64_t>((max_elems / 4 + 255) / 256, 4096), (unsigned)n_groups);
  project_tc_reduce_kernel<<<grid, 256, 0, st>>>(shapes, items, groups, a_out, ws);
  return cudaGetLastError();
}

}  // namespace fmap
