// Spectral projection on the tensor cores (Eq. 1) for FP32 features, three-pass TF32:
//
//   A_s^T (d x k) = F_s^T (d x n) . P_s (n x k),   P_s = diag(M_s) Phi_s
//
// TF32 keeps 10 explicit mantissa bits of each operand; a single pass would leave
// ~2^-11 relative error per product. Each operand is therefore split into a TF32 head
// (rounded to nearest) and the exact FP32 remainder, P = Ph + Pl and F = Fh + Fl, and
// three products are accumulated in FP32:
//   Ph.Fh + Pl.Fh + Ph.Fl,
// which drops Pl.Fl (~2^-22) and the TF32 truncation of the two correction terms
// (~2^-21 each): the accuracy class of an FP32 accumulation.
//
// Same schedule as the BF16 kernel (one persistent CTA per SM over a stream-K range of
// (shape, feature group) segments, partials reduced in a fixed order by a second
// kernel), with 32-vertex stages and two TMEM accumulators (segments are short, so the
// epilogue of one overlaps the MMAs of the next):
//   warp 0      TMA-loads the F tile (FP32, MN-major: 32-feature boxes, 128-byte
//               swizzle), the Phi tile (FP32, 32-column boxes) and the 32 masses;
//   warps 2-9   form P = M * Phi and write Ph, Pl as K-major 128-byte-swizzled B tiles
//               (the mass is fused into the operand load), and transpose the F tile into
//               K-major A tiles Fh (in place) and Fl (kind::tf32 takes K-major operands
//               only);
//   warp 1      issues tcgen05.mma kind::tf32 (M = 128 features, N = k rounded up to 16,
//               K = 8 vertices), three per K-step, into FP32 accumulators in TMEM.
// Waits are bounded like the BF16 kernel's.
#include "fmap_internal.cuh"
#include "tc_ptx.cuh"

namespace fmap {
namespace {

constexpr int kConvWarps = 8;
constexpr int kThreads = 32 * (2 + kConvWarps);
constexpr int kStageV = 32;                  // vertices per pipeline stage (one 128-byte row of FP32)
constexpr uint32_t kBoxBytes = 32 * 128;     // one TMA box: 32 vertices x 32 FP32 (features or basis)
constexpr uint32_t kGroupBytes = 4 * kBoxBytes;   // 128 features of one stage

constexpr int kMaxFg = 2;   // feature groups of 128 per CTA (the planner caps FP32 units at 2)

__global__ void __launch_bounds__(kThreads, 1) project_tc32_kernel(TcProjParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = P.stages;
  // per stage: [F tile | Fl] (f_stage_bytes = 2 * fg * kGroupBytes), then [Phi | Ph | Pl]
  uint8_t* sF = smem;
  uint8_t* sP = sF + (size_t)S * P.f_stage_bytes;
  float* sM = reinterpret_cast<float*>(sP + (size_t)S * P.p_stage_bytes);   // 32 masses per stage
  uint64_t* bars = reinterpret_cast<uint64_t*>(sM + (size_t)S * kStageV);
  uint64_t* full_f = bars;
  uint64_t* full_p = bars + S;
  uint64_t* empty = bars + 2 * S;
  uint64_t* acc_full = bars + 3 * S;    // [2]: accumulators double-buffered in TMEM
  uint64_t* acc_empty = acc_full + 2;   // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full_f[s], 1);
      tc::mbar_init(&full_p[s], kConvWarps);
      tc::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], kConvWarps);
    }
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
        const uint32_t bytes = (uint32_t)item.fg * kGroupBytes + (uint32_t)kb * kBoxBytes + kStageV * 4;
        for (int st = 0; st < nst; ++st) {
          if (!tc::mbar_wait(&empty[stage], phase ^ 1, abort_flag)) goto producer_done;
          tc::mbar_arrive_expect_tx(&full_f[stage], bytes);
          uint8_t* dst = sF + (size_t)stage * P.f_stage_bytes;
          uint8_t* pdst = sP + (size_t)stage * P.p_stage_bytes;
          const int y = (int)(item.v0 + (int64_t)st * kStageV);
          for (int m = 0; m < item.fg; ++m)
            for (int h = 0; h < 4; ++h)
              tc::tma_load_2d(dst + (m * 4 + h) * kBoxBytes, fmap, &full_f[stage], item.f0 + m * 128 + h * 32, y);
          for (int b = 0; b < kb; ++b)
            tc::tma_load_2d(pdst + b * kBoxBytes, pmap, &full_f[stage], item.n0 + b * 32, y);
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
      uint32_t stage = 0, phase = 0;
      uint32_t acc_phase[2] = {0, 0};
      int buf = 0;
      const uint32_t half_cols = P.tmem_cols / 2;
      for (int it = P.cta_first[blockIdx.x]; it < P.cta_first[blockIdx.x + 1]; ++it) {
        const TcItem item = P.items[it];
        if (!tc::mbar_wait(&acc_empty[buf], acc_phase[buf] ^ 1, abort_flag)) break;
        tc::tc_fence_after();
        const uint32_t idesc = tc::idesc_tf32(128, (uint32_t)item.npad);
        const int nst = (int)((item.v1 - item.v0 + kStageV - 1) / kStageV);
        const int kb = (item.npad + 31) / 32;
        bool ok = true;
        for (int st = 0; st < nst && ok; ++st) {
          ok = tc::mbar_wait(&full_f[stage], phase, abort_flag) && tc::mbar_wait(&full_p[stage], phase, abort_flag);
          if (!ok) break;
          tc::tc_fence_after();
          const uint32_t f_base = tc::smem_u32(sF + (size_t)stage * P.f_stage_bytes);
          const uint32_t fl_base = f_base + (uint32_t)item.fg * kGroupBytes;
          const uint32_t ph = tc::smem_u32(sP + (size_t)stage * P.p_stage_bytes) + (uint32_t)kb * kBoxBytes;
          const uint32_t pl = ph + (uint32_t)item.npad * 128u;
#pragma unroll
          for (int kk = 0; kk < kStageV / 8; ++kk) {
            const uint64_t bh = tc::smem_desc(ph + kk * 32, 16, 1024, tc::kLayoutSW128);
            const uint64_t bl = tc::smem_desc(pl + kk * 32, 16, 1024, tc::kLayoutSW128);
            for (int m = 0; m < item.fg; ++m) {
              const uint64_t af = tc::smem_desc(f_base + m * kGroupBytes + kk * 32, 16, 1024, tc::kLayoutSW128);
              const uint64_t al = tc::smem_desc(fl_base + m * kGroupBytes + kk * 32, 16, 1024, tc::kLayoutSW128);
              const uint32_t d = tmem_base + (uint32_t)buf * half_cols + (uint32_t)(m * item.npad);
              tc::mma_tf32(d, af, bh, idesc, (st | kk) != 0 ? 1u : 0u);
              tc::mma_tf32(d, af, bl, idesc, 1u);
              tc::mma_tf32(d, al, bh, idesc, 1u);
            }
          }
          tc::mma_commit(&empty[stage]);
          if (++stage == (uint32_t)S) { stage = 0; phase ^= 1; }
        }
        if (!ok) break;
        tc::mma_commit(&acc_full[buf]);
        acc_phase[buf] ^= 1;
        buf ^= 1;
      }
    }
  } else {
    // ------------------------------------------------------------ converters + epilogue
    const int ct = threadIdx.x - 64;   // 0 .. 255
    const int cw = warp - 2;
    uint32_t stage = 0, phase = 0;
    uint32_t acc_phase[2] = {0, 0};
    int buf = 0;
    const uint32_t half_cols = P.tmem_cols / 2;
    for (int it = P.cta_first[blockIdx.x]; it < P.cta_first[blockIdx.x + 1]; ++it) {
      const TcItem item = P.items[it];
      const ShapeDev s = P.shapes[item.shape];
      const int nst = (int)((item.v1 - item.v0 + kStageV - 1) / kStageV);
      const int kb = (item.npad + 31) / 32;
      for (int st = 0; st < nst; ++st) {
        if (!tc::mbar_wait(&full_f[stage], phase, abort_flag)) goto conv_done;
        uint8_t* ftile = sF + (size_t)stage * P.f_stage_bytes;
        uint8_t* phi = sP + (size_t)stage * P.p_stage_bytes;
        uint8_t* th = phi + (size_t)kb * kBoxBytes;
        uint8_t* tl = th + (size_t)item.npad * 128;
        const float* mst = sM + (size_t)stage * kStageV;
        const int64_t vbase = item.v0 + (int64_t)st * kStageV;
        // F: read this thread's chunks (feature row f, vertices 4c .. 4c+3) out of the
        // vertex-row TMA boxes, then (after every converter has read) write Fh in place and
        // Fl beside it as K-major 128-byte-swizzled A tiles (row f, 32 vertices). The 32
        // lanes of a warp take 32 consecutive features of one box and one vertex quad, so
        // each read touches 32 distinct banks.
        float fx[kMaxFg * 4][4];
        const int nfc = item.fg * 128 * 8;
#pragma unroll
        for (int r = 0; r < kMaxFg * 4; ++r) {
          const int q = ct + 32 * kConvWarps * r;
          if (q < nfc) {
            const int c = (q >> 5) & 7, box = q >> 8;
            const int ff = q & 31, f = 32 * box + ff;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int v = 4 * c + j;
              fx[r][j] = *reinterpret_cast<const float*>(ftile + box * kBoxBytes + v * 128 +
                                                         ((((ff >> 2) ^ (v & 7)) << 4) | ((ff & 3) << 2)));
            }
          }
        }
        tc::named_barrier_sync(1, 32 * kConvWarps);
#pragma unroll
        for (int r = 0; r < kMaxFg * 4; ++r) {
          const int q = ct + 32 * kConvWarps * r;
          if (q < nfc) {
            const int c = (q >> 5) & 7, f = 32 * (q >> 8) + (q & 31);
            float h[4], l[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              h[j] = tc::tf32_rna(fx[r][j]);
              l[j] = fx[r][j] - h[j];
            }
            const uint32_t off = (uint32_t)f * 128u + ((uint32_t)(c ^ (f & 7)) << 4);
            *reinterpret_cast<float4*>(ftile + off) = make_float4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<float4*>(ftile + (size_t)item.fg * kGroupBytes + off) = make_float4(l[0], l[1], l[2], l[3]);
          }
        }
        // Ph, Pl: 16-byte chunk (row n, vertices 4c .. 4c+3) of the K-major swizzled B tiles;
        // a warp takes 32 consecutive basis functions of one box and one vertex quad
        for (int q = ct; q < kb * 32 * 8; q += 32 * kConvWarps) {
          const int n = 32 * (q >> 8) + (q & 31), c = (q >> 5) & 7;
          if (n >= item.npad) continue;
          float hv[4], lv[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int v = 4 * c + j;
            const int b = n >> 5, nn = n & 31;
            const float ph = *reinterpret_cast<const float*>(phi + b * kBoxBytes + v * 128 +
                                                             ((((nn >> 2) ^ (v & 7)) << 4) | ((nn & 3) << 2)));
            const float p = (vbase + v < item.v1) ? ph * mst[v] : 0.f;
            hv[j] = tc::tf32_rna(p);
            lv[j] = p - hv[j];
          }
          const uint32_t off = (uint32_t)n * 128u + ((uint32_t)(c ^ (n & 7)) << 4);
          *reinterpret_cast<float4*>(th + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
          *reinterpret_cast<float4*>(tl + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
        }
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&full_p[stage]);
        if (++stage == (uint32_t)S) { stage = 0; phase ^= 1; }
      }
      // epilogue: accumulators -> this item's partial A (nk x stride, row-major)
      if (!tc::mbar_wait(&acc_full[buf], acc_phase[buf], abort_flag)) goto conv_done;
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
            tc::tmem_ld16(tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)buf * half_cols +
                              (uint32_t)(m * item.npad + ch * 16), v);
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
      if (lane == 0) tc::mbar_arrive(&acc_empty[buf]);
      acc_phase[buf] ^= 1;
      buf ^= 1;
    }
  conv_done:;
  }

  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem_base, P.tmem_cols);
  if (threadIdx.x == 0 && *abort_flag) atomicExch(P.err, (int)FMAP_ERR_TIMEOUT);
}

}  // namespace

cudaError_t project_tc32_set_smem(int bytes) {
  return cudaFuncSetAttribute(project_tc32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_project_tc32(const TcProjParams& p, int grid, int smem_bytes, cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  project_tc32_kernel<<<grid, kThreads, smem_bytes, st>>>(p);
  return cudaGetLastError();
}

}  // namespace fmap
