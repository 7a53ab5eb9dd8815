// Backward spectral projection on the tensor cores for FP32 features (chain rule of
// Eq. 1), three-pass TF32:
//
//   dF_s (n x d, FP32) = diag(M_s) Phi_s (n x k) . dA_s (k x d)
//
// Same split as the FP32 forward projection: Phi = Pt + Pr with Pt = Phi as the MMA
// truncates it and Pr = Phi - Pt (exact), dA^T = Bh + Bl with Bh = dA^T rounded to TF32
// and Bl the exact remainder; Pt.Bh + Pt.Bl + Pr.Bh is accumulated in FP32 (the dropped
// Pr.Bl and the truncation of the correction terms are ~2^-20 relative).
//
// kind::tf32 MMA, M = 128 vertices, N = one feature group (<= 64 features), K = the
// basis index in blocks of 32. One persistent CTA per SM walks its list of (shape,
// feature group, vertex chunk) items:
//   warp 0      TMA-loads the Phi tiles (FP32, K-major, 128-byte swizzle) and, once per
//               item, bulk-copies the group's Bh / Bl images (built once per backward
//               pass, K-major swizzled) into shared memory;
//   warps 10-13 write Pr beside every Phi stage (element by element, same layout);
//   warp 1      issues the three MMAs per K-step into a double-buffered TMEM accumulator;
//   warps 2-9   read the accumulator, scale each row (vertex) by its mass, and write dF
//               in FP32 through shared memory with TMA stores.
// Waits are bounded like the other tensor-core kernels'.
#include "fmap_internal.cuh"
#include "tc_ptx.cuh"

namespace fmap {
namespace {

constexpr int kEpiWarps = 8;
constexpr int kConvWarps = 4;
constexpr int kThreads = 32 * (2 + kEpiWarps + kConvWarps);
constexpr int kTileV = 128;                          // vertices per output tile (MMA M)
constexpr uint32_t kAStageBytes = kTileV * 128;      // 128 rows x 32 FP32
constexpr uint32_t kOutChunkBytes = 32 * 16 * 4;     // 32 rows x 16 FP32: one TMA store box
constexpr uint32_t kOutWarpBytes = 2 * kOutChunkBytes;   // <= 32 features per warp and tile

// x minus the TF32 value the tensor core reads for it (the low 13 bits dropped): exact.
__device__ __forceinline__ float tf32_trunc_rest(float x) {
  return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

__global__ void __launch_bounds__(kThreads, 1) project_bwd_tc32_kernel(TcBwdParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = P.stages;
  uint8_t* sB = smem;                                   // Bh then Bl image of the item's feature group
  uint8_t* sA = sB + 2 * (size_t)P.b_bytes_max;         // per stage: Phi tile, then Pr
  uint8_t* sOut = sA + (size_t)S * 2 * kAStageBytes;    // FP32 dF staging, kOutWarpBytes per epilogue warp
  uint64_t* bars = reinterpret_cast<uint64_t*>(sOut + (size_t)kEpiWarps * kOutWarpBytes);
  uint64_t* a_full = bars;
  uint64_t* a_conv = bars + S;
  uint64_t* a_empty = bars + 2 * S;
  uint64_t* b_full = bars + 3 * S;
  uint64_t* b_empty = b_full + 1;
  uint64_t* acc_full = b_empty + 1;      // [2]
  uint64_t* acc_empty = acc_full + 2;    // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int it_beg = P.cta_first[blockIdx.x], it_end = P.cta_first[blockIdx.x + 1];
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&a_full[s], 1);
      tc::mbar_init(&a_conv[s], kConvWarps);
      tc::mbar_init(&a_empty[s], 1);
    }
    tc::mbar_init(b_full, 1);
    tc::mbar_init(b_empty, 1);
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], kEpiWarps);
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
      uint32_t stage = 0, phase = 0, bphase = 0;
      for (int it = it_beg; it < it_end; ++it) {
        const TcBwdItem item = P.items[it];
        const CUtensorMap* map = P.phimaps + item.shape;
        tc::prefetch_tmap(map);
        if (!tc::mbar_wait(b_empty, bphase ^ 1, abort_flag)) goto producer_done;
        {
          // Bh then Bl, contiguous in the workspace; Bl at b_bytes_max in shared memory
          const uint32_t bbytes = (uint32_t)item.kb * (uint32_t)item.nf * 128u;   // one image
          tc::mbar_arrive_expect_tx(b_full, 2 * bbytes);
          const uint8_t* src = reinterpret_cast<const uint8_t*>(P.ws + item.img_off);
          for (int h = 0; h < 2; ++h)
            for (uint32_t off = 0; off < bbytes; off += 16384u)
              tc::bulk_g2s(sB + h * P.b_bytes_max + off, src + h * bbytes + off,
                           (bbytes - off) < 16384u ? (bbytes - off) : 16384u, b_full);
        }
        bphase ^= 1;
        const int ntiles = (int)((item.v1 - item.v0 + kTileV - 1) / kTileV);
        for (int t = 0; t < ntiles; ++t) {
          const int y = (int)(item.v0 + (int64_t)t * kTileV);
          for (int kb = 0; kb < item.kb; ++kb) {
            if (!tc::mbar_wait(&a_empty[stage], phase ^ 1, abort_flag)) goto producer_done;
            tc::mbar_arrive_expect_tx(&a_full[stage], kAStageBytes);
            uint8_t* dst = sA + (size_t)stage * 2 * kAStageBytes;
            tc::tma_load_2d(dst, map, &a_full[stage], kb * 32, y);
            tc::tma_load_2d(dst + kAStageBytes / 2, map, &a_full[stage], kb * 32, y + kTileV / 2);
            if (++stage == (uint32_t)S) { stage = 0; phase ^= 1; }
          }
        }
      }
    producer_done:
      if (*abort_flag) {
        const uint64_t t0 = tc::globaltimer();
        while (tc::globaltimer() - t0 < 2000000ull) {}
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t stage = 0, phase = 0, bphase = 0;
      uint32_t acc_phase[2] = {0, 0};
      int buf = 0;
      bool ok = true;
      for (int it = it_beg; it < it_end && ok; ++it) {
        const TcBwdItem item = P.items[it];
        if (!tc::mbar_wait(b_full, bphase, abort_flag)) break;
        bphase ^= 1;
        tc::tc_fence_after();
        const uint32_t idesc = tc::idesc_tf32(128, (uint32_t)item.nf);
        const uint32_t bh_base = tc::smem_u32(sB);
        const uint32_t bl_base = bh_base + P.b_bytes_max;
        const int ntiles = (int)((item.v1 - item.v0 + kTileV - 1) / kTileV);
        for (int t = 0; t < ntiles && ok; ++t) {
          if (!tc::mbar_wait(&acc_empty[buf], acc_phase[buf] ^ 1, abort_flag)) { ok = false; break; }
          tc::tc_fence_after();
          const uint32_t d = tmem_base + (uint32_t)(buf * (P.tmem_cols / 2));
          for (int kb = 0; kb < item.kb; ++kb) {
            if (!tc::mbar_wait(&a_conv[stage], phase, abort_flag)) { ok = false; break; }
            tc::tc_fence_after();
            const uint32_t a_base = tc::smem_u32(sA + (size_t)stage * 2 * kAStageBytes);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              const uint64_t at = tc::smem_desc(a_base + ks * 32, 16, 1024, tc::kLayoutSW128);
              const uint64_t ar = tc::smem_desc(a_base + kAStageBytes + ks * 32, 16, 1024, tc::kLayoutSW128);
              const uint32_t boff = (uint32_t)(kb * item.nf * 128) + ks * 32;
              const uint64_t bh = tc::smem_desc(bh_base + boff, 16, 1024, tc::kLayoutSW128);
              const uint64_t bl = tc::smem_desc(bl_base + boff, 16, 1024, tc::kLayoutSW128);
              tc::mma_tf32(d, at, bh, idesc, (kb | ks) != 0 ? 1u : 0u);
              tc::mma_tf32(d, at, bl, idesc, 1u);
              tc::mma_tf32(d, ar, bh, idesc, 1u);
            }
            tc::mma_commit(&a_empty[stage]);
            if (++stage == (uint32_t)S) { stage = 0; phase ^= 1; }
          }
          if (!ok) break;
          tc::mma_commit(&acc_full[buf]);
          acc_phase[buf] ^= 1;
          buf ^= 1;
        }
        if (!ok) break;
        tc::mma_commit(b_empty);
      }
    }
  } else if (warp >= 2 + kEpiWarps) {
    // ------------------------------------------------------------ Phi remainder (Pr)
    const int ct = threadIdx.x - 32 * (2 + kEpiWarps);   // 0 .. 127
    uint32_t stage = 0, phase = 0;
    for (int it = it_beg; it < it_end; ++it) {
      const TcBwdItem item = P.items[it];
      const int ntiles = (int)((item.v1 - item.v0 + kTileV - 1) / kTileV);
      for (int t = 0; t < ntiles; ++t)
        for (int kb = 0; kb < item.kb; ++kb) {
          if (!tc::mbar_wait(&a_full[stage], phase, abort_flag)) goto conv_done;
          const float4* src = reinterpret_cast<const float4*>(sA + (size_t)stage * 2 * kAStageBytes);
          float4* dst = reinterpret_cast<float4*>(sA + (size_t)stage * 2 * kAStageBytes + kAStageBytes);
#pragma unroll
          for (int r = 0; r < (int)(kAStageBytes / 16) / (32 * kConvWarps); ++r) {
            const float4 x = src[ct + 32 * kConvWarps * r];
            dst[ct + 32 * kConvWarps * r] =
                make_float4(tf32_trunc_rest(x.x), tf32_trunc_rest(x.y), tf32_trunc_rest(x.z), tf32_trunc_rest(x.w));
          }
          tc::fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) tc::mbar_arrive(&a_conv[stage]);
          if (++stage == (uint32_t)S) { stage = 0; phase ^= 1; }
        }
    }
  conv_done:;
  } else {
    // ------------------------------------------------------------ epilogue: TMEM -> M * acc -> FP32 dF
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    uint8_t* stage_out = sOut + (size_t)(warp - 2) * kOutWarpBytes;
    uint32_t acc_phase[2] = {0, 0};
    int buf = 0;
    for (int it = it_beg; it < it_end; ++it) {
      const TcBwdItem item = P.items[it];
      const ShapeDev s = P.shapes[item.shape];
      const CUtensorMap* dmap = P.dfmaps + item.shape;
      const int ntiles = (int)((item.v1 - item.v0 + kTileV - 1) / kTileV);
      for (int t = 0; t < ntiles; ++t) {
        const int64_t vrow0 = item.v0 + (int64_t)t * kTileV + quarter * 32;
        const int64_t v = vrow0 + lane;
        const float m = v < item.v1 ? __ldg(s.mass + v) : 0.f;
        if (!tc::mbar_wait(&acc_full[buf], acc_phase[buf], abort_flag)) goto epi_done;
        tc::tc_fence_after();
        if (lane == 0) tc::bulk_wait_group_read0();
        __syncwarp();
        int j = 0;
        for (int ch = half; ch < item.nf / 16; ch += 2, ++j) {
          float x[16];
          tc::tmem_ld16(tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * (P.tmem_cols / 2) + ch * 16),
                        x);
          float4* dst = reinterpret_cast<float4*>(stage_out + j * kOutChunkBytes + lane * 64);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            dst[q] = make_float4(x[4 * q] * m, x[4 * q + 1] * m, x[4 * q + 2] * m, x[4 * q + 3] * m);
        }
        tc::tc_fence_before();
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&acc_empty[buf]);
        if (lane == 0 && vrow0 < s.n) {
          j = 0;
          for (int ch = half; ch < item.nf / 16; ch += 2, ++j)
            tc::tma_store_2d(dmap, stage_out + j * kOutChunkBytes, item.f0 + ch * 16, (int)vrow0);
          tc::bulk_commit_group();
        }
        acc_phase[buf] ^= 1;
        buf ^= 1;
      }
    }
  epi_done:
    if (lane == 0) tc::bulk_wait_group0();
  }

  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem_base, P.tmem_cols);
  if (threadIdx.x == 0 && *abort_flag) atomicExch(P.err, (int)FMAP_ERR_TIMEOUT);
}

// dA_s^T of one feature group as two K-major, 128-byte-swizzled FP32 images, the TF32
// head Bh (rounded to nearest) and the exact remainder Bl right after it: block kb
// (basis 32kb..32kb+31) holds nf rows of 128 bytes, 16-byte chunk c of row f at c ^ (f & 7).
__global__ void build_dat_image32_kernel(const ShapeDev* shapes, const TcBwdGroup* groups, const float* d_a,
                                         float* ws) {
  const TcBwdGroup g = groups[blockIdx.y];
  const ShapeDev s = shapes[g.shape];
  const int total = g.kb * g.nf * 32;
  float* img = ws + g.img_off;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int kb = e / (g.nf * 32);
    const int rem = e % (g.nf * 32);
    const int f = rem / 32, nl = rem % 32;
    const int n = kb * 32 + nl, fg = g.f0 + f;
    const float val = (n < s.k && fg < s.d) ? d_a[s.a_off + (int64_t)n * s.d + fg] : 0.f;
    const int chunk = nl >> 2;
    const int64_t at = (int64_t)kb * g.nf * 32 + f * 32 + ((chunk ^ (f & 7)) << 2) + (nl & 3);
    const float h = tc::tf32_rna(val);
    img[at] = h;
    img[at + total] = val - h;
  }
}

}  // namespace

cudaError_t project_bwd_tc32_set_smem(int bytes) {
  return cudaFuncSetAttribute(project_bwd_tc32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_build_dat_image32(const ShapeDev* shapes, const TcBwdGroup* groups, int n_groups, int max_elems,
                                     const float* d_a, float* ws, cudaStream_t st) {
  if (n_groups <= 0) return cudaSuccess;
  dim3 grid((unsigned)std::max(1, std::min((max_elems + 255) / 256, 1024)), (unsigned)n_groups);
  build_dat_image32_kernel<<<grid, 256, 0, st>>>(shapes, groups, d_a, ws);
  return cudaGetLastError();
}

cudaError_t launch_project_bwd_tc32(const TcBwdParams& p, int grid, int smem_bytes, cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  project_bwd_tc32_kernel<<<grid, kThreads, smem_bytes, st>>>(p);
  return cudaGetLastError();
}

}  // namespace fmap
