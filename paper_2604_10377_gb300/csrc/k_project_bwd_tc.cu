// Backward spectral projection on the tensor cores (chain rule of Eq. 1), BF16 features:
//
//   dF_s (n x d) = diag(M_s) Phi_s (n x k) . dA_s (k x d)
//
// kind::tf32 MMA, M = 128 vertices, N = one feature group (<= 128 features),
// K = the basis index in blocks of 32. One persistent CTA per SM. CTAs 2c and 2c + 1
// take the two feature groups of the same (shape, vertex chunk) items in the same
// order, so they walk the same vertex tiles at about the same time: each loads the
// whole FP32 Phi tile with plain TMA loads, and the second of the two reads of a tile
// is served from L2, so HBM sees Phi about once per pair of groups. The B operand is
// dA_s^T of the CTA's feature group, prepared once per backward pass as a K-major
// swizzled FP32 image in the workspace and bulk-copied into shared memory per work
// item. The mass is a per-row (per-TMEM-lane) scale applied in the epilogue, which
// converts to BF16 and writes dF (and, when the shape asks for it, the same values
// before rounding as an FP32 copy). TF32 keeps ~2^-11 relative accuracy of each
// operand, far inside the BF16 storage of dF. Accumulators are double-buffered in
// TMEM so that the epilogue of one vertex tile overlaps the MMAs of the next.
//
// Waits are bounded like the forward kernel's; a timeout sets the workspace
// control word to FMAP_ERR_TIMEOUT.
#include "fmap_internal.cuh"
#include "tc_ptx.cuh"

namespace fmap {
namespace {

constexpr int kEpiWarps = 8;   // two per TMEM lane quarter, each storing half of the columns
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr int kTileV = 128;                       // vertices per output tile (MMA M)
constexpr uint32_t kAStageBytes = kTileV * 128;   // 128 rows x 32 fp32
constexpr uint32_t kOutChunkBytes = 32 * 32;      // 32 rows x 16 BF16: one TMA store box
constexpr uint32_t kOutWarpBytes = 4 * kOutChunkBytes;   // <= 4 chunks of 16 features per warp and tile

__global__ void __launch_bounds__(kThreads, 1) project_bwd_tc_kernel(TcBwdParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = P.stages;
  uint8_t* sB = smem;                                   // resident dA^T image of this CTA's feature group
  uint8_t* sA = sB + P.b_bytes_max;                     // Phi tiles, S stages
  uint8_t* sOut = sA + (size_t)S * kAStageBytes;        // BF16 dF staging, kOutWarpBytes per epilogue warp
  uint64_t* bars = reinterpret_cast<uint64_t*>(sOut + (size_t)kEpiWarps * kOutWarpBytes);
  uint64_t* a_full = bars;
  uint64_t* a_empty = bars + S;
  uint64_t* b_full = bars + 2 * S;
  uint64_t* b_empty = b_full + 1;
  uint64_t* acc_full = b_empty + 1;      // [2]
  uint64_t* acc_empty = acc_full + 2;    // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = blockIdx.x & 1u;           // 0 or 1: which feature group of the item pair
  const int cl = blockIdx.x >> 1;                  // CTA pair index
  const int it_beg = P.cta_first[cl], it_end = P.cta_first[cl + 1];
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&a_full[s], 1);
      tc::mbar_init(&a_empty[s], 1);     // released by this CTA's MMAs
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
    // The whole Phi tile (128 vertices) of every stage, as two boxes of 64 vertices.
    if (lane == 0) {
      uint32_t stage = 0, phase = 0, bphase = 0;
      for (int it = it_beg; it < it_end; ++it) {
        const TcBwdItem item = P.items[2 * it + rank];
        const CUtensorMap* map = P.phimaps + item.shape;
        tc::prefetch_tmap(map);
        if (!tc::mbar_wait(b_empty, bphase ^ 1, abort_flag)) goto producer_done;
        if (item.nf > 0) {
          const uint32_t bbytes = (uint32_t)item.kb * (uint32_t)item.nf * 128u;
          tc::mbar_arrive_expect_tx(b_full, bbytes);
          const uint8_t* src = reinterpret_cast<const uint8_t*>(P.ws + item.img_off);
          for (uint32_t off = 0; off < bbytes; off += 16384u)
            tc::bulk_g2s(sB + off, src + off, (bbytes - off) < 16384u ? (bbytes - off) : 16384u, b_full);
        } else {
          tc::mbar_arrive(b_full);
        }
        bphase ^= 1;
        const int ntiles = (int)((item.v1 - item.v0 + kTileV - 1) / kTileV);
        for (int t = 0; t < ntiles; ++t) {
          const int y = (int)(item.v0 + (int64_t)t * kTileV);
          for (int kb = 0; kb < item.kb; ++kb) {
            if (!tc::mbar_wait(&a_empty[stage], phase ^ 1, abort_flag)) goto producer_done;
            tc::mbar_arrive_expect_tx(&a_full[stage], kAStageBytes);
            uint8_t* dst = sA + (size_t)stage * kAStageBytes;
            tc::tma_load_2d(dst, map, &a_full[stage], kb * 32, y);
            tc::tma_load_2d(dst + kAStageBytes / 2, map, &a_full[stage], kb * 32, y + kTileV / 2);
            if (++stage == (uint32_t)S) { stage = 0; phase ^= 1; }
          }
        }
      }
      // every stage's last use has been released: no MMA still reads a stage when the
      // CTA leaves
      for (int s = 0; s < S; ++s) {
        if (!tc::mbar_wait(&a_empty[stage], phase ^ 1, abort_flag)) break;
        if (++stage == (uint32_t)S) { stage = 0; phase ^= 1; }
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
        const TcBwdItem item = P.items[2 * it + rank];
        if (!tc::mbar_wait(b_full, bphase, abort_flag)) break;
        bphase ^= 1;
        tc::tc_fence_after();
        const uint32_t idesc = tc::idesc_tf32(128, (uint32_t)(item.nf > 0 ? item.nf : 16));
        const uint32_t b_base = tc::smem_u32(sB);
        const int ntiles = (int)((item.v1 - item.v0 + kTileV - 1) / kTileV);
        for (int t = 0; t < ntiles && ok; ++t) {
          if (!tc::mbar_wait(&acc_empty[buf], acc_phase[buf] ^ 1, abort_flag)) { ok = false; break; }
          tc::tc_fence_after();
          const uint32_t d = tmem_base + (uint32_t)(buf * 128);
          for (int kb = 0; kb < item.kb; ++kb) {
            if (!tc::mbar_wait(&a_full[stage], phase, abort_flag)) { ok = false; break; }
            tc::tc_fence_after();
            const uint32_t a_base = tc::smem_u32(sA + (size_t)stage * kAStageBytes);
            if (item.nf > 0) {
#pragma unroll
              for (int ks = 0; ks < 4; ++ks) {
                const uint64_t ad = tc::smem_desc(a_base + ks * 32, 16, 1024, tc::kLayoutSW128);
                const uint64_t bd = tc::smem_desc(b_base + (uint32_t)(kb * item.nf * 128) + ks * 32, 16, 1024,
                                                  tc::kLayoutSW128);
                tc::mma_tf32(d, ad, bd, idesc, (kb | ks) != 0 ? 1u : 0u);
              }
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
  } else {
    // ------------------------------------------------------------ epilogue: TMEM -> M * acc -> BF16 dF
    // Each warp converts its 32 rows x (its chunks of 16 features) into shared memory
    // and one lane writes them with TMA stores (full-line writes, rows past n clipped).
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    uint8_t* stage_out = sOut + (size_t)(warp - 2) * kOutWarpBytes;
    uint32_t acc_phase[2] = {0, 0};
    int buf = 0;
    for (int it = it_beg; it < it_end; ++it) {
      const TcBwdItem item = P.items[2 * it + rank];
      const ShapeDev s = P.shapes[item.shape];
      const CUtensorMap* dmap = P.dfmaps + item.shape;
      const int ntiles = (int)((item.v1 - item.v0 + kTileV - 1) / kTileV);
      for (int t = 0; t < ntiles; ++t) {
        // the row's mass is loaded before the accumulator wait, so its latency is hidden
        const int64_t vrow0 = item.v0 + (int64_t)t * kTileV + quarter * 32;
        const int64_t v = vrow0 + lane;
        const float m = v < item.v1 ? __ldg(s.mass + v) : 0.f;
        if (!tc::mbar_wait(&acc_full[buf], acc_phase[buf], abort_flag)) goto epi_done;
        tc::tc_fence_after();
        // the previous tile's stores have read the staging buffer
        if (lane == 0) tc::bulk_wait_group_read0();
        __syncwarp();
        int j = 0;
        for (int ch = half; ch < item.nf / 16; ch += 2, ++j) {
          float x[16];
          tc::tmem_ld16(tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(buf * 128 + ch * 16), x);
          if (s.dfeat32 != nullptr && v < item.v1) {
            float4* d32 = reinterpret_cast<float4*>(s.dfeat32 + v * s.ld_feat + item.f0 + ch * 16);
#pragma unroll
            for (int q = 0; q < 4; ++q)
              d32[q] = make_float4(x[4 * q] * m, x[4 * q + 1] * m, x[4 * q + 2] * m, x[4 * q + 3] * m);
          }
          uint32_t w[8];
#pragma unroll
          for (int q = 0; q < 8; ++q)
            w[q] = __bfloat16_as_ushort(__float2bfloat16_rn(x[2 * q] * m)) |
                   ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x[2 * q + 1] * m)) << 16);
          uint4* dst = reinterpret_cast<uint4*>(stage_out + j * kOutChunkBytes + lane * 32);
          dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
          dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
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
    // every TMA store of this warp has completed before the CTA exits
    if (lane == 0) tc::bulk_wait_group0();
  }

  __syncthreads();
  if (warp == 1) tc::tmem_dealloc(tmem_base, P.tmem_cols);
  if (threadIdx.x == 0 && *abort_flag) atomicExch(P.err, (int)FMAP_ERR_TIMEOUT);
}

// dA_s^T of one feature group as the K-major, 128-byte-swizzled FP32 image the MMA
// reads: block kb (basis 32kb..32kb+31) holds nf rows of 128 bytes (one feature per
// row), 16-byte chunk c of row f stored at chunk c ^ (f & 7). Each value is rounded to
// the nearest TF32 here (the MMA would otherwise drop its low 13 bits), so the only
// truncated operand of the product is Phi.
__global__ void build_dat_image_kernel(const ShapeDev* shapes, const TcBwdGroup* groups, const float* d_a,
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
    const float raw = (n < s.k && fg < s.d) ? d_a[s.a_off + (int64_t)n * s.d + fg] : 0.f;
    uint32_t r32;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r32) : "f"(raw));
    const float val = __uint_as_float(r32);
    const int chunk = nl >> 2;
    img[(int64_t)kb * g.nf * 32 + f * 32 + ((chunk ^ (f & 7)) << 2) + (nl & 3)] = val;
  }
}

}  // namespace

cudaError_t project_bwd_tc_set_smem(int bytes) {
  return cudaFuncSetAttribute(project_bwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_build_dat_image(const ShapeDev* shapes, const TcBwdGroup* groups, int n_groups, int max_elems,
                                   const float* d_a, float* ws, cudaStream_t st) {
  if (n_groups <= 0) return cudaSuccess;
  dim3 grid((unsigned)std::max(1, std::min((max_elems + 255) / 256, 1024)), (unsigned)n_groups);
  build_dat_image_kernel<<<grid, 256, 0, st>>>(shapes, groups, d_a, ws);
  return cudaGetLastError();
}

cudaError_t launch_project_bwd_tc(const TcBwdParams& p, int grid, int smem_bytes, cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  // CTAs 2c and 2c + 1 (which walk the same Phi tiles) launch as a cluster of two: they
  // start together on one GPC, so the second read of each tile finds it in L2. The kernel
  // uses nothing of the cluster beyond that placement.
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = (size_t)smem_bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, project_bwd_tc_kernel, p);
}

}  // namespace fmap
