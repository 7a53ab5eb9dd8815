// Spatial gradient features (Sec. "Learned Scaling and Rotation in DiffusionNet"), fused
// in one kernel that writes the features straight into the projection's input layout:
//
//   z_v = sum_u G_vu X_u          (sparse complex gradient operator G, CSR; z = x + i y)
//   [P | Q] = [x | y] W           (W: the 2D x 2D real form of the learned complex A)
//   g_v = x o P + y o Q           (= Re(conj(z) o Az) for variant A)
//
// with P = (Az)_re = A_re x - A_im y and Q = (Az)_im = A_re y + A_im x (variant A) or
// A_re x + A_im y (variant B). One persistent CTA per SM walks 128-vertex tiles:
//   all 16 warps  gather x and y of the tile's vertices (lanes over channels, float4
//                 rows of X) into a K-major, 128-byte-swizzled FP32 tile in shared memory
//                 (K = the 2D channels x, y); each warp pass keeps eight rows of X in
//                 flight per lane and fetches the next pass's CSR offsets and first eight
//                 entries while the current rows load;
//   thread 0      streams the K-blocks of the W image (built once per call in the
//                 workspace, rounded to TF32) through two shared-memory stages (the first
//                 two issued before the gather) and issues tcgen05.mma kind::tf32
//                 (M = 128 vertices, N = 2D, K = 8) into TMEM;
//   warps 4-7     read P and Q from TMEM (one vertex per lane), x and y from the tile,
//                 and store g in FP32 or BF16 rows of the output.
// The x, y tile is the MMA operand and the epilogue's input, so a tile's gather starts
// after the previous tile's epilogue. Waits are bounded; a wait that gives up, or a CSR
// index out of range, sets the caller's status word.
#include "fmap_internal.cuh"
#include "tc_ptx.cuh"

namespace fmap {
namespace {

constexpr int kGfThreads = 512;
constexpr int kGfTileV = 128;
constexpr int kGfMaxDim = 128;

// Byte offset of (row r, K index kk) in a K-major tile of 128-byte rows with the 128-byte
// swizzle: K-block kk / 32 of `rows` rows, 16-byte chunk (kk % 32) / 4 of row r stored at
// chunk ((kk % 32) / 4) ^ (r % 8).
__device__ __forceinline__ uint32_t sw_off(int r, int kk, int rows) {
  const int kb = kk >> 5, ch = (kk & 31) >> 2;
  return (uint32_t)kb * (uint32_t)rows * 128u + (uint32_t)r * 128u + (uint32_t)((ch ^ (r & 7)) << 4) +
         (uint32_t)((kk & 3) << 2);
}

// W image: K-block kb holds the 2D output columns n (rows of 128 bytes, K-major),
// value W[k][n] for k = 32 kb + kk, rounded to TF32. Column n < D is P_n, n >= D is Q_{n-D};
// row k < D is x_k, k >= D is y_{k-D}.
__global__ void gradfeat_w_image_kernel(const float* a_re, const float* a_im, int dim, int variant, float* img) {
  const int n2 = 2 * dim;
  const int total = n2 * n2;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int kb = e / (n2 * 32);
    const int rem = e % (n2 * 32);
    const int n = rem / 32, kk = rem % 32;
    const int k = 32 * kb + kk;
    const bool kx = k < dim, nq = n >= dim;
    const int i = nq ? n - dim : n, j = kx ? k : k - dim;
    const float are = a_re[(int64_t)i * dim + j], aim = a_im[(int64_t)i * dim + j];
    float w;
    if (!nq)
      w = kx ? are : -aim;                                  // P_i = A_re x - A_im y
    else if (variant == 0)
      w = kx ? aim : are;                                   // Q_i = A_re y + A_im x
    else
      w = kx ? are : aim;                                   // Q_i = A_re x + A_im y
    img[(int64_t)(kb * n2 + n) * 32 + (((kk >> 2) ^ (n & 7)) << 2) + (kk & 3)] = tc::tf32_rna(w);
  }
}

struct GfParams {
  int64_t n, n_in, nnz;
  const int64_t* row_ptr;
  const int32_t* col_idx;
  const float2* vals;
  const float* x_in;
  int64_t ld_in;
  int32_t dim;
  void* out;
  int64_t ld_out;
  int32_t out_bf16;
  const float* w_img;
  int32_t* status;
  uint32_t tmem_cols;
};

__global__ void __launch_bounds__(kGfThreads, 1) gradfeat_kernel(GfParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int dim = P.dim, n2 = 2 * dim, nkb = n2 / 32;
  const uint32_t a_bytes = (uint32_t)kGfTileV * (uint32_t)n2 * 4u;   // x | y tile
  const uint32_t w_stage = (uint32_t)n2 * 128u;                       // one K-block of W
  uint8_t* sA = smem;
  uint8_t* sW = sA + a_bytes;
  uint64_t* w_full = reinterpret_cast<uint64_t*>(sW + 2 * w_stage);
  uint64_t* w_empty = w_full + 2;
  uint64_t* acc_full = w_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_full + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* bad_index = const_cast<int*>(reinterpret_cast<volatile int*>(tmem_slot + 2));

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(&w_full[s], 1);
      tc::mbar_init(&w_empty[s], 1);
    }
    tc::mbar_init(acc_full, 1);
    *abort_flag = 0;
    *bad_index = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, P.tmem_cols);
    tc::tmem_relinquish();
    tc::tc_fence_before();
  }
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  const uint32_t idesc = tc::idesc_tf32(128, (uint32_t)n2);

  // gather mapping: `lpv` lanes per vertex (4 channels each), `vpw` vertices per warp pass
  constexpr int kWarps = kGfThreads / 32;
  const int lpv = dim / 4, vpw = 32 / lpv;
  const int sub = lane / lpv, cl = lane % lpv;
  const bool lane_on = sub < vpw;
  const int npass = (kGfTileV + kWarps * vpw - 1) / (kWarps * vpw);
  const int64_t ntiles = (P.n + kGfTileV - 1) / kGfTileV;
  const uint8_t* wsrc = reinterpret_cast<const uint8_t*>(P.w_img);
  auto load_stage = [&](int kb) {
    const int s = kb & 1;
    tc::mbar_arrive_expect_tx(&w_full[s], w_stage);
    for (uint32_t off = 0; off < w_stage; off += 16384u)
      tc::bulk_g2s(sW + (size_t)s * w_stage + off, wsrc + (size_t)kb * w_stage + off,
                   (w_stage - off) < 16384u ? (w_stage - off) : 16384u, &w_full[s]);
  };
  // CSR offsets of the vertex of pass `ps` (length 0 outside the tile or the operator)
  auto meta = [&](int64_t v0, int ps, int64_t& e0, int& len) {
    const int r = (ps * kWarps + warp) * vpw + sub;
    const int64_t v = v0 + r;
    e0 = 0;
    len = 0;
    if (lane_on && r < kGfTileV && v < P.n) {
      const int64_t a = __ldg(P.row_ptr + v), b = __ldg(P.row_ptr + v + 1);
      if (a < 0 || b < a || b > P.nnz) {
        *bad_index = 1;
      } else {
        e0 = a;
        len = (b - a) < (int64_t)(1 << 30) ? (int)(b - a) : (1 << 30);
      }
    }
  };
  // entries q .. q+7 of a row (column -1: none); a column outside X is reported and skipped
  auto entries = [&](int64_t e0, int len, int q, int32_t (&c)[8], float2 (&g)[8]) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      c[u] = -1;
      g[u] = make_float2(0.f, 0.f);
      if (q + u < len) {
        const int32_t cc = __ldg(P.col_idx + e0 + q + u);
        if (cc >= 0 && cc < P.n_in) {
          c[u] = cc;
          g[u] = __ldg(P.vals + e0 + q + u);
        } else {
          *bad_index = 1;
        }
      }
    }
  };
  auto accumulate = [&](const int32_t (&c)[8], const float2 (&g)[8], float4& ax, float4& ay) {
    float4 xr[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      xr[u] = c[u] >= 0 ? __ldg(reinterpret_cast<const float4*>(P.x_in + (int64_t)c[u] * P.ld_in) + cl)
                        : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      ax.x = fmaf(g[u].x, xr[u].x, ax.x); ax.y = fmaf(g[u].x, xr[u].y, ax.y);
      ax.z = fmaf(g[u].x, xr[u].z, ax.z); ax.w = fmaf(g[u].x, xr[u].w, ax.w);
      ay.x = fmaf(g[u].y, xr[u].x, ay.x); ay.y = fmaf(g[u].y, xr[u].y, ay.y);
      ay.z = fmaf(g[u].y, xr[u].z, ay.z); ay.w = fmaf(g[u].y, xr[u].w, ay.w);
    }
  };
  uint32_t wphase[2] = {0, 0}, ephase[2] = {0, 0}, aphase = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t v0 = tile * kGfTileV;
    // the first two K-blocks of W stream in while the tile gathers (the previous tile's
    // MMAs have completed: their stages were drained)
    if (tid == 0) {
      load_stage(0);
      if (nkb > 1) load_stage(1);
    }
    // ---------------------------------------------------------------- gather x, y
    int64_t e0;
    int len;
    meta(v0, 0, e0, len);
    int32_t c_cur[8];
    float2 g_cur[8];
    entries(e0, len, 0, c_cur, g_cur);
    for (int ps = 0; ps < npass; ++ps) {
      const int r = (ps * kWarps + warp) * vpw + sub;
      int64_t e0n = 0;
      int lenn = 0;
      if (ps + 1 < npass) meta(v0, ps + 1, e0n, lenn);
      float4 ax = make_float4(0.f, 0.f, 0.f, 0.f), ay = ax;
      int mx = len;
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      // rows longer than eight entries: the rest first, one chunk of eight at a time
      for (int q = 8; q < mx; q += 8) {
        int32_t c_more[8];
        float2 g_more[8];
        entries(e0, len, q, c_more, g_more);
        accumulate(c_more, g_more, ax, ay);
      }
      // the next pass's first entries load while this pass's first eight rows of X do
      int32_t c_nxt[8];
      float2 g_nxt[8];
      entries(e0n, lenn, 0, c_nxt, g_nxt);
      accumulate(c_cur, g_cur, ax, ay);
      if (lane_on && r < kGfTileV) {
        *reinterpret_cast<float4*>(sA + sw_off(r, 4 * cl, kGfTileV)) = ax;
        *reinterpret_cast<float4*>(sA + sw_off(r, dim + 4 * cl, kGfTileV)) = ay;
      }
      e0 = e0n;
      len = lenn;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        c_cur[u] = c_nxt[u];
        g_cur[u] = g_nxt[u];
      }
    }
    tc::fence_proxy_async_smem();
    __syncthreads();
    // ---------------------------------------------------------------- MMAs
    if (tid == 0) {
      bool ok = true;
      const uint32_t a_base = tc::smem_u32(sA);
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int s = kb & 1;
        if (!tc::mbar_wait(&w_full[s], wphase[s], abort_flag)) { ok = false; break; }
        wphase[s] ^= 1;
        tc::tc_fence_after();
        const uint32_t b_base = tc::smem_u32(sW + (size_t)s * w_stage);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint64_t ad = tc::smem_desc(a_base + (uint32_t)kb * (kGfTileV * 128u) + ks * 32, 16, 1024,
                                            tc::kLayoutSW128);
          const uint64_t bd = tc::smem_desc(b_base + ks * 32, 16, 1024, tc::kLayoutSW128);
          tc::mma_tf32(tmem_base, ad, bd, idesc, (kb | ks) != 0 ? 1u : 0u);
        }
        tc::mma_commit(&w_empty[s]);
        if (kb + 2 < nkb) {
          // the stage is refilled once the MMAs that read it have completed
          if (!tc::mbar_wait(&w_empty[s], ephase[s], abort_flag)) { ok = false; break; }
          ephase[s] ^= 1;
          load_stage(kb + 2);
        }
      }
      tc::mma_commit(acc_full);
      // stages whose last MMAs were not waited for: drain their commits, so that the
      // phases stay in step for the next tile
      for (int kb = (nkb > 2 ? nkb - 2 : 0); kb < nkb && ok; ++kb) {
        const int s = kb & 1;
        if (!tc::mbar_wait(&w_empty[s], ephase[s], abort_flag)) break;
        ephase[s] ^= 1;
      }
    }
    // ---------------------------------------------------------------- epilogue
    if (warp >= 4 && warp < 8) {
      const int quarter = warp & 3;
      const int r = quarter * 32 + lane;
      const int64_t v = v0 + r;
      if (tc::mbar_wait(acc_full, aphase, abort_flag)) {
        tc::tc_fence_after();
        for (int c0 = 0; c0 < dim; c0 += 16) {
          float pv[16], qv[16];
          tc::tmem_ld16(tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, pv);
          tc::tmem_ld16(tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(dim + c0), qv);
          float g[16];
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const float4 xv = *reinterpret_cast<const float4*>(sA + sw_off(r, c0 + 4 * h, kGfTileV));
            const float4 yv = *reinterpret_cast<const float4*>(sA + sw_off(r, dim + c0 + 4 * h, kGfTileV));
            g[4 * h + 0] = fmaf(xv.x, pv[4 * h + 0], yv.x * qv[4 * h + 0]);
            g[4 * h + 1] = fmaf(xv.y, pv[4 * h + 1], yv.y * qv[4 * h + 1]);
            g[4 * h + 2] = fmaf(xv.z, pv[4 * h + 2], yv.z * qv[4 * h + 2]);
            g[4 * h + 3] = fmaf(xv.w, pv[4 * h + 3], yv.w * qv[4 * h + 3]);
          }
          if (v < P.n) {
            if (P.out_bf16) {
              uint32_t w[8];
#pragma unroll
              for (int q = 0; q < 8; ++q)
                w[q] = __bfloat16_as_ushort(__float2bfloat16_rn(g[2 * q])) |
                       ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(g[2 * q + 1])) << 16);
              uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(P.out) + v * P.ld_out + c0);
              dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
              dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
            } else {
              float4* dst = reinterpret_cast<float4*>(reinterpret_cast<float*>(P.out) + v * P.ld_out + c0);
#pragma unroll
              for (int h = 0; h < 4; ++h) dst[h] = make_float4(g[4 * h], g[4 * h + 1], g[4 * h + 2], g[4 * h + 3]);
            }
          }
        }
        tc::tc_fence_before();
      }
    }
    aphase ^= 1;
    __syncthreads();   // the tile's epilogue has read sA and TMEM before the next gather and MMAs
    if (*abort_flag) break;
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem_base, P.tmem_cols);
  if (tid == 0 && P.status) {
    if (*abort_flag) atomicCAS(P.status, 0, (int)FMAP_ERR_TIMEOUT);
    if (*bad_index) atomicCAS(P.status, 0, (int)FMAP_ERR_INVALID_ARG);
  }
}

size_t gf_smem_bytes(int dim) {
  return 1024 + (size_t)kGfTileV * 2 * dim * 4 + 2 * (size_t)(2 * dim) * 128 + 64;
}

}  // namespace
}  // namespace fmap

using namespace fmap;

extern "C" FMAP_API size_t fmap_gradient_features_ws_bytes(int32_t dim) {
  if (dim < 16 || dim > kGfMaxDim || dim % 16 != 0) return 0;
  return (size_t)(2 * dim) * (size_t)(2 * dim) * sizeof(float);
}

extern "C" FMAP_API int32_t fmap_gradient_features(int64_t n, const int64_t* row_ptr, const int32_t* col_idx,
                                                   const float* g_vals, int64_t nnz, int64_t n_in, const float* x_in,
                                                   int64_t ld_in, int32_t dim, const float* a_re, const float* a_im,
                                                   int32_t variant, void* out, int64_t ld_out, int32_t out_dtype,
                                                   int32_t* status, void* ws, size_t ws_bytes, void* stream) {
  if (n < 0 || nnz < 0 || n_in < 0) return FMAP_ERR_INVALID_ARG;
  if (variant != 0 && variant != 1) return FMAP_ERR_INVALID_ARG;
  if (out_dtype != FMAP_PREC_FP32 && out_dtype != FMAP_PREC_BF16) return FMAP_ERR_INVALID_ARG;
  if (dim < 16 || dim > kGfMaxDim || dim % 16 != 0) return FMAP_ERR_UNSUPPORTED;
  if (n == 0) return FMAP_OK;
  if (!row_ptr || !out || !a_re || !a_im || !status || (nnz > 0 && (!col_idx || !g_vals)) || (n_in > 0 && !x_in))
    return FMAP_ERR_INVALID_ARG;
  if (ld_in < dim || ld_out < dim) return FMAP_ERR_INVALID_ARG;
  if (ld_in % 4 != 0 || ld_out % 8 != 0) return FMAP_ERR_UNSUPPORTED;
  auto aligned = [](const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; };
  if (!aligned(x_in, 16) || !aligned(out, 16) || !aligned(g_vals, 8) || !aligned(row_ptr, 8) ||
      !aligned(col_idx, 4) || !aligned(a_re, 4) || !aligned(a_im, 4) || !aligned(status, 4))
    return FMAP_ERR_UNSUPPORTED;
  if (!ws || !aligned(ws, 256) || ws_bytes < fmap_gradient_features_ws_bytes(dim)) return FMAP_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return FMAP_ERR_CUDA;
  const size_t smem = gf_smem_bytes(dim);
  if (cudaFuncSetAttribute(gradfeat_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return FMAP_ERR_CUDA;
  if (cudaMemsetAsync(status, 0, sizeof(int32_t), st) != cudaSuccess) return FMAP_ERR_CUDA;
  float* img = static_cast<float*>(ws);
  const int img_elems = (2 * dim) * (2 * dim);
  gradfeat_w_image_kernel<<<std::max(1, std::min((img_elems + 255) / 256, 256)), 256, 0, st>>>(a_re, a_im, dim,
                                                                                                 variant, img);
  GfParams p{};
  p.n = n; p.n_in = n_in; p.nnz = nnz;
  p.row_ptr = row_ptr; p.col_idx = col_idx; p.vals = reinterpret_cast<const float2*>(g_vals);
  p.x_in = x_in; p.ld_in = ld_in; p.dim = dim;
  p.out = out; p.ld_out = ld_out; p.out_bf16 = out_dtype == FMAP_PREC_BF16 ? 1 : 0;
  p.w_img = img; p.status = status;
  uint32_t cols = 32;
  while (cols < (uint32_t)(2 * dim)) cols <<= 1;
  p.tmem_cols = cols;
  const int64_t ntiles = (n + kGfTileV - 1) / kGfTileV;
  const int grid = (int)std::min<int64_t>(ntiles, sms);
  gradfeat_kernel<<<grid, kGfThreads, smem, st>>>(p);
  return cudaGetLastError() == cudaSuccess ? FMAP_OK : FMAP_ERR_CUDA;
}
