// Host runtime of the functional-map library: argument validation, the batch
// plan (offsets, work lists), the device descriptor tables, and the launch
// sequence of every C ABI entry point declared in include/fmap.h.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cudaTypedefs.h>

#include "adjoint_tc.cuh"
#include "fmap_internal.cuh"

using namespace fmap;

namespace {

thread_local char g_last_cuda_error[256] = "no error";

int32_t cuda_fail(cudaError_t e, const char* where) {
  std::snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s: %s", where, cudaGetErrorString(e));
  return FMAP_ERR_CUDA;
}

constexpr int64_t kAlignFloats = 64;   // 256-byte alignment of workspace regions
constexpr int64_t kTcChunkV = 8192;    // vertices per work item of the tensor-core backward projection
constexpr int kTcCtas = 152;           // persistent CTAs of the projection (one per GB300 SM)
constexpr int64_t kStageV = 64;        // vertices per projection pipeline stage
constexpr int64_t kTcSegMaxV = 8192;   // longest projection segment (one TMEM accumulation), BF16 F
constexpr int64_t kTc32SegMaxV = 512;   // the same for FP32 F (accuracy of the TF32 passes)
constexpr int kSmemBudget = 227 * 1024;

int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// RAII switch of the calling thread's current device.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// One launch of the forward projection: the segments of one spectral-size class.
struct TcLaunch {
  int32_t cta_off;     // offset of its proj_ctas + 1 CTA boundaries in tc_cta_first
  int32_t stages;
  uint32_t f_stage, p_stage, tmem_cols;
  int32_t smem;
};

struct Plan {
  fmap_options opt{};
  std::vector<ShapeDev> shapes;
  std::vector<PairDev> pairs;
  std::vector<int64_t> a_off, c_off, slot_list;
  std::vector<int2> systems;
  std::vector<SolveGroup> groups;
  int max_k = 0, max_d = 0;
  int64_t max_kd = 0;
  int64_t da_int_off = 0;
  int64_t loss_part_off = 0;
  // tensor-core projection
  bool tc32 = false;      // FP32 features: three-pass TF32 kernel
  bool tc_bwd = false;    // backward projection on the tensor cores (BF16 features: CTA pairs)
  bool tc_bwd32 = false;  // backward projection on the tensor cores (FP32 features: three TF32 passes)
  std::vector<TcItem> tc_items;
  int proj_ctas = kTcCtas;             // persistent CTAs of the forward projection
  int bwd_ctas = kTcCtas;              // and of the backward projection
  std::vector<int32_t> tc_cta_first;   // proj_ctas + 1 entries per launch
  std::vector<TcLaunch> tc_launches;
  std::vector<TcRedGroup> tc_groups;
  int64_t tc_max_group_elems = 0;
  int tc_smem = 0;                     // the largest dynamic shared memory of the launches
  // tensor-core backward projection
  std::vector<TcBwdItem> bw_items;
  std::vector<int32_t> bw_cta_first;   // bwd_ctas + 1 (FP32) or bwd_ctas / 2 + 1 (BF16) boundaries
  std::vector<TcBwdGroup> bw_groups;
  int bw_max_img = 0, bw_stages = 0, bw_smem = 0;
  uint32_t bw_b_bytes = 0;
  // tensor-core adjoint GEMMs (built when the batch is created: the SM count sets the tiles)
  AdjTcPlan adj;
  AdjTcPlan loss_tc;        // the training loss's GEMMs on the same kernel (E, then dL/dC)
  bool row_grads = false;   // some pair has per-row lambda gradients to write
  fmap_sizes sizes{};
};

int32_t validate_options(const fmap_options& o) {
  if (o.precision != FMAP_PREC_FP32 && o.precision != FMAP_PREC_BF16) return FMAP_ERR_INVALID_ARG;
  if (o.ir_steps < 0 || o.ir_steps > 3) return FMAP_ERR_INVALID_ARG;
  if (o.hi_gram_min_k < 1 || o.store_factors_max_k < 0) return FMAP_ERR_INVALID_ARG;
  if (o.adjoint_ir_steps < 0 || o.adjoint_ir_steps > 3) return FMAP_ERR_INVALID_ARG;
  if (o.proj_max_stages != 0 && (o.proj_max_stages < 2 || o.proj_max_stages > 6)) return FMAP_ERR_INVALID_ARG;
  if (o.proj_seg_max_v != 0 && (o.proj_seg_max_v < 2048 || o.proj_seg_max_v > 16384 || o.proj_seg_max_v % 64))
    return FMAP_ERR_INVALID_ARG;
  if (o.bwd_group_features != 0 && o.bwd_group_features != 64 && o.bwd_group_features != 128)
    return FMAP_ERR_INVALID_ARG;
  if (o.bwd_chunk_v != 0 && (o.bwd_chunk_v < 1024 || o.bwd_chunk_v > 65536 || o.bwd_chunk_v % 128))
    return FMAP_ERR_INVALID_ARG;
  if (o.solve_threads_k64 != 0 && o.solve_threads_k64 != 64 && o.solve_threads_k64 != 128) return FMAP_ERR_INVALID_ARG;
  if (o.solve_threads_k128 != 0 && o.solve_threads_k128 != 128 && o.solve_threads_k128 != 256)
    return FMAP_ERR_INVALID_ARG;
  if (o.solve_no_g_copy != 0 && o.solve_no_g_copy != 1) return FMAP_ERR_INVALID_ARG;
  if (o.adjoint_kernel < 0 || o.adjoint_kernel > 2) return FMAP_ERR_INVALID_ARG;
  if (o.adjoint_features != 0 && o.adjoint_features != 64 && o.adjoint_features != 128 && o.adjoint_features != 256)
    return FMAP_ERR_INVALID_ARG;
  if (o.adjoint_stages < 0 || o.adjoint_stages > 2) return FMAP_ERR_INVALID_ARG;
  if (o.proj_ctas < 0 || o.proj_ctas > kTcCtas) return FMAP_ERR_INVALID_ARG;
  if (o.bwd_ctas < 0 || o.bwd_ctas > kTcCtas || (o.bwd_ctas & 1)) return FMAP_ERR_INVALID_ARG;
  return FMAP_OK;
}

int32_t make_plan(const fmap_options& opt, const fmap_shape_desc* shapes, int32_t n_shapes,
                  const fmap_pair_desc* pairs, int32_t n_pairs, Plan& P) {
  int32_t rc = validate_options(opt);
  if (rc) return rc;
  if (n_shapes < 0 || n_pairs < 0 || n_shapes > 65535 || n_pairs > 65535) return FMAP_ERR_INVALID_ARG;
  if ((n_shapes > 0 && !shapes) || (n_pairs > 0 && !pairs)) return FMAP_ERR_INVALID_ARG;
  P.opt = opt;
  P.proj_ctas = opt.proj_ctas ? opt.proj_ctas : kTcCtas;
  P.bwd_ctas = opt.bwd_ctas ? opt.bwd_ctas : kTcCtas;
  const size_t fsz = opt.precision == FMAP_PREC_BF16 ? 2 : 4;

  P.shapes.resize(n_shapes);
  P.a_off.assign(n_shapes + 1, 0);
  for (int s = 0; s < n_shapes; ++s) {
    const fmap_shape_desc& d = shapes[s];
    if (!d.phi || !d.mass || !d.feat) return FMAP_ERR_INVALID_ARG;
    if (d.n < 1 || d.k < 1 || d.d < 1) return FMAP_ERR_INVALID_ARG;
    if (d.k > kMaxK || d.d > kMaxD || d.d % 16 != 0) return FMAP_ERR_UNSUPPORTED;
    if (d.ld_phi < d.k || d.ld_feat < d.d) return FMAP_ERR_INVALID_ARG;
    if (d.ld_phi % 4 != 0 || d.ld_feat % 8 != 0) return FMAP_ERR_UNSUPPORTED;
    if (!aligned(d.phi, 16) || !aligned(d.feat, 16) || !aligned(d.mass, 4)) return FMAP_ERR_UNSUPPORTED;
    if (d.dfeat && !aligned(d.dfeat, 16)) return FMAP_ERR_UNSUPPORTED;
    if (d.dfeat_f32 && !aligned(d.dfeat_f32, 16)) return FMAP_ERR_UNSUPPORTED;
    if (d.evals && !aligned(d.evals, 4)) return FMAP_ERR_UNSUPPORTED;
    ShapeDev& sd = P.shapes[s];
    std::memset(&sd, 0, sizeof(sd));
    sd.n = d.n; sd.k = d.k; sd.d = d.d;
    sd.phi = d.phi; sd.ld_phi = d.ld_phi; sd.mass = d.mass; sd.evals = d.evals;
    sd.feat = d.feat; sd.ld_feat = d.ld_feat; sd.dfeat = d.dfeat;
    sd.dfeat32 = (opt.precision == FMAP_PREC_BF16 && d.dfeat) ? d.dfeat_f32 : nullptr;
    sd.a_off = P.a_off[s];
    P.a_off[s + 1] = P.a_off[s] + (int64_t)d.k * d.d;
    P.max_k = std::max(P.max_k, d.k);
    P.max_d = std::max(P.max_d, d.d);
    P.max_kd = std::max(P.max_kd, (int64_t)d.k * d.d);
  }
  (void)fsz;

  P.pairs.resize(n_pairs);
  P.c_off.assign(n_pairs + 1, 0);
  for (int p = 0; p < n_pairs; ++p) {
    const fmap_pair_desc& q = pairs[p];
    if (q.shape_x < 0 || q.shape_x >= n_shapes || q.shape_y < 0 || q.shape_y >= n_shapes) return FMAP_ERR_INVALID_ARG;
    const fmap_shape_desc& sx = shapes[q.shape_x];
    const fmap_shape_desc& sy = shapes[q.shape_y];
    if (sx.d != sy.d) return FMAP_ERR_INVALID_ARG;
    if (!(q.lambda >= 0.f) || !std::isfinite(q.lambda)) return FMAP_ERR_INVALID_ARG;
    if (!q.mask && (!sx.evals || !sy.evals)) return FMAP_ERR_INVALID_ARG;
    if (q.mask && !aligned(q.mask, 4)) return FMAP_ERR_UNSUPPORTED;
    PairDev& pd = P.pairs[p];
    std::memset(&pd, 0, sizeof(pd));
    pd.x = q.shape_x; pd.y = q.shape_y; pd.k = sx.k; pd.d = sx.d;   // C is sy.k x sx.k
    pd.lam = q.lambda; pd.mask = q.mask;
    if (q.lambda_rows && !aligned(q.lambda_rows, 4)) return FMAP_ERR_UNSUPPORTED;
    if (q.d_lambda_rows && !aligned(q.d_lambda_rows, 4)) return FMAP_ERR_UNSUPPORTED;
    pd.lam_rows = q.lambda_rows;
    pd.dlam_rows = q.lambda_rows ? q.d_lambda_rows : nullptr;
    if (pd.dlam_rows) P.row_grads = true;
    pd.hi_gram = sx.k >= opt.hi_gram_min_k ? 1 : 0;
    pd.c_off = P.c_off[p];
    P.c_off[p + 1] = P.c_off[p] + (int64_t)sy.k * sx.k;
  }

  // ---- workspace layout (floats, 256-byte aligned regions); the first 256 bytes
  // hold control words (word 0: error raised by a device-side wait that timed out)
  int64_t cur = kAlignFloats;
  P.tc32 = opt.precision == FMAP_PREC_FP32;
  P.tc_bwd = opt.precision == FMAP_PREC_BF16;
  P.tc_bwd32 = opt.precision == FMAP_PREC_FP32;
  {
    // (shape, feature group) units, grouped by spectral-size class (k padded to 32, 64,
    // 128, 256); every class is one launch with its own pipeline depth, and within a
    // class a stream-K split of the vertex ranges into proj_ctas ranges of equal cost
    // (64-vertex granularity)
    // A spectral size above the widest basis range of one unit (256, the MMA's largest
    // N, for BF16 features; 128 for FP32 features, whose stages are larger) is split
    // into basis ranges of equal width (a multiple of 32), each reading its own Phi
    // columns and all of F.
    struct Unit { int s, f0, fg, npad, n0, nk, dspan; double cpv; };
    std::vector<Unit> classes[4];
    const int nmax = P.tc32 ? 128 : 256;
    for (int s = 0; s < n_shapes; ++s) {
      const ShapeDev& sd = P.shapes[s];
      const int nsplit = (sd.k + nmax - 1) / nmax;
      const int width = ((sd.k + nsplit - 1) / nsplit + 31) / 32 * 32;
      for (int h = 0; h < nsplit; ++h) {
        const int n0 = h * width;
        const int nk = std::min(width, sd.k - n0);
        if (nk <= 0) continue;
        const int npad = (nk + 15) / 16 * 16;
        const int mt = (sd.d + 127) / 128;
        int fg_cap = std::max(1, std::min(4, 512 / npad));
        if (P.tc32) {
          // two stages of (F + its remainder: 32 KB per group) + Phi, Ph, Pl must fit
          const int pb = (npad + 31) / 32 * 4096 + npad * 256;
          fg_cap = std::max(1, std::min(std::min(fg_cap, 2), ((kSmemBudget - 1536) / 2 - pb - 128) / 32768));
          fg_cap = std::max(1, std::min(fg_cap, 256 / npad));   // two accumulators in 512 TMEM columns
        }
        const int groups = (mt + fg_cap - 1) / fg_cap;
        const int fg_s = (mt + groups - 1) / groups;
        const int cls = npad <= 32 ? 0 : (npad <= 64 ? 1 : (npad <= 128 ? 2 : 3));
        for (int g = 0; g < groups; ++g) {
          Unit u;
          u.s = s; u.f0 = g * fg_s * 128; u.fg = std::min(fg_s, mt - g * fg_s); u.npad = npad;
          u.n0 = n0; u.nk = nk;
          u.dspan = std::min(u.fg * 128, sd.d - u.f0);
          u.cpv = 4.0 * nk + 4.0 + 2.0 * u.dspan;   // HBM bytes per vertex
          classes[cls].push_back(u);
        }
      }
    }
    // The tensor cores accumulate a segment in TMEM; the FP32-feature kernel bounds that
    // chain to 512 vertices (64 K-steps) so that the accumulator's rounding stays in the
    // FP32 class (a longer chain drifts, ~6e-8 relative per K-step); partials are then
    // added in IEEE FP32 by the reduction. The tuning knob applies to BF16 features.
    const int64_t seg_max = P.tc32 ? kTc32SegMaxV : (opt.proj_seg_max_v ? (int64_t)opt.proj_seg_max_v : kTcSegMaxV);
    // vertices per pipeline stage: 64 (BF16 F, one 128-byte row of BF16) or 32 (FP32 F)
    const int64_t stage_v = P.tc32 ? 32 : kStageV;
    for (int cls = 0; cls < 4; ++cls) {
      const std::vector<Unit>& units = classes[cls];
      if (units.empty()) continue;
      uint32_t fmax = 0, pmax = 0, tmax = 0;
      double total = 0.0;
      for (const Unit& u : units) {
        total += u.cpv * (double)P.shapes[u.s].n;
        // BF16: F tile; Phi tile converted in place into P hi / lo.
        // FP32: F tile and its TF32 remainder; Phi tile, then P hi and P lo beside it.
        const uint32_t kbu = (uint32_t)((u.npad + 31) / 32);
        fmax = std::max<uint32_t>(fmax, (uint32_t)u.fg * (P.tc32 ? 32768u : 16384u));
        const uint32_t pb = P.tc32 ? kbu * 4096u + (uint32_t)u.npad * 256u
                                   : std::max<uint32_t>(kbu * 8192u, (uint32_t)u.npad * 256u);
        pmax = std::max<uint32_t>(pmax, pb);
        tmax = std::max<uint32_t>(tmax, (uint32_t)(u.fg * u.npad));
      }
      TcLaunch L{};
      L.cta_off = (int32_t)P.tc_cta_first.size();
      const int nctas = P.proj_ctas;
      P.tc_cta_first.resize(P.tc_cta_first.size() + nctas + 1, 0);
      int32_t* first = P.tc_cta_first.data() + L.cta_off;
      first[0] = (int32_t)P.tc_items.size();
      const double per_cta = total / nctas;
      int cta = 0;
      double budget = per_cta;
      for (const Unit& u : units) {
        const ShapeDev& sd = P.shapes[u.s];
        TcRedGroup rg{};
        rg.shape = u.s; rg.f0 = u.f0; rg.stride = u.fg * 128; rg.dspan = u.dspan;
        rg.n0 = u.n0; rg.nk = u.nk;
        rg.it_beg = (int32_t)P.tc_items.size();
        int64_t v = 0;
        while (v < sd.n) {
          int64_t take = (int64_t)std::ceil(std::max(budget, 0.0) / u.cpv);
          take = std::max<int64_t>(stage_v, (take + stage_v - 1) / stage_v * stage_v);
          if (cta == nctas - 1) take = sd.n - v;
          // a segment accumulates in TMEM; bounding its length bounds the accumulated
          // rounding of the tensor-core FP32 sums (partials are added in IEEE FP32)
          take = std::min<int64_t>(std::min<int64_t>(take, seg_max), sd.n - v);
          TcItem it{};
          it.shape = u.s; it.f0 = u.f0; it.fg = u.fg; it.npad = u.npad;
          it.n0 = u.n0; it.nk = u.nk;
          it.v0 = v; it.v1 = v + take;
          it.part_off = cur;
          cur = align_up(cur + (int64_t)u.nk * rg.stride, kAlignFloats);
          P.tc_items.push_back(it);
          v += take;
          budget -= u.cpv * (double)take;
          if (budget <= 1e-9 * per_cta && cta < nctas - 1) {
            ++cta;
            first[cta] = (int32_t)P.tc_items.size();
            budget += per_cta;
          }
        }
        rg.it_end = (int32_t)P.tc_items.size();
        P.tc_groups.push_back(rg);
        P.tc_max_group_elems = std::max<int64_t>(P.tc_max_group_elems, (int64_t)u.nk * rg.dspan);
      }
      for (int c = cta + 1; c <= nctas; ++c) first[c] = (int32_t)P.tc_items.size();
      L.f_stage = std::max<uint32_t>(fmax, 16384u);
      L.p_stage = (std::max<uint32_t>(pmax, 8192u) + 1023u) / 1024u * 1024u;
      uint32_t cols = 32;
      while (cols < (P.tc32 ? 2 * tmax : tmax)) cols <<= 1;   // FP32: two accumulators
      L.tmem_cols = cols;
      const int fixed = 1024 + 512;
      const int per_stage = (int)(L.f_stage + L.p_stage) + (int)stage_v * 4;
      L.stages = std::min(opt.proj_max_stages ? opt.proj_max_stages : 6, (kSmemBudget - fixed) / per_stage);
      if (L.stages < 2) return FMAP_ERR_UNSUPPORTED;
      L.smem = fixed + L.stages * per_stage;
      P.tc_smem = std::max(P.tc_smem, L.smem);
      P.tc_launches.push_back(L);
    }
  }
  for (auto& pd : P.pairs) {
    const int64_t ky = P.shapes[pd.y].k;   // rows of C (k_Y); pd.k = k_X
    const int64_t kk = (int64_t)pd.k * pd.k, yk = ky * pd.k, yy = ky * ky;
    pd.g_off = cur; cur = align_up(cur + gram_floats(pd.k), kAlignFloats);
    pd.r_off = cur; cur = align_up(cur + yk, kAlignFloats);
    pd.e_off = cur; cur = align_up(cur + yy, kAlignFloats);
    if (pd.hi_gram) {
      pd.g64_off = cur / 2;
      cur = align_up(cur + 2 * kk, kAlignFloats);
    } else {
      pd.g64_off = -1;
    }
  }
  P.loss_part_off = cur;   // per-pair, per-tile partial sums of the training loss
  cur = align_up(cur + (int64_t)n_pairs * kMaxLossTiles, kAlignFloats);
  const int64_t ws_fwd = cur;
  for (auto& pd : P.pairs) {
    const int64_t ky = P.shapes[pd.y].k;
    const int64_t kk = (int64_t)pd.k * pd.k, yk = ky * pd.k;
    pd.gam_off = cur; cur = align_up(cur + yk, kAlignFloats);
    pd.w_off = cur; cur = align_up(cur + kk, kAlignFloats);
    pd.sx_off = cur; cur = align_up(cur + (int64_t)pd.k * pd.d, kAlignFloats);
    pd.sy_off = cur; cur = align_up(cur + ky * pd.d, kAlignFloats);
  }
  P.da_int_off = cur;
  cur = align_up(cur + P.a_off[n_shapes], kAlignFloats);
  if (P.tc_bwd) {
    // Backward work runs on pairs of CTAs (2c, 2c + 1) that walk the same Phi tiles at
    // the same time, so the second read of each tile hits L2: a shape's features split
    // into an even number of groups of <= 128, and a work item is (shape, vertex chunk,
    // pair of groups), one group per CTA of the pair. Items are sorted by cost and dealt
    // to the CTA pairs round-robin.
    const int n_ctapairs = P.bwd_ctas / 2;
    int64_t bw_work = 0;
    for (int s = 0; s < n_shapes; ++s)
      if (P.shapes[s].dfeat) bw_work += P.shapes[s].n * (int64_t)((P.shapes[s].d + 255) / 256);
    const int64_t bw_chunk = opt.bwd_chunk_v ? (int64_t)opt.bwd_chunk_v
                                             : std::min<int64_t>(kTcChunkV, std::max<int64_t>(
                                                   1024, (bw_work / (4 * n_ctapairs) + 127) / 128 * 128));
    const int bw_gf = opt.bwd_group_features ? opt.bwd_group_features : 128;
    std::vector<TcBwdItem> items;   // pairs: [2 j] for CTA 2c, [2 j + 1] for CTA 2c + 1
    for (int s = 0; s < n_shapes; ++s) {
      const ShapeDev& sd = P.shapes[s];
      if (!sd.dfeat) continue;
      const int kb = (sd.k + 31) / 32;
      const int ngroups = 2 * ((sd.d + 2 * bw_gf - 1) / (2 * bw_gf));
      const int nf_s = ((sd.d + ngroups - 1) / ngroups + 15) / 16 * 16;
      std::vector<TcBwdGroup> gl(ngroups);
      for (int g = 0; g < ngroups; ++g) {
        TcBwdGroup& bg = gl[g];
        bg.shape = s; bg.f0 = g * nf_s; bg.nf = std::max(0, std::min(nf_s, sd.d - bg.f0)); bg.kb = kb;
        bg.img_off = -1;
        if (bg.nf <= 0) continue;
        bg.img_off = cur;
        cur = align_up(cur + (int64_t)kb * bg.nf * 32, kAlignFloats);
        P.bw_groups.push_back(bg);
        P.bw_max_img = std::max(P.bw_max_img, kb * bg.nf * 32);
        P.bw_b_bytes = std::max<uint32_t>(P.bw_b_bytes, (uint32_t)(kb * bg.nf * 128));
      }
      for (int gp = 0; gp < ngroups / 2; ++gp)
        for (int64_t v0 = 0; v0 < sd.n; v0 += bw_chunk)
          for (int r = 0; r < 2; ++r) {
            const TcBwdGroup& bg = gl[2 * gp + r];
            TcBwdItem it{};
            it.shape = s; it.f0 = bg.f0; it.nf = bg.nf; it.kb = kb;
            it.v0 = v0; it.v1 = std::min<int64_t>(sd.n, v0 + bw_chunk);
            it.img_off = bg.img_off;
            items.push_back(it);
          }
    }
    if (!items.empty()) {
      const size_t npi = items.size() / 2;
      std::vector<int32_t> order(npi);
      for (size_t i = 0; i < npi; ++i) order[i] = (int32_t)i;
      auto bcost = [&](size_t j) {
        const TcBwdItem& it = items[2 * j];
        return (double)(it.v1 - it.v0) * (4.0 * P.shapes[it.shape].k + 2.0 * (it.nf + items[2 * j + 1].nf));
      };
      std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        const double cx = bcost(a), cy = bcost(b);
        if (cx != cy) return cx > cy;
        return a < b;
      });
      // CTA pair c takes pair-items c, c + n_ctapairs, ... of the sorted list, stored contiguously
      P.bw_cta_first.assign(n_ctapairs + 1, 0);
      for (int c = 0; c < n_ctapairs; ++c) {
        P.bw_cta_first[c] = (int32_t)(P.bw_items.size() / 2);
        for (size_t j = c; j < order.size(); j += n_ctapairs) {
          P.bw_items.push_back(items[2 * order[j]]);
          P.bw_items.push_back(items[2 * order[j] + 1]);
        }
      }
      P.bw_cta_first[n_ctapairs] = (int32_t)(P.bw_items.size() / 2);
    }
    const int fixed = 1024 + 512;
    const int out_staging = 8 * 4096;   // BF16 dF staging of the eight epilogue warps
    P.bw_stages = std::min(6, (kSmemBudget - fixed - out_staging - (int)P.bw_b_bytes) / 16384);
    if (!P.bw_items.empty() && P.bw_stages < 2) return FMAP_ERR_UNSUPPORTED;
    P.bw_smem = fixed + out_staging + (int)P.bw_b_bytes + P.bw_stages * 16384;
  }
  if (P.tc_bwd32) {
    // FP32 features: one CTA per SM over (shape, feature group, vertex chunk) items; a
    // group is 64 features (32 when the basis needs more than 6 blocks of 32, so that the
    // TF32 head and remainder images of dA^T plus two Phi stages fit), with its two
    // images contiguous in the workspace. Items sorted by cost, dealt round-robin.
    int kb_max = 1;
    for (int s = 0; s < n_shapes; ++s)
      if (P.shapes[s].dfeat) kb_max = std::max(kb_max, (P.shapes[s].k + 31) / 32);
    const int nf_g = kb_max <= 6 ? 64 : 32;
    int64_t bw_work = 0;
    for (int s = 0; s < n_shapes; ++s)
      if (P.shapes[s].dfeat) bw_work += P.shapes[s].n * (int64_t)((P.shapes[s].d + nf_g - 1) / nf_g);
    const int64_t bw_chunk = opt.bwd_chunk_v ? (int64_t)opt.bwd_chunk_v
                                             : std::min<int64_t>(kTcChunkV, std::max<int64_t>(
                                                   1024, (bw_work / (4 * P.bwd_ctas) + 127) / 128 * 128));
    std::vector<TcBwdItem> items;
    for (int s = 0; s < n_shapes; ++s) {
      const ShapeDev& sd = P.shapes[s];
      if (!sd.dfeat) continue;
      const int kb = (sd.k + 31) / 32;
      for (int f0 = 0; f0 < sd.d; f0 += nf_g) {
        TcBwdGroup bg{};
        bg.shape = s; bg.f0 = f0; bg.nf = std::min(nf_g, sd.d - f0); bg.kb = kb;
        bg.img_off = cur;
        cur = align_up(cur + 2 * (int64_t)kb * bg.nf * 32, kAlignFloats);
        P.bw_groups.push_back(bg);
        P.bw_max_img = std::max(P.bw_max_img, kb * bg.nf * 32);
        P.bw_b_bytes = std::max<uint32_t>(P.bw_b_bytes, (uint32_t)(kb * bg.nf * 128));
        for (int64_t v0 = 0; v0 < sd.n; v0 += bw_chunk) {
          TcBwdItem it{};
          it.shape = s; it.f0 = f0; it.nf = bg.nf; it.kb = kb;
          it.v0 = v0; it.v1 = std::min<int64_t>(sd.n, v0 + bw_chunk);
          it.img_off = bg.img_off;
          items.push_back(it);
        }
      }
    }
    if (!items.empty()) {
      std::vector<int32_t> order(items.size());
      for (size_t i = 0; i < items.size(); ++i) order[i] = (int32_t)i;
      auto bcost = [&](const TcBwdItem& it) {
        return (double)(it.v1 - it.v0) * (4.0 * P.shapes[it.shape].k + 4.0 * it.nf);
      };
      std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        const double cx = bcost(items[a]), cy = bcost(items[b]);
        if (cx != cy) return cx > cy;
        return a < b;
      });
      const int nctas = P.bwd_ctas;
      P.bw_cta_first.assign(nctas + 1, 0);
      for (int c = 0; c < nctas; ++c) {
        P.bw_cta_first[c] = (int32_t)P.bw_items.size();
        for (size_t j = c; j < order.size(); j += nctas) P.bw_items.push_back(items[order[j]]);
      }
      P.bw_cta_first[nctas] = (int32_t)P.bw_items.size();
    }
    const int fixed = 1024 + 512;
    const int out_staging = 8 * 4096;   // FP32 dF staging of the eight epilogue warps
    P.bw_stages = std::min(6, (kSmemBudget - fixed - out_staging - 2 * (int)P.bw_b_bytes) / 32768);
    if (!P.bw_items.empty() && P.bw_stages < 2) return FMAP_ERR_UNSUPPORTED;
    P.bw_smem = fixed + out_staging + 2 * (int)P.bw_b_bytes + P.bw_stages * 32768;
  }
  const int64_t ws_bwd = std::max(cur, ws_fwd);

  // ---- saved factors
  int64_t fac = 0;
  for (auto& pd : P.pairs) {
    if (pd.k <= opt.store_factors_max_k) {
      pd.fac_off = fac;
      fac = align_up(fac + (int64_t)P.shapes[pd.y].k * chol_factor_floats(pd.k), kAlignFloats);
    } else {
      pd.fac_off = -1;
    }
  }

  // ---- dA contributions per shape, in pair order
  for (int s = 0; s < n_shapes; ++s) {
    P.shapes[s].slot_beg = (int32_t)P.slot_list.size();
    for (const auto& pd : P.pairs) {
      if (pd.x == s) P.slot_list.push_back(pd.sx_off);
      if (pd.y == s) P.slot_list.push_back(pd.sy_off);
    }
    P.shapes[s].slot_end = (int32_t)P.slot_list.size();
  }

  // ---- row systems, grouped by block size, largest k first
  // (k <= 64: 64 threads, <= 128: 128, <= 256: 256, <= kMaxK: 320 -- every block has at
  // least one thread per padded row)
  const int bounds[4] = {64, 128, 256, kMaxK};
  const int threads[4] = {opt.solve_threads_k64 ? opt.solve_threads_k64 : 64,
                          opt.solve_threads_k128 ? opt.solve_threads_k128 : 128, 256, 320};
  for (int gi = 0; gi < 4; ++gi) {
    SolveGroup g{};
    g.first = (int32_t)P.systems.size();
    g.threads = threads[gi];
    g.no_g_copy = opt.solve_no_g_copy;
    std::vector<int> members;
    for (int p = 0; p < n_pairs; ++p) {
      const int k = P.pairs[p].k;
      const int lo = gi == 0 ? 0 : bounds[gi - 1];
      if (k > lo && k <= bounds[gi]) members.push_back(p);
    }
    std::stable_sort(members.begin(), members.end(), [&](int a, int b) { return P.pairs[a].k > P.pairs[b].k; });
    for (int p : members) {
      g.kmax = std::max(g.kmax, P.pairs[p].k);
      const int ky = P.shapes[P.pairs[p].y].k;   // one row system per row of C
      for (int i = 0; i < ky; ++i) P.systems.push_back(make_int2(p, i));
    }
    g.count = (int32_t)P.systems.size() - g.first;
    if (g.count > 0) P.groups.push_back(g);
  }

  P.sizes.a_floats = P.a_off[n_shapes];
  P.sizes.c_floats = P.c_off[n_pairs];
  P.sizes.ws_bytes = ws_fwd * 4;
  P.sizes.ws_bwd_bytes = ws_bwd * 4;
  P.sizes.saved_bytes = fac * 4;
  P.sizes.n_shapes = n_shapes;
  P.sizes.n_pairs = n_pairs;
  return FMAP_OK;
}

}  // namespace

struct fmap_ctx {
  int device;
  fmap_options opt;
};

struct Timing {
  bool on = false;
  std::vector<cudaEvent_t> ev;   // start/stop pairs
  std::vector<int> kind;
  int used = 0;
};
constexpr int kMaxTimedLaunches = 16384;

struct fmap_batch {
  fmap_ctx* ctx;
  Plan plan;
  Timing timing;
  void* dev_mem = nullptr;
  BatchDev dev{};
  const int2* d_systems = nullptr;
  const CUtensorMap* d_fmaps = nullptr;
  const TcItem* d_tc_items = nullptr;
  const int32_t* d_tc_cta_first = nullptr;
  const TcRedGroup* d_tc_groups = nullptr;
  const CUtensorMap* d_phimaps_fwd = nullptr;
  const CUtensorMap* d_massmaps = nullptr;
  const CUtensorMap* d_dfmaps = nullptr;
  const CUtensorMap* d_phimaps_bwd = nullptr;
  const TcBwdItem* d_bw_items = nullptr;
  const int32_t* d_bw_cta_first = nullptr;
  const TcBwdGroup* d_bw_groups = nullptr;
  const AdjItem* d_adj_items = nullptr;
  const AdjItem* d_loss_items = nullptr;
  int sm_count = 152;
};

namespace {

// Brackets one kernel launch with CUDA events on its stream when timing is on.
struct TimedScope {
  fmap_batch* b;
  cudaStream_t st;
  int idx = -1;
  TimedScope(fmap_batch* batch, int kind, cudaStream_t stream) : b(batch), st(stream) {
    Timing& t = b->timing;
    if (!t.on || t.used >= kMaxTimedLaunches) return;
    const int i = t.used;
    while ((int)t.ev.size() < 2 * (i + 1)) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      t.ev.push_back(e);
    }
    if ((int)t.kind.size() < i + 1) t.kind.resize(i + 1);
    t.kind[i] = kind;
    if (cudaEventRecord(t.ev[2 * i], st) != cudaSuccess) return;
    idx = i;
    t.used = i + 1;
  }
  ~TimedScope() {
    if (idx >= 0) cudaEventRecord(b->timing.ev[2 * idx + 1], st);
  }
};

}  // namespace

namespace fmap {
// defined in k_overlap.cu
cudaError_t launch_overlap_metrics(const float* scores, const uint8_t* labels, const int64_t* seg_off, int n_seg,
                                   int64_t max_len, float thr, int64_t* counts, double* metrics, cudaStream_t st);
}  // namespace fmap

extern "C" {

const char* fmap_version(void) { return "fmap-gb300 0.1 (sm_103a)"; }

const char* fmap_error_string(int32_t code) {
  switch (code & 0xff) {
    case FMAP_OK: return "ok";
    case FMAP_ERR_INVALID_ARG: return "invalid argument";
    case FMAP_ERR_UNSUPPORTED: return "unsupported size or alignment";
    case FMAP_ERR_CUDA: return "CUDA error";
    case FMAP_ERR_NOT_SPD: return "row system not positive definite";
    case FMAP_ERR_NONFINITE: return "non-finite result";
    case FMAP_ERR_TIMEOUT: return "device-side wait timed out";
    case FMAP_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    default: return "unknown error";
  }
}

const char* fmap_last_cuda_error(void) { return g_last_cuda_error; }


int32_t fmap_overlap_metrics(const float* scores, const uint8_t* labels, const int64_t* seg_offsets,
                             int32_t n_segments, int64_t max_segment_len, float threshold, int64_t* counts,
                             double* metrics, void* stream) {
  if (n_segments < 0 || max_segment_len < 0 || !std::isfinite(threshold)) return FMAP_ERR_INVALID_ARG;
  if (n_segments == 0) return FMAP_OK;
  if (!seg_offsets || !counts || (max_segment_len > 0 && (!scores || !labels))) return FMAP_ERR_INVALID_ARG;
  if (n_segments > 65535) return FMAP_ERR_UNSUPPORTED;
  const cudaError_t e = launch_overlap_metrics(scores, labels, seg_offsets, n_segments, max_segment_len, threshold,
                                               counts, metrics, static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? FMAP_OK : cuda_fail(e, "overlap metrics");
}

int32_t fmap_default_options(fmap_options* opt) {
  if (!opt) return FMAP_ERR_INVALID_ARG;
  std::memset(opt, 0, sizeof(*opt));   // tuning knobs: 0 = built-in choice
  opt->precision = FMAP_PREC_FP32;
  opt->ir_steps = 1;
  opt->hi_gram_min_k = 200;
  opt->store_factors_max_k = kMaxK;
  opt->adjoint_ir_steps = 0;
  return FMAP_OK;
}

int32_t fmap_create(fmap_ctx** out, int32_t device, const fmap_options* opt) {
  if (!out) return FMAP_ERR_INVALID_ARG;
  *out = nullptr;
  if (device < 0) return FMAP_ERR_INVALID_ARG;
  fmap_options o;
  if (opt) o = *opt; else fmap_default_options(&o);
  int32_t rc = validate_options(o);
  if (rc) return rc;
  fmap_ctx* c = new (std::nothrow) fmap_ctx;
  if (!c) return FMAP_ERR_INVALID_ARG;
  c->device = device;
  c->opt = o;
  *out = c;
  return FMAP_OK;
}

int32_t fmap_destroy(fmap_ctx* ctx) {
  delete ctx;
  return FMAP_OK;
}

int32_t fmap_plan_sizes(const fmap_options* opt, const fmap_shape_desc* shapes, int32_t n_shapes,
                        const fmap_pair_desc* pairs, int32_t n_pairs, fmap_sizes* out) {
  if (!out) return FMAP_ERR_INVALID_ARG;
  fmap_options o;
  if (opt) o = *opt; else fmap_default_options(&o);
  Plan P;
  int32_t rc = make_plan(o, shapes, n_shapes, pairs, n_pairs, P);
  if (rc) return rc;
  *out = P.sizes;
  return FMAP_OK;
}

int32_t fmap_batch_create(fmap_ctx* ctx, const fmap_shape_desc* shapes, int32_t n_shapes,
                          const fmap_pair_desc* pairs, int32_t n_pairs, fmap_batch** out) {
  if (!ctx || !out) return FMAP_ERR_INVALID_ARG;
  *out = nullptr;
  fmap_batch* b = new (std::nothrow) fmap_batch;
  if (!b) return FMAP_ERR_INVALID_ARG;
  b->ctx = ctx;
  int32_t rc = make_plan(ctx->opt, shapes, n_shapes, pairs, n_pairs, b->plan);
  if (rc) { delete b; return rc; }
  Plan& P = b->plan;
  DeviceGuard dg(ctx->device);
  if (!dg.ok) { delete b; return cuda_fail(cudaErrorInvalidDevice, "cudaSetDevice"); }
  cudaError_t e = solve_set_smem_limits();
  if (e != cudaSuccess) { delete b; return cuda_fail(e, "cudaFuncSetAttribute"); }
  {
    int dev_sms = 0;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    b->sm_count = dev_sms > 0 ? dev_sms : kTcCtas;
  }
  if (ctx->opt.adjoint_kernel != 2 && n_pairs > 0) {
    std::vector<int3> pk(P.pairs.size());
    for (size_t p = 0; p < P.pairs.size(); ++p)
      pk[p] = make_int3(P.pairs[p].k, P.shapes[P.pairs[p].y].k, P.pairs[p].d);
    P.adj.stages = ctx->opt.adjoint_stages;
    P.adj.features = ctx->opt.adjoint_features;
    adjoint_tc_plan(pk, b->sm_count, P.adj);
    adjoint_tc_loss_plan(pk, P.loss_tc);
  }

  // one allocation for every table
  auto bytes_of = [](size_t n, size_t sz) { return (int64_t)align_up((int64_t)(n * sz), 256); };
  const int64_t o_sh = 0;
  const int64_t o_pr = o_sh + bytes_of(P.shapes.size(), sizeof(ShapeDev));
  const int64_t o_sl = o_pr + bytes_of(P.pairs.size(), sizeof(PairDev));
  const int64_t o_sy = o_sl + bytes_of(P.slot_list.size(), sizeof(int64_t));
  const int64_t o_tm = o_sy + bytes_of(P.systems.size(), sizeof(int2));
  const int64_t o_ti = o_tm + bytes_of(P.shapes.size(), sizeof(CUtensorMap));
  const int64_t o_to = o_ti + bytes_of(P.tc_items.size(), sizeof(TcItem));
  const int64_t o_tg = o_to + bytes_of(P.tc_cta_first.size(), sizeof(int32_t));
  const int64_t o_fp = o_tg + bytes_of(P.tc_groups.size(), sizeof(TcRedGroup));
  const int64_t o_mm = o_fp + bytes_of(P.shapes.size(), sizeof(CUtensorMap));
  const int64_t o_dm = o_mm + bytes_of(P.shapes.size(), sizeof(CUtensorMap));
  const int64_t o_pb = o_dm + bytes_of(P.shapes.size(), sizeof(CUtensorMap));
  const int64_t o_bi = o_pb + bytes_of(P.shapes.size(), sizeof(CUtensorMap));
  const int64_t o_bo = o_bi + bytes_of(P.bw_items.size(), sizeof(TcBwdItem));
  const int64_t o_bg = o_bo + bytes_of(P.bw_cta_first.size(), sizeof(int32_t));
  const int64_t o_ai = o_bg + bytes_of(P.bw_groups.size(), sizeof(TcBwdGroup));
  const int64_t o_li = o_ai + bytes_of(P.adj.items.size(), sizeof(AdjItem));
  const int64_t total = o_li + bytes_of(P.loss_tc.items.size(), sizeof(AdjItem)) + 256;
  e = cudaMalloc(&b->dev_mem, (size_t)total);
  if (e != cudaSuccess) { delete b; return cuda_fail(e, "cudaMalloc(batch tables)"); }
  char* base = static_cast<char*>(b->dev_mem);
  std::vector<char> host((size_t)total, 0);
  auto put = [&](int64_t off, const void* src, size_t n) { if (n) std::memcpy(host.data() + off, src, n); };
  put(o_sh, P.shapes.data(), P.shapes.size() * sizeof(ShapeDev));
  put(o_pr, P.pairs.data(), P.pairs.size() * sizeof(PairDev));
  put(o_sl, P.slot_list.data(), P.slot_list.size() * sizeof(int64_t));
  put(o_sy, P.systems.data(), P.systems.size() * sizeof(int2));
  put(o_ai, P.adj.items.data(), P.adj.items.size() * sizeof(AdjItem));
  put(o_li, P.loss_tc.items.data(), P.loss_tc.items.size() * sizeof(AdjItem));
  if (n_shapes > 0) {
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) { cudaFree(b->dev_mem); delete b; return cuda_fail(cudaErrorNotSupported, "cuTensorMapEncodeTiled"); }
    for (int s = 0; s < n_shapes; ++s) {
      const ShapeDev& sd = P.shapes[s];
      // features: BF16 box 64 features x 64 vertices, or FP32 box 32 features x 32 vertices
      // (a 128-byte row either way); the basis and mass boxes follow the stage length
      const cuuint32_t sv = P.tc32 ? 32 : 64;
      CUtensorMap m;
      cuuint64_t gdim[2] = {(cuuint64_t)sd.d, (cuuint64_t)sd.n};
      cuuint64_t gstride[1] = {(cuuint64_t)sd.ld_feat * (P.tc32 ? 4 : 2)};
      cuuint32_t box[2] = {P.tc32 ? 32u : 64u, sv};
      cuuint32_t estr[2] = {1, 1};
      CUresult r = encode(&m, P.tc32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                          const_cast<void*>(sd.feat), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) {
        cudaFree(b->dev_mem); delete b;
        std::snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "cuTensorMapEncodeTiled failed (%d)", (int)r);
        return FMAP_ERR_CUDA;
      }
      put(o_tm + s * (int64_t)sizeof(CUtensorMap), &m, sizeof(m));
      // FP32 basis, box 32 basis x sv vertices (the forward projection's tiles and, at 64
      // vertices, the halves of the backward projection's 128-vertex tiles)
      CUtensorMap pm;
      cuuint64_t pdim[2] = {(cuuint64_t)sd.k, (cuuint64_t)sd.n};
      cuuint64_t pstride[1] = {(cuuint64_t)sd.ld_phi * 4};
      cuuint32_t fbox[2] = {32, sv};
      r = encode(&pm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(sd.phi), pdim, pstride, fbox, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) {
        cudaFree(b->dev_mem); delete b;
        std::snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "cuTensorMapEncodeTiled(phi fwd) failed (%d)", (int)r);
        return FMAP_ERR_CUDA;
      }
      put(o_fp + s * (int64_t)sizeof(CUtensorMap), &pm, sizeof(pm));
      // mass: 1-D, box of sv
      CUtensorMap mm;
      cuuint64_t mdim[1] = {(cuuint64_t)sd.n};
      cuuint64_t mstride[1] = {4};
      cuuint32_t mbox[1] = {sv};
      cuuint32_t mestr[1] = {1};
      r = encode(&mm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 1, const_cast<float*>(sd.mass), mdim, mstride, mbox, mestr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) {
        cudaFree(b->dev_mem); delete b;
        std::snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "cuTensorMapEncodeTiled(mass) failed (%d)", (int)r);
        return FMAP_ERR_CUDA;
      }
      put(o_mm + s * (int64_t)sizeof(CUtensorMap), &mm, sizeof(mm));
      // FP32 basis, box 32 basis x 64 vertices: the halves of the backward projection's
      // 128-vertex tiles
      CUtensorMap pb;
      cuuint32_t bbox[2] = {32, 64};
      r = encode(&pb, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(sd.phi), pdim, pstride, bbox, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) {
        cudaFree(b->dev_mem); delete b;
        std::snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "cuTensorMapEncodeTiled(phi bwd) failed (%d)", (int)r);
        return FMAP_ERR_CUDA;
      }
      put(o_pb + s * (int64_t)sizeof(CUtensorMap), &pb, sizeof(pb));
      // dF (BF16 or FP32): box 16 features x 32 vertices, stored by the backward projection
      CUtensorMap dm;
      std::memset(&dm, 0, sizeof(dm));
      if (sd.dfeat && (P.tc_bwd || P.tc_bwd32)) {
        cuuint32_t dbox[2] = {16, 32};
        r = encode(&dm, P.tc_bwd32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, sd.dfeat,
                   gdim, gstride, dbox, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
          cudaFree(b->dev_mem); delete b;
          std::snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "cuTensorMapEncodeTiled(dF) failed (%d)", (int)r);
          return FMAP_ERR_CUDA;
        }
      }
      put(o_dm + s * (int64_t)sizeof(CUtensorMap), &dm, sizeof(dm));
    }
    put(o_bi, P.bw_items.data(), P.bw_items.size() * sizeof(TcBwdItem));
    put(o_bo, P.bw_cta_first.data(), P.bw_cta_first.size() * sizeof(int32_t));
    put(o_bg, P.bw_groups.data(), P.bw_groups.size() * sizeof(TcBwdGroup));
    if (!P.bw_items.empty()) {
      e = P.tc_bwd32 ? project_bwd_tc32_set_smem(P.bw_smem) : project_bwd_tc_set_smem(P.bw_smem);
      if (e != cudaSuccess) { cudaFree(b->dev_mem); delete b; return cuda_fail(e, "cudaFuncSetAttribute(project bwd)"); }
    }
    put(o_ti, P.tc_items.data(), P.tc_items.size() * sizeof(TcItem));
    put(o_to, P.tc_cta_first.data(), P.tc_cta_first.size() * sizeof(int32_t));
    put(o_tg, P.tc_groups.data(), P.tc_groups.size() * sizeof(TcRedGroup));
    e = P.tc32 ? project_tc32_set_smem(P.tc_smem) : project_tc_set_smem(P.tc_smem);
    if (e != cudaSuccess) { cudaFree(b->dev_mem); delete b; return cuda_fail(e, "cudaFuncSetAttribute(project)"); }
  }
  e = cudaMemcpy(b->dev_mem, host.data(), (size_t)total, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { cudaFree(b->dev_mem); delete b; return cuda_fail(e, "cudaMemcpy(batch tables)"); }
  b->dev.shapes = reinterpret_cast<const ShapeDev*>(base + o_sh);
  b->dev.pairs = reinterpret_cast<const PairDev*>(base + o_pr);
  b->dev.slot_list = reinterpret_cast<const int64_t*>(base + o_sl);
  b->dev.n_shapes = n_shapes;
  b->dev.n_pairs = n_pairs;
  b->dev.feat_bf16 = ctx->opt.precision == FMAP_PREC_BF16 ? 1 : 0;
  b->dev.ir_steps = ctx->opt.ir_steps;
  b->dev.ir_steps_adj = ctx->opt.adjoint_ir_steps;
  b->d_systems = reinterpret_cast<const int2*>(base + o_sy);
  b->d_fmaps = reinterpret_cast<const CUtensorMap*>(base + o_tm);
  b->d_tc_items = reinterpret_cast<const TcItem*>(base + o_ti);
  b->d_tc_cta_first = reinterpret_cast<const int32_t*>(base + o_to);
  b->d_tc_groups = reinterpret_cast<const TcRedGroup*>(base + o_tg);
  b->d_phimaps_fwd = reinterpret_cast<const CUtensorMap*>(base + o_fp);
  b->d_massmaps = reinterpret_cast<const CUtensorMap*>(base + o_mm);
  b->d_dfmaps = reinterpret_cast<const CUtensorMap*>(base + o_dm);
  b->d_phimaps_bwd = reinterpret_cast<const CUtensorMap*>(base + o_pb);
  b->d_bw_items = reinterpret_cast<const TcBwdItem*>(base + o_bi);
  b->d_bw_cta_first = reinterpret_cast<const int32_t*>(base + o_bo);
  b->d_bw_groups = reinterpret_cast<const TcBwdGroup*>(base + o_bg);
  b->d_adj_items = reinterpret_cast<const AdjItem*>(base + o_ai);
  b->d_loss_items = reinterpret_cast<const AdjItem*>(base + o_li);
  *out = b;
  return FMAP_OK;
}

int32_t fmap_batch_destroy(fmap_batch* b) {
  if (!b) return FMAP_OK;
  if (b->dev_mem || !b->timing.ev.empty()) {
    DeviceGuard dg(b->ctx->device);
    if (b->dev_mem) cudaFree(b->dev_mem);
    for (cudaEvent_t e : b->timing.ev) cudaEventDestroy(e);
  }
  delete b;
  return FMAP_OK;
}

int32_t fmap_batch_sizes(const fmap_batch* b, fmap_sizes* out) {
  if (!b || !out) return FMAP_ERR_INVALID_ARG;
  *out = b->plan.sizes;
  return FMAP_OK;
}

int32_t fmap_batch_offsets(const fmap_batch* b, int64_t* a_offsets, int64_t* c_offsets) {
  if (!b) return FMAP_ERR_INVALID_ARG;
  if (a_offsets) std::memcpy(a_offsets, b->plan.a_off.data(), b->plan.a_off.size() * sizeof(int64_t));
  if (c_offsets) std::memcpy(c_offsets, b->plan.c_off.data(), b->plan.c_off.size() * sizeof(int64_t));
  return FMAP_OK;
}

int32_t fmap_batch_set_timing(fmap_batch* b, int32_t enable) {
  if (!b) return FMAP_ERR_INVALID_ARG;
  b->timing.on = enable != 0;
  b->timing.used = 0;
  return FMAP_OK;
}

int32_t fmap_batch_read_timing(fmap_batch* b, float* ms, int32_t* launches, int32_t n_kinds) {
  if (!b || !ms || !launches || n_kinds < FMAP_KIND_COUNT) return FMAP_ERR_INVALID_ARG;
  for (int i = 0; i < n_kinds; ++i) { ms[i] = 0.f; launches[i] = 0; }
  Timing& t = b->timing;
  if (t.used == 0) return FMAP_OK;
  DeviceGuard dg(b->ctx->device);
  cudaError_t e = cudaEventSynchronize(t.ev[2 * t.used - 1]);
  if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize(timing)");
  for (int i = 0; i < t.used; ++i) {
    float x = 0.f;
    e = cudaEventElapsedTime(&x, t.ev[2 * i], t.ev[2 * i + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
    ms[t.kind[i]] += x;
    launches[t.kind[i]] += 1;
  }
  t.used = 0;
  return FMAP_OK;
}

static int32_t check_ws(void* ws, size_t ws_bytes, int64_t need) {
  if (need == 0) return FMAP_OK;
  if (!ws || !aligned(ws, 256) || (int64_t)ws_bytes < need) return FMAP_ERR_WORKSPACE;
  return FMAP_OK;
}

int32_t fmap_project(fmap_batch* b, float* a_out, void* ws, size_t ws_bytes, void* stream) {
  if (!b) return FMAP_ERR_INVALID_ARG;
  if (b->plan.sizes.n_shapes == 0) return FMAP_OK;
  if (!a_out) return FMAP_ERR_INVALID_ARG;
  int32_t rc = check_ws(ws, ws_bytes, b->plan.sizes.ws_bytes);
  if (rc) return rc;
  DeviceGuard dg(b->ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* w = static_cast<float*>(ws);
  cudaError_t e = cudaMemsetAsync(ws, 0, 256, st);   // control words
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(control)");
  const Plan& P = b->plan;
  for (const TcLaunch& L : P.tc_launches) {
    TcProjParams tp{};
    tp.shapes = b->dev.shapes;
    tp.fmaps = b->d_fmaps;
    tp.phimaps = b->d_phimaps_fwd;
    tp.massmaps = b->d_massmaps;
    tp.items = b->d_tc_items;
    tp.cta_first = b->d_tc_cta_first + L.cta_off;
    tp.stages = L.stages;
    tp.f_stage_bytes = L.f_stage;
    tp.p_stage_bytes = L.p_stage;
    tp.tmem_cols = L.tmem_cols;
    tp.ws = w;
    tp.err = static_cast<int*>(ws);
    {
      TimedScope ts(b, FMAP_KIND_PROJECT, st);
      e = P.tc32 ? launch_project_tc32(tp, P.proj_ctas, L.smem, st) : launch_project_tc(tp, P.proj_ctas, L.smem, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "project (tensor cores)");
  }
  {
    TimedScope ts(b, FMAP_KIND_PROJECT_REDUCE, st);
    e = launch_project_tc_reduce(b->dev.shapes, b->d_tc_items, b->d_tc_groups, (int)P.tc_groups.size(),
                                 P.tc_max_group_elems, a_out, w, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "project_reduce");
  return FMAP_OK;
}

int32_t fmap_solve(fmap_batch* b, const float* a, float* c_out, void* saved, int32_t* status, void* ws,
                   size_t ws_bytes, void* stream) {
  if (!b) return FMAP_ERR_INVALID_ARG;
  if (b->plan.sizes.n_pairs == 0) return FMAP_OK;
  if (!a || !c_out) return FMAP_ERR_INVALID_ARG;
  int32_t rc = check_ws(ws, ws_bytes, b->plan.sizes.ws_bytes);
  if (rc) return rc;
  if (saved && !aligned(saved, 256)) return FMAP_ERR_WORKSPACE;
  DeviceGuard dg(b->ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* w = static_cast<float*>(ws);
  cudaError_t e = cudaSuccess;
  if (status) {
    TimedScope ts(b, FMAP_KIND_STATUS, st);
    e = launch_status_clear(status, b->plan.sizes.n_pairs, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "status_clear");
  {
    TimedScope ts(b, FMAP_KIND_GRAM, st);
    e = launch_gram(b->dev, b->plan.max_k, a, w, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "gram");
  for (const auto& g : b->plan.groups) {
    TimedScope ts(b, FMAP_KIND_SOLVE, st);
    e = launch_solve(b->dev, g, b->d_systems, kSolveForward, nullptr, c_out, static_cast<float*>(saved), status, w, st);
    if (e != cudaSuccess) return cuda_fail(e, "solve");
  }
  return FMAP_OK;
}

}  // extern "C"

namespace {

// The adjoint part of the backward pass: dC -> Gamma (adjoint row solves) -> dA (and dD,
// dlambda), written to da.
// A bounded device wait that gave up in a kernel after the row solves (the adjoint GEMMs,
// the backward projection) leaves FMAP_ERR_TIMEOUT in the workspace's control word; this
// turns it into every pair's status (pairs that already hold an error keep it).
__global__ void status_from_control_kernel(const int* ctrl, int32_t* status, int n) {
  const int code = ctrl[0];
  if (code == 0) return;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
    atomicCAS(status + p, 0, code);
}

cudaError_t launch_status_from_control(const void* ws, int32_t* status, int n, cudaStream_t st) {
  if (!status || n <= 0) return cudaSuccess;
  status_from_control_kernel<<<(n + 255) / 256, 256, 0, st>>>(static_cast<const int*>(ws), status, n);
  return cudaGetLastError();
}

int32_t adjoint_impl(fmap_batch* b, const float* d_c, const float* a, const float* c, const void* saved, float* da,
                     float* d_mask, float* d_lambda, int32_t* status, float* w, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (status) {
    TimedScope ts(b, FMAP_KIND_STATUS, st);
    e = launch_status_clear(status, b->plan.sizes.n_pairs, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "status_clear");
  // the adjoint solves read G only to refactor a system whose factor was not saved,
  // or for adjoint refinement steps
  bool need_g = saved == nullptr || b->dev.ir_steps_adj > 0;
  for (const PairDev& pd : b->plan.pairs) need_g = need_g || pd.fac_off < 0;
  if (need_g) {
    TimedScope ts(b, FMAP_KIND_GRAM, st);
    e = launch_gram(b->dev, b->plan.max_k, a, w, st, /*with_r=*/false);
  }
  if (e != cudaSuccess) return cuda_fail(e, "gram");
  for (const auto& g : b->plan.groups) {
    TimedScope ts(b, FMAP_KIND_ADJ_SOLVE, st);
    e = launch_solve(b->dev, g, b->d_systems, kSolveAdjoint, d_c, nullptr,
                     const_cast<float*>(static_cast<const float*>(saved)), status, w, st);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint solve");
  }
  {
    TimedScope ts(b, FMAP_KIND_ADJ_GEMM, st);
    const int ak = b->plan.opt.adjoint_kernel;
    const bool simt = ak == 2 || (ak == 0 && !b->plan.adj.fills_sms);
    e = launch_adjoint_gemms(b->dev, b->plan.max_k, b->plan.max_d, a, c, d_mask, d_lambda, b->plan.row_grads, w,
                             simt, st);
    if (e == cudaSuccess && !simt) e = launch_adjoint_tc(b->dev, b->d_adj_items, b->plan.adj, a, c, w, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "adjoint gemms");
  {
    TimedScope ts(b, FMAP_KIND_GATHER, st);
    e = launch_gather_da(b->dev, (int)b->plan.max_kd, da, w, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "gather dA");
  return FMAP_OK;
}

// dF = diag(M) Phi dA for every shape with a dF buffer: the dA^T images, then the
// tensor-core backward projection.
int32_t project_backward_impl(fmap_batch* b, const float* da, float* w, void* ws, cudaStream_t st) {
  if (b->plan.bw_items.empty()) return FMAP_OK;
  const Plan& P = b->plan;
  cudaError_t e;
  {
    TimedScope ts(b, FMAP_KIND_GATHER, st);
    e = P.tc_bwd32
            ? launch_build_dat_image32(b->dev.shapes, b->d_bw_groups, (int)P.bw_groups.size(), P.bw_max_img, da, w, st)
            : launch_build_dat_image(b->dev.shapes, b->d_bw_groups, (int)P.bw_groups.size(), P.bw_max_img, da, w, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "dA image");
  TcBwdParams bp{};
  bp.shapes = b->dev.shapes;
  bp.phimaps = b->d_phimaps_bwd;
  bp.dfmaps = b->d_dfmaps;
  bp.items = b->d_bw_items;
  bp.cta_first = b->d_bw_cta_first;
  bp.stages = P.bw_stages;
  bp.b_bytes_max = P.bw_b_bytes;
  bp.tmem_cols = P.tc_bwd32 ? 128 : 256;   // two accumulators of <= 64 or <= 128 columns
  bp.ws = w;
  bp.err = static_cast<int*>(ws);
  {
    TimedScope ts(b, FMAP_KIND_PROJECT_BWD, st);
    e = P.tc_bwd32 ? launch_project_bwd_tc32(bp, P.bwd_ctas, P.bw_smem, st)
                   : launch_project_bwd_tc(bp, P.bwd_ctas, P.bw_smem, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "project backward");
  return FMAP_OK;
}

}  // namespace

extern "C" {

int32_t fmap_solve_backward(fmap_batch* b, const float* d_c, const float* a, const float* c, const void* saved,
                            float* d_a, float* d_mask, float* d_lambda, int32_t* status, void* ws,
                            size_t ws_bytes, void* stream) {
  if (!b) return FMAP_ERR_INVALID_ARG;
  if (b->plan.sizes.n_pairs == 0) return FMAP_OK;
  if (!d_c || !a || !c) return FMAP_ERR_INVALID_ARG;
  int32_t rc = check_ws(ws, ws_bytes, b->plan.sizes.ws_bwd_bytes);
  if (rc) return rc;
  if (saved && !aligned(saved, 256)) return FMAP_ERR_WORKSPACE;
  DeviceGuard dg(b->ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* w = static_cast<float*>(ws);
  float* da = d_a ? d_a : w + b->plan.da_int_off;
  rc = adjoint_impl(b, d_c, a, c, saved, da, d_mask, d_lambda, status, w, st);
  if (rc) return rc;
  rc = project_backward_impl(b, da, w, ws, st);
  if (rc) return rc;
  cudaError_t e;
  {
    TimedScope ts(b, FMAP_KIND_STATUS, st);
    e = launch_status_from_control(ws, status, b->plan.sizes.n_pairs, st);
  }
  return e == cudaSuccess ? FMAP_OK : cuda_fail(e, "status");
}

int32_t fmap_adjoint(fmap_batch* b, const float* d_c, const float* a, const float* c, const void* saved, float* d_a,
                     float* d_mask, float* d_lambda, int32_t* status, void* ws, size_t ws_bytes, void* stream) {
  if (!b) return FMAP_ERR_INVALID_ARG;
  if (b->plan.sizes.n_pairs == 0) return FMAP_OK;
  if (!d_c || !a || !c || !d_a) return FMAP_ERR_INVALID_ARG;
  int32_t rc = check_ws(ws, ws_bytes, b->plan.sizes.ws_bwd_bytes);
  if (rc) return rc;
  if (saved && !aligned(saved, 256)) return FMAP_ERR_WORKSPACE;
  DeviceGuard dg(b->ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc = adjoint_impl(b, d_c, a, c, saved, d_a, d_mask, d_lambda, status, static_cast<float*>(ws), st);
  if (rc) return rc;
  cudaError_t e;
  {
    TimedScope ts(b, FMAP_KIND_STATUS, st);
    e = launch_status_from_control(ws, status, b->plan.sizes.n_pairs, st);
  }
  return e == cudaSuccess ? FMAP_OK : cuda_fail(e, "status");
}

int32_t fmap_project_backward(fmap_batch* b, const float* d_a, int32_t* status, void* ws, size_t ws_bytes,
                              void* stream) {
  if (!b) return FMAP_ERR_INVALID_ARG;
  if (b->plan.sizes.n_pairs == 0) return FMAP_OK;
  if (!d_a) return FMAP_ERR_INVALID_ARG;
  int32_t rc = check_ws(ws, ws_bytes, b->plan.sizes.ws_bwd_bytes);
  if (rc) return rc;
  DeviceGuard dg(b->ctx->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc = project_backward_impl(b, d_a, static_cast<float*>(ws), ws, st);
  if (rc) return rc;
  cudaError_t e;
  {
    TimedScope ts(b, FMAP_KIND_STATUS, st);
    e = launch_status_from_control(ws, status, b->plan.sizes.n_pairs, st);
  }
  return e == cudaSuccess ? FMAP_OK : cuda_fail(e, "status");
}

int32_t fmap_loss_orth(fmap_batch* b, const float* c, const float* c_gt, float* loss, float* d_c, void* ws,
                       size_t ws_bytes, void* stream) {
  if (!b) return FMAP_ERR_INVALID_ARG;
  if (b->plan.sizes.n_pairs == 0) return FMAP_OK;
  if (!c || !c_gt || (!loss && !d_c)) return FMAP_ERR_INVALID_ARG;
  int32_t rc = check_ws(ws, ws_bytes, b->plan.sizes.ws_bytes);
  if (rc) return rc;
  DeviceGuard dg(b->ctx->device);
  cudaError_t e;
  {
    TimedScope ts(b, FMAP_KIND_LOSS, static_cast<cudaStream_t>(stream));
    // the GEMMs on the tensor cores when the adjoint's run there (both need dL/dC: its tiles
    // also carry ||C - C_gt||^2), else the FP32 FMA tiles
    const int ak = b->plan.opt.adjoint_kernel;
    const bool tc = d_c && !b->plan.loss_tc.items.empty() && (ak == 1 || (ak == 0 && b->plan.adj.fills_sms));
    float* w = static_cast<float*>(ws);
    e = tc ? launch_loss_tc(b->dev, b->d_loss_items, b->plan.loss_tc, c, c_gt, loss, d_c, w, w + b->plan.loss_part_off,
                            static_cast<cudaStream_t>(stream))
           : launch_loss_orth(b->dev, b->plan.max_k, c, c_gt, loss, d_c, w, w + b->plan.loss_part_off,
                              static_cast<cudaStream_t>(stream));
  }
  if (e != cudaSuccess) return cuda_fail(e, "loss");
  return FMAP_OK;
}

}  // extern "C"
