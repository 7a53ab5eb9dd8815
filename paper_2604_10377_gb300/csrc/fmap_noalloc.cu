// Allocation-free solve of one shape pair.
//
// fmap_solve_pair_noalloc runs the same Gram and row-system Cholesky kernels as
// fmap_solve, for a single pair given directly by its two spectral descriptor
// matrices, but takes all of its scratch from a fixed device array defined in this
// file instead of a caller workspace, and it never allocates device memory. It is
// meant for callers that cannot allocate device memory when they solve: code that
// runs while a memory pool it does not own is frozen, real-time threads that must
// not enter the allocator, or plug-ins whose host application owns all device
// memory. Such callers still pass their inputs and outputs.
//
// The scratch array lives on every GPU that loads the library until the process
// exits (kScratchBytes per device). Every call shares it and it keeps the last
// call's contents; the set-up kernel of each call clears what must start at zero.
// Calls that overlap on the GPU (different streams, or a graph replayed while
// another call runs) race on the array and must not be issued.
#include <mutex>

#include "fmap_internal.cuh"

namespace fmap {
namespace {

constexpr size_t kScratchBytes = size_t(2) << 20;   // 2 MiB per device
constexpr int kNoallocMaxK = 256;                     // the layout of one pair fits the scratch
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};
bool g_setup_done[kMaxDevices] = {};

constexpr int64_t kAlign = 64;   // floats (256 bytes)
int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Scratch layout in floats: [0, 64) control words, then the descriptor tables,
// then G, R and the (hi, lo) Gram.
struct Layout {
  int64_t shapes, pair, systems, g, r, ghl, end;
};

Layout layout_for(int k, bool hi) {
  Layout L;
  int64_t cur = kAlign;
  L.shapes = cur; cur = align_up(cur + (int64_t)(2 * sizeof(ShapeDev) + 3) / 4, kAlign);
  L.pair = cur; cur = align_up(cur + (int64_t)(sizeof(PairDev) + 3) / 4, kAlign);
  L.systems = cur; cur = align_up(cur + 2 * (int64_t)k, kAlign);
  L.g = cur; cur = align_up(cur + gram_floats(k), kAlign);
  L.r = cur; cur = align_up(cur + (int64_t)k * k, kAlign);
  if (hi) { L.ghl = cur; cur = align_up(cur + 2 * (int64_t)k * k, kAlign); } else { L.ghl = -1; }
  L.end = cur;
  return L;
}

struct SetupArgs {
  const float* a_x;
  const float* a_y;
  int32_t k, d;
  const float* evals_x;
  const float* evals_y;
  const float* mask;
  float lambda;
  int32_t hi;
  Layout lay;
};

// Writes the descriptor tables of the single pair into the scratch array and
// clears the control word the solve reads.
__global__ void noalloc_setup_kernel(SetupArgs s, float* scratch) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0) {
    reinterpret_cast<int*>(scratch)[0] = 0;
    ShapeDev* sh = reinterpret_cast<ShapeDev*>(scratch + s.lay.shapes);
    for (int j = 0; j < 2; ++j) {
      ShapeDev v = {};
      v.n = 0;
      v.k = s.k;
      v.d = s.d;
      v.evals = j == 0 ? s.evals_x : s.evals_y;
      // both descriptor matrices are addressed from a_x: A_y sits (a_y - a_x) / 4 floats away
      v.a_off = j == 0 ? 0
                       : (int64_t)(reinterpret_cast<uintptr_t>(s.a_y) - reinterpret_cast<uintptr_t>(s.a_x)) /
                             (int64_t)sizeof(float);
      sh[j] = v;
    }
    PairDev p = {};
    p.x = 0;
    p.y = 1;
    p.k = s.k;
    p.d = s.d;
    p.lam = s.lambda;
    p.hi_gram = s.hi;
    p.mask = s.mask;
    p.c_off = 0;
    p.g_off = s.lay.g;
    p.r_off = s.lay.r;
    p.g64_off = s.hi ? s.lay.ghl / 2 : -1;
    p.fac_off = -1;
    *reinterpret_cast<PairDev*>(scratch + s.lay.pair) = p;
  }
  int2* sys = reinterpret_cast<int2*>(scratch + s.lay.systems);
  for (int i = t; i < s.k; i += gridDim.x * blockDim.x) sys[i] = make_int2(0, i);
}

// Once per device, with that device current: the device address of the scratch
// array and the shared-memory limits of the solve kernels.
int32_t setup_device(int dev, float** scratch) {
  if (dev < 0 || dev >= kMaxDevices) return FMAP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_setup_done[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) return FMAP_ERR_CUDA;
    if (solve_set_smem_limits() != cudaSuccess) return FMAP_ERR_CUDA;
    g_scratch_addr[dev] = ptr;
    g_setup_done[dev] = true;
  }
  *scratch = static_cast<float*>(g_scratch_addr[dev]);
  return FMAP_OK;
}

}  // namespace
}  // namespace fmap

using namespace fmap;

extern "C" FMAP_API int32_t fmap_solve_pair_noalloc(const float* a_x, const float* a_y, int32_t k, int32_t d,
                                                    const float* evals_x, const float* evals_y, const float* mask,
                                                    float lambda, int32_t ir_steps, float* c_out, int32_t* status,
                                                    void* stream) {
  if (!a_x || !a_y || !c_out) return FMAP_ERR_INVALID_ARG;
  if (k < 1 || d < 1 || !(lambda >= 0.f) || ir_steps < 0 || ir_steps > 3) return FMAP_ERR_INVALID_ARG;
  if (!mask && (!evals_x || !evals_y)) return FMAP_ERR_INVALID_ARG;
  if (k > kNoallocMaxK) return FMAP_ERR_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(a_x) | reinterpret_cast<uintptr_t>(a_y)) % 4 != 0) return FMAP_ERR_UNSUPPORTED;
  const bool hi = k >= 200;
  const Layout lay = layout_for(k, hi);
  if ((size_t)lay.end * sizeof(float) > kScratchBytes) return FMAP_ERR_UNSUPPORTED;

  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return FMAP_ERR_CUDA;
  float* scratch = nullptr;
  int32_t rc = setup_device(dev, &scratch);
  if (rc) return rc;

  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SetupArgs sa;
  sa.a_x = a_x; sa.a_y = a_y; sa.k = k; sa.d = d;
  sa.evals_x = evals_x; sa.evals_y = evals_y; sa.mask = mask; sa.lambda = lambda;
  sa.hi = hi ? 1 : 0;
  sa.lay = lay;
  noalloc_setup_kernel<<<(k + 255) / 256, 256, 0, st>>>(sa, scratch);
  if (cudaGetLastError() != cudaSuccess) return FMAP_ERR_CUDA;

  BatchDev b{};
  b.shapes = reinterpret_cast<const ShapeDev*>(scratch + lay.shapes);
  b.pairs = reinterpret_cast<const PairDev*>(scratch + lay.pair);
  b.slot_list = nullptr;
  b.n_shapes = 2;
  b.n_pairs = 1;
  b.feat_bf16 = 0;
  b.ir_steps = ir_steps;
  if (launch_status_clear(status, 1, st) != cudaSuccess) return FMAP_ERR_CUDA;
  if (launch_gram(b, k, a_x, scratch, st) != cudaSuccess) return FMAP_ERR_CUDA;
  SolveGroup g{};
  g.first = 0;
  g.count = k;
  g.kmax = k;
  g.threads = k <= 64 ? 64 : (k <= 128 ? 128 : 256);
  if (launch_solve(b, g, reinterpret_cast<const int2*>(scratch + lay.systems), kSolveForward, nullptr, c_out,
                   nullptr, status, scratch, st) != cudaSuccess)
    return FMAP_ERR_CUDA;
  return FMAP_OK;
}
