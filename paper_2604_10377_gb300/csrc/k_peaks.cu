// Peak-throughput loops used as roofline denominators (instrumentation; no counterpart
// in the paper): FP32 and FP64 FMA on the SIMT pipes, and tcgen05 MMA of kind::tf32 and
// kind::f16 (BF16) on the tensor cores. Each launch does a fixed, documented amount of
// arithmetic; the caller times it with CUDA events.
//
//   FMA loops  every thread (512 per CTA) runs kChains = 8 independent multiply-add chains
//              for `iters` rounds of 4 steps: flops = blocks x 512 x iters x 4 x 8 x 2.
//   MMA loops  one CTA per SM; thread 0 issues `iters` MMAs of M = 128, N = 256 into a
//              TMEM accumulator (K = 8 for TF32, 16 for BF16; operand tiles of zeros in
//              shared memory, 128-byte swizzle, K-major), then waits on one commit with a
//              bounded wait: flops = blocks x iters x 2 x 128 x 256 x K.
#include "fmap_internal.cuh"
#include "tc_ptx.cuh"

namespace fmap {
namespace {

constexpr int kChains = 8;
constexpr int kMmaThreads = 128;
constexpr uint32_t kMmaN = 256;
constexpr uint32_t kATileBytes = 128 * 128;        // 128 rows x 128 bytes
constexpr uint32_t kBTileBytes = kMmaN * 128;      // 256 rows x 128 bytes
// more shared memory than the tiles need, so that one CTA holds an SM (one accumulator per SM)
constexpr uint32_t kMmaSmem = 120 * 1024;

__global__ void fma32_loop_kernel(int64_t iters, float mul, float add, float* sink) {
  float x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = (float)(threadIdx.x + j) * 1e-3f;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], mul, add);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  if (s == 12345.678f) sink[blockIdx.x] = s;   // keeps the chains alive; never true in practice
}

// The same chains as pairs of FP32 lanes through the packed fma.rn.f32x2 instruction.
__global__ void fma32x2_loop_kernel(int64_t iters, float mul, float add, float* sink) {
  uint64_t x[kChains / 2];
  const float2 m2 = make_float2(mul, mul), a2 = make_float2(add, add);
  const uint64_t mm = *reinterpret_cast<const uint64_t*>(&m2), aa = *reinterpret_cast<const uint64_t*>(&a2);
#pragma unroll
  for (int j = 0; j < kChains / 2; ++j) {
    const float2 v = make_float2((float)(threadIdx.x + 2 * j) * 1e-3f, (float)(threadIdx.x + 2 * j + 1) * 1e-3f);
    x[j] = *reinterpret_cast<const uint64_t*>(&v);
  }
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int j = 0; j < kChains / 2; ++j) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[j]) : "l"(mm), "l"(aa));
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains / 2; ++j) {
    const float2 v = *reinterpret_cast<const float2*>(&x[j]);
    s += v.x + v.y;
  }
  if (s == 12345.678f) sink[blockIdx.x] = s;
}

__global__ void fma64_loop_kernel(int64_t iters, double mul, double add, float* sink) {
  double x[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) x[j] = (double)(threadIdx.x + j) * 1e-3;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) x[j] = fma(x[j], mul, add);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += x[j];
  if (s == 12345.678) sink[blockIdx.x] = (float)s;
}

// bf16 = 0: kind::tf32 (K = 8 per MMA); 1: kind::f16 with BF16 operands (K = 16).
__global__ void __launch_bounds__(kMmaThreads, 1) mma_loop_kernel(int64_t iters, int bf16, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = sA + kATileBytes;
  uint64_t* done = reinterpret_cast<uint64_t*>(sB + kBTileBytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  __shared__ int s_abort;
  const int warp = threadIdx.x >> 5;
  for (uint32_t i = threadIdx.x; i < (kATileBytes + kBTileBytes) / 16; i += kMmaThreads)
    reinterpret_cast<uint4*>(sA)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (threadIdx.x == 0) {
    s_abort = 0;
    tc::mbar_init(done, 1);
    tc::fence_mbar_init();
  }
  tc::fence_proxy_async_smem();
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, kMmaN);
    tc::tmem_relinquish();
    tc::tc_fence_before();
  }
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t d = *tmem_slot;
  if (threadIdx.x == 0) {
    const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
    const uint32_t idesc = bf16 ? tc::idesc_bf16_f32(128, kMmaN, 0, 0) : tc::idesc_tf32(128, kMmaN);
    for (int64_t i = 0; i < iters; ++i) {
      const uint32_t ks = (uint32_t)(i & 3) * 32u;   // four K-steps of 32 bytes per 128-byte row
      const uint64_t ad = tc::smem_desc(a0 + ks, 16, 1024, tc::kLayoutSW128);
      const uint64_t bd = tc::smem_desc(b0 + ks, 16, 1024, tc::kLayoutSW128);
      if (bf16)
        tc::mma_bf16(d, ad, bd, idesc, i != 0 ? 1u : 0u);
      else
        tc::mma_tf32(d, ad, bd, idesc, i != 0 ? 1u : 0u);
    }
    tc::mma_commit(done);
    if (!tc::mbar_wait(done, 0, &s_abort)) atomicExch(err, (int)FMAP_ERR_TIMEOUT);
  }
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_dealloc(d, kMmaN);
}

}  // namespace
}  // namespace fmap

using namespace fmap;

extern "C" FMAP_API int32_t fmap_peak_loop(int32_t kind, int32_t blocks, int64_t iters, void* sink,
                                           double* flops_per_launch, void* stream) {
  if (blocks < 1 || blocks > 65535 || iters < 1 || sink == nullptr || flops_per_launch == nullptr)
    return FMAP_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int threads = 512;
  switch (kind) {
    case FMAP_PEAK_FP32_FMA:
      *flops_per_launch = (double)blocks * threads * (double)iters * 4.0 * kChains * 2.0;
      fma32_loop_kernel<<<blocks, threads, 0, st>>>(iters, 0.9999f, 1e-4f, static_cast<float*>(sink));
      break;
    case FMAP_PEAK_FP32X2_FMA:
      *flops_per_launch = (double)blocks * threads * (double)iters * 4.0 * kChains * 2.0;
      fma32x2_loop_kernel<<<blocks, threads, 0, st>>>(iters, 0.9999f, 1e-4f, static_cast<float*>(sink));
      break;
    case FMAP_PEAK_FP64_FMA:
      *flops_per_launch = (double)blocks * threads * (double)iters * 4.0 * kChains * 2.0;
      fma64_loop_kernel<<<blocks, threads, 0, st>>>(iters, 0.9999, 1e-4, static_cast<float*>(sink));
      break;
    case FMAP_PEAK_TF32_MMA:
    case FMAP_PEAK_BF16_MMA: {
      const int bf = kind == FMAP_PEAK_BF16_MMA ? 1 : 0;
      if (cudaFuncSetAttribute(mma_loop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMmaSmem) !=
          cudaSuccess)
        return FMAP_ERR_CUDA;
      *flops_per_launch = (double)blocks * (double)iters * 2.0 * 128.0 * kMmaN * (bf ? 16.0 : 8.0);
      mma_loop_kernel<<<blocks, kMmaThreads, kMmaSmem, st>>>(iters, bf, static_cast<int*>(sink));
      break;
    }
    default:
      return FMAP_ERR_INVALID_ARG;
  }
  return cudaGetLastError() == cudaSuccess ? FMAP_OK : FMAP_ERR_CUDA;
}
