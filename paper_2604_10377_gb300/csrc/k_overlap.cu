// Overlap-prediction metrics (Sec. "Overlap Prediction Metrics" of the paper): for each
// segment s (the vertices of one shape, or of one pair's overlap region) a vertex is
// predicted overlapping when its score exceeds the threshold (FP32 comparison), and the
// prediction is counted against the binary ground truth:
//   TP = #(pred & label), FP = #(pred & !label), FN = #(!pred & label), TN = the rest.
// From the counts, in FP64: IoU = TP / (TP + FP + FN), accuracy = (TP + TN) / n,
// precision = TP / (TP + FP), recall (sensitivity) = TP / (TP + FN),
// specificity = TN / (TN + FP), F1 = 2 TP / (2 TP + FP + FN) and balanced accuracy =
// (recall + specificity) / 2. A ratio whose denominator is zero is NaN.
//
// The count pass reads each vertex's score (4 bytes) and label (1 byte) once, so it is
// bound by HBM bandwidth: blocks take 4096-vertex chunks of a segment (coalesced scalar
// loads), reduce per warp with ballots, and add the block's counts with one integer
// atomic each (integer sums: exact and order-independent).
#include <stdint.h>

#include "fmap_internal.cuh"

namespace fmap {
namespace {

constexpr int kOvThreads = 256;
constexpr int kOvPerThread = 16;
constexpr int kOvChunk = kOvThreads * kOvPerThread;   // vertices per block

__global__ void __launch_bounds__(kOvThreads) overlap_count_kernel(const float* __restrict__ scores,
                                                                   const uint8_t* __restrict__ labels,
                                                                   const int64_t* __restrict__ seg_off, float thr,
                                                                   unsigned long long* counts) {
  __shared__ unsigned int red[3][kOvThreads / 32];
  const int s = blockIdx.y;
  const int64_t beg = seg_off[s], end = seg_off[s + 1];
  const int64_t c0 = beg + (int64_t)blockIdx.x * kOvChunk;
  if (c0 >= end) return;
  const int64_t c1 = c0 + kOvChunk < end ? c0 + kOvChunk : end;
  unsigned int tp = 0, fp = 0, fn = 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t v0 = c0; v0 < c1; v0 += 4 * kOvThreads) {
    // four loads in flight per thread, then four ballots
    float sc[4];
    uint8_t lb[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t v = v0 + u * kOvThreads + threadIdx.x;
      sc[u] = v < c1 ? scores[v] : 0.f;
      lb[u] = v < c1 ? labels[v] : 0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t v = v0 + u * kOvThreads + threadIdx.x;
      const bool pred = v < c1 && sc[u] > thr, lab = v < c1 && lb[u] != 0;
      const unsigned int bp = __ballot_sync(0xffffffffu, pred), bl = __ballot_sync(0xffffffffu, lab);
      if (lane == 0) {
        tp += __popc(bp & bl);
        fp += __popc(bp & ~bl);
        fn += __popc(~bp & bl);
      }
    }
  }
  if (lane == 0) {
    red[0][warp] = tp;
    red[1][warp] = fp;
    red[2][warp] = fn;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    unsigned long long t = 0;
    for (int w = 0; w < kOvThreads / 32; ++w) t += red[threadIdx.x][w];
    atomicAdd(&counts[4 * s + threadIdx.x], t);
  }
}

// num / den, or a quiet NaN when den is 0 (the ratio is undefined)
__device__ __forceinline__ double ratio(double num, double den) {
  return den > 0.0 ? num / den : __longlong_as_double(0x7ff8000000000000LL);
}

// One thread per segment: TN from the segment length, then the seven metrics.
__global__ void overlap_metrics_kernel(const int64_t* __restrict__ seg_off, int n_seg, unsigned long long* counts,
                                       double* metrics) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_seg) return;
  const unsigned long long n = (unsigned long long)(seg_off[s + 1] - seg_off[s]);
  const unsigned long long tpi = counts[4 * s], fpi = counts[4 * s + 1], fni = counts[4 * s + 2];
  const unsigned long long tni = n - tpi - fpi - fni;
  counts[4 * s + 3] = tni;
  if (metrics == nullptr) return;
  const double tp = (double)tpi, fp = (double)fpi, fn = (double)fni, tn = (double)tni;
  const double recall = ratio(tp, tp + fn), spec = ratio(tn, tn + fp);
  double* m = metrics + 7 * (int64_t)s;
  m[0] = ratio(tp, tp + fp + fn);             // IoU
  m[1] = (recall + spec) * 0.5;               // balanced accuracy
  m[2] = ratio(tp + tn, (double)n);           // accuracy
  m[3] = ratio(tp, tp + fp);                  // precision
  m[4] = recall;                              // recall (sensitivity)
  m[5] = spec;                                // specificity
  m[6] = ratio(2.0 * tp, 2.0 * tp + fp + fn); // F1
}

}  // namespace

cudaError_t launch_overlap_metrics(const float* scores, const uint8_t* labels, const int64_t* seg_off, int n_seg,
                                   int64_t max_len, float thr, int64_t* counts, double* metrics, cudaStream_t st) {
  if (n_seg <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int64_t) * 4 * (size_t)n_seg, st);
  if (e != cudaSuccess) return e;
  auto* cnt = reinterpret_cast<unsigned long long*>(counts);
  if (max_len > 0) {
    const int64_t chunks = (max_len + kOvChunk - 1) / kOvChunk;
    overlap_count_kernel<<<dim3((unsigned)chunks, (unsigned)n_seg), kOvThreads, 0, st>>>(scores, labels, seg_off, thr,
                                                                                         cnt);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  overlap_metrics_kernel<<<(n_seg + 127) / 128, 128, 0, st>>>(seg_off, n_seg, cnt, metrics);
  return cudaGetLastError();
}

}  // namespace fmap
