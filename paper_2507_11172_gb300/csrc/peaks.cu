// Arithmetic peaks of the device: FP32 and FP64 fused multiply-add throughput, measured with
// long independent FMA chains on a full grid.  The triplet kernel is bound by plain FP32 ALU work
// (no tensor cores: the ATM sum is not a dense contraction), so its roofline fraction divides its
// algorithmic flop rate by what this device's FMA pipes deliver at the clock of the moment; the FP64
// path is set against the DFMA rate the same way.  No counterpart in the paper.
//
// Each thread runs kChains independent recurrences acc = acc * a + b (|a| < 1, so the values stay
// bounded and normal), kUnroll steps per loop trip; the sum of the chains is stored only if it equals
// an impossible value, which keeps every FMA live without a store per thread.  Work per launch:
// 2 flop x kChains x kUnroll x iters per thread.
#include <algorithm>
#include <string>

#include "../../include/respa3b.h"
#include "md_internal.cuh"

namespace r3b {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma(float a, float b, int iters, float* out) {
  float acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = 1e-3f * (float)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) acc[c] = __fmaf_rn(acc[c], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  if (s == -1.2345f) out[0] = s;
}

// packed FP32x2 (two FMAs per instruction)
__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma2(float a, float b, int iters, float* out) {
  float2 acc[kChains / 2];
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
  for (int c = 0; c < kChains / 2; ++c) acc[c] = make_float2(1e-3f * (float)(threadIdx.x + c), 2e-3f * (float)c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains / 2; ++c) acc[c] = __ffma2_rn(acc[c], a2, b2);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains / 2; ++c) s += acc[c].x + acc[c].y;
  if (s == -1.2345f) out[0] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_dfma(double a, double b, int iters, float* out) {
  double acc[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc[c] = 1e-3 * (double)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) acc[c] = __fma_rn(acc[c], a, b);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += acc[c];
  if (s == -1.2345) out[0] = (float)s;
}

cudaError_t launch_peak(int kind, int grid, int iters, float* out, cudaStream_t st) {
  if (kind == 0)
    k_peak_ffma<<<grid, kPeakThreads, 0, st>>>(0.9999f, 1e-4f, iters, out);
  else if (kind == 1)
    k_peak_ffma2<<<grid, kPeakThreads, 0, st>>>(0.9999f, 1e-4f, iters, out);
  else
    k_peak_dfma<<<grid, kPeakThreads, 0, st>>>(0.9999, 1e-4, iters, out);
  return cudaGetLastError();
}

}  // namespace
}  // namespace r3b

using namespace r3b;

extern "C" md_status md_measure_fma_peak(int kind, double min_ms, double* flops_per_s, double* ms_out) {
  if (kind < 0 || kind > 2 || !flops_per_s || !(min_ms > 0) || !(min_ms <= 1e4)) return MD_ERR_ARG;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_last_error((std::string("md_measure_fma_peak: ") + cudaGetErrorString(e)).c_str());
    return MD_ERR_CUDA;
  }
  const void* kern = kind == 0 ? (const void*)k_peak_ffma : kind == 1 ? (const void*)k_peak_ffma2
                                                                       : (const void*)k_peak_dfma;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPeakThreads, 0);
  const int grid = std::max(1, sms) * std::max(1, per_sm);  // one full wave of resident CTAs
  cudaStream_t st = nullptr;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  md_status status = MD_OK;
  auto fail = [&](cudaError_t err, const char* what) {
    cudaGetLastError();
    set_last_error((std::string("md_measure_fma_peak: ") + what + ": " + cudaGetErrorString(err)).c_str());
    status = err == cudaErrorMemoryAllocation ? MD_ERR_OOM : MD_ERR_CUDA;
  };
  double best = 0.0, best_ms = 0.0;
  do {
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) { fail(e, "stream"); break; }
    if ((e = cudaMalloc(&out, sizeof(float))) != cudaSuccess) { fail(e, "cudaMalloc"); break; }
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
      fail(e, "event");
      break;
    }
    // calibrate: grow the trip count until one launch lasts at least min_ms, then time three launches
    int iters = kind == 2 ? 16 : 256;
    float ms = 0.f;
    for (int round = 0; round < 40; ++round) {
      if ((e = cudaEventRecord(e0, st)) != cudaSuccess) break;
      if ((e = launch_peak(kind, grid, iters, out, st)) != cudaSuccess) break;
      if ((e = cudaEventRecord(e1, st)) != cudaSuccess) break;
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
      if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
      if (ms >= min_ms || iters > (1 << 28)) break;
      const double grow = ms > 0.05f ? 1.2 * min_ms / ms : 8.0;
      iters = (int)std::min<double>((double)iters * std::max(2.0, grow), (double)(1 << 29));
    }
    if (e != cudaSuccess) { fail(e, "calibration launch"); break; }
    const double work = 2.0 * kChains * kUnroll * (double)iters * (double)grid * kPeakThreads;
    for (int r = 0; r < 3; ++r) {
      if ((e = cudaEventRecord(e0, st)) != cudaSuccess) break;
      if ((e = launch_peak(kind, grid, iters, out, st)) != cudaSuccess) break;
      if ((e = cudaEventRecord(e1, st)) != cudaSuccess) break;
      if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
      if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
      const double rate = work / ((double)ms * 1e-3);
      if (rate > best) {
        best = rate;
        best_ms = ms;
      }
    }
    if (e != cudaSuccess) fail(e, "timed launch");
  } while (false);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (st) cudaStreamDestroy(st);
  if (status != MD_OK) return status;
  *flops_per_s = best;
  if (ms_out) *ms_out = best_ms;
  return MD_OK;
}
