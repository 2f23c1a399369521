// FP64 throughput of the current GPU (hwswe.h: hw_measure_fp64_peak): the denominator of the FP64
// roofline of the scheme's kernels, measured rather than taken from a data sheet.
//
// Every thread runs CHAINS independent chains x <- fma(x, a, b); with eight resident blocks of 256
// threads on every SM the FP64 pipe always has independent work, so the launch time is set by the
// pipe's issue rate alone. a and b are kernel arguments (nothing folds at compile time); the chains
// converge to b / (1 - a) without overflow or subnormals; the sum of the chains is stored under a
// condition the compiler cannot decide, so no chain is removed.
#include <algorithm>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/hwswe.h"
#include "hw_internal.h"

namespace hw {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 8;

__global__ void __launch_bounds__(kThreads) k_dfma_peak(int iters, double a, double b, double* sink) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3 * threadIdx.x + c;
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (s == -1.0) sink[blockIdx.x] = s;  // the chains stay positive: never taken, never provable
}

}  // namespace
}  // namespace hw

extern "C" int hw_measure_fp64_peak(int reps, double* out) {
  if (reps < 1 || reps > 1000 || !out) return hw::set_last_error(HW_ERR_ARG, "hw_measure_fp64_peak: reps in 1..1000 and out required");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms < 1)
    return hw::set_last_error(HW_ERR_CUDA, "hw_measure_fp64_peak: no usable device");
  const int blocks = sms * hw::kBlocksPerSm;
  const int iters = 4096;
  double* sink = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&] {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (sink) cudaFree(sink);
  };
  cudaError_t e = cudaMalloc(&sink, blocks * sizeof(double));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  std::vector<float> ms;
  if (e == cudaSuccess) {
    hw::k_dfma_peak<<<blocks, hw::kThreads, 0, st>>>(iters, 0.9999999, 1e-7, sink);  // warm-up
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
      cudaEventRecord(e0, st);
      hw::k_dfma_peak<<<blocks, hw::kThreads, 0, st>>>(iters, 0.9999999, 1e-7, sink);
      cudaEventRecord(e1, st);
      e = cudaEventSynchronize(e1);
      float t = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      ms.push_back(t);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    cleanup();
    return hw::set_last_error(HW_ERR_CUDA, (std::string("hw_measure_fp64_peak: ") + cudaGetErrorString(e)).c_str());
  }
  cleanup();
  std::sort(ms.begin(), ms.end());
  const double dfma = (double)blocks * hw::kThreads * hw::kChains * iters;
  out[0] = dfma / (ms.front() * 1e-3);
  out[1] = dfma / (ms[ms.size() / 2] * 1e-3);
  out[2] = ms.front();
  return HW_OK;
}
