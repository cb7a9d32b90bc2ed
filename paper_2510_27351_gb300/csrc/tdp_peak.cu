// Measured rate of the binary64 pipe (a diagnostic of the library, not part
// of the method): the denominator of the binary64 kernels' ALU roofline.
//
// Every thread runs kChains independent chains x <- fma(x, y, z), so that
// each SM sub-partition always has independent binary64 instructions to
// issue; y and z arrive at run time (nothing folds), and the chains' sum is
// stored only under a condition the values never meet.
#include <algorithm>

#include "tdp_internal.h"

namespace tdp {
namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) k_fp64_pipe(double* __restrict__ sink, int iters, double y,
                                                            double z) {
  double x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 1e-3 * threadIdx.x + i;
  for (int k = 0; k < iters; ++k) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], y, z);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace tdp

using namespace tdp;

extern "C" int tdp_fp64_fma_rate(double* fma_per_s, double* ms_out, void* stream) {
  if (!fma_per_s) return set_last_error(TDP_EINVAL, "tdp_fp64_fma_rate: null output");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fp64_pipe, kPeakThreads, 0);
  if (e != cudaSuccess) return set_last_error(TDP_ECUDA, std::string("tdp_fp64_fma_rate: ") + cudaGetErrorString(e));
  const int grid = sms * std::max(1, per_sm) * 4;  // four waves of full occupancy
  const int iters = 2048;
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&sink, sizeof(double) * grid);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.0f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // rep 0 warms up
    e = cudaEventRecord(e0, st);
    launch_begin(st, "fp64_pipe", false);
    k_fp64_pipe<<<grid, kPeakThreads, 0, st>>>(sink, iters, 0.999999, 1e-6);
    launch_end(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return set_last_error(TDP_ECUDA, std::string("tdp_fp64_fma_rate: ") + cudaGetErrorString(e));
  const double fmas = double(grid) * kPeakThreads * kChains * double(iters);
  *fma_per_s = fmas / (double(best) * 1e-3);
  if (ms_out) *ms_out = best;
  return set_last_error(TDP_OK, "");
}
