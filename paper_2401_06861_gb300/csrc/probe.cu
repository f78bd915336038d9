// Arithmetic-pipe peak probes (measurement only, not part of the method).
//
// The FP64 sweeps are bound by the FP64 pipe and the double-float sweeps by
// the FP32 pipe; the benchmark reports their rates against peaks measured in
// the same run by these kernels: every thread runs independent FMA chains
// (enough chains to cover the pipe latency), the grid fills every SM several
// times over, and the rate is timed with CUDA events on a private stream.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/nwqgb.h"
#include "state.hpp"

namespace nwq {
namespace {

constexpr int kProbeThreads = 256;

template <class R, int CH>
__global__ void __launch_bounds__(kProbeThreads) fma_chains(int iters, R a, R b, R* __restrict__ out) {
  R v[CH];
#pragma unroll
  for (int c = 0; c < CH; c++) v[c] = (R)(threadIdx.x + c) * (R)1e-3;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < CH; c++) v[c] = fma(v[c], a, b);
  }
  R s = 0;
#pragma unroll
  for (int c = 0; c < CH; c++) s += v[c];
  out[blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

template <class R, int CH>
int probe(int iters, double* per_second) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return set_error(NWQ_ECUDA, cudaGetErrorString(e));
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chains<R, CH>, kProbeThreads, 0);
  if (e != cudaSuccess) return set_error(NWQ_ECUDA, cudaGetErrorString(e));
  const int blocks = sms * (per_sm < 1 ? 1 : per_sm) * 4;
  cudaStream_t s = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  R* out = nullptr;
  e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(R) * (size_t)blocks * kProbeThreads);
  float ms = 0.f;
  if (e == cudaSuccess) {
    // (a, b) keep every chain finite: v -> v * 0.999... + 1e-7 converges
    fma_chains<R, CH><<<blocks, kProbeThreads, 0, s>>>(iters / 8 + 1, (R)0.9999999, (R)1e-7, out);  // warm-up
    e = cudaEventRecord(t0, s);
    fma_chains<R, CH><<<blocks, kProbeThreads, 0, s>>>(iters, (R)0.9999999, (R)1e-7, out);
    if (e == cudaSuccess) e = cudaEventRecord(t1, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
  }
  if (out) cudaFree(out);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess) return set_error(NWQ_ECUDA, cudaGetErrorString(e));
  if (ms <= 0.f) return set_error(NWQ_ECUDA, "peak probe: no elapsed time");
  *per_second = (double)blocks * kProbeThreads * CH * (double)iters / (ms * 1e-3);
  return NWQ_OK;
}

}  // namespace
}  // namespace nwq

extern "C" int nwq_peak_probe(int what, double* fma_per_second) {
  if (!fma_per_second) return nwq::set_error(NWQ_EINVAL, "NULL argument");
  switch (what) {
    case NWQ_PROBE_FP64_FMA:
      return nwq::probe<double, 8>(4096, fma_per_second);
    case NWQ_PROBE_FP32_FMA:
      return nwq::probe<float, 16>(1 << 17, fma_per_second);
    default:
      return nwq::set_error(NWQ_EINVAL, "nwq_peak_probe: unknown probe");
  }
}
