// lise_probe.cu -- lise_measure_fp64_peak: the FP64 fused multiply-add throughput of the
// GPU under its current clock, measured with a kernel of independent FMA chains (CUDA
// events on a private stream).  It is the denominator of the FP64-pipe fraction that the
// benchmark reports beside the memory roofline.
#include <cuda_runtime.h>

#include "../../include/lise.h"

namespace {

constexpr int kChains = 8;      // independent FMA chains per thread (hide the FMA latency)
constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_dfma_probe(double* sink, int store, int iters, double a, double b) {
  double x[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) x[i] = 1e-3 * (double)threadIdx.x + (double)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += x[i];
  if (store) sink[blockIdx.x] = s;  // store = 0 at run time; the compiler must keep the chains
}

}  // namespace

extern "C" int lise_measure_fp64_peak(int device, double* tflops) {
  if (!tflops) return LISE_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return LISE_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return LISE_ECUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return LISE_ECUDA;
  const int blocks = sms * 8, iters = 4096;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = LISE_OK;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    rc = LISE_ECUDA;
  float best = 0.f;
  for (int rep = 0; rep < 6 && rc == LISE_OK; ++rep) {  // the first launch warms up
    cudaEventRecord(e0, s);
    k_dfma_probe<<<blocks, kThreads, 0, s>>>(nullptr, 0, iters, 0.9999999, 1e-7);
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      rc = LISE_ECUDA;
      break;
    }
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (rc != LISE_OK) return rc;
  const double flops = 2.0 * kChains * (double)iters * blocks * kThreads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return LISE_OK;
}
