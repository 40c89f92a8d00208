// Measured FP32 FMA throughput of the device, as a denominator beside the
// nominal one (SMs x 128 FP32 lanes x 2 flop x maximum SM clock) for the
// passes' FP32 roofline.  Each thread runs eight independent FMA chains
// (enough to cover the FMA latency at full occupancy); the chains stay
// bounded (x -> a x + b with 0 < a < 1) and their sum is stored so that
// nothing is optimised away.
#include <cuda_runtime.h>

#include <algorithm>

#include "pty_internal.h"
#include "../../include/pty.h"

namespace {

constexpr int kChains = 8, kUnroll = 16;

__global__ void __launch_bounds__(256) k_ffma(float* __restrict__ out, int iters, float a,
                                              float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1e-3f * (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int pty_measure_fp32_peak(double* tflops) {
  if (!tflops) return pty::set_error(PTY_EINVAL, "null argument");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return pty::set_error(PTY_ECUDA, "no device");
  const int threads = 256, blocks = sms * 8, iters = 4096;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t s = nullptr;
  int rc = PTY_OK;
  if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    rc = pty::set_error(PTY_ECUDA, "setup failed");
  } else {
    float best = 1e30f;
    for (int rep = 0; rep < 4 && rc == PTY_OK; ++rep) {  // the first launch warms up
      cudaEventRecord(e0, s);
      k_ffma<<<blocks, threads, 0, s>>>(out, iters, 0.9999999f, 1e-7f);
      cudaEventRecord(e1, s);
      float ms = 0.f;
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
        rc = pty::set_error(PTY_ECUDA, "timing failed");
      else if (rep > 0)
        best = std::min(best, ms);
    }
    if (rc == PTY_OK) {
      const double flop = 2.0 * kChains * kUnroll * (double)iters * blocks * threads;
      *tflops = flop / (best * 1e-3) / 1e12;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (out) cudaFree(out);
  cudaGetLastError();
  return rc;
}
