// FP32 FMA throughput probe (a measurement aid, not part of the training
// path): every thread runs 8 independent chains of packed dual FP32 FMAs,
// enough independent work per warp to keep the FMA pipes of every SM busy,
// so the kernel's FLOP rate is the device's attainable FP32 FMA peak at the
// clocks it runs at.  Timed with CUDA events around one launch.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/dpinn.h"

namespace {

__global__ void __launch_bounds__(256) k_ffma2_probe(float* out, long long iters) {
  float2 a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = make_float2(1e-3f * (threadIdx.x + i), 2e-3f * (blockIdx.x + i));
  const float2 m = make_float2(0.999999f, 0.999998f), c = make_float2(1e-7f, 2e-7f);
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = __ffma2_rn(a[i], m, c);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i].x + a[i].y;
  if (s == 1234.5f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains alive
}

}  // namespace

extern "C" int dpinn_probe_fp32(int device, int blocks_per_sm, long long iters, float* ms, double* flop) {
  if (!ms || !flop || blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 1 || iters > (1LL << 40))
    return DPINN_ERR_INVALID_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return DPINN_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return DPINN_ERR_CUDA;
  const int blocks = sms * blocks_per_sm, threads = 256;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&out, (size_t)blocks * threads * sizeof(float));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    k_ffma2_probe<<<blocks, threads>>>(out, std::min<long long>(iters, 64));   // warm-up
    cudaEventRecord(e0);
    k_ffma2_probe<<<blocks, threads>>>(out, iters);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
  }
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  // 8 chains x 4 packed FMAs x 2 lanes x 2 FLOP per iteration and thread
  *flop = (double)blocks * threads * (double)iters * 8 * 4 * 2 * 2;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  return e == cudaSuccess ? DPINN_OK : DPINN_ERR_CUDA;
}
