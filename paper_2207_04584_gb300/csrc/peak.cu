// FP32 FMA throughput of this GPU, measured: the ALU roofline of the plain
// FP32 gridding form (its peak is not among the measured copy and tensor
// peaks).  Each thread runs 8 independent FMA chains; the grid fills every SM
// with 8 CTAs of 256 threads.
#include <cuda_runtime.h>

#include "hegrid_internal.cuh"

namespace hg {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_fma_loop(float* __restrict__ sink, int iters, float c) {
  float v[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) v[k] = (float)(threadIdx.x + k) * 1e-3f;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < kChains; ++k) v[k] = __fmaf_rn(v[k], c, 1e-4f);
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += v[k];
  if (s == 12345.0f) sink[blockIdx.x] = s;  // keeps the chains alive; never true in practice
}

}  // namespace
}  // namespace hg

extern "C" hegrid_status hegrid_fp32_peak(double* tflops, void* stream) {
  hg::set_error("");
  HG_ARG_CHECK(tflops != nullptr, "tflops is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  HG_CUDA_TRY(cudaGetDevice(&dev));
  HG_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256, iters = 1 << 14;
  float* sink = nullptr;
  HG_CUDA_TRY(hg::pool_alloc((void**)&sink, sizeof(float) * blocks, s));
  cudaEvent_t e0, e1;
  HG_CUDA_TRY(cudaEventCreate(&e0));
  HG_CUDA_TRY(cudaEventCreate(&e1));
  hg::k_fma_loop<<<blocks, threads, 0, s>>>(sink, iters / 8, 0.999f);  // warm-up
  cudaEventRecord(e0, s);
  hg::k_fma_loop<<<blocks, threads, 0, s>>>(sink, iters, 0.999f);
  cudaEventRecord(e1, s);
  hg::count_launch(2);
  cudaError_t err = hg::launch_status();
  if (err == cudaSuccess) err = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(sink, s);
  HG_CUDA_TRY(err);
  const double flops = 2.0 * (double)blocks * threads * iters * hg::kChains;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return HEGRID_OK;
}
