// Measurement aid: the FP32 fused multiply-add rate this GPU sustains, the
// denominator of the CUDA-core kernels' roofline (the paper has no
// counterpart).  Every thread runs 16 independent FFMA chains, so issue, not
// latency, bounds the loop; the grid holds 8 blocks of 256 threads per SM.
#include "mcmg_internal.cuh"

namespace mcmg {

namespace {

constexpr int FFMA_CHAINS = 16;
constexpr int FFMA_ITERS = 4096;

__device__ float g_ffma_sink;   // written only if the chains' sum is negative: never

__global__ void __launch_bounds__(256) k_ffma_peak(float a, float b) {
  float v[FFMA_CHAINS];
#pragma unroll
  for (int i = 0; i < FFMA_CHAINS; ++i) v[i] = (float)(threadIdx.x + i);
#pragma unroll 4
  for (int it = 0; it < FFMA_ITERS; ++it) {
#pragma unroll
    for (int i = 0; i < FFMA_CHAINS; ++i) v[i] = fmaf(v[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < FFMA_CHAINS; ++i) s += v[i];
  // the chains start at 0 .. 270 and contract towards b / (1 - a) = 1, so the
  // sum stays positive; the test only keeps the compiler from dropping them
  if (s < 0.f) g_ffma_sink = s;
}

}  // namespace

}  // namespace mcmg

mcmg_status mcmg_fp32_ffma_tflops(void* stream, double* tflops) {
  using namespace mcmg;
  if (!tflops) {
    set_error("NULL result pointer");
    return MCMG_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  MCMG_CUDA(cudaGetDevice(&dev));
  MCMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256;
  cudaEvent_t e0, e1;
  MCMG_CUDA(cudaEventCreate(&e0));
  MCMG_CUDA(cudaEventCreate(&e1));
  for (int w = 0; w < 3; ++w) k_ffma_peak<<<blocks, threads, 0, st>>>(0.999f, 0.001f);
  MCMG_CUDA(cudaEventRecord(e0, st));
  const int reps = 20;
  for (int r = 0; r < reps; ++r) k_ffma_peak<<<blocks, threads, 0, st>>>(0.999f, 0.001f);
  MCMG_CUDA(cudaEventRecord(e1, st));
  MCMG_CUDA(cudaEventSynchronize(e1));
  count_launch(3 + reps);
  float ms = 0.f;
  MCMG_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 2.0 * FFMA_CHAINS * FFMA_ITERS * (double)blocks * threads * reps;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return MCMG_OK;
}
