// Plain-ALU throughput probe (FP64 and FP32 FMA), the denominator of the
// roofline for ALU-bound kernels.  Each thread runs eight independent FMA
// chains in registers; the result is kept alive through a device sink that is
// written only when the value matches an impossible bit pattern.
#include "msmg_internal.cuh"

namespace msmg {

__device__ double g_probe_sink;

template <typename T>
__global__ void k_fma_chain(int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if ((double)s == -1.2345e300) g_probe_sink = (double)s;
}

}  // namespace msmg

extern "C" int msmg_probe_alu_peaks(double* fp64_tflops, double* fp32_tflops, msmg_stream stream) {
  using namespace msmg;
  if (!fp64_tflops || !fp32_tflops) return MSMG_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = nsm * 8, threads = 256;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  double best64 = 0, best32 = 0;
  for (int rep = 0; rep < 3; ++rep) {
    const int it64 = 2048, it32 = 2048 * 16;
    float ms = 0;
    cudaEventRecord(e0, s);
    k_fma_chain<double><<<blocks, threads, 0, s>>>(it64, 0.999999, 1e-7);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    const double f64 = 2.0 * 8 * it64 * (double)blocks * threads / (ms * 1e-3) / 1e12;
    cudaEventRecord(e0, s);
    k_fma_chain<float><<<blocks, threads, 0, s>>>(it32, 0.999999f, 1e-7f);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    const double f32 = 2.0 * 8 * it32 * (double)blocks * threads / (ms * 1e-3) / 1e12;
    if (f64 > best64) best64 = f64;
    if (f32 > best32) best32 = f32;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *fp64_tflops = best64;
  *fp32_tflops = best32;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { set_last_cuda_error(e); return MSMG_ERR_CUDA; }
  return 0;
}
