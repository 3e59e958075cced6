// Dot product that allocates nothing: the same deterministic grid reduction as
// msmg_dot, with its scratch (per-CTA partial sums, the ticket counter and the
// result slot) in a fixed array in this library's device memory instead of a
// caller-provided buffer.  For callers that cannot allocate device memory.
#include "msmg_internal.cuh"
#include "reduce.cuh"

namespace msmg {

// One partial per CTA of 1024 elements: the array bounds the accepted length.
constexpr int64_t kNoAllocElemsPerCta = 1024;
constexpr int64_t kNoAllocMaxCtas = MSMG_DOT_NOALLOC_MAX_N / kNoAllocElemsPerCta;
// layout (doubles): [0, kNoAllocMaxCtas) partials | counter word | result
constexpr int64_t kNoAllocCounterSlot = kNoAllocMaxCtas;
constexpr int64_t kNoAllocResultSlot = kNoAllocMaxCtas + 1;

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) double g_dot_scratch[kNoAllocMaxCtas + 32];

__global__ void k_dot_noalloc(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                              double* scratch) {
  RedSlot red;
  red.partials = scratch;
  red.counter = reinterpret_cast<unsigned*>(scratch + kNoAllocCounterSlot);
  double* out = scratch + kNoAllocResultSlot;
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[0] += a[i] * b[i];
  grid_reduce<1>(v, red, [=] __device__(double* t) { *out = t[0]; });
}

// Device address of the array on the current device.  Looked up on every call
// (the lookup does not synchronise): a cached address would go stale if the
// caller reset the device, after which the module is loaded again.
static int scratch_address(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_dot_scratch);
  if (e != cudaSuccess || !p) { set_last_cuda_error(e); return MSMG_ERR_CUDA; }
  *out = static_cast<double*>(p);
  return 0;
}

}  // namespace msmg

extern "C" int msmg_dot_noalloc(const double* a, const double* b, int64_t n, double* result_host,
                                msmg_stream stream) {
  using namespace msmg;
  if (n < 0 || (n > 0 && (!a || !b)) || !result_host) return MSMG_ERR_INVALID_ARG;
  if (n > MSMG_DOT_NOALLOC_MAX_N) return MSMG_ERR_INVALID_ARG;
  double* scratch = nullptr;
  int st = scratch_address(&scratch);
  if (st) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // the ticket counter must start at zero; the previous call's contents stay otherwise
  MSMG_CUDA_TRY(cudaMemsetAsync(scratch + kNoAllocCounterSlot, 0, sizeof(double), s));
  int64_t grid = (n + kNoAllocElemsPerCta - 1) / kNoAllocElemsPerCta;
  if (grid < 1) grid = 1;
  k_dot_noalloc<<<(unsigned)grid, 256, 0, s>>>(a, b, n, scratch);
  MSMG_CUDA_TRY(cudaGetLastError());
  MSMG_CUDA_TRY(cudaMemcpyAsync(result_host, scratch + kNoAllocResultSlot, sizeof(double), cudaMemcpyDeviceToHost, s));
  MSMG_CUDA_TRY(cudaStreamSynchronize(s));
  return 0;
}
