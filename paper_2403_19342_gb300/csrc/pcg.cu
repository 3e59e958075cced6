// Preconditioned conjugate gradients on A x = b (Eq. (p)) with the V-cycle
// preconditioner, FP64 outer recurrence.  Scalars (alpha, beta, residual
// norms, iteration count, convergence flag) live on the device and are
// produced by the last CTA of each reducing kernel, so an iteration needs no
// host round trip; every kernel returns at once when the flag is set, so
// extra launches after convergence are no-ops and the iteration count stays
// exact.
#include "msmg_internal.cuh"
#include "reduce.cuh"
#include <cmath>

namespace msmg {

void pcg_step_vcycle(msmg_ctx* c, int update, const double* qv, PcgScalars* sc, cudaStream_t s);
void pcg_step_pmatvec(msmg_ctx* c, PcgScalars* sc, cudaStream_t s);

static constexpr int kVecThreads = 256;
static inline unsigned vec_grid(int64_t n) {
  int64_t g = (n + kVecThreads * 4 - 1) / (kVecThreads * 4);
  if (g > 152 * 8) g = 152 * 8;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// sum(b) -> sc->mean (as mean), then the host launches k_sub_mean
__global__ void k_sum(const double* __restrict__ b, int64_t n, RedSlot red, double* out, double scale) {
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[0] += b[i];
  grid_reduce<1>(v, red, [=] __device__(double* t) { *out = t[0] * scale; });
}

// b -= mean; r = b; x = 0; bb = b.b (initial residual for a zero guess)
__global__ void k_init_zero(double* __restrict__ b, double* __restrict__ r, double* __restrict__ x, int64_t n,
                            RedSlot red, PcgScalars* sc, double rtol2) {
  const double mean = sc->mean;
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i] - mean;
    b[i] = bi;
    r[i] = bi;
    x[i] = 0.0;
    v[0] += bi * bi;
  }
  grid_reduce<1>(v, red, [=] __device__(double* t) {
    sc->bb = t[0];
    sc->tol2 = rtol2 * t[0];
    sc->rr = t[0];
    sc->iter = 0;
    sc->rz = 0.0;
    sc->pq = 0.0;
    sc->done = (t[0] <= sc->tol2 || t[0] == 0.0) ? 1 : 0;
  });
}

// b -= mean; x given: r = b - q (q = A x computed before); bb, rr
__global__ void k_init_x0(double* __restrict__ b, double* __restrict__ r, const double* __restrict__ q, int64_t n,
                          RedSlot red, PcgScalars* sc, double rtol2) {
  const double mean = sc->mean;
  double v[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double bi = b[i] - mean;
    b[i] = bi;
    const double ri = bi - q[i];
    r[i] = ri;
    v[0] += bi * bi;
    v[1] += ri * ri;
  }
  grid_reduce<2>(v, red, [=] __device__(double* t) {
    sc->bb = t[0];
    sc->tol2 = rtol2 * t[0];
    sc->rr = t[1];
    sc->iter = 0;
    sc->rz = 0.0;
    sc->pq = 0.0;
    sc->done = (t[1] <= sc->tol2 || t[0] == 0.0) ? 1 : 0;
  });
}

// residual replacement: r = b - q (q = A x), rr; restart the recurrence
__global__ void k_restart(const double* __restrict__ b, const double* __restrict__ q, double* __restrict__ r,
                          int64_t n, RedSlot red, PcgScalars* sc) {
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = b[i] - q[i];
    r[i] = ri;
    v[0] += ri * ri;
  }
  grid_reduce<1>(v, red, [=] __device__(double* t) {
    sc->rr = t[0];
    sc->rz = 0.0;
    sc->pq = 0.0;
    sc->beta = 0.0;
    sc->done = t[0] <= sc->tol2 ? 1 : 0;
  });
}

__global__ void k_copy(const double* __restrict__ a, double* __restrict__ b, int64_t n, const PcgScalars* sc) {
  if (sc && sc->done) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

// x += alpha p; r -= alpha q; rr = r.r; iteration bookkeeping
__global__ void k_update(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                         const double* __restrict__ q, int64_t n, RedSlot red, PcgScalars* sc) {
  if (sc->done) return;
  const double alpha = sc->alpha;
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    v[0] += ri * ri;
  }
  grid_reduce<1>(v, red, [=] __device__(double* t) {
    sc->rr = t[0];
    sc->iter += 1;
    if (!isfinite(t[0])) sc->done = 2;
    else if (t[0] <= sc->tol2) sc->done = 1;
    else if (sc->iter >= sc->max_iter) sc->done = 3;
  });
}

// p_new = z + beta p_old
__global__ void k_pupdate(const double* __restrict__ z, const double* __restrict__ pold, double* __restrict__ pnew,
                          int64_t n, const PcgScalars* sc) {
  if (sc->done) return;
  const double beta = sc->beta;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    pnew[i] = z[i] + beta * pold[i];
}

// x -= mean(x) (uniqueness condition): out[0] holds the sum beforehand
__global__ void k_sub_scalar(double* __restrict__ x, int64_t n, const double* sum, double scale) {
  const double m = *sum * scale;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] -= m;
}

// ||b - q||^2 -> out
__global__ void k_resid_norm(const double* __restrict__ b, const double* __restrict__ q, int64_t n, RedSlot red,
                             double* out) {
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = b[i] - q[i];
    v[0] += d * d;
  }
  grid_reduce<1>(v, red, [=] __device__(double* t) { *out = t[0]; });
}

__global__ void k_dot(const double* __restrict__ a, const double* __restrict__ b, int64_t n, RedSlot red,
                      double* out) {
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[0] += a[i] * b[i];
  grid_reduce<1>(v, red, [=] __device__(double* t) { *out = t[0]; });
}

__global__ void k_set_scalars(PcgScalars* sc, int max_iter, int flexible) {
  sc->max_iter = max_iter;
  sc->flexible = flexible;
  sc->done = 0;
  sc->iter = 0;
}

void launch_dot(const double* a, const double* b, int64_t n, RedSlot red, double* out, cudaStream_t s) {
  k_dot<<<vec_grid(n), kVecThreads, 0, s>>>(a, b, n, red, out);
}

// Capture two consecutive PCG iterations (p0 -> p1 -> p0) into a CUDA graph on a
// private stream.  Returns 1 when the graph is ready, -1 when capture is not
// possible (the caller then launches kernel by kernel).
static int build_iteration_graph(msmg_ctx* c) {
  if (c->graph_state != 0) return c->graph_state;
  SolveBuffers& B = c->sb;
  const bool flexible = c->opts.precision == MSMG_MIXED;
  c->graph_state = -1;
  if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return -1;
  B.pcur = B.p0;
  B.pnext = B.p1;
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return -1;
  for (int k = 0; k < 2; ++k) {
    pcg_step_pmatvec(c, B.sc, c->cap_stream);
    double* t = B.pcur; B.pcur = B.pnext; B.pnext = t;
    pcg_step_vcycle(c, 1, flexible ? B.q : nullptr, B.sc, c->cap_stream);
  }
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  B.pcur = B.p0;
  B.pnext = B.p1;
  if (e != cudaSuccess || !g) { cudaGetLastError(); return -1; }
  e = cudaGraphInstantiate(&c->iter_graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { cudaGetLastError(); return -1; }
  c->graph_state = 1;
  return 1;
}

// One PCG solve for a single right-hand side already in block-major order in
// c->sb.b (FP64); x in c->sb.x (initial guess if use_x0).
//   init:      r0 = b - A x0 (mean removed), z0 = P^{-1} r0, beta = 0
//   iteration: p = z + beta p; q = A p; alpha = r.z / p.q        (k_pmatvec)
//              x += alpha p; r -= alpha q; stop on ||r|| <= rtol ||b||   (k_pre)
//              z = P^{-1} r; beta = r.z / r_old.z_old, or the flexible
//              (Polak-Ribiere) beta in the mixed form                (V-cycle)
static int pcg_one(msmg_ctx* c, double rtol, int max_iter, bool use_x0, int flags, cudaStream_t s,
                   msmg_solve_info* info) {
  SolveBuffers& B = c->sb;
  PcgScalars* sc = B.sc;
  const int64_t n = c->n;
  const unsigned vg = vec_grid(n);
  const bool flexible = c->opts.precision == MSMG_MIXED;
  k_set_scalars<<<1, 1, 0, s>>>(sc, max_iter, flexible ? 1 : 0);
  k_sum<<<vg, kVecThreads, 0, s>>>(B.b, n, c->red, &sc->mean, 1.0 / (double)n);
  if (use_x0) {
    launch_matvec(c, B.x, B.q, s);
    k_init_x0<<<vg, kVecThreads, 0, s>>>(B.b, B.r, B.q, n, c->red, sc, rtol * rtol);
  } else {
    k_init_zero<<<vg, kVecThreads, 0, s>>>(B.b, B.r, B.x, n, c->red, sc, rtol * rtol);
  }
  MSMG_CUDA_TRY(cudaMemsetAsync(B.p0, 0, n * sizeof(double), s));
  B.pcur = B.p0;
  B.pnext = B.p1;
  pcg_step_vcycle(c, 0, nullptr, sc, s);
  PcgScalars hsc;
  const int64_t vc_launches = 4 + 4 * (int64_t)(c->nL - 2) + 1;
  int64_t launches = 3 + (use_x0 ? 2 : 1) + vc_launches;
  const bool graph = !(flags & MSMG_FLAG_NO_GRAPH) && build_iteration_graph(c) == 1;
  auto iterate = [&](int budget) -> int {
    if (graph) {
      // two iterations per graph launch (the p buffers alternate); kernels are
      // no-ops once the device flag is set, so the count stays exact
      for (int it = 0; it < budget; it += 2) {
        launches += 2 * (1 + vc_launches);
        MSMG_CUDA_TRY(cudaGraphLaunch(c->iter_graph, s));
        if ((it & 7) == 6 || it + 2 >= budget) {
          MSMG_CUDA_TRY(cudaMemcpyAsync(&hsc, sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
          MSMG_CUDA_TRY(cudaStreamSynchronize(s));
          if (hsc.done) break;
        }
      }
    } else {
      for (int it = 0; it < budget; ++it) {
        launches += 1 + vc_launches;
        pcg_step_pmatvec(c, sc, s);
        double* t = B.pcur; B.pcur = B.pnext; B.pnext = t;
        pcg_step_vcycle(c, 1, flexible ? B.q : nullptr, sc, s);
        if ((it & 3) == 3 || it + 1 == budget) {
          MSMG_CUDA_TRY(cudaMemcpyAsync(&hsc, sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
          MSMG_CUDA_TRY(cudaStreamSynchronize(s));
          if (hsc.done) break;
        }
      }
    }
    MSMG_CUDA_TRY(cudaMemcpyAsync(&hsc, sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
    MSMG_CUDA_TRY(cudaStreamSynchronize(s));
    return 0;
  };
  int st = iterate(max_iter);
  if (st) return st;
  // The recurrence residual can drift from b - A x (FP32 V-cycle, flexible beta):
  // check the true residual in FP64 and, if it is above the tolerance, replace the
  // residual by it and continue (at most twice).
  double* scal = c->dtmp + 8;
  double hres[2] = {0.0, 0.0};
  for (int restart = 0;; ++restart) {
    launch_matvec(c, B.x, B.q, s);
    k_resid_norm<<<vg, kVecThreads, 0, s>>>(B.b, B.q, n, c->red, scal + 1);
    MSMG_CUDA_TRY(cudaMemcpyAsync(hres, scal, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    MSMG_CUDA_TRY(cudaStreamSynchronize(s));
    launches += 2;
    if (hsc.done != 1 || hres[1] <= hsc.tol2 || restart == 2 || hsc.iter >= max_iter) break;
    k_restart<<<vg, kVecThreads, 0, s>>>(B.b, B.q, B.r, n, c->red, sc);
    MSMG_CUDA_TRY(cudaMemsetAsync(B.p0, 0, n * sizeof(double), s));
    B.pcur = B.p0;
    B.pnext = B.p1;
    pcg_step_vcycle(c, 0, nullptr, sc, s);
    launches += 1 + vc_launches;
    st = iterate(max_iter - hsc.iter);
    if (st) return st;
  }
  // zero-mean solution (uniqueness condition, Section 2.1)
  k_sum<<<vg, kVecThreads, 0, s>>>(B.x, n, c->red, scal, 1.0);
  k_sub_scalar<<<vg, kVecThreads, 0, s>>>(B.x, n, scal, 1.0 / (double)n);
  launches += 2;
  MSMG_CUDA_TRY(cudaStreamSynchronize(s));
  if (info) {
    info->iterations = hsc.iter;
    info->converged = hsc.done == 1;
    info->rel_residual = hsc.bb > 0 ? std::sqrt(hsc.rr / hsc.bb) : 0.0;
    info->true_rel_residual = hsc.bb > 0 ? std::sqrt(hres[1] / hsc.bb) : 0.0;
    info->rhs_mean = hsc.mean;
    info->kernel_launches = launches;
  }
  if (hsc.done == 2) return MSMG_ERR_BREAKDOWN;
  if (hsc.done != 1) return MSMG_NOT_CONVERGED;
  return MSMG_OK;
}

int pcg_solve(msmg_ctx* c, const double* rhs, double* x, double rtol, int max_iter, int flags, cudaStream_t s,
              msmg_solve_info* info) {
  const int64_t n = c->n;
  const bool host = flags & MSMG_FLAG_HOST_IO;
  const bool x0 = flags & MSMG_FLAG_X0;
  SolveBuffers& B = c->sb;
  // natural-order staging: q and z serve as staging buffers
  if (host) {
    MSMG_CUDA_TRY(cudaMemcpyAsync(B.q, rhs, n * sizeof(double), cudaMemcpyHostToDevice, s));
    launch_nat_to_blk(c, B.q, B.b, s);
    if (x0) {
      MSMG_CUDA_TRY(cudaMemcpyAsync(B.q, x, n * sizeof(double), cudaMemcpyHostToDevice, s));
      launch_nat_to_blk(c, B.q, B.x, s);
    }
  } else {
    launch_nat_to_blk(c, rhs, B.b, s);
    if (x0) launch_nat_to_blk(c, x, B.x, s);
  }
  int st = pcg_one(c, rtol, max_iter, x0, flags, s, info);
  if (info) info->kernel_launches += (x0 ? 2 : 1) + 1;   // permutations in and out
  if (host) {
    launch_blk_to_nat(c, B.x, B.q, s);
    MSMG_CUDA_TRY(cudaMemcpyAsync(x, B.q, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    MSMG_CUDA_TRY(cudaStreamSynchronize(s));
  } else {
    launch_blk_to_nat(c, B.x, x, s);
  }
  return st;
}

double dot_host(msmg_ctx* c, const double* a, const double* b, int64_t n, cudaStream_t s) {
  double* out = c->dtmp + 12;
  launch_dot(a, b, n, c->red, out, s);
  double h = 0;
  cudaMemcpyAsync(&h, out, sizeof(double), cudaMemcpyDeviceToHost, s);
  cudaStreamSynchronize(s);
  return h;
}

}  // namespace msmg
