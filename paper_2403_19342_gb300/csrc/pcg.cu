// Preconditioned conjugate gradients on A x = b (Eq. (p)) with the V-cycle
// preconditioner, FP64 outer recurrence, for a batch of R right-hand sides in
// lockstep (one PcgScalars record each; vectors stored n apart).  Scalars
// (alpha, beta, residual norms, iteration count, convergence flag) live on the
// device and are produced by the last CTA of each reducing kernel, so an
// iteration needs no host round trip; every kernel returns at once for a
// right-hand side whose flag is set, so launches after convergence are no-ops
// and each iteration count stays exact.
//
// The host side (PcgRun) is resumable: it keeps two chunks of iterations in
// flight and polls the flags through pinned host memory, so one context runs
// without a bubble between chunks and several contexts (msmg_solve_batched)
// interleave on their own streams.
#include "msmg_internal.cuh"
#include "reduce.cuh"
#include <cmath>
#include <vector>
#include <algorithm>

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

// doubles between the PcgScalars records of consecutive right-hand sides
static_assert(sizeof(PcgScalars) % sizeof(double) == 0, "PcgScalars must be a whole number of doubles");
constexpr int64_t kScStride = sizeof(PcgScalars) / sizeof(double);

// grid-stride loop over one right-hand side's slice of a batched launch
#define MSMG_RHS_LOOP(i, bi, n) \
  for (int64_t i = (int64_t)(bi).blk * blockDim.x + threadIdx.x; i < (n); i += (int64_t)(bi).nblk * blockDim.x)

// out[r * ostride] = scale * sum(b_r)
__global__ void k_sum(const double* __restrict__ b, int64_t n, RedSlot red, double* out, int64_t ostride,
                      double scale, int R) {
  const BatchIdx bi = batch_idx(R);
  b += (int64_t)bi.r * n;
  out += (int64_t)bi.r * ostride;
  double v[1] = {0.0};
  MSMG_RHS_LOOP(i, bi, n) v[0] += b[i];
  grid_reduce_r<1>(v, red, bi, [=] __device__(double* t) { *out = t[0] * scale; });
}

// b -= mean; r = b; x = 0; bb = b.b (initial residual for a zero guess)
__global__ void k_init_zero(double* __restrict__ b, double* __restrict__ r, double* __restrict__ x, int64_t n,
                            RedSlot red, PcgScalars* sc, double rtol2, int R) {
  const BatchIdx bi = batch_idx(R);
  sc += bi.r;
  {
    const int64_t off = (int64_t)bi.r * n;
    b += off; r += off; x += off;
  }
  const double mean = sc->mean;
  double v[1] = {0.0};
  MSMG_RHS_LOOP(i, bi, n) {
    const double bi_ = b[i] - mean;
    b[i] = bi_;
    r[i] = bi_;
    x[i] = 0.0;
    v[0] += bi_ * bi_;
  }
  grid_reduce_r<1>(v, red, bi, [=] __device__(double* t) {
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
                          RedSlot red, PcgScalars* sc, double rtol2, int R) {
  const BatchIdx bi = batch_idx(R);
  sc += bi.r;
  {
    const int64_t off = (int64_t)bi.r * n;
    b += off; r += off; q += off;
  }
  const double mean = sc->mean;
  double v[2] = {0.0, 0.0};
  MSMG_RHS_LOOP(i, bi, n) {
    const double bi_ = b[i] - mean;
    b[i] = bi_;
    const double ri = bi_ - q[i];
    r[i] = ri;
    v[0] += bi_ * bi_;
    v[1] += ri * ri;
  }
  grid_reduce_r<2>(v, red, bi, [=] __device__(double* t) {
    sc->bb = t[0];
    sc->tol2 = rtol2 * t[0];
    sc->rr = t[1];
    sc->iter = 0;
    sc->rz = 0.0;
    sc->pq = 0.0;
    sc->done = (t[1] <= sc->tol2 || t[0] == 0.0) ? 1 : 0;
  });
}

// residual replacement for the right-hand sides with mask[r] != 0:
// r = b - q (q = A x), rr; restart the recurrence
__global__ void k_restart(const double* __restrict__ b, const double* __restrict__ q, double* __restrict__ r,
                          int64_t n, RedSlot red, PcgScalars* sc, const int* __restrict__ mask, int R) {
  const BatchIdx bi = batch_idx(R);
  if (!mask[bi.r]) return;
  sc += bi.r;
  {
    const int64_t off = (int64_t)bi.r * n;
    b += off; q += off; r += off;
  }
  double v[1] = {0.0};
  MSMG_RHS_LOOP(i, bi, n) {
    const double ri = b[i] - q[i];
    r[i] = ri;
    v[0] += ri * ri;
  }
  grid_reduce_r<1>(v, red, bi, [=] __device__(double* t) {
    sc->rr = t[0];
    sc->rz = 0.0;
    sc->pq = 0.0;
    sc->beta = 0.0;
    sc->done = t[0] <= sc->tol2 ? 1 : 0;
  });
}

// x_r -= scale * sum[r * sstride]
__global__ void k_sub_scalar(double* __restrict__ x, int64_t n, const double* sum, int64_t sstride, double scale,
                             int R) {
  const BatchIdx bi = batch_idx(R);
  x += (int64_t)bi.r * n;
  const double m = sum[(int64_t)bi.r * sstride] * scale;
  MSMG_RHS_LOOP(i, bi, n) x[i] -= m;
}

// out[2 r] = ||b_r - q_r||^2
__global__ void k_resid_norm(const double* __restrict__ b, const double* __restrict__ q, int64_t n, RedSlot red,
                             double* out, int R) {
  const BatchIdx bi = batch_idx(R);
  {
    const int64_t off = (int64_t)bi.r * n;
    b += off; q += off;
  }
  out += 2 * bi.r;
  double v[1] = {0.0};
  MSMG_RHS_LOOP(i, bi, n) {
    const double d = b[i] - q[i];
    v[0] += d * d;
  }
  grid_reduce_r<1>(v, red, bi, [=] __device__(double* t) { *out = t[0]; });
}

__global__ void k_dot(const double* __restrict__ a, const double* __restrict__ b, int64_t n, RedSlot red,
                      double* out) {
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[0] += a[i] * b[i];
  grid_reduce<1>(v, red, [=] __device__(double* t) { *out = t[0]; });
}

__global__ void k_set_scalars(PcgScalars* sc, int max_iter, int flexible, int R) {
  const int r = threadIdx.x;
  if (r >= R) return;
  sc[r].max_iter = max_iter;
  sc[r].flexible = flexible;
  sc[r].done = 0;
  sc[r].iter = 0;
  sc[r].mean = 0.0;   // stays 0 when A has a cell term (nonsingular: no mean to remove)
}

void launch_dot(const double* a, const double* b, int64_t n, RedSlot red, double* out, cudaStream_t s) {
  k_dot<<<vec_grid(n), kVecThreads, 0, s>>>(a, b, n, red, out);
}

// Capture two consecutive PCG iterations (p0 -> p1 -> p0) of the current batch
// width into a CUDA graph on a private stream.  Returns 1 when the graph is
// ready, -1 when capture is not possible (the caller then launches kernel by
// kernel).
static int build_iteration_graph(msmg_ctx* c) {
  SolveBuffers& B = c->sb;
  if (c->graph_state == 1 && c->graph_R == B.R) return 1;
  if (c->graph_state == -1) return -1;
  if (c->graph_state == 1) {
    cudaGraphExecDestroy(c->iter_graph);
    c->graph_state = 0;
  }
  const bool flexible = c->opts.precision == MSMG_MIXED;
  c->graph_state = -1;
  if (!c->cap_stream && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return -1;
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
  c->graph_R = B.R;
  return 1;
}

// One PCG solve of the batch of R right-hand sides already in block-major order
// in c->sb.b (FP64); x in c->sb.x (initial guess if use_x0).
//   init:      r0 = b - A x0 (mean removed), z0 = P^{-1} r0, beta = 0
//   iteration: p = z + beta p; q = A p; alpha = r.z / p.q        (k_pmatvec)
//              x += alpha p; r -= alpha q; stop on ||r|| <= rtol ||b||   (k_pre)
//              z = P^{-1} r; beta = r.z / r_old.z_old, or the flexible
//              (Polak-Ribiere) beta in the mixed form                (V-cycle)
//   exit:      the recurrence residual can drift from b - A x (FP32 V-cycle,
//              flexible beta): the true residual is checked in FP64 and, where
//              it is above the tolerance, replaces the recurrence residual and
//              the iteration continues (at most twice)
struct PcgRun {
  enum Phase { kIter, kCheck, kFinal, kDone };
  static constexpr int kChunk = 4;   // iterations per chunk (two graph launches)

  msmg_ctx* c = nullptr;
  cudaStream_t s = nullptr;
  int R = 1;
  double rtol = 0;
  int max_iter = 0;
  bool use_x0 = false;
  bool flexible = false;
  bool graph = false;
  Phase phase = kIter;
  int64_t launches = 0;
  int64_t vc_launches = 0;
  int launched = 0;        // iterations launched since the last (re)start
  int budget = 0;          // iterations that may still be launched
  int inflight = 0;        // chunks whose poll is outstanding (0, 1, 2)
  int head = 0;            // ring slot of the oldest outstanding chunk
  bool stop_launch = false;
  int restarts[MSMG_MAX_BATCH_RHS] = {};   // residual replacements per right-hand side

  PcgScalars* hsc_ring(int k) const { return c->hsc + (size_t)(1 + k) * c->max_rhs; }
  PcgScalars* hsc_last() const { return c->hsc; }
  cudaEvent_t ring_ev(int k) const { return c->poll_evs[k]; }

  int start() {
    SolveBuffers& B = c->sb;
    const int64_t n = c->n;
    const unsigned vg = vec_grid(n) * R;
    PcgScalars* sc = B.sc;
    flexible = c->opts.precision == MSMG_MIXED;
    vc_launches = 4 + 4 * (int64_t)(c->nL - 2) + 1;
    k_set_scalars<<<1, 32 * ((R + 31) / 32), 0, s>>>(sc, max_iter, flexible ? 1 : 0, R);
    // compatibility condition (Section 2.1) of the singular system; a cell term
    // (wells) makes A nonsingular and the right-hand side is taken as it is
    if (!c->fine.Wd) k_sum<<<vg, kVecThreads, 0, s>>>(B.b, n, c->red, &sc->mean, kScStride, 1.0 / (double)n, R);
    if (use_x0) {
      launch_matvec(c, B.x, B.q, s, R);
      k_init_x0<<<vg, kVecThreads, 0, s>>>(B.b, B.r, B.q, n, c->red, sc, rtol * rtol, R);
    } else {
      k_init_zero<<<vg, kVecThreads, 0, s>>>(B.b, B.r, B.x, n, c->red, sc, rtol * rtol, R);
    }
    launches += 3 + (use_x0 ? 2 : 1);
    MSMG_CUDA_TRY(cudaGetLastError());
    return restart_recurrence(max_iter);
  }

  // zero search direction and z = P^{-1} r for every right-hand side still running
  int restart_recurrence(int new_budget) {
    SolveBuffers& B = c->sb;
    MSMG_CUDA_TRY(cudaMemsetAsync(B.p0, 0, (size_t)R * c->n * sizeof(double), s));
    B.pcur = B.p0;
    B.pnext = B.p1;
    pcg_step_vcycle(c, 0, nullptr, B.sc, s);
    launches += 1 + vc_launches;
    launched = 0;
    budget = new_budget;
    inflight = 0;
    head = 0;
    stop_launch = budget <= 0;
    phase = kIter;
    MSMG_CUDA_TRY(cudaGetLastError());
    return 0;
  }

  int launch_chunk() {
    SolveBuffers& B = c->sb;
    int todo = budget - launched;
    if (todo > kChunk) todo = kChunk;
    if (graph) {
      // two iterations per graph launch (the p buffers alternate); kernels are
      // no-ops once a right-hand side's flag is set, so the counts stay exact
      for (int it = 0; it < todo; it += 2) {
        MSMG_CUDA_TRY(cudaGraphLaunch(c->iter_graph, s));
        launches += 2 * (1 + vc_launches);
      }
      launched += (todo + 1) / 2 * 2;
    } else {
      for (int it = 0; it < todo; ++it) {
        pcg_step_pmatvec(c, B.sc, s);
        double* t = B.pcur; B.pcur = B.pnext; B.pnext = t;
        pcg_step_vcycle(c, 1, flexible ? B.q : nullptr, B.sc, s);
        launches += 1 + vc_launches;
      }
      launched += todo;
    }
    const int slot = (head + inflight) % 2;
    MSMG_CUDA_TRY(cudaMemcpyAsync(hsc_ring(slot), B.sc, (size_t)R * sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
    MSMG_CUDA_TRY(cudaEventRecord(ring_ev(slot), s));
    ++inflight;
    if (launched >= budget) stop_launch = true;
    return 0;
  }

  // 1 when the event has completed, 0 when not yet (non-blocking), < 0 on error
  int wait(cudaEvent_t ev, bool block) {
    cudaError_t e = block ? cudaEventSynchronize(ev) : cudaEventQuery(ev);
    if (e == cudaSuccess) return 1;
    if (e == cudaErrorNotReady) return 0;
    set_last_cuda_error(e);
    return MSMG_ERR_CUDA;
  }

  bool all_done(const PcgScalars* h) const {
    for (int r = 0; r < R; ++r)
      if (!h[r].done) return false;
    return true;
  }

  // Advance the solve.  Returns 1 when finished, 0 when more work is pending,
  // < 0 on a CUDA error.  With block, waits for the device where needed.
  int step(bool block) {
    SolveBuffers& B = c->sb;
    const int64_t n = c->n;
    const unsigned vg = vec_grid(n) * R;
    switch (phase) {
      case kIter: {
        while (inflight < 2 && !stop_launch) {
          int st = launch_chunk();
          if (st) return st;
        }
        if (inflight == 0) {
          phase = kCheck;
          return enqueue_check();
        }
        int w = wait(ring_ev(head), block);
        if (w <= 0) return w;
        std::copy(hsc_ring(head), hsc_ring(head) + R, hsc_last());
        head = (head + 1) % 2;
        --inflight;
        if (all_done(hsc_last())) stop_launch = true;
        if (stop_launch && inflight == 0) {
          phase = kCheck;
          return enqueue_check();
        }
        return 0;
      }
      case kCheck: {
        int w = wait(c->poll_evs[2], block);
        if (w <= 0) return w;
        const PcgScalars* h = hsc_last();
        bool any = false;
        int min_iter = max_iter;
        for (int r = 0; r < R; ++r) {
          const bool need = h[r].done == 1 && c->hres[2 * r] > h[r].tol2 && h[r].iter < max_iter;
          c->hmask[r] = (need && restarts[r] < 2) ? 1 : 0;
          if (c->hmask[r]) {
            any = true;
            ++restarts[r];
            if (h[r].iter < min_iter) min_iter = h[r].iter;
          }
        }
        if (any) {
          MSMG_CUDA_TRY(cudaMemcpyAsync(B.dmask, c->hmask, (size_t)R * sizeof(int), cudaMemcpyHostToDevice, s));
          k_restart<<<vg, kVecThreads, 0, s>>>(B.b, B.q, B.r, n, c->red, B.sc, B.dmask, R);
          launches += 1;
          return restart_recurrence(max_iter - min_iter);
        }
        // zero-mean solution (uniqueness condition, Section 2.1)
        if (!c->fine.Wd) {
          k_sum<<<vg, kVecThreads, 0, s>>>(B.x, n, c->red, B.dres + 1, 2, 1.0, R);
          k_sub_scalar<<<vg, kVecThreads, 0, s>>>(B.x, n, B.dres + 1, 2, 1.0 / (double)n, R);
          launches += 2;
        }
        MSMG_CUDA_TRY(cudaEventRecord(c->poll_evs[2], s));
        phase = kFinal;
        return 0;
      }
      case kFinal: {
        int w = wait(c->poll_evs[2], block);
        if (w <= 0) return w;
        phase = kDone;
        return 1;
      }
      default:
        return 1;
    }
  }

  // true residual of every right-hand side and the latest scalars to the host
  int enqueue_check() {
    SolveBuffers& B = c->sb;
    const int64_t n = c->n;
    const unsigned vg = vec_grid(n) * R;
    launch_matvec(c, B.x, B.q, s, R);
    k_resid_norm<<<vg, kVecThreads, 0, s>>>(B.b, B.q, n, c->red, B.dres, R);
    launches += 2;
    MSMG_CUDA_TRY(cudaMemcpyAsync(hsc_last(), B.sc, (size_t)R * sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
    MSMG_CUDA_TRY(cudaMemcpyAsync(c->hres, B.dres, (size_t)2 * R * sizeof(double), cudaMemcpyDeviceToHost, s));
    // error words: [5] cooperative coarse cycle not launched, [6] a bounded wait gave up
    MSMG_CUDA_TRY(cudaMemcpyAsync(c->hmask + c->max_rhs, c->flags + 5, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    MSMG_CUDA_TRY(cudaEventRecord(c->poll_evs[2], s));
    return 0;
  }

  int finish(msmg_solve_info* info) const {
    if (c->hmask[c->max_rhs]) {
      set_last_cuda_error(cudaErrorLaunchFailure);   // the cooperative coarse cycle did not run
      return MSMG_ERR_CUDA;
    }
    if (c->hmask[c->max_rhs + 1]) return MSMG_ERR_DEVICE_TIMEOUT;   // staged data never landed
    const PcgScalars* h = hsc_last();
    int worst = MSMG_OK;
    for (int r = 0; r < R; ++r) {
      if (info) {
        msmg_solve_info& I = info[r];
        I.iterations = h[r].iter;
        I.converged = h[r].done == 1;
        I.rel_residual = h[r].bb > 0 ? std::sqrt(h[r].rr / h[r].bb) : 0.0;
        I.true_rel_residual = h[r].bb > 0 ? std::sqrt(c->hres[2 * r] / h[r].bb) : 0.0;
        I.rhs_mean = h[r].mean;
        I.kernel_launches = launches;
      }
      if (h[r].done == 2) worst = MSMG_ERR_BREAKDOWN;
      else if (h[r].done != 1 && worst == MSMG_OK) worst = MSMG_NOT_CONVERGED;
    }
    return worst;
  }
};

// Copy the batch's right-hand sides (and initial guesses) into block-major order.
static int stage_in(msmg_ctx* c, const double* rhs, const double* x, int R, bool host, bool x0, cudaStream_t s,
                    int64_t* launches) {
  SolveBuffers& B = c->sb;
  const int64_t n = c->n;
  if (host) {
    // natural-order staging through q
    MSMG_CUDA_TRY(cudaMemcpyAsync(B.q, rhs, (size_t)R * n * sizeof(double), cudaMemcpyHostToDevice, s));
    for (int r = 0; r < R; ++r) launch_nat_to_blk(c, B.q + r * n, B.b + r * n, s);
    if (x0) {
      MSMG_CUDA_TRY(cudaMemcpyAsync(B.q, x, (size_t)R * n * sizeof(double), cudaMemcpyHostToDevice, s));
      for (int r = 0; r < R; ++r) launch_nat_to_blk(c, B.q + r * n, B.x + r * n, s);
    }
  } else {
    for (int r = 0; r < R; ++r) launch_nat_to_blk(c, rhs + r * n, B.b + r * n, s);
    if (x0)
      for (int r = 0; r < R; ++r) launch_nat_to_blk(c, x + r * n, B.x + r * n, s);
  }
  *launches += (int64_t)R * (x0 ? 2 : 1);
  MSMG_CUDA_TRY(cudaGetLastError());
  return 0;
}

static int stage_out(msmg_ctx* c, double* x, int R, bool host, cudaStream_t s, int64_t* launches) {
  SolveBuffers& B = c->sb;
  const int64_t n = c->n;
  if (host) {
    for (int r = 0; r < R; ++r) launch_blk_to_nat(c, B.x + r * n, B.q + r * n, s);
    MSMG_CUDA_TRY(cudaMemcpyAsync(x, B.q, (size_t)R * n * sizeof(double), cudaMemcpyDeviceToHost, s));
  } else {
    for (int r = 0; r < R; ++r) launch_blk_to_nat(c, B.x + r * n, x + r * n, s);
  }
  *launches += R;
  MSMG_CUDA_TRY(cudaGetLastError());
  return 0;
}

// A solve in progress on one context: its batches of right-hand sides, one at a time.
struct CtxSolve {
  msmg_ctx* c;
  const double* rhs;
  double* x;
  int n_rhs;
  int next = 0;          // first right-hand side of the current batch
  int R = 0;
  PcgRun run;
  bool active = false;
  bool finished = false;
  int worst = MSMG_OK;
  int64_t stage_launches = 0;
  cudaEvent_t t0 = nullptr;
};

static int begin_batch(CtxSolve& J, double rtol, int max_iter, int flags, cudaStream_t s) {
  msmg_ctx* c = J.c;
  const bool host = flags & MSMG_FLAG_HOST_IO, x0 = flags & MSMG_FLAG_X0;
  J.R = J.n_rhs - J.next < c->max_rhs ? J.n_rhs - J.next : c->max_rhs;
  c->sb.R = J.R;
  J.stage_launches = 0;
  MSMG_CUDA_TRY(cudaEventRecord(c->ev0, s));
  MSMG_CUDA_TRY(cudaMemsetAsync(c->flags + 6, 0, sizeof(int), s));
  if (c->sb.iiters) MSMG_CUDA_TRY(cudaMemsetAsync(c->sb.iiters, 0, (size_t)J.R * sizeof(int), s));
  int st = stage_in(c, J.rhs + (int64_t)J.next * c->n, J.x + (int64_t)J.next * c->n, J.R, host, x0, s,
                    &J.stage_launches);
  if (st) return st;
  J.run = PcgRun{};
  J.run.c = c;
  J.run.s = s;
  J.run.R = J.R;
  J.run.rtol = rtol;
  J.run.max_iter = max_iter;
  J.run.use_x0 = x0;
  J.run.graph = !(flags & MSMG_FLAG_NO_GRAPH) && build_iteration_graph(c) == 1;
  J.active = true;
  return J.run.start();
}

static int end_batch(CtxSolve& J, int flags, cudaStream_t s, msmg_solve_info* info) {
  msmg_ctx* c = J.c;
  const bool host = flags & MSMG_FLAG_HOST_IO;
  int st = stage_out(c, J.x + (int64_t)J.next * c->n, J.R, host, s, &J.stage_launches);
  if (st) return st;
  MSMG_CUDA_TRY(cudaEventRecord(c->ev1, s));
  MSMG_CUDA_TRY(cudaEventSynchronize(c->ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  msmg_solve_info* I = info ? info + J.next : nullptr;
  const int res = J.run.finish(I);
  int inner[MSMG_MAX_BATCH_RHS] = {};
  if (I && c->sb.iiters)
    MSMG_CUDA_TRY(cudaMemcpy(inner, c->sb.iiters, (size_t)J.R * sizeof(int), cudaMemcpyDeviceToHost));
  if (I)
    for (int r = 0; r < J.R; ++r) {
      I[r].kernel_launches += J.stage_launches;
      I[r].solve_ms = ms;
      I[r].inner_iterations = inner[r];
    }
  if (res < 0) return res;
  if (res > J.worst) J.worst = res;
  J.next += J.R;
  J.active = false;
  J.finished = J.next >= J.n_rhs;
  return 0;
}

// Solve n_rhs systems on one context, max_rhs at a time, on stream s.
int pcg_solve(msmg_ctx* c, const double* rhs, double* x, int n_rhs, double rtol, int max_iter, int flags,
              cudaStream_t s, msmg_solve_info* info) {
  CtxSolve J{c, rhs, x, n_rhs};
  while (!J.finished) {
    int st = begin_batch(J, rtol, max_iter, flags, s);
    if (st) return st;
    for (;;) {
      st = J.run.step(true);
      if (st < 0) return st;
      if (st == 1) break;
    }
    st = end_batch(J, flags, s, info);
    if (st) return st;
  }
  return J.worst;
}

// Solve the systems of several contexts together: each context runs on its own
// stream (forked from s and joined back), and the host advances whichever
// context's device work has completed, so small problems overlap.
int pcg_solve_batched(msmg_ctx* const* ctxs, int n_ctx, const double* const* rhs, double* const* x,
                      const int* n_rhs, double rtol, int max_iter, int flags, cudaStream_t s,
                      msmg_solve_info* info) {
  std::vector<CtxSolve> jobs;
  std::vector<int64_t> info_off(n_ctx + 1, 0);
  for (int k = 0; k < n_ctx; ++k) info_off[k + 1] = info_off[k] + n_rhs[k];
  cudaEvent_t fork = nullptr;
  MSMG_CUDA_TRY(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  MSMG_CUDA_TRY(cudaEventRecord(fork, s));
  for (int k = 0; k < n_ctx; ++k) {
    msmg_ctx* c = ctxs[k];
    if (!c->run_stream) MSMG_CUDA_TRY(cudaStreamCreateWithFlags(&c->run_stream, cudaStreamNonBlocking));
    MSMG_CUDA_TRY(cudaStreamWaitEvent(c->run_stream, fork, 0));
    jobs.push_back(CtxSolve{c, rhs[k], x[k], n_rhs[k]});
  }
  int err = 0;
  size_t left = jobs.size();
  for (auto& J : jobs) {
    if (J.n_rhs <= 0) { J.finished = true; --left; }
  }
  // round robin: start batches, advance without blocking, finish batches
  while (left > 0 && !err) {
    bool progressed = false;
    for (size_t k = 0; k < jobs.size() && !err; ++k) {
      CtxSolve& J = jobs[k];
      if (J.finished) continue;
      if (!J.active) {
        err = begin_batch(J, rtol, max_iter, flags, J.c->run_stream);
        progressed = true;
        continue;
      }
      const int st = J.run.step(false);
      if (st < 0) { err = st; break; }
      if (st == 1) {
        err = end_batch(J, flags, J.c->run_stream, info ? info + info_off[k] : nullptr);
        if (J.finished) --left;
        progressed = true;
      }
    }
    if (!progressed && !err) {
      // nothing completed in this pass: block on the oldest outstanding work of one context
      for (auto& J : jobs) {
        if (J.finished || !J.active) continue;
        const int st = J.run.step(true);
        if (st < 0) err = st;
        break;
      }
    }
  }
  int worst = MSMG_OK;
  for (auto& J : jobs) {
    cudaEvent_t join = nullptr;
    if (cudaEventCreateWithFlags(&join, cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(join, J.c->run_stream);
      cudaStreamWaitEvent(s, join, 0);
      cudaEventDestroy(join);
    }
    if (J.worst > worst) worst = J.worst;
  }
  cudaEventDestroy(fork);
  if (err) return err;
  return worst;
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
