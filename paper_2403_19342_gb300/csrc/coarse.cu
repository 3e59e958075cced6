// Coarse-level steps of the V-cycle (Algorithm 1 applied on W_l, l >= 2) and
// the coarsest pseudo-inverse application, all in FP64.
//
// A_l is a block 7-point stencil: element a of E_{l-1} carries L coordinates;
// Ad[a] is its diagonal block and Ao[a][d] = A_l[a, a + e_d] its coupling to the
// +d neighbour (the -d coupling is the transpose of the neighbour's).  The
// smoother is block Jacobi over the parents (elements of E_l): one dense
// nP x nP inverse per parent, nP = children * L, applied as a GEMV.
#include "msmg_internal.cuh"

namespace msmg {

// r_i = f_i - (A_l u)_i for the rows i of one parent's children, into smem r[].
// Threads t < nP handle row t (child t / L, component t % L).
__device__ void coarse_residual_rows(const CoarseLevel& lv, int64_t P, const double* __restrict__ f,
                                     const double* __restrict__ u, double* r) {
  const int L = lv.L;
  const int t = threadIdx.x;
  if (t >= lv.nP) return;
  const int64_t a = P * lv.nchild + t / L;
  const int k = t % L;
  const int L2 = L * L;
  double acc = f[a * L + k];
  const double* ad = lv.Ad + a * L2 + (size_t)k * L;
  const double* ua = u + a * L;
  for (int mm = 0; mm < L; ++mm) acc -= ad[mm] * ua[mm];
  const int* nb = lv.nbr + a * 6;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int bp = nb[2 * d + 1];   // +d neighbour
    if (bp >= 0) {
      const double* ao = lv.Ao + ((size_t)a * 3 + d) * L2 + (size_t)k * L;
      const double* ub = u + (int64_t)bp * L;
      for (int mm = 0; mm < L; ++mm) acc -= ao[mm] * ub[mm];
    }
    const int bm = nb[2 * d];       // -d neighbour: A_l[a, bm] = Ao[bm][d]^T
    if (bm >= 0) {
      const double* ao = lv.Ao + ((size_t)bm * 3 + d) * L2 + k;
      const double* ub = u + (int64_t)bm * L;
      for (int mm = 0; mm < L; ++mm) acc -= ao[(size_t)mm * L] * ub[mm];
    }
  }
  r[t] = acc;
}

// Pre-smoothing from zero on level l: u_P = Minv_P f_P.
__global__ void k_coarse_smooth_first(CoarseLevel lv, const double* __restrict__ f, double* __restrict__ u,
                                      const PcgScalars* sc) {
  if (sc && sc->done) return;
  extern __shared__ double sm[];
  const int64_t P = blockIdx.x;
  const int nP = lv.nP;
  const int t = threadIdx.x;
  if (t < nP) sm[t] = f[P * nP + t];
  __syncthreads();
  if (t < nP) {
    const double* Mi = lv.Minv + (size_t)P * nP * nP;
    double acc = 0.0;
    for (int j = 0; j < nP; ++j) acc += Mi[(size_t)j * nP + t] * sm[j];   // Minv symmetric
    u[P * nP + t] = acc;
  }
}

// Residual and restriction to level l+1: fn[P][j] = sum_i Psi[P][j][i] (f - A_l u)_i.
__global__ void k_coarse_resid_restrict(CoarseLevel lv, const double* __restrict__ f, const double* __restrict__ u,
                                        double* __restrict__ fn, const PcgScalars* sc) {
  if (sc && sc->done) return;
  extern __shared__ double sm[];
  const int64_t P = blockIdx.x;
  coarse_residual_rows(lv, P, f, u, sm);
  __syncthreads();
  const int t = threadIdx.x;
  if (t < lv.Lnext) {
    const double* ps = lv.Psi + ((size_t)P * lv.Lnext + t) * lv.nP;
    double acc = 0.0;
    for (int i = 0; i < lv.nP; ++i) acc += ps[i] * sm[i];
    fn[P * lv.Lnext + t] = acc;
  }
}

// Prolongation: u_P += Psi_P^T e_P.
__global__ void k_coarse_prolong(CoarseLevel lv, double* __restrict__ u, const double* __restrict__ e,
                                 const PcgScalars* sc) {
  if (sc && sc->done) return;
  const int64_t P = blockIdx.x;
  const int t = threadIdx.x;
  if (t >= lv.nP) return;
  const double* ps = lv.Psi + (size_t)P * lv.Lnext * lv.nP;
  double acc = 0.0;
  for (int j = 0; j < lv.Lnext; ++j) acc += ps[(size_t)j * lv.nP + t] * e[P * lv.Lnext + j];
  u[P * lv.nP + t] += acc;
}

// Post-smoothing: out = u + Minv (f - A_l u)   (out must not alias u).
__global__ void k_coarse_resid_smooth(CoarseLevel lv, const double* __restrict__ f, const double* __restrict__ u,
                                      double* __restrict__ out, const PcgScalars* sc) {
  if (sc && sc->done) return;
  extern __shared__ double sm[];
  const int64_t P = blockIdx.x;
  coarse_residual_rows(lv, P, f, u, sm);
  __syncthreads();
  const int nP = lv.nP;
  const int t = threadIdx.x;
  if (t < nP) {
    const double* Mi = lv.Minv + (size_t)P * nP * nP;
    double acc = 0.0;
    for (int j = 0; j < nP; ++j) acc += Mi[(size_t)j * nP + t] * sm[j];
    out[P * nP + t] = u[P * nP + t] + acc;
  }
}

// Coarsest level: u = A^dagger f, dense symmetric GEMV (one warp per row group).
__global__ void k_dense_gemv(const double* __restrict__ A, const double* __restrict__ x, double* __restrict__ y,
                             int64_t n, const PcgScalars* sc) {
  if (sc && sc->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  const double* a = A + row * n;
  double acc = 0.0;
  for (int64_t j = lane; j < n; j += 32) acc += a[j] * x[j];
  acc = warp_sum(acc);
  if (lane == 0) y[row] = acc;
}

static inline unsigned coarse_threads(const CoarseLevel& lv) {
  int t = lv.nP > lv.Lnext ? lv.nP : lv.Lnext;
  return (unsigned)((t + 31) / 32 * 32);
}

// Level-l part of the V-cycle (l >= 2): on entry vf[l] holds the right side;
// returns the device pointer holding the level-l correction.
const double* coarse_cycle(msmg_ctx* c, int l, PcgScalars* sc, cudaStream_t s) {
  CoarseLevel& lv = c->lev[l];
  double* f = (double*)c->sb.vf[l];
  double* u = (double*)c->sb.vu[l];
  double* w = (double*)c->sb.vw[l];
  if (l == c->nL) {
    const unsigned grid = (unsigned)((lv.n * 32 + 255) / 256);
    k_dense_gemv<<<grid, 256, 0, s>>>(lv.pinv, f, u, lv.n, sc);
    return u;
  }
  const unsigned thr = coarse_threads(lv);
  const size_t sm = (size_t)lv.nP * sizeof(double);
  k_coarse_smooth_first<<<(unsigned)lv.mP, thr, sm, s>>>(lv, f, u, sc);
  double* fn = (double*)c->sb.vf[l + 1];
  k_coarse_resid_restrict<<<(unsigned)lv.mP, thr, sm, s>>>(lv, f, u, fn, sc);
  const double* e = coarse_cycle(c, l + 1, sc, s);
  k_coarse_prolong<<<(unsigned)lv.mP, thr, 0, s>>>(lv, u, e, sc);
  k_coarse_resid_smooth<<<(unsigned)lv.mP, thr, sm, s>>>(lv, f, u, w, sc);
  return w;
}

}  // namespace msmg
