// Two-phase flow by the improved IMPES scheme (Section 6): the pieces that run
// on the GPU around the pressure solve.
//
// Fluid model (Section 6): S* = (S - s_wc) / (1 - s_wc - s_or) clipped to
// [0, 1], relative permeabilities k_rw = S*^2 and k_ro = (1 - S*)^2, total
// mobility lambda = k_rw / mu_w + k_ro / mu_o, water fractional flow
// f_w = (k_rw / mu_w) / lambda.
//
// Pressure step, Eq. (IMP): div(-lambda(S^n) K grad p) = q(p).  Its two-point
// discretisation is the pressure system of this library with the permeability
// lambda(S^n) kappa (face coefficients harmonic averages of it), plus the
// producers' well terms: at a cell a producer crosses, q = W (p_BH - p) with
// W = WI kappa^x lambda, WI the well index.  So the system is (A + W) p = b,
// b = q_inj + W p_BH, W the library's cell term (options.cell_diag).
//
// Saturation sub-steps, Eq. (ES): phi (S^{m+1} - S^m) / dt + div(f_w(S^m) v) =
// q_w with the face flux f_w(S_up) v of the upstream cell (the cell the flow
// leaves) and q_w = q_inj at the injector, f_w(S) W (p_BH - p) at a producer;
// dt = DS_max / max |dS/dt| so that no cell changes by more than DS_max.
#include "msmg_internal.cuh"
#include "reduce.cuh"
#include <cmath>

namespace msmg {

struct Fluid {
  double mu_w, mu_o, s_wc, s_or;
};
__device__ __forceinline__ void fluid_eval(const Fluid& F, double S, double* lam, double* fw) {
  double s = (S - F.s_wc) / (1.0 - F.s_wc - F.s_or);
  s = s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
  const double mw = s * s / F.mu_w, mo = (1.0 - s) * (1.0 - s) / F.mu_o;
  *lam = mw + mo;
  *fw = mw / (mw + mo);
}

__global__ void k_pressure_terms(int64_t n, Fluid F, const double* __restrict__ S, const double* __restrict__ kappa,
                                 const double* __restrict__ wi, const double* __restrict__ q_inj, double p_bh,
                                 double* __restrict__ kappa_eff, double* __restrict__ w, double* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double lam, fw;
  fluid_eval(F, S[i], &lam, &fw);
  for (int d = 0; d < 3; ++d) kappa_eff[(int64_t)d * n + i] = lam * kappa[(int64_t)d * n + i];
  const double wc = wi[i] * kappa[i] * lam;
  w[i] = wc;
  b[i] = q_inj[i] + wc * p_bh;
}

// f_w of every cell at the sub-step's saturation: one evaluation of the fluid
// model per cell (the face fluxes read it for both sides of every face; evaluated
// there, its four FP64 divisions per face side made a sub-step FP64-bound)
__global__ void k_frac_flow(int64_t n, Fluid F, const double* __restrict__ S, double* __restrict__ fw) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double lam, f;
    fluid_eval(F, S[i], &lam, &f);
    fw[i] = f;
  }
}

// dS/dt of every cell into rate (natural order) and max |dS/dt| -> sc[0] = dt
__global__ void k_sat_rate(int nx, int ny, int nz, double hx, double hy, double hz,
                           const double* __restrict__ v, const double* __restrict__ p, const double* __restrict__ w,
                           double p_bh, const double* __restrict__ q_inj, const double* __restrict__ phi,
                           const double* __restrict__ fw, double* __restrict__ rate, RedSlot red, double ds_max,
                           double* sc) {
  const int64_t n = (int64_t)nx * ny * nz;
  const int64_t st[3] = {1, nx, (int64_t)nx * ny};
  const double h[3] = {hx, hy, hz};
  double vmax[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int gc[3] = {(int)(i % nx), (int)((i / nx) % ny), (int)(i / ((int64_t)nx * ny))};
    const int nn[3] = {nx, ny, nz};
    const double fwi = fw[i];
    double div = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double fp = 0.0, fm = 0.0;
      if (gc[d] + 1 < nn[d]) {                       // +d face: upstream is i when v >= 0
        const double vf = v[(int64_t)d * n + i];
        const double fw2 = vf >= 0.0 ? fwi : fw[i + st[d]];
        fp = fw2 * vf;
      }
      if (gc[d] > 0) {                               // -d face = +d face of the -d neighbour
        const double vf = v[(int64_t)d * n + i - st[d]];
        const double fw2 = vf >= 0.0 ? fw[i - st[d]] : fwi;
        fm = fw2 * vf;
      }
      div += (fp - fm) / h[d];
    }
    const double qw = q_inj[i] + fwi * w[i] * (p_bh - p[i]);
    const double r = (qw - div) / phi[i];
    rate[i] = r;
    vmax[0] = fmax(vmax[0], fabs(r));
  }
  // the largest |rate|: a max over each CTA, then over the CTAs by the last CTA to
  // finish (ticket counter), which sets the sub-step's dt
  __shared__ double sh[32];
  double t = vmax[0];
  for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  __shared__ int am_last;
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int k = 0; k < (int)((blockDim.x + 31) >> 5); ++k) m = fmax(m, sh[k]);
    red.partials[blockIdx.x] = m;
    __threadfence();
    const unsigned tk = atomicAdd(red.counter, 1u);
    am_last = tk == gridDim.x - 1;
  }
  __syncthreads();
  if (am_last && threadIdx.x == 0) {
    __threadfence();
    double m = 0.0;
    for (unsigned k = 0; k < gridDim.x; ++k) m = fmax(m, __ldcg(&red.partials[k]));
    sc[0] = m > 0.0 ? ds_max / m : 0.0;
    *red.counter = 0u;
    __threadfence();
  }
}

// S += dt rate; sc[1] accumulates the sub-steps' dt
__global__ void k_sat_update(int64_t n, double* __restrict__ S, const double* __restrict__ rate, double* sc) {
  const double dt = sc[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    S[i] = fma(dt, rate[i], S[i]);
  if (blockIdx.x == 0 && threadIdx.x == 0) sc[1] += dt;
}

}  // namespace msmg

using namespace msmg;

extern "C" {

int msmg_impes_pressure_terms(int64_t n, const msmg_fluid* fluid, const double* S, const double* kappa,
                              const double* wi, const double* q_inj, double p_bh, double* kappa_eff, double* w,
                              double* b, msmg_stream stream) {
  if (n < 1 || !fluid || !S || !kappa || !wi || !q_inj || !kappa_eff || !w || !b) return MSMG_ERR_INVALID_ARG;
  if (!(fluid->mu_w > 0) || !(fluid->mu_o > 0) || !(fluid->s_wc >= 0) || !(fluid->s_or >= 0) ||
      !(fluid->s_wc + fluid->s_or < 1))
    return MSMG_ERR_INVALID_ARG;
  const Fluid F{fluid->mu_w, fluid->mu_o, fluid->s_wc, fluid->s_or};
  k_pressure_terms<<<(unsigned)((n + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      n, F, S, kappa, wi, q_inj, p_bh, kappa_eff, w, b);
  MSMG_CUDA_TRY(cudaGetLastError());
  return 0;
}

int msmg_impes_transport(msmg_ctx* c, const msmg_fluid* fluid, const double* v, const double* p, const double* w,
                         double p_bh, const double* q_inj, const double* phi, double* S, int M, double ds_max,
                         double* dt_host, msmg_stream stream) {
  if (!c || !fluid || !v || !p || !w || !q_inj || !phi || !S || M < 0 || !(ds_max > 0)) return MSMG_ERR_INVALID_ARG;
  if (!(fluid->mu_w > 0) || !(fluid->mu_o > 0) || !(fluid->s_wc >= 0) || !(fluid->s_or >= 0) ||
      !(fluid->s_wc + fluid->s_or < 1))
    return MSMG_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const Fluid F{fluid->mu_w, fluid->mu_o, fluid->s_wc, fluid->s_or};
  const int64_t n = c->n;
  double* rate = c->sb.z;             // scratch: the solve buffers are free between solves
  double* fw = c->sb.q;
  double* sc = c->dtmp + 12;          // [0] dt of the sub-step, [1] their sum
  unsigned grid = (unsigned)((n + 1023) / 1024);
  if (grid > 152 * 8) grid = 152 * 8;
  MSMG_CUDA_TRY(cudaMemsetAsync(sc, 0, 2 * sizeof(double), s));
  for (int m = 0; m < M; ++m) {
    k_frac_flow<<<grid, 256, 0, s>>>(n, F, S, fw);
    k_sat_rate<<<grid, 256, 0, s>>>(c->grid.nx, c->grid.ny, c->grid.nz, c->grid.hx, c->grid.hy, c->grid.hz, v, p, w,
                                    p_bh, q_inj, phi, fw, rate, c->red, ds_max, sc);
    k_sat_update<<<grid, 256, 0, s>>>(n, S, rate, sc);
  }
  MSMG_CUDA_TRY(cudaGetLastError());
  if (dt_host) {
    MSMG_CUDA_TRY(cudaMemcpyAsync(dt_host, sc + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    MSMG_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return 0;
}

}  // extern "C"
