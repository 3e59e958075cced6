// Velocity recovery after a pressure solve and the discrete mass-balance check
// (Section 2.2).  Eliminating the velocity gave A = B M_t^{-1} B^T (Eq. (p));
// the velocity comes back as v = M_t^{-1} B^T p, which with the trapezoidal
// rule is the two-point flux of Eq. (velocity): on the face between cell i and
// its +d neighbour j,
//     v_f = -kappa_f (p_j - p_i) / h_d = -T_f h_d (p_j - p_i),
// T_f = kappa_f / h_d^2 the harmonic-average face coefficient (Fig. (kappa
// edge)); boundary faces carry no flow.  Mass conservation on a cell (the
// identity the paper derives from Eq. (discrete varia), in three directions):
//     sum_d (v_{i+e_d/2} - v_{i-e_d/2}) / h_d = f_i,
// the left side being (A p)_i.  The kernel walks the cells in block-major order
// (where the face coefficients live) and reads p and f in natural order.
#include "msmg_internal.cuh"
#include "reduce.cuh"
#include <cmath>

namespace msmg {

static constexpr int kVelThreads = 256;

static inline unsigned vel_grid(int64_t n) {
  int64_t g = (n + kVelThreads * 4 - 1) / (kVelThreads * 4);
  if (g > 152 * 8) g = 152 * 8;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// out[0] = sum_i f_i / n
__global__ void k_vel_mean(const double* __restrict__ f, int64_t n, RedSlot red, double* out) {
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[0] += f[i];
  grid_reduce<1>(v, red, [=] __device__(double* t) { out[0] = t[0] / (double)n; });
}

// v[d][c] for the +d face of every cell c (natural order), and the balance
// sums out[1] = sum_i (div_i - b_i)^2, out[2] = sum_i b_i^2, b = f - mean(f).
__global__ void k_velocity(const double* __restrict__ p, const double* __restrict__ f, const double* __restrict__ T,
                           const double* __restrict__ Wd,
                           int nx, int ny, int nz, double hx, double hy, double hz, int bx, int by, int bz,
                           const int* __restrict__ lex_of_hid, const int* __restrict__ nbr, int gx, int gy,
                           double* __restrict__ v, RedSlot red, double* out) {
  const int64_t n = (int64_t)nx * ny * nz;
  const int nb = bx * by * bz;
  const double mean = out[0];
  double acc[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / nb;
    const int q = (int)(i % nb);
    const int lex = lex_of_hid[e];
    const int ex = lex % gx, ey = (lex / gx) % gy, ez = lex / (gx * gy);
    const int lc[3] = {q % bx, (q / bx) % by, q / (bx * by)};
    const int gc[3] = {ex * bx + lc[0], ey * by + lc[1], ez * bz + lc[2]};
    const int nn[3] = {nx, ny, nz}, bd[3] = {bx, by, bz}, lst[3] = {1, bx, bx * by};
    const double h[3] = {hx, hy, hz};
    const int64_t st[3] = {1, nx, (int64_t)nx * ny};
    const int64_t c = gc[0] + (int64_t)nx * (gc[1] + (int64_t)ny * gc[2]);
    const double pc = p[c];
    double div = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      // +d face of this cell
      double vp = 0.0;
      if (gc[d] + 1 < nn[d]) vp = -T[(int64_t)d * n + i] * h[d] * (p[c + st[d]] - pc);
      v[(int64_t)d * n + c] = vp;
      // -d face: the +d face of the -d neighbour, whose coefficient sits at that cell
      double vm = 0.0;
      if (gc[d] > 0) {
        int64_t im;
        if (lc[d] > 0) {
          im = i - lst[d];
        } else {
          const int ne = nbr[e * 6 + 2 * d];
          im = (int64_t)ne * nb + q + (int64_t)(bd[d] - 1) * lst[d];
        }
        vm = -T[(int64_t)d * n + im] * h[d] * (pc - p[c - st[d]]);
      }
      div += (vp - vm) / h[d];
    }
    // the cell's net source: f - mean (the singular system), or f - W p with a cell
    // term (wells: the flow leaves through the well, not through a face)
    const double b = Wd ? f[c] - Wd[i] * pc : f[c] - mean;
    acc[0] = fma(div - b, div - b, acc[0]);
    acc[1] = fma(b, b, acc[1]);
  }
  grid_reduce<2>(acc, red, [=] __device__(double* t) {
    out[1] = t[0];
    out[2] = t[1];
  });
}

}  // namespace msmg

using namespace msmg;

extern "C" int msmg_velocity(msmg_ctx* c, const double* p, const double* f, double* v, double* balance,
                             msmg_stream stream) {
  if (!c || !p || !f || !v) return MSMG_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const FineLevel& F = c->fine;
  double* out = c->dtmp + 8 + 1;   // [0] mean of f, [1] sum (div - b)^2, [2] sum b^2
  const unsigned grid = vel_grid(c->n);
  RedSlot red = c->red;
  k_vel_mean<<<grid, kVelThreads, 0, s>>>(f, c->n, red, out);
  k_velocity<<<grid, kVelThreads, 0, s>>>(p, f, F.T, F.Wd, c->grid.nx, c->grid.ny, c->grid.nz, c->grid.hx, c->grid.hy,
                                          c->grid.hz, F.bx, F.by, F.bz, F.lex_of_hid, F.nbr, F.gx, F.gy, v, red,
                                          out);
  MSMG_CUDA_TRY(cudaGetLastError());
  if (balance) {
    double h[3];
    MSMG_CUDA_TRY(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, s));
    MSMG_CUDA_TRY(cudaStreamSynchronize(s));
    balance[0] = std::sqrt(h[1]);
    balance[1] = std::sqrt(h[2]);
  }
  return 0;
}
