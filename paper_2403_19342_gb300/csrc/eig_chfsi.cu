// Level-1 local eigensolver for large elements (Eq. (spepb)): Chebyshev-
// filtered subspace iteration (the filtered Rayleigh-Ritz scheme of Zhou,
// Saad, Tiago and Chelikowsky, 2006), FP64, one CTA per element, everything in
// shared memory.
//
// The generalised problem A_K phi = lambda S_K phi is solved in its symmetric
// form A~ y = lambda y, A~ = S^{-1/2} A_K S^{-1/2}, phi = S^{-1/2} y.  A~ is the
// element's 7-point operator with diagonal g_c = (sum of in-element face
// coefficients) / s_c and off-diagonals -T / sqrt(s_c s_c').  Its spectrum lies
// in [0, 8] and S^{1/2} 1 spans its kernel exactly, so that vector seeds the
// block and stays in it.
//
// One outer iteration: filter the K-vector block with the degree-m Chebyshev
// polynomial that damps [theta_{K-1}, b] (b a Gershgorin bound, theta the
// current Ritz values) and is normalised at 0; orthonormalise (classical
// Gram-Schmidt, two passes); Rayleigh-Ritz with a Jacobi eigensolve of the
// K x K projected matrix; stop when the L wanted Ritz pairs have residual
// ||A~ y - theta y||_2 <= tol.  K - L guard vectors keep the convergence rate
// set by the gap to theta_{K-1}, not by clusters at the L-th eigenvalue.
//
// Starting block: the constant S^{1/2} 1 and separable cosine modes ranked by
// frequency, or, with a learned warm start, the network's guesses for
// eigenvectors 1 .. L-1 in place of the first cosines (the guard vectors stay
// cosines).  The stopping test is the same either way.
#include "msmg_internal.cuh"
#include "reduce.cuh"
#include "linalg_small.cuh"

namespace msmg {

constexpr int kKMax = 16;

// Sum over the CTA of cnt (<= kKMax) values per thread; out[0..cnt) in smem,
// valid for every thread on return.
__device__ __forceinline__ void block_sum_many(const double (&vals)[kKMax], int cnt, double* out, double* scr) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < kKMax; ++i) {
    if (i < cnt) {
      const double t = warp_sum(vals[i]);
      if (lane == 0) scr[i * 32 + warp] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double acc = 0.0;
    for (int w = 0; w < nwarp; ++w) acc += scr[threadIdx.x * 32 + w];
    out[threadIdx.x] = acc;
  }
  __syncthreads();
}

struct ElemOp {
  const double *g, *wx, *wy, *wz;
  int bx, by, bz, bxy;
  __device__ __forceinline__ double apply(const double* v, int c, int lx, int ly, int lz) const {
    double r = g[c] * v[c];
    if (lx > 0) r -= wx[c - 1] * v[c - 1];
    if (lx < bx - 1) r -= wx[c] * v[c + 1];
    if (ly > 0) r -= wy[c - bx] * v[c - bx];
    if (ly < by - 1) r -= wy[c] * v[c + bx];
    if (lz > 0) r -= wz[c - bxy] * v[c - bxy];
    if (lz < bz - 1) r -= wz[c] * v[c + bxy];
    return r;
  }
};

__device__ __forceinline__ double hash_unit(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t h = a * 0x9E3779B1u ^ (b + 0x7F4A7C15u) * 0x85EBCA77u ^ (c + 0x165667B1u) * 0xC2B2AE3Du;
  h ^= h >> 15; h *= 0x2C1B3C6Du; h ^= h >> 12; h *= 0x297A2D39u; h ^= h >> 15;
  return (double)h * (1.0 / 4294967296.0) - 0.5;
}

__global__ void __launch_bounds__(512) k_eig_l1_chfsi(const double* __restrict__ T, const double* __restrict__ S, int64_t n, int bx, int by,
                               int bz, int64_t m, int L, int K, int mdeg, int max_iter, double tol,
                               const float* __restrict__ guess, double* __restrict__ Phi, double* __restrict__ lam,
                               double* stats, int* flags) {
  extern __shared__ double sm[];
  const int nb = bx * by * bz, bxy = bx * by;
  double* g = sm;
  double* wx = g + nb;
  double* wy = wx + nb;
  double* wz = wy + nb;
  double* X = wz + nb;               // [K][nb]
  double* Y = X + K * nb;            // [K][nb]
  double* H = Y + K * nb;            // [K][K]
  double* Q = H + K * K;             // [K][K]
  double* theta = Q + K * K;         // [K]
  double* proj = theta + kKMax;      // [kKMax]
  double* scr = proj + kKMax;        // [kKMax * 32]
  double* cs = scr + kKMax * 32;     // [K + 2]
  double* red = cs + kKMax + 2;      // [72]
  double* misc = red + 72;           // [8]
  int* pr = reinterpret_cast<int*>(misc + 8);   // [K + 2]
  int* order = pr + kKMax + 2;                  // [K]
  int* modes = order + kKMax;                   // [K][3]

  const int64_t e = blockIdx.x;
  const int c = threadIdx.x;
  const bool act = c < nb;
  const int lx = act ? c % bx : 0, ly = act ? (c / bx) % by : 0, lz = act ? c / bxy : 0;
  const double* Te = T + e * nb;
  double sq = 1.0;
  if (act) {
    sq = sqrt(S[e * nb + c]);
    Y[c] = 1.0 / sq;                 // isq staged in Y for the weights
  }
  __syncthreads();
  if (act) {
    const double isq = Y[c];
    double diag = 0.0;
    double w0 = 0.0, w1 = 0.0, w2 = 0.0;
    if (lx < bx - 1) { const double t = Te[c]; diag += t; w0 = t * isq * Y[c + 1]; }
    if (lx > 0) diag += Te[c - 1];
    if (ly < by - 1) { const double t = Te[n + c]; diag += t; w1 = t * isq * Y[c + bx]; }
    if (ly > 0) diag += Te[n + c - bx];
    if (lz < bz - 1) { const double t = Te[2 * n + c]; diag += t; w2 = t * isq * Y[c + bxy]; }
    if (lz > 0) diag += Te[2 * n + c - bxy];
    g[c] = diag * isq * isq;
    wx[c] = w0; wy[c] = w1; wz[c] = w2;
  }
  // starting modes: separable cosines ranked by sum (k_d / b_d)^2 (mode 0 = constant)
  const int cx = bx < 4 ? bx : 4, cy = by < 4 ? by : 4, cz = bz < 4 ? bz : 4;
  const int ncand = cx * cy * cz;
  if (c < ncand) {
    const int kx = c % cx, ky = (c / cx) % cy, kz = c / (cx * cy);
    const double key = (double)(kx * kx) / (bx * bx) + (double)(ky * ky) / (by * by) + (double)(kz * kz) / (bz * bz);
    int rank = 0;
    for (int j = 0; j < ncand; ++j) {
      const int jx = j % cx, jy = (j / cx) % cy, jz = j / (cx * cy);
      const double kj = (double)(jx * jx) / (bx * bx) + (double)(jy * jy) / (by * by) + (double)(jz * jz) / (bz * bz);
      rank += (kj < key) || (kj == key && j < c);
    }
    if (rank < K) { modes[3 * rank] = kx; modes[3 * rank + 1] = ky; modes[3 * rank + 2] = kz; }
  }
  __syncthreads();
  const ElemOp op{g, wx, wy, wz, bx, by, bz, bxy};
  // Gershgorin upper bound of the spectrum
  {
    double v[1] = {0.0};
    if (act) {
      double r = g[c] + wx[c] + wy[c] + wz[c];
      if (lx > 0) r += wx[c - 1];
      if (ly > 0) r += wy[c - bx];
      if (lz > 0) r += wz[c - bxy];
      v[0] = r;
    }
    // max via warp shuffles
    double t = v[0];
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    if ((threadIdx.x & 31) == 0) scr[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double mx = 0.0;
      for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) mx = fmax(mx, scr[w]);
      misc[0] = mx;
    }
    __syncthreads();
  }
  const double bup = misc[0];
  const double PI = 3.141592653589793238462643383279502884;
  if (act) {
    for (int q = 0; q < K; ++q) {
      if (guess && q >= 1 && q < L) {
        X[q * nb + c] = (double)guess[((size_t)e * (L - 1) + (q - 1)) * nb + c];
        continue;
      }
      const double v = cos(PI * modes[3 * q] * (lx + 0.5) / bx) * cos(PI * modes[3 * q + 1] * (ly + 0.5) / by) *
                       cos(PI * modes[3 * q + 2] * (lz + 0.5) / bz);
      X[q * nb + c] = sq * v;
    }
  }
  __syncthreads();

  double vals[kKMax];
  int it = 0;
  double rmax = 0.0;
  for (;; ++it) {
    // ---- orthonormalise X (two-pass classical Gram-Schmidt)
    for (int j = 0; j < K; ++j) {
      for (int tries = 0; tries < 3; ++tries) {
        for (int pass = 0; pass < 2; ++pass) {
          if (j == 0) break;
#pragma unroll
          for (int i = 0; i < kKMax; ++i) vals[i] = (act && i < j) ? X[i * nb + c] * X[j * nb + c] : 0.0;
          block_sum_many(vals, j, proj, scr);
          if (act) {
            double x = X[j * nb + c];
            for (int i = 0; i < j; ++i) x -= proj[i] * X[i * nb + c];
            X[j * nb + c] = x;
          }
          __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < kKMax; ++i) vals[i] = 0.0;
        vals[0] = act ? X[j * nb + c] * X[j * nb + c] : 0.0;
        block_sum_many(vals, 1, proj, scr);
        const double nrm2 = proj[0];
        if (nrm2 > 1e-24) {
          if (act) X[j * nb + c] *= 1.0 / sqrt(nrm2);
          __syncthreads();
          break;
        }
        // collapsed: reseed deterministically and project again
        if (act) X[j * nb + c] = sq * hash_unit((uint32_t)c, (uint32_t)j, (uint32_t)(it * 4 + tries));
        __syncthreads();
      }
    }
    // ---- Rayleigh-Ritz
    if (act)
      for (int q = 0; q < K; ++q) Y[q * nb + c] = op.apply(X + q * nb, c, lx, ly, lz);
    __syncthreads();
    const int npair = K * (K + 1) / 2;
    for (int b0 = 0; b0 < npair; b0 += kKMax) {
      const int cnt = npair - b0 < kKMax ? npair - b0 : kKMax;
#pragma unroll
      for (int t = 0; t < kKMax; ++t) {
        vals[t] = 0.0;
        if (t < cnt && act) {
          // pair index -> (i, j), i <= j
          int p = b0 + t, i = 0;
          while (p >= K - i) { p -= K - i; ++i; }
          const int j = i + p;
          vals[t] = X[i * nb + c] * Y[j * nb + c];
        }
      }
      block_sum_many(vals, cnt, proj, scr);
      if (threadIdx.x < cnt) {
        int p = b0 + threadIdx.x, i = 0;
        while (p >= K - i) { p -= K - i; ++i; }
        const int j = i + p;
        H[i * K + j] = proj[threadIdx.x];
        H[j * K + i] = proj[threadIdx.x];
      }
      __syncthreads();
    }
    jacobi_eig(H, Q, K, cs, pr, red, 30, 1e-15);
    sort_diag(H, K, order);
    if (threadIdx.x < K) theta[threadIdx.x] = H[order[threadIdx.x] * K + order[threadIdx.x]];
    if (act) {
      double xn[kKMax], yn[kKMax];
#pragma unroll
      for (int j = 0; j < kKMax; ++j) { xn[j] = 0.0; yn[j] = 0.0; }
      for (int i = 0; i < K; ++i) {
        const double xi = X[i * nb + c], yi = Y[i * nb + c];
#pragma unroll
        for (int j = 0; j < kKMax; ++j) {
          if (j < K) {
            const double qij = Q[i * K + order[j]];
            xn[j] += xi * qij;
            yn[j] += yi * qij;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kKMax; ++j)
        if (j < K) { X[j * nb + c] = xn[j]; Y[j * nb + c] = yn[j]; }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kKMax; ++j) {
      vals[j] = 0.0;
      if (j < L && act) {
        const double r = Y[j * nb + c] - theta[j] * X[j * nb + c];
        vals[j] = r * r;
      }
    }
    block_sum_many(vals, L, proj, scr);
    rmax = 0.0;
    for (int j = 0; j < L; ++j) rmax = fmax(rmax, sqrt(fmax(proj[j], 0.0)));
    if (rmax <= tol || it >= max_iter) break;
    // ---- Chebyshev filter of degree mdeg on [a, bup], normalised at 0
    double a = theta[K - 1];
    if (!(a < 0.95 * bup)) a = 0.5 * bup;
    const double c0 = 0.5 * (a + bup), e0 = 0.5 * (bup - a);
    const double sig = -e0 / c0;
    double* Yc = Y;   // current  (degree j)
    double* Xp = X;   // previous (degree j-1)
    if (act)
      for (int q = 0; q < K; ++q)
        Yc[q * nb + c] = (sig / e0) * (op.apply(Xp + q * nb, c, lx, ly, lz) - c0 * Xp[q * nb + c]);
    __syncthreads();
    double sj = sig;
    for (int step = 2; step <= mdeg; ++step) {
      const double sn = 1.0 / (2.0 / sig - sj);
      if (act)
        for (int q = 0; q < K; ++q)
          Xp[q * nb + c] = (2.0 * sn / e0) * (op.apply(Yc + q * nb, c, lx, ly, lz) - c0 * Yc[q * nb + c]) -
                           sj * sn * Xp[q * nb + c];
      __syncthreads();
      double* t = Yc; Yc = Xp; Xp = t;
      sj = sn;
    }
    X = Yc;
    Y = Xp;
  }
  // ---- output: Phi = S^{-1/2} y for the L smallest
  if (act)
    for (int k = 0; k < L; ++k) Phi[(e * L + k) * nb + c] = X[k * nb + c] / sq;
  if (threadIdx.x < L) lam[e * L + threadIdx.x] = theta[threadIdx.x];
  if (threadIdx.x == 0) {
    atomic_max_pos(&stats[0], rmax);
    atomicMax(&flags[3], it);
    atomicAdd(&flags[4], it);
    if (!(rmax <= tol)) atomicExch(&flags[2], 1);
  }
}

int launch_level1_chfsi(msmg_ctx* c, cudaStream_t s, const float* guess) {
  FineLevel& f = c->fine;
  const int L = f.L;
  int guard = L / 2 > 4 ? L / 2 : 4;
  int K = L + guard;
  if (K > kKMax) K = kKMax;
  if (K > f.nb) K = f.nb;
  const int cx = f.bx < 4 ? f.bx : 4, cy = f.by < 4 ? f.by : 4, cz = f.bz < 4 ? f.bz : 4;
  if (L >= kKMax || K > cx * cy * cz || f.nb > 512) return MSMG_ERR_UNSUPPORTED;
  const int max_iter = c->opts.eig_max_iter > 0 ? c->opts.eig_max_iter : 200;
  const double tol = c->opts.eig_tol > 0 ? c->opts.eig_tol : 1e-12;
  const size_t sm = (size_t)(4 * f.nb + 2 * K * f.nb + 2 * K * K + kKMax * 2 + kKMax * 32 + kKMax + 2 + 72 + 8) *
                        sizeof(double) + (size_t)(kKMax + 2 + kKMax + 3 * kKMax) * sizeof(int) + 64;
  cudaFuncSetAttribute(k_eig_l1_chfsi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const unsigned thr = (unsigned)((f.nb + 31) / 32 * 32);
  k_eig_l1_chfsi<<<(unsigned)f.m, thr, sm, s>>>(f.T, f.S, c->n, f.bx, f.by, f.bz, f.m, L, K, 10, max_iter, tol, guess,
                                                f.Phi, f.lam, c->dtmp, c->flags);
  return 0;
}

}  // namespace msmg
