// Level-1 local eigensolver for large elements (Eq. (spepb)): Chebyshev-
// filtered subspace iteration (the filtered Rayleigh-Ritz scheme of Zhou,
// Saad, Tiago and Chelikowsky, 2006), one CTA per element, everything in
// shared memory.  The FP64 form iterates in FP64 throughout; the mixed form
// first iterates in FP32 (vectors, filter, orthonormalisation, Rayleigh-Ritz
// projections; only the K x K eigensolve in FP64) to a residual near FP32's
// reach and then polishes the whole block in FP64 to the requested tolerance,
// so the bases it keeps are the FP64 form's to within that tolerance.
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
// valid for every thread on return.  A is the accumulation type; outr, if
// given, receives the sums (or, with rsq, their reciprocal square roots) in A,
// so that no thread converts or divides per use.
template <typename A>
__device__ __forceinline__ void block_sum_many(const A (&vals)[kKMax], int cnt, double* out, double* scr,
                                               A* outr = nullptr, bool rsq = false) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
  A* sa = reinterpret_cast<A*>(scr);
#pragma unroll
  for (int i = 0; i < kKMax; ++i) {
    if (i < cnt) {
      const A t = warp_sum_t(vals[i]);
      if (lane == 0) sa[i * 32 + warp] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    A acc = (A)0;
    for (int w = 0; w < nwarp; ++w) acc += sa[threadIdx.x * 32 + w];
    out[threadIdx.x] = (double)acc;
    if (outr) outr[threadIdx.x] = rsq ? (A)(1.0 / sqrt((double)acc)) : acc;
  }
  __syncthreads();
}

template <typename R>
struct ElemOp {
  const R *g, *wx, *wy, *wz;
  int bx, by, bz, bxy;
  __device__ __forceinline__ R apply(const R* v, int c, int lx, int ly, int lz) const {
    R r = g[c] * v[c];
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

// Shared memory: (4 + 2K) nb values of R, then the FP64 Rayleigh-Ritz work, then ints.
__host__ __device__ inline size_t chfsi_r_bytes(int nb, int K, size_t rsize) {
  return ((size_t)(4 + 2 * K) * nb * rsize + 15) / 16 * 16;
}
constexpr int kMdegMax = 32;
// R-typed scalars shared by the CTA: rotation Q (K x K, Ritz order), Ritz values,
// block sums, filter coefficients
constexpr int kRScal = kKMax * kKMax + kKMax + (kKMax + 1) + 2 + 2 * kMdegMax;
__host__ __device__ inline size_t chfsi_smem(int nb, int K, size_t rsize) {
  return chfsi_r_bytes(nb, K, rsize) +
         (size_t)(2 * K * K + kKMax * 2 + kKMax * 32 + kKMax + 2 + 72 + 8 + kRScal) * sizeof(double) +
         (size_t)(kKMax + 2 + kKMax + 3 * kKMax) * sizeof(int) + 64;
}

// R: arithmetic of the filter, orthonormalisation and residuals (FP64, or FP32
// for the first phase of the mixed form); the K x K Rayleigh-Ritz eigensolve is
// FP64 either way.
//   guess, guess_vecs   starting vectors (symmetric form, FP32): guess_vecs == L - 1
//                       fills slots 1 .. L-1 (learned warm start), == K fills every slot
//                       (the block a first phase left), 0: none
//   block_out           first phase: the K vectors of the final block (symmetric form,
//                       FP32) are written here and Phi, lam and the convergence flag
//                       are left to the second phase
template <typename R>
__global__ void __launch_bounds__(512, 2) k_eig_l1_chfsi(const double* __restrict__ T, const double* __restrict__ S,
                                                      int64_t n, int bx, int by, int bz, int64_t m, int L, int K,
                                                      int mdeg, int max_iter, double tol,
                                                      const float* __restrict__ guess, int guess_vecs,
                                                      float* __restrict__ block_out, double* __restrict__ Phi,
                                                      double* __restrict__ lam, double* stats, int* flags,
                                                      const double* __restrict__ Wd) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int nb = bx * by * bz, bxy = bx * by;
  R* g = reinterpret_cast<R*>(smraw);
  R* wx = g + nb;
  R* wy = wx + nb;
  R* wz = wy + nb;
  R* X = wz + nb;                    // [K][nb]
  R* Y = X + K * nb;                 // [K][nb]
  double* H = reinterpret_cast<double*>(smraw + chfsi_r_bytes(nb, K, sizeof(R)));   // [K][K]
  double* Q = H + K * K;             // [K][K]
  double* theta = Q + K * K;         // [K]
  double* proj = theta + kKMax;      // [kKMax]
  double* scr = proj + kKMax;        // [kKMax * 32]
  double* cs = scr + kKMax * 32;     // [K + 2]
  double* red = cs + kKMax + 2;      // [72]
  double* misc = red + 72;           // [8]
  R* Qr = reinterpret_cast<R*>(misc + 8);       // [K][K] in R, columns in Ritz order
  R* theta_r = Qr + kKMax * kKMax;              // [K]
  R* sum_r = theta_r + kKMax;                   // [kKMax + 1]
  R* coef = sum_r + kKMax + 1;                  // [2 + 2 mdeg]: sig/e, c, then (2 s_j/e, s_{j-1} s_j) per degree
  int* pr = reinterpret_cast<int*>(misc + 8 + kRScal);   // [K + 2]
  int* order = pr + kKMax + 2;                  // [K]
  int* modes = order + kKMax;                   // [K][3]

  const int64_t e = blockIdx.x;
  const int c = threadIdx.x;
  const bool act = c < nb;
  const int lx = act ? c % bx : 0, ly = act ? (c / bx) % by : 0, lz = act ? c / bxy : 0;
  const double* Te = T + e * nb;
  double sq = 1.0;
  double* isq_s = H;                 // 1 / sqrt(s) staged in the (not yet used) FP64 area
  if (act) {
    sq = sqrt(S[e * nb + c]);
    isq_s[c] = 1.0 / sq;
  }
  __syncthreads();
  if (act) {
    const double isq = isq_s[c];
    double diag = 0.0;
    double w0 = 0.0, w1 = 0.0, w2 = 0.0;
    if (lx < bx - 1) { const double t = Te[c]; diag += t; w0 = t * isq * isq_s[c + 1]; }
    if (lx > 0) diag += Te[c - 1];
    if (ly < by - 1) { const double t = Te[n + c]; diag += t; w1 = t * isq * isq_s[c + bx]; }
    if (ly > 0) diag += Te[n + c - bx];
    if (lz < bz - 1) { const double t = Te[2 * n + c]; diag += t; w2 = t * isq * isq_s[c + bxy]; }
    if (lz > 0) diag += Te[2 * n + c - bxy];
    if (Wd) diag += Wd[e * nb + c];   // cell term (wells), added to the left-hand form (Section 6)
    g[c] = (R)(diag * isq * isq);
    wx[c] = (R)w0; wy[c] = (R)w1; wz[c] = (R)w2;
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
  const ElemOp<R> op{g, wx, wy, wz, bx, by, bz, bxy};
  // Gershgorin upper bound of the spectrum
  {
    double t = 0.0;
    if (act) {
      double r = (double)g[c] + (double)wx[c] + (double)wy[c] + (double)wz[c];
      if (lx > 0) r += (double)wx[c - 1];
      if (ly > 0) r += (double)wy[c - bx];
      if (lz > 0) r += (double)wz[c - bxy];
      t = r;
    }
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
      if (guess && ((guess_vecs == K) || (guess_vecs == L - 1 && q >= 1 && q < L))) {
        const int slot = guess_vecs == K ? q : q - 1;
        X[q * nb + c] = (R)guess[((size_t)e * guess_vecs + slot) * nb + c];
        continue;
      }
      const double v = cos(PI * modes[3 * q] * (lx + 0.5) / bx) * cos(PI * modes[3 * q + 1] * (ly + 0.5) / by) *
                       cos(PI * modes[3 * q + 2] * (lz + 0.5) / bz);
      X[q * nb + c] = (R)(sq * v);
    }
  }
  __syncthreads();

  R vals[kKMax];
  int it = 0, stall = 0;
  double rmax = 0.0, rbest = 1e300;
  for (;; ++it) {
    // ---- orthonormalise X (two-pass classical Gram-Schmidt)
    for (int j = 0; j < K; ++j) {
      for (int tries = 0; tries < 3; ++tries) {
        for (int pass = 0; pass < 2; ++pass) {
          if (j == 0) break;
#pragma unroll
          for (int i = 0; i < kKMax; ++i) vals[i] = (act && i < j) ? X[i * nb + c] * X[j * nb + c] : (R)0;
          block_sum_many(vals, j, proj, scr, sum_r);
          if (act) {
            R x = X[j * nb + c];
            for (int i = 0; i < j; ++i) x -= sum_r[i] * X[i * nb + c];
            X[j * nb + c] = x;
          }
          __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < kKMax; ++i) vals[i] = (R)0;
        vals[0] = act ? X[j * nb + c] * X[j * nb + c] : (R)0;
        block_sum_many(vals, 1, proj, scr, sum_r, true);
        const double nrm2 = proj[0];
        if (nrm2 > (sizeof(R) == 4 ? 1e-12 : 1e-24)) {
          if (act) X[j * nb + c] *= sum_r[0];
          __syncthreads();
          break;
        }
        // collapsed: reseed deterministically and project again
        if (act) X[j * nb + c] = (R)(sq * hash_unit((uint32_t)c, (uint32_t)j, (uint32_t)(it * 4 + tries)));
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
        vals[t] = (R)0;
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
    if (threadIdx.x < K) {
      const double t = H[order[threadIdx.x] * K + order[threadIdx.x]];
      theta[threadIdx.x] = t;
      theta_r[threadIdx.x] = (R)t;
    }
    for (int t = threadIdx.x; t < K * K; t += blockDim.x) Qr[t] = (R)Q[(t / K) * K + order[t % K]];
    __syncthreads();
    if (act) {
      // each thread rotates its own cell of X, then of Y (one accumulator set live)
      for (int pass = 0; pass < 2; ++pass) {
        R* V = pass ? Y : X;
        R vn[kKMax];
#pragma unroll
        for (int j = 0; j < kKMax; ++j) vn[j] = (R)0;
        for (int i = 0; i < K; ++i) {
          const R vi = V[i * nb + c];
#pragma unroll
          for (int j = 0; j < kKMax; ++j)
            if (j < K) vn[j] += vi * Qr[i * K + j];
        }
#pragma unroll
        for (int j = 0; j < kKMax; ++j)
          if (j < K) V[j * nb + c] = vn[j];
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kKMax; ++j) {
      vals[j] = (R)0;
      if (j < L && act) {
        const R r = Y[j * nb + c] - theta_r[j] * X[j * nb + c];
        vals[j] = r * r;
      }
    }
    block_sum_many(vals, L, proj, scr);
    rmax = 0.0;
    for (int j = 0; j < L; ++j) rmax = fmax(rmax, sqrt(fmax(proj[j], 0.0)));
    if (rmax <= tol || it >= max_iter) break;
    // a first phase stops where its arithmetic stops making progress (three
    // iterations without a 10% gain): the second phase takes over from there
    if (block_out) {
      stall = rmax < 0.9 * rbest ? 0 : stall + 1;
      rbest = fmin(rbest, rmax);
      if (stall >= 3) break;
    }
    // ---- Chebyshev filter of degree mdeg on [a, bup], normalised at 0
    // (three-term recurrence with scaling sigma_j; the coefficients are
    // computed once by one thread)
    if (threadIdx.x == 0) {
      double a = theta[K - 1];
      if (!(a < 0.95 * bup)) a = 0.5 * bup;
      const double c0 = 0.5 * (a + bup), e0 = 0.5 * (bup - a);
      const double sig = -e0 / c0;
      coef[0] = (R)(sig / e0);
      coef[1] = (R)c0;
      double sj = sig;
      for (int step = 2; step <= mdeg; ++step) {
        const double sn = 1.0 / (2.0 / sig - sj);
        coef[2 * step - 2] = (R)(2.0 * sn / e0);
        coef[2 * step - 1] = (R)(sj * sn);
        sj = sn;
      }
    }
    __syncthreads();
    R* Yc = Y;   // current  (degree j)
    R* Xp = X;   // previous (degree j-1)
    const R cc = coef[1];
    if (act) {
      const R f0 = coef[0];
      for (int q = 0; q < K; ++q) Yc[q * nb + c] = f0 * (op.apply(Xp + q * nb, c, lx, ly, lz) - cc * Xp[q * nb + c]);
    }
    __syncthreads();
    for (int step = 2; step <= mdeg; ++step) {
      if (act) {
        const R f1 = coef[2 * step - 2], f2 = coef[2 * step - 1];
        for (int q = 0; q < K; ++q)
          Xp[q * nb + c] = f1 * (op.apply(Yc + q * nb, c, lx, ly, lz) - cc * Yc[q * nb + c]) - f2 * Xp[q * nb + c];
      }
      __syncthreads();
      R* t = Yc; Yc = Xp; Xp = t;
    }
    X = Yc;
    Y = Xp;
  }
  if (block_out) {
    // first phase: hand the whole block to the second
    if (act)
      for (int q = 0; q < K; ++q) block_out[((size_t)e * K + q) * nb + c] = (float)X[q * nb + c];
    if (threadIdx.x == 0) {
      atomicMax(&flags[3], it);
      atomicAdd(&flags[4], it);
    }
    return;
  }
  // ---- output: Phi = S^{-1/2} y for the L smallest
  if (act)
    for (int k = 0; k < L; ++k) Phi[(e * L + k) * nb + c] = (double)X[k * nb + c] / sq;
  if (threadIdx.x < L) lam[e * L + threadIdx.x] = theta[threadIdx.x];
  if (threadIdx.x == 0) {
    atomic_max_pos(&stats[0], rmax);
    atomicMax(&flags[3], it);
    atomicAdd(&flags[4], it);
    if (!(rmax <= tol)) atomicExch(&flags[2], 1);
  }
}

// Mixed form: a first FP32 phase to residual kMixedPhase1Tol (on the symmetric
// form, whose spectrum lies in [0, 8]: FP32 resolves residuals down to ~1e-6),
// then an FP64 phase from that block to eig_tol.  The FP64 form runs the FP64
// phase alone.  block is scratch for the FP32 block (m K nb floats) or null.
constexpr double kMixedPhase1Tol = 2e-5;

int launch_level1_chfsi(msmg_ctx* c, cudaStream_t s, const float* guess, float* block) {
  FineLevel& f = c->fine;
  const int L = f.L;
  int guard = L / 2 > 4 ? L / 2 : 4;
  int K = L + guard;
  if (K > kKMax) K = kKMax;
  if (K > f.nb) K = f.nb;
  const int cx = f.bx < 4 ? f.bx : 4, cy = f.by < 4 ? f.by : 4, cz = f.bz < 4 ? f.bz : 4;
  constexpr int mdeg = 10;
  static_assert(mdeg <= kMdegMax, "filter degree");
  if (L >= kKMax || K > cx * cy * cz || f.nb > 512) return MSMG_ERR_UNSUPPORTED;
  // the cap only matters for rare elements with clustered eigenvalues at the
  // cutoff: on 512^3 layered channels (262,144 elements, L = 12) one element of
  // the mixed form needs ~500 iterations; an element that iterates longer costs
  // its own CTA's time, not the launch's
  const int max_iter = c->opts.eig_max_iter > 0 ? c->opts.eig_max_iter : 1000;
  const double tol = c->opts.eig_tol > 0 ? c->opts.eig_tol : 1e-12;
  const unsigned thr = (unsigned)((f.nb + 31) / 32 * 32);
  const int guess_vecs = guess ? L - 1 : 0;
  if (block) {
    const size_t sm1 = chfsi_smem(f.nb, K, sizeof(float));
    cudaFuncSetAttribute(k_eig_l1_chfsi<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    const double tol1 = tol > kMixedPhase1Tol ? tol : kMixedPhase1Tol;
    k_eig_l1_chfsi<float><<<(unsigned)f.m, thr, sm1, s>>>(f.T, f.S, c->n, f.bx, f.by, f.bz, f.m, L, K, mdeg, max_iter,
                                                          tol1, guess, guess_vecs, block, nullptr, nullptr, c->dtmp,
                                                          c->flags, f.Wd);
  }
  const size_t sm = chfsi_smem(f.nb, K, sizeof(double));
  cudaFuncSetAttribute(k_eig_l1_chfsi<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_eig_l1_chfsi<double><<<(unsigned)f.m, thr, sm, s>>>(f.T, f.S, c->n, f.bx, f.by, f.bz, f.m, L, K, mdeg, max_iter, tol,
                                                        block ? block : guess, block ? K : guess_vecs, nullptr, f.Phi,
                                                        f.lam, c->dtmp, c->flags, f.Wd);
  return 0;
}

}  // namespace msmg
