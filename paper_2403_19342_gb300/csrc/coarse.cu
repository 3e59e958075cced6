// Coarse-level steps of the V-cycle (Algorithm 1 applied on W_l, l >= 2) and
// the coarsest pseudo-inverse application, in FP64 in both forms: with
// high-contrast coefficients the coarse block inverses are ill-conditioned
// (cond ~1e7 at contrast 1e6), and FP32 coarse levels doubled the mixed form's
// iteration count on the 128^3 inclusion workload.  In the mixed form the
// level-2 correction is also written in FP32 for the fine prolongation.
//
// A_l is a block 7-point stencil: element a of E_{l-1} carries L coordinates;
// Ad[a] is its diagonal block and Ao[a][d] = A_l[a, a + e_d] its coupling to the
// +d neighbour (the -d coupling is the transpose of the neighbour's).  The
// smoother is block Jacobi over the parents (elements of E_l): one dense
// nP x nP inverse per parent, nP = children * L, applied as a GEMV.
//
// One CTA per parent and right-hand side (R right-hand sides in lockstep,
// level-l vectors stored n_l apart; CTA b handles parent b / R of right-hand
// side b % R).  The parent's smoother inverse is staged in shared memory with
// asynchronous copies (all in flight at once); the per-row stencil loops are
// unrolled for the common block sizes L (template parameter, 0 = runtime).
#include "msmg_internal.cuh"
#include "reduce.cuh"
#include <cooperative_groups.h>
#include <type_traits>

namespace cg = cooperative_groups;

namespace msmg {

__device__ __forceinline__ void cp16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp8(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ void cp4(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_elem(double* dst, const double* src) { cp8(dst, src); }
__device__ __forceinline__ void cp_elem(float* dst, const float* src) { cp4(dst, src); }

// CTA-wide asynchronous copy of count values (16-byte chunks when aligned)
template <typename S>
__device__ __forceinline__ void cta_cp(S* dst, const S* src, int count) {
  constexpr int per = 16 / sizeof(S);
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0 && (count % per) == 0) {
    for (int i = threadIdx.x; i < count / per; i += blockDim.x) cp16(dst + per * i, src + per * i);
  } else {
    for (int i = threadIdx.x; i < count; i += blockDim.x) cp_elem(dst + i, src + i);
  }
}

// Threads of a per-parent CTA: max(nP, Lnext, 64) rounded up to a warp.
__host__ __device__ inline unsigned coarse_threads_d(int nP, int Ln) {
  int t = nP > Ln ? nP : Ln;
  if (t < 64) t = 64;
  return (unsigned)((t + 31) / 32 * 32);
}

// The level's operator data in the arithmetic type S.
template <typename S>
struct LevelData {
  const S *Ad, *Ao, *Minv, *Psi;
};

// r_i = f_i - (A_l u)_i for the rows i of one parent's children (thread t: row t).
template <int LT, typename S>
__device__ __forceinline__ S coarse_residual_row(const CoarseLevel& lv, const LevelData<S>& D, int64_t P, int t,
                                                 const S* __restrict__ f, const S* __restrict__ u) {
  const int L = LT ? LT : lv.L;
  const int64_t a = P * lv.nchild + t / L;
  const int k = t % L;
  const int L2 = L * L;
  const S* ad = D.Ad + a * L2 + (size_t)k * L;
  const S* ua = u + a * L;
  S acc = __ldg(f + a * L + k);
  int nb[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) nb[q] = __ldg(lv.nbr + a * 6 + q);
  if (LT) {
#pragma unroll
    for (int mm = 0; mm < LT; ++mm) acc -= __ldg(ad + mm) * __ldg(ua + mm);
  } else {
    for (int mm = 0; mm < L; ++mm) acc -= __ldg(ad + mm) * __ldg(ua + mm);
  }
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int bp = nb[2 * d + 1];   // +d neighbour: A_l[a, bp] = Ao[a][d]
    if (bp >= 0) {
      const S* ao = D.Ao + ((size_t)a * 3 + d) * L2 + (size_t)k * L;
      const S* ub = u + (int64_t)bp * L;
      if (LT) {
#pragma unroll
        for (int mm = 0; mm < LT; ++mm) acc -= __ldg(ao + mm) * __ldg(ub + mm);
      } else {
        for (int mm = 0; mm < L; ++mm) acc -= __ldg(ao + mm) * __ldg(ub + mm);
      }
    }
    const int bm = nb[2 * d];       // -d neighbour: A_l[a, bm] = Ao[bm][d]^T
    if (bm >= 0) {
      const S* ao = D.Ao + ((size_t)bm * 3 + d) * L2 + k;
      const S* ub = u + (int64_t)bm * L;
      if (LT) {
#pragma unroll
        for (int mm = 0; mm < LT; ++mm) acc -= __ldg(ao + (size_t)mm * LT) * __ldg(ub + mm);
      } else {
        for (int mm = 0; mm < L; ++mm) acc -= __ldg(ao + (size_t)mm * L) * __ldg(ub + mm);
      }
    }
  }
  return acc;
}

// y_t = sum_j M[j][t] x_j from shared memory (M symmetric, so column t = row t)
template <typename S>
__device__ __forceinline__ S smem_gemv_col(const S* M, const S* x, int nP, int t) {
  S a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  int j = 0;
  for (; j + 3 < nP; j += 4) {
    a0 = fma(M[(size_t)j * nP + t], x[j], a0);
    a1 = fma(M[(size_t)(j + 1) * nP + t], x[j + 1], a1);
    a2 = fma(M[(size_t)(j + 2) * nP + t], x[j + 2], a2);
    a3 = fma(M[(size_t)(j + 3) * nP + t], x[j + 3], a3);
  }
  for (; j < nP; ++j) a0 = fma(M[(size_t)j * nP + t], x[j], a0);
  return (a0 + a1) + (a2 + a3);
}

// Pre-smoothing from zero on level l: u_P = Minv_P f_P.
template <typename S>
__global__ void k_coarse_smooth_first(CoarseLevel lv, LevelData<S> D, const S* __restrict__ f, S* __restrict__ u,
                                      const PcgScalars* sc, int R) {
  const BatchIdx bi = batch_idx(R);
  if (sc) sc += bi.r;
  if (sc && sc->done) return;
  f += (int64_t)bi.r * lv.n;
  u += (int64_t)bi.r * lv.n;
  extern __shared__ __align__(16) unsigned char smraw[];
  S* sm = reinterpret_cast<S*>(smraw);
  const int64_t P = bi.blk;
  const int nP = lv.nP;
  S* Mi = sm;                      // [nP][nP]
  S* fs = sm + (size_t)nP * nP;
  cta_cp(Mi, D.Minv + (size_t)P * nP * nP, nP * nP);
  const int t = threadIdx.x;
  if (t < nP) fs[t] = __ldg(f + P * nP + t);
  cp_wait();
  __syncthreads();
  if (t < nP) u[P * nP + t] = smem_gemv_col(Mi, fs, nP, t);
}

// Residual and restriction to level l+1: fn[P][j] = sum_i Psi[P][j][i] (f - A_l u)_i.
template <int LT, typename S>
__global__ void k_coarse_resid_restrict(CoarseLevel lv, LevelData<S> D, const S* __restrict__ f,
                                        const S* __restrict__ u, S* __restrict__ fn, const PcgScalars* sc, int R) {
  const BatchIdx bi = batch_idx(R);
  if (sc) sc += bi.r;
  if (sc && sc->done) return;
  f += (int64_t)bi.r * lv.n;
  u += (int64_t)bi.r * lv.n;
  fn += (int64_t)bi.r * lv.mP * lv.Lnext;
  extern __shared__ __align__(16) unsigned char smraw[];
  S* sm = reinterpret_cast<S*>(smraw);
  const int64_t P = bi.blk;
  const int nP = lv.nP, Ln = lv.Lnext;
  const int nw = (blockDim.x + 31) >> 5;
  S* ps = sm;                            // [Ln][nP]
  S* red = sm + (size_t)Ln * nP;         // [Ln][nw]
  cta_cp(ps, D.Psi + (size_t)P * Ln * nP, Ln * nP);
  const int t = threadIdx.x;
  const S rt = t < nP ? coarse_residual_row<LT>(lv, D, P, t, f, u) : (S)0;
  cp_wait();
  __syncthreads();
  const int lane = t & 31, w = t >> 5;
  for (int j = 0; j < Ln; ++j) {
    S v = t < nP ? ps[(size_t)j * nP + t] * rt : (S)0;
    v = warp_sum_t(v);
    if (lane == 0) red[j * nw + w] = v;
  }
  __syncthreads();
  if (t < Ln) {
    S acc = 0;
    for (int q = 0; q < nw; ++q) acc += red[t * nw + q];
    fn[P * Ln + t] = acc;
  }
}

// Prolongation: u_P += Psi_P^T e_P.
template <typename S>
__global__ void k_coarse_prolong(CoarseLevel lv, LevelData<S> D, S* __restrict__ u, const S* __restrict__ e,
                                 const PcgScalars* sc, int R) {
  const BatchIdx bi = batch_idx(R);
  if (sc) sc += bi.r;
  if (sc && sc->done) return;
  u += (int64_t)bi.r * lv.n;
  e += (int64_t)bi.r * lv.mP * lv.Lnext;
  const int64_t P = bi.blk;
  const int t = threadIdx.x;
  if (t >= lv.nP) return;
  const S* ps = D.Psi + (size_t)P * lv.Lnext * lv.nP;
  S acc = 0;
#pragma unroll 4
  for (int j = 0; j < lv.Lnext; ++j) acc = fma(__ldg(ps + (size_t)j * lv.nP + t), __ldg(e + P * lv.Lnext + j), acc);
  u[P * lv.nP + t] += acc;
}

// Post-smoothing: out = u + Minv (f - A_l u)   (out must not alias u).
template <int LT, typename S>
__global__ void k_coarse_resid_smooth(CoarseLevel lv, LevelData<S> D, const S* __restrict__ f,
                                      const S* __restrict__ u, S* __restrict__ out, float* __restrict__ out32,
                                      const PcgScalars* sc, int R) {
  const BatchIdx bi = batch_idx(R);
  if (sc) sc += bi.r;
  if (sc && sc->done) return;
  {
    const int64_t off = (int64_t)bi.r * lv.n;
    f += off; u += off; out += off;
    if (out32) out32 += off;
  }
  extern __shared__ __align__(16) unsigned char smraw[];
  S* sm = reinterpret_cast<S*>(smraw);
  const int64_t P = bi.blk;
  const int nP = lv.nP;
  S* Mi = sm;
  S* rs = sm + (size_t)nP * nP;
  cta_cp(Mi, D.Minv + (size_t)P * nP * nP, nP * nP);
  const int t = threadIdx.x;
  if (t < nP) rs[t] = coarse_residual_row<LT>(lv, D, P, t, f, u);
  cp_wait();
  __syncthreads();
  if (t < nP) {
    const S v = u[P * nP + t] + smem_gemv_col(Mi, rs, nP, t);
    out[P * nP + t] = v;
    if (out32) out32[P * nP + t] = (float)v;
  }
}

// Coarsest level: u = A^dagger f, dense symmetric GEMV, one warp per row.
template <typename S>
__global__ void k_dense_gemv(const double* __restrict__ A, const S* __restrict__ x, S* __restrict__ y,
                             float* __restrict__ y32, int64_t n, const PcgScalars* sc, int R) {
  const BatchIdx bi = batch_idx(R);
  if (sc) sc += bi.r;
  if (sc && sc->done) return;
  x += (int64_t)bi.r * n;
  y += (int64_t)bi.r * n;
  if (y32) y32 += (int64_t)bi.r * n;
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)bi.blk * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  const double* a = A + row * n;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int64_t j = lane;
  for (; j + 96 < n; j += 128) {
    a0 = fma(__ldg(a + j), (double)__ldg(x + j), a0);
    a1 = fma(__ldg(a + j + 32), (double)__ldg(x + j + 32), a1);
    a2 = fma(__ldg(a + j + 64), (double)__ldg(x + j + 64), a2);
    a3 = fma(__ldg(a + j + 96), (double)__ldg(x + j + 96), a3);
  }
  for (; j < n; j += 32) a0 = fma(__ldg(a + j), (double)__ldg(x + j), a0);
  const double acc = warp_sum((a0 + a1) + (a2 + a3));
  if (lane == 0) {
    y[row] = (S)acc;
    if (y32) y32[row] = (float)acc;
  }
}

// ------------------------------------------------------------------ fused coarse cycle
// Levels l0 .. nL of the V-cycle (and the coarsest pseudo-inverse) in one
// launch, the phases separated by barriers.  On GB300 a warp issues one FP64
// instruction per 64 cycles on its SM sub-partition, so a level with a few
// hundred parents, launched as its own kernels, leaves most sub-partitions
// idle and pays a launch per phase.  Two forms:
//   cluster: a thread-block cluster per right-hand side (16 SMs), cluster
//            barriers; for a small tail of levels;
//   grid:    a cooperative launch over the whole GPU for all right-hand sides
//            and all coarse levels, grid barriers.
// Work items are (right-hand side, parent) pairs: each is handled by a group of
// ceil(max(nP, Lnext, 64) / 32) warps with thread t on row t; item i goes to
// CTA i mod ncta (group i / ncta), so a level with fewer items than group slots
// still spreads over every CTA's SM.  Every row,
// restriction and GEMV is evaluated by the same code and reduction order as the
// per-level kernels above, so every form gives the same bits.  A right-hand
// side that has converged skips its items but every thread reaches every
// barrier.
constexpr int kTailThreads = 256;
constexpr int kTailMaxLevels = kMaxLevels;

struct TailArgs {
  CoarseLevel lv[kTailMaxLevels + 1];   // indexed by level
  double* f[kTailMaxLevels + 1];
  double* u[kTailMaxLevels + 1];
  double* w[kTailMaxLevels + 1];
  float* out32;                          // FP32 copy of the level-2 correction (mixed form), or null
  int* err;                              // set when the grid form was not launched cooperatively
  int l0, nL;
};

struct ClusterBarrier {
  __device__ __forceinline__ void operator()() const {
    __threadfence();
    cg::this_cluster().sync();
  }
};
struct GridBarrier {
  __device__ __forceinline__ void operator()() const {
    __threadfence();
    cg::this_grid().sync();
  }
};

// item i of the level's R * mP (right-hand side, parent) pairs
struct TailItem {
  int r;
  int64_t P;
  bool live;
};
__device__ __forceinline__ TailItem tail_item(int64_t i, int64_t mP, int r0, int r1, const PcgScalars* sc) {
  TailItem it;
  it.live = i < (int64_t)(r1 - r0) * mP;
  it.r = it.live ? r0 + (int)(i / mP) : r0;
  it.P = it.live ? i % mP : 0;
  if (it.live && sc && sc[it.r].done) it.live = false;
  return it;
}

// asynchronous copy of count doubles by the nt threads of a parent group (thread t)
__device__ __forceinline__ void group_cp(double* dst, const double* src, int count, int t, int nt) {
  if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0 && (count & 1) == 0) {
    for (int i = t; i < count / 2; i += nt) cp16(dst + 2 * i, src + 2 * i);
  } else {
    for (int i = t; i < count; i += nt) cp8(dst + i, src + i);
  }
}

// per-group shared memory: [nP * nP] smoother inverse | [nP] vector | [Ln][gw] partials
__host__ __device__ inline int tail_group_doubles(int nP, int Ln, int gw) {
  return (nP * nP + nP + Ln * gw + 2 + 1) / 2 * 2;
}

template <int LT, typename Bar>
__device__ void tail_level_down(const TailArgs& A, int l, int r0, int r1, int cta, int ncta, double* sm,
                                const PcgScalars* sc, Bar bar) {
  const CoarseLevel& lv = A.lv[l];
  const LevelData<double> D{lv.Ad, lv.Ao, lv.Minv, lv.Psi};
  const int nP = lv.nP, Ln = lv.Lnext;
  const int gw = (int)(coarse_threads_d(nP, Ln) / 32);      // warps per parent group
  const int G = (kTailThreads / 32) / gw;                   // groups per CTA
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp / gw, t = (warp % gw) * 32 + lane;
  const int64_t items = (int64_t)(r1 - r0) * lv.mP;
  double* Mi = sm + (size_t)grp * tail_group_doubles(nP, Ln, gw);
  double* fs = Mi + (size_t)nP * nP;                        // [nP] right side, then [Ln][gw] partials
  // pre-smoothing from zero: u_P = Minv_P f_P (the inverse staged, all copies in flight)
  for (int64_t b0 = 0; b0 < items; b0 += (int64_t)ncta * G) {
    const TailItem it = tail_item(b0 + (int64_t)grp * ncta + cta, lv.mP, r0, r1, sc);
    const bool live = grp < G && it.live;
    const double* f = A.f[l] + (int64_t)it.r * lv.n;
    double* u = A.u[l] + (int64_t)it.r * lv.n;
    if (live) group_cp(Mi, D.Minv + (size_t)it.P * nP * nP, nP * nP, t, gw * 32);
    if (live && t < nP) fs[t] = f[it.P * nP + t];
    cp_wait();
    __syncthreads();
    if (live && t < nP) u[it.P * nP + t] = smem_gemv_col(Mi, fs, nP, t);
    __syncthreads();
  }
  bar();
  // residual and restriction: fn[P][j] = sum_i Psi[P][j][i] (f - A_l u)_i
  for (int64_t b0 = 0; b0 < items; b0 += (int64_t)ncta * G) {
    const TailItem it = tail_item(b0 + (int64_t)grp * ncta + cta, lv.mP, r0, r1, sc);
    const bool live = grp < G && it.live;
    const double* f = A.f[l] + (int64_t)it.r * lv.n;
    const double* u = A.u[l] + (int64_t)it.r * lv.n;
    double* fn = A.f[l + 1] + (int64_t)it.r * lv.mP * Ln;
    const double rt = (live && t < nP) ? coarse_residual_row<LT>(lv, D, it.P, t, f, u) : 0.0;
    double* red = fs + nP;
    for (int j = 0; j < Ln; ++j) {
      double v = (live && t < nP) ? __ldg(D.Psi + ((size_t)it.P * Ln + j) * nP + t) * rt : 0.0;
      v = warp_sum_t(v);
      if (live && lane == 0) red[j * gw + (warp % gw)] = v;
    }
    __syncthreads();
    if (live && t < Ln) {
      double acc = 0;
      for (int q = 0; q < gw; ++q) acc += red[t * gw + q];
      fn[it.P * Ln + t] = acc;
    }
    __syncthreads();
  }
  bar();
}

template <int LT, typename Bar>
__device__ void tail_level_up(const TailArgs& A, int l, int r0, int r1, int cta, int ncta, double* sm,
                              const PcgScalars* sc, Bar bar) {
  const CoarseLevel& lv = A.lv[l];
  const LevelData<double> D{lv.Ad, lv.Ao, lv.Minv, lv.Psi};
  const int nP = lv.nP, Ln = lv.Lnext;
  const int gw = (int)(coarse_threads_d(nP, Ln) / 32);
  const int G = (kTailThreads / 32) / gw;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = warp / gw, t = (warp % gw) * 32 + lane;
  const int64_t items = (int64_t)(r1 - r0) * lv.mP;
  const double* ebase = (l + 1 == A.nL) ? A.u[l + 1] : A.w[l + 1];
  double* Mi = sm + (size_t)grp * tail_group_doubles(nP, Ln, gw);
  double* rs = Mi + (size_t)nP * nP;
  // prolongation: u_P += Psi_P^T e_P
  for (int64_t b0 = 0; b0 < items; b0 += (int64_t)ncta * G) {
    const TailItem it = tail_item(b0 + (int64_t)grp * ncta + cta, lv.mP, r0, r1, sc);
    if (grp < G && it.live && t < nP) {
      const double* e = ebase + (int64_t)it.r * lv.mP * Ln;
      double* u = A.u[l] + (int64_t)it.r * lv.n;
      const double* ps = D.Psi + (size_t)it.P * Ln * nP;
      double acc = 0;
#pragma unroll 4
      for (int j = 0; j < Ln; ++j) acc = fma(__ldg(ps + (size_t)j * nP + t), e[it.P * Ln + j], acc);
      u[it.P * nP + t] += acc;
    }
  }
  bar();
  // post-smoothing: w = u + Minv (f - A_l u)
  for (int64_t b0 = 0; b0 < items; b0 += (int64_t)ncta * G) {
    const TailItem it = tail_item(b0 + (int64_t)grp * ncta + cta, lv.mP, r0, r1, sc);
    const bool live = grp < G && it.live;
    const double* f = A.f[l] + (int64_t)it.r * lv.n;
    const double* u = A.u[l] + (int64_t)it.r * lv.n;
    double* w = A.w[l] + (int64_t)it.r * lv.n;
    float* o32 = (l == 2 && A.out32) ? A.out32 + (int64_t)it.r * lv.n : nullptr;
    if (live) group_cp(Mi, D.Minv + (size_t)it.P * nP * nP, nP * nP, t, gw * 32);
    if (live && t < nP) rs[t] = coarse_residual_row<LT>(lv, D, it.P, t, f, u);
    cp_wait();
    __syncthreads();
    if (live && t < nP) {
      const double v = u[it.P * nP + t] + smem_gemv_col(Mi, rs, nP, t);
      w[it.P * nP + t] = v;
      if (o32) o32[it.P * nP + t] = (float)v;
    }
    __syncthreads();
  }
  bar();
}

// coarsest: u = A^dagger f, one warp per (right-hand side, row), the same
// arithmetic as k_dense_gemv
template <typename Bar>
__device__ void tail_coarsest(const TailArgs& A, int r0, int r1, int cta, int ncta, const PcgScalars* sc, Bar bar) {
  const CoarseLevel& lc = A.lv[A.nL];
  const int64_t n = lc.n;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)ncta * (kTailThreads / 32);
  const int64_t items = (int64_t)(r1 - r0) * n;
  for (int64_t i = (int64_t)cta * (kTailThreads / 32) + (threadIdx.x >> 5); i < items; i += nw) {
    const int r = r0 + (int)(i / n);
    const int64_t row = i % n;
    if (sc && sc[r].done) continue;
    const double* x = A.f[A.nL] + (int64_t)r * n;
    double* y = A.u[A.nL] + (int64_t)r * n;
    const double* a = lc.pinv + row * n;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int64_t j = lane;
    for (; j + 96 < n; j += 128) {
      a0 = fma(__ldg(a + j), x[j], a0);
      a1 = fma(__ldg(a + j + 32), x[j + 32], a1);
      a2 = fma(__ldg(a + j + 64), x[j + 64], a2);
      a3 = fma(__ldg(a + j + 96), x[j + 96], a3);
    }
    for (; j < n; j += 32) a0 = fma(__ldg(a + j), x[j], a0);
    const double acc = warp_sum((a0 + a1) + (a2 + a3));
    if (lane == 0) {
      y[row] = acc;
      if (A.nL == 2 && A.out32) A.out32[(int64_t)r * n + row] = (float)acc;
    }
  }
  bar();
}

template <int LT, typename Bar>
__device__ void tail_run(const TailArgs& A, int r0, int r1, int cta, int ncta, const PcgScalars* sc, Bar bar) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double* sm = reinterpret_cast<double*>(smraw);
  for (int l = A.l0; l < A.nL; ++l) tail_level_down<LT>(A, l, r0, r1, cta, ncta, sm, sc, bar);
  tail_coarsest(A, r0, r1, cta, ncta, sc, bar);
  for (int l = A.nL - 1; l >= A.l0; --l) tail_level_up<LT>(A, l, r0, r1, cta, ncta, sm, sc, bar);
}

// one cluster per right-hand side
template <int LT>
__global__ void __launch_bounds__(kTailThreads) k_coarse_tail(TailArgs A, const PcgScalars* sc, int R) {
  const int ncta = (int)cg::this_cluster().num_blocks();
  const int cta = (int)cg::this_cluster().block_rank();
  const int r = (int)(blockIdx.x / (unsigned)ncta) % R;
  tail_run<LT>(A, r, r + 1, cta, ncta, sc, ClusterBarrier{});
}

// one cooperative grid for every right-hand side
template <int LT>
__global__ void __launch_bounds__(kTailThreads) k_coarse_coop(TailArgs A, const PcgScalars* sc, int R) {
  // the grid barrier is defined only for a cooperative launch: otherwise every CTA
  // returns at once (nothing waits) and the solve reports the error
  if (!cg::this_grid().is_valid()) {
    if (threadIdx.x == 0) atomicExch(A.err, 1);
    return;
  }
  tail_run<LT>(A, 0, R, (int)blockIdx.x, (int)gridDim.x, sc, GridBarrier{});
}

static inline unsigned coarse_threads(const CoarseLevel& lv) { return coarse_threads_d(lv.nP, lv.Lnext); }
template <typename S>
static inline size_t smem_smooth(const CoarseLevel& lv) {
  return ((size_t)lv.nP * lv.nP + lv.nP) * sizeof(S) + 16;
}
template <typename S>
static inline size_t smem_restrict(const CoarseLevel& lv) {
  return ((size_t)lv.Lnext * lv.nP + (size_t)lv.Lnext * (coarse_threads(lv) / 32)) * sizeof(S) + 16;
}

template <typename F>
static void with_L(int L, F&& fn) {
  switch (L) {
    case 4: fn(std::integral_constant<int, 4>{}); break;
    case 6: fn(std::integral_constant<int, 6>{}); break;
    case 7: fn(std::integral_constant<int, 7>{}); break;
    case 8: fn(std::integral_constant<int, 8>{}); break;
    default: fn(std::integral_constant<int, 0>{}); break;
  }
}

template <typename S>
static LevelData<S> level_data(const CoarseLevel& lv);
template <>
LevelData<double> level_data<double>(const CoarseLevel& lv) { return {lv.Ad, lv.Ao, lv.Minv, lv.Psi}; }

template <typename S>
static void prepare_t(msmg_ctx* c) {
  for (int l = 2; l < c->nL; ++l) {
    CoarseLevel& lv = c->lev[l];
    const int sm1 = (int)smem_smooth<S>(lv), sm2 = (int)smem_restrict<S>(lv);
    cudaFuncSetAttribute(k_coarse_smooth_first<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm1);
    with_L(lv.L, [&](auto LC) {
      constexpr int LT = decltype(LC)::value;
      cudaFuncSetAttribute(k_coarse_resid_smooth<LT, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm1);
      cudaFuncSetAttribute(k_coarse_resid_restrict<LT, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2);
    });
  }
}

// Fused coarse cycle, cluster form: from the first level with at most
// kTailMaxParents parents (all later levels are smaller); grid form: every
// coarse level.  Both need a coarsest level small enough for its dense
// pseudo-inverse GEMV to run inside the launch.
constexpr int64_t kTailMaxParents = 256;
constexpr int64_t kTailMaxCoarsest = 1536;
constexpr int64_t kCoopMaxCoarsest = 4096;

// shared memory and the common compile-time L of levels l0 .. nL-1 (0: runtime)
static bool tail_shape(const msmg_ctx* c, int l0, int* lt_out, size_t* sm_out) {
  int lt = l0 < c->nL ? c->lev[l0].L : 4;
  size_t sm = 0;
  for (int l = l0; l < c->nL; ++l) {
    const CoarseLevel& lv = c->lev[l];
    if (lv.L != lt) lt = 0;
    const int gw = (int)(coarse_threads_d(lv.nP, lv.Lnext) / 32);
    if (gw > kTailThreads / 32) return false;
    const int G = (kTailThreads / 32) / gw;
    const size_t need = (size_t)G * tail_group_doubles(lv.nP, lv.Lnext, gw) * sizeof(double);
    if (need > sm) sm = need;
  }
  if (lt != 4 && lt != 6 && lt != 7 && lt != 8) lt = 0;
  if (sm + 64 > 200 * 1024) return false;        // keep well inside 227 KB per CTA
  *lt_out = lt;
  *sm_out = sm + 64;
  return true;
}

template <int LT>
static void cluster_prepare_lt(msmg_ctx* c) {
  cudaFuncSetAttribute(k_coarse_tail<LT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->tail_smem);
  cudaFuncSetAttribute(k_coarse_tail<LT>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  for (int cs : {16, 8}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cs);
    cfg.blockDim = dim3(kTailThreads);
    cfg.dynamicSmemBytes = c->tail_smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclus = 0;
    if (cudaOccupancyMaxActiveClusters(&nclus, k_coarse_tail<LT>, &cfg) == cudaSuccess && nclus >= 1) {
      c->tail_cs = cs;
      return;
    }
    cudaGetLastError();
  }
  c->tail_l0 = 0;
}

template <int LT>
static void coop_prepare_lt(msmg_ctx* c) {
  c->coop_grid = 0;
  int coop = 0, dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (!coop || nsm < 1) return;
  cudaFuncSetAttribute(k_coarse_coop<LT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->coop_smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_coarse_coop<LT>, kTailThreads, c->coop_smem) !=
          cudaSuccess || per < 1) {
    cudaGetLastError();
    return;
  }
  c->coop_grid = nsm * (per < 2 ? per : 2);   // every CTA co-resident, as the grid barrier needs
}

static void tail_prepare(msmg_ctx* c) {
  c->tail_l0 = 0;
  c->tail_cs = 0;
  c->coop_grid = 0;
  const int64_t nc = c->lev[c->nL].n;
  if (nc <= kTailMaxCoarsest) {
    int l0 = 0;
    for (int l = 2; l < c->nL; ++l)
      if (c->lev[l].mP <= kTailMaxParents) { l0 = l; break; }
    if (l0 && tail_shape(c, l0, &c->tail_lt, &c->tail_smem)) {
      c->tail_l0 = l0;
      with_L(c->tail_lt, [&](auto LC) { cluster_prepare_lt<decltype(LC)::value>(c); });
    }
  }
  if (nc <= kCoopMaxCoarsest && tail_shape(c, 2, &c->coop_lt, &c->coop_smem))
    with_L(c->coop_lt, [&](auto LC) { coop_prepare_lt<decltype(LC)::value>(c); });
}

static TailArgs tail_args(const msmg_ctx* c, int l0) {
  TailArgs A;
  for (int l = 0; l <= kTailMaxLevels; ++l) {
    const bool in = l >= 2 && l <= c->nL;
    A.lv[l] = in ? c->lev[l] : CoarseLevel{};
    A.f[l] = in ? (double*)c->sb.vf[l] : nullptr;
    A.u[l] = in ? (double*)c->sb.vu[l] : nullptr;
    A.w[l] = in ? (double*)c->sb.vw[l] : nullptr;
  }
  A.out32 = l0 == 2 ? c->sb.ec32 : nullptr;
  A.err = c->flags + 5;
  A.l0 = l0;
  A.nL = c->nL;
  return A;
}

// cluster form from level tail_l0
static int launch_tail(msmg_ctx* c, PcgScalars* sc, cudaStream_t s) {
  const TailArgs A = tail_args(c, c->tail_l0);
  const int R = c->sb.R;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(c->tail_cs * R));
  cfg.blockDim = dim3(kTailThreads);
  cfg.dynamicSmemBytes = c->tail_smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)c->tail_cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaSuccess;
  with_L(c->tail_lt, [&](auto LC) { e = cudaLaunchKernelEx(&cfg, k_coarse_tail<decltype(LC)::value>, A, sc, R); });
  if (e != cudaSuccess) { set_last_cuda_error(e); return MSMG_ERR_CUDA; }
  return 0;
}

// grid form: the coarse cycle from level l0 (2: all of it; tail_l0: the small
// levels), cooperative launch
static int launch_coop(msmg_ctx* c, int l0, PcgScalars* sc, cudaStream_t s) {
  const TailArgs A = tail_args(c, l0);
  const int R = c->sb.R;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)c->coop_grid);
  cfg.blockDim = dim3(kTailThreads);
  cfg.dynamicSmemBytes = c->coop_smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaSuccess;
  with_L(c->coop_lt, [&](auto LC) { e = cudaLaunchKernelEx(&cfg, k_coarse_coop<decltype(LC)::value>, A, sc, R); });
  if (e != cudaSuccess) { set_last_cuda_error(e); return MSMG_ERR_CUDA; }
  return 0;
}

// Shared-memory limits of the coarse kernels and the fused forms (set once per
// context, never during capture).
void prepare_coarse_kernels(msmg_ctx* c) {
  prepare_t<double>(c);
  tail_prepare(c);
  for (int k = 0; k < 2; ++k) {
    if (c->tune_tail[k] == 3 && !(c->coop_grid && c->tail_l0)) c->tune_tail[k] = c->coop_grid ? 2 : 0;
    if (c->tune_tail[k] == 2 && !c->coop_grid) c->tune_tail[k] = c->tail_l0 ? 1 : 0;
    if (c->tune_tail[k] == 1 && !c->tail_l0) c->tune_tail[k] = c->coop_grid ? 2 : 0;
  }
}

// available forms of the coarse cycle: bit 0 per level (always), bit 1 cluster tail,
// bit 2 grid (all coarse levels), bit 3 grid tail
int coarse_forms(const msmg_ctx* c) {
  return 1 | (c->tail_l0 ? 2 : 0) | (c->coop_grid ? 4 : 0) | (c->coop_grid && c->tail_l0 ? 8 : 0);
}


// Level-l part of the V-cycle (l >= 2): on entry vf[l] holds the right side;
// returns the device pointer holding the level-l correction.
template <typename S>
static const S* coarse_cycle_t(msmg_ctx* c, int l, PcgScalars* sc, cudaStream_t s) {
  CoarseLevel& lv = c->lev[l];
  S* f = (S*)c->sb.vf[l];
  S* u = (S*)c->sb.vu[l];
  S* w = (S*)c->sb.vw[l];
  const int R = c->sb.R;
  const int form = c->tune_tail[R > 1 ? 1 : 0];
  if (l == 2 && form == 2 && c->coop_grid) {
    launch_coop(c, 2, sc, s);
    return (const S*)(c->nL == 2 ? c->sb.vu[2] : c->sb.vw[2]);
  }
  if (l == c->tail_l0 && form == 1) {
    launch_tail(c, sc, s);
    return (const S*)c->sb.vw[l];
  }
  if (l == c->tail_l0 && form == 3 && c->coop_grid) {
    launch_coop(c, l, sc, s);
    return (const S*)c->sb.vw[l];
  }
  if (l == c->nL) {
    const unsigned grid = (unsigned)((lv.n * 32 + 255) / 256 * R);
    k_dense_gemv<S><<<grid, 256, 0, s>>>(lv.pinv, f, u, l == 2 ? c->sb.ec32 : nullptr, lv.n, sc, R);
    return u;
  }
  const LevelData<S> D = level_data<S>(lv);
  S* fn = (S*)c->sb.vf[l + 1];
  const unsigned thr = coarse_threads(lv);
  const unsigned grid = (unsigned)(lv.mP * R);
  k_coarse_smooth_first<S><<<grid, thr, smem_smooth<S>(lv), s>>>(lv, D, f, u, sc, R);
  with_L(lv.L, [&](auto LC) {
    k_coarse_resid_restrict<decltype(LC)::value, S><<<grid, thr, smem_restrict<S>(lv), s>>>(lv, D, f, u, fn, sc, R);
  });
  const S* e = coarse_cycle_t<S>(c, l + 1, sc, s);
  k_coarse_prolong<S><<<grid, thr, 0, s>>>(lv, D, u, e, sc, R);
  with_L(lv.L, [&](auto LC) {
    k_coarse_resid_smooth<decltype(LC)::value, S><<<grid, thr, smem_smooth<S>(lv), s>>>(
        lv, D, f, u, w, l == 2 ? c->sb.ec32 : nullptr, sc, R);
  });
  return w;
}

// Returns the level-2 correction in the V-cycle precision: FP64, or its FP32
// copy in the mixed form.
const void* coarse_cycle(msmg_ctx* c, int l, PcgScalars* sc, cudaStream_t s) {
  const double* e = coarse_cycle_t<double>(c, l, sc, s);
  return c->sb.ec32 ? (const void*)c->sb.ec32 : (const void*)e;
}

}  // namespace msmg
