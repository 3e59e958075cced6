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

// Loads of f and u: through the read-only path when they were written by an
// earlier launch (per-level kernels), coherent when an earlier phase of the same
// launch wrote them (the fused forms, the inner two-grid solve).
template <bool NC, typename S>
__device__ __forceinline__ S ld_vec(const S* p) {
  if constexpr (NC) return __ldg(p);
  else return *p;
}

// Partial s of r_i = f_i - (A_l u)_i for row t of parent P: s = 0 takes f and
// the element's own block, s = 1, 2, 3 its x, y, z neighbour blocks (+d, then
// -d).  The row is (p0 + p1) + (p2 + p3): four threads (per-level kernels) or
// one thread in turn (fused forms) give the same bits.
template <int LT, typename S, bool NC = true>
__device__ __forceinline__ S coarse_residual_part(const CoarseLevel& lv, const LevelData<S>& D, int64_t P, int t,
                                                  int s, const S* __restrict__ f, const S* __restrict__ u) {
  const int L = LT ? LT : lv.L;
  const int64_t a = P * lv.nchild + t / L;
  const int k = t % L;
  const int L2 = L * L;
  if (s == 0) {
    const S* ad = D.Ad + a * L2 + (size_t)k * L;
    const S* ua = u + a * L;
    S acc = ld_vec<NC>(f + a * L + k);
    if (LT) {
#pragma unroll
      for (int mm = 0; mm < LT; ++mm) acc -= __ldg(ad + mm) * ld_vec<NC>(ua + mm);
    } else {
      for (int mm = 0; mm < L; ++mm) acc -= __ldg(ad + mm) * ld_vec<NC>(ua + mm);
    }
    return acc;
  }
  const int d = s - 1;
  S acc = 0;
  const int bp = __ldg(lv.nbr + a * 6 + 2 * d + 1);   // +d neighbour: A_l[a, bp] = Ao[a][d]
  const int bm = __ldg(lv.nbr + a * 6 + 2 * d);       // -d neighbour: A_l[a, bm] = Ao[bm][d]^T
  if (bp >= 0) {
    const S* ao = D.Ao + ((size_t)a * 3 + d) * L2 + (size_t)k * L;
    const S* ub = u + (int64_t)bp * L;
    if (LT) {
#pragma unroll
      for (int mm = 0; mm < LT; ++mm) acc -= __ldg(ao + mm) * ld_vec<NC>(ub + mm);
    } else {
      for (int mm = 0; mm < L; ++mm) acc -= __ldg(ao + mm) * ld_vec<NC>(ub + mm);
    }
  }
  if (bm >= 0) {
    const S* ao = D.Ao + ((size_t)bm * 3 + d) * L2 + k;
    const S* ub = u + (int64_t)bm * L;
    if (LT) {
#pragma unroll
      for (int mm = 0; mm < LT; ++mm) acc -= __ldg(ao + (size_t)mm * LT) * ld_vec<NC>(ub + mm);
    } else {
      for (int mm = 0; mm < L; ++mm) acc -= __ldg(ao + (size_t)mm * L) * ld_vec<NC>(ub + mm);
    }
  }
  return acc;
}

template <int LT, typename S, bool NC = true>
__device__ __forceinline__ S coarse_residual_row(const CoarseLevel& lv, const LevelData<S>& D, int64_t P, int t,
                                                 const S* __restrict__ f, const S* __restrict__ u) {
  const S p0 = coarse_residual_part<LT, S, NC>(lv, D, P, t, 0, f, u);
  const S p1 = coarse_residual_part<LT, S, NC>(lv, D, P, t, 1, f, u);
  const S p2 = coarse_residual_part<LT, S, NC>(lv, D, P, t, 2, f, u);
  const S p3 = coarse_residual_part<LT, S, NC>(lv, D, P, t, 3, f, u);
  return (p0 + p1) + (p2 + p3);
}

// (q0 + q1) + (q2 + q3) of the four lanes 4t .. 4t+3 of a warp, in every one of them
// (IEEE addition commutes, so the four lanes agree bit for bit)
template <typename S>
__device__ __forceinline__ S quad_combine(S q) {
  const S a = q + __shfl_xor_sync(0xffffffffu, q, 1);
  return a + __shfl_xor_sync(0xffffffffu, a, 2);
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

// Partial s of smem_gemv_col: its accumulator a_s (terms j = s mod 4 of the first
// 4 floor(nP / 4), and for s = 0 the remainder), so that quad_combine of the four
// partials equals smem_gemv_col bit for bit.
template <typename S>
__device__ __forceinline__ S smem_gemv_part(const S* M, const S* x, int nP, int t, int s) {
  S a = 0;
  const int n4 = nP & ~3;
  for (int j = s; j < n4; j += 4) a = fma(M[(size_t)j * nP + t], x[j], a);
  if (s == 0)
    for (int j = n4; j < nP; ++j) a = fma(M[(size_t)j * nP + t], x[j], a);
  return a;
}

// Threads of the per-level smoothing and residual kernels: four per row of the
// parent (quad_combine), and at least the row-per-thread layout of
// coarse_threads_d, whose warps form the restriction sums.
__host__ __device__ inline unsigned coarse_threads4_d(int nP, int Ln) {
  int t = 4 * nP;
  const int t1 = (int)coarse_threads_d(nP, Ln);
  if (t < t1) t = t1;
  return (unsigned)((t + 31) / 32 * 32);
}

// Row layouts of the per-level kernels, the same bits either way: QUAD, four
// threads per row (a level with few parents: shorter dependent chains, more
// warps); otherwise thread t takes row t and forms the four partials in turn.
// Pre-smoothing from zero on level l: u_P = Minv_P f_P.
template <typename S, bool QUAD>
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
  if constexpr (QUAD) {
    const int row = t >> 2, sub = t & 3;
    S q = row < nP ? smem_gemv_part(Mi, fs, nP, row, sub) : (S)0;
    q = quad_combine(q);
    if (row < nP && sub == 0) u[P * nP + row] = q;
  } else {
    if (t < nP) u[P * nP + t] = smem_gemv_col(Mi, fs, nP, t);
  }
}

// Residual and restriction to level l+1: fn[P][j] = sum_i Psi[P][j][i] (f - A_l u)_i.
// The residual rows by four threads each; the sums over the rows in the warps of
// the row-per-thread layout (the order of the fused forms).
template <int LT, typename S, bool QUAD>
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
  const int nw = (int)(coarse_threads_d(nP, Ln) / 32);
  S* ps = sm;                            // [Ln][nP]
  S* red = sm + (size_t)Ln * nP;         // [Ln][nw]
  S* rs = red + (size_t)Ln * nw;         // [nP] residual rows
  cta_cp(ps, D.Psi + (size_t)P * Ln * nP, Ln * nP);
  const int t = threadIdx.x;
  if constexpr (QUAD) {
    const int row = t >> 2, sub = t & 3;
    S q = row < nP ? coarse_residual_part<LT>(lv, D, P, row, sub, f, u) : (S)0;
    q = quad_combine(q);
    if (row < nP && sub == 0) rs[row] = q;
  } else {
    if (t < nP) rs[t] = coarse_residual_row<LT>(lv, D, P, t, f, u);
  }
  cp_wait();
  __syncthreads();
  if (t < nw * 32) {
    const int lane = t & 31, w = t >> 5;
    const S rt = t < nP ? rs[t] : (S)0;
    for (int j = 0; j < Ln; ++j) {
      S v = t < nP ? ps[(size_t)j * nP + t] * rt : (S)0;
      v = warp_sum_t(v);
      if (lane == 0) red[j * nw + w] = v;
    }
  }
  __syncthreads();
  if (t < Ln) {
    S acc = 0;
    for (int qq = 0; qq < nw; ++qq) acc += red[t * nw + qq];
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

// Post-smoothing: out = u + Minv (f - A_l u)   (out must not alias u); the residual
// rows and the smoother GEMV by four threads per row.
template <int LT, typename S, bool QUAD>
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
  if constexpr (QUAD) {
    const int row = t >> 2, sub = t & 3;
    S q = row < nP ? coarse_residual_part<LT>(lv, D, P, row, sub, f, u) : (S)0;
    q = quad_combine(q);
    if (row < nP && sub == 0) rs[row] = q;
    cp_wait();
    __syncthreads();
    S g = row < nP ? smem_gemv_part(Mi, rs, nP, row, sub) : (S)0;
    g = quad_combine(g);
    if (row < nP && sub == 0) {
      const S v = u[P * nP + row] + g;
      out[P * nP + row] = v;
      if (out32) out32[P * nP + row] = (float)v;
    }
  } else {
    if (t < nP) rs[t] = coarse_residual_row<LT>(lv, D, P, t, f, u);
    cp_wait();
    __syncthreads();
    if (t < nP) {
      const S v = u[P * nP + t] + smem_gemv_col(Mi, rs, nP, t);
      out[P * nP + t] = v;
      if (out32) out32[P * nP + t] = (float)v;
    }
  }
}

// Coarsest level: u = A^dagger f, dense symmetric GEMV, one warp per row.  Under
// Strategy 2 the pseudo-inverse acts on the kept coordinates only (packed,
// nk x nk): row p of the padded output reads packed row cinv[p] and gathers x
// through cmap; unused slots get 0.
__device__ __forceinline__ double coarsest_row(const double* __restrict__ A, const double* x, int64_t q, int64_t nk,
                                               const int* __restrict__ cmap, int lane) {
  const double* a = A + q * nk;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int64_t j = lane;
  if (cmap) {
    for (; j + 96 < nk; j += 128) {
      a0 = fma(__ldg(a + j), x[cmap[j]], a0);
      a1 = fma(__ldg(a + j + 32), x[cmap[j + 32]], a1);
      a2 = fma(__ldg(a + j + 64), x[cmap[j + 64]], a2);
      a3 = fma(__ldg(a + j + 96), x[cmap[j + 96]], a3);
    }
    for (; j < nk; j += 32) a0 = fma(__ldg(a + j), x[cmap[j]], a0);
  } else {
    for (; j + 96 < nk; j += 128) {
      a0 = fma(__ldg(a + j), x[j], a0);
      a1 = fma(__ldg(a + j + 32), x[j + 32], a1);
      a2 = fma(__ldg(a + j + 64), x[j + 64], a2);
      a3 = fma(__ldg(a + j + 96), x[j + 96], a3);
    }
    for (; j < nk; j += 32) a0 = fma(__ldg(a + j), x[j], a0);
  }
  return warp_sum((a0 + a1) + (a2 + a3));
}

template <typename S>
__global__ void k_dense_gemv(const double* __restrict__ A, const S* __restrict__ x, S* __restrict__ y,
                             float* __restrict__ y32, int64_t n, int64_t nk, const int* __restrict__ cmap,
                             const int* __restrict__ cinv, const PcgScalars* sc, int R) {
  const BatchIdx bi = batch_idx(R);
  if (sc) sc += bi.r;
  if (sc && sc->done) return;
  x += (int64_t)bi.r * n;
  y += (int64_t)bi.r * n;
  if (y32) y32 += (int64_t)bi.r * n;
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)bi.blk * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  const int64_t q = cinv ? cinv[row] : row;
  const double acc = q >= 0 ? coarsest_row(A, x, q, nk, cmap, lane) : 0.0;
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

// Per right-hand-side stop flags the fused forms read: the PCG scalars' done
// words (stride between records in ints) or any other int array.
struct DoneFlags {
  const int* p;
  int stride;
  __device__ __forceinline__ bool operator()(int r) const { return p && p[(size_t)r * stride]; }
};
__host__ __device__ inline DoneFlags done_of(const PcgScalars* sc) {
  return DoneFlags{sc ? &sc->done : nullptr, (int)(sizeof(PcgScalars) / sizeof(int))};
}

// item i of the level's R * mP (right-hand side, parent) pairs
struct TailItem {
  int r;
  int64_t P;
  bool live;
};
__device__ __forceinline__ TailItem tail_item(int64_t i, int64_t mP, int r0, int r1, DoneFlags dn) {
  TailItem it;
  it.live = i < (int64_t)(r1 - r0) * mP;
  it.r = it.live ? r0 + (int)(i / mP) : r0;
  it.P = it.live ? i % mP : 0;
  if (it.live && dn(it.r)) it.live = false;
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
                                DoneFlags sc, Bar bar) {
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
    const double rt = (live && t < nP) ? coarse_residual_row<LT, double, false>(lv, D, it.P, t, f, u) : 0.0;
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
                              DoneFlags sc, Bar bar) {
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
    if (live && t < nP) rs[t] = coarse_residual_row<LT, double, false>(lv, D, it.P, t, f, u);
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
__device__ void tail_coarsest(const TailArgs& A, int r0, int r1, int cta, int ncta, DoneFlags sc, Bar bar) {
  const CoarseLevel& lc = A.lv[A.nL];
  const int64_t n = lc.n;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)ncta * (kTailThreads / 32);
  const int64_t items = (int64_t)(r1 - r0) * n;
  for (int64_t i = (int64_t)cta * (kTailThreads / 32) + (threadIdx.x >> 5); i < items; i += nw) {
    const int r = r0 + (int)(i / n);
    const int64_t row = i % n;
    if (sc(r)) continue;
    const double* x = A.f[A.nL] + (int64_t)r * n;
    double* y = A.u[A.nL] + (int64_t)r * n;
    const int64_t q = lc.cinv ? lc.cinv[row] : row;
    const double acc = q >= 0 ? coarsest_row(lc.pinv, x, q, lc.nk, lc.cmap, lane) : 0.0;
    if (lane == 0) {
      y[row] = acc;
      if (A.nL == 2 && A.out32) A.out32[(int64_t)r * n + row] = (float)acc;
    }
  }
  bar();
}

template <int LT, typename Bar>
__device__ void tail_run(const TailArgs& A, int r0, int r1, int cta, int ncta, DoneFlags sc, Bar bar) {
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
  tail_run<LT>(A, r, r + 1, cta, ncta, done_of(sc), ClusterBarrier{});
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
  tail_run<LT>(A, 0, R, (int)blockIdx.x, (int)gridDim.x, done_of(sc), GridBarrier{});
}

// ------------------------------------------------------------------ exact two-grid (P_TG)
// Eq. (B_TG) puts the exact A_c^dagger where the V-cycle has the recursive
// coarse cycle B_c^{-1} of Eq. (B_c).  A_2 e_c = r_c is solved here by PCG on
// level 2, preconditioned by the coarse cycle from level 2 down (the device code
// of the fused grid form), to ||r|| <= inner_rtol ||r_c||, in one cooperative
// launch that iterates on the device until every right-hand side has converged.
// The result is projected orthogonal to the null vector z of A_2 (the
// minimum-norm solution, as the pseudo-inverse gives).
//
// Work split: CTA k owns the level-2 rows [k chunk, (k+1) chunk) of every
// right-hand side; warp w takes the right-hand sides r = w (mod 8) and its lanes
// the rows.  Sums: lanes -> warp shuffle -> one partial per (CTA, right-hand
// side) -> grid barrier -> every CTA adds the partials in CTA order with the same
// fixed tree, so all CTAs hold the same scalars and take the same decisions.
struct InnerArgs {
  double* x;        // [R][n2] solution of A_2 x = r_c
  double* p0;       // [R][n2] search directions, alternating between iterations
  double* p1;
  double* q;        // [R][n2] A_2 p
  double* part;     // [ncta][R][2] per-CTA partial sums
  int* iters;       // [R] inner iterations, accumulated over the calls of a solve
  float* out32;     // FP32 copy of the solution (mixed form) or null
  double rtol2;
  int max_iter;
  int singular;     // A_2 has the constant's null vector (no cell term)
};

// (A_2 v)_i, i = (element a, coordinate k); v(j) returns the vector's entry j
template <int LT, typename Vf>
__device__ __forceinline__ double coarse_apply_row(const CoarseLevel& lv, int64_t a, int k, Vf v) {
  const int L = LT ? LT : lv.L;
  const int L2 = L * L;
  double acc = 0.0;
  const double* ad = lv.Ad + a * L2 + (size_t)k * L;
  for (int mm = 0; mm < L; ++mm) acc = fma(ad[mm], v(a * L + mm), acc);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int bp = lv.nbr[a * 6 + 2 * d + 1];
    if (bp >= 0) {
      const double* ao = lv.Ao + ((size_t)a * 3 + d) * L2 + (size_t)k * L;
      for (int mm = 0; mm < L; ++mm) acc = fma(ao[mm], v((int64_t)bp * L + mm), acc);
    }
    const int bm = lv.nbr[a * 6 + 2 * d];
    if (bm >= 0) {
      const double* ao = lv.Ao + ((size_t)bm * 3 + d) * L2 + k;
      for (int mm = 0; mm < L; ++mm) acc = fma(ao[(size_t)mm * L], v((int64_t)bm * L + mm), acc);
    }
  }
  return acc;
}

// sum over the CTAs of partial ``slot`` of right-hand side r (every lane gets it)
__device__ __forceinline__ double inner_total(const double* part, int ncta, int R, int r, int slot, int lane) {
  double v = 0.0;
  for (int k = lane; k < ncta; k += 32) v += __ldcg(part + ((size_t)k * R + r) * 2 + slot);
  return warp_sum(v);
}

template <int LT>
__global__ void __launch_bounds__(kTailThreads) k_inner_pcg(TailArgs A, InnerArgs I, const PcgScalars* osc, int R) {
  if (!cg::this_grid().is_valid()) {   // the grid barrier needs a cooperative launch
    if (threadIdx.x == 0) atomicExch(A.err, 1);
    return;
  }
  const GridBarrier bar{};
  const int cta = (int)blockIdx.x, ncta = (int)gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NW = kTailThreads / 32;
  const CoarseLevel& lv = A.lv[2];
  const int L = LT ? LT : lv.L;
  const int64_t n2 = lv.n;
  const int64_t chunk = (n2 + ncta - 1) / ncta;
  const int64_t row0 = (int64_t)cta * chunk;
  const int64_t row1 = row0 + chunk < n2 ? row0 + chunk : n2;
  __shared__ int s_done[MSMG_MAX_BATCH_RHS];
  __shared__ int s_it[MSMG_MAX_BATCH_RHS];
  __shared__ double s_tol2[MSMG_MAX_BATCH_RHS], s_rz[MSMG_MAX_BATCH_RHS], s_beta[MSMG_MAX_BATCH_RHS],
      s_alpha[MSMG_MAX_BATCH_RHS];
  double* const rv = A.f[2];        // the residual, r_c on entry
  const double* const z = A.w[2];   // the coarse cycle's output
  // The pseudo-inverse acts on the part of r_c in the range of A_2: r_c is
  // orthogonal to A_2's null vector z0 in exact arithmetic (z0 represents the
  // constant), but rounding (FP32 in the mixed form) leaves a component along
  // it, which would make the inner system inconsistent.  Remove it, set x = 0,
  // and take ||r_c||^2.
  for (int r = warp; r < R; r += NW) {
    double v0 = 0.0, v1 = 0.0;
    for (int64_t i = row0 + lane; i < row1; i += 32) {
      const double zi = lv.z[i];
      v0 = fma(zi, rv[(int64_t)r * n2 + i], v0);
      v1 = fma(zi, zi, v1);
    }
    v0 = warp_sum(v0);
    v1 = warp_sum(v1);
    if (lane == 0) {
      I.part[((size_t)cta * R + r) * 2] = v0;
      I.part[((size_t)cta * R + r) * 2 + 1] = v1;
    }
  }
  bar();
  for (int r = warp; r < R; r += NW) {
    const double zr = inner_total(I.part, ncta, R, r, 0, lane);
    const double zz = inner_total(I.part, ncta, R, r, 1, lane);
    const double cz = (I.singular && zz > 0.0) ? zr / zz : 0.0;
    double v = 0.0;
    for (int64_t i = row0 + lane; i < row1; i += 32) {
      const double t = fma(-cz, lv.z[i], rv[(int64_t)r * n2 + i]);
      rv[(int64_t)r * n2 + i] = t;
      I.x[(int64_t)r * n2 + i] = 0.0;
      v = fma(t, t, v);
    }
    v = warp_sum(v);
    s_tol2[r] = v;   // this warp's own partial, written below once every CTA has read slot 0
  }
  bar();   // every CTA has read the null-vector sums
  for (int r = warp; r < R; r += NW)
    if (lane == 0) I.part[((size_t)cta * R + r) * 2] = s_tol2[r];
  bar();
  for (int r = warp; r < R; r += NW) {
    const double t = inner_total(I.part, ncta, R, r, 0, lane);
    if (lane == 0) {
      s_done[r] = ((osc && osc[r].done) || !(t > 0.0)) ? 1 : 0;
      s_tol2[r] = I.rtol2 * t;
      s_rz[r] = 0.0;
      s_it[r] = 0;
    }
  }
  __syncthreads();
  const DoneFlags dn{s_done, 1};
  for (int it = 0; it < I.max_iter; ++it) {
    bool any = false;
    for (int r = 0; r < R; ++r) any |= !s_done[r];
    if (!any) break;
    // z = B_2^{-1} r (its grid barriers also separate the r.r reads above from
    // the next partial sums written below): the coarse cycle from level 2 (Algorithm 1 below level 1)
    tail_run<LT>(A, 0, R, cta, ncta, dn, bar);
    // r.z
    for (int r = warp; r < R; r += NW) {
      if (s_done[r]) continue;
      double v = 0.0;
      for (int64_t i = row0 + lane; i < row1; i += 32) v = fma(rv[(int64_t)r * n2 + i], z[(int64_t)r * n2 + i], v);
      v = warp_sum(v);
      if (lane == 0) I.part[((size_t)cta * R + r) * 2] = v;
    }
    bar();
    for (int r = warp; r < R; r += NW) {
      if (s_done[r]) continue;
      const double rz = inner_total(I.part, ncta, R, r, 0, lane);
      if (lane == 0) {
        s_beta[r] = (it > 0 && s_rz[r] != 0.0) ? rz / s_rz[r] : 0.0;
        s_rz[r] = rz;
        ++s_it[r];
      }
    }
    __syncthreads();
    // p = z + beta p_prev and q = A_2 p (neighbour entries of p formed on the fly
    // from z and p_prev, which are complete), p.q
    const double* pp = (it & 1) ? I.p0 : I.p1;
    double* pc = (it & 1) ? I.p1 : I.p0;
    for (int r = warp; r < R; r += NW) {
      if (s_done[r]) continue;
      const double beta = s_beta[r];
      const int64_t off = (int64_t)r * n2;
      auto pv = [&](int64_t j) { return it > 0 ? fma(beta, pp[off + j], z[off + j]) : z[off + j]; };
      double v = 0.0;
      for (int64_t i = row0 + lane; i < row1; i += 32) {
        const double pi = pv(i);
        const double qi = coarse_apply_row<LT>(lv, i / L, (int)(i % L), pv);
        pc[off + i] = pi;
        I.q[off + i] = qi;
        v = fma(pi, qi, v);
      }
      v = warp_sum(v);
      if (lane == 0) I.part[((size_t)cta * R + r) * 2 + 1] = v;
    }
    bar();
    for (int r = warp; r < R; r += NW) {
      if (s_done[r]) continue;
      const double pq = inner_total(I.part, ncta, R, r, 1, lane);
      if (lane == 0) {
        const double al = s_rz[r] / pq;
        s_alpha[r] = al;
        if (!(pq > 0.0) || !isfinite(al)) s_done[r] = 2;   // breakdown: keep the iterate
      }
    }
    __syncthreads();
    // x += alpha p, r -= alpha q, r.r
    for (int r = warp; r < R; r += NW) {
      if (s_done[r]) continue;
      const double al = s_alpha[r];
      const int64_t off = (int64_t)r * n2;
      double v = 0.0;
      for (int64_t i = row0 + lane; i < row1; i += 32) {
        I.x[off + i] = fma(al, pc[off + i], I.x[off + i]);
        const double ri = fma(-al, I.q[off + i], rv[off + i]);
        rv[off + i] = ri;
        v = fma(ri, ri, v);
      }
      v = warp_sum(v);
      if (lane == 0) I.part[((size_t)cta * R + r) * 2] = v;
    }
    bar();
    for (int r = warp; r < R; r += NW) {
      if (s_done[r]) continue;
      const double rr = inner_total(I.part, ncta, R, r, 0, lane);
      if (lane == 0 && rr <= s_tol2[r]) s_done[r] = 1;
    }
    __syncthreads();
  }
  // minimum-norm solution: x -= (z0.x / z0.z0) z0, z0 the null vector of A_2
  bar();   // every CTA has read the last partial sums
  for (int r = warp; r < R; r += NW) {
    if (osc && osc[r].done) continue;
    double v0 = 0.0, v1 = 0.0;
    for (int64_t i = row0 + lane; i < row1; i += 32) {
      const double zi = lv.z[i];
      v0 = fma(zi, I.x[(int64_t)r * n2 + i], v0);
      v1 = fma(zi, zi, v1);
    }
    v0 = warp_sum(v0);
    v1 = warp_sum(v1);
    if (lane == 0) {
      I.part[((size_t)cta * R + r) * 2] = v0;
      I.part[((size_t)cta * R + r) * 2 + 1] = v1;
    }
  }
  bar();
  for (int r = warp; r < R; r += NW) {
    if (osc && osc[r].done) continue;
    const double zx = inner_total(I.part, ncta, R, r, 0, lane);
    const double zz = inner_total(I.part, ncta, R, r, 1, lane);
    const double cz = (I.singular && zz > 0.0) ? zx / zz : 0.0;
    for (int64_t i = row0 + lane; i < row1; i += 32) {
      const double xi = fma(-cz, lv.z[i], I.x[(int64_t)r * n2 + i]);
      I.x[(int64_t)r * n2 + i] = xi;
      if (I.out32) I.out32[(int64_t)r * n2 + i] = (float)xi;
    }
    if (cta == 0 && lane == 0) I.iters[r] += s_it[r];
  }
}

static inline unsigned coarse_threads(const CoarseLevel& lv) { return coarse_threads_d(lv.nP, lv.Lnext); }
template <typename S>
static inline size_t smem_smooth(const CoarseLevel& lv) {
  return ((size_t)lv.nP * lv.nP + lv.nP) * sizeof(S) + 16;
}
template <typename S>
static inline size_t smem_restrict(const CoarseLevel& lv) {
  return ((size_t)lv.Lnext * lv.nP + (size_t)lv.Lnext * (coarse_threads(lv) / 32) + lv.nP) * sizeof(S) + 16;
}
static inline unsigned coarse_threads4(const CoarseLevel& lv) { return coarse_threads4_d(lv.nP, lv.Lnext); }

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
    cudaFuncSetAttribute(k_coarse_smooth_first<S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm1);
    cudaFuncSetAttribute(k_coarse_smooth_first<S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm1);
    with_L(lv.L, [&](auto LC) {
      constexpr int LT = decltype(LC)::value;
      cudaFuncSetAttribute(k_coarse_resid_smooth<LT, S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm1);
      cudaFuncSetAttribute(k_coarse_resid_smooth<LT, S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm1);
      cudaFuncSetAttribute(k_coarse_resid_restrict<LT, S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2);
      cudaFuncSetAttribute(k_coarse_resid_restrict<LT, S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm2);
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
constexpr int kInnerMaxCtas = 1024;   // CTAs of the exact two-grid solve (partials are sized for it)

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

template <int LT>
static void inner_prepare_lt(msmg_ctx* c) {
  c->inner_grid = 0;
  int coop = 0, dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (!coop || nsm < 1) return;
  cudaFuncSetAttribute(k_inner_pcg<LT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->coop_smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_inner_pcg<LT>, kTailThreads, c->coop_smem) !=
          cudaSuccess || per < 1) {
    cudaGetLastError();
    return;
  }
  int g = nsm * (per < 2 ? per : 2);
  if (g > kInnerMaxCtas) g = kInnerMaxCtas;
  c->inner_grid = g;
}

// Exact two-grid: the level-2 solve as one cooperative launch.  Returns the
// level-2 correction (FP64; its FP32 copy is written too in the mixed form).
static const double* launch_inner(msmg_ctx* c, PcgScalars* sc, cudaStream_t s) {
  TailArgs A = tail_args(c, 2);
  A.out32 = nullptr;
  const int R = c->sb.R;
  InnerArgs I;
  I.x = c->sb.ix;
  I.p0 = c->sb.ip0;
  I.p1 = c->sb.ip1;
  I.q = c->sb.iq;
  I.part = c->sb.ipart;
  I.iters = c->sb.iiters;
  I.out32 = c->sb.ec32;
  I.rtol2 = c->opts.inner_rtol * c->opts.inner_rtol;
  I.max_iter = c->opts.inner_max_iter;
  I.singular = c->fine.Wd == nullptr ? 1 : 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)c->inner_grid);
  cfg.blockDim = dim3(kTailThreads);
  cfg.dynamicSmemBytes = c->coop_smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaSuccess;
  with_L(c->coop_lt, [&](auto LC) { e = cudaLaunchKernelEx(&cfg, k_inner_pcg<decltype(LC)::value>, A, I, (const PcgScalars*)sc, R); });
  if (e != cudaSuccess) set_last_cuda_error(e);
  return c->sb.ix;
}

// Shared-memory limits of the coarse kernels and the fused forms (set once per
// context, never during capture).
void prepare_coarse_kernels(msmg_ctx* c) {
  prepare_t<double>(c);
  tail_prepare(c);
  c->inner_grid = 0;
  if (c->opts.two_grid && c->nL >= 3 && c->coop_smem)
    with_L(c->coop_lt, [&](auto LC) { inner_prepare_lt<decltype(LC)::value>(c); });
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
    k_dense_gemv<S><<<grid, 256, 0, s>>>(lv.pinv, f, u, l == 2 ? c->sb.ec32 : nullptr, lv.n, lv.nk, lv.cmap,
                                         lv.cinv, sc, R);
    return u;
  }
  const LevelData<S> D = level_data<S>(lv);
  S* fn = (S*)c->sb.vf[l + 1];
  const unsigned grid = (unsigned)(lv.mP * R);
  // four threads per row when the level's CTAs leave the GPU short of warps
  const bool quad = grid < (unsigned)(152 * 8);
  const unsigned thr = coarse_threads(lv), thrs = quad ? coarse_threads4(lv) : thr;
  if (quad) k_coarse_smooth_first<S, true><<<grid, thrs, smem_smooth<S>(lv), s>>>(lv, D, f, u, sc, R);
  else k_coarse_smooth_first<S, false><<<grid, thrs, smem_smooth<S>(lv), s>>>(lv, D, f, u, sc, R);
  with_L(lv.L, [&](auto LC) {
    constexpr int LT = decltype(LC)::value;
    if (quad)
      k_coarse_resid_restrict<LT, S, true><<<grid, thrs, smem_restrict<S>(lv), s>>>(lv, D, f, u, fn, sc, R);
    else
      k_coarse_resid_restrict<LT, S, false><<<grid, thrs, smem_restrict<S>(lv), s>>>(lv, D, f, u, fn, sc, R);
  });
  const S* e = coarse_cycle_t<S>(c, l + 1, sc, s);
  k_coarse_prolong<S><<<grid, thr, 0, s>>>(lv, D, u, e, sc, R);
  with_L(lv.L, [&](auto LC) {
    constexpr int LT = decltype(LC)::value;
    float* o32 = l == 2 ? c->sb.ec32 : nullptr;
    if (quad) k_coarse_resid_smooth<LT, S, true><<<grid, thrs, smem_smooth<S>(lv), s>>>(lv, D, f, u, w, o32, sc, R);
    else k_coarse_resid_smooth<LT, S, false><<<grid, thrs, smem_smooth<S>(lv), s>>>(lv, D, f, u, w, o32, sc, R);
  });
  return w;
}

// Returns the level-2 correction in the V-cycle precision: FP64, or its FP32
// copy in the mixed form.
const void* coarse_cycle(msmg_ctx* c, int l, PcgScalars* sc, cudaStream_t s) {
  const double* e = (l == 2 && c->opts.two_grid) ? launch_inner(c, sc, s) : coarse_cycle_t<double>(c, l, sc, s);
  return c->sb.ec32 ? (const void*)c->sb.ec32 : (const void*)e;
}

}  // namespace msmg
