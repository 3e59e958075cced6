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
#include <type_traits>

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

static inline unsigned coarse_threads(const CoarseLevel& lv) {
  int t = lv.nP > lv.Lnext ? lv.nP : lv.Lnext;
  if (t < 64) t = 64;
  return (unsigned)((t + 31) / 32 * 32);
}
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

// Shared-memory limits of the coarse kernels (set once per context, never during capture).
void prepare_coarse_kernels(msmg_ctx* c) { prepare_t<double>(c); }

// Level-l part of the V-cycle (l >= 2): on entry vf[l] holds the right side;
// returns the device pointer holding the level-l correction.
template <typename S>
static const S* coarse_cycle_t(msmg_ctx* c, int l, PcgScalars* sc, cudaStream_t s) {
  CoarseLevel& lv = c->lev[l];
  S* f = (S*)c->sb.vf[l];
  S* u = (S*)c->sb.vu[l];
  S* w = (S*)c->sb.vw[l];
  const int R = c->sb.R;
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
