// Fine-level PCG iteration kernels, one warp per element.
//
// Each element of E_1 (bx x by x bz cells) is handled by one warp: its data
// is one contiguous chunk of every block-major array, loaded with coalesced
// lane-strided accesses into a padded shared-memory tile together with the
// one-cell halo from the face-adjacent elements.  The incomplete-Cholesky
// solves of the block-Jacobi smoother (Section 5) sweep the element in
// wavefronts lx + ly + lz = const; the lanes own the x-lines (ly, lz) of the
// element, so consecutive wavefronts only need a warp-level barrier.
//
// One PCG iteration on the fine level is five kernels:
//   k_pmatvec  p = z + beta p_old (cells and halo), q = A p, reduce p.q -> alpha
//   k_pre      x += alpha p, r -= alpha q, reduce r.r (convergence), and the
//              pre-smoothing u = M^{-1} r of Algorithm 1 (from u = 0)
//   k_restrict r_c = Phi^T (r - A u) per element (Algorithm 1, restriction)
//   k_prolong  u += Phi e_c (Algorithm 1, prolongation)   [fine.cu]
//   k_post     z = u + M^{-T} (r - A u), reduce r.z (and z.q for the flexible beta)
#include "msmg_internal.cuh"
#include "reduce.cuh"

namespace msmg {

struct WGeo {
  int bx, by, bz, nb, nlines, P;
};

static inline WGeo make_wgeo(int bx, int by, int bz) {
  WGeo g;
  g.bx = bx; g.by = by; g.bz = bz; g.nb = bx * by * bz; g.nlines = by * bz;
  g.P = (bx + 2) * (by + 2) * (bz + 2);
  return g;
}

constexpr int kWarpsPerCta = 4;

__device__ __forceinline__ int wpad(const WGeo& g, int lx, int ly, int lz) {
  return (lx + 1) + (g.bx + 2) * ((ly + 1) + (g.by + 2) * (lz + 1));
}
__device__ __forceinline__ int wpad_cell(const WGeo& g, int c) {
  const int lx = c % g.bx, t = c / g.bx;
  return wpad(g, lx, t % g.by, t / g.by);
}

// Interior of element e of X into a padded tile (lane-strided, coalesced).
template <typename Src, typename Dst>
__device__ __forceinline__ void w_load_interior(Dst* tile, const Src* __restrict__ X, int64_t e, const WGeo& g,
                                                int lane) {
  const Src* src = X + e * g.nb;
  for (int c = lane; c < g.nb; c += 32) tile[wpad_cell(g, c)] = (Dst)src[c];
}

// Face halo of element e: faces selected by mask (bit f: -x,+x,-y,+y,-z,+z);
// zero outside the domain.  Optional per-cell transform for the halo value.
template <typename Src, typename Dst>
__device__ __forceinline__ void w_load_halo(Dst* tile, const Src* __restrict__ X, int64_t e, const int* __restrict__ nbr,
                                            const WGeo& g, int lane, int mask) {
  const int F0 = g.by * g.bz, F1 = g.bx * g.bz, F2 = g.bx * g.by;
  for (int f = 0; f < 6; ++f) {
    if (!((mask >> f) & 1)) continue;
    const int ne = nbr[e * 6 + f];
    const int d = f >> 1;
    const bool plus = f & 1;
    const int F = d == 0 ? F0 : (d == 1 ? F1 : F2);
    for (int h = lane; h < F; h += 32) {
      int dx, dy, dz, sx, sy, sz;
      if (d == 0) { const int u = h % g.by, v = h / g.by; dy = sy = u; dz = sz = v; dx = plus ? g.bx : -1; sx = plus ? 0 : g.bx - 1; }
      else if (d == 1) { const int u = h % g.bx, v = h / g.bx; dx = sx = u; dz = sz = v; dy = plus ? g.by : -1; sy = plus ? 0 : g.by - 1; }
      else { const int u = h % g.bx, v = h / g.bx; dx = sx = u; dy = sy = v; dz = plus ? g.bz : -1; sz = plus ? 0 : g.bz - 1; }
      Dst val = (Dst)0;
      if (ne >= 0) val = (Dst)X[(int64_t)ne * g.nb + sx + g.bx * (sy + g.by * sz)];
      tile[wpad(g, dx, dy, dz)] = val;
    }
  }
}

// Element context: base offset and the six neighbour element bases (-1: none).
struct WElem {
  int64_t base;
  int64_t nb6[6];
};

__device__ __forceinline__ WElem w_elem(int64_t e, const int* __restrict__ nbr, const WGeo& g) {
  WElem E;
  E.base = e * g.nb;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int ne = nbr[e * 6 + f];
    E.nb6[f] = ne >= 0 ? (int64_t)ne * g.nb : -1;
  }
  return E;
}

// Coefficient of the -d face of local cell (lx, ly, lz): in-element, or from the
// -d neighbour element, or zero on the domain boundary.  T is read through L1.
template <typename V>
__device__ __forceinline__ V w_Tminus(const V* __restrict__ Td, const WElem& E, const WGeo& g, int d, int c, int lc) {
  const int st = d == 0 ? 1 : (d == 1 ? g.bx : g.bx * g.by);
  const int bd = d == 0 ? g.bx : (d == 1 ? g.by : g.bz);
  if (lc > 0) return __ldg(Td + E.base + c - st);
  const int64_t nb = E.nb6[2 * d];
  return nb >= 0 ? __ldg(Td + nb + c + (bd - 1) * st) : (V)0;
}

// (A u)_c: u from the padded tile, coefficients from global memory (L1).
template <typename V>
__device__ __forceinline__ V w_apply_A(const V* ut, const V* __restrict__ T, int64_t n, const WElem& E, const WGeo& g,
                                       int c) {
  const int lx = c % g.bx, t = c / g.bx, ly = t % g.by, lz = t / g.by;
  const int pc = wpad(g, lx, ly, lz);
  const int sy = g.bx + 2, sz = (g.bx + 2) * (g.by + 2);
  const V uc = ut[pc];
  const V tx = __ldg(T + E.base + c), ty = __ldg(T + n + E.base + c), tz = __ldg(T + 2 * n + E.base + c);
  const V mx = w_Tminus(T, E, g, 0, c, lx), my = w_Tminus(T + n, E, g, 1, c, ly), mz = w_Tminus(T + 2 * n, E, g, 2, c, lz);
  V acc = tx * (uc - ut[pc + 1]) + mx * (uc - ut[pc - 1]);
  acc += ty * (uc - ut[pc + sy]) + my * (uc - ut[pc - sy]);
  acc += tz * (uc - ut[pc + sz]) + mz * (uc - ut[pc - sz]);
  return acc;
}

// y <- M^{-1} y on the element, M = (D~ + L) D~^{-1} (D~ + L^T): forward then
// backward wavefronts; lanes own x-lines; y indexed by the element-local cell.
template <typename V>
__device__ __forceinline__ void w_ic0(V* y, const V* __restrict__ T, const V* __restrict__ invd, int64_t n,
                                      const WElem& E, const WGeo& g, int lane) {
  const int smax = g.bx + g.by + g.bz - 3;
  const int bxy = g.bx * g.by;
  const V* T0 = T + E.base;
  const V* T1 = T + n + E.base;
  const V* T2 = T + 2 * n + E.base;
  const V* D = invd + E.base;
  for (int w = 0; w <= smax; ++w) {
    for (int l = lane; l < g.nlines; l += 32) {
      const int ly = l % g.by, lz = l / g.by;
      const int lx = w - ly - lz;
      if (lx < 0 || lx >= g.bx) continue;
      const int c = lx + g.bx * ly + bxy * lz;
      V acc = y[c];
      if (lx > 0) acc += __ldg(T0 + c - 1) * y[c - 1];
      if (ly > 0) acc += __ldg(T1 + c - g.bx) * y[c - g.bx];
      if (lz > 0) acc += __ldg(T2 + c - bxy) * y[c - bxy];
      y[c] = acc * __ldg(D + c);
    }
    __syncwarp();
  }
  for (int w = smax; w >= 0; --w) {
    for (int l = lane; l < g.nlines; l += 32) {
      const int ly = l % g.by, lz = l / g.by;
      const int lx = w - ly - lz;
      if (lx < 0 || lx >= g.bx) continue;
      const int c = lx + g.bx * ly + bxy * lz;
      V acc = (V)0;
      if (lx < g.bx - 1) acc += __ldg(T0 + c) * y[c + 1];
      if (ly < g.by - 1) acc += __ldg(T1 + c) * y[c + g.bx];
      if (lz < g.bz - 1) acc += __ldg(T2 + c) * y[c + bxy];
      y[c] += __ldg(D + c) * acc;
    }
    __syncwarp();
  }
}

template <typename V>
struct WTiles {
  V *ut, *y;
};

// per warp: padded u tile (P) and the wavefront vector (nb)
template <typename V>
__device__ __forceinline__ WTiles<V> w_carve(unsigned char* base, const WGeo& g, int warp) {
  V* p = reinterpret_cast<V*>(base) + (size_t)warp * (g.P + g.nb);
  WTiles<V> t;
  t.ut = p;
  t.y = p + g.P;
  return t;
}

// ------------------------------------------------------------------ k_pre
// update != 0: x += alpha p, r -= alpha q, rr = r.r (convergence bookkeeping);
// then f = r (in V precision, also written to rv) and u = M^{-1} f.
template <typename V>
__global__ void __launch_bounds__(kWarpsPerCta * 32) k_pre(double* __restrict__ x, double* __restrict__ r,
                                                           const double* __restrict__ p, const double* __restrict__ q,
                                                           const V* __restrict__ T, const V* __restrict__ invd,
                                                           V* __restrict__ rv, V* __restrict__ u, int64_t n, WGeo g,
                                                           int64_t m, const int* __restrict__ nbr, int update,
                                                           RedSlot red, PcgScalars* sc) {
  if (sc && sc->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * kWarpsPerCta + warp;
  const bool act = e < m;
  const WTiles<V> s = w_carve<V>(smem, g, warp);
  double acc = 0.0;
  if (act) {
    const double alpha = update ? sc->alpha : 0.0;
    const WElem E = w_elem(e, nbr, g);
    const int64_t base = E.base;
    for (int c = lane; c < g.nb; c += 32) {
      double rc = r[base + c];
      if (update) {
        x[base + c] += alpha * p[base + c];
        rc -= alpha * q[base + c];
        r[base + c] = rc;
        acc += rc * rc;
      }
      const V fv = (V)rc;
      s.y[c] = fv;
      rv[base + c] = fv;
    }
    __syncwarp();
    w_ic0(s.y, T, invd, n, E, g, lane);
    for (int c = lane; c < g.nb; c += 32) u[base + c] = s.y[c];
  }
  if (update) {
    double v[1] = {acc};
    grid_reduce<1>(v, red, [=] __device__(double* t) {
      sc->rr = t[0];
      sc->iter += 1;
      if (!isfinite(t[0])) sc->done = 2;
      else if (t[0] <= sc->tol2) sc->done = 1;
      else if (sc->iter >= sc->max_iter) sc->done = 3;
    });
  }
}

// ------------------------------------------------------------------ k_restrict
template <typename V, typename BT>
__global__ void __launch_bounds__(kWarpsPerCta * 32) k_restrict(const V* __restrict__ f, const V* __restrict__ u,
                                                                const V* __restrict__ T, const BT* __restrict__ Phi,
                                                                int L, double* __restrict__ rc, int64_t n, WGeo g,
                                                                int64_t m, const int* __restrict__ nbr,
                                                                const PcgScalars* sc) {
  if (sc && sc->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * kWarpsPerCta + warp;
  if (e >= m) return;
  const WTiles<V> s = w_carve<V>(smem, g, warp);
  const WElem E = w_elem(e, nbr, g);
  w_load_interior(s.ut, u, e, g, lane);
  w_load_halo(s.ut, u, e, nbr, g, lane, 0x3f);
  __syncwarp();
  const int64_t base = E.base;
  for (int c = lane; c < g.nb; c += 32) s.y[c] = f[base + c] - w_apply_A(s.ut, T, n, E, g, c);
  __syncwarp();
  // accumulate in the V-cycle precision (FP32 in the mixed form: the FP64 pipe of
  // this part is 1/64 of its FP32 rate)
  for (int k = 0; k < L; ++k) {
    const BT* ph = Phi + (e * L + k) * g.nb;
    V acc = (V)0;
    for (int c = lane; c < g.nb; c += 32) acc += (V)ph[c] * s.y[c];
    acc = warp_sum_t(acc);
    if (lane == 0) rc[e * L + k] = (double)acc;
  }
}

// ------------------------------------------------------------------ k_post
// z = u + M^{-1} (f - A u); reductions: r.z (FP64 r) and z.q (flexible beta).
template <typename V>
__global__ void __launch_bounds__(kWarpsPerCta * 32) k_post(const V* __restrict__ f, const double* __restrict__ r,
                                                            const V* __restrict__ u, const V* __restrict__ T,
                                                            const V* __restrict__ invd, V* __restrict__ z,
                                                            const double* __restrict__ qv, int64_t n, WGeo g,
                                                            int64_t m, const int* __restrict__ nbr, RedSlot red,
                                                            PcgScalars* sc) {
  if (sc && sc->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * kWarpsPerCta + warp;
  const bool act = e < m;
  const WTiles<V> s = w_carve<V>(smem, g, warp);
  double v[2] = {0.0, 0.0};
  if (act) {
    const WElem E = w_elem(e, nbr, g);
    const int64_t base = E.base;
    w_load_interior(s.ut, u, e, g, lane);
    w_load_halo(s.ut, u, e, nbr, g, lane, 0x3f);
    __syncwarp();
    for (int c = lane; c < g.nb; c += 32) s.y[c] = f[base + c] - w_apply_A(s.ut, T, n, E, g, c);
    __syncwarp();
    w_ic0(s.y, T, invd, n, E, g, lane);
    for (int c = lane; c < g.nb; c += 32) {
      const V zc = s.ut[wpad_cell(g, c)] + s.y[c];
      z[base + c] = zc;
      if (sc) {
        v[0] += r[base + c] * (double)zc;
        if (qv) v[1] += (double)zc * qv[base + c];
      }
    }
  }
  if (sc) {
    grid_reduce<2>(v, red, [=] __device__(double* t) {
      sc->rz_old = sc->rz;
      sc->rz = t[0];
      if (sc->flexible) sc->beta = sc->rz_old != 0.0 ? -sc->alpha * t[1] / sc->rz_old : 0.0;
      else sc->beta = sc->rz_old != 0.0 ? t[0] / sc->rz_old : 0.0;
      if (!isfinite(t[0])) sc->done = 2;
    });
  }
}

// ------------------------------------------------------------------ k_pmatvec
// p = z + beta p_old on the element and its halo, q = A p (FP64), reduce p.q.
template <typename V>
__global__ void __launch_bounds__(kWarpsPerCta * 32) k_pmatvec(const V* __restrict__ z, const double* __restrict__ pold,
                                                               double* __restrict__ pnew, double* __restrict__ q,
                                                               const double* __restrict__ T, int64_t n, WGeo g,
                                                               int64_t m, const int* __restrict__ nbr, RedSlot red,
                                                               PcgScalars* sc) {
  if (sc->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * kWarpsPerCta + warp;
  const bool act = e < m;
  const WTiles<double> s = w_carve<double>(smem, g, warp);
  double acc = 0.0;
  if (act) {
    const double beta = sc->beta;
    const int64_t base = e * g.nb;
    // p tile: interior and halo, p = z + beta pold
    for (int c = lane; c < g.nb; c += 32) {
      const double pv = (double)z[base + c] + beta * pold[base + c];
      s.ut[wpad_cell(g, c)] = pv;
      pnew[base + c] = pv;
    }
    {
      const int F0 = g.by * g.bz, F1 = g.bx * g.bz, F2 = g.bx * g.by;
      for (int f = 0; f < 6; ++f) {
        const int ne = nbr[e * 6 + f];
        const int d = f >> 1;
        const bool plus = f & 1;
        const int F = d == 0 ? F0 : (d == 1 ? F1 : F2);
        for (int h = lane; h < F; h += 32) {
          int dx, dy, dz, sx, sy, sz;
          if (d == 0) { const int uu = h % g.by, vv = h / g.by; dy = sy = uu; dz = sz = vv; dx = plus ? g.bx : -1; sx = plus ? 0 : g.bx - 1; }
          else if (d == 1) { const int uu = h % g.bx, vv = h / g.bx; dx = sx = uu; dz = sz = vv; dy = plus ? g.by : -1; sy = plus ? 0 : g.by - 1; }
          else { const int uu = h % g.bx, vv = h / g.bx; dx = sx = uu; dy = sy = vv; dz = plus ? g.bz : -1; sz = plus ? 0 : g.bz - 1; }
          double val = 0.0;
          if (ne >= 0) {
            const int64_t src = (int64_t)ne * g.nb + sx + g.bx * (sy + g.by * sz);
            val = (double)z[src] + beta * pold[src];
          }
          s.ut[wpad(g, dx, dy, dz)] = val;
        }
      }
    }
    __syncwarp();
    const WElem E = w_elem(e, nbr, g);
    for (int c = lane; c < g.nb; c += 32) {
      const int pc = wpad_cell(g, c);
      const double a = w_apply_A(s.ut, T, n, E, g, c);
      q[base + c] = a;
      acc += a * s.ut[pc];
    }
  }
  double v[1] = {acc};
  grid_reduce<1>(v, red, [=] __device__(double* t) {
    sc->pq = t[0];
    if (!(t[0] > 0.0) || !isfinite(t[0])) { sc->done = 2; sc->alpha = 0.0; }
    else sc->alpha = sc->rz / t[0];
  });
}

// z (V) -> FP64
template <typename V>
__global__ void k_widen(const V* __restrict__ a, double* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

// ------------------------------------------------------------------ host side
template <typename V, typename BT>
struct FineOps {
  const V* T;
  const V* invd;
  const BT* Phi;
};

static inline size_t wsmem(const WGeo& g, size_t vsize) {
  return (size_t)kWarpsPerCta * (g.P + g.nb) * vsize;
}

template <typename V, typename BT>
static void pre_t(msmg_ctx* c, const FineOps<V, BT>& o, int update, PcgScalars* sc, cudaStream_t s) {
  const WGeo g = make_wgeo(c->fine.bx, c->fine.by, c->fine.bz);
  const unsigned grid = (unsigned)((c->fine.m + kWarpsPerCta - 1) / kWarpsPerCta);
  const size_t sm = wsmem(g, sizeof(V));
  SolveBuffers& B = c->sb;
  k_pre<V><<<grid, kWarpsPerCta * 32, sm, s>>>(B.x, B.r, B.pcur, B.q, o.T, o.invd, (V*)B.rv, (V*)B.vu[1], c->n, g,
                                               c->fine.m, c->fine.nbr, update, c->red, sc);
}

template <typename V, typename BT>
static void restrict_t(msmg_ctx* c, const FineOps<V, BT>& o, PcgScalars* sc, cudaStream_t s) {
  const WGeo g = make_wgeo(c->fine.bx, c->fine.by, c->fine.bz);
  const unsigned grid = (unsigned)((c->fine.m + kWarpsPerCta - 1) / kWarpsPerCta);
  const size_t sm = wsmem(g, sizeof(V));
  SolveBuffers& B = c->sb;
  k_restrict<V, BT><<<grid, kWarpsPerCta * 32, sm, s>>>((const V*)B.rv, (const V*)B.vu[1], o.T, o.Phi, c->fine.L,
                                                        (double*)B.vf[2], c->n, g, c->fine.m, c->fine.nbr, sc);
}

template <typename V, typename BT>
static void post_t(msmg_ctx* c, const FineOps<V, BT>& o, const double* qv, PcgScalars* sc, cudaStream_t s) {
  const WGeo g = make_wgeo(c->fine.bx, c->fine.by, c->fine.bz);
  const unsigned grid = (unsigned)((c->fine.m + kWarpsPerCta - 1) / kWarpsPerCta);
  const size_t sm = wsmem(g, sizeof(V));
  SolveBuffers& B = c->sb;
  k_post<V><<<grid, kWarpsPerCta * 32, sm, s>>>((const V*)B.rv, B.r, (const V*)B.vu[1], o.T, o.invd, (V*)B.zv, qv,
                                                c->n, g, c->fine.m, c->fine.nbr, c->red, sc);
}

template <typename V>
static void pmatvec_t(msmg_ctx* c, PcgScalars* sc, cudaStream_t s) {
  const WGeo g = make_wgeo(c->fine.bx, c->fine.by, c->fine.bz);
  const unsigned grid = (unsigned)((c->fine.m + kWarpsPerCta - 1) / kWarpsPerCta);
  const size_t sm = wsmem(g, sizeof(double));
  SolveBuffers& B = c->sb;
  k_pmatvec<V><<<grid, kWarpsPerCta * 32, sm, s>>>((const V*)B.zv, B.pcur, B.pnext, B.q, c->fine.T, c->n, g,
                                                   c->fine.m, c->fine.nbr, c->red, sc);
}

template <typename V, typename BT>
void launch_prolong_fine(msmg_ctx* c, const BT* Phi, const double* ec, PcgScalars* sc, cudaStream_t s);

// Shared-memory limits of the fine-level kernels, set once per context (never
// during stream capture).
template <typename V, typename BT>
static void prepare_t(msmg_ctx* c) {
  const WGeo g = make_wgeo(c->fine.bx, c->fine.by, c->fine.bz);
  const int smv = (int)wsmem(g, sizeof(V)), smd = (int)wsmem(g, sizeof(double));
  cudaFuncSetAttribute(k_pre<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, smv);
  cudaFuncSetAttribute(k_restrict<V, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smv);
  cudaFuncSetAttribute(k_post<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, smv);
  cudaFuncSetAttribute(k_pmatvec<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, smd);
}

void prepare_fine_kernels(msmg_ctx* c) {
  if (c->opts.precision == MSMG_MIXED) prepare_t<float, float>(c);
  else prepare_t<double, double>(c);
}

const double* coarse_cycle(msmg_ctx* c, int l, PcgScalars* sc, cudaStream_t s);

// Fine-level V-cycle on the residual held in B.r (FP64); result in B.zv (V).
// update != 0 first performs the PCG update of x and r with the current alpha.
template <typename V, typename BT>
static void vcycle_t(msmg_ctx* c, const FineOps<V, BT>& o, int update, const double* qv, PcgScalars* sc,
                     cudaStream_t s) {
  pre_t<V, BT>(c, o, update, sc, s);
  restrict_t<V, BT>(c, o, sc, s);
  const double* ec = coarse_cycle(c, 2, sc, s);
  launch_prolong_fine<V, BT>(c, o.Phi, ec, sc, s);
  post_t<V, BT>(c, o, qv, sc, s);
}

void pcg_step_vcycle(msmg_ctx* c, int update, const double* qv, PcgScalars* sc, cudaStream_t s) {
  if (c->opts.precision == MSMG_MIXED) {
    FineOps<float, float> o{c->fine.T32, c->fine.invd32, c->fine.Phi32};
    vcycle_t<float, float>(c, o, update, qv, sc, s);
  } else {
    FineOps<double, double> o{c->fine.T, c->fine.invd, c->fine.Phi};
    vcycle_t<double, double>(c, o, update, qv, sc, s);
  }
}

template <typename V, typename BT>
static void vcycle_timed_t(msmg_ctx* c, const FineOps<V, BT>& o, int update, const double* qv, PcgScalars* sc,
                           cudaStream_t s, cudaEvent_t* ev) {
  cudaEventRecord(ev[0], s);
  pre_t<V, BT>(c, o, update, sc, s);
  cudaEventRecord(ev[1], s);
  restrict_t<V, BT>(c, o, sc, s);
  cudaEventRecord(ev[2], s);
  const double* ec = coarse_cycle(c, 2, sc, s);
  cudaEventRecord(ev[3], s);
  launch_prolong_fine<V, BT>(c, o.Phi, ec, sc, s);
  cudaEventRecord(ev[4], s);
  post_t<V, BT>(c, o, qv, sc, s);
  cudaEventRecord(ev[5], s);
}

void pcg_step_vcycle_timed(msmg_ctx* c, int update, const double* qv, PcgScalars* sc, cudaStream_t s,
                           cudaEvent_t* ev) {
  if (c->opts.precision == MSMG_MIXED) {
    FineOps<float, float> o{c->fine.T32, c->fine.invd32, c->fine.Phi32};
    vcycle_timed_t<float, float>(c, o, update, qv, sc, s, ev);
  } else {
    FineOps<double, double> o{c->fine.T, c->fine.invd, c->fine.Phi};
    vcycle_timed_t<double, double>(c, o, update, qv, sc, s, ev);
  }
}

void pcg_step_pmatvec(msmg_ctx* c, PcgScalars* sc, cudaStream_t s) {
  if (c->opts.precision == MSMG_MIXED) pmatvec_t<float>(c, sc, s);
  else pmatvec_t<double>(c, sc, s);
}

// z = P^{-1} r in FP64 (natural order handled by the caller): r in B.r, result in B.z.
void apply_vcycle_fp64_out(msmg_ctx* c, cudaStream_t s) {
  pcg_step_vcycle(c, 0, nullptr, nullptr, s);
  const unsigned g1 = (unsigned)((c->n + 255) / 256);
  if (c->opts.precision == MSMG_MIXED) k_widen<float><<<g1, 256, 0, s>>>((const float*)c->sb.zv, c->sb.z, c->n);
  else k_widen<double><<<g1, 256, 0, s>>>((const double*)c->sb.zv, c->sb.z, c->n);
}

int fine_warp_vcycle_launches(const msmg_ctx* c) { return 4; }

}  // namespace msmg
