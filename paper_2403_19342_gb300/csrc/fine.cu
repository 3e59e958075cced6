// Fine-level kernels: face coefficients (Section 2.2), IC(0) pivots of the
// block-Jacobi smoother (Section 5), the two-point-flux stencil
// (Eq. (discrete varia)), and the fine-level steps of the V-cycle
// (Algorithm 1: pre-smoothing, residual restriction with the local
// eigenbases, prolongation, post-smoothing).
//
// Every kernel works element by element: one group of nb threads per element
// (nb = cells per element), ``epc`` elements per CTA.  An element's cells and
// the one-cell halo on its six faces are staged in shared memory as a padded
// (bx+2)(by+2)(bz+2) tile; the halo comes from the face-adjacent elements
// (their data is one contiguous chunk each in the block-major layout).
#include "msmg_internal.cuh"
#include "reduce.cuh"
#include "linalg_small.cuh"

namespace msmg {

struct Geo {
  int bx, by, bz, nb, epc, P;   // P = padded tile size
};

__host__ __device__ inline Geo make_geo(int bx, int by, int bz) {
  Geo g;
  g.bx = bx; g.by = by; g.bz = bz; g.nb = bx * by * bz;
  g.epc = g.nb >= 256 ? 1 : 256 / g.nb;
  g.P = (bx + 2) * (by + 2) * (bz + 2);
  return g;
}

__device__ __forceinline__ int pad(const Geo& g, int lx, int ly, int lz) {
  return (lx + 1) + (g.bx + 2) * ((ly + 1) + (g.by + 2) * (lz + 1));
}

// Thread -> (element in CTA, local cell); ``valid`` false for padding threads
// and elements past the end.
struct Slot {
  int eloc;       // element index inside the CTA
  int p;          // local cell
  int64_t e;      // global (hierarchical) element
  int lx, ly, lz;
  bool valid;
};

__device__ __forceinline__ Slot make_slot(const Geo& g, int64_t m, unsigned blk) {
  Slot s;
  s.eloc = threadIdx.x / g.nb;
  s.p = threadIdx.x % g.nb;
  s.e = (int64_t)blk * g.epc + s.eloc;
  s.valid = (s.eloc < g.epc) && (s.e < m);
  s.lx = s.p % g.bx;
  int t = s.p / g.bx;
  s.ly = t % g.by;
  s.lz = t / g.by;
  return s;
}

// Stage field X (block-major) of element s.e into a padded tile, including the
// one-cell halo on the faces selected by ``face_mask`` (bit f for face f =
// -x,+x,-y,+y,-z,+z).  Halo cells outside the domain are zero.
template <typename Src, typename Dst>
__device__ void load_tile(Dst* tile, const Src* X, const Slot& s, const Geo& g, const int* nbr, int face_mask) {
  if (s.valid) tile[pad(g, s.lx, s.ly, s.lz)] = (Dst)X[s.e * g.nb + s.p];
  if (s.eloc >= g.epc) return;
  const int F0 = g.by * g.bz, F1 = g.bx * g.bz, F2 = g.bx * g.by;
  const int H = 2 * (F0 + F1 + F2);
  for (int h = s.p; h < H; h += g.nb) {
    int f, u, v;
    if (h < 2 * F0) { f = h / F0; int q = h % F0; u = q % g.by; v = q / g.by; }
    else if (h < 2 * (F0 + F1)) { int hh = h - 2 * F0; f = 2 + hh / F1; int q = hh % F1; u = q % g.bx; v = q / g.bx; }
    else { int hh = h - 2 * (F0 + F1); f = 4 + hh / F2; int q = hh % F2; u = q % g.bx; v = q / g.bx; }
    if (!((face_mask >> f) & 1)) continue;
    int dx, dy, dz, sx, sy, sz;   // destination (padded coords) and source local coords
    switch (f) {
      case 0: dx = -1; dy = u; dz = v; sx = g.bx - 1; sy = u; sz = v; break;
      case 1: dx = g.bx; dy = u; dz = v; sx = 0; sy = u; sz = v; break;
      case 2: dx = u; dy = -1; dz = v; sx = u; sy = g.by - 1; sz = v; break;
      case 3: dx = u; dy = g.by; dz = v; sx = u; sy = 0; sz = v; break;
      case 4: dx = u; dy = v; dz = -1; sx = u; sy = v; sz = g.bz - 1; break;
      default: dx = u; dy = v; dz = g.bz; sx = u; sy = v; sz = 0; break;
    }
    Dst val = (Dst)0;
    if (s.e < 0 || !s.valid) { /* element past the end: leave */ }
    else {
      int ne = nbr[s.e * 6 + f];
      if (ne >= 0) val = (Dst)X[(int64_t)ne * g.nb + sx + g.bx * (sy + g.by * sz)];
    }
    tile[pad(g, dx, dy, dz)] = val;
  }
}

// T tiles: interior of all three components plus the -d face halo of component d
// (the coefficient of the face between the element and its -d neighbour).
template <typename Src, typename Dst>
__device__ void load_T_tiles(Dst* t0, Dst* t1, Dst* t2, const Src* T, int64_t n, const Slot& s, const Geo& g,
                             const int* nbr) {
  load_tile(t0, T, s, g, nbr, 1 << 0);
  load_tile(t1, T + n, s, g, nbr, 1 << 2);
  load_tile(t2, T + 2 * n, s, g, nbr, 1 << 4);
}

// (A u)_c from padded tiles: sum over the six faces of T_f (u_c - u_nb).
template <typename V>
__device__ __forceinline__ V apply_A_cell(const V* ut, const V* t0, const V* t1, const V* t2, const Geo& g,
                                          int lx, int ly, int lz) {
  const int c = pad(g, lx, ly, lz);
  const int sy = g.bx + 2, sz = (g.bx + 2) * (g.by + 2);
  const V uc = ut[c];
  V acc = t0[c] * (uc - ut[c + 1]) + t0[c - 1] * (uc - ut[c - 1]);
  acc += t1[c] * (uc - ut[c + sy]) + t1[c - sy] * (uc - ut[c - sy]);
  acc += t2[c] * (uc - ut[c + sz]) + t2[c - sz] * (uc - ut[c - sz]);
  return acc;
}

// ============================================================== set-up kernels

// K1: face coefficients (harmonic average of kappa^d / h_d^2, Fig. (kappa edge))
// and Tr K~, written block-major.  flags[0] <- 1 on non-positive / non-finite kappa.
template <typename KT>
__global__ void k_faces(const KT* __restrict__ kappa, int comps, int nx, int ny, int nz, double ihx2, double ihy2,
                        double ihz2, Geo g, int64_t m, const int* __restrict__ lex_of_hid, int gx, int gy,
                        double* __restrict__ T, double* __restrict__ S, int* flags, double* tstats) {
  const int64_t n = (int64_t)nx * ny * nz;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double tmax = 0.0, tinv = 0.0;                  // largest face coefficient, largest 1 / coefficient
  if (i < n) {
  const int64_t e = i / g.nb;
  const int p = (int)(i % g.nb);
  const int lex = lex_of_hid[e];
  const int ex = lex % gx, ey = (lex / gx) % gy, ez = lex / (gx * gy);
  const int lx = p % g.bx, ly = (p / g.bx) % g.by, lz = p / (g.bx * g.by);
  const int ci = ex * g.bx + lx, cj = ey * g.by + ly, ck = ez * g.bz + lz;
  const int64_t c = ci + (int64_t)nx * (cj + (int64_t)ny * ck);
  const double ih[3] = {ihx2, ihy2, ihz2};
  const int64_t stride[3] = {1, nx, (int64_t)nx * ny};
  const bool has[3] = {ci + 1 < nx, cj + 1 < ny, ck + 1 < nz};
  double s = 0.0;
  bool bad = false;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int64_t comp = comps == 3 ? d : 0;
    const double kc = (double)kappa[comp * n + c];
    bad |= !(kc > 0.0) || !isfinite(kc);
    const double a = kc * ih[d];
    s += a;
    double t = 0.0;
    if (has[d]) {
      const double kn = (double)kappa[comp * n + c + stride[d]];
      const double b = kn * ih[d];
      t = (kn > 0.0 && isfinite(kn) && a > 0.0) ? 2.0 / (1.0 / a + 1.0 / b) : 0.0;
    }
    T[d * n + i] = t;
    if (t > 0.0) {
      tmax = fmax(tmax, t);
      tinv = fmax(tinv, 1.0 / t);
    }
  }
  S[i] = s;
  if (bad) atomicExch(&flags[0], 1);
  }
  // face-coefficient contrast of the field: one atomic per warp
  for (int o = 16; o > 0; o >>= 1) {
    tmax = fmax(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
    tinv = fmax(tinv, __shfl_xor_sync(0xffffffffu, tinv, o));
  }
  if ((threadIdx.x & 31) == 0 && tmax > 0.0) {
    atomic_max_pos(&tstats[0], tmax);
    atomic_max_pos(&tstats[1], tinv);
  }
}

// IC(0) pivots of each element's diagonal block of the global A:
// d_c = a_cc - sum_{j < c, j ~ c in element} T^2 / d_j, a_cc = sum of the six face
// coefficients.  Writes 1/d.  flags[1] <- 1 on a non-positive pivot.
__global__ void k_pivots(const double* __restrict__ T, int64_t n, Geo g, int64_t m, const int* __restrict__ nbr,
                         const double* __restrict__ Wd, double* __restrict__ invd, double* __restrict__ D, int* flags) {
  extern __shared__ double smem[];
  const Slot s = make_slot(g, m, blockIdx.x);
  double* t0 = smem + (size_t)s.eloc * (3 * g.P + g.nb);
  double* t1 = t0 + g.P;
  double* t2 = t1 + g.P;
  double* d = t2 + g.P;
  if (s.eloc < g.epc) load_T_tiles(t0, t1, t2, T, n, s, g, nbr);
  __syncthreads();
  const int c = pad(g, s.lx, s.ly, s.lz);
  const int sy = g.bx + 2, sz = (g.bx + 2) * (g.by + 2);
  double diag = 0.0;
  if (s.valid) diag = t0[c] + t0[c - 1] + t1[c] + t1[c - sy] + t2[c] + t2[c - sz];
  if (s.valid && Wd) diag += Wd[s.e * g.nb + s.p];   // cell term (wells)
  const int smax = g.bx + g.by + g.bz - 3;
  const int sc = s.lx + s.ly + s.lz;
  for (int w = 0; w <= smax; ++w) {
    if (s.valid && sc == w) {
      double v = diag;
      if (s.lx > 0) v -= t0[c - 1] * t0[c - 1] / d[s.p - 1];
      if (s.ly > 0) v -= t1[c - sy] * t1[c - sy] / d[s.p - g.bx];
      if (s.lz > 0) v -= t2[c - sz] * t2[c - sz] / d[s.p - g.bx * g.by];
      d[s.p] = v;
      if (!(v > 0.0)) atomicExch(&flags[1], 1);
    }
    __syncthreads();
  }
  if (s.valid) {
    invd[s.e * g.nb + s.p] = 1.0 / d[s.p];
    D[s.e * g.nb + s.p] = diag;
  }
}

// natural <-> block-major permutations
__device__ __forceinline__ int64_t nat_index(int64_t i, const Geo& g, const int* lex_of_hid, int gx, int gy, int nx,
                                             int ny) {
  const int64_t e = i / g.nb;
  const int p = (int)(i % g.nb);
  const int lex = lex_of_hid[e];
  const int ex = lex % gx, ey = (lex / gx) % gy, ez = lex / (gx * gy);
  const int lx = p % g.bx, ly = (p / g.bx) % g.by, lz = p / (g.bx * g.by);
  return (int64_t)(ex * g.bx + lx) + (int64_t)nx * ((ey * g.by + ly) + (int64_t)ny * (ez * g.bz + lz));
}

template <bool ToBlk, typename Tin, typename Tout>
__global__ void k_perm(const Tin* __restrict__ in, Tout* __restrict__ out, int64_t n, Geo g,
                       const int* __restrict__ lex_of_hid, int gx, int gy, int nx, int ny, int comps) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t j = nat_index(i, g, lex_of_hid, gx, gy, nx, ny);
  for (int c = 0; c < comps; ++c) {
    if (ToBlk) out[c * n + i] = (Tout)in[c * n + j];
    else out[c * n + j] = (Tout)in[c * n + i];
  }
}

// ============================================================== stencil

// q = A p (FP64) for R right-hand sides stored n apart.  With Reduce, also p.q
// and the PCG step length (finaliser).
template <bool Reduce>
__global__ void k_matvec(const double* __restrict__ p, double* __restrict__ q, const double* __restrict__ T, int64_t n,
                         Geo g, int64_t m, const int* __restrict__ nbr, const double* __restrict__ Wd, RedSlot red,
                         PcgScalars* sc, int R) {
  const BatchIdx bi = batch_idx(R);
  if (Reduce) sc += bi.r;
  if (Reduce && sc->done) return;
  p += (int64_t)bi.r * n;
  q += (int64_t)bi.r * n;
  extern __shared__ double smem[];
  const Slot s = make_slot(g, m, bi.blk);
  double* pt = smem + (size_t)s.eloc * 4 * g.P;
  double* t0 = pt + g.P;
  double* t1 = t0 + g.P;
  double* t2 = t1 + g.P;
  if (s.eloc < g.epc) {
    load_tile(pt, p, s, g, nbr, 0x3f);
    load_T_tiles(t0, t1, t2, T, n, s, g, nbr);
  }
  __syncthreads();
  double v[1] = {0.0};
  if (s.valid) {
    double a = apply_A_cell(pt, t0, t1, t2, g, s.lx, s.ly, s.lz);
    if (Wd) a += Wd[s.e * g.nb + s.p] * pt[pad(g, s.lx, s.ly, s.lz)];   // cell term (wells)
    q[s.e * g.nb + s.p] = a;
    v[0] = a * pt[pad(g, s.lx, s.ly, s.lz)];
  }
  if (Reduce) {
    grid_reduce_r<1>(v, red, bi, [=] __device__(double* t) {
      sc->pq = t[0];
      if (!(t[0] > 0.0) || !isfinite(t[0])) { sc->done = 2; sc->alpha = 0.0; }
      else sc->alpha = sc->rz / t[0];
    });
  }
}

// ============================================================== host launchers

static inline Geo fine_geo(const msmg_ctx* c) { return make_geo(c->fine.bx, c->fine.by, c->fine.bz); }
static inline unsigned fine_grid(const msmg_ctx* c, const Geo& g) { return (unsigned)((c->fine.m + g.epc - 1) / g.epc); }
static inline unsigned fine_threads(const Geo& g) { return (unsigned)(((g.epc * g.nb) + 31) / 32 * 32); }

void launch_faces(msmg_ctx* c, const void* kappa, int comps, int dtype, cudaStream_t s) {
  const Geo g = fine_geo(c);
  const int64_t n = c->n;
  const unsigned grid = (unsigned)((n + 255) / 256);
  const double ihx2 = 1.0 / (c->grid.hx * c->grid.hx), ihy2 = 1.0 / (c->grid.hy * c->grid.hy),
               ihz2 = 1.0 / (c->grid.hz * c->grid.hz);
  if (dtype == MSMG_F32)
    k_faces<float><<<grid, 256, 0, s>>>((const float*)kappa, comps, c->grid.nx, c->grid.ny, c->grid.nz, ihx2, ihy2,
                                        ihz2, g, c->fine.m, c->fine.lex_of_hid, c->fine.gx, c->fine.gy, c->fine.T,
                                        c->fine.S, c->flags, c->dtmp + 2);
  else
    k_faces<double><<<grid, 256, 0, s>>>((const double*)kappa, comps, c->grid.nx, c->grid.ny, c->grid.nz, ihx2, ihy2,
                                         ihz2, g, c->fine.m, c->fine.lex_of_hid, c->fine.gx, c->fine.gy, c->fine.T,
                                         c->fine.S, c->flags, c->dtmp + 2);
}

void launch_pivots(msmg_ctx* c, cudaStream_t s) {
  const Geo g = fine_geo(c);
  const size_t sm = (size_t)g.epc * (3 * g.P + g.nb) * sizeof(double);
  cudaFuncSetAttribute(k_pivots, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_pivots<<<fine_grid(c, g), fine_threads(g), sm, s>>>(c->fine.T, c->n, g, c->fine.m, c->fine.nbr, c->fine.Wd,
                                                         c->fine.invd, c->fine.D, c->flags);
}

void launch_nat_to_blk(msmg_ctx* c, const double* in, double* out, cudaStream_t s) {
  const Geo g = fine_geo(c);
  k_perm<true, double, double><<<(unsigned)((c->n + 255) / 256), 256, 0, s>>>(
      in, out, c->n, g, c->fine.lex_of_hid, c->fine.gx, c->fine.gy, c->grid.nx, c->grid.ny, 1);
}

void launch_blk_to_nat(msmg_ctx* c, const double* in, double* out, cudaStream_t s) {
  const Geo g = fine_geo(c);
  k_perm<false, double, double><<<(unsigned)((c->n + 255) / 256), 256, 0, s>>>(
      in, out, c->n, g, c->fine.lex_of_hid, c->fine.gx, c->fine.gy, c->grid.nx, c->grid.ny, 1);
}

void launch_faces_to_nat(msmg_ctx* c, double* out, cudaStream_t s) {
  const Geo g = fine_geo(c);
  k_perm<false, double, double><<<(unsigned)((c->n + 255) / 256), 256, 0, s>>>(
      c->fine.T, out, c->n, g, c->fine.lex_of_hid, c->fine.gx, c->fine.gy, c->grid.nx, c->grid.ny, 3);
}

void launch_matvec(msmg_ctx* c, const double* p, double* q, cudaStream_t s, int R) {
  const Geo g = fine_geo(c);
  const size_t sm = (size_t)g.epc * 4 * g.P * sizeof(double);
  cudaFuncSetAttribute(k_matvec<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_matvec<false><<<fine_grid(c, g) * R, fine_threads(g), sm, s>>>(p, q, c->fine.T, c->n, g, c->fine.m, c->fine.nbr,
                                                                    c->fine.Wd, c->red, nullptr, R);
}

// The cell term W (wells) in block-major order; a negative or non-finite value
// raises the same flag as a bad permeability.
__global__ void k_check_nonneg(const double* __restrict__ w, int64_t n, int* flags) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !(w[i] >= 0.0 && w[i] < INFINITY)) atomicExch(&flags[0], 1);
}
void launch_cell_diag(msmg_ctx* c, const double* w_nat, cudaStream_t s) {
  launch_nat_to_blk(c, w_nat, c->fine.Wd, s);
  k_check_nonneg<<<(unsigned)((c->n + 255) / 256), 256, 0, s>>>(c->fine.Wd, c->n, c->flags);
}

// ---- kernel timing (roofline figures)
__global__ void k_fill_pattern(double* __restrict__ v, int64_t n, double phase) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = sin(0.001 * (double)i + phase) + 0.25 * cos(0.0173 * (double)i);
}
__global__ void k_reset_scalars(PcgScalars* scs, int R) {
  if ((int)threadIdx.x >= R) return;
  PcgScalars* sc = scs + threadIdx.x;
  sc->done = 0;
  sc->iter = 1;
  sc->max_iter = 1 << 30;
  sc->tol2 = -1.0;
  sc->pq = 1.0;
  sc->rz = 1.0;
  sc->rz_old = 1.0;
  sc->alpha = 0.0;
  sc->beta = 0.0;
}

void pcg_step_vcycle_timed(msmg_ctx* c, int update, const double* qv, PcgScalars* sc, cudaStream_t s,
                           cudaEvent_t* ev);
void pcg_step_pmatvec(msmg_ctx* c, PcgScalars* sc, cudaStream_t s);
void pcg_step_vcycle(msmg_ctx* c, int update, const double* qv, PcgScalars* sc, cudaStream_t s);

// Per-kernel device times of one PCG iteration's fine-level work (events on s),
// for a batch of R right-hand sides.
int time_kernels(msmg_ctx* c, int R, int reps, double* acc, cudaStream_t s) {
  SolveBuffers& B = c->sb;
  if (R < 1 || R > B.n_rhs) return MSMG_ERR_INVALID_ARG;
  B.R = R;
  const int64_t n = c->n * R;
  const unsigned g1 = (unsigned)((n + 255) / 256);
  k_fill_pattern<<<g1, 256, 0, s>>>(B.r, n, 0.3);
  k_fill_pattern<<<g1, 256, 0, s>>>(B.p0, n, 1.1);
  k_fill_pattern<<<g1, 256, 0, s>>>(B.q, n, 2.0);
  k_fill_pattern<<<g1, 256, 0, s>>>(B.x, n, 0.7);
  B.pcur = B.p0;
  B.pnext = B.p1;
  cudaEvent_t ev[8];
  for (int i = 0; i < 8; ++i) cudaEventCreate(&ev[i]);
  for (int i = 0; i < 7; ++i) acc[i] = 0.0;
  const bool flexible = c->opts.precision == MSMG_MIXED;
  for (int r = 0; r < reps; ++r) {
    k_reset_scalars<<<1, 32 * ((R + 31) / 32), 0, s>>>(B.sc, R);
    pcg_step_vcycle_timed(c, 1, flexible ? B.q : nullptr, B.sc, s, ev);   // ev[0..5]
    k_reset_scalars<<<1, 32 * ((R + 31) / 32), 0, s>>>(B.sc, R);
    cudaEventRecord(ev[6], s);
    pcg_step_pmatvec(c, B.sc, s);
    cudaEventRecord(ev[7], s);
    cudaError_t e = cudaEventSynchronize(ev[7]);
    if (e != cudaSuccess) {
      set_last_cuda_error(e);
      for (int i = 0; i < 8; ++i) cudaEventDestroy(ev[i]);
      return MSMG_ERR_CUDA;
    }
    float ms;
    const int seg[5][2] = {{0, 1}, {1, 2}, {3, 4}, {4, 5}, {2, 3}};
    for (int k = 0; k < 5; ++k) {
      cudaEventElapsedTime(&ms, ev[seg[k][0]], ev[seg[k][1]]);
      acc[k] += ms;
    }
    cudaEventElapsedTime(&ms, ev[6], ev[7]);
    acc[5] += ms;
    cudaEventElapsedTime(&ms, ev[0], ev[5]);
    acc[6] += ms;
  }
  for (int i = 0; i < 7; ++i) acc[i] /= reps;
  for (int i = 0; i < 8; ++i) cudaEventDestroy(ev[i]);
  return 0;
}

// Mean time of one whole PCG iteration (V-cycle and the p / A p kernel),
// reps of them captured in one CUDA graph and launched as a solve launches its
// iterations (kernel by kernel if capture is not possible); the autotuner's
// criterion.  Same scratch contents as time_kernels.
int time_iterations(msmg_ctx* c, int R, int reps, double* ms_out, cudaStream_t s) {
  SolveBuffers& B = c->sb;
  if (R < 1 || R > B.n_rhs || reps < 1) return MSMG_ERR_INVALID_ARG;
  B.R = R;
  const int64_t n = c->n * R;
  const unsigned g1 = (unsigned)((n + 255) / 256);
  k_fill_pattern<<<g1, 256, 0, s>>>(B.r, n, 0.3);
  k_fill_pattern<<<g1, 256, 0, s>>>(B.p0, n, 1.1);
  k_fill_pattern<<<g1, 256, 0, s>>>(B.q, n, 2.0);
  k_fill_pattern<<<g1, 256, 0, s>>>(B.x, n, 0.7);
  B.pcur = B.p0;
  B.pnext = B.p1;
  const bool flexible = c->opts.precision == MSMG_MIXED;
  cudaEvent_t ev[2];
  cudaEventCreate(&ev[0]);
  cudaEventCreate(&ev[1]);
  cudaGraphExec_t ge = nullptr;
  if (!c->cap_stream) cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (c->cap_stream && cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    for (int r = 0; r < reps; ++r) {
      k_reset_scalars<<<1, 32 * ((R + 31) / 32), 0, c->cap_stream>>>(B.sc, R);
      pcg_step_vcycle(c, 1, flexible ? B.q : nullptr, B.sc, c->cap_stream);
      pcg_step_pmatvec(c, B.sc, c->cap_stream);
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(c->cap_stream, &g) == cudaSuccess && g) {
      if (cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) ge = nullptr;
      cudaGraphDestroy(g);
    }
  }
  cudaGetLastError();   // a failed capture leaves the eager path below
  if (ge) {
    cudaGraphLaunch(ge, s);              // warm-up
    cudaEventRecord(ev[0], s);
    cudaGraphLaunch(ge, s);
  } else {
    for (int r = 0; r <= reps; ++r) {    // the first iteration warms up
      if (r == 1) cudaEventRecord(ev[0], s);
      k_reset_scalars<<<1, 32 * ((R + 31) / 32), 0, s>>>(B.sc, R);
      pcg_step_vcycle(c, 1, flexible ? B.q : nullptr, B.sc, s);
      pcg_step_pmatvec(c, B.sc, s);
    }
  }
  cudaEventRecord(ev[1], s);
  const cudaError_t e = cudaEventSynchronize(ev[1]);
  float ms = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, ev[0], ev[1]);
  if (ge) cudaGraphExecDestroy(ge);
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (e != cudaSuccess) {
    set_last_cuda_error(e);
    return MSMG_ERR_CUDA;
  }
  *ms_out = ms / reps;
  return 0;
}

// ---- integer-pipe conversions, element by element (diagnostics)
__global__ void k_check_conversions(const double* __restrict__ in64, const float* __restrict__ in32, int64_t n,
                                    float* __restrict__ out32, double* __restrict__ out64) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out32[i] = f32_of_f64_rn(in64[i]);
  out64[i] = f64_of_f32(in32[i]);
}
int launch_check_conversions(const double* in64, const float* in32, int64_t n, float* out32, double* out64,
                             cudaStream_t s) {
  if (n <= 0) return 0;
  k_check_conversions<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in64, in32, n, out32, out64);
  MSMG_CUDA_TRY(cudaGetLastError());
  return 0;
}

// ---- mixed-precision copies
__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
void launch_mixed_copies(msmg_ctx* c, cudaStream_t s) {
  if (c->opts.precision != MSMG_MIXED) return;
  auto cvt = [&](const double* a, float* b, int64_t cnt) {
    if (cnt > 0) k_to_f32<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(a, b, cnt);
  };
  const int64_t n = c->n;
  cvt(c->fine.T, c->fine.T32, 3 * n);
  cvt(c->fine.invd, c->fine.invd32, n);
  if (c->fine.Wd) cvt(c->fine.Wd, c->fine.Wd32, n);
  cvt(c->fine.Phi, c->fine.Phi32, c->fine.m * c->fine.L * c->fine.nb);
}

}  // namespace msmg
