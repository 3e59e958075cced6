// C-ABI entry points of libmsmg (declared in include/msmg.h): validation, the
// workspace plan, set-up orchestration, solves and parity exports.
#include "msmg_internal.cuh"
#include "reduce.cuh"
#include <cstring>
#include <cstdio>
#include <new>

namespace msmg {

static thread_local cudaError_t g_last_cuda = cudaSuccess;
void set_last_cuda_error(cudaError_t e) { g_last_cuda = e; }

void launch_mixed_copies(msmg_ctx* c, cudaStream_t s);
void launch_cell_diag(msmg_ctx* c, const double* w_nat, cudaStream_t s);
void launch_kept_sums(msmg_ctx* c, cudaStream_t s);
void launch_dot(const double* a, const double* b, int64_t n, RedSlot red, double* out, cudaStream_t s);
int launch_level1_chfsi(msmg_ctx* c, cudaStream_t s, const float* guess, float* block);
int net_guesses(msmg_ctx* c, const msmg_net* net, float* x, float* g, cudaStream_t s);
bool net_matches(const msmg_ctx* c, const msmg_net* net);
int launch_coarse_setup_given(msmg_ctx* c, int l, cudaStream_t s);
int time_kernels(msmg_ctx* c, int R, int reps, double* acc, cudaStream_t s);
int time_iterations(msmg_ctx* c, int R, int reps, double* ms_out, cudaStream_t s);
int launch_check_conversions(const double* in64, const float* in32, int64_t n, float* out32, double* out64,
                             cudaStream_t s);
int pcg_solve_batched(msmg_ctx* const* ctxs, int n_ctx, const double* const* rhs, double* const* x,
                      const int* n_rhs, double rtol, int max_iter, int flags, cudaStream_t s,
                      msmg_solve_info* info);
void apply_vcycle_fp64_out(msmg_ctx* c, cudaStream_t s);
void prepare_fine_kernels(msmg_ctx* c);
void prepare_coarse_kernels(msmg_ctx* c);
int coarse_forms(const msmg_ctx* c);

struct LevelShape {
  int g[kMaxLevels + 1][3];    // element grid of E_l, l = 1 .. nL-1
  int64_t m[kMaxLevels + 1];
};

static int shapes(const msmg_grid* gr, const msmg_options* o, LevelShape& sh) {
  const int nL = o->n_levels;
  const int b[3] = {o->block[0], o->block[1], o->block[2]};
  const int nn[3] = {gr->nx, gr->ny, gr->nz};
  for (int d = 0; d < 3; ++d) {
    if (b[d] < 1) return MSMG_ERR_INVALID_ARG;
    if (nn[d] % b[d]) return MSMG_ERR_NOT_DIVISIBLE;
    sh.g[1][d] = nn[d] / b[d];
  }
  sh.m[1] = (int64_t)sh.g[1][0] * sh.g[1][1] * sh.g[1][2];
  for (int l = 2; l <= nL - 1; ++l) {
    for (int d = 0; d < 3; ++d) {
      const int r = o->ratio[l - 2][d];
      if (r < 1) return MSMG_ERR_INVALID_ARG;
      if (sh.g[l - 1][d] % r) return MSMG_ERR_NOT_DIVISIBLE;
      sh.g[l][d] = sh.g[l - 1][d] / r;
    }
    sh.m[l] = (int64_t)sh.g[l][0] * sh.g[l][1] * sh.g[l][2];
  }
  return 0;
}

int validate(const msmg_grid* g, const msmg_options* o) {
  if (!g || !o) return MSMG_ERR_INVALID_ARG;
  if (g->nx < 1 || g->ny < 1 || g->nz < 1) return MSMG_ERR_INVALID_ARG;
  if (!(g->hx > 0) || !(g->hy > 0) || !(g->hz > 0)) return MSMG_ERR_INVALID_ARG;
  if (o->n_levels < 2 || o->n_levels > kMaxLevels) return MSMG_ERR_INVALID_ARG;
  if (o->precision != MSMG_FP64 && o->precision != MSMG_MIXED) return MSMG_ERR_INVALID_ARG;
  if (o->coarse_smoother != MSMG_BLOCK_CHOL && o->coarse_smoother != MSMG_BLOCK_IC0) return MSMG_ERR_INVALID_ARG;
  if (o->two_grid != 0 && o->two_grid != 1) return MSMG_ERR_INVALID_ARG;
  if (o->two_grid && o->n_levels < 3) return MSMG_ERR_INVALID_ARG;   // two levels: the V-cycle is P_TG
  if (!(o->inner_rtol >= 0) || o->inner_max_iter < 0) return MSMG_ERR_INVALID_ARG;
  for (int l = 0; l < o->n_levels - 1; ++l)
    if (!(o->eig_threshold[l] >= 0) || !(o->eig_threshold[l] < 1e300)) return MSMG_ERR_INVALID_ARG;
  LevelShape sh;
  int st = shapes(g, o, sh);
  if (st) return st;
  const int nL = o->n_levels;
  for (int l = 1; l <= nL - 1; ++l)
    if (sh.m[l] < 2) return MSMG_ERR_SINGLE_BLOCK;
  const int nb = o->block[0] * o->block[1] * o->block[2];
  if (nb > 512) return MSMG_ERR_UNSUPPORTED;
  if (o->n_eig[0] < 1 || o->n_eig[0] > nb) return MSMG_ERR_INVALID_ARG;
  if (nb > 96 && o->n_eig[0] >= 16) return MSMG_ERR_UNSUPPORTED;   // subspace solver block limit
  for (int l = 2; l <= nL - 1; ++l) {
    const int nch = o->ratio[l - 2][0] * o->ratio[l - 2][1] * o->ratio[l - 2][2];
    const int nP = nch * o->n_eig[l - 2];
    if (o->n_eig[l - 1] < 1 || o->n_eig[l - 1] > nP) return MSMG_ERR_INVALID_ARG;
    if (nP > 96) return MSMG_ERR_UNSUPPORTED;
  }
  for (int l = 0; l < nL - 1; ++l)
    if (o->nu[l] != 1) return MSMG_ERR_UNSUPPORTED;
  if (o->eig_tol < 0) return MSMG_ERR_INVALID_ARG;
  if (g->nx * (int64_t)g->ny * g->nz > ((int64_t)1 << 31) - 1) return MSMG_ERR_UNSUPPORTED;
  return 0;
}

int plan_and_carve(const msmg_grid* g, const msmg_options* o, int n_rhs, Arena& ar, msmg_ctx* c) {
  LevelShape sh;
  int st = shapes(g, o, sh);
  if (st) return st;
  const int nL = o->n_levels;
  c->grid = *g;
  c->opts = *o;
  if (c->opts.inner_rtol <= 0) c->opts.inner_rtol = 1e-10;
  if (c->opts.inner_max_iter <= 0) c->opts.inner_max_iter = 200;
  c->nL = nL;
  c->n = (int64_t)g->nx * g->ny * g->nz;
  c->max_rhs = n_rhs < 1 ? 1 : n_rhs;
  const bool mixed = o->precision == MSMG_MIXED;
  FineLevel& f = c->fine;
  f.bx = o->block[0]; f.by = o->block[1]; f.bz = o->block[2];
  f.nb = f.bx * f.by * f.bz;
  f.gx = sh.g[1][0]; f.gy = sh.g[1][1]; f.gz = sh.g[1][2];
  f.m = sh.m[1];
  f.n = c->n;
  f.L = o->n_eig[0];
  f.nu = o->nu[0];
  for (int l = 2; l <= nL; ++l) {
    CoarseLevel& lv = c->lev[l];
    lv = CoarseLevel{};
    lv.l = l;
    lv.gx = sh.g[l - 1][0]; lv.gy = sh.g[l - 1][1]; lv.gz = sh.g[l - 1][2];
    lv.me = sh.m[l - 1];
    lv.L = o->n_eig[l - 2];
    lv.n = lv.me * lv.L;
    if (l < nL) {
      lv.nu = o->nu[l - 1];
      lv.rx = o->ratio[l - 2][0]; lv.ry = o->ratio[l - 2][1]; lv.rz = o->ratio[l - 2][2];
      lv.nchild = lv.rx * lv.ry * lv.rz;
      lv.mP = sh.m[l];
      lv.nP = lv.nchild * lv.L;
      lv.Lnext = o->n_eig[l - 1];
    }
  }
  const int64_t n = c->n;
  const int64_t nc = c->lev[nL].n;
  // common
  c->flags = ar.take<int>(16);
  c->kept = ar.take<unsigned long long>(kMaxLevels + 1);
  c->dtmp = ar.take<double>(16 + nc * nc + (4 * kGjBlock + 1) * nc + kGjBlock * kGjBlock + 64);
  // every reducing kernel launches at most one CTA per element and right-hand
  // side, or 1216 CTAs per right-hand side for the grid-stride vector kernels
  int64_t maxgrid = f.m;
  if (maxgrid < 152 * 8) maxgrid = 152 * 8;
  const int R = c->max_rhs;
  c->red.stride = maxgrid * kRedWidth;
  c->red.partials = ar.take<double>((size_t)c->red.stride * R);
  c->red.counter = ar.take<unsigned>(R);
  // fine level
  f.lex_of_hid = ar.take<int>(f.m);
  f.nbr = ar.take<int>(f.m * 6);
  f.T = ar.take<double>(3 * n);
  f.S = ar.take<double>(n);
  f.invd = ar.take<double>(n);
  f.D = ar.take<double>(n);
  f.Phi = ar.take<double>(f.m * f.L * f.nb);
  f.lam = ar.take<double>(f.m * f.L);
  if (mixed) {
    f.T32 = ar.take<float>(3 * n);
    f.invd32 = ar.take<float>(n);
    f.Phi32 = ar.take<float>(f.m * f.L * f.nb);
  }
  if (o->cell_diag) {
    f.Wd = ar.take<double>(n);
    if (mixed) f.Wd32 = ar.take<float>(n);
  }
  for (int l = 2; l <= nL; ++l) {
    CoarseLevel& lv = c->lev[l];
    const int64_t L2 = (int64_t)lv.L * lv.L;
    lv.lex_of_hid = ar.take<int>(lv.me);
    lv.nbr = ar.take<int>(lv.me * 6);
    lv.Ad = ar.take<double>(lv.me * L2);
    lv.Ao = ar.take<double>(lv.me * 3 * L2);
    lv.F = ar.take<double>(lv.me * 6 * L2);
    lv.z = ar.take<double>(lv.n);
    lv.cnt = ar.take<int>(lv.me);
    if (l < nL) {
      lv.Minv = ar.take<double>(lv.mP * lv.nP * lv.nP);
      lv.Psi = ar.take<double>(lv.mP * lv.Lnext * lv.nP);
      lv.lamP = ar.take<double>(lv.mP * lv.Lnext);
    } else {
      lv.pinv = ar.take<double>(lv.n * lv.n);
      lv.nk = lv.n;
      c->cmaps = ar.take<int>(2 * lv.n);   // launch_coarsest points cmap / cinv here when it packs
    }
  }
  // solve buffers
  // solve buffers: R copies of every vector, right-hand side r at offset r * n
  SolveBuffers& B = c->sb;
  const int64_t nR = n * R;
  B.b = ar.take<double>(nR);
  B.x = ar.take<double>(nR);
  B.r = ar.take<double>(nR);
  B.z = ar.take<double>(nR);
  B.p0 = ar.take<double>(nR);
  B.p1 = ar.take<double>(nR);
  B.q = ar.take<double>(nR);
  B.vu[1] = mixed ? (void*)ar.take<float>(nR) : (void*)ar.take<double>(nR);
  B.rv = mixed ? (void*)ar.take<float>(nR) : (void*)ar.take<double>(nR);
  for (int l = 2; l <= nL; ++l) {
    B.vf[l] = ar.take<double>(c->lev[l].n * R);
    B.vu[l] = ar.take<double>(c->lev[l].n * R);
    B.vw[l] = ar.take<double>(c->lev[l].n * R);
  }
  B.ec32 = mixed ? ar.take<float>(c->lev[2].n * R) : nullptr;
  B.sc = ar.take<PcgScalars>(R);
  B.dres = ar.take<double>(2 * R);
  B.dmask = ar.take<int>(R);
  if (o->two_grid) {
    const int64_t n2 = c->lev[2].n * R;
    B.ix = ar.take<double>(n2);
    B.ip0 = ar.take<double>(n2);
    B.ip1 = ar.take<double>(n2);
    B.iq = ar.take<double>(n2);
    B.ipart = ar.take<double>((size_t)1024 * R * 2);
    B.iiters = ar.take<int>(R);
  }
  B.n_rhs = R;
  B.R = 1;
  return 0;
}

// Hierarchical numbering of the element levels (see msmg_internal.cuh) and
// face-neighbour tables, built on the host.
static void build_tables(const msmg_ctx* c, const LevelShape& sh, std::vector<std::vector<int>>& lex_of_hid,
                         std::vector<std::vector<int>>& nbr) {
  const int nL = c->nL;
  std::vector<std::vector<int>> hid_of_lex(nL + 1);
  lex_of_hid.assign(nL + 1, {});
  nbr.assign(nL + 1, {});
  for (int l = nL - 1; l >= 1; --l) {
    const int gx = sh.g[l][0], gy = sh.g[l][1], gz = sh.g[l][2];
    const int64_t m = sh.m[l];
    hid_of_lex[l].resize(m);
    lex_of_hid[l].resize(m);
    for (int64_t lx = 0; lx < m; ++lx) {
      const int ex = (int)(lx % gx), ey = (int)((lx / gx) % gy), ez = (int)(lx / ((int64_t)gx * gy));
      int64_t hid;
      if (l == nL - 1) hid = lx;
      else {
        const int rx = c->opts.ratio[l - 1][0], ry = c->opts.ratio[l - 1][1], rz = c->opts.ratio[l - 1][2];
        const int px = ex / rx, py = ey / ry, pz = ez / rz;
        const int64_t plex = px + (int64_t)sh.g[l + 1][0] * (py + (int64_t)sh.g[l + 1][1] * pz);
        const int local = (ex % rx) + rx * ((ey % ry) + ry * (ez % rz));
        hid = (int64_t)hid_of_lex[l + 1][plex] * (rx * ry * rz) + local;
      }
      hid_of_lex[l][lx] = (int)hid;
      lex_of_hid[l][hid] = (int)lx;
    }
    nbr[l].resize(m * 6);
    for (int64_t lx = 0; lx < m; ++lx) {
      const int ex = (int)(lx % gx), ey = (int)((lx / gx) % gy), ez = (int)(lx / ((int64_t)gx * gy));
      const int64_t h = hid_of_lex[l][lx];
      const int cc[3] = {ex, ey, ez}, gg[3] = {gx, gy, gz};
      const int64_t st[3] = {1, gx, (int64_t)gx * gy};
      for (int d = 0; d < 3; ++d) {
        nbr[l][h * 6 + 2 * d] = cc[d] > 0 ? hid_of_lex[l][lx - st[d]] : -1;
        nbr[l][h * 6 + 2 * d + 1] = cc[d] + 1 < gg[d] ? hid_of_lex[l][lx + st[d]] : -1;
      }
    }
  }
}

static int check_flags(msmg_ctx* c, cudaStream_t s) {
  int h[8];
  double d[9];   // [0] eig residual max, [1] factorisation failure, [2] max T, [3] max 1/T,
                 // [8] a coarse IC(0) factor fell back to the exact block
  MSMG_CUDA_TRY(cudaMemcpyAsync(h, c->flags, sizeof(h), cudaMemcpyDeviceToHost, s));
  MSMG_CUDA_TRY(cudaMemcpyAsync(d, c->dtmp, sizeof(d), cudaMemcpyDeviceToHost, s));
  MSMG_CUDA_TRY(cudaStreamSynchronize(s));
  MSMG_CUDA_TRY(cudaGetLastError());
  if (h[0]) return MSMG_ERR_BAD_KAPPA;
  if (h[1] || d[1] != 0.0) return MSMG_ERR_NOT_FACTORIZABLE;
  {
    unsigned long long k[kMaxLevels + 1] = {};
    launch_kept_sums(c, s);
    MSMG_CUDA_TRY(cudaMemcpyAsync(k, c->kept, sizeof(k), cudaMemcpyDeviceToHost, s));
    MSMG_CUDA_TRY(cudaStreamSynchronize(s));
    c->info.dims_kept[0] = c->n;
    for (int l = 2; l <= c->nL; ++l) c->info.dims_kept[l - 1] = (int64_t)k[l];
  }
  c->info.eig_residual_max = d[0];
  c->info.face_contrast = d[2] * d[3];
  c->info.eig_iterations_max = h[3];
  c->info.eig_iterations_total = h[4];
  if (h[2]) return MSMG_ERR_EIG_NOT_CONVERGED;
  if (d[8] != 0.0) return MSMG_COARSE_IC_FALLBACK;
  return 0;
}

// Autotuner: time each result-preserving variant of the V-cycle at batch width R
// (CUDA events over reps repetitions on the context's own buffers) and keep the
// fastest for that width class.  Variants give the same bits, so the choice
// moves only the time.  Clobbers the solve buffers (call between solves).
static int autotune(msmg_ctx* c, int R, int reps, cudaStream_t s) {
  const int cls = R > 1 ? 1 : 0;
  int bf = c->tune_fused[cls], bt = c->tune_tail[cls];
  const int forms = coarse_forms(c);
  // every variant timed in three interleaved rounds, the best round kept: the
  // variants differ by a few percent, about what one short timing varies by
  double t[4][2];
  for (int tail = 0; tail < 4; ++tail)
    for (int v = 0; v < 2; ++v) t[tail][v] = 1e300;
  for (int round = 0; round < 3; ++round)
    for (int tail = 0; tail < 4; ++tail)
      for (int v = 0; v < 2; ++v) {
        if (!((forms >> tail) & 1)) continue;
        c->tune_fused[cls] = v;
        c->tune_tail[cls] = tail;
        double ms = 0.0;
        int st = time_iterations(c, R, reps, &ms, s);
        if (st) return st;
        if (ms < t[tail][v]) t[tail][v] = ms;
      }
  double best = 1e300;
  for (int tail = 0; tail < 4; ++tail)
    for (int v = 0; v < 2; ++v)
      if (((forms >> tail) & 1) && t[tail][v] < best) { best = t[tail][v]; bf = v; bt = tail; }
  c->tune_fused[cls] = bf;
  c->tune_tail[cls] = bt;
  c->tuned[cls] = 1;
  // a captured iteration graph holds the previous variant
  if (c->graph_state == 1) {
    cudaGraphExecDestroy(c->iter_graph);
    c->graph_state = 0;
  }
  return 0;
}

// Everything that depends on the bases: Galerkin operators, coarse smoothers,
// coarsest pseudo-inverse, reduced-precision copies.
static int build_from_bases(msmg_ctx* c, bool given, cudaStream_t s) {
  launch_level1_galerkin(c, s, !given);
  for (int l = 2; l <= c->nL - 1; ++l) {
    int st = given ? launch_coarse_setup_given(c, l, s) : launch_coarse_setup(c, l, s);
    if (st) return st;
  }
  int st = launch_coarsest(c, s);
  if (st) return st;
  launch_mixed_copies(c, s);
  prepare_fine_kernels(c);
  prepare_coarse_kernels(c);
  if (c->opts.two_grid && !c->inner_grid) return MSMG_ERR_UNSUPPORTED;   // needs the cooperative form
  return 0;
}

}  // namespace msmg

using namespace msmg;

extern "C" {

int msmg_workspace_size(const msmg_grid* grid, const msmg_options* opts, int n_rhs, size_t* bytes) {
  int st = validate(grid, opts);
  if (st) return st;
  if (!bytes) return MSMG_ERR_INVALID_ARG;
  msmg_ctx tmp{};
  Arena ar;
  st = plan_and_carve(grid, opts, n_rhs, ar, &tmp);
  if (st) return st;
  *bytes = ar.off + 256;
  return 0;
}

int msmg_setup(const msmg_grid* grid, const void* kappa, int kappa_components, int kappa_dtype,
               const msmg_options* opts, void* workspace, size_t workspace_bytes, msmg_stream stream,
               msmg_ctx** out) {
  if (!out || !kappa || !workspace) return MSMG_ERR_INVALID_ARG;
  *out = nullptr;
  int st = validate(grid, opts);
  if (st) return st;
  if (kappa_components != 1 && kappa_components != 3) return MSMG_ERR_INVALID_ARG;
  if (kappa_dtype != MSMG_F64 && kappa_dtype != MSMG_F32) return MSMG_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return MSMG_ERR_WORKSPACE;
  size_t need = 0;
  msmg_workspace_size(grid, opts, 1, &need);
  if (workspace_bytes < need) return MSMG_ERR_WORKSPACE;
  msmg_ctx* c = new (std::nothrow) msmg_ctx{};
  if (!c) return MSMG_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Arena ar;
  ar.base = static_cast<char*>(workspace);
  ar.cap = workspace_bytes;
  // the largest batch width that fits (the workspace grows linearly with it)
  int n_rhs = 1;
  {
    size_t b1 = 0, b2 = 0;
    msmg_workspace_size(grid, opts, 1, &b1);
    msmg_workspace_size(grid, opts, 2, &b2);
    const size_t per = b2 > b1 ? b2 - b1 : 1;
    size_t k = 1 + (workspace_bytes - b1) / per;
    if (k > MSMG_MAX_BATCH_RHS) k = MSMG_MAX_BATCH_RHS;
    n_rhs = (int)k;
    for (;;) {
      size_t b = 0;
      msmg_workspace_size(grid, opts, n_rhs, &b);
      if (b <= workspace_bytes || n_rhs == 1) break;
      --n_rhs;
    }
  }
  plan_and_carve(grid, opts, n_rhs, ar, c);
  c->ws_bytes = workspace_bytes;
  cudaGetDevice(&c->device);
  cudaEventCreate(&c->ev0);
  cudaEventCreate(&c->ev1);
  // untuned defaults: separate prolongation for single solves, fused for batches
  c->tune_fused[0] = 0;
  c->tune_fused[1] = 1;
  c->tune_tail[0] = c->tune_tail[1] = 2;   // the fused coarse cycle, where the hierarchy allows it
  for (int k = 0; k < 3; ++k) cudaEventCreateWithFlags(&c->poll_evs[k], cudaEventDisableTiming);
  *out = c;
  // pinned host mirrors of the PCG scalars (latest + two in-flight chunks),
  // residual norms and restart mask
  MSMG_CUDA_TRY(cudaMallocHost(&c->hsc, (size_t)3 * n_rhs * sizeof(PcgScalars)));
  MSMG_CUDA_TRY(cudaMallocHost(&c->hres, (size_t)2 * n_rhs * sizeof(double)));
  MSMG_CUDA_TRY(cudaMallocHost(&c->hmask, (size_t)(n_rhs + 2) * sizeof(int)));
  c->hmask[n_rhs] = c->hmask[n_rhs + 1] = 0;
  cudaEventRecord(c->ev0, s);
  LevelShape sh;
  shapes(grid, opts, sh);
  std::vector<std::vector<int>> lex, nbr;
  build_tables(c, sh, lex, nbr);
  MSMG_CUDA_TRY(cudaMemcpyAsync(c->fine.lex_of_hid, lex[1].data(), lex[1].size() * sizeof(int),
                                cudaMemcpyHostToDevice, s));
  MSMG_CUDA_TRY(cudaMemcpyAsync(c->fine.nbr, nbr[1].data(), nbr[1].size() * sizeof(int), cudaMemcpyHostToDevice, s));
  for (int l = 2; l <= c->nL; ++l) {
    MSMG_CUDA_TRY(cudaMemcpyAsync(c->lev[l].lex_of_hid, lex[l - 1].data(), lex[l - 1].size() * sizeof(int),
                                  cudaMemcpyHostToDevice, s));
    MSMG_CUDA_TRY(cudaMemcpyAsync(c->lev[l].nbr, nbr[l - 1].data(), nbr[l - 1].size() * sizeof(int),
                                  cudaMemcpyHostToDevice, s));
  }
  MSMG_CUDA_TRY(cudaStreamSynchronize(s));   // host tables go out of scope
  MSMG_CUDA_TRY(cudaMemsetAsync(c->flags, 0, 16 * sizeof(int), s));
  MSMG_CUDA_TRY(cudaMemsetAsync(c->dtmp, 0, 16 * sizeof(double), s));
  MSMG_CUDA_TRY(cudaMemsetAsync(c->red.counter, 0, (size_t)c->max_rhs * sizeof(unsigned), s));
  launch_faces(c, kappa, kappa_components, kappa_dtype, s);
  if (opts->cell_diag) launch_cell_diag(c, opts->cell_diag, s);
  {
    // stop before any eigensolve when the permeability is not positive and finite
    int h0 = 0;
    MSMG_CUDA_TRY(cudaMemcpyAsync(&h0, c->flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    MSMG_CUDA_TRY(cudaStreamSynchronize(s));
    if (h0) return MSMG_ERR_BAD_KAPPA;
  }
  launch_pivots(c, s);
  cudaEvent_t e_eig0, e_eig1;
  cudaEventCreate(&e_eig0);
  cudaEventCreate(&e_eig1);
  cudaEventRecord(e_eig0, s);
  // Dense Jacobi (all eigenpairs) for elements of at most 64 cells; above that the
  // filtered subspace iteration for the L wanted pairs (80-cell elements of the
  // IMPES workload: 731 -> 49 ms for 13,750 elements), Jacobi again up to 96 cells
  // where the subspace solver's block limits do not fit.
  bool dense = c->fine.nb <= 64;
  if (!dense && c->fine.nb <= 96) {
    const int L = c->fine.L, guard = L / 2 > 4 ? L / 2 : 4;
    const int K = L + guard < c->fine.nb ? L + guard : c->fine.nb;
    const int cx = c->fine.bx < 4 ? c->fine.bx : 4, cy = c->fine.by < 4 ? c->fine.by : 4,
              cz = c->fine.bz < 4 ? c->fine.bz : 4;
    dense = L >= 16 || (K < 16 ? K : 16) > cx * cy * cz;
  }
  if (dense) {
    st = launch_level1_eigen(c, s);
  } else {
    // Scratch in buffers that are still unused: the solve buffers span at
    // least 56 n bytes (64 n in the mixed form), Phi 8 L n bytes.
    //   FP64 form   features, then the learned guesses, in the solve buffers
    //   mixed form  features, then the FP32 block handed from the first phase
    //               to the second (4 K n <= 64 n bytes), in the solve buffers;
    //               the guesses in Phi, which only the second phase writes
    const bool mixed = c->opts.precision == MSMG_MIXED;
    float* span = reinterpret_cast<float*>(c->sb.b);
    const float* guess = nullptr;
    const msmg_net* net = opts->warm_start;
    if (net && net_matches(c, net) && (mixed || (size_t)4 * c->fine.L * c->n <= (size_t)56 * c->n)) {
      float* g = mixed ? reinterpret_cast<float*>(c->fine.Phi) : span + c->n;
      st = net_guesses(c, net, span, g, s);
      if (st) return st;
      guess = g;
      c->info.warm_started = 1;
    }
    st = launch_level1_chfsi(c, s, guess, mixed ? span : nullptr);
  }
  cudaEventRecord(e_eig1, s);
  if (st) return st;
  st = build_from_bases(c, false, s);
  if (st) return st;
  cudaEventRecord(c->ev1, s);
  int fl = check_flags(c, s);
  float ms = 0.f, ems = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  cudaEventElapsedTime(&ems, e_eig0, e_eig1);
  cudaEventDestroy(e_eig0);
  cudaEventDestroy(e_eig1);
  msmg_setup_info& I = c->info;
  I.n_levels = c->nL;
  I.dims[0] = c->n;
  for (int l = 2; l <= c->nL; ++l) I.dims[l - 1] = c->lev[l].n;
  for (int l = 1; l <= c->nL - 1; ++l) I.elements[l - 1] = sh.m[l];
  I.setup_ms = ms;
  I.eig_ms = ems;
  I.workspace_bytes = (int64_t)workspace_bytes;
  if (opts->autotune && fl >= 0) {
    int st2 = autotune(c, 1, 6, s);
    if (!st2 && c->max_rhs > 1) st2 = autotune(c, c->max_rhs, 3, s);
    if (st2) return st2;
  }
  for (int k = 0; k < 2; ++k) {
    I.tuning[k] = c->tune_fused[k];
    I.tuning[2 + k] = c->tune_tail[k];
  }
  return fl;
}

int msmg_solve(msmg_ctx* c, const double* rhs, double* x, int n_rhs, double rtol, int max_iter, int flags,
               msmg_stream stream, msmg_solve_info* info) {
  if (!c || !rhs || !x || n_rhs < 1 || max_iter < 0 || !(rtol >= 0)) return MSMG_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (info)
    for (int i = 0; i < n_rhs; ++i) info[i] = msmg_solve_info{};
  const int st = pcg_solve(c, rhs, x, n_rhs, rtol, max_iter, flags, s, info);
  if (st < 0) return st;
  cudaError_t e = cudaGetLastError();   // a NotReady left by an event poll is not an error
  if (e != cudaSuccess && e != cudaErrorNotReady) { set_last_cuda_error(e); return MSMG_ERR_CUDA; }
  return st;
}

int msmg_solve_batched(msmg_ctx* const* ctxs, int n_ctx, const double* const* rhs, double* const* x,
                       const int* n_rhs, double rtol, int max_iter, int flags, msmg_stream stream,
                       msmg_solve_info* info) {
  if (!ctxs || n_ctx < 1 || !rhs || !x || !n_rhs || max_iter < 0 || !(rtol >= 0)) return MSMG_ERR_INVALID_ARG;
  int64_t total = 0;
  for (int k = 0; k < n_ctx; ++k) {
    if (!ctxs[k] || !rhs[k] || !x[k] || n_rhs[k] < 0) return MSMG_ERR_INVALID_ARG;
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) return MSMG_ERR_INVALID_ARG;   // one solve per context at a time
    total += n_rhs[k];
  }
  if (info)
    for (int64_t i = 0; i < total; ++i) info[i] = msmg_solve_info{};
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int st = pcg_solve_batched(ctxs, n_ctx, rhs, x, n_rhs, rtol, max_iter, flags, s, info);
  if (st < 0) return st;
  cudaError_t e = cudaGetLastError();   // a NotReady left by an event poll is not an error
  if (e != cudaSuccess && e != cudaErrorNotReady) { set_last_cuda_error(e); return MSMG_ERR_CUDA; }
  return st;
}

int msmg_max_batch_rhs(const msmg_ctx* c) { return c ? c->max_rhs : 0; }

int msmg_set_tuning(msmg_ctx* c, const int* tuning) {
  if (!c || !tuning) return MSMG_ERR_INVALID_ARG;
  for (int k = 0; k < 2; ++k)
    if (tuning[k] != 0 && tuning[k] != 1) return MSMG_ERR_INVALID_ARG;
  for (int k = 2; k < 4; ++k) {
    if (tuning[k] < 0 || tuning[k] > 3) return MSMG_ERR_INVALID_ARG;
    if (!((coarse_forms(c) >> tuning[k]) & 1)) return MSMG_ERR_UNSUPPORTED;
  }
  for (int k = 0; k < 2; ++k) {
    c->tune_fused[k] = tuning[k];
    c->tune_tail[k] = tuning[2 + k];
  }
  for (int k = 0; k < 4; ++k) c->info.tuning[k] = tuning[k];
  if (c->graph_state == 1) {
    cudaGraphExecDestroy(c->iter_graph);
    c->graph_state = 0;
  }
  return 0;
}

int msmg_autotune(msmg_ctx* c, int n_rhs, int reps, msmg_stream stream) {
  if (!c || n_rhs < 1 || n_rhs > c->max_rhs || reps < 1) return MSMG_ERR_INVALID_ARG;
  const int st = autotune(c, n_rhs, reps, reinterpret_cast<cudaStream_t>(stream));
  for (int k = 0; k < 2; ++k) {
    c->info.tuning[k] = c->tune_fused[k];
    c->info.tuning[2 + k] = c->tune_tail[k];
  }
  return st;
}

int msmg_apply_A(msmg_ctx* c, const double* p, double* q, msmg_stream stream) {
  if (!c || !p || !q) return MSMG_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  c->sb.R = 1;
  launch_nat_to_blk(c, p, c->sb.p0, s);
  launch_matvec(c, c->sb.p0, c->sb.q, s);
  launch_blk_to_nat(c, c->sb.q, q, s);
  MSMG_CUDA_TRY(cudaGetLastError());
  return 0;
}

int msmg_apply_precond(msmg_ctx* c, const double* r, double* z, msmg_stream stream) {
  if (!c || !r || !z) return MSMG_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  c->sb.R = 1;
  MSMG_CUDA_TRY(cudaMemsetAsync(c->flags + 6, 0, sizeof(int), s));
  launch_nat_to_blk(c, r, c->sb.r, s);
  apply_vcycle_fp64_out(c, s);
  launch_blk_to_nat(c, c->sb.z, z, s);
  MSMG_CUDA_TRY(cudaGetLastError());
  // a bounded wait inside the V-cycle that gave up leaves its error word set
  int err = 0;
  MSMG_CUDA_TRY(cudaMemcpyAsync(&err, c->flags + 6, sizeof(int), cudaMemcpyDeviceToHost, s));
  MSMG_CUDA_TRY(cudaStreamSynchronize(s));
  return err ? MSMG_ERR_DEVICE_TIMEOUT : 0;
}

size_t msmg_dot_scratch_bytes(int64_t n) {
  (void)n;
  return (size_t)(152 * 8) * kRedWidth * sizeof(double) + 256;
}

int msmg_dot(const double* a, const double* b, int64_t n, void* scratch, double* result_host, msmg_stream stream) {
  if ((n > 0 && (!a || !b)) || !scratch || !result_host || n < 0) return MSMG_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(scratch) % 16) return MSMG_ERR_WORKSPACE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(scratch);
  RedSlot red;
  red.partials = reinterpret_cast<double*>(base + 256);
  red.counter = reinterpret_cast<unsigned*>(base);
  double* out = reinterpret_cast<double*>(base + 64);
  MSMG_CUDA_TRY(cudaMemsetAsync(base, 0, 256, s));
  launch_dot(a, b, n, red, out, s);
  MSMG_CUDA_TRY(cudaMemcpyAsync(result_host, out, sizeof(double), cudaMemcpyDeviceToHost, s));
  MSMG_CUDA_TRY(cudaStreamSynchronize(s));
  MSMG_CUDA_TRY(cudaGetLastError());
  return 0;
}

int msmg_export_basis(msmg_ctx* c, int level, double* basis, double* lam, msmg_stream stream) {
  if (!c || !basis || level < 1 || level > c->nL - 1) return MSMG_ERR_INVALID_ARG;
  launch_basis_export(c, level, basis, lam, false, reinterpret_cast<cudaStream_t>(stream));
  MSMG_CUDA_TRY(cudaGetLastError());
  return 0;
}

int msmg_import_bases(msmg_ctx* c, const double* const* bases, msmg_stream stream) {
  if (!c || !bases) return MSMG_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (int l = 1; l <= c->nL - 1; ++l) {
    if (!bases[l - 1]) return MSMG_ERR_INVALID_ARG;
    launch_basis_export(c, l, const_cast<double*>(bases[l - 1]), nullptr, true, s);
  }
  MSMG_CUDA_TRY(cudaMemsetAsync(c->dtmp, 0, 16 * sizeof(double), s));
  // level-by-level: each level's operator is needed before the next level's set-up
  launch_level1_galerkin(c, s, false);
  for (int l = 2; l <= c->nL - 1; ++l) {
    int st = launch_coarse_setup_given(c, l, s);
    if (st) return st;
  }
  int st = launch_coarsest(c, s);
  if (st) return st;
  launch_mixed_copies(c, s);
  prepare_fine_kernels(c);
  prepare_coarse_kernels(c);
  if (c->opts.two_grid && !c->inner_grid) return MSMG_ERR_UNSUPPORTED;
  return check_flags(c, s);
}

int msmg_export_operator(msmg_ctx* c, int level, double* out, msmg_stream stream) {
  if (!c || !out || level < 2 || level > c->nL) return MSMG_ERR_INVALID_ARG;
  launch_operator_export(c, level, out, reinterpret_cast<cudaStream_t>(stream));
  MSMG_CUDA_TRY(cudaGetLastError());
  return 0;
}

int msmg_export_faces(msmg_ctx* c, double* T, msmg_stream stream) {
  if (!c || !T) return MSMG_ERR_INVALID_ARG;
  launch_faces_to_nat(c, T, reinterpret_cast<cudaStream_t>(stream));
  MSMG_CUDA_TRY(cudaGetLastError());
  return 0;
}

int msmg_get_setup_info(msmg_ctx* c, msmg_setup_info* info) {
  if (!c || !info) return MSMG_ERR_INVALID_ARG;
  *info = c->info;
  return 0;
}

void msmg_destroy(msmg_ctx* c) {
  if (!c) return;
  if (c->graph_state == 1) cudaGraphExecDestroy(c->iter_graph);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->run_stream) cudaStreamDestroy(c->run_stream);
  cudaEventDestroy(c->ev0);
  cudaEventDestroy(c->ev1);
  for (int k = 0; k < 3; ++k)
    if (c->poll_evs[k]) cudaEventDestroy(c->poll_evs[k]);
  if (c->hsc) cudaFreeHost(c->hsc);
  if (c->hres) cudaFreeHost(c->hres);
  if (c->hmask) cudaFreeHost(c->hmask);
  delete c;
}

int msmg_time_kernels(msmg_ctx* c, int n_rhs, int reps, double* ms_out, int n_out, msmg_stream stream) {
  if (!c || !ms_out || reps < 1 || n_out < 1 || n_rhs < 1 || n_rhs > c->max_rhs) return MSMG_ERR_INVALID_ARG;
  double acc[7];
  int st = time_kernels(c, n_rhs, reps, acc, reinterpret_cast<cudaStream_t>(stream));
  if (st) return st;
  for (int i = 0; i < n_out && i < 7; ++i) ms_out[i] = acc[i];
  return 0;
}

int msmg_check_conversions(const double* in64, const float* in32, int64_t n, float* out32, double* out64,
                           msmg_stream stream) {
  if (n > 0 && (!in64 || !in32 || !out32 || !out64)) return MSMG_ERR_INVALID_ARG;
  return launch_check_conversions(in64, in32, n, out32, out64, reinterpret_cast<cudaStream_t>(stream));
}

const char* msmg_status_string(int s) {
  switch (s) {
    case MSMG_OK: return "ok";
    case MSMG_NOT_CONVERGED: return "not converged within max_iter";
    case MSMG_COARSE_IC_FALLBACK: return "a coarse IC(0) factor broke down; its parent uses the exact block";
    case MSMG_ERR_INVALID_ARG: return "invalid argument";
    case MSMG_ERR_NOT_DIVISIBLE: return "element sizes do not tile the grid";
    case MSMG_ERR_BAD_KAPPA: return "permeability not positive and finite";
    case MSMG_ERR_SINGLE_BLOCK: return "a smoothed level has a single element";
    case MSMG_ERR_BREAKDOWN: return "PCG breakdown (p^T A p <= 0 or non-finite)";
    case MSMG_ERR_EIG_NOT_CONVERGED: return "local eigensolve did not reach eig_tol";
    case MSMG_ERR_WORKSPACE: return "workspace too small or misaligned";
    case MSMG_ERR_CUDA: return cudaGetErrorString(g_last_cuda);
    case MSMG_ERR_NOT_FACTORIZABLE: return "smoother or coarsest factorisation failed";
    case MSMG_ERR_UNSUPPORTED: return "unsupported configuration";
    case MSMG_ERR_DEVICE_TIMEOUT: return "a bounded device-side wait gave up (data never arrived)";
    default: return "unknown status";
  }
}

}  // extern "C"
