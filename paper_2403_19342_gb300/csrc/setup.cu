// Set-up phase kernels (Section 3, Section 5), FP64.
//
//  * Level-1 local spectral problem (Eq. (spepb)) on small elements: the
//    symmetric form A~ = S^{-1/2} A_K S^{-1/2} is diagonalised by a parallel
//    cyclic Jacobi method in shared memory; Phi = S^{-1/2} Y keeps the L
//    smallest eigenvectors, which are then S-orthonormal.
//  * Level-1 Galerkin blocks of A_2 = R_1 A R_1^T: diagonal Phi_a^T A_aa Phi_a,
//    couplings -sum_faces T Phi_a(c) Phi_b(c')^T, and per-face terms
//    Phi_a^T diag(T on the face) Phi_a used to pose the next level's problems.
//  * Level l >= 2, per parent P: the left matrix of Eq. (spectral cc) equals
//    the parent's diagonal block of A_l minus the face terms of its children
//    on P's boundary (the right matrix is I); its smallest eigenvectors Psi_P;
//    the Galerkin blocks of A_{l+1}; the parent's face terms; and the inverse
//    of the parent's diagonal block (the block-Jacobi smoother of level l).
//  * Coarsest level: A_L + sigma z z^T / |z|^2 (z spans null(A_L)) is inverted
//    by Gauss-Jordan elimination and projected, giving the Moore-Penrose
//    inverse A_L^dagger used by Algorithm 1's coarsest correction.
#include "msmg_internal.cuh"
#include "reduce.cuh"
#include "linalg_small.cuh"
#include <cmath>
#include <vector>

namespace msmg {

// ------------------------------------------------------------------ level 1 eigen (dense)
// One CTA per element, nb <= 96.  stats[0] <- max eigen-residual.
__global__ void k_eig_l1_jacobi(const double* __restrict__ T, const double* __restrict__ S, int64_t n, int bx, int by,
                                int bz, int64_t m, int L, double* __restrict__ Phi, double* __restrict__ lam,
                                double* stats, const double* __restrict__ Wd) {
  extern __shared__ double sm[];
  const int nb = bx * by * bz;
  double* A = sm;
  double* V = A + nb * nb;
  double* isq = V + nb * nb;
  double* cs = isq + nb;
  double* red = cs + nb + 2;
  int* pr = reinterpret_cast<int*>(red + 72);
  int* order = pr + nb + 2;
  const int64_t e = blockIdx.x;
  const double* Te = T + e * nb;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) isq[i] = 1.0 / sqrt(S[e * nb + i]);
  for (int i = threadIdx.x; i < nb * nb; i += blockDim.x) A[i] = 0.0;
  __syncthreads();
  // A~ = S^{-1/2} A_K S^{-1/2}: faces inside the element only (Eq. (spepb))
  for (int c = threadIdx.x; c < nb; c += blockDim.x) {
    const int lx = c % bx, ly = (c / bx) % by, lz = c / (bx * by);
    const int lc[3] = {lx, ly, lz}, bd[3] = {bx, by, bz}, st[3] = {1, bx, bx * by};
    double diag = 0.0;
    for (int d = 0; d < 3; ++d) {
      if (lc[d] + 1 < bd[d]) {
        const double t = Te[(int64_t)d * n + c];
        diag += t;
        A[c * nb + c + st[d]] = -t * isq[c] * isq[c + st[d]];
      }
      if (lc[d] > 0) {
        const double t = Te[(int64_t)d * n + c - st[d]];
        diag += t;
        A[c * nb + c - st[d]] = -t * isq[c] * isq[c - st[d]];
      }
    }
    if (Wd) diag += Wd[e * nb + c];   // cell term (wells), added to the left-hand form (Section 6)
    A[c * nb + c] = diag * isq[c] * isq[c];
  }
  __syncthreads();
  jacobi_eig(A, V, nb, cs, pr, red, 40, 1e-15);
  sort_diag(A, nb, order);
  // Phi = S^{-1/2} y for the L smallest; eigen-residual ||A~ y - theta y||
  for (int idx = threadIdx.x; idx < L * nb; idx += blockDim.x) {
    const int k = idx / nb, c = idx % nb;
    const int col = order[k];
    Phi[(e * L + k) * nb + c] = V[c * nb + col] * isq[c];
  }
  for (int k = threadIdx.x; k < L; k += blockDim.x) lam[e * L + k] = A[order[k] * nb + order[k]];
  double res = 0.0;
  for (int k = 0; k < L; ++k) {
    const int col = order[k];
    const double th = A[col * nb + col];
    double v[1] = {0.0};
    // (A~ y)_c from the element's faces (the 7-point stencil), not from a dense copy
    // of A~: two matrices in shared memory instead of three, so two CTAs share an SM
    for (int c = threadIdx.x; c < nb; c += blockDim.x) {
      const int lx = c % bx, ly = (c / bx) % by, lz = c / (bx * by);
      const int lc[3] = {lx, ly, lz}, bd[3] = {bx, by, bz}, st[3] = {1, bx, bx * by};
      double diag = 0.0, off = 0.0;
      for (int d = 0; d < 3; ++d) {
        if (lc[d] + 1 < bd[d]) {
          const double t = Te[(int64_t)d * n + c];
          diag += t;
          off += t * isq[c + st[d]] * V[(c + st[d]) * nb + col];
        }
        if (lc[d] > 0) {
          const double t = Te[(int64_t)d * n + c - st[d]];
          diag += t;
          off += t * isq[c - st[d]] * V[(c - st[d]) * nb + col];
        }
      }
      if (Wd) diag += Wd[e * nb + c];
      const double acc = isq[c] * (diag * isq[c] * V[c * nb + col] - off) - th * V[c * nb + col];
      v[0] += acc * acc;
    }
    block_sum<1>(v, red + 2);
    if (threadIdx.x == 0) res = fmax(res, sqrt(v[0]));
  }
  if (threadIdx.x == 0) atomic_max_pos(&stats[0], res);
}

// ------------------------------------------------------------------ level-1 counts (Strategy 2)
// With a threshold B > 0 (B_c, Section 5) each element keeps its candidates with
// eigenvalue below B, at least one (the candidates come in ascending order), and
// the other slots become zero rows of Phi.  The count is then the number of
// leading nonzero rows (which also reads the counts of imported bases).  One
// warp per element.
__global__ void k_level1_counts(double* __restrict__ Phi, const double* __restrict__ lam, int64_t m, int L, int nb,
                                double B, int* __restrict__ cnt) {
  const int64_t e = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (e >= m) return;
  double* Pe = Phi + e * (int64_t)L * nb;
  if (B > 0.0) {
    int c = 0;
    for (int k = 0; k < L; ++k) c += lam[e * L + k] < B ? 1 : 0;
    if (c < 1) c = 1;
    for (int idx = c * nb + lane; idx < L * nb; idx += 32) Pe[idx] = 0.0;
    __syncwarp();
  }
  int last = 0;
  for (int k = 0; k < L; ++k) {
    bool nz = false;
    for (int i = lane; i < nb; i += 32) nz |= Pe[k * nb + i] != 0.0;
    if (__any_sync(0xffffffffu, nz)) last = k + 1;
  }
  if (lane == 0) cnt[e] = last;
}

__global__ void k_kept_sum(const int* __restrict__ cnt, int64_t m, unsigned long long* out) {
  unsigned long long v = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    v += (unsigned long long)cnt[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, v);
}

// ------------------------------------------------------------------ level 1 Galerkin
// One CTA per element a.  Outputs: Ad[a] = Phi_a^T A_aa Phi_a, Ao[a][d] = A_2[a, a+e_d],
// F[a][f] = Phi_a^T diag(T on face f) Phi_a, z[a] = Phi_a^T S 1.
__global__ void k_galerkin1(const double* __restrict__ T, const double* __restrict__ S, int64_t n, int bx, int by,
                            int bz, int64_t m, const int* __restrict__ nbr, int L, const double* __restrict__ Phi,
                            double* __restrict__ Ad, double* __restrict__ Ao, double* __restrict__ F,
                            double* __restrict__ z, const int* __restrict__ cnt, const double* __restrict__ Wd) {
  extern __shared__ double sm[];
  const int nb = bx * by * bz;
  double* Ph = sm;            // [L][nb]
  double* W = Ph + L * nb;    // [L][nb] = A_aa phi
  double* Tm = W + L * nb;    // [3][nb] coefficient of the -d face of each cell
  const int64_t a = blockIdx.x;
  for (int i = threadIdx.x; i < L * nb; i += blockDim.x) Ph[i] = Phi[a * L * nb + i];
  const int bd[3] = {bx, by, bz}, st[3] = {1, bx, bx * by};
  for (int c = threadIdx.x; c < nb; c += blockDim.x) {
    const int lc[3] = {c % bx, (c / bx) % by, c / (bx * by)};
    for (int d = 0; d < 3; ++d) {
      double t = 0.0;
      if (lc[d] > 0) t = T[(int64_t)d * n + a * nb + c - st[d]];
      else {
        const int nbm = nbr[a * 6 + 2 * d];
        if (nbm >= 0) t = T[(int64_t)d * n + (int64_t)nbm * nb + c + (bd[d] - 1) * st[d]];
      }
      Tm[d * nb + c] = t;
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < nb; c += blockDim.x) {
    const int lc[3] = {c % bx, (c / bx) % by, c / (bx * by)};
    double diag = 0.0;
    for (int d = 0; d < 3; ++d) diag += T[(int64_t)d * n + a * nb + c] + Tm[d * nb + c];
    if (Wd) diag += Wd[a * nb + c];   // cell term (wells)
    for (int k = 0; k < L; ++k) {
      double acc = diag * Ph[k * nb + c];
      for (int d = 0; d < 3; ++d) {
        if (lc[d] + 1 < bd[d]) acc -= T[(int64_t)d * n + a * nb + c] * Ph[k * nb + c + st[d]];
        if (lc[d] > 0) acc -= Tm[d * nb + c] * Ph[k * nb + c - st[d]];
      }
      W[k * nb + c] = acc;
    }
  }
  __syncthreads();
  const int L2 = L * L;
  const int nout = L2 + 6 * L2 + 3 * L2 + L;
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    if (o < L2) {
      const int k = o / L, mm = o % L;
      if (k > mm) continue;
      double acc = 0.0, acc2 = 0.0;
      for (int c = 0; c < nb; ++c) { acc += Ph[k * nb + c] * W[mm * nb + c]; acc2 += Ph[mm * nb + c] * W[k * nb + c]; }
      double v = 0.5 * (acc + acc2);
      if (k == mm && k >= cnt[a]) v = 1.0;   // unused slot (Strategy 2): a decoupled unknown
      Ad[a * L2 + k * L + mm] = v;
      Ad[a * L2 + mm * L + k] = v;
    } else if (o < 7 * L2) {
      const int oo = o - L2;
      const int f = oo / L2, k = (oo % L2) / L, mm = oo % L;
      const int d = f / 2;
      const bool plus = f & 1;
      const int u = (d + 1) % 3, w = (d + 2) % 3;
      double acc = 0.0;
      for (int iu = 0; iu < bd[u]; ++iu)
        for (int iw = 0; iw < bd[w]; ++iw) {
          const int c = (plus ? bd[d] - 1 : 0) * st[d] + iu * st[u] + iw * st[w];
          const double t = plus ? T[(int64_t)d * n + a * nb + c] : Tm[d * nb + c];
          acc += t * Ph[k * nb + c] * Ph[mm * nb + c];
        }
      F[(a * 6 + f) * L2 + k * L + mm] = acc;
    } else if (o < 10 * L2) {
      const int oo = o - 7 * L2;
      const int d = oo / L2, k = (oo % L2) / L, mm = oo % L;
      const int nbp = nbr[a * 6 + 2 * d + 1];
      double acc = 0.0;
      if (nbp >= 0) {
        const int u = (d + 1) % 3, w = (d + 2) % 3;
        const double* Pn = Phi + ((int64_t)nbp * L + mm) * nb;
        for (int iu = 0; iu < bd[u]; ++iu)
          for (int iw = 0; iw < bd[w]; ++iw) {
            const int c = (bd[d] - 1) * st[d] + iu * st[u] + iw * st[w];
            const int c2 = iu * st[u] + iw * st[w];
            acc -= T[(int64_t)d * n + a * nb + c] * Ph[k * nb + c] * Pn[c2];
          }
      }
      Ao[(a * 3 + d) * L2 + k * L + mm] = acc;
    } else {
      const int k = o - 10 * L2;
      double acc = 0.0;
      for (int c = 0; c < nb; ++c) acc += Ph[k * nb + c] * S[a * nb + c];
      z[a * L + k] = acc;
    }
  }
}

// ------------------------------------------------------------------ coarse levels
// Incomplete Cholesky with no fill (Section 5: incomplete Cholesky for the
// coarse smoother) of a parent's diagonal block A (nP x nP, shared memory) into
// the lower factor Lf.  The pattern is structural: A_l is a block 7-point
// stencil, so the block (child a, child b), L x L, is in it when the children
// (lexicographic inside the parent, rx x ry x rz) are equal or share a face.
// Right-looking order: pivot k, column k scaled, then the updates of the
// trailing pattern entries.  Returns false (every thread) on a pivot that is
// not positive.  flag: one shared int of scratch.
__device__ __forceinline__ bool sib_pat(int i, int j, int L, int rx, int ry) {
  const int a = i / L, b = j / L;
  const int ax = a % rx, ay = (a / rx) % ry, az = a / (rx * ry);
  const int bx = b % rx, by = (b / rx) % ry, bz = b / (rx * ry);
  return abs(ax - bx) + abs(ay - by) + abs(az - bz) <= 1;
}
__device__ bool ic0_factor(const double* A, double* Lf, int nP, int L, int rx, int ry, double* flag) {
  for (int idx = threadIdx.x; idx < nP * nP; idx += blockDim.x) {
    const int i = idx / nP, j = idx % nP;
    Lf[idx] = (j <= i && sib_pat(i, j, L, rx, ry)) ? A[idx] : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < nP; ++k) {
    if (threadIdx.x == 0) {
      const double d = Lf[k * nP + k];
      flag[0] = d > 0.0 ? 0.0 : 1.0;
      Lf[k * nP + k] = d > 0.0 ? sqrt(d) : d;
    }
    __syncthreads();
    if (flag[0] != 0.0) return false;
    const double dk = Lf[k * nP + k];
    for (int i = k + 1 + threadIdx.x; i < nP; i += blockDim.x)
      if (sib_pat(i, k, L, rx, ry)) Lf[i * nP + k] /= dk;
    __syncthreads();
    const int m = nP - k - 1;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      const int i = k + 1 + idx / m, j = k + 1 + idx % m;
      if (j > i) continue;
      if (sib_pat(j, k, L, rx, ry) && sib_pat(i, k, L, rx, ry) && sib_pat(i, j, L, rx, ry))
        Lf[i * nP + j] -= Lf[i * nP + k] * Lf[j * nP + k];
    }
    __syncthreads();
  }
  return true;
}

// One CTA per parent P of level l.  nP <= 96.
//
// Strategy 2 (Section 5): a child's unused slots (k >= lv.cnt[child]) are
// decoupled unit-diagonal unknowns; the local eigenproblem is posed on the kept
// coordinates only (compacted), and with a threshold B > 0 (B_cc) the parent
// keeps its candidates with eigenvalue below B, at least one; its other rows of
// Psi are zero and its count goes to nx.cnt.  With given (imported) bases the
// count is the number of leading nonzero rows of Psi.
__global__ void k_coarse_setup(CoarseLevel lv, CoarseLevel nx, double* stats, int given, int ic0, double B) {
  extern __shared__ double sm[];
  const int nP = lv.nP, L = lv.L, L2 = L * L, Ln = lv.Lnext, Ln2 = Ln * Ln;
  double* A = sm;                 // parent's diagonal block of A_l
  double* N = A + nP * nP;        // left matrix of Eq. (spectral cc); then Psi
  double* V = N + nP * nP;        // eigenvectors; then A Psi^T
  double* cs = V + nP * nP;
  double* red = cs + nP + 2;
  int* pr = reinterpret_cast<int*>(red + 72);
  int* order = pr + nP + 2;
  int* ridx = order + nP + 2;     // [nP] kept coordinates of the parent, in order
  int* cidx = ridx + nP;          // [nP] compact index of each coordinate (-1: unused slot)
  __shared__ int s_nr, s_cnt;
  const int64_t P = blockIdx.x;
  const int rx = lv.rx, ry = lv.ry;
  // assemble A_P
  for (int idx = threadIdx.x; idx < nP * nP; idx += blockDim.x) {
    const int i = idx / nP, j = idx % nP;
    const int ca = i / L, k = i % L, cb = j / L, mm = j % L;
    const int64_t a = P * lv.nchild + ca, b = P * lv.nchild + cb;
    double v = 0.0;
    if (ca == cb) v = lv.Ad[a * L2 + k * L + mm];
    else {
      for (int d = 0; d < 3; ++d) {
        if (lv.nbr[a * 6 + 2 * d + 1] == (int)b) v = lv.Ao[(a * 3 + d) * L2 + k * L + mm];
        if (lv.nbr[b * 6 + 2 * d + 1] == (int)a) v = lv.Ao[(b * 3 + d) * L2 + mm * L + k];
      }
    }
    A[idx] = v;
    // Neumann on P: remove the children's face terms on P's boundary
    double nv = v;
    if (ca == cb) {
      const int cx = ca % rx, cy = (ca / rx) % ry, cz = ca / (rx * ry);
      const int cc[3] = {cx, cy, cz}, rr[3] = {lv.rx, lv.ry, lv.rz};
      for (int d = 0; d < 3; ++d) {
        if (cc[d] == 0) nv -= lv.F[(a * 6 + 2 * d) * L2 + k * L + mm];
        if (cc[d] == rr[d] - 1) nv -= lv.F[(a * 6 + 2 * d + 1) * L2 + k * L + mm];
      }
    }
    N[idx] = nv;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nP * nP; idx += blockDim.x) {   // symmetrise
    const int i = idx / nP, j = idx % nP;
    if (i < j) {
      const double s = 0.5 * (N[idx] + N[j * nP + i]);
      N[idx] = s;
      N[j * nP + i] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int nr = 0;
    for (int i = 0; i < nP; ++i) {
      const bool kept = (i % L) < lv.cnt[P * lv.nchild + i / L];
      cidx[i] = kept ? nr : -1;
      if (kept) ridx[nr++] = i;
    }
    s_nr = nr;
  }
  __syncthreads();
  const int nR = s_nr;
  if (!given) {
    // the local problem on the kept coordinates (all of them under Strategy 1)
    for (int idx = threadIdx.x; idx < nR * nR; idx += blockDim.x)
      V[idx] = N[ridx[idx / nR] * nP + ridx[idx % nR]];
    __syncthreads();
    jacobi_eig(V, N, nR, cs, pr, red, 40, 1e-15);
    sort_diag(V, nR, order);
    const int nc = Ln < nR ? Ln : nR;
    if (threadIdx.x == 0) {
      int cn = nc;
      if (B > 0.0) {
        cn = 0;
        for (int j = 0; j < nc; ++j) cn += V[order[j] * nR + order[j]] < B ? 1 : 0;
        if (cn < 1) cn = 1;
      }
      s_cnt = cn;
    }
    for (int j = threadIdx.x; j < Ln; j += blockDim.x)
      lv.lamP[P * Ln + j] = j < nc ? V[order[j] * nR + order[j]] : INFINITY;
    __syncthreads();
    const int cn = s_cnt;
    // Psi (rows = eigenvectors), zero in unused rows and slots
    for (int idx = threadIdx.x; idx < Ln * nP; idx += blockDim.x) {
      const int j = idx / nP, i = idx % nP;
      lv.Psi[(P * Ln + j) * nP + i] = (j < cn && cidx[i] >= 0) ? N[cidx[i] * nR + order[j]] : 0.0;
    }
  } else if (threadIdx.x == 0) {
    int last = 0;
    for (int j = 0; j < Ln; ++j)
      for (int i = 0; i < nP; ++i)
        if (lv.Psi[(P * Ln + j) * nP + i] != 0.0) { last = j + 1; break; }
    s_cnt = last;
  }
  __syncthreads();
  const int cntP = s_cnt;
  if (threadIdx.x == 0) nx.cnt[P] = cntP;
  for (int idx = threadIdx.x; idx < Ln * nP; idx += blockDim.x) {
    const int j = idx / nP, i = idx % nP;
    N[j * nP + i] = lv.Psi[(P * Ln + j) * nP + i];
  }
  __syncthreads();
  // V <- A Psi^T  (nP x Ln)
  for (int idx = threadIdx.x; idx < nP * Ln; idx += blockDim.x) {
    const int i = idx / Ln, j = idx % Ln;
    double acc = 0.0;
    for (int q = 0; q < nP; ++q) acc += A[i * nP + q] * N[j * nP + q];
    V[idx] = acc;
  }
  __syncthreads();
  // next level: diagonal block, face terms, null vector
  for (int o = threadIdx.x; o < Ln2 + 6 * Ln2 + Ln; o += blockDim.x) {
    if (o < Ln2) {
      const int j = o / Ln, jj = o % Ln;
      if (j > jj) continue;
      double acc = 0.0, acc2 = 0.0;
      for (int i = 0; i < nP; ++i) { acc += N[j * nP + i] * V[i * Ln + jj]; acc2 += N[jj * nP + i] * V[i * Ln + j]; }
      double v = 0.5 * (acc + acc2);
      if (j == jj && j >= cntP) v = 1.0;   // unused slot (Strategy 2): a decoupled unknown
      nx.Ad[P * Ln2 + j * Ln + jj] = v;
      nx.Ad[P * Ln2 + jj * Ln + j] = v;
    } else if (o < 7 * Ln2) {
      const int oo = o - Ln2;
      const int f = oo / Ln2, j = (oo % Ln2) / Ln, jj = oo % Ln;
      const int d = f / 2;
      const bool plus = f & 1;
      const int rr[3] = {lv.rx, lv.ry, lv.rz};
      double acc = 0.0;
      for (int ca = 0; ca < lv.nchild; ++ca) {
        const int cc[3] = {ca % rx, (ca / rx) % ry, ca / (rx * ry)};
        if (cc[d] != (plus ? rr[d] - 1 : 0)) continue;
        const int64_t a = P * lv.nchild + ca;
        const double* Fa = lv.F + (a * 6 + f) * L2;
        for (int k = 0; k < L; ++k) {
          const double pj = N[j * nP + ca * L + k];
          if (pj == 0.0) continue;
          double t = 0.0;
          for (int mm = 0; mm < L; ++mm) t += Fa[k * L + mm] * N[jj * nP + ca * L + mm];
          acc += pj * t;
        }
      }
      nx.F[(P * 6 + f) * Ln2 + j * Ln + jj] = acc;
    } else {
      const int j = o - 7 * Ln2;
      double acc = 0.0;
      for (int i = 0; i < nP; ++i) acc += N[j * nP + i] * lv.z[P * nP + i];
      nx.z[P * Ln + j] = acc;
    }
  }
  __syncthreads();
  // smoother: the inverse of the parent's diagonal block (exact block Jacobi), or
  // of L L^T with L its incomplete Cholesky factor (IC(0) block Jacobi)
  if (ic0 && ic0_factor(A, N, nP, L, lv.rx, lv.ry, cs)) {
    // A <- L L^T (then inverted like the exact block)
    for (int idx = threadIdx.x; idx < nP * nP; idx += blockDim.x) {
      const int i = idx / nP, j = idx % nP;
      const int kmax = i < j ? i : j;
      double acc = 0.0;
      for (int k = 0; k <= kmax; ++k) acc += N[i * nP + k] * N[j * nP + k];
      A[idx] = acc;
    }
    __syncthreads();
  } else if (ic0 && threadIdx.x == 0) {
    atomic_max_pos(&stats[8], 1.0);   // this parent fell back to its exact block
  }
  gj_inverse(A, nP, cs, V);
  for (int idx = threadIdx.x; idx < nP * nP; idx += blockDim.x) {
    const double v = A[idx];
    if (!isfinite(v)) atomic_max_pos(&stats[1], 1.0);
    lv.Minv[(size_t)P * nP * nP + idx] = v;
  }
}

// Couplings of A_{l+1}: Ao[P][d] = sum over P's children a on its +d face of
// Psi_P[:, a]^T Ao_l[a][d] Psi_Q[:, a'], Q = P + e_d, a' = a's +d neighbour.
__global__ void k_coarse_galerkin_off(CoarseLevel lv, CoarseLevel nx) {
  const int64_t P = blockIdx.x;
  const int L = lv.L, L2 = L * L, Ln = lv.Lnext, Ln2 = Ln * Ln, nP = lv.nP;
  const int rr[3] = {lv.rx, lv.ry, lv.rz};
  for (int o = threadIdx.x; o < 3 * Ln2; o += blockDim.x) {
    const int d = o / Ln2, j = (o % Ln2) / Ln, jj = o % Ln;
    const int Q = nx.nbr[P * 6 + 2 * d + 1];
    double acc = 0.0;
    if (Q >= 0) {
      for (int ca = 0; ca < lv.nchild; ++ca) {
        const int cc[3] = {ca % lv.rx, (ca / lv.rx) % lv.ry, ca / (lv.rx * lv.ry)};
        if (cc[d] != rr[d] - 1) continue;
        int cb3[3] = {cc[0], cc[1], cc[2]};
        cb3[d] = 0;
        const int cb = cb3[0] + lv.rx * (cb3[1] + lv.ry * cb3[2]);
        const int64_t a = P * lv.nchild + ca;
        const double* ao = lv.Ao + (a * 3 + d) * L2;
        const double* psP = lv.Psi + ((size_t)P * Ln + j) * nP + ca * L;
        const double* psQ = lv.Psi + ((size_t)Q * Ln + jj) * nP + cb * L;
        for (int k = 0; k < L; ++k) {
          double t = 0.0;
          for (int mm = 0; mm < L; ++mm) t += ao[k * L + mm] * psQ[mm];
          acc += psP[k] * t;
        }
      }
    }
    nx.Ao[(P * 3 + d) * Ln2 + j * Ln + jj] = acc;
  }
}

// ------------------------------------------------------------------ coarsest
// Dense A_L (hierarchical order) from the block stencil.  out zeroed beforehand.
__global__ void k_assemble_dense(CoarseLevel lv, double* __restrict__ out) {
  const int64_t a = blockIdx.x;
  const int L = lv.L, L2 = L * L;
  const int64_t n = lv.n;
  for (int o = threadIdx.x; o < L2; o += blockDim.x) {
    const int k = o / L, mm = o % L;
    out[(a * L + k) * n + a * L + mm] = lv.Ad[a * L2 + o];
    for (int d = 0; d < 3; ++d) {
      const int b = lv.nbr[a * 6 + 2 * d + 1];
      if (b < 0) continue;
      const double v = lv.Ao[(a * 3 + d) * L2 + o];
      out[(a * L + k) * n + (int64_t)b * L + mm] = v;
      out[((int64_t)b * L + mm) * n + a * L + k] = v;
    }
  }
}

// Strategy 2 packing of the coarsest level: out[i][j] = B[cmap[i]][cmap[j]]
__global__ void k_pack_dense(const double* __restrict__ B, int64_t n, const int* __restrict__ cmap, int64_t nk,
                             double* __restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nk * nk) return;
  out[idx] = B[(int64_t)cmap[idx / nk] * n + cmap[idx % nk]];
}
__global__ void k_pack_vec(const double* __restrict__ z, const int* __restrict__ cmap, int64_t nk,
                           double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nk) out[i] = z[cmap[i]];
}

// scal[0] = |z|^2, scal[1] = trace(A)
__global__ void k_coarsest_scalars(const double* __restrict__ A, const double* __restrict__ z, int64_t n,
                                   double* scal) {
  double v[2] = {0.0, 0.0};
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    v[0] += z[i] * z[i];
    v[1] += A[i * n + i];
  }
  __shared__ double sh[64];
  block_sum<2>(v, sh);
  if (threadIdx.x == 0) { scal[0] = v[0]; scal[1] = v[1]; }
}

// A += sigma z z^T / |z|^2 with sigma = trace / n
__global__ void k_add_null_shift(double* __restrict__ A, const double* __restrict__ z, int64_t n,
                                 const double* scal) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int64_t i = idx / n, j = idx % n;
  const double sigma = scal[1] / (double)n;
  A[idx] += sigma * z[i] * z[j] / scal[0];
}

// Gauss-Jordan inversion in place (no pivoting: the matrix is symmetric positive
// definite, shifted along its null vector when singular), kGjBlock pivots per pass
// over the matrix, with the arithmetic of one pivot at a time.  Step k of the
// single-pivot form: with c_i = A[i][k] / A[k][k] and r_j = A[k][j],
//   A[i][j] = fma(-c_i, r_j, A[i][j]) for i, j != k,  A[k][j] = r_j / A[k][k],
//   A[i][k] = -c_i,  A[k][k] = 1 / A[k][k].
// For the pivots P = {k, .., k + b - 1} the first launch replays these b steps on
// the rows and columns of P (thread j owns row P's entries in column j and column
// P's entries in row j; every thread also replays the b x b pivot block) and
// records each step's c and r; the second applies the b rank-1 updates to the
// other entries in step order.  Every entry sees the same operations in the same
// order as with one pivot per pass, so the bits are the same, with one sweep of
// the matrix per b pivots instead of one per pivot (the 3740-unknown inverse of the
// IMPES hierarchy: 224 ms with one pivot per pass).
__global__ void k_gj_panel(const double* __restrict__ A, int64_t n, int64_t k, int b, double* __restrict__ cbuf,
                           double* __restrict__ rbuf, double* __restrict__ rfin, double* __restrict__ cfin,
                           double* __restrict__ ppfin, double* stats) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double PP[kGjBlock][kGjBlock];
#pragma unroll
  for (int s = 0; s < kGjBlock; ++s)
#pragma unroll
    for (int u = 0; u < kGjBlock; ++u) PP[s][u] = (s < b && u < b) ? A[(k + s) * n + k + u] : 0.0;
  const bool act = j < n && !(j >= k && j < k + b);
  double R[kGjBlock], Cj[kGjBlock];
#pragma unroll
  for (int s = 0; s < kGjBlock; ++s) {
    R[s] = (act && s < b) ? A[(k + s) * n + j] : 0.0;
    Cj[s] = (act && s < b) ? A[j * n + k + s] : 0.0;
  }
#pragma unroll
  for (int t = 0; t < kGjBlock; ++t) {
    if (t >= b) break;
    const double piv = PP[t][t];
    if (blockIdx.x == 0 && threadIdx.x == 0 && !(piv > 0.0)) atomic_max_pos(&stats[1], 1.0);
    if (act) {
      const double c = Cj[t] / piv, r = R[t];
      cbuf[(int64_t)t * n + j] = c;
      rbuf[(int64_t)t * n + j] = r;
#pragma unroll
      for (int s = 0; s < kGjBlock; ++s)
        if (s < b && s != t) R[s] = fma(-(PP[s][t] / piv), r, R[s]);
      R[t] = r / piv;
#pragma unroll
      for (int u = 0; u < kGjBlock; ++u)
        if (u < b && u != t) Cj[u] = fma(-c, PP[t][u], Cj[u]);
      Cj[t] = -c;
    }
    double cs[kGjBlock];
#pragma unroll
    for (int s = 0; s < kGjBlock; ++s) cs[s] = PP[s][t] / piv;
#pragma unroll
    for (int s = 0; s < kGjBlock; ++s)
#pragma unroll
      for (int u = 0; u < kGjBlock; ++u)
        if (s < b && u < b && s != t && u != t) PP[s][u] = fma(-cs[s], PP[t][u], PP[s][u]);
#pragma unroll
    for (int u = 0; u < kGjBlock; ++u)
      if (u < b && u != t) PP[t][u] = PP[t][u] / piv;
#pragma unroll
    for (int s = 0; s < kGjBlock; ++s)
      if (s < b && s != t) PP[s][t] = -cs[s];
    PP[t][t] = 1.0 / piv;
  }
  if (act) {
#pragma unroll
    for (int s = 0; s < kGjBlock; ++s)
      if (s < b) {
        rfin[(int64_t)s * n + j] = R[s];
        cfin[j * kGjBlock + s] = Cj[s];
      }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0)
    for (int s = 0; s < b; ++s)
      for (int u = 0; u < b; ++u) ppfin[s * b + u] = PP[s][u];
}

__global__ void k_gj_block_update(double* __restrict__ A, int64_t n, int64_t k, int b,
                                  const double* __restrict__ cbuf, const double* __restrict__ rbuf,
                                  const double* __restrict__ rfin, const double* __restrict__ cfin,
                                  const double* __restrict__ ppfin) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int64_t i = idx / n, j = idx % n;
  const bool pi = i >= k && i < k + b, pj = j >= k && j < k + b;
  double v;
  if (pi && pj) {
    v = ppfin[(i - k) * b + (j - k)];
  } else if (pi) {
    v = rfin[(i - k) * n + j];
  } else if (pj) {
    v = cfin[i * kGjBlock + (j - k)];
  } else {
    v = A[idx];
#pragma unroll
    for (int t = 0; t < kGjBlock; ++t)
      if (t < b) v = fma(-cbuf[(int64_t)t * n + i], rbuf[(int64_t)t * n + j], v);
  }
  A[idx] = v;
}

// w = B zhat (B the inverse), gamma = zhat^T w; zhat = z / |z|
__global__ void k_gemv_z(const double* __restrict__ B, const double* __restrict__ z, int64_t n, const double* scal,
                         double* __restrict__ w) {
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  const double inv = 1.0 / sqrt(scal[0]);
  double acc = 0.0;
  for (int64_t j = lane; j < n; j += 32) acc += B[row * n + j] * z[j] * inv;
  acc = warp_sum(acc);
  if (lane == 0) w[row] = acc;
}

__global__ void k_dot_zw(const double* __restrict__ z, const double* __restrict__ w, int64_t n, double* scal) {
  double v[1] = {0.0};
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v[0] += z[i] * w[i];
  __shared__ double sh[32];
  block_sum<1>(v, sh);
  if (threadIdx.x == 0) scal[2] = v[0] / sqrt(scal[0]);
}

// pinv = (I - zz^T) B (I - zz^T) = B - w z^T - z w^T + gamma z z^T  (zhat normalised)
__global__ void k_project(const double* __restrict__ B, const double* __restrict__ z, const double* __restrict__ w,
                          int64_t n, const double* scal, double* __restrict__ out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int64_t i = idx / n, j = idx % n;
  const double inv = 1.0 / sqrt(scal[0]);
  const double zi = z[i] * inv, zj = z[j] * inv;
  out[idx] = B[idx] - w[i] * zj - zi * w[j] + scal[2] * zi * zj;
}

// ------------------------------------------------------------------ export / import
// level 1: Phi[hid][L][nb] <-> out[lex][L][nb]; level >= 2: Psi[hidP][Ln][nP] <-> out[lexP][Ln][nP]
__global__ void k_basis_xfer(double* __restrict__ dev, double* __restrict__ ext, const int* __restrict__ lex_of_hid,
                             int64_t m, int64_t per, const double* __restrict__ lam_dev, double* __restrict__ lam_ext,
                             int64_t lper, bool import) {
  const int64_t e = blockIdx.x;
  const int64_t lx = lex_of_hid[e];
  for (int64_t i = threadIdx.x; i < per; i += blockDim.x) {
    if (import) dev[e * per + i] = ext[lx * per + i];
    else ext[lx * per + i] = dev[e * per + i];
  }
  if (!import && lam_ext)
    for (int64_t i = threadIdx.x; i < lper; i += blockDim.x) lam_ext[lx * lper + i] = lam_dev[e * lper + i];
}

// dense operator in the paper's coordinate order (lexicographic elements)
__global__ void k_operator_export(CoarseLevel lv, double* __restrict__ out) {
  const int64_t a = blockIdx.x;
  const int L = lv.L, L2 = L * L;
  const int64_t n = lv.n;
  const int64_t la = lv.lex_of_hid[a];
  for (int o = threadIdx.x; o < L2; o += blockDim.x) {
    const int k = o / L, mm = o % L;
    out[(la * L + k) * n + la * L + mm] = lv.Ad[a * L2 + o];
    for (int d = 0; d < 3; ++d) {
      const int b = lv.nbr[a * 6 + 2 * d + 1];
      if (b < 0) continue;
      const int64_t lb = lv.lex_of_hid[b];
      const double v = lv.Ao[(a * 3 + d) * L2 + o];
      out[(la * L + k) * n + lb * L + mm] = v;
      out[(lb * L + mm) * n + la * L + k] = v;
    }
  }
}

// ------------------------------------------------------------------ host launchers
static size_t jac_smem(int n, int extra_mats) {
  return (size_t)extra_mats * n * n * sizeof(double) + (size_t)(2 * n + 4 + 72) * sizeof(double) +
         (size_t)(4 * n + 4) * sizeof(int) + 64;
}

int launch_level1_eigen(msmg_ctx* c, cudaStream_t s) {
  FineLevel& f = c->fine;
  if (f.nb > 96) return MSMG_ERR_UNSUPPORTED;   // large elements use the subspace solver
  const size_t sm = jac_smem(f.nb, 2);
  cudaFuncSetAttribute(k_eig_l1_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_eig_l1_jacobi<<<(unsigned)f.m, 256, sm, s>>>(f.T, f.S, c->n, f.bx, f.by, f.bz, f.m, f.L, f.Phi, f.lam,
                                                  c->dtmp, f.Wd);
  return 0;
}

void launch_level1_galerkin(msmg_ctx* c, cudaStream_t s, bool threshold) {
  FineLevel& f = c->fine;
  CoarseLevel& l2 = c->lev[2];
  const double B = threshold ? c->opts.eig_threshold[0] : 0.0;
  k_level1_counts<<<(unsigned)((f.m + 7) / 8), 256, 0, s>>>(f.Phi, f.lam, f.m, f.L, f.nb, B, l2.cnt);
  const size_t sm = (size_t)(2 * f.L * f.nb + 3 * f.nb) * sizeof(double);
  cudaFuncSetAttribute(k_galerkin1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  const unsigned thr = f.nb >= 256 ? 256 : (unsigned)((f.nb + 31) / 32 * 32 < 64 ? 64 : (f.nb + 31) / 32 * 32);
  k_galerkin1<<<(unsigned)f.m, thr, sm, s>>>(f.T, f.S, c->n, f.bx, f.by, f.bz, f.m, f.nbr, f.L, f.Phi, l2.Ad, l2.Ao,
                                             l2.F, l2.z, l2.cnt, f.Wd);
}

int launch_coarse_setup(msmg_ctx* c, int l, cudaStream_t s) {
  CoarseLevel& lv = c->lev[l];
  CoarseLevel& nx = c->lev[l + 1];
  if (lv.nP > 96) return MSMG_ERR_UNSUPPORTED;
  const size_t sm = jac_smem(lv.nP, 3);
  cudaFuncSetAttribute(k_coarse_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_coarse_setup<<<(unsigned)lv.mP, 256, sm, s>>>(lv, nx, c->dtmp, 0, c->opts.coarse_smoother == MSMG_BLOCK_IC0,
                                                  c->opts.eig_threshold[l - 1]);
  k_coarse_galerkin_off<<<(unsigned)lv.mP, 128, 0, s>>>(lv, nx);
  return 0;
}

// Same with the bases Psi already in place (imported): no eigensolve.
int launch_coarse_setup_given(msmg_ctx* c, int l, cudaStream_t s) {
  CoarseLevel& lv = c->lev[l];
  CoarseLevel& nx = c->lev[l + 1];
  if (lv.nP > 96) return MSMG_ERR_UNSUPPORTED;
  const size_t sm = jac_smem(lv.nP, 3);
  cudaFuncSetAttribute(k_coarse_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_coarse_setup<<<(unsigned)lv.mP, 256, sm, s>>>(lv, nx, c->dtmp, 1, c->opts.coarse_smoother == MSMG_BLOCK_IC0,
                                                  0.0);
  k_coarse_galerkin_off<<<(unsigned)lv.mP, 128, 0, s>>>(lv, nx);
  return 0;
}

int launch_coarsest(msmg_ctx* c, cudaStream_t s) {
  CoarseLevel& lv = c->lev[c->nL];
  const int64_t n = lv.n;
  // Strategy 2: the pseudo-inverse is built and applied on the kept coordinates
  // only (packed), so unused slots cost the dense solve nothing
  {
    std::vector<int> cnt((size_t)lv.me), cmap, cinv((size_t)n, -1);
    MSMG_CUDA_TRY(cudaMemcpyAsync(cnt.data(), lv.cnt, (size_t)lv.me * sizeof(int), cudaMemcpyDeviceToHost, s));
    MSMG_CUDA_TRY(cudaStreamSynchronize(s));
    for (int64_t a = 0; a < lv.me; ++a)
      for (int k = 0; k < cnt[a] && k < lv.L; ++k) {
        cinv[a * lv.L + k] = (int)cmap.size();
        cmap.push_back((int)(a * lv.L + k));
      }
    lv.nk = (int64_t)cmap.size();
    if (lv.nk < n) {
      lv.cmap = c->cmaps;
      lv.cinv = c->cmaps + n;
      MSMG_CUDA_TRY(cudaMemcpyAsync(lv.cmap, cmap.data(), cmap.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      MSMG_CUDA_TRY(cudaMemcpyAsync(lv.cinv, cinv.data(), cinv.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      MSMG_CUDA_TRY(cudaStreamSynchronize(s));   // the host maps go out of scope
    } else {
      lv.cmap = lv.cinv = nullptr;
    }
  }
  const int64_t nk = lv.nk;
  double* B = c->dtmp + 16;
  double* cbuf = B + n * n;                  // [kGjBlock][n] each step's multipliers
  double* rbuf = cbuf + kGjBlock * n;         // [kGjBlock][n] each step's pivot row
  double* rfin = rbuf + kGjBlock * n;         // [kGjBlock][n] the pivot rows after the pass
  double* cfin = rfin + kGjBlock * n;         // [n][kGjBlock] the pivot columns after the pass
  double* ppfin = cfin + kGjBlock * n;        // [kGjBlock^2] the pivot block after the pass
  double* w = ppfin + kGjBlock * kGjBlock;
  double* scal = c->dtmp + 4;
  MSMG_CUDA_TRY(cudaMemsetAsync(B, 0, (size_t)n * n * sizeof(double), s));
  k_assemble_dense<<<(unsigned)lv.me, 64, 0, s>>>(lv, B);
  const double* z = lv.z;
  if (nk < n) {
    // packed matrix and null vector (the pinv array is scratch until the end)
    k_pack_dense<<<(unsigned)((nk * nk + 255) / 256), 256, 0, s>>>(B, n, lv.cmap, nk, lv.pinv);
    MSMG_CUDA_TRY(cudaMemcpyAsync(B, lv.pinv, (size_t)nk * nk * sizeof(double), cudaMemcpyDeviceToDevice, s));
    k_pack_vec<<<(unsigned)((nk + 255) / 256), 256, 0, s>>>(lv.z, lv.cmap, nk, lv.pinv + nk * nk);
    z = lv.pinv + nk * nk;
  }
  const unsigned g2 = (unsigned)((nk * nk + 255) / 256);
  const unsigned g1 = (unsigned)((nk + 255) / 256);
  const bool singular = c->fine.Wd == nullptr;   // a cell term (wells) removes the null space
  if (singular) {
    k_coarsest_scalars<<<1, 256, 0, s>>>(B, z, nk, scal);
    k_add_null_shift<<<g2, 256, 0, s>>>(B, z, nk, scal);
  }
  for (int64_t k = 0; k < nk; k += kGjBlock) {
    const int b = (int)(nk - k < kGjBlock ? nk - k : kGjBlock);
    k_gj_panel<<<g1, 256, 0, s>>>(B, nk, k, b, cbuf, rbuf, rfin, cfin, ppfin, c->dtmp);
    k_gj_block_update<<<g2, 256, 0, s>>>(B, nk, k, b, cbuf, rbuf, rfin, cfin, ppfin);
  }
  if (singular) {
    k_gemv_z<<<(unsigned)((nk * 32 + 255) / 256), 256, 0, s>>>(B, z, nk, scal, w);
    k_dot_zw<<<1, 256, 0, s>>>(z, w, nk, scal);
    k_project<<<g2, 256, 0, s>>>(B, z, w, nk, scal, lv.pinv);
  } else {
    MSMG_CUDA_TRY(cudaMemcpyAsync(lv.pinv, B, (size_t)nk * nk * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  return 0;
}

void launch_basis_export(msmg_ctx* c, int level, double* basis, double* lam, bool import, cudaStream_t s) {
  if (level == 1) {
    FineLevel& f = c->fine;
    k_basis_xfer<<<(unsigned)f.m, 256, 0, s>>>(f.Phi, basis, f.lex_of_hid, f.m, (int64_t)f.L * f.nb, f.lam, lam, f.L,
                                               import);
  } else {
    CoarseLevel& lv = c->lev[level];
    const CoarseLevel& up = c->lev[level + 1];
    k_basis_xfer<<<(unsigned)lv.mP, 256, 0, s>>>(lv.Psi, basis, up.lex_of_hid, lv.mP, (int64_t)lv.Lnext * lv.nP,
                                                 lv.lamP, lam, lv.Lnext, import);
  }
}

void launch_operator_export(msmg_ctx* c, int level, double* out, cudaStream_t s) {
  CoarseLevel& lv = c->lev[level];
  cudaMemsetAsync(out, 0, (size_t)lv.n * lv.n * sizeof(double), s);
  k_operator_export<<<(unsigned)lv.me, 64, 0, s>>>(lv, out);
}

}  // namespace msmg

namespace msmg {
// dims_kept: the number of kept coordinates of every coarse level
void launch_kept_sums(msmg_ctx* c, cudaStream_t s) {
  cudaMemsetAsync(c->kept, 0, (kMaxLevels + 1) * sizeof(unsigned long long), s);
  for (int l = 2; l <= c->nL; ++l) {
    const CoarseLevel& lv = c->lev[l];
    unsigned g = (unsigned)((lv.me + 255) / 256);
    if (g > 1024) g = 1024;
    k_kept_sum<<<g, 256, 0, s>>>(lv.cnt, lv.me, c->kept + l);
  }
}
}  // namespace msmg
