// Internal declarations shared by the msmg CUDA translation units.
//
// Data layout in device memory (all inside the caller's workspace):
//   * Element ordering is hierarchical at every level: the elements of E_l are
//     numbered parent-major (the r^3 children of one element of E_{l+1} are
//     consecutive, in lexicographic order inside the parent), and the elements
//     of the top element level E_{L-1} are lexicographic.  So every block of
//     every smoother and every local spectral problem is one contiguous range.
//   * Fine-level vectors are block-major: cell (element e, local p) sits at
//     e * nb + p with p = lx + bx*(ly + by*lz).  Each element's data is one
//     contiguous, coalesced chunk.
//   * A level-l vector (l >= 2) stores the coordinates of element e of E_{l-1}
//     at e * L + k, k < L.
#pragma once
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>
#include <vector>
#include "../../include/msmg.h"

namespace msmg {

constexpr int kMaxLevels = MSMG_MAX_LEVELS;

// ---------------------------------------------------------------- errors
#define MSMG_CUDA_TRY(expr)                                                   \
  do {                                                                        \
    cudaError_t _e = (expr);                                                  \
    if (_e != cudaSuccess) { ::msmg::set_last_cuda_error(_e); return MSMG_ERR_CUDA; } \
  } while (0)
void set_last_cuda_error(cudaError_t e);

// ---------------------------------------------------------------- arena
// Bump allocator over the caller's workspace.  With base == nullptr it only
// measures (used by msmg_workspace_size).
struct Arena {
  char* base = nullptr;
  size_t off = 0;
  size_t cap = 0;
  template <typename T>
  T* take(size_t count, size_t align = 256) {
    off = (off + align - 1) / align * align;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

// ---------------------------------------------------------------- PCG scalars
// One record per right-hand side, in device memory.  Written by the
// last-finishing CTA of each reducing kernel.
struct PcgScalars {
  double bb;         // ||b||^2 after mean removal
  double tol2;       // (rtol ||b||)^2
  double rz;         // r^T z (current)
  double rz_old;     // previous r^T z
  double rz_mix;     // z_new^T r_old (flexible beta)
  double pq;         // p^T A p
  double rr;         // ||r||^2
  double alpha, beta;
  double mean;       // removed rhs mean
  int iter;          // completed iterations
  int done;          // 1 converged, 2 breakdown, 3 max_iter
  int max_iter;
  int flexible;
};

// A deterministic grid reduction slot: per-CTA partials, a ticket counter and
// a result.  The last CTA to finish sums the partials in index order.
//
// A batched launch (R right-hand sides in lockstep) reduces each right-hand
// side separately: slice r of the partials starts at r * stride and uses
// counter[r].
struct RedSlot {
  double* partials;     // [R][max CTAs of a reducing launch per rhs][kRedWidth]
  unsigned* counter;    // [R], zero between uses
  int64_t stride;       // doubles per right-hand-side slice of partials
};
constexpr int kRedWidth = 4;   // up to 4 simultaneous sums per reduction

// Batched launches order their CTAs right-hand-side minor: CTA b works on block
// b / R of the data of right-hand side b % R, so the R CTAs that share an
// element's coefficients run next to each other and the coefficients are read
// from HBM once and from L2 R - 1 times.
struct BatchIdx {
  int r;              // right-hand side
  unsigned blk;       // block index within the right-hand side
  unsigned nblk;      // blocks per right-hand side
};
__device__ __forceinline__ BatchIdx batch_idx(int R) {
  BatchIdx b;
  b.r = (int)(blockIdx.x % (unsigned)R);
  b.blk = blockIdx.x / (unsigned)R;
  b.nblk = gridDim.x / (unsigned)R;
  return b;
}
__host__ __device__ __forceinline__ RedSlot red_for(const RedSlot& red, int r) {
  RedSlot o;
  o.partials = red.partials + (int64_t)r * red.stride;
  o.counter = red.counter + r;
  o.stride = red.stride;
  return o;
}

// ---------------------------------------------------------------- levels
struct FineLevel {
  int bx, by, bz, nb;           // element size and cells per element
  int gx, gy, gz;               // element grid
  int64_t m;                    // elements
  int64_t n;                    // cells
  int L;                        // eigenvectors per element (n_eig[0])
  int nu;
  int* lex_of_hid;              // [m] lexicographic element index of hierarchical index
  int* nbr;                     // [m][6] neighbour hid (-x,+x,-y,+y,-z,+z), -1 on boundary
  double* T;                    // [3][n] face coefficients (FP64, block-major)
  double* S;                    // [n] Tr K~
  double* invd;                 // [n] inverse IC(0) pivots
  double* D;                    // [n] diagonal of A (sum of the six face coefficients)
  double* Phi;                  // [m][L][nb] S-orthonormal basis
  double* lam;                  // [m][L]
  float* T32;                   // mixed-precision copies (nullptr in FP64 mode)
  float* invd32;
  float* Phi32;
  double* Wd;                   // [n] cell term W of A (wells), block-major; nullptr: none
  float* Wd32;                  // its FP32 copy (mixed form)
};

struct CoarseLevel {            // level l >= 2 (W_l)
  int l;
  int gx, gy, gz;               // grid of E_{l-1} (elements carrying L dofs each)
  int64_t me;                   // elements of E_{l-1}
  int L;                        // dofs per element = n_eig[l-2]
  int64_t n;                    // me * L
  int nu;
  int* lex_of_hid;              // [me]
  int* nbr;                     // [me][6]
  double* Ad;                   // [me][L][L] diagonal blocks of A_l
  double* Ao;                   // [me][3][L][L] A_l[a, a+e_d], d = x, y, z
  double* F;                    // [me][6][L][L] face terms (setup only)
  double* z;                    // [n] null vector of A_l
  int* cnt;                     // [me] coordinates each element keeps (Strategy 2; L otherwise):
                                //      slots k >= cnt are decoupled unit-diagonal unknowns that
                                //      stay zero (their basis rows one level down are zero)
  // smoother / restriction towards level l+1 (absent at the coarsest level)
  int rx, ry, rz, nchild;       // children per parent (ratio of E_l over E_{l-1})
  int64_t mP;                   // parents (elements of E_l)
  int nP;                       // dofs per parent = nchild * L
  int Lnext;                    // n_eig[l-1]
  double* Minv;                 // [mP][nP][nP] inverse of each parent's diagonal block
  double* Psi;                  // [mP][Lnext][nP]
  double* lamP;                 // [mP][Lnext]
  // coarsest only
  double* pinv;                 // [nk][nk] pseudo-inverse on the kept coordinates
  int64_t nk;                   // kept coordinates (n under Strategy 1)
  int* cmap;                    // [nk] packed -> padded coordinate, null when nk == n
  int* cinv;                    // [n] padded -> packed coordinate (-1: unused slot), null when nk == n
};

struct SolveBuffers {
  // fine level, FP64, block-major
  double *b, *x, *r, *z, *p0, *p1, *q;
  double *pcur, *pnext;         // ping-pong search directions of the current iteration
  void* rv;                     // residual in V-cycle precision
  float* ec32;                  // FP32 copy of the level-2 correction (mixed form), else nullptr
  // V-cycle work on every level: f (right side), u (iterate), w (scratch); level 1 in
  // the V-cycle precision, levels >= 2 in FP64
  void* vf[kMaxLevels + 1];     // indexed by level, 1 .. n_levels
  void* vu[kMaxLevels + 1];
  void* vw[kMaxLevels + 1];
  PcgScalars* sc;               // [n_rhs]
  int n_rhs;                    // capacity: every vector above holds n_rhs copies
  int R;                        // right-hand sides of the batch in flight (<= n_rhs)
  double* dres;                 // [n_rhs][2] true-residual norms, mean sums
  int* dmask;                   // [n_rhs] restart mask
  // exact two-grid (level-2 inner PCG), null otherwise: level-2 vectors x, p (two),
  // q; per-CTA partial sums; inner iteration counts
  double *ix, *ip0, *ip1, *iq, *ipart;
  int* iiters;
};

}  // namespace msmg

namespace msmg {
// pivots per pass of the blocked Gauss-Jordan inversion of the coarsest matrix
constexpr int kGjBlock = 4;
}

struct msmg_ctx {
  msmg_grid grid;
  msmg_options opts;
  int nL;                                       // n_levels
  int64_t n;                                    // fine cells
  msmg::FineLevel fine;
  msmg::CoarseLevel lev[msmg::kMaxLevels + 1];  // lev[l] for l = 2 .. nL (index by level)
  msmg::SolveBuffers sb;
  msmg::RedSlot red;                            // reduction scratch
  double* dtmp;                                 // setup scratch (dense coarsest work etc.)
  int* flags;                                   // [4] device error flags
  int* hflags;                                  // pinned host mirror
  size_t ws_bytes;
  msmg_setup_info info;
  cudaEvent_t ev0, ev1;
  int device;
  int max_rhs;
  cudaStream_t cap_stream;                      // private stream for graph capture
  cudaGraphExec_t iter_graph;                   // two captured PCG iterations
  int graph_state;                              // 0 not built, 1 ready, -1 capture failed
  int graph_R;                                  // batch width the graph was captured for
  msmg::PcgScalars* hsc;                        // pinned host mirror of sb.sc [max_rhs]
  double* hres;                                 // pinned host mirror of sb.dres [max_rhs][2]
  int* hmask;                                   // pinned host restart mask [max_rhs]
  cudaEvent_t poll_evs[3];                      // PCG polls: two in-flight chunks, exit checks
  cudaStream_t run_stream;                      // per-context stream of batched solves
  // autotuned variants (result-preserving), index 0: batch width 1, 1: wider batches
  int tune_fused[2];                            // prolongation inside k_post (1) or separate (0)
  int tune_tail[2];                             // coarse cycle: per level (0), cluster tail (1), one grid (2)
  int tuned[2];                                 // set once measured
  int pf_post[2];                               // resident CTAs of k_post (unfused, fused): its L2 prefetch distance
  int tail_l0;                                  // first level of the cluster tail (0: none)
  int tail_cs;                                  // CTAs per cluster
  int tail_lt;                                  // compile-time L of the tail levels (0: runtime)
  size_t tail_smem;
  int coop_grid;                                // CTAs of the cooperative coarse cycle (0: unavailable)
  int inner_grid;                               // CTAs of the exact two-grid inner solve (0: unavailable)
  unsigned long long* kept;                     // [kMaxLevels + 1] sum of cnt per level (device)
  int* cmaps;                                   // [2 n_L] storage of the coarsest packing maps
  int coop_lt;
  size_t coop_smem;
};

namespace msmg {
// ---------------------------------------------------------------- plan
int plan_and_carve(const msmg_grid* g, const msmg_options* o, int n_rhs, Arena& ar, msmg_ctx* ctx);
int validate(const msmg_grid* g, const msmg_options* o);

// ---------------------------------------------------------------- launchers (fine level)
void launch_faces(msmg_ctx* c, const void* kappa, int comps, int dtype, cudaStream_t s);
void launch_pivots(msmg_ctx* c, cudaStream_t s);
void launch_nat_to_blk(msmg_ctx* c, const double* in, double* out, cudaStream_t s);
void launch_blk_to_nat(msmg_ctx* c, const double* in, double* out, cudaStream_t s);
void launch_faces_to_nat(msmg_ctx* c, double* out, cudaStream_t s);
// q = A p (FP64, block-major) for R right-hand sides stored n apart.
void launch_matvec(msmg_ctx* c, const double* p, double* q, cudaStream_t s, int R = 1);

// ---------------------------------------------------------------- setup
int launch_level1_eigen(msmg_ctx* c, cudaStream_t s);
void launch_level1_galerkin(msmg_ctx* c, cudaStream_t s, bool threshold);
int launch_coarse_setup(msmg_ctx* c, int l, cudaStream_t s);
int launch_coarsest(msmg_ctx* c, cudaStream_t s);
void launch_basis_export(msmg_ctx* c, int level, double* basis, double* lam, bool import, cudaStream_t s);
void launch_operator_export(msmg_ctx* c, int level, double* out, cudaStream_t s);

// ---------------------------------------------------------------- solve
int pcg_solve(msmg_ctx* c, const double* rhs_nat, double* x_nat, int n_rhs, double rtol, int max_iter, int flags,
              cudaStream_t s, msmg_solve_info* info);
double dot_host(msmg_ctx* c, const double* a, const double* b, int64_t n, cudaStream_t s);

// ---------------------------------------------------------------- device helpers
template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP32 <-> FP64 conversions on the integer pipes.  GB300 runs conversions on
// its FP64 pipe (2 per clock per SM), which the FP64 PCG arithmetic already
// saturates; these rebuild the IEEE 754 encodings with integer operations.
// binary32: 1 sign, 8 exponent (bias 127), 23 fraction bits; binary64: 1, 11
// (bias 1023), 52.  Results equal the hardware conversions bit for bit
// (round to nearest, ties to even), NaNs stay NaNs.

// Exact widening.
__device__ __forceinline__ double f64_of_f32(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
  const uint32_t mag = u & 0x7fffffffu;
  uint64_t out;
  if (mag >= 0x00800000u && mag < 0x7f800000u) {
    // normal: exponent re-biased by 1023 - 127, fraction moved up 29 bits
    out = ((uint64_t)mag + ((uint64_t)(1023 - 127) << 23)) << 29;
  } else if (mag >= 0x7f800000u) {
    out = 0x7ff0000000000000ull | ((uint64_t)(mag & 0x007fffffu) << 29);   // inf, NaN
  } else if (mag == 0u) {
    out = 0;
  } else {
    // subnormal m 2^-149: the leading one at bit p gives exponent p - 149
    const int p = 31 - __clz((int)mag);
    out = ((uint64_t)(p - 149 + 1023) << 52) | (((uint64_t)mag << (52 - p)) & 0x000fffffffffffffull);
  }
  return __longlong_as_double((long long)(sign | out));
}

// Narrowing, round to nearest, ties to even.
__device__ __forceinline__ float f32_of_f64_rn(double d) {
  const uint64_t u = (uint64_t)__double_as_longlong(d);
  const uint32_t sign = (uint32_t)(u >> 32) & 0x80000000u;
  const int e = (int)((u >> 52) & 0x7ff);
  const uint64_t frac = u & 0x000fffffffffffffull;
  uint32_t out;
  if (e == 0x7ff) {
    out = frac ? (0x7fc00000u | (uint32_t)(frac >> 29)) : 0x7f800000u;
  } else {
    const int ef = e - 1023 + 127;        // binary32 biased exponent
    if (ef >= 0xff) {
      out = 0x7f800000u;                   // beyond the binary32 range
    } else if (ef >= 1) {
      const uint32_t m = (uint32_t)(frac >> 29);
      const uint32_t rem = (uint32_t)(frac & 0x1fffffffu);
      out = ((uint32_t)ef << 23) | m;
      // a carry out of the fraction steps the exponent (up to inf)
      out += (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
    } else {
      // binary32 subnormal or zero: significand with its leading one, shifted by 30 - ef
      const int sh = 30 - ef;
      if (e == 0 || sh > 54) {
        out = 0;                           // below half the smallest subnormal
      } else {
        const uint64_t sig = frac | 0x0010000000000000ull;
        const uint32_t m = (uint32_t)(sig >> sh);
        const uint64_t rem = sig & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        out = m + ((rem > half || (rem == half && (m & 1u))) ? 1u : 0u);
      }
    }
  }
  return __uint_as_float(sign | out);
}

}  // namespace msmg
