// Fine-level PCG iteration kernels, one warp per element (two in the FP64 k_post
// on 8^3 elements, see elem_threads).
//
// Each element of E_1 (bx x by x bz cells) is handled by one warp.  Its data is
// one contiguous chunk of every block-major array; the warp stages what it
// reuses (the iterate u with its one-cell face halo, the face coefficients T,
// the inverse IC(0) pivots) in shared memory with asynchronous copies, all in
// flight at once, then works out of shared memory.  The incomplete-Cholesky
// solves of the block-Jacobi smoother (Section 5) sweep the element in
// wavefronts lx + ly + lz = const; the element's threads take the cells of a
// wavefront (dealt from a plane table, or on fixed x-lines, see w_ic0_s), so
// consecutive wavefronts only need a barrier of the element's threads.
//
// The element shape is a template parameter: 8^3 and 4^3 elements are compiled
// with constant geometry (index arithmetic folds to shifts, loops unroll);
// other shapes use the same code with runtime geometry.
//
// One PCG iteration on the fine level is four kernels:
//   k_pmatvec  p = z + beta p_old (cells and halo), q = A p, reduce p.q -> alpha
//   k_pre      x += alpha p, r -= alpha q, reduce r.r (convergence), and the
//              pre-smoothing u = M^{-1} r of Algorithm 1 (from u = 0)
//   k_restrict r_c = Phi^T (r - A u) per element (Algorithm 1, restriction)
//   k_post     prolongation u' = u + Phi e_c (Algorithm 1) applied to the staged
//              tile (the element's cells and its face halo, the halo with the
//              neighbours' bases and coarse coordinates), then the
//              post-smoothing z = u' + M^{-T} (r - A u'); reduces r.z (and z.q
//              for the flexible beta)
// or, as two launches, k_prolong (u += Phi e_c, a thread per cell) and k_post
// without the prolongation.  Both give the same bits; the context's autotuner
// picks the faster per batch width.
//
// Every kernel also runs R right-hand sides in lockstep (vectors stored n
// apart, one PcgScalars record and one reduction slice each): CTA b handles
// element group b / R of right-hand side b % R, so an element's coefficients
// are read from HBM once per launch and from L2 by the other R - 1 CTAs.
#include "msmg_internal.cuh"
#include "reduce.cuh"
#include <type_traits>

namespace msmg {

// compile-time element geometry
template <int BX, int BY, int BZ>
struct GeoC {
  static constexpr int bx = BX, by = BY, bz = BZ, nb = BX * BY * BZ, nlines = BY * BZ;
  static constexpr int P = (BX + 2) * (BY + 2) * (BZ + 2);
};
// runtime element geometry
struct GeoR {
  int bx, by, bz, nb, nlines, P;
};
static inline GeoR make_geor(int bx, int by, int bz) {
  GeoR g;
  g.bx = bx; g.by = by; g.bz = bz; g.nb = bx * by * bz; g.nlines = by * bz;
  g.P = (bx + 2) * (by + 2) * (bz + 2);
  return g;
}

template <typename G>
struct IsCube8 : std::false_type {};
template <>
struct IsCube8<GeoC<8, 8, 8>> : std::true_type {};

// Threads per element of the staged kernels: two warps for an 8^3 element in
// the FP64 k_post (a wavefront has at most 48 cells, so each thread takes at
// most one cell of it, and an SM keeps twice the warps for the same staged
// bytes: 182 -> 168 us on 128^3), one warp otherwise (there the pair's
// barriers cost more than the extra warps gain).  A two-warp element is a CTA
// of its own, so that its barriers are the CTA's.
constexpr int kStageFull = 0, kStagePre = 1, kStageRestrict = 2, kStageRestrictT = 3;
template <int LAYOUT, typename G, typename V>
__host__ __device__ constexpr int elem_threads() {
  return IsCube8<G>::value && sizeof(V) == 8 && LAYOUT == kStageFull ? 64 : 32;
}

constexpr int kWarpsPerCta = 4;
constexpr int kProlongLMax = 8;   // local basis sizes with all loads of a cell in flight at once

template <typename G>
__device__ __forceinline__ int wpad(const G& g, int lx, int ly, int lz) {
  return (lx + 1) + (g.bx + 2) * ((ly + 1) + (g.by + 2) * (lz + 1));
}

// Element context: base offset and the six neighbour element bases (-1: none).
struct WElem {
  int64_t base;
  int64_t nb6[6];
};

template <typename G>
__device__ __forceinline__ WElem w_elem(int64_t e, const int* __restrict__ nbr, const G& g) {
  WElem E;
  E.base = e * g.nb;
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int ne = __ldg(nbr + e * 6 + f);
    E.nb6[f] = ne >= 0 ? (int64_t)ne * g.nb : -1;
  }
  return E;
}

// ------------------------------------------------------------------ staging
// Asynchronous global -> shared copies: every copy of an element's working set
// is in flight at once, so the element pays one memory latency before its
// wavefronts run out of shared memory.
__device__ __forceinline__ void cp_async_16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_async_elem(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_async_elem(double* dst, const double* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Bulk asynchronous copies (the TMA engine, untiled form) of contiguous arrays
// into shared memory, completion tracked by one mbarrier per warp: one lane
// issues them, every lane waits.  Addresses 16-byte aligned, sizes multiples of
// 16 bytes.
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned bar) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(d),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// Waits for phase ``parity`` of the barrier to complete; gives up (false) after
// about a million polls instead of waiting without bound.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  for (int it = 0; it < (1 << 20); ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Barrier of the NT threads that work on one element: the warp, or the CTA
// when the element has one to itself (NT > 32).
template <int NT>
__device__ __forceinline__ void ebar() {
  if constexpr (NT == 32) __syncwarp();
  else __syncthreads();
}
// AND of a predicate over the element's threads, the same answer in all of
// them; also a barrier.
template <int NT>
__device__ __forceinline__ bool eall(bool p) {
  if constexpr (NT == 32) {
    const bool r = __all_sync(0xffffffffu, p);
    __syncwarp();
    return r;
  } else {
    return __syncthreads_and(p) != 0;
  }
}

// Completion of an element's bulk copies, the same answer in all its threads.
// When the bounded wait gives up, the error word is set (whatever path
// launched the kernel), the right-hand side is marked as broken down, and the
// copies get a second bounded wait before the threads skip the element: they
// then use none of the staged data.
template <int NT>
__device__ __forceinline__ bool bulk_landed(bool bulk, unsigned bar, PcgScalars* sc, int* err, int et) {
  const bool ok = eall<NT>(!bulk || mbar_wait(bar, 0));
  if (!ok) {
    if (et == 0) {
      atomicExch(err, 1);
      if (sc) sc->done = 2;
    }
    mbar_wait(bar, 0);
  }
  ebar<NT>();
  return ok;
}

// L2 prefetch (bulk, nothing waits for it) of bytes at p: 16-byte aligned,
// a multiple of 16 bytes.
__device__ __forceinline__ void l2_prefetch(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}
// The element (e2, right-hand side r2) that slot ``slot`` of the CTA ``pf``
// places ahead will work on, if that CTA exists: with pf = the CTAs resident
// at once, each wave's CTAs prefetch the next wave's arrays into L2 while they
// compute.  k_post uses it for batched launches (many waves: 624 -> 536 us
// at 16 right-hand sides on 128^3); at one right-hand side (two waves) it
// cost 2 us, and the launch passes pf = 0.
__device__ __forceinline__ bool ahead_elem(int pf, int R, int W, int slot, int64_t m, int64_t* e2, int* r2) {
  if (pf <= 0) return false;
  const unsigned b = blockIdx.x + (unsigned)pf;
  if (b >= gridDim.x) return false;
  *r2 = (int)(b % (unsigned)R);
  *e2 = (int64_t)(b / (unsigned)R) * W + slot;
  return *e2 < m;
}

// The staging helpers below are run by the NT threads of an element (lane =
// the thread's index among them).

// one element's chunk of an array; 16-byte copies when the chunk allows it
template <int NT = 32, typename V, typename G>
__device__ __forceinline__ void w_cp_array(V* dst, const V* __restrict__ src, const G& g, int lane) {
  if ((g.nb * (int)sizeof(V)) % 16 == 0) {
    constexpr int per = 16 / sizeof(V);
#pragma unroll
    for (int i = 0; i < (g.nb / per + NT - 1) / NT; ++i) {
      const int k = lane + NT * i;
      if (k < g.nb / per) cp_async_16(dst + k * per, src + k * per);
    }
  } else {
    for (int i = lane; i < g.nb; i += NT) cp_async_elem(dst + i, src + i);
  }
}

// element interior into the padded tile
template <int NT = 32, typename V, typename G>
__device__ __forceinline__ void w_cp_padded(V* tile, const V* __restrict__ src, const G& g, int lane) {
#pragma unroll
  for (int i = 0; i < (g.nb + NT - 1) / NT; ++i) {
    const int c = lane + NT * i;
    if (c < g.nb) {
      const int lx = c % g.bx, t = c / g.bx;
      cp_async_elem(tile + wpad(g, lx, t % g.by, t / g.by), src + c);
    }
  }
}

// face halo f of X into the padded tile (zero on the domain boundary)
template <int NT = 32, typename V, typename G>
__device__ __forceinline__ void w_cp_face(V* tile, const V* __restrict__ X, const WElem& E, const G& g, int lane,
                                          int f) {
  const int d = f >> 1;
  const bool plus = f & 1;
  const int F = d == 0 ? g.by * g.bz : (d == 1 ? g.bx * g.bz : g.bx * g.by);
  const int64_t nb = E.nb6[f];
  for (int h = lane; h < F; h += NT) {
    int dx, dy, dz, sx, sy, sz;
    if (d == 0) { const int uu = h % g.by, vv = h / g.by; dy = sy = uu; dz = sz = vv; dx = plus ? g.bx : -1; sx = plus ? 0 : g.bx - 1; }
    else if (d == 1) { const int uu = h % g.bx, vv = h / g.bx; dx = sx = uu; dz = sz = vv; dy = plus ? g.by : -1; sy = plus ? 0 : g.by - 1; }
    else { const int uu = h % g.bx, vv = h / g.bx; dx = sx = uu; dy = sy = vv; dz = plus ? g.bz : -1; sz = plus ? 0 : g.bz - 1; }
    V* dst = tile + wpad(g, dx, dy, dz);
    if (nb >= 0) cp_async_elem(dst, X + nb + sx + g.bx * (sy + g.by * sz));
    else *dst = (V)0;
  }
}

template <int NT = 32, typename V, typename G>
__device__ __forceinline__ void w_cp_halo(V* tile, const V* __restrict__ X, const WElem& E, const G& g, int lane) {
#pragma unroll
  for (int f = 0; f < 6; ++f) w_cp_face<NT>(tile, X, E, g, lane, f);
}

// coefficients of the element's -d boundary faces (held by the -d neighbour)
template <int NT = 32, typename V, typename G>
__device__ __forceinline__ void w_cp_tminus(V* tm0, V* tm1, V* tm2, const V* __restrict__ T, int64_t n,
                                            const WElem& E, const G& g, int lane) {
  for (int h = lane; h < g.by * g.bz; h += NT) {          // (ly, lz) = h, source lx = bx - 1
    const int64_t nb = E.nb6[0];
    if (nb >= 0) cp_async_elem(tm0 + h, T + nb + (g.bx - 1) + g.bx * h);
    else tm0[h] = (V)0;
  }
  for (int h = lane; h < g.bx * g.bz; h += NT) {          // (lx, lz), source ly = by - 1
    const int64_t nb = E.nb6[2];
    const int lx = h % g.bx, lz = h / g.bx;
    if (nb >= 0) cp_async_elem(tm1 + h, T + n + nb + lx + g.bx * ((g.by - 1) + g.by * lz));
    else tm1[h] = (V)0;
  }
  for (int h = lane; h < g.bx * g.by; h += NT) {          // (lx, ly), source lz = bz - 1
    const int64_t nb = E.nb6[4];
    if (nb >= 0) cp_async_elem(tm2 + h, T + 2 * n + nb + h + g.bx * g.by * (g.bz - 1));
    else tm2[h] = (V)0;
  }
}

// per-warp shared-memory carve of the staged working set; each kernel carves
// only what it uses (more warps fit on an SM):
//   kStageFull      u tile with halo, T, 1/d, y, -d face coefficients (k_post)
//   kStagePre       T, 1/d, y                                     (k_pre)
//   kStageRestrict  u tile with halo                              (k_restrict FP32,
//                   which reads its face coefficients into registers)
//   kStageRestrictT u tile with halo, T, -d face coefficients     (k_restrict FP64,
//                   register-bound with the coefficients in registers)
template <typename V>
struct WStage {
  V *ut, *t0, *t1, *t2, *tm0, *tm1, *tm2, *dinv, *y;
};
template <typename V>
__host__ __device__ constexpr int restrict_layout() { return sizeof(V) == 8 ? kStageRestrictT : kStageRestrict; }
// Elements per CTA of the staged kernels: the CTA size that keeps the most
// elements resident per SM for the staging footprint of an 8^3 element (FP32:
// 10 KB for k_pre, 4 KB for k_restrict, 15 KB for k_post; FP64 twice that),
// which also sets how many elements one wave covers.
template <int LAYOUT, typename V, typename G = GeoR>
__host__ __device__ constexpr int stage_elems() {
  if (elem_threads<LAYOUT, G, V>() > 32) return 1;
  if (LAYOUT == kStageRestrict) return 4;
  if (LAYOUT == kStageRestrictT) return 2;
  if (sizeof(V) == 4) return LAYOUT == kStageFull ? 2 : 4;
  return LAYOUT == kStageFull ? 1 : 2;
}
// CTAs per SM the shared memory allows for k_post on 8^3 elements: the
// register cap that keeps them all resident; 0 leaves the register count to
// the compiler (an explicit minimum of 1 makes it take far more registers).
template <int LAYOUT, typename V, typename G>
__host__ __device__ constexpr int stage_min_ctas() {
  if (!IsCube8<G>::value || LAYOUT != kStageFull) return 0;
  return 7;
}
__host__ __device__ constexpr int r4(int x) { return (x + 3) / 4 * 4; }
template <int LAYOUT, typename G>
__host__ __device__ inline int wstage_elems(const G& g) {
  if (LAYOUT == kStageRestrict) return r4(g.P);
  const int tut = LAYOUT == kStagePre ? 0 : r4(g.P);
  const int nv = LAYOUT == kStageRestrictT ? 3 : 5;
  const int tm = LAYOUT == kStagePre ? 0 : r4(g.by * g.bz) + r4(g.bx * g.bz) + r4(g.bx * g.by);
  return tut + nv * r4(g.nb) + tm;
}
template <typename V, int LAYOUT = kStageFull, typename G>
__device__ __forceinline__ WStage<V> w_stage(unsigned char* base, const G& g, int warp) {
  V* p = reinterpret_cast<V*>(base) + (size_t)warp * wstage_elems<LAYOUT>(g);
  WStage<V> s;
  s.ut = nullptr;
  s.dinv = nullptr;
  s.y = nullptr;
  if (LAYOUT != kStagePre) { s.ut = p; p += r4(g.P); }
  s.t0 = p; p += r4(g.nb);
  s.t1 = p; p += r4(g.nb);
  s.t2 = p; p += r4(g.nb);
  if (LAYOUT != kStageRestrictT) {
    s.dinv = p; p += r4(g.nb);
    s.y = p; p += r4(g.nb);
  }
  if (LAYOUT == kStagePre) {   // k_pre's sweeps use no halo coefficients
    s.tm0 = s.tm1 = s.tm2 = nullptr;
    return s;
  }
  s.tm0 = p; p += r4(g.by * g.bz);
  s.tm1 = p; p += r4(g.bx * g.bz);
  s.tm2 = p;
  return s;
}

template <typename V, typename G>
__device__ __forceinline__ void w_stage_T(const WStage<V>& s, const V* __restrict__ T, const V* __restrict__ invd,
                                          int64_t n, const WElem& E, const G& g, int lane, bool with_dinv) {
  w_cp_array(s.t0, T + E.base, g, lane);
  w_cp_array(s.t1, T + n + E.base, g, lane);
  w_cp_array(s.t2, T + 2 * n + E.base, g, lane);
  if (with_dinv) w_cp_array(s.dinv, invd + E.base, g, lane);
  w_cp_tminus(s.tm0, s.tm1, s.tm2, T, n, E, g, lane);
}

// The same with the four in-element arrays (T[0..2], 1/d) as bulk copies on the
// element's mbarrier ``bar`` (its thread 0 issues them) where their size
// allows, the -d halo coefficients (gathered from three neighbours) by
// per-thread copies when asked for.  Returns whether the caller must wait on
// ``bar`` (phase 0).
template <int NT, typename V, typename G>
__device__ __forceinline__ bool w_stage_T_bulk(const WStage<V>& s, const V* __restrict__ T,
                                               const V* __restrict__ invd, int64_t n, const WElem& E, const G& g,
                                               int lane, unsigned bar, bool with_tm) {
  const bool bulk = (g.nb * (int)sizeof(V)) % 16 == 0;
  if (bulk) {
    if (lane == 0) {
      const unsigned bytes = (unsigned)(g.nb * sizeof(V));
      mbar_init(bar, 1);
      mbar_expect_tx(bar, 4 * bytes);
      bulk_g2s(s.t0, T + E.base, bytes, bar);
      bulk_g2s(s.t1, T + n + E.base, bytes, bar);
      bulk_g2s(s.t2, T + 2 * n + E.base, bytes, bar);
      bulk_g2s(s.dinv, invd + E.base, bytes, bar);
    }
    // the other threads poll the barrier only after thread 0 initialised it
    ebar<NT>();
  } else {
    w_cp_array<NT>(s.t0, T + E.base, g, lane);
    w_cp_array<NT>(s.t1, T + n + E.base, g, lane);
    w_cp_array<NT>(s.t2, T + 2 * n + E.base, g, lane);
    w_cp_array<NT>(s.dinv, invd + E.base, g, lane);
  }
  if (with_tm) w_cp_tminus<NT>(s.tm0, s.tm1, s.tm2, T, n, E, g, lane);
  return bulk;
}

// (A u)_c from the staged tiles
template <typename V, typename G>
__device__ __forceinline__ V w_apply_A_s(const WStage<V>& s, const G& g, int c) {
  const int lx = c % g.bx, t = c / g.bx, ly = t % g.by, lz = t / g.by;
  const int pc = wpad(g, lx, ly, lz);
  const int sy = g.bx + 2, sz = (g.bx + 2) * (g.by + 2);
  const V* ut = s.ut;
  const V uc = ut[pc];
  const V mx = lx > 0 ? s.t0[c - 1] : s.tm0[ly + g.by * lz];
  const V my = ly > 0 ? s.t1[c - g.bx] : s.tm1[lx + g.bx * lz];
  const V mz = lz > 0 ? s.t2[c - g.bx * g.by] : s.tm2[lx + g.bx * ly];
  V acc = s.t0[c] * (uc - ut[pc + 1]) + mx * (uc - ut[pc - 1]);
  acc += s.t1[c] * (uc - ut[pc + sy]) + my * (uc - ut[pc - sy]);
  acc += s.t2[c] * (uc - ut[pc + sz]) + mz * (uc - ut[pc - sz]);
  return acc;
}

// The cell term of A (wells) times u_c from the staged tile; 0 without one.
template <typename V, typename G>
__device__ __forceinline__ V w_cell_term(const V* __restrict__ Wd, int64_t base, const V* ut, const G& g, int c) {
  if (!Wd) return (V)0;
  const int lx = c % g.bx, t = c / g.bx;
  return __ldg(Wd + base + c) * ut[wpad(g, lx, t % g.by, t / g.by)];
}

// Cells of an 8^3 element by hyperplane lx + ly + lz = w (w = 0 .. 21), each plane in
// (lz, ly) order; off[w] is the first entry of plane w.  With these, a warp
// gives every lane at most two cells of the current plane (30 warp-steps per
// sweep instead of 44 with two fixed x-lines per lane).
struct Plane8 {
  unsigned short cell[512];
  unsigned short off[23];
};
constexpr Plane8 make_plane8() {
  Plane8 p{};
  int k = 0;
  for (int w = 0; w <= 21; ++w) {
    p.off[w] = (unsigned short)k;
    for (int lz = 0; lz < 8; ++lz)
      for (int ly = 0; ly < 8; ++ly) {
        const int lx = w - ly - lz;
        if (lx >= 0 && lx < 8) p.cell[k++] = (unsigned short)(lx + 8 * ly + 64 * lz);
      }
  }
  p.off[22] = (unsigned short)k;
  return p;
}
__device__ const Plane8 kPlane8 = make_plane8();

// Which sweep a kernel runs on 8^3 elements: the plane table (k_pre, and the
// FP64 k_post) or the unrolled fixed lines (the FP32 k_post, where it measured
// faster).  The table is read at every wavefront step, so each CTA keeps a
// copy in shared memory (after the elements' staging areas): a global read
// there would queue behind the kernel's outstanding loads.
template <int LAYOUT, typename V, typename G>
__host__ __device__ constexpr bool plane_sweeps() {
  return IsCube8<G>::value && (LAYOUT == kStagePre || (LAYOUT == kStageFull && sizeof(V) == 8));
}
constexpr int kPlaneShorts = 512 + 23;
constexpr size_t kPlaneSmemBytes = 1088;

// copy the table (all threads of the CTA; ends with a CTA barrier); returns it
template <bool TABLE>
__device__ __forceinline__ const unsigned short* w_plane_table(unsigned char* at) {
  if constexpr (TABLE) {
    unsigned short* t = reinterpret_cast<unsigned short*>(at);
    const unsigned short* src = reinterpret_cast<const unsigned short*>(&kPlane8);
    for (int i = threadIdx.x; i < kPlaneShorts; i += blockDim.x) t[i] = src[i];
    __syncthreads();
    return t;
  }
  return nullptr;
}

// y <- M^{-1} y from the staged tiles, M = (D~ + L) D~^{-1} (D~ + L^T):
// forward then backward wavefronts lx + ly + lz = w, run by the element's NT
// threads.  With the table (8^3 elements): the cells of each plane are dealt
// to the threads.  Otherwise thread l owns the x-lines l, l + NT, ... (line =
// ly + by * lz), so at wavefront w it updates cell lx = w - ly - lz of each of
// its lines; on 8^3 elements the 22 wavefronts are unrolled, which makes every
// address an immediate offset from the line's base (cell = 7 ly + 63 lz + w),
// and the x-neighbour is the value the thread produced at the previous
// wavefront (kept in a register).  The arithmetic per cell is the same in all
// forms.
template <int NT, bool TABLE, typename V, typename G>
__device__ __forceinline__ void w_ic0_s(const WStage<V>& s, const G& g, int lane, const unsigned short* tab) {
  V* y = s.y;
  if constexpr (TABLE) {
    const unsigned short* cell = tab;
    const unsigned short* off = tab + 512;
    for (int w = 0; w <= 21; ++w) {
      const int o0 = off[w], o1 = off[w + 1];
#pragma unroll
      for (int j = 0; j < (48 + NT - 1) / NT; ++j) {
        const int k = o0 + lane + NT * j;
        if (k >= o1) continue;
        const int c = cell[k];
        const int lx = c & 7, ly = (c >> 3) & 7, lz = c >> 6;
        V acc = y[c];
        if (lx > 0) acc += s.t0[c - 1] * y[c - 1];
        if (ly > 0) acc += s.t1[c - 8] * y[c - 8];
        if (lz > 0) acc += s.t2[c - 64] * y[c - 64];
        y[c] = acc * s.dinv[c];
      }
      ebar<NT>();
    }
    for (int w = 21; w >= 0; --w) {
      const int o0 = off[w], o1 = off[w + 1];
#pragma unroll
      for (int j = 0; j < (48 + NT - 1) / NT; ++j) {
        const int k = o0 + lane + NT * j;
        if (k >= o1) continue;
        const int c = cell[k];
        const int lx = c & 7, ly = (c >> 3) & 7, lz = c >> 6;
        V acc = (V)0;
        if (lx < 7) acc += s.t0[c] * y[c + 1];
        if (ly < 7) acc += s.t1[c] * y[c + 8];
        if (lz < 7) acc += s.t2[c] * y[c + 64];
        y[c] += s.dinv[c] * acc;
      }
      ebar<NT>();
    }
    return;
  } else if constexpr (IsCube8<G>::value) {
    constexpr int LPT = 64 / NT;              // lines per thread
    int base[LPT], off[LPT];
    bool hy[LPT], hz[LPT], ty[LPT], tz[LPT];
    V prev[LPT];
#pragma unroll
    for (int j = 0; j < LPT; ++j) {
      const int l = lane + NT * j, ly = l & 7, lz = l >> 3;
      base[j] = 7 * ly + 63 * lz;
      off[j] = ly + lz;
      hy[j] = ly > 0;
      hz[j] = lz > 0;
      ty[j] = ly < 7;
      tz[j] = lz < 7;
      prev[j] = (V)0;
    }
#pragma unroll
    for (int w = 0; w <= 21; ++w) {
#pragma unroll
      for (int j = 0; j < LPT; ++j) {
        const int lx = w - off[j];
        if ((unsigned)lx < 8u) {
          const int c = base[j] + w;
          V acc = y[c];
          if (lx > 0) acc += s.t0[c - 1] * prev[j];
          if (hy[j]) acc += s.t1[c - 8] * y[c - 8];
          if (hz[j]) acc += s.t2[c - 64] * y[c - 64];
          acc = acc * s.dinv[c];
          y[c] = acc;
          prev[j] = acc;
        }
      }
      ebar<NT>();
    }
#pragma unroll
    for (int w = 21; w >= 0; --w) {
#pragma unroll
      for (int j = 0; j < LPT; ++j) {
        const int lx = w - off[j];
        if ((unsigned)lx < 8u) {
          const int c = base[j] + w;
          V acc = (V)0;
          if (lx < 7) acc += s.t0[c] * prev[j];
          if (ty[j]) acc += s.t1[c] * y[c + 8];
          if (tz[j]) acc += s.t2[c] * y[c + 64];
          const V v = y[c] + s.dinv[c] * acc;
          y[c] = v;
          prev[j] = v;
        }
      }
      ebar<NT>();
    }
    return;
  }
  const int smax = g.bx + g.by + g.bz - 3;
  const int bxy = g.bx * g.by;
  for (int w = 0; w <= smax; ++w) {
#pragma unroll
    for (int i = 0; i < (g.nlines + NT - 1) / NT; ++i) {
      const int l = lane + NT * i;
      if (l >= g.nlines) continue;
      const int ly = l % g.by, lz = l / g.by;
      const int lx = w - ly - lz;
      if (lx < 0 || lx >= g.bx) continue;
      const int c = lx + g.bx * ly + bxy * lz;
      V acc = y[c];
      if (lx > 0) acc += s.t0[c - 1] * y[c - 1];
      if (ly > 0) acc += s.t1[c - g.bx] * y[c - g.bx];
      if (lz > 0) acc += s.t2[c - bxy] * y[c - bxy];
      y[c] = acc * s.dinv[c];
    }
    ebar<NT>();
  }
  for (int w = smax; w >= 0; --w) {
#pragma unroll
    for (int i = 0; i < (g.nlines + NT - 1) / NT; ++i) {
      const int l = lane + NT * i;
      if (l >= g.nlines) continue;
      const int ly = l % g.by, lz = l / g.by;
      const int lx = w - ly - lz;
      if (lx < 0 || lx >= g.bx) continue;
      const int c = lx + g.bx * ly + bxy * lz;
      V acc = (V)0;
      if (lx < g.bx - 1) acc += s.t0[c] * y[c + 1];
      if (ly < g.by - 1) acc += s.t1[c] * y[c + g.bx];
      if (lz < g.bz - 1) acc += s.t2[c] * y[c + bxy];
      y[c] += s.dinv[c] * acc;
    }
    ebar<NT>();
  }
}

// ------------------------------------------------------------------ k_pre
// update != 0: x += alpha p, r -= alpha q, rr = r.r (convergence bookkeeping);
// then f = r (in V precision, also written to rv) and u = M^{-1} f.
template <typename V, typename G>
__global__ void __launch_bounds__(stage_elems<kStagePre, V, G>() * elem_threads<kStagePre, G, V>(),
                                  stage_min_ctas<kStagePre, V, G>()) k_pre(double* __restrict__ x, double* __restrict__ r,
                                                           const double* __restrict__ p, const double* __restrict__ q,
                                                           const V* __restrict__ T, const V* __restrict__ invd,
                                                           V* __restrict__ rv, V* __restrict__ u, int64_t n, G g,
                                                           int64_t m, const int* __restrict__ nbr, int update,
                                                           RedSlot red, PcgScalars* sc, int* err, int R) {
  const BatchIdx bi = batch_idx(R);
  if (sc) sc += bi.r;
  if (sc && sc->done) return;
  {
    const int64_t off = (int64_t)bi.r * n;
    x += off; r += off; p += off; q += off; rv += off; u += off;
  }
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NT = elem_threads<kStagePre, G, V>();
  const int lane = threadIdx.x % NT, slot = threadIdx.x / NT;   // thread in the element, element in the CTA
  constexpr int W = stage_elems<kStagePre, V, G>();
  static_assert(NT == 32 || W == 1, "a two-warp element is a CTA of its own");
  const int64_t e = (int64_t)bi.blk * W + slot;
  const bool act = e < m;
  const WStage<V> s = w_stage<V, kStagePre>(smem, g, slot);
  __shared__ __align__(8) unsigned long long s_bar[W];   // one mbarrier per element
  const unsigned bar = (unsigned)__cvta_generic_to_shared(&s_bar[slot]);
  constexpr bool TABLE = plane_sweeps<kStagePre, V, G>();
  const unsigned short* tab = w_plane_table<TABLE>(smem + (size_t)W * wstage_elems<kStagePre>(g) * sizeof(V));
  double acc = 0.0;
  if (act) {
    const WElem E = w_elem(e, nbr, g);
    // the element's face coefficients and inverse pivots (the sweeps use no
    // halo coefficients)
    const bool bulk = w_stage_T_bulk<NT>(s, T, invd, n, E, g, lane, bar, false);
    const double alpha = update ? sc->alpha : 0.0;
    const int64_t base = E.base;
    // batches of kB cells per thread: all loads of a batch are issued before use
    constexpr int kB = NT == 64 ? 4 : 8;
    const int ncl = (g.nb + NT - 1) / NT;
    for (int b0 = 0; b0 < ncl; b0 += kB) {
      double rr[kB], qq[kB], xx[kB], pp[kB];
#pragma unroll
      for (int i = 0; i < kB; ++i) {
        const int c = lane + NT * (b0 + i);
        const bool in = b0 + i < ncl && c < g.nb;
        rr[i] = in ? r[base + c] : 0.0;
        qq[i] = (in && update) ? q[base + c] : 0.0;
        xx[i] = (in && update) ? x[base + c] : 0.0;
        pp[i] = (in && update) ? p[base + c] : 0.0;
      }
#pragma unroll
      for (int i = 0; i < kB; ++i) {
        const int c = lane + NT * (b0 + i);
        if (!(b0 + i < ncl && c < g.nb)) continue;
        double rc = rr[i];
        if (update) {
          x[base + c] = fma(alpha, pp[i], xx[i]);
          rc = fma(-alpha, qq[i], rc);
          r[base + c] = rc;
          acc = fma(rc, rc, acc);
        }
        V fv;
        if constexpr (std::is_same<V, float>::value) fv = f32_of_f64_rn(rc);   // integer pipes
        else fv = rc;
        s.y[c] = fv;
        rv[base + c] = fv;
      }
    }
    cp_async_wait_all();
    do {   // left early when the staged data never landed
    if (!bulk_landed<NT>(bulk, bar, sc, err, lane)) break;
    w_ic0_s<NT, TABLE>(s, g, lane, tab);
#pragma unroll 4
    for (int i = 0; i < (g.nb + NT - 1) / NT; ++i) {
      const int c = lane + NT * i;
      if (c < g.nb) u[base + c] = s.y[c];
    }
    } while (0);
  }
  if (update) {
    double v[1] = {acc};
    grid_reduce_r<1>(v, red, bi, [=] __device__(double* t) {
      sc->rr = t[0];
      sc->iter += 1;
      if (sc->done != 0) return;   // a warp of this launch already stopped the solve
      if (!isfinite(t[0])) sc->done = 2;
      else if (t[0] <= sc->tol2) sc->done = 1;
      else if (sc->iter >= sc->max_iter) sc->done = 3;
    });
  }
}

// ------------------------------------------------------------------ k_restrict
// Residual in registers (each lane's cells), then one warp reduction per local
// eigenvector.  Only the u tile is staged (4 KB per warp in FP32): the face
// coefficients of a group of cells are read straight into registers, so seven
// CTAs of four warps fit on an SM and the 4096 elements of a 128^3 grid take
// one wave.  The basis loads of all eigenvectors are issued cell by cell into
// L accumulators (the sum over each eigenvector's cells keeps its order).
template <typename V, typename BT, typename G>
__global__ void __launch_bounds__(stage_elems<restrict_layout<V>(), V>() * 32, sizeof(V) == 4 ? 7 : 1)
    k_restrict(const V* __restrict__ f, const V* __restrict__ u, const V* __restrict__ T, const V* __restrict__ Wd,
               const BT* __restrict__ Phi, int L, double* __restrict__ rc, int64_t nc, int64_t n, G g, int64_t m,
               const int* __restrict__ nbr, const PcgScalars* sc, int R, int pf) {
  const BatchIdx bi = batch_idx(R);
  if (sc) sc += bi.r;
  if (sc && sc->done) return;
  f += (int64_t)bi.r * n;
  u += (int64_t)bi.r * n;
  rc += (int64_t)bi.r * nc;
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int kC = 16;                                   // cells per lane held in registers
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int LAY = restrict_layout<V>();
  const int64_t e = (int64_t)bi.blk * stage_elems<LAY, V>() + warp;
  if (e >= m) return;
  const WStage<V> s = w_stage<V, kStageRestrictT>(smem, g, warp);   // used in the FP64 layout only
  V* ut = LAY == kStageRestrictT ? s.ut : reinterpret_cast<V*>(smem) + (size_t)warp * r4(g.P);
  const WElem E = w_elem(e, nbr, g);
  if (pf && lane == 0 && (g.nb * (int)sizeof(V)) % 16 == 0) {
    // the element's later loads into L2 now: batched launches (many waves) 215 -> 192 us
    // at 16 right-hand sides on 128^3; at one right-hand side (one wave) it cost 3 us
    const unsigned bv = (unsigned)(g.nb * sizeof(V));
    l2_prefetch(Phi + (size_t)e * L * g.nb, (unsigned)(L * g.nb * sizeof(BT)));
    l2_prefetch(T + E.base, bv);
    l2_prefetch(T + n + E.base, bv);
    l2_prefetch(T + 2 * n + E.base, bv);
    l2_prefetch(f + E.base, bv);
  }
  w_cp_padded(ut, u + E.base, g, lane);
  w_cp_halo(ut, u, E, g, lane);
  if constexpr (LAY == kStageRestrictT) w_stage_T(s, T, (const V*)nullptr, n, E, g, lane, false);
  const int ncl = (g.nb + 31) / 32;            // <= kC: elements have at most 512 cells
  const int bxy = g.bx * g.by;
  const int sy = g.bx + 2, sz = (g.bx + 2) * (g.by + 2);
  V w[kC];
#pragma unroll
  for (int i = 0; i < kC; ++i) {
    const int c = lane + 32 * i;
    w[i] = (i < ncl && c < g.nb) ? __ldg(f + E.base + c) : (V)0;
  }
  cp_async_wait_all();
  __syncwarp();
  if constexpr (LAY == kStageRestrictT) {
#pragma unroll
    for (int i = 0; i < kC; ++i) {
      const int c = lane + 32 * i;
      if (i < ncl && c < g.nb) w[i] -= w_apply_A_s(s, g, c) + w_cell_term(Wd, E.base, ut, g, c);
    }
  } else {
  // w -= A u: the six face coefficients of kG cells loaded before the products
  // (-d faces on the element boundary are held by the -d neighbour)
  constexpr int kG = 2;
#pragma unroll
  for (int i0 = 0; i0 < kC; i0 += kG) {
    V t0[kG], t1[kG], t2[kG], mx[kG], my[kG], mz[kG];
#pragma unroll
    for (int j = 0; j < kG; ++j) {
      const int c = lane + 32 * (i0 + j);
      t0[j] = t1[j] = t2[j] = mx[j] = my[j] = mz[j] = (V)0;
      if (!(i0 + j < ncl && c < g.nb)) continue;
      const int lx = c % g.bx, t = c / g.bx, ly = t % g.by, lz = t / g.by;
      t0[j] = __ldg(T + E.base + c);
      t1[j] = __ldg(T + n + E.base + c);
      t2[j] = __ldg(T + 2 * n + E.base + c);
      mx[j] = lx > 0 ? __ldg(T + E.base + c - 1) : (E.nb6[0] >= 0 ? __ldg(T + E.nb6[0] + c + g.bx - 1) : (V)0);
      my[j] = ly > 0 ? __ldg(T + n + E.base + c - g.bx)
                     : (E.nb6[2] >= 0 ? __ldg(T + n + E.nb6[2] + c + g.bx * (g.by - 1)) : (V)0);
      mz[j] = lz > 0 ? __ldg(T + 2 * n + E.base + c - bxy)
                     : (E.nb6[4] >= 0 ? __ldg(T + 2 * n + E.nb6[4] + c + bxy * (g.bz - 1)) : (V)0);
    }
#pragma unroll
    for (int j = 0; j < kG; ++j) {
      const int c = lane + 32 * (i0 + j);
      if (!(i0 + j < ncl && c < g.nb)) continue;
      const int lx = c % g.bx, t = c / g.bx;
      const int pc = wpad(g, lx, t % g.by, t / g.by);
      const V uc = ut[pc];
      V acc = t0[j] * (uc - ut[pc + 1]) + mx[j] * (uc - ut[pc - 1]);
      acc += t1[j] * (uc - ut[pc + sy]) + my[j] * (uc - ut[pc - sy]);
      acc += t2[j] * (uc - ut[pc + sz]) + mz[j] * (uc - ut[pc - sz]);
      if (Wd) acc += __ldg(Wd + E.base + c) * uc;   // cell term (wells)
      w[i0 + j] -= acc;
    }
  }
  }
  // rc_k = Phi_k . w, accumulated in the V-cycle precision (FP32 in the mixed
  // form: the FP64 pipe runs at 1/64 of the FP32 rate)
  const BT* ph = Phi + (size_t)e * L * g.nb;
  if (sizeof(V) == 4 && L <= kProlongLMax) {     // (FP64: one pass per eigenvector, fewer registers)
    V acc[kProlongLMax];
#pragma unroll
    for (int k = 0; k < kProlongLMax; ++k) acc[k] = (V)0;
#pragma unroll
    for (int i = 0; i < kC; ++i) {
      const int c = lane + 32 * i;
      if (!(i < ncl && c < g.nb)) continue;
#pragma unroll
      for (int k = 0; k < kProlongLMax; ++k)
        if (k < L) acc[k] += (V)__ldg(ph + (size_t)k * g.nb + c) * w[i];
    }
#pragma unroll
    for (int k = 0; k < kProlongLMax; ++k) {
      if (k >= L) break;
      const V a = warp_sum_t(acc[k]);
      if (lane == 0) rc[e * L + k] = (double)a;
    }
  } else {
    for (int k = 0; k < L; ++k) {
      V acc = (V)0;
#pragma unroll
      for (int i = 0; i < kC; ++i) {
        const int c = lane + 32 * i;
        if (i < ncl && c < g.nb) acc += (V)__ldg(ph + (size_t)k * g.nb + c) * w[i];
      }
      acc = warp_sum_t(acc);
      if (lane == 0) rc[e * L + k] = (double)acc;
    }
  }
}

// ------------------------------------------------------------------ prolongation
// Coarse correction (Algorithm 1, R_1^T e_c) added to the staged padded tile:
// the element's own cells and the face halo (cells of the six neighbours, with
// the neighbours' bases and coordinates).  Each cell's correction is
// sum_k Phi[ne][k][c] ec[ne][k], accumulated in the V-cycle precision in k
// order.  All L basis loads of a group of cells are issued before the first
// product (L <= kProlongLMax; larger L takes the plain loop).

template <typename V, typename BT>
__device__ __forceinline__ void w_corr_group(V* ut, const BT* __restrict__ ph, const V (&ev)[kProlongLMax], int L,
                                             int nb, const int (&src)[4], const int (&dst)[4], int cnt) {
  BT v[4][kProlongLMax];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int k = 0; k < kProlongLMax; ++k)
      if (j < cnt && k < L) v[j][k] = __ldg(ph + (size_t)k * nb + src[j]);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (j >= cnt) continue;
    V acc = (V)0;
#pragma unroll
    for (int k = 0; k < kProlongLMax; ++k)
      if (k < L) acc += (V)v[j][k] * ev[k];
    ut[dst[j]] += acc;
  }
}

template <typename V, typename BT>
__device__ __forceinline__ V w_coarse_corr(const BT* __restrict__ ph, const V* __restrict__ en, int L, int nb, int c) {
  V acc = (V)0;
  for (int k = 0; k < L; ++k) acc += (V)__ldg(ph + (size_t)k * nb + c) * __ldg(en + k);
  return acc;
}

template <int NT, typename V, typename BT, typename G>
__device__ __forceinline__ void w_prolong_tile(V* ut, const BT* __restrict__ Phi, const V* __restrict__ ec, int L,
                                               int64_t e, const WElem& E, const G& g, int lane) {
  if (L > kProlongLMax) {
    const V* en = ec + e * L;
    const BT* ph = Phi + (size_t)e * L * g.nb;
    for (int c = lane; c < g.nb; c += NT) {
      const int lx = c % g.bx, t = c / g.bx;
      ut[wpad(g, lx, t % g.by, t / g.by)] += w_coarse_corr(ph, en, L, g.nb, c);
    }
    for (int f = 0; f < 6; ++f) {
      const int64_t nbase = E.nb6[f];
      if (nbase < 0) continue;
      const int64_t ne = nbase / g.nb;
      const int d = f >> 1;
      const bool plus = f & 1;
      const int F = d == 0 ? g.by * g.bz : (d == 1 ? g.bx * g.bz : g.bx * g.by);
      for (int h = lane; h < F; h += NT) {
        int dx, dy, dz, sx, sy, sz;
        if (d == 0) { const int uu = h % g.by, vv = h / g.by; dy = sy = uu; dz = sz = vv; dx = plus ? g.bx : -1; sx = plus ? 0 : g.bx - 1; }
        else if (d == 1) { const int uu = h % g.bx, vv = h / g.bx; dx = sx = uu; dz = sz = vv; dy = plus ? g.by : -1; sy = plus ? 0 : g.by - 1; }
        else { const int uu = h % g.bx, vv = h / g.bx; dx = sx = uu; dy = sy = vv; dz = plus ? g.bz : -1; sz = plus ? 0 : g.bz - 1; }
        ut[wpad(g, dx, dy, dz)] += w_coarse_corr(Phi + (size_t)ne * L * g.nb, ec + ne * L, L, g.nb,
                                                 sx + g.bx * (sy + g.by * sz));
      }
    }
    return;
  }
  V ev[kProlongLMax];
#pragma unroll
  for (int k = 0; k < kProlongLMax; ++k) ev[k] = k < L ? ec[e * L + k] : (V)0;
  {
    const BT* ph = Phi + (size_t)e * L * g.nb;
    const int ncl = (g.nb + NT - 1) / NT;
    for (int i0 = 0; i0 < ncl; i0 += 4) {
      int src[4], dst[4];
      int cnt = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = lane + NT * (i0 + j);
        src[j] = c;
        dst[j] = 0;
        if (i0 + j < ncl && c < g.nb) {
          const int lx = c % g.bx, t = c / g.bx;
          dst[j] = wpad(g, lx, t % g.by, t / g.by);
          cnt = j + 1;
        }
      }
      w_corr_group(ut, ph, ev, L, g.nb, src, dst, cnt);
    }
  }
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    const int64_t nbase = E.nb6[f];
    if (nbase < 0) continue;
    const int64_t ne = nbase / g.nb;
#pragma unroll
    for (int k = 0; k < kProlongLMax; ++k) ev[k] = k < L ? ec[ne * L + k] : (V)0;
    const BT* pn = Phi + (size_t)ne * L * g.nb;
    const int d = f >> 1;
    const bool plus = f & 1;
    const int F = d == 0 ? g.by * g.bz : (d == 1 ? g.bx * g.bz : g.bx * g.by);
    for (int h0 = 0; h0 < F; h0 += 4 * NT) {
      int src[4], dst[4];
      int cnt = 0;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int h = h0 + lane + NT * j;
        src[j] = 0;
        dst[j] = 0;
        if (h < F) {
          int dx, dy, dz, sx, sy, sz;
          if (d == 0) { const int uu = h % g.by, vv = h / g.by; dy = sy = uu; dz = sz = vv; dx = plus ? g.bx : -1; sx = plus ? 0 : g.bx - 1; }
          else if (d == 1) { const int uu = h % g.bx, vv = h / g.bx; dx = sx = uu; dz = sz = vv; dy = plus ? g.by : -1; sy = plus ? 0 : g.by - 1; }
          else { const int uu = h % g.bx, vv = h / g.bx; dx = sx = uu; dy = sy = vv; dz = plus ? g.bz : -1; sz = plus ? 0 : g.bz - 1; }
          src[j] = sx + g.bx * (sy + g.by * sz);
          dst[j] = wpad(g, dx, dy, dz);
          cnt = j + 1;
        }
      }
      w_corr_group(ut, pn, ev, L, g.nb, src, dst, cnt);
    }
  }
}

// Separate prolongation: u_c += sum_k Phi[e][k][c] ec[e][k], a thread per cell,
// same accumulation order as the fused form.
template <typename V, typename BT, typename G>
__global__ void __launch_bounds__(256) k_prolong(V* __restrict__ u, const BT* __restrict__ Phi, int L,
                                                 const V* __restrict__ ec, int64_t n, int64_t nc, G g,
                                                 const PcgScalars* sc, int R) {
  const BatchIdx bi = batch_idx(R);
  if (sc) sc += bi.r;
  if (sc && sc->done) return;
  u += (int64_t)bi.r * n;
  ec += (int64_t)bi.r * nc;
  const int64_t i = (int64_t)bi.blk * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t e = i / g.nb;
  const int c = (int)(i - e * g.nb);
  const BT* ph = Phi + (size_t)e * L * g.nb + c;
  V acc = (V)0;
  if (L <= kProlongLMax) {
    BT v[kProlongLMax];
#pragma unroll
    for (int k = 0; k < kProlongLMax; ++k)
      if (k < L) v[k] = __ldg(ph + (size_t)k * g.nb);
#pragma unroll
    for (int k = 0; k < kProlongLMax; ++k)
      if (k < L) acc += (V)v[k] * __ldg(ec + e * L + k);
  } else {
    for (int k = 0; k < L; ++k) acc += (V)__ldg(ph + (size_t)k * g.nb) * __ldg(ec + e * L + k);
  }
  u[i] += acc;
}

// The same for FP32 vectors and bases, four consecutive cells of one element
// per thread (16-byte loads and stores; elements of a multiple of 4 cells):
// per cell the same products in the same order.
template <typename G>
__global__ void __launch_bounds__(256) k_prolong4(float* __restrict__ u, const float* __restrict__ Phi, int L,
                                                  const float* __restrict__ ec, int64_t n, int64_t nc, G g,
                                                  const PcgScalars* sc, int R) {
  const BatchIdx bi = batch_idx(R);
  if (sc) sc += bi.r;
  if (sc && sc->done) return;
  u += (int64_t)bi.r * n;
  ec += (int64_t)bi.r * nc;
  const int64_t i = ((int64_t)bi.blk * blockDim.x + threadIdx.x) * 4;
  if (i >= n) return;
  const int64_t e = i / g.nb;
  const int c = (int)(i - e * g.nb);
  const float* ph = Phi + (size_t)e * L * g.nb + c;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (L <= kProlongLMax) {
    float4 v[kProlongLMax];
    float ev[kProlongLMax];
#pragma unroll
    for (int k = 0; k < kProlongLMax; ++k)
      if (k < L) {
        v[k] = __ldg(reinterpret_cast<const float4*>(ph + (size_t)k * g.nb));
        ev[k] = __ldg(ec + e * L + k);
      }
#pragma unroll
    for (int k = 0; k < kProlongLMax; ++k)
      if (k < L) {
        acc.x += v[k].x * ev[k];
        acc.y += v[k].y * ev[k];
        acc.z += v[k].z * ev[k];
        acc.w += v[k].w * ev[k];
      }
  } else {
    for (int k = 0; k < L; ++k) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(ph + (size_t)k * g.nb));
      const float ek = __ldg(ec + e * L + k);
      acc.x += v.x * ek;
      acc.y += v.y * ek;
      acc.z += v.z * ek;
      acc.w += v.w * ek;
    }
  }
  float4* up = reinterpret_cast<float4*>(u + i);
  float4 uu = *up;
  uu.x += acc.x;
  uu.y += acc.y;
  uu.z += acc.z;
  uu.w += acc.w;
  *up = uu;
}

// ------------------------------------------------------------------ k_post
// z = u + M^{-1} (f - A u), written in FP64; reductions: r.z and z.q (flexible
// beta).  f, r and q are loaded into registers before the wavefronts start.
template <typename V, typename BT, typename G, bool FUSE>
__global__ void __launch_bounds__(stage_elems<kStageFull, V, G>() * elem_threads<kStageFull, G, V>(),
                                  stage_min_ctas<kStageFull, V, G>()) k_post(const V* __restrict__ f, const double* __restrict__ r,
                                                            const V* __restrict__ u, const V* __restrict__ T,
                                                            const V* __restrict__ Wd,
                                                            const V* __restrict__ invd, const BT* __restrict__ Phi,
                                                            const V* __restrict__ ec, int L, int64_t nc,
                                                            double* __restrict__ z, const double* __restrict__ qv,
                                                            int64_t n, G g, int64_t m, const int* __restrict__ nbr,
                                                            RedSlot red, PcgScalars* sc, int* err, int R, int pf) {
  const BatchIdx bi = batch_idx(R);
  if (sc) sc += bi.r;
  if (sc && sc->done) return;
  {
    const int64_t off = (int64_t)bi.r * n;
    f += off; r += off; u += off; z += off;
    if (qv) qv += off;
    ec += (int64_t)bi.r * nc;
  }
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NT = elem_threads<kStageFull, G, V>();
  constexpr int kC = 512 / NT;                 // cells per thread held in registers
  const int lane = threadIdx.x % NT, slot = threadIdx.x / NT;   // thread in the element, element in the CTA
  constexpr int W = stage_elems<kStageFull, V, G>();
  static_assert(NT == 32 || W == 1, "a two-warp element is a CTA of its own");
  const int64_t e = (int64_t)bi.blk * W + slot;
  const bool act = e < m;
  const WStage<V> s = w_stage<V>(smem, g, slot);
  __shared__ __align__(8) unsigned long long s_bar[W];   // one mbarrier per element
  const unsigned bar = (unsigned)__cvta_generic_to_shared(&s_bar[slot]);
  constexpr bool TABLE = plane_sweeps<kStageFull, V, G>();
  const unsigned short* tab = w_plane_table<TABLE>(smem + (size_t)W * wstage_elems<kStageFull>(g) * sizeof(V));
  const int ncl = (g.nb + NT - 1) / NT;
  double v[2] = {0.0, 0.0};
  if (act && ncl <= kC) {
    const WElem E = w_elem(e, nbr, g);
    const int64_t base = E.base;
    w_cp_padded<NT>(s.ut, u + base, g, lane);
    w_cp_halo<NT>(s.ut, u, E, g, lane);
    const bool bulk = w_stage_T_bulk<NT>(s, T, invd, n, E, g, lane, bar, true);
    cp_async_wait_all();
    do {   // left early when the staged data never landed
    if (!bulk_landed<NT>(bulk, bar, sc, err, lane)) break;
    {
      int64_t e2;
      int r2;
      if (lane == 0 && bulk && ahead_elem(pf, R, W, slot, m, &e2, &r2)) {
        const unsigned bv = (unsigned)(g.nb * sizeof(V)), bd = (unsigned)(g.nb * sizeof(double));
        const int64_t b2 = e2 * g.nb, o2 = (int64_t)(r2 - bi.r) * n + b2;
        l2_prefetch(T + b2, bv);
        l2_prefetch(T + n + b2, bv);
        l2_prefetch(T + 2 * n + b2, bv);
        l2_prefetch(invd + b2, bv);
        l2_prefetch(u + o2, bv);
        l2_prefetch(f + o2, bv);
        if (sc) l2_prefetch(r + o2, bd);
        if (qv) l2_prefetch(qv + o2, bd);
        if (FUSE) l2_prefetch(Phi + b2 * L, (unsigned)(L * g.nb * sizeof(BT)));
      }
    }
    if (FUSE) {
      w_prolong_tile<NT>(s.ut, Phi, ec, L, e, E, g, lane);
      ebar<NT>();
    }
    // The V-cycle's right-hand side f is r in V precision.  In FP64 that is r itself,
    // read once for both uses (182 -> 166 us on 128^3 with the other changes); in
    // FP32 the rounded copy k_pre stored is read (rounding r again here on the
    // integer pipes saved no time: the kernel waits on latency, not bytes).
    constexpr bool kFromR = sizeof(V) == 8;
    double rr[kC];
    {
      V fr[kC];
#pragma unroll
      for (int i = 0; i < kC; ++i) {
        const int c = lane + NT * i;
        const bool in = i < ncl && c < g.nb;
        if constexpr (kFromR) {
          rr[i] = in ? __ldg(r + base + c) : 0.0;
          fr[i] = (V)rr[i];
        } else {
          fr[i] = in ? __ldg(f + base + c) : (V)0;
        }
      }
#pragma unroll
      for (int i = 0; i < kC; ++i) {
        const int c = lane + NT * i;
        if (i < ncl && c < g.nb) s.y[c] = fr[i] - (w_apply_A_s(s, g, c) + w_cell_term(Wd, base, s.ut, g, c));
      }
    }
    // r (FP32 form) and q are needed only after the sweeps: their loads overlap them
    double qq[kC];
#pragma unroll
    for (int i = 0; i < kC; ++i) {
      const int c = lane + NT * i;
      const bool in = i < ncl && c < g.nb;
      if constexpr (!kFromR) rr[i] = (in && sc) ? __ldg(r + base + c) : 0.0;
      qq[i] = (in && qv) ? __ldg(qv + base + c) : 0.0;
    }
    ebar<NT>();
    w_ic0_s<NT, TABLE>(s, g, lane, tab);
#pragma unroll
    for (int i = 0; i < kC; ++i) {
      const int c = lane + NT * i;
      if (!(i < ncl && c < g.nb)) continue;
      const int lx = c % g.bx, t = c / g.bx;
      const V zv = s.ut[wpad(g, lx, t % g.by, t / g.by)] + s.y[c];
      double zc;
      if constexpr (std::is_same<V, float>::value) zc = f64_of_f32(zv);       // integer pipes
      else zc = zv;
      z[base + c] = zc;
      v[0] = fma(rr[i], zc, v[0]);
      v[1] = fma(zc, qq[i], v[1]);
    }
    } while (0);
  } else if (act) {
    const WElem E = w_elem(e, nbr, g);
    const int64_t base = E.base;
    w_cp_padded<NT>(s.ut, u + base, g, lane);
    w_cp_halo<NT>(s.ut, u, E, g, lane);
    const bool bulk = w_stage_T_bulk<NT>(s, T, invd, n, E, g, lane, bar, true);
    cp_async_wait_all();
    do {   // left early when the staged data never landed
    if (!bulk_landed<NT>(bulk, bar, sc, err, lane)) break;
    if (FUSE) {
      w_prolong_tile<NT>(s.ut, Phi, ec, L, e, E, g, lane);
      ebar<NT>();
    }
    for (int c = lane; c < g.nb; c += NT)
      s.y[c] = __ldg(f + base + c) - (w_apply_A_s(s, g, c) + w_cell_term(Wd, base, s.ut, g, c));
    ebar<NT>();
    w_ic0_s<NT, TABLE>(s, g, lane, tab);
    for (int c = lane; c < g.nb; c += NT) {
      const int lx = c % g.bx, t = c / g.bx;
      const double zc = (double)(s.ut[wpad(g, lx, t % g.by, t / g.by)] + s.y[c]);
      z[base + c] = zc;
      if (sc) {
        v[0] = fma(r[base + c], zc, v[0]);
        if (qv) v[1] = fma(zc, qv[base + c], v[1]);
      }
    }
    } while (0);
  }
  if (sc) {
    grid_reduce_r<2>(v, red, bi, [=] __device__(double* t) {
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
// FP64-rate bound on GB300, so it is built for residency: three warps per CTA
// (8 KB tile each) and at most 72 registers, nine CTAs per SM, 27 warps -- one
// wave for 4104 elements.
constexpr int kPmWarps = 3, kPmCtasPerSm = 9;
template <typename G>
__global__ void __launch_bounds__(kPmWarps * 32, kPmCtasPerSm) k_pmatvec(const double* __restrict__ z, const double* __restrict__ pold,
                                                               double* __restrict__ pnew, double* __restrict__ q,
                                                               const double* __restrict__ T,
                                                               const double* __restrict__ Dg, int64_t n, G g,
                                                               int64_t m, const int* __restrict__ nbr, RedSlot red,
                                                               PcgScalars* sc, int R) {
  const BatchIdx bi = batch_idx(R);
  sc += bi.r;
  if (sc->done) return;
  {
    const int64_t off = (int64_t)bi.r * n;
    z += off; pold += off; pnew += off; q += off;
  }
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t e = (int64_t)bi.blk * kPmWarps + warp;
  const bool act = e < m;
  double* ut = reinterpret_cast<double*>(smem) + (size_t)warp * r4(g.P);
  double acc = 0.0;
  if (act) {
    const double beta = sc->beta;
    const WElem E = w_elem(e, nbr, g);
    const int64_t base = E.base;
    constexpr int kC = 8;                        // cells per lane and batch
    const int ncl = (g.nb + 31) / 32;
    // p on the element: every load of a batch issued before the first use
    for (int i0 = 0; i0 < ncl; i0 += kC) {
      double zz[kC], po[kC];
#pragma unroll
      for (int i = 0; i < kC; ++i) {
        const int c = lane + 32 * (i0 + i);
        const bool in = i0 + i < ncl && c < g.nb;
        zz[i] = in ? __ldg(z + base + c) : 0.0;
        po[i] = in ? __ldg(pold + base + c) : 0.0;
      }
#pragma unroll
      for (int i = 0; i < kC; ++i) {
        const int c = lane + 32 * (i0 + i);
        if (!(i0 + i < ncl && c < g.nb)) continue;
        const double pv = fma(beta, po[i], zz[i]);
        const int lx = c % g.bx, t = c / g.bx;
        ut[wpad(g, lx, t % g.by, t / g.by)] = pv;
        pnew[base + c] = pv;
      }
    }
    // p on the face halo, recomputed from the neighbours' z and p_old
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      const int d = f >> 1;
      const bool plus = f & 1;
      const int F = d == 0 ? g.by * g.bz : (d == 1 ? g.bx * g.bz : g.bx * g.by);
      const int64_t nb = E.nb6[f];
      for (int h0 = 0; h0 < F; h0 += 64) {
        double zv[2], pv[2];
        int dst[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int h = h0 + lane + 32 * j;
          zv[j] = 0.0;
          pv[j] = 0.0;
          dst[j] = -1;
          if (h < F) {
            int dx, dy, dz, sx, sy, sz;
            if (d == 0) { const int uu = h % g.by, vv = h / g.by; dy = sy = uu; dz = sz = vv; dx = plus ? g.bx : -1; sx = plus ? 0 : g.bx - 1; }
            else if (d == 1) { const int uu = h % g.bx, vv = h / g.bx; dx = sx = uu; dz = sz = vv; dy = plus ? g.by : -1; sy = plus ? 0 : g.by - 1; }
            else { const int uu = h % g.bx, vv = h / g.bx; dx = sx = uu; dy = sy = vv; dz = plus ? g.bz : -1; sz = plus ? 0 : g.bz - 1; }
            dst[j] = wpad(g, dx, dy, dz);
            if (nb >= 0) {
              const int64_t src = nb + sx + g.bx * (sy + g.by * sz);
              zv[j] = __ldg(z + src);
              pv[j] = __ldg(pold + src);
            }
          }
        }
#pragma unroll
        for (int j = 0; j < 2; ++j)
          if (dst[j] >= 0) ut[dst[j]] = nb >= 0 ? fma(beta, pv[j], zv[j]) : 0.0;
      }
    }
    __syncwarp();
    const int sy = g.bx + 2, sz = (g.bx + 2) * (g.by + 2);
    // q = A p: coefficients of a group of kQ cells loaded before the products
    constexpr int kQ = 2;
    for (int i0 = 0; i0 < ncl; i0 += kQ) {
      double t0[kQ], t1[kQ], t2[kQ], dg[kQ], mx[kQ], my[kQ], mz[kQ];
#pragma unroll
      for (int j = 0; j < kQ; ++j) {
        const int c = lane + 32 * (i0 + j);
        t0[j] = t1[j] = t2[j] = dg[j] = mx[j] = my[j] = mz[j] = 0.0;
        if (!(i0 + j < ncl && c < g.nb)) continue;
        const int lx = c % g.bx, t = c / g.bx, ly = t % g.by, lz = t / g.by;
        t0[j] = __ldg(T + base + c);
        t1[j] = __ldg(T + n + base + c);
        t2[j] = __ldg(T + 2 * n + base + c);
        dg[j] = __ldg(Dg + base + c);
        // -d face coefficients: in-element, or held by the -d neighbour
        mx[j] = lx > 0 ? __ldg(T + base + c - 1) : (E.nb6[0] >= 0 ? __ldg(T + E.nb6[0] + c + g.bx - 1) : 0.0);
        my[j] = ly > 0 ? __ldg(T + n + base + c - g.bx)
                       : (E.nb6[2] >= 0 ? __ldg(T + n + E.nb6[2] + c + g.bx * (g.by - 1)) : 0.0);
        mz[j] = lz > 0 ? __ldg(T + 2 * n + base + c - g.bx * g.by)
                       : (E.nb6[4] >= 0 ? __ldg(T + 2 * n + E.nb6[4] + c + g.bx * g.by * (g.bz - 1)) : 0.0);
      }
#pragma unroll
      for (int j = 0; j < kQ; ++j) {
        const int c = lane + 32 * (i0 + j);
        if (!(i0 + j < ncl && c < g.nb)) continue;
        const int lx = c % g.bx, t = c / g.bx, ly = t % g.by, lz = t / g.by;
        const int pc = wpad(g, lx, ly, lz);
        const double pcv = ut[pc];
        // (A p)_c = D_c p_c - sum_f T_f p_nb: one multiply and six FMAs in FP64
        double a = dg[j] * pcv;
        a = fma(-t0[j], ut[pc + 1], a);
        a = fma(-mx[j], ut[pc - 1], a);
        a = fma(-t1[j], ut[pc + sy], a);
        a = fma(-my[j], ut[pc - sy], a);
        a = fma(-t2[j], ut[pc + sz], a);
        a = fma(-mz[j], ut[pc - sz], a);
        q[base + c] = a;
        acc = fma(a, pcv, acc);
      }
    }
  }
  double v[1] = {acc};
  grid_reduce_r<1>(v, red, bi, [=] __device__(double* t) {
    sc->pq = t[0];
    if (!(t[0] > 0.0) || !isfinite(t[0])) { sc->done = 2; sc->alpha = 0.0; }
    else sc->alpha = sc->rz / t[0];
  });
}

// ------------------------------------------------------------------ host side
template <typename V, typename BT>
struct FineOps {
  const V* T;
  const V* invd;
  const BT* Phi;
  const V* Wd;     // cell term (wells) or null
};

template <int LAYOUT, typename V, typename G>
static inline size_t wsmem(const G& g) {
  return (size_t)stage_elems<LAYOUT, V, G>() * wstage_elems<LAYOUT>(g) * sizeof(V) +
         (plane_sweeps<LAYOUT, V, G>() ? kPlaneSmemBytes : 0);
}
template <typename G>
static inline size_t wsmem_p(const G& g) {
  return (size_t)kPmWarps * r4(g.P) * sizeof(double);
}

// run f(geometry) with the compile-time geometry of the element when available
template <typename F>
static void with_geo(const msmg_ctx* c, F&& f) {
  const int bx = c->fine.bx, by = c->fine.by, bz = c->fine.bz;
  if (bx == 8 && by == 8 && bz == 8) f(GeoC<8, 8, 8>{});
  else if (bx == 4 && by == 4 && bz == 4) f(GeoC<4, 4, 4>{});
  else f(make_geor(bx, by, bz));
}

// CTAs of a batched fine-level launch: element groups x right-hand sides
static inline unsigned fine_wgrid(const msmg_ctx* c, int W = kWarpsPerCta) {
  return (unsigned)((c->fine.m + W - 1) / W * c->sb.R);
}

template <typename V, typename BT, typename G>
static void pre_t(msmg_ctx* c, const FineOps<V, BT>& o, int update, PcgScalars* sc, cudaStream_t s, const G& g) {
  SolveBuffers& B = c->sb;
  constexpr int W = stage_elems<kStagePre, V, G>();
  k_pre<V, G><<<fine_wgrid(c, W), W * elem_threads<kStagePre, G, V>(), wsmem<kStagePre, V>(g), s>>>(
      B.x, B.r, B.pcur, B.q, o.T, o.invd, (V*)B.rv, (V*)B.vu[1], c->n, g, c->fine.m, c->fine.nbr, update, c->red, sc,
      c->flags + 6, B.R);
}

template <typename V, typename BT, typename G>
static void restrict_t(msmg_ctx* c, const FineOps<V, BT>& o, PcgScalars* sc, cudaStream_t s, const G& g) {
  SolveBuffers& B = c->sb;
  constexpr int W = stage_elems<restrict_layout<V>(), V>();
  k_restrict<V, BT, G><<<fine_wgrid(c, W), W * 32, wsmem<restrict_layout<V>(), V>(g), s>>>(
      (const V*)B.rv, (const V*)B.vu[1], o.T, o.Wd, o.Phi, c->fine.L, (double*)B.vf[2], c->lev[2].n, c->n, g, c->fine.m,
      c->fine.nbr, sc, B.R, B.R > 1);
}

template <typename V, typename BT, typename G>
static void post_t(msmg_ctx* c, const FineOps<V, BT>& o, const V* ec, const double* qv, PcgScalars* sc,
                   cudaStream_t s, const G& g, bool fuse) {
  SolveBuffers& B = c->sb;
  constexpr int W = stage_elems<kStageFull, V, G>();
  constexpr int NT = elem_threads<kStageFull, G, V>();
  if (fuse)
    k_post<V, BT, G, true><<<fine_wgrid(c, W), W * NT, wsmem<kStageFull, V>(g), s>>>(
        (const V*)B.rv, B.r, (const V*)B.vu[1], o.T, o.Wd, o.invd, o.Phi, ec, c->fine.L, c->lev[2].n, B.z, qv, c->n, g,
        c->fine.m, c->fine.nbr, c->red, sc, c->flags + 6, B.R, B.R > 1 ? c->pf_post[1] : 0);
  else
    k_post<V, BT, G, false><<<fine_wgrid(c, W), W * NT, wsmem<kStageFull, V>(g), s>>>(
        (const V*)B.rv, B.r, (const V*)B.vu[1], o.T, o.Wd, o.invd, o.Phi, ec, c->fine.L, c->lev[2].n, B.z, qv, c->n, g,
        c->fine.m, c->fine.nbr, c->red, sc, c->flags + 6, B.R, B.R > 1 ? c->pf_post[0] : 0);
}

template <typename V, typename BT, typename G>
static void prolong_t(msmg_ctx* c, const FineOps<V, BT>& o, const V* ec, PcgScalars* sc, cudaStream_t s,
                      const G& g) {
  SolveBuffers& B = c->sb;
  if constexpr (std::is_same<V, float>::value && std::is_same<BT, float>::value) {
    if (c->fine.nb % 4 == 0) {
      const unsigned grid = (unsigned)((c->n / 4 + 255) / 256 * B.R);
      k_prolong4<G><<<grid, 256, 0, s>>>((float*)B.vu[1], o.Phi, c->fine.L, ec, c->n, c->lev[2].n, g, sc, B.R);
      return;
    }
  }
  const unsigned grid = (unsigned)((c->n + 255) / 256 * B.R);
  k_prolong<V, BT, G><<<grid, 256, 0, s>>>((V*)B.vu[1], o.Phi, c->fine.L, ec, c->n, c->lev[2].n, g, sc, B.R);
}

template <typename G>
static void pmatvec_t(msmg_ctx* c, PcgScalars* sc, cudaStream_t s, const G& g) {
  SolveBuffers& B = c->sb;
  k_pmatvec<G><<<fine_wgrid(c, kPmWarps), kPmWarps * 32, wsmem_p(g), s>>>(B.z, B.pcur, B.pnext, B.q, c->fine.T, c->fine.D,
                                                                      c->n, g, c->fine.m, c->fine.nbr, c->red, sc, B.R);
}


// Shared-memory limits of the fine-level kernels, set once per context (never
// during stream capture).
// CTAs of kernel k resident at once on the device (the launch's first wave)
static int resident_ctas(const void* k, int threads, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;   // no prefetch
  }
  return per * sms;
}

template <typename V, typename BT, typename G>
static void prepare_t(msmg_ctx* c, const G& g) {
  const int smv = (int)wsmem<kStageFull, V>(g), smd = (int)wsmem_p(g);
  cudaFuncSetAttribute(k_pre<V, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsmem<kStagePre, V>(g));
  cudaFuncSetAttribute(k_restrict<V, BT, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)wsmem<restrict_layout<V>(), V>(g));
  cudaFuncSetAttribute(k_restrict<V, BT, G>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(k_post<V, BT, G, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smv);
  cudaFuncSetAttribute(k_post<V, BT, G, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smv);
  cudaFuncSetAttribute(k_post<V, BT, G, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(k_post<V, BT, G, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  cudaFuncSetAttribute(k_pmatvec<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, smd);
  cudaFuncSetAttribute(k_pmatvec<G>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  constexpr int NT = elem_threads<kStageFull, G, V>();
  c->pf_post[0] = resident_ctas((const void*)k_post<V, BT, G, false>, stage_elems<kStageFull, V, G>() * NT, smv);
  c->pf_post[1] = resident_ctas((const void*)k_post<V, BT, G, true>, stage_elems<kStageFull, V, G>() * NT, smv);
}

void prepare_fine_kernels(msmg_ctx* c) {
  with_geo(c, [&](auto g) {
    if (c->opts.precision == MSMG_MIXED) prepare_t<float, float>(c, g);
    else prepare_t<double, double>(c, g);
  });
}

const void* coarse_cycle(msmg_ctx* c, int l, PcgScalars* sc, cudaStream_t s);

// Fine-level V-cycle on the residual held in B.r (FP64); result in B.z (FP64).
// update != 0 first performs the PCG update of x and r with the current alpha.
// With ev != nullptr, events ev[0..5] bracket the pieces (kernel timing).
template <typename V, typename BT>
static void vcycle_t(msmg_ctx* c, const FineOps<V, BT>& o, int update, const double* qv, PcgScalars* sc,
                     cudaStream_t s, cudaEvent_t* ev) {
  with_geo(c, [&](auto g) {
    if (ev) cudaEventRecord(ev[0], s);
    pre_t<V, BT>(c, o, update, sc, s, g);
    if (ev) cudaEventRecord(ev[1], s);
    restrict_t<V, BT>(c, o, sc, s, g);
    if (ev) cudaEventRecord(ev[2], s);
    const V* ec = (const V*)coarse_cycle(c, 2, sc, s);
    if (ev) cudaEventRecord(ev[3], s);
    // fused: the prolongation is part of k_post and the [3, 4] interval stays empty
    const bool fuse = c->tune_fused[c->sb.R > 1 ? 1 : 0] != 0;
    if (!fuse) prolong_t<V, BT>(c, o, ec, sc, s, g);
    if (ev) cudaEventRecord(ev[4], s);
    post_t<V, BT>(c, o, ec, qv, sc, s, g, fuse);
    if (ev) cudaEventRecord(ev[5], s);
  });
}

static void pcg_step_vcycle_ev(msmg_ctx* c, int update, const double* qv, PcgScalars* sc, cudaStream_t s,
                               cudaEvent_t* ev) {
  if (c->opts.precision == MSMG_MIXED) {
    FineOps<float, float> o{c->fine.T32, c->fine.invd32, c->fine.Phi32, c->fine.Wd32};
    vcycle_t<float, float>(c, o, update, qv, sc, s, ev);
  } else {
    FineOps<double, double> o{c->fine.T, c->fine.invd, c->fine.Phi, c->fine.Wd};
    vcycle_t<double, double>(c, o, update, qv, sc, s, ev);
  }
}

void pcg_step_vcycle(msmg_ctx* c, int update, const double* qv, PcgScalars* sc, cudaStream_t s) {
  pcg_step_vcycle_ev(c, update, qv, sc, s, nullptr);
}

void pcg_step_vcycle_timed(msmg_ctx* c, int update, const double* qv, PcgScalars* sc, cudaStream_t s,
                           cudaEvent_t* ev) {
  pcg_step_vcycle_ev(c, update, qv, sc, s, ev);
}

void pcg_step_pmatvec(msmg_ctx* c, PcgScalars* sc, cudaStream_t s) {
  with_geo(c, [&](auto g) { pmatvec_t(c, sc, s, g); });
}

// z = P^{-1} r in FP64 (natural order handled by the caller): r in B.r, result in B.z.
void apply_vcycle_fp64_out(msmg_ctx* c, cudaStream_t s) { pcg_step_vcycle(c, 0, nullptr, nullptr, s); }

}  // namespace msmg
