// Learned warm start for the level-1 local eigenproblems (Eq. (spepb)): a
// multilayer perceptron maps an element's standardised log-permeability patch
// to guesses for its eigenvectors 1 .. L-1 in the symmetric form
// y = S^{1/2} phi (eigenvector 0, the constant, is known exactly).  The guesses
// seed the subspace iteration, which still runs to the same eigen-residual
// tolerance, so the preconditioner is unchanged; only the set-up time moves.
//
// Network: x (n_in) -> relu(x W1 + b1) (h1) -> relu(. W2 + b2) (h2) -> o = . W3 + b3
// (n_vec * n_in) -> y_k = w * o_k.  The fixed output weighting
// w_c = sqrt(S_c / sum S), recovered from the input (S_c is proportional to
// exp(8 x_c)), makes the network predict the eigenvectors phi, which vary
// slowly across permeability jumps, while its output y = S^{1/2} phi stays in
// the symmetric form.  Weights are kept as FP32 masters (training, Adam) and
// BF16 copies that every product reads; activations and accumulation are FP32.
//
// Loss per sample and output vector k (sign-invariant: an eigenvector is only
// defined up to sign):  l = ||p||^2 + ||t||^2 - 2 |p . t|,  the smaller of
// ||p - t||^2 and ||p + t||^2;  the batch loss is the mean over samples and
// vectors.
//
// All kernels are deterministic (no atomics): a training run is reproducible.
#include "msmg_internal.cuh"
#include <cuda.h>
#include <cuda_bf16.h>
#include <new>

struct msmg_net {
  msmg_net_desc d;
  int n_out;                    // n_vec * n_in
  int64_t n_param;              // total parameters
  // parameter blocks inside one array: W1 [n_in][h1], b1, W2 [h1][h2], b2, W3 [h2][n_out], b3
  int64_t off_w[3], off_b[3];
  float* w32;                   // FP32 masters
  __nv_bfloat16* w16;           // BF16 copies (read by the products)
  float* grad;                  // gradients, same layout
  float* adam_m;
  float* adam_v;
  float* h1;                    // [batch_max][h1]
  float* h2;                    // [batch_max][h2]
  float* out;                   // [batch_max][n_out]
  float* d_out;                 // [batch_max][n_out]
  float* d_h2;                  // [batch_max][h2]
  float* d_h1;                  // [batch_max][h1]
  float* wgt;                   // [batch_max][n_in] output weighting of the current batch
  float* loss;                  // [batch_max * n_vec + 32]
  int64_t step;
  // tensor-core forward (tcgen05): layer widths multiples of 64
  bool tc;
  __nv_bfloat16* wt16;          // BF16 weights transposed, W_l^T [fan_out][fan_in], same offsets
  __nv_bfloat16* xb;            // [batch_max][n_in] BF16 input (the products' A operand)
  __nv_bfloat16* h1b;           // [batch_max][h1] BF16 activations
  __nv_bfloat16* h2b;           // [batch_max][h2]
  int* err;                     // device error word: a bounded tensor-core wait gave up
  int map_err;                  // host: a tensor map of the tensor-core products could not be encoded
  CUtensorMap tmap[3][2];               // per layer: A (activations) and Bt (weights), for batch tmap_batch
  int tmap_batch;                       // 0: not encoded
};

namespace msmg {

// ------------------------------------------------------------------ GEMM
// C[M][N] = op(A)[M][K] op(B)[K][N] (+ bias[N]) (ReLU), FP32 accumulation.
//   A element (m, k): TA ? A[k * lda + m] : A[m * lda + k]
//   B element (k, n): TB ? B[n * ldb + k] : B[k * ldb + n]
// 64 x 64 output tile per CTA of 256 threads, 4 x 4 outputs per thread, K in
// steps of 16 through shared memory.
constexpr int kBM = 64, kBN = 64, kBK = 16;

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename TAe, typename TBe, bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) k_gemm(const TAe* __restrict__ A, int lda, const TBe* __restrict__ B, int ldb,
                                              float* __restrict__ C, int ldc, const float* __restrict__ bias, int M,
                                              int N, int K) {
  __shared__ float As[kBK][kBM + 4];
  __shared__ float Bs[kBK][kBN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += kBK) {
    // 1024 values of each tile, 4 per thread
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = tid + 256 * q;
      // A tile: (mm, kk), mm < 64, kk < 16
      int mm, kk;
      if (TA) { mm = idx % kBM; kk = idx / kBM; }     // consecutive threads along m (contiguous in A^T layout)
      else { kk = idx % kBK; mm = idx / kBK; }        // consecutive threads along k
      const int gm = m0 + mm, gk = k0 + kk;
      float va = 0.f;
      if (gm < M && gk < K) va = to_f(TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk]);
      As[kk][mm] = va;
      // B tile: (kk, nn)
      int nn;
      if (TB) { kk = idx % kBK; nn = idx / kBK; }
      else { nn = idx % kBN; kk = idx / kBN; }
      const int gn = n0 + nn;
      const int gk2 = k0 + kk;
      float vb = 0.f;
      if (gn < N && gk2 < K) vb = to_f(TB ? B[(int64_t)gn * ldb + gk2] : B[(int64_t)gk2 * ldb + gn]);
      Bs[kk][nn] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      float v = acc[i][j];
      if (EPI >= 1) v += bias[gn];
      if (EPI == 2) v = v > 0.f ? v : 0.f;
      C[(int64_t)gm * ldc + gn] = v;
    }
  }
}

template <typename TAe, typename TBe, bool TA, bool TB, int EPI>
static void gemm(const TAe* A, int lda, const TBe* B, int ldb, float* C, int ldc, const float* bias, int M, int N,
                 int K, cudaStream_t s) {
  dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM);
  k_gemm<TAe, TBe, TA, TB, EPI><<<grid, 256, 0, s>>>(A, lda, B, ldb, C, ldc, bias, M, N, K);
}

// ------------------------------------------------------------------ tensor-core GEMM (tcgen05)
// C[M][N] = epi(A[M][K] . Bt[N][K]^T (+ bias)), A and Bt BF16 with K contiguous,
// FP32 accumulation in tensor memory (TMEM).  Persistent: one CTA per SM takes
// the 128 x BN output tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... (BN =
// 256, 128 or 64, the widest dividing N; N-tiles fastest, so consecutive tiles
// share their A rows in L2), with six warps in three roles:
//   warp 0, one thread: TMA (cp.async.bulk.tensor.2d) of the A and Bt blocks
//     (K in blocks of 64, 128-byte swizzle) into a ring of shared-memory stages,
//     completion counted in bytes on the stage's "full" mbarrier; a stage is
//     refilled once its "empty" mbarrier has fired;
//   warp 1, one thread: the four 128 x BN x 16 MMAs of each block (shared-memory
//     descriptors, K-major, 128-byte swizzle: 8-row groups 1024 bytes apart, the
//     16-wide K steps 32 bytes apart inside the swizzle atom), tcgen05.commit to
//     the stage's "empty" barrier, and after a tile's last block a commit to the
//     "accumulator full" barrier of the tile's TMEM buffer (two buffers of BN
//     columns, so the next tile accumulates while this one is written out);
//   warps 2-5: the epilogue (warp w reads TMEM lanes 32 (w mod 4) .. + 31, the
//     tile's rows): 64-column chunks by tcgen05.ld into a padded shared-memory
//     slice, the buffer released ("accumulator empty") once read, then bias, ReLU,
//     FP32 store and, when asked, a BF16 copy (the next layer's A operand), each
//     store writing whole row segments.
// Rows of A beyond M and of Bt beyond N read as zeros (TMA bounds).  Every wait
// is bounded: on timeout the error word is set, the loops stop, what was issued
// is drained with bounded waits, and the TMEM is freed before the CTA returns.
// K must be a multiple of 64, the row strides multiples of 8 elements and the
// bases 16-byte aligned (the tensor maps' rules).
constexpr int kTcM = 128, kTcK = 64, kTcThreads = 192, kTcChunk = 64;
template <int BN>
__host__ __device__ constexpr int tc_stages() { return BN == 256 ? 3 : (BN == 128 ? 4 : 6); }
template <int BN>
__host__ __device__ constexpr size_t tc_stage_bytes() { return (size_t)(kTcM + BN) * kTcK * 2; }
constexpr size_t kTcEpiBytes = (size_t)4 * 32 * (kTcChunk + 4) * 4;   // four warps' padded 32 x 64 slices
template <int BN>
__host__ __device__ constexpr size_t tc_smem_bytes() {
  return tc_stages<BN>() * tc_stage_bytes<BN>() + kTcEpiBytes + 1024;
}

// shared-memory matrix descriptor, K-major with 128-byte swizzle: start address,
// leading offset unused (1), stride between 8-row groups 1024 bytes, descriptor
// version 1, layout type 2 (128-byte swizzle)
__device__ __forceinline__ uint64_t tc_desc_sw128(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// instruction descriptor of kind::f16: F32 accumulator, BF16 A and B, both K-major, M x N
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void tc_mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ bool tc_mbar_wait(uint32_t bar, uint32_t parity) {
  for (int it = 0; it < (1 << 24); ++it) {
    uint32_t done;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done)
                 : "r"(bar), "r"(parity)
                 : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tc_tma_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar) : "memory");
}

template <int EPI, int BN>   // EPI 1: + bias; 2: + bias, ReLU
__global__ void __launch_bounds__(kTcThreads, 1) k_gemm_tc(const __grid_constant__ CUtensorMap mapA,
                                                           const __grid_constant__ CUtensorMap mapB,
                                                           float* __restrict__ C, int ldc,
                                                           __nv_bfloat16* __restrict__ Cb,
                                                           const float* __restrict__ bias, int M, int N, int K,
                                                           int* err) {
  constexpr int S = tc_stages<BN>();
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ __align__(8) unsigned long long full[S], empty[S], acc_full[2], acc_empty[2], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_fail;
  constexpr uint32_t kStage = (uint32_t)tc_stage_bytes<BN>();
  constexpr uint32_t kBytesA = kTcM * kTcK * 2;
  constexpr uint32_t kCols = 2 * BN;                      // two accumulator buffers
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_smem) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nk = K / kTcK;
  const int ntn = N / BN, ntiles = ntn * ((M + kTcM - 1) / kTcM);
  const int mytiles = blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (threadIdx.x == 32) {
    for (int i = 0; i < S; ++i) {
      tc_mbar_init(smem_u32(&full[i]), 1);
      tc_mbar_init(smem_u32(&empty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc_mbar_init(smem_u32(&acc_full[i]), 1);
      tc_mbar_init(smem_u32(&acc_empty[i]), 4);   // one arrival per epilogue warp
    }
    tc_mbar_init(smem_u32(&done_bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    s_fail = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  if (threadIdx.x == 0) {
    // producer: global block counter g runs across the CTA's tiles
    int g = 0;
    bool stop = false;
    for (int i = 0; i < mytiles && !stop; ++i) {
      const int t = (int)blockIdx.x + i * (int)gridDim.x;
      const int m0 = (t / ntn) * kTcM, n0 = (t % ntn) * BN;
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int st = g % S, use = g / S;
        if ((use > 0 && !tc_mbar_wait(smem_u32(&empty[st]), (uint32_t)((use - 1) & 1))) ||
            *(volatile int*)&s_fail) {
          atomicExch(&s_fail, 1);
          stop = true;
          break;
        }
        const uint32_t sA = smem_u32(smem + st * kStage), sB = sA + kBytesA;
        const uint32_t fb = smem_u32(&full[st]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(kStage) : "memory");
        tc_tma_2d(sA, &mapA, kb * kTcK, m0, fb);
        tc_tma_2d(sB, &mapB, kb * kTcK, n0, fb);
      }
    }
    // a load issued but not consumed must land before the CTA may exit (the last
    // S loads are the last completions of their barriers)
    for (int j = g - S < 0 ? 0 : g - S; j < g; ++j) tc_mbar_wait(smem_u32(&full[j % S]), (uint32_t)((j / S) & 1));
  } else if (threadIdx.x == 32) {
    // MMA issuer
    constexpr uint32_t idesc = tc_idesc(kTcM, BN);
    int g = 0;
    bool stop = false;
    for (int i = 0; i < mytiles && !stop; ++i) {
      const int a = i & 1, use = i >> 1;
      if ((use > 0 && !tc_mbar_wait(smem_u32(&acc_empty[a]), (uint32_t)((use - 1) & 1))) || *(volatile int*)&s_fail) {
        atomicExch(&s_fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t acc_tm = tmem + (uint32_t)(a * BN);
      for (int kb = 0; kb < nk; ++kb, ++g) {
        const int st = g % S, su = g / S;
        if (!tc_mbar_wait(smem_u32(&full[st]), (uint32_t)(su & 1)) || *(volatile int*)&s_fail) {
          atomicExch(&s_fail, 1);
          stop = true;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t sA = smem_u32(smem + st * kStage), sB = sA + kBytesA;
#pragma unroll
        for (int kk = 0; kk < kTcK / 16; ++kk) {
          const uint64_t da = tc_desc_sw128(sA + kk * 32), db = tc_desc_sw128(sB + kk * 32);
          const uint32_t accf = (kb > 0 || kk > 0) ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc_tm),
              "l"(da), "l"(db), "r"(idesc), "r"(accf));
        }
        tc_commit(smem_u32(&empty[st]));
      }
      if (!stop) tc_commit(smem_u32(&acc_full[a]));
    }
    tc_commit(smem_u32(&done_bar));   // covers every MMA this CTA issued
  } else if (warp >= 2) {
    // epilogue
    const int q = warp & 3;                                 // TMEM lane quarter = rows 32q .. 32q + 31
    float* sl = reinterpret_cast<float*>(smem + S * kStage) + (size_t)(warp - 2) * 32 * (kTcChunk + 4);
    for (int i = 0; i < mytiles; ++i) {
      const int t = (int)blockIdx.x + i * (int)gridDim.x;
      const int m0 = (t / ntn) * kTcM, n0 = (t % ntn) * BN;
      const int a = i & 1, use = i >> 1;
      bool ok = tc_mbar_wait(smem_u32(&acc_full[a]), (uint32_t)(use & 1));
      ok = __all_sync(0xffffffffu, ok && *(volatile int*)&s_fail == 0);
      if (!ok) {
        if (lane == 0) atomicExch(&s_fail, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t acc_tm = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(a * BN);
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += kTcChunk) {
#pragma unroll
        for (int c1 = 0; c1 < kTcChunk; c1 += 16) {
          uint32_t v[16];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
              "%14, %15}, [%16];\n"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(acc_tm + (uint32_t)(c0 + c1)));
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
          float4* dst = reinterpret_cast<float4*>(sl + (size_t)lane * (kTcChunk + 4) + c1);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            dst[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                 __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
        }
        if (c0 + kTcChunk >= BN) {
          // the whole accumulator of this tile has been read: release the buffer
          asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
          __syncwarp();
          if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&acc_empty[a])) : "memory");
        }
        __syncwarp();
        // lanes 0-15 row 2k, lanes 16-31 row 2k + 1, four columns each
        const int cl = (lane & 15) * 4;
        float4 bb = make_float4(0.f, 0.f, 0.f, 0.f);
        if (EPI >= 1) bb = __ldg(reinterpret_cast<const float4*>(bias + n0 + c0 + cl));
#pragma unroll 4
        for (int r2 = 0; r2 < 32; r2 += 2) {
          const int r = r2 + (lane >> 4);
          const int row = m0 + q * 32 + r;
          float4 v = *reinterpret_cast<const float4*>(sl + (size_t)r * (kTcChunk + 4) + cl);
          if (row < M) {
            if (EPI >= 1) { v.x += bb.x; v.y += bb.y; v.z += bb.z; v.w += bb.w; }
            if (EPI == 2) {
              v.x = v.x > 0.f ? v.x : 0.f; v.y = v.y > 0.f ? v.y : 0.f;
              v.z = v.z > 0.f ? v.z : 0.f; v.w = v.w > 0.f ? v.w : 0.f;
            }
            *reinterpret_cast<float4*>(C + (int64_t)row * ldc + n0 + c0 + cl) = v;
            if (Cb) {
              const __nv_bfloat162 h0 = __floats2bfloat162_rn(v.x, v.y), h1 = __floats2bfloat162_rn(v.z, v.w);
              uint2 w;
              w.x = *reinterpret_cast<const uint32_t*>(&h0);
              w.y = *reinterpret_cast<const uint32_t*>(&h1);
              *reinterpret_cast<uint2*>(Cb + (int64_t)row * ldc + n0 + c0 + cl) = w;
            }
          }
        }
        __syncwarp();   // the slice is rewritten by the next chunk
      }
    }
  }
  __syncwarp();
  __syncthreads();
  if (threadIdx.x == 0) {
    // every MMA complete before the TMEM is freed (at once unless a wait gave up)
    const bool d = tc_mbar_wait(smem_u32(&done_bar), 0u);
    if (s_fail || !d) atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols));
  }
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link against
// the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}
// 2-D BF16 map of a rows x cols matrix (cols contiguous, row stride ld elements),
// box of box_rows x 64, 128-byte swizzle, zero fill outside
static bool tc_map(CUtensorMap* map, const __nv_bfloat16* base, int rows, int cols, int ld, int box_rows) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// widest output tile dividing N (N a multiple of 64)
static inline int tc_bn(int N) { return N % 256 == 0 ? 256 : (N % 128 == 0 ? 128 : 64); }
static int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      n = 1;
    }
  }
  return n;
}
// persistent launch: one CTA per SM (or per tile, when there are fewer)
template <int EPI>
static void gemm_tc(const CUtensorMap& ma, const CUtensorMap& mb, float* C, int ldc, __nv_bfloat16* Cb,
                    const float* bias, int M, int N, int K, int* err, cudaStream_t s) {
  const int bn = tc_bn(N);
  const int tiles = (N / bn) * ((M + kTcM - 1) / kTcM);
  const unsigned grid = (unsigned)(tiles < sm_count() ? tiles : sm_count());
  if (bn == 256)
    k_gemm_tc<EPI, 256><<<grid, kTcThreads, tc_smem_bytes<256>(), s>>>(ma, mb, C, ldc, Cb, bias, M, N, K, err);
  else if (bn == 128)
    k_gemm_tc<EPI, 128><<<grid, kTcThreads, tc_smem_bytes<128>(), s>>>(ma, mb, C, ldc, Cb, bias, M, N, K, err);
  else
    k_gemm_tc<EPI, 64><<<grid, kTcThreads, tc_smem_bytes<64>(), s>>>(ma, mb, C, ldc, Cb, bias, M, N, K, err);
}
template <int EPI>
static void gemm_tc_prepare() {
  cudaFuncSetAttribute(k_gemm_tc<EPI, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes<256>());
  cudaFuncSetAttribute(k_gemm_tc<EPI, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes<128>());
  cudaFuncSetAttribute(k_gemm_tc<EPI, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes<64>());
}

// BF16 copy of an FP32 matrix (the tensor-core A operand of layer 1)
__global__ void k_bf16_copy(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16(a[i]);
}
// Wt[c][r] = bf16(W[r][c]) for a rows x cols FP32 matrix
__global__ void k_transpose_bf16(const float* __restrict__ W, int rows, int cols, __nv_bfloat16* __restrict__ Wt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)rows * cols) return;
  const int r = (int)(i / cols), c = (int)(i % cols);
  Wt[(int64_t)c * rows + r] = __float2bfloat16(W[i]);
}

// ------------------------------------------------------------------ output weighting
// w[b][c] = exp(4 (x_c - max x)) / sqrt(sum_c exp(8 (x_c - max x))) = sqrt(S_c / sum S)
// for x_c = (log S_c - mean) / 8; one CTA per row.
__global__ void k_out_weight(const float* __restrict__ x, int n_in, float* __restrict__ w) {
  const int64_t b = blockIdx.x;
  const float* xr = x + b * n_in;
  __shared__ float red[32];
  __shared__ float bc;
  float mx = -3.0e38f;
  for (int c = threadIdx.x; c < n_in; c += blockDim.x) mx = fmaxf(mx, xr[c]);
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = red[0];
    for (int i = 1; i < (int)((blockDim.x + 31) >> 5); ++i) m = fmaxf(m, red[i]);
    bc = m;
  }
  __syncthreads();
  mx = bc;
  float acc = 0.f;
  for (int c = threadIdx.x; c < n_in; c += blockDim.x) acc += expf(8.f * (xr[c] - mx));
  acc = warp_sum_t(acc);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) t += red[i];
    bc = rsqrtf(t);
  }
  __syncthreads();
  const float inv = bc;
  for (int c = threadIdx.x; c < n_in; c += blockDim.x) w[b * n_in + c] = expf(4.f * (xr[c] - mx)) * inv;
}

// y[b][k][c] *= w[b][c]  (forward: y = w o; backward: d o = w d y)
__global__ void k_apply_weight(float* __restrict__ y, const float* __restrict__ w, int batch, int n_vec, int n_in) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)batch * n_vec * n_in;
  if (i >= total) return;
  const int c = (int)(i % n_in);
  const int64_t b = i / ((int64_t)n_vec * n_in);
  y[i] *= w[b * n_in + c];
}

// ------------------------------------------------------------------ elementwise
// d_h *= (h > 0)   (ReLU derivative from the post-activation value)
__global__ void k_relu_back(float* __restrict__ dh, const float* __restrict__ h, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !(h[i] > 0.f)) dh[i] = 0.f;
}

// db[n] = sum_b d[b][n]  (thread per column, rows in order)
__global__ void k_colsum(const float* __restrict__ d, int rows, int cols, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= cols) return;
  float acc = 0.f;
  for (int b = 0; b < rows; ++b) acc += d[(int64_t)b * cols + n];
  db[n] = acc;
}

// Sign-invariant loss and its gradient; one warp per (sample, vector).
//   loss[b * n_vec + k] = ||p||^2 + ||t||^2 - 2 |p.t|
//   dp = 2 (p - sign(p.t) t) * scale
__global__ void k_loss(const float* __restrict__ out, const float* __restrict__ target, int batch, int n_vec, int n_in,
                       float scale, float* __restrict__ loss, float* __restrict__ d_out) {
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= (int64_t)batch * n_vec) return;
  const float* p = out + w * n_in;
  const float* t = target + w * n_in;
  float pt = 0.f, pp = 0.f, tt = 0.f;
  for (int i = lane; i < n_in; i += 32) {
    const float a = p[i], b = t[i];
    pt = fmaf(a, b, pt);
    pp = fmaf(a, a, pp);
    tt = fmaf(b, b, tt);
  }
  pt = warp_sum_t(pt);
  pp = warp_sum_t(pp);
  tt = warp_sum_t(tt);
  const float sg = pt >= 0.f ? 1.f : -1.f;
  if (lane == 0) loss[w] = pp + tt - 2.f * fabsf(pt);
  if (d_out) {
    float* dp = d_out + w * n_in;
    for (int i = lane; i < n_in; i += 32) dp[i] = 2.f * scale * (p[i] - sg * t[i]);
  }
}

// total = sum of n values, in order, one thread (n is batch * n_vec, small)
__global__ void k_sum_in_order(const float* __restrict__ v, int n, float* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double acc = 0.0;
  for (int i = 0; i < n; ++i) acc += v[i];
  *out = (float)acc;
}

// Adam (Kingma and Ba, 2015) on the FP32 masters; refresh the BF16 copies.
__global__ void k_adam(float* __restrict__ w, __nv_bfloat16* __restrict__ w16, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  w16[i] = __float2bfloat16(wi);
}

__global__ void k_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16(a[i]);
}

// Deterministic initial weights: uniform(-a, a), a = sqrt(6 / fan_in), from a
// counter-based hash of (seed, index) (the splitmix64 finaliser); biases zero.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void k_init_uniform(float* __restrict__ w, int64_t n, uint64_t seed, float a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t h = splitmix64(seed ^ splitmix64((uint64_t)i));
  const float u = (float)((h >> 40) * (1.0 / 16777216.0));   // [0, 1)
  w[i] = a * (2.f * u - 1.f);
}

static inline unsigned g256(int64_t n) { return (unsigned)((n + 255) / 256); }

// ------------------------------------------------------------------ passes
// The products' operands are BF16: the weights (the masters' BF16 copies) and
// the activations (x, h1, h2 rounded to BF16 before the product that reads them);
// accumulation and the stored activations are FP32.  With layer widths multiples
// of 64 the products run on the tensor cores (tcgen05, k_gemm_tc), otherwise on
// the CUDA cores (k_gemm) with the same operands.
static void net_refresh_bf16(msmg_net* t, cudaStream_t s) {
  const int64_t dims[4] = {t->d.n_in, t->d.hidden[0], t->d.hidden[1], t->n_out};
  for (int l = 0; l < 3; ++l)
    k_transpose_bf16<<<g256(dims[l] * dims[l + 1]), 256, 0, s>>>(t->w32 + t->off_w[l], (int)dims[l], (int)dims[l + 1],
                                                                  t->wt16 + t->off_w[l]);
}

// Tensor maps of the three products for `batch` rows (encoded when the batch
// size changes; the buffers and weights never move).
static bool net_encode_maps(msmg_net* t, int batch) {
  if (t->tmap_batch == batch) return true;
  const msmg_net_desc& d = t->d;
  const int dims[4] = {d.n_in, d.hidden[0], d.hidden[1], t->n_out};
  const __nv_bfloat16* acts[3] = {t->xb, t->h1b, t->h2b};
  for (int l = 0; l < 3; ++l) {
    const int K = dims[l], N = dims[l + 1];
    if (!tc_map(&t->tmap[l][0], acts[l], batch, K, K, kTcM) ||
        !tc_map(&t->tmap[l][1], t->wt16 + t->off_w[l], N, K, K, tc_bn(N))) {
      t->tmap_batch = 0;
      return false;
    }
  }
  t->tmap_batch = batch;
  return true;
}

// The three products on the tensor cores; with ev (6 events) each launch is
// bracketed by ev[2l], ev[2l + 1].
static void net_tc_products(msmg_net* t, int batch, cudaStream_t s, cudaEvent_t* ev) {
  const msmg_net_desc& d = t->d;
  const int h1 = d.hidden[0], h2 = d.hidden[1], no = t->n_out;
  if (!net_encode_maps(t, batch)) {
    t->map_err = 1;
    return;
  }
  if (ev) cudaEventRecord(ev[0], s);
  gemm_tc<2>(t->tmap[0][0], t->tmap[0][1], t->h1, h1, t->h1b, t->w32 + t->off_b[0], batch, h1, d.n_in, t->err, s);
  if (ev) cudaEventRecord(ev[1], s);
  if (ev) cudaEventRecord(ev[2], s);
  gemm_tc<2>(t->tmap[1][0], t->tmap[1][1], t->h2, h2, t->h2b, t->w32 + t->off_b[1], batch, h2, h1, t->err, s);
  if (ev) cudaEventRecord(ev[3], s);
  if (ev) cudaEventRecord(ev[4], s);
  gemm_tc<1>(t->tmap[2][0], t->tmap[2][1], t->out, no, nullptr, t->w32 + t->off_b[2], batch, no, h2, t->err, s);
  if (ev) cudaEventRecord(ev[5], s);
}

// forward for `batch` rows of x; output in net->out
static void net_forward(msmg_net* t, const float* x, int batch, cudaStream_t s) {
  const msmg_net_desc& d = t->d;
  const int h1 = d.hidden[0], h2 = d.hidden[1], no = t->n_out;
  k_bf16_copy<<<g256((int64_t)batch * d.n_in), 256, 0, s>>>(x, t->xb, (int64_t)batch * d.n_in);
  if (t->tc) {
    net_tc_products(t, batch, s, nullptr);
  } else {
    gemm<__nv_bfloat16, __nv_bfloat16, false, false, 2>(t->xb, d.n_in, t->w16 + t->off_w[0], h1, t->h1, h1,
                                                        t->w32 + t->off_b[0], batch, h1, d.n_in, s);
    k_bf16_copy<<<g256((int64_t)batch * h1), 256, 0, s>>>(t->h1, t->h1b, (int64_t)batch * h1);
    gemm<__nv_bfloat16, __nv_bfloat16, false, false, 2>(t->h1b, h1, t->w16 + t->off_w[1], h2, t->h2, h2,
                                                        t->w32 + t->off_b[1], batch, h2, h1, s);
    k_bf16_copy<<<g256((int64_t)batch * h2), 256, 0, s>>>(t->h2, t->h2b, (int64_t)batch * h2);
    gemm<__nv_bfloat16, __nv_bfloat16, false, false, 1>(t->h2b, h2, t->w16 + t->off_w[2], no, t->out, no,
                                                        t->w32 + t->off_b[2], batch, no, h2, s);
  }
  k_out_weight<<<(unsigned)batch, 128, 0, s>>>(x, d.n_in, t->wgt);
  k_apply_weight<<<g256((int64_t)batch * no), 256, 0, s>>>(t->out, t->wgt, batch, d.n_vec, d.n_in);
}

// loss and gradients for `batch` rows (forward included); loss total in t->loss[batch * n_vec]
static void net_backward(msmg_net* t, const float* x, const float* target, int batch, cudaStream_t s) {
  const msmg_net_desc& d = t->d;
  const int h1 = d.hidden[0], h2 = d.hidden[1], no = t->n_out;
  net_forward(t, x, batch, s);
  const int nl = batch * d.n_vec;
  const float scale = 1.f / (float)nl;
  k_loss<<<(unsigned)(((int64_t)nl * 32 + 255) / 256), 256, 0, s>>>(t->out, target, batch, d.n_vec, d.n_in, scale,
                                                                   t->loss, t->d_out);
  k_sum_in_order<<<1, 32, 0, s>>>(t->loss, nl, t->loss + nl);
  k_apply_weight<<<g256((int64_t)batch * no), 256, 0, s>>>(t->d_out, t->wgt, batch, d.n_vec, d.n_in);
  float* g = t->grad;
  // layer 3: dW3 = h2^T d_out, db3, d_h2 = d_out W3^T (relu mask)
  gemm<__nv_bfloat16, float, true, false, 0>(t->h2b, h2, t->d_out, no, g + t->off_w[2], no, nullptr, h2, no, batch,
                                             s);
  k_colsum<<<g256(no), 256, 0, s>>>(t->d_out, batch, no, g + t->off_b[2]);
  gemm<float, __nv_bfloat16, false, true, 0>(t->d_out, no, t->w16 + t->off_w[2], no, t->d_h2, h2, nullptr, batch, h2,
                                             no, s);
  k_relu_back<<<g256((int64_t)batch * h2), 256, 0, s>>>(t->d_h2, t->h2, (int64_t)batch * h2);
  // layer 2
  gemm<__nv_bfloat16, float, true, false, 0>(t->h1b, h1, t->d_h2, h2, g + t->off_w[1], h2, nullptr, h1, h2, batch,
                                             s);
  k_colsum<<<g256(h2), 256, 0, s>>>(t->d_h2, batch, h2, g + t->off_b[1]);
  gemm<float, __nv_bfloat16, false, true, 0>(t->d_h2, h2, t->w16 + t->off_w[1], h2, t->d_h1, h1, nullptr, batch, h1,
                                             h2, s);
  k_relu_back<<<g256((int64_t)batch * h1), 256, 0, s>>>(t->d_h1, t->h1, (int64_t)batch * h1);
  // layer 1
  gemm<__nv_bfloat16, float, true, false, 0>(t->xb, d.n_in, t->d_h1, h1, g + t->off_w[0], h1, nullptr, d.n_in, h1,
                                             batch, s);
  k_colsum<<<g256(h1), 256, 0, s>>>(t->d_h1, batch, h1, g + t->off_b[0]);
}

}  // namespace msmg

using namespace msmg;

static int64_t net_layout(const msmg_net_desc* d, int64_t off_w[3], int64_t off_b[3]) {
  const int n_out = d->n_vec * d->n_in;
  const int64_t dims[4] = {d->n_in, d->hidden[0], d->hidden[1], n_out};
  int64_t o = 0;
  for (int l = 0; l < 3; ++l) {
    off_w[l] = o;
    o += dims[l] * dims[l + 1];
    o = (o + 63) / 64 * 64;
    off_b[l] = o;
    o += dims[l + 1];
    o = (o + 63) / 64 * 64;
  }
  return o;
}

static bool desc_ok(const msmg_net_desc* d) {
  return d && d->n_in >= 1 && d->n_in <= 4096 && d->hidden[0] >= 1 && d->hidden[1] >= 1 && d->hidden[0] <= 16384 &&
         d->hidden[1] <= 16384 && d->n_vec >= 1 && d->n_vec <= 64 && d->batch_max >= 1 && d->batch_max <= 1 << 20;
}

static int64_t net_carve(const msmg_net_desc* d, Arena& ar, msmg_net* t) {
  int64_t ow[3], ob[3];
  const int64_t np = net_layout(d, ow, ob);
  const int no = d->n_vec * d->n_in;
  const int64_t B = d->batch_max;
  float* w32 = ar.take<float>(np);
  __nv_bfloat16* w16 = ar.take<__nv_bfloat16>(np);
  float* grad = ar.take<float>(np);
  float* am = ar.take<float>(np);
  float* av = ar.take<float>(np);
  float* h1 = ar.take<float>(B * d->hidden[0]);
  float* h2 = ar.take<float>(B * d->hidden[1]);
  float* out = ar.take<float>(B * no);
  float* dout = ar.take<float>(B * no);
  float* dh2 = ar.take<float>(B * d->hidden[1]);
  float* dh1 = ar.take<float>(B * d->hidden[0]);
  float* loss = ar.take<float>(B * d->n_vec + 32);
  float* wgt = ar.take<float>(B * d->n_in);
  __nv_bfloat16* wt16 = ar.take<__nv_bfloat16>(np);
  __nv_bfloat16* xb = ar.take<__nv_bfloat16>(B * d->n_in);
  __nv_bfloat16* h1b = ar.take<__nv_bfloat16>(B * d->hidden[0]);
  __nv_bfloat16* h2b = ar.take<__nv_bfloat16>(B * d->hidden[1]);
  int* err = ar.take<int>(4);
  if (t) {
    t->d = *d;
    t->n_out = no;
    t->n_param = np;
    for (int l = 0; l < 3; ++l) { t->off_w[l] = ow[l]; t->off_b[l] = ob[l]; }
    t->w32 = w32; t->w16 = w16; t->grad = grad; t->adam_m = am; t->adam_v = av;
    t->h1 = h1; t->h2 = h2; t->out = out; t->d_out = dout; t->d_h2 = dh2; t->d_h1 = dh1; t->loss = loss;
    t->wgt = wgt;
    t->step = 0;
    t->wt16 = wt16; t->xb = xb; t->h1b = h1b; t->h2b = h2b; t->err = err;
    t->tc = d->n_in % 64 == 0 && d->hidden[0] % 64 == 0 && d->hidden[1] % 64 == 0;
  }
  return np;
}

// --------------------------------------------------------------- set-up integration
namespace msmg {

// x[e][c] = clamp(log S_c - mean_e log S, -20, 20) / 8: the element's
// log-permeability pattern up to a constant factor (for isotropic kappa,
// log S = log kappa + const), the scale-free input of the network.
// Output row: the element itself, or its lexicographic index when lex_of_hid is given.
__global__ void k_net_features(const double* __restrict__ S, int nb, int64_t m, const int* __restrict__ lex_of_hid,
                               float* __restrict__ x) {
  const int64_t e = blockIdx.x;
  if (e >= m) return;
  const int64_t row = lex_of_hid ? (int64_t)lex_of_hid[e] : e;
  __shared__ double red[32];
  double acc = 0.0;
  for (int c = threadIdx.x; c < nb; c += blockDim.x) acc += log(S[e * nb + c]);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t += red[w];
    red[0] = t / nb;
  }
  __syncthreads();
  const double mean = red[0];
  for (int c = threadIdx.x; c < nb; c += blockDim.x) {
    double v = log(S[e * nb + c]) - mean;
    v = v < -20.0 ? -20.0 : (v > 20.0 ? 20.0 : v);
    x[row * nb + c] = (float)(v / 8.0);
  }
}

// y[e][k - 1][c] = sqrt(S_c) Phi[e][k][c], k = 1 .. L-1: the level-1 eigenvectors
// in the symmetric form (Euclidean-orthonormal), the network's targets.
__global__ void k_net_targets(const double* __restrict__ S, const double* __restrict__ Phi, int nb, int L, int64_t m,
                              const int* __restrict__ lex_of_hid, float* __restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = m * (L - 1) * nb;
  if (i >= total) return;
  const int c = (int)(i % nb);
  const int64_t ek = i / nb;
  const int k = (int)(ek % (L - 1)) + 1;
  const int64_t e = ek / (L - 1);
  const int64_t row = lex_of_hid ? (int64_t)lex_of_hid[e] : e;
  y[(row * (L - 1) + (k - 1)) * nb + c] = (float)(sqrt(S[e * nb + c]) * Phi[(e * L + k) * nb + c]);
}

void launch_net_features(msmg_ctx* c, float* x, const int* lex_of_hid, cudaStream_t s) {
  k_net_features<<<(unsigned)c->fine.m, 128, 0, s>>>(c->fine.S, c->fine.nb, c->fine.m, lex_of_hid, x);
}

int net_status(msmg_net* t, cudaStream_t s);

// Guesses for every element, in chunks of the network's batch: g[e][k-1][c].
int net_guesses(msmg_ctx* c, const msmg_net* net, float* x, float* g, cudaStream_t s) {
  msmg_net* t = const_cast<msmg_net*>(net);
  launch_net_features(c, x, nullptr, s);
  const int64_t m = c->fine.m;
  const int nb = c->fine.nb;
  for (int64_t e0 = 0; e0 < m; e0 += t->d.batch_max) {
    const int b = (int)((m - e0) < t->d.batch_max ? (m - e0) : t->d.batch_max);
    net_forward(t, x + e0 * nb, b, s);
    MSMG_CUDA_TRY(cudaMemcpyAsync(g + e0 * t->n_out, t->out, (size_t)b * t->n_out * sizeof(float),
                                  cudaMemcpyDeviceToDevice, s));
  }
  MSMG_CUDA_TRY(cudaGetLastError());
  return net_status(t, s);
}

// MSMG_ERR_DEVICE_TIMEOUT when a tensor-core wait of the network's products gave up
// (synchronises the stream; clears the word), MSMG_ERR_CUDA when a tensor map
// could not be encoded (the products were not launched)
int net_status(msmg_net* t, cudaStream_t s) {
  if (t->map_err) {
    t->map_err = 0;
    return MSMG_ERR_CUDA;
  }
  int e = 0;
  MSMG_CUDA_TRY(cudaMemcpyAsync(&e, t->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  MSMG_CUDA_TRY(cudaStreamSynchronize(s));
  if (e) {
    MSMG_CUDA_TRY(cudaMemsetAsync(t->err, 0, sizeof(int), s));
    return MSMG_ERR_DEVICE_TIMEOUT;
  }
  return 0;
}

bool net_matches(const msmg_ctx* c, const msmg_net* net) {
  return net && net->d.n_in == c->fine.nb && net->d.n_vec == c->fine.L - 1;
}

}  // namespace msmg

extern "C" {

size_t msmg_net_workspace_size(const msmg_net_desc* desc) {
  if (!desc_ok(desc)) return 0;
  Arena ar;
  net_carve(desc, ar, nullptr);
  return ar.off + 256;
}

int msmg_net_create(const msmg_net_desc* desc, void* workspace, size_t workspace_bytes, uint64_t seed,
                    msmg_stream stream, msmg_net** out) {
  if (!out || !desc_ok(desc) || !workspace) return MSMG_ERR_INVALID_ARG;
  *out = nullptr;
  if (reinterpret_cast<uintptr_t>(workspace) % 256) return MSMG_ERR_WORKSPACE;
  if (workspace_bytes < msmg_net_workspace_size(desc)) return MSMG_ERR_WORKSPACE;
  msmg_net* t = new (std::nothrow) msmg_net{};
  if (!t) return MSMG_ERR_INVALID_ARG;
  Arena ar;
  ar.base = static_cast<char*>(workspace);
  ar.cap = workspace_bytes;
  net_carve(desc, ar, t);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  MSMG_CUDA_TRY(cudaMemsetAsync(t->w32, 0, (size_t)t->n_param * sizeof(float), s));
  MSMG_CUDA_TRY(cudaMemsetAsync(t->adam_m, 0, (size_t)t->n_param * sizeof(float), s));
  MSMG_CUDA_TRY(cudaMemsetAsync(t->adam_v, 0, (size_t)t->n_param * sizeof(float), s));
  const int64_t dims[4] = {desc->n_in, desc->hidden[0], desc->hidden[1], t->n_out};
  for (int l = 0; l < 3; ++l) {
    const int64_t n = dims[l] * dims[l + 1];
    k_init_uniform<<<g256(n), 256, 0, s>>>(t->w32 + t->off_w[l], n, seed * 4 + (uint64_t)l,
                                           sqrtf(6.f / (float)dims[l]) * (l == 2 ? 0.25f : 1.f));
  }
  k_to_bf16<<<g256(t->n_param), 256, 0, s>>>(t->w32, t->w16, t->n_param);
  net_refresh_bf16(t, s);
  MSMG_CUDA_TRY(cudaMemsetAsync(t->err, 0, 4 * sizeof(int), s));
  gemm_tc_prepare<1>();
  gemm_tc_prepare<2>();
  MSMG_CUDA_TRY(cudaGetLastError());
  *out = t;
  return 0;
}

void msmg_net_destroy(msmg_net* net) { delete net; }

int64_t msmg_net_param_count(const msmg_net* net) { return net ? net->n_param : 0; }

int msmg_net_param_offsets(const msmg_net* net, int64_t* w_off, int64_t* b_off) {
  if (!net || !w_off || !b_off) return MSMG_ERR_INVALID_ARG;
  for (int l = 0; l < 3; ++l) { w_off[l] = net->off_w[l]; b_off[l] = net->off_b[l]; }
  return 0;
}

int msmg_net_get_params(const msmg_net* net, float* params, msmg_stream stream) {
  if (!net || !params) return MSMG_ERR_INVALID_ARG;
  MSMG_CUDA_TRY(cudaMemcpyAsync(params, net->w32, (size_t)net->n_param * sizeof(float), cudaMemcpyDeviceToDevice,
                                reinterpret_cast<cudaStream_t>(stream)));
  return 0;
}

int msmg_net_set_params(msmg_net* net, const float* params, msmg_stream stream) {
  if (!net || !params) return MSMG_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  MSMG_CUDA_TRY(cudaMemcpyAsync(net->w32, params, (size_t)net->n_param * sizeof(float), cudaMemcpyDeviceToDevice, s));
  k_to_bf16<<<g256(net->n_param), 256, 0, s>>>(net->w32, net->w16, net->n_param);
  net_refresh_bf16(net, s);
  MSMG_CUDA_TRY(cudaGetLastError());
  return 0;
}

int msmg_net_forward(msmg_net* net, const float* x, float* y, int batch, msmg_stream stream) {
  if (!net || !x || !y || batch < 0) return MSMG_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (int b0 = 0; b0 < batch; b0 += net->d.batch_max) {
    const int b = batch - b0 < net->d.batch_max ? batch - b0 : net->d.batch_max;
    net_forward(net, x + (int64_t)b0 * net->d.n_in, b, s);
    MSMG_CUDA_TRY(cudaMemcpyAsync(y + (int64_t)b0 * net->n_out, net->out, (size_t)b * net->n_out * sizeof(float),
                                  cudaMemcpyDeviceToDevice, s));
  }
  MSMG_CUDA_TRY(cudaGetLastError());
  return net_status(net, s);
}

int msmg_net_time_products(msmg_net* net, const float* x, int batch, double* ms, msmg_stream stream) {
  if (!net || !x || !ms || batch < 1 || batch > net->d.batch_max) return MSMG_ERR_INVALID_ARG;
  if (!net->tc) return MSMG_ERR_UNSUPPORTED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t ev[6];
  for (int i = 0; i < 6; ++i) MSMG_CUDA_TRY(cudaEventCreate(&ev[i]));
  net_forward(net, x, batch, s);   // the products' operands: BF16 input and activations
  net_tc_products(net, batch, s, ev);
  cudaError_t e = cudaStreamSynchronize(s);
  for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
    float t = 0.f;
    e = cudaEventElapsedTime(&t, ev[2 * l], ev[2 * l + 1]);
    ms[l] = t;
  }
  for (int i = 0; i < 6; ++i) cudaEventDestroy(ev[i]);
  MSMG_CUDA_TRY(e);
  return net_status(net, s);
}

int msmg_net_gradients(msmg_net* net, const float* x, const float* target, int batch, float* grad, float* loss_host,
                       msmg_stream stream) {
  if (!net || !x || !target || batch < 1 || batch > net->d.batch_max) return MSMG_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  net_backward(net, x, target, batch, s);
  if (grad)
    MSMG_CUDA_TRY(cudaMemcpyAsync(grad, net->grad, (size_t)net->n_param * sizeof(float), cudaMemcpyDeviceToDevice, s));
  {
    const int st = net_status(net, s);
    if (st) return st;
  }
  if (loss_host) {
    const int nl = batch * net->d.n_vec;
    MSMG_CUDA_TRY(cudaMemcpyAsync(loss_host, net->loss + nl, sizeof(float), cudaMemcpyDeviceToHost, s));
    MSMG_CUDA_TRY(cudaStreamSynchronize(s));
    *loss_host /= (float)nl;
  }
  MSMG_CUDA_TRY(cudaGetLastError());
  return 0;
}

int msmg_net_train_step(msmg_net* net, const float* x, const float* target, int batch, float lr, float* loss_host,
                        msmg_stream stream) {
  if (!net || !x || !target || batch < 1 || batch > net->d.batch_max || !(lr > 0.f)) return MSMG_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  net_backward(net, x, target, batch, s);
  net->step += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)net->step), c2 = 1.f - powf(b2, (float)net->step);
  k_adam<<<g256(net->n_param), 256, 0, s>>>(net->w32, net->w16, net->grad, net->adam_m, net->adam_v, net->n_param, lr,
                                            b1, b2, eps, c1, c2);
  net_refresh_bf16(net, s);
  {
    const int st = net_status(net, s);
    if (st) return st;
  }
  if (loss_host) {
    const int nl = batch * net->d.n_vec;
    MSMG_CUDA_TRY(cudaMemcpyAsync(loss_host, net->loss + nl, sizeof(float), cudaMemcpyDeviceToHost, s));
    MSMG_CUDA_TRY(cudaStreamSynchronize(s));
    *loss_host /= (float)nl;
  }
  MSMG_CUDA_TRY(cudaGetLastError());
  return 0;
}

int msmg_learning_data(msmg_ctx* c, float* x, float* y, msmg_stream stream) {
  if (!c || !x || !y || c->fine.L < 2) return MSMG_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  launch_net_features(c, x, c->fine.lex_of_hid, s);
  const int64_t total = c->fine.m * (c->fine.L - 1) * c->fine.nb;
  k_net_targets<<<g256(total), 256, 0, s>>>(c->fine.S, c->fine.Phi, c->fine.nb, c->fine.L, c->fine.m,
                                            c->fine.lex_of_hid, y);
  MSMG_CUDA_TRY(cudaGetLastError());
  return 0;
}

}  // extern "C"
