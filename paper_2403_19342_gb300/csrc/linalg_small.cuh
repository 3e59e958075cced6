// Small dense linear algebra inside one CTA (shared memory), FP64: parallel
// cyclic Jacobi eigensolver, stable ranking of a diagonal, Gauss-Jordan
// inverse.  Used by the local eigenproblems, Rayleigh-Ritz steps and the
// per-parent smoother inverses.
#pragma once
#include "msmg_internal.cuh"
#include "reduce.cuh"
#include <cmath>

namespace msmg {

// ------------------------------------------------------------------ Jacobi
// Parallel cyclic Jacobi (round-robin pairing) on the n x n symmetric matrix A
// in shared memory; V receives the eigenvectors (columns).  On return the
// diagonal of A holds the eigenvalues.
__device__ inline void jacobi_eig(double* A, double* V, int n, double* cs, int* pr, double* red, int max_sweeps,
                           double rtol) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int npad = n + (n & 1);
  const int half = npad / 2;
  for (int i = tid; i < n * n; i += nthr) V[i] = (i / n == i % n) ? 1.0 : 0.0;
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double v[2] = {0.0, 0.0};
    for (int i = tid; i < n * n; i += nthr) {
      const double a = A[i];
      v[1] += a * a;
      if (i / n != i % n) v[0] += a * a;
    }
    block_sum<2>(v, red + 2);
    if (tid == 0) { red[0] = v[0]; red[1] = v[1]; }
    __syncthreads();
    const bool conv = red[0] <= rtol * rtol * red[1];
    __syncthreads();
    if (conv) break;
    for (int r = 0; r < npad - 1; ++r) {
      for (int i = tid; i < half; i += nthr) {
        int pa = (i == 0) ? 0 : 1 + ((i - 1 + r) % (npad - 1));
        const int j = npad - 1 - i;
        int pb = 1 + ((j - 1 + r) % (npad - 1));
        if (pa > pb) { int t = pa; pa = pb; pb = t; }
        double c = 1.0, s = 0.0;
        if (pb < n) {
          const double apq = A[pa * n + pb];
          if (fabs(apq) > 1e-300) {
            const double theta = (A[pb * n + pb] - A[pa * n + pa]) / (2.0 * apq);
            const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        cs[2 * i] = c;
        cs[2 * i + 1] = s;
        pr[2 * i] = pa;
        pr[2 * i + 1] = pb;
      }
      __syncthreads();
      for (int idx = tid; idx < half * n; idx += nthr) {     // rows: A <- J^T A
        const int i = idx / n, col = idx % n;
        const int p = pr[2 * i], q = pr[2 * i + 1];
        if (q >= n) continue;
        const double c = cs[2 * i], s = cs[2 * i + 1];
        const double ap = A[p * n + col], aq = A[q * n + col];
        A[p * n + col] = c * ap - s * aq;
        A[q * n + col] = s * ap + c * aq;
      }
      __syncthreads();
      for (int idx = tid; idx < half * n; idx += nthr) {     // columns: A <- A J, V <- V J
        const int i = idx / n, row = idx % n;
        const int p = pr[2 * i], q = pr[2 * i + 1];
        if (q >= n) continue;
        const double c = cs[2 * i], s = cs[2 * i + 1];
        const double ap = A[row * n + p], aq = A[row * n + q];
        A[row * n + p] = c * ap - s * aq;
        A[row * n + q] = s * ap + c * aq;
        const double vp = V[row * n + p], vq = V[row * n + q];
        V[row * n + p] = c * vp - s * vq;
        V[row * n + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
}

// order[k] = index of the k-th smallest diagonal entry of A (stable).  NaN
// entries sort as +infinity, so the ranks always form a permutation of 0..n-1.
__device__ __forceinline__ double sort_key(double v) { return isnan(v) ? INFINITY : v; }
__device__ inline void sort_diag(const double* A, int n, int* order) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double di = sort_key(A[i * n + i]);
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double dj = sort_key(A[j * n + j]);
      rank += (dj < di) || (dj == di && j < i);
    }
    order[rank] = i;
  }
  __syncthreads();
}

// In-place Gauss-Jordan inverse of an SPD n x n matrix in shared memory.
__device__ inline void gj_inverse(double* A, int n, double* rowk, double* colk) {
  for (int k = 0; k < n; ++k) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      rowk[i] = A[k * n + i];
      colk[i] = A[i * n + k];
    }
    __syncthreads();
    const double piv = colk[k];
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int i = idx / n, j = idx % n;
      double v;
      if (i == k && j == k) v = 1.0 / piv;
      else if (i == k) v = rowk[j] / piv;
      else if (j == k) v = -colk[i] / piv;
      else v = A[idx] - colk[i] * rowk[j] / piv;
      A[idx] = v;
    }
    __syncthreads();
  }
}

// Positive double values order like their bit patterns: atomic max via int64.
__device__ __forceinline__ void atomic_max_pos(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

}  // namespace msmg
