// CTA-cooperative dense linear algebra on small matrices (n <= 80) for the
// GPU-SLS kernels (sm_103a).  All routines are called by every thread of a
// 256-thread CTA and end with __syncthreads(), so their outputs are visible to
// the whole CTA on return.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gsls {

constexpr int NT = 256;     // threads per CTA
constexpr int TILE = 80;    // max edge of a C tile (and of a GJ-inverted matrix)
constexpr int KT = 16;      // k-slab staged per step of the CTA GEMM
constexpr int GJ_LD = TILE + 1;

__host__ __device__ inline int rup4(int x) { return (x + 3) & ~3; }
__host__ __device__ inline int rup16(int x) { return (x + 15) & ~15; }

template <typename T> __device__ inline T tiny_pivot();
template <> __device__ inline double tiny_pivot<double>() { return 1e-280; }
template <> __device__ inline float tiny_pivot<float>() { return 1e-30f; }

// Shared-memory scratch needed by cta_gemm: 2*KT*TILE elements.
template <typename T> constexpr int gemm_smem_elems() { return 2 * KT * TILE; }

// C = alpha * op(A) * op(B) + beta * C0 (+ I if addI), with op(A) m x k and
// op(B) k x n.  tA: A is stored k x m (op(A) = A^T); tB likewise.  C may alias
// C0 but not A or B.  C0 may be null.  Operands may live in global or shared
// memory.  Any m, n (tiled by TILE), any k.
template <typename T>
__device__ __noinline__ void cta_gemm(int m, int n, int k, T alpha,
                         const T* A, int lda, bool tA,
                         const T* B, int ldb, bool tB,
                         T beta, const T* C0, int ldc0, bool addI,
                         T* C, int ldc, T* sm) {
  T* As = sm;               // As[kk * TILE + i] = op(A)[i][kk]
  T* Bs = sm + KT * TILE;   // Bs[kk * TILE + j] = op(B)[kk][j]
  const int t = threadIdx.x;
  const int ty = t >> 4, tx = t & 15;
  for (int i0 = 0; i0 < m; i0 += TILE) {
    for (int j0 = 0; j0 < n; j0 += TILE) {
      const int mt = min(TILE, m - i0), nt = min(TILE, n - j0);
      T acc[5][5];
#pragma unroll
      for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int b = 0; b < 5; ++b) acc[a][b] = T(0);
      for (int k0 = 0; k0 < k; k0 += KT) {
        const int kt = min(KT, k - k0);
        __syncthreads();
        for (int e = t; e < mt * KT; e += NT) {
          int i, kk;
          if (!tA) { i = e / KT; kk = e - i * KT; } else { kk = e / mt; i = e - kk * mt; }
          T v = T(0);
          if (kk < kt) v = tA ? A[(size_t)(k0 + kk) * lda + i0 + i] : A[(size_t)(i0 + i) * lda + k0 + kk];
          As[kk * TILE + i] = v;
        }
        for (int e = t; e < nt * KT; e += NT) {
          int j, kk;
          if (!tB) { kk = e / nt; j = e - kk * nt; } else { j = e / KT; kk = e - j * KT; }
          T v = T(0);
          if (kk < kt) v = tB ? B[(size_t)(j0 + j) * ldb + k0 + kk] : B[(size_t)(k0 + kk) * ldb + j0 + j];
          Bs[kk * TILE + j] = v;
        }
        __syncthreads();
        for (int kk = 0; kk < kt; ++kk) {
          T av[5], bv[5];
#pragma unroll
          for (int a = 0; a < 5; ++a) av[a] = As[kk * TILE + ty + 16 * a];
#pragma unroll
          for (int b = 0; b < 5; ++b) bv[b] = Bs[kk * TILE + tx + 16 * b];
#pragma unroll
          for (int a = 0; a < 5; ++a)
#pragma unroll
            for (int b = 0; b < 5; ++b) acc[a][b] += av[a] * bv[b];
        }
      }
#pragma unroll
      for (int a = 0; a < 5; ++a) {
#pragma unroll
        for (int b = 0; b < 5; ++b) {
          const int i = ty + 16 * a, j = tx + 16 * b;
          if (i < mt && j < nt) {
            T v = alpha * acc[a][b];
            if (C0) v += beta * C0[(size_t)(i0 + i) * ldc0 + j0 + j];
            if (addI && (i0 + i) == (j0 + j)) v += T(1);
            C[(size_t)(i0 + i) * ldc + j0 + j] = v;
          }
        }
      }
    }
  }
  __syncthreads();
}

// Y = X (copy an m x n block), optional transpose (Y = X^T, Y is n x m).
template <typename T>
__device__ void cta_copy(int m, int n, const T* X, int ldxs, bool trans, T* Y, int ldy) {
  for (int e = threadIdx.x; e < m * n; e += NT) {
    const int i = e / n, j = e - i * n;
    if (!trans) Y[(size_t)i * ldy + j] = X[(size_t)i * ldxs + j];
    else Y[(size_t)j * ldy + i] = X[(size_t)i * ldxs + j];
  }
  __syncthreads();
}

// Y = I (n x n) or Y = 0 (m x n).
template <typename T>
__device__ void cta_eye(int n, T* Y, int ldy) {
  for (int e = threadIdx.x; e < n * n; e += NT) {
    const int i = e / n, j = e - i * n;
    Y[(size_t)i * ldy + j] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
}

template <typename T>
__device__ void cta_zero(int m, int n, T* Y, int ldy) {
  for (int e = threadIdx.x; e < m * n; e += NT) {
    const int i = e / n, j = e - i * n;
    Y[(size_t)i * ldy + j] = T(0);
  }
  __syncthreads();
}

// In-place Gauss-Jordan inversion of the n x n matrix M (shared memory, leading
// dimension ldm).  pivot = true: partial (row) pivoting, failure if a pivot is
// below tiny_pivot.  pivot = false: no pivoting, failure if a pivot is not
// positive (the test that the matrix is symmetric positive definite).
// Returns 0 on success, 1 on failure (M is then garbage).
// buf: shared scratch of 2*TILE elements; perm: shared int[TILE]; flag: shared int.
template <typename T>
__device__ __noinline__ int cta_inverse(T* M, int ldm, int n, bool pivot, T* buf, int* perm, int* flag) {
  const int t = threadIdx.x;
  T* rowb = buf;
  T* colb = buf + TILE;
  if (t == 0) *flag = 0;
  __syncthreads();
  for (int kp = 0; kp < n; ++kp) {
    if (pivot) {
      if (t < 32) {
        T best = T(-1);
        int bi = kp;
        for (int i = kp + t; i < n; i += 32) {
          const T v = fabs(M[i * ldm + kp]);
          if (v > best) { best = v; bi = i; }
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) {
          const T ob = __shfl_down_sync(0xffffffffu, best, off);
          const int oi = __shfl_down_sync(0xffffffffu, bi, off);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (t == 0) perm[kp] = bi;
      }
      __syncthreads();
      const int p = perm[kp];
      if (p != kp) {
        for (int j = t; j < n; j += NT) {
          const T a = M[kp * ldm + j];
          M[kp * ldm + j] = M[p * ldm + j];
          M[p * ldm + j] = a;
        }
      }
      __syncthreads();
    }
    T piv = M[kp * ldm + kp];
    const bool bad = pivot ? !(fabs(piv) > tiny_pivot<T>()) : !(piv > T(0));
    if (bad) {
      if (t == 0) *flag = 1;
      piv = T(1);
    }
    const T ip = T(1) / piv;
    for (int j = t; j < n; j += NT) {
      rowb[j] = (j == kp) ? ip : M[kp * ldm + j] * ip;
      colb[j] = M[j * ldm + kp];
    }
    __syncthreads();
    for (int e = t; e < n * n; e += NT) {
      const int i = e / n, j = e - i * n;
      T v;
      if (i == kp) v = rowb[j];
      else if (j == kp) v = -colb[i] * ip;
      else v = M[i * ldm + j] - colb[i] * rowb[j];
      M[i * ldm + j] = v;
    }
    __syncthreads();
  }
  if (pivot) {
    for (int kp = n - 1; kp >= 0; --kp) {
      const int p = perm[kp];
      if (p != kp) {
        for (int i = t; i < n; i += NT) {
          const T a = M[i * ldm + kp];
          M[i * ldm + kp] = M[i * ldm + p];
          M[i * ldm + p] = a;
        }
      }
      __syncthreads();
    }
  }
  const int f = *flag;
  __syncthreads();
  return f;
}

// ---------------------------------------------------------------------------
// Warp helpers
// ---------------------------------------------------------------------------
template <typename T>
__device__ inline T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

template <typename T>
__device__ inline T warp_max(T v) {
#pragma unroll
  for (int off = 16; off; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

// dot(a, x) over n entries by one warp; result in every lane.
template <typename T>
__device__ inline T warp_dot(const T* a, const T* x, int n) {
  const int l = threadIdx.x & 31;
  T s = T(0);
  for (int j = l; j < n; j += 32) s += a[j] * x[j];
  return warp_sum(s);
}

// ---------------------------------------------------------------------------
// cp.async staging (16-byte chunks, L2 -> shared), used to prefetch the
// per-stage matrices of the dependent scan chains.
// ---------------------------------------------------------------------------
__device__ inline void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ inline void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Issue the copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// from global to shared by the whole CTA.
__device__ inline void cta_stage(void* dst, const void* src, int bytes) {
  const int n16 = bytes >> 4;
  const char* s = (const char*)src;
  char* d = (char*)dst;
  for (int i = threadIdx.x; i < n16; i += NT) cp_async16(d + 16 * i, s + 16 * i);
}

// y = M^T x + c  (M: rows x cols in shared memory, leading dim ld; x: rows;
// y, c: cols; y, x, c in shared memory; y must not alias x).  red: shared
// scratch of NT elements.
template <typename T>
__device__ void smem_mvT(const T* M, int ld, int rows, int cols, const T* x, const T* c, T* y, T* red) {
  const int t = threadIdx.x;
  const int W = rup16(cols);
  const int G = NT / W;
  const int j = t % W, g = t / W;
  if (g < G && j < cols) {
    T s = T(0);
    for (int i = g; i < rows; i += G) s += M[i * ld + j] * x[i];
    red[g * W + j] = s;
  }
  __syncthreads();
  if (t < cols) {
    T s = c ? c[t] : T(0);
    for (int gg = 0; gg < G; ++gg) s += red[gg * W + t];
    y[t] = s;
  }
  __syncthreads();
}

// y = M x + c  (M rows x cols in shared memory) -- one warp per row.
template <typename T>
__device__ void smem_mv(const T* M, int ld, int rows, int cols, const T* x, const T* c, T* y) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int i = w; i < rows; i += NT / 32) {
    T s = T(0);
    for (int jj = l; jj < cols; jj += 32) s += M[i * ld + jj] * x[jj];
    s = warp_sum(s);
    if (l == 0) y[i] = s + (c ? c[i] : T(0));
  }
  __syncthreads();
}

}  // namespace gsls
