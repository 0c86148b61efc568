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
constexpr int KT = 64;      // k-slab staged per step of the CTA GEMM (whole k for k <= 64)
constexpr int GJ_LD = TILE + 1;

__host__ __device__ inline int rup4(int x) { return (x + 3) & ~3; }
__host__ __device__ inline int rup16(int x) { return (x + 15) & ~15; }

template <typename T> __device__ inline T tiny_pivot();
template <> __device__ inline double tiny_pivot<double>() { return 1e-280; }
template <> __device__ inline float tiny_pivot<float>() { return 1e-30f; }

// Shared-memory scratch needed by cta_gemm: 2*KT*TILE elements (op(A) and
// op(B) k-slabs stored k-major).
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
        // one burst of independent loads per operand, 16 x 16 thread grid,
        // coalesced along the contiguous index of each operand
        if (!tA) {
          for (int i = ty; i < mt; i += 16)
            for (int kk = tx; kk < kt; kk += 16) As[kk * TILE + i] = A[(size_t)(i0 + i) * lda + k0 + kk];
        } else {
          for (int kk = ty; kk < kt; kk += 16)
            for (int i = tx; i < mt; i += 16) As[kk * TILE + i] = A[(size_t)(k0 + kk) * lda + i0 + i];
        }
        if (!tB) {
          for (int kk = ty; kk < kt; kk += 16)
            for (int j = tx; j < nt; j += 16) Bs[kk * TILE + j] = B[(size_t)(k0 + kk) * ldb + j0 + j];
        } else {
          for (int j = ty; j < nt; j += 16)
            for (int kk = tx; kk < kt; kk += 16) Bs[kk * TILE + j] = B[(size_t)(j0 + j) * ldb + k0 + kk];
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

// Gauss-Jordan inversion of the n x n matrix held in shared memory S (leading
// dimension lds), written to Wout (leading dimension ldw; shared or global).
// S is destroyed.  pivot = true: partial pivoting over the not-yet-used rows
// (the pivot row is recorded instead of swapped, and the result gathered
// through the permutation at the end); failure if a pivot is below
// tiny_pivot.  pivot = false: pivots taken on the diagonal, failure if one is
// not positive (the test that the matrix is symmetric positive definite).
// Returns 0 on success, 1 on failure.
// Thread map: warp w owns rows i = w (mod 8); lane l owns columns l, l+32, l+64.
// One step = [read pivot row and column into registers] barrier [update,
// and the owners of column k+1 propose its pivot candidates] barrier.
// buf: shared scratch of 2*TILE elements (candidate values and rows);
// perm: shared int[2*TILE]; flag: shared int[2].
template <typename T>
__device__ __noinline__ int cta_inverse(T* S, int lds, int n, bool pivot, T* Wout, int ldw, T* buf, int* perm,
                                        int* flag) {
  const int t = threadIdx.x, w = t >> 5, l = t & 31;
  int* used = perm + TILE;       // used[i]: physical row i already a pivot row
  T* cval = buf;                 // per-warp candidate |value|
  int* cand_row = reinterpret_cast<int*>(buf + TILE);
  if (t == 0) flag[0] = 0;
  for (int i = t; i < n; i += NT) used[i] = 0;
  __syncthreads();
  // candidates for column 0
  if (pivot && l == 0) {
    T best = T(-1);
    int bi = -1;
    for (int i = w; i < n; i += 8) {
      const T v = fabs(S[i * lds]);
      if (v > best) { best = v; bi = i; }
    }
    cval[w] = best;
    cand_row[w] = bi;
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    int p = k;
    if (pivot) {
      T best = T(-1);
      for (int q = 0; q < 8; ++q) {
        const int r = cand_row[q];
        const T v = cval[q];
        if (r >= 0 && (v > best || (v == best && r < p))) { best = v; p = r; }
      }
    }
    T piv = S[p * lds + k];
    const bool bad = pivot ? !(fabs(piv) > tiny_pivot<T>()) : !(piv > T(0));
    if (bad) piv = T(1);
    const T ip = T(1) / piv;
    // registers: pivot row entries of own columns, column-k entries of own rows
    T rowp[3], colk[10];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int j = l + 32 * c;
      rowp[c] = (j < n) ? S[p * lds + j] : T(0);
    }
#pragma unroll
    for (int a = 0; a < 10; ++a) {
      const int i = w + 8 * a;
      colk[a] = (i < n) ? S[i * lds + k] : T(0);
    }
    if (t == 0) {
      perm[k] = p;
      used[p] = 1;
      if (bad) flag[0] = 1;
    }
    __syncthreads();
    T best = T(-1);
    int bi = -1;
#pragma unroll
    for (int a = 0; a < 10; ++a) {
      const int i = w + 8 * a;
      if (i < n) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int j = l + 32 * c;
          if (j < n) {
            T v;
            if (i == p) v = (j == k) ? ip : rowp[c] * ip;
            else if (j == k) v = -colk[a] * ip;
            else v = S[i * lds + j] - colk[a] * rowp[c] * ip;
            S[i * lds + j] = v;
            if (pivot && j == k + 1 && !used[i]) {
              const T av = fabs(v);
              if (av > best) { best = av; bi = i; }
            }
          }
        }
      }
    }
    if (pivot && k + 1 < n && l == ((k + 1) & 31)) {
      cval[w] = best;
      cand_row[w] = bi;
    }
    __syncthreads();
  }
  // gather: W[a][b] = S[perm[a]][iperm[b]], iperm[perm[c]] = c (identity without pivoting)
  int* iperm = used;
  if (pivot) {
    for (int c = t; c < n; c += NT) iperm[perm[c]] = c;
  }
  __syncthreads();
  for (int a = w; a < n; a += 8) {
    const int ra = pivot ? perm[a] : a;
    for (int b = l; b < n; b += 32) Wout[a * ldw + b] = S[ra * lds + (pivot ? iperm[b] : b)];
  }
  __syncthreads();
  const int f = flag[0];
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

// Column sweep of one output: sum_{r < R} S[r * ld + j] x[r], four
// independent accumulators (consecutive j across a warp read consecutive
// shared-memory words).
template <typename T>
__device__ inline T col_dot(const T* S, int ld, int R, int j, const T* x) {
  T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
  int r = 0;
  for (; r + 3 < R; r += 4) {
    a0 += S[r * ld + j] * x[r];
    a1 += S[(r + 1) * ld + j] * x[r + 1];
    a2 += S[(r + 2) * ld + j] * x[r + 2];
    a3 += S[(r + 3) * ld + j] * x[r + 3];
  }
  for (; r < R; ++r) a0 += S[r * ld + j] * x[r];
  return (a0 + a1) + (a2 + a3);
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
