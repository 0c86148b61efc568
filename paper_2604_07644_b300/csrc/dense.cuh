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

// 16-byte vector of T (VW elements)
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int W = 2; };

template <typename T> __device__ inline T tiny_pivot();
template <> __device__ inline double tiny_pivot<double>() { return 1e-280; }
template <> __device__ inline float tiny_pivot<float>() { return 1e-30f; }

// Shared-memory scratch needed by cta_gemm: 2*KT*TILE elements (op(A) and
// op(B) k-slabs stored k-major).
template <typename T> constexpr int gemm_smem_elems() { return 2 * KT * TILE; }

// TF32 tensor-core pieces (the GPUSLS_TF32 precision mode): operands rounded
// to TF32, mma.sync m16n8k8 with FP32 accumulation.
__device__ inline unsigned tf32_rna(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(r) : "f"(x));
  return r;
}
__device__ inline void mma_tf32(float* c, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
constexpr int GEMM_NB = 4;   // n8 tiles per warp strip (16 x 32 outputs) of the TF32 path

// One element global -> shared without a register round trip (4 or 8
// bytes), so a thread's staging loads are all in flight at once.
template <typename T>
__device__ inline void cp_async_elem(T* dst_smem, const T* src_global) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  if (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src_global) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src_global) : "memory");
}

// dst[e] = f(e) for e < total by the whole CTA, eight elements per thread per
// round with all eight (independent) loads issued before the stores, so that
// global-memory latency is paid once per round rather than once per element.
template <typename T, typename F>
__device__ inline void cta_fill(T* dst, int total, F f) {
  for (int base = threadIdx.x; base < total; base += 8 * NT) {
    T v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = base + u * NT;
      v[u] = e < total ? f(e) : T(0);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = base + u * NT;
      if (e < total) dst[e] = v[u];
    }
  }
}

// acc[a][b] += sum_kk As[kk][ty + 16 a] Bs[kk][tx + 16 b] for a < RA, b < RB.
template <typename T, int RA, int RB>
__device__ __forceinline__ void gemm_mac(const T* As, const T* Bs, int kt, int ty, int tx, T (&acc)[5][5]) {
  for (int kk = 0; kk < kt; ++kk) {
    T av[RA], bv[RB];
#pragma unroll
    for (int a = 0; a < RA; ++a) av[a] = As[kk * TILE + ty + 16 * a];
#pragma unroll
    for (int b = 0; b < RB; ++b) bv[b] = Bs[kk * TILE + tx + 16 * b];
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
      for (int b = 0; b < RB; ++b) acc[a][b] += av[a] * bv[b];
  }
}

template <typename T, int RA>
__device__ __forceinline__ void gemm_mac_rb(int rb, const T* As, const T* Bs, int kt, int ty, int tx,
                                            T (&acc)[5][5]) {
  switch (rb) {
    case 1: gemm_mac<T, RA, 1>(As, Bs, kt, ty, tx, acc); break;
    case 2: gemm_mac<T, RA, 2>(As, Bs, kt, ty, tx, acc); break;
    case 3: gemm_mac<T, RA, 3>(As, Bs, kt, ty, tx, acc); break;
    case 4: gemm_mac<T, RA, 4>(As, Bs, kt, ty, tx, acc); break;
    default: gemm_mac<T, RA, 5>(As, Bs, kt, ty, tx, acc); break;
  }
}

template <typename T>
__device__ __forceinline__ void gemm_mac_dispatch(int ra, int rb, const T* As, const T* Bs, int kt, int ty, int tx,
                                                  T (&acc)[5][5]) {
  switch (ra) {
    case 1: gemm_mac_rb<T, 1>(rb, As, Bs, kt, ty, tx, acc); break;
    case 2: gemm_mac_rb<T, 2>(rb, As, Bs, kt, ty, tx, acc); break;
    case 3: gemm_mac_rb<T, 3>(rb, As, Bs, kt, ty, tx, acc); break;
    case 4: gemm_mac_rb<T, 4>(rb, As, Bs, kt, ty, tx, acc); break;
    default: gemm_mac_rb<T, 5>(rb, As, Bs, kt, ty, tx, acc); break;
  }
}

// C = alpha * op(A) * op(B) + beta * C0 (+ I if addI), with op(A) m x k and
// op(B) k x n.  tA: A is stored k x m (op(A) = A^T); tB likewise.  C may alias
// C0 but not A or B.  C0 may be null.  Operands may live in global or shared
// memory.  Any m, n (tiled by TILE), any k.  Operands are staged k-major in
// shared memory.  tc = false (or FP64): 5 x 5 register tiles per thread on a
// 16 x 16 thread grid.  tc = true (FP32 only): TF32 tensor-core MMAs, one
// 16 x 32 strip per warp.
template <typename T>
__device__ __noinline__ void cta_gemm(int m, int n, int k, T alpha,
                         const T* A, int lda, bool tA,
                         const T* B, int ldb, bool tB,
                         T beta, const T* C0, int ldc0, bool addI,
                         T* C, int ldc, T* sm, bool tc = false) {
  T* As = sm;               // As[kk * TILE + i] = op(A)[i][kk]
  T* Bs = sm + KT * TILE;   // Bs[kk * TILE + j] = op(B)[kk][j]
  const int t = threadIdx.x;
  const int ty = t >> 4, tx = t & 15;
  const bool gA = __isGlobal(A) != 0, gB = __isGlobal(B) != 0;
  const bool TC = tc && sizeof(T) == 4;
  const int lane = t & 31, w = t >> 5, gid = lane >> 2, tig = lane & 3;
  for (int i0 = 0; i0 < m; i0 += TILE) {
    for (int j0 = 0; j0 < n; j0 += TILE) {
      const int mt = min(TILE, m - i0), nt = min(TILE, n - j0);
      T acc[5][5];
      float fr[2][GEMM_NB][4];
      const int mt16 = (mt + 15) >> 4, nt8 = (nt + 7) >> 3;
      const int nstrip_n = (nt8 + GEMM_NB - 1) / GEMM_NB, nstrips = mt16 * nstrip_n;
#pragma unroll
      for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int b = 0; b < 5; ++b) acc[a][b] = T(0);
#pragma unroll
      for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
        for (int q = 0; q < GEMM_NB; ++q)
#pragma unroll
          for (int e = 0; e < 4; ++e) fr[s2][q][e] = 0.f;
      for (int k0 = 0; k0 < k; k0 += KT) {
        const int kt = min(KT, k - k0);
        const int kt8 = (kt + 7) & ~7;
        __syncthreads();
        // 16 x 16 thread grid, coalesced along the contiguous index of each
        // operand; global operands go by cp.async (every load of a thread in
        // flight at once), shared ones by plain copies
        if (!tA) {
          for (int i = ty; i < mt; i += 16)
            for (int kk = tx; kk < kt; kk += 16) {
              const T* src = A + (size_t)(i0 + i) * lda + k0 + kk;
              if (gA) cp_async_elem(As + kk * TILE + i, src);
              else As[kk * TILE + i] = *src;
            }
        } else {
          for (int kk = ty; kk < kt; kk += 16)
            for (int i = tx; i < mt; i += 16) {
              const T* src = A + (size_t)(k0 + kk) * lda + i0 + i;
              if (gA) cp_async_elem(As + kk * TILE + i, src);
              else As[kk * TILE + i] = *src;
            }
        }
        if (!tB) {
          for (int kk = ty; kk < kt; kk += 16)
            for (int j = tx; j < nt; j += 16) {
              const T* src = B + (size_t)(k0 + kk) * ldb + j0 + j;
              if (gB) cp_async_elem(Bs + kk * TILE + j, src);
              else Bs[kk * TILE + j] = *src;
            }
        } else {
          for (int j = ty; j < nt; j += 16)
            for (int kk = tx; kk < kt; kk += 16) {
              const T* src = B + (size_t)(j0 + j) * ldb + k0 + kk;
              if (gB) cp_async_elem(Bs + kk * TILE + j, src);
              else Bs[kk * TILE + j] = *src;
            }
        }
        if (TC) {
          // zero the k-padding up to a multiple of 8 and the row / column
          // padding of the 16 x 8 fragments (stale values could be Inf / NaN)
          for (int e = t; e < (kt8 - kt) * TILE; e += NT) {
            As[kt * TILE + e] = T(0);
            Bs[kt * TILE + e] = T(0);
          }
          for (int e = t; e < kt8 * 16; e += NT) {
            const int kk = e >> 4, r = e & 15;
            if (mt + r < TILE && mt + r < 16 * mt16) As[kk * TILE + mt + r] = T(0);
            if (nt + r < TILE && nt + r < 8 * nt8) Bs[kk * TILE + nt + r] = T(0);
          }
        }
        if (gA || gB) {
          cp_async_commit();
          cp_async_wait<0>();
        }
        __syncthreads();
        if (TC) {
          // fragments (m16n8k8, tf32): A row gid / gid+8, col tig / tig+4;
          // B row tig / tig+4, col gid; C rows gid / gid+8, cols 2 tig, 2 tig+1
          for (int s2 = 0; s2 < 2; ++s2) {
            const int st = w + 8 * s2;
            if (st < nstrips) {
              const int r0 = (st / nstrip_n) * 16, c0 = (st % nstrip_n) * (8 * GEMM_NB);
              for (int k8 = 0; k8 < kt8; k8 += 8) {
                const float* a_lo = reinterpret_cast<const float*>(As) + (k8 + tig) * TILE + r0 + gid;
                const float* a_hi = a_lo + 4 * TILE;
                const unsigned af[4] = {tf32_rna(a_lo[0]), tf32_rna(a_lo[8]), tf32_rna(a_hi[0]), tf32_rna(a_hi[8])};
#pragma unroll
                for (int q = 0; q < GEMM_NB; ++q) {
                  const int cb = c0 + 8 * q;
                  if (cb < 8 * nt8) {
                    const float* b_lo = reinterpret_cast<const float*>(Bs) + (k8 + tig) * TILE + cb + gid;
                    const unsigned bf[2] = {tf32_rna(b_lo[0]), tf32_rna(b_lo[4 * TILE])};
                    mma_tf32(fr[s2][q], af, bf);
                  }
                }
              }
            }
          }
        } else {
          // register tile sized to the block: rows ty + 16 a for a < RA =
          // ceil(mt / 16), columns tx + 16 b for b < RB = ceil(nt / 16), so no
          // arithmetic is spent on padding rows or columns
          gemm_mac_dispatch<T>((mt + 15) >> 4, (nt + 15) >> 4, As, Bs, kt, ty, tx, acc);
        }
      }
      if (TC) {
        for (int s2 = 0; s2 < 2; ++s2) {
          const int st = w + 8 * s2;
          if (st < nstrips) {
            const int r0 = (st / nstrip_n) * 16, c0 = (st % nstrip_n) * (8 * GEMM_NB);
#pragma unroll
            for (int q = 0; q < GEMM_NB; ++q) {
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const int i = r0 + gid + (e >> 1) * 8, j = c0 + 8 * q + 2 * tig + (e & 1);
                if (i < mt && j < nt) {
                  T v = alpha * (T)fr[s2][q][e];
                  if (C0) v += beta * C0[(size_t)(i0 + i) * ldc0 + j0 + j];
                  if (addI && (i0 + i) == (j0 + j)) v += T(1);
                  C[(size_t)(i0 + i) * ldc + j0 + j] = v;
                }
              }
            }
          }
        }
        continue;
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

// ---------------------------------------------------------------------------
// Register-tile GEMM on operands already in place (normally shared memory):
// no staging copies.  16 x 16 thread grid; thread (ty, tx) owns output rows
// ty + 16 a (a < ceil(m / 16)) and columns tx + 16 b (b < ceil(n / 16)).
// Every output is computed into registers before any is stored, with a CTA
// barrier in between, so the output may alias A, B or C0.
// ---------------------------------------------------------------------------
// One product term op(A) B with op(A) m x k (tA: A stored k x m) and B k x n.
template <typename T>
struct MTerm {
  const T* A;
  int lda;
  bool tA;
  const T* B;
  int ldb;
  int k;   // 0: no term
};

// acc[a][b] += sum_kk op(A)[ty + 16 a][kk] B[kk][tx + 16 b].  Row and column
// indices past m / n are clamped to m - 1 / n - 1 (their sums are discarded),
// so no read leaves the operands.
template <typename T, int RA, int RB, bool TA>
__device__ __forceinline__ void rt_mac(int m, int n, int k, const T* A, int lda, const T* B, int ldb,
                                       T (&acc)[5][5]) {
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const T* pa[RA];
  const T* pb[RB];
#pragma unroll
  for (int a = 0; a < RA; ++a) {
    const int i = min(ty + 16 * a, m - 1);
    pa[a] = TA ? A + i : A + (size_t)i * lda;
  }
#pragma unroll
  for (int b = 0; b < RB; ++b) pb[b] = B + min(tx + 16 * b, n - 1);
  const int sa = TA ? lda : 1;
#pragma unroll 2
  for (int kk = 0; kk < k; ++kk) {
    T av[RA], bv[RB];
#pragma unroll
    for (int a = 0; a < RA; ++a) av[a] = pa[a][kk * sa];
#pragma unroll
    for (int b = 0; b < RB; ++b) bv[b] = pb[b][kk * ldb];
#pragma unroll
    for (int a = 0; a < RA; ++a)
#pragma unroll
      for (int b = 0; b < RB; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
  }
}

template <typename T, int RA, bool TA>
__device__ __forceinline__ void rt_mac_rb(int rb, int m, int n, const MTerm<T>& p, T (&acc)[5][5]) {
  switch (rb) {
    case 1: rt_mac<T, RA, 1, TA>(m, n, p.k, p.A, p.lda, p.B, p.ldb, acc); break;
    case 2: rt_mac<T, RA, 2, TA>(m, n, p.k, p.A, p.lda, p.B, p.ldb, acc); break;
    case 3: rt_mac<T, RA, 3, TA>(m, n, p.k, p.A, p.lda, p.B, p.ldb, acc); break;
    case 4: rt_mac<T, RA, 4, TA>(m, n, p.k, p.A, p.lda, p.B, p.ldb, acc); break;
    default: rt_mac<T, RA, 5, TA>(m, n, p.k, p.A, p.lda, p.B, p.ldb, acc); break;
  }
}

template <typename T, bool TA>
__device__ __forceinline__ void rt_mac_dispatch(int m, int n, const MTerm<T>& p, T (&acc)[5][5]) {
  const int ra = (m + 15) >> 4, rb = (n + 15) >> 4;
  switch (ra) {
    case 1: rt_mac_rb<T, 1, TA>(rb, m, n, p, acc); break;
    case 2: rt_mac_rb<T, 2, TA>(rb, m, n, p, acc); break;
    case 3: rt_mac_rb<T, 3, TA>(rb, m, n, p, acc); break;
    case 4: rt_mac_rb<T, 4, TA>(rb, m, n, p, acc); break;
    default: rt_mac_rb<T, 5, TA>(rb, m, n, p, acc); break;
  }
}

// Vectorized register-tile body.  Thread t -> (ty, tx) = (t / GX, t % GX) of
// a GY x GX grid (GY = NT / GX); it owns rows ty + GY a (a < RA) and the
// 4-column groups starting at 4 tx + 4 GX bb (bb < RB).  B is read as 16-byte
// vectors along the columns; A (not transposed) as vectors along k, four
// k-steps per load, with a scalar tail for k % 4; a transposed A by scalars.
// Groups and rows past n / m are clamped onto the last valid ones for the
// reads and skipped by the stores.  Requires 16-byte aligned A, B and leading
// dims that are multiples of 4 elements (checked by the caller).
template <typename T>
__device__ __forceinline__ void ld4(const T* p, T* v) {
  using V16 = typename Vec16<T>::type;
  constexpr int VW = Vec16<T>::W;
#pragma unroll
  for (int h = 0; h < 4; h += VW) *reinterpret_cast<V16*>(v + h) = *reinterpret_cast<const V16*>(p + h);
}
template <typename T>
__device__ __forceinline__ void st4(T* p, const T* v) {
  using V16 = typename Vec16<T>::type;
  constexpr int VW = Vec16<T>::W;
#pragma unroll
  for (int h = 0; h < 4; h += VW) *reinterpret_cast<V16*>(p + h) = *reinterpret_cast<const V16*>(v + h);
}

template <typename T, int GX, int RA, int RB, bool TA>
__device__ __forceinline__ void mk_mac(int m, int n, const MTerm<T>& p, T (&acc)[RA][RB][4]) {
  constexpr int GY = NT / GX;
  const int ty = threadIdx.x / GX, tx = threadIdx.x % GX;
  const int k = p.k, lda = p.lda, ldb = p.ldb;
  const int lastg = (n - 1) & ~3;
  const T* pa[RA];
  const T* pb[RB];
#pragma unroll
  for (int a = 0; a < RA; ++a) {
    const int i = min(ty + GY * a, m - 1);
    pa[a] = TA ? p.A + i : p.A + (size_t)i * lda;
  }
#pragma unroll
  for (int bb = 0; bb < RB; ++bb) pb[bb] = p.B + min(4 * tx + 4 * GX * bb, lastg);
  if (!TA) {
    const int k4 = k & ~3;
#pragma unroll 1
    for (int kk = 0; kk < k4; kk += 4) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        T bv[RB][4];
#pragma unroll
        for (int bb = 0; bb < RB; ++bb) ld4<T>(pb[bb] + (size_t)(kk + q) * ldb, bv[bb]);
#pragma unroll
        for (int a = 0; a < RA; ++a) {
          const T aq = pa[a][kk + q];
#pragma unroll
          for (int bb = 0; bb < RB; ++bb)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][bb][c] = fma(aq, bv[bb][c], acc[a][bb][c]);
        }
      }
    }
    for (int kk = k4; kk < k; ++kk) {
      T bv[RB][4];
#pragma unroll
      for (int bb = 0; bb < RB; ++bb) ld4<T>(pb[bb] + (size_t)kk * ldb, bv[bb]);
#pragma unroll
      for (int a = 0; a < RA; ++a) {
        const T av = pa[a][kk];
#pragma unroll
        for (int bb = 0; bb < RB; ++bb)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[a][bb][c] = fma(av, bv[bb][c], acc[a][bb][c]);
      }
    }
  } else {
#pragma unroll 2
    for (int kk = 0; kk < k; ++kk) {
      T av[RA], bv[RB][4];
#pragma unroll
      for (int a = 0; a < RA; ++a) av[a] = pa[a][(size_t)kk * lda];
#pragma unroll
      for (int bb = 0; bb < RB; ++bb) ld4<T>(pb[bb] + (size_t)kk * ldb, bv[bb]);
#pragma unroll
      for (int a = 0; a < RA; ++a)
#pragma unroll
        for (int bb = 0; bb < RB; ++bb)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[a][bb][c] = fma(av[a], bv[bb][c], acc[a][bb][c]);
    }
  }
}

// Each shape is its own (non-inlined) function so that its registers are
// allocated for it alone.
template <typename T, int GX, int RA, int RB>
__device__ __noinline__ void sgemm_vec(int m, int n, T alpha, const MTerm<T> p1, const MTerm<T> p2, T beta,
                                       const T* C0, int ldc0, bool addI, T* C, int ldc, bool tC) {
  constexpr int GY = NT / GX;
  constexpr bool PRE = RA * RB <= 4;   // C0 prefetched into registers when they allow
  const int ty = threadIdx.x / GX, tx = threadIdx.x % GX;
  T acc[RA][RB][4];
  T c0v[PRE ? RA : 1][PRE ? RB : 1][4];
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int bb = 0; bb < RB; ++bb)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        acc[a][bb][c] = T(0);
        if (PRE) {
          const int i = ty + GY * a, j = 4 * tx + 4 * GX * bb + c;
          c0v[PRE ? a : 0][PRE ? bb : 0][c] = (C0 && i < m && j < n) ? C0[(size_t)i * ldc0 + j] : T(0);
        }
      }
  if (p1.k > 0) {
    if (p1.tA) mk_mac<T, GX, RA, RB, true>(m, n, p1, acc);
    else mk_mac<T, GX, RA, RB, false>(m, n, p1, acc);
  }
  if (p2.k > 0) {
    if (p2.tA) mk_mac<T, GX, RA, RB, true>(m, n, p2, acc);
    else mk_mac<T, GX, RA, RB, false>(m, n, p2, acc);
  }
  __syncthreads();   // every operand read before any output is written
  const bool vst = !tC && ((reinterpret_cast<uintptr_t>(C) & 15) == 0) && (ldc & 3) == 0;
#pragma unroll
  for (int a = 0; a < RA; ++a) {
    const int i = ty + GY * a;
    if (i >= m) continue;
#pragma unroll
    for (int bb = 0; bb < RB; ++bb) {
      const int j0 = 4 * tx + 4 * GX * bb;
      if (j0 >= n) continue;
      T v[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = j0 + c;
        T c0 = T(0);
        if (PRE) c0 = c0v[PRE ? a : 0][PRE ? bb : 0][c];
        else if (C0 && j < n) c0 = C0[(size_t)i * ldc0 + j];
        v[c] = alpha * acc[a][bb][c] + beta * c0;
        if (addI && i == j) v[c] += T(1);
      }
      if (vst && j0 + 3 < n) {
        st4<T>(C + (size_t)i * ldc + j0, v);
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int j = j0 + c;
          if (j < n) {
            if (tC) C[(size_t)j * ldc + i] = v[c];
            else C[(size_t)i * ldc + j] = v[c];
          }
        }
      }
    }
  }
  __syncthreads();
}

// 64 < n <= 80: the 16 x 16 grid's four vector columns per thread (0 .. 63)
// plus one scalar column 64 + tx, so 80 columns are covered with 88 % of the
// threads' outputs in use at n = 75 (two vector column groups would cover 128
// columns at 55 %).  The scalar column reuses the A values of the vector
// k-loop.
template <typename T, int RA, bool TA>
__device__ __forceinline__ void mk_mac_ex(int m, int n, const MTerm<T>& p, T (&acc)[RA][4], T (&ex)[RA]) {
  constexpr int GX = 16, GY = NT / GX;
  const int ty = threadIdx.x / GX, tx = threadIdx.x % GX;
  const int k = p.k, lda = p.lda, ldb = p.ldb;
  const T* const A = p.A;
  const T* const pb = p.B + 4 * tx;
  const T* const px = p.B + min(64 + tx, n - 1);
  int oa[RA];   // 32-bit row offsets keep the five-row tile in registers
#pragma unroll
  for (int a = 0; a < RA; ++a) {
    const int i = min(ty + GY * a, m - 1);
    oa[a] = TA ? i : i * lda;
  }
  if (!TA) {
    const int k4 = k & ~3;
#pragma unroll 1
    for (int kk = 0; kk < k4; kk += 4) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        T bv[4];
        ld4<T>(pb + (kk + q) * ldb, bv);
        const T bx = px[(kk + q) * ldb];
#pragma unroll
        for (int a = 0; a < RA; ++a) {
          const T aq = A[oa[a] + kk + q];
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[a][c] = fma(aq, bv[c], acc[a][c]);
          ex[a] = fma(aq, bx, ex[a]);
        }
      }
    }
    for (int kk = k4; kk < k; ++kk) {
      T bv[4];
      ld4<T>(pb + kk * ldb, bv);
      const T bx = px[kk * ldb];
#pragma unroll
      for (int a = 0; a < RA; ++a) {
        const T av = A[oa[a] + kk];
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = fma(av, bv[c], acc[a][c]);
        ex[a] = fma(av, bx, ex[a]);
      }
    }
  } else {
#pragma unroll 1
    for (int kk = 0; kk < k; ++kk) {
      T bv[4];
      ld4<T>(pb + kk * ldb, bv);
      const T bx = px[kk * ldb];
#pragma unroll
      for (int a = 0; a < RA; ++a) {
        const T av = A[kk * lda + oa[a]];
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = fma(av, bv[c], acc[a][c]);
        ex[a] = fma(av, bx, ex[a]);
      }
    }
  }
}

template <typename T, int RA>
__device__ __noinline__ void sgemm_vec_ex(int m, int n, T alpha, const MTerm<T> p1, const MTerm<T> p2, T beta,
                                          const T* C0, int ldc0, bool addI, T* C, int ldc, bool tC) {
  constexpr int GX = 16, GY = NT / GX;
  const int ty = threadIdx.x / GX, tx = threadIdx.x % GX;
  T acc[RA][4], ex[RA];
#pragma unroll
  for (int a = 0; a < RA; ++a) {
    ex[a] = T(0);
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = T(0);
  }
  if (p1.k > 0) {
    if (p1.tA) mk_mac_ex<T, RA, true>(m, n, p1, acc, ex);
    else mk_mac_ex<T, RA, false>(m, n, p1, acc, ex);
  }
  if (p2.k > 0) {
    if (p2.tA) mk_mac_ex<T, RA, true>(m, n, p2, acc, ex);
    else mk_mac_ex<T, RA, false>(m, n, p2, acc, ex);
  }
  __syncthreads();   // every operand read before any output is written
  const bool vst = !tC && ((reinterpret_cast<uintptr_t>(C) & 15) == 0) && (ldc & 3) == 0;
  const int jx = 64 + tx;
#pragma unroll
  for (int a = 0; a < RA; ++a) {
    const int i = ty + GY * a;
    if (i >= m) continue;
    const int j0 = 4 * tx;   // < 64 < n: all four columns exist
    T v[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + c;
      v[c] = alpha * acc[a][c] + (C0 ? beta * C0[(size_t)i * ldc0 + j] : T(0));
      if (addI && i == j) v[c] += T(1);
    }
    if (vst) {
      st4<T>(C + (size_t)i * ldc + j0, v);
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = j0 + c;
        if (tC) C[(size_t)j * ldc + i] = v[c];
        else C[(size_t)i * ldc + j] = v[c];
      }
    }
    if (jx < n) {
      T w = alpha * ex[a] + (C0 ? beta * C0[(size_t)i * ldc0 + jx] : T(0));
      if (addI && i == jx) w += T(1);
      if (tC) C[(size_t)jx * ldc + i] = w;
      else C[(size_t)i * ldc + jx] = w;
    }
  }
  __syncthreads();
}

// Scalar register-tile path for operands that are not 16-byte aligned.
template <typename T>
__device__ __noinline__ void sgemm_scalar(int m, int n, T alpha, const MTerm<T> p1, const MTerm<T> p2, T beta,
                                          const T* C0, int ldc0, bool addI, T* C, int ldc, bool tC) {
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  T acc[5][5];
#pragma unroll
  for (int a = 0; a < 5; ++a)
#pragma unroll
    for (int b = 0; b < 5; ++b) acc[a][b] = T(0);
  if (p1.k > 0) {
    if (p1.tA) rt_mac_dispatch<T, true>(m, n, p1, acc);
    else rt_mac_dispatch<T, false>(m, n, p1, acc);
  }
  if (p2.k > 0) {
    if (p2.tA) rt_mac_dispatch<T, true>(m, n, p2, acc);
    else rt_mac_dispatch<T, false>(m, n, p2, acc);
  }
  __syncthreads();   // every operand read before any output is written
#pragma unroll
  for (int a = 0; a < 5; ++a)
#pragma unroll
    for (int b = 0; b < 5; ++b) {
      const int i = ty + 16 * a, j = tx + 16 * b;
      if (i < m && j < n) {
        T v = alpha * acc[a][b] + (C0 ? beta * C0[(size_t)i * ldc0 + j] : T(0));
        if (addI && i == j) v += T(1);
        if (tC) C[(size_t)j * ldc + i] = v;
        else C[(size_t)i * ldc + j] = v;
      }
    }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Tensor-core GEMM with three TF32 products (the GPUSLS_MIXED mode): every
// operand is split a = a_hi + a_lo with a_hi = tf32(a), a_lo = tf32(a - a_hi),
// and op(A) B is accumulated in FP32 as a_lo b_hi + a_hi b_lo + a_hi b_hi by
// mma.sync m16n8k8 (the a_lo b_lo term is below FP32 rounding), which keeps
// FP32 accuracy on the tensor pipe.  Same contract as sgemm_vec: operands in
// place (shared or global memory, any alignment), m, n <= 80, output
// computed before any store (it may alias an operand), optional transposed
// A, transposed output, + I, two product terms.
//   Fragments (PTX ISA, mma.m16n8k8 .tf32, g = lane / 4, q = lane % 4):
//   A 16 x 8: (g, q) (g + 8, q) (g, q + 4) (g + 8, q + 4);  B 8 x 8: (q, g) (q + 4, g);
//   C 16 x 8: (g, 2q) (g, 2q + 1) (g + 8, 2q) (g + 8, 2q + 1).
// Warp w owns units u = w, w + 8 (a unit: one 16-row tile x four 8-column
// tiles); rows, columns and k past the operands are clamped for the reads
// and zeroed in k.
// ---------------------------------------------------------------------------
__device__ inline void split_tf32(float x, unsigned& hi, unsigned& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));
}

__device__ __forceinline__ void tc3_mac(int m, int n, const MTerm<float>& p, int mt, int ng, float (&acc)[4][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const int r0 = mt * 16 + g, r1 = r0 + 8;
  const int ra = min(r0, m - 1), rb = min(r1, m - 1);
  const int k = p.k;
  for (int k0 = 0; k0 < k; k0 += 8) {
    const int ka = k0 + q, kb = k0 + q + 4;
    const bool va = ka < k, vb = kb < k;
    const int kac = min(ka, k - 1), kbc = min(kb, k - 1);
    float av[4];
    if (p.tA) {
      av[0] = p.A[(size_t)kac * p.lda + ra];
      av[1] = p.A[(size_t)kac * p.lda + rb];
      av[2] = p.A[(size_t)kbc * p.lda + ra];
      av[3] = p.A[(size_t)kbc * p.lda + rb];
    } else {
      av[0] = p.A[(size_t)ra * p.lda + kac];
      av[1] = p.A[(size_t)rb * p.lda + kac];
      av[2] = p.A[(size_t)ra * p.lda + kbc];
      av[3] = p.A[(size_t)rb * p.lda + kbc];
    }
    if (!va) av[0] = av[1] = 0.f;
    if (!vb) av[2] = av[3] = 0.f;
    unsigned ah[4], al[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) split_tf32(av[e], ah[e], al[e]);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int col = min((ng * 4 + t) * 8 + g, n - 1);
      float b0 = p.B[(size_t)kac * p.ldb + col];
      float b1 = p.B[(size_t)kbc * p.ldb + col];
      if (!va) b0 = 0.f;
      if (!vb) b1 = 0.f;
      unsigned bh[2], bl[2];
      split_tf32(b0, bh[0], bl[0]);
      split_tf32(b1, bh[1], bl[1]);
      // the three passes of this k-step into a fresh accumulator, added to the
      // running sum by a rounded FP32 add: the tensor core's own accumulation
      // then spans 24 products, not the whole k (measured: it otherwise leaves
      // ~8x the FFMA path's error in the Riccati terms)
      float tmp[4] = {0.f, 0.f, 0.f, 0.f};
      mma_tf32(tmp, al, bh);
      mma_tf32(tmp, ah, bl);
      mma_tf32(tmp, ah, bh);
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[t][e] += tmp[e];
    }
  }
}

static __device__ __noinline__ void sgemm_tc3(int m, int n, float alpha, const MTerm<float> p1, const MTerm<float> p2,
                                       float beta, const float* C0, int ldc0, bool addI, float* C, int ldc, bool tC) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const int mtiles = (m + 15) >> 4, ngroups = (n + 31) >> 5, units = mtiles * ngroups;
  float acc[2][4][4];
#pragma unroll
  for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[s2][t][e] = 0.f;
#pragma unroll
  for (int s2 = 0; s2 < 2; ++s2) {
    const int u = w + 8 * s2;
    if (u < units) {
      const int mt = u / ngroups, ng = u - mt * ngroups;
      if (p1.k > 0) tc3_mac(m, n, p1, mt, ng, acc[s2]);
      if (p2.k > 0) tc3_mac(m, n, p2, mt, ng, acc[s2]);
    }
  }
  __syncthreads();   // every operand read before any output is written
#pragma unroll
  for (int s2 = 0; s2 < 2; ++s2) {
    const int u = w + 8 * s2;
    if (u >= units) continue;
    const int mt = u / ngroups, ng = u - mt * ngroups;
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = mt * 16 + g + (e >= 2 ? 8 : 0);
        const int j = (ng * 4 + t) * 8 + 2 * q + (e & 1);
        if (i < m && j < n) {
          float v = alpha * acc[s2][t][e] + (C0 ? beta * C0[(size_t)i * ldc0 + j] : 0.f);
          if (addI && i == j) v += 1.f;
          if (tC) C[(size_t)j * ldc + i] = v;
          else C[(size_t)i * ldc + j] = v;
        }
      }
  }
  __syncthreads();
}

template <typename T>
__device__ inline bool mterm_vec_ok(const MTerm<T>& p) {
  return p.k == 0 || ((((reinterpret_cast<uintptr_t>(p.A) | reinterpret_cast<uintptr_t>(p.B)) & 15) == 0) &&
                      ((p.lda | p.ldb) & 3) == 0);
}

// C = alpha (op(A1) B1 + op(A2) B2) + beta C0 (+ I if addI), m, n <= 80; the
// second term is skipped when p2.k == 0.  tC: C is written transposed
// (C[j][i]).  C0 (shared or global) is read before the products when the
// registers allow, so its global-memory latency overlaps them.  Ends with a
// CTA barrier.  Operands that are not 16-byte aligned take a scalar path.
// tc (FP32 only, the GPUSLS_MIXED mode): products that give every warp a
// unit (16 rows x 32 columns) and k >= 16 run on the tensor cores in three
// TF32 passes (sgemm_tc3); narrower ones keep the FFMA path, where the
// tensor path would leave warps waiting at the closing barrier.
template <typename T>
__device__ __noinline__ void sgemm(int m, int n, T alpha, MTerm<T> p1, MTerm<T> p2, T beta, const T* C0, int ldc0,
                                   bool addI, T* C, int ldc, bool tC, bool tc = false) {
  if (m <= 0 || n <= 0) {
    __syncthreads();
    return;
  }
  if constexpr (sizeof(T) == 4) {
    if (tc && ((m + 15) >> 4) * ((n + 31) >> 5) >= NT / 32 && p1.k >= 16 && (p2.k == 0 || p2.k >= 16)) {
      sgemm_tc3(m, n, alpha, p1, p2, beta, C0, ldc0, addI, C, ldc, tC);
      return;
    }
  }
  // FP64 products run at the FP64 FMA rate whatever the loads, so FP64 keeps
  // the scalar path (and the vector shapes are instantiated for FP32 only)
  if constexpr (sizeof(T) == 4) {
    if (mterm_vec_ok(p1) && mterm_vec_ok(p2)) {
      if (n <= 16) {
        // narrow outputs: 64 x 4 grid, one column group per thread
        if (m <= 64) sgemm_vec<T, 4, 1, 1>(m, n, alpha, p1, p2, beta, C0, ldc0, addI, C, ldc, tC);
        else sgemm_vec<T, 4, 2, 1>(m, n, alpha, p1, p2, beta, C0, ldc0, addI, C, ldc, tC);
      } else if (n <= 32) {
        // 32 x 8 grid: 32 columns, so fewer idle column groups than the 16 x 16 grid
        if (m <= 32) sgemm_vec<T, 8, 1, 1>(m, n, alpha, p1, p2, beta, C0, ldc0, addI, C, ldc, tC);
        else if (m <= 64) sgemm_vec<T, 8, 2, 1>(m, n, alpha, p1, p2, beta, C0, ldc0, addI, C, ldc, tC);
        else sgemm_vec<T, 8, 3, 1>(m, n, alpha, p1, p2, beta, C0, ldc0, addI, C, ldc, tC);
      } else if (n > 64 && n <= 80) {
        switch ((m + 15) >> 4) {
          case 1: sgemm_vec_ex<T, 1>(m, n, alpha, p1, p2, beta, C0, ldc0, addI, C, ldc, tC); break;
          case 2: sgemm_vec_ex<T, 2>(m, n, alpha, p1, p2, beta, C0, ldc0, addI, C, ldc, tC); break;
          case 3: sgemm_vec_ex<T, 3>(m, n, alpha, p1, p2, beta, C0, ldc0, addI, C, ldc, tC); break;
          case 4: sgemm_vec_ex<T, 4>(m, n, alpha, p1, p2, beta, C0, ldc0, addI, C, ldc, tC); break;
          default: sgemm_vec_ex<T, 5>(m, n, alpha, p1, p2, beta, C0, ldc0, addI, C, ldc, tC); break;
        }
      } else {
        // 32 < n <= 64: the 16 x 16 grid, four columns per thread
        switch ((m + 15) >> 4) {
          case 1: sgemm_vec<T, 16, 1, 1>(m, n, alpha, p1, p2, beta, C0, ldc0, addI, C, ldc, tC); break;
          case 2: sgemm_vec<T, 16, 2, 1>(m, n, alpha, p1, p2, beta, C0, ldc0, addI, C, ldc, tC); break;
          case 3: sgemm_vec<T, 16, 3, 1>(m, n, alpha, p1, p2, beta, C0, ldc0, addI, C, ldc, tC); break;
          case 4: sgemm_vec<T, 16, 4, 1>(m, n, alpha, p1, p2, beta, C0, ldc0, addI, C, ldc, tC); break;
          default: sgemm_vec<T, 16, 5, 1>(m, n, alpha, p1, p2, beta, C0, ldc0, addI, C, ldc, tC); break;
        }
      }
      return;
    }
  }
  sgemm_scalar<T>(m, n, alpha, p1, p2, beta, C0, ldc0, addI, C, ldc, tC);
}

// One-term convenience form.
template <typename T>
__device__ inline void sgemm1(int m, int n, int k, T alpha, const T* A, int lda, bool tA, const T* B, int ldb,
                              T beta, const T* C0, int ldc0, T* C, int ldc, bool tC = false, bool tc = false) {
  sgemm<T>(m, n, alpha, MTerm<T>{A, lda, tA, B, ldb, k}, MTerm<T>{nullptr, 0, false, nullptr, 0, 0}, beta, C0, ldc0,
           false, C, ldc, tC, tc);
}

// Y = X for an m x n block by 16-byte vectors: X, Y 16-byte aligned, leading
// dims multiples of 4 elements.  Columns n .. rup4(n) - 1 of Y are zeroed.
template <typename T>
__device__ void cta_copy_vec(int m, int n, const T* X, int ldxs, T* Y, int ldy) {
  const int c4 = (n + 3) >> 2, tot = m * c4;
  for (int e = threadIdx.x; e < tot; e += NT) {
    const int r = e / c4, cc = (e - r * c4) * 4;
    T v[4];
    ld4<T>(X + (size_t)r * ldxs + cc, v);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (cc + q >= n) v[q] = T(0);
    st4<T>(Y + (size_t)r * ldy + cc, v);
  }
  __syncthreads();
}

// Inverse of a symmetric positive definite n x n matrix, n <= CAP <= 32, by
// warp 0: Gauss-Jordan in place without pivoting (the diagonal pivots of an
// SPD matrix are positive), lane i holding row i in registers and pivot row
// k broadcast by shuffles, n columns per step:
//   g_kk <- 1/p,  g_kj <- g_kj / p,  g_ik <- -g_ik / p,  g_ij <- g_ij - g_ik g_kj / p.
// (Half the work of eliminating [G | I]; in FP64, GPUSLS_MIXED, the FP64
// pipe sets the cost.)  G and Gi: shared or global, may not alias.  Returns
// 1 in every thread (after the closing barrier) if a pivot was not positive.
// flag: shared int.  Loads T, computes in A (GPUSLS_MIXED: FP32 operands,
// FP64 arithmetic), stores T.
template <typename T, typename A, int CAP>
__device__ __noinline__ int warp_spd_inverse_as(const T* G, int ldg, int n, T* Gi, int ldgi, int* flag) {
  if (threadIdx.x < 32) {
    const int l = threadIdx.x;
    A g[CAP];
#pragma unroll
    for (int j = 0; j < CAP; ++j) g[j] = (l < n && j < n) ? (A)G[l * ldg + j] : (l == j ? A(1) : A(0));
    int bad = 0;
#pragma unroll
    for (int k = 0; k < CAP; ++k) {
      if (k < n) {
        A piv = __shfl_sync(0xffffffffu, g[k], k);
        if (!(piv > A(0))) {
          bad = 1;
          piv = A(1);
        }
        const A ip = A(1) / piv;
        const A f = g[k] * ip;   // g_lk / p (this lane's column-k entry before the step)
#pragma unroll
        for (int j = 0; j < CAP; ++j) {
          if (j < n) {
            const A rk = __shfl_sync(0xffffffffu, g[j], k);
            if (l == k) g[j] = j == k ? ip : rk * ip;
            else g[j] = j == k ? -f : fma(-f, rk, g[j]);
          }
        }
      }
    }
    if (l < n) {
#pragma unroll
      for (int j = 0; j < CAP; ++j)
        if (j < n) Gi[l * ldgi + j] = (T)g[j];
    }
    if (l == 0) flag[0] = bad;
  }
  __syncthreads();
  const int f = flag[0];
  __syncthreads();
  return f;
}

// Inverse of a symmetric positive definite n x n matrix by the whole CTA:
// Gauss-Jordan in place in Gi without pivoting (the diagonal pivots of an SPD
// matrix are positive).  Step k copies pivot row and column to prow / pcol
// (shared, >= n elements each), then every thread updates its elements:
//   g_kk <- 1/p,  g_kj <- g_kj / p,  g_ik <- -g_ik / p,  g_ij <- g_ij - g_ik g_kj / p.
// Two CTA barriers per pivot; used for n > 16, where one warp's unrolled
// chains of shuffles (warp_spd_inverse) grow with 32-wide registers rows.  G
// and Gi shared, not aliased.  Returns 1 in every thread if a pivot was not
// positive.  flag: shared int.
template <typename T>
__device__ __noinline__ int cta_spd_inverse(const T* G, int ldg, int n, T* Gi, int ldgi, int* flag, T* prow,
                                            T* pcol) {
  const int t = threadIdx.x, nn = n * n;
  for (int e = t; e < nn; e += NT) {
    const int i = e / n, j = e - i * n;
    Gi[i * ldgi + j] = G[i * ldg + j];
  }
  if (t == 0) flag[0] = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (t < n) {
      prow[t] = Gi[k * ldgi + t];
      pcol[t] = Gi[t * ldgi + k];
    }
    __syncthreads();
    T p = prow[k];
    if (!(p > T(0))) {
      if (t == 0) flag[0] = 1;
      p = T(1);
    }
    const T ip = T(1) / p;
    for (int e = t; e < nn; e += NT) {
      const int i = e / n, j = e - i * n;
      T v;
      if (i == k) v = j == k ? ip : prow[j] * ip;
      else if (j == k) v = -pcol[i] * ip;
      else v = fma(-(pcol[i] * ip), prow[j], Gi[i * ldgi + j]);
      Gi[i * ldgi + j] = v;
    }
    __syncthreads();
  }
  const int f = flag[0];
  __syncthreads();
  return f;
}

template <typename T, int CAP>
__device__ __noinline__ int warp_spd_inverse(const T* G, int ldg, int n, T* Gi, int ldgi, int* flag) {
  return warp_spd_inverse_as<T, T, CAP>(G, ldg, n, Gi, ldgi, flag);
}

// Issue (without waiting) the cp.async copy of an m-row block whose rows are
// `rowb` bytes (a multiple of 16) from global (row pitch gpitch bytes) to
// shared (row pitch spitch bytes); all addresses 16-byte aligned.
__device__ inline void cta_stage_rows(void* dst, int spitch, const void* src, int gpitch, int m, int rowb) {
  const int c16 = rowb >> 4, tot = m * c16;
  for (int e = threadIdx.x; e < tot; e += NT) {
    const int r = e / c16, cc = e - r * c16;
    cp_async16((char*)dst + (size_t)r * spitch + 16 * cc, (const char*)src + (size_t)r * gpitch + 16 * cc);
  }
}

// Y = X (copy an m x n block), optional transpose (Y = X^T, Y is n x m).
template <typename T>
__device__ void cta_copy(int m, int n, const T* X, int ldxs, bool trans, T* Y, int ldy) {
  // eight independent loads per thread before their stores
  const int total = m * n;
  for (int base = threadIdx.x; base < total; base += 8 * NT) {
    T v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = base + u * NT;
      if (e < total) {
        const int i = trans ? e % m : e / n, j = trans ? e / m : e % n;
        v[u] = X[(size_t)i * ldxs + j];
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = base + u * NT;
      if (e < total) {
        const int i = trans ? e % m : e / n, j = trans ? e / m : e % n;
        if (!trans) Y[(size_t)i * ldy + j] = v[u];
        else Y[(size_t)j * ldy + i] = v[u];
      }
    }
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
// pivot = true: partial pivoting over the not-yet-used rows (largest |value|
// up to a relative 2^-16 in FP32, 2^-13 in FP64, ties to the lower row; the
// pivot row is recorded instead of swapped and the result gathered through the
// permutation at the end); failure if a pivot is not above tiny_pivot.  pivot = false: pivots on the diagonal, failure if one
// is not positive (the test that the matrix is symmetric positive definite).
// Returns 0 on success, 1 on failure.  S is overwritten.
//
// One elimination step with pivot (p, k) replaces column k by e_p and then
// left-multiplies by L = I + g e_p^T, g = -(c - e_p) / c_p, c = column k.
// The steps are blocked by INV_PANEL columns:
//   * warp 0 runs the steps of a panel on the panel's columns only, held in
//     registers (lane l owns rows l, l+32, l+64); after the panel, column k_j
//     holds L_b ... L_1 e_{p_j};
//   * every other column x then needs x <- L_b ... L_1 x.  Since e_{p_j} is
//     untouched by the steps before j, L_b ... L_1 x = x + sum_j (PC_j -
//     e_{p_j}) x_{p_j} with PC_j the final panel column j, i.e.
//     x_i <- [i not a pivot row of the panel] x_i + sum_j PC[i][j] x_{p_j},
//     a rank-b update done by the whole CTA from a copy of the pivot rows.
// scratch: shared, >= INV_SCRATCH elements; perm: shared int[2*TILE];
// flag: shared int (flag[0] = failure).
constexpr int INV_PANEL = 16;
constexpr int INV_SCRATCH = INV_PANEL * TILE + INV_PANEL;

__device__ inline unsigned abs_hi32(float v) { return __float_as_uint(fabsf(v)); }
__device__ inline unsigned abs_hi32(double v) { return (unsigned)((unsigned long long)__double_as_longlong(fabs(v)) >> 32); }

// Rank-b update of the columns outside panel [k0, k0 + bw) (see cta_inverse),
// with an R x R register tile per thread of the 16 x 16 grid.
template <typename T, int R>
__device__ __forceinline__ void inv_trailing(T* S, int lds, int n, int k0, int bw, int pn, const int* panel_of,
                                             const T* XP) {
  const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
  T acc[R][R];
#pragma unroll
  for (int a = 0; a < R; ++a) {
    const int i = ty + 16 * a;
    const bool keep = i < n && panel_of[i] != pn;
#pragma unroll
    for (int b = 0; b < R; ++b) {
      const int col = tx + 16 * b;
      acc[a][b] = (keep && col < n) ? S[i * lds + col] : T(0);
    }
  }
  for (int j = 0; j < bw; ++j) {
    T xr[R], pc[R];
#pragma unroll
    for (int b = 0; b < R; ++b) {
      const int col = tx + 16 * b;
      xr[b] = col < n ? XP[j * TILE + col] : T(0);
    }
#pragma unroll
    for (int a = 0; a < R; ++a) {
      const int i = ty + 16 * a;
      pc[a] = i < n ? S[i * lds + k0 + j] : T(0);
    }
#pragma unroll
    for (int a = 0; a < R; ++a)
#pragma unroll
      for (int b = 0; b < R; ++b) acc[a][b] = fma(pc[a], xr[b], acc[a][b]);
  }
#pragma unroll
  for (int a = 0; a < R; ++a) {
    const int i = ty + 16 * a;
#pragma unroll
    for (int b = 0; b < R; ++b) {
      const int col = tx + 16 * b;
      if (i < n && col < n && (col < k0 || col >= k0 + bw)) S[i * lds + col] = acc[a][b];
    }
  }
}

// Gauss-Jordan steps of one panel [k0, k0 + bw) by warp 0 (see cta_inverse):
// lane l holds rows l + 32 q, q < QR (QR = 2 covers n <= 64, 3 covers 96).
template <typename T, int QR>
__device__ __forceinline__ void inv_panel(T* S, int lds, int n, int k0, int bw, int pn, bool pivot, unsigned& used,
                                          int& bad, int* perm, int* panel_of, T* rowbuf) {
  const int lane = threadIdx.x & 31;
  // Panel columns in registers, rotated so that the current step's
  // column is always slot 0: after a step every slot moves down by one
  // and the finished column goes to the last slot.  The step is then
  // the same code for every j (a rolled loop: the panel code stays small
  // enough for the instruction cache).  After bw steps slot m holds panel
  // column (m + bw) mod INV_PANEL.
  T pv[QR][INV_PANEL];
#pragma unroll
  for (int q = 0; q < QR; ++q) {
    const int i = lane + 32 * q;
#pragma unroll
    for (int l = 0; l < INV_PANEL; ++l) pv[q][l] = (i < n && l < bw) ? S[i * lds + k0 + l] : T(0);
  }
#pragma unroll 1
  for (int j = 0; j < bw; ++j) {
    const int k = k0 + j;
    int p = k;
    if (pivot) {
      // argmax |column| over unused rows in one warp max: the key is the
      // top 32 bits of |value| (non-negative floats order like unsigned
      // integers) with the low 7 bits replaced by 127 - row, so the
      // winner is a largest |value| up to a relative 2^-16 (FP32) or
      // 2^-13 (FP64) -- as good a partial pivot -- ties to the lower row
      unsigned key = 0u;
#pragma unroll
      for (int q = 0; q < QR; ++q) {
        const int i = lane + 32 * q;
        if (i < n && !((used >> q) & 1u)) {
          const unsigned kq = (abs_hi32(pv[q][0]) & ~127u) | (unsigned)(127 - i);
          key = kq > key ? kq : key;
        }
      }
      const unsigned kmax = __reduce_max_sync(0xffffffffu, key);
      p = 127 - (int)(kmax & 127u);
      p = (p >= 0 && p < n) ? p : n - 1;   // always in range: an unused row exists while k < n
    }
    const int pl = p & 31, pq = p >> 5;
    // pivot row of the panel, broadcast through shared memory by its owner
    using V16 = typename Vec16<T>::type;
    constexpr int VW = Vec16<T>::W;
    if (lane == pl) {
#pragma unroll
      for (int l0 = 0; l0 < INV_PANEL; l0 += VW) {
        V16 v;
        T* vp = reinterpret_cast<T*>(&v);
#pragma unroll
        for (int e = 0; e < VW; ++e)
        {
          T sel = pv[0][l0 + e];
#pragma unroll
          for (int q = 1; q < QR; ++q) sel = pq == q ? pv[q][l0 + e] : sel;   // constant indices only
          vp[e] = sel;
        }
        reinterpret_cast<V16*>(rowbuf)[l0 / VW] = v;
      }
    }
    __syncwarp();
    T rowp[INV_PANEL];
#pragma unroll
    for (int l0 = 0; l0 < INV_PANEL; l0 += VW) {
      const V16 v = reinterpret_cast<const V16*>(rowbuf)[l0 / VW];
      const T* vp = reinterpret_cast<const T*>(&v);
#pragma unroll
      for (int e = 0; e < VW; ++e) rowp[l0 + e] = vp[e];
    }
    __syncwarp();
    T piv = rowp[0];
    const bool badk = pivot ? !(fabs(piv) > tiny_pivot<T>()) : !(piv > T(0));
    if (badk) {
      bad = 1;
      piv = T(1);
    }
    const T ip = T(1) / piv;
#pragma unroll
    for (int q = 0; q < QR; ++q) {
      const bool isp = (lane + 32 * q) == p;
      const T g = -(pv[q][0] - (isp ? T(1) : T(0))) * ip;
      // slots 1.. get the step's update and move down; slot 0 (this
      // step's column, replaced by e_p + g) goes to the last slot
#pragma unroll
      for (int l = 1; l < INV_PANEL; ++l) pv[q][l - 1] = fma(g, rowp[l], pv[q][l]);
      pv[q][INV_PANEL - 1] = (isp ? T(1) : T(0)) + g;
    }
    if (lane == pl) used |= 1u << pq;
    if (lane == 0) {
      perm[k] = p;
      panel_of[p] = pn;
    }
  }
  // undo the rotation: slot m holds panel column (m + bw) mod INV_PANEL
#pragma unroll
  for (int q = 0; q < QR; ++q) {
    const int i = lane + 32 * q;
#pragma unroll
    for (int m = 0; m < INV_PANEL; ++m) {
      const int l = (m + bw) & (INV_PANEL - 1);
      if (i < n && l < bw) S[i * lds + k0 + l] = pv[q][m];
    }
  }
}

template <typename T>
__device__ __noinline__ int cta_inverse(T* S, int lds, int n, bool pivot, T* Wout, int ldw, T* scratch, int* perm,
                                        int* flag) {
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  int* panel_of = perm + TILE;   // panel index in which row i became a pivot row (-1: not yet)
  T* XP = scratch;               // pivot rows of the current panel, [INV_PANEL][TILE]
  T* rowbuf = scratch + INV_PANEL * TILE;   // warp 0: pivot row of the panel, [INV_PANEL]
  for (int i = t; i < n; i += NT) panel_of[i] = -1;
  if (t == 0) flag[0] = 0;
  __syncthreads();
  unsigned used = 0;             // warp 0: bit q = row lane + 32 q is a pivot row
  int bad = 0;
  const int npan = (n + INV_PANEL - 1) / INV_PANEL;
  for (int pn = 0; pn < npan; ++pn) {
    const int k0 = pn * INV_PANEL;
    const int bw = min(INV_PANEL, n - k0);
    if (w == 0) {
      if (n <= 64) inv_panel<T, 2>(S, lds, n, k0, bw, pn, pivot, used, bad, perm, panel_of, rowbuf);
      else inv_panel<T, 3>(S, lds, n, k0, bw, pn, pivot, used, bad, perm, panel_of, rowbuf);
    }
    __syncthreads();
    // pivot rows of this panel, before the rank-b update
    for (int e = t; e < bw * n; e += NT) {
      const int j = e / n, col = e - j * n;
      XP[j * TILE + col] = S[perm[k0 + j] * lds + col];
    }
    __syncthreads();
    // x_i <- [i not a pivot row of this panel] x_i + sum_j PC[i][j] XP[j] for
    // every column outside the panel: 16 x 16 thread grid, rows ty + 16 a and
    // columns tx + 16 b (4 x 4 per thread when n <= 64, else 5 x 5).  No
    // other thread reads what a thread writes: it owns its (row, column)
    // elements, and the panel columns it reads are not written in this phase.
    if (n <= 64) inv_trailing<T, 4>(S, lds, n, k0, bw, pn, panel_of, XP);
    else inv_trailing<T, 5>(S, lds, n, k0, bw, pn, panel_of, XP);
    __syncthreads();
  }
  if (t == 0 && bad) flag[0] = 1;
  // gather: W[a][b] = M[perm[a]][iperm[b]] (iperm[perm[c]] = c)
  int* iperm = perm + TILE;
  for (int q = t; q < n; q += NT) iperm[perm[q]] = q;
  __syncthreads();
  for (int e = t; e < n * n; e += NT) {
    const int a = e / n, b = e - a * n;
    Wout[a * ldw + b] = S[perm[a] * lds + iperm[b]];
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

// Inverse of an SPD n x n matrix (n <= CAP <= 32) to FP64 accuracy by
// mixed-precision iterative refinement: the FP32 Gauss-Jordan inverse X0 of
// warp_spd_inverse_as, the residual E = I - G X0 in FP64 arithmetic, then one
// Newton-Schulz step X1 = X0 + X0 E.  Since I - G X1 = E^2, X1 has relative
// error at most ||E||^2 (infinity norm); the step is taken when ||E|| <= 1e-4,
// so X1 is FP64-accurate to well below the output's rounding.  X0 E is a
// small correction, so its product runs in FP32; the sum X0 + X0 E is
// rounded once.  A failed FP32 pivot, or ||E|| > 1e-4 (an ill-conditioned
// block), takes the FP64 Gauss-Jordan instead.  B300 issues FP64 at a small
// fraction of the FP32 rate: this keeps FP64 to the n^3 residual products,
// one element per thread, and out of the pivot chain with its divisions.
// G, Gi as for warp_spd_inverse_as; E: shared scratch of n rows x lde >= n
// elements aliasing neither.  Ends with a CTA barrier.
template <typename T, int CAP>
__device__ __noinline__ int spd_inverse_refined(const T* G, int ldg, int n, T* Gi, int ldgi, int* flag, T* E,
                                                int lde) {
  if (warp_spd_inverse_as<T, T, CAP>(G, ldg, n, Gi, ldgi, flag))
    return warp_spd_inverse_as<T, double, CAP>(G, ldg, n, Gi, ldgi, flag);
  const int t = threadIdx.x, nn = n * n;
  for (int e = t; e < nn; e += NT) {
    const int i = e / n, j = e - i * n;
    double s = i == j ? 1.0 : 0.0;
    for (int q = 0; q < n; ++q) s = fma(-(double)G[i * ldg + q], (double)Gi[q * ldgi + j], s);
    E[i * lde + j] = (T)s;
  }
  __syncthreads();
  if (t < 32) {
    T r = T(0);
    if (t < n)
      for (int j = 0; j < n; ++j) r += fabs(E[t * lde + j]);
    r = warp_max(r);
    if (t == 0) flag[0] = r <= T(1e-4) ? 0 : 1;
  }
  __syncthreads();
  const int fall = flag[0];
  __syncthreads();
  if (fall) return warp_spd_inverse_as<T, double, CAP>(G, ldg, n, Gi, ldgi, flag);
  constexpr int PER = (CAP * CAP + NT - 1) / NT;
  T xr[PER];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = t + p * NT;
    xr[p] = T(0);
    if (e < nn) {
      const int i = e / n, j = e - i * n;
      T s = T(0);
      for (int l = 0; l < n; ++l) s = fma(Gi[i * ldgi + l], E[l * lde + j], s);
      xr[p] = Gi[i * ldgi + j] + s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = t + p * NT;
    if (e < nn) {
      const int i = e / n, j = e - i * n;
      Gi[i * ldgi + j] = xr[p];
    }
  }
  __syncthreads();
  return 0;
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

// ---------------------------------------------------------------------------
// Bulk (TMA) copies global -> shared with mbarrier completion.
// ---------------------------------------------------------------------------
__device__ inline unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ inline void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) accesses.
__device__ inline void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// One thread: expect `bytes` on `bar` and start the bulk copy (16-byte aligned
// addresses, bytes a multiple of 16).
__device__ inline void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Wait for the phase with the given parity to complete; gives up after
// `limit` polls and returns false.
__device__ inline bool mbar_wait(unsigned long long* bar, unsigned parity, int limit) {
  const unsigned a = smem_addr(bar);
  for (int k = 0; k < limit; ++k) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// ---------------------------------------------------------------------------
// One-round split sweep: y = [A | B]^T x with A (rows x na, leading dim lda)
// at the start of a shared block and B (rows x nb, leading dim ldb) at element
// offset offB.  Outputs are grouped in 16-byte vectors (VW elements); the
// rows are split into G contiguous groups, every (vector, group) pair is one
// thread, and the G partial vectors are summed by the output's owner thread
// (t < na + nb) after one barrier.  The role of each thread is computed once
// (sweep_plan) and reused for every block of a stream.
// ---------------------------------------------------------------------------

constexpr int SWEEP_MAXG = 16;
// shared scratch of a sweep: NT vectors of 16 bytes
constexpr int SWEEP_SMEM_BYTES = NT * 16;

struct SweepPlan {
  int nr;        // rows of this thread's group (0: no partial role)
  int moff;      // element offset of its first (row, vector) in the block
  int ld;        // leading dimension of its matrix
  int r0;        // first row
  int slot;      // vector slot of its partial
  int G;         // row groups
  int red_off;   // element offset of its output in a partial row (red_off < 0: no output)
  int pstride;   // elements per partial row (nq * VW)
};

template <typename T>
__device__ inline SweepPlan sweep_plan(int rows, int na, int lda, int nb, int ldb, int offB) {
  constexpr int VW = Vec16<T>::W;
  const int t = threadIdx.x;
  const int nqa = (na + VW - 1) / VW, nqb = (nb + VW - 1) / VW, nq = nqa + nqb;
  SweepPlan p;
  int G = NT / nq;
  G = G < 1 ? 1 : (G > SWEEP_MAXG ? SWEEP_MAXG : G);
  const int Rg = (rows + G - 1) / G;
  const int q = t % nq, g = t / nq;
  p.G = G;
  p.pstride = nq * VW;
  p.slot = g * nq + q;
  p.nr = 0;
  p.moff = 0;
  p.ld = lda;
  p.r0 = 0;
  if (g < G) {
    const bool isa = q < nqa;
    const int r0 = min(rows, g * Rg);
    p.r0 = r0;
    p.nr = min(rows, r0 + Rg) - r0;
    p.ld = isa ? lda : ldb;
    p.moff = (isa ? 0 : offB) + r0 * p.ld + (isa ? q : q - nqa) * VW;
  }
  p.red_off = t < na ? t : (t < na + nb ? nqa * VW + (t - na) : -1);
  return p;
}

template <typename T>
__device__ inline void vload16(const T* p, T* v);
template <> __device__ inline void vload16<float>(const float* p, float* v) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
template <> __device__ inline void vload16<double>(const double* p, double* v) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  v[0] = a.x; v[1] = a.y;
}

// Batched plan: nmat matrices of rows x ncols (leading dim ld, element stride
// `stride` between matrices) times the same x; output o = mat * ncols + col.
// Needs nmat * ceil(ncols / VW) <= NT and nmat * ncols <= NT.
template <typename T>
__device__ inline SweepPlan sweep_plan_batched(int rows, int ncols, int ld, int nmat, int stride) {
  constexpr int VW = Vec16<T>::W;
  const int t = threadIdx.x;
  const int nqc = (ncols + VW - 1) / VW, nq = nmat * nqc;
  SweepPlan p;
  int G = NT / nq;
  G = G < 1 ? 1 : (G > SWEEP_MAXG ? SWEEP_MAXG : G);
  const int Rg = (rows + G - 1) / G;
  const int q = t % nq, g = t / nq;
  p.G = G;
  p.pstride = nq * VW;
  p.slot = g * nq + q;
  p.nr = 0;
  p.moff = 0;
  p.ld = ld;
  p.r0 = 0;
  if (g < G) {
    const int mat = q / nqc, vq = q - mat * nqc;
    const int r0 = min(rows, g * Rg);
    p.r0 = r0;
    p.nr = min(rows, r0 + Rg) - r0;
    p.moff = mat * stride + r0 * ld + vq * VW;
  }
  if (t < nmat * ncols) {
    const int mat = t / ncols, col = t - mat * ncols;
    p.red_off = mat * nqc * VW + col;
  } else {
    p.red_off = -1;
  }
  return p;
}

// Partial sums of this thread's (vector, row group) on block `blk` with
// vector x (both shared), added into acc[VW].  No barrier.
template <typename T>
__device__ inline void sweep_partial(const SweepPlan& p, const T* blk, const T* x, T* acc) {
  constexpr int VW = Vec16<T>::W;
  if (p.nr <= 0) return;
  T b[VW], m0[VW], m1[VW];
#pragma unroll
  for (int e = 0; e < VW; ++e) b[e] = T(0);
  const T* mp = blk + p.moff;
  const T* xp = x + p.r0;
  const int ld2 = 2 * p.ld;
  int k = 0;
  for (; k + 1 < p.nr; k += 2) {
    vload16<T>(mp, m0);
    vload16<T>(mp + p.ld, m1);
    const T x0 = xp[k], x1 = xp[k + 1];
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      acc[e] = fma(m0[e], x0, acc[e]);
      b[e] = fma(m1[e], x1, b[e]);
    }
    mp += ld2;
  }
  if (k < p.nr) {
    vload16<T>(mp, m0);
    const T x0 = xp[k];
#pragma unroll
    for (int e = 0; e < VW; ++e) acc[e] = fma(m0[e], x0, acc[e]);
  }
#pragma unroll
  for (int e = 0; e < VW; ++e) acc[e] += b[e];
}

// Publishes the partial vectors (zero for threads of a row group without
// rows), one barrier, and returns the total for the owner of an output
// (red_off >= 0), else 0.  The caller must barrier before `swp` is reused.
template <typename T>
__device__ inline T sweep_reduce(const SweepPlan& p, const T* acc, T* swp) {
  constexpr int VW = Vec16<T>::W;
  using V = typename Vec16<T>::type;
  if (p.slot < p.G * (p.pstride / VW)) {
    V o;
    T* op = reinterpret_cast<T*>(&o);
#pragma unroll
    for (int e = 0; e < VW; ++e) op[e] = acc[e];
    reinterpret_cast<V*>(swp)[p.slot] = o;
  }
  __syncthreads();
  T sum = T(0);
  if (p.red_off >= 0) {
    const T* ps = swp + p.red_off;
#pragma unroll 4
    for (int g = 0; g < p.G; ++g) sum += ps[g * p.pstride];
  }
  return sum;
}

// One block: partial sums, one barrier, reduction.
template <typename T>
__device__ inline T sweep_run(const SweepPlan& p, const T* blk, const T* x, T* swp) {
  constexpr int VW = Vec16<T>::W;
  T acc[VW];
#pragma unroll
  for (int e = 0; e < VW; ++e) acc[e] = T(0);
  sweep_partial<T>(p, blk, x, acc);
  return sweep_reduce<T>(p, acc, swp);
}

}  // namespace gsls
