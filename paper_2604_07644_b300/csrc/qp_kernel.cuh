// Persistent ADMM solve kernel for the LTV-QP (Sec. IV-A), one thread-block
// cluster per QP.
//
// Layout of the work inside a cluster of `cs` CTAs:
//   * the stages 0..N-1 are split into nch <= cs contiguous chunks; CTA r owns
//     chunk [s_r, e_r) (and the terminal time point N if it owns the last chunk);
//   * the rho-dependent factorization (eq. augmented_matrices, eq. assoc_init,
//     the reverse scan of eq. combination_rules, eq. controller_cache) runs as
//     the paper's tree: an up-sweep of full combines and a down-sweep of
//     combines whose right operand is a complete suffix, level by level, with
//     the combines of a level spread over the cluster's CTAs;
//   * once the Riccati terms P_i are cached, one ADMM iteration is two affine
//     recursions with fixed matrices (backward p_i = Abar_i^T p_{i+1} + c_i,
//     forward x_{i+1} = Abar_i x_i + d_i).  Each is scanned in three phases:
//     a chunk-local chain with zero boundary, a chunk-boundary correction with
//     cached products of the chunk transfer matrices read through distributed
//     shared memory, and a fix-up folded into cached per-stage products.
#pragma once
#include <cooperative_groups.h>
#include <math.h>
#include "dense.cuh"

namespace cg = cooperative_groups;

namespace gsls {

// CTAs per QP: up to 8 is the portable cluster size; 9..16 are non-portable
// cluster sizes (long horizons: shorter chunk chains), launched only where
// the device schedules them.
constexpr int MAXCS = 16;
constexpr int MAXCS_PORTABLE = 8;

// Per-QP descriptor: dimensions and device pointers into the handle's pools.
// Pointers typed void* are in the solve precision T (padded layouts, leading
// dims ldx / ldu / ldc); double* pointers are FP64 copies of the caller's
// dense arrays (for the KKT check) or FP64 outputs.
struct QPDesc {
  int nx, nu, N, nc, nf, m;
  int ldx, ldu, ldc;
  int nch, Lc;      // number of non-empty chunks, chunk length
  int nlev;         // tree levels above the leaves
  int ldv, ldf;     // row strides of the stacked vectors [l; omega] and [x; k]
  int depth, slot;  // cp.async ring depth and slot size (elements)
  int fact;         // factorization schedule: 0 blocked (leaf-structured combines), 1 tree
  int vg;           // 1: per-chunk vectors in the global region vec (long horizons), 0: shared memory
  int vstride;      // bytes of one CTA's part of vec
  // problem (T)
  void *A, *B, *b, *Q, *R, *S, *q, *r, *C, *D, *CN, *lo, *hi, *x0;
  // factorization workspace (T)
  void *Rhi, *Sh, *VP, *VA, *VC, *IP, *scr;
  void *Rh, *S0;    // R^_i and R^_i^-1 S^_i per stage (blocked schedule)
  // cached iteration operators (T)
  void *Abar, *CK, *F, *FPi, *J, *K, *KSig, *CKSig, *Sig, *c0, *k0, *CNSig, *SigN, *Tch, *Uch,
      *Theta, *Xi, *Gam;
  // per-stage bundles streamed by the iteration (see bundle_sizes)
  void *BW, *FW, *CD;
  // ADMM state (T)
  void *z, *y;
  void* vec;        // vg: per-CTA vector regions [cluster][vstride bytes]
  // FP64 copies (dense, caller layout) and scratch
  double *A64, *B64, *b64, *Q64, *R64, *S64, *q64, *r64, *C64, *D64, *CN64, *lo64, *hi64, *x064;
  double *kg, *kh;
  double* rho;      // [1]
  int* flags;       // [0]: factorization valid for *rho; [1]: state set by a warm start
  const double* rho0;   // [1] setup penalty (cold restart)
  // outputs (set per call)
  double *ox, *ou, *olam;
  int* info_i;      // [4]: status, iters, refactors, -
  double* info_d;   // [4]: rho, r_prim, r_dual, kkt
};

// MODE_GAINS: the factorization for its gains alone (K_i, Abar_i, P_i,
// Gamma_i), without the iteration operators (bundles, chunk products,
// chunk-boundary operators): the SLS controller solves need no more, and
// the handle's factorization is left marked invalid for iterations.
enum Mode { MODE_SOLVE = 0, MODE_RICCATI = 1, MODE_KKT = 2, MODE_GAINS = 3 };

struct SolveArgs {
  unsigned long long* prof;   // optional per-phase cycle counters [cs][phases] of QP 0, else null
  int mode;
  int max_iter;
  int fixed_iters;
  int sigma;
  int check_every;
  int cs;
  double eps, eps_kkt, rho_min, rho_max, eps_floor;
  int max_refine;
  int fallback_iters;   // > 0: a warm-started QP not converged after this many iterations restarts cold
  const int* order;     // launch order: cluster b solves QP order[b] (null: QP b)
  int tc;               // 1: factorization block products on the tensor cores in TF32 (GPUSLS_TF32);
                        // 2: GPUSLS_MIXED (three TF32 passes, FP64 per-stage solves)
  int test_wait;        // test hook: one bounded wait on a copy barrier that nothing completes
};

// Per-stage operator bundles of the cached iteration (elements).  Every
// product of the iteration is a column sweep y[j] = sum_r M[r][j] x[r] over a
// row-major block, so blocks used as y = M x are stored transposed.
//   BW_i = [Abar_i ; CK_i] ((nx+nc) x ldx), [F_i | J_i]^T ((nx+nc) x ldu),
//          c0_i (ldx), k0_i (ldu)                    -- backward chain
//   FW_i = [Abar_i | B_i ; CK_i | D_i]^T ((nx+nu) x ldv), b_i (ldx) -- forward chain
//   CD_i = [C_i | D_i] (nc x ldf)                    -- dual residual
// with ldv = rup4(nx + nc), ldf = rup4(nx + nu).
__host__ __device__ inline void bundle_sizes(int nx, int nu, int nc, int ldx, int ldu, int ldv, int ldf, int* bw,
                                             int* fw, int* cd) {
  *bw = (nx + nc) * ldx + (nx + nc) * ldu + ldx + ldu;
  *fw = (nx + nu) * ldv + ldx;
  *cd = nc * ldf;
}

// Shared-memory carve-up (byte offsets, 16-byte aligned).
struct SmemLayout {
  int ring, gemm, gj, gjbuf;                 // union region
  int z, y, w, l, x, kt, v, d, u, pe, xs, slotL, slotX, tmp1, tmp2, tmp3, red;
  int part, perm, flag, bar, swp, gath;
  int uni;     // bytes of the union region (ring / dense scratch / factorization buffers)
  int total;
  int vbytes;  // vg: bytes of the per-CTA global region holding z, y, w, l, x, kt, v, d, u
};

constexpr int MAX_RING = 8;   // ring slots (mbarriers) at most
constexpr int BULK_BAR = MAX_RING - 1;   // mbarrier of the whole-region copies (ring depth < BULK_BAR)
constexpr int RING_FLAG = 8;  // index in the shared flag[] array: a ring wait gave up
constexpr int RING_WAIT_LIMIT = 1 << 22;   // polls of one bulk-copy completion before giving up

__host__ __device__ inline int al16(int x) { return (x + 15) & ~15; }

// Shared-memory buffers of the blocked factorization, element offsets into
// the union region (which the iteration's ring and the tree's GEMM staging
// use at other times).  Every buffer starts on a multiple of 4 elements
// (16 bytes in FP32, 32 in FP64).
struct FactLayout {
  int lds;   // row pitch of the nx-column buffers (ldx, or ldx + 4 when ldx is a multiple of 32: no bank conflicts
             // between the two rows a warp reads)
  int P, Aa, Xb, Bb[2], Rb[2], Db[2], S1, S2, S3, Gm, Gi, BG, CKb[2], JT, vec;
  int vlen;  // length of each of the 8 vectors at vec
  int total;
};

__host__ __device__ inline FactLayout fact_layout(int nx, int nu, int nc, int nf, int ldx, int ldu) {
  FactLayout f;
  f.lds = (ldx % 32 == 0) ? ldx + 4 : ldx;
  f.vlen = rup4(nx > nu ? nx : nu);
  int off = 0;
  const int big = rup4(nx * f.lds), bsz = rup4(nx * ldu), rsz = rup4(nu * ldu), dsz = rup4(nc * ldu),
            ssz = rup4(nu * f.lds), csz = rup4((nc > nf ? nc : nf) * f.lds);
  f.P = off; off += big;
  f.Aa = off; off += big;
  f.Xb = off; off += big;
  for (int k = 0; k < 2; ++k) { f.Bb[k] = off; off += bsz; }
  for (int k = 0; k < 2; ++k) { f.Rb[k] = off; off += rsz; }
  for (int k = 0; k < 2; ++k) { f.Db[k] = off; off += dsz; }
  f.S1 = off; off += ssz;
  f.S2 = off; off += ssz;
  f.S3 = off; off += ssz;
  f.Gm = off; off += rsz;
  f.Gi = off; off += rsz;
  f.BG = off; off += bsz;
  for (int k = 0; k < 2; ++k) { f.CKb[k] = off; off += csz; }
  f.JT = off; off += dsz;
  f.vec = off; off += 8 * f.vlen;
  f.total = off;
  return f;
}

// The blocked schedule runs when its buffers fit and nu is small enough for
// the one-warp inverse of the nu x nu blocks.
constexpr int FACT_MAX_NU = 32;

// vg = 1 (long horizons): the per-chunk vectors z, y, w, l, x, kt, v, d, u,
// whose size grows with the chunk length, live in a per-CTA region of global
// memory (offsets relative to its base, vbytes long) instead of shared
// memory; the kernel reaches them through the same generic pointers.
__host__ __device__ inline SmemLayout smem_layout(int nx, int nu, int nc, int nf, int Lc, int nch, int cs, int ldx,
                                                  int ldu, int ldv, int ldf, int depth, int slot, int esz, int fact,
                                                  int vg = 0) {
  SmemLayout s;
  int off = 0;
  const int ring_b = depth * slot * esz;
  const int dense_b = (2 * KT * TILE + TILE * GJ_LD + 3 * TILE) * esz;
  const int fact_b = fact == 0 ? fact_layout(nx, nu, nc, nf, ldx, ldu).total * esz : 0;
  int uni = ring_b > dense_b ? ring_b : dense_b;
  uni = uni > fact_b ? uni : fact_b;
  s.ring = 0;
  s.gemm = 0;
  s.gj = 2 * KT * TILE * esz;
  s.gjbuf = s.gj + TILE * GJ_LD * esz;
  off = al16(uni);
  const int rows = Lc * nc + nf;
  int voff = 0;
  int& vo = vg ? voff : off;
  s.z = vo; vo = al16(vo + rows * esz);
  s.y = vo; vo = al16(vo + rows * esz);
  s.w = vo; vo = al16(vo + rows * esz);
  s.l = vo; vo = al16(vo + (Lc + 1) * ldv * esz);
  s.x = vo; vo = al16(vo + (Lc + 1) * ldf * esz);
  s.kt = vo; vo = al16(vo + Lc * ldu * esz);
  s.v = vo; vo = al16(vo + rows * esz);
  s.d = vo; vo = al16(vo + (Lc + 1) * ldx * esz);
  s.u = vo; vo = al16(vo + Lc * ldu * esz);
  s.vbytes = vg ? (voff + 255) & ~255 : 0;
  s.pe = off; off = al16(off + TILE * esz);
  s.xs = off; off = al16(off + TILE * esz);
  s.slotL = off; off = al16(off + TILE * esz);
  s.slotX = off; off = al16(off + TILE * esz);
  s.tmp1 = off; off = al16(off + TILE * esz);
  s.tmp2 = off; off = al16(off + TILE * esz);
  s.tmp3 = off; off = al16(off + TILE * esz);
  s.red = off; off = al16(off + NT * esz);
  s.part = off; off = al16(off + (16 + cs * 8) * 8);   // cluster_max slots and its [cs][8] gather
  s.perm = off; off = al16(off + 2 * TILE * 4);
  s.flag = off; off = al16(off + 16 * 4);
  s.bar = off; off = al16(off + MAX_RING * 8);
  // sweep partials and the gathered chunk-boundary vectors go in the union
  // region's slack after the ring when the dense scratch is the larger part
  // of it, else in regions of their own
  int slack = al16(ring_b);
  const int uend = al16(uni);
  const int gath_b = (nch > 1 ? nch - 1 : 1) * ldx * esz;
  if (slack + SWEEP_SMEM_BYTES <= uend) {
    s.swp = slack; slack = al16(slack + SWEEP_SMEM_BYTES);
  } else {
    s.swp = off; off = al16(off + SWEEP_SMEM_BYTES);
  }
  if (slack + gath_b <= uend) {
    s.gath = slack; slack = al16(slack + gath_b);
  } else {
    s.gath = off; off = al16(off + gath_b);
  }
  s.uni = uend;
  s.total = off;
  return s;
}

template <typename T>
struct Ctx {
  QPDesc* d;
  int rank, cs;
  int s, e, L;
  bool active, first, last;
  T *gemm, *gj, *gjbuf, *ring;
  T *zS, *yS, *wS, *lS, *xS, *ktS, *vS, *dS, *uS, *pe, *xs, *slotL, *slotX, *tmp1, *tmp2, *tmp3, *red;
  double* part;
  int *perm, *flag;
  unsigned long long* bar;   // ring mbarriers, one per slot
  T* swp;                    // sweep partials
  T* gath;                   // chunk-boundary vectors gathered from the other CTAs
  unsigned ws, wp;           // ring: next slot to consume and its phase parity
  unsigned inflight, ipar;   // issuing thread: slots with a copy not yet seen complete, their parities
  unsigned bpar;             // whole-region copies: parity of the next completion of bar[BULK_BAR]
  int bulk_inflight;         // a whole-region copy was issued and not yet seen complete
  int cm_par;                // cluster_max: slot of part[] of the next call
  // per-launch iteration plan (iter_plan): bundle sizes, and the whole-region
  // rounds of the chunk-boundary corrections (P3: Theta blocks, then FPi
  // stages; P5: Xi blocks, then CKSig stages)
  int bws, fws, cds;
  int cap_bk, nb_th, nr_th, gs_fp, nr_fp, nb_xi, nr_xi, gs_ck, nr_ck;
  T* scr;   // per-CTA global scratch: 6 matrices nx x ldx
  int msz;  // nx * ldx
  int uni;  // bytes of the union region at ring
  unsigned long long* prof;  // non-null in each CTA of QP 0 when profiling (thread 0 records)
  bool tc;                   // factorization products in TF32 on the tensor cores (tree schedule)
  bool gains;                // MODE_GAINS: skip the iteration operators in the factorization
  bool mix;                  // GPUSLS_MIXED: blocked-schedule products in three TF32 passes on the
                             // tensor cores, per-stage nu x nu solves in FP64
  long long t_last;
};

// Phase timers (debug aid; compiled in, inactive unless SolveArgs.prof is set).
enum Phase { PH_P1 = 0, PH_BWD, PH_SYNC1, PH_P3, PH_FWD, PH_SYNC2, PH_P5, PH_CHECK, PH_RHO, PH_R1, PH_R2, PH_R3,
             PH_R4, PH_R5, PH_R6, PH_KKT, PH_RINGWAIT, PH_KKT_STAGES, PH_KKT_SYNC, PH_KKT_COSTATE,
             PH_FA1, PH_FA2, PH_FA3, PH_FC1, PH_FC2, PH_FC3, PH_FC4, PH_FC5, PH_COUNT };
template <typename T>
__device__ inline void prof_mark(Ctx<T>& c, int ph) {
  if (threadIdx.x == 0 && c.prof) {
    const long long now = clock64();
    c.prof[ph] += (unsigned long long)(now - c.t_last);
    c.t_last = now;
  }
}

template <typename T> __device__ inline T* TP(void* p) { return reinterpret_cast<T*>(p); }

__device__ inline int level_count(int n, int d) {  // n_d = ceil(n / 2^d)
  return (n + (1 << d) - 1) >> d;
}
__device__ inline int node_index(int n, int d, int m) {
  int off = 0;
  for (int i = 0; i < d; ++i) off += level_count(n, i);
  return off + m;
}

// ---------------------------------------------------------------------------
// global-memory CTA matvecs (operators streamed from L2 / HBM)
// ---------------------------------------------------------------------------
// y[i] (+)= alpha * sum_j M[i][j] x[j], i < rows (warp per row).  x, y shared.
template <typename T>
__device__ void g_mv(const T* M, int ld, int rows, int cols, const T* x, T alpha, bool acc, T* y) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int i = w; i < rows; i += NT / 32) {
    T s = T(0);
    for (int j = l; j < cols; j += 32) s += M[(size_t)i * ld + j] * x[j];
    s = warp_sum(s);
    if (l == 0) y[i] = (acc ? y[i] : T(0)) + alpha * s;
  }
  __syncthreads();
}
// y[j] (+)= alpha * sum_i M[i][j] x[i], j < cols (thread per column).
template <typename T>
__device__ void g_mvT(const T* M, int ld, int rows, int cols, const T* x, T alpha, bool acc, T* y) {
  for (int j = threadIdx.x; j < cols; j += NT) {
    T s = T(0);
    for (int i = 0; i < rows; ++i) s += M[(size_t)i * ld + j] * x[i];
    y[j] = (acc ? y[j] : T(0)) + alpha * s;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Combines of the reverse scan (eq. combination_rules).  Operands are tree
// nodes (P~, A~, C~) in global memory.  With W = (I + C~_ik P~_kj)^{-1}:
//   Ups P~_kj A~_ik = (P~_kj A~_ik)^T (W A~_ik)     (push-through identity)
//   Psi = A~_kj W,  A~_ij = Psi A~_ik,  C~_ij = Psi C~_ik A~_kj^T + C~_kj.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ int combine_full(Ctx<T>& c, const T* lP, const T* lA, const T* lC, const T* rP, const T* rA,
                                         const T* rC, T* oP, T* oA, T* oC) {
  const int n = c.d->nx, ld = c.d->ldx;
  T* X = c.scr;
  T* Psi = c.scr + c.msz;
  T* V = c.scr + 2 * c.msz;
  T* U = c.scr + 3 * c.msz;
  T* Wm = c.scr + 4 * c.msz;
  cta_gemm<T>(n, n, n, T(1), lC, ld, false, rP, ld, false, T(0), nullptr, 0, true, c.gj, GJ_LD, c.gemm, c.tc);
  const int bad = cta_inverse<T>(c.gj, GJ_LD, n, true, Wm, ld, c.gemm, c.perm, c.flag);
  cta_gemm<T>(n, n, n, T(1), Wm, ld, false, lA, ld, false, T(0), nullptr, 0, false, X, ld, c.gemm, c.tc);
  cta_gemm<T>(n, n, n, T(1), rA, ld, false, Wm, ld, false, T(0), nullptr, 0, false, Psi, ld, c.gemm, c.tc);
  cta_gemm<T>(n, n, n, T(1), rP, ld, false, lA, ld, false, T(0), nullptr, 0, false, V, ld, c.gemm, c.tc);
  cta_gemm<T>(n, n, n, T(1), V, ld, true, X, ld, false, T(1), lP, ld, false, oP, ld, c.gemm, c.tc);
  cta_gemm<T>(n, n, n, T(1), Psi, ld, false, lA, ld, false, T(0), nullptr, 0, false, oA, ld, c.gemm, c.tc);
  cta_gemm<T>(n, n, n, T(1), Psi, ld, false, lC, ld, false, T(0), nullptr, 0, false, U, ld, c.gemm, c.tc);
  cta_gemm<T>(n, n, n, T(1), U, ld, false, rA, ld, true, T(1), rC, ld, false, oC, ld, c.gemm, c.tc);
  return bad;
}

// Right operand is a complete suffix (A~ = C~ = 0, only P): P_out = (P A~)^T W A~ + P~.
template <typename T>
__device__ __noinline__ int combine_complete(Ctx<T>& c, const T* lP, const T* lA, const T* lC, const T* rP, T* oP) {
  const int n = c.d->nx, ld = c.d->ldx;
  T* X = c.scr;
  T* V = c.scr + 2 * c.msz;
  T* Wm = c.scr + 4 * c.msz;
  cta_gemm<T>(n, n, n, T(1), lC, ld, false, rP, ld, false, T(0), nullptr, 0, true, c.gj, GJ_LD, c.gemm, c.tc);
  const int bad = cta_inverse<T>(c.gj, GJ_LD, n, true, Wm, ld, c.gemm, c.perm, c.flag);
  cta_gemm<T>(n, n, n, T(1), Wm, ld, false, lA, ld, false, T(0), nullptr, 0, false, X, ld, c.gemm, c.tc);
  cta_gemm<T>(n, n, n, T(1), rP, ld, false, lA, ld, false, T(0), nullptr, 0, false, V, ld, c.gemm, c.tc);
  cta_gemm<T>(n, n, n, T(1), V, ld, true, X, ld, false, T(1), lP, ld, false, oP, ld, c.gemm, c.tc);
  return bad;
}

// Reduce an int flag (or) across the cluster through the part[] slots.
template <typename T>
__device__ int cluster_or(Ctx<T>& c, cg::cluster_group& cl, int v) {
  if (threadIdx.x == 0) c.part[15] = (double)v;
  cl.sync();
  int r = 0;
  for (int k = 0; k < c.cs; ++k) {
    double* p = cl.map_shared_rank(c.part, k);
    r |= (int)p[15];
  }
  cl.sync();
  return r;
}

// Tree schedule of the reverse scan (eq. combination_rules, App. A): up-sweep
// of full combines and down-sweep of complete-suffix combines level by level,
// then the gains (eq. controller_cache) and the iteration operators per stage.
template <typename T>
__device__ __noinline__ int tree_scan(Ctx<T>& c, cg::cluster_group& cl, T rho) {
  QPDesc& d = *c.d;
  const int nx = d.nx, nu = d.nu, nc = d.nc, N = d.N;
  const int ldx = d.ldx, ldu = d.ldu, ldc = d.ldc;
  const int msz = c.msz;
  const T *A = TP<T>(d.A), *B = TP<T>(d.B), *bb = TP<T>(d.b), *R = TP<T>(d.R);
  const T *q = TP<T>(d.q), *r = TP<T>(d.r), *C = TP<T>(d.C), *D = TP<T>(d.D);
  T *Sh = TP<T>(d.Sh), *VP = TP<T>(d.VP), *VA = TP<T>(d.VA), *VC = TP<T>(d.VC), *IP = TP<T>(d.IP);
  T *Abar = TP<T>(d.Abar), *CK = TP<T>(d.CK), *F = TP<T>(d.F), *J = TP<T>(d.J), *K = TP<T>(d.K);
  T *c0 = TP<T>(d.c0), *k0 = TP<T>(d.k0), *Gam = TP<T>(d.Gam);
  T* s0 = c.scr + 4 * msz;   // small temporaries (nu x nx etc.)
  T* s1 = c.scr + 5 * msz;
  int bad = 0;
  const int n = N + 1;
  // R2: up-sweep.  Block (d, m) covers leaves [m 2^d, min((m+1) 2^d, n)); the
  // last block of every level contains the terminal leaf and is complete.
  for (int lv = 0; lv < d.nlev; ++lv) {
    const int nd = level_count(n, lv), nd1 = level_count(n, lv + 1);
    for (int m = c.rank; m < nd1; m += c.cs) {
      const size_t li = (size_t)node_index(n, lv, 2 * m) * msz;
      const size_t oi = (size_t)node_index(n, lv + 1, m) * msz;
      if (2 * m + 1 >= nd) {
        cta_copy<T>(nx, nx, VP + li, ldx, false, VP + oi, ldx);
        cta_copy<T>(nx, nx, VA + li, ldx, false, VA + oi, ldx);
        cta_copy<T>(nx, nx, VC + li, ldx, false, VC + oi, ldx);
      } else {
        const size_t ri = (size_t)node_index(n, lv, 2 * m + 1) * msz;
        if (2 * m + 1 == nd - 1)
          bad |= combine_complete<T>(c, VP + li, VA + li, VC + li, VP + ri, VP + oi);
        else
          bad |= combine_full<T>(c, VP + li, VA + li, VC + li, VP + ri, VA + ri, VC + ri, VP + oi, VA + oi, VC + oi);
      }
    }
    cl.sync();
  }
  prof_mark(c, PH_R2);
  // R3: down-sweep of inclusive complete suffixes I(d, m) at block starts:
  // left children inherit the parent's, right children combine their own
  // block with the suffix after the parent block.
  if (c.rank == 0) {
    const size_t ri = (size_t)node_index(n, d.nlev, 0) * msz;
    cta_copy<T>(nx, nx, VP + ri, ldx, false, IP + ri, ldx);
  }
  cl.sync();
  for (int lv = d.nlev - 1; lv >= 0; --lv) {
    const int nd = level_count(n, lv), nd1 = level_count(n, lv + 1);
    // right children m = 2p+1 (the combines) spread evenly, then the copies
    const int nright = nd / 2;
    for (int p = c.rank; p < nright; p += c.cs) {
      const int m = 2 * p + 1;
      const size_t oi = (size_t)node_index(n, lv, m) * msz;
      if (p + 1 < nd1) {
        const size_t si = (size_t)node_index(n, lv + 1, p + 1) * msz;
        bad |= combine_complete<T>(c, VP + oi, VA + oi, VC + oi, IP + si, IP + oi);
      } else {
        cta_copy<T>(nx, nx, VP + oi, ldx, false, IP + oi, ldx);
      }
    }
    const int nleft = (nd + 1) / 2;
    for (int p = (c.rank + nright) % c.cs; p < nleft; p += c.cs) {
      const size_t oi = (size_t)node_index(n, lv, 2 * p) * msz;
      const size_t pi = (size_t)node_index(n, lv + 1, p) * msz;
      cta_copy<T>(nx, nx, IP + pi, ldx, false, IP + oi, ldx);
    }
    cl.sync();
  }
  prof_mark(c, PH_R3);
  // R4: gains (eq. controller_cache) and the per-stage iteration operators.
  if (c.active) {
    for (int i = c.s; i < c.e; ++i) {
      const T* Ai = A + (size_t)i * msz;
      const T* Bi = B + (size_t)i * nx * ldu;
      const T* Ci = C + (size_t)i * nc * ldx;
      const T* Di = D + (size_t)i * nc * ldu;
      const T* Pn = IP + (size_t)(i + 1) * msz;   // level-0 node i+1 = P_{i+1}
      T* Gi = Gam + (size_t)i * nu * ldu;
      T* Ki = K + (size_t)i * nu * ldx;
      T* Abi = Abar + (size_t)i * msz;
      // s0 = B^T P_{i+1} (nu x nx)
      cta_gemm<T>(nu, nx, nx, T(1), Bi, ldu, true, Pn, ldx, false, T(0), nullptr, 0, false, s0, ldx, c.gemm, c.tc);
      // Gamma^-1 = R^ + s0 B  (R^ rebuilt)
      cta_gemm<T>(nu, nu, nc, rho, Di, ldu, true, Di, ldu, false, T(1), R + (size_t)i * nu * ldu, ldu, false, c.gj, GJ_LD, c.gemm, c.tc);
      cta_gemm<T>(nu, nu, nx, T(1), s0, ldx, false, Bi, ldu, false, T(1), c.gj, GJ_LD, false, c.gj, GJ_LD, c.gemm, c.tc);
      bad |= cta_inverse<T>(c.gj, GJ_LD, nu, false, Gi, ldu, c.gemm, c.perm, c.flag);
      // s1 = S^ + s0 A ; K = -Gamma s1
      cta_gemm<T>(nu, nx, nx, T(1), s0, ldx, false, Ai, ldx, false, T(1), Sh + (size_t)i * nu * ldx, ldx, false, s1, ldx, c.gemm, c.tc);
      cta_gemm<T>(nu, nx, nu, T(-1), Gi, ldu, false, s1, ldx, false, T(0), nullptr, 0, false, Ki, ldx, c.gemm, c.tc);
      // Abar = A + B K ; CK = C + D K ; F = -Gamma B^T ; J = -Gamma D^T
      cta_gemm<T>(nx, nx, nu, T(1), Bi, ldu, false, Ki, ldx, false, T(1), Ai, ldx, false, Abi, ldx, c.gemm, c.tc);
      cta_gemm<T>(nc, nx, nu, T(1), Di, ldu, false, Ki, ldx, false, T(1), Ci, ldx, false, CK + (size_t)i * nc * ldx, ldx, c.gemm, c.tc);
      cta_gemm<T>(nu, nx, nu, T(-1), Gi, ldu, false, Bi, ldu, true, T(0), nullptr, 0, false, F + (size_t)i * nu * ldx, ldx, c.gemm, c.tc);
      cta_gemm<T>(nu, nc, nu, T(-1), Gi, ldu, false, Di, ldu, true, T(0), nullptr, 0, false, J + (size_t)i * nu * ldc, ldc, c.gemm, c.tc);
      // vectors: k0 = -Gamma (s0 b + r) ; c0 = Abar^T (P b) + q + K^T r
      const T* bi = bb + (size_t)i * ldx;
      for (int e2 = threadIdx.x; e2 < nx; e2 += NT) c.tmp3[e2] = bi[e2];
      __syncthreads();
      g_mv<T>(s0, ldx, nu, nx, c.tmp3, T(1), false, c.tmp1);          // tmp1 = s0 b
      for (int a = threadIdx.x; a < nu; a += NT) c.tmp1[a] += r[(size_t)i * ldu + a];
      __syncthreads();
      g_mv<T>(Gi, ldu, nu, nu, c.tmp1, T(-1), false, c.tmp2);          // tmp2 = k0
      for (int a = threadIdx.x; a < nu; a += NT) k0[(size_t)i * ldu + a] = c.tmp2[a];
      g_mv<T>(Pn, ldx, nx, nx, c.tmp3, T(1), false, c.tmp1);          // tmp1 = P b
      g_mvT<T>(Abi, ldx, nx, nx, c.tmp1, T(1), false, c.tmp2);        // tmp2 = Abar^T P b
      for (int a = threadIdx.x; a < nu; a += NT) c.tmp1[a] = r[(size_t)i * ldu + a];
      __syncthreads();
      g_mvT<T>(Ki, ldx, nu, nx, c.tmp1, T(1), true, c.tmp2);          // += K^T r
      for (int j = threadIdx.x; j < nx; j += NT) c0[(size_t)i * ldx + j] = c.tmp2[j] + q[(size_t)i * ldx + j];
      __syncthreads();
      // bundles of the cached iteration (layouts: see bundle_sizes)
      const int ldv = d.ldv, ldf = d.ldf, R = nx + nc;
      int bws, fws, cds;
      bundle_sizes(nx, nu, nc, ldx, ldu, ldv, ldf, &bws, &fws, &cds);
      T* bw = TP<T>(d.BW) + (size_t)i * bws;
      T* fw = TP<T>(d.FW) + (size_t)i * fws;
      T* cd = TP<T>(d.CD) + (size_t)i * cds;
      const T* CKi = CK + (size_t)i * nc * ldx;
      const T* Fi = F + (size_t)i * nu * ldx;
      const T* Ji = J + (size_t)i * nu * ldc;
      // (cta_fill: eight independent loads per thread before the stores)
      cta_fill<T>(bw, R * ldx, [&](int e2) {
        const int rr = e2 / ldx, j = e2 - rr * ldx;
        return (j >= nx) ? T(0) : (rr < nx ? Abi[(size_t)rr * ldx + j] : CKi[(size_t)(rr - nx) * ldx + j]);
      });
      T* fjt = bw + (size_t)R * ldx;           // [F | J]^T : row r, column a
      cta_fill<T>(fjt, R * ldu, [&](int e2) {
        const int rr = e2 / ldu, a = e2 - rr * ldu;
        return a >= nu ? T(0) : (rr < nx ? Fi[(size_t)a * ldx + rr] : Ji[(size_t)a * ldc + rr - nx]);
      });
      T* c0b = fjt + (size_t)R * ldu;
      cta_fill<T>(c0b, ldx + ldu, [&](int j) {
        return j < ldx ? (j < nx ? c0[(size_t)i * ldx + j] : T(0))
                       : (j - ldx < nu ? k0[(size_t)i * ldu + j - ldx] : T(0));
      });
      // FW^T: row cc < nx+nu (input index), column r < nx+nc (output index)
      cta_fill<T>(fw, (nx + nu) * ldv, [&](int e2) {
        const int cc = e2 / ldv, r2 = e2 - cc * ldv;
        T v = T(0);
        if (r2 < nx) v = cc < nx ? Abi[(size_t)r2 * ldx + cc] : Bi[(size_t)r2 * ldu + cc - nx];
        else if (r2 < R) v = cc < nx ? CKi[(size_t)(r2 - nx) * ldx + cc] : Di[(size_t)(r2 - nx) * ldu + cc - nx];
        return v;
      });
      cta_fill<T>(fw + (size_t)(nx + nu) * ldv, ldx, [&](int j) { return j < nx ? bb[(size_t)i * ldx + j] : T(0); });
      cta_fill<T>(cd, nc * ldf, [&](int e2) {
        const int rr = e2 / ldf, j = e2 - rr * ldf;
        return j < nx ? Ci[(size_t)rr * ldx + j] : (j < nx + nu ? Di[(size_t)rr * ldu + j - nx] : T(0));
      });
      __syncthreads();
    }
  }
  return bad;
}

// ---------------------------------------------------------------------------
// Blocked schedule of the reverse scan.
//
// The combine of eq. combination_rules with a stage leaf of eq. assoc_init as
// its left operand, e_ik = (P~_i, A~_i, C~_i = B_i R^_i^-1 B_i^T), and any
// right operand e_kj = (P_r, A_r, C_r): C~_i has rank nu, so with
//   Y^T = B_i^T P_r,  G = R^_i + Y^T B_i,  Gamma = G^-1,  H = Gamma Y^T A~_i,
// the Woodbury identity (I + C~_i P_r)^-1 = I - B_i Gamma Y^T gives
//   X = (I + C~_i P_r)^-1 A~_i = A~_i - B_i H,
//   P~_ij = P~_i + A~_i^T P_r X = P~_i + X^T P_r X + H^T R^_i H,
//   A~_ij = A_r X,
//   C~_ij = C_r + A_r (I + C~_i P_r)^-1 C~_i A_r^T = C_r + E Gamma E^T,  E = A_r B_i,
// inverting only the nu x nu block G.  With a complete right operand
// (P_r = P_{i+1}, A_r = C_r = 0) it is one Riccati step: X = Abar_i and
// K_i = -(R^_i^-1 S^_i + H) (eq. controller_cache).
//
// Schedule over the cluster's chunks [s_r, e_r):
//   A  chunks 1 .. nch-2 fold their leaves right to left into one element
//      T_r = e_{s_r} (x) ... (x) e_{e_r - 1}, while the last chunk, whose
//      suffix is complete from the terminal leaf on, runs its Riccati steps;
//   B  P_{s_r} = T_r (x) P_{s_{r+1}} for r = nch-2 .. 1, a general combine
//      with a complete right operand, one CTA after the other;
//   C  chunks 0 .. nch-2 run their Riccati steps from P_{e_r}.
// A Riccati step also forms its stage's gains and iteration operators.  The
// operands live in shared memory (the union region); only the stage inputs
// are fetched, by cp.async issued at the start of the step.
// ---------------------------------------------------------------------------
template <typename T>
struct FactBufs {
  T *P, *Aa, *Xb, *Bb[2], *Rb[2], *Db[2], *S1, *S2, *S3, *Gm, *Gi, *BG, *CKb[2], *JT, *v;
  int lds, vlen;
};

template <typename T>
__device__ inline FactBufs<T> fact_bufs(Ctx<T>& c) {
  const QPDesc& d = *c.d;
  const FactLayout f = fact_layout(d.nx, d.nu, d.nc, d.nf, d.ldx, d.ldu);
  T* b = c.ring;
  FactBufs<T> fb;
  fb.P = b + f.P;
  fb.Aa = b + f.Aa;
  fb.Xb = b + f.Xb;
  for (int k = 0; k < 2; ++k) {
    fb.Bb[k] = b + f.Bb[k];
    fb.Rb[k] = b + f.Rb[k];
    fb.Db[k] = b + f.Db[k];
  }
  fb.S1 = b + f.S1;
  fb.S2 = b + f.S2;
  fb.S3 = b + f.S3;
  fb.Gm = b + f.Gm;
  fb.Gi = b + f.Gi;
  fb.BG = b + f.BG;
  fb.CKb[0] = b + f.CKb[0];
  fb.CKb[1] = b + f.CKb[1];
  fb.JT = b + f.JT;
  fb.v = b + f.vec;
  fb.lds = f.lds;
  fb.vlen = f.vlen;
  return fb;
}

// cp.async (no wait) of stage i's B_i, R^_i and, for a Riccati step, D_i
// into buffer set k.
template <typename T>
__device__ inline void fact_prefetch(Ctx<T>& c, const FactBufs<T>& fb, int i, int k, bool withD) {
  const QPDesc& d = *c.d;
  const int esz = (int)sizeof(T);
  cta_stage(fb.Bb[k], TP<T>(d.B) + (size_t)i * d.nx * d.ldu, d.nx * d.ldu * esz);
  cta_stage(fb.Rb[k], TP<T>(d.Rh) + (size_t)i * d.nu * d.ldu, d.nu * d.ldu * esz);
  if (withD && d.nc > 0) cta_stage(fb.Db[k], TP<T>(d.D) + (size_t)i * d.nc * d.ldu, d.nc * d.ldu * esz);
}

// n x n (n <= FACT_MAX_NU) SPD inverse by one warp (the CTA for n > 16).
// GPUSLS_MIXED: the per-stage solve (Gamma_i, R^_i^-1) to FP64 accuracy: for
// n <= 16 the FP32 inverse refined with an FP64 residual (spd_inverse_refined,
// scratch E: n rows x lde, free shared memory), else the FP64 Gauss-Jordan.
template <typename T>
__device__ inline int small_spd_inverse(Ctx<T>& c, const T* G, int ldg, int n, T* Gi, int ldgi, T* E, int lde) {
  if (sizeof(T) == 4 && c.mix) {
    if (n <= 16 && n <= lde) return spd_inverse_refined<T, 16>(G, ldg, n, Gi, ldgi, c.flag + 1, E, lde);
    if (n <= 16) return warp_spd_inverse_as<T, double, 16>(G, ldg, n, Gi, ldgi, c.flag + 1);
    return warp_spd_inverse_as<T, double, FACT_MAX_NU>(G, ldg, n, Gi, ldgi, c.flag + 1);
  }
  if (n <= 16) return warp_spd_inverse<T, 16>(G, ldg, n, Gi, ldgi, c.flag + 1);
  return cta_spd_inverse<T>(G, ldg, n, Gi, ldgi, c.flag + 1, c.tmp1, c.tmp2);
}

// Phase A step: (P, Aa, Cacc) <- e_i (x) (P, Aa, Cacc).  Cacc stays in global
// memory (it is only ever updated, never a product operand).
template <typename T>
__device__ __noinline__ int fact_step_full(Ctx<T>& c, const FactBufs<T>& fb, int i, int k, T* Cacc) {
  const QPDesc& d = *c.d;
  const int nx = d.nx, nu = d.nu, ldx = d.ldx, ldu = d.ldu, lds = fb.lds;
  const int esz = (int)sizeof(T);
  T *Bb = fb.Bb[k], *Rb = fb.Rb[k];
  cta_stage_rows(fb.Xb, lds * esz, TP<T>(d.VA) + (size_t)i * c.msz, ldx * esz, nx, ldx * esz);   // A~_i
  if (i - 1 >= c.s) fact_prefetch<T>(c, fb, i - 1, k ^ 1, false);
  cp_async_commit();
  sgemm1<T>(nx, nu, nx, T(1), fb.P, lds, false, Bb, ldu, T(0), nullptr, 0, fb.S1, lds, true, c.mix);    // Y^T
  sgemm1<T>(nx, nu, nx, T(1), fb.Aa, lds, false, Bb, ldu, T(0), nullptr, 0, fb.S3, lds, true, c.mix);   // E^T
  sgemm1<T>(nu, nu, nx, T(1), fb.S1, lds, false, Bb, ldu, T(1), Rb, ldu, fb.Gm, ldu, false, c.mix);             // G
  const int bad = small_spd_inverse<T>(c, fb.Gm, ldu, nu, fb.Gi, ldu, fb.S2, lds);
  cp_async_wait<0>();
  __syncthreads();
  prof_mark(c, PH_FA1);
  sgemm1<T>(nu, nx, nx, T(1), fb.S1, lds, false, fb.Xb, lds, T(0), nullptr, 0, fb.S2, lds, false, c.mix);       // Y^T A~_i
  sgemm1<T>(nu, nx, nu, T(1), fb.Gi, ldu, false, fb.S2, lds, T(0), nullptr, 0, fb.S2, lds, false, c.mix);       // H
  sgemm1<T>(nx, nx, nu, T(-1), Bb, ldu, false, fb.S2, lds, T(1), fb.Xb, lds, fb.Xb, lds, false, c.mix);         // X
  sgemm1<T>(nu, nx, nu, T(1), fb.Gi, ldu, false, fb.S3, lds, T(0), nullptr, 0, fb.S1, lds, false, c.mix);       // Gamma E^T
  sgemm1<T>(nx, nx, nu, T(1), fb.S3, lds, true, fb.S1, lds, T(1), Cacc, ldx, Cacc, ldx, false, c.mix);          // C~_ij
  prof_mark(c, PH_FA2);
  sgemm1<T>(nx, nx, nx, T(1), fb.Aa, lds, false, fb.Xb, lds, T(0), nullptr, 0, fb.Aa, lds, false, c.mix);       // A~_ij
  sgemm1<T>(nx, nx, nx, T(1), fb.P, lds, false, fb.Xb, lds, T(0), nullptr, 0, fb.P, lds, false, c.mix);         // P_r X
  sgemm1<T>(nu, nx, nu, T(1), Rb, ldu, false, fb.S2, lds, T(0), nullptr, 0, fb.S1, lds, false, c.mix);          // R^ H
  sgemm<T>(nx, nx, T(1), MTerm<T>{fb.Xb, lds, true, fb.P, lds, nx}, MTerm<T>{fb.S2, lds, true, fb.S1, lds, nu},
           T(1), TP<T>(d.VP) + (size_t)i * c.msz, ldx, false, fb.P, lds, false, c.mix);                 // P~_ij
  prof_mark(c, PH_FA3);
  return bad;
}

// Iteration operators of stage i (layouts: see bundle_sizes) from the
// shared copies of Abar_i (Xb), B_i, D_i, CK_i, -B_i Gamma_i (= F_i^T),
// -D_i Gamma_i (= J_i^T), c0_i, k0_i and b_i; C_i from global memory.
template <typename T>
__device__ __noinline__ void fact_bundles(Ctx<T>& c, const FactBufs<T>& fb, int i, int k) {
  const QPDesc& d = *c.d;
  const int nx = d.nx, nu = d.nu, nc = d.nc, ldx = d.ldx, ldu = d.ldu, ldv = d.ldv, ldf = d.ldf;
  const int lds = fb.lds, R = nx + nc;
  int bws, fws, cds;
  bundle_sizes(nx, nu, nc, ldx, ldu, ldv, ldf, &bws, &fws, &cds);
  T* bw = TP<T>(d.BW) + (size_t)i * bws;
  T* fw = TP<T>(d.FW) + (size_t)i * fws;
  T* cd = TP<T>(d.CD) + (size_t)i * cds;
  const T* Ab = fb.Xb;
  const T* Bb = fb.Bb[k];
  const T* Db = fb.Db[k];
  const T* CKs = fb.CKb[0];
  const T* BG = fb.BG;
  const T* JT = fb.JT;
  const T* Ci = TP<T>(d.C) + (size_t)i * nc * ldx;
  const T* bv = fb.v;
  const T* c0v = fb.v + 5 * fb.vlen;
  const T* k0v = fb.v + 6 * fb.vlen;
  cta_fill<T>(bw, R * ldx, [&](int e2) {
    const int rr = e2 / ldx, j = e2 - rr * ldx;
    return (j >= nx) ? T(0) : (rr < nx ? Ab[rr * lds + j] : CKs[(rr - nx) * lds + j]);
  });
  T* fjt = bw + (size_t)R * ldx;   // [F | J]^T : row r, column a
  cta_fill<T>(fjt, R * ldu, [&](int e2) {
    const int rr = e2 / ldu, a = e2 - rr * ldu;
    return a >= nu ? T(0) : (rr < nx ? BG[rr * ldu + a] : JT[(rr - nx) * ldu + a]);
  });
  T* c0b = fjt + (size_t)R * ldu;
  cta_fill<T>(c0b, ldx + ldu, [&](int j) {
    return j < ldx ? (j < nx ? c0v[j] : T(0)) : (j - ldx < nu ? k0v[j - ldx] : T(0));
  });
  // FW^T: row cc < nx+nu (input index), column r < nx+nc (output index)
  cta_fill<T>(fw, (nx + nu) * ldv, [&](int e2) {
    const int cc = e2 / ldv, r2 = e2 - cc * ldv;
    T v = T(0);
    if (r2 < nx) v = cc < nx ? Ab[r2 * lds + cc] : Bb[r2 * ldu + cc - nx];
    else if (r2 < R) v = cc < nx ? CKs[(r2 - nx) * lds + cc] : Db[(r2 - nx) * ldu + cc - nx];
    return v;
  });
  cta_fill<T>(fw + (size_t)(nx + nu) * ldv, ldx, [&](int j) { return j < nx ? bv[j] : T(0); });
  cta_fill<T>(cd, nc * ldf, [&](int e2) {
    const int rr = e2 / ldf, j = e2 - rr * ldf;
    return j < nx ? Ci[(size_t)rr * ldx + j] : (j < nx + nu ? Db[rr * ldu + j - nx] : T(0));
  });
  __syncthreads();
}

// Riccati step of stage i from P_{i+1} (in P) to P_i, with the gains and
// the iteration operators of the stage (eq. controller_cache):
//   Gamma_i, K_i, Abar_i = X, CK_i = C_i + D_i K_i, F_i = -Gamma_i B_i^T,
//   J_i = -Gamma_i D_i^T, k0_i = -Gamma_i (B_i^T P_{i+1} b_i + r_i),
//   c0_i = Abar_i^T P_{i+1} b_i + q_i + K_i^T r_i,
// and, outside the last chunk, the backward chunk products with
// Pi_{i+1} (in Aa, Pi_e = I): FPi_i = F_i Pi_{i+1}, Pi_i = Abar_i^T Pi_{i+1}.
// ponly: the P recursion alone (P_i to IP, no gains, vectors or operators),
// by the same operations as the full step, so a later full pass from the same
// P_{i+1} reproduces it exactly.
template <typename T>
__device__ __noinline__ int fact_step_riccati(Ctx<T>& c, const FactBufs<T>& fb, int i, int k, bool ponly) {
  const QPDesc& d = *c.d;
  const int nx = d.nx, nu = d.nu, nc = d.nc, ldx = d.ldx, ldu = d.ldu, ldc = d.ldc, lds = fb.lds, msz = c.msz;
  const int esz = (int)sizeof(T), t = threadIdx.x;
  T *Bb = fb.Bb[k], *Rb = fb.Rb[k], *Db = fb.Db[k];
  T *bv = fb.v, *pb = fb.v + fb.vlen, *rv = fb.v + 2 * fb.vlen, *qv = fb.v + 3 * fb.vlen, *tv = fb.v + 4 * fb.vlen;
  T *c0v = fb.v + 5 * fb.vlen, *k0v = fb.v + 6 * fb.vlen;
  cta_stage_rows(fb.Xb, lds * esz, TP<T>(d.VA) + (size_t)i * msz, ldx * esz, nx, ldx * esz);    // A~_i
  cta_stage_rows(fb.S3, lds * esz, TP<T>(d.S0) + (size_t)i * nu * ldx, ldx * esz, nu, ldx * esz);  // R^-1 S^
  if (i - 1 >= c.s) fact_prefetch<T>(c, fb, i - 1, k ^ 1, true);
  cp_async_commit();
  if (!ponly) {
    for (int e = t; e < nx; e += NT) {
      bv[e] = TP<T>(d.b)[(size_t)i * ldx + e];
      qv[e] = TP<T>(d.q)[(size_t)i * ldx + e];
    }
    for (int e = t; e < nu; e += NT) rv[e] = TP<T>(d.r)[(size_t)i * ldu + e];
    __syncthreads();
    smem_mvT<T>(fb.P, lds, nx, nx, bv, nullptr, pb, c.red);                                       // P_{i+1} b_i (P symmetric)
  }
  sgemm1<T>(nx, nu, nx, T(1), fb.P, lds, false, Bb, ldu, T(0), nullptr, 0, fb.S1, lds, true, c.mix);    // Y^T
  sgemm1<T>(nu, nu, nx, T(1), fb.S1, lds, false, Bb, ldu, T(1), Rb, ldu, fb.Gm, ldu, false, c.mix);             // Gamma^-1
  const int bad = small_spd_inverse<T>(c, fb.Gm, ldu, nu, fb.Gi, ldu, fb.S2, lds);
  cp_async_wait<0>();
  __syncthreads();
  prof_mark(c, PH_FC1);
  sgemm1<T>(nu, nx, nx, T(1), fb.S1, lds, false, fb.Xb, lds, T(0), nullptr, 0, fb.S2, lds, false, c.mix);       // Y^T A~_i
  sgemm1<T>(nu, nx, nu, T(1), fb.Gi, ldu, false, fb.S2, lds, T(0), nullptr, 0, fb.S2, lds, false, c.mix);       // H
  sgemm1<T>(nx, nx, nu, T(-1), Bb, ldu, false, fb.S2, lds, T(1), fb.Xb, lds, fb.Xb, lds, false, c.mix);         // Abar_i
  if (!ponly) {
    T* Kg = TP<T>(d.K) + (size_t)i * nu * ldx;
    for (int e = t; e < nu * nx; e += NT) {
      const int a = e / nx, j = e - a * nx;
      const T v = -(fb.S3[a * lds + j] + fb.S2[a * lds + j]);
      fb.S1[a * lds + j] = v;
      Kg[(size_t)a * ldx + j] = v;
    }
    __syncthreads();
    smem_mvT<T>(Bb, ldu, nx, nu, pb, rv, tv, c.red);       // B^T P b + r
    smem_mvT<T>(fb.Xb, lds, nx, nx, pb, qv, c0v, c.red);   // Abar^T P b + q
    smem_mvT<T>(fb.S1, lds, nu, nx, rv, c0v, c0v, c.red);  // ... + K^T r
    smem_mv<T>(fb.Gi, ldu, nu, nu, tv, nullptr, k0v);
    if (t < nu) k0v[t] = -k0v[t];
    __syncthreads();
  }
  prof_mark(c, PH_FC2);
  // P_i = P~_i + X^T (P_{i+1} X) + H^T (R^ H)
  sgemm1<T>(nx, nx, nx, T(1), fb.P, lds, false, fb.Xb, lds, T(0), nullptr, 0, fb.P, lds, false, c.mix);
  sgemm1<T>(nu, nx, nu, T(1), Rb, ldu, false, fb.S2, lds, T(0), nullptr, 0, fb.S3, lds, false, c.mix);
  sgemm<T>(nx, nx, T(1), MTerm<T>{fb.Xb, lds, true, fb.P, lds, nx}, MTerm<T>{fb.S2, lds, true, fb.S3, lds, nu},
           T(1), TP<T>(d.VP) + (size_t)i * msz, ldx, false, fb.P, lds, false, c.mix);
  prof_mark(c, PH_FC3);
  if (ponly) {
    cta_copy_vec<T>(nx, nx, fb.P, lds, TP<T>(d.IP) + (size_t)i * msz, ldx);
    return bad;
  }
  // stage outputs: -B Gamma (= F_i^T), -D Gamma (= J_i^T), CK_i = C_i + D_i K_i
  sgemm1<T>(nx, nu, nu, T(-1), Bb, ldu, false, fb.Gi, ldu, T(0), nullptr, 0, fb.BG, ldu, false, c.mix);
  sgemm1<T>(nc, nu, nu, T(-1), Db, ldu, false, fb.Gi, ldu, T(0), nullptr, 0, fb.JT, ldu, false, c.mix);
  sgemm1<T>(nc, nx, nu, T(1), Db, ldu, false, fb.S1, lds, T(1), TP<T>(d.C) + (size_t)i * nc * ldx, ldx, fb.CKb[0], lds, false, c.mix);
  cta_copy_vec<T>(nx, nx, fb.P, lds, TP<T>(d.IP) + (size_t)i * msz, ldx);
  cta_copy_vec<T>(nx, nx, fb.Xb, lds, TP<T>(d.Abar) + (size_t)i * msz, ldx);
  cta_copy_vec<T>(nu, nu, fb.Gi, ldu, TP<T>(d.Gam) + (size_t)i * nu * ldu, ldu);
  cta_copy_vec<T>(nc, nx, fb.CKb[0], lds, TP<T>(d.CK) + (size_t)i * nc * ldx, ldx);
  for (int e = t; e < nx; e += NT) TP<T>(d.c0)[(size_t)i * ldx + e] = c0v[e];
  for (int e = t; e < nu; e += NT) TP<T>(d.k0)[(size_t)i * ldu + e] = k0v[e];
  if (c.gains) {
    prof_mark(c, PH_FC4);
    return bad;
  }
  if (!c.last) {
    // backward chunk products (Pi in Aa): FPi_i^T = Pi_{i+1}^T F_i^T, Pi_i = Abar_i^T Pi_{i+1}
    sgemm1<T>(nx, nu, nx, T(1), fb.Aa, lds, true, fb.BG, ldu, T(0), nullptr, 0,
              TP<T>(d.FPi) + (size_t)i * nx * ldu, ldu, false, c.mix);
    sgemm1<T>(nx, nx, nx, T(1), fb.Xb, lds, true, fb.Aa, lds, T(0), nullptr, 0, fb.Aa, lds, false, c.mix);
  }
  prof_mark(c, PH_FC4);
  fact_bundles<T>(c, fb, i, k);
  prof_mark(c, PH_FC5);
  return bad;
}

template <typename T>
__device__ __noinline__ int blocked_scan(Ctx<T>& c, cg::cluster_group& cl) {
  QPDesc& d = *c.d;
  const int nx = d.nx, ldx = d.ldx, msz = c.msz, N = d.N, nch = d.nch;
  const int esz = (int)sizeof(T);
  T *VP = TP<T>(d.VP), *VA = TP<T>(d.VA), *VC = TP<T>(d.VC), *IP = TP<T>(d.IP);
  const FactBufs<T> fb = fact_bufs<T>(c);
  const int lds = fb.lds;
  const int n = N + 1;   // leaves; chunk elements T_r are kept at tree nodes n + r
  int bad = 0;
  // With more than one chunk the last chunk runs only the P recursion in A,
  // beside the other chunks' folds (a full Riccati step, with its gains and
  // operators, costs about twice a fold step), and its full steps in C,
  // beside theirs.
  const bool split_last = nch > 1;
  if (c.active && c.last) {
    // A (last chunk): Riccati steps from the terminal leaf, P_N = Q^_N
    cta_stage_rows(fb.P, lds * esz, VP + (size_t)N * msz, ldx * esz, nx, ldx * esz);
    fact_prefetch<T>(c, fb, c.e - 1, 0, true);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    cta_copy_vec<T>(nx, nx, fb.P, lds, IP + (size_t)N * msz, ldx);
    int k = 0;
    for (int i = c.e - 1; i >= c.s; --i, k ^= 1) bad |= fact_step_riccati<T>(c, fb, i, k, split_last);
  } else if (c.active && c.rank >= 1) {
    // A: T_r, starting from the chunk's last leaf
    const int i0 = c.e - 1;
    T* Cacc = VC + (size_t)(n + c.rank) * msz;
    cta_stage_rows(fb.P, lds * esz, VP + (size_t)i0 * msz, ldx * esz, nx, ldx * esz);
    cta_stage_rows(fb.Aa, lds * esz, VA + (size_t)i0 * msz, ldx * esz, nx, ldx * esz);
    if (i0 - 1 >= c.s) fact_prefetch<T>(c, fb, i0 - 1, 0, false);
    cp_async_commit();
    cta_copy_vec<T>(nx, nx, VC + (size_t)i0 * msz, ldx, Cacc, ldx);
    cp_async_wait<0>();
    __syncthreads();
    int k = 0;
    for (int i = i0 - 1; i >= c.s; --i, k ^= 1) bad |= fact_step_full<T>(c, fb, i, k, Cacc);
    cta_copy_vec<T>(nx, nx, fb.P, lds, VP + (size_t)(n + c.rank) * msz, ldx);
    cta_copy_vec<T>(nx, nx, fb.Aa, lds, VA + (size_t)(n + c.rank) * msz, ldx);
  }
  cl.sync();
  prof_mark(c, PH_R2);
  // B: P_{s_r} = T_r (x) P_{e_r}, r = nch-2 .. 1
  for (int r = nch - 2; r >= 1; --r) {
    if (c.rank == r) {
      const size_t ti = (size_t)(n + r) * msz;
      bad |= combine_complete<T>(c, VP + ti, VA + ti, VC + ti, IP + (size_t)c.e * msz, IP + (size_t)c.s * msz);
    }
    cl.sync();
  }
  prof_mark(c, PH_R3);
  // C: Riccati steps of chunks 0 .. nch-2 from P_{e_r} (and of the last
  // chunk from P_N again, when A ran only its P recursion)
  if (c.active && (!c.last || split_last)) {
    cta_stage_rows(fb.P, lds * esz, IP + (size_t)(c.last ? N : c.e) * msz, ldx * esz, nx, ldx * esz);
    fact_prefetch<T>(c, fb, c.e - 1, 0, true);
    cp_async_commit();
    if (!c.last) cta_eye<T>(nx, fb.Aa, lds);   // Pi_e
    cp_async_wait<0>();
    __syncthreads();
    int k = 0;
    for (int i = c.e - 1; i >= c.s; --i, k ^= 1) bad |= fact_step_riccati<T>(c, fb, i, k, false);
    if (!c.last) cta_copy_vec<T>(nx, nx, fb.Aa, lds, TP<T>(d.Tch) + (size_t)c.rank * msz, ldx);   // T_r = Pi_s
  }
  return bad;
}

// R1 of the blocked schedule: the stage leaves of eq. assoc_init with
// shared-memory GEMMs,
//   Q^ = Q + rho C^T C,  R^ = R + rho D^T D,  S^ = S + rho D^T C,
//   s0 = R^^-1 S^,  P~ = Q^ - S^^T s0,  A~ = A - B s0,
// kept in global memory (P~, A~, R^, s0) for the phases of blocked_scan; C~ =
// B R^^-1 B^T only for the last leaf of chunks 1 .. nch-2 (the start of their
// fold); the last chunk also forms the terminal leaf P~_N = Q_N + rho C_N^T C_N.
template <typename T>
__device__ __noinline__ int leaves_blocked(Ctx<T>& c, T rho) {
  QPDesc& d = *c.d;
  if (!c.active) return 0;
  const int nx = d.nx, nu = d.nu, nc = d.nc, nf = d.nf, N = d.N, ldx = d.ldx, ldu = d.ldu, msz = c.msz;
  const int esz = (int)sizeof(T);
  const FactBufs<T> fb = fact_bufs<T>(c);
  const int lds = fb.lds;
  int bad = 0;
  const bool need_ct = c.rank >= 1 && !c.last;
  for (int i = c.s; i < c.e; ++i) {
    cta_stage_rows(fb.P, lds * esz, TP<T>(d.Q) + (size_t)i * msz, ldx * esz, nx, ldx * esz);
    cta_stage_rows(fb.Xb, lds * esz, TP<T>(d.A) + (size_t)i * msz, ldx * esz, nx, ldx * esz);
    cta_stage_rows(fb.S3, lds * esz, TP<T>(d.S) + (size_t)i * nu * ldx, ldx * esz, nu, ldx * esz);
    if (nc > 0) {
      cta_stage_rows(fb.CKb[0], lds * esz, TP<T>(d.C) + (size_t)i * nc * ldx, ldx * esz, nc, ldx * esz);
      cta_stage(fb.Db[0], TP<T>(d.D) + (size_t)i * nc * ldu, nc * ldu * esz);
    }
    cta_stage(fb.Bb[0], TP<T>(d.B) + (size_t)i * nx * ldu, nx * ldu * esz);
    cta_stage(fb.Rb[0], TP<T>(d.R) + (size_t)i * nu * ldu, nu * ldu * esz);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    sgemm1<T>(nx, nx, nc, rho, fb.CKb[0], lds, true, fb.CKb[0], lds, T(1), fb.P, lds, fb.P, lds, false, c.mix);      // Q^
    sgemm1<T>(nu, nu, nc, rho, fb.Db[0], ldu, true, fb.Db[0], ldu, T(1), fb.Rb[0], ldu, fb.Gm, ldu, false, c.mix);   // R^
    sgemm1<T>(nu, nx, nc, rho, fb.Db[0], ldu, true, fb.CKb[0], lds, T(1), fb.S3, lds, fb.S1, lds, false, c.mix);     // S^
    cta_copy_vec<T>(nu, nu, fb.Gm, ldu, TP<T>(d.Rh) + (size_t)i * nu * ldu, ldu);
    bad |= small_spd_inverse<T>(c, fb.Gm, ldu, nu, fb.Gi, ldu, fb.S2, lds);
    sgemm1<T>(nu, nx, nu, T(1), fb.Gi, ldu, false, fb.S1, lds, T(0), nullptr, 0, fb.S2, lds, false, c.mix);          // s0
    sgemm1<T>(nx, nx, nu, T(-1), fb.S1, lds, true, fb.S2, lds, T(1), fb.P, lds, fb.P, lds, false, c.mix);            // P~
    sgemm1<T>(nx, nx, nu, T(-1), fb.Bb[0], ldu, false, fb.S2, lds, T(1), fb.Xb, lds, fb.Xb, lds, false, c.mix);      // A~
    cta_copy_vec<T>(nu, nx, fb.S2, lds, TP<T>(d.S0) + (size_t)i * nu * ldx, ldx);
    cta_copy_vec<T>(nx, nx, fb.P, lds, TP<T>(d.VP) + (size_t)i * msz, ldx);
    cta_copy_vec<T>(nx, nx, fb.Xb, lds, TP<T>(d.VA) + (size_t)i * msz, ldx);
    if (need_ct && i == c.e - 1) {
      // C~ = B (B R^^-1)^T
      sgemm1<T>(nx, nu, nu, T(1), fb.Bb[0], ldu, false, fb.Gi, ldu, T(0), nullptr, 0, fb.S3, lds, true, c.mix);
      sgemm1<T>(nx, nx, nu, T(1), fb.Bb[0], ldu, false, fb.S3, lds, T(0), nullptr, 0,
                TP<T>(d.VC) + (size_t)i * msz, ldx, false, c.mix);
    }
  }
  if (c.last) {
    cta_stage_rows(fb.P, lds * esz, TP<T>(d.Q) + (size_t)N * msz, ldx * esz, nx, ldx * esz);
    if (nf > 0) cta_stage_rows(fb.CKb[0], lds * esz, TP<T>(d.CN), ldx * esz, nf, ldx * esz);
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    sgemm1<T>(nx, nx, nf, rho, fb.CKb[0], lds, true, fb.CKb[0], lds, T(1), fb.P, lds, fb.P, lds, false, c.mix);
    cta_copy_vec<T>(nx, nx, fb.P, lds, TP<T>(d.VP) + (size_t)N * msz, ldx);
  }
  return bad;
}

// Forward chunk products of the blocked schedule (not needed in the first
// chunk): Sig_s = I, Sig_{i+1} = Abar_i Sig_i, KSig_i = K_i Sig_i,
// CKSig_i = (CK_i Sig_i)^T (stored transposed), U_r = Sig_e; the last chunk
// also Sig_N and C_N Sig_N.  Sig stays in shared memory; the next stage's
// Abar, K and CK are fetched while the current one is used.
template <typename T>
__device__ __noinline__ void forward_products(Ctx<T>& c) {
  QPDesc& d = *c.d;
  if (!c.active || c.first) return;
  const int nx = d.nx, nu = d.nu, nc = d.nc, nf = d.nf, ldx = d.ldx, ldc = d.ldc, msz = c.msz;
  const int esz = (int)sizeof(T);
  const FactBufs<T> fb = fact_bufs<T>(c);
  const int lds = fb.lds;
  T* Sg = fb.P;
  T* const Ab[2] = {fb.Xb, fb.Aa};
  T* const Kb[2] = {fb.S1, fb.S2};
  auto issue = [&](int i, int k) {
    cta_stage_rows(Ab[k], lds * esz, TP<T>(d.Abar) + (size_t)i * msz, ldx * esz, nx, ldx * esz);
    cta_stage_rows(Kb[k], lds * esz, TP<T>(d.K) + (size_t)i * nu * ldx, ldx * esz, nu, ldx * esz);
    if (nc > 0) cta_stage_rows(fb.CKb[k], lds * esz, TP<T>(d.CK) + (size_t)i * nc * ldx, ldx * esz, nc, ldx * esz);
    cp_async_commit();
  };
  issue(c.s, 0);
  cta_eye<T>(nx, Sg, lds);
  int k = 0;
  for (int i = c.s; i < c.e; ++i, k ^= 1) {
    if (i + 1 < c.e) {
      issue(i + 1, k ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    cta_copy_vec<T>(nx, nx, Sg, lds, TP<T>(d.Sig) + (size_t)i * msz, ldx);
    sgemm1<T>(nu, nx, nx, T(1), Kb[k], lds, false, Sg, lds, T(0), nullptr, 0, TP<T>(d.KSig) + (size_t)i * nu * ldx, ldx, false, c.mix);
    sgemm1<T>(nc, nx, nx, T(1), fb.CKb[k], lds, false, Sg, lds, T(0), nullptr, 0,
              TP<T>(d.CKSig) + (size_t)i * nx * ldc, ldc, true, c.mix);
    sgemm1<T>(nx, nx, nx, T(1), Ab[k], lds, false, Sg, lds, T(0), nullptr, 0, Sg, lds, false, c.mix);
  }
  cta_copy_vec<T>(nx, nx, Sg, lds, TP<T>(d.Uch) + (size_t)c.rank * msz, ldx);
  if (c.last) {
    cta_copy_vec<T>(nx, nx, Sg, lds, TP<T>(d.SigN), ldx);
    if (nf > 0) {
      cta_stage_rows(fb.CKb[0], lds * esz, TP<T>(d.CN), ldx * esz, nf, ldx * esz);
      cp_async_commit();
      cp_async_wait<0>();
      __syncthreads();
      sgemm1<T>(nf, nx, nx, T(1), fb.CKb[0], lds, false, Sg, lds, T(0), nullptr, 0, TP<T>(d.CNSig), ldx, false, c.mix);
    }
  }
}

// ---------------------------------------------------------------------------
// rho-dependent factorization (the "refactor")
// ---------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ int refactor(Ctx<T>& c, cg::cluster_group& cl, T rho) {
  QPDesc& d = *c.d;
  const int nx = d.nx, nu = d.nu, nc = d.nc, nf = d.nf, N = d.N;
  const int ldx = d.ldx, ldu = d.ldu, ldc = d.ldc;
  const int msz = c.msz;
  const T *A = TP<T>(d.A), *B = TP<T>(d.B), *bb = TP<T>(d.b), *Q = TP<T>(d.Q), *R = TP<T>(d.R), *S = TP<T>(d.S);
  const T *q = TP<T>(d.q), *r = TP<T>(d.r), *C = TP<T>(d.C), *D = TP<T>(d.D), *CN = TP<T>(d.CN);
  T *Rhi = TP<T>(d.Rhi), *Sh = TP<T>(d.Sh), *VP = TP<T>(d.VP), *VA = TP<T>(d.VA), *VC = TP<T>(d.VC), *IP = TP<T>(d.IP);
  T *Abar = TP<T>(d.Abar), *CK = TP<T>(d.CK), *F = TP<T>(d.F), *FPi = TP<T>(d.FPi), *J = TP<T>(d.J), *K = TP<T>(d.K);
  T *KSig = TP<T>(d.KSig), *CKSig = TP<T>(d.CKSig), *Sig = TP<T>(d.Sig), *c0 = TP<T>(d.c0), *k0 = TP<T>(d.k0);
  T *CNSig = TP<T>(d.CNSig), *SigN = TP<T>(d.SigN), *Tch = TP<T>(d.Tch), *Uch = TP<T>(d.Uch);
  T *Theta = TP<T>(d.Theta), *Xi = TP<T>(d.Xi), *Gam = TP<T>(d.Gam);
  T* s1 = c.scr + 5 * msz;   // small temporary (nx x nu)
  T *Rh = TP<T>(d.Rh), *S0 = TP<T>(d.S0);
  int bad = 0;

  // R1: leaves (eq. assoc_init) for own stages, terminal by the last chunk.
  if (d.fact == 0) bad |= leaves_blocked<T>(c, rho);
  else if (c.active) {
    for (int i = c.s; i < c.e; ++i) {
      const T* Ai = A + (size_t)i * msz;
      const T* Bi = B + (size_t)i * nx * ldu;
      const T* Ci = C + (size_t)i * nc * ldx;
      const T* Di = D + (size_t)i * nc * ldu;
      T* Pl = VP + (size_t)i * msz;
      T* Al = VA + (size_t)i * msz;
      T* Cl = VC + (size_t)i * msz;
      T* Shi = Sh + (size_t)i * nu * ldx;
      T* Rhii = Rhi + (size_t)i * nu * ldu;
      // Q^ = Q + rho C^T C,  R^ = R + rho D^T D,  S^ = S + rho D^T C
      cta_gemm<T>(nx, nx, nc, rho, Ci, ldx, true, Ci, ldx, false, T(1), Q + (size_t)i * msz, ldx, false, Pl, ldx, c.gemm, c.tc);
      cta_gemm<T>(nu, nu, nc, rho, Di, ldu, true, Di, ldu, false, T(1), R + (size_t)i * nu * ldu, ldu, false, c.gj, GJ_LD, c.gemm, c.tc);
      cta_copy<T>(nu, nu, c.gj, GJ_LD, false, Rh + (size_t)i * nu * ldu, ldu);   // R^ kept for the blocked scan
      cta_gemm<T>(nu, nx, nc, rho, Di, ldu, true, Ci, ldx, false, T(1), S + (size_t)i * nu * ldx, ldx, false, Shi, ldx, c.gemm, c.tc);
      bad |= cta_inverse<T>(c.gj, GJ_LD, nu, false, Rhii, ldu, c.gemm, c.perm, c.flag);
      // s0 = R^-1 S^ (kept: K_i = -(s0 + H_i) in the blocked scan) ; P~ = Q^ - S^^T s0 ;
      // A~ = A - B s0 ; s1 = B R^-1 ; C~ = s1 B^T
      T* s0 = S0 + (size_t)i * nu * ldx;
      cta_gemm<T>(nu, nx, nu, T(1), Rhii, ldu, false, Shi, ldx, false, T(0), nullptr, 0, false, s0, ldx, c.gemm, c.tc);
      cta_gemm<T>(nx, nx, nu, T(-1), Shi, ldx, true, s0, ldx, false, T(1), Pl, ldx, false, Pl, ldx, c.gemm, c.tc);
      cta_gemm<T>(nx, nx, nu, T(-1), Bi, ldu, false, s0, ldx, false, T(1), Ai, ldx, false, Al, ldx, c.gemm, c.tc);
      cta_gemm<T>(nx, nu, nu, T(1), Bi, ldu, false, Rhii, ldu, false, T(0), nullptr, 0, false, s1, ldu, c.gemm, c.tc);
      cta_gemm<T>(nx, nx, nu, T(1), s1, ldu, false, Bi, ldu, true, T(0), nullptr, 0, false, Cl, ldx, c.gemm, c.tc);
    }
    if (c.last) {
      T* Pl = VP + (size_t)N * msz;
      cta_gemm<T>(nx, nx, nf, rho, CN, ldx, true, CN, ldx, false, T(1), Q + (size_t)N * msz, ldx, false, Pl, ldx, c.gemm, c.tc);
      cta_zero<T>(nx, nx, VA + (size_t)N * msz, ldx);
      cta_zero<T>(nx, nx, VC + (size_t)N * msz, ldx);
    }
  }
  cl.sync();
  prof_mark(c, PH_R1);

  if (d.fact == 0) bad |= blocked_scan<T>(c, cl);
  else bad |= tree_scan<T>(c, cl, rho);
  cl.sync();
  prof_mark(c, PH_R4);
  if (c.gains) {
    const int res = cluster_or<T>(c, cl, bad);
    prof_mark(c, PH_R6);
    return res;
  }
  // R5: chunk products.  Backward (not needed in the last chunk):
  //   FPi_i = F_i Pi_{i+1},  Pi_i = Abar_i^T Pi_{i+1},  Pi_e = I,  T_r = Pi_s.
  // Forward (not needed in the first chunk):
  //   Sig_s = I, Sig_{i+1} = Abar_i Sig_i, KSig_i = K_i Sig_i,
  //   CKSig_i = CK_i Sig_i, U_r = Sig_e; the last chunk also C_N Sig_N.
  if (d.fact == 0) forward_products<T>(c);   // backward products came with the Riccati steps
  else if (c.active) {
    if (!c.last) {
      T* Pc = c.scr;
      T* Pn2 = c.scr + c.msz;
      const int i1 = c.e - 1;
      // FPi stored transposed: FPi_i^T = Pi_{i+1}^T F_i^T  (nx x ldu)
      cta_copy<T>(nu, nx, F + (size_t)i1 * nu * ldx, ldx, true, FPi + (size_t)i1 * nx * ldu, ldu);
      cta_copy<T>(nx, nx, Abar + (size_t)i1 * msz, ldx, true, Pc, ldx);
      for (int i = c.e - 2; i >= c.s; --i) {
        cta_gemm<T>(nx, nu, nx, T(1), Pc, ldx, true, F + (size_t)i * nu * ldx, ldx, true, T(0), nullptr, 0, false,
                    FPi + (size_t)i * nx * ldu, ldu, c.gemm, c.tc);
        cta_gemm<T>(nx, nx, nx, T(1), Abar + (size_t)i * msz, ldx, true, Pc, ldx, false, T(0), nullptr, 0, false, Pn2,
                    ldx, c.gemm, c.tc);
        T* t_ = Pc; Pc = Pn2; Pn2 = t_;
      }
      cta_copy<T>(nx, nx, Pc, ldx, false, Tch + (size_t)c.rank * msz, ldx);
    }
    if (!c.first) {
      cta_eye<T>(nx, Sig + (size_t)c.s * msz, ldx);
      cta_copy<T>(nu, nx, K + (size_t)c.s * nu * ldx, ldx, false, KSig + (size_t)c.s * nu * ldx, ldx);
      // CKSig stored transposed: CKSig_i^T = Sig_i^T CK_i^T  (nx x ldc)
      cta_copy<T>(nc, nx, CK + (size_t)c.s * nc * ldx, ldx, true, CKSig + (size_t)c.s * nx * ldc, ldc);
      for (int i = c.s + 1; i < c.e; ++i) {
        T* Si = Sig + (size_t)i * msz;
        cta_gemm<T>(nx, nx, nx, T(1), Abar + (size_t)(i - 1) * msz, ldx, false, Sig + (size_t)(i - 1) * msz, ldx, false,
                    T(0), nullptr, 0, false, Si, ldx, c.gemm, c.tc);
        cta_gemm<T>(nu, nx, nx, T(1), K + (size_t)i * nu * ldx, ldx, false, Si, ldx, false, T(0), nullptr, 0, false,
                    KSig + (size_t)i * nu * ldx, ldx, c.gemm, c.tc);
        cta_gemm<T>(nx, nc, nx, T(1), Si, ldx, true, CK + (size_t)i * nc * ldx, ldx, true, T(0), nullptr, 0, false,
                    CKSig + (size_t)i * nx * ldc, ldc, c.gemm, c.tc);
      }
      T* Ur = Uch + (size_t)c.rank * msz;
      cta_gemm<T>(nx, nx, nx, T(1), Abar + (size_t)(c.e - 1) * msz, ldx, false, Sig + (size_t)(c.e - 1) * msz, ldx,
                  false, T(0), nullptr, 0, false, Ur, ldx, c.gemm, c.tc);
      if (c.last) {
        cta_copy<T>(nx, nx, Ur, ldx, false, SigN, ldx);
        cta_gemm<T>(nf, nx, nx, T(1), CN, ldx, false, SigN, ldx, false, T(0), nullptr, 0, false, CNSig, ldx, c.gemm, c.tc);
      }
    }
  }
  cl.sync();
  prof_mark(c, PH_R5);
  // R6: chunk-boundary operators Theta_{r,m} = T_{r+1} ... T_{m-1} (m >= r+2)
  // and Xi_{r,m} = U_{r-1} ... U_{m+1} (m <= r-2).
  if (c.active) {
    const int r0 = c.rank, nch = d.nch;
    // stored transposed: Theta_{r,m}^T = T_{m-1}^T Theta_{r,m-1}^T, Xi_{r,m-1}^T = U_m^T Xi_{r,m}^T
    for (int m = r0 + 2; m < nch; ++m) {
      T* Th = Theta + (size_t)(r0 * nch + m) * msz;
      if (m == r0 + 2) cta_copy<T>(nx, nx, Tch + (size_t)(r0 + 1) * msz, ldx, true, Th, ldx);
      else cta_gemm<T>(nx, nx, nx, T(1), Tch + (size_t)(m - 1) * msz, ldx, true,
                       Theta + (size_t)(r0 * nch + m - 1) * msz, ldx, false, T(0), nullptr, 0, false, Th, ldx, c.gemm, c.tc);
    }
    for (int m = r0 - 2; m >= 0; --m) {
      T* X = Xi + (size_t)(r0 * nch + m) * msz;
      if (m == r0 - 2) cta_copy<T>(nx, nx, Uch + (size_t)(r0 - 1) * msz, ldx, true, X, ldx);
      else cta_gemm<T>(nx, nx, nx, T(1), Uch + (size_t)(m + 1) * msz, ldx, true,
                       Xi + (size_t)(r0 * nch + m + 1) * msz, ldx, false, T(0), nullptr, 0, false, X, ldx, c.gemm, c.tc);
    }
  }
  const int res = cluster_or<T>(c, cl, bad);
  prof_mark(c, PH_R6);
  return res;
}

}  // namespace gsls
