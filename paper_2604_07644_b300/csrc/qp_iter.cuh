// ADMM iteration, residuals, rho rule and FP64 KKT check of the persistent
// solve kernel (Sec. IV-A).  See qp_kernel.cuh for the cluster layout.
#pragma once
#include "qp_kernel.cuh"

namespace gsls {

template <typename T>
__device__ T block_max(Ctx<T>& c, T v) {
  v = warp_max(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) c.red[w] = v;
  __syncthreads();
  T r = T(0);
  for (int k = 0; k < NT / 32; ++k) r = fmax(r, c.red[k]);
  __syncthreads();
  return r;
}

// Block-level max of three values in one round (three CTA barriers, not nine).
template <typename T>
__device__ void block_max3(Ctx<T>& c, T& a, T& b, T& d) {
  a = warp_max(a);
  b = warp_max(b);
  d = warp_max(d);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  constexpr int NW = NT / 32;
  __syncthreads();
  if (l == 0) {
    c.red[w] = a;
    c.red[NW + w] = b;
    c.red[2 * NW + w] = d;
  }
  __syncthreads();
  a = b = d = T(0);
#pragma unroll
  for (int k = 0; k < NW; ++k) {
    a = fmax(a, c.red[k]);
    b = fmax(b, c.red[NW + k]);
    d = fmax(d, c.red[2 * NW + k]);
  }
  __syncthreads();
}

// Number of constraint rows owned by this CTA (stage rows, plus terminal rows
// for the last chunk).  Owned row `lr` has global index s*nc + lr.
template <typename T>
__device__ inline int own_rows(Ctx<T>& c) {
  return c.active ? c.L * c.d->nc + (c.last ? c.d->nf : 0) : 0;
}

// ---------------------------------------------------------------------------
// Bulk-copy ring over the union region.  Blocks go round the `depth` slots in
// order; the k-th use of a slot completes phase k of its mbarrier, so a
// consumer waits on parity k & 1.  One thread issues the copies; every thread
// waits on the slot's mbarrier itself (no barrier between arrival and use).
// The ring position (slot, parity) is carried across streams in Ctx, so no
// division is needed per block.
// ---------------------------------------------------------------------------
template <typename T>
struct Blk {
  const T* ptr;
  int bytes;
};

__device__ inline void ring_advance(unsigned& slot, unsigned& par, unsigned depth) {
  if (++slot == depth) {
    slot = 0;
    par ^= 1u;
  }
}

// Stream nblk blocks (src(b) -> Blk) through the ring, depth-1 blocks ahead of
// the compute f(b, slot).  Every block must fit a slot; addresses 16-byte
// aligned, sizes multiples of 16 bytes.  A wait that gives up sets
// flag[RING_FLAG]; from then on the CTA issues and waits for nothing more (the
// iteration runs to its end on stale data and the solve reports
// GPUSLS_ERR_TIMEOUT).
template <typename T, typename Src, typename Fn>
__device__ __forceinline__ void stream_blocks(Ctx<T>& c, int nblk, Src src, Fn f) {
  const unsigned depth = (unsigned)c.d->depth;
  const size_t slot_el = (size_t)c.d->slot;
  T* const ring = c.ring;
  unsigned long long* const bar = c.bar;
  int* const flag = c.flag;
  unsigned long long* const prof = threadIdx.x == 0 ? c.prof : nullptr;
  const bool issuer = threadIdx.x == 0;
  fence_proxy_async();     // earlier generic accesses of the ring region come first
  __syncthreads();
  bool dead = flag[RING_FLAG] != 0;
  unsigned ws = c.ws, wp = c.wp;          // next slot to consume, its parity
  unsigned is = ws, ip = wp;              // next slot to fill (issuer)
  unsigned inflight = c.inflight, ipar = c.ipar;
  auto issue = [&](int b) {
    const Blk<T> k = src(b);
    bulk_g2s(ring + is * slot_el, k.ptr, (unsigned)k.bytes, &bar[is]);
    inflight |= 1u << is;
    ipar = (ipar & ~(1u << is)) | (ip << is);
    ring_advance(is, ip, depth);
  };
  if (issuer && !dead)
    for (int b = 0; b < nblk && b < (int)depth - 1; ++b) issue(b);
  for (int b = 0; b < nblk; ++b) {
    if (!dead) {
      if (issuer && b + (int)depth - 1 < nblk) issue(b + (int)depth - 1);
      const long long tw = prof ? clock64() : 0;
      if (mbar_wait(&bar[ws], wp, RING_WAIT_LIMIT)) inflight &= ~(1u << ws);
      else flag[RING_FLAG] = 1;
      if (prof) prof[PH_RINGWAIT] += (unsigned long long)(clock64() - tw);
    }
    f(b, (const T*)(ring + ws * slot_el));
    __syncthreads();
    dead = flag[RING_FLAG] != 0;
    ring_advance(ws, wp, depth);
  }
  if (issuer) {   // every thread holds the same ws, wp; inflight, ipar are the issuer's
    c.ws = ws;
    c.wp = wp;
    c.inflight = inflight;
    c.ipar = ipar;
  }
}

// Before the CTA exits: if a ring wait gave up, the issuing thread waits
// (bounded) for every copy it started that was not seen to complete, so that
// none lands after the CTA's shared memory is gone.
template <typename T>
__device__ void ring_drain(Ctx<T>& c) {
  if (threadIdx.x != 0 || c.flag[RING_FLAG] == 0) return;
  for (unsigned sl = 0; sl < (unsigned)c.d->depth; ++sl)
    if ((c.inflight >> sl) & 1u) mbar_wait(&c.bar[sl], (c.ipar >> sl) & 1u, RING_WAIT_LIMIT);
  if (c.bulk_inflight) mbar_wait(&c.bar[BULK_BAR], c.bpar, RING_WAIT_LIMIT);
}

// ---------------------------------------------------------------------------
// Whole-region copies.  The chunk-boundary corrections stream runs of
// contiguous blocks with little arithmetic per block, which the ring serves one
// slot at a time; here as many blocks as the ring region holds come in one
// bulk copy on a barrier of their own, so a run costs one copy latency (the
// first one issued before the cluster barrier that precedes its use).  The
// ring must be idle: no ring copy in flight.  Both calls are made by every
// thread of the CTA and contain a CTA barrier.
// ---------------------------------------------------------------------------
template <typename T>
__device__ inline int bulk_capacity(const Ctx<T>& c) {   // elements
  return c.d->depth * c.d->slot;
}

// Orders every thread's earlier accesses of the ring region before the copy of
// n_el elements from src (16-byte aligned, n_el * sizeof(T) a multiple of 16,
// n_el <= bulk_capacity) into it; thread 0 issues the copy.
template <typename T>
__device__ void bulk_issue(Ctx<T>& c, const T* src, int n_el) {
  fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0 && c.flag[RING_FLAG] == 0) {
    bulk_g2s(c.ring, src, (unsigned)(n_el * (int)sizeof(T)), &c.bar[BULK_BAR]);
    c.bulk_inflight = 1;
  }
}

// Waits (bounded) for the copy of the last bulk_issue.  A wait that gives up
// sets flag[RING_FLAG], as in the ring.  Returns after a CTA barrier.
template <typename T>
__device__ void bulk_wait(Ctx<T>& c) {
  const bool issued = c.flag[RING_FLAG] == 0;   // the flag is only set by waits, none since the issue
  bool ok = true;
  if (issued) {
    const long long tw = (threadIdx.x == 0 && c.prof) ? clock64() : 0;
    ok = mbar_wait(&c.bar[BULK_BAR], c.bpar, RING_WAIT_LIMIT);
    if (!ok) c.flag[RING_FLAG] = 1;
    if (threadIdx.x == 0 && c.prof) c.prof[PH_RINGWAIT] += (unsigned long long)(clock64() - tw);
  }
  __syncthreads();
  if (threadIdx.x == 0 && issued && ok) {
    c.bpar ^= 1u;
    c.bulk_inflight = 0;
  }
}

struct Partials {
  double rp, rd, vm, zm;
};

// The iteration's per-launch constants, computed once by thread 0 (the
// divisions would otherwise run in every iteration): bundle sizes, and the
// whole-region rounds of the chunk-boundary corrections.  A ring slot holds a
// Theta or Xi block, so cap_bk >= 1; a batched fix-up sweep takes at most
// NT / nu (NT / nc) stages.
template <typename T>
__device__ void iter_plan(Ctx<T>& c) {
  const QPDesc& d = *c.d;
  const int nx = d.nx, nu = d.nu, nc = d.nc, L = c.L;
  bundle_sizes(nx, nu, nc, d.ldx, d.ldu, d.ldv, d.ldf, &c.bws, &c.fws, &c.cds);
  const int cap_el = d.depth * d.slot;
  c.cap_bk = cap_el / c.msz;
  c.nb_th = max(0, d.nch - (c.rank + 2));
  c.nr_th = (c.nb_th + c.cap_bk - 1) / c.cap_bk;
  c.gs_fp = min(min(cap_el / (nx * d.ldu), NT / nu), max(L, 1));
  c.nr_fp = (L + c.gs_fp - 1) / c.gs_fp;
  c.nb_xi = max(0, c.rank - 1);
  c.nr_xi = (c.nb_xi + c.cap_bk - 1) / c.cap_bk;
  c.gs_ck = nc > 0 ? min(min(cap_el / (nx * d.ldc), NT / nc), max(L, 1)) : 1;
  c.nr_ck = nc > 0 ? (L + c.gs_ck - 1) / c.gs_ck : 0;
}

// One ADMM iteration (eq. augmented_linear, the LQ solve of eq. primal_update
// with the cached factorization, the z-projection and the scaled dual update).
//
// Backward chain, stage i = e-1 .. s, on the stacked vector [l_{i+1}; omega_i]:
//   l_i  = [Abar_i; CK_i]^T [l_{i+1}; omega_i] + c0_i   (p_i up to the fix-up)
//   k~_i = [F_i  J_i] [l_{i+1}; omega_i] + k0_i
// Forward chain, stage i = s .. e-1, on [lx_i; k_i]:
//   [lx_{i+1}; v~_i] = [Abar_i B_i; CK_i D_i] [lx_i; k_i] + [b_i; 0]
// with k_i = k~_i + FPi_i p_e and v_i = v~_i + CKSig_i x_s after the
// chunk-boundary exchanges.  On `check` iterations the dual-residual partial
// is formed too.
template <typename T>
__device__ void admm_iteration(Ctx<T>& c, cg::cluster_group& cl, T rho, bool check, Partials& pl) {
  QPDesc& d = *c.d;
  const int nx = d.nx, nu = d.nu, nc = d.nc, nf = d.nf, N = d.N, ldx = d.ldx, ldu = d.ldu;
  const int ldv = d.ldv, ldf = d.ldf, msz = c.msz, L = c.L, s = c.s;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const T *q = TP<T>(d.q), *CN = TP<T>(d.CN), *lo = TP<T>(d.lo), *hi = TP<T>(d.hi);
  const T *FPi = TP<T>(d.FPi), *CKSig = TP<T>(d.CKSig), *CNSig = TP<T>(d.CNSig);
  const T *Theta = TP<T>(d.Theta), *Xi = TP<T>(d.Xi);
  const T *BW = TP<T>(d.BW), *FW = TP<T>(d.FW), *CD = TP<T>(d.CD);
  const int bws = c.bws, fws = c.fws;
  const int nrows = own_rows(c);
  // The chunk-boundary corrections in whole-region rounds (bulk_issue), as
  // planned by iter_plan:
  // P3: nr_th rounds of Theta blocks (cap_bk per round), then nr_fp rounds of
  //     FPi stages (gs_fp per round);
  // P5: nr_xi rounds of Xi blocks, then nr_ck rounds of CKSig stages.
  const int cap_bk = c.cap_bk, m0 = c.rank + 2, nb_th = c.nb_th, nr_th = c.nr_th;
  const int per_fp = nx * ldu, gs_fp = c.gs_fp, nr_fp = c.nr_fp;
  const int nb_xi = c.nb_xi, nr_xi = c.nr_xi;
  const int ldc = d.ldc, per_ck = nx * ldc, gs_ck = c.gs_ck, nr_ck = c.nr_ck;
  T lo_a = T(0), hi_a = T(0), lo_b = T(0), hi_b = T(0);   // bounds of the first two own rows (P5)
  auto p3_src = [&](int r) -> const T* {
    return r < nr_th ? Theta + (size_t)(c.rank * d.nch + m0 + r * cap_bk) * msz
                     : FPi + (size_t)(s + (r - nr_th) * gs_fp) * per_fp;
  };
  auto p3_len = [&](int r) -> int {
    return r < nr_th ? min(cap_bk, nb_th - r * cap_bk) * msz : min(gs_fp, L - (r - nr_th) * gs_fp) * per_fp;
  };
  auto p5_src = [&](int r) -> const T* {
    return r < nr_xi ? Xi + (size_t)(c.rank * d.nch + r * cap_bk) * msz
                     : CKSig + (size_t)(s + (r - nr_xi) * gs_ck) * per_ck;
  };
  auto p5_len = [&](int r) -> int {
    return r < nr_xi ? min(cap_bk, nb_xi - r * cap_bk) * msz : min(gs_ck, L - (r - nr_xi) * gs_ck) * per_ck;
  };

  // P1: omega = rho (y - z) into the stacked rows; boundary of the backward
  // chain (p_N = q^_N = q_N + C_N^T omega_N for the last chunk, 0 otherwise).
  if (c.active) {
    // omega straight into the stacked rows (wS keeps the last dz for the dual
    // residual); the terminal omega_N is formed where it is used
    for (int e2 = t; e2 < L * nc; e2 += NT) {
      const int li = e2 / nc, rr = e2 - li * nc;
      c.lS[(size_t)(li + 1) * ldv + nx + rr] = rho * (c.yS[e2] - c.zS[e2]);
    }
    for (int j = t; j < nx; j += NT) {
      T a = T(0);
      if (c.last) {
        a = q[(size_t)N * ldx + j];
        for (int rr = 0; rr < nf; ++rr)
          a += CN[rr * ldx + j] * (rho * (c.yS[L * nc + rr] - c.zS[L * nc + rr]));
      }
      c.lS[(size_t)L * ldv + j] = a;
    }
    __syncthreads();
    prof_mark(c, PH_P1);
    // P2: backward chain over the BW bundles: one split sweep of
    // [Abar; CK | (F | J)^T] per stage gives l_i (t < nx) and k~_i.
    const int R = nx + nc;
    {
      const SweepPlan sp = sweep_plan<T>(R, nx, ldx, nu, ldu, R * ldx);
      T* const lS = c.lS;
      T* const ktS = c.ktS;
      T* const swp = c.swp;
      const int c0o = t < nx ? R * ldx + R * ldu + t : R * ldx + R * ldu + ldx + (t - nx);
      stream_blocks<T>(
          c, L, [&](int st) { return Blk<T>{BW + (size_t)(c.e - 1 - st) * bws, bws * (int)sizeof(T)}; },
          [&](int st, const T* S) {
            const int li = L - 1 - st;
            const T y = sweep_run<T>(sp, S, lS + (size_t)(li + 1) * ldv, swp);
            if (t < nx) lS[(size_t)li * ldv + t] = S[c0o] + y;
            else if (t < nx + nu) ktS[li * ldu + t - nx] = S[c0o] + y;
          });
    }
    for (int j = t; j < nx; j += NT) c.slotL[j] = c.lS[j];
    // the ring is idle: start the first copy of P3 before the cluster barrier
    if (!c.last) bulk_issue<T>(c, p3_src(0), p3_len(0));
    prof_mark(c, PH_BWD);
  }
  cl.sync();
  prof_mark(c, PH_SYNC1);
  // P3: boundary p_e from the later chunks, then k_i = k~_i + FPi_i p_e.
  if (c.active) {
    if (!c.last) {
      // the later chunks' local results l_m (m = rank+1 .. nch-1), gathered
      // in one round of distributed shared memory reads
      const int nlat = d.nch - 1 - c.rank;
      T* const gath = c.gath;
      for (int e2 = t; e2 < nlat * nx; e2 += NT) {
        const int m = e2 / nx;
        gath[e2] = cl.map_shared_rank(c.slotL, c.rank + 1 + m)[e2 - m * nx];
      }
      // p_e = l_{rank+1} + sum_m Theta_{rank,m} l_m over m = rank+2 ..: the
      // Theta blocks of a row are contiguous, so a round of k of them is one
      // tall (k nx) x nx block swept against the stacked l_m
      constexpr int VW = Vec16<T>::W;
      T acc[VW];
#pragma unroll
      for (int e = 0; e < VW; ++e) acc[e] = T(0);
      for (int r = 0; r < nr_th; ++r) {
        if (r > 0) bulk_issue<T>(c, p3_src(r), p3_len(r));
        bulk_wait<T>(c);   // also orders the gather before the sweep
        const int b0 = r * cap_bk, k = min(cap_bk, nb_th - b0);
        const SweepPlan sp = sweep_plan<T>(k * nx, nx, ldx, 0, ldx, 0);
        sweep_partial<T>(sp, c.ring, gath + (size_t)(b0 + 1) * nx, acc);
      }
      // the first FPi round's copy overlaps the reduction (it was the
      // prefetched round when there are no Theta rounds)
      if (nr_th > 0) bulk_issue<T>(c, p3_src(nr_th), p3_len(nr_th));
      {
        const SweepPlan sp = sweep_plan<T>(nx, nx, ldx, 0, ldx, 0);
        const T y = sweep_reduce<T>(sp, acc, c.swp);
        if (t < nx) c.pe[t] = gath[t] + y;
      }
      // k_i = k~_i + FPi_i p_e for own stages, gs_fp stages per round
      const int per = nx * ldu;   // FPi_i^T
      T* const xS = c.xS;
      const T* const ktS = c.ktS;
      const int ls_t = t / nu, a_t = t - ls_t * nu;
      for (int r = 0; r < nr_fp; ++r) {
        if (r > 0) bulk_issue<T>(c, p3_src(nr_th + r), p3_len(nr_th + r));
        bulk_wait<T>(c);   // also orders p_e before the sweep
        const int n_st = min(gs_fp, L - r * gs_fp);
        const SweepPlan fp = sweep_plan_batched<T>(nx, nu, ldu, n_st, per);
        const T y = sweep_run<T>(fp, c.ring, c.pe, c.swp);
        const int li = r * gs_fp + ls_t;
        if (t < n_st * nu) xS[(size_t)li * ldf + nx + a_t] = ktS[li * ldu + a_t] + y;
      }
    } else {
      for (int e2 = t; e2 < L * nu; e2 += NT) {
        const int li = e2 / nu, a = e2 - li * nu;
        c.xS[(size_t)li * ldf + nx + a] = c.ktS[li * ldu + a];
      }
    }
    __syncthreads();   // (xS row 0 = x0 or 0 is set once per launch)
    prof_mark(c, PH_P3);
    // P4: forward chain over the FW^T bundles: thread r < nx + nc sweeps
    // column r of FW^T for lx_{i+1} (r < nx) or v~_i (r >= nx).
    const int R = nx + nc, Cn = nx + nu;
    {
      const SweepPlan sp = sweep_plan<T>(Cn, R, ldv, 0, ldv, 0);
      T* const xS = c.xS;
      T* const vS = c.vS;
      T* const swp = c.swp;
      const int bo = Cn * ldv + t;
      stream_blocks<T>(
          c, L, [&](int st) { return Blk<T>{FW + (size_t)(s + st) * fws, fws * (int)sizeof(T)}; },
          [&](int st, const T* S) {
            const T y = sweep_run<T>(sp, S, xS + (size_t)st * ldf, swp);
            if (t < nx) xS[(size_t)(st + 1) * ldf + t] = y + S[bo];
            else if (t < R) vS[st * nc + t - nx] = y;
          });
    }
    for (int j = t; j < nx; j += NT) c.slotX[j] = c.xS[(size_t)L * ldf + j];
    // the ring is idle: start the first copy of P5 before the cluster barrier
    if (!c.first && nr_xi + nr_ck > 0) bulk_issue<T>(c, p5_src(0), p5_len(0));
    // the bounds of this thread's first two rows, loaded ahead of the projection
    if (t < nrows) {
      lo_a = lo[s * nc + t];
      hi_a = hi[s * nc + t];
    }
    if (t + NT < nrows) {
      lo_b = lo[s * nc + t + NT];
      hi_b = hi[s * nc + t + NT];
    }
    prof_mark(c, PH_FWD);
  }
  cl.sync();
  prof_mark(c, PH_SYNC2);
  // P5: boundary x_s from the earlier chunks, v_i = v~_i + CKSig_i x_s,
  // projection and scaled dual update.
  if (c.active) {
    if (!c.first) {
      // the earlier chunks' end states lx_m (m = 0 .. rank-1), gathered in one
      // round of distributed shared memory reads: gath row m = chunk m
      T* const gath = c.gath;
      for (int e2 = t; e2 < c.rank * nx; e2 += NT) {
        const int m = e2 / nx;
        gath[e2] = cl.map_shared_rank(c.slotX, m)[e2 - m * nx];
      }
      // x_s = lx_{rank-1} + sum_m Xi_{rank,m} lx_m over m = 0 .. rank-2, in
      // tall rounds of contiguous Xi blocks as in P3
      constexpr int VW = Vec16<T>::W;
      T acc[VW];
#pragma unroll
      for (int e = 0; e < VW; ++e) acc[e] = T(0);
      for (int r = 0; r < nr_xi; ++r) {
        if (r > 0) bulk_issue<T>(c, p5_src(r), p5_len(r));
        bulk_wait<T>(c);   // also orders the gather before the sweep
        const int b0 = r * cap_bk, k = min(cap_bk, nb_xi - b0);
        const SweepPlan sp = sweep_plan<T>(k * nx, nx, ldx, 0, ldx, 0);
        sweep_partial<T>(sp, c.ring, gath + (size_t)b0 * nx, acc);
      }
      if (nr_xi > 0 && nr_ck > 0) bulk_issue<T>(c, p5_src(nr_xi), p5_len(nr_xi));
      {
        const SweepPlan sp = sweep_plan<T>(nx, nx, ldx, 0, ldx, 0);
        const T y = sweep_reduce<T>(sp, acc, c.swp);
        if (t < nx) c.xs[t] = gath[(size_t)(c.rank - 1) * nx + t] + y;
      }
      // v_i += CKSig_i x_s for own stages, gs_ck stages per round
      T* const vS = c.vS;
      const int ls_t = nc > 0 ? t / nc : 0, r_t = t - ls_t * nc;
      for (int r = 0; r < nr_ck; ++r) {
        if (r > 0) bulk_issue<T>(c, p5_src(nr_xi + r), p5_len(nr_xi + r));
        bulk_wait<T>(c);   // also orders x_s before the sweep
        const int n_st = min(gs_ck, L - r * gs_ck);
        const SweepPlan cp = sweep_plan_batched<T>(nx, nc, ldc, n_st, per_ck);
        const T y = sweep_run<T>(cp, c.ring, c.xs, c.swp);
        const int li = r * gs_ck + ls_t;
        if (t < n_st * nc) vS[li * nc + r_t] += y;
      }
      if (nr_ck == 0) __syncthreads();   // x_s before the terminal rows
    }
    if (c.last) {
      // terminal rows, one warp each
      const T* xN = c.xS + (size_t)L * ldf;
      for (int rr = w; rr < nf; rr += NT / 32) {
        const T* Cr = CN + rr * ldx;
        const T* Sr = CNSig + rr * ldx;
        T a = T(0);
        for (int k = lane; k < nx; k += 32) {
          a = fma(Cr[k], xN[k], a);
          if (!c.first) a = fma(Sr[k], c.xs[k], a);
        }
        a = warp_sum(a);
        if (lane == 0) c.vS[L * nc + rr] = a;
      }
    }
    __syncthreads();
    T rp = T(0), vm = T(0), zm = T(0);
    for (int lr = t, k2 = 0; lr < nrows; lr += NT, ++k2) {
      const int gi = s * nc + lr;
      const T v = c.vS[lr];
      const T zo = c.zS[lr], yo = c.yS[lr];
      const T lo_r = k2 == 0 ? lo_a : (k2 == 1 ? lo_b : lo[gi]);
      const T hi_r = k2 == 0 ? hi_a : (k2 == 1 ? hi_b : hi[gi]);
      const T zn = fmin(fmax(v + yo, lo_r), hi_r);
      c.yS[lr] = yo + v - zn;
      c.zS[lr] = zn;
      c.wS[lr] = zn - zo;
      // a NaN or Inf in v (fmax would drop a NaN) makes r_prim infinite:
      // the check reports GPUSLS_ERR_NAN
      rp = isfinite(v) ? fmax(rp, fabs(v - zn)) : T(INFINITY);
      vm = fmax(vm, fabs(v));
      zm = fmax(zm, fabs(zn));
    }
    __syncthreads();
    prof_mark(c, PH_P5);
    if (check) {
      block_max3(c, rp, vm, zm);
      pl.rp = (double)rp;
      pl.vm = (double)vm;
      pl.zm = (double)zm;
      pl.rd = 0.0;   // formed by dual_residual_partial when the solve loop needs it
    }
  } else {
    pl.rp = pl.rd = pl.vm = pl.zm = 0.0;
  }
}

// Dual-residual partial of own rows, rho * ||G^T (z+ - z)||_inf = rho * max
// |[C D]^T dz| over own stages (dz = wS, left by the projection of the last
// iteration), block-level max.  Only the solve loop's checks that need it
// call it (the primal test passed, a rho update, the last iteration).
template <typename T>
__device__ double dual_residual_partial(Ctx<T>& c, T rho) {
  QPDesc& d = *c.d;
  const int nx = d.nx, nu = d.nu, nc = d.nc, nf = d.nf, ldx = d.ldx, ldu = d.ldu, ldv = d.ldv, ldf = d.ldf;
  const int L = c.L, s = c.s, t = threadIdx.x;
  const T *CD = TP<T>(d.CD), *CN = TP<T>(d.CN);
  int bws, fws, cds;
  bundle_sizes(nx, nu, nc, ldx, ldu, ldv, ldf, &bws, &fws, &cds);
  T rd = T(0);
  if (c.active) {
    const int Cn = nx + nu;
    if (cds > 0) {
      // the [C D] blocks of own stages are contiguous: whole-region rounds
      // (the ring is idle between iterations)
      const int cap = max(1, bulk_capacity(c) / cds);
      for (int st0 = 0; st0 < L; st0 += cap) {
        const int n_st = min(cap, L - st0);
        bulk_issue<T>(c, CD + (size_t)(s + st0) * cds, n_st * cds);
        bulk_wait<T>(c);
        for (int e2 = t; e2 < n_st * Cn; e2 += NT) {
          const int ls = e2 / Cn, col = e2 - ls * Cn, li = st0 + ls;
          const T* Sb = c.ring + (size_t)ls * cds;
          T a = T(0);
          for (int rr = 0; rr < nc; ++rr) a += Sb[rr * ldf + col] * c.wS[li * nc + rr];
          rd = fmax(rd, fabs(a));
        }
      }
    }
    if (c.last) {
      for (int j = t; j < nx; j += NT) {
        T a = T(0);
        for (int rr = 0; rr < nf; ++rr) a += CN[rr * ldx + j] * c.wS[L * nc + rr];
        rd = fmax(rd, fabs(a));
      }
    }
  }
  return (double)rho * (double)block_max(c, rd);
}

// Full state and input of own stages: x_i = lx_i + Sig_i x_s (into dS rows
// 0..L, row L = x_N for the last chunk), u_i = K_i lx_i + KSig_i x_s + k_i.
template <typename T>
__device__ void full_xu(Ctx<T>& c) {
  QPDesc& d = *c.d;
  const int nx = d.nx, nu = d.nu, ldx = d.ldx, ldu = d.ldu, ldf = d.ldf, msz = c.msz, L = c.L, s = c.s;
  const T *K = TP<T>(d.K), *KSig = TP<T>(d.KSig), *Sig = TP<T>(d.Sig), *SigN = TP<T>(d.SigN);
  if (!c.active) return;
  const int t = threadIdx.x;
  if (c.first) {
    const int nxr = (L + (c.last ? 1 : 0)) * nx;
    for (int pr = t; pr < nxr; pr += NT) {
      const int li = pr / nx, j = pr - li * nx;
      c.dS[(size_t)li * ldx + j] = c.xS[(size_t)li * ldf + j];
    }
  } else {
    // Sig_i of own stages are contiguous: whole-region rounds of cap stages
    // (the ring is idle between iterations), one thread per output row dot
    // product from shared memory.  Lane l starts its row at column l mod nx
    // and wraps, so a warp's reads of 32 rows fall in 32 different banks.
    const int cap = bulk_capacity(c) / msz;
    const int k0 = (t & 31) % nx;
    const T* const xs = c.xs;
    for (int st0 = 0; st0 < L; st0 += cap) {
      const int n_st = min(cap, L - st0);
      bulk_issue<T>(c, Sig + (size_t)(s + st0) * msz, n_st * msz);
      bulk_wait<T>(c);
      for (int pr = t; pr < n_st * nx; pr += NT) {
        const int lr = pr / nx, j = pr - lr * nx, li = st0 + lr;
        const T* Sr = c.ring + (size_t)lr * msz + j * ldx;
        T a0 = T(0), a1 = T(0);
        int k = k0;
        int it = 0;
        for (; it + 1 < nx; it += 2) {
          a0 = fma(Sr[k], xs[k], a0);
          k = (k + 1 == nx) ? 0 : k + 1;
          a1 = fma(Sr[k], xs[k], a1);
          k = (k + 1 == nx) ? 0 : k + 1;
        }
        if (it < nx) a0 = fma(Sr[k], xs[k], a0);
        c.dS[(size_t)li * ldx + j] = c.xS[(size_t)li * ldf + j] + a0 + a1;
      }
    }
    if (c.last) {   // x_N = lx_N + Sig_N x_s, from global memory
      for (int j = t; j < nx; j += NT) {
        const T* Sr = SigN + j * ldx;
        T a0 = T(0), a1 = T(0);
        int k = 0;
        for (; k + 1 < nx; k += 2) {
          a0 = fma(Sr[k], xs[k], a0);
          a1 = fma(Sr[k + 1], xs[k + 1], a1);
        }
        if (k < nx) a0 = fma(Sr[k], xs[k], a0);
        c.dS[(size_t)L * ldx + j] = c.xS[(size_t)L * ldf + j] + a0 + a1;
      }
    }
  }
  for (int pr = t; pr < L * nu; pr += NT) {
    const int li = pr / nu, a = pr - li * nu, i = s + li;
    const T* Kr = K + (size_t)i * nu * ldx + a * ldx;
    const T* KSr = KSig + (size_t)i * nu * ldx + a * ldx;
    const T* lx = c.xS + (size_t)li * ldf;
    T a0 = T(0), a1 = T(0);
    for (int k = 0; k < nx; ++k) {
      a0 = fma(Kr[k], lx[k], a0);
      if (!c.first) a1 = fma(KSr[k], c.xs[k], a1);
    }
    c.uS[li * ldu + a] = a0 + a1 + c.xS[(size_t)li * ldf + nx + a];
  }
  __syncthreads();
}

// Partials of the rho rule: ||H xi||_inf, ||G^T lambda||_inf, ||(q, r)||_inf
// over own stages (needs full_xu first).
template <typename T>
__device__ void rho_rule_partials(Ctx<T>& c, T rho, double& hm, double& gm, double& qm) {
  QPDesc& d = *c.d;
  const int nx = d.nx, nu = d.nu, nc = d.nc, N = d.N, ldx = d.ldx, ldu = d.ldu, msz = c.msz, L = c.L, s = c.s;
  const T *Q = TP<T>(d.Q), *R = TP<T>(d.R), *S = TP<T>(d.S), *C = TP<T>(d.C), *D = TP<T>(d.D), *CN = TP<T>(d.CN);
  const T *q = TP<T>(d.q), *r = TP<T>(d.r);
  const int t = threadIdx.x;
  T h = T(0), g = T(0), qq = T(0);
  if (c.active) {
    // Q_i x_i from whole-region rounds of the Q_i of own stages (contiguous;
    // the ring is idle between iterations), one thread per row dot product,
    // lane l starting at column l mod nx so that a warp's 32 rows fall in 32
    // banks; S_i^T u_i and C_i^T y_i by columns from global memory (the
    // threads of a warp, consecutive j, read consecutive addresses)
    const int capq = max(1, bulk_capacity(c) / msz);
    const int k0 = (t & 31) % nx;
    for (int st0 = 0; st0 < L; st0 += capq) {
      const int n_st = min(capq, L - st0);
      bulk_issue<T>(c, Q + (size_t)(s + st0) * msz, n_st * msz);
      bulk_wait<T>(c);
      for (int e2 = t; e2 < n_st * nx; e2 += NT) {
        const int lr = e2 / nx, j = e2 - lr * nx, li = st0 + lr, i = s + li;
        const T* Qr = c.ring + (size_t)lr * msz + j * ldx;
        const T* xi = c.dS + li * ldx;
        T a = T(0), a1 = T(0);
        int k = k0;
        int it = 0;
        for (; it + 1 < nx; it += 2) {
          a = fma(Qr[k], xi[k], a);
          k = (k + 1 == nx) ? 0 : k + 1;
          a1 = fma(Qr[k], xi[k], a1);
          k = (k + 1 == nx) ? 0 : k + 1;
        }
        if (it < nx) a = fma(Qr[k], xi[k], a);
        const T* Si = S + (size_t)i * nu * ldx;
        for (int k2 = 0; k2 < nu; ++k2) a1 = fma(Si[k2 * ldx + j], c.uS[li * ldu + k2], a1);
        a += a1;
        h = fmax(h, fabs(a));
        const T* Ci = C + (size_t)i * nc * ldx;
        T b2 = T(0);
        for (int rr = 0; rr < nc; ++rr) b2 += Ci[rr * ldx + j] * c.yS[li * nc + rr];
        g = fmax(g, fabs(rho * b2));
        qq = fmax(qq, fabs(q[(size_t)i * ldx + j]));
      }
    }
    for (int e2 = t; e2 < L * nu; e2 += NT) {
      const int li = e2 / nu, a2 = e2 - li * nu, i = s + li;
      const T* Ri = R + (size_t)i * nu * ldu + a2;   // column a2 = row a2 (R_i symmetric)
      T a = T(0), a1 = T(0);
      for (int k = 0; k < nu; ++k) a = fma(Ri[k * ldu], c.uS[li * ldu + k], a);
      const T* Si = S + (size_t)i * nu * ldx + a2 * ldx;
      const T* xi = c.dS + li * ldx;
      int k = 0;
      for (; k + 1 < nx; k += 2) {
        a = fma(Si[k], xi[k], a);
        a1 = fma(Si[k + 1], xi[k + 1], a1);
      }
      if (k < nx) a = fma(Si[k], xi[k], a);
      a += a1;
      h = fmax(h, fabs(a));
      const T* Di = D + (size_t)i * nc * ldu;
      T b2 = T(0);
      for (int rr = 0; rr < nc; ++rr) b2 += Di[rr * ldu + a2] * c.yS[li * nc + rr];
      g = fmax(g, fabs(rho * b2));
      qq = fmax(qq, fabs(r[(size_t)i * ldu + a2]));
    }
    if (c.last) {
      for (int j = t; j < nx; j += NT) {
        const T* Qi = Q + (size_t)N * msz + j;   // column j = row j (symmetric)
        T a = T(0);
        for (int k = 0; k < nx; ++k) a = fma(Qi[(size_t)k * ldx], c.dS[L * ldx + k], a);
        h = fmax(h, fabs(a));
        T b2 = T(0);
        for (int rr = 0; rr < d.nf; ++rr) b2 += CN[rr * ldx + j] * c.yS[L * nc + rr];
        g = fmax(g, fabs(rho * b2));
        qq = fmax(qq, fabs(q[(size_t)N * ldx + j]));
      }
    }
  }
  block_max3(c, h, g, qq);
  hm = (double)h;
  gm = (double)g;
  qm = (double)qq;
}

// Cluster-wide max (NaN-propagating) of N <= 7 doubles per CTA.  Thread 0
// publishes them in one of two slots of part[] that alternate between calls,
// every remote value is read by its own thread, and the values are combined
// from shared memory.  One cluster barrier per call: a CTA writes a slot again
// only two calls later, after every CTA has passed the barrier of the call in
// between (so after its reads of that slot).  part[15] belongs to cluster_or.
template <typename T, int N>
__device__ void cluster_max(Ctx<T>& c, cg::cluster_group& cl, double (&v)[N]) {
  static_assert(N <= 7, "cluster_max: at most 7 values");
  const int t = threadIdx.x;
  const int par = c.cm_par;
  double* const slot = c.part + 8 * par;
  if (t == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) slot[k] = v[k];
  }
  cl.sync();
  double* const gath = c.part + 16;   // [cs * N]
  if (t < c.cs * N) {
    const int rk = t / N;
    gath[t] = cl.map_shared_rank(slot, rk)[t - rk * N];
  }
  if (t == 0) c.cm_par = par ^ 1;   // every thread read par before the cluster barrier
  __syncthreads();
#pragma unroll
  for (int k = 0; k < N; ++k) {
    double r = 0.0;
    for (int rk = 0; rk < c.cs; ++rk) {
      const double a = gath[rk * N + k];
      r = (a != a || r != r) ? a + r : fmax(r, a);
    }
    v[k] = r;
  }
}

// Write full x, u and lambda = rho y of own stages to the FP64 outputs.
template <typename T>
__device__ void write_outputs(Ctx<T>& c, T rho) {
  QPDesc& d = *c.d;
  if (!c.active) return;
  const int nx = d.nx, nu = d.nu, nc = d.nc, ldx = d.ldx, ldu = d.ldu, L = c.L, s = c.s;
  const int t = threadIdx.x;
  const int nxr = (L + (c.last ? 1 : 0)) * nx;
  for (int e2 = t; e2 < nxr; e2 += NT) {
    const int li = e2 / nx, j = e2 - li * nx;
    d.ox[(size_t)(s + li) * nx + j] = (double)c.dS[li * ldx + j];
  }
  for (int e2 = t; e2 < L * nu; e2 += NT) {
    const int li = e2 / nu, a = e2 - li * nu;
    d.ou[(size_t)(s + li) * nu + a] = (double)c.uS[li * ldu + a];
  }
  const int nrows = own_rows(c);
  for (int e2 = t; e2 < nrows; e2 += NT) d.olam[(size_t)s * nc + e2] = (double)rho * (double)c.yS[e2];
  __syncthreads();
}

// FP64 KKT residual of the outputs written by write_outputs (the definition
// is the library's, see include/gpusls.h): dynamics, bound violation,
// u-stationarity after costate recovery and complementarity, max over the
// cluster.  Every CTA evaluates the stage-local parts of its chunk, with the
// stage's Q_i, A_i and C_i copied into shared memory (coalesced, by
// cp.async) when the union region holds them; CTA 0 then runs the costate
// recursion mu_k = g_k + A_k^T mu_{k+1} sequentially.
template <typename T>
__device__ __noinline__ double kkt_eval(Ctx<T>& c, cg::cluster_group& cl) {
  QPDesc& d = *c.d;
  const int nx = d.nx, nu = d.nu, nc = d.nc, nf = d.nf, N = d.N;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  double* xv = reinterpret_cast<double*>(c.ring);   // FP64 scratch in the union region
  double* xn = xv + 96;
  double* uv = xn + 96;
  double* lv = uv + 96;
  double* qx = lv + 96;   // Q x
  double* ax = qx + 96;   // A x
  double* bu = ax + 96;   // B u
  double* sx = bu + 96;   // S x
  double* ru = sx + 96;   // R u
  double* cx = ru + 96;   // C x
  double* du = cx + 96;   // D u
  double* gt = du + 96;   // C^T lam + S^T u
  double* ht = gt + 96;   // D^T lam
  // Q_i, A_i, C_i of the stage in shared memory after the vectors
  double* Qs = ht + 96;
  double* As = Qs + nx * nx;
  double* Cs = As + nx * nx;
  const bool stg = (13 * 96 + 2 * nx * nx + (nc > nf ? nc : nf) * nx) * 8 <= c.uni;
  double dyn = 0.0, viol = 0.0, comp = 0.0, stat = 0.0;
  long long kt0 = c.prof ? clock64() : 0;
  cl.sync();   // outputs of every chunk visible
  if (c.active) {
    const int iend = c.e + (c.last ? 1 : 0);
    for (int i = c.s; i < iend; ++i) {
      const bool term = (i == N);
      const int nr = term ? nf : nc;
      const double* Qg = d.Q64 + (size_t)i * nx * nx;
      const double* Cg = term ? d.CN64 : d.C64 + (size_t)i * nc * nx;
      const double* Ag = d.A64 + (size_t)i * nx * nx;
      if (stg) {   // the caller's rows are unpadded: 8-byte copies
        for (int e2 = t; e2 < nx * nx; e2 += NT) cp_async_elem<double>(Qs + e2, Qg + e2);
        if (!term)
          for (int e2 = t; e2 < nx * nx; e2 += NT) cp_async_elem<double>(As + e2, Ag + e2);
        for (int e2 = t; e2 < nr * nx; e2 += NT) cp_async_elem<double>(Cs + e2, Cg + e2);
        cp_async_commit();
      }
      for (int j = t; j < nx; j += NT) {
        xv[j] = d.ox[(size_t)i * nx + j];
        if (!term) xn[j] = d.ox[(size_t)(i + 1) * nx + j];
      }
      for (int a = t; a < nu; a += NT) uv[a] = term ? 0.0 : d.ou[(size_t)i * nu + a];
      for (int k = t; k < nr; k += NT) lv[k] = d.olam[(size_t)i * nc + k];
      if (stg) cp_async_wait<0>();
      __syncthreads();
      const double* Qi = stg ? Qs : Qg;
      const double* Ci = stg ? Cs : Cg;
      const double* Ai = stg ? As : Ag;
      const double* Bi = d.B64 + (size_t)i * nx * nu;
      const double* Si = d.S64 + (size_t)i * nu * nx;
      const double* Ri = d.R64 + (size_t)i * nu * nu;
      const double* Di = d.D64 + (size_t)i * nc * nu;
      // Every dot product of the stage is one work item walked by one thread
      // (rows: Q x, A x, B u, S x, R u, C x, D u; columns: C^T lam + S^T u,
      // D^T lam), so all their loads are in flight in one pass.
      const int nrow = term ? nx + nr : 3 * nx + 2 * nu + nr + nc;
      const int ncol = term ? nx : nx + nu;
      for (int it = t; it < nrow + ncol; it += NT) {
        const double* M;
        const double* x;
        int len, stride;
        double* out;
        if (it < nrow) {
          int r = it;
          stride = 1;
          if (r < nx) { M = Qi + (size_t)r * nx; x = xv; len = nx; out = qx + r; }
          else if (term) { r -= nx; M = Ci + (size_t)r * nx; x = xv; len = nx; out = cx + r; }
          else if ((r -= nx) < nx) { M = Ai + (size_t)r * nx; x = xv; len = nx; out = ax + r; }
          else if ((r -= nx) < nx) { M = Bi + (size_t)r * nu; x = uv; len = nu; out = bu + r; }
          else if ((r -= nx) < nu) { M = Si + (size_t)r * nx; x = xv; len = nx; out = sx + r; }
          else if ((r -= nu) < nu) { M = Ri + (size_t)r * nu; x = uv; len = nu; out = ru + r; }
          else if ((r -= nu) < nr) { M = Ci + (size_t)r * nx; x = xv; len = nx; out = cx + r; }
          else { r -= nr; M = Di + (size_t)r * nu; x = uv; len = nu; out = du + r; }
        } else {
          const int col = it - nrow;
          if (col < nx) { M = Ci + col; stride = nx; x = lv; len = nr; out = gt + col; }
          else { M = Di + (col - nx); stride = nu; x = lv; len = nc; out = ht + (col - nx); }
        }
        // eight independent partial sums: eight loads of the row in flight
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0, a4 = 0.0, a5 = 0.0, a6 = 0.0, a7 = 0.0;
        int k = 0;
        for (; k + 7 < len; k += 8) {
          const double* Mk = M + (size_t)k * stride;
          a0 = fma(Mk[0], x[k], a0);
          a1 = fma(Mk[(size_t)stride], x[k + 1], a1);
          a2 = fma(Mk[(size_t)2 * stride], x[k + 2], a2);
          a3 = fma(Mk[(size_t)3 * stride], x[k + 3], a3);
          a4 = fma(Mk[(size_t)4 * stride], x[k + 4], a4);
          a5 = fma(Mk[(size_t)5 * stride], x[k + 5], a5);
          a6 = fma(Mk[(size_t)6 * stride], x[k + 6], a6);
          a7 = fma(Mk[(size_t)7 * stride], x[k + 7], a7);
        }
        for (; k < len; ++k) a0 = fma(M[(size_t)k * stride], x[k], a0);
        a0 = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
        a1 = 0.0;
        if (it >= nrow && it - nrow < nx && !term) {
          // S^T u joins the column sum of C^T lam
          const int col = it - nrow;
          for (int q2 = 0; q2 < nu; ++q2) a1 = fma(Si[(size_t)q2 * nx + col], uv[q2], a1);
        }
        *out = a0 + a1;
      }
      __syncthreads();
      for (int j = t; j < nx; j += NT) d.kg[(size_t)i * nx + j] = qx[j] + gt[j] + d.q64[(size_t)i * nx + j];
      if (!term) {
        for (int j = t; j < nx; j += NT) dyn = fmax(dyn, fabs(xn[j] - ax[j] - bu[j] - d.b64[(size_t)i * nx + j]));
        for (int a = t; a < nu; a += NT) d.kh[(size_t)i * nu + a] = ru[a] + sx[a] + ht[a] + d.r64[(size_t)i * nu + a];
      }
      for (int k = t; k < nr; k += NT) {
        const size_t gi = (size_t)i * nc + k;
        const double v = cx[k] + (term ? 0.0 : du[k]), lo = d.lo64[gi], hi = d.hi64[gi], l = lv[k];
        viol = fmax(viol, fmax(fmax(v - hi, lo - v), 0.0));
        double cp = 0.0;
        if (l > 0) cp = isfinite(hi) ? l * fabs(hi - v) : fabs(l);
        else if (l < 0) cp = isfinite(lo) ? -l * fabs(v - lo) : fabs(l);
        comp = fmax(comp, cp);
      }
      __syncthreads();
    }
    if (c.first) {
      for (int j = t; j < nx; j += NT) dyn = fmax(dyn, fabs(d.ox[j] - d.x064[j]));
    }
  }
  long long kt1 = c.prof ? clock64() : 0;
  cl.sync();
  long long kt2 = c.prof ? clock64() : 0;
  if (c.rank == 0) {
    // costate recursion mu_i = g_i + A_i^T mu_{i+1}, with the u-residual
    // B_i^T mu_{i+1} + h_i at each stage.  Every stage is one split-row sweep
    // over the nx + nu outputs: thread (o, g) sums rows k of group g of
    // A_i(k, o) (o < nx) or B_i(k, o - nx) times mu(k), and the owners of the
    // outputs add the G partial sums.  When two stages' A_i, B_i fit the
    // union region after the vectors, the next stage's are copied into shared
    // memory (cp.async, 8-byte elements: the caller's arrays are unpadded)
    // while the current one is swept; otherwise they are read from global
    // memory in the sweep.
    const int no = nx + nu;
    int G = NT / no;
    G = G < 1 ? 1 : (G > SWEEP_MAXG ? SWEEP_MAXG : G);
    const int Rg = (nx + G - 1) / G;
    const int o = t % no, g = t / no;
    const int r0 = min(nx, g * Rg), r1 = min(nx, r0 + Rg);
    const int per = nx * nx + nx * nu;   // doubles of A_i then B_i
    // the stage scratch is dead here: the recursion reuses the region
    double* mu = xv;
    double* mu2 = xv + 96;
    double* part = xv + 192;              // [G][no] partial sums
    double* pbuf = part + NT;
    const bool pre = (int)((pbuf - xv) + 2 * per) * 8 <= c.uni;
    auto issue = [&](int i, int k) {
      double* dst = pbuf + (size_t)k * per;
      const double* Ai = d.A64 + (size_t)i * nx * nx;
      const double* Bi = d.B64 + (size_t)i * nx * nu;
      for (int e2 = t; e2 < nx * nx; e2 += NT) cp_async_elem<double>(dst + e2, Ai + e2);
      for (int e2 = t; e2 < nx * nu; e2 += NT) cp_async_elem<double>(dst + nx * nx + e2, Bi + e2);
      cp_async_commit();
    };
    for (int j = t; j < nx; j += NT) mu[j] = d.kg[(size_t)N * nx + j];
    double* mcur = mu;    // mu_{i+1}, read by the sweep of stage i
    double* mnext = mu2;  // mu_i, written by the owners (the two swap every stage)
    if (pre) issue(N - 1, 0);
    __syncthreads();
    int kb = 0;
    for (int i = N - 1; i >= 0; --i, kb ^= 1) {
      // the owner's term of this stage, loaded ahead of the copy wait and the sweep
      double own = 0.0;
      if (t < no) own = t < nx ? d.kg[(size_t)i * nx + t] : d.kh[(size_t)i * nu + (t - nx)];
      if (pre) {
        if (i > 0) {
          issue(i - 1, kb ^ 1);
          cp_async_wait<1>();
        } else {
          cp_async_wait<0>();
        }
        __syncthreads();
      }
      if (g < G) {
        const bool isA = o < nx;
        const double* base = pre ? pbuf + (size_t)kb * per
                                 : (isA ? d.A64 + (size_t)i * nx * nx : d.B64 + (size_t)i * nx * nu);
        const double* M = isA ? base + o : (pre ? base + nx * nx : base) + (o - nx);
        const int ld = isA ? nx : nu;
        double a0 = 0.0, a1 = 0.0;
        int k = r0;
        for (; k + 1 < r1; k += 2) {
          a0 = fma(M[(size_t)k * ld], mcur[k], a0);
          a1 = fma(M[(size_t)(k + 1) * ld], mcur[k + 1], a1);
        }
        if (k < r1) a0 = fma(M[(size_t)k * ld], mcur[k], a0);
        part[g * no + o] = a0 + a1;
      }
      __syncthreads();
      if (t < no) {
        double s2 = 0.0;
        for (int gg = 0; gg < G; ++gg) s2 += part[gg * no + t];
        if (t < nx) {
          mnext[t] = s2 + own;
        } else {
          const int a = t - nx;
          const double ru = s2 + own;
          stat = fmax(stat, fabs(ru));
          d.kh[(size_t)i * nu + a] = ru;   // u-stationarity residual, read by refine_linear_term
        }
      }
      __syncthreads();   // mu_i complete; part[] free again
      double* const sw = mcur;
      mcur = mnext;
      mnext = sw;
    }
  }
  if (threadIdx.x == 0 && c.prof) {
    c.prof[PH_KKT_STAGES] += (unsigned long long)(kt1 - kt0);
    c.prof[PH_KKT_SYNC] += (unsigned long long)(kt2 - kt1);
    c.prof[PH_KKT_COSTATE] += (unsigned long long)(clock64() - kt2);
  }
  double v4[4] = {dyn, viol, stat, comp};
  // block-level max of each (reuse red as double scratch)
  double* rd = reinterpret_cast<double*>(c.tmp3) ;
  (void)rd;
  for (int k = 0; k < 4; ++k) {
    double x = v4[k];
    x = warp_max(x);
    __syncthreads();
    if (lane == 0) xv[w] = x;
    __syncthreads();
    double r2 = 0.0;
    for (int q2 = 0; q2 < NT / 32; ++q2) r2 = fmax(r2, xv[q2]);
    v4[k] = r2;
    __syncthreads();
  }
  cluster_max(c, cl, v4);
  return fmax(fmax(v4[0], v4[1]), fmax(v4[2], v4[3]));
}

// Mixed-precision iterative refinement of the ADMM fixed point: fold the FP64
// u-stationarity residual ru_k left by kkt_eval (d.kh) into the linear term,
// r_k <- r_k + ru_k.  With the cached gains this shifts
//   k0_k <- k0_k - Gamma_k ru_k,   c0_k <- c0_k + K_k^T ru_k
// (c0 = Abar^T P b + q + K^T r, k0 = -Gamma (B^T P b + r)); the solve-precision
// copy of r is updated too so that a later refactor keeps the correction.
// The KKT check itself always uses the original FP64 data.
template <typename T>
__device__ void refine_linear_term(Ctx<T>& c) {
  QPDesc& d = *c.d;
  if (!c.active) return;
  const int nx = d.nx, nu = d.nu, nc = d.nc, ldx = d.ldx, ldu = d.ldu, ldv = d.ldv, ldf = d.ldf;
  int bws, fws, cds;
  bundle_sizes(nx, nu, nc, ldx, ldu, ldv, ldf, &bws, &fws, &cds);
  T* r = TP<T>(d.r);
  T* k0 = TP<T>(d.k0);
  T* c0 = TP<T>(d.c0);
  const T* Gam = TP<T>(d.Gam);
  const T* K = TP<T>(d.K);
  const int t = threadIdx.x;
  for (int i = c.s; i < c.e; ++i) {
    T* bw = TP<T>(d.BW) + (size_t)i * bws;
    T* c0b = bw + (size_t)(nx + nc) * ldx + (size_t)(nx + nc) * ldu;
    T* k0b = c0b + ldx;
    for (int a = t; a < nu; a += NT) c.tmp1[a] = (T)d.kh[(size_t)i * nu + a];
    __syncthreads();
    for (int a = t; a < nu; a += NT) {
      T g = T(0);
      for (int b = 0; b < nu; ++b) g += Gam[(size_t)i * nu * ldu + a * ldu + b] * c.tmp1[b];
      k0[(size_t)i * ldu + a] -= g;
      k0b[a] -= g;
      r[(size_t)i * ldu + a] += c.tmp1[a];
    }
    for (int j = t; j < nx; j += NT) {
      T g = T(0);
      for (int a = 0; a < nu; ++a) g += K[(size_t)i * nu * ldx + a * ldx + j] * c.tmp1[a];
      c0[(size_t)i * ldx + j] += g;
      c0b[j] += g;
    }
    __syncthreads();
  }
}

// Multipliers lambda = rho y of own rows into the FP64 output buffer: the
// reference point of the infeasibility certificate (infeas_eval), taken one
// check interval before max_iter.  The final write_outputs overwrites it.
template <typename T>
__device__ void save_multipliers(Ctx<T>& c, T rho) {
  QPDesc& d = *c.d;
  if (!c.active) return;
  const int nrows = own_rows(c);
  for (int e2 = threadIdx.x; e2 < nrows; e2 += NT) d.olam[(size_t)c.s * d.nc + e2] = (double)rho * (double)c.yS[e2];
}

// Block reduction in FP64 (op 0: max, 1: sum) through `scr` (>= NT / 32
// doubles of shared memory); the result is returned to every thread.
__device__ inline double block_reduce_d(double v, int op, double* scr) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  v = op == 0 ? warp_max(v) : warp_sum(v);
  __syncthreads();
  if (l == 0) scr[w] = v;
  __syncthreads();
  double r = 0.0;
  for (int k = 0; k < NT / 32; ++k) r = op == 0 ? fmax(r, scr[k]) : r + scr[k];
  __syncthreads();
  return r;
}

// Primal infeasibility certificate (Farkas) at a solve that reached max_iter.
// The constraints of eq. sqp_qp are the dynamics and initial state, E xi = e
// (rows x_0 = x0 and x_{k+1} - A_k x_k - B_k u_k = b_k), and the bounds
// lo <= G xi <= hi.  No feasible xi exists if some (mu, w) has
// E^T mu + G^T w = 0 and sigma(w) + e^T mu < 0, with the support function
// sigma(w) = sum_i (w_i > 0 ? hi_i w_i : lo_i w_i) of the box.  For a given w
// the x-components fix mu (nu_k the multiplier of stage k's dynamics row):
//   nu_{N-1} = -C_N^T w_N,  nu_{k-1} = A_k^T nu_k - C_k^T w_k (k = N-1 .. 1),
//   mu_0 = A_0^T nu_0 - C_0^T w_0,
// and the u-components are left as the residual r_k = D_k^T w_k - B_k^T nu_k.
// w is the change of the multipliers over the last check interval, lambda
// now minus the saved lambda (olam), which on an infeasible problem tends to
// a certificate direction.  Certified (returned in every thread of the
// cluster) when, with W = ||w||_inf > 0: every w_i pushing against an
// infinite bound is at most tol W, ||r||_inf <= tol W and
// sigma(w) + e^T mu < -tol W.  Every CTA forms w of its own rows in olam;
// CTA 0 runs the serial recursion over the stages in FP64.
template <typename T>
__device__ __noinline__ int infeas_eval(Ctx<T>& c, cg::cluster_group& cl, T rho, double tol) {
  QPDesc& d = *c.d;
  const int nx = d.nx, nu = d.nu, nc = d.nc, nf = d.nf, N = d.N, m = d.m;
  const int t = threadIdx.x;
  if (c.active) {
    const int nrows = own_rows(c);
    for (int e2 = t; e2 < nrows; e2 += NT) {
      const size_t gi = (size_t)c.s * nc + e2;
      d.olam[gi] = (double)rho * (double)c.yS[e2] - d.olam[gi];
    }
  }
  cl.sync();   // every CTA's w in olam
  int cert = 0;
  if (c.rank == 0) {
    double* nu_c = reinterpret_cast<double*>(c.ring);   // FP64 scratch in the union region
    double* nu_n = nu_c + 96;
    double* scr = nu_n + 96;
    const double* w = d.olam;
    // W, the push against infinite bounds, sigma(w)
    double W = 0.0, pinf = 0.0, sig = 0.0;
    for (int i = t; i < m; i += NT) {
      const double wi = w[i];
      W = fmax(W, fabs(wi));
      if (wi > 0.0) {
        const double h = d.hi64[i];
        if (isfinite(h)) sig += h * wi;
        else pinf = fmax(pinf, wi);
      } else if (wi < 0.0) {
        const double l = d.lo64[i];
        if (isfinite(l)) sig += l * wi;
        else pinf = fmax(pinf, -wi);
      }
    }
    W = block_reduce_d(W, 0, scr);
    pinf = block_reduce_d(pinf, 0, scr);
    sig = block_reduce_d(sig, 1, scr);
    // nu_{N-1} = -C_N^T w_N
    for (int j = t; j < nx; j += NT) {
      double a = 0.0;
      for (int k = 0; k < nf; ++k) a += d.CN64[(size_t)k * nx + j] * w[(size_t)N * nc + k];
      nu_c[j] = -a;
    }
    __syncthreads();
    double rmax = 0.0, val = 0.0;   // val: this thread's share of e^T mu
    for (int k = N - 1; k >= 0; --k) {
      const double* Ak = d.A64 + (size_t)k * nx * nx;
      const double* Bk = d.B64 + (size_t)k * nx * nu;
      const double* Ck = d.C64 + (size_t)k * nc * nx;
      const double* Dk = d.D64 + (size_t)k * nc * nu;
      const double* wk = w + (size_t)k * nc;
      if (t < nx) {
        // nu_{k-1} (mu_0 at k = 0) = A_k^T nu_k - C_k^T w_k; e^T mu: b_k^T nu_k
        double a = 0.0, b2 = 0.0;
        for (int i = 0; i < nx; ++i) a = fma(Ak[(size_t)i * nx + t], nu_c[i], a);
        for (int r = 0; r < nc; ++r) b2 = fma(Ck[(size_t)r * nx + t], wk[r], b2);
        nu_n[t] = a - b2;
        val = fma(d.b64[(size_t)k * nx + t], nu_c[t], val);
      } else if (t < nx + nu) {
        // r_k = D_k^T w_k - B_k^T nu_k
        const int q = t - nx;
        double a = 0.0, b2 = 0.0;
        for (int r = 0; r < nc; ++r) a = fma(Dk[(size_t)r * nu + q], wk[r], a);
        for (int i = 0; i < nx; ++i) b2 = fma(Bk[(size_t)i * nu + q], nu_c[i], b2);
        rmax = fmax(rmax, fabs(a - b2));
      }
      __syncthreads();
      double* sw = nu_c;
      nu_c = nu_n;
      nu_n = sw;
    }
    // nu_c = mu_0: e^T mu gains x0^T mu_0
    if (t < nx) val = fma(d.x064[t], nu_c[t], val);
    rmax = block_reduce_d(rmax, 0, scr);
    val = block_reduce_d(val, 1, scr);
    cert = (W > 0.0 && pinf <= tol * W && rmax <= tol * W && sig + val < -tol * W) ? 1 : 0;
  }
  return cluster_or<T>(c, cl, cert);
}

}  // namespace gsls
