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

// Number of constraint rows owned by this CTA (stage rows, plus terminal rows
// for the last chunk).  Owned row `lr` has global index s*nc + lr.
template <typename T>
__device__ inline int own_rows(Ctx<T>& c) {
  return c.active ? c.L * c.d->nc + (c.last ? c.d->nf : 0) : 0;
}

// Dependent chain over the chunk with the per-stage matrices Abar staged into a
// 3-slot shared-memory ring by cp.async (two stages ahead of the compute).
//   backward: l_i = Abar_i^T l_{i+1} + c_i for i = e-1 .. s
//   forward:  x_{i+1} = Abar_i x_i + d_i for i = s .. e-1
template <typename T>
__device__ void chain(Ctx<T>& c, bool backward) {
  QPDesc& d = *c.d;
  const int nx = d.nx, ldx = d.ldx, L = c.L, msz = c.msz;
  const T* Abar = TP<T>(d.Abar);
  const int bytes = msz * (int)sizeof(T);
  auto stage_of = [&](int st) { return backward ? (c.e - 1 - st) : (c.s + st); };
#pragma unroll 1
  for (int st = 0; st < 2; ++st) {
    if (st < L) cta_stage(c.ring + (size_t)st * msz, Abar + (size_t)stage_of(st) * msz, bytes);
    cp_async_commit();
  }
#pragma unroll 1
  for (int st = 0; st < L; ++st) {
    if (st + 2 < L) cta_stage(c.ring + (size_t)((st + 2) % 3) * msz, Abar + (size_t)stage_of(st + 2) * msz, bytes);
    cp_async_commit();
    cp_async_wait<2>();
    __syncthreads();
    const T* M = c.ring + (size_t)(st % 3) * msz;
    if (backward) {
      const int li = c.e - 1 - st - c.s;
      smem_mvT<T>(M, ldx, nx, nx, c.lS + (size_t)(li + 1) * ldx, c.cS + (size_t)li * ldx, c.lS + (size_t)li * ldx, c.red);
    } else {
      smem_mv<T>(M, ldx, nx, nx, c.xS + (size_t)st * ldx, c.dS + (size_t)st * ldx, c.xS + (size_t)(st + 1) * ldx);
    }
  }
  cp_async_wait<0>();
  __syncthreads();
}

struct Partials {
  double rp, rd, vm, zm;
};

// One ADMM iteration (eq. augmented_linear, the LQ solve of eq. primal_update
// with cached factorization, the z-projection and the scaled dual update).
// On `check` iterations the per-CTA dual-residual partial is also formed.
template <typename T>
__device__ void admm_iteration(Ctx<T>& c, cg::cluster_group& cl, T rho, bool check, Partials& pl) {
  QPDesc& d = *c.d;
  const int nx = d.nx, nu = d.nu, nc = d.nc, N = d.N, ldx = d.ldx, ldu = d.ldu, ldc = d.ldc;
  const int msz = c.msz, L = c.L, s = c.s;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const T *B = TP<T>(d.B), *bb = TP<T>(d.b), *q = TP<T>(d.q), *C = TP<T>(d.C), *D = TP<T>(d.D), *CN = TP<T>(d.CN);
  const T *lo = TP<T>(d.lo), *hi = TP<T>(d.hi), *x0 = TP<T>(d.x0);
  const T *CK = TP<T>(d.CK), *F = TP<T>(d.F), *FPi = TP<T>(d.FPi), *J = TP<T>(d.J);
  const T *CKSig = TP<T>(d.CKSig), *c0 = TP<T>(d.c0), *k0 = TP<T>(d.k0), *CNSig = TP<T>(d.CNSig);
  const T *Theta = TP<T>(d.Theta), *Xi = TP<T>(d.Xi);
  const int nrows = own_rows(c);

  // P1: omega = rho (y - z); c_i = c0_i + CK_i^T omega_i; boundary of the
  // backward chain (p_N = q^_N for the last chunk, 0 otherwise).
  if (c.active) {
    for (int e2 = t; e2 < nrows; e2 += NT) c.wS[e2] = rho * (c.yS[e2] - c.zS[e2]);
    __syncthreads();
    for (int e2 = t; e2 < L * nx; e2 += NT) {
      const int li = e2 / nx, j = e2 - li * nx, i = s + li;
      const T* CKi = CK + (size_t)i * nc * ldx;
      T a = c0[(size_t)i * ldx + j];
      for (int rr = 0; rr < nc; ++rr) a += CKi[rr * ldx + j] * c.wS[li * nc + rr];
      c.cS[li * ldx + j] = a;
    }
    for (int j = t; j < nx; j += NT) {
      T a = T(0);
      if (c.last) {
        a = q[(size_t)N * ldx + j];
        for (int rr = 0; rr < d.nf; ++rr) a += CN[rr * ldx + j] * c.wS[L * nc + rr];
      }
      c.lS[(size_t)L * ldx + j] = a;
    }
    __syncthreads();
    // P2: backward chunk-local chain
    chain<T>(c, true);
    for (int j = t; j < nx; j += NT) c.slotL[j] = c.lS[j];
  }
  cl.sync();
  // P3: boundary p_e from the later chunks, then k_i and d_i.
  if (c.active) {
    if (!c.last) {
      const T* rem = cl.map_shared_rank(c.slotL, c.rank + 1);
      for (int j = t; j < nx; j += NT) c.pe[j] = rem[j];
      __syncthreads();
      for (int m = c.rank + 2; m < d.nch; ++m) {
        const T* rm = cl.map_shared_rank(c.slotL, m);
        for (int j = t; j < nx; j += NT) c.tmp1[j] = rm[j];
        __syncthreads();
        g_mv<T>(Theta + (size_t)(c.rank * MAXCS + m) * msz, ldx, nx, nx, c.tmp1, T(1), true, c.pe);
      }
    }
    for (int pr = w; pr < L * nu; pr += NT / 32) {
      const int li = pr / nu, a = pr - li * nu, i = s + li;
      T v = warp_dot(F + (size_t)i * nu * ldx + a * ldx, c.lS + (size_t)(li + 1) * ldx, nx);
      if (!c.last) v += warp_dot(FPi + (size_t)i * nu * ldx + a * ldx, c.pe, nx);
      v += warp_dot(J + (size_t)i * nu * ldc + a * ldc, c.wS + li * nc, nc);
      if (lane == 0) c.kS[li * ldu + a] = v + k0[(size_t)i * ldu + a];
    }
    __syncthreads();
    for (int e2 = t; e2 < L * nx; e2 += NT) {
      const int li = e2 / nx, row = e2 - li * nx, i = s + li;
      const T* Bi = B + (size_t)i * nx * ldu + row * ldu;
      T a = bb[(size_t)i * ldx + row];
      for (int k = 0; k < nu; ++k) a += Bi[k] * c.kS[li * ldu + k];
      c.dS[li * ldx + row] = a;
    }
    for (int j = t; j < nx; j += NT) c.xS[j] = c.first ? x0[j] : T(0);
    __syncthreads();
    // P4: forward chunk-local chain
    chain<T>(c, false);
    for (int j = t; j < nx; j += NT) c.slotX[j] = c.xS[(size_t)L * ldx + j];
  }
  cl.sync();
  // P5: boundary x_s from the earlier chunks, G(dx, du), projection, dual update.
  if (c.active) {
    if (!c.first) {
      const T* rem = cl.map_shared_rank(c.slotX, c.rank - 1);
      for (int j = t; j < nx; j += NT) c.xs[j] = rem[j];
      __syncthreads();
      for (int m = c.rank - 2; m >= 0; --m) {
        const T* rm = cl.map_shared_rank(c.slotX, m);
        for (int j = t; j < nx; j += NT) c.tmp1[j] = rm[j];
        __syncthreads();
        g_mv<T>(Xi + (size_t)(c.rank * MAXCS + m) * msz, ldx, nx, nx, c.tmp1, T(1), true, c.xs);
      }
    }
    T rp = T(0), vm = T(0), zm = T(0);
    for (int lr = w; lr < nrows; lr += NT / 32) {
      T v;
      if (lr < L * nc) {
        const int li = lr / nc, rr = lr - li * nc, i = s + li;
        v = warp_dot(CK + (size_t)i * nc * ldx + rr * ldx, c.xS + (size_t)li * ldx, nx);
        if (!c.first) v += warp_dot(CKSig + (size_t)i * nc * ldx + rr * ldx, c.xs, nx);
        v += warp_dot(D + (size_t)i * nc * ldu + rr * ldu, c.kS + li * ldu, nu);
      } else {
        const int rr = lr - L * nc;
        v = warp_dot(CN + rr * ldx, c.xS + (size_t)L * ldx, nx);
        if (!c.first) v += warp_dot(CNSig + rr * ldx, c.xs, nx);
      }
      if (lane == 0) {
        const int g = s * nc + lr;
        const T zo = c.zS[lr], yo = c.yS[lr];
        const T zn = fmin(fmax(v + yo, lo[g]), hi[g]);
        c.yS[lr] = yo + v - zn;
        c.zS[lr] = zn;
        c.wS[lr] = zn - zo;
        rp = fmax(rp, fabs(v - zn));
        vm = fmax(vm, fabs(v));
        zm = fmax(zm, fabs(zn));
      }
    }
    __syncthreads();
    if (check) {
      pl.rp = (double)block_max(c, rp);
      pl.vm = (double)block_max(c, vm);
      pl.zm = (double)block_max(c, zm);
      // dual residual partial: rho * ||G^T (z+ - z)||_inf over own stages
      T rd = T(0);
      for (int e2 = t; e2 < L * nx; e2 += NT) {
        const int li = e2 / nx, j = e2 - li * nx, i = s + li;
        const T* Ci = C + (size_t)i * nc * ldx;
        T a = T(0);
        for (int rr = 0; rr < nc; ++rr) a += Ci[rr * ldx + j] * c.wS[li * nc + rr];
        rd = fmax(rd, fabs(a));
      }
      for (int e2 = t; e2 < L * nu; e2 += NT) {
        const int li = e2 / nu, a2 = e2 - li * nu, i = s + li;
        const T* Di = D + (size_t)i * nc * ldu;
        T a = T(0);
        for (int rr = 0; rr < nc; ++rr) a += Di[rr * ldu + a2] * c.wS[li * nc + rr];
        rd = fmax(rd, fabs(a));
      }
      if (c.last) {
        for (int j = t; j < nx; j += NT) {
          T a = T(0);
          for (int rr = 0; rr < d.nf; ++rr) a += CN[rr * ldx + j] * c.wS[L * nc + rr];
          rd = fmax(rd, fabs(a));
        }
      }
      pl.rd = (double)rho * (double)block_max(c, rd);
    }
  } else {
    pl.rp = pl.rd = pl.vm = pl.zm = 0.0;
  }
}

// Full state and input of own stages: x_i = lx_i + Sig_i x_s (into dS rows
// 0..L, row L = x_N for the last chunk), u_i = K_i lx_i + KSig_i x_s + k_i.
template <typename T>
__device__ void full_xu(Ctx<T>& c) {
  QPDesc& d = *c.d;
  const int nx = d.nx, nu = d.nu, ldx = d.ldx, ldu = d.ldu, msz = c.msz, L = c.L, s = c.s;
  const T *K = TP<T>(d.K), *KSig = TP<T>(d.KSig), *Sig = TP<T>(d.Sig), *SigN = TP<T>(d.SigN);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nxr = (L + (c.last ? 1 : 0)) * nx;
  for (int pr = w; pr < nxr; pr += NT / 32) {
    const int li = pr / nx, j = pr - li * nx;
    T v = T(0);
    if (!c.first) {
      const T* Sr = (li < L) ? Sig + (size_t)(s + li) * msz + j * ldx : SigN + j * ldx;
      v = warp_dot(Sr, c.xs, nx);
    }
    if (lane == 0) c.dS[(size_t)li * ldx + j] = c.xS[(size_t)li * ldx + j] + v;
  }
  for (int pr = w; pr < L * nu; pr += NT / 32) {
    const int li = pr / nu, a = pr - li * nu, i = s + li;
    T v = warp_dot(K + (size_t)i * nu * ldx + a * ldx, c.xS + (size_t)li * ldx, nx);
    if (!c.first) v += warp_dot(KSig + (size_t)i * nu * ldx + a * ldx, c.xs, nx);
    if (lane == 0) c.uS[li * ldu + a] = v + c.kS[li * ldu + a];
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
    for (int e2 = t; e2 < L * nx; e2 += NT) {
      const int li = e2 / nx, j = e2 - li * nx, i = s + li;
      const T* Qi = Q + (size_t)i * msz + j * ldx;
      T a = T(0);
      for (int k = 0; k < nx; ++k) a += Qi[k] * c.dS[li * ldx + k];
      const T* Si = S + (size_t)i * nu * ldx;
      for (int k = 0; k < nu; ++k) a += Si[k * ldx + j] * c.uS[li * ldu + k];
      h = fmax(h, fabs(a));
      const T* Ci = C + (size_t)i * nc * ldx;
      T b2 = T(0);
      for (int rr = 0; rr < nc; ++rr) b2 += Ci[rr * ldx + j] * c.yS[li * nc + rr];
      g = fmax(g, fabs(rho * b2));
      qq = fmax(qq, fabs(q[(size_t)i * ldx + j]));
    }
    for (int e2 = t; e2 < L * nu; e2 += NT) {
      const int li = e2 / nu, a2 = e2 - li * nu, i = s + li;
      const T* Ri = R + (size_t)i * nu * ldu + a2 * ldu;
      T a = T(0);
      for (int k = 0; k < nu; ++k) a += Ri[k] * c.uS[li * ldu + k];
      const T* Si = S + (size_t)i * nu * ldx + a2 * ldx;
      for (int k = 0; k < nx; ++k) a += Si[k] * c.dS[li * ldx + k];
      h = fmax(h, fabs(a));
      const T* Di = D + (size_t)i * nc * ldu;
      T b2 = T(0);
      for (int rr = 0; rr < nc; ++rr) b2 += Di[rr * ldu + a2] * c.yS[li * nc + rr];
      g = fmax(g, fabs(rho * b2));
      qq = fmax(qq, fabs(r[(size_t)i * ldu + a2]));
    }
    if (c.last) {
      for (int j = t; j < nx; j += NT) {
        const T* Qi = Q + (size_t)N * msz + j * ldx;
        T a = T(0);
        for (int k = 0; k < nx; ++k) a += Qi[k] * c.dS[L * ldx + k];
        h = fmax(h, fabs(a));
        T b2 = T(0);
        for (int rr = 0; rr < d.nf; ++rr) b2 += CN[rr * ldx + j] * c.yS[L * nc + rr];
        g = fmax(g, fabs(rho * b2));
        qq = fmax(qq, fabs(q[(size_t)N * ldx + j]));
      }
    }
  }
  hm = (double)block_max(c, h);
  gm = (double)block_max(c, g);
  qm = (double)block_max(c, qq);
}

// Cluster-wide max of up to 8 doubles through the part[] slots.
template <typename T>
__device__ void cluster_max(Ctx<T>& c, cg::cluster_group& cl, double* v, int n) {
  if (threadIdx.x < n) c.part[threadIdx.x] = v[threadIdx.x];
  cl.sync();
  for (int k = 0; k < n; ++k) v[k] = 0.0;
  for (int rk = 0; rk < c.cs; ++rk) {
    const double* p = cl.map_shared_rank(c.part, rk);
    for (int k = 0; k < n; ++k) {
      const double a = p[k];
      v[k] = (a != a || v[k] != v[k]) ? a + v[k] : fmax(v[k], a);
    }
  }
  cl.sync();
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

// FP64 KKT residual of (ox, ou, olam) -- see include/gpusls.h for the
// definition.  Every CTA evaluates the stage-local parts of its chunk; CTA 0
// then runs the costate recursion mu_k = g_k + A_k^T mu_{k+1} sequentially.
template <typename T>
__device__ __noinline__ double kkt_eval(Ctx<T>& c, cg::cluster_group& cl) {
  QPDesc& d = *c.d;
  const int nx = d.nx, nu = d.nu, nc = d.nc, nf = d.nf, N = d.N;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  double* xv = reinterpret_cast<double*>(c.ring);   // FP64 scratch in the union region
  double* xn = xv + 96;
  double* uv = xn + 96;
  double* lv = uv + 96;
  double* mu = lv + 96;
  double* mu2 = mu + 96;
  double dyn = 0.0, viol = 0.0, comp = 0.0, stat = 0.0;
  cl.sync();   // outputs of every chunk visible
  if (c.active) {
    const int iend = c.e + (c.last ? 1 : 0);
    for (int i = c.s; i < iend; ++i) {
      const bool term = (i == N);
      const int nr = term ? nf : nc;
      for (int j = t; j < nx; j += NT) {
        xv[j] = d.ox[(size_t)i * nx + j];
        if (!term) xn[j] = d.ox[(size_t)(i + 1) * nx + j];
      }
      for (int a = t; a < nu; a += NT) uv[a] = term ? 0.0 : d.ou[(size_t)i * nu + a];
      for (int k = t; k < nr; k += NT) lv[k] = d.olam[(size_t)i * nc + k];
      __syncthreads();
      const double* Qi = d.Q64 + (size_t)i * nx * nx;
      const double* Ci = term ? d.CN64 : d.C64 + (size_t)i * nc * nx;
      const double* Di = term ? nullptr : d.D64 + (size_t)i * nc * nu;
      // dynamics row j: x_{i+1} - A x - B u - b ;  g_i = Q x + S^T u + q + C^T lam
      for (int j = w; j < nx; j += NT / 32) {
        double gsum = warp_dot(Qi + (size_t)j * nx, xv, nx);
        if (!term) {
          const double* Ai = d.A64 + (size_t)i * nx * nx + (size_t)j * nx;
          const double* Bi = d.B64 + (size_t)i * nx * nu + (size_t)j * nu;
          const double ax = warp_dot(Ai, xv, nx) + warp_dot(Bi, uv, nu);
          if (lane == 0) dyn = fmax(dyn, fabs(xn[j] - ax - d.b64[(size_t)i * nx + j]));
          double st = 0.0;
          for (int a = lane; a < nu; a += 32) st += d.S64[(size_t)i * nu * nx + (size_t)a * nx + j] * uv[a];
          gsum += warp_sum(st);
        }
        double ct = 0.0;
        for (int k = lane; k < nr; k += 32) ct += Ci[(size_t)k * nx + j] * lv[k];
        gsum += warp_sum(ct);
        if (lane == 0) d.kg[(size_t)i * nx + j] = gsum + d.q64[(size_t)i * nx + j];
      }
      if (!term) {
        // h_i = R u + S x + r + D^T lam
        for (int a = w; a < nu; a += NT / 32) {
          double hs = warp_dot(d.R64 + (size_t)i * nu * nu + (size_t)a * nu, uv, nu) +
                      warp_dot(d.S64 + (size_t)i * nu * nx + (size_t)a * nx, xv, nx);
          double dt = 0.0;
          for (int k = lane; k < nc; k += 32) dt += Di[(size_t)k * nu + a] * lv[k];
          hs += warp_sum(dt);
          if (lane == 0) d.kh[(size_t)i * nu + a] = hs + d.r64[(size_t)i * nu + a];
        }
      }
      // rows: v = C x + D u ; violation and complementarity
      for (int k = w; k < nr; k += NT / 32) {
        double v = warp_dot(Ci + (size_t)k * nx, xv, nx);
        if (!term) v += warp_dot(Di + (size_t)k * nu, uv, nu);
        if (lane == 0) {
          const size_t gi = (size_t)i * nc + k;
          const double lo = d.lo64[gi], hi = d.hi64[gi], l = lv[k];
          viol = fmax(viol, fmax(fmax(v - hi, lo - v), 0.0));
          double cp = 0.0;
          if (l > 0) cp = isfinite(hi) ? l * fabs(hi - v) : fabs(l);
          else if (l < 0) cp = isfinite(lo) ? -l * fabs(v - lo) : fabs(l);
          comp = fmax(comp, cp);
        }
      }
      __syncthreads();
    }
    if (c.first) {
      for (int j = t; j < nx; j += NT) dyn = fmax(dyn, fabs(d.ox[j] - d.x064[j]));
    }
  }
  cl.sync();
  if (c.rank == 0) {
    for (int j = t; j < nx; j += NT) mu[j] = d.kg[(size_t)N * nx + j];
    __syncthreads();
    for (int i = N - 1; i >= 0; --i) {
      for (int a = w; a < nu; a += NT / 32) {
        double s2 = 0.0;
        for (int j = lane; j < nx; j += 32) s2 += d.B64[(size_t)i * nx * nu + (size_t)j * nu + a] * mu[j];
        s2 = warp_sum(s2);
        if (lane == 0) stat = fmax(stat, fabs(s2 + d.kh[(size_t)i * nu + a]));
      }
      for (int j = t; j < nx; j += NT) {
        double s2 = d.kg[(size_t)i * nx + j];
        const double* Ai = d.A64 + (size_t)i * nx * nx;
        for (int k = 0; k < nx; ++k) s2 += Ai[(size_t)k * nx + j] * mu[k];
        mu2[j] = s2;
      }
      __syncthreads();
      for (int j = t; j < nx; j += NT) mu[j] = mu2[j];
      __syncthreads();
    }
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
  cluster_max(c, cl, v4, 4);
  return fmax(fmax(v4[0], v4[1]), fmax(v4[2], v4[3]));
}

}  // namespace gsls
