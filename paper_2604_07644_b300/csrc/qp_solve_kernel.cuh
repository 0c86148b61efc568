// The persistent solve kernel (one thread-block cluster per QP), included by
// one translation unit per precision (qp_kernel_f32.cu, qp_kernel_f64.cu) so
// that the two compile in parallel; the host code launches it through
// qp_kernel_entry<T>().
#pragma once
#include "../../include/gpusls.h"
#include "qp_iter.cuh"

namespace gsls {

// ---------------------------------------------------------------------------
// the solve kernel
// ---------------------------------------------------------------------------
// FP32 solves fit two CTAs per SM (<= 128 registers, ~100 KB shared), which
// lets one cluster's barrier and latency stalls overlap another's work.
template <typename T> struct KernelOcc { static constexpr int value = sizeof(T) == 4 ? 2 : 1; };

constexpr int FP32_STALL_ITERS = 250;

template <typename T>
__global__ void __launch_bounds__(NT, KernelOcc<T>::value) qp_kernel(const QPDesc* __restrict__ descs, SolveArgs args) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ QPDesc dsh;
  const int cs = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int qi = args.order ? args.order[blockIdx.x / cs] : (int)(blockIdx.x / cs);
  if (threadIdx.x == 0) dsh = descs[qi];
  __syncthreads();
  QPDesc& d = dsh;

  const SmemLayout lay = smem_layout(d.nx, d.nu, d.nc, d.nf, d.Lc, d.nch, cs, d.ldx, d.ldu, d.ldv, d.ldf, d.depth, d.slot,
                                     (int)sizeof(T), d.fact, d.vg);
  // One context per CTA in shared memory, filled by thread 0: every thread
  // reads the same fields, and a per-thread copy would sit in local memory
  // that the L1 left beside two CTAs' shared memory cannot hold.
  __shared__ Ctx<T> csh;
  Ctx<T>& c = csh;
  const int t = threadIdx.x;
  if (t == 0) {
    c.d = &d;
    c.rank = rank;
    c.cs = cs;
    c.s = min(rank * d.Lc, d.N);
    c.e = min((rank + 1) * d.Lc, d.N);
    c.L = c.e - c.s;
    c.active = rank < d.nch;
    c.first = rank == 0;
    c.last = rank == d.nch - 1;
    c.gemm = reinterpret_cast<T*>(smem + lay.gemm);
    c.gj = reinterpret_cast<T*>(smem + lay.gj);
    c.gjbuf = reinterpret_cast<T*>(smem + lay.gjbuf);
    c.ring = reinterpret_cast<T*>(smem + lay.ring);
    // the per-chunk vectors: shared memory, or this CTA's global region (vg)
    unsigned char* vb = d.vg ? static_cast<unsigned char*>(d.vec) + (size_t)rank * d.vstride : smem;
    c.zS = reinterpret_cast<T*>(vb + lay.z);
    c.yS = reinterpret_cast<T*>(vb + lay.y);
    c.wS = reinterpret_cast<T*>(vb + lay.w);
    c.lS = reinterpret_cast<T*>(vb + lay.l);
    c.xS = reinterpret_cast<T*>(vb + lay.x);
    c.ktS = reinterpret_cast<T*>(vb + lay.kt);
    c.vS = reinterpret_cast<T*>(vb + lay.v);
    c.dS = reinterpret_cast<T*>(vb + lay.d);
    c.uS = reinterpret_cast<T*>(vb + lay.u);
    c.pe = reinterpret_cast<T*>(smem + lay.pe);
    c.xs = reinterpret_cast<T*>(smem + lay.xs);
    c.slotL = reinterpret_cast<T*>(smem + lay.slotL);
    c.slotX = reinterpret_cast<T*>(smem + lay.slotX);
    c.tmp1 = reinterpret_cast<T*>(smem + lay.tmp1);
    c.tmp2 = reinterpret_cast<T*>(smem + lay.tmp2);
    c.tmp3 = reinterpret_cast<T*>(smem + lay.tmp3);
    c.red = reinterpret_cast<T*>(smem + lay.red);
    c.part = reinterpret_cast<double*>(smem + lay.part);
    c.perm = reinterpret_cast<int*>(smem + lay.perm);
    c.flag = reinterpret_cast<int*>(smem + lay.flag);
    c.bar = reinterpret_cast<unsigned long long*>(smem + lay.bar);
    c.swp = reinterpret_cast<T*>(smem + lay.swp);
    c.gath = reinterpret_cast<T*>(smem + lay.gath);
    c.ws = c.wp = 0;
    c.inflight = c.ipar = 0;
    c.bpar = 0;
    c.bulk_inflight = 0;
    c.cm_par = 0;
    for (int k = 0; k < d.depth; ++k) mbar_init(&c.bar[k], 1);
    mbar_init(&c.bar[BULK_BAR], 1);
    mbar_init_fence();
    c.flag[RING_FLAG] = 0;
    c.msz = d.nx * d.ldx;
    c.uni = lay.uni;
    c.scr = TP<T>(d.scr) + (size_t)rank * 6 * c.msz;
    c.prof = (args.prof && qi == 0 && t == 0) ? args.prof + (size_t)rank * PH_COUNT : nullptr;
    c.t_last = clock64();
    c.gains = args.mode == MODE_GAINS;
    c.tc = args.tc == 1;
    c.mix = args.tc == 2;
    iter_plan<T>(c);
  }
  __syncthreads();

  if (args.mode == MODE_KKT) {
    const double kkt = kkt_eval<T>(c, cl);
    if (rank == 0 && t == 0) d.info_d[3] = kkt;
    cl.sync();   // no CTA leaves while another may still read its shared memory
    return;
  }

  T rho = (T)d.rho[0];
  int refactors = 0;
  int status = GPUSLS_MAX_ITER;
  if (args.mode == MODE_RICCATI || args.mode == MODE_GAINS || d.flags[0] == 0) {
    const int bad = refactor<T>(c, cl, rho);
    ++refactors;
    if (bad) status = GPUSLS_ERR_NOT_SPD;
  }
  if (args.mode == MODE_RICCATI || args.mode == MODE_GAINS) {
    // P_i = level-0 inclusive suffixes, K_i gains, as FP64 dense blocks.
    const int nx = d.nx, nu = d.nu, ldx = d.ldx, msz = c.msz;
    if (c.active && d.ox && d.ou) {
      const int iend = c.e + (c.last ? 1 : 0);
      for (int i = c.s; i < iend; ++i)
        for (int e2 = t; e2 < nx * nx; e2 += NT)
          d.ox[(size_t)i * nx * nx + e2] = (double)TP<T>(d.IP)[(size_t)i * msz + (e2 / nx) * ldx + e2 % nx];
      for (int i = c.s; i < c.e; ++i)
        for (int e2 = t; e2 < nu * nx; e2 += NT)
          d.ou[(size_t)i * nu * nx + e2] = (double)TP<T>(d.K)[(size_t)i * nu * ldx + (e2 / nx) * ldx + e2 % nx];
    }
    if (rank == 0 && t == 0) {
      d.info_i[0] = status == GPUSLS_ERR_NOT_SPD ? status : GPUSLS_OK;
      d.info_i[2] = refactors;
      d.flags[0] = (status == GPUSLS_ERR_NOT_SPD || args.mode == MODE_GAINS) ? 0 : 1;
    }
    cl.sync();
    return;
  }

  // load the ADMM state of own rows
  const int nrows = own_rows(c);
  const T* zg = TP<T>(d.z);
  const T* yg = TP<T>(d.y);
  for (int e2 = t; e2 < nrows; e2 += NT) {
    c.zS[e2] = zg[(size_t)c.s * d.nc + e2];
    c.yS[e2] = yg[(size_t)c.s * d.nc + e2];
  }
  // the forward chain's start lx_s (x0 for the first chunk, 0 for the others);
  // no phase writes row 0 of xS below column nx
  for (int j = t; j < d.nx; j += NT) c.xS[j] = c.first ? TP<T>(d.x0)[j] : T(0);
  __syncthreads();

  double eps = args.eps;
  const bool fixed = args.fixed_iters > 0;
  const int max_it = fixed ? args.fixed_iters : args.max_iter;
  double rp = INFINITY, rd = INFINITY, kkt = -1.0;
  int it = 0;
  int refines = 0;
  int floor_it = -1;   // FP32: iteration from which the gate has waited at the eps floor
  bool warm = d.flags[1] != 0;
  const int it_warm0 = 0;
  int fell_back = 0;
  if (status != GPUSLS_ERR_NOT_SPD) {
    if (args.test_wait) {
      // test hook: wait (bounded) for the next completion of the whole-region
      // copy barrier, which no copy is issued to; the wait gives up, the
      // flag stops every later copy and wait, and the first check reports
      // GPUSLS_ERR_TIMEOUT
      if (!mbar_wait(&c.bar[BULK_BAR], c.bpar, RING_WAIT_LIMIT)) c.flag[RING_FLAG] = 1;
      __syncthreads();
    }
    for (it = 1; it <= max_it; ++it) {
      const bool stop_iter = !fixed && (it % args.check_every == 0);
      const bool rho_iter = !fixed && args.sigma > 0 && (it % args.sigma == 0);
      const bool check = stop_iter || rho_iter || (it == max_it);
      Partials pl;
      admm_iteration<T>(c, cl, rho, check, pl);
      // the reference multipliers of the infeasibility certificate
      if (!fixed && it == max_it - args.check_every) save_multipliers<T>(c, rho);
      if (!check) continue;
      double v[5] = {pl.rp, 0.0, pl.vm, pl.zm, c.flag[RING_FLAG] ? 1.0 : 0.0};
      cluster_max(c, cl, v);
      rp = v[0];
      // the dual residual only where a decision reads it: the primal test
      // passed, a rho update, the last iteration (all uniform in the cluster)
      const bool need_rd = rho_iter || it == max_it || (stop_iter && rp <= eps);
      if (need_rd && v[4] == 0.0 && isfinite(rp)) {
        double u2[2] = {dual_residual_partial<T>(c, rho), c.flag[RING_FLAG] ? 1.0 : 0.0};
        cluster_max(c, cl, u2);
        rd = u2[0];
        v[4] = fmax(v[4], u2[1]);
      }
      prof_mark(c, PH_CHECK);
      if (v[4] > 0.0) {
        status = GPUSLS_ERR_TIMEOUT;
        break;
      }
      if (!isfinite(rp) || (need_rd && !isfinite(rd))) {
        status = GPUSLS_ERR_NAN;
        break;
      }
      // FP32 stall rule: rounding in the FP32 operators can hold r_prim or
      // r_dual just above the eps floor, where the gate below would never
      // run; after FP32_STALL_ITERS iterations at the floor it runs anyway
      // (and refines the linear term if the FP64 KKT check fails).
      // eps counts as at the floor within a relative 1e-9: repeated
      // multiplication by 0.1 does not land on the floor exactly in binary
      const bool at_floor = eps <= args.eps_floor * (1.0 + 1e-9);
      bool stalled = false;
      if (sizeof(T) == 4 && at_floor) {
        if (floor_it < 0) floor_it = it;
        stalled = it - floor_it >= FP32_STALL_ITERS;
      }
      if (stop_iter && ((rp <= eps && rd <= eps) || stalled)) {
        floor_it = -1;
        if (args.eps_kkt <= 0.0) {
          status = GPUSLS_OK;
          break;
        }
        full_xu<T>(c);
        write_outputs<T>(c, rho);
        kkt = kkt_eval<T>(c, cl);
        prof_mark(c, PH_KKT);
        if (kkt <= args.eps_kkt) {
          status = GPUSLS_OK;
          break;
        }
        if (!at_floor) {
          eps = fmax(eps * 0.1, args.eps_floor);
        } else if (refines < args.max_refine) {
          refine_linear_term<T>(c);
          ++refines;
        }
      }
      if (warm && args.fallback_iters > 0 && it - it_warm0 >= args.fallback_iters) {
        // cold-start fallback of a warm start that did not converge in time
        for (int e2 = t; e2 < nrows; e2 += NT) {
          c.zS[e2] = T(0);
          c.yS[e2] = T(0);
        }
        warm = false;
        fell_back = 1;
        eps = args.eps;
        const T rho_c = (T)d.rho0[0];
        __syncthreads();
        if (rho_c != rho) {
          rho = rho_c;
          const int bad = refactor<T>(c, cl, rho);
          ++refactors;
          if (bad) {
            status = GPUSLS_ERR_NOT_SPD;
            break;
          }
        }
        continue;
      }
      if (rho_iter) {
        full_xu<T>(c);
        double hm, gm, qm;
        rho_rule_partials<T>(c, rho, hm, gm, qm);
        double u[3] = {hm, gm, qm};
        cluster_max(c, cl, u);
        prof_mark(c, PH_RHO);
        const double prim_scale = fmax(v[2], v[3]);
        const double dual_scale = fmax(fmax(u[0], u[1]), u[2]);
        double rho_new = (double)rho;
        if (rp > 0.0 && rd > 0.0 && prim_scale > 0.0 && dual_scale > 0.0) {
          const double ratio = (rp / prim_scale) / (rd / dual_scale);
          rho_new = fmin(fmax((double)rho * sqrt(ratio), args.rho_min), args.rho_max);
        }
        if (rho_new > 5.0 * (double)rho || rho_new < (double)rho / 5.0) {
          const T scale = (T)((double)rho / rho_new);
          for (int e2 = t; e2 < nrows; e2 += NT) c.yS[e2] *= scale;
          rho = (T)rho_new;
          __syncthreads();
          const int bad = refactor<T>(c, cl, rho);
          ++refactors;
          if (bad) {
            status = GPUSLS_ERR_NOT_SPD;
            break;
          }
        }
      }
    }
    if (it > max_it) it = max_it;
    // a solve that ran out of iterations: a primal infeasibility certificate
    // from the multipliers' change over the last check interval
    if (status == GPUSLS_MAX_ITER && !fixed && max_it > args.check_every &&
        infeas_eval<T>(c, cl, rho, args.eps))
      status = GPUSLS_ERR_INFEASIBLE;
    full_xu<T>(c);
    write_outputs<T>(c, rho);
    if (status == GPUSLS_OK && args.eps_kkt <= 0.0) kkt = -1.0;
  }
  // store state
  T* zw = TP<T>(d.z);
  T* yw = TP<T>(d.y);
  for (int e2 = t; e2 < nrows; e2 += NT) {
    zw[(size_t)c.s * d.nc + e2] = c.zS[e2];
    yw[(size_t)c.s * d.nc + e2] = c.yS[e2];
  }
  if (rank == 0 && t == 0) {
    d.info_i[0] = status;
    d.info_i[1] = it;
    d.info_i[2] = refactors;
    d.info_i[3] = refines;
    d.info_i[4] = fell_back;
    d.info_d[0] = (double)rho;
    d.info_d[1] = rp;
    d.info_d[2] = rd;
    d.info_d[3] = kkt;
    d.rho[0] = (double)rho;
    d.flags[0] = (status == GPUSLS_ERR_NOT_SPD) ? 0 : 1;
    d.flags[1] = 0;
    d.flags[2] = fell_back;
  }
  ring_drain<T>(c);
  cl.sync();   // no CTA leaves while another may still read its shared memory
}

}  // namespace gsls
