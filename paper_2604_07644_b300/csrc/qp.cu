// Persistent ADMM solver for batches of LTV-QPs (Sec. IV-A) and its C ABI
// (include/gpusls.h).  Host code owns the workspace; one cluster launch solves
// every QP of a handle.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/gpusls.h"
#include "internal.h"
#include "qp_iter.cuh"

namespace gsls {

// The solve kernel lives in qp_kernel_f32.cu / qp_kernel_f64.cu.
template <typename T>
const void* qp_kernel_entry();
template <> const void* qp_kernel_entry<float>();
template <> const void* qp_kernel_entry<double>();
using QPKernelFn = void (*)(const QPDesc*, SolveArgs);

// ---------------------------------------------------------------------------
// launch order for the next solve: longest expected first
// ---------------------------------------------------------------------------
// Expected work of QP b = its last solve's iterations + 180 per factorization
// (a 61D factorization costs about as much as 180 iterations); order[r] = b
// for the rank r of b in decreasing work (ties by index), by counting.
__global__ void order_kernel(const int* __restrict__ info_i, int batch, int* __restrict__ order) {
  __shared__ int work[1024];
  for (int b0 = 0; b0 < batch; b0 += blockDim.x) {            // same trip count in every thread
    const int b = b0 + threadIdx.x;
    const bool valid = b < batch;
    const int wb = valid ? info_i[8 * b + 1] + 180 * info_i[8 * b + 2] : 0;
    int rank = 0;
    for (int j0 = 0; j0 < batch; j0 += 1024) {
      const int nj = min(1024, batch - j0);
      __syncthreads();
      for (int j = threadIdx.x; j < nj; j += blockDim.x)
        work[j] = info_i[8 * (j0 + j) + 1] + 180 * info_i[8 * (j0 + j) + 2];
      __syncthreads();
      if (valid)
        for (int j = 0; j < nj; ++j) {
          const int wj = work[j];
          rank += (wj > wb || (wj == wb && j0 + j < b)) ? 1 : 0;
        }
    }
    if (valid) order[rank] = b;
  }
}

// ---------------------------------------------------------------------------
// packing FP64 caller arrays into padded solve-precision layouts
// ---------------------------------------------------------------------------


template <typename T>
__global__ void pack_kernel(const PackJob* __restrict__ jobs) {
  const PackJob j = jobs[blockIdx.y];
  const size_t total = (size_t)j.count * j.rows * j.ld;
  T* dst = reinterpret_cast<T*>(j.dst);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t rowi = e / j.ld;
    const int col = (int)(e - rowi * j.ld);
    T v = T(0);
    if (col < j.cols && j.src) v = (T)j.src[rowi * j.cols + col];
    dst[e] = v;
  }
}

}  // namespace gsls

// ===========================================================================
// host side
// ===========================================================================
using namespace gsls;

static thread_local std::string g_err;
static int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}
int gsls::set_error(int code, const std::string& msg) { return fail(code, msg); }
// On a failing runtime call the error is also cleared (cudaGetLastError), so
// that it is not reported again by a later, unrelated call.
#define CU(x)                                                                                \
  do {                                                                                       \
    cudaError_t e_ = (x);                                                                    \
    if (e_ != cudaSuccess) {                                                                 \
      (void)cudaGetLastError();                                                              \
      return fail(GPUSLS_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_));         \
    }                                                                                        \
  } while (0)

static size_t al64(size_t x) { return (x + 63) & ~(size_t)63; }

extern "C" void qp_default_settings(qp_settings* s) {
  s->rho0 = 0.1;
  s->eps = 1e-4;
  s->eps_kkt = 1e-4;
  s->rho_min = 1e-6;
  s->rho_max = 1e6;
  s->sigma = 25;
  s->check_every = 5;
  s->max_iter = 4000;
  s->precision = GPUSLS_FP64;
  s->cluster = 0;
  s->fixed_iters = 0;
  s->max_refine = 3;
  s->fallback_iters = 0;
  s->eps_floor = 0.0;   // auto: 1e-7 for FP64 solves, 1e-5 for FP32 solves
  s->occupancy = 0;
  s->schedule = 0;
  s->factorization = 0;
}

extern "C" const char* gpusls_last_error(void) { return g_err.c_str(); }

static int auto_cluster(int N) {
  int cs = (N + 11) / 12;
  return std::max(1, std::min(MAXCS_PORTABLE, cs));
}

// Kernel attributes and launch configuration of a solve launch: one cluster
// of h->cs CTAs per QP; cluster sizes above 8 need the non-portable attribute.
template <typename T>
static cudaError_t prepare_launch(qp_handle* h, cudaLaunchConfig_t* cfg, cudaLaunchAttribute* attr) {
  const void* kern = qp_kernel_entry<T>();
  int smem = h->smem;
  // occupancy 1: ask for more than half of the SM's shared memory, so that
  // exactly one CTA of this kernel fits an SM
  if (h->set.occupancy == 1) smem = std::max(smem, 116 * 1024);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess && h->cs > MAXCS_PORTABLE)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  *cfg = {};
  cfg->gridDim = dim3(h->batch * h->cs, 1, 1);
  cfg->blockDim = dim3(NT, 1, 1);
  cfg->dynamicSmemBytes = smem;
  cfg->stream = h->stream;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = h->cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg->attrs = attr;
  cfg->numAttrs = 1;
  return e;
}

// Clusters of this handle's launch shape the device can hold at once (0: the
// shape cannot be scheduled, e.g. a non-portable cluster size the device does
// not offer at this shared-memory size).
template <typename T>
static int max_active_clusters(qp_handle* h) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  int n = 0;
  if (prepare_launch<T>(h, &cfg, attr) != cudaSuccess ||
      cudaOccupancyMaxActiveClusters(&n, qp_kernel_entry<T>(), &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <typename T>
static int launch_qp(qp_handle* h, const SolveArgs& a) {
  const QPKernelFn kern = reinterpret_cast<QPKernelFn>(const_cast<void*>(qp_kernel_entry<T>()));
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  CU(prepare_launch<T>(h, &cfg, attr));
  CU(cudaLaunchKernelEx(&cfg, kern, (const QPDesc*)h->ddesc, a));
  CU(cudaGetLastError());
  return GPUSLS_OK;
}

// Debug aid: GPUSLS_PROFILE=1 accumulates per-phase cycle counts of every CTA
// of QP 0 and prints them to stderr after each launch.
static int launch(qp_handle* h, const SolveArgs& a0) {
  SolveArgs a = a0;
  a.tc = h->set.precision == GPUSLS_TF32 ? 1 : (h->set.precision == GPUSLS_MIXED ? 2 : 0);
  // test hook of the bounded device waits (see include/gpusls.h)
  a.test_wait = getenv("GPUSLS_TEST_WAIT_TIMEOUT") != nullptr ? 1 : 0;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CU(cudaStreamIsCapturing(h->stream, &cap));
  const bool prof_on = getenv("GPUSLS_PROFILE") != nullptr && cap == cudaStreamCaptureStatusNone;
  unsigned long long* dprof = nullptr;
  const int nprof = MAXCS * PH_COUNT;
  if (prof_on) {
    CU(cudaMalloc(&dprof, nprof * sizeof(unsigned long long)));
    CU(cudaMemsetAsync(dprof, 0, nprof * sizeof(unsigned long long), h->stream));
    a.prof = dprof;
  }
  const int st = h->esz == 8 ? launch_qp<double>(h, a) : launch_qp<float>(h, a);
  if (prof_on) {
    unsigned long long hp[MAXCS * PH_COUNT];
    CU(cudaMemcpyAsync(hp, dprof, sizeof(hp), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    cudaFree(dprof);
    static const char* names[PH_COUNT] = {"P1", "bwd", "sync1", "P3", "fwd", "sync2", "P5", "check", "rho",
                                          "R1", "R2", "R3", "R4", "R5", "R6", "kkt", "ringwait(incl)", "kkt:stages(incl)",
                                          "kkt:sync(incl)", "kkt:costate(incl)", "fA:gamma", "fA:xhc", "fA:ap",
                                          "fC:gamma", "fC:xk", "fC:p", "fC:out", "fC:bundles"};
    for (int r = 0; r < MAXCS; ++r) {
      unsigned long long tot = 0;
      for (int k = 0; k < PH_COUNT; ++k) tot += hp[r * PH_COUNT + k];
      if (!tot) continue;
      fprintf(stderr, "[gpusls prof cycles rank %d]", r);
      for (int k = 0; k < PH_COUNT; ++k) fprintf(stderr, " %s=%llu", names[k], hp[r * PH_COUNT + k]);
      fprintf(stderr, "\n");
    }
  }
  return st;
}

static int run_pack(qp_handle* h, const std::vector<PackJob>& jobs) {
  if (jobs.empty()) return GPUSLS_OK;
  if (jobs.size() > h->njobs_cap) {
    if (h->djobs) cudaFree(h->djobs);
    CU(cudaMalloc(&h->djobs, jobs.size() * sizeof(PackJob)));
    h->njobs_cap = jobs.size();
  }
  CU(cudaMemcpyAsync(h->djobs, jobs.data(), jobs.size() * sizeof(PackJob), cudaMemcpyHostToDevice, h->stream));
  for (size_t j0 = 0; j0 < jobs.size(); j0 += 60000) {
    const int nj = (int)std::min<size_t>(60000, jobs.size() - j0);
    dim3 grid(32, nj);
    if (h->esz == 8) pack_kernel<double><<<grid, 256, 0, h->stream>>>(h->djobs + j0);
    else pack_kernel<float><<<grid, 256, 0, h->stream>>>(h->djobs + j0);
    CU(cudaGetLastError());
  }
  // the jobs buffer is reused by later calls: keep the upload ordered
  CU(cudaStreamSynchronize(h->stream));
  return GPUSLS_OK;
}

// Dynamic shared memory a CTA of the solve kernel may request: the device's
// opt-in maximum per block less the kernel's static shared memory.
static int smem_limit(int esz) {
  int dev = 0, optin = 227 * 1024;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa = {};
  const cudaError_t e = esz == 8 ? cudaFuncGetAttributes(&fa, qp_kernel_entry<double>())
                                 : cudaFuncGetAttributes(&fa, qp_kernel_entry<float>());
  (void)cudaGetLastError();
  const int stat = e == cudaSuccess ? (int)fa.sharedSizeBytes : 4096;
  return std::min(optin, 227 * 1024) - stat;
}

// Per-QP launch-shape plan for cluster size cs: chunk length and count, ring
// slot, factorization schedule (blocked unless asked for the tree, in TF32,
// or its buffers do not fit), ring depth, and the shared memory per CTA.
struct ShapePlan {
  int Lc, nch, slot, fact, depth, smem, vg, vbytes;
};
static ShapePlan plan_shape(const qp_dims& d, int cs, int esz, const qp_settings* s, int lim) {
  ShapePlan p;
  const int ldx = rup4(d.nx), ldu = rup4(d.nu), ldc = rup4(std::max(1, d.nc));
  const int ldv = rup4(d.nx + d.nc), ldf = rup4(d.nx + d.nu);
  const int msz = d.nx * ldx;
  int bws, fws, cds;
  bundle_sizes(d.nx, d.nu, d.nc, ldx, ldu, ldv, ldf, &bws, &fws, &cds);
  p.Lc = (d.N + cs - 1) / cs;
  p.nch = (d.N + p.Lc - 1) / p.Lc;
  p.slot = std::max(std::max(std::max(bws, fws), msz), std::max(std::max(d.nx * ldu, d.nx * ldc), cds));
  p.vg = 0;
  auto lay_total = [&](int depth, int fact) {
    return smem_layout(d.nx, d.nu, d.nc, d.nf, p.Lc, p.nch, cs, ldx, ldu, ldv, ldf, depth, p.slot, esz, fact, p.vg)
        .total;
  };
  // long horizons: when even the smallest layout (tree, ring depth 2) cannot
  // hold the per-chunk vectors, they move to a per-CTA global region
  if (lay_total(2, 1) > lim) p.vg = 1;
  p.fact = (s->factorization == 1 || s->precision == GPUSLS_TF32 || d.nu > FACT_MAX_NU) ? 1 : 0;
  if (p.fact == 0 && lay_total(1, 0) > lim) p.fact = 1;
  p.depth = lay_total(3, p.fact) > lim ? 2 : 3;
  p.smem = lay_total(p.depth, p.fact);
  p.vbytes =
      smem_layout(d.nx, d.nu, d.nc, d.nf, p.Lc, p.nch, cs, ldx, ldu, ldv, ldf, p.depth, p.slot, esz, p.fact, p.vg)
          .vbytes;
  return p;
}

static bool dims_ok(const qp_dims& d) {
  return d.nx >= 1 && d.nx <= TILE && d.nu >= 1 && d.nu <= 32 && d.nc >= 0 && d.nc <= 64 && d.nf >= 0 &&
         d.nf <= 64 && d.N >= 1 && d.N <= GPUSLS_MAX_N;
}

extern "C" int qp_batch_setup(qp_handle** out, int32_t batch, const qp_dims* dims, const double* A, const double* B,
                              const double* c, const double* Q, const double* R, const double* S, const double* q,
                              const double* r, const double* C, const double* D, const double* CN, const double* lo,
                              const double* hi, const double* rho, const qp_settings* s, void* stream) {
  gsls::NvtxRange nvtx_("gpusls/qp_batch_setup");
  if (!out || batch < 1 || !dims || !A || !B || !c || !Q || !R || !q || !r || !lo || !hi || !s)
    return fail(GPUSLS_ERR_INVALID, "qp_batch_setup: null argument or batch < 1");
  if (s->precision != GPUSLS_FP64 && s->precision != GPUSLS_FP32 && s->precision != GPUSLS_TF32 &&
      s->precision != GPUSLS_MIXED)
    return fail(GPUSLS_ERR_INVALID, "qp_batch_setup: unknown precision");
  if (s->cluster < 0 || s->cluster > MAXCS) return fail(GPUSLS_ERR_INVALID, "qp_batch_setup: cluster must be 0..16");
  if (s->occupancy < 0 || s->occupancy > 1 || s->schedule < 0 || s->schedule > 1 || s->factorization < 0 ||
      s->factorization > 1)
    return fail(GPUSLS_ERR_INVALID, "qp_batch_setup: occupancy, schedule and factorization must be 0 or 1");
  if (s->check_every < 1 || s->max_iter < 1 || s->sigma < 0)
    return fail(GPUSLS_ERR_INVALID, "qp_batch_setup: check_every, max_iter >= 1 and sigma >= 0 required");
  int needC = 0, needCN = 0;
  for (int b = 0; b < batch; ++b) {
    if (!dims_ok(dims[b])) return fail(GPUSLS_ERR_INVALID, "qp_batch_setup: dims out of range for QP " + std::to_string(b));
    needC |= dims[b].nc > 0;
    needCN |= dims[b].nf > 0;
  }
  if ((needC && (!C || !D)) || (needCN && !CN)) return fail(GPUSLS_ERR_INVALID, "qp_batch_setup: C/D/CN missing");

  qp_handle* h = new qp_handle();
  h->batch = batch;
  h->dims.assign(dims, dims + batch);
  h->set = *s;
  h->stream = (cudaStream_t)stream;
  h->esz = s->precision == GPUSLS_FP64 ? 8 : 4;
  int cs = s->cluster;
  if (cs == 0) {
    int Nmax = 1;
    for (auto& d : h->dims) Nmax = std::max(Nmax, d.N);
    cs = auto_cluster(Nmax);
  }
  h->cs = cs;

  // caller pool offsets
  h->off.resize(batch);
  QPOffsets o = {};
  for (int b = 0; b < batch; ++b) {
    const qp_dims& d = dims[b];
    h->off[b] = o;
    const size_t nx = d.nx, nu = d.nu, N = d.N, nc = d.nc, nf = d.nf, m = N * nc + nf;
    o.A += N * nx * nx; o.B += N * nx * nu; o.c += N * nx; o.Q += (N + 1) * nx * nx; o.R += N * nu * nu;
    o.S += N * nu * nx; o.q += (N + 1) * nx; o.r += N * nu; o.C += N * nc * nx; o.D += N * nc * nu;
    o.CN += nf * nx; o.lohi += m; o.x0 += nx; o.dx += (N + 1) * nx; o.du += N * nu; o.P += (N + 1) * nx * nx;
    o.K += N * nu * nx;
  }
  const QPOffsets tot = o;

  // workspace sizes
  const int esz = h->esz;
  const int lim = smem_limit(esz);
  // automatic launch shape for long horizons: when the per-chunk vectors of
  // 8-CTA clusters need the global-memory region, clusters of 16 CTAs (a
  // non-portable size) halve the chunk chains, if the device schedules them
  if (s->cluster == 0 && cs == MAXCS_PORTABLE) {
    bool vg8 = false;
    int smem16 = 0;
    for (int b = 0; b < batch; ++b) {
      vg8 = vg8 || plan_shape(dims[b], cs, esz, s, lim).vg != 0;
      smem16 = std::max(smem16, plan_shape(dims[b], MAXCS, esz, s, lim).smem);
    }
    if (vg8 && smem16 <= lim) {
      h->cs = MAXCS;
      h->smem = smem16;
      if ((esz == 8 ? max_active_clusters<double>(h) : max_active_clusters<float>(h)) >= 1) cs = MAXCS;
      h->cs = cs;
    }
  }
  std::vector<size_t> toff(batch), doff(batch);
  size_t tsz = 0, dsz = 0;
  int smem = 0;
  h->hdesc.resize(batch);
  struct Sizes {
    size_t A, B, b, Q, R, S, q, r, C, D, CN, lo, hi, x0, Rhi, Sh, Rh, S0, V, scr, Abar, CK, F, FPi, J, K, KSig, CKSig, Sig,
        c0, k0, CNSig, SigN, Tch, Uch, Theta, Xi, Gam, z, y, BW, FW, CD, vec;
  };
  std::vector<ShapePlan> plans(batch);
  std::vector<Sizes> sz(batch);
  for (int b = 0; b < batch; ++b) {
    const qp_dims& d = dims[b];
    const size_t nx = d.nx, nu = d.nu, N = d.N, nc = d.nc, nf = d.nf, m = N * nc + nf;
    const size_t ldx = rup4(d.nx), ldu = rup4(d.nu), ldc = rup4(std::max(1, d.nc));
    const size_t msz = nx * ldx;
    const int n = d.N + 1;
    int nlev = 0;
    while ((1 << nlev) < n) ++nlev;
    size_t nodes = 0;
    for (int lv = 0; lv <= nlev; ++lv) nodes += (n + (1 << lv) - 1) >> lv;
    Sizes& z = sz[b];
    z.A = al64(N * msz); z.B = al64(N * nx * ldu); z.b = al64(N * ldx); z.Q = al64((N + 1) * msz);
    z.R = al64(N * nu * ldu); z.S = al64(N * nu * ldx); z.q = al64((N + 1) * ldx); z.r = al64(N * ldu);
    z.C = al64(N * nc * ldx + 1); z.D = al64(N * nc * ldu + 1); z.CN = al64(nf * ldx + 1); z.lo = al64(m + 1);
    z.hi = al64(m + 1); z.x0 = al64(ldx); z.Rhi = al64(N * nu * ldu); z.Sh = al64(N * nu * ldx);
    z.Rh = al64(N * nu * ldu); z.S0 = al64(N * nu * ldx);
    plans[b] = plan_shape(d, cs, esz, s, lim);
    const size_t nch = plans[b].nch;
    z.V = al64(nodes * msz); z.scr = al64((size_t)cs * 6 * msz); z.Abar = al64(N * msz);
    z.CK = al64(N * nc * ldx + 1); z.F = al64(N * nu * ldx); z.FPi = al64(N * nx * ldu); z.J = al64(N * nu * ldc);
    z.K = al64(N * nu * ldx); z.KSig = al64(N * nu * ldx); z.CKSig = al64(N * nx * ldc + 1); z.Sig = al64(N * msz);
    z.c0 = al64(N * ldx); z.k0 = al64(N * ldu); z.CNSig = al64(nf * ldx + 1); z.SigN = al64(msz);
    z.Tch = al64(cs * msz); z.Uch = al64(cs * msz); z.Theta = al64(nch * nch * msz);
    z.Xi = al64(nch * nch * msz); z.Gam = al64(N * nu * ldu); z.z = al64(m + 1); z.y = al64(m + 1);
    const int ldv = rup4(d.nx + d.nc), ldf = rup4(d.nx + d.nu);
    int bws, fws, cds;
    bundle_sizes(d.nx, d.nu, d.nc, (int)ldx, (int)ldu, ldv, ldf, &bws, &fws, &cds);
    z.BW = al64(N * (size_t)bws); z.FW = al64(N * (size_t)fws); z.CD = al64(N * (size_t)cds + 1);
    z.vec = plans[b].vg ? al64((size_t)cs * plans[b].vbytes / esz) : 0;
    toff[b] = tsz;
    tsz += z.A + z.B + z.b + z.Q + z.R + z.S + z.q + z.r + z.C + z.D + z.CN + z.lo + z.hi + z.x0 + z.Rhi + z.Sh +
           z.Rh + z.S0 + 4 * z.V + z.scr + z.Abar + z.CK + z.F + z.FPi + z.J + z.K + z.KSig + z.CKSig + z.Sig + z.c0 + z.k0 +
           z.CNSig + z.SigN + z.Tch + z.Uch + z.Theta + z.Xi + z.Gam + z.z + z.y + z.BW + z.FW + z.CD + z.vec;
    doff[b] = dsz;
    dsz += al64((N + 1) * nx) + al64(N * nu) + 64;   // kg, kh, rho/flags slot
    // per-QP descriptor (pointers filled after allocation)
    QPDesc& D_ = h->hdesc[b];
    memset(&D_, 0, sizeof(D_));
    D_.nx = d.nx; D_.nu = d.nu; D_.N = d.N; D_.nc = d.nc; D_.nf = d.nf; D_.m = (int)m;
    D_.ldx = (int)ldx; D_.ldu = (int)ldu; D_.ldc = (int)ldc;
    const ShapePlan& sp = plans[b];
    D_.vg = sp.vg;
    D_.vstride = sp.vbytes;
    D_.Lc = sp.Lc;
    D_.nch = sp.nch;
    D_.nlev = nlev;
    D_.ldv = ldv;
    D_.ldf = ldf;
    D_.slot = sp.slot;
    D_.fact = sp.fact;
    D_.depth = sp.depth;
    smem = std::max(smem, sp.smem);
  }
  h->smem = smem;
  if (smem > lim) {
    delete h;
    return fail(GPUSLS_ERR_INVALID, "qp_batch_setup: shared memory per CTA (" + std::to_string(smem) +
                                        " B) exceeds the device's " + std::to_string(lim) +
                                        " B for this kernel (smaller nx, nc or nf)");
  }
  if (cs > MAXCS_PORTABLE && (esz == 8 ? max_active_clusters<double>(h) : max_active_clusters<float>(h)) < 1) {
    delete h;
    return fail(GPUSLS_ERR_INVALID, "qp_batch_setup: the device cannot schedule clusters of " + std::to_string(cs) +
                                        " CTAs with " + std::to_string(smem) + " B of shared memory each");
  }
  // FP64 copies of the caller's arrays live in dpool after the per-QP scratch
  const size_t d_copy = tot.A + tot.B + tot.c + tot.Q + tot.R + tot.S + tot.q + tot.r + tot.C + tot.D + tot.CN +
                        2 * tot.lohi + tot.x0 + 64;
  cudaError_t e1 = cudaMalloc(&h->tpool, tsz * esz + 256);
  cudaError_t e2 = cudaMalloc(&h->dpool, (dsz + d_copy) * sizeof(double) + 256);
  cudaError_t e3 = cudaMalloc(&h->ddesc, batch * sizeof(QPDesc));
  cudaError_t e4 = cudaMalloc(&h->info_i, batch * 8 * sizeof(int));
  cudaError_t e5 = cudaMalloc(&h->info_d, batch * 4 * sizeof(double));
  if (e1 || e2 || e3 || e4 || e5) {
    qp_destroy(h);
    return fail(GPUSLS_ERR_CUDA, "qp_batch_setup: cudaMalloc failed");
  }
  // FP64 copies
  double* dc = h->dpool + dsz;
  double *A64 = dc, *B64 = A64 + tot.A, *b64 = B64 + tot.B, *Q64 = b64 + tot.c, *R64 = Q64 + tot.Q,
         *S64 = R64 + tot.R, *q64 = S64 + tot.S, *r64 = q64 + tot.q, *C64 = r64 + tot.r, *D64 = C64 + tot.C,
         *CN64 = D64 + tot.D, *lo64 = CN64 + tot.CN, *hi64 = lo64 + tot.lohi, *x064 = hi64 + tot.lohi;
  auto cp = [&](double* dst, const double* src, size_t n) -> cudaError_t {
    if (n == 0) return cudaSuccess;
    if (!src) return cudaMemsetAsync(dst, 0, n * sizeof(double), h->stream);
    return cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
  };
  CU(cp(A64, A, tot.A)); CU(cp(B64, B, tot.B)); CU(cp(b64, c, tot.c)); CU(cp(Q64, Q, tot.Q)); CU(cp(R64, R, tot.R));
  CU(cp(S64, S, tot.S)); CU(cp(q64, q, tot.q)); CU(cp(r64, r, tot.r)); CU(cp(C64, C, tot.C)); CU(cp(D64, D, tot.D));
  CU(cp(CN64, CN, tot.CN)); CU(cp(lo64, lo, tot.lohi)); CU(cp(hi64, hi, tot.lohi));
  CU(cudaMemsetAsync(x064, 0, tot.x0 * sizeof(double), h->stream));

  std::vector<PackJob> jobs;
  char* tp = (char*)h->tpool;
  h->tx0.resize(batch);
  for (int b = 0; b < batch; ++b) {
    const qp_dims& d = dims[b];
    const Sizes& z = sz[b];
    QPDesc& D_ = h->hdesc[b];
    const QPOffsets& po = h->off[b];
    char* p = tp + toff[b] * esz;
    auto take = [&](size_t n) { void* r_ = p; p += n * esz; return r_; };
    D_.A = take(z.A); D_.B = take(z.B); D_.b = take(z.b); D_.Q = take(z.Q); D_.R = take(z.R); D_.S = take(z.S);
    D_.q = take(z.q); D_.r = take(z.r); D_.C = take(z.C); D_.D = take(z.D); D_.CN = take(z.CN); D_.lo = take(z.lo);
    D_.hi = take(z.hi); D_.x0 = take(z.x0); D_.Rhi = take(z.Rhi); D_.Sh = take(z.Sh); D_.Rh = take(z.Rh);
    D_.S0 = take(z.S0); D_.VP = take(z.V);
    D_.VA = take(z.V); D_.VC = take(z.V); D_.IP = take(z.V); D_.scr = take(z.scr); D_.Abar = take(z.Abar);
    D_.CK = take(z.CK); D_.F = take(z.F); D_.FPi = take(z.FPi); D_.J = take(z.J); D_.K = take(z.K);
    D_.KSig = take(z.KSig); D_.CKSig = take(z.CKSig); D_.Sig = take(z.Sig); D_.c0 = take(z.c0); D_.k0 = take(z.k0);
    D_.CNSig = take(z.CNSig); D_.SigN = take(z.SigN); D_.Tch = take(z.Tch); D_.Uch = take(z.Uch);
    D_.Theta = take(z.Theta); D_.Xi = take(z.Xi); D_.Gam = take(z.Gam); D_.z = take(z.z); D_.y = take(z.y);
    D_.BW = take(z.BW); D_.FW = take(z.FW); D_.CD = take(z.CD);
    D_.vec = z.vec ? take(z.vec) : nullptr;
    h->tx0[b] = D_.x0;
    D_.A64 = A64 + po.A; D_.B64 = B64 + po.B; D_.b64 = b64 + po.c; D_.Q64 = Q64 + po.Q; D_.R64 = R64 + po.R;
    D_.S64 = S64 + po.S; D_.q64 = q64 + po.q; D_.r64 = r64 + po.r; D_.C64 = C64 + po.C; D_.D64 = D64 + po.D;
    D_.CN64 = CN64 + po.CN; D_.lo64 = lo64 + po.lohi; D_.hi64 = hi64 + po.lohi; D_.x064 = x064 + po.x0;
    double* dp = h->dpool + doff[b];
    D_.kg = dp;
    D_.kh = dp + al64((size_t)(d.N + 1) * d.nx);
    D_.rho = D_.kh + al64((size_t)d.N * d.nu);
    D_.flags = reinterpret_cast<int*>(D_.rho + 8);
    D_.info_i = h->info_i + 8 * b;
    D_.info_d = h->info_d + 4 * b;
    const int nx = d.nx, nu = d.nu, N = d.N, nc = d.nc, nf = d.nf, m = N * nc + nf;
    const int ldx = D_.ldx, ldu = D_.ldu;
    jobs.push_back({A + po.A, D_.A, N, nx, nx, ldx});
    jobs.push_back({B + po.B, D_.B, N, nx, nu, ldu});
    jobs.push_back({c + po.c, D_.b, N, 1, nx, ldx});
    jobs.push_back({Q + po.Q, D_.Q, N + 1, nx, nx, ldx});
    jobs.push_back({R + po.R, D_.R, N, nu, nu, ldu});
    jobs.push_back({S ? S + po.S : nullptr, D_.S, N, nu, nx, ldx});
    jobs.push_back({q + po.q, D_.q, N + 1, 1, nx, ldx});
    jobs.push_back({r + po.r, D_.r, N, 1, nu, ldu});
    if (nc) {
      jobs.push_back({C + po.C, D_.C, N, nc, nx, ldx});
      jobs.push_back({D + po.D, D_.D, N, nc, nu, ldu});
    }
    if (nf) jobs.push_back({CN + po.CN, D_.CN, 1, nf, nx, ldx});
    if (m) {
      jobs.push_back({lo + po.lohi, D_.lo, 1, 1, m, m});
      jobs.push_back({hi + po.lohi, D_.hi, 1, 1, m, m});
      jobs.push_back({nullptr, D_.z, 1, 1, m, m});
      jobs.push_back({nullptr, D_.y, 1, 1, m, m});
    }
  }
  int st = run_pack(h, jobs);
  if (st) { qp_destroy(h); return st; }
  // rho and flags
  std::vector<double> r0(batch);
  for (int b = 0; b < batch; ++b) r0[b] = (rho && rho[b] > 0) ? rho[b] : s->rho0;
  if (cudaMalloc(&h->rho0_dev, batch * sizeof(double)) != cudaSuccess) {
    qp_destroy(h);
    return fail(GPUSLS_ERR_CUDA, "qp_batch_setup: cudaMalloc failed");
  }
  CU(cudaMemcpyAsync(h->rho0_dev, r0.data(), batch * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  for (int b = 0; b < batch; ++b) h->hdesc[b].rho0 = h->rho0_dev + b;
  // launch order: index order until a solve has run (schedule 1)
  std::vector<int> ord(batch);
  for (int b = 0; b < batch; ++b) ord[b] = b;
  if (cudaMalloc(&h->order_dev, batch * sizeof(int)) != cudaSuccess) {
    qp_destroy(h);
    return fail(GPUSLS_ERR_CUDA, "qp_batch_setup: cudaMalloc failed");
  }
  CU(cudaMemcpy(h->order_dev, ord.data(), batch * sizeof(int), cudaMemcpyHostToDevice));
  for (int b = 0; b < batch; ++b) {
    int fl[4] = {0, 0, 0, 0};
    CU(cudaMemcpyAsync(h->hdesc[b].rho, &r0[b], sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(h->hdesc[b].flags, fl, sizeof(fl), cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));
  }
  CU(cudaMemcpyAsync(h->ddesc, h->hdesc.data(), batch * sizeof(QPDesc), cudaMemcpyHostToDevice, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  *out = h;
  return GPUSLS_OK;
}

extern "C" int qp_setup(qp_handle** h, qp_dims d, const double* A, const double* B, const double* c, const double* Q,
                        const double* R, const double* S, const double* q, const double* r, const double* C,
                        const double* D, const double* CN, const double* lo, const double* hi, double rho,
                        const qp_settings* s, void* stream) {
  qp_settings def;
  if (!s) {
    qp_default_settings(&def);
    s = &def;
  }
  double rv = rho;
  return qp_batch_setup(h, 1, &d, A, B, c, Q, R, S, q, r, C, D, CN, lo, hi, rho > 0 ? &rv : nullptr, s, stream);
}

// Set the output pointers (caller pools) of every descriptor and upload.
static int set_outputs(qp_handle* h, double* ox, double* ou, double* olam, size_t stride_x, size_t stride_u,
                       bool riccati) {
  for (int b = 0; b < h->batch; ++b) {
    const QPOffsets& po = h->off[b];
    h->hdesc[b].ox = ox ? ox + (riccati ? po.P : po.dx) : nullptr;
    h->hdesc[b].ou = ou ? ou + (riccati ? po.K : po.du) : nullptr;
    h->hdesc[b].olam = olam ? olam + po.lohi : nullptr;
  }
  (void)stride_x;
  (void)stride_u;
  CU(cudaMemcpyAsync(h->ddesc, h->hdesc.data(), h->batch * sizeof(QPDesc), cudaMemcpyHostToDevice, h->stream));
  return GPUSLS_OK;
}

static int set_x0(qp_handle* h, const double* x0) {
  std::vector<PackJob> jobs;
  size_t tot = 0;
  for (int b = 0; b < h->batch; ++b) {
    jobs.push_back({x0 + h->off[b].x0, h->tx0[b], 1, 1, h->dims[b].nx, h->hdesc[b].ldx});
    tot += h->dims[b].nx;
  }
  // FP64 copy (pool layout matches the caller's x0 pool)
  CU(cudaMemcpyAsync(h->hdesc[0].x064, x0, tot * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  return run_pack(h, jobs);
}

static int collect(qp_handle* h, qp_info* info) {
  std::vector<int> ii(h->batch * 8);
  std::vector<double> dd(h->batch * 4);
  CU(cudaMemcpyAsync(ii.data(), h->info_i, ii.size() * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaMemcpyAsync(dd.data(), h->info_d, dd.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  int worst = GPUSLS_OK;
  for (int b = 0; b < h->batch; ++b) {
    const int st = ii[8 * b];
    if (info) {
      info[b].status = st;
      info[b].iters = ii[8 * b + 1];
      info[b].refactors = ii[8 * b + 2];
      info[b].refines = ii[8 * b + 3];
      info[b].fallback = ii[8 * b + 4];
      info[b].pad = 0;
      info[b].rho = dd[4 * b];
      info[b].r_prim = dd[4 * b + 1];
      info[b].r_dual = dd[4 * b + 2];
      info[b].kkt = dd[4 * b + 3];
    }
    // an infeasible QP is a result (info[b].status), not a failed call: it
    // counts as not converged
    if (st < 0 && st != GPUSLS_ERR_INFEASIBLE && (worst >= 0 || st < worst)) worst = st;
    else if ((st == GPUSLS_MAX_ITER || st == GPUSLS_ERR_INFEASIBLE) && worst == GPUSLS_OK) worst = GPUSLS_MAX_ITER;
  }
  return worst;
}

static SolveArgs solve_args(const qp_handle* h, int32_t iters, double tol) {
  SolveArgs a = {};
  a.mode = MODE_SOLVE;
  a.max_iter = iters > 0 ? iters : h->set.max_iter;
  a.fixed_iters = h->set.fixed_iters;
  a.sigma = h->set.sigma;
  a.check_every = h->set.check_every;
  a.cs = h->cs;
  a.eps = tol > 0 ? tol : h->set.eps;
  a.eps_kkt = h->set.eps_kkt > 0 ? (tol > 0 ? tol : h->set.eps_kkt) : -1.0;
  a.rho_min = h->set.rho_min;
  a.rho_max = h->set.rho_max;
  a.eps_floor = h->set.eps_floor > 0.0 ? h->set.eps_floor : (h->esz == 4 ? 1e-5 : 1e-7);
  a.max_refine = h->set.max_refine;
  a.fallback_iters = h->set.fallback_iters;
  a.order = h->set.schedule == 1 ? h->order_dev : nullptr;
  return a;
}

// The solve launch, followed (schedule 1) by the launch order of the next solve.
static int launch_solve(qp_handle* h, const SolveArgs& a) {
  int st = launch(h, a);
  if (st) return st;
  if (h->set.schedule == 1) {
    order_kernel<<<1, 256, 0, h->stream>>>(h->info_i, h->batch, h->order_dev);
    CU(cudaGetLastError());
  }
  return GPUSLS_OK;
}

extern "C" int qp_solve(qp_handle* h, const double* x0, int32_t iters, double tol, double* dx, double* du,
                        double* lam, qp_info* info) {
  gsls::NvtxRange nvtx_("gpusls/qp_solve");
  if (!h || !x0 || !dx || !du || !lam) return fail(GPUSLS_ERR_INVALID, "qp_solve: null argument");
  int st = set_x0(h, x0);
  if (st) return st;
  st = set_outputs(h, dx, du, lam, 0, 0, false);
  if (st) return st;
  st = launch_solve(h, solve_args(h, iters, tol));
  if (st) return st;
  return collect(h, info);
}

// ---------------------------------------------------------------------------
// serving graph
// ---------------------------------------------------------------------------
// qp_update: mark every QP's factorization stale (flags[0]) and its state
// as not warm-started (flags[1]).
__global__ void flags_clear_kernel(const QPDesc* __restrict__ descs, int batch) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < batch) {
    descs[b].flags[0] = 0;
    descs[b].flags[1] = 0;
  }
}

template <typename T>
__global__ void reset_kernel(const QPDesc* __restrict__ descs, const double* __restrict__ rho0);

struct qp_graph {
  qp_handle* q = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  PackJob* djobs = nullptr;   // x0 pack jobs (uploaded once)
  int njobs = 0;
  std::vector<float*> feat;   // per-head feature buffers (qp_graph_create_heads)
};

extern "C" void qp_graph_destroy(qp_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->djobs) cudaFree(g->djobs);
  for (float* f : g->feat) cudaFree(f);
  if (g->cap) cudaStreamDestroy(g->cap);
  delete g;
}

// Captures reset -> warm(stream) -> x0 pack -> solve -> info copies.
template <typename Warm>
static int graph_create(qp_graph** out, qp_graph* g, qp_handle* h, Warm warm, const double* x0, double* dx,
                        double* du, double* lam, int32_t* info_i, double* info_d) {
  *out = nullptr;
  g->q = h;
  auto bail = [&](int code, const std::string& msg) {
    qp_graph_destroy(g);
    return fail(code, msg);
  };
  // outputs and x0 pack jobs are fixed for the graph's life: set them now
  int st = set_outputs(h, dx, du, lam, 0, 0, false);
  if (st) return bail(st, gpusls_last_error());
  std::vector<PackJob> jobs;
  size_t tot = 0;
  for (int b = 0; b < h->batch; ++b) {
    jobs.push_back({x0 + h->off[b].x0, h->tx0[b], 1, 1, h->dims[b].nx, h->hdesc[b].ldx});
    tot += h->dims[b].nx;
  }
  g->njobs = (int)jobs.size();
  if (cudaMalloc(&g->djobs, jobs.size() * sizeof(PackJob)) != cudaSuccess)
    return bail(GPUSLS_ERR_CUDA, "qp_graph_create: cudaMalloc failed");
  if (cudaMemcpy(g->djobs, jobs.data(), jobs.size() * sizeof(PackJob), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess)
    return bail(GPUSLS_ERR_CUDA, "qp_graph_create: upload failed");
  if (cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking) != cudaSuccess)
    return bail(GPUSLS_ERR_CUDA, "qp_graph_create: cudaStreamCreate failed");
  // the kernel attributes are set before capture
  {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    const cudaError_t e = h->esz == 8 ? prepare_launch<double>(h, &cfg, attr) : prepare_launch<float>(h, &cfg, attr);
    if (e != cudaSuccess) return bail(GPUSLS_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
  }
  const cudaStream_t saved = h->stream;
  h->stream = g->cap;
  if (cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    h->stream = saved;
    return bail(GPUSLS_ERR_CUDA, "qp_graph_create: cudaStreamBeginCapture failed");
  }
  int est = GPUSLS_OK;
  if (h->esz == 8) reset_kernel<double><<<h->batch, 256, 0, g->cap>>>(h->ddesc, h->rho0_dev);
  else reset_kernel<float><<<h->batch, 256, 0, g->cap>>>(h->ddesc, h->rho0_dev);
  est = warm(g->cap);
  if (!est && cudaMemcpyAsync(h->hdesc[0].x064, x0, tot * sizeof(double), cudaMemcpyDeviceToDevice, g->cap))
    est = GPUSLS_ERR_CUDA;
  if (!est) {
    dim3 grid(32, g->njobs);
    if (h->esz == 8) pack_kernel<double><<<grid, 256, 0, g->cap>>>(g->djobs);
    else pack_kernel<float><<<grid, 256, 0, g->cap>>>(g->djobs);
    est = launch_solve(h, solve_args(h, 0, 0.0));
  }
  if (!est && info_i &&
      cudaMemcpyAsync(info_i, h->info_i, (size_t)h->batch * 8 * sizeof(int), cudaMemcpyDeviceToDevice, g->cap))
    est = GPUSLS_ERR_CUDA;
  if (!est && info_d &&
      cudaMemcpyAsync(info_d, h->info_d, (size_t)h->batch * 4 * sizeof(double), cudaMemcpyDeviceToDevice, g->cap))
    est = GPUSLS_ERR_CUDA;
  const cudaError_t ee = cudaStreamEndCapture(g->cap, &g->graph);
  h->stream = saved;
  if (est) return bail(est, std::string("qp_graph_create: capture failed: ") + gpusls_last_error());
  if (ee != cudaSuccess) return bail(GPUSLS_ERR_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(ee));
  const cudaError_t ei = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (ei != cudaSuccess) return bail(GPUSLS_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei));
  *out = g;
  return GPUSLS_OK;
}

extern "C" int qp_graph_create(qp_graph** out, qp_handle* h, mlp_handle* m, const float* features, const double* x0,
                               double* dx, double* du, double* lam, int32_t* info_i, double* info_d,
                               double rho_min, double rho_max) {
  if (!out || !h || !x0 || !dx || !du || !lam || (m && !features))
    return fail(GPUSLS_ERR_INVALID, "qp_graph_create: null argument");
  qp_graph* g = new qp_graph();
  auto warm = [&](cudaStream_t st) -> int {
    return m ? gsls::mlp_enqueue_warm_start(h, m, features, rho_min, rho_max, st) : GPUSLS_OK;
  };
  return graph_create(out, g, h, warm, x0, dx, du, lam, info_i, info_d);
}

extern "C" int qp_graph_create_heads(qp_graph** out, qp_handle* h, int32_t n_heads, mlp_handle* const* heads,
                                     const int32_t* const* idx, const int32_t* counts, const int32_t* n_stage,
                                     const double* x0, double* dx, double* du, double* lam, int32_t* info_i,
                                     double* info_d, double rho_min, double rho_max) {
  if (!out || !h || !x0 || !dx || !du || !lam || n_heads < 1 || !heads || !idx || !counts || !n_stage)
    return fail(GPUSLS_ERR_INVALID, "qp_graph_create_heads: null argument");
  // the host-side checks of qp_warm_start_heads
  std::vector<int> smem(n_heads);
  for (int hh = 0; hh < n_heads; ++hh) {
    if (!heads[hh] || !idx[hh] || counts[hh] < 1) return fail(GPUSLS_ERR_INVALID, "qp_graph_create_heads: bad head");
    std::vector<int32_t> hidx(counts[hh]);
    if (cudaMemcpy(hidx.data(), idx[hh], counts[hh] * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(GPUSLS_ERR_CUDA, "qp_graph_create_heads: index copy failed");
    for (int i = 0; i < counts[hh]; ++i)
      if (hidx[i] < 0 || hidx[i] >= h->batch || h->dims[hidx[i]].N > n_stage[hh])
        return fail(GPUSLS_ERR_INVALID, "qp_graph_create_heads: QP index or horizon out of range");
    smem[hh] = gsls::features_smem(h, hidx.data(), counts[hh]);
  }
  qp_graph* g = new qp_graph();
  for (int hh = 0; hh < n_heads; ++hh) {
    float* f = nullptr;
    if (cudaMalloc(&f, (size_t)counts[hh] * gsls::mlp_n_in(heads[hh]) * sizeof(float)) != cudaSuccess) {
      qp_graph_destroy(g);
      return fail(GPUSLS_ERR_CUDA, "qp_graph_create_heads: cudaMalloc failed");
    }
    g->feat.push_back(f);
  }
  if (cudaFuncSetAttribute(gsls::qp_features_kernel_ptr(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                           *std::max_element(smem.begin(), smem.end())) != cudaSuccess) {
    qp_graph_destroy(g);
    return fail(GPUSLS_ERR_CUDA, "qp_graph_create_heads: cudaFuncSetAttribute failed");
  }
  auto warm = [&](cudaStream_t st) -> int {
    for (int hh = 0; hh < n_heads; ++hh) {
      const int e = gsls::enqueue_head(h, heads[hh], idx[hh], counts[hh], smem[hh], n_stage[hh], x0, g->feat[hh],
                                       rho_min, rho_max, st);
      if (e) return e;
    }
    return GPUSLS_OK;
  };
  return graph_create(out, g, h, warm, x0, dx, du, lam, info_i, info_d);
}

extern "C" int qp_graph_launch(qp_graph* g, void* stream) {
  gsls::NvtxRange nvtx_("gpusls/qp_graph_launch");
  if (!g || !g->exec) return fail(GPUSLS_ERR_INVALID, "qp_graph_launch: null graph");
  CU(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
  return GPUSLS_OK;
}

extern "C" int qp_graph_kernel_count(qp_graph* g, int32_t* n) {
  if (!g || !g->graph || !n) return fail(GPUSLS_ERR_INVALID, "qp_graph_kernel_count: null argument");
  size_t count = 0;
  CU(cudaGraphGetNodes(g->graph, nullptr, &count));
  std::vector<cudaGraphNode_t> nodes(count);
  if (count) CU(cudaGraphGetNodes(g->graph, nodes.data(), &count));
  int k = 0;
  for (size_t i = 0; i < count; ++i) {
    cudaGraphNodeType ty;
    CU(cudaGraphNodeGetType(nodes[i], &ty));
    if (ty == cudaGraphNodeTypeKernel) ++k;
  }
  *n = k;
  return GPUSLS_OK;
}

extern "C" int qp_riccati(qp_handle* h, double* P, double* K) {
  if (!h || !P || !K) return fail(GPUSLS_ERR_INVALID, "qp_riccati: null argument");
  int st = set_outputs(h, P, K, nullptr, 0, 0, true);
  if (st) return st;
  SolveArgs a = {};
  a.mode = MODE_RICCATI;
  a.cs = h->cs;
  st = launch(h, a);
  if (st) return st;
  return collect(h, nullptr);
}

int gsls::qp_refactor_internal(qp_handle* h, bool gains_only) {
  int st = set_outputs(h, nullptr, nullptr, nullptr, 0, 0, true);
  if (st) return st;
  SolveArgs a = {};
  a.mode = gains_only ? MODE_GAINS : MODE_RICCATI;
  a.cs = h->cs;
  st = launch(h, a);
  if (st) return st;
  return collect(h, nullptr);
}

extern "C" int qp_kkt(qp_handle* h, const double* x0, const double* dx, const double* du, const double* lam,
                      double* out) {
  gsls::NvtxRange nvtx_("gpusls/qp_kkt");
  if (!h || !x0 || !dx || !du || !lam || !out) return fail(GPUSLS_ERR_INVALID, "qp_kkt: null argument");
  int st = set_x0(h, x0);
  if (st) return st;
  st = set_outputs(h, const_cast<double*>(dx), const_cast<double*>(du), const_cast<double*>(lam), 0, 0, false);
  if (st) return st;
  SolveArgs a = {};
  a.mode = MODE_KKT;
  a.cs = h->cs;
  st = launch(h, a);
  if (st) return st;
  std::vector<qp_info> inf(h->batch);
  collect(h, inf.data());
  for (int b = 0; b < h->batch; ++b) out[b] = inf[b].kkt;
  return GPUSLS_OK;
}

// ---------------------------------------------------------------------------
// state access
// ---------------------------------------------------------------------------
template <typename T>
__global__ void state_io_kernel(const QPDesc* __restrict__ descs, const double* z, const double* y, double* zo,
                                double* yo, const size_t* offs, int set) {
  const QPDesc d = descs[blockIdx.x];
  const size_t o = offs[blockIdx.x];
  T* zz = reinterpret_cast<T*>(d.z);
  T* yy = reinterpret_cast<T*>(d.y);
  for (int e = threadIdx.x; e < d.m; e += blockDim.x) {
    if (set && e == 0) d.flags[1] = 1;
    if (set) {
      zz[e] = z ? (T)z[o + e] : T(0);
      yy[e] = y ? (T)y[o + e] : T(0);
    } else {
      if (zo) zo[o + e] = (double)zz[e];
      if (yo) yo[o + e] = (double)yy[e];
    }
  }
}

static int state_io(qp_handle* h, const double* z, const double* y, double* zo, double* yo, int set) {
  std::vector<size_t> offs(h->batch);
  for (int b = 0; b < h->batch; ++b) offs[b] = h->off[b].lohi;
  size_t* doffs = nullptr;
  CU(cudaMalloc(&doffs, offs.size() * sizeof(size_t)));
  CU(cudaMemcpyAsync(doffs, offs.data(), offs.size() * sizeof(size_t), cudaMemcpyHostToDevice, h->stream));
  if (h->esz == 8) state_io_kernel<double><<<h->batch, 256, 0, h->stream>>>(h->ddesc, z, y, zo, yo, doffs, set);
  else state_io_kernel<float><<<h->batch, 256, 0, h->stream>>>(h->ddesc, z, y, zo, yo, doffs, set);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(h->stream));
  cudaFree(doffs);
  return GPUSLS_OK;
}

extern "C" int qp_set_warm_start(qp_handle* h, const double* z, const double* y, const double* rho) {
  if (!h) return fail(GPUSLS_ERR_INVALID, "qp_set_warm_start: null handle");
  int st = state_io(h, z, y, nullptr, nullptr, 1);
  if (st) return st;
  if (rho) {
    for (int b = 0; b < h->batch; ++b) {
      if (!(rho[b] > 0)) return fail(GPUSLS_ERR_INVALID, "qp_set_warm_start: rho must be > 0");
      double old = 0;
      CU(cudaMemcpyAsync(&old, h->hdesc[b].rho, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      CU(cudaStreamSynchronize(h->stream));
      if (old != rho[b]) {
        int fl0 = 0;   // factorization no longer valid (flags[1], the warm mark, stays set)
        CU(cudaMemcpyAsync(h->hdesc[b].rho, &rho[b], sizeof(double), cudaMemcpyHostToDevice, h->stream));
        CU(cudaMemcpyAsync(h->hdesc[b].flags, &fl0, sizeof(fl0), cudaMemcpyHostToDevice, h->stream));
        CU(cudaStreamSynchronize(h->stream));
      }
    }
  }
  return GPUSLS_OK;
}

extern "C" int qp_get_state(qp_handle* h, double* z, double* y, double* rho) {
  if (!h) return fail(GPUSLS_ERR_INVALID, "qp_get_state: null handle");
  int st = state_io(h, nullptr, nullptr, z, y, 0);
  if (st) return st;
  if (rho) {
    for (int b = 0; b < h->batch; ++b)
      CU(cudaMemcpyAsync(&rho[b], h->hdesc[b].rho, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
  }
  return GPUSLS_OK;
}

extern "C" int qp_update(qp_handle* h, const double* A, const double* B, const double* c, const double* Q,
                         const double* R, const double* S, const double* q, const double* r, const double* C,
                         const double* D, const double* CN, const double* lo, const double* hi) {
  gsls::NvtxRange nvtx_("gpusls/qp_update");
  if (!h) return fail(GPUSLS_ERR_INVALID, "qp_update: null handle");
  std::vector<PackJob> jobs;
  const bool refac = A || B || c || Q || R || S || q || r || C || D || CN;
  // the FP64 copies mirror the caller's pool layout (per-QP blocks
  // concatenated), so each array kind is one device-to-device copy for the
  // whole batch; the padded solve-precision copies are pack jobs per QP
  const double* srcs[13] = {A, B, c, Q, R, S, q, r, C, D, CN, lo, hi};
  size_t n64[13] = {};
  for (int b = 0; b < h->batch; ++b) {
    const qp_dims& d = h->dims[b];
    const QPDesc& D_ = h->hdesc[b];
    const QPOffsets& po = h->off[b];
    const int nx = d.nx, nu = d.nu, N = d.N, nc = d.nc, nf = d.nf, m = N * nc + nf;
    const int ldx = D_.ldx, ldu = D_.ldu;
    auto add = [&](int k, size_t o, void* dst, int count, int rows, int cols, int ld, size_t n) {
      n64[k] += n;
      if (srcs[k] && n > 0) jobs.push_back({srcs[k] + o, dst, count, rows, cols, ld});
    };
    add(0, po.A, D_.A, N, nx, nx, ldx, (size_t)N * nx * nx);
    add(1, po.B, D_.B, N, nx, nu, ldu, (size_t)N * nx * nu);
    add(2, po.c, D_.b, N, 1, nx, ldx, (size_t)N * nx);
    add(3, po.Q, D_.Q, N + 1, nx, nx, ldx, (size_t)(N + 1) * nx * nx);
    add(4, po.R, D_.R, N, nu, nu, ldu, (size_t)N * nu * nu);
    add(5, po.S, D_.S, N, nu, nx, ldx, (size_t)N * nu * nx);
    add(6, po.q, D_.q, N + 1, 1, nx, ldx, (size_t)(N + 1) * nx);
    add(7, po.r, D_.r, N, 1, nu, ldu, (size_t)N * nu);
    add(8, po.C, D_.C, N, nc, nx, ldx, (size_t)N * nc * nx);
    add(9, po.D, D_.D, N, nc, nu, ldu, (size_t)N * nc * nu);
    add(10, po.CN, D_.CN, 1, nf, nx, ldx, (size_t)nf * nx);
    add(11, po.lohi, D_.lo, 1, 1, m, m, (size_t)m);
    add(12, po.lohi, D_.hi, 1, 1, m, m, (size_t)m);
  }
  const QPDesc& D0 = h->hdesc[0];
  double* dst64[13] = {D0.A64, D0.B64, D0.b64, D0.Q64, D0.R64, D0.S64, D0.q64, D0.r64, D0.C64, D0.D64,
                       D0.CN64, D0.lo64, D0.hi64};
  for (int k = 0; k < 13; ++k)
    if (srcs[k] && n64[k] > 0)
      CU(cudaMemcpyAsync(dst64[k], srcs[k], n64[k] * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  if (refac) {   // the factorization of every QP is stale
    flags_clear_kernel<<<(h->batch + 255) / 256, 256, 0, h->stream>>>(h->ddesc, h->batch);
    CU(cudaGetLastError());
  }
  int st = run_pack(h, jobs);
  if (st) return st;
  CU(cudaStreamSynchronize(h->stream));
  return GPUSLS_OK;
}

template <typename T>
__global__ void reset_kernel(const QPDesc* __restrict__ descs, const double* __restrict__ rho0) {
  const QPDesc d = descs[blockIdx.x];
  T* zz = reinterpret_cast<T*>(d.z);
  T* yy = reinterpret_cast<T*>(d.y);
  for (int e = threadIdx.x; e < d.m; e += blockDim.x) {
    zz[e] = T(0);
    yy[e] = T(0);
  }
  // undo iterative-refinement corrections of the linear term r
  T* rr = reinterpret_cast<T*>(d.r);
  for (int e = threadIdx.x; e < d.N * d.ldu; e += blockDim.x) {
    const int i = e / d.ldu, a = e - i * d.ldu;
    rr[e] = a < d.nu ? (T)d.r64[(size_t)i * d.nu + a] : T(0);
  }
  if (threadIdx.x == 0) {
    d.rho[0] = rho0[blockIdx.x];
    d.flags[0] = 0;
    d.flags[1] = 0;
  }
}

extern "C" int qp_reset(qp_handle* h) {
  if (!h) return fail(GPUSLS_ERR_INVALID, "qp_reset: null handle");
  if (h->esz == 8) reset_kernel<double><<<h->batch, 256, 0, h->stream>>>(h->ddesc, h->rho0_dev);
  else reset_kernel<float><<<h->batch, 256, 0, h->stream>>>(h->ddesc, h->rho0_dev);
  CU(cudaGetLastError());
  return GPUSLS_OK;
}

extern "C" void qp_destroy(qp_handle* h) {
  if (!h) return;
  if (h->tpool) cudaFree(h->tpool);
  if (h->dpool) cudaFree(h->dpool);
  if (h->ddesc) cudaFree(h->ddesc);
  if (h->info_i) cudaFree(h->info_i);
  if (h->info_d) cudaFree(h->info_d);
  if (h->djobs) cudaFree(h->djobs);
  if (h->rho0_dev) cudaFree(h->rho0_dev);
  if (h->order_dev) cudaFree(h->order_dev);
  delete h;
}
