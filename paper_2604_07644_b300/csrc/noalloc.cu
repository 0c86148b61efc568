// Allocation-free FP64 KKT residual of one LTV-QP.
//
// Some callers cannot allocate GPU memory at the point where they need this
// check: a real-time control loop that must not call cudaMalloc (it can block
// and implicitly synchronize the device), code running inside a region that
// forbids allocation, or a host runtime that owns every device buffer itself.
// For them gpusls_kkt_noalloc evaluates the same residual as qp_kkt without a
// handle: the caller passes the problem, the candidate point and an output
// buffer, and the only scratch -- the per-stage gradient pieces g_k, h_k of the
// costate recursion -- lives in a fixed device array defined in this file.
#include <cuda_runtime.h>
#include <math.h>

#include <string>

#include "../../include/gpusls.h"
#include "dense.cuh"
#include "internal.h"

using namespace gsls;

// Scratch shared by every call: (N+1)*nx + N*nu doubles at most.  It stays
// allocated on every device that loads the library until the process exits.
static __device__ __align__(256) double g_kkt_noalloc_scratch[GPUSLS_NOALLOC_MAX_SCRATCH];

namespace {

struct NoAllocArgs {
  int nx, nu, N, nc, nf;
  const double *A, *B, *c, *Q, *R, *S, *q, *r, *C, *D, *CN, *lo, *hi, *x0, *x, *u, *lam;
  double* out;
  double* scratch;
};

__device__ inline double block_max_d(double v, double* red) {
  v = warp_max(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  for (int k = 0; k < NT / 32; ++k) r = fmax(r, red[k]);
  __syncthreads();
  return r;
}

// One CTA: stage-local parts for every stage, then the costate recursion
// mu_N = Q_N x_N + q_N + C_N^T lam_N, mu_k = g_k + A_k^T mu_{k+1}, with the
// u-stationarity residual h_k + B_k^T mu_{k+1} at each stage.  Same definition
// as qp_kkt (see include/gpusls.h).
__global__ void __launch_bounds__(NT) kkt_noalloc_kernel(NoAllocArgs a) {
  __shared__ double xv[TILE], xn[TILE], uv[64], lv[64], mu[TILE], mu2[TILE], red[NT / 32];
  const int nx = a.nx, nu = a.nu, N = a.N, nc = a.nc, nf = a.nf;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  double* g = a.scratch;                      // [(N+1)][nx]
  double* h = a.scratch + (size_t)(N + 1) * nx;   // [N][nu]
  double dyn = 0.0, viol = 0.0, comp = 0.0, stat = 0.0;
  for (int i = 0; i <= N; ++i) {
    const bool term = (i == N);
    const int nr = term ? nf : nc;
    for (int j = t; j < nx; j += NT) {
      xv[j] = a.x[(size_t)i * nx + j];
      if (!term) xn[j] = a.x[(size_t)(i + 1) * nx + j];
    }
    for (int k = t; k < nu; k += NT) uv[k] = term ? 0.0 : a.u[(size_t)i * nu + k];
    for (int k = t; k < nr; k += NT) lv[k] = a.lam[(size_t)i * nc + k];
    __syncthreads();
    const double* Qi = a.Q + (size_t)i * nx * nx;
    const double* Ci = term ? a.CN : a.C + (size_t)i * nc * nx;
    const double* Di = term ? nullptr : a.D + (size_t)i * nc * nu;
    for (int j = w; j < nx; j += NT / 32) {
      double gs = warp_dot(Qi + (size_t)j * nx, xv, nx);
      if (!term) {
        const double ax = warp_dot(a.A + (size_t)i * nx * nx + (size_t)j * nx, xv, nx) +
                          warp_dot(a.B + (size_t)i * nx * nu + (size_t)j * nu, uv, nu);
        if (lane == 0) dyn = fmax(dyn, fabs(xn[j] - ax - a.c[(size_t)i * nx + j]));
        if (a.S) {
          double st = 0.0;
          for (int k = lane; k < nu; k += 32) st += a.S[(size_t)i * nu * nx + (size_t)k * nx + j] * uv[k];
          gs += warp_sum(st);
        }
      }
      double ct = 0.0;
      for (int k = lane; k < nr; k += 32) ct += Ci[(size_t)k * nx + j] * lv[k];
      gs += warp_sum(ct);
      if (lane == 0) g[(size_t)i * nx + j] = gs + a.q[(size_t)i * nx + j];
    }
    if (!term) {
      for (int k = w; k < nu; k += NT / 32) {
        double hs = warp_dot(a.R + (size_t)i * nu * nu + (size_t)k * nu, uv, nu);
        if (a.S) hs += warp_dot(a.S + (size_t)i * nu * nx + (size_t)k * nx, xv, nx);
        double dt = 0.0;
        for (int l = lane; l < nc; l += 32) dt += Di[(size_t)l * nu + k] * lv[l];
        hs += warp_sum(dt);
        if (lane == 0) h[(size_t)i * nu + k] = hs + a.r[(size_t)i * nu + k];
      }
    }
    for (int k = w; k < nr; k += NT / 32) {
      double v = warp_dot(Ci + (size_t)k * nx, xv, nx);
      if (!term) v += warp_dot(Di + (size_t)k * nu, uv, nu);
      if (lane == 0) {
        const size_t gi = (size_t)i * nc + k;
        const double lo = a.lo[gi], hi = a.hi[gi], l = lv[k];
        viol = fmax(viol, fmax(fmax(v - hi, lo - v), 0.0));
        double cp = 0.0;
        if (l > 0) cp = isfinite(hi) ? l * fabs(hi - v) : fabs(l);
        else if (l < 0) cp = isfinite(lo) ? -l * fabs(v - lo) : fabs(l);
        comp = fmax(comp, cp);
      }
    }
    __syncthreads();
  }
  for (int j = t; j < nx; j += NT) dyn = fmax(dyn, fabs(a.x[j] - a.x0[j]));
  for (int j = t; j < nx; j += NT) mu[j] = g[(size_t)N * nx + j];
  __syncthreads();
  for (int i = N - 1; i >= 0; --i) {
    for (int k = w; k < nu; k += NT / 32) {
      double s2 = 0.0;
      for (int j = lane; j < nx; j += 32) s2 += a.B[(size_t)i * nx * nu + (size_t)j * nu + k] * mu[j];
      s2 = warp_sum(s2);
      if (lane == 0) stat = fmax(stat, fabs(s2 + h[(size_t)i * nu + k]));
    }
    for (int j = t; j < nx; j += NT) {
      double s2 = g[(size_t)i * nx + j];
      const double* Ai = a.A + (size_t)i * nx * nx;
      for (int k = 0; k < nx; ++k) s2 += Ai[(size_t)k * nx + j] * mu[k];
      mu2[j] = s2;
    }
    __syncthreads();
    for (int j = t; j < nx; j += NT) mu[j] = mu2[j];
    __syncthreads();
  }
  const double p0 = block_max_d(dyn, red), p1 = block_max_d(viol, red);
  const double p2 = block_max_d(stat, red), p3 = block_max_d(comp, red);
  if (t == 0) {
    a.out[0] = fmax(fmax(p0, p1), fmax(p2, p3));
    a.out[1] = p0;
    a.out[2] = p1;
    a.out[3] = p2;
    a.out[4] = p3;
  }
}

// Device address of the scratch array on the current device.  It is looked up
// on every call (the lookup allocates nothing): a cached address would dangle
// after cudaDeviceReset or any other re-creation of the primary context, which
// reloads the module and with it the array.
int scratch_for_current_device(double** ptr) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_kkt_noalloc_scratch);
  if (e != cudaSuccess || !p)
    return set_error(GPUSLS_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
  *ptr = static_cast<double*>(p);
  return GPUSLS_OK;
}

}  // namespace

extern "C" int gpusls_kkt_noalloc(qp_dims d, const double* A, const double* B, const double* c, const double* Q,
                                  const double* R, const double* S, const double* q, const double* r, const double* C,
                                  const double* D, const double* CN, const double* lo, const double* hi,
                                  const double* x0, const double* dx, const double* du, const double* lam,
                                  double* out, void* stream) {
  if (!A || !B || !c || !Q || !R || !q || !r || !lo || !hi || !x0 || !dx || !du || !lam || !out)
    return set_error(GPUSLS_ERR_INVALID, "gpusls_kkt_noalloc: null argument");
  if ((d.nc > 0 && (!C || !D)) || (d.nf > 0 && !CN))
    return set_error(GPUSLS_ERR_INVALID, "gpusls_kkt_noalloc: C/D/CN missing");
  if (d.nx < 1 || d.nx > TILE || d.nu < 1 || d.nu > 64 || d.nc < 0 || d.nc > 64 || d.nf < 0 || d.nf > 64 || d.N < 1)
    return set_error(GPUSLS_ERR_INVALID, "gpusls_kkt_noalloc: dims out of range (nx <= 80, nu, nc, nf <= 64)");
  const size_t need = (size_t)(d.N + 1) * d.nx + (size_t)d.N * d.nu;
  if (need > (size_t)GPUSLS_NOALLOC_MAX_SCRATCH)
    return set_error(GPUSLS_ERR_INVALID, "gpusls_kkt_noalloc: (N+1)*nx + N*nu = " + std::to_string(need) +
                                             " exceeds the fixed scratch of " +
                                             std::to_string(GPUSLS_NOALLOC_MAX_SCRATCH) + " doubles");
  double* scratch = nullptr;
  int st = scratch_for_current_device(&scratch);
  if (st) return st;
  NoAllocArgs a = {d.nx, d.nu, d.N, d.nc, d.nf, A, B, c, Q, R, S, q, r, C, D, CN, lo, hi, x0, dx, du, lam, out,
                   scratch};
  kkt_noalloc_kernel<<<1, NT, 0, (cudaStream_t)stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(GPUSLS_ERR_CUDA, std::string("kkt_noalloc_kernel: ") + cudaGetErrorString(e));
  return GPUSLS_OK;
}
