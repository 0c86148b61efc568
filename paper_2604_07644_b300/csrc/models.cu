// Analytic models of App. C (Dubins car) and App. D (planar quadrotor) and
// the SQP / RTI outer loop around the LTV-QP solver (Sec. III-B, Sec. IV-C).
//
//   model_linearize_kernel  one thread per (trajectory b, stage k): the
//       Jacobians A_k, B_k, the defect b_k = f(x_k, u_k) - x_{k+1}, the
//       Gauss-Newton cost blocks and gradients, and the linearized input-box
//       and obstacle rows of eq. sqp_qp -- every stage in parallel (the
//       "parallel linearization" of Fig. fig:schematic).
//   model_merit_kernel      one CTA per trajectory: the l1 merit of the trial
//       point X + alpha dX (cost + w x (defects + violations)), a block
//       reduction over the stages, for the step-size search of Sec. III-B.
//   model_axpy_kernel, model_simulate_kernel, model_shift_kernel: the step,
//       the disturbed plant x+ = f(x, u_0) + E w and the nominal shift of an
//       RTI control step (Sec. IV-C).
// The drivers sqp_solve and rti_step chain these with qp_update / qp_solve
// (and, for robust RTI, fastsls_solve) on one batch handle.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/gpusls.h"
#include "internal.h"

using namespace gsls;

#define CUM2(x)                                                                                     \
  do {                                                                                              \
    cudaError_t e_ = (x);                                                                           \
    if (e_ != cudaSuccess) return (void)cudaGetLastError(), set_error(GPUSLS_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

namespace {

__host__ __device__ inline int m_nx(const model_spec& m) { return m.kind == GPUSLS_MODEL_DUBINS ? 3 : 6; }
__host__ __device__ inline int m_nu(const model_spec& m) { return m.kind == GPUSLS_MODEL_DUBINS ? 1 : 2; }

// x_{k+1} = f(x, u): App. C; App. D with one explicit Euler step.
__device__ void f_eval(const model_spec& m, const double* x, const double* u, double* y) {
  if (m.kind == GPUSLS_MODEL_DUBINS) {
    y[0] = x[0] + m.v * cos(x[2]) * m.dt;
    y[1] = x[1] + m.v * sin(x[2]) * m.dt;
    y[2] = x[2] + u[0] * m.dt;
    return;
  }
  const double T = u[0] + u[1], s = sin(x[2]), c = cos(x[2]);
  y[0] = x[0] + m.dt * x[3];
  y[1] = x[1] + m.dt * x[4];
  y[2] = x[2] + m.dt * x[5];
  y[3] = x[3] + m.dt * (-T * s / m.mass);
  y[4] = x[4] + m.dt * (T * c / m.mass - m.grav);
  y[5] = x[5] + m.dt * (m.arm * (u[1] - u[0]) / m.inertia);
}

// A = df/dx [nx][nx], B = df/du [nx][nu] (row-major), by hand from f_eval.
__device__ void jac_eval(const model_spec& m, const double* x, const double* u, double* A, double* B) {
  const int nx = m_nx(m), nu = m_nu(m);
  for (int i = 0; i < nx * nx; ++i) A[i] = (i % (nx + 1) == 0) ? 1.0 : 0.0;
  for (int i = 0; i < nx * nu; ++i) B[i] = 0.0;
  if (m.kind == GPUSLS_MODEL_DUBINS) {
    A[0 * 3 + 2] = -m.v * sin(x[2]) * m.dt;
    A[1 * 3 + 2] = m.v * cos(x[2]) * m.dt;
    B[2] = m.dt;
    return;
  }
  const double T = u[0] + u[1], s = sin(x[2]), c = cos(x[2]);
  A[0 * 6 + 3] = m.dt;
  A[1 * 6 + 4] = m.dt;
  A[2 * 6 + 5] = m.dt;
  A[3 * 6 + 2] = -m.dt * T * c / m.mass;
  A[4 * 6 + 2] = -m.dt * T * s / m.mass;
  B[3 * 2 + 0] = B[3 * 2 + 1] = -m.dt * s / m.mass;
  B[4 * 2 + 0] = B[4 * 2 + 1] = m.dt * c / m.mass;
  B[5 * 2 + 0] = -m.dt * m.arm / m.inertia;
  B[5 * 2 + 1] = m.dt * m.arm / m.inertia;
}

// obstacle o: g = r^2 - (p_x - c_x)^2 - (p_y - c_y)^2 (<= 0 is safe)
__device__ inline double obs_g(const model_spec& m, int o, const double* x) {
  const double dx = x[0] - m.obs[3 * o], dy = x[1] - m.obs[3 * o + 1], r = m.obs[3 * o + 2];
  return r * r - dx * dx - dy * dy;
}

struct LinOut {
  double *A, *B, *c, *Q, *R, *S, *q, *r, *C, *D, *CN, *lo, *hi, *dx0;
};

__global__ void model_linearize_kernel(model_spec m, int batch, const double* __restrict__ X,
                                       const double* __restrict__ U, const double* __restrict__ x0bar, LinOut o) {
  const int N = m.N, nx = m_nx(m), nu = m_nu(m), no = m.n_obs, nc = nu + no, mrows = N * nc + no;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= batch * (N + 1)) return;
  const int b = e / (N + 1), k = e - b * (N + 1);
  const double* x = X + ((size_t)b * (N + 1) + k) * nx;
  double* lo = o.lo + (size_t)b * mrows;
  double* hi = o.hi + (size_t)b * mrows;
  double* Qk = o.Q + ((size_t)b * (N + 1) + k) * nx * nx;
  double* qk = o.q + ((size_t)b * (N + 1) + k) * nx;
  const double* Qw = k < N ? m.Qd : m.QNd;
  for (int i = 0; i < nx * nx; ++i) Qk[i] = (i % (nx + 1) == 0) ? Qw[i / (nx + 1)] : 0.0;
  for (int i = 0; i < nx; ++i) qk[i] = Qw[i] * (x[i] - m.xref[i]);
  if (k == N) {
    double* CN = o.CN + (size_t)b * no * nx;
    for (int j = 0; j < no; ++j) {
      for (int i = 0; i < nx; ++i) CN[j * nx + i] = 0.0;
      CN[j * nx + 0] = -2.0 * (x[0] - m.obs[3 * j]);
      CN[j * nx + 1] = -2.0 * (x[1] - m.obs[3 * j + 1]);
      lo[N * nc + j] = -INFINITY;
      hi[N * nc + j] = -obs_g(m, j, x);
    }
    const double* x0 = X + (size_t)b * (N + 1) * nx;
    for (int i = 0; i < nx; ++i) o.dx0[(size_t)b * nx + i] = x0bar[(size_t)b * nx + i] - x0[i];
    return;
  }
  const double* u = U + ((size_t)b * N + k) * nu;
  const size_t sk = (size_t)b * N + k;
  jac_eval(m, x, u, o.A + sk * nx * nx, o.B + sk * nx * nu);
  double fx[6];
  f_eval(m, x, u, fx);
  for (int i = 0; i < nx; ++i) o.c[sk * nx + i] = fx[i] - x[nx + i];   // x_{k+1} follows x_k in X
  double* Rk = o.R + sk * nu * nu;
  for (int i = 0; i < nu * nu; ++i) Rk[i] = (i % (nu + 1) == 0) ? m.Rd[i / (nu + 1)] : 0.0;
  for (int i = 0; i < nu * nx; ++i) o.S[sk * nu * nx + i] = 0.0;
  for (int i = 0; i < nu; ++i) o.r[sk * nu + i] = m.Rd[i] * (u[i] - m.uref[i]);
  double* Ck = o.C + sk * nc * nx;
  double* Dk = o.D + sk * nc * nu;
  for (int i = 0; i < nc * nx; ++i) Ck[i] = 0.0;
  for (int i = 0; i < nc * nu; ++i) Dk[i] = 0.0;
  for (int j = 0; j < nu; ++j) {
    Dk[j * nu + j] = 1.0;
    lo[k * nc + j] = m.u_lo[j] - u[j];
    hi[k * nc + j] = m.u_hi[j] - u[j];
  }
  for (int j = 0; j < no; ++j) {
    Ck[(nu + j) * nx + 0] = -2.0 * (x[0] - m.obs[3 * j]);
    Ck[(nu + j) * nx + 1] = -2.0 * (x[1] - m.obs[3 * j + 1]);
    lo[k * nc + nu + j] = -INFINITY;
    hi[k * nc + nu + j] = -obs_g(m, j, x);
  }
}

// l1 merit of (X + a dX, U + a dU), a = alpha[b]: one CTA per trajectory.
__global__ void model_merit_kernel(model_spec m, const double* __restrict__ X, const double* __restrict__ U,
                                   const double* __restrict__ dX, const double* __restrict__ dU,
                                   const double* __restrict__ alpha, const double* __restrict__ x0bar, double w,
                                   double* __restrict__ out) {
  const int N = m.N, nx = m_nx(m), nu = m_nu(m), no = m.n_obs;
  const int b = blockIdx.x;
  const double a = alpha ? alpha[b] : 0.0;
  const double* Xb = X + (size_t)b * (N + 1) * nx;
  const double* Ub = U + (size_t)b * N * nu;
  const double* dXb = dX ? dX + (size_t)b * (N + 1) * nx : nullptr;
  const double* dUb = dU ? dU + (size_t)b * N * nu : nullptr;
  double cost = 0.0, inf = 0.0;
  for (int k = threadIdx.x; k <= N; k += blockDim.x) {
    double x[6], x1[6], u[2], fx[6];
    for (int i = 0; i < nx; ++i) x[i] = Xb[k * nx + i] + (dXb ? a * dXb[k * nx + i] : 0.0);
    const double* Qw = k < N ? m.Qd : m.QNd;
    for (int i = 0; i < nx; ++i) cost += 0.5 * Qw[i] * (x[i] - m.xref[i]) * (x[i] - m.xref[i]);
    for (int j = 0; j < no; ++j) inf += fmax(obs_g(m, j, x), 0.0);
    if (k == 0)
      for (int i = 0; i < nx; ++i) inf += fabs(x[i] - x0bar[(size_t)b * nx + i]);
    if (k < N) {
      for (int i = 0; i < nu; ++i) u[i] = Ub[k * nu + i] + (dUb ? a * dUb[k * nu + i] : 0.0);
      for (int i = 0; i < nx; ++i) x1[i] = Xb[(k + 1) * nx + i] + (dXb ? a * dXb[(k + 1) * nx + i] : 0.0);
      for (int i = 0; i < nu; ++i) {
        cost += 0.5 * m.Rd[i] * (u[i] - m.uref[i]) * (u[i] - m.uref[i]);
        inf += fmax(u[i] - m.u_hi[i], 0.0) + fmax(m.u_lo[i] - u[i], 0.0);
      }
      f_eval(m, x, u, fx);
      for (int i = 0; i < nx; ++i) inf += fabs(fx[i] - x1[i]);
    }
  }
  // block reduction in a fixed order (deterministic)
  __shared__ double sc[256], si[256];
  sc[threadIdx.x] = cost;
  si[threadIdx.x] = inf;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sc[threadIdx.x] += sc[threadIdx.x + s];
      si[threadIdx.x] += si[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[b] = sc[0] + w * si[0];
}

// Y[b] += alpha[b] dY[b] over n values per trajectory
__global__ void model_axpy_kernel(int batch, int n, double* __restrict__ Y, const double* __restrict__ dY,
                                  const double* __restrict__ alpha) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (size_t)batch * n) return;
  Y[e] += (alpha ? alpha[e / n] : 1.0) * dY[e];
}

// x[b] <- f(x[b], U[b][0]) + E w[b]; u0[b] <- U[b][0]
__global__ void model_simulate_kernel(model_spec m, int batch, double* __restrict__ x, const double* __restrict__ U,
                                      const double* __restrict__ W, double* __restrict__ u0) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  const int nx = m_nx(m), nu = m_nu(m);
  double xb[6], y[6];
  const double* u = U + (size_t)b * m.N * nu;
  for (int i = 0; i < nx; ++i) xb[i] = x[(size_t)b * nx + i];
  f_eval(m, xb, u, y);
  for (int i = 0; i < nx; ++i) {
    double s = y[i];
    if (W)
      for (int j = 0; j < nx; ++j) s += m.E[i * nx + j] * W[(size_t)b * nx + j];
    x[(size_t)b * nx + i] = s;
  }
  if (u0)
    for (int i = 0; i < nu; ++i) u0[(size_t)b * nu + i] = u[i];
}

// Nominal for the next control step: X[b][k] <- X[b][k+1], U[b][k] <- U[b][k+1],
// the last stage kept (one thread per trajectory and component, in order).
__global__ void model_shift_kernel(model_spec m, int batch, double* __restrict__ X, double* __restrict__ U) {
  const int nx = m_nx(m), nu = m_nu(m), N = m.N;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= batch * (nx + nu)) return;
  const int b = e / (nx + nu), i = e - b * (nx + nu);
  if (i < nx) {
    double* Xb = X + (size_t)b * (N + 1) * nx;
    for (int k = 0; k < N; ++k) Xb[k * nx + i] = Xb[(k + 1) * nx + i];
  } else {
    double* Ub = U + (size_t)b * N * nu;
    const int j = i - nx;
    for (int k = 0; k + 1 < N; ++k) Ub[k * nu + j] = Ub[(k + 1) * nu + j];
  }
}

int check_spec(const model_spec* m) {
  if (!m) return set_error(GPUSLS_ERR_INVALID, "model: null spec");
  if (m->kind != GPUSLS_MODEL_DUBINS && m->kind != GPUSLS_MODEL_QUAD2D)
    return set_error(GPUSLS_ERR_INVALID, "model: unknown kind");
  if (m->N < 2 || m->N > GPUSLS_MAX_N || m->n_obs < 0 || m->n_obs > GPUSLS_MODEL_MAX_OBS || !(m->dt > 0.0))
    return set_error(GPUSLS_ERR_INVALID, "model: N, n_obs or dt out of range");
  return GPUSLS_OK;
}

int launch_linearize(const model_spec* m, int batch, const double* X, const double* U, const double* x0bar,
                     const LinOut& o, cudaStream_t st) {
  const int tot = batch * (m->N + 1);
  model_linearize_kernel<<<(tot + 127) / 128, 128, 0, st>>>(*m, batch, X, U, x0bar, o);
  CUM2(cudaGetLastError());
  return GPUSLS_OK;
}

}  // namespace

extern "C" int model_dims(const model_spec* m, qp_dims* d) {
  int st = check_spec(m);
  if (st) return st;
  if (!d) return set_error(GPUSLS_ERR_INVALID, "model_dims: null dims");
  d->nx = m_nx(*m);
  d->nu = m_nu(*m);
  d->N = m->N;
  d->nc = d->nu + m->n_obs;
  d->nf = m->n_obs;
  return GPUSLS_OK;
}

extern "C" int model_linearize(const model_spec* m, int32_t batch, const double* X, const double* U,
                               const double* x0bar, double* A, double* B, double* c, double* Q, double* R, double* S,
                               double* q, double* r, double* C, double* D, double* CN, double* lo, double* hi,
                               double* dx0, void* stream) {
  int st = check_spec(m);
  if (st) return st;
  if (batch < 1 || !X || !U || !x0bar || !A || !B || !c || !Q || !R || !S || !q || !r || !C || !D || !lo || !hi ||
      !dx0 || (m->n_obs > 0 && !CN))
    return set_error(GPUSLS_ERR_INVALID, "model_linearize: null argument or batch < 1");
  LinOut o = {A, B, c, Q, R, S, q, r, C, D, CN, lo, hi, dx0};
  st = launch_linearize(m, batch, X, U, x0bar, o, (cudaStream_t)stream);
  if (st) return st;
  CUM2(cudaStreamSynchronize((cudaStream_t)stream));
  return GPUSLS_OK;
}

extern "C" int model_merit(const model_spec* m, int32_t batch, const double* X, const double* U, const double* dX,
                           const double* dU, const double* alpha, const double* x0bar, double w, double* out,
                           void* stream) {
  int st = check_spec(m);
  if (st) return st;
  if (batch < 1 || !X || !U || !x0bar || !out) return set_error(GPUSLS_ERR_INVALID, "model_merit: null argument");
  model_merit_kernel<<<batch, 256, 0, (cudaStream_t)stream>>>(*m, X, U, dX, dU, alpha, x0bar, w, out);
  CUM2(cudaGetLastError());
  CUM2(cudaStreamSynchronize((cudaStream_t)stream));
  return GPUSLS_OK;
}

// ---------------------------------------------------------------------------
// SQP / RTI handle
// ---------------------------------------------------------------------------
struct sqp_handle {
  model_spec m{};
  int batch = 0, robust = 0;
  qp_dims d{};
  cudaStream_t st = nullptr;
  qp_handle* q = nullptr;
  sls_handle* s = nullptr;
  LinOut lin{};
  double *dX = nullptr, *dU = nullptr, *lam = nullptr, *alpha = nullptr, *merit = nullptr;
  double *E = nullptr, *Qbar = nullptr, *Rbar = nullptr, *QbarN = nullptr, *tau = nullptr, *hk = nullptr,
         *hf = nullptr;
  int have_tau = 0;
  std::vector<void*> allocs;
};

extern "C" void sqp_destroy(sqp_handle* h) {
  if (!h) return;
  if (h->q) qp_destroy(h->q);
  if (h->s) sls_destroy(h->s);
  for (void* p : h->allocs) cudaFree(p);
  delete h;
}

extern "C" int sqp_setup(sqp_handle** out, const model_spec* m, int32_t batch, const qp_settings* s, int32_t robust,
                         void* stream) {
  if (!out || !s) return set_error(GPUSLS_ERR_INVALID, "sqp_setup: null argument");
  int st = check_spec(m);
  if (st) return st;
  if (batch < 1) return set_error(GPUSLS_ERR_INVALID, "sqp_setup: batch < 1");
  if (robust && batch != 1) return set_error(GPUSLS_ERR_INVALID, "sqp_setup: robust RTI runs one trajectory");
  if (robust && m->N > 512) return set_error(GPUSLS_ERR_INVALID, "sqp_setup: robust RTI needs N <= 512");
  sqp_handle* h = new sqp_handle();
  h->m = *m;
  h->batch = batch;
  h->robust = robust ? 1 : 0;
  h->st = (cudaStream_t)stream;
  model_dims(m, &h->d);
  const size_t nx = h->d.nx, nu = h->d.nu, N = h->d.N, nc = h->d.nc, nf = h->d.nf, B = batch;
  const size_t mrows = N * nc + nf;
  auto alloc = [&](double** p, size_t n) -> bool {
    void* v = nullptr;
    if (cudaMalloc(&v, std::max<size_t>(n, 1) * sizeof(double)) != cudaSuccess) return false;
    cudaMemsetAsync(v, 0, std::max<size_t>(n, 1) * sizeof(double), h->st);
    h->allocs.push_back(v);
    *p = static_cast<double*>(v);
    return true;
  };
  bool ok = alloc(&h->lin.A, B * N * nx * nx) && alloc(&h->lin.B, B * N * nx * nu) && alloc(&h->lin.c, B * N * nx) &&
            alloc(&h->lin.Q, B * (N + 1) * nx * nx) && alloc(&h->lin.R, B * N * nu * nu) &&
            alloc(&h->lin.S, B * N * nu * nx) && alloc(&h->lin.q, B * (N + 1) * nx) && alloc(&h->lin.r, B * N * nu) &&
            alloc(&h->lin.C, B * N * nc * nx) && alloc(&h->lin.D, B * N * nc * nu) && alloc(&h->lin.CN, B * nf * nx) &&
            alloc(&h->lin.lo, B * mrows) && alloc(&h->lin.hi, B * mrows) && alloc(&h->lin.dx0, B * nx) &&
            alloc(&h->dX, B * (N + 1) * nx) && alloc(&h->dU, B * N * nu) && alloc(&h->lam, B * mrows) &&
            alloc(&h->alpha, B) && alloc(&h->merit, B);
  if (ok && h->robust)
    ok = alloc(&h->E, N * nx * nx) && alloc(&h->Qbar, nx * nx) && alloc(&h->Rbar, nu * nu) &&
         alloc(&h->QbarN, nx * nx) && alloc(&h->tau, (N + 1) * N * std::max<size_t>(std::max(nc, nf), 1)) &&
         alloc(&h->hk, N * nc) && alloc(&h->hf, std::max<size_t>(nf, 1));
  if (!ok) {
    sqp_destroy(h);
    return set_error(GPUSLS_ERR_CUDA, "sqp_setup: cudaMalloc failed");
  }
  // placeholder problem data for the handle (identity costs); every solve
  // replaces all of it through qp_update first
  std::vector<double> eye((size_t)B * (N + 1) * nx * nx, 0.0), eyeu((size_t)B * N * nu * nu, 0.0);
  for (size_t i = 0; i < B * (N + 1); ++i)
    for (size_t j = 0; j < nx; ++j) eye[i * nx * nx + j * (nx + 1)] = 1.0;
  for (size_t i = 0; i < B * N; ++i)
    for (size_t j = 0; j < nu; ++j) eyeu[i * nu * nu + j * (nu + 1)] = 1.0;
  CUM2(cudaMemcpyAsync(h->lin.Q, eye.data(), eye.size() * sizeof(double), cudaMemcpyHostToDevice, h->st));
  CUM2(cudaMemcpyAsync(h->lin.R, eyeu.data(), eyeu.size() * sizeof(double), cudaMemcpyHostToDevice, h->st));
  if (h->robust) {
    // SLS data: E_j = E for every j, Qbar = I, Rbar = I, QbarN = I
    std::vector<double> E((size_t)N * nx * nx);
    for (size_t j = 0; j < N; ++j)
      for (size_t i = 0; i < nx * nx; ++i) E[j * nx * nx + i] = m->E[i];
    CUM2(cudaMemcpyAsync(h->E, E.data(), E.size() * sizeof(double), cudaMemcpyHostToDevice, h->st));
    CUM2(cudaMemcpyAsync(h->Qbar, eye.data(), nx * nx * sizeof(double), cudaMemcpyHostToDevice, h->st));
    CUM2(cudaMemcpyAsync(h->QbarN, eye.data(), nx * nx * sizeof(double), cudaMemcpyHostToDevice, h->st));
    CUM2(cudaMemcpyAsync(h->Rbar, eyeu.data(), nu * nu * sizeof(double), cudaMemcpyHostToDevice, h->st));
  }
  CUM2(cudaStreamSynchronize(h->st));
  std::vector<qp_dims> dims(batch, h->d);
  st = qp_batch_setup(&h->q, batch, dims.data(), h->lin.A, h->lin.B, h->lin.c, h->lin.Q, h->lin.R, h->lin.S,
                      h->lin.q, h->lin.r, h->lin.C, h->lin.D, h->lin.CN, h->lin.lo, h->lin.hi, nullptr, s, stream);
  if (!st && h->robust) st = sls_setup(&h->s, h->d, s->precision == GPUSLS_FP64 ? GPUSLS_FP64 : GPUSLS_FP32, 1, stream);
  if (st) {
    sqp_destroy(h);
    return st;
  }
  *out = h;
  return GPUSLS_OK;
}

namespace {
int update_qp(sqp_handle* h) {
  const LinOut& l = h->lin;
  return qp_update(h->q, l.A, l.B, l.c, l.Q, l.R, l.S, l.q, l.r, l.C, l.D, l.CN, l.lo, l.hi);
}
}  // namespace

extern "C" int sqp_solve(sqp_handle* h, double* X, double* U, const double* x0bar, int32_t iters, double merit_w,
                         int32_t line_search, double* alpha_out, qp_info* info) {
  gsls::NvtxRange nvtx_("gpusls/sqp_solve");
  if (!h || !X || !U || !x0bar || iters < 1) return set_error(GPUSLS_ERR_INVALID, "sqp_solve: bad argument");
  const int B = h->batch, nx = h->d.nx, nu = h->d.nu, N = h->d.N;
  std::vector<double> a(B), phi0(B), phi(B);
  std::vector<int> done(B);
  int worst = GPUSLS_OK;
  for (int it = 0; it < iters; ++it) {
    int st = launch_linearize(&h->m, B, X, U, x0bar, h->lin, h->st);
    if (st) return st;
    CUM2(cudaStreamSynchronize(h->st));
    st = update_qp(h);
    if (st) return st;
    st = qp_solve(h->q, h->lin.dx0, 0, 0.0, h->dX, h->dU, h->lam, info);
    if (st < 0) return st;
    worst = std::max(worst, st);
    // step size: backtracking on the l1 merit, every trajectory its own alpha
    std::fill(a.begin(), a.end(), 1.0);
    if (line_search) {
      model_merit_kernel<<<B, 256, 0, h->st>>>(h->m, X, U, nullptr, nullptr, nullptr, x0bar, merit_w, h->merit);
      CUM2(cudaGetLastError());
      CUM2(cudaMemcpyAsync(phi0.data(), h->merit, B * sizeof(double), cudaMemcpyDeviceToHost, h->st));
      std::fill(done.begin(), done.end(), 0);
      for (int t = 0; t < 8; ++t) {
        CUM2(cudaMemcpyAsync(h->alpha, a.data(), B * sizeof(double), cudaMemcpyHostToDevice, h->st));
        model_merit_kernel<<<B, 256, 0, h->st>>>(h->m, X, U, h->dX, h->dU, h->alpha, x0bar, merit_w, h->merit);
        CUM2(cudaGetLastError());
        CUM2(cudaMemcpyAsync(phi.data(), h->merit, B * sizeof(double), cudaMemcpyDeviceToHost, h->st));
        CUM2(cudaStreamSynchronize(h->st));
        int open = 0;
        for (int b = 0; b < B; ++b) {
          if (done[b]) continue;
          if (phi[b] < phi0[b] || t == 7) done[b] = 1;
          else { a[b] *= 0.5; ++open; }
        }
        if (!open) break;
      }
    }
    CUM2(cudaMemcpyAsync(h->alpha, a.data(), B * sizeof(double), cudaMemcpyHostToDevice, h->st));
    const int nX = (N + 1) * nx, nU = N * nu;
    model_axpy_kernel<<<(B * nX + 255) / 256, 256, 0, h->st>>>(B, nX, X, h->dX, h->alpha);
    model_axpy_kernel<<<(B * nU + 255) / 256, 256, 0, h->st>>>(B, nU, U, h->dU, h->alpha);
    CUM2(cudaGetLastError());
    CUM2(cudaStreamSynchronize(h->st));
    if (alpha_out) std::copy(a.begin(), a.end(), alpha_out + (size_t)it * B);
  }
  return worst;
}

extern "C" int rti_step(sqp_handle* h, double* X, double* U, double* x, const double* W, double* u_applied,
                        double* hk, double* hf, qp_info* info) {
  gsls::NvtxRange nvtx_("gpusls/rti_step");
  if (!h || !X || !U || !x) return set_error(GPUSLS_ERR_INVALID, "rti_step: null argument");
  const int B = h->batch, nx = h->d.nx, nu = h->d.nu, N = h->d.N;
  int st = launch_linearize(&h->m, B, X, U, x, h->lin, h->st);
  if (st) return st;
  CUM2(cudaStreamSynchronize(h->st));
  st = update_qp(h);
  if (st) return st;
  int qs;
  if (h->robust) {
    // controller update from the previous step's duals, tightened nominal QP, new duals
    const LinOut& l = h->lin;
    qs = fastsls_solve(h->q, h->s, l.A, l.B, h->E, h->Qbar, h->Rbar, h->QbarN, l.C, l.D, l.CN, l.lo, l.hi, l.dx0, 1,
                       1e-8, h->have_tau ? h->tau : nullptr, h->tau, h->dX, h->dU, h->lam, nullptr, nullptr, h->hk,
                       h->d.nf ? h->hf : nullptr, info);
    if (qs < 0) return qs;
    h->have_tau = 1;
    if (hk) CUM2(cudaMemcpyAsync(hk, h->hk, (size_t)N * h->d.nc * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    if (hf && h->d.nf)
      CUM2(cudaMemcpyAsync(hf, h->hf, (size_t)h->d.nf * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  } else {
    qs = qp_solve(h->q, h->lin.dx0, 0, 0.0, h->dX, h->dU, h->lam, info);
    if (qs < 0) return qs;
  }
  const int nX = (N + 1) * nx, nU = N * nu;
  model_axpy_kernel<<<(B * nX + 255) / 256, 256, 0, h->st>>>(B, nX, X, h->dX, nullptr);
  model_axpy_kernel<<<(B * nU + 255) / 256, 256, 0, h->st>>>(B, nU, U, h->dU, nullptr);
  model_simulate_kernel<<<(B + 127) / 128, 128, 0, h->st>>>(h->m, B, x, U, W, u_applied);
  model_shift_kernel<<<(B * (nx + nu) + 127) / 128, 128, 0, h->st>>>(h->m, B, X, U);
  CUM2(cudaGetLastError());
  CUM2(cudaStreamSynchronize(h->st));
  return qs;
}

extern "C" int sqp_reset_duals(sqp_handle* h) {
  if (!h) return set_error(GPUSLS_ERR_INVALID, "sqp_reset_duals: null handle");
  h->have_tau = 0;
  return qp_reset(h->q);
}
