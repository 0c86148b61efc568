// SLS controller synthesis and reachability margins (Sec. III-D, Sec. IV-B)
// on top of the batched factorization of qp.cu (blocked schedule by default).
//
//   1. sls_build_kernel forms, for every disturbance index j, the LQR data of
//      the j-th controller problem (eq. fastsls_qp): stages k = j+1 .. N-1
//      with costs Qx = Qbar + C^T diag(tau) C, Qu = Rbar + D^T diag(tau) D,
//      Qux = D^T diag(tau) C and terminal Qx_N = QbarN + C_N^T diag(tau) C_N
//      (eq. sls_cost_matrices_tau).  With tau = 0 the costs do not depend on j
//      and one problem over stages 1 .. N-1 serves every j.
//   2. The reverse scans over the horizon (eq. robust_combin, the homogeneous
//      case of eq. combination_rules) and the gains K_k^(j) (eq. backward_prop)
//      run as one batched launch of the QP factorization kernel, one cluster
//      per problem.
//   3. sls_phi_kernel, one CTA per (j, column block), propagates Phi_x_{k+1,j} =
//      (A_k + B_k K_k^(j)) Phi_x_{k,j} from Phi_x_{j+1,j} = E_j and
//      Phi_u_{k,j} = K_k^(j) Phi_x_{k,j} (eq. forward_prop), and the row norms
//      of C_k Phi_x_{k,j} + D_k Phi_u_{k,j}; sls_margin_kernel sums them over j
//      in a fixed order into h_k and h^f (the tightenings of Sec. III-D).
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/gpusls.h"
#include "dense.cuh"
#include "internal.h"

using namespace gsls;

#define CUS(x)                                                                                      \
  do {                                                                                              \
    cudaError_t e_ = (x);                                                                           \
    if (e_ != cudaSuccess) return (void)cudaGetLastError(), set_error(GPUSLS_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct sls_handle {
  qp_dims d{};
  int precision = 0;
  int per_j = 0;
  int esz = 8;
  cudaStream_t stream = nullptr;
  qp_handle* qh = nullptr;   // internal batch of LQR problems (nc = nf = 0)
  int nq = 0;
  // FP64 pools of the internal problems (dense layouts)
  double *pA = nullptr, *pB = nullptr, *pQ = nullptr, *pR = nullptr, *pS = nullptr, *dummy = nullptr;
  size_t nA = 0, nB = 0, nQ = 0, nR = 0, nS = 0;
  // solve-precision copies of E, C, D, CN (padded)
  void *ET = nullptr, *CT = nullptr, *DT = nullptr, *CNT = nullptr;
  double *rn = nullptr, *rnf = nullptr;   // partial row sums of squares [N][N][nblk][nc], [N][nblk][nf]
  int nblk = 1;                           // column blocks of Phi_{.,j} propagated by separate CTAs
  int ldx = 0, ldu = 0;
  int solved = 0;                         // rn / rnf hold the last sls_solve
  // FastSLS alternation (per-j handles): working tau [N+1][N][max(nc, nf)],
  // tightened bounds [N nc + nf]
  double *tau = nullptr, *lo_t = nullptr, *hi_t = nullptr;
};

namespace gsls {

struct SLSBuild {
  const double *A, *B, *Qbar, *Rbar, *QbarN, *C, *D, *CN, *tau;
  double *pA, *pB, *pQ, *pR, *pS;
  int nx, nu, N, nc, nf, tw, per_j, nq;
};

// One CTA per (problem q, local stage i <= N_q): copies A_k, B_k and forms the
// cost blocks of stage k = first(q) + i (i == N_q: terminal), accumulating in
// Acc (FP64 handles: double; FP32 handles: float, whose solves round the
// blocks to FP32 anyway -- B300's FP64 rate made this kernel 7 % of a
// 75D solve).
template <typename Acc>
__global__ void sls_build_kernel(SLSBuild a) {
  extern __shared__ __align__(16) unsigned char bsm[];
  const int q = blockIdx.y, i = blockIdx.x;
  const int first = a.per_j ? q + 1 : 1;
  const int Nq = a.N - first;
  if (i > Nq) return;
  const int j = a.per_j ? q : 0;
  const int nx = a.nx, nu = a.nu, nc = a.nc, nf = a.nf;
  // offsets of problem q in the pools: problems are laid out in order
  size_t oA = 0, oQ = 0, oR = 0;
  for (int qq = 0; qq < q; ++qq) {
    const int n = a.N - (a.per_j ? qq + 1 : 1);
    oA += (size_t)n;
    oQ += (size_t)n + 1;
  }
  oR = oA;
  const int k = first + i;
  const double* tau = nullptr;
  if (a.tau) tau = a.tau + ((size_t)k * a.N + j) * a.tw;
  const int t = threadIdx.x;
  // the constraint rows in shared memory, once as loaded (Cs, Ds) and once
  // scaled by tau (CT = diag(tau) C, DT = diag(tau) D): every block entry is
  // then a short dot product over rows read from shared memory
  const int rows = i < Nq ? nc : nf;
  Acc* Cs = reinterpret_cast<Acc*>(bsm);
  Acc* CT = Cs + rows * nx;
  Acc* Ds = CT + rows * nx;
  Acc* DT = Ds + rows * nu;
  const double* Cg = i < Nq ? a.C + (size_t)k * nc * nx : a.CN;
  if (tau) {
    for (int e = t; e < rows * nx; e += blockDim.x) {
      Cs[e] = (Acc)Cg[e];
      CT[e] = (Acc)tau[e / nx] * Cs[e];
    }
    if (i < Nq)
      for (int e = t; e < nc * nu; e += blockDim.x) {
        Ds[e] = (Acc)a.D[(size_t)k * nc * nu + e];
        DT[e] = (Acc)tau[e / nu] * Ds[e];
      }
  }
  __syncthreads();
  if (i < Nq) {
    double* Ad = a.pA + (oA + i) * nx * nx;
    double* Bd = a.pB + (oA + i) * nx * nu;
    for (int e = t; e < nx * nx; e += blockDim.x) Ad[e] = a.A[(size_t)k * nx * nx + e];
    for (int e = t; e < nx * nu; e += blockDim.x) Bd[e] = a.B[(size_t)k * nx * nu + e];
    double* Qd = a.pQ + (oQ + i) * nx * nx;
    double* Rd = a.pR + (oR + i) * nu * nu;
    double* Sd = a.pS + (oR + i) * nu * nx;
    for (int e = t; e < nx * nx; e += blockDim.x) {
      const int r = e / nx, c = e - r * nx;
      Acc v = (Acc)a.Qbar[e];
      if (tau)
        for (int l = 0; l < nc; ++l) v += CT[l * nx + r] * Cs[l * nx + c];
      Qd[e] = v;
    }
    for (int e = t; e < nu * nu; e += blockDim.x) {
      const int r = e / nu, c = e - r * nu;
      Acc v = (Acc)a.Rbar[e];
      if (tau)
        for (int l = 0; l < nc; ++l) v += DT[l * nu + r] * Ds[l * nu + c];
      Rd[e] = v;
    }
    for (int e = t; e < nu * nx; e += blockDim.x) {
      const int r = e / nx, c = e - r * nx;
      Acc v = Acc(0);
      if (tau)
        for (int l = 0; l < nc; ++l) v += DT[l * nu + r] * Cs[l * nx + c];
      Sd[e] = v;
    }
  } else {
    double* Qd = a.pQ + (oQ + Nq) * nx * nx;
    for (int e = t; e < nx * nx; e += blockDim.x) {
      const int r = e / nx, c = e - r * nx;
      Acc v = (Acc)a.QbarN[e];
      if (tau)
        for (int l = 0; l < nf; ++l) v += CT[l * nx + r] * Cs[l * nx + c];
      Qd[e] = v;
    }
  }
}

// FP64 dense [count][rows][cols] -> solve precision [count][rows][ld] (zero padded)
template <typename T>
__global__ void sls_convert_kernel(const double* __restrict__ src, T* __restrict__ dst, int count, int rows, int cols,
                                   int ld) {
  const size_t total = (size_t)count * rows * ld;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t ri = e / ld;
    const int c = (int)(e - ri * ld);
    dst[e] = c < cols ? (T)src[ri * cols + c] : T(0);
  }
}

struct SLSPhi {
  const QPDesc* descs;
  const void *ET, *CT, *DT, *CNT;
  double *Phix, *Phiu, *rn, *rnf;
  int nx, nu, N, nc, nf, ldx, ldu, per_j, nblk;
};

// Shared-memory layout of sls_phi_kernel (element offsets): the block's
// columns of Phi_x_{k,j} (cur, nxt), Phi_u_{k,j} (xu) and the margin rows
// (mr), each with row pitch lw; then nbuf stage sets, each holding the
// stage's Abar_k^(j), K_k^(j), C_k (or C_N) and D_k with their padded
// pitches.  FP32 keeps two stage sets (the next stage's operands are copied
// while the current one is used); FP64, whose sets are twice the size, one.
struct PhiLayout {
  int lw, cur, nxt, xu, mr, stage, ab, kk, cc, dd, nbuf, total;
};
__host__ __device__ inline PhiLayout phi_layout(int nx, int nu, int nc, int nf, int ldx, int ldu, int nblk, int esz) {
  PhiLayout L;
  const int bw = (nx + nblk - 1) / nblk;
  const int ncf = nc > nf ? nc : nf;
  L.lw = rup4(bw);
  int off = 0;
  L.cur = off; off += rup4(nx * L.lw);
  L.nxt = off; off += rup4(nx * L.lw);
  L.xu = off; off += rup4(nu * L.lw);
  L.mr = off; off += rup4((ncf > 0 ? ncf : 1) * L.lw);
  L.ab = 0;
  L.kk = rup4(nx * ldx);
  L.cc = L.kk + rup4(nu * ldx);
  L.dd = L.cc + rup4((ncf > 0 ? ncf : 1) * ldx);
  L.stage = L.dd + rup4((nc > 0 ? nc : 1) * ldu);
  L.nbuf = esz == 4 ? 2 : 1;
  L.total = off + L.nbuf * L.stage;
  return L;
}

// One CTA per (disturbance index j, column block cb): the columns
// [c0, c1) of Phi_{.,j} evolve independently (Phi_x_{k+1,j} = Abar_k^(j)
// Phi_x_{k,j} acts on each column), so a block propagates them alone and
// leaves, per constraint row, its partial sum of squares of
// C_k Phi_x_{k,j} + D_k Phi_u_{k,j} (the block's columns) for the margins
// and duals to add up.  The block's columns stay in shared memory for the
// whole chain over k; each stage's operators are copied in (cp.async) and,
// in FP32, the next stage's while the current stage's products run.
template <typename T>
__global__ void __launch_bounds__(NT, 2) sls_phi_kernel(SLSPhi a) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* sm = reinterpret_cast<T*>(smem);
  const int j = blockIdx.x, cb = blockIdx.y, nblk = a.nblk;
  const int nx = a.nx, nu = a.nu, N = a.N, nc = a.nc, nf = a.nf, ldx = a.ldx, ldu = a.ldu;
  const int bw = (nx + nblk - 1) / nblk, c0 = cb * bw, w = min(nx, c0 + bw) - c0;
  if (w <= 0) return;
  const PhiLayout L = phi_layout(nx, nu, nc, nf, ldx, ldu, nblk, (int)sizeof(T));
  const int lw = L.lw, msz = nx * ldx, esz = (int)sizeof(T);
  const int NX = N * nx;
  const int t = threadIdx.x, wp = t >> 5, l = t & 31;
  T* cur = sm + L.cur;
  T* nxt = sm + L.nxt;
  T* Xu = sm + L.xu;
  T* M = sm + L.mr;
  T* const stg0 = sm + (L.total - L.nbuf * L.stage);
  const T* ET = reinterpret_cast<const T*>(a.ET);
  const T* CT = reinterpret_cast<const T*>(a.CT);
  const T* DT = reinterpret_cast<const T*>(a.DT);
  const T* CNT = reinterpret_cast<const T*>(a.CNT);
  const int q = a.per_j ? j : 0;
  const int first = a.per_j ? j + 1 : 1;
  const QPDesc* dq = (j + 1 < N || !a.per_j) ? &a.descs[q] : nullptr;
  // the operators of stage k into stage set sb (no wait)
  auto issue = [&](int k, int sb) {
    T* S = stg0 + (size_t)sb * L.stage;
    if (k < N) {
      const int i = k - first;   // local stage of problem q
      cta_stage(S + L.ab, reinterpret_cast<const T*>(dq->Abar) + (size_t)i * msz, msz * esz);
      cta_stage(S + L.kk, reinterpret_cast<const T*>(dq->K) + (size_t)i * nu * ldx, nu * ldx * esz);
      if (nc > 0) {
        cta_stage(S + L.cc, CT + (size_t)k * nc * ldx, nc * ldx * esz);
        cta_stage(S + L.dd, DT + (size_t)k * nc * ldu, nc * ldu * esz);
      }
    } else if (nf > 0) {
      cta_stage(S + L.cc, CNT, nf * ldx * esz);
    }
    cp_async_commit();
  };
  // Phi_x_{j+1,j} = E_j (columns c0 .. c0 + w, zero beyond w)
  for (int e = t; e < nx * lw; e += NT) {
    const int r = e / lw, c = e - r * lw;
    cur[e] = c < w ? ET[(size_t)j * msz + (size_t)r * ldx + c0 + c] : T(0);
  }
  issue(j + 1, 0);
  int sb = 0;
  for (int k = j + 1; k <= N; ++k) {
    const bool ahead = L.nbuf == 2 && k + 1 <= N;
    if (ahead) {
      issue(k + 1, sb ^ 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const T* S = stg0 + (size_t)sb * L.stage;
    // write Phi_x_{k,j} (block row k-1, block column j, columns c0 ..)
    if (a.Phix)
      for (int e = t; e < nx * w; e += NT) {
        const int r = e / w, c = e - r * w;
        a.Phix[(size_t)((k - 1) * nx + r) * NX + (size_t)j * nx + c0 + c] = (double)cur[r * lw + c];
      }
    if (k == N) {
      // terminal margin rows: C_N Phi_x_{N,j}
      if (nf > 0) {
        sgemm1<T>(nf, w, nx, T(1), S + L.cc, ldx, false, cur, lw, T(0), nullptr, 0, M, lw);
        for (int r = wp; r < nf; r += NT / 32) {
          T s2 = T(0);
          for (int c = l; c < w; c += 32) s2 += M[r * lw + c] * M[r * lw + c];
          s2 = warp_sum(s2);
          if (l == 0) a.rnf[((size_t)j * nblk + cb) * nf + r] = (double)s2;
        }
        __syncthreads();
      }
      break;
    }
    // Phi_u_{k,j} = K_k^(j) Phi_x_{k,j}
    sgemm1<T>(nu, w, nx, T(1), S + L.kk, ldx, false, cur, lw, T(0), nullptr, 0, Xu, lw);
    if (a.Phiu)
      for (int e = t; e < nu * w; e += NT) {
        const int r = e / w, c = e - r * w;
        a.Phiu[(size_t)(k * nu + r) * NX + (size_t)j * nx + c0 + c] = (double)Xu[r * lw + c];
      }
    // margin rows: C_k Phi_x + D_k Phi_u
    if (nc > 0) {
      sgemm<T>(nc, w, T(1), MTerm<T>{S + L.cc, ldx, false, cur, lw, nx}, MTerm<T>{S + L.dd, ldu, false, Xu, lw, nu},
               T(0), nullptr, 0, false, M, lw, false);
      for (int r = wp; r < nc; r += NT / 32) {
        T s2 = T(0);
        for (int c = l; c < w; c += 32) s2 += M[r * lw + c] * M[r * lw + c];
        s2 = warp_sum(s2);
        if (l == 0) a.rn[(((size_t)k * N + j) * nblk + cb) * nc + r] = (double)s2;
      }
    }
    // Phi_x_{k+1,j} = (A_k + B_k K_k^(j)) Phi_x_{k,j}
    sgemm1<T>(nx, w, nx, T(1), S + L.ab, ldx, false, cur, lw, T(0), nullptr, 0, nxt, lw);
    T* tmp = cur;
    cur = nxt;
    nxt = tmp;
    if (L.nbuf == 2) {
      sb ^= 1;
    } else if (k + 1 <= N) {
      issue(k + 1, 0);   // the products above ended with a CTA barrier: the set is free
    }
  }
}

// h_k[c] = sum_{j<k} sqrt(sum_cb rn[k][j][cb][c]) (j ascending),
// h^f[c] = sum_j sqrt(sum_cb rnf[j][cb][c]): the row norms of the column
// blocks' partial sums of squares, summed over j in a fixed order.
__global__ void sls_margin_kernel(const double* __restrict__ rn, const double* __restrict__ rnf, double* h, double* hf,
                                  int N, int nc, int nf, int nblk) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < N * nc) {
    const int k = e / nc, c = e - k * nc;
    double s = 0.0;
    for (int j = 0; j < k; ++j) {
      double q = 0.0;
      for (int b = 0; b < nblk; ++b) q += rn[(((size_t)k * N + j) * nblk + b) * nc + c];
      s += sqrt(q);
    }
    if (h) h[e] = s;
  } else if (e < N * nc + nf) {
    const int c = e - N * nc;
    double s = 0.0;
    for (int j = 0; j < N; ++j) {
      double q = 0.0;
      for (int b = 0; b < nblk; ++b) q += rnf[((size_t)j * nblk + b) * nf + c];
      s += sqrt(q);
    }
    if (hf) hf[c] = s;
  }
}

// FastSLS duals (App. B): tau_{k,j}[c] = |lam_{k,c}| / sqrt(beta_{k,j}[c] + eps)
// with beta the squared row norms of C_k Phi_x_{k,j} + D_k Phi_u_{k,j} (stage
// k < N) or C_N Phi_x_{N,j} (k = N): the sum of the column blocks' partial
// sums of squares that the last solve left in rn / rnf;
// zero for k <= j (Phi_{k,j} = 0 there) and beyond a stage's rows.  |lam|:
// a two-sided row is two one-sided rows of the same norm, at most one active.
__global__ void sls_tau_kernel(const double* __restrict__ rn, const double* __restrict__ rnf,
                               const double* __restrict__ lam, double eps, double* __restrict__ tau, int N, int nc,
                               int nf, int w, int nblk) {
  const size_t total = (size_t)(N + 1) * N * w;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / ((size_t)N * w));
    const int rem = (int)(e - (size_t)k * N * w);
    const int j = rem / w, c = rem - j * w;
    double v = 0.0;
    if (j < k) {
      if (k < N && c < nc) {
        double beta = 0.0;
        for (int b = 0; b < nblk; ++b) beta += rn[(((size_t)k * N + j) * nblk + b) * nc + c];
        v = fabs(lam[(size_t)k * nc + c]) / sqrt(beta + eps);
      } else if (k == N && c < nf) {
        double beta = 0.0;
        for (int b = 0; b < nblk; ++b) beta += rnf[((size_t)j * nblk + b) * nf + c];
        v = fabs(lam[(size_t)N * nc + c]) / sqrt(beta + eps);
      }
    }
    tau[e] = v;
  }
}

// Tightened bounds of eq. nmpc_problem_tightened: the rows of stage k move
// inwards by h_k (lo + h, hi - h), the terminal rows by h^f; infinite bounds
// stay infinite.
__global__ void fastsls_tighten_kernel(const double* __restrict__ lo, const double* __restrict__ hi,
                                       const double* __restrict__ hk, const double* __restrict__ hf,
                                       double* __restrict__ lo_t, double* __restrict__ hi_t, int N, int nc, int nf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= N * nc + nf) return;
  const double m = e < N * nc ? hk[e] : hf[e - N * nc];
  lo_t[e] = lo[e] + m;
  hi_t[e] = hi[e] - m;
}

}  // namespace gsls

extern "C" int sls_setup_ex(sls_handle** out, qp_dims d, int32_t precision, int32_t per_j_tau,
                            const qp_settings* inner, void* stream);

extern "C" int sls_setup(sls_handle** out, qp_dims d, int32_t precision, int32_t per_j_tau, void* stream) {
  return sls_setup_ex(out, d, precision, per_j_tau, nullptr, stream);
}

extern "C" int sls_setup_ex(sls_handle** out, qp_dims d, int32_t precision, int32_t per_j_tau,
                            const qp_settings* inner, void* stream) {
  if (!out) return set_error(GPUSLS_ERR_INVALID, "sls_setup: null handle pointer");
  if (d.nx < 1 || d.nx > TILE || d.nu < 1 || d.nu > 32 || d.nc < 0 || d.nc > 64 || d.nf < 0 || d.nf > 64 || d.N < 1 ||
      d.N > 512)
    return set_error(GPUSLS_ERR_INVALID, "sls_setup: dims out of range");
  if (precision != GPUSLS_FP64 && precision != GPUSLS_FP32)
    return set_error(GPUSLS_ERR_INVALID, "sls_setup: unknown precision");
  sls_handle* h = new sls_handle();
  h->d = d;
  h->precision = precision;
  h->per_j = per_j_tau ? 1 : 0;
  h->esz = precision == GPUSLS_FP64 ? 8 : 4;
  h->stream = (cudaStream_t)stream;
  h->ldx = rup4(d.nx);
  h->ldu = rup4(d.nu);
  // column blocks of about 16 columns (at most 5): more CTAs per disturbance
  // index and shorter products along each CTA's chain over k
  h->nblk = std::max(1, std::min(5, (d.nx + 15) / 16));
  const int nx = d.nx, nu = d.nu, N = d.N, nc = d.nc, nf = d.nf;
  h->nq = N >= 2 ? (h->per_j ? N - 1 : 1) : 0;
  std::vector<qp_dims> dims;
  for (int q = 0; q < h->nq; ++q) {
    const int first = h->per_j ? q + 1 : 1;
    dims.push_back({nx, nu, N - first, 0, 0});
    h->nA += (size_t)(N - first);
    h->nQ += (size_t)(N - first) + 1;
  }
  auto alloc = [&](double** p, size_t n) { return cudaMalloc(p, std::max<size_t>(n, 1) * sizeof(double)); };
  const int esz = h->esz;
  cudaError_t e = cudaSuccess;
  e = (cudaError_t)(e | alloc(&h->pA, h->nA * nx * nx));
  e = (cudaError_t)(e | alloc(&h->pB, h->nA * nx * nu));
  e = (cudaError_t)(e | alloc(&h->pQ, h->nQ * nx * nx));
  e = (cudaError_t)(e | alloc(&h->pR, h->nA * nu * nu));
  e = (cudaError_t)(e | alloc(&h->pS, h->nA * nu * nx));
  const size_t nzero = std::max<size_t>(std::max(h->nQ * nx, h->nA * nu), (size_t)std::max(N * nx, 16));
  e = (cudaError_t)(e | alloc(&h->dummy, nzero));
  e = (cudaError_t)(e | cudaMalloc(&h->ET, (size_t)N * nx * h->ldx * esz + 256));
  e = (cudaError_t)(e | cudaMalloc(&h->CT, (size_t)N * std::max(nc, 1) * h->ldx * esz + 256));
  e = (cudaError_t)(e | cudaMalloc(&h->DT, (size_t)N * std::max(nc, 1) * h->ldu * esz + 256));
  e = (cudaError_t)(e | cudaMalloc(&h->CNT, (size_t)std::max(nf, 1) * h->ldx * esz + 256));
  e = (cudaError_t)(e | alloc(&h->rn, (size_t)N * N * h->nblk * std::max(nc, 1)));
  e = (cudaError_t)(e | alloc(&h->rnf, (size_t)N * h->nblk * std::max(nf, 1)));
  if (h->per_j) {
    e = (cudaError_t)(e | alloc(&h->tau, (size_t)(N + 1) * N * std::max(std::max(nc, nf), 1)));
    e = (cudaError_t)(e | alloc(&h->lo_t, (size_t)N * nc + nf));
    e = (cudaError_t)(e | alloc(&h->hi_t, (size_t)N * nc + nf));
  }
  if (e != cudaSuccess) {
    sls_destroy(h);
    return set_error(GPUSLS_ERR_CUDA, "sls_setup: cudaMalloc failed");
  }
  cudaMemsetAsync(h->pA, 0, std::max<size_t>(h->nA * nx * nx, 1) * sizeof(double), h->stream);
  cudaMemsetAsync(h->pB, 0, std::max<size_t>(h->nA * nx * nu, 1) * sizeof(double), h->stream);
  cudaMemsetAsync(h->pQ, 0, std::max<size_t>(h->nQ * nx * nx, 1) * sizeof(double), h->stream);
  cudaMemsetAsync(h->pR, 0, std::max<size_t>(h->nA * nu * nu, 1) * sizeof(double), h->stream);
  cudaMemsetAsync(h->pS, 0, std::max<size_t>(h->nA * nu * nx, 1) * sizeof(double), h->stream);
  cudaMemsetAsync(h->dummy, 0, nzero * sizeof(double), h->stream);
  if (h->nq > 0) {
    qp_settings s;
    qp_default_settings(&s);
    // chunks of about 8 stages for the longest controller problem: measured
    // at 75D / N = 40 (39 stages), 4.40 ms at cluster 5 against 4.77 at 4,
    // 4.59 at 6 and 5.83 at 8 (more chunks mean more phase-B combines)
    s.cluster = std::min(8, std::max(1, (N - 1 + 7) / 8));
    if (inner) {   // launch shape and factorization schedule of the controller problems
      if (inner->cluster > 0) s.cluster = inner->cluster;
      s.occupancy = inner->occupancy;
      s.factorization = inner->factorization;
    }
    s.precision = precision;
    // placeholder data (zeros); every solve overwrites all problem data and
    // refactors before any use
    int st = qp_batch_setup(&h->qh, h->nq, dims.data(), h->pA, h->pB, h->dummy, h->pQ, h->pR, h->pS, h->dummy,
                            h->dummy, nullptr, nullptr, nullptr, h->dummy, h->dummy, nullptr, &s, stream);
    if (st) {
      sls_destroy(h);
      return st;
    }
  }
  *out = h;
  return GPUSLS_OK;
}

extern "C" int sls_solve(sls_handle* h, const double* A, const double* B, const double* E, const double* Qbar,
                         const double* Rbar, const double* QbarN, const double* C, const double* D, const double* CN,
                         const double* tau, double* Phi_x, double* Phi_u, double* hk, double* hf) {
  gsls::NvtxRange nvtx_("gpusls/sls_solve");
  if (!h || !A || !B || !E || !Qbar || !Rbar || !QbarN) return set_error(GPUSLS_ERR_INVALID, "sls_solve: null argument");
  const qp_dims d = h->d;
  const int nx = d.nx, nu = d.nu, N = d.N, nc = d.nc, nf = d.nf;
  if ((nc > 0 && (!C || !D)) || (nf > 0 && !CN)) return set_error(GPUSLS_ERR_INVALID, "sls_solve: C/D/CN missing");
  if (tau && !h->per_j) return set_error(GPUSLS_ERR_INVALID, "sls_solve: tau given to a handle set up without per-j tau");
  cudaStream_t st = h->stream;
  const size_t NX = (size_t)N * nx;
  if (Phi_x) CUS(cudaMemsetAsync(Phi_x, 0, NX * NX * sizeof(double), st));
  if (Phi_u) CUS(cudaMemsetAsync(Phi_u, 0, (size_t)N * nu * NX * sizeof(double), st));
  // 1. LQR data of every controller problem (cost blocks from tau)
  if (h->nq > 0) {
    SLSBuild a = {A, B, Qbar, Rbar, QbarN, C, D, CN, tau, h->pA, h->pB, h->pQ, h->pR, h->pS,
                  nx, nu, N, nc, nf, std::max(nc, nf), h->per_j, h->nq};
    dim3 grid(N, h->nq);
    const int brows = std::max(nc, nf);
    const size_t bsm = (size_t)(2 * brows * nx + 2 * nc * nu) * h->esz;
    if (h->esz == 8) {
      CUS(cudaFuncSetAttribute(sls_build_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm));
      sls_build_kernel<double><<<grid, 256, bsm, st>>>(a);
    } else {
      CUS(cudaFuncSetAttribute(sls_build_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsm));
      sls_build_kernel<float><<<grid, 256, bsm, st>>>(a);
    }
    CUS(cudaGetLastError());
    int s2 = qp_update(h->qh, h->pA, h->pB, nullptr, h->pQ, h->pR, h->pS, nullptr, nullptr, nullptr, nullptr, nullptr,
                       nullptr, nullptr);
    if (s2) return s2;
    // 2. reverse scans over the horizon and gains for every problem
    s2 = qp_refactor_internal(h->qh, true);   // gains K_k^(j) and Abar_k^(j) only
    if (s2) return s2;
  }
  // solve-precision copies of E, C, D, CN
  const int ldx = h->ldx, ldu = h->ldu;
  auto conv = [&](const double* src, void* dst, int count, int rows, int cols, int ld) {
    if (!src || count * rows == 0) return;
    if (h->esz == 8)
      sls_convert_kernel<double><<<64, 256, 0, st>>>(src, (double*)dst, count, rows, cols, ld);
    else
      sls_convert_kernel<float><<<64, 256, 0, st>>>(src, (float*)dst, count, rows, cols, ld);
  };
  conv(E, h->ET, N, nx, nx, ldx);
  conv(C, h->CT, N, nc, nx, ldx);
  conv(D, h->DT, N, nc, nu, ldu);
  conv(CN, h->CNT, 1, nf, nx, ldx);
  CUS(cudaGetLastError());
  // 3. Phi and margin row norms, one CTA per disturbance index j
  SLSPhi p = {h->qh ? h->qh->ddesc : nullptr, h->ET, h->CT, h->DT, h->CNT, Phi_x, Phi_u, h->rn, h->rnf,
              nx, nu, N, nc, nf, ldx, ldu, h->per_j, h->nblk};
  const dim3 pgrid(N, h->nblk);
  const int smem = phi_layout(nx, nu, nc, nf, ldx, ldu, h->nblk, h->esz).total * h->esz;
  if (h->esz == 8) {
    CUS(cudaFuncSetAttribute(sls_phi_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    sls_phi_kernel<double><<<pgrid, NT, smem, st>>>(p);
  } else {
    CUS(cudaFuncSetAttribute(sls_phi_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    sls_phi_kernel<float><<<pgrid, NT, smem, st>>>(p);
  }
  CUS(cudaGetLastError());
  const int tot = N * nc + nf;
  if (tot > 0) {
    sls_margin_kernel<<<(tot + 255) / 256, 256, 0, st>>>(h->rn, h->rnf, hk, hf, N, nc, nf, h->nblk);
    CUS(cudaGetLastError());
  }
  CUS(cudaStreamSynchronize(st));
  h->solved = 1;
  return GPUSLS_OK;
}

extern "C" int sls_tau(sls_handle* h, const double* lam, double eps, double* tau) {
  gsls::NvtxRange nvtx_("gpusls/sls_tau");
  if (!h || !lam || !tau) return set_error(GPUSLS_ERR_INVALID, "sls_tau: null argument");
  if (!h->solved) return set_error(GPUSLS_ERR_INVALID, "sls_tau: no sls_solve has run on this handle");
  if (!(eps > 0.0)) return set_error(GPUSLS_ERR_INVALID, "sls_tau: eps must be positive");
  const qp_dims d = h->d;
  const int w = std::max(std::max(d.nc, d.nf), 1);
  const size_t total = (size_t)(d.N + 1) * d.N * w;
  const int blocks = (int)std::min<size_t>((total + 255) / 256, 4096);
  sls_tau_kernel<<<blocks, 256, 0, h->stream>>>(h->rn, h->rnf, lam, eps, tau, d.N, d.nc, d.nf, w, h->nblk);
  CUS(cudaGetLastError());
  CUS(cudaStreamSynchronize(h->stream));
  return GPUSLS_OK;
}

extern "C" int fastsls_solve(qp_handle* q, sls_handle* s, const double* A, const double* B, const double* E,
                             const double* Qbar, const double* Rbar, const double* QbarN, const double* C,
                             const double* D, const double* CN, const double* lo, const double* hi, const double* x0,
                             int32_t iters, double eps_tau, const double* tau_in, double* tau_out, double* dx,
                             double* du, double* lam, double* Phi_x, double* Phi_u, double* hk, double* hf,
                             qp_info* info) {
  gsls::NvtxRange nvtx_("gpusls/fastsls_solve");
  if (!q || !s || !lo || !hi || !x0 || !dx || !du || !lam || !hk || (s->d.nf > 0 && !hf))
    return set_error(GPUSLS_ERR_INVALID, "fastsls_solve: null argument");
  if (!s->per_j || !s->tau) return set_error(GPUSLS_ERR_INVALID, "fastsls_solve: the SLS handle needs per-j tau");
  if (q->batch != 1) return set_error(GPUSLS_ERR_INVALID, "fastsls_solve: the QP handle must hold one QP");
  const qp_dims d = s->d, dq = q->dims[0];
  if (dq.nx != d.nx || dq.nu != d.nu || dq.N != d.N || dq.nc != d.nc || dq.nf != d.nf)
    return set_error(GPUSLS_ERR_INVALID, "fastsls_solve: QP and SLS dims differ");
  if (iters < 1) return set_error(GPUSLS_ERR_INVALID, "fastsls_solve: iters must be >= 1");
  if (!(eps_tau > 0.0)) return set_error(GPUSLS_ERR_INVALID, "fastsls_solve: eps_tau must be positive");
  const int rows = d.N * d.nc + d.nf;
  const int w = std::max(std::max(d.nc, d.nf), 1);
  const size_t ntau = (size_t)(d.N + 1) * d.N * w;
  int worst = GPUSLS_OK;
  for (int it = 0; it < iters; ++it) {
    // controller update from the previous duals (zero on the first step without tau_in)
    const double* tau_cur = it == 0 ? tau_in : s->tau;
    int st = sls_solve(s, A, B, E, Qbar, Rbar, QbarN, C, D, CN, tau_cur, Phi_x, Phi_u, hk, hf);
    if (st) return st;
    // tightened nominal QP
    if (rows > 0) {
      fastsls_tighten_kernel<<<(rows + 255) / 256, 256, 0, s->stream>>>(lo, hi, hk, d.nf > 0 ? hf : hk, s->lo_t,
                                                                         s->hi_t, d.N, d.nc, d.nf);
      CUS(cudaGetLastError());
      CUS(cudaStreamSynchronize(s->stream));
    }
    st = qp_update(q, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                   nullptr, s->lo_t, s->hi_t);
    if (st) return st;
    st = qp_solve(q, x0, 0, 0.0, dx, du, lam, info);
    if (st < 0) return st;
    if (st > worst) worst = st;
    // duals for the next controller update
    st = sls_tau(s, lam, eps_tau, s->tau);
    if (st) return st;
  }
  if (tau_out) {
    CUS(cudaMemcpyAsync(tau_out, s->tau, ntau * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
    CUS(cudaStreamSynchronize(s->stream));
  }
  return worst;
}

extern "C" void sls_destroy(sls_handle* h) {
  if (!h) return;
  if (h->qh) qp_destroy(h->qh);
  for (double* p : {h->pA, h->pB, h->pQ, h->pR, h->pS, h->dummy, h->rn, h->rnf, h->tau, h->lo_t, h->hi_t})
    if (p) cudaFree(p);
  for (void* p : {h->ET, h->CT, h->DT, h->CNT})
    if (p) cudaFree(p);
  delete h;
}
