// Learned ADMM warm start: a 2-hidden-layer ReLU MLP trained and evaluated on
// the GPU by the library's own kernels (no counterpart in the paper).
//
//   h1 = relu(X W1^T + b1), h2 = relu(h1 W2^T + b2), Y = h2 W3^T + b3
//   loss = (1 / 2B) sum (Y - T)^2 on normalized inputs/targets
//
// Every GEMM runs on the tensor cores (mma.sync m16n8k16, BF16 operands,
// FP32 accumulation): operands are FP32 in global memory and rounded to BF16
// (round to nearest even) when staged in shared memory.  Master weights and
// the Adam moments stay FP32.  The network maps the features of a QP
// instance (x0 and linearization parameters) to (z, lambda, log rho); the
// warm-start kernel projects z onto the bounds, clamps rho and sets
// y = lambda / rho in the QP handle's ADMM state.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/gpusls.h"
#include "internal.h"

using namespace gsls;

#define CUM(x)                                                                                      \
  do {                                                                                              \
    cudaError_t e_ = (x);                                                                           \
    if (e_ != cudaSuccess) return (void)cudaGetLastError(), set_error(GPUSLS_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct mlp_handle {
  int n_in = 0, hid = 0, n_out = 0, maxb = 0;
  cudaStream_t stream = nullptr;
  float* P = nullptr;   // params: W1 [hid][n_in], b1, W2 [hid][hid], b2, W3 [n_out][hid], b3
  float* G = nullptr;   // gradients (same layout)
  float* Mm = nullptr;  // Adam first moment
  float* Vm = nullptr;  // Adam second moment
  size_t np = 0;
  size_t oW1, ob1, oW2, ob2, oW3, ob3;
  int step = 0;
  // activations [maxb][.]
  float *Xn, *Z1, *H1, *Z2, *H2, *Y, *dY, *dH, *dZ;
  float *xm, *xs, *ym, *ys;   // normalization
  float* loss;                // [1]
};

namespace gsls {

// ---------------------------------------------------------------------------
// BF16 tensor-core GEMM (mma.sync m16n8k16), generic strides:
//   C[m][n] = alpha * sum_k A(m,k) B(k,n) + beta * Cin[m][n] + bias[n]
//   A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn], all FP32 in memory.
// 64 x 64 tile per CTA, 4 warps of 32 x 32, k-slab 32.
// ---------------------------------------------------------------------------
struct GemmArgs {
  const float* A;
  const float* B;
  const float* Cin;
  const float* bias;
  float* C;
  int M, N, K;
  long long sam, sak, sbk, sbn;
  int ldc, ldcin;
  float alpha, beta;
};

constexpr int GBM = 64, GBN = 64, GBK = 32, GPAD = 8;

__device__ inline unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat16 a = __float2bfloat16_rn(lo);
  const __nv_bfloat16 b = __float2bfloat16_rn(hi);
  return (unsigned)__bfloat16_as_ushort(a) | ((unsigned)__bfloat16_as_ushort(b) << 16);
}

__global__ void __launch_bounds__(128) mlp_gemm_kernel(GemmArgs g) {
  __shared__ __align__(16) __nv_bfloat16 As[GBM][GBK + GPAD];
  __shared__ __align__(16) __nv_bfloat16 Bs[GBN][GBK + GPAD];
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int wm = w >> 1, wn = w & 1;
  const int gid = lane >> 2, tq = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
  for (int k0 = 0; k0 < g.K; k0 += GBK) {
    // stage A tile (m, k) and B tile (n, k) as BF16
    for (int e = t; e < GBM * GBK; e += 128) {
      int m, kk;
      if (g.sak == 1) { m = e / GBK; kk = e % GBK; } else { kk = e / GBM; m = e % GBM; }
      const int gm = m0 + m, gk = k0 + kk;
      float v = 0.f;
      if (gm < g.M && gk < g.K) v = g.A[gm * g.sam + gk * g.sak];
      As[m][kk] = __float2bfloat16_rn(v);
    }
    for (int e = t; e < GBN * GBK; e += 128) {
      int n, kk;
      if (g.sbk == 1) { n = e / GBK; kk = e % GBK; } else { kk = e / GBN; n = e % GBN; }
      const int gn = n0 + n, gk = k0 + kk;
      float v = 0.f;
      if (gn < g.N && gk < g.K) v = g.B[gk * g.sbk + gn * g.sbn];
      Bs[n][kk] = __float2bfloat16_rn(v);
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < GBK; ks += 16) {
      unsigned af[2][4], bfr[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int r = wm * 32 + mi * 16 + gid;
        af[mi][0] = *reinterpret_cast<const unsigned*>(&As[r][ks + 2 * tq]);
        af[mi][1] = *reinterpret_cast<const unsigned*>(&As[r + 8][ks + 2 * tq]);
        af[mi][2] = *reinterpret_cast<const unsigned*>(&As[r][ks + 2 * tq + 8]);
        af[mi][3] = *reinterpret_cast<const unsigned*>(&As[r + 8][ks + 2 * tq + 8]);
      }
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int c = wn * 32 + ni * 8 + gid;
        bfr[ni][0] = *reinterpret_cast<const unsigned*>(&Bs[c][ks + 2 * tq]);
        bfr[ni][1] = *reinterpret_cast<const unsigned*>(&Bs[c][ks + 2 * tq + 8]);
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};\n"
              : "+f"(acc[mi][ni][0]), "+f"(acc[mi][ni][1]), "+f"(acc[mi][ni][2]), "+f"(acc[mi][ni][3])
              : "r"(af[mi][0]), "r"(af[mi][1]), "r"(af[mi][2]), "r"(af[mi][3]), "r"(bfr[ni][0]), "r"(bfr[ni][1]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int m = m0 + wm * 32 + mi * 16 + gid + (c >= 2 ? 8 : 0);
        const int n = n0 + wn * 32 + ni * 8 + 2 * tq + (c & 1);
        if (m < g.M && n < g.N) {
          float v = g.alpha * acc[mi][ni][c];
          if (g.Cin) v += g.beta * g.Cin[(size_t)m * g.ldcin + n];
          if (g.bias) v += g.bias[n];
          g.C[(size_t)m * g.ldc + n] = v;
        }
      }
}

// elementwise helpers
__global__ void relu_kernel(const float* __restrict__ Z, float* __restrict__ H, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    H[i] = fmaxf(Z[i], 0.f);
}
__global__ void relu_mask_kernel(const float* __restrict__ dH, const float* __restrict__ Z, float* __restrict__ dZ,
                                 size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dZ[i] = Z[i] > 0.f ? dH[i] : 0.f;
}
// column sums of an [rows][cols] matrix into out[cols] (fixed order per column)
__global__ void colsum_kernel(const float* __restrict__ X, float* __restrict__ out, int rows, int cols) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += X[(size_t)r * cols + c];
  out[c] = s;
}
// normalize rows: out = (X - mean) / std, or out = X * std + mean (inverse)
__global__ void affine_rows_kernel(const float* __restrict__ X, float* __restrict__ out, const float* __restrict__ mean,
                                   const float* __restrict__ sd, int rows, int cols, int inverse) {
  const size_t n = (size_t)rows * cols;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % cols);
    out[i] = inverse ? X[i] * sd[c] + mean[c] : (X[i] - mean[c]) / sd[c];
  }
}
// dY = (Y - T) / B ; loss partial sums of (Y - T)^2 (one block, fixed order)
__global__ void mse_kernel(const float* __restrict__ Y, const float* __restrict__ T, float* __restrict__ dY,
                           float* loss, int B, int n) {
  __shared__ float red[256];
  const size_t tot = (size_t)B * n;
  float s = 0.f;
  for (size_t i = threadIdx.x; i < tot; i += blockDim.x) {
    const float d = Y[i] - T[i];
    dY[i] = d / (float)B;
    s += d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = 0.5f * red[0] / (float)B;
}
__global__ void adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                            float* __restrict__ V, size_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float g = G[i];
    const float m = b1 * M[i] + (1.f - b1) * g;
    const float v = b2 * V[i] + (1.f - b2) * g * g;
    M[i] = m;
    V[i] = v;
    P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  }
}
// per-column mean and standard deviation over rows (std floored at 1e-6)
__global__ void moments_kernel(const float* __restrict__ X, float* mean, float* sd, int rows, int cols) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double s = 0.0, s2 = 0.0;
  for (int r = 0; r < rows; ++r) {
    const double v = X[(size_t)r * cols + c];
    s += v;
    s2 += v * v;
  }
  const double mu = s / rows;
  const double var = fmax(s2 / rows - mu * mu, 0.0);
  mean[c] = (float)mu;
  sd[c] = (float)fmax(sqrt(var), 1e-6);
}

}  // namespace gsls

static int gemm(cudaStream_t st, const float* A, long long sam, long long sak, const float* B, long long sbk,
                long long sbn, float* C, int ldc, int M, int N, int K, const float* bias = nullptr,
                const float* Cin = nullptr, int ldcin = 0, float alpha = 1.f, float beta = 0.f) {
  GemmArgs g = {A, B, Cin, bias, C, M, N, K, sam, sak, sbk, sbn, ldc, ldcin, alpha, beta};
  dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
  mlp_gemm_kernel<<<grid, 128, 0, st>>>(g);
  CUM(cudaGetLastError());
  return GPUSLS_OK;
}

static int blocks(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 4096); }

// forward on normalized inputs Xn [B][n_in] -> h->Y (normalized outputs)
static int forward(mlp_handle* h, const float* Xn, int B) {
  const float* P = h->P;
  int st = 0;
  st |= gemm(h->stream, Xn, h->n_in, 1, P + h->oW1, 1, h->n_in, h->Z1, h->hid, B, h->hid, h->n_in, P + h->ob1);
  relu_kernel<<<blocks((size_t)B * h->hid), 256, 0, h->stream>>>(h->Z1, h->H1, (size_t)B * h->hid);
  st |= gemm(h->stream, h->H1, h->hid, 1, P + h->oW2, 1, h->hid, h->Z2, h->hid, B, h->hid, h->hid, P + h->ob2);
  relu_kernel<<<blocks((size_t)B * h->hid), 256, 0, h->stream>>>(h->Z2, h->H2, (size_t)B * h->hid);
  st |= gemm(h->stream, h->H2, h->hid, 1, P + h->oW3, 1, h->hid, h->Y, h->n_out, B, h->n_out, h->hid, P + h->ob3);
  CUM(cudaGetLastError());
  return st ? GPUSLS_ERR_CUDA : GPUSLS_OK;
}

// gradients of the MSE loss for normalized (Xn, Tn) into h->G
static int backward(mlp_handle* h, const float* Xn, const float* Tn, int B) {
  const float* P = h->P;
  float* G = h->G;
  int st = forward(h, Xn, B);
  mse_kernel<<<1, 256, 0, h->stream>>>(h->Y, Tn, h->dY, h->loss, B, h->n_out);
  // layer 3: gW3 = dY^T H2 [n_out][hid], gb3 = colsum dY, dH2 = dY W3 [B][hid]
  st |= gemm(h->stream, h->dY, 1, h->n_out, h->H2, h->hid, 1, G + h->oW3, h->hid, h->n_out, h->hid, B);
  colsum_kernel<<<(h->n_out + 255) / 256, 256, 0, h->stream>>>(h->dY, G + h->ob3, B, h->n_out);
  st |= gemm(h->stream, h->dY, h->n_out, 1, P + h->oW3, h->hid, 1, h->dH, h->hid, B, h->hid, h->n_out);
  relu_mask_kernel<<<blocks((size_t)B * h->hid), 256, 0, h->stream>>>(h->dH, h->Z2, h->dZ, (size_t)B * h->hid);
  // layer 2
  st |= gemm(h->stream, h->dZ, 1, h->hid, h->H1, h->hid, 1, G + h->oW2, h->hid, h->hid, h->hid, B);
  colsum_kernel<<<(h->hid + 255) / 256, 256, 0, h->stream>>>(h->dZ, G + h->ob2, B, h->hid);
  st |= gemm(h->stream, h->dZ, h->hid, 1, P + h->oW2, h->hid, 1, h->dH, h->hid, B, h->hid, h->hid);
  relu_mask_kernel<<<blocks((size_t)B * h->hid), 256, 0, h->stream>>>(h->dH, h->Z1, h->dZ, (size_t)B * h->hid);
  // layer 1
  st |= gemm(h->stream, h->dZ, 1, h->hid, Xn, h->n_in, 1, G + h->oW1, h->n_in, h->hid, h->n_in, B);
  colsum_kernel<<<(h->hid + 255) / 256, 256, 0, h->stream>>>(h->dZ, G + h->ob1, B, h->hid);
  CUM(cudaGetLastError());
  return st ? GPUSLS_ERR_CUDA : GPUSLS_OK;
}

extern "C" int mlp_create(mlp_handle** out, int32_t n_in, int32_t hidden, int32_t n_out, int32_t max_batch,
                          void* stream) {
  if (!out || n_in < 1 || hidden < 1 || n_out < 1 || max_batch < 1)
    return set_error(GPUSLS_ERR_INVALID, "mlp_create: invalid dimensions");
  mlp_handle* h = new mlp_handle();
  h->n_in = n_in;
  h->hid = hidden;
  h->n_out = n_out;
  h->maxb = max_batch;
  h->stream = (cudaStream_t)stream;
  h->oW1 = 0;
  h->ob1 = h->oW1 + (size_t)hidden * n_in;
  h->oW2 = h->ob1 + hidden;
  h->ob2 = h->oW2 + (size_t)hidden * hidden;
  h->oW3 = h->ob2 + hidden;
  h->ob3 = h->oW3 + (size_t)n_out * hidden;
  h->np = h->ob3 + n_out;
  const size_t B = max_batch;
  size_t act = B * n_in + 4 * B * hidden + 2 * B * n_out + 2 * B * std::max(hidden, n_out);
  float* base = nullptr;
  const size_t tot = 4 * h->np + act + 2 * (size_t)n_in + 2 * (size_t)n_out + 16;
  if (cudaMalloc(&base, tot * sizeof(float)) != cudaSuccess) {
    delete h;
    return set_error(GPUSLS_ERR_CUDA, "mlp_create: cudaMalloc failed");
  }
  cudaMemsetAsync(base, 0, tot * sizeof(float), h->stream);
  float* p = base;
  auto take = [&](size_t n) { float* r = p; p += n; return r; };
  h->P = take(h->np); h->G = take(h->np); h->Mm = take(h->np); h->Vm = take(h->np);
  h->Xn = take(B * n_in); h->Z1 = take(B * hidden); h->H1 = take(B * hidden); h->Z2 = take(B * hidden);
  h->H2 = take(B * hidden); h->Y = take(B * n_out); h->dY = take(B * n_out);
  h->dH = take(B * std::max(hidden, n_out)); h->dZ = take(B * std::max(hidden, n_out));
  h->xm = take(n_in); h->xs = take(n_in); h->ym = take(n_out); h->ys = take(n_out); h->loss = take(16);
  // identity normalization until mlp_fit_normalization / mlp_set_normalization
  std::vector<float> ones(std::max(n_in, n_out), 1.f);
  cudaMemcpyAsync(h->xs, ones.data(), n_in * sizeof(float), cudaMemcpyHostToDevice, h->stream);
  cudaMemcpyAsync(h->ys, ones.data(), n_out * sizeof(float), cudaMemcpyHostToDevice, h->stream);
  cudaStreamSynchronize(h->stream);
  *out = h;
  return GPUSLS_OK;
}

static int params_io(mlp_handle* h, float* const* dst, const float* const* src, bool set) {
  const size_t offs[6] = {h->oW1, h->ob1, h->oW2, h->ob2, h->oW3, h->ob3};
  const size_t cnt[6] = {(size_t)h->hid * h->n_in, (size_t)h->hid, (size_t)h->hid * h->hid, (size_t)h->hid,
                         (size_t)h->n_out * h->hid, (size_t)h->n_out};
  for (int i = 0; i < 6; ++i) {
    if (set) {
      if (!src[i]) return set_error(GPUSLS_ERR_INVALID, "mlp_set_params: null parameter");
      CUM(cudaMemcpyAsync(h->P + offs[i], src[i], cnt[i] * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    } else if (dst[i]) {
      CUM(cudaMemcpyAsync(dst[i], h->P + offs[i], cnt[i] * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    }
  }
  if (set) {   // new parameters restart the optimizer state
    CUM(cudaMemsetAsync(h->Mm, 0, h->np * sizeof(float), h->stream));
    CUM(cudaMemsetAsync(h->Vm, 0, h->np * sizeof(float), h->stream));
    h->step = 0;
  }
  CUM(cudaStreamSynchronize(h->stream));
  return GPUSLS_OK;
}

extern "C" int mlp_set_params(mlp_handle* h, const float* W1, const float* b1, const float* W2, const float* b2,
                              const float* W3, const float* b3) {
  if (!h) return set_error(GPUSLS_ERR_INVALID, "mlp_set_params: null handle");
  const float* src[6] = {W1, b1, W2, b2, W3, b3};
  return params_io(h, nullptr, src, true);
}

extern "C" int mlp_get_params(mlp_handle* h, float* W1, float* b1, float* W2, float* b2, float* W3, float* b3) {
  if (!h) return set_error(GPUSLS_ERR_INVALID, "mlp_get_params: null handle");
  float* dst[6] = {W1, b1, W2, b2, W3, b3};
  return params_io(h, dst, nullptr, false);
}

extern "C" int mlp_fit_normalization(mlp_handle* h, const float* X, const float* T, int32_t count) {
  if (!h || !X || !T || count < 1) return set_error(GPUSLS_ERR_INVALID, "mlp_fit_normalization: invalid argument");
  moments_kernel<<<(h->n_in + 127) / 128, 128, 0, h->stream>>>(X, h->xm, h->xs, count, h->n_in);
  moments_kernel<<<(h->n_out + 127) / 128, 128, 0, h->stream>>>(T, h->ym, h->ys, count, h->n_out);
  CUM(cudaGetLastError());
  CUM(cudaStreamSynchronize(h->stream));
  return GPUSLS_OK;
}

extern "C" int mlp_set_normalization(mlp_handle* h, const float* xm, const float* xs, const float* ym, const float* ys) {
  if (!h || !xm || !xs || !ym || !ys) return set_error(GPUSLS_ERR_INVALID, "mlp_set_normalization: null argument");
  CUM(cudaMemcpyAsync(h->xm, xm, h->n_in * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  CUM(cudaMemcpyAsync(h->xs, xs, h->n_in * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  CUM(cudaMemcpyAsync(h->ym, ym, h->n_out * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  CUM(cudaMemcpyAsync(h->ys, ys, h->n_out * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  CUM(cudaStreamSynchronize(h->stream));
  return GPUSLS_OK;
}

extern "C" int mlp_get_normalization(mlp_handle* h, float* xm, float* xs, float* ym, float* ys) {
  if (!h) return set_error(GPUSLS_ERR_INVALID, "mlp_get_normalization: null handle");
  if (xm) CUM(cudaMemcpyAsync(xm, h->xm, h->n_in * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  if (xs) CUM(cudaMemcpyAsync(xs, h->xs, h->n_in * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  if (ym) CUM(cudaMemcpyAsync(ym, h->ym, h->n_out * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  if (ys) CUM(cudaMemcpyAsync(ys, h->ys, h->n_out * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  CUM(cudaStreamSynchronize(h->stream));
  return GPUSLS_OK;
}

// Host image of a network in the file layout of mlp_save: parameters in the
// mlp_set_params order, then the normalization.
static std::vector<std::pair<float*, size_t>> file_fields(mlp_handle* h) {
  return {{h->P + h->oW1, (size_t)h->hid * h->n_in}, {h->P + h->ob1, (size_t)h->hid},
          {h->P + h->oW2, (size_t)h->hid * h->hid}, {h->P + h->ob2, (size_t)h->hid},
          {h->P + h->oW3, (size_t)h->n_out * h->hid}, {h->P + h->ob3, (size_t)h->n_out},
          {h->xm, (size_t)h->n_in}, {h->xs, (size_t)h->n_in}, {h->ym, (size_t)h->n_out}, {h->ys, (size_t)h->n_out}};
}

static const char MLP_FILE_TAG[8] = {'G', 'S', 'L', 'S', 'M', 'L', 'P', '1'};

extern "C" int mlp_save(mlp_handle* h, const char* path) {
  if (!h || !path) return set_error(GPUSLS_ERR_INVALID, "mlp_save: null argument");
  std::vector<float> buf;
  for (auto& f : file_fields(h)) {
    const size_t o = buf.size();
    buf.resize(o + f.second);
    CUM(cudaMemcpyAsync(buf.data() + o, f.first, f.second * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  }
  CUM(cudaStreamSynchronize(h->stream));
  FILE* fp = fopen(path, "wb");
  if (!fp) return set_error(GPUSLS_ERR_INVALID, std::string("mlp_save: cannot open ") + path);
  const int32_t dims[3] = {h->n_in, h->hid, h->n_out};
  const bool ok = fwrite(MLP_FILE_TAG, 1, 8, fp) == 8 && fwrite(dims, sizeof(int32_t), 3, fp) == 3 &&
                  fwrite(buf.data(), sizeof(float), buf.size(), fp) == buf.size();
  if (fclose(fp) != 0 || !ok) return set_error(GPUSLS_ERR_INVALID, std::string("mlp_save: write failed: ") + path);
  return GPUSLS_OK;
}

extern "C" int mlp_load(mlp_handle* h, const char* path) {
  if (!h || !path) return set_error(GPUSLS_ERR_INVALID, "mlp_load: null argument");
  FILE* fp = fopen(path, "rb");
  if (!fp) return set_error(GPUSLS_ERR_INVALID, std::string("mlp_load: cannot open ") + path);
  char tag[8] = {};
  int32_t dims[3] = {};
  const auto fields = file_fields(h);
  size_t total = 0;
  for (auto& f : fields) total += f.second;
  std::vector<float> buf(total);
  bool ok = fread(tag, 1, 8, fp) == 8 && memcmp(tag, MLP_FILE_TAG, 8) == 0 && fread(dims, sizeof(int32_t), 3, fp) == 3;
  ok = ok && dims[0] == h->n_in && dims[1] == h->hid && dims[2] == h->n_out;
  ok = ok && fread(buf.data(), sizeof(float), total, fp) == total;
  char extra;
  ok = ok && fread(&extra, 1, 1, fp) == 0;   // nothing after the last field
  fclose(fp);
  if (!ok)
    return set_error(GPUSLS_ERR_INVALID, std::string("mlp_load: not a network of this handle's sizes: ") + path);
  size_t o = 0;
  for (auto& f : fields) {
    CUM(cudaMemcpyAsync(f.first, buf.data() + o, f.second * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    o += f.second;
  }
  // new parameters restart the optimizer state
  CUM(cudaMemsetAsync(h->Mm, 0, h->np * sizeof(float), h->stream));
  CUM(cudaMemsetAsync(h->Vm, 0, h->np * sizeof(float), h->stream));
  h->step = 0;
  CUM(cudaStreamSynchronize(h->stream));   // buf is released on return
  return GPUSLS_OK;
}

extern "C" int mlp_forward(mlp_handle* h, const float* X, int32_t B, float* Y) {
  if (!h || !X || !Y || B < 1 || B > h->maxb) return set_error(GPUSLS_ERR_INVALID, "mlp_forward: invalid argument");
  affine_rows_kernel<<<blocks((size_t)B * h->n_in), 256, 0, h->stream>>>(X, h->Xn, h->xm, h->xs, B, h->n_in, 0);
  int st = forward(h, h->Xn, B);
  if (st) return st;
  affine_rows_kernel<<<blocks((size_t)B * h->n_out), 256, 0, h->stream>>>(h->Y, Y, h->ym, h->ys, B, h->n_out, 1);
  CUM(cudaGetLastError());
  CUM(cudaStreamSynchronize(h->stream));
  return GPUSLS_OK;
}

extern "C" int mlp_gradients(mlp_handle* h, const float* Xn, const float* Tn, int32_t B, float* grads, float* loss) {
  if (!h || !Xn || !Tn || B < 1 || B > h->maxb) return set_error(GPUSLS_ERR_INVALID, "mlp_gradients: invalid argument");
  int st = backward(h, Xn, Tn, B);
  if (st) return st;
  if (grads) CUM(cudaMemcpyAsync(grads, h->G, h->np * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  if (loss) CUM(cudaMemcpyAsync(loss, h->loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  CUM(cudaStreamSynchronize(h->stream));
  return GPUSLS_OK;
}

extern "C" int mlp_train_step(mlp_handle* h, const float* X, const float* T, int32_t B, float lr, float* loss) {
  gsls::NvtxRange nvtx_("gpusls/mlp_train_step");
  if (!h || !X || !T || B < 1 || B > h->maxb) return set_error(GPUSLS_ERR_INVALID, "mlp_train_step: invalid argument");
  // normalized inputs and targets (targets into dH scratch region sized B * max(hid, n_out))
  affine_rows_kernel<<<blocks((size_t)B * h->n_in), 256, 0, h->stream>>>(X, h->Xn, h->xm, h->xs, B, h->n_in, 0);
  float* Tn = h->dZ;   // reuse: backward() overwrites dZ only after mse_kernel consumed Tn
  affine_rows_kernel<<<blocks((size_t)B * h->n_out), 256, 0, h->stream>>>(T, Tn, h->ym, h->ys, B, h->n_out, 0);
  int st = backward(h, h->Xn, Tn, B);
  if (st) return st;
  h->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)h->step), c2 = 1.f - powf(b2, (float)h->step);
  adam_kernel<<<blocks(h->np), 256, 0, h->stream>>>(h->P, h->G, h->Mm, h->Vm, h->np, lr, b1, b2, 1e-8f, c1, c2);
  CUM(cudaGetLastError());
  if (loss) CUM(cudaMemcpyAsync(loss, h->loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  CUM(cudaStreamSynchronize(h->stream));
  return GPUSLS_OK;
}

extern "C" void mlp_destroy(mlp_handle* h) {
  if (!h) return;
  if (h->P) cudaFree(h->P);
  delete h;
}

// ---------------------------------------------------------------------------
// warm start of a QP handle from the network's output
// ---------------------------------------------------------------------------
namespace gsls {
template <typename T>
__global__ void warm_assemble_kernel(const QPDesc* __restrict__ descs, const float* __restrict__ Y, int ldy,
                                     double rho_lo, double rho_hi) {
  const QPDesc d = descs[blockIdx.x];
  const float* y = Y + (size_t)blockIdx.x * ldy;
  const int m = d.m;
  double rho = exp((double)y[2 * m]);
  rho = fmin(fmax(rho, rho_lo), rho_hi);
  T* z = reinterpret_cast<T*>(d.z);
  T* yy = reinterpret_cast<T*>(d.y);
  const T* lo = reinterpret_cast<const T*>(d.lo);
  const T* hi = reinterpret_cast<const T*>(d.hi);
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const T zz = fmin(fmax((T)y[i], lo[i]), hi[i]);
    z[i] = zz;
    yy[i] = (T)((double)y[m + i] / rho);
  }
  if (threadIdx.x == 0) {
    if (d.rho[0] != rho) d.flags[0] = 0;
    d.rho[0] = rho;
    d.flags[1] = 1;   // warm-started: eligible for the cold fallback
  }
}
}  // namespace gsls

// Enqueues the learned warm start of every QP of q on `stream` (no host
// synchronization and no host copies, so it can be captured into a graph).
int gsls::mlp_enqueue_warm_start(qp_handle* q, mlp_handle* h, const float* features, double rho_min,
                                 double rho_max, cudaStream_t stream) {
  if (!q || !h || !features) return set_error(GPUSLS_ERR_INVALID, "qp_warm_start_mlp: null argument");
  if (q->batch > h->maxb) return set_error(GPUSLS_ERR_INVALID, "qp_warm_start_mlp: batch exceeds the network's max batch");
  for (int b = 0; b < q->batch; ++b) {
    const int m = q->dims[b].N * q->dims[b].nc + q->dims[b].nf;
    if (2 * m + 1 != h->n_out)
      return set_error(GPUSLS_ERR_INVALID, "qp_warm_start_mlp: network output size must be 2 m + 1 for every QP");
  }
  const cudaStream_t saved = h->stream;
  h->stream = stream;
  affine_rows_kernel<<<blocks((size_t)q->batch * h->n_in), 256, 0, stream>>>(features, h->Xn, h->xm, h->xs,
                                                                              q->batch, h->n_in, 0);
  int st = forward(h, h->Xn, q->batch);
  h->stream = saved;
  if (st) return st;
  float* Yd = h->dY;   // denormalized outputs
  affine_rows_kernel<<<blocks((size_t)q->batch * h->n_out), 256, 0, stream>>>(h->Y, Yd, h->ym, h->ys, q->batch,
                                                                               h->n_out, 1);
  if (q->esz == 8)
    warm_assemble_kernel<double><<<q->batch, 256, 0, stream>>>(q->ddesc, Yd, h->n_out, rho_min, rho_max);
  else
    warm_assemble_kernel<float><<<q->batch, 256, 0, stream>>>(q->ddesc, Yd, h->n_out, rho_min, rho_max);
  CUM(cudaGetLastError());
  return GPUSLS_OK;
}

extern "C" int qp_warm_start_mlp(qp_handle* q, mlp_handle* h, const float* features, double rho_min, double rho_max) {
  if (!h) return set_error(GPUSLS_ERR_INVALID, "qp_warm_start_mlp: null argument");
  const int st = gsls::mlp_enqueue_warm_start(q, h, features, rho_min, rho_max, h->stream);
  if (st) return st;
  CUM(cudaStreamSynchronize(h->stream));
  return GPUSLS_OK;
}

// ---------------------------------------------------------------------------
// Linearization features and per-family warm-start heads
// ---------------------------------------------------------------------------
namespace gsls {

// +-1 from a 32-bit mix of (salt, row l, input index e) (the finalizer of
// MurmurHash3): a fixed Rademacher projection that needs no stored matrix.
__device__ inline float rad_sign(unsigned salt, unsigned l, unsigned e) {
  unsigned h = salt * 0x9E3779B1u ^ (l + 0x7F4A7C15u) * 0x85EBCA77u ^ (e + 0x165667B1u) * 0xC2B2AE3Du;
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return (h & 1u) ? 1.f : -1.f;
}

// Block sum of one value per thread (blockDim.x == 256), result to all threads.
__device__ inline float feat_block_sum(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float s = 0.f;
  for (int w = 0; w < 8; ++w) s += red[w];
  return s;
}

// One CTA per listed QP: row i of out = [x0 (nx), p projections each of
// mean_k (A_k - I), mean_k B_k, mean_k q_k (k = 0..N) and the mean of the
// finite upper bounds of each stage row (clamped to +-10), N / 128].
__global__ void __launch_bounds__(256) qp_features_kernel(const QPDesc* __restrict__ descs, const int* __restrict__ idx,
                                                          const double* __restrict__ x064_base,
                                                          const double* __restrict__ x0, int p, int ld,
                                                          float* __restrict__ out) {
  extern __shared__ float fsm[];
  __shared__ float red[8];
  const int b = idx ? idx[blockIdx.x] : (int)blockIdx.x;
  const QPDesc& d = descs[b];
  const int nx = d.nx, nu = d.nu, N = d.N, nc = d.nc, t = threadIdx.x;
  float* row = out + (size_t)blockIdx.x * ld;
  const double* xb = x0 + (d.x064 - x064_base);
  for (int i = t; i < nx; i += blockDim.x) row[i] = (float)xb[i];
  float* mA = fsm;                      // [nx * nx]
  float* mB = mA + nx * nx;             // [nx * nu]
  float* mq = mB + nx * nu;             // [nx]
  float* mh = mq + nx;                  // [nc]
  const double invN = 1.0 / N;
  for (int e = t; e < nx * nx; e += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < N; ++k) s += d.A64[(size_t)k * nx * nx + e];
    mA[e] = (float)(s * invN - ((e % (nx + 1)) == 0 ? 1.0 : 0.0));
  }
  for (int e = t; e < nx * nu; e += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < N; ++k) s += d.B64[(size_t)k * nx * nu + e];
    mB[e] = (float)(s * invN);
  }
  for (int e = t; e < nx; e += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k <= N; ++k) s += d.q64[(size_t)k * nx + e];
    mq[e] = (float)(s / (N + 1));
  }
  for (int e = t; e < nc; e += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < N; ++k) {
      const double h = d.hi64[(size_t)k * nc + e];
      s += isfinite(h) ? fmin(fmax(h, -10.0), 10.0) : 0.0;
    }
    mh[e] = (float)(s * invN);
  }
  __syncthreads();
  const float sA = rsqrtf((float)(nx * nx)), sB = rsqrtf((float)(nx * nu)), sq = rsqrtf((float)nx),
              sh = nc > 0 ? rsqrtf((float)nc) : 0.f;
  for (int l = 0; l < p; ++l) {
    float a = 0.f, bb = 0.f, q = 0.f, h = 0.f;
    for (int e = t; e < nx * nx; e += blockDim.x) a += rad_sign(1u, l, e) * mA[e];
    for (int e = t; e < nx * nu; e += blockDim.x) bb += rad_sign(2u, l, e) * mB[e];
    for (int e = t; e < nx; e += blockDim.x) q += rad_sign(3u, l, e) * mq[e];
    for (int e = t; e < nc; e += blockDim.x) h += rad_sign(4u, l, e) * mh[e];
    a = feat_block_sum(a, red);
    bb = feat_block_sum(bb, red);
    q = feat_block_sum(q, red);
    h = feat_block_sum(h, red);
    if (t == 0) {
      row[nx + l] = a * sA;
      row[nx + p + l] = bb * sB;
      row[nx + 2 * p + l] = q * sq;
      row[nx + 3 * p + l] = h * sh;
    }
  }
  if (t == 0) row[nx + 4 * p] = (float)N / 128.f;
}

// Warm start of the listed QPs from a head's denormalized outputs Y [count]
// [ldy] laid out for horizon n_stage (>= each QP's N): z stage rows, z
// terminal rows, lambda stage rows, lambda terminal rows, log rho.
template <typename T>
__global__ void warm_assemble_heads_kernel(const QPDesc* __restrict__ descs, const int* __restrict__ idx,
                                           const float* __restrict__ Y, int ldy, int n_stage, double rho_lo,
                                           double rho_hi) {
  const int b = idx ? idx[blockIdx.x] : (int)blockIdx.x;
  const QPDesc d = descs[b];
  const float* y = Y + (size_t)blockIdx.x * ldy;
  const int m = d.m, ns = d.N * d.nc, mmax = n_stage * d.nc + d.nf;
  double rho = exp((double)y[2 * mmax]);
  rho = fmin(fmax(rho, rho_lo), rho_hi);
  T* z = reinterpret_cast<T*>(d.z);
  T* yy = reinterpret_cast<T*>(d.y);
  const T* lo = reinterpret_cast<const T*>(d.lo);
  const T* hi = reinterpret_cast<const T*>(d.hi);
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const int src = i < ns ? i : n_stage * d.nc + (i - ns);
    const T zz = fmin(fmax((T)y[src], lo[i]), hi[i]);
    z[i] = zz;
    yy[i] = (T)((double)y[mmax + src] / rho);
  }
  if (threadIdx.x == 0) {
    if (d.rho[0] != rho) d.flags[0] = 0;
    d.rho[0] = rho;
    d.flags[1] = 1;
  }
}

int features_smem(const qp_handle* q, const int32_t* host_idx, int count) {
  int mx = 0;
  for (int i = 0; i < (host_idx ? count : q->batch); ++i) {
    const qp_dims& d = q->dims[host_idx ? host_idx[i] : i];
    mx = std::max(mx, (d.nx * d.nx + d.nx * d.nu + d.nx + d.nc) * (int)sizeof(float));
  }
  return mx;
}

// Features of the QPs idx[0..count) into out [count][ld] on `stream`.
int enqueue_features(qp_handle* q, const int32_t* idx_dev, int count, int smem, const double* x0, int p, int ld,
                     float* out, cudaStream_t stream) {
  qp_features_kernel<<<count, 256, smem, stream>>>(q->ddesc, idx_dev, q->hdesc[0].x064, x0, p, ld, out);
  CUM(cudaGetLastError());
  return GPUSLS_OK;
}

// One head: features -> network -> warm start of its QPs, all on `stream`.
int enqueue_head(qp_handle* q, mlp_handle* h, const int32_t* idx_dev, int count, int smem, int n_stage,
                 const double* x0, float* feat, double rho_min, double rho_max, cudaStream_t stream) {
  if (count > h->maxb) return set_error(GPUSLS_ERR_INVALID, "warm-start head: more QPs than the network's max batch");
  int st = enqueue_features(q, idx_dev, count, smem, x0, GPUSLS_FEATURE_P, h->n_in, feat, stream);
  if (st) return st;
  const cudaStream_t saved = h->stream;
  h->stream = stream;
  affine_rows_kernel<<<blocks((size_t)count * h->n_in), 256, 0, stream>>>(feat, h->Xn, h->xm, h->xs, count, h->n_in,
                                                                           0);
  st = forward(h, h->Xn, count);
  h->stream = saved;
  if (st) return st;
  float* Yd = h->dY;
  affine_rows_kernel<<<blocks((size_t)count * h->n_out), 256, 0, stream>>>(h->Y, Yd, h->ym, h->ys, count, h->n_out, 1);
  if (q->esz == 8)
    warm_assemble_heads_kernel<double><<<count, 256, 0, stream>>>(q->ddesc, idx_dev, Yd, h->n_out, n_stage, rho_min,
                                                                  rho_max);
  else
    warm_assemble_heads_kernel<float><<<count, 256, 0, stream>>>(q->ddesc, idx_dev, Yd, h->n_out, n_stage, rho_min,
                                                                 rho_max);
  CUM(cudaGetLastError());
  return GPUSLS_OK;
}

int mlp_n_in(const mlp_handle* h) { return h->n_in; }
const void* qp_features_kernel_ptr() { return reinterpret_cast<const void*>(qp_features_kernel); }

}  // namespace gsls

extern "C" int qp_features(qp_handle* q, const double* x0, const int32_t* idx, int32_t count, int32_t ld,
                           float* out) {
  if (!q || !x0 || !out || count < 1 || (!idx && count != q->batch))
    return set_error(GPUSLS_ERR_INVALID, "qp_features: invalid argument");
  std::vector<int32_t> hidx;
  if (idx) {
    hidx.resize(count);
    CUM(cudaMemcpy(hidx.data(), idx, count * sizeof(int32_t), cudaMemcpyDeviceToHost));
  }
  for (int i = 0; i < count; ++i) {
    const int b = idx ? hidx[i] : i;
    if (b < 0 || b >= q->batch) return set_error(GPUSLS_ERR_INVALID, "qp_features: index out of range");
    if (q->dims[b].nx + 4 * GPUSLS_FEATURE_P + 1 > ld)
      return set_error(GPUSLS_ERR_INVALID, "qp_features: ld < nx + 4 GPUSLS_FEATURE_P + 1");
  }
  const int smem = gsls::features_smem(q, idx ? hidx.data() : nullptr, count);
  CUM(cudaFuncSetAttribute(gsls::qp_features_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int st = gsls::enqueue_features(q, idx, count, smem, x0, GPUSLS_FEATURE_P, ld, out, q->stream);
  if (st) return st;
  CUM(cudaStreamSynchronize(q->stream));
  return GPUSLS_OK;
}

namespace {
// host-side checks of a head list; fills the shared-memory need per head
int check_heads(qp_handle* q, int32_t n_heads, mlp_handle* const* heads, const int32_t* const* idx,
                const int32_t* counts, const int32_t* n_stage, std::vector<int>& smem) {
  if (!q || n_heads < 1 || !heads || !idx || !counts || !n_stage)
    return set_error(GPUSLS_ERR_INVALID, "warm-start heads: null argument");
  smem.assign(n_heads, 0);
  std::vector<int> seen(q->batch, 0);
  for (int hh = 0; hh < n_heads; ++hh) {
    mlp_handle* h = heads[hh];
    if (!h || !idx[hh] || counts[hh] < 1 || counts[hh] > h->maxb)
      return set_error(GPUSLS_ERR_INVALID, "warm-start heads: bad head, index list or count");
    std::vector<int32_t> hidx(counts[hh]);
    CUM(cudaMemcpy(hidx.data(), idx[hh], counts[hh] * sizeof(int32_t), cudaMemcpyDeviceToHost));
    for (int i = 0; i < counts[hh]; ++i) {
      const int b = hidx[i];
      if (b < 0 || b >= q->batch || seen[b]++)
        return set_error(GPUSLS_ERR_INVALID, "warm-start heads: QP index out of range or listed twice");
      const qp_dims& d = q->dims[b];
      if (d.N > n_stage[hh] || h->n_in != d.nx + 4 * GPUSLS_FEATURE_P + 1 ||
          h->n_out != 2 * (n_stage[hh] * d.nc + d.nf) + 1)
        return set_error(GPUSLS_ERR_INVALID, "warm-start heads: network sizes do not match QP " + std::to_string(b));
    }
    smem[hh] = gsls::features_smem(q, hidx.data(), counts[hh]);
  }
  CUM(cudaFuncSetAttribute(gsls::qp_features_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           *std::max_element(smem.begin(), smem.end())));
  return GPUSLS_OK;
}
}  // namespace

extern "C" int qp_warm_start_heads(qp_handle* q, int32_t n_heads, mlp_handle* const* heads,
                                   const int32_t* const* idx, const int32_t* counts, const int32_t* n_stage,
                                   const double* x0, double rho_min, double rho_max) {
  gsls::NvtxRange nvtx_("gpusls/qp_warm_start_heads");
  std::vector<int> smem;
  int st = check_heads(q, n_heads, heads, idx, counts, n_stage, smem);
  if (st) return st;
  if (!x0) return set_error(GPUSLS_ERR_INVALID, "qp_warm_start_heads: null x0");
  for (int hh = 0; hh < n_heads; ++hh) {
    float* feat = nullptr;
    CUM(cudaMalloc(&feat, (size_t)counts[hh] * heads[hh]->n_in * sizeof(float)));
    st = gsls::enqueue_head(q, heads[hh], idx[hh], counts[hh], smem[hh], n_stage[hh], x0, feat, rho_min, rho_max,
                            q->stream);
    cudaError_t e = cudaStreamSynchronize(q->stream);
    cudaFree(feat);
    if (st) return st;
    if (e != cudaSuccess) return set_error(GPUSLS_ERR_CUDA, std::string("qp_warm_start_heads: ") + cudaGetErrorString(e));
  }
  return GPUSLS_OK;
}
