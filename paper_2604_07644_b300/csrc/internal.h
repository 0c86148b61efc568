// Host-side internals shared by the solver and the SLS front end (not part
// of the public C ABI).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <string>
#include <vector>

#include "../../include/gpusls.h"
#include "qp_kernel.cuh"

namespace gsls {

struct PackJob {
  const double* src;  // null: zero fill
  void* dst;
  int count, rows, cols, ld;
};

struct QPOffsets {
  size_t A, B, c, Q, R, S, q, r, C, D, CN, lohi, x0, dx, du, P, K;
};

// NVTX range over a host entry point ("gpusls/<call>"): visible to profilers
// that record NVTX (e.g. `ncu --nvtx --nvtx-include "gpusls/qp_solve/"`),
// free otherwise.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace gsls

struct qp_handle {
  int batch = 0;
  std::vector<qp_dims> dims;
  std::vector<gsls::QPOffsets> off;   // offsets into the caller's pools (elements)
  qp_settings set;
  cudaStream_t stream = nullptr;
  int esz = 8;                  // bytes of the solve precision
  int cs = 1;
  int smem = 0;
  void* tpool = nullptr;        // solve-precision workspace
  double* dpool = nullptr;      // FP64 workspace
  gsls::QPDesc* ddesc = nullptr;      // device descriptors
  std::vector<gsls::QPDesc> hdesc;
  int* info_i = nullptr;
  double* info_d = nullptr;
  gsls::PackJob* djobs = nullptr;
  size_t njobs_cap = 0;
  std::vector<void*> tx0;       // per-QP x0 (solve precision)
  double* rho0_dev = nullptr;   // [batch] setup penalties (qp_reset)
  int* order_dev = nullptr;     // [batch] launch order (settings.schedule == 1)
};

namespace gsls {
int set_error(int code, const std::string& msg);
// Learned warm start of every QP of q, enqueued on `stream` without host
// synchronization (graph-capturable).
int mlp_enqueue_warm_start(qp_handle* q, mlp_handle* h, const float* features, double rho_min, double rho_max,
                           cudaStream_t stream);
// Factorization only (MODE_RICCATI) without copying results out; gains_only
// (MODE_GAINS) skips the iteration operators.
int qp_refactor_internal(qp_handle* h, bool gains_only = false);
// Linearization features and one warm-start head (features -> network ->
// warm start of the QPs idx_dev[0..count)), enqueued on `stream` without host
// synchronization; features_smem gives the features kernel's shared memory
// for the listed QPs (host indices).
int features_smem(const qp_handle* q, const int32_t* host_idx, int count);
int enqueue_head(qp_handle* q, mlp_handle* h, const int32_t* idx_dev, int count, int smem, int n_stage,
                 const double* x0, float* feat, double rho_min, double rho_max, cudaStream_t stream);
int mlp_n_in(const mlp_handle* h);
const void* qp_features_kernel_ptr();
}  // namespace gsls
