// FP64 instantiation of the persistent solve kernel.
#include "qp_solve_kernel.cuh"

namespace gsls {
template <typename T>
const void* qp_kernel_entry();
template <>
const void* qp_kernel_entry<double>() {
  return reinterpret_cast<const void*>(&qp_kernel<double>);
}
}  // namespace gsls
