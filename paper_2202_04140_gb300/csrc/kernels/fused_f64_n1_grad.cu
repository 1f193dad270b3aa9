// Instantiations of the fused kernel: FP64, one output channel, forward + adjoint.
#include "fused.cuh"
#include "launch.hpp"

namespace ace {

const void* fused_ptr_f64_n1_grad(int E, int ro, int* nt) {
  using namespace dev;
  if (E == 1 && ro == 0) {
    *nt = 512;
    return (const void*)&fused_kernel<double, 1, 1, true, 0, 512>;
  }
  if (E == 2 && ro == 0) {
    *nt = 512;
    return (const void*)&fused_kernel<double, 2, 1, true, 0, 512>;
  }
  if (E == 4 && ro == 0) {
    *nt = 512;
    return (const void*)&fused_kernel<double, 4, 1, true, 0, 512>;
  }
  if (E == 8 && ro == 0) {
    *nt = 512;
    return (const void*)&fused_kernel<double, 8, 1, true, 0, 512>;
  }
  return nullptr;
}

}  // namespace ace
