// Instantiations of the fused kernel: FP32, up to 16 output channels, forward + adjoint.
#include "fused.cuh"
#include "launch.hpp"

namespace ace {

const void* fused_ptr_f32_n16_grad(int E, int ro, int* nt) {
  using namespace dev;
  if (E == 1 && ro == 0) {
    *nt = 256;
    return (const void*)&fused_kernel<float, 1, 16, true, 0, 256>;
  }
  if (E == 1 && ro == 1) {
    *nt = 256;
    return (const void*)&fused_kernel<float, 1, 16, true, 1, 256>;
  }
  if (E == 1 && ro == 2) {
    *nt = 256;
    return (const void*)&fused_kernel<float, 1, 16, true, 2, 256>;
  }
  if (E == 2 && ro == 0) {
    *nt = 256;
    return (const void*)&fused_kernel<float, 2, 16, true, 0, 256>;
  }
  if (E == 2 && ro == 1) {
    *nt = 256;
    return (const void*)&fused_kernel<float, 2, 16, true, 1, 256>;
  }
  if (E == 2 && ro == 2) {
    *nt = 256;
    return (const void*)&fused_kernel<float, 2, 16, true, 2, 256>;
  }
  if (E == 4 && ro == 0) {
    *nt = 256;
    return (const void*)&fused_kernel<float, 4, 16, true, 0, 256>;
  }
  if (E == 4 && ro == 1) {
    *nt = 256;
    return (const void*)&fused_kernel<float, 4, 16, true, 1, 256>;
  }
  if (E == 4 && ro == 2) {
    *nt = 256;
    return (const void*)&fused_kernel<float, 4, 16, true, 2, 256>;
  }
  return nullptr;
}

}  // namespace ace
