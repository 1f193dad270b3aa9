// Instantiations of the fused kernel: FP32, one output channel, forward + adjoint.
#include "fused.cuh"
#include "launch.hpp"

namespace ace {

const void* fused_ptr_f32_n1_grad(int E, int ro, int* nt) {
  using namespace dev;
  if (E == 1 && ro == 0) {
    *nt = 1024;
    return (const void*)&fused_kernel<float, 1, 1, true, 0, 1024>;
  }
  if (E == 1 && ro == 1) {
    *nt = 1024;
    return (const void*)&fused_kernel<float, 1, 1, true, 1, 1024>;
  }
  if (E == 1 && ro == 2) {
    *nt = 1024;
    return (const void*)&fused_kernel<float, 1, 1, true, 2, 1024>;
  }
  if (E == 2 && ro == 0) {
    *nt = 1024;
    return (const void*)&fused_kernel<float, 2, 1, true, 0, 1024>;
  }
  if (E == 2 && ro == 1) {
    *nt = 1024;
    return (const void*)&fused_kernel<float, 2, 1, true, 1, 1024>;
  }
  if (E == 2 && ro == 2) {
    *nt = 1024;
    return (const void*)&fused_kernel<float, 2, 1, true, 2, 1024>;
  }
  if (E == 4 && ro == 0) {
    *nt = 768;  // 85 registers per thread (1024 threads would spill)
    return (const void*)&fused_kernel<float, 4, 1, true, 0, 768>;
  }
  if (E == 4 && ro == 1) {
    *nt = 768;  // 85 registers per thread (1024 threads would spill)
    return (const void*)&fused_kernel<float, 4, 1, true, 1, 768>;
  }
  if (E == 4 && ro == 2) {
    *nt = 768;  // 85 registers per thread (1024 threads would spill)
    return (const void*)&fused_kernel<float, 4, 1, true, 2, 768>;
  }
  if (E == 8 && ro == 0) {
    *nt = 512;
    return (const void*)&fused_kernel<float, 8, 1, true, 0, 512>;
  }
  if (E == 8 && ro == 1) {
    *nt = 512;
    return (const void*)&fused_kernel<float, 8, 1, true, 1, 512>;
  }
  if (E == 8 && ro == 2) {
    *nt = 512;
    return (const void*)&fused_kernel<float, 8, 1, true, 2, 512>;
  }
  if (E == 16 && ro == 0) {
    *nt = 512;
    return (const void*)&fused_kernel<float, 16, 1, true, 0, 512>;
  }
  if (E == 16 && ro == 1) {
    *nt = 512;
    return (const void*)&fused_kernel<float, 16, 1, true, 1, 512>;
  }
  if (E == 16 && ro == 2) {
    *nt = 512;
    return (const void*)&fused_kernel<float, 16, 1, true, 2, 512>;
  }
  return nullptr;
}

}  // namespace ace
