// Selects the compiled instantiation of the fused kernel.
#include "launch.hpp"

namespace ace {

const void* fused_ptr_f32_n1_fwd(int E, int ro, int* nt);
const void* fused_ptr_f32_n1_grad(int E, int ro, int* nt);
const void* fused_ptr_f32_n16_fwd(int E, int ro, int* nt);
const void* fused_ptr_f32_n16_grad(int E, int ro, int* nt);
const void* fused_ptr_f64_n1_fwd(int E, int ro, int* nt);
const void* fused_ptr_f64_n1_grad(int E, int ro, int* nt);
const void* fused_ptr_f64_n16_fwd(int E, int ro, int* nt);
const void* fused_ptr_f64_n16_grad(int E, int ro, int* nt);

const void* fused_kernel_ptr(int dtype, int E, int nout, bool grad, int readout, int* nt) {
  if (dtype == ACE_F32) {
    if (nout == 1) return grad ? fused_ptr_f32_n1_grad(E, readout, nt) : fused_ptr_f32_n1_fwd(E, readout, nt);
    if (nout == 16) return grad ? fused_ptr_f32_n16_grad(E, readout, nt) : fused_ptr_f32_n16_fwd(E, readout, nt);
  } else if (dtype == ACE_F64) {
    if (nout == 1) return grad ? fused_ptr_f64_n1_grad(E, 0, nt) : fused_ptr_f64_n1_fwd(E, 0, nt);
    if (nout == 16) return grad ? fused_ptr_f64_n16_grad(E, 0, nt) : fused_ptr_f64_n16_fwd(E, 0, nt);
  }
  return nullptr;
}

}  // namespace ace
