// Selects the compiled instantiation of the fused kernel.
#include "launch.hpp"

namespace ace {

const void* fused_ptr_f32_n1_fwd(int E, int ro);
const void* fused_ptr_f32_n1_grad(int E, int ro);
const void* fused_ptr_f32_n16_fwd(int E, int ro);
const void* fused_ptr_f32_n16_grad(int E, int ro);
const void* fused_ptr_f64_n1_fwd(int E, int ro);
const void* fused_ptr_f64_n1_grad(int E, int ro);
const void* fused_ptr_f64_n16_fwd(int E, int ro);
const void* fused_ptr_f64_n16_grad(int E, int ro);

const void* fused_kernel_ptr(int dtype, int E, int nout, bool grad, int readout, int* nt) {
  *nt = nout == 1 ? 512 : 256;
  if (dtype == ACE_F32) {
    if (nout == 1) return grad ? fused_ptr_f32_n1_grad(E, readout) : fused_ptr_f32_n1_fwd(E, readout);
    if (nout == 16) return grad ? fused_ptr_f32_n16_grad(E, readout) : fused_ptr_f32_n16_fwd(E, readout);
  } else if (dtype == ACE_F64) {
    if (nout == 1) return grad ? fused_ptr_f64_n1_grad(E, 0) : fused_ptr_f64_n1_fwd(E, 0);
    if (nout == 16) return grad ? fused_ptr_f64_n16_grad(E, 0) : fused_ptr_f64_n16_fwd(E, 0);
  }
  return nullptr;
}

}  // namespace ace
