// Fused forward + adjoint for small graphs, one environment per lane.
//
// Same arithmetic as fused.cuh (section 2.6, Eq. 4; sinks folded into the
// symmetric sink matrix, adjoint pushed back through the operand nodes), laid
// out the other way round: a CTA holds 32 environments, lane e of every warp
// owns environment e, and a whole warp works on one task at a time.  The
// stored values of the tile are AA[slot][e] with a row stride of 33 floats, so
// that a warp reading slot j touches 32 consecutive banks (no conflicts) and
// the transposed copies of A in and dA out hit distinct banks too.  Every warp
// reads its own contiguous stream of 16-byte items (a task header, then the
// task's entries {column, coefficient} two per item), each item one warp-uniform
// load (a broadcast): metadata costs half a load per entry and 32 environments,
// the gather one conflict-free wavefront.  Used when 32 environments of stored
// values (and adjoints) fit in shared memory; otherwise the same code keeps them
// in a global workspace.
#include <cstdint>
#include <cuda_runtime.h>

#include "launch.hpp"
#include "loe_device.cuh"

namespace ace {
namespace dev {

template <bool GRAD, int RO, int NT, bool GLOBAL>
__global__ void __launch_bounds__(NT) loe_kernel(const LoeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NW = NT / 32;
  constexpr int S = GLOBAL ? 32 : kLoeStride;
  float* AA;
  float* G;
  float* pb;
  if constexpr (GLOBAL) {
    AA = a.ws + (size_t)blockIdx.x * loe_global_floats(a.n_slots, a.n_g, GRAD);
    G = AA + (size_t)a.n_slots * S;
    pb = reinterpret_cast<float*>(smem_raw);
  } else {
    AA = reinterpret_cast<float*>(smem_raw);
    G = reinterpret_cast<float*>(smem_raw + align16((size_t)a.n_slots * S * 4));
    pb = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(G) + (GRAD ? align16((size_t)a.n_g * S * 4) : 0));
  }
  // per-lane phi partials of every warp: the readout's own accumulator (8 bytes reserved per slot)
  static_assert(sizeof(Acc<float, RO>) <= sizeof(double), "phi partial slot");
  Acc<float, RO>* red = reinterpret_cast<Acc<float, RO>*>(pb + 32);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = a.K;
  for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
    const int64_t env0 = tile * 32;
    const int n_here = (a.n_env - env0) < 32 ? (int)(a.n_env - env0) : 32;
    // 1. leaves: the tile's rows of A are one contiguous block
    for (int e = warp; e < 32; e += NW) {
      const float* row = a.A + (env0 + e) * K;
      for (int k = lane; k < K; k += 32) AA[k * S + e] = e < n_here ? row[k] : 0.f;
    }
    if constexpr (GRAD) {
      for (int i = tid; i < a.n_g * S; i += NT) G[i] = 0.f;
      if (tid < 32) pb[tid] = tid < n_here ? (a.phibar ? a.phibar[env0 + tid] : 1.f) : 0.f;
    }
    __syncthreads();
    // 2. operand nodes, order ascending (Eq. 4): one node per warp, one environment per lane
    loe_forward_levels<S, NW>(a, AA, warp, lane);
    // 3. tasks: each warp walks its own stream, one task at a time
    Acc<float, RO> phiacc;
    const float pbl = GRAD ? pb[lane] : 0.f;
    if (a.check)
      loe_tasks<GRAD, RO, S, true>(a, AA, G, pbl, phiacc, warp, lane);
    else
      loe_tasks<GRAD, RO, S, false>(a, AA, G, pbl, phiacc, warp, lane);
    __syncthreads();
    // 4. adjoint through the inner operand nodes, order descending
    if constexpr (GRAD) {
      loe_reverse_levels<S, NW>(a, AA, G, warp, lane);
      for (int e = warp; e < n_here; e += NW) {
        float* row = a.dA + (env0 + e) * K;
        for (int k = lane; k < K; k += 32) row[k] = G[k * S + e];
      }
    }
    // 5. phi: per-lane partials of every warp, combined in warp order by the readout's accumulator
    //    (plain FP32, Kahan FP32, or FP64 for the FP64 readout) and rounded once
    red[warp * 32 + lane] = phiacc;
    __syncthreads();
    if (tid < 32 && tid < n_here && a.phi) {
      Acc<float, RO> s;
      for (int w = 0; w < NW; ++w) s.add_acc(red[w * 32 + tid]);
      a.phi[env0 + tid] = (float)s.value();
    }
    __syncthreads();
  }
}

}  // namespace dev

const void* loe_kernel_ptr(bool grad, int readout, bool global, int* nt) {
  *nt = 1024;
  using namespace dev;
#define ACE_LOE_PICK(G)                                                              \
  if (grad) {                                                                        \
    if (readout == 0) return (const void*)&loe_kernel<true, 0, 1024, G>;            \
    if (readout == 1) return (const void*)&loe_kernel<true, 1, 1024, G>;            \
    if (readout == 2) return (const void*)&loe_kernel<true, 2, 1024, G>;            \
  } else {                                                                           \
    if (readout == 0) return (const void*)&loe_kernel<false, 0, 1024, G>;           \
    if (readout == 1) return (const void*)&loe_kernel<false, 1, 1024, G>;           \
    if (readout == 2) return (const void*)&loe_kernel<false, 2, 1024, G>;           \
  }
  if (global) {
    ACE_LOE_PICK(true)
  } else {
    ACE_LOE_PICK(false)
  }
#undef ACE_LOE_PICK
  return nullptr;
}

size_t loe_smem(int n_slots, int n_g, bool grad, int nt) { return dev::loe_smem_bytes(n_slots, n_g, grad, nt); }

size_t loe_global_smem(int nt) { return 32 * 4 + (size_t)(nt / 32) * 32 * sizeof(double); }

size_t loe_global_bytes_per_cta(int n_slots, int n_g, bool grad) {
  return dev::loe_global_floats(n_slots, n_g, grad) * sizeof(float);
}

// One thread per task: its header {target, (pairs << 8) | flags, second factor,
// row coefficient} and its entry pairs {column, c of the entry's basis function
// (doubled on the diagonal of the symmetric form; 0 for padding)}; for a block
// row (flag bit 3) the header without a pair count and its coefficients alone,
// four per item, in the block's column order.  The target of
// a top operand is its first factor (the kernel forms its value from both
// factors and pushes adjoints to them), otherwise the row itself; the row
// coefficient is c of the row when the task is the row's first and the row is a
// basis function.
__global__ void bind_loe_kernel(const float* __restrict__ c, const int4* __restrict__ tasks,
                                const int32_t* __restrict__ toff, const int32_t* __restrict__ col,
                                const int32_t* __restrict__ ebasis, const uint8_t* __restrict__ ew2,
                                const int32_t* __restrict__ slot_basis, const int32_t* __restrict__ hpos, int32_t n,
                                int4* __restrict__ stream) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int4 t = tasks[i];
    const int32_t q0 = toff[i], q1 = toff[i + 1];
    const int32_t b = slot_basis[t.x];
    const float lin = ((t.y & 5) == 5 && b >= 0) ? c[b] : 0.f;
    const bool top = (t.y & 2) != 0;
    int4* h = stream + hpos[i];
    const bool block_row = (t.y & 8) != 0;  // coefficients only, four per item (block column order)
    *h = make_int4(top ? t.z : t.x, block_row ? (t.y & 0xff) : ((((q1 - q0) >> 1) << 8) | (t.y & 0xff)),
                   top ? t.w : 0, __float_as_int(lin));
    int2* e = reinterpret_cast<int2*>(h + 1);
    float* f = reinterpret_cast<float*>(h + 1);
    for (int32_t q = q0; q < q1; ++q) {
      const int32_t eb = ebasis[q];
      const float v = eb >= 0 ? c[eb] * (ew2[q] ? 2.f : 1.f) : 0.f;
      if (block_row) f[q - q0] = v;
      else e[q - q0] = make_int2(col[q], __float_as_int(v));
    }
  }
}

__global__ void loe_static_kernel(const int32_t* __restrict__ pos, const int4* __restrict__ val, int32_t n,
                                  int4* __restrict__ stream) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) stream[pos[i]] = val[i];
}

cudaError_t launch_loe_static(const int32_t* pos, const int4* val, int32_t n, int4* stream, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>(((int64_t)n + 255) / 256, 4096);
  loe_static_kernel<<<blocks, 256, 0, st>>>(pos, val, n, stream);
  return cudaGetLastError();
}

cudaError_t launch_bind_loe(const float* c, const int4* tasks, const int32_t* toff, const int32_t* col,
                            const int32_t* ebasis, const uint8_t* ew2, const int32_t* slot_basis,
                            const int32_t* hpos, int32_t n_tasks, int4* stream, cudaStream_t st) {
  if (n_tasks == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>(((int64_t)n_tasks + 255) / 256, 4096);
  bind_loe_kernel<<<blocks, 256, 0, st>>>(c, tasks, toff, col, ebasis, ew2, slot_basis, hpos, n_tasks, stream);
  return cudaGetLastError();
}

}  // namespace ace
