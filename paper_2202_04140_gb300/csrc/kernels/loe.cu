// Fused forward + adjoint for small graphs, one environment per lane.
//
// Same arithmetic as fused.cuh (section 2.6, Eq. 4; sinks folded into the
// symmetric sink matrix, adjoint pushed back through the operand nodes), laid
// out the other way round: a CTA holds 32 environments, lane e of every warp
// owns environment e, and a whole warp works on one task at a time.  The
// stored values of the tile are AA[slot][e] with a row stride of 33 floats, so
// that a warp reading slot j touches 32 consecutive banks (no conflicts) and
// the transposed copies of A in and dA out hit distinct banks too.  Entries
// {column, coefficient} are read two at a time with one warp-uniform 16-byte
// load (a broadcast), so metadata costs half a shared-memory-pipe wavefront per
// entry and 32 environments; the gather is one conflict-free wavefront.  Used
// when 32 environments of stored values (and adjoints) fit in shared memory.
#include <cstdint>
#include <cuda_runtime.h>

#include "fused.cuh"
#include "launch.hpp"

namespace ace {
namespace dev {

constexpr int kLoeStride = 33;
constexpr int kPairBatch = 4;  // entry pairs loaded together per warp


__host__ __device__ inline size_t loe_smem_bytes(int n_slots, int n_g, bool grad, int nt) {
  size_t b = align16((size_t)n_slots * kLoeStride * 4);
  if (grad) b += align16((size_t)n_g * kLoeStride * 4);
  b += 32 * 4;
  b += (size_t)(nt / 32) * 32 * sizeof(double);
  return b;
}

// GLOBAL = false: the stored values AA and adjoints G of the CTA's 32
// environments live in shared memory, rows of 33 floats (conflict-free
// transposed copies).  GLOBAL = true (graphs too large for shared memory, e.g.
// millions of basis functions): they live in the CTA's slice of a global
// workspace, rows of 32 floats (one 128-byte line per slot, every gather
// coalesced), and the adjoint updates are global atomics.
__host__ __device__ inline size_t loe_global_floats(int n_slots, int n_g, bool grad) {
  return ((size_t)n_slots + (grad ? (size_t)n_g : 0)) * 32;
}

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
  double* red = reinterpret_cast<double*>(pb + 32);
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
    for (int lv = 0; lv < a.n_fwd_levels; ++lv) {
      // kNodeBatch nodes per warp at a time: their indices are loaded together
      for (int i0 = a.fwd_off[lv] + warp * kNodeBatch; i0 < a.fwd_off[lv + 1]; i0 += NW * kNodeBatch) {
        int s[kNodeBatch], l[kNodeBatch], r[kNodeBatch];
#pragma unroll
        for (int u = 0; u < kNodeBatch; ++u) {
          const bool in = i0 + u < a.fwd_off[lv + 1];
          s[u] = in ? __ldg(a.fwd_slot + i0 + u) : -1;
          l[u] = in ? __ldg(a.fwd_l + i0 + u) : 0;
          r[u] = in ? __ldg(a.fwd_r + i0 + u) : 0;
        }
#pragma unroll
        for (int u = 0; u < kNodeBatch; ++u) {
          if (s[u] < 0) continue;
          if (a.check && ((unsigned)s[u] >= (unsigned)a.n_slots || (unsigned)l[u] >= (unsigned)a.n_slots ||
                          (unsigned)r[u] >= (unsigned)a.n_slots)) {
            if (lane == 0) atomicOr(a.status, kStatusBounds);
            continue;
          }
          AA[s[u] * S + lane] = AA[l[u] * S + lane] * AA[r[u] * S + lane];
        }
      }
      __syncthreads();
    }
    // 3. tasks: one task per warp
    Acc<float, RO> phiacc;
    const float half = GRAD ? 0.5f : 1.f;
    const float pbl = GRAD ? pb[lane] : 0.f;
    // Most tasks hold at most 2 kPairBatch entries: the header and the first
    // kPairBatch entry pairs of the warp's next task are loaded while the current
    // task runs (the pairs once its header has arrived, before the epilogue).
    int t = warp;
    int4 task = make_int4(-1, 0, 0, 0);
    int q0 = 0, q1 = 0;
    float lin = 0.f;
    int4 cur[kPairBatch];
#pragma unroll
    for (int u = 0; u < kPairBatch; ++u) cur[u] = make_int4(0, 0, 0, 0);
    if (t < a.n_tasks) {
      task = __ldg(a.tasks + t);
      const int4 h = __ldg(a.thdr + t);
      q0 = h.x;
      q1 = h.y;
      lin = __int_as_float(h.z);
      const int np0 = (q1 - q0) >> 1;
#pragma unroll
      for (int u = 0; u < kPairBatch; ++u)
        if (u < np0) cur[u] = __ldg(a.ent + (q0 >> 1) + u);
    }
    while (t < a.n_tasks) {
      const int tn = t + NW;
      int4 task_n = make_int4(-1, 0, 0, 0);
      int q0n = 0, q1n = 0;
      float lin_n = 0.f;
      if (tn < a.n_tasks) {
        task_n = __ldg(a.tasks + tn);
        const int4 h = __ldg(a.thdr + tn);
        q0n = h.x;
        q1n = h.y;
        lin_n = __int_as_float(h.z);
      }
      const int4* ep = a.ent + (q0 >> 1);
      const int np = (q1 - q0) >> 1;
      float acc0 = 0.f, acc1 = 0.f;
      // the first batch, already loaded
#pragma unroll
      for (int u = 0; u < kPairBatch; ++u) {
        if (u < np) {
          int j0 = cur[u].x, j1 = cur[u].z;
          if (a.check && ((unsigned)j0 >= (unsigned)a.n_slots || (unsigned)j1 >= (unsigned)a.n_slots)) {
            if (lane == 0) atomicOr(a.status, kStatusBounds);
            j0 = j1 = 0;
          }
          acc0 = __fmaf_rn(__int_as_float(cur[u].y), AA[j0 * S + lane], acc0);
          acc1 = __fmaf_rn(__int_as_float(cur[u].w), AA[j1 * S + lane], acc1);
        }
      }
      // longer tasks: further batches, loaded together
      for (int b = kPairBatch; b < np; b += kPairBatch) {
        int4 bt[kPairBatch];
#pragma unroll
        for (int u = 0; u < kPairBatch; ++u) bt[u] = b + u < np ? __ldg(ep + b + u) : make_int4(0, 0, 0, 0);
#pragma unroll
        for (int u = 0; u < kPairBatch; ++u) {
          if (b + u < np) {
            int j0 = bt[u].x, j1 = bt[u].z;
            if (a.check && ((unsigned)j0 >= (unsigned)a.n_slots || (unsigned)j1 >= (unsigned)a.n_slots)) {
              if (lane == 0) atomicOr(a.status, kStatusBounds);
              j0 = j1 = 0;
            }
            acc0 = __fmaf_rn(__int_as_float(bt[u].y), AA[j0 * S + lane], acc0);
            acc1 = __fmaf_rn(__int_as_float(bt[u].w), AA[j1 * S + lane], acc1);
          }
        }
      }
      // the next task's first batch
      {
        const int npn = (q1n - q0n) >> 1;
#pragma unroll
        for (int u = 0; u < kPairBatch; ++u)
          cur[u] = u < npn ? __ldg(a.ent + (q0n >> 1) + u) : make_int4(0, 0, 0, 0);
      }
      const float acc = acc0 + acc1;
      const int row = task.x;
      const bool top = (task.y & 2) != 0;
      bool ok = true;
      if (a.check && (unsigned)row >= (unsigned)a.n_slots) {
        if (lane == 0) atomicOr(a.status, kStatusBounds);
        ok = false;
      }
      if (ok) {
        float ap, xl = 0.f, xr = 0.f;
        if (GRAD && top) {
          xl = AA[task.z * S + lane];
          xr = AA[task.w * S + lane];
          ap = xl * xr;
        } else {
          ap = AA[row * S + lane];
        }
        phiacc.add(ap * __fmaf_rn(half, acc, lin));
        if constexpr (GRAD) {
          const float g = pbl * (acc + lin);
          if (top) {
            atomicAdd(G + task.z * S + lane, g * xr);
            atomicAdd(G + task.w * S + lane, g * xl);
          } else {
            atomicAdd(G + row * S + lane, g);
          }
        }
      }
      t = tn;
      task = task_n;
      q0 = q0n;
      q1 = q1n;
      lin = lin_n;
    }
    __syncthreads();
    // 4. adjoint through the inner operand nodes, order descending
    if constexpr (GRAD) {
      for (int lv = 0; lv < a.n_rev_levels; ++lv) {
        for (int i0 = a.rev_off[lv] + warp * kNodeBatch; i0 < a.rev_off[lv + 1]; i0 += NW * kNodeBatch) {
          int s[kNodeBatch], l[kNodeBatch], r[kNodeBatch];
#pragma unroll
          for (int u = 0; u < kNodeBatch; ++u) {
            const bool in = i0 + u < a.rev_off[lv + 1];
            s[u] = in ? __ldg(a.rev_slot + i0 + u) : -1;
            l[u] = in ? __ldg(a.rev_l + i0 + u) : 0;
            r[u] = in ? __ldg(a.rev_r + i0 + u) : 0;
          }
#pragma unroll
          for (int u = 0; u < kNodeBatch; ++u) {
            if (s[u] < 0) continue;
            if (a.check && ((unsigned)s[u] >= (unsigned)a.n_g || (unsigned)l[u] >= (unsigned)a.n_g ||
                            (unsigned)r[u] >= (unsigned)a.n_g)) {
              if (lane == 0) atomicOr(a.status, kStatusBounds);
              continue;
            }
            const float g = G[s[u] * S + lane];
            atomicAdd(G + l[u] * S + lane, g * AA[r[u] * S + lane]);
            atomicAdd(G + r[u] * S + lane, g * AA[l[u] * S + lane]);
          }
        }
        __syncthreads();
      }
      for (int e = warp; e < n_here; e += NW) {
        float* row = a.dA + (env0 + e) * K;
        for (int k = lane; k < K; k += 32) row[k] = G[k * S + e];
      }
    }
    // 5. phi: per-lane partials of every warp, summed in FP64 in warp order
    red[warp * 32 + lane] = phiacc.value();
    __syncthreads();
    if (tid < 32 && tid < n_here && a.phi) {
      double s = 0.0;
      for (int w = 0; w < NW; ++w) s += red[w * 32 + tid];
      a.phi[env0 + tid] = (float)s;
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

__global__ void bind_rm_kernel(const float* __restrict__ c, const int32_t* __restrict__ col,
                               const int32_t* __restrict__ ebasis, const uint8_t* __restrict__ ew2, int64_t n,
                               int2* __restrict__ ent) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t b = ebasis[i];
    const float v = b >= 0 ? c[b] * (ew2[i] ? 2.f : 1.f) : 0.f;
    ent[i] = make_int2(col[i], __float_as_int(v));
  }
}

// thdr[t] = {first entry, end entry, coefficient bits, 0}: the coefficient is c of
// task t's row when t is the row's first task and the row is a basis function, else 0
__global__ void bind_thdr_kernel(const float* __restrict__ c, const int4* __restrict__ tasks,
                                 const int32_t* __restrict__ toff, const int32_t* __restrict__ slot_basis, int32_t n,
                                 int4* __restrict__ thdr) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int4 t = tasks[i];
    const int32_t b = slot_basis[t.x];
    const float lin = ((t.y & 5) == 5 && b >= 0) ? c[b] : 0.f;
    thdr[i] = make_int4(toff[i], toff[i + 1], __float_as_int(lin), 0);
  }
}

cudaError_t launch_bind_rm(const float* c, const int32_t* col, const int32_t* ebasis, const uint8_t* ew2, int64_t n,
                           int2* ent, const int4* tasks, const int32_t* toff, const int32_t* slot_basis,
                           int32_t n_tasks, int4* thdr, cudaStream_t st) {
  int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  if (blocks < 1) blocks = 1;
  bind_rm_kernel<<<blocks, 256, 0, st>>>(c, col, ebasis, ew2, n, ent);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || n_tasks == 0) return e;
  bind_thdr_kernel<<<(n_tasks + 255) / 256, 256, 0, st>>>(c, tasks, toff, slot_basis, n_tasks, thdr);
  return cudaGetLastError();
}

}  // namespace ace
