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

// u += c_j0 AA_j0 and c_j1 AA_j1 for one entry pair {j0, c0, j1, c1}.
template <int S, bool CHECK>
__device__ __forceinline__ void loe_pair(const LoeArgs& a, const float* AA, const int4 q, const int lane,
                                         float& acc0, float& acc1) {
  int j0 = q.x, j1 = q.z;
  if (CHECK && ((unsigned)j0 >= (unsigned)a.n_slots || (unsigned)j1 >= (unsigned)a.n_slots)) {
    if (lane == 0) atomicOr(a.status, kStatusBounds);
    j0 = j1 = 0;
  }
  acc0 = __fmaf_rn(__int_as_float(q.y), AA[j0 * S + lane], acc0);
  acc1 = __fmaf_rn(__int_as_float(q.w), AA[j1 * S + lane], acc1);
}

// The sink tasks of one warp (step 3 of the kernel).  Its stream holds, per task,
// a header h = {x, (pairs << 8) | flags, z, row coefficient} and the task's entry
// pairs right after it.  x is the row s, or for a top operand (flags bit 1) its
// first factor with z the second: the top operand's value is then formed from
// its factors and its adjoint pushed to them (its own adjoint is not kept).
// Epilogue: phi += AA_s (lin + half u); adjoint g = phibar (lin + u) to G_s, or
// G_x += g AA_z, G_z += g AA_x.  While a task runs, the next header and the
// items after it (the next task's first pairs, when it has that many) are loaded.
// Epilogue of a task or block row with header {x, flags, z, row coefficient} and row sum acc:
// phi += AA_s (lin + half acc); adjoint g = phibar (lin + acc) to G_s, or G_x += g AA_z,
// G_z += g AA_x for a top operand s = [x, z].
template <bool GRAD, int RO, int S, bool CHECK>
__device__ __forceinline__ void loe_epilogue(const LoeArgs& a, const float* AA, float* G, const float pbl,
                                             Acc<float, RO>& phiacc, const int4 h, const float acc, const int lane) {
  const float half = GRAD ? 0.5f : 1.f;
  const bool top = (h.y & 2) != 0;
  const int x = h.x, z = h.z;
  if (CHECK) {
    const unsigned lim = GRAD ? (unsigned)a.n_g : (unsigned)a.n_slots;
    if ((unsigned)x >= lim || (top && (unsigned)z >= lim)) {
      if (lane == 0) atomicOr(a.status, kStatusBounds);
      return;
    }
  }
  float ap, xl = 0.f, xr = 0.f;
  if (top) {
    xl = AA[x * S + lane];
    xr = AA[z * S + lane];
    ap = xl * xr;
  } else {
    ap = AA[x * S + lane];
  }
  const float lin = __int_as_float(h.w);
  phiacc.add(ap * __fmaf_rn(half, acc, lin));
  if constexpr (GRAD) {
    const float g = pbl * (acc + lin);
    if (top) {
      atomicAdd(G + x * S + lane, g * xr);
      atomicAdd(G + z * S + lane, g * xl);
    } else {
      atomicAdd(G + x * S + lane, g);
    }
  }
}

// A block unit at p (header h): the block's kLoeBlockCols column values of this lane's
// environment are read once into registers; every row is then its header, two items of
// coefficients and the epilogue (no gathers of its own).  Returns the item after the unit.
template <bool GRAD, int RO, int S, bool CHECK>
__device__ __forceinline__ const int4* loe_block(const LoeArgs& a, const float* AA, float* G, const float pbl,
                                                 Acc<float, RO>& phiacc, const int4* p, const int4 h,
                                                 const int4 c0, const int4 c1, const int lane) {
  static_assert(kLoeBlockCols == 8, "two items of columns and of coefficients per row");
  const int nrows = h.y >> 8;
  int col[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
  float q[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (CHECK && (unsigned)col[j] >= (unsigned)a.n_slots) {
      if (lane == 0) atomicOr(a.status, kStatusBounds);
      col[j] = 0;
    }
    q[j] = AA[col[j] * S + lane];
  }
  const int4* r = p + 3;
  int4 rh = __ldg(r);
  float4 f0 = __ldg(reinterpret_cast<const float4*>(r + 1));
  float4 f1 = __ldg(reinterpret_cast<const float4*>(r + 2));
  for (int i = 0; i < nrows; ++i) {
    // the next row's items (or the items after the unit: inside the stream and its padding)
    const int4 rhn = __ldg(r + 3);
    const float4 f0n = __ldg(reinterpret_cast<const float4*>(r + 4));
    const float4 f1n = __ldg(reinterpret_cast<const float4*>(r + 5));
    float s0 = f0.x * q[0], s1 = f0.y * q[1];
    s0 = __fmaf_rn(f0.z, q[2], s0);
    s1 = __fmaf_rn(f0.w, q[3], s1);
    s0 = __fmaf_rn(f1.x, q[4], s0);
    s1 = __fmaf_rn(f1.y, q[5], s1);
    s0 = __fmaf_rn(f1.z, q[6], s0);
    s1 = __fmaf_rn(f1.w, q[7], s1);
    loe_epilogue<GRAD, RO, S, CHECK>(a, AA, G, pbl, phiacc, rh, s0 + s1, lane);
    r += 3;
    rh = rhn;
    f0 = f0n;
    f1 = f1n;
  }
  return r;
}

template <bool GRAD, int RO, int S, bool CHECK>
__device__ __forceinline__ void loe_tasks(const LoeArgs& a, float* AA, float* G, const float pbl,
                                          Acc<float, RO>& phiacc, const int warp, const int lane) {
  // The stream is followed by kLoeStreamPad zero items, so every item read ahead
  // here (the next header, up to kPairBatch items after it, the last batch of a
  // task) lies inside the allocation; items past a task are loaded but not used.
  const int4* p = a.stream + a.wbeg[warp];
  const int4* const pend = a.stream + a.wbeg[warp + 1];
  if (p >= pend) return;
  int4 h = __ldg(p);
  int4 cur[kPairBatch];
#pragma unroll
  for (int u = 0; u < kPairBatch; ++u) cur[u] = __ldg(p + 1 + u);
  while (true) {
    if (h.y & kLoeBlockFlag) {
      const int4* const pn = loe_block<GRAD, RO, S, CHECK>(a, AA, G, pbl, phiacc, p, h, cur[0], cur[1], lane);
      if (pn >= pend) break;
      p = pn;
      h = __ldg(p);
#pragma unroll
      for (int u = 0; u < kPairBatch; ++u) cur[u] = __ldg(p + 1 + u);
      continue;
    }
    const int np = h.y >> 8;
    const int4* const pn = p + 1 + np;  // the next header
    const bool more = pn < pend;
    const int4 hn = __ldg(pn);
    float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
    for (int u = 0; u < kPairBatch; ++u)
      if (u < np) loe_pair<S, CHECK>(a, AA, cur[u], lane, acc0, acc1);
    // the next task's first pairs: the items after its header
#pragma unroll
    for (int u = 0; u < kPairBatch; ++u) cur[u] = __ldg(pn + 1 + u);
    // longer tasks: further batches, loaded together
    for (int b = kPairBatch; b < np; b += kPairBatch) {
      int4 bt[kPairBatch];
#pragma unroll
      for (int u = 0; u < kPairBatch; ++u) bt[u] = __ldg(p + 1 + b + u);
#pragma unroll
      for (int u = 0; u < kPairBatch; ++u)
        if (b + u < np) loe_pair<S, CHECK>(a, AA, bt[u], lane, acc0, acc1);
    }
    loe_epilogue<GRAD, RO, S, CHECK>(a, AA, G, pbl, phiacc, h, acc0 + acc1, lane);
    if (!more) break;
    p = pn;
    h = hn;
  }
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
