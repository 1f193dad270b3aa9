// Device code of the one-environment-per-lane kernels (loe.cu), shared with the fused
// forces kernel (pool.cu): layout helpers, the task and block walkers of the per-warp
// streams, and the forward and reverse level sweeps.  loe.cu describes the layout.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fused.cuh"

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
  if constexpr (S == 32) {
    // global-workspace variant: the warp's whole stream is requested into L2 at once, so that its
    // sequential reads do not wait on the workspace traffic that evicts it
    if (lane == 0)
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(p)),
                   "r"((unsigned)((pend - p) * (int)sizeof(int4)))
                   : "memory");
  }
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

// Operand nodes level by level, order ascending (Eq. 4): kNodeBatch nodes per warp at a time
// (their indices are loaded together), one environment per lane; AA rows of stride S.
template <int S, int NW>
__device__ __forceinline__ void loe_forward_levels(const LoeArgs& a, float* AA, const int warp, const int lane) {
  for (int lv = 0; lv < a.n_fwd_levels; ++lv) {
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
}

// Adjoint through the inner operand nodes, order descending: G_l += G_i AA_r, G_r += G_i AA_l.
template <int S, int NW>
__device__ __forceinline__ void loe_reverse_levels(const LoeArgs& a, const float* AA, float* G, const int warp,
                                                   const int lane) {
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
}

}  // namespace dev
}  // namespace ace
