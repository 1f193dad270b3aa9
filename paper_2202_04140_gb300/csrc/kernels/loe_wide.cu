// Global-workspace form of the one-environment-per-lane kernel with two environments per lane:
// a CTA holds 64 environments, lane j owns environments 2j and 2j + 1, and every stored value
// or adjoint row of the CTA's workspace slice is 64 floats (256 bytes), so that one gather
// brings a lane the values of both its environments (8 bytes).  Same per-warp task streams,
// arithmetic and order of operations as loe_kernel<GLOBAL = true> (section 2.6, Eq. 4, the
// symmetric sink form and its adjoint); the adjoint updates are 8-byte vector reductions in
// global memory.  Used for graphs whose 32 environments do not fit in shared memory, where the
// one-environment form waits on its gathers: per gather twice the environments.
#include <cstdint>
#include <cuda_runtime.h>

#include "launch.hpp"
#include "loe_device.cuh"

namespace ace {
namespace dev {

constexpr int kWideRow = 64;  // environments per CTA and floats per workspace row
// Entry pairs loaded together per warp: more gathers in flight (measured at D = 20: 2 pairs 33.1 ms,
// 4 34.8, 5 27.2, 6 27.4, 7 33.0, 8 32.0; from 7 on, register spills outweigh them).
constexpr int kWideBatch = 5;
// the next task's first kWideBatch pair items are read past its header: inside the stream padding
static_assert(kWideBatch < kLoeStreamPad, "read-ahead beyond the stream padding");
// Operand nodes of one level taken together per warp in the forward and reverse sweeps, their
// indices loaded before any gather (measured at D = 20: 4 nodes 26.95 ms, 8 nodes 26.42 ms).
constexpr int kWideNodes = 8;

__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }

// p[0] += v.x, p[1] += v.y, one vector reduction (global memory, 8-byte aligned)
__device__ __forceinline__ void red2(float* p, float2 v) {
  asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v.x), "f"(v.y) : "memory");
}

// u += c_j0 AA_j0 and c_j1 AA_j1 for one entry pair {j0, c0, j1, c1}, both environments of the lane.
template <bool CHECK>
__device__ __forceinline__ void wide_pair(const LoeArgs& a, const float* AA, const int4 q, const int lane,
                                          float2& acc0, float2& acc1) {
  int j0 = q.x, j1 = q.z;
  if (CHECK && ((unsigned)j0 >= (unsigned)a.n_slots || (unsigned)j1 >= (unsigned)a.n_slots)) {
    if (lane == 0) atomicOr(a.status, kStatusBounds);
    j0 = j1 = 0;
  }
  const float2 v0 = ld2(AA + (size_t)j0 * kWideRow + 2 * lane);
  const float2 v1 = ld2(AA + (size_t)j1 * kWideRow + 2 * lane);
  const float c0 = __int_as_float(q.y), c1 = __int_as_float(q.w);
  acc0.x = __fmaf_rn(c0, v0.x, acc0.x);
  acc0.y = __fmaf_rn(c0, v0.y, acc0.y);
  acc1.x = __fmaf_rn(c1, v1.x, acc1.x);
  acc1.y = __fmaf_rn(c1, v1.y, acc1.y);
}

// Epilogue of a task or block row with header {x, flags, z, row coefficient} and row sums acc of
// the lane's two environments: phi += AA_s (lin + half acc); adjoint g = phibar (lin + acc) to
// G_s, or G_x += g AA_z, G_z += g AA_x for a top operand s = [x, z].
template <bool GRAD, int RO, bool CHECK>
__device__ __forceinline__ void wide_epilogue(const LoeArgs& a, const float* AA, float* G, const float2 pbl,
                                              Acc<float, RO>& phi0, Acc<float, RO>& phi1, const int4 h,
                                              const float2 acc, const int lane) {
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
  float2 ap, xl = make_float2(0.f, 0.f), xr = make_float2(0.f, 0.f);
  if (top) {
    xl = ld2(AA + (size_t)x * kWideRow + 2 * lane);
    xr = ld2(AA + (size_t)z * kWideRow + 2 * lane);
    ap = make_float2(xl.x * xr.x, xl.y * xr.y);
  } else {
    ap = ld2(AA + (size_t)x * kWideRow + 2 * lane);
  }
  const float lin = __int_as_float(h.w);
  phi0.add(ap.x * __fmaf_rn(half, acc.x, lin));
  phi1.add(ap.y * __fmaf_rn(half, acc.y, lin));
  if constexpr (GRAD) {
    const float2 g = make_float2(pbl.x * (acc.x + lin), pbl.y * (acc.y + lin));
    if (top) {
      red2(G + (size_t)x * kWideRow + 2 * lane, make_float2(g.x * xr.x, g.y * xr.y));
      red2(G + (size_t)z * kWideRow + 2 * lane, make_float2(g.x * xl.x, g.y * xl.y));
    } else {
      red2(G + (size_t)x * kWideRow + 2 * lane, g);
    }
  }
}

// A block unit at p (header h): the block's kLoeBlockCols column values are read once into
// registers; every row is then its header, two items of coefficients and the epilogue.
// Returns the item after the unit.
template <bool GRAD, int RO, bool CHECK>
__device__ __forceinline__ const int4* wide_block(const LoeArgs& a, const float* AA, float* G, const float2 pbl,
                                                  Acc<float, RO>& phi0, Acc<float, RO>& phi1, const int4* p,
                                                  const int4 h, const int4 c0, const int4 c1, const int lane) {
  static_assert(kLoeBlockCols == 8, "two items of columns and of coefficients per row");
  const int nrows = h.y >> 8;
  int col[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
  float2 q[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (CHECK && (unsigned)col[j] >= (unsigned)a.n_slots) {
      if (lane == 0) atomicOr(a.status, kStatusBounds);
      col[j] = 0;
    }
    q[j] = ld2(AA + (size_t)col[j] * kWideRow + 2 * lane);
  }
  const int4* r = p + 3;
  int4 rh = __ldg(r);
  float4 f0 = __ldg(reinterpret_cast<const float4*>(r + 1));
  float4 f1 = __ldg(reinterpret_cast<const float4*>(r + 2));
  for (int i = 0; i < nrows; ++i) {
    const int4 rhn = __ldg(r + 3);
    const float4 f0n = __ldg(reinterpret_cast<const float4*>(r + 4));
    const float4 f1n = __ldg(reinterpret_cast<const float4*>(r + 5));
    const float f[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
    float2 s0 = make_float2(f[0] * q[0].x, f[0] * q[0].y), s1 = make_float2(f[1] * q[1].x, f[1] * q[1].y);
#pragma unroll
    for (int j = 2; j < 8; j += 2) {
      s0.x = __fmaf_rn(f[j], q[j].x, s0.x);
      s0.y = __fmaf_rn(f[j], q[j].y, s0.y);
      s1.x = __fmaf_rn(f[j + 1], q[j + 1].x, s1.x);
      s1.y = __fmaf_rn(f[j + 1], q[j + 1].y, s1.y);
    }
    wide_epilogue<GRAD, RO, CHECK>(a, AA, G, pbl, phi0, phi1, rh, make_float2(s0.x + s1.x, s0.y + s1.y), lane);
    r += 3;
    rh = rhn;
    f0 = f0n;
    f1 = f1n;
  }
  return r;
}

// The sink tasks of one warp's stream (as loe_tasks).
template <bool GRAD, int RO, bool CHECK>
__device__ __forceinline__ void wide_tasks(const LoeArgs& a, const float* AA, float* G, const float2 pbl,
                                           Acc<float, RO>& phi0, Acc<float, RO>& phi1, const int warp,
                                           const int lane) {
  const int4* p = a.stream + a.wbeg[warp];
  const int4* const pend = a.stream + a.wbeg[warp + 1];
  if (p >= pend) return;
  if (lane == 0)  // the warp's whole stream requested into L2 at once (as the one-environment form)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(__cvta_generic_to_global(p)),
                 "r"((unsigned)((pend - p) * (int)sizeof(int4)))
                 : "memory");
  int4 h = __ldg(p);
  int4 cur[kWideBatch];
#pragma unroll
  for (int u = 0; u < kWideBatch; ++u) cur[u] = __ldg(p + 1 + u);
  while (true) {
    if (h.y & kLoeBlockFlag) {
      const int4* const pn = wide_block<GRAD, RO, CHECK>(a, AA, G, pbl, phi0, phi1, p, h, cur[0], cur[1], lane);
      if (pn >= pend) break;
      p = pn;
      h = __ldg(p);
#pragma unroll
      for (int u = 0; u < kWideBatch; ++u) cur[u] = __ldg(p + 1 + u);
      continue;
    }
    const int np = h.y >> 8;
    const int4* const pn = p + 1 + np;  // the next header
    const bool more = pn < pend;
    const int4 hn = __ldg(pn);
    float2 acc0 = make_float2(0.f, 0.f), acc1 = make_float2(0.f, 0.f);
#pragma unroll
    for (int u = 0; u < kWideBatch; ++u)
      if (u < np) wide_pair<CHECK>(a, AA, cur[u], lane, acc0, acc1);
#pragma unroll
    for (int u = 0; u < kWideBatch; ++u) cur[u] = __ldg(pn + 1 + u);
    for (int b = kWideBatch; b < np; b += kWideBatch) {
      int4 bt[kWideBatch];
#pragma unroll
      for (int u = 0; u < kWideBatch; ++u) bt[u] = __ldg(p + 1 + b + u);
#pragma unroll
      for (int u = 0; u < kWideBatch; ++u)
        if (b + u < np) wide_pair<CHECK>(a, AA, bt[u], lane, acc0, acc1);
    }
    wide_epilogue<GRAD, RO, CHECK>(a, AA, G, pbl, phi0, phi1, h, make_float2(acc0.x + acc1.x, acc0.y + acc1.y),
                                   lane);
    if (!more) break;
    p = pn;
    h = hn;
  }
}

template <bool GRAD, int RO, int NT>
__global__ void __launch_bounds__(NT) loe_wide_kernel(const LoeArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NW = NT / 32, S = kWideRow;
  static_assert(NW == kLoeStreamWarps, "one stream per warp");
  float* AA = a.ws + (size_t)blockIdx.x * loe_global_floats(a.n_slots, a.n_g, GRAD) * 2;
  float* G = AA + (size_t)a.n_slots * S;
  float* pb = reinterpret_cast<float*>(smem_raw);  // [64]
  // per-lane phi partials of every warp, both environments: the readout's own accumulator
  static_assert(sizeof(Acc<float, RO>) <= sizeof(double), "phi partial slot");
  Acc<float, RO>* red = reinterpret_cast<Acc<float, RO>*>(pb + S);  // [NW][32][2]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = a.K;
  for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
    const int64_t env0 = tile * S;
    const int n_here = (a.n_env - env0) < S ? (int)(a.n_env - env0) : S;
    // 1. leaves: the tile's rows of A are one contiguous block
    for (int e = warp; e < S; e += NW) {
      const float* row = a.A + (env0 + e) * K;
      for (int k = lane; k < K; k += 32) AA[(size_t)k * S + e] = e < n_here ? row[k] : 0.f;
    }
    if constexpr (GRAD) {
      for (int64_t i = tid; i < (int64_t)a.n_g * S; i += NT) G[i] = 0.f;
      if (tid < S) pb[tid] = tid < n_here ? (a.phibar ? a.phibar[env0 + tid] : 1.f) : 0.f;
    }
    __syncthreads();
    // 2. operand nodes, order ascending (Eq. 4)
    for (int lv = 0; lv < a.n_fwd_levels; ++lv) {
      for (int i0 = a.fwd_off[lv] + warp * kWideNodes; i0 < a.fwd_off[lv + 1]; i0 += NW * kWideNodes) {
        int s[kWideNodes], l[kWideNodes], r[kWideNodes];
#pragma unroll
        for (int u = 0; u < kWideNodes; ++u) {
          const bool in = i0 + u < a.fwd_off[lv + 1];
          s[u] = in ? __ldg(a.fwd_slot + i0 + u) : -1;
          l[u] = in ? __ldg(a.fwd_l + i0 + u) : 0;
          r[u] = in ? __ldg(a.fwd_r + i0 + u) : 0;
        }
#pragma unroll
        for (int u = 0; u < kWideNodes; ++u) {
          if (s[u] < 0) continue;
          if (a.check && ((unsigned)s[u] >= (unsigned)a.n_slots || (unsigned)l[u] >= (unsigned)a.n_slots ||
                          (unsigned)r[u] >= (unsigned)a.n_slots)) {
            if (lane == 0) atomicOr(a.status, kStatusBounds);
            continue;
          }
          const float2 xl = ld2(AA + (size_t)l[u] * S + 2 * lane), xr = ld2(AA + (size_t)r[u] * S + 2 * lane);
          *reinterpret_cast<float2*>(AA + (size_t)s[u] * S + 2 * lane) = make_float2(xl.x * xr.x, xl.y * xr.y);
        }
      }
      __syncthreads();
    }
    // 3. tasks: each warp walks its own stream
    Acc<float, RO> phi0, phi1;
    const float2 pbl = GRAD ? make_float2(pb[2 * lane], pb[2 * lane + 1]) : make_float2(0.f, 0.f);
    if (a.check)
      wide_tasks<GRAD, RO, true>(a, AA, G, pbl, phi0, phi1, warp, lane);
    else
      wide_tasks<GRAD, RO, false>(a, AA, G, pbl, phi0, phi1, warp, lane);
    __syncthreads();
    // 4. adjoint through the inner operand nodes, order descending: G_l += G_i AA_r, G_r += G_i AA_l
    if constexpr (GRAD) {
      for (int lv = 0; lv < a.n_rev_levels; ++lv) {
        for (int i0 = a.rev_off[lv] + warp * kWideNodes; i0 < a.rev_off[lv + 1]; i0 += NW * kWideNodes) {
          int s[kWideNodes], l[kWideNodes], r[kWideNodes];
#pragma unroll
          for (int u = 0; u < kWideNodes; ++u) {
            const bool in = i0 + u < a.rev_off[lv + 1];
            s[u] = in ? __ldg(a.rev_slot + i0 + u) : -1;
            l[u] = in ? __ldg(a.rev_l + i0 + u) : 0;
            r[u] = in ? __ldg(a.rev_r + i0 + u) : 0;
          }
#pragma unroll
          for (int u = 0; u < kWideNodes; ++u) {
            if (s[u] < 0) continue;
            if (a.check && ((unsigned)s[u] >= (unsigned)a.n_g || (unsigned)l[u] >= (unsigned)a.n_g ||
                            (unsigned)r[u] >= (unsigned)a.n_g)) {
              if (lane == 0) atomicOr(a.status, kStatusBounds);
              continue;
            }
            const float2 g = ld2(G + (size_t)s[u] * S + 2 * lane);
            const float2 xl = ld2(AA + (size_t)l[u] * S + 2 * lane), xr = ld2(AA + (size_t)r[u] * S + 2 * lane);
            red2(G + (size_t)l[u] * S + 2 * lane, make_float2(g.x * xr.x, g.y * xr.y));
            red2(G + (size_t)r[u] * S + 2 * lane, make_float2(g.x * xl.x, g.y * xl.y));
          }
        }
        __syncthreads();
      }
      for (int e = warp; e < n_here; e += NW) {
        float* row = a.dA + (env0 + e) * K;
        for (int k = lane; k < K; k += 32) row[k] = G[(size_t)k * S + e];
      }
    }
    // 5. phi: per-lane partials of every warp, combined in warp order by the readout's accumulator
    red[(warp * 32 + lane) * 2] = phi0;
    red[(warp * 32 + lane) * 2 + 1] = phi1;
    __syncthreads();
    if (tid < n_here && a.phi) {
      Acc<float, RO> s;
      for (int w = 0; w < NW; ++w) s.add_acc(red[(w * 32 + (tid >> 1)) * 2 + (tid & 1)]);
      a.phi[env0 + tid] = (float)s.value();
    }
    __syncthreads();
  }
}

}  // namespace dev

const void* loe_wide_kernel_ptr(bool grad, int readout, int* nt) {
  *nt = 1024;
  if (grad) {
    if (readout == 0) return (const void*)&dev::loe_wide_kernel<true, 0, 1024>;
    if (readout == 1) return (const void*)&dev::loe_wide_kernel<true, 1, 1024>;
    if (readout == 2) return (const void*)&dev::loe_wide_kernel<true, 2, 1024>;
  } else {
    if (readout == 0) return (const void*)&dev::loe_wide_kernel<false, 0, 1024>;
    if (readout == 1) return (const void*)&dev::loe_wide_kernel<false, 1, 1024>;
    if (readout == 2) return (const void*)&dev::loe_wide_kernel<false, 2, 1024>;
  }
  return nullptr;
}

size_t loe_wide_smem(int nt) { return dev::kWideRow * 4 + (size_t)(nt / 32) * 32 * 2 * sizeof(double); }

size_t loe_wide_bytes_per_cta(int n_slots, int n_g, bool grad) {
  return dev::loe_global_floats(n_slots, n_g, grad) * 2 * sizeof(float);
}

}  // namespace ace
