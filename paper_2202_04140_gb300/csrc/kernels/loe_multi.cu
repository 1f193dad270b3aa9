// Forward evaluation with several output channels, one environment per lane.
//
// Same recursion as loe.cu (section 2.6, Eq. 4, sinks folded into the one-sided
// sparse contraction phi = sum_s AA_s (c_s + sum_q C_sq AA_q)), for requests with
// up to 16 channels.  The tile-per-lane kernel carries every entry's 16
// coefficients per lane for E environments; here a warp's 32 lanes are 32
// environments, so an entry's coefficient row is one warp-uniform (broadcast) load
// of 64 bytes serving all 32 of them.  The stored values of the CTA's 32
// environments live in its slice of a global workspace (rows of 32 floats, one
// 128-byte line per slot), which for graphs of a few thousand operands stays in L2.
//
// The per-warp streams have the layout of the one-channel kernel (tasks and block
// units, see kLoeBlockCols), bound with basis indices instead of coefficients:
//   task header {x, (pairs << 8) | flags, z, basis index of the row's coefficient or -1},
//   pairs {col0, idx0, col1, idx1}, block rows: header and 8 indices, four per item;
// an index is the basis function of the entry (-1: none), bit 30 doubles it.
// Coefficients are read from the bound table c[n_basis][16] (channels past n_out zero).
#include <cstdint>
#include <cuda_runtime.h>

#include "fused.cuh"
#include "launch.hpp"

namespace ace {
namespace dev {

constexpr int kMultiOut = 16;          // channels carried per lane (requests pad to 16)
constexpr int kIdxMask = 0x3fffffff;   // basis index bits of a bound index
constexpr int kIdxDouble = 0x40000000; // the entry's coefficient counts twice

struct LoeMultiArgs {
  LoeArgs b;              // geometry of the tile, forward levels, workspace, streams' warp ranges
  const int4* istream;    // index-bound per-warp streams (followed by kLoeStreamPad zero items)
  const float* cvals;     // [n_basis][kMultiOut]
  int32_t n_out;
};

// u += x * c[idx] (16 channels), for a bound index (no-op for -1)
__device__ __forceinline__ void add_row(const float* __restrict__ cvals, int idx, float x, float (&u)[kMultiOut]) {
  if (idx < 0) return;  // warp-uniform
  const float s = (idx & kIdxDouble) ? 2.f * x : x;
  const float4* row = reinterpret_cast<const float4*>(cvals + (size_t)(idx & kIdxMask) * kMultiOut);
#pragma unroll
  for (int q = 0; q < kMultiOut / 4; ++q) {
    const float4 v = __ldg(row + q);
    u[4 * q] = __fmaf_rn(v.x, s, u[4 * q]);
    u[4 * q + 1] = __fmaf_rn(v.y, s, u[4 * q + 1]);
    u[4 * q + 2] = __fmaf_rn(v.z, s, u[4 * q + 2]);
    u[4 * q + 3] = __fmaf_rn(v.w, s, u[4 * q + 3]);
  }
}

// phi[ch] += AA_s (c_s[ch] + u[ch]) for a row with header h (u already holds c_s, see the callers)
template <int RO, bool CHECK>
__device__ __forceinline__ void multi_epilogue(const LoeMultiArgs& a, const float* AA, const int4 h,
                                               const float (&u)[kMultiOut], Acc<float, RO> (&phiacc)[kMultiOut],
                                               const int lane) {
  const bool top = (h.y & 2) != 0;
  int x = h.x, z = h.z;
  if (CHECK && ((unsigned)x >= (unsigned)a.b.n_slots || (top && (unsigned)z >= (unsigned)a.b.n_slots))) {
    if (lane == 0) atomicOr(a.b.status, kStatusBounds);
    return;
  }
  const float ap = top ? AA[x * 32 + lane] * AA[z * 32 + lane] : AA[x * 32 + lane];
#pragma unroll
  for (int ch = 0; ch < kMultiOut; ++ch) phiacc[ch].add(ap * u[ch]);
}

// The rows of one of the kLoeStreamWarps per-warp streams.
template <int RO, bool CHECK>
__device__ __forceinline__ void multi_tasks(const LoeMultiArgs& a, const float* AA, Acc<float, RO> (&phiacc)[kMultiOut],
                                            const int stream, const int lane) {
  const int4* p = a.istream + a.b.wbeg[stream];
  const int4* const pend = a.istream + a.b.wbeg[stream + 1];
  auto col_ok = [&](int c) {
    if (CHECK && (unsigned)c >= (unsigned)a.b.n_slots) {
      if (lane == 0) atomicOr(a.b.status, kStatusBounds);
      return 0;
    }
    return c;
  };
  while (p < pend) {
    const int4 h = __ldg(p);
    if (h.y & kLoeBlockFlag) {  // a block: its 8 columns once, then every row from its indices
      const int4 c0 = __ldg(p + 1), c1 = __ldg(p + 2);
      const int col[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
      float q[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) q[j] = AA[col_ok(col[j]) * 32 + lane];
      const int4* r = p + 3;
      for (int i = 0; i < (h.y >> 8); ++i, r += 3) {
        const int4 rh = __ldg(r), i0 = __ldg(r + 1), i1 = __ldg(r + 2);
        const int idx[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
        float u[kMultiOut];
#pragma unroll
        for (int ch = 0; ch < kMultiOut; ++ch) u[ch] = 0.f;
        add_row(a.cvals, rh.w, 1.f, u);  // the row's own coefficient
#pragma unroll
        for (int j = 0; j < 8; ++j) add_row(a.cvals, idx[j], q[j], u);
        multi_epilogue<RO, CHECK>(a, AA, rh, u, phiacc, lane);
      }
      p = r;
      continue;
    }
    const int np = h.y >> 8;
    float u[kMultiOut];
#pragma unroll
    for (int ch = 0; ch < kMultiOut; ++ch) u[ch] = 0.f;
    add_row(a.cvals, h.w, 1.f, u);
    for (int k = 0; k < np; ++k) {
      const int4 e = __ldg(p + 1 + k);
      const float x0 = AA[col_ok(e.x) * 32 + lane], x1 = AA[col_ok(e.z) * 32 + lane];
      add_row(a.cvals, e.y, x0, u);
      add_row(a.cvals, e.w, x1, u);
    }
    multi_epilogue<RO, CHECK>(a, AA, h, u, phiacc, lane);
    p += 1 + np;
  }
}

template <int RO, int NT>
__global__ void __launch_bounds__(NT) loe_multi_kernel(const LoeMultiArgs a) {
  static_assert(kLoeStreamWarps % (NT / 32) == 0, "every warp walks the same number of streams");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NW = NT / 32;
  static_assert(sizeof(Acc<float, RO>) <= sizeof(double), "phi partial slot");
  Acc<float, RO>* red = reinterpret_cast<Acc<float, RO>*>(smem_raw);  // [NW][32][kMultiOut]
  float* AA = a.b.ws + (size_t)blockIdx.x * a.b.n_slots * 32;  // this CTA's slice of the workspace
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int K = a.b.K;
  for (int64_t tile = blockIdx.x; tile < a.b.n_tiles; tile += gridDim.x) {
    const int64_t env0 = tile * 32;
    const int n_here = (a.b.n_env - env0) < 32 ? (int)(a.b.n_env - env0) : 32;
    // 1. leaves: environment e's row of A into lane e of every slot's line
    for (int e = warp; e < 32; e += NW) {
      const float* row = a.b.A + (env0 + e) * K;
      for (int k = lane; k < K; k += 32) AA[k * 32 + e] = e < n_here ? row[k] : 0.f;
    }
    __syncthreads();
    // 2. operand nodes, order ascending (Eq. 4)
    for (int lv = 0; lv < a.b.n_fwd_levels; ++lv) {
      for (int i0 = a.b.fwd_off[lv] + warp * kNodeBatch; i0 < a.b.fwd_off[lv + 1]; i0 += NW * kNodeBatch) {
        int s[kNodeBatch], l[kNodeBatch], r[kNodeBatch];
#pragma unroll
        for (int u = 0; u < kNodeBatch; ++u) {
          const bool in = i0 + u < a.b.fwd_off[lv + 1];
          s[u] = in ? __ldg(a.b.fwd_slot + i0 + u) : -1;
          l[u] = in ? __ldg(a.b.fwd_l + i0 + u) : 0;
          r[u] = in ? __ldg(a.b.fwd_r + i0 + u) : 0;
        }
#pragma unroll
        for (int u = 0; u < kNodeBatch; ++u) {
          if (s[u] < 0) continue;
          if (a.b.check && ((unsigned)s[u] >= (unsigned)a.b.n_slots || (unsigned)l[u] >= (unsigned)a.b.n_slots ||
                            (unsigned)r[u] >= (unsigned)a.b.n_slots)) {
            if (lane == 0) atomicOr(a.b.status, kStatusBounds);
            continue;
          }
          AA[s[u] * 32 + lane] = AA[l[u] * 32 + lane] * AA[r[u] * 32 + lane];
        }
      }
      __syncthreads();
    }
    // 3. the sink rows: the plan lays out kLoeStreamWarps streams, warp w walks w, w + NW, ...
    Acc<float, RO> phiacc[kMultiOut];
    for (int sw = warp; sw < kLoeStreamWarps; sw += NW) {
      if (a.b.check)
        multi_tasks<RO, true>(a, AA, phiacc, sw, lane);
      else
        multi_tasks<RO, false>(a, AA, phiacc, sw, lane);
    }
    // 4. phi: per-lane partials of every warp, combined in warp order by the readout's accumulator
#pragma unroll
    for (int ch = 0; ch < kMultiOut; ++ch) red[(warp * 32 + lane) * kMultiOut + ch] = phiacc[ch];
    __syncthreads();
    for (int i = tid; i < 32 * kMultiOut; i += NT) {
      const int e = i / kMultiOut, ch = i - e * kMultiOut;
      if (e < n_here && ch < a.n_out && a.b.phi) {
        Acc<float, RO> s;
        for (int w = 0; w < NW; ++w) s.add_acc(red[(w * 32 + e) * kMultiOut + ch]);
        a.b.phi[(env0 + e) * a.n_out + ch] = (float)s.value();
      }
    }
    __syncthreads();
  }
}

// One thread per row-major task: as bind_loe_kernel, with basis indices in place of coefficients.
__global__ void bind_loe_idx_kernel(const int4* __restrict__ tasks, const int32_t* __restrict__ toff,
                                    const int32_t* __restrict__ col, const int32_t* __restrict__ ebasis,
                                    const uint8_t* __restrict__ ew2, const int32_t* __restrict__ slot_basis,
                                    const int32_t* __restrict__ hpos, int32_t n, int4* __restrict__ stream) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int4 t = tasks[i];
    const int32_t q0 = toff[i], q1 = toff[i + 1];
    const int32_t b = slot_basis[t.x];
    const int lin = ((t.y & 5) == 5 && b >= 0) ? b : -1;
    const bool top = (t.y & 2) != 0;
    const bool block_row = (t.y & 8) != 0;
    int4* h = stream + hpos[i];
    *h = make_int4(top ? t.z : t.x, block_row ? (t.y & 0xff) : ((((q1 - q0) >> 1) << 8) | (t.y & 0xff)),
                   top ? t.w : 0, lin);
    int* f = reinterpret_cast<int*>(h + 1);
    for (int32_t q = q0; q < q1; ++q) {
      const int32_t eb = ebasis[q];
      const int idx = eb >= 0 ? (eb | (ew2[q] ? kIdxDouble : 0)) : -1;
      if (block_row) {
        f[q - q0] = idx;
      } else {
        f[2 * (q - q0)] = col[q];
        f[2 * (q - q0) + 1] = idx;
      }
    }
  }
}

}  // namespace dev

const void* loe_multi_kernel_ptr(int readout, int* nt) {
  *nt = 512;
  if (readout == 0) return (const void*)&dev::loe_multi_kernel<0, 512>;
  if (readout == 1) return (const void*)&dev::loe_multi_kernel<1, 512>;
  if (readout == 2) return (const void*)&dev::loe_multi_kernel<2, 512>;
  return nullptr;
}

size_t loe_multi_smem(int nt) { return (size_t)(nt / 32) * 32 * dev::kMultiOut * sizeof(double); }

cudaError_t launch_loe_multi(const void* kernel, int grid, int nt, size_t smem, const dev::LoeArgs& base,
                             const int4* istream, const float* cvals, int n_out, cudaStream_t st) {
  dev::LoeMultiArgs a;
  a.b = base;
  a.istream = istream;
  a.cvals = cvals;
  a.n_out = n_out;
  void* args[] = {&a};
  return cudaLaunchKernel(kernel, dim3((unsigned)grid), dim3(nt), args, smem, st);
}

cudaError_t launch_bind_loe_idx(const int4* tasks, const int32_t* toff, const int32_t* col, const int32_t* ebasis,
                                const uint8_t* ew2, const int32_t* slot_basis, const int32_t* hpos, int32_t n_tasks,
                                int4* stream, cudaStream_t st) {
  if (n_tasks == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>(((int64_t)n_tasks + 255) / 256, 4096);
  dev::bind_loe_idx_kernel<<<blocks, 256, 0, st>>>(tasks, toff, col, ebasis, ew2, slot_basis, hpos, n_tasks, stream);
  return cudaGetLastError();
}

}  // namespace ace
