// Fused evaluation of the recursive contraction (section 2.6, Eq. 4) for a
// tile of E environments per CTA, with every stored value of the tile resident
// in shared memory.
//
// Per tile:
//  1. A rows -> AA[k][e] (leaves), transposed so that the E values of one slot
//     are contiguous (one vector load per slot).
//  2. Operand nodes level by level (correlation order ascending):
//     AA_i = AA_l * AA_r  (Eq. 4), for the stored slots; a graph too large for
//     shared memory leaves its least-used top operands out ("cold"), and the
//     entries that need them read their two factors instead.
//  3. Sink contraction: each lane owns one task (a piece of one row s of the
//     sink matrix), streams its (column, coefficient) entries, and forms
//     u = sum_j S_sj AA_j.  Its epilogue adds AA_s (c_s + u/2) (symmetric form)
//     or AA_s (c_s + u) (one-sided form) to the lane's phi accumulator, and in
//     the adjoint pass adds g = phibar . (c_s + u) to G_s, or pushes it to the
//     factors of s (G_l += g AA_r, G_r += g AA_l) when s is a top operand.
//  4. Adjoint through the inner operand nodes, order descending:
//     G_x += G_i AA_p for every inner operand i = [x, p], summed per target x
//     across the warp before one shared-memory update.
//  5. dA[e][k] = G[k][e]; phi[e] = block sum of the lane accumulators.
// No global scratch memory, no inter-CTA communication: tiles are assigned
// statically (tile = blockIdx.x + i * gridDim.x).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ace {
namespace dev {

constexpr int kMaxLevels = 8;
// Warps per CTA of the one-environment-per-lane kernel (its task streams are laid
// out per warp).
constexpr int kLoeStreamWarps = 32;
// Zero items allocated after the last stream (the kernel reads up to this many items ahead).
constexpr int kLoeStreamPad = 16;
// Block units of the streams: header {m, rows << 8 | kLoeBlockFlag, 0, 0}, kLoeBlockCols / 4
// items of columns, then per row a header {x, flags, z, row coefficient} and kLoeBlockCols / 4
// items of coefficients.
constexpr int kLoeBlockCols = 8;
constexpr int kLoeBlockFlag = 16;

enum : int { kReadPlain = 0, kReadComp = 1, kReadF64 = 2 };
enum : uint32_t { kStatusBounds = 1u, kStatusTimeout = 2u };

template <typename T>
struct FusedArgs {
  const T* A;
  const T* phibar;  // may be null (= ones)
  T* phi;           // may be null
  T* dA;            // adjoint output (GRAD)
  int64_t n_env;
  int64_t n_tiles;
  int32_t K, n_slots, n_g, n_out;  // n_slots: slots kept in shared memory (leaves, inner, stored top)
  int32_t gs;  // stride between environments in G (n_g rounded up to 32)
  // genc = 1: the adjoint targets of the tasks carry their adjoint row in the high 16 bits (the
  // slot in the low 16), the pull triples' consumer and target are adjoint rows, and gperm gives
  // the row of each leaf (rows permuted so that updates issued together fall in different banks)
  int32_t genc;
  const int32_t* gperm;
  const int32_t* fwd_slot;
  const int32_t* fwd_l;
  const int32_t* fwd_r;
  const int4* pull;  // adjoint sweep: {inner consumer, partner factor, target, rounds} by target level
  int32_t fwd_off[kMaxLevels + 1];
  int32_t pull_lvl[kMaxLevels + 1];
  int32_t n_fwd_levels, n_pull_levels;
  const int4* tasks;
  const int32_t* slice_off;
  const int32_t* slice_steps;
  int32_t n_slices;
  const uint16_t* col16;    // entry columns (slot indices)
  // FP32 one-channel kernels: the entries packed four steps per lane at a time
  // (group g of a slice at off4[slice] + 32 g + lane: 4 x uint16 columns, float4 coefficients)
  const uint2* col4;
  const int32_t* off4;
  const void* vals4;
  const T* vals;  // [entries][NOUT]
  const T* lin;   // [tasks][NOUT] row coefficient of each task (first task of a basis row), else 0
  // cold tasks (entries read through the two factors of a top operand not in shared memory)
  const int4* cold_tasks;
  const int32_t* cold_slice_off;
  const int32_t* cold_slice_steps;  // steps | (reduction rounds << 16)
  int32_t n_cold_slices;
  const uint32_t* cold_cab;         // factor slots ca | cb << 16
  const T* cold_vals;               // [cold entries][NOUT]
  int32_t check;
  int32_t stage;  // 1: bulk-copy staging of the next tile's A (needs 16-byte aligned A)
  int32_t stage_no_issue;  // test hook: wait for copies that are never issued (exercises the time-out)
  uint32_t* status;
};

// Arguments of the one-environment-per-lane variant (loe.cu).
struct LoeArgs {
  const float* A;
  const float* phibar;
  float* phi;
  float* dA;
  int64_t n_env, n_tiles;
  int32_t K, n_slots, n_g;
  const int32_t* fwd_slot;
  const int32_t* fwd_l;
  const int32_t* fwd_r;
  const int32_t* rev_slot;
  const int32_t* rev_l;
  const int32_t* rev_r;
  int32_t fwd_off[kMaxLevels + 1];
  int32_t rev_off[kMaxLevels + 1];
  int32_t n_fwd_levels, n_rev_levels;
  // One stream per warp of units: a task is a header {target slot, (entry pairs << 8) |
  // flags, second factor slot (top operands), row coefficient bits} followed by
  // its entry pairs {col0, coef0 bits, col1, coef1 bits}; a block of rows with the
  // same kLoeBlockCols columns is laid out as described at kLoeBlockCols.
  const int4* stream;                 // followed by kLoeStreamPad zero items
  int32_t wbeg[kLoeStreamWarps + 1];  // first item of each warp's stream
  float* ws;          // global-workspace variant: [gridDim.x][n_slots (+ n_g)][32] floats
  int32_t check;
  uint32_t* status;
};

// Byte offsets of the shared-memory regions of one CTA (each 16-byte aligned):
// AA [n_slots][E] (slot-major: the E values of one slot are one vector load),
// G [E][gs] (adjoint only, environment-major: the bank of an accumulator is
// its slot mod 32, gs = n_g rounded up to 32), phibar [E][NOUT], phi partials
// [warps][E][NOUT] (8 bytes each: the readout's accumulator, an FP32 (s, c) pair for the
// compensated readout, FP64 for the FP64 one), and, when staging is on, the bulk-copy buffer of
// the next tile's rows of A (E K values + 16 bytes) and its mbarrier.
struct SmemLayout {
  size_t g, pb, red, stage, mbar, total;
};

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

__host__ __device__ inline int g_stride(int n_g) { return (n_g + 31) & ~31; }


__host__ __device__ inline SmemLayout smem_layout(int E, int NOUT, bool grad, int n_slots, int n_g, int NT,
                                                  int tsize, int K, bool stage) {
  SmemLayout L;
  L.g = align16((size_t)n_slots * E * tsize);
  L.pb = L.g + (grad ? align16((size_t)g_stride(n_g) * E * tsize) : 0);
  L.red = L.pb + align16((size_t)E * NOUT * tsize);
  L.stage = align16(L.red + (size_t)(NT / 32) * E * NOUT * sizeof(double));
  L.mbar = L.stage + (stage ? align16((size_t)E * K * tsize + 16) : 0);
  L.total = L.mbar + (stage ? 16 : 0);
  return L;
}

// ---- bulk-copy staging of A (cp.async.bulk, completion on an mbarrier) ---------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* mb) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mb)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Copy the 16-byte aligned window [a0, a1) of the tile's bytes of A into the
// staging buffer (a1 - a0 may be 0: the barrier phase then completes by the
// arrival alone).  Called by one thread.
__device__ __forceinline__ void stage_issue(uint64_t* mb, void* buf, const unsigned char* src, uint32_t bytes) {
  const uint32_t m = smem_u32(mb);
  if (bytes > 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(m), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(buf)), "l"(src), "r"(bytes), "r"(m) : "memory");
  } else {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(m) : "memory");
  }
}

// Wait for the completion of phase `parity`, for at most about a second of
// SM clocks; returns false on time-out.
__device__ __forceinline__ bool stage_wait(uint64_t* mb, uint32_t parity) {
  const uint32_t m = smem_u32(mb);
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(m), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > 2000000000LL) return false;
  }
}

// Byte window of a tile's rows of A: [b0, b1) exactly, of which [b0 & ~15, b1 & ~15) is bulk-copied.
struct StageWindow {
  int64_t b0, b1, a0, a1;
};
__device__ __forceinline__ StageWindow stage_window(int64_t env0, int64_t n_env, int E, int K, int tsize) {
  const int64_t n_here = (n_env - env0) < E ? (n_env - env0) : E;
  StageWindow w;
  w.b0 = env0 * K * tsize;
  w.b1 = w.b0 + n_here * K * tsize;
  w.a0 = w.b0 & ~(int64_t)15;
  w.a1 = w.b1 & ~(int64_t)15;
  if (w.a1 < w.a0) w.a1 = w.a0;
  return w;
}

// Fused multiply-add in the arithmetic type T (no implicit conversions: a call
// with mixed types does not compile).
template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "fma_t: float or double");
  if constexpr (sizeof(T) == 4) return __fmaf_rn(a, b, c);
  else return __fma_rn(a, b, c);
}

// Shared-memory float atomicAdd runs at about a quarter of the throughput of an
// integer shared atomic on this GPU (measured), and explicit compare-and-swap
// loops are slower still: the kernel keeps the number of such updates low
// (segmented warp reduction of equal targets) and spreads concurrent ones over
// distinct banks (environment-major accumulators).

// ---- vector helpers ---------------------------------------------------------------

template <typename T, int E>
__device__ __forceinline__ void load_slot(const T* __restrict__ p, T (&x)[E]) {
  constexpr int bytes = E * (int)sizeof(T);
  if constexpr (bytes % 16 == 0) {
#pragma unroll
    for (int i = 0; i < bytes / 16; ++i) {
      float4 f = reinterpret_cast<const float4*>(p)[i];
      const T* q = reinterpret_cast<const T*>(&f);
#pragma unroll
      for (int j = 0; j < 16 / (int)sizeof(T); ++j) x[i * (16 / (int)sizeof(T)) + j] = q[j];
    }
  } else if constexpr (bytes == 8) {
    float2 f = *reinterpret_cast<const float2*>(p);
    const T* q = reinterpret_cast<const T*>(&f);
#pragma unroll
    for (int j = 0; j < E; ++j) x[j] = q[j];
  } else {
#pragma unroll
    for (int j = 0; j < E; ++j) x[j] = p[j];
  }
}

template <typename T, int E>
__device__ __forceinline__ void store_slot(T* __restrict__ p, const T (&x)[E]) {
  constexpr int bytes = E * (int)sizeof(T);
  if constexpr (bytes % 16 == 0) {
#pragma unroll
    for (int i = 0; i < bytes / 16; ++i) {
      float4 f;
      T* q = reinterpret_cast<T*>(&f);
#pragma unroll
      for (int j = 0; j < 16 / (int)sizeof(T); ++j) q[j] = x[i * (16 / (int)sizeof(T)) + j];
      reinterpret_cast<float4*>(p)[i] = f;
    }
  } else if constexpr (bytes == 8) {
    float2 f;
    T* q = reinterpret_cast<T*>(&f);
#pragma unroll
    for (int j = 0; j < E; ++j) q[j] = x[j];
    *reinterpret_cast<float2*>(p) = f;
  } else {
#pragma unroll
    for (int j = 0; j < E; ++j) p[j] = x[j];
  }
}

template <typename T, int N>
__device__ __forceinline__ void load_vals(const T* __restrict__ p, T (&x)[N]) {
  constexpr int bytes = N * (int)sizeof(T);
  if constexpr (bytes % 16 == 0) {
#pragma unroll
    for (int i = 0; i < bytes / 16; ++i) {
      float4 f = __ldg(reinterpret_cast<const float4*>(p) + i);
      const T* q = reinterpret_cast<const T*>(&f);
#pragma unroll
      for (int j = 0; j < 16 / (int)sizeof(T); ++j) x[i * (16 / (int)sizeof(T)) + j] = q[j];
    }
  } else {
#pragma unroll
    for (int j = 0; j < N; ++j) x[j] = __ldg(p + j);
  }
}

// ---- readout accumulators (FP32 plain, FP32 compensated, FP64) -----------------------

template <typename T, int RO>
struct Acc;

template <>
struct Acc<float, kReadPlain> {
  float s = 0.f;
  __device__ __forceinline__ void add(float x) { s += x; }
  __device__ __forceinline__ void add_acc(const Acc& o) { s += o.s; }
  __device__ __forceinline__ float value() const { return s; }
  __device__ __forceinline__ void shfl_down_add(int d) { s += __shfl_down_sync(0xffffffffu, s, d); }
};

// Kahan's compensated summation: c holds the negated low-order part that the
// running sum s lost, and is subtracted from the next term (four additions per
// term).  The error of the sum of x_1..x_n is at most (2u + O(n u^2)) sum |x_i|,
// u = 2^-24, whatever the order; each x here is a per-task partial, so the bound is
// a small multiple of u times the condition-aware scale sum_k |c_k| |AA_k|.
template <>
struct Acc<float, kReadComp> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ void add_acc(const Acc& o) {
    add(o.s);
    add(-o.c);
  }
  __device__ __forceinline__ float value() const { return s - c; }  // one rounding of s + (-c)
  __device__ __forceinline__ void shfl_down_add(int d) {
    Acc o;
    o.s = __shfl_down_sync(0xffffffffu, s, d);
    o.c = __shfl_down_sync(0xffffffffu, c, d);
    add_acc(o);
  }
};

template <typename T>
struct AccD {
  double s = 0.0;
  __device__ __forceinline__ void add(T x) { s += (double)x; }
  __device__ __forceinline__ void add_acc(const AccD& o) { s += o.s; }
  __device__ __forceinline__ double value() const { return s; }
  __device__ __forceinline__ void shfl_down_add(int d) { s += __shfl_down_sync(0xffffffffu, s, d); }
};
template <>
struct Acc<float, kReadF64> : AccD<float> {};
template <>
struct Acc<double, kReadPlain> : AccD<double> {};


// ---- the kernel ------------------------------------------------------------------------

// Entries of one lane's task, software-pipelined: the (column, coefficient)
// pairs of the next kBatch steps are loaded while the current kBatch are used.
constexpr int kBatch = 4;
// Operand nodes per thread whose indices are loaded together in the level loops.
constexpr int kNodeBatch = 4;
constexpr int kFwdBatch = 8;  // the tile-per-lane kernel's forward levels

template <typename T, int E, int NOUT, bool CHECK>
__device__ __forceinline__ void use_entry(const FusedArgs<T>& a, const T* __restrict__ AA, int j, const T (&v)[NOUT],
                                          T (&acc)[E][NOUT]) {
  if constexpr (CHECK) {
    if ((unsigned)j >= (unsigned)a.n_slots) {
      atomicOr(a.status, kStatusBounds);
      j = 0;
    }
  }
  T x[E];
  load_slot<T, E>(AA + (size_t)j * E, x);
#pragma unroll
  for (int e = 0; e < E; ++e)
#pragma unroll
    for (int c = 0; c < NOUT; ++c) acc[e][c] = fma_t(v[c], x[e], acc[e][c]);
}

template <typename T, int E, int NOUT, int NS, bool CHECK, typename C>
__device__ __forceinline__ void task_entries_impl(const FusedArgs<T>& a, const T* __restrict__ AA,
                                                  const C* __restrict__ colp, const T* __restrict__ valp, int steps,
                                                  T (&acc)[E][NOUT]) {
  // NOUT channels of an entry, at valp + entry * NS (NS: channels stored per entry)
  // colp / valp point at this lane's first entry; entry k is 32 k further on.
  // Whole batches of kBatch entries run without per-entry guards, the loads of
  // batch b + 1 in flight while batch b is used; the last steps % kBatch
  // entries follow one by one.
  const int nb = steps / kBatch;
  if (nb > 0) {
    int cur[kBatch];
    T vc[kBatch][NOUT];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      cur[u] = (int)__ldg(colp + u * 32);
      if constexpr (NOUT == 1) vc[u][0] = __ldg(valp + u * 32);
    }
    for (int b = 0; b < nb; ++b) {
      int nxt[kBatch];
      T vn[kBatch][NOUT];
      if (b + 1 < nb) {
        const C* cp = colp + (size_t)(b + 1) * kBatch * 32;
        const T* vp = valp + (size_t)(b + 1) * kBatch * 32 * NS;
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
          nxt[u] = (int)__ldg(cp + u * 32);
          if constexpr (NOUT == 1) vn[u][0] = __ldg(vp + u * 32);
        }
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        if constexpr (NOUT > 1) load_vals<T, NOUT>(valp + ((size_t)b * kBatch + u) * 32 * NS, vc[u]);
        use_entry<T, E, NOUT, CHECK>(a, AA, cur[u], vc[u], acc);
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        cur[u] = nxt[u];
        if constexpr (NOUT == 1) vc[u][0] = vn[u][0];
      }
    }
  }
  const int done = nb * kBatch;
#pragma unroll
  for (int u = 0; u < kBatch - 1; ++u) {
    if (done + u < steps) {
      const int j = (int)__ldg(colp + (size_t)(done + u) * 32);
      T v[NOUT];
      load_vals<T, NOUT>(valp + (size_t)(done + u) * 32 * NS, v);
      use_entry<T, E, NOUT, CHECK>(a, AA, j, v, acc);
    }
  }
}

template <typename T, int E, int NOUT, int NS, bool CHECK>
__device__ __forceinline__ void task_entries(const FusedArgs<T>& a, const T* __restrict__ AA, int32_t off,
                                             int steps, int lane, int c0, T (&acc)[E][NOUT]) {
  // 16-bit columns: a graph whose stored values per environment exceed 65535
  // could not hold one environment in shared memory anyway.
  const T* valp = a.vals + ((size_t)off + lane) * NS + c0;
  task_entries_impl<T, E, NOUT, NS, CHECK>(a, AA, a.col16 + off + lane, valp, steps, acc);
}

// Four packed entries of one lane: the first n (warp-uniform) are used.
template <int E, bool CHECK, bool FULL>
__device__ __forceinline__ void use_group(const FusedArgs<float>& a, const float* __restrict__ AA, uint2 c, float4 v,
                                          int n, float (&acc)[E][1]) {
  const int j[4] = {(int)(c.x & 0xffffu), (int)(c.x >> 16), (int)(c.y & 0xffffu), (int)(c.y >> 16)};
  const float w[4][1] = {{v.x}, {v.y}, {v.z}, {v.w}};
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (FULL || k < n) use_entry<float, E, 1, CHECK>(a, AA, j[k], w[k], acc);
}

// The entries of one lane's task in packed groups; (c0, v0) is the slice's first
// group, already loaded.  Groups alternate between two register sets, the next
// one loading while the current one is used.
template <int E, bool CHECK>
__device__ __forceinline__ void task_entries_packed(const FusedArgs<float>& a, const float* __restrict__ AA,
                                                    int32_t off4, int steps, int lane, uint2 c0, float4 v0,
                                                    float (&acc)[E][1]) {
  const int ng = (steps + 3) >> 2;
  if (ng == 0) return;
  const uint2* cp = a.col4 + off4 + lane;
  const float4* vp = static_cast<const float4*>(a.vals4) + off4 + lane;
  uint2 ca = c0, cb;
  float4 va = v0, vb;
  int g = 0;
  while (true) {
    if (g + 1 < ng) {
      cb = __ldg(cp + (size_t)(g + 1) * 32);
      vb = __ldg(vp + (size_t)(g + 1) * 32);
      use_group<E, CHECK, true>(a, AA, ca, va, 4, acc);
    } else {
      use_group<E, CHECK, false>(a, AA, ca, va, steps - 4 * g, acc);
      break;
    }
    ++g;
    if (g + 1 < ng) {
      ca = __ldg(cp + (size_t)(g + 1) * 32);
      va = __ldg(vp + (size_t)(g + 1) * 32);
      use_group<E, CHECK, true>(a, AA, cb, vb, 4, acc);
    } else {
      use_group<E, CHECK, false>(a, AA, cb, vb, steps - 4 * g, acc);
      break;
    }
    ++g;
  }
}

// Epilogue of one task (row s, partial row sum u in acc): phi += AA_s (lin +
// half u), and in the adjoint form g = phibar . (lin + u) goes to the row's
// accumulator or, for a top operand, to its factors (segmented warp sums over
// equal "A" targets, one shared-memory update per run).  Called by all lanes.
// phibar of the tile: in registers when it is small, else read from shared memory.
template <typename T, int E, int NOUT, int NS>
struct PhiBar {
  static constexpr bool kRegs = E * NOUT <= 8;  // measured: -2% on the stress step (E = 4, one channel)
  T r[kRegs ? E : 1][kRegs ? NOUT : 1];
  const T* p;
  __device__ __forceinline__ PhiBar(const T* pb, int c0) : p(pb) {
    if constexpr (kRegs) {
#pragma unroll
      for (int e = 0; e < E; ++e)
#pragma unroll
        for (int c = 0; c < NOUT; ++c) r[e][c] = pb[e * NS + c0 + c];
    }
  }
  __device__ __forceinline__ T get(int e, int c, int c0) const {
    if constexpr (kRegs) return r[e][c];
    else return p[e * NS + c0 + c];
  }
};

template <typename T, int E, int NOUT, int NS, bool GRAD, int RO, bool CHECK>
__device__ __forceinline__ void task_epilogue(const FusedArgs<T>& a, const T* __restrict__ AA, T* __restrict__ G,
                                              const PhiBar<T, E, NOUT, NS>& pb, Acc<T, RO> (&phiacc)[E][NOUT],
                                              const int4 task, const T (&acc)[E][NOUT], const T (&lin)[NOUT],
                                              const int rounds, const int lane, const int c0) {
  // channels c0 .. c0 + NOUT of NS; the adjoint seed g sums over them (the blocks of a
  // request add up in the accumulators)
  const int gs = a.gs;
  const bool top = (task.y & 2) != 0;
  bool valid = task.x >= 0;
  // slots (rows of AA) and adjoint rows (rows of G) of the task's targets: the row of a task that
  // is not a top operand, the two factors of one that is (a top operand may not be stored: its
  // value is the product of its factors)
  const bool enc = GRAD && a.genc;
  int row = enc && !top ? (task.x & 0xffff) : task.x, row_g = enc && !top ? (task.x >> 16) : task.x;
  int pl = enc ? (task.z & 0xffff) : task.z, pl_g = enc ? (task.z >> 16) : task.z;
  int pr = enc ? (task.w & 0xffff) : task.w, pr_g = enc ? (task.w >> 16) : task.w;
  if constexpr (CHECK) {
    bool bad = valid && !top && (unsigned)row >= (unsigned)a.n_slots;
    if (valid && top)
      bad |= (unsigned)pl >= (unsigned)a.n_g || (unsigned)pr >= (unsigned)a.n_g ||
             (unsigned)pl_g >= (unsigned)a.n_g || (unsigned)pr_g >= (unsigned)a.n_g;
    if (GRAD && valid && !top) bad |= (unsigned)row >= (unsigned)a.n_g || (unsigned)row_g >= (unsigned)a.n_g;
    if (bad) {
      atomicOr(a.status, kStatusBounds);
      valid = false;
    }
  }
  if (!valid) row = row_g = 0;
  if (!(valid && top)) pl = pl_g = pr = pr_g = 0;
  T xl[E], xr[E], ap[E];
  if (top) {
    load_slot<T, E>(AA + (size_t)pl * E, xl);
    load_slot<T, E>(AA + (size_t)pr * E, xr);
#pragma unroll
    for (int e = 0; e < E; ++e) ap[e] = xl[e] * xr[e];
  } else {
    load_slot<T, E>(AA + (size_t)row * E, ap);
#pragma unroll
    for (int e = 0; e < E; ++e) xl[e] = xr[e] = T(0);
  }
  const T half = GRAD ? T(0.5) : T(1);
  if (valid) {
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int c = 0; c < NOUT; ++c) phiacc[e][c].add(ap[e] * fma_t(half, acc[e][c], lin[c]));
  }
  if constexpr (GRAD) {
    // g = phibar . (c_s + u): the adjoint of this task's stored value
    T g[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      T s = T(0);
#pragma unroll
      for (int c = 0; c < NOUT; ++c) s = fma_t(pb.get(e, c, c0), acc[e][c] + lin[c], s);
      g[e] = valid ? s : T(0);
    }
    // "A" target: the row itself, or the first factor of a top operand.  Lanes
    // are ordered by A target, so equal targets form runs; a segmented suffix
    // sum leaves each run's total in its first lane, which does one atomic.  The
    // plan stores the runs with the task (bit 8 + r: lane + 2^r is in the same
    // run; bit 13: first lane of its run), so no target is shuffled here.
    const int key = valid ? (top ? pl_g : row_g) : 0;
    T va[E];
#pragma unroll
    for (int e = 0; e < E; ++e) va[e] = top ? g[e] * xr[e] : g[e];
    for (int r = 0, d = 1; r < rounds; ++r, d <<= 1) {  // rounds: warp-uniform, from the plan
      const bool same = (task.y >> (8 + r)) & 1;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const T y = __shfl_down_sync(0xffffffffu, va[e], d);
        if (same) va[e] += y;
      }
    }
    const bool head = (task.y >> 13) & 1;
    if (valid && head) {
#pragma unroll
      for (int e = 0; e < E; ++e) atomicAdd(G + (size_t)e * gs + key, va[e]);
    }
    // "B" target: the second factor of a top operand, one atomic per lane
    if (valid && top) {
#pragma unroll
      for (int e = 0; e < E; ++e) atomicAdd(G + (size_t)e * gs + pr_g, g[e] * xl[e]);
    }
  }
}

template <typename T, int E, int NOUT, int NS, bool GRAD, int RO, int NT, bool CHECK>
__device__ __forceinline__ void run_tasks(const FusedArgs<T>& a, const T* __restrict__ AA, T* __restrict__ G,
                                          const PhiBar<T, E, NOUT, NS>& pb, Acc<T, RO> (&phiacc)[E][NOUT],
                                          const int c0) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
  // The header of the warp's next slice (its tasks, length and entry offset) is
  // loaded while the current slice runs.
  // slice_steps holds the entry steps in its low 16 bits and the number of
  // rounds of the segmented adjoint sum in the high bits.
  // FP32 with one channel reads the packed entry groups, whose offsets replace
  // the entry offsets; the first group of the next slice is loaded before the
  // current slice's epilogue.
  constexpr bool PACK = sizeof(T) == 4 && NS == 1;
  const int32_t* offs = PACK ? a.off4 : a.slice_off;
  int4 task_n = make_int4(-1, 0, -1, -1);
  int hdr_n = 0;
  int32_t off_n = 0;
  T lin_n = T(0);  // one channel: the row coefficient is prefetched too
  uint2 c_n = make_uint2(0u, 0u);
  float4 v_n = make_float4(0.f, 0.f, 0.f, 0.f);
  if (warp < a.n_slices) {
    task_n = __ldg(a.tasks + (size_t)warp * 32 + lane);
    hdr_n = __ldg(a.slice_steps + warp);
    off_n = __ldg(offs + warp);
    if constexpr (NS == 1) lin_n = __ldg(a.lin + (size_t)warp * 32 + lane);
    if constexpr (PACK) {
      if ((hdr_n & 0xffff) > 0) {
        c_n = __ldg(a.col4 + off_n + lane);
        v_n = __ldg(static_cast<const float4*>(a.vals4) + off_n + lane);
      }
    }
  }
  for (int sl = warp; sl < a.n_slices; sl += NW) {
    const int4 task = task_n;
    const int steps = hdr_n & 0xffff, rounds = hdr_n >> 16;
    const int32_t off = off_n;
    T lin[NOUT];
    if constexpr (NS == 1) lin[0] = lin_n;
    const uint2 grp_c = c_n;  // the slice's first packed entry group
    const float4 grp_v = v_n;
    const bool has_next = sl + NW < a.n_slices;
    if (has_next) {
      task_n = __ldg(a.tasks + (size_t)(sl + NW) * 32 + lane);
      hdr_n = __ldg(a.slice_steps + sl + NW);
      off_n = __ldg(offs + sl + NW);
      if constexpr (NS == 1) lin_n = __ldg(a.lin + (size_t)(sl + NW) * 32 + lane);
    }
    T acc[E][NOUT];
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int c = 0; c < NOUT; ++c) acc[e][c] = T(0);
    if constexpr (PACK) {
      task_entries_packed<E, CHECK>(a, AA, off, steps, lane, grp_c, grp_v, acc);
      if (has_next && (hdr_n & 0xffff) > 0) {
        c_n = __ldg(a.col4 + off_n + lane);
        v_n = __ldg(static_cast<const float4*>(a.vals4) + off_n + lane);
      }
    } else {
      task_entries<T, E, NOUT, NS, CHECK>(a, AA, off, steps, lane, c0, acc);
    }
    if constexpr (NS > 1) load_vals<T, NOUT>(a.lin + ((size_t)sl * 32 + lane) * NS + c0, lin);
    task_epilogue<T, E, NOUT, NS, GRAD, RO, CHECK>(a, AA, G, pb, phiacc, task, acc, lin, rounds, lane, c0);
  }
}

// The cold tasks: entries whose column is a top operand not kept in shared
// memory read that operand's two factors (ca, cb) and use their product.  Same
// epilogue as the other tasks (no row coefficient).
template <typename T, int E, int NOUT, int NS, bool GRAD, int RO, int NT, bool CHECK>
__device__ __forceinline__ void run_cold_tasks(const FusedArgs<T>& a, const T* __restrict__ AA, T* __restrict__ G,
                                               const PhiBar<T, E, NOUT, NS>& pb, Acc<T, RO> (&phiacc)[E][NOUT],
                                               const int c0) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
  // entry steps whose factor slots and coefficients are loaded together (fewer when the
  // tile's accumulators already fill the registers: measured on 16 channels, E = 4)
  constexpr int CB = E * NOUT >= 64 ? 1 : (E >= 4 ? 2 : 4);
  // Hot slices go round-robin in order of decreasing length, so the last warps
  // carry the least hot work: cold slice i goes to warp NW - 1 - i (a fixed
  // assignment, so phi keeps its summation order).
  for (int sl = NW - 1 - warp; sl < a.n_cold_slices; sl += NW) {
    const int4 task = __ldg(a.cold_tasks + (size_t)sl * 32 + lane);
    const int hdr = __ldg(a.cold_slice_steps + sl);
    const int steps = hdr & 0xffff, rounds = hdr >> 16;
    const int32_t off = __ldg(a.cold_slice_off + sl);
    T acc[E][NOUT];
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
      for (int c = 0; c < NOUT; ++c) acc[e][c] = T(0);
    for (int k0 = 0; k0 < steps; k0 += CB) {
      uint32_t q[CB];
      T v[CB][NOUT];
#pragma unroll
      for (int u = 0; u < CB; ++u) {
        const size_t idx = (size_t)off + (size_t)(k0 + u) * 32 + lane;
        q[u] = k0 + u < steps ? __ldg(a.cold_cab + idx) : 0u;
        if (k0 + u < steps) {
          load_vals<T, NOUT>(a.cold_vals + idx * NS + c0, v[u]);
        } else {
#pragma unroll
          for (int c = 0; c < NOUT; ++c) v[u][c] = T(0);
        }
      }
#pragma unroll
      for (int u = 0; u < CB; ++u) {
        int ca = (int)(q[u] & 0xffffu), cb = (int)(q[u] >> 16);
        if constexpr (CHECK) {
          if ((unsigned)ca >= (unsigned)a.n_slots || (unsigned)cb >= (unsigned)a.n_slots) {
            atomicOr(a.status, kStatusBounds);
            ca = cb = 0;
          }
        }
        T xa[E], xb[E];
        load_slot<T, E>(AA + (size_t)ca * E, xa);
        load_slot<T, E>(AA + (size_t)cb * E, xb);
#pragma unroll
        for (int e = 0; e < E; ++e) {
          const T x = xa[e] * xb[e];
#pragma unroll
          for (int c = 0; c < NOUT; ++c) acc[e][c] = fma_t(v[u][c], x, acc[e][c]);
        }
      }
    }
    T lin[NOUT];
#pragma unroll
    for (int c = 0; c < NOUT; ++c) lin[c] = T(0);
    task_epilogue<T, E, NOUT, NS, GRAD, RO, CHECK>(a, AA, G, pb, phiacc, task, acc, lin, rounds, lane, c0);
  }
}

template <typename T, int E, int NOUT, bool GRAD, int RO, int NT>
__global__ void __launch_bounds__(NT) fused_kernel(const FusedArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NW = NT / 32;
  const SmemLayout L = smem_layout(E, NOUT, GRAD, a.n_slots, a.n_g, NT, (int)sizeof(T), a.K, a.stage != 0);
  T* AA = reinterpret_cast<T*>(smem_raw);
  T* G = reinterpret_cast<T*>(smem_raw + L.g);
  T* pb = reinterpret_cast<T*>(smem_raw + L.pb);
  // per-warp phi partials: the readout's own accumulator (FP32 sums stay FP32 across warps)
  static_assert(sizeof(Acc<T, RO>) <= sizeof(double), "phi partial slot");
  Acc<T, RO>* red = reinterpret_cast<Acc<T, RO>*>(smem_raw + L.red);
  T* sbuf = reinterpret_cast<T*>(smem_raw + L.stage);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_raw + L.mbar);
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int K = a.K;
  const unsigned char* Abytes = reinterpret_cast<const unsigned char*>(a.A);
  // The rows of A of a CTA's next tile are bulk-copied into the staging buffer
  // while the current tile computes.
  bool stage = a.stage != 0;
  uint32_t parity = 0, stale = 0xffffffffu;  // stale: parity of a copy that timed out
  if (stage) {
    if (tid == 0) {
      mbar_init(mbar);
      if (blockIdx.x < a.n_tiles && !a.stage_no_issue) {
        const StageWindow w = stage_window((int64_t)blockIdx.x * E, a.n_env, E, K, (int)sizeof(T));
        stage_issue(mbar, sbuf, Abytes + w.a0, (uint32_t)(w.a1 - w.a0));
      }
    }
    __syncthreads();
  }

  for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
    const int64_t env0 = tile * E;
    // 1. leaves (from the staging buffer, the unaligned last bytes from global memory)
    if (stage) {
      const bool late = !stage_wait(mbar, parity);
      if (__syncthreads_or(late)) {  // block-uniform decision
        if (tid == 0) atomicOr(a.status, kStatusTimeout);
        stage = false;  // this and later tiles read A directly; the copy is waited for at exit
        stale = parity;
      }
      parity ^= 1u;
    }
    if (stage) {
      const StageWindow w = stage_window(env0, a.n_env, E, K, (int)sizeof(T));
      const int shift = (int)((w.b0 - w.a0) / (int64_t)sizeof(T));
      const int in_buf = (int)((w.a1 - w.b0) / (int64_t)sizeof(T));  // tile elements held by the buffer
      for (int i = tid; i < E * K; i += NT) {
        const int e = i / K, k = i - e * K;
        const int64_t env = env0 + e;
        T v = T(0);
        if (env < a.n_env) v = i < in_buf ? sbuf[shift + i] : a.A[env * K + k];
        AA[(size_t)k * E + e] = v;
      }
    } else {
      for (int i = tid; i < E * K; i += NT) {
        const int e = i / K, k = i - e * K;
        const int64_t env = env0 + e;
        AA[(size_t)k * E + e] = env < a.n_env ? a.A[env * K + k] : T(0);
      }
    }
    if constexpr (GRAD) {
      for (int i = tid; i < a.gs * E; i += NT) G[i] = T(0);
      for (int i = tid; i < E * NOUT; i += NT) {
        const int e = i / NOUT, c = i - e * NOUT;
        const int64_t env = env0 + e;
        T v = T(0);
        if (env < a.n_env && c < a.n_out) v = a.phibar ? a.phibar[env * a.n_out + c] : T(1);
        pb[i] = v;
      }
    }
    __syncthreads();
    // the staging buffer is free again: start the copy of the next tile's rows
    if (stage && tid == 0 && tile + gridDim.x < a.n_tiles && !a.stage_no_issue) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const StageWindow w = stage_window((tile + gridDim.x) * E, a.n_env, E, K, (int)sizeof(T));
      stage_issue(mbar, sbuf, Abytes + w.a0, (uint32_t)(w.a1 - w.a0));
    }
    // 2. operand nodes, order ascending (Eq. 4)
    for (int lv = 0; lv < a.n_fwd_levels; ++lv) {
      const int b = a.fwd_off[lv], eidx = a.fwd_off[lv + 1];
      // kFwdBatch nodes per thread at a time, their indices loaded together
      for (int i0 = b + tid; i0 < eidx; i0 += NT * kFwdBatch) {
        int s[kFwdBatch], l[kFwdBatch], r[kFwdBatch];
#pragma unroll
        for (int u = 0; u < kFwdBatch; ++u) {
          const int i = i0 + u * NT;
          const bool in = i < eidx;
          s[u] = in ? __ldg(a.fwd_slot + i) : -1;
          l[u] = in ? __ldg(a.fwd_l + i) : 0;
          r[u] = in ? __ldg(a.fwd_r + i) : 0;
        }
#pragma unroll
        for (int u = 0; u < kFwdBatch; ++u) {
          if (s[u] < 0) continue;
          if (a.check && ((unsigned)s[u] >= (unsigned)a.n_slots || (unsigned)l[u] >= (unsigned)a.n_slots ||
                          (unsigned)r[u] >= (unsigned)a.n_slots)) {
            atomicOr(a.status, kStatusBounds);
            continue;
          }
          T xl[E], xr[E], y[E];
          load_slot<T, E>(AA + (size_t)l[u] * E, xl);
          load_slot<T, E>(AA + (size_t)r[u] * E, xr);
#pragma unroll
          for (int e = 0; e < E; ++e) y[e] = xl[e] * xr[e];
          store_slot<T, E>(AA + (size_t)s[u] * E, y);
        }
      }
      __syncthreads();
    }
    // 3. sink contraction + readout (+ adjoint seeds), in blocks of NB channels: the
    //    accumulators of a block live in registers; each block's per-warp phi partials
    //    go to shared memory.  Plain and FP64-partial readouts take blocks of 8 (fewer
    //    registers, more warps); the compensated readout keeps all channels in one pass
    //    (measured faster: its second pass costs more than the registers it frees).
    constexpr int NB = (NOUT > 8 && RO != kReadComp) ? 8 : NOUT;
    for (int c0 = 0; c0 < NOUT; c0 += NB) {
      Acc<T, RO> phiacc[E][NB];
      const PhiBar<T, E, NB, NOUT> pbv(pb, c0);
      if (a.check) {
        run_tasks<T, E, NB, NOUT, GRAD, RO, NT, true>(a, AA, G, pbv, phiacc, c0);
        run_cold_tasks<T, E, NB, NOUT, GRAD, RO, NT, true>(a, AA, G, pbv, phiacc, c0);
      } else {
        run_tasks<T, E, NB, NOUT, GRAD, RO, NT, false>(a, AA, G, pbv, phiacc, c0);
        run_cold_tasks<T, E, NB, NOUT, GRAD, RO, NT, false>(a, AA, G, pbv, phiacc, c0);
      }
#pragma unroll
      for (int e = 0; e < E; ++e)
#pragma unroll
        for (int c = 0; c < NB; ++c) {
#pragma unroll
          for (int d = 16; d >= 1; d >>= 1) phiacc[e][c].shfl_down_add(d);
          if (lane == 0) red[(warp * E + e) * NOUT + c0 + c] = phiacc[e][c];
        }
    }
    __syncthreads();
    // 4. adjoint through the inner operand nodes, order descending: one lane per
    //    (consumer i, partner p, target x) triple forms G_i AA_p; triples of equal
    //    target are contiguous, so a segmented warp sum leaves one update per run
    if constexpr (GRAD) {
      for (int lv = 0; lv < a.n_pull_levels; ++lv) {
        const int end = a.pull_lvl[lv + 1];
        // the next chunk's triples load while this chunk is summed
        int4 qn = a.pull_lvl[lv] + warp * 32 + lane < end ? __ldg(a.pull + a.pull_lvl[lv] + warp * 32 + lane)
                                                          : make_int4(0, 0, -1, 0);
        for (int j0 = a.pull_lvl[lv] + warp * 32; j0 < end; j0 += NT) {
          int4 q = qn;
          if (j0 + NT < end) qn = j0 + NT + lane < end ? __ldg(a.pull + j0 + NT + lane) : make_int4(0, 0, -1, 0);
          // rounds of the segmented sum: stored by the plan with every triple of the chunk
          const int rounds = __shfl_sync(0xffffffffu, q.w, 0);
          bool valid = q.z >= 0;
          if (a.check && valid &&
              ((unsigned)q.x >= (unsigned)a.n_g || (unsigned)q.y >= (unsigned)a.n_g || (unsigned)q.z >= (unsigned)a.n_g)) {
            atomicOr(a.status, kStatusBounds);
            valid = false;
          }
          if (!valid) q = make_int4(0, 0, -1 - lane, 0);
          T xp[E], v[E];
          load_slot<T, E>(AA + (size_t)q.y * E, xp);
#pragma unroll
          for (int e = 0; e < E; ++e) v[e] = valid ? G[(size_t)e * a.gs + q.x] * xp[e] : T(0);
          const int key = q.z;
          for (int r = 0, d = 1; r < rounds; ++r, d <<= 1) {
            const int k2 = __shfl_down_sync(0xffffffffu, key, d);
            const bool same = (lane + d < 32) && (k2 == key);
#pragma unroll
            for (int e = 0; e < E; ++e) {
              const T y = __shfl_down_sync(0xffffffffu, v[e], d);
              if (same) v[e] += y;
            }
          }
          const int kprev = __shfl_up_sync(0xffffffffu, key, 1);
          if (valid && (lane == 0 || kprev != key)) {
#pragma unroll
            for (int e = 0; e < E; ++e) atomicAdd(G + (size_t)e * a.gs + key, v[e]);
          }
        }
        __syncthreads();
      }
      for (int i = tid; i < E * K; i += NT) {
        const int e = i / K, k = i - e * K;
        const int64_t env = env0 + e;
        if (env < a.n_env) a.dA[env * K + k] = G[(size_t)e * a.gs + (a.gperm ? __ldg(a.gperm + k) : k)];
      }
    }
    // 5. phi: the per-warp partials (already in shared memory) combined in fixed warp order by the
    //    readout's own accumulator (plain FP32, Kahan FP32, or FP64), rounded once to T
    if (a.phi) {
      for (int i = tid; i < E * NOUT; i += NT) {
        const int e = i / NOUT, c = i - e * NOUT;
        Acc<T, RO> s;
        for (int w = 0; w < NW; ++w) s.add_acc(red[(w * E + e) * NOUT + c]);
        const int64_t env = env0 + e;
        if (env < a.n_env && c < a.n_out) a.phi[env * a.n_out + c] = (T)s.value();
      }
    }
    __syncthreads();
  }
  if (stale != 0xffffffffu) stage_wait(mbar, stale);  // a copy that timed out: wait once more (bounded)
}


}  // namespace dev
}  // namespace ace
