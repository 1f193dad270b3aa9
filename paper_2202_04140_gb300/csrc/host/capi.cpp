// extern "C" entry points of libace (include/ace.h).
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <tuple>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../kernels/fused.cuh"
#include "../kernels/launch.hpp"
#include "ace_internal.hpp"

namespace ace {

namespace {
thread_local std::string g_last_error;
}
static_assert(dev::kLoeBlockCols == kLoeBlockCols && dev::kLoeBlockFlag == kLoeBlockUnit &&
                  dev::kLoeStreamWarps == kLoeWarps,
              "stream layout of the plan and of the one-environment-per-lane kernel");

ace_status fail(ace_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

void clear_error() { g_last_error.clear(); }

const char* last_error_cstr() { return g_last_error.c_str(); }

}  // namespace ace

using namespace ace;

struct ace_spec {
  std::unique_ptr<Spec> s;
};

namespace {

// NVTX range over an entry point's host work (a no-op unless a profiler attaches to NVTX)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct DevTaskSet {
  int4* tasks = nullptr;
  int32_t* slice_off = nullptr;
  int32_t* slice_steps = nullptr;  // device copy: steps | (adjoint reduction rounds << 16)
  int32_t* tbasis = nullptr;       // per task: basis index of its row's own coefficient, or -1
  int32_t* col = nullptr;
  uint16_t* col16 = nullptr;  // columns as uint16 when every slot index fits
  // The same entries packed four steps at a time for the FP32 one-channel kernels:
  // group g of a slice holds steps 4g..4g+3 of each lane, columns as 4 x uint16 in
  // a uint2 and coefficients as a float4, at off4[slice] + 32 g + lane.
  uint2* col4 = nullptr;
  int32_t* off4 = nullptr;
  int32_t* ebasis4 = nullptr;
  uint8_t* ew2_4 = nullptr;
  int64_t n_pack = 0;  // packed entries (groups x 32 lanes x 4)
  void* vals4 = nullptr;
  size_t vals4_bytes = 0;
  // cold tasks (entries read through the two factors of a top operand not kept on chip)
  int4* cold_tasks = nullptr;
  int32_t* cold_slice_off = nullptr;
  int32_t* cold_slice_steps = nullptr;  // steps | (reduction rounds << 16)
  uint32_t* cold_cab = nullptr;
  int32_t* cold_ebasis = nullptr;
  uint8_t* cold_ew2 = nullptr;
  int32_t n_cold_slices = 0;
  int64_t n_cold_pad = 0;
  void* cold_vals = nullptr;
  size_t cold_vals_bytes = 0;
  int32_t* ebasis = nullptr;
  uint8_t* ew2 = nullptr;
  int32_t n_slices = 0;
  int64_t n_pad = 0;
  // row-major copy of the tasks (one-environment-per-lane kernel)
  int4* rm_tasks = nullptr;
  int32_t* rm_off = nullptr;
  int32_t* rm_col = nullptr;
  int32_t* rm_ebasis = nullptr;
  uint8_t* rm_ew2 = nullptr;
  int32_t n_rm = 0;
  int64_t n_rm_ent = 0;
  int32_t* loe_hpos = nullptr;  // item of each task's header in the per-warp streams
  int32_t* loe_spos = nullptr;  // items written once (block headers and columns) and their values
  int4* loe_sval = nullptr;
  int32_t n_loe_static = 0;
  int32_t loe_wbeg[kLoeWarps + 1] = {};
  int64_t n_loe_items = 0;
  int4* loe_stream = nullptr;   // bound streams: headers and {column, coefficient} pairs (FP32, one channel)
  int4* loe_istream = nullptr;  // the same layout bound with basis indices (FP32, several channels)
  float* cvals16 = nullptr;     // bound coefficients [n_basis][16] (channels past n_out zero)
  bool multi_bound = false;
  bool rm_bound = false;
  // coefficients bound into this task set
  void* vals = nullptr;
  size_t vals_bytes = 0;
  void* lin = nullptr;
  size_t lin_bytes = 0;
  bool bound = false;
  int bound_dtype = -1, bound_nout = -1;
};

}  // namespace

struct ace_dag {
  // autotuned kernel choice per (dtype, padded channel count, adjoint): kind 1 = tile per lane
  // (with tile size E), 2 = one environment per lane
  std::map<std::tuple<int, int, int>, std::pair<int, int>> tuned;
  int32_t K = 0;
  int64_t n_basis = 0;
  Graph g;
  GraphOptions opts;  // how g and plan were built
  Plan plan;
  int device = -1;
  int sm_count = 0, smem_optin = 0;
  int32_t *fwd_slot = nullptr, *fwd_l = nullptr, *fwd_r = nullptr;
  int32_t *fwds_slot = nullptr, *fwds_l = nullptr, *fwds_r = nullptr;  // stored slots only
  int32_t *rev_slot = nullptr, *rev_l = nullptr, *rev_r = nullptr;
  int4* pull = nullptr;  // {consumer slot, partner slot, target slot, 0}
  std::vector<int4> pull_host;
  bool genc = false;                 // the sym tasks and pull triples carry permuted adjoint rows
  int32_t* g_perm_dev = nullptr;     // [n_g] adjoint row of each slot (the dA copy of the leaves)
  int32_t *node_left = nullptr, *node_right = nullptr, *node_basis = nullptr, *slot_basis = nullptr;
  DevTaskSet sym, one;
  void* loe_ws = nullptr;  // global workspace of the one-environment-per-lane kernel for large graphs
  size_t loe_ws_bytes = 0;
  // host-buffer evaluation: copy-in, evaluate and copy-out streams, their events, two staging slots
  cudaStream_t hstream[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t hev_fork = nullptr, hev_in[2] = {nullptr, nullptr}, hev_done[2] = {nullptr, nullptr},
              hev_out[2] = {nullptr, nullptr}, hev_join[3] = {nullptr, nullptr, nullptr};
  void* hslot[2] = {nullptr, nullptr};
  size_t hslot_bytes = 0;
  void* fbuf = nullptr;  // host-buffer forces pipeline: whole-batch positions, offsets, forces, phi; two A/dA chunks
  size_t fbuf_bytes = 0;
  void* fwork = nullptr;  // device-buffer forces pipeline, three-kernel form: A and dA of the batch
  size_t fwork_bytes = 0;
  uint32_t* status = nullptr;
  std::vector<void*> allocations;
  std::vector<std::vector<uint16_t>> staging16;  // host copies kept alive until the upload completes
  std::vector<std::vector<int4>> staging_int4;
  std::vector<std::vector<int32_t>> staging32;
  std::vector<std::vector<uint2>> staging_u2;
  std::vector<std::vector<uint8_t>> staging8;
};

namespace {

ace_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? ACE_ERR_OOM : ACE_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename V>
ace_status upload_vec(ace_dag* d, const std::vector<V>& v, V** out, cudaStream_t st) {
  *out = nullptr;
  size_t bytes = std::max<size_t>(v.size() * sizeof(V), 16);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  d->allocations.push_back(p);
  if (!v.empty()) {
    e = cudaMemcpyAsync(p, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync");
  }
  *out = static_cast<V*>(p);
  return ACE_OK;
}

// Rounds of the segmented warp sum a slice needs: ceil(log2) of its longest run
// of lanes with equal "A" target (the row, or the first factor of a top operand).
int reduction_rounds(const std::vector<Task>& tasks, size_t sl) {
  int run = 1, longest = 1, prev_key = 0;
  for (int j = 0; j < 32; ++j) {
    const Task& t = tasks[sl * 32 + j];
    const int key = t.row < 0 ? -1 - j : ((t.flags & 2) ? t.pl : t.row);
    run = (j > 0 && key == prev_key) ? run + 1 : 1;
    longest = std::max(longest, run);
    prev_key = key;
  }
  int rounds = 0;
  while ((1 << rounds) < longest) ++rounds;
  return rounds;
}

// Per-lane structure of the segmented warp sum over equal "A" targets, as flag bits of the
// device task: bit 8 + r is set when lane + 2^r (r < 5) holds the same target (the sum at
// distance 2^r stays inside the run), bit 13 marks the first lane of a run (it does the update).
int32_t segment_bits(const std::vector<Task>& tasks, size_t sl, int j) {
  auto key = [&](int l) {
    const Task& t = tasks[sl * 32 + l];
    return t.row < 0 ? -1 - l : ((t.flags & 2) ? t.pl : t.row);
  };
  int32_t bits = 0;
  for (int r = 0; r < 5; ++r)
    if (j + (1 << r) < 32 && key(j + (1 << r)) == key(j)) bits |= 1 << (8 + r);
  if (j == 0 || key(j - 1) != key(j)) bits |= 1 << 13;
  return bits;
}

// perm (or NULL): adjoint row of each slot with an adjoint; the adjoint targets of a task (the row
// of a task that is not a top operand, the two factors of one that is) then carry their row in
// the high 16 bits above the slot (both below 2^15).
std::vector<int4> device_tasks(const std::vector<Task>& tasks, const int32_t* perm) {
  std::vector<int4> t4(tasks.size());
  auto enc = [&](int32_t v) { return perm && v >= 0 ? v | (perm[v] << 16) : v; };
  for (size_t i = 0; i < tasks.size(); ++i) {
    const Task& t = tasks[i];
    const bool top = (t.flags & 2) != 0;
    t4[i] = make_int4(top ? t.row : enc(t.row), t.flags | segment_bits(tasks, i / 32, (int)(i % 32)),
                      top ? enc(t.pl) : t.pl, top ? enc(t.pr) : t.pr);
  }
  return t4;
}

ace_status upload_tasks(ace_dag* d, const TaskSet& ts, DevTaskSet& dt, cudaStream_t st, const int32_t* perm) {
  std::vector<int4> t4 = device_tasks(ts.tasks, perm);
  d->staging_int4.push_back(std::move(t4));
  ace_status s;
  if ((s = upload_vec(d, d->staging_int4.back(), &dt.tasks, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, ts.slice_off, &dt.slice_off, st)) != ACE_OK) return s;
  // Per slice, the rounds of the segmented warp sum over equal adjoint targets
  // (ceil(log2) of the longest run of equal targets among its 32 tasks), and per
  // task the basis index of its row's own coefficient (first task of a row only).
  std::vector<int32_t> steps_dev(ts.slice_steps.size()), tb(ts.tasks.size(), -1);
  for (size_t sl = 0; sl < ts.slice_steps.size(); ++sl)
    steps_dev[sl] = ts.slice_steps[sl] | (reduction_rounds(ts.tasks, sl) << 16);
  for (size_t i = 0; i < ts.tasks.size(); ++i) {
    const Task& t = ts.tasks[i];
    if (t.row >= 0 && (t.flags & 5) == 5) tb[i] = d->plan.slot_basis[t.row];
  }
  d->staging32.push_back(std::move(steps_dev));
  if ((s = upload_vec(d, d->staging32.back(), &dt.slice_steps, st)) != ACE_OK) return s;
  d->staging32.push_back(std::move(tb));
  if ((s = upload_vec(d, d->staging32.back(), &dt.tbasis, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, ts.col, &dt.col, st)) != ACE_OK) return s;
  if (d->plan.n_stored <= kTileMaxStored) {
    d->staging16.emplace_back(ts.col.begin(), ts.col.end());
    if ((s = upload_vec(d, d->staging16.back(), &dt.col16, st)) != ACE_OK) return s;
    // packed copy: padding steps of a slice's last group get column 0 and no coefficient
    std::vector<int32_t> off4(ts.slice_steps.size() + 1, 0);
    for (size_t sl = 0; sl < ts.slice_steps.size(); ++sl)
      off4[sl + 1] = off4[sl] + 32 * ((ts.slice_steps[sl] + 3) / 4);
    const size_t n_groups = (size_t)off4.back();
    std::vector<uint2> c4(n_groups, make_uint2(0u, 0u));
    std::vector<int32_t> eb4(n_groups * 4, -1);
    std::vector<uint8_t> w4(n_groups * 4, 0);
    for (size_t sl = 0; sl < ts.slice_steps.size(); ++sl) {
      const int steps = ts.slice_steps[sl];
      for (int st4 = 0; st4 < steps; ++st4)
        for (int j = 0; j < 32; ++j) {
          const size_t src = (size_t)ts.slice_off[sl] + (size_t)st4 * 32 + j;
          const size_t gi = (size_t)off4[sl] + (size_t)(st4 / 4) * 32 + j;
          const uint32_t cv = (uint32_t)ts.col[src] << (16 * (st4 & 1));
          if ((st4 & 2) == 0) c4[gi].x |= cv;
          else c4[gi].y |= cv;
          eb4[gi * 4 + (st4 & 3)] = ts.ebasis[src];
          w4[gi * 4 + (st4 & 3)] = ts.ew2[src];
        }
    }
    d->staging32.push_back(std::move(off4));
    if ((s = upload_vec(d, d->staging32.back(), &dt.off4, st)) != ACE_OK) return s;
    d->staging_u2.push_back(std::move(c4));
    if ((s = upload_vec(d, d->staging_u2.back(), &dt.col4, st)) != ACE_OK) return s;
    d->staging32.push_back(std::move(eb4));
    if ((s = upload_vec(d, d->staging32.back(), &dt.ebasis4, st)) != ACE_OK) return s;
    d->staging8.push_back(std::move(w4));
    if ((s = upload_vec(d, d->staging8.back(), &dt.ew2_4, st)) != ACE_OK) return s;
    dt.n_pack = (int64_t)n_groups * 4;
  }
  if ((s = upload_vec(d, ts.ebasis, &dt.ebasis, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, ts.ew2, &dt.ew2, st)) != ACE_OK) return s;
  // cold tasks: slice headers with reduction rounds, factor pairs packed as ca | cb << 16
  dt.n_cold_slices = ts.n_cold_slices();
  dt.n_cold_pad = (int64_t)ts.cold_ca.size();
  if (dt.n_cold_slices > 0) {
    std::vector<int4> c4 = device_tasks(ts.cold_tasks, perm);
    std::vector<int32_t> hdr(ts.cold_slice_steps.size());
    for (size_t sl = 0; sl < hdr.size(); ++sl)
      hdr[sl] = ts.cold_slice_steps[sl] | (reduction_rounds(ts.cold_tasks, sl) << 16);
    std::vector<int32_t> cab(ts.cold_ca.size());
    for (size_t i = 0; i < cab.size(); ++i)
      cab[i] = (int32_t)((uint32_t)ts.cold_ca[i] | ((uint32_t)ts.cold_cb[i] << 16));
    d->staging_int4.push_back(std::move(c4));
    if ((s = upload_vec(d, d->staging_int4.back(), &dt.cold_tasks, st)) != ACE_OK) return s;
    d->staging32.push_back(std::move(hdr));
    if ((s = upload_vec(d, d->staging32.back(), &dt.cold_slice_steps, st)) != ACE_OK) return s;
    if ((s = upload_vec(d, ts.cold_slice_off, &dt.cold_slice_off, st)) != ACE_OK) return s;
    d->staging32.push_back(std::move(cab));
    int32_t* cab_dev = nullptr;
    if ((s = upload_vec(d, d->staging32.back(), &cab_dev, st)) != ACE_OK) return s;
    dt.cold_cab = reinterpret_cast<uint32_t*>(cab_dev);
    if ((s = upload_vec(d, ts.cold_ebasis, &dt.cold_ebasis, st)) != ACE_OK) return s;
    if ((s = upload_vec(d, ts.cold_ew2, &dt.cold_ew2, st)) != ACE_OK) return s;
  }
  dt.n_slices = ts.n_slices();
  dt.n_pad = (int64_t)ts.col.size();
  std::vector<int4> r4(ts.rm_tasks.size());
  for (size_t i = 0; i < ts.rm_tasks.size(); ++i)
    r4[i] = make_int4(ts.rm_tasks[i].row, ts.rm_tasks[i].flags, ts.rm_tasks[i].pl, ts.rm_tasks[i].pr);
  d->staging_int4.push_back(std::move(r4));
  if ((s = upload_vec(d, d->staging_int4.back(), &dt.rm_tasks, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, ts.rm_off, &dt.rm_off, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, ts.rm_col, &dt.rm_col, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, ts.rm_ebasis, &dt.rm_ebasis, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, ts.rm_ew2, &dt.rm_ew2, st)) != ACE_OK) return s;
  dt.n_rm = (int32_t)ts.rm_tasks.size();
  dt.n_rm_ent = (int64_t)ts.rm_col.size();
  if ((s = upload_vec(d, ts.loe_hpos, &dt.loe_hpos, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, ts.loe_spos, &dt.loe_spos, st)) != ACE_OK) return s;
  {
    std::vector<int4> sv(ts.loe_spos.size());
    for (size_t i = 0; i < sv.size(); ++i)
      sv[i] = make_int4(ts.loe_sval[4 * i], ts.loe_sval[4 * i + 1], ts.loe_sval[4 * i + 2], ts.loe_sval[4 * i + 3]);
    d->staging_int4.push_back(std::move(sv));
    if ((s = upload_vec(d, d->staging_int4.back(), &dt.loe_sval, st)) != ACE_OK) return s;
    dt.n_loe_static = (int32_t)ts.loe_spos.size();
  }
  for (int w = 0; w <= kLoeWarps; ++w) dt.loe_wbeg[w] = ts.loe_wbeg[w];
  dt.n_loe_items = ts.loe_wbeg[kLoeWarps];
  return ACE_OK;
}

// Host-side validation of every index the kernels read (done once, before upload).
ace_status validate_plan(const Plan& p) {
  auto in = [](int32_t v, int32_t hi) { return v >= 0 && v < hi; };
  for (size_t i = 0; i < p.fwd.slot.size(); ++i)
    if (!in(p.fwd.slot[i], p.n_slots) || !in(p.fwd.l[i], p.n_slots) || !in(p.fwd.r[i], p.n_slots))
      return fail(ACE_ERR_BOUNDS, "plan: forward index out of range");
  for (size_t i = 0; i < p.rev.slot.size(); ++i)
    if (!in(p.rev.slot[i], p.n_g) || !in(p.rev.l[i], p.n_g) || !in(p.rev.r[i], p.n_g))
      return fail(ACE_ERR_BOUNDS, "plan: adjoint index out of range");
  if (p.n_stored < p.n_g || p.n_stored > p.n_slots) return fail(ACE_ERR_BOUNDS, "plan: stored slot count");
  for (size_t i = 0; i < p.fwd_stored.slot.size(); ++i)
    if (!in(p.fwd_stored.slot[i], p.n_stored) || !in(p.fwd_stored.l[i], p.n_stored) ||
        !in(p.fwd_stored.r[i], p.n_stored))
      return fail(ACE_ERR_BOUNDS, "plan: stored forward index out of range");
  for (const TaskSet* ts : {&p.sym, &p.one}) {
    for (int32_t c : ts->col)
      if (!in(c, p.n_stored)) return fail(ACE_ERR_BOUNDS, "plan: entry column not stored");
    for (size_t i = 0; i < ts->cold_ca.size(); ++i)
      if (!in(ts->cold_ca[i], p.n_g) || !in(ts->cold_cb[i], p.n_g))
        return fail(ACE_ERR_BOUNDS, "plan: cold entry factor out of range");
    for (const Task& t : ts->cold_tasks) {
      if (t.row < 0) continue;
      if (!in(t.row, p.n_slots) || (t.flags & 5)) return fail(ACE_ERR_BOUNDS, "plan: cold task row or flags");
      if ((t.flags & 2) && (!in(t.pl, p.n_g) || !in(t.pr, p.n_g)))
        return fail(ACE_ERR_BOUNDS, "plan: cold task factor out of range");
      if (!(t.flags & 2) && !in(t.row, p.n_g)) return fail(ACE_ERR_BOUNDS, "plan: cold task row out of range");
    }
    if (ts->cold_slice_off.size() != ts->cold_slice_steps.size() + 1 ||
        ts->cold_slice_off.back() != (int32_t)ts->cold_ca.size())
      return fail(ACE_ERR_BOUNDS, "plan: cold slice offsets inconsistent");
  }
  const PullList& q = p.pull;
  if (q.src.size() != q.par.size() || q.src.size() != q.tgt.size() || q.lvl.empty() ||
      q.lvl.back() != (int32_t)q.src.size())
    return fail(ACE_ERR_BOUNDS, "plan: adjoint gather list inconsistent");
  for (size_t j = 0; j < q.src.size(); ++j)
    if (!in(q.src[j], p.n_g) || !in(q.par[j], p.n_g) || !in(q.tgt[j], p.n_g))
      return fail(ACE_ERR_BOUNDS, "plan: adjoint triple out of range");
  for (const TaskSet* ts : {&p.sym, &p.one}) {
    for (int32_t c : ts->col)
      if (!in(c, p.n_slots)) return fail(ACE_ERR_BOUNDS, "plan: entry column out of range");
    for (const Task& t : ts->tasks) {
      if (t.row < 0) continue;
      if (!in(t.row, p.n_slots)) return fail(ACE_ERR_BOUNDS, "plan: task row out of range");
      if ((t.flags & 2) && (!in(t.pl, p.n_g) || !in(t.pr, p.n_g)))
        return fail(ACE_ERR_BOUNDS, "plan: task factor out of range");
      if (ts == &p.sym && !(t.flags & 2) && !in(t.row, p.n_g))
        return fail(ACE_ERR_BOUNDS, "plan: adjoint row out of range");
      if (!(t.flags & 2) && !in(t.row, p.n_stored)) return fail(ACE_ERR_BOUNDS, "plan: task row not stored");
    }
    for (int32_t c : ts->rm_col)
      if (!in(c, p.n_slots)) return fail(ACE_ERR_BOUNDS, "plan: row-major entry column out of range");
    if (ts->rm_off.size() != ts->rm_tasks.size() + 1 || ts->rm_off.back() != (int32_t)ts->rm_col.size())
      return fail(ACE_ERR_BOUNDS, "plan: row-major offsets inconsistent");
    for (size_t i = 0; i < ts->rm_tasks.size(); ++i) {
      const Task& t = ts->rm_tasks[i];
      if ((ts->rm_off[i] & 1) || ts->rm_off[i + 1] < ts->rm_off[i]) return fail(ACE_ERR_BOUNDS, "plan: odd offset");
      if (!in(t.row, p.n_slots)) return fail(ACE_ERR_BOUNDS, "plan: row-major task row out of range");
      if ((t.flags & 2) && (!in(t.pl, p.n_g) || !in(t.pr, p.n_g)))
        return fail(ACE_ERR_BOUNDS, "plan: row-major task factor out of range");
      if (ts == &p.sym && !(t.flags & 2) && !in(t.row, p.n_g))
        return fail(ACE_ERR_BOUNDS, "plan: row-major adjoint row out of range");
    }
    // per-warp streams, decoded as the kernel walks them: every unit (a task, or a block header,
    // its columns and rows) inside its warp's stream, every rm task exactly once, in order
    if (ts->loe_wbeg.size() != (size_t)kLoeWarps + 1 || ts->loe_hpos.size() != ts->rm_tasks.size() ||
        ts->loe_wbeg[0] != 0 || ts->loe_sval.size() != 4 * ts->loe_spos.size())
      return fail(ACE_ERR_BOUNDS, "plan: per-warp stream sizes");
    size_t t = 0, si = 0;
    for (int w = 0; w < kLoeWarps; ++w) {
      int32_t pos = ts->loe_wbeg[w];
      while (pos < ts->loe_wbeg[w + 1]) {
        if (si < ts->loe_spos.size() && ts->loe_spos[si] == pos) {  // a block
          const int32_t* h = &ts->loe_sval[4 * si];
          const int32_t m = h[0], nrows = h[1] >> 8;
          if ((h[1] & 0xff) != kLoeBlockUnit || m < 1 || m > kLoeBlockCols || nrows < 1)
            return fail(ACE_ERR_BOUNDS, "plan: block header");
          ++si;
          ++pos;
          for (int k = 0; k < kLoeBlockCols / 4; ++k, ++si, ++pos) {
            if (si >= ts->loe_spos.size() || ts->loe_spos[si] != pos)
              return fail(ACE_ERR_BOUNDS, "plan: block columns");
            for (int c = 0; c < 4; ++c)
              if (!in(ts->loe_sval[4 * si + c], p.n_slots)) return fail(ACE_ERR_BOUNDS, "plan: block column");
          }
          for (int32_t r = 0; r < nrows; ++r, ++t) {
            if (t >= ts->rm_tasks.size() || ts->loe_hpos[t] != pos || !(ts->rm_tasks[t].flags & kTaskBlockRow) ||
                ts->rm_off[t + 1] - ts->rm_off[t] != kLoeBlockCols)
              return fail(ACE_ERR_BOUNDS, "plan: block row");
            pos += 1 + kLoeBlockCols / 4;
          }
        } else {                                                    // a task
          if (t >= ts->rm_tasks.size() || ts->loe_hpos[t] != pos || (ts->rm_tasks[t].flags & kTaskBlockRow))
            return fail(ACE_ERR_BOUNDS, "plan: per-warp stream header position");
          pos += 1 + (ts->rm_off[t + 1] - ts->rm_off[t]) / 2;
          ++t;
        }
      }
      if (pos != ts->loe_wbeg[w + 1]) return fail(ACE_ERR_BOUNDS, "plan: per-warp stream extent");
    }
    if (t != ts->rm_tasks.size() || si != ts->loe_spos.size())
      return fail(ACE_ERR_BOUNDS, "plan: per-warp streams do not cover the tasks");
  }
  return ACE_OK;
}

ace_status ensure_uploaded(ace_dag* d, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(ACE_ERR_NO_DEVICE, std::string("no CUDA device: ") + cudaGetErrorString(e));
  if (d->device >= 0) {
    if (d->device != dev) return fail(ACE_ERR_UNSUPPORTED, "graph was uploaded to another device");
    return ACE_OK;
  }
  cudaDeviceGetAttribute(&d->sm_count, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&d->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  ace_status s = validate_plan(d->plan);
  if (s != ACE_OK) return s;
  const Plan& p = d->plan;
  if ((s = upload_vec(d, p.fwd.slot, &d->fwd_slot, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, p.fwd.l, &d->fwd_l, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, p.fwd.r, &d->fwd_r, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, p.fwd_stored.slot, &d->fwds_slot, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, p.fwd_stored.l, &d->fwds_l, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, p.fwd_stored.r, &d->fwds_r, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, p.rev.slot, &d->rev_slot, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, p.rev.l, &d->rev_l, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, p.rev.r, &d->rev_r, st)) != ACE_OK) return s;
  // the tile-per-lane kernel's adjoint rows: permuted (Plan::g_perm) when every row fits 15 bits
  d->genc = p.n_g <= 32767 && p.g_perm.size() == (size_t)p.n_g;
  if (d->genc && (s = upload_vec(d, p.g_perm, &d->g_perm_dev, st)) != ACE_OK) return s;
  // {consumer, partner, target, rounds}: rounds of the segmented warp sum of the 32-triple chunk
  // (counted from the level's first triple, as the kernel walks them) holding the triple; the
  // consumer and the target as adjoint rows
  d->pull_host.resize(p.pull.src.size());
  for (size_t lv = 0; lv + 1 < p.pull.lvl.size(); ++lv)
    for (int32_t c0 = p.pull.lvl[lv]; c0 < p.pull.lvl[lv + 1]; c0 += 32) {
      const int32_t c1 = std::min<int32_t>(c0 + 32, p.pull.lvl[lv + 1]);
      int run = 1, longest = 1;
      for (int32_t j = c0 + 1; j < c1; ++j) {
        run = p.pull.tgt[j] == p.pull.tgt[j - 1] ? run + 1 : 1;
        longest = std::max(longest, run);
      }
      int rounds = 0;
      while ((1 << rounds) < longest) ++rounds;
      for (int32_t j = c0; j < c1; ++j)
        d->pull_host[j] = d->genc ? make_int4(p.g_perm[p.pull.src[j]], p.pull.par[j], p.g_perm[p.pull.tgt[j]], rounds)
                                  : make_int4(p.pull.src[j], p.pull.par[j], p.pull.tgt[j], rounds);
    }
  if ((s = upload_vec(d, d->pull_host, &d->pull, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, d->g.left, &d->node_left, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, d->g.right, &d->node_right, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, d->g.node_basis, &d->node_basis, st)) != ACE_OK) return s;
  if ((s = upload_vec(d, p.slot_basis, &d->slot_basis, st)) != ACE_OK) return s;
  if ((s = upload_tasks(d, p.sym, d->sym, st, d->genc ? p.g_perm.data() : nullptr)) != ACE_OK) return s;
  if ((s = upload_tasks(d, p.one, d->one, st, nullptr)) != ACE_OK) return s;
  void* stw = nullptr;
  if ((e = cudaMalloc(&stw, 16)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  d->allocations.push_back(stw);
  d->status = static_cast<uint32_t*>(stw);
  if ((e = cudaMemsetAsync(stw, 0, 16, st)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  // the host vectors above must outlive the copies
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  d->device = dev;
  return ACE_OK;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

int nout_pad_of(int n_out) { return n_out == 1 ? 1 : 16; }

ace_status bind(ace_dag* d, DevTaskSet& dt, const void* c, int n_out, int dtype, cudaStream_t st) {
  const int npad = nout_pad_of(n_out);
  const size_t tsz = dtype == ACE_F32 ? 4 : 8;
  if (c == nullptr) {
    if (!dt.bound || dt.bound_dtype != dtype || dt.bound_nout != n_out)
      return fail(ACE_ERR_INVALID_ARG, "c is NULL and no coefficients of this n_out/dtype are bound");
    return ACE_OK;
  }
  const size_t vb = std::max<size_t>((size_t)dt.n_pad * npad * tsz, 16);
  const size_t lb = std::max<size_t>((size_t)dt.n_slices * 32 * npad * tsz, 16);
  cudaError_t e;
  if (vb > dt.vals_bytes) {
    if (dt.vals) d->allocations.push_back(dt.vals);  // kept: a captured graph may read it
    dt.vals = nullptr;
    dt.vals_bytes = 0;
    if ((e = cudaMalloc(&dt.vals, vb)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    dt.vals_bytes = vb;
  }
  if (lb > dt.lin_bytes) {
    if (dt.lin) d->allocations.push_back(dt.lin);  // kept: a captured graph may read it
    dt.lin = nullptr;
    dt.lin_bytes = 0;
    if ((e = cudaMalloc(&dt.lin, lb)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    dt.lin_bytes = lb;
  }
  e = launch_bind(dtype, c, n_out, npad, dt.ebasis, dt.ew2, dt.n_pad, dt.vals, dt.tbasis, (int64_t)dt.n_slices * 32,
                  dt.lin, st);
  if (e != cudaSuccess) return cuda_fail(e, "coefficient binding launch");
  if (dtype == ACE_F32 && n_out == 1 && dt.col4) {
    const size_t b4 = std::max<size_t>((size_t)dt.n_pack * 4, 16);
    if (b4 > dt.vals4_bytes) {
      if (dt.vals4) d->allocations.push_back(dt.vals4);  // kept: a captured graph may read it
      dt.vals4 = nullptr;
      dt.vals4_bytes = 0;
      if ((e = cudaMalloc(&dt.vals4, b4)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
      dt.vals4_bytes = b4;
    }
    e = launch_bind(dtype, c, n_out, 1, dt.ebasis4, dt.ew2_4, dt.n_pack, dt.vals4, nullptr, 0, nullptr, st);
    if (e != cudaSuccess) return cuda_fail(e, "coefficient binding launch");
  }
  if (dt.n_cold_slices > 0) {
    const size_t cb = std::max<size_t>((size_t)dt.n_cold_pad * npad * tsz, 16);
    if (cb > dt.cold_vals_bytes) {
      if (dt.cold_vals) d->allocations.push_back(dt.cold_vals);  // kept: a captured graph may read it
      dt.cold_vals = nullptr;
      dt.cold_vals_bytes = 0;
      if ((e = cudaMalloc(&dt.cold_vals, cb)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
      dt.cold_vals_bytes = cb;
    }
    e = launch_bind(dtype, c, n_out, npad, dt.cold_ebasis, dt.cold_ew2, dt.n_cold_pad, dt.cold_vals, nullptr, 0,
                    nullptr, st);
    if (e != cudaSuccess) return cuda_fail(e, "coefficient binding launch");
  }
  dt.rm_bound = false;
  dt.multi_bound = false;
  if (dtype == ACE_F32 && n_out > 1) {
    // several channels, one environment per lane: streams of basis indices and the coefficient table
    const size_t sbytes = ((size_t)dt.n_loe_items + dev::kLoeStreamPad) * sizeof(int4);
    if (!dt.loe_istream) {
      void* p = nullptr;
      if ((e = cudaMalloc(&p, sbytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
      dt.loe_istream = static_cast<int4*>(p);
      if ((e = cudaMemsetAsync(p, 0, sbytes, st)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
      if ((e = launch_loe_static(dt.loe_spos, dt.loe_sval, dt.n_loe_static, dt.loe_istream, st)) != cudaSuccess)
        return cuda_fail(e, "stream layout launch");
      if ((e = launch_bind_loe_idx(dt.rm_tasks, dt.rm_off, dt.rm_col, dt.rm_ebasis, dt.rm_ew2, d->slot_basis,
                                   dt.loe_hpos, dt.n_rm, dt.loe_istream, st)) != cudaSuccess)
        return cuda_fail(e, "index binding launch");
    }
    if (!dt.cvals16) {
      void* p = nullptr;
      if ((e = cudaMalloc(&p, std::max<size_t>((size_t)d->n_basis * 16 * sizeof(float), 16))) != cudaSuccess)
        return cuda_fail(e, "cudaMalloc");
      dt.cvals16 = static_cast<float*>(p);
    }
    if ((e = cudaMemsetAsync(dt.cvals16, 0, (size_t)d->n_basis * 16 * sizeof(float), st)) != cudaSuccess ||
        (d->n_basis > 0 &&
         (e = cudaMemcpy2DAsync(dt.cvals16, 16 * sizeof(float), c, (size_t)n_out * sizeof(float),
                                (size_t)n_out * sizeof(float), (size_t)d->n_basis, cudaMemcpyDeviceToDevice, st)) !=
             cudaSuccess))
      return cuda_fail(e, "coefficient table copy");
    dt.multi_bound = true;
  }
  if (dtype == ACE_F32 && n_out == 1) {
    if (!dt.loe_stream) {
      void* p = nullptr;
      const size_t bytes = ((size_t)dt.n_loe_items + dev::kLoeStreamPad) * sizeof(int4);
      if ((e = cudaMalloc(&p, bytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc");
      dt.loe_stream = static_cast<int4*>(p);
      if ((e = cudaMemsetAsync(p, 0, bytes, st)) != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
      // block headers and columns: part of the plan, written once
      if ((e = launch_loe_static(dt.loe_spos, dt.loe_sval, dt.n_loe_static, dt.loe_stream, st)) != cudaSuccess)
        return cuda_fail(e, "stream layout launch");
    }
    e = launch_bind_loe(static_cast<const float*>(c), dt.rm_tasks, dt.rm_off, dt.rm_col, dt.rm_ebasis, dt.rm_ew2,
                        d->slot_basis, dt.loe_hpos, dt.n_rm, dt.loe_stream, st);
    if (e != cudaSuccess) return cuda_fail(e, "coefficient binding launch");
    dt.rm_bound = true;
  }
  dt.bound = true;
  dt.bound_dtype = dtype;
  dt.bound_nout = n_out;
  return ACE_OK;
}

bool checked_mode() {
  const char* v = std::getenv("ACE_CHECKED");
  return v && v[0] && v[0] != '0';
}

// Environments per CTA: the largest compiled E whose shared-memory tile fits,
// with E * NOUT <= 64 accumulators per lane, and not so large that fewer tiles
// than SMs remain.
// The shared-memory layout depends on the thread count of the exact kernel that
// will run (its phi partials take one row per warp), so the lookup uses the
// request's readout mode.
ace_status choose_tile(const ace_dag* d, int dtype, int npad, bool grad, int ro, int64_t n_env, int E_force, int* E_out,
                       int* nt_out, size_t* smem_out, const void** kern_out, bool* stage_out) {
  const int cands_f32_1[] = {16, 8, 4, 2, 1};
  const int cands_f32_16[] = {4, 2, 1};
  const int cands_f64_1[] = {8, 4, 2, 1};
  const int cands_f64_16[] = {2, 1};
  const int* cands;
  int nc;
  if (dtype == ACE_F32) {
    cands = npad == 1 ? cands_f32_1 : cands_f32_16;
    nc = npad == 1 ? 5 : 3;
  } else {
    cands = npad == 1 ? cands_f64_1 : cands_f64_16;
    nc = npad == 1 ? 4 : 2;
  }
  const size_t tsz = dtype == ACE_F32 ? 4 : 8;
  const int64_t per_sm = std::max<int64_t>(1, n_env / std::max(1, d->sm_count));
  for (int i = 0; i < nc; ++i) {
    const int E = cands[i];
    if (E_force > 0 && E != E_force) continue;
    if (E_force <= 0 && E > 1 && E > per_sm) continue;
    int nt = 0;
    const void* k = fused_kernel_ptr(dtype, E, npad, grad, ro, &nt);
    if (!k) continue;
    // with the bulk-copy staging buffer when it fits, else without
    bool stage = true;
    dev::SmemLayout L = dev::smem_layout(E, npad, grad, d->plan.n_stored, d->plan.n_g, nt, (int)tsz, d->K, true);
    if (L.total > (size_t)d->smem_optin) {
      stage = false;
      L = dev::smem_layout(E, npad, grad, d->plan.n_stored, d->plan.n_g, nt, (int)tsz, d->K, false);
    }
    if (L.total > (size_t)d->smem_optin) continue;
    *stage_out = stage;
    *E_out = E;
    *nt_out = nt;
    *smem_out = L.total;
    *kern_out = k;
    return ACE_OK;
  }
  return fail(ACE_ERR_UNSUPPORTED,
              "the stored values of one environment do not fit in shared memory (graph too large for the tiled "
              "kernel)");
}

// Which fused kernel: ACE_KERNEL=lon|loe forces one (tests), otherwise the
// one-environment-per-lane kernel whenever 32 environments fit in shared memory.
int kernel_choice() {
  const char* v = std::getenv("ACE_KERNEL");
  if (v && std::strcmp(v, "lon") == 0) return 1;
  if (v && std::strcmp(v, "loe") == 0) return 2;
  if (v && std::strcmp(v, "loeg") == 0) return 3;
  if (v && std::strcmp(v, "loem") == 0) return 4;
  if (v && std::strcmp(v, "loeg2") == 0) return 5;
  return 0;
}

ace_status grow_loe_workspace(ace_dag* d, size_t need) {
  if (need <= d->loe_ws_bytes) return ACE_OK;
  if (d->loe_ws) cudaFree(d->loe_ws);
  d->loe_ws = nullptr;
  d->loe_ws_bytes = 0;
  cudaError_t e = cudaMalloc(&d->loe_ws, need);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (stored-value workspace)");
  d->loe_ws_bytes = need;
  return ACE_OK;
}

void fill_loe_args(const ace_dag* d, const DevTaskSet& dt, const void* A, const void* phibar, int64_t n_env,
                   void* phi, void* dA, dev::LoeArgs& a) {
  const Plan& p = d->plan;
  a.ws = static_cast<float*>(d->loe_ws);
  a.A = static_cast<const float*>(A);
  a.phibar = static_cast<const float*>(phibar);
  a.phi = static_cast<float*>(phi);
  a.dA = static_cast<float*>(dA);
  a.n_env = n_env;
  a.n_tiles = (n_env + 31) / 32;
  a.K = p.K;
  a.n_slots = p.n_slots;
  a.n_g = p.n_g;
  a.fwd_slot = d->fwd_slot;
  a.fwd_l = d->fwd_l;
  a.fwd_r = d->fwd_r;
  a.rev_slot = d->rev_slot;
  a.rev_l = d->rev_l;
  a.rev_r = d->rev_r;
  a.n_fwd_levels = (int32_t)p.fwd.off.size() - 1;
  a.n_rev_levels = (int32_t)p.rev.off.size() - 1;
  for (int i = 0; i <= dev::kMaxLevels; ++i) {
    a.fwd_off[i] = i < (int)p.fwd.off.size() ? p.fwd.off[i] : 0;
    a.rev_off[i] = i < (int)p.rev.off.size() ? p.rev.off[i] : 0;
  }
  a.stream = dt.loe_stream;
  for (int w = 0; w <= kLoeWarps; ++w) a.wbeg[w] = dt.loe_wbeg[w];
  a.check = checked_mode() ? 1 : 0;
  a.status = d->status;
}

// Several channels, forward only, one environment per lane (stored values in the global workspace).
ace_status run_loe_multi(ace_dag* d, DevTaskSet& dt, const void* A, int64_t n_env, int n_out, int readout, void* phi,
                         cudaStream_t st) {
  int nt = 0;
  const void* k = loe_multi_kernel_ptr(readout, &nt);
  if (!k) return fail(ACE_ERR_UNSUPPORTED, "no kernel for this readout mode");
  const size_t smem = loe_multi_smem(nt);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  int bps = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, nt, smem)) != cudaSuccess)
    return cuda_fail(e, "occupancy query");
  if (bps < 1) return fail(ACE_ERR_UNSUPPORTED, "several-channel kernel cannot be resident");
  const int64_t n_tiles = (n_env + 31) / 32;
  const int64_t grid = std::min<int64_t>(n_tiles, (int64_t)d->sm_count * bps);
  ace_status s = grow_loe_workspace(d, (size_t)grid * d->plan.n_slots * 32 * sizeof(float));
  if (s != ACE_OK) return s;
  dev::LoeArgs a{};
  fill_loe_args(d, dt, A, nullptr, n_env, phi, nullptr, a);
  e = launch_loe_multi(k, (int)grid, nt, smem, a, dt.loe_istream, dt.cvals16, n_out, st);
  if (e != cudaSuccess) return cuda_fail(e, "several-channel kernel launch");
  return ACE_OK;
}

// One environment per lane (global: stored values in a global workspace; wide: two environments
// per lane, 64 per CTA, global workspace).
ace_status run_loe(ace_dag* d, DevTaskSet& dt, const void* A, const void* phibar, int64_t n_env, int readout,
                   void* phi, void* dA, bool grad, bool global, cudaStream_t st, bool wide = false) {
  int nt = 0;
  const void* k = wide ? loe_wide_kernel_ptr(grad, readout, &nt) : loe_kernel_ptr(grad, readout, global, &nt);
  if (!k) return fail(ACE_ERR_UNSUPPORTED, "no kernel for this readout mode");
  const int tile = wide ? 64 : 32;
  const size_t smem = wide ? loe_wide_smem(nt)
                           : global ? loe_global_smem(nt) : loe_smem(d->plan.n_slots, d->plan.n_g, grad, nt);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  int bps = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, nt, smem)) != cudaSuccess)
    return cuda_fail(e, "occupancy query");
  if (bps < 1) return fail(ACE_ERR_UNSUPPORTED, "one-environment-per-lane kernel cannot be resident");
  const int64_t n_tiles = (n_env + tile - 1) / tile;
  const int64_t grid = std::min<int64_t>(n_tiles, (int64_t)d->sm_count * bps);
  if (global || wide) {
    // one slice of stored values (and adjoints) per CTA, grown on demand and kept in the graph handle
    const size_t need = (size_t)grid * (wide ? loe_wide_bytes_per_cta(d->plan.n_slots, d->plan.n_g, grad)
                                             : loe_global_bytes_per_cta(d->plan.n_slots, d->plan.n_g, grad));
    if (need > d->loe_ws_bytes) {
      if (d->loe_ws) cudaFree(d->loe_ws);
      d->loe_ws = nullptr;
      d->loe_ws_bytes = 0;
      if ((e = cudaMalloc(&d->loe_ws, need)) != cudaSuccess) return cuda_fail(e, "cudaMalloc (stored-value workspace)");
      d->loe_ws_bytes = need;
    }
  }
  static_assert(kLoeWarps == dev::kLoeStreamWarps, "per-warp stream layout and kernel disagree");
  dev::LoeArgs a{};
  fill_loe_args(d, dt, A, phibar, n_env, phi, dA, a);
  a.n_tiles = n_tiles;  // 64 environments per tile for the two-environments-per-lane form
  void* args[] = {&a};
  e = cudaLaunchKernel(k, dim3((unsigned)grid), dim3(nt), args, smem, st);
  if (e != cudaSuccess) return cuda_fail(e, "fused kernel launch");
  return ACE_OK;
}

ace_status run_fused(ace_dag* d, const void* A, const void* c, const void* phibar, int64_t n_env, int n_out,
                     int dtype, int readout, void* phi, void* dA, bool grad, cudaStream_t st) {
  DevTaskSet& dt = grad ? d->sym : d->one;
  ace_status s = bind(d, dt, c, n_out, dtype, st);
  if (s != ACE_OK) return s;
  const int npad = nout_pad_of(n_out);
  // kernel choice: environment overrides (ACE_KERNEL, ACE_TILE_E), else the autotuned choice for
  // this (dtype, channels, adjoint), else one environment per lane whenever it fits
  int choice = kernel_choice(), E_force = 0;
  if (const char* v = std::getenv("ACE_TILE_E")) E_force = std::atoi(v);
  if (choice == 0 && E_force == 0) {
    auto it = d->tuned.find(std::make_tuple(dtype, npad, grad ? 1 : 0));
    if (it != d->tuned.end()) {
      choice = it->second.first;
      E_force = it->second.second;
    }
  }
  const bool multi_ok = dtype == ACE_F32 && n_out > 1 && !grad && dt.multi_bound;
  if (choice == 4 && !multi_ok)
    return fail(ACE_ERR_UNSUPPORTED, "ACE_KERNEL=loem: FP32 forward requests with several channels only");
  if (choice == 4) return run_loe_multi(d, dt, A, n_env, n_out, readout, phi, st);
  const bool loeg_ok = dtype == ACE_F32 && n_out == 1 && dt.rm_bound;
  const bool loe_ok = loeg_ok && loe_smem(d->plan.n_slots, d->plan.n_g, grad, 1024) <= (size_t)d->smem_optin;
  if (choice == 2 && !loe_ok) return fail(ACE_ERR_UNSUPPORTED, "ACE_KERNEL=loe: graph or request does not fit");
  if ((choice == 3 || choice == 5) && !loeg_ok)
    return fail(ACE_ERR_UNSUPPORTED, "ACE_KERNEL=loeg/loeg2: FP32 one-channel requests only");
  if (choice == 3) return run_loe(d, dt, A, phibar, n_env, readout, phi, dA, grad, true, st);
  if (choice == 5) return run_loe(d, dt, A, phibar, n_env, readout, phi, dA, grad, true, st, true);
  if (loe_ok && choice != 1) return run_loe(d, dt, A, phibar, n_env, readout, phi, dA, grad, false, st);
  int E = 0, nt = 0;
  size_t smem = 0;
  const void* k = nullptr;
  bool stage = false;
  const int ro = dtype == ACE_F32 ? readout : 0;
  s = dt.col16 ? choose_tile(d, dtype, npad, grad, ro, n_env, E_force, &E, &nt, &smem, &k, &stage)
               : fail(ACE_ERR_UNSUPPORTED, "more than 65535 stored values per environment");
  if (s != ACE_OK) {
    // the stored values of one environment do not fit on chip: keep them in global memory, two
    // environments per lane (measured faster than one: D = 20 34.7 against 41.2 ms, D = 24 433
    // against 527 ms, 16,384 environments)
    if (loeg_ok && choice != 1) return run_loe(d, dt, A, phibar, n_env, readout, phi, dA, grad, true, st, true);
    return s;
  }
  if (const char* v = std::getenv("ACE_STAGE")) stage = stage && v[0] != '0';  // ACE_STAGE=0: plain loads of A
  if (!k) return fail(ACE_ERR_UNSUPPORTED, "no kernel for this readout mode");
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  int bps = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, nt, smem);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  if (bps < 1) return fail(ACE_ERR_UNSUPPORTED, "fused kernel cannot be resident with this tile");
  const int64_t n_tiles = (n_env + E - 1) / E;
  const int64_t grid = std::min<int64_t>(n_tiles, (int64_t)d->sm_count * bps);
  const Plan& p = d->plan;
  auto fill = [&](auto& a) {
    using TT = std::remove_pointer_t<decltype(a.phi)>;
    a.A = static_cast<const TT*>(A);
    a.phibar = static_cast<const TT*>(phibar);
    a.phi = static_cast<TT*>(phi);
    a.dA = static_cast<TT*>(dA);
    a.n_env = n_env;
    a.n_tiles = n_tiles;
    a.K = p.K;
    a.n_slots = p.n_stored;  // the slots this kernel keeps in shared memory
    a.n_g = p.n_g;
    a.n_out = n_out;
    a.fwd_slot = d->fwds_slot;
    a.fwd_l = d->fwds_l;
    a.fwd_r = d->fwds_r;
    a.pull = d->pull;
    a.n_fwd_levels = (int32_t)p.fwd_stored.off.size() - 1;
    a.n_pull_levels = (int32_t)p.pull.lvl.size() - 1;
    for (int i = 0; i <= dev::kMaxLevels; ++i) {
      a.fwd_off[i] = i < (int)p.fwd_stored.off.size() ? p.fwd_stored.off[i] : 0;
      a.pull_lvl[i] = i < (int)p.pull.lvl.size() ? p.pull.lvl[i] : 0;
    }
    a.tasks = dt.tasks;
    a.slice_off = dt.slice_off;
    a.slice_steps = dt.slice_steps;
    a.n_slices = dt.n_slices;
    a.col16 = dt.col16;
    a.col4 = dt.col4;
    a.off4 = dt.off4;
    a.vals4 = dt.vals4;
    a.gs = dev::g_stride(p.n_g);
    a.genc = grad && d->genc ? 1 : 0;
    a.gperm = grad && d->genc ? d->g_perm_dev : nullptr;
    a.vals = static_cast<const TT*>(dt.vals);
    a.lin = static_cast<const TT*>(dt.lin);
    a.cold_tasks = dt.cold_tasks;
    a.cold_slice_off = dt.cold_slice_off;
    a.cold_slice_steps = dt.cold_slice_steps;
    a.n_cold_slices = dt.n_cold_slices;
    a.cold_cab = dt.cold_cab;
    a.cold_vals = static_cast<const TT*>(dt.cold_vals);
    a.check = checked_mode() ? 1 : 0;
    a.stage = stage ? 1 : 0;
    // test hook for the bounded wait: the staged copies are waited for but never issued, so every
    // CTA's first wait times out (about a second), reports ACE_ERR_TIMEOUT and reads A directly
    if (const char* v = std::getenv("ACE_TEST_STAGE_TIMEOUT")) a.stage_no_issue = v[0] == '1' ? 1 : 0;
    a.status = d->status;
  };
  if (dtype == ACE_F32) {
    dev::FusedArgs<float> a{};
    fill(a);
    void* args[] = {&a};
    e = cudaLaunchKernel(k, dim3((unsigned)grid), dim3(nt), args, smem, st);
  } else {
    dev::FusedArgs<double> a{};
    fill(a);
    void* args[] = {&a};
    e = cudaLaunchKernel(k, dim3((unsigned)grid), dim3(nt), args, smem, st);
  }
  if (e != cudaSuccess) return cuda_fail(e, "fused kernel launch");
  return ACE_OK;
}

// Environments per tile of the kernel form that an evaluation of this request takes
// (the same choice as run_fused: forced, tuned, else one environment per lane when it
// fits, else tile per lane, else the global workspace): 32 for the one-environment-per-lane
// forms, E for tile per lane.
int64_t tile_envs_of(const ace_dag* d, const DevTaskSet& dt, int dtype, int n_out, int readout, bool grad,
                     int64_t n_env) {
  const int npad = nout_pad_of(n_out);
  int choice = kernel_choice(), E_force = 0;
  if (const char* v = std::getenv("ACE_TILE_E")) E_force = std::atoi(v);
  if (choice == 0 && E_force == 0) {
    auto it = d->tuned.find(std::make_tuple(dtype, npad, grad ? 1 : 0));
    if (it != d->tuned.end()) {
      choice = it->second.first;
      E_force = it->second.second;
    }
  }
  const bool loeg_ok = dtype == ACE_F32 && n_out == 1 && dt.rm_bound;
  const bool loe_ok = loeg_ok && loe_smem(d->plan.n_slots, d->plan.n_g, grad, 1024) <= (size_t)d->smem_optin;
  if (choice == 5) return 64;
  if (choice == 2 || choice == 3 || choice == 4 || (loe_ok && choice != 1)) return 32;
  int E = 0, nt = 0;
  size_t smem = 0;
  const void* k = nullptr;
  bool stage = false;
  const int ro = dtype == ACE_F32 ? readout : 0;
  if (dt.col16 && choose_tile(d, dtype, npad, grad, ro, n_env, E_force, &E, &nt, &smem, &k, &stage) == ACE_OK)
    return std::max(E, 1);
  return loeg_ok ? 64 : 32;  // the global-workspace fallback: two environments per lane
}

// Automatic chunk size of the host-buffer entry points: a third of the batch, but at least
// 8 MiB of A (smaller evaluations are launch-bound) and 4 x SMs tiles of the kernel form
// (fewer tiles leave the last wave of a chunk's evaluation mostly idle).  Measured on the
// stress graph (16,384 environments, tiles of 4): thirds 2.98 ms, quarters 3.03, eighths
// 3.38, one piece 3.30; on the paper-degree graph (tiles of 32 environments, 44 ms of
// evaluation) thirds lost a quarter of the throughput to the tail.
int64_t auto_chunk(const ace_dag* d, const DevTaskSet& dt, int dtype, int n_out, int readout, bool grad,
                   int64_t n_env, size_t row_bytes) {
  const int64_t by_bytes = (int64_t)((8u << 20) / row_bytes) + 1;
  const int64_t by_tiles = 4 * (int64_t)std::max(d->sm_count, 1) * tile_envs_of(d, dt, dtype, n_out, readout, grad,
                                                                                 n_env);
  return std::max<int64_t>({(n_env + 2) / 3, by_bytes, by_tiles});
}

// Streams, events and two staging slots of `bytes` each for the host-buffer entry points.
ace_status ensure_host_pipeline(ace_dag* d, size_t bytes) {
  cudaError_t e;
  for (cudaStream_t& h : d->hstream)
    if (!h && (e = cudaStreamCreateWithFlags(&h, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_fail(e, "cudaStreamCreateWithFlags");
  for (cudaEvent_t* ev : {&d->hev_fork, &d->hev_in[0], &d->hev_in[1], &d->hev_done[0], &d->hev_done[1], &d->hev_out[0],
                          &d->hev_out[1], &d->hev_join[0], &d->hev_join[1], &d->hev_join[2]})
    if (!*ev && (e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "cudaEventCreateWithFlags");
  if (bytes > d->hslot_bytes) {
    for (void*& p : d->hslot) {
      if (p) cudaFree(p);
      p = nullptr;
    }
    d->hslot_bytes = 0;
    for (void*& p : d->hslot)
      if ((e = cudaMalloc(&p, bytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc (host-buffer staging)");
    d->hslot_bytes = bytes;
  }
  return ACE_OK;
}

// Chunk sizes of a host-buffer evaluation: equal chunks of `chunk` environments when the caller
// gives a size; otherwise a short first and last chunk (whole waves of the kernel form, SMs x
// environments per tile, at least 2 MiB of A) around two long ones that take the rest, because
// nothing overlaps the copy-in of the first chunk and the copy-out of the last (measured on the
// stress workload: end to end 5.72 M env/s with thirds, 5.85 with 8 MiB edges).  Batches too small
// for that take the automatic size of auto_chunk.
std::vector<int64_t> chunk_plan(const ace_dag* d, const DevTaskSet& dt, int dtype, int n_out, int readout, bool grad,
                                int64_t n_env, size_t row_bytes, int64_t chunk) {
  std::vector<int64_t> out;
  if (chunk == 0) {
    const int64_t wave = (int64_t)std::max(d->sm_count, 1) * tile_envs_of(d, dt, dtype, n_out, readout, grad, n_env);
    const int64_t by_bytes = (int64_t)((2u << 20) / row_bytes) + 1;
    const int64_t edge = (std::max<int64_t>(by_bytes, wave) + wave - 1) / wave * wave;
    const int64_t rest = n_env - 2 * edge;
    const int64_t mid = rest / (2 * wave) * wave;
    if (mid >= 2 * edge) return {edge, mid, rest - mid, edge};
    chunk = auto_chunk(d, dt, dtype, n_out, readout, grad, n_env, row_bytes);
  }
  chunk = std::min(chunk, n_env);
  for (int64_t off = 0; off < n_env; off += chunk) out.push_back(std::min(chunk, n_env - off));
  return out;
}

// Chunked evaluation with host buffers: chunk i is copied in on hstream[0], evaluated on
// hstream[1] and copied out on hstream[2]; slot i mod 2 is reused by chunk i + 2 once the
// evaluation of chunk i has read its A and the copy-out of chunk i has read its outputs.
ace_status eval_host(ace_dag* d, const void* A, const void* c, const void* phibar, int64_t n_env, int n_out,
                     int dtype, int readout, void* phi, void* dA, bool grad, int64_t chunk, cudaStream_t st) {
  ace_status s;
  if ((s = ensure_uploaded(d, st)) != ACE_OK) return s;
  DevTaskSet& dt = grad ? d->sym : d->one;
  if ((s = bind(d, dt, c, n_out, dtype, st)) != ACE_OK) return s;
  if (n_env == 0) return ACE_OK;
  const size_t tsz = dtype == ACE_F32 ? 4 : 8;
  const std::vector<int64_t> plan = chunk_plan(d, dt, dtype, n_out, readout, grad, n_env, (size_t)d->K * tsz, chunk);
  chunk = *std::max_element(plan.begin(), plan.end());
  const size_t a_bytes = dev::align16((size_t)chunk * d->K * tsz);
  const size_t o_bytes = dev::align16((size_t)chunk * n_out * tsz);
  const size_t slot_bytes = a_bytes * (grad ? 2 : 1) + o_bytes * (grad ? 2 : 1);
  if ((s = ensure_host_pipeline(d, slot_bytes)) != ACE_OK) return s;
  cudaStream_t hin = d->hstream[0], hev = d->hstream[1], hout = d->hstream[2];
  cudaError_t e = cudaEventRecord(d->hev_fork, st);
  for (cudaStream_t h : d->hstream)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h, d->hev_fork, 0);
  const unsigned char* Ah = static_cast<const unsigned char*>(A);
  const unsigned char* pbh = static_cast<const unsigned char*>(phibar);
  unsigned char* phih = static_cast<unsigned char*>(phi);
  unsigned char* dAh = static_cast<unsigned char*>(dA);
  const size_t row_a = (size_t)d->K * tsz, row_o = (size_t)n_out * tsz;
  s = ACE_OK;
  int64_t off = 0;
  for (size_t k = 0; k < plan.size() && e == cudaSuccess && s == ACE_OK; off += plan[k], ++k) {
    const int64_t n = plan[k];
    const int b = (int)(k & 1);
    unsigned char* slot = static_cast<unsigned char*>(d->hslot[b]);
    unsigned char* Ad = slot;
    unsigned char* dAd = grad ? slot + a_bytes : nullptr;
    unsigned char* phid = slot + a_bytes * (grad ? 2 : 1);
    unsigned char* pbd = grad ? phid + o_bytes : nullptr;
    // copy in (slot b is free once the evaluation of chunk k - 2 has run)
    if (k >= 2) e = cudaStreamWaitEvent(hin, d->hev_done[b], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Ad, Ah + off * row_a, n * row_a, cudaMemcpyHostToDevice, hin);
    if (e == cudaSuccess && grad && phibar)
      e = cudaMemcpyAsync(pbd, pbh + off * row_o, n * row_o, cudaMemcpyHostToDevice, hin);
    if (e == cudaSuccess) e = cudaEventRecord(d->hev_in[b], hin);
    // evaluate (after the copy-out of chunk k - 2 has read this slot's outputs)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hev, d->hev_in[b], 0);
    if (e == cudaSuccess && k >= 2) e = cudaStreamWaitEvent(hev, d->hev_out[b], 0);
    if (e != cudaSuccess) break;
    s = run_fused(d, Ad, nullptr, (grad && phibar) ? pbd : nullptr, n, n_out, dtype, readout, phi ? phid : nullptr,
                  dAd, grad, hev);
    if (s != ACE_OK) break;
    e = cudaEventRecord(d->hev_done[b], hev);
    // copy out
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hout, d->hev_done[b], 0);
    if (e == cudaSuccess && grad) e = cudaMemcpyAsync(dAh + off * row_a, dAd, n * row_a, cudaMemcpyDeviceToHost, hout);
    if (e == cudaSuccess && phi) e = cudaMemcpyAsync(phih + off * row_o, phid, n * row_o, cudaMemcpyDeviceToHost, hout);
    if (e == cudaSuccess) e = cudaEventRecord(d->hev_out[b], hout);
  }
  // join: `stream` waits for all three streams (also after an error, so nothing is left unjoined)
  for (int i = 0; i < 3; ++i) {
    if (cudaEventRecord(d->hev_join[i], d->hstream[i]) == cudaSuccess) cudaStreamWaitEvent(st, d->hev_join[i], 0);
  }
  if (s != ACE_OK) return s;
  if (e != cudaSuccess) return cuda_fail(e, "host-buffer evaluation");
  return ACE_OK;
}

ace_status check_eval_args(const ace_dag* d, const void* A, int64_t n_env, int n_out, int dtype, int readout) {
  if (!d) return fail(ACE_ERR_INVALID_ARG, "dag is NULL");
  if (n_env < 0) return fail(ACE_ERR_INVALID_ARG, "n_env must be >= 0");
  if (n_out < 1 || n_out > 16) return fail(ACE_ERR_INVALID_ARG, "n_out must be in [1, 16]");
  if (dtype != ACE_F32 && dtype != ACE_F64) return fail(ACE_ERR_INVALID_ARG, "dtype must be ACE_F32 or ACE_F64");
  if (readout < 0 || readout > 2) return fail(ACE_ERR_INVALID_ARG, "unknown readout mode");
  if (n_env > 0 && !A) return fail(ACE_ERR_INVALID_ARG, "A is NULL");
  if (A && !aligned16(A)) return fail(ACE_ERR_INVALID_ARG, "A must be 16-byte aligned");
  return ACE_OK;
}


// Which form the forces pipeline takes: the fused kernel (pooling, graph forward and adjoint and
// pooling adjoint in one launch, A and dA in shared memory) or the three kernels.  ACE_FORCES=fused
// or ACE_FORCES=split chooses; by default the three kernels, measured faster on GB300 (50,000
// environments of 10-60 neighbours, K = 392: 0.645 ms against 0.759 ms): with one tile per SM the
// fused kernel's phases cannot overlap, and its last wave of tiles leaves SMs idle.
constexpr bool kForcesFusedDefault = false;

// Shared memory of the fused forces kernel for this request, or 0 when the three kernels run
// (bound: the one-channel FP32 coefficients are bound, as the forces entry points make them;
// smem_optin: the device's shared memory limit per CTA).
size_t forces_fused_bytes(const ace_dag* d, int nmin, int nmax, int lmax, int kmax, bool bound, int smem_optin) {
  const char* v = std::getenv("ACE_FORCES");
  const bool fused = v && std::strcmp(v, "fused") == 0 ? true : v && std::strcmp(v, "split") == 0 ? false
                                                                                                 : kForcesFusedDefault;
  if (!fused || !bound) return 0;
  if (loe_smem(d->plan.n_slots, d->plan.n_g, true, 1024) > (size_t)smem_optin) return 0;
  const size_t fsmem = forces_fused_smem(d->plan.n_slots, d->plan.n_g, d->K, nmin, nmax, lmax, kmax);
  return fsmem <= (size_t)smem_optin ? fsmem : 0;
}

// The forces pipeline of n environments on stream st (device buffers; offsets index pos): the fused
// kernel when forces_fused_bytes allows it, else pooling -> forward + adjoint -> pooling adjoint
// through A_d and dA_d (n x K floats each, required then).
ace_status forces_pipeline(ace_dag* d, const float* pos_d, const float* mu_d, const int64_t* off_d, int64_t n,
                           float rc, int nmin, int nmax, int lmax, int kmax, int readout, float* phi_d, float* F_d,
                           float* A_d, float* dA_d, cudaStream_t st) {
  DevTaskSet& dt = d->sym;
  const size_t fsmem = forces_fused_bytes(d, nmin, nmax, lmax, kmax, dt.rm_bound, d->smem_optin);
  cudaError_t e;
  if (fsmem > 0) {
    dev::LoeArgs a{};
    fill_loe_args(d, dt, nullptr, nullptr, n, phi_d, nullptr, a);
    const int64_t grid = std::min<int64_t>(a.n_tiles, (int64_t)d->sm_count);
    e = launch_forces_fused(a, pos_d, off_d, rc, nmin, nmax, lmax, readout, F_d, (int)grid, fsmem, st);
    if (e != cudaSuccess) return cuda_fail(e, "fused forces launch");
    return ACE_OK;
  }
  if (!A_d || !dA_d) return fail(ACE_ERR_INVALID_ARG, "internal: no A/dA buffers for the three-kernel forces path");
  if ((e = launch_pool(pos_d, mu_d, off_d, n, rc, nmin, nmax, lmax, kmax, A_d, st)) != cudaSuccess)
    return cuda_fail(e, "pooling kernel launch");
  ace_status s = run_fused(d, A_d, nullptr, nullptr, n, 1, ACE_F32, readout, phi_d, dA_d, true, st);
  if (s != ACE_OK) return s;
  if ((e = launch_pool_grad(pos_d, mu_d, off_d, n, rc, nmin, nmax, lmax, kmax, dA_d, -1.f, F_d, st)) != cudaSuccess)
    return cuda_fail(e, "pooling adjoint launch");
  return ACE_OK;
}

}  // namespace

extern "C" {

const char* ace_last_error(void) { return ace::last_error_cstr(); }

int32_t ace_abi_version(void) { return ACE_ABI_VERSION; }

ace_status ace_build_spec(const ace_spec_params* params, ace_spec** out) {
  NvtxRange nvtx_range("ace_build_spec");
  if (!params || !out) return fail(ACE_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  try {
    std::unique_ptr<Spec> s;
    ace_status st = build_spec(*params, s);
    if (st != ACE_OK) return st;
    auto* h = new ace_spec;
    h->s = std::move(s);
    *out = h;
    return ACE_OK;
  } catch (const std::bad_alloc&) {
    return fail(ACE_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(ACE_ERR_INVALID_ARG, "unexpected error building the index set");
  }
}

ace_status ace_spec_info(const ace_spec* spec, int64_t* n_basis, int32_t* K, int64_t* counts_per_nu) {
  if (!spec) return fail(ACE_ERR_INVALID_ARG, "spec is NULL");
  if (n_basis) *n_basis = spec->s->n_basis();
  if (K) *K = spec->s->K;
  if (counts_per_nu)
    std::memcpy(counts_per_nu, spec->s->counts_per_nu.data(), spec->s->counts_per_nu.size() * sizeof(int64_t));
  return ACE_OK;
}

ace_status ace_spec_tuples(const ace_spec* spec, int32_t* tuples, int32_t* deg) {
  if (!spec) return fail(ACE_ERR_INVALID_ARG, "spec is NULL");
  if (tuples) std::memcpy(tuples, spec->s->tuples.data(), spec->s->tuples.size() * sizeof(int32_t));
  if (deg) std::memcpy(deg, spec->s->deg.data(), spec->s->deg.size() * sizeof(int32_t));
  return ACE_OK;
}

void ace_spec_free(ace_spec* spec) { delete spec; }

// Largest number of stored slots for which a tile of four environments (FP32,
// one channel, forward + adjoint, 1024 threads, with the staging buffer) fits in
// the 227 KB of shared memory a CTA can have on this GPU; ACE_PLAN_STORED=<n>
// sets the limit directly (tests: forces entries to the cold path).
int64_t stored_slot_limit(int32_t K, int32_t n_g) {
  if (const char* v = std::getenv("ACE_PLAN_STORED")) return std::max<int64_t>(0, std::atoll(v));
  constexpr size_t kSmemOptin = 232448;
  int64_t lo = 0, hi = 65535;
  while (lo < hi) {  // largest n with the layout inside the budget
    const int64_t mid = (lo + hi + 1) / 2;
    if (dev::smem_layout(4, 1, true, (int)mid, n_g, 1024, 4, K, true).total <= kSmemOptin) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

ace_status ace_build_dag(const ace_spec* spec, int32_t algo, int32_t split_rule, int32_t n_split, ace_dag** out) {
  NvtxRange nvtx_range("ace_build_dag");
  if (!spec || !out) return fail(ACE_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  try {
    auto d = std::make_unique<ace_dag>();
    ace_status st;
    {
      NvtxRange phase("graph");
      st = build_graph(*spec->s, algo, split_rule, n_split, d->g);
    }
    if (st != ACE_OK) return st;
    int task_len = 64;
    if (const char* v = std::getenv("ACE_TASK_LEN")) task_len = std::max(1, std::atoi(v));
    d->opts = GraphOptions{algo, split_rule, n_split, task_len};
    {
      NvtxRange phase("plan");
      st = build_plan(*spec->s, d->g, task_len, stored_slot_limit, d->plan);
    }
    if (st != ACE_OK) return st;
    d->K = spec->s->K;
    d->n_basis = spec->s->n_basis();
    *out = d.release();
    return ACE_OK;
  } catch (const std::bad_alloc&) {
    return fail(ACE_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(ACE_ERR_INVALID_ARG, "unexpected error building the graph");
  }
}

ace_status ace_dag_save(const ace_spec* spec, const ace_dag* dag, const char* path) {
  NvtxRange nvtx_range("ace_dag_save");
  if (!spec || !dag || !path) return fail(ACE_ERR_INVALID_ARG, "NULL argument");
  if (spec->s->K != dag->K || spec->s->n_basis() != dag->n_basis ||
      (int64_t)dag->g.basis_node.size() != dag->n_basis)
    return fail(ACE_ERR_INVALID_ARG, "the graph was not built from this index set");
  try {
    return save_graph(path, *spec->s, dag->g, dag->opts);
  } catch (const std::bad_alloc&) {
    return fail(ACE_ERR_OOM, "host allocation failed");
  }
}

ace_status ace_dag_load(const char* path, ace_spec_params* params, ace_spec** spec_out, ace_dag** dag_out) {
  NvtxRange nvtx_range("ace_dag_load");
  if (!path || !spec_out || !dag_out) return fail(ACE_ERR_INVALID_ARG, "NULL argument");
  *spec_out = nullptr;
  *dag_out = nullptr;
  try {
    std::unique_ptr<Spec> s;
    auto d = std::make_unique<ace_dag>();
    ace_status st = load_graph(path, s, d->g, d->opts);
    if (st != ACE_OK) return st;
    st = build_plan(*s, d->g, d->opts.task_len, stored_slot_limit, d->plan);
    if (st != ACE_OK) return st;
    d->K = s->K;
    d->n_basis = s->n_basis();
    if (params) *params = s->p;
    auto* h = new ace_spec;
    h->s = std::move(s);
    *spec_out = h;
    *dag_out = d.release();
    return ACE_OK;
  } catch (const std::bad_alloc&) {
    return fail(ACE_ERR_OOM, "host allocation failed");
  } catch (...) {
    return fail(ACE_ERR_INVALID_ARG, "unexpected error reading the graph file");
  }
}

ace_status ace_dag_info(const ace_dag* dag, int64_t* n_nodes, int64_t* n_aux, int64_t* n_operands,
                        int32_t* n_levels) {
  if (!dag) return fail(ACE_ERR_INVALID_ARG, "dag is NULL");
  const Graph& g = dag->g;
  if (n_nodes) *n_nodes = g.n_nodes();
  if (n_aux) {
    int64_t a = 0;
    for (uint8_t x : g.is_aux) a += x;
    *n_aux = a;
  }
  if (n_operands) *n_operands = dag->plan.n_slots - dag->plan.K;
  if (n_levels) {
    int32_t m = 1;
    for (int32_t o : g.order) m = std::max(m, o);
    *n_levels = m;
  }
  return ACE_OK;
}

ace_status ace_dag_export(const ace_dag* dag, int32_t* left, int32_t* right, int32_t* level, uint8_t* is_aux,
                          int32_t* basis_node) {
  if (!dag) return fail(ACE_ERR_INVALID_ARG, "dag is NULL");
  const Graph& g = dag->g;
  const size_t n = (size_t)g.n_nodes();
  if (left) std::memcpy(left, g.left.data(), n * sizeof(int32_t));
  if (right) std::memcpy(right, g.right.data(), n * sizeof(int32_t));
  if (level) std::memcpy(level, g.order.data(), n * sizeof(int32_t));
  if (is_aux) std::memcpy(is_aux, g.is_aux.data(), n);
  if (basis_node) std::memcpy(basis_node, g.basis_node.data(), g.basis_node.size() * sizeof(int32_t));
  return ACE_OK;
}

ace_status ace_dag_plan_info(const ace_dag* dag, int64_t* n_slots, int64_t* n_sinks, int64_t* n_entries,
                             int64_t* smem_bytes_f32) {
  if (!dag) return fail(ACE_ERR_INVALID_ARG, "dag is NULL");
  const Plan& p = dag->plan;
  if (n_slots) *n_slots = p.n_slots;
  if (n_sinks) *n_sinks = p.n_sinks;
  if (n_entries) *n_entries = p.sym.n_entries;
  if (smem_bytes_f32) *smem_bytes_f32 = (int64_t)(p.n_stored + p.n_g) * 4;
  return ACE_OK;
}

ace_status ace_dag_validate(const ace_dag* dag) {
  if (!dag) return fail(ACE_ERR_INVALID_ARG, "dag is NULL");
  return validate_plan(dag->plan);
}

ace_status ace_dag_plan_array(const ace_dag* dag, const char* name, int32_t* out, int64_t* count) {
  if (!dag || !name || !count) return fail(ACE_ERR_INVALID_ARG, "NULL argument");
  const Plan& p = dag->plan;
  std::vector<int32_t> tmp;
  const std::vector<int32_t>* v = nullptr;
  const std::string n(name);
  auto from_ts = [&](const TaskSet& ts, const std::string& field) -> bool {
    if (field == "tasks") {
      for (const Task& t : ts.tasks) tmp.insert(tmp.end(), {t.row, t.flags, t.pl, t.pr});
      v = &tmp;
    } else if (field == "slice_off") v = &ts.slice_off;
    else if (field == "slice_steps") v = &ts.slice_steps;
    else if (field == "col") v = &ts.col;
    else if (field == "ebasis") v = &ts.ebasis;
    else if (field == "ew2") {
      tmp.assign(ts.ew2.begin(), ts.ew2.end());
      v = &tmp;
    } else if (field == "rm_tasks") {
      for (const Task& t : ts.rm_tasks) tmp.insert(tmp.end(), {t.row, t.flags, t.pl, t.pr});
      v = &tmp;
    } else if (field == "cold_tasks") {
      for (const Task& t : ts.cold_tasks) tmp.insert(tmp.end(), {t.row, t.flags, t.pl, t.pr});
      v = &tmp;
    } else if (field == "cold_slice_off") v = &ts.cold_slice_off;
    else if (field == "cold_slice_steps") v = &ts.cold_slice_steps;
    else if (field == "cold_ca") v = &ts.cold_ca;
    else if (field == "cold_cb") v = &ts.cold_cb;
    else if (field == "cold_ebasis") v = &ts.cold_ebasis;
    else if (field == "cold_ew2") {
      tmp.assign(ts.cold_ew2.begin(), ts.cold_ew2.end());
      v = &tmp;
    } else if (field == "rm_off") v = &ts.rm_off;
    else if (field == "rm_col") v = &ts.rm_col;
    else if (field == "loe_wbeg") v = &ts.loe_wbeg;
    else if (field == "loe_hpos") v = &ts.loe_hpos;
    else if (field == "loe_spos") v = &ts.loe_spos;
    else if (field == "loe_sval") v = &ts.loe_sval;
    else if (field == "rm_ebasis") v = &ts.rm_ebasis;
    else if (field == "rm_ew2") {
      tmp.assign(ts.rm_ew2.begin(), ts.rm_ew2.end());
      v = &tmp;
    } else return false;
    return true;
  };
  if (n == "slot_node") v = &p.slot_node;
  else if (n == "slot_basis") v = &p.slot_basis;
  else if (n == "n_g") {
    tmp = {p.n_g};
    v = &tmp;
  } else if (n == "fwd_slot") v = &p.fwd.slot;
  else if (n == "fwd_l") v = &p.fwd.l;
  else if (n == "fwd_r") v = &p.fwd.r;
  else if (n == "fwd_off") v = &p.fwd.off;
  else if (n == "rev_slot") v = &p.rev.slot;
  else if (n == "rev_l") v = &p.rev.l;
  else if (n == "rev_r") v = &p.rev.r;
  else if (n == "rev_off") v = &p.rev.off;
  else if (n == "n_stored") {
    tmp = {p.n_stored};
    v = &tmp;
  } else if (n == "fwd_stored_slot") v = &p.fwd_stored.slot;
  else if (n == "fwd_stored_l") v = &p.fwd_stored.l;
  else if (n == "fwd_stored_r") v = &p.fwd_stored.r;
  else if (n == "fwd_stored_off") v = &p.fwd_stored.off;
  else if (n == "pull_tgt") v = &p.pull.tgt;
  else if (n == "pull_src") v = &p.pull.src;
  else if (n == "pull_par") v = &p.pull.par;
  else if (n == "pull_lvl") v = &p.pull.lvl;
  else if (n == "g_perm") v = &p.g_perm;
  else if (n.rfind("sym_", 0) == 0) {
    if (!from_ts(p.sym, n.substr(4))) v = nullptr;
  } else if (n.rfind("one_", 0) == 0) {
    if (!from_ts(p.one, n.substr(4))) v = nullptr;
  }
  if (!v) return fail(ACE_ERR_INVALID_ARG, "unknown plan array: " + n);
  *count = (int64_t)v->size();
  if (out && !v->empty()) std::memcpy(out, v->data(), v->size() * sizeof(int32_t));
  return ACE_OK;
}

void ace_dag_free(ace_dag* dag) {
  if (!dag) return;
  if (dag->device >= 0) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(dag->device);
    for (void* p : dag->allocations) cudaFree(p);
    if (dag->loe_ws) cudaFree(dag->loe_ws);
    for (void* p : dag->hslot)
      if (p) cudaFree(p);
    if (dag->fbuf) cudaFree(dag->fbuf);
    if (dag->fwork) cudaFree(dag->fwork);
    for (cudaStream_t h : dag->hstream)
      if (h) cudaStreamDestroy(h);
    for (cudaEvent_t ev : {dag->hev_fork, dag->hev_in[0], dag->hev_in[1], dag->hev_done[0], dag->hev_done[1],
                           dag->hev_out[0], dag->hev_out[1], dag->hev_join[0], dag->hev_join[1], dag->hev_join[2]})
      if (ev) cudaEventDestroy(ev);
    for (DevTaskSet* t : {&dag->sym, &dag->one}) {
      if (t->vals) cudaFree(t->vals);
      if (t->lin) cudaFree(t->lin);
      if (t->vals4) cudaFree(t->vals4);
      if (t->cold_vals) cudaFree(t->cold_vals);
      if (t->loe_stream) cudaFree(t->loe_stream);
      if (t->loe_istream) cudaFree(t->loe_istream);
      if (t->cvals16) cudaFree(t->cvals16);
    }
    cudaSetDevice(cur);
  }
  delete dag;
}

ace_status ace_dag_upload(ace_dag* dag, void* stream) {
  NvtxRange nvtx_range("ace_dag_upload");
  if (!dag) return fail(ACE_ERR_INVALID_ARG, "dag is NULL");
  return ensure_uploaded(dag, (cudaStream_t)stream);
}

ace_status ace_eval(ace_dag* dag, const void* A, const void* c, int64_t n_env, int32_t n_out, int32_t dtype,
                    int32_t readout, void* phi, void* stream) {
  NvtxRange nvtx_range("ace_eval");
  ace_status s = check_eval_args(dag, A, n_env, n_out, dtype, readout);
  if (s != ACE_OK) return s;
  if (n_env > 0 && !phi) return fail(ACE_ERR_INVALID_ARG, "phi is NULL");
  if (phi && !aligned16(phi)) return fail(ACE_ERR_INVALID_ARG, "phi must be 16-byte aligned");
  if (c && !aligned16(c)) return fail(ACE_ERR_INVALID_ARG, "c must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  if ((s = ensure_uploaded(dag, st)) != ACE_OK) return s;
  if (n_env == 0) return bind(dag, dag->one, c, n_out, dtype, st);
  return run_fused(dag, A, c, nullptr, n_env, n_out, dtype, readout, phi, nullptr, false, st);
}

ace_status ace_eval_grad(ace_dag* dag, const void* A, const void* c, const void* phi_bar, int64_t n_env,
                         int32_t n_out, int32_t dtype, int32_t readout, void* phi, void* dA, void* stream) {
  NvtxRange nvtx_range("ace_eval_grad");
  ace_status s = check_eval_args(dag, A, n_env, n_out, dtype, readout);
  if (s != ACE_OK) return s;
  if (n_env > 0 && !dA) return fail(ACE_ERR_INVALID_ARG, "dA is NULL");
  for (const void* p : {(const void*)phi, (const void*)dA, phi_bar, c})
    if (p && !aligned16(p)) return fail(ACE_ERR_INVALID_ARG, "pointers must be 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  if ((s = ensure_uploaded(dag, st)) != ACE_OK) return s;
  if (n_env == 0) return bind(dag, dag->sym, c, n_out, dtype, st);
  return run_fused(dag, A, c, phi_bar, n_env, n_out, dtype, readout, phi, dA, true, st);
}

ace_status ace_eval_host(ace_dag* dag, const void* A, const void* c, int64_t n_env, int32_t n_out, int32_t dtype,
                         int32_t readout, void* phi, int64_t chunk_env, void* stream) {
  NvtxRange nvtx_range("ace_eval_host");
  ace_status s = check_eval_args(dag, nullptr, 0, n_out, dtype, readout);
  if (s != ACE_OK) return s;
  if (n_env < 0 || chunk_env < 0) return fail(ACE_ERR_INVALID_ARG, "n_env and chunk_env must be >= 0");
  if (n_env > 0 && (!A || !phi)) return fail(ACE_ERR_INVALID_ARG, "A or phi is NULL");
  if (c && !aligned16(c)) return fail(ACE_ERR_INVALID_ARG, "c must be 16-byte aligned");
  return eval_host(dag, A, c, nullptr, n_env, n_out, dtype, readout, phi, nullptr, false, chunk_env,
                   (cudaStream_t)stream);
}

ace_status ace_eval_grad_host(ace_dag* dag, const void* A, const void* c, const void* phi_bar, int64_t n_env,
                              int32_t n_out, int32_t dtype, int32_t readout, void* phi, void* dA, int64_t chunk_env,
                              void* stream) {
  NvtxRange nvtx_range("ace_eval_grad_host");
  ace_status s = check_eval_args(dag, nullptr, 0, n_out, dtype, readout);
  if (s != ACE_OK) return s;
  if (n_env < 0 || chunk_env < 0) return fail(ACE_ERR_INVALID_ARG, "n_env and chunk_env must be >= 0");
  if (n_env > 0 && (!A || !dA)) return fail(ACE_ERR_INVALID_ARG, "A or dA is NULL");
  if (c && !aligned16(c)) return fail(ACE_ERR_INVALID_ARG, "c must be 16-byte aligned");
  return eval_host(dag, A, c, phi_bar, n_env, n_out, dtype, readout, phi, dA, true, chunk_env, (cudaStream_t)stream);
}

ace_status ace_dag_autotune(ace_dag* dag, int64_t n_env, int32_t n_out, int32_t dtype, int32_t grad, int32_t readout,
                            void* stream, int32_t* best_kind, int32_t* best_E, float* best_ms) {
  NvtxRange nvtx_range("ace_dag_autotune");
  ace_status s = check_eval_args(dag, nullptr, 0, n_out, dtype, readout);
  if (s != ACE_OK) return s;
  if (n_env < 1) return fail(ACE_ERR_INVALID_ARG, "n_env must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  if ((s = ensure_uploaded(dag, st)) != ACE_OK) return s;
  const size_t tsz = dtype == ACE_F32 ? 4 : 8;
  void *A = nullptr, *c = nullptr, *phi = nullptr, *dA = nullptr;
  cudaError_t e;
  auto cleanup = [&]() {
    for (void* p : {A, c, phi, dA})
      if (p) cudaFree(p);
  };
  if ((e = cudaMalloc(&A, (size_t)n_env * dag->K * tsz)) != cudaSuccess ||
      (e = cudaMalloc(&c, (size_t)dag->n_basis * n_out * tsz)) != cudaSuccess ||
      (e = cudaMalloc(&phi, (size_t)n_env * n_out * tsz)) != cudaSuccess ||
      (e = cudaMalloc(&dA, (size_t)n_env * dag->K * tsz)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "cudaMalloc (autotune buffers)");
  }
  // small non-zero inputs (every byte 0x3c: 0.0115 in FP32, 1.6e-18 in FP64), so that the
  // timed arithmetic and shared-memory updates are those of real data
  cudaMemsetAsync(A, 0x3c, (size_t)n_env * dag->K * tsz, st);
  cudaMemsetAsync(c, 0x3c, (size_t)dag->n_basis * n_out * tsz, st);
  const int npad = nout_pad_of(n_out);
  const auto key = std::make_tuple((int)dtype, npad, grad ? 1 : 0);
  dag->tuned.erase(key);
  std::vector<std::pair<int, int>> cands = {{2, 0}, {3, 0}, {4, 0}, {5, 0}};
  for (int E : {1, 2, 4, 8, 16}) cands.push_back({1, E});
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = -1.f;
  std::pair<int, int> pick{0, 0};
  bool first = true;
  for (auto cand : cands) {
    dag->tuned[key] = cand;
    auto run = [&]() {
      const void* cc = first ? c : nullptr;
      const ace_status r = grad ? ace_eval_grad(dag, A, cc, nullptr, n_env, n_out, dtype, readout, phi, dA, stream)
                                : ace_eval(dag, A, cc, n_env, n_out, dtype, readout, phi, stream);
      if (r == ACE_OK) first = false;
      return r;
    };
    if (run() != ACE_OK) continue;  // configuration not compiled or does not fit
    cudaEventRecord(a, st);
    bool ok = true;
    for (int r = 0; r < 3 && ok; ++r) ok = run() == ACE_OK;
    cudaEventRecord(b, st);
    if (!ok || cudaEventSynchronize(b) != cudaSuccess) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    ms /= 3.f;
    if (best < 0.f || ms < best) {
      best = ms;
      pick = cand;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  dag->tuned.erase(key);
  DevTaskSet& used = grad ? dag->sym : dag->one;  // the zero coefficients must not serve a later NULL c
  used.bound = false;
  used.rm_bound = false;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "autotune");
  }
  cleanup();
  clear_error();
  if (best < 0.f) return fail(ACE_ERR_UNSUPPORTED, "no kernel configuration runs this request");
  dag->tuned[key] = pick;
  if (best_kind) *best_kind = pick.first;
  if (best_E) *best_E = pick.second;
  if (best_ms) *best_ms = best;
  return ACE_OK;
}

ace_status ace_eval_plain_workspace_bytes(const ace_dag* dag, int64_t n_env, int32_t with_grad, size_t* bytes) {
  if (!dag || !bytes) return fail(ACE_ERR_INVALID_ARG, "NULL argument");
  if (n_env < 0) return fail(ACE_ERR_INVALID_ARG, "n_env must be >= 0");
  // n_nodes x n_env x 8 (x 2) bytes, refused where size_t would wrap
  const size_t per_env = (size_t)dag->g.n_nodes() * sizeof(double) * (with_grad ? 2 : 1);
  if (per_env > 0 && (size_t)n_env > SIZE_MAX / per_env)
    return fail(ACE_ERR_INVALID_ARG, "workspace size overflows size_t for n_env = " + std::to_string(n_env));
  *bytes = per_env * (size_t)n_env;
  return ACE_OK;
}

ace_status ace_eval_plain_f64(ace_dag* dag, const double* A, const double* c, const double* phi_bar,
                              int64_t n_env, int32_t n_out, double* phi, double* dA, void* workspace,
                              size_t workspace_bytes, void* stream) {
  NvtxRange nvtx_range("ace_eval_plain_f64");
  ace_status s = check_eval_args(dag, A, n_env, n_out, ACE_F64, 0);
  if (s != ACE_OK) return s;
  if (n_env == 0) return ACE_OK;
  if (!c) return fail(ACE_ERR_INVALID_ARG, "c is NULL");
  if (!phi && !dA) return fail(ACE_ERR_INVALID_ARG, "nothing to compute: phi and dA are NULL");
  size_t need = 0;
  if ((s = ace_eval_plain_workspace_bytes(dag, n_env, dA != nullptr, &need)) != ACE_OK) return s;
  if (!workspace || workspace_bytes < need) return fail(ACE_ERR_INVALID_ARG, "workspace missing or too small");
  cudaStream_t st = (cudaStream_t)stream;
  if ((s = ensure_uploaded(dag, st)) != ACE_OK) return s;
  double* AA = static_cast<double*>(workspace);
  double* abar = dA ? AA + (size_t)dag->g.n_nodes() * n_env : nullptr;
  cudaError_t e = launch_plain_f64(A, c, phi_bar, n_env, n_out, dag->K, dag->g.n_nodes(), dag->node_left,
                                   dag->node_right, dag->node_basis, phi, dA, AA, abar, st);
  if (e != cudaSuccess) return cuda_fail(e, "plain kernel launch");
  return ACE_OK;
}

ace_status ace_eval_plain_f64_static(ace_dag* dag, const double* A, const double* c, const double* phi_bar,
                                     int64_t n_env, int32_t n_out, double* phi, double* dA, void* stream) {
  ace_status s = check_eval_args(dag, A, n_env, n_out, ACE_F64, 0);
  if (s != ACE_OK) return s;
  if (n_env == 0) return ACE_OK;
  if (!c) return fail(ACE_ERR_INVALID_ARG, "c is NULL");
  if (!phi && !dA) return fail(ACE_ERR_INVALID_ARG, "nothing to compute: phi and dA are NULL");
  const int64_t N = dag->g.n_nodes();
  const size_t graph_bytes = (size_t(3) * (size_t)N * sizeof(int32_t) + 255) & ~size_t(255);
  const size_t per_env = (size_t)N * sizeof(double) * (dA ? 2 : 1);
  const size_t cap = static_scratch_bytes();
  // compared by division, so that no product of n_env can wrap around
  const size_t max_env = graph_bytes >= cap ? 0 : (cap - graph_bytes) / per_env;
  if ((uint64_t)n_env > (uint64_t)max_env)
    return fail(ACE_ERR_INVALID_ARG,
                "ace_eval_plain_f64_static: " + std::to_string(n_env) + " environments need " +
                    std::to_string(graph_bytes) + " bytes of graph plus " + std::to_string(per_env) +
                    " bytes per environment; the static scratch holds " + std::to_string(cap) + " bytes (at most " +
                    std::to_string(max_env) + " environments for this graph)");
  void* base = nullptr;
  cudaError_t e = static_scratch_ptr(&base);
  if (e != cudaSuccess) return cuda_fail(e, "static scratch lookup");
  cudaStream_t st = (cudaStream_t)stream;
  int32_t* left = static_cast<int32_t*>(base);
  int32_t* right = left + N;
  int32_t* nbasis = right + N;
  double* AA = reinterpret_cast<double*>(static_cast<unsigned char*>(base) + graph_bytes);
  double* abar = dA ? AA + (size_t)N * n_env : nullptr;
  if ((e = cudaMemcpyAsync(left, dag->g.left.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(right, dag->g.right.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice, st)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(nbasis, dag->g.node_basis.data(), N * sizeof(int32_t), cudaMemcpyHostToDevice, st)) !=
          cudaSuccess)
    return cuda_fail(e, "graph copy into the static scratch");
  e = launch_plain_f64(A, c, phi_bar, n_env, n_out, dag->K, N, left, right, nbasis, phi, dA, AA, abar, st);
  if (e != cudaSuccess) return cuda_fail(e, "plain kernel launch");
  return ACE_OK;
}

static ace_status check_pool_args(const float* pos, const int64_t* offsets, int64_t n_env, int64_t n_pairs, float rc,
                                  int32_t nmin, int32_t nmax, int32_t lmax, const float* mu, int32_t kmax) {
  if (n_env < 0 || n_pairs < 0) return fail(ACE_ERR_INVALID_ARG, "sizes must be >= 0");
  if (!offsets && n_env > 0) return fail(ACE_ERR_INVALID_ARG, "offsets is NULL");
  if (!pos && n_pairs > 0) return fail(ACE_ERR_INVALID_ARG, "pos is NULL");
  if (!(rc > 0.f)) return fail(ACE_ERR_INVALID_ARG, "rc must be > 0");
  if (nmin < 0 || nmax < nmin) return fail(ACE_ERR_INVALID_ARG, "need 0 <= nmin <= nmax");
  if (kmax < 0) return fail(ACE_ERR_INVALID_ARG, "kmax must be >= 0");
  if (kmax > 3) return fail(ACE_ERR_UNSUPPORTED, "feature degree kmax > 3 is not compiled");
  if (kmax > 0 && !mu && n_pairs > 0) return fail(ACE_ERR_INVALID_ARG, "mu is NULL while kmax > 0");
  if ((nmax - nmin + 1) * (kmax + 1) > 16)
    return fail(ACE_ERR_UNSUPPORTED, "at most 16 radial x feature functions per neighbour");
  if (lmax < 0) return fail(ACE_ERR_INVALID_ARG, "lmax must be >= 0");
  if (lmax > 8) return fail(ACE_ERR_UNSUPPORTED, "lmax > 8 is not compiled");
  return ACE_OK;
}

ace_status ace_pool_A_feat(const float* pos, const float* mu, const int64_t* offsets, int64_t n_env, int64_t n_pairs,
                           float rc, int32_t nmin, int32_t nmax, int32_t lmax, int32_t kmax, float* A, void* stream) {
  NvtxRange nvtx_range("ace_pool_A_feat");
  ace_status s = check_pool_args(pos, offsets, n_env, n_pairs, rc, nmin, nmax, lmax, mu, kmax);
  if (s != ACE_OK) return s;
  if (n_env == 0) return ACE_OK;
  if (!A) return fail(ACE_ERR_INVALID_ARG, "A is NULL");
  cudaError_t e = launch_pool(pos, kmax > 0 ? mu : nullptr, offsets, n_env, rc, nmin, nmax, lmax, kmax, A,
                              (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pooling kernel launch");
  return ACE_OK;
}

ace_status ace_pool_A_feat_grad(const float* pos, const float* mu, const int64_t* offsets, int64_t n_env,
                                int64_t n_pairs, float rc, int32_t nmin, int32_t nmax, int32_t lmax, int32_t kmax,
                                const float* dA, float alpha, float* dpos, void* stream) {
  NvtxRange nvtx_range("ace_pool_A_feat_grad");
  ace_status s = check_pool_args(pos, offsets, n_env, n_pairs, rc, nmin, nmax, lmax, mu, kmax);
  if (s != ACE_OK) return s;
  if (n_env == 0) return ACE_OK;
  if (!dA || (!dpos && n_pairs > 0)) return fail(ACE_ERR_INVALID_ARG, "dA or dpos is NULL");
  cudaError_t e = launch_pool_grad(pos, kmax > 0 ? mu : nullptr, offsets, n_env, rc, nmin, nmax, lmax, kmax, dA,
                                   alpha, dpos, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "pooling adjoint launch");
  return ACE_OK;
}

ace_status ace_pool_A(const float* pos, const int64_t* offsets, int64_t n_env, int64_t n_pairs, float rc,
                      int32_t nmin, int32_t nmax, int32_t lmax, float* A, void* stream) {
  NvtxRange nvtx_range("ace_pool_A");
  return ace_pool_A_feat(pos, nullptr, offsets, n_env, n_pairs, rc, nmin, nmax, lmax, 0, A, stream);
}

ace_status ace_pool_A_grad(const float* pos, const int64_t* offsets, int64_t n_env, int64_t n_pairs, float rc,
                           int32_t nmin, int32_t nmax, int32_t lmax, const float* dA, float alpha, float* dpos,
                           void* stream) {
  NvtxRange nvtx_range("ace_pool_A_grad");
  return ace_pool_A_feat_grad(pos, nullptr, offsets, n_env, n_pairs, rc, nmin, nmax, lmax, 0, dA, alpha, dpos,
                              stream);
}

ace_status ace_energy_forces_host(ace_dag* dag, const float* pos, const float* mu, const int64_t* offsets,
                                  int64_t n_env, int64_t n_pairs, const void* c, int32_t readout, float rc,
                                  int32_t nmin, int32_t nmax, int32_t lmax, int32_t kmax, float* phi, float* forces,
                                  int64_t chunk_env, void* stream) {
  NvtxRange nvtx_range("ace_energy_forces_host");
  ace_status s = check_pool_args(pos, offsets, n_env, n_pairs, rc, nmin, nmax, lmax, mu, kmax);
  if (s != ACE_OK) return s;
  if ((s = check_eval_args(dag, nullptr, 0, 1, ACE_F32, readout)) != ACE_OK) return s;
  if (chunk_env < 0) return fail(ACE_ERR_INVALID_ARG, "chunk_env must be >= 0");
  if (n_env > 0 && (!phi || (!forces && n_pairs > 0))) return fail(ACE_ERR_INVALID_ARG, "phi or forces is NULL");
  if (c && !aligned16(c)) return fail(ACE_ERR_INVALID_ARG, "c must be 16-byte aligned");
  const int64_t K = (int64_t)(nmax - nmin + 1) * (kmax + 1) * (lmax + 1) * (lmax + 1);
  if (K != dag->K) return fail(ACE_ERR_INVALID_ARG, "the graph's K does not match the pooling's one-particle set");
  if (n_env > 0) {  // the host holds the offsets: check them before any copy
    if (offsets[0] != 0 || offsets[n_env] != n_pairs)
      return fail(ACE_ERR_INVALID_ARG, "offsets must start at 0 and end at n_pairs");
    for (int64_t e = 0; e < n_env; ++e)
      if (offsets[e + 1] < offsets[e]) return fail(ACE_ERR_INVALID_ARG, "offsets must not decrease");
  }
  cudaStream_t st = (cudaStream_t)stream;
  if ((s = ensure_uploaded(dag, st)) != ACE_OK) return s;
  if ((s = bind(dag, dag->sym, c, 1, ACE_F32, st)) != ACE_OK) return s;
  if (n_env == 0) return ACE_OK;
  const std::vector<int64_t> plan = chunk_plan(dag, dag->sym, ACE_F32, 1, readout, true, n_env, (size_t)K * 4, chunk_env);
  const int64_t chunk = *std::max_element(plan.begin(), plan.end());
  // one allocation: positions, mu, offsets, forces, phi of the batch, then A and dA of two chunks
  const size_t b_pos = dev::align16((size_t)n_pairs * 12), b_mu = kmax > 0 ? dev::align16((size_t)n_pairs * 4) : 0;
  const size_t b_off = dev::align16((size_t)(n_env + 1) * 8), b_phi = dev::align16((size_t)n_env * 4);
  const bool fused = forces_fused_bytes(dag, nmin, nmax, lmax, kmax, dag->sym.rm_bound, dag->smem_optin) > 0;
  const size_t b_a = fused ? 0 : dev::align16((size_t)chunk * K * 4);
  const size_t need = 2 * b_pos + b_mu + b_off + b_phi + 4 * b_a;
  if ((s = ensure_host_pipeline(dag, 0)) != ACE_OK) return s;
  cudaError_t e;
  if (need > dag->fbuf_bytes) {
    if (dag->fbuf) cudaFree(dag->fbuf);
    dag->fbuf = nullptr;
    dag->fbuf_bytes = 0;
    if ((e = cudaMalloc(&dag->fbuf, need)) != cudaSuccess) return cuda_fail(e, "cudaMalloc (forces pipeline)");
    dag->fbuf_bytes = need;
  }
  unsigned char* base = static_cast<unsigned char*>(dag->fbuf);
  float* pos_d = reinterpret_cast<float*>(base);
  float* F_d = reinterpret_cast<float*>(base + b_pos);
  float* mu_d = kmax > 0 ? reinterpret_cast<float*>(base + 2 * b_pos) : nullptr;
  int64_t* off_d = reinterpret_cast<int64_t*>(base + 2 * b_pos + b_mu);
  float* phi_d = reinterpret_cast<float*>(base + 2 * b_pos + b_mu + b_off);
  unsigned char* slots = base + 2 * b_pos + b_mu + b_off + b_phi;
  cudaStream_t hin = dag->hstream[0], hk = dag->hstream[1], hout = dag->hstream[2];
  e = cudaEventRecord(dag->hev_fork, st);
  for (cudaStream_t h : dag->hstream)
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h, dag->hev_fork, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(off_d, offsets, (size_t)(n_env + 1) * 8, cudaMemcpyHostToDevice, hin);
  s = ACE_OK;
  int64_t e0 = 0;
  for (size_t k = 0; k < plan.size() && e == cudaSuccess && s == ACE_OK; e0 += plan[k], ++k) {
    const int64_t n = plan[k];
    const int64_t p0 = offsets[e0], p1 = offsets[e0 + n];
    const int b = (int)(k & 1);
    float* A_d = reinterpret_cast<float*>(slots + (size_t)b * 2 * b_a);
    float* dA_d = reinterpret_cast<float*>(slots + (size_t)b * 2 * b_a + b_a);
    // copy in this chunk's neighbours (the slots of A and dA are only used on the kernel stream)
    if (p1 > p0) e = cudaMemcpyAsync(pos_d + 3 * p0, pos + 3 * p0, (size_t)(p1 - p0) * 12, cudaMemcpyHostToDevice, hin);
    if (e == cudaSuccess && kmax > 0 && p1 > p0)
      e = cudaMemcpyAsync(mu_d + p0, mu + p0, (size_t)(p1 - p0) * 4, cudaMemcpyHostToDevice, hin);
    if (e == cudaSuccess) e = cudaEventRecord(dag->hev_in[b], hin);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hk, dag->hev_in[b], 0);
    // the forces pipeline of the chunk (offsets index the whole batch's positions)
    if (e != cudaSuccess) break;
    s = forces_pipeline(dag, pos_d, mu_d, off_d + e0, n, rc, nmin, nmax, lmax, kmax, readout, phi_d + e0, F_d,
                        fused ? nullptr : A_d, fused ? nullptr : dA_d, hk);
    if (s != ACE_OK) break;
    e = cudaEventRecord(dag->hev_done[b], hk);
    // copy out
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hout, dag->hev_done[b], 0);
    if (e == cudaSuccess && p1 > p0)
      e = cudaMemcpyAsync(forces + 3 * p0, F_d + 3 * p0, (size_t)(p1 - p0) * 12, cudaMemcpyDeviceToHost, hout);
    if (e == cudaSuccess) e = cudaMemcpyAsync(phi + e0, phi_d + e0, (size_t)n * 4, cudaMemcpyDeviceToHost, hout);
  }
  for (int i = 0; i < 3; ++i) {
    if (cudaEventRecord(dag->hev_join[i], dag->hstream[i]) == cudaSuccess) cudaStreamWaitEvent(st, dag->hev_join[i], 0);
  }
  if (s != ACE_OK) return s;
  if (e != cudaSuccess) return cuda_fail(e, "host-buffer forces pipeline");
  return ACE_OK;
}

ace_status ace_energy_forces(ace_dag* dag, const float* pos, const float* mu, const int64_t* offsets, int64_t n_env,
                             int64_t n_pairs, const void* c, int32_t readout, float rc, int32_t nmin, int32_t nmax,
                             int32_t lmax, int32_t kmax, float* phi, float* forces, void* stream) {
  NvtxRange nvtx_range("ace_energy_forces");
  ace_status s = check_pool_args(pos, offsets, n_env, n_pairs, rc, nmin, nmax, lmax, mu, kmax);
  if (s != ACE_OK) return s;
  if ((s = check_eval_args(dag, nullptr, 0, 1, ACE_F32, readout)) != ACE_OK) return s;
  if (n_env > 0 && (!phi || (!forces && n_pairs > 0))) return fail(ACE_ERR_INVALID_ARG, "phi or forces is NULL");
  if (c && !aligned16(c)) return fail(ACE_ERR_INVALID_ARG, "c must be 16-byte aligned");
  const int64_t K = (int64_t)(nmax - nmin + 1) * (kmax + 1) * (lmax + 1) * (lmax + 1);
  if (K != dag->K) return fail(ACE_ERR_INVALID_ARG, "the graph's K does not match the pooling's one-particle set");
  cudaStream_t st = (cudaStream_t)stream;
  if ((s = ensure_uploaded(dag, st)) != ACE_OK) return s;
  if ((s = bind(dag, dag->sym, c, 1, ACE_F32, st)) != ACE_OK) return s;
  if (n_env == 0) return ACE_OK;
  float *A_d = nullptr, *dA_d = nullptr;
  if (forces_fused_bytes(dag, nmin, nmax, lmax, kmax, dag->sym.rm_bound, dag->smem_optin) == 0) {
    // the three-kernel form keeps A and dA of the batch in the handle
    const size_t half = dev::align16((size_t)n_env * K * sizeof(float));
    if (2 * half > dag->fwork_bytes) {
      if (dag->fwork) cudaFree(dag->fwork);
      dag->fwork = nullptr;
      dag->fwork_bytes = 0;
      cudaError_t e = cudaMalloc(&dag->fwork, 2 * half);
      if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (forces work buffer)");
      dag->fwork_bytes = 2 * half;
    }
    A_d = static_cast<float*>(dag->fwork);
    dA_d = A_d + half / sizeof(float);
  }
  return forces_pipeline(dag, pos, kmax > 0 ? mu : nullptr, offsets, n_env, rc, nmin, nmax, lmax, kmax, readout, phi,
                         forces, A_d, dA_d, st);
}

ace_status ace_energy_forces_plan(ace_dag* dag, int32_t nmin, int32_t nmax, int32_t lmax, int32_t kmax,
                                  int32_t* fused, int64_t* smem_bytes) {
  if (!dag) return fail(ACE_ERR_INVALID_ARG, "dag is NULL");
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return fail(ACE_ERR_NO_DEVICE, std::string("no CUDA device: ") + cudaGetErrorString(e));
  const size_t b = forces_fused_bytes(dag, nmin, nmax, lmax, kmax, true, optin);
  if (fused) *fused = b > 0 ? 1 : 0;
  if (smem_bytes) *smem_bytes = (int64_t)b;
  return ACE_OK;
}

ace_status ace_stream_status(ace_dag* dag, void* stream) {
  if (!dag) return fail(ACE_ERR_INVALID_ARG, "dag is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  if (dag->device < 0) return ACE_OK;
  uint32_t w = 0;
  if ((e = cudaMemcpy(&w, dag->status, sizeof(w), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return cuda_fail(e, "status read");
  if ((e = cudaMemset(dag->status, 0, sizeof(uint32_t))) != cudaSuccess) return cuda_fail(e, "status clear");
  if (w & dev::kStatusBounds) return fail(ACE_ERR_BOUNDS, "a checked kernel saw an out-of-range index");
  if (w & dev::kStatusTimeout) return fail(ACE_ERR_TIMEOUT, "a bounded device wait gave up");
  return ACE_OK;
}

ace_status ace_device_info(int32_t* sm_count, int32_t* smem_optin_bytes, int32_t* cc_major, int32_t* cc_minor) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(ACE_ERR_NO_DEVICE, std::string("no CUDA device: ") + cudaGetErrorString(e));
  int v = 0;
  if (sm_count) {
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    *sm_count = v;
  }
  if (smem_optin_bytes) {
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    *smem_optin_bytes = v;
  }
  if (cc_major) {
    cudaDeviceGetAttribute(&v, cudaDevAttrComputeCapabilityMajor, dev);
    *cc_major = v;
  }
  if (cc_minor) {
    cudaDeviceGetAttribute(&v, cudaDevAttrComputeCapabilityMinor, dev);
    *cc_minor = v;
  }
  return ACE_OK;
}

ace_status ace_fma_peak(int64_t iters, double* ms, double* fma_count, void* stream) {
  if (iters < 1 || !ms || !fma_count) return fail(ACE_ERR_INVALID_ARG, "bad argument");
  int32_t sms = 0;
  ace_status s = ace_device_info(&sms, nullptr, nullptr, nullptr);
  if (s != ACE_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  const int threads = 256, blocks = sms * 8;
  float* out = nullptr;
  cudaError_t e = cudaMalloc(&out, (size_t)blocks * sizeof(float));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  launch_fma_probe(iters / 10 + 1, blocks, threads, out, st);  // warm-up
  cudaEventRecord(a, st);
  e = launch_fma_probe(iters, blocks, threads, out, st);
  cudaEventRecord(b, st);
  cudaError_t e2 = cudaEventSynchronize(b);
  float t = 0.f;
  cudaEventElapsedTime(&t, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(out);
  if (e != cudaSuccess) return cuda_fail(e, "probe launch");
  if (e2 != cudaSuccess) return cuda_fail(e2, "probe sync");
  *ms = t;
  *fma_count = (double)iters * 8.0 * threads * blocks;
  return ACE_OK;
}

}  // extern "C"
