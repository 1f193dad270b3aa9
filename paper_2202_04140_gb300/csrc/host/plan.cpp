// Evaluation plan: the recursion of Eq. 4 laid out for the fused GPU kernels.
//
// phi = sum_k c_k AA_k splits into
//   * a linear part sum_s c_s AA_s over the stored values (leaves and operand
//     nodes that are basis functions), and
//   * the sinks: a node i = [p, q] of order >= 2 that no other node consumes is
//     never stored; it contributes c_i AA_p AA_q.
// Writing S for the symmetric matrix over slots with S_pq = S_qp = c_i for
// every sink i = [p, q] (2 c_i on the diagonal when p = q), and u = S AA:
//   phi     = sum_s AA_s (c_s + u_s / 2)
//   dphi/dAA_s (through the sinks and the linear part) = c_s + u_s,
// after which the adjoint runs back through the operand nodes
// (g_l += g_i AA_r, g_r += g_i AA_l).  Forward-only evaluation uses the
// one-sided form (each sink stored once, in the row of its factor with more
// sinks): phi = sum_s AA_s (c_s + t_s), t = C AA.
//
// Rows are cut into tasks of at most `task_len` entries; tasks are sorted by
// length and grouped 32 at a time (one per lane), their entries interleaved so
// that a warp reads one contiguous 128-byte line of indices per step.
#include <algorithm>
#include <numeric>

#include "ace_internal.hpp"

namespace ace {

namespace {

struct Entry {
  int32_t col, basis;
  uint8_t w2;
};

void build_tasks(const std::vector<std::vector<Entry>>& rows, const std::vector<int32_t>& slot_basis,
                 int32_t n_g, bool sym, const std::vector<int32_t>& slot_l, const std::vector<int32_t>& slot_r,
                 int task_len, TaskSet& ts) {
  struct Proto {
    Task t;
    int32_t begin, len;
  };
  std::vector<Proto> protos;
  const int32_t n_slots = (int32_t)rows.size();
  for (int32_t s = 0; s < n_slots; ++s) {
    const auto& r = rows[s];
    const bool lin = slot_basis[s] >= 0;
    if (r.empty() && !lin) continue;
    const bool top = sym && s >= n_g;
    int32_t n = (int32_t)r.size();
    int32_t begin = 0;
    bool first = true;
    do {
      int32_t len = std::min<int32_t>(task_len, n - begin);
      Proto p;
      p.t.row = s;
      p.t.flags = (first ? 1 : 0) | (top ? 2 : 0);
      p.t.pl = top ? slot_l[s] : -1;
      p.t.pr = top ? slot_r[s] : -1;
      p.begin = begin;
      p.len = len;
      protos.push_back(p);
      begin += len;
      first = false;
    } while (begin < n);
  }
  std::stable_sort(protos.begin(), protos.end(), [](const Proto& a, const Proto& b) { return a.len > b.len; });
  const int32_t n_tasks = (int32_t)protos.size();
  const int32_t n_slices = (n_tasks + 31) / 32;
  ts = TaskSet();
  ts.tasks.resize((size_t)n_slices * 32, Task{-1, 0, -1, -1});
  ts.slice_off.assign(n_slices + 1, 0);
  ts.slice_steps.assign(n_slices, 0);
  int64_t off = 0;
  for (int32_t s = 0; s < n_slices; ++s) {
    int32_t steps = 0;
    for (int j = 0; j < 32; ++j) {
      int32_t ti = s * 32 + j;
      if (ti < n_tasks) steps = std::max(steps, protos[ti].len);
    }
    ts.slice_off[s] = (int32_t)off;
    ts.slice_steps[s] = steps;
    off += (int64_t)steps * 32;
  }
  ts.slice_off[n_slices] = (int32_t)off;
  ts.col.assign(off, 0);
  ts.ebasis.assign(off, -1);
  ts.ew2.assign(off, 0);
  ts.n_entries = 0;
  for (int32_t s = 0; s < n_slices; ++s) {
    for (int j = 0; j < 32; ++j) {
      int32_t ti = s * 32 + j;
      if (ti >= n_tasks) continue;
      const Proto& p = protos[ti];
      ts.tasks[ti] = p.t;
      const auto& r = rows[p.t.row];
      for (int32_t k = 0; k < p.len; ++k) {
        const Entry& e = r[p.begin + k];
        int64_t idx = (int64_t)ts.slice_off[s] + (int64_t)k * 32 + j;
        ts.col[idx] = e.col;
        ts.ebasis[idx] = e.basis;
        ts.ew2[idx] = e.w2;
      }
      ts.n_entries += p.len;
    }
  }
}

}  // namespace

ace_status build_plan(const Spec& spec, const Graph& g, int task_len, Plan& plan) {
  if (task_len < 1) return fail(ACE_ERR_INVALID_ARG, "task_len must be >= 1");
  const int32_t K = g.K;
  const int64_t N = g.n_nodes();
  std::vector<int32_t> cons(N, 0), opcons(N, 0);
  for (int64_t i = K; i < N; ++i) {
    cons[g.left[i]]++;
    cons[g.right[i]]++;
  }
  std::vector<uint8_t> operand(N, 0), inner(N, 0);
  for (int64_t i = K; i < N; ++i) operand[i] = cons[i] > 0;
  for (int64_t i = K; i < N; ++i)
    if (operand[i]) {
      opcons[g.left[i]]++;
      opcons[g.right[i]]++;
    }
  for (int64_t i = K; i < N; ++i) inner[i] = operand[i] && opcons[i] > 0;

  plan = Plan();
  plan.K = K;
  plan.node_slot.assign(N, -1);
  for (int32_t k = 0; k < K; ++k) {
    plan.node_slot[k] = k;
    plan.slot_node.push_back(k);
  }
  auto by_order = [&](std::vector<int32_t>& ids) {
    std::stable_sort(ids.begin(), ids.end(), [&](int32_t a, int32_t b) { return g.order[a] < g.order[b]; });
  };
  std::vector<int32_t> inner_ids, top_ids;
  for (int64_t i = K; i < N; ++i) {
    if (inner[i]) inner_ids.push_back((int32_t)i);
    else if (operand[i]) top_ids.push_back((int32_t)i);
  }
  by_order(inner_ids);
  by_order(top_ids);
  for (int32_t id : inner_ids) {
    plan.node_slot[id] = (int32_t)plan.slot_node.size();
    plan.slot_node.push_back(id);
  }
  plan.n_g = (int32_t)plan.slot_node.size();
  for (int32_t id : top_ids) {
    plan.node_slot[id] = (int32_t)plan.slot_node.size();
    plan.slot_node.push_back(id);
  }
  plan.n_slots = (int32_t)plan.slot_node.size();
  const int32_t n_slots = plan.n_slots;

  plan.slot_basis.assign(n_slots, -1);
  std::vector<int32_t> slot_l(n_slots, -1), slot_r(n_slots, -1);
  for (int32_t s = 0; s < n_slots; ++s) {
    int32_t id = plan.slot_node[s];
    plan.slot_basis[s] = g.node_basis[id];
    if (id >= K) {
      slot_l[s] = plan.node_slot[g.left[id]];
      slot_r[s] = plan.node_slot[g.right[id]];
      if (slot_l[s] < 0 || slot_r[s] < 0) return fail(ACE_ERR_INVALID_ARG, "internal: operand factor not stored");
    }
  }

  // forward: all operand nodes by increasing order; reverse: inner operand nodes by decreasing order
  const int nu_max = g.nu_max;
  auto fill_levels = [&](const std::vector<int32_t>& slots_in_order, LevelList& L, bool descending) {
    std::vector<int32_t> ord = slots_in_order;
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) {
      int32_t oa = g.order[plan.slot_node[a]], ob = g.order[plan.slot_node[b]];
      return descending ? oa > ob : oa < ob;
    });
    L = LevelList();
    int32_t cur = -1;
    for (int32_t s : ord) {
      int32_t o = g.order[plan.slot_node[s]];
      if (o != cur) {
        L.off.push_back((int32_t)L.slot.size());
        cur = o;
      }
      L.slot.push_back(s);
      L.l.push_back(slot_l[s]);
      L.r.push_back(slot_r[s]);
    }
    L.off.push_back((int32_t)L.slot.size());
  };
  std::vector<int32_t> all_ops, inner_slots;
  for (int32_t s = K; s < n_slots; ++s) all_ops.push_back(s);
  for (int32_t s = K; s < plan.n_g; ++s) inner_slots.push_back(s);
  fill_levels(all_ops, plan.fwd, false);
  fill_levels(inner_slots, plan.rev, true);
  if ((int)plan.fwd.off.size() - 1 > nu_max || (int)plan.rev.off.size() - 1 > nu_max)
    return fail(ACE_ERR_INVALID_ARG, "internal: too many levels");

  // sinks -> sparse rows
  std::vector<std::vector<Entry>> sym_rows(n_slots), one_rows(n_slots);
  std::vector<int32_t> sink_deg(n_slots, 0);
  struct Sink {
    int32_t p, q, b;
  };
  std::vector<Sink> sinks;
  for (int64_t i = K; i < N; ++i) {
    if (operand[i]) continue;
    int32_t b = g.node_basis[i];
    if (b < 0) continue;  // auxiliary node nobody uses: contributes nothing
    int32_t p = plan.node_slot[g.left[i]], q = plan.node_slot[g.right[i]];
    if (p < 0 || q < 0) return fail(ACE_ERR_INVALID_ARG, "internal: sink factor not stored");
    sinks.push_back({p, q, b});
    sink_deg[p]++;
    if (q != p) sink_deg[q]++;
  }
  plan.n_sinks = (int64_t)sinks.size();
  for (const Sink& s : sinks) {
    if (s.p == s.q) {
      sym_rows[s.p].push_back({s.p, s.b, 1});
    } else {
      sym_rows[s.p].push_back({s.q, s.b, 0});
      sym_rows[s.q].push_back({s.p, s.b, 0});
    }
    int32_t row = s.p, other = s.q;
    if (sink_deg[s.q] > sink_deg[s.p] || (sink_deg[s.q] == sink_deg[s.p] && s.q < s.p)) {
      row = s.q;
      other = s.p;
    }
    one_rows[row].push_back({other, s.b, 0});
  }
  build_tasks(sym_rows, plan.slot_basis, plan.n_g, true, slot_l, slot_r, task_len, plan.sym);
  build_tasks(one_rows, plan.slot_basis, plan.n_g, false, slot_l, slot_r, task_len, plan.one);
  return ACE_OK;
}

}  // namespace ace
