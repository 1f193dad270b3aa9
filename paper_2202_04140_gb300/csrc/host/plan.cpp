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
#include <array>
#include <map>
#include <numeric>

#include "ace_internal.hpp"

namespace ace {

namespace {

struct Entry {
  int32_t col, basis;
  uint8_t w2;
};

// Slices of 32 tasks (one per lane).  Tasks are taken longest first.  In the
// adjoint form every task adds into one "A" target (its row, or the first
// factor of a top operand), combined across lanes by a segmented warp
// reduction (lanes are ordered by A target), and top-operand tasks also add
// into a "B" target (their second factor) with one shared-memory atomic per
// lane; a task joins the slice being filled only if no other lane has its B
// target (the banks of the targets are chosen afterwards, by the adjoint-row
// permutation of choose_g_perm).  The search looks at most `kWindow` tasks ahead;
// a slice that cannot be completed without a repeat takes the next tasks.
constexpr int kWindow = 512;

// Bank schedule of the entries: the tile-per-lane kernel gathers E values per
// lane and entry; with E >= 4 (16 bytes or more per lane) a warp's load is
// served a quarter-warp at a time, 8 lanes over 8 groups of 16-byte banks, so
// the schedule keeps the columns of every 8 consecutive lanes in distinct
// groups (column mod 8) or equal (broadcast).  Tiles of 4 environments are the
// target of the plan (see Plan::n_stored).
constexpr int kPhaseLanes = 8;
constexpr int kBankGroups = 8;

void form_slices(const std::vector<Task>& tasks, const std::vector<int32_t>& order, const std::vector<int32_t>& len,
                 bool atomics, std::vector<std::vector<int32_t>>& slices) {
  std::vector<uint8_t> taken(order.size(), 0);
  size_t head = 0;
  while (true) {
    while (head < order.size() && taken[head]) ++head;
    if (head >= order.size()) break;
    std::vector<int32_t> sl;
    // candidates stay within a length band of the slice's longest task (padding stays small)
    const int32_t band = len[order[head]] - std::max<int32_t>(1, len[order[head]] / 16);
    std::vector<size_t> cand;
    for (size_t i = head; i < order.size() && cand.size() < (size_t)kWindow; ++i) {
      if (taken[i]) continue;
      if (len[order[i]] < band) break;
      cand.push_back(i);
    }
    auto a_key = [&](int32_t ti) { return (tasks[ti].flags & 2) ? tasks[ti].pl : tasks[ti].row; };
    auto take = [&](size_t i) {
      const Task& t = tasks[order[i]];
      if (atomics && (t.flags & 2))
        for (int32_t q : sl)
          if ((tasks[q].flags & 2) && tasks[q].pr == t.pr) return false;
      taken[i] = 1;
      sl.push_back(order[i]);
      return true;
    };
    // Fill in candidate order, but after each task first take the other candidates with the
    // same first atomic target, so that equal targets form long runs (one atomic per run).
    for (size_t ci = 0; ci < cand.size() && sl.size() < 32; ++ci) {
      if (taken[cand[ci]] || !take(cand[ci])) continue;
      if (!atomics) continue;
      const int32_t key = a_key(order[cand[ci]]);
      for (size_t cj = ci + 1; cj < cand.size() && sl.size() < 32; ++cj)
        if (!taken[cand[cj]] && a_key(order[cand[cj]]) == key) take(cand[cj]);
    }
    for (size_t i = head; i < order.size() && sl.size() < 32; ++i) {
      if (taken[i]) continue;
      taken[i] = 1;
      sl.push_back(order[i]);
    }
    if (atomics) {  // lanes ordered by A target so that equal targets are contiguous
      std::stable_sort(sl.begin(), sl.end(), [&](int32_t a, int32_t b) {
        const int32_t ka = (tasks[a].flags & 2) ? tasks[a].pl : tasks[a].row;
        const int32_t kb = (tasks[b].flags & 2) ? tasks[b].pl : tasks[b].row;
        return ka < kb;
      });
    }
    slices.push_back(std::move(sl));
  }
}

// Interleave the entries of one slice step by step.  The lanes of a phase
// (`phase_lanes` consecutive lanes, served by one vector shared-memory load of E
// values per lane) gather without bank conflict when, for every bank group
// (column mod `bank_mod`), all of them read the same column: different columns
// of one group cost one extra wavefront each, the same column is a broadcast.
// So at every step each group is given at most one column: lanes are visited
// most-constrained first (entries left against steps left); a lane reads a
// column already given to its group if it has one, else opens a free group
// with its column that most lanes of the phase still need (so that they can
// share it), else, if it has no slack, takes a conflicting entry, and otherwise
// waits a step.  A waiting or finished lane reads a zero coefficient at a
// column already given out (a broadcast) or in a group nobody uses.
// key(entry) is the slot the entry gathers (the scheduled column); emit(lane j,
// step k, entry or nullptr, padding column) writes the schedule.
template <typename Key, typename Emit>
void interleave(const std::vector<const std::vector<Entry>*>& lane_entries, int32_t steps, int phase_lanes,
                int bank_mod, int32_t n_slots, Key key, Emit emit) {
  const int nl = (int)lane_entries.size();
  // remaining entries of every lane as (column, entry index), sorted by column
  std::vector<std::vector<std::pair<int32_t, int32_t>>> rem(32);
  for (int j = 0; j < nl; ++j) {
    const auto& v = *lane_entries[j];
    for (int32_t q = 0; q < (int32_t)v.size(); ++q) rem[j].push_back({key(v[q]), q});
    std::sort(rem[j].begin(), rem[j].end());
  }
  std::vector<int32_t> chosen(bank_mod);
  std::vector<int> order;
  std::vector<std::pair<int32_t, int>> pop;  // (column, lanes of the phase still needing it)
  for (int32_t k = 0; k < steps; ++k) {
    const int32_t steps_left = steps - k;
    for (int p0 = 0; p0 < 32; p0 += phase_lanes) {
      std::fill(chosen.begin(), chosen.end(), -1);
      pop.clear();
      order.clear();
      for (int j = p0; j < p0 + phase_lanes && j < nl; ++j) {
        if (rem[j].empty()) continue;
        order.push_back(j);
        for (size_t t = 0; t < rem[j].size(); ++t)
          if (t == 0 || rem[j][t].first != rem[j][t - 1].first) pop.push_back({rem[j][t].first, 1});
      }
      std::sort(pop.begin(), pop.end());
      {  // merge equal columns
        size_t w = 0;
        for (size_t t = 0; t < pop.size(); ++t) {
          if (w > 0 && pop[w - 1].first == pop[t].first) pop[w - 1].second += pop[t].second;
          else pop[w++] = pop[t];
        }
        pop.resize(w);
      }
      auto popularity = [&](int32_t c) {
        auto it = std::lower_bound(pop.begin(), pop.end(), std::make_pair(c, 0));
        return (it != pop.end() && it->first == c) ? it->second : 0;
      };
      std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const int32_t sx = (int32_t)rem[x].size() - steps_left, sy = (int32_t)rem[y].size() - steps_left;
        if (sx != sy) return sx > sy;  // least slack first
        return x < y;
      });
      std::vector<int32_t> lane_col(32, -1);
      for (int j : order) {
        const int32_t left = (int32_t)rem[j].size();
        int pick = -1;
        for (size_t t = 0; t < rem[j].size() && pick < 0; ++t)
          if (chosen[rem[j][t].first % bank_mod] == rem[j][t].first) pick = (int)t;
        if (pick < 0) {
          int best_pop = -1;
          for (size_t t = 0; t < rem[j].size(); ++t) {
            const int32_t c = rem[j][t].first;
            if (chosen[c % bank_mod] >= 0) continue;
            const int pc = popularity(c);
            if (pc > best_pop) {
              best_pop = pc;
              pick = (int)t;
            }
          }
          if (pick >= 0) chosen[rem[j][pick].first % bank_mod] = rem[j][pick].first;
        }
        if (pick < 0 && left >= steps_left) pick = 0;  // no slack: a conflicting entry
        if (pick < 0) continue;                         // wait a step
        lane_col[j] = pick;
      }
      // a column already given out (broadcast), else a group nobody uses, for lanes without an entry
      int32_t pad = -1;
      for (int b = 0; b < bank_mod && pad < 0; ++b)
        if (chosen[b] >= 0) pad = chosen[b];
      if (pad < 0) pad = 0;
      for (int j = p0; j < p0 + phase_lanes; ++j) {
        if (j < nl && lane_col[j] >= 0) {
          const int t = lane_col[j];
          const int32_t q = rem[j][t].second;
          rem[j].erase(rem[j].begin() + t);
          emit(j, k, &(*lane_entries[j])[q], 0);
        } else {
          emit(j, k, nullptr, pad < n_slots ? pad : 0);
        }
      }
    }
  }
}

// Task protos of a set of rows: each row with entries (or, if with_lin, a row
// coefficient) is cut into equal pieces of at most task_len entries.
struct Proto {
  int32_t begin, len;
};

void make_tasks(const std::vector<std::vector<Entry>>& rows, const std::vector<int32_t>& slot_basis, int32_t n_g,
                bool with_lin, const std::vector<int32_t>& slot_l, const std::vector<int32_t>& slot_r, int task_len,
                std::vector<Task>& tasks, std::vector<Proto>& protos) {
  const int32_t n_slots = (int32_t)rows.size();
  for (int32_t s = 0; s < n_slots; ++s) {
    const auto& r = rows[s];
    const bool lin = with_lin && slot_basis[s] >= 0;
    if (r.empty() && !lin) continue;
    // a top operand's value is the product of its factors (adjoint: pushed to them)
    const bool top = s >= n_g;
    const int32_t n = (int32_t)r.size();
    const int32_t pieces = std::max<int32_t>(1, (n + task_len - 1) / task_len);
    for (int32_t p = 0; p < pieces; ++p) {
      const int32_t b = (int32_t)((int64_t)n * p / pieces), e = (int32_t)((int64_t)n * (p + 1) / pieces);
      Task t;
      t.row = s;
      t.flags = (p == 0 && with_lin ? 1 : 0) | (top ? 2 : 0) | (lin ? 4 : 0);
      t.pl = top ? slot_l[s] : -1;
      t.pr = top ? slot_r[s] : -1;
      tasks.push_back(t);
      protos.push_back({b, e - b});
    }
  }
}

// Slices of the protos, longest first.
void slice_tasks(const std::vector<Task>& tasks, const std::vector<Proto>& protos, bool sym,
                 std::vector<std::vector<int32_t>>& slices, std::vector<int32_t>& steps) {
  std::vector<int32_t> order(tasks.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return protos[a].len > protos[b].len; });
  std::vector<int32_t> lens(protos.size());
  for (size_t i = 0; i < protos.size(); ++i) lens[i] = protos[i].len;
  form_slices(tasks, order, lens, sym, slices);
  steps.assign(slices.size(), 0);
  for (size_t s = 0; s < slices.size(); ++s)
    for (int32_t ti : slices[s]) steps[s] = std::max(steps[s], protos[ti].len);
}

void build_tasks(const std::vector<std::vector<Entry>>& rows, const std::vector<int32_t>& slot_basis, int32_t n_g,
                 int32_t n_stored, bool sym, const std::vector<int32_t>& slot_l, const std::vector<int32_t>& slot_r,
                 int task_len, TaskSet& ts) {
  const int32_t n_slots = (int32_t)rows.size();
  ts = TaskSet();
  for (const auto& r : rows) ts.n_entries += (int64_t)r.size();
  // the tile-per-lane layout, only where that kernel can run (every stored column below 2^16);
  // otherwise no slices: both offset lists hold their final 0
  const bool tile = n_stored <= kTileMaxStored;
  if (!tile) {
    ts.slice_off.assign(1, 0);
    ts.cold_slice_off.assign(1, 0);
  }
  // hot entries (column kept in shared memory) and cold ones
  std::vector<std::vector<Entry>> hot(tile ? n_slots : 0), cold(tile ? n_slots : 0);
  if (tile)
    for (int32_t s = 0; s < n_slots; ++s)
      for (const Entry& e : rows[s]) (e.col < n_stored ? hot : cold)[s].push_back(e);

  // ---- hot tasks: interleaved, bank-scheduled entries
  if (tile) {
    std::vector<Task> tasks;
    std::vector<Proto> protos;
    make_tasks(hot, slot_basis, n_g, true, slot_l, slot_r, task_len, tasks, protos);
    std::vector<std::vector<int32_t>> slices;
    std::vector<int32_t> steps;
    slice_tasks(tasks, protos, sym, slices, steps);
    const int32_t n_slices = (int32_t)slices.size();
    ts.tasks.resize((size_t)n_slices * 32, Task{-1, 0, -1, -1});
    ts.slice_off.assign(n_slices + 1, 0);
    ts.slice_steps = steps;
    int64_t off = 0;
    for (int32_t s = 0; s < n_slices; ++s) {
      ts.slice_off[s] = (int32_t)off;
      off += (int64_t)steps[s] * 32;
    }
    ts.slice_off[n_slices] = (int32_t)off;
    ts.col.assign(off, 0);
    ts.ebasis.assign(off, -1);
    ts.ew2.assign(off, 0);
    std::vector<std::vector<Entry>> lane_store(32);
    for (int32_t s = 0; s < n_slices; ++s) {
      std::vector<const std::vector<Entry>*> lanes;
      for (size_t j = 0; j < slices[s].size(); ++j) {
        const int32_t ti = slices[s][j];
        ts.tasks[(size_t)s * 32 + j] = tasks[ti];
        const auto& r = hot[tasks[ti].row];
        lane_store[j].assign(r.begin() + protos[ti].begin, r.begin() + protos[ti].begin + protos[ti].len);
        lanes.push_back(&lane_store[j]);
      }
      const int64_t base = ts.slice_off[s];
      interleave(
          lanes, ts.slice_steps[s], kPhaseLanes, kBankGroups, n_stored, [](const Entry& e) { return e.col; },
          [&](int j, int32_t k, const Entry* e, int32_t pad) {
            const int64_t idx = base + (int64_t)k * 32 + j;
            ts.col[idx] = e ? e->col : pad;
            ts.ebasis[idx] = e ? e->basis : -1;
            ts.ew2[idx] = e ? e->w2 : 0;
          });
    }
  }

  // ---- cold tasks: the operand's two factors per entry, entries in task order
  if (tile) {
    std::vector<Task> tasks;
    std::vector<Proto> protos;
    make_tasks(cold, slot_basis, n_g, false, slot_l, slot_r, task_len, tasks, protos);
    std::vector<std::vector<int32_t>> slices;
    std::vector<int32_t> steps;
    slice_tasks(tasks, protos, sym, slices, steps);
    const int32_t n_slices = (int32_t)slices.size();
    ts.cold_tasks.resize((size_t)n_slices * 32, Task{-1, 0, -1, -1});
    ts.cold_slice_off.assign(n_slices + 1, 0);
    ts.cold_slice_steps = steps;
    int64_t off = 0;
    for (int32_t s = 0; s < n_slices; ++s) {
      ts.cold_slice_off[s] = (int32_t)off;
      off += (int64_t)steps[s] * 32;
    }
    ts.cold_slice_off[n_slices] = (int32_t)off;
    ts.cold_ca.assign(off, 0);
    ts.cold_cb.assign(off, 0);
    ts.cold_ebasis.assign(off, -1);
    ts.cold_ew2.assign(off, 0);
    // entries scheduled on their first factor (the second factor's banks are left to chance)
    std::vector<std::vector<Entry>> lane_store(32);
    for (int32_t s = 0; s < n_slices; ++s) {
      std::vector<const std::vector<Entry>*> lanes;
      for (size_t j = 0; j < slices[s].size(); ++j) {
        const int32_t ti = slices[s][j];
        ts.cold_tasks[(size_t)s * 32 + j] = tasks[ti];
        const auto& r = cold[tasks[ti].row];
        lane_store[j].assign(r.begin() + protos[ti].begin, r.begin() + protos[ti].begin + protos[ti].len);
        lanes.push_back(&lane_store[j]);
      }
      const int64_t base = ts.cold_slice_off[s];
      interleave(
          lanes, steps[s], kPhaseLanes, kBankGroups, n_g, [&](const Entry& e) { return slot_l[e.col]; },
          [&](int j, int32_t k, const Entry* e, int32_t pad) {
            const int64_t idx = base + (int64_t)k * 32 + j;
            ts.cold_ca[idx] = e ? slot_l[e->col] : pad;
            ts.cold_cb[idx] = e ? slot_r[e->col] : pad;
            ts.cold_ebasis[idx] = e ? e->basis : -1;
            ts.cold_ew2[idx] = e ? e->w2 : 0;
          });
    }
  }

  // ---- row-major copy of all entries (kernels that keep every slot), laid out as one stream per
  //      warp of the one-environment-per-lane kernel
  {
    std::vector<Task> tasks;
    std::vector<Proto> protos;
    make_tasks(rows, slot_basis, n_g, true, slot_l, slot_r, task_len, tasks, protos);
    // Blocks: whole rows of at most kLoeBlockCols entries whose column sets are equal.  Such a
    // row needs no gathers of its own: the block's columns are read once per warp, and each
    // row is a header, its coefficients and the epilogue.
    std::map<std::vector<int32_t>, std::vector<int32_t>> by_cols;
    std::vector<uint8_t> in_block(tasks.size(), 0);
    for (size_t ti = 0; ti < tasks.size(); ++ti) {
      const auto& r = rows[tasks[ti].row];
      const int32_t len = protos[ti].len;
      if (len < 1 || len > kLoeBlockCols || len != (int32_t)r.size()) continue;
      std::vector<int32_t> cols;
      for (const Entry& e : r) cols.push_back(e.col);
      std::sort(cols.begin(), cols.end());
      by_cols[cols].push_back((int32_t)ti);
    }
    struct Unit {
      std::vector<int32_t> tis;  // one task, or the rows of a block
      std::vector<int32_t> cols; // block columns (empty: a task)
      int64_t cost;
    };
    std::vector<Unit> units;
    for (auto& kv : by_cols) {
      if ((int32_t)kv.second.size() < kLoeBlockMinRows) continue;
      for (size_t i0 = 0; i0 < kv.second.size(); i0 += kLoeBlockRows) {
        Unit u;
        u.cols = kv.first;
        for (size_t i = i0; i < std::min(kv.second.size(), i0 + kLoeBlockRows); ++i) {
          u.tis.push_back(kv.second[i]);
          in_block[kv.second[i]] = 1;
        }
        u.cost = 20 + 30 * (int64_t)u.tis.size();  // measured against 40 + 40 rows, 40 + 60 rows: best
        units.push_back(std::move(u));
      }
    }
    for (size_t ti = 0; ti < tasks.size(); ++ti)
      if (!in_block[ti]) units.push_back(Unit{{(int32_t)ti}, {}, 60 + 6 * (int64_t)protos[ti].len});
    // longest processing time first onto the least loaded warp (ties: lowest warp); units of
    // equal cost keep their order, so the layout is deterministic
    std::vector<int32_t> uorder(units.size());
    std::iota(uorder.begin(), uorder.end(), 0);
    std::stable_sort(uorder.begin(), uorder.end(),
                     [&](int32_t x, int32_t y) { return units[x].cost > units[y].cost; });
    std::vector<int64_t> load(kLoeWarps, 0);
    std::vector<std::vector<int32_t>> wunits(kLoeWarps);
    for (int32_t ui : uorder) {
      const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      load[w] += units[ui].cost;
      wunits[w].push_back(ui);
    }
    // rm order: warp by warp, unit by unit; every task's entries padded to an even count (pairs),
    // every block row's to 2 * 4 coefficients (two items)
    ts.rm_off.push_back(0);
    ts.loe_wbeg.assign(kLoeWarps + 1, 0);
    int32_t pos = 0;
    auto push_entries = [&](int32_t ti, const std::vector<int32_t>* cols) {
      const Task& t = tasks[ti];
      const auto& r = rows[t.row];
      Task rt = t;
      if (cols) rt.flags |= kTaskBlockRow;
      ts.rm_tasks.push_back(rt);
      ts.loe_hpos.push_back(pos);
      if (cols) {
        for (int32_t c : *cols) {  // the block's column order
          const Entry* e = nullptr;
          for (const Entry& x : r)
            if (x.col == c) e = &x;
          ts.rm_col.push_back(c);
          ts.rm_ebasis.push_back(e->basis);
          ts.rm_ew2.push_back(e->w2);
        }
        for (size_t k = cols->size(); k < (size_t)kLoeBlockCols; ++k) {
          ts.rm_col.push_back(0);
          ts.rm_ebasis.push_back(-1);
          ts.rm_ew2.push_back(0);
        }
        pos += 1 + kLoeBlockCols / 4;
      } else {
        for (int32_t q = protos[ti].begin; q < protos[ti].begin + protos[ti].len; ++q) {
          ts.rm_col.push_back(r[q].col);
          ts.rm_ebasis.push_back(r[q].basis);
          ts.rm_ew2.push_back(r[q].w2);
        }
        if (protos[ti].len % 2) {
          ts.rm_col.push_back(0);
          ts.rm_ebasis.push_back(-1);
          ts.rm_ew2.push_back(0);
        }
        pos += 1 + (protos[ti].len + 1) / 2;
      }
      ts.rm_off.push_back((int32_t)ts.rm_col.size());
    };
    for (int w = 0; w < kLoeWarps; ++w) {
      ts.loe_wbeg[w] = pos;
      for (int32_t ui : wunits[w]) {
        const Unit& u = units[ui];
        if (u.cols.empty()) {
          push_entries(u.tis[0], nullptr);
          continue;
        }
        // block header {m, rows << 8 | kLoeBlockUnit, 0, 0}, then the columns, kLoeBlockCols / 4 items
        ts.loe_spos.push_back(pos);
        ts.loe_sval.insert(ts.loe_sval.end(),
                           {(int32_t)u.cols.size(), ((int32_t)u.tis.size() << 8) | kLoeBlockUnit, 0, 0});
        ++pos;
        for (int k = 0; k < kLoeBlockCols; k += 4) {
          ts.loe_spos.push_back(pos++);
          for (int c = k; c < k + 4; ++c) ts.loe_sval.push_back(c < (int)u.cols.size() ? u.cols[c] : 0);
        }
        for (int32_t ti : u.tis) push_entries(ti, &u.cols);
      }
    }
    ts.loe_wbeg[kLoeWarps] = pos;
  }
}

}  // namespace

namespace {

// Adjoint rows of the tile-per-lane kernel: its accumulators live in shared memory
// environment-major, row r of environment e at e x gs + r (gs a multiple of 32), so row r is in
// bank r mod 32, and the adjoint updates that one warp issues together are serialised by bank
// conflicts: the distinct first targets of a slice's 32 tasks (one update per run), the second
// factors of its top-operand tasks, the distinct targets of a 32-triple chunk of the pull sweep.
// The permutation slot -> row puts the slots of such groups in different banks where it can:
// slots in decreasing order of the number of groups they belong to, each placed in the bank
// (with rows left) that raises the fewest groups' largest bank load, ties to the bank least used
// by its groups.  Rows of one bank are handed out in slot order.
void choose_g_perm(Plan& plan) {
  const int32_t n_g = plan.n_g;
  plan.g_perm.resize(n_g);
  std::iota(plan.g_perm.begin(), plan.g_perm.end(), 0);
  if (n_g <= 32) return;
  std::vector<std::vector<int32_t>> groups;
  auto add = [&](std::vector<int32_t>& v) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    if (v.size() > 1) groups.push_back(v);
  };
  auto add_slices = [&](const std::vector<Task>& tasks) {
    for (size_t s0 = 0; s0 + 32 <= tasks.size(); s0 += 32) {
      std::vector<int32_t> a, b;
      for (int j = 0; j < 32; ++j) {
        const Task& t = tasks[s0 + j];
        if (t.row < 0) continue;
        if (t.flags & 2) {
          a.push_back(t.pl);
          b.push_back(t.pr);
        } else {
          a.push_back(t.row);
        }
      }
      add(a);
      add(b);
    }
  };
  add_slices(plan.sym.tasks);
  add_slices(plan.sym.cold_tasks);
  const PullList& P = plan.pull;
  for (size_t lv = 0; lv + 1 < P.lvl.size(); ++lv)
    for (int32_t c0 = P.lvl[lv]; c0 < P.lvl[lv + 1]; c0 += 32) {
      std::vector<int32_t> t(P.tgt.begin() + c0, P.tgt.begin() + std::min<int32_t>(c0 + 32, P.lvl[lv + 1]));
      add(t);
    }
  std::vector<std::vector<int32_t>> member(n_g);
  for (size_t gi = 0; gi < groups.size(); ++gi)
    for (int32_t k : groups[gi])
      if (k >= 0 && k < n_g) member[k].push_back((int32_t)gi);
  std::vector<std::array<uint8_t, 32>> cnt(groups.size());
  for (auto& c : cnt) c.fill(0);
  std::vector<uint8_t> mx(groups.size(), 0);
  std::array<int32_t, 32> cap;
  for (int b = 0; b < 32; ++b) cap[b] = (n_g - b + 31) / 32;
  std::vector<int32_t> order(n_g);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return member[a].size() > member[b].size(); });
  std::vector<int32_t> bank(n_g, 0);
  for (int32_t k : order) {
    int best = -1;
    int64_t best_add = 0, best_tie = 0;
    for (int b = 0; b < 32; ++b) {
      if (cap[b] == 0) continue;
      int64_t add_max = 0, tie = 0;
      for (int32_t gi : member[k]) {
        if (cnt[gi][b] >= mx[gi]) ++add_max;
        tie += cnt[gi][b];
      }
      if (best < 0 || add_max < best_add || (add_max == best_add && tie < best_tie)) {
        best = b;
        best_add = add_max;
        best_tie = tie;
      }
    }
    bank[k] = best;
    --cap[best];
    for (int32_t gi : member[k]) {
      ++cnt[gi][best];
      mx[gi] = std::max(mx[gi], cnt[gi][best]);
    }
  }
  std::array<int32_t, 32> next;
  for (int b = 0; b < 32; ++b) next[b] = b;
  for (int32_t k = 0; k < n_g; ++k) {
    plan.g_perm[k] = next[bank[k]];
    next[bank[k]] += 32;
  }
}

}  // namespace

ace_status build_plan(const Spec& spec, const Graph& g, int task_len, StoredLimitFn stored_limit_fn, Plan& plan) {
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
  // Stored slots for the tile-per-lane kernel: when not every top operand fits,
  // keep those that appear in the most sink entries (entries are symmetric:
  // a sink [p, q] is an entry of row p in column q and of row q in column p).
  {
    const int64_t n_all = (int64_t)plan.n_g + (int64_t)top_ids.size();
    const int64_t stored_limit = stored_limit_fn ? stored_limit_fn(K, plan.n_g) : 0;
    int64_t keep = (int64_t)top_ids.size();
    if (stored_limit > 0 && n_all > stored_limit && stored_limit > plan.n_g && n_all <= kTileMaxStored)
      keep = stored_limit - plan.n_g;
    if (keep < (int64_t)top_ids.size()) {
      std::vector<int32_t> deg(N, 0);
      for (int64_t i = K; i < N; ++i) {
        if (operand[i] || g.node_basis[i] < 0) continue;
        deg[g.left[i]]++;
        if (g.right[i] != g.left[i]) deg[g.right[i]]++;
      }
      std::vector<int32_t> by_use = top_ids;
      std::stable_sort(by_use.begin(), by_use.end(), [&](int32_t a, int32_t b) { return deg[a] > deg[b]; });
      std::vector<uint8_t> hot(N, 0);
      for (int64_t t = 0; t < keep; ++t) hot[by_use[t]] = 1;
      std::stable_partition(top_ids.begin(), top_ids.end(), [&](int32_t id) { return hot[id] != 0; });
    }
    plan.n_stored = (int32_t)(plan.n_g + keep);
  }
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
  std::vector<int32_t> all_ops, stored_ops, inner_slots;
  for (int32_t s = K; s < n_slots; ++s) all_ops.push_back(s);
  for (int32_t s = K; s < plan.n_stored; ++s) stored_ops.push_back(s);
  for (int32_t s = K; s < plan.n_g; ++s) inner_slots.push_back(s);
  fill_levels(all_ops, plan.fwd, false);
  fill_levels(stored_ops, plan.fwd_stored, false);
  // Within each stored level, order the nodes so that every 8 consecutive ones (a
  // quarter-warp of the 16-byte loads and stores of 4-environment tiles) read and
  // write distinct bank groups (slot mod 8), or read the same slot (a broadcast).
  {
    LevelList& F = plan.fwd_stored;
    constexpr int kGroup = 8, kLook = 256;
    for (size_t lv = 0; lv + 1 < F.off.size(); ++lv) {
      const int32_t b = F.off[lv], e = F.off[lv + 1];
      std::vector<int32_t> pool;
      for (int32_t i = b; i < e; ++i) pool.push_back(i);
      std::vector<int32_t> out;
      out.reserve(pool.size());
      std::vector<uint8_t> used(pool.size(), 0);
      size_t head = 0;
      while (out.size() < pool.size()) {
        int32_t gl[kGroup], gr[kGroup], gs[kGroup];
        int n = 0;
        for (size_t t = head; t < pool.size() && n < kGroup && t < head + kLook; ++t) {
          if (used[t]) continue;
          const int32_t i = pool[t];
          bool ok = true;
          for (int q = 0; q < n && ok; ++q) {
            ok &= (F.l[i] % kGroup != gl[q] % kGroup) || F.l[i] == gl[q];
            ok &= (F.r[i] % kGroup != gr[q] % kGroup) || F.r[i] == gr[q];
            ok &= F.slot[i] % kGroup != gs[q] % kGroup;
          }
          if (!ok) continue;
          used[t] = 1;
          gl[n] = F.l[i];
          gr[n] = F.r[i];
          gs[n] = F.slot[i];
          ++n;
          out.push_back(i);
        }
        for (size_t t = head; t < pool.size() && n < kGroup; ++t)  // no fit in the window: next nodes
          if (!used[t]) {
            used[t] = 1;
            ++n;
            out.push_back(pool[t]);
          }
        while (head < pool.size() && used[head]) ++head;
      }
      std::vector<int32_t> ns(out.size()), nl(out.size()), nr(out.size());
      for (size_t q = 0; q < out.size(); ++q) {
        ns[q] = F.slot[out[q]];
        nl[q] = F.l[out[q]];
        nr[q] = F.r[out[q]];
      }
      std::copy(ns.begin(), ns.end(), F.slot.begin() + b);
      std::copy(nl.begin(), nl.end(), F.l.begin() + b);
      std::copy(nr.begin(), nr.end(), F.r.begin() + b);
    }
  }
  fill_levels(inner_slots, plan.rev, true);
  if ((int)plan.fwd.off.size() - 1 > nu_max || (int)plan.rev.off.size() - 1 > nu_max)
    return fail(ACE_ERR_INVALID_ARG, "internal: too many levels");

  // gather form of the reverse sweep: consumers of each factor among the inner operands
  {
    std::vector<std::vector<std::pair<int32_t, int32_t>>> cons(plan.n_g);
    for (int32_t i = K; i < plan.n_g; ++i) {
      cons[slot_l[i]].push_back({i, slot_r[i]});
      cons[slot_r[i]].push_back({i, slot_l[i]});
    }
    std::vector<int32_t> tg;
    for (int32_t x = 0; x < plan.n_g; ++x)
      if (!cons[x].empty()) tg.push_back(x);
    auto order_of = [&](int32_t x) { return g.order[plan.slot_node[x]]; };
    // order descending, then by slot
    std::stable_sort(tg.begin(), tg.end(), [&](int32_t a, int32_t b) {
      if (order_of(a) != order_of(b)) return order_of(a) > order_of(b);
      return a < b;
    });
    PullList& P = plan.pull;
    P = PullList();
    int32_t cur = -1;
    for (int32_t x : tg) {
      if (order_of(x) != cur) {
        P.lvl.push_back((int32_t)P.src.size());
        cur = order_of(x);
      }
      for (auto& pr : cons[x]) {
        P.src.push_back(pr.first);
        P.par.push_back(pr.second);
        P.tgt.push_back(x);
      }
    }
    P.lvl.push_back((int32_t)P.src.size());
    if ((int)P.lvl.size() - 1 > nu_max) return fail(ACE_ERR_INVALID_ARG, "internal: too many levels");
  }

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
  build_tasks(sym_rows, plan.slot_basis, plan.n_g, plan.n_stored, true, slot_l, slot_r, task_len, plan.sym);
  build_tasks(one_rows, plan.slot_basis, plan.n_g, plan.n_stored, false, slot_l, slot_r, task_len, plan.one);
  // the tile-per-lane kernel's adjoint rows (it carries them in 15-bit fields: larger graphs keep
  // the identity; measured on the stress graph: slices formed again with the second targets in
  // distinct banks under the permutation raise the bank conflicts, 2,232 or 2,307 against 2,065)
  plan.g_perm.resize(plan.n_g);
  std::iota(plan.g_perm.begin(), plan.g_perm.end(), 0);
  if (plan.n_g <= 32767) choose_g_perm(plan);
  return ACE_OK;
}

}  // namespace ace
