// Internal host-side structures of libace: index set, graph and evaluation plan.
//
// The index set follows sections 2.2-2.5 (Eq. 3), the graph section 2.6 with
// Algorithm 1 (section 3.2) / Algorithm 2 (section 3.3), and the plan is the
// GPU layout of the recursive evaluation of Eq. 4 (not in the paper).
#pragma once

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "../../../include/ace.h"

namespace ace {

constexpr int kMaxNu = 8;

// Error reporting: a status plus a thread-local message.
ace_status fail(ace_status st, const std::string& msg);
void clear_error();

struct Spec {
  ace_spec_params p{};
  int32_t K = 0;                      // one-particle functions
  std::vector<int32_t> one_deg;       // per one-particle id: degree
  std::vector<int32_t> one_m;         // per id: m
  std::vector<int32_t> one_l;         // per id: l (O(3)), 0 otherwise
  int32_t nu_max = 0;
  std::vector<int32_t> tuples;        // [n_basis][nu_max], -1 padded, canonical order
  std::vector<int32_t> nu;            // [n_basis]
  std::vector<int32_t> deg;           // [n_basis] total degree (sum of one-particle degrees)
  std::vector<int64_t> counts_per_nu; // [nu_max]
  int64_t n_basis() const { return (int64_t)nu.size(); }
};

ace_status build_spec(const ace_spec_params& p, std::unique_ptr<Spec>& out);

// Graph G in canonical (insertion) ids.
struct Graph {
  int32_t K = 0;
  int32_t nu_max = 0;
  std::vector<int32_t> left, right;   // -1 for leaves
  std::vector<int32_t> order;         // correlation order (topological level)
  std::vector<uint8_t> is_aux;
  std::vector<int32_t> basis_node;    // basis index -> node id
  std::vector<int32_t> node_basis;    // node id -> basis index or -1
  int64_t n_nodes() const { return (int64_t)left.size(); }
};

ace_status build_graph(const Spec& spec, int algo, int split_rule, int n_split, Graph& g);

// Options a graph and its plan were built with (kept with the graph, written to graph files).
struct GraphOptions {
  int32_t algo = 1, split_rule = 0, n_split = 2, task_len = 64;
};

// Graph files (checkpoint.cpp): the index set's parameters, the options and the graph, with a
// checksum; load_graph rebuilds the index set, checks it and the graph, and fills g.
ace_status save_graph(const std::string& path, const Spec& spec, const Graph& g, const GraphOptions& o);
ace_status load_graph(const std::string& path, std::unique_ptr<Spec>& spec, Graph& g, GraphOptions& o);

// Evaluation plan (section 2.6 recursion laid out for the fused kernels).
//
// Slots are the values kept per environment: [0, K) the leaves A_k, then the
// operand nodes (order >= 2 with at least one consumer).  Operand nodes whose
// consumers include other operand nodes ("inner" operands) come first, so that
// the adjoint accumulators G exist exactly for slots [0, n_g).  Sink nodes
// (order >= 2, no consumer) are never stored: sink i = [p, q] contributes
// c_i AA_p AA_q to phi, which is folded into a sparse contraction over slots.
struct Task {
  int32_t row;    // slot whose sparse row this task covers (-1: padding)
  int32_t flags;  // bit0: first task of its row (adds the row's own coefficient)
                  // bit1: row is a top operand (push to its factors) else G row
                  // bit2: the row's stored value is a basis function (has a coefficient)
  int32_t pl, pr; // factor slots of a top operand row, else -1
};

// Warps per CTA of the one-environment-per-lane kernel (1024 threads).
constexpr int kLoeWarps = 32;
// Blocks of that kernel's streams: rows with equal column sets of at most kLoeBlockCols
// columns, kLoeBlockMinRows or more of them, in units of at most kLoeBlockRows rows.
constexpr int kLoeBlockCols = 8;
constexpr int kLoeBlockMinRows = 2;
constexpr int kLoeBlockRows = 16;
// Flag bits beyond those of Task::flags: a row-major task that is a block row (its
// coefficients follow its header four per item, in the block's column order), and a
// stream item that is a block header.
constexpr int kTaskBlockRow = 8;
constexpr int kLoeBlockUnit = 16;
// Most slots the tile-per-lane kernel can keep (its columns are 16-bit): a plan with more has
// no tile-per-lane layout (the hot and cold tasks below stay empty).
constexpr int32_t kTileMaxStored = 65535;

struct TaskSet {
  // Tasks grouped in slices of 32 (one per lane); entries of a slice are
  // interleaved: entry k of lane j sits at slice_off[s] + 32 k + j.  Built only
  // when the plan keeps at most kTileMaxStored slots.
  std::vector<Task> tasks;            // [n_slices * 32]
  std::vector<int32_t> slice_off;     // [n_slices + 1] entry offsets
  std::vector<int32_t> slice_steps;   // [n_slices]
  std::vector<int32_t> col;           // [n_entries_padded] slot index
  std::vector<int32_t> ebasis;        // [n_entries_padded] basis index (-1 padding)
  std::vector<uint8_t> ew2;           // [n_entries_padded] 1: weight 2 (diagonal of the symmetric form)
  int64_t n_entries = 0;              // real (unpadded) entries of all rows
  // Cold entries: entries whose column is a top operand that the tile-per-lane
  // kernel does not keep in shared memory (slots >= n_stored).  Such an entry
  // reads the operand's two factor slots (ca, cb < n_g) and multiplies them.
  // They form their own tasks (no row coefficient), sliced like the others,
  // entry k of lane j at cold_slice_off[s] + 32 k + j.
  std::vector<Task> cold_tasks;       // [n_cold_slices * 32]
  std::vector<int32_t> cold_slice_off, cold_slice_steps;
  std::vector<int32_t> cold_ca, cold_cb, cold_ebasis;
  std::vector<uint8_t> cold_ew2;
  int32_t n_cold_slices() const { return (int32_t)cold_slice_steps.size(); }
  // The same tasks with their entries contiguous (for the kernel in which a
  // whole warp works on one task, one environment per lane); every task's
  // entry count is padded to an even number (entries are read in pairs).
  std::vector<Task> rm_tasks;         // [n_rm] in slice order, padding tasks dropped
  std::vector<int32_t> rm_off;        // [n_rm + 1]
  std::vector<int32_t> rm_col, rm_ebasis;
  std::vector<uint8_t> rm_ew2;
  // Their layout as one stream per warp of that kernel (kLoeWarps warps per CTA;
  // units spread over the warps longest first): a unit is either a task (a 16-byte
  // header followed by its entry pairs, 16 bytes each) or a block (a header
  // {m, rows << 8 | kLoeBlockUnit, 0, 0}, kLoeBlockCols / 4 items of columns, then
  // per row its header and kLoeBlockCols / 4 items of coefficients).  The rm tasks
  // are in stream order.  Positions count 16-byte items.
  std::vector<int32_t> loe_wbeg;      // [kLoeWarps + 1] first item of each warp's stream
  std::vector<int32_t> loe_hpos;      // [n_rm] item of each task's (or block row's) header
  std::vector<int32_t> loe_spos;      // items written once, not by the binding: block headers, columns
  std::vector<int32_t> loe_sval;      // [4 per loe_spos] their values
  int32_t n_slices() const { return (int32_t)slice_steps.size(); }
};

struct LevelList {
  std::vector<int32_t> slot, l, r;    // node slot and its two factor slots
  std::vector<int32_t> off;           // level offsets (size n_levels + 1)
};

// The adjoint sweep through the inner operand nodes as one flat list of
// (consumer, partner, target) triples: every inner operand i = [x, p]
// contributes G_i AA_p to G_x (and G_i AA_x to G_p).  Triples are grouped by the
// correlation order of their target, descending (every consumer of a target has
// a higher order, so its G is final when the target's level runs), and sorted
// by target within a level, so that equal targets are contiguous and can be
// summed before one update.
struct PullList {
  std::vector<int32_t> src, par, tgt; // consumer slot i, partner factor slot p, target slot x
  std::vector<int32_t> lvl;           // level offsets into the triples (size n_levels + 1)
};

struct Plan {
  int32_t K = 0, n_slots = 0, n_g = 0;
  // Slots [0, n_stored) are kept in shared memory by the tile-per-lane kernel:
  // leaves, inner operands and the top operands used by the most sink entries;
  // the rest (cold top operands) are read through their factors.  n_stored is
  // chosen so that a tile of four environments fits in 227 KB of shared memory.
  int32_t n_stored = 0;
  int64_t n_sinks = 0;
  std::vector<int32_t> node_slot;     // node id -> slot or -1
  std::vector<int32_t> slot_node;     // slot -> node id
  std::vector<int32_t> slot_basis;    // slot -> basis index or -1 (linear coefficient)
  LevelList fwd;                      // operand nodes by increasing order
  LevelList fwd_stored;               // the same, restricted to slots < n_stored
  LevelList rev;                      // inner operand nodes by decreasing order
  PullList pull;                      // the same sweep, gathered per target
  TaskSet sym;                        // symmetric sink form (forward + adjoint)
  TaskSet one;                        // one-sided sink form (forward only)
  // Adjoint row of each slot with an adjoint (a permutation of [0, n_g)) for the tile-per-lane
  // kernel, chosen so that the adjoint updates issued together fall in different banks.
  std::vector<int32_t> g_perm;
};

// stored_limit(K, n_g): at most this many slots are kept for the tile-per-lane
// kernel (0: no limit); see Plan::n_stored.
using StoredLimitFn = int64_t (*)(int32_t K, int32_t n_g);
ace_status build_plan(const Spec& spec, const Graph& g, int task_len, StoredLimitFn stored_limit, Plan& plan);

}  // namespace ace
