// Computational graph G (section 2.6) built by Algorithm 1 (section 3.2) or
// Algorithm 2 (section 3.3).
//
// Rules fixed where the paper leaves a choice (the oracle states the same
// readings in its own code):
//  * Decompositions k = [k1, k2] are tried with |k1| = s for s = nu/2 down to 1
//    (balanced) or 1 up to nu/2 (peel); for each s the positions of k1 run
//    over the s-subsets of tuple positions in lexicographic order, skipping a
//    k1 multiset already tried for this s.  The first pair with both parts in
//    G is used; left = k1, right = the complement.
//  * Fallback of Algorithm 1: split off the element of largest one-particle
//    degree, ties broken towards the largest position; insert the rest, then
//    run the insertion of k again from the start.
//  * Fallback of Algorithm 2: the s = min(n, nu-1) elements of largest degree
//    (same tie rule) form the head, inserted with Algorithm 1; then the rest
//    with Algorithm 2; then k again.
//  * Node ids follow insertion order; leaves (the K one-particle nodes) are
//    0..K-1; auxiliary = order >= 2 and not in the basis set.
#include <algorithm>
#include <vector>

#include "ace_internal.hpp"

namespace ace {

namespace {

struct Key {
  uint64_t a, b;  // up to 8 ids of 16 bits, 0xFFFF padded
  bool operator==(const Key& o) const { return a == o.a && b == o.b; }
};

struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t h = k.a * 0x9E3779B97F4A7C15ULL ^ (k.b + 0x632BE59BD9B4E019ULL + (k.a << 6) + (k.a >> 2));
    h ^= h >> 33;
    h *= 0xFF51AFD7ED558CCDULL;
    h ^= h >> 33;
    return (size_t)h;
  }
};

// Node ids by tuple: open addressing with linear probing over a power-of-two table.  The empty
// slot holds the all-padding key, which no tuple has (ids are below 0xFFFF and a tuple has at
// least one).  Grown by doubling past a load of 3/4.
class NodeTable {
 public:
  void reserve(size_t n) {
    size_t cap = 1024;
    while (3 * cap < 4 * n) cap <<= 1;
    if (cap > keys_.size()) rehash(cap);
  }
  int32_t find(const Key& k) const {
    if (keys_.empty()) return -1;
    for (size_t i = KeyHash()(k) & mask_;; i = (i + 1) & mask_) {
      if (keys_[i] == k) return vals_[i];
      if (keys_[i] == kEmpty) return -1;
    }
  }
  void insert(const Key& k, int32_t v) {  // k not present
    if (4 * (used_ + 1) > 3 * keys_.size()) rehash(keys_.empty() ? 1024 : 2 * keys_.size());
    size_t i = KeyHash()(k) & mask_;
    while (!(keys_[i] == kEmpty)) i = (i + 1) & mask_;
    keys_[i] = k;
    vals_[i] = v;
    ++used_;
  }

 private:
  static constexpr Key kEmpty{~0ULL, ~0ULL};
  std::vector<Key> keys_;
  std::vector<int32_t> vals_;
  size_t mask_ = 0, used_ = 0;

  void rehash(size_t cap) {
    std::vector<Key> ok = std::move(keys_);
    std::vector<int32_t> ov = std::move(vals_);
    keys_.assign(cap, kEmpty);
    vals_.assign(cap, -1);
    mask_ = cap - 1;
    used_ = 0;
    for (size_t i = 0; i < ok.size(); ++i)
      if (!(ok[i] == kEmpty)) insert(ok[i], ov[i]);
  }
};

struct Tup {
  int32_t n = 0;
  int32_t v[kMaxNu];
  Key key() const {
    uint64_t w[2] = {~0ULL, ~0ULL};
    for (int i = 0; i < n; ++i) {
      int word = i >> 2, sh = (i & 3) * 16;
      w[word] &= ~(0xFFFFULL << sh);
      w[word] |= (uint64_t)(uint16_t)v[i] << sh;
    }
    return Key{w[0], w[1]};
  }
};

// Most k1 position sets of one size: C(8, 4) for tuples of at most 8 elements.
static_assert(kMaxNu <= 8, "Key packs at most 8 ids");
constexpr int kMaxSubsets = 70;

struct Builder {
  const Spec& s;
  int split_rule;
  int n_split;
  Graph& g;
  NodeTable ids;

  Builder(const Spec& s_, int rule, int ns, Graph& g_) : s(s_), split_rule(rule), n_split(ns), g(g_) {}

  int32_t add(const Tup& t, int32_t l, int32_t r) {
    int32_t id = (int32_t)g.left.size();
    ids.insert(t.key(), id);
    g.left.push_back(l);
    g.right.push_back(r);
    g.order.push_back(t.n);
    return id;
  }

  int32_t find(const Tup& t) const { return ids.find(t.key()); }

  // Try every decomposition in the fixed order; add k with the first pair found.
  bool try_pairs(const Tup& t) {
    const int nu = t.n;
    for (int step = 0; step < nu / 2; ++step) {
      const int sz = split_rule == ACE_SPLIT_PEEL ? step + 1 : nu / 2 - step;
      Key seen[kMaxSubsets];  // the k1 multisets already tried for this size
      int n_seen = 0;
      int pos[kMaxNu];
      for (int i = 0; i < sz; ++i) pos[i] = i;
      while (true) {
        Tup a, b;
        a.n = sz;
        b.n = nu - sz;
        int pi = 0, bi = 0;
        for (int i = 0; i < nu; ++i) {
          if (pi < sz && pos[pi] == i) a.v[pi++] = t.v[i];
          else b.v[bi++] = t.v[i];
        }
        Key ka = a.key();
        bool dup = std::find(seen, seen + n_seen, ka) != seen + n_seen;
        if (!dup) {
          seen[n_seen++] = ka;
          int32_t ia = find(a);
          if (ia >= 0) {
            int32_t ib = find(b);
            if (ib >= 0) {
              add(t, ia, ib);
              return true;
            }
          }
        }
        // next combination in lexicographic order
        int i = sz - 1;
        while (i >= 0 && pos[i] == nu - sz + i) --i;
        if (i < 0) break;
        ++pos[i];
        for (int j = i + 1; j < sz; ++j) pos[j] = pos[j - 1] + 1;
      }
    }
    return false;
  }

  // positions of the s largest one-particle degrees, ties to larger positions; ascending
  void top_positions(const Tup& t, int s_cnt, int* out) const {
    int idx[kMaxNu];
    for (int i = 0; i < t.n; ++i) idx[i] = i;
    std::sort(idx, idx + t.n, [&](int x, int y) {
      int dx = s.one_deg[t.v[x]], dy = s.one_deg[t.v[y]];
      if (dx != dy) return dx > dy;
      return x > y;
    });
    std::copy(idx, idx + s_cnt, out);
    std::sort(out, out + s_cnt);
  }

  void insert1(const Tup& t) {
    if (find(t) >= 0) return;
    if (try_pairs(t)) return;
    int j;
    top_positions(t, 1, &j);
    Tup rest;
    rest.n = t.n - 1;
    for (int i = 0, o = 0; i < t.n; ++i)
      if (i != j) rest.v[o++] = t.v[i];
    insert1(rest);  // [t_j] is a leaf, always present
    insert1(t);
  }

  void insert2(const Tup& t) {
    if (find(t) >= 0) return;
    if (try_pairs(t)) return;
    int s_cnt = std::min(n_split, t.n - 1);
    int pos[kMaxNu];
    top_positions(t, s_cnt, pos);
    Tup head, rest;
    head.n = s_cnt;
    rest.n = t.n - s_cnt;
    int pi = 0, ri = 0;
    for (int i = 0; i < t.n; ++i) {
      if (pi < s_cnt && pos[pi] == i) head.v[pi++] = t.v[i];
      else rest.v[ri++] = t.v[i];
    }
    insert1(head);
    insert2(rest);
    insert2(t);
  }
};

}  // namespace

ace_status build_graph(const Spec& spec, int algo, int split_rule, int n_split, Graph& g) {
  if (algo != ACE_ALGO_1 && algo != ACE_ALGO_2) return fail(ACE_ERR_INVALID_ARG, "algo must be 1 or 2");
  if (split_rule != ACE_SPLIT_BALANCED && split_rule != ACE_SPLIT_PEEL)
    return fail(ACE_ERR_INVALID_ARG, "unknown split rule");
  if (algo == ACE_ALGO_2 && n_split < 1) return fail(ACE_ERR_INVALID_ARG, "n_split must be >= 1");
  g = Graph();
  g.K = spec.K;
  g.nu_max = spec.nu_max;
  Builder b(spec, split_rule, n_split, g);
  b.ids.reserve((size_t)spec.n_basis() + (size_t)spec.n_basis() / 16 + spec.K);  // basis, auxiliary, leaves
  for (int32_t k = 0; k < spec.K; ++k) {
    Tup t;
    t.n = 1;
    t.v[0] = k;
    b.add(t, -1, -1);
  }
  const int nu_max = spec.nu_max;
  for (int64_t i = 0; i < spec.n_basis(); ++i) {
    Tup t;
    t.n = spec.nu[i];
    for (int j = 0; j < t.n; ++j) t.v[j] = spec.tuples[i * nu_max + j];
    if (t.n < 2) continue;
    if (algo == ACE_ALGO_1) b.insert1(t);
    else b.insert2(t);
  }
  const int64_t N = g.n_nodes();
  g.is_aux.assign(N, 0);
  g.node_basis.assign(N, -1);
  g.basis_node.assign(spec.n_basis(), -1);
  for (int64_t i = 0; i < spec.n_basis(); ++i) {
    Tup t;
    t.n = spec.nu[i];
    for (int j = 0; j < t.n; ++j) t.v[j] = spec.tuples[i * nu_max + j];
    int32_t id = b.find(t);
    if (id < 0) return fail(ACE_ERR_INVALID_ARG, "internal: basis tuple missing from graph");
    g.basis_node[i] = id;
    g.node_basis[id] = (int32_t)i;
  }
  for (int64_t i = spec.K; i < N; ++i) g.is_aux[i] = g.node_basis[i] < 0 ? 1 : 0;
  return ACE_OK;
}

}  // namespace ace
