// Graph files: the index set's parameters, the build options and the graph G (section 2.6), so
// that a graph built once (seconds to minutes for millions of basis functions) is read back
// instead of searched again.  The evaluation plan is not stored; it is rebuilt from the graph.
//
// Layout (little-endian, written byte by byte so that it is the same on every host):
//   8 bytes   magic "ACEGRAPH"
//   u32       format version (1)
//   i32 x 12  ace_spec_params in declaration order
//   i32 x 4   algorithm, split rule, head size n of Algorithm 2, task length of the plan
//   i32       K;  i64 n_basis;  u64 FNV-1a 64 of the index set (tuples, then degrees, as i32)
//   i64       N, the node count
//   i32 x N   left, right, order (correlation order) of every node;  i32 x n_basis basis node
//   u64       FNV-1a 64 of every byte before it
#include <cstdio>
#include <cstring>

#include "ace_internal.hpp"

namespace ace {

namespace {

constexpr char kMagic[8] = {'A', 'C', 'E', 'G', 'R', 'A', 'P', 'H'};
constexpr uint32_t kVersion = 1;

// FNV-1a, 64-bit (offset basis 14695981039346656037, prime 1099511628211)
struct Fnv {
  uint64_t h = 14695981039346656037ULL;
  void add(const uint8_t* p, size_t n) {
    for (size_t i = 0; i < n; ++i) h = (h ^ p[i]) * 1099511628211ULL;
  }
};

struct Writer {
  std::vector<uint8_t> b;
  void u(uint64_t v, int bytes) {
    for (int i = 0; i < bytes; ++i) b.push_back((uint8_t)(v >> (8 * i)));
  }
  void i32(int32_t v) { u((uint32_t)v, 4); }
  void i64(int64_t v) { u((uint64_t)v, 8); }
  void i32s(const std::vector<int32_t>& v) {
    size_t at = b.size();
    b.resize(at + 4 * v.size());
    for (int32_t x : v) {
      const uint32_t y = (uint32_t)x;
      b[at] = (uint8_t)y;
      b[at + 1] = (uint8_t)(y >> 8);
      b[at + 2] = (uint8_t)(y >> 16);
      b[at + 3] = (uint8_t)(y >> 24);
      at += 4;
    }
  }
};

struct Reader {
  const std::vector<uint8_t>& b;
  size_t pos = 0, end;
  bool ok = true;
  Reader(const std::vector<uint8_t>& b_, size_t end_) : b(b_), end(end_) {}
  uint64_t u(int bytes) {
    if (!ok || end - pos < (size_t)bytes) {
      ok = false;
      return 0;
    }
    uint64_t v = 0;
    for (int i = 0; i < bytes; ++i) v |= (uint64_t)b[pos + i] << (8 * i);
    pos += bytes;
    return v;
  }
  int32_t i32() { return (int32_t)(uint32_t)u(4); }
  int64_t i64() { return (int64_t)u(8); }
  bool i32s(std::vector<int32_t>& v, int64_t n) {
    if (!ok || n < 0 || (uint64_t)n > (end - pos) / 4) return ok = false;
    v.resize((size_t)n);
    const uint8_t* p = b.data() + pos;
    for (int64_t i = 0; i < n; ++i, p += 4)
      v[(size_t)i] = (int32_t)((uint32_t)p[0] | (uint32_t)p[1] << 8 | (uint32_t)p[2] << 16 | (uint32_t)p[3] << 24);
    pos += 4 * (size_t)n;
    return ok;
  }
};

uint64_t spec_digest(const Spec& s) {
  Writer w;
  w.i32s(s.tuples);
  w.i32s(s.deg);
  Fnv f;
  f.add(w.b.data(), w.b.size());
  return f.h;
}

void put_params(Writer& w, const ace_spec_params& p) {
  for (int32_t v : {p.group, p.nmin, p.nmax, p.lmax, p.nu_max, p.deg_max, p.wn, p.wl, p.p_norm, p.require_l_even,
                    p.kmax, p.wk})
    w.i32(v);
}

ace_spec_params get_params(Reader& r) {
  ace_spec_params p{};
  for (int32_t* f : {&p.group, &p.nmin, &p.nmax, &p.lmax, &p.nu_max, &p.deg_max, &p.wn, &p.wl, &p.p_norm,
                     &p.require_l_even, &p.kmax, &p.wk})
    *f = r.i32();
  return p;
}

// splitmix64 finaliser: the per-id values of the multiset hash below
uint64_t id_value(int32_t id) {
  uint64_t z = (uint64_t)id + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Structural checks of a graph read from a file against its index set: leaves first, every
// other node the product of two earlier nodes with the sum of their orders, and every basis
// node distinct, of its function's order, and (by a multiset hash: a node's value is the sum
// over its tuple of a per-id value, so a product adds its factors' values) of its function's
// tuple.
ace_status check_graph(const Spec& s, const Graph& g) {
  const int64_t N = g.n_nodes(), K = s.K;
  if (N < K) return fail(ACE_ERR_INVALID_ARG, "graph file: fewer nodes than one-particle functions");
  std::vector<uint64_t> h((size_t)N);
  for (int64_t i = 0; i < N; ++i) {
    if (i < K) {
      if (g.left[i] != -1 || g.right[i] != -1 || g.order[i] != 1)
        return fail(ACE_ERR_INVALID_ARG, "graph file: leaf " + std::to_string(i) + " is not a leaf");
      h[i] = id_value((int32_t)i);
      continue;
    }
    const int32_t l = g.left[i], r = g.right[i];
    if (l < 0 || r < 0 || l >= i || r >= i)
      return fail(ACE_ERR_INVALID_ARG, "graph file: node " + std::to_string(i) + " has a factor that is not earlier");
    if (g.order[i] != g.order[l] + g.order[r] || g.order[i] > s.nu_max)
      return fail(ACE_ERR_INVALID_ARG, "graph file: order of node " + std::to_string(i));
    h[i] = h[l] + h[r];
  }
  std::vector<uint8_t> used((size_t)N, 0);
  const int nu_max = s.nu_max;
  for (int64_t b = 0; b < s.n_basis(); ++b) {
    const int32_t id = g.basis_node[b];
    if (id < 0 || id >= N || used[id] || g.order[id] != s.nu[b])
      return fail(ACE_ERR_INVALID_ARG, "graph file: basis node of function " + std::to_string(b));
    used[id] = 1;
    uint64_t want = 0;
    for (int t = 0; t < s.nu[b]; ++t) want += id_value(s.tuples[(size_t)b * nu_max + t]);
    if (h[id] != want)
      return fail(ACE_ERR_INVALID_ARG, "graph file: node of function " + std::to_string(b) + " is another product");
  }
  return ACE_OK;
}

}  // namespace

ace_status save_graph(const std::string& path, const Spec& s, const Graph& g, const GraphOptions& o) {
  Writer w;
  w.b.reserve(128 + 4 * (3 * (size_t)g.n_nodes() + g.basis_node.size()));
  w.b.insert(w.b.end(), kMagic, kMagic + 8);
  w.u(kVersion, 4);
  put_params(w, s.p);
  w.i32(o.algo);
  w.i32(o.split_rule);
  w.i32(o.n_split);
  w.i32(o.task_len);
  w.i32(s.K);
  w.i64(s.n_basis());
  w.u(spec_digest(s), 8);
  w.i64(g.n_nodes());
  w.i32s(g.left);
  w.i32s(g.right);
  w.i32s(g.order);
  w.i32s(g.basis_node);
  Fnv f;
  f.add(w.b.data(), w.b.size());
  w.u(f.h, 8);
  std::FILE* fp = std::fopen(path.c_str(), "wb");
  if (!fp) return fail(ACE_ERR_INVALID_ARG, "cannot open " + path + " for writing");
  const size_t n = std::fwrite(w.b.data(), 1, w.b.size(), fp);
  const bool closed = std::fclose(fp) == 0;
  if (n != w.b.size() || !closed) return fail(ACE_ERR_INVALID_ARG, "cannot write " + path);
  return ACE_OK;
}

ace_status load_graph(const std::string& path, std::unique_ptr<Spec>& spec, Graph& g, GraphOptions& o) {
  std::vector<uint8_t> b;
  {
    std::FILE* fp = std::fopen(path.c_str(), "rb");
    if (!fp) return fail(ACE_ERR_INVALID_ARG, "cannot open " + path);
    uint8_t buf[1 << 16];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof(buf), fp)) > 0) b.insert(b.end(), buf, buf + n);
    const bool err = std::ferror(fp) != 0;
    std::fclose(fp);
    if (err) return fail(ACE_ERR_INVALID_ARG, "cannot read " + path);
  }
  if (b.size() < 8 + 4 + 8 || std::memcmp(b.data(), kMagic, 8) != 0)
    return fail(ACE_ERR_INVALID_ARG, path + " is not a graph file");
  Reader tail(b, b.size());
  tail.pos = b.size() - 8;
  const uint64_t stored = tail.u(8);
  Fnv f;
  f.add(b.data(), b.size() - 8);
  if (f.h != stored) return fail(ACE_ERR_INVALID_ARG, "graph file: checksum mismatch (damaged or truncated)");
  Reader r(b, b.size() - 8);
  r.pos = 8;
  const uint32_t version = (uint32_t)r.u(4);
  if (version != kVersion)
    return fail(ACE_ERR_INVALID_ARG, "graph file: format version " + std::to_string(version) + ", this library reads " +
                                         std::to_string(kVersion));
  const ace_spec_params p = get_params(r);
  o.algo = r.i32();
  o.split_rule = r.i32();
  o.n_split = r.i32();
  o.task_len = r.i32();
  const int32_t K = r.i32();
  const int64_t n_basis = r.i64();
  const uint64_t digest = r.u(8);
  const int64_t N = r.i64();
  if (!r.ok) return fail(ACE_ERR_INVALID_ARG, "graph file: truncated header");
  if (o.task_len < 1) return fail(ACE_ERR_INVALID_ARG, "graph file: task length");
  ace_status st = build_spec(p, spec);
  if (st != ACE_OK) return st;
  if (spec->K != K || spec->n_basis() != n_basis || spec_digest(*spec) != digest)
    return fail(ACE_ERR_INVALID_ARG, "graph file: this library builds another index set from the stored parameters");
  g = Graph();
  g.K = K;
  g.nu_max = spec->nu_max;
  if (!r.i32s(g.left, N) || !r.i32s(g.right, N) || !r.i32s(g.order, N) || !r.i32s(g.basis_node, n_basis) ||
      r.pos != r.end)
    return fail(ACE_ERR_INVALID_ARG, "graph file: array sizes do not match the header");
  if ((st = check_graph(*spec, g)) != ACE_OK) return st;
  g.node_basis.assign((size_t)N, -1);
  for (int64_t i = 0; i < n_basis; ++i) g.node_basis[g.basis_node[i]] = (int32_t)i;
  g.is_aux.assign((size_t)N, 0);
  for (int64_t i = K; i < N; ++i) g.is_aux[i] = g.node_basis[i] < 0 ? 1 : 0;
  return ACE_OK;
}

}  // namespace ace
