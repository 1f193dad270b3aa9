// Index set K_G^p(D): sorted, degree-truncated, invariant multi-indices.
//
// Sections 2.2 (SO(2)), 2.3 (torus), 2.4 (O(3)): one-particle bases and the
// invariance constraints sum m = 0 (and sum l even for O(3)); section 2.5,
// Eq. 3: truncation ||k||_p <= D.  Permutation symmetry (section 1) keeps only
// non-decreasing id tuples.  The tuples are produced by a depth-first walk that
// extends a tuple only with ids >= its last id and only while the degree budget
// allows; for a fixed length the walk visits tuples in lexicographic order, so
// the canonical order (nu, lexicographic) needs no sort.
#include <algorithm>
#include <cmath>
#include <functional>

#include "ace_internal.hpp"

namespace ace {

namespace {

struct Walker {
  const Spec& s;
  int32_t D;
  int32_t pnorm;  // 1, 2 or 0 (max)
  bool l_even;
  int32_t maxd = 0;
  // next[b * (K + 1) + k]: the smallest id >= k of one-particle degree <= b (K if none)
  std::vector<int32_t> next;
  std::vector<std::vector<int32_t>> found;  // per nu: flattened tuples
  int32_t cur[kMaxNu];

  Walker(const Spec& s_, int32_t D_, int32_t p_, bool le) : s(s_), D(D_), pnorm(p_), l_even(le) {
    for (int32_t d : s.one_deg) maxd = std::max(maxd, d);
    const int32_t K = s.K;
    next.assign((size_t)(maxd + 1) * (K + 1), K);
    for (int32_t b = 0; b <= maxd; ++b) {
      int32_t* nb = next.data() + (size_t)b * (K + 1);
      for (int32_t k = K - 1; k >= 0; --k) nb[k] = s.one_deg[k] <= b ? k : nb[k + 1];
    }
    found.assign(s.nu_max + 1, {});
  }

  // acc: accumulated norm measure (sum d, sum d^2, or max d)
  void walk(int depth, int32_t last, int64_t acc, int32_t msum, int32_t lsum) {
    if (depth > 0) {
      if (msum == 0 && (!l_even || (lsum % 2) == 0)) {
        auto& v = found[depth];
        v.insert(v.end(), cur, cur + depth);
      }
    }
    if (depth == s.nu_max) return;
    // children: ids >= last whose degree d keeps the tuple within the budget, in ascending id
    // order; the budget is a largest admissible degree dlim (sum d <= D, sum d^2 <= D^2, max d <= D)
    int64_t dlim;
    if (pnorm == 1) dlim = (int64_t)D - acc;
    else if (pnorm == 2) {
      const int64_t r = (int64_t)D * D - acc;
      dlim = r < 0 ? -1 : (int64_t)std::sqrt((double)r);
      while (dlim >= 0 && dlim * dlim > r) --dlim;
      while ((dlim + 1) * (dlim + 1) <= r) ++dlim;
    } else dlim = D;
    if (dlim < 0) return;
    const int32_t* nb = next.data() + (size_t)std::min<int64_t>(dlim, maxd) * (s.K + 1);
    for (int32_t k = nb[last]; k < s.K; k = nb[k + 1]) {
      int64_t d = s.one_deg[k];
      int64_t nacc = (pnorm == 1) ? acc + d : (pnorm == 2) ? acc + d * d : std::max<int64_t>(acc, d);
      cur[depth] = k;
      walk(depth + 1, k, nacc, msum + s.one_m[k], lsum + s.one_l[k]);
    }
  }
};

}  // namespace

ace_status build_spec(const ace_spec_params& p, std::unique_ptr<Spec>& out) {
  if (p.nu_max < 1 || p.nu_max > kMaxNu) return fail(ACE_ERR_INVALID_ARG, "nu_max must be in [1, 8]");
  if (p.deg_max < 0) return fail(ACE_ERR_INVALID_ARG, "deg_max must be >= 0");
  if (p.lmax < 0) return fail(ACE_ERR_INVALID_ARG, "lmax must be >= 0");
  if (p.p_norm != 0 && p.p_norm != 1 && p.p_norm != 2)
    return fail(ACE_ERR_INVALID_ARG, "p_norm must be 1, 2 or 0 (max)");
  auto s = std::make_unique<Spec>();
  s->p = p;
  s->nu_max = p.nu_max;
  if (p.group == ACE_GROUP_O3) {
    if (p.nmin < 0 || p.nmax < p.nmin) return fail(ACE_ERR_INVALID_ARG, "need 0 <= nmin <= nmax");
    if (p.wn < 0 || p.wl < 0 || p.wk < 0) return fail(ACE_ERR_INVALID_ARG, "degree weights must be >= 0");
    if (p.kmax < 0) return fail(ACE_ERR_INVALID_ARG, "kmax must be >= 0");
    // id order: n, then the feature degree k, then l, then m
    for (int32_t n = p.nmin; n <= p.nmax; ++n)
      for (int32_t k = 0; k <= p.kmax; ++k)
        for (int32_t l = 0; l <= p.lmax; ++l)
          for (int32_t m = -l; m <= l; ++m) {
            s->one_deg.push_back(p.wn * n + p.wl * l + p.wk * k);
            s->one_m.push_back(m);
            s->one_l.push_back(l);
          }
  } else if (p.group == ACE_GROUP_SO2) {
    if (p.nmin < 0 || p.nmax < p.nmin) return fail(ACE_ERR_INVALID_ARG, "need 0 <= nmin <= nmax");
    for (int32_t n = p.nmin; n <= p.nmax; ++n)
      for (int32_t m = -p.lmax; m <= p.lmax; ++m) {
        s->one_deg.push_back(p.wn * n + p.wl * std::abs(m));
        s->one_m.push_back(m);
        s->one_l.push_back(0);
      }
  } else if (p.group == ACE_GROUP_TORUS) {
    for (int32_t m = -p.lmax; m <= p.lmax; ++m) {
      s->one_deg.push_back(std::abs(m));
      s->one_m.push_back(m);
      s->one_l.push_back(0);
    }
  } else {
    return fail(ACE_ERR_INVALID_ARG, "unknown group");
  }
  s->K = (int32_t)s->one_deg.size();
  if (s->K == 0 || s->K > 65535) return fail(ACE_ERR_INVALID_ARG, "K must be in [1, 65535]");
  bool l_even = (p.group == ACE_GROUP_O3) && p.require_l_even;
  Walker w(*s, p.deg_max, p.p_norm, l_even);
  w.walk(0, 0, 0, 0, 0);
  s->counts_per_nu.assign(p.nu_max, 0);
  for (int nu = 1; nu <= p.nu_max; ++nu) {
    const auto& v = w.found[nu];
    int64_t cnt = (int64_t)v.size() / nu;
    s->counts_per_nu[nu - 1] = cnt;
    for (int64_t i = 0; i < cnt; ++i) {
      int32_t dsum = 0;
      for (int t = 0; t < p.nu_max; ++t) {
        int32_t k = t < nu ? v[i * nu + t] : -1;
        s->tuples.push_back(k);
        if (k >= 0) dsum += s->one_deg[k];
      }
      s->nu.push_back(nu);
      s->deg.push_back(dsum);
    }
  }
  out = std::move(s);
  return ACE_OK;
}

}  // namespace ace
