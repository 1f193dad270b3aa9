// Accuracy of the pooling geometry (paper_2202_04140_gb300/csrc/kernels/pool_geometry.cuh)
// against long-double values, on the host.  Compiled and run by tests/test_pool_geometry.py
// with floating-point contraction off, so each float operation is rounded once, as the
// device intrinsics are.  The device's rsqrtf is an approximation (a few ulp); here the seed
// of 1/r is the correctly rounded value moved by -2..+2 ulp, chosen per input, so that the
// Newton step has real work to do.
//
// Output: one line per region "region n max_ulp_ir max_ulp_unit max_ulp_t max_abs_t
// max_rel_w max_abs_w", the errors of 1/r, of the unit vector components (in ulp of the
// exact value), of t = 2r/rc - 1 and of w = 1 - r/rc.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

static float seed_rsqrt(float a) {
  float y = 1.0f / std::sqrt(a);
  uint32_t h;
  std::memcpy(&h, &a, 4);
  h ^= h >> 13;
  h *= 0x9e3779b1u;
  const int k = (int)(h >> 29) % 5 - 2;
  for (int i = 0; i < (k < 0 ? -k : k); ++i) y = std::nextafter(y, k < 0 ? 0.0f : 1e30f);
  return y;
}
#define ACE_GEO_HOST_RSQRT seed_rsqrt
#include "../paper_2202_04140_gb300/csrc/kernels/pool_geometry.cuh"

typedef long double LD;

static LD ulp_of(LD x) {
  const float f = (float)x;
  const float a = std::fabs(f);
  const float up = std::nextafter(a, 1e30f);
  return (LD)(up - a);
}

static uint64_t rng_state = 0x243f6a8885a308d3ull;
static double uniform() {  // splitmix64 -> [0, 1)
  uint64_t z = (rng_state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

int main() {
  const float rc = 5.0f;
  const ace::geo::Cut cut = ace::geo::make_cut(rc);
  const char* names[4] = {"centre", "bulk", "cutoff", "axes"};
  const int per_region = 1000000;
  for (int region = 0; region < 4; ++region) {
    LD e_ir = 0, e_u = 0, e_t = 0, e_ta = 0, e_w = 0, e_wa = 0;
    int n = 0;
    for (int i = 0; i < per_region; ++i) {
      double d[3];
      double nn = 0;
      for (int c = 0; c < 3; ++c) {
        // direction: Gaussian by Box-Muller; the axes region zeroes one or two components
        const double u1 = uniform() + 1e-300, u2 = uniform();
        d[c] = std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
      }
      if (region == 3) {
        const int z1 = (int)(uniform() * 3), z2 = (int)(uniform() * 3);
        d[z1] = 0.0;
        if (uniform() < 0.5) d[z2] = 0.0;
      }
      for (int c = 0; c < 3; ++c) nn += d[c] * d[c];
      if (nn == 0.0) continue;
      double r;
      if (region == 0) r = std::pow(10.0, -6.0 + 4.0 * uniform());                 // 1e-6 .. 1e-2
      else if (region == 2) r = rc * (1.0 - std::pow(10.0, -7.0 + 5.0 * uniform()));  // rc (1 - 1e-7 .. 1e-2)
      else r = rc * std::cbrt(uniform());
      const float x = (float)(d[0] / std::sqrt(nn) * r), y = (float)(d[1] / std::sqrt(nn) * r),
                  z = (float)(d[2] / std::sqrt(nn) * r);
      const LD R2 = (LD)x * x + (LD)y * y + (LD)z * z;
      const LD R = std::sqrt(R2);
      if (!(R > 0) || !(R < (LD)rc)) continue;
      const ace::geo::Geo g = ace::geo::geometry(x, y, z, cut);
      if (!g.ok) {  // only r = 0 or r >= rc may be refused
        std::printf("refused %a %a %a\n", x, y, z);
        return 1;
      }
      ++n;
      const LD ir = 1.0L / R;
      if (std::fabs((LD)g.ir - ir) / ulp_of(ir) > e_ir) e_ir = std::fabs((LD)g.ir - ir) / ulp_of(ir);
      const float comp[3] = {g.xh, g.yh, g.u};
      const float in[3] = {x, y, z};
      for (int c = 0; c < 3; ++c) {
        const LD ex = (LD)in[c] / R;
        const LD err = ex == 0 ? std::fabs((LD)comp[c]) : std::fabs((LD)comp[c] - ex) / ulp_of(ex);
        if (err > e_u) e_u = err;
      }
      const LD t = 2.0L * R / (LD)rc - 1.0L;
      const LD w = 1.0L - R / (LD)rc;
      const LD et = std::fabs((LD)g.t - t);
      if (et / ulp_of(t) > e_t) e_t = et / ulp_of(t);
      if (et > e_ta) e_ta = et;
      const LD ew = std::fabs((LD)g.w - w);
      if (ew / w > e_wa) e_wa = ew / w;
      if (ew > e_w) e_w = ew;
    }
    std::printf("%s %d %.3Lf %.3Lf %.3Lf %.3Le %.3Le %.3Le\n", names[region], n, e_ir, e_u, e_t, e_ta, e_wa, e_w);
  }
  return 0;
}
