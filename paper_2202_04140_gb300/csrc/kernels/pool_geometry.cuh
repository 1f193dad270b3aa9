// Neighbour geometry for the pooling kernels, in FP32 only.
//
// FP64 runs at about 1/64 of the FP32 rate on this GPU, so the digits that plain
// FP32 would lose are carried as unevaluated sums hi + lo of two floats, built from
// two error-free transformations:
//   TwoSum (Knuth): s = fl(a + b) and e = (a + b) - s exactly, six additions;
//   TwoProduct (Dekker, with a fused multiply-add): p = fl(a b), e = fma(a, b, -p) = a b - p.
// The intrinsics (__fadd_rn, __fmul_rn, __fmaf_rn) keep the compiler from contracting
// a product and a sum into an FMA, which would break the exactness of both.
//
// What needs the extra digits:
//  * r^2 and rc^2 - r^2: 1 - r/rc = (rc^2 - r^2) / ((rc + r) rc) must keep its relative
//    accuracy next to the cutoff, where rc^2 - r^2 cancels;
//  * 1/r: the reciprocal square root refined by one Newton-Raphson step
//    y0 (1 + rho/2), rho = 1 - r^2 y0^2 formed exactly, and the unit vector from it,
//    each component rounded once (high-l harmonics amplify direction errors);
//  * t = 2r/rc - 1, rounded once (T_n(t) has slope n^2 at the ends).
// All products of two floats and the squares are exact as hi + lo, so each output is
// the exact value up to terms of relative size ~2^-44 before its one final rounding.
#pragma once

#if defined(__CUDACC__)
#define ACE_HD __host__ __device__ __forceinline__
#else
#define ACE_HD inline
#endif

namespace ace {
namespace geo {

#if defined(__CUDA_ARCH__)
ACE_HD float add(float a, float b) { return __fadd_rn(a, b); }
ACE_HD float mul(float a, float b) { return __fmul_rn(a, b); }
ACE_HD float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
ACE_HD float rsqrt(float a) { return rsqrtf(a); }
ACE_HD float div(float a, float b) { return __fdiv_rn(a, b); }
#else
// Host build (accuracy checks): the same operations, each rounded to float; the
// translation unit must be compiled without floating-point contraction.
ACE_HD float add(float a, float b) { return a + b; }
ACE_HD float mul(float a, float b) { return a * b; }
ACE_HD float fma(float a, float b, float c) { return __builtin_fmaf(a, b, c); }
#ifdef ACE_GEO_HOST_RSQRT
// an accuracy check may stand in an approximate seed, as the device's rsqrtf is one
ACE_HD float rsqrt(float a) { return ACE_GEO_HOST_RSQRT(a); }
#else
ACE_HD float rsqrt(float a) { return 1.0f / __builtin_sqrtf(a); }
#endif
ACE_HD float div(float a, float b) { return a / b; }
#endif

// TwoSum: s + e = a + b exactly.
ACE_HD void two_sum(float a, float b, float& s, float& e) {
  s = add(a, b);
  const float bb = add(s, -a);
  e = add(add(a, -add(s, -bb)), add(b, -bb));
}

// TwoProduct: p + e = a b exactly.
ACE_HD void two_prod(float a, float b, float& p, float& e) {
  p = mul(a, b);
  e = fma(a, b, -p);
}

// Per-thread constants of the cutoff: rc^2 = rc2h + rc2l, 2/rc = qh + ql.
struct Cut {
  float rc, rc2h, rc2l, qh, ql;
};

ACE_HD Cut make_cut(float rc) {
  Cut c;
  c.rc = rc;
  two_prod(rc, rc, c.rc2h, c.rc2l);
  c.qh = div(2.0f, rc);
  c.ql = div(fma(-c.qh, rc, 2.0f), rc);  // 2 - qh rc is exact (residual of a rounded quotient)
  return c;
}

struct Geo {
  bool ok;                // 0 < r < rc (a neighbour at the centre or beyond rc adds nothing)
  float ir, xh, yh, u, t, w;  // 1/r, unit vector (xh, yh, u), 2r/rc - 1, 1 - r/rc
};

ACE_HD Geo geometry(float x, float y, float z, const Cut& c) {
  Geo g;
  // r^2 = hi + lo
  float px, ex, py, ey, pz, ez, s1, e1, hi, e2;
  two_prod(x, x, px, ex);
  two_prod(y, y, py, ey);
  two_prod(z, z, pz, ez);
  two_sum(px, py, s1, e1);
  two_sum(s1, pz, hi, e2);
  float lo = add(add(ex, ey), add(ez, add(e1, e2)));
  {
    const float s = add(hi, lo);  // renormalise: hi = fl(r^2)
    lo = add(lo, -add(s, -hi));
    hi = s;
  }
  // rc^2 - r^2 = d + dl
  float d, de;
  two_sum(c.rc2h, -hi, d, de);
  const float d2 = add(d, add(de, add(c.rc2l, -lo)));
  g.ok = hi >= 1e-30f && d2 > 0.0f;
  // 1/r = y0 + il with rho = 1 - r^2 y0^2 formed exactly up to second-order terms
  const float y0 = rsqrt(g.ok ? hi : 1.0f);
  float a, b, cc, dd;
  two_prod(y0, y0, a, b);   // y0^2 = a + b
  two_prod(hi, a, cc, dd);  // hi a = cc + dd
  const float rho = add(add(add(1.0f, -cc), -dd), -fma(hi, b, mul(lo, a)));  // 1 - cc is exact
  const float il = g.ok ? mul(mul(0.5f, y0), rho) : 0.0f;
  const float y0k = g.ok ? y0 : 0.0f;
  g.ir = add(y0k, il);
  g.xh = fma(x, y0k, mul(x, il));
  g.yh = fma(y, y0k, mul(y, il));
  g.u = fma(z, y0k, mul(z, il));
  // r = r^2 / r = rh + rl
  float rh, re;
  two_prod(hi, y0k, rh, re);
  const float rl = add(re, fma(hi, il, mul(lo, y0k)));
  const float r = add(rh, rl);
  g.w = g.ok ? div(d2, mul(add(c.rc, r), c.rc)) : 0.0f;
  // t = r (2/rc) - 1
  float p, pe, s, se;
  two_prod(rh, c.qh, p, pe);
  two_sum(p, -1.0f, s, se);
  g.t = add(s, add(add(se, pe), fma(rh, c.ql, mul(rl, c.qh))));
  return g;
}

}  // namespace geo
}  // namespace ace
