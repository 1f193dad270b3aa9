// Neighbour pooling A_nlm = sum_j R_n(r_j) Y_lm(r_j/|r_j|) (Eq. 2, section 2.4)
// and its adjoint (forces).
//
// Basis (the paper fixes neither R_n nor a real form of Y_l^m):
//   R_n(r) = T_n(2r/rc - 1) (1 - r/rc)^2, T_n by T_{n+1} = 2t T_n - T_{n-1};
//   dR_n/dr by T'_{n+1} = 2 T_n + 2t T'_n - T'_{n-1}.
//   Y_l0 = N_l0 Q_l^0(u), Y_lm = sqrt2 N_lm Q_l^m(u) C_m, Y_l-m = sqrt2 N_lm Q_l^m(u) S_m
//   (m > 0), with u = z/r, C_m + i S_m = ((x + i y)/r)^m and Q_l^m = d^m P_l/du^m,
//   computed by Q_m^m = (2m-1)!!, Q_{m+1}^m = (2m+1) u Q_m^m,
//   (l-m) Q_l^m = (2l-1) u Q_{l-1}^m - (l+m-1) Q_{l-2}^m.  This is the real
//   orthonormal harmonic without Condon-Shortley phase, evaluated from the
//   Cartesian direction (no angles).
// Invariant features (phi_nlmk = R_n Y_l^m T_k(mu), section "Invariant
// features"): the radial factor becomes R_n(r) T_k(mu_j) with T_k the Chebyshev
// polynomial of the neighbour's feature value, radial-feature index
// q = (n - nmin)(kmax+1) + k, one-particle id q (lmax+1)^2 + l^2 + l + m.
// Gradients treat Y as a polynomial in the unit vector (xh, yh, zh):
//   dY/dxh = K Q m C_{m-1} (cos) or K Q m S_{m-1} (sin),
//   dY/dyh = -K Q m S_{m-1} (cos) or K Q m C_{m-1} (sin),
//   dY/dzh = K Q_l^{m+1} C_m (cos) or K Q_l^{m+1} S_m (sin),
// and grad_r Y = (g - rh (rh . g)) / r.
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "launch.hpp"
#include "loe_device.cuh"
#include "pool_geometry.cuh"

namespace ace {
namespace dev {

constexpr int kPoolLmax = 8;
constexpr int kPoolMaxR = 16;  // radial x feature factors per neighbour
constexpr int kPoolMaxF = 4;   // feature degrees 0..3
constexpr int kPoolQ = (kPoolLmax + 2) * (kPoolLmax + 3) / 2;  // Q_l^m for 0 <= m <= l+1 <= lmax+1
constexpr int kPoolWarps = 4;
constexpr int kPoolChunk = 32;  // neighbours staged per pass
constexpr int kPoolGroupEnvs = 4;  // adjoint: consecutive environments per warp, neighbours walked as one list

// K_lm (sqrt2 N_lm for m > 0, N_l0 for m = 0) and the recurrence coefficients,
// filled once from the host in double precision.
__constant__ float c_norm[kPoolLmax + 1][kPoolLmax + 1];
__constant__ float c_ra[kPoolLmax + 1][kPoolLmax + 1];  // (2l-1)/(l-m)
__constant__ float c_rb[kPoolLmax + 1][kPoolLmax + 1];  // (l+m-1)/(l-m)
__constant__ float c_dfac[kPoolLmax + 2];               // (2m-1)!!

__device__ __forceinline__ int qidx(int l, int m) { return l * (l + 1) / 2 + m; }

// Q[qidx(l,m)] = Q_l^m(u) for 0 <= m <= l <= lmax.
template <int LMAX>
__device__ __forceinline__ void legendre_q(float u, float (&Q)[kPoolQ]) {
#pragma unroll
  for (int m = 0; m <= LMAX; ++m) {
    Q[qidx(m, m)] = c_dfac[m];
    if (m + 1 <= LMAX) Q[qidx(m + 1, m)] = (2 * m + 1) * u * c_dfac[m];
#pragma unroll
    for (int l = m + 2; l <= LMAX; ++l)
      Q[qidx(l, m)] = c_ra[l][m] * u * Q[qidx(l - 1, m)] - c_rb[l][m] * Q[qidx(l - 2, m)];
  }
}

// A: one warp per environment; lanes compute R and Y of one neighbour each into
// shared memory, then lane owns lm = lane + 32 i for all radial n.
// T_k(mu) for k < kf (<= kPoolMaxF), T_0 = 1, T_1 = mu, T_{k+1} = 2 mu T_k - T_{k-1}.
__device__ __forceinline__ void feature_poly(float mu, int kf, float (&Tf)[kPoolMaxF]) {
  Tf[0] = 1.f;
#pragma unroll
  for (int k = 1; k < kPoolMaxF; ++k) Tf[k] = k == 1 ? mu : 2.f * mu * Tf[k - 1] - Tf[k - 2];
  (void)kf;
}

// Slot of radial factor n of staged neighbour jj in sR: the four 16-byte groups of a
// row are permuted by (jj / 2) mod 4, so that the 32 lanes writing factor n of their own
// neighbours hit 8 banks (4-way) instead of 2, while a row stays readable as float4s.
__device__ __forceinline__ int rslot(int jj, int n) { return ((((n >> 2) ^ (jj >> 1)) & 3) << 2) | (n & 3); }

template <int LMAX>
__global__ void __launch_bounds__(kPoolWarps * 32) pool_kernel(const float* __restrict__ pos,
                                                               const float* __restrict__ mu,
                                                               const int64_t* __restrict__ offsets, int64_t n_env,
                                                               float rc, int nmin, int nmax, int kf,
                                                               float* __restrict__ A) {
  constexpr int NL = (LMAX + 1) * (LMAX + 1);
  constexpr int NI = (NL + 31) / 32;
  __shared__ __align__(16) float sR[kPoolWarps][kPoolChunk][kPoolMaxR];
  __shared__ float sY[kPoolWarps][kPoolChunk][NL];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const geo::Cut cut = geo::make_cut(rc);
  const int nR0 = nmax - nmin + 1;
  const int nR = nR0 * kf;  // radial x feature factors
  const int K = nR * NL;
  for (int64_t env = blockIdx.x * (int64_t)kPoolWarps + warp; env < n_env; env += (int64_t)gridDim.x * kPoolWarps) {
    float acc[NI][kPoolMaxR];
#pragma unroll
    for (int i = 0; i < NI; ++i)
#pragma unroll
      for (int n = 0; n < kPoolMaxR; ++n) acc[i][n] = 0.f;
    const int64_t j0 = offsets[env], j1 = offsets[env + 1];
    for (int64_t jb = j0; jb < j1; jb += kPoolChunk) {
      const int64_t j = jb + lane;
      const int cnt = (int)((j1 - jb) < kPoolChunk ? (j1 - jb) : kPoolChunk);
      if (lane < cnt) {
        const float x = pos[3 * j], y = pos[3 * j + 1], z = pos[3 * j + 2];
        const geo::Geo g = geo::geometry(x, y, z, cut);
        const bool ok = g.ok;
        const float xh = g.xh, yh = g.yh, u = g.u, t = g.t;
        const float env2 = ok ? g.w * g.w : 0.f;
        float Tm1 = 1.f, T = t;
        for (int n = 1; n <= nmax; ++n) {
          if (n >= nmin) sR[warp][lane][rslot(lane, n - nmin)] = T * env2;
          const float Tn = 2.f * t * T - Tm1;
          Tm1 = T;
          T = Tn;
        }
        if (nmin == 0) sR[warp][lane][rslot(lane, 0)] = env2;
        if (kf > 1) {  // expand R_n into R_n T_k(mu_j), in place from the last factor down
          float Tf[kPoolMaxF];
          feature_poly(mu[j], kf, Tf);
          for (int i = nR0 - 1; i >= 0; --i) {
            const float rn = sR[warp][lane][rslot(lane, i)];
#pragma unroll
            for (int k = kPoolMaxF - 1; k >= 0; --k)
              if (k < kf) sR[warp][lane][rslot(lane, i * kf + k)] = rn * Tf[k];
          }
        }
        float Q[kPoolQ];
        legendre_q<LMAX>(u, Q);
        float C = 1.f, S = 0.f;
#pragma unroll
        for (int m = 0; m <= LMAX; ++m) {
#pragma unroll
          for (int l = m; l <= LMAX; ++l) {
            const float q = c_norm[l][m] * Q[qidx(l, m)];
            if (m == 0) {
              sY[warp][lane][l * l + l] = ok ? q : 0.f;
            } else {
              sY[warp][lane][l * l + l + m] = ok ? q * C : 0.f;
              sY[warp][lane][l * l + l - m] = ok ? q * S : 0.f;
            }
          }
          const float Cn = C * xh - S * yh;
          S = S * xh + C * yh;
          C = Cn;
        }
      }
      __syncwarp();
      for (int jj = 0; jj < cnt; ++jj) {
        float y[NI];
#pragma unroll
        for (int i = 0; i < NI; ++i) y[i] = (lane + 32 * i < NL) ? sY[warp][jj][lane + 32 * i] : 0.f;
        // factors n >= nR of the last group are stale; their sums are never stored
#pragma unroll
        for (int q = 0; q < kPoolMaxR / 4; ++q) {
          if (4 * q < nR) {
            const float4 rv = *reinterpret_cast<const float4*>(&sR[warp][jj][rslot(jj, 4 * q)]);
            const float r4[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
              for (int i = 0; i < NI; ++i) acc[i][4 * q + c] = __fmaf_rn(r4[c], y[i], acc[i][4 * q + c]);
          }
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int n = 0; n < kPoolMaxR; ++n) {
      if (n < nR) {
#pragma unroll
        for (int i = 0; i < NI; ++i) {
          const int lm = lane + 32 * i;
          if (lm < NL) A[env * K + n * NL + lm] = acc[i][n];
        }
      }
    }
  }
}

// Adjoint: one warp per group of environments, one lane per neighbour.  With
// G_q,lm = dphi/dA_q,lm (q the radial x feature factor) the force on neighbour j is
// built from
//   h_lm = sum_q G_q,lm R_q(r_j),   hd_lm = sum_q G_q,lm dR_q/dr(r_j)
// (49 + 49 values per lane for lmax = 6, held in registers; the radial index runs
// outside, each row of G read with 16-byte broadcast loads), then
//   dphi/dr_j = rh sum_lm hd_lm Y_lm + (grad_u - rh (rh . grad_u)) / r,
//   grad_u = sum_lm h_lm dY_lm/d(unit vector).
// A warp takes kPoolGroupEnvs consecutive environments at a time and walks their
// neighbours as one list (lane i: neighbour i, i + 32, ...), so that short
// neighbour lists do not leave most lanes of a second pass idle; G of the group
// is staged in dynamic shared memory, [warp][environment][q][NLP].
template <int LMAX>
__global__ void __launch_bounds__(kPoolWarps * 32) pool_grad_kernel(const float* __restrict__ pos,
                                                                    const float* __restrict__ mu,
                                                                    const int64_t* __restrict__ offsets,
                                                                    int64_t n_env, float rc, int nmin, int nmax,
                                                                    int kf, const float* __restrict__ dA,
                                                                    float alpha, float* __restrict__ dpos) {
  constexpr int NL = (LMAX + 1) * (LMAX + 1);
  constexpr int NL4 = (NL + 3) / 4;  // 16-byte groups per row of G
  constexpr int NLP = 4 * NL4;       // row stride in shared memory
  extern __shared__ __align__(16) float pool_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const geo::Cut cut = geo::make_cut(rc);
  const float two_over_rc = 2.f / rc;
  const int nR = nmax - nmin + 1;
  const int K = nR * kf * NL;
  const int env_floats = nR * kf * NLP;
  float* const sGw = pool_smem + (size_t)warp * kPoolGroupEnvs * env_floats;
  const int64_t n_groups = (n_env + kPoolGroupEnvs - 1) / kPoolGroupEnvs;
  for (int64_t grp = blockIdx.x * (int64_t)kPoolWarps + warp; grp < n_groups; grp += (int64_t)gridDim.x * kPoolWarps) {
    const int64_t e0 = grp * kPoolGroupEnvs;
    const int ne = (int)(n_env - e0 < kPoolGroupEnvs ? n_env - e0 : kPoolGroupEnvs);
    __syncwarp();
    for (int b = 0; b < ne; ++b)
      for (int i = lane; i < K; i += 32) {
        const int row = i / NL;
        sGw[b * env_floats + row * NLP + (i - row * NL)] = dA[(e0 + b) * K + i];
      }
    __syncwarp();
    // neighbour offsets of the group (environments past the end repeat the last one)
    int64_t ob[kPoolGroupEnvs + 1];
#pragma unroll
    for (int b = 0; b <= kPoolGroupEnvs; ++b) ob[b] = offsets[e0 + (b < ne ? b : ne)];
    for (int64_t j = ob[0] + lane; j < ob[kPoolGroupEnvs]; j += 32) {
      int slot = 0;
#pragma unroll
      for (int b = 1; b < kPoolGroupEnvs; ++b) slot += j >= ob[b] ? 1 : 0;
      const float* const sG = sGw + slot * env_floats;
      const float x = pos[3 * j], y = pos[3 * j + 1], z = pos[3 * j + 2];
      const geo::Geo gm = geo::geometry(x, y, z, cut);
      if (!gm.ok) {
        dpos[3 * j] = 0.f;
        dpos[3 * j + 1] = 0.f;
        dpos[3 * j + 2] = 0.f;
        continue;
      }
      const float ir = gm.ir;
      const float xh = gm.xh, yh = gm.yh, u = gm.u, t = gm.t;
      const float w = gm.w;
      const float env2 = w * w, denv = -2.f * w / rc;
      float Tf[kPoolMaxF];
      feature_poly(kf > 1 ? mu[j] : 0.f, kf, Tf);
      float h[NL], hd[NL];
#pragma unroll
      for (int i = 0; i < NL; ++i) {
        h[i] = 0.f;
        hd[i] = 0.f;
      }
      // T_n(t) and T_n'(t) from n = 0 upwards; R_n = T_n env2, dR_n/dr = (2/rc) T_n' env2 + T_n denv.
      float T = 1.f, dT = 0.f, Tm1 = 0.f, dTm1 = 0.f;
      for (int n = 0; n <= nmax; ++n) {
        if (n >= nmin) {
          const float rn = T * env2, drn = dT * two_over_rc * env2 + T * denv;
          const float4* row = reinterpret_cast<const float4*>(sG + (n - nmin) * kf * NLP);
#pragma unroll
          for (int q = 0; q < NL4; ++q) {
            float4 v = row[q];
            if (kf > 1) {  // sum the feature degrees with weights T_k(mu_j)
#pragma unroll
              for (int k = 1; k < kPoolMaxF; ++k)
                if (k < kf) {
                  const float4 vk = row[k * NL4 + q];
                  v.x = __fmaf_rn(vk.x, Tf[k], v.x);
                  v.y = __fmaf_rn(vk.y, Tf[k], v.y);
                  v.z = __fmaf_rn(vk.z, Tf[k], v.z);
                  v.w = __fmaf_rn(vk.w, Tf[k], v.w);
                }
            }
            const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int c = 0; c < 4; ++c)
              if (4 * q + c < NL) {
                h[4 * q + c] = __fmaf_rn(vv[c], rn, h[4 * q + c]);
                hd[4 * q + c] = __fmaf_rn(vv[c], drn, hd[4 * q + c]);
              }
          }
        }
        // advance: T_{n+1} = 2t T_n - T_{n-1} (T_1 = t), T'_{n+1} = 2 T_n + 2t T'_n - T'_{n-1}
        const float Tn = n == 0 ? t : 2.f * t * T - Tm1;
        const float dTn = n == 0 ? 1.f : 2.f * T + 2.f * t * dT - dTm1;
        Tm1 = T;
        T = Tn;
        dTm1 = dT;
        dT = dTn;
      }
      float Q[kPoolQ];
      legendre_q<LMAX>(u, Q);
      float gx = 0.f, gy = 0.f, gz = 0.f, ys = 0.f;
      float C = 1.f, S = 0.f, Cp = 0.f, Sp = 0.f;  // (x+iy)^m and (x+iy)^(m-1)
#pragma unroll
      for (int m = 0; m <= LMAX; ++m) {
#pragma unroll
        for (int l = m; l <= LMAX; ++l) {
          const float kq = c_norm[l][m] * Q[qidx(l, m)];
          const float kq1 = (m + 1 <= l) ? c_norm[l][m] * Q[qidx(l, m + 1)] : 0.f;
          const int base = l * l + l;
          if (m == 0) {
            ys = __fmaf_rn(hd[base], kq, ys);
            gz = __fmaf_rn(h[base], kq1, gz);
          } else {
            const float fm = (float)m;
            const float h1 = h[base + m], hd1 = hd[base + m], h2 = h[base - m], hd2 = hd[base - m];
            // cos part
            ys = __fmaf_rn(hd1, kq * C, ys);
            gx = __fmaf_rn(h1, kq * fm * Cp, gx);
            gy = __fmaf_rn(h1, -kq * fm * Sp, gy);
            gz = __fmaf_rn(h1, kq1 * C, gz);
            // sin part
            ys = __fmaf_rn(hd2, kq * S, ys);
            gx = __fmaf_rn(h2, kq * fm * Sp, gx);
            gy = __fmaf_rn(h2, kq * fm * Cp, gy);
            gz = __fmaf_rn(h2, kq1 * S, gz);
          }
        }
        Cp = C;
        Sp = S;
        const float Cn = C * xh - S * yh;
        S = S * xh + C * yh;
        C = Cn;
      }
      const float rg = xh * gx + yh * gy + u * gz;
      dpos[3 * j] = alpha * (ys * xh + (gx - xh * rg) * ir);
      dpos[3 * j + 1] = alpha * (ys * yh + (gy - yh * rg) * ir);
      dpos[3 * j + 2] = alpha * (ys * u + (gz - u * rg) * ir);
    }
  }
}

// ---- fused forces pipeline ---------------------------------------------------------------

// Entries of the adjoint rows of the fused kernel, lmax 6, ordered by m groups: group A holds
// the (l, m) of m = 0, 1, 2 (29 entries, padded to 32), group B those of m = 3..6 (20); inside a
// group m ascending, l ascending, cos entry then sin entry.  A lane then holds the h sums of one
// group at a time (29 or 20 registers instead of 49) and reads the group with 16-byte loads.
constexpr int kFLmax = 6;
constexpr int kFGroupB = 32;   // first entry of group B
constexpr int kFRow = 52;      // entries per adjoint row (32 + 20)
constexpr int kFMaxR = 8;      // radial factors of the fused kernel (nmax - nmin + 1 <= 8)
constexpr int kFChunk = 32;      // neighbours staged per pooling warp per pass
constexpr int kFPoolWarps = 16;  // warps that pool (the others wait at the barrier)

__host__ __device__ constexpr int fgroup_size(int m0, int m1) {
  int n = 0;
  for (int m = m0; m <= m1; ++m) n += m == 0 ? kFLmax + 1 : 2 * (kFLmax + 1 - m);
  return n;
}
// position of (l, m, sin?) inside the group that starts at m0
__host__ __device__ constexpr int fgroup_pos(int m0, int m, int l, int sn) {
  return fgroup_size(m0, m - 1) + (m == 0 ? l : 2 * (l - m) + sn);
}

__constant__ int c_fperm[kFRow];  // adjoint-row entry -> lm = l^2 + l + m (or -1: padding)

// Part of the pooling adjoint of one neighbour from the m group [M0, M1] of its environment's
// adjoint rows (row n - nmin at rows + (n - nmin) kFRow + goff).  PASS 0 sums h = sum_n G_n R_n(r)
// and contracts it with the gradient of Y in the unit vector into (gx, gy, gz); PASS 1 sums
// hd = sum_n G_n dR_n/dr and contracts it with Y into ys.  The columns Q_l^m, Q_l^{m+1} of
// d^m P_l/du^m follow their recurrence in l inside the contraction.
template <int PASS, int M0, int M1>
__device__ __forceinline__ void adjoint_group(const float* __restrict__ rows, int goff, int nmin, int nmax,
                                              float t, float env2, float denv, float two_over_rc, float u, float xh,
                                              float yh, float& gx, float& gy, float& gz, float& ys) {
  constexpr int NH = fgroup_size(M0, M1);
  constexpr int NH4 = (NH + 3) / 4;
  float h[NH];
#pragma unroll
  for (int i = 0; i < NH; ++i) h[i] = 0.f;
  float T = 1.f, dT = 0.f, Tm1 = 0.f, dTm1 = 0.f;
  for (int n = 0; n <= nmax; ++n) {
    if (n >= nmin) {
      const float wn = PASS == 0 ? T * env2 : dT * two_over_rc * env2 + T * denv;
      const float4* row = reinterpret_cast<const float4*>(rows + (n - nmin) * kFRow + goff);
#pragma unroll
      for (int q = 0; q < NH4; ++q) {
        const float4 v = row[q];
        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (4 * q + c < NH) h[4 * q + c] = __fmaf_rn(vv[c], wn, h[4 * q + c]);
      }
    }
    const float Tn = n == 0 ? t : 2.f * t * T - Tm1;
    const float dTn = n == 0 ? 1.f : 2.f * T + 2.f * t * dT - dTm1;
    Tm1 = T;
    T = Tn;
    dTm1 = dT;
    dT = dTn;
  }
  float C = 1.f, S = 0.f, Cp = 0.f, Sp = 0.f;  // (x+iy)^m and (x+iy)^(m-1)
#pragma unroll
  for (int m = 0; m <= M1; ++m) {
    if (m >= M0) {
      float q0m2 = 0.f, q0m1 = 0.f, q1m2 = 0.f, q1m1 = 0.f;  // Q_{l-2}, Q_{l-1} of columns m, m+1
#pragma unroll
      for (int l = m; l <= kFLmax; ++l) {
        float q0;
        if (l == m) q0 = c_dfac[m];
        else if (l == m + 1) q0 = (2 * m + 1) * u * q0m1;
        else q0 = c_ra[l][m] * u * q0m1 - c_rb[l][m] * q0m2;
        q0m2 = q0m1;
        q0m1 = q0;
        const float kq = c_norm[l][m] * q0;
        const int pc = fgroup_pos(M0, m, l, 0), ps = fgroup_pos(M0, m, l, 1);
        if constexpr (PASS == 1) {
          if (m == 0) {
            ys = __fmaf_rn(h[pc], kq, ys);
          } else {
            ys = __fmaf_rn(h[pc], kq * C, ys);
            ys = __fmaf_rn(h[ps], kq * S, ys);
          }
        } else {
          float q1 = 0.f;
          if (l >= m + 1) {
            if (l == m + 1) q1 = c_dfac[m + 1];
            else if (l == m + 2) q1 = (2 * m + 3) * u * q1m1;
            else q1 = c_ra[l][m + 1] * u * q1m1 - c_rb[l][m + 1] * q1m2;
            q1m2 = q1m1;
            q1m1 = q1;
          }
          const float kq1 = c_norm[l][m] * q1;
          if (m == 0) {
            gz = __fmaf_rn(h[pc], kq1, gz);
          } else {
            const float fm = (float)m;
            const float h1 = h[pc], h2 = h[ps];
            gx = __fmaf_rn(h1, kq * fm * Cp, gx);  // cos part
            gy = __fmaf_rn(h1, -kq * fm * Sp, gy);
            gz = __fmaf_rn(h1, kq1 * C, gz);
            gx = __fmaf_rn(h2, kq * fm * Sp, gx);  // sin part
            gy = __fmaf_rn(h2, kq * fm * Cp, gy);
            gz = __fmaf_rn(h2, kq1 * S, gz);
          }
        }
      }
    }
    Cp = C;
    Sp = S;
    const float Cn = C * xh - S * yh;
    S = S * xh + C * yh;
    C = Cn;
  }
}

// Slot of radial factor n of staged neighbour jj in a row of kFMaxR: the two 16-byte halves
// of a row swap for every other pair of neighbours (8 banks instead of 4 for the staging writes).
__device__ __forceinline__ int rslot8(int jj, int n) { return ((((n >> 2) ^ (jj >> 1)) & 1) << 2) | (n & 3); }

// Environment of neighbour j of the tile: the largest e with off[e] <= j (off: 33 offsets).
__device__ __forceinline__ int tile_env(const int64_t* off, int64_t j) {
  int lo = 0, hi = 32;
#pragma unroll
  for (int it = 0; it < 5; ++it) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= j) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Fused forces pipeline for one tile of 32 environments per CTA (no invariant features, lmax 6,
// at most 8 radial factors), 1024 threads:
//   1. pooling (Eq. 2) into the leaf rows of the one-environment-per-lane layout: the tile's
//      neighbours (contiguous in the CSR order) are cut into 16 equal ranges, one per pooling
//      warp; a warp stages 32 neighbours at a time (R_n, Y_lm in shared memory), sums them per
//      environment in registers and adds each environment's sums to its leaf rows (shared
//      atomics: a range can span several environments, an environment several ranges);
//   2.-4. the graph's forward levels, sink rows and reverse sweep (as loe_kernel, one stream per
//      warp);
//   5. phi, and the leaves' adjoints copied to rows [e][n][kFRow] in m-group order;
//   6. forces: one thread per (neighbour, m group) of the tile, each adding its part of the
//      pooling adjoint to the neighbour's force (zeroed at the start of the tile).
// A and dA stay in shared memory.  Scratch: the staging areas lie after the leaf rows (operand
// rows, adjoints, phi partials: unused until the forward levels); the adjoint rows go to the
// operand rows, dead after the reverse sweep; the tile's offsets follow the loe layout.  The
// host checks that all of it fits.
struct ForcesArgs {
  LoeArgs b;
  const float* pos;
  const int64_t* offsets;
  float rc;
  int32_t nmin, nmax;
  float* forces;
};

constexpr int kForcesThreads = 1024;
constexpr int kForcesOffBytes = 480;  // 33 int64 offsets (272 bytes), then the 52-entry row permutation

template <int RO>
__global__ void __launch_bounds__(kForcesThreads, 1) forces_fused_kernel(const ForcesArgs f) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int NT = kForcesThreads, NW = NT / 32, S = kLoeStride;
  constexpr int NL = (kFLmax + 1) * (kFLmax + 1);
  constexpr int NI = (NL + 31) / 32;
  static_assert(NW == kLoeStreamWarps, "one stream per warp");
  const LoeArgs& a = f.b;
  float* AA = reinterpret_cast<float*>(smem_raw);
  float* G = reinterpret_cast<float*>(smem_raw + align16((size_t)a.n_slots * S * 4));
  float* pb = G + align16((size_t)a.n_g * S * 4) / 4;
  Acc<float, RO>* red = reinterpret_cast<Acc<float, RO>*>(pb + 32);
  int64_t* soff = reinterpret_cast<int64_t*>(smem_raw + loe_smem_bytes(a.n_slots, a.n_g, true, NT));
  int* sperm = reinterpret_cast<int*>(soff + 34);  // c_fperm in shared memory (lanes read different entries)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid < kFRow) sperm[tid] = c_fperm[tid];
  const int K = a.K;
  const int nR = f.nmax - f.nmin + 1;
  float* scratch = AA + align16((size_t)K * S * 4) / 4;  // after the leaf rows, 16-byte aligned
  float* sR = scratch + (size_t)(warp % kFPoolWarps) * kFChunk * (kFMaxR + NL);
  float* sY = sR + kFChunk * kFMaxR;
  const geo::Cut cut = geo::make_cut(f.rc);
  const float two_over_rc = 2.f / f.rc;
  for (int64_t tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x) {
    const int64_t env0 = tile * 32;
    const int n_here = (a.n_env - env0) < 32 ? (int)(a.n_env - env0) : 32;
    if (tid <= 32) soff[tid] = f.offsets[env0 + (tid < n_here ? tid : n_here)];
    for (int i = tid; i < K * S; i += NT) AA[i] = 0.f;
    __syncthreads();
    const int64_t base = soff[0], N = soff[32] - base;
    // the forces of the tile's neighbours receive two partial sums each (step 6)
    for (int64_t i = tid; i < 3 * N; i += NT) f.forces[3 * base + i] = 0.f;
    // 1. pooling over warp ranges of the tile's neighbours
    if (warp < kFPoolWarps) {
      float acc[NI][kFMaxR];
#pragma unroll
      for (int i = 0; i < NI; ++i)
#pragma unroll
        for (int n = 0; n < kFMaxR; ++n) acc[i][n] = 0.f;
      int cur = -1;  // environment whose sums acc holds (warp-uniform)
      const int64_t lo = base + N * warp / kFPoolWarps, hi = base + N * (warp + 1) / kFPoolWarps;
      for (int64_t jb = lo; jb < hi; jb += kFChunk) {
        const int cnt = (int)((hi - jb) < kFChunk ? (hi - jb) : kFChunk);
        const int64_t j = jb + lane;
        int my_e = 0;
        if (lane < cnt) {
          my_e = tile_env(soff, j);
          const geo::Geo g = geo::geometry(f.pos[3 * j], f.pos[3 * j + 1], f.pos[3 * j + 2], cut);
          const float env2 = g.ok ? g.w * g.w : 0.f;
          float Tm1 = 1.f, T = g.t;
          for (int n = 1; n <= f.nmax; ++n) {
            if (n >= f.nmin) sR[lane * kFMaxR + rslot8(lane, n - f.nmin)] = T * env2;
            const float Tn = 2.f * g.t * T - Tm1;
            Tm1 = T;
            T = Tn;
          }
          if (f.nmin == 0) sR[lane * kFMaxR + rslot8(lane, 0)] = env2;
          float C = 1.f, Sn = 0.f;
#pragma unroll
          for (int m = 0; m <= kFLmax; ++m) {
            float qm2 = 0.f, qm1 = 0.f;
#pragma unroll
            for (int l = m; l <= kFLmax; ++l) {
              float q;
              if (l == m) q = c_dfac[m];
              else if (l == m + 1) q = (2 * m + 1) * g.u * qm1;
              else q = c_ra[l][m] * g.u * qm1 - c_rb[l][m] * qm2;
              qm2 = qm1;
              qm1 = q;
              const float kq = g.ok ? c_norm[l][m] * q : 0.f;
              if (m == 0) {
                sY[lane * NL + l * l + l] = kq;
              } else {
                sY[lane * NL + l * l + l + m] = kq * C;
                sY[lane * NL + l * l + l - m] = kq * Sn;
              }
            }
            const float Cn = C * g.xh - Sn * g.yh;
            Sn = Sn * g.xh + C * g.yh;
            C = Cn;
          }
        }
        __syncwarp();
        for (int jj = 0; jj < cnt; ++jj) {
          const int e = __shfl_sync(0xffffffffu, my_e, jj);
          if (e != cur) {
            if (cur >= 0) {
#pragma unroll
              for (int n = 0; n < kFMaxR; ++n)
#pragma unroll
                for (int i = 0; i < NI; ++i) {
                  const int lm = lane + 32 * i;
                  if (n < nR && lm < NL) atomicAdd(&AA[(n * NL + lm) * S + cur], acc[i][n]);
                  acc[i][n] = 0.f;
                }
            }
            cur = e;
          }
          float y[NI];
#pragma unroll
          for (int i = 0; i < NI; ++i) y[i] = (lane + 32 * i < NL) ? sY[jj * NL + lane + 32 * i] : 0.f;
#pragma unroll
          for (int q = 0; q < kFMaxR / 4; ++q) {
            const float4 rv = *reinterpret_cast<const float4*>(&sR[jj * kFMaxR + rslot8(jj, 4 * q)]);
            const float r4[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
              for (int i = 0; i < NI; ++i) acc[i][4 * q + c] = __fmaf_rn(r4[c], y[i], acc[i][4 * q + c]);
          }
        }
        __syncwarp();
      }
      if (cur >= 0) {
#pragma unroll
        for (int n = 0; n < kFMaxR; ++n)
#pragma unroll
          for (int i = 0; i < NI; ++i) {
            const int lm = lane + 32 * i;
            if (n < nR && lm < NL) atomicAdd(&AA[(n * NL + lm) * S + cur], acc[i][n]);
          }
      }
    }
    __syncthreads();
    for (int i = tid; i < a.n_g * S; i += NT) G[i] = 0.f;
    if (tid < 32) pb[tid] = tid < n_here ? 1.f : 0.f;  // phibar = 1: the forces of phi
    __syncthreads();
    // 2. operand nodes (Eq. 4), 3. sink rows of the warp's stream, 4. reverse sweep
    loe_forward_levels<S, NW>(a, AA, warp, lane);
    Acc<float, RO> phiacc;
    const float pbl = pb[lane];
    if (a.check)
      loe_tasks<true, RO, S, true>(a, AA, G, pbl, phiacc, warp, lane);
    else
      loe_tasks<true, RO, S, false>(a, AA, G, pbl, phiacc, warp, lane);
    __syncthreads();
    loe_reverse_levels<S, NW>(a, AA, G, warp, lane);
    // 5. phi, and the leaves' adjoints as rows [e][n][kFRow] in the operand rows
    red[warp * 32 + lane] = phiacc;
    float* rows = scratch;
    for (int r = warp; r < 32 * nR; r += NW) {  // row r = e nR + n, one warp per row
      const int e = r / nR, n = r - e * nR;
      for (int p = lane; p < kFRow; p += 32) {
        const int lm = sperm[p];
        rows[r * kFRow + p] = lm >= 0 ? G[(n * NL + lm) * S + e] : 0.f;
      }
    }
    __syncthreads();
    if (tid < 32 && tid < n_here && a.phi) {
      Acc<float, RO> s;
      for (int w = 0; w < NW; ++w) s.add_acc(red[w * 32 + tid]);
      a.phi[env0 + tid] = (float)s.value();
    }
    // 6. forces: items (neighbour, m group), group A of every neighbour first, so that a warp
    //    runs one group; each item adds its part of F_j (linear in the contractions) to F_j,
    //    zeroed above.  Two addends onto zero: the result does not depend on their order.
    for (int64_t t = tid; t < 2 * N; t += NT) {
      const bool gb = t >= N;
      const int64_t j = base + (gb ? t - N : t);
      const geo::Geo gm = geo::geometry(f.pos[3 * j], f.pos[3 * j + 1], f.pos[3 * j + 2], cut);
      if (!gm.ok) continue;
      const float* er = rows + (size_t)tile_env(soff, j) * nR * kFRow;
      const float env2 = gm.w * gm.w, denv = -2.f * gm.w / f.rc;
      float gx = 0.f, gy = 0.f, gz = 0.f, ys = 0.f;
      if (!gb) {
        adjoint_group<0, 0, 2>(er, 0, f.nmin, f.nmax, gm.t, env2, denv, two_over_rc, gm.u, gm.xh, gm.yh, gx, gy, gz,
                               ys);
        adjoint_group<1, 0, 2>(er, 0, f.nmin, f.nmax, gm.t, env2, denv, two_over_rc, gm.u, gm.xh, gm.yh, gx, gy, gz,
                               ys);
      } else {
        adjoint_group<0, 3, 6>(er, kFGroupB, f.nmin, f.nmax, gm.t, env2, denv, two_over_rc, gm.u, gm.xh, gm.yh, gx,
                               gy, gz, ys);
        adjoint_group<1, 3, 6>(er, kFGroupB, f.nmin, f.nmax, gm.t, env2, denv, two_over_rc, gm.u, gm.xh, gm.yh, gx,
                               gy, gz, ys);
      }
      const float rg = gm.xh * gx + gm.yh * gy + gm.u * gz;
      atomicAdd(&f.forces[3 * j], -(ys * gm.xh + (gx - gm.xh * rg) * gm.ir));
      atomicAdd(&f.forces[3 * j + 1], -(ys * gm.yh + (gy - gm.yh * rg) * gm.ir));
      atomicAdd(&f.forces[3 * j + 2], -(ys * gm.u + (gz - gm.u * rg) * gm.ir));
    }
    __syncthreads();
  }
}

}  // namespace dev

namespace {

bool g_pool_consts_ready = false;

cudaError_t ensure_pool_constants() {
  if (g_pool_consts_ready) return cudaSuccess;
  float norm[dev::kPoolLmax + 1][dev::kPoolLmax + 1] = {};
  float ra[dev::kPoolLmax + 1][dev::kPoolLmax + 1] = {};
  float rb[dev::kPoolLmax + 1][dev::kPoolLmax + 1] = {};
  float dfac[dev::kPoolLmax + 2] = {};
  const double pi = 3.14159265358979323846;
  for (int l = 0; l <= dev::kPoolLmax; ++l)
    for (int m = 0; m <= l; ++m) {
      double ratio = 1.0;  // (l-m)!/(l+m)!
      for (int i = l - m + 1; i <= l + m; ++i) ratio /= (double)i;
      double N = std::sqrt((2.0 * l + 1.0) / (4.0 * pi) * ratio);
      norm[l][m] = (float)(m == 0 ? N : std::sqrt(2.0) * N);
      if (l > m) {
        ra[l][m] = (float)((2.0 * l - 1.0) / (double)(l - m));
        rb[l][m] = (float)((double)(l + m - 1) / (double)(l - m));
      }
    }
  double df = 1.0;
  for (int m = 0; m <= dev::kPoolLmax + 1; ++m) {
    if (m > 0) df *= (2.0 * m - 1.0);
    dfac[m] = (float)df;
  }
  cudaError_t e;
  if ((e = cudaMemcpyToSymbol(dev::c_norm, norm, sizeof(norm))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(dev::c_ra, ra, sizeof(ra))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(dev::c_rb, rb, sizeof(rb))) != cudaSuccess) return e;
  if ((e = cudaMemcpyToSymbol(dev::c_dfac, dfac, sizeof(dfac))) != cudaSuccess) return e;
  int fperm[dev::kFRow];
  for (int p = 0; p < dev::kFRow; ++p) fperm[p] = -1;
  for (int m = 0; m <= dev::kFLmax; ++m)
    for (int l = m; l <= dev::kFLmax; ++l) {
      const int m0 = m < 3 ? 0 : 3, goff = m < 3 ? 0 : dev::kFGroupB;
      fperm[goff + dev::fgroup_pos(m0, m, l, 0)] = l * l + l + m;
      if (m > 0) fperm[goff + dev::fgroup_pos(m0, m, l, 1)] = l * l + l - m;
    }
  if ((e = cudaMemcpyToSymbol(dev::c_fperm, fperm, sizeof(fperm))) != cudaSuccess) return e;
  g_pool_consts_ready = true;
  return cudaSuccess;
}

// CTAs for n_groups warp work items (environments, or groups of them): at most as many as are
// resident at once (kernel's occupancy with smem bytes of shared memory), so that no partial
// second wave of CTAs leaves SMs idle; the warps take their items round-robin.
int pool_grid(int64_t n_groups, const void* kernel, size_t smem) {
  int dev_id = 0, sms = 148, bps = 0;
  cudaGetDevice(&dev_id);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kernel, dev::kPoolWarps * 32, smem) != cudaSuccess || bps < 1)
    bps = 1;
  int64_t need = (n_groups + dev::kPoolWarps - 1) / dev::kPoolWarps;
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * bps));
}

}  // namespace

namespace {

template <int LMAX>
cudaError_t launch_pool_l(cudaStream_t st, const float* pos, const float* mu, const int64_t* offsets, int64_t n_env,
                          float rc, int nmin, int nmax, int kf, float* A) {
  const int grid = pool_grid(n_env, (const void*)&dev::pool_kernel<LMAX>, 0);
  dev::pool_kernel<LMAX><<<grid, dev::kPoolWarps * 32, 0, st>>>(pos, mu, offsets, n_env, rc, nmin, nmax, kf, A);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pool(const float* pos, const float* mu, const int64_t* offsets, int64_t n_env, float rc, int nmin,
                        int nmax, int lmax, int kmax, float* A, cudaStream_t st) {
  cudaError_t e = ensure_pool_constants();
  if (e != cudaSuccess) return e;
  const int kf = kmax + 1;
  switch (lmax) {
    case 0: return launch_pool_l<0>(st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, A);
    case 1: return launch_pool_l<1>(st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, A);
    case 2: return launch_pool_l<2>(st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, A);
    case 3: return launch_pool_l<3>(st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, A);
    case 4: return launch_pool_l<4>(st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, A);
    case 5: return launch_pool_l<5>(st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, A);
    case 6: return launch_pool_l<6>(st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, A);
    case 7: return launch_pool_l<7>(st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, A);
    case 8: return launch_pool_l<8>(st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, A);
    default: return cudaErrorInvalidValue;
  }
}

namespace {

// The adjoint kernel for one lmax: its shared memory (G of kPoolGroupEnvs environments
// per warp) can pass the 48 KB default (16 radial x feature rows at lmax 8 take 86 KB).
template <int LMAX>
cudaError_t launch_pool_grad_l(int64_t n_groups, size_t smem, cudaStream_t st, const float* pos, const float* mu,
                               const int64_t* offsets, int64_t n_env, float rc, int nmin, int nmax, int kf,
                               const float* dA, float alpha, float* dpos) {
  if (smem > 48 * 1024) {  // a per-device attribute: set on every such launch
    const cudaError_t e =
        cudaFuncSetAttribute(dev::pool_grad_kernel<LMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int grid = pool_grid(n_groups, (const void*)&dev::pool_grad_kernel<LMAX>, smem);
  dev::pool_grad_kernel<LMAX><<<grid, dev::kPoolWarps * 32, smem, st>>>(pos, mu, offsets, n_env, rc, nmin, nmax, kf,
                                                                         dA, alpha, dpos);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pool_grad(const float* pos, const float* mu, const int64_t* offsets, int64_t n_env, float rc,
                             int nmin, int nmax, int lmax, int kmax, const float* dA, float alpha, float* dpos,
                             cudaStream_t st) {
  cudaError_t e = ensure_pool_constants();
  if (e != cudaSuccess) return e;
  const int kf = kmax + 1;
  const int64_t n_groups = (n_env + dev::kPoolGroupEnvs - 1) / dev::kPoolGroupEnvs;
  const int NLP = 4 * (((lmax + 1) * (lmax + 1) + 3) / 4);
  const size_t smem = (size_t)dev::kPoolWarps * dev::kPoolGroupEnvs * (nmax - nmin + 1) * kf * NLP * sizeof(float);
  switch (lmax) {
    case 0: return launch_pool_grad_l<0>(n_groups, smem, st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, dA, alpha, dpos);
    case 1: return launch_pool_grad_l<1>(n_groups, smem, st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, dA, alpha, dpos);
    case 2: return launch_pool_grad_l<2>(n_groups, smem, st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, dA, alpha, dpos);
    case 3: return launch_pool_grad_l<3>(n_groups, smem, st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, dA, alpha, dpos);
    case 4: return launch_pool_grad_l<4>(n_groups, smem, st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, dA, alpha, dpos);
    case 5: return launch_pool_grad_l<5>(n_groups, smem, st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, dA, alpha, dpos);
    case 6: return launch_pool_grad_l<6>(n_groups, smem, st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, dA, alpha, dpos);
    case 7: return launch_pool_grad_l<7>(n_groups, smem, st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, dA, alpha, dpos);
    case 8: return launch_pool_grad_l<8>(n_groups, smem, st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, dA, alpha, dpos);
    default: return cudaErrorInvalidValue;
  }
}

// Shared memory of the fused forces kernel and whether its scratch areas fit (see
// forces_fused_kernel): 0 when the request cannot take the fused kernel.
size_t forces_fused_smem(int n_slots, int n_g, int K, int nmin, int nmax, int lmax, int kmax) {
  static_assert(dev::fgroup_size(0, 2) <= dev::kFGroupB && dev::kFGroupB + dev::fgroup_size(3, 6) == dev::kFRow,
                "adjoint row layout");
  if (kmax != 0 || lmax != dev::kFLmax || nmin < 0 || nmax < nmin || nmax - nmin + 1 > dev::kFMaxR) return 0;
  const size_t S = dev::kLoeStride, NL = (size_t)(lmax + 1) * (lmax + 1);
  const size_t nR = (size_t)(nmax - nmin + 1);
  if ((size_t)K != nR * NL) return 0;
  // the staging areas start at the first 16-byte boundary after the leaf rows and must end before
  // the tile's offsets; the adjoint rows must end before the adjoint accumulators G (they are
  // written while G is read)
  const size_t total = dev::loe_smem_bytes(n_slots, n_g, true, dev::kForcesThreads);
  const size_t leaves = dev::align16((size_t)K * S * 4), operands_end = dev::align16((size_t)n_slots * S * 4);
  const size_t staging = (size_t)dev::kFPoolWarps * dev::kFChunk * (dev::kFMaxR + NL) * 4;
  const size_t rows = 32 * nR * dev::kFRow * 4;
  if (leaves + staging > total || leaves + rows > operands_end) return 0;
  return total + dev::kForcesOffBytes;
}

cudaError_t launch_forces_fused(const dev::LoeArgs& b, const float* pos, const int64_t* offsets, float rc, int nmin,
                                int nmax, int lmax, int readout, float* forces, int grid, size_t smem,
                                cudaStream_t st) {
  cudaError_t e = ensure_pool_constants();
  if (e != cudaSuccess) return e;
  const void* k = nullptr;
  if (lmax == dev::kFLmax && nmax - nmin + 1 <= dev::kFMaxR) {
    if (readout == 0) k = (const void*)&dev::forces_fused_kernel<0>;
    if (readout == 1) k = (const void*)&dev::forces_fused_kernel<1>;
    if (readout == 2) k = (const void*)&dev::forces_fused_kernel<2>;
  }
  if (!k) return cudaErrorInvalidValue;
  if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess) return e;
  dev::ForcesArgs f;
  f.b = b;
  f.pos = pos;
  f.offsets = offsets;
  f.rc = rc;
  f.nmin = nmin;
  f.nmax = nmax;
  f.forces = forces;
  void* args[] = {&f};
  return cudaLaunchKernel(k, dim3((unsigned)grid), dim3(dev::kForcesThreads), args, smem, st);
}

}  // namespace ace
