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
  g_pool_consts_ready = true;
  return cudaSuccess;
}

// CTAs for n_groups warp work items (environments, or groups of them), at most 8 per SM.
int pool_grid(int64_t n_groups) {
  int dev_id = 0, sms = 148;
  cudaGetDevice(&dev_id);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id);
  int64_t need = (n_groups + dev::kPoolWarps - 1) / dev::kPoolWarps;
  return (int)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)sms * 8));
}

}  // namespace

#define ACE_POOL_DISPATCH(KERNEL, ...)                                                              \
  switch (lmax) {                                                                                   \
    case 0: dev::KERNEL<0><<<grid, dev::kPoolWarps * 32, 0, st>>>(__VA_ARGS__); break;              \
    case 1: dev::KERNEL<1><<<grid, dev::kPoolWarps * 32, 0, st>>>(__VA_ARGS__); break;              \
    case 2: dev::KERNEL<2><<<grid, dev::kPoolWarps * 32, 0, st>>>(__VA_ARGS__); break;              \
    case 3: dev::KERNEL<3><<<grid, dev::kPoolWarps * 32, 0, st>>>(__VA_ARGS__); break;              \
    case 4: dev::KERNEL<4><<<grid, dev::kPoolWarps * 32, 0, st>>>(__VA_ARGS__); break;              \
    case 5: dev::KERNEL<5><<<grid, dev::kPoolWarps * 32, 0, st>>>(__VA_ARGS__); break;              \
    case 6: dev::KERNEL<6><<<grid, dev::kPoolWarps * 32, 0, st>>>(__VA_ARGS__); break;              \
    case 7: dev::KERNEL<7><<<grid, dev::kPoolWarps * 32, 0, st>>>(__VA_ARGS__); break;              \
    case 8: dev::KERNEL<8><<<grid, dev::kPoolWarps * 32, 0, st>>>(__VA_ARGS__); break;              \
    default: return cudaErrorInvalidValue;                                                          \
  }

cudaError_t launch_pool(const float* pos, const float* mu, const int64_t* offsets, int64_t n_env, float rc, int nmin,
                        int nmax, int lmax, int kmax, float* A, cudaStream_t st) {
  cudaError_t e = ensure_pool_constants();
  if (e != cudaSuccess) return e;
  const int grid = pool_grid(n_env);
  const int kf = kmax + 1;
  ACE_POOL_DISPATCH(pool_kernel, pos, mu, offsets, n_env, rc, nmin, nmax, kf, A)
  return cudaGetLastError();
}

namespace {

// The adjoint kernel for one lmax: its shared memory (G of kPoolGroupEnvs environments
// per warp) can pass the 48 KB default (16 radial x feature rows at lmax 8 take 86 KB).
template <int LMAX>
cudaError_t launch_pool_grad_l(int grid, size_t smem, cudaStream_t st, const float* pos, const float* mu,
                               const int64_t* offsets, int64_t n_env, float rc, int nmin, int nmax, int kf,
                               const float* dA, float alpha, float* dpos) {
  if (smem > 48 * 1024) {  // a per-device attribute: set on every such launch
    const cudaError_t e =
        cudaFuncSetAttribute(dev::pool_grad_kernel<LMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
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
  const int grid = pool_grid(n_groups);
  const int NLP = 4 * (((lmax + 1) * (lmax + 1) + 3) / 4);
  const size_t smem = (size_t)dev::kPoolWarps * dev::kPoolGroupEnvs * (nmax - nmin + 1) * kf * NLP * sizeof(float);
  switch (lmax) {
    case 0: return launch_pool_grad_l<0>(grid, smem, st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, dA, alpha, dpos);
    case 1: return launch_pool_grad_l<1>(grid, smem, st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, dA, alpha, dpos);
    case 2: return launch_pool_grad_l<2>(grid, smem, st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, dA, alpha, dpos);
    case 3: return launch_pool_grad_l<3>(grid, smem, st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, dA, alpha, dpos);
    case 4: return launch_pool_grad_l<4>(grid, smem, st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, dA, alpha, dpos);
    case 5: return launch_pool_grad_l<5>(grid, smem, st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, dA, alpha, dpos);
    case 6: return launch_pool_grad_l<6>(grid, smem, st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, dA, alpha, dpos);
    case 7: return launch_pool_grad_l<7>(grid, smem, st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, dA, alpha, dpos);
    case 8: return launch_pool_grad_l<8>(grid, smem, st, pos, mu, offsets, n_env, rc, nmin, nmax, kf, dA, alpha, dpos);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ace
