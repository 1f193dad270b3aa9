"""Density projection A_nlm = sum_j R_n(r_j) Y_lm(r_j/|r_j|) and forces (oracle; test infrastructure only).

Paper passages followed:
  * Eq. 2 (section 2.1): A_k = sum_j phi_k(r_j), the pooling of a one-particle
    basis over the neighbours of an environment.
  * section 2.4: phi_nlm(r) = R_n(r) Y_l^m(r / |r|).
The paper fixes neither the radial basis nor a real form of Y_l^m; the workload
uses (readings, applied identically in the GPU path):
  * R_n(r) = T_n(2 r / rc - 1) (1 - r / rc)^2, T_n the Chebyshev polynomial of the
    first kind, n = nmin..nmax.
  * Real orthonormal spherical harmonics without the Condon-Shortley phase:
        Y_l0  = N_l0 P_l(z/r)
        Y_lm  = sqrt(2) N_lm P_l^m(z/r) cos(m phi)      (m > 0)
        Y_l-m = sqrt(2) N_lm P_l^m(z/r) sin(m phi)      (m > 0)
    with N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) and
    P_l^m(u) = (1 - u^2)^{m/2} d^m P_l/du^m.
    Since (1 - u^2)^{m/2} cos(m phi) = Re((x + i y)^m) / r^m (and Im for sin),
    Y_lm = sqrt(2) N_lm Q_lm(z/r) Re/Im((x+iy)^m) r^{-m} with Q_lm = d^m P_l/du^m;
    the gradient below differentiates exactly this product.
  * Cutoff: a neighbour at r >= rc (or at r = 0, where r/|r| is undefined) contributes
    nothing, and its force is zero.  The envelope (1 - r/rc)^2 has a double root at rc, so
    R_n and dR_n/dr both reach 0 there: the zero continuation is C^1 at the cutoff.
  * One-particle id = (n - nmin)(lmax+1)^2 + l^2 + (l + m).
  * Invariant features (section "Invariant features"): phi_nlmk(r, mu) =
    R_n(r) Y_l^m(r/|r|) T_k(mu), T_k the Chebyshev polynomial of the first kind
    (the paper only asks for a polynomial basis of degree k) of the neighbour's
    feature value mu in [-1, 1]; id = ((n - nmin)(kmax+1) + k)(lmax+1)^2 + l^2 + (l + m).
    The feature is a label of the neighbour, not a coordinate: forces are
    derivatives with respect to positions only.
Forces are F_j = -dphi/dr_j = -sum_k G_k grad(R_n Y_lm)(r_j) with G = dphi/dA.
"""
from __future__ import annotations

from math import factorial, pi, sqrt
import numpy as np
from numpy.polynomial import chebyshev as C
from numpy.polynomial import legendre as L


def lm_index(l: int, m: int) -> int:
    return l * l + l + m


def real_sph_harm(P: np.ndarray, lmax: int, with_grad: bool = False, bound: bool = False):
    """Y (n, (lmax+1)^2) at the directions of the rows of P (not necessarily unit), and dY/dP (n, L, 3).

    The value depends on the direction only, so the gradient is the gradient of
    Y(r / |r|) with respect to r.  With bound=True the gradient returned is the
    same expression with every product term replaced by its absolute value (an
    error scale for finite-precision evaluations, not a derivative).
    """
    P = np.asarray(P, dtype=np.float64)
    x, y, z = P[:, 0], P[:, 1], P[:, 2]
    r = np.sqrt(x * x + y * y + z * z)
    u = z / r
    w = x + 1j * y
    n = P.shape[0]
    nL = (lmax + 1) ** 2
    Y = np.zeros((n, nL))
    dY = np.zeros((n, nL, 3)) if with_grad else None
    rhat = P / r[:, None]
    grad_u = (np.array([0.0, 0.0, 1.0])[None, :] - u[:, None] * rhat) / r[:, None]
    for l in range(lmax + 1):
        Pl = np.zeros(l + 1)
        Pl[l] = 1.0                                  # Legendre series of P_l
        for m in range(0, l + 1):
            N = sqrt((2 * l + 1) / (4 * pi) * factorial(l - m) / factorial(l + m))
            Qc = L.legder(Pl, m) if m else Pl        # d^m P_l / du^m
            Q = L.legval(u, Qc)
            dQ = L.legval(u, L.legder(Qc, 1)) if l - m >= 1 else np.zeros(n)
            h = r ** (-m)
            grad_h = (-m) * r[:, None] ** (-m - 2) * P
            wm = w ** m
            wm1 = m * w ** (m - 1) if m >= 1 else np.zeros(n, complex)
            if m == 0:
                parts = [(0, N, np.ones(n), np.zeros((n, 3)))]
            else:
                s2 = sqrt(2.0) * N
                g_re = wm.real
                dg_re = np.stack([wm1.real, -wm1.imag, np.zeros(n)], axis=1)
                g_im = wm.imag
                dg_im = np.stack([wm1.imag, wm1.real, np.zeros(n)], axis=1)
                parts = [(m, s2, g_re, dg_re), (-m, s2, g_im, dg_im)]
            for mm, fac, g, dg in parts:
                idx = lm_index(l, mm)
                Y[:, idx] = fac * Q * g * h
                if with_grad and not bound:
                    dY[:, idx, :] = fac * (dQ[:, None] * grad_u * (g * h)[:, None]
                                           + Q[:, None] * dg * h[:, None]
                                           + (Q * g)[:, None] * grad_h)
                elif with_grad:
                    dY[:, idx, :] = fac * (np.abs(dQ[:, None] * grad_u * (g * h)[:, None])
                                           + np.abs(Q[:, None] * dg * h[:, None])
                                           + np.abs((Q * g)[:, None] * grad_h))
    return Y, dY


def radial(r: np.ndarray, nmin: int, nmax: int, rc: float, with_grad: bool = False, bound: bool = False):
    """R_n(r) = T_n(2r/rc - 1)(1 - r/rc)^2 for n = nmin..nmax, and dR_n/dr (or, with bound=True,
    the derivative's two product terms in absolute value)."""
    r = np.asarray(r, dtype=np.float64)
    x = 2.0 * r / rc - 1.0
    env = (1.0 - r / rc) ** 2
    denv = -2.0 * (1.0 - r / rc) / rc
    R = np.zeros((r.shape[0], nmax - nmin + 1))
    dR = np.zeros_like(R) if with_grad else None
    for i, nn in enumerate(range(nmin, nmax + 1)):
        coef = np.zeros(nn + 1)
        coef[nn] = 1.0
        T = C.chebval(x, coef)
        R[:, i] = T * env
        if with_grad:
            dT = C.chebval(x, C.chebder(coef))
            dR[:, i] = (np.abs(dT * (2.0 / rc) * env) + np.abs(T * denv)) if bound else \
                dT * (2.0 / rc) * env + T * denv
    return R, dR


def feature_poly(mu: np.ndarray, kmax: int) -> np.ndarray:
    """(n, kmax+1): T_k(mu_j), the Chebyshev polynomials of the first kind."""
    mu = np.asarray(mu, dtype=np.float64)
    out = np.zeros((mu.shape[0], kmax + 1))
    for k in range(kmax + 1):
        coef = np.zeros(k + 1)
        coef[k] = 1.0
        out[:, k] = C.chebval(mu, coef)
    return out


def _with_features(R, dR, mu, kmax):
    """Radial factors R_n -> R_n T_k(mu_j) in (n, k) order (and their r-derivatives)."""
    if mu is None:
        return R, dR
    T = feature_poly(mu, kmax)
    RF = (R[:, :, None] * T[:, None, :]).reshape(R.shape[0], -1)
    dRF = None if dR is None else (dR[:, :, None] * T[:, None, :]).reshape(R.shape[0], -1)
    return RF, dRF


def one_particle(P: np.ndarray, nmin: int, nmax: int, lmax: int, rc: float, with_grad: bool = False,
                 mu: np.ndarray | None = None, kmax: int = 0):
    """phi_k(r_j) for all neighbours j and one-particle ids k, and grad phi_k (n, K, 3).
    With mu (one feature value per neighbour) the ids include the feature degree k <= kmax."""
    P, inside = _inside(P, rc)
    r = np.linalg.norm(P, axis=1)
    Y, dY = real_sph_harm(P, lmax, with_grad)
    R, dR = radial(r, nmin, nmax, rc, with_grad)
    R, dR = _with_features(R, dR, mu, kmax)
    nR, nL = R.shape[1], Y.shape[1]
    phi = (R[:, :, None] * Y[:, None, :]).reshape(P.shape[0], nR * nL) * inside[:, None]
    if not with_grad:
        return phi, None
    rhat = P / r[:, None]
    g = (dR[:, :, None, None] * Y[:, None, :, None] * rhat[:, None, None, :]
         + R[:, :, None, None] * dY[:, None, :, :])
    return phi, g.reshape(P.shape[0], nR * nL, 3) * inside[:, None, None]


def _inside(P: np.ndarray, rc: float):
    """(P', inside): neighbours with 0 < r < rc; the others are replaced by a point inside the
    ball (their contributions are multiplied by inside = 0 afterwards)."""
    P = np.array(P, dtype=np.float64)
    r = np.linalg.norm(P, axis=1)
    inside = (r > 0.0) & (r < rc)
    P[~inside] = (0.5 * rc, 0.0, 0.0)
    return P, inside.astype(np.float64)


def one_particle_grad_bound(P: np.ndarray, nmin: int, nmax: int, lmax: int, rc: float,
                            mu: np.ndarray | None = None, kmax: int = 0) -> np.ndarray:
    """(n, K, 3): grad phi_k written as in ``one_particle`` with every product term in absolute value.

    Used as the scale of the force error: |F_hat - F| / sum_k |G_k| bound_k is the
    force analogue of |phi_hat - phi| / sum_k |c_k| |AA_k|.
    """
    P, inside = _inside(P, rc)
    r = np.linalg.norm(P, axis=1)
    Y, dYb = real_sph_harm(P, lmax, True, bound=True)
    R, dRb = radial(r, nmin, nmax, rc, True, bound=True)
    if mu is not None:
        T = np.abs(feature_poly(mu, kmax))
        R = (R[:, :, None] * T[:, None, :]).reshape(R.shape[0], -1)
        dRb = (dRb[:, :, None] * T[:, None, :]).reshape(dRb.shape[0], -1)
    rhat = np.abs(P / r[:, None])
    g = (dRb[:, :, None, None] * np.abs(Y)[:, None, :, None] * rhat[:, None, None, :]
         + np.abs(R)[:, :, None, None] * dYb[:, None, :, :])
    return g.reshape(P.shape[0], R.shape[1] * Y.shape[1], 3) * inside[:, None, None]


def pool_A(P: np.ndarray, offsets: np.ndarray, nmin: int, nmax: int, lmax: int, rc: float,
           mu: np.ndarray | None = None, kmax: int = 0) -> np.ndarray:
    """A[e, k] = sum over the neighbours j of environment e of phi_k(r_j) (Eq. 2)."""
    offsets = np.asarray(offsets, dtype=np.int64)
    phi, _ = one_particle(P, nmin, nmax, lmax, rc, mu=mu, kmax=kmax)
    A = np.zeros((offsets.shape[0] - 1, phi.shape[1]))
    for e in range(A.shape[0]):
        A[e] = phi[offsets[e]:offsets[e + 1]].sum(axis=0)
    return A


def forces(P: np.ndarray, offsets: np.ndarray, G: np.ndarray, nmin: int, nmax: int, lmax: int,
           rc: float, mu: np.ndarray | None = None, kmax: int = 0) -> np.ndarray:
    """F_j = -sum_k G[e(j), k] grad phi_k(r_j), with G = dphi/dA of the environment of j."""
    offsets = np.asarray(offsets, dtype=np.int64)
    _, g = one_particle(P, nmin, nmax, lmax, rc, with_grad=True, mu=mu, kmax=kmax)
    F = np.zeros((P.shape[0], 3))
    for e in range(offsets.shape[0] - 1):
        a, b = offsets[e], offsets[e + 1]
        F[a:b] = -np.einsum("k,jkd->jd", G[e], g[a:b])
    return F
