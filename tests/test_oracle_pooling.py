"""Pins for the oracle's one-particle basis R_n Y_lm, the pooling A_nlm and the forces.

Convention-free identities (addition theorem, orthonormality by exact
quadrature), scipy's complex harmonics, Chebyshev's closed form, finite
differences and neighbour-permutation invariance.
"""
from math import pi

import numpy as np
import pytest
import scipy.special as sps

from oracle.pooling import forces, lm_index, one_particle, pool_A, radial, real_sph_harm
from oracle.basis import o3_basis, index_set
from oracle.evaluate import grad_naive, phi_naive
import workloads as W

LMAX = 6


def unit(n, seed):
    d = np.random.default_rng(seed).standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1)[:, None]


def test_addition_theorem():
    """sum_m Y_lm(u)^2 = (2l + 1) / (4 pi) for every direction u."""
    Y, _ = real_sph_harm(unit(50, 1) * 2.3, LMAX)
    for l in range(LMAX + 1):
        s = sum(Y[:, lm_index(l, m)] ** 2 for m in range(-l, l + 1))
        assert np.allclose(s, (2 * l + 1) / (4 * pi), rtol=1e-12)


def test_orthonormality_by_quadrature():
    """Gauss-Legendre in cos(theta) x uniform phi grid integrates Y Y' exactly for l, l' <= 6."""
    nu, nphi = 16, 32
    x, wx = np.polynomial.legendre.leggauss(nu)
    phis = 2 * pi * np.arange(nphi) / nphi
    X, PH = np.meshgrid(x, phis, indexing="ij")
    st = np.sqrt(1 - X ** 2)
    P = np.stack([st * np.cos(PH), st * np.sin(PH), X], axis=-1).reshape(-1, 3)
    w = (wx[:, None] * np.full(nphi, 2 * pi / nphi)[None, :]).reshape(-1)
    Y, _ = real_sph_harm(P, LMAX)
    G = (Y * w[:, None]).T @ Y
    assert np.allclose(G, np.eye(G.shape[0]), atol=1e-12)


def test_against_scipy_complex_harmonics():
    """Ours (no Condon-Shortley phase): Y_lm = sqrt2 (-1)^m Re Y_l^m, Y_l-m = sqrt2 (-1)^m Im Y_l^m."""
    P = unit(40, 2) * 0.7
    Y, _ = real_sph_harm(P, LMAX)
    theta = np.arccos(np.clip(P[:, 2] / np.linalg.norm(P, axis=1), -1, 1))
    phi = np.arctan2(P[:, 1], P[:, 0])
    for l in range(LMAX + 1):
        ref0 = sps.sph_harm_y(l, 0, theta, phi)
        assert np.allclose(Y[:, lm_index(l, 0)], ref0.real, atol=1e-12)
        for m in range(1, l + 1):
            ref = sps.sph_harm_y(l, m, theta, phi)
            assert np.allclose(Y[:, lm_index(l, m)], np.sqrt(2) * (-1) ** m * ref.real, atol=1e-12)
            assert np.allclose(Y[:, lm_index(l, -m)], np.sqrt(2) * (-1) ** m * ref.imag, atol=1e-12)


def test_radial_chebyshev_closed_form():
    """T_n(cos t) = cos(n t): R_n(r) = cos(n t)(1 - r/rc)^2 with cos t = 2 r/rc - 1."""
    rc = 5.0
    r = np.linspace(0.01, 4.99, 37)
    R, _ = radial(r, 1, 8, rc)
    t = np.arccos(2 * r / rc - 1)
    for i, n in enumerate(range(1, 9)):
        assert np.allclose(R[:, i], np.cos(n * t) * (1 - r / rc) ** 2, atol=1e-13)


def test_gradients_by_finite_differences():
    rc, h = 5.0, 1e-6
    P = unit(7, 3) * np.random.default_rng(5).uniform(0.5, 4.5, 7)[:, None]
    phi0, g = one_particle(P, 1, 8, LMAX, rc, with_grad=True)
    for d in range(3):
        Pp, Pm = P.copy(), P.copy()
        Pp[:, d] += h
        Pm[:, d] -= h
        fd = (one_particle(Pp, 1, 8, LMAX, rc)[0] - one_particle(Pm, 1, 8, LMAX, rc)[0]) / (2 * h)
        assert np.allclose(fd, g[:, :, d], atol=2e-8)


def test_pooling_forces_permutation_and_fd():
    """A is invariant under permutation of neighbours, F permutes with them; F = -dphi/dr by FD."""
    rc = 5.0
    b = o3_basis(1, 3, 2, 1, 2)
    s = index_set(b, 3, 8)
    c = W.draw_c(s.deg, 1)
    offsets, P = W.draw_neighbours(3, rc=rc, j_range=(4, 7))
    A = pool_A(P, offsets, 1, 3, 2, rc)
    G = grad_naive(A, s, c)
    F = forces(P, offsets, G, 1, 3, 2, rc)
    perm = np.arange(P.shape[0])
    a, bb = offsets[1], offsets[2]
    perm[a:bb] = perm[a:bb][::-1]
    A2 = pool_A(P[perm], offsets, 1, 3, 2, rc)
    assert np.allclose(A2, A, rtol=1e-13, atol=1e-14)
    F2 = forces(P[perm], offsets, G, 1, 3, 2, rc)
    assert np.allclose(F2, F[perm], rtol=1e-12, atol=1e-14)
    h = 1e-6
    for j in (0, a + 1, P.shape[0] - 1):
        for d in range(3):
            Pp, Pm = P.copy(), P.copy()
            Pp[j, d] += h
            Pm[j, d] -= h
            fp = phi_naive(pool_A(Pp, offsets, 1, 3, 2, rc), s, c).sum()
            fm = phi_naive(pool_A(Pm, offsets, 1, 3, 2, rc), s, c).sum()
            assert abs(-(fp - fm) / (2 * h) - F[j, d]) < 1e-7 * max(1.0, abs(F[j, d]))


def test_gradient_bound_dominates_gradient():
    """The force error scale is at least the magnitude of the gradient it bounds, term by term."""
    from oracle.pooling import one_particle_grad_bound
    P = unit(9, 6) * np.random.default_rng(8).uniform(0.2, 4.9, 9)[:, None]
    _, g = one_particle(P, 1, 8, LMAX, 5.0, with_grad=True)
    b = one_particle_grad_bound(P, 1, 8, LMAX, 5.0)
    assert np.all(b >= np.abs(g) * (1 - 1e-12) - 1e-300)


# ---- the force-error scale, pinned from above: equal to |grad phi_k| where one product term is left ----

def _k(n, l, m, nmin=1, lmax=LMAX):
    return (n - nmin) * (lmax + 1) ** 2 + lm_index(l, m)


def test_gradient_bound_equals_gradient_where_one_term_is_left():
    """grad(R_n Y_lm) is a sum of product terms; where all but one vanish, the bound must equal |grad|.

    (a) l = 0 (Y constant) at a zero of T_n: only dT_n/dr (1 - r/rc)^2 Y rhat is left;
    (b) l = 0 at an interior extremum of T_n: only T_n d(1 - r/rc)^2/dr Y rhat;
    (c) z-component in the plane z = 0 (rhat_z = 0, and the r^-m factor has no z-derivative there);
    (d) sine parts (m < 0) on the x-axis, y-component; (e) cosine parts (m > 0) on the y-axis, x-component.
    """
    from oracle.pooling import one_particle_grad_bound
    rc, nmax = 5.0, 8
    d = unit(3, 11)
    for n in range(1, nmax + 1):
        xs = [np.cos((2 * k - 1) * pi / (2 * n)) for k in range(1, n + 1)]          # T_n = 0
        xs += [np.cos(k * pi / n) for k in range(1, n)]                            # T_n' = 0
        for x in xs:
            P = d * (rc * (x + 1) / 2)
            _, g = one_particle(P, 1, nmax, LMAX, rc, with_grad=True)
            b = one_particle_grad_bound(P, 1, nmax, LMAX, rc)
            k = _k(n, 0, 0)
            assert np.allclose(b[:, k], np.abs(g[:, k]), rtol=1e-12, atol=1e-15), (n, x)
    rng = np.random.default_rng(12)
    r = rng.uniform(0.3, 4.7, 6)
    phi = rng.uniform(0, 2 * pi, 6)
    planes = {"z": (np.stack([np.cos(phi), np.sin(phi), 0 * phi], 1) * r[:, None], 2, None),
              "x-axis": (np.stack([r, 0 * r, 0 * r], 1), 1, -1),
              "y-axis": (np.stack([0 * r, r, 0 * r], 1), 0, +1)}
    for name, (P, comp, sign) in planes.items():
        _, g = one_particle(P, 1, nmax, LMAX, rc, with_grad=True)
        b = one_particle_grad_bound(P, 1, nmax, LMAX, rc)
        ks = [_k(n, l, m) for n in range(1, nmax + 1) for l in range(LMAX + 1) for m in range(-l, l + 1)
              if sign is None or (m != 0 and np.sign(m) == sign)]
        gk, bk = np.abs(g[:, ks, comp]), b[:, ks, comp]
        assert np.allclose(bk, gk, rtol=1e-12, atol=1e-13), name
        assert np.mean(gk > 1e-6) > 0.2, name    # a fair share of the compared values is not zero


def test_harmonic_gradient_bound_r_power_term():
    """l = m: d^m P_m/du^m is constant, so the z-derivative of Y_mm has the r^-m term only."""
    P = unit(20, 13) * 1.7
    _, dY = real_sph_harm(P, LMAX, with_grad=True)
    _, dYb = real_sph_harm(P, LMAX, with_grad=True, bound=True)
    for m in range(1, LMAX + 1):
        for mm in (m, -m):
            i = lm_index(m, mm)
            assert np.allclose(dYb[:, i, 2], np.abs(dY[:, i, 2]), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("old,new", [
    ("(np.abs(dT * (2.0 / rc) * env) + np.abs(T * denv))", "(np.abs(dT * (4.0 / rc) * env) + np.abs(T * denv))"),
    ("(np.abs(dT * (2.0 / rc) * env) + np.abs(T * denv))", "(np.abs(dT * (2.0 / rc) * env) + 2 * np.abs(T * denv))"),
    ("+ np.abs(Q[:, None] * dg * h[:, None])", "+ 2 * np.abs(Q[:, None] * dg * h[:, None])"),
    ("+ np.abs((Q * g)[:, None] * grad_h))", "+ 2 * np.abs((Q * g)[:, None] * grad_h))"),
    ("fac * (np.abs(dQ[:, None]", "2 * fac * (np.abs(dQ[:, None]"),
    ("+ np.abs(R)[:, :, None, None] * dYb", "+ 2 * np.abs(R)[:, :, None, None] * dYb"),
])
def test_gradient_bound_pins_catch_planted_factors(old, new):
    """A stray factor in any term of the bound (plausible slips) fails one of the equalities above."""
    import inspect
    import sys
    import oracle.pooling as Pm
    src = inspect.getsource(Pm)
    assert src.count(old) == 1, old
    mod = type(Pm)("mutant_pooling")
    sys.modules["mutant_pooling"] = mod
    try:
        exec(compile(src.replace(old, new), "mutant_pooling", "exec"), mod.__dict__)
    finally:
        del sys.modules["mutant_pooling"]
    saved = {k: globals()[k] for k in ("one_particle", "real_sph_harm")}
    import oracle.pooling
    orig_bound = oracle.pooling.one_particle_grad_bound
    globals()["real_sph_harm"] = mod.real_sph_harm
    oracle.pooling.one_particle_grad_bound = mod.one_particle_grad_bound
    try:
        failed = 0
        for t in (test_gradient_bound_equals_gradient_where_one_term_is_left,
                  test_harmonic_gradient_bound_r_power_term):
            try:
                t()
            except AssertionError:
                failed += 1
        assert failed > 0, new
    finally:
        oracle.pooling.one_particle_grad_bound = orig_bound
        globals().update(saved)


def test_cutoff_zero_continuation_is_c1_and_drops_the_neighbour():
    """Neighbours at r >= rc or r = 0 contribute nothing.  The envelope's double root makes this the
    C^1 continuation: R_n = O(eps^2) and dR_n/dr = O(eps) at r = rc(1 - eps), so phi_k and grad phi_k
    of a neighbour just inside the cutoff are already within O(eps^2), O(eps) of the zero outside."""
    rc = 5.0
    for eps in (1e-2, 1e-3):
        R, dR = radial(np.array([rc * (1 - eps)]), 1, 8, rc, with_grad=True)
        assert np.all(np.abs(R) <= 1.01 * eps ** 2) and np.all(np.abs(dR) <= 2.01 * eps / rc * 8 ** 2)
        u = unit(1, 7)
        phi_in, g_in = one_particle(u * rc * (1 - eps), 1, 8, LMAX, rc, with_grad=True)
        assert np.abs(phi_in).max() <= 2 * eps ** 2 and np.abs(g_in).max() <= 200 * eps
    P = unit(5, 8) * np.array([1.0, 2.0, 4.0, 3.0, 2.5])[:, None]
    extra = np.concatenate([P, unit(2, 9) * np.array([[rc], [1.5 * rc]]), np.zeros((1, 3))])
    phi, g = one_particle(extra, 1, 8, LMAX, rc, with_grad=True)
    assert np.all(phi[5:] == 0.0) and np.all(g[5:] == 0.0)
    A = pool_A(P, np.array([0, 5]), 1, 8, LMAX, rc)
    A2 = pool_A(extra, np.array([0, 8]), 1, 8, LMAX, rc)
    assert np.array_equal(A, A2)
