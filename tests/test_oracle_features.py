"""Oracle pins for invariant features (section "Invariant features": phi_nlmk = R_n Y_l^m T_k(mu),
degree l + n + k): the feature-free case, brute force on a tiny set, the Chebyshev identity,
single-species factorisation, finite differences of the forces, and permutation invariance."""
import itertools

import numpy as np
import pytest

import workloads as W
from oracle.basis import index_set, o3_basis
from oracle.evaluate import grad_naive, phi_naive
from oracle.pooling import feature_poly, forces, pool_A


def test_kmax0_is_the_plain_o3_basis():
    a, b = o3_basis(1, 3, 2, 1, 2), o3_basis(1, 3, 2, 1, 2, kmax=0, wk=5)
    assert np.array_equal(a.labels, b.labels) and np.array_equal(a.deg, b.deg) and b.k is None
    rows = [(n, l, m) for n in range(1, 4) for l in range(3) for m in range(-l, l + 1)]
    assert np.array_equal(a.labels, np.array(rows))


def test_feature_ids_and_degrees():
    b = o3_basis(1, 2, 1, 1, 1, kmax=2, wk=1)
    assert b.K == 2 * 3 * 4
    for idx in range(b.K):       # id = ((n - nmin)(kmax+1) + k)(lmax+1)^2 + l^2 + l + m
        n, l, m = b.labels[idx]
        k = b.k[idx]
        assert idx == ((n - 1) * 3 + k) * 4 + l * l + l + m
        assert b.deg[idx] == n + l + k and b.m[idx] == m and b.l[idx] == l


def test_feature_index_set_brute_force():
    """All multisets of one-particle functions (n, k, l, m) with sum m = 0, sum l even, sum degree <= D."""
    nu_max, D = 3, 6
    b = o3_basis(1, 2, 1, 1, 1, kmax=1, wk=1)
    got = set(index_set(b, nu_max, D).as_tuples())
    want = set()
    for nu in range(1, nu_max + 1):
        for t in itertools.combinations_with_replacement(range(b.K), nu):
            if b.m[list(t)].sum() == 0 and b.l[list(t)].sum() % 2 == 0 and b.deg[list(t)].sum() <= D:
                want.add(t)
    assert got == want and len(want) > 50


def test_chebyshev_feature_polynomials():
    th = np.linspace(0.0, np.pi, 17)
    T = feature_poly(np.cos(th), 3)
    for k in range(4):
        assert np.allclose(T[:, k], np.cos(k * th), atol=1e-14)


def test_single_species_factorises():
    """With one feature value mu for every neighbour, A_nlmk = T_k(mu) A_nlm."""
    offsets, P = W.draw_neighbours(5, rc=5.0, j_range=(3, 9))
    mu0 = 0.3
    A = pool_A(P, offsets, 1, 3, 2, 5.0)
    AF = pool_A(P, offsets, 1, 3, 2, 5.0, mu=np.full(P.shape[0], mu0), kmax=2).reshape(5, 3, 3, 9)
    T = [1.0, mu0, 2 * mu0 * mu0 - 1.0]
    for k in range(3):
        assert np.allclose(AF[:, :, k, :], T[k] * A.reshape(5, 3, 9), rtol=1e-13, atol=1e-14)


@pytest.fixture(scope="module")
def tiny():
    w = W.workload("species_forces_k375", nmax=2, lmax=2, deg_max=5, nu_max=3)
    b = o3_basis(w.nmin, w.nmax, w.lmax, w.wn, w.wl, w.kmax, w.wk)
    o = index_set(b, w.nu_max, w.deg_max)
    offsets, P = W.draw_neighbours(3, rc=w.rc, j_range=(4, 7))
    mu = W.draw_species(P.shape[0], w.n_species)
    c = W.draw_c(o.deg, 1)
    return w, o, offsets, P, mu, c


def test_feature_forces_finite_differences(tiny):
    w, o, offsets, P, mu, c = tiny
    args = (w.nmin, w.nmax, w.lmax, w.rc)

    def energy(Q):
        return phi_naive(pool_A(Q, offsets, *args, mu=mu, kmax=w.kmax), o, c).sum()

    A = pool_A(P, offsets, *args, mu=mu, kmax=w.kmax)
    F = forces(P, offsets, grad_naive(A, o, c), *args, mu=mu, kmax=w.kmax)
    h = 1e-6
    for j in range(0, P.shape[0], 3):
        for d in range(3):
            Pp, Pm = P.copy(), P.copy()
            Pp[j, d] += h
            Pm[j, d] -= h
            fd = -(energy(Pp) - energy(Pm)) / (2 * h)
            assert abs(F[j, d] - fd) <= 1e-7 * max(1.0, abs(fd))


def test_feature_permutation_invariance(tiny):
    """Permuting the neighbours of an environment together with their features leaves phi unchanged."""
    w, o, offsets, P, mu, c = tiny
    args = (w.nmin, w.nmax, w.lmax, w.rc)
    perm = np.arange(P.shape[0])
    for e in range(len(offsets) - 1):
        a, b = offsets[e], offsets[e + 1]
        perm[a:b] = a + np.random.default_rng(e).permutation(b - a)
    p1 = phi_naive(pool_A(P, offsets, *args, mu=mu, kmax=w.kmax), o, c)
    p2 = phi_naive(pool_A(P[perm], offsets, *args, mu=mu[perm], kmax=w.kmax), o, c)
    assert np.allclose(p1, p2, rtol=1e-12, atol=1e-14)
    # and a species relabelling that is not a permutation changes it
    p3 = phi_naive(pool_A(P, offsets, *args, mu=-mu, kmax=w.kmax), o, c)
    assert not np.allclose(p1, p3)
