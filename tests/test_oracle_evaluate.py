"""Pins for the oracle's phi, dphi/dA and recursive evaluation (Eq. 1, Eq. 2, Eq. 4).

Brute force over unordered tuples, closed forms at special inputs, homogeneity,
Euler's identity for the gradient and central finite differences.
"""
from itertools import product
from math import factorial
from collections import Counter

import numpy as np
import pytest

from oracle.basis import index_set, o3_basis, workload_index_set
from oracle.dag import build_dag
from oracle.evaluate import (dag_forward, dag_reverse, error_scale, grad_naive, phi_naive,
                             phi_per_order)
import workloads as W


@pytest.fixture(scope="module")
def small():
    w = W.WORKLOADS["plain_fp64_k64"]
    s = workload_index_set(w)
    A = W.draw_A(6, s.basis.K)
    c = W.draw_c(s.deg, 2)
    return s, A, c


def test_brute_force_over_ordered_tuples(small):
    """phi = sum over ordered tuples of c_{sort(k)} prod A / (number of orderings of sort(k))."""
    s, A, c = small
    coef = {t: c[i] for i, t in enumerate(s.as_tuples())}
    K = s.basis.K
    phi = np.zeros((A.shape[0], c.shape[1]))
    for nu in range(1, s.nu_max + 1):
        for t in product(range(K), repeat=nu):
            key = tuple(sorted(t))
            if key not in coef:
                continue
            mult = Counter(key)
            n_orderings = factorial(nu)
            for v in mult.values():
                n_orderings //= factorial(v)
            phi += np.prod(A[:, list(t)], axis=1)[:, None] * coef[key][None, :] / n_orderings
    ref = phi_naive(A, s, c)
    assert np.allclose(phi, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_special_inputs(small):
    """phi(A = 1) = sum_k c_k; phi(A = 0) = 0; single non-zero A_j = a gives sum_{k = (j,...,j)} c_k a^nu."""
    s, _, c = small
    K = s.basis.K
    assert np.allclose(phi_naive(np.ones((1, K)), s, c)[0], c.sum(axis=0), rtol=1e-13)
    assert np.all(phi_naive(np.zeros((1, K)), s, c) == 0.0)
    tuples = s.as_tuples()
    for j in (0, 5, 17):
        a = 1.7
        A = np.zeros((1, K))
        A[0, j] = a
        expect = sum(c[i] * a ** len(t) for i, t in enumerate(tuples) if set(t) == {j})
        expect = np.zeros(c.shape[1]) + expect
        assert np.allclose(phi_naive(A, s, c)[0], expect, rtol=1e-13, atol=1e-15)


def test_homogeneity_per_order(small):
    """phi_nu(lambda A) = lambda^nu phi_nu(A) for each correlation order nu."""
    s, A, c = small
    lam = 1.37
    p1 = phi_per_order(A, s, c)
    p2 = phi_per_order(lam * A, s, c)
    for v in range(s.nu_max):
        assert np.allclose(p2[v], lam ** (v + 1) * p1[v], rtol=1e-12, atol=1e-14)
    assert np.allclose(p1.sum(axis=0), phi_naive(A, s, c), rtol=1e-12)


@pytest.mark.parametrize("name,rule", [("plain_fp64_k64", "balanced"), ("fwd_grad_k392", "balanced"),
                                       ("fwd_grad_k392", "peel")])
def test_recursive_equals_naive(name, rule):
    """Evaluating the graph (Eq. 4) reaches the plain sum (Eq. 2) up to rounding."""
    w = W.WORKLOADS[name]
    s = workload_index_set(w)
    dag = build_dag(s, rule=rule)
    A = W.draw_A(8, s.basis.K)
    c = W.draw_c(s.deg, 3)
    _, phi = dag_forward(dag, A, c)
    ref = phi_naive(A, s, c)
    scale = error_scale(A, s, c)
    assert np.max(np.abs(phi - ref) / scale) < 1e-13


def test_reverse_sweep_equals_product_rule():
    w = W.WORKLOADS["fwd_grad_k392"]
    s = workload_index_set(w)
    dag = build_dag(s)
    A = W.draw_A(5, s.basis.K)
    c = W.draw_c(s.deg, 2)
    pb = np.random.default_rng(7).standard_normal((5, 2))
    AA, _ = dag_forward(dag, A, c)
    g1 = dag_reverse(dag, AA, c, pb)
    g2 = grad_naive(A, s, c, pb)
    assert np.allclose(g1, g2, rtol=1e-11, atol=1e-13 * np.abs(g2).max())


def test_euler_identity():
    """sum_k A_k dphi/dA_k = sum_nu nu phi_nu (Euler, each order homogeneous of degree nu)."""
    w = W.WORKLOADS["fwd_grad_k392"]
    s = workload_index_set(w)
    A = W.draw_A(4, s.basis.K)
    c = W.draw_c(s.deg, 1)
    g = grad_naive(A, s, c)
    lhs = (A * g).sum(axis=1)
    per = phi_per_order(A, s, c)[:, :, 0]
    rhs = sum((v + 1) * per[v] for v in range(s.nu_max))
    assert np.allclose(lhs, rhs, rtol=1e-11)


def test_finite_differences():
    """Central differences, h = 1e-6 in FP64, on a fixed random subset of (env, k)."""
    w = W.WORKLOADS["fwd_grad_k392"]
    s = workload_index_set(w)
    A = W.draw_A(3, s.basis.K)
    c = W.draw_c(s.deg, 1)
    g = grad_naive(A, s, c)
    rng = np.random.default_rng(4)
    h = 1e-6
    for _ in range(12):
        e, k = int(rng.integers(3)), int(rng.integers(s.basis.K))
        Ap, Am = A.copy(), A.copy()
        Ap[e, k] += h
        Am[e, k] -= h
        fd = (phi_naive(Ap[e:e + 1], s, c) - phi_naive(Am[e:e + 1], s, c))[0, 0] / (2 * h)
        assert abs(fd - g[e, k]) <= 1e-7 * max(1.0, abs(g[e, k]))


def test_planted_mistakes_are_caught():
    """A dropped term, a wrong index or a transposed operand each changes phi measurably."""
    b = o3_basis(1, 2, 2, 1, 2)
    s = index_set(b, 3, 9)
    A = W.draw_A(3, b.K)
    c = W.draw_c(s.deg, 1)
    ref = phi_naive(A, s, c)
    scale = error_scale(A, s, c)
    dropped = s.tuples.copy()
    bad = index_set(b, 3, 9)
    bad.tuples = dropped[1:]
    bad.nu = s.nu[1:]
    c2 = c[1:]
    assert np.max(np.abs(phi_naive(A, bad, c2) - ref) / scale) > 1e-6
    shifted = index_set(b, 3, 9)
    shifted.tuples = np.where(s.tuples >= 0, (s.tuples + 1) % b.K, -1)
    assert np.max(np.abs(phi_naive(A, shifted, c) - ref) / scale) > 1e-6
