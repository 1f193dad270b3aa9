"""Pins for the oracle's index set (sections 2.2-2.5, Eq. 3) against brute force and the paper's counts."""
from itertools import product

import numpy as np
import pytest

from oracle.basis import index_set, o3_basis, so2_basis, torus_basis, workload_index_set
from tests.paper_formulas import k_torus
import workloads as W


def brute_force(basis, nu_max, D, l_even, p=1):
    """Every ordered nu-tuple over [0, K)^nu, filtered, sorted and de-duplicated."""
    out = []
    for nu in range(1, nu_max + 1):
        seen = set()
        for t in product(range(basis.K), repeat=nu):
            d = [int(basis.deg[k]) for k in t]
            if p == 1:
                ok_d = sum(d) <= D
            elif p == np.inf:
                ok_d = max(d) <= D
            else:
                ok_d = sum(x ** p for x in d) <= D ** p + 1e-9
            if not ok_d or sum(int(basis.m[k]) for k in t) != 0:
                continue
            if l_even and sum(int(basis.l[k]) for k in t) % 2:
                continue
            seen.add(tuple(sorted(t)))
        out += sorted(seen)
    return out


def test_o3_brute_force_small():
    b = o3_basis(1, 3, 2, 1, 2)
    s = index_set(b, 3, 9)
    assert s.as_tuples() == brute_force(b, 3, 9, True)


def test_o3_brute_force_paper_degree():
    b = o3_basis(1, 2, 2, 1, 1)           # the paper's n + l degree
    s = index_set(b, 3, 6)
    assert s.as_tuples() == brute_force(b, 3, 6, True)


@pytest.mark.parametrize("p", [2, np.inf])
def test_o3_brute_force_other_norms(p):
    b = o3_basis(1, 2, 2, 1, 1)
    s = index_set(b, 3, 4, p=p)
    assert s.as_tuples() == brute_force(b, 3, 4, True, p=p)


def test_so2_brute_force():
    b = so2_basis(1, 2, 3)
    s = index_set(b, 3, 6)
    assert s.as_tuples() == brute_force(b, 3, 6, False)


def test_plain_fp64_k64_counts():
    """K = 64, nu <= 3, D = 10: brute force gives 8, 50, 64 tuples of order 1, 2, 3."""
    w = W.WORKLOADS["plain_fp64_k64"]
    s = workload_index_set(w)
    assert s.basis.K == 64
    assert s.counts_per_nu() == [8, 50, 64]
    assert s.as_tuples() == brute_force(s.basis, 3, 10, True)


@pytest.mark.parametrize("nu,D", [(2, 6), (3, 8), (4, 10), (5, 12), (6, 12)])
def test_torus_counts_closed_form(nu, D):
    """#K_T(nu, D) = 1 + sum_h sum_k #E_T(k, h) (section 5.2) for every order up to nu."""
    s = index_set(torus_basis(D), nu, D)
    assert s.counts_per_nu() == [k_torus(v, D) for v in range(1, nu + 1)]


def test_basis_invariance_and_order():
    s = workload_index_set(W.WORKLOADS["fwd_grad_k392"])
    b = s.basis
    for row, nu in zip(s.tuples, s.nu):
        t = row[:nu]
        assert np.all(np.diff(t) >= 0)
        assert b.m[t].sum() == 0 and b.l[t].sum() % 2 == 0
        assert b.deg[t].sum() <= 16
    keys = [(int(n),) + tuple(int(x) for x in r[:n]) for r, n in zip(s.tuples, s.nu)]
    assert keys == sorted(keys)            # canonical order (nu, lexicographic)


def test_one_particle_ids():
    b = o3_basis(1, 4, 3, 1, 2)
    for k, (n, l, m) in enumerate(b.labels):
        assert k == (n - 1) * 16 + l * l + l + m
        assert b.deg[k] == n + 2 * l


@pytest.mark.parametrize("make,nu,D", [
    (lambda: o3_basis(1, 4, 3, 1, 2), 3, 10),
    (lambda: o3_basis(1, 8, 6, 1, 2), 4, 16),
    (lambda: o3_basis(1, 3, 2, 1, 1, 2, 1), 4, 7),
    (lambda: o3_basis(1, 6, 5, 1, 1), 5, 12),
    (lambda: so2_basis(1, 3, 4), 4, 8),
    (lambda: torus_basis(10), 5, 10),
])
def test_blockwise_enumeration_equals_index_set(make, nu, D):
    """index_set_by_first (one block per first element, for the multi-million sets) is index_set, p = 1."""
    from oracle.basis import index_set_by_first
    b = make()
    a, c = index_set(b, nu, D), index_set_by_first(b, nu, D)
    assert np.array_equal(a.tuples, c.tuples) and np.array_equal(a.nu, c.nu) and np.array_equal(a.deg, c.deg)
