"""Pins for the oracle's graph builder (sections 2.6, 3.2, 3.3) against the paper's worked examples and Theorem 3.2."""
import numpy as np
import pytest

from oracle.basis import index_set, torus_basis, workload_index_set
from oracle.dag import build_dag, decompositions, is_dependent
from tests.paper_formulas import aux_torus_alg1, catalan
import workloads as W


def torus_ids(ms, mmax):
    return tuple(sorted(m + mmax for m in ms))


def check_structure(dag, index):
    K = dag.K
    seen = set()
    basis = set(index.as_tuples())
    for i, t in enumerate(dag.tuples):
        assert t not in seen
        seen.add(t)
        if i < K:
            assert t == (i,) and dag.left[i] == -1
            continue
        l, r = dag.left[i], dag.right[i]
        assert 0 <= l < i and 0 <= r < i
        assert tuple(sorted(dag.tuples[l] + dag.tuples[r])) == t        # mset union, Eq. 4
        assert dag.is_aux[i] == (t not in basis)
    basis_tuples = index.as_tuples()
    for b, node in enumerate(dag.basis_node):
        assert dag.tuples[node] == basis_tuples[b]


def test_worked_examples_section_2_6():
    """[1,0,-1] = [[1,-1],[0]] is dependent; [1,1,-2] is independent and needs the aux node [1,1]."""
    mmax = 3
    s = index_set(torus_basis(mmax), 3, 4)
    b = s.basis
    assert is_dependent(torus_ids([1, 0, -1], mmax), b)
    assert not is_dependent(torus_ids([1, 1, -2], mmax), b)
    dag = build_dag(s)
    assert torus_ids([1, 1], mmax) in dag.tuples
    i = dag.tuples.index(torus_ids([1, 1], mmax))
    assert dag.is_aux[i]
    j = dag.tuples.index(torus_ids([1, 1, -2], mmax))
    parts = {dag.tuples[dag.left[j]], dag.tuples[dag.right[j]]}
    assert parts == {torus_ids([1, 1], mmax), torus_ids([-2], mmax)}
    k = dag.tuples.index(torus_ids([1, 0, -1], mmax))
    parts = {dag.tuples[dag.left[k]], dag.tuples[dag.right[k]]}
    assert torus_ids([0], mmax) in parts and torus_ids([1, -1], mmax) in parts


def test_multiple_decompositions_section_5_2():
    """[3,2,1,-1,-2,-3] splits as [[3,-3],[2,1,-1,-2]] and as [[2,-2],[3,1,-1,-3]]."""
    mmax = 3
    t = torus_ids([3, 2, 1, -1, -2, -3], mmax)
    pairs = {(a, b) for a, b in decompositions(t)}
    assert (torus_ids([3, -3], mmax), torus_ids([2, 1, -1, -2], mmax)) in pairs
    assert (torus_ids([2, -2], mmax), torus_ids([3, 1, -1, -3], mmax)) in pairs


@pytest.mark.parametrize("nu", [3, 4, 5, 6])
@pytest.mark.parametrize("D", [4, 6, 8, 11, 12, 14])
def test_torus_aux_count_theorem_3_2(nu, D):
    """Theorem 3.2(ii): Algorithm 1 inserts exactly 2 sum_{k=2}^{nu-1} sum_{n<=D/2} pi(k, n) aux nodes."""
    s = index_set(torus_basis(D), nu, D)
    dag = build_dag(s)
    assert dag.n_aux == aux_torus_alg1(nu, D)
    check_structure(dag, s)


@pytest.mark.parametrize("D", [6, 10, 14])
def test_torus_nu3_one_aux_per_independent(D):
    """Section 3.4: for nu = 3 every independent node needs its own auxiliary node."""
    s = index_set(torus_basis(D), 3, D)
    dag = build_dag(s)
    n_indep = sum(1 for t in s.as_tuples() if len(t) == 3 and not is_dependent(t, s.basis))
    assert dag.n_aux == n_indep


def test_torus_zero_lower_bound_section_5_2():
    """Every torus tuple [0, m] (m invariant) is dependent (proof of Theorem 5.3)."""
    D = 8
    s = index_set(torus_basis(D), 4, D)
    zero = D                               # id of m = 0
    for t in s.as_tuples():
        if len(t) >= 2 and zero in t:
            assert is_dependent(t, s.basis)


def test_torus_aux_ratio_trend():
    """#A/#V for Algorithm 1 on the torus moves towards 1/(1 + C_{nu-1}/2) (Theorem 3.2(ii))."""
    nu = 4
    limit = 1.0 / (1.0 + catalan(nu - 1) / 2.0)
    ratios = []
    for D in (8, 16, 24):
        s = index_set(torus_basis(D), nu, D)
        dag = build_dag(s)
        ratios.append(dag.n_aux / (dag.n_nodes - dag.K + s.counts_per_nu()[0]))
    errs = [abs(r - limit) for r in ratios]
    assert errs[2] < errs[0]


@pytest.mark.parametrize("name", ["plain_fp64_k64", "fwd_grad_k392"])
def test_o3_structure_and_rule_independence(name):
    """The node set of Algorithm 1 does not depend on the decomposition order; edges may."""
    s = workload_index_set(W.WORKLOADS[name])
    a = build_dag(s, rule="balanced")
    b = build_dag(s, rule="peel")
    check_structure(a, s)
    check_structure(b, s)
    assert a.tuples == b.tuples
    assert np.array_equal(a.is_aux, b.is_aux)


def test_o3_fwd_grad_k392_counts():
    """K = 392, nu <= 4, D = 16 (deg n + 2l): 92 aux nodes (88 of order 2, 4 of order 3)."""
    s = workload_index_set(W.WORKLOADS["fwd_grad_k392"])
    dag = build_dag(s)
    assert dag.aux_per_order(4) == [88, 4, 0]
    assert int((dag.order >= 2).sum()) == 3337
    assert dag.n_operands() == 560


def test_algorithm2_structure_and_fewer_aux_at_high_degree():
    """Algorithm 2 (n = 2) builds a valid graph; on the torus at nu = 5 it needs fewer aux nodes (section 3.4)."""
    D = 16
    s = index_set(torus_basis(D), 5, D)
    d1 = build_dag(s, algo=1)
    d2 = build_dag(s, algo=2, n_split=2)
    check_structure(d2, s)
    assert d2.n_aux < d1.n_aux
