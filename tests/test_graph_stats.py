"""Auxiliary-node counts of Algorithms 1 and 2 against the statements of section 3.4,
Theorem 3.1 (ii) and Theorem 3.3 (host library only, no GPU)."""
from math import comb

import numpy as np
import pytest

from oracle.basis import index_set, o3_basis, torus_basis
from oracle.dag import build_dag
from paper_2202_04140_gb300.graph_stats import aux_ratio


def aux(group, nu, D, algo, p=1):
    return aux_ratio(group, nu, D, algo, 2, p)["aux"]


@pytest.mark.parametrize("D", [8, 16, 24])
def test_torus_nu3_needs_the_same_aux_under_both_schemes(D):
    # Section 3.4 on the torus: at nu = 3 each independent node needs exactly one auxiliary node,
    # whichever insertion scheme is used.
    assert aux("torus", 3, D, 1) == aux("torus", 3, D, 2)


@pytest.mark.parametrize("nu,D", [(4, 16), (4, 24), (4, 30), (5, 24), (5, 30)])
def test_torus_algorithm2_inserts_fewer_aux_at_nu4_nu5(nu, D):
    # Section 3.4: clear improvement of the generalised heuristic (n = 2) for nu = 4, 5 as D grows
    # (Theorem 3.3: #A/#V = O(D^(1-n)) against the nonzero limit of Theorem 3.1 (ii)).
    assert aux("torus", nu, D, 2) < aux("torus", nu, D, 1)


def limit_alg1_torus(nu):
    # Theorem 3.1 (ii): lim_{D -> inf} #A/#V = 1 / (1 + C_{nu-1} / 2), C_j the Catalan number
    # (1/j) binom(2j, j - 1).
    j = nu - 1
    return 1.0 / (1.0 + comb(2 * j, j - 1) / j / 2.0)


def test_torus_algorithm1_ratio_approaches_theorem_limit():
    # nu = 3: the ratio rises towards 1/2; nu = 4: it falls back towards 2/7 from above.
    assert limit_alg1_torus(3) == pytest.approx(0.5)
    assert limit_alg1_torus(4) == pytest.approx(2.0 / 7.0)
    r3 = [aux_ratio("torus", 3, D, 1)["ratio"] for D in (40, 80, 120)]
    assert r3[0] < r3[1] < r3[2] < 0.5 and 0.5 - r3[2] < 0.02
    r4 = [aux_ratio("torus", 4, D, 1)["ratio"] for D in (60, 120)]
    lim4 = limit_alg1_torus(4)
    assert r4[0] > r4[1] > lim4 and r4[1] - lim4 < 0.01


@pytest.mark.parametrize("nu,D", [(3, 10), (3, 12), (4, 10), (4, 12), (5, 14)])
def test_o3_total_degree_algorithm2_not_better_preasymptotically(nu, D):
    # Section 3.4 on O(3), p = 1: the generalised heuristic is slightly worse before the asymptotic regime.
    assert aux("o3", nu, D, 2) >= aux("o3", nu, D, 1)


@pytest.mark.parametrize("p,nu,D", [(0, 3, 4), (0, 3, 6), (0, 4, 5), (2, 3, 8), (2, 3, 12)])
def test_o3_p_greater_than_one_algorithm2_inserts_fewer_aux(p, nu, D):
    # Section 3.4 on O(3), p = 2 and p = inf (tuples with ||k||_1 > D present): Algorithm 2 does better.
    assert aux("o3", nu, D, 2, p) < aux("o3", nu, D, 1, p)


def test_ratio_is_aux_over_aux_plus_basis():
    # #V = #A + |K(1..nu, D)| (section 3.1); leaves outside K are not counted.
    r = aux_ratio("torus", 4, 12, 1)
    assert r["V"] == r["aux"] + r["basis"] and r["ratio"] == pytest.approx(r["aux"] / r["V"])


@pytest.mark.parametrize("group,p,nu,D,ob", [
    ("torus", 1, 4, 16, lambda: torus_basis(16)),
    ("o3", 0, 3, 4, lambda: o3_basis(1, 4, 3, 1, 1)),
    ("o3", 1, 3, 10, lambda: o3_basis(1, 10, 9, 1, 1)),
])
@pytest.mark.parametrize("algo", [1, 2])
def test_statistics_graphs_match_the_oracle_builder(group, p, nu, D, ob, algo):
    # the sets the tables use, built by the oracle's own Algorithm 1 / 2 (section 3.2, 3.3)
    o = index_set(ob(), nu, D, p={1: 1, 2: 2, 0: np.inf}[p])
    od = build_dag(o, algo=algo, rule="balanced", n_split=2)
    r = aux_ratio(group, nu, D, algo, 2, p)
    assert r["basis"] == len(o.deg) and r["aux"] == od.n_aux
