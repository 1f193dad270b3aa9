"""Hand-worked graphs of Algorithms 1 and 2 (sections 3.2 and 3.3) on tiny sets, as literals.

Each expected graph below was derived by hand, step by step, from the
algorithms as the paper states them, under the readings the builders document
(balanced-first decomposition order, ties in degree broken towards the larger
tuple position, Algorithm 2's sub-tuple = the s = min(n, len - 1) elements of
largest degree, inserted with Algorithm 1; the rest with Algorithm 2; then k
again).  Each graph is listed as its nodes of order >= 2 in insertion order,
(node, left, right), left being the part tried first.  They are checked
against the oracle and against the C++ builder in libace.

What these literals tell apart (each a plausible misreading):
  * Algorithm 1 vs Algorithm 2 (different auxiliary nodes on every set);
  * splitting off the elements of largest degree vs smallest (the torus
    [-2, 1, 1] and the O(3) [1, 1, 8] would get Algorithm 1's auxiliary node);
  * ties towards the larger position vs the smaller (the O(3) [4, 7, 7]);
  * the sub-tuple inserted with Algorithm 1 vs Algorithm 2 (the single tuple
    [-3, 1, 1, 1] with n = 3: Algorithm 2 would insert [-3, 1] first);
  * s = min(n, len - 1) vs s = n (n = 3 on an order-3 set must equal n = 2).
"""
import numpy as np
import pytest

from oracle.basis import IndexSet, index_set, o3_basis, torus_basis
from oracle.dag import build_dag

# ---- torus, nu <= 4, D = 4 (ids m + 4); tuples written as m values -------------------
TORUS_BASE = [  # order 2 and the order-3/4 nodes that decompose directly (same for both)
    ((-2, 2), (-2,), (2,)), ((-1, 1), (-1,), (1,)), ((0, 0), (0,), (0,)),
    ((-2, 0, 2), (0,), (-2, 2)),
]
TORUS_ALG1 = TORUS_BASE + [
    ((1, 1), (1,), (1,)),                      # aux: [-2] split off [-2, 1, 1]
    ((-2, 1, 1), (-2,), (1, 1)),
    ((-1, -1), (-1,), (-1,)),                  # aux: [2] split off [-1, -1, 2]
    ((-1, -1, 2), (2,), (-1, -1)),
    ((-1, 0, 1), (0,), (-1, 1)),
    ((0, 0, 0), (0,), (0, 0)),
    ((-2, 0, 0, 2), (-2, 2), (0, 0)),
    ((-2, 0, 1, 1), (0,), (-2, 1, 1)),
    ((-1, -1, 0, 2), (0,), (-1, -1, 2)),
    ((-1, -1, 1, 1), (-1, -1), (1, 1)),        # both halves are the auxiliary nodes
    ((-1, 0, 0, 1), (-1, 1), (0, 0)),
    ((0, 0, 0, 0), (0, 0), (0, 0)),
]
TORUS_ALG2 = TORUS_BASE + [
    ((-2, 1), (-2,), (1,)),                    # aux: the two largest degrees of [-2, 1, 1]
    ((-2, 1, 1), (1,), (-2, 1)),
    ((-1, 2), (-1,), (2,)),                    # aux: the two largest degrees of [-1, -1, 2]
    ((-1, -1, 2), (-1,), (-1, 2)),
    ((-1, 0, 1), (0,), (-1, 1)),
    ((0, 0, 0), (0,), (0, 0)),
    ((-2, 0, 0, 2), (-2, 2), (0, 0)),
    ((-2, 0, 1, 1), (0,), (-2, 1, 1)),
    ((-1, -1, 0, 2), (0,), (-1, -1, 2)),
    ((-1, -1, 1, 1), (-1, 1), (-1, 1)),        # [-1, -1] and [1, 1] do not exist here
    ((-1, 0, 0, 1), (-1, 1), (0, 0)),
    ((0, 0, 0, 0), (0, 0), (0, 0)),
]

# ---- O(3), n = 1, l <= 2, degree n + l, p = inf, D = 3, nu <= 3 --------------------------
# ids: 0 = (1,0,0); 1, 2, 3 = (1,1,-1..1); 4..8 = (1,2,-2..2); degrees 1, 2, 3.
O3_ORDER2 = [((0, 0), (0,), (0,)), ((0, 6), (0,), (6,)), ((1, 3), (1,), (3,)), ((2, 2), (2,), (2,)),
             ((4, 8), (4,), (8,)), ((5, 7), (5,), (7,)), ((6, 6), (6,), (6,))]
O3_DEP_HEAD = [((0, 0, 0), (0,), (0, 0)), ((0, 0, 6), (0,), (0, 6)), ((0, 1, 3), (0,), (1, 3)),
               ((0, 2, 2), (0,), (2, 2)), ((0, 4, 8), (0,), (4, 8)), ((0, 5, 7), (0,), (5, 7)),
               ((0, 6, 6), (0,), (6, 6))]
O3_DEP_TAIL = [((4, 6, 8), (6,), (4, 8))]
O3_ALG1 = O3_ORDER2 + O3_DEP_HEAD + [
    ((1, 1), (1,), (1,)), ((1, 1, 8), (8,), (1, 1)),
    ((1, 2), (1,), (2,)), ((1, 2, 7), (7,), (1, 2)),
    ((1, 3, 6), (6,), (1, 3)), ((2, 2, 6), (6,), (2, 2)),
    ((2, 3), (2,), (3,)), ((2, 3, 5), (5,), (2, 3)),
    ((3, 3), (3,), (3,)), ((3, 3, 4), (4,), (3, 3)),
] + O3_DEP_TAIL + [
    ((4, 7), (4,), (7,)), ((4, 7, 7), (7,), (4, 7)),   # all degree 3: the last position is split off
    ((5, 5), (5,), (5,)), ((5, 5, 8), (8,), (5, 5)),
    ((5, 6, 7), (6,), (5, 7)), ((6, 6, 6), (6,), (6, 6)),
]
O3_ALG2 = O3_ORDER2 + O3_DEP_HEAD + [
    ((1, 8), (1,), (8,)), ((1, 1, 8), (1,), (1, 8)),
    ((2, 7), (2,), (7,)), ((1, 2, 7), (1,), (2, 7)),
    ((1, 3, 6), (6,), (1, 3)), ((2, 2, 6), (6,), (2, 2)),
    ((3, 5), (3,), (5,)), ((2, 3, 5), (2,), (3, 5)),
    ((3, 4), (3,), (4,)), ((3, 3, 4), (3,), (3, 4)),
] + O3_DEP_TAIL + [
    ((7, 7), (7,), (7,)), ((4, 7, 7), (4,), (7, 7)),   # ties: the two last positions
    ((5, 8), (5,), (8,)), ((5, 5, 8), (5,), (5, 8)),
    ((5, 6, 7), (6,), (5, 7)), ((6, 6, 6), (6,), (6, 6)),
]

# ---- a set holding the single torus tuple [-3, 1, 1, 1] (ids m + 3) -------------------
SINGLE = (-3, 1, 1, 1)
SINGLE_BY_N = {
    1: [((1, 1), (1,), (1,)), ((1, 1, 1), (1,), (1, 1)), (SINGLE, (-3,), (1, 1, 1))],
    2: [((-3, 1), (-3,), (1,)), ((1, 1), (1,), (1,)), (SINGLE, (-3, 1), (1, 1))],
    # the sub-tuple [-3, 1, 1] goes in by Algorithm 1, which splits off [-3] and inserts [1, 1]
    3: [((1, 1), (1,), (1,)), ((-3, 1, 1), (-3,), (1, 1)), (SINGLE, (1,), (-3, 1, 1))],
}


def oracle_graph(dag, to_label):
    out = []
    for i in range(dag.K, dag.n_nodes):
        out.append((to_label(dag.tuples[i]), to_label(dag.tuples[dag.left[i]]),
                    to_label(dag.tuples[dag.right[i]])))
    return out


def torus_labels(mmax):
    return lambda t: tuple(int(k) - mmax for k in t)


def ids(t):
    return tuple(int(k) for k in t)


def test_torus_nu4_d4_by_hand():
    s = index_set(torus_basis(4), 4, 4)
    lab = torus_labels(4)
    assert oracle_graph(build_dag(s, algo=1), lab) == TORUS_ALG1
    assert oracle_graph(build_dag(s, algo=2, n_split=2), lab) == TORUS_ALG2
    assert build_dag(s, algo=1).n_aux == 2 and build_dag(s, algo=2).n_aux == 2


def o3_pinf_set():
    return index_set(o3_basis(1, 1, 2, 1, 1), 3, 3, p=np.inf)


def test_o3_p_inf_by_hand():
    s = o3_pinf_set()
    assert s.counts_per_nu() == [2, 7, 18]          # [0] and [6] are invariant alone
    assert oracle_graph(build_dag(s, algo=1), ids) == O3_ALG1
    assert oracle_graph(build_dag(s, algo=2, n_split=2), ids) == O3_ALG2
    # s = min(n, len - 1): on an order-3 set n = 3 splits off two elements, as n = 2 does
    assert oracle_graph(build_dag(s, algo=2, n_split=3), ids) == O3_ALG2


def single_tuple_set():
    b = torus_basis(3)
    t = np.array([[m + 3 for m in SINGLE]], dtype=np.int64)
    return IndexSet(b, 4, 6, t, np.array([4]), np.array([6]))


@pytest.mark.parametrize("n", [1, 2, 3])
def test_single_tuple_by_hand(n):
    s = single_tuple_set()
    dag = build_dag(s, algo=1) if n == 1 else build_dag(s, algo=2, n_split=n)
    assert oracle_graph(dag, torus_labels(3)) == SINGLE_BY_N[n]
    assert build_dag(s, algo=2, n_split=1).tuples == build_dag(s, algo=1).tuples   # n = 1 is Algorithm 1


def lib_graph(spec, algo, n_split, to_label, tuples_of_node):
    from paper_2202_04140_gb300.torch_api import Dag
    d = Dag(spec, algo=algo, n_split=n_split)
    e = d.export()
    out = []
    for i in range(d.K, d.n_nodes):
        out.append((to_label(tuples_of_node[i]), to_label(tuples_of_node[e["left"][i]]),
                    to_label(tuples_of_node[e["right"][i]])))
    return out


def lib_node_tuples(spec, algo, n_split):
    """Node tuples of the C++ graph, rebuilt from its own left/right arrays."""
    from paper_2202_04140_gb300.torch_api import Dag
    d = Dag(spec, algo=algo, n_split=n_split)
    e = d.export()
    tup = [(k,) for k in range(d.K)]
    for i in range(d.K, d.n_nodes):
        tup.append(tuple(sorted(tup[e["left"][i]] + tup[e["right"][i]])))
    return tup


@pytest.mark.parametrize("algo,n_split,expected", [(1, 2, TORUS_ALG1), (2, 2, TORUS_ALG2)])
def test_cpp_builder_torus_by_hand(algo, n_split, expected):
    pytest.importorskip("paper_2202_04140_gb300.ace")
    from paper_2202_04140_gb300.torch_api import Spec
    spec = Spec("T", 0, 0, 4, 4, 4, 1, 1, 1, False)
    tup = lib_node_tuples(spec, algo, n_split)
    assert lib_graph(spec, algo, n_split, torus_labels(4), tup) == expected


@pytest.mark.parametrize("algo,n_split,expected", [(1, 2, O3_ALG1), (2, 2, O3_ALG2), (2, 3, O3_ALG2)])
def test_cpp_builder_o3_p_inf_by_hand(algo, n_split, expected):
    pytest.importorskip("paper_2202_04140_gb300.ace")
    from paper_2202_04140_gb300.torch_api import Spec
    spec = Spec("O3", 1, 1, 2, 3, 3, 1, 1, 0, True)
    tup = lib_node_tuples(spec, algo, n_split)
    assert lib_graph(spec, algo, n_split, ids, tup) == expected


MUTATIONS = {
    "sub-tuple inserted by Algorithm 2": ("        insert1(head)\n", "        insert2(head)\n"),
    "s = n instead of min(n, len - 1)": ("s = min(n_split, len(t) - 1)", "s = n_split"),
    "smallest degrees split off": ("key=lambda i: (deg1[t[i]], i), reverse=True",
                                   "key=lambda i: (-deg1[t[i]], i), reverse=True"),
    "ties towards the smaller position": ("key=lambda i: (deg1[t[i]], i), reverse=True",
                                          "key=lambda i: (deg1[t[i]], -i), reverse=True"),
    "Algorithm 2 runs Algorithm 1": ("insert = insert1 if algo == 1 else insert2", "insert = insert1"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_misreadings(name):
    """Plant each misreading in a copy of the oracle's graph builder: some hand-worked literal must fail."""
    import inspect
    import sys
    import oracle.dag as D
    old, new = MUTATIONS[name]
    src = inspect.getsource(D)
    assert src.count(old) == 1, name
    mod = type(D)("mutant_dag")
    sys.modules["mutant_dag"] = mod     # dataclasses look their module up by name
    try:
        exec(compile(src.replace(old, new), "mutant_dag", "exec"), mod.__dict__)
    finally:
        del sys.modules["mutant_dag"]
    limit = sys.getrecursionlimit()
    sys.setrecursionlimit(200)          # a mutant that recurses without end fails fast

    def agrees(s, algo, n, lab, expected):
        try:
            return oracle_graph(mod.build_dag(s, algo=algo, n_split=n), lab) == expected
        except (RecursionError, IndexError):   # a mutant that breaks down also fails its pin
            return False

    try:
        results = [agrees(index_set(torus_basis(4), 4, 4), 1, 2, torus_labels(4), TORUS_ALG1),
                   agrees(index_set(torus_basis(4), 4, 4), 2, 2, torus_labels(4), TORUS_ALG2),
                   agrees(o3_pinf_set(), 1, 2, ids, O3_ALG1),
                   agrees(o3_pinf_set(), 2, 2, ids, O3_ALG2),
                   agrees(o3_pinf_set(), 2, 3, ids, O3_ALG2)]
        results += [agrees(single_tuple_set(), 1 if n == 1 else 2, n, torus_labels(3), SINGLE_BY_N[n])
                    for n in (1, 2, 3)]
    finally:
        sys.setrecursionlimit(limit)
    assert not all(results), name
