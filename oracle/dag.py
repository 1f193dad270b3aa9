"""The recursive computational graph and its insertion heuristics (oracle; test infrastructure only).

Paper passages followed:
  * section 2.6: a tuple k decomposes as k = [k1, k2] when it is the multiset
    union of k1 and k2, so that AA_k = AA_{k1} * AA_{k2} (Eq. 4); the graph G
    holds one node per basis function, every node of order >= 2 has exactly two
    in-edges (Eq. 5); the one-particle nodes [k] are inserted first, further
    nodes in increasing correlation order; nodes that are not invariant
    (auxiliary nodes) carry a zero coefficient.
  * Definition 2.1 (section 2.6): k is dependent when it splits into two
    invariant tuples, independent otherwise.
  * Algorithm 1 (section 3.2): insert k; try every decomposition; if none has
    both halves in G, split off the one-particle element of maximal degree,
    insert the rest recursively, then insert k again.
  * Algorithm 2 (section 3.3): as Algorithm 1, but the fallback splits off the
    sub-tuple of length s <= min(n, len(k) - 1) of maximal norm, inserted with
    Algorithm 1, then inserts the rest with Algorithm 2 and finally k again.

Readings of points the paper leaves open (the C++ builder follows the same ones):
  * Decomposition order ("for all decompositions" is unordered in the paper):
    "balanced" tries part sizes s = floor(nu/2) down to 1, "peel" tries
    s = 1 up to floor(nu/2); for each s the positions of k1 run over
    combinations of tuple positions in lexicographic order; a repeated k1
    multiset is not tried twice.  The first pair with both halves in G is
    taken, left = k1 (the size-s part), right = its complement.
  * Fallback tie-break: among elements of maximal one-particle degree, the one
    at the largest position of the sorted tuple is split off.
  * Algorithm 2's maximal-norm sub-tuple: the s = min(n, nu - 1) elements of
    largest degree (ties: largest positions first), kept in tuple order.
  * After the recursive insertion the full decomposition loop is run again for
    k (the pair finally chosen need not be the fallback split).
  * Node ids are insertion order; leaves are the K one-particle functions with
    ids 0..K-1.  Auxiliary nodes are the nodes of order >= 2 that are not in
    the basis set.
"""
from __future__ import annotations

from dataclasses import dataclass
from itertools import combinations
import numpy as np


def decompositions(t: tuple, rule: str = "balanced"):
    """All splits t = [t1, t2] with 1 <= |t1| <= |t|/2, in the builder's order (section 2.6)."""
    nu = len(t)
    sizes = range(nu // 2, 0, -1) if rule == "balanced" else range(1, nu // 2 + 1)
    for s in sizes:
        seen = set()
        for pos in combinations(range(nu), s):
            t1 = tuple(t[i] for i in pos)
            if t1 in seen:
                continue
            seen.add(t1)
            chosen = set(pos)
            t2 = tuple(t[i] for i in range(nu) if i not in chosen)
            yield t1, t2


@dataclass
class Dag:
    """The graph G in canonical (insertion) ids."""
    K: int
    tuples: list          # node id -> sorted tuple of one-particle ids
    left: np.ndarray      # (N,) int64, -1 for leaves
    right: np.ndarray     # (N,) int64, -1 for leaves
    is_aux: np.ndarray    # (N,) bool
    basis_node: np.ndarray  # (n_basis,) node id of every basis tuple
    order: np.ndarray     # (N,) correlation order of every node

    @property
    def n_nodes(self) -> int:
        return len(self.tuples)

    @property
    def n_aux(self) -> int:
        return int(self.is_aux.sum())

    def aux_per_order(self, nu_max: int) -> list[int]:
        return [int(np.sum(self.is_aux & (self.order == v))) for v in range(2, nu_max + 1)]

    def consumers(self) -> np.ndarray:
        """Number of nodes that use each node as a factor."""
        cnt = np.zeros(self.n_nodes, dtype=np.int64)
        inner = self.left >= 0
        np.add.at(cnt, self.left[inner], 1)
        np.add.at(cnt, self.right[inner], 1)
        return cnt

    def n_operands(self) -> int:
        """Nodes of order >= 2 used as a factor of another node."""
        return int(np.sum((self.consumers() > 0) & (self.order >= 2)))


def build_dag(index, algo: int = 1, rule: str = "balanced", n_split: int = 2) -> Dag:
    """Build G for an ``IndexSet`` with Algorithm 1 (algo=1) or Algorithm 2 (algo=2)."""
    deg1 = index.basis.deg
    K = index.basis.K
    ids: dict[tuple, int] = {}
    tuples, left, right = [], [], []

    def add(t, a, b):
        ids[t] = len(tuples)
        tuples.append(t)
        left.append(a)
        right.append(b)

    for k in range(K):                       # the one-particle nodes [k]
        add((k,), -1, -1)

    def try_pairs(t) -> bool:
        for t1, t2 in decompositions(t, rule):
            if t1 in ids and t2 in ids:
                add(t, ids[t1], ids[t2])
                return True
        return False

    def top_positions(t, s):
        # positions of the s largest one-particle degrees; ties -> larger position first
        order = sorted(range(len(t)), key=lambda i: (deg1[t[i]], i), reverse=True)
        return sorted(order[:s])

    def insert1(t):                           # Algorithm 1
        if t in ids:
            return
        if try_pairs(t):
            return
        j = top_positions(t, 1)[0]
        rest = t[:j] + t[j + 1:]
        insert1(rest)                         # [t_j] is a leaf, always in G
        insert1(t)

    def insert2(t):                           # Algorithm 2 with parameter n_split
        if t in ids:
            return
        if try_pairs(t):
            return
        s = min(n_split, len(t) - 1)
        pos = top_positions(t, s)
        head = tuple(t[i] for i in pos)
        rest = tuple(t[i] for i in range(len(t)) if i not in set(pos))
        insert1(head)
        insert2(rest)
        insert2(t)

    insert = insert1 if algo == 1 else insert2
    basis_tuples = index.as_tuples()
    for t in basis_tuples:                    # increasing correlation order
        if len(t) >= 2:
            insert(t)
    basis_set = set(basis_tuples)
    is_aux = np.array([len(t) >= 2 and t not in basis_set for t in tuples], dtype=bool)
    basis_node = np.array([ids[t] for t in basis_tuples], dtype=np.int64)
    order = np.array([len(t) for t in tuples], dtype=np.int64)
    return Dag(K, tuples, np.array(left, np.int64), np.array(right, np.int64),
               is_aux, basis_node, order)


def is_dependent(t: tuple, basis) -> bool:
    """Definition 2.1: t splits into two invariant tuples (m sums zero, l sums even)."""
    def invariant(u):
        if sum(int(basis.m[k]) for k in u) != 0:
            return False
        if basis.group == "O3" and sum(int(basis.l[k]) for k in u) % 2:
            return False
        return True
    return any(invariant(a) and invariant(b) for a, b in decompositions(t, "balanced"))
