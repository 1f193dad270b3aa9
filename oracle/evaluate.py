"""phi = sum_k c_k prod_t A_{k_t}, its gradient, and the recursive graph evaluation (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Everything is FP64.

Paper passages followed:
  * Eq. 1 / Eq. 2 (sections 1 and 2.1): phi = sum_{k in K} c_k AA_k with
    AA_k = prod_{t=1}^{nu(k)} A_{k_t}.  ``phi_naive`` evaluates this sum term by
    term; ``grad_naive`` differentiates every term by the product rule.
  * Eq. 4 / Eq. 5 (section 2.6): every node of order >= 2 is the product of its
    two in-edge nodes; auxiliary nodes carry c = 0.  ``dag_forward`` evaluates
    the nodes in id order (a topological order) and reads out sum c_k AA_k;
    ``dag_reverse`` is the reverse sweep of that recursion (the adjoint is not
    in the paper; it is the product rule applied to Eq. 4).

Shapes: A (n_env, K); c (n_basis, n_out); phi (n_env, n_out); phibar like phi;
dA like A.  dA = sum_ch phibar[:, ch] * dphi[:, ch]/dA.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

_CHUNK = 64


def _groups(index):
    for v in range(1, index.nu_max + 1):
        sel = np.nonzero(index.nu == v)[0]
        if sel.size:
            yield v, sel, index.tuples[sel, :v]


def phi_naive(A: np.ndarray, index, c: np.ndarray) -> np.ndarray:
    """Eq. 2 term by term: phi[e, ch] = sum_k c[k, ch] prod_t A[e, k_t]."""
    A = np.asarray(A, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64).reshape(index.n_basis, -1)
    phi = np.zeros((A.shape[0], c.shape[1]))
    for e0 in range(0, A.shape[0], _CHUNK):
        Ae = A[e0:e0 + _CHUNK]
        for v, sel, T in _groups(index):
            AA = np.prod(Ae[:, T], axis=2)            # (chunk, n_v): AA_k per term
            phi[e0:e0 + _CHUNK] += AA @ c[sel]
    return phi


def grad_naive(A: np.ndarray, index, c: np.ndarray, phibar: np.ndarray | None = None) -> np.ndarray:
    """Product rule on every term of Eq. 2.

    d/dA_j prod_t A_{k_t} = sum_{t : k_t = j} prod_{s != t} A_{k_s}; the sum over
    positions t handles repeated indices (multiplicity) without division.
    """
    A = np.asarray(A, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64).reshape(index.n_basis, -1)
    n_env, K = A.shape
    if phibar is None:
        phibar = np.ones((n_env, c.shape[1]))
    phibar = np.asarray(phibar, dtype=np.float64).reshape(n_env, -1)
    dA = np.zeros_like(A)
    scatter = {}
    for v, sel, T in _groups(index):
        for t in range(v):                       # sparse (n_v, K) indicator of k_t
            scatter[(v, t)] = sp.csr_matrix(
                (np.ones(sel.size), (np.arange(sel.size), T[:, t])), shape=(sel.size, K))
    for e0 in range(0, n_env, _CHUNK):
        Ae = A[e0:e0 + _CHUNK]
        w_all = phibar[e0:e0 + _CHUNK] @ c.T       # (chunk, n_basis): sum_ch phibar c
        for v, sel, T in _groups(index):
            F = Ae[:, T]                          # (chunk, n_v, v) factors
            w = w_all[:, sel]
            for t in range(v):
                others = np.prod(np.delete(F, t, axis=2), axis=2) if v > 1 else np.ones(F.shape[:2])
                dA[e0:e0 + _CHUNK] += (scatter[(v, t)].T @ (others * w).T).T
    return dA


def phi_per_order(A: np.ndarray, index, c: np.ndarray) -> np.ndarray:
    """phi split by correlation order: out[v-1] = sum_{k : nu(k) = v} c_k AA_k."""
    c = np.asarray(c, dtype=np.float64).reshape(index.n_basis, -1)
    out = np.zeros((index.nu_max, A.shape[0], c.shape[1]))
    for v, sel, T in _groups(index):
        out[v - 1] = np.prod(np.asarray(A, np.float64)[:, T], axis=2) @ c[sel]
    return out


def node_coefficients(dag, c: np.ndarray) -> np.ndarray:
    """c per graph node: the basis coefficient, 0 for auxiliary and non-basis leaves (section 2.6)."""
    c = np.asarray(c, dtype=np.float64).reshape(dag.basis_node.shape[0], -1)
    cn = np.zeros((dag.n_nodes, c.shape[1]))
    cn[dag.basis_node] = c
    return cn


def dag_forward(dag, A: np.ndarray, c: np.ndarray):
    """Recursive evaluation AA_k = AA_{k1} * AA_{k2} in id order (Eq. 4), then phi = sum c AA.

    Returns (AA, phi) with AA of shape (n_env, n_nodes).
    """
    A = np.asarray(A, dtype=np.float64)
    AA = np.empty((A.shape[0], dag.n_nodes))
    AA[:, :dag.K] = A
    for i in range(dag.K, dag.n_nodes):
        AA[:, i] = AA[:, dag.left[i]] * AA[:, dag.right[i]]
    phi = AA @ node_coefficients(dag, c)
    return AA, phi


def dag_reverse(dag, AA: np.ndarray, c: np.ndarray, phibar: np.ndarray | None = None) -> np.ndarray:
    """Reverse sweep of the recursion: abar_i = sum_ch c_i phibar; abar_l += abar_i AA_r, abar_r += abar_i AA_l."""
    cn = node_coefficients(dag, c)
    n_env = AA.shape[0]
    if phibar is None:
        phibar = np.ones((n_env, cn.shape[1]))
    abar = np.asarray(phibar, np.float64).reshape(n_env, -1) @ cn.T     # (n_env, n_nodes)
    for i in range(dag.n_nodes - 1, dag.K - 1, -1):
        l, r = dag.left[i], dag.right[i]
        g = abar[:, i]
        abar[:, l] += g * AA[:, r]
        abar[:, r] += g * AA[:, l]
    return abar[:, :dag.K].copy()


def error_scale(A: np.ndarray, index, c: np.ndarray) -> np.ndarray:
    """Condition-aware normaliser sum_k |c_k| |AA_k| per environment and channel.

    phi evaluated with |A| and |c|.  An FP32 product of nu factors carries a
    relative error of at most about (nu - 1) u, so |phi_hat - phi| / this scale
    is the error measure that a correct FP32 evaluation keeps near u, whatever
    the cancellation in phi itself.
    """
    return phi_naive(np.abs(A), index, np.abs(c))


def grad_error_scale(A: np.ndarray, index, c: np.ndarray, phibar: np.ndarray | None = None) -> np.ndarray:
    """The same normaliser for dphi/dA: the product-rule gradient with |A|, |c|, |phibar|."""
    pb = None if phibar is None else np.abs(phibar)
    return grad_naive(np.abs(A), index, np.abs(c), pb)
