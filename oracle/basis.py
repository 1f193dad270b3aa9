"""One-particle bases and the sparse invariant index set (oracle; test infrastructure only).

Paper passages followed:
  * section 2.4: O(3) one-particle basis phi_nlm = R_n Y_l^m, k = (n, l, m),
    invariance requires sum_t m_t = 0 and sum_t l_t even.
  * section 2.2: SO(2) basis R_n e^{-i m theta}, k = (n, m), sum_t m_t = 0.
  * section 2.3: torus basis e^{i m theta}, k = m, sum_t m_t = 0.
  * section 2.5, Eq. 3: K_G^p(D) = {k invariant : ||k||_p <= D}; for p = 1 the
    degree of a tuple is the sum of its one-particle degrees (n + l for O(3),
    n + |m| for SO(2), |m| for the torus).
  * section 1 / section 2.6: permutation symmetry, so only sorted tuples
    (multisets) are kept.
  * section "Invariant features": phi_nlmk(r, mu) = R_n Y_l^m T_k(mu) with the
    degree l + n + k; the feature index k carries no symmetry charge.

Readings of points the paper leaves open:
  * The one-particle degree is wn*n + wl*l (the paper's n + l is wn = wl = 1;
    the workloads use n + 2l).
  * One-particle ids: O(3) id = (n - nmin)(lmax+1)^2 + l^2 + (l + m), i.e. n
    outer, then l, then m ascending; with invariant features of degree
    0 <= k <= kmax, id = ((n - nmin)(kmax+1) + k)(lmax+1)^2 + l^2 + (l + m)
    (n, then k, then l, then m), degree wn*n + wl*l + wk*k.  Torus id = m + mmax.  SO(2) id =
    (n - nmin)(2 mmax + 1) + (m + mmax).
  * A tuple is stored non-decreasing in id; the basis order is (nu, then
    lexicographic on ids).  This one order fixes the coefficient draws and the
    insertion order of Algorithm 1.
  * p = 1 only (the sum of one-particle degrees) on the evaluated path; p = 2 and
    p = infinity are provided for counting.
"""
from __future__ import annotations

from dataclasses import dataclass
import numpy as np


@dataclass
class OneParticleBasis:
    """A finite one-particle basis: per id its labels, degree and symmetry charges."""
    group: str            # "O3", "SO2" or "T"
    labels: np.ndarray    # (K, 3) rows (n, l, m); unused labels are 0
    deg: np.ndarray       # (K,) int64 one-particle degree
    m: np.ndarray         # (K,) int64
    l: np.ndarray         # (K,) int64 (zeros outside O(3))
    k: np.ndarray | None = None  # (K,) int64 invariant-feature degree (None: no feature index)

    @property
    def K(self) -> int:
        return int(self.deg.shape[0])


def o3_basis(nmin: int, nmax: int, lmax: int, wn: int = 1, wl: int = 1, kmax: int = 0,
             wk: int = 1) -> OneParticleBasis:
    """k = (n, l, m), nmin <= n <= nmax, 0 <= l <= lmax, |m| <= l (section 2.4); with kmax > 0
    also the invariant-feature degree 0 <= k <= kmax (phi_nlmk, degree wn n + wl l + wk k)."""
    rows = [(n, l, m, k) for n in range(nmin, nmax + 1) for k in range(kmax + 1)
            for l in range(lmax + 1) for m in range(-l, l + 1)]
    lab = np.array(rows, dtype=np.int64)
    return OneParticleBasis("O3", lab[:, :3].copy(), wn * lab[:, 0] + wl * lab[:, 1] + wk * lab[:, 3],
                            lab[:, 2].copy(), lab[:, 1].copy(), lab[:, 3].copy() if kmax > 0 else None)


def so2_basis(nmin: int, nmax: int, mmax: int, wn: int = 1, wm: int = 1) -> OneParticleBasis:
    """k = (n, m), degree wn*n + wm*|m| (section 2.2, degree of section 2.5)."""
    rows = [(n, 0, m) for n in range(nmin, nmax + 1) for m in range(-mmax, mmax + 1)]
    lab = np.array(rows, dtype=np.int64)
    return OneParticleBasis("SO2", lab, wn * lab[:, 0] + wm * np.abs(lab[:, 2]),
                            lab[:, 2].copy(), np.zeros(len(rows), dtype=np.int64))


def torus_basis(mmax: int) -> OneParticleBasis:
    """k = m, -mmax <= m <= mmax, degree |m| (section 2.3 and section 2.5)."""
    m = np.arange(-mmax, mmax + 1, dtype=np.int64)
    lab = np.stack([np.zeros_like(m), np.zeros_like(m), m], axis=1)
    return OneParticleBasis("T", lab, np.abs(m), m.copy(), np.zeros_like(m))


def _sorted_tuples_within_degree(deg: np.ndarray, nu_max: int, deg_max: float, p: float):
    """All non-decreasing id tuples of length 1..nu_max with ||deg||_p <= deg_max.

    Yields (nu, T) with T an int64 array (count, nu).  Degree truncation is the
    only filter here: a non-invariant tuple can still extend to an invariant one.
    """
    K = deg.shape[0]
    ids = np.arange(K, dtype=np.int64)

    def measure(d):       # per-tuple accumulated degree in the p-norm
        if p == 1:
            return d
        if p == np.inf:
            return d
        return d ** p

    def within(acc):
        if p == 1:
            return acc <= deg_max
        if p == np.inf:
            return acc <= deg_max
        return acc <= deg_max ** p + 1e-9

    def combine(acc, d):
        if p == np.inf:
            return np.maximum(acc, d)
        return acc + d

    dm = measure(deg.astype(np.float64))
    keep = within(dm)
    T = ids[keep][:, None]
    acc = dm[keep]
    yield 1, T
    for nu in range(2, nu_max + 1):
        last = T[:, -1]
        new_T, new_acc = [], []
        for j in range(K):
            a = combine(acc, dm[j])
            sel = (last <= j) & within(a)
            if np.any(sel):
                rows = T[sel]
                new_T.append(np.concatenate([rows, np.full((rows.shape[0], 1), j, np.int64)], axis=1))
                new_acc.append(a[sel])
        if not new_T:
            return
        T = np.concatenate(new_T, axis=0)
        acc = np.concatenate(new_acc, axis=0)
        order = np.lexsort(T.T[::-1])        # lexicographic on (k_1, ..., k_nu)
        T, acc = T[order], acc[order]
        yield nu, T


@dataclass
class IndexSet:
    """The basis set K: sorted tuples in canonical order (nu, lexicographic)."""
    basis: OneParticleBasis
    nu_max: int
    deg_max: int
    tuples: np.ndarray     # (n_basis, nu_max) int64, -1 padded
    nu: np.ndarray         # (n_basis,) int64 correlation order
    deg: np.ndarray        # (n_basis,) int64 summed one-particle degree

    @property
    def n_basis(self) -> int:
        return int(self.nu.shape[0])

    def counts_per_nu(self) -> list[int]:
        return [int(np.sum(self.nu == v)) for v in range(1, self.nu_max + 1)]

    def as_tuples(self) -> list[tuple]:
        return [tuple(int(x) for x in row[:n]) for row, n in zip(self.tuples, self.nu)]


def index_set(basis: OneParticleBasis, nu_max: int, deg_max: int, p: float = 1,
              require_l_even: bool | None = None) -> IndexSet:
    """K_G^p(D) restricted to 1 <= nu <= nu_max (section 2.5, Eq. 3).

    Invariance filter: sum_t m_t = 0 for every group (sections 2.2-2.4); for O(3)
    additionally sum_t l_t even (section 2.4).
    """
    if require_l_even is None:
        require_l_even = basis.group == "O3"
    blocks, nus = [], []
    for nu, T in _sorted_tuples_within_degree(basis.deg, nu_max, deg_max, p):
        ok = basis.m[T].sum(axis=1) == 0
        if require_l_even:
            ok &= (basis.l[T].sum(axis=1) % 2) == 0
        T = T[ok]
        pad = np.full((T.shape[0], nu_max), -1, dtype=np.int64)
        pad[:, :nu] = T
        blocks.append(pad)
        nus.append(np.full(T.shape[0], nu, dtype=np.int64))
    tuples = np.concatenate(blocks, axis=0) if blocks else np.zeros((0, nu_max), np.int64)
    nu = np.concatenate(nus) if nus else np.zeros(0, np.int64)
    d = np.where(tuples >= 0, basis.deg[np.maximum(tuples, 0)], 0).sum(axis=1)
    return IndexSet(basis, nu_max, deg_max, tuples, nu, d.astype(np.int64))


def workload_index_set(w) -> IndexSet:
    """Index set of a ``workloads.Workload`` (O(3), p = 1, degree wn*n + wl*l [+ wk*k]).

    Enumerated block by block (``index_set_by_first``, the same set as ``index_set``)."""
    b = o3_basis(w.nmin, w.nmax, w.lmax, w.wn, w.wl, w.kmax, w.wk)
    return index_set_by_first(b, w.nu_max, w.deg_max)


def index_set_by_first(basis: OneParticleBasis, nu_max: int, deg_max: int,
                       require_l_even: bool | None = None) -> IndexSet:
    """The same set as ``index_set`` with p = 1, enumerated one block at a time (section 2.5, Eq. 3).

    For large sets (millions of tuples) ``index_set`` holds every degree-bounded
    tuple of an order at once.  Here, for each order nu and each first element
    k_1 in increasing id order, the non-decreasing tuples starting with k_1 are
    grown one element at a time: a row with last element a and degree sum d
    extends by every id j >= a with d + deg(j) <= deg_max (rows that share (a, d)
    share that candidate list).  The completed rows are filtered by the same
    invariance rule as ``index_set`` and sorted lexicographically; since every
    tuple of the block starts with k_1, the blocks in k_1 order give the
    canonical (nu, lexicographic) order.
    """
    if require_l_even is None:
        require_l_even = basis.group == "O3"
    deg = basis.deg.astype(np.int64)
    K = deg.shape[0]
    blocks, nus = [], []
    for nu in range(1, nu_max + 1):
        for k1 in range(K):
            if deg[k1] > deg_max:
                continue
            T = np.array([[k1]], dtype=np.int64)
            acc = deg[[k1]]
            for _ in range(1, nu):
                key = T[:, -1] * (deg_max + 1) + acc
                order = np.argsort(key, kind="stable")
                T, acc, key = T[order], acc[order], key[order]
                starts = np.flatnonzero(np.r_[True, key[1:] != key[:-1]])
                ends = np.r_[starts[1:], key.shape[0]]
                new_T, new_acc = [], []
                for s, e in zip(starts, ends):
                    a, d = int(T[s, -1]), int(acc[s])
                    cand = np.arange(a, K, dtype=np.int64)
                    cand = cand[deg[cand] + d <= deg_max]
                    if cand.size == 0:
                        continue
                    rows = np.repeat(T[s:e], cand.size, axis=0)
                    new_T.append(np.concatenate([rows, np.tile(cand, e - s)[:, None]], axis=1))
                    new_acc.append(np.repeat(acc[s:e], cand.size) + np.tile(deg[cand], e - s))
                if not new_T:
                    T = np.zeros((0, T.shape[1] + 1), np.int64)
                    break
                T, acc = np.concatenate(new_T), np.concatenate(new_acc)
            if T.shape[0] == 0:
                continue
            ok = basis.m[T].sum(axis=1) == 0
            if require_l_even:
                ok &= (basis.l[T].sum(axis=1) % 2) == 0
            T = T[ok]
            if T.shape[0] == 0:
                continue
            T = T[np.lexsort(T.T[::-1])]
            pad = np.full((T.shape[0], nu_max), -1, dtype=np.int64)
            pad[:, :nu] = T
            blocks.append(pad)
            nus.append(np.full(T.shape[0], nu, dtype=np.int64))
    tuples = np.concatenate(blocks, axis=0) if blocks else np.zeros((0, nu_max), np.int64)
    nu_arr = np.concatenate(nus) if nus else np.zeros(0, np.int64)
    d = np.where(tuples >= 0, basis.deg[np.maximum(tuples, 0)], 0).sum(axis=1)
    return IndexSet(basis, nu_max, deg_max, tuples, nu_arr, d.astype(np.int64))
