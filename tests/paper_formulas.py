"""Closed forms printed in the paper, retyped for use as pins (no oracle code here).

  * pi(k, n): integer partitions of n into exactly k parts (section 5.1); the
    paper sets pi(0, n) = 0.
  * E-slice size (section 5.2, proof of Lemma 5.1):
        #E_T(nu, D) = sum_{k=0}^{nu} pi(k, D/2) pi(nu-k, D/2) for even D, 0 for odd D.
  * #K_T(nu, D) = 1 + sum_{h=1}^{D} sum_{k=1}^{nu} #E_T(k, h)   (proof of Lemma 5.2);
    K_T(nu, D) holds the tuples of length exactly nu.
  * Theorem 3.2(ii): Algorithm 1 inserts exactly
        #A_T(nu, D) = 2 sum_{k=2}^{nu-1} sum_{n=1}^{floor(D/2)} pi(k, n)
    auxiliary nodes on the torus.
  * Theorem 3.2(ii) limit: #A/#V -> 1 / (1 + C_{nu-1}/2), C the Catalan numbers.
"""
from functools import lru_cache
from math import comb


@lru_cache(maxsize=None)
def partitions_exact(k: int, n: int) -> int:
    """pi(k, n) by the recursion p(k, n) = p(k-1, n-1) + p(k, n-k) (parts >= 1)."""
    if k <= 0 or n <= 0:
        return 0
    if k == 1:
        return 1
    if k > n:
        return 0
    return partitions_exact(k - 1, n - 1) + partitions_exact(k, n - k)


def e_slice(nu: int, D: int) -> int:
    if D % 2:
        return 0
    h = D // 2
    return sum(partitions_exact(k, h) * partitions_exact(nu - k, h) for k in range(nu + 1))


def k_torus(nu: int, D: int) -> int:
    return 1 + sum(e_slice(k, h) for h in range(1, D + 1) for k in range(1, nu + 1))


def aux_torus_alg1(nu: int, D: int) -> int:
    return 2 * sum(partitions_exact(k, n) for k in range(2, nu) for n in range(1, D // 2 + 1))


def catalan(n: int) -> int:
    return comb(2 * n, n) // (n + 1)
