"""Plain, slow, FP64 CPU oracle for the recursive ACE contraction (arXiv 2202.04140).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call, link
or execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` use it.  It shares no code with
the C++/CUDA library (no kernels, headers, helpers, tables or generators); the
only module both sides use is ``workloads`` (seeded random draws, no method
arithmetic).

Contents (each function cites the passage of the paper it follows):
  basis     one-particle bases (O(3), SO(2), torus) and the invariant,
            degree-truncated index set K_G^p(D)      (sections 2.2-2.5, Eq. 3)
  dag       Algorithm 1 (and Algorithm 2) building the computational graph,
            node / auxiliary counts                   (sections 2.6, 3.2, 3.3)
  evaluate  phi = sum_k c_k prod_t A_{k_t} term by term, its product-rule
            gradient, and the recursive graph evaluation with its reverse sweep
                                                      (Eq. 1, Eq. 2, Eq. 4)
  pooling   A_nlm = sum_j R_n(r_j) Y_lm(r_j/|r_j|) and the forces -dphi/dr_j
                                                      (Eq. 2, section 2.4)

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
brute force, the paper's closed forms, graphs worked out by hand from the
algorithms' steps, or identities of the mathematics.  The O(3) auxiliary-node
counts of the larger workloads have no printed value in the paper (its figures
carry no data); they are outputs of the pinned graph builder.
"""
