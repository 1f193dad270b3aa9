"""Auxiliary-node statistics of the contraction graph (sections 3.2-3.4).

For a correlation order nu and degree D the paper measures the insertion
heuristics by #A_G(nu, D) / #V_G(nu, D): the auxiliary nodes over all nodes,
V = A united with K(1, D), ..., K(nu, D) (section 3.1; Theorems 3.1 and 3.3,
Figures 1-3).  This module builds the graphs with libace (Algorithm 1, or
Algorithm 2 with parameter n) and reports that ratio.

    python -m paper_2202_04140_gb300.graph_stats            # the tables of both groups
    python -m paper_2202_04140_gb300.graph_stats --group torus --nu 4 --deg 8 12 16

The one-particle sets are taken large enough that the degree bound alone
truncates them: torus |m| <= D; O(3) with the paper's degree n + l, n >= 1,
so 1 <= n <= D and l <= D - 1.  p selects the tuple norm (1, 2, or 0 for the
maximum, section 2.5).
"""
from __future__ import annotations

import argparse
import time

from . import ace as L

_GROUPS = {"torus": L.ACE_GROUP_TORUS, "so2": L.ACE_GROUP_SO2, "o3": L.ACE_GROUP_O3}


def spec_params(group: str, nu: int, D: int, p_norm: int = 1) -> dict:
    """ace_build_spec arguments for K_G(nu, D) with a one-particle set cut by the degree only."""
    if group == "torus":
        return dict(group=L.ACE_GROUP_TORUS, nmin=0, nmax=0, lmax=D, nu_max=nu, deg_max=D, wn=1, wl=1,
                    p_norm=p_norm)
    if group == "so2":  # k = (n, m), degree n + |m|, n >= 0
        return dict(group=L.ACE_GROUP_SO2, nmin=0, nmax=D, lmax=D, nu_max=nu, deg_max=D, wn=1, wl=1,
                    p_norm=p_norm)
    if group == "o3":  # k = (n, l, m), degree n + l, n >= 1
        return dict(group=L.ACE_GROUP_O3, nmin=1, nmax=D, lmax=max(D - 1, 0), nu_max=nu, deg_max=D, wn=1, wl=1,
                    p_norm=p_norm)
    raise ValueError(f"unknown group {group!r}")


def aux_ratio(group: str, nu: int, D: int, algo: int = 1, n_split: int = 2, p_norm: int = 1) -> dict:
    """#A, #V = #A + |K(1..nu, D)| and their ratio for one graph."""
    spec = L.ace_build_spec(**spec_params(group, nu, D, p_norm))
    try:
        n_basis, K, _ = L.ace_spec_info(spec, nu)
        dag = L.ace_build_dag(spec, algo, L.ACE_SPLIT_BALANCED, n_split)
        try:
            _, n_aux, _, _ = L.ace_dag_info(dag)
        finally:
            L.ace_dag_free(dag)
    finally:
        L.ace_spec_free(spec)
    n_v = n_aux + n_basis
    return {"group": group, "nu": nu, "D": D, "p": p_norm, "algo": algo, "n": n_split if algo == 2 else 1,
            "K": K, "basis": n_basis, "aux": n_aux, "V": n_v, "ratio": n_aux / n_v if n_v else 0.0}


# Ranges that build in seconds on one core: (group, p, [(nu, [D, ...]), ...]).
DEFAULT_TABLES = [
    ("torus", 1, [(3, [8, 16, 24, 30]), (4, [8, 16, 24, 30]), (5, [8, 16, 24, 30]), (6, [8, 16, 24, 30])]),
    ("o3", 1, [(3, [8, 12, 16, 20]), (4, [8, 12, 16]), (5, [10, 12, 14, 16])]),
    ("o3", 2, [(3, [6, 8, 10, 12]), (4, [6, 8])]),
    ("o3", 0, [(3, [3, 4, 6, 8]), (4, [3, 4, 5])]),
]


def table(group: str, p_norm: int, rows, n_split: int = 2) -> str:
    """Markdown rows: #A/#V for Algorithm 1 and Algorithm 2 (parameter n_split) side by side.

    rows: [(nu, [D, ...]), ...]."""
    pname = {1: "1", 2: "2", 0: "inf"}[p_norm]
    lines = [f"### {group}, p = {pname}", "",
             f"| nu | D | basis | #A (Alg. 1) | #A/#V (Alg. 1) | #A (Alg. 2, n = {n_split}) | #A/#V (Alg. 2) |",
             "|---|---|---|---|---|---|---|"]
    for nu, degs in rows:
        for D in degs:
            a1 = aux_ratio(group, nu, D, 1, n_split, p_norm)
            a2 = aux_ratio(group, nu, D, 2, n_split, p_norm)
            lines.append(f"| {nu} | {D} | {a1['basis']:,} | {a1['aux']:,} | {a1['ratio']:.4f} | "
                         f"{a2['aux']:,} | {a2['ratio']:.4f} |")
    return "\n".join(lines)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--group", choices=sorted(_GROUPS))
    ap.add_argument("--p", type=int, default=1, choices=[0, 1, 2], help="tuple norm: 1, 2 or 0 (maximum)")
    ap.add_argument("--nu", type=int, nargs="+")
    ap.add_argument("--deg", type=int, nargs="+")
    ap.add_argument("--n-split", type=int, default=2, help="parameter n of Algorithm 2")
    a = ap.parse_args(argv)
    t0 = time.time()
    if a.group:
        print(table(a.group, a.p, [(nu, a.deg or [8, 12]) for nu in (a.nu or [3, 4])], a.n_split))
    else:
        for g, p, rows in DEFAULT_TABLES:
            print(table(g, p, rows, a.n_split))
            print()
    print(f"({time.time() - t0:.1f} s)")


if __name__ == "__main__":
    main()
