"""Write tests/golden/dag_summaries.json from the oracle alone.

For every workload and decomposition rule this records the index-set counts,
the Algorithm 1 graph counts, and SHA-256 digests of the canonical arrays:
  spec digest: int32 little-endian tuples (n_basis x nu_max, -1 padded), then int32 deg
  dag digest : int32 left, int32 right (N each, -1 for leaves), uint8 is_aux (N),
               int32 basis_node (n_basis)
The C++ builder is compared with these digests bit for bit.

Run:  python tests/golden/make_golden.py   (about 10 minutes; the largest set needs ~15 GB)
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.basis import workload_index_set   # noqa: E402
from oracle.dag import build_dag               # noqa: E402
import workloads as W                          # noqa: E402


def spec_digest(s) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(s.tuples, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(s.deg, dtype="<i4").tobytes())
    return h.hexdigest()


def dag_digest(d) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(d.left, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(d.right, dtype="<i4").tobytes())
    h.update(np.ascontiguousarray(d.is_aux, dtype="u1").tobytes())
    h.update(np.ascontiguousarray(d.basis_node, dtype="<i4").tobytes())
    return h.hexdigest()


def main():
    out = {}
    for name in ["plain_fp64_k64", "fwd_grad_k392", "uneven_16ch_k392", "stress_k810", "species_forces_k375",
                 "paper_degree_d20_k810", "paper_degree_k810"]:
        w = W.WORKLOADS[name]
        t0 = time.time()
        s = workload_index_set(w)
        rec = {"K": s.basis.K, "n_basis": s.n_basis, "counts_per_nu": s.counts_per_nu(),
               "spec_sha256": spec_digest(s), "rules": {}}
        # the 1.5- and 17.3-million-function sets: the balanced rule only (the oracle's graph build is
        # slow: about 5 minutes and 15 GB for the 17.3 million set)
        for rule in (["balanced"] if name.startswith("paper_degree") else ["balanced", "peel"]):
            d = build_dag(s, rule=rule)
            rec["rules"][rule] = {
                "n_nodes": d.n_nodes, "n_aux": d.n_aux,
                "aux_per_order": d.aux_per_order(w.nu_max),
                "nodes_order_ge2": int((d.order >= 2).sum()),
                "n_operands": d.n_operands(), "dag_sha256": dag_digest(d)}
        out[name] = rec
        print(name, rec["n_basis"], rec["rules"]["balanced"]["n_aux"],
              rec["rules"]["balanced"]["n_operands"], f"{time.time() - t0:.1f}s", flush=True)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "dag_summaries.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
