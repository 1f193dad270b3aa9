"""Graph files (ace_dag_save / ace_dag_load): a saved graph reads back identical, with the same
plan, and a damaged or foreign file is refused with ACE_ERR_INVALID_ARG before it is used.

The file layout tested here is the one ace_dag_save documents: a 104-byte header (magic,
version, the 12 index-set parameters, 4 build options, K, n_basis, the index set's checksum, N),
then left, right and order of the N nodes and the basis nodes as int32, then the FNV-1a 64-bit
checksum of everything before it.  Tampered files get a correct checksum, so that the checks
behind it are the ones exercised."""
import os
import struct

import numpy as np
import pytest

import workloads as W

L = pytest.importorskip("paper_2202_04140_gb300.ace")
from paper_2202_04140_gb300.torch_api import Dag, Spec  # noqa: E402

HEADER = 104


def fnv1a64(data: bytes) -> int:
    """FNV-1a, 64-bit (offset basis 14695981039346656037, prime 1099511628211)."""
    h = 14695981039346656037
    for b in data:
        h = ((h ^ b) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def rewrite(path: str, body: bytes):
    """Write body followed by its FNV-1a checksum (a tampered but well-formed file)."""
    with open(path, "wb") as f:
        f.write(body + struct.pack("<Q", fnv1a64(body)))


def small_dag(**kw):
    return Dag(Spec.from_workload(W.WORKLOADS["plain_fp64_k64"]), **kw)


def plan_arrays(dag):
    names = ["slot_node", "slot_basis", "fwd_slot", "rev_slot", "sym_tasks", "sym_col", "sym_rm_tasks",
             "sym_rm_col", "sym_loe_wbeg", "one_rm_tasks", "g_perm", "n_stored"]
    return {k: L.ace_dag_plan_array(dag.handle, k) for k in names}


@pytest.mark.parametrize("make", [
    lambda: Dag(Spec.from_workload(W.WORKLOADS["fwd_grad_k392"])),
    lambda: Dag(Spec.from_workload(W.WORKLOADS["fwd_grad_k392"]), rule="peel"),
    lambda: Dag(Spec.from_workload(W.WORKLOADS["fwd_grad_k392"]), algo=2, n_split=2),
    lambda: Dag(Spec.from_workload(W.WORKLOADS["species_forces_k375"])),
    lambda: Dag(Spec("SO2", nmin=0, nmax=4, lmax=4, nu_max=4, deg_max=8, wn=1, wl=1)),
    lambda: Dag(Spec("T", lmax=6, nu_max=5, deg_max=10), algo=2, n_split=1),
    lambda: Dag(Spec("O3", nmin=1, nmax=4, lmax=3, nu_max=4, deg_max=5, p_norm=0)),
    lambda: Dag(Spec.from_workload(W.WORKLOADS["paper_degree_d20_k810"])),
], ids=["fwd_grad", "fwd_grad_peel", "fwd_grad_alg2", "species", "so2", "torus_alg2", "o3_pinf", "paper_d20"])
def test_saved_graph_reads_back_identical(make, tmp_path):
    d = make()
    p = str(tmp_path / "g.acegraph")
    d.save(p)
    e = Dag.load(p)
    assert (e.spec.group, e.spec.n_basis, e.spec.K) == (d.spec.group, d.spec.n_basis, d.spec.K)
    assert list(e.spec.counts_per_nu) == list(d.spec.counts_per_nu)
    assert np.array_equal(e.spec.tuples()[0], d.spec.tuples()[0])
    assert (e.n_nodes, e.n_aux, e.n_operands, e.n_levels) == (d.n_nodes, d.n_aux, d.n_operands, d.n_levels)
    a, b = d.export(), e.export()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    pa, pb = plan_arrays(d), plan_arrays(e)
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k
    L.ace_dag_validate(e.handle)


def test_damaged_and_foreign_files_are_refused(tmp_path):
    d = small_dag()
    p = str(tmp_path / "g.acegraph")
    d.save(p)
    raw = open(p, "rb").read()
    body = raw[:-8]
    assert struct.unpack("<Q", raw[-8:])[0] == fnv1a64(body)          # the documented checksum
    N, nb = d.n_nodes, d.n_basis
    assert struct.unpack_from("<q", body, HEADER - 8)[0] == N
    assert len(body) == HEADER + 4 * (3 * N + nb)
    left = np.frombuffer(body, "<i4", N, HEADER).copy()
    bnode = np.frombuffer(body, "<i4", nb, HEADER + 12 * N).copy()
    order = np.frombuffer(body, "<i4", N, HEADER + 8 * N).copy()
    bad = str(tmp_path / "bad.acegraph")

    def refused(data, words, write=None):
        if write is None:
            open(bad, "wb").write(data)
        else:
            rewrite(bad, data)
        with pytest.raises(L.AceError) as err:
            Dag.load(bad)
        assert err.value.status == L.ACE_ERR_INVALID_ARG and words in str(err.value), str(err.value)

    # a flipped byte, a truncated file, another file type
    flipped = bytearray(raw)
    flipped[HEADER + 4 * (N // 2)] ^= 1
    refused(bytes(flipped), "checksum")
    refused(raw[:-100], "checksum")
    refused(b"not a graph file at all", "not a graph file")
    # well-formed files with a wrong version, other index-set parameters, a wrong graph
    refused(body[:8] + struct.pack("<I", 99) + body[12:], "version", write=True)
    deg_max_at = 8 + 4 + 4 * 5
    other = struct.unpack_from("<i", body, deg_max_at)[0] + 1
    refused(body[:deg_max_at] + struct.pack("<i", other) + body[deg_max_at + 4:], "another index set", write=True)
    i = int(np.flatnonzero(left >= 0)[0])                               # first node of order >= 2
    self_ref = left.copy()
    self_ref[i] = i
    refused(body[:HEADER] + self_ref.astype("<i4").tobytes() + body[HEADER + 4 * N:], "not earlier", write=True)
    # two basis functions of the same order exchange their nodes: each node is now another product
    nu = order[bnode]
    same = np.flatnonzero(nu == nu.max())
    swapped = bnode.copy()
    swapped[same[0]], swapped[same[1]] = bnode[same[1]], bnode[same[0]]
    refused(body[:HEADER + 12 * N] + swapped.astype("<i4").tobytes(), "another product", write=True)
    # a node listed twice as a basis node
    twice = bnode.copy()
    twice[same[1]] = bnode[same[0]]
    refused(body[:HEADER + 12 * N] + twice.astype("<i4").tobytes(), "basis node", write=True)
    # sizes that do not match the header
    refused(body + b"\0\0\0\0", "sizes", write=True)


def test_save_and_load_check_their_arguments(tmp_path):
    d = small_dag()
    other = Spec.from_workload(W.WORKLOADS["fwd_grad_k392"])
    with pytest.raises(L.AceError) as err:
        L.ace_dag_save(other.handle, d.handle, str(tmp_path / "x"))
    assert err.value.status == L.ACE_ERR_INVALID_ARG and "not built from this index set" in str(err.value)
    with pytest.raises(L.AceError) as err:
        L.ace_dag_load(str(tmp_path / "missing.acegraph"))
    assert err.value.status == L.ACE_ERR_INVALID_ARG and "cannot open" in str(err.value)
    with pytest.raises(L.AceError) as err:
        d.save(str(tmp_path / "no_such_dir" / "g.acegraph"))
    assert err.value.status == L.ACE_ERR_INVALID_ARG and "cannot open" in str(err.value)
    assert os.path.exists(str(tmp_path)) and not os.path.exists(str(tmp_path / "x"))
