"""Host side of libace (no GPU): exported symbols, index set and graph bit-exact against the oracle,
and the evaluation plan checked by emulating the fused kernel's arithmetic on the CPU."""
import hashlib
import json
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.basis import index_set, o3_basis, so2_basis, torus_basis, workload_index_set
from oracle.dag import build_dag
from oracle.evaluate import error_scale, grad_error_scale, grad_naive, phi_naive
import workloads as W
from tests.metrics import normalized_error

L = pytest.importorskip("paper_2202_04140_gb300.ace")
from paper_2202_04140_gb300.torch_api import Dag, Spec  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = json.load(open(os.path.join(ROOT, "tests", "golden", "dag_summaries.json")))


def header_symbols():
    text = open(os.path.join(ROOT, "include", "ace.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ace_[A-Za-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    names = header_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L._lib, n), n
    assert sorted(L.EXPORTED) == names
    assert L.ace_abi_version() == 2


def spec_of(basis_kind, **kw):
    if basis_kind == "O3":
        return Spec("O3", kw["nmin"], kw["nmax"], kw["lmax"], kw["nu"], kw["D"], kw["wn"], kw["wl"],
                    kw.get("p", 1), True, kw.get("kmax", 0), kw.get("wk", 1))
    if basis_kind == "SO2":
        return Spec("SO2", kw["nmin"], kw["nmax"], kw["mmax"], kw["nu"], kw["D"], 1, 1, 1, False)
    return Spec("T", 0, 0, kw["mmax"], kw["nu"], kw["D"], 1, 1, 1, False)


CASES = [
    ("O3", dict(nmin=1, nmax=4, lmax=3, nu=3, D=10, wn=1, wl=2), lambda: o3_basis(1, 4, 3, 1, 2)),
    ("O3", dict(nmin=1, nmax=3, lmax=3, nu=4, D=9, wn=1, wl=1), lambda: o3_basis(1, 3, 3, 1, 1)),
    ("O3", dict(nmin=1, nmax=3, lmax=2, nu=3, D=5, wn=1, wl=1, p=2), lambda: o3_basis(1, 3, 2, 1, 1)),
    ("O3", dict(nmin=1, nmax=3, lmax=2, nu=3, D=3, wn=1, wl=1, p=0), lambda: o3_basis(1, 3, 2, 1, 1)),
    ("O3", dict(nmin=1, nmax=3, lmax=2, nu=4, D=7, wn=1, wl=1, kmax=2, wk=1),
     lambda: o3_basis(1, 3, 2, 1, 1, kmax=2, wk=1)),
    ("SO2", dict(nmin=1, nmax=3, mmax=4, nu=4, D=8), lambda: so2_basis(1, 3, 4)),
    ("T", dict(mmax=10, nu=5, D=10), lambda: torus_basis(10)),
]


@pytest.mark.parametrize("kind,kw,ob", CASES)
def test_spec_matches_oracle(kind, kw, ob):
    s = spec_of(kind, **kw)
    p = {1: 1, 2: 2, 0: np.inf}[kw.get("p", 1)]
    o = index_set(ob(), kw["nu"], kw["D"], p=p)
    t, d = s.tuples()
    assert np.array_equal(t, o.tuples.astype(np.int32))
    assert np.array_equal(d, o.deg.astype(np.int32))


@pytest.mark.parametrize("kind,kw,ob", CASES)
@pytest.mark.parametrize("algo,rule", [(1, "balanced"), (1, "peel"), (2, "balanced")])
def test_dag_matches_oracle(kind, kw, ob, algo, rule):
    s = spec_of(kind, **kw)
    o = index_set(ob(), kw["nu"], kw["D"], p={1: 1, 2: 2, 0: np.inf}[kw.get("p", 1)])
    od = build_dag(o, algo=algo, rule=rule, n_split=2)
    d = Dag(s, algo=algo, rule=rule, n_split=2)
    ex = d.export()
    assert d.n_nodes == od.n_nodes and d.n_aux == od.n_aux
    assert np.array_equal(ex["left"], od.left.astype(np.int32))
    assert np.array_equal(ex["right"], od.right.astype(np.int32))
    assert np.array_equal(ex["is_aux"], od.is_aux.astype(np.uint8))
    assert np.array_equal(ex["basis_node"], od.basis_node.astype(np.int32))
    assert np.array_equal(ex["level"], od.order.astype(np.int32))


# every workload, the 17.3-million-function set included (about 25 s to build)
@pytest.mark.parametrize("name", sorted(GOLDEN))
def test_workload_digests(name):
    """Bit-exact against the oracle's digests (written by tests/golden/make_golden.py)."""
    g = GOLDEN[name]
    s = Spec.from_workload(W.WORKLOADS[name])
    t, d = s.tuples()
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(t, "<i4").tobytes())
    h.update(np.ascontiguousarray(d, "<i4").tobytes())
    assert s.n_basis == g["n_basis"] and list(s.counts_per_nu) == g["counts_per_nu"]
    assert h.hexdigest() == g["spec_sha256"]
    for rule, rec in g["rules"].items():
        dag = Dag(s, rule=rule)
        ex = dag.export()
        h = hashlib.sha256()
        h.update(np.ascontiguousarray(ex["left"], "<i4").tobytes())
        h.update(np.ascontiguousarray(ex["right"], "<i4").tobytes())
        h.update(np.ascontiguousarray(ex["is_aux"], "u1").tobytes())
        h.update(np.ascontiguousarray(ex["basis_node"], "<i4").tobytes())
        assert dag.n_aux == rec["n_aux"] and dag.n_nodes == rec["n_nodes"]
        assert dag.n_operands == rec["n_operands"]
        assert h.hexdigest() == rec["dag_sha256"]


# ---- plan emulation: the fused kernel's arithmetic, in FP64 numpy, on the exported plan -----

def plan_arrays(dag, mode):
    P = {k: L.ace_dag_plan_array(dag.handle, k) for k in
         ["slot_node", "slot_basis", "n_g", "n_stored", "fwd_slot", "fwd_l", "fwd_r", "fwd_off", "rev_slot",
          "rev_l", "rev_r", "rev_off", "pull_tgt", "pull_src", "pull_par", "pull_lvl", "fwd_stored_slot",
          "fwd_stored_l", "fwd_stored_r", "fwd_stored_off"]}
    for k in ["tasks", "slice_off", "slice_steps", "col", "ebasis", "ew2", "cold_tasks", "cold_slice_off",
              "cold_slice_steps", "cold_ca", "cold_cb", "cold_ebasis", "cold_ew2"]:
        P[k] = L.ace_dag_plan_array(dag.handle, f"{mode}_{k}")
    P["tasks"] = P["tasks"].reshape(-1, 4)
    P["cold_tasks"] = P["cold_tasks"].reshape(-1, 4)
    return P


def emulate(dag, mode, A, c, phibar=None, sweep="push"):
    P = plan_arrays(dag, mode)
    n_env, K = A.shape
    n_slots = len(P["slot_node"])
    n_g = int(P["n_g"][0])
    n_stored = int(P["n_stored"][0])
    c = c.reshape(dag.n_basis, -1)
    # the tile-per-lane kernel's view: only stored slots are computed, by the stored levels
    AA = np.full((n_env, n_slots), np.nan)
    AA[:, :K] = A
    off = P["fwd_stored_off"]
    for lv in range(len(off) - 1):
        s = slice(off[lv], off[lv + 1])
        AA[:, P["fwd_stored_slot"][s]] = AA[:, P["fwd_stored_l"][s]] * AA[:, P["fwd_stored_r"][s]]
    assert not np.isnan(AA[:, :n_stored]).any()
    lin = np.where(P["slot_basis"][:, None] >= 0, c[np.maximum(P["slot_basis"], 0)], 0.0)

    def sums(pre, cols):
        """Per task and channel: the sum over its entries of coefficient x column value."""
        eb = P[pre + "ebasis"]
        vals = np.where(eb[:, None] >= 0, c[np.maximum(eb, 0)], 0.0) * np.where(P[pre + "ew2"] > 0, 2.0, 1.0)[:, None]
        n_tasks = P[pre + "tasks"].shape[0]
        task_of = np.zeros(len(eb), dtype=np.int64)
        for s_ in range(len(P[pre + "slice_steps"])):
            o, st = P[pre + "slice_off"][s_], P[pre + "slice_steps"][s_]
            idx = o + np.arange(32 * st)
            task_of[idx] = s_ * 32 + (np.arange(32 * st) % 32)
        u = np.zeros((n_env, n_tasks, c.shape[1]))
        for ch in range(c.shape[1]):
            M = sp.csr_matrix((vals[:, ch], (task_of, np.arange(len(eb)))), shape=(n_tasks, len(eb)))
            u[:, :, ch] = (M @ cols.T).T
        return u

    ucold = sums("cold_", np.nan_to_num(AA[:, P["cold_ca"]]) * np.nan_to_num(AA[:, P["cold_cb"]]))
    assert not np.isnan(AA[:, P["col"]]).any()
    u = np.concatenate([sums("", AA[:, P["col"]]), ucold], axis=1)
    T = np.concatenate([P["tasks"], P["cold_tasks"]], axis=0)
    assert np.all((T[len(P["tasks"]):, 1] & 5) == 0)          # cold tasks carry no row coefficient
    valid = T[:, 0] >= 0
    row, first, top = T[:, 0], (T[:, 1] & 1) > 0, (T[:, 1] & 2) > 0
    linr = np.where((valid & first)[:, None], lin[np.maximum(row, 0)], 0.0)
    half = 0.5 if mode == "sym" else 1.0
    # a top operand's value from its factors (it may not be stored)
    ap = np.where(top[None, :], AA[:, np.maximum(T[:, 2], 0)] * AA[:, np.maximum(T[:, 3], 0)],
                  AA[:, np.maximum(row, 0)])
    ap = np.where(valid[None, :], ap, 0.0)
    phi = np.einsum("et,etc->ec", ap * valid, linr[None] + half * u)
    if mode == "one":
        return phi, None
    pb = np.ones((n_env, c.shape[1])) if phibar is None else phibar
    g = np.einsum("ec,etc->et", pb, linr[None] + u) * valid
    G = np.zeros((n_env, n_g))
    gt = g[:, top]
    pl, pr = T[top, 2], T[top, 3]
    np.add.at(G.T, pl, (gt * AA[:, pr]).T)
    np.add.at(G.T, pr, (gt * AA[:, pl]).T)
    np.add.at(G.T, row[valid & ~top], g[:, valid & ~top].T)
    if sweep == "push":
        off = P["rev_off"]
        for lv in range(len(off) - 1):
            s = slice(off[lv], off[lv + 1])
            gs = G[:, P["rev_slot"][s]]
            np.add.at(G.T, P["rev_l"][s], (gs * AA[:, P["rev_r"][s]]).T)
            np.add.at(G.T, P["rev_r"][s], (gs * AA[:, P["rev_l"][s]]).T)
    else:
        # gather form: per level, every triple reads a consumer whose value is final
        lvl, tgt, src = P["pull_lvl"], P["pull_tgt"], P["pull_src"]
        for lv in range(len(lvl) - 1):
            j = slice(lvl[lv], lvl[lv + 1])
            assert not set(src[j].tolist()) & set(tgt[j].tolist())
            assert np.all(np.diff(tgt[j]) >= 0)
            upd = G[:, src[j]] * AA[:, P["pull_par"][j]]
            np.add.at(G.T, tgt[j], upd.T)
    return phi, G[:, :K]


@pytest.mark.parametrize("name,n_out,rule,stored", [("plain_fp64_k64", 1, "balanced", None),
                                                    ("fwd_grad_k392", 1, "balanced", None),
                                                    ("fwd_grad_k392", 3, "peel", None),
                                                    ("uneven_16ch_k392", 16, "balanced", None),
                                                    ("fwd_grad_k392", 1, "balanced", 600),
                                                    ("plain_fp64_k64", 2, "peel", 70)])
def test_plan_emulation_matches_oracle(name, n_out, rule, stored, monkeypatch):
    """The tile-per-lane kernel's arithmetic on the exported plan; with `stored` the plan keeps only
    that many slots and reads the other top operands through their factors (cold tasks)."""
    if stored is not None:
        monkeypatch.setenv("ACE_PLAN_STORED", str(stored))
    w = W.WORKLOADS[name]
    o = workload_index_set(w)
    s = Spec.from_workload(w)
    dag = Dag(s, rule=rule)
    n_stored = int(L.ace_dag_plan_array(dag.handle, "n_stored")[0])
    if stored is not None:
        assert n_stored == stored < dag.n_slots
        assert len(L.ace_dag_plan_array(dag.handle, "sym_cold_ca")) > 0
    else:
        assert n_stored == dag.n_slots
    A = W.draw_A(4, s.K, env_scale=w.env_scale)
    c = W.draw_c(o.deg, n_out)
    pb = np.random.default_rng(9).standard_normal((4, n_out))
    ref = phi_naive(A, o, c)
    scale = error_scale(A, o, c)
    for mode in ["one", "sym"]:
        phi, _ = emulate(dag, mode, A, c, pb)
        assert normalized_error(phi, ref, scale) < 1e-12
    gref = grad_naive(A, o, c, pb)
    gscale = grad_error_scale(A, o, c, pb)
    for sweep in ["push", "pull"]:
        _, dA = emulate(dag, "sym", A, c, pb, sweep=sweep)
        assert normalized_error(dA, gref, gscale) < 1e-12


def emulate_row_major(dag, mode, A, c, phibar=None):
    """The one-environment-per-lane kernel's arithmetic on the row-major task copy (one channel)."""
    P = plan_arrays(dag, mode)
    R = {k: L.ace_dag_plan_array(dag.handle, f"{mode}_rm_{k}") for k in ["tasks", "off", "col", "ebasis", "ew2"]}
    T = R["tasks"].reshape(-1, 4)
    n_env, K = A.shape
    n_g = int(P["n_g"][0])
    c = c.reshape(-1)
    AA = np.zeros((n_env, len(P["slot_node"])))
    AA[:, :K] = A
    off = P["fwd_off"]
    for lv in range(len(off) - 1):
        s = slice(off[lv], off[lv + 1])
        AA[:, P["fwd_slot"][s]] = AA[:, P["fwd_l"][s]] * AA[:, P["fwd_r"][s]]
    eb = R["ebasis"]
    vals = np.where(eb >= 0, c[np.maximum(eb, 0)], 0.0) * np.where(R["ew2"] > 0, 2.0, 1.0)
    lin = np.where(P["slot_basis"] >= 0, c[np.maximum(P["slot_basis"], 0)], 0.0)
    phi = np.zeros(n_env)
    G = np.zeros((n_env, n_g))
    pb = np.ones(n_env) if phibar is None else phibar.reshape(-1)
    for t, (row, flags, pl, pr) in enumerate(T):
        q = slice(R["off"][t], R["off"][t + 1])
        u = AA[:, R["col"][q]] @ vals[q]
        li = lin[row] if (flags & 5) == 5 else 0.0
        top = (flags & 2) > 0 and mode == "sym"
        ap = AA[:, pl] * AA[:, pr] if top else AA[:, row]
        phi += ap * (li + (0.5 if mode == "sym" else 1.0) * u)
        if mode == "sym":
            g = pb * (u + li)
            if top:
                G[:, pl] += g * AA[:, pr]
                G[:, pr] += g * AA[:, pl]
            else:
                G[:, row] += g
    if mode == "one":
        return phi, None
    off = P["rev_off"]
    for lv in range(len(off) - 1):
        for i in range(off[lv], off[lv + 1]):
            s_, l_, r_ = P["rev_slot"][i], P["rev_l"][i], P["rev_r"][i]
            gs = G[:, s_].copy()
            G[:, l_] += gs * AA[:, r_]
            G[:, r_] += gs * AA[:, l_]
    return phi, G[:, :K]


@pytest.mark.parametrize("name", ["plain_fp64_k64", "fwd_grad_k392"])
def test_row_major_plan_emulation_matches_oracle(name):
    w = W.WORKLOADS[name]
    o = workload_index_set(w)
    s = Spec.from_workload(w)
    dag = Dag(s)
    A = W.draw_A(3, s.K)
    c = W.draw_c(o.deg, 1)
    pb = np.random.default_rng(3).standard_normal((3, 1))
    ref = phi_naive(A, o, c)
    for mode in ["one", "sym"]:
        phi, _ = emulate_row_major(dag, mode, A, c, pb)
        assert normalized_error(phi[:, None], ref, error_scale(A, o, c)) < 1e-12
    _, dA = emulate_row_major(dag, "sym", A, c, pb)
    assert normalized_error(dA, grad_naive(A, o, c, pb), grad_error_scale(A, o, c, pb)) < 1e-12
    R = L.ace_dag_plan_array(dag.handle, "sym_rm_off")
    assert np.all(R % 2 == 0)


def loe_streams(dag, mode, c):
    """The per-warp streams as the plan lays them out and the binding fills them.  A task is a
    header (x, pairs << 8 | flags, z, lin) then its pairs; a block is a header (m, rows << 8 | 16)
    and two items of 4 columns (written once from the plan), then per row (flag 8) a header and
    two items of 4 coefficients in the block's column order.  Task t of the row-major copy has its
    header at loe_hpos[t]."""
    P = plan_arrays(dag, mode)
    R = {k: L.ace_dag_plan_array(dag.handle, f"{mode}_rm_{k}") for k in ["tasks", "off", "col", "ebasis", "ew2"]}
    wbeg = L.ace_dag_plan_array(dag.handle, f"{mode}_loe_wbeg")
    hpos = L.ace_dag_plan_array(dag.handle, f"{mode}_loe_hpos")
    spos = L.ace_dag_plan_array(dag.handle, f"{mode}_loe_spos")
    sval = L.ace_dag_plan_array(dag.handle, f"{mode}_loe_sval").reshape(-1, 4)
    T = R["tasks"].reshape(-1, 4)
    c = c.reshape(-1)
    items = [None] * int(wbeg[-1])
    for i in range(0, len(spos), 3):
        items[spos[i]] = ("b",) + tuple(int(v) for v in sval[i])
        for k in (1, 2):
            items[spos[i + k]] = ("cols",) + tuple(int(v) for v in sval[i + k])
    for t, (row, flags, pl, pr) in enumerate(T):
        q0, q1 = R["off"][t], R["off"][t + 1]
        b = P["slot_basis"][row]
        lin = c[b] if ((flags & 5) == 5 and b >= 0) else 0.0
        top = (flags & 2) > 0
        v = [c[R["ebasis"][q]] * (2.0 if R["ew2"][q] else 1.0) if R["ebasis"][q] >= 0 else 0.0 for q in range(q0, q1)]
        assert items[hpos[t]] is None
        if flags & 8:
            assert q1 - q0 == 8
            items[hpos[t]] = ("r", pl if top else row, flags, pr if top else 0, lin)
            for k in (0, 1):
                assert items[hpos[t] + 1 + k] is None
                items[hpos[t] + 1 + k] = ("c",) + tuple(v[4 * k:4 * k + 4])
            continue
        items[hpos[t]] = ("h", pl if top else row, ((q1 - q0) // 2) << 8 | flags, pr if top else 0, lin)
        for k in range(q0, q1, 2):
            j = hpos[t] + 1 + (k - q0) // 2
            assert items[j] is None
            items[j] = ("p", R["col"][k], v[k - q0], R["col"][k + 1], v[k + 1 - q0])
    assert all(it is not None for it in items)
    return wbeg, items, T


def emulate_loe_streams(dag, mode, A, c, phibar=None):
    """The one-environment-per-lane kernel's task loop: every warp walks its stream header by header."""
    P = plan_arrays(dag, mode)
    wbeg, items, T = loe_streams(dag, mode, c)
    n_env, K = A.shape
    n_g = int(P["n_g"][0])
    AA = np.zeros((n_env, len(P["slot_node"])))
    AA[:, :K] = A
    off = P["fwd_off"]
    for lv in range(len(off) - 1):
        s = slice(off[lv], off[lv + 1])
        AA[:, P["fwd_slot"][s]] = AA[:, P["fwd_l"][s]] * AA[:, P["fwd_r"][s]]
    phi = np.zeros(n_env)
    G = np.zeros((n_env, n_g))
    pb = np.ones(n_env) if phibar is None else phibar.reshape(-1)
    half = 0.5 if mode == "sym" else 1.0
    seen = 0

    def epilogue(x, y, z, lin, u):
        top = (y & 2) > 0
        ap = AA[:, x] * AA[:, z] if top else AA[:, x]
        phi[:] += ap * (lin + half * u)
        if mode == "sym":
            g = pb * (u + lin)
            if top:
                G[:, x] += g * AA[:, z]
                G[:, z] += g * AA[:, x]
            else:
                G[:, x] += g

    for w in range(len(wbeg) - 1):
        p = wbeg[w]
        while p < wbeg[w + 1]:
            if items[p][0] == "b":                   # a block: columns once, then its rows
                _, m, y, _, _ = items[p]
                assert y & 0xff == 16 and 1 <= m <= 8
                cols = list(items[p + 1][1:]) + list(items[p + 2][1:])
                p += 3
                for _ in range(y >> 8):
                    kind, x, yr, z, lin = items[p]
                    assert kind == "r" and yr & 8
                    cf = list(items[p + 1][1:]) + list(items[p + 2][1:])
                    u = sum(cf[j] * AA[:, cols[j]] for j in range(8))
                    epilogue(x, yr, z, lin, u)
                    p += 3
                    seen += 1
                continue
            kind, x, y, z, lin = items[p]
            assert kind == "h"
            npair = y >> 8
            u = np.zeros(n_env)
            for q in range(p + 1, p + 1 + npair):
                kind2, j0, c0, j1, c1 = items[q]
                assert kind2 == "p"
                u += c0 * AA[:, j0] + c1 * AA[:, j1]
            epilogue(x, y, z, lin, u)
            p += 1 + npair
            seen += 1
    assert seen == len(T)
    if mode == "one":
        return phi, None
    off = P["rev_off"]
    for lv in range(len(off) - 1):
        for i in range(off[lv], off[lv + 1]):
            s_, l_, r_ = P["rev_slot"][i], P["rev_l"][i], P["rev_r"][i]
            gs = G[:, s_].copy()
            G[:, l_] += gs * AA[:, r_]
            G[:, r_] += gs * AA[:, l_]
    return phi, G[:, :K]


@pytest.mark.parametrize("name", ["plain_fp64_k64", "fwd_grad_k392"])
def test_per_warp_stream_emulation_matches_oracle(name):
    w = W.WORKLOADS[name]
    o = workload_index_set(w)
    s = Spec.from_workload(w)
    dag = Dag(s)
    A = W.draw_A(3, s.K)
    c = W.draw_c(o.deg, 1)
    pb = np.random.default_rng(3).standard_normal((3, 1))
    ref = phi_naive(A, o, c)
    for mode in ["one", "sym"]:
        phi, _ = emulate_loe_streams(dag, mode, A, c, pb)
        assert normalized_error(phi[:, None], ref, error_scale(A, o, c)) < 1e-12
    _, dA = emulate_loe_streams(dag, "sym", A, c, pb)
    assert normalized_error(dA, grad_naive(A, o, c, pb), grad_error_scale(A, o, c, pb)) < 1e-12
    # the row-major tasks are in stream order; most rows of this graph are block rows
    hpos = L.ace_dag_plan_array(dag.handle, "sym_loe_hpos")
    wbeg = L.ace_dag_plan_array(dag.handle, "sym_loe_wbeg")
    assert len(wbeg) == 33 and np.all(np.diff(hpos) > 0) and hpos[-1] < wbeg[-1]
    if name == "fwd_grad_k392":
        flags = L.ace_dag_plan_array(dag.handle, "sym_rm_tasks").reshape(-1, 4)[:, 1]
        assert np.mean((flags & 8) > 0) > 0.5


def test_plan_emulation_stress_sample():
    """Largest workload (K = 810, nu <= 6): plan arithmetic against the oracle on 2 environments."""
    w = W.WORKLOADS["stress_k810"]
    s = Spec.from_workload(w)
    dag = Dag(s)
    t, d = s.tuples()
    from oracle.basis import IndexSet
    o = IndexSet(o3_basis(1, 10, 8, 1, 2), 6, 24, t.astype(np.int64), (t >= 0).sum(1).astype(np.int64),
                 d.astype(np.int64))
    A = W.draw_A(2, s.K)
    c = W.draw_c(d, 1)
    phi, dA = emulate(dag, "sym", A, c)
    ref = phi_naive(A, o, c)
    assert normalized_error(phi, ref, error_scale(A, o, c)) < 1e-12
    gref = grad_naive(A, o, c)
    assert normalized_error(dA, gref, grad_error_scale(A, o, c)) < 1e-12


def test_plan_tasks_cover_every_sink_once():
    s = Spec.from_workload(W.WORKLOADS["fwd_grad_k392"])
    dag = Dag(s)
    for mode, per_sink in [("one", 1), ("sym", 2)]:
        P = plan_arrays(dag, mode)
        eb = P["ebasis"]
        real = eb >= 0
        counts = np.bincount(eb[real], weights=np.where(P["ew2"][real] > 0, 2, 1), minlength=s.n_basis)
        sink_basis = np.unique(eb[real])
        assert np.all(counts[sink_basis] == per_sink)
        assert np.all(P["col"] < len(P["slot_node"])) and np.all(P["col"] >= 0)


def test_invalid_arguments_fail_cleanly():
    with pytest.raises(L.AceError) as e:
        L.ace_build_spec(L.ACE_GROUP_O3, 1, 2, 1, 9, 5)          # nu_max > 8
    assert e.value.status == -1
    with pytest.raises(L.AceError):
        L.ace_build_spec(7, 1, 2, 1, 2, 5)                         # unknown group
    s = Spec("O3", 1, 2, 1, 2, 5, 1, 1)
    with pytest.raises(L.AceError):
        L.ace_build_dag(s.handle, 3, 0, 2)                         # unknown algorithm
    d = Dag(s)
    with pytest.raises(L.AceError):
        L.ace_dag_plan_array(d.handle, "nonsense")
    with pytest.raises(L.AceError):                                # n_out out of range, before any CUDA call
        L.ace_eval(d.handle, 0, 0, 1, 17, L.ACE_F32, 0, 0)
    with pytest.raises(L.AceError):                                # misaligned A
        L.ace_eval(d.handle, 8, 0, 1, 1, L.ACE_F32, 0, 16)
    with pytest.raises(L.AceError):
        L.ace_pool_A(0, 0, 1, 0, 5.0, 1, 8, 9, 0)                  # lmax > 8 unsupported
    with pytest.raises(L.AceError):
        L.ace_pool_A_grad(0, 0, 1, 0, 5.0, 1, 20, 2, 0, -1.0, 0)   # more than 16 radial functions


def test_host_buffer_entry_points_check_arguments_before_the_device():
    """The host-buffer entry points reject bad requests before any CUDA call (no GPU needed):
    the CSR offsets (which the host holds), a graph over another one-particle set, the chunk size."""
    w = W.WORKLOADS["forces_k392"]
    d = Dag(Spec.from_workload(w))
    n_env = 3
    pos = np.zeros((6, 3), np.float32)
    phi = np.zeros(n_env, np.float32)
    F = np.zeros((6, 3), np.float32)
    ptr = lambda a: a.ctypes.data

    def call(off, lmax=w.lmax, chunk=0, n_pairs=6):
        L.ace_energy_forces_host(d.handle, ptr(pos), 0, ptr(off), n_env, n_pairs, 0, 0, w.rc, w.nmin, w.nmax,
                                 lmax, 0, ptr(phi), ptr(F), chunk, 0)

    for bad in ([0, 4, 2, 6], [1, 2, 4, 6], [0, 2, 4, 5]):      # decreasing, not from 0, not to n_pairs
        with pytest.raises(L.AceError) as e:
            call(np.array(bad, np.int64))
        assert e.value.status == -1 and "offsets" in str(e.value)
    good = np.array([0, 2, 4, 6], np.int64)
    with pytest.raises(L.AceError) as e:
        call(good, lmax=w.lmax - 1)                               # K of the graph != pooling basis
    assert e.value.status == -1 and "K" in str(e.value)
    with pytest.raises(L.AceError) as e:
        call(good, chunk=-1)
    assert e.value.status == -1
    A = np.zeros((2, d.K), np.float32)
    with pytest.raises(L.AceError) as e:
        L.ace_eval_grad_host(d.handle, ptr(A), 0, 0, 2, 1, L.ACE_F32, 0, 0, 0, 0, 0)   # dA NULL
    assert e.value.status == -1
    with pytest.raises(L.AceError) as e:
        L.ace_eval_host(d.handle, ptr(A), 0, 2, 1, L.ACE_F32, 0, ptr(phi), -5, 0)      # chunk_env < 0
    assert e.value.status == -1


def test_plain_f64_sizes_refused_without_wrapping():
    """Huge n_env: the workspace query and the allocation-free entry point refuse it before any CUDA
    call, also where n_env x bytes per environment wraps around size_t to a small number."""
    d = Dag(Spec.from_workload(W.WORKLOADS["fwd_grad_k392"]))
    per_env = d.n_nodes * 8 * 2                                   # FP64 values and adjoints
    wrap = (2 ** 64 + per_env - 1) // per_env                     # n_env * per_env = 2^64 + small
    assert (wrap * per_env) % 2 ** 64 < 2 ** 25
    buf = np.zeros(64, np.float64)
    p = buf.ctypes.data
    for n_env in (wrap, 2 ** 62, 2 ** 63 - 1):
        with pytest.raises(L.AceError) as e:
            L.ace_eval_plain_workspace_bytes(d.handle, n_env, 1)
        assert e.value.status == -1
        with pytest.raises(L.AceError) as e:
            L.ace_eval_plain_f64_static(d.handle, p, p, 0, n_env, 1, p, p, 0)
        assert e.value.status == -1 and "static scratch" in str(e.value)
    assert L.ace_eval_plain_workspace_bytes(d.handle, 10, 1) == 10 * per_env


def _slice_bank_loads(tasks, rows):
    """Per slice of 32 tasks: the largest number of distinct first targets (run heads) and of second
    targets that share a bank (row mod 32) once mapped through rows."""
    a_load = b_load = 0
    for sl in tasks.reshape(-1, 32, 4):
        v = sl[:, 0] >= 0
        if not v.any():
            continue
        top = ((sl[:, 1] & 2) != 0) & v
        heads = np.unique(np.where(top, sl[:, 2], sl[:, 0])[v])
        a_load += np.bincount(rows[heads] % 32, minlength=32).max()
        if top.any():
            b_load += np.bincount(rows[sl[top, 3]] % 32, minlength=32).max()
    return a_load, b_load


@pytest.mark.parametrize("name", ["fwd_grad_k392", "stress_k810"])
def test_adjoint_row_permutation(name):
    """The tile kernel's adjoint rows: g_perm is a permutation of the n_g slots with an adjoint; slices
    repeat a second target only where the slice had to be completed from the tasks that followed
    (a repeat is two updates of one address, still correct); and the rows spread the updates one
    warp issues together over the banks better than the slots themselves do."""
    d = Dag(Spec.from_workload(W.WORKLOADS[name]))
    n_g = int(L.ace_dag_plan_array(d.handle, "n_g")[0])
    perm = L.ace_dag_plan_array(d.handle, "g_perm")
    assert sorted(perm.tolist()) == list(range(n_g))
    tasks = L.ace_dag_plan_array(d.handle, "sym_tasks")
    slices = tasks.reshape(-1, 32, 4)
    repeats = 0
    for sl in slices:
        top = ((sl[:, 1] & 2) != 0) & (sl[:, 0] >= 0)
        repeats += len(np.unique(sl[top, 3])) < int(top.sum())
    if name == "stress_k810":   # 8 of 736 slices with this plan
        assert repeats <= 0.02 * len(slices)
    ident = _slice_bank_loads(tasks, np.arange(n_g))
    permuted = _slice_bank_loads(tasks, perm)
    assert sum(permuted) < sum(ident)
    if name == "stress_k810":   # measured with this plan: 826 + 1,239 against 1,206 + 2,071
        assert sum(permuted) <= 0.7 * sum(ident)


def test_device_forces_entry_point_checks_arguments_before_the_device():
    """ace_energy_forces (device buffers) rejects bad requests before any CUDA call (no GPU needed): a
    graph over another one-particle set, missing outputs, a non-positive cutoff, sizes out of range;
    ace_energy_forces_plan rejects a missing graph."""
    w = W.WORKLOADS["forces_k392"]
    d = Dag(Spec.from_workload(w))
    buf = np.zeros(64, np.float32)
    off = np.zeros(4, np.int64)
    p = buf.ctypes.data

    def call(lmax=w.lmax, rc=w.rc, phi=p, forces=p, n_env=3, n_pairs=6, nmin=w.nmin):
        L.ace_energy_forces(d.handle, p, 0, off.ctypes.data, n_env, n_pairs, 0, 0, rc, nmin, w.nmax, lmax, 0,
                            phi, forces, 0)

    for kw, word in ((dict(lmax=w.lmax - 1), "K"), (dict(phi=0), "NULL"), (dict(forces=0), "NULL"),
                     (dict(rc=0.0), "rc"), (dict(n_env=-1), ">= 0"), (dict(nmin=w.nmax + 1), "nmin")):
        with pytest.raises(L.AceError) as e:
            call(**kw)
        assert e.value.status == -1 and word in str(e.value), (kw, str(e.value))
    with pytest.raises(L.AceError) as e:
        L.ace_energy_forces_plan(0, w.nmin, w.nmax, w.lmax, 0)
    assert e.value.status == -1


def test_binding_without_the_library_fails_loudly(tmp_path):
    """The product path has no fallback: a copy of the package without libace.so cannot be imported
    (the ctypes binding and the tensor API both raise ImportError naming the missing library)."""
    import shutil
    import subprocess
    import sys
    pkg = tmp_path / "paper_2202_04140_gb300"
    pkg.mkdir()
    for name in os.listdir(os.path.join(ROOT, "paper_2202_04140_gb300")):
        if name.endswith(".py"):
            shutil.copy(os.path.join(ROOT, "paper_2202_04140_gb300", name), pkg / name)
    assert not (pkg / "libace.so").exists()
    for mod in ("paper_2202_04140_gb300.ace", "paper_2202_04140_gb300.torch_api"):
        r = subprocess.run([sys.executable, "-c", f"import {mod}"], cwd=tmp_path, capture_output=True, text=True,
                           env={**os.environ, "PYTHONPATH": str(tmp_path)})
        assert r.returncode != 0, mod
        assert "ImportError" in r.stderr and "libace.so is not built" in r.stderr, r.stderr[-500:]


def test_tile_layout_only_where_the_tile_kernel_can_run():
    """A plan that keeps more than 65,535 slots (the 1.5-million-function set, D = 20) has no
    tile-per-lane layout: no hot or cold tasks, offset lists holding only their final 0, every
    entry still in the row-major streams.  A plan within the limit (K = 392, nu <= 4) keeps its layout."""
    for name, big in (("paper_degree_d20_k810", True), ("fwd_grad_k392", False)):
        dag = Dag(Spec.from_workload(W.WORKLOADS[name]))
        n_stored = int(L.ace_dag_plan_array(dag.handle, "n_stored")[0])
        assert (n_stored > 65535) == big
        for mode in ("sym", "one"):
            tasks = L.ace_dag_plan_array(dag.handle, f"{mode}_tasks")
            slice_off = L.ace_dag_plan_array(dag.handle, f"{mode}_slice_off")
            cold_off = L.ace_dag_plan_array(dag.handle, f"{mode}_cold_slice_off")
            rm_off = L.ace_dag_plan_array(dag.handle, f"{mode}_rm_off")
            assert len(rm_off) > 1 and rm_off[-1] > 0
            if big:
                assert len(tasks) == 0 and list(slice_off) == [0] and list(cold_off) == [0]
                assert len(L.ace_dag_plan_array(dag.handle, f"{mode}_col")) == 0
            else:
                assert len(tasks) > 0 and slice_off[-1] == len(L.ace_dag_plan_array(dag.handle, f"{mode}_col"))
        assert dag.n_entries > 0


@pytest.mark.parametrize("name,algo,stored", [(n, 1, None) for n in sorted(W.WORKLOADS)] +
                         [("fwd_grad_k392", 2, None), ("stress_k810", 2, None), ("fwd_grad_k392", 1, "600"),
                          ("stress_k810", 1, "6000")])
def test_plan_passes_the_library_validation(name, algo, stored, monkeypatch):
    """Every workload's plan (Algorithm 1 and 2; the paper-degree sets without a tile layout; plans
    forced onto the cold path by a small stored-slot limit) passes the host check
    that the first upload runs before anything reaches the device."""
    if stored:
        monkeypatch.setenv("ACE_PLAN_STORED", stored)
    dag = Dag(Spec.from_workload(W.WORKLOADS[name]), algo=algo)
    L.ace_dag_validate(dag.handle)
    if stored:
        assert len(L.ace_dag_plan_array(dag.handle, "sym_cold_tasks")) > 0


def test_per_warp_stream_emulation_paper_degree_d20():
    """The streams the global-workspace kernels walk for the 1.5-million-function set (a plan
    without a tile layout): forward and adjoint in FP64 on 2 environments against the oracle's
    term-by-term sums (about 35 s)."""
    w = W.WORKLOADS["paper_degree_d20_k810"]
    o = workload_index_set(w)
    s = Spec.from_workload(w)
    dag = Dag(s)
    A = W.draw_A(2, s.K, env_scale=w.env_scale)
    c = W.draw_c(o.deg, 1)
    pb = np.random.default_rng(3).standard_normal((2, 1))
    phi, dA = emulate_loe_streams(dag, "sym", A, c, pb)
    assert normalized_error(phi[:, None], phi_naive(A, o, c), error_scale(A, o, c)) < 1e-12
    assert normalized_error(dA, grad_naive(A, o, c, pb), grad_error_scale(A, o, c, pb)) < 1e-12
