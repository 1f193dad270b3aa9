"""The paper's degree n + l at K = 810, nu <= 6 (section 2.5, the regime where the basis reaches
millions): the stored values of one environment no longer fit on chip, and the graph runs on
the one-environment-per-lane kernel with its stored values in a global-memory workspace.

D = 16 (107,104 basis functions) is compared on every environment with the oracle's own index
set.  D = 20 (1,529,070 basis functions, 136,721 stored values per environment) takes the
automatic fallback; the library's index set and graph are first
checked bit for bit against the oracle's digests (tests/golden/dag_summaries.json, written by
the oracle alone), and only then are its tuples used to evaluate the oracle's naive sum on
sampled environments (building the oracle's own 1.5-million set here would take minutes)."""
import hashlib
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle.basis import IndexSet, o3_basis, workload_index_set
from oracle.evaluate import error_scale, grad_error_scale, grad_naive, phi_naive
from tests.metrics import normalized_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL32 = 1e-5
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("kernel", ["loeg", "loeg2"])
def test_paper_degree_d16_global_workspace(dev, monkeypatch, kernel):
    """Both global-workspace forms (one and two environments per lane) on the D = 16 paper-degree set."""
    from paper_2202_04140_gb300.torch_api import Dag, Spec
    monkeypatch.setenv("ACE_KERNEL", kernel)
    w = W.workload("paper_degree_d20_k810", deg_max=16)
    o = workload_index_set(w)
    s = Spec.from_workload(w)
    assert s.n_basis == o.n_basis == 107104
    d = Dag(s)
    n_env = 45
    A = W.round_to(W.draw_A(n_env, s.K), "f32")
    c = W.round_to(W.draw_c(o.deg, 1), "f32")
    At, ct = torch.tensor(A, dtype=torch.float32, device=dev), torch.tensor(c, dtype=torch.float32, device=dev)
    phi, dA = d.evaluate_grad(At, ct)
    assert normalized_error(phi.cpu().numpy(), phi_naive(A, o, c), error_scale(A, o, c)) < TOL32
    assert normalized_error(dA.cpu().numpy(), grad_naive(A, o, c), grad_error_scale(A, o, c)) < TOL32
    phi1 = d.evaluate(At, ct)
    assert normalized_error(phi1.cpu().numpy(), phi_naive(A, o, c), error_scale(A, o, c)) < TOL32
    assert d.status() == 0


def test_paper_degree_d20_automatic_fallback_sampled(dev):
    from paper_2202_04140_gb300.torch_api import Dag, Spec
    golden = json.load(open(os.path.join(ROOT, "tests", "golden", "dag_summaries.json")))
    if "paper_degree_d20_k810" not in golden:
        pytest.skip("no oracle digest for the D = 20 set")
    g = golden["paper_degree_d20_k810"]
    w = W.WORKLOADS["paper_degree_d20_k810"]
    s = Spec.from_workload(w)
    t, deg = s.tuples()
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(t, "<i4").tobytes())
    h.update(np.ascontiguousarray(deg, "<i4").tobytes())
    assert s.n_basis == g["n_basis"] and list(s.counts_per_nu) == g["counts_per_nu"]
    assert h.hexdigest() == g["spec_sha256"]          # the oracle's index set, bit for bit
    d = Dag(s)
    assert d.n_aux == g["rules"]["balanced"]["n_aux"] and d.n_nodes == g["rules"]["balanced"]["n_nodes"]
    ex = d.export()
    h = hashlib.sha256()
    for key, dt in (("left", "<i4"), ("right", "<i4"), ("is_aux", "u1"), ("basis_node", "<i4")):
        h.update(np.ascontiguousarray(ex[key], dt).tobytes())
    assert h.hexdigest() == g["rules"]["balanced"]["dag_sha256"]   # the oracle's Algorithm 1 graph
    assert d.n_slots > 65535                         # beyond the shared-memory kernels
    # the oracle's view of the same set: its own one-particle degrees, the verified tuples
    b = o3_basis(w.nmin, w.nmax, w.lmax, w.wn, w.wl)
    T = t.astype(np.int64)
    nu = (T >= 0).sum(axis=1)
    o = IndexSet(b, w.nu_max, w.deg_max, T, nu, np.where(T >= 0, b.deg[np.maximum(T, 0)], 0).sum(axis=1))
    n_env = 40
    A = W.round_to(W.draw_A(n_env, s.K), "f32")
    c = W.round_to(W.draw_c(o.deg, 1), "f32")
    phi, dA = d.evaluate_grad(torch.tensor(A, dtype=torch.float32, device=dev),
                              torch.tensor(c, dtype=torch.float32, device=dev))
    idx = [0, 31, 32, n_env - 1]                      # both tiles, first and last lanes
    sub = A[idx]
    assert normalized_error(phi.cpu().numpy()[idx], phi_naive(sub, o, c), error_scale(sub, o, c)) < TOL32
    assert normalized_error(dA.cpu().numpy()[idx], grad_naive(sub, o, c), grad_error_scale(sub, o, c)) < TOL32
    assert d.status() == 0


def test_paper_degree_d24_full_batch_sampled(dev):
    """D = 24 with the paper's degree n + l: 17,311,177 basis functions, 40,597 auxiliary nodes,
    1,104,019 stored values per environment.  The library's index set and Algorithm 1 graph are
    checked bit for bit against the oracle's digests (tests/golden/make_golden.py), then the whole
    16,384-environment batch runs in one launch (so the global workspace has its full size, one
    slice of ~1.1 M x 128 bytes per CTA) and sampled environments are compared with the oracle's
    naive sum and product-rule gradient over the verified tuples."""
    from paper_2202_04140_gb300.torch_api import Dag, Spec
    golden = json.load(open(os.path.join(ROOT, "tests", "golden", "dag_summaries.json")))
    if "paper_degree_k810" not in golden:
        pytest.skip("no oracle digest for the D = 24 set")
    g = golden["paper_degree_k810"]
    w = W.WORKLOADS["paper_degree_k810"]
    s = Spec.from_workload(w)
    t, deg = s.tuples()
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(t, "<i4").tobytes())
    h.update(np.ascontiguousarray(deg, "<i4").tobytes())
    assert s.n_basis == g["n_basis"] == 17311177 and list(s.counts_per_nu) == g["counts_per_nu"]
    assert h.hexdigest() == g["spec_sha256"]
    d = Dag(s)
    rb = g["rules"]["balanced"]
    assert d.n_aux == rb["n_aux"] == 40597 and d.n_nodes == rb["n_nodes"]
    ex = d.export()
    h = hashlib.sha256()
    for key, dt in (("left", "<i4"), ("right", "<i4"), ("is_aux", "u1"), ("basis_node", "<i4")):
        h.update(np.ascontiguousarray(ex[key], dt).tobytes())
    assert h.hexdigest() == rb["dag_sha256"]
    del ex
    b = o3_basis(w.nmin, w.nmax, w.lmax, w.wn, w.wl)
    T = t.astype(np.int64)
    del t
    nu = (T >= 0).sum(axis=1)
    o = IndexSet(b, w.nu_max, w.deg_max, T, nu, np.where(T >= 0, b.deg[np.maximum(T, 0)], 0).sum(axis=1))
    n_env = w.n_env
    A = W.round_to(W.draw_A(n_env, s.K), "f32")
    c = W.round_to(W.draw_c(o.deg, 1), "f32")
    phi, dA = d.evaluate_grad(torch.tensor(A, dtype=torch.float32, device=dev),
                              torch.tensor(c, dtype=torch.float32, device=dev))
    torch.cuda.synchronize()
    assert d.status() == 0
    idx = [0, 31, 8192, n_env - 1]                   # first and last lanes of tiles, the middle, the end
    sub = A[idx]
    assert normalized_error(phi.cpu().numpy()[idx], phi_naive(sub, o, c), error_scale(sub, o, c)) < TOL32
    dA_h = dA.cpu().numpy()[idx]
    for j in range(len(idx)):                        # one environment at a time keeps the oracle's memory low
        e = sub[j:j + 1]
        assert normalized_error(dA_h[j:j + 1], grad_naive(e, o, c), grad_error_scale(e, o, c)) < TOL32, idx[j]
