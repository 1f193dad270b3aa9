"""CUDA-graph capture of the library's launches: the fused forward + adjoint
kernels (both forms) and the full pooling -> graph -> forces pipeline are
captured once on static buffers and replayed with new inputs copied in; every
replay must match the FP64 oracle on those inputs."""
import numpy as np
import pytest

import workloads as W
from oracle.basis import workload_index_set
from oracle.evaluate import error_scale, grad_error_scale, grad_naive, phi_naive
from tests.metrics import normalized_error
from tests.test_gpu_pool import abs_pool, force_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL32 = 1e-5


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _capture(fn):
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        fn()
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        out = fn()
    return g, out


@pytest.mark.parametrize("kernel", ["lon", "loe", "loeg", "loeg2"])
def test_graph_replay_fused_grad(dev, kernel, monkeypatch):
    from paper_2202_04140_gb300.torch_api import Dag, Spec
    monkeypatch.setenv("ACE_KERNEL", kernel)
    w = W.WORKLOADS["fwd_grad_k392"]
    o = workload_index_set(w)
    d = Dag(Spec.from_workload(w))
    n_env = 200
    c = W.round_to(W.draw_c(o.deg, 1), "f32")
    ct = torch.tensor(c, dtype=torch.float32, device=dev)
    A_static = torch.zeros((n_env, d.K), dtype=torch.float32, device=dev)
    g, (phi, dA) = _capture(lambda: d.evaluate_grad(A_static, ct))
    for seed in (21, 22):
        A = W.round_to(W.draw_A(n_env, d.K, seed=seed), "f32")
        A_static.copy_(torch.tensor(A, device=dev))
        g.replay()
        torch.cuda.synchronize()
        assert normalized_error(phi.cpu().numpy(), phi_naive(A, o, c), error_scale(A, o, c)) < TOL32
        assert normalized_error(dA.cpu().numpy(), grad_naive(A, o, c), grad_error_scale(A, o, c)) < TOL32


def test_graph_replay_forces_pipeline(dev):
    from oracle.pooling import forces as oracle_forces, pool_A as oracle_pool
    from paper_2202_04140_gb300.torch_api import Dag, Spec, energy_and_forces
    w = W.WORKLOADS["forces_k392"]
    o = workload_index_set(w)
    d = Dag(Spec.from_workload(w))
    n_env = 40
    offsets, P = W.draw_neighbours(n_env, rc=w.rc, j_range=w.j_range)
    c = W.round_to(W.draw_c(o.deg, 1), "f32")
    ct = torch.tensor(c, dtype=torch.float32, device=dev)
    off_t = torch.tensor(offsets, device=dev)
    P_static = torch.zeros((P.shape[0], 3), dtype=torch.float32, device=dev)
    P_static.copy_(torch.tensor(W.round_to(P, "f32"), device=dev))
    g, (phi, F) = _capture(lambda: energy_and_forces(d, P_static, off_t, ct, w.nmin, w.nmax, w.lmax, w.rc))
    for seed in (0, 1):
        Pi = W.round_to(P if seed == 0 else P[np.random.default_rng(7).permutation(P.shape[0])], "f32")
        P_static.copy_(torch.tensor(Pi, device=dev))
        g.replay()
        torch.cuda.synchronize()
        A = oracle_pool(Pi, offsets, w.nmin, w.nmax, w.lmax, w.rc)
        Aabs = abs_pool(Pi, offsets, w)
        assert normalized_error(phi.cpu().numpy(), phi_naive(A, o, c), error_scale(Aabs, o, c)) < TOL32
        ref_F = oracle_forces(Pi, offsets, grad_naive(A, o, c), w.nmin, w.nmax, w.lmax, w.rc)
        Gabs = grad_naive(Aabs, o, np.abs(c))
        assert normalized_error(F.cpu().numpy(), ref_F, force_scale(Pi, offsets, Gabs, w)) < TOL32
