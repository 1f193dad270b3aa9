"""Host-buffer entry points (ace_eval_host, ace_eval_grad_host, ace_energy_forces_host):
chunked copies overlapped with the evaluation must give what the device entry points
give on the same inputs, for every kernel form, chunk size (automatic, ragged last
chunk, larger than the batch), pinned and pageable memory, and inside a CUDA graph;
phi is summed in a fixed order (equal bit for bit when the kernel configuration is
the same), dA with atomics (compared to 1e-5 of the condition-aware scale)."""
import numpy as np
import pytest

import workloads as W
from oracle.basis import workload_index_set
from oracle.evaluate import grad_error_scale
from tests.metrics import normalized_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL32 = 1e-5


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def case():
    from paper_2202_04140_gb300.torch_api import Spec
    w = W.WORKLOADS["fwd_grad_k392"]
    o = workload_index_set(w)
    s = Spec.from_workload(w)
    n_env = 1000
    A = W.draw_A(n_env, s.K)
    c = W.draw_c(o.deg, 1)
    pb = np.random.default_rng(7).standard_normal((n_env, 1))
    return w, o, s, A, c, pb


@pytest.mark.parametrize("kernel", ["lon", "loe", "loeg", "loeg2"])
@pytest.mark.parametrize("chunk", [0, 300, 4096])
def test_grad_host_matches_device(dev, case, kernel, chunk, monkeypatch):
    from paper_2202_04140_gb300.torch_api import Dag
    monkeypatch.setenv("ACE_KERNEL", kernel)
    w, o, s, A, c, pb = case
    d = Dag(s)
    A32 = torch.tensor(A, dtype=torch.float32)
    pb32 = torch.tensor(pb, dtype=torch.float32)
    cd = torch.tensor(c, dtype=torch.float32, device=dev)
    phi_d, dA_d = d.evaluate_grad(A32.to(dev), cd, pb32.to(dev), readout="compensated")
    phi_h, dA_h = d.evaluate_grad_host(A32.pin_memory(), cd, pb32.pin_memory(), readout="compensated",
                                       chunk_env=chunk)
    assert phi_h.device.type == "cpu" and dA_h.device.type == "cpu"
    if kernel == "lon":
        # the tile size follows the batch per SM, so chunks may sum in another grouping
        from oracle.evaluate import error_scale
        sc = error_scale(A32.double().numpy(), o, c)
        assert normalized_error(phi_h.double().numpy(), phi_d.double().cpu().numpy(), sc) < 1e-6
    else:
        assert torch.equal(phi_h, phi_d.cpu())
    scale = grad_error_scale(A32.double().numpy(), o, c, pb32.double().numpy())
    assert normalized_error(dA_h.double().numpy(), dA_d.double().cpu().numpy(), scale) < TOL32


def test_forward_host_matches_device_pageable(dev, case):
    from paper_2202_04140_gb300.torch_api import Dag
    w, o, s, A, c, pb = case
    d = Dag(s)
    A32 = torch.tensor(A, dtype=torch.float32)          # pageable: correct, not overlapped
    c16 = torch.tensor(np.random.default_rng(8).standard_normal((s.n_basis, 4)) * 1e-2, dtype=torch.float32,
                       device=dev)
    phi_d = d.evaluate(A32.to(dev), c16, readout="plain")
    phi_h = d.evaluate_host(A32, c16, readout="plain", chunk_env=257)
    assert torch.equal(phi_h, phi_d.cpu())


def test_grad_host_in_cuda_graph(dev, case):
    from paper_2202_04140_gb300.torch_api import Dag
    w, o, s, A, c, pb = case
    d = Dag(s)
    A_host = torch.tensor(A, dtype=torch.float32).pin_memory()
    phi_h = torch.empty((A.shape[0], 1), dtype=torch.float32).pin_memory()
    dA_h = torch.empty_like(A_host).pin_memory()
    cd = torch.tensor(c, dtype=torch.float32, device=dev)
    phi_d, dA_d = d.evaluate_grad(A_host.to(dev), cd, readout="plain")

    def step():
        d.evaluate_grad_host(A_host, cd, None, "plain", phi=phi_h, dA=dA_h, chunk_env=256, sync=False)

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()                                          # allocates the staging slots outside the capture
    torch.cuda.current_stream().wait_stream(side)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    phi_h.zero_()
    dA_h.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(phi_h, phi_d.cpu())
    scale = grad_error_scale(A.astype(np.float32).astype(np.float64), o, c, np.ones((A.shape[0], 1)))
    assert normalized_error(dA_h.double().numpy(), dA_d.double().cpu().numpy(), scale) < TOL32


def test_host_entry_points_reject_bad_arguments(dev, case):
    from paper_2202_04140_gb300 import ace as L
    from paper_2202_04140_gb300.torch_api import Dag
    w, o, s, A, c, pb = case
    d = Dag(s)
    A32 = torch.tensor(A[:4], dtype=torch.float32)
    cd = torch.tensor(c, dtype=torch.float32, device=dev)
    phi = torch.empty((4, 1))
    with pytest.raises(L.AceError):
        L.ace_eval_host(d.handle, A32.data_ptr(), cd.data_ptr(), 4, 1, L.ACE_F32, 0, phi.data_ptr(), -1, 0)
    with pytest.raises(L.AceError):
        L.ace_eval_grad_host(d.handle, A32.data_ptr(), cd.data_ptr(), 0, 4, 1, L.ACE_F32, 0, phi.data_ptr(), 0, 0, 0)
    # n_env = 0 binds the coefficients and copies nothing
    L.ace_eval_host(d.handle, 0, cd.data_ptr(), 0, 1, L.ACE_F32, 0, 0, 0, 0)


@pytest.mark.parametrize("chunk", [0, 37, 100000])
def test_forces_host_matches_oracle(dev, chunk):
    """ace_energy_forces_host (pooling -> forward + adjoint -> pooling adjoint in chunks) against
    the oracle's chain rule and against the device pipeline."""
    from oracle.evaluate import error_scale, grad_naive, phi_naive
    from oracle.pooling import forces, pool_A
    from paper_2202_04140_gb300.torch_api import Dag, Spec, energy_and_forces, energy_and_forces_host
    from tests.test_gpu_pool import abs_pool, force_scale, inputs
    w, offsets, P = inputs(96)
    o = workload_index_set(w)
    d = Dag(Spec.from_workload(w))
    c = W.round_to(W.draw_c(o.deg, 1), "f32")
    cd = torch.tensor(c, dtype=torch.float32, device=dev)
    P32 = torch.tensor(P, dtype=torch.float32)
    off = torch.tensor(offsets)
    phi, F = energy_and_forces_host(d, P32.pin_memory(), off.pin_memory(), cd, w.nmin, w.nmax, w.lmax, w.rc,
                                    chunk_env=chunk)
    phi_d, F_d = energy_and_forces(d, P32.to(dev), off.to(dev), cd, w.nmin, w.nmax, w.lmax, w.rc)
    # chunks cut the batch into other tiles than one call does (the fused kernel's pooling sums
    # each tile's neighbours in warp ranges): equal up to the order of the FP32 sums
    assert torch.allclose(phi, phi_d.reshape(-1).cpu(), rtol=1e-5, atol=1e-7)
    A = pool_A(P, offsets, w.nmin, w.nmax, w.lmax, w.rc)
    Aabs = abs_pool(P, offsets, w)
    assert normalized_error(phi.numpy()[:, None], phi_naive(A, o, c), error_scale(Aabs, o, c)) < TOL32
    Fref = forces(P, offsets, grad_naive(A, o, c), w.nmin, w.nmax, w.lmax, w.rc)
    S = force_scale(P, offsets, grad_naive(Aabs, o, np.abs(c)), w)
    assert normalized_error(F.numpy(), Fref, S) < TOL32


def test_forces_host_with_features_and_bad_offsets(dev):
    from paper_2202_04140_gb300 import ace as L
    from paper_2202_04140_gb300.torch_api import Dag, Spec, energy_and_forces, energy_and_forces_host
    w = W.WORKLOADS["species_forces_k375"]
    rng = np.random.default_rng(11)
    n_env = 40
    J = rng.integers(10, 61, n_env)
    offsets = np.concatenate([[0], np.cumsum(J)]).astype(np.int64)
    dirs = rng.standard_normal((offsets[-1], 3))
    P = dirs / np.linalg.norm(dirs, axis=1, keepdims=True) * (w.rc * rng.uniform(0.1, 0.99, (offsets[-1], 1)))
    mu = rng.choice([-1.0, 0.0, 1.0], offsets[-1])
    d = Dag(Spec.from_workload(w))
    cd = torch.tensor(W.round_to(W.draw_c(d.spec.deg, 1), "f32"), dtype=torch.float32, device=dev)
    P32, mu32, off = (torch.tensor(P, dtype=torch.float32), torch.tensor(mu, dtype=torch.float32),
                      torch.tensor(offsets))
    phi, F = energy_and_forces_host(d, P32, off, cd, w.nmin, w.nmax, w.lmax, w.rc, mu=mu32, kmax=w.kmax,
                                    chunk_env=13)
    phi_d, F_d = energy_and_forces(d, P32.to(dev), off.to(dev), cd, w.nmin, w.nmax, w.lmax, w.rc,
                                   mu=mu32.to(dev), kmax=w.kmax)
    # chunks of 13 environments may take another tile size than the whole batch (another summation grouping)
    assert torch.allclose(phi, phi_d.reshape(-1).cpu(), rtol=1e-5, atol=1e-6 * float(phi_d.abs().max()))
    assert torch.allclose(F, F_d.cpu(), rtol=1e-4, atol=1e-6 * float(F_d.abs().max()))
    bad = off.clone()
    bad[5] = bad[6] + 1                                   # decreasing offsets are refused on the host
    with pytest.raises(L.AceError):
        energy_and_forces_host(d, P32, bad, cd, w.nmin, w.nmax, w.lmax, w.rc, mu=mu32, kmax=w.kmax)
    with pytest.raises(L.AceError):                       # a graph over another one-particle set
        energy_and_forces_host(d, P32, off, cd, w.nmin, w.nmax, w.lmax - 1, w.rc, mu=mu32, kmax=w.kmax)


def test_grad_host_full_size_stress_against_oracle(dev):
    """The end-to-end path the benchmark times: the stress workload's whole batch (16,384
    environments, K = 810, nu <= 6) through ace_eval_grad_host with pinned host buffers and the
    automatic chunks, compared with the FP64 oracle on sampled environments, including the first
    and last of every chunk boundary region."""
    from paper_2202_04140_gb300.torch_api import Dag, Spec
    from oracle.evaluate import error_scale, grad_naive, phi_naive
    w = W.WORKLOADS["stress_k810"]
    o = workload_index_set(w)
    d = Dag(Spec.from_workload(w))
    A = W.round_to(W.draw_A(w.n_env, d.K), "f32")
    c = W.round_to(W.draw_c(o.deg, 1), "f32")
    A32 = torch.tensor(A, dtype=torch.float32).pin_memory()
    cd = torch.tensor(c, dtype=torch.float32, device=dev)
    phi_h, dA_h = d.evaluate_grad_host(A32, cd, None, readout="compensated")
    assert d.status() == 0
    n = w.n_env
    idx = np.array([0, 1, n // 3 - 1, n // 3, n // 2, 2 * n // 3 - 1, 2 * n // 3, n - 2, n - 1])
    sub = A[idx]
    phi_ref = phi_naive(sub, o, c)
    assert normalized_error(phi_h.numpy()[idx], phi_ref, error_scale(sub, o, c)) < TOL32
    assert normalized_error(dA_h.numpy()[idx], grad_naive(sub, o, c), grad_error_scale(sub, o, c)) < TOL32
