"""GPU parity of the pooling kernels and the full forces pipeline against the FP64 oracle (C ABI).

A is gated by |A - ref| / sum_j |R_n Y_lm|; forces by |F - ref| / (the oracle's
forces assembled from |G| and |grad phi_k|); phi by the usual normaliser.
"""
import numpy as np
import pytest

import workloads as W
from oracle.basis import workload_index_set
from oracle.evaluate import error_scale, grad_naive, phi_naive
from oracle.pooling import forces, one_particle, one_particle_grad_bound, pool_A
from tests.metrics import normalized_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL32 = 1e-5


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def abs_pool(P, offsets, w):
    phi, _ = one_particle(P, w.nmin, w.nmax, w.lmax, w.rc)
    A = np.zeros((len(offsets) - 1, phi.shape[1]))
    for e in range(A.shape[0]):
        A[e] = np.abs(phi[offsets[e]:offsets[e + 1]]).sum(axis=0)
    return A


def force_scale(P, offsets, G, w):
    g = one_particle_grad_bound(P, w.nmin, w.nmax, w.lmax, w.rc)
    S = np.zeros((P.shape[0], 3))
    for e in range(len(offsets) - 1):
        a, b = offsets[e], offsets[e + 1]
        S[a:b] = np.einsum("k,jkd->jd", np.abs(G[e]), np.abs(g[a:b]))
    return S


def inputs(n_env, seed=3, j_range=(10, 60)):
    w = W.WORKLOADS["forces_k392"]
    offsets, P = W.draw_neighbours(n_env, seed=seed, rc=w.rc, j_range=j_range)
    return w, offsets, W.round_to(P, "f32")


def test_pool_matches_oracle(dev):
    from paper_2202_04140_gb300.torch_api import pool_A as gpu_pool
    w, offsets, P = inputs(200)
    A = gpu_pool(torch.tensor(P, dtype=torch.float32, device=dev), torch.tensor(offsets, device=dev),
                 w.nmin, w.nmax, w.lmax, w.rc).cpu().numpy()
    ref = pool_A(P, offsets, w.nmin, w.nmax, w.lmax, w.rc)
    assert normalized_error(A, ref, abs_pool(P, offsets, w)) < TOL32


@pytest.mark.parametrize("lmax,nmin,nmax", [(0, 1, 3), (3, 0, 5), (8, 1, 16)])
def test_pool_other_shapes(dev, lmax, nmin, nmax):
    from paper_2202_04140_gb300.torch_api import pool_A as gpu_pool, pool_A_grad
    offsets, P = W.draw_neighbours(9, seed=8, rc=5.0, j_range=(0, 40))
    P = W.round_to(P, "f32")
    Pt, ot = torch.tensor(P, dtype=torch.float32, device=dev), torch.tensor(offsets, device=dev)
    A = gpu_pool(Pt, ot, nmin, nmax, lmax, 5.0).cpu().numpy()
    ref = pool_A(P, offsets, nmin, nmax, lmax, 5.0)
    phi, _ = one_particle(P, nmin, nmax, lmax, 5.0)
    g = one_particle_grad_bound(P, nmin, nmax, lmax, 5.0)
    scale = np.zeros_like(ref)
    for e in range(len(offsets) - 1):
        scale[e] = np.abs(phi[offsets[e]:offsets[e + 1]]).sum(axis=0)
    assert normalized_error(A, ref, scale) < TOL32
    G = np.random.default_rng(2).standard_normal(ref.shape)
    dpos = pool_A_grad(Pt, ot, torch.tensor(G, dtype=torch.float32, device=dev), nmin, nmax, lmax, 5.0)
    Fref = -forces(P, offsets, G, nmin, nmax, lmax, 5.0)
    S = np.zeros_like(Fref)
    for e in range(len(offsets) - 1):
        a, b = offsets[e], offsets[e + 1]
        S[a:b] = np.einsum("k,jkd->jd", np.abs(G[e]), np.abs(g[a:b]))
    assert normalized_error(dpos.cpu().numpy(), Fref, S) < TOL32


def test_forces_pipeline_small_batch(dev):
    """pooling -> fused forward + adjoint -> pooling adjoint, against the oracle's chain rule."""
    from paper_2202_04140_gb300.torch_api import Dag, Spec, energy_and_forces
    w, offsets, P = inputs(96)
    o = workload_index_set(w)
    s = Spec.from_workload(w)
    d = Dag(s)
    c = W.round_to(W.draw_c(o.deg, 1), "f32")
    phi, F = energy_and_forces(d, torch.tensor(P, dtype=torch.float32, device=dev),
                               torch.tensor(offsets, device=dev), torch.tensor(c, dtype=torch.float32, device=dev),
                               w.nmin, w.nmax, w.lmax, w.rc)
    A = pool_A(P, offsets, w.nmin, w.nmax, w.lmax, w.rc)
    ref = phi_naive(A, o, c)
    Aabs = abs_pool(P, offsets, w)
    assert normalized_error(phi.cpu().numpy(), ref, error_scale(Aabs, o, c)) < TOL32
    G = grad_naive(A, o, c)
    Fref = forces(P, offsets, G, w.nmin, w.nmax, w.lmax, w.rc)
    Gabs = grad_naive(Aabs, o, np.abs(c))
    assert normalized_error(F.cpu().numpy(), Fref, force_scale(P, offsets, Gabs, w)) < TOL32


def test_forces_permutation_invariance(dev):
    from paper_2202_04140_gb300.torch_api import Dag, Spec, energy_and_forces
    w, offsets, P = inputs(8)
    s = Spec.from_workload(w)
    d = Dag(s)
    c = torch.tensor(W.round_to(W.draw_c(s.deg, 1), "f32"), dtype=torch.float32, device=dev)
    perm = np.arange(P.shape[0])
    for e in range(len(offsets) - 1):
        a, b = offsets[e], offsets[e + 1]
        perm[a:b] = a + np.random.default_rng(e).permutation(b - a)
    ot = torch.tensor(offsets, device=dev)
    phi1, F1 = energy_and_forces(d, torch.tensor(P, dtype=torch.float32, device=dev), ot, c,
                                 w.nmin, w.nmax, w.lmax, w.rc)
    phi2, F2 = energy_and_forces(d, torch.tensor(P[perm], dtype=torch.float32, device=dev), ot, c,
                                 w.nmin, w.nmax, w.lmax, w.rc)
    assert torch.allclose(phi1, phi2, rtol=1e-5, atol=1e-6)
    assert torch.allclose(F1[torch.tensor(perm, device=dev)], F2, rtol=1e-4, atol=1e-6)


def test_forces_full_size_sampled(dev):
    """50k environments in one pipeline call; sampled environments against the oracle."""
    from paper_2202_04140_gb300.torch_api import Dag, Spec, energy_and_forces
    w, offsets, P = inputs(w_n := W.WORKLOADS["forces_k392"].n_env)
    o = workload_index_set(w)
    d = Dag(Spec.from_workload(w))
    c = W.round_to(W.draw_c(o.deg, 1), "f32")
    phi, F = energy_and_forces(d, torch.tensor(P, dtype=torch.float32, device=dev),
                               torch.tensor(offsets, device=dev), torch.tensor(c, dtype=torch.float32, device=dev),
                               w.nmin, w.nmax, w.lmax, w.rc)
    phi, F = phi.cpu().numpy(), F.cpu().numpy()
    for e in [0, 12345, w_n - 1]:
        a, b = offsets[e], offsets[e + 1]
        Pe, oe = P[a:b], np.array([0, b - a])
        A = pool_A(Pe, oe, w.nmin, w.nmax, w.lmax, w.rc)
        Aabs = abs_pool(Pe, oe, w)
        assert normalized_error(phi[e:e + 1], phi_naive(A, o, c), error_scale(Aabs, o, c)) < TOL32
        G = grad_naive(A, o, c)
        Gabs = grad_naive(Aabs, o, np.abs(c))
        Fref = forces(Pe, oe, G, w.nmin, w.nmax, w.lmax, w.rc)
        assert normalized_error(F[a:b], Fref, force_scale(Pe, oe, Gabs, w)) < TOL32


def test_pool_and_adjoint_next_to_centre_and_cutoff(dev):
    """Neighbours at r ~ 1e-6 and at r ~ rc (1 - 1e-6), also on the coordinate axes: the FP32
    geometry (error-free r^2, Newton-refined 1/r, 1 - r/rc from rc^2 - r^2) keeps A and the
    adjoint within the gate even where R_n(r) ~ (1 - r/rc)^2 ~ 1e-12."""
    from paper_2202_04140_gb300.torch_api import pool_A as gpu_pool, pool_A_grad
    w = W.WORKLOADS["forces_k392"]
    rc = w.rc
    rng = np.random.default_rng(31)

    def cloud(n, radii, axes=False):
        d = rng.standard_normal((n, 3))
        if axes:                                    # +-x, +-y or +-z, per point
            d = np.zeros((n, 3))
            d[np.arange(n), rng.integers(0, 3, n)] = rng.choice([-1.0, 1.0], n)
        d /= np.linalg.norm(d, axis=1)[:, None]
        return d * radii[:, None]

    clouds = [cloud(20, 1e-6 * rng.uniform(1, 10, 20)),                       # next to the centre
              cloud(20, rc * (1 - 1e-6 * rng.uniform(1, 10, 20))),            # next to the cutoff
              cloud(12, np.concatenate([1e-6 * rng.uniform(1, 10, 6), rc * (1 - 1e-6 * rng.uniform(1, 10, 6))]),
                    axes=True),
              np.concatenate([cloud(10, rc * (1 - 1e-6 * rng.uniform(1, 10, 10))),
                              cloud(10, rc * rng.uniform(0, 1, 10) ** (1 / 3))])]
    P = W.round_to(np.concatenate(clouds), "f32")
    assert np.all(np.linalg.norm(P, axis=1) < rc) and np.all(np.linalg.norm(P, axis=1) > 0)
    offsets = np.concatenate([[0], np.cumsum([len(c) for c in clouds])]).astype(np.int64)
    Pt, ot = torch.tensor(P, dtype=torch.float32, device=dev), torch.tensor(offsets, device=dev)
    A = gpu_pool(Pt, ot, w.nmin, w.nmax, w.lmax, rc).cpu().numpy()
    ref = pool_A(P, offsets, w.nmin, w.nmax, w.lmax, rc)
    assert normalized_error(A, ref, abs_pool(P, offsets, w)) < TOL32
    G = rng.standard_normal(ref.shape)
    dpos = pool_A_grad(Pt, ot, torch.tensor(G, dtype=torch.float32, device=dev), w.nmin, w.nmax, w.lmax, rc)
    Fref = -forces(P, offsets, G, w.nmin, w.nmax, w.lmax, rc)
    assert normalized_error(dpos.cpu().numpy(), Fref, force_scale(P, offsets, G, w)) < TOL32


def _ragged_cloud(n_env, rc, seed):
    """Neighbour clouds with an empty environment, one of 150 neighbours (several staging passes
    and warp ranges) and one neighbour outside the cutoff (its forces are zero)."""
    rng = np.random.default_rng(seed)
    J = rng.integers(1, 71, size=n_env)
    J[3] = 0
    J[min(40, n_env - 1)] = 150
    offsets = np.concatenate([[0], np.cumsum(J)]).astype(np.int64)
    d = rng.standard_normal((int(offsets[-1]), 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    r = rc * rng.uniform(0.05, 1.0, d.shape[0]) ** (1.0 / 3.0)
    r[offsets[5]] = 1.2 * rc
    return offsets, W.round_to(d * r[:, None], "f32")


def _kernels_run(fn):
    """fn() and the names of the kernels it launched (the first profiler session of a process can
    come back empty, so a throwaway session runs first)."""
    from torch.profiler import ProfilerActivity, profile
    for _ in range(2):
        with profile(activities=[ProfilerActivity.CUDA]) as prof:
            out = fn()
            torch.cuda.synchronize()
    return out, {e.key for e in prof.key_averages()}


@pytest.mark.parametrize("readout", ["plain", "compensated", "fp64"])
def test_fused_forces_kernel_matches_three_kernels_and_oracle(dev, monkeypatch, readout):
    """ace_energy_forces in both forms: the one-kernel pipeline (pooling, graph forward and adjoint,
    pooling adjoint per tile of 32 environments in shared memory, ACE_FORCES=fused) and the three
    kernels (ACE_FORCES=split), against the oracle's chain rule on a ragged batch: 77 environments
    (two full tiles and 13), an empty environment, one of 150 neighbours, one neighbour beyond the
    cutoff."""
    from paper_2202_04140_gb300 import ace as L
    from paper_2202_04140_gb300.torch_api import Dag, Spec, energy_and_forces
    w = W.WORKLOADS["forces_k392"]
    offsets, P = _ragged_cloud(77, w.rc, seed=8)
    o = workload_index_set(w)
    d = Dag(Spec.from_workload(w))
    c = W.round_to(W.draw_c(o.deg, 1, seed=9), "f32")
    ct = torch.tensor(c, dtype=torch.float32, device=dev)
    Pt, ot = torch.tensor(P, dtype=torch.float32, device=dev), torch.tensor(offsets, device=dev)
    run = lambda: energy_and_forces(d, Pt, ot, ct, w.nmin, w.nmax, w.lmax, w.rc, readout=readout)
    monkeypatch.setenv("ACE_FORCES", "fused")
    fused, smem = L.ace_energy_forces_plan(d.handle, w.nmin, w.nmax, w.lmax, w.kmax)
    assert fused and smem > 0
    (phi_f, F_f), k_fused = _kernels_run(run)
    monkeypatch.setenv("ACE_FORCES", "split")
    assert L.ace_energy_forces_plan(d.handle, w.nmin, w.nmax, w.lmax, w.kmax) == (False, 0)
    (phi_s, F_s), k_split = _kernels_run(run)
    monkeypatch.delenv("ACE_FORCES")
    if any("pool_grad_kernel" in k for k in k_split):   # the profiler sees the library's kernels
        assert any("forces_fused_kernel" in k for k in k_fused), sorted(k_fused)
        assert not any("forces_fused_kernel" in k for k in k_split), sorted(k_split)
    A = pool_A(P, offsets, w.nmin, w.nmax, w.lmax, w.rc)
    Aabs = abs_pool(P, offsets, w)
    ref = phi_naive(A, o, c)
    Fref = forces(P, offsets, grad_naive(A, o, c), w.nmin, w.nmax, w.lmax, w.rc)
    S = force_scale(P, offsets, grad_naive(Aabs, o, np.abs(c)), w)
    for phi, F in ((phi_f, F_f), (phi_s, F_s)):
        phi, F = phi.cpu().numpy().reshape(-1, 1), F.cpu().numpy()
        assert normalized_error(phi, ref, error_scale(Aabs, o, c)) < TOL32
        assert normalized_error(F, Fref, S) < TOL32
        assert phi[3, 0] == 0.0
        assert np.all(F[offsets[5]] == 0.0)


@pytest.mark.parametrize("form", ["fused", "split"])
def test_forces_empty_batch_and_full_size_forms_agree(dev, monkeypatch, form):
    """No environments: nothing launched, nothing written.  50k environments: both forms agree
    within the FP32 gate on every environment and every neighbour."""
    from paper_2202_04140_gb300.torch_api import Dag, Spec, energy_and_forces
    w = W.WORKLOADS["forces_k392"]
    s = Spec.from_workload(w)
    d = Dag(s)
    c = torch.tensor(W.round_to(W.draw_c(s.deg, 1), "f32"), dtype=torch.float32, device=dev)
    monkeypatch.setenv("ACE_FORCES", form)
    phi, F = energy_and_forces(d, torch.zeros((0, 3), device=dev), torch.zeros(1, dtype=torch.int64, device=dev), c,
                               w.nmin, w.nmax, w.lmax, w.rc)
    assert phi.shape == (0, 1) and F.shape == (0, 3)
    if form == "split":
        return
    offsets, P = W.draw_neighbours(w.n_env, seed=3, rc=w.rc, j_range=w.j_range)
    Pt = torch.tensor(W.round_to(P, "f32"), dtype=torch.float32, device=dev)
    ot = torch.tensor(offsets, device=dev)
    phi_f, F_f = energy_and_forces(d, Pt, ot, c, w.nmin, w.nmax, w.lmax, w.rc)
    monkeypatch.setenv("ACE_FORCES", "split")
    phi_s, F_s = energy_and_forces(d, Pt, ot, c, w.nmin, w.nmax, w.lmax, w.rc)
    monkeypatch.delenv("ACE_FORCES")
    assert (phi_f - phi_s).abs().max().item() <= 1e-4 * phi_s.abs().max().item()
    assert (F_f - F_s).abs().max().item() <= 1e-4 * F_s.abs().max().item()
