"""GPU parity with invariant features (phi_nlmk = R_n Y_lm T_k(mu), section "Invariant features"):
feature pooling and its adjoint for several shapes, and the full pooling -> graph -> forces
pipeline on the species workload, against the FP64 oracle through the C ABI."""
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


def scales(P, offsets, mu, kmax, nmin, nmax, lmax, rc, G):
    """Normalisers: sum_j |phi_k(r_j)| for A, sum_k |G_k| |grad phi_k| (term-wise) for forces."""
    phi, _ = one_particle(P, nmin, nmax, lmax, rc, mu=mu, kmax=kmax)
    g = one_particle_grad_bound(P, nmin, nmax, lmax, rc, mu=mu, kmax=kmax)
    SA = np.zeros((len(offsets) - 1, phi.shape[1]))
    SF = np.zeros((P.shape[0], 3))
    for e in range(len(offsets) - 1):
        a, b = offsets[e], offsets[e + 1]
        SA[e] = np.abs(phi[a:b]).sum(axis=0)
        SF[a:b] = np.einsum("k,jkd->jd", np.abs(G[e]), np.abs(g[a:b]))
    return SA, SF


@pytest.mark.parametrize("nmin,nmax,lmax,kmax,n_species", [(1, 5, 4, 2, 3), (0, 3, 6, 3, 4), (1, 8, 2, 1, 2),
                                                          (1, 4, 8, 0, 0)])
def test_feature_pool_and_adjoint(dev, nmin, nmax, lmax, kmax, n_species):
    from paper_2202_04140_gb300.torch_api import pool_A as gpu_pool, pool_A_grad
    offsets, P = W.draw_neighbours(23, seed=8, rc=5.0, j_range=(0, 45))
    P = W.round_to(P, "f32")
    mu = W.round_to(W.draw_species(P.shape[0], n_species), "f32") if kmax > 0 else None
    Pt, ot = torch.tensor(P, dtype=torch.float32, device=dev), torch.tensor(offsets, device=dev)
    mt = torch.tensor(mu, dtype=torch.float32, device=dev) if mu is not None else None
    A = gpu_pool(Pt, ot, nmin, nmax, lmax, 5.0, mt, kmax).cpu().numpy()
    ref = pool_A(P, offsets, nmin, nmax, lmax, 5.0, mu=mu, kmax=kmax)
    G = np.random.default_rng(2).standard_normal(ref.shape)
    SA, SF = scales(P, offsets, mu, kmax, nmin, nmax, lmax, 5.0, G)
    assert normalized_error(A, ref, SA) < TOL32
    dpos = pool_A_grad(Pt, ot, torch.tensor(G, dtype=torch.float32, device=dev), nmin, nmax, lmax, 5.0,
                       mu=mt, kmax=kmax)
    Fref = -forces(P, offsets, G, nmin, nmax, lmax, 5.0, mu=mu, kmax=kmax)
    assert normalized_error(dpos.cpu().numpy(), Fref, SF) < TOL32


def test_species_forces_pipeline(dev):
    from paper_2202_04140_gb300.torch_api import Dag, Spec, energy_and_forces
    w = W.WORKLOADS["species_forces_k375"]
    o = workload_index_set(w)
    s = Spec.from_workload(w)
    assert s.n_basis == o.n_basis and s.K == w.K
    d = Dag(s)
    offsets, P = W.draw_neighbours(64, rc=w.rc, j_range=w.j_range)
    P = W.round_to(P, "f32")
    mu = W.round_to(W.draw_species(P.shape[0], w.n_species), "f32")
    c = W.round_to(W.draw_c(o.deg, 1), "f32")
    phi, F = energy_and_forces(d, torch.tensor(P, dtype=torch.float32, device=dev), torch.tensor(offsets, device=dev),
                               torch.tensor(c, dtype=torch.float32, device=dev), w.nmin, w.nmax, w.lmax, w.rc,
                               mu=torch.tensor(mu, dtype=torch.float32, device=dev), kmax=w.kmax)
    A = pool_A(P, offsets, w.nmin, w.nmax, w.lmax, w.rc, mu=mu, kmax=w.kmax)
    SA, _ = scales(P, offsets, mu, w.kmax, w.nmin, w.nmax, w.lmax, w.rc, np.zeros_like(A))
    assert normalized_error(phi.cpu().numpy(), phi_naive(A, o, c), error_scale(SA, o, c)) < TOL32
    G = grad_naive(A, o, c)
    Gabs = grad_naive(SA, o, np.abs(c))
    _, SF = scales(P, offsets, mu, w.kmax, w.nmin, w.nmax, w.lmax, w.rc, Gabs)
    Fref = forces(P, offsets, G, w.nmin, w.nmax, w.lmax, w.rc, mu=mu, kmax=w.kmax)
    assert normalized_error(F.cpu().numpy(), Fref, SF) < TOL32
