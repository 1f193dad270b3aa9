"""The fused kernels on graphs other than the five workloads: Algorithm 2 (section 3.3), the
SO(2) and torus bases (sections 2.2, 2.3), the paper's own O(3) degree n + l and the p = 2 and
p = infinity degree sets (section 2.5).  The graph evaluation does not depend on what the
one-particle functions are, so A is drawn directly; phi and dphi/dA are compared with the
oracle's naive sum over its own index set."""
import numpy as np
import pytest

import workloads as W
from oracle.basis import index_set, o3_basis, so2_basis, torus_basis
from oracle.evaluate import error_scale, grad_error_scale, grad_naive, phi_naive
from tests.metrics import normalized_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL32, TOL64 = 1e-5, 1e-12

CASES = {
    "torus_nu5_D10": (dict(group="T", nmin=0, nmax=0, lmax=10, nu_max=5, deg_max=10, wn=1, wl=1, p_norm=1,
                           require_l_even=False), lambda: (torus_basis(10), 5, 10, 1)),
    "so2_nu4_D10": (dict(group="SO2", nmin=1, nmax=4, lmax=6, nu_max=4, deg_max=10, wn=1, wl=1, p_norm=1,
                         require_l_even=False), lambda: (so2_basis(1, 4, 6), 4, 10, 1)),
    "o3_paper_degree_nu4_D8": (dict(group="O3", nmin=1, nmax=5, lmax=4, nu_max=4, deg_max=8, wn=1, wl=1, p_norm=1,
                                    require_l_even=True), lambda: (o3_basis(1, 5, 4, 1, 1), 4, 8, 1)),
    "o3_p2_nu3_D5": (dict(group="O3", nmin=1, nmax=4, lmax=3, nu_max=3, deg_max=5, wn=1, wl=1, p_norm=2,
                          require_l_even=True), lambda: (o3_basis(1, 4, 3, 1, 1), 3, 5, 2)),
    "o3_pinf_nu3_D3": (dict(group="O3", nmin=1, nmax=3, lmax=2, nu_max=3, deg_max=3, wn=1, wl=1, p_norm=0,
                            require_l_even=True), lambda: (o3_basis(1, 3, 2, 1, 1), 3, 3, np.inf)),
}


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


@pytest.mark.parametrize("algo", [1, 2])
@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("kernel", ["lon", "loe", "loeg", "loeg2"])
def test_graph_variants(dev, case, algo, kernel, monkeypatch):
    from paper_2202_04140_gb300.torch_api import Dag, Spec
    monkeypatch.setenv("ACE_KERNEL", kernel)
    params, oracle_args = CASES[case]
    basis, nu, D, p = oracle_args()
    o = index_set(basis, nu, D, p=p)
    s = Spec(**params)
    assert s.n_basis == o.n_basis
    d = Dag(s, algo=algo, n_split=2)
    n_env = 70
    A = W.round_to(W.draw_A(n_env, s.K, seed=5), "f32")
    c = W.round_to(W.draw_c(o.deg, 1, seed=6), "f32")
    At = torch.tensor(A, dtype=torch.float32, device=dev)
    ct = torch.tensor(c, dtype=torch.float32, device=dev)
    phi, dA = d.evaluate_grad(At, ct)
    assert normalized_error(phi.cpu().numpy(), phi_naive(A, o, c), error_scale(A, o, c)) < TOL32
    assert normalized_error(dA.cpu().numpy(), grad_naive(A, o, c), grad_error_scale(A, o, c)) < TOL32
    phi1 = d.evaluate(At, ct)
    assert normalized_error(phi1.cpu().numpy(), phi_naive(A, o, c), error_scale(A, o, c)) < TOL32
    if kernel == "lon":     # FP64 runs on the tile-per-lane kernel only
        phi64, dA64 = d.evaluate_grad(At.double(), ct.double())
        assert normalized_error(phi64.cpu().numpy(), phi_naive(A, o, c), error_scale(A, o, c)) < TOL64
        assert normalized_error(dA64.cpu().numpy(), grad_naive(A, o, c), grad_error_scale(A, o, c)) < TOL64
