"""GPU parity of the fused graph kernels against the FP64 oracle, through the C ABI.

Gates (normalised error |x - ref| / scale, scale = the oracle with |A|, |c|, |phibar|):
FP64 paths 1e-12, FP32 paths 1e-5.  Small workloads are compared on every
environment; full-size workloads run in the launch configuration the benchmark
uses and are compared on sampled environments the oracle evaluates one by one.
"""
import numpy as np
import pytest

import workloads as W
from oracle.basis import workload_index_set
from oracle.evaluate import error_scale, grad_error_scale, grad_naive, phi_naive
from tests.metrics import normalized_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32, TOL64 = 1e-5, 1e-12


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


_CACHE = {}


def setup(name, n_env=None, n_out=None, rule="balanced"):
    """Oracle index set, the library's graph, and the workload's inputs (FP64 draws)."""
    from paper_2202_04140_gb300.torch_api import Dag, Spec
    key = (name, rule)
    if key not in _CACHE:
        w = W.WORKLOADS[name]
        o = workload_index_set(w)
        s = Spec.from_workload(w)
        _CACHE[key] = (w, o, s, Dag(s, rule=rule))
    w, o, s, d = _CACHE[key]
    n_env = n_env or w.n_env
    n_out = n_out or w.n_out
    A = W.draw_A(n_env, s.K, env_scale=w.env_scale)
    c = W.draw_c(o.deg, n_out)
    return w, o, d, A, c


def t(x, dtype, dev):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=dev)


def to_f32(x):
    return W.round_to(x, "f32")


# ---- FP64 ----------------------------------------------------------------------------------

def test_plain_fp64_k64_fused_and_plain(dev):
    w, o, d, A, c = setup("plain_fp64_k64")
    ref = phi_naive(A, o, c)
    scale = error_scale(A, o, c)
    phi = d.evaluate(t(A, torch.float64, dev), t(c, torch.float64, dev)).cpu().numpy()
    assert normalized_error(phi, ref, scale) < TOL64
    phi_p, dA_p = d.evaluate_plain_f64(t(A, torch.float64, dev), t(c, torch.float64, dev), grad=True)
    assert normalized_error(phi_p.cpu().numpy(), ref, scale) < TOL64
    gref = grad_naive(A, o, c)
    gscale = grad_error_scale(A, o, c)
    assert normalized_error(dA_p.cpu().numpy(), gref, gscale) < TOL64
    phi_g, dA = d.evaluate_grad(t(A, torch.float64, dev), t(c, torch.float64, dev))
    assert normalized_error(phi_g.cpu().numpy(), ref, scale) < TOL64
    assert normalized_error(dA.cpu().numpy(), gref, gscale) < TOL64


@pytest.mark.parametrize("n_out", [1, 3, 16])
def test_fwd_grad_k392_fp64(dev, n_out):
    w, o, d, A, c = setup("fwd_grad_k392", n_env=257, n_out=n_out)
    pb = np.random.default_rng(11).standard_normal((A.shape[0], n_out))
    phi, dA = d.evaluate_grad(t(A, torch.float64, dev), t(c, torch.float64, dev), t(pb, torch.float64, dev))
    assert normalized_error(phi.cpu().numpy(), phi_naive(A, o, c), error_scale(A, o, c)) < TOL64
    assert normalized_error(dA.cpu().numpy(), grad_naive(A, o, c, pb), grad_error_scale(A, o, c, pb)) < TOL64


# ---- FP32: the forward + adjoint workload (K = 392, nu <= 4, D = 16, 4096 environments) ---------

@pytest.mark.parametrize("kernel", ["lon", "loe", "loeg", "loeg2"])
@pytest.mark.parametrize("readout", ["plain", "compensated", "fp64"])
def test_fwd_grad_k392_fp32_all_envs(dev, readout, kernel, monkeypatch):
    """Both fused kernels (tiles of tasks per lane, and one environment per lane) on every environment."""
    monkeypatch.setenv("ACE_KERNEL", kernel)
    w, o, d, A, c = setup("fwd_grad_k392")
    A32, c32 = to_f32(A), to_f32(c)
    phi, dA = d.evaluate_grad(t(A32, torch.float32, dev), t(c32, torch.float32, dev), readout=readout)
    assert normalized_error(phi.cpu().numpy(), phi_naive(A32, o, c32), error_scale(A32, o, c32)) < TOL32
    assert normalized_error(dA.cpu().numpy(), grad_naive(A32, o, c32), grad_error_scale(A32, o, c32)) < TOL32
    phi1 = d.evaluate(t(A32, torch.float32, dev), t(c32, torch.float32, dev), readout=readout)
    assert normalized_error(phi1.cpu().numpy(), phi_naive(A32, o, c32), error_scale(A32, o, c32)) < TOL32


def test_fwd_grad_k392_autograd_and_finite_differences(dev):
    """autograd.Function backward = the adjoint kernel; central differences (h = 1e-6, FP64 path) agree."""
    w, o, d, A, c = setup("fwd_grad_k392", n_env=64)
    A32, c32 = to_f32(A), to_f32(c)
    At = t(A32, torch.float32, dev).requires_grad_(True)
    e = d.energy(At, t(c32, torch.float32, dev))
    e.sum().backward()
    g32 = At.grad.cpu().numpy()
    gscale = grad_error_scale(A32, o, c32)
    assert normalized_error(g32, grad_naive(A32, o, c32), gscale) < TOL32
    A64 = t(A32, torch.float64, dev)
    c64 = t(c32, torch.float64, dev)
    rng = np.random.default_rng(4)
    h = 1e-6
    for _ in range(32):
        ei, k = int(rng.integers(A.shape[0])), int(rng.integers(A.shape[1]))
        Ap, Am = A64.clone(), A64.clone()
        Ap[ei, k] += h
        Am[ei, k] -= h
        fd = (d.evaluate(Ap, c64) - d.evaluate(Am, c64))[ei, 0].item() / (2 * h)
        assert abs(fd - g32[ei, k]) <= TOL32 * gscale[ei, k] + 1e-7 * abs(fd)


@pytest.mark.parametrize("kernel", ["lon", "loe", "loeg", "loeg2"])
def test_coefficient_rebinding_and_edge_sizes(dev, kernel, monkeypatch):
    """n_env = 0 is a no-op; n_env = 1 and ragged tiles; c bound once then reused; new c rebinds."""
    monkeypatch.setenv("ACE_KERNEL", kernel)
    from paper_2202_04140_gb300 import ace as L
    w, o, d, A, c = setup("fwd_grad_k392", n_env=37)
    A32, c32 = to_f32(A), to_f32(c)
    At, ct = t(A32, torch.float32, dev), t(c32, torch.float32, dev)
    for n in [1, 2, 5, 17, 37]:
        phi = d.evaluate(At[:n], ct).cpu().numpy()
        assert normalized_error(phi, phi_naive(A32[:n], o, c32), error_scale(A32[:n], o, c32)) < TOL32
    c2 = to_f32(2.0 * c32)
    phi2 = d.evaluate(At, t(c2, torch.float32, dev)).cpu().numpy()
    assert normalized_error(phi2, phi_naive(A32, o, c2), error_scale(A32, o, c2)) < TOL32
    # a new coefficient tensor at a recycled address is bound again (no stale coefficients)
    for scale in (3.0, 5.0):
        cs = to_f32(scale * c32)
        phis = d.evaluate(At, t(cs, torch.float32, dev)).cpu().numpy()
        assert normalized_error(phis, phi_naive(A32, o, cs), error_scale(A32, o, cs)) < TOL32
    # an in-place update of the bound tensor is seen (its version changes)
    cin = t(c32, torch.float32, dev)
    d.evaluate(At, cin)
    cin.mul_(2.0)
    phii = d.evaluate(At, cin).cpu().numpy()
    assert normalized_error(phii, phi_naive(A32, o, c2), error_scale(A32, o, c2)) < TOL32
    empty = torch.empty((0, d.K), dtype=torch.float32, device=dev)
    assert d.evaluate(empty, ct).shape == (0, 1)          # binds c32 again, evaluates nothing
    # c = NULL reuses the coefficients bound by the previous call (c32 here)
    phi3 = torch.empty((37, 1), dtype=torch.float32, device=dev)
    L.ace_eval(d.handle, At.data_ptr(), 0, 37, 1, L.ACE_F32, 0, phi3.data_ptr(),
               torch.cuda.current_stream().cuda_stream)
    assert normalized_error(phi3.cpu().numpy(), phi_naive(A32, o, c32), error_scale(A32, o, c32)) < TOL32


@pytest.mark.parametrize("kernel", ["lon", "loe", "loeg", "loeg2"])
def test_checked_mode_status_word(dev, monkeypatch, kernel):
    """Bounds-checked kernels run clean on a valid plan and leave the status word at ACE_OK."""
    monkeypatch.setenv("ACE_CHECKED", "1")
    monkeypatch.setenv("ACE_KERNEL", kernel)
    w, o, d, A, c = setup("fwd_grad_k392", n_env=33)
    A32, c32 = to_f32(A), to_f32(c)
    phi, dA = d.evaluate_grad(t(A32, torch.float32, dev), t(c32, torch.float32, dev))
    assert d.status() == 0
    assert normalized_error(dA.cpu().numpy(), grad_naive(A32, o, c32), grad_error_scale(A32, o, c32)) < TOL32


# ---- FP32: 16 output channels, per-environment scales (K = 392, nu <= 5, D = 20) ---------------

@pytest.mark.parametrize("readout", ["plain", "compensated"])
def test_uneven_16ch_small_batch(dev, readout):
    w, o, d, A, c = setup("uneven_16ch_k392", n_env=301)
    A32, c32 = to_f32(A), to_f32(c)
    phi = d.evaluate(t(A32, torch.float32, dev), t(c32, torch.float32, dev), readout=readout).cpu().numpy()
    assert normalized_error(phi, phi_naive(A32, o, c32), error_scale(A32, o, c32)) < TOL32


def test_uneven_16ch_full_size_sampled(dev):
    w, o, d, A, c = setup("uneven_16ch_k392")
    A32, c32 = to_f32(A), to_f32(c)
    phi = d.evaluate(t(A32, torch.float32, dev), t(c32, torch.float32, dev), readout="compensated").cpu().numpy()
    idx = np.sort(np.random.default_rng(5).choice(A.shape[0], 48, replace=False))
    idx = np.concatenate([[0], idx, [A.shape[0] - 1]])
    sub = A32[idx]
    assert normalized_error(phi[idx], phi_naive(sub, o, c32), error_scale(sub, o, c32)) < TOL32
    assert np.all(np.isfinite(phi))


@pytest.mark.parametrize("readout", ["plain", "compensated", "fp64"])
@pytest.mark.parametrize("n_out", [2, 3, 16])
def test_several_channels_env_per_lane(dev, readout, n_out, monkeypatch):
    """The several-channel forward kernel (one environment per lane, coefficient rows read once per
    warp, stored values in the global workspace): 301 environments (a ragged last tile of 13)."""
    monkeypatch.setenv("ACE_KERNEL", "loem")
    w, o, d, A, c = setup("uneven_16ch_k392", n_env=301, n_out=n_out)
    A32, c32 = to_f32(A), to_f32(c)
    phi = d.evaluate(t(A32, torch.float32, dev), t(c32, torch.float32, dev), readout=readout).cpu().numpy()
    assert phi.shape == (301, n_out)
    assert normalized_error(phi, phi_naive(A32, o, c32), error_scale(A32, o, c32)) < TOL32
    assert d.status() == 0


def test_several_channels_env_per_lane_full_size_and_refusals(dev, monkeypatch):
    """All 100,000 environments of the 16-channel workload in one launch (every CTA's workspace
    slice in use), sampled against the oracle; the form refuses adjoint and one-channel requests."""
    monkeypatch.setenv("ACE_KERNEL", "loem")
    w, o, d, A, c = setup("uneven_16ch_k392")
    A32, c32 = to_f32(A), to_f32(c)
    At, ct = t(A32, torch.float32, dev), t(c32, torch.float32, dev)
    phi = d.evaluate(At, ct, readout="compensated").cpu().numpy()
    idx = np.sort(np.random.default_rng(6).choice(A.shape[0], 48, replace=False))
    idx = np.concatenate([[0, 31, 32], idx, [A.shape[0] - 1]])
    sub = A32[idx]
    assert normalized_error(phi[idx], phi_naive(sub, o, c32), error_scale(sub, o, c32)) < TOL32
    assert np.all(np.isfinite(phi)) and d.status() == 0
    from paper_2202_04140_gb300.ace import AceError
    with pytest.raises(AceError):
        d.evaluate_grad(At[:64], ct)
    with pytest.raises(AceError):
        d.evaluate(At[:64], ct[:, :1].contiguous())


# ---- FP32: the stress workload (K = 810, nu <= 6, D = 24, 16384 environments) ----------------------

def test_stress_k810_full_size_sampled(dev):
    w, o, d, A, c = setup("stress_k810")
    A32, c32 = to_f32(A), to_f32(c)
    phi, dA = d.evaluate_grad(t(A32, torch.float32, dev), t(c32, torch.float32, dev))
    phi, dA = phi.cpu().numpy(), dA.cpu().numpy()
    idx = np.sort(np.random.default_rng(6).choice(A.shape[0], 10, replace=False))
    idx = np.concatenate([[0], idx, [A.shape[0] - 1]])
    sub = A32[idx]
    assert normalized_error(phi[idx], phi_naive(sub, o, c32), error_scale(sub, o, c32)) < TOL32
    assert normalized_error(dA[idx], grad_naive(sub, o, c32), grad_error_scale(sub, o, c32)) < TOL32
    assert np.all(np.isfinite(phi)) and np.all(np.isfinite(dA))


def test_stress_k810_forward_only_matches_adjoint_pass(dev):
    w, o, d, A, c = setup("stress_k810", n_env=600)
    A32, c32 = to_f32(A), to_f32(c)
    At, ct = t(A32, torch.float32, dev), t(c32, torch.float32, dev)
    phi1 = d.evaluate(At, ct).cpu().numpy()
    phi2, _ = d.evaluate_grad(At, ct)
    sub = A32[:6]
    ref = phi_naive(sub, o, c32)
    scale = error_scale(sub, o, c32)
    assert normalized_error(phi1[:6], ref, scale) < TOL32
    assert normalized_error(phi2.cpu().numpy()[:6], ref, scale) < TOL32


def test_stress_k810_fp64_sampled(dev):
    w, o, d, A, c = setup("stress_k810", n_env=40)
    phi, dA = d.evaluate_grad(t(A, torch.float64, dev), t(c, torch.float64, dev))
    sub = slice(0, 4)
    assert normalized_error(phi.cpu().numpy()[sub], phi_naive(A[sub], o, c), error_scale(A[sub], o, c)) < TOL64
    assert normalized_error(dA.cpu().numpy()[sub], grad_naive(A[sub], o, c),
                            grad_error_scale(A[sub], o, c)) < TOL64


# ---- kernel configurations: every tile size, and the autotuner ---------------------------------

@pytest.mark.parametrize("dtype,E", [("f32", 1), ("f32", 2), ("f32", 4), ("f32", 8), ("f32", 16),
                                     ("f64", 1), ("f64", 2), ("f64", 4), ("f64", 8)])
def test_every_tile_size(dev, dtype, E, monkeypatch):
    """The tile-per-lane kernel with each compiled environments-per-CTA E (ragged last tile)."""
    from paper_2202_04140_gb300.ace import AceError
    monkeypatch.setenv("ACE_KERNEL", "lon")
    monkeypatch.setenv("ACE_TILE_E", str(E))
    w, o, d, A, c = setup("fwd_grad_k392", n_env=8 * E + 3)
    tol = TOL32 if dtype == "f32" else TOL64
    if dtype == "f32":
        A, c = to_f32(A), to_f32(c)
    td = torch.float32 if dtype == "f32" else torch.float64
    try:
        phi, dA = d.evaluate_grad(t(A, td, dev), t(c, td, dev))
    except AceError as e:
        assert "shared memory" in str(e)
        pytest.skip(f"E={E} does not fit in shared memory for this graph")
    assert normalized_error(phi.cpu().numpy(), phi_naive(A, o, c), error_scale(A, o, c)) < tol
    assert normalized_error(dA.cpu().numpy(), grad_naive(A, o, c), grad_error_scale(A, o, c)) < tol


@pytest.mark.parametrize("name,n_out,grad", [("fwd_grad_k392", 1, True), ("uneven_16ch_k392", 16, False)])
def test_autotune_then_evaluate(dev, name, n_out, grad):
    from paper_2202_04140_gb300.torch_api import Dag
    w, o, _, A, c = setup(name, n_env=301)
    d = Dag(_CACHE[(name, "balanced")][2])          # own graph handle: the tuned choice stays local
    res = d.autotune(n_env=4096, n_out=n_out, dtype=torch.float32, grad=grad)
    assert res["kernel"] in ("tile_per_lane", "env_per_lane", "env_per_lane_global", "env_per_lane_multi",
                             "env_pair_per_lane_global") and res["ms"] > 0
    if res["kernel"] == "tile_per_lane":
        assert res["E"] in (1, 2, 4, 8, 16)
    if n_out > 1:
        assert res["kernel"] in ("tile_per_lane", "env_per_lane_multi")
    else:
        assert res["kernel"] != "env_per_lane_multi"
    A32, c32 = to_f32(A), to_f32(c)
    At, ct = t(A32, torch.float32, dev), t(c32, torch.float32, dev)
    ref, scale = phi_naive(A32, o, c32), error_scale(A32, o, c32)
    if grad:
        phi, dA = d.evaluate_grad(At, ct)
        assert normalized_error(dA.cpu().numpy(), grad_naive(A32, o, c32), grad_error_scale(A32, o, c32)) < TOL32
    else:
        phi = d.evaluate(At, ct)
    assert normalized_error(phi.cpu().numpy(), ref, scale) < TOL32


@pytest.mark.parametrize("name,n_env", [("stress_k810", 301), ("fwd_grad_k392", 77), ("uneven_16ch_k392", 45)])
def test_bulk_copy_staging_matches_plain_loads(dev, name, n_env, monkeypatch):
    """Tiles read through the bulk-copy staging buffer give the same results as direct loads of A
    (K = 810 rows are not 16-byte multiples: every tile has an unaligned head and tail).  phi is
    bit-identical (fixed summation order); dphi/dA is summed with shared-memory atomics, whose
    order varies from run to run, so both are compared with the oracle."""
    monkeypatch.setenv("ACE_KERNEL", "lon")
    w, o, d, A, c = setup(name, n_env=n_env)
    At, ct = t(to_f32(A), torch.float32, dev), t(to_f32(c), torch.float32, dev)
    run = (lambda: d.evaluate_grad(At, ct)) if w.grad else (lambda: (d.evaluate(At, ct), None))
    monkeypatch.setenv("ACE_STAGE", "1")
    p1, g1 = run()
    monkeypatch.setenv("ACE_STAGE", "0")
    p0, g0 = run()
    assert torch.equal(p1, p0)
    assert d.status() == 0
    sub, c32 = to_f32(A)[[0, 1, n_env - 1]], to_f32(c)
    assert normalized_error(p1.cpu().numpy()[[0, 1, n_env - 1]], phi_naive(sub, o, c32),
                            error_scale(sub, o, c32)) < TOL32
    if g1 is not None:
        ref, scale = grad_naive(sub, o, c32), grad_error_scale(sub, o, c32)
        for g in (g1, g0):
            assert normalized_error(g.cpu().numpy()[[0, 1, n_env - 1]], ref, scale) < TOL32


def test_staging_wait_times_out_and_reports(dev, monkeypatch):
    """The bounded wait of the staged copy: with the copies never issued (test hook), the first wait
    of every CTA gives up after about a second, the kernel reads A directly, the results are still
    right, and the status word reports the time-out (ACE_ERR_TIMEOUT) with the context usable."""
    from paper_2202_04140_gb300 import ace as L
    monkeypatch.setenv("ACE_KERNEL", "lon")
    monkeypatch.setenv("ACE_TILE_E", "2")
    monkeypatch.setenv("ACE_STAGE", "1")
    w, o, d, A, c = setup("fwd_grad_k392", n_env=37)
    A32, c32 = to_f32(A), to_f32(c)
    At, ct = t(A32, torch.float32, dev), t(c32, torch.float32, dev)
    monkeypatch.setenv("ACE_TEST_STAGE_TIMEOUT", "1")
    phi, dA = d.evaluate_grad(At, ct)
    assert L.ace_stream_status(d.handle, torch.cuda.current_stream().cuda_stream) == L.ACE_ERR_TIMEOUT
    assert normalized_error(phi.cpu().numpy(), phi_naive(A32, o, c32), error_scale(A32, o, c32)) < TOL32
    assert normalized_error(dA.cpu().numpy(), grad_naive(A32, o, c32), grad_error_scale(A32, o, c32)) < TOL32
    monkeypatch.delenv("ACE_TEST_STAGE_TIMEOUT")
    phi2, _ = d.evaluate_grad(At, ct)             # the context is usable and the status clean again
    assert d.status() == 0
    assert torch.equal(phi2, phi)
