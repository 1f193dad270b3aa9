"""PyTorch-facing API over libace: tensors in, tensors out, every step in libace.

PyTorch supplies device memory, streams and autograd only.  ``Spec`` and ``Dag``
own the library handles; ``Dag.energy`` is differentiable (its backward is the
fused adjoint kernel); ``pool_A`` / ``forces`` wrap the neighbour pooling.
"""
from __future__ import annotations

import numpy as np
import torch

from . import ace as L

_DTYPE = {torch.float32: L.ACE_F32, torch.float64: L.ACE_F64}
_READOUT = {"plain": L.ACE_READOUT_PLAIN, "compensated": L.ACE_READOUT_COMPENSATED,
            "fp64": L.ACE_READOUT_FP64_FINAL}
_RULE = {"balanced": L.ACE_SPLIT_BALANCED, "peel": L.ACE_SPLIT_PEEL}
_GROUP = {"O3": L.ACE_GROUP_O3, "SO2": L.ACE_GROUP_SO2, "T": L.ACE_GROUP_TORUS}


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _dev(t: torch.Tensor, name: str, dtype=None) -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}")
    return t.contiguous()


class Spec:
    """The index set K (sections 2.2-2.5, Eq. 3), built by libace."""

    def __init__(self, group="O3", nmin=1, nmax=1, lmax=0, nu_max=1, deg_max=0, wn=1, wl=1, p_norm=1,
                 require_l_even=True, kmax=0, wk=1):
        self.group = group
        self.nu_max = nu_max
        self.handle = L.ace_build_spec(_GROUP[group], nmin, nmax, lmax, nu_max, deg_max, wn, wl, p_norm,
                                       int(require_l_even), kmax, wk)
        self.n_basis, self.K, self.counts_per_nu = L.ace_spec_info(self.handle, nu_max)
        self._tuples = None

    @classmethod
    def _from_handle(cls, handle: int, params: dict) -> "Spec":
        """Wrap an index-set handle the library built (params: its ace_spec_params)."""
        self = cls.__new__(cls)
        self.group = {v: k for k, v in _GROUP.items()}[params["group"]]
        self.nu_max = params["nu_max"]
        self.handle = handle
        self.n_basis, self.K, self.counts_per_nu = L.ace_spec_info(handle, self.nu_max)
        self._tuples = None
        return self

    @classmethod
    def from_workload(cls, w) -> "Spec":
        return cls("O3", w.nmin, w.nmax, w.lmax, w.nu_max, w.deg_max, w.wn, w.wl, 1, True, w.kmax, w.wk)

    def tuples(self):
        if self._tuples is None:
            self._tuples = L.ace_spec_tuples(self.handle, self.n_basis, self.nu_max)
        return self._tuples

    @property
    def deg(self) -> np.ndarray:
        return self.tuples()[1]

    def __del__(self, _free=L.ace_spec_free):
        h = getattr(self, "handle", None)
        if h:
            _free(h)
            self.handle = None


class Dag:
    """The computational graph G (section 2.6, Algorithm 1 or 2) and its device plan."""

    def __init__(self, spec: Spec, algo: int = 1, rule: str = "balanced", n_split: int = 2):
        self._attach(spec, L.ace_build_dag(spec.handle, algo, _RULE[rule], n_split))

    def save(self, path: str):
        """Write the graph and its index set's parameters to a file (ace_dag_save)."""
        L.ace_dag_save(self.spec.handle, self.handle, path)

    @classmethod
    def load(cls, path: str) -> "Dag":
        """A graph read from a file written by save (ace_dag_load); .spec is its index set."""
        params, sh, dh = L.ace_dag_load(path)
        self = cls.__new__(cls)
        self._attach(Spec._from_handle(sh, params), dh)
        return self

    def _attach(self, spec: Spec, handle: int):
        self.spec = spec
        self.handle = handle
        self.n_nodes, self.n_aux, self.n_operands, self.n_levels = L.ace_dag_info(self.handle)
        self.n_slots, self.n_sinks, self.n_entries, self.smem_bytes_f32 = L.ace_dag_plan_info(self.handle)
        self.K = spec.K
        self.n_basis = spec.n_basis
        self._bound = {}

    def export(self) -> dict:
        left, right, level, aux, bnode = L.ace_dag_export(self.handle, self.n_nodes, self.n_basis)
        return {"left": left, "right": right, "level": level, "is_aux": aux, "basis_node": bnode}

    def upload(self):
        L.ace_dag_upload(self.handle, _stream())

    def autotune(self, n_env: int, n_out: int = 1, dtype=torch.float32, grad: bool = True,
                 readout: str = "plain") -> dict:
        """Time every kernel configuration for this request and keep the fastest (see ace_dag_autotune)."""
        kind, E, ms = L.ace_dag_autotune(self.handle, n_env, n_out, _DTYPE[dtype], grad, _READOUT[readout],
                                         _stream())
        self._bound.clear()          # the tuner leaves no coefficients bound
        names = {1: "tile_per_lane", 2: "env_per_lane", 3: "env_per_lane_global", 4: "env_per_lane_multi",
                 5: "env_pair_per_lane_global"}
        return {"kernel": names[kind], "E": E, "ms": ms}

    def _c_arg(self, mode: str, c: torch.Tensor, c2: torch.Tensor, n_out: int) -> int:
        """Device pointer of c, or 0 when this very tensor, unmodified, is already bound for this mode.

        The bound tensor is kept referenced, so its memory cannot be handed to a
        different tensor while the library still holds coefficients gathered from it.
        """
        prev = self._bound.get(mode)
        if prev is not None and prev[0] is c and prev[1] == c._version and prev[2] == n_out:
            return 0
        self._bound[mode] = (c, c._version, n_out)
        return c2.data_ptr()

    def evaluate(self, A: torch.Tensor, c: torch.Tensor, readout: str = "plain") -> torch.Tensor:
        """phi[e][ch] = sum_k c[k][ch] prod_t A[e][k_t] (Eq. 2) through G (Eq. 4)."""
        A = _dev(A, "A")
        c = _dev(c, "c", A.dtype)
        n_env = A.shape[0]
        c2 = c.reshape(self.n_basis, -1)
        n_out = c2.shape[1]
        phi = torch.empty((n_env, n_out), dtype=A.dtype, device=A.device)
        L.ace_eval(self.handle, A.data_ptr(), self._c_arg("one", c, c2, n_out), n_env, n_out, _DTYPE[A.dtype],
                   _READOUT[readout], phi.data_ptr(), _stream())
        return phi

    def evaluate_grad(self, A: torch.Tensor, c: torch.Tensor, phi_bar: torch.Tensor | None = None,
                      readout: str = "plain", want_phi: bool = True):
        """(phi, dA) with dA[e][k] = sum_ch phi_bar[e][ch] dphi[e][ch]/dA[e][k] (phi_bar = 1 if None)."""
        A = _dev(A, "A")
        c = _dev(c, "c", A.dtype)
        n_env = A.shape[0]
        c2 = c.reshape(self.n_basis, -1)
        n_out = c2.shape[1]
        pb = 0
        if phi_bar is not None:
            phi_bar = _dev(phi_bar, "phi_bar", A.dtype).reshape(n_env, n_out)
            pb = phi_bar.data_ptr()
        phi = torch.empty((n_env, n_out), dtype=A.dtype, device=A.device) if want_phi else None
        dA = torch.empty_like(A)
        L.ace_eval_grad(self.handle, A.data_ptr(), self._c_arg("sym", c, c2, n_out), pb, n_env, n_out,
                        _DTYPE[A.dtype], _READOUT[readout], phi.data_ptr() if want_phi else 0, dA.data_ptr(),
                        _stream())
        return phi, dA

    def evaluate_host(self, A: torch.Tensor, c: torch.Tensor, readout: str = "plain", phi: torch.Tensor | None = None,
                      chunk_env: int = 0, sync: bool = True) -> torch.Tensor:
        """phi for host (CPU) A: copies in, evaluation and copies out overlapped in chunks
        (ace_eval_host).  Pin A (and phi) for the overlap.  With sync=False the result is complete
        once the current CUDA stream has been synchronised (the call can be captured in a graph)."""
        return self._host_call(False, A, c, None, readout, phi, None, chunk_env, sync)[0]

    def evaluate_grad_host(self, A: torch.Tensor, c: torch.Tensor, phi_bar: torch.Tensor | None = None,
                           readout: str = "plain", phi: torch.Tensor | None = None, dA: torch.Tensor | None = None,
                           chunk_env: int = 0, sync: bool = True):
        """(phi, dA) for host (CPU) A, as evaluate_grad, through ace_eval_grad_host."""
        return self._host_call(True, A, c, phi_bar, readout, phi, dA, chunk_env, sync)

    def _host_call(self, grad, A, c, phi_bar, readout, phi, dA, chunk_env, sync):
        if A.device.type != "cpu" or not A.is_contiguous():
            raise ValueError("A must be a contiguous CPU tensor")
        c = _dev(c, "c", A.dtype)
        n_env = A.shape[0]
        c2 = c.reshape(self.n_basis, -1)
        n_out = c2.shape[1]
        pin = A.is_pinned()

        def host_out(t, shape, name):
            if t is None:
                return torch.empty(shape, dtype=A.dtype, pin_memory=pin)
            if t.device.type != "cpu" or not t.is_contiguous() or t.dtype != A.dtype or tuple(t.shape) != shape:
                raise ValueError(f"{name} must be a contiguous CPU tensor of shape {shape} and A's dtype")
            return t

        phi = host_out(phi, (n_env, n_out), "phi")
        if grad:
            dA = host_out(dA, tuple(A.shape), "dA")
            pb = 0
            if phi_bar is not None:
                phi_bar = phi_bar.reshape(n_env, n_out)
                if phi_bar.device.type != "cpu" or not phi_bar.is_contiguous() or phi_bar.dtype != A.dtype:
                    raise ValueError("phi_bar must be a contiguous CPU tensor of A's dtype")
                pb = phi_bar.data_ptr()
            L.ace_eval_grad_host(self.handle, A.data_ptr(), self._c_arg("sym", c, c2, n_out), pb, n_env, n_out,
                                 _DTYPE[A.dtype], _READOUT[readout], phi.data_ptr(), dA.data_ptr(), chunk_env,
                                 _stream())
        else:
            L.ace_eval_host(self.handle, A.data_ptr(), self._c_arg("one", c, c2, n_out), n_env, n_out,
                            _DTYPE[A.dtype], _READOUT[readout], phi.data_ptr(), chunk_env, _stream())
        if sync:
            torch.cuda.current_stream().synchronize()
        return phi, dA

    def evaluate_plain_f64(self, A: torch.Tensor, c: torch.Tensor, phi_bar: torch.Tensor | None = None,
                           grad: bool = False, workspace: torch.Tensor | None = None):
        """The plain FP64 graph walk (one thread per environment, node values in global memory)."""
        A = _dev(A, "A", torch.float64)
        c = _dev(c, "c", torch.float64)
        n_env = A.shape[0]
        c2 = c.reshape(self.n_basis, -1)
        n_out = c2.shape[1]
        need = L.ace_eval_plain_workspace_bytes(self.handle, n_env, grad)
        if workspace is None or workspace.numel() * workspace.element_size() < need:
            workspace = torch.empty(max(need, 16), dtype=torch.uint8, device=A.device)
        phi = torch.empty((n_env, n_out), dtype=torch.float64, device=A.device)
        dA = torch.empty_like(A) if grad else None
        pb = _dev(phi_bar, "phi_bar", torch.float64).data_ptr() if phi_bar is not None else 0
        L.ace_eval_plain_f64(self.handle, A.data_ptr(), c2.data_ptr(), pb, n_env, n_out, phi.data_ptr(),
                             dA.data_ptr() if grad else 0, workspace.data_ptr(),
                             workspace.numel() * workspace.element_size(), _stream())
        return phi, dA

    def status(self) -> int:
        """Synchronise and read the device status word (0, or -5 bounds / -4 timeout)."""
        return L.ace_stream_status(self.handle, _stream())

    def energy(self, A: torch.Tensor, c: torch.Tensor, readout: str = "plain") -> torch.Tensor:
        """Differentiable phi (w.r.t. A): backward runs the fused forward+adjoint kernel."""
        return _AceEnergy.apply(A, c, self, readout)

    def __del__(self, _free=L.ace_dag_free):
        h = getattr(self, "handle", None)
        if h:
            _free(h)
            self.handle = None


class _AceEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, c, dag, readout):
        ctx.save_for_backward(A, c)
        ctx.dag = dag
        ctx.readout = readout
        return dag.evaluate(A, c, readout)

    @staticmethod
    def backward(ctx, gphi):
        A, c = ctx.saved_tensors
        _, dA = ctx.dag.evaluate_grad(A, c, gphi.contiguous(), ctx.readout, want_phi=False)
        return dA, None, None, None


def pool_A(pos: torch.Tensor, offsets: torch.Tensor, nmin: int, nmax: int, lmax: int, rc: float,
           mu: torch.Tensor | None = None, kmax: int = 0) -> torch.Tensor:
    """A[e][id(n,[k,]l,m)] = sum_{j in e} R_n(|r_j|) [T_k(mu_j)] Y_lm(r_j/|r_j|) on the GPU."""
    pos = _dev(pos, "pos", torch.float32)
    offsets = _dev(offsets, "offsets", torch.int64)
    mu_p = _dev(mu, "mu", torch.float32).data_ptr() if mu is not None else 0
    n_env = offsets.numel() - 1
    K = (nmax - nmin + 1) * (kmax + 1) * (lmax + 1) ** 2
    A = torch.empty((n_env, K), dtype=torch.float32, device=pos.device)
    L.ace_pool_A_feat(pos.data_ptr(), mu_p, offsets.data_ptr(), n_env, pos.shape[0], rc, nmin, nmax, lmax, kmax,
                      A.data_ptr(), _stream())
    return A


def pool_A_grad(pos: torch.Tensor, offsets: torch.Tensor, dA: torch.Tensor, nmin: int, nmax: int, lmax: int,
                rc: float, alpha: float = 1.0, mu: torch.Tensor | None = None, kmax: int = 0) -> torch.Tensor:
    """dpos[j] = alpha sum_k dA[e(j)][k] grad phi_k(r_j); alpha = -1 with dA = dphi/dA gives the forces."""
    pos = _dev(pos, "pos", torch.float32)
    offsets = _dev(offsets, "offsets", torch.int64)
    dA = _dev(dA, "dA", torch.float32)
    mu_p = _dev(mu, "mu", torch.float32).data_ptr() if mu is not None else 0
    n_env = offsets.numel() - 1
    dpos = torch.empty_like(pos)
    L.ace_pool_A_feat_grad(pos.data_ptr(), mu_p, offsets.data_ptr(), n_env, pos.shape[0], rc, nmin, nmax, lmax, kmax,
                           dA.data_ptr(), alpha, dpos.data_ptr(), _stream())
    return dpos


def energy_and_forces(dag: Dag, pos: torch.Tensor, offsets: torch.Tensor, c: torch.Tensor, nmin: int, nmax: int,
                      lmax: int, rc: float, readout: str = "plain", mu: torch.Tensor | None = None, kmax: int = 0):
    """Full pipeline through ace_energy_forces: pooling -> forward + adjoint -> pooling adjoint (one fused
    kernel per tile of 32 environments when it applies).  Returns (phi [n_env, 1], F = -dphi/dr [n_pairs, 3]).
    With mu (one invariant feature value per neighbour) the one-particle basis is R_n Y_lm T_k(mu)."""
    pos = _dev(pos, "pos", torch.float32)
    offsets = _dev(offsets, "offsets", torch.int64)
    mu_p = _dev(mu, "mu", torch.float32).data_ptr() if mu is not None else 0
    n_env = offsets.numel() - 1
    c = _dev(c, "c", torch.float32)
    c2 = c.reshape(dag.n_basis, -1)
    if c2.shape[1] != 1:
        raise ValueError("one output channel")
    phi = torch.empty((n_env, 1), dtype=torch.float32, device=pos.device)
    F = torch.empty((pos.shape[0], 3), dtype=torch.float32, device=pos.device)
    L.ace_energy_forces(dag.handle, pos.data_ptr(), mu_p, offsets.data_ptr(), n_env, pos.shape[0],
                        dag._c_arg("sym", c, c2, 1), _READOUT[readout], float(rc), nmin, nmax, lmax, kmax,
                        phi.data_ptr(), F.data_ptr(), _stream())
    return phi, F


def energy_and_forces_host(dag: Dag, pos: torch.Tensor, offsets: torch.Tensor, c: torch.Tensor, nmin: int, nmax: int,
                           lmax: int, rc: float, readout: str = "plain", mu: torch.Tensor | None = None,
                           kmax: int = 0, phi: torch.Tensor | None = None, forces: torch.Tensor | None = None,
                           chunk_env: int = 0, sync: bool = True):
    """energy_and_forces for host (CPU) positions, offsets (and mu) through ace_energy_forces_host:
    the batch in chunks, copies overlapped with the kernels.  Returns CPU (phi [n_env], F [n_pairs, 3]);
    pin pos and the outputs for the overlap.  With sync=False the results are complete once the
    current CUDA stream has been synchronised."""
    for t, name in ((pos, "pos"), (offsets, "offsets")):
        if t.device.type != "cpu" or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous CPU tensor")
    if pos.dtype != torch.float32 or offsets.dtype != torch.int64:
        raise ValueError("pos must be float32 and offsets int64")
    n_env = offsets.numel() - 1
    n_pairs = pos.shape[0]
    pin = pos.is_pinned()
    def host_out(t, shape, name):
        if t is None:
            return torch.empty(shape, dtype=torch.float32, pin_memory=pin)
        if t.device.type != "cpu" or not t.is_contiguous() or t.dtype != torch.float32 or tuple(t.shape) != shape:
            raise ValueError(f"{name} must be a contiguous float32 CPU tensor of shape {shape}")
        return t

    phi = host_out(phi, (n_env,), "phi")
    forces = host_out(forces, (n_pairs, 3), "forces")
    if mu is not None and (mu.device.type != "cpu" or not mu.is_contiguous() or mu.dtype != torch.float32
                           or mu.numel() != n_pairs):
        raise ValueError("mu must be a contiguous float32 CPU tensor with one value per neighbour")
    c = _dev(c, "c", torch.float32)
    c2 = c.reshape(dag.n_basis, -1)
    if c2.shape[1] != 1:
        raise ValueError("one output channel")
    L.ace_energy_forces_host(dag.handle, pos.data_ptr(), mu.data_ptr() if mu is not None else 0, offsets.data_ptr(),
                             n_env, n_pairs, dag._c_arg("sym", c, c2, 1), _READOUT[readout], float(rc), nmin, nmax,
                             lmax, kmax, phi.data_ptr(), forces.data_ptr(), chunk_env, _stream())
    if sync:
        torch.cuda.current_stream().synchronize()
    return phi, forces
