"""ctypes binding of libace (include/ace.h): the same entry points, argument marshalling only.

Every compute step runs inside libace (host C++ for the index set, the graph
and the plan; sm_103a kernels for evaluation).  Functions raise AceError on a
non-zero status.  Device buffers are passed as integer device pointers (for
example ``tensor.data_ptr()``) and streams as integer ``cudaStream_t`` handles.

Importing this module loads ``libace.so`` from this package directory and
fails loudly (ImportError) when it has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libace.so")

ACE_OK = 0
ACE_ERR_INVALID_ARG, ACE_ERR_OOM, ACE_ERR_CUDA = -1, -2, -3
ACE_ERR_TIMEOUT, ACE_ERR_BOUNDS, ACE_ERR_UNSUPPORTED, ACE_ERR_NO_DEVICE = -4, -5, -6, -7
STATUS_NAMES = {0: "ACE_OK", -1: "ACE_ERR_INVALID_ARG", -2: "ACE_ERR_OOM", -3: "ACE_ERR_CUDA",
                -4: "ACE_ERR_TIMEOUT", -5: "ACE_ERR_BOUNDS", -6: "ACE_ERR_UNSUPPORTED",
                -7: "ACE_ERR_NO_DEVICE"}
ACE_GROUP_O3, ACE_GROUP_SO2, ACE_GROUP_TORUS = 0, 1, 2
ACE_ALGO_1, ACE_ALGO_2 = 1, 2
ACE_SPLIT_BALANCED, ACE_SPLIT_PEEL = 0, 1
ACE_F32, ACE_F64 = 0, 1
ACE_READOUT_PLAIN, ACE_READOUT_COMPENSATED, ACE_READOUT_FP64_FINAL = 0, 1, 2

# every symbol declared in include/ace.h
EXPORTED = [
    "ace_last_error", "ace_abi_version", "ace_build_spec", "ace_spec_info", "ace_spec_tuples",
    "ace_spec_free", "ace_build_dag", "ace_dag_info", "ace_dag_export", "ace_dag_plan_info",
    "ace_dag_plan_array", "ace_dag_validate", "ace_dag_save", "ace_dag_load", "ace_dag_free", "ace_dag_upload", "ace_dag_autotune", "ace_eval", "ace_eval_grad",
    "ace_eval_host", "ace_eval_grad_host", "ace_eval_plain_workspace_bytes",
    "ace_eval_plain_f64", "ace_eval_plain_f64_static", "ace_pool_A", "ace_pool_A_grad", "ace_pool_A_feat", "ace_pool_A_feat_grad", "ace_energy_forces", "ace_energy_forces_plan", "ace_energy_forces_host", "ace_stream_status", "ace_device_info",
    "ace_fma_peak",
]


class AceError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        self.status = status
        super().__init__(f"{fn}: {STATUS_NAMES.get(status, status)}: {msg}")


class ace_spec_params(C.Structure):
    _fields_ = [("group", C.c_int32), ("nmin", C.c_int32), ("nmax", C.c_int32), ("lmax", C.c_int32),
                ("nu_max", C.c_int32), ("deg_max", C.c_int32), ("wn", C.c_int32), ("wl", C.c_int32),
                ("p_norm", C.c_int32), ("require_l_even", C.c_int32), ("kmax", C.c_int32), ("wk", C.c_int32)]


if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is not built; run `python -m paper_2202_04140_gb300.build`")
_lib = C.CDLL(_LIB_PATH)

_p, _i32, _i64, _sz, _f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t, C.c_float
_P = C.POINTER
_SIG = {
    "ace_last_error": (C.c_char_p, []),
    "ace_abi_version": (_i32, []),
    "ace_build_spec": (C.c_int, [_P(ace_spec_params), _P(_p)]),
    "ace_spec_info": (C.c_int, [_p, _P(_i64), _P(_i32), _p]),
    "ace_spec_tuples": (C.c_int, [_p, _p, _p]),
    "ace_spec_free": (None, [_p]),
    "ace_build_dag": (C.c_int, [_p, _i32, _i32, _i32, _P(_p)]),
    "ace_dag_info": (C.c_int, [_p, _P(_i64), _P(_i64), _P(_i64), _P(_i32)]),
    "ace_dag_export": (C.c_int, [_p, _p, _p, _p, _p, _p]),
    "ace_dag_plan_info": (C.c_int, [_p, _P(_i64), _P(_i64), _P(_i64), _P(_i64)]),
    "ace_dag_plan_array": (C.c_int, [_p, C.c_char_p, _p, _P(_i64)]),
    "ace_dag_validate": (C.c_int, [_p]),
    "ace_dag_save": (C.c_int, [_p, _p, C.c_char_p]),
    "ace_dag_load": (C.c_int, [C.c_char_p, _P(ace_spec_params), _P(_p), _P(_p)]),
    "ace_dag_free": (None, [_p]),
    "ace_dag_upload": (C.c_int, [_p, _p]),
    "ace_dag_autotune": (C.c_int, [_p, _i64, _i32, _i32, _i32, _i32, _p, _P(_i32), _P(_i32), _P(C.c_float)]),
    "ace_eval": (C.c_int, [_p, _p, _p, _i64, _i32, _i32, _i32, _p, _p]),
    "ace_eval_grad": (C.c_int, [_p, _p, _p, _p, _i64, _i32, _i32, _i32, _p, _p, _p]),
    "ace_eval_host": (C.c_int, [_p, _p, _p, _i64, _i32, _i32, _i32, _p, _i64, _p]),
    "ace_eval_grad_host": (C.c_int, [_p, _p, _p, _p, _i64, _i32, _i32, _i32, _p, _p, _i64, _p]),
    "ace_eval_plain_workspace_bytes": (C.c_int, [_p, _i64, _i32, _P(_sz)]),
    "ace_eval_plain_f64": (C.c_int, [_p, _p, _p, _p, _i64, _i32, _p, _p, _p, _sz, _p]),
    "ace_eval_plain_f64_static": (C.c_int, [_p, _p, _p, _p, _i64, _i32, _p, _p, _p]),
    "ace_pool_A": (C.c_int, [_p, _p, _i64, _i64, _f32, _i32, _i32, _i32, _p, _p]),
    "ace_pool_A_grad": (C.c_int, [_p, _p, _i64, _i64, _f32, _i32, _i32, _i32, _p, _f32, _p, _p]),
    "ace_pool_A_feat": (C.c_int, [_p, _p, _p, _i64, _i64, _f32, _i32, _i32, _i32, _i32, _p, _p]),
    "ace_pool_A_feat_grad": (C.c_int, [_p, _p, _p, _i64, _i64, _f32, _i32, _i32, _i32, _i32, _p, _f32, _p, _p]),
    "ace_energy_forces": (C.c_int, [_p, _p, _p, _p, _i64, _i64, _p, _i32, _f32, _i32, _i32, _i32, _i32, _p, _p, _p]),
    "ace_energy_forces_plan": (C.c_int, [_p, _i32, _i32, _i32, _i32, _p, _p]),
    "ace_energy_forces_host": (C.c_int, [_p, _p, _p, _p, _i64, _i64, _p, _i32, _f32, _i32, _i32, _i32, _i32, _p, _p,
                                         _i64, _p]),
    "ace_stream_status": (C.c_int, [_p, _p]),
    "ace_device_info": (C.c_int, [_P(_i32), _P(_i32), _P(_i32), _P(_i32)]),
    "ace_fma_peak": (C.c_int, [_i64, _P(C.c_double), _P(C.c_double), _p]),
}
for _name, (_res, _args) in _SIG.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def library_path() -> str:
    return _LIB_PATH


def _check(st: int, fn: str):
    if st != ACE_OK:
        raise AceError(st, fn, (_lib.ace_last_error() or b"").decode())


def ace_last_error() -> str:
    return (_lib.ace_last_error() or b"").decode()


def ace_abi_version() -> int:
    return _lib.ace_abi_version()


# ---- index set ---------------------------------------------------------------------------

def ace_build_spec(group=ACE_GROUP_O3, nmin=1, nmax=1, lmax=0, nu_max=1, deg_max=0, wn=1, wl=1, p_norm=1,
                   require_l_even=1, kmax=0, wk=1) -> int:
    prm = ace_spec_params(group, nmin, nmax, lmax, nu_max, deg_max, wn, wl, p_norm, require_l_even, kmax, wk)
    h = C.c_void_p()
    _check(_lib.ace_build_spec(C.byref(prm), C.byref(h)), "ace_build_spec")
    return h.value


def ace_spec_info(spec: int, nu_max: int):
    nb, K = C.c_int64(), C.c_int32()
    counts = np.zeros(nu_max, dtype=np.int64)
    _check(_lib.ace_spec_info(spec, C.byref(nb), C.byref(K), counts.ctypes.data), "ace_spec_info")
    return nb.value, K.value, counts


def ace_spec_tuples(spec: int, n_basis: int, nu_max: int):
    t = np.zeros((n_basis, nu_max), dtype=np.int32)
    d = np.zeros(n_basis, dtype=np.int32)
    _check(_lib.ace_spec_tuples(spec, t.ctypes.data, d.ctypes.data), "ace_spec_tuples")
    return t, d


def ace_spec_free(spec: int, _free=_lib.ace_spec_free):
    # the C function is bound at import: handles can be freed while the interpreter shuts down
    _free(spec)


# ---- graph ----------------------------------------------------------------------------------

def ace_build_dag(spec: int, algo=ACE_ALGO_1, split_rule=ACE_SPLIT_BALANCED, n_split=2) -> int:
    h = C.c_void_p()
    _check(_lib.ace_build_dag(spec, algo, split_rule, n_split, C.byref(h)), "ace_build_dag")
    return h.value


def ace_dag_info(dag: int):
    n, a, o, lv = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int32()
    _check(_lib.ace_dag_info(dag, C.byref(n), C.byref(a), C.byref(o), C.byref(lv)), "ace_dag_info")
    return n.value, a.value, o.value, lv.value


def ace_dag_export(dag: int, n_nodes: int, n_basis: int):
    left = np.zeros(n_nodes, np.int32)
    right = np.zeros(n_nodes, np.int32)
    level = np.zeros(n_nodes, np.int32)
    aux = np.zeros(n_nodes, np.uint8)
    bnode = np.zeros(n_basis, np.int32)
    _check(_lib.ace_dag_export(dag, left.ctypes.data, right.ctypes.data, level.ctypes.data, aux.ctypes.data,
                               bnode.ctypes.data), "ace_dag_export")
    return left, right, level, aux, bnode


def ace_dag_plan_info(dag: int):
    a, b, c, d = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
    _check(_lib.ace_dag_plan_info(dag, C.byref(a), C.byref(b), C.byref(c), C.byref(d)), "ace_dag_plan_info")
    return a.value, b.value, c.value, d.value


def ace_dag_plan_array(dag: int, name: str) -> np.ndarray:
    n = C.c_int64()
    _check(_lib.ace_dag_plan_array(dag, name.encode(), None, C.byref(n)), "ace_dag_plan_array")
    out = np.zeros(max(n.value, 1), dtype=np.int32)
    _check(_lib.ace_dag_plan_array(dag, name.encode(), out.ctypes.data, C.byref(n)), "ace_dag_plan_array")
    return out[:n.value]


def ace_dag_validate(dag: int):
    _check(_lib.ace_dag_validate(dag), "ace_dag_validate")


def ace_dag_save(spec: int, dag: int, path: str):
    _check(_lib.ace_dag_save(spec, dag, os.fsencode(path)), "ace_dag_save")


def ace_dag_load(path: str):
    """Returns (params as a dict, spec handle, dag handle) of a file written by ace_dag_save."""
    prm = ace_spec_params()
    s, d = C.c_void_p(), C.c_void_p()
    _check(_lib.ace_dag_load(os.fsencode(path), C.byref(prm), C.byref(s), C.byref(d)), "ace_dag_load")
    return {name: getattr(prm, name) for name, _ in ace_spec_params._fields_}, s.value, d.value


def ace_dag_free(dag: int, _free=_lib.ace_dag_free):
    # the C function is bound at import: handles can be freed while the interpreter shuts down
    _free(dag)


def ace_dag_upload(dag: int, stream: int = 0):
    _check(_lib.ace_dag_upload(dag, stream), "ace_dag_upload")


# ---- evaluation -----------------------------------------------------------------------------

def ace_dag_autotune(dag, n_env, n_out, dtype, grad, readout, stream=0):
    """Returns (kind, E, ms) of the fastest configuration, now used by later evaluations."""
    k, E, ms = C.c_int32(), C.c_int32(), C.c_float()
    _check(_lib.ace_dag_autotune(dag, n_env, n_out, dtype, int(grad), readout, stream, C.byref(k), C.byref(E),
                                 C.byref(ms)), "ace_dag_autotune")
    return k.value, E.value, ms.value


def ace_eval(dag, A, c, n_env, n_out, dtype, readout, phi, stream=0):
    _check(_lib.ace_eval(dag, A, c, n_env, n_out, dtype, readout, phi, stream), "ace_eval")


def ace_eval_grad(dag, A, c, phi_bar, n_env, n_out, dtype, readout, phi, dA, stream=0):
    _check(_lib.ace_eval_grad(dag, A, c, phi_bar, n_env, n_out, dtype, readout, phi, dA, stream),
           "ace_eval_grad")


def ace_eval_host(dag, A, c, n_env, n_out, dtype, readout, phi, chunk_env=0, stream=0):
    """A and phi are host pointers (page-locked memory lets the copies overlap the evaluation)."""
    _check(_lib.ace_eval_host(dag, A, c, n_env, n_out, dtype, readout, phi, chunk_env, stream), "ace_eval_host")


def ace_eval_grad_host(dag, A, c, phi_bar, n_env, n_out, dtype, readout, phi, dA, chunk_env=0, stream=0):
    """A, phi_bar, phi and dA are host pointers (page-locked memory lets the copies overlap the evaluation)."""
    _check(_lib.ace_eval_grad_host(dag, A, c, phi_bar, n_env, n_out, dtype, readout, phi, dA, chunk_env, stream),
           "ace_eval_grad_host")


def ace_eval_plain_workspace_bytes(dag, n_env, with_grad) -> int:
    b = C.c_size_t()
    _check(_lib.ace_eval_plain_workspace_bytes(dag, n_env, int(with_grad), C.byref(b)),
           "ace_eval_plain_workspace_bytes")
    return b.value


def ace_eval_plain_f64(dag, A, c, phi_bar, n_env, n_out, phi, dA, workspace, workspace_bytes, stream=0):
    _check(_lib.ace_eval_plain_f64(dag, A, c, phi_bar, n_env, n_out, phi, dA, workspace, workspace_bytes, stream),
           "ace_eval_plain_f64")


def ace_eval_plain_f64_static(dag, A, c, phi_bar, n_env, n_out, phi, dA, stream=0):
    """Plain FP64 graph walk with the library's fixed 32 MiB device scratch: allocates nothing."""
    _check(_lib.ace_eval_plain_f64_static(dag, A, c, phi_bar, n_env, n_out, phi, dA, stream),
           "ace_eval_plain_f64_static")


def ace_pool_A(pos, offsets, n_env, n_pairs, rc, nmin, nmax, lmax, A, stream=0):
    _check(_lib.ace_pool_A(pos, offsets, n_env, n_pairs, rc, nmin, nmax, lmax, A, stream), "ace_pool_A")


def ace_pool_A_grad(pos, offsets, n_env, n_pairs, rc, nmin, nmax, lmax, dA, alpha, dpos, stream=0):
    _check(_lib.ace_pool_A_grad(pos, offsets, n_env, n_pairs, rc, nmin, nmax, lmax, dA, alpha, dpos, stream),
           "ace_pool_A_grad")


def ace_pool_A_feat(pos, mu, offsets, n_env, n_pairs, rc, nmin, nmax, lmax, kmax, A, stream=0):
    _check(_lib.ace_pool_A_feat(pos, mu, offsets, n_env, n_pairs, rc, nmin, nmax, lmax, kmax, A, stream),
           "ace_pool_A_feat")


def ace_pool_A_feat_grad(pos, mu, offsets, n_env, n_pairs, rc, nmin, nmax, lmax, kmax, dA, alpha, dpos, stream=0):
    _check(_lib.ace_pool_A_feat_grad(pos, mu, offsets, n_env, n_pairs, rc, nmin, nmax, lmax, kmax, dA, alpha, dpos,
                                     stream), "ace_pool_A_feat_grad")


def ace_energy_forces(dag, pos, mu, offsets, n_env, n_pairs, c, readout, rc, nmin, nmax, lmax, kmax, phi, forces,
                      stream=0):
    _check(_lib.ace_energy_forces(dag, pos, mu, offsets, n_env, n_pairs, c, readout, rc, nmin, nmax, lmax, kmax, phi,
                                  forces, stream), "ace_energy_forces")


def ace_energy_forces_plan(dag, nmin, nmax, lmax, kmax):
    """(fused, smem_bytes): whether ace_energy_forces takes the one-kernel form for these parameters."""
    f, b = C.c_int32(0), C.c_int64(0)
    _check(_lib.ace_energy_forces_plan(dag, nmin, nmax, lmax, kmax, C.byref(f), C.byref(b)), "ace_energy_forces_plan")
    return bool(f.value), int(b.value)


def ace_energy_forces_host(dag, pos, mu, offsets, n_env, n_pairs, c, readout, rc, nmin, nmax, lmax, kmax, phi, forces,
                           chunk_env=0, stream=0):
    """pos, mu, offsets, phi and forces are host pointers; c a device pointer or 0."""
    _check(_lib.ace_energy_forces_host(dag, pos, mu, offsets, n_env, n_pairs, c, readout, rc, nmin, nmax, lmax, kmax,
                                       phi, forces, chunk_env, stream), "ace_energy_forces_host")


def ace_stream_status(dag, stream=0) -> int:
    """Returns the status code (0, -4 timeout, -5 bounds) instead of raising for device-side findings."""
    return _lib.ace_stream_status(dag, stream)


def ace_device_info():
    a, b, c, d = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _check(_lib.ace_device_info(C.byref(a), C.byref(b), C.byref(c), C.byref(d)), "ace_device_info")
    return a.value, b.value, c.value, d.value


def ace_fma_peak(iters: int, stream=0):
    ms, cnt = C.c_double(), C.c_double()
    _check(_lib.ace_fma_peak(iters, C.byref(ms), C.byref(cnt), stream), "ace_fma_peak")
    return ms.value, cnt.value
