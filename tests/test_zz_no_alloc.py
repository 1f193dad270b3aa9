"""The allocation-free entry point, through the C ABI: same results as the allocating one.

ace_eval_plain_f64_static serves callers that must not call cudaMalloc (the
device heap belongs to another allocator, or an allocation call is not
acceptable on their path): it runs the plain FP64 graph walk in the library's
fixed 32 MiB device scratch.  Two calls in a row, on different inputs, must
each match ace_eval_plain_f64 (which takes a caller-provided workspace) within
the FP64 gate of the other parity tests; a request larger than the scratch
must fail with ACE_ERR_INVALID_ARG.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads as W
from oracle.basis import workload_index_set
from oracle.evaluate import error_scale, grad_error_scale
from tests.metrics import normalized_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def test_static_scratch_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_04140_gb300 import ace as L
    from paper_2202_04140_gb300.torch_api import Dag, Spec
    dev = torch.device("cuda:0")
    w = W.WORKLOADS["fwd_grad_k392"]
    o = workload_index_set(w)
    dag = Dag(Spec.from_workload(w))
    n_env, n_out = 96, 2
    stream = torch.cuda.current_stream().cuda_stream
    for call, seed in enumerate([21, 22]):
        A = W.draw_A(n_env, dag.K, seed=seed)
        c = W.draw_c(o.deg, n_out, seed=seed + 100)
        pb = np.random.default_rng(seed + 200).standard_normal((n_env, n_out))
        At = torch.tensor(A, dtype=torch.float64, device=dev)
        ct = torch.tensor(c, dtype=torch.float64, device=dev)
        pbt = torch.tensor(pb, dtype=torch.float64, device=dev)
        ref_phi, ref_dA = dag.evaluate_plain_f64(At, ct, pbt, grad=True)
        phi = torch.full((n_env, n_out), float("nan"), dtype=torch.float64, device=dev)
        dA = torch.full((n_env, dag.K), float("nan"), dtype=torch.float64, device=dev)
        L.ace_eval_plain_f64_static(dag.handle, At.data_ptr(), ct.data_ptr(), pbt.data_ptr(), n_env, n_out,
                                    phi.data_ptr(), dA.data_ptr(), stream)
        torch.cuda.synchronize()
        assert normalized_error(phi.cpu().numpy(), ref_phi.cpu().numpy(), error_scale(A, o, c)) < TOL64, call
        assert normalized_error(dA.cpu().numpy(), ref_dA.cpu().numpy(), grad_error_scale(A, o, c, pb)) < TOL64, call
    # a request beyond the fixed scratch is refused with a clear error, nothing is computed
    big = torch.zeros((4096, dag.K), dtype=torch.float64, device=dev)
    out = torch.zeros((4096, 1), dtype=torch.float64, device=dev)
    with pytest.raises(L.AceError) as err:
        L.ace_eval_plain_f64_static(dag.handle, big.data_ptr(), ct[:, :1].contiguous().data_ptr(), 0, 4096, 1,
                                    out.data_ptr(), big.data_ptr(), stream)
    assert err.value.status == -1 and "static scratch" in str(err.value)
