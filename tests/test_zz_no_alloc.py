"""The allocation-free entry point, through the C ABI: same results as the allocating one and the oracle.

ace_eval_plain_f64_static serves callers that must not call cudaMalloc (the
device heap belongs to another allocator, or an allocation call is not
acceptable on their path): it runs the plain FP64 graph walk in the library's
fixed 32 MiB device scratch.  Two calls in a row, on different graphs and
inputs (so that a graph left in the scratch by the first call cannot serve the
second), must each match ace_eval_plain_f64 (which takes a caller-provided
workspace) and the FP64 oracle within the FP64 gate of the other parity tests;
a request larger than the scratch must fail with ACE_ERR_INVALID_ARG.  This
file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads as W
from oracle.basis import workload_index_set
from oracle.evaluate import error_scale, grad_error_scale, grad_naive, phi_naive
from tests.metrics import normalized_error

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def test_static_scratch_matches_allocating_entry_point_and_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_04140_gb300 import ace as L
    from paper_2202_04140_gb300.torch_api import Dag, Spec
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream().cuda_stream
    # two different graphs: the K = 392 graph by Algorithm 1, then the K = 64 graph by Algorithm 2
    cases = [("fwd_grad_k392", 1, 96, 2, 21), ("plain_fp64_k64", 2, 40, 3, 22)]
    dags = []
    for call, (name, algo, n_env, n_out, seed) in enumerate(cases):
        w = W.WORKLOADS[name]
        o = workload_index_set(w)
        dag = Dag(Spec.from_workload(w), algo=algo)
        dags.append(dag)
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
        phi_h, dA_h = phi.cpu().numpy(), dA.cpu().numpy()
        s_phi, s_dA = error_scale(A, o, c), grad_error_scale(A, o, c, pb)
        assert normalized_error(phi_h, ref_phi.cpu().numpy(), s_phi) < TOL64, call
        assert normalized_error(dA_h, ref_dA.cpu().numpy(), s_dA) < TOL64, call
        assert normalized_error(phi_h, phi_naive(A, o, c), s_phi) < TOL64, call
        assert normalized_error(dA_h, grad_naive(A, o, c, pb), s_dA) < TOL64, call
    # a request beyond the fixed scratch is refused with a clear error, nothing is computed:
    # 4096 environments of the K = 392 graph need 3,729 nodes x 4096 x 16 bytes > 32 MiB
    dag = dags[0]
    big = torch.zeros((4096, dag.K), dtype=torch.float64, device=dev)
    out = torch.zeros((4096, 1), dtype=torch.float64, device=dev)
    c1 = torch.zeros((dag.n_basis, 1), dtype=torch.float64, device=dev)
    with pytest.raises(L.AceError) as err:
        L.ace_eval_plain_f64_static(dag.handle, big.data_ptr(), c1.data_ptr(), 0, 4096, 1,
                                    out.data_ptr(), big.data_ptr(), stream)
    assert err.value.status == -1 and "static scratch" in str(err.value)
