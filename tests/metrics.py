"""Error measure used by every parity test.

e = |x - ref| / scale, where scale is the oracle evaluated with |A|, |c| (and
|phibar| for gradients): sum_k |c_k| |AA_k| for phi.  Entries whose scale is
exactly zero (an input no basis function touches) must match exactly.
"""
import numpy as np


def normalized_error(x, ref, scale) -> float:
    x, ref, scale = (np.asarray(v, dtype=np.float64) for v in (x, ref, scale))
    d = np.abs(x - ref)
    zero = scale == 0
    if np.any(d[zero] != 0):
        return float("inf")
    return float(np.max(np.where(zero, 0.0, d / np.where(zero, 1.0, scale)), initial=0.0))
