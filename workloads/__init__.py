"""Seeded synthetic workloads for the ACE contraction (arXiv 2202.04140).

This module is shared by the oracle, the tests and the benchmark.  It holds the
five workload definitions and the random draws only: it contains none of the
method's arithmetic (no index set, no graph, no product, no basis function).
Anything that depends on the index set (the per-basis degree used to scale the
coefficients) is passed in by the caller, who computes it on its own side.

Recipe (all draws are numpy PCG64 `default_rng(seed)`):
  * A_k       : seed 0, standard normal, shape (n_env, K), drawn in FP64.
                The "uneven batch" workload multiplies row e by s_e ~ U(0.5, 2)
                drawn from seed 2.
  * c_k       : seed 1, standard normal, shape (n_basis, n_out), divided by
                (1 + deg(k))^2 where deg(k) is the total degree of basis tuple k
                (given by the caller, in canonical basis order).
  * neighbours: seed 3.  J_e ~ U{10..60} for every environment, then all unit
                directions (normalised standard normals, 3 per neighbour), then
                all radii r = rc * U^(1/3) (uniform in the ball), in that order.
                A radius below 1e-6 is redrawn (probability ~1e-19 per draw).
  * species   : seed 4.  s_j ~ U{0..S-1} per neighbour; the feature value is
                mu_j = -1 + 2 s_j / (S - 1) (S species spread over [-1, 1]).
FP32 workloads round the FP64 draws to FP32 once; the oracle receives the same
FP32 values promoted to FP64, so input rounding is never counted as error.
"""
from __future__ import annotations

from dataclasses import dataclass, field, asdict
import numpy as np

__all__ = ["Workload", "WORKLOADS", "draw_A", "draw_c", "draw_neighbours", "draw_species",
           "round_to", "workload"]


@dataclass(frozen=True)
class Workload:
    """One synthetic workload: index-set parameters plus batch shape.

    The one-particle basis is (n, l, m) with nmin <= n <= nmax,
    0 <= l <= lmax, -l <= m <= l; the one-particle degree is wn*n + wl*l and a
    tuple is kept when its summed degree is at most deg_max (p = 1 norm).
    """
    name: str
    description: str
    nmin: int
    nmax: int
    lmax: int
    nu_max: int
    deg_max: int
    n_env: int
    n_out: int = 1
    wn: int = 1
    wl: int = 2
    dtype: str = "f32"            # arithmetic type of the GPU path
    grad: bool = False             # forward plus dphi/dA
    env_scale: tuple | None = None  # per-environment scale range for A rows
    pooling: bool = False          # A built from neighbour positions
    rc: float = 5.0
    j_range: tuple = (10, 60)
    kmax: int = 0                  # invariant-feature degree range (0: no feature index)
    wk: int = 1                    # weight of the feature degree in the one-particle degree
    n_species: int = 0             # neighbours carry one of n_species feature values (pooling)

    @property
    def K(self) -> int:
        return (self.nmax - self.nmin + 1) * (self.kmax + 1) * (self.lmax + 1) ** 2

    def as_dict(self) -> dict:
        return asdict(self)


WORKLOADS = {
    "plain_fp64_k64": Workload(
        "plain_fp64_k64", "plain forward FP64, K=64, nu<=3, D=10, 32 environments",
        nmin=1, nmax=4, lmax=3, nu_max=3, deg_max=10, n_env=32, dtype="f64"),
    "fwd_grad_k392": Workload(
        "fwd_grad_k392", "forward + dphi/dA FP32, K=392, nu<=4, D=16, 4096 environments",
        nmin=1, nmax=8, lmax=6, nu_max=4, deg_max=16, n_env=4096, grad=True),
    "uneven_16ch_k392": Workload(
        "uneven_16ch_k392", "forward FP32, 16 output channels, K=392, nu<=5, D=20, "
        "100k environments with per-environment scale U(0.5,2)",
        nmin=1, nmax=8, lmax=6, nu_max=5, deg_max=20, n_env=100_000, n_out=16,
        env_scale=(0.5, 2.0)),
    "stress_k810": Workload(
        "stress_k810", "forward + dphi/dA FP32, K=810, nu<=6, D=24, 16384 environments",
        nmin=1, nmax=10, lmax=8, nu_max=6, deg_max=24, n_env=16_384, grad=True),
    "forces_k392": Workload(
        "forces_k392", "pooling + forward + forces FP32, K=392, nu<=4, D=16, "
        "50k environments of 10-60 neighbours in a ball of radius 5",
        nmin=1, nmax=8, lmax=6, nu_max=4, deg_max=16, n_env=50_000, grad=True,
        pooling=True),
    "paper_degree_k810": Workload(
        "paper_degree_k810", "forward + dphi/dA FP32, K=810, nu<=6, D=24 with the paper's degree n + l "
        "(17.3 million basis functions), 16384 environments",
        nmin=1, nmax=10, lmax=8, nu_max=6, deg_max=24, n_env=16_384, wl=1, grad=True),
    "paper_degree_d20_k810": Workload(
        "paper_degree_d20_k810", "forward + dphi/dA FP32, K=810, nu<=6, D=20 with the paper's degree n + l "
        "(1.5 million basis functions), 16384 environments",
        nmin=1, nmax=10, lmax=8, nu_max=6, deg_max=20, n_env=16_384, wl=1, grad=True),
    "species_forces_k375": Workload(
        "species_forces_k375", "pooling + forward + forces FP32 with an invariant feature per neighbour "
        "(3 species, phi_nlmk = R_n Y_lm T_k(mu), k <= 2, degree n + l + k), K=375, nu<=4, D=12, "
        "20k environments of 10-60 neighbours in a ball of radius 5",
        nmin=1, nmax=5, lmax=4, nu_max=4, deg_max=12, n_env=20_000, wl=1, grad=True, pooling=True,
        kmax=2, wk=1, n_species=3),
}


def workload(name: str, **overrides) -> Workload:
    """Return a named workload, optionally with fields replaced (e.g. n_env)."""
    w = WORKLOADS[name]
    if overrides:
        d = w.as_dict()
        d.update(overrides)
        w = Workload(**d)
    return w


def round_to(x: np.ndarray, dtype: str) -> np.ndarray:
    """Round FP64 draws to the path's arithmetic type and promote back to FP64."""
    if dtype == "f32":
        return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)
    return np.asarray(x, dtype=np.float64)


def draw_A(n_env: int, K: int, seed: int = 0, env_scale=None,
           scale_seed: int = 2) -> np.ndarray:
    """A ~ N(0,1) of shape (n_env, K) in FP64; optional per-row scale U(lo, hi)."""
    A = np.random.default_rng(seed).standard_normal((n_env, K))
    if env_scale is not None:
        lo, hi = env_scale
        s = np.random.default_rng(scale_seed).uniform(lo, hi, n_env)
        A = A * s[:, None]
    return A


def draw_c(deg: np.ndarray, n_out: int = 1, seed: int = 1) -> np.ndarray:
    """c ~ N(0,1)/(1+deg)^2, shape (n_basis, n_out); deg supplied by the caller."""
    deg = np.asarray(deg, dtype=np.float64)
    z = np.random.default_rng(seed).standard_normal((deg.shape[0], n_out))
    return z / ((1.0 + deg) ** 2)[:, None]


def draw_neighbours(n_env: int, seed: int = 3, rc: float = 5.0,
                    j_range=(10, 60)):
    """Neighbour clouds: CSR offsets (n_env+1,) int64 and positions (sum J, 3) FP64."""
    rng = np.random.default_rng(seed)
    J = rng.integers(j_range[0], j_range[1] + 1, size=n_env)
    offsets = np.zeros(n_env + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(J)
    n = int(offsets[-1])
    d = rng.standard_normal((n, 3))
    norms = np.linalg.norm(d, axis=1)
    while np.any(norms < 1e-12):
        bad = norms < 1e-12
        d[bad] = rng.standard_normal((int(bad.sum()), 3))
        norms = np.linalg.norm(d, axis=1)
    d = d / norms[:, None]
    r = rc * rng.uniform(0.0, 1.0, n) ** (1.0 / 3.0)
    while np.any(r < 1e-6):
        bad = r < 1e-6
        r[bad] = rc * rng.uniform(0.0, 1.0, int(bad.sum())) ** (1.0 / 3.0)
    return offsets, d * r[:, None]


def draw_species(n_pairs: int, n_species: int, seed: int = 4) -> np.ndarray:
    """Feature value per neighbour: mu_j = -1 + 2 s_j / (S - 1), s_j ~ U{0..S-1} (S >= 2)."""
    s = np.random.default_rng(seed).integers(0, n_species, size=n_pairs)
    return -1.0 + 2.0 * s / (n_species - 1)
