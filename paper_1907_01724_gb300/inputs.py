"""Seeded synthetic inputs shaped like the paper's workloads (random charges in the cavity, Sec. 4.2).

This module holds no arithmetic of the method: it only draws charge positions, charge
values and system parameters.  Both the CUDA path's tests/benchmark and the oracle
receive the arrays it returns.

Recipes (seed = 190701 + workload index):
  * positions uniform in the ball of radius a: r = a U^(1/3), direction = normalised
    Gaussian 3-vector; a "shell" population has r^3 uniform in [(a-w)^3, a^3);
  * charges are exactly half +1 and half -1 (net neutral; odd N is rounded up to even),
    randomly permuted;
  * per-system parameters of the batched and serving workloads are drawn from the
    stated laws (log-uniform N, uniform a, uniform kappa*a, eps1 in {1, 78.5}).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 190701


@dataclass
class System:
    """One cavity: geometry, dielectric data, numerical parameters and charges."""
    a: float
    eps1: float
    eps2: float
    kappa: float
    p: int
    M: int
    xyz: np.ndarray          # (N, 3) float64
    q: np.ndarray            # (N,)  float64
    tau: float = 0.1
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.q.shape[0])


def _directions(rng: np.random.Generator, n: int) -> np.ndarray:
    v = rng.standard_normal((n, 3))
    nrm = np.linalg.norm(v, axis=1, keepdims=True)
    bad = nrm[:, 0] == 0.0
    while np.any(bad):
        v[bad] = rng.standard_normal((int(bad.sum()), 3))
        nrm = np.linalg.norm(v, axis=1, keepdims=True)
        bad = nrm[:, 0] == 0.0
    return v / nrm


def uniform_ball(rng: np.random.Generator, n: int, a: float) -> np.ndarray:
    r = a * rng.random(n) ** (1.0 / 3.0)
    return _directions(rng, n) * r[:, None]


def shell(rng: np.random.Generator, n: int, a: float, width: float) -> np.ndarray:
    lo = (a - width) ** 3
    r = (lo + (a ** 3 - lo) * rng.random(n)) ** (1.0 / 3.0)
    r = np.minimum(r, np.nextafter(a, 0.0))
    return _directions(rng, n) * r[:, None]


def neutral_charges(rng: np.random.Generator, n: int) -> np.ndarray:
    q = np.ones(n)
    q[n // 2:] = -1.0
    return rng.permutation(q)


def even(n: int) -> int:
    return n + (n % 2)


def small_system(seed_offset: int = 0) -> System:
    """N=200 unit charges uniform in a=1; eps1=1, eps2=80, kappa a=1, M=400, p=20."""
    rng = np.random.default_rng(SEED_BASE + 0 + seed_offset)
    n = 200
    return System(1.0, 1.0, 80.0, 1.0, 20, 400, uniform_ball(rng, n, 1.0), neutral_charges(rng, n),
                  name="N200_uniform_eps1_80_ka1_M400_p20")


def near_interface_system(kappa_a: float = 0.5, p: int = 20, n: int = 2000, seed_offset: int = 0) -> System:
    """N=2000, 25% with r in (0.95a, a), rest uniform; eps1=1, eps2=80, M=1000."""
    rng = np.random.default_rng(SEED_BASE + 1 + seed_offset)
    n = even(n)
    n_shell = n // 4
    xyz = np.concatenate([shell(rng, n_shell, 1.0, 0.05), uniform_ball(rng, n - n_shell, 1.0)])
    xyz = xyz[rng.permutation(n)]
    return System(1.0, 1.0, 80.0, kappa_a, p, 1000, xyz, neutral_charges(rng, n),
                  name=f"N{n}_shell25_eps1_80_ka{kappa_a:g}_M1000_p{p}")


def primitive_system(n: int = 20000, seed_offset: int = 0) -> System:
    """N=20000 uniform in a=1; eps1=eps2=78.5, kappa a=3, M=2000, p=30."""
    rng = np.random.default_rng(SEED_BASE + 2 + seed_offset)
    n = even(n)
    return System(1.0, 78.5, 78.5, 3.0, 30, 2000, uniform_ball(rng, n, 1.0), neutral_charges(rng, n),
                  name=f"N{n}_uniform_eps78.5_78.5_ka3_M2000_p30")


def far_field_system(n: int = 1_000_000, seed_offset: int = 0) -> System:
    """The paper's CPU-time workload (Sec. 4.2): N random charges in the unit sphere, p = 20,
    tau = 0.1, F1/F2 = 987/1597 (M = 3196 points per shell), with the accuracy study's dielectric
    data eps1 = 2, eps2 = 80, kappa a = 5 (Sec. 4)."""
    rng = np.random.default_rng(SEED_BASE + 5 + seed_offset)
    n = even(n)
    return System(1.0, 2.0, 80.0, 5.0, 20, 3196, uniform_ball(rng, n, 1.0), neutral_charges(rng, n),
                  name=f"N{n}_uniform_eps2_80_ka5_M3196_p20")


def _loguniform_int(rng, lo: int, hi: int, size: int) -> np.ndarray:
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size))).astype(np.int64)


def batched_systems(count: int = 512, n_lo: int = 100, n_hi: int = 10000, M: int = 1000, p: int = 20,
                    seed_offset: int = 0) -> list[System]:
    """Independent cavities: N log-uniform, a ~ U[0.8,1.5], kappa a ~ U[0.5,3], eps1 in {1, 78.5}, eps2 = 78.5."""
    rng = np.random.default_rng(SEED_BASE + 3 + seed_offset)
    ns = _loguniform_int(rng, n_lo, n_hi, count)
    out = []
    for s in range(count):
        n = even(int(ns[s]))
        a = float(rng.uniform(0.8, 1.5))
        ka = float(rng.uniform(0.5, 3.0))
        eps1 = 1.0 if rng.random() < 0.5 else 78.5
        xyz = uniform_ball(rng, n, a)
        q = neutral_charges(rng, n)
        out.append(System(a, eps1, 78.5, ka / a, p, M, xyz, q, name=f"batch{s}"))
    return out


@dataclass
class ServingWorkload:
    """Monte Carlo chains plus a seeded request stream (single-charge moves and full energies)."""
    chains: list[System]
    seed: int
    frac_delta: float = 0.9
    step_frac: float = 0.05
    rng: np.random.Generator = field(default=None, repr=False)

    def __post_init__(self):
        if self.rng is None:
            self.rng = np.random.default_rng(self.seed)

    def next_request(self, chain_positions: list[np.ndarray]) -> dict:
        """Draw one request: kind, chain, and for moves the charge index and its new position."""
        rng = self.rng
        c = int(rng.integers(len(self.chains)))
        if rng.random() >= self.frac_delta:
            return {"kind": "energy", "chain": c}
        sysc = self.chains[c]
        xyz = chain_positions[c]
        k = int(rng.integers(sysc.n))
        while True:
            step = uniform_ball(rng, 1, self.step_frac * sysc.a)[0]
            x_new = xyz[k] + step
            if float(np.dot(x_new, x_new)) < (sysc.a * (1.0 - 1e-9)) ** 2:
                break
        accept = bool(rng.random() < 0.5)
        return {"kind": "delta", "chain": c, "k": k, "x_new": x_new, "accept": accept}

    def interarrival(self, rate: float) -> float:
        return float(self.rng.exponential(1.0 / rate))


def serving_workload(count: int = 64, n_lo: int = 500, n_hi: int = 50000, M: int = 1000, p: int = 20,
                     seed_offset: int = 0) -> ServingWorkload:
    rng = np.random.default_rng(SEED_BASE + 4 + seed_offset)
    ns = _loguniform_int(rng, n_lo, n_hi, count)
    chains = []
    for s in range(count):
        n = even(int(ns[s]))
        a = float(rng.uniform(0.8, 1.5))
        ka = float(rng.uniform(0.5, 3.0))
        eps1 = 1.0 if rng.random() < 0.5 else 78.5
        chains.append(System(a, eps1, 78.5, ka / a, p, M, uniform_ball(rng, n, a), neutral_charges(rng, n),
                             name=f"chain{s}"))
    return ServingWorkload(chains, seed=SEED_BASE + 4 + 1000 + seed_offset)
