"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle's tests.

This module holds data only: the Hamiltonian term lists of the benchmark systems
(Eqs. H0WithCoupling and Hc of the paper, Sec. II.B, and the XXZ/all-pairs variants the
workloads use), the time grids, and seeded random pulses and states.  It contains none of
the method's arithmetic (no operators, no symmetry transforms, no propagation), so both the
oracle and the CUDA path can draw identical inputs from it without sharing any code.

Random numbers come from numpy's PCG64 with explicit seeds.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

# ---------------------------------------------------------------------------------------
# Term kinds.  Each term is (kind, coeff, dist).  Qubits are indexed i = 1..n, qubit 1 is
# the most significant bit of a computational-basis index, |0> = |up> (sigma_z = +1).
#   SUM_a       : sum_i sigma_a^(i)                                   (Sec. II.A)
#   ALLPAIRS_aa : sum_{i<j} sigma_a^(i) sigma_a^(j)                   (S_n-invariant)
#   RING_aa     : sum_{i=1..n} sigma_a^(i) sigma_a^(i+dist), periodic (Eq. H0MoreCoupling1)
# The numeric values are part of the C ABI (include/qoc.h, enum qoc_term_kind).
# ---------------------------------------------------------------------------------------
SUM_X, SUM_Y, SUM_Z = 0, 1, 2
ALLPAIRS_XX, ALLPAIRS_YY, ALLPAIRS_ZZ = 3, 4, 5
RING_XX, RING_YY, RING_ZZ = 6, 7, 8

GROUP_SN, GROUP_DN = 0, 1

Term = Tuple[int, float, int]


@dataclass
class System:
    """A control problem's static description: H0 and the control Hamiltonians Hc_j."""
    n: int
    group: int
    h0: List[Term]
    hc: List[List[Term]]
    T: float
    N: int
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n_ctrl(self) -> int:
        return len(self.hc)

    @property
    def tau(self) -> float:
        return self.T / self.N


def ising_ring(n: int, Bz: float, c_cpl: float, T: float, N: int) -> System:
    """Eqs. H0WithCoupling / Hc: H0 = Bz/2 sum Z + c/4 sum Z_i Z_{i+1}; Hc = Bx/2 sum X + By/2 sum Y."""
    h0 = [(SUM_Z, 0.5 * Bz, 0)]
    group = GROUP_SN
    if c_cpl != 0.0:
        h0.append((RING_ZZ, 0.25 * c_cpl, 1))
        group = GROUP_DN
    hc = [[(SUM_X, 0.5, 0)], [(SUM_Y, 0.5, 0)]]
    return System(n, group, h0, hc, T, N, name=f"ising_ring_n{n}")


def ising_ring_full(n: int, Bz: float, c_cpl: List[float], T: float, N: int) -> System:
    """Eq. H0MoreCoupling1: H0 = Bz/2 sum Z + sum_{d=1..floor(n/2)} c^(d)/4 sum_i Z_i Z_{i+d} (every
    ring distance, taken literally, so d = n/2 counts each pair twice for even n); Hc as in Eq. Hc."""
    assert len(c_cpl) == n // 2
    h0 = [(SUM_Z, 0.5 * Bz, 0)] + [(RING_ZZ, 0.25 * c, d + 1) for d, c in enumerate(c_cpl) if c != 0.0]
    hc = [[(SUM_X, 0.5, 0)], [(SUM_Y, 0.5, 0)]]
    return System(n, GROUP_DN, h0, hc, T, N, name=f"ising_ring_full_n{n}")


def sn_allpairs(n: int, J: float, h: float, T: float, N: int) -> System:
    """S_n-invariant H0 = J sum_{i<j} Z_i Z_j + h sum Z_i; controls u_x sum X, u_y sum Y."""
    return System(n, GROUP_SN, [(ALLPAIRS_ZZ, J, 0), (SUM_Z, h, 0)],
                  [[(SUM_X, 1.0, 0)], [(SUM_Y, 1.0, 0)]], T, N, name=f"sn_allpairs_n{n}")


def xxz_ring(n: int, T: float, N: int, delta: float = 0.5) -> System:
    """D_n ring H0 = sum_i (X_i X_{i+1} + Y_i Y_{i+1} + delta Z_i Z_{i+1}); controls sum X, sum Y, sum Z."""
    return System(n, GROUP_DN, [(RING_XX, 1.0, 1), (RING_YY, 1.0, 1), (RING_ZZ, delta, 1)],
                  [[(SUM_X, 1.0, 0)], [(SUM_Y, 1.0, 0)], [(SUM_Z, 1.0, 0)]], T, N,
                  name=f"xxz_ring_n{n}")


# The five workloads.  c1 and c2 are the small / benchmark cases; c3 is the long adjoint case.
def c1_system() -> System:
    """n=4, S_n: H0 = 1.0 sum_{i<j} ZZ + 0.5 sum Z; T=10, N=100."""
    return sn_allpairs(4, 1.0, 0.5, 10.0, 100)


def c2_system() -> System:
    """n=10 XXZ ring (D_n), T=20, N=500."""
    return xxz_ring(10, 20.0, 500)


def c3_system() -> System:
    """n=14 XXZ ring (D_n), T=40, N=2000."""
    return xxz_ring(14, 40.0, 2000)


# ---------------------------------------------------------------------------------------
# Seeded generators
# ---------------------------------------------------------------------------------------
def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def pulses_uniform(seed: int, N: int, nc: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """u[k, j] ~ U[lo, hi], shape [N, nc], float64."""
    return rng(seed).uniform(lo, hi, size=(N, nc))


def pulses_normal(seed: int, N: int, nc: int, sigma: float = 0.3) -> np.ndarray:
    """u[k, j] ~ N(0, sigma^2), shape [N, nc], float64."""
    return rng(seed).normal(0.0, sigma, size=(N, nc))


def random_state(seed: int, dim: int) -> np.ndarray:
    """A complex Gaussian vector of length dim, scaled to unit 2-norm (Haar-random direction)."""
    g = rng(seed)
    v = g.normal(size=dim) + 1j * g.normal(size=dim)
    return v / np.linalg.norm(v)


def basis_state(n: int, index: int) -> np.ndarray:
    """The computational-basis state |index> of n qubits as a complex vector of length 2^n."""
    v = np.zeros(1 << n, dtype=np.complex128)
    v[index] = 1.0
    return v


def fd_entries(seed: int, N: int, nc: int, count: int = 20) -> List[Tuple[int, int]]:
    """count distinct seeded (k, j) entries of an [N, nc] pulse array."""
    g = rng(seed)
    flat = g.choice(N * nc, size=min(count, N * nc), replace=False)
    return [(int(f // nc), int(f % nc)) for f in flat]


@dataclass
class SnProblem:
    """One S_n control problem of the many-problem workload (all-pairs ZZ + field)."""
    n: int
    J: float
    h: float
    N: int
    k_target: int
    seed: int


def sn_problem_batch(count: int, base_seed: int = 10_000, n_lo: int = 8, n_hi: int = 64,
                     N_lo: int = 200, N_hi: int = 1000) -> List[SnProblem]:
    """Problem i uses seed base_seed+i: n~U{n_lo..n_hi}, J~U[0.5,2], h~U[0,1], N~U{N_lo..N_hi}, k~U{0..n}."""
    out = []
    for i in range(count):
        g = rng(base_seed + i)
        n = int(g.integers(n_lo, n_hi + 1))
        J = float(g.uniform(0.5, 2.0))
        h = float(g.uniform(0.0, 1.0))
        N = int(g.integers(N_lo, N_hi + 1))
        k = int(g.integers(0, n + 1))
        out.append(SnProblem(n, J, h, N, k, base_seed + i))
    return out
