"""Oracle: Pauli operators and full-space Hamiltonians (test infrastructure only).

Definitions (paper Sec. II.A): sigma_a^(i) = I_2^{(i-1)} (x) sigma_a (x) I_2^{(n-i)} with qubit 1
the leftmost (most significant) Kronecker factor; H_x, H_y, H_z are sums over qubits; the ring
coupling sum_i sigma^(i) sigma^(i+1) is periodic (sigma^(n+i) = sigma^(i)).  Eq.
H0MoreCoupling1 extends the ring coupling to distance d.

Pins: tests/test_oracle_operators.py (Pauli algebra; the XXZ ring's one-magnon spectrum
4 cos(2 pi k d / n) + Delta (n - 4) on the full space and per D_n irrep; exact Z-ring values at every
distance d <= n/2; the all-pairs Heisenberg coupling as 2 J (J + 1) - 3 n / 2; collective-field
spectra) and tests/test_oracle_grape.py (Rabi closed forms).
"""
from __future__ import annotations

from functools import reduce

import numpy as np
import scipy.sparse as sp

SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
I2 = np.eye(2, dtype=np.complex128)
PAULI = {"x": SX, "y": SY, "z": SZ}

# Term kinds, same numbering as the seeded-input module and the C header.
SUM_X, SUM_Y, SUM_Z = 0, 1, 2
ALLPAIRS_XX, ALLPAIRS_YY, ALLPAIRS_ZZ = 3, 4, 5
RING_XX, RING_YY, RING_ZZ = 6, 7, 8
_AXIS = {SUM_X: "x", SUM_Y: "y", SUM_Z: "z", ALLPAIRS_XX: "x", ALLPAIRS_YY: "y",
         ALLPAIRS_ZZ: "z", RING_XX: "x", RING_YY: "y", RING_ZZ: "z"}


def kron_chain(mats):
    return reduce(lambda a, b: sp.kron(a, b, format="csr"), mats)


def sigma(n: int, i: int, a: str) -> sp.csr_matrix:
    """sigma_a^(i) for 1-based qubit index i on n qubits, as a sparse 2^n x 2^n matrix."""
    mats = [sp.csr_matrix(I2)] * n
    mats = list(mats)
    mats[i - 1] = sp.csr_matrix(PAULI[a])
    return kron_chain(mats)


def term_matrix(n: int, kind: int, dist: int = 1) -> sp.csr_matrix:
    """The operator of one term kind (coefficient 1), as a sparse 2^n x 2^n matrix."""
    a = _AXIS[kind]
    dim = 1 << n
    out = sp.csr_matrix((dim, dim), dtype=np.complex128)
    if kind in (SUM_X, SUM_Y, SUM_Z):
        for i in range(1, n + 1):
            out = out + sigma(n, i, a)
    elif kind in (ALLPAIRS_XX, ALLPAIRS_YY, ALLPAIRS_ZZ):
        for i in range(1, n + 1):
            for j in range(i + 1, n + 1):
                out = out + sigma(n, i, a) @ sigma(n, j, a)
    elif kind in (RING_XX, RING_YY, RING_ZZ):
        for i in range(1, n + 1):
            j = (i - 1 + dist) % n + 1
            out = out + sigma(n, i, a) @ sigma(n, j, a)
    else:
        raise ValueError(f"unknown term kind {kind}")
    return out.tocsr()


def hamiltonian(n: int, terms) -> sp.csr_matrix:
    """sum_t coeff_t * term_t for a list of (kind, coeff, dist)."""
    dim = 1 << n
    out = sp.csr_matrix((dim, dim), dtype=np.complex128)
    for kind, coeff, dist in terms:
        out = out + coeff * term_matrix(n, kind, dist)
    return out.tocsr()


def system_operators(system):
    """(H0, [Hc_j]) for a System of the seeded-input module, as sparse full-space matrices."""
    H0 = hamiltonian(system.n, system.h0)
    Hc = [hamiltonian(system.n, t) for t in system.hc]
    return H0, Hc


def dicke_state(n: int, k: int) -> np.ndarray:
    """|D(n,k)>: the normalised equal superposition of all n-qubit basis states with k ones."""
    dim = 1 << n
    v = np.zeros(dim, dtype=np.complex128)
    for x in range(dim):
        if bin(x).count("1") == k:
            v[x] = 1.0
    return v / np.linalg.norm(v)
