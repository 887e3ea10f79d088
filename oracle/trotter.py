"""Oracle: the Trotterised propagator for per-qubit controls and the trace fidelity that compares
propagators (Sec. IV; test infrastructure only).

With one pair of pulses per qubit (Eq. Hcprime) and the ring coupling (Eq. completeH_cpl), slice j has
    H_j = sum_i h^(i)_j + H_cpl,  h^(i)_j = Bz/2 sigma_z^(i) + 1/2 (Bx^(i)_j sigma_x^(i) + By^(i)_j sigma_y^(i)),
    H_cpl = c/4 sum_i sigma_z^(i) sigma_z^(i+1),
and the original step is U_j = exp(-i tau H_j) (Eq. exppropagator).  The Trotterised step (Eq.
propagator_cpl) is the ordered product over qubits i = 1..n (factor i = 1 leftmost) of
exp(-i tau h^(i)_j) exp(-i tau/n H_cpl); its local error is O(n^2 tau^2).  In the transformed form
(Eq. propagator_cpl_transformed) each single-qubit factor is A_i exp(-i tau A_i^dagger h^(i) A_i)
A_i^dagger, where A_i swaps qubits i and n, so that A_i^dagger sigma^(i) A_i = sigma^(n) =
I_{2^{n-1}} (x) sigma (2^{n-1} identical 2 x 2 blocks: one 2 x 2 exponential per qubit and slice),
and the coupling factor is A_D exp(-i tau/n A_D^dagger H_cpl A_D) A_D^dagger with the D_n adjoint
matrix (one exponential per D_n block, computed once).  Propagators K, K' of the full space are
compared by F = |Tr(K^dagger K') / 2^n|^2.

Pins: tests/test_oracle_trotter.py (exact without coupling, the swap identity, transformed ==
untransformed, second-order convergence of the infidelity in tau).
"""
from __future__ import annotations

import numpy as np

from . import operators as op
from . import symmetry as sy


def expm_herm(H: np.ndarray, t: float) -> np.ndarray:
    """exp(-i t H) of a Hermitian matrix, by its eigendecomposition."""
    w, V = np.linalg.eigh(H)
    return (V * np.exp(-1j * t * w)) @ V.conj().T


def swap_permutation(n: int, i: int) -> np.ndarray:
    """A_(i,n): the permutation of computational states that exchanges qubits i and n (1-based)."""
    dim = 1 << n
    P = np.zeros((dim, dim))
    bi, bn = n - i, 0  # bit positions of qubits i and n (qubit 1 is the most significant bit)
    for x in range(dim):
        a, b = (x >> bi) & 1, (x >> bn) & 1
        y = x & ~((1 << bi) | (1 << bn)) | (b << bi) | (a << bn)
        P[y, x] = 1.0
    return P


def qubit_term(Bz: float, bx: float, by: float) -> np.ndarray:
    """The 2 x 2 single-qubit Hamiltonian Bz/2 sigma_z + 1/2 (bx sigma_x + by sigma_y)."""
    return 0.5 * (Bz * op.SZ + bx * op.SX + by * op.SY)


def coupling(n: int, c: float) -> np.ndarray:
    """H_cpl = c/4 sum_i sigma_z^(i) sigma_z^(i+1) (periodic), dense."""
    return 0.25 * c * op.term_matrix(n, op.RING_ZZ, 1).toarray()


def slice_hamiltonian(n: int, Bz: float, c: float, bx, by) -> np.ndarray:
    """H_j of Eq. completeH_cpl for the per-qubit pulse values bx[i], by[i] of one slice."""
    H = coupling(n, c).astype(np.complex128)
    for i in range(1, n + 1):
        H = H + 0.5 * (Bz * op.sigma(n, i, "z") + bx[i - 1] * op.sigma(n, i, "x") + by[i - 1] * op.sigma(n, i, "y"))
    return np.asarray(H)


def original_step(n, Bz, c, bx, by, tau):
    return expm_herm(slice_hamiltonian(n, Bz, c, bx, by), tau)


def trotter_step(n, Bz, c, bx, by, tau):
    """Eq. propagator_cpl: prod_{i=1..n} exp(-i tau h^(i)) exp(-i tau/n H_cpl), full-space factors."""
    Ec = expm_herm(coupling(n, c), tau / n)
    U = np.eye(1 << n, dtype=np.complex128)
    for i in range(1, n + 1):
        hi = np.asarray(0.5 * (Bz * op.sigma(n, i, "z") + bx[i - 1] * op.sigma(n, i, "x")
                               + by[i - 1] * op.sigma(n, i, "y")).toarray())
        U = U @ expm_herm(hi, tau) @ Ec
    return U


def coupling_factor_by_blocks(n: int, c: float, tau: float) -> np.ndarray:
    """A_D exp(-i tau/n A_D^dagger H_cpl A_D) A_D^dagger with one exponential per D_n block."""
    blocks = sy.dn_blocks(n)
    Hc = coupling(n, c)
    out = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for _, V in blocks:
        Eb = expm_herm(sy.block_operator(V[0], Hc), tau / n)
        for r in range(V.shape[0]):
            Vr = V[r].T  # [2^n, m]: the copy's basis vectors as columns
            out += Vr @ Eb @ Vr.conj().T
    return out


def trotter_step_transformed(n, Bz, c, bx, by, tau, coupling_factor=None):
    """Eq. propagator_cpl_transformed: the single-qubit factors as A_i (I (x) e_i) A_i^dagger with the
    2 x 2 exponential e_i = exp(-i tau h^(i)), the coupling factor from the D_n blocks."""
    Ec = coupling_factor_by_blocks(n, c, tau) if coupling_factor is None else coupling_factor
    eye = np.eye(1 << (n - 1))
    U = np.eye(1 << n, dtype=np.complex128)
    for i in range(1, n + 1):
        A = swap_permutation(n, i)
        e = expm_herm(qubit_term(Bz, bx[i - 1], by[i - 1]), tau)
        U = U @ (A @ np.kron(eye, e) @ A.T) @ Ec
    return U


def evolve(step, n, Bz, c, bx, by, tau) -> np.ndarray:
    """K = U_N ... U_1 for the per-slice pulse arrays bx, by of shape [N, n]."""
    K = np.eye(1 << n, dtype=np.complex128)
    for j in range(bx.shape[0]):
        K = step(n, Bz, c, bx[j], by[j], tau) @ K
    return K


def trace_fidelity(K1: np.ndarray, K2: np.ndarray) -> float:
    """F = |Tr(K1^dagger K2) / d|^2 (Sec. IV)."""
    return abs(np.trace(K1.conj().T @ K2) / K1.shape[0]) ** 2
