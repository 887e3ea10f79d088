"""Pins of the oracle's Trotterised propagator for per-qubit controls (Sec. IV, Eqs. propagator_cpl and
propagator_cpl_transformed) and of the trace fidelity that compares it with the original propagator."""
import numpy as np
import pytest

from oracle import operators as op
from oracle import trotter as tr
from paper_2309_05884_gb300 import inputs as I

BZ, C, T = 1.0, 0.8, 2.0


def smooth_pulses(seed, n, N):
    """Per-qubit pulses Bx^(i)(t), By^(i)(t) = a cos(w t + phi) (seeded a, w, phi), sampled at the slice
    midpoints (j + 1/2) tau, so that refining tau samples the same functions."""
    g = I.rng(seed)
    amp = g.uniform(0.5, 1.5, (2, n))
    w = g.uniform(0.5, 2.0, (2, n))
    ph = g.uniform(0.0, 2 * np.pi, (2, n))
    t = (np.arange(N) + 0.5) * T / N
    return [amp[a] * np.cos(w[a] * t[:, None] + ph[a]) for a in range(2)]


@pytest.mark.parametrize("n", [3, 4, 5])
def test_swap_moves_a_qubit_term_to_the_last_qubit(n):
    # A_(i,n)^dagger sigma_a^(i) A_(i,n) = sigma_a^(n) = I_{2^{n-1}} (x) sigma_a: 2^{n-1} identical 2 x 2 blocks
    for i in range(1, n + 1):
        A = tr.swap_permutation(n, i)
        assert np.array_equal(A.T @ A, np.eye(2 ** n))
        for a in "xyz":
            moved = A.T @ op.sigma(n, i, a).toarray() @ A
            assert np.abs(moved - np.kron(np.eye(2 ** (n - 1)), op.PAULI[a])).max() == 0.0


@pytest.mark.parametrize("n", [3, 5])
def test_exact_without_coupling(n):
    # c = 0: the single-qubit terms commute, so the Trotterised step is the exact step
    bx, by = smooth_pulses(1, n, 12)
    tau = T / 12
    Ko = tr.evolve(tr.original_step, n, BZ, 0.0, bx, by, tau)
    Kt = tr.evolve(tr.trotter_step, n, BZ, 0.0, bx, by, tau)
    assert np.abs(Ko - Kt).max() < 1e-12
    assert abs(tr.trace_fidelity(Kt, Ko) - 1.0) < 1e-12


def test_transformed_equals_untransformed():
    # Eq. propagator_cpl_transformed is Eq. propagator_cpl written through A_i and A_D
    n = 5
    bx, by = smooth_pulses(2, n, 6)
    tau = T / 6
    Kt = tr.evolve(tr.trotter_step, n, BZ, C, bx, by, tau)
    Ec = tr.coupling_factor_by_blocks(n, C, tau)
    Kx = tr.evolve(lambda *a: tr.trotter_step_transformed(*a, coupling_factor=Ec), n, BZ, C, bx, by, tau)
    assert np.abs(Kt - Kx).max() < 1e-12
    assert np.abs(Ec - tr.expm_herm(tr.coupling(n, C), tau / n)).max() < 1e-12


def test_infidelity_is_second_order_in_tau():
    # a local error O(n^2 tau^2) per step accumulates to O(tau) in K, so 1 - F = O(tau^2): halving tau
    # over the same time divides the infidelity by 4
    n = 4
    infid = []
    for N in (20, 40, 80):
        bx, by = smooth_pulses(5, n, N)
        tau = T / N
        Ko = tr.evolve(tr.original_step, n, BZ, C, bx, by, tau)
        Kt = tr.evolve(tr.trotter_step, n, BZ, C, bx, by, tau)
        infid.append(1.0 - tr.trace_fidelity(Kt, Ko))
    assert infid[0] > 1e-5
    for a, b in zip(infid, infid[1:]):
        assert 3.8 < a / b < 4.2


def test_trace_fidelity_basics():
    n = 3
    bx, by = smooth_pulses(7, n, 5)
    K = tr.evolve(tr.original_step, n, BZ, C, bx, by, T / 5)
    assert abs(tr.trace_fidelity(K, K) - 1.0) < 1e-12
    assert abs(tr.trace_fidelity(K, np.exp(0.7j) * K) - 1.0) < 1e-12  # global phase drops out
    X = tr.swap_permutation(n, 1) @ K
    assert tr.trace_fidelity(K, X) <= 1.0 + 1e-12
