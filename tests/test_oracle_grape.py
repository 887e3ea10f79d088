"""Pins of the oracle's propagation, fidelity and gradient (Eqs. exppropagator, probability,
propagator_differentiation) against closed forms, invariants and finite differences."""
from math import comb

import numpy as np
import pytest

from oracle import grape as gr
from oracle import operators as op
from oracle import symmetry as sy
from paper_2309_05884_gb300 import inputs as I


def full_problem(system, psi0, psif):
    H0, Hc = op.system_operators(system)
    return [dict(h0=H0.toarray(), hc=[h.toarray() for h in Hc],
                 psi0=psi0[:, None], psif=psif[:, None])]


def block_problem(system, psi0, psif):
    H0, Hc = op.system_operators(system)
    return sy.block_problem(system, H0, Hc, sy.symmetry_blocks(system), psi0, psif)


def c1_states():
    return I.basis_state(4, 0), op.dicke_state(4, 2)


def test_single_qubit_rabi():
    # H = u sigma_x held for time T: P(|1>) = sin^2(u T)
    u0, T, N = 0.37, 3.0, 40
    s = I.System(1, I.GROUP_SN, [], [[(I.SUM_X, 1.0, 0)]], T, N)
    prob = full_problem(s, I.basis_state(1, 0), I.basis_state(1, 1))
    u = np.full((N, 1), u0)
    assert abs(gr.fidelity(prob, u, s.tau) - np.sin(u0 * T) ** 2) < 1e-13


@pytest.mark.parametrize("n", [3, 6, 12, 40])
def test_collective_rabi_in_symmetric_block(n):
    # H = u sum_i X_i: |<D(n,k)|psi(T)>|^2 = C(n,k) cos^{2(n-k)}(uT) sin^{2k}(uT), from the
    # J = n/2 block alone (no 2^n space), using the collective-spin form of sum X.
    u0, T, N = 0.21, 2.5, 25
    Jz, Jp, Jm = sy.spin_matrices(n)
    m = n + 1
    for k in (0, 1, n // 2, n):
        psi0 = np.zeros((m, 1), complex)
        psi0[0] = 1
        psif = np.zeros((m, 1), complex)
        psif[k] = 1
        prob = [dict(h0=np.zeros((m, m)), hc=[Jp + Jm], psi0=psi0, psif=psif)]
        F = gr.fidelity(prob, np.full((N, 1), u0), T / N)
        want = comb(n, k) * np.cos(u0 * T) ** (2 * (n - k)) * np.sin(u0 * T) ** (2 * k)
        assert abs(F - want) < 1e-12


def test_detuned_rabi_all_flip():
    # H = h sum Z + u sum X (separable): each qubit flips with p = (u/Omega)^2 sin^2(Omega T)
    n, h, u0, T, N = 3, 0.4, 0.3, 5.0, 50
    s = I.System(n, I.GROUP_SN, [(I.SUM_Z, h, 0)], [[(I.SUM_X, 1.0, 0)]], T, N)
    prob = full_problem(s, I.basis_state(n, 0), I.basis_state(n, 2 ** n - 1))
    Om = np.hypot(u0, h)
    p = (u0 / Om) ** 2 * np.sin(Om * T) ** 2
    assert abs(gr.fidelity(prob, np.full((N, 1), u0), s.tau) - p ** n) < 1e-12


def test_sigma_x_transfer_all_up_to_all_down():
    # u T = pi/2 under H = u sum X realises sigma_x^{(x)n} up to phase: F(up^n -> down^n) = 1
    n, N, T = 5, 10, 1.0
    s = I.System(n, I.GROUP_SN, [], [[(I.SUM_X, 1.0, 0)]], T, N)
    prob = block_problem(s, I.basis_state(n, 0), I.basis_state(n, 2 ** n - 1))
    assert len(prob) == 1 and prob[0]["h0"].shape == (n + 1, n + 1)
    assert abs(gr.fidelity(prob, np.full((N, 1), np.pi / 2 / T), s.tau) - 1.0) < 1e-12


def test_propagators_unitary():
    s = I.c1_system()
    prob = block_problem(s, *c1_states())
    u = I.pulses_uniform(0, s.N, 2)
    for b in prob:
        U = gr.propagators(b, u, s.tau)
        eye = np.eye(U.shape[1])
        assert np.abs(np.conj(np.swapaxes(U, -1, -2)) @ U - eye).max() < 1e-12


def test_diagonal_case_analytic_phases():
    # u == 0 and c1's H0 = 2 Jz^2 - 2 + Jz (n = 4) is diagonal in |J=2, M>: U_k are phases
    s = I.c1_system()
    psi0 = I.random_state(7, 5)[:, None]
    M = np.array([2, 1, 0, -1, -2], dtype=float)
    E = 2 * M ** 2 - 2 + M
    Jz, Jp, Jm = sy.spin_matrices(4)
    blk = dict(h0=np.diag(E), hc=[Jp + Jm, -1j * (Jp - Jm)], psi0=psi0, psif=psi0)
    psiN = gr.final_states([blk], np.zeros((s.N, 2)), s.tau)[0]
    assert np.abs(psiN[:, 0] - np.exp(-1j * s.T * E) * psi0[:, 0]).max() < 1e-12
    # and the oracle's own S_4 block of H0 is that diagonal
    prob = block_problem(s, *c1_states())
    assert np.abs(prob[0]["h0"] - np.diag(E)).max() < 1e-12


def _fd_check(prob, u, tau, seed, tol=1e-6):
    _, _, g = gr.fidelity_and_grad(prob, u, tau)
    entries = I.fd_entries(seed, *u.shape)
    fd = gr.gradient_fd(prob, u, tau, entries)
    ge = np.array([g[k, j] for k, j in entries])
    scale = np.abs(g).max()
    assert np.abs(ge - fd).max() <= tol * scale
    return g


def test_gradient_fd_c1_full_space():
    s = I.c1_system()
    prob = full_problem(s, *c1_states())
    _fd_check(prob, I.pulses_uniform(0, s.N, 2), s.tau, seed=3)


def test_gradient_fd_dn_all_blocks():
    s = I.xxz_ring(6, 4.0, 40)
    prob = block_problem(s, I.random_state(11, 64), I.random_state(12, 64))
    assert len(prob) == 6
    _fd_check(prob, I.pulses_normal(1, s.N, 3), s.tau, seed=3)


def test_gradient_fd_large_norm_slices():
    # slices with |tau H| of order 10 exercise the degenerate-free DK quotient far from 0
    s = I.sn_allpairs(8, 2.0, 1.0, 10.0, 20)
    prob = block_problem(s, I.basis_state(8, 0), op.dicke_state(8, 3))
    _fd_check(prob, I.pulses_uniform(4, s.N, 2), s.tau, seed=5, tol=2e-6)


@pytest.mark.parametrize("system_fn,seed", [
    (I.c1_system, 0), (lambda: I.xxz_ring(6, 4.0, 40), 2),
    (lambda: I.ising_ring_full(8, 1.0, [0.8, 0.37, 0.23, 0.11], 3.0, 12), 4),
    pytest.param(lambda: I.xxz_ring(10, 1.0, 4), 6, marks=pytest.mark.slow)],
    ids=["c1", "xxz6", "ising8_full", "xxz10"])
def test_full_space_equals_block_space(system_fn, seed):
    s = system_fn()
    dim = 2 ** s.n
    psi0, psif = I.random_state(seed + 20, dim), I.random_state(seed + 21, dim)
    u = I.pulses_uniform(seed, s.N, s.n_ctrl)
    Ff, of, gf = gr.fidelity_and_grad(full_problem(s, psi0, psif), u, s.tau)
    Fb, ob, gb = gr.fidelity_and_grad(block_problem(s, psi0, psif), u, s.tau)
    assert abs(of - ob) < 1e-12
    assert np.abs(gf - gb).max() < 1e-12 * max(1.0, np.abs(gf).max())
    # full-space evolution A (+) U_b A^dagger psi0 equals prod U_k psi0
    blocks = sy.symmetry_blocks(s)
    prob_all = [dict(h0=sy.block_operator(V[0], op.system_operators(s)[0]),
                     hc=[sy.block_operator(V[0], h) for h in op.system_operators(s)[1]],
                     psi0=c, psif=c)
                for (_, V), c in zip(blocks, sy.to_blocks(blocks, psi0))]
    psiN_blocks = gr.final_states(prob_all, u, s.tau)
    psiN_full = gr.final_states(full_problem(s, psi0, psi0), u, s.tau)[0][:, 0]
    assert np.abs(sy.from_blocks(blocks, psiN_blocks) - psiN_full).max() < 1e-12


def test_first_order_gradient_limit():
    # exact minus first-order slice derivative is O(tau) relative: halving tau halves it
    s = I.c1_system()
    prob = full_problem(s, *c1_states())
    rels = []
    for N in (100, 200, 400):
        u = np.repeat(I.pulses_uniform(0, 100, 2), N // 100, axis=0)
        _, _, g = gr.fidelity_and_grad(prob, u, s.T / N)
        g1 = gr.gradient_first_order(prob, u, s.T / N)
        rels.append(np.linalg.norm(g - g1) / np.linalg.norm(g))
    assert rels[0] > 1e-4
    for a, b in zip(rels, rels[1:]):
        assert 1.7 < a / b < 2.3


def test_grape_invariance_full_vs_block():
    # Sec. II.B: original and transformed Hamiltonians give the same optimal pulses
    s = I.c1_system()
    u0 = I.pulses_uniform(0, s.N, 2)
    uf, hf, _ = gr.grape(full_problem(s, *c1_states()), u0, s.tau, 200, 0.2)
    ub, hb, _ = gr.grape(block_problem(s, *c1_states()), u0, s.tau, 200, 0.2)
    assert np.abs(uf - ub).max() < 1e-10
    assert hf[-1] > hf[0]


def test_adam_first_step_is_signed_step():
    # with zero moments, the first Adam step moves every coordinate by step * sign(g) (up to eps)
    g = np.array([[0.3, -2.0], [1e-3, 5.0]])
    u, m, v = gr.adam_update(np.zeros_like(g), g, np.zeros_like(g), np.zeros_like(g), 1, 0.1)
    assert np.allclose(u, 0.1 * np.sign(g), atol=1e-6)
    # and the second step with the same gradient again moves by step * sign(g)
    u2, _, _ = gr.adam_update(u, g, m, v, 2, 0.1)
    assert np.allclose(u2 - u, 0.1 * np.sign(g), atol=1e-6)


def test_grape_adam_escapes_tiny_overlap():
    # |0...0> -> D(6, 3) with weak random pulses: F starts near 0, fixed steps barely move, Adam
    # (scale-free steps) reaches F >= 0.999
    n, N, T = 6, 60, 1.0
    Jz, Jp, Jm = sy.spin_matrices(n)
    m = n + 1
    p0 = np.zeros((m, 1), complex)
    p0[0] = 1
    pf = np.zeros((m, 1), complex)
    pf[3] = 1
    prob = [dict(h0=0.8 * (2 * Jz @ Jz - n / 2 * np.eye(m)) + 0.4 * 2 * Jz, hc=[Jp + Jm, -1j * (Jp - Jm)],
                 psi0=p0, psif=pf)]
    u0 = I.pulses_uniform(1, N, 2, -0.1, 0.1)
    _, hist, reached = gr.grape_adam(prob, u0, T / N, 2000, 0.5, f_target=0.999)
    assert hist[0] < 1e-3 and reached >= 0 and hist[-1] >= 0.999
