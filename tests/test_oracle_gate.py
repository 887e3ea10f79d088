"""Pins of the oracle's gate (unitary) objective F = |Tr(W^dagger U_N...U_1) / d|^2 (the trace fidelity
of Sec. IV with a gate as the target; sigma_x^{(x)n} and U_sq^{(x)n} gates of Sec. III): closed forms
for tensor-power gates, full space == block form with copy multiplicities, the maximum at W = U, and
central finite differences of the plain trace definition."""
import numpy as np
import pytest

from oracle import grape as gr
from oracle import operators as op
from oracle import symmetry as sy
from paper_2309_05884_gb300 import inputs as I

X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def tensor_power(a, n):
    out = np.ones((1, 1), dtype=np.complex128)
    for _ in range(n):
        out = np.kron(out, a)
    return out


def expm_herm(h, t):
    """exp(-i t h) of a Hermitian matrix by its eigendecomposition."""
    w, V = np.linalg.eigh(h)
    return (V * np.exp(-1j * t * w)) @ V.conj().T


def seeded_unitary(seed, m=2):
    g = I.rng(seed)
    q, r = np.linalg.qr(g.standard_normal((m, m)) + 1j * g.standard_normal((m, m)))
    return q * (np.diag(r) / np.abs(np.diag(r)))


def full_form(s):
    H0, Hc = op.system_operators(s)
    return [dict(h0=H0.toarray(), hc=[h.toarray() for h in Hc])]


def block_form(s, W_full):
    """Blocks of H0, Hc_j and of the symmetric gate W in the oracle's adapted basis, with the copy
    multiplicities; W must not couple blocks."""
    H0, Hc = op.system_operators(s)
    blocks = sy.symmetry_blocks(s)
    A = sy.adjoint_matrix(blocks)
    Wa = A.conj().T @ W_full @ A
    mask = np.zeros_like(Wa, dtype=bool)
    o = 0
    for _, V in blocks:
        for _r in range(V.shape[0]):
            m = V.shape[1]
            mask[o:o + m, o:o + m] = True
            o += m
    assert np.abs(Wa[~mask]).max(initial=0.0) < 1e-12  # a symmetric gate stays in its blocks
    blks = [dict(h0=sy.block_operator(V[0], H0), hc=[sy.block_operator(V[0], h) for h in Hc]) for _, V in blocks]
    Ws = [sy.block_operator(V[0], W_full) for _, V in blocks]
    mult = [V.shape[0] for _, V in blocks]
    return blks, Ws, mult


def no_drift(n, T, N):
    return I.System(n, I.GROUP_SN, [], [[(I.SUM_X, 1.0, 0)], [(I.SUM_Y, 1.0, 0)]], T, N)


@pytest.mark.parametrize("n", [3, 4, 5])
def test_sigma_x_power_gate_at_quarter_period(n):
    # H = u sum X with u T = pi/2: U = exp(-i pi/2 sum X) = (-i)^n X^{(x)n}, so F(X^{(x)n}) = 1, and
    # Tr(X^{(x)n}) = 0 gives F(I) = 0
    T, N = 2.0, 8
    s = no_drift(n, T, N)
    u = np.zeros((N, 2))
    u[:, 0] = np.pi / (2 * T)
    Xn = tensor_power(X, n)
    for blks, Ws, mult in [(full_form(s), [Xn], [1]), block_form(s, Xn)]:
        assert abs(gr.gate_fidelity(blks, Ws, mult, u, s.tau) - 1.0) < 1e-12
        g = gr.gate_overlap(blks, Ws, mult, u, s.tau)
        assert abs(g - (-1j) ** n) < 1e-12
    blks, Ws, mult = block_form(s, np.eye(2 ** n))
    assert gr.gate_fidelity(blks, Ws, mult, u, s.tau) < 1e-24


@pytest.mark.parametrize("n", [2, 4, 5])
def test_product_gate_closed_form(n):
    # no coupling: H = a sum X + b sum Y + c sum Z is a sum of one-qubit terms, U = u1^{(x)n} with
    # u1 = exp(-i T (a X + b Y + c Z)), and Tr(A^{(x)n}) = Tr(A)^n gives, for the gate V^{(x)n},
    # F = |Tr(V^dagger u1) / 2|^{2n}.  The block form must weight every S_n sector by its multiplicity.
    a, b, c, T, N = 0.37, -0.21, 0.55, 1.7, 6
    s = I.System(n, I.GROUP_SN, [(I.SUM_Z, c, 0)], [[(I.SUM_X, 1.0, 0)], [(I.SUM_Y, 1.0, 0)]], T, N)
    u = np.tile([a, b], (N, 1))
    u1 = expm_herm(a * X + b * Y + c * Z, T)
    V = seeded_unitary(17)
    want = abs(np.trace(V.conj().T @ u1) / 2) ** (2 * n)
    Vn = tensor_power(V, n)
    for blks, Ws, mult in [(full_form(s), [Vn], [1]), block_form(s, Vn)]:
        assert abs(gr.gate_fidelity(blks, Ws, mult, u, s.tau) - want) < 1e-12
        F, _, _ = gr.gate_fidelity_and_grad(blks, Ws, mult, u, s.tau)
        assert abs(F - want) < 1e-12
    if n >= 4:
        # the sectors' multiplicities differ here, so dropping them changes F
        blks, Ws, mult = block_form(s, Vn)
        assert len(set(mult)) > 1
        assert abs(gr.gate_fidelity(blks, Ws, [1] * len(mult), u, s.tau) - want) > 1e-6


def test_block_form_equals_full_space_dn_ring():
    # D_6 XXZ ring; V^{(x)n} commutes with every qubit permutation, so it is block diagonal
    s = I.xxz_ring(6, 1.5, 12)
    u = I.pulses_normal(5, s.N, 3)
    W = tensor_power(seeded_unitary(23), s.n)
    Ff, gf, df = gr.gate_fidelity_and_grad(full_form(s), [W], [1], u, s.tau)
    blks, Ws, mult = block_form(s, W)
    Fb, gb, db = gr.gate_fidelity_and_grad(blks, Ws, mult, u, s.tau)
    assert abs(gf - gb) < 1e-12
    assert abs(Ff - Fb) < 1e-12
    assert np.abs(df - db).max() < 1e-12 * max(1.0, np.abs(df).max())
    assert abs(gr.gate_overlap(blks, Ws, mult, u, s.tau) - gb) < 1e-12


def test_maximum_at_the_reached_gate():
    # W = U(u) itself: F = 1 and dF/du = 0 (a maximum of |g|^2 <= 1)
    s = I.xxz_ring(5, 1.0, 10)
    u = I.pulses_normal(6, s.N, 3)
    H0, Hc = op.system_operators(s)
    blocks = sy.symmetry_blocks(s)
    blks = [dict(h0=sy.block_operator(V[0], H0), hc=[sy.block_operator(V[0], h) for h in Hc]) for _, V in blocks]
    Ws = []
    for blk in blks:
        K = np.eye(blk["h0"].shape[0], dtype=np.complex128)
        for U in gr.propagators(blk, u, s.tau):
            K = U @ K
        Ws.append(K)
    mult = [V.shape[0] for _, V in blocks]
    F, g, grad = gr.gate_fidelity_and_grad(blks, Ws, mult, u, s.tau)
    assert abs(F - 1.0) < 1e-12 and abs(g - 1.0) < 1e-12
    assert np.abs(grad).max() < 1e-10


def test_gradient_matches_central_differences_of_the_trace():
    # the exact gradient (costate form) against central differences of the plain trace definition,
    # h = 1e-6 on 20 seeded entries
    s = I.ising_ring(5, 1.0, 0.8, 2.0, 20)
    u = I.pulses_uniform(8, s.N, 2)
    blks, Ws, mult = block_form(s, tensor_power(seeded_unitary(29), s.n))
    F, _, grad = gr.gate_fidelity_and_grad(blks, Ws, mult, u, s.tau)
    assert F > 1e-4
    entries = I.fd_entries(3, s.N, 2)
    h = 1e-6
    fd = []
    for k, j in entries:
        up, dn = u.copy(), u.copy()
        up[k, j] += h
        dn[k, j] -= h
        fd.append((gr.gate_fidelity(blks, Ws, mult, up, s.tau) - gr.gate_fidelity(blks, Ws, mult, dn, s.tau)) / (2 * h))
    sel = np.array([grad[k, j] for k, j in entries])
    assert np.linalg.norm(np.array(fd) - sel) / np.linalg.norm(sel) < 1e-6
