"""Oracle: piecewise-constant propagation, fidelity and its gradient (test infrastructure only).

Paper Sec. II.A: with tau = T/N and the control held constant on each slice,
    psi_k = U_k psi_{k-1},  U_k = exp(-i tau (H0 + sum_j u_kj Hc_j))            (Eq. exppropagator)
and the objective is the state-transfer probability
    F = |<psi_f|psi_N>|^2                                                      (Eq. probability).
A problem is a list of blocks (the full space is the one-block case); block b carries its own
H0_b, Hc_jb and copies psi0_b, psif_b of shape [m_b, c_b]; the overlap sums over blocks and copies.

Propagators come from numpy.linalg.eigh: U = V diag(exp(-i tau w)) V^dagger.  The exact slice
derivative is the Daleckii-Krein form of the Frechet derivative of exp at X = -i tau H:
    L(X, E) = V [(V^dagger E V) o Phi] V^dagger,  Phi_ab = e^{mu_b} (e^{mu_a-mu_b} - 1)/(mu_a-mu_b),
with mu = -i tau w and E = -i tau Hc_j; the costates are lam_N = psi_f, lam_{k-1} = U_k^dagger lam_k
(unitarity, Appendix B), and
    dF/du_kj = 2 Re( conj(o) * sum_b,r lam_k^dagger L(X_k, E_j) psi_{k-1} ),  o = <psi_f|psi_N>.
The paper's own derivative (Eq. propagator_differentiation) keeps only the first-order term
-i tau Hc_j U_k; gradient_first_order implements it for the O(tau^2) comparison.

Pins (tests/test_oracle_grape.py): single-qubit and collective Rabi closed forms, detuned Rabi,
sigma_x^{(x)n} transfer, unitarity, the analytic diagonal case, central finite differences, the
first-order limit, and full-space == block-space trajectories.  The gate objective at the end of
this file (trace fidelity of Sec. IV against a target gate) is pinned in tests/test_oracle_gate.py:
tensor-power closed forms, full space == block form with copy multiplicities, the maximum at the
reached gate, and central differences of the plain trace.
"""
from __future__ import annotations

import numpy as np


def _as_blocks(problem):
    return problem if isinstance(problem, (list, tuple)) else [problem]


def slice_hamiltonians(blk, u: np.ndarray) -> np.ndarray:
    """H_k = H0 + sum_j u_kj Hc_j for all slices k: [N, m, m]."""
    h0 = np.asarray(blk["h0"], dtype=np.complex128)
    H = np.broadcast_to(h0, (u.shape[0],) + h0.shape).copy()
    for j, hc in enumerate(blk["hc"]):
        H += u[:, j, None, None] * np.asarray(hc, dtype=np.complex128)
    return H


def slice_eigs(blk, u: np.ndarray):
    H = slice_hamiltonians(blk, u)
    H = 0.5 * (H + np.conj(np.swapaxes(H, -1, -2)))
    return np.linalg.eigh(H)


def propagators(blk, u: np.ndarray, tau: float) -> np.ndarray:
    """U_k = exp(-i tau H_k), [N, m, m]."""
    w, V = slice_eigs(blk, u)
    ph = np.exp(-1j * tau * w)
    return (V * ph[:, None, :]) @ np.conj(np.swapaxes(V, -1, -2))


def forward_states(U: np.ndarray, psi0: np.ndarray) -> np.ndarray:
    """psi_k for k = 0..N: [N+1, m, c]."""
    out = np.empty((U.shape[0] + 1,) + psi0.shape, dtype=np.complex128)
    out[0] = psi0
    for k in range(U.shape[0]):
        out[k + 1] = U[k] @ out[k]
    return out


def backward_costates(U: np.ndarray, psif: np.ndarray) -> np.ndarray:
    """lam_k for k = 0..N with lam_N = psi_f and lam_{k-1} = U_k^dagger lam_k: [N+1, m, c]."""
    N = U.shape[0]
    out = np.empty((N + 1,) + psif.shape, dtype=np.complex128)
    out[N] = psif
    for k in range(N, 0, -1):
        out[k - 1] = np.conj(U[k - 1].T) @ out[k]
    return out


def final_states(problem, u: np.ndarray, tau: float):
    return [forward_states(propagators(b, u, tau), b["psi0"])[-1] for b in _as_blocks(problem)]


def overlap(problem, u: np.ndarray, tau: float) -> complex:
    """o = sum_b sum_r <psif_br | psi_N,br>."""
    o = 0.0 + 0.0j
    for b, psiN in zip(_as_blocks(problem), final_states(problem, u, tau)):
        o += np.vdot(b["psif"], psiN)
    return complex(o)


def fidelity(problem, u: np.ndarray, tau: float) -> float:
    """F = |<psi_f|psi_N>|^2 (Eq. probability)."""
    return abs(overlap(problem, u, tau)) ** 2


def _dk_phi(mu: np.ndarray) -> np.ndarray:
    """Phi_ab = e^{mu_b} * expm1(mu_a - mu_b)/(mu_a - mu_b), with the limit e^{mu_b} at 0."""
    z = mu[..., :, None] - mu[..., None, :]
    small = np.abs(z) < 1e-300
    zs = np.where(small, 1.0, z)
    phi1 = np.where(small, 1.0, np.expm1(zs) / zs)
    return np.exp(mu)[..., None, :] * phi1


def fidelity_and_grad(problem, u: np.ndarray, tau: float):
    """(F, o, dF/du [N, nc]) with the exact (Daleckii-Krein) slice derivative."""
    blocks = _as_blocks(problem)
    N, nc = u.shape
    per_block = []
    o = 0.0 + 0.0j
    for b in blocks:
        w, V = slice_eigs(b, u)
        mu = -1j * tau * w
        U = (V * np.exp(mu)[:, None, :]) @ np.conj(np.swapaxes(V, -1, -2))
        psi = forward_states(U, b["psi0"])
        lam = backward_costates(U, b["psif"])
        o += np.vdot(b["psif"], psi[-1])
        per_block.append((b, w, V, mu, psi, lam))
    do = np.zeros((N, nc), dtype=np.complex128)
    for b, w, V, mu, psi, lam in per_block:
        Phi = _dk_phi(mu)
        Vh = np.conj(np.swapaxes(V, -1, -2))
        a = Vh @ psi[:-1]          # V_k^dagger psi_{k-1}: [N, m, c]
        l = Vh @ lam[1:]           # V_k^dagger lam_k:     [N, m, c]
        for j, hc in enumerate(b["hc"]):
            E = -1j * tau * np.asarray(hc, dtype=np.complex128)
            Et = Vh @ E @ V        # [N, m, m]
            M = Et * Phi
            do[:, j] += np.einsum("kar,kab,kbr->k", np.conj(l), M, a)
    grad = 2.0 * np.real(np.conj(o) * do)
    return abs(o) ** 2, complex(o), grad


def gradient_first_order(problem, u: np.ndarray, tau: float):
    """dF/du with the paper's first-order slice derivative dU_k/du_kj ~ -i tau Hc_j U_k
    (Eq. propagator_differentiation)."""
    blocks = _as_blocks(problem)
    N, nc = u.shape
    o = 0.0 + 0.0j
    do = np.zeros((N, nc), dtype=np.complex128)
    data = []
    for b in blocks:
        U = propagators(b, u, tau)
        psi = forward_states(U, b["psi0"])
        lam = backward_costates(U, b["psif"])
        o += np.vdot(b["psif"], psi[-1])
        data.append((b, psi, lam))
    for b, psi, lam in data:
        for j, hc in enumerate(b["hc"]):
            E = -1j * tau * np.asarray(hc, dtype=np.complex128)
            # lam_k^dagger (E U_k psi_{k-1}) = lam_k^dagger E psi_k
            do[:, j] += np.einsum("kar,ab,kbr->k", np.conj(lam[1:]), E, psi[1:])
    return 2.0 * np.real(np.conj(o) * do)


def gradient_fd(problem, u: np.ndarray, tau: float, entries, h: float = 1e-6) -> np.ndarray:
    """Central differences (F(u + h e_kj) - F(u - h e_kj)) / 2h at the listed (k, j)."""
    out = []
    for k, j in entries:
        up = u.copy()
        dn = u.copy()
        up[k, j] += h
        dn[k, j] -= h
        out.append((fidelity(problem, up, tau) - fidelity(problem, dn, tau)) / (2 * h))
    return np.array(out)


def adam_update(u, g, m, v, t, step, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam ascent step (Kingma & Ba, 2015) on u with gradient g; t counts from 1.  The paper
    leaves the optimiser to its supplement; this is the library's documented choice besides the
    fixed step.  Returns (u, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return u + step * mh / (np.sqrt(vh) + eps), m, v


def grape_adam(problem, u0: np.ndarray, tau: float, iters: int, step: float, f_target: float = 2.0,
               beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """Adam ascent on F; stops updating once F >= f_target.  Returns (u, [F per iteration], first
    iteration with F >= f_target or -1)."""
    u = np.array(u0, dtype=np.float64, copy=True)
    m = np.zeros_like(u)
    v = np.zeros_like(u)
    hist = []
    reached = -1
    for it in range(iters):
        F, _, g = fidelity_and_grad(problem, u, tau)
        hist.append(F)
        if F >= f_target:
            reached = it
            break
        u, m, v = adam_update(u, g, m, v, it + 1, step, beta1, beta2, eps)
    return u, hist, reached


def grape(problem, u0: np.ndarray, tau: float, iters: int, step: float, f_target: float = 2.0):
    """Fixed-step gradient ascent u <- u + step * dF/du; stops early once F >= f_target.
    Returns (u, [F before each update], iterations run)."""
    u = np.array(u0, dtype=np.float64, copy=True)
    hist = []
    it = 0
    for it in range(iters):
        F, _, g = fidelity_and_grad(problem, u, tau)
        hist.append(F)
        if F >= f_target:
            return u, hist, it
        u = u + step * g
    return u, hist, iters


# ------------------------------------------------------------------------------------------------
# Gate (unitary) objective.  Sec. IV compares two propagators K, K' of the full space by the trace
# fidelity F = |Tr(K^dagger K') / 2^n|^2; as a control objective the target is a gate W and
# K' = U_N ... U_1.  With a symmetric W (one that commutes with the group, e.g. U_sq^{(x)n}, Sec.
# III) both are block diagonal in the adapted basis, every copy of block b carries the same block,
# and the full-space trace is the sum over blocks of mult_b Tr(W_b^dagger U_b).
# ------------------------------------------------------------------------------------------------
def gate_overlap(blocks, W_blocks, mult, u: np.ndarray, tau: float) -> complex:
    """g = sum_b mult_b Tr(W_b^dagger U_bN ... U_b1) / d with d = sum_b mult_b m_b; the plain product
    of the propagators, block by block."""
    d = sum(c * np.asarray(W).shape[0] for W, c in zip(W_blocks, mult))
    g = 0.0 + 0.0j
    for blk, W, c in zip(blocks, W_blocks, mult):
        K = np.eye(np.asarray(W).shape[0], dtype=np.complex128)
        for U in propagators(blk, u, tau):
            K = U @ K
        g += c * np.trace(np.conj(np.asarray(W, dtype=np.complex128)).T @ K)
    return complex(g / d)


def gate_fidelity(blocks, W_blocks, mult, u: np.ndarray, tau: float) -> float:
    """F = |Tr(W^dagger U) / d|^2 (the trace fidelity of Sec. IV with the gate as the target)."""
    return abs(gate_overlap(blocks, W_blocks, mult, u, tau)) ** 2


def gate_problem(blocks, W_blocks, mult):
    """The gate objective as a state-transfer problem: in block b the identity columns, weighted by
    sqrt(mult_b / d), are carried to the target's columns W_b e_r with the same weight, so that
    sum_b sum_r <psif_br|psi_N,br> = sum_b (mult_b / d) Tr(W_b^dagger U_b) = g.  The exact gradient
    of F then follows from fidelity_and_grad's costate formula with m columns per block."""
    d = sum(c * np.asarray(W).shape[0] for W, c in zip(W_blocks, mult))
    out = []
    for blk, W, c in zip(blocks, W_blocks, mult):
        W = np.asarray(W, dtype=np.complex128)
        s = np.sqrt(c / d)
        out.append(dict(h0=blk["h0"], hc=blk["hc"], psi0=s * np.eye(W.shape[0], dtype=np.complex128), psif=s * W))
    return out


def gate_fidelity_and_grad(blocks, W_blocks, mult, u: np.ndarray, tau: float):
    """(F, g, dF/du [N, nc]) of the gate objective with the exact slice derivative."""
    return fidelity_and_grad(gate_problem(blocks, W_blocks, mult), u, tau)
