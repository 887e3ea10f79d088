"""The gate (unitary) objective on the GPU: F = |Tr(W^dagger U_N ... U_1) / d|^2, the trace fidelity of
Sec. IV with a symmetric target gate (Sec. III), every column of every block propagated.

Against the oracle's gate objective (its own adapted basis, plain products of eigendecomposition
propagators, exact gradient) within 1e-10 (FP64) and 1e-5 (FP32) on F and the relative gradient
error, with every D_n block taking part; the sigma_x^{(x)n} closed form (u T = pi/2 under sum X:
F = 1, zero gradient); GRAPE on the gate objective follows the oracle's trajectory.
"""
import numpy as np
import pytest

from oracle import grape as gr
from oracle import operators as op
from oracle import symmetry as sy
from paper_2309_05884_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2309_05884_gb300 import _lib, api  # noqa: E402

DEV = torch.device("cuda", 0)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Hd = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2)


def tensor_power(a, n):
    out = np.ones((1, 1), dtype=np.complex128)
    for _ in range(n):
        out = np.kron(out, a)
    return out


def oracle_gate(s, W_full, u):
    """The oracle's blocks of H0, Hc_j and W (its own basis), then its gate objective."""
    H0, Hc = op.system_operators(s)
    blocks = sy.symmetry_blocks(s)
    blks = [dict(h0=sy.block_operator(V[0], H0), hc=[sy.block_operator(V[0], h) for h in Hc]) for _, V in blocks]
    Ws = [sy.block_operator(V[0], W_full) for _, V in blocks]
    mult = [V.shape[0] for _, V in blocks]
    return gr.gate_fidelity_and_grad(blks, Ws, mult, u, s.tau), (blks, Ws, mult)


def gpu_gate(s, W_full, prec, **kw):
    B = api.Basis(s)
    plan = api.Plan(B, s.N, s.tau, prec=prec, objective="gate", **kw)
    p0, pf = plan.gate_states(B.gate_blocks(W_full))
    assert plan.state_len == sum(m * m for _, m, _, _ in B.blocks)
    return B, plan, api.to_device(p0, DEV), api.to_device(pf, DEV)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-10), ("f32", 1e-5)])
@pytest.mark.parametrize("gate", ["hadamard", "xpow"])
def test_gate_objective_matches_oracle_all_blocks(prec, tol, gate):
    s = I.xxz_ring(8, 2.0, 30)
    W = tensor_power(Hd if gate == "hadamard" else X, s.n)
    u = I.pulses_normal(5, s.N, s.n_ctrl)
    (F, g_o, gref), _ = oracle_gate(s, W, u)
    B, plan, d0, df = gpu_gate(s, W, prec)
    assert len(plan.active_blocks()) == B.n_blocks  # every block takes part
    out3, g = plan.fidelity_and_grad(torch.from_numpy(u).to(DEV), d0, df)
    torch.cuda.synchronize()
    plan.sync_status()
    o = out3.cpu().numpy()
    assert abs(o[0] - F) <= tol
    assert abs((o[1] + 1j * o[2]) - g_o) <= tol
    assert rel(g.cpu().numpy(), gref) <= tol


@pytest.mark.parametrize("n", [4, 6, 8])
def test_sigma_x_power_closed_form(n):
    # H = u sum X, u T = pi/2: U = (-i)^n X^{(x)n}, so F = 1 for W = X^{(x)n} and dF/du = 0 (a maximum)
    T, N = 2.0, 16
    s = I.System(n, I.GROUP_DN, [(I.RING_ZZ, 0.0, 1)], [[(I.SUM_X, 1.0, 0)], [(I.SUM_Y, 1.0, 0)]], T, N)
    u = np.zeros((N, 2))
    u[:, 0] = np.pi / (2 * T)
    B, plan, d0, df = gpu_gate(s, tensor_power(X, n), "f64")
    out3, g = plan.fidelity_and_grad(torch.from_numpy(u).to(DEV), d0, df)
    torch.cuda.synchronize()
    plan.sync_status()
    o = out3.cpu().numpy()
    assert abs(o[0] - 1.0) <= 1e-12
    assert abs((o[1] + 1j * o[2]) - (-1j) ** n) <= 1e-12
    assert np.abs(g.cpu().numpy()).max() <= 1e-10


def test_gate_grape_follows_oracle():
    s = I.xxz_ring(6, 1.5, 20)
    W = tensor_power(Hd, s.n)
    u0 = I.pulses_normal(7, s.N, s.n_ctrl)
    _, (blks, Ws, mult) = oracle_gate(s, W, u0)
    prob = gr.gate_problem(blks, Ws, mult)
    iters, step = 15, 0.3
    u_ref, hist = u0.copy(), []
    for _ in range(iters):
        F, _, g = gr.fidelity_and_grad(prob, u_ref, s.tau)
        hist.append(F)
        u_ref = u_ref + step * g
    B, plan, d0, df = gpu_gate(s, W, "f64")
    ut = torch.from_numpy(u0.copy()).to(DEV)
    Fh, done, _ = plan.optimize(ut, d0, df, iters=iters, step=step)
    torch.cuda.synchronize()
    assert done == iters
    assert np.abs(Fh.cpu().numpy() - np.array(hist)).max() <= 1e-10
    assert np.abs(ut.cpu().numpy() - u_ref).max() <= 1e-9
    assert hist[-1] > hist[0]


def test_gate_plan_rejects_active_mask():
    s = I.xxz_ring(4, 1.0, 4)
    B = api.Basis(s)
    with pytest.raises(_lib.QocError) as e:
        api.Plan(B, s.N, s.tau, objective="gate", active=np.ones(B.n_copies, np.uint8))
    assert e.value.code == _lib.QOC_EINVAL


def test_gate_blocks_reject_asymmetric_gate():
    s = I.xxz_ring(4, 1.0, 4)
    B = api.Basis(s)
    W = np.kron(X, np.eye(8))  # acts on qubit 1 only: not D_4-symmetric
    with pytest.raises(ValueError):
        B.gate_blocks(W)
