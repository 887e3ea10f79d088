"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on identical seeded inputs.

Tolerances: FP64 path 1e-10 on F and on the relative gradient error ||g - g_ref|| / ||g_ref||;
FP32 path (complex FP32 polynomial and sweeps, FP64 squaring and accumulation) 1e-5.
Gauge: the library's block basis and the oracle's differ by block-internal rotations, so states
are compared in the full space and propagators through their spectra."""
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

from paper_2309_05884_gb300 import api  # noqa: E402

DEV = torch.device("cuda", 0)
TOL64 = 1e-10
TOL32 = 1e-5


def a1_target(system, seed):
    """Normalised projection of a seeded random state onto the trivial irrep (A1 / J=n/2) block,
    computed by each side in its own basis (the projection itself is basis independent)."""
    x = I.random_state(seed, 2 ** system.n)
    ob = sy.symmetry_blocks(system)
    coords = sy.to_blocks(ob, x)
    coords = [c if i == 0 else np.zeros_like(c) for i, c in enumerate(coords)]
    full = sy.from_blocks(ob, coords)
    return x, full / np.linalg.norm(full)


def gpu_side(system, psi0_full, psif_full, prec, grad_mode=0, blk_f=None):
    B = api.Basis(system)
    b0 = B.state_to_blocks(psi0_full)
    bf = B.state_to_blocks(psif_full) if blk_f is None else blk_f
    plan = api.Plan(B, system.N, system.tau, prec=prec, grad_mode=grad_mode, active=B.active_copies(b0, bf))
    return B, plan, api.to_device(b0, DEV), api.to_device(bf, DEV)


def run(plan, u, d0, df):
    ut = torch.from_numpy(np.ascontiguousarray(u)).to(DEV)
    out3, g = plan.fidelity_and_grad(ut, d0, df)
    torch.cuda.synchronize()
    plan.sync_status()
    o = out3.cpu().numpy()
    return o[0], o[1] + 1j * o[2], g.cpu().numpy()


def oracle_side(system, psi0_full, psif_full, u, mode="exact"):
    H0, Hc = op.system_operators(system)
    prob = sy.block_problem(system, H0, Hc, sy.symmetry_blocks(system), psi0_full, psif_full)
    F, o, g = gr.fidelity_and_grad(prob, u, system.tau)
    if mode == "first":
        g = gr.gradient_first_order(prob, u, system.tau)
    return F, o, g


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def check(system, psi0, psif, u, prec, tol, grad_mode=0, blk_f=None):
    _, plan, d0, df = gpu_side(system, psi0, psif, prec, grad_mode, blk_f)
    F, o, g = run(plan, u, d0, df)
    Fr, orf, gr_ = oracle_side(system, psi0, psif, u, "first" if grad_mode else "exact")
    assert abs(F - Fr) <= tol, (F, Fr)
    assert abs(o - orf) <= tol * max(1.0, abs(orf)) * 10, (o, orf)
    assert rel(g, gr_) <= tol, rel(g, gr_)
    assert np.abs(g - gr_).max() <= tol * np.abs(gr_).max() * 10
    return F, g


# ------------------------------------------------------------------------------------------ FP64
def test_c1_fp64_dicke_target():
    s = I.c1_system()
    check(s, I.basis_state(4, 0), op.dicke_state(4, 2), I.pulses_uniform(0, s.N, 2), "f64", TOL64)


def test_c1_fp64_all_blocks():
    s = I.c1_system()
    check(s, I.random_state(30, 16), I.random_state(31, 16), I.pulses_uniform(0, s.N, 2), "f64", TOL64)


@pytest.mark.parametrize("n,N,T", [(5, 30, 3.0), (6, 40, 4.0), (8, 20, 1.0)])
def test_dn_ring_fp64_all_blocks(n, N, T):
    s = I.xxz_ring(n, T, N)
    dim = 2 ** n
    check(s, I.random_state(40 + n, dim), I.random_state(50 + n, dim), I.pulses_normal(n, N, 3), "f64", TOL64)


def test_dn10_fp64_multi_tile_blocks():
    # blocks of 30..105 exceed one 64x64 FP64 tile: exercises the tiled GEMM's ragged edges
    s = I.xxz_ring(10, 0.4, 10)
    check(s, I.random_state(60, 1024), I.random_state(61, 1024), I.pulses_normal(1, 10, 3), "f64", TOL64)


def test_first_order_mode_fp64():
    s = I.c1_system()
    check(s, I.basis_state(4, 0), op.dicke_state(4, 2), I.pulses_uniform(0, s.N, 2), "f64", TOL64, grad_mode=1)


def test_single_slice_and_size_one_block():
    # N = 1 and the 1x1 J=0 blocks of S_4
    s = I.System(4, I.GROUP_SN, I.c1_system().h0, I.c1_system().hc, 0.3, 1)
    check(s, I.random_state(70, 16), I.random_state(71, 16), I.pulses_uniform(3, 1, 2), "f64", TOL64)


def test_ising_ring_paper_model_fp64():
    # Eqs. H0WithCoupling / Hc, up^n -> down^n, first D_n block only (Sec. II.B)
    s = I.ising_ring(7, 1.0, 0.8, 5.0, 50)
    check(s, I.basis_state(7, 0), I.basis_state(7, 127), I.pulses_uniform(5, 50, 2), "f64", TOL64)


def test_propagate_fp64_elementwise_full_space():
    s = I.xxz_ring(6, 2.0, 25)
    psi0 = I.random_state(80, 64)
    u = I.pulses_normal(2, s.N, 3)
    B, plan, d0, _ = gpu_side(s, psi0, psi0, "f64")
    psiN = plan.propagate(torch.from_numpy(u).to(DEV), d0)
    torch.cuda.synchronize()
    full_gpu = B.blocks_to_state(psiN.cpu().numpy())
    H0, Hc = op.system_operators(s)
    ref = gr.final_states([dict(h0=H0.toarray(), hc=[h.toarray() for h in Hc], psi0=psi0[:, None],
                                psif=psi0[:, None])], u, s.tau)[0][:, 0]
    assert np.abs(full_gpu - ref).max() <= 1e-11


def test_expm_spectra_and_unitarity_fp64():
    s = I.xxz_ring(6, 2.0, 12)
    psi0 = I.random_state(81, 64)
    u = I.pulses_normal(3, s.N, 3)
    B, plan, _, _ = gpu_side(s, psi0, psi0, "f64")
    ut = torch.from_numpy(u).to(DEV)
    U = plan.expm(ut).cpu().numpy()
    A = plan.assemble(ut).cpu().numpy()
    H0, Hc = op.system_operators(s)
    ob = sy.symmetry_blocks(s)
    off = 0
    for b in plan.active_blocks():
        m = B.blocks[b][1]
        Ub = U[off: off + s.N * m * m].reshape(s.N, m, m)
        Ab = A[off: off + s.N * m * m].reshape(s.N, m, m)
        off += s.N * m * m
        V = ob[b][1][0]
        blk = dict(h0=sy.block_operator(V, H0), hc=[sy.block_operator(V, h) for h in Hc])
        w = np.linalg.eigvalsh(gr.slice_hamiltonians(blk, u))          # [N, m]
        for k in range(s.N):
            assert np.abs(Ub[k].conj().T @ Ub[k] - np.eye(m)).max() < 1e-12
            # eigenphases of U_k are exp(-i tau w); eigenvalues of i A_k / tau are w
            ph = np.sort(np.angle(np.linalg.eigvals(Ub[k])))
            assert np.abs(ph - np.sort(np.angle(np.exp(-1j * s.tau * w[k])))).max() < 1e-10
            wa = np.sort(np.linalg.eigvalsh(0.5 * (1j * Ab[k] / s.tau + (1j * Ab[k] / s.tau).conj().T)))
            assert np.abs(wa - w[k]).max() < 1e-12


def test_large_norm_slices_use_fp64_squaring():
    # |tau H| ~ 40: scaling and squaring with s ~ 4 (propagation only; the gradient series is
    # limited to moderate norms and reports it)
    s = I.sn_allpairs(8, 2.0, 1.0, 10.0, 20)
    psi0 = I.basis_state(8, 0)
    u = I.pulses_uniform(4, s.N, 2)
    B, plan, d0, _ = gpu_side(s, psi0, psi0, "f64")
    psiN = plan.propagate(torch.from_numpy(u).to(DEV), d0)
    torch.cuda.synchronize()
    plan.sync_status()
    full_gpu = B.blocks_to_state(psiN.cpu().numpy())
    ob = sy.symmetry_blocks(s)
    H0, Hc = op.system_operators(s)
    prob = sy.block_problem(s, H0, Hc, ob, psi0, psi0)
    ref = sy.from_blocks(ob, [gr.final_states(prob, u, s.tau)[0]] + [np.zeros((V.shape[1], V.shape[0]))
                                                                     for _, V in ob[1:]])
    assert np.abs(full_gpu - ref).max() <= 1e-10


def test_grape_trajectory_matches_oracle_fp64():
    s = I.c1_system()
    psi0, psif = I.basis_state(4, 0), op.dicke_state(4, 2)
    u0 = I.pulses_uniform(0, s.N, 2)
    _, plan, d0, df = gpu_side(s, psi0, psif, "f64")
    ut = torch.from_numpy(u0.copy()).to(DEV)
    Fh, done, _ = plan.optimize(ut, d0, df, iters=200, step=0.3)
    torch.cuda.synchronize()
    H0, Hc = op.system_operators(s)
    prob = sy.block_problem(s, H0, Hc, sy.symmetry_blocks(s), psi0, psif)
    ur, hr, _ = gr.grape(prob, u0, s.tau, 200, 0.3)
    assert done == 200
    assert np.abs(ut.cpu().numpy() - ur).max() <= 1e-9
    assert np.abs(Fh.cpu().numpy() - np.array(hr)).max() <= 1e-10
    assert hr[-1] > 0.999


def test_autograd_function_fp64():
    s = I.c1_system()
    psi0, psif = I.basis_state(4, 0), op.dicke_state(4, 2)
    u0 = I.pulses_uniform(0, s.N, 2)
    _, plan, d0, df = gpu_side(s, psi0, psif, "f64")
    ut = torch.from_numpy(u0).to(DEV).requires_grad_(True)
    F = api.FidelityGrad.apply(ut, plan, d0, df)
    (3.0 * F).backward()
    Fr, _, gref = oracle_side(s, psi0, psif, u0)
    assert abs(F.item() - Fr) <= TOL64
    assert rel(ut.grad.cpu().numpy(), 3.0 * gref) <= TOL64


def test_nan_pulse_is_reported():
    s = I.c1_system()
    _, plan, d0, df = gpu_side(s, I.basis_state(4, 0), op.dicke_state(4, 2), "f64")
    u = I.pulses_uniform(0, s.N, 2)
    u[7, 1] = np.nan
    plan.fidelity_and_grad(torch.from_numpy(u).to(DEV), d0, df)
    with pytest.raises(RuntimeError, match="non-finite"):
        plan.sync_status()
    plan.sync_status()  # cleared


def test_workspace_too_small_is_rejected():
    from paper_2309_05884_gb300 import _lib
    import ctypes as C
    s = I.c1_system()
    _, plan, d0, df = gpu_side(s, I.basis_state(4, 0), op.dicke_state(4, 2), "f64")
    ut = torch.from_numpy(I.pulses_uniform(0, s.N, 2)).to(DEV)
    out3 = torch.empty(3, dtype=torch.float64, device=DEV)
    ws = plan.workspace
    rc = plan.lib.qoc_fidelity_and_grad(plan.handle, C.c_void_p(ut.data_ptr()), C.c_void_p(d0.data_ptr()),
                                        C.c_void_p(df.data_ptr()), C.c_void_p(out3.data_ptr()), None,
                                        C.c_void_p(ws.data_ptr()), plan.workspace_bytes - 1, None)
    assert rc == _lib.QOC_ENOMEM


# ------------------------------------------------------------------------------------------ FP32
def test_c2_fp32_first_block():
    # the paper's "first block only" setting: |0...0> and an A1 target
    s = I.c2_system()
    _, psif = a1_target(s, 102)
    F, _ = check(s, I.basis_state(10, 0), psif, I.pulses_normal(1, s.N, 3), "f32", TOL32)
    assert F > 0


def test_c2_fp32_all_blocks_full_size():
    s = I.c2_system()
    check(s, I.random_state(101, 1024), I.random_state(102, 1024), I.pulses_normal(1, s.N, 3), "f32", TOL32)


def test_c2_fp32_short_elementwise_states():
    s = I.xxz_ring(10, 2.0, 50)
    psi0 = I.random_state(103, 1024)
    u = I.pulses_normal(7, s.N, 3)
    B, plan, d0, _ = gpu_side(s, psi0, psi0, "f32")
    psiN = plan.propagate(torch.from_numpy(u).to(DEV), d0)
    torch.cuda.synchronize()
    full_gpu = B.blocks_to_state(psiN.cpu().numpy())
    ob = sy.symmetry_blocks(s)
    H0, Hc = op.system_operators(s)
    prob = sy.block_problem(s, H0, Hc, ob, psi0, psi0)
    ref = sy.from_blocks(ob, gr.final_states(prob, u, s.tau))
    assert np.abs(full_gpu - ref).max() <= TOL32


def test_fp32_dn_ragged_sizes():
    # n = 9: blocks of 14..58 (one to four 16-row tiles, ragged tails)
    s = I.xxz_ring(9, 3.0, 60)
    check(s, I.random_state(110, 512), I.random_state(111, 512), I.pulses_normal(9, s.N, 3), "f32", TOL32)


def test_ising_ring_full_coupling_fp64():
    # Eq. H0MoreCoupling1 (every ring distance up to floor(n/2)), |up^n> to a seeded target in the
    # first D_n block (Sec. II.B), and up^n -> down^n
    s = I.ising_ring_full(8, 1.0, [0.8, 0.37, 0.23, 0.11], 6.0, 60)
    _, psif = a1_target(s, 112)
    F, _ = check(s, I.basis_state(8, 0), psif, I.pulses_uniform(6, 60, 2), "f64", TOL64)
    assert F > 1e-3
    check(s, I.basis_state(8, 0), I.basis_state(8, 255), I.pulses_uniform(6, 60, 2), "f64", TOL64)


def test_ising_ring_full_coupling_fp32_all_blocks():
    s = I.ising_ring_full(9, 1.0, [0.8, 0.37, 0.23, 0.11], 2.0, 40)
    check(s, I.random_state(90, 512), I.random_state(91, 512), I.pulses_uniform(7, 40, 2), "f32", TOL32)
