"""Tensor-core (tcgen05) complex products at about FP32 accuracy, against numpy complex128."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2309_05884_gb300 import _lib  # noqa: E402

DEV = torch.device("cuda", 0)


def tc_products(A, B):
    lib = _lib.load()
    count, m, _ = A.shape
    a = torch.from_numpy(A.astype(np.complex64)).to(DEV)
    b = torch.from_numpy(B.astype(np.complex64)).to(DEV)
    c = torch.zeros_like(a)
    st = torch.zeros(1, dtype=torch.int32, device=DEV)
    rc = lib.qoc_tc_cgemm(C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), C.c_void_p(c.data_ptr()), m, count,
                          C.c_void_p(st.data_ptr()), None)
    assert rc == 0, lib.qoc_last_error()
    torch.cuda.synchronize()
    assert st.item() == 0
    return c.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("m", [1, 9, 16, 30, 64, 78, 105, 112])
def test_tc_complex_products_match_fp64(m):
    rng = np.random.default_rng(m)
    A = (rng.normal(size=(5, m, m)) + 1j * rng.normal(size=(5, m, m))) / np.sqrt(m)
    B = (rng.normal(size=(5, m, m)) + 1j * rng.normal(size=(5, m, m))) / np.sqrt(m)
    A = A.astype(np.complex64).astype(np.complex128)
    B = B.astype(np.complex64).astype(np.complex128)
    Cg = tc_products(A, B)
    Cr = A @ B
    err = np.abs(Cg - Cr).max() / np.abs(Cr).max()
    assert err < 1e-5, err


def test_tc_products_of_wide_dynamic_range():
    # entries spanning 1e-4 .. 10 (as in powers of a scaled Hamiltonian): error relative to the norms
    rng = np.random.default_rng(3)
    m = 64
    scale = np.exp(rng.uniform(np.log(1e-4), np.log(10.0), size=(2, m, m)))
    A = (scale[0] * (rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m))))[None]
    B = (scale[1] * (rng.normal(size=(m, m)) + 1j * rng.normal(size=(m, m))))[None]
    A = A.astype(np.complex64).astype(np.complex128)
    B = B.astype(np.complex64).astype(np.complex128)
    Cg = tc_products(A, B)
    Cr = A @ B
    bound = np.abs(A[0]) @ np.abs(B[0])
    assert (np.abs(Cg[0] - Cr[0]) / bound).max() < 4e-6


@pytest.mark.parametrize("prec", ["f32", "f32_all"])
def test_tensor_core_expm_matches_tiled_and_oracle(prec):
    from oracle import grape as gr
    from oracle import operators as op
    from oracle import symmetry as sy
    from paper_2309_05884_gb300 import api
    from paper_2309_05884_gb300 import inputs as I
    s = I.xxz_ring(10, 4.0, 100)   # blocks of 30..105
    psi0, psif = I.random_state(301, 1024), I.random_state(302, 1024)
    B = api.Basis(s)
    b0, bf = B.state_to_blocks(psi0), B.state_to_blocks(psif)
    plan = api.Plan(B, s.N, s.tau, prec=prec, active=B.active_copies(b0, bf))
    u = torch.from_numpy(I.pulses_normal(9, s.N, 3)).to(DEV)
    d0, df = api.to_device(b0, DEV), api.to_device(bf, DEV)
    plan.set_expm_rules([(1 << 30, 0, 0)])
    o_t, g_t = plan.fidelity_and_grad(u, d0, df)
    plan.set_expm_rules([(112, 2, 0)])
    assert all(c[0] == 2 for c in plan.expm_classes())
    o_c, g_c = plan.fidelity_and_grad(u, d0, df)
    torch.cuda.synchronize()
    plan.sync_status()
    H0, Hc = op.system_operators(s)
    F, _, gref = gr.fidelity_and_grad(sy.block_problem(s, H0, Hc, sy.symmetry_blocks(s), psi0, psif),
                                      u.cpu().numpy(), s.tau)
    assert abs(o_c[0].item() - F) <= 1e-5
    gc = g_c.cpu().numpy()
    assert np.linalg.norm(gc - gref) / np.linalg.norm(gref) <= 1e-5
    assert np.linalg.norm(gc - g_t.cpu().numpy()) / np.linalg.norm(gref) <= 1e-5


def _propagator_errors(system, prec, u, tc_param=1):
    """Max |U - U_oracle| over every slice and block, for the tensor-core rule (tc_param 1: every
    slice on the tensor cores; 0: the slices without squarings) and the tiled kernel.  The oracle
    exponentiates the basis builder's block Hamiltonians by eigendecomposition in FP64."""
    from oracle import grape as gr
    from paper_2309_05884_gb300 import api
    B = api.Basis(system)
    plan = api.Plan(B, system.N, system.tau, prec=prec)
    ut = torch.from_numpy(np.ascontiguousarray(u)).to(DEV)
    plan.set_expm_rules([(1 << 30, 0, 0)])
    U_t = plan.expm(ut).cpu().numpy()
    plan.set_expm_rules([(112, 2, tc_param)])
    assert all(c[0] == 2 and c[1] == tc_param for c in plan.expm_classes())
    U_c = plan.expm(ut).cpu().numpy()
    torch.cuda.synchronize()
    plan.sync_status()
    off, e_c, e_t = 0, 0.0, 0.0
    for b in plan.active_blocks():
        m = B.blocks[b][1]
        h0, hc = B.block_matrices(b)
        Uref = gr.propagators(dict(h0=h0, hc=list(hc)), u, system.tau)
        n = system.N * m * m
        e_c = max(e_c, np.abs(U_c[off:off + n].reshape(system.N, m, m) - Uref).max())
        e_t = max(e_t, np.abs(U_t[off:off + n].reshape(system.N, m, m) - Uref).max())
        off += n
    return e_c, e_t


@pytest.mark.parametrize("case", ["tiny_norm", "moderate", "squarings_tc", "squarings_fp64", "small_blocks",
                                  "mid_blocks"])
def test_tensor_core_propagators_match_oracle(case):
    # tiny_norm: degree 1 (no product); moderate: Horner in X^2 only; squarings_tc: |tau H| ~ 50 with
    # the squarings on the tensor cores (FP32 plan); squarings_fp64: the same norms with the FP64
    # squaring chain; small/mid blocks: several CTAs per SM (operand sizes 16..48)
    from paper_2309_05884_gb300 import inputs as I
    if case == "tiny_norm":
        s, prec, tol = I.xxz_ring(8, 4e-5, 4), "f32", 2e-6
    elif case == "moderate":
        s, prec, tol = I.xxz_ring(10, 0.5, 10), "f32", 1e-5
    elif case == "squarings_tc":
        s, prec, tol = I.xxz_ring(8, 20.0, 5), "f32_all", 2e-4
    elif case == "squarings_fp64":
        s, prec, tol = I.xxz_ring(8, 20.0, 5), "f32", 2e-5
    elif case == "small_blocks":
        s, prec, tol = I.sn_allpairs(12, 1.0, 0.5, 3.0, 12), "f32_all", 2e-5
    else:
        s, prec, tol = I.xxz_ring(8, 2.0, 12), "f32_all", 2e-5
    u = I.pulses_normal(17, s.N, s.n_ctrl) if s.n_ctrl == 3 else I.pulses_uniform(17, s.N, s.n_ctrl)
    e_c, e_t = _propagator_errors(s, prec, u)
    assert e_c <= tol, (e_c, e_t)
    # and close to the FP32 CUDA-core kernel on the same slices (two FP16 halves per operand, all four
    # split products: a product errs up to about 2x an FP32 one, more through many squarings)
    assert e_c <= max(8 * e_t, tol / 4), (e_c, e_t)


@pytest.mark.parametrize("prec", ["f32", "f32_all"])
def test_tensor_core_rule_keeps_squared_slices_on_cuda_cores(prec):
    # |tau H| ~ 50: every slice needs squarings, so the default tensor-core rule (param 0) leaves them
    # all to the tiled kernel and the result has its accuracy
    from paper_2309_05884_gb300 import inputs as I
    s = I.xxz_ring(8, 20.0, 5)
    u = I.pulses_normal(17, s.N, 3)
    e_c, e_t = _propagator_errors(s, prec, u, tc_param=0)
    assert e_c <= 1.0001 * e_t + 1e-12, (e_c, e_t)


def test_tensor_core_expm_in_checkpoint_windows():
    # the windowed launches (slice windows of one problem) give the gradient of the whole-problem launch
    from paper_2309_05884_gb300 import api
    from paper_2309_05884_gb300 import inputs as I
    s = I.xxz_ring(8, 4.0, 40)
    psi0, psif = I.random_state(311, 256), I.random_state(312, 256)
    B = api.Basis(s)
    b0, bf = B.state_to_blocks(psi0), B.state_to_blocks(psif)
    act = B.active_copies(b0, bf)
    d0, df = api.to_device(b0, DEV), api.to_device(bf, DEV)
    u = torch.from_numpy(I.pulses_normal(19, s.N, 3)).to(DEV)
    res = []
    for seg in (0, 7):
        plan = api.Plan(B, s.N, s.tau, prec="f32_all", active=act, ckpt_segment=seg)
        plan.set_expm_rules([(112, 2, 0)])
        o, g = plan.fidelity_and_grad(u, d0, df)
        torch.cuda.synchronize()
        plan.sync_status()
        res.append((o.cpu().numpy(), g.cpu().numpy()))
    assert abs(res[0][0][0] - res[1][0][0]) <= 1e-12
    assert np.abs(res[0][1] - res[1][1]).max() <= 1e-12 * max(1.0, np.abs(res[0][1]).max())


@pytest.mark.parametrize("T", [0.12, 0.003, 0.6])
def test_large_block_tensor_core_propagators_match_oracle(T):
    # D_12 blocks of 128..346 states (one to three 128-row tiles, ragged tails), 6 slices of tau = T / 6
    # (0.02: Taylor degree 9-11; 0.0005: degree 3, no Y^2; 0.1: degree 13-15 or squarings): the tiled
    # tensor-core GEMMs (rule kind 3) against the FP64 oracle and the CUDA-core tiles
    from oracle import grape as gr
    from paper_2309_05884_gb300 import api
    from paper_2309_05884_gb300 import inputs as I
    s = I.xxz_ring(12, T, 6)
    B = api.Basis(s)
    u = I.pulses_normal(29, s.N, 3)
    plan = api.Plan(B, s.N, s.tau, prec="f32")
    ut = torch.from_numpy(u).to(DEV)
    plan.set_expm_rules([(1 << 30, 0, 0)])
    U_t = plan.expm(ut).cpu().numpy()
    plan.set_expm_rules([(2048, 3, 0)])
    assert all(c[0] == 3 for c in plan.expm_classes())
    U_c = plan.expm(ut).cpu().numpy()
    torch.cuda.synchronize()
    plan.sync_status()
    off, e_c, e_t = 0, 0.0, 0.0
    for b in plan.active_blocks():
        m = B.blocks[b][1]
        h0, hc = B.block_matrices(b)
        Uref = gr.propagators(dict(h0=h0, hc=list(hc)), u, s.tau)
        n = s.N * m * m
        e_c = max(e_c, np.abs(U_c[off:off + n].reshape(s.N, m, m) - Uref).max())
        e_t = max(e_t, np.abs(U_t[off:off + n].reshape(s.N, m, m) - Uref).max())
        off += n
    assert e_c <= 2e-5, (e_c, e_t)
    assert e_c <= max(8 * e_t, 5e-6), (e_c, e_t)


@pytest.mark.slow
def test_large_block_tensor_core_gradient_d14_first_block():
    # D_14 A1 (687 states), checkpointed FP32 gradient with the tiled tensor-core expm against the
    # same plan on the CUDA-core tiles (the CUDA-core path itself is checked against the oracle in
    # test_gpu_checkpoint)
    from paper_2309_05884_gb300 import api
    from paper_2309_05884_gb300 import inputs as I
    s = I.xxz_ring(14, 4.0, 200)
    B = api.Basis(s, first_block_only=True)
    x = I.random_state(203, 2 ** 14)
    blk = B.state_to_blocks(x)
    blk[687:] = 0
    blk /= np.linalg.norm(blk)
    b0 = B.state_to_blocks(I.basis_state(14, 0))
    u = torch.from_numpy(I.pulses_normal(2, s.N, 3)).to(DEV)
    d0, df = api.to_device(b0, DEV), api.to_device(blk, DEV)
    res = []
    for rules in ([(1 << 30, 0, 0)], [(2048, 3, 0)]):
        plan = api.Plan(B, s.N, s.tau, prec="f32", ckpt_segment=-1)
        plan.set_expm_rules(rules)
        o, g = plan.fidelity_and_grad(u, d0, df)
        torch.cuda.synchronize()
        plan.sync_status()
        res.append((o.cpu().numpy(), g.cpu().numpy()))
    (o_t, g_t), (o_c, g_c) = res
    assert abs(o_c[0] - o_t[0]) <= 1e-5
    assert np.linalg.norm(g_c - g_t) / np.linalg.norm(g_t) <= 1e-5
