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
