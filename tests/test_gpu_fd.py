"""The GPU gradient (FP64 plans, exact slice derivative; Eq. propagator_differentiation and Appendix B)
against central finite differences of the GPU's own fidelity F = |<psi_f|psi_N>|^2 (Eq. probability):
h = 1e-6 on 20 seeded (k, j) entries, relative error <= 1e-6 (the FD rounding floor is about
1e-16 / h = 1e-10 absolute)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2309_05884_gb300 import api  # noqa: E402
from paper_2309_05884_gb300 import inputs as I  # noqa: E402

DEV = torch.device("cuda", 0)
H_FD = 1e-6
N_ENTRIES = 20
FD_SEED = 3


def _fd_check(plan, u, b0, bf):
    d0, df = api.to_device(b0, DEV), api.to_device(bf, DEV)
    ut = torch.from_numpy(u).to(DEV)
    out, g = plan.fidelity_and_grad(ut, d0, df)
    torch.cuda.synchronize()
    plan.sync_status()
    g = g.cpu().numpy()
    N, nc = u.shape
    picks = I.fd_entries(FD_SEED, N, nc, N_ENTRIES)
    fd = np.empty(len(picks))
    for i, (k, j) in enumerate(picks):
        vals = []
        for sgn in (1.0, -1.0):
            up = u.copy()
            up[k, j] += sgn * H_FD
            o, _ = plan.fidelity_and_grad(torch.from_numpy(up).to(DEV), d0, df, want_grad=False)
            torch.cuda.synchronize()
            vals.append(o[0].item())
        fd[i] = (vals[0] - vals[1]) / (2 * H_FD)
    sel = np.array([g[k, j] for k, j in picks])
    assert np.abs(sel).max() > 1e-3  # a gradient well above the FD rounding floor
    rel = np.linalg.norm(fd - sel) / np.linalg.norm(sel)
    assert rel <= 1e-6, rel
    return out[0].item()


@pytest.mark.parametrize("ckpt", [0, -1])
def test_d8_all_blocks_gradient_matches_central_differences(ckpt):
    # D_8 XXZ ring, every irrep block active: psi_0 = psi_f = a seeded random full-space state, so
    # F (the return probability) is O(0.1) and the gradient is far above the FD floor
    s = I.xxz_ring(8, 4.0, 60)
    B = api.Basis(s)
    x = B.state_to_blocks(I.random_state(2, 2 ** s.n))
    plan = api.Plan(B, s.N, s.tau, prec="f64", ckpt_segment=ckpt)
    F = _fd_check(plan, I.pulses_normal(2, s.N, s.n_ctrl), x, x)
    assert 0.0 < F <= 1.0


def test_d12_first_block_gradient_matches_central_differences():
    # D_12 XXZ ring, first block A1 (224 states, two 128-row tiles), tau = 0.02 as in the D_n
    # workloads: |0...0> -> |0...0> in FP64 (FP64 runs on the CUDA cores at a small fraction of the
    # FP32 rate, which keeps the FD check off the 687-state D_14 block; the FP32 path is checked
    # against the oracle there)
    s = I.xxz_ring(12, 0.4, 20)
    B = api.Basis(s, first_block_only=True)
    assert B.blocks[0][1] == 224
    b0 = B.state_to_blocks(I.basis_state(12, 0))
    plan = api.Plan(B, s.N, s.tau, prec="f64")
    F = _fd_check(plan, I.pulses_normal(2, s.N, s.n_ctrl), b0, b0)
    assert 0.0 < F <= 1.0
