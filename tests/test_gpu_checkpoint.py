"""sqrt(N) checkpointing (keep psi every S slices, recompute each segment's propagators during the
costate pass): results equal the stored-propagator path bit for bit, and the oracle within the
path's tolerance."""
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


def make(system, psi0, psif, prec, seg, first_block=False):
    B = api.Basis(system, first_block_only=first_block)
    b0 = B.state_to_blocks(psi0)
    bf = B.state_to_blocks(psif)
    plan = api.Plan(B, system.N, system.tau, prec=prec, active=B.active_copies(b0, bf), ckpt_segment=seg)
    return B, plan, api.to_device(b0, DEV), api.to_device(bf, DEV)


def eval_(plan, u, d0, df):
    out3, g = plan.fidelity_and_grad(torch.from_numpy(u).to(DEV), d0, df)
    torch.cuda.synchronize()
    plan.sync_status()
    return out3.cpu().numpy(), g.cpu().numpy()


@pytest.mark.parametrize("seg", [-1, 7, 1])
def test_checkpointed_equals_stored_fp64(seg):
    s = I.c1_system()
    psi0, psif = I.random_state(5, 16), I.random_state(6, 16)
    u = I.pulses_uniform(0, s.N, 2)
    _, p0, d0, df = make(s, psi0, psif, "f64", 0)
    _, p1, _, _ = make(s, psi0, psif, "f64", seg)
    assert p1.workspace_bytes < p0.workspace_bytes or seg == 1
    o0, g0 = eval_(p0, u, d0, df)
    o1, g1 = eval_(p1, u, d0, df)
    assert np.array_equal(o0, o1) and np.array_equal(g0, g1)
    H0, Hc = op.system_operators(s)
    F, o, g = gr.fidelity_and_grad(sy.block_problem(s, H0, Hc, sy.symmetry_blocks(s), psi0, psif), u, s.tau)
    assert abs(o1[0] - F) <= 1e-10
    assert np.linalg.norm(g1 - g) / np.linalg.norm(g) <= 1e-10


def test_checkpointed_equals_stored_fp32_c2_full_size():
    s = I.c2_system()
    psi0, psif = I.random_state(101, 1024), I.random_state(102, 1024)
    u = I.pulses_normal(1, s.N, 3)
    _, p0, d0, df = make(s, psi0, psif, "f32", 0)
    _, p1, _, _ = make(s, psi0, psif, "f32", -1)   # S = 23, 22 segments, last one ragged (17 slices)
    # the stored propagators (500 slices x 53 764 complex64 = 215 MB) shrink to one segment's worth
    assert p0.workspace_bytes - p1.workspace_bytes > 0.9 * 500 * 53764 * 8
    o0, g0 = eval_(p0, u, d0, df)
    o1, g1 = eval_(p1, u, d0, df)
    assert np.array_equal(o0, o1) and np.array_equal(g0, g1)


def test_checkpointed_propagate_and_autograd():
    s = I.xxz_ring(8, 2.0, 30)
    psi0, psif = I.random_state(7, 256), I.random_state(8, 256)
    u = I.pulses_normal(2, s.N, 3)
    B, p1, d0, df = make(s, psi0, psif, "f64", 4)
    psiN = p1.propagate(torch.from_numpy(u).to(DEV), d0)
    torch.cuda.synchronize()
    H0, Hc = op.system_operators(s)
    ref = gr.final_states([dict(h0=H0.toarray(), hc=[h.toarray() for h in Hc], psi0=psi0[:, None],
                                psif=psi0[:, None])], u, s.tau)[0][:, 0]
    assert np.abs(B.blocks_to_state(psiN.cpu().numpy()) - ref).max() <= 1e-11
    ut = torch.from_numpy(u).to(DEV).requires_grad_(True)
    F = api.FidelityGrad.apply(ut, p1, d0, df)
    F.backward()
    Fr, _, gref = gr.fidelity_and_grad(sy.block_problem(s, H0, Hc, sy.symmetry_blocks(s), psi0, psif), u, s.tau)
    assert abs(F.item() - Fr) <= 1e-10
    assert np.linalg.norm(ut.grad.cpu().numpy() - gref) / np.linalg.norm(gref) <= 1e-10


@pytest.mark.slow
def test_d14_first_block_checkpointed_fp32():
    # D_14 XXZ ring, first block A1 (687 states), |0...0> -> seeded A1 target, tau = 0.02 as in the
    # T = 40, N = 2000 workload but N = 200 so that the oracle's eigendecompositions stay short
    s = I.xxz_ring(14, 4.0, 200)
    B = api.Basis(s, first_block_only=True)
    assert B.blocks[0][1] == 687
    x = I.random_state(203, 2 ** 14)
    blk = B.state_to_blocks(x)
    blk[687:] = 0
    blk /= np.linalg.norm(blk)
    b0 = B.state_to_blocks(I.basis_state(14, 0))
    u = I.pulses_normal(2, s.N, 3)
    plans = [api.Plan(B, s.N, s.tau, prec="f32", ckpt_segment=seg) for seg in (0, -1)]
    d0, df = api.to_device(b0, DEV), api.to_device(blk, DEV)
    (o0, g0), (o1, g1) = [eval_(p, u, d0, df) for p in plans]
    assert np.array_equal(o0, o1) and np.array_equal(g0, g1)
    # oracle: its own D_14 basis, first block; the target is the same full-space state
    from oracle import symmetry as osy
    psif_full = B.blocks_to_state(blk)
    H0, Hc = op.system_operators(s)
    # A1 of the oracle: orbit sums (one vector per orbit), built from the oracle's own orbits
    orbits = osy.dn_orbits(14)
    V = np.zeros((len(orbits), 2 ** 14))
    for i, orb in enumerate(orbits):
        V[i, orb] = 1.0 / np.sqrt(len(orb))
    prob = [dict(h0=osy.block_operator(V, H0), hc=[osy.block_operator(V, h) for h in Hc],
                 psi0=(V @ I.basis_state(14, 0))[:, None], psif=(V.conj() @ psif_full)[:, None])]
    F, o, g = gr.fidelity_and_grad(prob, u, s.tau)
    assert abs(o1[0] - F) <= 1e-5
    assert np.linalg.norm(g1 - g) / np.linalg.norm(g) <= 1e-5
