"""Forward/backward sweeps split over thread-block clusters, against the one-CTA-per-chain kernel and
the FP64 oracle (Sec. II.A propagation; costates through U_k^dagger, Appendix B)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import grape as gr  # noqa: E402
from oracle import operators as op  # noqa: E402
from oracle import symmetry as sy  # noqa: E402
from paper_2309_05884_gb300 import api  # noqa: E402
from paper_2309_05884_gb300 import inputs as I  # noqa: E402

DEV = torch.device("cuda", 0)
TOL = {"f64": 1e-10, "f32": 1e-5}


def _setup(s, seed, prec, seg=0):
    dim = 2 ** s.n
    psi0, psif = I.random_state(seed, dim), I.random_state(seed + 1, dim)
    B = api.Basis(s)
    b0, bf = B.state_to_blocks(psi0), B.state_to_blocks(psif)
    plan = api.Plan(B, s.N, s.tau, prec=prec, active=B.active_copies(b0, bf), ckpt_segment=seg)
    return psi0, psif, B, plan, api.to_device(b0, DEV), api.to_device(bf, DEV)


def _fg(plan, u, d0, df):
    o, g = plan.fidelity_and_grad(u, d0, df)
    torch.cuda.synchronize()
    plan.sync_status()
    return o.cpu().numpy(), g.cpu().numpy()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("cl", [2, 4, 8])
def test_cluster_sweeps_match_oracle(prec, cl):
    s = I.xxz_ring(8, 3.0, 40)  # blocks of 6..33 states
    psi0, psif, B, plan, d0, df = _setup(s, 401, prec)
    u = torch.from_numpy(I.pulses_normal(23, s.N, 3)).to(DEV)
    plan.set_sweep_cluster(0)
    o_1, g_1 = _fg(plan, u, d0, df)
    plan.set_sweep_cluster(cl)
    assert plan.sweep_cluster() == cl
    o_c, g_c = _fg(plan, u, d0, df)
    H0, Hc = op.system_operators(s)
    F, _, gref = gr.fidelity_and_grad(sy.block_problem(s, H0, Hc, sy.symmetry_blocks(s), psi0, psif),
                                      u.cpu().numpy(), s.tau)
    tol = TOL[prec]
    assert abs(o_c[0] - F) <= tol
    assert np.linalg.norm(g_c - gref) / np.linalg.norm(gref) <= tol
    assert abs(o_c[0] - o_1[0]) <= tol
    # the final state, element by element, against the full 2^n evolution
    psiN = plan.propagate(u, d0)
    torch.cuda.synchronize()
    full = B.blocks_to_state(psiN.cpu().numpy())
    ref = gr.final_states([dict(h0=H0.toarray(), hc=[h.toarray() for h in Hc], psi0=psi0[:, None],
                                psif=psi0[:, None])], u.cpu().numpy(), s.tau)[0][:, 0]
    assert np.abs(full - ref).max() <= (1e-11 if prec == "f64" else 2e-5)


def test_cluster_sweeps_in_checkpoint_windows():
    s = I.xxz_ring(8, 3.0, 45)
    psi0, psif, B, plan, d0, df = _setup(s, 405, "f64", seg=7)
    u = torch.from_numpy(I.pulses_normal(29, s.N, 3)).to(DEV)
    plan.set_sweep_cluster(4)
    o_w, g_w = _fg(plan, u, d0, df)
    _, _, _, whole, d0b, dfb = _setup(s, 405, "f64")
    whole.set_sweep_cluster(0)
    o_1, g_1 = _fg(whole, u, d0b, dfb)
    assert abs(o_w[0] - o_1[0]) <= 1e-12
    assert np.abs(g_w - g_1).max() <= 1e-12 * max(1.0, np.abs(g_1).max())


def test_cluster_size_rejections():
    s = I.xxz_ring(8, 3.0, 10)
    _, _, _, plan, _, _ = _setup(s, 409, "f32")
    for bad in (1, 9, -2):
        with pytest.raises(Exception):
            plan.set_sweep_cluster(bad)
    plan.set_sweep_cluster(3)
    assert plan.sweep_cluster() == 3
    plan.set_sweep_cluster(-1)
    assert plan.sweep_cluster() in (0, 2, 3, 4, 5, 6, 7, 8)


@pytest.mark.parametrize("prec,cl", [("f64", 3), ("f64", 8), ("f32", 5), ("f32", 8)])
def test_cluster_sweeps_stream_large_blocks_in_row_subblocks(prec, cl):
    # D_12 blocks of up to 346 states: a CTA's rows of U_k exceed the 8-slot ring, so they pass
    # through 4 slots in sub-blocks (ragged last one); states against the oracle's per-block
    # propagation, F and dF/du against the one-CTA-per-chain kernel
    s = I.xxz_ring(12, 2.0, 8)
    dim = 2 ** s.n
    B = api.Basis(s)
    b0 = B.state_to_blocks(I.random_state(411, dim))
    bf = B.state_to_blocks(I.random_state(412, dim))
    plan = api.Plan(B, s.N, s.tau, prec=prec)
    d0, df = api.to_device(b0, DEV), api.to_device(bf, DEV)
    un = I.pulses_normal(31, s.N, 3)
    u = torch.from_numpy(un).to(DEV)
    plan.set_sweep_cluster(0)
    o_1, g_1 = _fg(plan, u, d0, df)
    plan.set_sweep_cluster(cl)
    o_c, g_c = _fg(plan, u, d0, df)
    psiN = plan.propagate(u, d0)
    torch.cuda.synchronize()
    psiN = psiN.cpu().numpy()
    ov, err = 0.0 + 0.0j, 0.0
    for b, (_, m, c, off) in enumerate(B.blocks):
        h0, hc = B.block_matrices(b)
        x0 = b0[off:off + c * m].reshape(c, m).T
        ref = gr.forward_states(gr.propagators(dict(h0=h0, hc=list(hc)), un, s.tau), x0)[-1]
        got = psiN[off:off + c * m].reshape(c, m).T
        err = max(err, np.abs(got - ref).max())
        ov += np.vdot(bf[off:off + c * m].reshape(c, m).T, ref)
    tol = TOL[prec]
    assert err <= (1e-11 if prec == "f64" else 2e-5)
    assert abs(o_c[0] - abs(ov) ** 2) <= tol
    assert abs(o_c[0] - o_1[0]) <= (1e-13 if prec == "f64" else 1e-6)
    assert np.linalg.norm(g_c - g_1) / np.linalg.norm(g_1) <= (1e-12 if prec == "f64" else 1e-5)
