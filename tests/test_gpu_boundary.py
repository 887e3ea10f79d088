"""The C ABI's error behaviour and the split adjoint (forward half / backward half) on the GPU.

- Initial and target states must have norm 1 (to 1e-8) per problem: checked on the device, the
  error is latched and returned by qoc_plan_sync_status or by the next call on the plan.
- Latched kernel errors (non-finite pulse, squaring cap, bounded wait) come back from the next call.
- The bounded-wait path: a wait on an mbarrier that nothing completes gives up and reports
  QOC_ETIMEOUT; the context stays usable (the next evaluation still matches the oracle).
- FidelityGrad's forward runs no costate or derivative kernel; its backward does, and scales dF/du
  by dL/dF on the device; the gradient equals qoc_fidelity_and_grad's bit for bit.
"""
import ctypes as C

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


def c1_plan(prec="f64", **kw):
    s = I.c1_system()
    B = api.Basis(s)
    b0 = B.state_to_blocks(I.basis_state(4, 0))
    bf = B.state_to_blocks(op.dicke_state(4, 2))
    plan = api.Plan(B, s.N, s.tau, prec=prec, active=B.active_copies(b0, bf), **kw)
    return s, B, plan, b0, bf


def d8_plan(prec="f32", seg=0):
    s = I.xxz_ring(8, 3.0, 40)
    psi0, psif = I.random_state(401, 256), I.random_state(402, 256)
    B = api.Basis(s)
    b0, bf = B.state_to_blocks(psi0), B.state_to_blocks(psif)
    plan = api.Plan(B, s.N, s.tau, prec=prec, active=B.active_copies(b0, bf), ckpt_segment=seg)
    return s, plan, psi0, psif, api.to_device(b0, DEV), api.to_device(bf, DEV)


def ut_of(u):
    return torch.from_numpy(np.ascontiguousarray(u)).to(DEV)


def code_of(excinfo):
    return excinfo.value.code


@pytest.mark.parametrize("which", ["psi0", "psif"])
def test_unnormalised_state_is_rejected(which):
    s, B, plan, b0, bf = c1_plan()
    u = ut_of(I.pulses_uniform(0, s.N, 2))
    good0, goodf = api.to_device(b0, DEV), api.to_device(bf, DEV)
    plan.fidelity_and_grad(u, good0, goodf)
    plan.sync_status()  # normalised states pass
    bad = (b0 if which == "psi0" else bf) * 1.01
    d0 = api.to_device(bad, DEV) if which == "psi0" else good0
    df = api.to_device(bad, DEV) if which == "psif" else goodf
    plan.fidelity_and_grad(u, d0, df)
    with pytest.raises(_lib.QocError, match="norm") as e:
        plan.sync_status()
    assert code_of(e) == _lib.QOC_EINVAL
    plan.sync_status()  # cleared
    # a deviation inside the 1e-8 tolerance is accepted
    plan.fidelity_and_grad(u, api.to_device(b0 * (1 + 2e-9), DEV), goodf)
    plan.sync_status()


def test_unnormalised_state_in_propagate_and_batch():
    s, B, plan, b0, bf = c1_plan()
    u = ut_of(I.pulses_uniform(0, s.N, 2))
    plan.propagate(u, api.to_device(b0 * 0.5, DEV))
    with pytest.raises(_lib.QocError) as e:
        plan.sync_status()
    assert code_of(e) == _lib.QOC_EINVAL
    # batch: only problem 1 of 2 is off
    probs = I.sn_problem_batch(2, n_lo=8, n_hi=10)
    bases = [api.Basis(I.sn_allpairs(p.n, p.J, p.h, 10.0, p.N), first_block_only=True) for p in probs]
    bp = api.Plan(bases, [p.N for p in probs], [10.0 / p.N for p in probs], prec="f64")
    psi0 = np.concatenate([b.dicke_state(0) for b in bases])
    psif = np.concatenate([b.dicke_state(p.k_target) for b, p in zip(bases, probs)])
    ub = ut_of(np.concatenate([I.pulses_uniform(p.seed, p.N, 2) for p in probs]))
    bp.fidelity_and_grad(ub, api.to_device(psi0, DEV), api.to_device(psif, DEV))
    bp.sync_status()
    psif_bad = psif.copy()
    psif_bad[bases[0].state_len:] *= 1.001
    bp.fidelity_and_grad(ub, api.to_device(psi0, DEV), api.to_device(psif_bad, DEV))
    with pytest.raises(_lib.QocError) as e:
        bp.sync_status()
    assert code_of(e) == _lib.QOC_EINVAL


def test_latched_error_is_returned_by_the_next_call():
    s, B, plan, b0, bf = c1_plan()
    u = I.pulses_uniform(0, s.N, 2)
    u[3, 0] = np.inf
    d0, df = api.to_device(b0, DEV), api.to_device(bf, DEV)
    plan.fidelity_and_grad(ut_of(u), d0, df)
    torch.cuda.synchronize()  # the failing call has finished
    with pytest.raises(_lib.QocError, match="non-finite") as e:
        plan.fidelity_and_grad(ut_of(I.pulses_uniform(0, s.N, 2)), d0, df)
    assert code_of(e) == _lib.QOC_EINVAL
    # returned once: the next call and the status word are clean
    out3, g = plan.fidelity_and_grad(ut_of(I.pulses_uniform(0, s.N, 2)), d0, df)
    plan.sync_status()
    assert np.isfinite(g.cpu().numpy()).all()


def test_squaring_cap_is_reported():
    # a slice norm of about 2e3 needs ~10 halvings; the plan allows one
    s, B, plan, b0, bf = c1_plan(max_squarings=1)
    u = I.pulses_uniform(0, s.N, 2) * 1000.0
    plan.fidelity_and_grad(ut_of(u), api.to_device(b0, DEV), api.to_device(bf, DEV))
    with pytest.raises(_lib.QocError, match="squarings") as e:
        plan.sync_status()
    assert code_of(e) == _lib.QOC_EUNSUPPORTED


def test_optimize_stops_on_latched_error():
    s, B, plan, b0, bf = c1_plan()
    u = I.pulses_uniform(0, s.N, 2)
    u[10, 1] = np.nan
    ut = ut_of(u)
    with pytest.raises(_lib.QocError, match="non-finite") as e:
        plan.optimize(ut, api.to_device(b0, DEV), api.to_device(bf, DEV), iters=50, step=0.1, f_target=0.999,
                      check_every=5)
    assert code_of(e) == _lib.QOC_EINVAL


def test_bounded_wait_times_out_and_context_survives():
    s, B, plan, b0, bf = c1_plan()
    plan.selftest_wait(limit_ms=2.0)
    with pytest.raises(_lib.QocError) as e:
        plan.sync_status()
    assert code_of(e) == _lib.QOC_ETIMEOUT
    # returned by the next call too, once the waiting kernel has finished
    plan.selftest_wait(limit_ms=1.0)
    torch.cuda.synchronize()
    u = I.pulses_uniform(0, s.N, 2)
    d0, df = api.to_device(b0, DEV), api.to_device(bf, DEV)
    with pytest.raises(_lib.QocError) as e:
        plan.fidelity_and_grad(ut_of(u), d0, df)
    assert code_of(e) == _lib.QOC_ETIMEOUT
    # the context is still usable: an evaluation matches the oracle
    out3, g = plan.fidelity_and_grad(ut_of(u), d0, df)
    torch.cuda.synchronize()
    plan.sync_status()
    H0, Hc = op.system_operators(s)
    prob = sy.block_problem(s, H0, Hc, sy.symmetry_blocks(s), I.basis_state(4, 0), op.dicke_state(4, 2))
    F, _, gref = gr.fidelity_and_grad(prob, u, s.tau)
    assert abs(out3[0].item() - F) <= 1e-10
    assert np.linalg.norm(g.cpu().numpy() - gref) / np.linalg.norm(gref) <= 1e-10


def test_selftest_rejects_bad_limits():
    _, _, plan, _, _ = c1_plan()
    for bad in (0.0, -1.0, 5000.0, float("nan")):
        with pytest.raises(_lib.QocError) as e:
            plan.selftest_wait(limit_ms=bad)
        assert code_of(e) == _lib.QOC_EINVAL


# ------------------------------------------------------------------ split adjoint behind autograd
@pytest.mark.parametrize("prec,seg", [("f32", 0), ("f32", -1), ("f64", 0), ("f64", 7)])
def test_split_halves_equal_fused_call(prec, seg):
    s, plan, psi0, psif, d0, df = d8_plan(prec, seg)
    u = ut_of(I.pulses_normal(23, s.N, 3))
    out3, g = plan.fidelity_and_grad(u, d0, df)
    o1, serial = plan.forward(u, d0, df)
    g1 = plan.backward(u, df, serial)
    torch.cuda.synchronize()
    plan.sync_status()
    assert np.array_equal(out3.cpu().numpy(), o1.cpu().numpy())
    assert np.array_equal(g.cpu().numpy(), g1.cpu().numpy())


@pytest.mark.parametrize("seg", [0, -1])
def test_forward_runs_no_derivative_kernel(seg):
    s, plan, psi0, psif, d0, df = d8_plan("f32", seg)
    u = ut_of(I.pulses_normal(23, s.N, 3)).requires_grad_(True)
    plan.set_profiling(True)
    with torch.no_grad():
        F = api.FidelityGrad.apply(u, plan, d0, df)
    torch.cuda.synchronize()
    c_fwd = plan.work_counts()
    assert c_fwd[2] > 0          # propagators were computed
    assert c_fwd[3] == 0         # no slice-derivative series ran
    assert 0 <= c_fwd[5] <= c_fwd[0] + c_fwd[1]  # three-term products are a part of all products
    F = api.FidelityGrad.apply(u, plan, d0, df)
    torch.cuda.synchronize()
    c_mid = plan.work_counts()
    assert c_mid[3] == 0
    F.backward()
    torch.cuda.synchronize()
    c_bwd = plan.work_counts()
    assert c_bwd[3] > 0          # the derivatives ran in backward
    if seg != 0:                 # checkpointed: backward recomputed every propagator once more
        assert c_bwd[2] - c_mid[2] == c_mid[2] - c_fwd[2]
    plan.set_profiling(False)
    H0, Hc = op.system_operators(s)
    prob = sy.block_problem(s, H0, Hc, sy.symmetry_blocks(s), psi0, psif)
    Fr, _, gref = gr.fidelity_and_grad(prob, I.pulses_normal(23, s.N, 3), s.tau)
    assert abs(F.item() - Fr) <= 1e-5
    assert np.linalg.norm(u.grad.cpu().numpy() - gref) / np.linalg.norm(gref) <= 1e-5


def test_backward_after_reuse_raises():
    s, plan, psi0, psif, d0, df = d8_plan("f32")
    u = ut_of(I.pulses_normal(23, s.N, 3)).requires_grad_(True)
    F1 = api.FidelityGrad.apply(u, plan, d0, df)
    F2 = api.FidelityGrad.apply(u, plan, d0, df)  # overwrites the workspace F1's backward needs
    with pytest.raises(RuntimeError, match="reused"):
        F1.backward()
    F2.backward()


def test_batched_autograd_scales_each_problem():
    probs = I.sn_problem_batch(3, n_lo=8, n_hi=12)
    T = 10.0
    bases = [api.Basis(I.sn_allpairs(p.n, p.J, p.h, T, p.N), first_block_only=True) for p in probs]
    plan = api.Plan(bases, [p.N for p in probs], [T / p.N for p in probs], prec="f64")
    psi0 = api.to_device(np.concatenate([b.dicke_state(0) for b in bases]), DEV)
    psif = api.to_device(np.concatenate([b.dicke_state(p.k_target) for b, p in zip(bases, probs)]), DEV)
    u0 = np.concatenate([I.pulses_uniform(p.seed, p.N, 2) for p in probs])
    u = ut_of(u0).requires_grad_(True)
    F = api.FidelityGrad.apply(u, plan, psi0, psif)
    assert F.shape == (3,)
    w = torch.tensor([0.5, -2.0, 3.0], dtype=torch.float64, device=DEV)
    (w * F).sum().backward()
    out3, g = plan.fidelity_and_grad(ut_of(u0), psi0, psif)
    torch.cuda.synchronize()
    plan.sync_status()
    rows = np.cumsum([0] + [p.N for p in probs])
    ga, gb = u.grad.cpu().numpy(), g.cpu().numpy()
    for i in range(3):
        sl = slice(rows[i], rows[i + 1])
        assert np.allclose(ga[sl], w[i].item() * gb[sl], rtol=1e-14, atol=0)
    assert np.array_equal(F.detach().cpu().numpy(), out3.view(3, 3)[:, 0].cpu().numpy())
