"""One persistent launch per GRAPE iteration (FP64 plans): the cooperative kernel that runs the norm
check, propagators, sweeps, overlaps, reverse-mode slice derivatives, gradient and update of every
problem and block against the oracle (1e-10) and against the multi-launch path; one launch per
iteration; graph replay of the persistent iteration follows the oracle's Adam trajectory."""
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


def oracle_block(n, J, h, k):
    Jz, Jp, Jm = sy.spin_matrices(n)
    m = n + 1
    p0 = np.zeros((m, 1), complex)
    p0[0] = 1
    pf = np.zeros((m, 1), complex)
    pf[k] = 1
    return [dict(h0=J * (2 * Jz @ Jz - n / 2 * np.eye(m)) + h * 2 * Jz, hc=[Jp + Jm, -1j * (Jp - Jm)],
                 psi0=p0, psif=pf)]


def sn_batch(probs, T):
    bases = [api.Basis(I.sn_allpairs(p.n, p.J, p.h, T, p.N), first_block_only=True, vectors=False) for p in probs]
    plan = api.Plan(bases, [p.N for p in probs], [T / p.N for p in probs], prec="f64")
    d0 = api.to_device(np.concatenate([b.dicke_state(0) for b in bases]), DEV)
    df = api.to_device(np.concatenate([b.dicke_state(p.k_target) for b, p in zip(bases, probs)]), DEV)
    us = [I.pulses_uniform(p.seed, p.N, 2) for p in probs]
    return plan, d0, df, us


def run(plan, u, d0, df):
    out3, g = plan.fidelity_and_grad(torch.from_numpy(np.ascontiguousarray(u)).to(DEV), d0, df)
    torch.cuda.synchronize()
    plan.sync_status()
    return out3.cpu().numpy().reshape(-1, 3), g.cpu().numpy()


def test_persistent_batch_matches_oracle_and_multi_launch():
    # T = 10 regime: many squarings (reverse mode), mixed block sizes (R = 1..4 tiles), ragged N
    probs = I.sn_problem_batch(12, base_seed=26_000, n_lo=4, n_hi=40, N_lo=40, N_hi=120)
    T = 10.0
    plan, d0, df, us = sn_batch(probs, T)
    u = np.concatenate(us)
    out_m, g_m = run(plan, u, d0, df)
    plan.set_persistent(True)
    assert plan.kernel_launches(True) == 1
    out_p, g_p = run(plan, u, d0, df)
    row = 0
    for i, p in enumerate(probs):
        F, o, gref = gr.fidelity_and_grad(oracle_block(p.n, p.J, p.h, p.k_target), us[i], T / p.N)
        gi = g_p[row: row + p.N]
        gn = np.linalg.norm(gref)
        assert abs(out_p[i, 0] - F) <= 1e-10 * max(F, 1e-3), (i, out_p[i, 0], F)
        assert np.linalg.norm(gi - gref) <= 1e-10 * max(gn, 1e-8), (i, p)
        row += p.N
    assert np.abs(out_p - out_m).max() <= 1e-14
    assert np.linalg.norm(g_p - g_m) <= 1e-11 * np.linalg.norm(g_m)
    # phase times come from the kernel's own stamps
    plan.set_profiling(True)
    run(plan, u, d0, df)
    ph = plan.phase_times()
    assert all(t >= 0 for t in ph) and ph[0] > 0 and ph[3] > 0
    plan.set_profiling(False)


def test_persistent_dn_all_blocks_fp64():
    s = I.xxz_ring(6, 1.5, 25)
    psi0, psif = I.random_state(41, 64), I.random_state(42, 64)
    B = api.Basis(s)
    b0, bf = B.state_to_blocks(psi0), B.state_to_blocks(psif)
    plan = api.Plan(B, s.N, s.tau, prec="f64", active=B.active_copies(b0, bf))
    plan.set_persistent(True)
    u = I.pulses_normal(9, s.N, 3)
    out, g = run(plan, u, api.to_device(b0, DEV), api.to_device(bf, DEV))
    H0, Hc = op.system_operators(s)
    F, o, gref = gr.fidelity_and_grad(sy.block_problem(s, H0, Hc, sy.symmetry_blocks(s), psi0, psif), u, s.tau)
    assert abs(out[0, 0] - F) <= 1e-10
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) <= 1e-10


def test_persistent_graph_adam_follows_oracle():
    probs = I.sn_problem_batch(5, base_seed=27_000, n_lo=4, n_hi=12, N_lo=30, N_hi=60)
    T = 10.0
    plan, d0, df, us = sn_batch(probs, T)
    plan.set_persistent(True)
    u = torch.from_numpy(np.concatenate(us)).to(DEV)
    iters, step = 12, 0.05
    Fh, done, _ = plan.optimize(u, d0, df, iters=iters, step=step, rule="adam", use_graph=True)
    torch.cuda.synchronize()
    plan.sync_status()
    Fh = Fh.cpu().numpy()
    for i, p in enumerate(probs):
        prob = oracle_block(p.n, p.J, p.h, p.k_target)
        _, hist, _ = gr.grape_adam(prob, us[i], T / p.N, iters, step)
        assert np.abs(Fh[:, i] - np.array(hist[:iters])).max() <= 1e-9, i


def test_persistent_rejects_unsupported_plans():
    s = I.xxz_ring(6, 1.5, 25)
    B = api.Basis(s)
    for kw in (dict(prec="f32"), dict(prec="f64", ckpt_segment=5), dict(prec="f64", grad_mode=1)):
        plan = api.Plan(B, s.N, s.tau, **kw)
        with pytest.raises(_lib.QocError) as e:
            plan.set_persistent(True)
        assert e.value.code == _lib.QOC_EUNSUPPORTED
