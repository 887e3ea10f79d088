"""Parity at the shapes the headline workloads run (FP32 paths, tolerance 1e-5 on F and on the
relative gradient error, states element-wise in the full space):

- the D_14 XXZ ring's two-dimensional irreps E1 (1161 states) and E2 (1179 states), both copies,
  through the default FP32 kernels: tiled tcgen05 GEMM exponentials (blocks above 112 states),
  cluster sweeps with 197-row slices (clusters of 6) and the automatic choice, sqrt(N) checkpointing;
- the batched S_n workload's largest problems (n = 32, 48, 64; N up to 1000; T = 10), where slice
  norms reach |tau H| ~ 200: this regime runs in FP64 (tolerance 1e-10).  An FP32 polynomial loses
  about 2^s sqrt(m) eps_32 per slice after s halvings, ~1e-3 in the final state, whether the squaring
  chain is FP32 or FP64, because the error enters before the squarings;
- the warm-start network at its trained widths 4-256-256-256-400.

The oracle builds its own E1/E2 basis (projectors of the dihedral group on the orbits) and works in
it; the library's basis differs by a rotation inside each block, so states are compared in the full
space.  The D_14 target is the oracle's own final state mixed with a seeded random one, so that
|<psi_f|psi_N>| is of order one and a relative gradient error measures the arithmetic rather than
the conditioning of a near-zero overlap.
"""
import numpy as np
import pytest

from oracle import grape as gr
from oracle import mlp as omlp
from oracle import operators as op
from oracle import symmetry as sy
from paper_2309_05884_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2309_05884_gb300 import api  # noqa: E402
from paper_2309_05884_gb300 import warmstart as ws  # noqa: E402

DEV = torch.device("cuda", 0)
TOL32 = 1e-5


def _project(B, full, labels):
    """Block coordinates of a full-space state kept on the named blocks only, normalised."""
    blk = B.state_to_blocks(full)
    for label, m, c, off in B.blocks:
        if label not in labels:
            blk[off: off + m * c] = 0
    return blk / np.linalg.norm(blk)


@pytest.fixture(scope="module")
def d14_e_blocks():
    # tau = 0.02 as in the T = 40, N = 2000 workload; 16 slices keep the oracle's 1161/1179-state
    # eigendecompositions short
    s = I.xxz_ring(14, 0.32, 16)
    labels = ("E1", "E2")
    B = api.Basis(s)
    sizes = {l: (m, c) for l, m, c, _ in B.blocks}
    assert sizes["E1"] == (1161, 2) and sizes["E2"] == (1179, 2)
    b0 = _project(B, I.random_state(311, 2 ** 14), labels)
    psi0 = B.blocks_to_state(b0)
    u = I.pulses_normal(2, s.N, 3)
    H0, Hc = op.system_operators(s)
    ob = sy.dn_blocks(14, labels=list(labels))
    # oracle final state from psi0 alone (target-independent), then a target close to it
    p0 = sy.block_problem(s, H0, Hc, ob, psi0, psi0)
    fin = gr.final_states(p0, u, s.tau)
    psiN_ref = sy.from_blocks(ob, fin)
    bf = _project(B, psiN_ref + 0.6 * I.random_state(312, 2 ** 14), labels)
    psif = B.blocks_to_state(bf)
    prob = sy.block_problem(s, H0, Hc, ob, psi0, psif)
    F, o, g = gr.fidelity_and_grad(prob, u, s.tau)
    assert 0.2 < F < 0.95
    return dict(s=s, B=B, b0=b0, bf=bf, u=u, F=F, g=g, psiN=psiN_ref)


@pytest.mark.slow
@pytest.mark.parametrize("cl,seg", [(6, -1), (-1, 0)])
def test_d14_e_blocks_fp32(d14_e_blocks, cl, seg):
    d = d14_e_blocks
    s, B = d["s"], d["B"]
    plan = api.Plan(B, s.N, s.tau, prec="f32", active=B.active_copies(d["b0"], d["bf"]), ckpt_segment=seg)
    classes = plan.expm_classes()
    assert any(k == 3 and mx >= 1161 for k, _, _, mx, _ in classes), classes  # tiled tensor-core GEMMs
    plan.set_sweep_cluster(cl)
    if cl == 6:
        assert plan.sweep_cluster() == 6  # rows per CTA: ceil(1179 / 6) = 197
    d0, df = api.to_device(d["b0"], DEV), api.to_device(d["bf"], DEV)
    ut = torch.from_numpy(d["u"]).to(DEV)
    out3, g = plan.fidelity_and_grad(ut, d0, df)
    psiN = plan.propagate(ut, d0)
    torch.cuda.synchronize()
    plan.sync_status()
    assert abs(out3[0].item() - d["F"]) <= TOL32
    gg = g.cpu().numpy()
    assert np.linalg.norm(gg - d["g"]) / np.linalg.norm(d["g"]) <= TOL32
    full = B.blocks_to_state(psiN.cpu().numpy())
    assert np.abs(full - d["psiN"]).max() <= TOL32
    # the split adjoint behind autograd gives the same gradient
    ua = ut.clone().requires_grad_(True)
    F = api.FidelityGrad.apply(ua, plan, d0, df)
    F.backward()
    assert np.array_equal(ua.grad.cpu().numpy(), gg)


def _sn_oracle_block(n, J, h, k):
    """The oracle's own J = n/2 block of J sum_{i<j} Z_i Z_j + h sum Z_i with controls sum X, sum Y."""
    Jz, Jp, Jm = sy.spin_matrices(n)
    m = n + 1
    p0 = np.zeros((m, 1), complex)
    p0[0] = 1
    pf = np.zeros((m, 1), complex)
    pf[k] = 1
    return [dict(h0=J * (2 * Jz @ Jz - n / 2 * np.eye(m)) + h * 2 * Jz, hc=[Jp + Jm, -1j * (Jp - Jm)],
                 psi0=p0, psif=pf)]


def test_sn_batch_largest_problems_fp64():
    T = 10.0
    shapes = [(32, 400), (48, 700), (64, 1000), (64, 200), (40, 1000), (56, 300)]
    probs = []
    for i, (n, N) in enumerate(shapes):
        g = I.rng(30_000 + i)
        probs.append(I.SnProblem(n, float(g.uniform(0.5, 2)), float(g.uniform(0, 1)), N, int(g.integers(0, n + 1)),
                                 30_000 + i))
    bases = [api.Basis(I.sn_allpairs(p.n, p.J, p.h, T, p.N), first_block_only=True, vectors=False) for p in probs]
    plan = api.Plan(bases, [p.N for p in probs], [T / p.N for p in probs], prec="f64")
    d0 = api.to_device(np.concatenate([b.dicke_state(0) for b in bases]), DEV)
    df = api.to_device(np.concatenate([b.dicke_state(p.k_target) for b, p in zip(bases, probs)]), DEV)
    us = [I.pulses_uniform(p.seed, p.N, 2) for p in probs]
    out3, g = plan.fidelity_and_grad(torch.from_numpy(np.concatenate(us)).to(DEV), d0, df)
    torch.cuda.synchronize()
    plan.sync_status()
    out, g = out3.cpu().numpy().reshape(-1, 3), g.cpu().numpy()
    row = 0
    for i, p in enumerate(probs):
        F, o, gref = gr.fidelity_and_grad(_sn_oracle_block(p.n, p.J, p.h, p.k_target), us[i], T / p.N)
        gi = g[row: row + p.N]
        row += p.N
        assert abs(out[i, 0] - F) <= 1e-10 * max(F, 1e-3)
        # a target the pulses cannot reach leaves a gradient at rounding level (|g| ~ 1e-17): there the
        # absolute error is what is bounded
        gn = np.linalg.norm(gref)
        assert np.linalg.norm(gi - gref) <= 1e-10 * max(gn, 1e-8), (i, p, gn)


@pytest.mark.parametrize("batch", [512, 37])
def test_mlp_trained_widths_match_oracle(batch):
    net = ws.WarmStartMLP(dims=(4, 256, 256, 256, 400), seed=5, device=DEV)
    rng = np.random.default_rng(11)
    X = rng.uniform(0, 1, size=(batch, 4)).astype(np.float32)
    T = rng.normal(size=(batch, 400)).astype(np.float32)
    for b in net.b:
        b.copy_(torch.from_numpy(rng.normal(size=b.shape).astype(np.float32) * 0.1))
    Xd, Td = torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV)
    Y, _ = net.forward(Xd)
    params = net.params_for_oracle()
    Yr, cr = omlp.forward(params, X.astype(np.float64))
    assert np.abs(Y.cpu().numpy() - Yr).max() <= 1e-5 * max(1.0, np.abs(Yr).max())
    loss, grads = net.loss_and_grads(Xd, Td)
    Lr, dYr = omlp.mse(Yr, T.astype(np.float64))
    assert abs(loss.item() - Lr) <= 1e-5 * Lr
    for (dW, db), (dWr, dbr) in zip(grads, omlp.backward(params, cr, dYr)):
        assert np.linalg.norm(dW.cpu().numpy() - dWr) <= 1e-4 * np.linalg.norm(dWr)
        assert np.linalg.norm(db.cpu().numpy() - dbr) <= 1e-4 * max(np.linalg.norm(dbr), 1e-12)


@pytest.mark.parametrize("n,first,seg", [(12, True, 0), (12, False, -1), (11, False, 7), (10, False, 0)])
def test_derivatives_gemm_paths_match_series_kernels(n, first, seg):
    # the tall-GEMM derivative path on the FP32 CUDA cores and on the tensor cores, for the blocks above
    # 128 states and (threshold 24) for every block, against the per-slice series kernels and the
    # oracle (D_12: A1 224 states; D_10, D_11, D_12 with every block, ragged chunks)
    s = I.xxz_ring(n, 0.02 * 30, 30)
    B = api.Basis(s, first_block_only=first)
    x, y = I.random_state(321, 2 ** n), I.random_state(322, 2 ** n)
    b0, bf = B.state_to_blocks(x), B.state_to_blocks(y)
    b0, bf = b0 / np.linalg.norm(b0), bf / np.linalg.norm(bf)
    u = torch.from_numpy(I.pulses_normal(4, s.N, 3)).to(DEV)
    d0, df = api.to_device(b0, DEV), api.to_device(bf, DEV)
    res = {}
    for mode, min_m in ((0, 129), (1, 129), (2, 129), (1, 24), (2, 24)):
        plan = api.Plan(B, s.N, s.tau, prec="f32", active=B.active_copies(b0, bf), ckpt_segment=seg)
        plan.set_deriv_gemm(mode, min_m)
        assert (plan.deriv_gemm_blocks() > 0) == (mode > 0 and max(m for _, m, _, _ in B.blocks) >= min_m)
        out3, g = plan.fidelity_and_grad(u, d0, df)
        torch.cuda.synchronize()
        plan.sync_status()
        res[(mode, min_m)] = (out3.cpu().numpy(), g.cpu().numpy())
    o0, g0 = res[(0, 129)]
    for key, (o1, g1) in res.items():
        assert np.array_equal(o1, o0)
        assert np.linalg.norm(g1 - g0) / np.linalg.norm(g0) <= 5e-6, key
    if not first:
        H0, Hc = op.system_operators(s)
        prob = sy.block_problem(s, H0, Hc, sy.symmetry_blocks(s), B.blocks_to_state(b0), B.blocks_to_state(bf))
        F, o, gref = gr.fidelity_and_grad(prob, u.cpu().numpy(), s.tau)
        for key, (o1, g1) in res.items():
            assert abs(o1[0] - F) <= TOL32
            assert np.linalg.norm(g1 - gref) / np.linalg.norm(gref) <= TOL32, key


def test_autotuner_every_choice_keeps_results(tmp_path):
    # D_11 (blocks of 126 and 186 states, FP32): exponential kinds per bucket, sweep cluster size and
    # the derivative path are tuned and cached; results stay within the FP32 tolerance
    from paper_2309_05884_gb300 import autotune
    s = I.xxz_ring(11, 0.02 * 24, 24)
    B = api.Basis(s)
    b0 = B.state_to_blocks(I.random_state(331, 2 ** 11))
    bf = B.state_to_blocks(I.random_state(332, 2 ** 11))
    plan = api.Plan(B, s.N, s.tau, prec="f32", active=B.active_copies(b0, bf))
    d0, df = api.to_device(b0, DEV), api.to_device(bf, DEV)
    u = torch.from_numpy(I.pulses_normal(8, s.N, 3)).to(DEV)
    o0, g0 = plan.fidelity_and_grad(u, d0, df)
    o0, g0 = o0.cpu().numpy(), g0.cpu().numpy()
    cache = str(tmp_path / "tune.json")
    rep = autotune.tune(plan, u, d0, df, reps=2, cache_path=cache)
    assert rep["expm"]["rules"] and len(rep["sweeps"]["trials"]) >= 2 and len(rep["derivatives"]["trials"]) >= 3
    o1, g1 = plan.fidelity_and_grad(u, d0, df)
    torch.cuda.synchronize()
    plan.sync_status()
    o1, g1 = o1.cpu().numpy(), g1.cpu().numpy()
    assert abs(o1[0] - o0[0]) <= 1e-5
    assert np.linalg.norm(g1 - g0) / np.linalg.norm(g0) <= 1e-5
    rep2 = autotune.tune(plan, u, d0, df, cache_path=cache)
    assert rep2["expm"]["cached"] and rep2["sweeps"]["cached"] and rep2["derivatives"]["cached"]
    assert rep2["sweeps"]["cl"] == rep["sweeps"]["cl"] and rep2["derivatives"]["mode"] == rep["derivatives"]["mode"]
