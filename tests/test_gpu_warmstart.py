"""The warm-start network's kernels against the FP64 oracle network (same BF16 weights)."""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2309_05884_gb300 import warmstart as ws  # noqa: E402

DEV = torch.device("cuda", 0)


def test_mlp_forward_backward_match_oracle():
    net = ws.WarmStartMLP(dims=(4, 40, 33, 17, 10), seed=3, device=DEV)
    rng = np.random.default_rng(7)
    X = rng.normal(size=(37, 4)).astype(np.float32)
    T = rng.normal(size=(37, 10)).astype(np.float32)
    Xd, Td = torch.from_numpy(X).to(DEV), torch.from_numpy(T).to(DEV)
    for b in net.b:  # nonzero biases
        b.copy_(torch.from_numpy(rng.normal(size=b.shape).astype(np.float32) * 0.1))
    Y, cache = net.forward(Xd)
    params = net.params_for_oracle()
    Yr, cr = omlp.forward(params, X.astype(np.float64))
    assert np.abs(Y.cpu().numpy() - Yr).max() <= 1e-5 * max(1.0, np.abs(Yr).max())
    loss, grads = net.loss_and_grads(Xd, Td)
    Lr, dYr = omlp.mse(Yr, T.astype(np.float64))
    assert abs(loss.item() - Lr) <= 1e-5 * Lr
    gr_ = omlp.backward(params, cr, dYr)
    for (dW, db), (dWr, dbr) in zip(grads, gr_):
        assert np.linalg.norm(dW.cpu().numpy() - dWr) <= 1e-4 * np.linalg.norm(dWr)
        assert np.linalg.norm(db.cpu().numpy() - dbr) <= 1e-4 * max(np.linalg.norm(dbr), 1e-12)
    # one Adam step: the BF16 shadow is the round-to-nearest of the FP32 master weights
    net.step(grads, 1e-2)
    for W, Wb in zip(net.W, net.Wb):
        assert torch.equal(W.to(torch.bfloat16).view(torch.int16), Wb.view(torch.int16))


def test_mlp_fit_reduces_loss():
    net = ws.WarmStartMLP(dims=(4, 64, 64, 8), seed=1, device=DEV)
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, size=(512, 4)).astype(np.float32)
    T = np.stack([np.sin(2 * X[:, 0]) * X[:, 1] + 0.3 * X[:, k % 4] for k in range(8)], axis=1).astype(np.float32)
    hist = net.fit(X, T, epochs=60, batch=128, lr=3e-3)
    assert hist[-1] < 0.1 * hist[0]


@pytest.mark.slow
def test_trained_network_gains_over_random_start():
    # T = 4: GRAPE from U[-1,1] pulses often starts at F ~ 1e-4 and stalls; the network, trained on
    # pulses the batched solver optimised, starts held-out problems in a far better place
    from paper_2309_05884_gb300 import inputs as I
    X, Y, kept, _ = ws.generate_dataset(1024, 100_000, N=200, T=4.0, n_lo=8, n_hi=16, iters=600, lr=0.05,
                                        init_seed=0)
    assert len(kept) > 700
    net = ws.WarmStartMLP(seed=0, device=DEV)
    hist = net.fit(X, Y, epochs=300, batch=256, lr=1e-3)
    assert hist[-1] < 0.5 * hist[0]
    held = I.sn_problem_batch(64, base_seed=900_000, n_lo=8, n_hi=16, N_lo=200, N_hi=200)
    u_pred = net.predict(ws.features(held)).reshape(len(held), 200, 2)
    u_rand = np.stack([I.pulses_uniform(p.seed, 200, 2) for p in held])
    F_pred = ws.solve_batch(held, u_pred, 4.0, 1, 0.0, f_target=2.0, use_graph=False).F_final
    F_rand = ws.solve_batch(held, u_rand, 4.0, 1, 0.0, f_target=2.0, use_graph=False).F_final
    assert np.median(F_pred) > 10 * np.median(F_rand)
    ev = ws.evaluate(net, held, T=4.0, cap=1500, warm_budget=200, lr=0.05)
    assert ev["warm"]["iters_mean"] < ev["plain"]["iters_mean"]
