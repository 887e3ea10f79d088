"""Learned warm start for batched GRAPE on S_n problems (not in the paper; scored by the method's own
fidelity).

A network maps a problem's parameters (n, J, h, target Dicke index k) to the N x 2 initial pulses
of GRAPE; it is trained on pulses that this library's batched GRAPE optimised to F >= f_target.
All arithmetic runs in the library's kernels (qoc_dense_forward / qoc_dense_backward / qoc_adam_step /
qoc_mse); torch only holds the device memory.

Pulse gauge: H0 = J sum_{i<j} Z_i Z_j + h sum Z_i, |0...0> and every Dicke state commute with sum Z, so
multiplying the complex pulse u_x + i u_y by a constant phase changes no fidelity.  Training targets
are rotated so that sum_k (u_x,k + i u_y,k) is real and positive; otherwise the regression would
average optima that differ only by that phase.
"""
from __future__ import annotations

import ctypes as C
import time
from dataclasses import dataclass
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

from . import _lib as L
from . import api
from . import inputs as I

FEATURES = 4


def features(probs: Sequence[I.SnProblem]) -> np.ndarray:
    """(n/32, J/2, h, k/n) per problem."""
    return np.array([[p.n / 32.0, p.J / 2.0, p.h, p.k_target / p.n] for p in probs], dtype=np.float32)


def canonicalize(u: np.ndarray) -> np.ndarray:
    """Rotate pulses [N, 2] so that sum_k (u_x + i u_y) is real and positive (a symmetry of F)."""
    z = u[:, 0] + 1j * u[:, 1]
    s = z.sum()
    if abs(s) > 0:
        z = z * np.exp(-1j * np.angle(s))
    return np.stack([z.real, z.imag], axis=1)


def _p(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


class WarmStartMLP:
    """Fully connected network: GELU hidden layers, identity output; BF16 weights, FP32 master copy."""

    def __init__(self, dims=(FEATURES, 256, 256, 256, 400), seed: int = 0, device=None):
        self.lib = L.load()
        self.dims = list(dims)
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else device
        g = np.random.default_rng(seed)
        self.W, self.Wb, self.b, self.m, self.v = [], [], [], [], []
        for i in range(len(dims) - 1):
            fan_in = dims[i]
            W = (g.normal(size=(dims[i + 1], dims[i])) * np.sqrt(2.0 / fan_in)).astype(np.float32)
            Wt = torch.from_numpy(W).to(self.device)
            self.W.append(Wt)
            self.b.append(torch.zeros(dims[i + 1], dtype=torch.float32, device=self.device))
            Wb = torch.empty(W.shape, dtype=torch.bfloat16, device=self.device)
            L.check(self.lib.qoc_to_bf16(_p(Wt), _p(Wb), Wt.numel(), self._s()), "qoc_to_bf16")
            self.Wb.append(Wb)
        self.m = [torch.zeros_like(t) for t in self.W + self.b]
        self.v = [torch.zeros_like(t) for t in self.W + self.b]
        self.t = 0
        self.scale = 1.0  # output scaling of the targets

    def _s(self):
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)

    @property
    def n_layers(self):
        return len(self.W)

    def forward(self, X: torch.Tensor):
        """Returns (Y, cache); cache[l] = (input, Z) of layer l."""
        y = X.contiguous()
        cache = []
        for l in range(self.n_layers):
            B = y.shape[0]
            out = self.dims[l + 1]
            Z = torch.empty(B, out, dtype=torch.float32, device=self.device)
            Y = torch.empty_like(Z)
            act = 1 if l < self.n_layers - 1 else 0
            L.check(self.lib.qoc_dense_forward(_p(y), _p(self.Wb[l]), _p(self.b[l]), _p(Z), _p(Y), B,
                                               self.dims[l], out, act, self._s()), "qoc_dense_forward")
            cache.append((y, Z))
            y = Y
        return y, cache

    def backward(self, cache, dY: torch.Tensor):
        grads = [None] * self.n_layers
        g = dY.contiguous()
        for l in range(self.n_layers - 1, -1, -1):
            x, Z = cache[l]
            B = x.shape[0]
            dZ = torch.empty_like(Z)
            dX = torch.empty_like(x) if l > 0 else None
            dW = torch.empty_like(self.W[l])
            db = torch.empty_like(self.b[l])
            act = 1 if l < self.n_layers - 1 else 0
            L.check(self.lib.qoc_dense_backward(_p(x), _p(self.Wb[l]), _p(Z), _p(g), _p(dZ), _p(dX), _p(dW), _p(db), B,
                                                self.dims[l], self.dims[l + 1], act, self._s()), "qoc_dense_backward")
            grads[l] = (dW, db)
            g = dX
        return grads

    def loss_and_grads(self, X: torch.Tensor, T: torch.Tensor):
        Y, cache = self.forward(X)
        dY = torch.empty_like(Y)
        loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        L.check(self.lib.qoc_mse(_p(Y), _p(T), _p(dY), _p(loss), Y.numel(), self._s()), "qoc_mse")
        return loss, self.backward(cache, dY)

    def step(self, grads, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
        self.t += 1
        params = self.W + self.b
        gl = [g[0] for g in grads] + [g[1] for g in grads]
        shadows = self.Wb + [None] * len(self.b)
        for p, sh, g, m, v in zip(params, shadows, gl, self.m, self.v):
            L.check(self.lib.qoc_adam_step(_p(p), _p(sh), _p(g), _p(m), _p(v), p.numel(), lr, beta1, beta2, eps,
                                           self.t, self._s()), "qoc_adam_step")

    def fit(self, X: np.ndarray, T: np.ndarray, epochs: int = 200, batch: int = 512, lr: float = 1e-3,
            seed: int = 0) -> List[float]:
        """Minibatch Adam on the MSE between the network and the (scaled) targets."""
        self.scale = float(np.std(T)) or 1.0
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T / self.scale, dtype=np.float32)
        g = np.random.default_rng(seed)
        hist = []
        n = X.shape[0]
        for ep in range(epochs):
            perm = g.permutation(n)  # shuffled on the host, uploaded once per epoch
            Xd = torch.from_numpy(X[perm]).to(self.device)
            Td = torch.from_numpy(T[perm]).to(self.device)
            tot = 0.0
            for i in range(0, n, batch):
                loss, grads = self.loss_and_grads(Xd[i:i + batch], Td[i:i + batch])
                self.step(grads, lr)
                tot += float(loss.item()) * min(batch, n - i)
            hist.append(tot / n)
        return hist

    def predict(self, X: np.ndarray) -> np.ndarray:
        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(self.device)
        Y, _ = self.forward(Xd)
        return Y.cpu().numpy().astype(np.float64) * self.scale

    def params_for_oracle(self):
        """[(W as the BF16 values the device uses, b)] in float64."""
        out = []
        for Wb, b in zip(self.Wb, self.b):
            bits = Wb.view(torch.int16).cpu().numpy().view(np.uint16).astype(np.uint32) << 16
            out.append((bits.view(np.float32).astype(np.float64), b.cpu().numpy().astype(np.float64)))
        return out


# ------------------------------------------------------------------------------ GRAPE on S_n batches
@dataclass
class SolveResult:
    pulses: np.ndarray       # [P, N, 2]
    reached: np.ndarray      # first iteration with F >= f_target, -1 if never
    F_final: np.ndarray
    iters: int
    seconds: float


def sn_batch_plan(probs: Sequence[I.SnProblem], T: float, prec: str = "f32_all"):
    systems = [I.sn_allpairs(p.n, p.J, p.h, T, p.N) for p in probs]
    bases = [api.Basis(s, first_block_only=True, vectors=False) for s in systems]
    psi0 = np.concatenate([b.dicke_state(0) for b in bases])
    psif = np.concatenate([b.dicke_state(p.k_target) for b, p in zip(bases, probs)])
    plan = api.Plan(bases, [p.N for p in probs], [T / p.N for p in probs], prec=prec)
    return plan, api.to_device(psi0), api.to_device(psif)


def solve_batch(probs: Sequence[I.SnProblem], u0: np.ndarray, T: float, iters: int, lr: float,
                f_target: float = 0.999, check_every: int = 20, prec: str = "f32_all", use_graph: bool = True,
                plan_cache: Optional[Dict] = None) -> SolveResult:
    """Batched Adam GRAPE on S_n problems of equal N from pulses u0 [P, N, 2]; converged problems freeze."""
    key = (tuple((p.n, p.J, p.h, p.N, p.k_target) for p in probs), T, prec)
    if plan_cache is not None and key in plan_cache:
        plan, d0, df = plan_cache[key]
    else:
        plan, d0, df = sn_batch_plan(probs, T, prec)
        if plan_cache is not None:
            plan_cache[key] = (plan, d0, df)
    u = torch.from_numpy(np.ascontiguousarray(u0.reshape(-1, 2), dtype=np.float64)).to(plan.device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Fh, done, _ = plan.optimize(u, d0, df, iters, lr, f_target=f_target, check_every=check_every, rule="adam",
                                use_graph=use_graph)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    reached = plan.last_reached.cpu().numpy()
    F_last = Fh[-1].cpu().numpy() if done > 0 else np.zeros(len(probs))
    return SolveResult(u.cpu().numpy().reshape(len(probs), -1, 2), reached, np.atleast_1d(F_last), done, secs)


def solve_compacting(probs: Sequence[I.SnProblem], u0: np.ndarray, T: float, cap: int, lr: float,
                     f_target: float = 0.999, round_iters: int = 100, prec: str = "f32_all"):
    """Batched Adam GRAPE in rounds of round_iters; after each round the converged problems leave the
    batch (their pulses are kept) and the rest continue from where they are.  Returns (pulses [P,N,2],
    iterations to f_target per problem (-1 if not within cap), seconds)."""
    P = len(probs)
    pulses = np.array(u0, dtype=np.float64, copy=True)
    reached = np.full(P, -1, dtype=np.int64)
    active = np.arange(P)
    done, secs = 0, 0.0
    while len(active) and done < cap:
        it = min(round_iters, cap - done)
        res = solve_batch([probs[i] for i in active], pulses[active], T, it, lr, f_target, check_every=it,
                          prec=prec, use_graph=True)
        secs += res.seconds
        pulses[active] = res.pulses
        hit = res.reached >= 0
        reached[active[hit]] = done + res.reached[hit]
        active = active[~hit]
        done += it
    return pulses, reached, secs


def generate_dataset(count: int, base_seed: int, N: int = 200, T: float = 10.0, n_lo: int = 8, n_hi: int = 32,
                     iters: int = 400, lr: float = 0.05, f_target: float = 0.999, init_seed: Optional[int] = 0):
    """Optimise `count` seeded problems and keep the converged ones as (features, canonical pulses).

    init_seed: every problem starts from the same U[-1,1] pulse shape (seed init_seed), so that the
    optimum reached varies smoothly with the problem's parameters; None = each problem's own seed."""
    probs = I.sn_problem_batch(count, base_seed=base_seed, n_lo=n_lo, n_hi=n_hi, N_lo=N, N_hi=N)
    if init_seed is None:
        u0 = np.stack([I.pulses_uniform(p.seed, N, 2) for p in probs])
    else:
        u0 = np.broadcast_to(I.pulses_uniform(init_seed, N, 2), (count, N, 2)).copy()
    pulses, reached, seconds = solve_compacting(probs, u0, T, iters, lr, f_target)
    keep = np.nonzero(reached >= 0)[0]
    X = features([probs[i] for i in keep])
    Y = np.array([canonicalize(pulses[i]).reshape(-1) for i in keep], np.float32)
    return X, Y, [probs[i] for i in keep], seconds


def evaluate(model: Optional[WarmStartMLP], probs: Sequence[I.SnProblem], T: float = 10.0, cap: int = 5000,
             warm_budget: int = 300, lr: float = 0.05, f_target: float = 0.999) -> Dict:
    """Iterations and wall time to F >= f_target: plain GRAPE from U[-1,1] pulses (each problem's own
    seed) versus the network's pulses followed by GRAPE, falling back to plain GRAPE for problems the
    warm start leaves below f_target after warm_budget iterations (their plain iterations and time are
    added).  Both arms run batched with compaction."""
    N = probs[0].N
    u_rand = np.stack([I.pulses_uniform(p.seed, N, 2) for p in probs])
    _, r_plain, s_plain = solve_compacting(probs, u_rand, T, cap, lr, f_target)
    it_plain = np.where(r_plain >= 0, r_plain, cap)
    out = {"problems": len(probs),
           "plain": {"iters_median": float(np.median(it_plain)), "iters_mean": float(np.mean(it_plain)),
                     "failures": int((r_plain < 0).sum()), "seconds": s_plain}}
    if model is None:
        return out
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    u_warm = model.predict(features(probs)).reshape(len(probs), N, 2)
    torch.cuda.synchronize()
    t_inf = time.perf_counter() - t0
    _, r_warm, s_warm = solve_compacting(probs, u_warm, T, warm_budget, lr, f_target)
    iters = np.where(r_warm >= 0, r_warm, -1).astype(float)
    fb = np.nonzero(r_warm < 0)[0]
    s_fb, fails = 0.0, 0
    if len(fb):
        _, r_fb, s_fb = solve_compacting([probs[i] for i in fb], u_rand[fb], T, cap, lr, f_target)
        iters[fb] = warm_budget + np.where(r_fb >= 0, r_fb, cap)
        fails = int((r_fb < 0).sum())
    out["warm"] = {"iters_median": float(np.median(iters)), "iters_mean": float(np.mean(iters)),
                   "fallbacks": int(len(fb)), "failures": fails, "seconds": t_inf + s_warm + s_fb,
                   "inference_seconds": t_inf}
    out["speedup_wall"] = s_plain / out["warm"]["seconds"] if out["warm"]["seconds"] > 0 else None
    return out
