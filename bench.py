"""Benchmark: GRAPE gradient evaluations per second on the largest single-GPU workload, the D_14 XXZ
ring with sqrt(N) checkpointing.

Workload (default, --workload d14): n = 14 qubits, H0 = sum_i (X_i X_{i+1} + Y_i Y_{i+1} + 0.5 Z_i
Z_{i+1}) on a periodic ring, controls u_x sum X, u_y sum Y, u_z sum Z, T = 40, N = 2000 slices,
pulses ~ N(0, 0.3^2) (seed 1).  All ten D_14 irrep blocks (A1 687, A2 495, B1 613, B2 549, E1-E6
1161/1179 x2 copies) carry amplitude: the initial and target states are seeded random full-space
states.  sqrt(N) checkpointing (45-slice segments): the costate pass recomputes each segment's
propagators.  Complex FP32 Taylor polynomial (tcgen05 tensor cores for blocks of 25..2048 states)
and sweeps, FP64 squaring chain, overlap and gradient accumulation.  One step = one GRAPE iteration:
F, dF/du (exact slice derivatives) and the update u <- u + eps dF/du, all on the device.
Other workloads: d10 (n = 10, T = 20, N = 500, every propagator stored), sn-batch (256 batched S_n
problems), warmstart (time to F >= 0.999 with and without the learned warm start).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload ...]

Prints one JSON line.  --impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (a few slices per step, scaled to whole gradient evaluations).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2309_05884_gb300 import inputs as I  # noqa: E402

METRIC = "GRAPE grad evals/s"
UNIT = "grad_evals/s"
WORKLOAD = ("D_10 XXZ ring (n=10, T=20, N=500, 3 controls), all 8 D_10 irrep blocks active "
            "(A1 78, A2 30, B1 58, B2 42, E1-E4 99/105 x2 copies)")
EPS = 0.5          # GRAPE step
SEED_U, SEED_PSI0, SEED_PSIF = 1, 101, 102
FP32_PEAK_NOTE = "FP32 FMA peak = 152 SMs x 128 lanes x 2 flop x 2.07 GHz (max SM clock) = 80.5 TFLOP/s"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# FP64 on GB300: 1.25 TFLOP/s nominal = 152 SMs x 2 FP64 FMA per clock x 2 flop x 2.07 GHz
FP64_PEAK_NOTE = "FP64 FMA peak = 152 SMs x 2 lanes x 2 flop x 2.07 GHz (max SM clock) = 1.26 TFLOP/s"
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def measured_peaks(long_step: bool = False):
    """HBM and dense tensor peaks from MEASURED_PEAKS.json (the profiling recipe's fallback if absent).
    long_step: the kernel runs inside a step of seconds, so the sustained tensor rate applies."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        key = "bf16_tflops_sustained" if long_step and "bf16_tflops_sustained" in d else "bf16_tflops"
        how = "sustained" if key.endswith("sustained") else "burst"
        return {"hbm_gbs": float(d["hbm_gbs"]), "hbm_note": "of measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "tensor_tflops": float(d[key]),
                "tensor_note": f"of measured dense BF16 {how} rate (MEASURED_PEAKS.json {key}); FP16 x 1"}
    except (OSError, KeyError, ValueError):
        t = 1700.0 if long_step else 1900.0
        return {"hbm_gbs": 6800.0, "hbm_note": "of fallback 6.8 TB/s", "tensor_tflops": t,
                "tensor_note": f"of fallback {t / 1000:.1f} PFLOP/s BF16; FP16 x 1"}


# DRAM bytes (read + write) of one launch of a workload's dominant kernel, from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum), with the launch it was taken on and that launch's
# algorithmic bytes; None where the kernel changed after the capture.  The profiles/ summaries
# name the commands.
# The last D_14 capture (profiles/xl_gemm_kernel_d14.md: the final product of the first chunk, 1273.7 MB
# against 1160.2 MB algorithmic) predates a change of that kernel's epilogue, so no figure is reported.
NCU_TRAFFIC = {
    "d14": None,
}


def workload():
    s = I.c2_system()
    psi0 = I.random_state(SEED_PSI0, 2 ** s.n)
    psif = I.random_state(SEED_PSIF, 2 ** s.n)
    u = I.pulses_normal(SEED_U, s.N, s.n_ctrl)
    return s, psi0, psif, u


SN_BATCH = 256
SN_T = 10.0
SN_WORKLOAD = (f"{SN_BATCH} independent S_n problems (H0 = J sum_{{i<j}} Z_i Z_j + h sum Z_i, controls sum X, sum Y), "
               f"n ~ U{{8..64}}, J ~ U[0.5,2], h ~ U[0,1], N ~ U{{200..1000}}, T = {SN_T}, |0...0> -> Dicke "
               f"D(n,k), k ~ U{{0..n}}, pulses U[-1,1], seeds 10000+i; block J = n/2 (size n+1) per problem")


def sn_batch_problems(count: int = SN_BATCH):
    return I.sn_problem_batch(count, base_seed=10_000)


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            try:
                rows.append(dict(sm=float(f[1]), smax=float(f[2]), power=float(f[3]),
                                 hw=f[5], hwt=f[6], swt=f[7], pcap=f[8], util=float(f[9])))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        loaded = [r for r in rows if r["util"] > 0] or rows
        reasons = set()
        for r in loaded:
            if r["hw"].startswith("Active"):
                reasons.add("hw_slowdown")
            if r["hwt"].startswith("Active"):
                reasons.add("hw_thermal_slowdown")
            if r["swt"].startswith("Active"):
                reasons.add("sw_thermal_slowdown")
            if r["pcap"].startswith("Active"):
                reasons.add("sw_power_cap")
        return {"sm_mhz": float(np.median([r["sm"] for r in loaded])), "sm_max_mhz": loaded[0]["smax"],
                "power_w_max": max(r["power"] for r in loaded), "reasons": sorted(reasons),
                "samples": len(loaded)}


# --------------------------------------------------------------------------- oracle (CPU) legs
def oracle_problem(s, psi0, psif, N_sample):
    from oracle import operators as op
    from oracle import symmetry as sy
    sub = I.System(s.n, s.group, s.h0, s.hc, s.tau * N_sample, N_sample)
    H0, Hc = op.system_operators(sub)
    return sub, sy.block_problem(sub, H0, Hc, sy.symmetry_blocks(sub), psi0, psif)


def cpu_oracle_rate(s, psi0, psif, u, N_sample, reps=1):
    """Grad evals/s of the oracle on the first N_sample slices, scaled to the whole workload."""
    from oracle import grape as gr
    sub, prob = oracle_problem(s, psi0, psif, N_sample)
    t0 = time.perf_counter()
    for _ in range(reps):
        gr.fidelity_and_grad(prob, u[:N_sample], sub.tau)
    dt = time.perf_counter() - t0
    return reps * (N_sample / s.N) / dt, dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    if args.workload == "d14":
        s, psi0, psif, u = d14_workload()
        Ns, name = 2, D14_WORKLOAD
    else:
        s, psi0, psif, u = workload()
        Ns, name = 50, WORKLOAD
    from oracle import grape as gr
    sub, prob = oracle_problem(s, psi0, psif, Ns)
    uu = u[:Ns].copy()
    for _ in range(args.warmup):
        _, _, g = gr.fidelity_and_grad(prob, uu, sub.tau)
        uu += EPS * g
    t0 = time.perf_counter()
    for _ in range(args.steps):
        _, _, g = gr.fidelity_and_grad(prob, uu, sub.tau)
        uu += EPS * g
    dt = time.perf_counter() - t0
    value = args.steps * (Ns / s.N) / dt
    cores = os.cpu_count()
    sample = (f"each step: oracle F + exact gradient + update on the first {Ns} of {s.N} slices "
              f"(all blocks), scaled by {Ns}/{s.N}")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": name},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# --------------------------------------------------------------------------- workloads
class D10:
    """The D_10 XXZ ring, all irrep blocks (default)."""
    name = WORKLOAD
    problems = 1
    prec = "f32"
    step_kw = dict(step=EPS, rule="fixed")
    key = "d10"
    default_steps = 300

    def build(self, api, dev):
        s, psi0_full, psif_full, u0 = workload()
        B = api.Basis(s)
        b0, bf = B.state_to_blocks(psi0_full), B.state_to_blocks(psif_full)
        plan = api.Plan(B, s.N, s.tau, prec=self.prec, active=B.active_copies(b0, bf))
        self._s, self._p0, self._pf, self._u = s, psi0_full, psif_full, u0
        return plan, u0, b0, bf

    def sweep_bytes(self, plan):
        # FP32 complex propagators (8 B per element), read by the forward and the backward sweep
        return 2 * 8 * plan.export_elems()

    def cpu_rate(self):
        Ns = 250
        rate, secs = cpu_oracle_rate(self._s, self._p0, self._pf, self._u, Ns)
        return rate, (f"one FP64 oracle F + exact gradient over the first {Ns} of {self._s.N} slices "
                      f"(all blocks, numpy/BLAS default threads), {secs:.1f} s, scaled by {Ns}/{self._s.N}")


class SnBatch:
    """256 independent S_n problems per launch (batched many-problem solve)."""
    name = SN_WORKLOAD
    problems = SN_BATCH
    # FP64: at T = 10 slice norms reach |tau H| ~ 200, where an FP32 polynomial leaves ~1e-3 in the
    # final states (the parity bound is met in FP64 only)
    prec = "f64"
    step_kw = dict(step=0.02, rule="fixed")
    key = "sn-batch"
    default_steps = 3

    def build(self, api, dev):
        probs = sn_batch_problems(self.problems)
        self._probs = probs
        systems = [I.sn_allpairs(p.n, p.J, p.h, SN_T, p.N) for p in probs]
        bases = [api.Basis(s, first_block_only=True, vectors=False) for s in systems]
        b0 = np.concatenate([bb.dicke_state(0) for bb in bases])
        bf = np.concatenate([bb.dicke_state(p.k_target) for bb, p in zip(bases, probs)])
        u0 = np.concatenate([I.pulses_uniform(p.seed, p.N, 2) for p in probs])
        plan = api.Plan(bases, [p.N for p in probs], [SN_T / p.N for p in probs], prec=self.prec)
        if self.prec == "f64":
            plan.set_persistent(True)  # one cooperative launch per GRAPE iteration
        return plan, u0, b0, bf

    def sweep_bytes(self, plan):
        return 2 * 8 * sum(p.N * (p.n + 1) ** 2 for p in self._probs)

    def cpu_rate(self):
        from oracle import grape as gr
        from oracle import symmetry as sy
        sample = self._probs[:8]
        t0 = time.perf_counter()
        for p in sample:
            Jz, Jp, Jm = sy.spin_matrices(p.n)
            m = p.n + 1
            p0 = np.zeros((m, 1), complex)
            p0[0] = 1
            pf = np.zeros((m, 1), complex)
            pf[p.k_target] = 1
            prob = [dict(h0=p.J * (2 * Jz @ Jz - p.n / 2 * np.eye(m)) + p.h * 2 * Jz, hc=[Jp + Jm, -1j * (Jp - Jm)],
                         psi0=p0, psif=pf)]
            gr.fidelity_and_grad(prob, I.pulses_uniform(p.seed, p.N, 2), SN_T / p.N)
        secs = time.perf_counter() - t0
        return len(sample) / secs, (f"FP64 oracle F + exact gradient of the first {len(sample)} of the "
                                    f"{SN_BATCH} problems ({secs:.1f} s), problems per second")


D14_N, D14_T = 2000, 40.0
D14_WORKLOAD = (f"D_14 XXZ ring (n=14, T={D14_T:g}, N={D14_N}, 3 controls), seeded random states: all 10 D_14 "
                "irrep blocks active (A1 687, A2 495, B1 613, B2 549, E1-E6 1161/1179 x2 copies); sqrt(N) "
                "checkpoint segments (45 slices), the costate pass recomputes each segment")


def d14_workload():
    s = I.xxz_ring(14, D14_T, D14_N)
    psi0 = I.random_state(SEED_PSI0, 2 ** s.n)
    psif = I.random_state(SEED_PSIF, 2 ** s.n)
    u0 = I.pulses_normal(SEED_U, s.N, s.n_ctrl)
    return s, psi0, psif, u0


class D14:
    """The D_14 XXZ ring with sqrt(N) checkpointing (adjoint + recomputation)."""
    name = D14_WORKLOAD
    problems = 1
    prec = "f32"
    step_kw = dict(step=EPS, rule="fixed")
    ckpt = True
    key = "d14"
    default_steps = 4
    e2e_steps = 2
    long_step = True   # a step of seconds: the sustained tensor peak applies

    def build(self, api, dev):
        s, psi0, psif, u0 = d14_workload()
        B = api.Basis(s)
        b0, bf = B.state_to_blocks(psi0), B.state_to_blocks(psif)
        plan = api.Plan(B, s.N, s.tau, prec=self.prec, active=B.active_copies(b0, bf), ckpt_segment=-1)
        self._s, self._p0, self._pf, self._u = s, psi0, psif, u0
        return plan, u0, b0, bf

    def sweep_bytes(self, plan):
        # FP32 complex propagators, read three times: the first pass's forward sweep, and in the costate
        # pass each segment's forward re-sweep (from its checkpoint) and its backward sweep
        return 3 * 8 * plan.export_elems()

    def cpu_rate(self):
        Ns = 4  # about 15 s of oracle work on 16 host cores
        rate, secs = cpu_oracle_rate(self._s, self._p0, self._pf, self._u, Ns)
        return rate, (f"one FP64 oracle F + exact gradient over the first {Ns} of {self._s.N} slices "
                      f"(all blocks, numpy/BLAS default threads; block set-up not timed), {secs:.1f} s, "
                      f"scaled by {Ns}/{self._s.N}")


WS_T = 4.0
WS_TRAIN, WS_HELD = 20000, 1024


def run_warmstart(args, rank, world):
    """Learned warm start: train on GRAPE-optimised pulses, then time-to-F>=0.999 on held-out problems
    for network + batched GRAPE (with plain-GRAPE fallback) versus batched GRAPE from random pulses."""
    if rank != 0:
        return
    import torch
    from paper_2309_05884_gb300 import warmstart as ws
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    X, Y, kept, gen_s = ws.generate_dataset(args.ws_train, 100_000, N=200, T=WS_T, iters=600, lr=0.05, init_seed=0)
    net = ws.WarmStartMLP(seed=0)
    t1 = time.perf_counter()
    hist = net.fit(X, Y, epochs=400, batch=256, lr=1e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    held = I.sn_problem_batch(args.ws_held, base_seed=900_000, n_lo=8, n_hi=32, N_lo=200, N_hi=200)
    with ClockSampler(0) as clk:
        ev = ws.evaluate(net, held, T=WS_T, cap=5000, warm_budget=300, lr=0.05)
    print(json.dumps({
        "metric": "time-to-F>=0.999 (learned warm start + batched GRAPE)", "value": ev["warm"]["seconds"],
        "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64/f64 (GRAPE), bf16/f32 (network)", "data": "synthetic",
        "config": {"workload": f"{args.ws_held} held-out S_n problems (seeds 900000+), n ~ U{{8..32}}, N = 200, "
                               f"T = {WS_T}, |0...0> -> D(n,k); network 4-256-256-256-400 GELU trained on "
                               f"{len(kept)} pulses optimised from one shared U[-1,1] start (seeds 100000+)",
                   "optimizer": "Adam ascent, step 0.05; warm budget 300 iterations then plain fallback; cap 5000"},
        "plain_grape": ev["plain"], "warm_start": ev["warm"], "speedup_wall": ev["speedup_wall"],
        "training": {"examples": len(kept), "generation_s": gen_s, "train_s": train_s, "final_mse": hist[-1],
                     "total_s": time.perf_counter() - t0},
        "clocks": clk.summary(),
    }), flush=True)


WORKLOADS = {"d10": D10, "d14": D14, "sn-batch": SnBatch, "warmstart": None}


# --------------------------------------------------------------------------- replicas
def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over all ranks (every rank gets it); x itself on one rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, problems: int, steps: int, total_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return world * problems * steps / (total_ms / 1e3)


# --------------------------------------------------------------------------- GPU leg
def run_ours(args, rank, world):
    import torch
    from paper_2309_05884_gb300 import api

    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    wl = WORKLOADS[args.workload]()
    if args.prec != "default":
        wl.prec = args.prec
    if args.sn_problems and args.workload == "sn-batch":
        wl.problems = args.sn_problems
    plan, u0, b0, bf = wl.build(api, dev)
    if args.ncu:
        # profiling mode: one GRAPE step and nothing else (no warm-up, timing, copies or CPU leg), so
        # that a launch list or a capture covers exactly one step; its output is not a bench line
        u = torch.from_numpy(u0.copy()).to(dev)
        plan.optimize(u, api.to_device(b0, dev), api.to_device(bf, dev), iters=1, **wl.step_kw)
        torch.cuda.synchronize()
        plan.sync_status()
        if rank == 0:
            launches = plan.kernel_launches(True)
            print(json.dumps({"ncu_profile_step": wl.name, "launches": launches + (0 if launches == 1 else 2)}),
                  flush=True)
        return
    if args.deriv != "default":
        mode, min_m = {"off": (0, 0), "cuda": (1, 129), "tc": (2, 129), "tc-all": (2, 24)}[args.deriv]
        plan.set_deriv_gemm(mode, min_m)
    if args.expm_kernel == "tc":
        plan.set_expm_rules([(112, 2, 0)])      # tcgen05 tensor cores where the block fits
    elif args.expm_kernel == "tiled":
        plan.set_expm_rules([(1 << 30, 0, 0)])
    if args.autotune:
        from paper_2309_05884_gb300 import autotune
        autotune.tune(plan, torch.from_numpy(u0).to(dev), api.to_device(b0, dev), api.to_device(bf, dev),
                      cache_path=os.path.join(tempfile.gettempdir(), "qoc_autotune.json"))
    d0, df = api.to_device(b0, dev), api.to_device(bf, dev)
    u = torch.from_numpy(u0.copy()).to(dev)
    ws = plan.workspace  # allocate before timing
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def step():
        plan.optimize(u, d0, df, iters=1, **wl.step_kw)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    plan.sync_status()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # timed region: K steps, each bracketed by events on the launching stream, L2 flushed between
    plan.set_profiling(True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    phases = []
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
            phases.append(plan.phase_times())
        torch.cuda.synchronize()
        barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    counts = plan.work_counts()
    plan.set_profiling(False)
    plan.sync_status()
    total_ms = max_over_ranks(float(np.sum(step_ms)), world, dev)
    value = job_rate(world, wl.problems, args.steps, total_ms)
    ph = np.mean(np.array(phases), axis=0)

    # rooflines per phase, from algorithmic work per call (complex multiply-add = 8 flop) and the
    # in-step CUDA-event phase times (each the sum of that phase's launch durations on the launching
    # stream); the line's "roofline" is the phase that takes longest
    peaks = measured_peaks(getattr(wl, "long_step", False))
    n = args.steps
    phase_ms = {"expm": float(ph[0]), "sweeps": float(ph[1]), "overlap": float(ph[2]),
                "slice_derivatives": float(ph[3]), "reduce_update": float(ph[4])}
    classes = plan.expm_classes()
    kinds = {c[0] for c in classes}
    ckpt = getattr(wl, "ckpt", False)
    expm_flop = 8.0 * (counts[0] + counts[1]) / n   # both passes when checkpointing
    roofs = {}
    if kinds & {2, 3}:
        # kind::f16 MMAs: the measured BF16 dense rate (FP16 has the same nominal rate)
        tc_peak, tc_src = peaks["tensor_tflops"], peaks["tensor_note"]
        kern = ("xl_gemm_kernel (tcgen05 128 x 128 tiles, pre-split FP16 plane slabs)" if 3 in kinds
                else "expm_tc_kernel (tcgen05, FP16 hi/lo split)")
        roofs["expm"] = {"bound": "tensor", "kernel": kern,
                         "achieved": expm_flop / (phase_ms["expm"] * 1e-3) / 1e12, "peak": tc_peak,
                         "unit": "TFLOP/s", "peak_source": tc_src,
                         "flops_per_step": expm_flop,
                         "note": "algorithmic complex-FP32 flop (8 m^3 per product; a Hermitian product of the "
                                 "large-block path, formed on the upper tiles and mirrored, counts as half) over "
                                 "the summed durations of the exponential launches; the split issues 16 real FP16 "
                                 "products per complex product (12 where lo*lo is left out) on padded operands"
                                 + ("; checkpointed: every exponential is computed twice (forward pass and "
                                    "costate pass), both counted" if ckpt else "")}
        # a complex product is 4 real products of 4 (or, without lo*lo, 3) split FP16 products each:
        # 32 m^3 (24 m^3) tensor flop per 8 m^3 algorithmic, so a kernel that kept the tensor pipe busy
        # all the time would reach 1/4 (1/3) of the peak in these algorithmic units
        prods = counts[0] + counts[1]
        three = min(counts[5], prods)
        ratio = 8.0 * prods / (32.0 * (prods - three) + 24.0 * three) if prods else 0.25
        roofs["expm"]["split_ceiling"] = {
            "peak": tc_peak * ratio, "frac": roofs["expm"]["achieved"] / (tc_peak * ratio),
            "three_term_share": three / prods if prods else 0.0,
            "note": "algorithmic rate of a split-FP16 kernel with the tensor pipe always busy, for this "
                    "step's mix of four-term and three-term products"}
    else:
        f64 = wl.prec == "f64"
        roofs["expm"] = {"bound": "alu", "kernel": "expm_kernel (CUDA-core tiles, %s)" % ("FP64" if f64 else "FP32"),
                         "achieved": expm_flop / (phase_ms["expm"] * 1e-3) / 1e12,
                         "peak": FP64_PEAK_TFLOPS if f64 else FP32_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "peak_source": FP64_PEAK_NOTE if f64 else FP32_PEAK_NOTE,
                         "flops_per_step": expm_flop}
    grad_flop = 8.0 * counts[3] / n
    if grad_flop > 0:
        roofs["slice_derivatives"] = {
            "bound": "alu", "kernel": "grad_fast_kernel (register tiles, FP32 FMA)",
            "achieved": grad_flop / (phase_ms["slice_derivatives"] * 1e-3) / 1e12, "peak": FP32_PEAK_TFLOPS,
            "unit": "TFLOP/s", "peak_source": FP32_PEAK_NOTE, "flops_per_step": grad_flop,
            "note": "series work (c (3P+1) + n_ctrl) m^2 complex multiply-adds per (slice, block) item"}
    gemm_flop = 8.0 * counts[4] / n
    if gemm_flop > 0 and "slice_derivatives" not in roofs:
        tc = args.deriv != "cuda"  # the plans' default derivative GEMM runs on the tensor cores
        roofs["slice_derivatives"] = {
            "bound": "tensor" if tc else "alu",
            "kernel": "gg_tc_kernel (tall GEMMs [H0; Hc_j] X on tcgen05, split FP16)" if tc
            else "gg_gemm_kernel (tall GEMMs on CUDA cores)",
            "achieved": gemm_flop / (phase_ms["slice_derivatives"] * 1e-3) / 1e12,
            "peak": peaks["tensor_tflops"] if tc else FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "peak_source": peaks["tensor_note"] if tc else FP32_PEAK_NOTE, "flops_per_step": gemm_flop,
            "note": "series work per (slice, block) item: (1 + n_ctrl) m^2 2c (P + 1) complex multiply-adds for the "
                    "chains, c n_ctrl m (P + 1)(P + 2) / 2 for the contraction; the tensor-core GEMM issues 12 real "
                    "FP16 products (three split terms) per complex multiply-add, so 1/3 of the peak is its ceiling"}
    sweep_bytes = wl.sweep_bytes(plan)
    if sweep_bytes:
        roofs["sweeps"] = {"bound": "hbm", "kernel": "sweep_cluster_kernel" if plan.sweep_cluster() else "sweep_kernel",
                           "achieved": sweep_bytes / (phase_ms["sweeps"] * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                           "unit": "GB/s", "peak_source": peaks["hbm_note"], "bytes_per_step": sweep_bytes,
                           "note": "every stored propagator read once forward and once backward"}
    for r in roofs.values():
        r["frac"] = r["achieved"] / r["peak"]
        r["traffic"] = None
    tr = NCU_TRAFFIC.get(getattr(wl, "key", ""))
    if tr and "expm" in roofs and roofs["expm"]["kernel"].startswith(tr["kernel"]):
        roofs["expm"]["traffic"] = tr["bytes"]
        roofs["expm"]["traffic_launch"] = {k: tr[k] for k in ("launch", "algorithmic_bytes", "source")}
    dominant = max((k for k in roofs), key=lambda k: phase_ms[k])
    roof = dict(roofs[dominant])
    roof["phase"] = dominant
    roof["phase_ms"] = phase_ms

    # end to end through the C ABI with host buffers: H2D of u and both states, D2H of F and dF/du
    u_h = torch.from_numpy(u0.copy()).pin_memory()
    b0_h = torch.from_numpy(b0).pin_memory()
    bf_h = torch.from_numpy(bf).pin_memory()
    out_h = torch.empty(3 * plan.n_prob, dtype=torch.float64).pin_memory()
    g_h = torch.empty_like(u_h).pin_memory()
    u_d, d0e, dfe = torch.empty_like(u), torch.empty_like(d0), torch.empty_like(df)
    out3 = torch.empty(3 * plan.n_prob, dtype=torch.float64, device=dev)
    gd = torch.empty_like(u)
    e2e_steps = getattr(wl, "e2e_steps", None) or max(3, args.steps // 2)
    lr = wl.step_kw["step"]
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        u_d.copy_(u_h, non_blocking=True)
        d0e.copy_(b0_h, non_blocking=True)
        dfe.copy_(bf_h, non_blocking=True)
        plan.fidelity_and_grad(u_d, d0e, dfe, out3=out3, grad=gd)
        out_h.copy_(out3, non_blocking=True)
        g_h.copy_(gd, non_blocking=True)
        torch.cuda.synchronize()
        u_h += lr * g_h
    e2e_s = time.perf_counter() - t0
    h2d = u_h.numel() * 8 + b0_h.numel() * 16 + bf_h.numel() * 16
    d2h = out_h.numel() * 8 + g_h.numel() * 8

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, sample = wl.cpu_rate()
        cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle", "sample": sample}

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128" if wl.prec == "f64" else "c64/f64", "data": "synthetic",
            "config": {"workload": wl.name, "precision": {"f32": "complex FP32 polynomial + sweeps; FP64 squaring, "
                                                                  "overlap, gradient accumulation",
                                                           "f32_all": "complex FP32 polynomial, squaring and sweeps; "
                                                                      "FP64 overlap and gradient accumulation",
                                                           "f64": "complex FP64 throughout"}[wl.prec],
                       "problems_per_step": wl.problems, "l2": "flushed between timed steps (256 MB write)",
                       "expm_kernels": [list(c) for c in plan.expm_classes()],
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roof,
            "rooflines": roofs,
            "cpu_baseline": cpu,
            "e2e": {"value": world * wl.problems * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            # per step: the plan's launches, plus (multi-launch path) the norm check and the iteration counter
            "gpu_launches": (plan.kernel_launches(True) + (0 if plan.kernel_launches(True) == 1 else 2)) * args.steps,
            "clocks": clk.summary(),
        }), flush=True)


def build_parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default: the workload's)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="d14")
    ap.add_argument("--prec", choices=["default", "f64", "f32", "f32_all"], default="default",
                    help="override the workload's precision")
    ap.add_argument("--deriv", choices=["default", "off", "cuda", "tc", "tc-all"], default="default",
                    help="slice-derivative path: per-slice series (off), tall GEMMs on CUDA cores or tensor cores for "
                         "blocks above 128 states, or tensor cores for every block of 24 states or more")
    ap.add_argument("--autotune", action="store_true",
                    help="tune the exponential, sweep and derivative kernels before timing")
    ap.add_argument("--ncu", action="store_true",
                    help="profiling mode: run one step of the workload and exit (for ncu launch lists and captures)")
    ap.add_argument("--sn-problems", type=int, default=0, help="problems of the sn-batch workload (default 256)")
    ap.add_argument("--expm-kernel", choices=["default", "tiled", "tc"], default="default",
                    help="force the exponential kernel: tiled CUDA-core or tcgen05 tensor-core")
    ap.add_argument("--ws-train", type=int, default=WS_TRAIN, help="warm-start training problems")
    ap.add_argument("--ws-held", type=int, default=WS_HELD, help="warm-start held-out problems")
    return ap


def main():
    args = build_parser().parse_args()
    if args.steps is None:
        wl_cls = WORKLOADS.get(args.workload)
        args.steps = wl_cls.default_steps if wl_cls is not None else 1
    args.warmup = max(args.warmup, 3) if args.impl == "ours" and not args.ncu else args.warmup
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "warmstart":
        run_warmstart(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
