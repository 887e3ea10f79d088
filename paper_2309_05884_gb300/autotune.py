"""Autotuner for a plan's kernel choices, timed on the plan's real work and cached per GPU, precision
and block sizes:
  - exponentials, per block-size bucket: tiled CTA kernel with register tiles R, warp-packed kernel
    with 1..32/MP matrices per warp, tcgen05 kernel one CTA per slice (unsquared slices or all), tiled
    tcgen05 GEMMs for large blocks;
  - sweeps: one CTA per chain or thread-block clusters of 2..8 CTAs;
  - slice derivatives: the per-slice series kernels, or tall GEMMs shared by a chunk's slices (FP32
    CUDA cores or tensor cores) for the blocks above a size threshold.
Each choice is timed by the device time of its own phase of qoc_fidelity_and_grad (CUDA events the
library records around that phase's launches), median of a few repetitions; the choices are made in
that order, each with the earlier ones applied.
"""
from __future__ import annotations

import json
import os
from typing import Dict, List, Optional, Tuple

import torch

Rule = Tuple[int, int, int]  # (m_max, kind, param)


def _buckets(plan) -> List[int]:
    return sorted({c[3] for c in plan.expm_classes()})


def _block_sizes(plan) -> List[int]:
    """Sizes of the plan's active blocks (independent of the current kernel rules)."""
    out = set()
    for basis, act in zip(plan.bases, plan._acts):
        i = 0
        for _, m, c, _ in basis.blocks:
            if act is None or act[i:i + c].any():
                out.add(m)
            i += c
    return sorted(out)


def _candidates(m_max: int, prec: str) -> List[Tuple[int, int]]:
    rmax = 4 if prec == "f64" else 7
    r0 = max(1, min(rmax, -(-m_max // 16)))
    out = [(0, r) for r in sorted({max(1, r0 - 1), r0, min(rmax, r0 + 1)})]
    if prec == "f32" and m_max <= 112:
        out += [(2, 0), (2, 1)]  # tcgen05, one CTA per slice: unsquared slices / every slice
    if prec == "f32" and 24 < m_max <= 2048:
        out.append((3, 0))  # tiled tcgen05 GEMMs
    warp_ok = prec != "f32" and m_max <= (16 if prec == "f64" else 32)
    if warp_ok:
        mp = 8 if m_max <= 8 else 16 if m_max <= 16 else 32
        out += [(1, w) for w in sorted({1, max(1, 32 // mp // 2), 32 // mp})]
    return out


def _time_phase(plan, u, psi0, psif, reps: int, phase: int, want_grad: bool) -> float:
    plan.set_profiling(True)
    times = []
    for _ in range(reps + 1):
        plan.fidelity_and_grad(u, psi0, psif, want_grad=want_grad)
        times.append(plan.phase_times()[phase])
    plan.set_profiling(False)
    plan.sync_status()
    times = sorted(times[1:])
    return times[len(times) // 2]


def _time_expm(plan, u, psi0, psif, reps: int) -> float:
    return _time_phase(plan, u, psi0, psif, reps, 0, False)


def tune_expm(plan, u: torch.Tensor, psi0: torch.Tensor, psif: torch.Tensor, reps: int = 3,
              cache_path: Optional[str] = None) -> Dict:
    """Greedy per-bucket search; applies the best rules to the plan and returns a report."""
    key = f"{torch.cuda.get_device_name()}|{plan.prec}|" + ",".join(map(str, _block_sizes(plan)))
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    if key in cache:
        rules = [tuple(r) for r in cache[key]["rules"]]
        plan.set_expm_rules(rules)
        return dict(cache[key], cached=True)
    plan.set_expm_rules([(1 << 30, 0, 0)])  # the default rules (tiled kernels by size)
    buckets = _buckets(plan)
    chosen: Dict[int, Tuple[int, int]] = {}
    report = []
    base = _time_expm(plan, u, psi0, psif, reps)
    for b in buckets:
        best = None
        for cand in _candidates(b, plan.prec):
            rules = [(bb, *chosen[bb]) for bb in buckets if bb in chosen] + [(b, *cand)]
            plan.set_expm_rules(rules)
            t = _time_expm(plan, u, psi0, psif, reps)
            report.append({"bucket": b, "kind": cand[0], "param": cand[1], "ms": t})
            if best is None or t < best[0]:
                best = (t, cand)
        chosen[b] = best[1]
    rules: List[Rule] = [(b, *chosen[b]) for b in buckets]
    plan.set_expm_rules(rules)
    tuned = _time_expm(plan, u, psi0, psif, reps)
    out = {"rules": rules, "default_ms": base, "tuned_ms": tuned, "trials": report, "cached": False}
    if cache_path:
        cache[key] = {k: v for k, v in out.items() if k != "cached"}
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return out


def _cached(cache_path, key):
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            return json.load(f).get(key)
    return None


def _store(cache_path, key, value):
    if not cache_path:
        return
    cache = {}
    if os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    cache[key] = value
    with open(cache_path, "w") as f:
        json.dump(cache, f, indent=1)


def tune_sweeps(plan, u: torch.Tensor, psi0: torch.Tensor, psif: torch.Tensor, reps: int = 3,
                cache_path: Optional[str] = None) -> Dict:
    """Cluster size of the forward/backward sweeps (0 = one CTA per chain), timed on the sweep phase."""
    key = f"sweeps|{torch.cuda.get_device_name()}|{plan.prec}|{plan.n_prob}|" + ",".join(map(str, _block_sizes(plan)))
    hit = _cached(cache_path, key)
    if hit is not None:
        plan.set_sweep_cluster(hit["cl"])
        return dict(hit, cached=True)
    trials = []
    for cl in (0, 2, 3, 4, 6, 8):
        try:
            plan.set_sweep_cluster(cl)
        except RuntimeError:
            continue  # the cluster's buffers do not fit
        trials.append({"cl": cl, "ms": _time_phase(plan, u, psi0, psif, reps, 1, True)})
    best = min(trials, key=lambda t: t["ms"])
    plan.set_sweep_cluster(best["cl"])
    out = {"cl": best["cl"], "trials": trials}
    _store(cache_path, key, out)
    return dict(out, cached=False)


def tune_derivatives(plan, u: torch.Tensor, psi0: torch.Tensor, psif: torch.Tensor, reps: int = 3,
                     cache_path: Optional[str] = None) -> Dict:
    """Slice-derivative path: per-slice series kernels, or tall GEMMs (FP32 CUDA cores or tensor cores)
    for the blocks above a size threshold, timed on the derivative phase."""
    key = f"deriv|{torch.cuda.get_device_name()}|{plan.prec}|{plan.n_prob}|" + ",".join(map(str, _block_sizes(plan)))
    hit = _cached(cache_path, key)
    if hit is not None:
        plan.set_deriv_gemm(hit["mode"], hit["min_m"])
        return dict(hit, cached=True)
    trials = []
    for mode, min_m in ((0, 129), (1, 129), (2, 129), (2, 24)):
        plan.set_deriv_gemm(mode, min_m)
        if mode and plan.deriv_gemm_blocks() == 0:
            continue  # no block that large: same as off
        trials.append({"mode": mode, "min_m": min_m, "ms": _time_phase(plan, u, psi0, psif, reps, 3, True)})
    best = min(trials, key=lambda t: t["ms"])
    plan.set_deriv_gemm(best["mode"], best["min_m"])
    out = {"mode": best["mode"], "min_m": best["min_m"], "trials": trials}
    _store(cache_path, key, out)
    return dict(out, cached=False)


def tune(plan, u: torch.Tensor, psi0: torch.Tensor, psif: torch.Tensor, reps: int = 3,
         cache_path: Optional[str] = None) -> Dict:
    """Every choice in turn: exponentials, sweeps, derivatives.  The plan's workspace size may change
    (the Python Plan reallocates it)."""
    return {"expm": tune_expm(plan, u, psi0, psif, reps, cache_path),
            "sweeps": tune_sweeps(plan, u, psi0, psif, reps, cache_path),
            "derivatives": tune_derivatives(plan, u, psi0, psif, reps, cache_path)}
