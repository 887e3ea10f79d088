"""Autotuner for the batched exponentials: per block-size bucket, time the candidate kernels (tiled
CTA kernel with register tiles R, or the warp-packed kernel with 1..32/MP matrices per warp) on
the plan's real work and keep the fastest, then cache the choice per GPU, precision and bucket.

The timing is the device time of the exponential phase of qoc_fidelity_and_grad (CUDA events the
library records on the call's stream), median of a few repetitions.
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
    if prec != "f64" and m_max <= 112:
        out.append((2, 0))  # tcgen05 tensor cores
    warp_ok = prec != "f32" and m_max <= (16 if prec == "f64" else 32)
    if warp_ok:
        mp = 8 if m_max <= 8 else 16 if m_max <= 16 else 32
        out += [(1, w) for w in sorted({1, max(1, 32 // mp // 2), 32 // mp})]
    return out


def _time_expm(plan, u, psi0, psif, reps: int) -> float:
    plan.set_profiling(True)
    times = []
    for _ in range(reps + 1):
        plan.fidelity_and_grad(u, psi0, psif, want_grad=False)
        times.append(plan.phase_times()[0])
    plan.set_profiling(False)
    plan.sync_status()
    times = sorted(times[1:])
    return times[len(times) // 2]


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
