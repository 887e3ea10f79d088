"""Python binding of libqoc (include/qoc.h): Basis, Plan and the autograd wrapper.

Argument marshalling only: every step of the hot path runs in the library's CUDA kernels; torch
supplies device memory and streams.  Complex device buffers are torch.complex128 tensors (the
interleaved (re, im) double layout of the C ABI).
"""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Tuple

import numpy as np
import torch

from . import _lib as L


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


class Basis:
    """Symmetry-adapted block decomposition of H0 and the Hc_j (Appendix A); built on the host once.

    system: an object with fields n, group, h0 (list of (kind, coeff, dist)), hc (list of such lists)
    such as paper_2309_05884_gb300.inputs.System."""

    def __init__(self, system, first_block_only: bool = False, vectors: bool = True):
        self.lib = L.load()
        self.system = system
        h0 = (L.qoc_term * max(1, len(system.h0)))(*[L.qoc_term(k, d, c) for k, c, d in system.h0])
        hcs = [(L.qoc_term * len(t))(*[L.qoc_term(k, d, c) for k, c, d in t]) for t in system.hc]
        n_hc = (C.c_int * len(hcs))(*[len(t) for t in system.hc])
        hc_ptrs = (C.POINTER(L.qoc_term) * len(hcs))(*[C.cast(a, C.POINTER(L.qoc_term)) for a in hcs])
        desc = L.qoc_system_desc(system.n, system.group, len(system.h0), C.cast(h0, C.POINTER(L.qoc_term)),
                                 len(hcs), C.cast(n_hc, C.POINTER(C.c_int)),
                                 C.cast(hc_ptrs, C.POINTER(C.POINTER(L.qoc_term))))
        flags = (L.QOC_BASIS_FIRST_BLOCK_ONLY if first_block_only else 0) | (0 if vectors else L.QOC_BASIS_NO_VECTORS)
        h = C.c_void_p()
        L.check(self.lib.qoc_build_symmetry_basis(C.byref(desc), flags, C.byref(h)), "qoc_build_symmetry_basis")
        self.handle = h
        nb, nc, sl, fd = C.c_int(), C.c_int(), C.c_int64(), C.c_int64()
        L.check(self.lib.qoc_basis_info(h, C.byref(nb), C.byref(nc), C.byref(sl), C.byref(fd)), "qoc_basis_info")
        self.n_blocks, self.n_ctrl, self.state_len, self.full_dim = nb.value, nc.value, sl.value, fd.value
        self.blocks: List[Tuple[str, int, int, int]] = []
        for b in range(self.n_blocks):
            m, c, off = C.c_int(), C.c_int(), C.c_int64()
            lab = C.create_string_buffer(16)
            L.check(self.lib.qoc_basis_block(h, b, C.byref(m), C.byref(c), C.byref(off), lab), "qoc_basis_block")
            self.blocks.append((lab.value.decode(), m.value, c.value, off.value))

    def __del__(self):
        if getattr(self, "handle", None):
            self.lib.qoc_basis_free(self.handle)
            self.handle = None

    @property
    def n_copies(self) -> int:
        return sum(c for _, _, c, _ in self.blocks)

    def block_matrices(self, b: int):
        _, m, _, _ = self.blocks[b]
        h0 = np.zeros((m, m), np.complex128)
        hc = np.zeros((self.n_ctrl, m, m), np.complex128)
        L.check(self.lib.qoc_basis_block_matrices(self.handle, b, h0.ctypes.data_as(C.c_void_p),
                                                  hc.ctypes.data_as(C.c_void_p)), "qoc_basis_block_matrices")
        return h0, hc

    def norm_bounds(self, b: int) -> np.ndarray:
        """[bound of |H0_b|_2, bound of |Hc_jb|_2 for each j]: what the slice norm bound is built from."""
        out = np.zeros(1 + self.n_ctrl, np.float64)
        L.check(self.lib.qoc_basis_norm_bounds(self.handle, b, out.ctypes.data_as(C.c_void_p)),
                "qoc_basis_norm_bounds")
        return out

    def state_to_blocks(self, full: np.ndarray) -> np.ndarray:
        full = np.ascontiguousarray(full, dtype=np.complex128)
        assert full.shape == (self.full_dim,)
        out = np.zeros(self.state_len, np.complex128)
        L.check(self.lib.qoc_state_to_blocks(self.handle, full.ctypes.data_as(C.c_void_p),
                                             out.ctypes.data_as(C.c_void_p)), "qoc_state_to_blocks")
        return out

    def blocks_to_state(self, blk: np.ndarray) -> np.ndarray:
        blk = np.ascontiguousarray(blk, dtype=np.complex128)
        out = np.zeros(self.full_dim, np.complex128)
        L.check(self.lib.qoc_blocks_to_state(self.handle, blk.ctypes.data_as(C.c_void_p),
                                             out.ctypes.data_as(C.c_void_p)), "qoc_blocks_to_state")
        return out

    def dicke_state(self, k: int) -> np.ndarray:
        out = np.zeros(self.state_len, np.complex128)
        L.check(self.lib.qoc_dicke_state(self.handle, k, out.ctypes.data_as(C.c_void_p)), "qoc_dicke_state")
        return out

    def copy_norms(self, blk: np.ndarray) -> np.ndarray:
        """2-norm of every block copy of a block state, in block-state order."""
        out = []
        for _, m, c, off in self.blocks:
            for r in range(c):
                out.append(np.linalg.norm(blk[off + r * m: off + (r + 1) * m]))
        return np.array(out)

    def gate_blocks(self, W: np.ndarray, tol: float = 1e-10) -> List[np.ndarray]:
        """W_b = V_b^dagger W V_b (copy 0) of a full-space gate W that commutes with the symmetry group;
        raises if W mixes blocks (it is then not a symmetric gate)."""
        W = np.asarray(W, dtype=np.complex128)
        assert W.shape == (self.full_dim, self.full_dim)
        out = []
        for b, (_, m, c, off) in enumerate(self.blocks):
            Wb = np.zeros((m, m), np.complex128)
            for a in range(m):
                e = np.zeros(self.state_len, np.complex128)
                e[off + a] = 1.0
                col = self.state_to_blocks(W @ self.blocks_to_state(e))
                Wb[:, a] = col[off: off + m]
                col[off: off + m] = 0
                if np.abs(col).max(initial=0.0) > tol:
                    raise ValueError("the gate mixes symmetry blocks (it does not commute with the group)")
            out.append(Wb)
        return out

    def active_copies(self, psi0_blk: np.ndarray, psif_blk: np.ndarray, tol: float = 1e-13) -> np.ndarray:
        """Copies with support in both states (only those can contribute to <psi_f|psi_N>)."""
        return ((self.copy_norms(psi0_blk) > tol) & (self.copy_norms(psif_blk) > tol)).astype(np.uint8)


class Plan:
    """A GPU plan: one problem (basis, N slices of length dt, active copies) or a batch of them that
    run together in every launch.  Batched device buffers concatenate the problems in order."""

    PRECS = {"f64": L.QOC_PREC_F64, "f32": L.QOC_PREC_F32, "f32_all": L.QOC_PREC_F32_ALL}

    def __init__(self, basis, N, dt, prec: str = "f64", grad_mode: int = 0, active=None,
                 max_squarings: int = 16, ckpt_segment: int = 0, device=None, objective: str = "state"):
        self.lib = L.load()
        batch = not isinstance(basis, Basis)
        self.bases = list(basis) if batch else [basis]
        self.basis = self.bases[0]
        n = len(self.bases)
        Ns = list(N) if batch else [N]
        dts = list(dt) if batch else [dt]
        acts = (list(active) if active is not None else [None] * n) if batch else [active]
        self.N, self.dt = (Ns[0], dts[0]) if not batch else (Ns, dts)
        self.Ns, self.dts = Ns, dts
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        opts = L.qoc_plan_opts()
        self.lib.qoc_plan_opts_default(C.byref(opts))
        opts.prec = self.PRECS[prec]
        opts.grad_mode = grad_mode
        opts.max_squarings = max_squarings
        opts.ckpt_segment = ckpt_segment
        opts.objective = {"state": L.QOC_OBJ_STATE, "gate": L.QOC_OBJ_GATE}[objective]
        self.objective = objective
        self.prec = prec
        self._acts = [None if a_ is None else np.ascontiguousarray(a_, dtype=np.uint8) for a_ in acts]
        for a_, b_ in zip(self._acts, self.bases):
            assert a_ is None or a_.shape == (b_.n_copies,)
        self._active = self._acts[0]
        act_ptrs = (C.c_void_p * n)(*[None if a_ is None else a_.ctypes.data_as(C.c_void_p).value for a_ in self._acts])
        base_ptrs = (C.c_void_p * n)(*[b_.handle.value for b_ in self.bases])
        Ns_c = (C.c_int * n)(*Ns)
        dts_c = (C.c_double * n)(*dts)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            L.check(self.lib.qoc_plan_create_batch(base_ptrs, n, Ns_c, dts_c, C.byref(opts), act_ptrs, C.byref(h)),
                    "qoc_plan_create_batch")
        self.handle = h
        npb, rows, sl = C.c_int(), C.c_int64(), C.c_int64()
        L.check(self.lib.qoc_plan_info(h, C.byref(npb), C.byref(rows), C.byref(sl)), "qoc_plan_info")
        self.n_prob, self.rows, self.state_len = npb.value, rows.value, sl.value
        nbytes = C.c_size_t()
        L.check(self.lib.qoc_plan_workspace_bytes(h, C.byref(nbytes)), "qoc_plan_workspace_bytes")
        self.workspace_bytes = nbytes.value
        self._ws = None
        self._graph_stream = None
        self.last_reached = None
        self._fwd_serial = 0  # counts forward halves; a backward half must follow its own forward

    def __del__(self):
        if getattr(self, "handle", None):
            self.lib.qoc_plan_free(self.handle)
            self.handle = None

    @property
    def workspace(self) -> torch.Tensor:
        if self._ws is None:
            self._ws = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8, device=self.device)
        return self._ws

    def release_workspace(self):
        self._ws = None

    def _check_u(self, u: torch.Tensor):
        assert u.dtype == torch.float64 and u.is_cuda and u.is_contiguous()
        assert tuple(u.shape) == (self.rows, self.basis.n_ctrl), (tuple(u.shape), (self.rows, self.basis.n_ctrl))

    def _check_state(self, s: torch.Tensor):
        assert s.dtype == torch.complex128 and s.is_cuda and s.is_contiguous()
        assert s.numel() == self.state_len

    def fidelity_and_grad(self, u: torch.Tensor, psi0: torch.Tensor, psif: torch.Tensor, want_grad: bool = True,
                          out3: Optional[torch.Tensor] = None, grad: Optional[torch.Tensor] = None, stream=None):
        """(out3 = [F, Re o, Im o] per problem, grad [rows, nc]) on the device, asynchronously."""
        self._check_u(u)
        self._check_state(psi0)
        self._check_state(psif)
        if out3 is None:
            out3 = torch.empty(3 * self.n_prob, dtype=torch.float64, device=u.device)
        if want_grad and grad is None:
            grad = torch.empty_like(u)
        ws = self.workspace
        L.check(self.lib.qoc_fidelity_and_grad(self.handle, _ptr(u), _ptr(psi0), _ptr(psif), _ptr(out3),
                                               _ptr(grad) if want_grad else None, _ptr(ws), ws.numel(),
                                               _stream(stream)), "qoc_fidelity_and_grad")
        return out3, (grad if want_grad else None)

    def forward(self, u: torch.Tensor, psi0: torch.Tensor, psif: torch.Tensor, out3: Optional[torch.Tensor] = None,
                stream=None) -> Tuple[torch.Tensor, int]:
        """Forward half (qoc_fidelity_forward): out3 = [F, Re o, Im o] per problem and a serial number
        that backward() must be given; the workspace keeps the states backward() needs."""
        self._check_u(u)
        self._check_state(psi0)
        self._check_state(psif)
        if out3 is None:
            out3 = torch.empty(3 * self.n_prob, dtype=torch.float64, device=u.device)
        ws = self.workspace
        L.check(self.lib.qoc_fidelity_forward(self.handle, _ptr(u), _ptr(psi0), _ptr(psif), _ptr(out3), _ptr(ws),
                                              ws.numel(), _stream(stream)), "qoc_fidelity_forward")
        self._fwd_serial += 1
        return out3, self._fwd_serial

    def backward(self, u: torch.Tensor, psif: torch.Tensor, serial: int, gF: Optional[torch.Tensor] = None,
                 grad: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """Backward half (qoc_fidelity_backward): grad = gF_p dF_p/du from the workspace that the forward
        half numbered 'serial' left; raises if another forward half ran on this plan since."""
        if serial != self._fwd_serial:
            raise RuntimeError("the plan's workspace was reused by a later forward pass; run forward again")
        self._check_u(u)
        self._check_state(psif)
        if grad is None:
            grad = torch.empty_like(u)
        if gF is not None:
            assert gF.dtype == torch.float64 and gF.is_cuda and gF.is_contiguous() and gF.numel() == self.n_prob
        ws = self.workspace
        L.check(self.lib.qoc_fidelity_backward(self.handle, _ptr(u), _ptr(psif), _ptr(gF), _ptr(grad), _ptr(ws),
                                               ws.numel(), _stream(stream)), "qoc_fidelity_backward")
        return grad

    def selftest_wait(self, limit_ms: float = 1.0, stream=None) -> None:
        """Launch a bounded wait that nothing completes (qoc_plan_selftest_wait); sync_status() then
        raises QOC_ETIMEOUT."""
        L.check(self.lib.qoc_plan_selftest_wait(self.handle, float(limit_ms), _stream(stream)), "qoc_plan_selftest_wait")

    def propagate(self, u: torch.Tensor, psi0: torch.Tensor, psiN: Optional[torch.Tensor] = None, stream=None):
        self._check_u(u)
        self._check_state(psi0)
        if psiN is None:
            psiN = torch.empty_like(psi0)
        ws = self.workspace
        L.check(self.lib.qoc_propagate(self.handle, _ptr(u), _ptr(psi0), _ptr(psiN), _ptr(ws), ws.numel(),
                                       _stream(stream)), "qoc_propagate")
        return psiN

    def assemble(self, u: torch.Tensor, stream=None) -> torch.Tensor:
        """A[b][k] = -i dt (H0_b + sum_j u_kj Hc_jb), packed block-major over active blocks."""
        self._check_u(u)
        out = torch.empty(self.export_elems(), dtype=torch.complex128, device=u.device)
        L.check(self.lib.qoc_assemble_blocks(self.handle, _ptr(u), _ptr(out), _stream(stream)), "qoc_assemble_blocks")
        return out

    def expm(self, u: torch.Tensor, stream=None) -> torch.Tensor:
        """U[b][k] = exp(A[b][k]) in the layout of assemble()."""
        self._check_u(u)
        out = torch.empty(self.export_elems(), dtype=torch.complex128, device=u.device)
        ws = self.workspace
        L.check(self.lib.qoc_expm_blocks(self.handle, _ptr(u), _ptr(out), _ptr(ws), ws.numel(), _stream(stream)),
                "qoc_expm_blocks")
        return out

    def gate_states(self, W_blocks) -> Tuple[np.ndarray, np.ndarray]:
        """(psi0, psif) block states of a gate plan (one problem): in block b the identity columns and
        the columns of W_b, both weighted by sqrt(c_b / d), d = sum_b c_b m_b."""
        assert self.objective == "gate"
        B = self.basis
        d = sum(c * m for _, m, c, _ in B.blocks)
        psi0, psif = [], []
        for (_, m, c, _), Wb in zip(B.blocks, W_blocks):
            w = np.sqrt(c / d)
            psi0.append((w * np.eye(m, dtype=np.complex128)).T.reshape(-1))   # column r at [r*m, (r+1)*m)
            psif.append((w * np.asarray(Wb, dtype=np.complex128)).T.reshape(-1))
        return np.concatenate(psi0), np.concatenate(psif)

    def active_blocks(self) -> List[int]:
        """Basis indices of blocks with at least one active copy (the export layout's order)."""
        if getattr(self, "_active", None) is None:
            return list(range(self.basis.n_blocks))
        out, i = [], 0
        for b, (_, m, c, off) in enumerate(self.basis.blocks):
            if self._active[i:i + c].any():
                out.append(b)
            i += c
        return out

    def export_elems(self) -> int:
        return sum(self.N * self.basis.blocks[b][1] ** 2 for b in self.active_blocks())

    def optimize(self, u: torch.Tensor, psi0: torch.Tensor, psif: torch.Tensor, iters: int, step: float,
                 f_target: float = 2.0, check_every: int = 10, rule: str = "fixed", beta1: float = 0.9,
                 beta2: float = 0.999, eps: float = 1e-8, use_graph: bool = False, freeze: bool = True,
                 stream=None):
        """GRAPE ascent in place on u.  Returns (F history [iters_done] for one problem, else
        [iters_done, n_prob], iterations done, converged); self.last_reached holds, per problem, the
        first iteration whose F reached f_target (-1 if none)."""
        self._check_u(u)
        self._check_state(psi0)
        self._check_state(psif)
        F_hist = torch.zeros(max(iters, 1) * self.n_prob, dtype=torch.float64, device=u.device)
        reached = torch.empty(self.n_prob, dtype=torch.int32, device=u.device)
        o = L.qoc_opt_opts()
        self.lib.qoc_opt_opts_default(C.byref(o))
        o.iters, o.rule, o.step = iters, (L.QOC_RULE_ADAM if rule == "adam" else L.QOC_RULE_FIXED), step
        o.beta1, o.beta2, o.eps, o.f_target = beta1, beta2, eps, f_target
        o.check_every, o.use_graph, o.freeze_converged = check_every, int(use_graph), int(freeze)
        done = C.c_int(0)
        ws = self.workspace
        cur = torch.cuda.current_stream() if stream is None else stream
        run_stream = cur
        if use_graph:
            if self._graph_stream is None:
                self._graph_stream = torch.cuda.Stream(device=self.device)
            run_stream = self._graph_stream
            run_stream.wait_stream(cur)
        rc = self.lib.qoc_optimize_pulses(self.handle, _ptr(u), _ptr(psi0), _ptr(psif), C.byref(o), _ptr(F_hist),
                                          _ptr(reached), C.byref(done), _ptr(ws), ws.numel(), _stream(run_stream))
        if use_graph:
            cur.wait_stream(run_stream)
        converged = rc == L.QOC_OK
        if rc not in (L.QOC_OK, L.QOC_ENOTCONVERGED):
            L.check(rc, "qoc_optimize_pulses")
        self.last_reached = reached
        Fh = F_hist[: done.value * self.n_prob].view(done.value, self.n_prob)
        return (Fh[:, 0] if self.n_prob == 1 else Fh), done.value, converged

    def set_profiling(self, on: bool = True) -> None:
        L.check(self.lib.qoc_plan_set_profiling(self.handle, int(on)), "qoc_plan_set_profiling")

    def phase_times(self) -> List[float]:
        """[expm, sweeps, overlap, slice derivatives, reduction] of the last call, in ms."""
        ms = (C.c_float * 5)()
        L.check(self.lib.qoc_plan_phase_times(self.handle, ms, 5), "qoc_plan_phase_times")
        return list(ms)

    def work_counts(self) -> List[int]:
        """[sum m^3 * polynomial products, sum m^3 * squarings, items, complex multiply-adds of the
        register-tile derivative series, complex multiply-adds of the GEMM-path derivative series,
        sum m^3 * tensor-core products taken with three split terms] since profiling was enabled."""
        out = (C.c_longlong * 6)()
        L.check(self.lib.qoc_plan_work_counts(self.handle, out, 6), "qoc_plan_work_counts")
        return list(out)

    def set_expm_rules(self, rules) -> None:
        """rules: [(m_max, kind, param)], kind 0 = tiled CTA kernel (param R), 1 = warp-packed (param =
        matrices per warp), 2 = tensor cores, one CTA per slice (m <= 112; param 0: slices without
        squarings, 1: all), 3 = tiled tensor-core GEMMs (m <= 2048, slices without squarings).
        Reallocates the workspace if its size changes."""
        n = len(rules)
        mx = (C.c_int * n)(*[r[0] for r in rules])
        kd = (C.c_int * n)(*[r[1] for r in rules])
        pm = (C.c_int * n)(*[r[2] for r in rules])
        L.check(self.lib.qoc_plan_set_expm_rules(self.handle, n, mx, kd, pm), "qoc_plan_set_expm_rules")
        nbytes = C.c_size_t()
        L.check(self.lib.qoc_plan_workspace_bytes(self.handle, C.byref(nbytes)), "qoc_plan_workspace_bytes")
        if nbytes.value != self.workspace_bytes:
            self.workspace_bytes = nbytes.value
            self._ws = None

    def set_sweep_cluster(self, cl: int) -> None:
        """Sweep kernel: cl = 2, 4 or 8 CTAs per chain in a thread-block cluster, 0 one CTA per
        chain, -1 the automatic choice."""
        L.check(self.lib.qoc_plan_set_sweep_cluster(self.handle, cl), "qoc_plan_set_sweep_cluster")

    def set_deriv_gemm(self, mode, min_m: int = 0) -> None:
        """Slice derivatives as tall GEMMs shared by a chunk's slices: mode 0 / False off (per-slice
        series kernels), 1 FP32 CUDA cores, 2 / True tensor cores (the default); min_m: the smallest
        block on the path (0 keeps the current threshold).  Reallocates the workspace if its size
        changes."""
        mode = 2 if mode is True else 0 if mode is False else int(mode)
        L.check(self.lib.qoc_plan_set_deriv_gemm(self.handle, mode, int(min_m)), "qoc_plan_set_deriv_gemm")
        nbytes = C.c_size_t()
        L.check(self.lib.qoc_plan_workspace_bytes(self.handle, C.byref(nbytes)), "qoc_plan_workspace_bytes")
        if nbytes.value != self.workspace_bytes:
            self.workspace_bytes = nbytes.value
            self._ws = None

    def set_persistent(self, on: bool) -> None:
        """One cooperative launch per evaluation / GRAPE iteration (FP64 plans without checkpointing);
        reallocates the workspace if its size changes."""
        L.check(self.lib.qoc_plan_set_persistent(self.handle, int(on)), "qoc_plan_set_persistent")
        nbytes = C.c_size_t()
        L.check(self.lib.qoc_plan_workspace_bytes(self.handle, C.byref(nbytes)), "qoc_plan_workspace_bytes")
        if nbytes.value != self.workspace_bytes:
            self.workspace_bytes = nbytes.value
            self._ws = None

    def deriv_gemm_blocks(self) -> int:
        n = C.c_int()
        L.check(self.lib.qoc_plan_deriv_gemm(self.handle, C.byref(n)), "qoc_plan_deriv_gemm")
        return n.value

    def sweep_cluster(self) -> int:
        n = C.c_int()
        L.check(self.lib.qoc_plan_sweep_cluster(self.handle, C.byref(n)), "qoc_plan_sweep_cluster")
        return n.value

    def expm_classes(self):
        """[(kind, param, per_warp, m_max, n_blocks)] of the plan's exponential launches."""
        n = C.c_int()
        cap = 32
        arrs = [(C.c_int * cap)() for _ in range(5)]
        L.check(self.lib.qoc_plan_expm_classes(self.handle, cap, C.byref(n), *arrs), "qoc_plan_expm_classes")
        return [tuple(a[i] for a in arrs) for i in range(n.value)]

    def kernel_launches(self, with_grad: bool = True) -> int:
        n = C.c_int()
        L.check(self.lib.qoc_plan_kernel_launches(self.handle, int(with_grad), C.byref(n)), "qoc_plan_kernel_launches")
        return n.value

    def sync_status(self, stream=None) -> None:
        L.check(self.lib.qoc_plan_sync_status(self.handle, _stream(stream)), "device status")


class FidelityGrad(torch.autograd.Function):
    """F(u) = |<psi_f|psi_N(u)>|^2 (one problem: a scalar; a batch plan: [n_prob]) with its
    hand-written adjoint.  forward runs the propagators, the forward states (kept per slice, or at
    checkpoints) and the overlap; backward runs the costate sweep and the exact slice derivatives
    (recomputing checkpointed segments) and scales dF_p/du by the incoming dL/dF_p on the device.
    Under torch.no_grad, or when no gradient is asked for, no costate kernel runs."""

    @staticmethod
    def forward(ctx, u: torch.Tensor, plan: Plan, psi0: torch.Tensor, psif: torch.Tensor):
        uc = u.detach().contiguous()
        out3, serial = plan.forward(uc, psi0, psif)
        ctx.plan, ctx.u, ctx.psif, ctx.serial = plan, uc, psif, serial
        F = out3.view(plan.n_prob, 3)[:, 0].clone()
        return F[0] if plan.n_prob == 1 else F

    @staticmethod
    def backward(ctx, gF):
        plan = ctx.plan
        gFd = gF.detach().to(torch.float64).reshape(-1).contiguous()
        if gFd.numel() == 1 and plan.n_prob > 1:
            gFd = gFd.expand(plan.n_prob).contiguous()
        g = plan.backward(ctx.u, ctx.psif, ctx.serial, gF=gFd)
        return g, None, None, None


class Trotter:
    """Trotterised propagation with one pulse pair per qubit (Sec. IV): slice j applies
    prod_{i=1..n} exp(-i tau h_i^(j)) E with E = exp(-i tau/n H_cpl) from the D_n blocks of the coupling
    (qoc_trotter_create / qoc_trotter_propagate).  cpl: a D_n Basis whose H0 is H_cpl."""

    def __init__(self, cpl: Basis, tau: float, device=None):
        self.lib = L.load()
        self.n, self.dim, self.tau = cpl.system.n, 1 << cpl.system.n, tau
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            L.check(self.lib.qoc_trotter_create(cpl.handle, float(tau), C.byref(h)), "qoc_trotter_create")
        self.handle = h

    def __del__(self):
        if getattr(self, "handle", None):
            self.lib.qoc_trotter_free(self.handle)
            self.handle = None

    def propagate(self, pulses: torch.Tensor, psi_in: torch.Tensor, stream=None) -> torch.Tensor:
        """pulses [N, n, 3] (Bz, Bx, By) float64; psi_in [ncols, 2^n] complex128 -> U_N ... U_1 psi_in."""
        assert pulses.dtype == torch.float64 and pulses.is_cuda and pulses.is_contiguous()
        assert pulses.dim() == 3 and pulses.shape[1] == self.n and pulses.shape[2] == 3
        assert psi_in.dtype == torch.complex128 and psi_in.is_cuda and psi_in.is_contiguous()
        assert psi_in.shape[-1] == self.dim
        out = torch.empty_like(psi_in)
        ncols = psi_in.numel() // self.dim
        L.check(self.lib.qoc_trotter_propagate(self.handle, _ptr(pulses), pulses.shape[0], _ptr(psi_in), _ptr(out),
                                               ncols, _stream(stream)), "qoc_trotter_propagate")
        return out


def to_device(blk: np.ndarray, device=None) -> torch.Tensor:
    """A host block state (complex128, length state_len) as a device tensor."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else device
    return torch.from_numpy(np.ascontiguousarray(blk, dtype=np.complex128)).to(dev)
