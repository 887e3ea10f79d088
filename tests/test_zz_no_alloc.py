"""The allocation-free batched exponential (qoc_expm_batch_noalloc), called through the C ABI, gives
the same propagators as the plan-based entry point qoc_expm_blocks, on two calls in a row.

It exists for callers that cannot allocate device memory while they run; its scratch is a fixed
array inside the library.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_2309_05884_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2309_05884_gb300 import _lib, api  # noqa: E402

DEV = torch.device("cuda", 0)
TOL64 = 1e-10


def test_noalloc_matches_plan_expm_two_calls():
    lib = _lib.load()
    s = I.xxz_ring(6, 2.0, 12)   # blocks of 1..13 (FP64 path)
    B = api.Basis(s)
    plan = api.Plan(B, s.N, s.tau, prec="f64")
    for seed in (21, 22):        # two calls in a row, different inputs
        ut = torch.from_numpy(I.pulses_normal(seed, s.N, 3)).to(DEV)
        A = plan.assemble(ut)
        U_ref = plan.expm(ut)
        U = torch.empty_like(A)
        off = 0
        for b in plan.active_blocks():
            m = B.blocks[b][1]
            n_el = s.N * m * m
            rc = lib.qoc_expm_batch_noalloc(C.c_void_p(A.data_ptr() + 16 * off), C.c_void_p(U.data_ptr() + 16 * off),
                                            m, s.N, None)
            assert rc == _lib.QOC_OK, lib.qoc_last_error()
            off += n_el
        torch.cuda.synchronize()
        err = (U - U_ref).abs().max().item()
        assert err <= TOL64, err


def test_noalloc_larger_blocks_and_limits():
    lib = _lib.load()
    s = I.xxz_ring(10, 0.4, 6)   # blocks of 30..105: several CTAs share the array, multi-tile GEMMs
    B = api.Basis(s)
    plan = api.Plan(B, s.N, s.tau, prec="f64")
    ut = torch.from_numpy(I.pulses_normal(5, s.N, 3)).to(DEV)
    A, U_ref = plan.assemble(ut), plan.expm(ut)
    U = torch.empty_like(A)
    off = 0
    for b in plan.active_blocks():
        m = B.blocks[b][1]
        assert lib.qoc_expm_batch_noalloc(C.c_void_p(A.data_ptr() + 16 * off), C.c_void_p(U.data_ptr() + 16 * off),
                                          m, s.N, None) == _lib.QOC_OK
        off += s.N * m * m
    torch.cuda.synchronize()
    assert (U - U_ref).abs().max().item() <= TOL64
    # sizes beyond the fixed array's limit are rejected before any launch
    rc = lib.qoc_expm_batch_noalloc(C.c_void_p(A.data_ptr()), C.c_void_p(U.data_ptr()), 129, 1, None)
    assert rc == _lib.QOC_EUNSUPPORTED and b"1..128" in lib.qoc_last_error()
