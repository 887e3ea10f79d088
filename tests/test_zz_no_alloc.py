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


def test_noalloc_largest_size_persistent_slots():
    # m = 128, the largest size the fixed array takes: six slots of 10 m^2 complex, so 13 matrices make
    # the CTAs loop over the batch; one matrix has a large norm (squarings).  Reference: the
    # eigendecomposition of each Hermitian H, U = V exp(-i tau w) V^dagger.
    lib = _lib.load()
    m, count, tau = 128, 13, 0.05
    g = I.rng(77)
    Hs = []
    for i in range(count):
        X = g.normal(size=(m, m)) + 1j * g.normal(size=(m, m))
        H = (X + X.conj().T) / 2 * (40.0 if i == 5 else 1.0)
        Hs.append(H)
    A = np.stack([-1j * tau * H for H in Hs])
    ref = []
    for H in Hs:
        w, V = np.linalg.eigh(H)
        ref.append((V * np.exp(-1j * tau * w)) @ V.conj().T)
    At = torch.from_numpy(A).to(DEV)
    for _ in range(2):   # two calls in a row on the shared array
        U = torch.zeros_like(At)
        rc = lib.qoc_expm_batch_noalloc(C.c_void_p(At.data_ptr()), C.c_void_p(U.data_ptr()), m, count, None)
        assert rc == _lib.QOC_OK, lib.qoc_last_error()
        torch.cuda.synchronize()
        assert np.abs(U.cpu().numpy() - np.stack(ref)).max() <= 1e-10
