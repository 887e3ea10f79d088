"""The C-ABI library loads, exports every symbol include/qoc.h declares, and its host-side
symmetry builder agrees with the oracle on gauge-invariant quantities (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2309_05884_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qoc.h")


def declared_symbols():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qoc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2309_05884_gb300 import _lib
    return _lib.load()


def test_header_symbols_exported(lib):
    from paper_2309_05884_gb300 import _lib
    syms = declared_symbols()
    assert len(syms) >= 20
    for s in syms:
        assert hasattr(lib, s), s
        assert s in _lib.SIGNATURES, s


def test_errors_are_reported(lib):
    from paper_2309_05884_gb300 import _lib
    h = C.c_void_p()
    assert lib.qoc_build_symmetry_basis(None, 0, C.byref(h)) == _lib.QOC_EINVAL
    assert b"null" in lib.qoc_last_error()
    assert lib.qoc_strerror(_lib.QOC_ETIMEOUT) == b"device wait timed out"


def test_ring_rejected_for_sn():
    from paper_2309_05884_gb300 import api
    s = I.System(5, I.GROUP_SN, [(I.RING_ZZ, 1.0, 1)], [[(I.SUM_X, 1.0, 0)]], 1.0, 10)
    with pytest.raises(RuntimeError, match="S_n"):
        api.Basis(s)


def _oracle_blocks(system):
    from oracle import operators as op
    from oracle import symmetry as sy
    H0, Hc = op.system_operators(system)
    return H0, Hc, sy.symmetry_blocks(system)


@pytest.mark.parametrize("system", [I.c1_system(), I.xxz_ring(6, 1.0, 10), I.xxz_ring(8, 1.0, 10),
                                    I.ising_ring(7, 1.0, 0.6, 1.0, 10), I.sn_allpairs(6, 0.7, 0.3, 1.0, 10),
                                    I.ising_ring_full(8, 1.0, [0.8, 0.37, 0.23, 0.11], 1.0, 10)],
                         ids=["c1", "xxz6", "xxz8", "ising7", "sn6", "ising8_full"])
def test_host_blocks_match_oracle(system):
    from oracle import symmetry as sy
    from paper_2309_05884_gb300 import api
    B = api.Basis(system)
    H0, Hc, ob = _oracle_blocks(system)
    # same block structure (sizes, copies) in the same order
    assert [(m, c) for _, m, c, _ in B.blocks] == [(V.shape[1], V.shape[0]) for _, V in ob]
    assert B.state_len == 2 ** system.n
    for b, (_, V) in enumerate(ob):
        h0, hc = B.block_matrices(b)
        # Hermitian, and spectra equal to the oracle's blocks (gauge invariant)
        for mine, full in [(h0, H0)] + [(hc[j], Hc[j]) for j in range(len(Hc))]:
            assert np.abs(mine - mine.conj().T).max() < 1e-12
            ref = sy.block_operator(V[0], full)
            assert np.allclose(np.linalg.eigvalsh(mine), np.linalg.eigvalsh(ref), atol=1e-10)
        # a mixed operator too (the eigenvalues of sums are not fixed by those of the terms)
        mix = h0 + 0.37 * hc[0] - 0.81 * hc[-1]
        ref = sy.block_operator(V[0], H0 + 0.37 * Hc[0] - 0.81 * Hc[-1])
        assert np.allclose(np.linalg.eigvalsh(mix), np.linalg.eigvalsh(ref), atol=1e-10)


@pytest.mark.parametrize("system", [I.c1_system(), I.xxz_ring(7, 1.0, 10)], ids=["c1", "xxz7"])
def test_host_state_conversion(system):
    from oracle import operators as op
    from paper_2309_05884_gb300 import api
    B = api.Basis(system)
    H0, Hc = op.system_operators(system)
    psi = I.random_state(3, 2 ** system.n)
    blk = B.state_to_blocks(psi)
    assert abs(np.linalg.norm(blk) - 1.0) < 1e-12
    assert np.abs(B.blocks_to_state(blk) - psi).max() < 1e-12
    # <psi|H|psi> from the blocks equals the full-space value
    for Hfull, j in [(H0, None)] + [(h, i) for i, h in enumerate(Hc)]:
        want = np.vdot(psi, Hfull @ psi)
        got = 0.0
        for b, (_, m, c, off) in enumerate(B.blocks):
            h0, hc = B.block_matrices(b)
            Hb = h0 if j is None else hc[j]
            for r in range(c):
                x = blk[off + r * m: off + (r + 1) * m]
                got += np.vdot(x, Hb @ x)
        assert abs(got - want) < 1e-11


def test_table1_from_host_builder():
    from paper_2309_05884_gb300 import api
    rows = [tuple(int(x) for x in l.split()) for l in open(os.path.join(ROOT, "tests", "golden", "table1.txt"))
            if l.strip() and not l.startswith("#")]
    for n, full, dimS, dimD in rows:
        s = I.xxz_ring(n, 1.0, 10)
        B = api.Basis(s, first_block_only=True, vectors=False)
        assert B.blocks[0][1] == dimD and B.blocks[0][0] == "A1"
        t = I.sn_allpairs(n, 1.0, 0.5, 1.0, 10)
        Bs = api.Basis(t, first_block_only=True, vectors=False)
        assert Bs.blocks[0][1] == dimS


def test_dicke_state_in_block_coordinates():
    from oracle import operators as op
    from paper_2309_05884_gb300 import api
    s = I.sn_allpairs(6, 1.0, 0.5, 1.0, 10)
    B = api.Basis(s)
    for k in range(7):
        blk = B.dicke_state(k)
        assert np.abs(B.blocks_to_state(blk) - op.dicke_state(6, k)).max() < 1e-12
    big = api.Basis(I.sn_allpairs(40, 1.0, 0.5, 1.0, 10))
    assert big.n_blocks == 1 and big.state_len == 41


def test_host_first_block_resonances_full_coupling():
    # Sec. III / Fig. 4d on the library's own blocks: n = 4, nearest-neighbour coupling gives three
    # resonance frequencies in the first subspace, the full coupling of Eq. H0MoreCoupling1 six
    from paper_2309_05884_gb300 import api

    def resonances(s):
        B = api.Basis(s, first_block_only=True)
        h0, hc = B.block_matrices(0)
        w, Q = np.linalg.eigh(h0)
        X = Q.conj().T @ hc[0] @ Q
        return {round(abs(w[a] - w[b]), 9) for a in range(len(w)) for b in range(a) if abs(X[a, b]) > 1e-9}

    assert len(resonances(I.ising_ring(4, 1.0, 0.8, 1.0, 1))) == 3
    assert len(resonances(I.ising_ring_full(4, 1.0, [0.8, 0.37], 1.0, 1))) == 6


@pytest.mark.parametrize("system", [I.c1_system(), I.xxz_ring(8, 1.0, 10), I.ising_ring(7, 1.0, 0.6, 1.0, 10),
                                    I.sn_allpairs(6, 0.7, 0.3, 1.0, 10), I.xxz_ring(10, 0.32, 10)],
                         ids=["c1", "xxz8", "ising7", "sn6", "xxz10"])
def test_norm_bounds_enclose_spectral_norms(system):
    # The per-block bounds that fix the Taylor degree: never below the spectral norm (the truncation
    # bound stays rigorous), never above the 1-norm (no slice needs more products than with it), and
    # equal to it where the moduli of a block are the block up to a diagonal sign change (real
    # blocks with one sign pattern, e.g. the S_n J blocks), where rho(|M|) = rho(M).
    from paper_2309_05884_gb300 import api
    B = api.Basis(system)
    tighter = 0
    for b, (_, m, _, _) in enumerate(B.blocks):
        h0, hc = B.block_matrices(b)
        bounds = B.norm_bounds(b)
        for M, nb in zip([h0] + list(hc), bounds):
            two = np.abs(np.linalg.eigvalsh(M)).max() if m > 0 else 0.0
            one = np.abs(M).sum(axis=0).max()
            assert two - 1e-12 * max(1.0, one) <= nb <= one * (1 + 1e-12) + 1e-300, (b, two, nb, one)
            rho_abs = np.abs(np.linalg.eigvals(np.abs(M))).max()
            assert nb <= rho_abs * (1 + 1e-2) + 1e-12, (b, nb, rho_abs)  # converged to rho(|M|)
            tighter += nb < one * (1 - 1e-3)
    if system.n >= 8:
        assert tighter > 0  # the bound improves on the 1-norm somewhere
