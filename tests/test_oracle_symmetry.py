"""Pins of the oracle's symmetry-adapted bases (Sec. II.A, Table I, Fig. 2, Appendix A)."""
import os
from math import comb

import numpy as np
import pytest

from oracle import operators as op
from oracle import symmetry as sy
from paper_2309_05884_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1.txt")


def table1():
    rows = []
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(int(x) for x in line.split()))
    return rows


@pytest.mark.parametrize("row", table1(), ids=lambda r: f"n{r[0]}")
def test_table1_by_characters(row):
    n, full, dimS, dimD = row
    assert full == 2 ** n
    dims = sy.dn_block_dims_by_characters(n)
    assert dims["A1"] == dimD
    sizes = dict(zip(dims, [2 if k.startswith("E") else 1 for k in dims]))
    assert sum(dims[k] * sizes[k] for k in dims) == 2 ** n
    sn = sy.sn_block_dims(n)
    assert sn[0] == (dimS, 1)
    assert sum(m * c for m, c in sn) == 2 ** n


@pytest.mark.parametrize("row", [r for r in table1() if r[0] <= 10], ids=lambda r: f"n{r[0]}")
def test_table1_by_constructed_basis(row):
    n, full, dimS, dimD = row
    bd = sy.dn_blocks(n)
    assert bd[0][0] == "A1" and bd[0][1].shape[1] == dimD
    chars = sy.dn_block_dims_by_characters(n)
    for label, V in bd:
        assert V.shape[1] == chars[label]
    if n <= 8:
        bs = sy.sn_blocks(n)
        assert bs[0][1].shape[1] == dimS
        assert [(V.shape[1], V.shape[0]) for _, V in bs] == sy.sn_block_dims(n)


def test_c1_sector_sizes():
    # the S_4 spin sectors J=2,1,0: sizes 5,3,1 with multiplicities 1,3,2
    assert sy.sn_block_dims(4) == [(5, 1), (3, 3), (1, 2)]


def test_c2_block_sizes():
    d = sy.dn_block_dims_by_characters(10)
    assert d == {"A1": 78, "A2": 30, "B1": 58, "B2": 42, "E1": 99, "E2": 105, "E3": 99, "E4": 105}


def _offblock_norm(blocks, X):
    A = sy.adjoint_matrix(blocks)
    B = A.conj().T @ X @ A
    mask = np.zeros(B.shape, dtype=bool)
    o = 0
    for _, V in blocks:
        for r in range(V.shape[0]):
            m = V.shape[1]
            mask[o:o + m, o:o + m] = True
            o += m
    return np.linalg.norm(B[~mask]), B


@pytest.mark.parametrize("n", [3, 4, 5, 6])
def test_sn_unitary_and_block_diagonal(n):
    blocks = sy.sn_blocks(n)
    A = sy.adjoint_matrix(blocks)
    assert np.abs(A.conj().T @ A - np.eye(2 ** n)).max() < 1e-12
    for kind in (I.SUM_X, I.SUM_Y, I.SUM_Z, I.ALLPAIRS_ZZ, I.ALLPAIRS_XX, I.ALLPAIRS_YY):
        X = op.term_matrix(n, kind).toarray()
        off, _ = _offblock_norm(blocks, X)
        assert off < 1e-12


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 8])
def test_dn_unitary_and_block_diagonal(n):
    blocks = sy.dn_blocks(n)
    A = sy.adjoint_matrix(blocks)
    assert np.abs(A.conj().T @ A - np.eye(2 ** n)).max() < 1e-12
    # every ring distance of Eq. H0MoreCoupling1 keeps the D_n blocks
    kinds = [(I.SUM_X, 0), (I.SUM_Y, 0), (I.SUM_Z, 0), (I.RING_XX, 1), (I.RING_YY, 1)] + \
        [(I.RING_ZZ, d) for d in range(1, n // 2 + 1)]
    for kind, d in kinds:
        X = op.term_matrix(n, kind, d).toarray()
        off, B = _offblock_norm(blocks, X)
        assert off < 1e-12
        # both copies of a 2-dimensional irrep carry the identical block
        o = 0
        for _, V in blocks:
            m = V.shape[1]
            blks = []
            for r in range(V.shape[0]):
                blks.append(B[o:o + m, o:o + m])
                o += m
            for b in blks[1:]:
                assert np.abs(b - blks[0]).max() < 1e-12


def test_ring_breaks_sn():
    # the ring coupling is D_n- but not S_n-invariant (Sec. II.A): its S_n off-block norm is nonzero
    off, _ = _offblock_norm(sy.sn_blocks(4), op.term_matrix(4, I.RING_ZZ, 1).toarray())
    assert off > 0.1


@pytest.mark.parametrize("n", [2, 4, 5])
def test_sn_blocks_are_collective_spin(n):
    # sum Z = 2 Jz, sum X = J+ + J-, sum Y = -i (J+ - J-), sum_{i<j} Z Z = 2 Jz^2 - n/2
    blocks = sy.sn_blocks(n)
    ops = {k: op.term_matrix(n, k).toarray() for k in (I.SUM_Z, I.SUM_X, I.SUM_Y, I.ALLPAIRS_ZZ)}
    for J2, V in blocks:
        Jz, Jp, Jm = sy.spin_matrices(J2)
        want = {I.SUM_Z: 2 * Jz, I.SUM_X: Jp + Jm, I.SUM_Y: -1j * (Jp - Jm),
                I.ALLPAIRS_ZZ: 2 * Jz @ Jz - n / 2 * np.eye(J2 + 1)}
        for r in range(V.shape[0]):
            for k, X in ops.items():
                assert np.abs(sy.block_operator(V[r], X) - want[k]).max() < 1e-12


def test_dicke_is_symmetric_block_vector():
    n = 6
    blocks = sy.sn_blocks(n)
    J2, V = blocks[0]
    for k in range(n + 1):
        d = op.dicke_state(n, k)
        assert abs(abs(np.vdot(V[0, k], d)) - 1.0) < 1e-12
        assert comb(n, k) == int(round(1.0 / abs(d[np.nonzero(d)[0][0]]) ** 2))


def test_round_trip_blocks():
    n = 6
    blocks = sy.dn_blocks(n)
    psi = I.random_state(5, 2 ** n)
    c = sy.to_blocks(blocks, psi)
    assert np.abs(sy.from_blocks(blocks, c) - psi).max() < 1e-12


def _first_block_resonances(s):
    """Distinct transition energies |E_a - E_b| between eigenstates of H0 in the first D_n block that
    the control sum X connects (the resonance frequencies of Sec. III)."""
    H0, Hc = op.system_operators(s)
    _, V = sy.symmetry_blocks(s)[0]
    w, Q = np.linalg.eigh(sy.block_operator(V[0], H0))
    X = Q.conj().T @ sy.block_operator(V[0], Hc[0]) @ Q
    return len(w), {round(abs(w[a] - w[b]), 9) for a in range(len(w)) for b in range(a) if abs(X[a, b]) > 1e-9}


def _golden_resonances():
    path = os.path.join(os.path.dirname(__file__), "golden", "resonances.txt")
    out = {}
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                kind, n, count = line.split()
                out[(kind, int(n))] = int(count)
    return out


@pytest.mark.parametrize("n", [3, 4, 5, 6])
def test_resonances_nearest_neighbour_vs_full_coupling(n):
    # Sec. III: with the nearest-neighbour coupling of Eq. H0WithCoupling the first subspace has three
    # resonance frequencies for every n >= 3; the full coupling of Eq. H0MoreCoupling1 breaks the
    # degeneracy, giving six for n = 4 (Fig. 4d); for n = 3 the two forms coincide (floor(n/2) = 1)
    gold = _golden_resonances()
    m, nn = _first_block_resonances(I.ising_ring(n, 1.0, 0.8, 1.0, 1))
    assert m == {3: 4, 4: 6, 5: 8, 6: 13}[n]  # Table I
    assert len(nn) == gold[("nn", n)]
    couplings = [0.8, 0.37, 0.23][: n // 2]
    _, full = _first_block_resonances(I.ising_ring_full(n, 1.0, couplings, 1.0, 1))
    if n == 3:
        assert full == nn
    else:
        assert len(full) > len(nn)
    if ("full", n) in gold:
        assert len(full) == gold[("full", n)]
