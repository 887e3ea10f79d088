"""Pins of the oracle's Pauli operators and coupling terms (Sec. II.A; Eq. H0MoreCoupling1).

Every coupling weight is fixed here by a closed form that does not restate the term's own sum:
  - the one-magnon spectrum of the XXZ ring, E_k = 4 cos(2 pi k d / n) + Delta (n - 4), on the full
    space and inside the oracle's D_n blocks (which irrep carries which momentum k);
  - exact diagonal values of the distance-d Z ring on computational states (n on |0...0>, n - 4 on
    every single flip, also at d = n/2 where the literal sum counts every pair twice);
  - the all-pairs Heisenberg coupling as a function of the total spin, 2 J (J + 1) - 3 n / 2.
A weight error (1/2 on XX + YY, a dropped or doubled wrap bond, a wrong sign) fails one of them.
"""
import itertools
from math import comb

import numpy as np
import pytest

from oracle import operators as op
from oracle import symmetry as sy


def _dense(A):
    return np.asarray(A.todense())


def _weight_states(n, w):
    return [x for x in range(1 << n) if bin(x).count("1") == w]


def test_pauli_algebra_single_site():
    P = [op.SX, op.SY, op.SZ]
    eps = np.zeros((3, 3, 3))
    for a, b, c in itertools.permutations(range(3)):
        eps[a, b, c] = np.linalg.det(np.eye(3)[[a, b, c]])
    for a in range(3):
        for b in range(3):
            want = (a == b) * np.eye(2) + 1j * sum(eps[a, b, c] * P[c] for c in range(3))
            assert np.allclose(P[a] @ P[b], want, atol=0)


def test_sigma_sites_hermitian_commuting():
    n = 4
    for i in range(1, n + 1):
        for a in "xyz":
            S = _dense(op.sigma(n, i, a))
            assert np.allclose(S, S.conj().T)
            assert np.allclose(S @ S, np.eye(1 << n))
        for j in range(i + 1, n + 1):
            A, B = _dense(op.sigma(n, i, "x")), _dense(op.sigma(n, j, "y"))
            assert np.allclose(A @ B, B @ A)
    # same site, different axes anticommute
    A, B = _dense(op.sigma(n, 2, "x")), _dense(op.sigma(n, 2, "z"))
    assert np.allclose(A @ B, -B @ A)


def test_qubit_one_is_most_significant():
    # sigma_z^(1) is -1 exactly on the indices whose top bit is set (qubit 1 in |1>)
    n = 5
    d = np.real(np.diag(_dense(op.sigma(n, 1, "z"))))
    assert np.array_equal(d < 0, np.arange(1 << n) >= (1 << (n - 1)))


def _xxz(n, delta, dist=1):
    return _dense(op.term_matrix(n, op.RING_XX, dist) + op.term_matrix(n, op.RING_YY, dist)
                  + delta * op.term_matrix(n, op.RING_ZZ, dist))


@pytest.mark.parametrize("n", [3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("delta", [0.0, 0.5, -1.3])
def test_one_magnon_spectrum_nearest_neighbour(n, delta):
    H = _xxz(n, delta)
    one = _weight_states(n, 1)
    zero = _weight_states(n, 0)
    # the coupling conserves the number of flipped spins: no amplitude leaves the one-magnon sector
    rest = [x for x in range(1 << n) if x not in one]
    assert np.abs(H[np.ix_(rest, one)]).max() < 1e-14
    E = np.sort(np.linalg.eigvalsh(H[np.ix_(one, one)]))
    want = np.sort([4 * np.cos(2 * np.pi * k / n) + delta * (n - 4) for k in range(n)])
    assert np.allclose(E, want, atol=1e-12)
    # all spins up: every bond aligned
    assert abs(H[zero[0], zero[0]] - delta * n) < 1e-14


@pytest.mark.parametrize("n", [4, 5, 6, 7, 8])
def test_ring_distance_d_z_values(n):
    for d in range(1, n // 2 + 1):
        Z = np.real(np.diag(_dense(op.term_matrix(n, op.RING_ZZ, d))))
        assert Z[0] == n
        for x in _weight_states(n, 1):
            assert Z[x] == n - 4, (n, d, x)


@pytest.mark.parametrize("n", [4, 5, 6, 7, 8])
def test_ring_distance_d_hopping(n):
    # XX + YY at distance d moves a single flip by +-d: E_k = 4 cos(2 pi k d / n) (literal sum; at
    # d = n/2 both terms of a pair hop to the same site and the amplitude doubles, as the formula says)
    one = _weight_states(n, 1)
    for d in range(1, n // 2 + 1):
        H = _xxz(n, 0.0, d)
        E = np.sort(np.linalg.eigvalsh(H[np.ix_(one, one)]))
        want = np.sort([4 * np.cos(2 * np.pi * k * d / n) for k in range(n)])
        assert np.allclose(E, want, atol=1e-12), (n, d)


def _one_magnon_part(V, n):
    """Rows of the block basis V [m, 2^n] supported on single flips only."""
    one = np.array(_weight_states(n, 1))
    keep = [a for a in range(V.shape[0]) if np.abs(np.delete(V[a], one)).max() < 1e-14
            and np.abs(V[a, one]).max() > 1e-14]
    return V[keep]


@pytest.mark.parametrize("n", [5, 6, 8])
def test_one_magnon_energies_per_dn_irrep(n):
    """Inside the oracle's D_n blocks, the one-magnon vector of irrep A1 has k = 0, that of E_m has
    k = +-m, and for even n one of B1/B2 has k = n/2; A2 has none (a reflection through the flipped
    site leaves a single flip unchanged)."""
    delta = 0.5
    H = _xxz(n, delta)
    E = lambda k: 4 * np.cos(2 * np.pi * k / n) + delta * (n - 4)
    found = {}
    for label, V in sy.dn_blocks(n):
        for r in range(V.shape[0]):
            W = _one_magnon_part(V[r], n)
            if W.shape[0] == 0:
                continue
            assert W.shape[0] == 1, label
            w = W[0]
            Hw = H @ w
            e = np.vdot(w, Hw).real
            assert np.allclose(Hw, e * w, atol=1e-12), label  # an eigenvector of the coupling
            found.setdefault(label, set()).add(round(e, 10))
    assert found["A1"] == {round(E(0), 10)}
    assert "A2" not in found
    for m in range(1, (n - 1) // 2 + 1):
        assert found[f"E{m}"] == {round(E(m), 10)}
    if n % 2 == 0:
        bs = [found.get(l) for l in ("B1", "B2")]
        assert sorted(map(bool, bs)) == [False, True]
        assert [b for b in bs if b][0] == {round(E(n // 2), 10)}


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_allpairs_heisenberg_is_total_spin(n):
    """sum_{i<j} (XX + YY + ZZ) = 2 J (J + 1) - 3 n / 2 with the S_n multiplicities of each J."""
    H = _dense(op.term_matrix(n, op.ALLPAIRS_XX) + op.term_matrix(n, op.ALLPAIRS_YY)
               + op.term_matrix(n, op.ALLPAIRS_ZZ))
    E = np.sort(np.linalg.eigvalsh(H))
    want = []
    for J2 in range(n % 2, n + 1, 2):
        J = J2 / 2
        mult = comb(n, (n - J2) // 2) - (comb(n, (n - J2) // 2 - 1) if (n - J2) // 2 >= 1 else 0)
        want += [2 * J * (J + 1) - 1.5 * n] * int((J2 + 1) * mult)
    assert np.allclose(E, np.sort(want), atol=1e-12)


@pytest.mark.parametrize("kind", [op.SUM_X, op.SUM_Y, op.SUM_Z])
def test_collective_field_spectrum(kind):
    # sum_i sigma_a^(i) has eigenvalue n - 2w with multiplicity C(n, w)
    n = 5
    E = np.sort(np.linalg.eigvalsh(_dense(op.term_matrix(n, kind))))
    want = np.sort(sum([[n - 2 * w] * comb(n, w) for w in range(n + 1)], []))
    assert np.allclose(E, want, atol=1e-12)
