"""Oracle: S_n and D_n symmetry-adapted bases and block Hamiltonians (test infrastructure only).

Paper, Sec. II.A and Appendix A.  The Hilbert space of n qubits splits into orthogonal subspaces
labelled by irreps of the symmetry group; stacking orthonormal bases of those subspaces as
columns gives the adjoint matrix A, and A^dagger H A is block diagonal for every H that commutes
with the group (Fig. 2).

S_n (Appendix A, first paragraph; the Clebsch-Gordan |J,M> route): for each weight w (number of
ones, M = n/2 - w) the highest-weight vectors of spin J = n/2 - w are the kernel of the total
raising operator J+ inside that weight space; lowering them with J- gives |J,M,r>.  Copy r runs
over an orthonormal basis of the kernel, so every copy carries the same (2J+1)-dimensional block.

D_n (Eq. groupAlgebraElementsDn): the group-algebra element O_j^theta = sum_g A_jj^theta(g) g,
normalised as the projector P_jj = (d_theta/2n) sum_g A_jj^theta(g) rho(g), is applied inside the
span of each orbit of computational states; its eigenvectors with eigenvalue 1 are the orbit's
row-1 vectors of irrep theta.  For 2-dimensional irreps the second copy is P_21 applied to the
row-1 vectors, which gives a block identical to the first.  Irreps are taken in real orthogonal
form (rotation by 2 pi m t/n, reflection diag(1,-1)); the paper only says "unitary irreps".

Block ordering: D_n: A1, A2, (B1, B2 for even n), E1, E2, ...; S_n: J = n/2, n/2-1, ...
B1 is +1 on reflections that fix a vertex (i -> t-i, t even), B2 on those that fix none.

Pins (tests/test_oracle_symmetry.py): Table I dimensions (tests/golden/table1.txt), block sizes
against a character count, A^dagger A = I, vanishing off-block norm, identical copies, S_n blocks
equal to the collective-spin matrices.
"""
from __future__ import annotations

from math import comb, gcd

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


# ----------------------------------------------------------------------------- helpers
def _bit(x: int, p: int, n: int) -> int:
    """Bit of qubit p+1 (0-based position p) in basis index x; qubit 1 is the MSB."""
    return (x >> (n - 1 - p)) & 1


def _popcount(x: int) -> int:
    return bin(x).count("1")


# ----------------------------------------------------------------------------- S_n
def sn_blocks(n: int):
    """S_n-adapted basis.  Returns a list of (J2, V) with J2 = 2J and V of shape
    [copies, 2J+1, 2^n]; V[r, a] is |J, M = J - a, r> as a full-space vector."""
    dim = 1 << n
    # J- = sum_i sigma_-^(i), sigma_- = |1><0| (|0> = up): lowers the weight by flipping a 0 to a 1.
    rows, cols = [], []
    for x in range(dim):
        for p in range(n):
            if _bit(x, p, n) == 0:
                rows.append(x | (1 << (n - 1 - p)))
                cols.append(x)
    Jm = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(dim, dim))
    Jp = Jm.T.tocsr()
    out = []
    for w in range(0, n // 2 + 1):
        states_w = [x for x in range(dim) if _popcount(x) == w]
        if w == 0:
            hw = np.ones((1, 1))
        else:
            states_prev = [x for x in range(dim) if _popcount(x) == w - 1]
            Jp_w = Jp[states_prev][:, states_w].toarray()
            hw = sla.null_space(Jp_w)
        if hw.shape[1] == 0:
            continue
        J2 = n - 2 * w  # 2J
        copies = hw.shape[1]
        V = np.zeros((copies, J2 + 1, dim), dtype=np.complex128)
        for r in range(copies):
            v = np.zeros(dim, dtype=np.complex128)
            v[states_w] = hw[:, r]
            V[r, 0] = v
            for a in range(1, J2 + 1):
                # |J, M-1> = J- |J, M> / sqrt(J(J+1) - M(M-1)), M = J - (a-1)
                J = J2 / 2.0
                M = J - (a - 1)
                V[r, a] = (Jm @ V[r, a - 1]) / np.sqrt(J * (J + 1) - M * (M - 1))
        out.append((J2, V))
    return out


def sn_block_dims(n: int):
    """(size, copies) of every S_n block: size 2J+1, copies C(n, n/2-J) - C(n, n/2-J-1)."""
    out = []
    for w in range(0, n // 2 + 1):
        copies = comb(n, w) - (comb(n, w - 1) if w >= 1 else 0)
        if copies > 0:
            out.append((n - 2 * w + 1, copies))
    return out


def spin_matrices(J2: int):
    """Jz, J+, J- for spin J = J2/2 in the |J, M = J - a> basis, a = 0..2J (Condon-Shortley)."""
    J = J2 / 2.0
    m = J2 + 1
    Ms = J - np.arange(m)
    Jz = np.diag(Ms).astype(np.complex128)
    Jm = np.zeros((m, m), dtype=np.complex128)
    for a in range(m - 1):
        M = Ms[a]
        Jm[a + 1, a] = np.sqrt(J * (J + 1) - M * (M - 1))
    return Jz, Jm.conj().T, Jm


# ----------------------------------------------------------------------------- D_n
def dn_group(n: int):
    """The 2n elements g = rho^t sigma^e of D_n as (t, e, perm), perm[i] = g(i) on positions
    0..n-1, with rho: i -> i+1 and sigma: i -> -i (mod n)."""
    out = []
    for e in (0, 1):
        for t in range(n):
            perm = [((-i if e else i) + t) % n for i in range(n)]
            out.append((t, e, perm))
    return out


def dn_act(perm, x: int, n: int) -> int:
    """rho(g)|x> = |g.x>, where the bit at position g(i) of g.x is the bit at position i of x."""
    y = 0
    for i in range(n):
        if _bit(x, i, n):
            y |= 1 << (n - 1 - perm[i])
    return y


def dn_irreps(n: int):
    """Real orthogonal irreps of D_n: list of (label, d, D) with D(t, e) -> d x d array."""
    irr = [("A1", 1, lambda t, e: np.array([[1.0]])),
           ("A2", 1, lambda t, e: np.array([[(-1.0) ** e]]))]
    if n % 2 == 0:
        irr.append(("B1", 1, lambda t, e: np.array([[(-1.0) ** t]])))
        irr.append(("B2", 1, lambda t, e: np.array([[(-1.0) ** (t + e)]])))
    for m in range(1, (n - 1) // 2 + 1):
        def D(t, e, m=m):
            a = 2 * np.pi * m * t / n
            R = np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])
            return R @ np.diag([1.0, -1.0]) if e else R
        irr.append((f"E{m}", 2, D))
    return irr


def dn_orbits(n: int):
    """Orbits of the computational states under D_n, each sorted, ordered by smallest element."""
    G = dn_group(n)
    seen = np.zeros(1 << n, dtype=bool)
    orbits = []
    for x in range(1 << n):
        if seen[x]:
            continue
        orb = sorted({dn_act(perm, x, n) for (_, _, perm) in G})
        seen[orb] = True
        orbits.append(orb)
    return orbits


def dn_blocks(n: int, labels=None):
    """D_n-adapted basis.  Returns a list of (label, V) with V of shape [copies, m, 2^n]
    (copies = irrep dimension); V[r, a] is the a-th basis vector of row r+1 of the irrep.
    labels (optional): build only the irreps named there (same vectors as the full build)."""
    G = dn_group(n)
    orbits = dn_orbits(n)
    irreps = dn_irreps(n)
    dim = 1 << n
    out = []
    for label, d, D in irreps:
        if labels is not None and label not in labels:
            continue
        rows = [[] for _ in range(d)]
        for orb in orbits:
            idx = {x: i for i, x in enumerate(orb)}
            L = len(orb)
            # P_jk restricted to the orbit span, as an L x L matrix
            P = np.zeros((d, d, L, L))
            for (t, e, perm) in G:
                Dg = D(t, e)
                for i, x in enumerate(orb):
                    P[:, :, idx[dn_act(perm, x, n)], i] += Dg
            P *= d / (2.0 * n)
            w, U = np.linalg.eigh(0.5 * (P[0, 0] + P[0, 0].T))
            sel = U[:, w > 0.5]
            for c in range(sel.shape[1]):
                for r in range(d):
                    vec = sel[:, c] if r == 0 else P[r, 0] @ sel[:, c]
                    full = np.zeros(dim, dtype=np.complex128)
                    full[orb] = vec
                    rows[r].append(full)
        m = len(rows[0])
        if m == 0:
            continue
        V = np.array([np.array(rows[r]) for r in range(d)])
        out.append((label, V))
    return out


def dn_block_dims_by_characters(n: int):
    """Multiplicity of every D_n irrep in the permutation representation on {0,1}^n, by
    characters: m_theta = (1/2n) sum_g chi_theta(g) 2^{cycles(g)}.  Returns {label: m}."""
    G = dn_group(n)

    def cycles(perm):
        seen, c = [False] * n, 0
        for i in range(n):
            if not seen[i]:
                c += 1
                j = i
                while not seen[j]:
                    seen[j] = True
                    j = perm[j]
        return c

    out = {}
    for label, d, D in dn_irreps(n):
        s = sum(np.trace(D(t, e)) * 2.0 ** cycles(perm) for (t, e, perm) in G)
        out[label] = int(round(s / (2 * n)))
    return out


# ----------------------------------------------------------------------------- blocks of H
def adjoint_matrix(blocks) -> np.ndarray:
    """A: all basis vectors as columns, in block order then copy order then index."""
    cols = []
    for _, V in blocks:
        for r in range(V.shape[0]):
            cols.extend(V[r])
    return np.array(cols).T


def block_operator(V_r: np.ndarray, H) -> np.ndarray:
    """The block V_r^dagger H V_r of one copy, V_r of shape [m, 2^n]."""
    HV = H @ V_r.T
    return V_r.conj() @ HV


def to_blocks(blocks, psi: np.ndarray):
    """Block coordinates of a full-space state: list over blocks of arrays [m, copies]."""
    return [np.stack([V[r].conj() @ psi for r in range(V.shape[0])], axis=1) for _, V in blocks]


def from_blocks(blocks, coords) -> np.ndarray:
    """Inverse of to_blocks."""
    psi = np.zeros(blocks[0][1].shape[2], dtype=np.complex128)
    for (_, V), c in zip(blocks, coords):
        for r in range(V.shape[0]):
            psi += V[r].T @ c[:, r]
    return psi


def symmetry_blocks(system):
    """The oracle's own adapted basis for a System: S_n or D_n by its group field."""
    return sn_blocks(system.n) if system.group == 0 else dn_blocks(system.n)


def block_problem(system, H0, Hc, blocks, psi0, psif, tol: float = 1e-13):
    """Restrict a full-space problem to the blocks where both psi0 and psif have support.

    Returns a list of dicts {h0, hc:[...], psi0:[m, c], psif:[m, c]} with only the copies that
    carry amplitude in both states (others cannot contribute to <psif|U|psi0>)."""
    c0 = to_blocks(blocks, psi0)
    cf = to_blocks(blocks, psif)
    out = []
    for (label, V), a0, af in zip(blocks, c0, cf):
        keep = [r for r in range(V.shape[0])
                if np.linalg.norm(a0[:, r]) > tol and np.linalg.norm(af[:, r]) > tol]
        if not keep:
            continue
        Vr = V[0]
        out.append(dict(label=label,
                        h0=block_operator(Vr, H0),
                        hc=[block_operator(Vr, h) for h in Hc],
                        psi0=a0[:, keep], psif=af[:, keep]))
    return out
