"""Trotterised propagation with per-qubit controls on the GPU (Sec. IV, Eqs. propagator_cpl and
propagator_cpl_transformed) against the oracle's Trotterised propagator, element by element on the
full-space propagator K (FP64, 1e-11); exactness without coupling; the second-order convergence of
the infidelity against the original propagator; the coupling factor from the D_n blocks."""
import numpy as np
import pytest

from oracle import trotter as tr
from paper_2309_05884_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2309_05884_gb300 import _lib, api  # noqa: E402

DEV = torch.device("cuda", 0)
BZ, T = 1.0, 2.0


def smooth_pulses(seed, n, N):
    """Bx, By per qubit: a cos(w t + phi) at the slice midpoints (seeded a, w, phi)."""
    g = I.rng(seed)
    amp = g.uniform(0.5, 1.5, (2, n))
    w = g.uniform(0.5, 2.0, (2, n))
    ph = g.uniform(0.0, 2 * np.pi, (2, n))
    t = (np.arange(N) + 0.5) * T / N
    return [amp[a] * np.cos(w[a] * t[:, None] + ph[a]) for a in range(2)]


def coupling_basis(n, c):
    # H_cpl = c/4 sum_i Z_i Z_{i+1} (Eq. completeH_cpl); one control term is required and not used
    s = I.System(n, I.GROUP_DN, [(I.RING_ZZ, c / 4.0, 1)], [[(I.SUM_Z, 1.0, 0)]], T, 1)
    return api.Basis(s)


def gpu_K(n, c, bx, by, tau):
    N = bx.shape[0]
    pl = np.zeros((N, n, 3))
    pl[:, :, 0] = BZ
    pl[:, :, 1] = bx
    pl[:, :, 2] = by
    trot = api.Trotter(coupling_basis(n, c), tau)
    eye = torch.eye(2 ** n, dtype=torch.complex128, device=DEV)  # rows = columns of the identity
    out = trot.propagate(torch.from_numpy(pl).to(DEV), eye.contiguous())
    torch.cuda.synchronize()
    return out.cpu().numpy().T  # column c of K = U (e_c)


@pytest.mark.parametrize("n,N", [(4, 6), (5, 5), (6, 4), (8, 2)])
def test_trotter_propagator_matches_oracle(n, N):
    c = 0.8
    bx, by = smooth_pulses(2, n, N)
    tau = T / N
    Kg = gpu_K(n, c, bx, by, tau)
    Ec = tr.coupling_factor_by_blocks(n, c, tau)
    Ko = tr.evolve(lambda *a: tr.trotter_step_transformed(*a, coupling_factor=Ec), n, BZ, c, bx, by, tau)
    assert np.abs(Kg - Ko).max() <= 1e-11
    assert np.abs(Kg.conj().T @ Kg - np.eye(2 ** n)).max() <= 1e-11


def test_exact_without_coupling():
    n, N = 5, 8
    bx, by = smooth_pulses(1, n, N)
    tau = T / N
    Kg = gpu_K(n, 0.0, bx, by, tau)
    Ko = tr.evolve(tr.original_step, n, BZ, 0.0, bx, by, tau)
    assert np.abs(Kg - Ko).max() <= 1e-11


def test_infidelity_second_order_against_original():
    n = 4
    infid = []
    for N in (20, 40, 80):
        bx, by = smooth_pulses(5, n, N)
        tau = T / N
        Kg = gpu_K(n, 0.8, bx, by, tau)
        Ko = tr.evolve(tr.original_step, n, BZ, 0.8, bx, by, tau)
        infid.append(1.0 - tr.trace_fidelity(Kg, Ko))
    assert infid[0] > 1e-5
    for a, b in zip(infid, infid[1:]):
        assert 3.8 < a / b < 4.2


def test_trotter_rejects_bad_bases():
    s = I.System(4, I.GROUP_DN, [(I.RING_ZZ, 0.2, 1)], [[(I.SUM_Z, 1.0, 0)]], T, 1)
    with pytest.raises(_lib.QocError):
        api.Trotter(api.Basis(s, first_block_only=True), 0.1)
    with pytest.raises(_lib.QocError):
        api.Trotter(api.Basis(s), -1.0)
