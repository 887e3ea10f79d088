"""Host-side pieces of the warm start: the pulse gauge used to canonicalise training targets is a
symmetry of F (checked with the oracle), and the feature map."""
import numpy as np

from oracle import grape as gr
from oracle import symmetry as sy
from paper_2309_05884_gb300 import inputs as I


def test_global_pulse_phase_is_a_symmetry():
    from paper_2309_05884_gb300 import warmstart as ws
    p = I.SnProblem(n=7, J=1.3, h=0.4, N=30, k_target=3, seed=5)
    Jz, Jp, Jm = sy.spin_matrices(p.n)
    m = p.n + 1
    p0 = np.zeros((m, 1), complex)
    p0[0] = 1
    pf = np.zeros((m, 1), complex)
    pf[p.k_target] = 1
    prob = [dict(h0=p.J * (2 * Jz @ Jz - p.n / 2 * np.eye(m)) + p.h * 2 * Jz, hc=[Jp + Jm, -1j * (Jp - Jm)],
                 psi0=p0, psif=pf)]
    u = I.pulses_uniform(1, p.N, 2)
    uc = ws.canonicalize(u)
    z = uc[:, 0] + 1j * uc[:, 1]
    assert abs(z.sum().imag) < 1e-12 and z.sum().real > 0
    assert abs(gr.fidelity(prob, u, 10.0 / p.N) - gr.fidelity(prob, uc, 10.0 / p.N)) < 1e-12
    F, _, g = gr.fidelity_and_grad(prob, u, 10.0 / p.N)
    assert F > 0 and np.abs(g).max() > 0


def test_features():
    from paper_2309_05884_gb300 import warmstart as ws
    f = ws.features([I.SnProblem(n=16, J=1.0, h=0.5, N=200, k_target=4, seed=0)])
    assert f.shape == (1, 4) and np.allclose(f[0], [0.5, 0.5, 0.5, 0.25])
