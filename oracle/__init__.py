"""Oracle for the symmetry-block GRAPE hot path — TEST INFRASTRUCTURE ONLY.

A plain, slow, FP64 CPU restatement of what the paper computes, written from the paper's
equations and shared with nothing on the CUDA side.  Only the tests, the package's smoke()
check and bench.py's CPU-baseline leg may import it; the product path never does.

Modules
- operators : Pauli strings and full 2^n-dimensional Hamiltonians (Sec. II.A, Eqs. H0WithCoupling, Hc)
- symmetry  : S_n and D_n adapted bases (Appendix A, Eqs. groupAlgebraElementsSn/Dn), block
              dimensions by characters, block Hamiltonians A^dagger H A
- grape     : piecewise-constant propagation (Eq. exppropagator), state-transfer fidelity
              (Eq. probability), exact and first-order (Eq. propagator_differentiation)
              gradients, finite differences, gradient ascent; the gate (trace) fidelity objective
- trotter   : the Trotterised propagator for per-qubit controls and its transformed form (Sec. IV,
              Eqs. propagator_cpl, propagator_cpl_transformed), trace fidelity of propagators
- mlp       : the warm-start network's forward and backward pass

Every function is pinned by a test in tests/ against values the paper prints (Table I) or
against closed forms and invariants; see each module's header.
"""
