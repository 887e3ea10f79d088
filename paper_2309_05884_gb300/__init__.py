"""Symmetry-block GRAPE on one GB300: a C-ABI CUDA library (libqoc.so) and its Python binding.

- paper_2309_05884_gb300.api     : Basis, Plan, FidelityGrad (binding of include/qoc.h)
- paper_2309_05884_gb300.inputs  : seeded synthetic systems, pulses and states
- paper_2309_05884_gb300.build   : compiles libqoc.so in-tree for sm_103a
"""
__all__ = ["api", "inputs", "build"]
