"""GB300-native electrostatic FEM-PIC cycle (Veske et al., Phys. Rev. E 101,
053307, arXiv 1906.08125): field-emission injection, P1 field gather and
leapfrog push, tetrahedron-walk relocation, fixed-point charge deposition and
the preconditioned-CG Poisson solve, as hand-written CUDA for sm_103a behind a
C ABI (``libpicfem.so``).

Importing the package loads nothing; ``picfem`` holds the binding and loads
the CUDA library on first use.
"""
