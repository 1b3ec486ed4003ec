"""Plain FP64 CPU oracle of the electrostatic FEM-PIC cycle.

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke entry and the CPU
baseline of the benchmark; the CUDA library never imports it.
"""
