"""GB300-native (sm_103a) lattice Boltzmann solver for Bingham fluids.

Two collision formulations from Regulski, Leonardi & Szumbarski
(arXiv:1610.01388): Papanastasiou regularisation with an explicitly updated
relaxation time (PR, Sec. 3.1) and the locally implicit model (IR, Sec. 2.3 and
3.2).  The hot path is a fused pull stream-and-collide CUDA kernel behind the C
ABI declared in include/bingham_lbm.h; ``paper_1610_01388_gb300.lbm`` is a thin
ctypes binding with the same names, and ``workloads`` holds the seeded input
generators.
"""
