// Batch kernel instantiations for the D3Q27 lattice (a translation unit of its
// own, compiled in parallel with the single-domain kernels of kern_d3q27.cu).
#include "kernels.cuh"

BLBM_DEFINE_BATCH_LAUNCHERS(D3Q27)
