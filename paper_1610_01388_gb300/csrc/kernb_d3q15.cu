// Batch kernel instantiations for the D3Q15 lattice (a translation unit of its
// own, compiled in parallel with the single-domain kernels of kern_d3q15.cu).
#include "kernels.cuh"

BLBM_DEFINE_BATCH_LAUNCHERS(D3Q15)
