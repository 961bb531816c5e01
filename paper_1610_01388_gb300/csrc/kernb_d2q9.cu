// Batch kernel instantiations for the D2Q9 lattice (a translation unit of its
// own, compiled in parallel with the single-domain kernels of kern_d2q9.cu).
#include "kernels.cuh"

BLBM_DEFINE_BATCH_LAUNCHERS(D2Q9)
