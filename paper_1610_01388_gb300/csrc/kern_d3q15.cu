// Kernel instantiations for the D3Q15 lattice (one translation unit per lattice
// so the build compiles them in parallel).
#include "kernels.cuh"

BLBM_DEFINE_LAUNCHERS(D3Q15)
