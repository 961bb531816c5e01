// Kernel instantiations for the D2Q9 lattice (one translation unit per lattice
// so the build compiles them in parallel).
#include "kernels.cuh"

BLBM_DEFINE_LAUNCHERS(D2Q9)
