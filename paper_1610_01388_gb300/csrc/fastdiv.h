// Division of cell indices by a fixed divisor with one multiply-high, add and
// shift (Granlund & Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, round-up method).  For a divisor d >= 1 pick
// s = ceil(log2 d) and m = floor(2^32 (2^s - d) / d) + 1 (< 2^32); then for
// every 0 <= n < 2^31:  n / d = (mulhi(n, m) + n) >> s.
// Host code builds the constants; the kernels only evaluate div().
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define BLBM_HD __host__ __device__ __forceinline__
#else
#define BLBM_HD inline
#endif

namespace blbm {

struct FastDiv {
    uint32_t d, m, s;

    static FastDiv make(uint32_t d) {
        FastDiv f{d, 0u, 0u};
        uint32_t s = 0;
        while ((uint64_t(1) << s) < d) ++s;
        f.s = s;
        f.m = uint32_t(((uint64_t(1) << 32) * ((uint64_t(1) << s) - d)) / d + 1);
        return f;
    }

    BLBM_HD uint32_t div(uint32_t n) const {
#if defined(__CUDA_ARCH__)
        const uint32_t hi = __umulhi(n, m);
#else
        const uint32_t hi = uint32_t((uint64_t(n) * m) >> 32);
#endif
        return (hi + n) >> s;
    }
};

}  // namespace blbm
