// Velocity sets of the four lattices (Sec. 4.1), c_s^2 = 1/3.
//
// Order used throughout the CUDA path and at the C ABI: index 0 is the rest
// velocity, then opposite pairs sit next to each other, i odd -> opp(i) = i+1.
// That puts the two members of every TRT pair (Sec. 2.1) in adjacent
// registers and lets the collision loop over pairs.  Weights are the textbook
// ones (the paper does not print them): they make the lattice moments
// isotropic to fourth order.
//
// w3f(i) are the FP32 constants used for 3 w_i in the odd (momentum
// carrying) part of the collision.  The floats nearest to 3 w_i do not sum
// to an exact first moment (sum_i 3 w_i c_ix^2 = 1 + O(1e-8) in binary), and
// that error would add or remove O(1e-8) of the momentum at every collision,
// a drift that accumulates linearly in time.  These values are the FP32
// numbers within 6e-8 of 3 w_i for which that sum is exactly 1 (checked at
// compile time below), so the odd equilibrium carries exactly the momentum.
#pragma once

namespace blbm {

template <int Q_, int D_> struct LatticeBase {
    static constexpr int Q = Q_;
    static constexpr int D = D_;
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
};

struct D2Q9 : LatticeBase<9, 2> {
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int t[9] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int t[9] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    __host__ __device__ static constexpr float w3f(int i) {
        return i == 0 ? 0.0f : (i < 5 ? 0x1.555556p-2f : 0x1.555554p-4f);
    }
};

struct D3Q15 : LatticeBase<15, 3> {
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int t[15] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int t[15] = {0, 0, 0, 1, -1, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int i) {
        constexpr int t[15] = {0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, 1, -1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 2.0 / 9.0 : (i < 7 ? 1.0 / 9.0 : 1.0 / 72.0);
    }
    __host__ __device__ static constexpr float w3f(int i) {
        return i == 0 ? 0.0f : (i < 7 ? 0x1.555556p-2f : 0x1.555554p-5f);
    }
};

struct D3Q19 : LatticeBase<19, 3> {
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int i) {
        constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    __host__ __device__ static constexpr float w3f(int i) {
        return i == 0 ? 0.0f : (i < 7 ? 0x1.555554p-3f : 0x1.555556p-4f);
    }
};

struct D3Q27 : LatticeBase<27, 3> {
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int t[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1,
                               0, 0, 0, 0, 1, -1, 1, -1, 1, -1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int t[27] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0,
                               1, -1, 1, -1, 1, -1, 1, -1, -1, 1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int i) {
        constexpr int t[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1,
                               1, -1, -1, 1, 1, -1, -1, 1, 1, -1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 8.0 / 27.0 : (i < 7 ? 2.0 / 27.0 : (i < 19 ? 1.0 / 54.0 : 1.0 / 216.0));
    }
    __host__ __device__ static constexpr float w3f(int i) {
        return i == 0 ? 0.0f : (i < 7 ? 0x1.c71c72p-3f : (i < 19 ? 0x1.c71c72p-5f : 0x1.c71c70p-7f));
    }
};

// 3 w_i for the odd part in arithmetic type R (exact double for FP64).
template <class L, class R> __host__ __device__ constexpr R odd_w(int i) {
    if constexpr (sizeof(R) == 4)
        return L::w3f(i);
    else
        return 3.0 * L::w(i);
}

// Exactness of the FP32 odd weights: sum_i w3f_i c_ia^2 == 1 for every axis
// (sums of these floats are exact in double).
template <class L> constexpr bool odd_weights_exact() {
    for (int a = 0; a < L::D; ++a) {
        double s = 0.0;
        for (int i = 0; i < L::Q; ++i) {
            const int c = a == 0 ? L::cx(i) : (a == 1 ? L::cy(i) : L::cz(i));
            s += double(c * c) * double(L::w3f(i));
        }
        if (s != 1.0) return false;
    }
    for (int i = 1; i < L::Q; ++i) {
        const double d = double(L::w3f(i)) / (3.0 * L::w(i)) - 1.0;
        if (d > 1e-7 || d < -1e-7) return false;
    }
    return true;
}
static_assert(odd_weights_exact<D2Q9>(), "D2Q9 odd weights");
static_assert(odd_weights_exact<D3Q15>(), "D3Q15 odd weights");
static_assert(odd_weights_exact<D3Q19>(), "D3Q19 odd weights");
static_assert(odd_weights_exact<D3Q27>(), "D3Q27 odd weights");

}  // namespace blbm
