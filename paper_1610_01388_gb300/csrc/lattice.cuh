// Velocity sets of the four lattices (Sec. 4.1), c_s^2 = 1/3.
//
// Order used throughout the CUDA path and at the C ABI: index 0 is the rest
// velocity, then opposite pairs sit next to each other, i odd -> opp(i) = i+1.
// That puts the two members of every TRT pair (Sec. 2.1) in adjacent
// registers and lets the collision loop over pairs.  Weights are the textbook
// ones (the paper does not print them): they make the lattice moments
// isotropic to fourth order.
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
};

}  // namespace blbm
