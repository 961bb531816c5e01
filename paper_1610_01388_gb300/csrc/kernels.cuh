// Fused pull stream-and-collide kernels for the PR and IR Bingham models.
//
// One thread owns one cell (k_step; k_step2 runs two cells per thread with
// the collision in packed two-wide FP32).  Per fluid cell and time step it
//   1. gathers the Q incoming populations (eq. 8, pull form): population i
//      comes from the cell at x - c_i (periodic wrap) or, when that cell is
//      solid, is the cell's own outgoing population in the opposite direction
//      (halfway bounce-back, Sec. 4.3);
//   2. forms the moments rho, j, Pi (eq. MomentsLBM) in registers;
//   3. collides:
//      PR  T = Pi - rho c_s^2 I - rho u u, D = -T/(2 tau_old c_s^2)
//          (eq. LBM_strain_rate), gdot = sqrt(2 D:D), nu_app from eqs.
//          (Pap_reg_1)/(PR_interpolation), tau = 1/2 + nu_app/c_s^2
//          (eq. tau_visc), or the Newton-implicit tau of Sec. 3; TRT with
//          tau_odd from Lambda (Sec. 2.1) and the exact-difference force of
//          eq. (14);
//      IR  u = (j + F/2)/rho, T as above, the closed-form solution of
//          eq. (Vikh_main_short) (eqs. Vikh_sigmaS_formula/tensor, yield where
//          |T| >= sqrt2 sigma_y), A = -sigma_bar + s/2, and the post-collision
//          populations f_eq + w/(2 c_s^4)(cc - c_s^2 I):A + Phi/2 of
//          eqs. (Vikh_postCol)/(Vikh_f_stress)/(Vikh_force);
//   4. stores the Q outgoing populations (and, PR, the new tau in place).
//
// Populations are stored as offsets f_i - w_i from the rest state (scaled per
// direction for the 16-bit forms), so every moment is formed from small
// numbers (no cancellation against the weights).  On check steps the same
// launch also accumulates the flow-rate sums and the residual against the
// previous snapshot into per-block partials, summed in FP64 in a fixed order.
#pragma once

#include <algorithm>
#include <cstdint>
#include <type_traits>
#include <utility>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/bingham_lbm.h"
#include "lattice.cuh"
#include "lbm_internal.h"

namespace blbm {

// ---------------------------------------------------------------------------
// compile-time loop
template <int I, int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, N>(std::forward<F>(f));
    }
}

// Sums with compile-time integer coefficients.  Terms with a zero
// coefficient are left out entirely (IEEE arithmetic forbids the compiler to
// drop 0 * x or x + 0 by itself), +-1 become adds and subtracts.
template <class R, bool Started> struct CSum {
    R v;
};

template <int c, class R, bool S>
__device__ __forceinline__ auto cadd(CSum<R, S> a, R x) {
    if constexpr (c == 0) {
        return a;
    } else if constexpr (!S) {
        if constexpr (c == 1) return CSum<R, true>{x};
        else if constexpr (c == -1) return CSum<R, true>{-x};
        else return CSum<R, true>{R(c) * x};
    } else {
        if constexpr (c == 1) return CSum<R, true>{a.v + x};
        else if constexpr (c == -1) return CSum<R, true>{a.v - x};
        else return CSum<R, true>{a.v + R(c) * x};
    }
}

template <class R, bool S> __device__ __forceinline__ R cval(CSum<R, S> a) {
    if constexpr (S) return a.v;
    else return R(0);
}

// a x + b y + c z
template <int a, int b, int c, class R>
__device__ __forceinline__ R cdot(R x, R y, R z) {
    return cval(cadd<c>(cadd<b>(cadd<a>(CSum<R, false>{R(0)}, x), y), z));
}

// a x + b y + c z + d p + e q + g r
template <int a, int b, int c, int d, int e, int g, class R>
__device__ __forceinline__ R cdot6(R x, R y, R z, R p, R q, R r) {
    return cval(cadd<g>(cadd<e>(cadd<d>(cadd<c>(cadd<b>(cadd<a>(CSum<R, false>{R(0)}, x), y), z), p), q), r));
}

// ---------------------------------------------------------------------------
// Random bits for stochastic rounding.  Per cell and launch one hash of
// (cell index, launch counter) with the PCG-based hash of Jarzynski & Olano,
// "Hash Functions for GPU Rendering" (JCGT 9(3), 2020).  Population pair p
// takes that word times a distinct odd constant (a bijection of 32-bit words,
// so every pair's word is exactly as uniform as the hash; one multiply).
__device__ __forceinline__ uint32_t pcg_hash(uint32_t v) {
    const uint32_t state = v * 747796405u + 2891336453u;
    const uint32_t word = ((state >> ((state >> 28u) + 4u)) ^ state) * 277803737u;
    return (word >> 22u) ^ word;
}
template <int p>
__device__ __forceinline__ uint32_t pair_bits(uint32_t h) {
    constexpr uint32_t k = 0x9e3779b9u * uint32_t(2 * p + 1);   // odd
    return h * k;
}
// Hardware stochastic rounding of two FP32 values to a packed 16-bit pair
// (PTX cvt.rs, sm_100a and later): the high half holds `hi`, the low half
// `lo`; rbits supplies the random bits.
__device__ __forceinline__ uint32_t cvt_rs_f16x2(float hi, float lo, uint32_t rbits) {
    uint32_t d;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
    return d;
}
__device__ __forceinline__ uint32_t cvt_rs_bf16x2(float hi, float lo, uint32_t rbits) {
    uint32_t d;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
    return d;
}
__device__ __forceinline__ void st_u16(void* p, uint32_t v) { *reinterpret_cast<uint16_t*>(p) = (uint16_t)v; }

// ---------------------------------------------------------------------------
// Two cells in one register pair.  F2 holds one FP32 quantity of two cells;
// its +, -, * issue the packed f32x2 forms (PTX add/sub/mul/fma .f32x2,
// sm_100a and later): one instruction for both cells.  A product stays
// unevaluated (F2P) until it is used, so a following add or subtract becomes
// one fused multiply-add, the contraction nvcc applies to scalar code.
struct F2 {
    unsigned long long v;
    F2() = default;
    __device__ __forceinline__ F2(float a) { asm("mov.b64 %0, {%1, %1};" : "=l"(v) : "f"(a)); }
    __device__ __forceinline__ F2(double a) : F2((float)a) {}
    __device__ __forceinline__ F2(int a) : F2((float)a) {}
    __device__ __forceinline__ F2(float a, float b) { asm("mov.b64 %0, {%1, %2};" : "=l"(v) : "f"(a), "f"(b)); }
    __device__ __forceinline__ float lo() const { return __uint_as_float((unsigned)v); }
    __device__ __forceinline__ float hi() const { return __uint_as_float((unsigned)(v >> 32)); }
};
__device__ __forceinline__ F2 f2_bits(unsigned long long b) {
    F2 r;
    r.v = b;
    return r;
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a.v), "l"(b.v));
    return f2_bits(d);
}
__device__ __forceinline__ F2 f2_sub(F2 a, F2 b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a.v), "l"(b.v));
    return f2_bits(d);
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a.v), "l"(b.v));
    return f2_bits(d);
}
__device__ __forceinline__ F2 f2_fma(F2 a, F2 b, F2 c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a.v), "l"(b.v), "l"(c.v));
    return f2_bits(d);
}
__device__ __forceinline__ F2 operator-(F2 a) { return f2_bits(a.v ^ 0x8000000080000000ull); }
struct F2P {   // a * b, not yet rounded
    F2 a, b;
    __device__ __forceinline__ operator F2() const { return f2_mul(a, b); }
};
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return f2_add(a, b); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return f2_sub(a, b); }
__device__ __forceinline__ F2P operator*(F2 a, F2 b) { return F2P{a, b}; }
__device__ __forceinline__ F2P operator*(F2P p, F2 b) { return F2P{F2(p), b}; }
__device__ __forceinline__ F2P operator*(F2 a, F2P p) { return F2P{a, F2(p)}; }
__device__ __forceinline__ F2P operator*(F2P p, F2P q) { return F2P{F2(p), F2(q)}; }
__device__ __forceinline__ F2 operator+(F2P p, F2 c) { return f2_fma(p.a, p.b, c); }
__device__ __forceinline__ F2 operator+(F2 c, F2P p) { return f2_fma(p.a, p.b, c); }
__device__ __forceinline__ F2 operator-(F2 c, F2P p) { return f2_fma(-p.a, p.b, c); }
__device__ __forceinline__ F2 operator-(F2P p, F2 c) { return f2_fma(p.a, p.b, -c); }
__device__ __forceinline__ F2 operator+(F2P p, F2P q) { return f2_fma(p.a, p.b, F2(q)); }
__device__ __forceinline__ F2 operator-(F2P p, F2P q) { return f2_fma(p.a, p.b, -F2(q)); }
__device__ __forceinline__ F2P operator-(F2P p) { return F2P{-p.a, p.b}; }
__device__ __forceinline__ F2& operator+=(F2& a, F2 b) { return a = a + b; }
__device__ __forceinline__ F2& operator-=(F2& a, F2 b) { return a = a - b; }
__device__ __forceinline__ F2& operator+=(F2& a, F2P p) { return a = a + p; }

// The scalar type of an arithmetic type, and lane access: the parts of the
// collision with no packed form (sqrt, divisions, expm1, branches) run per
// cell on the lanes.
template <class R> struct Lanes {
    using Sc = R;
    static constexpr int n = 1;
    __device__ __forceinline__ static R get(R x, int) { return x; }
    __device__ __forceinline__ static R make(const R (&v)[1]) { return v[0]; }
};
template <> struct Lanes<F2> {
    using Sc = float;
    static constexpr int n = 2;
    __device__ __forceinline__ static float get(F2 x, int k) { return k ? x.hi() : x.lo(); }
    __device__ __forceinline__ static F2 make(const float (&v)[2]) { return F2(v[0], v[1]); }
};
__device__ __forceinline__ float recip(float x) { return 1.0f / x; }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ F2 recip(F2 x) { return F2(1.0f / x.lo(), 1.0f / x.hi()); }

// ---------------------------------------------------------------------------
// storage.  R is the arithmetic type.  ld / st move population i between
// memory and registers; enc / dec convert full FP64 populations at the ABI
// (set/get populations).
//
// The 16-bit forms store the offset normalised by its lattice weight,
// (f_i - w_i) / w_i, which is O(Ma) in every direction; FP16 also scales it
// by 2^14 (exact) so offsets down to ~4e-9 stay out of FP16's subnormal range
// while |(f_i - w_i)/w_i| up to 4 stays below its largest finite value.
template <class S> struct Store;
//
// The collision works on populations in MEMORY UNITS x_i = alpha_i (f_i - w_i),
// so loads and stores need no scaling.  Three per-direction constants carry
// the units: beta_i = 1 / alpha_i turns x_i into an offset (moments),
// gam_i = alpha_i w_i scales the equilibrium-type terms (which all carry a
// factor w_i) and god_i = alpha_i 3 w_i their odd part.  For the 16-bit forms
// alpha_i is proportional to 1 / w_i, so gam_i and god_i are the same for
// every direction and the weights drop out of the collision arithmetic.
template <> struct Store<float> {
    using R = float;
    template <class L, int i> __host__ __device__ static constexpr R beta() { return 1.0f; }
    template <class L, int i> __host__ __device__ static constexpr R gam() { return R(L::w(i)); }
    template <class L, int i> __host__ __device__ static constexpr R god() { return L::w3f(i); }
    template <class L, int i> static __device__ __forceinline__ R ld(const float* p) { return __ldg(p); }
    static constexpr bool kStochastic = false;
    template <class L, int i> static __device__ __forceinline__ void st(float* p, R v, uint32_t) { *p = v; }
    template <class L, int i>
    static __device__ __forceinline__ void st2(float* pi, float* po, R vi, R vo, uint32_t) { *pi = vi; *po = vo; }
    static __device__ __forceinline__ float enc(double off, double) { return (float)off; }
    static __device__ __forceinline__ double dec(float v, double) { return (double)v; }
};
template <> struct Store<double> {
    using R = double;
    template <class L, int i> __host__ __device__ static constexpr R beta() { return 1.0; }
    template <class L, int i> __host__ __device__ static constexpr R gam() { return L::w(i); }
    template <class L, int i> __host__ __device__ static constexpr R god() { return 3.0 * L::w(i); }
    template <class L, int i> static __device__ __forceinline__ R ld(const double* p) { return __ldg(p); }
    static constexpr bool kStochastic = false;
    template <class L, int i> static __device__ __forceinline__ void st(double* p, R v, uint32_t) { *p = v; }
    template <class L, int i>
    static __device__ __forceinline__ void st2(double* pi, double* po, R vi, R vo, uint32_t) { *pi = vi; *po = vo; }
    static __device__ __forceinline__ double enc(double off, double) { return off; }
    static __device__ __forceinline__ double dec(double v, double) { return v; }
};
template <> struct Store<__half> {
    using R = float;
    static constexpr double kScale = 16384.0;   // 2^14: alpha_i = 2^14 / w_i
    template <class L, int i> __host__ __device__ static constexpr R beta() { return float(L::w(i) / kScale); }
    template <class L, int i> __host__ __device__ static constexpr R gam() { return float(kScale); }
    template <class L, int i> __host__ __device__ static constexpr R god() { return float(3.0 * kScale); }
    template <class L, int i> static __device__ __forceinline__ R ld(const __half* p) {
        return __half2float(__ldg(p));
    }
    static constexpr bool kStochastic = true;
    // stochastic rounding (unbiased: a value moves by less than half an ulp per
    // step in slowly relaxing flows, and round-to-nearest would freeze it)
    template <class L, int i> static __device__ __forceinline__ void st(__half* p, R v, uint32_t rnd) {
        st_u16(p, cvt_rs_f16x2(v, 0.0f, rnd) >> 16);
    }
    // populations i and its opposite (same weight) in one conversion
    template <class L, int i>
    // pi and po = pi + 1 are the two halves of one 4-byte-aligned word (the
    // interleaved pair layout): f_i in the low half, f_o in the high half
    static __device__ __forceinline__ void st2(__half* pi, __half*, R vi, R vo, uint32_t rnd) {
        *reinterpret_cast<uint32_t*>(pi) = cvt_rs_f16x2(vo, vi, rnd);
    }
    static __device__ __forceinline__ __half enc(double off, double w) { return __double2half(off / w * kScale); }
    static __device__ __forceinline__ double dec(__half v, double w) { return (double)__half2float(v) * (w / kScale); }
};
template <> struct Store<__nv_bfloat16> {
    using R = float;   // alpha_i = 1 / w_i
    template <class L, int i> __host__ __device__ static constexpr R beta() { return float(L::w(i)); }
    template <class L, int i> __host__ __device__ static constexpr R gam() { return 1.0f; }
    template <class L, int i> __host__ __device__ static constexpr R god() { return 3.0f; }
    template <class L, int i> static __device__ __forceinline__ R ld(const __nv_bfloat16* p) {
        return __bfloat162float(__ldg(p));
    }
    static constexpr bool kStochastic = true;
    template <class L, int i> static __device__ __forceinline__ void st(__nv_bfloat16* p, R v, uint32_t rnd) {
        st_u16(p, cvt_rs_bf16x2(v, 0.0f, rnd) >> 16);
    }
    template <class L, int i>
    static __device__ __forceinline__ void st2(__nv_bfloat16* pi, __nv_bfloat16*, R vi, R vo,
                                               uint32_t rnd) {
        *reinterpret_cast<uint32_t*>(pi) = cvt_rs_bf16x2(vo, vi, rnd);
    }
    static __device__ __forceinline__ __nv_bfloat16 enc(double off, double w) { return __double2bfloat16(off / w); }
    static __device__ __forceinline__ double dec(__nv_bfloat16 v, double w) { return (double)__bfloat162float(v) * w; }
};

// Rheology constants in the arithmetic type, derived on the host in FP64.
template <class R> struct Coef {
    R nu_p, sigma_y, m, gdot_c, inv_gc, e_c, magic;
    R g[3];
    R s2y;     // sqrt(2) sigma_y
    R ir_a;    // 1 / (1/2 + 3 nu_p)
    R ir_b;    // 1 / (1 + 6 nu_p)
    R six_nu;  // 6 nu_p
    int newton;  // PR: Newton iterations of the implicit tau update
    R cg[13];   // c_i . g of direction i = 2p + 1 (PR force terms), per pair p
    R cgg[13];  // (c_i . g)^2
};

struct KArgs {
    KParams kp;
    Coef<float> cf;
    Coef<double> cd;
};

template <class R> __device__ __forceinline__ const Coef<R>& coef(const KArgs& a);
template <> __device__ __forceinline__ const Coef<float>& coef<float>(const KArgs& a) { return a.cf; }
template <> __device__ __forceinline__ const Coef<double>& coef<double>(const KArgs& a) { return a.cd; }

// Base pointer of every population plane, passed by value in the kernel
// parameters: an address is then one multiply-add of the 32-bit cell index.
// Population layout.  FP32 / FP64: plane i holds population i of every cell.
// 16-bit forms: the rest population has plane 0; an opposite pair (i, i + 1),
// i odd, shares planes i and i + 1 as one plane of 32-bit words holding f_i
// in the low and f_{i+1} in the high half of cell n's word, so the pair's
// packed stochastic-rounding result is one aligned 32-bit store.  Element
// (i, n) is at pop_base(i) + pop_step(i) n; the total is Q planes either way.
template <class S> __host__ __device__ constexpr bool pairs_interleaved() { return sizeof(S) == 2; }
template <class S> __host__ __device__ constexpr int64_t pop_base(int i, int64_t plane) {
    return (!pairs_interleaved<S>() || i == 0) ? i * plane : (i - ((i - 1) & 1)) * plane + ((i - 1) & 1);
}
template <class S> __host__ __device__ constexpr int pop_step(int i) {
    return (pairs_interleaved<S>() && i > 0) ? 2 : 1;
}

template <class S> struct SrcPlanes {
    const S* p[27];   // p[i] = buffer + pop_base(i)
    template <int i> __device__ __forceinline__ const S* at(int n) const {
        return p[i] + (int64_t)pop_step<S>(i) * n;
    }
};
template <class S> struct DstPlanes {
    S* p[27];
    template <int i> __device__ __forceinline__ S* at(int n) const {
        return p[i] + (int64_t)pop_step<S>(i) * n;
    }
};
// Planes of one buffer addressed by a stride (batched launches, where the
// pointers differ per domain), in 32-bit arithmetic (the batch admits only
// domains with Q * plane < 2^31, and every element index is below that).
template <class S> struct SrcStride {
    const S* base;
    int plane;
    template <int i> __device__ __forceinline__ const S* at(int n) const {
        return base + ((int)pop_base<S>(i, plane) + pop_step<S>(i) * n);
    }
};
template <class S> struct DstStride {
    S* base;
    int plane;
    template <int i> __device__ __forceinline__ S* at(int n) const {
        return base + ((int)pop_base<S>(i, plane) + pop_step<S>(i) * n);
    }
};

// cell index -> (x, y, z)
__device__ __forceinline__ void cell_xyz(const KParams& kp, int idx, int& x, int& y, int& z) {
    const uint32_t t = kp.div_nx.div((uint32_t)idx);
    x = idx - (int)t * kp.nx;
    z = (int)kp.div_ny.div(t);
    y = (int)t - z * kp.ny;
}

// ---------------------------------------------------------------------------
// streaming (pull) with halfway bounce-back
// 1: the gather path is chosen per warp (see gather); 0 restores the
// per-thread choice, for comparison builds.
#ifndef BLBM_WARP_UNIFORM_GATHER
#define BLBM_WARP_UNIFORM_GATHER 1
#endif
// Offsets from a cell's index to its pull sources x - c (periodic wrap):
// m for a velocity component +1, p for -1.
struct PullOffsets {
    int dxm, dxp, dym, dyp, dzm, dzp;
    template <class L, int i> __device__ __forceinline__ int of() const {
        constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        int off = 0;
        if constexpr (cx > 0) off += dxm;
        if constexpr (cx < 0) off += dxp;
        if constexpr (cy > 0) off += dym;
        if constexpr (cy < 0) off += dyp;
        if constexpr (cz > 0) off += dzm;
        if constexpr (cz < 0) off += dzp;
        return off;
    }
};

__device__ __forceinline__ PullOffsets pull_offsets(const KParams& kp, int idx) {
    const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
    int x, y, z;
    cell_xyz(kp, idx, x, y, z);
    const int sy = nx, sz = nx * ny;
    PullOffsets o;
    o.dxm = (x == 0) ? nx - 1 : -1;
    o.dxp = (x == nx - 1) ? -(nx - 1) : 1;
    o.dym = (y == 0) ? (ny - 1) * sy : -sy;
    o.dyp = (y == ny - 1) ? -(ny - 1) * sy : sy;
    o.dzm = (z == 0) ? (nz - 1) * sz : -sz;
    o.dzp = (z == nz - 1) ? -(nz - 1) * sz : sz;
    return o;
}

// self = true loads the cell's own populations, plane by plane (all offsets
// 0; lk must be 0): the copy-through of a solid cell.
template <class L, class S, class Src>
__device__ __forceinline__ void gather(const KParams& kp, const Src& P, uint32_t lk,
                                       int idx, typename Store<S>::R (&v)[L::Q],
                                       bool self = false) {
    PullOffsets o = pull_offsets(kp, idx);
    if (self) o = PullOffsets{0, 0, 0, 0, 0, 0};
    auto offset = [&](auto I) { return o.template of<L, decltype(I)::value>(); };
    // The path is chosen per warp: a warp takes the plain pull only when none
    // of its cells has a solid neighbour.  A per-thread choice makes a warp
    // that mixes wall and interior cells run both paths one after the other,
    // which is most warps in a porous medium; the select path is exact for
    // interior cells too (their link bits are 0).
#if BLBM_WARP_UNIFORM_GATHER
    const bool plain = __all_sync(__activemask(), lk == 0u);
#else
    const bool plain = lk == 0u;
#endif
    if (plain) {
        // no solid neighbour: plain pull, no per-population selects
        static_for<0, L::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            v[i] = Store<S>::template ld<L, i>(P.template at<i>(idx + offset(I)));
        });
    } else {
        static_for<0, L::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const S* p = ((lk >> i) & 1u) ? P.template at<L::opp(i)>(idx)
                                          : P.template at<i>(idx + offset(I));
            v[i] = Store<S>::template ld<L, i>(p);   // opposite planes share w_i
        });
    }
}

// ---------------------------------------------------------------------------
// moments of the offsets: d = sum df, j = sum c df, p = sum c c df
template <class R> struct Mom {
    R d, jx, jy, jz, xx, yy, zz, xy, xz, yz;
};

// Grouped sums: populations are added once per velocity class (c_x = +1, -1,
// 0; c_y = +-1; c_z = +-1; sign of c_x c_y, c_x c_z, c_y c_z) and the moments
// are sums and differences of those class sums.  Each class sum starts as its
// first member (no add to a zero).  f is in memory units; beta_i turns each
// value into an offset.  Where beta_i != 1 it is applied inside each class
// sum's multiply-add (one instruction per class membership, no separate
// multiply per population).
enum { kXp, kXm, kX0, kYp, kYm, kZp, kZm, kPxy, kMxy, kPxz, kMxz, kPyz, kMyz, kNumClasses };

__host__ __device__ constexpr bool in_class(int k, int cx, int cy, int cz) {
    return k == kXp ? cx == 1 : k == kXm ? cx == -1 : k == kX0 ? cx == 0
         : k == kYp ? cy == 1 : k == kYm ? cy == -1 : k == kZp ? cz == 1 : k == kZm ? cz == -1
         : k == kPxy ? cx * cy == 1 : k == kMxy ? cx * cy == -1
         : k == kPxz ? cx * cz == 1 : k == kMxz ? cx * cz == -1
         : k == kPyz ? cy * cz == 1 : cy * cz == -1;
}
template <class L> __host__ __device__ constexpr int first_in_class(int k) {
    for (int i = 0; i < L::Q; ++i)
        if (in_class(k, L::cx(i), L::cy(i), L::cz(i))) return i;
    return -1;
}

template <class L, class S, class R = typename Store<S>::R>
__device__ __forceinline__ Mom<R> moments(const R (&f)[L::Q]) {
    R acc[kNumClasses];
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        constexpr auto beta = Store<S>::template beta<L, i>();
        static_for<0, kNumClasses>([&](auto K) {
            constexpr int k = decltype(K)::value;
            if constexpr (in_class(k, cx, cy, cz)) {
                if constexpr (beta == 1) {
                    if constexpr (first_in_class<L>(k) == i) acc[k] = f[i];
                    else acc[k] += f[i];
                } else {
                    if constexpr (first_in_class<L>(k) == i) acc[k] = R(f[i] * R(beta));
                    else acc[k] = acc[k] + f[i] * R(beta);
                }
            }
        });
    });
    Mom<R> m;
    m.xx = acc[kXp] + acc[kXm];
    m.jx = acc[kXp] - acc[kXm];
    m.d = m.xx + acc[kX0];
    m.yy = acc[kYp] + acc[kYm];
    m.jy = acc[kYp] - acc[kYm];
    m.xy = acc[kPxy] - acc[kMxy];
    if constexpr (L::D == 3) {
        m.zz = acc[kZp] + acc[kZm];
        m.jz = acc[kZp] - acc[kZm];
        m.xz = acc[kPxz] - acc[kMxz];
        m.yz = acc[kPyz] - acc[kMyz];
    } else {
        m.zz = R(0);
        m.jz = R(0);
        m.xz = R(0);
        m.yz = R(0);
    }
    return m;
}

// Non-equilibrium second moment T = Pi - rho c_s^2 I - rho u u written with
// offsets: Pi = c_s^2 I + p, rho = 1 + d.
template <class R> struct Tens {
    R xx, yy, zz, xy, xz, yz;
};

template <class L, class R>
__device__ __forceinline__ Tens<R> noneq(const Mom<R>& m, R rho, R ux, R uy, R uz, uint32_t flags) {
    const R d3 = m.d * R(1.0 / 3.0);
    Tens<R> t;
    t.xx = m.xx - d3 - rho * ux * ux;
    t.yy = m.yy - d3 - rho * uy * uy;
    t.xy = m.xy - rho * ux * uy;
    if constexpr (L::D == 3) {
        t.zz = m.zz - d3 - rho * uz * uz;
        t.xz = m.xz - rho * ux * uz;
        t.yz = m.yz - rho * uy * uz;
    } else {
        t.zz = R(0);
        t.xz = R(0);
        t.yz = R(0);
    }
    if (flags & LBM_FLAG_BURNETT_X) t.xx = R(0);
    return t;
}

template <class L, class R> __device__ __forceinline__ R tnorm2(const Tens<R>& T) {
    R s = T.xx * T.xx + T.yy * T.yy + R(2) * T.xy * T.xy;
    if constexpr (L::D == 3) s += T.zz * T.zz + R(2) * (T.xz * T.xz + T.yz * T.yz);
    return s;
}

// c.T.c for a lattice velocity, from T and the doubled off-diagonals
template <int cx, int cy, int cz, class R>
__device__ __forceinline__ R ctc(const Tens<R>& T, R t2xy, R t2xz, R t2yz) {
    return cdot6<cx * cx, cy * cy, cz * cz, cx * cy, cx * cz, cy * cz>(T.xx, T.yy, T.zz, t2xy,
                                                                        t2xz, t2yz);
}

// ---------------------------------------------------------------------------
// IR yield solve, per cell: s = as T, sigma = asg T (eq. Vikh_sigmaS_tensor)
// from |T|^2.
template <class R>
__device__ __forceinline__ void ir_yield(const Coef<typename Lanes<R>::Sc>& c, R tn2, R& as_out,
                                         R& asg_out) {
    using Sc = typename Lanes<R>::Sc;
    Sc as[Lanes<R>::n], asg[Lanes<R>::n];
#pragma unroll
    for (int k = 0; k < Lanes<R>::n; ++k) {
        const Sc tn = sqrt(Lanes<R>::get(tn2, k));
        as[k] = Sc(0);
        asg[k] = Sc(-1);
        if (tn > Sc(0) && tn >= c.s2y) {
            const Sc it = Sc(1) / tn;
            as[k] = -(tn - c.s2y) * c.ir_a * it;
            asg[k] = -(c.six_nu * tn + c.s2y) * c.ir_b * it;
        }
    }
    as_out = Lanes<R>::make(as);
    asg_out = Lanes<R>::make(asg);
}

// ---------------------------------------------------------------------------
// IR collision (Secs. 2.3, 3.2).  f: memory units in, memory units out.  R is
// the arithmetic type: one cell (float, double) or two cells (F2).
template <class L, class S, class R = typename Store<S>::R>
__device__ __forceinline__ void collide_ir(const Coef<typename Lanes<R>::Sc>& c, uint32_t flags,
                                           R (&f)[L::Q], R& drho, R (&ur)[3]) {
    const Mom<R> m = moments<L, S, R>(f);
    const R rho = R(1) + m.d;
    const R inv = recip(rho);
    const R Fx = rho * R(c.g[0]), Fy = rho * R(c.g[1]);
    R Fz = R(0);
    if constexpr (L::D == 3) Fz = rho * R(c.g[2]);
    const R ux = (m.jx + R(0.5) * Fx) * inv;
    const R uy = (m.jy + R(0.5) * Fy) * inv;
    R uz = R(0);
    if constexpr (L::D == 3) uz = (m.jz + R(0.5) * Fz) * inv;
    const Tens<R> T = noneq<L, R>(m, rho, ux, uy, uz, flags);
    R as, asg;
    ir_yield<R>(c, tnorm2<L, R>(T), as, asg);
    // A = -sigma_bar + s/2 = k1 T + k2 I with sigma_bar = sigma - tr(sigma)/D I
    const R trT = T.xx + T.yy + T.zz;
    const R k1 = R(0.5) * as - asg;
    const R k2 = asg * trT * R(1.0 / L::D);
    // (c c - c_s^2 I):A = k1 (cTc - trT/3) + k2 (|c|^2 - D/3) = h0 + k1 cTc + k2 |c|^2
    const R h0 = -(k1 * trT + k2 * R(L::D)) * R(1.0 / 3.0);
    const R uu = ux * ux + uy * uy + uz * uz;
    const R base = m.d - R(1.5) * rho * uu;
    const R r45 = R(4.5) * rho;
    const R k145 = R(4.5) * k1;
    const R t2xy = R(2) * T.xy, t2xz = R(2) * T.xz, t2yz = R(2) * T.yz;
    // odd part: w_i (3 rho c.u + 3/2 c.F) = 3 w_i c.(j + F), since rho u = j + F/2
    const R qx = m.jx + Fx, qy = m.jy + Fy, qz = m.jz + Fz;
    f[0] = R(Store<S>::template gam<L, 0>()) * (base + R(4.5) * h0);
    static_for<0, (L::Q - 1) / 2>([&](auto P) {
        constexpr int i = 2 * decltype(P)::value + 1;
        constexpr int o = i + 1;
        constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        constexpr int c2 = cx * cx + cy * cy + cz * cz;
        const R w = R(Store<S>::template gam<L, i>());   // w_i in memory units
        // even part e = w (base + 4.5 rho cu^2 + 4.5 h) = A + B cu^2 + C cTc (per class A, B, C)
        const R A = w * (base + R(4.5) * (h0 + k2 * R(c2)));
        const R B = w * r45;
        const R C = w * k145;
        const R cu = cdot<cx, cy, cz>(ux, uy, uz);
        const R e = A + B * (cu * cu) + C * ctc<cx, cy, cz>(T, t2xy, t2xz, t2yz);
        const R od = R(Store<S>::template god<L, i>()) * cdot<cx, cy, cz>(qx, qy, qz);
        f[i] = e + od;
        f[o] = e - od;
    });
    drho = m.d;
    ur[0] = ux;
    ur[1] = uy;
    ur[2] = uz;
}

// ---------------------------------------------------------------------------
// Implicit PR update (Sec. 3, Newton iterations).  With the unknown tau the
// strain rate of eq. (LBM_strain_rate) is gdot = a / tau, a = 1.5 sqrt(2 T:T);
// tau = 1/2 + 3 nu_app(gdot).  Consistency is the root of
// H(gdot) = gdot tau(gdot) - a = gdot / 2 + 3 gdot nu_app(gdot) - a, whose
// derivative is 1/2 + 3 d(gdot nu_app)/d gdot: nu_p + (sigma_y / rho) m e^(-m gdot)
// above the cut-off, nu_0 + 2 gdot (nu_c - nu_0) / gdot_C on the linear part
// below it.  Iterates are clamped at 0, H' floored at 1/2.
template <class R>
__device__ __forceinline__ R pr_newton(const Coef<R>& c, R a, R gd, R sy_rho) {
    const R nu0 = c.nu_p + c.m * sy_rho;
    const R nuc = c.nu_p + sy_rho * c.e_c;
    for (int k = 0; k < c.newton; ++k) {
        R gnu, dgnu;   // gdot nu_app(gdot) and its derivative
        if (gd >= c.gdot_c) {
            const R em = expm1(-c.m * gd);
            gnu = c.nu_p * gd - sy_rho * em;
            dgnu = c.nu_p + sy_rho * c.m * (R(1) + em);
        } else {
            const R s = gd * c.inv_gc;
            gnu = gd * ((R(1) - s) * nu0 + s * nuc);
            dgnu = nu0 + R(2) * s * (nuc - nu0);
        }
        const R h = R(0.5) * gd + R(3) * gnu - a;
        const R dh = fmax(R(0.5) + R(3) * dgnu, R(0.5));
        gd = fmax(gd - h / dh, R(0));
    }
    return gd;
}

// ---------------------------------------------------------------------------
// PR relaxation rates, per cell: strain rate with the previous step's tau
// (or the Newton-implicit one), apparent viscosity, tau and the two TRT rates.
template <bool IMPLICIT, class R>
__device__ __forceinline__ void pr_rates(const Coef<typename Lanes<R>::Sc>& c, R tn2, R inv, R& tau,
                                         R& wp_out, R& wm_out) {
    using Sc = typename Lanes<R>::Sc;
    Sc tau_[Lanes<R>::n], wp_[Lanes<R>::n], wm_[Lanes<R>::n];
#pragma unroll
    for (int k = 0; k < Lanes<R>::n; ++k) {
        // D = -T / (2 tau_old c_s^2) = -1.5 T / tau_old ; gdot = sqrt(2 D:D)
        const Sc tt = sqrt(Sc(2) * Lanes<R>::get(tn2, k));
        Sc gd = Sc(1.5) / Lanes<R>::get(tau, k) * tt;
        const Sc sy_rho = c.sigma_y * Lanes<R>::get(inv, k);
        if constexpr (IMPLICIT) gd = pr_newton(c, Sc(1.5) * tt, gd, sy_rho);
        Sc nu;
        if (gd >= c.gdot_c) {
            nu = c.nu_p + sy_rho * (-expm1(-c.m * gd)) / gd;
        } else {
            const Sc nu0 = c.nu_p + c.m * sy_rho;
            const Sc nuc = c.nu_p + sy_rho * c.e_c;
            nu = (c.gdot_c - gd) * c.inv_gc * nu0 + gd * c.inv_gc * nuc;
        }
        const Sc tn = Sc(0.5) + Sc(3) * nu;
        wp_[k] = Sc(1) / tn;
        // 1 / tau_odd with tau_odd = 1/2 + Lambda / (tau - 1/2), as one division
        const Sc tm = tn - Sc(0.5);
        wm_[k] = tm / (Sc(0.5) * tm + c.magic);
        tau_[k] = tn;
    }
    tau = Lanes<R>::make(tau_);
    wp_out = Lanes<R>::make(wp_);
    wm_out = Lanes<R>::make(wm_);
}

// ---------------------------------------------------------------------------
// PR collision (Sec. 3.1 + TRT + EDM).  tau: previous step's relaxation time
// in, this step's out.  f: memory units in, memory units out (the TRT update is
// linear and opposite populations share their unit).  R as for collide_ir.
template <class L, class S, bool IMPLICIT, class R = typename Store<S>::R>
__device__ __forceinline__ void collide_pr(const Coef<typename Lanes<R>::Sc>& c, uint32_t flags,
                                           R (&f)[L::Q], R& tau, R& drho, R (&ur)[3]) {
    const Mom<R> m = moments<L, S, R>(f);
    const R rho = R(1) + m.d;
    const R inv = recip(rho);
    const R ux = m.jx * inv, uy = m.jy * inv;
    R uz = R(0);
    if constexpr (L::D == 3) uz = m.jz * inv;
    const Tens<R> T = noneq<L, R>(m, rho, ux, uy, uz, flags);
    R wp, wm;
    pr_rates<IMPLICIT, R>(c, tnorm2<L, R>(T), inv, tau, wp, wm);
    const R gx = R(c.g[0]), gy = R(c.g[1]);
    R gz = R(0);
    if constexpr (L::D == 3) gz = R(c.g[2]);
    const R Fx = rho * gx, Fy = rho * gy, Fz = rho * gz;
    const R uu = ux * ux + uy * uy + uz * uz;
    const R ug = ux * gx + uy * gy + uz * gz;
    const R gg = gx * gx + gy * gy + gz * gz;
    const R base = m.d - R(1.5) * rho * uu;                 // even part of f_eq - w, direction-free
    const R fbase = R(-1.5) * rho * (R(2) * ug + gg);      // even part of the EDM difference
    const R r45 = R(4.5) * rho;
    // Per pair (i, o = opposite), with f^+- = (f_i +- f_o) / 2:
    //   E = f^+ - wp (f^+ - f_eq^+) + F^+ = (1 - wp)/2 (f_i + f_o) + w_i (K0 + 4.5 rho t),
    //       K0 = wp base + fbase,  t = wp cu^2 + cg (2 cu + cg) = cu (wp cu + 2 cg) + cg^2;
    //   O = f^- - wm (f^- - f_eq^-) + F^- = (1 - wm)/2 (f_i - f_o) + 3 w_i c.(wm j + F),
    // the odd equilibrium and force parts from j and F directly (3 w_i rho c.u
    // = 3 w_i c.j exactly).  cg = c_i.g and cg^2 are per-launch constants.
    const R omp = R(0.5) - R(0.5) * wp;
    const R omm = R(0.5) - R(0.5) * wm;
    const R K0 = wp * base + fbase;
    const R qx = wm * m.jx + Fx, qy = wm * m.jy + Fy, qz = wm * m.jz + Fz;
    {
        const R w0 = R(Store<S>::template gam<L, 0>());
        f[0] = (R(1) - wp) * f[0] + w0 * K0;
    }
    static_for<0, (L::Q - 1) / 2>([&](auto P) {
        constexpr int p = decltype(P)::value;
        constexpr int i = 2 * p + 1;
        constexpr int o = i + 1;
        constexpr int cx = L::cx(i), cy = L::cy(i), cz = L::cz(i);
        const R w = R(Store<S>::template gam<L, i>());    // w_i and 3 w_i in memory units
        const R w3 = R(Store<S>::template god<L, i>());
        const R cu = cdot<cx, cy, cz>(ux, uy, uz);
        const R cg = R(c.cg[p]);
        const R t = cu * (wp * cu + R(2) * cg) + R(c.cgg[p]);
        const R E = omp * (f[i] + f[o]) + w * (K0 + r45 * t);
        const R O = omm * (f[i] - f[o]) + w3 * cdot<cx, cy, cz>(qx, qy, qz);
        f[i] = E + O;
        f[o] = E - O;
    });
    drho = m.d;
    ur[0] = ux + R(0.5) * gx;
    ur[1] = uy + R(0.5) * gy;
    ur[2] = uz + R(0.5) * gz;
}

// ---------------------------------------------------------------------------
// deterministic block reduction of kNumStats values (fixed shuffle tree).
// The warp and block stages run in the type of v (the arithmetic type on
// check steps: at most 256 terms); each block's sums are stored as FP64
// partials and summed in FP64 in a fixed order by the finaliser.  Keeping the
// block stage off the FP64 pipe matters on GB300, whose FP64 rate is a small
// fraction of FP32: a serial FP64 shuffle chain per block made check steps
// four to five times slower than plain steps.
template <class V>
__device__ __forceinline__ void block_sum_store(V (&v)[kNumStats], double* __restrict__ out) {
    __shared__ V sm[kBlock / 32][kNumStats];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kNumStats; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kNumStats; ++k) sm[warp][k] = v[k];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < kNumStats; ++k) {
            V t = (lane < kBlock / 32) ? sm[lane][k] : V(0);
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (lane == 0) out[k] = (double)t;
        }
    }
}

// ---------------------------------------------------------------------------
// the fused step
//
// Minimum resident blocks per SM requested from the register allocator (0 =
// let it choose).  PR in FP32 arithmetic (FP32 and 16-bit storage): D3Q27
// keeps 1024 threads resident per SM at 256 and 512 threads per block (64
// registers) and 9 blocks at 128 (56 registers); a tighter cap spills.  The
// smaller lattices keep 1280 (10 x 128, 5 x 256, 2 x 512): D3Q19 PR then
// takes 48 registers without spilling and measured 7-9 % faster than at 64
// (porous box 256^3: FP32 466 -> 430 us, FP16 440 -> 401 us; duct
// 256 x 128 x 128: FP32 113.5 -> 105.7 us).  IR (40-48 registers) and FP64
// arithmetic (which these caps would make spill) are left to the allocator.
// BLBM_PR_MINB / BLBM_IR_MINB override at build time.
#ifndef BLBM_PR_MINB
#define BLBM_PR_MINB -1
#endif
#ifndef BLBM_IR_MINB
#define BLBM_IR_MINB 0
#endif
template <class L, int MODEL, class S, bool CHECK, int BLOCK> constexpr int step_min_blocks() {
    if (MODEL == LBM_MODEL_IR) return BLBM_IR_MINB;
    if (std::is_same<typename Store<S>::R, double>::value) return 0;
    if (BLBM_PR_MINB >= 0) return BLBM_PR_MINB;
    if (L::Q == 27 || CHECK) return BLOCK == 128 ? 9 : 1024 / BLOCK;   // check steps: no spill
    return 1280 / BLOCK;
}

// Stores one cell's outgoing populations at element n of the planes: the
// rest population, then the opposite pairs (i, i + 1), one random word each.
template <class L, class S, class Dst>
__device__ __forceinline__ void store_cell(const Dst& dst, int n,
                                           const typename Store<S>::R (&f)[L::Q], uint32_t rnd) {
    Store<S>::template st<L, 0>(dst.template at<0>(n), f[0], rnd);
    static_for<0, (L::Q - 1) / 2>([&](auto P) {
        constexpr int i = 2 * decltype(P)::value + 1;
        Store<S>::template st2<L, i>(dst.template at<i>(n), dst.template at<i + 1>(n), f[i],
                                     f[i + 1], pair_bits<decltype(P)::value + 1>(rnd));
    });
}

// A cell's check-step contributions (velocity, its change since the previous
// snapshot up, density offset, non-finite flag); its velocity becomes element
// n of the snapshot.
template <class R>
__device__ __forceinline__ void check_stats(const R (&ur)[3], const R (&up)[3], R drho,
                                            R* __restrict__ usnap, int64_t plane, int n,
                                            R (&acc)[kNumStats]) {
    R du2 = R(0), u2 = R(0);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        acc[kStatUx + d] = ur[d];
        du2 += (ur[d] - up[d]) * (ur[d] - up[d]);
        u2 += ur[d] * ur[d];
        usnap[(int64_t)d * plane + n] = ur[d];
    }
    acc[kStatDu2] = du2;
    acc[kStatU2] = u2;
    acc[kStatDrho] = drho;
    acc[kStatNonFinite] = isfinite(drho) ? R(0) : R(1);
}

// One cell of one time step: pull, collide, store; on check steps the cell's
// contributions to the flow-rate and residual sums go to acc.  Shared by the
// single-domain and the batched kernels so both do identical arithmetic.
// fluid = false copies a solid cell's populations through unchanged, the
// step's definition for solid cells: the stores of a group of cells that
// holds fluid cells then fill whole 32-byte sectors.  A sector the stores
// cover only in part costs a DRAM read before its write; at the edges of a
// porous medium's grains that doubled the reads.
template <class L, int MODEL, class S, bool CHECK, class Src, class Dst>
__device__ __forceinline__ void cell_step(const KParams& kp, const Coef<typename Store<S>::R>& c,
                                          const Src& src, const Dst& dst, uint32_t lk, int idx,
                                          typename Store<S>::R* __restrict__ tau,
                                          typename Store<S>::R* __restrict__ usnap, uint32_t rnd,
                                          typename Store<S>::R (&acc)[kNumStats],
                                          bool fluid = true) {
    using R = typename Store<S>::R;
    // check steps: the previous snapshot is read first, so its latency overlaps
    // the gather (after the population stores the compiler could not move
    // these loads up past them: the pointers may alias)
    R up[3] = {R(0), R(0), R(0)};
    if constexpr (CHECK) {
#pragma unroll
        for (int d = 0; d < 3; ++d) up[d] = usnap[(int64_t)d * kp.plane + idx];
    }
    R f[L::Q];
    gather<L, S>(kp, src, fluid ? lk : 0u, idx, f, !fluid);
    R drho = R(0), ur[3] = {R(0), R(0), R(0)};
    if (fluid) {
        if constexpr (MODEL != LBM_MODEL_IR) {
            R t = tau[idx];
            collide_pr<L, S, MODEL == kModelPRImplicit>(c, kp.flags, f, t, drho, ur);
            tau[idx] = t;
        } else {
            collide_ir<L, S>(c, kp.flags, f, drho, ur);
        }
    }
    store_cell<L, S>(dst, idx, f, rnd);
    if constexpr (CHECK) check_stats(ur, up, drho, usnap, kp.plane, idx, acc);
}

// Copy-through: the solid cells that share an aligned group of 8 consecutive
// cells (one 32-byte sector of a plane of 4-byte words) with a fluid cell run
// cell_step with fluid = false, which stores their populations unchanged, so
// the stores fill whole sectors (plain and check steps).  Groups without fluid
// cells are neither read nor written.  (The earlier rule, every solid cell of
// a warp that holds fluid cells, also moved the all-solid sectors of mixed
// warps: on a porous box of porosity 0.7 with grains of radius 6-10 it
// touched 1.43x the fluid cells' bytes, the 8-cell groups 1.27x.)  For the PR
// step of the 16-bit forms it is a per-solver choice (COPY), because there
// its path costs registers: on the D3Q27 duct, which has no warp mixing
// solid and fluid cells, it spills and the step is 6 % slower, while on a
// porous box it saves 7 % (256^3 D3Q19: 431 -> 401 us).  The solver takes it
// when at least 1 % of its warps with fluid cells also hold solid ones.
// (Solid lanes copying their raw words in a branch of their own keep the
// fluid path's registers, but a mixed warp then runs both branches one after
// the other: 40 % slower on the porous box in FP32.)
template <int MODEL, class S> __host__ __device__ constexpr bool copy_is_choice() {
    return MODEL != LBM_MODEL_IR && sizeof(S) == 2;
}

// Whether the aligned group of kCopyGroup cells holding cell idx has a fluid
// cell among the warp's active lanes.  Lane l holds cell idx - (threadIdx.x &
// 31) + l; cells of the group outside the warp count as solid (possible only
// when a launch does not start on a group boundary, a step taken in parts).
constexpr int kCopyGroup = 8;
__device__ __forceinline__ bool group_has_fluid(bool fluid, int idx) {
    const uint32_t b = __ballot_sync(__activemask(), fluid);
    const int first = (int)(threadIdx.x & 31) - (idx & (kCopyGroup - 1));   // -7 .. 31
    return ((((uint64_t)b << 32) >> (first + 32)) & ((1u << kCopyGroup) - 1u)) != 0;
}

// BLOCK: threads per block, chosen per (lattice, model, storage, size class)
// by the tuning table; check steps always run with kBlock so their reduction
// order does not depend on the tuning.
// RANGE: the launch covers cells [cell_begin, cell_end) only, one part of a
// step taken in parts (lbm_step_cells; 256 threads, plain steps).  Its own
// instantiation, so the whole-domain kernels carry no range arithmetic: under
// the 48-register budget of the smaller lattices it made the D3Q19 FP32 PR
// step spill and run 4 % slower.
template <class L, int MODEL, class S, bool CHECK, int BLOCK = kBlock, bool COPY = true,
          bool RANGE = false>
__global__ void __launch_bounds__(BLOCK, step_min_blocks<L, MODEL, S, CHECK, BLOCK>())
k_step(const KArgs a, const SrcPlanes<S> src, const DstPlanes<S> dst,
       const uint32_t* __restrict__ links, typename Store<S>::R* __restrict__ tau,
       typename Store<S>::R* __restrict__ usnap, double* __restrict__ partials,
       uint32_t* __restrict__ rng_ctr, int parity) {
    static_assert(!CHECK || BLOCK == kBlock, "check steps use the fixed block size");
    using R = typename Store<S>::R;
    const KParams& kp = a.kp;
    const int idx = (RANGE ? kp.cell_begin : 0) + (int)(blockIdx.x * BLOCK + threadIdx.x);
    const bool inside = idx < (RANGE ? kp.cell_end : kp.ncells);
    uint32_t rnd = 0u;
    if constexpr (Store<S>::kStochastic) {
        // this launch reads counter[parity] and leaves counter + 1 for the next
        const uint32_t seed = __ldg(rng_ctr + parity);
        if (blockIdx.x == 0 && threadIdx.x == 0) rng_ctr[parity ^ 1] = seed + 1u;
        rnd = pcg_hash(((uint32_t)idx + kp.hash_offset) ^ (seed * 0x9e3779b9u));
    }
    const uint32_t lk = inside ? __ldg(links + idx) : kSolidBit;
    const bool active = !(lk & kSolidBit);
    R acc[kNumStats];
    if constexpr (!CHECK) {
        if constexpr (COPY) {
            // a group without fluid cells has nothing to do; in any other group
            // the solid cells inside the domain copy their populations through
            if (!group_has_fluid(active, idx) || !inside) return;
            cell_step<L, MODEL, S, false>(kp, coef<R>(a), src, dst, lk, idx, tau, usnap, rnd, acc,
                                          active);
        } else {
            if (!active) return;
            cell_step<L, MODEL, S, false>(kp, coef<R>(a), src, dst, lk, idx, tau, usnap, rnd, acc);
        }
    } else {
#pragma unroll
        for (int k = 0; k < kNumStats; ++k) acc[k] = R(0);
        if constexpr (COPY) {
            // solid cells add nothing to the sums: their velocity and snapshot are 0
            if (group_has_fluid(active, idx) && inside)
                cell_step<L, MODEL, S, true>(kp, coef<R>(a), src, dst, lk, idx, tau, usnap, rnd, acc,
                                             active);
        } else {
            if (active)
                cell_step<L, MODEL, S, true>(kp, coef<R>(a), src, dst, lk, idx, tau, usnap, rnd, acc);
        }
        block_sum_store(acc, partials + (int64_t)blockIdx.x * kNumStats);
    }
}

// ---------------------------------------------------------------------------
// Two cells per thread.  Thread t of a block works on cells base + t and
// base + t + BLOCK, so every load and store instruction of a warp stays
// contiguous; it gathers and stores each cell as cell_step does and runs one
// collision on F2 values (packed f32x2 arithmetic for both cells).  A lane
// whose cell is solid or past the end repeats the other cell's work and
// stores nothing.  Plain steps of the FP32 and 16-bit forms only.
template <class L, int MODEL, class S, class Src, class Dst>
__device__ __forceinline__ void cell_step2(const KParams& kp, const Coef<float>& c, const Src& src,
                                           const Dst& dst, const uint32_t (&lk)[2],
                                           const int (&idx)[2], const bool (&act)[2],
                                           float* __restrict__ tau, const uint32_t (&rnd)[2]) {
    float a[L::Q], b[L::Q];
    gather<L, S>(kp, src, lk[0], idx[0], a);
    gather<L, S>(kp, src, lk[1], idx[1], b);
    F2 f[L::Q];
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        f[i] = F2(a[i], b[i]);
    });
    F2 drho, ur[3];
    if constexpr (MODEL != LBM_MODEL_IR) {
        F2 t(tau[idx[0]], tau[idx[1]]);
        collide_pr<L, S, MODEL == kModelPRImplicit, F2>(c, kp.flags, f, t, drho, ur);
        if (act[0]) tau[idx[0]] = t.lo();
        if (act[1]) tau[idx[1]] = t.hi();
    } else {
        collide_ir<L, S, F2>(c, kp.flags, f, drho, ur);
    }
    static_for<0, 2>([&](auto K) {
        constexpr int k = decltype(K)::value;
        if (act[k]) {
            const int n = idx[k];
            Store<S>::template st<L, 0>(dst.template at<0>(n), Lanes<F2>::get(f[0], k), rnd[k]);
            static_for<0, (L::Q - 1) / 2>([&](auto P) {
                constexpr int i = 2 * decltype(P)::value + 1;
                Store<S>::template st2<L, i>(dst.template at<i>(n), dst.template at<i + 1>(n),
                                             Lanes<F2>::get(f[i], k), Lanes<F2>::get(f[i + 1], k),
                                             pair_bits<decltype(P)::value + 1>(rnd[k]));
            });
        }
    });
}

// PR: at most 128 registers a thread, so 16 warps (1024 cells) stay resident
// per SM, the memory-level parallelism of the one-cell PR kernel.  IR needs
// fewer registers unbounded.
template <int MODEL, int BLOCK> constexpr int step2_min_blocks() {
    return MODEL == LBM_MODEL_IR ? 0 : 512 / BLOCK;
}

template <class L, int MODEL, class S, int BLOCK>
__global__ void __launch_bounds__(BLOCK, step2_min_blocks<MODEL, BLOCK>())
k_step2(const KArgs a, const SrcPlanes<S> src, const DstPlanes<S> dst,
        const uint32_t* __restrict__ links, float* __restrict__ tau,
        uint32_t* __restrict__ rng_ctr, int parity) {
    static_assert(std::is_same<typename Store<S>::R, float>::value, "two-cell steps need FP32 arithmetic");
    const KParams& kp = a.kp;
    const int i0 = blockIdx.x * (2 * BLOCK) + threadIdx.x;
    const int i1 = i0 + BLOCK;
    uint32_t seed = 0u;
    if constexpr (Store<S>::kStochastic) {
        // this launch reads counter[parity] and leaves counter + 1 for the next
        seed = __ldg(rng_ctr + parity);
        if (blockIdx.x == 0 && threadIdx.x == 0) rng_ctr[parity ^ 1] = seed + 1u;
    }
    const uint32_t l0 = i0 < kp.ncells ? __ldg(links + i0) : kSolidBit;
    const uint32_t l1 = i1 < kp.ncells ? __ldg(links + i1) : kSolidBit;
    const bool a0 = !(l0 & kSolidBit), a1 = !(l1 & kSolidBit);
    if (!a0 && !a1) return;
    const int idx[2] = {a0 ? i0 : i1, a1 ? i1 : i0};
    const uint32_t lk[2] = {a0 ? l0 : l1, a1 ? l1 : l0};
    const bool act[2] = {a0, a1};
    uint32_t rnd[2] = {0u, 0u};
    if constexpr (Store<S>::kStochastic) {
        rnd[0] = pcg_hash(((uint32_t)idx[0] + kp.hash_offset) ^ (seed * 0x9e3779b9u));
        rnd[1] = pcg_hash(((uint32_t)idx[1] + kp.hash_offset) ^ (seed * 0x9e3779b9u));
    }
    cell_step2<L, MODEL, S>(kp, a.cf, src, dst, lk, idx, act, tau, rnd);
}

// ---------------------------------------------------------------------------
// Compact layout (LBM_FLAG_COMPACT).  The population planes, the link words,
// tau and the check-step snapshot hold the stepped fluid cells only: slot k is
// the k-th fluid cell in cell-index order, cellidx[k] its cell index, and
// rank[n] the slot of cell n (-1 for a solid cell).  One thread per slot, so
// every lane of a warp is a fluid cell and every store fills whole sectors,
// whereas on a porous medium the dense layout also moves the solid cells that
// share a DRAM access with fluid ones.  The pull reads population i of the
// cell at x - c_i from slot rank[x - c_i] (a solid source: the cell's own
// opposite population, as in the dense layout); the rank words a warp reads
// lie in a few rows and mostly come from L1.  Per cell the arithmetic is the
// dense step's (the same collision code, the same stochastic-rounding hash of
// the cell index); compiled into another kernel, it may differ from it by the
// compiler's multiply-add contraction, i.e. to round-off.
template <class L, class S, class Src>
__device__ __forceinline__ void gather_compact(const KParams& kp, const Src& P, uint32_t lk,
                                               int idx, int slot, const int* __restrict__ rank,
                                               typename Store<S>::R (&v)[L::Q]) {
    const PullOffsets o = pull_offsets(kp, idx);
    // the cell's own rank word: each neighbour's is one multiply-add from it
    // (against an add and a sign-extended 64-bit address per neighbour: 2-8 %
    // faster steps on 256^3 porous boxes)
    const int* __restrict__ rk = rank + idx;
    v[0] = Store<S>::template ld<L, 0>(P.template at<0>(slot));
    if (__all_sync(__activemask(), lk == 0u)) {
        static_for<1, L::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const int k = __ldg(rk + o.template of<L, i>());
            v[i] = Store<S>::template ld<L, i>(P.template at<i>(k));
        });
    } else {
        static_for<1, L::Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const S* p;
            if ((lk >> i) & 1u)
                p = P.template at<L::opp(i)>(slot);
            else
                p = P.template at<i>(__ldg(rk + o.template of<L, i>()));
            v[i] = Store<S>::template ld<L, i>(p);   // opposite planes share w_i
        });
    }
}

// One fluid cell of one time step in the compact layout (as cell_step).
template <class L, int MODEL, class S, bool CHECK, class Src, class Dst>
__device__ __forceinline__ void compact_cell(const KParams& kp, const Coef<typename Store<S>::R>& c,
                                             const Src& src, const Dst& dst, uint32_t lk, int idx,
                                             int slot, const int* __restrict__ rank,
                                             typename Store<S>::R* __restrict__ tau,
                                             typename Store<S>::R* __restrict__ usnap, uint32_t rnd,
                                             typename Store<S>::R (&acc)[kNumStats]) {
    using R = typename Store<S>::R;
    R up[3] = {R(0), R(0), R(0)};
    if constexpr (CHECK) {
#pragma unroll
        for (int d = 0; d < 3; ++d) up[d] = usnap[(int64_t)d * kp.plane + slot];
    }
    R f[L::Q];
    gather_compact<L, S>(kp, src, lk, idx, slot, rank, f);
    R drho, ur[3];
    if constexpr (MODEL != LBM_MODEL_IR) {
        R t = tau[slot];
        collide_pr<L, S, MODEL == kModelPRImplicit>(c, kp.flags, f, t, drho, ur);
        tau[slot] = t;
    } else {
        collide_ir<L, S>(c, kp.flags, f, drho, ur);
    }
    store_cell<L, S>(dst, slot, f, rnd);
    if constexpr (CHECK) check_stats(ur, up, drho, usnap, kp.plane, slot, acc);
}

// Register budget of the compact step: the dense step's (BLBM_COMPACT_MINB
// overrides it at build time for the FP32-arithmetic forms).
#ifndef BLBM_COMPACT_MINB
#define BLBM_COMPACT_MINB -1
#endif
template <class L, int MODEL, class S, bool CHECK> constexpr int compact_min_blocks() {
    if (std::is_same<typename Store<S>::R, double>::value) return 0;
    if (BLBM_COMPACT_MINB >= 0) return BLBM_COMPACT_MINB;
    // IR up to 19 velocities: 6 blocks of 256 (40 registers): on the 256^3
    // porous box, D3Q19, 378 -> 361 us (FP32) and 318 -> 302 us (FP16) against
    // the allocator's 38 registers.  D3Q27 IR: 4 blocks (64 registers; 48
    // spilled and ran slower).  PR keeps the dense step's budget (6 blocks
    // spilled and made the D3Q19 FP16 step 7 % slower).
    if (MODEL == LBM_MODEL_IR && !CHECK) return L::Q <= 19 ? 6 : 4;
    return step_min_blocks<L, MODEL, S, CHECK, kBlock>();
}

// Threads per block of the plain compact step (check steps: kBlock).  A
// block's rank words come from the rows next to its cells, so a wider block
// reuses more of them from L1; the register budget per SM stays the same.
// 256^3 porous box, D3Q19: IR (FP32) 373 / 361 / 349 us at 128 / 256 / 512
// threads; PR, whose budget at 512 threads loses occupancy, 400 / 405 / 500
// (FP32) and 331 / 338 / 406 (FP16).  D3Q27 IR, whose 64 registers allow
// only two blocks of 512 per SM: 581 us at 512 threads, 512 us at 256 (256^3
// box, porosity 0.7).  BLBM_COMPACT_BLOCK overrides it.
#ifndef BLBM_COMPACT_BLOCK
#define BLBM_COMPACT_BLOCK 0
#endif
template <class L, int MODEL> constexpr int compact_block() {
    if (BLBM_COMPACT_BLOCK > 0) return BLBM_COMPACT_BLOCK;
    if (MODEL != LBM_MODEL_IR) return 128;
    return L::Q <= 19 ? 512 : 256;
}

template <class L, int MODEL, class S, bool CHECK, int BLOCK = kBlock>
__global__ void __launch_bounds__(BLOCK, compact_min_blocks<L, MODEL, S, CHECK>() * kBlock / BLOCK)
k_step_compact(const KArgs a, const SrcPlanes<S> src, const DstPlanes<S> dst,
               const uint32_t* __restrict__ links, const int* __restrict__ cellidx,
               const int* __restrict__ rank, typename Store<S>::R* __restrict__ tau,
               typename Store<S>::R* __restrict__ usnap, double* __restrict__ partials,
               uint32_t* __restrict__ rng_ctr, int parity) {
    static_assert(!CHECK || BLOCK == kBlock, "check steps use the fixed block size");
    using R = typename Store<S>::R;
    const KParams& kp = a.kp;
    const int slot = blockIdx.x * BLOCK + threadIdx.x;
    uint32_t seed = 0u;
    if constexpr (Store<S>::kStochastic) {
        // this launch reads counter[parity] and leaves counter + 1 for the next
        seed = __ldg(rng_ctr + parity);
        if (blockIdx.x == 0 && threadIdx.x == 0) rng_ctr[parity ^ 1] = seed + 1u;
    }
    R acc[kNumStats];
    if constexpr (CHECK) {
#pragma unroll
        for (int k = 0; k < kNumStats; ++k) acc[k] = R(0);
    }
    if (slot < kp.nslots) {
        const int idx = __ldg(cellidx + slot);
        const uint32_t lk = __ldg(links + slot);
        uint32_t rnd = 0u;
        if constexpr (Store<S>::kStochastic)
            rnd = pcg_hash(((uint32_t)idx + kp.hash_offset) ^ (seed * 0x9e3779b9u));
        compact_cell<L, MODEL, S, CHECK>(kp, coef<R>(a), src, dst, lk, idx, slot, rank, tau, usnap,
                                         rnd, acc);
    }
    if constexpr (CHECK) block_sum_store(acc, partials + (int64_t)blockIdx.x * kNumStats);
}

// Plain compact step over a persistent grid: each thread walks the slots
// slot, slot + stride, ... and loads the next slot's cell index and link word
// before it steps the current one, so of the three dependent loads of a slot
// (cell index, neighbour slots, populations) only the last two are on the
// critical path.  It pays for the IR step of the 16-bit forms (256^3 porous
// box, D3Q19 FP16: 306 -> 268 us).  The FP32 forms need more registers for it
// than their budgets hold: IR spilled at 6 blocks per SM (417 us) and ran at
// 391 us with 5, against 364 us for the one-slot kernel; PR gained nothing.
template <int MODEL, class S> constexpr bool compact_loop() {
    return MODEL == LBM_MODEL_IR && sizeof(S) == 2;
}
// (BLBM_COMPACT_LOOP_MINB overrides its register budget at build time.)
#ifndef BLBM_COMPACT_LOOP_MINB
#define BLBM_COMPACT_LOOP_MINB -1
#endif
// D3Q27: 4 blocks (64 registers; at 5 blocks it spills 68 bytes).
template <class L, int MODEL, class S> constexpr int compact_loop_min_blocks() {
    if (BLBM_COMPACT_LOOP_MINB >= 0) return BLBM_COMPACT_LOOP_MINB;
    if (L::Q == 27) return 4;
    return compact_min_blocks<L, MODEL, S, false>();
}

template <class L, int MODEL, class S>
__global__ void __launch_bounds__(kBlock, compact_loop_min_blocks<L, MODEL, S>())
k_step_compact_loop(const KArgs a, const SrcPlanes<S> src, const DstPlanes<S> dst,
                    const uint32_t* __restrict__ links, const int* __restrict__ cellidx,
                    const int* __restrict__ rank, typename Store<S>::R* __restrict__ tau,
                    uint32_t* __restrict__ rng_ctr, int parity) {
    using R = typename Store<S>::R;
    const KParams& kp = a.kp;
    const int n = kp.nslots, stride = gridDim.x * kBlock;
    uint32_t seed = 0u;
    if constexpr (Store<S>::kStochastic) {
        // this launch reads counter[parity] and leaves counter + 1 for the next
        seed = __ldg(rng_ctr + parity);
        if (blockIdx.x == 0 && threadIdx.x == 0) rng_ctr[parity ^ 1] = seed + 1u;
    }
    int slot = blockIdx.x * kBlock + threadIdx.x;
    int idx = 0;
    uint32_t lk = 0u;
    if (slot < n) {
        idx = __ldg(cellidx + slot);
        lk = __ldg(links + slot);
    }
    R acc[kNumStats];
    for (; slot < n; slot += stride) {
        const int next = slot + stride;
        int nidx = 0;
        uint32_t nlk = 0u;
        if (next < n) {
            nidx = __ldg(cellidx + next);
            nlk = __ldg(links + next);
        }
        uint32_t rnd = 0u;
        if constexpr (Store<S>::kStochastic)
            rnd = pcg_hash(((uint32_t)idx + kp.hash_offset) ^ (seed * 0x9e3779b9u));
        compact_cell<L, MODEL, S, false>(kp, coef<R>(a), src, dst, lk, idx, slot, rank, tau,
                                         nullptr, rnd, acc);
        idx = nidx;
        lk = nlk;
    }
}

// link words of the compact layout: slot k gets the bits of cell cellidx[k]
template <class L>
__global__ void __launch_bounds__(kBlock)
k_links_compact(const KParams kp, const uint8_t* __restrict__ mask,
                const int* __restrict__ cellidx, uint32_t* __restrict__ links) {
    const int slot = blockIdx.x * kBlock + threadIdx.x;
    if (slot >= kp.nslots) return;
    const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
    int x, y, z;
    cell_xyz(kp, cellidx[slot], x, y, z);
    uint32_t bits = 0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int xs = (x - L::cx(i) + nx) % nx;
        const int ys = (y - L::cy(i) + ny) % ny;
        const int zs = (z - L::cz(i) + nz) % nz;
        if (mask[xs + nx * (ys + ny * zs)]) bits |= 1u << i;
    }
    links[slot] = bits;
}

// ---------------------------------------------------------------------------
// Batched step: all resident domains of one (lattice, model, storage) in one
// launch.  Block b works on domain block_dom[b]; each domain's blocks are
// contiguous from desc.block_begin.  The current buffer of a domain is
// phase ^ desc.parity0, so a captured graph that alternates the phase stays
// valid for every domain.
struct BatchDesc {
    KParams kp;
    Coef<float> cf;
    Coef<double> cd;
    void* f[2];
    const uint32_t* links;
    void* tau;
    void* usnap;
    uint32_t* rng;      // two launch counters (16-bit storage)
    int parity0;
    int block_begin;    // first 256-cell tile of this domain (check steps)
    int nblocks;        // its 256-cell tiles
    int slot;           // row of this domain in the batch's per-domain stats
    int pblock_begin;   // first tile of this domain in the plain-step tile map
};

template <class R> __device__ __forceinline__ const Coef<R>& bcoef(const BatchDesc& d);
template <> __device__ __forceinline__ const Coef<float>& bcoef<float>(const BatchDesc& d) { return d.cf; }
template <> __device__ __forceinline__ const Coef<double>& bcoef<double>(const BatchDesc& d) { return d.cd; }

// One check step of one tile (kBlock consecutive cells of one domain): as
// k_step's check step, with the copy-through for every form (the solid cells
// of a group with fluid cells copy their populations through).
template <class L, int MODEL, class S>
__device__ __forceinline__ void batch_tile_check(const BatchDesc& D, int tile, int phase,
                                                 double* __restrict__ partials) {
    using R = typename Store<S>::R;
    const KParams& kp = D.kp;
    const int lb = tile - D.block_begin;
    const int idx = lb * kBlock + threadIdx.x;
    const int cur = phase ^ D.parity0;
    const SrcStride<S> src{(const S*)D.f[cur], (int)kp.plane};
    const DstStride<S> dst{(S*)D.f[cur ^ 1], (int)kp.plane};
    const bool inside = idx < kp.ncells;
    uint32_t rnd = 0u;
    if constexpr (Store<S>::kStochastic) {
        // reads counter[cur], leaves counter + 1 in the other slot for the next launch
        const uint32_t seed = D.rng[cur];
        if (lb == 0 && threadIdx.x == 0) D.rng[cur ^ 1] = seed + 1u;
        rnd = pcg_hash(((uint32_t)idx + kp.hash_offset) ^ (seed * 0x9e3779b9u));
    }
    const uint32_t lk = inside ? __ldg(D.links + idx) : kSolidBit;
    const bool active = !(lk & kSolidBit);
    const bool group_fluid = group_has_fluid(active, idx);
    R acc[kNumStats];
#pragma unroll
    for (int k = 0; k < kNumStats; ++k) acc[k] = R(0);
    if (group_fluid && inside)
        cell_step<L, MODEL, S, true>(kp, bcoef<R>(D), src, dst, lk, idx, (R*)D.tau, (R*)D.usnap,
                                     rnd, acc, active);
    block_sum_store(acc, partials + (int64_t)tile * kNumStats);
}

// One plain step of one tile of T x C cells of one domain (the tile shape the
// batch schedule sets per group): thread t steps cells base + t, base + t + T,
// ... (C of them, one after the other), so every warp access stays
// contiguous.  Per cell as k_step, with the copy-through for every form.
template <class L, int MODEL, class S, int T, int C>
__device__ __forceinline__ void batch_tile_plain(const BatchDesc& D, int tile, int phase) {
    using R = typename Store<S>::R;
    const KParams& kp = D.kp;
    const int lb = tile - D.pblock_begin;
    const int cur = phase ^ D.parity0;
    const SrcStride<S> src{(const S*)D.f[cur], (int)kp.plane};
    const DstStride<S> dst{(S*)D.f[cur ^ 1], (int)kp.plane};
    uint32_t seed = 0u;
    if constexpr (Store<S>::kStochastic) {
        // reads counter[cur], leaves counter + 1 in the other slot for the next launch
        seed = D.rng[cur];
        if (lb == 0 && threadIdx.x == 0) D.rng[cur ^ 1] = seed + 1u;
    }
#pragma unroll 1
    for (int c = 0; c < C; ++c) {
        const int idx = (lb * C + c) * T + (int)threadIdx.x;
        const bool inside = idx < kp.ncells;
        uint32_t rnd = 0u;
        if constexpr (Store<S>::kStochastic) rnd = pcg_hash(((uint32_t)idx + kp.hash_offset) ^ (seed * 0x9e3779b9u));
        const uint32_t lk = inside ? __ldg(D.links + idx) : kSolidBit;
        const bool active = !(lk & kSolidBit);
        const bool group_fluid = group_has_fluid(active, idx);
        R acc[kNumStats];
        if (group_fluid && inside)
            cell_step<L, MODEL, S, false>(kp, bcoef<R>(D), src, dst, lk, idx, (R*)D.tau,
                                          (R*)D.usnap, rnd, acc, active);
    }
}

// Batch steps: the CTAs walk the tiles of every domain of the group (tile t,
// t + gridDim.x, ...).  With one CTA per tile this is the plain launch; with
// fewer CTAs it is a persistent grid.  Check-step partials are indexed by
// 256-cell tile, so check steps reduce in the same order for every grid size
// and every plain-step tile shape.
// Register budget of the batch kernels, as resident 256-thread blocks (scaled
// to the tile's threads): plain PR steps in FP32 arithmetic keep 4 (64
// registers).  Without it the 16-bit forms take 72 registers and FP32
// storage 70 (the descriptor's coefficients are loaded, not kernel-parameter
// operands), leaving 3 blocks; on a single D3Q27 duct the FP32 PR batch step
// measured 170 us without and 154 us with the budget.  Plain IR steps of the
// 16-bit forms keep 5 (48 registers; their copy-through path takes 58 and 4
// blocks otherwise).  FP32 IR, check steps and FP64 are left to the
// allocator.  BLBM_BATCH_PR_MINB (16-bit PR), BLBM_BATCH_PR32_MINB (FP32 PR)
// and BLBM_BATCH_IR16_MINB override at build time.
#ifndef BLBM_BATCH_PR_MINB
#define BLBM_BATCH_PR_MINB 4
#endif
#ifndef BLBM_BATCH_PR32_MINB
#define BLBM_BATCH_PR32_MINB 4
#endif
#ifndef BLBM_BATCH_IR16_MINB
#define BLBM_BATCH_IR16_MINB 5
#endif
template <int MODEL, class S, bool CHECK> constexpr int batch_min_blocks() {
    return CHECK ? 0
         : MODEL == LBM_MODEL_IR ? (sizeof(S) == 2 ? BLBM_BATCH_IR16_MINB : 0)
         : sizeof(S) == 2 ? BLBM_BATCH_PR_MINB
         : sizeof(S) == 4 ? BLBM_BATCH_PR32_MINB : 0;
}

template <class L, int MODEL, class S>
__global__ void __launch_bounds__(kBlock)
k_step_batch_check(const BatchDesc* __restrict__ descs, const int* __restrict__ block_dom,
                   int ntiles, int phase, double* __restrict__ partials) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        batch_tile_check<L, MODEL, S>(descs[block_dom[t]], t, phase, partials);
        __syncthreads();   // block_sum_store's shared rows are reused
    }
}

template <class L, int MODEL, class S, int T, int C>
__global__ void __launch_bounds__(T, batch_min_blocks<MODEL, S, false>() * kBlock / T)
k_step_batch(const BatchDesc* __restrict__ descs, const int* __restrict__ tile_dom, int ntiles,
             int phase) {
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x)
        batch_tile_plain<L, MODEL, S, T, C>(descs[tile_dom[t]], t, phase);
}

// density and velocity u = (j + F/2) / rho of gathered populations
template <class L, class S>
__device__ __forceinline__ void fields_of(const KArgs& a, const typename Store<S>::R (&v)[L::Q],
                                          double& r, double (&u)[3]) {
    using R = typename Store<S>::R;
    const Mom<R> m = moments<L, S>(v);
    const Coef<R>& c = coef<R>(a);
    const R rr = R(1) + m.d;
    const R inv = R(1) / rr;
    r = (double)rr;
    u[0] = (double)((m.jx + R(0.5) * rr * c.g[0]) * inv);
    u[1] = (double)((m.jy + R(0.5) * rr * c.g[1]) * inv);
    if constexpr (L::D == 3) u[2] = (double)((m.jz + R(0.5) * rr * c.g[2]) * inv);
}

// macroscopic fields of the streamed populations (solid cells: 0)
template <class L, class S>
__global__ void __launch_bounds__(kBlock)
k_fields(const KArgs a, const SrcPlanes<S> f, const uint32_t* __restrict__ links,
         double* __restrict__ rho, double* __restrict__ ux, double* __restrict__ uy,
         double* __restrict__ uz) {
    using R = typename Store<S>::R;
    const KParams& kp = a.kp;
    const int idx = blockIdx.x * kBlock + threadIdx.x;
    if (idx >= kp.ncells) return;
    const uint32_t lk = links[idx];
    double r = 0.0, u[3] = {0.0, 0.0, 0.0};
    if (!(lk & kSolidBit)) {
        R v[L::Q];
        gather<L, S>(kp, f, lk, idx, v);
        fields_of<L, S>(a, v, r, u);
    }
    if (rho) rho[idx] = r;
    if (ux) ux[idx] = u[0];
    if (uy) uy[idx] = u[1];
    if (uz) uz[idx] = u[2];
}

// the same from the compact layout, one thread per cell of the box
template <class L, class S>
__global__ void __launch_bounds__(kBlock)
k_fields_compact(const KArgs a, const SrcPlanes<S> f, const uint32_t* __restrict__ links,
                 const int* __restrict__ rank, double* __restrict__ rho, double* __restrict__ ux,
                 double* __restrict__ uy, double* __restrict__ uz) {
    using R = typename Store<S>::R;
    const KParams& kp = a.kp;
    const int idx = blockIdx.x * kBlock + threadIdx.x;
    if (idx >= kp.ncells) return;
    const int slot = rank[idx];
    double r = 0.0, u[3] = {0.0, 0.0, 0.0};
    if (slot >= 0) {
        R v[L::Q];
        gather_compact<L, S>(kp, f, links[slot], idx, slot, rank, v);
        fields_of<L, S>(a, v, r, u);
    }
    if (rho) rho[idx] = r;
    if (ux) ux[idx] = u[0];
    if (uy) uy[idx] = u[1];
    if (uz) uz[idx] = u[2];
}

// grid-stride reductions: flow sums of u_real (gathered) or state totals,
// over the cells of the box (dense layout) or the slots (COMPACT)
template <class L, class S, int MODE, bool COMPACT>
__global__ void __launch_bounds__(kBlock)
k_reduce(const KArgs a, const SrcPlanes<S> f, const uint32_t* __restrict__ links,
         const int* __restrict__ cellidx, const int* __restrict__ rank,
         double* __restrict__ partials) {
    using R = typename Store<S>::R;
    const KParams& kp = a.kp;
    double acc[kNumStats];
#pragma unroll
    for (int k = 0; k < kNumStats; ++k) acc[k] = 0.0;
    const int stride = gridDim.x * kBlock;
    const int n_end = COMPACT ? kp.nslots : kp.ncells;
    for (int n = blockIdx.x * kBlock + threadIdx.x; n < n_end; n += stride) {
        const uint32_t lk = links[n];
        if (!COMPACT && (lk & kSolidBit)) continue;
        R v[L::Q];
        if constexpr (MODE == kReduceFlow) {
            if constexpr (COMPACT)
                gather_compact<L, S>(kp, f, lk, cellidx[n], n, rank, v);
            else
                gather<L, S>(kp, f, lk, n, v);
        } else {
            static_for<0, L::Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                v[i] = Store<S>::template ld<L, i>(f.template at<i>(n));
            });
        }
        const Mom<R> m = moments<L, S>(v);
        if constexpr (MODE == kReduceFlow) {
            const Coef<R>& c = coef<R>(a);
            const R rr = R(1) + m.d;
            const R inv = R(1) / rr;
            acc[kStatUx] += (double)((m.jx + R(0.5) * rr * c.g[0]) * inv);
            acc[kStatUy] += (double)((m.jy + R(0.5) * rr * c.g[1]) * inv);
            if constexpr (L::D == 3) acc[kStatUz] += (double)((m.jz + R(0.5) * rr * c.g[2]) * inv);
            acc[kStatDrho] += (double)m.d;
        } else {
            acc[kTotMass] += (double)m.d;
            acc[kTotJx] += (double)m.jx;
            acc[kTotJy] += (double)m.jy;
            acc[kTotJz] += (double)m.jz;
        }
    }
    block_sum_store(acc, partials + (int64_t)blockIdx.x * kNumStats);
}

// solid / bounce-back link bits: bit i set if the cell at x - c_i is solid
// (With LBM_FLAG_Z_GHOSTS the first and last z-planes are ghost planes: they
// are never stepped, like solid cells, while their mask rows, the
// neighbouring slabs' own, still set the link bits of the planes next to them.)
template <class L>
__global__ void __launch_bounds__(kBlock)
k_links(const KParams kp, const uint8_t* __restrict__ mask, uint32_t* __restrict__ links) {
    const int idx = blockIdx.x * kBlock + threadIdx.x;
    if (idx >= kp.ncells) return;
    const int nx = kp.nx, ny = kp.ny, nz = kp.nz;
    int x, y, z;
    cell_xyz(kp, idx, x, y, z);
    const bool ghost = (kp.flags & LBM_FLAG_Z_GHOSTS) && (z == 0 || z == nz - 1);
    if (mask[idx] || ghost) {
        links[idx] = kSolidBit;
        return;
    }
    uint32_t bits = 0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const int xs = (x - L::cx(i) + nx) % nx;
        const int ys = (y - L::cy(i) + ny) % ny;
        const int zs = (z - L::cz(i) + nz) % nz;
        if (mask[xs + nx * (ys + ny * zs)]) bits |= 1u << i;
    }
    links[idx] = bits;
}

// FP64 full populations <-> stored offsets, one population plane at a time.
// Compact layout (rank != nullptr): the fluid cells' values move through
// their slots; solid cells are not stored and read back as the rest state w_q.
template <class L, class S>
__global__ void __launch_bounds__(kBlock)
k_convert(const KParams kp, int q, bool to_device, S* __restrict__ f, double* __restrict__ buf,
          const int* __restrict__ rank) {
    const int idx = blockIdx.x * kBlock + threadIdx.x;
    if (idx >= kp.ncells) return;
    double w = 0.0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
        if (i == q) w = L::w(i);
    const int n = rank ? rank[idx] : idx;
    if (n < 0) {
        if (!to_device) buf[idx] = w;
        return;
    }
    S* p = f + pop_base<S>(q, kp.plane) + (int64_t)pop_step<S>(q) * n;
    if (to_device)
        *p = Store<S>::enc(buf[idx] - w, w);
    else
        buf[idx] = Store<S>::dec(*p, w) + w;
}

// Slab faces (LBM_FLAG_Z_GHOSTS).  The populations that cross a z-face are
// those with c_z = +1 (moving up) and c_z = -1 (moving down).  side 1 packs
// the last interior plane's c_z = +1 populations (the upper neighbour's lower
// ghost plane receives them: its side 0 unpack); side 0 packs the first
// interior plane's c_z = -1 populations (the lower neighbour's side 1
// unpack, into its upper ghost plane).  buf holds the stored values (no
// conversion), [j][cell of the plane] for the j-th crossing population in the
// lattice's order.
template <class L> __host__ __device__ constexpr int face_count() {
    int n = 0;
    for (int i = 0; i < L::Q; ++i) n += L::cz(i) == 1;
    return n;
}
template <class L> __device__ __forceinline__ int face_pop(int j, int cz) {
    int n = 0;
    for (int i = 0; i < L::Q; ++i)
        if (L::cz(i) == cz && n++ == j) return i;
    return -1;
}

template <class L, class S>
__global__ void __launch_bounds__(kBlock)
k_halo(const KParams kp, S* __restrict__ f, S* __restrict__ buf, int side, bool pack) {
    const int nxy = kp.nx * kp.ny;
    const int k = blockIdx.x * kBlock + threadIdx.x;
    if (k >= face_count<L>() * nxy) return;
    const int j = k / nxy, xy = k - j * nxy;
    // pack: interior plane next to the face, populations leaving through it;
    // unpack: ghost plane of the face, populations entering through it
    const int cz = (side == 1) == pack ? 1 : -1;
    const int z = pack ? (side == 1 ? kp.nz - 2 : 1) : (side == 1 ? kp.nz - 1 : 0);
    const int i = face_pop<L>(j, cz);
    S* p = f + pop_base<S>(i, kp.plane) + (int64_t)pop_step<S>(i) * ((int64_t)z * nxy + xy);
    if (pack)
        buf[k] = *p;
    else
        *p = buf[k];
}

// full FP64 populations of listed cells: out[i * n + k] = f_i(cells[k])
// (compact layout: a solid cell reads as the rest state w_i)
template <class L, class S>
__global__ void __launch_bounds__(kBlock)
k_gather_cells(const KParams kp, const S* __restrict__ f, const int64_t* __restrict__ cells,
               int n, double* __restrict__ out, const int* __restrict__ rank) {
    const int k = blockIdx.x * kBlock + threadIdx.x;
    if (k >= n) return;
    const int64_t c = rank ? (int64_t)rank[cells[k]] : cells[k];
    static_for<0, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        out[(int64_t)i * n + k] =
            c < 0 ? L::w(i)
                  : Store<S>::dec(f[pop_base<S>(i, kp.plane) + (int64_t)pop_step<S>(i) * c], L::w(i)) + L::w(i);
    });
}

// ---------------------------------------------------------------------------
// host-side helpers for the per-lattice launchers
template <class L, class R> inline void fill_force_dirs(Coef<R>& c, const KParams& kp) {
    for (int p = 0; p < 13; ++p) {
        c.cg[p] = R(0);
        c.cgg[p] = R(0);
    }
    for (int p = 0; p < (L::Q - 1) / 2; ++p) {
        const int i = 2 * p + 1;
        const double cg = L::cx(i) * kp.g[0] + L::cy(i) * kp.g[1] + L::cz(i) * kp.g[2];
        c.cg[p] = (R)cg;
        c.cgg[p] = (R)(cg * cg);
    }
}

template <class R> inline Coef<R> make_coef(const KParams& kp) {
    Coef<R> c;
    const double nu = kp.nu_p;
    c.nu_p = (R)nu;
    c.sigma_y = (R)kp.sigma_y;
    c.m = (R)kp.m;
    c.gdot_c = (R)kp.gdot_c;
    c.inv_gc = (R)(1.0 / kp.gdot_c);
    c.e_c = (R)(kp.m * kp.gdot_c > 0.0 ? -expm1(-kp.m * kp.gdot_c) / kp.gdot_c : 0.0);
    c.magic = (R)kp.magic;
    for (int d = 0; d < 3; ++d) c.g[d] = (R)kp.g[d];
    c.s2y = (R)(1.4142135623730951 * kp.sigma_y);
    c.ir_a = (R)(1.0 / (0.5 + 3.0 * nu));
    c.ir_b = (R)(1.0 / (1.0 + 6.0 * nu));
    c.six_nu = (R)(6.0 * nu);
    c.newton = kp.newton;
    return c;
}

template <class L> inline KArgs make_args(const KParams& kp) {
    KArgs a;
    a.kp = kp;
    a.cf = make_coef<float>(kp);
    a.cd = make_coef<double>(kp);
    fill_force_dirs<L>(a.cf, kp);
    fill_force_dirs<L>(a.cd, kp);
    return a;
}

// Coefficients of a domain of lattice `lat` (host code without the lattice
// as a template parameter: the batch tables).
template <class R> inline Coef<R> make_coef_lat(const KParams& kp, int lat) {
    Coef<R> c = make_coef<R>(kp);
    switch (lat) {
    case LBM_D2Q9: fill_force_dirs<D2Q9>(c, kp); break;
    case LBM_D3Q15: fill_force_dirs<D3Q15>(c, kp); break;
    case LBM_D3Q19: fill_force_dirs<D3Q19>(c, kp); break;
    default: fill_force_dirs<D3Q27>(c, kp); break;
    }
    return c;
}

template <class L, class S> inline SrcPlanes<S> src_planes(const void* f, int64_t plane) {
    SrcPlanes<S> P{};
    for (int i = 0; i < L::Q; ++i) P.p[i] = (const S*)f + pop_base<S>(i, plane);
    return P;
}
template <class L, class S> inline DstPlanes<S> dst_planes(void* f, int64_t plane) {
    DstPlanes<S> P{};
    for (int i = 0; i < L::Q; ++i) P.p[i] = (S*)f + pop_base<S>(i, plane);
    return P;
}

template <class L, int MODEL, class S, bool COPY>
cudaError_t launch_step_c(bool check, const KParams& kp, const StepArgs& s, cudaStream_t st) {
    using R = typename Store<S>::R;
    const KArgs a = make_args<L>(kp);
    const int ncell = kp.cell_end - kp.cell_begin;   // the cells this launch covers
    const int grid = step_grid(ncell);
    const SrcPlanes<S> src = src_planes<L, S>(s.fsrc, kp.plane);
    const DstPlanes<S> dst = dst_planes<L, S>(s.fdst, kp.plane);
    const int block = (check || MODEL == kModelPRImplicit) ? kBlock : s.block;   // implicit: untuned
    if constexpr (MODEL != kModelPRImplicit && std::is_same<typename Store<S>::R, float>::value) {
        if (!check && s.cpt == 2) {   // two cells per thread
            if (block == 128)
                k_step2<L, MODEL, S, 128><<<(kp.ncells + 255) / 256, 128, 0, st>>>(
                    a, src, dst, s.links, (R*)s.tau, s.rng_ctr, s.parity);
            else
                k_step2<L, MODEL, S, 256><<<(kp.ncells + 511) / 512, 256, 0, st>>>(
                    a, src, dst, s.links, (R*)s.tau, s.rng_ctr, s.parity);
            return cudaGetLastError();
        }
    }
    if (check) {
        k_step<L, MODEL, S, true, kBlock, COPY><<<grid, kBlock, 0, st>>>(
            a, src, dst, s.links, (R*)s.tau, (R*)s.usnap, s.partials, s.rng_ctr, s.parity);
    } else if (kp.cell_begin != 0 || kp.cell_end != kp.ncells) {
        // one part of a step taken in parts (256 threads)
        k_step<L, MODEL, S, false, kBlock, COPY, true><<<grid, kBlock, 0, st>>>(
            a, src, dst, s.links, (R*)s.tau, (R*)s.usnap, s.partials, s.rng_ctr, s.parity);
    } else if constexpr (MODEL != kModelPRImplicit) {
        if (block == 128) {
            k_step<L, MODEL, S, false, 128, COPY><<<(ncell + 127) / 128, 128, 0, st>>>(
                a, src, dst, s.links, (R*)s.tau, (R*)s.usnap, s.partials, s.rng_ctr, s.parity);
        } else if (block == 512) {
            k_step<L, MODEL, S, false, 512, COPY><<<(ncell + 511) / 512, 512, 0, st>>>(
                a, src, dst, s.links, (R*)s.tau, (R*)s.usnap, s.partials, s.rng_ctr, s.parity);
        } else {
            k_step<L, MODEL, S, false, kBlock, COPY><<<grid, kBlock, 0, st>>>(
                a, src, dst, s.links, (R*)s.tau, (R*)s.usnap, s.partials, s.rng_ctr, s.parity);
        }
    } else {
        k_step<L, MODEL, S, false, kBlock, COPY><<<grid, kBlock, 0, st>>>(
            a, src, dst, s.links, (R*)s.tau, (R*)s.usnap, s.partials, s.rng_ctr, s.parity);
    }
    return cudaGetLastError();
}

template <class L, int MODEL, class S>
cudaError_t launch_step_compact(bool check, const KParams& kp, const StepArgs& s, cudaStream_t st) {
    using R = typename Store<S>::R;
    const KArgs a = make_args<L>(kp);
    const int grid = step_grid(kp.nslots);
    const SrcPlanes<S> src = src_planes<L, S>(s.fsrc, kp.plane);
    const DstPlanes<S> dst = dst_planes<L, S>(s.fdst, kp.plane);
    if (check) {
        k_step_compact<L, MODEL, S, true><<<grid, kBlock, 0, st>>>(
            a, src, dst, s.links, s.cellidx, s.rank, (R*)s.tau, (R*)s.usnap, s.partials,
            s.rng_ctr, s.parity);
    } else if constexpr (compact_loop<MODEL, S>()) {
        // persistent: as many blocks as are resident at once, at most one per 256 slots
        static const int resident = [] {   // blocks per SM (per instantiation)
            int r = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, k_step_compact_loop<L, MODEL, S>,
                                                              kBlock, 0) != cudaSuccess) {
                cudaGetLastError();
                r = 1;
            }
            return r < 1 ? 1 : r;
        }();
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int pgrid = std::min(grid, std::max(1, resident * sms));
        k_step_compact_loop<L, MODEL, S><<<pgrid, kBlock, 0, st>>>(
            a, src, dst, s.links, s.cellidx, s.rank, (R*)s.tau, s.rng_ctr, s.parity);
    } else {
        constexpr int B = compact_block<L, MODEL>();
        k_step_compact<L, MODEL, S, false, B><<<(kp.nslots + B - 1) / B, B, 0, st>>>(
            a, src, dst, s.links, s.cellidx, s.rank, (R*)s.tau, (R*)s.usnap, s.partials,
            s.rng_ctr, s.parity);
    }
    return cudaGetLastError();
}

// The compact layout has its own kernel.  In the dense one the copy-through
// is on for every form but the PR step of the 16-bit ones, which follows the
// solver's geometry (s.copy).
template <class L, int MODEL, class S>
cudaError_t launch_step_t(bool check, const KParams& kp, const StepArgs& s, cudaStream_t st) {
    if (s.rank) return launch_step_compact<L, MODEL, S>(check, kp, s, st);
    if constexpr (copy_is_choice<MODEL, S>()) {
        if (!s.copy) return launch_step_c<L, MODEL, S, false>(check, kp, s, st);
    }
    return launch_step_c<L, MODEL, S, true>(check, kp, s, st);
}

template <class L, class S>
cudaError_t launch_step_model(int model, bool check, const KParams& kp, const StepArgs& s,
                              cudaStream_t st) {
    if (model == kModelPRImplicit) return launch_step_t<L, kModelPRImplicit, S>(check, kp, s, st);
    if (model == LBM_MODEL_PR) return launch_step_t<L, LBM_MODEL_PR, S>(check, kp, s, st);
    return launch_step_t<L, LBM_MODEL_IR, S>(check, kp, s, st);
}

template <class L>
cudaError_t launch_step_lat(int model, int storage, bool check, const KParams& kp,
                            const StepArgs& s, cudaStream_t st) {
    switch (storage) {
    case LBM_F32: return launch_step_model<L, float>(model, check, kp, s, st);
    case LBM_F64: return launch_step_model<L, double>(model, check, kp, s, st);
    case LBM_F16_OFS: return launch_step_model<L, __half>(model, check, kp, s, st);
    case LBM_BF16_OFS: return launch_step_model<L, __nv_bfloat16>(model, check, kp, s, st);
    default: return cudaErrorNotSupported;
    }
}

// Plain-step tile shapes of the batch (threads per CTA x cells per thread);
// FP64 storage and the Newton-implicit PR step run 256 x 1 only.
template <int MODEL, class S> constexpr bool batch_shapes_all() {
    return MODEL != kModelPRImplicit && !std::is_same<S, double>::value;
}

template <class L, int MODEL, class S>
cudaError_t launch_batch_t(bool check, const BatchDesc* descs, const int* block_dom, int nblocks,
                           int grid, int phase, double* partials, int threads, int cpt,
                           cudaStream_t st) {
    if (check) {
        k_step_batch_check<L, MODEL, S><<<grid, kBlock, 0, st>>>(descs, block_dom, nblocks, phase, partials);
    } else if (threads == 256 && cpt == 1) {
        k_step_batch<L, MODEL, S, 256, 1><<<grid, 256, 0, st>>>(descs, block_dom, nblocks, phase);
    } else if constexpr (batch_shapes_all<MODEL, S>()) {
        if (threads == 128 && cpt == 1)
            k_step_batch<L, MODEL, S, 128, 1><<<grid, 128, 0, st>>>(descs, block_dom, nblocks, phase);
        else if (threads == 512 && cpt == 1)
            k_step_batch<L, MODEL, S, 512, 1><<<grid, 512, 0, st>>>(descs, block_dom, nblocks, phase);
        else if (threads == 128 && cpt == 2)
            k_step_batch<L, MODEL, S, 128, 2><<<grid, 128, 0, st>>>(descs, block_dom, nblocks, phase);
        else if (threads == 256 && cpt == 2)
            k_step_batch<L, MODEL, S, 256, 2><<<grid, 256, 0, st>>>(descs, block_dom, nblocks, phase);
        else
            return cudaErrorInvalidValue;
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t launch_batch_model(int model, bool check, const BatchDesc* descs, const int* block_dom,
                               int nblocks, int grid, int phase, double* partials, int threads,
                               int cpt, cudaStream_t st) {
    if (model == kModelPRImplicit)
        return launch_batch_t<L, kModelPRImplicit, S>(check, descs, block_dom, nblocks, grid, phase, partials, threads, cpt, st);
    if (model == LBM_MODEL_PR)
        return launch_batch_t<L, LBM_MODEL_PR, S>(check, descs, block_dom, nblocks, grid, phase, partials, threads, cpt, st);
    return launch_batch_t<L, LBM_MODEL_IR, S>(check, descs, block_dom, nblocks, grid, phase, partials, threads, cpt, st);
}

template <class L>
cudaError_t launch_batch_lat(int model, int storage, bool check, const BatchDesc* descs,
                             const int* block_dom, int nblocks, int grid, int phase,
                             double* partials, int threads, int cpt, cudaStream_t st) {
    switch (storage) {
    case LBM_F32: return launch_batch_model<L, float>(model, check, descs, block_dom, nblocks, grid, phase, partials, threads, cpt, st);
    case LBM_F64: return launch_batch_model<L, double>(model, check, descs, block_dom, nblocks, grid, phase, partials, threads, cpt, st);
    case LBM_F16_OFS: return launch_batch_model<L, __half>(model, check, descs, block_dom, nblocks, grid, phase, partials, threads, cpt, st);
    case LBM_BF16_OFS: return launch_batch_model<L, __nv_bfloat16>(model, check, descs, block_dom, nblocks, grid, phase, partials, threads, cpt, st);
    default: return cudaErrorNotSupported;
    }
}

template <class L>
cudaError_t launch_links_lat(const KParams& kp, const uint8_t* mask, uint32_t* links,
                             const int* cellidx, cudaStream_t st) {
    if (cellidx)
        k_links_compact<L><<<step_grid(kp.nslots), kBlock, 0, st>>>(kp, mask, cellidx, links);
    else
        k_links<L><<<step_grid(kp.ncells), kBlock, 0, st>>>(kp, mask, links);
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t launch_fields_s(const KArgs& a, const void* f, const uint32_t* links, const int* rank,
                            double* rho, double* ux, double* uy, double* uz, cudaStream_t st) {
    const int grid = step_grid(a.kp.ncells);
    const SrcPlanes<S> P = src_planes<L, S>(f, a.kp.plane);
    if (rank)
        k_fields_compact<L, S><<<grid, kBlock, 0, st>>>(a, P, links, rank, rho, ux, uy, uz);
    else
        k_fields<L, S><<<grid, kBlock, 0, st>>>(a, P, links, rho, ux, uy, uz);
    return cudaGetLastError();
}

template <class L>
cudaError_t launch_fields_lat(int storage, const KParams& kp, const void* f, const uint32_t* links,
                              const int* rank, double* rho, double* ux, double* uy, double* uz,
                              cudaStream_t st) {
    const KArgs a = make_args<L>(kp);
    switch (storage) {
    case LBM_F32: return launch_fields_s<L, float>(a, f, links, rank, rho, ux, uy, uz, st);
    case LBM_F64: return launch_fields_s<L, double>(a, f, links, rank, rho, ux, uy, uz, st);
    case LBM_F16_OFS: return launch_fields_s<L, __half>(a, f, links, rank, rho, ux, uy, uz, st);
    case LBM_BF16_OFS: return launch_fields_s<L, __nv_bfloat16>(a, f, links, rank, rho, ux, uy, uz, st);
    default: return cudaErrorNotSupported;
    }
}

template <class L, class S>
cudaError_t launch_reduce_s(int mode, const KArgs& a, const void* f, const uint32_t* links,
                            const int* cellidx, const int* rank, double* partials, int nblocks,
                            cudaStream_t st) {
    const SrcPlanes<S> P = src_planes<L, S>(f, a.kp.plane);
    if (cellidx) {
        if (mode == kReduceFlow)
            k_reduce<L, S, kReduceFlow, true><<<nblocks, kBlock, 0, st>>>(a, P, links, cellidx, rank, partials);
        else
            k_reduce<L, S, kReduceTotals, true><<<nblocks, kBlock, 0, st>>>(a, P, links, cellidx, rank, partials);
    } else {
        if (mode == kReduceFlow)
            k_reduce<L, S, kReduceFlow, false><<<nblocks, kBlock, 0, st>>>(a, P, links, nullptr, nullptr, partials);
        else
            k_reduce<L, S, kReduceTotals, false><<<nblocks, kBlock, 0, st>>>(a, P, links, nullptr, nullptr, partials);
    }
    return cudaGetLastError();
}

template <class L>
cudaError_t launch_reduce_lat(int storage, int mode, const KParams& kp, const void* f,
                              const uint32_t* links, const int* cellidx, const int* rank,
                              double* partials, int nblocks, cudaStream_t st) {
    const KArgs a = make_args<L>(kp);
    switch (storage) {
    case LBM_F32: return launch_reduce_s<L, float>(mode, a, f, links, cellidx, rank, partials, nblocks, st);
    case LBM_F64: return launch_reduce_s<L, double>(mode, a, f, links, cellidx, rank, partials, nblocks, st);
    case LBM_F16_OFS: return launch_reduce_s<L, __half>(mode, a, f, links, cellidx, rank, partials, nblocks, st);
    case LBM_BF16_OFS: return launch_reduce_s<L, __nv_bfloat16>(mode, a, f, links, cellidx, rank, partials, nblocks, st);
    default: return cudaErrorNotSupported;
    }
}

template <class L>
cudaError_t launch_convert_lat(int storage, bool to_device, const KParams& kp, int q, void* f,
                               double* buf, const int* rank, cudaStream_t st) {
    const int grid = step_grid(kp.ncells);
    switch (storage) {
    case LBM_F32: k_convert<L, float><<<grid, kBlock, 0, st>>>(kp, q, to_device, (float*)f, buf, rank); break;
    case LBM_F64: k_convert<L, double><<<grid, kBlock, 0, st>>>(kp, q, to_device, (double*)f, buf, rank); break;
    case LBM_F16_OFS: k_convert<L, __half><<<grid, kBlock, 0, st>>>(kp, q, to_device, (__half*)f, buf, rank); break;
    case LBM_BF16_OFS: k_convert<L, __nv_bfloat16><<<grid, kBlock, 0, st>>>(kp, q, to_device, (__nv_bfloat16*)f, buf, rank); break;
    default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

template <class L>
cudaError_t launch_gather_lat(int storage, const KParams& kp, const void* f, const int64_t* cells,
                              int n, double* out, const int* rank, cudaStream_t st) {
    const int grid = (n + kBlock - 1) / kBlock;
    switch (storage) {
    case LBM_F32: k_gather_cells<L, float><<<grid, kBlock, 0, st>>>(kp, (const float*)f, cells, n, out, rank); break;
    case LBM_F64: k_gather_cells<L, double><<<grid, kBlock, 0, st>>>(kp, (const double*)f, cells, n, out, rank); break;
    case LBM_F16_OFS: k_gather_cells<L, __half><<<grid, kBlock, 0, st>>>(kp, (const __half*)f, cells, n, out, rank); break;
    case LBM_BF16_OFS: k_gather_cells<L, __nv_bfloat16><<<grid, kBlock, 0, st>>>(kp, (const __nv_bfloat16*)f, cells, n, out, rank); break;
    default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

template <class L>
cudaError_t launch_halo_lat(int storage, const KParams& kp, void* f, void* buf, int side,
                            bool pack, cudaStream_t st) {
    const int n = face_count<L>() * kp.nx * kp.ny;
    const int grid = (n + kBlock - 1) / kBlock;
    switch (storage) {
    case LBM_F32: k_halo<L, float><<<grid, kBlock, 0, st>>>(kp, (float*)f, (float*)buf, side, pack); break;
    case LBM_F64: k_halo<L, double><<<grid, kBlock, 0, st>>>(kp, (double*)f, (double*)buf, side, pack); break;
    case LBM_F16_OFS: k_halo<L, __half><<<grid, kBlock, 0, st>>>(kp, (__half*)f, (__half*)buf, side, pack); break;
    case LBM_BF16_OFS: k_halo<L, __nv_bfloat16><<<grid, kBlock, 0, st>>>(kp, (__nv_bfloat16*)f, (__nv_bfloat16*)buf, side, pack); break;
    default: return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

template <class L> int face_count_lat() { return face_count<L>(); }

template <class L> void lattice_table(int* c, double* w) {
    for (int i = 0; i < L::Q; ++i) {
        if (c) {
            c[3 * i] = L::cx(i);
            c[3 * i + 1] = L::cy(i);
            c[3 * i + 2] = L::cz(i);
        }
        if (w) w[i] = L::w(i);
    }
}

}  // namespace blbm

#define BLBM_DEFINE_LAUNCHERS(L)                                                               \
    namespace blbm {                                                                            \
    cudaError_t launch_step_##L(int model, int storage, bool check, const KParams& kp,         \
                                const StepArgs& a, cudaStream_t st) {                           \
        return launch_step_lat<L>(model, storage, check, kp, a, st);                            \
    }                                                                                           \
    cudaError_t launch_links_##L(const KParams& kp, const uint8_t* mask, uint32_t* links,      \
                                 const int* cellidx, cudaStream_t st) {                         \
        return launch_links_lat<L>(kp, mask, links, cellidx, st);                               \
    }                                                                                           \
    cudaError_t launch_fields_##L(int storage, const KParams& kp, const void* f,               \
                                  const uint32_t* links, const int* rank, double* rho,         \
                                  double* ux, double* uy, double* uz, cudaStream_t st) {        \
        return launch_fields_lat<L>(storage, kp, f, links, rank, rho, ux, uy, uz, st);          \
    }                                                                                           \
    cudaError_t launch_reduce_##L(int storage, int mode, const KParams& kp, const void* f,     \
                                  const uint32_t* links, const int* cellidx, const int* rank,  \
                                  double* partials, int nblocks, cudaStream_t st) {             \
        return launch_reduce_lat<L>(storage, mode, kp, f, links, cellidx, rank, partials,       \
                                    nblocks, st);                                               \
    }                                                                                           \
    cudaError_t launch_convert_##L(int storage, bool to_device, const KParams& kp, int q,      \
                                   void* f, double* plane_buf, const int* rank,                 \
                                   cudaStream_t st) {                                           \
        return launch_convert_lat<L>(storage, to_device, kp, q, f, plane_buf, rank, st);        \
    }                                                                                           \
    void lattice_table_##L(int* c, double* w) { lattice_table<L>(c, w); }                       \
    cudaError_t launch_gather_##L(int storage, const KParams& kp, const void* f,               \
                                  const int64_t* cells, int n, double* out, const int* rank,   \
                                  cudaStream_t st) {                                            \
        return launch_gather_lat<L>(storage, kp, f, cells, n, out, rank, st);                   \
    }                                                                                           \
    cudaError_t launch_halo_##L(int storage, const KParams& kp, void* f, void* buf, int side,  \
                                bool pack, cudaStream_t st) {                                   \
        return launch_halo_lat<L>(storage, kp, f, buf, side, pack, st);                         \
    }                                                                                           \
    int face_count_##L() { return face_count_lat<L>(); }                                        \
    }

// The batch kernels of a lattice, in a translation unit of their own.
#define BLBM_DEFINE_BATCH_LAUNCHERS(L)                                                         \
    namespace blbm {                                                                            \
    cudaError_t launch_step_batch_##L(int model, int storage, bool check, const BatchDesc* descs,\
                                      const int* block_dom, int nblocks, int grid, int phase,  \
                                      double* partials, int threads, int cpt, cudaStream_t st) {\
        return launch_batch_lat<L>(model, storage, check, descs, block_dom, nblocks, grid,      \
                                   phase, partials, threads, cpt, st);                          \
    }                                                                                           \
    }
