// Device helpers shared by the FD stage kernels (one launch per stage) and
// the temporally blocked FD kernel (all stages of a step in one launch): the
// WENO-5 interface value (Sec. 2, Jiang-Shu) evaluated two at a time, and
// periodic index wrapping.
#pragma once

#include <cuda_runtime.h>

namespace lbm {

// Pairs of values evaluated together: the x-face and the y-face of a node
// are two independent WENO-5 reconstructions, computed side by side. For
// float they map to the packed FP32x2 instructions of sm_100+ (one
// instruction, two results); for double they are two scalar operations.
template <typename T>
struct Pr;

template <>
struct Pr<float> {
    using V = float2;
    static __device__ __forceinline__ V mk(float a, float b) { return make_float2(a, b); }
    static __device__ __forceinline__ V sp(float a) { return make_float2(a, a); }
    static __device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
    // a / b through the approximate reciprocal (relative error ~2^-23):
    // b is a normal number far from the range limits here
    static __device__ __forceinline__ float rcp(float x) {
        float r;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ V div(V a, V b) { return __fmul2_rn(a, make_float2(rcp(b.x), rcp(b.y))); }
};

template <>
struct Pr<double> {
    using V = double2;
    static __device__ __forceinline__ V mk(double a, double b) { return make_double2(a, b); }
    static __device__ __forceinline__ V sp(double a) { return make_double2(a, a); }
    static __device__ __forceinline__ V add(V a, V b) { return make_double2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ V mul(V a, V b) { return make_double2(a.x * b.x, a.y * b.y); }
    static __device__ __forceinline__ V fma(V a, V b, V c) { return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y)); }
    static __device__ __forceinline__ V div(V a, V b) { return make_double2(a.x / b.x, a.y / b.y); }
};

// WENO-5 interface values (Jiang-Shu) of two faces at once, from their
// upwind-ordered stencils (a, b, c, d, e) = (f_{i-2}, f_{i-1}, f_i, f_{i+1},
// f_{i+2}) for the face i+1/2:
//   candidates q0 = (2a - 7b + 11c)/6, q1 = (-b + 5c + 2d)/6, q2 = (2c + 5d - e)/6,
//   smoothness beta_r = 13/12 t_r^2 + 1/4 u_r^2 with the second differences
//     t_r and the first differences u0 = a - 4b + 3c, u1 = b - d,
//     u2 = 3c - 4d + e of the three stencils,
//   weights alpha_r = d_r / (eps + beta_r)^2, d = (1/10, 6/10, 3/10),
//   face = sum alpha_r q_r / sum alpha_r.
// The normalised weights do not change when every alpha_r is multiplied by
// one common factor, so the kernel uses s_r = (12/13)(eps + beta_r) =
// t_r^2 + (3/13) u_r^2 + e (e = 12 eps / 13, passed in), d = (1, 6, 3), and
// multiplies numerator and denominator by s0^2 s1^2 s2^2: one reciprocal per
// face. All differences come from the four node differences D_i = f_{i+1} - f_i
// of the stencil (exact for close values). With q_r = c + (t_r + 3 u_r')/12
// (u_r' = u0, -u1, -u2) the function returns 12 (face - c): a small number
// next to c, so its rounding is small next to the flux differences it feeds.
template <typename T>
__device__ __forceinline__ typename Pr<T>::V weno5_pair(typename Pr<T>::V a, typename Pr<T>::V b, typename Pr<T>::V c,
                                                        typename Pr<T>::V d, typename Pr<T>::V e, typename Pr<T>::V eps_s) {
    using P = Pr<T>;
    using V = typename P::V;
    const V m1 = P::sp(T(-1));
    const V D1 = P::fma(a, m1, b), D2 = P::fma(b, m1, c), D3 = P::fma(c, m1, d), D4 = P::fma(d, m1, e);
    const V t0 = P::fma(D1, m1, D2), t1 = P::fma(D2, m1, D3), t2 = P::fma(D3, m1, D4);
    const V u0 = P::fma(D2, P::sp(T(-3)), D1);   // -(a - 4b + 3c)
    const V u1 = P::add(D2, D3);                  // d - b
    const V u2 = P::fma(D3, P::sp(T(-3)), D4);   // 3c - 4d + e
    const V q0 = P::fma(u0, P::sp(T(-3)), t0);   // 12 (q0 - c)
    const V q1 = P::fma(u1, P::sp(T(3)), t1);    // 12 (q1 - c)
    const V q2 = P::fma(u2, P::sp(T(-3)), t2);   // 12 (q2 - c)
    const V k = P::sp(T(3.0 / 13.0));
    V s0 = P::fma(t0, t0, P::fma(P::mul(u0, k), u0, eps_s));
    V s1 = P::fma(t1, t1, P::fma(P::mul(u1, k), u1, eps_s));
    V s2 = P::fma(t2, t2, P::fma(P::mul(u2, k), u2, eps_s));
    s0 = P::mul(s0, s0);
    s1 = P::mul(s1, s1);
    s2 = P::mul(s2, s2);
    const V w0 = P::mul(s1, s2);                          // d0 s1^2 s2^2
    const V w1 = P::mul(P::mul(s0, s2), P::sp(T(6)));     // d1 s0^2 s2^2
    const V w2 = P::mul(P::mul(s0, s1), P::sp(T(3)));     // d2 s0^2 s1^2
    const V num = P::fma(q2, w2, P::fma(q1, w1, P::mul(q0, w0)));
    const V den = P::add(P::add(w0, w1), w2);
    return P::div(num, den);
}

__device__ __forceinline__ int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

}  // namespace lbm
