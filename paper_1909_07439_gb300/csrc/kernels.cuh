// Smoothing kernels (Sect. 2.3): W(r, h) = C f(q) / h^3 with q = r / h, zero
// for q >= R (the support radius in units of h), F(r, h) = C f'(q) / h^4
// (Eq. 14).  The paper offers three kernels chosen at compile time so that
// their constants fold; here each is a specialisation of SphKernel<K>, the
// pair kernels are templates on K, and sph_params.kernel selects the
// instantiation:
//   K = 0  M4 cubic spline,  R = 2, C = 1/pi
//          f = 1 - 3/2 q^2 + 3/4 q^3 (q < 1), (2 - q)^3 / 4 (1 <= q < 2)
//   K = 1  M6 quintic spline, R = 3, C = 1/(120 pi)
//          f = a^5 - 6 b^5 + 15 c^5, a = (3 - q)+, b = (2 - q)+, c = (1 - q)+
//   K = 2  Wendland C6, R = 2, C = 1365/(512 pi)
//          f = s^8 (4 q^3 + 25/4 q^2 + 4 q + 1), s = (1 - q/2)+
// (x)+ = max(x, 0): each form is branch-free and vanishes beyond the support.
// Members: f_df(q) -> f, f'; df(q) = f'; d2f(q) = f''; and, in the variable
// p = r / (R h) = r rsqrt((R h)^2) that the force pass evaluates,
// f'(R p) = G g_p(p) with the constant G kept apart so that it folds into a
// per-particle factor.
#pragma once

#include "sph_internal.cuh"

namespace sph {

// Two-lane FP32 arithmetic in the packed FP32x2 instructions (add, multiply,
// fused multiply-add, each rounded to nearest per element).
__device__ __forceinline__ float2 f2(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <int K>
struct SphKernel;

template <>
struct SphKernel<0> {
    static constexpr float R = 2.f;
    static constexpr float C = 0.318309886183790671538f;
    __device__ static __forceinline__ void f_df(float q, float &f, float &df)
    {
        const float fi = 1.f + q * q * (-1.5f + 0.75f * q);
        const float dfi = q * (-3.f + 2.25f * q);
        const float t = fmaxf(2.f - q, 0.f);
        const float t2 = t * t;
        const bool in = q < 1.f;
        f = in ? fi : 0.25f * t2 * t;
        df = in ? dfi : -0.75f * t2;
    }
    __device__ static __forceinline__ float d2f(float q)
    {
        // f' = -3/4 t^2 + 3 s^2, t = (2 - q)+, s = (1 - q)+
        return 1.5f * fmaxf(2.f - q, 0.f) - 6.f * fmaxf(1.f - q, 0.f);
    }
    __device__ static __forceinline__ float df(float q)
    {
        const float inner = q * (-3.f + 2.25f * q);
        const float t = fmaxf(2.f - q, 0.f);
        return q < 1.f ? inner : -0.75f * t * t;
    }
    // f'(2 p) = -3 ((1 - p)+^2 - (1 - 2 p)+^2)
    static constexpr float G = -3.f;
    __device__ static __forceinline__ float g_p(float p)
    {
        const float a = fmaxf(1.f - p, 0.f), b = fmaxf(fmaf(-2.f, p, 1.f), 0.f);
        return fmaf(a, a, -b * b);
    }
};

template <>
struct SphKernel<1> {
    static constexpr float R = 3.f;
    static constexpr float C = 0.00265258238486492226282f;  // 1 / (120 pi)
    __device__ static __forceinline__ void f_df(float q, float &f, float &df)
    {
        const float a = fmaxf(3.f - q, 0.f), b = fmaxf(2.f - q, 0.f), c = fmaxf(1.f - q, 0.f);
        const float a2 = a * a, b2 = b * b, c2 = c * c;
        const float a4 = a2 * a2, b4 = b2 * b2, c4 = c2 * c2;
        f = fmaf(15.f * c4, c, fmaf(-6.f * b4, b, a4 * a));
        df = -5.f * fmaf(15.f, c4, fmaf(-6.f, b4, a4));
    }
    __device__ static __forceinline__ float df(float q)
    {
        const float a = fmaxf(3.f - q, 0.f), b = fmaxf(2.f - q, 0.f), c = fmaxf(1.f - q, 0.f);
        const float a2 = a * a, b2 = b * b, c2 = c * c;
        return -5.f * fmaf(15.f * c2, c2, fmaf(-6.f * b2, b2, a2 * a2));
    }
    __device__ static __forceinline__ float d2f(float q)
    {
        const float a = fmaxf(3.f - q, 0.f), b = fmaxf(2.f - q, 0.f), c = fmaxf(1.f - q, 0.f);
        return 20.f * fmaf(15.f * c * c, c, fmaf(-6.f * b * b, b, a * a * a));
    }
    // q = 3 p: f' = -5 (a^4 - 6 b^4 + 15 c^4), a = 3 (1 - p)+, b = (2 - 3 p)+, c = (1 - 3 p)+
    static constexpr float G = -5.f;
    __device__ static __forceinline__ float g_p(float p)
    {
        const float a = 3.f * fmaxf(1.f - p, 0.f), b = fmaxf(fmaf(-3.f, p, 2.f), 0.f),
                    c = fmaxf(fmaf(-3.f, p, 1.f), 0.f);
        const float a2 = a * a, b2 = b * b, c2 = c * c;
        return fmaf(15.f * c2, c2, fmaf(-6.f * b2, b2, a2 * a2));
    }
};

template <>
struct SphKernel<2> {
    static constexpr float R = 2.f;
    static constexpr float C = 0.848619130157957545f;  // 1365 / (512 pi)
    // f = s^8 P, P = 4 q^3 + 25/4 q^2 + 4 q + 1; f' = -11/2 q s^7 (4 q^2 + 7/2 q + 1)
    __device__ static __forceinline__ void f_df(float q, float &f, float &df)
    {
        const float s = fmaxf(fmaf(-0.5f, q, 1.f), 0.f);
        const float s2 = s * s, s4 = s2 * s2, s7 = s4 * s2 * s;
        const float P = fmaf(fmaf(fmaf(4.f, q, 6.25f), q, 4.f), q, 1.f);
        f = s7 * s * P;
        df = -5.5f * q * s7 * fmaf(fmaf(4.f, q, 3.5f), q, 1.f);
    }
    __device__ static __forceinline__ float df(float q)
    {
        const float s = fmaxf(fmaf(-0.5f, q, 1.f), 0.f);
        const float s2 = s * s, s7 = s2 * s2 * s2 * s;
        return -5.5f * q * s7 * fmaf(fmaf(4.f, q, 3.5f), q, 1.f);
    }
    // f'' = 11/2 s^6 (20 q^3 + 15/4 q^2 - 3 q - 1)
    __device__ static __forceinline__ float d2f(float q)
    {
        const float s = fmaxf(fmaf(-0.5f, q, 1.f), 0.f);
        const float s2 = s * s, s6 = s2 * s2 * s2;
        return 5.5f * s6 * fmaf(fmaf(fmaf(20.f, q, 3.75f), q, -3.f), q, -1.f);
    }
    // q = 2 p: f' = -11 p (1 - p)+^7 (16 p^2 + 7 p + 1)
    static constexpr float G = -11.f;
    __device__ static __forceinline__ float g_p(float p)
    {
        const float s = fmaxf(1.f - p, 0.f);
        const float s2 = s * s, s7 = s2 * s2 * s2 * s;
        return p * s7 * fmaf(fmaf(16.f, p, 7.f), p, 1.f);
    }
};

// support radius, normalisation and G C of kernel k on the host
inline float kernel_support(int k) { return k == 1 ? 3.f : 2.f; }
inline float kernel_norm(int k)
{
    return k == 1 ? SphKernel<1>::C : k == 2 ? SphKernel<2>::C : SphKernel<0>::C;
}
// largest h whose support R h stays below half of every periodic period
// (INFINITY without periodic axes)
inline float periodic_h_limit(const sph_params &p)
{
    float lim = INFINITY;
    const float R = kernel_support(p.kernel);
    for (int a = 0; a < 3; ++a)
        if (p.box_len[a] > 0.f) lim = fminf(lim, 0.5f * p.box_len[a] / R);
    return lim;
}

inline float kernel_gc(int k)
{
    return k == 1 ? SphKernel<1>::G * SphKernel<1>::C
         : k == 2 ? SphKernel<2>::G * SphKernel<2>::C
                  : SphKernel<0>::G * SphKernel<0>::C;
}

}  // namespace sph
