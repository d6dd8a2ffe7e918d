// device_math.cuh -- small device helpers: Philox4x32-10, float-float
// arithmetic, complex multiply, fixed-point cell lookup.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "fdf_internal.cuh"

namespace fdf {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, each two
// 32x32 -> 64-bit products mixed with the other two words and the key; the key
// is bumped by the Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// ---- float-float (Dekker / Knuth error-free transforms on the FP32 pipe) ----
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e)  // |a| >= |b|
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    FF r;
    fast_two_sum(s, e, r.hi, r.lo);
    return r;
}

__device__ __forceinline__ FF ff_mul(FF a, FF b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    FF r;
    fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

// 1/sqrt(s) to about 2^-44 relative: hardware seed and one Newton step whose
// residual 1 - s y^2 is formed exactly enough in float-float.
__device__ __forceinline__ FF ff_rsqrt(FF s)
{
    const float y = rsqrtf(s.hi);
    const float y2 = __fmul_rn(y, y);
    const float y2e = __fmaf_rn(y, y, -y2);
    const float p = __fmul_rn(s.hi, y2);
    const float pe = __fmaf_rn(s.hi, y2, -p);
    const float res = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, p), pe), __fmaf_rn(s.hi, y2e, __fmul_rn(s.lo, y2)));
    FF r;
    fast_two_sum(y, __fmul_rn(__fmul_rn(0.5f, y), res), r.hi, r.lo);
    return r;
}

// ---- FP64 <-> FP32 on the integer pipe ---------------------------------------
// GB300 converts between FP64 and FP32 at its FP64 rate (two per clock per SM, the
// rate of its FMAs), so the FP64-state particle pass converts with bit operations,
// which run on the integer pipe.  Both follow the IEEE-754 binary64 and binary32
// layouts (sign, biased exponent, fraction; the biases differ by 1023 - 127 = 896).
//
// d2f_bits: a double in the FP32 normal range (or a value below 2^-126 in
// magnitude, returned as a signed zero) to the nearest float, ties away from zero.
__device__ __forceinline__ float d2f_bits(double d)
{
    const uint32_t hi = (uint32_t)__double2hiint(d), lo = (uint32_t)__double2loint(d);
    const uint32_t sign = hi & 0x80000000u, mag = hi & 0x7FFFFFFFu;
    // exponent rebias (896 << 20 in the high word, then << 3 into binary32's field),
    // the top 23 fraction bits, and the next bit to round; a carry out of the fraction
    // moves into the exponent, as it must
    uint32_t f = (((mag - 0x38000000u) << 3) | (lo >> 29)) + ((lo >> 28) & 1u);
    f = mag < 0x38100000u ? 0u : f;
    return __uint_as_float(sign | f);
}

// f2d_bits: a float (normal or zero; subnormals flush to zero) to the equal double.
__device__ __forceinline__ double f2d_bits(float f)
{
    const uint32_t b = __float_as_uint(f);
    const uint32_t mag = b & 0x7FFFFFFFu;
    const uint32_t hi = mag < 0x00800000u ? (b & 0x80000000u) : (((mag >> 3) + 0x38000000u) | (b & 0x80000000u));
    const uint32_t lo = mag < 0x00800000u ? 0u : (b << 29);
    return __hiloint2double((int)hi, (int)lo);
}

// 1/sqrt(u) for u > 0 in the FP32 normal range, to FP64 accuracy with four FP64
// instructions: the FP32 hardware estimate y (relative error below ~2^-21) and one
// Newton-Raphson step for u^(-1/2) taken to second order,
//   r = y (1 + e/2 + 3 e^2 / 8),  e = 1 - u y^2,
// whose error is 5 e^3 / 16 (below 2^-62).  e/2 = 1/2 - u y (y/2) is formed with one
// fused multiply-add in FP64; 3 e^2 / 8 (below 2^-40) is formed in FP32.
__device__ __forceinline__ double rsqrt_fp64(double u)
{
    const float yf = rsqrtf(d2f_bits(u));
    const double y = f2d_bits(yf), yh = f2d_bits(0.5f * yf);
    const double eh = fma(-(u * y), yh, 0.5);                 // e/2
    const float ehf = d2f_bits(eh);
    const double s = eh + f2d_bits(1.5f * ehf * ehf);         // e/2 + 3 e^2 / 8
    return fma(y, s, y);
}

// The same to first order, r = y (1 + e/2), three FP64 instructions, relative error
// 3 e^2 / 8 (below 2^-40): for the kick integrals, which scale a kick of at most ~1e-3
// of |q| and are needed to ~1e-9.
__device__ __forceinline__ double rsqrt_fp64_1(double u)
{
    const float yf = rsqrtf(d2f_bits(u));
    const double y = f2d_bits(yf), yh = f2d_bits(0.5f * yf);
    return fma(y, fma(-(u * y), yh, 0.5), y);
}

// ---- complex ----
__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <typename V> struct Real;
template <> struct Real<float2> { using T = float; };
template <> struct Real<double2> { using T = double; };

template <typename V> __device__ __forceinline__ V mk(typename Real<V>::T x, typename Real<V>::T y);
template <> __device__ __forceinline__ float2 mk<float2>(float x, float y) { return make_float2(x, y); }
template <> __device__ __forceinline__ double2 mk<double2>(double x, double y) { return make_double2(x, y); }

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return mk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return mk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmuli(V a) { return mk<V>(-a.y, a.x); }  // i a

// ---- fixed-point periodic coordinate -> (cell, fraction) on an N grid -------
// X / 2^32 is the position in units of L; cell = floor(X N / 2^32), fraction =
// ((X N) mod 2^32) / 2^32.
__device__ __forceinline__ void fixed_cell(uint32_t X, uint32_t N, uint32_t& i0, uint32_t& i1, float& f)
{
    i0 = __umulhi(X, N);
    f = __uint2float_rn(X * N) * 2.3283064365386963e-10f;
    i1 = (i0 + 1u == N) ? 0u : i0 + 1u;
}

// |q| with the sampler's exactly rounded evaluation order, so that an
// untouched momentum reproduces p = |q_sampled| bit for bit.
__device__ __forceinline__ double norm3_rn(const double q[3])
{
    return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(q[0], q[0]), __dmul_rn(q[1], q[1])), __dmul_rn(q[2], q[2])));
}

// delta-f weight (Sec. 2.2), w = 1 - fbar(|q|)/fbar(p), in the cancellation-free form
// w = -expm1((p - |q|)/T) / (1 + exp(-|q|/T)).
__device__ __forceinline__ double dfweight(double qm, double p, double T)
{
    return -expm1((p - qm) / T) / (1.0 + exp(-qm / T));
}

// The same weight as the FP32/BF16-grid forms compute it: the small difference p - |q| in
// FP64 (|q| from norm3_rn), the rest in FP32 (their momenta carry FP32 rounding
// already, and GB300's FP64 transcendental functions are slow).
__device__ __forceinline__ float dfweight_split(double qm, double p, double T)
{
    const float arg = (float)((p - qm) / T);
    return -expm1f(arg) / (1.f + expf(-(float)qm / (float)T));
}

}  // namespace fdf
