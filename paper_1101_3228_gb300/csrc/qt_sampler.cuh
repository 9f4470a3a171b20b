// qt_sampler.cuh -- device sampler for the pair draw of Algorithm III.
//
// Prop. 1 (Sec. 3): X_{k+1} = A_k X_k + T_k eps_k.  Algorithm III draws the
// pair (X_k, eps_k) directly for every layer, so layers are independent.  The
// paper leaves the generator open (Sec. 3.1 compares block and skip-ahead
// streams); here a counter-based generator gives every (layer, sample) its
// own stream with no state: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
//
// Every floating-point step below is an explicitly rounded IEEE operation
// (__fadd_rn, __fmul_rn, __fdiv_rn, __fsqrt_rn and their double versions), in a
// fixed order, so the samples are identical bit for bit to those of any other
// correct implementation of the same definition:
//   uniform  FP32: u = (2*(w >> 9) + 1) * 2^-24
//            FP64: u = (2*((w_a >> 6) * 2^26 + (w_b >> 6)) + 1) * 2^-53
//   ln u     split u = 2^e f with f in (sqrt(1/2), sqrt(2)], s = (f-1)/(f+1),
//            ln f = 2 atanh(s) = 2 (s + s z P(z)), z = s^2, P the odd-reciprocal
//            series 1/3 + z/5 + ... (Horner), ln u = e ln2 + ln f
//   sin/cos  2 pi u = q pi/2 + theta with the quarter q and the remainder taken
//            exactly from 4u; theta folded to [0, pi/4]; Taylor polynomials
//   normals  Box & Muller (1958): z0 = sqrt(-2 ln u0) cos(2 pi u1),
//            z1 = sqrt(-2 ln u0) sin(2 pi u1); FP32 calls give two pairs,
//            FP64 calls one.
#pragma once
#include <cstdint>

namespace qt {

struct Philox4 {
    uint32_t v[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    Philox4 r;
    r.v[0] = c0;
    r.v[1] = c1;
    r.v[2] = c2;
    r.v[3] = c3;
    return r;
}

__device__ __forceinline__ float uniform_f32(uint32_t w)
{
    const uint32_t j = w >> 9;
    return __fmul_rn((float)(2u * j + 1u), 0x1p-24f);
}

__device__ __forceinline__ double uniform_f64(uint32_t wa, uint32_t wb)
{
    const unsigned long long j = ((unsigned long long)(wa >> 6) << 26) | (unsigned long long)(wb >> 6);
    return __dmul_rn((double)(2ull * j + 1ull), 0x1p-53);
}

__device__ __forceinline__ float ln_f32(float u)
{
    const uint32_t bits = __float_as_uint(u);
    int e = (int)((bits >> 23) & 0xFFu) - 127;
    float f = __uint_as_float((bits & 0x007FFFFFu) | 0x3F800000u);
    if (f > 1.41421354f) {
        f = __fmul_rn(f, 0.5f);
        e += 1;
    }
    const float s = __fdiv_rn(__fsub_rn(f, 1.0f), __fadd_rn(f, 1.0f));
    const float z = __fmul_rn(s, s);
    float p = (1.0f / 11.0f);
    p = __fadd_rn(__fmul_rn(p, z), (1.0f / 9.0f));
    p = __fadd_rn(__fmul_rn(p, z), (1.0f / 7.0f));
    p = __fadd_rn(__fmul_rn(p, z), (1.0f / 5.0f));
    p = __fadd_rn(__fmul_rn(p, z), (1.0f / 3.0f));
    const float t = __fmul_rn(__fmul_rn(s, z), p);
    const float at = __fadd_rn(s, t);
    const float lnf = __fadd_rn(at, at);
    return __fadd_rn(__fmul_rn((float)e, 0.693147182f), lnf);
}

__device__ __forceinline__ double ln_f64(double u)
{
    const unsigned long long bits = (unsigned long long)__double_as_longlong(u);
    int e = (int)((bits >> 52) & 0x7FFull) - 1023;
    double f = __longlong_as_double((long long)((bits & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull));
    if (f > 1.4142135623730951) {
        f = __dmul_rn(f, 0.5);
        e += 1;
    }
    const double s = __ddiv_rn(__dsub_rn(f, 1.0), __dadd_rn(f, 1.0));
    const double z = __dmul_rn(s, s);
    double p = (1.0 / 21.0);
    p = __dadd_rn(__dmul_rn(p, z), (1.0 / 19.0));
    p = __dadd_rn(__dmul_rn(p, z), (1.0 / 17.0));
    p = __dadd_rn(__dmul_rn(p, z), (1.0 / 15.0));
    p = __dadd_rn(__dmul_rn(p, z), (1.0 / 13.0));
    p = __dadd_rn(__dmul_rn(p, z), (1.0 / 11.0));
    p = __dadd_rn(__dmul_rn(p, z), (1.0 / 9.0));
    p = __dadd_rn(__dmul_rn(p, z), (1.0 / 7.0));
    p = __dadd_rn(__dmul_rn(p, z), (1.0 / 5.0));
    p = __dadd_rn(__dmul_rn(p, z), (1.0 / 3.0));
    const double t = __dmul_rn(__dmul_rn(s, z), p);
    const double at = __dadd_rn(s, t);
    const double lnf = __dadd_rn(at, at);
    return __dadd_rn(__dmul_rn((double)e, 0.6931471805599453), lnf);
}

__device__ __forceinline__ void quarter_sincos_f32(float t, float& s, float& c)
{
    const float t2 = __fmul_rn(t, t);
    float ps = (1.0f / 362880.0f);
    ps = __fadd_rn(__fmul_rn(ps, t2), (-1.0f / 5040.0f));
    ps = __fadd_rn(__fmul_rn(ps, t2), (1.0f / 120.0f));
    ps = __fadd_rn(__fmul_rn(ps, t2), (-1.0f / 6.0f));
    s = __fadd_rn(t, __fmul_rn(__fmul_rn(t, t2), ps));
    float pc = (-1.0f / 3628800.0f);
    pc = __fadd_rn(__fmul_rn(pc, t2), (1.0f / 40320.0f));
    pc = __fadd_rn(__fmul_rn(pc, t2), (-1.0f / 720.0f));
    pc = __fadd_rn(__fmul_rn(pc, t2), (1.0f / 24.0f));
    pc = __fadd_rn(__fmul_rn(pc, t2), (-1.0f / 2.0f));
    c = __fadd_rn(1.0f, __fmul_rn(t2, pc));
}

__device__ __forceinline__ void sincos2pi_f32(float u, float& sn, float& cs)
{
    const float v = __fmul_rn(u, 4.0f);
    const int q = (int)v;
    const float f = __fsub_rn(v, (float)q);
    float st, ct, s0, c0;
    if (f > 0.5f) {
        quarter_sincos_f32(__fmul_rn(__fsub_rn(1.0f, f), 1.57079637f), st, ct);
        s0 = ct;
        c0 = st;
    } else {
        quarter_sincos_f32(__fmul_rn(f, 1.57079637f), st, ct);
        s0 = st;
        c0 = ct;
    }
    switch (q & 3) {
    case 0: sn = s0; cs = c0; break;
    case 1: sn = c0; cs = -s0; break;
    case 2: sn = -s0; cs = -c0; break;
    default: sn = -c0; cs = s0; break;
    }
}

__device__ __forceinline__ void quarter_sincos_f64(double t, double& s, double& c)
{
    const double t2 = __dmul_rn(t, t);
    double ps = (1.0 / 355687428096000.0);
    ps = __dadd_rn(__dmul_rn(ps, t2), (-1.0 / 1307674368000.0));
    ps = __dadd_rn(__dmul_rn(ps, t2), (1.0 / 6227020800.0));
    ps = __dadd_rn(__dmul_rn(ps, t2), (-1.0 / 39916800.0));
    ps = __dadd_rn(__dmul_rn(ps, t2), (1.0 / 362880.0));
    ps = __dadd_rn(__dmul_rn(ps, t2), (-1.0 / 5040.0));
    ps = __dadd_rn(__dmul_rn(ps, t2), (1.0 / 120.0));
    ps = __dadd_rn(__dmul_rn(ps, t2), (-1.0 / 6.0));
    s = __dadd_rn(t, __dmul_rn(__dmul_rn(t, t2), ps));
    double pc = (-1.0 / 6402373705728000.0);
    pc = __dadd_rn(__dmul_rn(pc, t2), (1.0 / 20922789888000.0));
    pc = __dadd_rn(__dmul_rn(pc, t2), (-1.0 / 87178291200.0));
    pc = __dadd_rn(__dmul_rn(pc, t2), (1.0 / 479001600.0));
    pc = __dadd_rn(__dmul_rn(pc, t2), (-1.0 / 3628800.0));
    pc = __dadd_rn(__dmul_rn(pc, t2), (1.0 / 40320.0));
    pc = __dadd_rn(__dmul_rn(pc, t2), (-1.0 / 720.0));
    pc = __dadd_rn(__dmul_rn(pc, t2), (1.0 / 24.0));
    pc = __dadd_rn(__dmul_rn(pc, t2), (-1.0 / 2.0));
    c = __dadd_rn(1.0, __dmul_rn(t2, pc));
}

__device__ __forceinline__ void sincos2pi_f64(double u, double& sn, double& cs)
{
    const double v = __dmul_rn(u, 4.0);
    const int q = (int)v;
    const double f = __dsub_rn(v, (double)q);
    double st, ct, s0, c0;
    if (f > 0.5) {
        quarter_sincos_f64(__dmul_rn(__dsub_rn(1.0, f), 1.5707963267948966), st, ct);
        s0 = ct;
        c0 = st;
    } else {
        quarter_sincos_f64(__dmul_rn(f, 1.5707963267948966), st, ct);
        s0 = st;
        c0 = ct;
    }
    switch (q & 3) {
    case 0: sn = s0; cs = c0; break;
    case 1: sn = c0; cs = -s0; break;
    case 2: sn = -s0; cs = -c0; break;
    default: sn = -c0; cs = s0; break;
    }
}

// Normal stream of (layer k, sample m): g[0 .. count) in FP32.
template <int CNT>
__device__ __forceinline__ void normals_f32(uint64_t seed, int k, uint64_t m, int count, float (&g)[CNT])
{
    const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
    const uint32_t m0 = (uint32_t)m, m1 = (uint32_t)(m >> 32);
#pragma unroll
    for (int r = 0; r < (CNT + 3) / 4; ++r) {
        if (4 * r < count) {
            const Philox4 w = philox4x32_10(m0, m1, (uint32_t)k, (uint32_t)r, key0, key1);
#pragma unroll
            for (int pair = 0; pair < 2; ++pair) {
                const float u0 = uniform_f32(w.v[2 * pair]);
                const float u1 = uniform_f32(w.v[2 * pair + 1]);
                const float rad = __fsqrt_rn(__fmul_rn(-2.0f, ln_f32(u0)));
                float sn, cs;
                sincos2pi_f32(u1, sn, cs);
                const int q = 4 * r + 2 * pair;
                if (q < CNT) g[q] = __fmul_rn(rad, cs);
                if (q + 1 < CNT) g[q + 1] = __fmul_rn(rad, sn);
            }
        }
    }
}

template <int CNT>
__device__ __forceinline__ void normals_f64(uint64_t seed, int k, uint64_t m, int count, double (&g)[CNT])
{
    const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
    const uint32_t m0 = (uint32_t)m, m1 = (uint32_t)(m >> 32);
#pragma unroll
    for (int r = 0; r < (CNT + 1) / 2; ++r) {
        if (2 * r < count) {
            const Philox4 w = philox4x32_10(m0, m1, (uint32_t)k, (uint32_t)r, key0, key1);
            const double u0 = uniform_f64(w.v[0], w.v[1]);
            const double u1 = uniform_f64(w.v[2], w.v[3]);
            const double rad = __dsqrt_rn(__dmul_rn(-2.0, ln_f64(u0)));
            double sn, cs;
            sincos2pi_f64(u1, sn, cs);
            if (2 * r < CNT) g[2 * r] = __dmul_rn(rad, cs);
            if (2 * r + 1 < CNT) g[2 * r + 1] = __dmul_rn(rad, sn);
        }
    }
}

// Per-layer sampler parameters, packed: m[d], b[d], L[d*d], A[d*d], T[d*d].
__host__ __device__ constexpr int param_count(int d) { return 2 * d + 3 * d * d; }

// X = m + L z, Y = b + A X + T eps, rounded step by step in FP32 (DM >= d).
template <int DM>
__device__ __forceinline__ void pair_f32(const float* __restrict__ P, int d, uint64_t seed, int k, uint64_t m,
                                         float (&X)[DM], float (&Y)[DM])
{
    float g[2 * DM];
    normals_f32<2 * DM>(seed, k, m, 2 * d, g);
    const float* pm = P;
    const float* pb = P + d;
    const float* pL = P + 2 * d;
    const float* pA = pL + d * d;
    const float* pT = pA + d * d;
#pragma unroll
    for (int l = 0; l < DM; ++l) {
        float acc = 0.0f;
        if (l < d) {
            acc = pm[l];
#pragma unroll
            for (int q = 0; q <= l; ++q) acc = __fadd_rn(acc, __fmul_rn(pL[l * d + q], g[q]));
        }
        X[l] = acc;
    }
#pragma unroll
    for (int l = 0; l < DM; ++l) {
        float acc = 0.0f;
        if (l < d) {
            acc = pb[l];
#pragma unroll
            for (int q = 0; q < DM; ++q)
                if (q < d) acc = __fadd_rn(acc, __fmul_rn(pA[l * d + q], X[q]));
#pragma unroll
            for (int q = 0; q <= l; ++q) acc = __fadd_rn(acc, __fmul_rn(pT[l * d + q], g[d + q]));
        }
        Y[l] = acc;
    }
}

template <int DM>
__device__ __forceinline__ void pair_f64(const double* __restrict__ P, int d, uint64_t seed, int k, uint64_t m,
                                         double (&X)[DM], double (&Y)[DM])
{
    double g[2 * DM];
    normals_f64<2 * DM>(seed, k, m, 2 * d, g);
    const double* pm = P;
    const double* pb = P + d;
    const double* pL = P + 2 * d;
    const double* pA = pL + d * d;
    const double* pT = pA + d * d;
#pragma unroll
    for (int l = 0; l < DM; ++l) {
        double acc = 0.0;
        if (l < d) {
            acc = pm[l];
#pragma unroll
            for (int q = 0; q <= l; ++q) acc = __dadd_rn(acc, __dmul_rn(pL[l * d + q], g[q]));
        }
        X[l] = acc;
    }
#pragma unroll
    for (int l = 0; l < DM; ++l) {
        double acc = 0.0;
        if (l < d) {
            acc = pb[l];
#pragma unroll
            for (int q = 0; q < DM; ++q)
                if (q < d) acc = __dadd_rn(acc, __dmul_rn(pA[l * d + q], X[q]));
#pragma unroll
            for (int q = 0; q <= l; ++q) acc = __dadd_rn(acc, __dmul_rn(pT[l * d + q], g[d + q]));
        }
        Y[l] = acc;
    }
}

}  // namespace qt
