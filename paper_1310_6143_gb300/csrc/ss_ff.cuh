// The thermal Gaussians of the FP32-mixed form: the Box-Muller transform of ss_math.cuh
// evaluated in double-float arithmetic (a value held as the unevaluated sum hi + lo of two
// floats, combined with error-free transformations: Dekker's product via FMA, Knuth's
// TwoSum and the fast two-sum for ordered operands), with a certified rounding to FP32.
//
// The FP32-mixed form stores the thermal field in FP32, so what its kernels need of the FP64
// transform is that transform's result rounded to FP32.  The double-float evaluation gets
// each Gaussian to within about 2^-44.5 (relative) of the exact value, on the FP32 pipes,
// and rounds it to FP32.  That rounding is accepted only when the double-float value lies
// further from the nearest rounding boundary (the midpoint between two floats) than an
// error bound that covers both the double-float evaluation and the FP64 transform
// (2^-41 |g| + 2^-43 R, R the Box-Muller radius; over 20 times the largest error seen in
// tests, and over 10 times the sum of the largest errors of each part over all 2^32
// inputs).  Both then round to the same float.  Otherwise (about four values in 10^5) the
// caller evaluates the FP64 transform and rounds its result.  Either way
// the float is exactly the FP64 transform's result rounded to nearest: the thermal field
// is bit for bit the same as with the FP64 transform, at a fraction of its cost on GB300,
// whose FP64 pipe issues two instructions per cycle per SM against 128 for FP32.
//
// Pieces (notation of ss_math.cuh: u = (w + 1/2) 2^-32 = m 2^-33, m = 2w + 1):
//   * -2 ln u: u = 2^-n f, f in [0.75, 1.5), nearest centre c = J/2048; f - c is an exact
//     multiple of 2^-33 (an integer below 2^23 times a power of two), r = (f - c)(1/c) with
//     1/c a double-float table entry; -2 ln(1 + r) = -2r + r^2 - r^3 (2/3 - r/2 + 2r^2/5)
//     (|r| < 3.3e-4, the r^3 tail in single precision); then + (-2 ln c) + 2 n ln 2, both
//     double-float table entries, added smallest first with the fast two-sum (each sum's
//     larger operand is known).
//   * sqrt(L): s0 = L rsqrt(L) in single precision, then two Newton corrections
//     c_k = (L - (s0 + c_1 + ..)^2) / (2 s0) whose residuals are formed exactly (Dekker's
//     product, FMAs).
//   * sin/cos of 2 pi u: the nearest of 4096 table angles a (one octant tabulated in
//     double-float, the rest by the exact symmetries of ss_math.cuh) and the remainder
//     d = 2 pi rho / 2^33 (|d| <= pi/4096) as a double-float product; sin(a + d) =
//     sin a + sin a (cos d - 1) + cos a sin d and its cosine counterpart, with
//     cos d - 1 = -d^2/2 + d^4/24 and sin d = d - d^3/6 (dropped terms below 1e-17).
//   * g = R cos, R sin: the double-float product, rounded to float with the check above.
#pragma once

#include <stdint.h>

#include "ss_math.cuh"

namespace ss {

// Shared-memory copy of the double-float tables (build_ff_tables):
//   lg[t]   = (1/c hi, 1/c lo, -2 ln c hi, -2 ln c lo), c = (kLogFirst + t) / kLogScale;
//   trig[m] = (sin hi, sin lo, cos hi, cos lo) of pi m / 2048, m = 0..512;
//   ln2[n]  = 2 n ln 2 (hi, lo), n = 0..33.
struct FFTables {
    float4 lg[kLogTab];
    float4 trig[kTrigTab];
    float2 ln2[kLn2Tab];
};

__device__ __forceinline__ void stage_ff_tables(const float4 *src, FFTables &t) {
    float4 *dst = reinterpret_cast<float4 *>(&t);
    for (int i = threadIdx.x; i < kLogTab + kTrigTab; i += blockDim.x) dst[i] = src[i];
    const float2 *s2 = reinterpret_cast<const float2 *>(src + kLogTab + kTrigTab);
    for (int i = threadIdx.x; i < kLn2Tab; i += blockDim.x) t.ln2[i] = s2[i];
}

struct FF {
    float hi, lo;
};

// a b = p + e exactly (Dekker's product through the FMA).
__device__ __forceinline__ FF ff_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return FF{p, fmaf(a, b, -p)};
}

// a + b = s + e exactly (Knuth's TwoSum; no ordering of the operands needed).
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return FF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// a + b = s + e exactly when |a| >= |b| or a = 0 (the fast two-sum).
__device__ __forceinline__ FF ff_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return FF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a + b for |a| >= |b| (or a = 0), normalised.
__device__ __forceinline__ FF ff_add_ordered(FF a, FF b) {
    const FF s = ff_fast_two_sum(a.hi, b.hi);
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

// -2 ln((w + 1/2) 2^-32) in double-float.
__device__ __forceinline__ FF ff_neg2log(uint32_t w, const FFTables &t) {
    const int lz = __clz(w);
    // m = 2w + 1 with its leading one moved to bit 31 (exact for lz >= 1; for lz = 0, m's
    // last bit, a one, falls below bit 0 and `half` keeps it): f = (x + half/2) 2^-31
    const uint32_t x = (w << (lz & 31)) | (lz ? 1u << ((lz - 1) & 31) : 0u);
    const int32_t half = lz == 0 ? 1 : 0;
    const bool big = x >= 0xC0000000u;          // f >= 1.5: use f/2
    const int n = lz + (big ? 0 : 1);           // u = 2^-n f', f' in [0.75, 1.5)
    const int sh = big ? 21 : 20;
    const uint32_t J = (x >> sh) + ((x >> (sh - 1)) & 1u);  // nearest centre c = J / 2048
    // f' - c = (2 (x - J 2^sh) + half) 2^-(32 + big), an integer below 2^22 in magnitude
    const int32_t D = (int32_t)(x - (J << sh));
    const float dk = __int2float_rn(2 * D + half) * (big ? 0x1p-33f : 0x1p-32f);
    const float4 L = t.lg[J - (uint32_t)kLogFirst];
    // r = (f' - c) / c
    const float rh = __fmul_rn(dk, L.x);
    const float rl = fmaf(dk, L.y, fmaf(dk, L.x, -rh));
    // B = -2 ln(1 + r) = -2r + r^2 - r^3 (2/3 - r/2 + 2r^2/5): -2rh + rh^2 by the fast
    // two-sum (|2 rh| >= rh^2), the rest in single precision
    const float p = __fmul_rn(rh, rh);
    const float pe = fmaf(rh, rh, -p);
    const float tail = __fmul_rn(p, rh) * fmaf(rh, fmaf(rh, -0.4f, 0.5f), -2.0f / 3.0f);
    const float bh = fmaf(-2.0f, rh, p);
    const float be = __fsub_rn(p, fmaf(2.0f, rh, bh));
    const float bl = __fadd_rn(__fadd_rn(__fsub_rn(be, 2.0f * rl), fmaf(2.0f * rh, rl, pe)), tail);
    // -2 ln c + B: |-2 ln c| >= 9.7e-4 > |B| unless c = 1 (then -2 ln c = 0); then
    // 2 n ln 2 + (..): 2 n ln 2 >= 1.38 > 0.82 unless n = 0
    const FF X = ff_add_ordered(FF{L.z, L.w}, FF{bh, bl});
    const float2 A = t.ln2[n];
    return ff_add_ordered(FF{A.x, A.y}, X);
}

// sqrt(L) for a normalised double-float 2^-33 < L < 64.
__device__ __forceinline__ FF ff_sqrt(FF L) {
    const float y = rsqrtf(L.hi);
    const float s0 = __fmul_rn(L.hi, y);
    const float hy = 0.5f * y;
    const FF p = ff_two_prod(s0, s0);
    const float r0 = __fadd_rn(__fsub_rn(__fsub_rn(L.hi, p.hi), p.lo), L.lo);  // L - s0^2
    const float c1 = __fmul_rn(r0, hy);
    const float r1 = fmaf(-c1, c1, fmaf(-2.0f * s0, c1, r0));                  // L - (s0 + c1)^2
    const float c2 = r1 * hy;
    const FF s = ff_fast_two_sum(s0, c1);
    return FF{s.hi, __fadd_rn(s.lo, c2)};
}

// The binary angle 2 pi (2w + 1) / 2^33 split into an octant o, a table angle a of the first
// octant (its double-float sine and cosine in tv) and the remainder d as sin d = dh + sdl,
// cos d - 1 = cmh + cml, taken with the sign that makes theta = (octant symmetry)(a + d).
struct FFTurn {
    uint32_t o;
    float4 tv;
    float dh, sdl, cmh, cml;
};

__device__ __forceinline__ FFTurn ff_turn(uint32_t w, const FFTables &t) {
    constexpr double C = 6.283185307179586 / 8589934592.0;  // 2 pi / 2^33
    constexpr float Ch = (float)C;
    constexpr float Cl = (float)(C - (double)Ch);
    const uint32_t q = (w >> 20) + ((w >> 19) & 1u);        // nearest multiple of 2^21 of 2w + 1
    const int32_t rho = (int32_t)(2u * w + 1u - (q << 21));  // |rho| < 2^20, exact in float
    const uint32_t j = q & 4095u, o = j >> 9, m = j & 511u;
    const bool odd = o & 1u;                                 // reflected octant: a = pi/4 - ..
    FFTurn r;
    r.o = o;
    r.tv = t.trig[odd ? 512u - m : m];
    const float rf = __int2float_rn(odd ? -rho : rho);
    r.dh = __fmul_rn(rf, Ch);
    const float dl = fmaf(rf, Cl, fmaf(rf, Ch, -r.dh));
    const FF p = ff_two_prod(r.dh, r.dh);
    r.cmh = -0.5f * p.hi;
    r.cml = fmaf(-r.dh, dl, fmaf(p.hi, p.hi * (1.0f / 24.0f), -0.5f * p.lo));
    r.sdl = fmaf(-r.dh, p.hi * (1.0f / 6.0f), dl);
    return r;
}

// P (1 + (cos d - 1)) + Q sin d for table values P, Q (double-float): sin(a + d) with
// (P, Q) = (sin a, cos a), cos(a + d) with (cos a, -sin a).
__device__ __forceinline__ FF ff_rot(float Ph, float Pl, float Qh, float Ql, const FFTurn &r) {
    const FF x = ff_two_prod(Qh, r.dh);
    const FF y = ff_two_prod(Ph, r.cmh);
    const FF d = ff_two_sum(x.hi, y.hi);
    const float small = fmaf(Qh, r.sdl, fmaf(Ql, r.dh, fmaf(Ph, r.cml, __fmul_rn(Pl, r.cmh))));
    const float dl = __fadd_rn(__fadd_rn(d.lo, __fadd_rn(x.lo, y.lo)), small);
    const FF s = ff_two_sum(Ph, d.hi);
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(Pl, dl)));
}

__device__ __forceinline__ FF ff_neg(FF a) { return FF{-a.hi, -a.lo}; }

// R V rounded to float; ok is cleared when the rounding is not certain (the value lies within
// the error bound of a midpoint between two floats, or the result is a power of two).
__device__ __forceinline__ float ff_mul_round(FF R, FF V, bool &ok) {
    const float gh = __fmul_rn(R.hi, V.hi);
    const float ge = __fadd_rn(fmaf(R.hi, V.hi, -gh), fmaf(R.hi, V.lo, __fmul_rn(R.lo, V.hi)));
    const float f = __fadd_rn(gh, ge);
    const float e = __fadd_rn(__fsub_rn(gh, f), ge);  // (gh + ge) - f
    const uint32_t fb = __float_as_uint(f);
    const float half_ulp = __uint_as_float((fb & 0x7F800000u) - (24u << 23));
    const float bound = fmaf(fabsf(f), 0x1p-41f, R.hi * 0x1p-43f);
    ok = ok && (fb & 0x7FFFFFu) != 0u && fabsf(e) + bound < half_ulp;
    return f;
}

// Three standard Gaussians of one Philox block rounded to float (the values of box_muller3
// rounded to nearest); false when a rounding is not certain, and the caller must then take
// the FP64 transform's rounded values instead.
__device__ __forceinline__ bool box_muller3_ff(const Philox4 &w, const FFTables &t, float &g0, float &g1,
                                               float &g2) {
    const FF R1 = ff_sqrt(ff_neg2log(w.w0, t));
    const FF R2 = ff_sqrt(ff_neg2log(w.w2, t));
    const FFTurn a = ff_turn(w.w1, t);
    const FF sb = ff_rot(a.tv.x, a.tv.y, a.tv.z, a.tv.w, a);    // sin(a + d)
    const FF cb = ff_rot(a.tv.z, a.tv.w, -a.tv.x, -a.tv.y, a);  // cos(a + d)
    // octant o: (sin, cos) = (s, c), (c, s), (c, -s), (s, -c), (-s, -c), (-c, -s), (-c, s), (-s, c)
    const bool swap = ((a.o + 1u) >> 1) & 1u;
    FF S = swap ? cb : sb, Co = swap ? sb : cb;
    if (a.o & 4u) S = ff_neg(S);
    if ((a.o + 2u) & 4u) Co = ff_neg(Co);
    const FFTurn b = ff_turn(w.w3, t);
    const bool swap2 = ((b.o + 1u) >> 1) & 1u;
    FF C2 = swap2 ? ff_rot(b.tv.x, b.tv.y, b.tv.z, b.tv.w, b) : ff_rot(b.tv.z, b.tv.w, -b.tv.x, -b.tv.y, b);
    if ((b.o + 2u) & 4u) C2 = ff_neg(C2);
    bool ok = true;
    g0 = ff_mul_round(R1, Co, ok);
    g1 = ff_mul_round(R1, S, ok);
    g2 = ff_mul_round(R2, C2, ok);
    return ok;
}

// The FP64 transform's Gaussians rounded to float (reading the FP64 tables from global
// memory): the rare draws whose double-float rounding is not certain.
static __device__ __noinline__ void box_muller3_fp64_rounded(Philox4 w, const double2 *tab, float *g) {
    const SmemTables &t = *reinterpret_cast<const SmemTables *>(tab);
    double d0, d1, d2;
    box_muller3(w, t, d0, d1, d2);
    g[0] = d2f_bits(d0);
    g[1] = d2f_bits(d1);
    g[2] = d2f_bits(d2);
}

// Three standard Gaussians rounded to float: the FP64 transform's values, bit for bit.
__device__ __forceinline__ void gaussians_f32(const Philox4 &w, const FFTables &t, const double2 *tab64, float &g0,
                                              float &g1, float &g2) {
    if (!box_muller3_ff(w, t, g0, g1, g2)) {
        float g[3];
        box_muller3_fp64_rounded(w, tab64, g);
        g0 = g[0];
        g1 = g[1];
        g2 = g[2];
    }
}

}  // namespace ss
