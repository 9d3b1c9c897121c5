// Device arithmetic of the thermal field: Philox4x32-10 and an FP64 Box-Muller transform.
//
// Philox4x32-10 follows Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy
// as 1, 2, 3" (SC'11): ten rounds, each two 32x32->64 multiplications by the published
// multipliers, the key advanced by the published Weyl increments between rounds.
//
// The Box-Muller transform (Box and Muller, 1958) takes the four words w0..w3 of one
// Philox block as uniforms u_k = (w_k + 1/2) 2^-32 and returns
//   gx = sqrt(-2 ln u0) cos(2 pi u1), gy = sqrt(-2 ln u0) sin(2 pi u1),
//   gz = sqrt(-2 ln u2) cos(2 pi u3).
// It is evaluated in FP64 with the project's own table-driven functions (GB300's FP64
// pipe is narrow, so every FP64 instruction counts):
//   * -2 ln u by Tang's table-driven method (P. T. P. Tang, "Table-driven implementation
//     of the logarithm function in IEEE floating-point arithmetic", ACM TOMS 16, 1990):
//     u = 2^-n f with f in [0.75, 1.5) taken exactly from the integer 2w+1; f is reduced
//     against the nearest table centre c = k/2048 through r = f (1/c) - 1, where the
//     table's 1/c is rounded to 21 bits so that the product of the integers behind f and
//     1/c is exact in 64-bit integer arithmetic (r is then exact, and its double is
//     assembled from the bits), and
//     -2 ln u = 2 n ln 2 - 2 ln c - 2r + r^2 - r^3 (2/3 - r/2 + 2r^2/5) (Taylor series of
//     2 log1p(r), |r| < 6.6e-4).  The r^3 tail is below 1.9e-10, so single precision
//     evaluates it to an absolute 2e-17; the leading terms stay in FP64.  The tables hold
//     2 n ln 2 and -2 ln c as integer multiples of 2^-45 plus small remainders, so the sum
//     of the two leading constants is an exact integer difference whose double is built
//     from its bits (no FP64 instruction); the remainders join the single-precision tail.
//     Near u = 1 (n = 0, c = 1, r exact) the result keeps its relative accuracy.
//   * sqrt(x): 1/sqrt(x) refined to about 2^-45 in single precision with error-free float
//     products, s = sqrt(x) from it as a float pair whose double is assembled from the
//     bits, then one Newton step in FP64, sqrt(x) = s + (x - s^2) / (2s), the residual
//     from one FMA (the same seed serves the FP64 form's renormalisation, rsqrt_pos).
//   * sin/cos of 2 pi t / 2^33 (t = 2w+1, an exact binary angle) by the nearest of 4096
//     angles a (tabulated for one octant, the rest by exact symmetries) and the remainder
//     d = 2 pi rho / 2^33, |d| <= pi/4096: sin(a+d) = cos a sin d + sin a cos d,
//     cos(a+d) = cos a cos d - sin a sin d, with sin d = d - d^3/6 and
//     cos d = (1 - d^2/2) + d^4/24 (dropped terms below 2.2e-18).  d is carried as a pair
//     of floats (rho is exact in single precision); only the products of the table values
//     with the leading parts of sin d and cos d run in FP64, the rest in single precision
//     (those parts are below 1e-10, so within 1e-17 absolute).  1 - p/2 (p = d^2 rounded
//     to float) is exact in double for p >= 2^-29 and is built from the bits of p.
// All results are within a few units in the last place of the correctly rounded values;
// the tests compare them with CUDA's own log, sqrt and sincospi and with the CPU oracle.
#pragma once

#include <stdint.h>

#include "ss_internal.h"

namespace ss {

struct Philox4 {
    uint32_t w0, w1, w2, w3;
};

// Shared-memory copy of the Box-Muller tables (build_bm_tables):
//   log_[t] = (C_t, M_t, both as int64 bits), C_t = round(2^20 / c_t) (1/c_t rounded to
//             21 bits: 2^-20 C_t), M_t = round(2^45 T_t), T_t = -2 ln(2^-20 C_t);
//   lolog[t] = T_t - 2^-45 M_t (|.| <= 2^-46);
//   ln2[n] = (N_n as int64 bits, 2 n ln 2 - 2^-45 N_n), N_n = round(2^45 2 n ln 2);
//   trig[m] = (sin, cos) of pi m / 2048.
struct SmemTables {
    double2 log_[kLogTab];
    double2 ln2[kLn2Tab];
    double2 trig[kTrigTab];
    float lolog[kLogTab];
};

__device__ __forceinline__ void stage_bm_tables(const double2 *tab, SmemTables &t) {
    for (int i = threadIdx.x; i < kLogTab; i += blockDim.x) t.log_[i] = tab[i];
    for (int i = threadIdx.x; i < kLn2Tab; i += blockDim.x) t.ln2[i] = tab[kLogTab + i];
    for (int i = threadIdx.x; i < kTrigTab; i += blockDim.x) t.trig[i] = tab[kLogTab + kLn2Tab + i];
    const float *lo = reinterpret_cast<const float *>(tab + kLogTab + kLn2Tab + kTrigTab);
    for (int i = threadIdx.x; i < kLogTab; i += blockDim.x) t.lolog[i] = lo[i];
}

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return Philox4{c0, c1, c2, c3};
}

// Exact float -> double from the bits (no FP64 instruction).  Subnormal floats become
// signed zero; infinities and NaN keep their class.
__device__ __forceinline__ double f2d_bits(float f) {
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xFFu;
    const uint32_t E = e == 0xFFu ? 0x7FFu : e + 896u;
    const uint32_t hi = (b & 0x80000000u) | (e ? (E << 20) | ((b & 0x7FFFFFu) >> 3) : 0u);
    const uint32_t lo = e ? b << 29 : 0u;
    return __hiloint2double((int)hi, (int)lo);
}

// double -> float rounded to nearest-even, from the bits, for finite non-zero x with
// 2^-126 <= |x| < 2^127 (no FP64 instruction).
__device__ __forceinline__ float d2f_bits(double x) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const uint32_t e = (uint32_t)((b >> 52) & 0x7FFu) - 896u;
    const uint64_t m = b & 0x000FFFFFFFFFFFFFull;
    const uint64_t mr = (m + 0x0FFFFFFFull + ((m >> 29) & 1ull)) >> 29;  // may carry into the exponent
    return __uint_as_float(sign | ((e << 23) + (uint32_t)mr));
}

// double -> float rounded to nearest for |x| < 2^127; values below 2^-126 in magnitude
// (including zero) give zero (no FP64 instruction).
__device__ __forceinline__ float d2f_small(double x) {
    const uint32_t ex = (uint32_t)(__double2hiint(x) >> 20) & 0x7FFu;
    return ex >= 897u ? d2f_bits(x) : 0.0f;
}

// v 2^-q as a double for |v| < 2^53 and 0 <= q <= 60 (exact), assembled from the integer
// bits.
__device__ __forceinline__ double fixed_to_double(int64_t v, int q) {
    const uint64_t sign = (uint64_t)v & 0x8000000000000000ull;
    const uint64_t a = v < 0 ? (uint64_t)(-v) : (uint64_t)v;
    const int lz = __clzll((long long)a);                        // a in [2^(63-lz), 2^(64-lz))
    const uint64_t mn = a << ((lz - 11) & 63);                   // leading one at bit 52
    const uint64_t bits = sign | (((uint64_t)(1023 + 63 - lz - q - 1) << 52) + mn);
    return a ? __longlong_as_double((long long)bits) : 0.0;
}

// -2 ln((w + 1/2) 2^-32) from the tables of SmemTables.  Three FP64 instructions.
__device__ __forceinline__ double neg2log_u(uint32_t w, const SmemTables &tab) {
    const uint64_t m = 2ull * w + 1ull;              // u = m 2^-33, m odd, < 2^33
    const int lz = __clzll((long long)m);
    const int k = 63 - lz;                           // m in [2^k, 2^(k+1)), k <= 32
    const uint64_t frac = (m << (52 - k)) & 0x000FFFFFFFFFFFFFull;  // f = 1.frac in [1, 2)
    const bool big = frac >= (1ull << 51);           // f >= 1.5: use f/2 and k + 1
    const int n = 33 - k - (big ? 1 : 0);            // u = 2^-n f'
    const int K = k + (big ? 1 : 0);                 // f' = m 2^-K in [0.75, 1.5)
    // nearest centre c = j/2048: j = round(2048 f')
    const uint32_t j = big ? (uint32_t)(1024u + (uint32_t)((frac + (1ull << 41)) >> 42))
                           : (uint32_t)(2048u + (uint32_t)((frac + (1ull << 40)) >> 41));
    const double2 tl = tab.log_[j - (uint32_t)kLogFirst];
    const double2 tn = tab.ln2[n];
    // r = f' 2^-20 C - 1 = (m C - 2^(K+20)) 2^-(K+20): m < 2^33 and C < 2^21, so the
    // integer product is exact; |r| < 3.3e-4
    const uint64_t C = (uint64_t)__double_as_longlong(tl.x);
    const int64_t Dr = (int64_t)(m * C) - (int64_t)(1ull << (K + 20));
    const double r = fixed_to_double(Dr, K + 20);
    const float rf = d2f_small(r);
    const float tail = ((rf * rf) * rf) * fmaf(rf, fmaf(rf, 0.4f, -0.5f), 2.0f / 3.0f);
    // 2 n ln 2 - T = 2^-45 (N - M) + (remainders); N - M >= 0 (the result is positive
    // for n >= 1, and c <= 1 for n = 0) and < 2^51
    const uint64_t nm = (uint64_t)__double_as_longlong(tn.x) - (uint64_t)__double_as_longlong(tl.y);
    const float lo = d2f_small(tn.y) - tab.lolog[j - (uint32_t)kLogFirst];
    const double c = f2d_bits(lo - tail);                // remainders minus the tail
    const double b = fma(-2.0, r, fma(r, r, c));         // -2r + r^2 + c
    return fixed_to_double((int64_t)nm, 45) + b;
}

// 1/sqrt(x) for 2^-100 < x < 2^100, refined in single precision carried as a float pair:
// x = xh + xl (both taken from the bits of x), y0 = rsqrtf(xh), r = 1 - x y0^2 evaluated
// with error-free products, y = y0 + yl = y0 (1 + r/2 + 3r^2/8) ~ 1/sqrt(x) to about 2^-45.
struct RsqrtPair {
    float xh, xl, y0, yl;
};

__device__ __forceinline__ RsqrtPair rsqrt_pair(double x) {
    const uint64_t b = (uint64_t)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    const float xh = __uint_as_float(((uint32_t)(E - 896) << 23) | (uint32_t)((b >> 29) & 0x7FFFFFu));
    const float scale = __uint_as_float((uint32_t)(E - 1075 + 127) << 23);  // 2^(E - 1075)
    const float xl = __int2float_rn((int)(b & 0x1FFFFFFFu)) * scale;          // x - xh to 2^-48 x
    const float y0 = rsqrtf(xh);
    const float p = y0 * y0;
    const float q = fmaf(y0, y0, -p);        // y0^2 = p + q exactly
    const float P = xh * p;
    const float Pe = fmaf(xh, p, -P);        // xh p = P + Pe exactly
    const float r = ((1.0f - P) - Pe) - fmaf(xh, q, xl * p);
    const float yl = y0 * (r * fmaf(0.375f, r, 0.5f));
    return RsqrtPair{xh, xl, y0, yl};
}

// The refined 1/sqrt(x) as a double (one FP64 add).
__device__ __forceinline__ double rsqrt_seed(double x) {
    const RsqrtPair p = rsqrt_pair(x);
    return f2d_bits(p.y0) + f2d_bits(p.yl);
}

__device__ __forceinline__ double half_of(double y) {  // y / 2 for normal y, from the bits
    return __longlong_as_double(__double_as_longlong(y) - (1ll << 52));
}

// sqrt(x), 2^-100 < x < 2^100: s = x (y0 + yl) as a float pair S + sl (xh y0 = S + Se
// exactly, the cross terms in single precision; about 2^-44), then one Newton step in
// FP64, sqrt(x) = s + (x - s^2) h with h = (y0 + yl)/2 rounded to float, the residual
// x - s^2 from one FMA -- two FP64 instructions, within half an ulp but for the last
// rounding.  The double s is S + sl placed on the double grid of S from the bits (bits
// of sl below that grid are dropped; just below a power of two the grid is twice as
// fine): a start within about 2^-44, where the step needs 2^-30.
__device__ __forceinline__ double sqrt_pos(double x) {
    const RsqrtPair p = rsqrt_pair(x);
    const float S = p.xh * p.y0;
    const float Se = fmaf(p.xh, p.y0, -S);
    const float sl = Se + fmaf(p.xh, p.yl, p.xl * p.y0);
    const uint64_t Sb = (uint64_t)__double_as_longlong(f2d_bits(S));
    const uint32_t lb = __float_as_uint(sl);
    const int el = (int)((lb >> 23) & 0xFFu);
    const int sh = (el - 150) - ((int)(Sb >> 52) - 1075);     // sl = M 2^(el-150), grid 2^(eS-1075)
    const uint32_t M = (lb & 0x7FFFFFu) | 0x800000u;
    int64_t delta = sh >= 0 ? (int64_t)((uint64_t)M << (sh & 31)) : (sh > -32 ? (int64_t)(M >> (-sh)) : 0);
    delta = el == 0 ? 0 : ((lb >> 31) ? -delta : delta);
    if ((Sb & 0x000FFFFFFFFFFFFFull) == 0 && delta < 0) delta *= 2;
    const double s = __longlong_as_double((long long)(Sb + (uint64_t)delta));
    const double e = fma(-s, s, x);
    return fma(e, f2d_bits(0.5f * (p.y0 + p.yl)), s);
}

// 1/sqrt(x), 2^-100 < x < 2^100: one FP64 Newton step from the refined seed -- four FP64
// instructions, about one ulp.
__device__ __forceinline__ double rsqrt_pos(double x) {
    const double y = rsqrt_seed(x);
    const double e = fma(-(x * y), y, 1.0);
    return fma(half_of(y), e, y);
}

// Exact int32 -> double for v != 0, assembled from the integer bits (no FP64 instruction).
__device__ __forceinline__ double int_to_double(int32_t v) {
    const uint32_t sign = (uint32_t)v & 0x80000000u;
    const uint32_t a = v < 0 ? (uint32_t)(-v) : (uint32_t)v;
    const int k = 31 - __clz(a);                                   // a in [2^k, 2^(k+1))
    const uint64_t m = ((uint64_t)a << (52 - k)) & 0x000FFFFFFFFFFFFFull;
    const uint64_t bits = ((uint64_t)sign << 32) | ((uint64_t)(1023 + k) << 52) | m;
    return __longlong_as_double((long long)bits);
}

// Reduction of the binary angle 2 pi (2w+1) / 2^33 to the nearest of 4096 table angles
// (index j) and a remainder d = 2 pi rho / 2^33, |rho| < 2^20 (odd).  rho is exact in
// single precision, so d is formed as a float pair dh + dl (about 2^-48 relative) and
// sin d = dh + sdl, cos d = (1 - p/2) + T with p = dh^2 rounded and sdl, T small floats.
struct TurnSplit {
    uint32_t j;   // angle 2 pi j / 4096
    float dh;     // leading part of d (exact as a double)
    float sdl;    // sin d - dh
    float p;      // dh^2 rounded to float
    float T;      // cos d - (1 - p/2)
};

__device__ __forceinline__ TurnSplit split_turn(uint32_t w) {
    constexpr double C = 6.283185307179586 / 8589934592.0;  // 2 pi / 2^33 (exact scaling)
    constexpr float Ch = (float)C;
    constexpr float Cl = (float)(C - (double)Ch);
    const uint64_t t = 2ull * w + 1ull;
    const uint64_t q = (t + (1ull << 20)) >> 21;            // nearest multiple of 2^21
    const float rho = __int2float_rn((int)(int64_t)(t - (q << 21)));
    TurnSplit s;
    s.j = (uint32_t)q & 4095u;
    s.dh = rho * Ch;
    const float dl = fmaf(rho, Ch, -s.dh) + rho * Cl;        // d = dh + dl
    s.p = s.dh * s.dh;
    const float d2l = fmaf(s.dh, s.dh, -s.p) + 2.0f * (s.dh * dl);  // d^2 = p + d2l
    s.sdl = dl - (s.p * s.dh) * (1.0f / 6.0f);               // sin d = d - d^3/6
    s.T = (s.p * s.p) * (1.0f / 24.0f) - 0.5f * d2l;         // cos d = 1 - d^2/2 + d^4/24
    return s;
}

// 1 - p/2 for 0 <= p < 2^-20 from the bits of p: 2^53 (1 - p/2) = 2^53 - P 2^(e+29) for
// p = P 2^(e-23) (P the 24-bit significand), exact for e >= -29, rounded to nearest below.
__device__ __forceinline__ double one_minus_half(float p) {
    const uint32_t pb = __float_as_uint(p);
    const int sh = (int)(pb >> 23) - 127 + 29;                 // e + 29 <= 8
    const uint32_t P = pb ? ((pb & 0x7FFFFFu) | 0x800000u) : 0u;
    const int k = -sh;                                         // right shift when > 0
    const uint32_t v = sh >= 0 ? P << sh : (k < 32 ? (P + (1u << (k - 1))) >> k : 0u);
    return __longlong_as_double((long long)(0x3FF0000000000000ull - (uint64_t)v));
}

// (sin, cos) of 2 pi j / 4096 from the first-octant table (pi m / 2048, m = 0..512):
// reflect within the octant, swap sine and cosine, flip signs.
__device__ __forceinline__ void octant_lookup(uint32_t j, const double2 *tab_trig, double &sa, double &ca) {
    const uint32_t o = j >> 9, m = j & 511u;
    const double2 v = tab_trig[(o & 1u) ? 512u - m : m];
    const bool swap = ((o + 1u) >> 1) & 1u;
    const double s = swap ? v.y : v.x;
    const double c = swap ? v.x : v.y;
    const long long sbit = (long long)((o & 4u) != 0) << 63;
    const long long cbit = (long long)(((o + 2u) & 4u) != 0) << 63;
    sa = __longlong_as_double(__double_as_longlong(s) ^ sbit);
    ca = __longlong_as_double(__double_as_longlong(c) ^ cbit);
}

// sin(a + d) = cos a sin d + sin a cos d, cos(a + d) = cos a cos d - sin a sin d: the
// FP64 parts are cos a dh, sin a (1 - p/2) and their cosine counterparts; the products of
// the table values with the small float parts are formed in single precision (below
// 1e-10 in size, so within 1e-17 absolute).  Four FP64 instructions for both outputs.
__device__ __forceinline__ void sincos_turn(uint32_t w, const double2 *tab_trig, double &sv, double &cv) {
    const TurnSplit ts = split_turn(w);
    double sa, ca;
    octant_lookup(ts.j, tab_trig, sa, ca);
    const float saf = d2f_small(sa), caf = d2f_small(ca);
    const double cd = one_minus_half(ts.p);
    const double dh = f2d_bits(ts.dh);
    sv = fma(ca, dh, fma(sa, cd, f2d_bits(saf * ts.T + caf * ts.sdl)));
    cv = fma(-sa, dh, fma(ca, cd, f2d_bits(caf * ts.T - saf * ts.sdl)));
}

// cos(a + d) alone: two FP64 instructions.
__device__ __forceinline__ double cos_turn(uint32_t w, const double2 *tab_trig) {
    const TurnSplit ts = split_turn(w);
    double sa, ca;
    octant_lookup(ts.j, tab_trig, sa, ca);
    const float saf = d2f_small(sa), caf = d2f_small(ca);
    const double cd = one_minus_half(ts.p);
    return fma(-sa, f2d_bits(ts.dh), fma(ca, cd, f2d_bits(caf * ts.T - saf * ts.sdl)));
}

// Three standard Gaussians of one Philox block (project transform, see the file header):
// 19 FP64 instructions.
__device__ __forceinline__ void box_muller3(const Philox4 &w, const SmemTables &tab, double &gx, double &gy,
                                            double &gz) {
    const double r1 = sqrt_pos(neg2log_u(w.w0, tab));
    const double r2 = sqrt_pos(neg2log_u(w.w2, tab));
    double s1, c1;
    sincos_turn(w.w1, tab.trig, s1, c1);
    const double c2 = cos_turn(w.w3, tab.trig);
    gx = r1 * c1;
    gy = r1 * s1;
    gz = r2 * c2;
}

// The same transform through CUDA's own double-precision functions; used only by the
// diagnostic entry point that checks the table-driven functions above.
__device__ __forceinline__ void box_muller3_libm(const Philox4 &w, double &gx, double &gy, double &gz) {
    const double u0 = ((double)w.w0 + 0.5) * 2.3283064365386963e-10;
    const double u1 = ((double)w.w1 + 0.5) * 2.3283064365386963e-10;
    const double u2 = ((double)w.w2 + 0.5) * 2.3283064365386963e-10;
    const double u3 = ((double)w.w3 + 0.5) * 2.3283064365386963e-10;
    const double r1 = sqrt(-2.0 * log(u0));
    const double r2 = sqrt(-2.0 * log(u2));
    double s1, c1;
    sincospi(2.0 * u1, &s1, &c1);
    gx = r1 * c1;
    gy = r1 * s1;
    gz = r2 * cospi(2.0 * u3);
}

}  // namespace ss
