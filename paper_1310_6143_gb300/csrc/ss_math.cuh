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
//     against the nearest table centre c = k/256 through r = f (1/c) - 1 (one FMA, so
//     the table's rounded 1/c defines the split exactly), and
//     -2 ln u = 2 n ln 2 - 2 ln c - 2 log1p(r), with log1p(r) the Taylor series to r^6
//     (|r| < 2^-8.4, truncation below 2^-60 relative).  Near u = 1 (n = 0, c = 1) the
//     result is -2 log1p(r) with r exact, so it keeps full relative accuracy.
//   * sqrt by two coupled Newton (Goldschmidt) iterations from the single-precision
//     reciprocal square root, each squaring the relative error (2^-21 -> 2^-42 -> 2^-84).
//   * sin/cos of 2 pi t / 2^33 (t = 2w+1, an exact binary angle) by the nearest of 512
//     table angles a and the remainder d = 2 pi rho / 2^33, |d| <= pi/512:
//     sin(a+d) = sin a + (sin a (cos d - 1) + cos a sin d), and likewise for cos, with
//     sin d, cos d - 1 from their Taylor series (errors below 2^-56).
// All results are within a few units in the last place of the correctly rounded values;
// the tests compare them with CUDA's own log, sqrt and sincospi and with the CPU oracle.
#pragma once

#include <stdint.h>

namespace ss {

struct Philox4 {
    uint32_t w0, w1, w2, w3;
};

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

// -2 ln((w + 1/2) 2^-32).  tab_log[t] = (1/c_t rounded, -2 ln(that rounded value)),
// tab_ln2[n] = 2 n ln 2 as (hi, lo).
__device__ __forceinline__ double neg2log_u(uint32_t w, const double2 *tab_log, const double2 *tab_ln2) {
    const uint64_t m = 2ull * w + 1ull;              // u = m 2^-33, m odd, < 2^33
    const int lz = __clzll((long long)m);
    const int k = 63 - lz;                           // m in [2^k, 2^(k+1)), k <= 32
    const uint64_t frac = (m << (52 - k)) & 0x000FFFFFFFFFFFFFull;  // f = 1.frac in [1, 2)
    const bool big = frac >= (1ull << 51);           // f >= 1.5: use f/2 and k + 1
    const int n = 33 - k - (big ? 1 : 0);            // u = 2^-n f'
    const uint64_t ebits = big ? (1022ull << 52) : (1023ull << 52);
    const double fp = __longlong_as_double((long long)(ebits | frac));    // f' in [0.75, 1.5)
    // nearest centre c = j/256: j = round(256 f')
    const uint32_t j = big ? (uint32_t)(128u + (uint32_t)((frac + (1ull << 44)) >> 45))
                           : (uint32_t)(256u + (uint32_t)((frac + (1ull << 43)) >> 44));
    const double2 tl = tab_log[j - 192u];
    const double2 tn = tab_ln2[n];
    const double r = fma(fp, tl.x, -1.0);            // f'/c - 1 up to one rounding
    const double r2 = r * r;
    // 2 log1p(r) = 2r - r^2 + (2/3) r^3 - (1/2) r^4 + (2/5) r^5 - (1/3) r^6
    double t = fma(r, -1.0 / 3.0, 0.4);
    t = fma(r, t, -0.5);
    t = fma(r, t, 2.0 / 3.0);
    t = fma(r, t, -1.0);
    const double p2 = fma(r2, t, r + r);
    const double a = tn.x - tl.y;                    // 2 n ln2 - 2 ln c (leading part)
    return a + (tn.y - p2);
}

// sqrt(x) for 1e-30 < x < 1e30.
__device__ __forceinline__ double sqrt_pos(double x) {
    // single-precision seed from the high word (exponent rebiased, mantissa truncated)
    const int hi = __double2hiint(x);
    const int fe = ((hi >> 20) & 0x7FF) - 1023 + 127;
    const float xf = __int_as_float((fe << 23) | ((hi & 0xFFFFF) << 3));
    const float yf = rsqrtf(xf);
    const int yb = __float_as_int(yf);
    const int ye = ((yb >> 23) & 0xFF) - 127 + 1023;
    const double y = __hiloint2double((ye << 20) | ((yb & 0x7FFFFF) >> 3), (yb & 7) << 29);
    // Goldschmidt: s -> sqrt(x), h -> 1/(2 sqrt(x))
    double s = x * y;
    double h = __hiloint2double(((ye - 1) << 20) | ((yb & 0x7FFFFF) >> 3), (yb & 7) << 29);  // y/2
    double e = fma(-s, h, 0.5);
    s = fma(s, e, s);
    h = fma(h, e, h);
    e = fma(-s, h, 0.5);
    return fma(s, e, s);
}

// Exact int32 -> double through the 2^52 + 2^31 bias (one FP64 add).
__device__ __forceinline__ double int_to_double(int32_t v) {
    const double biased = __hiloint2double(0x43300000, (int)((uint32_t)v ^ 0x80000000u));
    return biased - 4503601774854144.0;  // 2^52 + 2^31
}

// Reduction of the binary angle 2 pi (2w+1) / 2^33 to a table angle and a remainder.
struct TurnSplit {
    uint32_t j;   // table index, angle 2 pi j / 512
    double d;     // remainder angle, |d| <= pi/512
};

__device__ __forceinline__ TurnSplit split_turn(uint32_t w) {
    const uint64_t t = 2ull * w + 1ull;
    const uint64_t q = (t + (1ull << 23)) >> 24;     // nearest multiple of 2^24
    const int32_t rho = (int32_t)(int64_t)(t - (q << 24));
    TurnSplit s;
    s.j = (uint32_t)q & 511u;
    s.d = int_to_double(rho) * (6.283185307179586 / 8589934592.0);  // 2 pi / 2^33 (exact scaling)
    return s;
}

__device__ __forceinline__ void sincos_turn(uint32_t w, const double2 *tab_trig, double &sv, double &cv) {
    const TurnSplit ts = split_turn(w);
    const double d = ts.d;
    const double d2 = d * d;
    const double sd = fma(d2 * d, fma(d2, 1.0 / 120.0, -1.0 / 6.0), d);  // sin d
    const double cm1 = d2 * fma(d2, 1.0 / 24.0, -0.5);                     // cos d - 1
    const double2 sc = tab_trig[ts.j];
    sv = sc.x + fma(sc.y, sd, sc.x * cm1);
    cv = sc.y + fma(-sc.x, sd, sc.y * cm1);
}

__device__ __forceinline__ double cos_turn(uint32_t w, const double2 *tab_trig) {
    const TurnSplit ts = split_turn(w);
    const double d = ts.d;
    const double d2 = d * d;
    const double sd = fma(d2 * d, fma(d2, 1.0 / 120.0, -1.0 / 6.0), d);
    const double cm1 = d2 * fma(d2, 1.0 / 24.0, -0.5);
    const double2 sc = tab_trig[ts.j];
    return sc.y + fma(-sc.x, sd, sc.y * cm1);
}

// Three standard Gaussians of one Philox block (project transform, see the file header).
__device__ __forceinline__ void box_muller3(const Philox4 &w, const double2 *tab_log, const double2 *tab_ln2,
                                            const double2 *tab_trig, double &gx, double &gy, double &gz) {
    const double r1 = sqrt_pos(neg2log_u(w.w0, tab_log, tab_ln2));
    const double r2 = sqrt_pos(neg2log_u(w.w2, tab_log, tab_ln2));
    double s1, c1;
    sincos_turn(w.w1, tab_trig, s1, c1);
    const double c2 = cos_turn(w.w3, tab_trig);
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
