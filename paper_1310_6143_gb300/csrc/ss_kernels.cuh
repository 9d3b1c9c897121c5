// Step kernels of the stochastic Heun-LLG integrator (templated on the working type R).
//
// One step (Section "Time Integration of the LLG Equation" of arXiv:1310.6143):
//   predictor pass, every spin i:
//     H_i  = (1/mu) sum_j J_ij S_j + (2 k_u/mu)(S_i.e) e + H_app [+ (2/mu) K S_i] + H_th,i
//            (Eq. Heff applied to the Hamiltonian; H_th,i from Philox + Box-Muller, drawn
//            once per step at T(t_n) and stored for the corrector)
//     dS_i = -gamma/(1+lambda^2) [S_i x H_i + lambda S_i x (S_i x H_i)]       (Eq. LLG)
//     S'_i = normalise(S_i + dt dS_i),  Q_i = S_i + dt/2 dS_i
//     + FP64 partial sums of sum mu S, E_exc, E_ani, E_app of the state S(t_n)
//   -- every predictor finishes before any corrector starts (kernel boundary, or a grid
//      barrier in the persistent kernel) --
//   corrector pass, every spin i:
//     H'_i from S' with the same H_th,i; dS'_i = LLG(S'_i, H'_i)
//     S_i <- normalise(Q_i + dt/2 dS'_i)   (= S_i + dt/2 (dS_i + dS'_i), then renormalised)
//
// Data layout: spins as structure-of-arrays (three arrays per vector); the neighbour list
// in CSR (int32 offsets and columns, J in the working type); one material index per spin.
// Work is split into tiles (contiguous spins of one system); each tile yields one FP64
// partial of the reductions, summed per system in a fixed order, so the record is
// bitwise reproducible.
#pragma once

#include <cooperative_groups.h>
#include <stdint.h>

#include "ss_internal.h"
#include "ss_ff.cuh"
#include "ss_math.cuh"

namespace ss {

// Loads of data written earlier in the same launch must bypass the non-coherent L1
// (the persistent kernel); everything else may use the read-only path.
template <bool Coherent, typename T>
__device__ __forceinline__ T ld(const T *p) {
    if constexpr (Coherent) {
        return __ldcg(p);
    } else {
        return __ldg(p);
    }
}

// Working-type views of the system's double-precision parameters and of FP64 results:
// the FP32-mixed form reads float copies prepared on the host and converts with integer
// bit operations, so that the narrow FP64 pipe only runs the Box-Muller transform and the
// reduction sums.
__device__ __forceinline__ float sys_H(const SysDesc &sd, int c, float) { return sd.Hf[c]; }
__device__ __forceinline__ double sys_H(const SysDesc &sd, int c, double) { return sd.H[c]; }
__device__ __forceinline__ double widen(float v) { return f2d_bits(v); }
__device__ __forceinline__ double widen(double v) { return v; }
template <typename R> __device__ __forceinline__ R narrow(double v);
// double -> working type for any finite value (the hardware conversion; off the hot path)
template <typename R> __device__ __forceinline__ R narrow_any(double v) { return (R)v; }
template <> __device__ __forceinline__ float narrow<float>(double v) { return d2f_bits(v); }
template <> __device__ __forceinline__ double narrow<double>(double v) { return v; }

template <typename R>
__device__ __forceinline__ R rsqrt_r(R x);
template <>
__device__ __forceinline__ float rsqrt_r<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_r<double>(double x) {
    // |v|^2 of a renormalised spin plus a small step: well inside the range of rsqrt_pos
    return rsqrt_pos(x);
}

// a b rounded, never fused into a following add: the thermal field sigma g is formed this way
// wherever it is used, so that the predictor's and the corrector's fields are the same value.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// True when the reciprocal length of a renormalised spin is NaN or infinite.
__device__ __forceinline__ bool bad_inv(float v) { return !(v < 3.0e38f); }
__device__ __forceinline__ bool bad_inv(double v) { return ((__double2hiint(v) >> 20) & 0x7FF) == 0x7FF; }

template <typename R>
__device__ __forceinline__ void stage_tables(const KArgs<R> &a, SmemTables &t) {
    stage_bm_tables(a.tab, t);
}

// Tables of the Heun step kernels' thermal transform: the FP64 tables for the FP64 form, the
// double-float tables for the FP32-mixed form (whose rare uncertain roundings read the FP64
// tables from global memory).
template <typename R> struct StepTab { using type = SmemTables; };
template <> struct StepTab<float> { using type = FFTables; };
template <typename R> using StepTabT = typename StepTab<R>::type;

__device__ __forceinline__ void stage_step_tables(const KArgs<double> &a, SmemTables &t) { stage_bm_tables(a.tab, t); }
__device__ __forceinline__ void stage_step_tables(const KArgs<float> &a, FFTables &t) { stage_ff_tables(a.fftab, t); }

// Three standard Gaussians of one Philox block in the working type: the FP64 transform, and
// in the FP32-mixed form its values rounded to float (bit for bit, see ss_ff.cuh).
__device__ __forceinline__ void thermal_gaussians(const KArgs<double> &, const SmemTables &tab, const Philox4 &w,
                                                  double &g0, double &g1, double &g2) {
    box_muller3(w, tab, g0, g1, g2);
}
__device__ __forceinline__ void thermal_gaussians(const KArgs<float> &a, const FFTables &tab, const Philox4 &w,
                                                  float &g0, float &g1, float &g2) {
    gaussians_f32(w, tab, a.tab, g0, g1, g2);
}

// H_app + sum_j (J_ij / mu_s,i) X_j over row i (CSR order, one FMA per term and
// component): the exchange plus applied field, in tesla.
// Variants of the step kernels, fixed at compile time so that a plain lattice's kernels carry
// no code for the other cases: kPlain (scalar J, no cubic anisotropy), kGeneral (tensor bonds
// and cubic anisotropy decided per launch / material), kRows (the exchange field summed
// beforehand by k_rows_sell / k_rows_field; cubic per material).
constexpr int kPlain = 0, kGeneral = 1, kRows = 2;
// kUniform: kPlain with a single material, read from the kernel arguments (the Heun step
// kernels only; everything else treats it as kPlain).
constexpr int kUniform = 3;
__host__ __device__ constexpr int base_mode(int mode) { return mode == kUniform ? kPlain : mode; }

// The material index of spin i (stored in one, two or four bytes by the number of materials).
template <typename R>
__device__ __forceinline__ int32_t mat_of(const KArgs<R> &a, int64_t i) {
    if (a.mat_bytes == 1) return __ldg(static_cast<const uint8_t *>(a.mat) + i);
    if (a.mat_bytes == 2) return __ldg(static_cast<const uint16_t *>(a.mat) + i);
    return __ldg(static_cast<const int32_t *>(a.mat) + i);
}

template <int Mode, typename R>
__device__ __forceinline__ const MatDesc<R> &mat_at(const KArgs<R> &a, int64_t i) {
    if constexpr (Mode == kUniform) {
        (void)i;
        return a.mat0;
    } else {
        return a.mats[mat_of(a, i)];
    }
}

// Checked builds (SS_CHECKED): an index about to be gathered with is checked against [0, n);
// a bad one sets kErrBounds in the error word and is replaced by 0, so nothing outside the
// arrays is read.  Other builds return it unchanged.
__device__ __forceinline__ int32_t chk(int64_t j, int64_t n, unsigned int *err) {
#ifdef SS_CHECKED
    if (j < 0 || j >= n) {
        atomicOr(err, kErrBounds);
        return 0;
    }
#else
    (void)n;
    (void)err;
#endif
    return (int32_t)j;
}

template <typename R, bool Coherent, int Mode = kGeneral>
__device__ __forceinline__ void exchange_sum_h(const KArgs<R> &a, R hx, R hy, R hz, const R *X, const R *Y,
                                               const R *Z, int64_t i, R &e0, R &e1, R &e2);

// The exchange sum of a row stored as a row pattern (NS slots: kShortRow or kPatRow): the
// pattern's offsets and length come as vector loads, every slot is summed, and the slots past
// the row's end carry the spin's own index and J = 0, adding exact zeros after the row's CSR
// terms (so the sum is the CSR sum).
template <typename R, bool Coherent, int NS>
__device__ __forceinline__ void pattern_sum(const KArgs<R> &a, const R *X, const R *Y, const R *Z, int64_t i, R &x,
                                            R &y, R &z) {
    constexpr int W = NS == kShortRow ? 8 : 16;
    const int p = a.pat_wide ? (int)__ldg(reinterpret_cast<const uint16_t *>(a.pat) + i) : (int)__ldg(a.pat + i);
    int32_t off[W];
    const int4 *row = reinterpret_cast<const int4 *>(a.pat_off) + (int64_t)p * (W / 4);
#pragma unroll
    for (int v = 0; v < W / 4; ++v) {
        const int4 t = __ldg(row + v);
        off[4 * v] = t.x;
        off[4 * v + 1] = t.y;
        off[4 * v + 2] = t.z;
        off[4 * v + 3] = t.w;
    }
    const int len = off[NS];
    R Jr[NS];
    if (a.J_uniform) {
#pragma unroll
        for (int q = 0; q < NS; ++q) Jr[q] = q < len ? a.J_value : (R)0;
    } else {
#pragma unroll
        for (int q = 0; q < NS; ++q) Jr[q] = __ldg(a.pat_J + (int64_t)p * W + q);
    }
    const int32_t ii = (int32_t)i;
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        const int32_t j = chk((int64_t)ii + off[q], a.n, a.err);
        x = fma(Jr[q], ld<Coherent>(X + j), x);
        y = fma(Jr[q], ld<Coherent>(Y + j), y);
        z = fma(Jr[q], ld<Coherent>(Z + j), z);
    }
}

template <typename R, bool Coherent, int Mode = kGeneral>
__device__ __forceinline__ void exchange_sum(const KArgs<R> &a, const SysDesc &sd, const R *X, const R *Y,
                                             const R *Z, int64_t i, R &e0, R &e1, R &e2) {
    exchange_sum_h<R, Coherent, Mode>(a, sys_H(sd, 0, R()), sys_H(sd, 1, R()), sys_H(sd, 2, R()), X, Y, Z, i, e0,
                                      e1, e2);
}

// The exchange sum of a row of tensor bonds stored as a row pattern: the form's offsets, length
// and tensor entries come as vector loads, and the row's bonds (the slots before its length)
// are summed as the CSR loop sums them, the tensor of bond k applied to S_j.
template <typename R, bool Coherent, int NS>
__device__ __forceinline__ void pattern_sum_tensor(const KArgs<R> &a, const R *X, const R *Y, const R *Z, int64_t i,
                                                   R &x, R &y, R &z) {
    constexpr int W = NS == kShortRow ? 8 : 16;
    const int p = a.pat_wide ? (int)__ldg(reinterpret_cast<const uint16_t *>(a.pat) + i) : (int)__ldg(a.pat + i);
    int32_t off[W], tid[W];
    const int4 *row = reinterpret_cast<const int4 *>(a.pat_off) + (int64_t)p * (W / 4);
    // the form's Jt entries: W int32 at the start of its W * sizeof(R) bytes of pat_J
    const int4 *trow = reinterpret_cast<const int4 *>(a.pat_J) + (int64_t)p * (W / 4) * ((int)sizeof(R) / 4);
#pragma unroll
    for (int v = 0; v < W / 4; ++v) {
        const int4 t = __ldg(row + v), u = __ldg(trow + v);
        off[4 * v] = t.x;
        off[4 * v + 1] = t.y;
        off[4 * v + 2] = t.z;
        off[4 * v + 3] = t.w;
        tid[4 * v] = u.x;
        tid[4 * v + 1] = u.y;
        tid[4 * v + 2] = u.z;
        tid[4 * v + 3] = u.w;
    }
    const int len = off[NS];
    const int32_t ii = (int32_t)i;
#pragma unroll
    for (int q = 0; q < NS; ++q) {
        if (q < len) {
            const int32_t j = chk((int64_t)ii + off[q], a.n, a.err);
            const R *t = a.Jt + 9 * (int64_t)tid[q];
            const R sx = ld<Coherent>(X + j), sy = ld<Coherent>(Y + j), sz = ld<Coherent>(Z + j);
            x = fma(__ldg(t + 0), sx, fma(__ldg(t + 1), sy, fma(__ldg(t + 2), sz, x)));
            y = fma(__ldg(t + 3), sx, fma(__ldg(t + 4), sy, fma(__ldg(t + 5), sz, y)));
            z = fma(__ldg(t + 6), sx, fma(__ldg(t + 7), sy, fma(__ldg(t + 8), sz, z)));
        }
    }
}

// The sum started at the system's applied field (hx, hy, hz), passed in by callers that hold
// it in registers for a whole tile.
template <typename R, bool Coherent, int Mode>
__device__ __forceinline__ void exchange_sum_h(const KArgs<R> &a, R hx, R hy, R hz, const R *X, const R *Y,
                                               const R *Z, int64_t i, R &e0, R &e1, R &e2) {
    if constexpr (Mode == kRows) {  // long rows: summed beforehand by k_rows_sell / k_rows_field
        e0 = ld<Coherent>(a.ex + i);
        e1 = ld<Coherent>(a.ey + i);
        e2 = ld<Coherent>(a.ez + i);
        return;
    }
    R x = hx, y = hy, z = hz;
    if (a.pat && !(Mode == kGeneral && a.J_tensor)) {
        if (a.pat_w == 8)
            pattern_sum<R, Coherent, kShortRow>(a, X, Y, Z, i, x, y, z);
        else
            pattern_sum<R, Coherent, kPatRow>(a, X, Y, Z, i, x, y, z);
        e0 = x;
        e1 = y;
        e2 = z;
        return;
    }
    if (Mode == kGeneral && a.J_tensor && a.pat) {
        if (a.pat_w == 8)
            pattern_sum_tensor<R, Coherent, kShortRow>(a, X, Y, Z, i, x, y, z);
        else
            pattern_sum_tensor<R, Coherent, kPatRow>(a, X, Y, Z, i, x, y, z);
        e0 = x;
        e1 = y;
        e2 = z;
        return;
    }
    const int32_t b = __ldg(a.row_ptr + i);
    const int32_t e = __ldg(a.row_ptr + i + 1);
    if (Mode == kGeneral && a.J_tensor) {  // Eq. HJijSMS: the tensor of bond k applied to S_j
        for (int32_t k = b; k < e; ++k) {
            const int32_t j = chk(__ldg(a.col + k), a.n, a.err);
            const R *t = a.Jt + 9 * (int64_t)__ldg(a.Jtidx + k);
            const R sx = ld<Coherent>(X + j), sy = ld<Coherent>(Y + j), sz = ld<Coherent>(Z + j);
            x = fma(__ldg(t + 0), sx, fma(__ldg(t + 1), sy, fma(__ldg(t + 2), sz, x)));
            y = fma(__ldg(t + 3), sx, fma(__ldg(t + 4), sy, fma(__ldg(t + 5), sz, y)));
            z = fma(__ldg(t + 6), sx, fma(__ldg(t + 7), sy, fma(__ldg(t + 8), sz, z)));
        }
        e0 = x;
        e1 = y;
        e2 = z;
        return;
    }
    if (a.short_rows) {  // at most kShortRow bonds: unrolled, so the row's loads issue together
#pragma unroll
        for (int q = 0; q < kShortRow; ++q) {
            if (b + q < e) {
                const int32_t j = chk(__ldg(a.col + b + q), a.n, a.err);
                const R Jk = a.J_uniform ? a.J_value : __ldg(a.J + b + q);
                x = fma(Jk, ld<Coherent>(X + j), x);
                y = fma(Jk, ld<Coherent>(Y + j), y);
                z = fma(Jk, ld<Coherent>(Z + j), z);
            }
        }
    } else {
        for (int32_t k = b; k < e; ++k) {
            const int32_t j = chk(__ldg(a.col + k), a.n, a.err);
            const R Jk = a.J_uniform ? a.J_value : __ldg(a.J + k);
            x = fma(Jk, ld<Coherent>(X + j), x);
            y = fma(Jk, ld<Coherent>(Y + j), y);
            z = fma(Jk, ld<Coherent>(Z + j), z);
        }
    }
    e0 = x;
    e1 = y;
    e2 = z;
}

// Deterministic field (tesla): the exchange + applied field h from exchange_sum, then
// the anisotropy and Neel terms.  Returns S.e for the anisotropy energy.  Here and in llg_rhs
// and spin_terms_r every product and sum is spelled out (fma, products rounded on their own),
// so that no kernel variant that inlines them contracts them differently: the step kernels'
// variants (split or fused, any launch mode) give bitwise the same states and records.
template <typename R, bool Cubic = true>
__device__ __forceinline__ R det_field(const MatDesc<R> &m, R s0, R s1, R s2, R e0, R e1, R e2, R &H0, R &H1,
                                       R &H2) {
    const R sde = fma(s2, m.e[2], fma(s1, m.e[1], mul_rn(s0, m.e[0])));
    const R an = mul_rn(m.ani, sde);
    H0 = fma(an, m.e[0], e0);
    H1 = fma(an, m.e[1], e1);
    H2 = fma(an, m.e[2], e2);
    if (Cubic && m.has_cubic) {  // -(2 k_c / mu_s) S^3
        H0 = fma(mul_rn(mul_rn(m.kcf, s0), s0), s0, H0);
        H1 = fma(mul_rn(mul_rn(m.kcf, s1), s1), s1, H1);
        H2 = fma(mul_rn(mul_rn(m.kcf, s2), s2), s2, H2);
    }
    if (m.has_neel) {
        H0 = H0 + fma(m.kf[4], s2, fma(m.kf[3], s1, mul_rn(m.kf[0], s0)));
        H1 = H1 + fma(m.kf[5], s2, fma(m.kf[1], s1, mul_rn(m.kf[3], s0)));
        H2 = H2 + fma(m.kf[2], s2, fma(m.kf[5], s1, mul_rn(m.kf[4], s0)));
    }
    return sde;
}

// The macrocell demagnetising field of spin i's cell, added to its field (Eq. demag; the
// field is held between updates, so it is read like a parameter).
template <typename R>
__device__ __forceinline__ void add_demag(const KArgs<R> &a, int64_t i, R &H0, R &H1, R &H2) {
    const int32_t c = chk(__ldg(a.mc_of + i), a.ncell, a.err);
    H0 += __ldg(a.hdx + c);
    H1 += __ldg(a.hdy + c);
    H2 += __ldg(a.hdz + c);
}

// dS = -gamma/(1+lambda^2) [S x H + lambda S x (S x H)]  (Eq. LLG)
template <typename R>
__device__ __forceinline__ void llg_rhs(R gp, R lam, R s0, R s1, R s2, R H0, R H1, R H2, R &d0, R &d1, R &d2) {
    const R c0 = fma(s1, H2, -mul_rn(s2, H1));
    const R c1 = fma(s2, H0, -mul_rn(s0, H2));
    const R c2 = fma(s0, H1, -mul_rn(s1, H0));
    const R x0 = fma(s1, c2, -mul_rn(s2, c1));
    const R x1 = fma(s2, c0, -mul_rn(s0, c2));
    const R x2 = fma(s0, c1, -mul_rn(s1, c0));
    d0 = mul_rn(-gp, fma(lam, x0, c0));
    d1 = mul_rn(-gp, fma(lam, x1, c1));
    d2 = mul_rn(-gp, fma(lam, x2, c2));
}

// Per-spin contributions to the reductions of the state S: mu S (3), -mu S.h/2 with h the
// exchange + applied field, and the anisotropy energy.  The applied-field energy is
// -H.M (H is uniform within a system) and the exchange energy sum(-mu S.h/2) + H.M/2;
// both are formed from the FP64 sums when a system's record is finalised.
// -mu S.h/2 of one spin (h: exchange + applied field).
template <typename R>
__device__ __forceinline__ R exchange_term(const MatDesc<R> &m, R s0, R s1, R s2, R e0, R e1, R e2) {
    return mul_rn((R)-0.5 * m.mu, fma(s2, e2, fma(s1, e1, mul_rn(s0, e0))));
}

// The anisotropy energy of one spin (uniaxial from S.e, cubic, Neel).
template <typename R, bool Cubic = true>
__device__ __forceinline__ R anisotropy_term(const MatDesc<R> &m, R s0, R s1, R s2, R sde) {
    R ea = mul_rn(-m.ku, mul_rn(sde, sde));
    if (Cubic && m.has_cubic) {
        const R x2 = mul_rn(s0, s0), y2 = mul_rn(s1, s1), z2 = mul_rn(s2, s2);
        ea = fma((R)0.5 * m.kc, fma(z2, z2, fma(y2, y2, mul_rn(x2, x2))), ea);
    }
    if (m.has_neel) {
        const R d = fma(mul_rn(m.K[2], s2), s2, fma(mul_rn(m.K[1], s1), s1, mul_rn(mul_rn(m.K[0], s0), s0)));
        const R o = fma(mul_rn(m.K[5], s1), s2, fma(mul_rn(m.K[4], s0), s2, mul_rn(mul_rn(m.K[3], s0), s1)));
        ea = ea - fma((R)2, o, d);
    }
    return ea;
}

template <typename R, bool Cubic = true>
__device__ __forceinline__ void spin_terms_r(const MatDesc<R> &m, R s0, R s1, R s2, R e0, R e1, R e2, R sde,
                                             R v[5]) {
    const R mu = m.mu;
    v[0] = mul_rn(mu, s0);
    v[1] = mul_rn(mu, s1);
    v[2] = mul_rn(mu, s2);
    v[3] = exchange_term(m, s0, s1, s2, e0, e1, e2);
    v[4] = anisotropy_term<R, Cubic>(m, s0, s1, s2, sde);
}

template <typename R, bool Cubic = true>
__device__ __forceinline__ void spin_terms(const MatDesc<R> &m, R s0, R s1, R s2, R e0, R e1, R e2, R sde,
                                           double v[5]) {
    R t[5];
    spin_terms_r<R, Cubic>(m, s0, s1, s2, e0, e1, e2, sde, t);
#pragma unroll
    for (int c = 0; c < 5; ++c) v[c] = widen(t[c]);
}

// A thread's sums of the five record terms over its spins of a tile.  FP64 form: FP64 sums.
// FP32-mixed form: each float term is added by TwoSum, the running sum hi keeping the float
// sum and lo the sum of TwoSum's exact rounding errors, so that hi + lo is the exact sum up
// to lo's own rounding (a relative 2^-48 of the sum); hi and lo are widened to FP64 once per
// tile, and every later stage sums in FP64.  The FP64 pipe then runs no per-spin work.
template <typename R>
struct TermAcc;

template <>
struct TermAcc<double> {
    double s[5];
    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int c = 0; c < 5; ++c) s[c] = 0.0;
    }
    __device__ __forceinline__ void add(const double v[5]) {
#pragma unroll
        for (int c = 0; c < 5; ++c) s[c] += v[c];
    }
    __device__ __forceinline__ void out(double (&acc)[8]) const {
#pragma unroll
        for (int c = 0; c < 5; ++c) acc[c] = s[c];
        acc[5] = acc[6] = acc[7] = 0.0;
    }
};

template <>
struct TermAcc<float> {
    float h[5], l[5];
    __device__ __forceinline__ void reset() {
#pragma unroll
        for (int c = 0; c < 5; ++c) h[c] = l[c] = 0.0f;
    }
    __device__ __forceinline__ void add(const float v[5]) {
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            const FF t = ff_two_sum(h[c], v[c]);
            h[c] = t.hi;
            l[c] = __fadd_rn(l[c], t.lo);
        }
    }
    __device__ __forceinline__ void out(double (&acc)[8]) const {
        // once per tile; the floats widened from their bits (integer instructions, exact for the
        // normal floats these sums hold) rather than by conversions on the FP64 pipe
#pragma unroll
        for (int c = 0; c < 5; ++c) acc[c] = f2d_bits(h[c]) + f2d_bits(l[c]);
        acc[5] = acc[6] = acc[7] = 0.0;
    }
};

// Sum of eight FP64 values over a warp by a transposing butterfly: 9 additions per lane
// instead of 40.  Afterwards lane L holds component ((L>>4)&1)*4 + ((L>>3)&1)*2 + ((L>>2)&1).
__device__ __forceinline__ double warp_sum8(const double v[8]) {
    const int lane = threadIdx.x & 31;
    double w4[4], w2[2];
    const bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double send = u16 ? v[k] : v[k + 4];
        const double keep = u16 ? v[k + 4] : v[k];
        w4[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const double send = u8 ? w4[k] : w4[k + 2];
        const double keep = u8 ? w4[k + 2] : w4[k];
        w2[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    double x;
    {
        const double send = u4 ? w2[0] : w2[1];
        const double keep = u4 ? w2[1] : w2[0];
        x = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    x += __shfl_xor_sync(0xffffffffu, x, 2);
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    return x;
}

__device__ __forceinline__ int warp_sum8_component(int lane) {
    return ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
}

// Block sum of eight FP64 values in a fixed order; the result is valid in thread 0..7
// (component = thread index) after the call.  red must hold (BS/32)*8 doubles.
template <int BS>
__device__ __forceinline__ double block_sum8(const double v[8], double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double x = warp_sum8(v);
    if ((lane & 3) == 0) red[warp * 8 + warp_sum8_component(lane)] = x;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 8) {
#pragma unroll 4
        for (int w = 0; w < BS / 32; ++w) r += red[w * 8 + threadIdx.x];
    }
    __syncthreads();
    return r;
}

// sqrt(T) of a step in the working type: the schedule entry when a schedule is set.
template <typename R>
__device__ __forceinline__ R sqrtT_of_step(const KArgs<R> &a, uint64_t step, const SysDesc &sd) {
    const bool f32 = sizeof(R) == 4;
    if (a.sched_len <= 0) return f32 ? (R)sd.sqrtTf : (R)sd.sqrtT;
    int64_t k = (int64_t)step - a.sched_step0;
    k = k < 0 ? 0 : (k >= a.sched_len ? a.sched_len - 1 : k);
    return f32 ? (R)a.sqrtT_sched_f[k] : (R)a.sqrtT_sched[k];
}

// Tiles whose per-warp partial sums a block keeps in shared memory between two barriers.
constexpr int kTileChunk = 8;

// The warp's sums of eight per-thread values go to red[(q * warps + warp) * 8 + component]
// (tile slot q of the block's current chunk).
template <int BS>
__device__ __forceinline__ void warp_partials(const double v[8], double *red, int q) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double x = warp_sum8(v);
    if ((lane & 3) == 0) red[(q * (BS / 32) + warp) * 8 + warp_sum8_component(lane)] = x;
}

// After a barrier: the partial of chunk slot q is the sum of its warps' entries in warp
// order (the order of block_sum8), written for tile t0 + q * stride.
template <int BS>
__device__ __forceinline__ void flush_partials(const double *red, int nq, double *partials, int64_t t0,
                                               int64_t stride) {
    for (int idx = threadIdx.x; idx < nq * 8; idx += BS) {  // (blocks of fewer than 64 threads loop)
        const int q = idx >> 3, c = idx & 7;
        double r = 0.0;
#pragma unroll 4
        for (int w = 0; w < BS / 32; ++w) r += red[(q * (BS / 32) + w) * 8 + c];
        partials[(t0 + q * stride) * kPartComps + c] = r;
    }
}

// Predictor over one tile.  Writes S', Q and H_th; acc receives this thread's sums of the
// per-spin reduction terms.  Split: the step's Gaussians were written beforehand by k_gauss
// (every spin reads them, nothing is drawn here) and H_th is not stored (the corrector forms
// the same product again).
template <typename R, int BS, bool Coherent, int Mode = kGeneral, bool Split = false>
__device__ __forceinline__ void predictor_tile(const KArgs<R> &a, const TileDesc &td, uint64_t step,
                                               const StepTabT<R> *tab, int pre_slot, double (&acc)[8],
                                               const R *Gx, const R *Gy, const R *Gz) {
    constexpr int BM = base_mode(Mode);
    const SysDesc &sd = a.sys[td.sys];
    const R sqrtT = sqrtT_of_step(a, step, sd);
    const uint32_t key0 = sd.key0, key1 = sd.key1, ctr2 = sd.ctr2;
    const int64_t off = sd.offset - sd.pbase;  // Philox spin index i - off
    const R ha0 = sys_H(sd, 0, R()), ha1 = sys_H(sd, 1, R()), ha2 = sys_H(sd, 2, R());
    TermAcc<R> ta;
    ta.reset();
    // The slot index is rotated by the warp index, so that the warps of a block reach their
    // transform-heavy slots (the Gaussians not drawn ahead) at different times.
    int rot = (threadIdx.x >> 5) % a.slots;
    for (int k = threadIdx.x; k < td.count; k += BS, rot = rot + 1 == a.slots ? 0 : rot + 1) {
        const int64_t i = td.start + k;
        const MatDesc<R> &m = mat_at<Mode>(a, i);
        const R s0 = ld<Coherent>(a.sx + i), s1 = ld<Coherent>(a.sy + i), s2 = ld<Coherent>(a.sz + i);
        R e0, e1, e2;
        exchange_sum_h<R, Coherent, BM>(a, ha0, ha1, ha2, a.sx, a.sy, a.sz, i, e0, e1, e2);
        R H0, H1, H2;
        const R sde = det_field<R, BM != kPlain>(m, s0, s1, s2, e0, e1, e2, H0, H1, H2);
        if (a.demag) add_demag(a, i, H0, H1, H2);
        R t0 = 0, t1 = 0, t2 = 0;
        if (sqrtT > (R)0) {
            const R sig = m.sig * sqrtT;
            if (Split || rot >= pre_slot) {  // drawn beforehand (k_gauss, or the previous corrector)
                t0 = mul_rn(sig, ld<Coherent>(Gx + i));
                t1 = mul_rn(sig, ld<Coherent>(Gy + i));
                t2 = mul_rn(sig, ld<Coherent>(Gz + i));
            } else if constexpr (!Split) {
                const Philox4 w = philox4x32_10((uint32_t)(i - off), (uint32_t)step, ctr2, 0u, key0, key1);
                R g0, g1, g2;
                thermal_gaussians(a, *tab, w, g0, g1, g2);
                t0 = mul_rn(sig, g0);
                t1 = mul_rn(sig, g1);
                t2 = mul_rn(sig, g2);
            }
        }
        if constexpr (!Split) {
            a.hx[i] = t0;
            a.hy[i] = t1;
            a.hz[i] = t2;
        }
        H0 += t0;
        H1 += t1;
        H2 += t2;
        R d0, d1, d2;
        llg_rhs(m.gp, m.lambda, s0, s1, s2, H0, H1, H2, d0, d1, d2);
        const R dt = m.dt;
        const R v0 = fma(dt, d0, s0), v1 = fma(dt, d1, s1), v2 = fma(dt, d2, s2);
        const R inv = rsqrt_r(fma(v2, v2, fma(v1, v1, mul_rn(v0, v0))));
        a.px[i] = mul_rn(v0, inv);
        a.py[i] = mul_rn(v1, inv);
        a.pz[i] = mul_rn(v2, inv);
        const R hdt = (R)0.5 * dt;
        a.qx[i] = fma(hdt, d0, s0);
        a.qy[i] = fma(hdt, d1, s1);
        a.qz[i] = fma(hdt, d2, s2);
        if constexpr (sizeof(R) == 4) {
            R v[5];
            spin_terms_r<R, BM != kPlain>(m, s0, s1, s2, e0, e1, e2, sde, v);
            ta.add(v);
        } else {
            double v[5];
            spin_terms<R, BM != kPlain>(m, s0, s1, s2, e0, e1, e2, sde, v);
            ta.add(v);
        }
    }
    ta.out(acc);
}

template <typename R, int BS, bool Coherent, int Mode = kGeneral, bool Split = false>
__device__ __forceinline__ void corrector_tile(const KArgs<R> &a, const TileDesc &td, uint64_t step,
                                               const StepTabT<R> *tab, const R *Gx = nullptr,
                                               const R *Gy = nullptr, const R *Gz = nullptr) {
    constexpr int BM = base_mode(Mode);
    const SysDesc &sd = a.sys[td.sys];
    const R sqrtT = Split ? sqrtT_of_step(a, step, sd) : (R)0;  // the thermal field from the Gaussians
    // Gaussians of step + 1 for the slots the next predictor will not draw (FP32-mixed):
    // this puts transform work next to the corrector's memory traffic.
    const R sqrtT_next = tab ? sqrtT_of_step(a, step + 1, sd) : (R)0;
    const uint32_t key0 = sd.key0, key1 = sd.key1, ctr2 = sd.ctr2;
    const int64_t off = sd.offset - sd.pbase;  // Philox spin index i - off
    const R ha0 = sys_H(sd, 0, R()), ha1 = sys_H(sd, 1, R()), ha2 = sys_H(sd, 2, R());
    int rot = (threadIdx.x >> 5) % a.slots;  // the predictor's rotated slot index
    for (int k = threadIdx.x; k < td.count; k += BS, rot = rot + 1 == a.slots ? 0 : rot + 1) {
        const int64_t i = td.start + k;
        const MatDesc<R> &m = mat_at<Mode>(a, i);
        const R s0 = ld<Coherent>(a.px + i), s1 = ld<Coherent>(a.py + i), s2 = ld<Coherent>(a.pz + i);
        R e0, e1, e2;
        exchange_sum_h<R, Coherent, BM>(a, ha0, ha1, ha2, a.px, a.py, a.pz, i, e0, e1, e2);
        R H0, H1, H2;
        det_field<R, BM != kPlain>(m, s0, s1, s2, e0, e1, e2, H0, H1, H2);
        if (a.demag) add_demag(a, i, H0, H1, H2);
        if constexpr (Split) {  // the predictor's H_th, formed the same way
            if (sqrtT > (R)0) {
                const R sig = m.sig * sqrtT;
                H0 += mul_rn(sig, ld<Coherent>(Gx + i));
                H1 += mul_rn(sig, ld<Coherent>(Gy + i));
                H2 += mul_rn(sig, ld<Coherent>(Gz + i));
            }
        } else {
            H0 += ld<Coherent>(a.hx + i);
            H1 += ld<Coherent>(a.hy + i);
            H2 += ld<Coherent>(a.hz + i);
        }
        R d0, d1, d2;
        llg_rhs(m.gp, m.lambda, s0, s1, s2, H0, H1, H2, d0, d1, d2);
        const R hdt = (R)0.5 * m.dt;
        const R v0 = fma(hdt, d0, ld<Coherent>(a.qx + i));
        const R v1 = fma(hdt, d1, ld<Coherent>(a.qy + i));
        const R v2 = fma(hdt, d2, ld<Coherent>(a.qz + i));
        const R inv = rsqrt_r(fma(v2, v2, fma(v1, v1, mul_rn(v0, v0))));
        if (bad_inv(inv)) atomicOr(a.err, kErrNonFinite);  // NaN or infinite length
        a.sx[i] = mul_rn(v0, inv);
        a.sy[i] = mul_rn(v1, inv);
        a.sz[i] = mul_rn(v2, inv);
        if (!Split && rot >= a.pre_slot && sqrtT_next > (R)0) {
            const Philox4 w = philox4x32_10((uint32_t)(i - off), (uint32_t)(step + 1), ctr2, 0u, key0, key1);
            R g0, g1, g2;
            thermal_gaussians(a, *tab, w, g0, g1, g2);
            a.gx[i] = g0;
            a.gy[i] = g1;
            a.gz[i] = g2;
        }
    }
}

// One record (8 doubles) from the block sums of the per-spin terms (valid in threads 0..7
// on entry): sum mu S (3), sum mu, E_exc = sum(-mu S.h/2) + H.M/2, E_ani, E_app = -H.M,
// E_total.  Called by every thread of the block.
__device__ __forceinline__ void write_record(const SysDesc &sd, double r, double *dst) {
    __shared__ double comp[8];
    if (threadIdx.x < 8) comp[threadIdx.x] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        const double *H = sd.H;
        const double hm = (H[0] * comp[0] + H[1] * comp[1]) + H[2] * comp[2];  // H.M
        const double e_app = -hm;
        const double e_exc = comp[3] + 0.5 * hm;
        dst[0] = comp[0];
        dst[1] = comp[1];
        dst[2] = comp[2];
        dst[3] = sd.msum;
        dst[4] = e_exc;
        dst[5] = comp[4];
        dst[6] = e_app;
        dst[7] = (e_exc + comp[4]) + e_app;
    }
    __syncthreads();
}

// Sum the tile partials of system s in tile order and write one record (8 doubles).
template <int BS, bool Coherent, bool Chains4 = false>
__device__ __forceinline__ void finalize_system(const SysDesc *sys, const int32_t *sys_tiles, const double *partials,
                                                int s, double *dst, double *red) {
    const int32_t t0 = sys_tiles[s], t1 = sys_tiles[s + 1];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if constexpr (Chains4) {
        // four independent chains per thread (tiles t, t + BS, t + 2 BS, t + 3 BS of each
        // round), joined in a fixed order: deterministic, and the loads overlap (the
        // stand-alone finalisation kernels; inside the step kernels the registers cost more)
        double a4[4][5] = {};
        for (int32_t t = t0 + threadIdx.x; t < t1; t += 4 * BS) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int32_t u = t + q * BS;
                if (u < t1) {
#pragma unroll
                    for (int c = 0; c < 5; ++c) a4[q][c] += ld<Coherent>(partials + (int64_t)u * kPartComps + c);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 5; ++c) acc[c] = (a4[0][c] + a4[1][c]) + (a4[2][c] + a4[3][c]);
    } else {
        for (int32_t t = t0 + threadIdx.x; t < t1; t += BS) {
#pragma unroll
            for (int c = 0; c < 5; ++c) acc[c] += ld<Coherent>(partials + (int64_t)t * kPartComps + c);
        }
    }
    const double r = block_sum8<BS>(acc, red);
    write_record(sys[s], r, dst);
}

// ----------------------------------------------------------------------------------
// Kernels
// ----------------------------------------------------------------------------------

// Predictor passes over the block's tiles t = blockIdx.x + j gridDim.x, in chunks of
// kTileChunk tiles whose partials are summed after one barrier.
template <typename R, int BS, bool Coherent, int Mode = kGeneral, bool Split = false>
__device__ __forceinline__ void predictor_pass(const KArgs<R> &a, uint64_t step, const StepTabT<R> *tab,
                                               int pre_slot, double *red, const R *Gx, const R *Gy,
                                               const R *Gz) {
    const int64_t stride = gridDim.x;
    for (int64_t t0 = blockIdx.x; t0 < a.ntiles; t0 += (int64_t)kTileChunk * stride) {
        int nq = 0;
        for (; nq < kTileChunk; ++nq) {
            const int64_t t = t0 + nq * stride;
            if (t >= a.ntiles) break;
            double acc[8];
            predictor_tile<R, BS, Coherent, Mode, Split>(a, a.tiles[t], step, tab, pre_slot, acc, Gx, Gy, Gz);
            warp_partials<BS>(acc, red, nq);
        }
        __syncthreads();
        flush_partials<BS>(red, nq, a.partials, t0, stride);
        __syncthreads();
    }
}

// FP64: one resident block per SM is enough for the FP64 pipe, and the minimum-blocks bound
// lets the compiler keep the transform in registers (without it the FP64 form spills at 64).
template <typename R, int BS, int Mode = kGeneral>
#ifndef SS_PRED_WARPS
#define SS_PRED_WARPS 32
#endif
#ifndef SS_CORR_WARPS
#define SS_CORR_WARPS 32
#endif
__global__ void __launch_bounds__(BS, sizeof(R) == 8 ? 1 : SS_PRED_WARPS * 32 / BS) k_predictor(const KArgs<R> a) {
    __shared__ StepTabT<R> tab;
    __shared__ double red[kTileChunk * (BS / 32) * 8];
    stage_step_tables(a, tab);
    __syncthreads();
    const uint64_t step = *a.step;
    // Gaussians drawn ahead are valid only if the previous corrector ran for this step.
    const int pre_slot = (a.g_step != nullptr && *a.g_step == step) ? a.pre_slot : 1 << 30;
    predictor_pass<R, BS, false, Mode>(a, step, &tab, pre_slot, red, a.gx, a.gy, a.gz);
}

// Blocks [0, nfin) sum the predictor's tile partials into the record ring; the rest run
// the corrector over the tiles.  The last block to finish advances the step counter.
template <typename R, int BS, bool DrawAhead, int Mode = kGeneral>
__global__ void __launch_bounds__(BS, sizeof(R) == 8 ? 0 : SS_CORR_WARPS * 32 / BS) k_corrector(const KArgs<R> a, int nfin) {
    __shared__ double red[(BS / 32) * 8];
    const uint64_t step = *a.step;
    if ((int)blockIdx.x < nfin) {
        for (int s = blockIdx.x; s < a.nsys; s += nfin) {
            double *dst = a.rec + ((int64_t)(step % (uint64_t)a.rec_cap) * a.nsys + s) * kRecComps;
            finalize_system<BS, false>(a.sys, a.sys_tiles, a.partials, s, dst, red);
        }
    } else if constexpr (DrawAhead) {
        __shared__ StepTabT<R> tab;
        stage_step_tables(a, tab);
        __syncthreads();
        const int64_t nb = gridDim.x - nfin;
        for (int64_t t = blockIdx.x - nfin; t < a.ntiles; t += nb)
            corrector_tile<R, BS, false, Mode>(a, a.tiles[t], step, &tab);
    } else {
        const int64_t nb = gridDim.x - nfin;
        for (int64_t t = blockIdx.x - nfin; t < a.ntiles; t += nb)
            corrector_tile<R, BS, false, Mode>(a, a.tiles[t], step, nullptr);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int done = atomicAdd(a.ticket, 1u);
        if (done == gridDim.x - 1) {
            *a.ticket = 0u;
            if (a.advance) {
                if (DrawAhead) *a.g_step = step + 1ull;
                *a.step = step + 1ull;
            }
            __threadfence();
        }
    }
}

// The split FP32-mixed step: k_gauss writes the step's Gaussians for every spin, then the
// predictor and the corrector read them.  The transform is pure arithmetic and the two Heun
// passes are memory-bound; apart, the passes carry no transform code, hold fewer registers and
// keep more warps in flight.  The Gaussians move 12 bytes per spin out and 24 back per step,
// what the stored thermal field and the drawn-ahead Gaussians of the fused step moved.
template <int BS>
__global__ void __launch_bounds__(BS) k_gauss(const KArgs<float> a) {
    __shared__ FFTables tab;
    stage_ff_tables(a.fftab, tab);
    __syncthreads();
    // The step comes from the Gaussian pass's own counter: the pass may run while the previous
    // step's Heun passes (which advance the step counter) are still running.
    const uint64_t step = *a.gstep;
    float *Gx = (step & 1) ? a.g2x : a.gx, *Gy = (step & 1) ? a.g2y : a.gy, *Gz = (step & 1) ? a.g2z : a.gz;
    // the buffers no longer hold Gaussians drawn ahead by a fused corrector
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.g_step) *a.g_step = ~0ull;
    for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const TileDesc td = a.tiles[t];
        const SysDesc &sd = a.sys[td.sys];
        if (!(sqrtT_of_step(a, step, sd) > 0.0f)) continue;  // no thermal field: nothing reads them
        const uint32_t key0 = sd.key0, key1 = sd.key1, ctr2 = sd.ctr2;
        const int64_t off = sd.offset - sd.pbase;  // Philox spin index i - off
        for (int k = threadIdx.x; k < td.count; k += BS) {
            const int64_t i = td.start + k;
            const Philox4 w = philox4x32_10((uint32_t)(i - off), (uint32_t)step, ctr2, 0u, key0, key1);
            float g0, g1, g2;
            gaussians_f32(w, tab, a.tab, g0, g1, g2);
            Gx[i] = g0;
            Gy[i] = g1;
            Gz[i] = g2;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // the last block to finish moves the counter to the next step
        __threadfence();
        const unsigned int done = atomicAdd(a.gticket, 1u);
        if (done == gridDim.x - 1) {
            *a.gticket = 0u;
            *a.gstep = step + 1ull;
            __threadfence();
        }
    }
}

// Start of a run of split steps: the Gaussian pass's counter joins the step counter.
static __global__ void k_gstep_sync(unsigned long long *gstep, const unsigned long long *step) { *gstep = *step; }

template <typename R, int BS, int Mode = kGeneral>
__global__ void __launch_bounds__(BS) k_predictor_split(const KArgs<R> a) {
    __shared__ double red[kTileChunk * (BS / 32) * 8];
    const uint64_t step = *a.step;
    // (no tables: nothing is drawn in this pass)
    const bool odd = step & 1;
    predictor_pass<R, BS, false, Mode, true>(a, step, nullptr, 0, red, odd ? a.g2x : a.gx, odd ? a.g2y : a.gy,
                                             odd ? a.g2z : a.gz);
}

template <typename R, int BS, int Mode = kGeneral>
__global__ void __launch_bounds__(BS) k_corrector_split(const KArgs<R> a, int nfin) {
    __shared__ double red[(BS / 32) * 8];
    const uint64_t step = *a.step;
    if ((int)blockIdx.x < nfin) {
        for (int s = blockIdx.x; s < a.nsys; s += nfin) {
            double *dst = a.rec + ((int64_t)(step % (uint64_t)a.rec_cap) * a.nsys + s) * kRecComps;
            finalize_system<BS, false>(a.sys, a.sys_tiles, a.partials, s, dst, red);
        }
    } else {
        const int64_t nb = gridDim.x - nfin;
        const bool odd = step & 1;
        for (int64_t t = blockIdx.x - nfin; t < a.ntiles; t += nb)
            corrector_tile<R, BS, false, Mode, true>(a, a.tiles[t], step, nullptr, odd ? a.g2x : a.gx,
                                                     odd ? a.g2y : a.gy, odd ? a.g2z : a.gz);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int done = atomicAdd(a.ticket, 1u);
        if (done == gridDim.x - 1) {
            *a.ticket = 0u;
            *a.step = step + 1ull;
            __threadfence();
        }
    }
}

// Tile partials of the current state (no integration): the on-demand measurement.
template <typename R, int BS>
__global__ void __launch_bounds__(BS) k_measure(const KArgs<R> a) {
    __shared__ double red[(BS / 32) * 8];
    for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const TileDesc td = a.tiles[t];
        const SysDesc &sd = a.sys[td.sys];
        TermAcc<R> ta;  // summed as in the step kernels
        ta.reset();
        for (int k = threadIdx.x; k < td.count; k += BS) {
            const int64_t i = td.start + k;
            const MatDesc<R> &m = a.mats[mat_of(a, i)];
            const R s0 = a.sx[i], s1 = a.sy[i], s2 = a.sz[i];
            R e0, e1, e2;
            if (a.ex)
                exchange_sum<R, false, kRows>(a, sd, a.sx, a.sy, a.sz, i, e0, e1, e2);
            else
                exchange_sum<R, false>(a, sd, a.sx, a.sy, a.sz, i, e0, e1, e2);
            R H0, H1, H2;
            const R sde = det_field(m, s0, s1, s2, e0, e1, e2, H0, H1, H2);
            if constexpr (sizeof(R) == 4) {
                R v[5];
                spin_terms_r(m, s0, s1, s2, e0, e1, e2, sde, v);
                ta.add(v);
            } else {
                double v[5];
                spin_terms(m, s0, s1, s2, e0, e1, e2, sde, v);
                ta.add(v);
            }
        }
        double acc[8];
        ta.out(acc);
        const double r = block_sum8<BS>(acc, red);
        if (threadIdx.x < kPartComps) a.partials[t * kPartComps + threadIdx.x] = r;
    }
}

// As k_finalize, into the record ring's entry of the current device step (so that the
// launch holds no host-side step and can be captured once and replayed).
template <int BS>
__global__ void __launch_bounds__(BS) k_finalize_ring(const SysDesc *sys, const int32_t *sys_tiles, int nsys,
                                                      const double *partials, double *rec, int64_t rec_cap,
                                                      const unsigned long long *step) {
    __shared__ double red[(BS / 32) * 8];
    double *dst = rec + (int64_t)(*step % (unsigned long long)rec_cap) * nsys * kRecComps;
    for (int s = blockIdx.x; s < nsys; s += gridDim.x)
        finalize_system<BS, false, true>(sys, sys_tiles, partials, s, dst + (int64_t)s * kRecComps, red);
}

template <int BS>
__global__ void __launch_bounds__(BS) k_finalize(const SysDesc *sys, const int32_t *sys_tiles, int nsys,
                                                 const double *partials, double *dst) {
    __shared__ double red[(BS / 32) * 8];
    for (int s = blockIdx.x; s < nsys; s += gridDim.x)
        finalize_system<BS, false, true>(sys, sys_tiles, partials, s, dst + (int64_t)s * kRecComps, red);
}

// Random unit spins from the reserved stream: counter (i, 0xFFFFFFFF, system, 1).
template <typename R>
__global__ void k_init_sphere(const KArgs<R> a) {
    __shared__ SmemTables tab;
    stage_tables(a, tab);
    __syncthreads();
    for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const TileDesc td = a.tiles[t];
        const SysDesc &sd = a.sys[td.sys];
        for (int k = threadIdx.x; k < td.count; k += blockDim.x) {
            const int64_t i = td.start + k;
            const Philox4 w =
                philox4x32_10((uint32_t)(i - sd.offset + sd.pbase), 0xFFFFFFFFu, sd.ctr2, 1u, sd.key0, sd.key1);
            double g0, g1, g2;
            box_muller3(w, tab, g0, g1, g2);
            const double inv = 1.0 / sqrt(g0 * g0 + g1 * g1 + g2 * g2);
            a.sx[i] = (R)(g0 * inv);
            a.sy[i] = (R)(g1 * inv);
            a.sz[i] = (R)(g2 * inv);
        }
    }
}

// Bounded grid barrier: waits at most bar_timeout_ns (globaltimer) and then reports a
// timeout instead of hanging.  Returns false on timeout (uniform within the block).
__device__ __forceinline__ bool grid_barrier(unsigned int *count, unsigned int *gen, unsigned int expected,
                                             long long timeout_ns, unsigned int *err) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned int *vgen = gen;
        const unsigned int g = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(count, 1u);
        if (arrived == expected - 1u) {
            *count = 0u;
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            unsigned long long t0;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
            while (*vgen == g) {
                unsigned long long t1;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
                if ((long long)(t1 - t0) > timeout_ns) {
                    atomicOr(err, kErrTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Many steps in one cooperative launch: predictor phase, barrier, corrector phase (with
// the record of the step summed by blocks [0, nfin), and in the FP32-mixed form the back
// half of the next step's Gaussians drawn ahead), barrier.
template <typename R, int BS, int Mode = kGeneral>
__global__ void __launch_bounds__(BS) k_persistent(const KArgs<R> a, int nfin, long long nsteps) {
    __shared__ StepTabT<R> tab;
    __shared__ double red[kTileChunk * (BS / 32) * 8];
    stage_step_tables(a, tab);
    __syncthreads();
    const uint64_t step0 = __ldcg(a.step);
    const bool ahead = a.g_step != nullptr;
    const int pre_first = (ahead && __ldcg(a.g_step) == step0) ? a.pre_slot : 1 << 30;
    const unsigned int expected = gridDim.x + a.bar_extra;
    for (long long k = 0; k < nsteps; ++k) {
        const uint64_t step = step0 + (uint64_t)k;
        const int pre_slot = k == 0 ? pre_first : (ahead ? a.pre_slot : 1 << 30);
        predictor_pass<R, BS, true, Mode>(a, step, &tab, pre_slot, red, a.gx, a.gy, a.gz);
        if (!grid_barrier(a.bar_count, a.bar_gen, expected, a.bar_timeout_ns, a.err)) return;
        if ((int)blockIdx.x < nfin) {
            for (int s = blockIdx.x; s < a.nsys; s += nfin) {
                double *dst = a.rec + ((int64_t)(step % (uint64_t)a.rec_cap) * a.nsys + s) * kRecComps;
                finalize_system<BS, true>(a.sys, a.sys_tiles, a.partials, s, dst, red);
            }
        }
        for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x)
            corrector_tile<R, BS, true, Mode>(a, a.tiles[t], step, ahead ? &tab : nullptr);
        if (!grid_barrier(a.bar_count, a.bar_gen, expected, a.bar_timeout_ns, a.err)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (ahead) *a.g_step = step0 + (uint64_t)nsteps;
        *a.step = step0 + (uint64_t)nsteps;
    }
}

// Whole systems per block: block b advances systems b, b + gridDim.x, ... for nsteps steps
// each, with block barriers between the Heun passes and no grid-wide synchronisation (the
// systems are independent).  Every spin a block reads was written by the same block, after
// a block barrier; loads bypass the non-coherent L1.  Each step's record is summed in the
// block directly.  The last block to finish advances the step counter.
template <typename R, int BS, int Mode = kGeneral>
__global__ void __launch_bounds__(BS) k_system_blocks(const KArgs<R> a, long long nsteps) {
    __shared__ StepTabT<R> tab;
    __shared__ double red[(BS / 32) * 8];
    stage_step_tables(a, tab);
    __syncthreads();
    const uint64_t step0 = __ldcg(a.step);
    for (int s = blockIdx.x; s < a.nsys; s += gridDim.x) {
        const SysDesc &sd = a.sys[s];
        TileDesc whole;
        whole.start = sd.offset;
        whole.count = (int32_t)sd.n;
        whole.sys = s;
        for (long long k = 0; k < nsteps; ++k) {
            const uint64_t step = step0 + (uint64_t)k;
            double acc[8];
            predictor_tile<R, BS, true, Mode>(a, whole, step, &tab, 1 << 30, acc, a.gx, a.gy, a.gz);
            const double r = block_sum8<BS>(acc, red);
            write_record(sd, r, a.rec + ((int64_t)(step % (uint64_t)a.rec_cap) * a.nsys + s) * kRecComps);
            corrector_tile<R, BS, true, Mode>(a, whole, step, nullptr);
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int done = atomicAdd(a.ticket, 1u);
        if (done == gridDim.x - 1) {
            *a.ticket = 0u;
            *a.step = step0 + (uint64_t)nsteps;
            __threadfence();
        }
    }
}

// ----------------------------------------------------------------------------------
// Long exchange rows (hundreds to thousands of neighbours, Eq. HJij): a warp per row.
// The warp takes 32 consecutive rows; for each, its lanes stride over the row's bonds
// (coalesced bond loads), gather the neighbours' spins and sum; a butterfly gives every lane
// the row's total and lane q keeps row q's.  Each lane then writes its row's field
// H_app + sum_j (J_ij / mu_s,i) X_j (coalesced).  Mode 1: col + J (or the uniform J);
// 2: tensors.  (Packed scalar bonds go through k_rows_sell below.)
// ----------------------------------------------------------------------------------
// Packed bonds in slices (the scalar-J case with at most 255 distinct J_ij / mu_s,i): lane l
// of the warp owning slice s sums row 32 s + l, all lanes stepping through bond k together,
// so the bond words load coalesced and the neighbours' spins come as one 16-byte (FP32) or
// 32-byte (FP64) gather from the (x, y, z, 0) copy.  Consecutive rows keep the slice's
// neighbourhood compact (on a lattice numbered cell by cell, a few cells), which is what
// L1 reuse of the gathered spins depends on.  Each row is summed in its CSR order from
// H_app, like the thread-per-row sum (padding adds 0 * S exactly).
template <typename R>
__global__ void k_pack4(const KArgs<R> a, const R *X, const R *Y, const R *Z) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        if constexpr (sizeof(R) == 4) {
            reinterpret_cast<float4 *>(a.x4)[i] = make_float4(X[i], Y[i], Z[i], 0.f);
        } else {
            double2 *d = reinterpret_cast<double2 *>(a.x4) + 2 * i;
            d[0] = make_double2(X[i], Y[i]);
            d[1] = make_double2(Z[i], 0.0);
        }
    }
}

template <typename R>
__device__ __forceinline__ void load_spin4(const R *x4, int32_t j, R &s0, R &s1, R &s2) {
    if constexpr (sizeof(R) == 4) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(x4) + j);
        s0 = v.x;
        s1 = v.y;
        s2 = v.z;
    } else {
        const double2 *d = reinterpret_cast<const double2 *>(x4) + 2 * (int64_t)j;
        const double2 u = __ldg(d), v = __ldg(d + 1);
        s0 = u.x;
        s1 = u.y;
        s2 = v.x;
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_rows_sell(const KArgs<R> a) {
    __shared__ R jd[256];
    for (int t = threadIdx.x; t < a.nJd; t += blockDim.x) jd[t] = a.Jd[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t s = warp; s < a.nslice; s += nwarps) {
        const int64_t row = s * 32 + lane;
        const int64_t o = __ldg(a.sell_off + s);
        const int w = (int)((__ldg(a.sell_off + s + 1) - o) >> 5);
        const uint32_t *p = a.sell + o + lane;
        R x = 0, y = 0, z = 0;
        const SysDesc *sd = nullptr;
        if (row < a.n && !a.rows_bare) {
            sd = &a.sys[a.mats[mat_of(a, row)].sys];
            x = sys_H(*sd, 0, R());
            y = sys_H(*sd, 1, R());
            z = sys_H(*sd, 2, R());
        }
        if constexpr (sizeof(R) == 8) {
            // FP64: eight bonds at a time, their words, then their gathers, then the sums in
            // bond order (5.80 against 6.34 ms per pass on fcc 64^3 to 4a; sixteen at a time
            // gives 5.83 ms; in FP32 the plain loop below is faster, 1.52 against 1.70 ms with
            // eight and 1.99 ms with four)
            constexpr int U = 8;
            int k = 0;
            for (; k + U <= w; k += U) {
                uint32_t bw[U];
#pragma unroll
                for (int u = 0; u < U; ++u) bw[u] = __ldg(p + 32 * (int64_t)(k + u));
                R s0[U], s1[U], s2[U];
#pragma unroll
                for (int u = 0; u < U; ++u) load_spin4(a.x4, chk(bw[u] >> 8, a.n, a.err), s0[u], s1[u], s2[u]);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const R Jk = jd[chk(bw[u] & 255u, a.nJd, a.err)];
                    x = fma(Jk, s0[u], x);
                    y = fma(Jk, s1[u], y);
                    z = fma(Jk, s2[u], z);
                }
            }
            for (; k < w; ++k) {
                const uint32_t b = __ldg(p + 32 * (int64_t)k);
                const R Jk = jd[chk(b & 255u, a.nJd, a.err)];
                R s0, s1, s2;
                load_spin4(a.x4, chk(b >> 8, a.n, a.err), s0, s1, s2);
                x = fma(Jk, s0, x);
                y = fma(Jk, s1, y);
                z = fma(Jk, s2, z);
            }
        } else {
#pragma unroll 8
            for (int k = 0; k < w; ++k) {
                const uint32_t b = __ldg(p + 32 * (int64_t)k);
                const R Jk = jd[chk(b & 255u, a.nJd, a.err)];
                R s0, s1, s2;
                load_spin4(a.x4, chk(b >> 8, a.n, a.err), s0, s1, s2);
                x = fma(Jk, s0, x);
                y = fma(Jk, s1, y);
                z = fma(Jk, s2, z);
            }
        }
        if (row < a.n) {
            a.ex[row] = x;
            a.ey[row] = y;
            a.ez[row] = z;
        }
    }
}

template <typename R, int Mode>
__global__ void __launch_bounds__(256) k_rows_field(const KArgs<R> a, const R *X, const R *Y, const R *Z) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r0 = warp * 32; r0 < a.n; r0 += nwarps * 32) {
        const int64_t row = r0 + lane;
        int32_t rb = 0, re = 0;
        if (row < a.n) {
            rb = __ldg(a.row_ptr + row);
            re = __ldg(a.row_ptr + row + 1);
        }
        const int nr = a.n - r0 < 32 ? (int)(a.n - r0) : 32;
        R mx = 0, my = 0, mz = 0;
        for (int q = 0; q < nr; ++q) {
            const int32_t b = __shfl_sync(FULL, rb, q), e = __shfl_sync(FULL, re, q);
            R x = 0, y = 0, z = 0;
#pragma unroll 4
            for (int32_t k = b + lane; k < e; k += 32) {
                if (Mode == 1) {
                    const int32_t j = chk(__ldg(a.col + k), a.n, a.err);
                    const R Jk = a.J_uniform ? a.J_value : __ldg(a.J + k);
                    x = fma(Jk, X[j], x);
                    y = fma(Jk, Y[j], y);
                    z = fma(Jk, Z[j], z);
                } else {
                    const int32_t j = chk(__ldg(a.col + k), a.n, a.err);
                    const R *t = a.Jt + 9 * (int64_t)__ldg(a.Jtidx + k);
                    const R s0 = X[j], s1 = Y[j], s2 = Z[j];
                    x = fma(__ldg(t + 0), s0, fma(__ldg(t + 1), s1, fma(__ldg(t + 2), s2, x)));
                    y = fma(__ldg(t + 3), s0, fma(__ldg(t + 4), s1, fma(__ldg(t + 5), s2, y)));
                    z = fma(__ldg(t + 6), s0, fma(__ldg(t + 7), s1, fma(__ldg(t + 8), s2, z)));
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                x += __shfl_xor_sync(FULL, x, o);
                y += __shfl_xor_sync(FULL, y, o);
                z += __shfl_xor_sync(FULL, z, o);
            }
            if (lane == q) {
                mx = x;
                my = y;
                mz = z;
            }
        }
        if (row < a.n) {
            if (a.rows_bare) {
                a.ex[row] = mx;
                a.ey[row] = my;
                a.ez[row] = mz;
            } else {
                const SysDesc &sd = a.sys[a.mats[mat_of(a, row)].sys];
                a.ex[row] = sys_H(sd, 0, R()) + mx;
                a.ey[row] = sys_H(sd, 1, R()) + my;
                a.ez[row] = sys_H(sd, 2, R()) + mz;
            }
        }
    }
}

// ----------------------------------------------------------------------------------
// Midpoint rule (the alternative integrator the paper's time-integration section cites):
// S_{n+1} = S_n + dt f(m), m = (S_n + S_{n+1})/2, solved by fixed-point iterations from the
// Euler predictor; the thermal field is drawn once per step (counters as the Heun step) and
// held; nothing is renormalised (f(m) is perpendicular to m).
// ----------------------------------------------------------------------------------

// sum_j (J_ij / mu_s,i) X_j over row i (scalar or tensor bonds, kPlain: scalar only), without
// the applied field; one FMA per bond and component in CSR order.
template <typename R, int Mode>
__device__ __forceinline__ void exchange_bare(const KArgs<R> &a, const R *X, const R *Y, const R *Z, int64_t i,
                                              R &e0, R &e1, R &e2) {
    if constexpr (Mode == kRows) {  // long rows: summed beforehand (without H_app) by the row passes
        e0 = a.ex[i];
        e1 = a.ey[i];
        e2 = a.ez[i];
        return;
    }
    const int32_t b = __ldg(a.row_ptr + i);
    const int32_t e = __ldg(a.row_ptr + i + 1);
    R x = 0, y = 0, z = 0;
    if (Mode != kPlain && a.J_tensor) {
        for (int32_t k = b; k < e; ++k) {
            const int32_t j = chk(__ldg(a.col + k), a.n, a.err);
            const R m0 = X[j], m1 = Y[j], m2 = Z[j];
            const R *t = a.Jt + 9 * (int64_t)__ldg(a.Jtidx + k);
            x = fma(__ldg(t + 0), m0, fma(__ldg(t + 1), m1, fma(__ldg(t + 2), m2, x)));
            y = fma(__ldg(t + 3), m0, fma(__ldg(t + 4), m1, fma(__ldg(t + 5), m2, y)));
            z = fma(__ldg(t + 6), m0, fma(__ldg(t + 7), m1, fma(__ldg(t + 8), m2, z)));
        }
    } else if (a.J_uniform) {
        const R Jk = a.J_value;
        for (int32_t k = b; k < e; ++k) {
            const int32_t j = chk(__ldg(a.col + k), a.n, a.err);
            x = fma(Jk, X[j], x);
            y = fma(Jk, Y[j], y);
            z = fma(Jk, Z[j], z);
        }
    } else {
        for (int32_t k = b; k < e; ++k) {
            const int32_t j = chk(__ldg(a.col + k), a.n, a.err);
            const R Jk = __ldg(a.J + k);
            x = fma(Jk, X[j], x);
            y = fma(Jk, Y[j], y);
            z = fma(Jk, Z[j], z);
        }
    }
    e0 = x;
    e1 = y;
    e2 = z;
}

// ----------------------------------------------------------------------------------
// Semi-implicit predictor-corrector (the modified predictor-corrector midpoint scheme of
// Mentink et al. that the paper's time-integration section cites): with Eq. LLG written as
// dS/dt = S x A(S), A = -gamma/(1+lambda^2) (H + lambda S x H), each half-step solves
// X = S_n + (dt/2)(S_n + X) x A in closed form, a rotation of S_n.  The predictor takes A at
// S_n, the corrector at Sb = (S_n + S')/2; the thermal field is drawn once per step and held.
// ----------------------------------------------------------------------------------

// X = (c - b x c + (b.c) b)/(1 + |b|^2), b = (dt/2) A, c = S + S x b.
template <typename R>
__device__ __forceinline__ void sib_solve(R hdt, R s0, R s1, R s2, R a0, R a1, R a2, R &x0, R &x1, R &x2) {
    const R b0 = hdt * a0, b1 = hdt * a1, b2 = hdt * a2;
    const R c0 = s0 + (s1 * b2 - s2 * b1), c1 = s1 + (s2 * b0 - s0 * b2), c2 = s2 + (s0 * b1 - s1 * b0);
    const R bc = b0 * c0 + b1 * c1 + b2 * c2;
    const R den = (R)1 + (b0 * b0 + b1 * b1 + b2 * b2);
    x0 = (c0 - (b1 * c2 - b2 * c1) + bc * b0) / den;
    x1 = (c1 - (b2 * c0 - b0 * c2) + bc * b1) / den;
    x2 = (c2 - (b0 * c1 - b1 * c0) + bc * b2) / den;
}

// A = -gp (H + lambda v x H).
template <typename R>
__device__ __forceinline__ void sib_a(R gp, R lam, R v0, R v1, R v2, R H0, R H1, R H2, R &a0, R &a1, R &a2) {
    a0 = -gp * fma(lam, v1 * H2 - v2 * H1, H0);
    a1 = -gp * fma(lam, v2 * H0 - v0 * H2, H1);
    a2 = -gp * fma(lam, v0 * H1 - v1 * H0, H2);
}

// Threads per block of the first pass of the alternative integrators.
constexpr int kAltBlock = 256;

// First pass of the alternative integrators, tile by tile: the step's thermal field (counters
// as the Heun step), the part of the second pass's field that is fixed over the step,
// C = H_app + H_th + (1/2) sum_j J_ij S_j (the exchange field is linear, so the field of
// (S + X)/2 is C + (1/2) sum_j J_ij X_j plus the on-site terms), into (hx, hy, hz); the first new
// spin into (px, py, pz): the semi-implicit predictor (Sib) or the Euler predictor of the
// midpoint rule; and the tile partials of the record of S, the state at the start of the step.
template <typename R, int Mode, bool Sib>
__device__ __forceinline__ void alt_first_pass(const KArgs<R> &a, const SmemTables &tab, double *red) {
    const uint64_t step = *a.step;
    for (int64_t t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
        const TileDesc td = a.tiles[t];
        const SysDesc &sd = a.sys[td.sys];
        const R sqrtT = sqrtT_of_step(a, step, sd);
        const R ha0 = sys_H(sd, 0, R()), ha1 = sys_H(sd, 1, R()), ha2 = sys_H(sd, 2, R());
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int k = threadIdx.x; k < td.count; k += kAltBlock) {
            const int64_t i = td.start + k;
            const MatDesc<R> &m = a.mats[mat_of(a, i)];
            R t0 = 0, t1 = 0, t2 = 0;
            if (sqrtT > (R)0) {
                const R sig = m.sig * sqrtT;
                const Philox4 w =
                    philox4x32_10((uint32_t)(i - sd.offset + sd.pbase), (uint32_t)step, sd.ctr2, 0u, sd.key0, sd.key1);
                double g0, g1, g2;
                box_muller3(w, tab, g0, g1, g2);
                t0 = sig * narrow<R>(g0);
                t1 = sig * narrow<R>(g1);
                t2 = sig * narrow<R>(g2);
            }
            const R s0 = a.sx[i], s1 = a.sy[i], s2 = a.sz[i];
            R x0, x1, x2;
            exchange_bare<R, Mode>(a, a.sx, a.sy, a.sz, i, x0, x1, x2);
            const R c0 = ha0 + t0, c1 = ha1 + t1, c2 = ha2 + t2;
            a.hx[i] = fma((R)0.5, x0, c0);
            a.hy[i] = fma((R)0.5, x1, c1);
            a.hz[i] = fma((R)0.5, x2, c2);
            R H0, H1, H2;
            const R sde = det_field<R, Mode != kPlain>(m, s0, s1, s2, x0 + c0, x1 + c1, x2 + c2, H0, H1, H2);
            if (a.demag) add_demag(a, i, H0, H1, H2);
            double v[5];
            spin_terms<R, Mode != kPlain>(m, s0, s1, s2, x0 + ha0, x1 + ha1, x2 + ha2, sde, v);
#pragma unroll
            for (int c = 0; c < 5; ++c) acc[c] += v[c];
            R p0, p1, p2;
            if constexpr (Sib) {
                R a0, a1, a2;
                sib_a(m.gp, m.lambda, s0, s1, s2, H0, H1, H2, a0, a1, a2);
                sib_solve((R)0.5 * m.dt, s0, s1, s2, a0, a1, a2, p0, p1, p2);
            } else {
                R d0, d1, d2;
                llg_rhs(m.gp, m.lambda, s0, s1, s2, H0, H1, H2, d0, d1, d2);
                p0 = fma(m.dt, d0, s0);
                p1 = fma(m.dt, d1, s1);
                p2 = fma(m.dt, d2, s2);
            }
            a.px[i] = p0;
            a.py[i] = p1;
            a.pz[i] = p2;
        }
        const double r = block_sum8<kAltBlock>(acc, red);
        if (threadIdx.x < kPartComps) a.partials[t * kPartComps + threadIdx.x] = r;
    }
}

// Midpoint rule, first pass: the Euler predictor X = S + dt f(S).
template <typename R, int Mode>
__global__ void __launch_bounds__(kAltBlock) k_mid_euler(const KArgs<R> a) {
    __shared__ SmemTables tab;
    __shared__ double red[(kAltBlock / 32) * 8];
    stage_tables(a, tab);
    __syncthreads();
    alt_first_pass<R, Mode, false>(a, tab, red);
}

// One fixed-point iteration: Y = S + dt f(m), m = (S + X)/2, with the field C + (1/2) sum_j J_ij X_j
// plus the on-site terms of m.  A thread reads S only at its own spin, so the last iteration
// writes Y over S (Last: and flags non-finite spins).
template <typename R, int Mode, bool Last>
__global__ void k_mid_iter(const KArgs<R> a, const R *xx, const R *xy, const R *xz, R *yx, R *yy, R *yz) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        const MatDesc<R> &m = a.mats[mat_of(a, i)];
        const R s0 = a.sx[i], s1 = a.sy[i], s2 = a.sz[i];
        const R m0 = (R)0.5 * (s0 + xx[i]), m1 = (R)0.5 * (s1 + xy[i]), m2 = (R)0.5 * (s2 + xz[i]);
        R x0, x1, x2;
        exchange_bare<R, Mode>(a, xx, xy, xz, i, x0, x1, x2);
        R H0, H1, H2;
        det_field<R, Mode != kPlain>(m, m0, m1, m2, fma((R)0.5, x0, a.hx[i]), fma((R)0.5, x1, a.hy[i]),
                                     fma((R)0.5, x2, a.hz[i]), H0, H1, H2);
        if (a.demag) add_demag(a, i, H0, H1, H2);
        R d0, d1, d2;
        llg_rhs(m.gp, m.lambda, m0, m1, m2, H0, H1, H2, d0, d1, d2);
        const R v0 = fma(m.dt, d0, s0), v1 = fma(m.dt, d1, s1), v2 = fma(m.dt, d2, s2);
        if (Last && bad_inv(v0 * v0 + v1 * v1 + v2 * v2)) atomicOr(a.err, kErrNonFinite);
        yx[i] = v0;
        yy[i] = v1;
        yz[i] = v2;
    }
}

// Semi-implicit predictor: S' = S_n + (dt/2)(S_n + S') x A(S_n), with the first-pass outputs above.
template <typename R, int Mode>
__global__ void __launch_bounds__(kAltBlock) k_sib_pred(const KArgs<R> a) {
    __shared__ SmemTables tab;
    __shared__ double red[(kAltBlock / 32) * 8];
    stage_tables(a, tab);
    __syncthreads();
    alt_first_pass<R, Mode, true>(a, tab, red);
}

// Corrector: A at Sb = (S + S')/2 with the field C + (1/2) sum_j J_ij S'_j plus the on-site
// terms of Sb; the new spin overwrites S (a thread reads S only at its own spin).
template <typename R, int Mode>
__global__ void k_sib_corr(const KArgs<R> a) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        const MatDesc<R> &m = a.mats[mat_of(a, i)];
        const R s0 = a.sx[i], s1 = a.sy[i], s2 = a.sz[i];
        const R m0 = (R)0.5 * (s0 + a.px[i]), m1 = (R)0.5 * (s1 + a.py[i]), m2 = (R)0.5 * (s2 + a.pz[i]);
        R x0, x1, x2;
        exchange_bare<R, Mode>(a, a.px, a.py, a.pz, i, x0, x1, x2);
        R H0, H1, H2;
        det_field<R, Mode != kPlain>(m, m0, m1, m2, fma((R)0.5, x0, a.hx[i]), fma((R)0.5, x1, a.hy[i]),
                                     fma((R)0.5, x2, a.hz[i]), H0, H1, H2);
        if (a.demag) add_demag(a, i, H0, H1, H2);
        R a0, a1, a2;
        sib_a(m.gp, m.lambda, m0, m1, m2, H0, H1, H2, a0, a1, a2);
        R v0, v1, v2;
        sib_solve((R)0.5 * m.dt, s0, s1, s2, a0, a1, a2, v0, v1, v2);
        if (bad_inv(v0 * v0 + v1 * v1 + v2 * v2)) atomicOr(a.err, kErrNonFinite);
        a.sx[i] = v0;
        a.sy[i] = v1;
        a.sz[i] = v2;
    }
}

// ----------------------------------------------------------------------------------
// Macrocell demagnetising field (Section "Demagnetising fields")
// ----------------------------------------------------------------------------------

// Moment of every macrocell, m_c = sum_i mu_s,i S_i over its spins (the moment equation):
// one warp per cell, FP64, summed in a fixed order (lane-strided, then a fixed butterfly).
template <typename R>
__global__ void k_demag_moments(const KArgs<R> a, const DemagArgs d) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = warp; c < d.ncell; c += nwarps) {
        double m0 = 0.0, m1 = 0.0, m2 = 0.0;
        for (int32_t k = d.cell_start[c] + lane; k < d.cell_start[c + 1]; k += 32) {
            const int32_t i = d.cell_spins[k];
            const double mu = widen(a.mats[mat_of(a, i)].mu);
            m0 += mu * widen(a.sx[i]);
            m1 += mu * widen(a.sy[i]);
            m2 += mu * widen(a.sz[i]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            m0 += __shfl_xor_sync(0xffffffffu, m0, o);
            m1 += __shfl_xor_sync(0xffffffffu, m1, o);
            m2 += __shfl_xor_sync(0xffffffffu, m2, o);
        }
        if (lane == 0) {
            d.m[3 * c + 0] = m0;
            d.m[3 * c + 1] = m1;
            d.m[3 * c + 2] = m2;
        }
    }
}

// Field of every macrocell p (Eq. demag): mu0/(4 pi) sum over the other cells q of the same
// system of [3 (m_q . u) u - m_q] / r^3, u the unit vector from p to q, minus the self term
// mu0/3 m_p / V_p.  One warp per cell: lane-strided over q, the lane sums in FP64 combined by
// a fixed butterfly.  The separations are formed in FP64; the rest of a pair's arithmetic runs
// in the working type.  Also writes the working-type copy the step kernels read.
template <typename R>
__global__ void k_demag_field(const KArgs<R> a, const DemagArgs d) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = warp; p < d.ncell; p += nwarps) {
        const double px = d.pos[3 * p], py = d.pos[3 * p + 1], pz = d.pos[3 * p + 2];
        double hx = 0.0, hy = 0.0, hz = 0.0;
        for (int32_t q = d.cell_first[p] + lane; q < d.cell_end[p]; q += 32) {
            if (q == p) continue;
            const R rx = narrow_any<R>(d.pos[3 * q] - px), ry = narrow_any<R>(d.pos[3 * q + 1] - py);
            const R rz = narrow_any<R>(d.pos[3 * q + 2] - pz);
            const R rinv = rsqrt_r(rx * rx + ry * ry + rz * rz);
            const R ux = rx * rinv, uy = ry * rinv, uz = rz * rinv;
            const R mx = narrow_any<R>(d.m[3 * q]), my = narrow_any<R>(d.m[3 * q + 1]);
            const R mz = narrow_any<R>(d.m[3 * q + 2]);
            const R mu3 = (R)3 * (mx * ux + my * uy + mz * uz);
            const R r3inv = rinv * rinv * rinv;
            hx += widen((mu3 * ux - mx) * r3inv);
            hy += widen((mu3 * uy - my) * r3inv);
            hz += widen((mu3 * uz - mz) * r3inv);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            hx += __shfl_xor_sync(0xffffffffu, hx, o);
            hy += __shfl_xor_sync(0xffffffffu, hy, o);
            hz += __shfl_xor_sync(0xffffffffu, hz, o);
        }
        if (lane == 0) {
            const double c1 = kMu0 / (4.0 * 3.14159265358979323846), c2 = kMu0 / 3.0 / d.vol[p];
            const double H0 = c1 * hx - c2 * d.m[3 * p], H1 = c1 * hy - c2 * d.m[3 * p + 1];
            const double H2 = c1 * hz - c2 * d.m[3 * p + 2];
            d.H[3 * p] = H0;
            d.H[3 * p + 1] = H1;
            d.H[3 * p + 2] = H2;
            R *hx_ = const_cast<R *>(a.hdx), *hy_ = const_cast<R *>(a.hdy), *hz_ = const_cast<R *>(a.hdz);
            hx_[p] = narrow_any<R>(H0);
            hy_[p] = narrow_any<R>(H1);
            hz_[p] = narrow_any<R>(H2);
        }
    }
}

// ----------------------------------------------------------------------------------
// Monte Carlo (Section "Monte Carlo Methods")
// ----------------------------------------------------------------------------------

// One Hinzke-Nowak trial move (spin flip, Gaussian move Eq. MCgaussian, random move
// Eq. MCrandom, picked with equal odds) for every spin of one colour class, accepted by
// the Metropolis criterion Eq. AMCP as dE <= -kB T ln u.  Per (spin i, step n): Philox
// block (i, n, system, 2) gives the Gaussian triple, block (i, n, system, 3) the move type
// (from the first word, floor(3 w0 / 2^32)) and the acceptance uniform (second word).
// Spins of one colour share no bond, so each trial reads only spins of other colours.
// dE is the change of site i's Hamiltonian terms: exchange and applied field through the
// field h = H_app + sum_j (J_ij / mu_s,i) S_j, then anisotropy and the Neel term.
// One Hinzke-Nowak trial move of spin i (Section "Monte Carlo Methods"): spin flip, Gaussian
// or random move by a Philox draw, accepted by Eq. AMCP.  Returns whether it was accepted;
// sysid receives the spin's system.  Rec (0: none) also gives the spin's record terms of the
// pre-step state in v: mu S (3), the exchange term (1: -mu S.(h - H_app) - mu S.H_app/2 for
// the first colour class, whose bonds all end on unchanged spins; 2: -mu S.H_app/2), and
// the anisotropy energy.
// The FP64 Box-Muller tables of a kernel: its shared-memory copy in the FP64 form; in the
// FP32-mixed form (whose kernels stage the double-float tables) the global buffer itself, laid
// out as SmemTables (log | ln2 | trig | log remainders), read through the caches.
__device__ __forceinline__ const SmemTables &fp64_tables(const KArgs<double> &, const SmemTables &t) { return t; }
__device__ __forceinline__ const SmemTables &fp64_tables(const KArgs<float> &a, const FFTables &) {
    return *reinterpret_cast<const SmemTables *>(a.tab);
}

// The random part of spin i's trial at `step`: the move type (0 flip, 1 Gaussian, 2 random),
// the Gaussian triple (drawn for moves 1 and 2) and the acceptance factor -(-2 ln u)/2.
template <typename R>
__device__ __forceinline__ int mc_randoms(const KArgs<R> &a, int64_t i, uint64_t step, const StepTabT<R> &tab,
                                          R &g0, R &g1, R &g2, double &lnu) {
    const MatDesc<R> &mt = a.mats[mat_of(a, i)];
    const SysDesc &sd = a.sys[mt.sys];
    const uint32_t spin = (uint32_t)(i - sd.offset + sd.pbase);
    const Philox4 wa = philox4x32_10(spin, (uint32_t)step, sd.ctr2, 2u, sd.key0, sd.key1);
    const Philox4 wb = philox4x32_10(spin, (uint32_t)step, sd.ctr2, 3u, sd.key0, sd.key1);
    const int move = (int)(((uint64_t)wb.w0 * 3u) >> 32);
    if (move != 0) {
        if constexpr (sizeof(R) == 8) {
            box_muller3(wa, tab, g0, g1, g2);
        } else {  // the FP64 transform's values rounded to float, from the double-float transform
            gaussians_f32(wa, tab, a.tab, g0, g1, g2);
        }
    }
    lnu = -0.5 * neg2log_u(wb.w1, fp64_tables(a, tab));
    return move;
}

template <typename R, int Mode, int Rec, bool GivenH = false, bool Pre = false>
__device__ __forceinline__ bool mc_trial(const KArgs<R> &a, const McArgs &m, int64_t i, uint64_t step,
                                         const StepTabT<R> *tab, int &sysid, double v[5], R gh0 = 0, R gh1 = 0,
                                         R gh2 = 0) {
    bool accept;
    const MatDesc<R> &mt = a.mats[mat_of(a, i)];
    const SysDesc &sd = a.sys[mt.sys];
    double2 par;
    if (a.sched_len > 0) {
        int64_t q = (int64_t)step - a.sched_step0;
        q = q < 0 ? 0 : (q >= a.sched_len ? a.sched_len - 1 : q);
        par = m.par_sched[q];
    } else {
        par = m.par_sys[mt.sys];
    }
    R g0 = (R)0, g1 = (R)0, g2 = (R)0;
    double lnu;
    int move;
    if constexpr (Pre) {  // drawn beforehand by k_mc_prep
        move = m.pre_move[i];
        const R *pg = static_cast<const R *>(m.pre_g);
        g0 = pg[i];
        g1 = pg[a.n + i];
        g2 = pg[2 * a.n + i];
        lnu = m.pre_acc[i];
    } else {
        move = mc_randoms(a, i, step, *tab, g0, g1, g2, lnu);
    }
    const R s0 = a.sx[i], s1 = a.sy[i], s2 = a.sz[i];
    R n0, n1, n2;
    if (move == 0) {  // spin flip
        n0 = -s0;
        n1 = -s1;
        n2 = -s2;
    } else if (move == 1 && par.y == 0.0) {  // T = 0: a Gaussian cone of width 0
        n0 = s0;
        n1 = s1;
        n2 = s2;
    } else {
        if (move == 1) {  // Gaussian move: S + sigma_g Gamma, normalised
            if constexpr (sizeof(R) == 8) {
                const double sg = par.y;
                n0 = fma(sg, g0, s0);
                n1 = fma(sg, g1, s1);
                n2 = fma(sg, g2, s2);
            } else {
                const float sgf = narrow<float>(par.y);
                n0 = fmaf(sgf, g0, s0);
                n1 = fmaf(sgf, g1, s1);
                n2 = fmaf(sgf, g2, s2);
            }
        } else {  // random move: Gamma normalised
            n0 = g0;
            n1 = g1;
            n2 = g2;
        }
        const R inv = rsqrt_r(n0 * n0 + n1 * n1 + n2 * n2);
        n0 *= inv;
        n1 *= inv;
        n2 *= inv;
    }
    R h0 = gh0, h1 = gh1, h2 = gh2;  // GivenH: H_app + sum_j (J_ij/mu_s,i) S_j summed by the caller
    if constexpr (!GivenH) exchange_sum<R, false, Mode>(a, sd, a.sx, a.sy, a.sz, i, h0, h1, h2);
    // quadratic terms as (n - s).(A (n + s)): exactly zero when the spin is unchanged or
    // flipped, whatever the contraction of products into FMAs
    const R d0 = n0 - s0, d1 = n1 - s1, d2 = n2 - s2;
    const R p0 = n0 + s0, p1 = n1 + s1, p2 = n2 + s2;
    const R de = d0 * mt.e[0] + d1 * mt.e[1] + d2 * mt.e[2];
    const R pe = p0 * mt.e[0] + p1 * mt.e[1] + p2 * mt.e[2];
    R dE = -mt.mu * (d0 * h0 + d1 * h1 + d2 * h2) - mt.ku * (de * pe);
    if (Mode != kPlain && mt.has_cubic) {  // (k_c/2) sum (n^4 - s^4), n^4 - s^4 = (n - s)(n + s)(n^2 + s^2)
        dE += (R)0.5 * mt.kc * (d0 * p0 * (n0 * n0 + s0 * s0) + d1 * p1 * (n1 * n1 + s1 * s1)
                                + d2 * p2 * (n2 * n2 + s2 * s2));
    }
    if (mt.has_neel) {
        const R k0 = mt.K[0] * p0 + mt.K[3] * p1 + mt.K[4] * p2;
        const R k1 = mt.K[3] * p0 + mt.K[1] * p1 + mt.K[5] * p2;
        const R k2 = mt.K[4] * p0 + mt.K[5] * p1 + mt.K[2] * p2;
        dE -= d0 * k0 + d1 * k1 + d2 * k2;
    }
    // accept when dE <= -kB T ln u = (-kB T)(-1/2)(-2 ln u); at T = 0 when dE <= 0
    const double dEd = widen(dE);
    accept = par.x < 0.0 ? dEd <= par.x * lnu : dEd <= 0.0;
    if (accept) {
        a.sx[i] = n0;
        a.sy[i] = n1;
        a.sz[i] = n2;
    }
    if constexpr (Rec != 0) {  // terms in the working type, summed in FP64 (as spin_terms)
        const R mu = mt.mu;
        v[0] = widen(mu * s0);
        v[1] = widen(mu * s1);
        v[2] = widen(mu * s2);
        const R sh = s0 * sys_H(sd, 0, R()) + s1 * sys_H(sd, 1, R()) + s2 * sys_H(sd, 2, R());  // S.H_app
        if (Rec == 1)
            v[3] = widen(-mu * (s0 * h0 + s1 * h1 + s2 * h2) + (R)0.5 * mu * sh);
        else
            v[3] = widen((R)-0.5 * mu * sh);
        const R se = s0 * mt.e[0] + s1 * mt.e[1] + s2 * mt.e[2];
        R ea = -mt.ku * se * se;
        if (Mode != kPlain && mt.has_cubic) {
            const R x2 = s0 * s0, y2 = s1 * s1, z2 = s2 * s2;
            ea += (R)0.5 * mt.kc * (x2 * x2 + y2 * y2 + z2 * z2);
        }
        if (mt.has_neel) {
            ea -= mt.K[0] * s0 * s0 + mt.K[1] * s1 * s1 + mt.K[2] * s2 * s2
                + (R)2 * (mt.K[3] * s0 * s1 + mt.K[4] * s0 * s2 + mt.K[5] * s1 * s2);
        }
        v[4] = widen(ea);
    }
    sysid = mt.sys;
    return accept;
}

template <typename R, int BS, int Mode = kGeneral>
__global__ void __launch_bounds__(BS) k_mc_colour(const KArgs<R> a, const McArgs m) {
    __shared__ StepTabT<R> tab;
    stage_step_tables(a, tab);
    __syncthreads();
    const uint64_t step = *a.step;
    for (int64_t k = m.c0 + (int64_t)blockIdx.x * BS + threadIdx.x; k < m.c1; k += (int64_t)gridDim.x * BS) {
        int sysid;
        double v[5];
        const bool accept = mc_trial<R, Mode, 0>(a, m, chk(__ldg(m.order + k), a.n, a.err), step, &tab, sysid, v);
        // accepted moves per system, one atomic per (warp, system)
        const unsigned act = __activemask();
        const unsigned same = __match_any_sync(act, sysid);
        const unsigned yes = __ballot_sync(act, accept);
        if ((int)(threadIdx.x & 31) == __ffs(same) - 1)
            atomicAdd(m.acc + sysid, (unsigned long long)__popc(yes & same));
    }
}

// A colour pass for long exchange rows: each warp takes 32 trials of the class, sums their
// rows one by one with its lanes striding over the row's bonds (col + J, or tensors) and a
// butterfly, and each lane then runs its own trial with its row's field (the neighbours of a
// class are of other classes, unchanged during the pass).
// Lane `lane`'s share of the scalar exchange sum of row [b, e) (bonds b + lane, b + lane + 32,
// ... in order): eight bonds at a time, their columns first, then their gathers, then the
// sums in bond order, so that the loads of a lane overlap.
template <typename R>
__device__ __forceinline__ void mc_row_sum8(const KArgs<R> &a, int32_t b, int32_t e, int lane, R &x, R &y, R &z) {
    constexpr int U = 8;
    for (int32_t t0 = b + lane; t0 < e; t0 += 32 * U) {
        int32_t jj[U];
        R Jk[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int32_t t = t0 + 32 * u;
            jj[u] = t < e ? chk(__ldg(a.col + t), a.n, a.err) : -1;
            Jk[u] = a.J_uniform ? a.J_value : (t < e ? __ldg(a.J + t) : (R)0);
        }
        R sx[U], sy[U], sz[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int32_t j = jj[u] >= 0 ? jj[u] : 0;
            sx[u] = a.sx[j];
            sy[u] = a.sy[j];
            sz[u] = a.sz[j];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (jj[u] >= 0) {
                x = fma(Jk[u], sx[u], x);
                y = fma(Jk[u], sy[u], y);
                z = fma(Jk[u], sz[u], z);
            }
        }
    }
}

// The trial randoms of the device's current step for every spin (move type, Gaussian triple,
// acceptance factor), for the long-row colour passes: their trials then run without the
// transform's tables or its serial work (mc_randoms is what mc_trial draws otherwise).
template <typename R, int BS>
__global__ void __launch_bounds__(BS) k_mc_prep(const KArgs<R> a, const McArgs m) {
    __shared__ StepTabT<R> tab;
    stage_step_tables(a, tab);
    __syncthreads();
    const uint64_t step = *a.step;
    uint8_t *mv = const_cast<uint8_t *>(m.pre_move);
    R *pg = static_cast<R *>(const_cast<void *>(m.pre_g));
    double *pa = const_cast<double *>(m.pre_acc);
    for (int64_t i = (int64_t)blockIdx.x * BS + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * BS) {
        R g0 = (R)0, g1 = (R)0, g2 = (R)0;
        double lnu;
        mv[i] = (uint8_t)mc_randoms(a, i, step, tab, g0, g1, g2, lnu);
        pg[i] = g0;
        pg[a.n + i] = g1;
        pg[2 * a.n + i] = g2;
        pa[i] = lnu;
    }
}

template <typename R, int BS, int Mode>
__global__ void __launch_bounds__(BS) k_mc_colour_warp(const KArgs<R> a, const McArgs m) {
    // the trial randoms come from k_mc_prep: no tables
    const uint64_t step = *a.step;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * BS + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * BS) >> 5;
    for (int64_t k0 = m.c0 + warp * 32; k0 < m.c1; k0 += nwarps * 32) {
        const int64_t k = k0 + lane;
        const int64_t i = k < m.c1 ? (int64_t)chk(__ldg(m.order + k), a.n, a.err) : -1;
        int32_t rb = 0, re = 0;
        if (i >= 0) {
            rb = __ldg(a.row_ptr + i);
            re = __ldg(a.row_ptr + i + 1);
        }
        const int nr = m.c1 - k0 < 32 ? (int)(m.c1 - k0) : 32;
        R mx = 0, my = 0, mz = 0;
        for (int q = 0; q < nr; ++q) {
            const int32_t b = __shfl_sync(FULL, rb, q), e = __shfl_sync(FULL, re, q);
            R x = 0, y = 0, z = 0;
            if (Mode == kPlain || !a.J_tensor) {
                mc_row_sum8(a, b, e, lane, x, y, z);
            } else {
#pragma unroll 4
                for (int32_t t = b + lane; t < e; t += 32) {
                    const int32_t j = chk(__ldg(a.col + t), a.n, a.err);
                    const R s0 = a.sx[j], s1 = a.sy[j], s2 = a.sz[j];
                    const R *tt = a.Jt + 9 * (int64_t)__ldg(a.Jtidx + t);
                    x = fma(__ldg(tt + 0), s0, fma(__ldg(tt + 1), s1, fma(__ldg(tt + 2), s2, x)));
                    y = fma(__ldg(tt + 3), s0, fma(__ldg(tt + 4), s1, fma(__ldg(tt + 5), s2, y)));
                    z = fma(__ldg(tt + 6), s0, fma(__ldg(tt + 7), s1, fma(__ldg(tt + 8), s2, z)));
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                x += __shfl_xor_sync(FULL, x, o);
                y += __shfl_xor_sync(FULL, y, o);
                z += __shfl_xor_sync(FULL, z, o);
            }
            if (lane == q) {
                mx = x;
                my = y;
                mz = z;
            }
        }
        bool accept = false;
        int sysid = -1;
        if (i >= 0) {
            const SysDesc &sd = a.sys[a.mats[mat_of(a, i)].sys];
            double v[5];
            accept = mc_trial<R, Mode, 0, true, true>(a, m, i, step, nullptr, sysid, v, sys_H(sd, 0, R()) + mx,
                                                 sys_H(sd, 1, R()) + my, sys_H(sd, 2, R()) + mz);
        }
        const unsigned same = __match_any_sync(FULL, sysid);
        const unsigned yes = __ballot_sync(FULL, accept);
        if (sysid >= 0 && lane == __ffs(same) - 1) atomicAdd(m.acc + sysid, (unsigned long long)__popc(yes & same));
    }
}

// As k_mc_colour_warp for colour classes too small to fill the GPU 32 trials to a warp: each
// warp takes one trial, sums its row across the lanes, and lane 0 runs the trial.
template <typename R, int BS, int Mode>
__global__ void __launch_bounds__(BS) k_mc_colour_warp1(const KArgs<R> a, const McArgs m) {
    // the trial randoms come from k_mc_prep: no tables
    const uint64_t step = *a.step;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * BS + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * BS) >> 5;
    for (int64_t k = m.c0 + warp; k < m.c1; k += nwarps) {
        const int64_t i = chk(__ldg(m.order + k), a.n, a.err);
        const int32_t b = __ldg(a.row_ptr + i), e = __ldg(a.row_ptr + i + 1);
        R x = 0, y = 0, z = 0;
        if (Mode == kPlain || !a.J_tensor) {
            mc_row_sum8(a, b, e, lane, x, y, z);
        } else {
#pragma unroll 4
            for (int32_t t = b + lane; t < e; t += 32) {
                const int32_t j = chk(__ldg(a.col + t), a.n, a.err);
                const R s0 = a.sx[j], s1 = a.sy[j], s2 = a.sz[j];
                const R *tt = a.Jt + 9 * (int64_t)__ldg(a.Jtidx + t);
                x = fma(__ldg(tt + 0), s0, fma(__ldg(tt + 1), s1, fma(__ldg(tt + 2), s2, x)));
                y = fma(__ldg(tt + 3), s0, fma(__ldg(tt + 4), s1, fma(__ldg(tt + 5), s2, y)));
                z = fma(__ldg(tt + 6), s0, fma(__ldg(tt + 7), s1, fma(__ldg(tt + 8), s2, z)));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_xor_sync(FULL, x, o);
            y += __shfl_xor_sync(FULL, y, o);
            z += __shfl_xor_sync(FULL, z, o);
        }
        if (lane == 0) {
            const SysDesc &sd = a.sys[a.mats[mat_of(a, i)].sys];
            int sysid;
            double v[5];
            const bool accept = mc_trial<R, Mode, 0, true, true>(a, m, i, step, nullptr, sysid, v, sys_H(sd, 0, R()) + x,
                                                           sys_H(sd, 1, R()) + y, sys_H(sd, 2, R()) + z);
            if (accept) atomicAdd(m.acc + sysid, 1ull);
        }
    }
}

// A colour pass tile by tile that also sums the record terms of the pre-step state of its
// spins (tile partials in the block's fixed order), for lattices of at most two classes.
template <typename R, int BS, int Mode, bool First>
__global__ void __launch_bounds__(BS) k_mc_colour_rec(const KArgs<R> a, const McArgs m) {
    __shared__ StepTabT<R> tab;
    __shared__ double red[(BS / 32) * 8];
    stage_step_tables(a, tab);
    __syncthreads();
    const uint64_t step = *a.step;
    for (int64_t t = blockIdx.x; t < m.ntiles; t += gridDim.x) {
        const TileDesc td = m.tiles[t];
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int k = threadIdx.x; k < td.count; k += BS) {
            int sysid;
            double v[5];
            const bool accept = mc_trial<R, Mode, First ? 1 : 2>(a, m, chk(__ldg(m.order + td.start + k), a.n, a.err),
                                                                 step, &tab, sysid, v);
#pragma unroll
            for (int c = 0; c < 5; ++c) acc[c] += v[c];
            // a tile lies in one system: one atomic per warp
            const unsigned act = __activemask();
            const unsigned yes = __ballot_sync(act, accept);
            if ((int)(threadIdx.x & 31) == __ffs(act) - 1) atomicAdd(m.acc + sysid, (unsigned long long)__popc(yes));
        }
        const double r = block_sum8<BS>(acc, red);
        if (threadIdx.x < kPartComps) m.partials[(int64_t)m.slot[t] * kPartComps + threadIdx.x] = r;
    }
}

}  // namespace ss
