/*
 * spinsys_oracle.c -- plain, slow, FP64 CPU oracle of the stochastic Heun-LLG step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this
 * file; only tests, the smoke check and the benchmark's CPU-baseline leg use it.  It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * What it computes (Evans et al., "Atomistic spin model simulations of magnetic
 * nanomaterials", arXiv:1310.6143):
 *   - Hamiltonian H = H_exc + H_ani + H_app                       (Eq. spinhamiltonian)
 *       H_exc = -sum_{i!=j} J_ij S_i.S_j, each bond counted once   (Eq. HJij, reading below)
 *       H_ani = -k_u sum_i (S_i.e)^2                              (uniaxial anisotropy eq.)
 *       H_app = -sum_i mu_s S_i.H_app                             (applied-field eq.)
 *       H_ani also takes the cubic term (k_c/2) sum_i (Sx^4+Sy^4+Sz^4) (cubic-anisotropy eq.)
 *       and H_exc the tensorial form of Eq. HJijSMS when tensors are given (T1, T2);
 *     plus an optional per-site Neel surface tensor term -S_i^T K_i S_i (not in the
 *     paper; a project extension for surface anisotropy, folded into the anisotropy
 *     energy).
 *   - Effective field H_eff = -(1/mu_s) dH/dS_i                    (Eq. Heff)
 *   - Langevin thermal field Gamma(t) sqrt(2 lambda kB T/(gamma mu_s dt))  (thermal-field eq.)
 *   - LLG right-hand side -gamma/(1+lambda^2)[S x H + lambda S x (S x H)]  (Eq. LLG)
 *   - Heun predictor / corrector with renormalisation after both passes and the thermal
 *     field held fixed between them; predictor over all spins before any corrector
 *     (Section "Time Integration of the LLG Equation").
 *
 * Readings of the paper that this file takes (the paper is silent or ambiguous):
 *   R1  H_exc counts each bond once: the field is (1/mu_s) sum_j J_ij S_j and the energy
 *       is -1/2 sum_i sum_j J_ij S_i.S_j over the (symmetric) neighbour list.
 *   R2  Constants are the paper's Table I values (gamma = 1.76e11, kB = 1.3807e-23).
 *   R3  Noise variance 2 lambda kB T/(gamma mu_s dt) carries no (1+lambda^2) factor.
 *   R4  The thermal field for step n is drawn once, at temperature T(t_n), t_n = n dt,
 *       and used unchanged by predictor and corrector.
 *   R5  The corrector starts from the un-normalised sum S + dt/2 (dS + dS') and is then
 *       renormalised; dS' is evaluated at the renormalised predictor spin S'.
 *   R6  Random numbers: the paper's Mersenne Twister + Ziggurat is replaced by a
 *       counter-based Philox4x32-10 generator (Salmon, Moraes, Dror and Shaw, SC'11)
 *       followed by the Box-Muller transform (Box and Muller, 1958).  One Philox call per
 *       (spin, step): counter (i, n, system, 0), key (seed low word, seed high word);
 *       u_k = (w_k + 1/2) 2^-32;  gx = sqrt(-2 ln u0) cos(2 pi u1),
 *       gy = sqrt(-2 ln u0) sin(2 pi u1),  gz = sqrt(-2 ln u2) cos(2 pi u3).
 *       Initial random spins use counter (i, 0xFFFFFFFF, system, 1) and normalise the
 *       same three Gaussians.
 *   R7  Magnetisation is sum_i mu_s,i S_i (and sum_i mu_s,i); the per-step record holds
 *       the state at the start of the step, S(t_n).
 *
 * Monte Carlo (Section "Monte Carlo Methods": the Metropolis criterion, Eq. AMCP, with
 * the Hinzke-Nowak trial moves: spin flip, Gaussian move Eq. MCgaussian with the cone
 * width Eq. MCgaussianSigma, random move Eq. MCrandom), readings:
 *   M1  One Monte Carlo step gives every spin exactly one trial move, colour class by
 *       colour class of a proper colouring of the neighbour graph (no two neighbours share
 *       a colour), colours in increasing order, the spins of one colour in site order (they
 *       do not interact, so their order does not change the result).  The colouring is
 *       greedy in site order: each site takes the smallest colour no earlier neighbour
 *       holds.  (The paper picks N random sites per step; every single-spin Metropolis
 *       update keeps the Boltzmann distribution invariant either way.)
 *   M2  Random numbers per (spin i, Monte Carlo step n): Philox block A with counter
 *       (i, n, system, 2) gives the Gaussian triple Gamma by the Box-Muller transform of R6;
 *       block B with counter (i, n, system, 3) gives the move type from its first word w0,
 *       floor(3 w0 / 2^32) (0 spin flip, 1 Gaussian, 2 random), and the acceptance uniform
 *       u = (w1 + 1/2) 2^-32 from its second word.
 *   M3  A move is accepted when dE <= -kB T ln u, i.e. u <= exp(-dE/(kB T)) (Eq. AMCP);
 *       energy-lowering moves are always accepted; at T = 0 exactly the moves with dE <= 0.
 *       At T = 0 the cone width is 0 and the Gaussian move leaves the spin exactly as it is
 *       (dE = 0, counted as accepted) rather than renormalising it.
 *   M4  The energy change is that of site i's terms of the Hamiltonian: exchange with its
 *       neighbours, its anisotropy, its applied-field term and its Neel term.
 *   M5  The record of Monte Carlo step n holds the state at the start of the step.
 *
 * Demagnetising field (Section "Demagnetising fields": Eqs. macrocellpos, mc_volume, demag,
 * demag-fast), readings:
 *   D1  Macrocells are cubes of edge `demag_cell` on a grid anchored at the smallest atomic
 *       coordinate of the system on each axis; an atom belongs to the cube holding its
 *       position; empty cubes are not macrocells.  Macrocells are numbered in the order of
 *       their grid index (x fastest, then y, then z).
 *   D2  Position of a macrocell: the moment-weighted centre of mass (Eq. macrocellpos);
 *       moment: sum_i mu_s,i S_i; volume: n_atoms * V_atom (Eq. mc_volume), with V_atom =
 *       V_uc / n_uc given per system (`demag_vatom`).
 *   D3  H_p = mu0/(4 pi) sum_{q != p} [3 (m_q . r) r - m_q] / |r_pq|^3 - (mu0/3) m_p / V_p with
 *       r the unit vector from p to q (Eq. demag); Eq. demag-fast is the same sum with the
 *       dipole tensors precomputed (its printed diagonal "-1/3" and the missing 1/r^3 on its
 *       off-diagonal entries are read as garbled: the self term is the separate -mu0/3 m/V).
 *       mu0 = 4 pi 1e-7 T m/A.  H_p acts on every atom of macrocell p as an added field.
 *   D4  The field is recomputed from the state at the start of step n when n is a multiple
 *       of `demag_every` and at the first step of each call, and held fixed in between; both
 *       Heun passes of a step use the same field.
 *   D5  The recorded energies exclude the demagnetising energy.
 *
 * Tensorial exchange (Eqs. HJijM, HJijSMS) and cubic anisotropy (the cubic-anisotropy
 * equation), readings:
 *   T1  A bond k of row i (i -> j = col[k]) may carry a 3x3 exchange tensor J_k, stored row
 *       by row (Jxx Jxy Jxz Jyx Jyy Jyz Jzx Jzy Jzz).  The field on i is (1/mu_s,i) sum_k J_k S_j
 *       and the energy -1/2 sum_i S_i . sum_k J_k S_j (each bond once, as R1); the field is
 *       the gradient of that energy when the reverse bond carries the transpose.  A scalar J
 *       is the tensor J times the identity.
 *   T2  The cubic anisotropy energy is +(k_c/2)(Sx^4 + Sy^4 + Sz^4) per atom as printed (the
 *       sign of k_c picks the easy axes) in the lattice frame, with the field
 *       -(2 k_c/mu_s)(Sx^3, Sy^3, Sz^3); it is part of the anisotropy energy.
 *
 * Midpoint integrator (the midpoint rule the paper's time-integration section cites,
 * d'Aquino et al. 2005), readings:
 *   I1  S_{n+1} = S_n + dt f(m), m = (S_n + S_{n+1})/2, f the right-hand side of Eq. LLG with
 *       the deterministic field of m and the thermal field of R4 (drawn once per step from
 *       the same Philox counters, held over the step).  f(m) is perpendicular to m, so the
 *       rule keeps |S| without renormalisation.
 *   I2  The implicit equation is solved by K fixed-point iterations from the Euler predictor
 *       S^(0) = S_n + dt f(S_n): S^(k+1) = S_n + dt f((S_n + S^(k))/2), k = 0 .. K-1, and
 *       S_{n+1} = S^(K); nothing is renormalised.
 *   I3  The record holds the state at the start of each step (R7); the demagnetising field,
 *       when on, is updated as for Heun (D4) and held, like the thermal field, over the step.
 *
 * Semi-implicit predictor-corrector (the modified predictor-corrector midpoint scheme the
 * paper cites, Mentink et al. 2010, their scheme B), readings:
 *   P1  Eq. LLG written as dS/dt = S x A(S), A(S) = -gamma/(1+lambda^2) (H + lambda S x H),
 *       H the deterministic field of S plus the thermal field of R4 (drawn once per step from
 *       the same Philox counters, held over the step).
 *   P2  Predictor: S' = S_n + (dt/2) (S_n + S') x A(S_n); corrector: S_{n+1} = S_n +
 *       (dt/2) (S_n + S_{n+1}) x A(Sb), Sb = (S_n + S')/2 (the field and the damping term
 *       both at Sb, which is not renormalised).  Each is a 3x3 linear equation in the new
 *       spin, solved in closed form: with b = (dt/2) A and c = S_n + S_n x b, the new spin is
 *       (c - b x c + (b.c) b)/(1 + |b|^2), a rotation of S_n, so |S| is kept without
 *       renormalisation.
 *   P3  The record holds the state at the start of each step (R7); the demagnetising field as I3.
 *
 * Layout: spins and vectors are array-of-structures, 3 doubles per site (x, y, z).
 * Neel tensors are 6 doubles per site in the order xx, yy, zz, xy, xz, yz.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no fused multiply-add, so
 * every product and sum is rounded as written).  The spin loops may run on several
 * threads; every site is computed independently and every sum over sites runs serially
 * in site order, so the result does not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_KB 1.3807e-23      /* Boltzmann constant, J/K (Table I) */
#define ORC_GAMMA 1.76e11      /* gyromagnetic ratio, 1/(T s) (Table I) */
#define ORC_PI 3.14159265358979323846
#define ORC_MUB 9.2740e-24     /* Bohr magneton, J/T (Table I) */
#define ORC_MU0 (4.0e-7 * ORC_PI) /* vacuum permeability, T m/A (reading D3) */

typedef struct {
    int64_t n;                /* number of spins                                  */
    const int64_t *row_ptr;   /* [n+1] CSR row offsets                             */
    const int32_t *col;       /* [nnz] neighbour indices                           */
    const double *J;          /* [nnz] exchange constants, J/link                  */
    const double *mu_s;       /* [n] atomic moments, J/T                           */
    const double *k_u;        /* [n] uniaxial anisotropy, J/atom                   */
    const double *easy_axis;  /* [3n] unit easy axes                               */
    const double *K_neel;     /* [6n] Neel tensors (xx,yy,zz,xy,xz,yz) or NULL     */
    double alpha;             /* Gilbert damping lambda                            */
    double dt;                /* time step, s                                      */
    double gamma;             /* gyromagnetic ratio, 1/(T s)                       */
    double H_app[3];          /* applied field, T                                  */
    uint64_t seed;            /* Philox key                                        */
    uint32_t sys;             /* system id (third counter word)                    */
    const uint32_t *ids;      /* [n] Philox spin word of each site, or NULL (= i); lets a
                                 test run a cut-out neighbourhood of a large system     */
    const double *pos;        /* [3n] atomic positions, m (needed by the demag field)   */
    double demag_cell;        /* macrocell edge, m; <= 0: no demagnetising field        */
    double demag_vatom;       /* volume per atom V_uc / n_uc, m^3                       */
    int64_t demag_every;      /* steps between updates of the demagnetising field       */
    const double *Jt;         /* [9 nnz] exchange tensors (T1) or NULL (scalar J)       */
    const double *k_c;        /* [n] cubic anisotropy, J/atom (T2), or NULL             */
} orc_system;

static int g_threads = 1;

void orc_set_threads(int t) { g_threads = t < 1 ? 1 : t; }

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 multiplications   */
/* with the published multipliers, the key bumped by the published Weyl increments     */
/* between rounds.                                                                      */
/* ---------------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        x0 = y0;
        x1 = lo1;
        x2 = y2;
        x3 = lo0;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static double orc_uniform(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

/* Three standard Gaussians from one Philox block (reading R6). */
static void orc_box_muller3(const uint32_t w[4], double g[3]) {
    double u0 = orc_uniform(w[0]), u1 = orc_uniform(w[1]);
    double u2 = orc_uniform(w[2]), u3 = orc_uniform(w[3]);
    double r1 = sqrt(-2.0 * log(u0));
    double r2 = sqrt(-2.0 * log(u2));
    double phi1 = 2.0 * ORC_PI * u1;
    double phi2 = 2.0 * ORC_PI * u3;
    g[0] = r1 * cos(phi1);
    g[1] = r1 * sin(phi1);
    g[2] = r2 * cos(phi2);
}

void orc_thermal_gaussians(uint64_t seed, uint32_t sys, uint32_t spin, uint32_t step, double g[3]) {
    uint32_t ctr[4] = {spin, step, sys, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    orc_box_muller3(w, g);
}

/* Random-on-sphere initial state: normalised Gaussian triple from the reserved stream. */
void orc_init_sphere(uint64_t seed, uint32_t sys, int64_t n, double *S) {
    for (int64_t i = 0; i < n; ++i) {
        uint32_t ctr[4] = {(uint32_t)i, 0xFFFFFFFFu, sys, 1u};
        uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
        uint32_t w[4];
        double g[3];
        orc_philox4x32_10(ctr, key, w);
        orc_box_muller3(w, g);
        double len = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        S[3 * i + 0] = g[0] / len;
        S[3 * i + 1] = g[1] / len;
        S[3 * i + 2] = g[2] / len;
    }
}

/* ---------------------------------------------------------------------------------- */
/* Deterministic field of one site, Eq. Heff applied to the Hamiltonian terms.         */
/* hex receives the raw exchange sum sum_j J_ij S_j (J), H the field in tesla.         */
/* Terms are added in the order: exchange, anisotropy, applied, Neel.                  */
/* ---------------------------------------------------------------------------------- */
/* sum_k J_k S_j over row i: scalar J (R1) or exchange tensors (T1). */
static void orc_exchange_sum(const orc_system *s, const double *S, int64_t i, double h[3]) {
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int64_t k = s->row_ptr[i]; k < s->row_ptr[i + 1]; ++k) {
        int64_t j = s->col[k];
        if (s->Jt) {
            const double *t = s->Jt + 9 * k;
            sx += t[0] * S[3 * j + 0] + t[1] * S[3 * j + 1] + t[2] * S[3 * j + 2];
            sy += t[3] * S[3 * j + 0] + t[4] * S[3 * j + 1] + t[5] * S[3 * j + 2];
            sz += t[6] * S[3 * j + 0] + t[7] * S[3 * j + 1] + t[8] * S[3 * j + 2];
        } else {
            sx += s->J[k] * S[3 * j + 0];
            sy += s->J[k] * S[3 * j + 1];
            sz += s->J[k] * S[3 * j + 2];
        }
    }
    h[0] = sx; h[1] = sy; h[2] = sz;
}

static void orc_site_field(const orc_system *s, const double *S, int64_t i, double hex[3], double H[3]) {
    double hs[3];
    orc_exchange_sum(s, S, i, hs);
    double sx = hs[0], sy = hs[1], sz = hs[2];
    hex[0] = sx; hex[1] = sy; hex[2] = sz;
    double mu = s->mu_s[i];
    /* exchange: -(1/mu) d/dS_i of -sum_{bonds} J S_i.S_j */
    H[0] = sx / mu;
    H[1] = sy / mu;
    H[2] = sz / mu;
    /* uniaxial anisotropy: -(1/mu) d/dS of -k_u (S.e)^2 = (2 k_u/mu)(S.e) e */
    const double *e = s->easy_axis + 3 * i;
    double sdote = S[3 * i + 0] * e[0] + S[3 * i + 1] * e[1] + S[3 * i + 2] * e[2];
    double a = 2.0 * s->k_u[i] / mu * sdote;
    H[0] += a * e[0];
    H[1] += a * e[1];
    H[2] += a * e[2];
    /* cubic anisotropy (T2): -(1/mu) d/dS of (k_c/2)(Sx^4+Sy^4+Sz^4) = -(2 k_c/mu) S^3 */
    if (s->k_c) {
        double c = -2.0 * s->k_c[i] / mu;
        double x = S[3 * i + 0], y = S[3 * i + 1], z = S[3 * i + 2];
        H[0] += c * x * x * x;
        H[1] += c * y * y * y;
        H[2] += c * z * z * z;
    }
    /* applied field: -(1/mu) d/dS of -mu S.H_app = H_app */
    H[0] += s->H_app[0];
    H[1] += s->H_app[1];
    H[2] += s->H_app[2];
    /* Neel tensor: -(1/mu) d/dS of -S^T K S = (2/mu) K S */
    if (s->K_neel) {
        const double *K = s->K_neel + 6 * i;
        double x = S[3 * i + 0], y = S[3 * i + 1], z = S[3 * i + 2];
        double kx = K[0] * x + K[3] * y + K[4] * z;
        double ky = K[3] * x + K[1] * y + K[5] * z;
        double kz = K[4] * x + K[5] * y + K[2] * z;
        H[0] += 2.0 / mu * kx;
        H[1] += 2.0 / mu * ky;
        H[2] += 2.0 / mu * kz;
    }
}

/* Deterministic fields of all sites (tesla), AoS [3n]; exposed for tests. */
void orc_fields(const orc_system *s, const double *S, double *H) {
    for (int64_t i = 0; i < s->n; ++i) {
        double hex[3];
        orc_site_field(s, S, i, hex, H + 3 * i);
    }
}

/* Magnetisation and energy of a state (reading R7, energy per R1):
 * out = {sum mu Sx, sum mu Sy, sum mu Sz, sum mu, E_exc, E_ani, E_app, E_total} (J/T, J). */
void orc_moment_energy(const orc_system *s, const double *S, double out[8]) {
    double m0 = 0, m1 = 0, m2 = 0, msum = 0, eex = 0, ean = 0, eap = 0;
    for (int64_t i = 0; i < s->n; ++i) {
        double hex[3], H[3];
        orc_site_field(s, S, i, hex, H);
        const double *Si = S + 3 * i;
        double mu = s->mu_s[i];
        m0 += mu * Si[0];
        m1 += mu * Si[1];
        m2 += mu * Si[2];
        msum += mu;
        eex += -0.5 * (Si[0] * hex[0] + Si[1] * hex[1] + Si[2] * hex[2]);
        const double *e = s->easy_axis + 3 * i;
        double sdote = Si[0] * e[0] + Si[1] * e[1] + Si[2] * e[2];
        double ea = -s->k_u[i] * sdote * sdote;
        if (s->k_c) {
            double x2 = Si[0] * Si[0], y2 = Si[1] * Si[1], z2 = Si[2] * Si[2];
            ea += 0.5 * s->k_c[i] * (x2 * x2 + y2 * y2 + z2 * z2);
        }
        if (s->K_neel) {
            const double *K = s->K_neel + 6 * i;
            double x = Si[0], y = Si[1], z = Si[2];
            double q = K[0] * x * x + K[1] * y * y + K[2] * z * z
                     + 2.0 * (K[3] * x * y + K[4] * x * z + K[5] * y * z);
            ea += -q;
        }
        ean += ea;
        eap += -mu * (Si[0] * s->H_app[0] + Si[1] * s->H_app[1] + Si[2] * s->H_app[2]);
    }
    out[0] = m0; out[1] = m1; out[2] = m2; out[3] = msum;
    out[4] = eex; out[5] = ean; out[6] = eap; out[7] = eex + ean + eap;
}

/* LLG right-hand side, Eq. LLG. */
static void orc_llg(double gamma, double lambda, const double S[3], const double H[3], double dS[3]) {
    double c0 = S[1] * H[2] - S[2] * H[1];
    double c1 = S[2] * H[0] - S[0] * H[2];
    double c2 = S[0] * H[1] - S[1] * H[0];
    double d0 = S[1] * c2 - S[2] * c1;
    double d1 = S[2] * c0 - S[0] * c2;
    double d2 = S[0] * c1 - S[1] * c0;
    double pre = -gamma / (1.0 + lambda * lambda);
    dS[0] = pre * (c0 + lambda * d0);
    dS[1] = pre * (c1 + lambda * d1);
    dS[2] = pre * (c2 + lambda * d2);
}

static void orc_normalise(double v[3]) {
    double len = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] = v[0] / len;
    v[1] = v[1] / len;
    v[2] = v[2] / len;
}

/* ---------------------------------------------------------------------------------- */
/* Macrocell demagnetising field, readings D1-D5 in the file header.                   */
/* ---------------------------------------------------------------------------------- */

/* Macrocell of every atom (D1): cell[i] in 0..ncell-1.  Returns ncell, or -1 if memory
 * could not be allocated. */
int64_t orc_macrocells(const orc_system *s, int64_t *cell) {
    int64_t n = s->n;
    if (n == 0) return 0;
    double lo[3] = {s->pos[0], s->pos[1], s->pos[2]}, hi[3] = {s->pos[0], s->pos[1], s->pos[2]};
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            if (s->pos[3 * i + a] < lo[a]) lo[a] = s->pos[3 * i + a];
            if (s->pos[3 * i + a] > hi[a]) hi[a] = s->pos[3 * i + a];
        }
    int64_t dim[3];
    for (int a = 0; a < 3; ++a) dim[a] = (int64_t)floor((hi[a] - lo[a]) / s->demag_cell) + 1;
    int64_t ngrid = dim[0] * dim[1] * dim[2];
    int64_t *id = (int64_t *)malloc(sizeof(int64_t) * (size_t)ngrid);
    if (!id) return -1;
    for (int64_t g = 0; g < ngrid; ++g) id[g] = -1;
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3];
        for (int a = 0; a < 3; ++a) c[a] = (int64_t)floor((s->pos[3 * i + a] - lo[a]) / s->demag_cell);
        cell[i] = c[0] + dim[0] * (c[1] + dim[1] * c[2]);
        id[cell[i]] = 0;
    }
    int64_t ncell = 0;
    for (int64_t g = 0; g < ngrid; ++g)
        if (id[g] == 0) id[g] = ncell++;
    for (int64_t i = 0; i < n; ++i) cell[i] = id[cell[i]];
    free(id);
    return ncell;
}

/* Demagnetising field of every atom (tesla, AoS [3n]) for the state S (D2, D3).  If
 * Hmc is not NULL it receives the field of each macrocell [3 ncell].  Returns ncell, or -1
 * if memory could not be allocated. */
int64_t orc_demag_fields(const orc_system *s, const double *S, double *Hd, double *Hmc) {
    int64_t n = s->n;
    int64_t *cell = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!cell) return -1;
    int64_t nc = orc_macrocells(s, cell);
    if (nc < 0) {
        free(cell);
        return -1;
    }
    double *m = (double *)calloc((size_t)(3 * nc + 1), sizeof(double));
    double *p = (double *)calloc((size_t)(3 * nc + 1), sizeof(double));
    double *w = (double *)calloc((size_t)(nc + 1), sizeof(double));
    double *na = (double *)calloc((size_t)(nc + 1), sizeof(double));
    double *H = (double *)calloc((size_t)(3 * nc + 1), sizeof(double));
    if (!m || !p || !w || !na || !H) {
        free(cell); free(m); free(p); free(w); free(na); free(H);
        return -1;
    }
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = cell[i];
        double mu = s->mu_s[i];
        for (int a = 0; a < 3; ++a) {
            m[3 * c + a] += mu * S[3 * i + a];
            p[3 * c + a] += mu * s->pos[3 * i + a];
        }
        w[c] += mu;
        na[c] += 1.0;
    }
    for (int64_t c = 0; c < nc; ++c)
        for (int a = 0; a < 3; ++a) p[3 * c + a] = p[3 * c + a] / w[c];
#pragma omp parallel for schedule(static) num_threads(g_threads)
    for (int64_t a = 0; a < nc; ++a) {
        double hx = 0.0, hy = 0.0, hz = 0.0;
        for (int64_t b = 0; b < nc; ++b) {
            if (b == a) continue;
            double rx = p[3 * b + 0] - p[3 * a + 0];
            double ry = p[3 * b + 1] - p[3 * a + 1];
            double rz = p[3 * b + 2] - p[3 * a + 2];
            double r = sqrt(rx * rx + ry * ry + rz * rz);
            double ux = rx / r, uy = ry / r, uz = rz / r;
            double mdotu = m[3 * b + 0] * ux + m[3 * b + 1] * uy + m[3 * b + 2] * uz;
            double r3 = r * r * r;
            hx += (3.0 * mdotu * ux - m[3 * b + 0]) / r3;
            hy += (3.0 * mdotu * uy - m[3 * b + 1]) / r3;
            hz += (3.0 * mdotu * uz - m[3 * b + 2]) / r3;
        }
        double V = na[a] * s->demag_vatom;
        H[3 * a + 0] = ORC_MU0 / (4.0 * ORC_PI) * hx - ORC_MU0 / 3.0 * m[3 * a + 0] / V;
        H[3 * a + 1] = ORC_MU0 / (4.0 * ORC_PI) * hy - ORC_MU0 / 3.0 * m[3 * a + 1] / V;
        H[3 * a + 2] = ORC_MU0 / (4.0 * ORC_PI) * hz - ORC_MU0 / 3.0 * m[3 * a + 2] / V;
    }
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) Hd[3 * i + a] = H[3 * cell[i] + a];
    if (Hmc) memcpy(Hmc, H, sizeof(double) * 3 * (size_t)nc);
    free(cell); free(m); free(p); free(w); free(na); free(H);
    return nc;
}

/* Thermal field of every site for step `step` at temperature Tn (the thermal-field
 * equation; readings R3, R4, R6): sqrt(2 lambda kB T / (gamma mu_s dt)) times the Gaussian
 * triple of the site. */
static void orc_thermal_field(const orc_system *s, uint32_t step, double Tn, double gamma, double lambda,
                              double *Hth) {
#pragma omp parallel for schedule(static) num_threads(g_threads)
    for (int64_t i = 0; i < s->n; ++i) {
        double g[3];
        orc_thermal_gaussians(s->seed, s->sys, s->ids ? s->ids[i] : (uint32_t)i, step, g);
        double sigma = sqrt(2.0 * lambda * ORC_KB * Tn / (gamma * s->mu_s[i] * s->dt));
        Hth[3 * i + 0] = sigma * g[0];
        Hth[3 * i + 1] = sigma * g[1];
        Hth[3 * i + 2] = sigma * g[2];
    }
}

/*
 * Advance nsteps Heun steps from step index step0.  S [3n] is updated in place.
 * T[k] is the temperature of step step0+k (K).  If rec is not NULL it receives
 * 8 doubles per step: orc_moment_energy of the state at the start of that step.
 * Returns 0, or -1 if memory could not be allocated.
 */
int orc_heun_run(const orc_system *s, double *S, int64_t step0, int64_t nsteps, const double *T, double *rec) {
    int64_t n = s->n;
    double *Hth = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *dS = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *Sp = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    int demag = s->demag_cell > 0.0;
    double *Hd = demag ? (double *)calloc(3 * (size_t)(n > 0 ? n : 1), sizeof(double)) : NULL;
    if (!Hth || !dS || !Sp || (demag && !Hd)) {
        free(Hth); free(dS); free(Sp); free(Hd);
        return -1;
    }
    double gamma = s->gamma > 0.0 ? s->gamma : ORC_GAMMA;
    double lambda = s->alpha;
    for (int64_t k = 0; k < nsteps; ++k) {
        uint32_t step = (uint32_t)(step0 + k);
        double Tn = T[k];
        if (rec) orc_moment_energy(s, S, rec + 8 * k);
        /* demagnetising field from the state at the start of the step (D4) */
        if (demag && (k == 0 || (step0 + k) % (s->demag_every > 0 ? s->demag_every : 1) == 0)) {
            if (orc_demag_fields(s, S, Hd, NULL) < 0) {
                free(Hth); free(dS); free(Sp); free(Hd);
                return -1;
            }
        }
        /* thermal field, drawn once per step (R4) */
        orc_thermal_field(s, step, Tn, gamma, lambda, Hth);
        /* predictor on every spin */
#pragma omp parallel for schedule(static) num_threads(g_threads)
        for (int64_t i = 0; i < n; ++i) {
            double hex[3], H[3];
            orc_site_field(s, S, i, hex, H);
            if (demag) {
                H[0] += Hd[3 * i + 0];
                H[1] += Hd[3 * i + 1];
                H[2] += Hd[3 * i + 2];
            }
            H[0] += Hth[3 * i + 0];
            H[1] += Hth[3 * i + 1];
            H[2] += Hth[3 * i + 2];
            orc_llg(gamma, lambda, S + 3 * i, H, dS + 3 * i);
            double v[3];
            v[0] = S[3 * i + 0] + dS[3 * i + 0] * s->dt;
            v[1] = S[3 * i + 1] + dS[3 * i + 1] * s->dt;
            v[2] = S[3 * i + 2] + dS[3 * i + 2] * s->dt;
            orc_normalise(v);
            Sp[3 * i + 0] = v[0];
            Sp[3 * i + 1] = v[1];
            Sp[3 * i + 2] = v[2];
        }
        /* corrector on every spin, field re-evaluated at S' with the same thermal field */
#pragma omp parallel for schedule(static) num_threads(g_threads)
        for (int64_t i = 0; i < n; ++i) {
            double hex[3], H[3], dSp[3];
            orc_site_field(s, Sp, i, hex, H);
            if (demag) {
                H[0] += Hd[3 * i + 0];
                H[1] += Hd[3 * i + 1];
                H[2] += Hd[3 * i + 2];
            }
            H[0] += Hth[3 * i + 0];
            H[1] += Hth[3 * i + 1];
            H[2] += Hth[3 * i + 2];
            orc_llg(gamma, lambda, Sp + 3 * i, H, dSp);
            double v[3];
            v[0] = S[3 * i + 0] + 0.5 * (dS[3 * i + 0] + dSp[0]) * s->dt;
            v[1] = S[3 * i + 1] + 0.5 * (dS[3 * i + 1] + dSp[1]) * s->dt;
            v[2] = S[3 * i + 2] + 0.5 * (dS[3 * i + 2] + dSp[2]) * s->dt;
            orc_normalise(v);
            /* S_i is only read by site i in this pass, so it can be overwritten here */
            S[3 * i + 0] = v[0];
            S[3 * i + 1] = v[1];
            S[3 * i + 2] = v[2];
        }
    }
    free(Hth); free(dS); free(Sp); free(Hd);
    return 0;
}

/*
 * Advance nsteps midpoint steps (I1-I3) with K = iters fixed-point iterations each, from
 * step index step0; arguments as orc_heun_run.  Returns 0, or -1 on allocation failure.
 */
int orc_midpoint_run(const orc_system *s, double *S, int64_t step0, int64_t nsteps, const double *T, int iters,
                     double *rec) {
    int64_t n = s->n;
    size_t sz = sizeof(double) * 3 * (size_t)(n > 0 ? n : 1);
    double *Hth = (double *)malloc(sz), *X = (double *)malloc(sz), *Y = (double *)malloc(sz);
    double *M = (double *)malloc(sz);
    int demag = s->demag_cell > 0.0;
    int64_t every = s->demag_every > 0 ? s->demag_every : 1;
    double *Hd = demag ? (double *)calloc(3 * (size_t)(n > 0 ? n : 1), sizeof(double)) : NULL;
    if (!Hth || !X || !Y || !M || (demag && !Hd)) {
        free(Hth); free(X); free(Y); free(M); free(Hd);
        return -1;
    }
    double gamma = s->gamma > 0.0 ? s->gamma : ORC_GAMMA;
    double lambda = s->alpha;
    for (int64_t k = 0; k < nsteps; ++k) {
        uint32_t step = (uint32_t)(step0 + k);
        double Tn = T[k];
        if (rec) orc_moment_energy(s, S, rec + 8 * k);
        orc_thermal_field(s, step, Tn, gamma, lambda, Hth);
        /* demagnetising field from the state at the start of the step, held (D4) */
        if (demag && (k == 0 || (step0 + k) % every == 0)) {
            if (orc_demag_fields(s, S, Hd, NULL) < 0) {
                free(Hth); free(X); free(Y); free(M); free(Hd);
                return -1;
            }
        }
        if (demag)
            for (int64_t q = 0; q < 3 * n; ++q) Hth[q] += Hd[q];  /* both are held over the step */
        /* Euler predictor S^(0) = S_n + dt f(S_n) (I2), into X */
#pragma omp parallel for schedule(static) num_threads(g_threads)
        for (int64_t i = 0; i < n; ++i) {
            double hex[3], H[3], d[3];
            orc_site_field(s, S, i, hex, H);
            for (int c = 0; c < 3; ++c) H[c] += Hth[3 * i + c];
            orc_llg(gamma, lambda, S + 3 * i, H, d);
            for (int c = 0; c < 3; ++c) X[3 * i + c] = S[3 * i + c] + d[c] * s->dt;
        }
        /* fixed-point iterations on the midpoint m = (S_n + S^(k))/2 */
        for (int it = 0; it < iters; ++it) {
#pragma omp parallel for schedule(static) num_threads(g_threads)
            for (int64_t i = 0; i < 3 * n; ++i) M[i] = 0.5 * (S[i] + X[i]);
#pragma omp parallel for schedule(static) num_threads(g_threads)
            for (int64_t i = 0; i < n; ++i) {
                double hex[3], H[3], d[3];
                orc_site_field(s, M, i, hex, H);
                for (int c = 0; c < 3; ++c) H[c] += Hth[3 * i + c];
                orc_llg(gamma, lambda, M + 3 * i, H, d);
                for (int c = 0; c < 3; ++c) Y[3 * i + c] = S[3 * i + c] + d[c] * s->dt;
            }
            double *t = X;
            X = Y;
            Y = t;
        }
        memcpy(S, X, sz);
    }
    free(Hth); free(X); free(Y); free(M); free(Hd);
    return 0;
}

/* A(S) of P1 at spin S with field H, and the solution X of X = S_n + (dt/2)(S_n + X) x A (P2). */
static void orc_sib_a(double gamma, double lambda, const double S[3], const double H[3], double A[3]) {
    double g = -gamma / (1.0 + lambda * lambda);
    double sxh0 = S[1] * H[2] - S[2] * H[1];
    double sxh1 = S[2] * H[0] - S[0] * H[2];
    double sxh2 = S[0] * H[1] - S[1] * H[0];
    A[0] = g * (H[0] + lambda * sxh0);
    A[1] = g * (H[1] + lambda * sxh1);
    A[2] = g * (H[2] + lambda * sxh2);
}

static void orc_sib_solve(double dt, const double Sn[3], const double A[3], double X[3]) {
    double b[3] = {0.5 * dt * A[0], 0.5 * dt * A[1], 0.5 * dt * A[2]};
    /* c = S_n + S_n x b */
    double c[3] = {Sn[0] + (Sn[1] * b[2] - Sn[2] * b[1]), Sn[1] + (Sn[2] * b[0] - Sn[0] * b[2]),
                   Sn[2] + (Sn[0] * b[1] - Sn[1] * b[0])};
    double bc = b[0] * c[0] + b[1] * c[1] + b[2] * c[2];
    double bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    double bxc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2], b[0] * c[1] - b[1] * c[0]};
    for (int k = 0; k < 3; ++k) X[k] = (c[k] - bxc[k] + bc * b[k]) / (1.0 + bb);
}

/*
 * Advance nsteps semi-implicit predictor-corrector steps (P1-P3) from step index step0; S [3n]
 * is updated in place, T and rec as orc_heun_run.  Returns 0, or -1 if memory could not be
 * allocated.
 */
int orc_sib_run(const orc_system *s, double *S, int64_t step0, int64_t nsteps, const double *T, double *rec) {
    int64_t n = s->n;
    size_t sz = sizeof(double) * 3 * (size_t)(n > 0 ? n : 1);
    double *Hth = (double *)malloc(sz), *P = (double *)malloc(sz), *M = (double *)malloc(sz);
    double *X = (double *)malloc(sz);
    int demag = s->demag_cell > 0.0;
    int64_t every = s->demag_every > 0 ? s->demag_every : 1;
    double *Hd = demag ? (double *)calloc(3 * (size_t)(n > 0 ? n : 1), sizeof(double)) : NULL;
    if (!Hth || !P || !M || !X || (demag && !Hd)) {
        free(Hth); free(P); free(M); free(X); free(Hd);
        return -1;
    }
    double gamma = s->gamma > 0.0 ? s->gamma : ORC_GAMMA;
    double lambda = s->alpha;
    for (int64_t k = 0; k < nsteps; ++k) {
        uint32_t step = (uint32_t)(step0 + k);
        if (rec) orc_moment_energy(s, S, rec + 8 * k);
        orc_thermal_field(s, step, T[k], gamma, lambda, Hth);
        /* demagnetising field from the state at the start of the step, held (D4) */
        if (demag && (k == 0 || (step0 + k) % every == 0)) {
            if (orc_demag_fields(s, S, Hd, NULL) < 0) {
                free(Hth); free(P); free(M); free(X); free(Hd);
                return -1;
            }
        }
        if (demag)
            for (int64_t q = 0; q < 3 * n; ++q) Hth[q] += Hd[q];  /* both are held over the step */
        /* predictor with A(S_n) */
#pragma omp parallel for schedule(static) num_threads(g_threads)
        for (int64_t i = 0; i < n; ++i) {
            double hex[3], H[3], A[3];
            orc_site_field(s, S, i, hex, H);
            for (int c = 0; c < 3; ++c) H[c] += Hth[3 * i + c];
            orc_sib_a(gamma, lambda, S + 3 * i, H, A);
            orc_sib_solve(s->dt, S + 3 * i, A, P + 3 * i);
        }
#pragma omp parallel for schedule(static) num_threads(g_threads)
        for (int64_t i = 0; i < 3 * n; ++i) M[i] = 0.5 * (S[i] + P[i]);
        /* corrector with A(Sb), Sb = (S_n + S')/2 */
#pragma omp parallel for schedule(static) num_threads(g_threads)
        for (int64_t i = 0; i < n; ++i) {
            double hex[3], H[3], A[3];
            orc_site_field(s, M, i, hex, H);
            for (int c = 0; c < 3; ++c) H[c] += Hth[3 * i + c];
            orc_sib_a(gamma, lambda, M + 3 * i, H, A);
            orc_sib_solve(s->dt, S + 3 * i, A, X + 3 * i);
        }
        memcpy(S, X, sz);
    }
    free(Hth); free(P); free(M); free(X); free(Hd);
    return 0;
}

/* Bulk helpers for statistical tests: Philox blocks of counters (c0+k, c1, c2, c3), and
 * the thermal Gaussians of spins 0..n-1 at one step, both in the definitions above. */
void orc_philox_bulk(const uint32_t ctr0[4], const uint32_t key[2], int64_t count, uint32_t *out) {
    for (int64_t k = 0; k < count; ++k) {
        uint32_t c[4] = {ctr0[0] + (uint32_t)k, ctr0[1], ctr0[2], ctr0[3]};
        orc_philox4x32_10(c, key, out + 4 * k);
    }
}

void orc_gaussians_bulk(uint64_t seed, uint32_t sys, uint32_t step, int64_t n, double *g) {
    for (int64_t i = 0; i < n; ++i) orc_thermal_gaussians(seed, sys, (uint32_t)i, step, g + 3 * i);
}

/* ---------------------------------------------------------------------------------- */
/* Monte Carlo (Section "Monte Carlo Methods"), readings M1-M5 in the file header.     */
/* ---------------------------------------------------------------------------------- */

/* Greedy colouring in site order (M1).  colour[i] receives the colour of site i; the
 * return value is the number of colours, or -1 if memory could not be allocated. */
int orc_colour_greedy(const orc_system *s, int32_t *colour) {
    int64_t n = s->n;
    int32_t ncol = 0;
    int32_t cap = 64;
    int64_t *seen = (int64_t *)malloc(sizeof(int64_t) * (size_t)cap);
    if (!seen) return -1;
    for (int32_t c = 0; c < cap; ++c) seen[c] = -1;
    for (int64_t i = 0; i < n; ++i) {
        /* mark the colours of the neighbours coloured before i */
        for (int64_t k = s->row_ptr[i]; k < s->row_ptr[i + 1]; ++k) {
            int64_t j = s->col[k];
            if (j < i) {
                int32_t c = colour[j];
                if (c >= cap) {
                    int32_t ncap = 2 * c + 2;
                    int64_t *m = (int64_t *)realloc(seen, sizeof(int64_t) * (size_t)ncap);
                    if (!m) {
                        free(seen);
                        return -1;
                    }
                    seen = m;
                    for (int32_t q = cap; q < ncap; ++q) seen[q] = -1;
                    cap = ncap;
                }
                seen[c] = i;
            }
        }
        int32_t c = 0;
        while (c < cap && seen[c] == i) ++c;
        if (c == cap) {
            int32_t ncap = 2 * cap;
            int64_t *m = (int64_t *)realloc(seen, sizeof(int64_t) * (size_t)ncap);
            if (!m) {
                free(seen);
                return -1;
            }
            seen = m;
            for (int32_t q = cap; q < ncap; ++q) seen[q] = -1;
            cap = ncap;
        }
        colour[i] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(seen);
    return ncol;
}

/* Width of the Gaussian trial cone, Eq. MCgaussianSigma. */
double orc_mc_sigma_g(double T) { return 2.0 / 25.0 * pow(ORC_KB * T / ORC_MUB, 0.2); }

/* Energy of site i's terms of the Hamiltonian with its spin set to X (M4):
 * -sum_j J_ij X.S_j - k_u (X.e)^2 - mu_s X.H_app - X^T K X. */
static double orc_site_energy(const orc_system *s, const double *S, int64_t i, const double X[3]) {
    double h[3];
    orc_exchange_sum(s, S, i, h);
    double hx = h[0], hy = h[1], hz = h[2];
    double e = -(X[0] * hx + X[1] * hy + X[2] * hz);
    const double *a = s->easy_axis + 3 * i;
    double xe = X[0] * a[0] + X[1] * a[1] + X[2] * a[2];
    e += -s->k_u[i] * xe * xe;
    if (s->k_c) {
        double x2 = X[0] * X[0], y2 = X[1] * X[1], z2 = X[2] * X[2];
        e += 0.5 * s->k_c[i] * (x2 * x2 + y2 * y2 + z2 * z2);
    }
    e += -s->mu_s[i] * (X[0] * s->H_app[0] + X[1] * s->H_app[1] + X[2] * s->H_app[2]);
    if (s->K_neel) {
        const double *K = s->K_neel + 6 * i;
        double q = K[0] * X[0] * X[0] + K[1] * X[1] * X[1] + K[2] * X[2] * X[2]
                 + 2.0 * (K[3] * X[0] * X[1] + K[4] * X[0] * X[2] + K[5] * X[1] * X[2]);
        e += -q;
    }
    return e;
}

/* One Hinzke-Nowak trial move of site i at Monte Carlo step n and temperature T
 * (Eqs. AMCP, MCgaussian, MCrandom; readings M2-M4).  Returns 1 if accepted. */
static int orc_mc_trial(const orc_system *s, double *S, int64_t i, uint32_t n, double T, double sigma_g) {
    uint32_t spin = s->ids ? s->ids[i] : (uint32_t)i;
    uint32_t key[2] = {(uint32_t)(s->seed & 0xFFFFFFFFu), (uint32_t)(s->seed >> 32)};
    uint32_t ca[4] = {spin, n, s->sys, 2u}, cb[4] = {spin, n, s->sys, 3u};
    uint32_t wa[4], wb[4];
    orc_philox4x32_10(ca, key, wa);
    orc_philox4x32_10(cb, key, wb);
    double g[3];
    orc_box_muller3(wa, g);
    int move = (int)(((uint64_t)wb[0] * 3u) >> 32);
    double u = orc_uniform(wb[1]);
    const double *Si = S + 3 * i;
    double Sn[3];
    if (move == 0) {            /* spin flip */
        Sn[0] = -Si[0];
        Sn[1] = -Si[1];
        Sn[2] = -Si[2];
    } else if (move == 1 && sigma_g == 0.0) {  /* T = 0: a cone of width 0 (M3) */
        Sn[0] = Si[0];
        Sn[1] = Si[1];
        Sn[2] = Si[2];
    } else if (move == 1) {     /* Gaussian move, Eq. MCgaussian */
        Sn[0] = Si[0] + sigma_g * g[0];
        Sn[1] = Si[1] + sigma_g * g[1];
        Sn[2] = Si[2] + sigma_g * g[2];
        orc_normalise(Sn);
    } else {                    /* random move, Eq. MCrandom */
        Sn[0] = g[0];
        Sn[1] = g[1];
        Sn[2] = g[2];
        orc_normalise(Sn);
    }
    double dE = orc_site_energy(s, S, i, Sn) - orc_site_energy(s, S, i, Si);
    int accept = T > 0.0 ? (dE <= -ORC_KB * T * log(u)) : (dE <= 0.0);
    if (accept) {
        S[3 * i + 0] = Sn[0];
        S[3 * i + 1] = Sn[1];
        S[3 * i + 2] = Sn[2];
    }
    return accept;
}

/*
 * Advance nsteps Monte Carlo steps from step index step0 (M1-M5).  colour[i] and ncol
 * come from orc_colour_greedy.  T[k] is the temperature of step step0+k (K).  If rec is
 * not NULL it receives orc_moment_energy of the state at the start of each step; if
 * accepted is not NULL it receives the accepted trial moves of each step.  Returns 0, or
 * -1 if memory could not be allocated.
 */
int orc_mc_run(const orc_system *s, double *S, int64_t step0, int64_t nsteps, const double *T,
               const int32_t *colour, int32_t ncol, double *rec, int64_t *accepted) {
    int64_t n = s->n;
    /* the sites of each colour, in site order */
    int64_t *start = (int64_t *)calloc((size_t)ncol + 1, sizeof(int64_t));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *fill = (int64_t *)calloc((size_t)ncol + 1, sizeof(int64_t));
    if (!start || !order || !fill) {
        free(start); free(order); free(fill);
        return -1;
    }
    for (int64_t i = 0; i < n; ++i) start[colour[i] + 1]++;
    for (int32_t c = 0; c < ncol; ++c) start[c + 1] += start[c];
    for (int64_t i = 0; i < n; ++i) order[start[colour[i]] + fill[colour[i]]++] = i;
    for (int64_t k = 0; k < nsteps; ++k) {
        uint32_t step = (uint32_t)(step0 + k);
        double Tn = T[k];
        double sg = orc_mc_sigma_g(Tn);
        if (rec) orc_moment_energy(s, S, rec + 8 * k);
        int64_t acc = 0;
        for (int32_t c = 0; c < ncol; ++c) {
            /* sites of one colour have no bonds between them: each trial reads only spins of
               other colours, so the loop may run on several threads */
#pragma omp parallel for schedule(static) num_threads(g_threads) reduction(+ : acc)
            for (int64_t q = start[c]; q < start[c + 1]; ++q) acc += orc_mc_trial(s, S, order[q], step, Tn, sg);
        }
        if (accepted) accepted[k] = acc;
    }
    free(start); free(order); free(fill);
    return 0;
}
