/*
 * spinsys.h -- C ABI of the GB300 stochastic Heun-LLG spin-dynamics library
 * (libspinsys.so).  Plain C types only: host pointers, sizes and opaque handles.
 *
 * The library integrates the stochastic Landau-Lifshitz-Gilbert equation of an atomistic
 * classical Heisenberg spin model (Evans et al., "Atomistic spin model simulations of
 * magnetic nanomaterials", arXiv:1310.6143):
 *
 *   Hamiltonian     H = -sum_{bonds} J_ij S_i.S_j - sum_i k_u (S_i.e_i)^2
 *                       - sum_i mu_s S_i.H_app [- sum_i S_i^T K_i S_i]
 *                   (Eq. spinhamiltonian, Eq. HJij, the uniaxial and applied-field terms;
 *                   each bond of the symmetric neighbour list counted once; the Neel
 *                   surface tensor K_i is an optional extension)
 *   effective field H_eff = -(1/mu_s) dH/dS_i + H_th                    (Eqs. Heff, Heffth)
 *   thermal field   H_th = Gamma sqrt(2 lambda kB T / (gamma mu_s dt))   (Langevin dynamics)
 *   equation        dS/dt = -gamma/(1+lambda^2) [S x H + lambda S x (S x H)]     (Eq. LLG)
 *   integrator      Heun predictor-corrector, |S| renormalised after both passes, the
 *                   thermal field held fixed between them, predictor over all spins
 *                   before any corrector (Section "Time Integration of the LLG Equation").
 *
 * The paper's Mersenne Twister + Ziggurat generator is replaced by Philox4x32-10
 * (Salmon et al., SC'11) with counter (spin index within its system, step, system id, 0)
 * and key (seed low word, seed high word), followed by an FP64 Box-Muller transform:
 * u_k = (w_k + 1/2) 2^-32, gx = sqrt(-2 ln u0) cos(2 pi u1), gy = sqrt(-2 ln u0)
 * sin(2 pi u1), gz = sqrt(-2 ln u2) cos(2 pi u3).  The FP32-mixed form uses exactly that
 * transform's values rounded to float (evaluated in double-float arithmetic with a
 * certified rounding, the rare uncertain roundings by the FP64 transform itself).  Steps
 * are counted modulo 2^32 in the counter.  Constants are those of Table I:
 * gamma = 1.76e11 1/(T s), kB = 1.3807e-23 J/K.
 *
 * Units: SI throughout -- moments J/T, energies J, fields T, temperatures K, time s.
 * Layouts: vectors are array-of-structures on the host (x, y, z per site); Neel tensors
 * are 6 doubles per site (xx, yy, zz, xy, xz, yz).  On the device spins are stored as
 * structure-of-arrays in the working precision.
 *
 * Ownership: every host array passed in is caller-owned and copied during the call.
 * Device memory is owned by the handle and released by spin_system_destroy.  Device
 * pointers returned by get_spins_device stay valid until the next call that changes the
 * state (llg_heun_step, set_spins) or spin_system_destroy.
 *
 * Errors: every call returns an ss_status and never aborts the process.  A message for
 * the last failure of a handle is available from ss_last_error.  After a CUDA error the
 * handle answers SS_ERR_STATE to every call but spin_system_destroy.  Calls on one handle
 * must not run concurrently from several host threads.
 *
 * Streams: all device work of a handle is issued on its stream (a private non-blocking
 * stream unless spin_system_set_stream names another).  Calls that return host data
 * synchronise that stream; llg_heun_step and the set_* calls are asynchronous.
 */
#ifndef SPINSYS_H
#define SPINSYS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ss_system ss_system; /* opaque, library-owned */

typedef enum {
    SS_OK = 0,
    SS_ERR_INVALID_ARG = 1, /* a pointer, size or value is out of range          */
    SS_ERR_CUDA = 2,        /* a CUDA runtime call failed                         */
    SS_ERR_OOM = 3,         /* device or host allocation failed                   */
    SS_ERR_TIMEOUT = 4,     /* a bounded device-side wait ran out                 */
    SS_ERR_NONFINITE = 5,   /* a spin became NaN or infinite                      */
    SS_ERR_STATE = 6,       /* the handle is unusable after an earlier failure    */
    SS_ERR_UNSUPPORTED = 7  /* a valid request the library cannot serve here     */
} ss_status;

typedef enum {
    SS_FP64 = 0,      /* every step in FP64                                          */
    SS_FP32_MIXED = 1 /* FP32 storage, field and LLG arithmetic; FP64 Philox-to-Gaussian
                         transform and FP64 moment/energy sums                        */
} ss_precision;

/* ss_params.flags */
#define SS_FLAG_CHECK_SYMMETRY 1u /* reject a neighbour list with J_ij != J_ji      */
#define SS_FLAG_INIT_RANDOM 2u    /* start from random unit spins drawn from the
                                     reserved Philox stream (counter (i, 0xFFFFFFFF,
                                     system, 1)); S0 is then ignored                 */

typedef struct {
    int64_t n;                /* spins, 1 <= n < 2^31                                  */
    const double *pos;        /* [3n] positions (m) or NULL; validated; kept (with mu_s)
                                 when every system has them, for set_demag              */
    const double *mu_s;       /* [n] atomic moments, J/T, > 0                          */
    const double *k_u;        /* [n] uniaxial anisotropy, J/atom                       */
    const double *easy_axis;  /* [3n] easy axes (normalised on copy) or NULL for +z    */
    const int64_t *row_ptr;   /* [n+1] CSR offsets, row_ptr[0] = 0, non-decreasing,
                                 nnz = row_ptr[n] < 2^31                               */
    const int32_t *col;       /* [nnz] neighbour indices in [0, n), no self bonds      */
    const double *J;          /* [nnz] exchange, J/link; the list holds both j->i and
                                 i->j of each bond (symmetric)                        */
    const double *K_neel;     /* [6n] Neel surface tensors or NULL                     */
    const double *S0;         /* [3n] initial spins or NULL (+z); normalised on copy
                                 unless already of unit length within 1e-6 (FP32-mixed)
                                 or 1e-14 (FP64), so stored states round-trip bitwise */
    double alpha;             /* Gilbert damping lambda, >= 0                          */
    double dt;                /* time step, s, > 0                                     */
    double gamma;             /* gyromagnetic ratio 1/(T s); 0 selects 1.76e11         */
    double H_app[3];          /* initial applied field, T                              */
    double T;                 /* initial temperature, K, >= 0                          */
    uint64_t seed;            /* Philox key                                            */
    uint32_t sys_id;          /* third Philox counter word of this system              */
    ss_precision precision;   /* must be equal for all systems of a batch              */
    uint32_t flags;           /* SS_FLAG_*                                             */
    const double *J_tensor;   /* [9 nnz] exchange tensors (Eqs. HJijM, HJijSMS) or NULL:
                                 bond k (row i -> j = col[k]) carries J_k row by row
                                 (Jxx Jxy Jxz Jyx Jyy Jyz Jzx Jzy Jzz); the field on i is
                                 (1/mu_s,i) sum_k J_k S_j, the energy -1/2 sum_i S_i.(...)
                                 (each bond once); the reverse bond should carry the
                                 transpose (checked with SS_FLAG_CHECK_SYMMETRY).  When
                                 given, J may be NULL and is not used; systems of a batch
                                 without tensors use J times the identity             */
    const double *k_c;        /* [n] cubic anisotropy, J/atom, or NULL: energy
                                 +(k_c/2)(Sx^4+Sy^4+Sz^4) per atom (cubic-anisotropy eq.),
                                 field -(2 k_c/mu_s)(Sx^3, Sy^3, Sz^3)                 */
} ss_params;

/* Execution modes of llg_heun_step (spin_system_set_exec). */
typedef enum {
    SS_EXEC_AUTO = 0,      /* SS_EXEC_CLUSTER for a single system it takes, else
                              graphs for long runs, direct launches for short ones  */
    SS_EXEC_KERNELS = 1,   /* one predictor and one corrector launch per step       */
    SS_EXEC_GRAPH = 2,     /* CUDA graphs of captured step launches                 */
    SS_EXEC_PERSISTENT = 3, /* one cooperative launch runs many steps, with a bounded
                              grid barrier between the Heun passes                  */
    SS_EXEC_SYSTEM_BLOCKS = 4, /* one thread block advances whole systems for many steps
                              with block barriers only (batches of small systems)   */
    SS_EXEC_CLUSTER = 5    /* one small system (at most 2048 spins, rows of at most 12
                              scalar bonds, no demagnetising field) in one thread-block
                              cluster holding the spins in shared memory: chunks of 256
                              steps, their thermal fields drawn beforehand and their
                              records summed afterwards on other SMs, beside the cluster;
                              states and records bitwise those of the other modes     */
} ss_exec;

typedef struct {
    int64_t n;            /* total spins                                              */
    int64_t nnz;          /* total neighbour entries                                  */
    int32_t num_systems;  /* systems in the handle (1 unless batched)                 */
    int32_t num_materials;/* distinct (system, mu_s, k_u, axis, Neel) combinations    */
    int32_t precision;    /* ss_precision                                             */
    int32_t exec;         /* ss_exec currently selected                               */
    int32_t block;        /* threads per block of the step kernels                    */
    int32_t tile;         /* spins per tile (one tile never spans two systems)        */
    int64_t num_tiles;
    int64_t step;         /* index of the next step                                   */
    int64_t record_capacity; /* steps kept in the per-step record ring               */
    int64_t device_bytes; /* device memory held by the handle                         */
    int32_t draw_ahead;   /* eighths of each tile's spins whose next-step Gaussians the
                             corrector draws (FP32-mixed form; see spin_system_set_draw_ahead) */
    int32_t exchange_rows;/* 1: a thread per exchange row; 2: a warp per row; 3: a warp per
                             row reading packed bonds (see spin_system_set_exchange_rows)  */
    int32_t row_patterns; /* row forms the thread-per-row exchange sums read instead of the
                             CSR (see spin_system_set_row_patterns); 0: the CSR is read    */
    int32_t gaussian_pass;/* graph and plain-launch steps: 0 Gaussians drawn in the Heun
                             passes, 1 a Gaussian pass before them, 2 that pass overlapping
                             the previous step (see spin_system_set_gaussian_pass)        */
} ss_info;

/* Create one system.  Validates and copies every array (SS_ERR_INVALID_ARG on bad
 * input: n out of range, non-monotone row_ptr, column out of range, self bond,
 * non-positive mu_s or dt, negative alpha or T, non-finite values, or an asymmetric
 * list when SS_FLAG_CHECK_SYMMETRY is set). */
ss_status spin_system_create(const ss_params *p, ss_system **out);

/* Create one handle holding `count` independent systems (statistical parallelism,
 * Appendix C): each system keeps its own neighbour list, moments, anisotropy, field,
 * temperature, seed and system id, and is advanced exactly as if it were alone.  All
 * systems share one step counter and one precision. */
ss_status spin_batch_create(const ss_params *systems, int32_t count, ss_system **out);

/* Release all device and host memory of the handle (NULL is accepted). */
ss_status spin_system_destroy(ss_system *h);

/* Issue all further work of the handle on this cudaStream_t (NULL = the library's own
 * stream).  The handle synchronises its previous stream first. */
ss_status spin_system_set_stream(ss_system *h, void *cuda_stream);

/* Applied field (T) of system `sys`, or of every system when sys < 0: the H_app of the
 * Zeeman term -sum_i mu_s S_i.H_app of Eq. spinhamiltonian, entering every spin's effective
 * field (Eq. Heff) unchanged.  Asynchronous; SS_ERR_INVALID_ARG for sys >= number of systems
 * or a non-finite component. */
ss_status set_field(ss_system *h, int32_t sys, const double H_app[3]);

/* Temperature (K) of every system; removes any temperature schedule.  T sets the variance
 * 2 lambda kB T / (gamma mu_s dt) of the thermal field of the Langevin-dynamics section
 * (the paper's thermal-field equation, each component a zero-mean Gaussian, drawn once per
 * step and held over both Heun passes).  Asynchronous; SS_ERR_INVALID_ARG for a negative or
 * non-finite T. */
ss_status set_temperature(ss_system *h, double T);

/* Temperatures of systems 0..count-1 (count = number of systems). */
ss_status set_temperature_batch(ss_system *h, const double *T, int32_t count);

/* Temperature schedule shared by all systems: step k uses T_per_step[k - step0] for
 * step0 <= k < step0 + nsteps, T_per_step[0] before and T_per_step[nsteps-1] after.
 * The temperature of a step is taken at its start, t_n = n dt. */
ss_status set_temperature_schedule(ss_system *h, const double *T_per_step, int64_t nsteps, int64_t step0);

/* Advance every system by n >= 0 Heun steps (asynchronous): the stochastic LLG equation
 * (Eq. LLG with the effective field of Eq. Heff plus the thermal field) integrated by the
 * Heun predictor-corrector scheme of the section "Time Integration of the LLG Equation" --
 * predictor S' = norm(S + dt dS(S, H)) over every spin, then corrector
 * S <- norm(S + dt/2 (dS(S, H) + dS(S', H'))) with the same thermal field in H and H'.
 * Each step records the moment and energy of the state at its start (Eq. spinhamiltonian)
 * into the per-step record ring.  SS_ERR_INVALID_ARG for n < 0; a non-finite spin raised
 * on the device is reported as SS_ERR_NONFINITE by the next synchronising call. */
ss_status llg_heun_step(ss_system *h, int64_t n);

/* Advance every system by n >= 0 Monte Carlo steps (asynchronous; Section "Monte Carlo
 * Methods": the Metropolis criterion Eq. AMCP with the Hinzke-Nowak mixture of spin-flip,
 * Gaussian (Eq. MCgaussian, cone width Eq. MCgaussianSigma) and random (Eq. MCrandom)
 * trial moves).  One Monte Carlo step gives every spin exactly one trial move, colour
 * class by colour class of a greedy colouring of the neighbour graph (in site order: each
 * site takes the smallest colour no lower-indexed neighbour holds), so that spins updated
 * together share no bond.  Per (spin i, step n) the trial uses Philox blocks
 * (i, n, system id, 2) for the Gaussian triple and (i, n, system id, 3) for the move type
 * floor(3 w0 / 2^32) (0 flip, 1 Gaussian, 2 random) and the acceptance uniform
 * u = (w1 + 1/2) 2^-32; a move is accepted when dE <= -kB T ln u (at T = 0 when dE <= 0),
 * dE being the change of the spin's Hamiltonian terms.  Temperatures, the schedule, the
 * step counter and the per-step record ring are shared with llg_heun_step: each Monte
 * Carlo step advances the counter by one and records the moment and energy of the state
 * at its start.  The first call builds the colouring (a copy of the neighbour list to the
 * host, one int32 per spin of device memory).  SS_ERR_INVALID_ARG for n < 0. */
ss_status mc_step(ss_system *h, int64_t n);

/* Macrocell demagnetising field (Section "Demagnetising fields"; Eqs. macrocellpos,
 * mc_volume, demag).  Needs the atomic positions (ss_params.pos) of every system.  Each
 * system is divided into cubic macrocells of edge `cell_size` (m) on a grid anchored at its
 * smallest coordinate on each axis; occupied cubes are the macrocells.  A macrocell sits at
 * the moment-weighted mean position of its atoms, has the moment sum_i mu_s,i S_i and the
 * volume n_atoms * atom_volume (atom_volume = V_uc / n_uc, m^3).  Its field is
 * mu0/(4 pi) sum over the other macrocells of the same system of [3 (m.u) u - m] / r^3 minus
 * the self term mu0/3 m_p / V_p (FP64), and it is added to the field of every atom in the
 * cell.  The field is recomputed from the state at the start of every step whose index is a
 * multiple of `every` (and at the first step after set_demag, set_spins or set_step) and held
 * in between; llg_heun_step uses it (mc_step does not); the recorded energies exclude it.
 * cell_size <= 0 switches the field off.  SS_ERR_INVALID_ARG without positions or for
 * atom_volume <= 0 or every < 1.  The all-pairs sum costs O(macrocells^2) per update. */
ss_status set_demag(ss_system *h, double cell_size, double atom_volume, int32_t every);

/* The demagnetising field in force for the next step, per atom (AoS [3n], tesla); computed
 * from the current state first if it is due (synchronous). */
ss_status get_demag_field(ss_system *h, double *out3n);

/* Monte Carlo acceptance of system `sys` since the handle was created: out[0] accepted
 * trial moves, out[1] attempted trial moves (synchronous). */
ss_status get_mc_stats(ss_system *h, int32_t sys, int64_t out[2]);

/* Advance every system by n >= 0 steps of the midpoint rule instead of Heun (asynchronous;
 * the alternative integrator the paper's time-integration section cites):
 * S_{n+1} = S_n + dt f(m), m = (S_n + S_{n+1})/2, f the right-hand side of Eq. LLG with the
 * field of the midpoint spins and the step's thermal field (drawn once per step from the same
 * Philox counters as llg_heun_step, held over the step).  Solved by `iterations` (1..1000)
 * fixed-point iterations from the Euler predictor; nothing is renormalised (the rule keeps
 * |S| when converged; the residual of the iteration shows in |S| - 1).  Shares the step
 * counter, record ring, temperatures and demagnetising field (set_demag: updated at the same
 * steps, held over each step) with llg_heun_step; runs iterations + 3 launches per step (the
 * first also sums the step's record).  SS_ERR_INVALID_ARG for n < 0 or iterations out of
 * range. */
ss_status llg_midpoint_step(ss_system *h, int64_t n, int32_t iterations);

/* Advance every system by n >= 0 steps of the semi-implicit predictor-corrector scheme
 * (asynchronous; the modified predictor-corrector midpoint scheme of Mentink et al. that the
 * paper's time-integration section cites).  With Eq. LLG written as dS/dt = S x A(S),
 * A = -gamma/(1+alpha^2) (H + alpha S x H), the predictor solves
 * S' = S_n + (dt/2)(S_n + S') x A(S_n) and the corrector S_{n+1} = S_n + (dt/2)(S_n + S_{n+1})
 * x A(Sb), Sb = (S_n + S')/2, each in closed form (a rotation of S_n: |S| is kept without
 * renormalisation); H includes the step's thermal field, drawn once per step from the same
 * Philox counters as llg_heun_step and held over the step.  Shares the step counter, record
 * ring, temperatures and demagnetising field (as llg_midpoint_step) with llg_heun_step; 4
 * launches per step (the predictor also sums the step's record), captured in CUDA graphs for
 * runs of whole graphs.  SS_ERR_INVALID_ARG for n < 0. */
ss_status llg_semi_implicit_step(ss_system *h, int64_t n);

/* Copy all spins (concatenated over systems) to out3n [3n], AoS, FP64 (synchronous): the
 * unit vectors S_i of the classical Heisenberg model (Eq. spinhamiltonian), |S_i| = 1 after
 * every Heun step (renormalised as the time-integration section prescribes).
 * out3n is caller-owned; SS_ERR_INVALID_ARG for NULL. */
ss_status get_spins(ss_system *h, double *out3n);

/* Device pointers of the x, y, z spin arrays (SoA, float or double as the precision). */
ss_status get_spins_device(ss_system *h, const void **sx, const void **sy, const void **sz);

/* Magnetisation of the current state of system `sys`: out = (mx, my, mz, |m|) with
 * m = sum_i mu_s,i S_i / sum_i mu_s,i (FP64 sums; synchronous) -- the reduced magnetisation
 * whose time average the paper's m(T) curves (Monte Carlo vs LLG, the Curie-temperature
 * fit) report.  SS_ERR_INVALID_ARG for sys out of range or NULL out. */
ss_status get_magnetisation(ss_system *h, int32_t sys, double out[4]);

/* Energy of the current state of system `sys` (J, FP64 sums, thermal field excluded):
 * out = (total, exchange, anisotropy incl. Neel, applied-field) -- the terms of the
 * Hamiltonian Eq. spinhamiltonian: exchange -1/2 sum_i sum_j J_ij S_i.S_j (Eq. HJij, each
 * bond of the symmetric list once), uniaxial anisotropy -sum_i k_u (S_i.e_i)^2, applied
 * field -sum_i mu_s S_i.H_app.  SS_ERR_INVALID_ARG for sys out of range or NULL out. */
ss_status get_energy(ss_system *h, int32_t sys, double out[4]);

/* Per-step record of steps first_step .. first_step+count-1 (all still in the ring):
 * out[(k * num_systems + s) * 8 + c] with c = (sum mu Sx, sum mu Sy, sum mu Sz,
 * sum mu, E_exchange, E_anisotropy, E_applied, E_total) of the state at the start of
 * step first_step+k.  Synchronous. */
ss_status get_record(ss_system *h, int64_t first_step, int64_t count, double *out);

/* Overwrite all spins from in3n [3n] AoS (normalised on copy as S0 is). */
ss_status set_spins(ss_system *h, const double *in3n);

/* Set the index of the next step (selects the Philox counter and schedule entry). */
ss_status set_step(ss_system *h, int64_t step);
ss_status get_step(ss_system *h, int64_t *step);

/* Select how llg_heun_step launches its work (see ss_exec).  SS_ERR_INVALID_ARG for an unknown
 * mode; SS_ERR_UNSUPPORTED for SS_EXEC_PERSISTENT / SS_EXEC_SYSTEM_BLOCKS with warp-per-row
 * exchange, and for SS_EXEC_CLUSTER when the handle is not one system of at most 2,048 spins
 * with rows of at most 12 scalar bonds and no demagnetising field (the message says which).
 * Every mode gives bitwise the same states; the records too, except SS_EXEC_SYSTEM_BLOCKS,
 * which sums them in another order. */
ss_status spin_system_set_exec(ss_system *h, ss_exec mode);

/* Threads per block (32, 64, 128, 256 or 512) and spins per tile (a multiple of the
 * block size, at most 16 blocks' worth) of the step kernels; rebuilds the tile list.
 * SS_ERR_INVALID_ARG for other values.  Single-warp blocks put each warp of a small system
 * on an SM of its own; a single small system runs faster still in SS_EXEC_CLUSTER (an FP64
 * warp instruction holds its SM sub-partition's pipe about 64 cycles whatever the number of
 * active lanes, so what counts is the FP64 work per warp, which that mode splits up). */
ss_status spin_system_set_launch(ss_system *h, int32_t block, int32_t tile);

/* How the exchange sum of Eq. HJij is split over threads: mode 0 automatic (the default: a
 * warp per row when the rows average at least 24 bonds in the FP32-mixed form or 128 in the
 * FP64 form with packed bonds, 64 or 256 without -- exchange beyond the nearest neighbours,
 * up to the over 1,000 neighbours per atom of the long-ranged exchange the paper's scaling
 * section runs), 1 a thread per row (the step kernels sum their own rows), 2 a warp per row.  With a warp per row, each Heun pass is preceded by a pass that sums the exchange
 * field of every spin into a buffer of 3n values.  For scalar J with at most 255 distinct
 * J_ij / mu_s,i and fewer than 2^24 spins (checked at creation, when the rows average 16 or
 * more bonds) the bonds are stored as packed 32-bit words (neighbour index and dictionary
 * entry, 4 bytes per bond) in slices of 32 consecutive rows, bond k of the slice's rows
 * interleaved and each slice padded to its longest row with zero bonds; lane l of a warp
 * sums row l of its slice in CSR order from H_app, exactly as a thread per row does, so the
 * results are identical to mode 1 (ss_info.exchange_rows = 3).  Otherwise (tensors, more
 * values) each warp sums 32 consecutive rows one by one, its lanes striding over the row's
 * bonds (exchange_rows = 2): only the summation order differs.  The midpoint and
 * semi-implicit steps use the same passes (sums without H_app) before each of their passes;
 * Monte Carlo steps sum each trial's row across a warp (32 trials a warp, or one when a
 * colour class is small).  A warp per row runs with graph or plain launches:
 * spin_system_set_exec refuses the persistent and system-block modes (SS_ERR_UNSUPPORTED),
 * and turning it on resets those to SS_EXEC_AUTO.  SS_ERR_INVALID_ARG for another mode. */
ss_status spin_system_set_exchange_rows(ss_system *h, int32_t mode);

/* Neighbour-list storage read by the thread-per-row exchange sums (Eq. HJij) of the Heun
 * steps, the on-demand measurement and Monte Carlo.  At creation, when the rows take few
 * distinct forms -- a form being a row's length (at most 12) and its (column - row,
 * J_ij/mu_s,i) pairs in CSR order, as on a lattice whose interior rows all look alike and
 * whose boundary rows come in a few kinds (the film: 27 forms; a batch of 256 grains: 6,846) --
 * each spin stores a form index (one byte up to 256 forms, else two) and the forms are kept in
 * tables; the sums then read one or two bytes per spin instead of the row's offsets and
 * columns, and add the same terms in the same order, so the results are identical.  "Few"
 * means at most 65,536 forms and at most one form slot (8 per form for rows of up to 6 bonds,
 * 16 beyond) per two bonds, so that the tables stay well below the CSR's size (the 20 nm
 * core-shell sphere, 76,795 forms, reads the CSR).  on = 1 (the default) uses the forms when they were built, 0 reads the CSR;
 * ss_info.row_patterns gives the number of forms in use (0: CSR).  With tensor bonds (Eq.
 * HJijSMS) a form holds each bond's tensor, as an entry of the handle's tensor dictionary, in
 * place of J_ij/mu_s,i.  SS_ERR_INVALID_ARG for another value. */
ss_status spin_system_set_row_patterns(ss_system *h, int32_t on);

/* FP32-mixed form, thread-per-row exchange, graph and plain-launch execution.  mode 0 (the
 * default; the persistent and system-block modes always work this way): the Heun passes draw
 * the thermal Gaussians themselves.  mode 1: each step runs a pass that writes the step's
 * Gaussians (the transform of ss_debug_gaussians mode 2) for every spin at a non-zero
 * temperature, then the predictor and the corrector, both forming the thermal field
 * sigma_i sqrt(T_n) g from them -- so the field is the same in both passes and the same as in
 * mode 0.  mode 2: as mode 1, with the Gaussian pass of step n+1 running on a second,
 * low-priority stream beside the Heun passes of step n (Gaussians of even and odd steps in two
 * buffers, the pass's step held in its own device counter; the Heun passes then take one block
 * per SM less, leaving room for it).  The transform is pure arithmetic and the Heun passes are
 * memory-bound.  Results do not depend on the mode.  Modes 1 and 2 allocate a second Gaussian
 * buffer (12 bytes per spin) on first use.  SS_ERR_INVALID_ARG for another value. */
ss_status spin_system_set_gaussian_pass(ss_system *h, int32_t mode);

/* FP32-mixed form: the corrector of step n draws the thermal Gaussians of step n+1 for
 * `eighths`/8 of each tile's spins (rounded down to whole blocks), so that their FP64
 * transform overlaps the corrector's memory traffic; the predictor draws the rest.
 * 0..8; the default is 4 when the default tile gives each thread 8 spins, else 6.
 * Results do not depend on it (the same Gaussians are drawn). */
ss_status spin_system_set_draw_ahead(ss_system *h, int32_t eighths);

/* Time the candidate (exec, block, tile, draw-ahead, Gaussian pass) choices on this handle over `trial_steps`
 * steps each, keep the fastest, and write it to *out_info.  The spins and the step
 * counter are restored afterwards, so the trajectory is unchanged.  With the environment
 * variable SPINSYS_AUTOTUNE_CACHE naming a file, a workload tuned before on the same device
 * (same precision, spins, bonds, systems, largest system, exchange-row mode and kernel
 * variant) takes its stored choice without trial runs, and a new result is appended. */
ss_status spin_system_autotune(ss_system *h, int32_t trial_steps, ss_info *out_info);

/* The handle's sizes and current launch settings into *out (caller-owned).  `exec` is the mode
 * selected (SS_EXEC_AUTO stays AUTO: the library picks the cluster step, graphs or plain
 * launches per call).
 * Host-only, no synchronisation; SS_ERR_INVALID_ARG for a NULL out. */
ss_status spin_system_info(ss_system *h, ss_info *out);

/* Advance `nsteps` steps with one predictor and one corrector launch each, timing every
 * launch with CUDA events on the handle's stream.  out_ms receives the mean duration of
 * (predictor, corrector) launches and the mean wall time of one step, in milliseconds; with
 * a warp per exchange row each includes the exchange pass before it.  The steps are real
 * steps: the state and the step counter advance. */
ss_status spin_system_time_kernels(ss_system *h, int32_t nsteps, double out_ms[3]);

/* As spin_system_time_kernels, with the Gaussian pass of the split FP32-mixed step timed on
 * its own: out_ms receives the mean duration of (Gaussian pass, predictor, corrector) launches
 * and the mean wall time of one step (the first is 0 without a Gaussian pass). */
ss_status spin_system_time_passes(ss_system *h, int32_t nsteps, double out_ms[4]);

/* Time `launches` (>= 1) passes of the warp-per-row exchange sum over the current spins
 * (spin_system_set_exchange_rows), CUDA events on the handle's stream; *out_ms receives the
 * mean duration of one pass.  The spins and step counter do not change.  SS_ERR_STATE when
 * the handle sums a thread per row. */
ss_status spin_system_time_rows(ss_system *h, int32_t launches, double *out_ms);

/* Test hook for the bounded grid barrier: when nonzero, the next persistent launches
 * wait for `extra` blocks that do not exist and give up after `timeout_ns`; the step then
 * fails with SS_ERR_TIMEOUT and the handle stays usable. */
ss_status spin_system_set_barrier_test(ss_system *h, int32_t extra, int64_t timeout_ns);

/* Wait for the handle's queued work and report any device-side failure (non-finite
 * spin, barrier timeout) raised since the last check; the flag is then cleared. */
ss_status spin_system_sync(ss_system *h);

/* Diagnostics (synchronous, default device, no handle).  ss_debug_philox writes the
 * Philox4x32-10 blocks of counters (ctr0[0]+k, ctr0[1], ctr0[2], ctr0[3]), k < count,
 * to out[4*count].  ss_debug_gaussians writes the thermal Gaussian triples of spins
 * 0..n-1 at one (seed, system id, step) to out[3n]; mode 0 uses the FP64 form's
 * table-driven FP64 transform, mode 1 CUDA's own log/sqrt/sincospi; modes 2-4 the FP32-mixed
 * form's transform: 2 the float Gaussians its step kernels use (the FP64 transform's values
 * rounded to float), 3 the double-float values before that rounding, 4 a flag (1.0 in the
 * first slot) for draws whose rounding the double-float evaluation could not certify. */
ss_status ss_debug_philox(const uint32_t ctr0[4], const uint32_t key[2], int64_t count, uint32_t *out);
ss_status ss_debug_gaussians(uint64_t seed, uint32_t sys_id, uint32_t step, int64_t n, int32_t mode, double *out);

/* Measured FP64 instruction throughput of the current device (instructions per second)
 * from a probe kernel of eight independent chains per thread: mode 0 DFMA with shared
 * multiplier and addend, mode 1 DFMA with three distinct register operands, mode 2 DADD.
 * The step kernels are bound by this pipe; the benchmark reports it beside the nominal
 * rate.  Synchronous; allocates and frees a small device buffer. */
ss_status ss_debug_fp64_rate(int32_t mode, double *inst_per_s);

/* Test hooks for failure handling (process-wide, thread-safe).  ss_debug_fail_allocations:
 * after `after` (>= 0) more successful device allocations by the handles of this process,
 * every device allocation fails as if the device were out of memory, so the calls that
 * allocate (create, set_demag, the first mc_step, ...) return SS_ERR_OOM; a negative value
 * switches the injection off.  ss_debug_live_bytes: the device bytes currently held by all
 * handles of this process (a failed create holds none). */
ss_status ss_debug_fail_allocations(int64_t after);
int64_t ss_debug_live_bytes(void);

/* ---------------------------------------------------------------------------------
 * Allocation-free stepping.  The paper has no counterpart of this entry point.
 *
 * Some callers cannot call cudaMalloc: code running inside a memory pool or arena that
 * owns all device memory of the process, callers that must not allocate after start-up
 * (real-time loops), or host code that receives device buffers from another runtime.
 * llg_heun_step_noalloc advances one FP64 system whose arrays the caller already holds in
 * device memory, and keeps its working buffers (predictor spins, half steps, thermal field,
 * reduction partials, Box-Muller tables) in one statically sized device array inside the
 * library instead of allocating them.  It never calls cudaMalloc, cudaFree or any allocating
 * library routine.
 *
 * Limits and behaviour:
 *  - n <= SS_NOALLOC_MAX_SPINS (131072); larger systems are rejected with
 *    SS_ERR_INVALID_ARG before any device work.  The static array holds 9.5 MB on every
 *    GPU that loads the library, until the process exits.
 *  - Every call looks up the array's device address on the current device
 *    (cudaGetSymbolAddress, which allocates nothing).  The first call on a device, and any
 *    call that finds the address changed, uploads the function tables with a synchronous
 *    copy.  Other calls are asynchronous on `cuda_stream`.  After cudaDeviceReset (or a
 *    torn-down and recreated context) the array comes back zeroed; if it comes back at the
 *    same address the tables are not uploaded again and the results are wrong: do not use
 *    the entry point after a reset in the same process.
 *  - All calls share the one array, which keeps the last call's contents.  Nothing in it
 *    needs clearing: every word a step reads (predictor spins, half steps, thermal field,
 *    reduction partials) is written earlier in the same step.  Calls whose work overlaps on
 *    the GPU (on different streams or devices sharing no order) race on the array and give
 *    wrong results: order them on one stream.
 *  - step0 + nsteps <= 2^32 - 1: the step index is the 32-bit Philox counter word (larger
 *    values are rejected with SS_ERR_INVALID_ARG).
 *  - Launch failures are checked after the first step's launches and after the last; an
 *    error left pending by earlier, unrelated work in the process is reported (and cleared)
 *    by this call as SS_ERR_CUDA.
 *  - The result equals llg_heun_step on a handle created from the same arrays with
 *    precision SS_FP64 (same Philox stream, same Heun step, same reductions).
 *  - Non-finite spins are not reported by this call; inspect the spins or the record.
 * ------------------------------------------------------------------------------- */
#define SS_NOALLOC_MAX_SPINS 131072

typedef struct {
    int64_t n;               /* spins, 1 <= n <= SS_NOALLOC_MAX_SPINS                   */
    const int32_t *row_ptr;  /* device [n+1] CSR offsets, row_ptr[0] = 0                */
    const int32_t *col;      /* device [nnz] neighbour indices in [0, n)                 */
    const double *J;         /* device [nnz] exchange, J/link                             */
    const double *mu_s;      /* device [n] atomic moments, J/T                            */
    const double *k_u;       /* device [n] uniaxial anisotropy, J                         */
    const double *easy_axis; /* device [3n] unit easy axes, AoS                           */
    double *sx, *sy, *sz;    /* device [n] each: spins, read and overwritten (SoA)        */
    double *record;          /* device [8 * nsteps] per-step record as in get_record, or
                                NULL                                                    */
    double alpha, dt, gamma; /* gamma 0 selects 1.76e11                                   */
    double H_app[3];         /* T                                                         */
    double T;                /* K                                                         */
    uint64_t seed;
    uint32_t sys_id;
    int64_t step0;           /* index of the first step (Philox counter)                  */
} ss_noalloc_step;

ss_status llg_heun_step_noalloc(const ss_noalloc_step *p, int64_t nsteps, void *cuda_stream);

/* ---------------------------------------------------------------------------------
 * Slab decomposition of one system (the paper's parallelisation, Appendix C: each
 * processor owns a geometric slab of the system, sorted into core spins, boundary spins
 * and halo copies of its neighbours' boundary spins, and the halo is passed between
 * processors twice per time step -- after the predictor, before the corrector, and after
 * the corrector, before the next predictor -- while core spins hide the transfer).
 *
 * spin_slab_create makes the handle of slab `slab` (0 <= slab < nslabs) of the system `p`:
 * it owns the contiguous global index range [lo, hi), lo = n slab / nslabs, hi = n (slab+1)
 * / nslabs -- a slab along the slowest index of a lattice numbered plane by plane, as the
 * workloads' lattices are.  Its arrays hold the owned spins first (local index g - lo), then
 * halo copies of every other spin an owned row names, in global order; the owned rows are
 * kept in CSR order with renumbered columns, the halo copies have no rows.  Every owned spin
 * draws its thermal field from the Philox counter of its GLOBAL index, so a decomposed run
 * gives, spin for spin and bit for bit, the states of the undecomposed run once the halos are
 * refreshed as above.  Scalar exchange only (SS_ERR_UNSUPPORTED for tensors); llg_heun_step,
 * Monte Carlo, the alternative integrators, the demagnetising field, warp-per-row exchange,
 * the kernel timers and the autotuner are refused on a slab (SS_ERR_UNSUPPORTED): a slab
 * sums a row per thread and advances by spin_system_heun_pass.
 * Tiles hold owned spins only, those with a halo neighbour (boundary tiles) first.
 * --------------------------------------------------------------------------------- */
typedef struct {
    int64_t lo, hi;          /* owned global index range                               */
    int64_t n_halo;          /* halo copies (local indices hi - lo .. hi - lo + n_halo - 1) */
    int64_t num_runs;        /* maximal runs of consecutive global indices in the halo  */
    int64_t boundary_tiles;  /* tiles 0 .. boundary_tiles-1 hold spins with halo neighbours */
    int64_t num_tiles;
    int32_t nslabs, slab;
} ss_slab_info;

ss_status spin_slab_create(const ss_params *p, int32_t nslabs, int32_t slab, ss_system **out);
ss_status spin_slab_info(ss_system *h, ss_slab_info *out);

/* The halo runs of a slab into out3[3 * num_runs] (cap >= num_runs): (first global index,
 * length, first local index) per run, in global order. */
ss_status spin_slab_halo_runs(ss_system *h, int64_t *out3, int64_t cap);

/* Device pointers of the x, y, z arrays of the state S (which = 0) or of the predictor
 * spins S' (which = 1), SoA in the working precision; valid until spin_system_destroy. */
ss_status get_state_device(ss_system *h, int32_t which, const void **x, const void **y, const void **z);

/* One pass of the Heun step over tiles [tile0, tile0 + ntiles) (asynchronous): pass 0 the
 * predictor, 1 the corrector (S' of the halo must be current), 2 the end of the step (the
 * record of the step's state from every tile's predictor sums, then the step counter
 * advances).  A step is pass 0 over all tiles, a halo refresh of S', pass 1 over all tiles,
 * pass 2, a halo refresh of S -- with the boundary tiles' passes first, so that the halo
 * transfer overlaps the core tiles' passes.  Thread-per-row exchange only; SS_ERR_INVALID_ARG
 * for a bad pass or tile range. */
ss_status spin_system_heun_pass(ss_system *h, int32_t pass, int64_t tile0, int64_t ntiles);

/* Human-readable message of the last failure on this handle ("" if none). */
const char *ss_last_error(ss_system *h);
const char *ss_status_string(ss_status s);

#ifdef __cplusplus
}
#endif

#endif /* SPINSYS_H */
