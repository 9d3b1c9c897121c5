// Internal structures shared by the host API (ss_api.cu) and the step kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ss {

// Table I of the paper.
constexpr double kBoltzmann = 1.3807e-23;   // J/K
constexpr double kGammaDefault = 1.76e11;   // 1/(T s)
constexpr double kBohrMagneton = 9.2740e-24;  // J/T
constexpr double kMu0 = 4.0e-7 * 3.14159265358979323846;  // vacuum permeability, T m/A

// Sizes of the Box-Muller function tables held in shared memory.
constexpr int kLogTab = 1537;  // centres c_t = (kLogFirst + t)/kLogScale, t = 0..1536: [0.75, 1.5]
constexpr int kLogFirst = 1536;
constexpr int kLogScale = 2048;
constexpr int kLn2Tab = 34;    // 2 n ln 2, n = 0..33, as a multiple of 2^-45 and a remainder
constexpr int kTrigTab = 513;  // (sin, cos) of pi m / 2048, m = 0..512: one octant of a 4096-point circle
constexpr int kLogLo = (kLogTab + 3) / 4;  // double2 slots holding the kLogTab float remainders
// One table buffer of double2: log | ln2 | trig | log remainders (floats, packed four per slot).
constexpr int kTabCount = kLogTab + kLn2Tab + kTrigTab + kLogLo;
// The double-float tables of the FP32-mixed transform (build_ff_tables), in float4 slots after
// the kTabCount double2 slots of the same buffer: log | trig | 2 n ln 2 (two per slot).
constexpr int kFFTabFloat4 = kLogTab + kTrigTab + (kLn2Tab + 1) / 2;
constexpr int kShortRow = 6;   // rows of at most this many bonds take the unrolled exchange sum
constexpr int kPatRow = 12;    // longest row a row pattern holds
constexpr int kMaxPatterns = 65536;  // most row forms kept (and at most half the bonds' worth)
constexpr int kBytePatterns = 256;   // up to this many forms the index is one byte, else two
constexpr int kRecComps = 8;   // record: sum mu S (3), sum mu, E_exc, E_ani, E_app, E_total
constexpr int kPartComps = 8;  // tile partials: sum mu S (3), sum -mu S.h/2, E_ani, 0, 0, 0

// One system of a handle (several when batched).  Lives in device memory; the field and
// temperature entries are rewritten by set_field / set_temperature between launches.
struct SysDesc {
    int64_t offset;      // first spin of the system in the concatenated arrays
    int64_t n;           // spins
    uint32_t key0, key1; // Philox key = (seed low word, seed high word)
    uint32_t ctr2;       // third counter word (system id)
    uint32_t pad;
    int64_t pbase;       // Philox spin index of the system's first spin (a slab's first global
                         // index; 0 otherwise): spin i draws with word i - offset + pbase
    double H[3];         // applied field, T
    double sqrtT;        // square root of the temperature, sqrt(K)
    double msum;         // sum of mu_s over the system, J/T
    float Hf[3];         // H rounded to float (FP32-mixed field arithmetic)
    float sqrtTf;        // sqrtT rounded to float
};

// One material: a distinct (system, mu_s, k_u, easy axis, Neel tensor) combination.
// Per-spin arrays are replaced by a material index per spin; identical sites share an
// entry, so a homogeneous lattice reads one broadcast entry.
template <typename R>
struct MatDesc {
    R inv_mu;     // 1 / mu_s                                      (1/(J/T))
    R ani;        // 2 k_u / mu_s                                  (T)
    R e[3];       // easy axis
    R kf[6];      // (2 / mu_s) K, field tensor of the Neel term    (T)
    R gp;         // gamma / (1 + lambda^2)
    R lambda;     // damping
    R dt;         // time step
    R sig;        // sqrt(2 lambda kB / (gamma mu_s dt)); sigma = sig * sqrt(T)
    R mu;         // mu_s
    R ku;         // k_u
    R K[6];       // Neel tensor (energy)
    R kc;         // cubic anisotropy k_c (energy (k_c/2) sum S^4)
    R kcf;        // -2 k_c / mu_s (field factor of S^3)
    int32_t sys;
    int32_t has_neel;
    int32_t has_cubic;
    int32_t pad;
};

// A contiguous range of spins of one system, processed by one block per pass.
struct TileDesc {
    int64_t start;
    int32_t count;
    int32_t sys;
};

// Everything a step kernel reads or writes.  Passed by value.
template <typename R>
struct KArgs {
    int64_t n;
    const int32_t *row_ptr;   // [n+1]
    const int32_t *col;       // [nnz]
    const R *J;               // [nnz] J_ij / mu_s,i (the exchange field per unit spin, T)
    R J_value;                // the common value when every entry of J is the same
    int J_uniform;            // 1: J is not read, every bond has J_value
    int short_rows;           // 1: no row has more than kShortRow bonds
    const uint8_t *pat;       // [n] row pattern of each spin (uint8, or uint16 when pat_wide), or
                              // nullptr (the CSR is read)
    int pat_wide;             // 1: pat holds uint16 indices (more than 256 forms)
    const int32_t *pat_off;   // [npat][pat_w] column - row of each bond in CSR order, 0 past the
                              // row's end, then the row length at slot pat_w - 2 (short) or
                              // pat_w - 4 (long); 32- or 64-byte aligned rows
    const R *pat_J;           // [npat][pat_w] J_ij / mu_s,i of each bond, 0 past the row's end;
                              // with tensor bonds int32 Jt entries instead (J is not read)
    int pat_w;                // 8: rows of at most kShortRow bonds; 16: at most kPatRow
    MatDesc<R> mat0;          // the only material when mat_uniform is set
    int mat_uniform;          // 1: every spin has material 0 (mat is not read)
    const R *Jt;              // [9 ndict] distinct exchange tensors / mu_s,i, row by row
    const int32_t *Jtidx;     // [nnz] tensor of each bond (J_tensor = 1)
    int J_tensor;             // 1: the exchange sum uses Jt[Jtidx[k]] instead of J
    int any_cubic;            // 1: some material has cubic anisotropy
    int rows_bare;            // 1: the long-row passes write sum_j J_ij X_j alone (no H_app)
    R *ex, *ey, *ez;          // [n] exchange + applied field of the spins being updated, computed
                              // beforehand by k_rows_field (a warp per row), or nullptr
    const uint32_t *sell;     // packed bonds col << 8 | entry of Jd in slices of 32 rows: bond k of
                              // row 32 s + l at sell[sell_off[s] + 32 k + l], padded with J = 0;
                              // or nullptr
    const int64_t *sell_off;  // [nslice + 1]
    int64_t nslice;
    R *x4;                    // [4n] the spins read by the sliced pass, (x, y, z, 0) per spin
    const R *Jd;              // [nJd <= 256] distinct J_ij / mu_s,i of the packed bonds (and 0)
    int nJd;
    const int32_t *mc_of;     // [n] macrocell of each spin (demagnetising field)
    const R *hdx, *hdy, *hdz; // [ncell] demagnetising field of each macrocell (T)
    int demag;                // 1: add the macrocell field to every spin's field
    int64_t ncell;            // macrocells (index bound of mc_of)
    const void *mat;          // [n] material index: uint8 (mat_bytes 1), uint16 (2) or int32 (4)
    int mat_bytes;
    const MatDesc<R> *mats;
    const SysDesc *sys;
    const TileDesc *tiles;
    int64_t ntiles;
    const int32_t *sys_tiles; // [nsys+1] tile range of each system
    int32_t nsys;
    R *sx, *sy, *sz;          // S (state)
    R *px, *py, *pz;          // S' (predictor, renormalised)
    R *qx, *qy, *qz;          // S + dt/2 dS (predictor half step)
    R *hx, *hy, *hz;          // thermal field of the current step
    R *gx, *gy, *gz;          // Gaussians of the next step drawn by the corrector (FP32-mixed);
                              // the split step's Gaussians of even steps
    R *g2x, *g2y, *g2z;       // the split step's Gaussians of odd steps (FP32-mixed)
    unsigned long long *gstep;  // step whose Gaussians the next Gaussian pass writes
    unsigned int *gticket;    // completion counter of the Gaussian pass
    unsigned long long *g_step; // step whose Gaussians gx..gz hold (tile slots >= pre_slot)
    int pre_slot;             // Gaussians of a tile slot (spin k of a tile: slot k / block) are
                              // drawn ahead by the corrector when its rotated index
                              // (slot + warp) mod slots is >= pre_slot; >= slots: none
    int slots;                // tile / block
    double *partials;         // [ntiles * kPartComps]
    double *rec;              // ring [rec_cap][nsys][kRecComps]
    int64_t rec_cap;
    double *cur;              // [nsys][kRecComps] on-demand measurement
    unsigned long long *step; // index of the next step
    const double *sqrtT_sched;
    const float *sqrtT_sched_f;  // the schedule rounded to float
    int64_t sched_len;
    int64_t sched_step0;
    unsigned int *err;        // bit 0: non-finite spin, bit 1: barrier timeout
    unsigned int *ticket;     // completion counter of the corrector launch
    int advance;              // 1: the corrector's last block advances the step counter (0 for a
                              // corrector pass over part of the tiles)
    const double2 *tab;       // Box-Muller tables, kTabCount entries (build_bm_tables)
    const float4 *fftab;      // double-float tables, kFFTabFloat4 entries (build_ff_tables)
    unsigned int *bar_count;  // grid barrier of the persistent kernel
    unsigned int *bar_gen;
    unsigned int bar_extra;   // test hook: phantom blocks the barrier waits for
    long long bar_timeout_ns;
};

// Monte Carlo colour pass (Section "Monte Carlo Methods"): the spins order[c0..c1) of one
// colour class, each given one Hinzke-Nowak trial move.
struct McArgs {
    const int32_t *order;     // spins sorted by colour, then index
    int64_t c0, c1;           // range of this colour class in order
    const double2 *par_sys;   // per system (-kB T, sigma_g) when no schedule is set
    const double2 *par_sched; // per schedule step (-kB T_k, sigma_g(T_k))
    unsigned long long *acc;  // accepted trial moves per system
    // The step's trial randoms drawn beforehand for every spin by k_mc_prep (long-row passes),
    // or nullptr (each trial draws its own): move type, the Gaussian triple in the working type
    // ([3][n]), and the acceptance factor -ln(u)/... as the trial uses it (-1/2 of -2 ln u).
    const uint8_t *pre_move;
    const void *pre_g;
    const double *pre_acc;
    // Record of the state at the start of the step summed in the colour passes (lattices with
    // at most two colour classes): the class's tiles, each a run of order[] within one system
    // whose record terms go to partials[slot]; slots run system by system.
    const TileDesc *tiles;    // tiles of this colour class (start and count in order[])
    const int32_t *slot;      // partial slot of each tile
    int64_t ntiles;
    double *partials;         // [slots * kPartComps]
    int first;                // 1: the first class (its rows' bonds are summed, both ends unchanged)
};

// Macrocell demagnetising field (Section "Demagnetising fields").
struct DemagArgs {
    int64_t ncell;
    const int32_t *cell_start;  // [ncell+1] spins of cell c: cell_spins[cell_start[c] .. cell_start[c+1])
    const int32_t *cell_spins;  // spins sorted by cell, then index
    const int32_t *cell_first;  // [ncell] first macrocell of the cell's system
    const int32_t *cell_end;    // [ncell] one past the last macrocell of the cell's system
    const double *pos;          // [3 ncell] moment-weighted centre of each cell, m
    const double *vol;          // [ncell] effective volume n_atoms V_atom, m^3
    double *m;                  // [3 ncell] moment of each cell, J/T
    double *H;                  // [3 ncell] field of each cell, T
};

constexpr unsigned int kErrNonFinite = 1u;
constexpr unsigned int kErrTimeout = 2u;
constexpr unsigned int kErrBounds = 4u;   // checked builds: an index out of its range was met

// Host helper (ss_api.cu): sets the message returned by ss_last_error(NULL).
void set_global_error(const char *msg);

// Launchers (ss_kernels_f32.cu / ss_kernels_f64.cu).
template <typename R> cudaError_t launch_predictor(const KArgs<R> &a, int block, int grid, cudaStream_t s);
template <typename R> cudaError_t launch_corrector(const KArgs<R> &a, int block, int grid, int nfin, cudaStream_t s);
template <typename R> cudaError_t launch_measure(const KArgs<R> &a, int block, int grid, cudaStream_t s);
// The split FP32-mixed step: the Gaussian pass, then the Heun passes reading it (FP32 only).
template <typename R> cudaError_t launch_gauss(const KArgs<R> &a, int block, int grid, cudaStream_t s, int priority);
template <typename R> cudaError_t launch_gstep_sync(const KArgs<R> &a, cudaStream_t s);
template <typename R> cudaError_t launch_predictor_split(const KArgs<R> &a, int block, int grid, cudaStream_t s);
template <typename R>
cudaError_t launch_corrector_split(const KArgs<R> &a, int block, int grid, int nfin, cudaStream_t s);
// Resident blocks per SM of the split step's kernels (which: 0 Gaussian pass, 1 predictor,
// 2 corrector; mode: the kernel variant).
template <typename R> int split_blocks_per_sm(int block, int mode, int which);
template <typename R> cudaError_t launch_init_sphere(const KArgs<R> &a, cudaStream_t s);
template <typename R> cudaError_t launch_persistent(const KArgs<R> &a, int block, int grid, int nfin,
                                                    long long nsteps, cudaStream_t s);
template <typename R> cudaError_t launch_system_blocks(const KArgs<R> &a, int block, int grid, long long nsteps,
                                                       cudaStream_t s);
template <typename R> int persistent_blocks_per_sm(int block, int mode);
// mode: the step-kernel variant (0 plain, 1 general, 2 rows; kPlain / kGeneral / kRows)
template <typename R> int step_blocks_per_sm(int block, int mode);
template <typename R> int corrector_blocks_per_sm(int block, bool draw_ahead, int mode);
// One colour pass for long exchange rows: a warp sums the rows of 32 trials cooperatively.
template <typename R> cudaError_t launch_mc_colour_warp(const KArgs<R> &a, const McArgs &m, int grid, cudaStream_t s);
// The trial randoms of the device's current step for every spin (McArgs.pre_*).
template <typename R> cudaError_t launch_mc_prep(const KArgs<R> &a, const McArgs &m, cudaStream_t s);
// One colour pass over the tiles of m that also sums the record terms of the pre-step state.
template <typename R> cudaError_t launch_mc_colour_rec(const KArgs<R> &a, const McArgs &m, int grid, cudaStream_t s);
template <typename R> cudaError_t launch_mc_colour(const KArgs<R> &a, const McArgs &m, int block, int grid,
                                                   cudaStream_t s);
template <typename R> int mc_blocks_per_sm(int block, int mode);  // mode: kPlain or kGeneral
cudaError_t launch_advance_step(unsigned long long *step, cudaStream_t s);
template <typename R> cudaError_t launch_demag(const KArgs<R> &a, const DemagArgs &d, cudaStream_t s);
// One midpoint step's launches after its record: Euler predictor, `iters` fixed-point
// iterations, copy back (the step counter is advanced separately).
// (rgrid: grid of the long-row passes, used when a.ex is set)
// (igrid: grid of the fixed-point iterations, at most one resident wave)
template <typename R> cudaError_t launch_midpoint(const KArgs<R> &a, int iters, int grid, int igrid, int rgrid,
                                                  cudaStream_t s);
// One semi-implicit predictor-corrector step's launches after its record (predictor, corrector;
// the step counter is advanced separately).
// (cgrid: grid of the corrector, at most one resident wave)
template <typename R> cudaError_t launch_sib(const KArgs<R> &a, int grid, int cgrid, int rgrid, cudaStream_t s);
// Resident 256-thread blocks per SM of the midpoint iterations (which = 0) or of the
// semi-implicit corrector (which = 1) in the kernel variant `mode`.
template <typename R> int alt_pass_blocks_per_sm(int which, int mode);
// Exchange + applied field of (X, Y, Z) into (a.ex, a.ey, a.ez), a warp per row (long rows).
template <typename R>
cudaError_t launch_rows_field(const KArgs<R> &a, const R *X, const R *Y, const R *Z, int grid, cudaStream_t s);
template <typename R> int rows_blocks_per_sm();
// The record of the current device step (ring entry step % rec_cap).
cudaError_t launch_finalize_ring(const SysDesc *sys, const int32_t *sys_tiles, int nsys, const double *partials,
                                 double *rec, int64_t rec_cap, const unsigned long long *step, cudaStream_t s);
cudaError_t launch_finalize(const SysDesc *sys, const int32_t *sys_tiles, int nsys, const double *partials,
                            double *dst, cudaStream_t s);
cudaError_t launch_debug_philox(const uint32_t *ctr0, const uint32_t *key, long long count, uint32_t *out,
                                cudaStream_t s);
cudaError_t fp64_rate(int mode, double *inst_per_s);
cudaError_t launch_debug_gaussians(uint64_t seed, uint32_t sys, uint32_t step, long long n, int mode,
                                   const double2 *tab, double *out, cudaStream_t s);

// The cluster step of one small system (ss_cluster.cuh): a chunk of m steps advanced by one
// thread-block cluster whose CTAs hold the spins in shared memory.
template <typename R>
struct ClusterArgs {
    R *G;               // [m][3][n] the chunk's thermal fields sigma g (k_cluster_gauss)
    R *T;               // [m][5][n] the per-spin record terms of the chunk's states
    double *partials;   // [m][ntiles][kPartComps] tile partials of the chunk's records
    uint64_t step0;     // first step of the chunk
    int m;              // steps of the chunk
    int span;           // spins per CTA (32 groups)
    int groups;         // groups of 32 spins per CTA (four warps each)
};
constexpr int kClusterChunk = 256;    // steps per cluster launch
constexpr int kClusterMaxGroups = 4;  // groups of 32 spins per CTA (512 threads)
constexpr int kClusterAutoMax = 2048; // largest system the automatic launch mode steps in a cluster
template <typename R> cudaError_t launch_cluster_gauss(const KArgs<R> &a, const ClusterArgs<R> &c, cudaStream_t s);
template <typename R>
cudaError_t launch_cluster_steps(const KArgs<R> &a, const ClusterArgs<R> &c, int ctas, int row_slots, cudaStream_t s);
template <typename R>
cudaError_t launch_cluster_record(const KArgs<R> &a, const ClusterArgs<R> &c, int block, cudaStream_t s);
// Largest cluster the step kernel can be launched with for `groups` groups per CTA (0: none).
template <typename R> int cluster_max_ctas(const KArgs<R> &a, int groups, int row_slots);

// Host (ss_common.cu): fills the kTabCount entries of the Box-Muller tables.
void build_bm_tables(double2 *t);
// Host (ss_common.cu): fills the kFFTabFloat4 entries of the double-float tables.
void build_ff_tables(float4 *t);

}  // namespace ss
