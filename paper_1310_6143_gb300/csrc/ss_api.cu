// Host implementation of the C ABI declared in include/spinsys.h.
//
// A handle owns the device image of one or more spin systems (concatenated), the working
// buffers of the Heun step, a per-step record ring and the launch state (stream, tile
// list, captured graph).  Everything that touches spins runs in the CUDA kernels of
// ss_kernels_f32.cu / ss_kernels_f64.cu; this file validates, converts and launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/spinsys.h"
#include "ss_internal.h"

using namespace ss;

namespace {
thread_local std::string g_create_error;
}  // namespace

namespace ss {

void set_global_error(const char *msg) { g_create_error = msg; }

}  // namespace ss

namespace {


struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Host-side description of one system after validation.
struct HostSys {
    const ss_params *p;
    int64_t offset;
    int64_t nnz_offset;
};

// Material key: compared bitwise.
struct MatKey {
    int32_t sys;
    int32_t has_neel;
    double v[12];  // mu, ku, e[3], K[6], k_c
    bool operator==(const MatKey &o) const {
        return sys == o.sys && has_neel == o.has_neel && std::memcmp(v, o.v, sizeof(v)) == 0;
    }
};

struct MatKeyHash {
    size_t operator()(const MatKey &k) const {
        uint64_t h = 1469598103934665603ull ^ (uint64_t)(uint32_t)k.sys;
        const unsigned char *b = reinterpret_cast<const unsigned char *>(k.v);
        for (size_t i = 0; i < sizeof(k.v); ++i) h = (h ^ b[i]) * 1099511628211ull;
        return (size_t)h;
    }
};

}  // namespace

struct ss_system {
    int precision = SS_FP64;
    int64_t n = 0, nnz = 0;
    int32_t nsys = 0, nmat = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    int device = 0, sm_count = 0;
    int block = 256, tile = 256;
    int64_t ntiles = 0;
    int exec = SS_EXEC_AUTO;
    int64_t step = 0;
    bool bad = false;
    std::string err;
    std::vector<DevBuf> bufs;
    size_t device_bytes = 0;

    // device arrays
    int32_t *row_ptr = nullptr, *col = nullptr, *sys_tiles = nullptr;
    void *mat = nullptr;   // material index per spin, mat_bytes each (1 up to 256 materials, 2 up to 65,536)
    int mat_bytes = 4;
    void *J = nullptr, *mats = nullptr;
    void *state[12] = {};  // sx sy sz px py pz qx qy qz hx hy hz
    void *ahead[3] = {};   // Gaussians drawn ahead by the corrector (FP32-mixed only)
    int pre_slot = 1 << 30;
    int ahead_q = 6;       // eighths of each tile drawn ahead by the corrector
    bool J_uniform = false;  // every bond has the same J_ij / mu_s,i (J_value)
    bool J_tensor = false;   // bonds carry exchange tensors (Jt dictionary, Jtidx per bond)
    bool any_cubic = false;  // some material has cubic anisotropy
    void *Jt = nullptr;
    int32_t *Jtidx = nullptr;
    double J_value = 0.0;
    bool zero_T = true;    // some temperature in force could be zero (the corrector then
                           // skips drawing those spins ahead)
    SysDesc *sys = nullptr;
    TileDesc *tiles = nullptr;
    double *partials = nullptr, *rec = nullptr, *cur = nullptr, *sched = nullptr;
    float *sched_f = nullptr;
    int64_t rec_cap = 0, sched_len = 0, sched_step0 = 0, sched_cap = 0;
    unsigned long long *ctl = nullptr;  // [0] step, [1] err|ticket, [2] barrier count|gen
    double2 *tab = nullptr;             // Box-Muller tables (build_bm_tables), then the
                                        // double-float tables (build_ff_tables)
    int32_t max_row = 0;                // longest CSR row
    // Row patterns (the CSR stored as one or two bytes per row, see build_patterns)
    uint8_t *pat = nullptr;
    int32_t *pat_off = nullptr;
    void *pat_J = nullptr;              // J of the forms' bonds, or their Jt entries (tensor bonds)
    int32_t npat = 0;                   // 0: no patterns (too many forms, rows too long)
    int32_t pat_w = 8;                  // slots of a pattern row (8 or 16, see KArgs)
    bool pat_wide = false;              // two-byte pattern indices (more than 256 forms)
    bool use_pat = true;                // spin_system_set_row_patterns
    // Slab of a decomposed system (spin_slab_create): the owned spins are the first slab_own
    // of the arrays, the halo copies follow; tiles cover the owned spins, boundary tiles first
    int64_t slab_own = -1;              // -1: not a slab
    int64_t slab_lo = 0, slab_hi = 0;   // owned global index range
    int32_t nslabs = 0, slab_index = 0;
    int64_t slab_boundary_tiles = 0;
    std::vector<int64_t> slab_runs;     // halo runs: (global start, length, local start)
    std::vector<uint8_t> slab_edge;     // owned spin with a neighbour in the halo
    int gauss_mode = 0;                 // spin_system_set_gaussian_pass: 0 fused, 1 split, 2 split
                                        // with the next step's Gaussian pass running concurrently
    void *ahead2[3] = {};               // the split step's Gaussians of odd steps (allocated on use)
    cudaStream_t side = nullptr;        // the concurrent Gaussian passes' stream
    int side_priority = 0;              // their launch priority (the device's lowest)
    cudaEvent_t ev_fork = nullptr, ev_gauss = nullptr, ev_corr = nullptr;
    alignas(16) unsigned char mat0[sizeof(MatDesc<double>)] = {};  // MatDesc<R> of material 0

    std::vector<SysDesc> hsys;
    std::vector<int64_t> sys_offset, sys_n;
    std::vector<double> Tsys;     // temperature of each system when no schedule is set, K
    std::vector<double> sched_T;  // the schedule's temperatures, K

    // Monte Carlo state (built on the first mc_step)
    int32_t *mc_order = nullptr;             // spins sorted by colour, then index
    std::vector<int64_t> mc_cstart;          // colour class c is mc_order[mc_cstart[c] .. mc_cstart[c+1])
    double2 *mc_par = nullptr;               // per system (-kB T, sigma_g)
    double2 *mc_sched = nullptr;             // per schedule step (-kB T_k, sigma_g(T_k))
    int64_t mc_sched_cap = 0;
    bool mc_par_dirty = true;
    unsigned long long *mc_acc = nullptr;    // accepted trial moves per system (device)
    uint8_t *mc_pre_move = nullptr;          // the step's trial randoms for the long-row passes
    void *mc_pre_g = nullptr;                // (k_mc_prep): move type, Gaussians [3][n], acceptance
    double *mc_pre_acc = nullptr;
    // record summed in the colour passes (at most two colour classes): per class its tiles
    // (runs of mc_order within one system) and their partial slots, slots system by system
    bool mc_rec = false;
    TileDesc *mc_tiles[2] = {};
    int32_t *mc_slot[2] = {};
    int64_t mc_ntiles[2] = {};
    int32_t *mc_sys_slots = nullptr;         // [nsys + 1] first slot of each system
    double *mc_partials = nullptr;
    std::vector<int64_t> mc_tried;           // trial moves per system (host count)

    // Macrocell demagnetising field (set_demag)
    std::vector<double> hpos, hmu;           // positions [3n] and moments [n] when given at create
    bool demag_on = false, demag_stale = true;
    double demag_cell = 0.0, demag_vatom = 0.0;
    int64_t demag_every = 1, ncell = 0;
    std::vector<int32_t> hcell_of;           // macrocell of each spin (host copy)
    int32_t *d_cell_of = nullptr, *d_cell_start = nullptr, *d_cell_spins = nullptr, *d_cell_first = nullptr,
            *d_cell_end = nullptr;
    double *d_cpos = nullptr, *d_cvol = nullptr, *d_cm = nullptr, *d_cH = nullptr;
    void *d_hd[3] = {};

    // Long exchange rows: the exchange field summed by a warp per row (k_rows_field) before
    // each step pass, when the rows are long enough (set_rows) or on request
    int rows_req = 0;            // 0 automatic, 1 a thread per row, 2 a warp per row
    bool rows = false;           // a warp per row in force
    uint32_t *sell = nullptr;    // packed bonds col << 8 | dictionary entry, slices of 32 rows
    int64_t *sell_off = nullptr; // [nslice + 1] word offset of each slice
    int64_t nslice = 0;
    void *Jd = nullptr;          // the dictionary of J_ij / mu_s,i (with 0 for the padding)
    int nJd = 0;
    void *x4 = nullptr;          // (x, y, z, 0) copy of the spins the sliced pass reads
    void *E[3] = {};             // field of the spins a pass reads

    // launch state
    int nfin = 1;
    cudaGraphExec_t graph = nullptr;
    cudaGraphExec_t midgraph = nullptr; // captured midpoint (midgraph_iters iterations each) or
                                        // semi-implicit (midgraph_iters = -1) steps
    int midgraph_steps = 0, midgraph_iters = 0;
    bool midgraph_failed = false;
    cudaGraphExec_t mcgraph = nullptr;  // captured Monte Carlo steps
    int mcgraph_steps = 0;
    bool mcgraph_failed = false;
    int graph_steps = 0;
    cudaGraphExec_t pgraph = nullptr;  // captured persistent launch (barrier reset + kernel)
    long long pgraph_steps = 0;
    bool pgraph_failed = false;
    bool graph_failed = false;
    unsigned int bar_extra = 0;
    long long bar_timeout_ns = 2000000000ll;
    long long persist_chunk = 64;  // steps per persistent launch
    // The cluster step of a small single system (SS_EXEC_CLUSTER): geometry and the chunk's
    // Gaussians, record terms and tile partials
    int cl_ctas = 0, cl_groups = 0;   // 0: not set up
    void *cl_G = nullptr, *cl_T = nullptr;  // two chunks each (double-buffered)
    double *cl_part = nullptr;
    int64_t cl_ntiles = 0;            // tiles cl_part was sized for
    cudaStream_t cl_side = nullptr;   // the thermal-field and record passes, beside the cluster
    cudaEvent_t cl_ev[7] = {};        // fields ready (2), chunk done (2), records done (2), start
};

namespace {

ss_status fail(ss_system *h, ss_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) {
        h->err = buf;
    } else {
        g_create_error = buf;
    }
    return s;
}

ss_status cuda_fail(ss_system *h, cudaError_t e, const char *what) {
    if (h) h->bad = true;
    return fail(h, e == cudaErrorMemoryAllocation ? SS_ERR_OOM : SS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SS_CUDA(h, call)                                      \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call); \
    } while (0)

// Allocation-failure injection (ss_debug_fail_allocations): < 0 off, else the successful
// allocations left before every allocation fails; and the bytes held by all handles.
std::atomic<int64_t> g_fail_after{-1};
std::atomic<int64_t> g_live_bytes{0};

cudaError_t dalloc(ss_system *h, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    int64_t left = g_fail_after.load();
    while (left >= 0) {
        if (left == 0) return cudaErrorMemoryAllocation;
        if (g_fail_after.compare_exchange_weak(left, left - 1)) break;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return e;
    h->bufs.push_back({*p, bytes});
    h->device_bytes += bytes;
    g_live_bytes += (int64_t)bytes;
    return cudaSuccess;
}

void dfree(ss_system *h, void *p) {
    for (size_t i = 0; i < h->bufs.size(); ++i) {
        if (h->bufs[i].p == p) {
            cudaFree(p);
            h->device_bytes -= h->bufs[i].bytes;
            g_live_bytes -= (int64_t)h->bufs[i].bytes;
            h->bufs.erase(h->bufs.begin() + (long)i);
            return;
        }
    }
}

size_t real_size(const ss_system *h) { return h->precision == SS_FP32_MIXED ? 4 : 8; }

// Unit vector of v.  A vector already of unit length within `tol` is kept as given, so
// that spins read with get_spins and written back with set_spins round-trip bitwise.
void unit_in(const double *v, double out[3], double tol) {
    const double len = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (std::fabs(len - 1.0) <= tol) {
        out[0] = v[0];
        out[1] = v[1];
        out[2] = v[2];
    } else {
        out[0] = v[0] / len;
        out[1] = v[1] / len;
        out[2] = v[2] / len;
    }
}

double unit_tol(int precision) { return precision == SS_FP32_MIXED ? 1e-6 : 1e-14; }

bool finite3(const double *v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

ss_status validate(const ss_params *p, int idx) {
    if (!p) return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: params is NULL", idx);
    if (p->n < 1 || p->n >= (int64_t(1) << 31))
        return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: n = %lld out of range [1, 2^31)", idx, (long long)p->n);
    if (!p->row_ptr || !p->mu_s || !p->k_u)
        return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: row_ptr, mu_s and k_u are required", idx);
    if (p->precision != SS_FP64 && p->precision != SS_FP32_MIXED)
        return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: unknown precision %d", idx, (int)p->precision);
    const int64_t n = p->n;
    if (p->row_ptr[0] != 0) return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: row_ptr[0] != 0", idx);
    for (int64_t i = 0; i < n; ++i)
        if (p->row_ptr[i + 1] < p->row_ptr[i])
            return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: row_ptr decreases at row %lld", idx, (long long)i);
    const int64_t nnz = p->row_ptr[n];
    if (nnz >= (int64_t(1) << 31)) return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: nnz >= 2^31", idx);
    if (nnz > 0 && (!p->col || (!p->J && !p->J_tensor)))
        return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: col and J (or J_tensor) are required when nnz > 0", idx);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k) {
            const int32_t j = p->col[k];
            if (j < 0 || j >= n)
                return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: col[%lld] = %d out of range", idx, (long long)k, j);
            if (j == i) return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: self bond at row %lld", idx, (long long)i);
            if (p->J_tensor) {
                for (int c = 0; c < 9; ++c)
                    if (!std::isfinite(p->J_tensor[9 * k + c]))
                        return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: J_tensor[%lld] not finite", idx,
                                    (long long)k);
            } else if (!std::isfinite(p->J[k])) {
                return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: J[%lld] not finite", idx, (long long)k);
            }
        }
        if (!(p->mu_s[i] > 0.0) || !std::isfinite(p->mu_s[i]))
            return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: mu_s[%lld] must be finite and > 0", idx, (long long)i);
        if (!std::isfinite(p->k_u[i]))
            return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: k_u[%lld] not finite", idx, (long long)i);
        if (p->k_c && !std::isfinite(p->k_c[i]))
            return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: k_c[%lld] not finite", idx, (long long)i);
        if (p->easy_axis) {
            const double *e = p->easy_axis + 3 * i;
            if (!finite3(e) || e[0] * e[0] + e[1] * e[1] + e[2] * e[2] == 0.0)
                return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: easy_axis[%lld] invalid", idx, (long long)i);
        }
        if (p->K_neel)
            for (int c = 0; c < 6; ++c)
                if (!std::isfinite(p->K_neel[6 * i + c]))
                    return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: K_neel[%lld] not finite", idx, (long long)i);
        if (p->S0 && !(p->flags & SS_FLAG_INIT_RANDOM)) {
            const double *s = p->S0 + 3 * i;
            if (!finite3(s) || s[0] * s[0] + s[1] * s[1] + s[2] * s[2] == 0.0)
                return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: S0[%lld] invalid", idx, (long long)i);
        }
        if (p->pos && !finite3(p->pos + 3 * i))
            return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: pos[%lld] not finite", idx, (long long)i);
    }
    if (!(p->alpha >= 0.0) || !std::isfinite(p->alpha))
        return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: alpha must be finite and >= 0", idx);
    if (!(p->dt > 0.0) || !std::isfinite(p->dt))
        return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: dt must be finite and > 0", idx);
    if (!(p->gamma >= 0.0) || !std::isfinite(p->gamma))
        return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: gamma must be finite and >= 0", idx);
    if (!(p->T >= 0.0) || !std::isfinite(p->T))
        return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: T must be finite and >= 0", idx);
    if (!finite3(p->H_app)) return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: H_app not finite", idx);
    if ((p->flags & SS_FLAG_CHECK_SYMMETRY) && p->J_tensor) {
        // each bond's tensor must be the transpose of its reverse bond's
        std::unordered_map<uint64_t, int64_t> where;
        where.reserve((size_t)nnz);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k)
                where[((uint64_t)i << 32) | (uint32_t)p->col[k]] = k;
        for (const auto &b : where) {
            const uint64_t rev = ((b.first & 0xffffffffull) << 32) | (b.first >> 32);
            auto it = where.find(rev);
            bool ok = it != where.end();
            for (int r = 0; ok && r < 3; ++r)
                for (int c = 0; ok && c < 3; ++c)
                    ok = p->J_tensor[9 * b.second + 3 * r + c] == p->J_tensor[9 * it->second + 3 * c + r];
            if (!ok)
                return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: exchange tensors not transposed at (%llu, %llu)",
                            idx, (unsigned long long)(b.first >> 32), (unsigned long long)(b.first & 0xffffffffull));
        }
    } else if (p->flags & SS_FLAG_CHECK_SYMMETRY) {
        std::unordered_map<uint64_t, double> bonds;
        bonds.reserve((size_t)nnz);
        for (int64_t i = 0; i < n; ++i)
            for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k)
                bonds[((uint64_t)i << 32) | (uint32_t)p->col[k]] += p->J[k];
        for (const auto &b : bonds) {
            const uint64_t rev = ((b.first & 0xffffffffull) << 32) | (b.first >> 32);
            auto it = bonds.find(rev);
            if (it == bonds.end() || it->second != b.second)
                return fail(nullptr, SS_ERR_INVALID_ARG, "system %d: neighbour list not symmetric at (%llu, %llu)",
                            idx, (unsigned long long)(b.first >> 32), (unsigned long long)(b.first & 0xffffffffull));
        }
    }
    return SS_OK;
}

// Function tables of the table-driven FP64 Box-Muller transform, followed by the double-float
// tables of the FP32-mixed transform (16-byte slots both).
void build_tables(std::vector<double2> &t) {
    static_assert(sizeof(float4) == sizeof(double2), "table slots");
    t.resize(kTabCount + kFFTabFloat4);
    build_bm_tables(t.data());
    build_ff_tables(reinterpret_cast<float4 *>(t.data() + kTabCount));
}

// Row patterns: when the rows take few distinct forms -- a form being the row's length and its
// (column - row, J_ij / mu_s,i) pairs in CSR order, as on a lattice whose interior rows all look
// alike and whose boundary rows come in a few kinds -- each spin stores the index of its row's
// form (one byte up to 256 forms: the film has 27; two bytes up to 65,536: a batch of 256
// grains has 6,846) and the forms are kept in tables, so a pass reads one or two bytes per spin
// instead of the row's offsets and columns (27.5 bytes on the film).  The exchange sum is then the CSR sum term for term.  With tensor
// bonds a form holds each bond's tensor entry (tidx, the Jt dictionary index) in place of J.
// Rows longer than kPatRow, or more forms than kMaxPatterns or than half the bonds fill
// (npat W > nnz / 2: the tables would rival the CSR), keep the CSR (npat = 0).
template <typename R>
ss_status build_patterns(ss_system *h, const std::vector<int32_t> &rp, const std::vector<int32_t> &col,
                         const std::vector<R> &J, const std::vector<int32_t> &tidx) {
    h->npat = 0;
    const bool tensor = h->J_tensor;
    if (h->nnz <= 0 || h->max_row > kPatRow) return SS_OK;
    const int NS = h->max_row <= kShortRow ? kShortRow : kPatRow;  // offset slots, then the length
    const int W = NS == kShortRow ? 8 : 16;
    const int64_t n = h->n;
    std::vector<uint16_t> pat((size_t)n);
    const int64_t max_forms = std::min<int64_t>(kMaxPatterns, h->nnz / (2 * W));
    std::vector<int32_t> poff, ptid;
    std::vector<R> pJ;
    std::unordered_map<uint64_t, int32_t> id_of;  // row hash -> pattern (contents verified)
    for (int64_t i = 0; i < n; ++i) {
        const int32_t b = rp[i], len = rp[i + 1] - rp[i];
        uint64_t hsh = 0x9E3779B97F4A7C15ull ^ (uint64_t)len;
        for (int32_t q = 0; q < len; ++q) {
            uint64_t jb = 0;
            if (tensor) jb = (uint64_t)(uint32_t)tidx[(size_t)(b + q)];
            else std::memcpy(&jb, &J[(size_t)(b + q)], sizeof(R));
            const uint64_t v = (uint64_t)(uint32_t)(col[(size_t)(b + q)] - (int32_t)i) * 0xBF58476D1CE4E5B9ull ^ jb;
            hsh = (hsh ^ v) * 0x94D049BB133111EBull;
            hsh ^= hsh >> 31;
        }
        auto it = id_of.find(hsh);
        int32_t id;
        if (it == id_of.end()) {
            if ((int64_t)(poff.size() / W) >= max_forms) return SS_OK;  // too many forms: keep the CSR
            id = (int32_t)(poff.size() / W);
            id_of.emplace(hsh, id);
            poff.resize(poff.size() + W, 0);
            pJ.resize(pJ.size() + W, (R)0);
            if (tensor) ptid.resize(ptid.size() + W, 0);
            for (int32_t q = 0; q < len; ++q) {
                poff[(size_t)id * W + q] = col[(size_t)(b + q)] - (int32_t)i;
                if (tensor) ptid[(size_t)id * W + q] = tidx[(size_t)(b + q)];
                else pJ[(size_t)id * W + q] = J[(size_t)(b + q)];
            }
            poff[(size_t)id * W + NS] = len;
        } else {
            id = it->second;
            bool same = poff[(size_t)id * W + NS] == len;
            for (int32_t q = 0; q < len && same; ++q)
                same = poff[(size_t)id * W + q] == col[(size_t)(b + q)] - (int32_t)i &&
                       (tensor ? ptid[(size_t)id * W + q] == tidx[(size_t)(b + q)]
                               : std::memcmp(&pJ[(size_t)id * W + q], &J[(size_t)(b + q)], sizeof(R)) == 0);
            if (!same) return SS_OK;  // a hash collision: keep the CSR
        }
        pat[(size_t)i] = (uint16_t)id;
    }
    const bool wide = poff.size() / W > (size_t)kBytePatterns;
    std::vector<uint8_t> pat8;
    if (!wide) pat8.assign(pat.begin(), pat.end());
    const void *psrc = wide ? (const void *)pat.data() : (const void *)pat8.data();
    const size_t pbytes = (size_t)n * (wide ? 2 : 1);
    SS_CUDA(h, dalloc(h, (void **)&h->pat, pbytes));
    SS_CUDA(h, dalloc(h, (void **)&h->pat_off, poff.size() * sizeof(int32_t)));
    // tensor bonds: the forms' Jt entries (int32) take the place of J, W of them per form, at the
    // start of each form's W * sizeof(R) bytes
    if (tensor)
        for (size_t f = 0; f < poff.size() / W; ++f)
            std::memcpy(reinterpret_cast<char *>(pJ.data()) + f * W * sizeof(R), &ptid[f * W], W * sizeof(int32_t));
    SS_CUDA(h, dalloc(h, &h->pat_J, pJ.size() * sizeof(R)));
    SS_CUDA(h, cudaMemcpyAsync(h->pat, psrc, pbytes, cudaMemcpyHostToDevice, h->stream));
    SS_CUDA(h, cudaMemcpyAsync(h->pat_off, poff.data(), poff.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                               h->stream));
    SS_CUDA(h, cudaMemcpyAsync(h->pat_J, pJ.data(), pJ.size() * sizeof(R), cudaMemcpyHostToDevice, h->stream));

    SS_CUDA(h, cudaStreamSynchronize(h->stream));  // the host vectors go out of scope
    h->npat = (int32_t)(poff.size() / W);
    h->pat_w = W;
    h->pat_wide = wide;
    return SS_OK;
}

template <typename R>
KArgs<R> make_args(const ss_system *h) {
    KArgs<R> a{};
    a.n = h->n;
    a.row_ptr = h->row_ptr;
    a.col = h->col;
    a.J = static_cast<const R *>(h->J);
    a.J_value = (R)h->J_value;
    a.J_uniform = h->J_uniform ? 1 : 0;
    a.short_rows = h->max_row <= kShortRow ? 1 : 0;
    const bool pat = h->npat > 0 && h->use_pat;
    a.pat = pat ? h->pat : nullptr;
    a.pat_off = pat ? h->pat_off : nullptr;
    a.pat_J = pat ? static_cast<const R *>(h->pat_J) : nullptr;
    a.pat_w = h->pat_w;
    a.pat_wide = h->pat_wide ? 1 : 0;
    a.mat_uniform = h->nmat == 1 ? 1 : 0;
    std::memcpy(&a.mat0, h->mat0, sizeof(MatDesc<R>));
    a.Jt = static_cast<const R *>(h->Jt);
    a.Jtidx = h->Jtidx;
    a.J_tensor = h->J_tensor ? 1 : 0;
    a.any_cubic = h->any_cubic ? 1 : 0;
    a.ex = a.ey = a.ez = nullptr;
    a.rows_bare = 0;
    a.sell = h->sell;
    a.sell_off = h->sell_off;
    a.nslice = h->nslice;
    a.x4 = static_cast<R *>(h->x4);
    a.Jd = static_cast<const R *>(h->Jd);
    a.nJd = h->nJd;
    a.demag = h->demag_on ? 1 : 0;
    a.ncell = h->ncell;
    a.mc_of = h->d_cell_of;
    a.hdx = static_cast<const R *>(h->d_hd[0]);
    a.hdy = static_cast<const R *>(h->d_hd[1]);
    a.hdz = static_cast<const R *>(h->d_hd[2]);
    a.mat = h->mat;
    a.mat_bytes = h->mat_bytes;
    a.mats = static_cast<const MatDesc<R> *>(h->mats);
    a.sys = h->sys;
    a.tiles = h->tiles;
    a.ntiles = h->ntiles;
    a.sys_tiles = h->sys_tiles;
    a.nsys = h->nsys;
    R **s = reinterpret_cast<R **>(const_cast<void **>(h->state));
    a.sx = s[0]; a.sy = s[1]; a.sz = s[2];
    a.px = s[3]; a.py = s[4]; a.pz = s[5];
    a.qx = s[6]; a.qy = s[7]; a.qz = s[8];
    a.hx = s[9]; a.hy = s[10]; a.hz = s[11];
    a.gx = static_cast<R *>(h->ahead[0]);
    a.gy = static_cast<R *>(h->ahead[1]);
    a.gz = static_cast<R *>(h->ahead[2]);
    a.g_step = h->ahead[0] ? h->ctl + 3 : nullptr;
    a.g2x = static_cast<R *>(h->ahead2[0]);
    a.g2y = static_cast<R *>(h->ahead2[1]);
    a.g2z = static_cast<R *>(h->ahead2[2]);
    a.gstep = h->ctl + 4;
    a.gticket = reinterpret_cast<unsigned int *>(h->ctl + 5);
    a.pre_slot = h->pre_slot;
    a.slots = std::max(1, h->tile / h->block);
    a.partials = h->partials;
    a.rec = h->rec;
    a.rec_cap = h->rec_cap;
    a.cur = h->cur;
    a.step = h->ctl;
    a.sqrtT_sched = h->sched;
    a.sqrtT_sched_f = h->sched_f;
    a.sched_len = h->sched_len;
    a.sched_step0 = h->sched_step0;
    a.err = reinterpret_cast<unsigned int *>(h->ctl + 1);
    a.ticket = reinterpret_cast<unsigned int *>(h->ctl + 1) + 1;
    a.advance = 1;
    a.bar_count = reinterpret_cast<unsigned int *>(h->ctl + 2);
    a.bar_gen = reinterpret_cast<unsigned int *>(h->ctl + 2) + 1;
    a.tab = h->tab;
    a.fftab = reinterpret_cast<const float4 *>(h->tab + kTabCount);
    a.bar_extra = h->bar_extra;
    a.bar_timeout_ns = h->bar_timeout_ns;
    return a;
}

// The step passes read the exchange field that k_rows_field sums beforehand (long rows).
template <typename R>
void use_rows(const ss_system *h, KArgs<R> &a) {
    if (!h->rows) return;
    a.ex = static_cast<R *>(h->E[0]);
    a.ey = static_cast<R *>(h->E[1]);
    a.ez = static_cast<R *>(h->E[2]);
}

int rows_grid(const ss_system *h) {
    const int per_sm = h->precision == SS_FP32_MIXED ? rows_blocks_per_sm<float>() : rows_blocks_per_sm<double>();
    const int64_t g = (int64_t)h->sm_count * std::max(per_sm, 1);
    return (int)std::max<int64_t>(1, std::min<int64_t>((h->n + 255) / 256, g));
}

// Forget Gaussians drawn ahead: needed when the tile shape changes (the drawn slots depend
// on it) and when a temperature that could have been zero becomes non-zero (the corrector
// draws only where the next temperature is non-zero).  Gaussians do not depend on spins,
// on the temperature's value or on the step counter itself.
cudaError_t invalidate_ahead(ss_system *h) {
    return cudaMemsetAsync(h->ctl + 3, 0xFF, sizeof(unsigned long long), h->stream);
}

void drop_graph(ss_system *h) {
    if (h->midgraph) cudaGraphExecDestroy(h->midgraph);
    h->midgraph = nullptr;
    h->midgraph_steps = 0;
    if (h->mcgraph) cudaGraphExecDestroy(h->mcgraph);
    h->mcgraph = nullptr;
    h->mcgraph_steps = 0;
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    h->graph_steps = 0;
    if (h->pgraph) cudaGraphExecDestroy(h->pgraph);
    h->pgraph = nullptr;
    h->pgraph_steps = 0;
}

// The Heun step-kernel variant the launchers pick for this handle (0 plain, 1 general, 2 rows,
// 3 plain with a single material).
int step_mode(const ss_system *h) {
    return h->rows ? 2 : (h->J_tensor || h->any_cubic) ? 1 : (h->nmat == 1 ? 3 : 0);
}
// The variant of the kernels that sum their own rows (Monte Carlo, persistent, system blocks).
int own_rows_mode(const ss_system *h) { return (h->J_tensor || h->any_cubic) ? 1 : 0; }

int step_grid(const ss_system *h) {
    const int mode = step_mode(h);
    const int per_sm = h->precision == SS_FP32_MIXED ? step_blocks_per_sm<float>(h->block, mode)
                                                     : step_blocks_per_sm<double>(h->block, mode);
    const int64_t g = (int64_t)h->sm_count * std::max(per_sm, 1);
    return (int)std::max<int64_t>(1, std::min<int64_t>(h->ntiles, g));
}

// One wave of resident corrector blocks (the finalisation blocks come on top).
int corrector_grid(const ss_system *h) {
    const bool ahead = h->ahead[0] != nullptr;
    const int mode = step_mode(h);
    const int per_sm = h->precision == SS_FP32_MIXED ? corrector_blocks_per_sm<float>(h->block, ahead, mode)
                                                     : corrector_blocks_per_sm<double>(h->block, ahead, mode);
    const int64_t g = (int64_t)h->sm_count * std::max(per_sm, 1);
    return (int)std::max<int64_t>(1, std::min<int64_t>(h->ntiles, g));
}

// The split FP32-mixed step (a Gaussian pass before the Heun passes) is used by the graph and
// plain-launch modes of FP32-mixed handles that sum a thread per exchange row.
bool split_step(const ss_system *h) {
    return h->gauss_mode > 0 && h->ahead2[0] && h->precision == SS_FP32_MIXED && !h->rows;
}

// One wave of resident blocks of the split step's kernel `which` (0 Gaussian pass, 1 predictor,
// 2 corrector; the corrector's finalisation blocks come on top).  With the Gaussian pass running
// concurrently (mode 2) the Heun passes take one block per SM less, leaving room for one block
// of the Gaussian pass on every SM.
int split_grid(const ss_system *h, int which) {
    int per_sm = std::max(1, split_blocks_per_sm<float>(h->block, step_mode(h), which));
    if (h->gauss_mode == 2) per_sm = which == 0 ? 1 : std::max(1, per_sm - 1);
    const int64_t g = (int64_t)h->sm_count * per_sm;
    return (int)std::max<int64_t>(1, std::min<int64_t>(h->ntiles, g));
}

int persistent_grid(const ss_system *h) {
    const int mode = own_rows_mode(h) == 0 && h->nmat == 1 ? 3 : own_rows_mode(h);
    const int per_sm = h->precision == SS_FP32_MIXED ? persistent_blocks_per_sm<float>(h->block, mode)
                                                     : persistent_blocks_per_sm<double>(h->block, mode);
    const int64_t g = (int64_t)h->sm_count * per_sm;
    return (int)std::max<int64_t>(0, std::min<int64_t>(h->ntiles, g));
}

template <typename R>
cudaError_t enqueue_steps_kernels(ss_system *h, int64_t n) {
    KArgs<R> a = make_args<R>(h);
    use_rows(h, a);
    if (split_step(h)) {
        const int gg = split_grid(h, 0), gp = split_grid(h, 1), gc = split_grid(h, 2);
        if (n <= 0) return cudaSuccess;
        cudaError_t e = launch_gstep_sync<R>(a, h->stream);
        if (h->gauss_mode == 1) {  // Gaussian pass, predictor, corrector, in order
            for (int64_t k = 0; k < n && e == cudaSuccess; ++k) {
                e = launch_gauss<R>(a, h->block, gg, h->stream, 0);
                if (e == cudaSuccess) e = launch_predictor_split<R>(a, h->block, gp, h->stream);
                if (e == cudaSuccess) e = launch_corrector_split<R>(a, h->block, gc, h->nfin, h->stream);
            }
            return e;
        }
        // Concurrent: the first step's Gaussians on the handle's stream; then the pass of step
        // s + 1 runs on the side stream beside step s's Heun passes, once the corrector of step
        // s - 1 (the last reader of its buffer) is done; the predictor of step s + 1 waits for it.
        {
            const int full = (int)std::max<int64_t>(  // the first pass has the GPU to itself
                1, std::min<int64_t>(h->ntiles, (int64_t)h->sm_count *
                                                    std::max(1, split_blocks_per_sm<float>(h->block, step_mode(h), 0))));
            if (e == cudaSuccess) e = launch_gauss<R>(a, h->block, full, h->stream, 0);
        }
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_fork, h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->ev_fork, 0);
        for (int64_t k = 0; k < n && e == cudaSuccess; ++k) {
            if (k + 1 < n) {
                if (k >= 1) e = cudaStreamWaitEvent(h->side, h->ev_corr, 0);
                if (e == cudaSuccess) e = launch_gauss<R>(a, h->block, gg, h->side, h->side_priority);
                if (e == cudaSuccess) e = cudaEventRecord(h->ev_gauss, h->side);
            }
            if (e == cudaSuccess && k >= 1) e = cudaStreamWaitEvent(h->stream, h->ev_gauss, 0);
            if (e == cudaSuccess) e = launch_predictor_split<R>(a, h->block, gp, h->stream);
            if (e == cudaSuccess) e = launch_corrector_split<R>(a, h->block, gc, h->nfin, h->stream);
            if (e == cudaSuccess) e = cudaEventRecord(h->ev_corr, h->stream);
        }
        // join the side stream (needed when it ran nothing after the fork)
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_fork, h->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_fork, 0);
        return e;
    }
    const int gp = step_grid(h), gc = corrector_grid(h), gr = h->rows ? rows_grid(h) : 0;
    for (int64_t k = 0; k < n; ++k) {
        cudaError_t e = h->rows ? launch_rows_field<R>(a, a.sx, a.sy, a.sz, gr, h->stream) : cudaSuccess;
        if (e == cudaSuccess) e = launch_predictor<R>(a, h->block, gp, h->stream);
        if (e != cudaSuccess) return e;
        if (h->rows) e = launch_rows_field<R>(a, a.px, a.py, a.pz, gr, h->stream);
        if (e == cudaSuccess) e = launch_corrector<R>(a, h->block, gc, h->nfin, h->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template <typename R>
cudaError_t enqueue_persistent(ss_system *h, int64_t n) {
    const KArgs<R> a = make_args<R>(h);
    const int grid = persistent_grid(h);
    if (grid < 1) return cudaErrorCooperativeLaunchTooLarge;
    const int nfin = std::min(h->nsys, grid);
    while (n > 0) {
        const long long k = std::min<long long>(n, h->persist_chunk);
        cudaError_t e = cudaMemsetAsync(h->ctl + 2, 0, sizeof(unsigned long long), h->stream);
        if (e != cudaSuccess) return e;
        e = launch_persistent<R>(a, h->block, grid, nfin, k, h->stream);
        if (e != cudaSuccess) return e;
        n -= k;
    }
    return cudaSuccess;
}

cudaError_t enqueue_kernels(ss_system *h, int64_t n) {
    return h->precision == SS_FP32_MIXED ? enqueue_steps_kernels<float>(h, n) : enqueue_steps_kernels<double>(h, n);
}

template <typename R>
cudaError_t enqueue_system_blocks(ss_system *h, int64_t n) {
    const KArgs<R> a = make_args<R>(h);
    const int per_sm = std::max(1, step_blocks_per_sm<R>(h->block, own_rows_mode(h)));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(h->nsys, (int64_t)h->sm_count * per_sm));
    while (n > 0) {
        const long long k = std::min<long long>(n, 1ll << 20);
        const cudaError_t e = launch_system_blocks<R>(a, h->block, grid, k, h->stream);
        if (e != cudaSuccess) return e;
        n -= k;
    }
    return cudaSuccess;
}

cudaError_t enqueue_sysblocks(ss_system *h, int64_t n) {
    return h->precision == SS_FP32_MIXED ? enqueue_system_blocks<float>(h, n) : enqueue_system_blocks<double>(h, n);
}

cudaError_t enqueue_persist(ss_system *h, int64_t n) {
    return h->precision == SS_FP32_MIXED ? enqueue_persistent<float>(h, n) : enqueue_persistent<double>(h, n);
}

// The cluster step (ss_cluster.cuh) for this handle: why it cannot run, or nullptr.  The
// geometry is the fewest 32-spin groups per CTA whose cluster the device can launch.
template <typename R>
const char *cluster_setup(ss_system *h) {
    if (h->nsys != 1) return "the cluster step takes one system";
    if (h->slab_own >= 0) return "not available on a slab handle";
    if (h->rows || h->J_tensor || h->demag_on)
        return "the cluster step takes a thread-per-row scalar exchange sum and no demagnetising field";
    if (h->max_row > kPatRow) return "the cluster step takes rows of at most 12 bonds";
    if (h->cl_groups == 0) {
        const KArgs<R> a = make_args<R>(h);
        for (int g = 1; g <= kClusterMaxGroups && h->cl_groups == 0; g *= 2) {
            const int64_t ctas = (h->n + 32 * g - 1) / (32 * g);
            if (ctas <= cluster_max_ctas<R>(a, g, h->max_row)) {
                h->cl_groups = g;
                h->cl_ctas = (int)ctas;
            }
        }
        if (h->cl_groups == 0) return "the system does not fit one thread-block cluster";
    }
    const size_t rs = sizeof(R);
    if (!h->cl_G) {
        if (dalloc(h, &h->cl_G, (size_t)2 * kClusterChunk * 3 * h->n * rs) != cudaSuccess ||
            dalloc(h, &h->cl_T, (size_t)2 * kClusterChunk * 5 * h->n * rs) != cudaSuccess)
            return "out of device memory";
    }
    if (!h->cl_side) {
        if (cudaStreamCreateWithFlags(&h->cl_side, cudaStreamNonBlocking) != cudaSuccess) return "no stream";
        for (cudaEvent_t &ev : h->cl_ev)
            if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return "no event";
    }
    if (h->cl_ntiles < h->ntiles) {
        if (h->cl_part) dfree(h, h->cl_part);
        h->cl_part = nullptr;
        h->cl_ntiles = 0;
        if (dalloc(h, (void **)&h->cl_part, (size_t)kClusterChunk * h->ntiles * kPartComps * sizeof(double)) !=
            cudaSuccess)
            return "out of device memory";
        h->cl_ntiles = h->ntiles;
    }
    return nullptr;
}

const char *cluster_ready(ss_system *h) {
    return h->precision == SS_FP32_MIXED ? cluster_setup<float>(h) : cluster_setup<double>(h);
}

// Chunks of kClusterChunk steps.  The cluster advances chunk after chunk on the handle's
// stream; beside it, on other SMs, a second stream draws the thermal fields of the next chunk
// and sums the records of the last one (two buffers of each, handed over by events).
template <typename R>
cudaError_t enqueue_cluster_steps(ss_system *h, int64_t n) {
    const KArgs<R> a = make_args<R>(h);
    const int64_t chunk = std::min<int64_t>(kClusterChunk, h->rec_cap);
    const int64_t nk = (n + chunk - 1) / chunk;
    auto args = [&](int64_t k) {
        ClusterArgs<R> c{};
        c.G = (R *)h->cl_G + (k & 1) * kClusterChunk * 3 * h->n;
        c.T = (R *)h->cl_T + (k & 1) * kClusterChunk * 5 * h->n;
        c.partials = h->cl_part;
        c.span = 32 * h->cl_groups;
        c.groups = h->cl_groups;
        c.step0 = (uint64_t)(h->step + k * chunk);
        c.m = (int)std::min<int64_t>(chunk, n - k * chunk);
        return c;
    };
    cudaEvent_t *eg = h->cl_ev, *ec = h->cl_ev + 2, *er = h->cl_ev + 4;
    cudaStream_t side = h->cl_side;
    cudaError_t e = cudaEventRecord(h->cl_ev[6], h->stream);  // parameters and state written before
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, h->cl_ev[6], 0);
    if (e == cudaSuccess) e = launch_cluster_gauss<R>(a, args(0), side);
    if (e == cudaSuccess) e = cudaEventRecord(eg[0], side);
    for (int64_t k = 0; k < nk && e == cudaSuccess; ++k) {
        const int b = (int)(k & 1), nb = (int)((k + 1) & 1);
        if (k + 1 < nk) {  // the next chunk's thermal fields, once chunk k - 1 has read that buffer
            e = cudaStreamWaitEvent(side, ec[nb], 0);
            if (e == cudaSuccess) e = launch_cluster_gauss<R>(a, args(k + 1), side);
            if (e == cudaSuccess) e = cudaEventRecord(eg[nb], side);
        }
        // chunk k, once its fields are drawn and the records of chunk k - 2 are summed
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, eg[b], 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, er[b], 0);
        if (e == cudaSuccess) e = launch_cluster_steps<R>(a, args(k), h->cl_ctas, h->max_row, h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ec[b], h->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ec[b], 0);
        if (e == cudaSuccess) e = launch_cluster_record<R>(a, args(k), h->block, side);
        if (e == cudaSuccess) e = cudaEventRecord(er[b], side);
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, er[(nk - 1) & 1], 0);  // every record summed
    return e;
}

cudaError_t enqueue_cluster(ss_system *h, int64_t n) {
    return h->precision == SS_FP32_MIXED ? enqueue_cluster_steps<float>(h, n) : enqueue_cluster_steps<double>(h, n);
}

// The persistent launch of `persist_chunk` steps (barrier reset + cooperative kernel),
// captured once into a CUDA graph and replayed.  Returns an error if capture is refused;
// the caller then launches directly.
cudaError_t persistent_graph_run(ss_system *h, int64_t &n) {
    const long long k = h->persist_chunk;
    if (n < k) return cudaSuccess;
    if (!h->pgraph) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        cudaError_t ek = enqueue_persist(h, k);
        e = cudaStreamEndCapture(h->stream, &g);
        if (ek != cudaSuccess || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return ek != cudaSuccess ? ek : e;
        }
        e = cudaGraphInstantiate(&h->pgraph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            h->pgraph = nullptr;
            return e;
        }
        h->pgraph_steps = k;
    }
    while (n >= h->pgraph_steps) {
        cudaError_t e = cudaGraphLaunch(h->pgraph, h->stream);
        if (e != cudaSuccess) return e;
        n -= h->pgraph_steps;
    }
    return cudaSuccess;
}

int graph_len(const ss_system *h) {
    // enough steps per graph that the launch cost is amortised, few enough that capture
    // stays cheap
    return h->n >= (int64_t(1) << 22) ? 8 : 64;
}

cudaError_t ensure_graph(ss_system *h) {
    if (h->graph) return cudaSuccess;
    const int g = graph_len(h);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t ek = enqueue_kernels(h, g);
    e = cudaStreamEndCapture(h->stream, &graph);
    if (ek != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return ek;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(&h->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        h->graph = nullptr;
        return e;
    }
    h->graph_steps = g;
    return cudaSuccess;
}

ss_status check_device_flags(ss_system *h) {
    unsigned long long ctl[3];
    SS_CUDA(h, cudaMemcpyAsync(ctl, h->ctl, sizeof(ctl), cudaMemcpyDeviceToHost, h->stream));
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    const unsigned int err = (unsigned int)(ctl[1] & 0xffffffffull);
    h->step = (int64_t)ctl[0];
    if (err) {
        const unsigned long long zero[3] = {ctl[0], 0ull, 0ull};
        SS_CUDA(h, cudaMemcpyAsync(h->ctl, zero, sizeof(zero), cudaMemcpyHostToDevice, h->stream));
        SS_CUDA(h, cudaStreamSynchronize(h->stream));
        if (err & kErrBounds)
            return fail(h, SS_ERR_STATE, "a kernel met an index out of its range (checked build); step counter at %lld",
                        (long long)h->step);
        if (err & kErrTimeout) {
            SS_CUDA(h, invalidate_ahead(h));  // an aborted launch may have drawn part of a step
            SS_CUDA(h, cudaStreamSynchronize(h->stream));
            return fail(h, SS_ERR_TIMEOUT, "grid barrier of the persistent kernel timed out; step counter at %lld",
                        (long long)h->step);
        }
        return fail(h, SS_ERR_NONFINITE, "a spin became non-finite (NaN/inf or zero length)");
    }
    return SS_OK;
}

ss_status build_tiles(ss_system *h) {
    std::vector<TileDesc> tiles;
    std::vector<int32_t> st(h->nsys + 1);
    for (int s = 0; s < h->nsys; ++s) {
        st[s] = (int32_t)tiles.size();
        for (int64_t b = 0; b < h->sys_n[s]; b += h->tile) {
            TileDesc t;
            t.start = h->sys_offset[s] + b;
            t.count = (int32_t)std::min<int64_t>(h->tile, h->sys_n[s] - b);
            t.sys = s;
            tiles.push_back(t);
        }
    }
    if (h->slab_own >= 0) {  // a slab: the tiles holding spins with halo neighbours first
        std::vector<TileDesc> edge, inner;
        for (const TileDesc &t : tiles) {
            bool e = false;
            for (int32_t k = 0; k < t.count && !e; ++k) e = h->slab_edge[(size_t)(t.start + k)] != 0;
            (e ? edge : inner).push_back(t);
        }
        h->slab_boundary_tiles = (int64_t)edge.size();
        tiles = edge;
        tiles.insert(tiles.end(), inner.begin(), inner.end());
    }
    st[h->nsys] = (int32_t)tiles.size();
    if (h->tiles) dfree(h, h->tiles);
    if (h->sys_tiles) dfree(h, h->sys_tiles);
    if (h->partials) dfree(h, h->partials);
    h->tiles = nullptr;
    h->sys_tiles = nullptr;
    h->partials = nullptr;
    h->ntiles = (int64_t)tiles.size();
    SS_CUDA(h, dalloc(h, (void **)&h->tiles, tiles.size() * sizeof(TileDesc)));
    SS_CUDA(h, dalloc(h, (void **)&h->sys_tiles, st.size() * sizeof(int32_t)));
    SS_CUDA(h, dalloc(h, (void **)&h->partials, tiles.size() * kPartComps * sizeof(double)));
    SS_CUDA(h, cudaMemcpyAsync(h->tiles, tiles.data(), tiles.size() * sizeof(TileDesc), cudaMemcpyHostToDevice,
                               h->stream));
    SS_CUDA(h, cudaMemcpyAsync(h->sys_tiles, st.data(), st.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                               h->stream));
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    h->nfin = std::max(1, std::min(h->nsys, 64));
    const int slots = h->tile / h->block;
    const int ahead = (h->ahead_q * slots) / 8;                // slots the corrector draws ahead
    h->pre_slot = ahead >= 1 ? slots - ahead : 1 << 30;
    SS_CUDA(h, invalidate_ahead(h));
    drop_graph(h);
    return SS_OK;
}

template <typename R>
void fill_material(MatDesc<R> &m, const MatKey &k, const ss_params *p) {
    const double mu = k.v[0], ku = k.v[1];
    const double gamma = p->gamma > 0.0 ? p->gamma : kGammaDefault;
    const double lam = p->alpha;
    std::memset(&m, 0, sizeof(m));
    m.inv_mu = (R)(1.0 / mu);
    m.ani = (R)(2.0 * ku / mu);
    for (int c = 0; c < 3; ++c) m.e[c] = (R)k.v[2 + c];
    for (int c = 0; c < 6; ++c) {
        m.kf[c] = (R)(2.0 / mu * k.v[5 + c]);
        m.K[c] = (R)k.v[5 + c];
    }
    m.gp = (R)(gamma / (1.0 + lam * lam));
    m.lambda = (R)lam;
    m.dt = (R)p->dt;
    m.sig = (R)std::sqrt(2.0 * lam * kBoltzmann / (gamma * mu * p->dt));
    m.mu = (R)mu;
    m.ku = (R)ku;
    m.kc = (R)k.v[11];
    m.kcf = (R)(-2.0 * k.v[11] / mu);
    m.sys = k.sys;
    m.has_neel = k.has_neel;
    m.has_cubic = k.v[11] != 0.0 ? 1 : 0;
}

// Rows averaging this many bonds or more get a warp each for the exchange sum (FP32-mixed,
// without packed slices; see set_rows).
constexpr int64_t kRowsAuto = 64;
// Packed slices are built for rows averaging this many bonds or more.
constexpr int64_t kSellMin = 16;

template <typename R>
ss_status upload_system(ss_system *h, const std::vector<HostSys> &hs) {
    const int64_t n = h->n, nnz = h->nnz;
    // CSR with global indices
    std::vector<int32_t> rp((size_t)n + 1), col((size_t)std::max<int64_t>(nnz, 1));
    std::vector<R> J((size_t)std::max<int64_t>(nnz, 1));
    bool tensor = false;
    for (int s = 0; s < h->nsys; ++s) tensor = tensor || hs[s].p->J_tensor != nullptr;
    std::vector<R> Jt;                                   // distinct tensors, 9 values each
    std::vector<int32_t> Jtidx(tensor ? (size_t)std::max<int64_t>(nnz, 1) : 0);
    std::unordered_map<std::string, int32_t> Jt_id;      // tensor bits -> dictionary entry
    std::vector<int32_t> mat((size_t)n);
    std::vector<MatDesc<R>> mats;
    std::unordered_map<MatKey, int32_t, MatKeyHash> mat_id;
    for (int s = 0; s < h->nsys; ++s) {
        const ss_params *p = hs[s].p;
        const int64_t off = hs[s].offset, noff = hs[s].nnz_offset;
        for (int64_t i = 0; i < p->n; ++i) rp[off + i] = (int32_t)(noff + p->row_ptr[i]);
        // J stored divided by the row's moment: the exchange sum then is the field (tesla)
        for (int64_t i = 0; i < p->n; ++i)
            for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k) {
                col[noff + k] = (int32_t)(off + p->col[k]);
                J[noff + k] = p->J ? (R)(p->J[k] / p->mu_s[i]) : (R)0;
                if (tensor) {  // tensors (or J times the identity) divided by the row's moment,
                               // stored once per distinct value
                    R t[9];
                    for (int c = 0; c < 9; ++c)
                        t[c] = p->J_tensor ? (R)(p->J_tensor[9 * k + c] / p->mu_s[i])
                                           : (c % 4 == 0 ? (R)(p->J[k] / p->mu_s[i]) : (R)0);
                    const std::string key(reinterpret_cast<const char *>(t), sizeof(t));
                    auto it = Jt_id.find(key);
                    int32_t id;
                    if (it == Jt_id.end()) {
                        id = (int32_t)(Jt.size() / 9);
                        Jt_id.emplace(key, id);
                        Jt.insert(Jt.end(), t, t + 9);
                    } else {
                        id = it->second;
                    }
                    Jtidx[(size_t)(noff + k)] = id;
                }
            }
        MatKey last{};
        int32_t last_id = -1;
        for (int64_t i = 0; i < p->n; ++i) {
            MatKey key{};
            key.sys = s;
            key.v[0] = p->mu_s[i];
            key.v[1] = p->k_u[i];
            double e[3] = {0.0, 0.0, 1.0};
            if (p->easy_axis) {
                const double *a = p->easy_axis + 3 * i;
                const double len = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
                e[0] = a[0] / len;
                e[1] = a[1] / len;
                e[2] = a[2] / len;
            }
            for (int c = 0; c < 3; ++c) key.v[2 + c] = e[c];
            if (p->K_neel) {
                bool any = false;
                for (int c = 0; c < 6; ++c) {
                    key.v[5 + c] = p->K_neel[6 * i + c];
                    any = any || key.v[5 + c] != 0.0;
                }
                key.has_neel = any ? 1 : 0;
            }
            key.v[11] = p->k_c ? p->k_c[i] : 0.0;
            int32_t id;
            if (last_id >= 0 && key == last) {
                id = last_id;
            } else {
                auto it = mat_id.find(key);
                if (it == mat_id.end()) {
                    id = (int32_t)mats.size();
                    mat_id.emplace(key, id);
                    MatDesc<R> m;
                    fill_material(m, key, p);
                    mats.push_back(m);
                } else {
                    id = it->second;
                }
                last = key;
                last_id = id;
            }
            mat[off + i] = id;
        }
    }
    rp[n] = (int32_t)nnz;
    h->nmat = (int32_t)mats.size();
    if (!mats.empty()) std::memcpy(h->mat0, &mats[0], sizeof(MatDesc<R>));
    h->max_row = 0;
    for (int64_t i = 0; i < n; ++i) h->max_row = std::max<int32_t>(h->max_row, rp[i + 1] - rp[i]);
    h->any_cubic = false;
    for (const MatDesc<R> &m : mats) h->any_cubic = h->any_cubic || m.has_cubic;
    // Homogeneous exchange (one J_ij / mu_s,i for every bond): the kernels skip the J loads.
    h->J_tensor = tensor;
    if (tensor) {
        if (Jt.empty()) Jt.assign(9, (R)0);
        SS_CUDA(h, dalloc(h, &h->Jt, Jt.size() * sizeof(R)));
        SS_CUDA(h, cudaMemcpyAsync(h->Jt, Jt.data(), Jt.size() * sizeof(R), cudaMemcpyHostToDevice, h->stream));
        SS_CUDA(h, dalloc(h, (void **)&h->Jtidx, Jtidx.size() * sizeof(int32_t)));
        SS_CUDA(h, cudaMemcpyAsync(h->Jtidx, Jtidx.data(), Jtidx.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                   h->stream));
        SS_CUDA(h, cudaStreamSynchronize(h->stream));  // the host vectors go out of scope
    }
    // Packed bonds for rows long enough to go a warp per row: col (< 2^24) and one byte naming
    // the bond's J_ij / mu_s,i in a dictionary of at most 255 values plus 0, stored in slices
    // of 32 rows (bond k of the slice's row l at 32 k + l), each padded to its longest row with
    // J = 0 bonds.
    if (!tensor && nnz >= kSellMin * n && n < (int64_t(1) << 24)) {
        using Bits = typename std::conditional<sizeof(R) == 8, uint64_t, uint32_t>::type;
        constexpr int kSlots = 1024;
        std::vector<Bits> key(kSlots);
        std::vector<int> id(kSlots, -1);
        std::vector<R> dict;
        std::vector<uint8_t> bid((size_t)nnz);
        bool ok = true;
        int zero = -1;
        for (int64_t k = 0; k < nnz && ok; ++k) {
            Bits b;
            std::memcpy(&b, &J[k], sizeof(R));
            uint32_t hsh = (uint32_t)(((uint64_t)b * 0x9E3779B97F4A7C15ull) >> 54);  // 10 bits
            while (id[hsh] >= 0 && key[hsh] != b) hsh = (hsh + 1) & (kSlots - 1);
            if (id[hsh] < 0) {
                if (dict.size() == 255) {
                    ok = false;
                    break;
                }
                key[hsh] = b;
                id[hsh] = (int)dict.size();
                if (b == 0) zero = id[hsh];
                dict.push_back(J[k]);
            }
            bid[(size_t)k] = (uint8_t)id[hsh];
        }
        if (ok) {
            if (zero < 0) {
                zero = (int)dict.size();
                dict.push_back((R)0);
            }
            const int64_t nsl = (n + 31) / 32;
            std::vector<int64_t> off((size_t)nsl + 1, 0);
            for (int64_t s = 0; s < nsl; ++s) {
                int32_t w = 0;
                for (int64_t i = 32 * s; i < std::min<int64_t>(n, 32 * s + 32); ++i) w = std::max(w, rp[i + 1] - rp[i]);
                off[(size_t)s + 1] = off[(size_t)s] + 32 * (int64_t)w;
            }
            std::vector<uint32_t> sell((size_t)std::max<int64_t>(off[(size_t)nsl], 1));
            for (int64_t s = 0; s < nsl; ++s) {
                const int64_t w = (off[(size_t)s + 1] - off[(size_t)s]) / 32;
                for (int l = 0; l < 32; ++l) {
                    const int64_t i = 32 * s + l;
                    const int64_t len = i < n ? rp[i + 1] - rp[i] : 0;
                    const uint32_t pad = ((uint32_t)(i < n ? i : 0) << 8) | (uint32_t)zero;
                    for (int64_t k = 0; k < w; ++k)
                        sell[(size_t)(off[(size_t)s] + 32 * k + l)] =
                            k < len ? ((uint32_t)col[rp[i] + k] << 8) | bid[(size_t)(rp[i] + k)] : pad;
                }
            }
            SS_CUDA(h, dalloc(h, &h->Jd, dict.size() * sizeof(R)));
            SS_CUDA(h, dalloc(h, (void **)&h->sell, sell.size() * sizeof(uint32_t)));
            SS_CUDA(h, dalloc(h, (void **)&h->sell_off, off.size() * sizeof(int64_t)));
            SS_CUDA(h, cudaMemcpyAsync(h->Jd, dict.data(), dict.size() * sizeof(R), cudaMemcpyHostToDevice, h->stream));
            SS_CUDA(h, cudaMemcpyAsync(h->sell, sell.data(), sell.size() * sizeof(uint32_t), cudaMemcpyHostToDevice,
                                       h->stream));
            SS_CUDA(h, cudaMemcpyAsync(h->sell_off, off.data(), off.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                                       h->stream));
            SS_CUDA(h, cudaStreamSynchronize(h->stream));
            h->nJd = (int)dict.size();
            h->nslice = nsl;
        }
    }
    h->J_uniform = nnz > 0 && !tensor;
    for (int64_t k = 1; k < nnz && h->J_uniform; ++k) h->J_uniform = std::memcmp(&J[k], &J[0], sizeof(R)) == 0;
    h->J_value = nnz > 0 ? (double)J[0] : 0.0;
    const size_t rs = sizeof(R);
    SS_CUDA(h, dalloc(h, (void **)&h->row_ptr, rp.size() * sizeof(int32_t)));
    SS_CUDA(h, dalloc(h, (void **)&h->col, col.size() * sizeof(int32_t)));
    SS_CUDA(h, dalloc(h, &h->J, J.size() * rs));
    h->mat_bytes = mats.size() <= 256 ? 1 : (mats.size() <= 65536 ? 2 : 4);
    std::vector<uint8_t> mat_packed(mat.size() * (size_t)h->mat_bytes);
    for (size_t k = 0; k < mat.size(); ++k) {
        if (h->mat_bytes == 1) mat_packed[k] = (uint8_t)mat[k];
        else if (h->mat_bytes == 2) reinterpret_cast<uint16_t *>(mat_packed.data())[k] = (uint16_t)mat[k];
        else reinterpret_cast<int32_t *>(mat_packed.data())[k] = mat[k];
    }
    SS_CUDA(h, dalloc(h, (void **)&h->mat, mat_packed.size()));
    SS_CUDA(h, dalloc(h, &h->mats, mats.size() * sizeof(MatDesc<R>)));
    SS_CUDA(h, cudaMemcpyAsync(h->row_ptr, rp.data(), rp.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    SS_CUDA(h, cudaMemcpyAsync(h->col, col.data(), col.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    SS_CUDA(h, cudaMemcpyAsync(h->J, J.data(), J.size() * rs, cudaMemcpyHostToDevice, h->stream));
    SS_CUDA(h, cudaMemcpyAsync(h->mat, mat_packed.data(), mat_packed.size(), cudaMemcpyHostToDevice, h->stream));
    SS_CUDA(h, cudaMemcpyAsync(h->mats, mats.data(), mats.size() * sizeof(MatDesc<R>), cudaMemcpyHostToDevice,
                               h->stream));
    {
        const ss_status ps = build_patterns<R>(h, rp, col, J, Jtidx);
        if (ps != SS_OK) return ps;
    }
    for (int b = 0; b < 12; ++b) SS_CUDA(h, dalloc(h, &h->state[b], (size_t)n * rs));
    if (h->precision == SS_FP32_MIXED)
        for (int b = 0; b < 3; ++b) SS_CUDA(h, dalloc(h, &h->ahead[b], (size_t)n * rs));
    // initial spins
    std::vector<R> s0((size_t)n), s1((size_t)n), s2((size_t)n);
    for (int s = 0; s < h->nsys; ++s) {
        const ss_params *p = hs[s].p;
        const int64_t off = hs[s].offset;
        for (int64_t i = 0; i < p->n; ++i) {
            double v[3] = {0.0, 0.0, 1.0};
            if (p->S0 && !(p->flags & SS_FLAG_INIT_RANDOM)) unit_in(p->S0 + 3 * i, v, unit_tol(h->precision));
            s0[off + i] = (R)v[0];
            s1[off + i] = (R)v[1];
            s2[off + i] = (R)v[2];
        }
    }
    SS_CUDA(h, cudaMemcpyAsync(h->state[0], s0.data(), (size_t)n * rs, cudaMemcpyHostToDevice, h->stream));
    SS_CUDA(h, cudaMemcpyAsync(h->state[1], s1.data(), (size_t)n * rs, cudaMemcpyHostToDevice, h->stream));
    SS_CUDA(h, cudaMemcpyAsync(h->state[2], s2.data(), (size_t)n * rs, cudaMemcpyHostToDevice, h->stream));
    for (int b = 3; b < 12; ++b) SS_CUDA(h, cudaMemsetAsync(h->state[b], 0, (size_t)n * rs, h->stream));
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    return SS_OK;
}

template <typename R>
ss_status init_random(ss_system *h, const std::vector<HostSys> &hs) {
    // random start for the systems that asked for it: draw for all, then restore the others
    bool any = false;
    for (const auto &x : hs) any = any || (x.p->flags & SS_FLAG_INIT_RANDOM);
    if (!any) return SS_OK;
    const size_t rs = sizeof(R);
    const int64_t n = h->n;
    std::vector<R> keep(3 * (size_t)n);
    for (int c = 0; c < 3; ++c)
        SS_CUDA(h, cudaMemcpyAsync(keep.data() + c * n, h->state[c], (size_t)n * rs, cudaMemcpyDeviceToHost, h->stream));
    SS_CUDA(h, launch_init_sphere<R>(make_args<R>(h), h->stream));
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    for (const auto &x : hs) {
        if (x.p->flags & SS_FLAG_INIT_RANDOM) continue;
        for (int c = 0; c < 3; ++c)
            SS_CUDA(h, cudaMemcpyAsync((char *)h->state[c] + x.offset * rs, keep.data() + c * n + x.offset,
                                       (size_t)x.p->n * rs, cudaMemcpyHostToDevice, h->stream));
    }
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    return SS_OK;
}

// A warp per row for the exchange sums (mode 2), a thread per row (1), or the automatic
// choice (0): a warp per row when rows average at least 24 bonds (FP32-mixed) or 128 (FP64)
// with packed slices, 64 or 256 without (measured crossovers on GB300).
ss_status set_rows(ss_system *h, int32_t mode) {
    const bool packed = h->sell != nullptr;
    const int64_t thr = h->precision == SS_FP32_MIXED ? (packed ? 24 : kRowsAuto) : (packed ? 128 : 256);
    const bool on = mode == 2 || (mode == 0 && h->n > 0 && h->nnz >= thr * h->n);
    if (on && !h->E[0]) {
        const size_t rs = real_size(h);
        for (int c = 0; c < 3; ++c) SS_CUDA(h, dalloc(h, &h->E[c], (size_t)h->n * rs));
        if (h->sell) SS_CUDA(h, dalloc(h, &h->x4, 4 * (size_t)h->n * rs));
    }
    h->rows_req = mode;
    if (on != h->rows) drop_graph(h);
    h->rows = on;
    if (on && (h->exec == SS_EXEC_PERSISTENT || h->exec == SS_EXEC_SYSTEM_BLOCKS || h->exec == SS_EXEC_CLUSTER))
        h->exec = SS_EXEC_AUTO;
    return SS_OK;
}

// A slab's owned range and Philox base, passed from spin_slab_create to create_impl.
struct SlabInit {
    int64_t n_own;                   // owned spins (the first n_own of the local arrays)
    int64_t pbase;                   // global index of the first owned spin
    const std::vector<uint8_t> *edge;  // [n_own] owned spins with a halo neighbour
};

ss_status create_impl(const ss_params *systems, int32_t count, ss_system **out, const SlabInit *slab = nullptr) {
    if (!out) return fail(nullptr, SS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!systems || count < 1) return fail(nullptr, SS_ERR_INVALID_ARG, "need at least one system");
    std::vector<HostSys> hs((size_t)count);
    int64_t n = 0, nnz = 0;
    for (int s = 0; s < count; ++s) {
        ss_status st = validate(systems + s, s);
        if (st != SS_OK) return st;
        if (systems[s].precision != systems[0].precision)
            return fail(nullptr, SS_ERR_INVALID_ARG, "all systems of a batch must share one precision");
        hs[s].p = systems + s;
        hs[s].offset = n;
        hs[s].nnz_offset = nnz;
        n += systems[s].n;
        nnz += systems[s].row_ptr[systems[s].n];
    }
    if (n >= (int64_t(1) << 31) || nnz >= (int64_t(1) << 31))
        return fail(nullptr, SS_ERR_INVALID_ARG, "total spins and total neighbour entries must be < 2^31");

    ss_system *h = new (std::nothrow) ss_system();
    if (!h) return fail(nullptr, SS_ERR_OOM, "host allocation failed");
    h->precision = systems[0].precision;
    h->n = n;
    h->nnz = nnz;
    h->nsys = count;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        ss_status st = fail(nullptr, e == cudaErrorNoDevice ? SS_ERR_UNSUPPORTED : SS_ERR_CUDA, "CUDA: %s",
                            cudaGetErrorString(e));
        delete h;
        return st;
    }
    h->stream = h->own_stream;
    bool all_pos = true;
    for (int s = 0; s < count; ++s) {
        h->sys_offset.push_back(hs[s].offset);
        h->sys_n.push_back(slab ? slab->n_own : systems[s].n);  // a slab integrates its owned spins
        all_pos = all_pos && systems[s].pos != nullptr;
    }
    if (slab) {
        h->slab_own = slab->n_own;
        h->slab_edge = *slab->edge;
    }
    if (all_pos) {  // kept for the macrocell demagnetising field
        for (int s = 0; s < count; ++s) {
            h->hpos.insert(h->hpos.end(), systems[s].pos, systems[s].pos + 3 * systems[s].n);
            h->hmu.insert(h->hmu.end(), systems[s].mu_s, systems[s].mu_s + systems[s].n);
        }
    }
    // system table
    h->hsys.resize((size_t)count);
    for (int s = 0; s < count; ++s) {
        const ss_params *p = systems + s;
        SysDesc &d = h->hsys[s];
        std::memset(&d, 0, sizeof(d));
        d.offset = hs[s].offset;
        d.n = slab ? slab->n_own : p->n;
        d.pbase = slab ? slab->pbase : 0;
        d.key0 = (uint32_t)(p->seed & 0xffffffffull);
        d.key1 = (uint32_t)(p->seed >> 32);
        d.ctr2 = p->sys_id;
        for (int c = 0; c < 3; ++c) {
            d.H[c] = p->H_app[c];
            d.Hf[c] = (float)p->H_app[c];
        }
        d.sqrtT = std::sqrt(p->T);
        d.sqrtTf = (float)d.sqrtT;
        h->Tsys.push_back(p->T);
        double ms = 0.0;
        for (int64_t i = 0; i < d.n; ++i) ms += p->mu_s[i];
        d.msum = ms;
    }
    auto cleanup = [&](ss_status st) {
        std::string msg = h->err;
        spin_system_destroy(h);
        g_create_error = msg;
        return st;
    };
    ss_status st;
    if ((e = dalloc(h, (void **)&h->sys, (size_t)count * sizeof(SysDesc))) != cudaSuccess)
        return cleanup(cuda_fail(h, e, "cudaMalloc"));
    if ((e = cudaMemcpyAsync(h->sys, h->hsys.data(), (size_t)count * sizeof(SysDesc), cudaMemcpyHostToDevice,
                             h->stream)) != cudaSuccess)
        return cleanup(cuda_fail(h, e, "cudaMemcpyAsync"));
    // control words, tables, record ring, current measurement
    if ((e = dalloc(h, (void **)&h->ctl, 6 * sizeof(unsigned long long))) != cudaSuccess)
        return cleanup(cuda_fail(h, e, "cudaMalloc"));
    if ((e = cudaMemsetAsync(h->ctl, 0, 6 * sizeof(unsigned long long), h->stream)) != cudaSuccess)
        return cleanup(cuda_fail(h, e, "cudaMemsetAsync"));
    std::vector<double2> tab;
    build_tables(tab);
    if ((e = dalloc(h, (void **)&h->tab, tab.size() * sizeof(double2))) != cudaSuccess)
        return cleanup(cuda_fail(h, e, "cudaMalloc"));
    if ((e = cudaMemcpyAsync(h->tab, tab.data(), tab.size() * sizeof(double2), cudaMemcpyHostToDevice, h->stream)) !=
        cudaSuccess)
        return cleanup(cuda_fail(h, e, "cudaMemcpyAsync"));
    h->rec_cap = std::max<int64_t>(16, std::min<int64_t>(4096, (int64_t(1) << 22) / ((int64_t)count * kRecComps)));
    if ((e = dalloc(h, (void **)&h->rec, (size_t)h->rec_cap * count * kRecComps * sizeof(double))) != cudaSuccess)
        return cleanup(cuda_fail(h, e, "cudaMalloc"));
    if ((e = cudaMemsetAsync(h->rec, 0, (size_t)h->rec_cap * count * kRecComps * sizeof(double), h->stream)) !=
        cudaSuccess)
        return cleanup(cuda_fail(h, e, "cudaMemsetAsync"));
    if ((e = dalloc(h, (void **)&h->cur, (size_t)count * kRecComps * sizeof(double))) != cudaSuccess)
        return cleanup(cuda_fail(h, e, "cudaMalloc"));
    st = h->precision == SS_FP32_MIXED ? upload_system<float>(h, hs) : upload_system<double>(h, hs);
    if (st != SS_OK) return cleanup(st);
    // Launch shape: 512-thread blocks for large systems; spins per thread (a power of two,
    // at most 8) chosen so that there are about eight tiles per resident block.
    h->block = n >= (int64_t(1) << 22) ? 512 : 256;
    {
        int64_t spt = n / ((int64_t)std::max(h->sm_count, 1) * 8 * h->block);
        int slots = 1;
        while (slots < 8 && 2 * slots <= spt) slots *= 2;
        h->tile = slots * h->block;
        h->ahead_q = slots >= 8 ? 4 : 6;  // the faster split on GB300 for each case
        if (slab) h->ahead_q = 0;         // a slab's passes draw their own Gaussians
    }
    st = build_tiles(h);
    if (st == SS_OK) st = set_rows(h, slab ? 1 : 0);  // a slab's passes sum a row per thread
    if (st != SS_OK) return cleanup(st);
    st = h->precision == SS_FP32_MIXED ? init_random<float>(h, hs) : init_random<double>(h, hs);
    if (st != SS_OK) return cleanup(st);
    *out = h;
    return SS_OK;
}

ss_status usable(ss_system *h) {
    if (!h) return fail(nullptr, SS_ERR_INVALID_ARG, "handle is NULL");
    if (h->bad) return fail(h, SS_ERR_STATE, "handle unusable after an earlier CUDA error: %s", h->err.c_str());
    return SS_OK;
}

template <typename R>
ss_status measure(ss_system *h) {
    KArgs<R> a = make_args<R>(h);
    use_rows(h, a);
    if (h->rows) SS_CUDA(h, launch_rows_field<R>(a, a.sx, a.sy, a.sz, rows_grid(h), h->stream));
    SS_CUDA(h, launch_measure<R>(a, h->block, step_grid(h), h->stream));
    SS_CUDA(h, launch_finalize(h->sys, h->sys_tiles, h->nsys, h->partials, h->cur, h->stream));
    return SS_OK;
}

ss_status current_record(ss_system *h, int32_t sys, double rec[kRecComps]) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (sys < 0 || sys >= h->nsys) return fail(h, SS_ERR_INVALID_ARG, "system %d out of range", sys);
    st = h->precision == SS_FP32_MIXED ? measure<float>(h) : measure<double>(h);
    if (st != SS_OK) return st;
    SS_CUDA(h, cudaMemcpyAsync(rec, h->cur + (int64_t)sys * kRecComps, kRecComps * sizeof(double),
                               cudaMemcpyDeviceToHost, h->stream));
    return check_device_flags(h);
}

template <typename R>
ss_status time_kernels_impl(ss_system *h, int32_t nsteps, double out_ms[4]) {
    KArgs<R> a = make_args<R>(h);
    use_rows(h, a);
    const bool split = split_step(h);
    const int gp = split ? split_grid(h, 1) : step_grid(h), gc = split ? split_grid(h, 2) : corrector_grid(h);
    const int gg = split ? split_grid(h, 0) : 0, gr = h->rows ? rows_grid(h) : 0;
    // per step: [Gaussian pass] ev[3k+1] predictor ev[3k+2] corrector ev[3k+3]
    std::vector<cudaEvent_t> ev(3 * (size_t)nsteps + 1);
    for (auto &e : ev) SS_CUDA(h, cudaEventCreate(&e));
    SS_CUDA(h, cudaEventRecord(ev[0], h->stream));
    for (int32_t k = 0; k < nsteps; ++k) {
        if (split && k == 0) SS_CUDA(h, launch_gstep_sync<R>(a, h->stream));
        if (split) SS_CUDA(h, launch_gauss<R>(a, h->block, gg, h->stream, 0));
        SS_CUDA(h, cudaEventRecord(ev[3 * k + 1], h->stream));
        if (h->rows) SS_CUDA(h, launch_rows_field<R>(a, a.sx, a.sy, a.sz, gr, h->stream));
        if (split)
            SS_CUDA(h, launch_predictor_split<R>(a, h->block, gp, h->stream));
        else
            SS_CUDA(h, launch_predictor<R>(a, h->block, gp, h->stream));
        SS_CUDA(h, cudaEventRecord(ev[3 * k + 2], h->stream));
        if (h->rows) SS_CUDA(h, launch_rows_field<R>(a, a.px, a.py, a.pz, gr, h->stream));
        if (split)
            SS_CUDA(h, launch_corrector_split<R>(a, h->block, gc, h->nfin, h->stream));
        else
            SS_CUDA(h, launch_corrector<R>(a, h->block, gc, h->nfin, h->stream));
        SS_CUDA(h, cudaEventRecord(ev[3 * k + 3], h->stream));
    }
    SS_CUDA(h, cudaEventSynchronize(ev.back()));
    double tg = 0.0, tp = 0.0, tc = 0.0;
    for (int32_t k = 0; k < nsteps; ++k) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        cudaEventElapsedTime(&a0, ev[3 * k], ev[3 * k + 1]);
        cudaEventElapsedTime(&a1, ev[3 * k + 1], ev[3 * k + 2]);
        cudaEventElapsedTime(&a2, ev[3 * k + 2], ev[3 * k + 3]);
        tg += a0;
        tp += a1;
        tc += a2;
    }
    float all = 0.f;
    cudaEventElapsedTime(&all, ev[0], ev.back());
    for (auto &e : ev) cudaEventDestroy(e);
    h->step += nsteps;
    out_ms[0] = tg / nsteps;
    out_ms[1] = tp / nsteps;
    out_ms[2] = tc / nsteps;
    out_ms[3] = all / nsteps;
    return check_device_flags(h);
}

template <typename R>
ss_status heun_pass_impl(ss_system *h, int32_t pass, int64_t tile0, int64_t ntiles) {
    KArgs<R> a = make_args<R>(h);
    if (pass == 2) {  // the step's record from every tile's partials, then the next step
        SS_CUDA(h, launch_finalize_ring(h->sys, h->sys_tiles, h->nsys, h->partials, h->rec, h->rec_cap, h->ctl,
                                        h->stream));
        SS_CUDA(h, launch_advance_step(h->ctl, h->stream));
        h->step += 1;
        return SS_OK;
    }
    if (ntiles == 0) return SS_OK;
    a.tiles = h->tiles + tile0;
    a.ntiles = ntiles;
    a.partials = h->partials + tile0 * kPartComps;
    a.advance = 0;
    if (pass == 0) {
        const int g = (int)std::min<int64_t>(ntiles, step_grid(h));
        SS_CUDA(h, launch_predictor<R>(a, h->block, g, h->stream));
    } else {
        const int g = (int)std::min<int64_t>(ntiles, corrector_grid(h));
        SS_CUDA(h, launch_corrector<R>(a, h->block, g, 0, h->stream));
    }
    return SS_OK;
}

// ----------------------------------------------------------------------------------
// Macrocell demagnetising field (Section "Demagnetising fields")
// ----------------------------------------------------------------------------------

void demag_free(ss_system *h) {
    void *bufs[] = {h->d_cell_of, h->d_cell_start, h->d_cell_spins, h->d_cell_first, h->d_cell_end, h->d_cpos,
                    h->d_cvol, h->d_cm, h->d_cH, h->d_hd[0], h->d_hd[1], h->d_hd[2]};
    for (void *b : bufs)
        if (b) dfree(h, b);
    h->d_cell_of = h->d_cell_start = h->d_cell_spins = h->d_cell_first = h->d_cell_end = nullptr;
    h->d_cpos = h->d_cvol = h->d_cm = h->d_cH = nullptr;
    h->d_hd[0] = h->d_hd[1] = h->d_hd[2] = nullptr;
    h->ncell = 0;
    h->hcell_of.clear();
}

// Macrocells of every system: cubes of edge `cell` on a grid anchored at the system's
// smallest coordinate on each axis, numbered by grid index (x fastest) among the occupied
// cubes, systems one after another.  Centre: the moment-weighted mean position; volume:
// n_atoms * vatom.
ss_status demag_build(ss_system *h, double cell, double vatom) {
    const int64_t n = h->n;
    std::vector<int32_t> cell_of((size_t)n);
    std::vector<int32_t> first, end;
    std::vector<double> cpos, cw, cvol;
    int64_t ncell = 0;
    for (int s = 0; s < h->nsys; ++s) {
        const int64_t off = h->sys_offset[s], ns = h->sys_n[s];
        if (ns == 0) continue;
        double lo[3], hi[3];
        for (int a = 0; a < 3; ++a) lo[a] = hi[a] = h->hpos[3 * off + a];
        for (int64_t i = off; i < off + ns; ++i)
            for (int a = 0; a < 3; ++a) {
                lo[a] = std::min(lo[a], h->hpos[3 * i + a]);
                hi[a] = std::max(hi[a], h->hpos[3 * i + a]);
            }
        int64_t dim[3];
        for (int a = 0; a < 3; ++a) dim[a] = (int64_t)std::floor((hi[a] - lo[a]) / cell) + 1;
        std::vector<int64_t> g((size_t)ns);
        for (int64_t k = 0; k < ns; ++k) {
            int64_t c[3];
            for (int a = 0; a < 3; ++a) c[a] = (int64_t)std::floor((h->hpos[3 * (off + k) + a] - lo[a]) / cell);
            g[k] = c[0] + dim[0] * (c[1] + dim[1] * c[2]);
        }
        std::vector<int64_t> occupied(g);
        std::sort(occupied.begin(), occupied.end());
        occupied.erase(std::unique(occupied.begin(), occupied.end()), occupied.end());
        const int64_t c0 = ncell;
        ncell += (int64_t)occupied.size();
        cpos.resize(3 * (size_t)ncell, 0.0);
        cw.resize((size_t)ncell, 0.0);
        cvol.resize((size_t)ncell, 0.0);
        for (int64_t k = 0; k < ns; ++k) {
            const int64_t c = c0 + (std::lower_bound(occupied.begin(), occupied.end(), g[k]) - occupied.begin());
            cell_of[off + k] = (int32_t)c;
            const double mu = h->hmu[off + k];
            for (int a = 0; a < 3; ++a) cpos[3 * c + a] += mu * h->hpos[3 * (off + k) + a];
            cw[c] += mu;
            cvol[c] += 1.0;
        }
        for (int64_t c = c0; c < ncell; ++c) {
            for (int a = 0; a < 3; ++a) cpos[3 * c + a] = cpos[3 * c + a] / cw[c];
            cvol[c] = cvol[c] * vatom;
            first.push_back((int32_t)c0);
            end.push_back((int32_t)ncell);
        }
    }
    if (ncell >= (int64_t(1) << 31)) return fail(h, SS_ERR_INVALID_ARG, "too many macrocells");
    std::vector<int32_t> start((size_t)ncell + 1, 0), spins((size_t)std::max<int64_t>(n, 1));
    for (int64_t i = 0; i < n; ++i) start[cell_of[i] + 1]++;
    for (int64_t c = 0; c < ncell; ++c) start[c + 1] += start[c];
    std::vector<int32_t> fill(start.begin(), start.end() - 1);
    for (int64_t i = 0; i < n; ++i) spins[fill[cell_of[i]]++] = (int32_t)i;
    demag_free(h);
    const size_t rs = real_size(h), nc = (size_t)std::max<int64_t>(ncell, 1);
    SS_CUDA(h, dalloc(h, (void **)&h->d_cell_of, cell_of.size() * sizeof(int32_t)));
    SS_CUDA(h, dalloc(h, (void **)&h->d_cell_start, start.size() * sizeof(int32_t)));
    SS_CUDA(h, dalloc(h, (void **)&h->d_cell_spins, spins.size() * sizeof(int32_t)));
    SS_CUDA(h, dalloc(h, (void **)&h->d_cell_first, nc * sizeof(int32_t)));
    SS_CUDA(h, dalloc(h, (void **)&h->d_cell_end, nc * sizeof(int32_t)));
    SS_CUDA(h, dalloc(h, (void **)&h->d_cpos, 3 * nc * sizeof(double)));
    SS_CUDA(h, dalloc(h, (void **)&h->d_cvol, nc * sizeof(double)));
    SS_CUDA(h, dalloc(h, (void **)&h->d_cm, 3 * nc * sizeof(double)));
    SS_CUDA(h, dalloc(h, (void **)&h->d_cH, 3 * nc * sizeof(double)));
    for (int c = 0; c < 3; ++c) SS_CUDA(h, dalloc(h, &h->d_hd[c], nc * rs));
    auto up = [&](void *dst, const void *src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->stream) : cudaSuccess;
    };
    SS_CUDA(h, up(h->d_cell_of, cell_of.data(), cell_of.size() * sizeof(int32_t)));
    SS_CUDA(h, up(h->d_cell_start, start.data(), start.size() * sizeof(int32_t)));
    SS_CUDA(h, up(h->d_cell_spins, spins.data(), (size_t)n * sizeof(int32_t)));
    SS_CUDA(h, up(h->d_cell_first, first.data(), first.size() * sizeof(int32_t)));
    SS_CUDA(h, up(h->d_cell_end, end.data(), end.size() * sizeof(int32_t)));
    SS_CUDA(h, up(h->d_cpos, cpos.data(), cpos.size() * sizeof(double)));
    SS_CUDA(h, up(h->d_cvol, cvol.data(), cvol.size() * sizeof(double)));
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    h->ncell = ncell;
    h->hcell_of.swap(cell_of);
    return SS_OK;
}

template <typename R>
cudaError_t enqueue_demag_update(ss_system *h) {
    const KArgs<R> a = make_args<R>(h);
    DemagArgs d{};
    d.ncell = h->ncell;
    d.cell_start = h->d_cell_start;
    d.cell_spins = h->d_cell_spins;
    d.cell_first = h->d_cell_first;
    d.cell_end = h->d_cell_end;
    d.pos = h->d_cpos;
    d.vol = h->d_cvol;
    d.m = h->d_cm;
    d.H = h->d_cH;
    return launch_demag<R>(a, d, h->stream);
}

cudaError_t demag_update(ss_system *h) {
    cudaError_t e = h->precision == SS_FP32_MIXED ? enqueue_demag_update<float>(h) : enqueue_demag_update<double>(h);
    if (e == cudaSuccess) h->demag_stale = false;
    return e;
}

// ----------------------------------------------------------------------------------
// Monte Carlo (Section "Monte Carlo Methods")
// ----------------------------------------------------------------------------------

// Colour classes of the neighbour graph, built on the first Monte Carlo call: greedy in
// site order (each site takes the smallest colour that no lower-indexed neighbour holds);
// systems share no bonds, so over the concatenated batch this is each system's own
// colouring.  The spins are listed by colour, in index order within a colour.
ss_status mc_prepare(ss_system *h) {
    if (h->mc_order) return SS_OK;
    const int64_t n = h->n;
    std::vector<int32_t> rp((size_t)n + 1), col((size_t)std::max<int64_t>(h->nnz, 1));
    SS_CUDA(h, cudaMemcpyAsync(rp.data(), h->row_ptr, rp.size() * sizeof(int32_t), cudaMemcpyDeviceToHost,
                               h->stream));
    if (h->nnz > 0)
        SS_CUDA(h, cudaMemcpyAsync(col.data(), h->col, (size_t)h->nnz * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                   h->stream));
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    std::vector<int32_t> colour((size_t)n, 0);
    std::vector<int64_t> taken;  // taken[c] == i: a lower-indexed neighbour of i holds colour c
    int32_t ncol = n > 0 ? 1 : 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
            const int64_t j = col[k];
            if (j >= i) continue;
            const int32_t cj = colour[j];
            if (cj >= (int32_t)taken.size()) taken.resize((size_t)cj + 1, -1);
            taken[cj] = i;
        }
        int32_t c = 0;
        while (c < (int32_t)taken.size() && taken[c] == i) ++c;
        colour[i] = c;
        ncol = std::max(ncol, c + 1);
    }
    h->mc_cstart.assign((size_t)ncol + 1, 0);
    for (int64_t i = 0; i < n; ++i) h->mc_cstart[colour[i] + 1]++;
    for (int32_t c = 0; c < ncol; ++c) h->mc_cstart[c + 1] += h->mc_cstart[c];
    std::vector<int32_t> order((size_t)std::max<int64_t>(n, 1));
    std::vector<int64_t> fill(h->mc_cstart.begin(), h->mc_cstart.end() - 1);
    for (int64_t i = 0; i < n; ++i) order[fill[colour[i]]++] = (int32_t)i;
    int32_t *dorder = nullptr;
    SS_CUDA(h, dalloc(h, (void **)&dorder, order.size() * sizeof(int32_t)));
    SS_CUDA(h, cudaMemcpyAsync(dorder, order.data(), order.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                               h->stream));
    if (ncol <= 2 && n > 0) {
        // tiles of at most `tile` trials within one system, per colour class (1,024, or 256 when
        // a class would give fewer than four tiles per SM); partial slots system by system
        // (class 0's tiles of the system, then class 1's)
        const int64_t kMcTile = h->mc_cstart[1] >= (int64_t)h->sm_count * 4 * 1024 ? 1024 : 256;
        std::vector<TileDesc> tl[2];
        std::vector<int32_t> sl[2];
        std::vector<int32_t> sys_slots((size_t)h->nsys + 1, 0);
        int32_t next = 0;
        for (int s = 0; s < h->nsys; ++s) {
            sys_slots[(size_t)s] = next;
            for (int c = 0; c < ncol; ++c) {
                // the spins of system s in class c: a contiguous run of order[] (sorted by index)
                const int64_t lo = h->sys_offset[s], hi = lo + h->sys_n[s];
                const int32_t *b0 = order.data() + h->mc_cstart[c], *b1 = order.data() + h->mc_cstart[c + 1];
                const int64_t r0 = std::lower_bound(b0, b1, (int32_t)lo) - order.data();
                const int64_t r1 = std::lower_bound(b0, b1, (int32_t)std::min<int64_t>(hi, INT32_MAX)) - order.data();
                for (int64_t q = r0; q < r1; q += kMcTile) {
                    TileDesc t;
                    t.start = q;
                    t.count = (int32_t)std::min<int64_t>(kMcTile, r1 - q);
                    t.sys = s;
                    tl[c].push_back(t);
                    sl[c].push_back(next++);
                }
            }
        }
        sys_slots[(size_t)h->nsys] = next;
        for (int c = 0; c < ncol; ++c) {
            h->mc_ntiles[c] = (int64_t)tl[c].size();
            if (tl[c].empty()) continue;
            SS_CUDA(h, dalloc(h, (void **)&h->mc_tiles[c], tl[c].size() * sizeof(TileDesc)));
            SS_CUDA(h, dalloc(h, (void **)&h->mc_slot[c], sl[c].size() * sizeof(int32_t)));
            SS_CUDA(h, cudaMemcpyAsync(h->mc_tiles[c], tl[c].data(), tl[c].size() * sizeof(TileDesc),
                                       cudaMemcpyHostToDevice, h->stream));
            SS_CUDA(h, cudaMemcpyAsync(h->mc_slot[c], sl[c].data(), sl[c].size() * sizeof(int32_t),
                                       cudaMemcpyHostToDevice, h->stream));
        }
        SS_CUDA(h, dalloc(h, (void **)&h->mc_sys_slots, sys_slots.size() * sizeof(int32_t)));
        SS_CUDA(h, cudaMemcpyAsync(h->mc_sys_slots, sys_slots.data(), sys_slots.size() * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, h->stream));
        SS_CUDA(h, dalloc(h, (void **)&h->mc_partials, (size_t)std::max(next, 1) * kPartComps * sizeof(double)));
        SS_CUDA(h, cudaStreamSynchronize(h->stream));
        h->mc_rec = true;
    }
    SS_CUDA(h, dalloc(h, (void **)&h->mc_acc, (size_t)h->nsys * sizeof(unsigned long long)));
    SS_CUDA(h, cudaMemsetAsync(h->mc_acc, 0, (size_t)h->nsys * sizeof(unsigned long long), h->stream));
    SS_CUDA(h, dalloc(h, (void **)&h->mc_par, (size_t)h->nsys * sizeof(double2)));
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    h->mc_order = dorder;
    h->mc_tried.assign((size_t)h->nsys, 0);
    h->mc_par_dirty = true;
    return SS_OK;
}

// (-kB T, sigma_g) with the cone width of Eq. MCgaussianSigma, sigma_g = (2/25)(kB T/muB)^(1/5).
double2 mc_params(double T) {
    return make_double2(-kBoltzmann * T, 2.0 / 25.0 * std::pow(kBoltzmann * T / kBohrMagneton, 0.2));
}

ss_status mc_upload_params(ss_system *h) {
    if (!h->mc_par_dirty) return SS_OK;
    std::vector<double2> ps((size_t)h->nsys);
    for (int s = 0; s < h->nsys; ++s) ps[s] = mc_params(h->Tsys[s]);
    SS_CUDA(h, cudaMemcpyAsync(h->mc_par, ps.data(), ps.size() * sizeof(double2), cudaMemcpyHostToDevice,
                               h->stream));
    if (h->sched_len > 0) {
        if (h->sched_len > h->mc_sched_cap) {
            SS_CUDA(h, cudaStreamSynchronize(h->stream));
            drop_graph(h);  // captured launches hold the old table's address
            if (h->mc_sched) dfree(h, h->mc_sched);
            h->mc_sched = nullptr;
            h->mc_sched_cap = 0;
            SS_CUDA(h, dalloc(h, (void **)&h->mc_sched, (size_t)h->sched_len * sizeof(double2)));
            h->mc_sched_cap = h->sched_len;
        }
        std::vector<double2> pk((size_t)h->sched_len);
        for (int64_t k = 0; k < h->sched_len; ++k) pk[k] = mc_params(h->sched_T[k]);
        SS_CUDA(h, cudaMemcpyAsync(h->mc_sched, pk.data(), pk.size() * sizeof(double2), cudaMemcpyHostToDevice,
                                   h->stream));
    }
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    h->mc_par_dirty = false;
    return SS_OK;
}

// The kernel variant the alternative integrators launch for these arguments.
template <typename R>
int alt_mode(const KArgs<R> &a) {
    return a.ex ? 2 : (a.J_tensor || a.any_cubic) ? 1 : 0;  // rows, general, plain (as step_mode)
}

// A grid-stride grid capped at one wave of `per_sm` resident blocks on every SM: more blocks
// than fit would leave a partial second wave running at low occupancy.
int one_wave(const ss_system *h, int grid, int per_sm) {
    const int64_t wave = (int64_t)per_sm * h->sm_count;
    return per_sm > 0 && wave < grid ? (int)wave : grid;
}

// Midpoint steps: per step the midpoint launches (the first of which leaves the tile partials
// of the record of the state at the start of the step, finalised into the ring at the
// device's step) and the step counter.
template <typename R>
cudaError_t enqueue_midpoint(ss_system *h, int64_t nsteps, int iterations) {
    KArgs<R> a = make_args<R>(h);
    use_rows(h, a);  // long rows: bare exchange sums from the row passes
    a.rows_bare = 1;
    const int rgrid = h->rows ? rows_grid(h) : 0;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((h->n + 255) / 256, (int64_t)h->sm_count * 8));
    const int igrid = one_wave(h, grid, alt_pass_blocks_per_sm<R>(0, alt_mode(a)));
    cudaError_t e = cudaSuccess;
    for (int64_t k = 0; k < nsteps && e == cudaSuccess; ++k) {
        e = launch_midpoint<R>(a, iterations, grid, igrid, rgrid, h->stream);
        if (e == cudaSuccess) e = launch_advance_step(a.step, h->stream);
    }
    return e;
}

// Steps of an alternative integrator, enqueued by `enqueue` (k steps per call): runs of whole
// graphs are captured once (per integrator variant `key`) and replayed; the launches hold no
// host-side step.
template <typename F>
ss_status integrate_captured(ss_system *h, int64_t n, int key, F enqueue, const char *what) {
    cudaError_t e = cudaSuccess;
    int64_t left = n;
    const int g = graph_len(h);
    if (left >= g && !h->midgraph_failed && h->exec != SS_EXEC_KERNELS) {
        if (h->midgraph && h->midgraph_iters != key) {
            cudaGraphExecDestroy(h->midgraph);
            h->midgraph = nullptr;
        }
        if (!h->midgraph) {
            cudaGraph_t graph = nullptr;
            e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const cudaError_t ek = enqueue(g);
                e = cudaStreamEndCapture(h->stream, &graph);
                if (ek != cudaSuccess) e = ek;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&h->midgraph, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                cudaGetLastError();
                h->midgraph = nullptr;
                h->midgraph_failed = true;  // capture refused: launch directly from now on
                e = cudaSuccess;
            } else {
                h->midgraph_steps = g;
                h->midgraph_iters = key;
            }
        }
        while (h->midgraph && left >= h->midgraph_steps && e == cudaSuccess) {
            e = cudaGraphLaunch(h->midgraph, h->stream);
            left -= h->midgraph_steps;
        }
    }
    if (e == cudaSuccess && left > 0) e = enqueue(left);
    if (e != cudaSuccess) return cuda_fail(h, e, what);
    h->step += n;
    return SS_OK;
}

// As integrate_captured, with the demagnetising field (when on) recomputed at multiples of its
// interval (and when stale) and held in between: the steps between two updates run as one chunk.
template <typename F>
ss_status integrate_with_demag(ss_system *h, int64_t n, int key, F enqueue, const char *what) {
    if (!h->demag_on) return integrate_captured(h, n, key, enqueue, what);
    while (n > 0) {
        const int64_t r = h->step % h->demag_every;
        if (r == 0 || h->demag_stale) {
            const cudaError_t e = demag_update(h);
            if (e != cudaSuccess) return cuda_fail(h, e, "demagnetising field");
        }
        const int64_t chunk = std::min<int64_t>(n, h->demag_every - r);
        const ss_status st = integrate_captured(h, chunk, key, enqueue, what);
        if (st != SS_OK) return st;
        n -= chunk;
    }
    return SS_OK;
}

// Semi-implicit predictor-corrector steps: predictor (with the record's tile partials),
// record, corrector, step counter.
template <typename R>
cudaError_t enqueue_sib(ss_system *h, int64_t nsteps) {
    KArgs<R> a = make_args<R>(h);
    use_rows(h, a);  // long rows: bare exchange sums from the row passes
    a.rows_bare = 1;
    const int rgrid = h->rows ? rows_grid(h) : 0;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((h->n + 255) / 256, (int64_t)h->sm_count * 8));
    const int cgrid = one_wave(h, grid, alt_pass_blocks_per_sm<R>(1, alt_mode(a)));
    cudaError_t e = cudaSuccess;
    for (int64_t k = 0; k < nsteps && e == cudaSuccess; ++k) {
        e = launch_sib<R>(a, grid, cgrid, rgrid, h->stream);
        if (e == cudaSuccess) e = launch_advance_step(a.step, h->stream);
    }
    return e;
}

// Per Monte Carlo step: the record of the state at the start of the step (measure and
// finalise into the ring), one launch per colour class, then the step counter advances.
template <typename R>
cudaError_t enqueue_mc(ss_system *h, int64_t nsteps) {
    const KArgs<R> a = make_args<R>(h);
    McArgs m{};
    m.order = h->mc_order;
    m.par_sys = h->mc_par;
    m.par_sched = h->mc_sched;
    m.acc = h->mc_acc;
    const int block = 256;
    const int64_t resident = (int64_t)h->sm_count * std::max(1, mc_blocks_per_sm<R>(block, own_rows_mode(h)));
    const int gmeas = step_grid(h);
    const int ncol = (int)h->mc_cstart.size() - 1;
    cudaError_t e = cudaSuccess;
    if (h->mc_rec && !h->rows) {  // the record summed in the colour passes
        m.partials = h->mc_partials;
        for (int64_t k = 0; k < nsteps && e == cudaSuccess; ++k) {
            for (int c = 0; c < ncol && e == cudaSuccess; ++c) {
                m.c0 = h->mc_cstart[c];
                m.c1 = h->mc_cstart[c + 1];
                m.tiles = h->mc_tiles[c];
                m.slot = h->mc_slot[c];
                m.ntiles = h->mc_ntiles[c];
                m.first = c == 0 ? 1 : 0;
                if (m.ntiles == 0) continue;
                const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(m.ntiles, resident));
                e = launch_mc_colour_rec<R>(a, m, grid, h->stream);
            }
            if (e == cudaSuccess)
                e = launch_finalize_ring(h->sys, h->mc_sys_slots, h->nsys, h->mc_partials, h->rec, h->rec_cap, a.step,
                                         h->stream);
            if (e == cudaSuccess) e = launch_advance_step(a.step, h->stream);
        }
        return e;
    }
    KArgs<R> ar = a;  // the record's measurement reads the row passes' field on long rows
    use_rows(h, ar);
    const int rgrid = h->rows ? rows_grid(h) : 0;
    if (h->rows) {  // the long-row passes read each step's trial randoms, drawn for all spins first
        if (!h->mc_pre_move) return cudaErrorInvalidValue;  // allocated by mc_step
        m.pre_move = h->mc_pre_move;
        m.pre_g = h->mc_pre_g;
        m.pre_acc = h->mc_pre_acc;
    }
    for (int64_t k = 0; k < nsteps && e == cudaSuccess; ++k) {
        if (h->rows) e = launch_rows_field<R>(ar, ar.sx, ar.sy, ar.sz, rgrid, h->stream);
        if (e == cudaSuccess) e = launch_measure<R>(ar, h->block, gmeas, h->stream);
        if (e == cudaSuccess)
            e = launch_finalize_ring(h->sys, h->sys_tiles, h->nsys, h->partials, h->rec, h->rec_cap, a.step, h->stream);
        if (h->rows && e == cudaSuccess) e = launch_mc_prep<R>(a, m, h->stream);
        for (int c = 0; c < ncol && e == cudaSuccess; ++c) {
            m.c0 = h->mc_cstart[c];
            m.c1 = h->mc_cstart[c + 1];
            const int64_t need = (m.c1 - m.c0 + block - 1) / block;
            const int grid = (int)std::max<int64_t>(1, std::min(need, resident));
            e = h->rows ? launch_mc_colour_warp<R>(a, m, grid, h->stream)  // long rows: a warp per 32 trials
                        : launch_mc_colour<R>(a, m, block, grid, h->stream);
        }
        if (e == cudaSuccess) e = launch_advance_step(a.step, h->stream);
    }
    return e;
}

}  // namespace

extern "C" {

ss_status spin_system_create(const ss_params *p, ss_system **out) { return create_impl(p, 1, out); }

ss_status spin_batch_create(const ss_params *systems, int32_t count, ss_system **out) {
    return create_impl(systems, count, out);
}

ss_status spin_system_destroy(ss_system *h) {
    if (!h) return SS_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graph(h);
    for (auto &b : h->bufs) {
        cudaFree(b.p);
        g_live_bytes -= (int64_t)b.bytes;
    }
    h->bufs.clear();
    if (h->side) {
        cudaStreamSynchronize(h->side);
        cudaStreamDestroy(h->side);
    }
    for (cudaEvent_t ev : {h->ev_fork, h->ev_gauss, h->ev_corr})
        if (ev) cudaEventDestroy(ev);
    if (h->cl_side) {
        cudaStreamSynchronize(h->cl_side);
        cudaStreamDestroy(h->cl_side);
    }
    for (cudaEvent_t ev : h->cl_ev)
        if (ev) cudaEventDestroy(ev);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
    return SS_OK;
}

ss_status spin_system_set_stream(ss_system *h, void *cuda_stream) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    h->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : h->own_stream;
    return SS_OK;
}

ss_status set_field(ss_system *h, int32_t sys, const double H_app[3]) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (!H_app || !finite3(H_app)) return fail(h, SS_ERR_INVALID_ARG, "H_app must be 3 finite values");
    if (sys >= h->nsys) return fail(h, SS_ERR_INVALID_ARG, "system %d out of range", sys);
    for (int s = 0; s < h->nsys; ++s) {
        if (sys >= 0 && s != sys) continue;
        for (int c = 0; c < 3; ++c) {
            h->hsys[s].H[c] = H_app[c];
            h->hsys[s].Hf[c] = (float)H_app[c];
        }
        SS_CUDA(h, cudaMemcpyAsync(&h->sys[s], &h->hsys[s], sizeof(SysDesc), cudaMemcpyHostToDevice, h->stream));
    }
    return SS_OK;
}

static ss_status upload_sqrtT(ss_system *h) {
    if (h->zero_T) SS_CUDA(h, invalidate_ahead(h));
    h->zero_T = false;
    for (auto &d : h->hsys) {
        d.sqrtTf = (float)d.sqrtT;
        h->zero_T = h->zero_T || d.sqrtT == 0.0;
    }
    SS_CUDA(h, cudaMemcpyAsync(h->sys, h->hsys.data(), h->hsys.size() * sizeof(SysDesc), cudaMemcpyHostToDevice,
                               h->stream));
    return SS_OK;
}

static ss_status clear_schedule(ss_system *h) {
    if (h->sched_len != 0) {
        h->sched_len = 0;
        drop_graph(h);
    }
    return SS_OK;
}

ss_status set_temperature(ss_system *h, double T) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (!(T >= 0.0) || !std::isfinite(T)) return fail(h, SS_ERR_INVALID_ARG, "T must be finite and >= 0");
    for (auto &d : h->hsys) d.sqrtT = std::sqrt(T);
    for (auto &t : h->Tsys) t = T;
    h->mc_par_dirty = true;
    clear_schedule(h);
    return upload_sqrtT(h);
}

ss_status set_temperature_batch(ss_system *h, const double *T, int32_t count) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (!T || count != h->nsys) return fail(h, SS_ERR_INVALID_ARG, "need one temperature per system (%d)", h->nsys);
    for (int s = 0; s < count; ++s)
        if (!(T[s] >= 0.0) || !std::isfinite(T[s])) return fail(h, SS_ERR_INVALID_ARG, "T[%d] invalid", s);
    for (int s = 0; s < count; ++s) h->hsys[s].sqrtT = std::sqrt(T[s]);
    for (int s = 0; s < count; ++s) h->Tsys[s] = T[s];
    h->mc_par_dirty = true;
    clear_schedule(h);
    return upload_sqrtT(h);
}

ss_status set_temperature_schedule(ss_system *h, const double *T_per_step, int64_t nsteps, int64_t step0) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (!T_per_step || nsteps < 1) return fail(h, SS_ERR_INVALID_ARG, "schedule needs at least one entry");
    std::vector<double> r((size_t)nsteps);
    std::vector<float> rf((size_t)nsteps);
    for (int64_t k = 0; k < nsteps; ++k) {
        if (!(T_per_step[k] >= 0.0) || !std::isfinite(T_per_step[k]))
            return fail(h, SS_ERR_INVALID_ARG, "T_per_step[%lld] invalid", (long long)k);
        r[k] = std::sqrt(T_per_step[k]);
        rf[k] = (float)r[k];
    }
    if (nsteps > h->sched_cap) {
        SS_CUDA(h, cudaStreamSynchronize(h->stream));
        if (h->sched) dfree(h, h->sched);
        if (h->sched_f) dfree(h, h->sched_f);
        h->sched = nullptr;
        h->sched_f = nullptr;
        h->sched_cap = 0;
        SS_CUDA(h, dalloc(h, (void **)&h->sched, (size_t)nsteps * sizeof(double)));
        SS_CUDA(h, dalloc(h, (void **)&h->sched_f, (size_t)nsteps * sizeof(float)));
        h->sched_cap = nsteps;
        drop_graph(h);
    }
    SS_CUDA(h, cudaMemcpyAsync(h->sched, r.data(), (size_t)nsteps * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    SS_CUDA(h, cudaMemcpyAsync(h->sched_f, rf.data(), (size_t)nsteps * sizeof(float), cudaMemcpyHostToDevice,
                               h->stream));
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    if (h->zero_T) SS_CUDA(h, invalidate_ahead(h));
    h->zero_T = std::any_of(r.begin(), r.end(), [](double v) { return v == 0.0; });
    if (h->sched_len != nsteps || h->sched_step0 != step0) drop_graph(h);
    h->sched_len = nsteps;
    h->sched_step0 = step0;
    h->sched_T.assign(T_per_step, T_per_step + nsteps);
    h->mc_par_dirty = true;
    return SS_OK;
}

static ss_status advance_steps(ss_system *h, int64_t n);

ss_status llg_heun_step(ss_system *h, int64_t n) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (h->slab_own >= 0)
        return fail(h, SS_ERR_UNSUPPORTED, "a slab advances by spin_system_heun_pass with halo exchanges");
    if (n < 0) return fail(h, SS_ERR_INVALID_ARG, "n must be >= 0");
    if (n == 0) return SS_OK;
    if (!h->demag_on) return advance_steps(h, n);
    // demagnetising field: recomputed at multiples of the interval (and when stale), held in
    // between; the steps between two updates run as one chunk
    while (n > 0) {
        const int64_t r = h->step % h->demag_every;
        if (r == 0 || h->demag_stale) {
            const cudaError_t e = demag_update(h);
            if (e != cudaSuccess) return cuda_fail(h, e, "demagnetising field");
        }
        const int64_t chunk = std::min<int64_t>(n, h->demag_every - r);
        st = advance_steps(h, chunk);
        if (st != SS_OK) return st;
        n -= chunk;
    }
    return SS_OK;
}

static ss_status advance_steps(ss_system *h, int64_t n) {
    cudaError_t e = cudaSuccess;
    int mode = h->exec;
    // automatic: the cluster step for a small single system that it takes (on GB300 a few
    // times faster than any per-step launch there), else graphs for long runs
    if (mode == SS_EXEC_AUTO && h->n <= kClusterAutoMax && h->nsys == 1 && !cluster_ready(h))
        mode = SS_EXEC_CLUSTER;
    if (mode == SS_EXEC_AUTO) mode = n >= graph_len(h) ? SS_EXEC_GRAPH : SS_EXEC_KERNELS;
    if (mode == SS_EXEC_GRAPH && !h->graph_failed) {
        e = ensure_graph(h);
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->graph_failed = true;
            mode = SS_EXEC_KERNELS;
        }
    } else if (mode == SS_EXEC_GRAPH) {
        mode = SS_EXEC_KERNELS;
    }
    if (mode == SS_EXEC_GRAPH) {
        int64_t left = n;
        while (left >= h->graph_steps) {
            e = cudaGraphLaunch(h->graph, h->stream);
            if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
            left -= h->graph_steps;
        }
        e = enqueue_kernels(h, left);
    } else if (mode == SS_EXEC_SYSTEM_BLOCKS) {
        e = enqueue_sysblocks(h, n);
    } else if (mode == SS_EXEC_CLUSTER) {
        const char *why = cluster_ready(h);
        if (why) return fail(h, SS_ERR_UNSUPPORTED, "%s", why);
        e = enqueue_cluster(h, n);
    } else if (mode == SS_EXEC_PERSISTENT) {
        int64_t left = n;
        if (!h->pgraph_failed) {
            e = persistent_graph_run(h, left);
            if (e != cudaSuccess) {
                cudaGetLastError();
                h->pgraph_failed = true;  // capture refused: launch directly from now on
                left = n;
                e = cudaSuccess;
            }
        }
        if (e == cudaSuccess && left > 0) e = enqueue_persist(h, left);
        if (e == cudaErrorCooperativeLaunchTooLarge || e == cudaErrorNotSupported) {
            cudaGetLastError();
            return fail(h, SS_ERR_UNSUPPORTED, "persistent launch not possible: %s", cudaGetErrorString(e));
        }
    } else {
        e = enqueue_kernels(h, n);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "step launch");
    h->step += n;
    return SS_OK;
}

ss_status llg_midpoint_step(ss_system *h, int64_t n, int32_t iterations) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (h->slab_own >= 0) return fail(h, SS_ERR_UNSUPPORTED, "not available on a slab handle");
    if (n < 0) return fail(h, SS_ERR_INVALID_ARG, "n must be >= 0");
    if (iterations < 1 || iterations > 1000) return fail(h, SS_ERR_INVALID_ARG, "iterations must be 1..1000");
    auto enqueue = [h, iterations](int64_t k) {
        return h->precision == SS_FP32_MIXED ? enqueue_midpoint<float>(h, k, iterations)
                                             : enqueue_midpoint<double>(h, k, iterations);
    };
    return integrate_with_demag(h, n, iterations, enqueue, "midpoint step");
}

ss_status llg_semi_implicit_step(ss_system *h, int64_t n) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (h->slab_own >= 0) return fail(h, SS_ERR_UNSUPPORTED, "not available on a slab handle");
    if (n < 0) return fail(h, SS_ERR_INVALID_ARG, "n must be >= 0");
    auto enqueue = [h](int64_t k) {
        return h->precision == SS_FP32_MIXED ? enqueue_sib<float>(h, k) : enqueue_sib<double>(h, k);
    };
    return integrate_with_demag(h, n, -1, enqueue, "semi-implicit step");
}

ss_status set_demag(ss_system *h, double cell_size, double atom_volume, int32_t every) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (h->slab_own >= 0) return fail(h, SS_ERR_UNSUPPORTED, "not available on a slab handle");
    if (!std::isfinite(cell_size)) return fail(h, SS_ERR_INVALID_ARG, "cell_size must be finite");
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    drop_graph(h);  // captured launches hold the previous arguments
    if (cell_size <= 0.0) {
        h->demag_on = false;
        demag_free(h);
        return SS_OK;
    }
    if (h->hpos.empty()) return fail(h, SS_ERR_INVALID_ARG, "the demagnetising field needs atomic positions (pos)");
    if (!(atom_volume > 0.0) || !std::isfinite(atom_volume))
        return fail(h, SS_ERR_INVALID_ARG, "atom_volume must be finite and > 0");
    if (every < 1) return fail(h, SS_ERR_INVALID_ARG, "every must be >= 1");
    h->demag_on = false;
    st = demag_build(h, cell_size, atom_volume);
    if (st != SS_OK) return st;
    h->demag_cell = cell_size;
    h->demag_vatom = atom_volume;
    h->demag_every = every;
    h->demag_on = true;
    h->demag_stale = true;
    return SS_OK;
}

ss_status get_demag_field(ss_system *h, double *out3n) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (!out3n) return fail(h, SS_ERR_INVALID_ARG, "out3n is NULL");
    if (!h->demag_on) return fail(h, SS_ERR_INVALID_ARG, "the demagnetising field is not enabled (set_demag)");
    if (h->demag_stale) {
        const cudaError_t e = demag_update(h);
        if (e != cudaSuccess) return cuda_fail(h, e, "demagnetising field");
    }
    std::vector<double> H(3 * (size_t)std::max<int64_t>(h->ncell, 1));
    SS_CUDA(h, cudaMemcpyAsync(H.data(), h->d_cH, 3 * (size_t)h->ncell * sizeof(double), cudaMemcpyDeviceToHost,
                               h->stream));
    st = check_device_flags(h);
    if (st != SS_OK) return st;
    for (int64_t i = 0; i < h->n; ++i)
        for (int c = 0; c < 3; ++c) out3n[3 * i + c] = H[3 * (size_t)h->hcell_of[i] + c];
    return SS_OK;
}

ss_status mc_step(ss_system *h, int64_t nsteps) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (h->slab_own >= 0) return fail(h, SS_ERR_UNSUPPORTED, "not available on a slab handle");
    if (nsteps < 0) return fail(h, SS_ERR_INVALID_ARG, "nsteps must be >= 0");
    if (nsteps == 0) return SS_OK;
    st = mc_prepare(h);
    if (st != SS_OK) return st;
    st = mc_upload_params(h);
    if (st != SS_OK) return st;
    if (h->rows && !h->mc_pre_move) {  // the long-row passes' trial randoms (before any capture)
        SS_CUDA(h, dalloc(h, (void **)&h->mc_pre_move, (size_t)h->n));
        SS_CUDA(h, dalloc(h, &h->mc_pre_g, 3 * (size_t)h->n * real_size(h)));
        SS_CUDA(h, dalloc(h, (void **)&h->mc_pre_acc, (size_t)h->n * sizeof(double)));
    }
    cudaError_t e = cudaSuccess;
    int64_t left = nsteps;
    // Captured steps (the launches hold no host-side step): replayed while whole graphs fit
    const int g = graph_len(h);
    if (left >= g && !h->mcgraph_failed && h->exec != SS_EXEC_KERNELS) {
        if (!h->mcgraph) {
            cudaGraph_t graph = nullptr;
            e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                const cudaError_t ek =
                    h->precision == SS_FP32_MIXED ? enqueue_mc<float>(h, g) : enqueue_mc<double>(h, g);
                e = cudaStreamEndCapture(h->stream, &graph);
                if (ek != cudaSuccess) e = ek;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&h->mcgraph, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess) {
                cudaGetLastError();
                h->mcgraph = nullptr;
                h->mcgraph_failed = true;  // capture refused: launch directly from now on
                e = cudaSuccess;
            } else {
                h->mcgraph_steps = g;
            }
        }
        while (h->mcgraph && left >= h->mcgraph_steps && e == cudaSuccess) {
            e = cudaGraphLaunch(h->mcgraph, h->stream);
            left -= h->mcgraph_steps;
        }
    }
    if (e == cudaSuccess && left > 0)
        e = h->precision == SS_FP32_MIXED ? enqueue_mc<float>(h, left) : enqueue_mc<double>(h, left);
    if (e != cudaSuccess) return cuda_fail(h, e, "Monte Carlo launch");
    h->step += nsteps;
    for (int s = 0; s < h->nsys; ++s) h->mc_tried[s] += h->sys_n[s] * nsteps;
    return SS_OK;
}

ss_status get_mc_stats(ss_system *h, int32_t sys, int64_t out[2]) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (!out) return fail(h, SS_ERR_INVALID_ARG, "out is NULL");
    if (sys < 0 || sys >= h->nsys) return fail(h, SS_ERR_INVALID_ARG, "system %d out of range", sys);
    out[0] = out[1] = 0;
    if (!h->mc_acc) return check_device_flags(h);
    unsigned long long acc = 0;
    SS_CUDA(h, cudaMemcpyAsync(&acc, h->mc_acc + sys, sizeof(acc), cudaMemcpyDeviceToHost, h->stream));
    st = check_device_flags(h);
    out[0] = (int64_t)acc;
    out[1] = h->mc_tried[sys];
    return st;
}

ss_status spin_system_sync(ss_system *h) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    return check_device_flags(h);
}

ss_status get_spins(ss_system *h, double *out3n) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (!out3n) return fail(h, SS_ERR_INVALID_ARG, "out3n is NULL");
    const int64_t n = h->n;
    if (h->precision == SS_FP32_MIXED) {
        std::vector<float> b(3 * (size_t)n);
        for (int c = 0; c < 3; ++c)
            SS_CUDA(h, cudaMemcpyAsync(b.data() + c * n, h->state[c], n * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
        st = check_device_flags(h);
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < 3; ++c) out3n[3 * i + c] = (double)b[c * n + i];
    } else {
        std::vector<double> b(3 * (size_t)n);
        for (int c = 0; c < 3; ++c)
            SS_CUDA(h, cudaMemcpyAsync(b.data() + c * n, h->state[c], n * sizeof(double), cudaMemcpyDeviceToHost,
                                       h->stream));
        st = check_device_flags(h);
        for (int64_t i = 0; i < n; ++i)
            for (int c = 0; c < 3; ++c) out3n[3 * i + c] = b[c * n + i];
    }
    return st;
}

ss_status get_spins_device(ss_system *h, const void **sx, const void **sy, const void **sz) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (!sx || !sy || !sz) return fail(h, SS_ERR_INVALID_ARG, "NULL output pointer");
    *sx = h->state[0];
    *sy = h->state[1];
    *sz = h->state[2];
    return SS_OK;
}

ss_status get_magnetisation(ss_system *h, int32_t sys, double out[4]) {
    if (!out) return fail(h, SS_ERR_INVALID_ARG, "out is NULL");
    double r[kRecComps];
    ss_status st = current_record(h, sys, r);
    if (st != SS_OK) return st;
    for (int c = 0; c < 3; ++c) out[c] = r[c] / r[3];
    out[3] = std::sqrt(out[0] * out[0] + out[1] * out[1] + out[2] * out[2]);
    return SS_OK;
}

ss_status get_energy(ss_system *h, int32_t sys, double out[4]) {
    if (!out) return fail(h, SS_ERR_INVALID_ARG, "out is NULL");
    double r[kRecComps];
    ss_status st = current_record(h, sys, r);
    if (st != SS_OK) return st;
    out[0] = r[7];
    out[1] = r[4];
    out[2] = r[5];
    out[3] = r[6];
    return SS_OK;
}

ss_status get_record(ss_system *h, int64_t first_step, int64_t count, double *out) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (count < 0 || (count > 0 && !out)) return fail(h, SS_ERR_INVALID_ARG, "bad count or NULL out");
    st = check_device_flags(h);
    if (st != SS_OK) return st;
    if (first_step < 0 || first_step + count > h->step || first_step < h->step - h->rec_cap)
        return fail(h, SS_ERR_INVALID_ARG, "steps [%lld, %lld) not in the record ring [%lld, %lld)",
                    (long long)first_step, (long long)(first_step + count),
                    (long long)std::max<int64_t>(0, h->step - h->rec_cap), (long long)h->step);
    const size_t per = (size_t)h->nsys * kRecComps;
    int64_t k = 0;
    while (k < count) {
        const int64_t slot = (first_step + k) % h->rec_cap;
        const int64_t run = std::min<int64_t>(count - k, h->rec_cap - slot);
        SS_CUDA(h, cudaMemcpyAsync(out + k * per, h->rec + slot * per, (size_t)run * per * sizeof(double),
                                   cudaMemcpyDeviceToHost, h->stream));
        k += run;
    }
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    return SS_OK;
}

ss_status set_spins(ss_system *h, const double *in3n) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (!in3n) return fail(h, SS_ERR_INVALID_ARG, "in3n is NULL");
    const int64_t n = h->n;
    for (int64_t i = 0; i < n; ++i) {
        const double *v = in3n + 3 * i;
        if (!finite3(v) || v[0] * v[0] + v[1] * v[1] + v[2] * v[2] == 0.0)
            return fail(h, SS_ERR_INVALID_ARG, "spin %lld invalid", (long long)i);
    }
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    if (h->precision == SS_FP32_MIXED) {
        std::vector<float> b(3 * (size_t)n);
        for (int64_t i = 0; i < n; ++i) {
            double u[3];
            unit_in(in3n + 3 * i, u, unit_tol(h->precision));
            for (int c = 0; c < 3; ++c) b[c * n + i] = (float)u[c];
        }
        for (int c = 0; c < 3; ++c)
            SS_CUDA(h, cudaMemcpyAsync(h->state[c], b.data() + c * n, n * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        SS_CUDA(h, cudaStreamSynchronize(h->stream));
    } else {
        std::vector<double> b(3 * (size_t)n);
        for (int64_t i = 0; i < n; ++i) {
            double u[3];
            unit_in(in3n + 3 * i, u, unit_tol(h->precision));
            for (int c = 0; c < 3; ++c) b[c * n + i] = u[c];
        }
        for (int c = 0; c < 3; ++c)
            SS_CUDA(h, cudaMemcpyAsync(h->state[c], b.data() + c * n, n * sizeof(double), cudaMemcpyHostToDevice,
                                       h->stream));
        SS_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    h->demag_stale = true;  // the held demagnetising field belongs to the previous state
    return SS_OK;
}

ss_status set_step(ss_system *h, int64_t step) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (step < 0) return fail(h, SS_ERR_INVALID_ARG, "step must be >= 0");
    const unsigned long long v = (unsigned long long)step;
    SS_CUDA(h, cudaMemcpyAsync(h->ctl, &v, sizeof(v), cudaMemcpyHostToDevice, h->stream));
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    h->step = step;
    h->demag_stale = true;
    return SS_OK;
}

ss_status get_step(ss_system *h, int64_t *step) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (!step) return fail(h, SS_ERR_INVALID_ARG, "step is NULL");
    st = check_device_flags(h);
    *step = h->step;
    return st;
}

ss_status spin_system_set_exec(ss_system *h, ss_exec mode) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (mode < SS_EXEC_AUTO || mode > SS_EXEC_CLUSTER) return fail(h, SS_ERR_INVALID_ARG, "unknown exec mode");
    if (mode == SS_EXEC_CLUSTER) {
        const char *why = cluster_ready(h);
        if (why) return fail(h, SS_ERR_UNSUPPORTED, "%s", why);
    }
    if ((mode == SS_EXEC_PERSISTENT || mode == SS_EXEC_SYSTEM_BLOCKS) && h->rows)
        return fail(h, SS_ERR_UNSUPPORTED, "long exchange rows (a warp per row) run as graph or plain launches");
    if (mode == SS_EXEC_PERSISTENT && persistent_grid(h) < 1)
        return fail(h, SS_ERR_UNSUPPORTED, "persistent kernel cannot be made co-resident with block %d", h->block);
    h->exec = mode;
    return SS_OK;
}

ss_status spin_system_set_launch(ss_system *h, int32_t block, int32_t tile) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (block != 32 && block != 64 && block != 128 && block != 256 && block != 512)
        return fail(h, SS_ERR_INVALID_ARG, "block must be 32, 64, 128, 256 or 512");
    if (tile < block || tile % block != 0 || tile > 16 * block)
        return fail(h, SS_ERR_INVALID_ARG, "tile must be a multiple of block, at most 16 blocks");
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    h->block = block;
    h->tile = tile;
    return build_tiles(h);
}

ss_status spin_system_set_exchange_rows(ss_system *h, int32_t mode) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (h->slab_own >= 0) return fail(h, SS_ERR_UNSUPPORTED, "not available on a slab handle");
    if (mode < 0 || mode > 2) return fail(h, SS_ERR_INVALID_ARG, "mode must be 0 (automatic), 1 or 2");
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    return set_rows(h, mode);
}

ss_status spin_system_set_gaussian_pass(ss_system *h, int32_t mode) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (mode < 0 || mode > 2) return fail(h, SS_ERR_INVALID_ARG, "mode must be 0, 1 or 2");
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    if (mode > 0 && h->precision == SS_FP32_MIXED && !h->ahead2[0])
        for (int b = 0; b < 3; ++b) SS_CUDA(h, dalloc(h, &h->ahead2[b], (size_t)h->n * sizeof(float)));
    if (mode == 2 && !h->side) {
        int least = 0, greatest = 0;
        SS_CUDA(h, cudaDeviceGetStreamPriorityRange(&least, &greatest));
        h->side_priority = least;
        SS_CUDA(h, cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, least));
        SS_CUDA(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        SS_CUDA(h, cudaEventCreateWithFlags(&h->ev_gauss, cudaEventDisableTiming));
        SS_CUDA(h, cudaEventCreateWithFlags(&h->ev_corr, cudaEventDisableTiming));
    }
    h->gauss_mode = mode;
    drop_graph(h);  // captured launches hold the other step's kernels
    SS_CUDA(h, invalidate_ahead(h));
    return SS_OK;
}

ss_status spin_system_set_row_patterns(ss_system *h, int32_t on) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (on != 0 && on != 1) return fail(h, SS_ERR_INVALID_ARG, "on must be 0 or 1");
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    h->use_pat = on != 0;
    drop_graph(h);  // captured launches hold the old arguments
    return SS_OK;
}

ss_status spin_system_set_draw_ahead(ss_system *h, int32_t eighths) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (eighths < 0 || eighths > 8) return fail(h, SS_ERR_INVALID_ARG, "eighths must be 0..8");
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    h->ahead_q = eighths;
    return build_tiles(h);
}

// ----------------------------------------------------------------------------------
// Slab decomposition of one system (Appendix C: geometric decomposition with core, boundary
// and halo spins, the halo passed between processors twice per time step)
// ----------------------------------------------------------------------------------

ss_status spin_slab_create(const ss_params *p, int32_t nslabs, int32_t slab, ss_system **out) {
    if (!out) return fail(nullptr, SS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!p) return fail(nullptr, SS_ERR_INVALID_ARG, "params is NULL");
    ss_status st = validate(p, 0);
    if (st != SS_OK) return st;
    if (nslabs < 1 || slab < 0 || slab >= nslabs || nslabs > p->n)
        return fail(nullptr, SS_ERR_INVALID_ARG, "need 1 <= nslabs <= n and 0 <= slab < nslabs");
    if (p->J_tensor) return fail(nullptr, SS_ERR_UNSUPPORTED, "slabs take scalar exchange");
    const int64_t n = p->n;
    const int64_t lo = n * slab / nslabs, hi = n * (slab + 1) / nslabs, own = hi - lo;
    // halo: every neighbour of an owned spin outside [lo, hi), sorted
    std::vector<int64_t> halo;
    std::vector<uint8_t> edge((size_t)own, 0);
    for (int64_t i = lo; i < hi; ++i)
        for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k) {
            const int64_t j = p->col[k];
            if (j < lo || j >= hi) {
                halo.push_back(j);
                edge[(size_t)(i - lo)] = 1;
            }
        }
    std::sort(halo.begin(), halo.end());
    halo.erase(std::unique(halo.begin(), halo.end()), halo.end());
    const int64_t nh = (int64_t)halo.size(), nt = own + nh;
    auto local = [&](int64_t g) -> int64_t {
        if (g >= lo && g < hi) return g - lo;
        return own + (int64_t)(std::lower_bound(halo.begin(), halo.end(), g) - halo.begin());
    };
    // local arrays: the owned rows (columns renumbered), empty rows for the halo copies
    std::vector<int64_t> rp((size_t)nt + 1, 0);
    std::vector<int32_t> col;
    std::vector<double> J, mu((size_t)nt), ku((size_t)nt), ea, kn, kc, S0, pos;
    col.reserve((size_t)(p->row_ptr[hi] - p->row_ptr[lo]));
    for (int64_t i = lo; i < hi; ++i) {
        for (int64_t k = p->row_ptr[i]; k < p->row_ptr[i + 1]; ++k) {
            col.push_back((int32_t)local(p->col[k]));
            J.push_back(p->J[k]);
        }
        rp[(size_t)(i - lo) + 1] = (int64_t)col.size();
    }
    for (int64_t i = own; i < nt; ++i) rp[(size_t)i + 1] = (int64_t)col.size();
    auto global = [&](int64_t l) { return l < own ? lo + l : halo[(size_t)(l - own)]; };
    auto take = [&](const double *src, int w, std::vector<double> &dst) {
        if (!src) return;
        dst.resize((size_t)nt * w);
        for (int64_t l = 0; l < nt; ++l)
            for (int c = 0; c < w; ++c) dst[(size_t)l * w + c] = src[global(l) * w + c];
    };
    for (int64_t l = 0; l < nt; ++l) {
        mu[(size_t)l] = p->mu_s[global(l)];
        ku[(size_t)l] = p->k_u[global(l)];
    }
    take(p->easy_axis, 3, ea);
    take(p->K_neel, 6, kn);
    take(p->k_c, 1, kc);
    take(p->S0, 3, S0);
    take(p->pos, 3, pos);
    ss_params q = *p;
    q.n = nt;
    q.row_ptr = rp.data();
    q.col = col.data();
    q.J = J.data();
    q.mu_s = mu.data();
    q.k_u = ku.data();
    q.easy_axis = p->easy_axis ? ea.data() : nullptr;
    q.K_neel = p->K_neel ? kn.data() : nullptr;
    q.k_c = p->k_c ? kc.data() : nullptr;
    q.S0 = p->S0 ? S0.data() : nullptr;
    q.pos = p->pos ? pos.data() : nullptr;
    q.flags &= ~(uint32_t)SS_FLAG_CHECK_SYMMETRY;  // the local list is one-sided at the halo
    const SlabInit init{own, lo, &edge};
    ss_system *h = nullptr;
    st = create_impl(&q, 1, &h, &init);
    if (st != SS_OK) return st;
    h->slab_lo = lo;
    h->slab_hi = hi;
    h->nslabs = nslabs;
    h->slab_index = slab;
    for (size_t r = 0; r < halo.size();) {  // maximal runs of consecutive global indices
        size_t e = r + 1;
        while (e < halo.size() && halo[e] == halo[e - 1] + 1) ++e;
        h->slab_runs.push_back(halo[r]);
        h->slab_runs.push_back((int64_t)(e - r));
        h->slab_runs.push_back(own + (int64_t)r);
        r = e;
    }
    *out = h;
    return SS_OK;
}

ss_status spin_slab_info(ss_system *h, ss_slab_info *o) {
    if (!h || !o) return fail(h, SS_ERR_INVALID_ARG, "NULL argument");
    if (h->slab_own < 0) return fail(h, SS_ERR_INVALID_ARG, "not a slab handle");
    o->lo = h->slab_lo;
    o->hi = h->slab_hi;
    o->n_halo = h->n - h->slab_own;
    o->num_runs = (int64_t)h->slab_runs.size() / 3;
    o->boundary_tiles = h->slab_boundary_tiles;
    o->num_tiles = h->ntiles;
    o->nslabs = h->nslabs;
    o->slab = h->slab_index;
    return SS_OK;
}

ss_status spin_slab_halo_runs(ss_system *h, int64_t *out3, int64_t cap) {
    if (!h || !out3) return fail(h, SS_ERR_INVALID_ARG, "NULL argument");
    if (h->slab_own < 0) return fail(h, SS_ERR_INVALID_ARG, "not a slab handle");
    const int64_t nr = (int64_t)h->slab_runs.size() / 3;
    if (cap < nr) return fail(h, SS_ERR_INVALID_ARG, "cap %lld below the %lld runs", (long long)cap, (long long)nr);
    std::copy(h->slab_runs.begin(), h->slab_runs.end(), out3);
    return SS_OK;
}

ss_status get_state_device(ss_system *h, int32_t which, const void **x, const void **y, const void **z) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (which < 0 || which > 1 || !x || !y || !z) return fail(h, SS_ERR_INVALID_ARG, "which must be 0 or 1");
    *x = h->state[3 * which];
    *y = h->state[3 * which + 1];
    *z = h->state[3 * which + 2];
    return SS_OK;
}

ss_status spin_system_heun_pass(ss_system *h, int32_t pass, int64_t tile0, int64_t ntiles) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (pass < 0 || pass > 2) return fail(h, SS_ERR_INVALID_ARG, "pass must be 0, 1 or 2");
    if (tile0 < 0 || ntiles < 0 || tile0 + ntiles > h->ntiles)
        return fail(h, SS_ERR_INVALID_ARG, "tiles [%lld, %lld) outside [0, %lld)", (long long)tile0,
                    (long long)(tile0 + ntiles), (long long)h->ntiles);
    if (h->rows || h->demag_on) return fail(h, SS_ERR_UNSUPPORTED, "passes take thread-per-row exchange, no demag");
    return h->precision == SS_FP32_MIXED ? heun_pass_impl<float>(h, pass, tile0, ntiles)
                                         : heun_pass_impl<double>(h, pass, tile0, ntiles);
}

ss_status spin_system_info(ss_system *h, ss_info *o) {
    if (!h || !o) return fail(h, SS_ERR_INVALID_ARG, "NULL argument");
    o->n = h->n;
    o->nnz = h->nnz;
    o->num_systems = h->nsys;
    o->num_materials = h->nmat;
    o->precision = h->precision;
    o->exec = h->exec;
    o->block = h->block;
    o->tile = h->tile;
    o->num_tiles = h->ntiles;
    o->step = h->step;
    o->record_capacity = h->rec_cap;
    o->device_bytes = (int64_t)h->device_bytes;
    o->draw_ahead = h->ahead_q;
    o->exchange_rows = h->rows ? (h->sell ? 3 : 2) : 1;
    o->row_patterns = h->use_pat ? h->npat : 0;
    o->gaussian_pass = split_step(h) ? h->gauss_mode : 0;
    return SS_OK;
}

ss_status spin_system_time_kernels(ss_system *h, int32_t nsteps, double out_ms[3]) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (h->slab_own >= 0) return fail(h, SS_ERR_UNSUPPORTED, "not available on a slab handle");
    if (nsteps < 1 || !out_ms) return fail(h, SS_ERR_INVALID_ARG, "nsteps >= 1 and out_ms needed");
    double t[4];
    st = h->precision == SS_FP32_MIXED ? time_kernels_impl<float>(h, nsteps, t) : time_kernels_impl<double>(h, nsteps, t);
    out_ms[0] = t[0] + t[1];  // the Gaussian pass (split step) counted with the predictor
    out_ms[1] = t[2];
    out_ms[2] = t[3];
    return st;
}

ss_status spin_system_time_passes(ss_system *h, int32_t nsteps, double out_ms[4]) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (h->slab_own >= 0) return fail(h, SS_ERR_UNSUPPORTED, "not available on a slab handle");
    if (nsteps < 1 || !out_ms) return fail(h, SS_ERR_INVALID_ARG, "nsteps >= 1 and out_ms needed");
    return h->precision == SS_FP32_MIXED ? time_kernels_impl<float>(h, nsteps, out_ms)
                                         : time_kernels_impl<double>(h, nsteps, out_ms);
}

ss_status spin_system_time_rows(ss_system *h, int32_t launches, double *out_ms) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (launches < 1 || !out_ms) return fail(h, SS_ERR_INVALID_ARG, "launches >= 1 and out_ms needed");
    if (!h->rows) return fail(h, SS_ERR_STATE, "the handle sums a thread per exchange row");
    cudaEvent_t e0, e1;
    SS_CUDA(h, cudaEventCreate(&e0));
    SS_CUDA(h, cudaEventCreate(&e1));
    const int gr = rows_grid(h);
    cudaError_t e = cudaEventRecord(e0, h->stream);
    for (int32_t k = 0; k < launches && e == cudaSuccess; ++k) {
        if (h->precision == SS_FP32_MIXED) {
            KArgs<float> a = make_args<float>(h);
            use_rows(h, a);
            e = launch_rows_field<float>(a, a.sx, a.sy, a.sz, gr, h->stream);
        } else {
            KArgs<double> a = make_args<double>(h);
            use_rows(h, a);
            e = launch_rows_field<double>(a, a.sx, a.sy, a.sz, gr, h->stream);
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(h, e, "exchange pass timing");
    *out_ms = ms / launches;
    return SS_OK;
}

// The autotune cache (SPINSYS_AUTOTUNE_CACHE): one line per tuned workload, "key<TAB>exec block
// tile draw-ahead", the key naming the device and what the launch shape depends on.
static std::string autotune_key(const ss_system *h) {
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, h->device) != cudaSuccess) cudaGetLastError();
    int64_t nmax = 0;
    for (int64_t v : h->sys_n) nmax = std::max(nmax, v);
    char buf[512];
    std::snprintf(buf, sizeof(buf), "v2|%s|%d|%lld|%lld|%d|%lld|%d|%d", prop.name, h->precision, (long long)h->n,
                  (long long)h->nnz, h->nsys, (long long)nmax, h->rows ? (h->sell ? 3 : 2) : 1, step_mode(h));
    for (char *c = buf; *c; ++c)
        if (*c == '\t' || *c == '\n') *c = ' ';
    return buf;
}

static bool autotune_lookup(const std::string &path, const std::string &key, int v[5]) {
    FILE *f = std::fopen(path.c_str(), "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        char *tab = std::strchr(line, '\t');
        if (!tab || std::string(line, (size_t)(tab - line)) != key) continue;
        found = std::sscanf(tab + 1, "%d %d %d %d %d", &v[0], &v[1], &v[2], &v[3], &v[4]) == 5;  // the last entry wins
    }
    std::fclose(f);
    return found;
}

ss_status spin_system_autotune(ss_system *h, int32_t trial_steps, ss_info *out_info) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (h->slab_own >= 0) return fail(h, SS_ERR_UNSUPPORTED, "not available on a slab handle");
    if (trial_steps < 1) return fail(h, SS_ERR_INVALID_ARG, "trial_steps must be >= 1");
    st = check_device_flags(h);
    if (st != SS_OK) return st;
    const char *cache = std::getenv("SPINSYS_AUTOTUNE_CACHE");
    const std::string key = cache && *cache ? autotune_key(h) : std::string();
    if (!key.empty()) {
        int v[5];
        if (autotune_lookup(cache, key, v) && v[3] >= 0 && v[3] <= 8 && v[4] >= 0 && v[4] <= 2) {
            h->ahead_q = v[3];
            st = spin_system_set_gaussian_pass(h, v[4]);
            if (st == SS_OK) st = spin_system_set_launch(h, v[1], v[2]);
            if (st == SS_OK) st = spin_system_set_exec(h, (ss_exec)v[0]);
            if (st == SS_OK) return out_info ? spin_system_info(h, out_info) : SS_OK;
            h->bad = false;  // a stale entry: tune afresh
        }
    }
    const size_t rs = real_size(h);
    const int64_t n = h->n;
    const int64_t step0 = h->step;
    void *save = nullptr;
    SS_CUDA(h, dalloc(h, &save, 3 * (size_t)n * rs));
    for (int c = 0; c < 3; ++c)
        SS_CUDA(h, cudaMemcpyAsync((char *)save + c * n * rs, h->state[c], n * rs, cudaMemcpyDeviceToDevice, h->stream));
    struct Cand { int exec, block, tile, ahead, gauss; };
    std::vector<Cand> cands;
    const bool mixed = h->precision == SS_FP32_MIXED;
    // 128-thread blocks, with up to four spins per thread, for systems of at most 4,096 spins
    // per SM: a small system spread over twice the SMs has twice the FP64 lanes for its thermal
    // draws, and a mid-sized one (the 20 nm core-shell sphere, 2,518 spins per SM) keeps every
    // SM busy while each tile's record reduction is shared by four spins per thread (0.045
    // against 0.051 ms per step with one spin per thread of 256-thread blocks)
    const bool medium = n <= (int64_t)h->sm_count * 4096;
    // single- and two-warp blocks for systems of at most 64 spins per SM: one warp per SM
    const bool tiny = n <= (int64_t)h->sm_count * 64;
    for (int b : {32, 64, 128, 256, 512})
        for (int m : {1, 2, 4, 8})
            for (int q : {4, 5, 6}) {
                if (!mixed && q != 6) continue;  // no draw-ahead in the FP64 form
                if (b == 128 && (!medium || m > 4)) continue;
                if (b <= 64 && (!tiny || m > 2)) continue;
                cands.push_back({SS_EXEC_GRAPH, b, b * m, q, 0});
                cands.push_back({SS_EXEC_PERSISTENT, b, b * m, q, 0});
            }
    // the split step (a Gaussian pass, then the lean Heun passes)
    if (mixed && !h->rows)
        for (int b : {256, 512})
            for (int m : {4, 8}) cands.push_back({SS_EXEC_GRAPH, b, b * m, h->ahead_q, 1});
    // whole systems per block pays when every system fits a few blocks' worth of threads
    int64_t biggest = 0;
    for (int64_t v : h->sys_n) biggest = std::max(biggest, v);
    if (biggest <= 16384)
        for (int b : {128, 256, 512}) cands.push_back({SS_EXEC_SYSTEM_BLOCKS, b, b, h->ahead_q, 0});
    // one small system in one thread-block cluster
    if (!cluster_ready(h)) cands.push_back({SS_EXEC_CLUSTER, h->block, h->tile, h->ahead_q, 0});
    cudaEvent_t e0, e1;
    SS_CUDA(h, cudaEventCreate(&e0));
    SS_CUDA(h, cudaEventCreate(&e1));
    float best = 1e30f;
    Cand bestc{h->exec, h->block, h->tile, h->ahead_q, h->gauss_mode};
    for (const Cand &c : cands) {
        h->ahead_q = c.ahead;
        if (spin_system_set_gaussian_pass(h, c.gauss) != SS_OK) { h->bad = false; continue; }
        if (spin_system_set_launch(h, c.block, c.tile) != SS_OK) continue;
        if (spin_system_set_exec(h, (ss_exec)c.exec) != SS_OK) continue;
        if (llg_heun_step(h, std::min(trial_steps, 4)) != SS_OK) { h->bad = false; continue; }
        // the shorter of two timed runs: one run of a few steps of a small system is noisy
        float ms = 1e30f;
        bool ok = true;
        for (int r = 0; r < 2 && ok; ++r) {
            cudaEventRecord(e0, h->stream);
            if (llg_heun_step(h, trial_steps) != SS_OK) { h->bad = false; ok = false; break; }
            cudaEventRecord(e1, h->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) { cudaGetLastError(); ok = false; break; }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            ms = std::min(ms, t);
        }
        if (!ok || check_device_flags(h) != SS_OK) continue;
        if (ms < best) {
            best = ms;
            bestc = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->ahead_q = bestc.ahead;
    st = spin_system_set_gaussian_pass(h, bestc.gauss);
    if (st == SS_OK) st = spin_system_set_launch(h, bestc.block, bestc.tile);
    if (st == SS_OK) st = spin_system_set_exec(h, (ss_exec)bestc.exec);
    for (int c = 0; c < 3; ++c)
        SS_CUDA(h, cudaMemcpyAsync(h->state[c], (char *)save + c * n * rs, n * rs, cudaMemcpyDeviceToDevice, h->stream));
    SS_CUDA(h, cudaStreamSynchronize(h->stream));
    dfree(h, save);
    if (st == SS_OK) st = set_step(h, step0);
    if (st == SS_OK && !key.empty()) {
        if (FILE *f = std::fopen(cache, "a")) {
            std::fprintf(f, "%s\t%d %d %d %d %d\n", key.c_str(), h->exec, h->block, h->tile, h->ahead_q,
                         h->gauss_mode);
            std::fclose(f);
        }
    }
    if (st == SS_OK && out_info) st = spin_system_info(h, out_info);
    return st;
}

ss_status spin_system_set_barrier_test(ss_system *h, int32_t extra, int64_t timeout_ns) {
    ss_status st = usable(h);
    if (st != SS_OK) return st;
    if (extra < 0 || timeout_ns < 1000) return fail(h, SS_ERR_INVALID_ARG, "extra >= 0 and timeout_ns >= 1000 needed");
    h->bar_extra = (unsigned int)extra;
    h->bar_timeout_ns = extra ? timeout_ns : 2000000000ll;
    if (!extra && timeout_ns != 2000000000ll) h->bar_timeout_ns = timeout_ns;
    drop_graph(h);
    return SS_OK;
}

ss_status ss_debug_fail_allocations(int64_t after) {
    g_fail_after.store(after < 0 ? -1 : after);
    return SS_OK;
}

int64_t ss_debug_live_bytes(void) { return g_live_bytes.load(); }

ss_status ss_debug_philox(const uint32_t ctr0[4], const uint32_t key[2], int64_t count, uint32_t *out) {
    if (!ctr0 || !key || !out || count < 0) return fail(nullptr, SS_ERR_INVALID_ARG, "bad arguments");
    uint32_t *d = nullptr;
    cudaError_t e = cudaMalloc(&d, (size_t)std::max<int64_t>(count, 1) * 16);
    if (e == cudaSuccess) e = launch_debug_philox(ctr0, key, count, d, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, d, (size_t)count * 16, cudaMemcpyDeviceToHost);
    if (d) cudaFree(d);
    return e == cudaSuccess ? SS_OK : fail(nullptr, SS_ERR_CUDA, "%s", cudaGetErrorString(e));
}

ss_status ss_debug_gaussians(uint64_t seed, uint32_t sys, uint32_t step, int64_t n, int32_t mode, double *out) {
    if (!out || n < 0 || mode < 0 || mode > 4) return fail(nullptr, SS_ERR_INVALID_ARG, "bad arguments");
    std::vector<double2> tab;
    build_tables(tab);
    double2 *dt = nullptr;
    double *d = nullptr;
    cudaError_t e = cudaMalloc(&dt, tab.size() * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&d, (size_t)std::max<int64_t>(n, 1) * 3 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(dt, tab.data(), tab.size() * sizeof(double2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = launch_debug_gaussians(seed, sys, step, n, mode, dt, d, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, d, (size_t)n * 3 * sizeof(double), cudaMemcpyDeviceToHost);
    if (d) cudaFree(d);
    if (dt) cudaFree(dt);
    return e == cudaSuccess ? SS_OK : fail(nullptr, SS_ERR_CUDA, "%s", cudaGetErrorString(e));
}

ss_status ss_debug_fp64_rate(int32_t mode, double *inst_per_s) {
    if (!inst_per_s || mode < 0 || mode > 2) return fail(nullptr, SS_ERR_INVALID_ARG, "bad arguments");
    const cudaError_t e = fp64_rate(mode, inst_per_s);
    return e == cudaSuccess ? SS_OK : fail(nullptr, SS_ERR_CUDA, "%s", cudaGetErrorString(e));
}

const char *ss_last_error(ss_system *h) { return h ? h->err.c_str() : g_create_error.c_str(); }

const char *ss_status_string(ss_status s) {
    switch (s) {
        case SS_OK: return "ok";
        case SS_ERR_INVALID_ARG: return "invalid argument";
        case SS_ERR_CUDA: return "CUDA error";
        case SS_ERR_OOM: return "out of memory";
        case SS_ERR_TIMEOUT: return "device wait timed out";
        case SS_ERR_NONFINITE: return "non-finite spin";
        case SS_ERR_STATE: return "handle unusable";
        case SS_ERR_UNSUPPORTED: return "unsupported";
    }
    return "unknown status";
}

}  // extern "C"
