// llg_heun_step_noalloc: the FP64 Heun step for callers that cannot allocate device
// memory.  The paper has no counterpart of this entry point.
//
// Callers such as code that lives inside a memory arena owning all device memory, loops
// that must not allocate after start-up, or hosts handed device buffers by another
// runtime cannot call cudaMalloc.  This file keeps every working buffer of the step in
// one file-scope static device array of fixed size, so the entry point allocates
// nothing: the caller passes its inputs and outputs as device pointers, and the
// predictor spins, half steps, thermal field, reduction partials and Box-Muller tables
// live in `g_noalloc_scratch`.
//
// In host code the name g_noalloc_scratch is only a host-side stand-in for the device
// array; its device address is obtained with cudaGetSymbolAddress on every call (the tables
// are uploaded again whenever the address differs from the last one seen on the device) and
// passed to the kernels.  Calls share the array; calls that overlap on the GPU race.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "../../include/spinsys.h"
#include "ss_kernels.cuh"

namespace ss {
namespace {

constexpr int64_t kNaMax = SS_NOALLOC_MAX_SPINS;
constexpr int kNaBlock = 256;
constexpr int64_t kNaTiles = (kNaMax + kNaBlock - 1) / kNaBlock;
constexpr size_t kNaTabCount = (size_t)kTabCount;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
// Layout of the static array (byte offsets, each 256-byte aligned).
constexpr size_t kNaTabOff = 0;
constexpr size_t kNaPartOff = align256(kNaTabOff + kNaTabCount * sizeof(double2));
constexpr size_t kNaStateOff = align256(kNaPartOff + (size_t)kNaTiles * kPartComps * sizeof(double));
constexpr size_t kNaBytes = kNaStateOff + 9 * (size_t)kNaMax * sizeof(double);  // S', Q, H_th (x, y, z each)

__device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Device address of g_noalloc_scratch per device ordinal at the last table upload.
std::mutex g_na_mutex;
unsigned char *g_na_base[128] = {};

struct NaArgs {
    int64_t n;
    int64_t ntiles;
    const int32_t *row_ptr;
    const int32_t *col;
    const double *J;
    const double *mu_s;
    const double *k_u;
    const double *ea;
    double *sx, *sy, *sz;
    double *px, *py, *pz;
    double *qx, *qy, *qz;
    double *hx, *hy, *hz;
    double *partials;
    double *record;  // this step's 8 doubles, or NULL
    const double2 *tab;
    double lambda, gp, dt, gamma, sig_num, sqrtT;  // sig_num = 2 lambda kB
    double H[3];
    uint32_t key0, key1, ctr2, step;
};

__device__ __forceinline__ void na_field(const NaArgs &a, int64_t i, const double *X, const double *Y,
                                         const double *Z, double s0, double s1, double s2, double &e0, double &e1,
                                         double &e2, double &H0, double &H1, double &H2) {
    const int32_t b = __ldg(a.row_ptr + i), e = __ldg(a.row_ptr + i + 1);
    double x = 0, y = 0, z = 0;
    for (int32_t k = b; k < e; ++k) {
        const int32_t j = __ldg(a.col + k);
        const double Jk = __ldg(a.J + k);
        x = fma(Jk, __ldg(X + j), x);
        y = fma(Jk, __ldg(Y + j), y);
        z = fma(Jk, __ldg(Z + j), z);
    }
    e0 = x;
    e1 = y;
    e2 = z;
    const double mu = __ldg(a.mu_s + i);
    const double im = 1.0 / mu;
    H0 = x * im;
    H1 = y * im;
    H2 = z * im;
    const double u0 = __ldg(a.ea + 3 * i), u1 = __ldg(a.ea + 3 * i + 1), u2 = __ldg(a.ea + 3 * i + 2);
    const double sde = s0 * u0 + s1 * u1 + s2 * u2;
    const double an = (2.0 * __ldg(a.k_u + i) / mu) * sde;
    H0 = fma(an, u0, H0);
    H1 = fma(an, u1, H1);
    H2 = fma(an, u2, H2);
    H0 += a.H[0];
    H1 += a.H[1];
    H2 += a.H[2];
}

__global__ void __launch_bounds__(kNaBlock) k_na_predictor(const NaArgs a) {
    __shared__ SmemTables tab;
    __shared__ double red[(kNaBlock / 32) * 8];
    stage_bm_tables(a.tab, tab);
    __syncthreads();
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int64_t i = (int64_t)blockIdx.x * kNaBlock + threadIdx.x;
    if (i < a.n) {
        const double s0 = a.sx[i], s1 = a.sy[i], s2 = a.sz[i];
        double e0, e1, e2, H0, H1, H2;
        na_field(a, i, a.sx, a.sy, a.sz, s0, s1, s2, e0, e1, e2, H0, H1, H2);
        const double mu = __ldg(a.mu_s + i);
        double t0 = 0, t1 = 0, t2 = 0;
        if (a.sqrtT > 0.0) {
            const Philox4 w = philox4x32_10((uint32_t)i, a.step, a.ctr2, 0u, a.key0, a.key1);
            double g0, g1, g2;
            box_muller3(w, tab, g0, g1, g2);
            const double sig = sqrt(a.sig_num / (a.gamma * mu * a.dt)) * a.sqrtT;
            t0 = sig * g0;
            t1 = sig * g1;
            t2 = sig * g2;
        }
        a.hx[i] = t0;
        a.hy[i] = t1;
        a.hz[i] = t2;
        H0 += t0;
        H1 += t1;
        H2 += t2;
        double d0, d1, d2;
        llg_rhs(a.gp, a.lambda, s0, s1, s2, H0, H1, H2, d0, d1, d2);
        const double v0 = fma(a.dt, d0, s0), v1 = fma(a.dt, d1, s1), v2 = fma(a.dt, d2, s2);
        const double inv = rsqrt(v0 * v0 + v1 * v1 + v2 * v2);
        a.px[i] = v0 * inv;
        a.py[i] = v1 * inv;
        a.pz[i] = v2 * inv;
        const double hdt = 0.5 * a.dt;
        a.qx[i] = fma(hdt, d0, s0);
        a.qy[i] = fma(hdt, d1, s1);
        a.qz[i] = fma(hdt, d2, s2);
        const double u0 = __ldg(a.ea + 3 * i), u1 = __ldg(a.ea + 3 * i + 1), u2 = __ldg(a.ea + 3 * i + 2);
        const double sde = s0 * u0 + s1 * u1 + s2 * u2;
        acc[0] = mu * s0;
        acc[1] = mu * s1;
        acc[2] = mu * s2;
        acc[3] = -0.5 * (s0 * e0 + s1 * e1 + s2 * e2);
        acc[4] = -__ldg(a.k_u + i) * sde * sde;
        acc[5] = -mu * (s0 * a.H[0] + s1 * a.H[1] + s2 * a.H[2]);
        acc[6] = mu;
    }
    const double r = block_sum8<kNaBlock>(acc, red);
    if (threadIdx.x < kPartComps) a.partials[(int64_t)blockIdx.x * kPartComps + threadIdx.x] = r;
}

// Block 0 sums the predictor's partials into the step's record; blocks 1.. correct.
__global__ void __launch_bounds__(kNaBlock) k_na_corrector(const NaArgs a) {
    __shared__ double red[(kNaBlock / 32) * 8];
    if (blockIdx.x == 0) {
        if (a.record == nullptr) return;
        double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t t = threadIdx.x; t < a.ntiles; t += kNaBlock)
            for (int c = 0; c < 7; ++c) acc[c] += a.partials[t * kPartComps + c];
        const double r = block_sum8<kNaBlock>(acc, red);
        __shared__ double comp[8];
        if (threadIdx.x < 8) comp[threadIdx.x] = r;
        __syncthreads();
        if (threadIdx.x == 0) {
            a.record[0] = comp[0];
            a.record[1] = comp[1];
            a.record[2] = comp[2];
            a.record[3] = comp[6];
            a.record[4] = comp[3];
            a.record[5] = comp[4];
            a.record[6] = comp[5];
            a.record[7] = (comp[3] + comp[4]) + comp[5];
        }
        return;
    }
    const int64_t i = (int64_t)(blockIdx.x - 1) * kNaBlock + threadIdx.x;
    if (i >= a.n) return;
    const double s0 = a.px[i], s1 = a.py[i], s2 = a.pz[i];
    double e0, e1, e2, H0, H1, H2;
    na_field(a, i, a.px, a.py, a.pz, s0, s1, s2, e0, e1, e2, H0, H1, H2);
    H0 += a.hx[i];
    H1 += a.hy[i];
    H2 += a.hz[i];
    double d0, d1, d2;
    llg_rhs(a.gp, a.lambda, s0, s1, s2, H0, H1, H2, d0, d1, d2);
    const double hdt = 0.5 * a.dt;
    const double v0 = fma(hdt, d0, a.qx[i]);
    const double v1 = fma(hdt, d1, a.qy[i]);
    const double v2 = fma(hdt, d2, a.qz[i]);
    const double inv = rsqrt(v0 * v0 + v1 * v1 + v2 * v2);
    a.sx[i] = v0 * inv;
    a.sy[i] = v1 * inv;
    a.sz[i] = v2 * inv;
}

ss_status na_error(ss_status s, const char *msg) {
    set_global_error(msg);
    return s;
}

// Device address of the static array on the current device, looked up on every call (no
// allocation); the tables are uploaded (synchronous copy) at the first call on the device and
// again whenever the address has changed since.
ss_status na_base(unsigned char **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_error(SS_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= 128) return na_error(SS_ERR_UNSUPPORTED, "device ordinal out of range");
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return na_error(SS_ERR_CUDA, "cudaGetSymbolAddress(g_noalloc_scratch) failed");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (g_na_base[dev] != (unsigned char *)p) {
        static double2 tab[kNaTabCount];
        build_bm_tables(tab);
        e = cudaMemcpy((unsigned char *)p + kNaTabOff, tab, sizeof(tab), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return na_error(SS_ERR_CUDA, cudaGetErrorString(e));
        g_na_base[dev] = (unsigned char *)p;
    }
    *out = g_na_base[dev];
    return SS_OK;
}

bool finite_d(double v) { return std::isfinite(v); }

}  // namespace
}  // namespace ss

extern "C" ss_status llg_heun_step_noalloc(const ss_noalloc_step *p, int64_t nsteps, void *cuda_stream) {
    using namespace ss;
    if (!p) return na_error(SS_ERR_INVALID_ARG, "llg_heun_step_noalloc: params is NULL");
    if (p->n < 1 || p->n > kNaMax) {
        char msg[160];
        std::snprintf(msg, sizeof(msg), "llg_heun_step_noalloc: n = %lld outside [1, %lld] (SS_NOALLOC_MAX_SPINS)",
                      (long long)p->n, (long long)kNaMax);
        return na_error(SS_ERR_INVALID_ARG, msg);
    }
    if (nsteps < 0) return na_error(SS_ERR_INVALID_ARG, "llg_heun_step_noalloc: nsteps < 0");
    if (!p->row_ptr || !p->col || !p->J || !p->mu_s || !p->k_u || !p->easy_axis || !p->sx || !p->sy || !p->sz)
        return na_error(SS_ERR_INVALID_ARG, "llg_heun_step_noalloc: a required device pointer is NULL");
    if (!(p->alpha >= 0.0) || !finite_d(p->alpha) || !(p->dt > 0.0) || !finite_d(p->dt) || !(p->gamma >= 0.0) ||
        !finite_d(p->gamma) || !(p->T >= 0.0) || !finite_d(p->T) || !finite_d(p->H_app[0]) ||
        !finite_d(p->H_app[1]) || !finite_d(p->H_app[2]))
        return na_error(SS_ERR_INVALID_ARG, "llg_heun_step_noalloc: alpha, dt, gamma, T or H_app out of range");
    if (p->step0 < 0) return na_error(SS_ERR_INVALID_ARG, "llg_heun_step_noalloc: step0 < 0");
    // the step index is the 32-bit Philox counter word: every step of the call must fit it
    if (p->step0 > 0xFFFFFFFFll || nsteps > 0xFFFFFFFFll - p->step0)
        return na_error(SS_ERR_INVALID_ARG, "llg_heun_step_noalloc: step0 + nsteps exceeds 2^32 - 1");
    if (nsteps == 0) return SS_OK;
    unsigned char *base = nullptr;
    ss_status st = na_base(&base);
    if (st != SS_OK) return st;
    const cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int64_t n = p->n;
    const double gamma = p->gamma > 0.0 ? p->gamma : kGammaDefault;
    NaArgs a{};
    a.n = n;
    a.ntiles = (n + kNaBlock - 1) / kNaBlock;
    a.row_ptr = p->row_ptr;
    a.col = p->col;
    a.J = p->J;
    a.mu_s = p->mu_s;
    a.k_u = p->k_u;
    a.ea = p->easy_axis;
    a.sx = p->sx;
    a.sy = p->sy;
    a.sz = p->sz;
    double *state = reinterpret_cast<double *>(base + kNaStateOff);
    double *bufs[9];
    for (int b = 0; b < 9; ++b) bufs[b] = state + (size_t)b * kNaMax;
    a.px = bufs[0]; a.py = bufs[1]; a.pz = bufs[2];
    a.qx = bufs[3]; a.qy = bufs[4]; a.qz = bufs[5];
    a.hx = bufs[6]; a.hy = bufs[7]; a.hz = bufs[8];
    a.partials = reinterpret_cast<double *>(base + kNaPartOff);
    a.tab = reinterpret_cast<const double2 *>(base + kNaTabOff);
    a.lambda = p->alpha;
    a.gp = gamma / (1.0 + p->alpha * p->alpha);
    a.dt = p->dt;
    a.gamma = gamma;
    a.sig_num = 2.0 * p->alpha * kBoltzmann;
    a.sqrtT = std::sqrt(p->T);
    for (int c = 0; c < 3; ++c) a.H[c] = p->H_app[c];
    a.key0 = (uint32_t)(p->seed & 0xffffffffull);
    a.key1 = (uint32_t)(p->seed >> 32);
    a.ctr2 = p->sys_id;
    const int grid = (int)a.ntiles;
    for (int64_t k = 0; k < nsteps; ++k) {
        a.step = (uint32_t)(p->step0 + k);
        a.record = p->record ? p->record + 8 * k : nullptr;
        k_na_predictor<<<grid, kNaBlock, 0, s>>>(a);
        k_na_corrector<<<grid + 1, kNaBlock, 0, s>>>(a);
        if (k == 0 || k + 1 == nsteps) {  // a launch failure stops the call at the first step
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return na_error(SS_ERR_CUDA, cudaGetErrorString(e));
        }
    }
    return SS_OK;
}
