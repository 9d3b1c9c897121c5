// Precision-independent kernels: the per-system finalisation of on-demand measurements
// and the diagnostic Philox / Gaussian kernels used by the tests.
#include <cmath>
#include <cstring>

#include "ss_ff.cuh"
#include "ss_kernels.cuh"

namespace ss {

__global__ void k_advance_step(unsigned long long *step) { *step += 1ull; }

cudaError_t launch_advance_step(unsigned long long *step, cudaStream_t s) {
    k_advance_step<<<1, 1, 0, s>>>(step);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const SysDesc *sys, const int32_t *sys_tiles, int nsys, const double *partials,
                            double *dst, cudaStream_t s) {
    const int grid = nsys < 1024 ? nsys : 1024;
    k_finalize<256><<<grid > 0 ? grid : 1, 256, 0, s>>>(sys, sys_tiles, nsys, partials, dst);
    return cudaGetLastError();
}

cudaError_t launch_finalize_ring(const SysDesc *sys, const int32_t *sys_tiles, int nsys, const double *partials,
                                 double *rec, int64_t rec_cap, const unsigned long long *step, cudaStream_t s) {
    const int grid = nsys < 1024 ? nsys : 1024;
    k_finalize_ring<256><<<grid > 0 ? grid : 1, 256, 0, s>>>(sys, sys_tiles, nsys, partials, rec, rec_cap, step);
    return cudaGetLastError();
}

__global__ void k_debug_philox(uint4 ctr0, uint2 key, long long count, uint32_t *out) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x) {
        const Philox4 w = philox4x32_10(ctr0.x + (uint32_t)k, ctr0.y, ctr0.z, ctr0.w, key.x, key.y);
        out[4 * k + 0] = w.w0;
        out[4 * k + 1] = w.w1;
        out[4 * k + 2] = w.w2;
        out[4 * k + 3] = w.w3;
    }
}

cudaError_t launch_debug_philox(const uint32_t *ctr0, const uint32_t *key, long long count, uint32_t *out,
                                cudaStream_t s) {
    const uint4 c = make_uint4(ctr0[0], ctr0[1], ctr0[2], ctr0[3]);
    const uint2 k = make_uint2(key[0], key[1]);
    k_debug_philox<<<256, 256, 0, s>>>(c, k, count, out);
    return cudaGetLastError();
}

// mode 0: the FP64 form's table-driven transform; mode 1: CUDA's log/sqrt/sincospi.
__global__ void k_debug_gaussians(uint64_t seed, uint32_t sys, uint32_t step, long long n, int mode,
                                  const double2 *tabs, double *out) {
    __shared__ SmemTables tab;
    stage_bm_tables(tabs, tab);
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const Philox4 w = philox4x32_10((uint32_t)i, step, sys, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
        double g0, g1, g2;
        if (mode == 0) {
            box_muller3(w, tab, g0, g1, g2);
        } else {
            box_muller3_libm(w, g0, g1, g2);
        }
        out[3 * i + 0] = g0;
        out[3 * i + 1] = g1;
        out[3 * i + 2] = g2;
    }
}

// The FP32-mixed form's transform.  mode 2: the Gaussians the step kernels use (rounded to
// float, uncertain roundings resolved by the FP64 transform); mode 3: the double-float values
// hi + lo before rounding; mode 4: 1 where a rounding of the draw was uncertain, else 0 (in
// the first of the three slots).
__global__ void k_debug_gaussians_ff(uint64_t seed, uint32_t sys, uint32_t step, long long n, int mode,
                                     const double2 *tabs, double *out) {
    __shared__ FFTables tab;
    stage_ff_tables(reinterpret_cast<const float4 *>(tabs + kTabCount), tab);
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const Philox4 w = philox4x32_10((uint32_t)i, step, sys, 0u, (uint32_t)seed, (uint32_t)(seed >> 32));
        double v[3] = {0.0, 0.0, 0.0};
        if (mode == 2) {
            float g0, g1, g2;
            gaussians_f32(w, tab, tabs, g0, g1, g2);
            v[0] = g0;
            v[1] = g1;
            v[2] = g2;
        } else {
            const FF R1 = ff_sqrt(ff_neg2log(w.w0, tab));
            const FF R2 = ff_sqrt(ff_neg2log(w.w2, tab));
            float g[3];
            const bool ok = box_muller3_ff(w, tab, g[0], g[1], g[2]);
            if (mode == 4) {
                v[0] = ok ? 0.0 : 1.0;
            } else {
                // the unrounded double-float products, as box_muller3_ff forms them
                const FFTurn a = ff_turn(w.w1, tab);
                const FF sb = ff_rot(a.tv.x, a.tv.y, a.tv.z, a.tv.w, a);
                const FF cb = ff_rot(a.tv.z, a.tv.w, -a.tv.x, -a.tv.y, a);
                const bool swap = ((a.o + 1u) >> 1) & 1u;
                FF S = swap ? cb : sb, Co = swap ? sb : cb;
                if (a.o & 4u) S = ff_neg(S);
                if ((a.o + 2u) & 4u) Co = ff_neg(Co);
                const FFTurn b = ff_turn(w.w3, tab);
                const bool swap2 = ((b.o + 1u) >> 1) & 1u;
                FF C2 = swap2 ? ff_rot(b.tv.x, b.tv.y, b.tv.z, b.tv.w, b)
                              : ff_rot(b.tv.z, b.tv.w, -b.tv.x, -b.tv.y, b);
                if ((b.o + 2u) & 4u) C2 = ff_neg(C2);
                const FF R[3] = {R1, R1, R2}, V[3] = {Co, S, C2};
                for (int c = 0; c < 3; ++c) {
                    const float gh = __fmul_rn(R[c].hi, V[c].hi);
                    const float ge = __fadd_rn(fmaf(R[c].hi, V[c].hi, -gh), fmaf(R[c].hi, V[c].lo, __fmul_rn(R[c].lo, V[c].hi)));
                    v[c] = (double)gh + (double)ge;
                }
            }
        }
        out[3 * i + 0] = v[0];
        out[3 * i + 1] = v[1];
        out[3 * i + 2] = v[2];
    }
}

cudaError_t launch_debug_gaussians(uint64_t seed, uint32_t sys, uint32_t step, long long n, int mode,
                                   const double2 *tab, double *out, cudaStream_t s) {
    if (mode <= 1)
        k_debug_gaussians<<<256, 256, 0, s>>>(seed, sys, step, n, mode, tab, out);
    else
        k_debug_gaussians_ff<<<256, 256, 0, s>>>(seed, sys, step, n, mode, tab, out);
    return cudaGetLastError();
}

// Box-Muller tables (layout in SmemTables), evaluated in long double.  The log and ln 2
// constants are split as 2^-45 M + remainder with M an integer stored in the bits of a
// double slot (so is the 21-bit reciprocal C); the remainders of the log table are floats
// packed after the trig table.
void build_bm_tables(double2 *t) {
    const long double q = 35184372088832.0L;  // 2^45
    float *lolog = reinterpret_cast<float *>(t + kLogTab + kLn2Tab + kTrigTab);
    for (int i = 0; i < 4 * kLogLo; ++i) lolog[i] = 0.0f;
    for (int i = 0; i < kLogTab; ++i) {
        // 1/c = kLogScale / j rounded to 21 bits: C 2^-20, C = round(2^20 kLogScale / j)
        const long long j = kLogFirst + i;
        const long long C = ((2ll << 20) * kLogScale / j + 1) / 2;
        const long double T = -2.0L * logl((long double)C / 1048576.0L);
        const long long M = llroundl(T * q);
        double cbits, mbits;
        std::memcpy(&cbits, &C, sizeof(cbits));
        std::memcpy(&mbits, &M, sizeof(mbits));
        t[i] = make_double2(cbits, mbits);
        lolog[i] = (float)(T - (long double)M / q);
    }
    const long double ln2 = 0.693147180559945309417232121458176568L;
    for (int i = 0; i < kLn2Tab; ++i) {
        const long double v = 2.0L * (long double)i * ln2;
        const long long N = llroundl(v * q);
        double nbits;
        std::memcpy(&nbits, &N, sizeof(nbits));
        t[kLogTab + i] = make_double2(nbits, (double)(v - (long double)N / q));
    }
    const long double twopi = 6.283185307179586476925286766559005768L;
    for (int j = 0; j < kTrigTab; ++j) {
        const long double a = twopi * (long double)j / 4096.0L;  // first octant of 4096 points
        t[kLogTab + kLn2Tab + j] = make_double2((double)sinl(a), (double)cosl(a));
    }
}

// Double-float tables of the FP32-mixed transform (layout in FFTables), evaluated in long
// double and split as hi = the value rounded to float, lo = the remainder rounded to float.
void build_ff_tables(float4 *t) {
    auto split = [](long double v, float &hi, float &lo) {
        hi = (float)v;
        lo = (float)(v - (long double)hi);
    };
    for (int i = 0; i < kLogTab; ++i) {
        const long double c = (long double)(kLogFirst + i) / (long double)kLogScale;
        split(1.0L / c, t[i].x, t[i].y);
        split(-2.0L * logl(c), t[i].z, t[i].w);
    }
    const long double twopi = 6.283185307179586476925286766559005768L;
    for (int m = 0; m < kTrigTab; ++m) {
        const long double a = twopi * (long double)m / 4096.0L;  // first octant of 4096 points
        float4 &e = t[kLogTab + m];
        split(sinl(a), e.x, e.y);
        split(cosl(a), e.z, e.w);
    }
    const long double ln2 = 0.693147180559945309417232121458176568L;
    float *l2 = reinterpret_cast<float *>(t + kLogTab + kTrigTab);
    for (int i = 0; i < 4 * ((kLn2Tab + 1) / 2); ++i) l2[i] = 0.0f;
    for (int n = 0; n < kLn2Tab; ++n) split(2.0L * (long double)n * ln2, l2[2 * n], l2[2 * n + 1]);
}

// FP64 instruction throughput probe: eight independent chains per thread.  mode 0: DFMA
// with the multiplier and addend shared by all chains; mode 1: DFMA with three distinct
// register operands (the pattern of general code); mode 2: DADD.
template <int MODE>
__global__ void k_fp64_rate(double *out, int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-3 + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (MODE == 0) x[k] = fma(x[k], a, b);
            else if (MODE == 1) x[k] = fma(x[k], x[(k + 1) & 7], (k & 1) ? a : b);
            else x[k] = x[k] + ((k & 1) ? a : b);
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FP64 instructions per second of the probe (grid: 4 blocks of 256 threads per SM).
cudaError_t fp64_rate(int mode, double *inst_per_s) {
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    if (e != cudaSuccess) return e;
    const int block = 256, grid = 4 * sms, iters = 4096, reps = 5;
    double *out = nullptr;
    e = cudaMalloc(&out, sizeof(double) * (size_t)grid * block);
    if (e != cudaSuccess) return e;
    auto launch = [&]() {
        if (mode == 0) k_fp64_rate<0><<<grid, block>>>(out, iters, 0.999, 1e-3);
        else if (mode == 1) k_fp64_rate<1><<<grid, block>>>(out, iters, 0.999, 1e-3);
        else k_fp64_rate<2><<<grid, block>>>(out, iters, 0.999, 1e-3);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch();
    cudaEventRecord(e0);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e == cudaSuccess) *inst_per_s = (double)reps * grid * block * iters * 8.0 / (ms * 1e-3);
    return e;
}

}  // namespace ss
