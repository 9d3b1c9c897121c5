// Host launchers of the step kernels for one working type; included by
// ss_kernels_f32.cu and ss_kernels_f64.cu (one translation unit per precision).
#pragma once

#include "ss_kernels.cuh"

namespace ss {

#define SS_BLOCK_SWITCH(block, ...)                      \
    switch (block) {                                     \
        case 32: { constexpr int BS = 32; __VA_ARGS__; } break; \
        case 64: { constexpr int BS = 64; __VA_ARGS__; } break; \
        case 128: { constexpr int BS = 128; __VA_ARGS__; } break; \
        case 256: { constexpr int BS = 256; __VA_ARGS__; } break; \
        case 512: { constexpr int BS = 512; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;           \
    }

// The Heun step-kernel variant for these arguments: kRows, kGeneral, kUniform (plain lattice,
// one material) or kPlain.
template <typename R>
int heun_mode(const KArgs<R> &a) {
    if (a.ex) return kRows;
    if (a.J_tensor || a.any_cubic) return kGeneral;
    return a.mat_uniform ? kUniform : kPlain;
}

template <typename R>
cudaError_t launch_predictor(const KArgs<R> &a, int block, int grid, cudaStream_t s) {
    switch (heun_mode(a)) {
        case kRows: SS_BLOCK_SWITCH(block, k_predictor<R, BS, kRows><<<grid, BS, 0, s>>>(a)); break;
        case kGeneral: SS_BLOCK_SWITCH(block, k_predictor<R, BS, kGeneral><<<grid, BS, 0, s>>>(a)); break;
        case kUniform: SS_BLOCK_SWITCH(block, k_predictor<R, BS, kUniform><<<grid, BS, 0, s>>>(a)); break;
        default: SS_BLOCK_SWITCH(block, k_predictor<R, BS, kPlain><<<grid, BS, 0, s>>>(a)); break;
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_corrector(const KArgs<R> &a, int block, int grid, int nfin, cudaStream_t s) {
    const int mode = heun_mode(a);
    const bool ahead = a.g_step != nullptr;
#define SS_CORRECTOR(DA, MODE) SS_BLOCK_SWITCH(block, k_corrector<R, BS, DA, MODE><<<grid + nfin, BS, 0, s>>>(a, nfin))
    if (mode == kRows) {
        if (ahead) { SS_CORRECTOR(true, kRows); } else { SS_CORRECTOR(false, kRows); }
    } else if (mode == kGeneral) {
        if (ahead) { SS_CORRECTOR(true, kGeneral); } else { SS_CORRECTOR(false, kGeneral); }
    } else if (mode == kUniform) {
        if (ahead) { SS_CORRECTOR(true, kUniform); } else { SS_CORRECTOR(false, kUniform); }
    } else {
        if (ahead) { SS_CORRECTOR(true, kPlain); } else { SS_CORRECTOR(false, kPlain); }
    }
#undef SS_CORRECTOR
    return cudaGetLastError();
}

// The split FP32-mixed step (a Gaussian pass, then the two Heun passes reading it): variants
// kUniform, kPlain and kGeneral of the thread-per-row exchange sum.
// priority: the launch's scheduling priority (cudaLaunchAttributePriority; 0 = the stream's)
template <typename R>
cudaError_t launch_gauss(const KArgs<R> &a, int block, int grid, cudaStream_t s, int priority) {
    if constexpr (sizeof(R) == 4) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributePriority;
        attr[0].val.priority = priority;
        cfg.attrs = attr;
        cfg.numAttrs = priority ? 1 : 0;
        switch (block) {
            case 32: cfg.blockDim = dim3(32); return cudaLaunchKernelEx(&cfg, k_gauss<32>, a);
            case 64: cfg.blockDim = dim3(64); return cudaLaunchKernelEx(&cfg, k_gauss<64>, a);
            case 128: cfg.blockDim = dim3(128); return cudaLaunchKernelEx(&cfg, k_gauss<128>, a);
            case 256: cfg.blockDim = dim3(256); return cudaLaunchKernelEx(&cfg, k_gauss<256>, a);
            case 512: cfg.blockDim = dim3(512); return cudaLaunchKernelEx(&cfg, k_gauss<512>, a);
            default: return cudaErrorInvalidValue;
        }
    } else {
        return cudaErrorNotSupported;
    }
}

template <typename R>
cudaError_t launch_gstep_sync(const KArgs<R> &a, cudaStream_t s) {
    k_gstep_sync<<<1, 1, 0, s>>>(a.gstep, a.step);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_predictor_split(const KArgs<R> &a, int block, int grid, cudaStream_t s) {
    if constexpr (sizeof(R) == 4) {
        switch (heun_mode(a)) {
            case kGeneral: SS_BLOCK_SWITCH(block, k_predictor_split<R, BS, kGeneral><<<grid, BS, 0, s>>>(a)); break;
            case kUniform: SS_BLOCK_SWITCH(block, k_predictor_split<R, BS, kUniform><<<grid, BS, 0, s>>>(a)); break;
            case kPlain: SS_BLOCK_SWITCH(block, k_predictor_split<R, BS, kPlain><<<grid, BS, 0, s>>>(a)); break;
            default: return cudaErrorNotSupported;
        }
        return cudaGetLastError();
    } else {
        return cudaErrorNotSupported;
    }
}

template <typename R>
cudaError_t launch_corrector_split(const KArgs<R> &a, int block, int grid, int nfin, cudaStream_t s) {
    if constexpr (sizeof(R) == 4) {
        switch (heun_mode(a)) {
            case kGeneral:
                SS_BLOCK_SWITCH(block, k_corrector_split<R, BS, kGeneral><<<grid + nfin, BS, 0, s>>>(a, nfin));
                break;
            case kUniform:
                SS_BLOCK_SWITCH(block, k_corrector_split<R, BS, kUniform><<<grid + nfin, BS, 0, s>>>(a, nfin));
                break;
            case kPlain:
                SS_BLOCK_SWITCH(block, k_corrector_split<R, BS, kPlain><<<grid + nfin, BS, 0, s>>>(a, nfin));
                break;
            default: return cudaErrorNotSupported;
        }
        return cudaGetLastError();
    } else {
        return cudaErrorNotSupported;
    }
}

// Resident blocks per SM of the split step's kernels: which = 0 the Gaussian pass, 1 the
// predictor, 2 the corrector, in the variant `mode` (1 general, 3 uniform, else plain).
template <typename R>
int split_blocks_per_sm(int block, int mode, int which) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if constexpr (sizeof(R) == 4) {
#define SS_OCC(MODE)                                                                                                  \
    if (which == 0) {                                                                                                 \
        SS_BLOCK_SWITCH(block, e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gauss<BS>, BS, 0));           \
    } else if (which == 1) {                                                                                          \
        SS_BLOCK_SWITCH(block, e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_predictor_split<R, BS, MODE>, \
                                                                                 BS, 0));                             \
    } else {                                                                                                          \
        SS_BLOCK_SWITCH(block, e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_corrector_split<R, BS, MODE>, \
                                                                                 BS, 0));                             \
    }
        if (mode == kGeneral) {
            SS_OCC(kGeneral)
        } else if (mode == kUniform) {
            SS_OCC(kUniform)
        } else {
            SS_OCC(kPlain)
        }
#undef SS_OCC
    }
    return e == cudaSuccess ? nb : 0;
}

template <typename R>
cudaError_t launch_measure(const KArgs<R> &a, int block, int grid, cudaStream_t s) {
    SS_BLOCK_SWITCH(block, k_measure<R, BS><<<grid, BS, 0, s>>>(a));
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_init_sphere(const KArgs<R> &a, cudaStream_t s) {
    const int64_t g = a.ntiles < 4096 ? a.ntiles : 4096;
    k_init_sphere<R><<<(int)(g > 0 ? g : 1), 256, 0, s>>>(a);
    return cudaGetLastError();
}

// (the persistent and system-block kernels come as kPlain, kUniform and kGeneral variants)
template <typename R>
int persistent_blocks_per_sm(int block, int mode) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (mode == kPlain) {
        SS_BLOCK_SWITCH(block, e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_persistent<R, BS, kPlain>, BS, 0));
    } else if (mode == kUniform) {
        SS_BLOCK_SWITCH(block, e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_persistent<R, BS, kUniform>, BS, 0));
    } else {
        SS_BLOCK_SWITCH(block, e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_persistent<R, BS, kGeneral>, BS, 0));
    }
    return e == cudaSuccess ? nb : 0;
}

// Resident blocks per SM of the predictor variant (kPlain / kGeneral / kRows) launched.
template <typename R>
int step_blocks_per_sm(int block, int mode) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define SS_OCC(MODE) SS_BLOCK_SWITCH(block, e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_predictor<R, BS, MODE>, BS, 0))
    if (mode == kRows) {
        SS_OCC(kRows);
    } else if (mode == kGeneral) {
        SS_OCC(kGeneral);
    } else if (mode == kUniform) {
        SS_OCC(kUniform);
    } else {
        SS_OCC(kPlain);
    }
#undef SS_OCC
    return e == cudaSuccess ? nb : 0;
}

// Resident blocks per SM of the corrector variant the handle launches.
template <typename R>
int corrector_blocks_per_sm(int block, bool draw_ahead, int mode) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define SS_OCC(DA, MODE) \
    SS_BLOCK_SWITCH(block, e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_corrector<R, BS, DA, MODE>, BS, 0))
    if (mode == kRows) {
        if (draw_ahead) { SS_OCC(true, kRows); } else { SS_OCC(false, kRows); }
    } else if (mode == kGeneral) {
        if (draw_ahead) { SS_OCC(true, kGeneral); } else { SS_OCC(false, kGeneral); }
    } else if (mode == kUniform) {
        if (draw_ahead) { SS_OCC(true, kUniform); } else { SS_OCC(false, kUniform); }
    } else {
        if (draw_ahead) { SS_OCC(true, kPlain); } else { SS_OCC(false, kPlain); }
    }
#undef SS_OCC
    return e == cudaSuccess ? nb : 0;
}

template <typename R>
cudaError_t launch_mc_colour_warp(const KArgs<R> &a, const McArgs &m, int grid, cudaStream_t s) {
    constexpr int BS = 256;
    const bool general = a.J_tensor || a.any_cubic;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (m.c1 - m.c0 < (int64_t)sms * 64 * 32) {  // a warp per trial: enough warps to fill the SMs
        const int64_t blocks = (m.c1 - m.c0 + BS / 32 - 1) / (BS / 32);
        const int g = (int)(blocks < (int64_t)sms * 8 ? (blocks > 0 ? blocks : 1) : (int64_t)sms * 8);
        if (general)
            k_mc_colour_warp1<R, BS, kGeneral><<<g, BS, 0, s>>>(a, m);
        else
            k_mc_colour_warp1<R, BS, kPlain><<<g, BS, 0, s>>>(a, m);
    } else if (general) {
        k_mc_colour_warp<R, BS, kGeneral><<<grid, BS, 0, s>>>(a, m);
    } else {
        k_mc_colour_warp<R, BS, kPlain><<<grid, BS, 0, s>>>(a, m);
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_mc_prep(const KArgs<R> &a, const McArgs &m, cudaStream_t s) {
    constexpr int BS = 256;
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (a.n + BS - 1) / BS;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 4));
    k_mc_prep<R, BS><<<g, BS, 0, s>>>(a, m);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_mc_colour_rec(const KArgs<R> &a, const McArgs &m, int grid, cudaStream_t s) {
    constexpr int BS = 256;
    const bool general = a.J_tensor || a.any_cubic;
    if (m.first) {
        if (general)
            k_mc_colour_rec<R, BS, kGeneral, true><<<grid, BS, 0, s>>>(a, m);
        else
            k_mc_colour_rec<R, BS, kPlain, true><<<grid, BS, 0, s>>>(a, m);
    } else {
        if (general)
            k_mc_colour_rec<R, BS, kGeneral, false><<<grid, BS, 0, s>>>(a, m);
        else
            k_mc_colour_rec<R, BS, kPlain, false><<<grid, BS, 0, s>>>(a, m);
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_mc_colour(const KArgs<R> &a, const McArgs &m, int block, int grid, cudaStream_t s) {
    if (a.J_tensor || a.any_cubic) {
        SS_BLOCK_SWITCH(block, k_mc_colour<R, BS, kGeneral><<<grid, BS, 0, s>>>(a, m));
    } else {
        SS_BLOCK_SWITCH(block, k_mc_colour<R, BS, kPlain><<<grid, BS, 0, s>>>(a, m));
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_demag(const KArgs<R> &a, const DemagArgs &d, cudaStream_t s) {
    if (d.ncell <= 0) return cudaSuccess;
    const int64_t wblocks = (d.ncell * 32 + 255) / 256;
    k_demag_moments<R><<<(int)(wblocks < 4096 ? wblocks : 4096), 256, 0, s>>>(a, d);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_demag_field<R><<<(int)(wblocks < 4096 ? wblocks : 4096), 256, 0, s>>>(a, d);
    return cudaGetLastError();
}

// The first pass of the alternative integrators over the tiles, then the record of the state
// at the start of the step from its tile partials.
template <typename R>
int alt_first_grid(const KArgs<R> &a, int grid) {
    return (int)(a.ntiles < (int64_t)grid ? (a.ntiles > 0 ? a.ntiles : 1) : grid);
}

template <typename R, int Mode>
cudaError_t launch_midpoint_mode(const KArgs<R> &a, int iters, int grid, int igrid, int rgrid, cudaStream_t s) {
    cudaError_t e = Mode == kRows ? launch_rows_field<R>(a, a.sx, a.sy, a.sz, rgrid, s) : cudaSuccess;
    if (e != cudaSuccess) return e;
    k_mid_euler<R, Mode><<<alt_first_grid(a, grid), kAltBlock, 0, s>>>(a);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_finalize_ring(a.sys, a.sys_tiles, a.nsys, a.partials, a.rec, a.rec_cap, a.step, s);
    R *x[3] = {a.px, a.py, a.pz}, *y[3] = {a.qx, a.qy, a.qz};
    for (int k = 0; k + 1 < iters && e == cudaSuccess; ++k) {
        if (Mode == kRows && (e = launch_rows_field<R>(a, x[0], x[1], x[2], rgrid, s)) != cudaSuccess) break;
        k_mid_iter<R, Mode, false><<<igrid, 256, 0, s>>>(a, x[0], x[1], x[2], y[0], y[1], y[2]);
        e = cudaGetLastError();
        for (int c = 0; c < 3; ++c) {
            R *t = x[c];
            x[c] = y[c];
            y[c] = t;
        }
    }
    if (e == cudaSuccess && Mode == kRows) e = launch_rows_field<R>(a, x[0], x[1], x[2], rgrid, s);
    if (e == cudaSuccess) {  // the last iterate goes straight to S
        k_mid_iter<R, Mode, true><<<igrid, 256, 0, s>>>(a, x[0], x[1], x[2], a.sx, a.sy, a.sz);
        e = cudaGetLastError();
    }
    return e;
}

template <typename R>
cudaError_t launch_midpoint(const KArgs<R> &a, int iters, int grid, int igrid, int rgrid, cudaStream_t s) {
    if (a.ex) return launch_midpoint_mode<R, kRows>(a, iters, grid, igrid, rgrid, s);
    return (a.J_tensor || a.any_cubic) ? launch_midpoint_mode<R, kGeneral>(a, iters, grid, igrid, rgrid, s)
                                       : launch_midpoint_mode<R, kPlain>(a, iters, grid, igrid, rgrid, s);
}

// Resident 256-thread blocks per SM of the second-pass kernels of the alternative integrators
// (which = 0: the midpoint iterations, the smaller of their two variants; 1: the semi-implicit
// corrector) in the variant `mode` (kPlain, kGeneral or kRows); 0 if the query fails.
template <typename R>
int alt_pass_blocks_per_sm(int which, int mode) {
    int n0 = 0, n1 = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define SS_OCC(MODE)                                                                              \
    if (which == 0) {                                                                             \
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n0, k_mid_iter<R, MODE, false>, 256, 0); \
        if (e == cudaSuccess)                                                                     \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n1, k_mid_iter<R, MODE, true>, 256, 0); \
        n0 = n1 < n0 ? n1 : n0;                                                                   \
    } else {                                                                                      \
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n0, k_sib_corr<R, MODE>, 256, 0);      \
    }
    if (mode == kRows) {
        SS_OCC(kRows)
    } else if (mode == kGeneral) {
        SS_OCC(kGeneral)
    } else {
        SS_OCC(kPlain)
    }
#undef SS_OCC
    return e == cudaSuccess ? n0 : 0;
}

template <typename R>
cudaError_t launch_sib(const KArgs<R> &a, int grid, int cgrid, int rgrid, cudaStream_t s) {
    const int mode = a.ex ? kRows : (a.J_tensor || a.any_cubic) ? kGeneral : kPlain;
    cudaError_t e = mode == kRows ? launch_rows_field<R>(a, a.sx, a.sy, a.sz, rgrid, s) : cudaSuccess;
    if (e != cudaSuccess) return e;
    if (mode == kRows)
        k_sib_pred<R, kRows><<<alt_first_grid(a, grid), kAltBlock, 0, s>>>(a);
    else if (mode == kGeneral)
        k_sib_pred<R, kGeneral><<<alt_first_grid(a, grid), kAltBlock, 0, s>>>(a);
    else
        k_sib_pred<R, kPlain><<<alt_first_grid(a, grid), kAltBlock, 0, s>>>(a);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_finalize_ring(a.sys, a.sys_tiles, a.nsys, a.partials, a.rec, a.rec_cap, a.step, s);
    if (e == cudaSuccess && mode == kRows) e = launch_rows_field<R>(a, a.px, a.py, a.pz, rgrid, s);
    if (e != cudaSuccess) return e;
    if (mode == kRows)
        k_sib_corr<R, kRows><<<cgrid, 256, 0, s>>>(a);
    else if (mode == kGeneral)
        k_sib_corr<R, kGeneral><<<cgrid, 256, 0, s>>>(a);
    else
        k_sib_corr<R, kPlain><<<cgrid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_rows_field(const KArgs<R> &a, const R *X, const R *Y, const R *Z, int grid, cudaStream_t s) {
    if (a.sell) {
        const int64_t pb = (a.n + 255) / 256;
        k_pack4<R><<<(int)(pb < 4 * (int64_t)grid ? pb : 4 * (int64_t)grid), 256, 0, s>>>(a, X, Y, Z);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_rows_sell<R><<<grid, 256, 0, s>>>(a);
    } else if (a.J_tensor)
        k_rows_field<R, 2><<<grid, 256, 0, s>>>(a, X, Y, Z);
    else
        k_rows_field<R, 1><<<grid, 256, 0, s>>>(a, X, Y, Z);
    return cudaGetLastError();
}

template <typename R>
int rows_blocks_per_sm() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_rows_field<R, 1>, 256, 0) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb;
}

template <typename R>
int mc_blocks_per_sm(int block, int mode) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (mode == kPlain) {
        SS_BLOCK_SWITCH(block, e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_mc_colour<R, BS, kPlain>, BS, 0));
    } else {
        SS_BLOCK_SWITCH(block, e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_mc_colour<R, BS, kGeneral>, BS, 0));
    }
    return e == cudaSuccess ? nb : 0;
}

template <typename R>
cudaError_t launch_persistent(const KArgs<R> &a, int block, int grid, int nfin, long long nsteps, cudaStream_t s) {
    KArgs<R> args = a;
    void *params[] = {(void *)&args, (void *)&nfin, (void *)&nsteps};
    if (a.J_tensor || a.any_cubic) {
        SS_BLOCK_SWITCH(block, return cudaLaunchCooperativeKernel((const void *)k_persistent<R, BS, kGeneral>, dim3(grid),
                                                                  dim3(BS), params, 0, s));
    } else if (a.mat_uniform) {
        SS_BLOCK_SWITCH(block, return cudaLaunchCooperativeKernel((const void *)k_persistent<R, BS, kUniform>, dim3(grid),
                                                                  dim3(BS), params, 0, s));
    } else {
        SS_BLOCK_SWITCH(block, return cudaLaunchCooperativeKernel((const void *)k_persistent<R, BS, kPlain>, dim3(grid),
                                                                  dim3(BS), params, 0, s));
    }
    return cudaSuccess;
}

template <typename R>
cudaError_t launch_system_blocks(const KArgs<R> &a, int block, int grid, long long nsteps, cudaStream_t s) {
    if (a.J_tensor || a.any_cubic) {
        SS_BLOCK_SWITCH(block, k_system_blocks<R, BS, kGeneral><<<grid, BS, 0, s>>>(a, nsteps));
    } else {
        SS_BLOCK_SWITCH(block, k_system_blocks<R, BS, kPlain><<<grid, BS, 0, s>>>(a, nsteps));
    }
    return cudaGetLastError();
}

// Explicit instantiations, split over translation units per precision (SS_PART) so that the
// build compiles them in parallel (part 4, the cluster step, instantiates in ss_cluster.cuh).
#if SS_PART == 1  // the Heun passes, the split step, the measurement, the long-row passes
template cudaError_t launch_predictor<SS_REAL>(const KArgs<SS_REAL> &, int, int, cudaStream_t);
template cudaError_t launch_corrector<SS_REAL>(const KArgs<SS_REAL> &, int, int, int, cudaStream_t);
template cudaError_t launch_gauss<SS_REAL>(const KArgs<SS_REAL> &, int, int, cudaStream_t, int);
template cudaError_t launch_gstep_sync<SS_REAL>(const KArgs<SS_REAL> &, cudaStream_t);
template cudaError_t launch_predictor_split<SS_REAL>(const KArgs<SS_REAL> &, int, int, cudaStream_t);
template cudaError_t launch_corrector_split<SS_REAL>(const KArgs<SS_REAL> &, int, int, int, cudaStream_t);
template int split_blocks_per_sm<SS_REAL>(int, int, int);
template cudaError_t launch_measure<SS_REAL>(const KArgs<SS_REAL> &, int, int, cudaStream_t);
template cudaError_t launch_init_sphere<SS_REAL>(const KArgs<SS_REAL> &, cudaStream_t);
template int step_blocks_per_sm<SS_REAL>(int, int);
template int corrector_blocks_per_sm<SS_REAL>(int, bool, int);
template cudaError_t launch_rows_field<SS_REAL>(const KArgs<SS_REAL> &, const SS_REAL *, const SS_REAL *,
                                                const SS_REAL *, int, cudaStream_t);
template int rows_blocks_per_sm<SS_REAL>();
#elif SS_PART == 2  // many steps per launch, the demagnetising field
template cudaError_t launch_system_blocks<SS_REAL>(const KArgs<SS_REAL> &, int, int, long long, cudaStream_t);
template cudaError_t launch_persistent<SS_REAL>(const KArgs<SS_REAL> &, int, int, int, long long, cudaStream_t);
template int persistent_blocks_per_sm<SS_REAL>(int, int);
template cudaError_t launch_demag<SS_REAL>(const KArgs<SS_REAL> &, const DemagArgs &, cudaStream_t);
#elif SS_PART == 3  // Monte Carlo and the alternative integrators
template cudaError_t launch_mc_colour<SS_REAL>(const KArgs<SS_REAL> &, const McArgs &, int, int, cudaStream_t);
template cudaError_t launch_mc_colour_rec<SS_REAL>(const KArgs<SS_REAL> &, const McArgs &, int, cudaStream_t);
template cudaError_t launch_mc_colour_warp<SS_REAL>(const KArgs<SS_REAL> &, const McArgs &, int, cudaStream_t);
template cudaError_t launch_mc_prep<SS_REAL>(const KArgs<SS_REAL> &, const McArgs &, cudaStream_t);
template int mc_blocks_per_sm<SS_REAL>(int, int);
template cudaError_t launch_midpoint<SS_REAL>(const KArgs<SS_REAL> &, int, int, int, int, cudaStream_t);
template cudaError_t launch_sib<SS_REAL>(const KArgs<SS_REAL> &, int, int, int, cudaStream_t);
template int alt_pass_blocks_per_sm<SS_REAL>(int, int);
#endif

}  // namespace ss
