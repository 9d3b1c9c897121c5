// The cluster step: one small system (up to a few thousand spins) advanced a chunk of steps
// by one thread-block cluster.
//
// On GB300 an FP64 warp instruction holds its SM sub-partition's FP64 pipe for about 64
// cycles, whatever the number of active lanes.  A system of a thousand spins, one spin per
// thread, is therefore bound by the FP64 instructions each warp issues per step (the
// Gaussian transform and the record sums included), not by memory, and spreading the spins
// thinner over more SMs does not shorten it.  This path takes the per-warp work apart:
//   * k_cluster_gauss draws the thermal fields of a whole chunk of steps beforehand, over
//     the whole GPU, with the Philox counters, the transform and the product sigma g of the
//     step kernels (so the values are theirs);
//   * k_cluster_steps runs the chunk in one cluster of up to 16 CTAs.  CTA r holds spins
//     [r P, r P + P) of S and S' in shared memory; a neighbour in another CTA is read through
//     distributed shared memory (mapa + ld.shared::cluster), and the two Heun passes of a step
//     are separated by cluster barriers instead of kernel boundaries or grid barriers.  Each
//     group of 32 spins has four warps: three take one Cartesian component each of the
//     exchange sum, the field, the LLG right-hand side and the update (their shares of S x H
//     and S x (S x H) meet in shared memory); the fourth takes the spins' scalars (S.e, the
//     squared length and its reciprocal square root, the record terms);
//   * k_cluster_record sums the chunk's record terms afterwards, tile by tile in the
//     predictor kernel's order, so each record is the other launch modes' bit for bit.
// Every value is formed by the operations of det_field, llg_rhs and spin_terms_r in their
// order, so the states are bitwise those of the other launch modes.
#pragma once

#include "ss_launch.cuh"

namespace ss {

__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// The cluster-window address of shared-memory byte address `addr` of this CTA, in CTA `rank`.
__device__ __forceinline__ uint32_t cluster_map(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ double ld_cluster(uint32_t addr, double) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ float ld_cluster(uint32_t addr, float) {
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
    return v;
}

// Every thread of every CTA of the cluster: this CTA's shared-memory writes are released,
// the other CTAs' acquired.
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The four warps of one group of 32 spins (named barrier 1 + group): between two cluster
// barriers the groups of a CTA touch only their own spins' entries, so they need not wait
// for one another.
__device__ __forceinline__ void group_sync(int grp) {
    asm volatile("bar.sync %0, 128;" ::"r"(grp + 1) : "memory");
}

template <typename R>
__device__ __forceinline__ R pick3(int c, R x, R y, R z) {
    return c == 0 ? x : (c == 1 ? y : z);
}

// The thermal field sigma g of steps step0 .. step0 + m - 1 of every spin: the step kernels'
// product mul_rn(sig sqrt(T), g) of its Gaussians, or 0 at zero temperature (where the step
// kernels add 0).
template <typename R, int BS>
__global__ void __launch_bounds__(BS) k_cluster_gauss(const KArgs<R> a, const ClusterArgs<R> c) {
    __shared__ StepTabT<R> tab;
    stage_step_tables(a, tab);
    __syncthreads();
    const SysDesc &sd = a.sys[0];
    const int64_t off = sd.offset - sd.pbase;  // Philox spin index i - off
    const int64_t n = a.n, total = (int64_t)c.m * n;
    for (int64_t idx = (int64_t)blockIdx.x * BS + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * BS) {
        const int s = (int)(idx / n);
        const int64_t i = idx - (int64_t)s * n;
        const uint64_t step = c.step0 + (uint64_t)s;
        const R sqrtT = sqrtT_of_step(a, step, sd);
        R t0 = (R)0, t1 = (R)0, t2 = (R)0;
        if (sqrtT > (R)0) {
            const R sig = (a.mat_uniform ? a.mat0.sig : a.mats[mat_of(a, i)].sig) * sqrtT;
            const Philox4 w = philox4x32_10((uint32_t)(i - off), (uint32_t)step, sd.ctr2, 0u, sd.key0, sd.key1);
            R g0, g1, g2;
            thermal_gaussians(a, tab, w, g0, g1, g2);
            t0 = mul_rn(sig, g0);
            t1 = mul_rn(sig, g1);
            t2 = mul_rn(sig, g2);
        }
        R *G = c.G + (int64_t)s * 3 * n + i;
        G[0] = t0;
        G[n] = t1;
        G[2 * n] = t2;
    }
}

// m Heun steps of the single system of `a` in one cluster (gridDim.x CTAs of 128 groups
// threads).  NR: the row slots (kShortRow or kPatRow, at least the longest row).
// A pass has five phases, separated by barriers of the group's four warps:
//   A  exchange sums (components);              S.e (scalars)
//   B  the field component (det_field + H_th);  record terms mu S, E_ani (scalars, predictor)
//   C  this component of S x H;                 record term -mu S.h/2 (scalars, predictor)
//   D  S x (S x H), dS and the update;          --
//   E  --                                       1/|v| and the renormalised spin (scalars)
// then a cluster barrier.  Two component warps share one SM sub-partition, a scalar and a
// component warp each of the others; the scalar warps' record terms fill phases whose
// critical path is the component warps'.
template <typename R, int Mode, int NR>
__global__ void __launch_bounds__(32 * 4 * kClusterMaxGroups) k_cluster_steps(const KArgs<R> a, const ClusterArgs<R> c) {
    extern __shared__ __align__(16) unsigned char cl_smem[];
    R *const sm = reinterpret_cast<R *>(cl_smem);
    const int P = c.span;
    // S | S' | exchange sums | field | S x H | unnormalised update, per component | an
    R *const S = sm;
    R *const Sp = sm + 3 * P;
    R *const E = sm + 6 * P;
    R *const Hs = sm + 9 * P;
    R *const Cs = sm + 12 * P;
    R *const Vs = sm + 15 * P;
    R *const AN = sm + 18 * P;
    constexpr bool Cubic = Mode == kGeneral;
    // FP32-mixed form: this component's thermal field loaded a step ahead, the record terms
    // stored in phase C; FP64 form: the load where it is used, the terms stored after the
    // cluster barrier (the faster arrangement of each, measured on GB300)
    constexpr bool kAhead = sizeof(R) == 4;
    const uint32_t rank = cluster_ctarank();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = warp >> 2;
    // warp roles rotate with the group, so that the scalar warps sit on different SM
    // sub-partitions (warp w runs on sub-partition w mod 4)
    const int role = (warp + grp) & 3;  // 0..2: that component of the group's spins; 3: scalars
    const int ls = grp * 32 + lane;
    const int64_t n = a.n;
    const int64_t i = (int64_t)rank * P + ls;
    const bool act = i < n;
    const bool comp = role < 3;
    const SysDesc &sd = a.sys[0];
    const MatDesc<R> &m = mat_at<Mode>(a, act ? i : 0);

    // per-role constants: the component's applied field, easy-axis entry and Neel row
    const int rc = comp ? role : 0;
    const R hC = sys_H(sd, rc, R());
    const R eC = pick3(rc, m.e[0], m.e[1], m.e[2]);
    const R k0 = pick3(rc, m.kf[0], m.kf[3], m.kf[4]);
    const R k1 = pick3(rc, m.kf[3], m.kf[1], m.kf[5]);
    const R k2 = pick3(rc, m.kf[4], m.kf[5], m.kf[2]);
    // the material's constants in registers for the whole chunk
    const R ex = m.e[0], ey = m.e[1], ez = m.e[2], ani = m.ani, mgp = -m.gp, lam = m.lambda, dt = m.dt;
    const R hdt = (R)0.5 * dt, kcf = m.kcf, mu = m.mu;
    const bool cubic = Cubic && m.has_cubic, neel = m.has_neel != 0;

    if (act && comp) S[role * P + ls] = pick3(role, a.sx, a.sy, a.sz)[i];
    // the neighbours: cluster-window address of this component of each one's S (S' lies
    // 3 P elements further in every CTA) and J_ij / mu_s,i
    uint32_t nb[NR];
    R Jn[NR];
    int len = 0;
    if (act && comp) {
        const int32_t b = __ldg(a.row_ptr + i);
        len = __ldg(a.row_ptr + i + 1) - b;
        const uint32_t base = (uint32_t)__cvta_generic_to_shared(S + role * P);
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            nb[q] = 0u;
            Jn[q] = (R)0;
            if (q < len) {
                const int32_t j = chk(__ldg(a.col + b + q), n, a.err);
                const int32_t r = j / P;
                nb[q] = cluster_map(base + (uint32_t)(j - r * P) * (uint32_t)sizeof(R), (uint32_t)r);
                Jn[q] = a.J_uniform ? a.J_value : __ldg(a.J + b + q);
            }
        }
    }
    const uint32_t sp_off = 3u * (uint32_t)P * (uint32_t)sizeof(R);
    // H_app + sum_j (J_ij / mu_s,i) X_j of this component, in CSR order (exchange_sum_h)
    auto xsum = [&](uint32_t shift) -> R {
        R x = hC;
#pragma unroll
        for (int q = 0; q < NR; ++q)
            if (q < len) x = fma(Jn[q], ld_cluster(nb[q] + shift, R()), x);
        return x;
    };
    // the scalar warp's last phase: 1/|v| of the group's update and the renormalised spin
    auto renormalise = [&](R *dst, bool check) {
        const R v0 = Vs[ls], v1 = Vs[P + ls], v2 = Vs[2 * P + ls];
        const R inv = rsqrt_r(fma(v2, v2, fma(v1, v1, mul_rn(v0, v0))));
        if (check && bad_inv(inv)) atomicOr(a.err, kErrNonFinite);
        dst[ls] = mul_rn(v0, inv);
        dst[P + ls] = mul_rn(v1, inv);
        dst[2 * P + ls] = mul_rn(v2, inv);
    };
    auto store_terms = [&](int s, const R (&tv)[5]) {
        R *T = c.T + (int64_t)s * 5 * n + i;
#pragma unroll
        for (int k = 0; k < 5; ++k) T[k * n] = tv[k];
    };
    R t_next = (kAhead && act && comp) ? c.G[(int64_t)role * n + i] : (R)0;
    cluster_barrier();  // every CTA's S is in place before the first remote read

    for (int s = 0; s < c.m; ++s) {
        R t = t_next;  // this component's thermal field of the step
        if (kAhead && act && comp && s + 1 < c.m) t_next = c.G[((int64_t)(s + 1) * 3 + role) * n + i];
        R s0 = (R)0, s1 = (R)0, s2 = (R)0, ec = (R)0, cc = (R)0, qc = (R)0, sde = (R)0;
        R tv[5];
        // ---- predictor.  A
        if (act) {
            s0 = S[ls];
            s1 = S[P + ls];
            s2 = S[2 * P + ls];
            if (comp) {
                ec = xsum(0u);
                E[role * P + ls] = ec;
            } else {
                sde = fma(s2, ez, fma(s1, ey, mul_rn(s0, ex)));
                AN[ls] = mul_rn(ani, sde);
            }
        }
        group_sync(grp);
        // B
        if (act) {
            if (comp) {
                const R sc = pick3(role, s0, s1, s2);
                R H = fma(AN[ls], eC, ec);
                if (cubic) H = fma(mul_rn(mul_rn(kcf, sc), sc), sc, H);
                if (neel) H = H + fma(k2, s2, fma(k1, s1, mul_rn(k0, s0)));
                if (!kAhead) t = c.G[((int64_t)s * 3 + role) * n + i];
                H += t;
                Hs[role * P + ls] = H;
            } else {
                tv[0] = mul_rn(mu, s0);
                tv[1] = mul_rn(mu, s1);
                tv[2] = mul_rn(mu, s2);
                tv[4] = anisotropy_term<R, Cubic>(m, s0, s1, s2, sde);
            }
        }
        group_sync(grp);
        // C
        if (act) {
            if (comp) {
                const R H0 = Hs[ls], H1 = Hs[P + ls], H2 = Hs[2 * P + ls];
                cc = role == 0 ? fma(s1, H2, -mul_rn(s2, H1))
                               : (role == 1 ? fma(s2, H0, -mul_rn(s0, H2)) : fma(s0, H1, -mul_rn(s1, H0)));
                Cs[role * P + ls] = cc;
            } else {
                tv[3] = exchange_term(m, s0, s1, s2, E[ls], E[P + ls], E[2 * P + ls]);
                if (kAhead) store_terms(s, tv);
            }
        }
        group_sync(grp);
        // D
        if (act && comp) {
            const R c0 = Cs[ls], c1 = Cs[P + ls], c2 = Cs[2 * P + ls];
            const R xc = role == 0 ? fma(s1, c2, -mul_rn(s2, c1))
                                   : (role == 1 ? fma(s2, c0, -mul_rn(s0, c2)) : fma(s0, c1, -mul_rn(s1, c0)));
            const R dc = mul_rn(mgp, fma(lam, xc, cc));
            const R sc = pick3(role, s0, s1, s2);
            qc = fma(hdt, dc, sc);
            Vs[role * P + ls] = fma(dt, dc, sc);
        }
        group_sync(grp);
        // E: S' = v / |v|
        if (act && !comp) renormalise(Sp, false);
        cluster_barrier();
        if (!kAhead && act && !comp) store_terms(s, tv);  // after the barrier: its release waits for no store

        // ---- corrector (the same phases on S', with the predictor's thermal field).  A
        R p0 = (R)0, p1 = (R)0, p2 = (R)0;
        if (act) {
            p0 = Sp[ls];
            p1 = Sp[P + ls];
            p2 = Sp[2 * P + ls];
            if (comp)
                ec = xsum(sp_off);
            else
                AN[ls] = mul_rn(ani, fma(p2, ez, fma(p1, ey, mul_rn(p0, ex))));
        }
        group_sync(grp);
        // B
        if (act && comp) {
            const R pc = pick3(role, p0, p1, p2);
            R H = fma(AN[ls], eC, ec);
            if (cubic) H = fma(mul_rn(mul_rn(kcf, pc), pc), pc, H);
            if (neel) H = H + fma(k2, p2, fma(k1, p1, mul_rn(k0, p0)));
            H += t;
            Hs[role * P + ls] = H;
        }
        group_sync(grp);
        // C
        if (act && comp) {
            const R H0 = Hs[ls], H1 = Hs[P + ls], H2 = Hs[2 * P + ls];
            cc = role == 0 ? fma(p1, H2, -mul_rn(p2, H1))
                           : (role == 1 ? fma(p2, H0, -mul_rn(p0, H2)) : fma(p0, H1, -mul_rn(p1, H0)));
            Cs[role * P + ls] = cc;
        }
        group_sync(grp);
        // D
        if (act && comp) {
            const R c0 = Cs[ls], c1 = Cs[P + ls], c2 = Cs[2 * P + ls];
            const R xc = role == 0 ? fma(p1, c2, -mul_rn(p2, c1))
                                   : (role == 1 ? fma(p2, c0, -mul_rn(p0, c2)) : fma(p0, c1, -mul_rn(p1, c0)));
            const R dc = mul_rn(mgp, fma(lam, xc, cc));
            Vs[role * P + ls] = fma(hdt, dc, qc);
        }
        group_sync(grp);
        // E: S = v / |v|, with the corrector kernel's non-finite check
        if (act && !comp) renormalise(S, true);
        cluster_barrier();
    }
    if (act && comp) pick3(role, a.sx, a.sy, a.sz)[i] = S[role * P + ls];
    if (rank == 0 && threadIdx.x == 0) *a.step = c.step0 + (uint64_t)c.m;
}

// The records of the chunk's steps (block s: step step0 + s) from the stored terms, tile by
// tile with the predictor kernel's thread order and partial sums, then the record as the
// corrector kernel finalises it.  BS must be the step kernels' block.
template <typename R, int BS>
__global__ void __launch_bounds__(BS) k_cluster_record(const KArgs<R> a, const ClusterArgs<R> c) {
    __shared__ double red[(BS / 32) * 8];
    const int s = blockIdx.x;
    const uint64_t step = c.step0 + (uint64_t)s;
    const int64_t n = a.n;
    const R *T = c.T + (int64_t)s * 5 * n;
    double *part = c.partials + (int64_t)s * a.ntiles * kPartComps;
    for (int64_t t = 0; t < a.ntiles; ++t) {
        const TileDesc td = a.tiles[t];
        TermAcc<R> ta;
        ta.reset();
        for (int k = threadIdx.x; k < td.count; k += BS) {
            const int64_t i = td.start + k;
            if constexpr (sizeof(R) == 4) {
                R v[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) v[q] = T[q * n + i];
                ta.add(v);
            } else {
                double v[5];
#pragma unroll
                for (int q = 0; q < 5; ++q) v[q] = widen(T[q * n + i]);
                ta.add(v);
            }
        }
        double acc[8];
        ta.out(acc);
        warp_partials<BS>(acc, red, 0);
        __syncthreads();
        flush_partials<BS>(red, 1, part, t, 1);
        __syncthreads();
    }
    double *dst = a.rec + (int64_t)(step % (uint64_t)a.rec_cap) * a.nsys * kRecComps;
    finalize_system<BS, true>(a.sys, a.sys_tiles, part, 0, dst, red);
}

// ----------------------------------------------------------------------------------
// Host launchers
// ----------------------------------------------------------------------------------

template <typename R>
size_t cluster_smem(int groups) {
    return (size_t)19 * 32 * groups * sizeof(R);
}

template <typename R, int Mode, int NR>
cudaError_t cluster_config(int ctas, int groups, cudaLaunchConfig_t &cfg, cudaLaunchAttribute *at, cudaStream_t s) {
    const void *k = (const void *)k_cluster_steps<R, Mode, NR>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3((unsigned)(128 * groups));
    cfg.dynamicSmemBytes = cluster_smem<R>(groups);
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)ctas;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaSuccess;
}

template <typename R, int Mode, int NR>
cudaError_t cluster_launch(const KArgs<R> &a, const ClusterArgs<R> &c, int ctas, cudaStream_t s) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    cudaError_t e = cluster_config<R, Mode, NR>(ctas, c.groups, cfg, at, s);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, k_cluster_steps<R, Mode, NR>, a, c);
}

template <typename R, int Mode, int NR>
int cluster_max_for(int groups) {
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    if (cluster_config<R, Mode, NR>(1, groups, cfg, at, nullptr) != cudaSuccess) return 0;
    cfg.numAttrs = 0;  // the query takes the cluster size from its own search
    int size = 0;
    if (cudaOccupancyMaxPotentialClusterSize(&size, k_cluster_steps<R, Mode, NR>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return size;
}

template <typename R>
cudaError_t launch_cluster_gauss(const KArgs<R> &a, const ClusterArgs<R> &c, cudaStream_t s) {
    constexpr int BS = 256;
    const int64_t total = (int64_t)c.m * a.n;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (total + BS - 1) / BS;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, 4ll * std::max(sms, 1)));
    k_cluster_gauss<R, BS><<<grid, BS, 0, s>>>(a, c);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_cluster_steps(const KArgs<R> &a, const ClusterArgs<R> &c, int ctas, int row_slots, cudaStream_t s) {
    const int mode = heun_mode(a);
    if (mode == kRows) return cudaErrorInvalidValue;
#define SS_CLUSTER(MODE)                                                                                  \
    return row_slots <= kShortRow ? cluster_launch<R, MODE, kShortRow>(a, c, ctas, s)                    \
                                  : cluster_launch<R, MODE, kPatRow>(a, c, ctas, s)
    if (mode == kGeneral) SS_CLUSTER(kGeneral);
    if (mode == kUniform) SS_CLUSTER(kUniform);
    SS_CLUSTER(kPlain);
#undef SS_CLUSTER
}

template <typename R>
cudaError_t launch_cluster_record(const KArgs<R> &a, const ClusterArgs<R> &c, int block, cudaStream_t s) {
    SS_BLOCK_SWITCH(block, k_cluster_record<R, BS><<<c.m, BS, 0, s>>>(a, c));
    return cudaGetLastError();
}

template <typename R>
int cluster_max_ctas(const KArgs<R> &a, int groups, int row_slots) {
    const int mode = heun_mode(a);
    if (mode == kRows) return 0;
#define SS_CLUSTER_MAX(MODE)                                                                  \
    return row_slots <= kShortRow ? cluster_max_for<R, MODE, kShortRow>(groups)               \
                                  : cluster_max_for<R, MODE, kPatRow>(groups)
    if (mode == kGeneral) SS_CLUSTER_MAX(kGeneral);
    if (mode == kUniform) SS_CLUSTER_MAX(kUniform);
    SS_CLUSTER_MAX(kPlain);
#undef SS_CLUSTER_MAX
}

template cudaError_t launch_cluster_gauss<SS_REAL>(const KArgs<SS_REAL> &, const ClusterArgs<SS_REAL> &, cudaStream_t);
template cudaError_t launch_cluster_steps<SS_REAL>(const KArgs<SS_REAL> &, const ClusterArgs<SS_REAL> &, int, int,
                                                   cudaStream_t);
template cudaError_t launch_cluster_record<SS_REAL>(const KArgs<SS_REAL> &, const ClusterArgs<SS_REAL> &, int,
                                                    cudaStream_t);
template int cluster_max_ctas<SS_REAL>(const KArgs<SS_REAL> &, int, int);

}  // namespace ss
