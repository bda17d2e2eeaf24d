// Persistent APC iteration kernel (Eq. (cons), Algorithm 1) for sm_103a.
//
// Work split.  The paper gives machine i the rows [A_i, b_i]; here the unknowns
// j = 0..n-1 are split into contiguous row ranges, one per thread-block
// cluster, and the m machines ("workers") into the CTAs of each cluster, one
// warp per worker.  Q is stored [n][m][P]: row j holds, for every worker i, the
// j-th row of Q_i (padded with zeros to P = 32*CPL columns).
//
// One pass over Q per iteration.  For each row j of its range a cluster has
// every worker's slice Q_i[j,:] on chip, so both skinny products of
// P_i y = y - Q_i (Q_i^T y) use it while it is resident:
//   w_i[j]   = Q_i[j,:] . z_i               (z_i = Q_i^T (xbar - x_i), last pass)
//   x_i[j]  += gamma (xbar[j] - x_i[j] - w_i[j])                    (cons1)
//   xbar[j]  = (eta/m) sum_i x_i[j] + (1 - eta) xbar[j]             (cons2)
//   z_i'    += Q_i[j,:]^T (xbar[j] - x_i[j])   (next pass's z_i, partial over j)
// The sum over workers in (cons2) is a per-row reduction across the warps of a
// CTA (shared memory) and across the CTAs of the cluster (st.async into the
// peers' shared memory, completing on their mbarriers).  The partial z_i' of
// all clusters are summed with global atomics, followed by one grid-wide
// barrier per iteration.  Q rows stream into a ring of shared-memory stages
// through TMA bulk copies with an L2 evict-first policy.
//
// The same pass structure computes the transpose of the step (reverse sweep
// for gradients), the least-norm initialisation and products with
// X = (1/m) sum_i Q_i Q_i^T (Eq. 3); `mode` selects the per-row arithmetic.
//
// Every wait is bounded by a_.timeout_ns (globaltimer); on expiry the kernel
// records an error word, drains its own bulk copies, joins a final cluster
// barrier and returns.
#include "apc_internal.h"
#include "apc_ptx.cuh"

namespace apc {

namespace {

template <typename TC>
struct RowOps {
    // Per (row, worker): new state xn and the worker's term of the row sum.
    __device__ static inline void update(int mode, TC xo, TC xb, TC d, TC g, TC e, TC im, TC &xn, TC &contrib) {
        switch (mode) {
            case MODE_APC: xn = xo + g * (xb - xo - d); contrib = xn; break;
            case MODE_INIT: xn = d; contrib = d; break;
            case MODE_ADJ: {
                const TC mu = xo + e * im * xb;
                xn = (TC(1) - g) * mu + g * d;
                contrib = mu - d;
            } break;
            case MODE_ADJ_SEED: xn = TC(0); contrib = TC(0); break;
            case MODE_ADJ_FINAL: xn = xo; contrib = TC(0); break;
            default: /* MODE_POWER */ xn = TC(0); contrib = d; break;
        }
    }
    // Per row: the master's new value from the row sum S.
    __device__ static inline TC master(int mode, TC S, TC xb, TC g, TC e, TC im) {
        switch (mode) {
            case MODE_APC: return e * im * S + (TC(1) - e) * xb;
            case MODE_INIT: return im * S;
            case MODE_ADJ: return (TC(1) - e) * xb + g * S;
            case MODE_ADJ_SEED:
            case MODE_ADJ_FINAL: return xb;
            default: return im * S;
        }
    }
    // Per (row, worker): the coefficient multiplying Q_i[j,:]^T in the next z_i.
    __device__ static inline TC coef(int mode, TC xn, TC xbn, TC e, TC im) {
        switch (mode) {
            case MODE_APC:
            case MODE_INIT: return xbn - xn;
            case MODE_ADJ:
            case MODE_ADJ_SEED: return xn + e * im * xbn;
            case MODE_ADJ_FINAL: return xn + im * xbn;
            default: return xbn;
        }
    }
    __device__ static inline bool reads_x(int mode) {
        return mode == MODE_APC || mode == MODE_ADJ || mode == MODE_ADJ_FINAL;
    }
    __device__ static inline bool writes_x(int mode) {
        return mode == MODE_APC || mode == MODE_INIT || mode == MODE_ADJ || mode == MODE_ADJ_SEED;
    }
};

template <typename TQ, typename TC, int V>
__device__ __forceinline__ void load_vec(const TQ *p, TC *out) {
    if constexpr (V * sizeof(TQ) == 16) {
        Elem<TQ>::load16(p, out);
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if constexpr (sizeof(TQ) == 2) out[v] = __bfloat162float(p[v]);
            else out[v] = static_cast<TC>(p[v]);
        }
    }
}

template <typename TS>
__device__ __forceinline__ void atomic_add_vec(TS *dst, const TS *v, int count) {
    if constexpr (sizeof(TS) == 4) {
        if (count % 4 == 0) {
            for (int i = 0; i < count; i += 4)
                atomicAdd(reinterpret_cast<float4 *>(dst + i), make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]));
            return;
        }
    }
    for (int i = 0; i < count; ++i) atomicAdd(dst + i, v[i]);
}

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

template <typename TQ, typename TS, int R>
struct SmemLayout {
    size_t stage_elems, off_xbs, off_red, off_sloc, off_bars, total;
    __host__ __device__ SmemLayout(int nw, int P, int stages, int64_t rpc) {
        stage_elems = size_t(R) * nw * P;
        off_xbs = align_up(size_t(stages) * stage_elems * sizeof(TQ), 128);
        off_red = align_up(off_xbs + 2 * size_t(rpc) * sizeof(TS), 16);
        off_sloc = off_red + 2 * R * 32 * sizeof(TS);
        off_bars = align_up(off_sloc + 2 * 8 * R * sizeof(TS), 8);
        total = off_bars + (stages + 2) * sizeof(uint64_t);
    }
};

template <typename TQ, typename TS, int CPL, int R, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) apc_iter_kernel(const IterArgs a) {
    using TC = TS;
    constexpr int VE = Elem<TQ>::V;
    constexpr int V = CPL < VE ? CPL : VE;  // elements per lane per vector
    constexpr int H = CPL / V;              // vectors per lane per row

    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int abort_flag;
    __shared__ int abort_code;

    const int P = a.P, nw = a.nw, S = a.stages, m = a.m, cs = a.cs;
    const int64_t rpc = a.rows_per_cluster;
    const SmemLayout<TQ, TS, R> L(nw, P, S, rpc);
    TQ *stage_base = reinterpret_cast<TQ *>(smem);
    TS *xbs = reinterpret_cast<TS *>(smem + L.off_xbs);  // [2][rpc]
    TS *red = reinterpret_cast<TS *>(smem + L.off_red);  // [2][R][32]
    TS *sloc = reinterpret_cast<TS *>(smem + L.off_sloc);  // [2][8][R]
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L.off_bars);  // [S]
    uint64_t *xchg = full + S;  // [2]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nwarps = blockDim.x >> 5;
    const uint32_t rank = cluster_rank();
    const int64_t cl = cluster_id_x();
    const int w0 = int(rank) * nw;
    const int nw_cta = max(0, min(nw, m - w0));
    const bool active = warp < nw_cta;
    const int wk = w0 + warp;
    const int64_t row0 = cl * rpc;
    const int64_t row1 = min(a.n, row0 + rpc);
    const int64_t nrows = max(int64_t(0), row1 - row0);
    const int64_t ngroups = (nrows + R - 1) / R;
    const int64_t total = ngroups * a.iters;
    const uint32_t rowbytes = uint32_t(nw_cta) * P * sizeof(TQ);
    const TQ *Q = reinterpret_cast<const TQ *>(a.Q);
    TS *xw = reinterpret_cast<TS *>(a.xw);
    TS *xbar = reinterpret_cast<TS *>(a.xbar);
    TS *zbuf = reinterpret_cast<TS *>(a.zbuf);
    const TC g = TC(a.gamma), e = TC(a.eta), im = TC(a.inv_m);
    const int mode = a.mode;
    const bool rx = RowOps<TC>::reads_x(mode), wx = RowOps<TC>::writes_x(mode);
    const size_t mP = size_t(m) * P;

    if (tid == 0) {
        abort_flag = 0;
        abort_code = 0;
        for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
        mbar_init(&xchg[0], R);
        mbar_init(&xchg[1], R);
        fence_mbar_init_cluster();
    }
    for (int64_t i = tid; i < nrows; i += blockDim.x) xbs[i] = xbar[row0 + i];
    __syncthreads();
    cluster_sync_all();  // peers' barriers are initialised before any st.async

    uint64_t policy = 0;
    int64_t issued = 0;
    auto issue = [&](int64_t qq) {
        const int s = int(qq % S);
        const int64_t gi = qq % ngroups;
        const int64_t r0 = row0 + gi * R;
        const int nr = int(min(int64_t(R), row1 - r0));
        mbar_arrive_expect_tx(&full[s], uint32_t(nr) * rowbytes);
        TQ *dst = stage_base + size_t(s) * L.stage_elems;
        for (int r = 0; r < nr; ++r)
            tma_load_1d(dst + size_t(r) * nw * P, Q + (size_t(r0 + r) * m + w0) * P, rowbytes, &full[s], policy);
    };
    if (tid == 0 && nw_cta > 0) {
        policy = policy_evict_first();
        for (; issued < min(int64_t(S - 1), total); ++issued) issue(issued);
    }

    // Register state: z_i (this pass's input) and the partial z_i' (output).
    TC z[CPL], acc[CPL];
    auto load_z = [&](int64_t t) {
        const TS *zin = zbuf + size_t(t % 3) * mP + size_t(wk) * P;
#pragma unroll
        for (int h = 0; h < H; ++h)
#pragma unroll
            for (int v = 0; v < V; ++v)
                z[h * V + v] = active ? __ldcg(zin + (h * 32 + lane) * V + v) : TC(0);
#pragma unroll
        for (int c = 0; c < CPL; ++c) acc[c] = TC(0);
    };
    load_z(a.t0);

    auto xload = [&](int64_t qq) -> TC {
        if (!rx || !active || lane >= R || qq >= total) return TC(0);
        const int64_t row = row0 + (qq % ngroups) * R + lane;
        return row < row1 ? xw[size_t(row) * m + wk] : TC(0);
    };
    TC xpre = xload(0);
    int cur = 0;
    int64_t q = 0;

    for (int64_t it = 0; it < a.iters; ++it) {
        for (int64_t gi = 0; gi < ngroups; ++gi, ++q) {
            const int s = int(q % S);
            const uint32_t par = uint32_t((q / S) & 1);
            const int64_t r0 = row0 + gi * R;
            const int nr = int(min(int64_t(R), row1 - r0));
            const int b = int(q & 1);
            if (nw_cta > 0 && !mbar_wait(&full[s], par, a.timeout_ns)) { abort_flag = 1; abort_code = DEV_TIMEOUT_TMA; }
            const TQ *st = stage_base + size_t(s) * L.stage_elems + size_t(warp) * P;

            // phase 1: w_i[j] = Q_i[j,:] . z_i for the R rows of the group
            TC d[R];
#pragma unroll
            for (int r = 0; r < R; ++r) d[r] = TC(0);
            if (active) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (r < nr) {
#pragma unroll
                        for (int h = 0; h < H; ++h) {
                            TC qv[V];
                            load_vec<TQ, TC, V>(st + size_t(r) * nw * P + (h * 32 + lane) * V, qv);
#pragma unroll
                            for (int v = 0; v < V; ++v) d[r] = fma(qv[v], z[h * V + v], d[r]);
                        }
                    }
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
#pragma unroll
                for (int r = 0; r < R; ++r) d[r] += __shfl_xor_sync(0xffffffffu, d[r], off);
            TC myd = TC(0);
#pragma unroll
            for (int r = 0; r < R; ++r) myd = (lane == r) ? d[r] : myd;

            const TC xo = xpre;
            xpre = xload(q + 1);
            TC xn = TC(0), contrib = TC(0);
            if (active && lane < nr) {
                const TC xb = xbs[size_t(cur) * rpc + gi * R + lane];
                RowOps<TC>::update(mode, xo, xb, myd, g, e, im, xn, contrib);
                if (wx) xw[size_t(r0 + lane) * m + wk] = xn;
            }
            if (lane < R) red[(b * R + lane) * 32 + warp] = (active && lane < nr) ? contrib : TC(0);

            if (__syncthreads_or(abort_flag)) goto abort_exit;
            if (tid == 0 && nw_cta > 0 && issued < total && issued == q + S - 1) { issue(issued); ++issued; }

            // row sums: this CTA's part, then the cluster's through st.async
            for (int r = warp; r < R; r += nwarps) {
                TC v = (lane < nwarps) ? red[(b * R + r) * 32 + lane] : TC(0);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                if (lane == 0) {
                    if (r < nr) {
                        TS *slot = &sloc[(b * 8 + rank) * R + r];
                        *slot = v;
                        for (int k = 0; k < cs; ++k) {
                            if (k == int(rank)) continue;
                            const uint32_t ra = map_shared_rank(smem_u32(slot), k);
                            const uint32_t rb = map_shared_rank(smem_u32(&xchg[b]), k);
                            if constexpr (sizeof(TS) == 4) st_async_f32(ra, v, rb);
                            else st_async_f64(ra, v, rb);
                        }
                    }
                    mbar_arrive_expect_tx(&xchg[b], r < nr ? uint32_t((cs - 1) * sizeof(TS)) : 0u);
                }
            }
            if (!mbar_wait(&xchg[b], uint32_t((q >> 1) & 1), a.timeout_ns)) { abort_flag = 1; abort_code = DEV_TIMEOUT_XCHG; }

            TC xbn[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                xbn[r] = TC(0);
                if (r < nr) {
                    TC Ssum = TC(0);
                    for (int k = 0; k < cs; ++k) Ssum += sloc[(b * 8 + k) * R + r];
                    xbn[r] = RowOps<TC>::master(mode, Ssum, xbs[size_t(cur) * rpc + gi * R + r], g, e, im);
                }
            }
            if (warp == 0 && lane < nr) {
                TC v = TC(0);
#pragma unroll
                for (int r = 0; r < R; ++r) v = (lane == r) ? xbn[r] : v;
                xbs[size_t(cur ^ 1) * rpc + gi * R + lane] = v;
            }

            // phase 2: z_i' += Q_i[j,:]^T coef_i[j]
            if (active) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const TC xr = __shfl_sync(0xffffffffu, xn, r);
                    if (r < nr) {
                        const TC cr = RowOps<TC>::coef(mode, xr, xbn[r], e, im);
#pragma unroll
                        for (int h = 0; h < H; ++h) {
                            TC qv[V];
                            load_vec<TQ, TC, V>(st + size_t(r) * nw * P + (h * 32 + lane) * V, qv);
#pragma unroll
                            for (int v = 0; v < V; ++v) acc[h * V + v] = fma(qv[v], cr, acc[h * V + v]);
                        }
                    }
                }
            }
        }

        // end of pass: publish z', clear the spare buffer, grid barrier
        {
            const int64_t t = a.t0 + it;
            TS *zout = zbuf + size_t((t + 1) % 3) * mP;
            TS *zsp = zbuf + size_t((t + 2) % 3) * mP;
            if (active) {
#pragma unroll
                for (int h = 0; h < H; ++h)
                    atomic_add_vec<TS>(zout + size_t(wk) * P + (h * 32 + lane) * V, acc + h * V, V);
            }
            for (size_t i = size_t(blockIdx.x) * blockDim.x + tid; i < mP; i += size_t(gridDim.x) * blockDim.x)
                zsp[i] = TS(0);
            cur ^= 1;
            if (it + 1 < a.iters) {
                __syncthreads();
                if (tid == 0) {
                    __threadfence();
                    red_release_add_u32(a.bar, 1u);
                    const uint32_t target = uint32_t(it + 1) * gridDim.x;
                    if (ld_acquire_u32(a.bar) < target) {
                        const uint64_t t_start = globaltimer_ns();
                        while (ld_acquire_u32(a.bar) < target) {
                            if (globaltimer_ns() - t_start > a.timeout_ns) {
                                abort_flag = 1;
                                abort_code = DEV_TIMEOUT_GRID;
                                break;
                            }
                        }
                    }
                    __threadfence();
                }
                if (__syncthreads_or(abort_flag)) goto abort_exit;
                load_z(t + 1);
            }
        }
    }

    // write the master's estimate for this cluster's rows
    if (rank == 0)
        for (int64_t i = tid; i < nrows; i += blockDim.x) xbar[row0 + i] = xbs[size_t(cur) * rpc + i];
    __syncthreads();
    cluster_sync_all();
    return;

abort_exit:
    if (tid == 0) {
        atomicCAS(a.err, 0, abort_code ? abort_code : DEV_TIMEOUT_TMA);
        // drain this CTA's bulk copies still in flight (bounded)
        for (int64_t qq = max(int64_t(0), issued - S); qq < issued; ++qq)
            (void)mbar_wait(&full[qq % S], uint32_t((qq / S) & 1), a.timeout_ns);
    }
    __syncthreads();
    cluster_sync_all();
}

template <int P_> struct Dummy {};

template <typename TQ, typename TS, int CPL>
constexpr int rows_per_group() { return sizeof(TQ) == 8 ? 2 : 4; }

template <typename TQ, typename TS, int CPL>
constexpr int max_threads() { return sizeof(TQ) == 8 ? 512 : 1024; }

template <typename TQ, typename TS, int CPL>
void *kernel_ptr() {
    return reinterpret_cast<void *>(
        &apc_iter_kernel<TQ, TS, CPL, rows_per_group<TQ, TS, CPL>(), max_threads<TQ, TS, CPL>()>);
}

template <typename TQ, typename TS>
void *kernel_for_cpl(int cpl) {
    switch (cpl) {
        case 1: return kernel_ptr<TQ, TS, 1>();
        case 2: return kernel_ptr<TQ, TS, 2>();
        case 4: return kernel_ptr<TQ, TS, 4>();
        case 8: return kernel_ptr<TQ, TS, 8>();
        default: return nullptr;
    }
}

void *kernel_for(int precision, int cpl) {
    switch (precision) {
        case 0: return kernel_for_cpl<double, double>(cpl);
        case 1: return kernel_for_cpl<float, float>(cpl);
        case 2: return kernel_for_cpl<__nv_bfloat16, float>(cpl);
        default: return nullptr;
    }
}

}  // namespace

int iter_rows_per_group(int precision) { return precision == 0 ? 2 : 4; }

size_t iter_smem_bytes(int precision, int cpl, int nw, int stages, int64_t rows_per_cluster) {
    const int P = 32 * cpl;
    switch (precision) {
        case 0: return SmemLayout<double, double, 2>(nw, P, stages, rows_per_cluster).total;
        case 1: return SmemLayout<float, float, 4>(nw, P, stages, rows_per_cluster).total;
        default: return SmemLayout<__nv_bfloat16, float, 4>(nw, P, stages, rows_per_cluster).total;
    }
}

static cudaLaunchConfig_t make_config(int cs, int nw, int clusters, size_t smem, cudaStream_t s,
                                      cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(clusters * cs), 1, 1);
    cfg.blockDim = dim3(unsigned(nw * 32), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(cs);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

int iter_max_clusters(int precision, int cpl, int cs, int nw, size_t smem) {
    void *k = kernel_for(precision, cpl);
    if (!k) return 0;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = make_config(cs, nw, 1, smem, nullptr, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_iter(int precision, int cpl, const IterArgs &a, int clusters, size_t smem, cudaStream_t s) {
    void *k = kernel_for(precision, cpl);
    if (!k) return cudaErrorInvalidValue;
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (err != cudaSuccess) return err;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = make_config(a.cs, a.nw, clusters, smem, s, attr);
    void *args[] = {const_cast<IterArgs *>(&a)};
    return cudaLaunchKernelExC(&cfg, k, args);
}

}  // namespace apc
