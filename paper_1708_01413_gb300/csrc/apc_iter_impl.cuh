// Persistent APC iteration kernel (Eq. (cons), Algorithm 1) for sm_103a.
//
// Work split.  The paper gives machine i the rows [A_i, b_i]; here the unknowns
// j = 0..n-1 are split into contiguous row ranges, one per thread-block
// cluster, and the m machines ("workers") into the CTAs of each cluster, one
// or two workers per warp.  Q is stored [n][m][P]: row j holds, for every
// worker i, the j-th row of Q_i (zero padded to P = 32*CPL columns).
//
// One pass over Q per iteration.  A cluster holds every worker's slice
// Q_i[j,:] of its rows on chip, so both skinny products of
// P_i y = y - Q_i (Q_i^T y) use it while it is resident:
//   w_i[j]   = Q_i[j,:] . z_i            (z_i = Q_i^T (xbar - x_i) from the last pass)
//   x_i[j]  += gamma (xbar[j] - x_i[j] - w_i[j])                      (cons1)
//   xbar[j]  = (eta/m) sum_i x_i[j] + (1 - eta) xbar[j]               (cons2)
//   z_i'    += Q_i[j,:]^T (xbar[j] - x_i[j])    (next pass's z_i, partial over j)
// The sum over workers in (cons2) is reduced across the warps of a CTA
// (shared memory) and across the CTAs of the cluster (st.async into the peers'
// shared memory, completing on their mbarriers).  Partial z_i' of all clusters
// are summed with global atomics, then one grid-wide barrier per iteration.
//
// Pipeline.  Rows go in groups of R = 2; one __syncthreads per step.  Step t
// computes the first product and the machines' updates of group t and sends
// the group's row sums to the cluster, and finishes group t-2: the master's
// new xbar (FP64, one lane per row) and the second product.  The two steps in
// between hide the cluster exchange.  Q rows stream into a ring of S
// shared-memory stages through TMA bulk copies (L2 evict-first); three stages
// are in use, S-3 are loading.
//
// Arithmetic (FP32 / BF16 Q).  Products accumulate in FP32 with packed FFMA2.
// xbar is kept in FP64 and as an FP32 hi+lo pair.  The row sums travel as
// compensated FP32 pairs and the master's update is FP64: with eta ~ 10..100
// a plain FP32 update would amplify rounding of the row sum by eta.  The
// machines' update x_i += gamma*v uses an error-free product and sum, so gamma
// enters with ~48 bits: near the optimum the roots of p_i are double and the
// iterates are very sensitive to gamma itself.
//
// MODE_APC is specialised; the other pass modes (least-norm initialisation,
// reverse sweep, products with X = (1/m) sum_i Q_i Q_i^T) share one
// instantiation with FP64 per-row arithmetic selected at run time.
//
// Every wait is bounded by timeout_ns (globaltimer); on expiry the kernel
// records an error word, drains its own bulk copies, joins a final cluster
// barrier and returns.
#pragma once
#include "apc_internal.h"
#include "apc_ptx.cuh"

namespace apc {
namespace iterk {

constexpr int R = kRowsPerGroup;   // rows per group (= 2, hard-wired below)
static_assert(R == 2, "the transposed butterfly and lane roles assume 2 rows per group");
constexpr int NX = 4;              // cluster exchange buffers (groups in flight)
constexpr int DELAY = 2;           // steps between a group's first and second product

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct SmemLayout {
    size_t stage_elems, row_stride, off_xbd, off_xbf, off_red, off_sloc, off_xbn, off_bars, total;
    __host__ __device__ SmemLayout(size_t q_elem, size_t s_elem, int slots, int P, int stages, int64_t rpc) {
        row_stride = size_t(slots) * P;               // elements per staged row
        stage_elems = size_t(R) * row_stride;
        // xbar [2][rpc], 8 bytes per row: FP64, or an FP32 hi/lo pair on the
        // double-float path (one launch uses one of the two views)
        off_xbd = align_up(size_t(stages) * stage_elems * q_elem, 128);
        off_xbf = off_xbd;
        off_red = align_up(off_xbd + 2 * size_t(rpc) * 8, 16);         // per-slot row terms [2][R][32]
        off_sloc = align_up(off_red + 2 * R * 32 * s_elem, 16);        // cluster row sums [NX][8][R]
        off_xbn = off_sloc + size_t(NX) * 8 * R * 8;                   // new xbar of a group [2][R] (hi/lo)
        off_bars = align_up(off_xbn + 2 * R * 8, 8);
        total = off_bars + (stages + NX) * sizeof(uint64_t);
    }
};

// Per-row arithmetic of the pass modes, FP64 (generic instantiation).
struct Row {
    __device__ static inline void update(int mode, double xo, double xb, double d, double g, double e, double im,
                                         double &xn, double &contrib) {
        switch (mode) {
            case MODE_APC: xn = xo + g * (xb - xo - d); contrib = xn; break;
            case MODE_INIT: xn = d; contrib = d; break;
            case MODE_ADJ: {
                const double mu = xo + e * im * xb;
                xn = (1.0 - g) * mu + g * d;
                contrib = mu - d;
            } break;
            case MODE_ADJ_SEED: xn = 0.0; contrib = 0.0; break;
            case MODE_ADJ_FINAL: xn = xo; contrib = 0.0; break;
            default: xn = 0.0; contrib = d; break;  // MODE_POWER
        }
    }
    __device__ static inline double master(int mode, double S, double xb, double g, double e, double im) {
        switch (mode) {
            case MODE_APC: return e * im * S + (1.0 - e) * xb;
            case MODE_INIT: return im * S;
            case MODE_ADJ: return (1.0 - e) * xb + g * S;
            case MODE_ADJ_SEED:
            case MODE_ADJ_FINAL: return xb;
            default: return im * S;
        }
    }
    __device__ static inline double coef(int mode, double xn, double xbn, double e, double im) {
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

// x + (gh + gl) * v with an error-free product and sum (FP32): gamma enters
// with ~48 bits and the result is rounded about once.
__device__ __forceinline__ float axpy_exact(float x, float gh, float gl, float v) {
    const float p = gh * v;
    const float pe = fmaf(gh, v, -p);
    const float c = fmaf(gl, v, pe);
    const float s = x + p;
    const float bb = s - x;
    const float se = (x - (s - bb)) + (p - bb);
    return s + (c + se);
}

// Load V elements of Q (16 bytes or fewer) and widen them to the compute type.
template <typename TQ, typename TC, int V>
__device__ __forceinline__ void load_row(const TQ *p, TC *out) {
    if constexpr (V * sizeof(TQ) == 16) {
        Elem<TQ>::load16(p, out);
    } else if constexpr (sizeof(TQ) == 2 && V == 4) {
        const uint2 w = *reinterpret_cast<const uint2 *>(p);
        out[0] = __uint_as_float(w.x << 16); out[1] = __uint_as_float(w.x & 0xffff0000u);
        out[2] = __uint_as_float(w.y << 16); out[3] = __uint_as_float(w.y & 0xffff0000u);
    } else if constexpr (sizeof(TQ) == 2 && V == 2) {
        const uint32_t w = *reinterpret_cast<const uint32_t *>(p);
        out[0] = __uint_as_float(w << 16); out[1] = __uint_as_float(w & 0xffff0000u);
    } else if constexpr (sizeof(TQ) == 4 && V == 2) {
        const float2 w = *reinterpret_cast<const float2 *>(p);
        out[0] = w.x; out[1] = w.y;
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) out[v] = static_cast<TC>(p[v]);
    }
}

// acc[0..V) += q[0..V) * c  (packed FFMA2 for FP32)
template <typename TC, int V>
__device__ __forceinline__ void axpy_vec(TC *acc, const TC *q, TC c) {
    if constexpr (sizeof(TC) == 4 && V % 2 == 0) {
        const float2 cc = make_float2(c, c);
#pragma unroll
        for (int v = 0; v < V; v += 2) {
            const float2 r = __ffma2_rn(make_float2(q[v], q[v + 1]), cc, make_float2(acc[v], acc[v + 1]));
            acc[v] = r.x;
            acc[v + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = fma(q[v], c, acc[v]);
    }
}

// two partial dot products (even / odd elements) of q and z
template <typename TC, int V>
__device__ __forceinline__ void dot_vec(TC &d0, TC &d1, const TC *q, const TC *z) {
    if constexpr (sizeof(TC) == 4 && V % 2 == 0) {
        float2 a = make_float2(d0, d1);
#pragma unroll
        for (int v = 0; v < V; v += 2) a = __ffma2_rn(make_float2(q[v], q[v + 1]), make_float2(z[v], z[v + 1]), a);
        d0 = a.x;
        d1 = a.y;
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if (v & 1) d1 = fma(q[v], z[v], d1);
            else d0 = fma(q[v], z[v], d0);
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

// compensated sum of a and b: returns a+b rounded, adds the rounding error to c
__device__ __forceinline__ float two_sum(float a, float b, float &c) {
    const float s = a + b;
    const float bb = s - a;
    c += (a - (s - bb)) + (b - bb);
    return s;
}

__device__ __forceinline__ uint64_t pack2(float hi, float lo) {
    return (uint64_t(__float_as_uint(lo)) << 32) | __float_as_uint(hi);
}

// double-float (hi + lo FP32 pair) arithmetic for the master's update
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    const float s = a.x + b.x;
    const float bb = s - a.x;
    float e = (a.x - (s - bb)) + (b.x - bb);
    e += a.y + b.y;
    const float hi = s + e;
    return make_float2(hi, e - (hi - s));
}

__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float hi = p + e;
    return make_float2(hi, e - (hi - p));
}

__device__ __forceinline__ float2 df_from(double v) {
    const float hi = float(v);
    return make_float2(hi, float(v - double(hi)));
}

template <typename TQ, typename TS, int CPL, int WPW, bool kAPC>
__global__ void __launch_bounds__(kMaxThreads, 1) apc_iter_kernel(const IterArgs a) {
    using TC = TS;
    constexpr bool kF64 = sizeof(TS) == 8;
    constexpr bool kDF = kAPC && !kF64;     // master update in double-float
    constexpr int VE = Elem<TQ>::V;
    constexpr int V = CPL < VE ? CPL : VE;  // elements per lane per vector
    constexpr int H = CPL / V;              // vectors per lane per row

    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int abort_flag;
    __shared__ int abort_code;

    const int P = a.P, nwe = a.nw, S = a.stages, m = a.m, cs = a.cs;
    const int W = nwe * WPW;  // worker slots per CTA
    const int rpc = int(a.rows_per_cluster);
    const SmemLayout L(sizeof(TQ), sizeof(TS), W, P, S, rpc);
    TQ *stage_base = reinterpret_cast<TQ *>(smem);
    double *xbd = reinterpret_cast<double *>(smem + L.off_xbd);   // [2][rpc]  FP64 xbar
    float2 *xbf = reinterpret_cast<float2 *>(smem + L.off_xbf);   // [2][rpc]  double-float xbar
    TS *red = reinterpret_cast<TS *>(smem + L.off_red);           // [2][R][32]
    uint64_t *sloc = reinterpret_cast<uint64_t *>(smem + L.off_sloc);  // [NX][8][R]
    float2 *xbn = reinterpret_cast<float2 *>(smem + L.off_xbn);   // [2][R] (double-float path)
    double *xbn_d = reinterpret_cast<double *>(smem + L.off_xbn);  // [2][R] (FP64 / generic path)
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L.off_bars);  // [S]
    uint64_t *xchg = full + S;                                          // [NX]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // warps [0, nwe) stream Q; warp nwe + r owns row r of each group (row sums,
    // cluster exchange, master update); lane 0 of warp nwe + 1 issues the TMA copies
    const bool is_ctl = warp >= nwe;
    const int ctl_r = warp - nwe;
    const int issuer = (nwe + 1) * 32;
    const uint32_t rank = cluster_rank();
    const int cl = int(cluster_id_x());
    const int w0 = int(rank) * W;
    const int W_cta = max(0, min(W, m - w0));
    const int64_t row0 = int64_t(cl) * rpc;
    const int nrows = int(max(int64_t(0), min(a.n, row0 + rpc) - row0));
    const int G = (nrows + R - 1) / R;  // groups per pass
    const int64_t total = int64_t(G) * a.iters;
    const uint32_t rowbytes = uint32_t(W_cta) * P * sizeof(TQ);
    const TQ *Qbase = reinterpret_cast<const TQ *>(a.Q) + size_t(w0) * P;  // this CTA's workers
    TS *xw = reinterpret_cast<TS *>(a.xw) + w0;
    TS *zbuf = reinterpret_cast<TS *>(a.zbuf);
    const int mode = kAPC ? int(MODE_APC) : a.mode;
    const bool rx = Row::reads_x(mode), wx = Row::writes_x(mode);
    const size_t mP = size_t(m) * P;
    const size_t qrow = size_t(m) * P;  // elements per row of Q
    const float g_hi = a.g_hi, g_lo = a.g_lo;
    const float2 c_em = make_float2(a.em_hi, a.em_lo);  // eta / m
    const float2 c_1e = make_float2(a.e1_hi, a.e1_lo);  // 1 - eta

    // byte offsets of this lane's Q vectors within a stage: [slot][row][vector]
    uint32_t qoff[WPW][R][H];
#pragma unroll
    for (int sl = 0; sl < WPW; ++sl)
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int h = 0; h < H; ++h)
                qoff[sl][r][h] = uint32_t((r * L.row_stride + (warp * WPW + sl) * P + (h * 32 + lane) * V) * sizeof(TQ));
    const uint32_t stage_bytes = uint32_t(L.stage_elems * sizeof(TQ));
    const unsigned char *stage_bytes_base = smem;

    // element warps: lane (r_l, s_l) updates row r_l of worker slot s_l
    const int r_l = lane >> 4, s_l = lane & 15;
    const bool upd_lane = !is_ctl && s_l < WPW;
    const int wl_upd = warp * WPW + s_l;  // CTA-local worker slot
    const bool upd_active = upd_lane && wl_upd < W_cta;

    if (tid == 0) {
        abort_flag = 0;
        abort_code = 0;
        for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
        for (int s = 0; s < NX; ++s) mbar_init(&xchg[s], R);
        fence_mbar_init_cluster();
    }
    for (int i = tid; i < nrows; i += blockDim.x) {
        const double v = a.xbar[row0 + i];
        if constexpr (kDF) xbf[i] = df_from(v);
        else xbd[i] = v;
    }
    // Zero the stage ring once: rows past the end of a group and worker slots
    // past the CTA's last worker are never written by TMA, so the element loops
    // below read finite values there and need no per-row or per-slot guards
    // (their results are discarded or multiplied by zero).
    {
        uint4 *p = reinterpret_cast<uint4 *>(smem);
        const size_t n16 = size_t(S) * L.stage_elems * sizeof(TQ) / 16;
        for (size_t i = tid; i < n16; i += blockDim.x) p[i] = make_uint4(0, 0, 0, 0);
        fence_proxy_async_shared();
    }
    __syncthreads();
    cluster_sync_all();  // peers' barriers are initialised before any st.async

    // ---- TMA producer state (thread `issuer`) ----
    uint64_t policy = 0;
    int64_t issued = 0;
    int is_stage = 0, is_k = 0;
    auto issue_next = [&]() {
        const int r0 = is_k * R;
        const int nr = min(R, nrows - r0);
        mbar_arrive_expect_tx(&full[is_stage], uint32_t(nr) * rowbytes);
        TQ *dst = stage_base + size_t(is_stage) * L.stage_elems;
        const TQ *src = Qbase + size_t(row0 + r0) * qrow;
        for (int r = 0; r < nr; ++r) tma_load_1d(dst + size_t(r) * L.row_stride, src + size_t(r) * qrow, rowbytes,
                                                 &full[is_stage], policy);
        ++issued;
        if (++is_stage == S) is_stage = 0;
        if (++is_k == G) is_k = 0;
    };
    if (tid == issuer && W_cta > 0 && G > 0) {
        policy = policy_evict_first();
        while (issued < min(int64_t(S - 3), total)) issue_next();
    }

    // z_i (this pass's input) and the partial z_i' (output), per worker slot
    TC z[WPW][CPL], acc[WPW][CPL];
    auto load_z = [&](int64_t t) {
        const TS *zin = zbuf + size_t(t % 3) * mP + size_t(w0) * P;
#pragma unroll
        for (int s = 0; s < WPW; ++s) {
            const int wl = warp * WPW + s;
            const bool act = !is_ctl && wl < W_cta;
#pragma unroll
            for (int h = 0; h < H; ++h)
#pragma unroll
                for (int v = 0; v < V; ++v)
                    z[s][h * V + v] = act ? __ldcg(zin + size_t(wl) * P + (h * 32 + lane) * V + v) : TC(0);
#pragma unroll
            for (int c = 0; c < CPL; ++c) acc[s][c] = TC(0);
        }
    };
    load_z(a.t0);

    // previous x_i of (row r_l, slot s_l) of pass-local group k, loaded ahead
    auto xload = [&](int k) -> TS {
        if (!rx || !upd_active) return TS(0);
        const int li = k * R + r_l;
        return li < nrows ? xw[size_t(row0 + li) * m + wl_upd] : TS(0);
    };
    TS xpre = G > 0 ? xload(0) : TS(0);
    TS x1 = TS(0), x2 = TS(0);  // this lane's x_i' of groups t-1 and t-2
    int nr1 = 0, nr2 = 0;       // row counts of groups t-1 and t-2
    int st1 = 0, ph1 = 0;       // stage / parity of the next first-product group
    int st2 = 0;                // stage of the next second-product group
    int cur = 0;

    for (int64_t it = 0; it < a.iters; ++it) {
        const int64_t gbase = it * G;
        for (int t = 0; t < G + DELAY && G > 0; ++t) {
            const bool has1 = t < G, has2 = t >= DELAY;
            const int nr = has1 ? min(R, nrows - t * R) : 0;
            const int64_t g = gbase + t;   // global index of group t (first product)
            const int64_t g2 = g - DELAY;  // global index of group t-2 (second product)
            TS xn_cur = TS(0);

            if (!is_ctl) {
                // ---- first product and machines' updates of group t ----
                if (has1) {
                    if (W_cta > 0 && !mbar_wait(&full[st1], uint32_t(ph1), a.timeout_ns)) {
                        abort_flag = 1;
                        abort_code = DEV_TIMEOUT_TMA;
                    }
                    const unsigned char *stb = stage_bytes_base + uint32_t(st1) * stage_bytes;
                    TC dsum[WPW];
#pragma unroll
                    for (int sl = 0; sl < WPW; ++sl) {
                        TC dr[R];
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            TC d0 = TC(0), d1 = TC(0);
#pragma unroll
                            for (int h = 0; h < H; ++h) {
                                TC qv[V];
                                load_row<TQ, TC, V>(reinterpret_cast<const TQ *>(stb + qoff[sl][r][h]), qv);
                                dot_vec<TC, V>(d0, d1, qv, &z[sl][h * V]);
                            }
                            dr[r] = d0 + d1;
                        }
                        // transposed butterfly: lanes 0-15 end with row 0, lanes 16-31 with row 1
                        TC keep = (lane & 16) ? dr[1] : dr[0];
                        const TC send = (lane & 16) ? dr[0] : dr[1];
                        keep += __shfl_xor_sync(0xffffffffu, send, 16);
#pragma unroll
                        for (int off = 8; off > 0; off >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, off);
                        dsum[sl] = keep;
                    }
                    TC myd = dsum[0];
#pragma unroll
                    for (int sl = 1; sl < WPW; ++sl) myd = (s_l == sl) ? dsum[sl] : myd;
                    TS contrib = TS(0);
                    if (upd_active && r_l < nr) {
                        const int li = t * R + r_l;
                        if constexpr (kDF) {
                            const float2 xb = xbf[cur * rpc + li];
                            const float xo = xpre;
                            const float v = ((xb.x - xo) + xb.y) - myd;
                            xn_cur = axpy_exact(xo, g_hi, g_lo, v);
                            contrib = xn_cur;
                        } else {
                            double xn, cb;
                            Row::update(mode, double(xpre), xbd[cur * rpc + li], double(myd), a.gamma, a.eta,
                                        a.inv_m, xn, cb);
                            xn_cur = TS(xn);
                            contrib = (mode == MODE_APC || mode == MODE_INIT) ? xn_cur : TS(cb);
                        }
                        if (wx) xw[size_t(row0 + li) * m + wl_upd] = xn_cur;
                    }
                    if (upd_lane) red[((int(g) & 1) * R + r_l) * 32 + wl_upd] = contrib;
                    // x_i of the next group, loaded after the store above (with one
                    // group per pass the next group is the same rows)
                    xpre = xload(t + 1 < G ? t + 1 : 0);
                }
            } else if (has2 && ctl_r < R && lane == 0) {
                // ---- master of row ctl_r of group t-2: cluster row sums -> new xbar ----
                const int r = ctl_r;
                const int bx = int(g2 & (NX - 1));
                if (!mbar_wait(&xchg[bx], uint32_t((g2 >> 2) & 1), a.timeout_ns)) {
                    abort_flag = 1;
                    abort_code = DEV_TIMEOUT_XCHG;
                }
                if (r < nr2) {
                    const int li = (t - DELAY) * R + r;
                    if constexpr (kDF) {
                        float2 Ssum = make_float2(0.0f, 0.0f);
                        for (int kk = 0; kk < cs; ++kk) {
                            const uint64_t w = sloc[(bx * 8 + kk) * R + r];
                            Ssum = df_add(Ssum, make_float2(__uint_as_float(uint32_t(w)), __uint_as_float(uint32_t(w >> 32))));
                        }
                        const float2 xnew = df_add(df_mul(c_em, Ssum), df_mul(c_1e, xbf[cur * rpc + li]));
                        xbf[(cur ^ 1) * rpc + li] = xnew;
                        xbn[(int(g2) & 1) * R + r] = xnew;
                    } else {
                        double Ssum = 0.0;
                        for (int kk = 0; kk < cs; ++kk) {
                            const uint64_t w = sloc[(bx * 8 + kk) * R + r];
                            if constexpr (kF64) Ssum += __longlong_as_double(static_cast<long long>(w));
                            else Ssum += double(__uint_as_float(uint32_t(w))) + double(__uint_as_float(uint32_t(w >> 32)));
                        }
                        const double xnew = Row::master(mode, Ssum, xbd[cur * rpc + li], a.gamma, a.eta, a.inv_m);
                        xbd[(cur ^ 1) * rpc + li] = xnew;
                        xbn_d[(int(g2) & 1) * R + r] = xnew;
                    }
                }
            }

            if (__syncthreads_or(abort_flag)) goto abort_exit;

            if (!is_ctl) {
                // ---- second product of group t-2: z_i' += Q_i[j,:]^T coef_i[j] ----
                if (has2) {
                    const unsigned char *stb = stage_bytes_base + uint32_t(st2) * stage_bytes;
                    TC myc = TC(0);
                    if (upd_active && r_l < nr2) {
                        if constexpr (kDF) {
                            const float2 xb = xbn[(int(g2) & 1) * R + r_l];
                            myc = (xb.x - x2) + xb.y;
                        } else {
                            myc = TC(Row::coef(mode, double(x2), xbn_d[(int(g2) & 1) * R + r_l], a.eta, a.inv_m));
                        }
                    }
#pragma unroll
                    for (int sl = 0; sl < WPW; ++sl) {
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            const TC cr = __shfl_sync(0xffffffffu, myc, r * 16 + sl);
#pragma unroll
                            for (int h = 0; h < H; ++h) {
                                TC qv[V];
                                load_row<TQ, TC, V>(reinterpret_cast<const TQ *>(stb + qoff[sl][r][h]), qv);
                                axpy_vec<TC, V>(&acc[sl][h * V], qv, cr);
                            }
                        }
                    }
                }
            } else if (has1 && ctl_r < R) {
                if (tid == issuer && W_cta > 0 && issued < total) issue_next();
                // ---- this CTA's sum of row ctl_r of group t, sent to every CTA of the cluster ----
                const int r = ctl_r;
                const int bx = int(g & (NX - 1));
                uint64_t payload;
                if constexpr (kF64) {
                    double v = (lane < W) ? double(red[((int(g) & 1) * R + r) * 32 + lane]) : 0.0;
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                    payload = uint64_t(__double_as_longlong(v));
                } else {
                    float sv = (lane < W) ? float(red[((int(g) & 1) * R + r) * 32 + lane]) : 0.0f;
                    float cv = 0.0f;
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) {
                        const float so = __shfl_xor_sync(0xffffffffu, sv, off);
                        const float co = __shfl_xor_sync(0xffffffffu, cv, off);
                        cv += co;
                        sv = two_sum(sv, so, cv);
                    }
                    payload = pack2(sv, cv);
                }
                if (lane == 0) {
                    if (r < nr) {
                        uint64_t *slot = &sloc[(bx * 8 + rank) * R + r];
                        *slot = payload;
                        for (int kk = 0; kk < cs; ++kk) {
                            if (kk == int(rank)) continue;
                            st_async_b64(map_shared_rank(smem_u32(slot), kk), payload,
                                         map_shared_rank(smem_u32(&xchg[bx]), kk));
                        }
                    }
                    mbar_arrive_expect_tx(&xchg[bx], r < nr ? uint32_t((cs - 1) * 8) : 0u);
                }
            }
            if (has2 && ++st2 == S) st2 = 0;
            if (has1 && ++st1 == S) {
                st1 = 0;
                ph1 ^= 1;
            }
            // shift this lane's per-group history: group t becomes t-1, t-1 becomes t-2
            x2 = x1;
            x1 = xn_cur;
            nr2 = nr1;
            nr1 = nr;
        }

        // ---- end of pass: publish z', clear the spare buffer, grid barrier ----
        {
            const int64_t tp = a.t0 + it;
            TS *zout = zbuf + size_t((tp + 1) % 3) * mP + size_t(w0) * P;
            TS *zsp = zbuf + size_t((tp + 2) % 3) * mP;
            if (!is_ctl) {
#pragma unroll
                for (int sl = 0; sl < WPW; ++sl) {
                    const int wl = warp * WPW + sl;
                    if (wl < W_cta) {
#pragma unroll
                        for (int h = 0; h < H; ++h)
                            atomic_add_vec<TS>(zout + size_t(wl) * P + (h * 32 + lane) * V, &acc[sl][h * V], V);
                    }
                }
            }
            for (size_t i = size_t(blockIdx.x) * blockDim.x + tid; i < mP; i += size_t(gridDim.x) * blockDim.x)
                zsp[i] = TS(0);
            cur ^= 1;
            if (it + 1 < a.iters) {
                __syncthreads();
                if (tid == 0) {
                    __threadfence();
                    red_release_add_u32(a.bar, 1u);
                    const uint32_t target = uint32_t(it + 1) * gridDim.x + a.barrier_skew;
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
                load_z(tp + 1);
            }
        }
    }

    // the master's estimate for this cluster's rows
    if (rank == 0) {
        for (int i = tid; i < nrows; i += blockDim.x) {
            if constexpr (kDF) {
                const float2 v = xbf[cur * rpc + i];
                a.xbar[row0 + i] = double(v.x) + double(v.y);
            } else {
                a.xbar[row0 + i] = xbd[cur * rpc + i];
            }
        }
    }
    __syncthreads();
    cluster_sync_all();
    return;

abort_exit:
    if (tid == issuer) {
        atomicCAS(a.err, 0, abort_code ? abort_code : DEV_TIMEOUT_TMA);
        // drain this CTA's bulk copies still in flight (bounded)
        for (int64_t qq = max(int64_t(0), issued - S); qq < issued; ++qq)
            (void)mbar_wait(&full[qq % S], uint32_t((qq / S) & 1), a.timeout_ns);
    }
    if (tid == 0) atomicCAS(a.err, 0, abort_code ? abort_code : DEV_TIMEOUT_TMA);
    __syncthreads();
    cluster_sync_all();
}

template <typename TQ, typename TS>
void *kernel_for(int cpl, int wpw, bool apc) {
#define APC_K(C, WP) (apc ? reinterpret_cast<void *>(&apc_iter_kernel<TQ, TS, C, WP, true>) \
                          : reinterpret_cast<void *>(&apc_iter_kernel<TQ, TS, C, WP, false>))
    if (wpw == 1) {
        switch (cpl) {
            case 2: return APC_K(2, 1);
            case 4: return APC_K(4, 1);
            case 8: return APC_K(8, 1);
        }
    } else if (wpw == 2) {
        switch (cpl) {
            case 2: return APC_K(2, 2);
            case 4: return APC_K(4, 2);
            case 8: return APC_K(8, 2);
        }
    }
#undef APC_K
    return nullptr;
}

}  // namespace iterk
}  // namespace apc
