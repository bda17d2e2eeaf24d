// Persistent APC iteration kernel (Eq. (cons), Algorithm 1) for sm_103a.
//
// Work split.  The paper gives machine i the rows [A_i, b_i]; here the unknowns
// j = 0..n-1 are split into contiguous row ranges, one per thread-block
// cluster, and the m machines ("workers") into the CTAs of each cluster, one,
// two or four workers per warp.  Q is stored [n][m][P]: row j holds, for every
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
// Pipeline.  Rows go in groups of R = 2 (or R = 1 where two rows of Q per
// stage would not leave a deep enough ring); one __syncthreads per step.
// Element warps stream Q: step t computes the first product of group t and
// the second product of group t-3.  Each row of a group has two control warps,
// one lane per worker slot: after the barrier of step t one finishes the
// master's update of group t-2 (its cluster exchange was sent two steps
// earlier) and writes the second product's coefficients, the other applies
// the machines' updates of group t, forms the CTA row sum and sends it to the
// cluster.  Q rows stream
// into a ring of S shared-memory stages through TMA bulk copies (L2
// evict-first); four stages are in use, S-4 are loading.
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
#include <type_traits>

#include "apc_internal.h"
#include "apc_ptx.cuh"

namespace apc {
namespace iterk {

// Cluster exchange buffers (groups in flight).  A peer writes group g + NX's
// row sums into the slot of group g only after its master has seen this CTA's
// sums of group g + NX - 2, which this CTA's update warps send in step
// t + NX - 2; this CTA's master reads group g in step t + 2.  NX >= 5 keeps the
// read before the overwrite (and one mbarrier phase per slot in flight).
constexpr int NX_LOG2 = 3;
constexpr int NX = 1 << NX_LOG2;

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct SmemLayout {
    size_t stage_elems, row_stride, off_xb, off_d, off_coef, off_sloc, off_xh, off_bars, total;
    // R = rows per group (1 or 2)
    __host__ __device__ SmemLayout(size_t q_elem, size_t s_elem, int slots, int P, int stages, int64_t rpc, int R) {
        row_stride = size_t(slots) * P;               // elements per staged row
        stage_elems = size_t(R) * row_stride;
        // xbar [2][rpc], 8 bytes per row: FP64, or an FP32 hi/lo pair on the
        // double-float path (one launch uses one of the two views)
        off_xb = align_up(size_t(stages) * stage_elems * q_elem, 128);
        off_d = align_up(off_xb + 2 * size_t(rpc) * 8, 16);        // first-product results [2][R][32]
        off_coef = align_up(off_d + 2 * R * 32 * s_elem, 16);      // second-product coefficients [2][32][R]
        off_sloc = align_up(off_coef + 2 * 32 * R * s_elem, 16);   // cluster row sums [NX][8][R]
        off_xh = align_up(off_sloc + size_t(NX) * 8 * R * 8, 16);  // machines' x_i' by group [4][R][32]
        off_bars = align_up(off_xh + size_t(4) * R * 32 * s_elem, 8);
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

template <typename TQ, typename TS, int CPL, int WPW, bool kAPC, int R, bool kDet>
// At most 32 worker slots per CTA: 32 / WPW element warps (16 for one worker
// per warp) plus the control warps and the producer warp.  Four workers per
// warp run 8 element warps with up to ~150 registers per thread.
__global__ void __launch_bounds__(((WPW >= 2 ? 32 / WPW : kMaxElemWarps) + kCtlWarps + kProducerWarps) * 32, 1)
    apc_iter_kernel(const IterArgs a) {
    static_assert(R == 1 || R == 2, "one or two rows per group");
    using TC = TS;
    constexpr bool kF64 = sizeof(TS) == 8;
    constexpr bool kDF = kAPC && !kF64;     // master update in double-float
    constexpr int VE = Elem<TQ>::V;
    constexpr int V = CPL < VE ? CPL : VE;  // elements per lane per vector
    constexpr int H = CPL / V;              // vectors per lane per row
    constexpr int NV = WPW * R;             // dot products per element warp and step
    constexpr int LNV = NV >= 8 ? 3 : NV >= 4 ? 2 : NV >= 2 ? 1 : 0;
    static_assert(NV == 1 << LNV, "workers per warp times rows per group must be a power of two");

    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int abort_flag;
    __shared__ int abort_code;

    const int P = a.P, nwe = a.nw, S = a.stages, m = a.m, cs = a.cs;
    const int W = nwe * WPW;  // worker slots per CTA (<= 32)
    const int rpc = int(a.rows_per_cluster);
    const SmemLayout L(sizeof(TQ), sizeof(TS), W, P, S, rpc, R);
    TQ *stage_base = reinterpret_cast<TQ *>(smem);
    double *xbd = reinterpret_cast<double *>(smem + L.off_xb);  // [2][rpc] FP64 xbar
    float2 *xbf = reinterpret_cast<float2 *>(smem + L.off_xb);  // [2][rpc] double-float xbar (same bytes)
    TS *dsh = reinterpret_cast<TS *>(smem + L.off_d);           // [2][R][32]  w_i[j] from the first product
    TS *coefs = reinterpret_cast<TS *>(smem + L.off_coef);      // [2][32][R]  coefficients of the second product
    uint64_t *sloc = reinterpret_cast<uint64_t *>(smem + L.off_sloc);  // [NX][8][R] cluster row sums
    TS *xhist = reinterpret_cast<TS *>(smem + L.off_xh);               // [4][R][32] x_i' of recent groups
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L.off_bars);  // [S]
    uint64_t *xchg = full + S;                                          // [NX]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // Warps [0, nwe) stream Q (both products).  2R control warps own the
    // rows of a group; lane s handles worker slot s.  Control warp r (r < R)
    // runs the master's update of row r of group t-2 and the second product's
    // coefficients; control warp R + r runs the machines' updates of row r of
    // group t, the CTA row sum and the cluster exchange.  The two chains are
    // independent within a step (they meet through shared memory two steps
    // apart), so a step waits for the longer of them, not their sum.  The last
    // warp only produces: its lane 0 issues the TMA copies of the ring.  A
    // bulk copy of a 16 KB row takes a few hundred cycles to issue, which on a
    // control warp delayed that warp's chain by as much every step.
    const bool is_ctl = warp >= nwe;  // every warp that is not an element warp
    const int ctl_r = warp - nwe;
    const int ctl_row = R == 2 ? (ctl_r & 1) : 0;
    const bool ctl_master = is_ctl && ctl_r < R;
    const bool ctl_update = is_ctl && ctl_r >= R && ctl_r < 2 * R;
    const bool is_prod = ctl_r == 2 * R;
    const int issuer = (nwe + 2 * R) * 32;
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
    // read finite values there and need no guards (their results are discarded
    // or multiplied by a zero coefficient).
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
        while (issued < min(int64_t(S - 4), total)) issue_next();
    }

    // ---- element warps: z_i (this pass's input) and the partial z_i' (output) ----
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
    // after the butterfly, lane group k = lane >> (5 - LNV) holds dot product k
    // (worker slot k / R, row k % R); its first lane publishes it
    const int k_l = lane >> (5 - LNV);
    const int r_l = k_l % R, s_l = k_l / R;
    const bool d_lane = !is_ctl && (lane & ((32 >> LNV) - 1)) == 0;
    const int wl_d = warp * WPW + s_l;

    // ---- control warps: x_i of (row ctl_r, slot lane), one group ahead ----
    const bool c_act = is_ctl && lane < W_cta;
    TS *const cx0 = xw + size_t(row0 + ctl_row) * m + lane;
    const size_t xstep = size_t(R) * m;
    const bool cx_ok = rx && c_act && ctl_update;
    TS *cx_next = cx0;
    int k_next = 0;
    auto cx_load_next = [&]() -> TS {
        TS v = TS(0);
        if (cx_ok && k_next * R + ctl_row < nrows) v = *cx_next;
        if (++k_next == G) {
            k_next = 0;
            cx_next = cx0;
        } else {
            cx_next += xstep;
        }
        return v;
    };
    TS cxpre = (ctl_update && G > 0) ? cx_load_next() : TS(0);
    TS *cx_cur = cx0;

    uint32_t sb1 = 0, sb2 = 0;  // stage byte offsets: first product (group t), second (group t-3)
    int st1 = 0, ph1 = 0;
    int gpass = 0;              // global index of group 0 of the current pass
    int cur = 0;

    // Step t: first product of group t; master and coefficients of group t-2
    // (control warps); second product of group t-3.  Returns true on a timeout.
    auto step = [&](int t) -> bool {
        const bool e1 = t < G, mm = t >= 2 && t - 2 < G, e2 = t >= 3;
        const int g = gpass + t;
        const int nr = e1 ? min(R, nrows - t * R) : 0;
        if (!is_ctl) {
            if (e1) {
                if (W_cta > 0 && !mbar_wait(&full[st1], uint32_t(ph1), a.timeout_ns)) {
                    abort_flag = 1;
                    abort_code = DEV_TIMEOUT_TMA;
                }
                const unsigned char *stb = smem + sb1;
                // the lane's partial sums of the warp's NV = WPW * R dot products
                // (k = slot * R + row)
                TC dv[NV];
#pragma unroll
                for (int sl = 0; sl < WPW; ++sl) {
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        TC d0 = TC(0), d1 = TC(0);
#pragma unroll
                        for (int h = 0; h < H; ++h) {
                            TC qv[V];
                            load_row<TQ, TC, V>(reinterpret_cast<const TQ *>(stb + qoff[sl][r][h]), qv);
                            dot_vec<TC, V>(d0, d1, qv, &z[sl][h * V]);
                        }
                        dv[sl * R + r] = d0 + d1;
                    }
                }
                // Transposed butterfly: at offsets 16, 8, ... each lane keeps half
                // of its values and receives its partner's partial sums of them,
                // so NV sums over 32 lanes take NV - 1 + 5 - log2(NV) shuffles
                // (one sum per lane group of 32 / NV lanes at the end).
#pragma unroll
                for (int lv = 0; lv < LNV; ++lv) {
                    const int half = NV >> (lv + 1);
                    const bool up = (lane >> (4 - lv)) & 1;
#pragma unroll
                    for (int k = 0; k < half; ++k) {
                        const TC keep = up ? dv[k + half] : dv[k];
                        const TC send = up ? dv[k] : dv[k + half];
                        dv[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16 >> lv);
                    }
                }
#pragma unroll
                for (int off = 16 >> LNV; off > 0; off >>= 1) dv[0] += __shfl_xor_sync(0xffffffffu, dv[0], off);
                if (d_lane) dsh[((g & 1) * R + r_l) * 32 + wl_d] = dv[0];
            }
        }

        if (__syncthreads_or(abort_flag)) return true;

        if (!is_ctl) {
            if (e2) {
                // ---- second product of group t-3: z_i' += Q_i[j,:]^T coef_i[j] ----
                const int g3 = g - 3;
                const unsigned char *stb = smem + sb2;
#pragma unroll
                for (int sl = 0; sl < WPW; ++sl) {
                    const TS *cp = coefs + ((g3 & 1) * 32 + warp * WPW + sl) * R;
                    TC cr[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) cr[r] = cp[r];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
#pragma unroll
                        for (int h = 0; h < H; ++h) {
                            TC qv[V];
                            load_row<TQ, TC, V>(reinterpret_cast<const TQ *>(stb + qoff[sl][r][h]), qv);
                            axpy_vec<TC, V>(&acc[sl][h * V], qv, cr[r]);
                        }
                    }
                }
                sb2 += stage_bytes;
                if (sb2 == uint32_t(S) * stage_bytes) sb2 = 0;
            }
            if (e1 && ++st1 == S) {
                st1 = 0;
                ph1 ^= 1;
            }
            sb1 = uint32_t(st1) * stage_bytes;
        } else {
            const int r = ctl_row;
            if (is_prod) {
                if (e1 && tid == issuer && W_cta > 0 && issued < total) issue_next();
            }
            const int nrh2 = (t >= 2 && t - 2 < G) ? min(R, nrows - (t - 2) * R) : 0;
            if (ctl_master && mm) {
                // ---- master of row r of group t-2: cluster row sums -> new xbar, coefficients ----
                const int g2 = g - 2;
                const int bx = g2 & (NX - 1);
                const int li = (t - 2) * R + r;
                if constexpr (kDF) {
                    if (lane == 0 && !mbar_wait(&xchg[bx], uint32_t((g2 >> NX_LOG2) & 1), a.timeout_ns)) {
                        abort_flag = 1;
                        abort_code = DEV_TIMEOUT_XCHG;
                    }
                    __syncwarp();
                    // lane kk < cs reads the row sum of cluster rank kk; a double-float
                    // tree over lanes 0-7, then every lane takes the total and forms
                    // xbar' itself (shorter than a serial sum in lane 0 and a broadcast:
                    // this chain paces the step)
                    float2 Ssum = make_float2(0.0f, 0.0f);
                    if (lane < cs && r < nrh2) {
                        const uint64_t w = sloc[(bx * 8 + lane) * R + r];
                        Ssum = make_float2(__uint_as_float(uint32_t(w)), __uint_as_float(uint32_t(w >> 32)));
                    }
                    // Only the rounds the cluster size needs (2 for 4 CTAs, 1 for 2): two-row
                    // steps gain 4-7 %.  The one-row instantiation keeps the unrolled three
                    // rounds: with the shorter loop it measured 4 % slower.
                    if constexpr (R == 2) {
                        for (int off = 1; off < cs; off <<= 1)
                            Ssum = df_add(Ssum, make_float2(__shfl_xor_sync(0xffffffffu, Ssum.x, off),
                                                            __shfl_xor_sync(0xffffffffu, Ssum.y, off)));
                    } else {
#pragma unroll
                        for (int off = 1; off < 8; off <<= 1)
                            Ssum = df_add(Ssum, make_float2(__shfl_xor_sync(0xffffffffu, Ssum.x, off),
                                                            __shfl_xor_sync(0xffffffffu, Ssum.y, off)));
                    }
                    Ssum.x = __shfl_sync(0xffffffffu, Ssum.x, 0);
                    Ssum.y = __shfl_sync(0xffffffffu, Ssum.y, 0);
                    float2 xnew = make_float2(0.0f, 0.0f);
                    if (r < nrh2) {
                        xnew = df_add(df_mul(c_em, Ssum), df_mul(c_1e, xbf[cur * rpc + li]));
                        if (lane == 0) xbf[(cur ^ 1) * rpc + li] = xnew;
                    }
                    const TS xh2 = xhist[((g2 & 3) * R + r) * 32 + lane];
                    const TS c = (r < nrh2 && lane < W_cta) ? TS((xnew.x - float(xh2)) + xnew.y) : TS(0);
                    coefs[((g2 & 1) * 32 + lane) * R + r] = c;
                } else {
                    double xnew = 0.0;
                    if (lane == 0) {
                        if (!mbar_wait(&xchg[bx], uint32_t((g2 >> NX_LOG2) & 1), a.timeout_ns)) {
                            abort_flag = 1;
                            abort_code = DEV_TIMEOUT_XCHG;
                        }
                        if (r < nrh2) {
                            double Ssum = 0.0;
                            for (int kk = 0; kk < cs; ++kk) {
                                const uint64_t w = sloc[(bx * 8 + kk) * R + r];
                                if constexpr (kF64) Ssum += __longlong_as_double(static_cast<long long>(w));
                                else Ssum += double(__uint_as_float(uint32_t(w))) +
                                             double(__uint_as_float(uint32_t(w >> 32)));
                            }
                            xnew = Row::master(mode, Ssum, xbd[cur * rpc + li], a.gamma, a.eta, a.inv_m);
                            xbd[(cur ^ 1) * rpc + li] = xnew;
                        }
                    }
                    xnew = __shfl_sync(0xffffffffu, xnew, 0);
                    const TS xh2 = xhist[((g2 & 3) * R + r) * 32 + lane];
                    const TS c = (r < nrh2 && lane < W_cta)
                                     ? TS(Row::coef(mode, double(xh2), xnew, a.eta, a.inv_m)) : TS(0);
                    coefs[((g2 & 1) * 32 + lane) * R + r] = c;
                }
            }
            if (ctl_update && e1) {
                // ---- machines' updates of row r of group t and the CTA row sum ----
                TS xn = TS(0), contrib = TS(0);
                if (r < nr && c_act) {
                    const int li = t * R + r;
                    const TS d = dsh[((g & 1) * R + r) * 32 + lane];
                    if constexpr (kDF) {
                        const float2 xb = xbf[cur * rpc + li];
                        const float xo = cxpre;
                        const float v = ((xb.x - xo) + xb.y) - d;
                        xn = axpy_exact(xo, g_hi, g_lo, v);
                        contrib = xn;
                    } else {
                        double xnd, cb;
                        Row::update(mode, double(cxpre), xbd[cur * rpc + li], double(d), a.gamma, a.eta, a.inv_m,
                                    xnd, cb);
                        xn = TS(xnd);
                        contrib = (mode == MODE_APC || mode == MODE_INIT) ? xn : TS(cb);
                    }
                    if (wx) *cx_cur = xn;
                }
                // x_i of the next group, loaded after the store above (with one
                // group per pass the next group is the same rows)
                cxpre = cx_load_next();
                cx_cur = (t + 1 < G) ? cx_cur + xstep : cx0;
                xhist[((g & 3) * R + r) * 32 + lane] = xn;  // read by the master's warp two steps later
                const int bx = g & (NX - 1);
                uint64_t payload;
                if constexpr (kF64) {
                    double v = double(contrib);
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
                    payload = uint64_t(__double_as_longlong(v));
                } else {
                    float sv = float(contrib), cv = 0.0f;
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
        }
        return false;
    };

    for (int64_t it = 0; it < a.iters; ++it) {
        cx_cur = cx0;
        for (int t = 0; t < G + 3 && G > 0; ++t)
            if (step(t)) goto abort_exit;
        gpass += G;

        // ---- end of pass: publish z', clear the spare buffer, grid barrier ----
        if constexpr (kDet) {
            // deterministic (a separate instantiation): this cluster's partial
            // z' for its workers; after a grid barrier (every partial visible)
            // the CTAs sum the partials in cluster order into the z buffer
            // (each a strided slice), then a second barrier before the next
            // pass reads it.  Barriers per launch: two per pass.
            const int64_t tp = a.t0 + it;
            TS *zp = reinterpret_cast<TS *>(a.zpart) + size_t(cl) * mP + size_t(w0) * P;
            if (!is_ctl) {
#pragma unroll
                for (int sl = 0; sl < WPW; ++sl) {
                    const int wl = warp * WPW + sl;
                    if (wl < W_cta) {
#pragma unroll
                        for (int h = 0; h < H; ++h)
#pragma unroll
                            for (int v = 0; v < V; ++v)
                                __stcg(zp + size_t(wl) * P + (h * 32 + lane) * V + v, acc[sl][h * V + v]);
                    }
                }
            }
            cur ^= 1;
            for (int pass2 = 0; pass2 < 2; ++pass2) {
                if (pass2 == 1) {
                    const TS *zpa = reinterpret_cast<const TS *>(a.zpart);
                    TS *zfull = zbuf + size_t((tp + 1) % 3) * mP;
                    const int ncl = int(gridDim.x) / cs;
                    for (size_t i = size_t(blockIdx.x) * blockDim.x + tid; i < mP;
                         i += size_t(gridDim.x) * blockDim.x) {
                        TS sum = TS(0);
                        for (int c2 = 0; c2 < ncl; ++c2) sum += __ldcg(zpa + size_t(c2) * mP + i);
                        zfull[i] = sum;
                    }
                    if (it + 1 == a.iters) break;
                }
                __syncthreads();
                if (tid == 0) {
                    __threadfence();
                    red_release_add_u32(a.bar, 1u);
                    const uint32_t target = uint32_t(2 * it + 1 + pass2) * gridDim.x + a.barrier_skew;
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
            }
            if (it + 1 < a.iters) load_z(tp + 1);
            continue;
        }
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

    // a wait that ran out in the last step is reported like any other
    if (__syncthreads_or(abort_flag)) goto abort_exit;
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

template <typename TQ, typename TS, int RG, bool DET>
void *kernel_for_rg(int cpl, int wpw, bool apc) {
#define APC_K(C, WP) (apc ? reinterpret_cast<void *>(&apc_iter_kernel<TQ, TS, C, WP, true, RG, DET>) \
                          : reinterpret_cast<void *>(&apc_iter_kernel<TQ, TS, C, WP, false, RG, DET>))
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
    } else if (wpw == 4) {
        // FP32 arithmetic only: FP64 z and z' for four workers would not fit
        // the register budget of a 384-thread CTA
        if constexpr (sizeof(TS) == 4) {
            switch (cpl) {
                case 2: return APC_K(2, 4);
                case 4: return APC_K(4, 4);
                case 8: return APC_K(8, 4);
            }
        }
    }
#undef APC_K
    return nullptr;
}

template <typename TQ, typename TS, bool DET>
void *kernel_for(int cpl, int wpw, bool apc, int rg) {
    return rg == 1 ? kernel_for_rg<TQ, TS, 1, DET>(cpl, wpw, apc)
                   : rg == 2 ? kernel_for_rg<TQ, TS, 2, DET>(cpl, wpw, apc) : nullptr;
}

}  // namespace iterk
}  // namespace apc
