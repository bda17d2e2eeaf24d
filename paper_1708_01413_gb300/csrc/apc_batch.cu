// Batched APC on the tensor cores: many independent systems A_s X_s = B_s,
// each with k <= 32 right-hand sides, uneven sizes n_s and uneven row blocks
// p_i, advanced together by one persistent kernel.
//
// Iteration.  Every machine keeps x_i (n x k) and the master keeps xbar.
// The machines' update is taken in the form of App. A, Eq. (e_i(t+1))
// written for x:
//     z_i = Q_i^T xbar - c_i,   x_i <- x_i + gamma (xbar - x_i - Q_i z_i),
// where c_i = R_i^{-T} b_i are the coordinates of every solution of
// A_i x = b_i in the basis Q_i (so Q_i^T x_i = c_i, and this equals
// Eq. (cons1)); then xbar <- (eta/m) sum_i x_i + (1 - eta) xbar, Eq. (cons2).
// z_i does not depend on x_i, so the second product is one GEMM per system,
// Y = Q^T xbar, over the packed basis Q = [Q_1 .. Q_m] (n x C).
//
// One iteration is two sweeps separated by grid barriers:
//   sweep A  unit = (system, tile of 256 rows); a consumer warp owns 32 rows.
//            The packed columns are walked in 64-column windows; for every
//            16-column chunk of machine i, W^T += Z_i^T Q_i^T (mma.sync
//            m16n8k16; A = z_i split into two BF16 planes, B = the basis via
//            ldmatrix), and after the machine's last chunk its update and the
//            running row sum; at the end of the unit the master's row update
//            (double-float) and xbar' split into three BF16 planes, stored in
//            the A-fragment order of sweep B.
//   sweep B  unit = (system, 512 columns); a consumer warp owns 64 columns,
//            all rows: Y^T = xbar'^T Q (A = the planes, B = the basis via
//            ldmatrix.trans), then Z = Y - c split into two planes, stored in
//            the A-fragment order of sweep A.
// The accumulator fragment of one sweep is, lane for lane, the operand
// fragment of the other, so no transposes are needed.
//
// Data movement.  The basis is stored tile-major and pre-swizzled: for each
// 256-row tile and 64-column window a contiguous [rows][64] BF16 block whose
// 16-byte chunks are XOR-permuted by (row & 7), the order ldmatrix reads
// without bank conflicts.  A machine's x_i tile is likewise one contiguous
// block ([k][rows + 8] FP32).  So every stage is one or a few 1-D TMA bulk
// copies, issued by a producer warp into a ring of 4 basis slots and 2 x_i
// slots; 8 consumer warps wait on the slots' mbarriers (bounded waits) and
// release them with per-warp arrivals, so no CTA-wide barrier sits in the
// streaming loop.  The CTAs claim units at run time from one counter per
// sweep, longest units first.
//
// Precision: Q_i is BF16 (rounded once from the FP64 QR); products accumulate
// in FP32 on the tensor cores; an operand split into planes keeps 16 (sweep
// A) or 24 (sweep B) significant bits of its FP32 value.  z_i tends to zero
// as the iteration converges, so its error is relative to the step; xbar does
// not, hence the third plane there.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <queue>
#include <string>
#include <vector>

#include "../../include/apc.h"
#include "../../include/apc_batch.h"
#include "apc_ctx.h"
#include "apc_internal.h"
#include "apc_ptx.cuh"

namespace apc {
void set_global_error_text(const char *msg);  // apc_api.cu
}

namespace {

using namespace apc;

constexpr int kConsumerWarps = 8;
constexpr int kThreads = 32 * (kConsumerWarps + 1);  // + one producer warp
constexpr int kTileRows = 256;   // rows of a sweep-A unit (32 per consumer warp)
constexpr int kWin = 64;         // basis columns per sweep-A window (one 128-byte row)
constexpr int kColsB = 512;      // columns of a sweep-B unit (64 per consumer warp)
constexpr int kRowsStageB = 32;  // rows per sweep-B stage
constexpr int kQSlots = 4, kXSlots = 2;
constexpr int kUQ = 4;           // depth of the queue of claimed units (producer -> consumers)
constexpr int kPlanesA = 2, kPlanesB = 3;
constexpr int kSlotQBytes = kTileRows * kWin * 2;  // 32 KB: 256 x 64 or 8 x (32 x 64) BF16
constexpr int kSlotZBytes = 8192;                  // operand planes of one stage
constexpr int kSlotBytes = kSlotQBytes + kSlotZBytes;
constexpr int kXPad = 8;                           // FP32 padding per right-hand-side row of an x_i tile
constexpr int kXSlotBytes = 32 * (kTileRows + kXPad) * 4;
constexpr int kBarOffset = kQSlots * kSlotBytes + kXSlots * kXSlotBytes;
// mbarriers: Q slots full/empty, x slots full/empty, unit queue full/empty; then the queue
constexpr size_t kSmemBytes = size_t(kBarOffset) + 2 * (kQSlots + kXSlots + kUQ) * sizeof(uint64_t) + kUQ * sizeof(int);

struct SysDesc {
    const __nv_bfloat16 *Q;  // tile-major, pre-swizzled (see q_block)
    float *X;                // tile-major x_i blocks (see x_block)
    float2 *Xb;              // [kp][npad]  master estimate, double-float
    uint4 *Xfrag;            // [npad/16][MT][kPlanesB][32]  xbar' operand planes
    uint2 *Zfrag;            // [Cq/8][MT][kPlanesA][32]     z operand planes
    const float4 *Cfrag;     // [Cq/8][MT][32]               c_i, FP32
    const int *coloff;       // [m + 1], multiples of 16
    float2 *Mb;              // [kp][npad]  heavy-ball momentum, double-float
    int npad, m, Cq, C;
    float g_hi, g_lo, em_hi, em_lo, e1_hi, e1_lo, im_hi, im_lo;
    float na_hi, na_lo, hb_hi, hb_lo;  // heavy ball: -alpha and beta
};

struct BatchArgs {
    const SysDesc *sys;
    const int2 *unitsA;  // (system, first row of the tile), longest first
    const int2 *unitsB;  // (system, first column), longest first
    int nA, nB;
    uint32_t *ctr;       // [3] claim counters, one per sweep, rotating (zero at launch)
    int64_t iters;
    int init;
    int hb;              // 1: distributed-preconditioned heavy ball instead of APC
    uint32_t barrier_skew;
    uint32_t *bar;
    int *err;
    uint64_t timeout_ns;
};

// rows of tile t
__host__ __device__ __forceinline__ int tile_rows(int npad, int t) { return min(kTileRows, npad - kTileRows * t); }
// first element of the basis block (tile t, window w): [tile_rows][64] BF16
__host__ __device__ __forceinline__ size_t q_block(int Cq, int npad, int t, int w) {
    return size_t(t) * kTileRows * Cq + size_t(w) * tile_rows(npad, t) * kWin;
}
// first element of machine i's x_i block in tile t: [kp][tile_rows + kXPad] FP32
__host__ __device__ __forceinline__ size_t x_block(int m, int kp, int npad, int t, int i) {
    return size_t(t) * m * kp * (kTileRows + kXPad) + size_t(i) * kp * (tile_rows(npad, t) + kXPad);
}

// ---- PTX wrappers ------------------------------------------------------------
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(addr));
}
__device__ __forceinline__ void lds64(uint32_t addr, uint32_t &x, uint32_t &y) {
    asm volatile("ld.shared.v2.u32 {%0,%1}, [%2];" : "=r"(x), "=r"(y) : "r"(addr));
}
__device__ __forceinline__ void lds128(uint32_t addr, uint32_t (&v)[4]) {
    asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]) : "r"(addr));
}
// D += A B, m16n8k16, BF16 operands, FP32 accumulators.  Not volatile: the
// compiler may interleave independent accumulations (a chain of MMAs on one
// accumulator would otherwise wait out the pipe latency at every step).
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// pull [src, src + bytes) into L2 ahead of its bulk copy into shared memory
__device__ __forceinline__ void prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// order this thread's generic-proxy global writes before later async-proxy
// (bulk copy) reads of them
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// ---- arithmetic ----------------------------------------------------------------
// bf16x2 with `lo` in the low half (the even k index) and `hi` in the high half
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}
// Split (x0, x1) into P BF16 planes: x = sum_p plane_p, each plane the nearest
// BF16 of what the previous planes left (every residual is exact in FP32).
template <int P>
__device__ __forceinline__ void split2(float x0, float x1, uint32_t (&w)[P]) {
#pragma unroll
    for (int p = 0; p < P; ++p) {
        w[p] = pack_bf16(x0, x1);
        x0 -= __uint_as_float(w[p] << 16);
        x1 -= __uint_as_float(w[p] & 0xffff0000u);
    }
}
// x + (g_hi + g_lo) v with the product g_hi v formed exactly (TwoProd) and the
// sum compensated (TwoSum): gamma enters with about 48 bits.
__device__ __forceinline__ float upd_exact(float x, float gh, float gl, float v) {
    const float p = gh * v;
    const float pe = fmaf(gh, v, -p);
    const float c = fmaf(gl, v, pe);
    const float s = x + p;
    const float bb = s - x;
    const float se = (x - (s - bb)) + (p - bb);
    return s + (c + se);
}
__device__ __forceinline__ float2 dfa(float2 a, float2 b) {
    const float s = a.x + b.x;
    const float bb = s - a.x;
    float e = (a.x - (s - bb)) + (b.x - bb);
    e += a.y + b.y;
    const float hi = s + e;
    return make_float2(hi, e - (hi - s));
}
__device__ __forceinline__ float2 dfm(float2 a, float2 b) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float hi = p + e;
    return make_float2(hi, e - (hi - p));
}

// ---- the ring ------------------------------------------------------------------
struct Ring {
    uint8_t *smem;
    uint64_t *full, *empty, *xfull, *xempty;  // [kQSlots], [kQSlots], [kXSlots], [kXSlots]
    int *abort_flag;
    uint64_t timeout_ns;

    __device__ uint8_t *qslot(int s) const { return smem + size_t(s) * kSlotBytes; }
    __device__ uint8_t *xslot(int s) const { return smem + size_t(kQSlots) * kSlotBytes + size_t(s) * kXSlotBytes; }
    // one non-blocking poll of a phase
    __device__ static bool test(uint64_t *bar, uint32_t parity) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
        return ok != 0;
    }
    // Bounded wait on a phase, spinning on test_wait (a suspended try_wait
    // wakes up late enough to cost a quarter of the sweep time); on time-out
    // raise the CTA's abort flag.
    __device__ bool wait(uint64_t *bar, uint32_t parity) const {
        if (*reinterpret_cast<volatile int *>(abort_flag)) return false;
        if (test(bar, parity)) return true;
        const uint64_t t0 = globaltimer_ns();
        while (globaltimer_ns() - t0 <= timeout_ns)
            if (test(bar, parity)) return true;
        atomicExch(abort_flag, 1);
        return false;
    }
    __device__ bool aborted() const { return *reinterpret_cast<volatile int *>(abort_flag) != 0; }
};

// Cursor over the stages of the ring, kept identically by the producer and by
// every consumer warp: stage q uses slot q % S with phase parity (q / S) & 1.
struct Cursor {
    uint32_t q = 0, x = 0;
};

// Producer: wait until slot of stage q is free (its previous use consumed).
__device__ __forceinline__ bool acquire_slot(const Ring &R, uint64_t *empty, int S, uint32_t q) {
    if (q < uint32_t(S)) return true;
    return R.wait(&empty[q % S], ((q / S) - 1) & 1);
}

// ---- sweep A ---------------------------------------------------------------------
template <int MT>
__device__ void sweep_a_producer(const Ring &R, Cursor &cur, const SysDesc &d, int row0, bool no_x,
                                 uint64_t policy) {
    constexpr int KP = 16 * MT;
    const int t = row0 / kTileRows, rows = tile_rows(d.npad, t);
    const int nwin = d.Cq / kWin;
    const uint32_t qbytes = uint32_t(rows) * kWin * 2, zbytes = 8 * MT * kPlanesA * 256;
    const uint32_t xbytes = uint32_t(KP) * (rows + kXPad) * 4;
    int pi = 0;  // next machine whose x_i tile is due
    // L2 prefetch runs kPrefetch windows / machines ahead of the shared-memory ring
    constexpr int kPrefetch = 4;
    for (int w = 0; w < min(kPrefetch, nwin); ++w) prefetch_l2(d.Q + q_block(d.Cq, d.npad, t, w), qbytes);
    if (!no_x)
        for (int j = 0; j < min(kPrefetch, d.m); ++j) prefetch_l2(d.X + x_block(d.m, KP, d.npad, t, j), xbytes);
    for (int w = 0; w < nwin; ++w) {
        const uint32_t s = cur.q % kQSlots;
        if (!acquire_slot(R, R.empty, kQSlots, cur.q)) return;
        mbar_arrive_expect_tx(&R.full[s], qbytes + zbytes);
        tma_load_1d(R.qslot(s), d.Q + q_block(d.Cq, d.npad, t, w), qbytes, &R.full[s], policy);
        tma_load_1d(R.qslot(s) + kSlotQBytes, d.Zfrag + size_t(8 * w) * MT * kPlanesA * 32, zbytes, &R.full[s],
                    policy);
        if (w + kPrefetch < nwin) prefetch_l2(d.Q + q_block(d.Cq, d.npad, t, w + kPrefetch), qbytes);
        ++cur.q;
        // x_i tiles of the machines whose last chunk lies in this window
        while (!no_x && pi < d.m && (__ldg(d.coloff + pi + 1) - 16) / kWin == w) {
            const uint32_t xs = cur.x % kXSlots;
            if (!acquire_slot(R, R.xempty, kXSlots, cur.x)) return;
            mbar_arrive_expect_tx(&R.xfull[xs], xbytes);
            tma_load_1d(R.xslot(xs), d.X + x_block(d.m, KP, d.npad, t, pi), xbytes, &R.xfull[xs], policy);
            if (pi + kPrefetch < d.m) prefetch_l2(d.X + x_block(d.m, KP, d.npad, t, pi + kPrefetch), xbytes);
            ++cur.x;
            ++pi;
        }
    }
}

template <int MT>
__device__ void sweep_a_consumer(const Ring &R, Cursor &cur, const SysDesc &d, int row0, bool init, bool hb,
                                 float gh, float gl) {
    constexpr int KP = 16 * MT;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tq = lane & 3;
    const int t = row0 / kTileRows, rows = tile_rows(d.npad, t);
    const bool wact = 32 * warp < rows;
    const int wrow = row0 + 32 * warp;  // first row of this warp
    const int nwin = d.Cq / kWin, nchunk = d.C / 16;
    const int xstride = rows + kXPad;   // floats per right-hand side in an x_i tile
    float xbh[MT][4][4], xbl[MT][4][4], S[MT][4][4], acc[MT][4][4];
    // accumulator element e of (mt, nt): right-hand side 16 mt + g + 8 (e >> 1),
    // row wrow + 8 nt + 2 tq + (e & 1)
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                S[mt][nt][e] = 0.0f;
                acc[mt][nt][e] = 0.0f;
                xbh[mt][nt][e] = 0.0f;
                xbl[mt][nt][e] = 0.0f;
            }
    if (wact && !init && !hb) {
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int rhs = 16 * mt + g + 8 * h;
                    const float4 v = __ldcg(reinterpret_cast<const float4 *>(
                        d.Xb + size_t(rhs) * d.npad + wrow + 8 * nt + 2 * tq));  // {hi, lo} of two rows
                    xbh[mt][nt][2 * h] = v.x;
                    xbl[mt][nt][2 * h] = v.y;
                    xbh[mt][nt][2 * h + 1] = v.z;
                    xbl[mt][nt][2 * h + 1] = v.w;
                }
    }
    int i = 0, iend = __ldg(d.coloff + 1) >> 4;  // machine of the current chunk, its end chunk
    for (int w = 0; w < nwin; ++w) {
        const uint32_t s = cur.q % kQSlots;
        if (!R.wait(&R.full[s], (cur.q / kQSlots) & 1)) return;
        const uint32_t sq = smem_u32(R.qslot(s)), sz = sq + kSlotQBytes;
#pragma unroll 1
        for (int kc = 0; kc < 4; ++kc) {
            const int c16 = 4 * w + kc;
            if (c16 >= nchunk) break;
            if (wact) {
                uint32_t a[MT][kPlanesA][4];
#pragma unroll
                for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                    for (int p = 0; p < kPlanesA; ++p) {
                        lds64(sz + (((2 * kc) * MT + mt) * kPlanesA + p) * 256 + lane * 8, a[mt][p][0], a[mt][p][1]);
                        lds64(sz + (((2 * kc + 1) * MT + mt) * kPlanesA + p) * 256 + lane * 8, a[mt][p][2],
                              a[mt][p][3]);
                    }
                uint32_t b[4][2];
#pragma unroll
                for (int ntp = 0; ntp < 4; ntp += 2) {
                    const int q = lane >> 3, r = lane & 7;
                    const int row = 32 * warp + 8 * (ntp + (q >> 1)) + r;
                    const int ch = 2 * kc + (q & 1);
                    ldsm_x4(sq + row * 128 + ((ch ^ (row & 7)) << 4), b[ntp][0], b[ntp][1], b[ntp + 1][0],
                            b[ntp + 1][1]);
                }
#pragma unroll
                for (int p = 0; p < kPlanesA; ++p)
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                        for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], a[mt][p], b[nt][0], b[nt][1]);
            }
            if (c16 + 1 == iend && hb) {
                // heavy ball: the accumulator keeps summing over the machines
                ++i;
                if (i < d.m) iend = __ldg(d.coloff + i + 1) >> 4;
            } else if (c16 + 1 == iend) {
                // machine i is complete: x_i <- x_i + gamma (xbar - x_i - w_i), row sums
                uint32_t xs = 0, sx = 0;
                if (!init) {
                    xs = cur.x % kXSlots;
                    if (!R.wait(&R.xfull[xs], (cur.x / kXSlots) & 1)) return;
                    sx = smem_u32(R.xslot(xs));
                }
                if (wact) {
                    float *xg = d.X + x_block(d.m, KP, d.npad, t, i);
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int rhs = 16 * mt + g + 8 * h;
                                const int rr = 32 * warp + 8 * nt + 2 * tq;  // row within the tile
                                uint32_t x0 = 0u, x1 = 0u;
                                if (!init) lds64(sx + (rhs * xstride + rr) * 4, x0, x1);
                                const float xo[2] = {__uint_as_float(x0), __uint_as_float(x1)};
                                float xn[2];
#pragma unroll
                                for (int u = 0; u < 2; ++u) {
                                    const int e = 2 * h + u;
                                    const float v = ((xbh[mt][nt][e] - xo[u]) + xbl[mt][nt][e]) - acc[mt][nt][e];
                                    xn[u] = upd_exact(xo[u], gh, gl, v);
                                    S[mt][nt][e] += xn[u];
                                    acc[mt][nt][e] = 0.0f;
                                }
                                __stcg(reinterpret_cast<float2 *>(xg + rhs * xstride + rr), make_float2(xn[0], xn[1]));
                            }
                }
                if (!init) {
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&R.xempty[xs]);
                    ++cur.x;
                }
                ++i;
                if (i < d.m) iend = __ldg(d.coloff + i + 1) >> 4;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&R.empty[s]);
        ++cur.q;
    }
    if (!wact) return;
    float xo[MT][4][4];
    if (hb) {
        // heavy ball on the preconditioned system (Sec. 4.3 update, Sec. 6):
        // the accumulator holds the gradient sum_i Q_i (Q_i^T x - c_i);
        // zeta <- beta zeta + gradient, x <- x - alpha zeta
        const float2 beta = make_float2(d.hb_hi, d.hb_lo), nalpha = make_float2(d.na_hi, d.na_lo);
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int rhs = 16 * mt + g + 8 * h;
                    const size_t off = size_t(rhs) * d.npad + wrow + 8 * nt + 2 * tq;
                    const float4 xv = __ldcg(reinterpret_cast<const float4 *>(d.Xb + off));
                    const float4 mv = __ldcg(reinterpret_cast<const float4 *>(d.Mb + off));
                    const float2 x2[2] = {make_float2(xv.x, xv.y), make_float2(xv.z, xv.w)};
                    const float2 m2[2] = {make_float2(mv.x, mv.y), make_float2(mv.z, mv.w)};
                    float2 xn[2], zn[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        zn[u] = dfa(dfm(beta, m2[u]), make_float2(acc[mt][nt][2 * h + u], 0.0f));
                        xn[u] = dfa(x2[u], dfm(nalpha, zn[u]));
                        xo[mt][nt][2 * h + u] = xn[u].x;
                    }
                    __stcg(reinterpret_cast<float4 *>(d.Mb + off), make_float4(zn[0].x, zn[0].y, zn[1].x, zn[1].y));
                    __stcg(reinterpret_cast<float4 *>(d.Xb + off), make_float4(xn[0].x, xn[0].y, xn[1].x, xn[1].y));
                }
    } else {
        // master: xbar' = (eta/m) S + (1 - eta) xbar   (initialisation: S / m)
        const float2 em = make_float2(init ? d.im_hi : d.em_hi, init ? d.im_lo : d.em_lo);
        const float2 e1 = make_float2(d.e1_hi, d.e1_lo);
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float2 xn[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const int e = 2 * h + u;
                        xn[u] = dfm(em, make_float2(S[mt][nt][e], 0.0f));
                        if (!init) xn[u] = dfa(xn[u], dfm(e1, make_float2(xbh[mt][nt][e], xbl[mt][nt][e])));
                        xo[mt][nt][e] = xn[u].x;
                    }
                    const int rhs = 16 * mt + g + 8 * h;
                    __stcg(reinterpret_cast<float4 *>(d.Xb + size_t(rhs) * d.npad + wrow + 8 * nt + 2 * tq),
                           make_float4(xn[0].x, xn[0].y, xn[1].x, xn[1].y));
                }
    }
    // xbar' operand planes of sweep B: in the 16-row chunk kc of this warp,
    // a0/a1 are n-tile 2kc (rhs g / g+8) and a2/a3 n-tile 2kc+1
#pragma unroll
    for (int kc = 0; kc < 2; ++kc)
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
            uint32_t w0[kPlanesB], w1[kPlanesB], w2[kPlanesB], w3[kPlanesB];
            split2<kPlanesB>(xo[mt][2 * kc][0], xo[mt][2 * kc][1], w0);
            split2<kPlanesB>(xo[mt][2 * kc][2], xo[mt][2 * kc][3], w1);
            split2<kPlanesB>(xo[mt][2 * kc + 1][0], xo[mt][2 * kc + 1][1], w2);
            split2<kPlanesB>(xo[mt][2 * kc + 1][2], xo[mt][2 * kc + 1][3], w3);
            const size_t kcg = size_t(wrow >> 4) + kc;
#pragma unroll
            for (int p = 0; p < kPlanesB; ++p)
                __stcg(d.Xfrag + ((kcg * MT + mt) * kPlanesB + p) * 32 + lane, make_uint4(w0[p], w1[p], w2[p], w3[p]));
        }
}

// ---- sweep B -----------------------------------------------------------------------
template <int MT>
__device__ void sweep_b_producer(const Ring &R, Cursor &cur, const SysDesc &d, int col0, uint64_t policy) {
    const int nwin = min(kColsB, d.Cq - col0) / kWin;
    const uint32_t xbytes = 2 * MT * kPlanesB * 512;
    for (int r0 = 0; r0 < d.npad; r0 += kRowsStageB) {
        const uint32_t s = cur.q % kQSlots;
        if (!acquire_slot(R, R.empty, kQSlots, cur.q)) return;
        const int t = r0 / kTileRows, rr = r0 % kTileRows;
        mbar_arrive_expect_tx(&R.full[s], uint32_t(nwin) * kRowsStageB * kWin * 2 + xbytes);
        for (int j = 0; j < nwin; ++j)
            tma_load_1d(R.qslot(s) + j * (kRowsStageB * kWin * 2),
                        d.Q + q_block(d.Cq, d.npad, t, col0 / kWin + j) + size_t(rr) * kWin,
                        kRowsStageB * kWin * 2, &R.full[s], policy);
        tma_load_1d(R.qslot(s) + kSlotQBytes, d.Xfrag + size_t(r0 >> 4) * MT * kPlanesB * 32, xbytes, &R.full[s],
                    policy);
        ++cur.q;
    }
}

template <int MT>
__device__ void store_z(const SysDesc &d, int col0, float (&acc)[MT][8][4], bool zero_y) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const size_t G = size_t(col0 >> 3) + 8 * warp + nt;
            const float4 c = __ldg(d.Cfrag + (G * MT + mt) * 32 + lane);
            const float y0 = zero_y ? 0.0f : acc[mt][nt][0], y1 = zero_y ? 0.0f : acc[mt][nt][1];
            const float y2 = zero_y ? 0.0f : acc[mt][nt][2], y3 = zero_y ? 0.0f : acc[mt][nt][3];
            uint32_t w01[kPlanesA], w23[kPlanesA];
            split2<kPlanesA>(y0 - c.x, y1 - c.y, w01);
            split2<kPlanesA>(y2 - c.z, y3 - c.w, w23);
#pragma unroll
            for (int p = 0; p < kPlanesA; ++p)
                __stcg(d.Zfrag + ((G * MT + mt) * kPlanesA + p) * 32 + lane, make_uint2(w01[p], w23[p]));
        }
}

template <int MT>
__device__ void sweep_b_consumer(const Ring &R, Cursor &cur, const SysDesc &d, int col0) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool wact = 64 * warp < min(kColsB, d.Cq - col0);
    float acc[MT][8][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.0f;
    for (int r0 = 0; r0 < d.npad; r0 += kRowsStageB) {
        const uint32_t s = cur.q % kQSlots;
        if (!R.wait(&R.full[s], (cur.q / kQSlots) & 1)) return;
        if (wact) {
            // this warp's 64 columns: a [32][64] block, chunks XOR-permuted by (row & 7)
            const uint32_t sq = smem_u32(R.qslot(s)) + warp * (kRowsStageB * kWin * 2);
            const uint32_t sx = smem_u32(R.qslot(s)) + kSlotQBytes;
#pragma unroll
            for (int kc = 0; kc < 2; ++kc) {
                uint32_t a[MT][kPlanesB][4];
#pragma unroll
                for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                    for (int p = 0; p < kPlanesB; ++p)
                        lds128(sx + ((kc * MT + mt) * kPlanesB + p) * 512 + lane * 16, a[mt][p]);
                uint32_t b[8][2];
#pragma unroll
                for (int ntp = 0; ntp < 8; ntp += 2) {
                    const int q = lane >> 3, r = lane & 7;
                    const int row = 16 * kc + 8 * (q & 1) + r;
                    const int ch = ntp + (q >> 1);
                    ldsm_x4_t(sq + row * 128 + ((ch ^ (row & 7)) << 4), b[ntp][0], b[ntp][1], b[ntp + 1][0],
                              b[ntp + 1][1]);
                }
#pragma unroll
                for (int p = 0; p < kPlanesB; ++p)
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                        for (int nt = 0; nt < 8; ++nt) mma_bf16(acc[mt][nt], a[mt][p], b[nt][0], b[nt][1]);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&R.empty[s]);
        ++cur.q;
    }
    if (wact) store_z<MT>(d, col0, acc, false);
}

// Bounded grid barrier over all CTAs: false when the wait ran out of time.
__device__ bool grid_barrier(uint32_t *bar, uint32_t target, uint64_t timeout_ns, int *abort_flag) {
    fence_proxy_async_global();  // this sweep's global writes are read by bulk copies in the next
    __syncthreads();
    if (threadIdx.x == 0 && !*reinterpret_cast<volatile int *>(abort_flag)) {
        __threadfence();
        red_release_add_u32(bar, 1u);
        if (ld_acquire_u32(bar) < target) {
            const uint64_t t0 = globaltimer_ns();
            while (ld_acquire_u32(bar) < target) {
                if (globaltimer_ns() - t0 > timeout_ns) {
                    atomicExch(abort_flag, 1);
                    break;
                }
            }
        }
        __threadfence();
    }
    return !__syncthreads_or(*reinterpret_cast<volatile int *>(abort_flag));
}

template <int MT>
__global__ void __launch_bounds__(kThreads, 1) apc_batch_kernel(const BatchArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int abort_flag;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kBarOffset);
    Ring R{smem, bars, bars + kQSlots, bars + 2 * kQSlots, bars + 2 * kQSlots + kXSlots, &abort_flag,
           a.timeout_ns};
    uint64_t *uqfull = bars + 2 * kQSlots + 2 * kXSlots;  // [kUQ] a claimed unit is in the queue
    uint64_t *uqempty = uqfull + kUQ;                     // [kUQ] every consumer warp has read it
    volatile int *uq = reinterpret_cast<volatile int *>(uqempty + kUQ);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool producer = warp == kConsumerWarps;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < kQSlots; ++s) {
            mbar_init(&R.full[s], 1);
            mbar_init(&R.empty[s], kConsumerWarps);
        }
        for (int s = 0; s < kXSlots; ++s) {
            mbar_init(&R.xfull[s], 1);
            mbar_init(&R.xempty[s], kConsumerWarps);
        }
        for (int s = 0; s < kUQ; ++s) {
            mbar_init(&uqfull[s], 1);
            mbar_init(&uqempty[s], kConsumerWarps);
        }
        fence_mbar_init_cluster();
    }
    __syncthreads();
    const uint64_t policy = policy_evict_first();
    Cursor cur;
    uint32_t uk = 0;  // units handed over so far (same count in the producer and every consumer warp)
    uint32_t episode = 0;
    bool ok = true;

    // One sweep.  The CTAs claim units from a global counter (the lists are
    // sorted longest first, so this is list scheduling with the longest units
    // first and the imbalance at the grid barrier is at most the shortest
    // units).  The producer claims ahead of the consumers and hands each unit
    // over through a small queue, so the ring keeps streaming across unit
    // boundaries; a claim past the end hands over -1 and ends the sweep.
    auto sweep = [&](bool is_a, uint32_t e, bool init, bool hb) {
        const int nunits = is_a ? a.nA : a.nB;
        const int2 *units = is_a ? a.unitsA : a.unitsB;
        // the counter of two sweeps ago: every claim on it ended before the last grid barrier
        if (blockIdx.x == 0 && threadIdx.x == 0) a.ctr[(e + 1) % 3] = 0u;
        if (producer) {
            if (lane != 0) return;
            for (;;) {
                const int s = int(uk % kUQ);
                int u = -1;
                if (uk < uint32_t(kUQ) || R.wait(&uqempty[s], ((uk / kUQ) - 1) & 1)) {
                    u = int(atomicAdd(&a.ctr[e % 3], 1u));
                    if (u >= nunits) u = -1;
                }
                uq[s] = u;
                mbar_arrive(&uqfull[s]);
                ++uk;
                if (u < 0) return;
                const int2 U = units[u];
                if (is_a) sweep_a_producer<MT>(R, cur, a.sys[U.x], U.y, init || hb, policy);
                else sweep_b_producer<MT>(R, cur, a.sys[U.x], U.y, policy);
            }
        } else {
            for (;;) {
                const int s = int(uk % kUQ);
                if (!R.wait(&uqfull[s], (uk / kUQ) & 1)) return;
                const int u = uq[s];
                __syncwarp();
                if (lane == 0) mbar_arrive(&uqempty[s]);
                ++uk;
                if (u < 0) return;
                const int2 U = units[u];
                const SysDesc &d = a.sys[U.x];
                if (is_a) sweep_a_consumer<MT>(R, cur, d, U.y, init, hb, init ? 1.0f : d.g_hi, init ? 0.0f : d.g_lo);
                else sweep_b_consumer<MT>(R, cur, d, U.y);
            }
        }
    };

    if (a.init) {
        // z_i(0) = -c_i, so that sweep A with gamma = 1 and x = xbar = 0 forms
        // the least-norm x_i(0) = Q_i c_i (Algorithm 1) and xbar(0) their mean
        if (!producer)
            for (int u = blockIdx.x; u < a.nB; u += gridDim.x) {
                const int2 U = a.unitsB[u];
                const SysDesc &d = a.sys[U.x];
                if (64 * warp < min(kColsB, d.Cq - U.y)) {
                    float acc[MT][8][4] = {};
                    store_z<MT>(d, U.y, acc, true);
                }
            }
        ++episode;
        ok = grid_barrier(a.bar, episode * gridDim.x + a.barrier_skew, a.timeout_ns, &abort_flag);
    }
    for (int64_t it = 0; ok && it < a.iters; ++it) {
        const bool init = a.init && it == 0;
        sweep(true, episode, init, a.hb && !init);
        ++episode;
        if (!(ok = grid_barrier(a.bar, episode * gridDim.x + a.barrier_skew, a.timeout_ns, &abort_flag))) break;
        sweep(false, episode, false, false);
        if (it + 1 < a.iters) {
            ++episode;
            ok = grid_barrier(a.bar, episode * gridDim.x + a.barrier_skew, a.timeout_ns, &abort_flag);
        }
    }
    // no bulk copy may still be writing this CTA's shared memory at exit: the
    // producer waits (bounded) for the last phase of every slot it filled
    __syncthreads();
    if (producer && lane == 0) {
        for (uint32_t q = cur.q > uint32_t(kQSlots) ? cur.q - kQSlots : 0; q < cur.q; ++q)
            (void)mbar_wait(&R.full[q % kQSlots], (q / kQSlots) & 1, a.timeout_ns);
        for (uint32_t x = cur.x > uint32_t(kXSlots) ? cur.x - kXSlots : 0; x < cur.x; ++x)
            (void)mbar_wait(&R.xfull[x % kXSlots], (x / kXSlots) & 1, a.timeout_ns);
    }
    __syncthreads();
    if (threadIdx.x == 0 && abort_flag) atomicCAS(a.err, 0, DEV_TIMEOUT_GRID);
}

// ---- set-up kernels -----------------------------------------------------------------
// Qs [n][m][P] (single-system layout) -> the tile-major, pre-swizzled packed
// basis: element (row j, packed column col) of block b = colblk[col / 16].
__global__ void repack_kernel(const __nv_bfloat16 *Qs, int64_t n, int m, int P, const int *colblk,
                              const int *coloff, const int32_t *pcount, int npad, int Cq, __nv_bfloat16 *Q) {
    const int64_t total = int64_t(npad) * Cq;
    for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int j = int(idx / Cq);
        const int col = int(idx - int64_t(j) * Cq);
        const int b = colblk[col >> 4];
        __nv_bfloat16 v = __float2bfloat16(0.0f);
        if (b >= 0 && j < n) {
            const int c = col - coloff[b];
            if (c < pcount[b]) v = Qs[(size_t(j) * m + b) * P + c];
        }
        const int t = j / kTileRows, r = j % kTileRows, w = col / kWin, cc = col % kWin;
        Q[q_block(Cq, npad, t, w) + size_t(r) * kWin + (((cc >> 3) ^ (r & 7)) << 3) + (cc & 7)] = v;
    }
}

// c_b = R2^T R1^T (d .* B_b) for one right-hand side (grid m x k), written as
// FP32 into the accumulator-fragment order of sweep B: column col and
// right-hand side rhs go to group col/8, m-tile rhs/16, lane 4 (rhs%8) +
// (col%8)/2, element 2 ((rhs%16)/8) + col%2.
__global__ void batch_coef_kernel(const double *B, int k, const int64_t *row_start, const int32_t *pcount,
                                  const double *dinv, const double *Rinv1, const double *Rinv2, int P,
                                  const int *coloff, int MT, float *Cfrag) {
    extern __shared__ double sh[];  // y[P], u[P]
    const int b = blockIdx.x, rhs = blockIdx.y;
    const int p = pcount[b];
    const int64_t r0 = row_start[b];
    const double *R1 = Rinv1 + size_t(b) * P * P, *R2 = Rinv2 + size_t(b) * P * P;
    double *y = sh, *u = sh + P;
    for (int r = threadIdx.x; r < P; r += blockDim.x) y[r] = r < p ? dinv[r0 + r] * B[(r0 + r) * k + rhs] : 0.0;
    __syncthreads();
    for (int c = threadIdx.x; c < P; c += blockDim.x) {
        double s = 0.0;
        for (int r = 0; r <= c && r < p; ++r) s = fma(R1[size_t(r) * P + c], y[r], s);
        u[c] = c < p ? s : 0.0;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < p; c += blockDim.x) {
        double s = 0.0;
        for (int r = 0; r <= c; ++r) s = fma(R2[size_t(r) * P + c], u[r], s);
        const int col = coloff[b] + c;
        const int G = col >> 3, w = col & 7;
        const int mt = rhs >> 4, rr = rhs & 15;
        Cfrag[((size_t(G) * MT + mt) * 32 + (rr & 7) * 4 + (w >> 1)) * 4 + (rr >> 3) * 2 + (w & 1)] = float(s);
    }
}

__global__ void xbar_out_kernel(const float2 *Xb, int64_t n, int64_t npad, int k, double *out, int64_t ldx) {
    const int64_t total = n * k;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t j = i / k;
        const int r = int(i - j * k);
        const float2 v = Xb[size_t(r) * npad + j];
        out[j * ldx + r] = double(v.x) + double(v.y);
    }
}

__global__ void x_out_kernel(const float *X, int64_t n, int npad, int m, int kp, int k, int worker, double *out,
                             int64_t ldx) {
    const int64_t total = n * k;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int j = int(i / k);
        const int r = int(i - int64_t(j) * k);
        const int t = j / kTileRows;
        const size_t off = x_block(m, kp, npad, t, worker) + size_t(r) * (tile_rows(npad, t) + kXPad) + j % kTileRows;
        out[int64_t(j) * ldx + r] = double(X[off]);
    }
}

void split_f64(double v, float &hi, float &lo) {
    hi = float(v);
    lo = float(v - double(hi));
}

}  // namespace

struct apc_batch {
    int device = 0, k = 1, kp = 16, MT = 1, nsys = 0, grid = 0;
    int units_a = 0, units_b = 0;
    std::vector<apc_ctx *> ctx;
    std::vector<SysDesc> desc;
    std::vector<int64_t> n;
    std::vector<int> m;
    std::vector<double *> B;  // FP64 right-hand sides (kept for apc_batch_reset)
    std::vector<void *> owned;
    SysDesc *d_desc = nullptr;
    int2 *d_unitsA = nullptr, *d_unitsB = nullptr;
    uint32_t *bar = nullptr;  // [4]: grid barrier counter, then the three claim counters
    int *err = nullptr;
    bool reset_done = false, params_set = false;
    int method = 0;  // 0: APC, 1: heavy ball (apc_batch_set_hb_params)
    int64_t q_bytes = 0, state_bytes = 0;
    double timeout_s = 2.0;
    uint32_t barrier_skew = 0;
    cudaGraphExec_t graph = nullptr;
    int64_t graph_iters = -1;
    int graph_method = -1;
    std::string last_error;
};

namespace {

int bfail(apc_batch *b, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (b) b->last_error = buf;
    apc::set_global_error_text(buf);
    return code;
}

#define BCK(b, call)                                                                                     \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) return bfail((b), APC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
int balloc(apc_batch *b, T **p, size_t bytes) {
    if (cudaMalloc(reinterpret_cast<void **>(p), bytes ? bytes : 16) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return bfail(b, APC_ERR_NOMEM, "cudaMalloc of %zu bytes failed", bytes);
    }
    b->owned.push_back(*p);
    return APC_OK;
}

const void *kernel_ptr(int MT) {
    return MT == 1 ? reinterpret_cast<const void *>(&apc_batch_kernel<1>)
                   : reinterpret_cast<const void *>(&apc_batch_kernel<2>);
}

// Units sorted longest first (by bytes streamed); the CTAs claim them in this
// order at run time.
std::vector<int2> longest_first(std::vector<std::pair<double, int2>> items) {
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<double, int2> &x, const std::pair<double, int2> &y) { return x.first > y.first; });
    std::vector<int2> units;
    units.reserve(items.size());
    for (const auto &it : items) units.push_back(it.second);
    return units;
}

int launch(apc_batch *b, int init, int64_t iters, cudaStream_t s) {
    BatchArgs a = {};
    a.sys = b->d_desc;
    a.unitsA = b->d_unitsA;
    a.unitsB = b->d_unitsB;
    a.nA = b->units_a;
    a.nB = b->units_b;
    a.ctr = b->bar + 1;
    a.iters = iters;
    a.init = init;
    a.hb = init ? 0 : b->method;
    a.barrier_skew = b->barrier_skew;
    a.bar = b->bar;
    a.err = b->err;
    a.timeout_ns = uint64_t(b->timeout_s * 1e9);
    BCK(b, cudaMemsetAsync(b->bar, 0, sizeof(uint32_t) * 4, s));
    if (b->MT == 1)
        apc_batch_kernel<1><<<b->grid, kThreads, kSmemBytes, s>>>(a);
    else
        apc_batch_kernel<2><<<b->grid, kThreads, kSmemBytes, s>>>(a);
    BCK(b, cudaGetLastError());
    return APC_OK;
}

int check_err(apc_batch *b, cudaStream_t s) {
    int h = 0;
    BCK(b, cudaMemcpyAsync(&h, b->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BCK(b, cudaStreamSynchronize(s));
    if (h) {
        BCK(b, cudaMemsetAsync(b->err, 0, sizeof(int), s));
        BCK(b, cudaStreamSynchronize(s));
        return bfail(b, APC_ERR_TIMEOUT, "a grid barrier wait ran out of time (%.3g s)", b->timeout_s);
    }
    return APC_OK;
}

int compute_coefficients(apc_batch *b, int sys, cudaStream_t s) {
    apc_ctx *c = b->ctx[sys];
    const SysDesc &d = b->desc[sys];
    float4 *Cf = const_cast<float4 *>(d.Cfrag);
    BCK(b, cudaMemsetAsync(Cf, 0, sizeof(float4) * size_t(d.Cq / 8) * b->MT * 32, s));
    const size_t sh = sizeof(double) * 2 * c->P;
    batch_coef_kernel<<<dim3(unsigned(c->m), unsigned(b->k)), 128, sh, s>>>(
        b->B[sys], b->k, c->d_rowstart, c->d_p, c->dinv, c->Rinv1, c->Rinv2, c->P, d.coloff, b->MT,
        reinterpret_cast<float *>(Cf));
    BCK(b, cudaGetLastError());
    return APC_OK;
}

}  // namespace

extern "C" {

int apc_batch_setup(apc_batch **out, int32_t nsys, const int64_t *n_host, const int32_t *m_host,
                    const int64_t *row_offsets_host, const double *const *A_dev_host,
                    const double *const *B_dev_host, int32_t k, const apc_options *opt, void *stream) {
    if (!out) return bfail(nullptr, APC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (nsys < 1 || !n_host || !m_host || !row_offsets_host || !A_dev_host || !B_dev_host)
        return bfail(nullptr, APC_ERR_INVALID_ARG, "apc_batch_setup: NULL argument or nsys < 1");
    if (k < 1 || k > 32) return bfail(nullptr, APC_ERR_UNSUPPORTED, "apc_batch_setup: k=%d outside 1..32", k);
    if (opt && opt->precision != APC_BF16)
        return bfail(nullptr, APC_ERR_UNSUPPORTED, "apc_batch_setup: the batched solver stores Q_i in BF16 only");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    apc_batch *b = new apc_batch();
    double *bcol = nullptr;
    auto bail = [&](int code) {
        if (bcol) cudaFree(bcol);
        const std::string msg = b->last_error;
        apc_batch_destroy(b);
        apc::set_global_error_text(msg.c_str());
        return code;
    };
    cudaGetDevice(&b->device);
    b->k = k;
    b->MT = k <= 16 ? 1 : 2;
    b->kp = 16 * b->MT;
    b->nsys = nsys;
    b->timeout_s = opt && opt->timeout_s > 0 ? opt->timeout_s : 2.0;
    const int MT = b->MT, kp = b->kp;
    const int64_t *offs = row_offsets_host;
    int rc = APC_OK;
    for (int sys = 0; sys < nsys; ++sys) {
        const int64_t n = n_host[sys];
        const int m = m_host[sys];
        if (n < 1 || m < 1 || n > (int64_t(1) << 24) || !A_dev_host[sys] || !B_dev_host[sys] || offs[0] != 0 ||
            offs[m] != n) {
            bfail(b, APC_ERR_INVALID_ARG, "system %d: bad size, pointer or offsets", sys);
            return bail(APC_ERR_INVALID_ARG);
        }
        // FP64 set-up of the single-system solver: row scaling and two passes
        // of Cholesky QR per block (Sec. 3.3); Q_i rounded to BF16 once
        if (bcol) cudaFree(bcol);
        bcol = nullptr;
        if (cudaMalloc(&bcol, sizeof(double) * n) != cudaSuccess) {
            cudaGetLastError();
            bcol = nullptr;
            bfail(b, APC_ERR_NOMEM, "cudaMalloc failed");
            return bail(APC_ERR_NOMEM);
        }
        if (cudaMemcpy2DAsync(bcol, sizeof(double), B_dev_host[sys], sizeof(double) * k, sizeof(double), n,
                              cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            bfail(b, APC_ERR_CUDA, "copy of B failed");
            return bail(APC_ERR_CUDA);
        }
        apc_options o = {APC_BF16, 0, 0, b->timeout_s};
        apc_ctx *c = nullptr;
        rc = apc_setup(&c, A_dev_host[sys], n, n, n, bcol, offs, m, &o, stream);
        if (rc != APC_OK) {
            bfail(b, rc, "system %d: %s", sys, apc_last_error(nullptr));
            return bail(rc);
        }
        b->ctx.push_back(c);
        b->n.push_back(n);
        b->m.push_back(m);
        // packed column layout: block i at coloff[i], width rounded up to 16
        // (one k16 chunk never spans two blocks)
        std::vector<int> co(m + 1, 0);
        for (int i = 0; i < m; ++i) co[i + 1] = co[i] + int((offs[i + 1] - offs[i] + 15) / 16 * 16);
        const int C = co[m];
        const int Cq = (C + kWin - 1) / kWin * kWin;
        const int64_t npad = (n + 31) / 32 * 32;
        const int ntiles = int((npad + kTileRows - 1) / kTileRows);
        std::vector<int> colblk(Cq / 16, -1);
        for (int i = 0; i < m; ++i)
            for (int g16 = co[i] / 16; g16 < co[i + 1] / 16; ++g16) colblk[g16] = i;
        SysDesc d = {};
        d.npad = int(npad);
        d.m = m;
        d.Cq = Cq;
        d.C = C;
        const size_t x_elems = x_block(m, kp, int(npad), ntiles, 0);
        int *d_co = nullptr, *d_cb = nullptr;
        __nv_bfloat16 *Q = nullptr;
        float4 *Cf = nullptr;
        double *Bc = nullptr;
        if ((rc = balloc(b, &d_co, sizeof(int) * (m + 1))) || (rc = balloc(b, &d_cb, sizeof(int) * (Cq / 16))) ||
            (rc = balloc(b, &Q, sizeof(__nv_bfloat16) * size_t(npad) * Cq)) ||
            (rc = balloc(b, &d.X, sizeof(float) * x_elems)) ||
            (rc = balloc(b, &d.Xb, sizeof(float2) * size_t(kp) * npad)) ||
            (rc = balloc(b, &d.Xfrag, sizeof(uint4) * size_t(npad / 16) * MT * kPlanesB * 32)) ||
            (rc = balloc(b, &d.Zfrag, sizeof(uint2) * size_t(Cq / 8) * MT * kPlanesA * 32)) ||
            (rc = balloc(b, &Cf, sizeof(float4) * size_t(Cq / 8) * MT * 32)) ||
            (rc = balloc(b, &d.Mb, sizeof(float2) * size_t(kp) * npad)) ||
            (rc = balloc(b, &Bc, sizeof(double) * size_t(n) * k)))
            return bail(rc);
        d.Q = Q;
        d.Cfrag = Cf;
        d.coloff = d_co;
        b->B.push_back(Bc);
        b->q_bytes += int64_t(sizeof(__nv_bfloat16)) * npad * Cq;
        b->state_bytes += int64_t(sizeof(float)) * m * kp * npad;  // unpadded iterate bytes
        cudaMemcpyAsync(d_co, co.data(), sizeof(int) * (m + 1), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_cb, colblk.data(), sizeof(int) * (Cq / 16), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(Bc, B_dev_host[sys], sizeof(double) * n * k, cudaMemcpyDeviceToDevice, s);
        cudaMemsetAsync(d.X, 0, sizeof(float) * x_elems, s);
        cudaMemsetAsync(d.Xb, 0, sizeof(float2) * size_t(kp) * npad, s);
        cudaMemsetAsync(d.Mb, 0, sizeof(float2) * size_t(kp) * npad, s);
        const unsigned grid = unsigned(std::min<int64_t>((npad * Cq + 255) / 256, 152 * 32));
        repack_kernel<<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(c->Q), n, m, c->P, d_cb, d_co, c->d_p,
                                           int(npad), Cq, Q);
        if (cudaGetLastError() != cudaSuccess) {
            bfail(b, APC_ERR_CUDA, "repack launch failed");
            return bail(APC_ERR_CUDA);
        }
        split_f64(1.0 / m, d.im_hi, d.im_lo);
        b->desc.push_back(d);
        if ((rc = compute_coefficients(b, sys, s)) != APC_OK) return bail(rc);
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            bfail(b, APC_ERR_CUDA, "set-up of system %d failed", sys);
            return bail(APC_ERR_CUDA);
        }
        // the single-system iteration buffers and the FP64 copy of A (kept
        // there for residuals) are not used by the batch
        cudaFree(c->A);
        c->A = nullptr;
        cudaFree(c->Q);
        c->Q = nullptr;
        cudaFree(c->xw);
        c->xw = nullptr;
        cudaFree(c->zbuf);
        c->zbuf = nullptr;
        offs += m + 1;
    }
    if (bcol) cudaFree(bcol);
    bcol = nullptr;
    if ((rc = balloc(b, &b->d_desc, sizeof(SysDesc) * nsys)) || (rc = balloc(b, &b->bar, sizeof(uint32_t) * 4)) ||
        (rc = balloc(b, &b->err, sizeof(int) * 4)))
        return bail(rc);
    if (cudaMemsetAsync(b->err, 0, sizeof(int) * 4, s) != cudaSuccess) {
        bfail(b, APC_ERR_CUDA, "memset failed");
        return bail(APC_ERR_CUDA);
    }
    // one CTA per SM, all resident at once (the grid barriers need that)
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    if (cudaFuncSetAttribute(kernel_ptr(MT), cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmemBytes)) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_ptr(MT), kThreads, kSmemBytes) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        bfail(b, APC_ERR_LAUNCH, "the batched kernel cannot be resident (%zu bytes of shared memory)", kSmemBytes);
        return bail(APC_ERR_LAUNCH);
    }
    b->grid = sms;
    // work lists: cost ~ bytes streamed per unit
    std::vector<std::pair<double, int2>> ia, ib;
    for (int sys = 0; sys < nsys; ++sys) {
        const SysDesc &d = b->desc[sys];
        for (int r0 = 0; r0 < d.npad; r0 += kTileRows) {
            const int rows = std::min(kTileRows, d.npad - r0);
            ia.push_back({double(rows) * (2.0 * d.Cq + 8.0 * d.m * kp + 64.0), make_int2(sys, r0)});
        }
        for (int c0 = 0; c0 < d.Cq; c0 += kColsB) {
            const int cols = std::min(kColsB, d.Cq - c0);
            ib.push_back({double(d.npad) * (2.0 * cols + 32.0), make_int2(sys, c0)});
        }
    }
    const std::vector<int2> ua = longest_first(ia), ub = longest_first(ib);
    b->units_a = int(ua.size());
    b->units_b = int(ub.size());
    if ((rc = balloc(b, &b->d_unitsA, sizeof(int2) * ua.size())) ||
        (rc = balloc(b, &b->d_unitsB, sizeof(int2) * ub.size())))
        return bail(rc);
    cudaMemcpyAsync(b->d_unitsA, ua.data(), sizeof(int2) * ua.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b->d_unitsB, ub.data(), sizeof(int2) * ub.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b->d_desc, b->desc.data(), sizeof(SysDesc) * nsys, cudaMemcpyHostToDevice, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        bfail(b, APC_ERR_CUDA, "set-up failed: %s", cudaGetErrorString(cudaGetLastError()));
        return bail(APC_ERR_CUDA);
    }
    *out = b;
    return APC_OK;
}

int apc_batch_set_params(apc_batch *b, const double *gamma_host, const double *eta_host) {
    if (!b || !gamma_host || !eta_host) return bfail(b, APC_ERR_INVALID_ARG, "NULL argument");
    for (int sys = 0; sys < b->nsys; ++sys) {
        const double g = gamma_host[sys], e = eta_host[sys];
        if (!(g > 0.0 && g < 2.0) || !std::isfinite(e))
            return bfail(b, APC_ERR_PARAMS, "system %d: gamma=%g must lie in (0, 2) and eta must be finite", sys, g);
    }
    for (int sys = 0; sys < b->nsys; ++sys) {
        SysDesc &d = b->desc[sys];
        const double g = gamma_host[sys], e = eta_host[sys];
        split_f64(g, d.g_hi, d.g_lo);
        split_f64(e / b->m[sys], d.em_hi, d.em_lo);
        split_f64(1.0 - e, d.e1_hi, d.e1_lo);
    }
    BCK(b, cudaMemcpy(b->d_desc, b->desc.data(), sizeof(SysDesc) * b->nsys, cudaMemcpyHostToDevice));
    b->params_set = true;
    b->method = 0;
    return APC_OK;
}

int apc_batch_set_hb_params(apc_batch *b, const double *alpha_host, const double *beta_host) {
    if (!b || !alpha_host || !beta_host) return bfail(b, APC_ERR_INVALID_ARG, "NULL argument");
    for (int sys = 0; sys < b->nsys; ++sys) {
        const double a = alpha_host[sys], be = beta_host[sys];
        if (!(a > 0.0) || !std::isfinite(a) || !(be >= 0.0 && be < 1.0))
            return bfail(b, APC_ERR_PARAMS, "system %d: need alpha > 0 and 0 <= beta < 1 (alpha=%g, beta=%g)", sys, a,
                         be);
    }
    for (int sys = 0; sys < b->nsys; ++sys) {
        SysDesc &d = b->desc[sys];
        split_f64(-alpha_host[sys], d.na_hi, d.na_lo);
        split_f64(beta_host[sys], d.hb_hi, d.hb_lo);
    }
    BCK(b, cudaMemcpy(b->d_desc, b->desc.data(), sizeof(SysDesc) * b->nsys, cudaMemcpyHostToDevice));
    b->params_set = true;
    b->method = 1;
    return APC_OK;
}

int apc_batch_reset(apc_batch *b, const double *const *B_dev_host, void *stream) {
    if (!b) return bfail(b, APC_ERR_INVALID_ARG, "NULL batch");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (B_dev_host) {
        for (int sys = 0; sys < b->nsys; ++sys)
            if (!B_dev_host[sys]) return bfail(b, APC_ERR_INVALID_ARG, "system %d: NULL right-hand side", sys);
        for (int sys = 0; sys < b->nsys; ++sys) {
            BCK(b, cudaMemcpyAsync(b->B[sys], B_dev_host[sys], sizeof(double) * b->n[sys] * b->k,
                                   cudaMemcpyDeviceToDevice, s));
            int rc = compute_coefficients(b, sys, s);
            if (rc != APC_OK) return rc;
        }
    }
    for (int sys = 0; sys < b->nsys; ++sys)
        BCK(b, cudaMemsetAsync(b->desc[sys].Mb, 0, sizeof(float2) * size_t(b->kp) * b->desc[sys].npad, s));
    int rc = launch(b, 1, 1, s);
    if (rc != APC_OK) return rc;
    if ((rc = check_err(b, s)) != APC_OK) return rc;
    b->reset_done = true;
    return APC_OK;
}

int apc_batch_iterate(apc_batch *b, int64_t iters, void *stream) {
    if (!b) return bfail(b, APC_ERR_INVALID_ARG, "NULL batch");
    if (iters < 0) return bfail(b, APC_ERR_INVALID_ARG, "iters < 0");
    if (iters == 0) return APC_OK;
    if (!b->params_set) return bfail(b, APC_ERR_PARAMS, "apc_batch_set_params must precede apc_batch_iterate");
    if (!b->reset_done) return bfail(b, APC_ERR_INVALID_ARG, "apc_batch_reset must precede apc_batch_iterate");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // one persistent launch (barrier reset + kernel), captured once per
    // iteration count and replayed as a CUDA graph
    if (!b->graph || b->graph_iters != iters || b->graph_method != b->method) {
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        cudaStream_t cs;
        BCK(b, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        const int rc = e == cudaSuccess ? launch(b, 0, iters, cs) : APC_ERR_CUDA;
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (rc == APC_OK && e2 == cudaSuccess) e2 = cudaGraphInstantiate(&b->graph, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess || rc != APC_OK || e2 != cudaSuccess) {
            cudaGetLastError();
            b->graph = nullptr;
            return bfail(b, APC_ERR_CUDA, "graph capture of the batched launch failed");
        }
        b->graph_iters = iters;
        b->graph_method = b->method;
    }
    BCK(b, cudaGraphLaunch(b->graph, s));
    return check_err(b, s);
}

int apc_batch_get_xbar(apc_batch *b, int32_t sys, double *X_dev, int64_t ldx, void *stream) {
    if (!b || !X_dev || sys < 0 || sys >= b->nsys || ldx < b->k) return bfail(b, APC_ERR_INVALID_ARG, "bad argument");
    const SysDesc &d = b->desc[sys];
    xbar_out_kernel<<<256, 256, 0, static_cast<cudaStream_t>(stream)>>>(d.Xb, b->n[sys], d.npad, b->k, X_dev, ldx);
    BCK(b, cudaGetLastError());
    return APC_OK;
}

int apc_batch_get_x(apc_batch *b, int32_t sys, int32_t worker, double *X_dev, int64_t ldx, void *stream) {
    if (!b || !X_dev || sys < 0 || sys >= b->nsys || worker < 0 || worker >= b->m[sys] || ldx < b->k)
        return bfail(b, APC_ERR_INVALID_ARG, "bad argument");
    const SysDesc &d = b->desc[sys];
    x_out_kernel<<<256, 256, 0, static_cast<cudaStream_t>(stream)>>>(d.X, b->n[sys], d.npad, d.m, b->kp, b->k, worker,
                                                                     X_dev, ldx);
    BCK(b, cudaGetLastError());
    return APC_OK;
}

int apc_batch_set_test_hooks(apc_batch *b, int32_t grid_barrier_skew, double timeout_s) {
    if (!b || grid_barrier_skew < 0 || !(timeout_s >= 0.0)) return bfail(b, APC_ERR_INVALID_ARG, "bad argument");
    b->barrier_skew = uint32_t(grid_barrier_skew);
    b->timeout_s = timeout_s > 0 ? timeout_s : 2.0;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return APC_OK;
}

int apc_batch_info(const apc_batch *b, int32_t *nsys, int32_t *k, int64_t *q_bytes, int64_t *state_bytes,
                   int32_t *grid, int32_t *units_a, int32_t *units_b) {
    if (!b) return APC_ERR_INVALID_ARG;
    if (nsys) *nsys = b->nsys;
    if (k) *k = b->k;
    if (q_bytes) *q_bytes = b->q_bytes;
    if (state_bytes) *state_bytes = b->state_bytes;
    if (grid) *grid = b->grid;
    if (units_a) *units_a = b->units_a;
    if (units_b) *units_b = b->units_b;
    return APC_OK;
}

const char *apc_batch_last_error(const apc_batch *b) { return b ? b->last_error.c_str() : apc_last_error(nullptr); }

void apc_batch_destroy(apc_batch *b) {
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (void *p : b->owned) cudaFree(p);
    for (apc_ctx *c : b->ctx) apc_destroy(c);
    delete b;
}

}  // extern "C"
