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
//   sweep A  unit = (system, 256 rows); warp = 32 rows.  For every machine i:
//            W^T = Z_i^T Q_i^T (mma.sync m16n8k16; A = Z_i^T split into two
//            BF16 planes, B = the BF16 basis from shared memory), then the
//            update of x_i and the running row sum; at the end the master's
//            row update (double-float) and xbar' split into three BF16
//            planes, stored in the A-fragment order of sweep B.
//   sweep B  unit = (system, 512 columns); warp = 64 columns, all rows.
//            Y^T = xbar'^T Q (A = xbar'^T in three planes, B = the basis via
//            ldmatrix.trans), then Z = Y - c split into two planes, stored in
//            the A-fragment order of sweep A.
// The accumulator fragment of one sweep is, lane for lane, the operand
// fragment of the other, so no transposes are needed.  The basis is staged
// through a 4-deep cp.async ring of XOR-swizzled tiles.  Units are assigned
// to CTAs on the host, longest first (LPT).
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

constexpr int kThreads = 256;
constexpr int kRowsA = 256;        // rows of a sweep-A unit (32 per warp)
constexpr int kColsStageA = 64;    // basis columns per sweep-A stage
constexpr int kColsB = 512;        // columns of a sweep-B unit (64 per warp)
constexpr int kRowsStageB = 32;    // rows per sweep-B stage
constexpr int kStages = 4;         // cp.async ring depth
constexpr int kPlanesA = 2, kPlanesB = 3;
constexpr int kStageQBytes = 32768;  // 256 x 64 or 32 x 512 BF16
constexpr int kStageBytes = 40960;   // basis tile + operand planes
constexpr size_t kSmemBytes = size_t(kStages) * kStageBytes;

struct SysDesc {
    const __nv_bfloat16 *Q;  // [npad][Cq], zero outside the blocks
    float *X;                // [m][kp][npad]   machines' iterates, transposed
    float2 *Xb;              // [kp][npad]      master estimate, double-float
    uint4 *Xfrag;            // [npad/16][MT][kPlanesB][32]  xbar' operand planes
    uint2 *Zfrag;            // [Cq/8][MT][kPlanesA][32]     z operand planes
    const float4 *Cfrag;     // [Cq/8][MT][32]               c_i, FP32
    const int *coloff;       // [m + 1], multiples of 8
    int npad, m, Cq, pad;
    float g_hi, g_lo, em_hi, em_lo, e1_hi, e1_lo, im_hi, im_lo;
};

struct BatchArgs {
    const SysDesc *sys;
    const int2 *unitsA;  // (system, first row)
    const int *offA;     // [grid + 1]
    const int2 *unitsB;  // (system, first column)
    const int *offB;     // [grid + 1]
    int64_t iters;
    int init;
    uint32_t barrier_skew;
    uint32_t *bar;
    int *err;
    uint64_t timeout_ns;
};

// ---- PTX wrappers ------------------------------------------------------------
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
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
// D += A B, m16n8k16, BF16 operands, FP32 accumulators
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
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

// Bounded grid barrier: false when the wait ran out of time.
__device__ bool grid_barrier(uint32_t *bar, uint32_t target, uint64_t timeout_ns, int *abort_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        red_release_add_u32(bar, 1u);
        if (ld_acquire_u32(bar) < target) {
            const uint64_t t0 = globaltimer_ns();
            while (ld_acquire_u32(bar) < target) {
                if (globaltimer_ns() - t0 > timeout_ns) {
                    *abort_flag = 1;
                    break;
                }
            }
        }
        __threadfence();
    }
    return !__syncthreads_or(*abort_flag);
}

// ---- sweep A: machines' first product, update, master ----------------------------
template <int MT>
struct SweepA {
    static constexpr int KP = 16 * MT;
    const SysDesc d;
    const int row0, rows, tid, warp, lane, g, t;
    const bool wact;
    const uint32_t sbase;
    int pi, ps, pc0, pw16;  // producer cursor: worker, sub-stage, its columns

    __device__ SweepA(const SysDesc &d_, int row0_, uint32_t sbase_)
        : d(d_), row0(row0_), rows(min(kRowsA, d_.npad - row0_)), tid(threadIdx.x), warp(threadIdx.x >> 5),
          lane(threadIdx.x & 31), g((threadIdx.x & 31) >> 2), t(threadIdx.x & 3),
          wact(32 * int(threadIdx.x >> 5) < min(kRowsA, d_.npad - row0_)), sbase(sbase_), pi(0), ps(0) {
        load_worker(0, pc0, pw16);
    }

    // first column and width (rounded up to 16) of worker i
    __device__ void load_worker(int i, int &c0, int &w16) const {
        if (i < d.m) {
            c0 = __ldg(d.coloff + i);
            w16 = (__ldg(d.coloff + i + 1) - c0 + 15) & ~15;
        } else {
            c0 = 0;
            w16 = 0;
        }
    }

    // Issue the next stage into ring slot `slot` (an empty group past the end).
    __device__ void issue(int slot) {
        if (pi < d.m) {
            const int cs = pc0 + kColsStageA * ps;
            const int nch = min(kColsStageA, pw16 - kColsStageA * ps) >> 3;  // 16-byte chunks per row
            const uint32_t sq = sbase + slot * kStageBytes;
            const __nv_bfloat16 *src = d.Q + size_t(row0) * d.Cq + cs;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int idx = tid + kThreads * k;
                const int r = idx >> 3, ch = idx & 7;
                if (ch < nch && r < rows)
                    cp_async16(sq + r * 128 + ((ch ^ (r & 7)) << 4), src + size_t(r) * d.Cq + 8 * ch);
            }
            const int zchunks = nch * MT * kPlanesA * 16;  // 16-byte pieces of the z planes
            const uint8_t *zsrc = reinterpret_cast<const uint8_t *>(d.Zfrag + size_t(cs >> 3) * MT * kPlanesA * 32);
            for (int idx = tid; idx < zchunks; idx += kThreads)
                cp_async16(sq + kStageQBytes + idx * 16, zsrc + size_t(idx) * 16);
            if (++ps * kColsStageA >= pw16) {
                ps = 0;
                ++pi;
                load_worker(pi, pc0, pw16);
            }
        }
        cp_async_commit();
    }

    __device__ void run(bool init, float gh, float gl) {
        float xbh[MT][4][4], xbl[MT][4][4], S[MT][4][4], acc[MT][4][4], xr[MT][4][4];
        const int wrow = row0 + 32 * warp;
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
                    xr[mt][nt][e] = 0.0f;
                }
        // accumulator element e of (mt, nt): rhs 16 mt + g + 8 (e >> 1),
        // row wrow + 8 nt + 2 t + (e & 1)
        if (wact && !init) {
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int rhs = 16 * mt + g + 8 * h;
                        const float4 v = __ldcg(reinterpret_cast<const float4 *>(
                            d.Xb + size_t(rhs) * d.npad + wrow + 8 * nt + 2 * t));  // {hi, lo} of two rows
                        xbh[mt][nt][2 * h] = v.x;
                        xbl[mt][nt][2 * h] = v.y;
                        xbh[mt][nt][2 * h + 1] = v.z;
                        xbl[mt][nt][2 * h + 1] = v.w;
                    }
        }
        for (int s = 0; s < kStages - 1; ++s) issue(s);
        int ci = 0, cs = 0, cc0, cw16;
        load_worker(0, cc0, cw16);
        int slot = 0;
        while (ci < d.m) {
            cp_async_wait<kStages - 2>();
            __syncthreads();
            issue((slot + kStages - 1) % kStages);
            const uint32_t sq = sbase + slot * kStageBytes, sz = sq + kStageQBytes;
            const int width = min(kColsStageA, cw16 - kColsStageA * cs);
            const bool first = cs == 0, last = (cs + 1) * kColsStageA >= cw16;
            // an odd number of 8-column groups: the second half of the last
            // 16-column chunk holds the next block's columns and gets zero weight
            const bool odd_tail = last && (((__ldg(d.coloff + ci + 1) - cc0) >> 3) & 1);
            if (wact) {
                if (first && !init) {
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                const int rhs = 16 * mt + g + 8 * h;
                                const float2 v = __ldcg(reinterpret_cast<const float2 *>(
                                    d.X + (size_t(ci) * KP + rhs) * d.npad + wrow + 8 * nt + 2 * t));
                                xr[mt][nt][2 * h] = v.x;
                                xr[mt][nt][2 * h + 1] = v.y;
                            }
                }
                const int nkc = width >> 4;
                for (int kc = 0; kc < nkc; ++kc) {
                    uint32_t a[MT][kPlanesA][4];
                    const bool zero_hi = odd_tail && kc == nkc - 1;
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                        for (int p = 0; p < kPlanesA; ++p) {
                            lds64(sz + (((2 * kc) * MT + mt) * kPlanesA + p) * 256 + lane * 8, a[mt][p][0],
                                  a[mt][p][1]);
                            if (zero_hi) {
                                a[mt][p][2] = 0u;
                                a[mt][p][3] = 0u;
                            } else {
                                lds64(sz + (((2 * kc + 1) * MT + mt) * kPlanesA + p) * 256 + lane * 8, a[mt][p][2],
                                      a[mt][p][3]);
                            }
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
                    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                            for (int p = 0; p < kPlanesA; ++p) mma_bf16(acc[mt][nt], a[mt][p], b[nt][0], b[nt][1]);
                }
                if (last) {
                    // x_i <- x_i + gamma (xbar - x_i - w_i); row sums over machines
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                float xn[2];
#pragma unroll
                                for (int u = 0; u < 2; ++u) {
                                    const int e = 2 * h + u;
                                    const float x = xr[mt][nt][e];
                                    const float v = ((xbh[mt][nt][e] - x) + xbl[mt][nt][e]) - acc[mt][nt][e];
                                    xn[u] = upd_exact(x, gh, gl, v);
                                    S[mt][nt][e] += xn[u];
                                    acc[mt][nt][e] = 0.0f;
                                }
                                const int rhs = 16 * mt + g + 8 * h;
                                __stcg(reinterpret_cast<float2 *>(d.X + (size_t(ci) * KP + rhs) * d.npad + wrow +
                                                                  8 * nt + 2 * t),
                                       make_float2(xn[0], xn[1]));
                            }
                }
            }
            slot = (slot + 1) % kStages;
            if (last) {
                cs = 0;
                ++ci;
                load_worker(ci, cc0, cw16);
            } else {
                ++cs;
            }
        }
        cp_async_wait<0>();
        __syncthreads();
        if (!wact) return;
        // master: xbar' = (eta/m) S + (1 - eta) xbar   (initialisation: S / m)
        const float2 em = make_float2(init ? d.im_hi : d.em_hi, init ? d.im_lo : d.em_lo);
        const float2 e1 = make_float2(d.e1_hi, d.e1_lo);
        float xo[MT][4][4];
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
                    __stcg(reinterpret_cast<float4 *>(d.Xb + size_t(rhs) * d.npad + wrow + 8 * nt + 2 * t),
                           make_float4(xn[0].x, xn[0].y, xn[1].x, xn[1].y));
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
                    __stcg(d.Xfrag + ((kcg * MT + mt) * kPlanesB + p) * 32 + lane,
                           make_uint4(w0[p], w1[p], w2[p], w3[p]));
            }
    }
};

// ---- sweep B: second product Y^T = xbar'^T Q, then Z = Y - c -----------------------
template <int MT>
struct SweepB {
    const SysDesc d;
    const int col0, ncols, tid, warp, lane;
    const bool wact;
    const uint32_t sbase;
    int pr;  // first row of the next stage to issue

    __device__ SweepB(const SysDesc &d_, int col0_, uint32_t sbase_)
        : d(d_), col0(col0_), ncols(min(kColsB, d_.Cq - col0_)), tid(threadIdx.x), warp(threadIdx.x >> 5),
          lane(threadIdx.x & 31), wact(64 * int(threadIdx.x >> 5) < min(kColsB, d_.Cq - col0_)), sbase(sbase_),
          pr(0) {}

    __device__ void issue(int slot) {
        if (pr < d.npad) {
            const uint32_t sq = sbase + slot * kStageBytes;
            const int nch = ncols >> 3;
            const __nv_bfloat16 *src = d.Q + size_t(pr) * d.Cq + col0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int idx = tid + kThreads * k;
                const int r = idx >> 6, ch = idx & 63;
                if (ch < nch) cp_async16(sq + r * 1024 + ((ch ^ (r & 7)) << 4), src + size_t(r) * d.Cq + 8 * ch);
            }
            const int xchunks = 2 * MT * kPlanesB * 32;  // two 16-row chunks of 16-byte lane vectors
            const uint8_t *xsrc = reinterpret_cast<const uint8_t *>(d.Xfrag + size_t(pr >> 4) * MT * kPlanesB * 32);
            for (int idx = tid; idx < xchunks; idx += kThreads)
                cp_async16(sq + kStageQBytes + idx * 16, xsrc + size_t(idx) * 16);
            pr += kRowsStageB;
        }
        cp_async_commit();
    }

    __device__ void run() {
        float acc[MT][8][4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
            for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.0f;
        for (int s = 0; s < kStages - 1; ++s) issue(s);
        int slot = 0;
        for (int r0 = 0; r0 < d.npad; r0 += kRowsStageB) {
            cp_async_wait<kStages - 2>();
            __syncthreads();
            issue((slot + kStages - 1) % kStages);
            if (wact) {
                const uint32_t sq = sbase + slot * kStageBytes, sx = sq + kStageQBytes;
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
                        const int ch = 8 * warp + ntp + (q >> 1);
                        ldsm_x4_t(sq + row * 1024 + ((ch ^ (row & 7)) << 4), b[ntp][0], b[ntp][1], b[ntp + 1][0],
                                  b[ntp + 1][1]);
                    }
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
                            for (int p = 0; p < kPlanesB; ++p) mma_bf16(acc[mt][nt], a[mt][p], b[nt][0], b[nt][1]);
                }
            }
            slot = (slot + 1) % kStages;
        }
        cp_async_wait<0>();
        __syncthreads();
        if (wact) store_z(acc, false);
    }

    // Z = Y - c into the sweep-A operand planes (zero_y: the initial z = -c)
    __device__ void store_z(float (&acc)[MT][8][4], bool zero_y) const {
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
};

template <int MT>
__global__ void __launch_bounds__(kThreads, 1) apc_batch_kernel(const BatchArgs a) {
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ int abort_flag;
    if (threadIdx.x == 0) abort_flag = 0;
    __syncthreads();
    const uint32_t sbase = smem_u32(smem);
    uint32_t episode = 0;
    bool ok = true;
    if (a.init) {
        // z_i(0) = -c_i, so that sweep A with gamma = 1 and x = xbar = 0 forms
        // the least-norm x_i(0) = Q_i c_i (Algorithm 1) and xbar(0) = their mean
        for (int u = a.offB[blockIdx.x]; u < a.offB[blockIdx.x + 1]; ++u) {
            const int2 U = a.unitsB[u];
            SweepB<MT> sb(a.sys[U.x], U.y, sbase);
            if (sb.wact) {
                float acc[MT][8][4] = {};
                sb.store_z(acc, true);
            }
        }
        ++episode;
        ok = grid_barrier(a.bar, episode * gridDim.x + a.barrier_skew, a.timeout_ns, &abort_flag);
    }
    for (int64_t it = 0; ok && it < a.iters; ++it) {
        const bool init = a.init && it == 0;
        for (int u = a.offA[blockIdx.x]; u < a.offA[blockIdx.x + 1]; ++u) {
            const int2 U = a.unitsA[u];
            SweepA<MT> sa(a.sys[U.x], U.y, sbase);
            sa.run(init, init ? 1.0f : sa.d.g_hi, init ? 0.0f : sa.d.g_lo);
        }
        ++episode;
        if (!(ok = grid_barrier(a.bar, episode * gridDim.x + a.barrier_skew, a.timeout_ns, &abort_flag))) break;
        for (int u = a.offB[blockIdx.x]; u < a.offB[blockIdx.x + 1]; ++u) {
            const int2 U = a.unitsB[u];
            SweepB<MT> sb(a.sys[U.x], U.y, sbase);
            sb.run();
        }
        if (it + 1 < a.iters) {
            ++episode;
            ok = grid_barrier(a.bar, episode * gridDim.x + a.barrier_skew, a.timeout_ns, &abort_flag);
        }
    }
    if (threadIdx.x == 0 && abort_flag) atomicCAS(a.err, 0, DEV_TIMEOUT_GRID);
}

// ---- set-up kernels -----------------------------------------------------------------
// Qs [n][m][P] (single-system layout) -> Q [npad][Cq], block b at coloff[b]
__global__ void repack_kernel(const __nv_bfloat16 *Qs, int64_t n, int m, int P, const int *colblk,
                              const int *coloff, const int32_t *pcount, int64_t npad, int Cq, __nv_bfloat16 *Q) {
    const int64_t total = npad * Cq;
    for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t j = idx / Cq;
        const int cc = int(idx - j * Cq);
        const int b = colblk[cc >> 3];
        __nv_bfloat16 v = __float2bfloat16(0.0f);
        if (b >= 0 && j < n) {
            const int c = cc - coloff[b];
            if (c < pcount[b]) v = Qs[(size_t(j) * m + b) * P + c];
        }
        Q[idx] = v;
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

__global__ void x_out_kernel(const float *X, int64_t n, int64_t npad, int kp, int k, int worker, double *out,
                             int64_t ldx) {
    const int64_t total = n * k;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t j = i / k;
        const int r = int(i - j * k);
        out[j * ldx + r] = double(X[(size_t(worker) * kp + r) * npad + j]);
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
    int *d_offA = nullptr, *d_offB = nullptr;
    uint32_t *bar = nullptr;
    int *err = nullptr;
    bool reset_done = false, params_set = false;
    int64_t q_bytes = 0, state_bytes = 0;
    double timeout_s = 2.0;
    uint32_t barrier_skew = 0;
    cudaGraphExec_t graph = nullptr;
    int64_t graph_iters = -1;
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

// Longest-processing-time assignment of units to CTAs, as CSR lists.
void lpt(std::vector<std::pair<double, int2>> items, int bins, std::vector<int2> &units, std::vector<int> &off) {
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<double, int2> &x, const std::pair<double, int2> &y) { return x.first > y.first; });
    std::vector<std::vector<int2>> per(bins);
    using P = std::pair<double, int>;
    std::priority_queue<P, std::vector<P>, std::greater<P>> heap;
    for (int i = 0; i < bins; ++i) heap.push({0.0, i});
    for (const auto &it : items) {
        P top = heap.top();
        heap.pop();
        per[top.second].push_back(it.second);
        heap.push({top.first + it.first, top.second});
    }
    units.clear();
    off.assign(1, 0);
    for (auto &v : per) {
        std::sort(v.begin(), v.end(), [](int2 x, int2 y) { return x.x != y.x ? x.x < y.x : x.y < y.y; });
        units.insert(units.end(), v.begin(), v.end());
        off.push_back(int(units.size()));
    }
}

int launch(apc_batch *b, int init, int64_t iters, cudaStream_t s) {
    BatchArgs a = {};
    a.sys = b->d_desc;
    a.unitsA = b->d_unitsA;
    a.offA = b->d_offA;
    a.unitsB = b->d_unitsB;
    a.offB = b->d_offB;
    a.iters = iters;
    a.init = init;
    a.barrier_skew = b->barrier_skew;
    a.bar = b->bar;
    a.err = b->err;
    a.timeout_ns = uint64_t(b->timeout_s * 1e9);
    BCK(b, cudaMemsetAsync(b->bar, 0, sizeof(uint32_t), s));
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
        // packed column layout: block i at coloff[i], width rounded up to 8
        std::vector<int> co(m + 1, 0);
        for (int i = 0; i < m; ++i) co[i + 1] = co[i] + int((offs[i + 1] - offs[i] + 7) / 8 * 8);
        const int C = co[m];
        const int Cq = (C + 8 + 63) / 64 * 64;
        const int64_t npad = (n + 31) / 32 * 32;
        std::vector<int> colblk(Cq / 8, -1);
        for (int i = 0; i < m; ++i)
            for (int g8 = co[i] / 8; g8 < co[i + 1] / 8; ++g8) colblk[g8] = i;
        SysDesc d = {};
        d.npad = int(npad);
        d.m = m;
        d.Cq = Cq;
        int *d_co = nullptr, *d_cb = nullptr;
        __nv_bfloat16 *Q = nullptr;
        float4 *Cf = nullptr;
        double *Bc = nullptr;
        if ((rc = balloc(b, &d_co, sizeof(int) * (m + 1))) || (rc = balloc(b, &d_cb, sizeof(int) * (Cq / 8))) ||
            (rc = balloc(b, &Q, sizeof(__nv_bfloat16) * size_t(npad) * Cq)) ||
            (rc = balloc(b, &d.X, sizeof(float) * size_t(m) * kp * npad)) ||
            (rc = balloc(b, &d.Xb, sizeof(float2) * size_t(kp) * npad)) ||
            (rc = balloc(b, &d.Xfrag, sizeof(uint4) * size_t(npad / 16) * MT * kPlanesB * 32)) ||
            (rc = balloc(b, &d.Zfrag, sizeof(uint2) * size_t(Cq / 8) * MT * kPlanesA * 32)) ||
            (rc = balloc(b, &Cf, sizeof(float4) * size_t(Cq / 8) * MT * 32)) ||
            (rc = balloc(b, &Bc, sizeof(double) * size_t(n) * k)))
            return bail(rc);
        d.Q = Q;
        d.Cfrag = Cf;
        d.coloff = d_co;
        b->B.push_back(Bc);
        b->q_bytes += int64_t(sizeof(__nv_bfloat16)) * npad * Cq;
        b->state_bytes += int64_t(sizeof(float)) * m * kp * npad;
        cudaMemcpyAsync(d_co, co.data(), sizeof(int) * (m + 1), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_cb, colblk.data(), sizeof(int) * (Cq / 8), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(Bc, B_dev_host[sys], sizeof(double) * n * k, cudaMemcpyDeviceToDevice, s);
        cudaMemsetAsync(d.X, 0, sizeof(float) * size_t(m) * kp * npad, s);
        cudaMemsetAsync(d.Xb, 0, sizeof(float2) * size_t(kp) * npad, s);
        const unsigned grid = unsigned(std::min<int64_t>((npad * Cq + 255) / 256, 152 * 32));
        repack_kernel<<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(c->Q), n, m, c->P, d_cb, d_co, c->d_p,
                                           npad, Cq, Q);
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
        // the single-system iteration buffers are not used by the batch
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
        for (int r0 = 0; r0 < d.npad; r0 += kRowsA) {
            const int rows = std::min(kRowsA, d.npad - r0);
            ia.push_back({double(rows) * (2.0 * d.Cq + 8.0 * d.m * kp + 64.0), make_int2(sys, r0)});
        }
        for (int c0 = 0; c0 < d.Cq; c0 += kColsB) {
            const int cols = std::min(kColsB, d.Cq - c0);
            ib.push_back({double(d.npad) * (2.0 * cols + 32.0), make_int2(sys, c0)});
        }
    }
    std::vector<int2> ua, ub;
    std::vector<int> oa, ob;
    lpt(ia, b->grid, ua, oa);
    lpt(ib, b->grid, ub, ob);
    b->units_a = int(ua.size());
    b->units_b = int(ub.size());
    if ((rc = balloc(b, &b->d_unitsA, sizeof(int2) * ua.size())) ||
        (rc = balloc(b, &b->d_offA, sizeof(int) * oa.size())) ||
        (rc = balloc(b, &b->d_unitsB, sizeof(int2) * ub.size())) ||
        (rc = balloc(b, &b->d_offB, sizeof(int) * ob.size())))
        return bail(rc);
    cudaMemcpyAsync(b->d_unitsA, ua.data(), sizeof(int2) * ua.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b->d_offA, oa.data(), sizeof(int) * oa.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b->d_unitsB, ub.data(), sizeof(int2) * ub.size(), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b->d_offB, ob.data(), sizeof(int) * ob.size(), cudaMemcpyHostToDevice, s);
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
    if (!b->graph || b->graph_iters != iters) {
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
    x_out_kernel<<<256, 256, 0, static_cast<cudaStream_t>(stream)>>>(d.X, b->n[sys], d.npad, b->kp, b->k, worker,
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
