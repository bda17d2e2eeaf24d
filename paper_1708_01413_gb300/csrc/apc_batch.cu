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
// One iteration is two sweeps, both on the 5th generation tensor cores
// (tcgen05.mma, BF16 operands in shared memory, FP32 accumulators in tensor
// memory), issued by one thread of a tensor-core warp:
//   sweep A  unit = (system, tile of 256 rows).  The packed columns are walked
//            in 64-column windows; for every 16-column chunk of machine i,
//            D += Q[rows, chunk] Z[chunk, 2 planes x k] (M = 128 rows per
//            instruction, N = 2k; z_i split into two BF16 planes), into one
//            of two accumulator buffers.  After the machine's last chunk the
//            consumers (thread = row) read its w_i = Q_i z_i from tensor
//            memory, update x_i and the running row sum while the tensor
//            cores go on with the next machine in the other buffer; at the end
//            of the unit the master's row update (double-float) and xbar'
//            split into three BF16 planes.
//   sweep B  unit = (system, 512 columns): D += Q[rows, cols]^T xbar'[rows,
//            3 planes x k] over all rows (M = 128 columns per instruction, the
//            basis read MN-major), then the consumers (thread = column) form
//            Z = Y - c split into two planes for sweep A.
// Operands: the basis windows are 128-byte swizzled K-major (sweep A) and
// MN-major (sweep B) matrices as stored; the plane operands are K-major core
// matrices (op_offset), written so by the other sweep's epilogue.
//
// Data movement.  The basis is stored tile-major and pre-swizzled: for each
// 256-row tile and 64-column window a contiguous [rows][64] BF16 block whose
// 16-byte chunks are XOR-permuted by (row & 7), the 128-byte swizzle of the
// tensor cores.  A machine's x_i tile is likewise one contiguous block ([k][rows]
// FP32).  So every stage is one or a few 1-D TMA bulk copies, issued by a
// producer warp into a ring of 4 basis slots and 2 x_i slots; the tensor-core
// warp waits on the slots' mbarriers and releases them with tcgen05.commit,
// the 8 consumer warps wait on the accumulators and x_i slots and release
// them with per-warp arrivals (every wait bounded), so no CTA-wide barrier
// sits in the streaming loop.  The CTAs claim units at run time from one
// stream (per iteration: sweep A, then sweep B, each system-major with the
// largest systems first); a unit waits only for the units of its own system
// that write its inputs, so no grid-wide barrier separates the sweeps.
//
// Precision: Q_i is BF16 (rounded once from the FP64 QR); products accumulate
// in FP32 in tensor memory; an operand split into planes keeps 16 (sweep
// A) or 24 (sweep B) significant bits of its FP32 value.  z_i tends to zero
// as the iteration converges, so its error is relative to the step; xbar does
// not, hence the third plane there.
#include <algorithm>
#include <array>
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
// right-hand sides whose state a consumer thread loads together in the heavy-ball
// and reverse-sweep row updates (their stores come after the loads)
constexpr int kRowBatch = 4;
constexpr int kProducerWarp = kConsumerWarps;       // issues the bulk copies
constexpr int kMmaWarp = kConsumerWarps + 1;        // issues the tensor-core instructions
constexpr int kThreads = 32 * (kConsumerWarps + 2);
constexpr int kTileRows = 256;   // rows of a basis storage tile (the largest sweep-A unit; 32 per consumer warp)
constexpr int kXRows = 128;      // rows of an x_i storage block (the smallest sweep-A unit)
constexpr int kWin = 64;         // basis columns per sweep-A window (one 128-byte row)
constexpr int kColsB = 512;      // columns of the largest sweep-B unit (64 per consumer warp)
constexpr int kRowsStageB = 32;  // rows per sweep-B stage
constexpr int kQSlots = 4, kXSlots = 2;
constexpr int kUQ = 4;           // depth of the queue of claimed units (producer -> consumers)
constexpr int kPlanesA = 2, kPlanesB = 3;
constexpr int kSlotQBytes = kTileRows * kWin * 2;  // 32 KB: 256 x 64 or 8 x (32 x 64) BF16
constexpr int kSlotZBytes = 8192;                  // operand planes of one stage
constexpr int kSlotBytes = kSlotQBytes + kSlotZBytes;
constexpr int kXSlotBytes = 32 * kTileRows * 4;    // x_i of one machine: two [32][128] FP32 blocks
constexpr int kBarOffset = kQSlots * kSlotBytes + kXSlots * kXSlotBytes;
// mbarriers: Q slots full/empty, x slots full/empty, unit queue full/empty,
// sweep-A accumulators full/free (two buffers), sweep-B accumulator full/free,
// drain; then the unit queue (64-bit unit indices) and the tensor-memory address
constexpr int kNumBars = 2 * kQSlots + 2 * kXSlots + 2 * kUQ + 4 + 3;
constexpr int kMaxSplit = 8;                       // parts per unit at most (apc_batch_set_tiles)
constexpr size_t kSmemUsed = size_t(kBarOffset) + kNumBars * sizeof(uint64_t) + kUQ * sizeof(long long) + sizeof(int);
constexpr size_t kSmemBytes = kSmemUsed + 1024;     // slack to align the slots to 1024 bytes
constexpr int kTmemCols = 512;                      // sweep A: 4 x 2k columns, sweep B: 4 x 3k

struct SysDesc {
    const __nv_bfloat16 *Q;  // tile-major, pre-swizzled (see q_block)
    const __nv_bfloat16 *QB; // the same 4 KB pieces ordered for sweep B (see qb_block), or null
    float *X;                // x_i in blocks of 128 rows (see x_block)
    float2 *Xb;              // [kp][npad]  master estimate, double-float
    uint8_t *Xop;            // xbar' planes, B operand of sweep B (see op_offset), npad x 3kp BF16
    uint8_t *Zop;            // z planes, B operand of sweep A (see op_offset), Cq x 2kp BF16
    const float *Ct;         // [kp][Cq] c_i, FP32
    const int *coloff;       // [m + 1], multiples of 16
    float2 *Mb;              // [kp][npad]  heavy-ball momentum, double-float; reverse sweep: ell
    float *Gc;               // [kp][Cq]  reverse sweep: dL/dc_i accumulated (FP32)
    float *Spart;            // [spA][kp][npad] split sweep A: the parts' row sums (or gradients)
    float *Ypart;            // [spB][kp][Cq]   split sweep B: the parts' products Q^T xbar'
    int *cntA, *cntB;        // split sweeps: parts done per (row unit, warp) / (column unit, warp, M-tile)
    int spA, spB, chunkB;    // parts per unit (machines in sweep A, rows in sweep B); rows per sweep-B part
    int npad, m, Cq, C;
    int nuA, nuB;            // units of this system in sweep A and in sweep B
    float g_hi, g_lo, em_hi, em_lo, e1_hi, e1_lo, im_hi, im_lo;
    float na_hi, na_lo, hb_hi, hb_lo;  // heavy ball: -alpha and beta
    float omg_hi, omg_lo, gm_hi, gm_lo;  // reverse sweep: 1 - gamma and gamma m
};

struct BatchArgs {
    const SysDesc *sys;
    const int2 *unitsA;  // (system, first row of the tile), system-major, largest systems first
    const int2 *unitsB;  // (system, first column), same order of systems
    int nA, nB;
    unsigned long long *claim;  // units claimed so far (zero at launch)
    unsigned long long *done;   // [2 nsys] per system: sweep-A, sweep-B unit completions x 8 (zero at launch)
    int64_t iters;
    int init;
    int hb;              // 1: distributed-preconditioned heavy ball instead of APC
    int adj;             // 1: reverse sweep through `iters` steps (apc_batch_backward)
    int rowsA;           // rows of a sweep-A unit: 128 or 256
    int colsB;           // columns of a sweep-B unit: 128, 256 or 512
    int prefetch;        // sweep A: L2 prefetch distance in windows / machines (0..8)
    int l2;              // L2 policy of the bulk copies: 0 evict-first (stream), 1 normal, 2 evict-last
    uint32_t barrier_skew;  // test hook: added to every cross-CTA wait target (0 = normal)
    uint32_t *bar;          // grid barrier after the initialisation (zero at launch)
    int *err;
    uint64_t timeout_ns;
};

// rows of tile t
__host__ __device__ __forceinline__ int tile_rows(int npad, int t) { return min(kTileRows, npad - kTileRows * t); }
// first element of the basis block (tile t, window w): [tile_rows][64] BF16
__host__ __device__ __forceinline__ size_t q_block(int Cq, int npad, int t, int w) {
    return size_t(t) * kTileRows * Cq + size_t(w) * tile_rows(npad, t) * kWin;
}
// Sweep B's copy of the basis: the [32 rows][64 columns] pieces of q_block
// reordered so that a 32-row group's windows are contiguous, [tile][group of
// 32 rows][window][32][64] (the same bytes, pre-swizzled alike).  A sweep-B
// stage of up to 8 windows is then one bulk copy per 32 rows instead of one
// per window (each copy costs the issuing thread 100+ cycles).  Built only
// when the batch's bases are far larger than L2: when they fit, sweep B
// re-reads from L2 what sweep A streamed, and a second copy would lose that
// (one 8192 system, 134 MB: 44.7 -> 37.6 % L2 hits, forward 20 -> 24 ms).
// First element of the piece (row group G = row / 32, window w):
__host__ __device__ __forceinline__ size_t qb_block(int Cq, int G, int w) {
    return (size_t(G) * (Cq / kWin) + w) * 32 * kWin;
}
// first element of machine i's x_i block for rows 128 u .. 128 u + 127:
// [kp][128] FP32 (the last block of a system padded to 128 rows with zeros).
// A machine's blocks are contiguous (nxs = blocks per machine, n_pad / 128
// rounded up), so a 256-row unit's x_i tile is one bulk copy.
__host__ __device__ __forceinline__ int x_blocks(int npad) { return (npad + kXRows - 1) / kXRows; }
__host__ __device__ __forceinline__ size_t x_block(int nxs, int kp, int u, int i) {
    return (size_t(i) * nxs + u) * kp * kXRows;
}

// ---- PTX wrappers ------------------------------------------------------------
__device__ __forceinline__ float lds_f32(uint32_t addr) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(addr));
    return v;
}
// Byte offset of element (n, kk) of a B operand stored as K-major core
// matrices without swizzle: for every 16 values of kk a block of `nrows` x 16
// BF16, made of 8 x 8 core matrices (n-group n/8 at 256 bytes, k-group at 128
// bytes, 16 bytes per row).  In the descriptor: leading-dimension offset 128
// (between k-groups), stride-dimension offset 256 (between n-groups).
__host__ __device__ __forceinline__ size_t op_offset(int nrows, int n, int64_t kk) {
    return size_t(kk >> 4) * nrows * 32 + size_t(n >> 3) * 256 + size_t((kk >> 3) & 1) * 128 + size_t(n & 7) * 16 +
           size_t(kk & 7) * 2;
}

// ---- tensor cores (tcgen05): operands in shared memory, accumulators in tensor memory ----
// Shared-memory matrix descriptor: start address, leading- and stride-dimension
// byte offsets, swizzle mode (0: none, 2: 128-byte).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t swz) {
    return uint64_t((saddr & 0x3FFFFu) >> 4) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46) | (uint64_t(swz & 7u) << 61);
}
// Instruction descriptor, kind::f16: FP32 accumulators, BF16 A and B, B
// K-major, A K-major (a_mn = 0) or MN-major (1), M = 128, N = n.
__host__ __device__ constexpr uint32_t instr_desc(int n, uint32_t a_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (a_mn << 15) | (uint32_t(n >> 3) << 17) | (uint32_t(128 >> 4) << 24);
}
// D (+)= A B^T on the tensor cores (kind::f16), and the arrival on an
// mbarrier once every tcgen05 operation issued so far has completed: both
// executed by the whole converged tensor-core warp, one elected lane issuing.
// The operands stay warp-uniform, which makes an MMA cheaper to issue than
// from a single lane in divergent code (measured: about 110-170 cycles per
// instruction from lane 0 alone).
__device__ __forceinline__ void tc_mma_w(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, bool accumulate) {
    asm volatile(
        "{\n\t.reg .pred p, e;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "elect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate ? 1u : 0u)
        : "memory");
}
__device__ __forceinline__ void tc_commit_w(uint64_t *bar) {
    asm volatile(
        "{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\t"
        "@e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n\t}"
        ::"r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 16 consecutive FP32 columns of this thread's tensor-memory lane (warp-wide)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
// L2 cache policy of the bulk copies: evict-first for operands streamed once
// per sweep (many systems, far more bytes than L2), normal or evict-last so
// that a single system's basis (about the size of L2) may stay on chip
// between the two sweeps and across iterations
__device__ __forceinline__ uint64_t l2_policy(int mode) {
    uint64_t p;
    if (mode == 2)
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    else if (mode == 1)
        asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    else
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
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

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// x, opaque to the compiler: a stride passed through this is not hoisted out
// of a loop as a set of per-right-hand-side offsets held in registers
__device__ __forceinline__ uint32_t opaque_u32(uint32_t x) {
    uint32_t y;
    asm volatile("mov.b32 %0, %1;" : "=r"(y) : "r"(x));
    return y;
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
};

// A bounded wait made warp-uniform (the tensor-core warp runs converged: its
// elected issues need every lane)
__device__ __forceinline__ bool wait_w(const Ring &R, uint64_t *bar, uint32_t parity) {
    return __all_sync(0xffffffffu, R.wait(bar, parity));
}

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

// ---- split units -------------------------------------------------------------------
// A unit may be split into parts that run on different CTAs: the machines of
// a sweep-A unit (each part updates its machines' x_i and forms a partial row
// sum) and the rows of a sweep-B unit (each part a partial product).  Each
// consumer warp stores its part's values, counts the parts done, and the last
// one adds all parts in part order (a fixed order) and finishes the unit.
struct PartA {
    int i_lo, i_hi;  // machines
    int c_lo, c_hi;  // their 16-column chunks
};
template <bool kSplit>
__device__ __forceinline__ PartA part_a(const SysDesc &d, int p) {
    PartA r;
    if constexpr (kSplit) {
        const int mc = (d.m + d.spA - 1) / d.spA;
        r.i_lo = p * mc;
        r.i_hi = min(d.m, r.i_lo + mc);
        r.c_lo = __ldg(d.coloff + r.i_lo) >> 4;
        r.c_hi = __ldg(d.coloff + r.i_hi) >> 4;
    } else {
        r.i_lo = 0;
        r.i_hi = d.m;
        r.c_lo = 0;
        r.c_hi = d.C >> 4;
    }
    return r;
}
template <bool kSplit>
__device__ __forceinline__ int2 part_b(const SysDesc &d, int p) {  // rows [x, y)
    if constexpr (kSplit) {
        const int lo = p * d.chunkB;
        return make_int2(lo, min(d.npad, lo + d.chunkB));
    } else {
        return make_int2(0, d.npad);
    }
}
// Store this part's KP values (part p of np, element q at part + (p KP + q)
// stride), count the part in *cnt; the warp that completes the count sums
// the np parts in order into v and resets the count.  True for that warp.
template <int KP>
__device__ __forceinline__ bool combine_parts(float (&v)[KP], float *part, size_t stride, int np, int p, int *cnt) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < KP; ++q) __stcg(part + (size_t(p) * KP + q) * stride, v[q]);
    __threadfence();
    __syncwarp();
    int old = 0;
    if (lane == 0) old = atomicAdd(cnt, 1);
    old = __shfl_sync(0xffffffffu, old, 0);
    if (old != np - 1) return false;
    __threadfence();
    // part after part, each part's KP values loaded together (one round trip
    // per part instead of one per value); every sum still adds the parts in
    // part order, starting from zero
#pragma unroll
    for (int q = 0; q < KP; ++q) v[q] = 0.0f;
    for (int pp = 0; pp < np; ++pp) {
        const float *pq = part + size_t(pp) * KP * stride;
#pragma unroll
        for (int q = 0; q < KP; ++q) v[q] += __ldcg(pq + size_t(q) * stride);
    }
    __syncwarp();
    if (lane == 0) atomicExch(cnt, 0);
    return true;
}

// ---- sweep A ---------------------------------------------------------------------
template <int MT, bool kSplit>
__device__ void sweep_a_producer(const Ring &R, Cursor &cur, const SysDesc &d, int row0, int part, int rowsA, int pf,
                                 bool no_x, uint64_t policy) {
    constexpr int KP = 16 * MT;
    // the unit's rows within their 256-row basis tile (the window blocks are
    // [tile rows][64] row-major, so any 128-row part of one is contiguous)
    const int t = row0 / kTileRows, ro = row0 - t * kTileRows;
    const int rows = min(rowsA, d.npad - row0);
    const PartA pa = part_a<kSplit>(d, part);
    const int w_lo = pa.c_lo >> 2, w_hi = (pa.c_hi + 3) >> 2;  // windows holding the part's chunks
    const uint32_t qbytes = uint32_t(rows) * kWin * 2, zbytes = kPlanesA * KP * 128;
    const int u0 = row0 / kXRows, nxb = (rows + kXRows - 1) / kXRows;  // x_i blocks of 128 rows per machine
    const int nxs = x_blocks(d.npad);
    const uint32_t xblk = uint32_t(KP) * kXRows * 4;
    auto qsrc = [&](int w) { return d.Q + q_block(d.Cq, d.npad, t, w) + size_t(ro) * kWin; };
    int pi = pa.i_lo;  // next machine whose x_i tile is due
    // L2 prefetch runs `pf` windows / machines ahead of the shared-memory ring
    // (measured on 256 systems with 256-row units: 2 is 1.5 % faster than 4, 8
    // is 13 % slower, none 4 % slower; an L2 prefetch in sweep B made it 40 %
    // slower); the tile tuner may pick another distance
    for (int w = w_lo; w < min(w_lo + pf, w_hi); ++w) prefetch_l2(qsrc(w), qbytes);
    if (!no_x)
        for (int i = pa.i_lo; i < min(pa.i_lo + pf, pa.i_hi); ++i)
            prefetch_l2(d.X + x_block(nxs, KP, u0, i), uint32_t(nxb) * xblk);
    for (int w = w_lo; w < w_hi; ++w) {
        const uint32_t s = cur.q % kQSlots;
        if (!acquire_slot(R, R.empty, kQSlots, cur.q)) return;
        mbar_arrive_expect_tx(&R.full[s], qbytes + zbytes);
        tma_load_1d(R.qslot(s), qsrc(w), qbytes, &R.full[s], policy);
        tma_load_1d(R.qslot(s) + kSlotQBytes, d.Zop + size_t(w) * zbytes, zbytes, &R.full[s], policy);
        if (w + pf < w_hi) prefetch_l2(qsrc(w + pf), qbytes);
        ++cur.q;
        // x_i tiles of the machines whose last chunk lies in this window
        while (!no_x && pi < pa.i_hi && (__ldg(d.coloff + pi + 1) - 16) / kWin == w) {
            const uint32_t xs = cur.x % kXSlots;
            if (!acquire_slot(R, R.xempty, kXSlots, cur.x)) return;
            mbar_arrive_expect_tx(&R.xfull[xs], uint32_t(nxb) * xblk);
            tma_load_1d(R.xslot(xs), d.X + x_block(nxs, KP, u0, pi), uint32_t(nxb) * xblk, &R.xfull[xs], policy);
            if (pi + pf < pa.i_hi)
                prefetch_l2(d.X + x_block(nxs, KP, u0, pi + pf), uint32_t(nxb) * xblk);
            ++cur.x;
            ++pi;
        }
    }
}

// Tensor-core warp, sweep A: for every 16-column chunk of machine i,
// D_b += Q[tile rows, chunk] Z[chunk, planes x rhs] into accumulator buffer
// b = (machine count) mod 2, one M = 128 instruction per 128 rows of the tile
// (A: the window block, 128-byte swizzled K-major; B: the z planes, core
// matrices).  After the machine's last chunk the buffer is handed to the
// consumers; a Q slot is released when the instructions reading it are done.
// Heavy ball: one accumulation over every machine of the tile.
template <int MT, bool kSplit>
__device__ void sweep_a_mma(const Ring &R, Cursor &cur, uint32_t &mc, uint64_t *dfull, uint64_t *dfree,
                            const SysDesc &d, int row0, int part, int rowsA, bool hb, uint32_t tmem) {
    constexpr int NA = kPlanesA * 16 * MT;
    constexpr uint32_t idesc = instr_desc(NA, 0);
    const int rows = min(rowsA, d.npad - row0);
    const int nmt = rows > 128 ? 2 : 1;
    const PartA pa = part_a<kSplit>(d, part);
    const int w_lo = pa.c_lo >> 2, w_hi = (pa.c_hi + 3) >> 2;
    int i = pa.i_lo, iend = __ldg(d.coloff + pa.i_lo + 1) >> 4;
    bool first = true;
    uint32_t b = 0;
    for (int w = w_lo; w < w_hi; ++w) {
        const uint32_t s = cur.q % kQSlots;
        if (!wait_w(R, &R.full[s], (cur.q / kQSlots) & 1)) return;
        tc_fence_after();
        const uint32_t sq = smem_u32(R.qslot(s)), sz = sq + kSlotQBytes;
        for (int kc = 0; kc < 4; ++kc) {
            const int c16 = 4 * w + kc;
            if constexpr (kSplit)
                if (c16 < pa.c_lo) continue;
            if (c16 >= pa.c_hi) break;
            if (first) {
                b = mc & 1;
                if (mc >= 2 && !wait_w(R, &dfree[b], ((mc >> 1) - 1) & 1)) return;
                tc_fence_after();
            }
            for (int h = 0; h < nmt; ++h)
                tc_mma_w(tmem + uint32_t((2 * b + h) * NA), smem_desc(sq + h * 16384 + kc * 32, 16, 1024, 2),
                       smem_desc(sz + kc * (NA * 32), 128, 256, 0), idesc, !first);
            first = false;
            if (hb ? c16 + 1 == pa.c_hi : c16 + 1 == iend) {
                tc_commit_w(&dfull[b]);
                ++mc;
                first = true;
                if (!hb && ++i < pa.i_hi) iend = __ldg(d.coloff + i + 1) >> 4;
            }
        }
        tc_commit_w(&R.empty[s]);
        ++cur.q;
    }
}

// xbar' (FP32, the hi part) of row `row` split into three BF16 planes for
// sweep B: element (plane p, right-hand side q) at op_offset(3 kp, p kp + q,
// row); two adjacent rows (even lane, odd lane) go into one 32-bit store.
template <int MT>
__device__ void store_xop(const SysDesc &d, int64_t row, const float (&xo)[16 * MT]) {
    constexpr int KP = 16 * MT, NB = kPlanesB * KP;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < KP; ++q) {
        const float x1 = __shfl_down_sync(0xffffffffu, xo[q], 1);
        if ((lane & 1) == 0) {
            uint32_t w[kPlanesB];
            split2<kPlanesB>(xo[q], x1, w);
#pragma unroll
            for (int p = 0; p < kPlanesB; ++p)
                __stcg(reinterpret_cast<uint32_t *>(d.Xop + op_offset(NB, p * KP + q, row)), w[p]);
        }
    }
}

// Consumers, sweep A: thread = one row of the tile (warp w: rows 128 (w/4) +
// 32 (w%4) .. + 31, the tensor-memory lanes of its quarter).  Per machine:
// w_i = the two planes' accumulators summed, then
// x_i <- x_i + gamma (xbar - x_i - w_i) and the running row sum; at the end
// the master's row update (double-float) and the xbar' planes of sweep B.
// Reverse sweep (kAdj, one accumulation over every machine, like heavy ball):
// the step's row update of (ell, lbar) and the planes of the next mu.
template <int MT, bool kAdj, bool kSplit>
__device__ void sweep_a_consumer(const Ring &R, Cursor &cur, uint32_t &mc, uint64_t *dfull, uint64_t *dfree,
                                 const SysDesc &d, int row0, int part, int rowsA, bool init, bool hb, float gh,
                                 float gl, uint32_t tmem, bool last) {
    constexpr int KP = 16 * MT, NA = kPlanesA * KP;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int h = warp >> 2, quad = warp & 3;
    const int rows = min(rowsA, d.npad - row0);
    const int r = 128 * h + 32 * quad + lane;         // row within the tile
    const bool wact = 128 * h + 32 * quad < rows;     // rows is a multiple of 32: warp-uniform
    const int64_t grow = int64_t(row0) + r;           // row within the system
    const uint32_t tl = tmem + (uint32_t(32 * quad) << 16);
    float xbh[KP], xbl[KP], S[KP], W[KP];
#pragma unroll
    for (int q = 0; q < KP; ++q) {
        xbh[q] = xbl[q] = S[q] = W[q] = 0.0f;
    }
    if (wact && !init && !hb) {
#pragma unroll
        for (int q = 0; q < KP; ++q) {
            const float2 v = __ldcg(d.Xb + size_t(q) * d.npad + grow);
            xbh[q] = v.x;
            xbl[q] = v.y;
        }
    }
    const PartA pa = part_a<kSplit>(d, part);
    const int nm = hb ? 1 : pa.i_hi - pa.i_lo;
    for (int ii = 0; ii < nm; ++ii) {
        const int i = pa.i_lo + ii;
        const uint32_t b = mc & 1;
        if (!R.wait(&dfull[b], (mc >> 1) & 1)) return;
        tc_fence_after();
        if (wact) {
            const uint32_t col = uint32_t((2 * b + h) * NA);
#pragma unroll
            for (int c0 = 0; c0 < KP; c0 += 16) {
                float p0[16], p1[16];
                tc_ld16(tl + col + c0, p0);
                tc_ld16(tl + col + KP + c0, p1);
#pragma unroll
                for (int j = 0; j < 16; ++j) W[c0 + j] = p0[j] + p1[j];
            }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&dfree[b]);
        ++mc;
        if (hb) break;
        // machine i is complete: x_i <- x_i + gamma (xbar - x_i - w_i), row sums
        uint32_t xs = 0, sx = 0;
        if (!init) {
            xs = cur.x % kXSlots;
            if (!R.wait(&R.xfull[xs], (cur.x / kXSlots) & 1)) return;
            sx = smem_u32(R.xslot(xs));
        }
        if (wact) {
            // the x_i tile holds [kp][128] blocks of 128 rows: the row's value
            // for right-hand side q sits 512 q bytes after its first one
            const uint32_t sxr = sx + uint32_t(h) * uint32_t(KP * kXRows * 4) + uint32_t(r & (kXRows - 1)) * 4u;
            float *xg = d.X + x_block(x_blocks(d.npad), KP, (row0 >> 7) + h, i) + (r & (kXRows - 1));
#pragma unroll
            for (int q = 0; q < KP; ++q) {
                const float xo = init ? 0.0f : lds_f32(sxr + uint32_t(q) * (kXRows * 4));
                const float v = ((xbh[q] - xo) + xbl[q]) - W[q];
                const float xn = upd_exact(xo, gh, gl, v);
                S[q] += xn;
                __stcg(xg + q * kXRows, xn);
            }
        }
        if (!init) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&R.xempty[xs]);
            ++cur.x;
        }
    }
    if (!wact) return;
    if constexpr (kSplit) {
        // a part of a split unit: only the warp that completes the row unit's
        // parts goes on, with the sum over all parts
        if (d.spA > 1) {
            int *cnt = d.cntA + (row0 / rowsA) * kConsumerWarps + (threadIdx.x >> 5);
            if (!(hb ? combine_parts<KP>(W, d.Spart + grow, size_t(d.npad), d.spA, part, cnt)
                     : combine_parts<KP>(S, d.Spart + grow, size_t(d.npad), d.spA, part, cnt)))
                return;
        }
    }
    float (&xo)[KP] = S;  // the new xbar (hi part), in place of the row sums
    if constexpr (kAdj) {
        // one step of the reverse sweep through the affine form of App. A.
        // Every machine's adjoint is the same vector ell (all start at zero and
        // follow the same recursion), so per row, with W = sum_i Q_i v_i and
        // v = Q^T mu from sweep B:
        //   mu = ell + (eta/m) lbar,  ell' = (1 - gamma) mu,
        //   lbar' = (1 - eta) lbar + gamma (m mu - W),
        // and the next mu (ell' + lbar'/m after the last step) to sweep B
        const float2 em = make_float2(d.em_hi, d.em_lo), e1 = make_float2(d.e1_hi, d.e1_lo);
        const float2 om = make_float2(d.omg_hi, d.omg_lo), gm = make_float2(d.gm_hi, d.gm_lo);
        const float2 ng = make_float2(-d.g_hi, -d.g_lo);
        const float2 nx = last ? make_float2(d.im_hi, d.im_lo) : em;
        char *xb = reinterpret_cast<char *>(d.Xb + grow), *mb = reinterpret_cast<char *>(d.Mb + grow);
        const uint32_t ns = opaque_u32(uint32_t(d.npad) * 8u);
#pragma unroll
        for (int q0 = 0; q0 < KP; q0 += kRowBatch) {
            // (ell, lbar) of kRowBatch right-hand sides loaded ahead of their stores
            float2 l[kRowBatch], lb[kRowBatch];
#pragma unroll
            for (int j = 0; j < kRowBatch; ++j) {
                l[j] = __ldcg(reinterpret_cast<const float2 *>(mb + size_t(q0 + j) * ns));
                lb[j] = __ldcg(reinterpret_cast<const float2 *>(xb + size_t(q0 + j) * ns));
            }
#pragma unroll
            for (int j = 0; j < kRowBatch; ++j) {
                const int q = q0 + j;
                const float2 mu = dfa(l[j], dfm(em, lb[j]));
                const float2 ln = dfm(om, mu);
                const float2 lbn = dfa(dfa(dfm(e1, lb[j]), dfm(gm, mu)), dfm(ng, make_float2(W[q], 0.0f)));
                __stcg(reinterpret_cast<float2 *>(mb + size_t(q) * ns), ln);
                __stcg(reinterpret_cast<float2 *>(xb + size_t(q) * ns), lbn);
                xo[q] = dfa(ln, dfm(nx, lbn)).x;
            }
        }
    } else if (hb) {
        // heavy ball on the preconditioned system (Sec. 4.3 update, Sec. 6):
        // W holds the gradient sum_i Q_i (Q_i^T x - c_i);
        // zeta <- beta zeta + gradient, x <- x - alpha zeta
        const float2 beta = make_float2(d.hb_hi, d.hb_lo), nalpha = make_float2(d.na_hi, d.na_lo);
        char *xb = reinterpret_cast<char *>(d.Xb + grow), *mb = reinterpret_cast<char *>(d.Mb + grow);
        const uint32_t ns = opaque_u32(uint32_t(d.npad) * 8u);
#pragma unroll
        for (int q0 = 0; q0 < KP; q0 += kRowBatch) {
            // (zeta, x) of kRowBatch right-hand sides loaded ahead of their stores
            float2 z[kRowBatch], x[kRowBatch];
#pragma unroll
            for (int j = 0; j < kRowBatch; ++j) {
                z[j] = __ldcg(reinterpret_cast<const float2 *>(mb + size_t(q0 + j) * ns));
                x[j] = __ldcg(reinterpret_cast<const float2 *>(xb + size_t(q0 + j) * ns));
            }
#pragma unroll
            for (int j = 0; j < kRowBatch; ++j) {
                const int q = q0 + j;
                const float2 zn = dfa(dfm(beta, z[j]), make_float2(W[q], 0.0f));
                const float2 xn = dfa(x[j], dfm(nalpha, zn));
                __stcg(reinterpret_cast<float2 *>(mb + size_t(q) * ns), zn);
                __stcg(reinterpret_cast<float2 *>(xb + size_t(q) * ns), xn);
                xo[q] = xn.x;
            }
        }
    } else {
        // master: xbar' = (eta/m) S + (1 - eta) xbar   (initialisation: S / m)
        const float2 em = make_float2(init ? d.im_hi : d.em_hi, init ? d.im_lo : d.em_lo);
        const float2 e1 = make_float2(d.e1_hi, d.e1_lo);
#pragma unroll
        for (int q = 0; q < KP; ++q) {
            float2 xn = dfm(em, make_float2(S[q], 0.0f));
            if (!init) xn = dfa(xn, dfm(e1, make_float2(xbh[q], xbl[q])));
            __stcg(d.Xb + size_t(q) * d.npad + grow, xn);
            xo[q] = xn.x;
        }
    }
    store_xop<MT>(d, grow, xo);
}

// ---- sweep B -----------------------------------------------------------------------
// Rows of Q per sweep-B stage: 32 (eight 4 KB pieces at 512 columns), or 64
// when the unit is at most 256 columns wide and the xbar' planes of 64 rows
// (3 x 16 right-hand sides) still fit the slot's 8 KB: a narrow unit then
// keeps twice the bytes in flight per stage.  Never past the system's rows.
template <int MT>
__device__ __forceinline__ int rows_stage_b(int nwin, int npad, int r0) {
    const int rs = (MT == 1 && nwin <= 4) ? 2 * kRowsStageB : kRowsStageB;
    return min(rs, npad - r0);
}

template <int MT, bool kSplit>
__device__ void sweep_b_producer(const Ring &R, Cursor &cur, const SysDesc &d, int col0, int part, int colsB,
                                 uint64_t policy) {
    const int nwin = min(colsB, d.Cq - col0) / kWin;
    const int2 pr = part_b<kSplit>(d, part);
    constexpr uint32_t prow = kPlanesB * 16 * MT * 2;  // bytes of the xbar' planes per row
    for (int r0 = pr.x, rs; r0 < pr.y; r0 += rs) {
        rs = rows_stage_b<MT>(nwin, pr.y, r0);
        const uint32_t s = cur.q % kQSlots;
        if (!acquire_slot(R, R.empty, kQSlots, cur.q)) return;
        if (d.QB) {
            // sweep B's copy, [group of 32 rows][window][32][64]: one copy of
            // nwin pieces per group
            const uint32_t gbytes = uint32_t(nwin) * 32 * kWin * 2;
            mbar_arrive_expect_tx(&R.full[s], uint32_t(rs / 32) * gbytes + uint32_t(rs) * prow);
            for (int gg = 0; gg < rs / 32; ++gg)
                tma_load_1d(R.qslot(s) + gg * gbytes, d.QB + qb_block(d.Cq, r0 / 32 + gg, col0 / kWin), gbytes,
                            &R.full[s], policy);
        } else {
            // the shared basis: one [rs rows][64] piece per window
            const int t = r0 / kTileRows, rr = r0 % kTileRows;
            const uint32_t blk = uint32_t(rs) * kWin * 2;
            mbar_arrive_expect_tx(&R.full[s], uint32_t(nwin) * blk + uint32_t(rs) * prow);
            for (int j = 0; j < nwin; ++j)
                tma_load_1d(R.qslot(s) + j * blk, d.Q + q_block(d.Cq, d.npad, t, col0 / kWin + j) + size_t(rr) * kWin,
                            blk, &R.full[s], policy);
        }
        tma_load_1d(R.qslot(s) + kSlotQBytes, d.Xop + size_t(r0) * prow, uint32_t(rs) * prow, &R.full[s], policy);
        ++cur.q;
    }
}

// z = Y - c of column `col` split into two BF16 planes for sweep A: element
// (plane p, right-hand side q) at op_offset(2 kp, p kp + q, col); two adjacent
// columns (even lane, odd lane) go into one 32-bit store.  zero_y: z = -c.
template <int MT>
__device__ void store_z(const SysDesc &d, int col, const float (&Y)[16 * MT], bool zero_y) {
    constexpr int KP = 16 * MT, NA = kPlanesA * KP;
    const int lane = threadIdx.x & 31;
    const char *ct = reinterpret_cast<const char *>(d.Ct + col);
    const uint32_t cs = opaque_u32(uint32_t(d.Cq) * 4u);
#pragma unroll
    for (int q = 0; q < KP; ++q) {
        const float z = (zero_y ? 0.0f : Y[q]) - __ldg(reinterpret_cast<const float *>(ct + size_t(q) * cs));
        const float z1 = __shfl_down_sync(0xffffffffu, z, 1);
        if ((lane & 1) == 0) {
            uint32_t w[kPlanesA];
            split2<kPlanesA>(z, z1, w);
#pragma unroll
            for (int p = 0; p < kPlanesA; ++p)
                __stcg(reinterpret_cast<uint32_t *>(d.Zop + op_offset(NA, p * KP + q, col)), w[p]);
        }
    }
}

// Reverse sweep: v = Y of column `col` (Y = Q^T mu) added to dL/dc with
// weight gamma (1 at the end of the sweep, the initialisation's term) and, except
// at the end, split into two BF16 planes for sweep A (the layout of store_z).
template <int MT>
__device__ void store_v(const SysDesc &d, int col, const float (&Y)[16 * MT], bool fin) {
    constexpr int KP = 16 * MT, NA = kPlanesA * KP;
    const int lane = threadIdx.x & 31;
    char *gc = reinterpret_cast<char *>(d.Gc + col);
    const uint32_t cs = opaque_u32(uint32_t(d.Cq) * 4u);
    const float gh = fin ? 1.0f : d.g_hi, gl = fin ? 0.0f : d.g_lo;
#pragma unroll
    for (int q0 = 0; q0 < KP; q0 += kRowBatch) {
        // dL/dc of kRowBatch right-hand sides loaded ahead of their stores
        float g[kRowBatch];
#pragma unroll
        for (int j = 0; j < kRowBatch; ++j) g[j] = __ldcg(reinterpret_cast<const float *>(gc + size_t(q0 + j) * cs));
#pragma unroll
        for (int j = 0; j < kRowBatch; ++j) {
            const int q = q0 + j;
            const float y = Y[q];
            __stcg(reinterpret_cast<float *>(gc + size_t(q) * cs), g[j] + fmaf(gh, y, gl * y));
            if (!fin) {
                const float y1 = __shfl_down_sync(0xffffffffu, y, 1);
                if ((lane & 1) == 0) {
                    uint32_t w[kPlanesA];
                    split2<kPlanesA>(y, y1, w);
#pragma unroll
                    for (int p = 0; p < kPlanesA; ++p)
                        __stcg(reinterpret_cast<uint32_t *>(d.Zop + op_offset(NA, p * KP + q, col)), w[p]);
                }
            }
        }
    }
}

// Tensor-core warp, sweep B: D_h += Q[rows, 128 columns]^T Xop[rows, planes x
// rhs] for the unit's M-tiles h (A: the stage's 64-column blocks read
// MN-major, 128-byte swizzle, 4 KB between blocks; B: the xbar' planes, core
// matrices), over all row stages; the accumulators go to the consumers once
// per unit and are reused after they release them.
template <int MT, bool kSplit>
__device__ void sweep_b_mma(const Ring &R, Cursor &cur, uint32_t &ubc, uint64_t *bfull, uint64_t *bfree,
                            const SysDesc &d, int col0, int part, int colsB, uint32_t tmem) {
    constexpr int NB = kPlanesB * 16 * MT;
    constexpr uint32_t idesc = instr_desc(NB, 1);
    const int nwin = min(colsB, d.Cq - col0) / kWin;
    const int nmt = (nwin * kWin + 127) / 128;
    if (ubc > 0 && !wait_w(R, bfree, (ubc - 1) & 1)) return;
    tc_fence_after();
    bool first = true;
    const int2 pr = part_b<kSplit>(d, part);
    for (int r0 = pr.x, rs; r0 < pr.y; r0 += rs) {
        rs = rows_stage_b<MT>(nwin, pr.y, r0);
        // stage layout, sweep B's copy (qb_block): [group of 32 rows][window][32][64],
        // 4 KB between windows (the M direction), nwin x 4 KB between 32-row
        // groups; the shared basis: [window][rs rows][64], rs x 128 bytes
        // between windows
        const uint32_t wstr = d.QB ? 4096u : uint32_t(rs) * 128u;
        const uint32_t gbytes = d.QB ? uint32_t(nwin) * 4096u : 4096u;
        const uint32_t s = cur.q % kQSlots;
        if (!wait_w(R, &R.full[s], (cur.q / kQSlots) & 1)) return;
        tc_fence_after();
        const uint32_t sq = smem_u32(R.qslot(s)), sx = sq + kSlotQBytes;
        for (int ks = 0; ks < rs / 16; ++ks) {
            for (int h = 0; h < nmt; ++h)
                tc_mma_w(tmem + uint32_t(h * NB),
                         smem_desc(sq + 2 * h * wstr + (ks >> 1) * gbytes + (ks & 1) * 2048, wstr, 1024, 2),
                       smem_desc(sx + ks * (NB * 32), 128, 256, 0), idesc, !first);
            first = false;
        }
        tc_commit_w(&R.empty[s]);
        ++cur.q;
    }
    tc_commit_w(bfull);
    ++ubc;
}

// Consumers, sweep B: thread = one column (warp w: M-tiles w/4 and w/4 + 2,
// columns 32 (w%4) .. + 31 of each, the tensor-memory lanes of its quarter):
// Y = the three planes' accumulators summed, then z = Y - c to sweep A
// (reverse sweep: v = Y, see store_v).
template <int MT, bool kAdj, bool kSplit>
__device__ void sweep_b_consumer(const Ring &R, uint32_t &ubc, uint64_t *bfull, uint64_t *bfree, const SysDesc &d,
                                 int col0, int part, int colsB, uint32_t tmem, bool fin) {
    constexpr int KP = 16 * MT, NB = kPlanesB * KP;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, quad = warp & 3;
    const int ncols = min(colsB, d.Cq - col0);
    if (!R.wait(bfull, ubc & 1)) return;
    tc_fence_after();
    const uint32_t tl = tmem + (uint32_t(32 * quad) << 16);
    // both M-tiles' sums are read before the accumulators are released, so
    // the tensor cores can start the next unit while z is formed and stored
    float Y[2][KP];
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
        const int h = (warp >> 2) + 2 * hh;
        if (128 * h + 32 * quad >= ncols) continue;  // ncols is a multiple of 64: warp-uniform
#pragma unroll
        for (int c0 = 0; c0 < KP; c0 += 16) {
            // (plane 0 + plane 1) + plane 2, one plane's 16 columns at a time
#pragma unroll
            for (int pl = 0; pl < kPlanesB; ++pl) {
                float pv[16];
                tc_ld16(tl + uint32_t(h * NB + pl * KP + c0), pv);
#pragma unroll
                for (int j = 0; j < 16; ++j) Y[hh][c0 + j] = pl == 0 ? pv[j] : Y[hh][c0 + j] + pv[j];
            }
        }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(bfree);
    ++ubc;
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
        const int h = (warp >> 2) + 2 * hh;
        const int cl = 128 * h + 32 * quad;
        if (cl < ncols) {
            if constexpr (kSplit) {
                // a part of a split unit: only the warp that completes the
                // column unit's parts goes on, with the sum over all parts
                if (d.spB > 1) {
                    int *cnt = d.cntB + ((col0 / colsB) * kConsumerWarps + warp) * 2 + hh;
                    if (!combine_parts<KP>(Y[hh], d.Ypart + col0 + cl + lane, size_t(d.Cq), d.spB, part, cnt))
                        continue;
                }
            }
            if constexpr (kAdj) store_v<MT>(d, col0 + cl + lane, Y[hh], fin);
            else store_z<MT>(d, col0 + cl + lane, Y[hh], false);
        }
    }
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

// Bounded wait until a completion counter reaches `target` (acquire); gives
// up early when another CTA has already reported a time-out.
__device__ bool wait_count(const unsigned long long *p, unsigned long long target, const BatchArgs &a,
                           int *abort_flag) {
    if (ld_acquire_u64(p) >= target) return true;
    const uint64_t t0 = globaltimer_ns();
    for (;;) {
        if (ld_acquire_u64(p) >= target) return true;
        if (*reinterpret_cast<volatile int *>(a.err) != 0 || globaltimer_ns() - t0 > a.timeout_ns) break;
    }
    atomicExch(abort_flag, 1);
    atomicCAS(a.err, 0, DEV_TIMEOUT_GRID);
    return false;
}

template <int MT, bool kAdj, bool kSplit>
__global__ void __launch_bounds__(kThreads, 1) apc_batch_kernel(const BatchArgs a) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ int abort_flag;
    // the 128-byte swizzle is applied to absolute shared addresses: slots start on 1024 bytes
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kBarOffset);
    Ring R{smem, bars, bars + kQSlots, bars + 2 * kQSlots, bars + 2 * kQSlots + kXSlots, &abort_flag,
           a.timeout_ns};
    uint64_t *uqfull = bars + 2 * kQSlots + 2 * kXSlots;  // [kUQ] a claimed unit is in the queue
    uint64_t *uqempty = uqfull + kUQ;                     // [kUQ] consumers and tensor-core warp have read it
    uint64_t *dfull = uqempty + kUQ;                      // [2] sweep-A accumulator buffer ready
    uint64_t *dfree = dfull + 2;                          // [2] sweep-A accumulator buffer read
    uint64_t *bfull = dfree + 2, *bfree = bfull + 1;      // sweep-B accumulators ready / read
    uint64_t *drain = bfree + 1;                          // every tensor-core operation done (exit)
    volatile long long *uq = reinterpret_cast<volatile long long *>(drain + 1);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1 + kUQ);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool producer = warp == kProducerWarp, mma_warp = warp == kMmaWarp;
    const bool consumer = warp < kConsumerWarps;
    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < kQSlots; ++s) {
            mbar_init(&R.full[s], 1);
            mbar_init(&R.empty[s], 1);  // tcgen05.commit of the instructions that read the slot
        }
        for (int s = 0; s < kXSlots; ++s) {
            mbar_init(&R.xfull[s], 1);
            mbar_init(&R.xempty[s], kConsumerWarps);
        }
        for (int s = 0; s < kUQ; ++s) {
            mbar_init(&uqfull[s], 1);
            mbar_init(&uqempty[s], kConsumerWarps + 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&dfull[s], 1);
            mbar_init(&dfree[s], kConsumerWarps);
        }
        mbar_init(bfull, 1);
        mbar_init(bfree, kConsumerWarps);
        mbar_init(drain, 1);
        fence_mbar_init_cluster();
    }
    if (mma_warp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "n"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t *>(tmem_slot);
    const uint64_t policy = l2_policy(a.l2);
    Cursor cur;
    uint32_t uk = 0;   // units handed over so far (same count in every role)
    uint32_t mc = 0;   // sweep-A accumulations (machines) so far (tensor-core warp and consumers)
    uint32_t ubc = 0;  // sweep-B units so far (tensor-core warp and consumers)
    bool ok = true;

    // The units of one launch form one stream: iteration it is the sweep-A
    // units of every system (system-major), then the sweep-B units.  The
    // CTAs claim from it with one counter.  The producer claims ahead of the
    // other roles, waits until the units of the same system that write the
    // unit's inputs are complete (sweep A of iteration it: sweep A of it - 1
    // (x_i, xbar) and sweep B of it - 1 (z); sweep B of it: sweep A of it
    // (xbar')), then hands the unit over through a small queue, so the ring
    // keeps streaming across unit boundaries and across sweeps; systems are
    // independent, so no grid-wide barrier separates the sweeps.  Every
    // dependency lies earlier in the stream and every CTA takes its units in
    // stream order, so the earliest incomplete unit can always proceed.  A
    // claim past the end hands over -1 and ends the stream.
    // Reverse sweep (kAdj): step it is its sweep-B units (v = Q^T mu), then its
    // sweep-A units (sum_i Q_i v_i and the row update); `iters` steps and a
    // last sweep B for the initialisation's term.  Sweep B of step it needs
    // sweep A of it - 1 (mu), sweep A of it needs sweep B of it (v).
    const long long per_it = (long long)a.nA + a.nB;
    const long long total = kAdj ? ((long long)a.iters + 1) * per_it - a.nA : (long long)a.iters * per_it;
    struct Unit {
        long long it;
        bool is_a, init, hb, edge;  // edge: last step's sweep A / final sweep B of a reverse sweep
        int2 U;                     // (system, first row or column | part << 24)
        int pos, part;
    };
    auto decode = [&](long long g) {
        Unit u;
        u.it = g / per_it;
        const int r = int(g - u.it * per_it);
        if constexpr (kAdj) {
            u.is_a = r >= a.nB;
            u.U = u.is_a ? a.unitsA[r - a.nB] : a.unitsB[r];
            u.init = false;
            u.hb = true;
            u.edge = u.is_a ? u.it + 1 == a.iters : u.it == a.iters;
        } else {
            u.is_a = r < a.nA;
            u.U = u.is_a ? a.unitsA[r] : a.unitsB[r - a.nA];
            u.init = a.init && u.it == 0;
            u.hb = a.hb && !u.init;
            u.edge = false;
        }
        u.pos = u.U.y & 0xFFFFFF;
        u.part = u.U.y >> 24;
        return u;
    };
    auto run = [&]() {
        if (producer) {
            if (lane != 0) return;
            for (;;) {
                const int s = int(uk % kUQ);
                long long g = -1;
                if (uk < uint32_t(kUQ) || R.wait(&uqempty[s], ((uk / kUQ) - 1) & 1)) {
                    g = (long long)atomicAdd(a.claim, 1ull);
                    if (g >= total) g = -1;
                }
                Unit u = {};
                if (g >= 0) {
                    u = decode(g);
                    const SysDesc &d = a.sys[u.U.x];
                    // completions are counted per consumer warp: kConsumerWarps per unit
                    const unsigned long long na = (unsigned long long)kConsumerWarps * unsigned(d.nuA);
                    const unsigned long long nb = (unsigned long long)kConsumerWarps * unsigned(d.nuB);
                    const unsigned long long it = (unsigned long long)u.it, sk = a.barrier_skew;
                    const unsigned long long *dn = a.done + 2 * u.U.x;
                    bool ready;
                    if constexpr (kAdj)
                        ready = u.is_a ? wait_count(dn + 1, (it + 1) * nb + sk, a, &abort_flag)
                                       : wait_count(dn, it * na + sk, a, &abort_flag);
                    else
                        ready = u.is_a ? wait_count(dn, it * na + sk, a, &abort_flag) &&
                                             wait_count(dn + 1, it * nb + sk, a, &abort_flag)
                                       : wait_count(dn, (it + 1) * na + sk, a, &abort_flag);
                    if (ready) __threadfence();
                    else g = -1;
                }
                uq[s] = g;
                mbar_arrive(&uqfull[s]);
                ++uk;
                if (g < 0) return;
                const SysDesc &d = a.sys[u.U.x];
                if (u.is_a)
                    sweep_a_producer<MT, kSplit>(R, cur, d, u.pos, u.part, a.rowsA, a.prefetch, u.init || u.hb, policy);
                else
                    sweep_b_producer<MT, kSplit>(R, cur, d, u.pos, u.part, a.colsB, policy);
            }
        } else if (mma_warp) {
            // the whole warp, converged: its MMAs and commits are issued by one
            // elected lane, with warp-uniform operands and waits
            int prev = -1;  // sweep of the previous unit (0: A, 1: B)
            for (;;) {
                const int s = int(uk % kUQ);
                if (!wait_w(R, &uqfull[s], (uk / kUQ) & 1)) return;
                const long long g = uq[s];
                __syncwarp();  // every lane has read the entry before it is released
                if (lane == 0) mbar_arrive(&uqempty[s]);
                ++uk;
                if (g < 0) return;
                const Unit u = decode(g);
                const SysDesc &d = a.sys[u.U.x];
                // sweep A's two accumulator buffers and sweep B's accumulators
                // share tensor memory: a change of sweep waits until the
                // consumers have read the other sweep's accumulators
                if (u.is_a && prev == 1) {
                    if (!wait_w(R, bfree, (ubc - 1) & 1)) return;
                    tc_fence_after();
                } else if (!u.is_a && prev == 0) {
                    for (uint32_t j = mc >= 2 ? mc - 2 : 0; j < mc; ++j)
                        if (!wait_w(R, &dfree[j & 1], (j >> 1) & 1)) return;
                    tc_fence_after();
                }
                prev = u.is_a ? 0 : 1;
                if (u.is_a) sweep_a_mma<MT, kSplit>(R, cur, mc, dfull, dfree, d, u.pos, u.part, a.rowsA, u.hb, tmem);
                else sweep_b_mma<MT, kSplit>(R, cur, ubc, bfull, bfree, d, u.pos, u.part, a.colsB, tmem);
            }
        } else {
            for (;;) {
                const int s = int(uk % kUQ);
                if (!R.wait(&uqfull[s], (uk / kUQ) & 1)) return;
                const long long g = uq[s];
                __syncwarp();
                if (lane == 0) mbar_arrive(&uqempty[s]);
                ++uk;
                if (g < 0) return;
                const Unit u = decode(g);
                const SysDesc &d = a.sys[u.U.x];
                if (u.is_a)
                    sweep_a_consumer<MT, kAdj, kSplit>(R, cur, mc, dfull, dfree, d, u.pos, u.part, a.rowsA, u.init,
                                                       u.hb, u.init ? 1.0f : d.g_hi, u.init ? 0.0f : d.g_lo, tmem,
                                                       u.edge);
                else
                    sweep_b_consumer<MT, kAdj, kSplit>(R, ubc, bfull, bfree, d, u.pos, u.part, a.colsB, tmem, u.edge);
                __syncwarp();
                if (*reinterpret_cast<volatile int *>(&abort_flag)) return;
                // the unit's global writes are read by other CTAs (bulk
                // copies and loads): publish them, one arrival per warp
                fence_proxy_async_global();
                __threadfence();
                __syncwarp();
                if (lane == 0) red_release_add_u64(a.done + 2 * u.U.x + (u.is_a ? 0 : 1), 1ull);
            }
        }
    };

    if (!kAdj && a.init) {
        // z_i(0) = -c_i, so that sweep A with gamma = 1 and x = xbar = 0 forms
        // the least-norm x_i(0) = Q_i c_i (Algorithm 1) and xbar(0) their mean
        if (consumer)
            for (int u = blockIdx.x; u < a.nB; u += gridDim.x) {
                const int2 U = a.unitsB[u];
                if ((U.y >> 24) != 0) continue;  // the columns once, not once per part
                const int col0 = U.y & 0xFFFFFF;
                const SysDesc &d = a.sys[U.x];
                const int ncols = min(a.colsB, d.Cq - col0);
                for (int hh = 0; hh < 2; ++hh) {
                    const int cl = 128 * ((warp >> 2) + 2 * hh) + 32 * (warp & 3);
                    if (cl < ncols) {
                        float Y[16 * MT] = {};
                        store_z<MT>(d, col0 + cl + lane, Y, true);
                    }
                }
            }
        ok = grid_barrier(a.bar, gridDim.x + a.barrier_skew, a.timeout_ns, &abort_flag);
    }
    if (ok) run();
    // no bulk copy may still be writing this CTA's shared memory and no
    // tensor-core operation may still be using tensor memory at exit: the
    // producer waits (bounded) for the last phase of every slot it filled, the
    // tensor-core warp for a final commit
    __syncthreads();
    if (producer && lane == 0) {
        for (uint32_t q = cur.q > uint32_t(kQSlots) ? cur.q - kQSlots : 0; q < cur.q; ++q)
            (void)mbar_wait(&R.full[q % kQSlots], (q / kQSlots) & 1, a.timeout_ns);
        for (uint32_t x = cur.x > uint32_t(kXSlots) ? cur.x - kXSlots : 0; x < cur.x; ++x)
            (void)mbar_wait(&R.xfull[x % kXSlots], (x / kXSlots) & 1, a.timeout_ns);
    }
    if (mma_warp) {
        tc_commit_w(drain);  // the elected lane is the one that issued the MMAs
        if (lane == 0) (void)mbar_wait(drain, 0, a.timeout_ns);
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (mma_warp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(kTmemCols) : "memory");
    if (threadIdx.x == 0 && abort_flag) atomicCAS(a.err, 0, DEV_TIMEOUT_GRID);
}

// ---- set-up kernels -----------------------------------------------------------------
// QB (qb_block) from Q (q_block): block b copies piece (row group b / (Cq/64),
// window b % (Cq/64)), 4 KB, as 256 x 16 bytes
__global__ void qb_permute_kernel(const __nv_bfloat16 *Q, int npad, int Cq, __nv_bfloat16 *QB) {
    const int nw = Cq / kWin;
    const int G = int(blockIdx.x) / nw, w = int(blockIdx.x) % nw;
    const int t = G * 32 / kTileRows, rr = G * 32 % kTileRows;
    const uint4 *src = reinterpret_cast<const uint4 *>(Q + q_block(Cq, npad, t, w) + size_t(rr) * kWin);
    uint4 *dst = reinterpret_cast<uint4 *>(QB + qb_block(Cq, G, w));
    dst[threadIdx.x] = src[threadIdx.x];
}

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
// FP32 into Ct[rhs][column] (Cq columns per right-hand side).
__global__ void batch_coef_kernel(const double *B, int k, const int64_t *row_start, const int32_t *pcount,
                                  const double *dinv, const double *Rinv1, const double *Rinv2, int P,
                                  const int *coloff, int Cq, float *Ct) {
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
        Ct[size_t(rhs) * Cq + coloff[b] + c] = float(s);
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
        const size_t off = x_block(x_blocks(npad), kp, j / kXRows, worker) + size_t(r) * kXRows + j % kXRows;
        out[int64_t(j) * ldx + r] = double(X[off]);
    }
}

// Start of the reverse sweep for one system: lbar = g (double-float), ell = 0,
// and the three BF16 planes of mu = coef * g (the B operand of sweep B, layout
// of store_xop), zero on padded rows and right-hand sides.  G is n x k, ld k.
__global__ void adj_seed_kernel(const double *G, int64_t n, int k, int kp, int npad, double coef, float2 *Xb,
                                float2 *Mb, uint8_t *Xop) {
    const int NB = kPlanesB * kp;
    const int64_t total = int64_t(npad) * kp;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int q = int(i / npad);
        const int64_t j = i - int64_t(q) * npad;
        const double gv = (j < n && q < k) ? G[j * k + q] : 0.0;
        const float hi = float(gv);
        Xb[size_t(q) * npad + j] = make_float2(hi, float(gv - double(hi)));
        Mb[size_t(q) * npad + j] = make_float2(0.0f, 0.0f);
        float x = float(coef * gv);
        for (int p = 0; p < kPlanesB; ++p) {
            const __nv_bfloat16 v = __float2bfloat16_rn(x);
            x -= __bfloat162float(v);
            *reinterpret_cast<__nv_bfloat16 *>(Xop + op_offset(NB, p * kp + q, j)) = v;
        }
    }
}

// End of the reverse sweep: dL/db_b = d .* (R1inv_b (R2inv_b dL/dc_b)) (the
// transpose of c_b = R2inv_b^T R1inv_b^T (d .* b_b), batch_coef_kernel), one
// block and right-hand side per CTA, FP64; DB is n x k, ld k.
__global__ void batch_grad_kernel(const float *Gc, int Cq, const int *coloff, const int64_t *row_start,
                                  const int32_t *pcount, const double *dinv, const double *Rinv1,
                                  const double *Rinv2, int P, int k, double *DB) {
    extern __shared__ double sh[];  // g[P], w[P]
    const int b = blockIdx.x, rhs = blockIdx.y;
    const int p = pcount[b];
    const int64_t r0 = row_start[b];
    const double *R1 = Rinv1 + size_t(b) * P * P, *R2 = Rinv2 + size_t(b) * P * P;
    double *g = sh, *w = sh + P;
    for (int c = threadIdx.x; c < P; c += blockDim.x) g[c] = c < p ? double(Gc[size_t(rhs) * Cq + coloff[b] + c]) : 0.0;
    __syncthreads();
    for (int r = threadIdx.x; r < p; r += blockDim.x) {
        double acc = 0.0;
        for (int c = r; c < p; ++c) acc = fma(R2[size_t(r) * P + c], g[c], acc);
        w[r] = acc;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < p; r += blockDim.x) {
        double acc = 0.0;
        for (int c = r; c < p; ++c) acc = fma(R1[size_t(r) * P + c], w[c], acc);
        DB[(r0 + r) * k + rhs] = dinv[r0 + r] * acc;
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
    int rowsA = 256, colsB = 512, prefetch = 2;  // unit shape (apc_batch_set_tiles)
    int l2 = 0;                                  // L2 policy of the bulk copies (apc_batch_set_tiles)
    int splitA = 1, splitB = 1;                  // parts per unit (apc_batch_set_tiles)
    int split_cap_a = 1, split_cap_b = 1;        // parts the Spart / Ypart buffers hold
    std::vector<void *> split_bufs;              // Spart / Ypart of every system
    int *cnt = nullptr;                          // split-part counters of all systems
    size_t cnt_count = 0;
    std::vector<apc_ctx *> ctx;
    std::vector<SysDesc> desc;
    std::vector<int64_t> n;
    std::vector<int> m;
    std::vector<double *> B;  // FP64 right-hand sides (kept for apc_batch_reset)
    std::vector<void *> owned;
    SysDesc *d_desc = nullptr;
    int2 *d_unitsA = nullptr, *d_unitsB = nullptr;
    // launch counters, zeroed before every launch: [0] grid barrier (32 bit),
    // [1] units claimed, [2 + 2 s], [3 + 2 s] completions of system s (64 bit)
    unsigned long long *ctr = nullptr;
    int *err = nullptr;
    bool reset_done = false, params_set = false;
    int method = 0;  // 0: APC, 1: heavy ball (apc_batch_set_hb_params)
    int64_t q_bytes = 0, state_bytes = 0;
    double timeout_s = 2.0;
    uint32_t barrier_skew = 0;
    cudaGraphExec_t graph = nullptr;  // forward launch (APC or heavy ball)
    int64_t graph_iters = -1;
    int graph_method = -1;            // method of the captured forward launch
    cudaGraphExec_t graph_adj = nullptr;  // reverse sweep (apc_batch_backward)
    int64_t graph_adj_iters = -1;
    std::vector<double> eta;  // eta_s of apc_batch_set_params (the reverse sweep's seed)
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

template <int MT>
const void *kernel_ptr_mt(bool adj, bool split) {
    if (adj)
        return split ? reinterpret_cast<const void *>(&apc_batch_kernel<MT, true, true>)
                     : reinterpret_cast<const void *>(&apc_batch_kernel<MT, true, false>);
    return split ? reinterpret_cast<const void *>(&apc_batch_kernel<MT, false, true>)
                 : reinterpret_cast<const void *>(&apc_batch_kernel<MT, false, false>);
}
const void *kernel_ptr(int MT, bool adj, bool split) {
    return MT == 1 ? kernel_ptr_mt<1>(adj, split) : kernel_ptr_mt<2>(adj, split);
}

// Units sorted by decreasing key, equal keys in insertion order; the CTAs
// claim them in this order at run time.
std::vector<int2> by_key_desc(std::vector<std::pair<double, int2>> items) {
    using Item = std::pair<double, int2>;
    std::stable_sort(items.begin(), items.end(), [](const Item &x, const Item &y) { return x.first > y.first; });
    std::vector<int2> units;
    units.reserve(items.size());
    for (const auto &it : items) units.push_back(it.second);
    return units;
}

int launch(apc_batch *b, int init, int64_t iters, cudaStream_t s, bool adj = false) {
    BatchArgs a = {};
    a.sys = b->d_desc;
    a.unitsA = b->d_unitsA;
    a.unitsB = b->d_unitsB;
    a.nA = b->units_a;
    a.nB = b->units_b;
    a.claim = b->ctr + 1;
    a.done = b->ctr + 2;
    a.iters = iters;
    a.init = init;
    a.hb = init || adj ? 0 : b->method;
    a.adj = adj ? 1 : 0;
    a.rowsA = b->rowsA;
    a.colsB = b->colsB;
    a.prefetch = b->prefetch;
    a.l2 = b->l2;
    a.barrier_skew = b->barrier_skew;
    a.bar = reinterpret_cast<uint32_t *>(b->ctr);
    a.err = b->err;
    a.timeout_ns = uint64_t(b->timeout_s * 1e9);
    BCK(b, cudaMemsetAsync(b->ctr, 0, sizeof(unsigned long long) * (2 + 2 * size_t(b->nsys)), s));
    const bool split = b->splitA > 1 || b->splitB > 1;
    if (split) BCK(b, cudaMemsetAsync(b->cnt, 0, sizeof(int) * b->cnt_count, s));
    void *args[] = {&a};
    BCK(b, cudaLaunchKernel(kernel_ptr(b->MT, adj, split), dim3(b->grid), dim3(kThreads), args, kSmemBytes, s));
    return APC_OK;
}

int check_err(apc_batch *b, cudaStream_t s) {
    int h = 0;
    BCK(b, cudaMemcpyAsync(&h, b->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    BCK(b, cudaStreamSynchronize(s));
    if (h) {
        BCK(b, cudaMemsetAsync(b->err, 0, sizeof(int), s));
        BCK(b, cudaStreamSynchronize(s));
        return bfail(b, APC_ERR_TIMEOUT, "a wait on another CTA's work ran out of time (%.3g s)", b->timeout_s);
    }
    return APC_OK;
}

// One persistent launch (counter reset + kernel) of `iters` iterations, or of
// a reverse sweep through `iters` steps, captured once per (count, method)
// and replayed as a CUDA graph; then the device error flag is read.
int run_graph(apc_batch *b, int64_t iters, bool adj, cudaStream_t s) {
    cudaGraphExec_t &exec = adj ? b->graph_adj : b->graph;
    const bool stale = adj ? b->graph_adj_iters != iters : (b->graph_iters != iters || b->graph_method != b->method);
    if (!exec || stale) {
        if (exec) {
            cudaGraphExecDestroy(exec);
            exec = nullptr;
        }
        cudaStream_t cs;
        BCK(b, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        const int rc = e == cudaSuccess ? launch(b, 0, iters, cs, adj) : APC_ERR_CUDA;
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (rc == APC_OK && e2 == cudaSuccess) e2 = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess || rc != APC_OK || e2 != cudaSuccess) {
            cudaGetLastError();
            exec = nullptr;
            return bfail(b, APC_ERR_CUDA, "graph capture of the batched launch failed");
        }
        if (adj) {
            b->graph_adj_iters = iters;
        } else {
            b->graph_iters = iters;
            b->graph_method = b->method;
        }
    }
    BCK(b, cudaGraphLaunch(exec, s));
    return check_err(b, s);
}

// Work lists for the current unit shape, system-major: the systems with the
// most bytes first, each system's units together (stable sort on the
// system's bytes); the per-system unit counts go to the descriptors.
int build_units(apc_batch *b, cudaStream_t s) {
    std::vector<std::pair<double, int2>> ia, ib;
    for (int sys = 0; sys < b->nsys; ++sys) {
        SysDesc &d = b->desc[sys];
        // parts: machines of a sweep-A unit in groups of ceil(m / splitA);
        // rows of a sweep-B unit in chunks of a multiple of 64 rows (no part empty)
        const int mchunk = (d.m + b->splitA - 1) / b->splitA;
        d.spA = (d.m + mchunk - 1) / mchunk;
        d.chunkB = ((d.npad + b->splitB - 1) / b->splitB + 63) / 64 * 64;
        d.spB = (d.npad + d.chunkB - 1) / d.chunkB;
        d.nuA = (d.npad + b->rowsA - 1) / b->rowsA * d.spA;
        d.nuB = (d.Cq + b->colsB - 1) / b->colsB * d.spB;
        const double bytes = double(d.npad) * (4.0 * d.Cq + 8.0 * d.m * b->kp);
        for (int r0 = 0; r0 < d.npad; r0 += b->rowsA)
            for (int p = 0; p < d.spA; ++p) ia.push_back({bytes, make_int2(sys, r0 | (p << 24))});
        for (int c0 = 0; c0 < d.Cq; c0 += b->colsB)
            for (int p = 0; p < d.spB; ++p) ib.push_back({bytes, make_int2(sys, c0 | (p << 24))});
    }
    const std::vector<int2> ua = by_key_desc(ia), ub = by_key_desc(ib);
    b->units_a = int(ua.size());
    b->units_b = int(ub.size());
    BCK(b, cudaMemcpyAsync(b->d_unitsA, ua.data(), sizeof(int2) * ua.size(), cudaMemcpyHostToDevice, s));
    BCK(b, cudaMemcpyAsync(b->d_unitsB, ub.data(), sizeof(int2) * ub.size(), cudaMemcpyHostToDevice, s));
    BCK(b, cudaMemcpyAsync(b->d_desc, b->desc.data(), sizeof(SysDesc) * b->nsys, cudaMemcpyHostToDevice, s));
    BCK(b, cudaStreamSynchronize(s));
    return APC_OK;
}

int compute_coefficients(apc_batch *b, int sys, cudaStream_t s) {
    apc_ctx *c = b->ctx[sys];
    const SysDesc &d = b->desc[sys];
    float *Ct = const_cast<float *>(d.Ct);
    BCK(b, cudaMemsetAsync(Ct, 0, sizeof(float) * size_t(b->kp) * d.Cq, s));
    const size_t sh = sizeof(double) * 2 * c->P;
    batch_coef_kernel<<<dim3(unsigned(c->m), unsigned(b->k)), 128, sh, s>>>(
        b->B[sys], b->k, c->d_rowstart, c->d_p, c->dinv, c->Rinv1, c->Rinv2, c->P, d.coloff, d.Cq, Ct);
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
    // sweep B's copy of the bases (qb_block) when all packed bases together
    // exceed twice the L2 cache
    bool use_qb = false;
    {
        int l2 = 0;
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, b->device);
        int64_t total = 0;
        const int64_t *o = row_offsets_host;
        for (int sys = 0; sys < nsys; ++sys) {
            const int m = m_host[sys];
            if (m < 1) break;  // rejected in the loop below
            int64_t C = 0;
            for (int i = 0; i < m; ++i) C += (o[i + 1] - o[i] + 15) / 16 * 16;
            total += int64_t(2) * ((n_host[sys] + 31) / 32 * 32) * ((C + kWin - 1) / kWin * kWin);
            o += m + 1;
        }
        use_qb = l2 > 0 && total > int64_t(2) * l2;
    }
    for (int sys = 0; sys < nsys; ++sys) {
        const int64_t n = n_host[sys];
        const int m = m_host[sys];
        if (n < 1 || m < 1 || n > (int64_t(1) << 24) || !A_dev_host[sys] || !B_dev_host[sys] || offs[0] != 0 ||
            offs[m] != n) {
            bfail(b, APC_ERR_INVALID_ARG, "system %d: bad size, pointer or offsets", sys);
            return bail(APC_ERR_INVALID_ARG);
        }
        // FP64 set-up of the single-system solver: row scaling and Cholesky QR
        // per block (Sec. 3.3); Q_i rounded to BF16 once
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
        apc_options o = {APC_BF16, 0, 0, b->timeout_s, 0};
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
        const int nxblocks = int((npad + kXRows - 1) / kXRows);
        std::vector<int> colblk(Cq / 16, -1);
        for (int i = 0; i < m; ++i)
            for (int g16 = co[i] / 16; g16 < co[i + 1] / 16; ++g16) colblk[g16] = i;
        SysDesc d = {};
        d.npad = int(npad);
        d.m = m;
        d.Cq = Cq;
        d.C = C;
        const size_t x_elems = x_block(nxblocks, kp, 0, m);
        int *d_co = nullptr, *d_cb = nullptr;
        __nv_bfloat16 *Q = nullptr, *QB = nullptr;
        float *Cf = nullptr;
        double *Bc = nullptr;
        if ((rc = balloc(b, &d_co, sizeof(int) * (m + 1))) || (rc = balloc(b, &d_cb, sizeof(int) * (Cq / 16))) ||
            (rc = balloc(b, &Q, sizeof(__nv_bfloat16) * size_t(npad) * Cq)) ||
            (use_qb && (rc = balloc(b, &QB, sizeof(__nv_bfloat16) * size_t(npad) * Cq))) ||
            (rc = balloc(b, &d.X, sizeof(float) * x_elems)) ||
            (rc = balloc(b, &d.Xb, sizeof(float2) * size_t(kp) * npad)) ||
            (rc = balloc(b, &d.Xop, size_t(npad) * kPlanesB * kp * 2)) ||
            (rc = balloc(b, &d.Zop, size_t(Cq) * kPlanesA * kp * 2)) ||
            (rc = balloc(b, &Cf, sizeof(float) * size_t(kp) * Cq)) ||
            (rc = balloc(b, &d.Mb, sizeof(float2) * size_t(kp) * npad)) ||
            (rc = balloc(b, &Bc, sizeof(double) * size_t(n) * k)))
            return bail(rc);
        d.Q = Q;
        d.QB = QB;
        d.Ct = Cf;
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
        cudaMemsetAsync(d.Xop, 0, size_t(npad) * kPlanesB * kp * 2, s);
        cudaMemsetAsync(d.Zop, 0, size_t(Cq) * kPlanesA * kp * 2, s);
        const unsigned grid = unsigned(std::min<int64_t>((npad * Cq + 255) / 256, 152 * 32));
        repack_kernel<<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(c->Q), n, m, c->P, d_cb, d_co, c->d_p,
                                           int(npad), Cq, Q);
        if (use_qb) qb_permute_kernel<<<unsigned(npad / 32 * (Cq / kWin)), 256, 0, s>>>(Q, int(npad), Cq, QB);
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
    if ((rc = balloc(b, &b->d_desc, sizeof(SysDesc) * nsys)) ||
        (rc = balloc(b, &b->ctr, sizeof(unsigned long long) * (2 + 2 * size_t(nsys)))) ||
        (rc = balloc(b, &b->err, sizeof(int) * 4)))
        return bail(rc);
    if (cudaMemsetAsync(b->err, 0, sizeof(int) * 4, s) != cudaSuccess) {
        bfail(b, APC_ERR_CUDA, "memset failed");
        return bail(APC_ERR_CUDA);
    }
    // one CTA per SM, all resident at once (the CTAs wait on one another's units)
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    bool resident = true;
    for (int v = 0; v < 4 && resident; ++v) {
        const void *k = kernel_ptr(MT, v & 1, v & 2);
        per_sm = 0;
        resident = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmemBytes)) == cudaSuccess &&
                   cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, kSmemBytes) == cudaSuccess &&
                   per_sm >= 1;
    }
    if (!resident) {
        cudaGetLastError();
        bfail(b, APC_ERR_LAUNCH, "the batched kernel cannot be resident (%zu bytes of shared memory)", kSmemBytes);
        return bail(APC_ERR_LAUNCH);
    }
    b->grid = sms;
    // work lists, sized for the smallest units and the most parts (the tile
    // tuner may pick them), and the split-part counters
    size_t max_a = 0, max_b = 0;
    for (const SysDesc &d : b->desc) {
        max_a += size_t((d.npad + kXRows - 1) / kXRows) * kMaxSplit;
        max_b += size_t((d.Cq + 127) / 128) * kMaxSplit;
        b->cnt_count += size_t((d.npad + kXRows - 1) / kXRows) * kConsumerWarps +
                        size_t((d.Cq + 127) / 128) * kConsumerWarps * 2;
    }
    if ((rc = balloc(b, &b->d_unitsA, sizeof(int2) * max_a)) || (rc = balloc(b, &b->d_unitsB, sizeof(int2) * max_b)) ||
        (rc = balloc(b, &b->cnt, sizeof(int) * b->cnt_count)))
        return bail(rc);
    {
        size_t off = 0;
        for (SysDesc &d : b->desc) {
            d.cntA = b->cnt + off;
            off += size_t((d.npad + kXRows - 1) / kXRows) * kConsumerWarps;
            d.cntB = b->cnt + off;
            off += size_t((d.Cq + 127) / 128) * kConsumerWarps * 2;
        }
    }
    if ((rc = build_units(b, s)) != APC_OK) return bail(rc);
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
        split_f64(1.0 - g, d.omg_hi, d.omg_lo);
        split_f64(g * b->m[sys], d.gm_hi, d.gm_lo);
    }
    BCK(b, cudaMemcpy(b->d_desc, b->desc.data(), sizeof(SysDesc) * b->nsys, cudaMemcpyHostToDevice));
    b->eta.assign(eta_host, eta_host + b->nsys);
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
    return run_graph(b, iters, false, static_cast<cudaStream_t>(stream));
}

int apc_batch_set_tiles(apc_batch *b, int32_t rows_a, int32_t cols_b, int32_t prefetch, int32_t l2, int32_t split_a,
                        int32_t split_b) {
    if (!b) return bfail(b, APC_ERR_INVALID_ARG, "NULL batch");
    auto pow2 = [](int v) { return v >= 1 && v <= kMaxSplit && (v & (v - 1)) == 0; };
    if ((rows_a != kXRows && rows_a != kTileRows) || (cols_b != 128 && cols_b != 256 && cols_b != kColsB) ||
        prefetch < 0 || prefetch > 8 || l2 < 0 || l2 > 2 || !pow2(split_a) || !pow2(split_b))
        return bfail(b, APC_ERR_INVALID_ARG,
                     "tiles: rows_a in {128, 256}, cols_b in {128, 256, 512}, prefetch 0..8, l2 0..2, splits 1, 2, 4 "
                     "or 8");
    if (rows_a == b->rowsA && cols_b == b->colsB && prefetch == b->prefetch && l2 == b->l2 && split_a == b->splitA &&
        split_b == b->splitB)
        return APC_OK;
    BCK(b, cudaDeviceSynchronize());  // no launch may still read the work lists
    if (split_a > b->split_cap_a || split_b > b->split_cap_b) {
        // partial sums of the parts: [parts][kp][npad] (sweep A), [parts][kp][Cq] (sweep B)
        for (void *p : b->split_bufs) cudaFree(p);
        b->split_bufs.clear();
        const int ca = std::max(split_a, b->split_cap_a), cb = std::max(split_b, b->split_cap_b);
        for (SysDesc &d : b->desc) {
            void *pa = nullptr, *pb = nullptr;
            if (cudaMalloc(&pa, sizeof(float) * size_t(ca) * b->kp * d.npad) != cudaSuccess ||
                cudaMalloc(&pb, sizeof(float) * size_t(cb) * b->kp * d.Cq) != cudaSuccess) {
                cudaGetLastError();
                if (pa) cudaFree(pa);
                for (void *p : b->split_bufs) cudaFree(p);
                b->split_bufs.clear();
                for (SysDesc &e : b->desc) e.Spart = e.Ypart = nullptr;
                b->split_cap_a = b->split_cap_b = 1;
                b->splitA = b->splitB = 1;
                build_units(b, nullptr);
                return bfail(b, APC_ERR_NOMEM, "buffers of the split units");
            }
            b->split_bufs.push_back(pa);
            b->split_bufs.push_back(pb);
            d.Spart = static_cast<float *>(pa);
            d.Ypart = static_cast<float *>(pb);
        }
        b->split_cap_a = ca;
        b->split_cap_b = cb;
    }
    b->rowsA = rows_a;
    b->colsB = cols_b;
    b->prefetch = prefetch;
    b->l2 = l2;
    b->splitA = split_a;
    b->splitB = split_b;
    for (cudaGraphExec_t *g : {&b->graph, &b->graph_adj})
        if (*g) {
            cudaGraphExecDestroy(*g);
            *g = nullptr;
        }
    return build_units(b, nullptr);
}

int apc_batch_get_tiles(const apc_batch *b, int32_t *rows_a, int32_t *cols_b, int32_t *prefetch, int32_t *l2,
                        int32_t *split_a, int32_t *split_b) {
    if (!b) return APC_ERR_INVALID_ARG;
    if (rows_a) *rows_a = b->rowsA;
    if (cols_b) *cols_b = b->colsB;
    if (prefetch) *prefetch = b->prefetch;
    if (l2) *l2 = b->l2;
    if (split_a) *split_a = b->splitA;
    if (split_b) *split_b = b->splitB;
    return APC_OK;
}

int apc_batch_autotune(apc_batch *b, int64_t iters, int32_t reps, int32_t *tiles_out, double *ms_best,
                       double *ms_default, void *stream) {
    if (!b || iters < 1 || reps < 1) return bfail(b, APC_ERR_INVALID_ARG, "bad argument");
    if (!b->params_set || !b->reset_done)
        return bfail(b, APC_ERR_INVALID_ARG, "apc_batch_set_params and apc_batch_reset must precede the tuning");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    typedef std::array<int, 6> Tiles;  // rows_a, cols_b, prefetch, l2, split_a, split_b
    const Tiles dflt_t = {b->rowsA, b->colsB, b->prefetch, b->l2, b->splitA, b->splitB};
    Tiles best_t = dflt_t;
    double best = 1e300, dflt = -1.0;
    cudaEvent_t e0, e1;
    BCK(b, cudaEventCreate(&e0));
    BCK(b, cudaEventCreate(&e1));
    // time one choice: ms per iteration into *per
    auto time_tiles = [&](const Tiles &t, double *per) -> int {
        int rc = apc_batch_set_tiles(b, t[0], t[1], t[2], t[3], t[4], t[5]);
        if (rc == APC_OK) rc = run_graph(b, iters, false, s);  // capture and warm-up
        if (rc != APC_OK) return rc;
        if (cudaEventRecord(e0, s) != cudaSuccess) return APC_ERR_CUDA;
        for (int r = 0; r < reps; ++r)
            if (cudaGraphLaunch(b->graph, s) != cudaSuccess) return APC_ERR_CUDA;
        if (cudaEventRecord(e1, s) != cudaSuccess) return APC_ERR_CUDA;
        if ((rc = check_err(b, s)) != APC_OK) return rc;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        *per = double(ms) / double(reps * iters);
        if (t == dflt_t) dflt = *per;
        if (*per < best) {
            best = *per;
            best_t = t;
        }
        return APC_OK;
    };
    // stage 1: unit shapes with every split of their units over several
    // CTAs (the current prefetch distance and L2 policy); stage 2: the other
    // prefetch distances on the best; stage 3: the other L2 policies
    const int cand_a[] = {256, 128}, cand_b[] = {512, 256, 128}, cand_p[] = {0, 1, 2, 4}, cand_s[] = {1, 2, 4, 8};
    int rc = APC_OK;
    double per = 0.0;
    // splits only pay when a shape leaves SMs without units: a sweep's units
    // are multiplied by its split only while the unsplit count is below twice
    // the grid (many systems already give every SM several units)
    auto units = [&](int ra, int cb, int *na, int *nb) {
        *na = *nb = 0;
        for (const SysDesc &d : b->desc) {
            *na += (d.npad + ra - 1) / ra;
            *nb += (d.Cq + cb - 1) / cb;
        }
    };
    for (int ra : cand_a)
        for (int cb : cand_b) {
            int na = 0, nb = 0;
            units(ra, cb, &na, &nb);
            for (int sa : cand_s)
                for (int sb : cand_s) {
                    if ((sa > 1 && na >= 2 * b->grid) || (sb > 1 && nb >= 2 * b->grid)) continue;
                    if (rc == APC_OK) rc = time_tiles({ra, cb, dflt_t[2], dflt_t[3], sa, sb}, &per);
                }
        }
    const Tiles s1 = best_t;
    for (int pf : cand_p)
        if (rc == APC_OK && pf != s1[2]) rc = time_tiles({s1[0], s1[1], pf, s1[3], s1[4], s1[5]}, &per);
    const Tiles s2 = best_t;
    for (int l2m = 0; l2m <= 2 && rc == APC_OK; ++l2m)
        if (l2m != s2[3]) rc = time_tiles({s2[0], s2[1], s2[2], l2m, s2[4], s2[5]}, &per);
    if (rc == APC_OK && dflt < 0.0) rc = time_tiles(dflt_t, &per);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != APC_OK) {
        cudaGetLastError();
        apc_batch_set_tiles(b, dflt_t[0], dflt_t[1], dflt_t[2], dflt_t[3], dflt_t[4], dflt_t[5]);
        return rc == APC_ERR_CUDA ? bfail(b, rc, "tuning launch failed") : rc;
    }
    if ((rc = apc_batch_set_tiles(b, best_t[0], best_t[1], best_t[2], best_t[3], best_t[4], best_t[5])) != APC_OK)
        return rc;
    b->reset_done = false;  // the tuning advanced the iteration state
    if (tiles_out)
        for (int j = 0; j < 6; ++j) tiles_out[j] = best_t[j];
    if (ms_best) *ms_best = best;
    if (ms_default) *ms_default = dflt;
    return APC_OK;
}

int apc_batch_forward(apc_batch *b, const double *const *B_dev_host, int64_t T, double *const *X_dev_host,
                      void *stream) {
    if (!b || !X_dev_host || T < 0) return bfail(b, APC_ERR_INVALID_ARG, "bad argument");
    for (int sys = 0; sys < b->nsys; ++sys)
        if (!X_dev_host[sys]) return bfail(b, APC_ERR_INVALID_ARG, "system %d: NULL output", sys);
    if (!b->params_set || b->method != 0)
        return bfail(b, APC_ERR_PARAMS, "apc_batch_set_params must precede apc_batch_forward");
    int rc = apc_batch_reset(b, B_dev_host, stream);
    if (rc == APC_OK) rc = apc_batch_iterate(b, T, stream);
    for (int sys = 0; rc == APC_OK && sys < b->nsys; ++sys) rc = apc_batch_get_xbar(b, sys, X_dev_host[sys], b->k, stream);
    return rc;
}

int apc_batch_backward(apc_batch *b, const double *const *G_dev_host, int64_t T, double *const *DB_dev_host,
                       void *stream) {
    if (!b || !G_dev_host || !DB_dev_host || T < 0) return bfail(b, APC_ERR_INVALID_ARG, "bad argument");
    for (int sys = 0; sys < b->nsys; ++sys)
        if (!G_dev_host[sys] || !DB_dev_host[sys])
            return bfail(b, APC_ERR_INVALID_ARG, "system %d: NULL gradient or output", sys);
    if (!b->params_set || b->method != 0)
        return bfail(b, APC_ERR_PARAMS, "the reverse sweep needs APC parameters (apc_batch_set_params)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // dL/dc_i accumulators, allocated on first use
    if (!b->desc[0].Gc) {
        for (int sys = 0; sys < b->nsys; ++sys) {
            int rc = balloc(b, &b->desc[sys].Gc, sizeof(float) * size_t(b->kp) * b->desc[sys].Cq);
            if (rc != APC_OK) return rc;
        }
        BCK(b, cudaMemcpyAsync(b->d_desc, b->desc.data(), sizeof(SysDesc) * b->nsys, cudaMemcpyHostToDevice, s));
    }
    // lbar = g, ell = 0, dL/dc = 0, and the planes of mu = ell + (eta/m) lbar
    // (lbar/m for T = 0: the initialisation's term alone)
    for (int sys = 0; sys < b->nsys; ++sys) {
        const SysDesc &d = b->desc[sys];
        BCK(b, cudaMemsetAsync(d.Gc, 0, sizeof(float) * size_t(b->kp) * d.Cq, s));
        const double coef = (T == 0 ? 1.0 : b->eta[sys]) / b->m[sys];
        const unsigned grid = unsigned(std::min<int64_t>((int64_t(d.npad) * b->kp + 255) / 256, 152 * 16));
        adj_seed_kernel<<<grid, 256, 0, s>>>(G_dev_host[sys], b->n[sys], b->k, b->kp, d.npad, coef, d.Xb, d.Mb,
                                             d.Xop);
        BCK(b, cudaGetLastError());
    }
    b->reset_done = false;  // the iteration state now holds the reverse sweep
    int rc = run_graph(b, T, true, s);
    if (rc != APC_OK) return rc;
    for (int sys = 0; sys < b->nsys; ++sys) {
        apc_ctx *c = b->ctx[sys];
        const SysDesc &d = b->desc[sys];
        const size_t sh = sizeof(double) * 2 * c->P;
        batch_grad_kernel<<<dim3(unsigned(c->m), unsigned(b->k)), 128, sh, s>>>(
            d.Gc, d.Cq, d.coloff, c->d_rowstart, c->d_p, c->dinv, c->Rinv1, c->Rinv2, c->P, b->k, DB_dev_host[sys]);
        BCK(b, cudaGetLastError());
    }
    return APC_OK;
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
    for (cudaGraphExec_t *g : {&b->graph, &b->graph_adj})
        if (*g) {
            cudaGraphExecDestroy(*g);
            *g = nullptr;
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

}  // extern "C"

// ---- k right-hand sides through a single-system context ------------------------

namespace {

int cfail(apc_ctx *c, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->last_error = buf;
    apc::set_global_error_text(buf);
    return code;
}

#define CCK(c, call)                                                                                     \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess) return cfail((c), APC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// The tensor-core form applies to a BF16 context of a square system with
// contiguous blocks and 2..32 right-hand sides; other contexts take the
// columns one after another through the single-system kernel.
bool use_tensor_cores(const apc_ctx *c, int64_t k) {
    return c->precision == APC_BF16 && c->N == c->n && !c->d_perm && k >= 2 && k <= 32;
}

// The context's one-system batch for k right-hand sides (built on first use,
// rebuilt when k changes) with (gamma, eta) set.
int multi_rhs_batch(apc_ctx *c, int64_t k, double gamma, double eta, cudaStream_t s) {
    if (!c->mrhs || c->mrhs_k != k) {
        apc::destroy_multi_rhs(c);
        if (cudaMalloc(&c->mrhs_in, sizeof(double) * c->n * k) != cudaSuccess ||
            cudaMalloc(&c->mrhs_out, sizeof(double) * c->N * k) != cudaSuccess) {
            cudaGetLastError();
            apc::destroy_multi_rhs(c);
            return cfail(c, APC_ERR_NOMEM, "staging buffers for %lld right-hand sides", (long long)k);
        }
        CCK(c, cudaMemsetAsync(c->mrhs_in, 0, sizeof(double) * c->n * k, s));
        const int64_t n = c->n;
        const int32_t m = c->m;
        const double *A = c->A;
        const double *B = c->mrhs_in;
        apc_options o = {APC_BF16, 0, 0, c->timeout_s, 0};
        const int rc = apc_batch_setup(&c->mrhs, 1, &n, &m, c->offs.data(), &A, &B, int32_t(k), &o, s);
        if (rc != APC_OK) {
            c->mrhs = nullptr;
            apc::destroy_multi_rhs(c);
            return cfail(c, rc, "%s", apc_batch_last_error(nullptr));
        }
        c->mrhs_k = int(k);
        // one system: units split over four CTAs each give the SMs work (the
        // tile tuner's choice for an 8192 system, k = 16: 0.11 ms per iteration
        // against 0.35 ms with the many-system default)
        const int rc2 = apc_batch_set_tiles(c->mrhs, 256, 256, 1, 0, 4, 4);
        if (rc2 != APC_OK) return cfail(c, rc2, "%s", apc_batch_last_error(c->mrhs));
        c->mrhs_params_set = false;
    }
    // the parameters' upload is synchronous: repeat it only when they change,
    // so that calls with the same (gamma, eta) queue back to back on the stream
    if (!c->mrhs_params_set || gamma != c->mrhs_gamma || eta != c->mrhs_eta) {
        const int rc = apc_batch_set_params(c->mrhs, &gamma, &eta);
        if (rc != APC_OK) return cfail(c, rc, "%s", apc_batch_last_error(c->mrhs));
        c->mrhs_gamma = gamma;
        c->mrhs_eta = eta;
        c->mrhs_params_set = true;
    }
    return APC_OK;
}

}  // namespace

namespace apc {
void destroy_multi_rhs(apc_ctx *c) {
    if (c->mrhs) apc_batch_destroy(c->mrhs);
    if (c->mrhs_in) cudaFree(c->mrhs_in);
    if (c->mrhs_out) cudaFree(c->mrhs_out);
    c->mrhs = nullptr;
    c->mrhs_in = c->mrhs_out = nullptr;
    c->mrhs_k = 0;
    c->mrhs_params_set = false;
}
}  // namespace apc

extern "C" {

int apc_forward_rhs(apc_ctx *c, const double *B_dev, int64_t k, int64_t ldb, int64_t T, double gamma, double eta,
                    double *X_dev, int64_t ldx, void *stream) {
    if (!c) return apc::set_global_error_text("NULL context"), APC_ERR_INVALID_ARG;
    if (!B_dev || !X_dev || k < 1 || ldb < k || ldx < k || T < 0)
        return cfail(c, APC_ERR_INVALID_ARG, "apc_forward_rhs: bad pointer, k, leading dimension or T");
    if (!(gamma > 0.0 && gamma < 2.0) || !std::isfinite(eta))
        return cfail(c, APC_ERR_PARAMS, "gamma=%g must lie in (0, 2) and eta must be finite", gamma);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (use_tensor_cores(c, k)) {
        int rc = multi_rhs_batch(c, k, gamma, eta, s);
        if (rc != APC_OK) return rc;
        CCK(c, cudaMemcpy2DAsync(c->mrhs_in, sizeof(double) * k, B_dev, sizeof(double) * ldb, sizeof(double) * k,
                                 c->N, cudaMemcpyDeviceToDevice, s));
        const double *Bp = c->mrhs_in;
        double *Xp = c->mrhs_out;
        rc = apc_batch_forward(c->mrhs, &Bp, T, &Xp, stream);
        if (rc != APC_OK) return cfail(c, rc, "%s", apc_batch_last_error(c->mrhs));
        CCK(c, cudaMemcpy2DAsync(X_dev, sizeof(double) * ldx, c->mrhs_out, sizeof(double) * k, sizeof(double) * k,
                                 c->n, cudaMemcpyDeviceToDevice, s));
        return APC_OK;
    }
    for (int64_t j = 0; j < k; ++j) {
        CCK(c, cudaMemcpy2DAsync(c->rhs, sizeof(double), B_dev + j, sizeof(double) * ldb, sizeof(double), c->N,
                                 cudaMemcpyDeviceToDevice, s));
        int rc = apc_reset(c, c->rhs, stream);
        if (rc == APC_OK && T > 0) rc = apc_iterate(c, gamma, eta, T, stream);
        if (rc != APC_OK) return rc;
        CCK(c, cudaMemcpy2DAsync(X_dev + j, sizeof(double) * ldx, c->xbar, sizeof(double), sizeof(double), c->n,
                                 cudaMemcpyDeviceToDevice, s));
    }
    return APC_OK;
}

int apc_backward_rhs(apc_ctx *c, const double *G_dev, int64_t k, int64_t ldg, int64_t T, double gamma, double eta,
                     double *DB_dev, int64_t lddb, void *stream) {
    if (!c) return apc::set_global_error_text("NULL context"), APC_ERR_INVALID_ARG;
    if (!G_dev || !DB_dev || k < 1 || ldg < k || lddb < k || T < 0)
        return cfail(c, APC_ERR_INVALID_ARG, "apc_backward_rhs: bad pointer, k, leading dimension or T");
    if (!(gamma > 0.0 && gamma < 2.0) || !std::isfinite(eta))
        return cfail(c, APC_ERR_PARAMS, "gamma=%g must lie in (0, 2) and eta must be finite", gamma);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (use_tensor_cores(c, k)) {
        int rc = multi_rhs_batch(c, k, gamma, eta, s);
        if (rc != APC_OK) return rc;
        CCK(c, cudaMemcpy2DAsync(c->mrhs_in, sizeof(double) * k, G_dev, sizeof(double) * ldg, sizeof(double) * k,
                                 c->n, cudaMemcpyDeviceToDevice, s));
        const double *Gp = c->mrhs_in;
        double *Dp = c->mrhs_out;
        rc = apc_batch_backward(c->mrhs, &Gp, T, &Dp, stream);
        if (rc != APC_OK) return cfail(c, rc, "%s", apc_batch_last_error(c->mrhs));
        CCK(c, cudaMemcpy2DAsync(DB_dev, sizeof(double) * lddb, c->mrhs_out, sizeof(double) * k, sizeof(double) * k,
                                 c->N, cudaMemcpyDeviceToDevice, s));
        return APC_OK;
    }
    for (int64_t j = 0; j < k; ++j) {
        CCK(c, cudaMemcpy2DAsync(c->xtmp, sizeof(double), G_dev + j, sizeof(double) * ldg, sizeof(double), c->n,
                                 cudaMemcpyDeviceToDevice, s));
        const int rc = apc_backward(c, c->xtmp, T, gamma, eta, c->rhs, stream);
        if (rc != APC_OK) return rc;
        CCK(c, cudaMemcpy2DAsync(DB_dev + j, sizeof(double) * lddb, c->rhs, sizeof(double), sizeof(double), c->N,
                                 cudaMemcpyDeviceToDevice, s));
    }
    return APC_OK;
}

const char *apc_batch_last_error(const apc_batch *b) { return b ? b->last_error.c_str() : apc_last_error(nullptr); }

void apc_batch_destroy(apc_batch *b) {
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->graph_adj) cudaGraphExecDestroy(b->graph_adj);
    for (void *p : b->split_bufs) cudaFree(p);
    for (void *p : b->owned) cudaFree(p);
    for (apc_ctx *c : b->ctx) apc_destroy(c);
    delete b;
}

}  // extern "C"
