// FP64 setup kernels: the QR of each block (Sec. 3.3), the least-norm
// initialisation (Sec. 3.1, Algorithm 1), the FP64 residual b - A x and small
// vector helpers.
//
// QR by two passes of Cholesky QR.  For block i with rows scaled to unit
// length (D_i A_i; the scaling leaves the row space, hence P_i, unchanged):
//   G = (D A_i)(D A_i)^T = R1^T R1,  Q1^T = R1^{-T} D A_i,
//   G2 = Q1^T Q1 = R2^T R2,           Q^T  = R2^{-T} Q1^T,
// so D A_i = (R2 R1)^T Q^T and A_i x = b_i  <=>  Q^T x = R2^{-T} R1^{-T} D b_i.
// The second pass restores orthogonality lost in the first.  GB300 has few
// FP64 units, so these kernels are plain register-tiled FP64 FMA loops; their
// cost is paid once per system.
#include <algorithm>
#include <cstdio>
#include "apc_internal.h"

namespace apc {

namespace {

constexpr int TB = 32;   // output tile edge of the FP64 GEMM-like kernels
constexpr int TK = 32;   // depth of one shared-memory K slice

// ---- row scaling ------------------------------------------------------------
__global__ void rownorm_kernel(const double *A, int64_t lda, int64_t N, int64_t n, double *dinv, int *err) {
    const int64_t row = int64_t(blockIdx.x) * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (row >= N) return;
    const double *a = A + row * lda;
    double s = 0.0;
    for (int64_t j = lane; j < n; j += 32) s = fma(a[j], a[j], s);
    for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) {
        if (!(s > 0.0) || !isfinite(s)) {
            atomicCAS(err, 0, isfinite(s) ? 2 : 3);  // 2: zero row, 3: non-finite
            dinv[row] = 0.0;
        } else {
            dinv[row] = 1.0 / sqrt(s);
        }
    }
}

// ---- Gram matrix G_b = (D X_b)(D X_b)^T, upper-triangular tiles mirrored ----
__global__ void gram_kernel(const double *X, int64_t ldx, const int64_t *row_start, const int32_t *pcount,
                            const double *dinv, int P, int64_t n, double *G) {
    const int b = blockIdx.z;
    const int ti = blockIdx.y, tj = blockIdx.x;
    double *Gb = G + size_t(b) * P * P;
    if (ti > tj) return;
    const int p = pcount[b];
    const int64_t r0 = row_start[b];
    __shared__ double As[TB][TK + 1], Bs[TB][TK + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;  // 16 x 16 threads, 2 x 2 outputs each
    double c00 = 0, c01 = 0, c10 = 0, c11 = 0;
    for (int64_t k0 = 0; k0 < n; k0 += TK) {
        for (int idx = threadIdx.x; idx < TB * TK; idx += blockDim.x) {
            const int r = idx / TK, k = idx % TK;
            const int ri = ti * TB + r, rj = tj * TB + r;
            const int64_t kk = k0 + k;
            double va = 0, vb = 0;
            if (kk < n) {
                if (ri < p) va = X[(r0 + ri) * ldx + kk] * (dinv ? dinv[r0 + ri] : 1.0);
                if (rj < p) vb = X[(r0 + rj) * ldx + kk] * (dinv ? dinv[r0 + rj] : 1.0);
            }
            As[r][k] = va;
            Bs[r][k] = vb;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < TK; ++k) {
            const double a0 = As[ty][k], a1 = As[ty + 16][k];
            const double b0 = Bs[tx][k], b1 = Bs[tx + 16][k];
            c00 = fma(a0, b0, c00); c01 = fma(a0, b1, c01);
            c10 = fma(a1, b0, c10); c11 = fma(a1, b1, c11);
        }
        __syncthreads();
    }
    const int i0 = ti * TB + ty, j0 = tj * TB + tx;
    const double cv[2][2] = {{c00, c01}, {c10, c11}};
    for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) {
            const int i = i0 + 16 * u, j = j0 + 16 * v;
            Gb[size_t(i) * P + j] = cv[u][v];
            Gb[size_t(j) * P + i] = cv[u][v];
        }
}

// ---- Cholesky (upper, G = R^T R) and R^{-1}, one CTA per block --------------
__global__ void chol_kernel(double *G, double *Rinv, const int32_t *pcount, int P, double pivot_tol, int *err) {
    const int b = blockIdx.x;
    const int p = pcount[b];
    double *R = G + size_t(b) * P * P;
    double *Ri = Rinv + size_t(b) * P * P;
    __shared__ double piv;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int k = 0; k < p; ++k) {
        if (threadIdx.x == 0) {
            const double g = R[size_t(k) * P + k];
            if (!(g > pivot_tol) || !isfinite(g)) {
                bad = 1;
                piv = 1.0;
            } else {
                piv = sqrt(g);
            }
            R[size_t(k) * P + k] = piv;
        }
        __syncthreads();
        if (bad) break;
        const double rk = piv;
        for (int j = k + 1 + threadIdx.x; j < p; j += blockDim.x) R[size_t(k) * P + j] /= rk;
        __syncthreads();
        // trailing update of the upper triangle: R[i][j] -= R[k][i] R[k][j], k < i <= j
        const int m2 = p - k - 1;
        for (int64_t idx = threadIdx.x; idx < int64_t(m2) * m2; idx += blockDim.x) {
            const int i = k + 1 + int(idx / m2), j = k + 1 + int(idx % m2);
            if (j >= i) R[size_t(i) * P + j] -= R[size_t(k) * P + i] * R[size_t(k) * P + j];
        }
        __syncthreads();
    }
    if (bad) {
        if (threadIdx.x == 0) atomicCAS(err, 0, 1 + b);
        return;
    }
    // zero the strict lower triangle and the padding
    for (int64_t idx = threadIdx.x; idx < int64_t(P) * P; idx += blockDim.x) {
        const int i = int(idx / P), j = int(idx % P);
        if (i >= p || j >= p || j < i) R[idx] = 0.0;
        Ri[idx] = 0.0;
    }
    __syncthreads();
    // R^{-1} column by column (back substitution), one thread per column
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
        Ri[size_t(j) * P + j] = 1.0 / R[size_t(j) * P + j];
        for (int i = j - 1; i >= 0; --i) {
            double s = 0.0;
            for (int k = i + 1; k <= j; ++k) s = fma(R[size_t(i) * P + k], Ri[size_t(k) * P + j], s);
            Ri[size_t(i) * P + j] = -s / R[size_t(i) * P + i];
        }
    }
}

// ---- QT_b[c][j] = sum_{r <= c} Rinv_b[r][c] d_r X_b[r][j] -------------------
__global__ void qt_kernel(const double *X, int64_t ldx, const int64_t *row_start, const int32_t *pcount,
                          const double *dinv, const double *Rinv, int P, int64_t n, double *QT) {
    const int b = blockIdx.z;
    const int tc = blockIdx.y;             // tile of output rows c
    const int64_t j_base = int64_t(blockIdx.x) * TB;  // tile of columns j
    const int p = pcount[b];
    const int64_t r0 = row_start[b];
    const double *Rb = Rinv + size_t(b) * P * P;
    double *Qb = QT + size_t(b) * P * n;
    __shared__ double Ms[TK][TB + 1];  // Ms[r][c] = Rinv[r][c]
    __shared__ double Xs[TK][TB + 1];  // Xs[r][j] = d_r X[r][j]
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double c00 = 0, c01 = 0, c10 = 0, c11 = 0;
    const int c_hi = min(p, (tc + 1) * TB);
    for (int k0 = 0; k0 < c_hi; k0 += TK) {
        for (int idx = threadIdx.x; idx < TK * TB; idx += blockDim.x) {
            const int r = idx / TB, c = idx % TB;
            const int rr = k0 + r, cc = tc * TB + c;
            Ms[r][c] = (rr < p && cc < p) ? Rb[size_t(rr) * P + cc] : 0.0;
            const int64_t jj = j_base + c;
            Xs[r][c] = (rr < p && jj < n) ? X[(r0 + rr) * ldx + jj] * (dinv ? dinv[r0 + rr] : 1.0) : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < TK; ++k) {
            const double m0 = Ms[k][ty], m1 = Ms[k][ty + 16];
            const double x0 = Xs[k][tx], x1 = Xs[k][tx + 16];
            c00 = fma(m0, x0, c00); c01 = fma(m0, x1, c01);
            c10 = fma(m1, x0, c10); c11 = fma(m1, x1, c11);
        }
        __syncthreads();
    }
    const double cv[2][2] = {{c00, c01}, {c10, c11}};
    for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v) {
            const int c = tc * TB + ty + 16 * u;
            const int64_t j = j_base + tx + 16 * v;
            if (j < n) Qb[size_t(c) * n + j] = cv[u][v];
        }
}

// ---- pack QT [m][P][n] (FP64) into Q [n][m][P] (iteration precision) --------
template <typename TQ>
__global__ void pack_kernel(const double *QT, int m, int P, int64_t n, TQ *Q) {
    __shared__ double tile[TB][TB + 1];
    const int b = blockIdx.z;
    const int c0 = blockIdx.y * TB;
    const int64_t j0 = int64_t(blockIdx.x) * TB;
    const double *src = QT + size_t(b) * P * n;
    for (int idx = threadIdx.x; idx < TB * TB; idx += blockDim.x) {
        const int c = idx / TB, jj = idx % TB;
        tile[c][jj] = (j0 + jj < n) ? src[size_t(c0 + c) * n + j0 + jj] : 0.0;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < TB * TB; idx += blockDim.x) {
        const int jj = idx / TB, c = idx % TB;
        if (j0 + jj < n) Q[(size_t(j0 + jj) * m + b) * P + c0 + c] = TQ(tile[c][jj]);
    }
}

template <>
__global__ void pack_kernel<__nv_bfloat16>(const double *QT, int m, int P, int64_t n, __nv_bfloat16 *Q) {
    __shared__ double tile[TB][TB + 1];
    const int b = blockIdx.z;
    const int c0 = blockIdx.y * TB;
    const int64_t j0 = int64_t(blockIdx.x) * TB;
    const double *src = QT + size_t(b) * P * n;
    for (int idx = threadIdx.x; idx < TB * TB; idx += blockDim.x) {
        const int c = idx / TB, jj = idx % TB;
        tile[c][jj] = (j0 + jj < n) ? src[size_t(c0 + c) * n + j0 + jj] : 0.0;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < TB * TB; idx += blockDim.x) {
        const int jj = idx / TB, c = idx % TB;
        if (j0 + jj < n) Q[(size_t(j0 + jj) * m + b) * P + c0 + c] = __double2bfloat16(tile[c][jj]);
    }
}

// ---- c_b = Rinv2^T Rinv1^T (d .* rhs_b) --------------------------------------
template <typename TS>
__global__ void csolve_kernel(const double *rhs, const int64_t *row_start, const int32_t *pcount,
                              const double *dinv, const double *Rinv1, const double *Rinv2, int P, TS *z) {
    extern __shared__ double sh[];  // y[P], u[P]
    const int b = blockIdx.x;
    const int p = pcount[b];
    const int64_t r0 = row_start[b];
    const double *R1 = Rinv1 + size_t(b) * P * P, *R2 = Rinv2 + size_t(b) * P * P;
    double *y = sh, *u = sh + P;
    for (int r = threadIdx.x; r < P; r += blockDim.x) y[r] = r < p ? dinv[r0 + r] * rhs[r0 + r] : 0.0;
    __syncthreads();
    // u[c] = sum_{r <= c} R1[r][c] y[r]
    for (int c = threadIdx.x; c < P; c += blockDim.x) {
        double s = 0.0;
        for (int r = 0; r <= c && r < p; ++r) s = fma(R1[size_t(r) * P + c], y[r], s);
        u[c] = c < p ? s : 0.0;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < P; c += blockDim.x) {
        double s = 0.0;
        for (int r = 0; r <= c && r < p; ++r) s = fma(R2[size_t(r) * P + c], u[r], s);
        z[size_t(b) * P + c] = TS(c < p ? s : 0.0);
    }
}

// ---- db_b = d .* (Rinv1 (Rinv2 v_b)) ------------------------------------------
template <typename TS>
__global__ void bsolve_kernel(const TS *z, const int64_t *row_start, const int32_t *pcount, const double *dinv,
                              const double *Rinv1, const double *Rinv2, int P, double *db) {
    extern __shared__ double sh[];
    const int b = blockIdx.x;
    const int p = pcount[b];
    const int64_t r0 = row_start[b];
    const double *R1 = Rinv1 + size_t(b) * P * P, *R2 = Rinv2 + size_t(b) * P * P;
    double *v = sh, *u = sh + P;
    for (int c = threadIdx.x; c < P; c += blockDim.x) v[c] = c < p ? double(z[size_t(b) * P + c]) : 0.0;
    __syncthreads();
    // u[r] = sum_{c >= r} R2[r][c] v[c]
    for (int r = threadIdx.x; r < P; r += blockDim.x) {
        double s = 0.0;
        for (int c = r; c < p; ++c) s = fma(R2[size_t(r) * P + c], v[c], s);
        u[r] = r < p ? s : 0.0;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < p; r += blockDim.x) {
        double s = 0.0;
        for (int c = r; c < p; ++c) s = fma(R1[size_t(r) * P + c], u[c], s);
        db[r0 + r] = dinv[r0 + r] * s;
    }
}

// ---- orthogonality probe of a first Cholesky-QR pass ----------------------------
// With v the +-1 vector v_c = sign pattern of a hash of c (c < p), Y_b = Q_b v
// (Q_b = QT_b^T, n x p) and u_b = Q_b^T Y_b; ||u_b - v|| / ||v|| is the
// departure of Q_b^T Q_b from the identity along v.
__device__ __forceinline__ double probe_sign(int c) { return ((uint32_t(c) * 0x9E3779B1u) >> 31) ? 1.0 : -1.0; }

__global__ void probe_y_kernel(const double *QT, const int32_t *pcount, int P, int64_t n, double *Y) {
    const int b = blockIdx.y;
    const int p = pcount[b];
    const double *Qb = QT + size_t(b) * P * n;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x) {
        double y = 0.0;
        for (int c = 0; c < p; ++c) y = fma(probe_sign(c), Qb[size_t(c) * n + j], y);
        Y[size_t(b) * n + j] = y;
    }
}

// err[b] = ||Q_b^T Y_b - v|| / ||v||, one CTA per block, one warp per row c
__global__ void probe_u_kernel(const double *QT, const double *Y, const int32_t *pcount, int P, int64_t n,
                               double *err) {
    __shared__ double part[32];
    const int b = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int p = pcount[b];
    const double *Qb = QT + size_t(b) * P * n, *Yb = Y + size_t(b) * n;
    double acc = 0.0;
    for (int c = warp; c < p; c += nw) {
        double u = 0.0;
        for (int64_t j = lane; j < n; j += 32) u = fma(Qb[size_t(c) * n + j], Yb[j], u);
        for (int off = 16; off; off >>= 1) u += __shfl_xor_sync(0xffffffffu, u, off);
        const double d = u - probe_sign(c);
        acc = fma(d, d, acc);
    }
    if (lane == 0) part[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += part[w];
        err[b] = sqrt(t / double(p > 0 ? p : 1));
    }
}

// R_b = I (p x p, zero padding): the second Cholesky-QR pass left out
__global__ void identity_kernel(double *R, const int32_t *pcount, int P) {
    const int b = blockIdx.x;
    const int p = pcount[b];
    for (int64_t idx = threadIdx.x; idx < int64_t(P) * P; idx += blockDim.x) {
        const int i = int(idx / P), j = int(idx % P);
        R[size_t(b) * P * P + idx] = (i == j && i < p) ? 1.0 : 0.0;
    }
}

// ---- free residual monitor -------------------------------------------------------
// Row block b of the residual of xbar: A_b xbar - rhs_b = D^{-1} R'^T (Q_b^T xbar - c_b)
// with (D A_b)^T = Q_b R', R' = R2 R1 the two Cholesky factors, and
// c_b = R'^{-T} D rhs_b.  While every x_i solves its block (App. A),
// Q_b^T xbar - c_b = Q_b^T (xbar - x_b) = z_b, the coefficients the iteration
// kernel already holds; so ||residual||^2 = sum_b ||D^{-1} R1^T R2^T z_b||^2, a
// p x p product per block.  sums[0] += that sum.
template <typename TS>
__global__ void monitor_kernel(const TS *z, const int64_t *row_start, const int32_t *pcount, const double *dinv,
                               const double *R1f, const double *R2f, int P, double *sums) {
    extern __shared__ double sh[];  // v[P], w[P]
    __shared__ double part[32];
    const int b = blockIdx.x;
    const int p = pcount[b];
    const int64_t r0 = row_start[b];
    const double *R1 = R1f + size_t(b) * P * P, *R2 = R2f + size_t(b) * P * P;
    double *v = sh, *w = sh + P;
    for (int c = threadIdx.x; c < P; c += blockDim.x) v[c] = c < p ? double(z[size_t(b) * P + c]) : 0.0;
    __syncthreads();
    // w = R2^T v: w[c] = sum_{r <= c} R2[r][c] v[r]
    for (int c = threadIdx.x; c < P; c += blockDim.x) {
        double s = 0.0;
        for (int r = 0; r <= c && r < p; ++r) s = fma(R2[size_t(r) * P + c], v[r], s);
        w[c] = c < p ? s : 0.0;
    }
    __syncthreads();
    double acc = 0.0;
    for (int c = threadIdx.x; c < p; c += blockDim.x) {
        double s = 0.0;
        for (int r = 0; r <= c; ++r) s = fma(R1[size_t(r) * P + c], w[r], s);
        const double res = s / dinv[r0 + c];
        acc = fma(res, res, acc);
    }
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < int(blockDim.x >> 5); ++i) t += part[i];
        atomicAdd(sums, t);
    }
}

// sums[0] += ||v||^2
__global__ void sumsq_kernel(const double *v, int64_t count, double *sums) {
    double acc = 0.0;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
        acc = fma(v[i], v[i], acc);
    for (int off = 16; off; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(sums, acc);
}

// ---- residual out = rhs - A x; sums += (||out||^2, ||rhs||^2) -----------------
// One warp per row, RPW rows per warp, x staged through shared memory in
// chunks shared by the CTA's warps.
constexpr int RES_WARPS = 8, RES_RPW = 4, RES_CHUNK = 2048;
__global__ void __launch_bounds__(RES_WARPS * 32) residual_kernel(const double *A, int64_t lda, int64_t N,
                                                                  int64_t n, const double *x, const double *rhs,
                                                                  double *out, double *sums) {
    __shared__ double xs[RES_CHUNK];
    __shared__ double part[2][RES_WARPS];
    const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
    const int64_t row_base = (int64_t(blockIdx.x) * RES_WARPS + warp) * RES_RPW;
    double acc[RES_RPW];
    for (int r = 0; r < RES_RPW; ++r) acc[r] = 0.0;
    for (int64_t k0 = 0; k0 < n; k0 += RES_CHUNK) {
        const int kn = int(min(int64_t(RES_CHUNK), n - k0));
        __syncthreads();
        for (int k = threadIdx.x; k < kn; k += blockDim.x) xs[k] = x[k0 + k];
        __syncthreads();
        for (int r = 0; r < RES_RPW; ++r) {
            const int64_t row = row_base + r;
            if (row >= N) break;
            const double *a = A + row * lda + k0;
            double s = acc[r];
            for (int k = lane; k < kn; k += 32) s = fma(a[k], xs[k], s);
            acc[r] = s;
        }
    }
    double s_out = 0.0, s_rhs = 0.0;
    for (int r = 0; r < RES_RPW; ++r) {
        double v = acc[r];
        for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        const int64_t row = row_base + r;
        if (lane == 0 && row < N) {
            const double rr = rhs[row] - v;
            out[row] = rr;
            s_out = fma(rr, rr, s_out);
            s_rhs = fma(rhs[row], rhs[row], s_rhs);
        }
    }
    if (lane == 0) {
        part[0][warp] = s_out;
        part[1][warp] = s_rhs;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a0 = 0.0, a1 = 0.0;
        for (int w = 0; w < RES_WARPS; ++w) {
            a0 += part[0][w];
            a1 += part[1][w];
        }
        atomicAdd(&sums[0], a0);
        atomicAdd(&sums[1], a1);
    }
}

template <typename TS>
__global__ void to_f64_kernel(const TS *src, int64_t count, double *dst) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
        dst[i] = double(src[i]);
}

template <typename TS>
__global__ void from_f64_kernel(const double *src, int64_t count, TS *dst) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
        dst[i] = TS(src[i]);
}

template <typename TS>
__global__ void unpack_x_kernel(const TS *xw, int64_t n, int m, double *out, int64_t ld) {
    for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < n * m;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t j = idx / m;
        const int i = int(idx % m);
        out[size_t(i) * ld + j] = double(xw[idx]);
    }
}

template <typename TQ>
__global__ void get_basis_kernel(const TQ *Q, int64_t n, int m, int P, int b, int p, double *out, int64_t ldq) {
    for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < n * p;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t j = idx / p;
        const int c = int(idx % p);
        out[j * ldq + c] = double(Q[(size_t(j) * m + b) * P + c]);
    }
}

template <>
__global__ void get_basis_kernel<__nv_bfloat16>(const __nv_bfloat16 *Q, int64_t n, int m, int P, int b, int p,
                                                double *out, int64_t ldq) {
    for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < n * p;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t j = idx / p;
        const int c = int(idx % p);
        out[j * ldq + c] = double(__bfloat162float(Q[(size_t(j) * m + b) * P + c]));
    }
}

__global__ void axpy_kernel(double *y, const double *x, double a, int64_t count) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
        y[i] = fma(a, x[i], y[i]);
}

// out[k][:] = A[perm[k]][:]  (rows of an N x n row-major matrix)
__global__ void gather_rows_kernel(const double *A, int64_t lda, int64_t N, int64_t n, const int64_t *perm,
                                   double *out) {
    const int64_t total = N * n;
    for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const int64_t k = idx / n, j = idx - k * n;
        out[idx] = A[perm[k] * lda + j];
    }
}

// out[k] = v[perm[k]] (gather) or out[perm[k]] = v[k] (scatter)
__global__ void permute_vec_kernel(const double *v, const int64_t *perm, int64_t N, int scatter, double *out) {
    for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < N; k += int64_t(gridDim.x) * blockDim.x) {
        if (scatter)
            out[perm[k]] = v[k];
        else
            out[k] = v[perm[k]];
    }
}

__global__ void finite_kernel(const double *v, int64_t count, int *flag) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
        if (!isfinite(v[i])) atomicOr(flag, 1);
}

inline unsigned grid1d(int64_t count, int threads) {
    int64_t g = (count + threads - 1) / threads;
    return unsigned(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

}  // namespace

cudaError_t launch_gather_rows(const double *A, int64_t lda, int64_t N, int64_t n, const int64_t *perm,
                               double *out, cudaStream_t s) {
    const unsigned g = unsigned(std::min<int64_t>((N * n + 255) / 256, 152 * 64));
    gather_rows_kernel<<<g, 256, 0, s>>>(A, lda, N, n, perm, out);
    return cudaGetLastError();
}

cudaError_t launch_permute_vec(const double *v, const int64_t *perm, int64_t N, int scatter, double *out,
                               cudaStream_t s) {
    const unsigned g = unsigned(std::min<int64_t>((N + 255) / 256, 152 * 16));
    permute_vec_kernel<<<g, 256, 0, s>>>(v, perm, N, scatter, out);
    return cudaGetLastError();
}

cudaError_t launch_rownorm(const double *A, int64_t lda, int64_t N, int64_t n, double *dinv, int *err,
                           cudaStream_t s) {
    rownorm_kernel<<<unsigned((N + 7) / 8), 256, 0, s>>>(A, lda, N, n, dinv, err);
    return cudaGetLastError();
}

cudaError_t launch_gram(const double *X, int64_t ldx, const int64_t *row_start_dev, const int32_t *p_dev,
                        const double *dinv, int m, int P, int64_t n, double *G, cudaStream_t s) {
    dim3 grid(unsigned(P / TB), unsigned(P / TB), unsigned(m));
    gram_kernel<<<grid, 256, 0, s>>>(X, ldx, row_start_dev, p_dev, dinv, P, n, G);
    return cudaGetLastError();
}

cudaError_t launch_chol(double *G, double *Rinv, const int32_t *p_dev, int m, int P, double pivot_tol, int *err,
                        cudaStream_t s) {
    chol_kernel<<<unsigned(m), 256, 0, s>>>(G, Rinv, p_dev, P, pivot_tol, err);
    return cudaGetLastError();
}

cudaError_t launch_qt(const double *X, int64_t ldx, const int64_t *row_start_dev, const int32_t *p_dev,
                      const double *dinv, const double *Rinv, int m, int P, int64_t n, double *QT, cudaStream_t s) {
    dim3 grid(unsigned((n + TB - 1) / TB), unsigned(P / TB), unsigned(m));
    qt_kernel<<<grid, 256, 0, s>>>(X, ldx, row_start_dev, p_dev, dinv, Rinv, P, n, QT);
    return cudaGetLastError();
}

cudaError_t launch_pack(const double *QT, int m, int P, int64_t n, int precision, void *Q, cudaStream_t s) {
    dim3 grid(unsigned((n + TB - 1) / TB), unsigned(P / TB), unsigned(m));
    switch (precision) {
        case 0: pack_kernel<double><<<grid, 256, 0, s>>>(QT, m, P, n, static_cast<double *>(Q)); break;
        case 1: pack_kernel<float><<<grid, 256, 0, s>>>(QT, m, P, n, static_cast<float *>(Q)); break;
        default: pack_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(QT, m, P, n, static_cast<__nv_bfloat16 *>(Q));
    }
    return cudaGetLastError();
}

cudaError_t launch_csolve(const double *rhs, const int64_t *row_start_dev, const int32_t *p_dev, const double *dinv,
                          const double *Rinv1, const double *Rinv2, int m, int P, int precision, void *z,
                          cudaStream_t s) {
    const size_t sh = 2 * size_t(P) * sizeof(double);
    if (precision == 0)
        csolve_kernel<double><<<unsigned(m), 256, sh, s>>>(rhs, row_start_dev, p_dev, dinv, Rinv1, Rinv2, P,
                                                          static_cast<double *>(z));
    else
        csolve_kernel<float><<<unsigned(m), 256, sh, s>>>(rhs, row_start_dev, p_dev, dinv, Rinv1, Rinv2, P,
                                                         static_cast<float *>(z));
    return cudaGetLastError();
}

cudaError_t launch_bsolve(const void *z, const int64_t *row_start_dev, const int32_t *p_dev, const double *dinv,
                          const double *Rinv1, const double *Rinv2, int m, int P, int precision, double *db,
                          cudaStream_t s) {
    const size_t sh = 2 * size_t(P) * sizeof(double);
    if (precision == 0)
        bsolve_kernel<double><<<unsigned(m), 256, sh, s>>>(static_cast<const double *>(z), row_start_dev, p_dev,
                                                          dinv, Rinv1, Rinv2, P, db);
    else
        bsolve_kernel<float><<<unsigned(m), 256, sh, s>>>(static_cast<const float *>(z), row_start_dev, p_dev,
                                                         dinv, Rinv1, Rinv2, P, db);
    return cudaGetLastError();
}

cudaError_t launch_orth_probe(const double *QT, const int32_t *p_dev, int m, int P, int64_t n, double *Y, double *err,
                              cudaStream_t s) {
    probe_y_kernel<<<dim3(unsigned(std::min<int64_t>((n + 255) / 256, 256)), unsigned(m)), 256, 0, s>>>(QT, p_dev, P, n,
                                                                                                     Y);
    probe_u_kernel<<<unsigned(m), 256, 0, s>>>(QT, Y, p_dev, P, n, err);
    return cudaGetLastError();
}

cudaError_t launch_identity(double *R, const int32_t *p_dev, int m, int P, cudaStream_t s) {
    identity_kernel<<<unsigned(m), 256, 0, s>>>(R, p_dev, P);
    return cudaGetLastError();
}

cudaError_t launch_monitor(const void *z, int precision, const int64_t *row_start_dev, const int32_t *p_dev,
                           const double *dinv, const double *R1, const double *R2, int m, int P, double *sums,
                           cudaStream_t s) {
    const size_t sh = sizeof(double) * 2 * P;
    if (precision == 0)
        monitor_kernel<double><<<m, 256, sh, s>>>(static_cast<const double *>(z), row_start_dev, p_dev, dinv, R1, R2, P,
                                                  sums);
    else
        monitor_kernel<float><<<m, 256, sh, s>>>(static_cast<const float *>(z), row_start_dev, p_dev, dinv, R1, R2, P,
                                                 sums);
    return cudaGetLastError();
}

cudaError_t launch_sumsq(const double *v, int64_t count, double *sums, cudaStream_t s) {
    const unsigned grid = unsigned(std::min<int64_t>((count + 255) / 256, 1024));
    sumsq_kernel<<<grid, 256, 0, s>>>(v, count, sums);
    return cudaGetLastError();
}

cudaError_t launch_residual(const double *A, int64_t lda, int64_t N, int64_t n, const double *x, const double *rhs,
                            double *out, double *sums, cudaStream_t s) {
    const int64_t rows_per_cta = RES_WARPS * RES_RPW;
    residual_kernel<<<unsigned((N + rows_per_cta - 1) / rows_per_cta), RES_WARPS * 32, 0, s>>>(A, lda, N, n, x, rhs,
                                                                                              out, sums);
    return cudaGetLastError();
}

cudaError_t launch_to_f64(const void *src, int precision, int64_t count, double *dst, cudaStream_t s) {
    if (precision == 0)
        to_f64_kernel<double><<<grid1d(count, 256), 256, 0, s>>>(static_cast<const double *>(src), count, dst);
    else
        to_f64_kernel<float><<<grid1d(count, 256), 256, 0, s>>>(static_cast<const float *>(src), count, dst);
    return cudaGetLastError();
}

cudaError_t launch_from_f64(const double *src, int precision, int64_t count, void *dst, cudaStream_t s) {
    if (precision == 0)
        from_f64_kernel<double><<<grid1d(count, 256), 256, 0, s>>>(src, count, static_cast<double *>(dst));
    else
        from_f64_kernel<float><<<grid1d(count, 256), 256, 0, s>>>(src, count, static_cast<float *>(dst));
    return cudaGetLastError();
}

cudaError_t launch_unpack_x(const void *xw, int precision, int64_t n, int m, double *out, int64_t ld,
                            cudaStream_t s) {
    if (precision == 0)
        unpack_x_kernel<double><<<grid1d(n * m, 256), 256, 0, s>>>(static_cast<const double *>(xw), n, m, out, ld);
    else
        unpack_x_kernel<float><<<grid1d(n * m, 256), 256, 0, s>>>(static_cast<const float *>(xw), n, m, out, ld);
    return cudaGetLastError();
}

cudaError_t launch_get_basis(const void *Q, int precision, int64_t n, int m, int P, int b, int p, double *out,
                             int64_t ldq, cudaStream_t s) {
    const unsigned g = grid1d(n * p, 256);
    if (precision == 0)
        get_basis_kernel<double><<<g, 256, 0, s>>>(static_cast<const double *>(Q), n, m, P, b, p, out, ldq);
    else if (precision == 1)
        get_basis_kernel<float><<<g, 256, 0, s>>>(static_cast<const float *>(Q), n, m, P, b, p, out, ldq);
    else
        get_basis_kernel<__nv_bfloat16><<<g, 256, 0, s>>>(static_cast<const __nv_bfloat16 *>(Q), n, m, P, b, p,
                                                          out, ldq);
    return cudaGetLastError();
}

namespace {
// acc[0] += sum_j sum_i (lam[j][i] + em lbar[j]) (x1[j][i] - x0[j][i]),
// acc[1] += sum_j lbar[j] ((1/m) sum_i x1[j][i] - xb0[j])   (FP64 sums; [n][m] states)
template <typename TS>
__global__ void adj_dots_kernel(const TS *lam, const double *lbar, const TS *x1, const TS *x0, const double *xb0,
                                int64_t n, int m, double em, double *acc) {
    double sg = 0.0, se = 0.0;
    for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += int64_t(gridDim.x) * blockDim.x) {
        const double lb = lbar[j];
        double mean = 0.0;
        for (int i = 0; i < m; ++i) {
            const size_t k = size_t(j) * m + i;
            sg += (double(lam[k]) + em * lb) * (double(x1[k]) - double(x0[k]));
            mean += double(x1[k]);
        }
        se += lb * (mean / m - xb0[j]);
    }
    for (int off = 16; off > 0; off >>= 1) {
        sg += __shfl_xor_sync(0xffffffffu, sg, off);
        se += __shfl_xor_sync(0xffffffffu, se, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(acc, sg);
        atomicAdd(acc + 1, se);
    }
}
}  // namespace

cudaError_t launch_adj_dots(const void *lam, const double *lbar, const void *x1, const void *x0, const double *xb0,
                            int64_t n, int m, double em, int precision, double *acc, cudaStream_t s) {
    const unsigned g = unsigned(std::min<int64_t>((n + 255) / 256, 1024));
    if (precision == 0)
        adj_dots_kernel<double><<<g, 256, 0, s>>>(static_cast<const double *>(lam), lbar,
                                                  static_cast<const double *>(x1), static_cast<const double *>(x0),
                                                  xb0, n, m, em, acc);
    else
        adj_dots_kernel<float><<<g, 256, 0, s>>>(static_cast<const float *>(lam), lbar,
                                                 static_cast<const float *>(x1), static_cast<const float *>(x0), xb0,
                                                 n, m, em, acc);
    return cudaGetLastError();
}

cudaError_t launch_axpy_f64(double *y, const double *x, double a, int64_t count, cudaStream_t s) {
    axpy_kernel<<<grid1d(count, 256), 256, 0, s>>>(y, x, a, count);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const double *v, int64_t count, int *flag, cudaStream_t s) {
    finite_kernel<<<grid1d(count, 256), 256, 0, s>>>(v, count, flag);
    return cudaGetLastError();
}

}  // namespace apc
