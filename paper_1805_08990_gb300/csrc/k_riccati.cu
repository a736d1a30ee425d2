// T3, the exact flow of dP/dt = -P B R^{-1} B^T P (Eq. nonlinear):
//     T3(t) P = (I + t P B R^{-1} B^T)^{-1} P.
// With Bt = B L_R^{-T} (B R^{-1} B^T = Bt Bt^T) and Z = P Bt (n x m), the
// Sherman-Morrison-Woodbury identity gives the m x m form
//     T3(t) P = P - t Z (I_m + t Bt^T Z)^{-1} Z^T,
// which only needs the small SPD matrix M = I_m + t Bt^T P Bt (the dense
// counterpart of the r x r solve of §2.2).  With M = L L^T and Y = Z L^{-T}:
//     T3(t) P = P - t Y Y^T.
// Four kernels: (1) Z = P Bt with per-block partial Gram sums Bt^T Z,
// (2) M, its Cholesky and L^{-1} (one warp, FP64, deterministic reduction
// order), (3) Y = Z L^{-T}, (4) the rank-m update P <- P - t Y Y^T (+ q Q).
// Everything is FP64.  (1) and (4) stream P once each with coalesced,
// 16-byte vector loads; the row dot-products of (1) are warp reductions.
#include "dme_internal.h"

#include <algorithm>

namespace dme {

constexpr int RZ_ROWS = 32;     // rows of P per block in kernel (1)
constexpr int RZ_MB = 8;        // columns of Bt per pass

static int rz_blocks(int n) { return (n + RZ_ROWS - 1) / RZ_ROWS; }

size_t riccati_work_doubles(int n, int m) {
    // Z (n m) | Y (n m) | Gpart (blocks m m) | Linv (m m)
    return (size_t)2 * n * m + (size_t)rz_blocks(n) * m * m + (size_t)m * m + 8;
}

// (1) Z[r][c] = sum_k P[r][k] Bt[k][c] for the block's 32 rows, columns
// c0 .. c0+MB-1; Bt chunks are staged in shared memory.
__global__ void __launch_bounds__(256) riccati_z_kernel(const double* __restrict__ P, const double* __restrict__ Bt,
                                                        double* __restrict__ Z, int n, int m, int c0) {
    constexpr int KC = 256;
    __shared__ double sB[KC][RZ_MB];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rbase = blockIdx.x * RZ_ROWS + warp * 4;
    const int mb = min(RZ_MB, m - c0);
    double acc[4][RZ_MB];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < RZ_MB; ++c) acc[r][c] = 0.0;

    for (int k0 = 0; k0 < n; k0 += KC) {
        __syncthreads();
        for (int e = threadIdx.x; e < KC * RZ_MB; e += blockDim.x) {
            int k = e / RZ_MB, c = e % RZ_MB;
            sB[k][c] = (k0 + k < n && c < mb) ? Bt[(size_t)(k0 + k) * m + c0 + c] : 0.0;
        }
        __syncthreads();
        const int kend = min(KC, n - k0);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int row = rbase + r;
            if (row >= n) continue;
            const double* prow = P + (size_t)row * n + k0;
            // 2 consecutive doubles per lane per iteration: a warp covers 64 columns
            for (int k = 2 * lane; k < kend; k += 64) {
                double p0, p1;
                if (k + 1 < kend && (((size_t)(prow + k)) & 15) == 0) {
                    double2 v = *reinterpret_cast<const double2*>(prow + k);
                    p0 = v.x;
                    p1 = v.y;
                } else {
                    p0 = prow[k];
                    p1 = (k + 1 < kend) ? prow[k + 1] : 0.0;
                }
#pragma unroll
                for (int c = 0; c < RZ_MB; ++c) {
                    acc[r][c] = fma(p0, sB[k][c], acc[r][c]);
                    if (k + 1 < kend) acc[r][c] = fma(p1, sB[k + 1][c], acc[r][c]);
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
#pragma unroll
        for (int c = 0; c < RZ_MB; ++c) {
            double v = acc[r][c];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            acc[r][c] = v;
        }
        const int row = rbase + r;
        if (row < n && lane < mb) {
            double v = 0.0;
#pragma unroll
            for (int c = 0; c < RZ_MB; ++c)
                if (c == lane) v = acc[r][c];
            Z[(size_t)row * m + c0 + lane] = v;
        }
    }
}

// (1b) Gpart[b][i][j] = sum over the block's rows r of Bt[r][i] Z[r][j], fixed order.
__global__ void riccati_gram_part_kernel(const double* __restrict__ Bt, const double* __restrict__ Z,
                                         double* __restrict__ Gpart, int n, int m) {
    const int b = blockIdx.x;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        int i = e / m, j = e % m;
        double s = 0.0;
        for (int r = b * RZ_ROWS; r < min(n, (b + 1) * RZ_ROWS); ++r) s = fma(Bt[(size_t)r * m + i], Z[(size_t)r * m + j], s);
        Gpart[(size_t)b * m * m + e] = s;
    }
}

// (2) M = I + t sym(sum_b Gpart[b]); M = L L^T; Linv = L^{-1}.  One warp.
__global__ void riccati_small_kernel(const double* __restrict__ Gpart, int nblocks, int m, double t,
                                     double* __restrict__ Linv, int* status) {
    __shared__ double M[32][33];
    __shared__ double L[32][33];
    const int lane = threadIdx.x;
    for (int e = lane; e < m * m; e += 32) {
        int i = e / m, j = e % m;
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += Gpart[(size_t)b * m * m + e];
        M[i][j] = s;
    }
    __syncwarp();
    for (int e = lane; e < m * m; e += 32) {
        int i = e / m, j = e % m;
        L[i][j] = (i == j ? 1.0 : 0.0) + t * 0.5 * (M[i][j] + M[j][i]);
    }
    __syncwarp();
    // Cholesky in place (lower)
    for (int j = 0; j < m; ++j) {
        double d = L[j][j];
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        if (!(d > 0.0)) {
            if (lane == 0) atomicOr(status, DEV_NOTSPD);
            return;
        }
        d = sqrt(d);
        __syncwarp();
        for (int i = j + 1 + lane; i < m; i += 32) {
            double s = L[i][j];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            L[i][j] = s / d;
        }
        __syncwarp();
        if (lane == 0) L[j][j] = d;
        __syncwarp();
    }
    // Linv column by column (forward substitution on e_c); lane c owns column c
    for (int c = lane; c < m; c += 32) {
        double x[32];
        for (int r = 0; r < m; ++r) {
            double s = (r == c) ? 1.0 : 0.0;
            for (int k = 0; k < r; ++k) s -= L[r][k] * x[k];
            x[r] = (r < c) ? 0.0 : s / L[r][r];
        }
        for (int r = 0; r < m; ++r) Linv[r * m + c] = x[r];
    }
}

// (3) Y[i][r] = sum_{c <= r} Linv[r][c] Z[i][c]   (Y = Z L^{-T}).
__global__ void riccati_y_kernel(const double* __restrict__ Z, const double* __restrict__ Linv,
                                 double* __restrict__ Y, int n, int m, const int* status) {
    if (*status & DEV_NOTSPD) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int r = 0; r < m; ++r) {
        double s = 0.0;
        for (int c = 0; c <= r; ++c) s = fma(Linv[r * m + c], Z[(size_t)i * m + c], s);
        Y[(size_t)i * m + r] = s;
    }
}

// (4) P[i][j] <- P[i][j] - t sum_r Y[i][r] Y[j][r] (+ q Q[i][j]).  The sum is
// taken in the same order for (i, j) and (j, i), so a symmetric P stays
// exactly symmetric.  64 x 64 tiles, 256 threads, Y rows staged in shared memory.
__global__ void __launch_bounds__(256) riccati_update_kernel(double* __restrict__ P, const double* __restrict__ Y,
                                                             int n, int m, double t, const double* __restrict__ Qadd,
                                                             double q, const int* status) {
    if (*status & DEV_NOTSPD) return;
    __shared__ double Yi[64][33];
    __shared__ double Yj[64][33];
    const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
    for (int e = threadIdx.x; e < 64 * m; e += blockDim.x) {
        int r = e / m, c = e % m;
        Yi[r][c] = (i0 + r < n) ? Y[(size_t)(i0 + r) * m + c] : 0.0;
        Yj[r][c] = (j0 + r < n) ? Y[(size_t)(j0 + r) * m + c] : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    for (int di = ty; di < 64; di += 8) {
        const int i = i0 + di;
        if (i >= n) break;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int dj = tx + 32 * h, j = j0 + dj;
            if (j >= n) continue;
            double s = 0.0;
            for (int c = 0; c < m; ++c) s = fma(Yi[di][c], Yj[dj][c], s);
            const size_t off = (size_t)i * n + j;
            double v = P[off] - t * s;
            if (Qadd) v += q * Qadd[off];
            P[off] = v;
        }
    }
}

void launch_riccati(double* P, const double* Bt, int n, int m, double t, const double* Qadd, double q,
                    double* work, int* status, cudaStream_t st) {
    double* Z = work;
    double* Y = Z + (size_t)n * m;
    double* Gpart = Y + (size_t)n * m;
    const int nb = rz_blocks(n);
    double* Linv = Gpart + (size_t)nb * m * m;
    for (int c0 = 0; c0 < m; c0 += RZ_MB) riccati_z_kernel<<<nb, 256, 0, st>>>(P, Bt, Z, n, m, c0);
    riccati_gram_part_kernel<<<nb, 64, 0, st>>>(Bt, Z, Gpart, n, m);
    riccati_small_kernel<<<1, 32, 0, st>>>(Gpart, nb, m, t, Linv, status);
    riccati_y_kernel<<<(n + 127) / 128, 128, 0, st>>>(Z, Linv, Y, n, m, status);
    dim3 g((n + 63) / 64, (n + 63) / 64);
    riccati_update_kernel<<<g, 256, 0, st>>>(P, Y, n, m, t, Qadd, q, status);
}

}  // namespace dme
