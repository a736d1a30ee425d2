// The action of the matrix exponential on a block of vectors by Newton
// interpolation at Leja points (the `expleja` step of the paper's low-rank
// algorithms, §3), for a sparse A^T in CSR.  One term of the Newton series
//     w_{k+1} = (A^T - c I) w_k / g - x_k w_k,   p <- p + d_{k+1} w_{k+1}
// is one fused, HBM-bound kernel: a warp per row of the n x r block (lanes
// over the r columns, so the rows of w read through the sparse row are
// contiguous; for r < 32 a thread per entry instead, so no lane idles),
// writing w_{k+1}, updating p, and leaving per-block partial sums
// of |w_{k+1}|^2 and |p|^2 that a second kernel reduces in a fixed order (the
// host stops the series on them, so the stopping point is reproducible).
#include "dme_internal.h"

#include <algorithm>

namespace dme {

namespace {

constexpr int LJ_ROWS = 8;      // rows per 256-thread block (one warp each)

__global__ void __launch_bounds__(256) leja_term_kernel(const int* __restrict__ ptr, const int* __restrict__ idx,
                                                        const double* __restrict__ val, int n, int r,
                                                        const double* __restrict__ W, double* __restrict__ Wn,
                                                        int ldw, double* __restrict__ Pacc, int ldp, double c,
                                                        double invg, double xk, double dk,
                                                        double* __restrict__ part) {
    __shared__ double sw[LJ_ROWS], sp[LJ_ROWS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = blockIdx.x * LJ_ROWS + warp;
    double aw = 0.0, ap = 0.0;
    if (row < n) {
        const int b = ptr[row], e = ptr[row + 1];
        for (int j = lane; j < r; j += 32) {
            double y = 0.0;
            for (int q = b; q < e; ++q) y = fma(val[q], W[(size_t)idx[q] * ldw + j], y);
            const double w = W[(size_t)row * ldw + j];
            const double wn = (y - c * w) * invg - xk * w;
            Wn[(size_t)row * ldw + j] = wn;
            const double pv = fma(dk, wn, Pacc[(size_t)row * ldp + j]);
            Pacc[(size_t)row * ldp + j] = pv;
            aw = fma(wn, wn, aw);
            ap = fma(pv, pv, ap);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        aw += __shfl_xor_sync(0xffffffffu, aw, off);
        ap += __shfl_xor_sync(0xffffffffu, ap, off);
    }
    if (lane == 0) {
        sw[warp] = aw;
        sp[warp] = ap;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, p = 0.0;
        for (int w = 0; w < LJ_ROWS; ++w) {
            a += sw[w];
            p += sp[w];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = p;
    }
}

// out[0], out[1] = sums of the partial pairs, strided then by a fixed tree.
__global__ void __launch_bounds__(1024) leja_reduce_kernel(const double* __restrict__ part, int nb,
                                                           double* __restrict__ out) {
    __shared__ double a[1024], p[1024];
    const int t = threadIdx.x;
    double sa = 0.0, sp = 0.0;
    for (int i = t; i < nb; i += 1024) {
        sa += part[2 * i];
        sp += part[2 * i + 1];
    }
    a[t] = sa;
    p[t] = sp;
    __syncthreads();
    for (int h = 512; h > 0; h >>= 1) {
        if (t < h) {
            a[t] += a[t + h];
            p[t] += p[t + h];
        }
        __syncthreads();
    }
    if (t == 0) {
        out[0] = a[0];
        out[1] = p[0];
    }
}

// Narrow blocks (r < 32): one thread per entry (row, j) of the block, 256
// entries per CTA, so no lane idles; same arithmetic and outputs.
__global__ void __launch_bounds__(256) leja_term_narrow_kernel(const int* __restrict__ ptr,
                                                               const int* __restrict__ idx,
                                                               const double* __restrict__ val, int n, int r,
                                                               const double* __restrict__ W, double* __restrict__ Wn,
                                                               int ldw, double* __restrict__ Pacc, int ldp, double c,
                                                               double invg, double xk, double dk,
                                                               double* __restrict__ part) {
    __shared__ double sw[8], sp[8];
    const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    double aw = 0.0, ap = 0.0;
    if (e < (size_t)n * r) {
        const int row = (int)(e / r), j = (int)(e % r);
        const int b = ptr[row], end = ptr[row + 1];
        double y = 0.0;
        for (int q = b; q < end; ++q) y = fma(val[q], W[(size_t)idx[q] * ldw + j], y);
        const double w = W[(size_t)row * ldw + j];
        const double wn = (y - c * w) * invg - xk * w;
        Wn[(size_t)row * ldw + j] = wn;
        const double pv = fma(dk, wn, Pacc[(size_t)row * ldp + j]);
        Pacc[(size_t)row * ldp + j] = pv;
        aw = wn * wn;
        ap = pv * pv;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        aw += __shfl_xor_sync(0xffffffffu, aw, off);
        ap += __shfl_xor_sync(0xffffffffu, ap, off);
    }
    if (lane == 0) {
        sw[warp] = aw;
        sp[warp] = ap;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, p = 0.0;
        for (int w = 0; w < 8; ++w) {
            a += sw[w];
            p += sp[w];
        }
        part[2 * blockIdx.x] = a;
        part[2 * blockIdx.x + 1] = p;
    }
}

}  // namespace

int leja_blocks(int n) { return (n + LJ_ROWS - 1) / LJ_ROWS; }

int leja_part_blocks(int n, int rmax) {
    // the larger of the two launch shapes' block counts (narrow form for r < 32)
    const size_t narrow = ((size_t)n * 31 + 255) / 256;
    return (int)std::max<size_t>((size_t)leja_blocks(n), narrow);
}

void launch_leja_term(const int* ptr, const int* idx, const double* val, int n, int r, const double* W, double* Wn,
                      int ldw, double* Pacc, int ldp, double c, double invg, double xk, double dk, double* part,
                      double* norms2, cudaStream_t st) {
    if (r < 32) {
        const int nb = (int)(((size_t)n * r + 255) / 256);
        leja_term_narrow_kernel<<<nb, 256, 0, st>>>(ptr, idx, val, n, r, W, Wn, ldw, Pacc, ldp, c, invg, xk, dk,
                                                    part);
        leja_reduce_kernel<<<1, 1024, 0, st>>>(part, nb, norms2);
        return;
    }
    const int nb = leja_blocks(n);
    leja_term_kernel<<<nb, 256, 0, st>>>(ptr, idx, val, n, r, W, Wn, ldw, Pacc, ldp, c, invg, xk, dk, part);
    leja_reduce_kernel<<<1, 1024, 0, st>>>(part, nb, norms2);
}

}  // namespace dme
