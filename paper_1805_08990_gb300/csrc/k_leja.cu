// The action of the matrix exponential on a block of vectors by Newton
// interpolation at Leja points (the `expleja` step of the paper's low-rank
// algorithms, §3), for a sparse A^T in CSR.  Over each substep the series
//     w_0 = v,  w_{k+1} = (A^T - c I) w_k / g - x_k w_k,   p = sum_k d_k w_k
// needs one SpMM of the n x r block per term and a stopping test on the norms
// of the newest term and of the partial sum.  The block is small (a few MB) and
// the terms are many (the count grows with t ||A||), so one launch per term
// would be bound by launch and host round-trip latency: instead one persistent
// cooperative launch runs every term of every substep of an application.  Each
// thread owns the same entries (row, j) throughout; a term is a grid-stride
// pass (SpMM row, recurrence, accumulation, per-block partial norms) followed
// by a grid barrier (grid_sync.cuh) whose last arriving block sums the
// partials in a fixed order, so every block takes the same, reproducible
// stopping decision.
#include "dme_internal.h"
#include "grid_sync.cuh"

#include <algorithm>

namespace dme {

namespace {

constexpr int LJ_THREADS = 256;

// Block sum of two values; the result is valid in every thread.
__device__ __forceinline__ void block_sum2(double& a, double& b, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, off);
        b += __shfl_xor_sync(0xffffffffu, b, off);
    }
    __syncthreads();                         // sh may still be read from the previous call
    if (lane == 0) {
        sh[2 * warp] = a;
        sh[2 * warp + 1] = b;
    }
    __syncthreads();
    a = 0.0;
    b = 0.0;
    for (int w = 0; w < LJ_THREADS / 32; ++w) {   // fixed order
        a += sh[2 * w];
        b += sh[2 * w + 1];
    }
}

// Grid barrier number `b`.  If part != nullptr the last block to arrive first
// sums part[2i], part[2i+1] over the grid (fixed order) into sums[0..1].
// Returns false after a timeout (status set).
__device__ bool grid_barrier(unsigned* bar, unsigned b, const double* part, double* sums, int* status,
                             double* sh) {
    __shared__ int s_last, s_ok;
    if (gs_arrive(bar, b, &s_last)) {
        if (part) {
            double a = 0.0, p = 0.0;
            for (int i = threadIdx.x; i < (int)gridDim.x; i += LJ_THREADS) {
                a += __ldcg(part + 2 * i);
                p += __ldcg(part + 2 * i + 1);
            }
            block_sum2(a, p, sh);
            if (threadIdx.x == 0) {
                sums[0] = a;
                sums[1] = p;
            }
        }
        gs_release(bar, b);
        __syncthreads();
        return true;
    }
    return gs_wait(bar, b, status, &s_ok);
}

struct LejaArgs {
    const int* ptr;
    const int* idx;
    const double* val;
    int n, r;
    const double* X;
    int ldx;
    double* Y;
    int ldy;
    double* Wa;
    double* Wb;
    int ldw;
    double c, invg, scale, tol;
    int substeps, terms;
    double* part;       // 2 buffers x 2 gridDim doubles
    double* sums;       // 2 buffers x 2 doubles
    unsigned* bar;      // arrival counter, release generation (zeroed before the launch)
    int* status;
    double xi[80];
    double dd[80];
};

// The entries (row, j) a thread owns: e = first, first + stride, ... < n r in
// row-major order, walked without a division per entry.
struct Entries {
    int row0, j0, drow, dj, n, r;
    __device__ Entries(int n_, int r_) : n(n_), r(r_) {
        const size_t first = (size_t)blockIdx.x * LJ_THREADS + threadIdx.x;
        const size_t stride = (size_t)gridDim.x * LJ_THREADS;
        row0 = (int)(first / r_);
        j0 = (int)(first % r_);
        drow = (int)(stride / r_);
        dj = (int)(stride % r_);
    }
    __device__ __forceinline__ void next(int& row, int& j) const {
        row += drow;
        j += dj;
        if (j >= r) {
            j -= r;
            ++row;
        }
    }
};

__global__ void __launch_bounds__(LJ_THREADS) leja_persistent_kernel(const LejaArgs a) {
    __shared__ double sh[2 * (LJ_THREADS / 32)];
    const Entries it(a.n, a.r);
    unsigned b = 0;
    // v = X (Y may be X: every entry is read and written by its own thread)
    for (int row = it.row0, j = it.j0; row < a.n; it.next(row, j))
        a.Wa[(size_t)row * a.ldw + j] = a.X[(size_t)row * a.ldx + j];
    for (int sub = 0; sub < a.substeps; ++sub) {
        for (int row = it.row0, j = it.j0; row < a.n; it.next(row, j))   // p = d_0 v
            a.Y[(size_t)row * a.ldy + j] = a.dd[0] * a.Wa[(size_t)row * a.ldw + j];
        if (!grid_barrier(a.bar, ++b, nullptr, nullptr, a.status, sh)) return;
        const double* W = a.Wa;
        double* Wn = a.Wb;
        int small = 0;
        for (int k = 1; k < a.terms; ++k) {
            // val holds A^T / g, so w_{k+1} = val w_k - (c/g + x_k) w_k: one FP64
            // FMA per stored entry plus one (FP64 issue is the bound on this part)
            const double beta = a.c * a.invg + a.xi[k - 1], dk = a.dd[k];
            double aw = 0.0, ap = 0.0;
            for (int row = it.row0, j = it.j0; row < a.n; it.next(row, j)) {
                double wn = -beta * __ldcg(W + (size_t)row * a.ldw + j);
                for (int q = a.ptr[row]; q < a.ptr[row + 1]; ++q)
                    wn = fma(a.val[q], __ldcg(W + (size_t)a.idx[q] * a.ldw + j), wn);
                Wn[(size_t)row * a.ldw + j] = wn;
                const double pv = fma(dk, wn, a.Y[(size_t)row * a.ldy + j]);
                a.Y[(size_t)row * a.ldy + j] = pv;
                aw = fma(wn, wn, aw);
                ap = fma(pv, pv, ap);
            }
            block_sum2(aw, ap, sh);
            double* part = a.part + (size_t)(k & 1) * 2 * gridDim.x;
            double* sums = a.sums + 2 * (k & 1);
            if (threadIdx.x == 0) {
                part[2 * blockIdx.x] = aw;
                part[2 * blockIdx.x + 1] = ap;
            }
            if (!grid_barrier(a.bar, ++b, part, sums, a.status, sh)) return;
            const double nw = __ldcg(sums), np = __ldcg(sums + 1);
            // stop after two consecutive terms |d_k| |w_k| <= tol |p|
            if (fabs(dk) * sqrt(nw) <= a.tol * sqrt(np)) ++small;
            else small = 0;
            double* t = const_cast<double*>(W);
            W = Wn;
            Wn = t;
            if (small == 2) break;
        }
        // the next substep starts from v = scale p; the last one leaves Y = scale p
        const bool last = sub + 1 == a.substeps;
        for (int row = it.row0, j = it.j0; row < a.n; it.next(row, j)) {
            const double v = a.scale * a.Y[(size_t)row * a.ldy + j];
            if (last) a.Y[(size_t)row * a.ldy + j] = v;
            else a.Wa[(size_t)row * a.ldw + j] = v;
        }
    }
}

// Y = alpha S X for a sparse S (CSR) and an n x r block X: one thread per entry.
__global__ void __launch_bounds__(256) spmm_kernel(const int* __restrict__ ptr, const int* __restrict__ idx,
                                                   const double* __restrict__ val, int n, int r,
                                                   const double* __restrict__ X, int ldx, double* __restrict__ Y,
                                                   int ldy, double alpha) {
    const size_t total = (size_t)n * r;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int row = (int)(e / r), j = (int)(e % r);
        double y = 0.0;
        for (int q = ptr[row]; q < ptr[row + 1]; ++q) y = fma(val[q], X[(size_t)idx[q] * ldx + j], y);
        Y[(size_t)row * ldy + j] = alpha * y;
    }
}

}  // namespace

void launch_spmm(const int* ptr, const int* idx, const double* val, int n, int r, const double* X, int ldx, double* Y,
                 int ldy, double alpha, cudaStream_t st) {
    if (n <= 0 || r <= 0) return;
    const size_t total = (size_t)n * r;
    const int grid = (int)std::min<size_t>((total + 255) / 256, 152 * 32);
    spmm_kernel<<<grid, 256, 0, st>>>(ptr, idx, val, n, r, X, ldx, Y, ldy, alpha);
}

// Resident blocks per SM (at most eight) and the SM count.
static int leja_per_sm() {
    static const int per = [] {
        int p = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, leja_persistent_kernel, LJ_THREADS, 0);
        return std::max(1, std::min(p, 8));
    }();
    return per;
}

int leja_grid_max() {
    static const int g = [] {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        // as many resident blocks as fit, up to eight per SM
        return std::max(1, sms) * leja_per_sm();
    }();
    return g;
}

dme_status launch_leja_apply(const LejaCall& c, cudaStream_t st) {
    if (c.n <= 0 || c.r <= 0) return DME_OK;
    if (c.terms > 80 || c.terms < 1) return set_error("Leja apply: 1 <= terms <= 80"), DME_EINVAL;
    LejaArgs a;
    a.ptr = c.ptr;
    a.idx = c.idx;
    a.val = c.val;
    a.n = c.n;
    a.r = c.r;
    a.X = c.X;
    a.ldx = c.ldx;
    a.Y = c.Y;
    a.ldy = c.ldy;
    a.Wa = c.Wa;
    a.Wb = c.Wb;
    a.ldw = c.ldw;
    a.c = c.c;
    a.invg = c.invg;
    a.scale = c.scale;
    a.tol = c.tol;
    a.substeps = c.substeps;
    a.terms = c.terms;
    a.part = c.part;
    a.sums = c.sums;
    a.bar = c.bar;
    a.status = c.status;
    for (int i = 0; i < 80; ++i) {
        a.xi[i] = i < c.terms ? c.xi[i] : 0.0;
        a.dd[i] = i < c.terms ? c.dd[i] : 0.0;
    }
    const size_t total = (size_t)c.n * c.r;
    const int grid = (int)std::min<size_t>((total + LJ_THREADS - 1) / LJ_THREADS, (size_t)leja_grid_max());
    // the barrier counter reaches (barriers per launch) x grid: keep it below 2^31
    const long long per_sub = (long long)c.terms * grid;
    const int chunk = (int)std::max<long long>(1, std::min<long long>(c.substeps, (1ll << 31) / per_sub - 1));
    for (int done = 0; done < c.substeps; done += chunk) {
        a.substeps = std::min(chunk, c.substeps - done);
        if (done > 0) {            // continue from the previous launch's result
            a.X = c.Y;
            a.ldx = c.ldy;
        }
        DME_CUDA_TRY(cudaMemsetAsync(c.bar, 0, 2 * sizeof(unsigned), st));
        void* args[] = {&a};
        DME_TRY(coop_launch(reinterpret_cast<const void*>(leja_persistent_kernel), dim3(grid), dim3(LJ_THREADS),
                            args, 0, st, leja_per_sm()));
    }
    return DME_OK;
}

}  // namespace dme
