// X = M^{-1} B by Gauss-Jordan elimination with partial pivoting, all n
// columns in one persistent cooperative launch: the two dense solves of the
// Pade step of the exponential (q R = p, and p^T R12 = p12 - q12 R22).  One
// launch per column (or three, for an LU factorisation and its two triangular
// sweeps) would make a plan of a small matrix a chain of thousands of tiny
// launches; here a column costs one grid barrier.
//
// Column k: every warp scans its own rows (rows gw, gw + W, ... for warp gw of
// W) for the largest |M[i][k]|, i >= k (ties: the smallest row), the blocks
// post their candidates, and the last block to reach the barrier picks the
// pivot row p, swaps rows k and p (columns >= k of M, all of B), scales row k
// by 1 / M[p][k] and releases the others (grid_sync.cuh).  Then every warp
// eliminates column k from its rows i != k:  row_i -= M[i][k] row_k.  After
// the last column B holds M^{-1} B in natural row order.  A zero or NaN
// column sets DEV_SINGULAR and is skipped.
#include "dme_internal.h"
#include "grid_sync.cuh"

#include <algorithm>
#include <condition_variable>
#include <functional>
#include <memory>
#include <mutex>

namespace dme {

namespace {

constexpr int GJ_THREADS = 256;
constexpr int GJ_WARPS = GJ_THREADS / 32;

struct GJArgs {
    double* M;
    int ldm;
    double* B;
    int ldb;
    int n, nrhs;
    double* pv;      // [gridDim] the blocks' candidate |M[i][k]|
    int* pi;         // [gridDim] their rows
    double* info;    // [0]: 1 / pivot of the current column (0: singular, skipped)
    unsigned* bar;   // grid barrier words, zeroed before the launch
    int* status;
    int staged;      // the pivot row goes to shared memory (n + nrhs doubles)
};

// (v, i) beats (w, j): larger value, then smaller row (a total order, so any
// reduction order gives the same winner).
__device__ __forceinline__ bool gj_better(double v, int i, double w, int j) { return v > w || (v == w && i < j); }

__device__ __forceinline__ void gj_warp_best(double& v, int& i) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, off);
        const int oi = __shfl_xor_sync(0xffffffffu, i, off);
        if (gj_better(ov, oi, v, i)) {
            v = ov;
            i = oi;
        }
    }
}

constexpr int GJ_U = 4;   // columns per lane whose loads are in flight together

// x[j] += c y[j] for j < len (lanes over j); y in shared memory when staged.
__device__ __forceinline__ void axpy_row(double* x, const double* y, int len, double c, int lane, bool staged) {
    for (int j0 = lane; j0 < len; j0 += 32 * GJ_U) {
        double xv[GJ_U], yv[GJ_U];
#pragma unroll
        for (int u = 0; u < GJ_U; ++u) {
            const int j = j0 + 32 * u;
            xv[u] = j < len ? __ldcg(x + j) : 0.0;
            yv[u] = j < len ? (staged ? y[j] : __ldcg(y + j)) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < GJ_U; ++u) {
            const int j = j0 + 32 * u;
            if (j < len) x[j] = fma(c, yv[u], xv[u]);
        }
    }
}

// Columns [j0, j1) of rows k and p: swap them (if swap) and scale row k by r.
__device__ __forceinline__ void swap_scale(double* rk, double* rp, int j0, int j1, bool swap, double r) {
    for (int jb = j0 + threadIdx.x; jb < j1; jb += GJ_THREADS * GJ_U) {
        double x[GJ_U], y[GJ_U];
#pragma unroll
        for (int u = 0; u < GJ_U; ++u) {
            const int j = jb + GJ_THREADS * u;
            x[u] = j < j1 ? __ldcg(rk + j) : 0.0;
            y[u] = (j < j1 && swap) ? __ldcg(rp + j) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < GJ_U; ++u) {
            const int j = jb + GJ_THREADS * u;
            if (j < j1) {
                if (swap) rp[j] = x[u];
                rk[j] = (swap ? y[u] : x[u]) * r;
            }
        }
    }
}

__global__ void __launch_bounds__(GJ_THREADS) gj_kernel(const GJArgs a) {
    extern __shared__ double srow[];
    __shared__ double s_v[GJ_WARPS];
    __shared__ int s_i[GJ_WARPS];
    __shared__ int s_last, s_ok, s_p;
    __shared__ double s_piv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int W = gridDim.x * GJ_WARPS, gw = blockIdx.x * GJ_WARPS + warp;
    const int n = a.n;
    unsigned b = 0;
    for (int k = 0; k < n; ++k) {
        // this warp's best candidate row (lanes take every 32nd of its rows)
        double best = -1.0;
        int bi = n;
        const int t0 = k > gw ? (k - gw + W - 1) / W : 0;
        for (long long t = t0 + lane; gw + (long long)W * t < n; t += 32) {
            const int i = (int)(gw + (long long)W * t);
            const double v = fabs(__ldcg(a.M + (size_t)i * a.ldm + k));
            if (gj_better(v, i, best, bi)) {
                best = v;
                bi = i;
            }
        }
        gj_warp_best(best, bi);
        if (lane == 0) {
            s_v[warp] = best;
            s_i[warp] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < GJ_WARPS; ++w)
                if (gj_better(s_v[w], s_i[w], best, bi)) {
                    best = s_v[w];
                    bi = s_i[w];
                }
            a.pv[blockIdx.x] = best;
            a.pi[blockIdx.x] = bi;
        }
        if (gs_arrive(a.bar, ++b, &s_last)) {
            // the pivot over all blocks (strided, then warp and block steps)
            double v = -1.0;
            int p = n;
            for (int g = threadIdx.x; g < (int)gridDim.x; g += GJ_THREADS) {
                const double gv = __ldcg(a.pv + g);
                const int gi = __ldcg(a.pi + g);
                if (gj_better(gv, gi, v, p)) {
                    v = gv;
                    p = gi;
                }
            }
            gj_warp_best(v, p);
            __syncthreads();
            if (lane == 0) {
                s_v[warp] = v;
                s_i[warp] = p;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int w = 0; w < GJ_WARPS; ++w)
                    if (gj_better(s_v[w], s_i[w], v, p)) {
                        v = s_v[w];
                        p = s_i[w];
                    }
                if (!(v > 0.0) || p < k || p >= n) {
                    atomicOr(a.status, DEV_SINGULAR);
                    s_p = k;
                    s_piv = 0.0;
                } else {
                    s_p = p;
                    s_piv = __ldcg(a.M + (size_t)p * a.ldm + k);
                }
            }
            __syncthreads();
            const int pr = s_p;
            const double r = s_piv != 0.0 ? 1.0 / s_piv : 0.0;
            double* Mk = a.M + (size_t)k * a.ldm;
            double* Mp = a.M + (size_t)pr * a.ldm;
            double* Bk = a.B + (size_t)k * a.ldb;
            double* Bp = a.B + (size_t)pr * a.ldb;
            // swap rows k and p, then scale row k (each thread owns its columns j;
            // GJ_U columns' loads are issued before any store)
            swap_scale(Mk, Mp, k + 1, n, pr != k, r);
            swap_scale(Bk, Bp, 0, a.nrhs, pr != k, r);
            if (threadIdx.x == 0) {
                if (pr != k) {            // column k itself: row p takes row k's entry
                    const double x = __ldcg(Mk + k);
                    Mk[k] = s_piv;
                    Mp[k] = x;
                }
                a.info[0] = r;
            }
            gs_release(a.bar, b);
            __syncthreads();
        } else if (!gs_wait(a.bar, b, a.status, &s_ok)) {
            return;
        }
        // eliminate column k from this warp's rows i != k; the pivot row is staged
        // in shared memory once per block when it fits
        const double r = __ldcg(a.info);
        if (r != 0.0) {
            const double* Mk = a.M + (size_t)k * a.ldm + (k + 1);
            const double* Bk = a.B + (size_t)k * a.ldb;
            const int lm = n - k - 1;
            if (a.staged) {
                for (int j = threadIdx.x; j < lm; j += GJ_THREADS) srow[j] = __ldcg(Mk + j);
                for (int j = threadIdx.x; j < a.nrhs; j += GJ_THREADS) srow[lm + j] = __ldcg(Bk + j);
                __syncthreads();
                Mk = srow;
                Bk = srow + lm;
            }
            for (int i = gw; i < n; i += W) {
                if (i == k) continue;
                double* Mi = a.M + (size_t)i * a.ldm + (k + 1);
                double* Bi = a.B + (size_t)i * a.ldb;
                const double f = __ldcg(a.M + (size_t)i * a.ldm + k);
                if (f == 0.0) continue;
                axpy_row(Mi, Mk, lm, -f, lane, a.staged);
                axpy_row(Bi, Bk, a.nrhs, -f, lane, a.staged);
            }
        }
        __syncthreads();
    }
}

constexpr size_t kGJMaxSmem = 200 * 1024;   // largest staged pivot row

int gj_sms() {
    static const int sms = [] {
        int dev = 0, c = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
        return std::max(c, 1);
    }();
    return sms;
}

// Blocks per SM, at most four (the grid is sized by the rows anyway).
int gj_blocks_per_sm(size_t smem) {
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, gj_kernel, GJ_THREADS, smem);
    return std::max(0, std::min(per, 4));
}

// One block waits at a grid barrier whose release word nothing writes: the
// bounded wait of grid_sync.cuh must give up and report DEV_TIMEOUT.
__global__ void wait_timeout_selftest_kernel(unsigned* bar, int* status) {
    __shared__ int s_ok;
    gs_wait(bar, 1u, status, &s_ok);
}

}  // namespace

dme_status wait_timeout_selftest(int* timed_out) {
    cudaStream_t st = nullptr;
    DME_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    std::unique_ptr<CUstream_st, void (*)(cudaStream_t)> sg(st, [](cudaStream_t x) { cudaStreamDestroy(x); });
    int* words = nullptr;
    DME_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&words), 4 * sizeof(int), st));
    std::unique_ptr<int, std::function<void(int*)>> wg(words, [st](int* p) {
        cudaFreeAsync(p, st);
        cudaStreamSynchronize(st);
    });
    DME_CUDA_TRY(cudaMemsetAsync(words, 0, 4 * sizeof(int), st));
    wait_timeout_selftest_kernel<<<1, 32, 0, st>>>(reinterpret_cast<unsigned*>(words), words + 2);
    DME_CUDA_TRY(cudaGetLastError());
    int hs = 0;
    DME_CUDA_TRY(cudaMemcpyAsync(&hs, words + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
    DME_CUDA_TRY(cudaStreamSynchronize(st));
    *timed_out = (hs & DEV_TIMEOUT) ? 1 : 0;
    return DME_OK;
}

dme_status coop_launch(const void* func, dim3 grid, dim3 block, void** args, size_t smem, cudaStream_t st,
                       int blocks_per_sm) {
    // Admission: kernels with at least 4 blocks per SM run together while their grids sum
    // to at most 4 blocks per SM (every such mix is co-resident); any other launch runs alone.
    static std::mutex mu;
    static std::condition_variable cv;
    static long inflight = 0;
    const long cap = 4L * gj_sms();
    const long weight = (blocks_per_sm >= 4 && (long)grid.x <= cap) ? (long)grid.x : cap;
    DME_CUDA_TRY(cudaStreamSynchronize(st));
    {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return inflight == 0 || inflight + weight <= cap; });
        inflight += weight;
    }
    cudaError_t e = cudaLaunchCooperativeKernel(func, grid, block, args, smem, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    {
        std::lock_guard<std::mutex> g(mu);
        inflight -= weight;
    }
    cv.notify_all();
    if (e != cudaSuccess) return set_error(std::string("cooperative launch: ") + cudaGetErrorString(e)), DME_ECUDA;
    return DME_OK;
}

size_t gj_work_doubles() { return 2 * (size_t)gj_sms() * 4 + 4; }

dme_status launch_gj_solve(double* M, int n, int ldm, double* B, int nrhs, int ldb, double* work, int* status,
                           cudaStream_t st) {
    if (n <= 0) return DME_OK;
    static const cudaError_t attr =
        cudaFuncSetAttribute(gj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGJMaxSmem);
    DME_CUDA_TRY(attr);
    const size_t row = sizeof(double) * ((size_t)n + nrhs);
    const bool staged = row <= kGJMaxSmem;
    const size_t smem = staged ? row : 0;
    const int per = gj_blocks_per_sm(smem);
    if (per < 1) return set_error("Gauss-Jordan solve: no block fits on an SM"), DME_EINVAL;
    const int gmax = gj_sms() * per;
    const int grid = std::max(1, std::min(gmax, (n + GJ_WARPS - 1) / GJ_WARPS));
    GJArgs a;
    a.M = M;
    a.ldm = ldm;
    a.B = B;
    a.ldb = ldb;
    a.n = n;
    a.nrhs = nrhs;
    const size_t cap = (size_t)gj_sms() * 4;   // layout of work: pv[cap], pi[cap], info, bar
    a.pv = work;
    a.pi = reinterpret_cast<int*>(work + cap);
    a.info = work + 2 * cap;
    a.bar = reinterpret_cast<unsigned*>(work + 2 * cap + 2);
    a.status = status;
    a.staged = staged ? 1 : 0;
    DME_CUDA_TRY(cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), st));
    void* args[] = {&a};
    return coop_launch(reinterpret_cast<const void*>(gj_kernel), dim3(grid), dim3(GJ_THREADS), args, smem, st,
                       per);
}

}  // namespace dme
