// X = M^{-1} B by Gauss-Jordan elimination with partial pivoting, blocked by
// panels of GJ_NB columns: the two dense solves of the Pade step of the
// exponential (q R = p, and p^T R12 = p12 - q12 R22), and dme_plan_mass's
// inverse.  For n <= GJP_MAX_N the panel path further down (a cluster launch
// per panel, no grid barriers); above it one persistent cooperative launch:
//
// Panel [k0, k1), k1 = min(k0 + GJ_NB, n).  Column k of the panel: every
// thread scans its rows i >= k for the largest |M[i][k]| (ties: the smallest
// row), the blocks post their candidates, and the last block to reach the
// grid barrier picks the pivot row p, exchanges rows k and p within the
// panel's columns, scales row k's panel entries right of k by 1 / pivot
// (keeping the pivot itself at (k, k)) and releases the others; each thread
// then eliminates column k from its rows i != k within the panel's columns,
// leaving the multiplier f = M[i][k] in place.  After the last column the
// panel's columns hold every row's multipliers, and the pivot rows also their
// pivots.  The remaining columns (M's right of the panel, then B's: the
// trailing block R) are brought up to date in two passes instead of GJ_NB:
//   S/V (a thread per trailing column): apply the panel's row exchanges in
//     order, then form the pivot rows as sequential elimination would leave
//     them when they are scaled,
//       V_c = (R_{k0+c} - sum_{c' < c} M[k0+c][k0+c'] V_{c'}) / M[k0+c][k0+c];
//   U (tiles of rows x columns): R_i -= sum_c M[i][k0+c] V_c for the other
//     rows, and R_{k0+c} = V_c - sum_{c' > c} M[k0+c][k0+c'] V_{c'} for the
//     pivot rows (the later columns of the panel eliminate them too).
// This is the same elimination as column by column (the multipliers travel
// with their rows through the exchanges), with the trailing block read and
// written once per panel; its sums run in a fixed order, so the result does
// not depend on the grid.  GJ_NB + 2 grid barriers per panel.  After the last
// panel B holds M^{-1} B in natural row order.  A zero or NaN pivot column
// sets DEV_SINGULAR; its pivot is stored as 0 and its row of V is 0.
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
constexpr int GJ_NB = 16;          // panel width

struct GJArgs {
    double* M;
    int ldm;
    double* B;
    int ldb;
    int n, nrhs;
    double* pv;      // [gridDim] the blocks' candidate |M[i][k]|
    int* pi;         // [gridDim] their rows
    double* info;    // [0]: the pivot of the current column (0: singular, skipped)
    unsigned* bar;   // grid barrier words, zeroed before the launch
    int* status;
    int* perm;       // [GJ_NB] the current panel's pivot rows, in column order
    double* V;       // [GJ_NB][ldv] the panel's transformed pivot rows over the trailing columns
    int ldv;         // n + nrhs
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

// The block's best (v, i) into pv/pi[blockIdx.x] (thread 0 writes).
__device__ __forceinline__ void gj_post_candidate(const GJArgs& a, double v, int i, double* s_v, int* s_i) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    gj_warp_best(v, i);
    __syncthreads();
    if (lane == 0) {
        s_v[warp] = v;
        s_i[warp] = i;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < GJ_WARPS; ++w)
            if (gj_better(s_v[w], s_i[w], v, i)) {
                v = s_v[w];
                i = s_i[w];
            }
        a.pv[blockIdx.x] = v;
        a.pi[blockIdx.x] = i;
    }
}

// Entry (i, t) of the trailing block of a panel ending at column k1: M's
// columns k1 .. n-1, then B's columns.
__device__ __forceinline__ double* gj_trail(const GJArgs& a, int k1, int i, int t) {
    const int mt = a.n - k1;
    return t < mt ? a.M + (size_t)i * a.ldm + k1 + t : a.B + (size_t)i * a.ldb + (t - mt);
}

// Update tiles of TM rows x TM trailing columns, (TM / 16)^2 outputs per thread.
template <int TM>
__global__ void __launch_bounds__(GJ_THREADS, 4) gj_kernel(const GJArgs a) {
    constexpr int RM = TM / 16;
    __shared__ double sF[TM][GJ_NB + 1];       // U: the tile rows' multipliers
    __shared__ double sV[GJ_NB][TM];           // U: the panel's V over the tile's columns
    __shared__ double sL[GJ_NB][GJ_NB + 1];    // S/V: the pivot rows' panel entries
    __shared__ double sR[GJ_NB];               // S/V: 1 / pivot (0: singular column)
    __shared__ double sP[GJ_NB];               // the current pivot row right of its column
    __shared__ int sPerm[GJ_NB];
    __shared__ double s_v[GJ_WARPS];
    __shared__ int s_i[GJ_WARPS];
    __shared__ int s_last, s_ok, s_p;
    __shared__ double s_piv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = a.n;
    const int T = gridDim.x * GJ_THREADS, gt = blockIdx.x * GJ_THREADS + threadIdx.x;
    unsigned b = 0;
    for (int k0 = 0; k0 < n; k0 += GJ_NB) {
        const int k1 = min(k0 + GJ_NB, n), nbk = k1 - k0;
        // candidates for the panel's first column (its values after the last update)
        double best = -1.0;
        int bi = n;
        for (int i = gt; i < n; i += T) {
            if (i < k0) continue;
            const double v = fabs(__ldcg(a.M + (size_t)i * a.ldm + k0));
            if (gj_better(v, i, best, bi)) {
                best = v;
                bi = i;
            }
        }
        for (int k = k0; k < k1; ++k) {
            gj_post_candidate(a, best, bi, s_v, s_i);
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
                    const bool singular = !(v > 0.0) || p < k || p >= n;
                    if (singular) {
                        atomicOr(a.status, DEV_SINGULAR);
                        p = k;
                    }
                    s_p = p;
                    s_piv = singular ? 0.0 : __ldcg(a.M + (size_t)p * a.ldm + k);
                    a.perm[k - k0] = p;
                    a.info[0] = s_piv;
                }
                __syncthreads();
                // rows k and p exchange their panel entries; row k's entries right of k are
                // scaled by 1 / pivot, the pivot stays at (k, k), the multipliers left of k stay
                const int pr = s_p;
                const double piv = s_piv;
                const double r = piv != 0.0 ? 1.0 / piv : 0.0;
                if (threadIdx.x < nbk) {
                    const int c = k0 + threadIdx.x;
                    double* Mk = a.M + (size_t)k * a.ldm;
                    double* Mp = a.M + (size_t)pr * a.ldm;
                    const double x = __ldcg(Mk + c);
                    const double y = pr != k ? __ldcg(Mp + c) : x;
                    if (pr != k) Mp[c] = x;
                    Mk[c] = c > k ? y * r : (c == k ? piv : y);
                }
                gs_release(a.bar, b);
                __syncthreads();
            } else if (!gs_wait(a.bar, b, a.status, &s_ok)) {
                return;
            }
            // eliminate column k from this thread's rows within the panel (the multiplier
            // stays at (i, k)), and find the next column's candidates among them
            if (threadIdx.x < GJ_NB) {
                const int c = k + 1 + threadIdx.x;
                sP[threadIdx.x] = c < k1 ? __ldcg(a.M + (size_t)k * a.ldm + c) : 0.0;
            }
            __syncthreads();
            const double piv = __ldcg(a.info);
            best = -1.0;
            bi = n;
            for (int i = gt; i < n; i += T) {
                double* Mi = a.M + (size_t)i * a.ldm;
                if (i != k && piv != 0.0) {
                    const double f = __ldcg(Mi + k);
                    if (f != 0.0)
                        for (int c = k + 1; c < k1; ++c) Mi[c] = fma(-f, sP[c - k - 1], __ldcg(Mi + c));
                }
                if (k + 1 < k1 && i > k) {
                    const double v = fabs(__ldcg(Mi + k + 1));
                    if (gj_better(v, i, best, bi)) {
                        best = v;
                        bi = i;
                    }
                }
            }
        }
        // S/V: a thread per trailing column applies the panel's row exchanges in order and
        // forms the transformed pivot rows V (kept in a.V; the pivot rows are written in U)
        const int mtt = n - k1 + a.nrhs;
        {
            const int c = threadIdx.x / GJ_NB, c2 = threadIdx.x % GJ_NB;   // GJ_THREADS == GJ_NB^2
            sL[c][c2] = (c < nbk && c2 < nbk) ? __ldcg(a.M + (size_t)(k0 + c) * a.ldm + k0 + c2) : 0.0;
            if (threadIdx.x < GJ_NB) sPerm[threadIdx.x] = threadIdx.x < nbk ? __ldcg(a.perm + threadIdx.x) : 0;
        }
        __syncthreads();
        if (threadIdx.x < GJ_NB) {
            const double pv = sL[threadIdx.x][threadIdx.x];
            sR[threadIdx.x] = pv != 0.0 ? 1.0 / pv : 0.0;
        }
        __syncthreads();
        for (int t = gt; t < mtt; t += T) {
            for (int c = 0; c < nbk; ++c) {
                const int p = sPerm[c], r = k0 + c;
                if (p != r) {
                    double* x = gj_trail(a, k1, r, t);
                    double* y = gj_trail(a, k1, p, t);
                    const double xv = __ldcg(x), yv = __ldcg(y);
                    *x = yv;
                    *y = xv;
                }
            }
            double v[GJ_NB];
#pragma unroll
            for (int c = 0; c < GJ_NB; ++c) {
                v[c] = 0.0;
                if (c < nbk) {
                    double x = __ldcg(gj_trail(a, k1, k0 + c, t));
#pragma unroll
                    for (int c2 = 0; c2 < c; ++c2) x = fma(-sL[c][c2], v[c2], x);
                    v[c] = x * sR[c];
                    a.V[(size_t)c * a.ldv + t] = v[c];
                }
            }
        }
        if (gs_arrive(a.bar, ++b, &s_last)) {
            gs_release(a.bar, b);
        } else if (!gs_wait(a.bar, b, a.status, &s_ok)) {
            return;
        }
        // U: R_i -= sum_c M[i][k0+c] V_c (other rows); R_{k0+c} = V_c - sum_{c' > c} ... (pivot rows)
        const int ntc = (mtt + TM - 1) / TM, ntiles = ((n + TM - 1) / TM) * ntc;
        const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int row0 = (tile / ntc) * TM, t0 = (tile % ntc) * TM;
            __syncthreads();
            for (int e = threadIdx.x; e < TM * GJ_NB; e += GJ_THREADS) {
                const int r = e / GJ_NB, c = e % GJ_NB, i = row0 + r;
                const bool live = i < n && c < nbk && !(i >= k0 && i < k1 && c <= i - k0);
                sF[r][c] = live ? __ldcg(a.M + (size_t)i * a.ldm + k0 + c) : 0.0;
            }
            for (int e = threadIdx.x; e < GJ_NB * TM; e += GJ_THREADS) {
                const int c = e / TM, tt = e % TM, t = t0 + tt;
                sV[c][tt] = (c < nbk && t < mtt) ? __ldcg(a.V + (size_t)c * a.ldv + t) : 0.0;
            }
            __syncthreads();
            double acc[RM][RM];
#pragma unroll
            for (int rr = 0; rr < RM; ++rr) {
                const int i = row0 + ty + 16 * rr;
#pragma unroll
                for (int cc = 0; cc < RM; ++cc) {
                    const int tt = tx + 16 * cc, t = t0 + tt;
                    acc[rr][cc] = 0.0;
                    if (i < n && t < mtt)
                        acc[rr][cc] = (i >= k0 && i < k1) ? sV[i - k0][tt] : __ldcg(gj_trail(a, k1, i, t));
                }
            }
#pragma unroll
            for (int c = 0; c < GJ_NB; ++c) {
                double fr[RM], vc[RM];
#pragma unroll
                for (int rr = 0; rr < RM; ++rr) fr[rr] = sF[ty + 16 * rr][c];
#pragma unroll
                for (int cc = 0; cc < RM; ++cc) vc[cc] = sV[c][tx + 16 * cc];
#pragma unroll
                for (int rr = 0; rr < RM; ++rr)
#pragma unroll
                    for (int cc = 0; cc < RM; ++cc) acc[rr][cc] = fma(-fr[rr], vc[cc], acc[rr][cc]);
            }
#pragma unroll
            for (int rr = 0; rr < RM; ++rr) {
                const int i = row0 + ty + 16 * rr;
#pragma unroll
                for (int cc = 0; cc < RM; ++cc) {
                    const int t = t0 + tx + 16 * cc;
                    if (i < n && t < mtt) *gj_trail(a, k1, i, t) = acc[rr][cc];
                }
            }
        }
        if (k1 < n) {
            // the next panel reads the updated columns
            if (gs_arrive(a.bar, ++b, &s_last)) {
                gs_release(a.bar, b);
            } else if (!gs_wait(a.bar, b, a.status, &s_ok)) {
                return;
            }
        }
    }
}

// Blocks per SM, at most four (the grid is sized by the work anyway).
template <int TM>
int gj_blocks_per_sm() {
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, gj_kernel<TM>, GJ_THREADS, 0);
    return std::max(0, std::min(per, 4));
}

int gj_sms() {
    static const int sms = [] {
        int dev = 0, c = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev);
        return std::max(c, 1);
    }();
    return sms;
}

// ---------------------------------------------------------------------------
// The same elimination for n <= GJP_MAX_N without grid barriers: per panel,
// one launch factors the panel in a thread-block cluster, one forms V, one
// updates the trailing block, all stream-ordered.  Rows are not exchanged:
// the pivot of column k is a physical row pr[k] marked used, every other row
// (used or not) is eliminated, and after the last panel the solution of
// unknown k is row pr[k] of B, gathered into place.  The arithmetic per
// entry is that of the exchanging form above.

constexpr int GJP_MAX_N = 4096;
constexpr int GJP_LD = GJ_NB + 1;       // shared-memory row stride of a panel (doubles)
constexpr int GJP_MAX_ROWS = 512;       // panel rows per CTA of the cluster

struct GJPanelArgs {
    double* M;
    int ldm;
    int n, k0, nbk;
    int rows_per;    // panel rows per CTA
    int* used;       // [n] rows already chosen as pivots
    int* pr;         // [n] pivot row of each column
    int* status;
};

__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_nrank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_map(const void* p, uint32_t rank) {
    uint32_t r;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ double cl_ld_f64(uint32_t a) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ int cl_ld_s32(uint32_t a) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
// Every thread of every CTA of the cluster; orders shared-memory writes before it
// with reads after it, across the cluster.
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Factor panel [k0, k0 + nbk) of rows 0..n-1: CTA `rank` of the cluster holds rows
// [rank * rows_per, ...) of the panel in shared memory.  Column c: each CTA's best
// unused row, one cluster barrier, every CTA reads all candidates and the winning
// row's entries from its owner (distributed shared memory) and eliminates column c
// from its own rows with the scaled pivot row; the owner writes the pivot row's
// scaled entries after the next barrier (other CTAs may still be reading them).
__global__ void __launch_bounds__(GJ_THREADS) gj_panel_kernel(const GJPanelArgs a) {
    extern __shared__ double sP[];                       // [rows_per][GJP_LD], then used flags
    int* sU = reinterpret_cast<int*>(sP + (size_t)a.rows_per * GJP_LD);
    __shared__ double s_cv[2];                           // this CTA's candidate, by column parity
    __shared__ int s_ci[2];
    __shared__ double s_wv[GJ_WARPS];
    __shared__ int s_wi[GJ_WARPS];
    __shared__ double s_raw[GJ_NB];                      // the pivot row's panel entries
    __shared__ double s_sc[GJ_NB];                       // ... scaled right of the pivot
    __shared__ double s_pend[GJ_NB];                     // deferred write of this CTA's last pivot row
    __shared__ int s_p, s_pend_r, s_pend_c;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rank = (int)cl_rank(), ncl = (int)cl_nrank();
    const int n = a.n, nbk = a.nbk, k0 = a.k0;
    const int r0 = rank * a.rows_per;
    const int nr = max(0, min(a.rows_per, n - r0));
    for (int e = threadIdx.x; e < nr * nbk; e += GJ_THREADS) {
        const int r = e / nbk, c = e % nbk;
        sP[r * GJP_LD + c] = __ldcg(a.M + (size_t)(r0 + r) * a.ldm + k0 + c);
    }
    for (int r = threadIdx.x; r < nr; r += GJ_THREADS) sU[r] = __ldcg(a.used + r0 + r);
    if (threadIdx.x == 0) s_pend_r = -1;
    __syncthreads();
    for (int c = 0; c < nbk; ++c) {
        double best = -1.0;
        int bi = n;
        for (int r = threadIdx.x; r < nr; r += GJ_THREADS) {
            if (sU[r]) continue;
            double v = fabs(sP[r * GJP_LD + c]);
            if (!(v == v)) v = 0.0;                      // NaN: a zero pivot if nothing better
            if (gj_better(v, r0 + r, best, bi)) {
                best = v;
                bi = r0 + r;
            }
        }
        gj_warp_best(best, bi);
        if (lane == 0) {
            s_wv[warp] = best;
            s_wi[warp] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < GJ_WARPS; ++w)
                if (gj_better(s_wv[w], s_wi[w], best, bi)) {
                    best = s_wv[w];
                    bi = s_wi[w];
                }
            s_cv[c & 1] = best;
            s_ci[c & 1] = bi;
        }
        cl_sync();
        // the previous column's pivot row (owned here) takes its scaled entries before
        // this column eliminates it (no other CTA reads that row any more)
        if (s_pend_r >= 0 && threadIdx.x < nbk && threadIdx.x >= s_pend_c)
            sP[s_pend_r * GJP_LD + threadIdx.x] = s_pend[threadIdx.x];
        __syncthreads();
        // the pivot over the cluster, then its row's entries from its owner
        if (warp == 0) {
            double v = -1.0;
            int p = n;
            if (lane < ncl) {
                v = cl_ld_f64(cl_map(&s_cv[c & 1], lane));
                p = cl_ld_s32(cl_map(&s_ci[c & 1], lane));
            }
            gj_warp_best(v, p);
            const bool singular = !(v > 0.0);
            if (p >= n) p = n - 1;                       // cannot happen: an unused row remains
            const int owner = p / a.rows_per, pl = p - owner * a.rows_per;
            if (lane < nbk) s_raw[lane] = cl_ld_f64(cl_map(&sP[pl * GJP_LD + lane], owner));
            __syncwarp();
            const double piv = singular ? 0.0 : s_raw[c];
            const double rp = piv != 0.0 ? 1.0 / piv : 0.0;
            if (lane < nbk) s_sc[lane] = lane > c ? s_raw[lane] * rp : 0.0;
            if (owner == rank && lane < nbk) s_pend[lane] = lane > c ? s_raw[lane] * rp : (lane == c ? piv : 0.0);
            if (lane == 0) {
                s_p = p;
                s_pend_r = owner == rank ? pl : -1;
                s_pend_c = c;
                if (singular && rank == 0) atomicOr(a.status, DEV_SINGULAR);
                if (owner == rank) {
                    sU[pl] = 1;
                    a.pr[k0 + c] = p;
                }
            }
        }
        __syncthreads();
        // eliminate column c from this CTA's rows other than the pivot row
        const int p = s_p;
        for (int r = threadIdx.x; r < nr; r += GJ_THREADS) {
            if (r0 + r == p) continue;
            double* row = sP + r * GJP_LD;
            const double f = row[c];
            if (f == 0.0) continue;
            for (int c2 = c + 1; c2 < nbk; ++c2) row[c2] = fma(-f, s_sc[c2], row[c2]);
        }
        __syncthreads();
    }
    cl_sync();                                           // nobody reads this CTA's rows any more
    if (s_pend_r >= 0 && threadIdx.x < nbk && threadIdx.x >= s_pend_c)
        sP[s_pend_r * GJP_LD + threadIdx.x] = s_pend[threadIdx.x];
    __syncthreads();
    for (int e = threadIdx.x; e < nr * nbk; e += GJ_THREADS) {
        const int r = e / nbk, c = e % nbk;
        a.M[(size_t)(r0 + r) * a.ldm + k0 + c] = sP[r * GJP_LD + c];
    }
    for (int r = threadIdx.x; r < nr; r += GJ_THREADS) a.used[r0 + r] = sU[r];
}

struct GJTrailArgs {
    double* M;
    int ldm;
    double* B;
    int ldb;
    int n, nrhs;
    int k0, k1;
    const int* pr;   // [n] pivot rows (this panel's at k0 .. k1-1)
    double* V;       // [GJ_NB][ldv]
    int ldv;
};

__device__ __forceinline__ double* gjt_at(const GJTrailArgs& a, int i, int t) {
    const int mt = a.n - a.k1;
    return t < mt ? a.M + (size_t)i * a.ldm + a.k1 + t : a.B + (size_t)i * a.ldb + (t - mt);
}

// V_c = (R[pr_c] - sum_{c' < c} M[pr_c][k0+c'] V_{c'}) / M[pr_c][k0+c], a thread per
// trailing column.
__global__ void __launch_bounds__(GJ_THREADS) gj_v_kernel(const GJTrailArgs a) {
    __shared__ double sL[GJ_NB][GJ_NB + 1];
    __shared__ double sR[GJ_NB];
    __shared__ int sPr[GJ_NB];
    const int nbk = a.k1 - a.k0;
    {
        const int c = threadIdx.x / GJ_NB, c2 = threadIdx.x % GJ_NB;
        sL[c][c2] = (c < nbk && c2 < nbk) ? __ldcg(a.M + (size_t)__ldcg(a.pr + a.k0 + c) * a.ldm + a.k0 + c2) : 0.0;
        if (threadIdx.x < GJ_NB) sPr[threadIdx.x] = threadIdx.x < nbk ? __ldcg(a.pr + a.k0 + threadIdx.x) : 0;
    }
    __syncthreads();
    if (threadIdx.x < GJ_NB) {
        const double pv = sL[threadIdx.x][threadIdx.x];
        sR[threadIdx.x] = pv != 0.0 ? 1.0 / pv : 0.0;
    }
    __syncthreads();
    const int mtt = a.n - a.k1 + a.nrhs;
    const int t = blockIdx.x * GJ_THREADS + threadIdx.x;
    if (t >= mtt) return;
    double v[GJ_NB];
#pragma unroll
    for (int c = 0; c < GJ_NB; ++c) {
        v[c] = 0.0;
        if (c < nbk) {
            double x = __ldcg(gjt_at(a, sPr[c], t));
#pragma unroll
            for (int c2 = 0; c2 < c; ++c2) x = fma(-sL[c][c2], v[c2], x);
            v[c] = x * sR[c];
            a.V[(size_t)c * a.ldv + t] = v[c];
        }
    }
}

// One TM x TM tile of the trailing update: R_i -= sum_c M[i][k0+c] V_c for rows that
// are not this panel's pivots, R_{pr_c} = V_c - sum_{c' > c} M[pr_c][k0+c'] V_{c'}.
template <int TM>
__global__ void __launch_bounds__(GJ_THREADS) gj_update_kernel(const GJTrailArgs a) {
    constexpr int RM = TM / 16;
    __shared__ double sF[TM][GJ_NB + 1];
    __shared__ double sV[GJ_NB][TM];
    __shared__ int sPr[GJ_NB];
    __shared__ int sC[TM];                               // the tile row's panel column, or -1
    const int nbk = a.k1 - a.k0;
    const int mtt = a.n - a.k1 + a.nrhs;
    const int ntc = (mtt + TM - 1) / TM;
    const int row0 = (blockIdx.x / ntc) * TM, t0 = (blockIdx.x % ntc) * TM;
    if (threadIdx.x < GJ_NB) sPr[threadIdx.x] = threadIdx.x < nbk ? __ldcg(a.pr + a.k0 + threadIdx.x) : -1;
    __syncthreads();
    for (int r = threadIdx.x; r < TM; r += GJ_THREADS) {
        int cr = -1;
        for (int c = 0; c < nbk; ++c)
            if (sPr[c] == row0 + r) cr = c;
        sC[r] = cr;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TM * GJ_NB; e += GJ_THREADS) {
        const int r = e / GJ_NB, c = e % GJ_NB, i = row0 + r;
        const bool live = i < a.n && c < nbk && c > sC[r];
        sF[r][c] = live ? __ldcg(a.M + (size_t)i * a.ldm + a.k0 + c) : 0.0;
    }
    for (int e = threadIdx.x; e < GJ_NB * TM; e += GJ_THREADS) {
        const int c = e / TM, tt = e % TM, t = t0 + tt;
        sV[c][tt] = (c < nbk && t < mtt) ? __ldcg(a.V + (size_t)c * a.ldv + t) : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[RM][RM];
#pragma unroll
    for (int rr = 0; rr < RM; ++rr) {
        const int r = ty + 16 * rr, i = row0 + r;
#pragma unroll
        for (int cc = 0; cc < RM; ++cc) {
            const int tt = tx + 16 * cc, t = t0 + tt;
            acc[rr][cc] = 0.0;
            if (i < a.n && t < mtt) acc[rr][cc] = sC[r] >= 0 ? sV[sC[r]][tt] : __ldcg(gjt_at(a, i, t));
        }
    }
#pragma unroll
    for (int c = 0; c < GJ_NB; ++c) {
        double fr[RM], vc[RM];
#pragma unroll
        for (int rr = 0; rr < RM; ++rr) fr[rr] = sF[ty + 16 * rr][c];
#pragma unroll
        for (int cc = 0; cc < RM; ++cc) vc[cc] = sV[c][tx + 16 * cc];
#pragma unroll
        for (int rr = 0; rr < RM; ++rr)
#pragma unroll
            for (int cc = 0; cc < RM; ++cc) acc[rr][cc] = fma(-fr[rr], vc[cc], acc[rr][cc]);
    }
#pragma unroll
    for (int rr = 0; rr < RM; ++rr) {
        const int i = row0 + ty + 16 * rr;
#pragma unroll
        for (int cc = 0; cc < RM; ++cc) {
            const int t = t0 + tx + 16 * cc;
            if (i < a.n && t < mtt) *gjt_at(a, i, t) = acc[rr][cc];
        }
    }
}

// X[k][j] = B[pr[k]][j] (row k of the solution sits in pivot row pr[k]).
__global__ void gj_gather_kernel(const double* B, int ldb, const int* pr, int n, int nrhs, double* X) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)n * nrhs) return;
    const int k = (int)(e / nrhs), j = (int)(e % nrhs);
    X[e] = B[(size_t)__ldg(pr + k) * ldb + j];
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

// Layout of work: pv[cap], pi[cap], info[2], bar (2 words), perm (GJ_NB ints),
// V[GJ_NB][n + nrhs], then (panel path) used and pr (n ints each) and the
// gathered solution (n x nrhs); cap = 4 blocks per SM.
size_t gj_work_doubles(int n, int nrhs) {
    const size_t nn = (size_t)std::max(n, 0), nr = (size_t)std::max(nrhs, 0);
    return 2 * (size_t)gj_sms() * 4 + 16 + (size_t)GJ_NB * (nn + nr) + nn + nn * nr;
}

// The panel path: per panel a cluster launch (factor), then V and the trailing
// update; finally the gather of the solution rows.
static dme_status gj_solve_panels(double* M, int n, int ldm, double* B, int nrhs, int ldb, double* V, int* used,
                                  int* pr, double* X, int* status, cudaStream_t st) {
    const int cl = std::max(1, std::min(8, (n + 127) / 128));
    const int rows_per = (n + cl - 1) / cl;
    const size_t smem = (size_t)rows_per * GJP_LD * sizeof(double) + (size_t)rows_per * sizeof(int);
    static const cudaError_t attr = cudaFuncSetAttribute(
        gj_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)((size_t)GJP_MAX_ROWS * GJP_LD * sizeof(double) + GJP_MAX_ROWS * sizeof(int)));
    DME_CUDA_TRY(attr);
    if (rows_per > GJP_MAX_ROWS) return set_error("Gauss-Jordan solve: panel too tall"), DME_EINVAL;
    DME_CUDA_TRY(cudaMemsetAsync(used, 0, sizeof(int) * (size_t)n, st));
    const int sms = gj_sms();
    for (int k0 = 0; k0 < n; k0 += GJ_NB) {
        const int k1 = std::min(k0 + GJ_NB, n);
        GJPanelArgs pa;
        pa.M = M;
        pa.ldm = ldm;
        pa.n = n;
        pa.k0 = k0;
        pa.nbk = k1 - k0;
        pa.rows_per = rows_per;
        pa.used = used;
        pa.pr = pr;
        pa.status = status;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cl);
        cfg.blockDim = dim3(GJ_THREADS);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        DME_CUDA_TRY(cudaLaunchKernelEx(&cfg, gj_panel_kernel, pa));
        const int mtt = n - k1 + nrhs;
        if (mtt <= 0) continue;
        GJTrailArgs ta;
        ta.M = M;
        ta.ldm = ldm;
        ta.B = B;
        ta.ldb = ldb;
        ta.n = n;
        ta.nrhs = nrhs;
        ta.k0 = k0;
        ta.k1 = k1;
        ta.pr = pr;
        ta.V = V;
        ta.ldv = n + nrhs;
        gj_v_kernel<<<(mtt + GJ_THREADS - 1) / GJ_THREADS, GJ_THREADS, 0, st>>>(ta);
        const long t64 = (long)((n + 63) / 64) * ((mtt + 63) / 64);
        if (t64 >= 2L * sms)
            gj_update_kernel<64><<<(unsigned)t64, GJ_THREADS, 0, st>>>(ta);
        else
            gj_update_kernel<32><<<(unsigned)(((n + 31) / 32) * ((mtt + 31) / 32)), GJ_THREADS, 0, st>>>(ta);
        DME_CUDA_TRY(cudaGetLastError());
    }
    if (nrhs > 0) {
        const size_t tot = (size_t)n * nrhs;
        gj_gather_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(B, ldb, pr, n, nrhs, X);
        DME_CUDA_TRY(cudaGetLastError());
        DME_CUDA_TRY(cudaMemcpy2DAsync(B, sizeof(double) * ldb, X, sizeof(double) * nrhs, sizeof(double) * nrhs, n,
                                       cudaMemcpyDeviceToDevice, st));
    }
    return DME_OK;
}

dme_status launch_gj_solve(double* M, int n, int ldm, double* B, int nrhs, int ldb, double* work, int* status,
                           cudaStream_t st) {
    if (n <= 0) return DME_OK;
    const int sms = gj_sms();
    const size_t cap = (size_t)sms * 4;
    double* V = work + 2 * cap + 16;
    if (n <= GJP_MAX_N) {
        int* used = reinterpret_cast<int*>(V + (size_t)GJ_NB * ((size_t)n + nrhs));
        double* X = V + (size_t)GJ_NB * ((size_t)n + nrhs) + n;
        return gj_solve_panels(M, n, ldm, B, nrhs, ldb, V, used, used + n, X, status, st);
    }
    // 64-wide update tiles when the first panel's update has two waves of them, else 32-wide
    const long mt0 = (long)n - std::min(GJ_NB, n) + nrhs;
    const long tiles64 = (long)((n + 63) / 64) * ((mt0 + 63) / 64);
    const bool wide = tiles64 >= 2L * sms;
    const long tiles = wide ? tiles64 : (long)((n + 31) / 32) * ((mt0 + 31) / 32);
    const int per = wide ? gj_blocks_per_sm<64>() : gj_blocks_per_sm<32>();
    if (per < 1) return set_error("Gauss-Jordan solve: no block fits on an SM"), DME_EINVAL;
    const long gmax = (long)sms * per;
    const int grid = (int)std::max(1L, std::min(gmax, std::max((long)(n + GJ_THREADS - 1) / GJ_THREADS, tiles)));
    GJArgs a;
    a.M = M;
    a.ldm = ldm;
    a.B = B;
    a.ldb = ldb;
    a.n = n;
    a.nrhs = nrhs;
    a.pv = work;
    a.pi = reinterpret_cast<int*>(work + cap);
    a.info = work + 2 * cap;
    a.bar = reinterpret_cast<unsigned*>(work + 2 * cap + 2);
    a.status = status;
    a.perm = reinterpret_cast<int*>(work + 2 * cap + 4);
    a.V = V;
    a.ldv = n + nrhs;
    DME_CUDA_TRY(cudaMemsetAsync(a.bar, 0, 2 * sizeof(unsigned), st));
    void* args[] = {&a};
    const void* fn = wide ? reinterpret_cast<const void*>(gj_kernel<64>) : reinterpret_cast<const void*>(gj_kernel<32>);
    return coop_launch(fn, dim3(grid), dim3(GJ_THREADS), args, 0, st, per);
}

}  // namespace dme
