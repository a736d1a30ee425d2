// T3, the exact flow of dP/dt = -P B R^{-1} B^T P (Eq. nonlinear):
//     T3(t) P = (I + t P B R^{-1} B^T)^{-1} P.
// With Bt = B L_R^{-T} (B R^{-1} B^T = Bt Bt^T) and Z = P Bt (n x m), the
// Sherman-Morrison-Woodbury identity gives the m x m form
//     T3(t) P = P - t Z (I_m + t Bt^T Z)^{-1} Z^T,
// which only needs the small SPD matrix M = I_m + t Bt^T P Bt (the dense
// counterpart of the r x r solve of §2.2).  With M = L L^T and Y = Z L^{-T}:
//     T3(t) P = P - t Y Y^T.
// Four kernels: (1) Z = P Bt with per-block partial Gram sums Bt^T Z,
// (2) M from the partials (deterministic reduction order), its Cholesky and
// L^{-1} (FP64), (3) Y = Z L^{-T}, (4) the rank-m update P <- P - t Y Y^T (+ q Q).
// Each kernel takes a batch of independent problems (grouped launch): the
// blocks of every problem are laid end to end and each block finds its
// problem by a binary search over the per-problem block offsets, so a
// problem is computed identically alone or in a batch.
// Everything is FP64.  (1) and (4) stream P once each with coalesced,
// 16-byte vector loads; the row dot-products of (1) are warp reductions.
#include "dme_internal.h"

#include <algorithm>
#include <cstring>
#include <vector>

namespace dme {

constexpr int RZ_ROWS = 8;      // rows of P per block in kernel (1): one per warp
constexpr int RZ_MB = 8;        // columns of Bt per pass
constexpr int RU_TILE = 64;     // update tile

__host__ __device__ __forceinline__ int rz_blocks(int n) { return (n + RZ_ROWS - 1) / RZ_ROWS; }

size_t riccati_work_doubles(int n, int m) {
    // Z (n m) | Y (n m) | Gpart (blocks m m) | Linv (m m)
    return (size_t)2 * n * m + (size_t)rz_blocks(n) * m * m + (size_t)m * m + 8;
}

// One problem of a (possibly grouped) Riccati update; the block-prefix fields
// map a global block index of each kernel to (problem, local block).
struct RicDesc {
    double* P;
    const double* Bt;
    double* Z;
    double* Y;
    double* Gpart;
    double* Linv;
    const double* Qadd;
    double t, q;
    int n, m;
    int* status;
    int sz, sy, su;     // first block of this problem in the z, y and update grids
};

constexpr int kRicLocal = 8;
struct RicBatch {
    RicDesc local[kRicLocal];
    const RicDesc* dev;     // used instead of `local` when nd > kRicLocal
    int nd;
};

__device__ __forceinline__ const RicDesc* ric_descs(const RicBatch& b) { return b.dev ? b.dev : b.local; }

// largest i with start(i) <= blk
template <int FIELD>
__device__ __forceinline__ int ric_find(const RicDesc* d, int nd, int blk) {
    int lo = 0, hi = nd - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int st = FIELD == 0 ? d[mid].sz : (FIELD == 1 ? d[mid].sy : d[mid].su);
        if (st <= blk) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// (1) Z[r][c] = sum_k P[r][k] Bt[k][c] for the block's 8 rows (one per warp),
// in passes of 8 columns; Bt chunks staged in shared memory; then the block's
// partial Gram sums Gpart[b][i][c] = sum_{r in block} Bt[r][i] Z[r][c] in a
// fixed order (deterministic, no atomics).
__global__ void __launch_bounds__(256) riccati_z_kernel(const __grid_constant__ RicBatch batch) {
    constexpr int KC = 512;
    // Bt chunk stored column-major in pairs: sB2[c][k/2] = (Bt[k][c], Bt[k+1][c]), so the lanes of a
    // warp (consecutive k pairs) read consecutive 16-byte words of one column
    __shared__ double2 sB2[RZ_MB][KC / 2];
    __shared__ double sZ[RZ_ROWS][RZ_MB];
    const RicDesc* ds = ric_descs(batch);
    const int ip = ric_find<0>(ds, batch.nd, blockIdx.x);
    const RicDesc& d = ds[ip];
    const int lb = blockIdx.x - d.sz;
    const int n = d.n, m = d.m;
    const double* __restrict__ P = d.P;
    const double* __restrict__ Bt = d.Bt;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = lb * RZ_ROWS + warp;
    const bool vec = (n % 2) == 0;
    for (int c0 = 0; c0 < m; c0 += RZ_MB) {
        const int mb = min(RZ_MB, m - c0);
        double acc[RZ_MB];
#pragma unroll
        for (int c = 0; c < RZ_MB; ++c) acc[c] = 0.0;
        for (int k0 = 0; k0 < n; k0 += KC) {
            __syncthreads();
            for (int e = threadIdx.x; e < (KC / 2) * RZ_MB; e += blockDim.x) {
                const int c = e / (KC / 2), kp = e % (KC / 2), k = 2 * kp;
                double2 v;
                v.x = (k0 + k < n && c < mb) ? Bt[(size_t)(k0 + k) * m + c0 + c] : 0.0;
                v.y = (k0 + k + 1 < n && c < mb) ? Bt[(size_t)(k0 + k + 1) * m + c0 + c] : 0.0;
                sB2[c][kp] = v;
            }
            __syncthreads();
            if (row >= n) continue;
            const int kend = min(KC, n - k0);
            const double* prow = P + (size_t)row * n + k0;
            // 2 consecutive doubles per lane per iteration: a warp covers 64 columns
            for (int k = 2 * lane; k < kend; k += 64) {
                double p0, p1 = 0.0;
                if (vec && k + 1 < kend) {
                    double2 v = *reinterpret_cast<const double2*>(prow + k);
                    p0 = v.x;
                    p1 = v.y;
                } else {
                    p0 = prow[k];
                    if (k + 1 < kend) p1 = prow[k + 1];
                }
                // k is even; past the row end p1 = 0 and the staged Bt is zero-filled
#pragma unroll
                for (int c = 0; c < RZ_MB; ++c) {
                    const double2 b = sB2[c][k >> 1];
                    acc[c] = fma(p1, b.y, fma(p0, b.x, acc[c]));
                }
            }
        }
#pragma unroll
        for (int c = 0; c < RZ_MB; ++c) {
            double v = acc[c];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            acc[c] = v;
        }
        __syncthreads();
        if (lane == 0) {
#pragma unroll
            for (int c = 0; c < RZ_MB; ++c) sZ[warp][c] = (row < n) ? acc[c] : 0.0;
        }
        if (row < n && lane < mb) {
            double v = 0.0;
#pragma unroll
            for (int c = 0; c < RZ_MB; ++c)
                if (c == lane) v = acc[c];
            d.Z[(size_t)row * m + c0 + lane] = v;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < m * mb; e += blockDim.x) {
            const int i = e / mb, jj = e % mb;
            double sacc = 0.0;
            for (int r = 0; r < RZ_ROWS; ++r) {
                const int rr = lb * RZ_ROWS + r;
                if (rr < n) sacc = fma(Bt[(size_t)rr * m + i], sZ[r][jj], sacc);
            }
            d.Gpart[(size_t)lb * m * m + (size_t)i * m + c0 + jj] = sacc;
        }
    }
}

// (2) M = I + t sym(sum_b Gpart[b]); M = L L^T; Linv = L^{-1}.  One block per
// problem.  The sum over blocks is a fixed two-level order (strided partial
// sums, then a tree), so the result does not depend on scheduling.
__global__ void __launch_bounds__(1024) riccati_small_kernel(const __grid_constant__ RicBatch batch) {
    __shared__ double red[1024];
    __shared__ double L[32][33];
    const RicDesc& d = ric_descs(batch)[blockIdx.x];
    const int m = d.m;
    const int nblocks = rz_blocks(d.n);
    const double t = d.t;
    const int E = m * m;
    const int G = max(1, 1024 / E);
    const int tid = threadIdx.x;
    const int e = tid % E, g = tid / E;
    double sacc = 0.0;
    if (g < G)
        for (int b = g; b < nblocks; b += G) sacc += d.Gpart[(size_t)b * E + e];
    red[tid] = (g < G) ? sacc : 0.0;
    __syncthreads();
    // tree over groups: group g adds group g + half (fixed order)
    for (int half = 1; half < G; half <<= 1) {
        if (g < G && (g % (2 * half)) == 0 && g + half < G) red[tid] += red[tid + half * E];
        __syncthreads();
    }
    if (tid < E) L[tid / m][tid % m] = red[tid];
    __syncthreads();
    if (tid >= 32) return;
    const int lane = tid;
    // symmetrise and add the identity: M = I + t (G + G^T)/2
    double Mv[32];
    for (int e2 = lane; e2 < E; e2 += 32) {
        const int i = e2 / m, j = e2 % m;
        Mv[e2 / 32] = (i == j ? 1.0 : 0.0) + t * 0.5 * (L[i][j] + L[j][i]);
    }
    __syncwarp();
    for (int e2 = lane; e2 < E; e2 += 32) L[e2 / m][e2 % m] = Mv[e2 / 32];
    __syncwarp();
    // Cholesky in place (lower)
    for (int j = 0; j < m; ++j) {
        double dj = L[j][j];
        for (int k = 0; k < j; ++k) dj -= L[j][k] * L[j][k];
        if (!(dj > 0.0)) {
            if (lane == 0) atomicOr(d.status, DEV_NOTSPD);
            return;
        }
        dj = sqrt(dj);
        __syncwarp();
        for (int i = j + 1 + lane; i < m; i += 32) {
            double s2 = L[i][j];
            for (int k = 0; k < j; ++k) s2 -= L[i][k] * L[j][k];
            L[i][j] = s2 / dj;
        }
        __syncwarp();
        if (lane == 0) L[j][j] = dj;
        __syncwarp();
    }
    // Linv column by column (forward substitution on e_c); lane c owns column c
    for (int c = lane; c < m; c += 32) {
        double x[32];
        for (int r = 0; r < m; ++r) {
            double s2 = (r == c) ? 1.0 : 0.0;
            for (int k = 0; k < r; ++k) s2 -= L[r][k] * x[k];
            x[r] = (r < c) ? 0.0 : s2 / L[r][r];
        }
        for (int r = 0; r < m; ++r) d.Linv[r * m + c] = x[r];
    }
}

// (1b) The partial Gram sums of (1) from a Z computed elsewhere (same blocks of
// RZ_ROWS rows, same fixed order).
__global__ void riccati_gpart_kernel(const __grid_constant__ RicBatch batch) {
    const RicDesc* ds = ric_descs(batch);
    const RicDesc& d = ds[ric_find<0>(ds, batch.nd, blockIdx.x)];
    const int lb = blockIdx.x - d.sz, n = d.n, m = d.m;
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int i = e / m, c = e % m;
        double sacc = 0.0;
        for (int r = 0; r < RZ_ROWS; ++r) {
            const int rr = lb * RZ_ROWS + r;
            if (rr < n) sacc = fma(d.Bt[(size_t)rr * m + i], d.Z[(size_t)rr * m + c], sacc);
        }
        d.Gpart[(size_t)lb * m * m + e] = sacc;
    }
}

// (3) Y[i][r] = sum_{c <= r} Linv[r][c] Z[i][c]   (Y = Z L^{-T}); Y = 0 when the
// m x m matrix was not SPD (an update with Y then leaves P as it is).
__global__ void riccati_y_kernel(const __grid_constant__ RicBatch batch) {
    const RicDesc* ds = ric_descs(batch);
    const RicDesc& d = ds[ric_find<1>(ds, batch.nd, blockIdx.x)];
    const int i = (blockIdx.x - d.sy) * blockDim.x + threadIdx.x;
    const int m = d.m;
    if (i >= d.n) return;
    if (*d.status & DEV_NOTSPD) {
        for (int r = 0; r < m; ++r) d.Y[(size_t)i * m + r] = 0.0;
        return;
    }
    for (int r = 0; r < m; ++r) {
        double s = 0.0;
        for (int c = 0; c <= r; ++c) s = fma(d.Linv[r * m + c], d.Z[(size_t)i * m + c], s);
        d.Y[(size_t)i * m + r] = s;
    }
}

// (4) P[i][j] <- P[i][j] - t sum_r Y[i][r] Y[j][r] (+ q Q[i][j]).  The result is
// symmetric (the sum is taken in the same order for (i, j) and (j, i)), so only
// the 64 x 64 tiles on or above the diagonal are computed: each reads its
// upper block of P, writes it, and for an off-diagonal tile also writes the
// transposed block below the diagonal from a shared-memory copy (coalesced).
// Half of the FP64 work and of the traffic on P of a full update.
constexpr int RU_LD = RU_TILE + 1;
constexpr size_t RU_SMEM = sizeof(double) * (2 * RU_TILE * 33 + RU_TILE * RU_LD);

__global__ void __launch_bounds__(256) riccati_update_kernel(const __grid_constant__ RicBatch batch) {
    const RicDesc* ds = ric_descs(batch);
    const RicDesc& d = ds[ric_find<2>(ds, batch.nd, blockIdx.x)];
    if (*d.status & DEV_NOTSPD) return;
    extern __shared__ double ru_smem[];
    double(*Yi)[33] = reinterpret_cast<double(*)[33]>(ru_smem);
    double(*Yj)[33] = reinterpret_cast<double(*)[33]>(ru_smem + RU_TILE * 33);
    double* Vt = ru_smem + 2 * RU_TILE * 33;           // [RU_TILE][RU_LD]
    const int n = d.n, m = d.m;
    const int T = (n + RU_TILE - 1) / RU_TILE;
    // upper-triangle tile (ti <= tj), row by row
    int rem = blockIdx.x - d.su, ti = 0;
    while (rem >= T - ti) {
        rem -= T - ti;
        ++ti;
    }
    const int tj = ti + rem;
    const int i0 = ti * RU_TILE, j0 = tj * RU_TILE;
    for (int e = threadIdx.x; e < RU_TILE * m; e += blockDim.x) {
        int r = e / m, c = e % m;
        Yi[r][c] = (i0 + r < n) ? d.Y[(size_t)(i0 + r) * m + c] : 0.0;
        Yj[r][c] = (j0 + r < n) ? d.Y[(size_t)(j0 + r) * m + c] : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    for (int di = ty; di < RU_TILE; di += 8) {
        const int i = i0 + di;
        if (i >= n) break;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int dj = tx + 32 * h, j = j0 + dj;
            if (j >= n) continue;
            double s = 0.0;
            for (int c = 0; c < m; ++c) s = fma(Yi[di][c], Yj[dj][c], s);
            const size_t off = (size_t)i * n + j;
            double v = d.P[off] - d.t * s;
            if (d.Qadd) v += d.q * d.Qadd[off];
            d.P[off] = v;
            Vt[di * RU_LD + dj] = v;
        }
    }
    if (ti == tj) return;
    __syncthreads();
    // mirror: P[j][i] = V[i][j] for the block below the diagonal
    for (int dj = ty; dj < RU_TILE; dj += 8) {
        const int j = j0 + dj;
        if (j >= n) break;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int di = tx + 32 * h, i = i0 + di;
            if (i >= n) continue;
            d.P[(size_t)j * n + i] = Vt[di * RU_LD + dj];
        }
    }
}

dme_status launch_riccati_from_z(const double* Bt, int n, int m, double t, double* work, int* status,
                                 cudaStream_t st) {
    RicBatch b;
    std::memset(&b, 0, sizeof(b));
    b.nd = 1;
    RicDesc& d = b.local[0];
    d.P = nullptr;
    d.Bt = Bt;
    d.Z = work;
    d.Y = d.Z + (size_t)n * m;
    d.Gpart = d.Y + (size_t)n * m;
    d.Linv = d.Gpart + (size_t)rz_blocks(n) * m * m;
    d.t = t;
    d.n = n;
    d.m = m;
    d.status = status;
    riccati_gpart_kernel<<<rz_blocks(n), 64, 0, st>>>(b);
    riccati_small_kernel<<<1, 1024, 0, st>>>(b);
    riccati_y_kernel<<<(n + 127) / 128, 128, 0, st>>>(b);
    DME_CUDA_TRY(cudaGetLastError());
    return DME_OK;
}

RicItem make_ric_item(double* P, const double* Bt, int n, int m, double t, const double* Qadd, double q,
                      double* work, int* status) {
    RicItem it;
    it.P = P;
    it.Bt = Bt;
    it.n = n;
    it.m = m;
    it.t = t;
    it.Qadd = Qadd;
    it.q = q;
    it.work = work;
    it.status = status;
    return it;
}

dme_status launch_riccati_grouped(const std::vector<RicItem>& items, void* dev_desc, cudaStream_t st,
                                  DescArena* arena) {
    if (items.empty()) return DME_OK;
    std::vector<RicDesc> ds(items.size());
    int sz = 0, sy = 0, su = 0;
    for (size_t k = 0; k < items.size(); ++k) {
        const RicItem& it = items[k];
        RicDesc& d = ds[k];
        const int n = it.n, m = it.m;
        d.P = it.P;
        d.Bt = it.Bt;
        d.Z = it.work;
        d.Y = d.Z + (size_t)n * m;
        d.Gpart = d.Y + (size_t)n * m;
        d.Linv = d.Gpart + (size_t)rz_blocks(n) * m * m;
        d.Qadd = it.Qadd;
        d.t = it.t;
        d.q = it.q;
        d.n = n;
        d.m = m;
        d.status = it.status;
        d.sz = sz;
        d.sy = sy;
        d.su = su;
        sz += rz_blocks(n);
        sy += (n + 127) / 128;
        const int tn = (n + RU_TILE - 1) / RU_TILE;
        su += tn * (tn + 1) / 2;
    }
    RicBatch b;
    std::memset(&b, 0, sizeof(b));
    b.nd = (int)ds.size();
    if (ds.size() <= (size_t)kRicLocal) {
        for (size_t k = 0; k < ds.size(); ++k) b.local[k] = ds[k];
        b.dev = nullptr;
    } else {
        if (arena) {
            dev_desc = arena->put(ds.data(), ds.size() * sizeof(RicDesc));
            if (!dev_desc) return set_error("grouped Riccati: descriptor arena full"), DME_ENOMEM;
        } else {
            if (!dev_desc) {
                set_error("grouped Riccati: more than 8 problems need a device descriptor buffer");
                return DME_EINVAL;
            }
            DME_CUDA_TRY(cudaMemcpyAsync(dev_desc, ds.data(), ds.size() * sizeof(RicDesc), cudaMemcpyHostToDevice, st));
        }
        b.dev = reinterpret_cast<const RicDesc*>(dev_desc);
    }
    riccati_z_kernel<<<sz, 256, 0, st>>>(b);
    riccati_small_kernel<<<b.nd, 1024, 0, st>>>(b);
    riccati_y_kernel<<<sy, 128, 0, st>>>(b);
    static const cudaError_t attr =
        cudaFuncSetAttribute(riccati_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)RU_SMEM);
    DME_CUDA_TRY(attr);
    riccati_update_kernel<<<su, 256, RU_SMEM, st>>>(b);
    DME_CUDA_TRY(cudaGetLastError());
    return DME_OK;
}

size_t riccati_desc_bytes() { return sizeof(RicDesc); }

// K = R^{-1} B^T P for symmetric P, with R = L L^T and Bt = B L^{-T}:
// B^T P = L Bt^T P = L Z^T (Z = P Bt), so K = L^{-T} Z^T, i.e. L^T K = Z^T,
// solved by back substitution for each column j of K (one thread per column).
__global__ void lqr_gain_kernel(const double* __restrict__ Z, const double* __restrict__ L, double* __restrict__ K,
                                int n, int m) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double x[32];
    for (int r = m - 1; r >= 0; --r) {
        double s = Z[(size_t)j * m + r];
        for (int c = r + 1; c < m; ++c) s -= L[c * m + r] * x[c];
        x[r] = s / L[r * m + r];
        K[(size_t)r * n + j] = x[r];
    }
}

// The gain of step *ctr into Kbase + (*ctr) m n, then ++*ctr (a single thread,
// after the gain kernel in stream order): one record per replayed step.
__global__ void lqr_gain_hist_kernel(const double* __restrict__ Z, const double* __restrict__ L,
                                     double* __restrict__ Kbase, int n, int m, const int* __restrict__ ctr,
                                     int cap) {
    const int k = *ctr;
    if (k >= cap) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double* K = Kbase + (size_t)k * m * n;
    double x[32];
    for (int r = m - 1; r >= 0; --r) {
        double s = Z[(size_t)j * m + r];
        for (int c = r + 1; c < m; ++c) s -= L[c * m + r] * x[c];
        x[r] = s / L[r * m + r];
        K[(size_t)r * n + j] = x[r];
    }
}

__global__ void counter_inc_kernel(int* ctr) { *ctr += 1; }

dme_status launch_lqr_gain_hist(const double* P, const double* Bt, const double* LR, int n, int m, double* work,
                                double* Kbase, int* ctr, int cap, cudaStream_t st) {
    RicBatch b;
    std::memset(&b, 0, sizeof(b));
    RicDesc& d = b.local[0];
    d.P = const_cast<double*>(P);
    d.Bt = Bt;
    d.Z = work;
    d.Y = d.Z + (size_t)n * m;
    d.Gpart = d.Y + (size_t)n * m;
    d.n = n;
    d.m = m;
    b.nd = 1;
    riccati_z_kernel<<<rz_blocks(n), 256, 0, st>>>(b);       // Z = P Bt (P is only read)
    lqr_gain_hist_kernel<<<(n + 127) / 128, 128, 0, st>>>(d.Z, LR, Kbase, n, m, ctr, cap);
    counter_inc_kernel<<<1, 1, 0, st>>>(ctr);
    DME_CUDA_TRY(cudaGetLastError());
    return DME_OK;
}

dme_status launch_lqr_gain(const double* P, const double* Bt, const double* LR, int n, int m, double* work,
                           double* K, cudaStream_t st) {
    RicBatch b;
    std::memset(&b, 0, sizeof(b));
    RicDesc& d = b.local[0];
    d.P = const_cast<double*>(P);
    d.Bt = Bt;
    d.Z = work;
    d.Y = d.Z + (size_t)n * m;
    d.Gpart = d.Y + (size_t)n * m;
    d.n = n;
    d.m = m;
    b.nd = 1;
    riccati_z_kernel<<<rz_blocks(n), 256, 0, st>>>(b);       // Z = P Bt (P is only read)
    lqr_gain_kernel<<<(n + 127) / 128, 128, 0, st>>>(d.Z, LR, K, n, m);
    DME_CUDA_TRY(cudaGetLastError());
    return DME_OK;
}

void launch_riccati(double* P, const double* Bt, int n, int m, double t, const double* Qadd, double q,
                    double* work, int* status, cudaStream_t st) {
    std::vector<RicItem> v{make_ric_item(P, Bt, n, m, t, Qadd, q, work, status)};
    launch_riccati_grouped(v, nullptr, st);
}

}  // namespace dme
