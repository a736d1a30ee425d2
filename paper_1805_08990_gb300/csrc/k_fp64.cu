// FP64 kernels of libdme: grouped GEMM with a symmetric-triangle mode and a
// fused additive epilogue, the elementwise helpers of the plan step, dense LU
// with partial pivoting and its triangular sweeps, and the small m x m
// Cholesky used for R.
//
// GB300 executes FP64 on a narrow pipe (about 1.25 TFLOP/s for the whole
// chip), so these kernels are ALU-bound: the GEMM keeps a 4 x 4 register
// tile per thread fed from shared memory and spends its effort on coalesced
// tile loads, not on latency hiding.
#include "dme_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace dme {

// ============================================================== grouped GEMM
constexpr int kMaxBatch = 8;
struct GemmBatch {
    GemmProb p[kMaxBatch];
    int nprobs;
};

__device__ __forceinline__ void tile_coords(const GemmProb& pb, int lt, int& ti, int& tj) {
    if (pb.tri) {
        int T = pb.tiles_n, r = 0, rem = lt;
        while (rem >= T - r) {
            rem -= T - r;
            ++r;
        }
        ti = r;
        tj = r + rem;
    } else {
        ti = lt / pb.tiles_n;
        tj = lt % pb.tiles_n;
    }
}

// One BM x BM output tile (BM = 32 or 64) with 256 threads, each holding a
// TM x TM register tile (TM = BM / 16).  Every output is accumulated over k in
// increasing order with fma, whatever BM is; gemm64_accum covers [kbeg, kend).
template <int BM>
__device__ __forceinline__ void gemm64_accum(const GemmProb& pb, int row0, int col0, int kbeg, int kend,
                                             double (&As)[G64_BK][BM + 1], double (&Bs)[G64_BK][BM + 1],
                                             double (&acc)[BM / 16][BM / 16]) {
    constexpr int TM = BM / 16;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TM; ++j) acc[i][j] = 0.0;

    for (int k0 = kbeg; k0 < kend; k0 += G64_BK) {
#pragma unroll
        for (int q = 0; q < TM; ++q) {
            const int e = tid + 256 * q;     // BM x 16 elements of each operand tile
            int r, k;
            double v = 0.0;
            if (!pb.transA) {
                r = e >> 4;
                k = e & 15;
                int gr = row0 + r, gk = k0 + k;
                if (gr < pb.M && gk < kend) v = pb.A[(size_t)gr * pb.lda + gk];
            } else {
                r = e % BM;
                k = e / BM;
                int gr = row0 + r, gk = k0 + k;
                if (gr < pb.M && gk < kend) v = pb.A[(size_t)gk * pb.lda + gr];
            }
            As[k][r] = v;
            int c;
            double w = 0.0;
            if (!pb.transB) {
                c = e % BM;
                k = e / BM;
                int gc = col0 + c, gk = k0 + k;
                if (gc < pb.N && gk < kend) w = pb.B[(size_t)gk * pb.ldb + gc];
            } else {
                c = e >> 4;
                k = e & 15;
                int gc = col0 + c, gk = k0 + k;
                if (gc < pb.N && gk < kend) w = pb.B[(size_t)gc * pb.ldb + gk];
            }
            Bs[k][c] = w;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < G64_BK; ++k) {
            double a[TM], b[TM];
#pragma unroll
            for (int i = 0; i < TM; ++i) a[i] = As[k][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < TM; ++j) b[j] = Bs[k][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TM; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
}

// C = alpha acc + b1 D1 + b2 D2 + b3 D3 (a triangle problem writes (r, c), r <= c,
// and its mirror).
__device__ __forceinline__ void gemm64_out(const GemmProb& pb, int r, int c, double sum) {
    const size_t off = (size_t)r * pb.ldd + c;
    double v = pb.alpha * sum;
    if (pb.D1) v += pb.b1 * pb.D1[off];
    if (pb.D2) v += pb.b2 * pb.D2[off];
    if (pb.D3) v += pb.b3 * pb.D3[off];
    pb.C[(size_t)r * pb.ldc + c] = v;
    if (pb.tri && r != c) pb.C[(size_t)c * pb.ldc + r] = v;
}

template <int BM>
__device__ __forceinline__ void gemm64_tile(const GemmProb& pb, int lt, double (&As)[G64_BK][BM + 1],
                                            double (&Bs)[G64_BK][BM + 1]) {
    constexpr int TM = BM / 16;
    int ti, tj;
    tile_coords(pb, lt, ti, tj);
    const int row0 = ti * BM, col0 = tj * BM;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[TM][TM];
    gemm64_accum<BM>(pb, row0, col0, 0, pb.K, As, Bs, acc);
#pragma unroll
    for (int i = 0; i < TM; ++i) {
        const int r = row0 + ty + 16 * i;
        if (r >= pb.M) continue;
#pragma unroll
        for (int j = 0; j < TM; ++j) {
            const int c = col0 + tx + 16 * j;
            if (c >= pb.N) continue;
            if (pb.tri && r > c) continue;
            gemm64_out(pb, r, c, acc[i][j]);
        }
    }
}

__device__ __forceinline__ int find_prob(const GemmProb* probs, int nprobs, int t) {
    int lo = 0, hi = nprobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (probs[mid].tile_start <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Persistent: CTA b takes tiles b, b + gridDim.x, ... of the concatenated tile list.
template <int BM>
__global__ void __launch_bounds__(256) gemm64_batch_kernel(const __grid_constant__ GemmBatch batch, int total) {
    __shared__ double As[G64_BK][BM + 1];
    __shared__ double Bs[G64_BK][BM + 1];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int ip = find_prob(batch.p, batch.nprobs, t);
        gemm64_tile<BM>(batch.p[ip], t - batch.p[ip].tile_start, As, Bs);
    }
}

template <int BM>
__global__ void __launch_bounds__(256) gemm64_desc_kernel(const GemmProb* __restrict__ probs, int nprobs, int total) {
    __shared__ double As[G64_BK][BM + 1];
    __shared__ double Bs[G64_BK][BM + 1];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int ip = find_prob(probs, nprobs, t);
        GemmProb pb = probs[ip];
        gemm64_tile<BM>(pb, t - pb.tile_start, As, Bs);
    }
}

// Split K for products of fewer tiles than SMs (the plan's small products, whose
// tiles would otherwise each run the whole K on one SM's narrow FP64 pipe): CTA
// (tile, part) writes its partial sums over K range `part` to ws[part][M][N];
// the reduction adds the parts in order and applies the epilogue.
__global__ void __launch_bounds__(256) gemm64_splitk_kernel(const __grid_constant__ GemmProb pb, int ntiles,
                                                            int kchunk, double* __restrict__ ws) {
    __shared__ double As[G64_BK][33];
    __shared__ double Bs[G64_BK][33];
    const int lt = blockIdx.x % ntiles, part = blockIdx.x / ntiles;
    int ti, tj;
    tile_coords(pb, lt, ti, tj);
    const int row0 = ti * 32, col0 = tj * 32;
    const int kb = part * kchunk, ke = min(pb.K, kb + kchunk);
    double acc[2][2];
    gemm64_accum<32>(pb, row0, col0, kb, ke, As, Bs, acc);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double* w = ws + (size_t)part * pb.M * pb.N;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int r = row0 + ty + 16 * i;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int c = col0 + tx + 16 * j;
            if (r < pb.M && c < pb.N) w[(size_t)r * pb.N + c] = acc[i][j];
        }
    }
}

__global__ void gemm64_splitk_reduce_kernel(const __grid_constant__ GemmProb pb, int parts,
                                            const double* __restrict__ ws) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t mn = (size_t)pb.M * pb.N;
    if (e >= mn) return;
    const int r = (int)(e / pb.N), c = (int)(e % pb.N);
    if (pb.tri && r > c) return;
    double sum = 0.0;
    for (int q = 0; q < parts; ++q) sum += ws[(size_t)q * mn + e];
    gemm64_out(pb, r, c, sum);
}

static int prepare_tiles(std::vector<GemmProb>& probs, int bm) {
    int total = 0;
    for (auto& p : probs) {
        int tm = (p.M + bm - 1) / bm, tn = (p.N + bm - 1) / bm;
        p.tiles_n = tn;
        p.ntiles = (p.M <= 0 || p.N <= 0) ? 0 : (p.tri ? tn * (tn + 1) / 2 : tm * tn);
        p.tile_start = total;
        total += p.ntiles;
    }
    return total;
}

void* DescArena::put(const void* src, size_t bytes) {
    size_t off = (host.size() + 255) & ~size_t(255);
    if (off + bytes > cap || !dev) return nullptr;
    host.resize(off + bytes);
    std::memcpy(host.data() + off, src, bytes);
    return dev + off;
}

// Resident CTAs of a kernel on the whole device (persistent grid size).
template <typename K>
static int resident_ctas(K kernel, int threads) {
    int dev = 0, nsm = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1 << 20;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1 << 20;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return nsm * per_sm;
}

template <int BM>
static int batch_cap() {
    static int cap = resident_ctas(gemm64_batch_kernel<BM>, 256);
    return cap;
}

template <int BM>
static int desc_cap() {
    static int cap = resident_ctas(gemm64_desc_kernel<BM>, 256);
    return cap;
}

void gemm64_prepare() {
    batch_cap<32>();
    batch_cap<64>();
    desc_cap<32>();
    desc_cap<64>();
}

template <int BM>
static dme_status gemm64_launch(std::vector<GemmProb>& live, GemmProb* dev_desc, cudaStream_t st, DescArena* arena) {
    const int total = prepare_tiles(live, BM);
    if (total == 0) return DME_OK;
    if ((int)live.size() <= kMaxBatch) {
        const int cap = batch_cap<BM>();
        GemmBatch b;
        std::memset(&b, 0, sizeof(b));
        b.nprobs = (int)live.size();
        for (int i = 0; i < b.nprobs; ++i) b.p[i] = live[i];
        gemm64_batch_kernel<BM><<<std::min(total, cap), 256, 0, st>>>(b, total);
    } else {
        const int cap = desc_cap<BM>();
        const size_t bytes = live.size() * sizeof(GemmProb);
        GemmProb* d = dev_desc;
        if (arena) {
            d = static_cast<GemmProb*>(arena->put(live.data(), bytes));
            if (!d) return set_error("gemm64: descriptor arena full"), DME_ENOMEM;
        } else {
            if (!d) return set_error("gemm64: more than 8 problems need a device descriptor buffer"), DME_EINVAL;
            DME_CUDA_TRY(cudaMemcpyAsync(d, live.data(), bytes, cudaMemcpyHostToDevice, st));
        }
        gemm64_desc_kernel<BM><<<std::min(total, cap), 256, 0, st>>>(d, (int)live.size(), total);
    }
    DME_CUDA_TRY(cudaGetLastError());
    return DME_OK;
}

dme_status gemm64_grouped(std::vector<GemmProb>& probs, GemmProb* dev_desc, cudaStream_t st, DescArena* arena,
                          int tile) {
    for (auto& p : probs) {
        if (p.tri && p.M != p.N) {
            set_error("gemm64: triangle mode needs M == N");
            return DME_EINVAL;
        }
    }
    if (tile != 32 && tile != 64) return set_error("gemm64: tile must be 32 or 64"), DME_EINVAL;
    // drop empty problems, keep order
    std::vector<GemmProb> live;
    for (auto& p : probs)
        if (p.M > 0 && p.N > 0) live.push_back(p);
    if (live.empty()) return DME_OK;
    return tile == 32 ? gemm64_launch<32>(live, dev_desc, st, arena) : gemm64_launch<64>(live, dev_desc, st, arena);
}

size_t gemm64_splitk_ws_doubles(int M, int N) { return (size_t)8 * M * N; }

dme_status gemm64_splitk(const GemmProb& g, double* ws, size_t ws_len, cudaStream_t st) {
    std::vector<GemmProb> v{g};
    if (g.M <= 0 || g.N <= 0) return DME_OK;
    if (g.tri && g.M != g.N) return set_error("gemm64: triangle mode needs M == N"), DME_EINVAL;
    const int tm = (g.M + 31) / 32, tn = (g.N + 31) / 32;
    const int tiles = g.tri ? tn * (tn + 1) / 2 : tm * tn;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // parts of at least one 16-deep K block, up to 8, for about two CTAs per SM
    int parts = std::min(8, std::min(g.K / G64_BK, std::max(1, 2 * nsm / std::max(tiles, 1))));
    if (tiles >= nsm / 2 || parts < 2 || !ws || ws_len < (size_t)parts * g.M * g.N) {
        long tiles64 = (long)((g.M + 63) / 64) * ((g.N + 63) / 64);
        if (g.tri) tiles64 = (tiles64 + (g.M + 63) / 64) / 2;
        return gemm64_grouped(v, nullptr, st, nullptr, tiles64 < nsm ? 32 : 64);
    }
    const int kchunk = ((g.K + parts - 1) / parts + G64_BK - 1) / G64_BK * G64_BK;
    parts = (g.K + kchunk - 1) / kchunk;
    GemmProb pb = g;
    pb.tiles_n = tn;
    gemm64_splitk_kernel<<<tiles * parts, 256, 0, st>>>(pb, tiles, kchunk, ws);
    const size_t mn = (size_t)g.M * g.N;
    gemm64_splitk_reduce_kernel<<<(unsigned)((mn + 255) / 256), 256, 0, st>>>(pb, parts, ws);
    DME_CUDA_TRY(cudaGetLastError());
    return DME_OK;
}

// ============================================================== elementwise
__global__ void axpy_kernel(double* P, const double* Q, double a, int n, int ld) {
    for (int i = blockIdx.x; i < n; i += gridDim.x)
        for (int j = threadIdx.x; j < n; j += blockDim.x) P[(size_t)i * ld + j] += a * Q[(size_t)i * ld + j];
}


void launch_axpy_sym(double* P, const double* Q, double a, int n, int ld, cudaStream_t st) {
    if (n <= 0) return;
    axpy_kernel<<<std::min(n, 152 * 16), 256, 0, st>>>(P, Q, a, n, ld);
}

__global__ void transpose_kernel(const double* X, double* Y, int rows, int cols, int ldx, int ldy) {
    __shared__ double tile[32][33];
    int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        int r = by + k, c = bx + threadIdx.x;
        if (r < rows && c < cols) tile[k][threadIdx.x] = X[(size_t)r * ldx + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        int r = bx + k, c = by + threadIdx.x;   // Y is cols x rows
        if (r < cols && c < rows) Y[(size_t)r * ldy + c] = tile[threadIdx.x][k];
    }
}

void launch_transpose(const double* X, double* Y, int rows, int cols, int ldx, int ldy, cudaStream_t st) {
    dim3 g((cols + 31) / 32, (rows + 31) / 32), b(32, 8);
    transpose_kernel<<<g, b, 0, st>>>(X, Y, rows, cols, ldx, ldy);
}


// A block per row (grid-stride over rows), threads over the columns.
__global__ void lincomb_kernel(double* Y, int n, int ld, const double* X1, double c1, const double* X2,
                               double c2, const double* X3, double c3, double cI) {
    for (int i = blockIdx.x; i < n; i += gridDim.x)
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const size_t off = (size_t)i * ld + j;
            double v = 0.0;
            if (X1) v += c1 * X1[off];
            if (X2) v += c2 * X2[off];
            if (X3) v += c3 * X3[off];
            if (i == j) v += cI;
            Y[off] = v;
        }
}

void launch_lincomb(double* Y, int n, int ld, const double* X1, double c1, const double* X2, double c2,
                    const double* X3, double c3, double cI, cudaStream_t st) {
    if (n <= 0) return;
    lincomb_kernel<<<std::min(n, 152 * 16), 256, 0, st>>>(Y, n, ld, X1, c1, X2, c2, X3, c3, cI);
}

__global__ void symmetrize_kernel(double* X, int n, int ld) {
    // a block per row i, threads over j > i: both entries of a pair get the same average
    for (int i = blockIdx.x; i < n; i += gridDim.x)
        for (int j = i + 1 + threadIdx.x; j < n; j += blockDim.x) {
            const double v = 0.5 * (X[(size_t)i * ld + j] + X[(size_t)j * ld + i]);
            X[(size_t)i * ld + j] = v;
            X[(size_t)j * ld + i] = v;
        }
}

void launch_symmetrize(double* X, int n, int ld, cudaStream_t st) {
    if (n <= 0) return;
    symmetrize_kernel<<<std::min(n, 152 * 16), 256, 0, st>>>(X, n, ld);
}

// Column abs-sums of the Van Loan matrix [[-A^T, Q], [0, A]] (2n columns).
__global__ void block_norm1_kernel(const double* A, const double* Q, int n, double* colsum) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s1 = 0.0, s2 = 0.0;
    for (int i = 0; i < n; ++i) {
        s1 += fabs(A[(size_t)j * n + i]);                                  // column j of -A^T = row j of A
        s2 += fabs(Q[(size_t)i * n + j]) + fabs(A[(size_t)i * n + j]);    // column n+j
    }
    colsum[j] = s1;
    colsum[n + j] = s2;
}

void launch_block_norm1(const double* A, const double* Q, int n, double* colsum_out, cudaStream_t st) {
    block_norm1_kernel<<<(n + 127) / 128, 128, 0, st>>>(A, Q, n, colsum_out);
}

__global__ void max_reduce_kernel(const double* x, int len, double* out) {
    __shared__ double red[1024];
    double m = 0.0;
    for (int i = threadIdx.x; i < len; i += blockDim.x) m = fmax(m, x[i]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

void launch_max_reduce(const double* x, int len, double* out, cudaStream_t st) {
    max_reduce_kernel<<<1, 1024, 0, st>>>(x, len, out);
}

// ============================================================== small Cholesky
// R = L L^T in place (lower triangle; the strict upper part is zeroed).  One warp.
__global__ void small_cholesky_kernel(double* R, int m, int* status) {
    const int lane = threadIdx.x;
    for (int j = 0; j < m; ++j) {
        double d = R[j * m + j];
        for (int k = 0; k < j; ++k) d -= R[j * m + k] * R[j * m + k];
        if (!(d > 0.0)) {
            if (lane == 0) atomicOr(status, DEV_NOTSPD);
            return;
        }
        d = sqrt(d);
        __syncwarp();
        for (int i = j + 1 + lane; i < m; i += 32) {
            double s = R[i * m + j];
            for (int k = 0; k < j; ++k) s -= R[i * m + k] * R[j * m + k];
            R[i * m + j] = s / d;
        }
        __syncwarp();
        if (lane == 0) R[j * m + j] = d;
        __syncwarp();
    }
    for (int e = lane; e < m * m; e += 32) {
        int i = e / m, j = e % m;
        if (j > i) R[e] = 0.0;
    }
}

void launch_small_cholesky(double* R, int m, int* status, cudaStream_t st) {
    small_cholesky_kernel<<<1, 32, 0, st>>>(R, m, status);
}

// Bt[i][:] = (L^{-1} B[i][:]^T)^T by forward substitution.
__global__ void apply_linv_rows_kernel(const double* B, const double* L, double* Bt, int n, int m) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double y[32];
    for (int r = 0; r < m; ++r) {
        double s = B[(size_t)i * m + r];
        for (int c = 0; c < r; ++c) s -= L[r * m + c] * y[c];
        y[r] = s / L[r * m + r];
        Bt[(size_t)i * m + r] = y[r];
    }
}

void launch_apply_linv_rows(const double* B, const double* L, double* Bt, int n, int m, cudaStream_t st) {
    apply_linv_rows_kernel<<<(n + 127) / 128, 128, 0, st>>>(B, L, Bt, n, m);
}

}  // namespace dme
