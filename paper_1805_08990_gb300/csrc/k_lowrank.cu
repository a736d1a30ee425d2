// Kernels of the low-rank (LDL^T) path: a one-CTA parallel Jacobi
// eigensolver for the small symmetric systems of the column compression and
// of the factored Riccati flow, the eigenvalue selection that builds the
// compressed basis, and column scaling / copying helpers.
//
// The compression only needs the eigen-decomposition of an r x r Gram matrix
// (r <= 224), so one CTA holds its upper triangle packed in shared memory and
// applies r/2 disjoint rotations per sub-sweep (round-robin pairing); the
// eigenvector matrix is accumulated transposed (rows p, q of V^T change per
// rotation, so the updates are contiguous), in shared memory up to r = 112 and
// in global memory beyond.
#include "dme_internal.h"

#include <algorithm>
#include <cmath>

namespace dme {

namespace {

__device__ __forceinline__ int pk(int a, int b, int r) {   // packed upper triangle, a <= b
    return a * r - (a * (a - 1)) / 2 + (b - a);
}

template <typename T>
__device__ __forceinline__ T pget(const T* A, int x, int y, int r) {
    return x <= y ? A[pk(x, y, r)] : A[pk(y, x, r)];
}

template <typename T>
__device__ __forceinline__ void pset(T* A, int x, int y, int r, T v) {
    if (x <= y) A[pk(x, y, r)] = v;
    else A[pk(y, x, r)] = v;
}

// Round-robin pairing of R (even) indices in sub-sweep t: index 0 stays, the
// others rotate on a circle of R - 1 positions.
__device__ __forceinline__ void rr_pair(int i, int t, int R, int& p, int& q) {
    int a, b;
    if (i == 0) {
        a = 0;
        b = 1 + (t % (R - 1));
    } else {
        a = 1 + ((i + t) % (R - 1));
        b = 1 + ((R - 1 - i + t) % (R - 1));
    }
    p = min(a, b);
    q = max(a, b);
}

constexpr int kJacobiSweeps = 60;

// Symmetric eigen-decomposition of the r x r matrix G (only (G + G^T)/2 is
// used): lam[i] = eigenvalue i, row i of V^T (ldv) = its eigenvector.  A
// rotation is skipped when |a_pq| <= max(1e-14 sqrt(|a_pp a_qq|), 1e-15 max_i
// |a_ii|): what the compression drops with the off-diagonal part is then below
// 1e-14 of the kept terms (the factored path's bar is 1e-11), the FP64 pass
// after the single-precision one (off-diagonal about 1e-7) needs one rotating
// sweep instead of two, and rounding noise below the floor is not chased (a
// Gram matrix formed in floating point carries absolute errors of that size).  The sweeps stop after
// one with no rotation (DEV_NONFINITE in *status after 60 sweeps or on a
// non-finite entry).
// T: the arithmetic (float for a fast first pass, double for the result).
// VS: V^T is accumulated in shared memory too (r <= 112 for double) and copied
// out at the end; otherwise in global memory (Vt_out, double only).
template <typename T, bool VS>
__global__ void __launch_bounds__(1024) jacobi_eig_kernel(const double* __restrict__ G, int ldg, int r,
                                                          double* __restrict__ Vt_out, int ldv_out,
                                                          double* __restrict__ lam, int* status) {
    extern __shared__ __align__(16) unsigned char jsm[];
    const int R = r + (r & 1), P = R / 2;
    T* A = reinterpret_cast<T*>(jsm);
    T* cs = A + (size_t)r * (r + 1) / 2;
    T* sn = cs + P;
    T* tt = sn + P;
    T* Vt = VS ? tt + P : reinterpret_cast<T*>(Vt_out);
    const int ldv = VS ? r : ldv_out;
    constexpr T kRel = sizeof(T) == 4 ? T(1e-7) : T(1e-14);
    constexpr T kFloor = sizeof(T) == 4 ? T(1e-8) : T(1e-15);
    int* pp = reinterpret_cast<int*>(VS ? tt + P + (size_t)r * r : tt + P);
    int* qq = pp + P;
    // (i, j), i <= j, of every rotation block, packed as i << 8 | j (P <= 112)
    unsigned short* blk = reinterpret_cast<unsigned short*>(qq + P);
    const int nblk = P * (P + 1) / 2;
    __shared__ int rotated;
    __shared__ int bad;
    __shared__ T floor_abs;
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) bad = 0;
    for (int i = tid; i < P; i += nt) {
        const int base = i * P - i * (i - 1) / 2;      // blocks (i, i..P-1) start here
        for (int j = i; j < P; ++j) blk[base + j - i] = (unsigned short)((i << 8) | j);
    }
    for (int e = tid; e < r * r; e += nt) {
        const int i = e / r, j = e % r;
        if (i <= j) {
            const double v = 0.5 * (G[(size_t)i * ldg + j] + G[(size_t)j * ldg + i]);
            A[pk(i, j, r)] = (T)v;
            if (!isfinite(v)) bad = 1;
        }
        Vt[(size_t)i * ldv + j] = (i == j) ? T(1) : T(0);
    }
    __syncthreads();
    if (bad) {
        if (tid == 0) atomicOr(status, DEV_NONFINITE);
        return;
    }
    int sweep = 0;
    for (; sweep < kJacobiSweeps; ++sweep) {
        if (tid == 0) {
            rotated = 0;
            T dm = 0;
            for (int i = 0; i < r; ++i) dm = max(dm, abs(A[pk(i, i, r)]));
            floor_abs = kFloor * dm;
        }
        __syncthreads();
        for (int t = 0; t < R - 1; ++t) {
            for (int i = tid; i < P; i += nt) {
                int p, q;
                rr_pair(i, t, R, p, q);
                T c = 1, s = 0, tv = 0;
                if (q < r) {
                    const T apq = A[pk(p, q, r)];
                    const T app = A[pk(p, p, r)], aqq = A[pk(q, q, r)];
                    if (abs(apq) > max(kRel * sqrt(abs(app * aqq)), floor_abs)) {
                        const T th = (aqq - app) / (T(2) * apq);
                        tv = (th >= T(0) ? T(1) : T(-1)) / (abs(th) + sqrt(T(1) + th * th));
                        c = T(1) / sqrt(T(1) + tv * tv);
                        s = tv * c;
                        rotated = 1;
                    }
                }
                pp[i] = p;
                qq[i] = q;
                cs[i] = c;
                sn[i] = s;
                tt[i] = tv;
            }
            __syncthreads();
            // every 2 x 2 block between pairs i <= j: X <- J_i^T X J_j
            for (int e = tid; e < nblk; e += nt) {
                const int i = blk[e] >> 8, j = blk[e] & 0xFF;
                const int pi = pp[i], qi = qq[i], pj = pp[j], qj = qq[j];
                const T ci = cs[i], si = sn[i], cj = cs[j], sj = sn[j];
                if (si == T(0) && sj == T(0)) continue;
                if (i == j) {
                    if (qi >= r) continue;
                    const T apq = A[pk(pi, qi, r)];
                    A[pk(pi, pi, r)] -= tt[i] * apq;
                    A[pk(qi, qi, r)] += tt[i] * apq;
                    A[pk(pi, qi, r)] = T(0);
                    continue;
                }
                const bool qiok = qi < r, qjok = qj < r;
                const T x00 = pget(A, pi, pj, r);
                const T x01 = qjok ? pget(A, pi, qj, r) : T(0);
                const T x10 = qiok ? pget(A, qi, pj, r) : T(0);
                const T x11 = (qiok && qjok) ? pget(A, qi, qj, r) : T(0);
                const T y00 = ci * x00 - si * x10, y01 = ci * x01 - si * x11;
                const T y10 = si * x00 + ci * x10, y11 = si * x01 + ci * x11;
                pset(A, pi, pj, r, cj * y00 - sj * y01);
                if (qjok) pset(A, pi, qj, r, sj * y00 + cj * y01);
                if (qiok) pset(A, qi, pj, r, cj * y10 - sj * y11);
                if (qiok && qjok) pset(A, qi, qj, r, sj * y10 + cj * y11);
            }
            // V <- V J: rows p, q of V^T
            for (int e = tid; e < P * r; e += nt) {
                const int i = e / r, k = e % r;
                const T s = sn[i];
                if (s == T(0)) continue;
                const T c = cs[i];
                const int p = pp[i], q = qq[i];
                const T vp = Vt[(size_t)p * ldv + k], vq = Vt[(size_t)q * ldv + k];
                Vt[(size_t)p * ldv + k] = c * vp - s * vq;
                Vt[(size_t)q * ldv + k] = s * vp + c * vq;
            }
            __syncthreads();
        }
        const int any = rotated;
        __syncthreads();
        if (!any) break;
    }
    for (int i = tid; i < r; i += nt) lam[i] = (double)A[pk(i, i, r)];
    if (VS)
        for (int e = tid; e < r * r; e += nt) Vt_out[(size_t)(e / r) * ldv_out + e % r] = (double)Vt[e];
    if (tid == 0 && sweep == kJacobiSweeps && sizeof(T) == 8) atomicOr(status, DEV_NONFINITE);
}

// Order the eigenvalues decreasingly and keep those above tol * max (max > 0):
// k_out = their count, d_out[rank] = lambda, T[a][rank] = V[a][i] * w with
// w = lambda^{-1/2} (inv_sqrt) or 1.  T has r rows (ldt).
__global__ void __launch_bounds__(256) select_kernel(const double* __restrict__ lam, const double* __restrict__ Vt,
                                                     int ldv, int r, double tol, int inv_sqrt, double* __restrict__ T,
                                                     int ldt, double* d_out, int* k_out, const double* rowscale) {
    __shared__ double smax;
    __shared__ int kcount;
    __shared__ double rs[LR_MAX_RANK];   // sqrt(rowscale), read before d_out (which may alias it) is written
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int a = tid; a < r; a += nt) rs[a] = rowscale ? sqrt(rowscale[a]) : 1.0;
    if (tid == 0) {
        double m = 0.0;
        for (int i = 0; i < r; ++i) m = fmax(m, lam[i]);
        smax = m;
        kcount = 0;
    }
    __syncthreads();
    const double thr = tol * smax;
    for (int i = tid; i < r; i += nt) {
        const double li = lam[i];
        if (!(smax > 0.0) || !(li > thr)) continue;
        int rank = 0;
        for (int j = 0; j < r; ++j) {
            const double lj = lam[j];
            rank += (lj > li) || (lj == li && j < i);
        }
        atomicAdd(&kcount, 1);
        d_out[rank] = li;
        const double w = inv_sqrt ? 1.0 / sqrt(li) : 1.0;
        for (int a = 0; a < r; ++a) T[(size_t)a * ldt + rank] = Vt[(size_t)i * ldv + a] * w * rs[a];
    }
    __syncthreads();
    if (tid == 0) *k_out = kcount;
}

// F = V diag(psi) V^T, psi_i = -t / (sqrt(1 + t l_i) (1 + sqrt(1 + t l_i))), l_i >= 0:
// the matrix function with G F G^T = (I + t G G^T)^{-1/2} - I.
__global__ void ric_weights_kernel(const double* __restrict__ lam, const double* __restrict__ Vt, int ldv, int m,
                                   double t, double* __restrict__ F, int ldf) {
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
        const int a = e / m, b = e % m;
        double acc = 0.0;
        for (int i = 0; i < m; ++i) {
            const double l = fmax(lam[i], 0.0);
            const double sq = sqrt(1.0 + t * l);
            const double psi = -t / (sq * (1.0 + sq));
            acc += Vt[(size_t)i * ldv + a] * psi * Vt[(size_t)i * ldv + b];
        }
        F[(size_t)a * ldf + b] = acc;
    }
}

// Y[i][j] = alpha * X[i][j] * (d ? sqrt(d[j]) : 1) for an n x k block.
// The entries (i, j) of an n x k block a thread visits in a grid-stride loop over
// e = i k + j, walked without a division per entry.
struct BlockEntries {
    int i0, j0, di, dj;
    __device__ BlockEntries(int k) {
        const size_t first = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
        const size_t stride = (size_t)gridDim.x * blockDim.x;
        i0 = (int)(first / k);
        j0 = (int)(first % k);
        di = (int)(stride / k);
        dj = (int)(stride % k);
    }
    __device__ __forceinline__ void next(int& i, int& j, int k) const {
        i += di;
        j += dj;
        if (j >= k) {
            j -= k;
            ++i;
        }
    }
};

// Y = alpha X diag(d)^{1/2} (d NULL: alpha X); the column scales are formed once
// per block (a square root per entry would be FP64-issue bound).
__global__ void __launch_bounds__(256) copy_cols_kernel(double* __restrict__ Y, int ldy, const double* __restrict__ X,
                                                        int ldx, int n, int k, double alpha,
                                                        const double* __restrict__ d) {
    __shared__ double sc[LR_MAX_RANK];
    const bool staged = k <= LR_MAX_RANK;
    if (staged)
        for (int j = threadIdx.x; j < k; j += blockDim.x) sc[j] = d ? alpha * sqrt(d[j]) : alpha;
    __syncthreads();
    const BlockEntries it(k);
    for (int i = it.i0, j = it.j0; i < n; it.next(i, j, k)) {
        const double s = staged ? sc[j] : (d ? alpha * sqrt(d[j]) : alpha);
        Y[(size_t)i * ldy + j] = s * X[(size_t)i * ldx + j];
    }
}

// G_ij *= sqrt(d_i d_j): the Gram matrix of L diag(d)^{1/2} from that of L.
__global__ void sym_scale_kernel(double* __restrict__ G, int ldg, int r, const double* __restrict__ d) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * r; e += gridDim.x * blockDim.x) {
        const int i = e / r, j = e % r;
        G[(size_t)i * ldg + j] *= sqrt(d[i]) * sqrt(d[j]);
    }
}

// C = alpha * sum_s W[s] (+ b1 D1), summed in s order; tri: C symmetric from the upper part.
__global__ void splitk_reduce_kernel(const double* __restrict__ Wk, int S, int M, int N, double* __restrict__ C,
                                     int ldc, double alpha, const double* __restrict__ D1, double b1, int tri) {
    const size_t total = (size_t)M * N;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / N), j = (int)(e % N);
        if (tri && i > j) continue;
        double acc = 0.0;
        for (int s = 0; s < S; ++s) acc += Wk[(size_t)s * total + e];
        double v = alpha * acc;
        if (D1) v += b1 * D1[(size_t)i * ldc + j];
        C[(size_t)i * ldc + j] = v;
        if (tri && i != j) C[(size_t)j * ldc + i] = v;
    }
}

// Partial products of X^T Y for tall X (K x M) and Y (K x N), M N <= 1024:
// block s sums the rows [s chunk, (s + 1) chunk).  The 256 threads form G =
// 256 / E groups (E = M N rounded up to a power of two, at least 32 so a group
// is whole warps, or 256 / 4 entries per thread when M N > 256); group g takes
// the rows k0 + g, k0 + g + G, ..., and the groups' sums are added in group
// order in shared memory.  part: [S][M][N].
__global__ void __launch_bounds__(256) tsgemm_kernel(const double* __restrict__ X, int ldx, int M,
                                                     const double* __restrict__ Y, int ldy, int N, int K, int chunk,
                                                     double* __restrict__ part, int sym) {
    __shared__ double red[1024];
    const int k0 = blockIdx.x * chunk, k1 = min(K, k0 + chunk);
    // sym (X = Y, M = N): only the M (M + 1) / 2 entries i <= j (half the FP64 FMAs)
    const int MN = sym ? M * (M + 1) / 2 : M * N;
    int E = 32;
    while (E < MN && E < 256) E <<= 1;
    const int per = (MN + 255) / 256;                 // entries per thread when E = 256
    const int G = 256 / E;
    const int g = threadIdx.x / E, t = threadIdx.x % E;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int ea[4], eb[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int e = t + E * u;
        ea[u] = 0;
        eb[u] = 0;
        if (e < MN && !sym) {
            ea[u] = e / N;
            eb[u] = e % N;
        } else if (e < MN) {                          // e-th entry of the upper triangle, row by row
            int i = 0, rem = e;
            while (rem >= M - i) {
                rem -= M - i;
                ++i;
            }
            ea[u] = i;
            eb[u] = i + rem;
        }
    }
    for (int k = k0 + g; k < k1; k += G) {
        const double* xr = X + (size_t)k * ldx;
        const double* yr = Y + (size_t)k * ldy;
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (u < per && t + E * u < MN) acc[u] = fma(xr[ea[u]], yr[eb[u]], acc[u]);
    }
    const size_t base = (size_t)blockIdx.x * M * N;   // part keeps the [M][N] layout (sym: i <= j written)
    if (G == 1) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = t + E * u;
            if (u < per && e < MN) part[base + (size_t)ea[u] * N + eb[u]] = acc[u];
        }
        return;
    }
    // G > 1: E <= 128, one entry per thread
    red[threadIdx.x] = acc[0];
    __syncthreads();
    if (g == 0 && t < MN) {
        double v = red[t];
        for (int q = 1; q < G; ++q) v += red[q * E + t];
        part[base + (size_t)ea[0] * N + eb[0]] = v;
    }
}

// C (n x N, ldc) = alpha X op(T) (+ beta D) for X n x K (ldx) and a small op(T)
// (K x N; T stored K x N, or N x K when tT, leading dimension ldt; K, N <= 64)
// staged in shared memory; one thread per output entry.
__global__ void __launch_bounds__(256) tall_small_kernel(const double* __restrict__ X, int ldx, int n, int K,
                                                         const double* __restrict__ Tm, int ldt, int tT, int N,
                                                         double* __restrict__ C, int ldc, double alpha,
                                                         const double* __restrict__ D, double beta) {
    __shared__ double sT[64 * 64];
    for (int e = threadIdx.x; e < K * N; e += blockDim.x) {
        const int k = e / N, j = e % N;
        sT[e] = tT ? Tm[(size_t)j * ldt + k] : Tm[(size_t)k * ldt + j];
    }
    __syncthreads();
    const BlockEntries it(N);
    for (int i = it.i0, j = it.j0; i < n; it.next(i, j, N)) {
        const double* xr = X + (size_t)i * ldx;
        double acc = 0.0;
        for (int k = 0; k < K; ++k) acc = fma(xr[k], sT[k * N + j], acc);
        double v = alpha * acc;
        if (D) v += beta * D[(size_t)i * ldc + j];
        C[(size_t)i * ldc + j] = v;
    }
}

__global__ void fill_kernel(double* __restrict__ x, int k, double v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) x[i] = v;
}

int grid_of(size_t total) { return (int)std::min<size_t>((total + 255) / 256, 152 * 8); }

}  // namespace

constexpr int kJacobiSmemV = 112;    // largest r whose V^T also fits in shared memory (double)
constexpr int kJacobiF32Max = LR_JACOBI_F32_MAX;   // single-precision pass: V^T in shared memory

template <typename T>
static size_t jacobi_smem(int r, bool vs) {
    const int P = (r + (r & 1)) / 2;
    return sizeof(T) * ((size_t)r * (r + 1) / 2 + 3 * (size_t)P + (vs ? (size_t)r * r : 0)) +
           sizeof(int) * 2 * (size_t)P + sizeof(unsigned short) * (size_t)P * (P + 1) / 2;
}

size_t jacobi_smem_bytes(int r) { return jacobi_smem<double>(r, r <= kJacobiSmemV); }

dme_status launch_jacobi_eig(const double* G, int ldg, int r, double* Vt, int ldv, double* lam, int* status,
                             cudaStream_t st, bool fp32) {
    if (r < 1 || r > LR_MAX_RANK) return set_error("jacobi: size must be in [1, 224]"), DME_EINVAL;
    if (fp32 && r > kJacobiF32Max) return set_error("jacobi: the single-precision pass needs r <= 176"), DME_EINVAL;
    // shared-memory limits, set once (thread-safe static initialisation)
    static const cudaError_t attr = [] {
        cudaError_t e = cudaFuncSetAttribute(jacobi_eig_kernel<double, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)jacobi_smem<double>(LR_MAX_RANK, false));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(jacobi_eig_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)jacobi_smem<double>(kJacobiSmemV, true));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(jacobi_eig_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)jacobi_smem<float>(kJacobiF32Max, true));
        return e;
    }();
    DME_CUDA_TRY(attr);
    // enough threads for the P(P+1)/2 rotation blocks of a sub-sweep, no more (fewer warps
    // make the two barriers per sub-sweep cheaper)
    const int P = (r + 1) / 2;
    const int threads = std::min(1024, std::max(64, (P * (P + 1) / 2 + 31) / 32 * 32));
    if (fp32)
        jacobi_eig_kernel<float, true><<<1, threads, jacobi_smem<float>(r, true), st>>>(G, ldg, r, Vt, ldv, lam,
                                                                                     status);
    else if (r <= kJacobiSmemV)
        jacobi_eig_kernel<double, true><<<1, threads, jacobi_smem<double>(r, true), st>>>(G, ldg, r, Vt, ldv, lam,
                                                                                       status);
    else
        jacobi_eig_kernel<double, false><<<1, threads, jacobi_smem<double>(r, false), st>>>(G, ldg, r, Vt, ldv,
                                                                                         lam, status);
    DME_CUDA_TRY(cudaGetLastError());
    return DME_OK;
}

void launch_lr_select(const double* lam, const double* Vt, int ldv, int r, double tol, int inv_sqrt, double* T,
                      int ldt, double* d_out, int* k_out, cudaStream_t st, const double* rowscale) {
    select_kernel<<<1, 256, 0, st>>>(lam, Vt, ldv, r, tol, inv_sqrt, T, ldt, d_out, k_out, rowscale);
}

void launch_sym_scale(double* G, int ldg, int r, const double* d, cudaStream_t st) {
    if (r <= 0) return;
    sym_scale_kernel<<<std::min(1024, (r * r + 255) / 256), 256, 0, st>>>(G, ldg, r, d);
}

void launch_ric_weights(const double* lam, const double* Vt, int ldv, int m, double t, double* F, int ldf,
                        cudaStream_t st) {
    ric_weights_kernel<<<1, 256, 0, st>>>(lam, Vt, ldv, m, t, F, ldf);
}

void launch_copy_cols(double* Y, int ldy, const double* X, int ldx, int n, int k, double alpha, const double* d,
                      cudaStream_t st) {
    if (n <= 0 || k <= 0) return;
    copy_cols_kernel<<<grid_of((size_t)n * k), 256, 0, st>>>(Y, ldy, X, ldx, n, k, alpha, d);
}

// Many partials of a small result: one block per entry, strided sums then a
// fixed tree (deterministic); same outputs as splitk_reduce_kernel.
__global__ void __launch_bounds__(256) splitk_reduce_wide_kernel(const double* __restrict__ Wk, int S, int M, int N,
                                                                 double* __restrict__ C, int ldc, double alpha,
                                                                 const double* __restrict__ D1, double b1, int tri) {
    __shared__ double red[256];
    const size_t total = (size_t)M * N;
    const int e = blockIdx.x;
    const int i = e / N, j = e % N;
    if (tri && i > j) return;
    double acc = 0.0;
    for (int s = threadIdx.x; s < S; s += 256) acc += Wk[(size_t)s * total + e];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double v = alpha * red[0];
        if (D1) v += b1 * D1[(size_t)i * ldc + j];
        C[(size_t)i * ldc + j] = v;
        if (tri && i != j) C[(size_t)j * ldc + i] = v;
    }
}

void launch_splitk_reduce(const double* W, int S, int M, int N, double* C, int ldc, double alpha, const double* D1,
                          double b1, int tri, cudaStream_t st) {
    if (M <= 0 || N <= 0) return;
    if (S >= 64 && (size_t)M * N <= 4096) {
        splitk_reduce_wide_kernel<<<M * N, 256, 0, st>>>(W, S, M, N, C, ldc, alpha, D1, b1, tri);
        return;
    }
    splitk_reduce_kernel<<<grid_of((size_t)M * N), 256, 0, st>>>(W, S, M, N, C, ldc, alpha, D1, b1, tri);
}

void launch_tsgemm(const double* X, int ldx, int M, const double* Y, int ldy, int N, int K, int chunk, double* part,
                   cudaStream_t st, int sym) {
    const int S = (K + chunk - 1) / chunk;
    if (S <= 0 || M * N <= 0) return;
    tsgemm_kernel<<<S, 256, 0, st>>>(X, ldx, M, Y, ldy, N, K, chunk, part, sym && X == Y && ldx == ldy && M == N);
}

void launch_tall_small(const double* X, int ldx, int n, int K, const double* Tm, int ldt, int tT, int N, double* C,
                       int ldc, double alpha, const double* D, double beta, cudaStream_t st) {
    if (n <= 0 || N <= 0) return;
    const size_t total = (size_t)n * N;
    const int grid = (int)std::min<size_t>((total + 255) / 256, 152 * 16);
    tall_small_kernel<<<grid, 256, 0, st>>>(X, ldx, n, K, Tm, ldt, tT, N, C, ldc, alpha, D, beta);
}

void launch_fill(double* x, int k, double v, cudaStream_t st) {
    if (k <= 0) return;
    fill_kernel<<<grid_of((size_t)k), 256, 0, st>>>(x, k, v);
}

}  // namespace dme
