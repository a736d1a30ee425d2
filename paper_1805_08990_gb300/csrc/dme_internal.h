// Internal declarations shared by the libdme translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "dme.h"

namespace dme {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
const char* get_error();

#define DME_CUDA_TRY(expr)                                                          \
    do {                                                                            \
        cudaError_t _e = (expr);                                                    \
        if (_e != cudaSuccess) {                                                    \
            ::dme::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));   \
            return DME_ECUDA;                                                       \
        }                                                                           \
    } while (0)

#define DME_TRY(expr)                                   \
    do {                                                \
        dme_status _s = (expr);                         \
        if (_s != DME_OK) return _s;                    \
    } while (0)

// Device status word bits written by kernels (read back after a sync).
enum : int { DEV_OK = 0, DEV_NOTSPD = 1, DEV_SINGULAR = 2, DEV_NONFINITE = 4, DEV_TIMEOUT = 8 };

// ---------------------------------------------------------------- FP64 GEMM
// One GEMM problem for the grouped FP64 kernel:
//   C = alpha * op(A) op(B) + b1*D1 + b2*D2 + b3*D3
// op(X) = X or X^T.  If tri != 0 the output is symmetric (M == N): only tiles
// on or above the diagonal are computed, and each value (i, j), i <= j, is
// written to both C[i][j] and C[j][i].  D1..D3 are then read on i <= j only.
struct GemmProb {
    const double* A;
    const double* B;
    double* C;
    const double* D1;
    const double* D2;
    const double* D3;
    int M, N, K;
    int lda, ldb, ldc, ldd;
    double alpha, b1, b2, b3;
    int transA, transB, tri;
    int tiles_n;       // filled by the launcher
    int tile_start;    // filled by the launcher
    int ntiles;        // filled by the launcher
};

constexpr int G64_BM = 64, G64_BN = 64, G64_BK = 16;

// Launch descriptors staged on the host and uploaded in one copy before the
// launches that read them run (used when a launch sequence is captured into a
// CUDA graph, where a per-launch host-to-device copy cannot be recorded).
struct DescArena {
    unsigned char* dev = nullptr;        // device block of `cap` bytes
    size_t cap = 0;
    std::vector<unsigned char> host;     // staged bytes; host[i] goes to dev[i]
    // Stage `bytes` from src (256-byte aligned); returns the device address, or
    // nullptr when the block is full.
    void* put(const void* src, size_t bytes);
};

// Enqueue a grouped FP64 GEMM over `probs` (host array).  Descriptors of more
// than 8 problems go to device memory: staged in `arena` when given, else
// copied to `dev_desc` with cudaMemcpyAsync (which must then stay untouched
// until the kernel finished).  `tile` is the square output tile, 32 or 64: both
// accumulate every output over k in the same order, so they give bit-identical
// results and the choice is purely a matter of speed.  The grid is persistent
// (at most the resident CTA count; CTAs stride over the tiles).
dme_status gemm64_grouped(std::vector<GemmProb>& probs, GemmProb* dev_desc, cudaStream_t st,
                          DescArena* arena = nullptr, int tile = 64);
// Query the persistent grid sizes ahead of any stream capture.
void gemm64_prepare();
// One product of fewer 32-wide tiles than half the SMs (the plan's products for
// small n) with K split in up to 8 parts (each at least 16 deep), their partial
// sums in ws, added in part order by a second kernel that applies the epilogue;
// larger products, or ws shorter than the parts need, take gemm64_grouped.  The
// result depends only on the problem's shape, not on the stream or the batch.
dme_status gemm64_splitk(const GemmProb& g, double* ws, size_t ws_len, cudaStream_t st);
size_t gemm64_splitk_ws_doubles(int M, int N);

// ---------------------------------------------------------------- small kernels
void launch_axpy_sym(double* P, const double* Q, double a, int n, int ld, cudaStream_t st);
void launch_transpose(const double* X, double* Y, int rows, int cols, int ldx, int ldy, cudaStream_t st);
void launch_lincomb(double* Y, int n, int ld, const double* X1, double c1, const double* X2, double c2,
                    const double* X3, double c3, double cI, cudaStream_t st);  // Y = c1X1+c2X2+c3X3+cI I
void launch_symmetrize(double* X, int n, int ld, cudaStream_t st);   // X = (X + X^T)/2
void launch_block_norm1(const double* A, const double* Q, int n, double* colsum_out, cudaStream_t st);
void launch_max_reduce(const double* x, int len, double* out, cudaStream_t st);

// B (n x nrhs, ldb) <- M^{-1} B by Gauss-Jordan elimination with partial
// pivoting, blocked by panels of 16 columns (n <= 4096: stream-ordered
// launches per panel; larger: one cooperative launch).  M (n x n with ldm) is
// overwritten.  work: gj_work_doubles(n, nrhs) doubles.
// A zero pivot column sets DEV_SINGULAR.
dme_status launch_gj_solve(double* M, int n, int ldm, double* B, int nrhs, int ldb, double* work, int* status,
                           cudaStream_t st);
size_t gj_work_doubles(int n, int nrhs);
// Self-test of the bounded grid-barrier wait: one block waits for a release
// that never comes; *timed_out = 1 once the wait gave up with DEV_TIMEOUT.
dme_status wait_timeout_selftest(int* timed_out);
// A cooperative launch of a kernel whose blocks wait on one another at grid
// barriers: it needs all its blocks resident, and such kernels running at once
// (plans built on several host threads) could each hold part of the GPU while
// waiting for the rest.  So these launches are admitted process-wide: kernels
// that fit at least 4 blocks per SM (blocks_per_sm) run together while their
// grids sum to at most 4 blocks per SM, which every mix of them can hold at
// once; any other runs alone.  The stream's earlier work is waited for before
// admission, the kernel's completion before release.  Synchronises st; not for
// use under capture.
dme_status coop_launch(const void* func, dim3 grid, dim3 block, void** args, size_t smem, cudaStream_t st,
                       int blocks_per_sm);

// Cholesky of a small SPD matrix (m <= 32) in place (lower), one warp.
void launch_small_cholesky(double* R, int m, int* status, cudaStream_t st);
// Bt = B L^{-T} (rows of B solved against lower L), n x m.
void launch_apply_linv_rows(const double* B, const double* L, double* Bt, int n, int m, cudaStream_t st);

// ---------------------------------------------------------------- low-rank path
constexpr int LR_MAX_RANK = 224;   // columns of L before a compression (shared-memory Jacobi)
constexpr int LR_JACOBI_F32_MAX = 176;   // largest size of the single-precision Jacobi pass
size_t jacobi_smem_bytes(int r);
// Eigen-decomposition of the symmetric r x r matrix G: lam (r), V^T (r x r, ldv).
// fp32: a single-precision pass (converged to about 1e-7), a starting basis for
// the double-precision one; the output is double either way.
dme_status launch_jacobi_eig(const double* G, int ldg, int r, double* Vt, int ldv, double* lam, int* status,
                             cudaStream_t st, bool fp32 = false);
// Keep eigenvalues > tol * max, ordered decreasingly: d_out, k_out, and the
// r x k basis T (columns = eigenvectors, times lambda^{-1/2} if inv_sqrt; row a
// also times sqrt(rowscale[a]) when rowscale is given, which may alias d_out).
void launch_lr_select(const double* lam, const double* Vt, int ldv, int r, double tol, int inv_sqrt, double* T,
                      int ldt, double* d_out, int* k_out, cudaStream_t st, const double* rowscale = nullptr);
// G_ij *= sqrt(d_i d_j) for the r x r matrix G.
void launch_sym_scale(double* G, int ldg, int r, const double* d, cudaStream_t st);
// F = V diag(psi(lam)) V^T (m x m) for the factored Riccati flow over t.
void launch_ric_weights(const double* lam, const double* Vt, int ldv, int m, double t, double* F, int ldf,
                        cudaStream_t st);
// Y = alpha X (n x k block), columns scaled by sqrt(d[j]) when d is given.
void launch_copy_cols(double* Y, int ldy, const double* X, int ldx, int n, int k, double alpha, const double* d,
                      cudaStream_t st);
void launch_fill(double* x, int k, double v, cudaStream_t st);
// part[s] (M x N) = sum over rows k in [s chunk, (s+1) chunk) of X[k]^T Y[k], for
// X (K x M), Y (K x N), M N <= 1024; ceil(K / chunk) partial products.  sym
// (with X = Y): only entries i <= j are formed and written, M (M+1)/2 <= 1024.
void launch_tsgemm(const double* X, int ldx, int M, const double* Y, int ldy, int N, int K, int chunk, double* part,
                   cudaStream_t st, int sym = 0);
// C (n x N) = alpha X op(T) (+ beta D, leading dimension ldc) for a tall X (n x K)
// and a small op(T) (K x N; T^T stored when tT), K, N <= 64; C must not overlap X.
void launch_tall_small(const double* X, int ldx, int n, int K, const double* Tm, int ldt, int tT, int N, double* C,
                       int ldc, double alpha, const double* D, double beta, cudaStream_t st);
// C (M x N) = alpha * sum_{s < S} W[s] (+ b1 D1) with W[s] M x N contiguous; tri mirrors the upper part.
void launch_splitk_reduce(const double* W, int S, int M, int N, double* C, int ldc, double alpha, const double* D1,
                          double b1, int tri, cudaStream_t st);

// Y (n x r, ldy) = alpha S X for S in CSR and X (n x r, ldx); Y must not overlap X.
void launch_spmm(const int* ptr, const int* idx, const double* val, int n, int r, const double* X, int ldx, double* Y,
                 int ldy, double alpha, cudaStream_t st);

// Y (n x r, ldy) = e^{t A^T} X (n x r, ldx) by Newton interpolation at Leja
// points, all substeps in one persistent cooperative launch: per substep
// p = d_0 v, w_{k+1} = (A^T w_k - c w_k) invg - xi_k w_k, p += d_{k+1} w_{k+1}
// (val holds the values of A^T already multiplied by invg = 1/g),
// stopping after two consecutive terms with |d_k| |w_k|_F <= tol |p|_F (at most
// `terms` - 1 terms), then v = scale p.  Y may be X.  Wa, Wb: n x r scratch
// (ldw); part: 4 leja_grid_max() doubles; sums: 4 doubles; bar: 2 unsigned.
struct LejaCall {
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
    const double* xi;    // host, `terms` Leja points
    const double* dd;    // host, `terms` divided differences
    double* part;
    double* sums;
    unsigned* bar;
    int* status;         // DEV_TIMEOUT if a grid barrier wait ran out
};
int leja_grid_max();
dme_status launch_leja_apply(const LejaCall& c, cudaStream_t st);

// ---------------------------------------------------------------- Riccati (T3)
// P <- P - t Z (I + t Bt^T Z)^{-1} Z^T + q * Qadd, Z = P Bt  (Woodbury form
// of (I + t P Bt Bt^T)^{-1} P).  Work buffers sized by riccati_work_doubles.
size_t riccati_work_doubles(int n, int m);
void launch_riccati(double* P, const double* Bt, int n, int m, double t, const double* Qadd,
                    double q, double* work, int* status, cudaStream_t st);
struct RicItem {
    double* P;
    const double* Bt;
    int n, m;
    double t;
    const double* Qadd;
    double q;
    double* work;
    int* status;
};
RicItem make_ric_item(double* P, const double* Bt, int n, int m, double t, const double* Qadd, double q,
                      double* work, int* status);
// Grouped launch over independent problems; more than 8 need `dev_desc`
// (riccati_desc_bytes() per problem, untouched until the kernels finish).
dme_status launch_riccati_grouped(const std::vector<RicItem>& items, void* dev_desc, cudaStream_t st,
                                  DescArena* arena = nullptr);
size_t riccati_desc_bytes();
// Kernels (2)-(3) of the Riccati flow for one problem whose Z = P Bt (n x m) is
// already in work (its first n m doubles): Gram partials, M = I + t Bt^T Z, its
// Cholesky, Y = Z L^{-T} (Y = 0 if M is not SPD, with DEV_NOTSPD set).
dme_status launch_riccati_from_z(const double* Bt, int n, int m, double t, double* work, int* status,
                                 cudaStream_t st);
// As launch_lqr_gain, into Kbase + (*ctr) m n (skipped once *ctr >= cap), then
// ++*ctr on the device: for a launch sequence replayed once per step.
dme_status launch_lqr_gain_hist(const double* P, const double* Bt, const double* LR, int n, int m, double* work,
                                double* Kbase, int* ctr, int cap, cudaStream_t st);
// K (m x n) = R^{-1} B^T P from Bt = B L^{-T} and L (R = L L^T); work as for launch_riccati.
dme_status launch_lqr_gain(const double* P, const double* Bt, const double* LR, int n, int m, double* work,
                           double* K, cudaStream_t st);

}  // namespace dme
