// Low-rank (factored) splitting schemes: the state P = L diag(d) L^T stays in
// factored form and every sub-flow acts on the factors (§2.1-2.3 factor forms;
// Alg. 1-4).  The dense FP64 plan underneath supplies the data (A, Q = C^T C,
// Bt = B L_R^{-T}, S) and the exponentials E_t = e^{tA} of its Pade path.
//
//   T_1(t):  L <- E_t^T L                         (Eq. F_sol_LDL with e^{tA^T} = E_t^T)
//   T_2(t):  L <- [L, C^T], d <- [d, t 1_p]       then compression
//   T_12(t): L <- [E_t^T L, L_I], d <- [d, d_I]   then compression; (L_I, d_I) is the
//            compressed Gauss-Legendre factor of W_t (Alg. 2), built once per t
//   T_3(t):  with Lt = L diag(d)^{1/2} and G = Lt^T Bt (r x m):
//            L <- Lt (I + t G G^T)^{-1/2} = Lt + (Lt G) F(G^T G) G^T, d <- 1, where
//            F(x) = -t / (sqrt(1 + t x)(1 + sqrt(1 + t x))); equal to the §2.2 form
//            L (I + t D L^T B R^{-1} B^T L)^{-1} D L^T by the push-through identity
//   T_4(t):  L <- [L, sqrt(t) S L, sqrt(t/2) S (sqrt(t) S L)], d <- [d, d, d] (midpoint)
//            or [L, sqrt(t) S L], [d, d] (Euler), then compression
//   compression: Lt = L diag(d)^{1/2}; Lt^T Lt = V Lambda V^T (Jacobi);
//            L <- Lt V_k Lambda_k^{-1/2}, d <- lambda_k for lambda > tol * max lambda,
//            i.e. the eigen-decomposition of P restricted to its numerical range
//            (the paper's reduced SVD followed by the small diagonalisation).
// d stays positive throughout (P is positive semidefinite).
#include "plan_internal.h"

#include <cmath>
#include <cstring>
#include <memory>
#include <utility>
#include <vector>

using namespace dme;

namespace {

struct WFactor {
    double tau;
    double* L;   // n x k, leading dimension k
    double* d;   // k
    int k;
};

}  // namespace

struct LejaTab {          // e^{tau A^T} by Leja interpolation: per step length tau
    double tau;
    int s;                   // substeps
    double scale;            // e^{t c}, t = tau / s
    std::vector<double> dd;  // divided differences of exp(t g x) at the Leja points
};

struct dme_lr_s {
    dme_plan_t P = nullptr;   // dense plan (data, E_t); NULL for a sparse A
    dme_plan_desc desc;       // the descriptor
    cudaStream_t st = nullptr;
    bool own_st = false;
    int* status = nullptr;    // device status word (the dense plan's, or own)
    const double* Bt = nullptr;   // B L_R^{-T} (n x m)
    // sparse A: A^T in CSR (device), Gershgorin data and Leja tables
    bool sparse = false;
    int nnz = 0;
    int *at_ptr = nullptr, *at_idx = nullptr;
    double* at_val = nullptr;   // values of A^T / g
    int *s_ptr = nullptr, *s_idx = nullptr;   // sparse S (CSR, device), for T4
    double* s_val = nullptr;
    double lc = 0.0, lg = 0.0;       // A^T = lc I + lg X, spectrum of X in [-2, 2] (Gershgorin)
    std::vector<double> xi;          // Leja points
    std::vector<LejaTab> ltab;
    double *Wa = nullptr, *Wb = nullptr;   // Leja work (n x rcap)
    double *lpart = nullptr, *lnorm = nullptr;  // per-block partial norms; norms and grid-barrier words
    int n = 0, m = 0, p = 0, rcap = 0, q = 7;
    double tol = 1e-13;
    double *L = nullptr, *L2 = nullptr, *d = nullptr, *d2 = nullptr;   // n x rcap, rcap
    double* LQ = nullptr;                                            // C^T, n x p
    double *G = nullptr, *Vt = nullptr, *lam = nullptr, *T = nullptr;  // rcap x rcap work
    double *J1 = nullptr, *J2 = nullptr, *J3 = nullptr, *J4 = nullptr;  // rcap x rcap eigensolver work
    double *Gm = nullptr, *H = nullptr, *VtH = nullptr, *lamH = nullptr, *F = nullptr, *Y = nullptr, *Z = nullptr;
    double* Pout = nullptr;   // n x n, allocated on the first dense output
    int* kdev = nullptr;
    bool split = false;            // the products with E_t and S on the tensor cores
    SliceBuf xsl;                  // split: slices of X^T for M X (rows = rmax, k = n)
    double* Xtr = nullptr;         // split: X^T (rmax x n)
    double* ws = nullptr;          // split-K partial products
    size_t ws_doubles = 0;
    GemmProb* wsdesc = nullptr;    // their descriptors (kSplitMax)
    std::vector<WFactor> wf;
    std::vector<void*> allocs;
    int r = 0;
};

namespace {

dme_status lr_alloc(dme_lr_t lr, double** out, size_t count) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(out), std::max<size_t>(count, 1) * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("low-rank plan: cudaMalloc: ") + cudaGetErrorString(e));
        return DME_ENOMEM;
    }
    lr->allocs.push_back(*out);
    return DME_OK;
}

GemmProb mk(int M, int N, int K, const double* A, int lda, int tA, const double* B, int ldb, int tB, double* C,
            int ldc, double alpha, int tri = 0, const double* D1 = nullptr, double b1 = 0.0) {
    GemmProb g;
    std::memset(&g, 0, sizeof(g));
    g.A = A;
    g.B = B;
    g.C = C;
    g.D1 = D1;
    g.M = M;
    g.N = N;
    g.K = K;
    g.lda = lda;
    g.ldb = ldb;
    g.ldc = ldc;
    g.ldd = ldc;
    g.alpha = alpha;
    g.b1 = b1;
    g.transA = tA;
    g.transB = tB;
    g.tri = tri;
    return g;
}

constexpr int kSplitMax = 64;   // K chunks of a split-K product

dme_status gemm_ws(dme_lr_t lr, const GemmProb& g, cudaStream_t st);

// FP64 product of the low-rank path.  Skinny outputs (N <= 64) use 32-wide
// tiles; a small output with a long K (Gram matrices L^T L, L^T Bt) is split
// into K chunks, one grouped launch, then summed in chunk order.
dme_status gemm(dme_lr_t lr, const GemmProb& g, cudaStream_t st) {
    if (g.M <= 0 || g.N <= 0) return DME_OK;
    const bool sym = g.tri && g.A == g.B && g.lda == g.ldb && g.M == g.N;
    if (g.transA && !g.transB && (g.M * g.N <= 1024 || (sym && g.M * (g.M + 1) / 2 <= 1024)) && g.K >= 1024) {
        // X^T Y of two tall blocks with a small result: row chunks summed per CTA
        // (a Gram matrix X^T X: its upper triangle only)
        const size_t mn = (size_t)g.M * g.N;
        const int smax = (int)std::min<size_t>(2048, lr->ws_doubles / mn);
        const int chunk = std::max(64, (g.K + smax - 1) / smax);
        const int S = (g.K + chunk - 1) / chunk;
        launch_tsgemm(g.A, g.lda, g.M, g.B, g.ldb, g.N, g.K, chunk, lr->ws, st, sym);
        launch_splitk_reduce(lr->ws, S, g.M, g.N, g.C, g.ldc, g.alpha, g.D1, g.b1, g.tri, st);
        return DME_OK;
    }
    if (!g.transA && !g.tri && !g.D2 && !g.D3 && g.K <= 64 && g.N <= 64 && g.M >= 2048 && g.C != g.A) {
        // tall X times a small matrix: one thread per output entry, the small factor in shared memory
        launch_tall_small(g.A, g.lda, g.M, g.K, g.B, g.ldb, g.transB, g.N, g.C, g.ldc, g.alpha, g.D1, g.b1, st);
        return DME_OK;
    }
    const long tiles64 = (long)((g.M + 63) / 64) * ((g.N + 63) / 64);
    if (tiles64 <= 16 && g.K >= 1024) return gemm_ws(lr, g, st);
    std::vector<GemmProb> v{g};
    return gemm64_grouped(v, nullptr, st, nullptr, g.N <= 64 ? 32 : 64);
}

dme_status gemm_ws(dme_lr_t lr, const GemmProb& g, cudaStream_t st) {
    const size_t mn = (size_t)g.M * g.N;
    int S = std::min(kSplitMax, std::max(1, g.K / 128));
    S = std::max(1, std::min<int>(S, (int)(lr->ws_doubles / mn)));
    const int chunk = ((g.K + S - 1) / S + 15) / 16 * 16;
    S = (g.K + chunk - 1) / chunk;
    std::vector<GemmProb> parts;
    for (int s = 0; s < S; ++s) {
        const int k0 = s * chunk, kc = std::min(chunk, g.K - k0);
        GemmProb q = g;
        q.K = kc;
        q.A = g.transA ? g.A + (size_t)k0 * g.lda : g.A + k0;
        q.B = g.transB ? g.B + k0 : g.B + (size_t)k0 * g.ldb;
        q.C = lr->ws + (size_t)s * mn;
        q.ldc = q.ldd = g.N;
        q.alpha = 1.0;
        q.tri = 0;
        q.D1 = q.D2 = q.D3 = nullptr;
        parts.push_back(q);
    }
    DME_TRY(gemm64_grouped(parts, lr->wsdesc, st, nullptr, g.N <= 64 ? 32 : 64));
    launch_splitk_reduce(lr->ws, S, g.M, g.N, g.C, g.ldc, g.alpha, g.D1, g.b1, g.tri, st);
    return DME_OK;
}

// Eigen-decomposition of the r x r Gram matrix lr->G: eigenvalues in lr->lam,
// eigenvectors in the rows of lr->Vt.  Two passes for 8 <= r <= 176: a
// single-precision Jacobi solve gives X (rows about orthonormal to 1e-7); two
// Newton-Schulz steps X <- (3X - (X X^T) X) / 2 make the rows orthonormal in
// FP64; the FP64 Jacobi solver then diagonalises X G X^T, which is diagonal to
// about 1e-7 already, in a few sweeps; the eigenvectors are the rows of V2 X.
dme_status eig_gram(dme_lr_t lr, int r) {
    cudaStream_t st = lr->st;
    const int rc = lr->rcap;
    if (r < 8 || r > LR_JACOBI_F32_MAX)
        return launch_jacobi_eig(lr->G, rc, r, lr->Vt, rc, lr->lam, lr->status, st);
    DME_TRY(launch_jacobi_eig(lr->G, rc, r, lr->J1, rc, lr->lam, lr->status, st, true));
    double* X = lr->J1;
    double* Xn = lr->J3;
    for (int it = 0; it < 2; ++it) {
        DME_TRY(gemm(lr, mk(r, r, r, X, rc, 0, X, rc, 1, lr->J2, rc, 1.0, 1), st));                  // X X^T
        DME_TRY(gemm(lr, mk(r, r, r, lr->J2, rc, 0, X, rc, 0, Xn, rc, -0.5, 0, X, 1.5), st));        // (3X - YX)/2
        std::swap(X, Xn);
    }
    DME_TRY(gemm(lr, mk(r, r, r, lr->G, rc, 0, X, rc, 1, lr->J2, rc, 1.0), st));                     // G X^T
    DME_TRY(gemm(lr, mk(r, r, r, X, rc, 0, lr->J2, rc, 0, lr->J4, rc, 1.0, 1), st));                 // X G X^T
    DME_TRY(launch_jacobi_eig(lr->J4, rc, r, lr->J2, rc, lr->lam, lr->status, st));
    return gemm(lr, mk(r, r, r, lr->J2, rc, 0, X, rc, 0, lr->Vt, rc, 1.0), st);                      // V2 X
}

// Compress the factor (L, d) with r columns (leading dimension ld) in place;
// L2 is an n x ld work buffer.  Reads the new rank back to the host.
// With Lt = L diag(d)^{1/2}, Lt is never formed: its Gram matrix is diag(d)^{1/2}
// (L^T L) diag(d)^{1/2}, and the new factor Lt V_k Lambda^{-1/2} is L times the
// small matrix diag(d)^{1/2} V_k Lambda^{-1/2}, written to L2; the two buffers
// then trade places (L names the result).
dme_status compress(dme_lr_t lr, double*& L, double*& L2, double* d, int ld, int& r) {
    if (r == 0) return DME_OK;
    cudaStream_t st = lr->st;
    const int n = lr->n;
    DME_TRY(gemm(lr, mk(r, r, n, L, ld, 1, L, ld, 0, lr->G, lr->rcap, 1.0, 1), st));            // L^T L
    launch_sym_scale(lr->G, lr->rcap, r, d, st);                                              // Lt^T Lt
    DME_TRY(eig_gram(lr, r));
    launch_lr_select(lr->lam, lr->Vt, lr->rcap, r, lr->tol, 1, lr->T, lr->rcap, d, lr->kdev, st, d);
    int k = 0;
    DME_CUDA_TRY(cudaMemcpyAsync(&k, lr->kdev, sizeof(int), cudaMemcpyDeviceToHost, st));
    DME_CUDA_TRY(cudaStreamSynchronize(st));
    DME_TRY(gemm(lr, mk(n, k, r, L, ld, 0, lr->T, lr->rcap, 0, L2, ld, 1.0), st));              // Lt V_k Lambda^-1/2
    std::swap(L, L2);
    r = k;
    return DME_OK;
}

dme_status need_cols(dme_lr_t lr, int cols) {
    if (cols > lr->rcap)
        return set_error("low-rank path: " + std::to_string(cols) + " columns exceed the capacity " +
                         std::to_string(lr->rcap) + " (raise rmax up to 224, or tol)"),
               DME_ENOMEM;
    return DME_OK;
}

// Gauss-Legendre nodes and weights on [0, t] (Newton on the Legendre recurrence).
void gauss_legendre(int q, double t, std::vector<double>& s, std::vector<double>& w) {
    s.assign(q, 0.0);
    w.assign(q, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (q + 1) / 2; ++i) {
        double x = std::cos(pi * (i + 0.75) / (q + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= q; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (q == 1) {
                p1 = x;
                p0 = 1.0;
            }
            dp = q * (x * p1 - p0) / (x * x - 1.0);
            const double dx = p1 / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = x;
            for (int k = 2; k <= q; ++k) {
                const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (q == 1) p0 = 1.0, p1 = x;
            dp = q * (x * p1 - p0) / (x * x - 1.0);
        }
        const double wi = 2.0 / ((1.0 - x * x) * dp * dp);
        // nodes x_i (descending) and -x_i, mapped to [0, t]
        s[i] = 0.5 * t * (1.0 + x);
        s[q - 1 - i] = 0.5 * t * (1.0 - x);
        w[i] = w[q - 1 - i] = 0.5 * t * wi;
    }
}

// ---------------------------------------------------------------- Leja action (sparse A)
constexpr int kLejaTerms = 80;        // interpolation points per substep
constexpr double kLejaRho = 4.0;      // largest t g per substep
constexpr double kLejaTol = 1e-15;    // series stops after two terms below tol |p|
constexpr int kLejaGrid = 20001;      // candidate points for the greedy Leja sequence

// Leja points of [-2, 2] from 2: x_k maximises prod_{i<k} |x - x_i| over a grid.
std::vector<double> leja_points_host(int m) {
    std::vector<double> xs(kLejaGrid), lp(kLejaGrid);
    const double step = 4.0 / (kLejaGrid - 1);
    for (int i = 0; i < kLejaGrid; ++i) {
        xs[i] = -2.0 + i * step;
        lp[i] = std::log(std::fabs(xs[i] - 2.0));
    }
    std::vector<double> pts{2.0};
    for (int k = 1; k < m; ++k) {
        int best = 0;
        for (int i = 1; i < kLejaGrid; ++i)
            if (lp[i] > lp[best]) best = i;
        pts.push_back(xs[best]);
        for (int i = 0; i < kLejaGrid; ++i) lp[i] += std::log(std::fabs(xs[i] - xs[best]));
    }
    return pts;
}

// First column of exp(a Z), Z lower bidiagonal with x on the diagonal and ones
// below: the divided differences of exp(a x) at x_0, x_1, ... (Opitz).  Taylor
// series of degree 30 after scaling to 1-norm <= 1/2, then repeated squaring
// (lower-triangular products).
std::vector<double> dd_exp_host(const std::vector<double>& x, double a) {
    const int m = (int)x.size();
    std::vector<double> M((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) {
        M[(size_t)i * m + i] = a * x[i];
        if (i > 0) M[(size_t)i * m + i - 1] = a;
    }
    double nrm = 0.0;
    for (int j = 0; j < m; ++j) nrm = std::max(nrm, std::fabs(M[(size_t)j * m + j]) + (j + 1 < m ? std::fabs(a) : 0.0));
    int sq = 0;
    while (nrm > 0.5) {
        nrm *= 0.5;
        ++sq;
    }
    const double f = std::ldexp(1.0, -sq);
    for (double& v : M) v *= f;
    auto mul = [m](const std::vector<double>& X, const std::vector<double>& Y) {
        std::vector<double> Zm((size_t)m * m, 0.0);
        for (int i = 0; i < m; ++i)
            for (int k = 0; k <= i; ++k) {
                const double xv = X[(size_t)i * m + k];
                if (xv == 0.0) continue;
                for (int j = 0; j <= k; ++j) Zm[(size_t)i * m + j] += xv * Y[(size_t)k * m + j];
            }
        return Zm;
    };
    std::vector<double> E((size_t)m * m, 0.0), T((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) E[(size_t)i * m + i] = T[(size_t)i * m + i] = 1.0;
    for (int k = 1; k <= 30; ++k) {
        T = mul(T, M);
        for (double& v : T) v /= k;
        for (size_t e = 0; e < E.size(); ++e) E[e] += T[e];
    }
    for (int i = 0; i < sq; ++i) E = mul(E, E);
    std::vector<double> col(m);
    for (int i = 0; i < m; ++i) col[i] = E[(size_t)i * m];
    return col;
}

const LejaTab& leja_table(dme_lr_t lr, double tau) {
    for (auto& t : lr->ltab)
        if (t.tau == tau) return t;
    LejaTab t;
    t.tau = tau;
    t.s = std::max(1, (int)std::ceil(tau * lr->lg / kLejaRho));
    const double sub = tau / t.s;
    t.scale = std::exp(sub * lr->lc);
    t.dd = dd_exp_host(lr->xi, sub * lr->lg);
    lr->ltab.push_back(t);
    return lr->ltab.back();
}

// Y (n x k, ldy) = e^{tau A^T} X (n x k, ldx) by Leja interpolation; Y may be X.
dme_status leja_apply(dme_lr_t lr, const double* X, int ldx, int k, double* Y, int ldy, double tau) {
    if (k == 0) return DME_OK;
    cudaStream_t st = lr->st;
    const int n = lr->n, rc = lr->rcap;
    if (!(lr->lg > 0.0)) {                              // A = c I
        launch_copy_cols(Y, ldy, X, ldx, n, k, std::exp(tau * lr->lc), nullptr, st);
        return DME_OK;
    }
    const LejaTab& tb = leja_table(lr, tau);
    LejaCall c;
    c.ptr = lr->at_ptr;
    c.idx = lr->at_idx;
    c.val = lr->at_val;
    c.n = n;
    c.r = k;
    c.X = X;
    c.ldx = ldx;
    c.Y = Y;
    c.ldy = ldy;
    c.Wa = lr->Wa;
    c.Wb = lr->Wb;
    c.ldw = rc;
    c.c = lr->lc;
    c.invg = 1.0 / lr->lg;
    c.scale = tb.scale;
    c.tol = kLejaTol;
    c.substeps = tb.s;
    c.terms = kLejaTerms;
    c.xi = lr->xi.data();
    c.dd = tb.dd.data();
    c.part = lr->lpart;
    c.sums = lr->lnorm;
    c.bar = reinterpret_cast<unsigned*>(lr->lnorm + 4);
    c.status = lr->status;
    DME_TRY(launch_leja_apply(c, st));
    DME_CUDA_TRY(cudaGetLastError());
    return DME_OK;
}

dme_status wfactor(dme_lr_t lr, double tau, const WFactor** out) {
    for (auto& f : lr->wf)
        if (f.tau == tau) {
            *out = &f;
            return DME_OK;
        }
    cudaStream_t st = lr->st;
    const int n = lr->n, p = lr->p, q = lr->q, k0 = q * p;
    DME_TRY(need_cols(lr, k0));
    std::vector<double> s, w;
    gauss_legendre(q, tau, s, w);
    // temporaries, freed (after the stream drained) when this function returns
    struct Tmp {
        cudaStream_t st;
        std::vector<void*> v;
        ~Tmp() {
            cudaStreamSynchronize(st);
            for (void* x : v) cudaFree(x);
        }
        dme_status get(double** o, size_t count) {
            if (cudaMalloc(reinterpret_cast<void**>(o), count * sizeof(double)) != cudaSuccess) {
                cudaGetLastError();
                set_error("low-rank plan: cudaMalloc (quadrature factor) failed");
                return DME_ENOMEM;
            }
            v.push_back(*o);
            return DME_OK;
        }
    } tmp{st, {}};
    double *WL = nullptr, *WL2 = nullptr, *wd = nullptr;
    DME_TRY(tmp.get(&WL, (size_t)n * lr->rcap));
    DME_TRY(tmp.get(&WL2, (size_t)n * lr->rcap));
    DME_TRY(tmp.get(&wd, (size_t)lr->rcap));
    for (int k = 0; k < q; ++k) {
        if (lr->sparse) {
            DME_TRY(leja_apply(lr, lr->LQ, p, p, WL + (size_t)k * p, lr->rcap, s[k]));                 // e^{s A^T} C^T
        } else {
            int idx;
            DME_TRY(plan_ew(lr->P, s[k], &idx));
            const double* E = lr->P->ew[idx].E;
            DME_TRY(gemm(lr, mk(n, p, n, E, n, 1, lr->LQ, p, 0, WL + (size_t)k * p, lr->rcap, 1.0), st));   // E_s^T C^T
        }
        launch_fill(wd + (size_t)k * p, p, w[k], st);
    }
    int r = k0;
    DME_TRY(compress(lr, WL, WL2, wd, lr->rcap, r));
    WFactor f;
    f.tau = tau;
    f.k = r;
    DME_TRY(lr_alloc(lr, &f.L, (size_t)n * std::max(r, 1)));
    DME_TRY(lr_alloc(lr, &f.d, (size_t)std::max(r, 1)));
    launch_copy_cols(f.L, std::max(r, 1), WL, lr->rcap, n, r, 1.0, nullptr, st);
    if (r > 0) DME_CUDA_TRY(cudaMemcpyAsync(f.d, wd, sizeof(double) * r, cudaMemcpyDeviceToDevice, st));
    DME_CUDA_TRY(cudaStreamSynchronize(st));
    lr->wf.push_back(f);
    *out = &lr->wf.back();
    return DME_OK;
}

// Split precision: C (n x k, ldc) = alpha M X for X (n x k, ldx), M given by the
// bf16 slices of its rows (E_t^T or S of the plan): X^T is sliced and the
// tcgen05 GEMM forms M (X^T)^T with FP64 output.
dme_status apply_split(dme_lr_t lr, const SliceBuf& Msl, const double* X, int ldx, int k, double* C, int ldc,
                       double alpha) {
    if (k == 0) return DME_OK;
    cudaStream_t st = lr->st;
    const int n = lr->n;
    launch_transpose(X, lr->Xtr, n, k, ldx, n, st);
    launch_slice_rows_f64(lr->Xtr, k, n, n, lr->xsl, st);
    OzParams p;
    DME_TRY(oz_params(Msl, lr->xsl, OZ_P14, &p));
    p.M = n;
    p.N = k;                     // the first k of the buffer's rows
    p.mode = OZ_OUT_F64;
    p.ldc = ldc;
    p.Cd = C;
    p.alpha = alpha;
    p.status = lr->status;
    p.ws = lr->P->kws;
    p.ws_cnt = lr->P->kcnt;
    return launch_ozaki_gemm(oz_tmap_a(Msl, OZ_P14), oz_tmap_b(lr->xsl, OZ_P14), p, st);
}

dme_status lr_T1(dme_lr_t lr, double tau) {
    if (lr->r == 0) return DME_OK;
    if (lr->sparse) {
        DME_TRY(leja_apply(lr, lr->L, lr->rcap, lr->r, lr->L2, lr->rcap, tau));
        std::swap(lr->L, lr->L2);
        return DME_OK;
    }
    int idx;
    DME_TRY(plan_ew(lr->P, tau, &idx));
    const EWEntry& e = lr->P->ew[idx];
    if (lr->split)
        DME_TRY(apply_split(lr, e.Gsl, lr->L, lr->rcap, lr->r, lr->L2, lr->rcap, 1.0));
    else
        DME_TRY(gemm(lr, mk(lr->n, lr->r, lr->n, e.E, lr->n, 1, lr->L, lr->rcap, 0, lr->L2, lr->rcap, 1.0),
                     lr->st));
    std::swap(lr->L, lr->L2);
    return DME_OK;
}

dme_status lr_append(dme_lr_t lr, const double* X, int ldx, int k, const double* dsrc, double dval) {
    DME_TRY(need_cols(lr, lr->r + k));
    cudaStream_t st = lr->st;
    launch_copy_cols(lr->L + lr->r, lr->rcap, X, ldx, lr->n, k, 1.0, nullptr, st);
    if (dsrc) DME_CUDA_TRY(cudaMemcpyAsync(lr->d + lr->r, dsrc, sizeof(double) * k, cudaMemcpyDeviceToDevice, st));
    else launch_fill(lr->d + lr->r, k, dval, st);
    lr->r += k;
    return DME_OK;
}

dme_status lr_T2(dme_lr_t lr, double tau) {
    DME_TRY(lr_append(lr, lr->LQ, lr->p, lr->p, nullptr, tau));
    return compress(lr, lr->L, lr->L2, lr->d, lr->rcap, lr->r);
}

dme_status lr_T12(dme_lr_t lr, double tau) {
    const WFactor* f = nullptr;
    DME_TRY(wfactor(lr, tau, &f));
    DME_TRY(lr_T1(lr, tau));
    if (f->k > 0) DME_TRY(lr_append(lr, f->L, f->k, f->k, f->d, 0.0));
    return compress(lr, lr->L, lr->L2, lr->d, lr->rcap, lr->r);
}

dme_status lr_T3(dme_lr_t lr, double tau) {
    if (lr->r == 0) return DME_OK;
    cudaStream_t st = lr->st;
    const int n = lr->n, m = lr->m, r = lr->r, rc = lr->rcap;
    launch_copy_cols(lr->L2, rc, lr->L, rc, n, r, 1.0, lr->d, st);                              // Lt
    DME_TRY(gemm(lr, mk(r, m, n, lr->L2, rc, 1, lr->Bt, m, 0, lr->Gm, m, 1.0), st));              // G = Lt^T Bt
    DME_TRY(gemm(lr, mk(m, m, r, lr->Gm, m, 1, lr->Gm, m, 0, lr->H, m, 1.0, 1), st));                // G^T G
    DME_TRY(launch_jacobi_eig(lr->H, m, m, lr->VtH, m, lr->lamH, lr->status, st));
    launch_ric_weights(lr->lamH, lr->VtH, m, m, tau, lr->F, m, st);                               // F(G^T G)
    DME_TRY(gemm(lr, mk(r, m, m, lr->Gm, m, 0, lr->F, m, 0, lr->Y, m, 1.0), st));                    // Y = G F
    DME_TRY(gemm(lr, mk(n, m, r, lr->L2, rc, 0, lr->Gm, m, 0, lr->Z, m, 1.0), st));                  // Z = Lt G
    DME_TRY(gemm(lr, mk(n, r, m, lr->Z, m, 0, lr->Y, m, 1, lr->L, rc, 1.0, 0, lr->L2, 1.0), st));    // L = Lt + Z Y^T
    launch_fill(lr->d, r, 1.0, st);
    return DME_OK;
}

dme_status lr_T4(dme_lr_t lr, double tau, int rule) {
    if (lr->r == 0) return DME_OK;
    cudaStream_t st = lr->st;
    const int n = lr->n, r = lr->r, rc = lr->rcap;
    const int blocks = rule == DME_T4_EULER ? 2 : 3;
    DME_TRY(need_cols(lr, blocks * r));
    if (lr->sparse) {
        launch_spmm(lr->s_ptr, lr->s_idx, lr->s_val, n, r, lr->L, rc, lr->L + r, rc, std::sqrt(tau), st);
        if (blocks == 3)
            launch_spmm(lr->s_ptr, lr->s_idx, lr->s_val, n, r, lr->L + r, rc, lr->L + 2 * r, rc, std::sqrt(0.5 * tau),
                        st);
        for (int b = 1; b < blocks; ++b)
            DME_CUDA_TRY(cudaMemcpyAsync(lr->d + b * r, lr->d, sizeof(double) * r, cudaMemcpyDeviceToDevice, st));
        lr->r = blocks * r;
        return compress(lr, lr->L, lr->L2, lr->d, rc, lr->r);
    }
    const double* S = lr->P->S;
    if (lr->split) {
        DME_TRY(apply_split(lr, lr->P->Ssl, lr->L, rc, r, lr->L + r, rc, std::sqrt(tau)));
        if (blocks == 3) DME_TRY(apply_split(lr, lr->P->Ssl, lr->L + r, rc, r, lr->L + 2 * r, rc, std::sqrt(0.5 * tau)));
    } else {
        DME_TRY(gemm(lr, mk(n, r, n, S, n, 0, lr->L, rc, 0, lr->L + r, rc, std::sqrt(tau)), st));          // sqrt(t) S L
        if (blocks == 3)
            DME_TRY(gemm(lr, mk(n, r, n, S, n, 0, lr->L + r, rc, 0, lr->L + 2 * r, rc, std::sqrt(0.5 * tau)), st));
    }
    for (int b = 1; b < blocks; ++b)
        DME_CUDA_TRY(cudaMemcpyAsync(lr->d + b * r, lr->d, sizeof(double) * r, cudaMemcpyDeviceToDevice, st));
    lr->r = blocks * r;
    return compress(lr, lr->L, lr->L2, lr->d, rc, lr->r);
}

int t4_rule(const dme_plan_desc& d) {
    if (d.t4_rule == DME_T4_MIDPOINT || d.t4_rule == DME_T4_EULER) return d.t4_rule;
    return d.comp == DME_STRANG ? DME_T4_MIDPOINT : DME_T4_EULER;
}

dme_status lr_apply(dme_lr_t lr, int flow, double tau) {
    switch (flow) {
        case DME_F1: return lr_T1(lr, tau);
        case DME_F2: return lr_T2(lr, tau);
        case DME_F12: return lr_T12(lr, tau);
        case DME_F3: return lr_T3(lr, tau);
        case DME_F4: return lr_T4(lr, tau, t4_rule(lr->desc));
    }
    set_error("low-rank path: unknown flow");
    return DME_EINVAL;
}

void lr_free(dme_lr_t lr) {
    if (!lr) return;
    if (lr->st) cudaStreamSynchronize(lr->st);
    for (void* q : lr->allocs) cudaFree(q);
    if (lr->P) free_plan(lr->P);
    if (lr->own_st && lr->st) cudaStreamDestroy(lr->st);
    delete lr;
}

// Report and clear the device status word (synchronises the stream).
dme_status lr_check(dme_lr_t lr, const char* where) {
    if (lr->P) return plan_check(lr->P, where);
    int hs = 0;
    DME_CUDA_TRY(cudaMemcpyAsync(&hs, lr->status, sizeof(int), cudaMemcpyDeviceToHost, lr->st));
    DME_CUDA_TRY(cudaStreamSynchronize(lr->st));
    if (!hs) return DME_OK;
    DME_CUDA_TRY(cudaMemsetAsync(lr->status, 0, sizeof(int), lr->st));
    DME_CUDA_TRY(cudaStreamSynchronize(lr->st));
    if (hs & DEV_NOTSPD) return set_error(std::string(where) + ": R is not positive definite"), DME_ENOTSPD;
    if (hs & DEV_TIMEOUT) return set_error(std::string(where) + ": a bounded device wait ran out"), DME_ECUDA;
    return set_error(std::string(where) + ": device status " + std::to_string(hs)), DME_ECUDA;
}

template <typename F>
dme_status guarded(F&& f) {
    try {
        return f();
    } catch (const std::bad_alloc&) {
        set_error("host allocation failed");
        return DME_ENOMEM;
    } catch (...) {
        set_error("internal error");
        return DME_EINVAL;
    }
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

dme_status lr_opts(const dme_lr_opts* opts, int* q, int* rmax, double* tol) {
    *q = opts && opts->quad_nodes > 0 ? opts->quad_nodes : 7;
    *rmax = opts && opts->rmax > 0 ? opts->rmax : LR_MAX_RANK;
    *tol = opts && opts->tol > 0.0 ? opts->tol : 1e-13;
    if (*q > 64 || *rmax > LR_MAX_RANK || !(*tol < 1.0))
        return set_error("low-rank path: need quad_nodes <= 64, rmax <= 224, tol < 1"), DME_EINVAL;
    return DME_OK;
}

// Buffers shared by the dense and the sparse forms, and L_Q = C^T.
dme_status lr_setup(dme_lr_t lr, const dme_plan_desc* desc, const double* C, int q, int rmax, double tol) {
    lr->desc = *desc;
    lr->n = desc->n;
    lr->m = desc->m;
    lr->p = desc->p;
    lr->q = q;
    lr->rcap = rmax;
    lr->tol = tol;
    const size_t n = desc->n, rc = rmax, m = std::max(desc->m, 1);
    cudaStream_t st = lr->st;
    DME_TRY(lr_alloc(lr, &lr->L, n * rc));
    DME_TRY(lr_alloc(lr, &lr->L2, n * rc));
    DME_TRY(lr_alloc(lr, &lr->d, rc));
    DME_TRY(lr_alloc(lr, &lr->d2, rc));
    DME_TRY(lr_alloc(lr, &lr->LQ, n * desc->p));
    DME_TRY(lr_alloc(lr, &lr->G, rc * rc));
    DME_TRY(lr_alloc(lr, &lr->Vt, rc * rc));
    DME_TRY(lr_alloc(lr, &lr->lam, rc));
    DME_TRY(lr_alloc(lr, &lr->T, rc * rc));
    DME_TRY(lr_alloc(lr, &lr->J1, rc * rc));
    DME_TRY(lr_alloc(lr, &lr->J2, rc * rc));
    DME_TRY(lr_alloc(lr, &lr->J3, rc * rc));
    DME_TRY(lr_alloc(lr, &lr->J4, rc * rc));
    DME_TRY(lr_alloc(lr, &lr->Gm, rc * m));
    DME_TRY(lr_alloc(lr, &lr->H, m * m));
    DME_TRY(lr_alloc(lr, &lr->VtH, m * m));
    DME_TRY(lr_alloc(lr, &lr->lamH, m));
    DME_TRY(lr_alloc(lr, &lr->F, m * m));
    DME_TRY(lr_alloc(lr, &lr->Y, rc * m));
    DME_TRY(lr_alloc(lr, &lr->Z, n * m));
    lr->ws_doubles = std::max<size_t>((size_t)8 * rc * rc, (size_t)kSplitMax * rc * m);
    DME_TRY(lr_alloc(lr, &lr->ws, lr->ws_doubles));
    double* wd = nullptr;
    DME_TRY(lr_alloc(lr, &wd, (sizeof(GemmProb) * kSplitMax + 7) / 8));
    lr->wsdesc = reinterpret_cast<GemmProb*>(wd);
    lr->split = desc->prec == DME_SPLIT_BF16;
    if (lr->split) {
        DME_TRY(lr_alloc(lr, &lr->Xtr, rc * n));
        lr->xsl.rows = (int)rc;
        lr->xsl.k = (int)n;
        lr->xsl.Kp = slice_kpad((int)n);
        lr->xsl.ns = OZ_SLICES_STEP;
        lr->xsl.scheme = OZ_DIG9;
        double* xd = nullptr;
        DME_TRY(lr_alloc(lr, &xd, (slice_buf_bytes((int)rc, (int)n, OZ_SLICES_STEP) + 7) / 8));
        lr->xsl.data = reinterpret_cast<__nv_bfloat16*>(xd);
        double* xs = nullptr;
        DME_TRY(lr_alloc(lr, &xs, (rc + 1) / 2));
        lr->xsl.scale = reinterpret_cast<float*>(xs);
        DME_CUDA_TRY(cudaMemsetAsync(xd, 0, slice_buf_bytes((int)rc, (int)n, OZ_SLICES_STEP), st));
        DME_CUDA_TRY(cudaMemsetAsync(xs, 0, sizeof(float) * rc, st));
        DME_TRY(make_slice_tmaps(lr->xsl));
    }
    double* kd = nullptr;
    DME_TRY(lr_alloc(lr, &kd, 1));
    lr->kdev = reinterpret_cast<int*>(kd);
    double* Cd = nullptr;
    DME_TRY(lr_alloc(lr, &Cd, (size_t)desc->p * n));
    DME_CUDA_TRY(cudaMemcpyAsync(Cd, C, sizeof(double) * desc->p * n, cudaMemcpyDefault, st));
    launch_transpose(Cd, lr->LQ, desc->p, (int)n, (int)n, desc->p, st);
    DME_CUDA_TRY(cudaStreamSynchronize(st));
    return DME_OK;
}

}  // namespace

extern "C" {

dme_status dme_lr_plan(const dme_plan_desc* desc, const double* A, const double* C, const double* B, const double* R,
                       const double* S, const dme_lr_opts* opts, void* cuda_stream, dme_lr_t* out) {
    if (!out) return set_error("out is NULL"), DME_EINVAL;
    *out = nullptr;
    set_error("");
    if (!desc || !A || !C) return set_error("desc, A and C are required"), DME_EINVAL;
    if (!desc->q_is_factor) return set_error("low-rank path: give Q as its factor C (q_is_factor = 1)"), DME_EINVAL;
    if (desc->prec != DME_FP64 && desc->prec != DME_SPLIT_BF16)
        return set_error("low-rank path: prec must be DME_FP64 or DME_SPLIT_BF16 (DME_SPLIT_TF32 is not built)"),
               DME_EINVAL;
    if (desc->fsal || desc->extrap > 1) return set_error("low-rank path: no fsal / extrapolation"), DME_EINVAL;
    int q, rmax;
    double tol;
    DME_TRY(lr_opts(opts, &q, &rmax, &tol));
    if (desc->p > rmax) return set_error("low-rank path: p exceeds rmax"), DME_EINVAL;
    DME_TRY(plan_validate(desc, A, C, B, R, S));
    return guarded([&]() -> dme_status {
        std::unique_ptr<dme_lr_s, void (*)(dme_lr_t)> lr(new dme_lr_s(), lr_free);
        // the dense plan only supplies E_t, S and their slices: no slice-pair probe
        dme_plan_desc d2 = *desc;
        if (d2.prec == DME_SPLIT_BF16) d2.pairs = 14;
        DME_TRY(plan_create(&d2, A, C, B, R, S, cuda_stream, &lr->P));
        lr->st = lr->P->st;
        lr->status = lr->P->status;
        lr->Bt = lr->P->Bt;
        DME_TRY(lr_setup(lr.get(), desc, C, q, rmax, tol));
        DME_TRY(lr_check(lr.get(), "dme_lr_plan"));
        *out = lr.release();
        return DME_OK;
    });
}

dme_status dme_lr_plan_csr(const dme_plan_desc* desc, int nnz, const int* rowptr, const int* colidx,
                           const double* vals, const double* C, const double* B, const double* R, int nnz_s,
                           const int* s_rowptr, const int* s_colidx, const double* s_vals, const dme_lr_opts* opts,
                           void* cuda_stream, dme_lr_t* out) {
    if (!out) return set_error("out is NULL"), DME_EINVAL;
    *out = nullptr;
    set_error("");
    if (!desc || !rowptr || (nnz > 0 && (!colidx || !vals)) || !C)
        return set_error("desc, the CSR arrays and C are required"), DME_EINVAL;
    if (nnz < 0) return set_error("nnz must be >= 0"), DME_EINVAL;
    if (!desc->q_is_factor) return set_error("low-rank path: give Q as its factor C (q_is_factor = 1)"), DME_EINVAL;
    if (desc->prec != DME_FP64) return set_error("sparse low-rank path: prec must be DME_FP64"), DME_EINVAL;
    if (desc->fsal || desc->extrap > 1) return set_error("low-rank path: no fsal / extrapolation"), DME_EINVAL;
    const bool gen = desc->eq == DME_GDLE || desc->eq == DME_GDRE;
    if (gen && (!s_rowptr || nnz_s < 0 || (nnz_s > 0 && (!s_colidx || !s_vals))))
        return set_error("sparse low-rank path: generalised equations need S in CSR"), DME_EINVAL;
    if (desc->n < 1 || desc->nflows < 1 || desc->nflows > 4) return set_error("bad n or nflows"), DME_EINVAL;
    if (desc->comp != DME_LIE && desc->comp != DME_STRANG) return set_error("bad comp"), DME_EINVAL;
    if (!(desc->h > 0.0) || !std::isfinite(desc->h)) return set_error("h must be positive"), DME_EINVAL;
    const bool ric = desc->eq == DME_DRE || desc->eq == DME_GDRE;
    for (int i = 0; i < desc->nflows; ++i) {
        const int f = desc->flows[i];
        if (f < DME_F1 || f > DME_F4) return set_error("bad flow id"), DME_EINVAL;
        if (f == DME_F3 && !ric) return set_error("F3 needs eq = DRE or GDRE"), DME_EINVAL;
        if (f == DME_F4 && !gen) return set_error("F4 needs eq = GDLE or GDRE"), DME_EINVAL;
    }
    if (ric && (desc->m < 1 || desc->m > 32 || !B || !R)) return set_error("DRE needs B, R and 1 <= m <= 32"), DME_EINVAL;
    if (desc->p < 1) return set_error("p must be >= 1"), DME_EINVAL;
    int q, rmax;
    double tol;
    DME_TRY(lr_opts(opts, &q, &rmax, &tol));
    if (desc->p > rmax) return set_error("low-rank path: p exceeds rmax"), DME_EINVAL;
    return guarded([&]() -> dme_status {
        const int n = desc->n;
        // the CSR arrays on the host (they may be device pointers), checked
        std::vector<int> ptr(n + 1), idx(nnz);
        std::vector<double> val(nnz);
        DME_CUDA_TRY(cudaMemcpy(ptr.data(), rowptr, sizeof(int) * (n + 1), cudaMemcpyDefault));
        if (nnz) {
            DME_CUDA_TRY(cudaMemcpy(idx.data(), colidx, sizeof(int) * nnz, cudaMemcpyDefault));
            DME_CUDA_TRY(cudaMemcpy(val.data(), vals, sizeof(double) * nnz, cudaMemcpyDefault));
        }
        if (ptr[0] != 0 || ptr[n] != nnz) return set_error("CSR: rowptr[0] must be 0 and rowptr[n] = nnz"), DME_EINVAL;
        for (int i = 0; i < n; ++i)
            if (ptr[i + 1] < ptr[i]) return set_error("CSR: rowptr must be non-decreasing"), DME_EINVAL;
        for (int e = 0; e < nnz; ++e)
            if (idx[e] < 0 || idx[e] >= n) return set_error("CSR: column index out of range"), DME_EINVAL;
        // A^T in CSR (a counting sort by column)
        std::vector<int> tptr(n + 1, 0), tidx(nnz);
        std::vector<double> tval(nnz);
        for (int e = 0; e < nnz; ++e) tptr[idx[e] + 1]++;
        for (int i = 0; i < n; ++i) tptr[i + 1] += tptr[i];
        std::vector<int> fill(tptr.begin(), tptr.end() - 1);
        for (int i = 0; i < n; ++i)
            for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
                const int dst = fill[idx[e]]++;
                tidx[dst] = i;
                tval[dst] = val[e];
            }
        std::unique_ptr<dme_lr_s, void (*)(dme_lr_t)> lr(new dme_lr_s(), lr_free);
        lr->sparse = true;
        lr->nnz = nnz;
        // Gershgorin interval of A^T (rows of A^T): A^T = c I + g X, X's spectrum in [-2, 2]
        double a = 0.0, b = 0.0;
        for (int i = 0; i < n; ++i) {
            double di = 0.0, ri = 0.0;
            for (int e = tptr[i]; e < tptr[i + 1]; ++e) {
                if (tidx[e] == i) di += tval[e];
                else ri += std::fabs(tval[e]);
            }
            if (i == 0 || di - ri < a) a = di - ri;
            if (i == 0 || di + ri > b) b = di + ri;
        }
        lr->lc = 0.5 * (a + b);
        lr->lg = 0.25 * (b - a);
        lr->xi = leja_points_host(kLejaTerms);
        // the device copy of A^T holds A^T / g (the Leja recurrence's operator up to the shift)
        if (lr->lg > 0.0)
            for (double& v : tval) v /= lr->lg;
        if (cuda_stream) {
            lr->st = reinterpret_cast<cudaStream_t>(cuda_stream);
        } else {
            DME_CUDA_TRY(cudaStreamCreateWithFlags(&lr->st, cudaStreamNonBlocking));
            lr->own_st = true;
        }
        cudaStream_t st = lr->st;
        double* sd = nullptr;
        DME_TRY(lr_alloc(lr.get(), &sd, 1));
        lr->status = reinterpret_cast<int*>(sd);
        DME_CUDA_TRY(cudaMemsetAsync(lr->status, 0, sizeof(int), st));
        double *tp = nullptr, *ti = nullptr;
        DME_TRY(lr_alloc(lr.get(), &tp, ((size_t)n + 2) / 2));
        DME_TRY(lr_alloc(lr.get(), &ti, ((size_t)nnz + 1) / 2));
        DME_TRY(lr_alloc(lr.get(), &lr->at_val, (size_t)nnz));
        lr->at_ptr = reinterpret_cast<int*>(tp);
        lr->at_idx = reinterpret_cast<int*>(ti);
        DME_CUDA_TRY(cudaMemcpyAsync(lr->at_ptr, tptr.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st));
        if (nnz) {
            DME_CUDA_TRY(cudaMemcpyAsync(lr->at_idx, tidx.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice, st));
            DME_CUDA_TRY(cudaMemcpyAsync(lr->at_val, tval.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, st));
        }
        DME_CUDA_TRY(cudaStreamSynchronize(st));       // the host copies above go out of scope
        if (gen) {
            // S in CSR: checked on the host, then copied as given (T4 applies S, not S^T)
            std::vector<int> sp(n + 1), si(nnz_s);
            std::vector<double> sv(nnz_s);
            DME_CUDA_TRY(cudaMemcpy(sp.data(), s_rowptr, sizeof(int) * (n + 1), cudaMemcpyDefault));
            if (nnz_s) {
                DME_CUDA_TRY(cudaMemcpy(si.data(), s_colidx, sizeof(int) * nnz_s, cudaMemcpyDefault));
                DME_CUDA_TRY(cudaMemcpy(sv.data(), s_vals, sizeof(double) * nnz_s, cudaMemcpyDefault));
            }
            if (sp[0] != 0 || sp[n] != nnz_s) return set_error("CSR of S: rowptr[0] must be 0, rowptr[n] = nnz"), DME_EINVAL;
            for (int i = 0; i < n; ++i)
                if (sp[i + 1] < sp[i]) return set_error("CSR of S: rowptr must be non-decreasing"), DME_EINVAL;
            for (int e = 0; e < nnz_s; ++e)
                if (si[e] < 0 || si[e] >= n) return set_error("CSR of S: column index out of range"), DME_EINVAL;
            double *p1 = nullptr, *p2 = nullptr;
            DME_TRY(lr_alloc(lr.get(), &p1, ((size_t)n + 2) / 2));
            DME_TRY(lr_alloc(lr.get(), &p2, ((size_t)nnz_s + 1) / 2));
            DME_TRY(lr_alloc(lr.get(), &lr->s_val, (size_t)nnz_s));
            lr->s_ptr = reinterpret_cast<int*>(p1);
            lr->s_idx = reinterpret_cast<int*>(p2);
            DME_CUDA_TRY(cudaMemcpyAsync(lr->s_ptr, sp.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st));
            if (nnz_s) {
                DME_CUDA_TRY(cudaMemcpyAsync(lr->s_idx, si.data(), sizeof(int) * nnz_s, cudaMemcpyHostToDevice, st));
                DME_CUDA_TRY(cudaMemcpyAsync(lr->s_val, sv.data(), sizeof(double) * nnz_s, cudaMemcpyHostToDevice, st));
            }
            DME_CUDA_TRY(cudaStreamSynchronize(st));
        }
        if (ric) {
            const int m = desc->m;
            double *Bd = nullptr, *Rd = nullptr, *Btd = nullptr;
            DME_TRY(lr_alloc(lr.get(), &Bd, (size_t)n * m));
            DME_TRY(lr_alloc(lr.get(), &Rd, (size_t)m * m));
            DME_TRY(lr_alloc(lr.get(), &Btd, (size_t)n * m));
            DME_CUDA_TRY(cudaMemcpyAsync(Bd, B, sizeof(double) * n * m, cudaMemcpyDefault, st));
            DME_CUDA_TRY(cudaMemcpyAsync(Rd, R, sizeof(double) * m * m, cudaMemcpyDefault, st));
            launch_small_cholesky(Rd, m, lr->status, st);
            launch_apply_linv_rows(Bd, Rd, Btd, n, m, st);
            lr->Bt = Btd;
            DME_TRY(lr_check(lr.get(), "dme_lr_plan_csr (Cholesky of R)"));
        }
        DME_TRY(lr_setup(lr.get(), desc, C, q, rmax, tol));
        const size_t rc = rmax;
        DME_TRY(lr_alloc(lr.get(), &lr->Wa, (size_t)n * rc));
        DME_TRY(lr_alloc(lr.get(), &lr->Wb, (size_t)n * rc));
        DME_TRY(lr_alloc(lr.get(), &lr->lpart, 4 * (size_t)leja_grid_max()));
        DME_TRY(lr_alloc(lr.get(), &lr->lnorm, 8));   // 4 sums, then the barrier words
        DME_TRY(lr_check(lr.get(), "dme_lr_plan_csr"));
        *out = lr.release();
        return DME_OK;
    });
}

dme_status dme_lr_solve(dme_lr_t lr, const double* L0, const double* D0, int r0, double T, int nsteps, double* P_out,
                        int* r_out) {
    if (!lr) return set_error("plan is NULL"), DME_EINVAL;
    if (nsteps < 1 || !(T > 0.0) || !std::isfinite(T)) return set_error("need nsteps >= 1 and T > 0"), DME_EINVAL;
    if (r0 < 0 || r0 > lr->rcap || (r0 > 0 && (!L0 || !D0)))
        return set_error("need 0 <= r0 <= rmax and L0, D0 when r0 > 0"), DME_EINVAL;
    return guarded([&]() -> dme_status {
        cudaStream_t st = lr->st;
        const int n = lr->n, rc = lr->rcap;
        lr->r = 0;
        if (r0 > 0) {
            // P0 = L0 D0 L0^T with D0 symmetric: L0 V, d = eigenvalues (> 0), then compress
            DME_CUDA_TRY(cudaMemcpy2DAsync(lr->L2, sizeof(double) * rc, L0, sizeof(double) * r0, sizeof(double) * r0, n,
                                           cudaMemcpyDefault, st));
            DME_CUDA_TRY(cudaMemcpy2DAsync(lr->G, sizeof(double) * rc, D0, sizeof(double) * r0, sizeof(double) * r0, r0,
                                           cudaMemcpyDefault, st));
            DME_TRY(launch_jacobi_eig(lr->G, rc, r0, lr->Vt, rc, lr->lam, lr->status, st));
            launch_lr_select(lr->lam, lr->Vt, rc, r0, 0.0, 0, lr->T, rc, lr->d, lr->kdev, st);
            int k = 0;
            DME_CUDA_TRY(cudaMemcpyAsync(&k, lr->kdev, sizeof(int), cudaMemcpyDeviceToHost, st));
            DME_CUDA_TRY(cudaStreamSynchronize(st));
            DME_TRY(gemm(lr, mk(n, k, r0, lr->L2, rc, 0, lr->T, rc, 0, lr->L, rc, 1.0), st));
            lr->r = k;
            DME_TRY(compress(lr, lr->L, lr->L2, lr->d, rc, lr->r));
        }
        const double h = T / nsteps;
        const auto seq = plan_step_sequence(lr->desc, h);
        for (int s = 0; s < nsteps; ++s)
            for (auto& ft : seq) DME_TRY(lr_apply(lr, ft.first, ft.second));
        if (P_out && n > 16384) return set_error("dme_lr_solve: P_out needs n <= 16384 (use dme_lr_factors)"), DME_EINVAL;
        if (P_out) {
            const size_t nn = (size_t)n * n;
            if (!lr->Pout) DME_TRY(lr_alloc(lr, &lr->Pout, nn));
            if (lr->r > 0) {
                launch_copy_cols(lr->L2, rc, lr->L, rc, n, lr->r, 1.0, lr->d, st);
                DME_TRY(gemm(lr, mk(n, n, lr->r, lr->L2, rc, 0, lr->L2, rc, 1, lr->Pout, n, 1.0, 1), st));
            } else {
                DME_CUDA_TRY(cudaMemsetAsync(lr->Pout, 0, nn * sizeof(double), st));
            }
            DME_CUDA_TRY(cudaMemcpyAsync(P_out, lr->Pout, nn * sizeof(double), cudaMemcpyDefault, st));
        }
        if (r_out) *r_out = lr->r;
        return lr_check(lr, "dme_lr_solve");
    });
}

dme_status dme_lr_factors(dme_lr_t lr, double* L_out, double* d_out, int* r) {
    if (!lr || !r) return set_error("plan and r are required"), DME_EINVAL;
    return guarded([&]() -> dme_status {
        cudaStream_t st = lr->st;
        *r = lr->r;
        if (lr->r > 0 && L_out)
            DME_CUDA_TRY(cudaMemcpy2DAsync(L_out, sizeof(double) * lr->r, lr->L, sizeof(double) * lr->rcap,
                                           sizeof(double) * lr->r, lr->n, cudaMemcpyDefault, st));
        if (lr->r > 0 && d_out)
            DME_CUDA_TRY(cudaMemcpyAsync(d_out, lr->d, sizeof(double) * lr->r, cudaMemcpyDefault, st));
        DME_CUDA_TRY(cudaStreamSynchronize(st));
        return DME_OK;
    });
}

dme_status dme_lr_destroy(dme_lr_t lr) {
    lr_free(lr);
    return DME_OK;
}

}  // extern "C"
