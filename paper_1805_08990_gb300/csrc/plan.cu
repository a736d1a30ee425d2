// Plan, exponential, stepping and the C ABI of libdme.
//
// A plan holds the problem on the device and, per step length t used by T1 or
// T12, the pair (E_t, W_t) of Eq. full:  E_t = e^{tA},
// W_t = int_0^t e^{sA^T} Q e^{sA} ds.  Both come from the Van Loan block
// exponential e^{t M}, M = [[-A^T, Q], [0, A]] (F22 = E_t, F22^T F12 = W_t),
// evaluated with Higham's [13/13] Pade approximant and scaling and squaring.
// Everything is done on n x n blocks, never on the 2n x 2n matrix:
//  * every polynomial in the block upper-triangular X = M/2^s is block upper
//    triangular, and its (1,1) block is determined by its (2,2) block
//    (X11 = -X22^T, so an even power has (1,1) = (2,2)^T and an odd one
//    (1,1) = -(2,2)^T); a product therefore costs three n x n GEMMs;
//  * the Pade denominator q = V - U has q11 = p22^T, so q R = p splits into
//    R22 = q22^{-1} p22 and R12 = p22^{-T} (p12 - q12 R22): two n x n LU
//    solves in FP64;
//  * squaring the block matrix is the semigroup law of T12 (Eq. full):
//    E_{2t} = E_t^2, W_{2t} = W_t + E_t^T W_t E_t.
#include "plan_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

namespace dme {

static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }
const char* get_error() { return g_err.c_str(); }

// theta_13 (Higham 2005): largest ||X||_1 for which the [13/13] approximant
// meets unit-roundoff backward error in double precision.
static const double kTheta13 = 5.371920351148152;

// c_0 = 1, c_{j+1} = c_j (m - j) / ((2m - j)(j + 1)), m = 13: the numerator
// coefficients of the [m/m] Pade approximant of e^x.
static void pade13(double c[14]) {
    c[0] = 1.0;
    for (int j = 0; j < 13; ++j) c[j + 1] = c[j] * (13.0 - j) / ((26.0 - j) * (j + 1.0));
}

}  // namespace dme

using namespace dme;

namespace {

dme_status palloc(dme_plan_t p, void** out, size_t bytes) {
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(out, bytes, p->st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
        return DME_ENOMEM;
    }
    p->allocs.push_back(*out);
    p->bytes += bytes;
    return DME_OK;
}

template <typename T>
dme_status palloc_t(dme_plan_t p, T** out, size_t count) {
    return palloc(p, reinterpret_cast<void**>(out), count * sizeof(T));
}

// Temporary device buffers released at scope exit (plan-time only), stream ordered.
struct TmpPool {
    cudaStream_t st;
    std::vector<void*> v;
    explicit TmpPool(cudaStream_t s) : st(s) {}
    ~TmpPool() {
        for (void* q : v) cudaFreeAsync(q, st);
    }
    dme_status get(double** out, size_t count) {
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(out), std::max<size_t>(count, 2) * sizeof(double), st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error(std::string("cudaMalloc (temporary): ") + cudaGetErrorString(e));
            return DME_ENOMEM;
        }
        v.push_back(*out);
        return DME_OK;
    }
};

GemmProb gp(int M, int N, int K, const double* A, int lda, int tA, const double* B, int ldb, int tB, double* C,
            int ldc, double alpha, int tri = 0, const double* D1 = nullptr, double b1 = 0.0,
            const double* D2 = nullptr, double b2 = 0.0, const double* D3 = nullptr, double b3 = 0.0) {
    GemmProb g;
    std::memset(&g, 0, sizeof(g));
    g.A = A;
    g.B = B;
    g.C = C;
    g.D1 = D1;
    g.D2 = D2;
    g.D3 = D3;
    g.M = M;
    g.N = N;
    g.K = K;
    g.lda = lda;
    g.ldb = ldb;
    g.ldc = ldc;
    g.ldd = ldc;
    g.alpha = alpha;
    g.b1 = b1;
    g.b2 = b2;
    g.b3 = b3;
    g.transA = tA;
    g.transB = tB;
    g.tri = tri;
    return g;
}

// One FP64 product; 32-wide output tiles when 64-wide ones would not fill one
// wave of the SMs (both tile shapes give bit-identical results).
dme_status gemm1(const GemmProb& g, cudaStream_t st) {
    std::vector<GemmProb> v{g};
    long tiles64 = (long)((g.M + 63) / 64) * ((g.N + 63) / 64);
    if (g.tri) tiles64 = (tiles64 + (g.M + 63) / 64) / 2;
    return gemm64_grouped(v, nullptr, st, nullptr, tiles64 < 152 ? 32 : 64);
}

// out = G^T P G + addends, symmetric, with G = E (so out = E^T P E); X is n x n work.
dme_status cong64(int n, const double* P, const double* E, double* X, double* out, const double* D1, double b1,
                  const double* D2, double b2, const double* D3, double b3, cudaStream_t st) {
    DME_TRY(gemm1(gp(n, n, n, P, n, 0, E, n, 0, X, n, 1.0), st));                       // X = P E
    DME_TRY(gemm1(gp(n, n, n, E, n, 1, X, n, 0, out, n, 1.0, 1, D1, b1, D2, b2, D3, b3), st));  // E^T X
    return DME_OK;
}

dme_status check_status(dme_plan_t p, const char* where) {
    DME_CUDA_TRY(cudaStreamSynchronize(p->st));
    int hs = 0;
    DME_CUDA_TRY(cudaMemcpyAsync(&hs, p->status, sizeof(int), cudaMemcpyDeviceToHost, p->st));
    DME_CUDA_TRY(cudaStreamSynchronize(p->st));
    if (hs) {
        DME_CUDA_TRY(cudaMemsetAsync(p->status, 0, sizeof(int), p->st));
        DME_CUDA_TRY(cudaStreamSynchronize(p->st));
        if (hs & DEV_NOTSPD) {
            set_error(std::string(where) + ": I_m + t Bt^T P Bt (or R) is not positive definite");
            return DME_ENOTSPD;
        }
        if (hs & DEV_SINGULAR) {
            set_error(std::string(where) + ": singular Pade denominator");
            return DME_ECUDA;
        }
        set_error(std::string(where) + ": device status " + std::to_string(hs));
        return DME_ECUDA;
    }
    return DME_OK;
}

// Products of the plan-time exponential on split plans with n >= kAccMinN: the
// accurate tensor-core mode (six 7-bit slices per operand, exact K chunks of
// 512 combined in fp64).  A product C = alpha op(L) op(R) + b1 D1 slices the rows
// of op(L) and the rows of op(R)^T, transposing first where needed.
constexpr int kAccMinN = 512;

struct AccWork {
    SliceBuf a, b;          // slices of the A operand (rows of op(L)) and B operand (rows of op(R)^T)
    double* t = nullptr;    // transpose scratch (n x n)
    double* wsd = nullptr;  // chunk workspace
    int* status = nullptr;
};

dme_status acc_prod(int n, AccWork& w, const double* L, int tL, const double* R, int tR, double* C, double alpha,
                    const double* D1, double b1, cudaStream_t st) {
    if (tL) {
        launch_transpose(L, w.t, n, n, n, n, st);
        launch_slice_rows_f64(w.t, n, n, n, w.a, st);
    } else {
        launch_slice_rows_f64(L, n, n, n, w.a, st);
    }
    if (tR) {
        launch_slice_rows_f64(R, n, n, n, w.b, st);
    } else {
        launch_transpose(R, w.t, n, n, n, n, st);
        launch_slice_rows_f64(w.t, n, n, n, w.b, st);
    }
    OzParams o;
    DME_TRY(oz_params(w.a, w.b, OZ_A21, &o));
    o.mode = OZ_OUT_F64;
    o.ldc = n;
    o.Cd = C;
    o.alpha = alpha;
    o.D1 = D1;
    o.b1 = b1;
    o.wsd = w.wsd;
    o.status = w.status;
    return launch_ozaki_gemm(oz_tmap_a(w.a, OZ_A21), oz_tmap_b(w.b, OZ_A21), o, st);
}

// Scratch of the accurate mode for n x n products, from a plan-time pool.
dme_status acc_setup(TmpPool& tp, int n, int* status, AccWork* w) {
    const size_t nn = (size_t)n * n;
    double *ad, *bd, *sc;
    const size_t sl = (slice_buf_bytes(n, n, OZ_SLICES_ACC) + 7) / 8;
    DME_TRY(tp.get(&ad, sl));
    DME_TRY(tp.get(&bd, sl));
    DME_TRY(tp.get(&sc, (size_t)n));
    DME_TRY(tp.get(&w->t, nn));
    DME_TRY(tp.get(&w->wsd, oz_acc_ws_doubles(n, n, n)));
    for (SliceBuf* b : {&w->a, &w->b}) {
        b->rows = n;
        b->k = n;
        b->Kp = slice_kpad(n);
        b->ns = OZ_SLICES_ACC;
        b->scheme = OZ_DIG7;
    }
    w->a.data = reinterpret_cast<__nv_bfloat16*>(ad);
    w->b.data = reinterpret_cast<__nv_bfloat16*>(bd);
    w->a.scale = reinterpret_cast<float*>(sc);
    w->b.scale = reinterpret_cast<float*>(sc) + n;
    DME_TRY(make_slice_tmaps(w->a));
    DME_TRY(make_slice_tmaps(w->b));
    w->status = status;
    return DME_OK;
}

// C = alpha op(L) op(R) + b1 D1 (n x n): the accurate tensor mode with aw, else FP64.
dme_status prod(int n, AccWork* aw, const double* L, int tL, const double* R, int tR, double* C, double alpha,
                const double* D1, double b1, cudaStream_t st, double* skw = nullptr, size_t skl = 0) {
    if (aw) return acc_prod(n, *aw, L, tL, R, tR, C, alpha, D1, b1, st);
    return gemm64_splitk(gp(n, n, n, L, n, tL, R, n, tR, C, n, alpha, 0, D1, b1), skw, skl, st);
}

// (O22, O12) = (L, L11 = ls L22^T) * (R):  O22 = L22 R22, O12 = ls L22^T R12 + L12 R22.
dme_status bprod(int n, AccWork* aw, const double* L22, const double* L12, double ls, const double* R22,
                 const double* R12, double* O22, double* O12, cudaStream_t st, double* skw = nullptr,
                 size_t skl = 0) {
    DME_TRY(prod(n, aw, L22, 0, R22, 0, O22, 1.0, nullptr, 0.0, st, skw, skl));
    DME_TRY(prod(n, aw, L22, 1, R12, 0, O12, ls, nullptr, 0.0, st, skw, skl));
    DME_TRY(prod(n, aw, L12, 0, R22, 0, O12, 1.0, O12, 1.0, st, skw, skl));
    return DME_OK;
}

cudaEvent_t ev_get(dme_plan_t p) {
    if (!p->evpool.empty()) {
        cudaEvent_t e = p->evpool.back();
        p->evpool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Bracket the launches of one kernel kind with events (profiling mode only).
struct ProfScope {
    dme_plan_t p;
    int kind;
    cudaEvent_t a = nullptr;
    ProfScope(dme_plan_t p_, int kind_) : p(p_), kind(kind_) {
        if (!p->prof) return;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(p->st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
        a = ev_get(p);
        cudaEventRecord(a, p->st);
    }
    ~ProfScope() {
        if (!a) return;
        cudaEvent_t b = ev_get(p);
        cudaEventRecord(b, p->st);
        p->evrec.push_back({kind, a, b});
    }
};

dme_status alloc_slices(dme_plan_t p, SliceBuf* sb, int rows, int k, int ns, int scheme = OZ_DIG9) {
    sb->rows = rows;
    sb->k = k;
    sb->Kp = slice_kpad(k);
    sb->ns = ns;
    sb->scheme = scheme;
    DME_TRY(palloc(p, reinterpret_cast<void**>(&sb->data), slice_buf_bytes(rows, k, ns)));
    DME_TRY(palloc_t(p, &sb->scale, (size_t)rows));
    return make_slice_tmaps(*sb);
}

// out = alpha G P G^T + b1 D1 + b2 D2 + b3 D3 on the split-precision path (P
// symmetric, G given by its row slices; the addends symmetric).  U = G P
// (P^T = P), then G U^T, both with slice-pair configuration cfg.
dme_status split_cong(dme_plan_t p, const double* P, const SliceBuf& G, double* out, double alpha, const double* D1,
                      double b1, const double* D2, double b2, const double* D3, double b3, int cfg) {
    const int n = p->n;
    cudaStream_t st = p->st;
    {
        ProfScope ps(p, DME_KIND_SLICE);
        launch_slice_rows_f64(P, n, n, n, p->psl, st);
    }
    OzParams a;
    DME_TRY(oz_params(G, p->psl, cfg, &a));
    a.mode = OZ_OUT_PAIR;
    a.ldc = n;
    a.Cp = p->U;
    a.status = p->status;
    a.ws = p->kws;
    a.ws_cnt = p->kcnt;
    {
        ProfScope ps(p, DME_KIND_SPLIT_GEMM);
        DME_TRY(launch_ozaki_gemm(oz_tmap_a(G, cfg), oz_tmap_b(p->psl, cfg), a, st));
    }
    {
        ProfScope ps(p, DME_KIND_SLICE);
        launch_slice_rows_pair(p->U, n, n, n, p->usl, st);
    }
    OzParams b;
    DME_TRY(oz_params(G, p->usl, cfg, &b));
    b.mode = OZ_OUT_F64;
    b.tri = 1;
    b.ldc = n;
    b.Cd = out;
    b.alpha = alpha;
    b.D1 = D1;
    b.b1 = b1;
    b.D2 = D2;
    b.b2 = b2;
    b.D3 = D3;
    b.b3 = b3;
    b.status = p->status;
    b.ws = p->kws;
    b.ws_cnt = p->kcnt;
    ProfScope ps(p, DME_KIND_SPLIT_GEMM);
    return launch_ozaki_gemm(oz_tmap_a(G, cfg), oz_tmap_b(p->usl, cfg), b, st);
}

// T3 on the split path for n > 1536: Z^T = Bt^T P (P symmetric) on the tensor
// cores (Bt^T with 5 slices as the fixed operand, P with 4), then the m x m
// part in FP64 (Gram partials, M = I + t Bt^T Z, Cholesky, Y = Z L^{-T}), then
// P <- P - t Y Y^T (+ q Q) as a triangle tensor GEMM with K = m and the FP64
// epilogue adding P.  Same formula as launch_riccati, other rounding.
dme_status split_riccati(dme_plan_t p, double* P, double tau, double qcoef) {
    const int n = p->n, m = p->m;
    cudaStream_t st = p->st;
    double* Z = p->rwork;
    double* Y = Z + (size_t)n * m;
    launch_slice_rows_f64(P, n, n, n, p->psl, st);
    OzParams a;
    DME_TRY(oz_params(p->btsl, p->psl, p->cfg, &a));
    a.mode = OZ_OUT_F64;
    a.ldc = n;
    a.Cd = p->Zt;
    a.alpha = 1.0;
    a.status = p->status;
    a.ws = p->kws;
    a.ws_cnt = p->kcnt;
    DME_TRY(launch_ozaki_gemm(oz_tmap_a(p->btsl, p->cfg), oz_tmap_b(p->psl, p->cfg), a, st));
    launch_transpose(p->Zt, Z, m, n, n, m, st);
    DME_TRY(launch_riccati_from_z(p->Bt, n, m, tau, p->rwork, p->status, st));
    launch_slice_rows_f64(Y, n, m, m, p->ysla, st);
    launch_slice_rows_f64(Y, n, m, m, p->yslb, st);
    OzParams b;
    DME_TRY(oz_params(p->ysla, p->yslb, p->cfg, &b));
    b.mode = OZ_OUT_F64;
    b.tri = 1;
    b.ldc = n;
    b.Cd = P;
    b.alpha = -tau;
    b.D1 = P;
    b.b1 = 1.0;
    if (qcoef != 0.0) {
        b.D2 = p->Q;
        b.b2 = qcoef;
    }
    b.status = p->status;
    return launch_ozaki_gemm(oz_tmap_a(p->ysla, p->cfg), oz_tmap_b(p->yslb, p->cfg), b, st);
}

dme_status compute_ew(dme_plan_t p, double tau, int* idx) {
    for (size_t i = 0; i < p->ew.size(); ++i)
        if (p->ew[i].tau == tau) {
            *idx = (int)i;
            return DME_OK;
        }
    const int n = p->n;
    const size_t nn = (size_t)n * n;
    cudaStream_t st = p->st;
    double c[14];
    pade13(c);
    const double nrm = std::fabs(tau) * p->normM;
    int s = 0;
    if (nrm > kTheta13) s = (int)std::ceil(std::log2(nrm / kTheta13));
    const double sc = std::ldexp(tau, -s);

    TmpPool tp(st);
    double *X22, *X12, *A22, *A12, *B22, *B12, *C22, *C12, *Y22, *Y12, *T22, *T12, *U22, *U12, *V22, *V12;
    double *LUq, *LUp, *R22, *R12;
    DME_TRY(tp.get(&X22, nn));
    DME_TRY(tp.get(&X12, nn));
    DME_TRY(tp.get(&A22, nn));
    DME_TRY(tp.get(&A12, nn));
    DME_TRY(tp.get(&B22, nn));
    DME_TRY(tp.get(&B12, nn));
    DME_TRY(tp.get(&C22, nn));
    DME_TRY(tp.get(&C12, nn));
    DME_TRY(tp.get(&Y22, nn));
    DME_TRY(tp.get(&Y12, nn));
    DME_TRY(tp.get(&T22, nn));
    DME_TRY(tp.get(&T12, nn));
    DME_TRY(tp.get(&U22, nn));
    DME_TRY(tp.get(&U12, nn));
    DME_TRY(tp.get(&V22, nn));
    DME_TRY(tp.get(&V12, nn));
    double* gjw = nullptr;
    DME_TRY(tp.get(&gjw, gj_work_doubles(n, n)));
    // split-K partial sums of the small FP64 products (n <= 288: fewer 32-wide tiles than half the SMs)
    double* skw = nullptr;
    size_t skl = 0;
    if (n <= 288) {
        skl = gemm64_splitk_ws_doubles(n, n);
        DME_TRY(tp.get(&skw, skl));
    }
    // split plans of n >= kAccMinN: the Pade products on the tensor cores (accurate mode)
    AccWork accw;
    AccWork* aw = nullptr;
    if (p->split && n >= kAccMinN) {
        DME_TRY(acc_setup(tp, n, p->status, &accw));
        aw = &accw;
    }

    // X = sc M:  X22 = sc A, X12 = sc Q, X11 = -X22^T (implicit)
    launch_lincomb(X22, n, n, p->A, sc, nullptr, 0, nullptr, 0, 0.0, st);
    launch_lincomb(X12, n, n, p->Q, sc, nullptr, 0, nullptr, 0, 0.0, st);
    // X2 = X X (odd * odd -> even), X4 = X2 X2, X6 = X4 X2
    DME_TRY(bprod(n, aw, X22, X12, -1.0, X22, X12, A22, A12, st, skw, skl));
    DME_TRY(bprod(n, aw, A22, A12, 1.0, A22, A12, B22, B12, st, skw, skl));
    DME_TRY(bprod(n, aw, B22, B12, 1.0, A22, A12, C22, C12, st, skw, skl));
    // odd part: U = X (X6 (c13 X6 + c11 X4 + c9 X2) + c7 X6 + c5 X4 + c3 X2 + c1 I)
    launch_lincomb(Y22, n, n, C22, c[13], B22, c[11], A22, c[9], 0.0, st);
    launch_lincomb(Y12, n, n, C12, c[13], B12, c[11], A12, c[9], 0.0, st);
    DME_TRY(bprod(n, aw, C22, C12, 1.0, Y22, Y12, T22, T12, st, skw, skl));
    launch_lincomb(U22, n, n, C22, c[7], B22, c[5], A22, c[3], c[1], st);
    launch_lincomb(U12, n, n, C12, c[7], B12, c[5], A12, c[3], 0.0, st);
    launch_lincomb(T22, n, n, T22, 1.0, U22, 1.0, nullptr, 0, 0.0, st);
    launch_lincomb(T12, n, n, T12, 1.0, U12, 1.0, nullptr, 0, 0.0, st);
    DME_TRY(bprod(n, aw, X22, X12, -1.0, T22, T12, U22, U12, st, skw, skl));
    // even part: V = X6 (c12 X6 + c10 X4 + c8 X2) + c6 X6 + c4 X4 + c2 X2 + c0 I
    launch_lincomb(Y22, n, n, C22, c[12], B22, c[10], A22, c[8], 0.0, st);
    launch_lincomb(Y12, n, n, C12, c[12], B12, c[10], A12, c[8], 0.0, st);
    DME_TRY(bprod(n, aw, C22, C12, 1.0, Y22, Y12, V22, V12, st, skw, skl));
    launch_lincomb(T22, n, n, C22, c[6], B22, c[4], A22, c[2], c[0], st);
    launch_lincomb(T12, n, n, C12, c[6], B12, c[4], A12, c[2], 0.0, st);
    launch_lincomb(V22, n, n, V22, 1.0, T22, 1.0, nullptr, 0, 0.0, st);
    launch_lincomb(V12, n, n, V12, 1.0, T12, 1.0, nullptr, 0, 0.0, st);
    // p = V + U, q = V - U (reuse X, A, B buffers)
    double* p22 = X22;
    double* p12 = X12;
    double* q22 = A22;
    double* q12 = A12;
    launch_lincomb(p22, n, n, V22, 1.0, U22, 1.0, nullptr, 0, 0.0, st);
    launch_lincomb(p12, n, n, V12, 1.0, U12, 1.0, nullptr, 0, 0.0, st);
    launch_lincomb(q22, n, n, V22, 1.0, U22, -1.0, nullptr, 0, 0.0, st);
    launch_lincomb(q12, n, n, V12, 1.0, U12, -1.0, nullptr, 0, 0.0, st);
    // R22 = q22^{-1} p22 (Gauss-Jordan with partial pivoting on a copy of q22)
    LUq = B22;
    R22 = B12;
    launch_lincomb(LUq, n, n, q22, 1.0, nullptr, 0, nullptr, 0, 0.0, st);
    launch_lincomb(R22, n, n, p22, 1.0, nullptr, 0, nullptr, 0, 0.0, st);
    DME_TRY(launch_gj_solve(LUq, n, n, R22, n, n, gjw, p->status, st));
    // R12 = p22^{-T} (p12 - q12 R22)
    R12 = C12;
    DME_TRY(prod(n, aw, q12, 0, R22, 0, R12, -1.0, p12, 1.0, st, skw, skl));
    LUp = C22;
    launch_transpose(p22, LUp, n, n, n, n, st);
    DME_TRY(launch_gj_solve(LUp, n, n, R12, n, n, gjw, p->status, st));
    // E = R22, W = R22^T R12 (symmetrised), then s doublings
    double* E = Y22;
    double* Wm = Y12;
    double* tmp = T22;
    double* E2 = T12;
    launch_lincomb(E, n, n, R22, 1.0, nullptr, 0, nullptr, 0, 0.0, st);
    DME_TRY(prod(n, aw, R22, 1, R12, 0, Wm, 1.0, nullptr, 0.0, st, skw, skl));
    launch_symmetrize(Wm, n, n, st);
    for (int i = 0; i < s; ++i) {
        DME_TRY(gemm64_splitk(gp(n, n, n, Wm, n, 0, E, n, 0, tmp, n, 1.0), skw, skl, st));   // tmp = W E
        DME_TRY(gemm64_splitk(gp(n, n, n, E, n, 1, tmp, n, 0, Wm, n, 1.0, 1, Wm, 1.0), skw, skl, st));   // W = E^T tmp + W
        DME_TRY(gemm64_splitk(gp(n, n, n, E, n, 0, E, n, 0, E2, n, 1.0), skw, skl, st));     // E2 = E E
        std::swap(E, E2);
    }
    EWEntry ent;
    ent.tau = tau;
    ent.s = s;
    DME_TRY(palloc_t(p, &ent.E, nn));
    DME_TRY(palloc_t(p, &ent.W, nn));
    DME_CUDA_TRY(cudaMemcpyAsync(ent.E, E, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
    DME_CUDA_TRY(cudaMemcpyAsync(ent.W, Wm, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (p->split) {
        launch_transpose(ent.E, tmp, n, n, n, n, st);          // tmp = E^T
        DME_TRY(alloc_slices(p, &ent.Gsl, n, n, OZ_SLICES_FIXED));
        launch_slice_rows_f64(tmp, n, n, n, ent.Gsl, st);
    }
    DME_CUDA_TRY(cudaGetLastError());
    DME_TRY(check_status(p, "dme_expm"));
    p->ew.push_back(ent);
    *idx = (int)p->ew.size() - 1;
    return DME_OK;
}

// Sums of (a - b)^2 and b^2 over len entries: per-block partials (fixed order),
// then one block adds them in order, so the result does not depend on timing.
__global__ void __launch_bounds__(256) diff_norms_partial_kernel(const double* __restrict__ a,
                                                                 const double* __restrict__ b, size_t len,
                                                                 double* __restrict__ part) {
    __shared__ double sd[256], sr[256];
    double d = 0.0, r = 0.0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (size_t)gridDim.x * blockDim.x) {
        const double x = a[e] - b[e];
        d += x * x;
        r += b[e] * b[e];
    }
    sd[threadIdx.x] = d;
    sr[threadIdx.x] = r;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sd[threadIdx.x] += sd[threadIdx.x + w];
            sr[threadIdx.x] += sr[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sd[0];
        part[2 * blockIdx.x + 1] = sr[0];
    }
}

__global__ void diff_norms_final_kernel(const double* __restrict__ part, int nb, double* __restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double d = 0.0, r = 0.0;
    for (int k = 0; k < nb; ++k) {
        d += part[2 * k];
        r += part[2 * k + 1];
    }
    out[0] = d;
    out[1] = r;
}

// ||a - b||_F / ||b||_F of two n x n device matrices (synchronises st).
dme_status rel_diff(const double* a, const double* b, size_t len, double* work, cudaStream_t st, double* out) {
    constexpr int nb = 256;
    diff_norms_partial_kernel<<<nb, 256, 0, st>>>(a, b, len, work);
    diff_norms_final_kernel<<<1, 32, 0, st>>>(work, nb, work + 2 * nb);
    double h[2] = {0.0, 0.0};
    DME_CUDA_TRY(cudaMemcpyAsync(h, work + 2 * nb, sizeof(h), cudaMemcpyDeviceToHost, st));
    DME_CUDA_TRY(cudaStreamSynchronize(st));
    *out = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
    return DME_OK;
}

int cfg_of_pairs(int pairs) { return pairs == 10 ? OZ_P10 : (pairs == 13 ? OZ_P13 : OZ_P14); }

__global__ void fill_kernel(double* x, int n, double v) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = v;
}

// y = M x (M n x n row-major): a warp per row.
__global__ void __launch_bounds__(256) gemv_rows_kernel(const double* __restrict__ M, const double* __restrict__ x,
                                                        int n, double* __restrict__ y) {
    const int lane = threadIdx.x & 31;
    for (int r = blockIdx.x * 8 + (threadIdx.x >> 5); r < n; r += gridDim.x * 8) {
        double a = 0.0;
        for (int k = lane; k < n; k += 32) a += M[(size_t)r * n + k] * x[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
        if (lane == 0) y[r] = a;
    }
}

// One block: rq[0] = x . z (the Rayleigh quotient of M^T M at the unit x), then
// x = z / ||z|| (fixed-order reductions; x left unchanged if z = 0).
__global__ void __launch_bounds__(1024) rayleigh_normalize_kernel(double* __restrict__ x,
                                                                  const double* __restrict__ z, int n,
                                                                  double* __restrict__ rq) {
    __shared__ double sa[1024], sb[1024];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a += x[i] * z[i];
        b += z[i] * z[i];
    }
    sa[threadIdx.x] = a;
    sb[threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sa[threadIdx.x] += sa[threadIdx.x + w];
            sb[threadIdx.x] += sb[threadIdx.x + w];
        }
        __syncthreads();
    }
    const double xz = sa[0], zz = sb[0];
    if (threadIdx.x == 0) rq[0] = xz;
    if (zz > 0.0) {
        const double sc = rsqrt(zz);
        for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = z[i] * sc;
    }
}

// Doubles of norm2_sq's work vector.
size_t norm2_work_doubles(int n) { return (size_t)n * n + 3 * (size_t)n + 2; }

// The largest eigenvalue of M^T M (M n x n), i.e. ||M||_2^2, by 20 steps of the
// power iteration from the unit vector of equal entries, returned as the last
// Rayleigh quotient: an estimate from below that converges to the eigenvalue.
// work: norm2_work_doubles(n) doubles (M^T, x, y, z and two scalars).
dme_status norm2_sq(const double* M, int n, double* work, size_t work_len, cudaStream_t st, double* out) {
    if (work_len < norm2_work_doubles(n)) return set_error("norm2_sq: work vector too short"), DME_EINVAL;
    double* Mt = work;
    double* x = Mt + (size_t)n * n;
    double* y = x + n;
    double* z = y + n;
    double* s = z + n;
    const int gr = std::min((n + 7) / 8, 1024);
    launch_transpose(M, Mt, n, n, n, n, st);
    fill_kernel<<<(n + 255) / 256, 256, 0, st>>>(x, n, 1.0 / std::sqrt((double)n));
    for (int it = 0; it < 20; ++it) {
        gemv_rows_kernel<<<gr, 256, 0, st>>>(M, x, n, y);                     // y = M x
        gemv_rows_kernel<<<gr, 256, 0, st>>>(Mt, y, n, z);                    // z = M^T y
        rayleigh_normalize_kernel<<<1, 1024, 0, st>>>(x, z, n, s);            // rq = x.z; x = z/|z|
    }
    DME_CUDA_TRY(cudaGetLastError());
    double h = 0.0;
    DME_CUDA_TRY(cudaMemcpyAsync(&h, s, sizeof(h), cudaMemcpyDeviceToHost, st));
    DME_CUDA_TRY(cudaStreamSynchronize(st));
    *out = h;
    return DME_OK;
}

// The split path's slice-pair configuration (dme_plan with pairs = 0): for
// every fixed operand G the plan's steps use (E_t^T per step length, S), one
// congruence G X G^T of the probe X = W_t (Q if W_t = 0, I if both are) under
// P10, P13 and P14 (cheapest first, stopping at the first that meets the
// target) against the FP64 congruence (from n = 512 the accurate tensor mode)
// gives the worst relative error e of one application.  An error made at some step reaches the end of the
// horizon through the later steps, which shrink it at most by
// rho = prod ||E_t||_2^2 over the step's congruences (times 1 + t ||S||^2 +
// t^2 ||S||^4 / 2 per S-flow; T2 and T3 counted as 1, and rho = 1 for the
// extrapolated schemes), so the estimate of the error over H steps is
//     4 e c (1 + rho + ... + rho^(H-1)),   c = congruences per step
// (the worst case of errors adding up in phase; the factor 4 covers the
// probe standing in for the states of the solve).  The cheapest configuration
// whose estimate is within tol is kept.
dme_status choose_pairs(dme_plan_t p) {
    if (!p->split) return DME_OK;
    if (p->d.pairs != 0) {
        p->cfg = cfg_of_pairs(p->d.pairs);
        p->cfg_est = -1.0;
        return DME_OK;
    }
    const int n = p->n;
    const size_t nn = (size_t)n * n;
    cudaStream_t st = p->st;
    long apps = 0;
    for (const Op& o : p->ops) {
        if (o.kind == OP_CONG) apps += 1;
        if (o.kind == OP_SFLOW) apps += (o.rule == DME_T4_EULER) ? 1 : 2;
    }
    const int cands[3] = {OZ_P10, OZ_P13, OZ_P14};
    p->cfg = OZ_P14;
    if (apps == 0) {                      // no tensor-core congruence in a step
        p->cfg_est = 0.0;
        return DME_OK;
    }
    TmpPool tp(st);
    double *X, *out, *tmp, *work, *vec;
    DME_TRY(tp.get(&X, nn));
    DME_TRY(tp.get(&out, nn));
    DME_TRY(tp.get(&tmp, nn));
    DME_TRY(tp.get(&work, 2 * 256 + 2));
    const size_t vec_len = norm2_work_doubles(n);
    DME_TRY(tp.get(&vec, vec_len));
    bool sflow = false;
    for (const Op& o : p->ops) sflow = sflow || o.kind == OP_SFLOW;
    // contraction of one step: ||E_t||_2^2 per congruence, the S-flow's growth
    std::vector<double> e2(p->ew.size(), 1.0);
    for (size_t k = 0; k < p->ew.size(); ++k) DME_TRY(norm2_sq(p->ew[k].E, n, vec, vec_len, st, &e2[k]));
    double s2 = 0.0;
    if (sflow && p->S) DME_TRY(norm2_sq(p->S, n, vec, vec_len, st, &s2));
    double rho = 1.0;
    for (const Op& o : p->ops) {
        if (o.kind == OP_CONG) rho *= e2[o.ew];
        if (o.kind == OP_SFLOW)
            rho *= 1.0 + std::fabs(o.tau) * s2 + (o.rule == DME_T4_EULER ? 0.0 : 0.5 * o.tau * o.tau * s2 * s2);
    }
    if (p->d.extrap > 1 || !(rho >= 0.0)) rho = 1.0;
    const int H = p->d.horizon > 0 ? p->d.horizon : 1024;
    const double tol = p->d.tol > 0.0 ? p->d.tol : 1e-7;
    const double G = rho < 1.0 ? (1.0 - std::pow(rho, (double)H)) / (1.0 - rho) : (double)H;
    const double N = (double)apps * G;
    p->cfg_rho = rho;
    // probe state: W_t of the first step length, else Q, else I (rel_diff against a
    // zero matrix returns the Frobenius norm)
    const double* probe_src = p->ew.empty() ? nullptr : p->ew.front().W;
    double nrm = 0.0;
    DME_CUDA_TRY(cudaMemsetAsync(tmp, 0, nn * sizeof(double), st));
    if (probe_src) DME_TRY(rel_diff(probe_src, tmp, nn, work, st, &nrm));
    if (!(nrm > 0.0)) {
        probe_src = p->Q;
        DME_TRY(rel_diff(p->Q, tmp, nn, work, st, &nrm));
    }
    if (nrm > 0.0) {
        DME_CUDA_TRY(cudaMemcpyAsync(X, probe_src, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
        launch_lincomb(X, n, n, nullptr, 0.0, nullptr, 0.0, nullptr, 0.0, 1.0, st);
    }
    // references of the probe congruence for every fixed operand, E_t^T X E_t and S X S^T:
    // FP64, or from n = kAccMinN on the accurate tensor mode (about 2^-39 of the row
    // scales per product, two orders below the errors measured against it)
    AccWork accw;
    AccWork* aw = nullptr;
    if (n >= kAccMinN) {
        DME_TRY(acc_setup(tp, n, p->status, &accw));
        aw = &accw;
    }
    std::vector<double*> refs;
    std::vector<const SliceBuf*> gs;
    for (const EWEntry& e : p->ew) {
        double* r = nullptr;
        DME_TRY(tp.get(&r, nn));
        DME_TRY(prod(n, aw, X, 0, e.E, 0, tmp, 1.0, nullptr, 0.0, st));
        DME_TRY(prod(n, aw, e.E, 1, tmp, 0, r, 1.0, nullptr, 0.0, st));
        refs.push_back(r);
        gs.push_back(&e.Gsl);
    }
    if (sflow && p->S) {
        double* r = nullptr;
        DME_TRY(tp.get(&r, nn));
        DME_TRY(prod(n, aw, X, 0, p->S, 1, tmp, 1.0, nullptr, 0.0, st));
        DME_TRY(prod(n, aw, p->S, 0, tmp, 0, r, 1.0, nullptr, 0.0, st));
        refs.push_back(r);
        gs.push_back(&p->Ssl);
    }
    // the candidates cheapest first; the first whose estimate meets tol is kept
    for (int c = 0; c < 3; ++c) {
        double worst = 0.0;
        for (size_t k = 0; k < refs.size(); ++k) {
            DME_TRY(split_cong(p, X, *gs[k], out, 1.0, nullptr, 0.0, nullptr, 0.0, nullptr, 0.0, cands[c]));
            double e = 0.0;
            DME_TRY(rel_diff(out, refs[k], nn, work, st, &e));
            worst = std::max(worst, e);
        }
        p->cfg_err[c] = worst;
        p->cfg = cands[c];
        p->cfg_est = 4.0 * N * worst;
        if (p->cfg_est <= tol) break;
    }
    DME_TRY(check_status(p, "dme_plan (slice-pair probe)"));
    return DME_OK;
}

// One composition step as (flow, t) pairs, in application order (§2):
// Lie: each flow over h; Strang: outer flows over h/2 around the last over h.
std::vector<std::pair<int, double>> step_sequence(const dme_plan_desc& d, double h) {
    std::vector<std::pair<int, double>> seq;
    const int k = d.nflows;
    if (k == 1) {
        seq.push_back({d.flows[0], h});
    } else if (d.comp == DME_LIE) {
        for (int i = 0; i < k; ++i) seq.push_back({d.flows[i], h});
    } else {
        for (int i = 0; i < k - 1; ++i) seq.push_back({d.flows[i], 0.5 * h});
        seq.push_back({d.flows[k - 1], h});
        for (int i = k - 2; i >= 0; --i) seq.push_back({d.flows[i], 0.5 * h});
    }
    return seq;
}

int t4_rule_of(const dme_plan_desc& d) {
    if (d.t4_rule == DME_T4_MIDPOINT || d.t4_rule == DME_T4_EULER) return d.t4_rule;
    return d.comp == DME_STRANG ? DME_T4_MIDPOINT : DME_T4_EULER;
}

}  // namespace

namespace {

// Weights of the extrapolated Strang scheme of order 2q (§2 "higher-order
// schemes"): the Lagrange basis at x = 0 on the nodes x_k = 1/k^2, so that
// sum_k gamma_k (S_{h/k})^k cancels the h^2 .. h^(2q-2) terms of Strang's even
// error expansion: gamma_k = prod_{j != k} k^2 / (k^2 - j^2).
double extrap_weight(int q, int k) {
    double g = 1.0;
    for (int j = 1; j <= q; ++j)
        if (j != k) g *= static_cast<double>(k * k) / static_cast<double>(k * k - j * j);
    return g;
}

// Append the ops of one flow sequence acting on state `buf`.  T2 (P + tQ) is
// fused into the epilogue of the op before it in the same sequence when there
// is one, else it is a standalone axpy.
dme_status compile_seq(dme_plan_t p, const std::vector<std::pair<int, double>>& seq, int buf, std::vector<Op>& ops) {
    const size_t first = ops.size();
    for (auto& ft : seq) {
        Op o;
        std::memset(&o, 0, sizeof(o));
        o.tau = ft.second;
        o.buf = buf;
        o.src = -1;
        switch (ft.first) {
            case DME_F1:
            case DME_F12: {
                int idx;
                DME_TRY(compute_ew(p, ft.second, &idx));
                o.kind = OP_CONG;
                o.ew = idx;
                o.wcoef = (ft.first == DME_F12) ? 1.0 : 0.0;
                ops.push_back(o);
                break;
            }
            case DME_F2:
                if (ops.size() > first) {
                    ops.back().qcoef += ft.second;
                } else {
                    o.kind = OP_AXPY;
                    o.qcoef = ft.second;
                    ops.push_back(o);
                }
                break;
            case DME_F3:
                o.kind = OP_RICC;
                ops.push_back(o);
                break;
            case DME_F4:
                o.kind = OP_SFLOW;
                o.rule = t4_rule_of(p->d);
                ops.push_back(o);
                break;
            default:
                set_error("unknown flow");
                return DME_EINVAL;
        }
    }
    return DME_OK;
}

Op state_op(int kind, int buf, int src, double c1, double c2) {
    Op o;
    std::memset(&o, 0, sizeof(o));
    o.kind = kind;
    o.buf = buf;
    o.src = src;
    o.c1 = c1;
    o.c2 = c2;
    return o;
}

void drop_graph(GraphSlot& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.P = nullptr;
    g.kernels = -1;
}

}  // namespace

// Compile one step of size h into ops (and, with fsal, its head / interior /
// closing parts).  Extrapolated scheme of order 2q, one step:
//   acc <- P; k = 1 Strang step of h on acc; acc <- g_1 acc
//   for 1 < k < q: work <- P; k steps of h/k on work; acc <- acc + g_k work
//   k = q steps of h/q on P; P <- g_q P + acc.
dme_status dme::build_ops(dme_plan_t p, double h) {
    if (p->ops_h == h) return DME_OK;
    std::vector<Op> ops, head, body, tail;
    const int q = p->d.extrap > 1 ? p->d.extrap : 1;
    if (q == 1) {
        DME_TRY(compile_seq(p, step_sequence(p->d, h), BUF_P, ops));
    } else {
        const size_t nn = (size_t)p->n * p->n;
        if (!p->xacc) DME_TRY(palloc_t(p, &p->xacc, nn));
        if (q >= 3 && !p->xwork) DME_TRY(palloc_t(p, &p->xwork, nn));
        for (int k = 1; k <= q; ++k) {
            const int buf = (k == q) ? BUF_P : (k == 1 ? BUF_ACC : BUF_WORK);
            if (k < q) ops.push_back(state_op(OP_COPY, buf, BUF_P, 0.0, 0.0));
            const auto seq = step_sequence(p->d, h / k);
            for (int r = 0; r < k; ++r) DME_TRY(compile_seq(p, seq, buf, ops));
            const double g = extrap_weight(q, k);
            if (k == 1)
                ops.push_back(state_op(OP_COMBINE, BUF_ACC, -1, g, 0.0));
            else if (k < q)
                ops.push_back(state_op(OP_COMBINE, BUF_ACC, BUF_WORK, 1.0, g));
            else
                ops.push_back(state_op(OP_COMBINE, BUF_P, BUF_ACC, g, 1.0));
        }
    }
    if (p->d.fsal) {
        // Strang [f0(h/2), inner..., f0(h/2)]: head = f0(h/2) inner, body = f0(h) inner, tail = f0(h/2)
        const auto seq = step_sequence(p->d, h);
        const std::vector<std::pair<int, double>> inner(seq.begin() + 1, seq.end() - 1);
        std::vector<std::pair<int, double>> hs{seq.front()}, bs{{seq.front().first, h}}, ts{seq.back()};
        hs.insert(hs.end(), inner.begin(), inner.end());
        bs.insert(bs.end(), inner.begin(), inner.end());
        DME_TRY(compile_seq(p, hs, BUF_P, head));
        DME_TRY(compile_seq(p, bs, BUF_P, body));
        DME_TRY(compile_seq(p, ts, BUF_P, tail));
    }
    p->ops = ops;
    p->ops_head = head;
    p->ops_body = body;
    p->ops_tail = tail;
    p->ops_h = h;
    drop_graph(p->g_step);
    drop_graph(p->g_head);
    drop_graph(p->g_body);
    drop_graph(p->g_tail);
    return DME_OK;
}

namespace {

dme_status run_sflow(dme_plan_t p, double* P, double tau, int rule, double qcoef) {
    const int n = p->n;
    cudaStream_t st = p->st;
    const double* Qd = qcoef != 0.0 ? p->Q : nullptr;
    // X1 = P S^T ; Xs = S X1  (= S P S^T, symmetric)
    DME_TRY(gemm1(gp(n, n, n, P, n, 0, p->S, n, 1, p->X, n, 1.0), st));
    if (rule == DME_T4_EULER) {
        // P <- P + t S P S^T (+ q Q)
        DME_TRY(gemm1(gp(n, n, n, p->S, n, 0, p->X, n, 0, P, n, tau, 1, P, 1.0, Qd, qcoef), st));
        return DME_OK;
    }
    DME_TRY(gemm1(gp(n, n, n, p->S, n, 0, p->X, n, 0, p->Xs, n, 1.0, 1), st));
    // Y1 = Xs S^T ; P <- P + t Xs + t^2/2 S Y1 (+ q Q)
    DME_TRY(gemm1(gp(n, n, n, p->Xs, n, 0, p->S, n, 1, p->Y1, n, 1.0), st));
    DME_TRY(gemm1(gp(n, n, n, p->S, n, 0, p->Y1, n, 0, P, n, 0.5 * tau * tau, 1, P, 1.0, p->Xs, tau, Qd, qcoef),
                  st));
    return DME_OK;
}

dme_status run_sflow_split(dme_plan_t p, double* P, double tau, int rule, double qcoef) {
    const double* Qd = qcoef != 0.0 ? p->Q : nullptr;
    if (rule == DME_T4_EULER) return split_cong(p, P, p->Ssl, P, tau, P, 1.0, Qd, qcoef, nullptr, 0.0, p->cfg);
    DME_TRY(split_cong(p, P, p->Ssl, p->Xs, 1.0, nullptr, 0.0, nullptr, 0.0, nullptr, 0.0, p->cfg));  // S P S^T
    return split_cong(p, p->Xs, p->Ssl, P, 0.5 * tau * tau, P, 1.0, p->Xs, tau, Qd, qcoef, p->cfg);  // + t^2/2 S Xs S^T
}

}  // namespace

dme_status dme::run_op(dme_plan_t p, const Op& o, double* Pcaller) {
    const int n = p->n;
    cudaStream_t st = p->st;
    auto state = [&](int b) { return b == BUF_ACC ? p->xacc : (b == BUF_WORK ? p->xwork : Pcaller); };
    double* P = state(o.buf);
    if (o.kind == OP_COPY) {
        DME_CUDA_TRY(cudaMemcpyAsync(P, state(o.src), (size_t)n * n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        return DME_OK;
    }
    if (o.kind == OP_COMBINE) {
        launch_lincomb(P, n, n, P, o.c1, o.src >= 0 ? state(o.src) : nullptr, o.c2, nullptr, 0.0, 0.0, st);
        return DME_OK;
    }
    if (p->split && o.kind == OP_CONG) {
        const EWEntry& e = p->ew[o.ew];
        return split_cong(p, P, e.Gsl, P, 1.0, o.wcoef != 0.0 ? e.W : nullptr, o.wcoef,
                          o.qcoef != 0.0 ? p->Q : nullptr, o.qcoef, nullptr, 0.0, p->cfg);
    }
    if (p->split && o.kind == OP_SFLOW) return run_sflow_split(p, P, o.tau, o.rule, o.qcoef);
    switch (o.kind) {
        case OP_CONG: {
            const EWEntry& e = p->ew[o.ew];
            ProfScope ps(p, DME_KIND_FP64_GEMM);
            return cong64(n, P, e.E, p->X, P, o.wcoef != 0.0 ? e.W : nullptr, o.wcoef,
                          o.qcoef != 0.0 ? p->Q : nullptr, o.qcoef, nullptr, 0.0, st);
        }
        case OP_AXPY:
            launch_axpy_sym(P, p->Q, o.qcoef, n, n, st);
            return DME_OK;
        case OP_RICC: {
            ProfScope ps(p, DME_KIND_RICCATI);
            if (p->tric) return split_riccati(p, P, o.tau, o.qcoef);
            launch_riccati(P, p->Bt, n, p->m, o.tau, o.qcoef != 0.0 ? p->Q : nullptr, o.qcoef, p->rwork, p->status,
                           st);
            return DME_OK;
        }
        case OP_SFLOW:
            return run_sflow(p, P, o.tau, o.rule, o.qcoef);
    }
    set_error("bad op");
    return DME_EINVAL;
}

namespace {

dme_status run_ops(dme_plan_t p, const std::vector<Op>& ops, double* P) {
    for (const Op& o : ops) DME_TRY(run_op(p, o, P));
    DME_CUDA_TRY(cudaGetLastError());
    return DME_OK;
}

dme_status validate(const dme_plan_desc* d, const double* A, const double* QorC, const double* B, const double* R,
                    const double* S) {
    if (!d || !A || !QorC) return set_error("desc, A and QorC are required"), DME_EINVAL;
    if (d->n < 1 || d->n > 16384) return set_error("n must be in [1, 16384]"), DME_EINVAL;
    if (d->eq < DME_DLE || d->eq > DME_GDRE) return set_error("bad eq"), DME_EINVAL;
    if (d->comp != DME_LIE && d->comp != DME_STRANG) return set_error("bad comp"), DME_EINVAL;
    if (d->nflows < 1 || d->nflows > 4) return set_error("nflows must be 1..4"), DME_EINVAL;
    if (d->prec == DME_SPLIT_TF32)
        return set_error("DME_SPLIT_TF32 is not built: an 11-bit TF32 digit keeps the fp32 tensor-core sum of "
                         "K digit products exact only for K <= 4 (use DME_SPLIT_BF16)"),
               DME_EINVAL;
    if (d->prec != DME_FP64 && d->prec != DME_SPLIT_BF16) return set_error("bad prec"), DME_EINVAL;
    if (!(d->h > 0.0) || !std::isfinite(d->h)) return set_error("h must be positive and finite"), DME_EINVAL;
    if (d->q_is_factor && (d->p < 1 || d->p > 16384)) return set_error("p must be >= 1 with q_is_factor"), DME_EINVAL;
    const bool ric = (d->eq == DME_DRE || d->eq == DME_GDRE);
    const bool gen = (d->eq == DME_GDLE || d->eq == DME_GDRE);
    for (int i = 0; i < d->nflows; ++i) {
        int f = d->flows[i];
        if (f < DME_F1 || f > DME_F4) return set_error("bad flow id"), DME_EINVAL;
        if (f == DME_F3 && !ric) return set_error("F3 needs eq = DRE or GDRE"), DME_EINVAL;
        if (f == DME_F4 && !gen) return set_error("F4 needs eq = GDLE or GDRE"), DME_EINVAL;
    }
    if (ric && (d->m < 1 || d->m > 32 || !B || !R)) return set_error("DRE needs B, R and 1 <= m <= 32"), DME_EINVAL;
    if (gen && !S) return set_error("generalised equations need S"), DME_EINVAL;
    bool has_f4 = false;
    for (int i = 0; i < d->nflows; ++i) has_f4 = has_f4 || d->flows[i] == DME_F4;
    if (d->extrap < 0 || d->extrap > 4) return set_error("extrap must be 0..4"), DME_EINVAL;
    if (d->extrap > 1 && (d->comp != DME_STRANG || has_f4 || d->fsal))
        return set_error("extrapolation needs Strang over exact flows (no F4) and fsal = 0"), DME_EINVAL;
    if (d->fsal && (d->comp != DME_STRANG || d->nflows < 2 || d->flows[0] == DME_F4))
        return set_error("fsal needs Strang with >= 2 flows and an exact outer flow (not F4)"), DME_EINVAL;
    return DME_OK;
}

}  // namespace

void dme::free_plan(dme_plan_t p) {
    if (!p) return;
    for (GraphSlot* g : {&p->g_step, &p->g_head, &p->g_body, &p->g_tail})
        if (g->exec) cudaGraphExecDestroy(g->exec);
    if (p->st) cudaStreamSynchronize(p->st);
    for (auto& r : p->evrec) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : p->evpool) cudaEventDestroy(e);
    for (void* q : p->allocs) cudaFreeAsync(q, p->st);
    if (p->st) cudaStreamSynchronize(p->st);
    if (p->own_st && p->st) cudaStreamDestroy(p->st);
    delete p;
}

// Split plans from this size on hold a split-K workspace (their products have K >= 512).
constexpr int kSplitKMinN = 512;

size_t dme::plan_estimate_bytes(const dme_plan_desc& d, bool serving) {
    const size_t nn = (size_t)d.n * d.n * sizeof(double);
    int taus = 0;
    for (int i = 0; i < d.nflows; ++i) taus += (d.flows[i] == DME_F1 || d.flows[i] == DME_F12) ? 1 : 0;
    taus = std::max(taus, 1);
    const size_t persistent = (3 + 2 * (size_t)taus + 3) * nn;           // A, Q, X, (E, W) per t, S-flow work
    const size_t transient = 17 * nn;                                   // Pade chain blocks and LU copies
    size_t split = 0;
    if (d.prec == DME_SPLIT_BF16) {
        const size_t sl = (size_t)d.n * slice_kpad(d.n) * 2;           // one bf16 slice plane
        split = (5 * (size_t)taus + 5 + 8) * sl + nn;                   // E^T / S slices, P and U slices, U pairs
        if (d.n >= kSplitKMinN && (!serving || d.n > 1536)) split += OZ_SPLIT_WS_FLOAT2 * sizeof(float2);
    }
    return persistent + transient + split + (size_t)d.n * 64 * sizeof(double) + (1u << 20);
}

namespace {

}  // namespace

dme_status dme::plan_create(const dme_plan_desc* d, const double* A, const double* QorC, const double* B,
                            const double* R, const double* S, void* stream, dme_plan_t* out, bool serving) {
    DME_TRY(validate(d, A, QorC, B, R, S));
    if (d->prec == DME_SPLIT_BF16 && d->n > OZ_MAX_K) {
        set_error("DME_SPLIT_BF16 supports n <= 4096 (exact slice accumulation over K <= 4096)");
        return DME_EINVAL;
    }
    if (d->prec == DME_SPLIT_BF16 && d->pairs != 0 && d->pairs != 10 && d->pairs != 13 && d->pairs != 14) {
        set_error("DME_SPLIT_BF16: pairs must be 0 (chosen at plan time), 10, 13 or 14");
        return DME_EINVAL;
    }
    if (d->horizon < 0 || !(d->tol >= 0.0) || !std::isfinite(d->tol)) {
        set_error("horizon must be >= 0 and tol finite and >= 0");
        return DME_EINVAL;
    }
    dme_plan_t p = new (std::nothrow) dme_plan_s();
    if (!p) return set_error("host allocation failed"), DME_ENOMEM;
    std::unique_ptr<dme_plan_s, void (*)(dme_plan_t)> guard(p, free_plan);
    p->d = *d;
    const int n = d->n;
    const bool ric = (d->eq == DME_DRE || d->eq == DME_GDRE);
    const bool gen = (d->eq == DME_GDLE || d->eq == DME_GDRE);
    p->n = n;
    p->m = ric ? d->m : 0;
    p->split = (d->prec == DME_SPLIT_BF16);
    if (stream) {
        p->st = reinterpret_cast<cudaStream_t>(stream);
    } else {
        DME_CUDA_TRY(cudaStreamCreateWithFlags(&p->st, cudaStreamNonBlocking));
        p->own_st = true;
    }
    const size_t nn = (size_t)n * n;
    cudaStream_t st = p->st;
    DME_TRY(palloc_t(p, &p->status, 4));
    DME_CUDA_TRY(cudaMemsetAsync(p->status, 0, 4 * sizeof(int), st));
    DME_TRY(palloc_t(p, &p->A, nn));
    DME_TRY(palloc_t(p, &p->Q, nn));
    DME_TRY(palloc_t(p, &p->X, nn));
    DME_TRY(palloc_t(p, &p->small, 2 * (size_t)n + 16));
    DME_CUDA_TRY(cudaMemcpyAsync(p->A, A, nn * sizeof(double), cudaMemcpyDefault, st));
    if (d->q_is_factor) {
        TmpPool tp(st);
        double* C = nullptr;
        DME_TRY(tp.get(&C, (size_t)d->p * n));
        DME_CUDA_TRY(cudaMemcpyAsync(C, QorC, (size_t)d->p * n * sizeof(double), cudaMemcpyDefault, st));
        DME_TRY(gemm1(gp(n, n, d->p, C, n, 1, C, n, 0, p->Q, n, 1.0), st));   // Q = C^T C
        DME_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
        DME_CUDA_TRY(cudaMemcpyAsync(p->Q, QorC, nn * sizeof(double), cudaMemcpyDefault, st));
    }
    if (ric) {
        const int m = d->m;
        TmpPool tp(st);
        double *Bd = nullptr, *Rd = nullptr;
        DME_TRY(tp.get(&Bd, (size_t)n * m));
        DME_TRY(palloc_t(p, &p->LR, (size_t)m * m));
        Rd = p->LR;
        DME_CUDA_TRY(cudaMemcpyAsync(Bd, B, (size_t)n * m * sizeof(double), cudaMemcpyDefault, st));
        DME_CUDA_TRY(cudaMemcpyAsync(Rd, R, (size_t)m * m * sizeof(double), cudaMemcpyDefault, st));
        DME_TRY(palloc_t(p, &p->Bt, (size_t)n * m));
        launch_small_cholesky(Rd, m, p->status, st);
        launch_apply_linv_rows(Bd, Rd, p->Bt, n, m, st);
        DME_TRY(check_status(p, "dme_plan (Cholesky of R)"));
        DME_TRY(palloc_t(p, &p->rwork, riccati_work_doubles(n, m)));
    }
    if (gen) {
        DME_TRY(palloc_t(p, &p->S, nn));
        DME_TRY(palloc_t(p, &p->Xs, nn));
        DME_TRY(palloc_t(p, &p->Y1, nn));
        DME_CUDA_TRY(cudaMemcpyAsync(p->S, S, nn * sizeof(double), cudaMemcpyDefault, st));
    }
    if (p->split) {
        DME_TRY(alloc_slices(p, &p->psl, n, n, OZ_SLICES_STEP));
        DME_TRY(alloc_slices(p, &p->usl, n, n, OZ_SLICES_STEP));
        DME_TRY(palloc_t(p, &p->U, nn));
        if (n >= kSplitKMinN && (!serving || n > 1536)) {
            // split K (K >= 512): the single partial wave of a product of at most 76 tiles
            // (n <= 1024 here), or the last partial wave of one with more tiles than SMs
            // (n > 1536; the plan's own tensor Riccati products need it in serving too)
            DME_TRY(palloc_t(p, &p->kws, OZ_SPLIT_WS_FLOAT2));
            DME_TRY(palloc_t(p, &p->kcnt, (size_t)OZ_SPLIT_MAX_TAIL));
            DME_CUDA_TRY(cudaMemsetAsync(p->kcnt, 0, sizeof(int) * OZ_SPLIT_MAX_TAIL, st));
        }
        if (n > 1536) {
            if (ric) {
                // the Riccati products on the tensor cores (below 1537 the FP64 kernels are
                // cheap, and serving, which uses them, stays bit-identical to single plans)
                const int m = p->m;
                p->tric = true;
                DME_TRY(palloc_t(p, &p->Zt, (size_t)m * n));
                DME_TRY(alloc_slices(p, &p->btsl, m, n, OZ_SLICES_FIXED));
                DME_TRY(alloc_slices(p, &p->ysla, n, m, OZ_SLICES_FIXED));
                DME_TRY(alloc_slices(p, &p->yslb, n, m, OZ_SLICES_STEP));
                launch_transpose(p->Bt, p->Zt, n, m, m, n, st);
                launch_slice_rows_f64(p->Zt, m, n, n, p->btsl, st);
            }
        }
        if (gen) {
            DME_TRY(alloc_slices(p, &p->Ssl, n, n, OZ_SLICES_FIXED));
            launch_slice_rows_f64(p->S, n, n, n, p->Ssl, st);
        }
    }
    // ||[[-A^T, Q], [0, A]]||_1 for the scaling of every t
    launch_block_norm1(p->A, p->Q, n, p->small, st);
    launch_max_reduce(p->small, 2 * n, p->small + 2 * n, st);
    DME_CUDA_TRY(cudaMemcpyAsync(&p->normM, p->small + 2 * n, sizeof(double), cudaMemcpyDeviceToHost, st));
    DME_CUDA_TRY(cudaStreamSynchronize(st));
    DME_TRY(build_ops(p, d->h));
    DME_TRY(check_status(p, "dme_plan"));
    DME_TRY(choose_pairs(p));
    *out = guard.release();
    return DME_OK;
}

namespace {

// Replay the op list `ops` `count` times on P from its CUDA graph (captured
// on first use for this P).
dme_status replay(dme_plan_t p, GraphSlot& slot, const std::vector<Op>& ops, double* P, int count) {
    if (count <= 0) return DME_OK;
    if (!slot.exec || slot.P != P) {
        if (slot.exec) {
            cudaGraphExecDestroy(slot.exec);
            slot.exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        DME_CUDA_TRY(cudaStreamBeginCapture(p->st, cudaStreamCaptureModeThreadLocal));
        dme_status s = run_ops(p, ops, P);
        cudaError_t e = cudaStreamEndCapture(p->st, &g);
        if (s != DME_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) return set_error(std::string("graph capture: ") + cudaGetErrorString(e)), DME_ECUDA;
        size_t nn = 0;
        int kernels = 0;
        if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
            std::vector<cudaGraphNode_t> nodes(nn);
            if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
                for (size_t i = 0; i < nn; ++i) {
                    cudaGraphNodeType ty;
                    if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kernels;
                }
        }
        slot.kernels = kernels;
        e = cudaGraphInstantiate(&slot.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return set_error(std::string("graph instantiate: ") + cudaGetErrorString(e)), DME_ECUDA;
        slot.P = P;
    }
    for (int k = 0; k < count; ++k) DME_CUDA_TRY(cudaGraphLaunch(slot.exec, p->st));
    return DME_OK;
}

// nsteps composition steps on P.  With fsal and nsteps >= 2 the outer half
// steps of neighbouring steps are merged: head, nsteps - 1 interior parts, tail.
dme_status step_graph(dme_plan_t p, double* P, int nsteps) {
    if (!p->d.fsal || nsteps < 2) return replay(p, p->g_step, p->ops, P, nsteps);
    DME_TRY(replay(p, p->g_head, p->ops_head, P, 1));
    DME_TRY(replay(p, p->g_body, p->ops_body, P, nsteps - 1));
    return replay(p, p->g_tail, p->ops_tail, P, 1);
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

dme_status dme_plan(const dme_plan_desc* desc, const double* A, const double* QorC, const double* B,
                    const double* R, const double* S, void* cuda_stream, dme_plan_t* out) {
    if (!out) return set_error("out is NULL"), DME_EINVAL;
    *out = nullptr;
    set_error("");
    return guarded([&] { return plan_create(desc, A, QorC, B, R, S, cuda_stream, out); });
}

dme_status dme_plan_mass(const dme_plan_desc* desc, const double* M, const double* A, const double* QorC,
                         const double* B, const double* R, const double* S, void* cuda_stream, dme_plan_t* out) {
    if (!out) return set_error("out is NULL"), DME_EINVAL;
    *out = nullptr;
    set_error("");
    if (!M) return set_error("dme_plan_mass: M is required"), DME_EINVAL;
    if (S) return set_error("dme_plan_mass: the mass-matrix form has no S term"), DME_EINVAL;
    DME_TRY(validate(desc, A, QorC, B, R, S));
    return guarded([&]() -> dme_status {
        const int n = desc->n;
        const size_t nn = (size_t)n * n;
        cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
        bool own = false;
        if (!st) {
            DME_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            own = true;
        }
        std::unique_ptr<CUstream_st, void (*)(cudaStream_t)> sg(own ? st : nullptr, [](cudaStream_t x) {
            if (x) {
                cudaStreamSynchronize(x);
                cudaStreamDestroy(x);
            }
        });
        TmpPool tp(st);
        double *Mt, *At, *Qt, *X, *Y, *Mi, *gjw, *stat;
        DME_TRY(tp.get(&Mt, nn));
        DME_TRY(tp.get(&At, nn));
        DME_TRY(tp.get(&Qt, nn));
        DME_TRY(tp.get(&X, nn));
        DME_TRY(tp.get(&Y, nn));
        DME_TRY(tp.get(&Mi, nn));
        DME_TRY(tp.get(&gjw, gj_work_doubles(n, n)));
        DME_TRY(tp.get(&stat, 2));
        int* status = reinterpret_cast<int*>(stat);
        DME_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
        DME_CUDA_TRY(cudaMemcpyAsync(X, M, nn * sizeof(double), cudaMemcpyDefault, st));
        DME_CUDA_TRY(cudaMemcpyAsync(Y, A, nn * sizeof(double), cudaMemcpyDefault, st));
        if (desc->q_is_factor) {
            double* C = nullptr;
            DME_TRY(tp.get(&C, (size_t)desc->p * n));
            DME_CUDA_TRY(cudaMemcpyAsync(C, QorC, (size_t)desc->p * n * sizeof(double), cudaMemcpyDefault, st));
            DME_TRY(gemm1(gp(n, n, desc->p, C, n, 1, C, n, 0, Qt, n, 1.0), st));   // Q = C^T C
        } else {
            DME_CUDA_TRY(cudaMemcpyAsync(Qt, QorC, nn * sizeof(double), cudaMemcpyDefault, st));
        }
        // M^-T by Gauss-Jordan with partial pivoting (a mass matrix is well conditioned)
        launch_transpose(X, Mt, n, n, n, n, st);                                   // Mt = M^T
        launch_lincomb(Mi, n, n, nullptr, 0.0, nullptr, 0.0, nullptr, 0.0, 1.0, st);   // Mi = I
        DME_TRY(launch_gj_solve(Mt, n, n, Mi, n, n, gjw, status, st));             // Mi = M^-T
        DME_TRY(gemm1(gp(n, n, n, Y, n, 0, Mi, n, 1, At, n, 1.0), st));           // A~ = A M^-1
        DME_TRY(gemm1(gp(n, n, n, Qt, n, 0, Mi, n, 1, Y, n, 1.0), st));           // Q M^-1
        DME_TRY(gemm1(gp(n, n, n, Mi, n, 0, Y, n, 0, X, n, 1.0), st));            // Q~ = M^-T Q M^-1
        launch_symmetrize(X, n, n, st);
        DME_CUDA_TRY(cudaGetLastError());
        int hs = 0;
        DME_CUDA_TRY(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
        DME_CUDA_TRY(cudaStreamSynchronize(st));
        if (hs) return set_error("dme_plan_mass: M is singular"), DME_EINVAL;
        dme_plan_desc d2 = *desc;
        d2.q_is_factor = 0;
        return plan_create(&d2, At, X, B, R, nullptr, cuda_stream, out);
    });
}

dme_status dme_wait_selftest(int* timed_out) {
    set_error("");
    if (!timed_out) return set_error("dme_wait_selftest: timed_out is NULL"), DME_EINVAL;
    *timed_out = 0;
    return guarded([&]() -> dme_status { return wait_timeout_selftest(timed_out); });
}

dme_status dme_dense_solve(const double* M, int n, double* B, int nrhs, void* cuda_stream) {
    set_error("");
    if (!M || !B || n < 1 || nrhs < 0) return set_error("dme_dense_solve: need M, B, n >= 1, nrhs >= 0"), DME_EINVAL;
    if (nrhs == 0) return DME_OK;
    return guarded([&]() -> dme_status {
        cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
        bool own = false;
        if (!st) {
            DME_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            own = true;
        }
        std::unique_ptr<CUstream_st, void (*)(cudaStream_t)> sg(own ? st : nullptr, [](cudaStream_t x) {
            if (x) {
                cudaStreamSynchronize(x);
                cudaStreamDestroy(x);
            }
        });
        TmpPool tp(st);
        const size_t nn = (size_t)n * n, nb = (size_t)n * nrhs;
        double *Md, *Bd, *gjw, *stat;
        DME_TRY(tp.get(&Md, nn));
        DME_TRY(tp.get(&Bd, nb));
        DME_TRY(tp.get(&gjw, gj_work_doubles(n, nrhs)));
        DME_TRY(tp.get(&stat, 2));
        int* status = reinterpret_cast<int*>(stat);
        DME_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), st));
        DME_CUDA_TRY(cudaMemcpyAsync(Md, M, nn * sizeof(double), cudaMemcpyDefault, st));
        DME_CUDA_TRY(cudaMemcpyAsync(Bd, B, nb * sizeof(double), cudaMemcpyDefault, st));
        DME_TRY(launch_gj_solve(Md, n, n, Bd, nrhs, nrhs, gjw, status, st));
        int hs = 0;
        DME_CUDA_TRY(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
        DME_CUDA_TRY(cudaStreamSynchronize(st));
        if (hs & DEV_SINGULAR) return set_error("dme_dense_solve: M is singular"), DME_EINVAL;
        if (hs) return set_error("dme_dense_solve: device status " + std::to_string(hs)), DME_ECUDA;
        DME_CUDA_TRY(cudaMemcpyAsync(B, Bd, nb * sizeof(double), cudaMemcpyDefault, st));
        DME_CUDA_TRY(cudaStreamSynchronize(st));
        return DME_OK;
    });
}

dme_status dme_expm(dme_plan_t plan, double t, double* E_out, double* W_out) {
    if (!plan) return set_error("plan is NULL"), DME_EINVAL;
    if (!std::isfinite(t)) return set_error("t must be finite"), DME_EINVAL;
    return guarded([&]() -> dme_status {
        int idx;
        DME_TRY(compute_ew(plan, t, &idx));
        const size_t bytes = (size_t)plan->n * plan->n * sizeof(double);
        if (E_out) DME_CUDA_TRY(cudaMemcpyAsync(E_out, plan->ew[idx].E, bytes, cudaMemcpyDefault, plan->st));
        if (W_out) DME_CUDA_TRY(cudaMemcpyAsync(W_out, plan->ew[idx].W, bytes, cudaMemcpyDefault, plan->st));
        DME_CUDA_TRY(cudaStreamSynchronize(plan->st));
        return DME_OK;
    });
}

static dme_status apply_impl(dme_plan_t plan, int flow, double t, double* P, bool sync) {
    if (!plan || !P) return set_error("plan and P are required"), DME_EINVAL;
    if (!std::isfinite(t)) return set_error("t must be finite"), DME_EINVAL;
    return guarded([&]() -> dme_status {
        Op o;
        std::memset(&o, 0, sizeof(o));
        o.tau = t;
        switch (flow) {
            case DME_F1:
            case DME_F12: {
                int idx;
                DME_TRY(compute_ew(plan, t, &idx));
                o.kind = OP_CONG;
                o.ew = idx;
                o.wcoef = flow == DME_F12 ? 1.0 : 0.0;
                break;
            }
            case DME_F2:
                o.kind = OP_AXPY;
                o.qcoef = t;
                break;
            case DME_F3:
                if (!plan->Bt) return set_error("F3 needs a DRE/GDRE plan"), DME_EINVAL;
                o.kind = OP_RICC;
                break;
            case DME_F4:
                if (!plan->S) return set_error("F4 needs a GDLE/GDRE plan"), DME_EINVAL;
                o.kind = OP_SFLOW;
                o.rule = t4_rule_of(plan->d);
                break;
            default:
                return set_error("bad flow id"), DME_EINVAL;
        }
        DME_TRY(run_op(plan, o, P));
        DME_CUDA_TRY(cudaGetLastError());
        return sync ? check_status(plan, "dme_apply") : DME_OK;
    });
}

dme_status dme_apply(dme_plan_t plan, int flow, double t, double* P) { return apply_impl(plan, flow, t, P, true); }

dme_status dme_apply_async(dme_plan_t plan, int flow, double t, double* P) {
    return apply_impl(plan, flow, t, P, false);
}

dme_status dme_sync(dme_plan_t plan) {
    if (!plan) return set_error("plan is NULL"), DME_EINVAL;
    return guarded([&] { return check_status(plan, "dme_sync"); });
}

int dme_plan_kernels_per_step(dme_plan_t plan) {
    if (!plan) return -1;
    return plan->d.fsal && plan->g_body.exec ? plan->g_body.kernels : plan->g_step.kernels;
}

dme_status dme_gain(dme_plan_t plan, const double* P, double* K_out) {
    if (!plan || !P || !K_out) return set_error("plan, P and K_out are required"), DME_EINVAL;
    if (!plan->Bt) return set_error("dme_gain needs a DRE/GDRE plan (B, R)"), DME_EINVAL;
    return guarded([&]() -> dme_status {
        const int n = plan->n, m = plan->m;
        if (!plan->Kbuf) DME_TRY(palloc_t(plan, &plan->Kbuf, (size_t)m * n));
        DME_TRY(launch_lqr_gain(P, plan->Bt, plan->LR, n, m, plan->rwork, plan->Kbuf, plan->st));
        DME_CUDA_TRY(cudaMemcpyAsync(K_out, plan->Kbuf, sizeof(double) * m * n, cudaMemcpyDefault, plan->st));
        return check_status(plan, "dme_gain");
    });
}

dme_status dme_plan_profile(dme_plan_t plan, int enable) {
    if (!plan) return set_error("plan is NULL"), DME_EINVAL;
    plan->prof = enable != 0;
    return DME_OK;
}

dme_status dme_plan_timing(dme_plan_t plan, int kind, double* ms, int* launches) {
    if (!plan || !ms || !launches) return set_error("plan, ms and launches are required"), DME_EINVAL;
    DME_CUDA_TRY(cudaStreamSynchronize(plan->st));
    double tot = 0.0;
    int cnt = 0;
    std::vector<dme_plan_s::EvRec> keep;
    for (auto& r : plan->evrec) {
        if (r.kind != kind) {
            keep.push_back(r);
            continue;
        }
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) tot += t;
        ++cnt;
        plan->evpool.push_back(r.a);
        plan->evpool.push_back(r.b);
    }
    plan->evrec.swap(keep);
    *ms = tot;
    *launches = cnt;
    return DME_OK;
}

dme_status dme_step(dme_plan_t plan, double* P, int nsteps) {
    if (!plan || !P) return set_error("plan and P are required"), DME_EINVAL;
    if (nsteps < 0) return set_error("nsteps must be >= 0"), DME_EINVAL;
    return guarded([&]() -> dme_status {
        DME_TRY(build_ops(plan, plan->d.h));
        DME_TRY(step_graph(plan, P, nsteps));
        return check_status(plan, "dme_step");
    });
}

dme_status dme_step_async(dme_plan_t plan, double* P, int nsteps) {
    if (!plan || !P) return set_error("plan and P are required"), DME_EINVAL;
    if (nsteps < 0) return set_error("nsteps must be >= 0"), DME_EINVAL;
    return guarded([&]() -> dme_status {
        DME_TRY(build_ops(plan, plan->d.h));
        DME_TRY(step_graph(plan, P, nsteps));
        DME_CUDA_TRY(cudaGetLastError());
        return DME_OK;
    });
}

dme_status dme_solve(dme_plan_t plan, const double* P0, double T, int nsteps, double* P_out) {
    if (!plan || !P0 || !P_out) return set_error("plan, P0 and P_out are required"), DME_EINVAL;
    if (nsteps < 1 || !(T > 0.0) || !std::isfinite(T)) return set_error("need nsteps >= 1 and T > 0"), DME_EINVAL;
    return guarded([&]() -> dme_status {
        const size_t bytes = (size_t)plan->n * plan->n * sizeof(double);
        if (!plan->state) DME_TRY(palloc_t(plan, &plan->state, (size_t)plan->n * plan->n));
        DME_TRY(build_ops(plan, T / nsteps));
        DME_CUDA_TRY(cudaMemcpyAsync(plan->state, P0, bytes, cudaMemcpyDefault, plan->st));
        DME_TRY(step_graph(plan, plan->state, nsteps));
        DME_CUDA_TRY(cudaMemcpyAsync(P_out, plan->state, bytes, cudaMemcpyDefault, plan->st));
        return check_status(plan, "dme_solve");
    });
}

size_t dme_plan_bytes(dme_plan_t plan) { return plan ? plan->bytes : 0; }

dme_status dme_plan_destroy(dme_plan_t plan) {
    free_plan(plan);
    return DME_OK;
}

const char* dme_last_error(void) { return get_error(); }

static dme_status gemm_split_impl(int M, int N, int K, const double* A, const double* B, double* C,
                                  void* cuda_stream, bool acc) {
    if (M < 0 || N < 0 || K < 1 || K > OZ_MAX_K || !A || !B || !C)
        return set_error("dme_gemm_split: need 1 <= K <= 4096 and non-null A, B, C"), DME_EINVAL;
    if (M == 0 || N == 0) return DME_OK;
    return guarded([&]() -> dme_status {
        cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
        const int Kp = slice_kpad(K);
        std::vector<void*> tmp;
        auto cleanup = [&] {
            cudaStreamSynchronize(st);
            for (void* q : tmp) cudaFree(q);
        };
        auto get = [&](size_t bytes, void** out) -> dme_status {
            if (cudaMalloc(out, bytes) != cudaSuccess) {
                cudaGetLastError();
                set_error("dme_gemm_split: cudaMalloc failed");
                return DME_ENOMEM;
            }
            tmp.push_back(*out);
            return DME_OK;
        };
        SliceBuf sa, sb;
        sa.rows = M;
        sa.k = K;
        sa.Kp = Kp;
        sa.ns = acc ? OZ_SLICES_ACC : OZ_SLICES_FIXED;
        sa.scheme = acc ? OZ_DIG7 : OZ_DIG9;
        sb.rows = N;
        sb.k = K;
        sb.Kp = Kp;
        sb.ns = acc ? OZ_SLICES_ACC : OZ_SLICES_STEP;
        sb.scheme = sa.scheme;
        int* status = nullptr;
        dme_status s = DME_OK;
        if ((s = get(slice_buf_bytes(M, K, sa.ns), reinterpret_cast<void**>(&sa.data))) != DME_OK ||
            (s = get(slice_buf_bytes(N, K, sb.ns), reinterpret_cast<void**>(&sb.data))) != DME_OK ||
            (s = get(sizeof(float) * M, reinterpret_cast<void**>(&sa.scale))) != DME_OK ||
            (s = get(sizeof(float) * N, reinterpret_cast<void**>(&sb.scale))) != DME_OK ||
            (s = get(sizeof(int), reinterpret_cast<void**>(&status))) != DME_OK ||
            (s = make_slice_tmaps(sa)) != DME_OK || (s = make_slice_tmaps(sb)) != DME_OK) {
            cleanup();
            return s;
        }
        double* wsd = nullptr;
        if (acc && (s = get(sizeof(double) * oz_acc_ws_doubles(M, N, K), reinterpret_cast<void**>(&wsd))) != DME_OK) {
            cleanup();
            return s;
        }
        cudaMemsetAsync(status, 0, sizeof(int), st);
        launch_slice_rows_f64(A, M, K, K, sa, st);
        launch_slice_rows_f64(B, N, K, K, sb, st);
        OzParams o;
        s = oz_params(sa, sb, acc ? OZ_A21 : OZ_P14, &o);
        o.mode = OZ_OUT_F64;
        o.ldc = N;
        o.Cd = C;
        o.status = status;
        o.wsd = wsd;
        if (s == DME_OK) s = launch_ozaki_gemm(oz_tmap_a(sa, o.cfg), oz_tmap_b(sb, o.cfg), o, st);
        int hs = 0;
        if (s == DME_OK) {
            cudaError_t e = cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) {
                set_error(std::string("dme_gemm_split: ") + cudaGetErrorString(e));
                s = DME_ECUDA;
            } else if (hs) {
                set_error("dme_gemm_split: device status " + std::to_string(hs));
                s = DME_ECUDA;
            }
        }
        cleanup();
        return s;
    });
}

dme_status dme_gemm_split(int M, int N, int K, const double* A, const double* B, double* C, void* cuda_stream) {
    return gemm_split_impl(M, N, K, A, B, C, cuda_stream, false);
}

dme_status dme_gemm_split_acc(int M, int N, int K, const double* A, const double* B, double* C, void* cuda_stream) {
    return gemm_split_impl(M, N, K, A, B, C, cuda_stream, true);
}

dme_status dme_plan_split_choice(dme_plan_t plan, int* pairs, double* est) {
    if (!plan) return set_error("plan is NULL"), DME_EINVAL;
    if (pairs) *pairs = plan->split ? oz_cfg_pairs(plan->cfg) : 0;
    if (est) *est = plan->split ? plan->cfg_est : 0.0;
    return DME_OK;
}

dme_status dme_plan_split_probe(dme_plan_t plan, double* err, double* rho) {
    if (!plan) return set_error("plan is NULL"), DME_EINVAL;
    if (!plan->split || plan->d.pairs != 0 || plan->cfg_est < 0.0)
        return set_error("dme_plan_split_probe: the plan did not choose its slice products (pairs = 0, split)"),
               DME_EINVAL;
    if (err)
        for (int c = 0; c < 3; ++c) err[c] = plan->cfg_err[c];
    if (rho) *rho = plan->cfg_rho;
    return DME_OK;
}

}  // extern "C"

dme_status dme::plan_ew(dme_plan_t p, double t, int* idx) { return compute_ew(p, t, idx); }
dme_status dme::plan_check(dme_plan_t p, const char* where) { return check_status(p, where); }
std::vector<std::pair<int, double>> dme::plan_step_sequence(const dme_plan_desc& d, double h) {
    return step_sequence(d, h);
}
dme_status dme::plan_validate(const dme_plan_desc* d, const double* A, const double* QorC, const double* B,
                              const double* R, const double* S) {
    return validate(d, A, QorC, B, R, S);
}
