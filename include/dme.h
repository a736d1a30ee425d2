/*
 * dme.h -- C ABI of libdme.so: dense splitting schemes for differential
 * Lyapunov and Riccati equations on one GB300 (sm_103a).
 *
 * Problem class (Mena, Pfurtscheller & Stillfjord, arXiv:1805.08990, §1):
 *     dP/dt = A^T P + P A + Q + G(P),   P(0) = P0,
 *     G = 0 (DLE, Eq. lyap), G(P) = -P B R^{-1} B^T P (DRE, Eq. ricc),
 *     plus S P S^T in the generalised forms (Eq. lyapGen, §2.4).
 *
 * Sub-flows (§2): T1(t)P = e^{tA^T} P e^{tA}; T2(t)P = P + tQ;
 * T12(t)P = E^T P E + W with E = e^{tA}, W = int_0^t e^{sA^T} Q e^{sA} ds
 * (Eq. full); T3(t)P = (I + t P B R^{-1} B^T)^{-1} P (Eq. nonlinear), applied
 * through an m x m solve; T4(t)P ~ P + t S(P + t/2 S P S^T)S^T (midpoint, §2.3)
 * or P + t S P S^T (explicit Euler, enough for Lie).  Compositions (§2, §3):
 * Lie applies the listed flows in order, each over h; Strang "Fa Fb Fc" applies
 * Ta(h/2) Tb(h/2) Tc(h) Tb(h/2) Ta(h/2).
 *
 * Conventions for every entry point:
 *  - Matrices are float64, row-major, dense, leading dimension = column count.
 *  - Pointers may be host or device memory (detected per pointer); the caller
 *    owns them and keeps them valid for the duration of the call.  The plan
 *    copies A, Q/C, B, R, S into plan-owned device buffers.
 *  - Functions return a dme_status and never throw across the ABI; the text
 *    of the last error of the calling thread is returned by dme_last_error().
 *  - Work is enqueued on the plan's CUDA stream; every entry point that
 *    reports a device status synchronises that stream before returning.
 */
#ifndef DME_H
#define DME_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DME_OK = 0,
    DME_EINVAL = 1,     /* bad argument (sizes, flags, null where required)      */
    DME_ENOMEM = 2,     /* device allocation failed or HBM budget exceeded       */
    DME_ENOTSPD = 3,    /* R, or I_m + t Bt^T P Bt, failed its Cholesky           */
    DME_ECUDA = 4,      /* a CUDA runtime/driver call failed                      */
    DME_ETIMEOUT = 5,   /* dme_poll waited longer than its timeout                */
    DME_EBUSY = 6,      /* server has no free slot and the queue is full          */
    DME_ENOTREADY = 7   /* request not finished (dme_poll with timeout 0)         */
} dme_status;

typedef enum { DME_DLE = 0, DME_DRE = 1, DME_GDLE = 2, DME_GDRE = 3 } dme_eq;
/* sub-flows T1, T2, T12, T3, T4 of §2 */
typedef enum { DME_F1 = 1, DME_F2 = 2, DME_F12 = 3, DME_F3 = 4, DME_F4 = 5 } dme_flow;
typedef enum { DME_LIE = 1, DME_STRANG = 2 } dme_comp;
/* DME_FP64: every product in float64 on the FP64 pipe.
 * DME_SPLIT_TF32: reserved; not built.  A TF32 slice carries an 11-bit digit,
 *   so the fp32 tensor-core sum of K products of two such digits is exact
 *   only for K <= 4; plans asking for it fail with DME_EINVAL and say so in
 *   dme_last_error().
 * DME_SPLIT_BF16: congruences (T1, T12, T4) as error-free bf16 slice products
 *   on tcgen05 tensor cores accumulated in fp32, exactly for the leading
 *   level (Ozaki splitting), combined in fp64; n <= 4096.  The Riccati m x m
 *   solve, the Pade denominator solve and the squarings of the exponential
 *   stay fp64. */
typedef enum { DME_FP64 = 0, DME_SPLIT_TF32 = 1, DME_SPLIT_BF16 = 2 } dme_prec;
/* T4 rule; AUTO = midpoint for Strang, explicit Euler for Lie (§2.3). */
typedef enum { DME_T4_AUTO = 0, DME_T4_MIDPOINT = 1, DME_T4_EULER = 2 } dme_t4_rule;

typedef struct {
    int n;              /* state dimension, 1 <= n <= 16384 (<= 4096 with DME_SPLIT_BF16) */
    int m;              /* columns of B (DRE/GDRE), 0 otherwise, m <= 32             */
    int p;              /* rows of C when q_is_factor = 1 (Q = C^T C)                 */
    int eq;             /* dme_eq                                                     */
    int comp;           /* dme_comp                                                   */
    int nflows;         /* 1..4                                                       */
    int flows[4];       /* dme_flow list in application order (e.g. F12,F3)          */
    int prec;           /* dme_prec                                                   */
    double h;           /* step size                                                  */
    int q_is_factor;    /* 1: QorC is C (p x n); 0: QorC is Q (n x n, symmetric)      */
    int t4_rule;        /* dme_t4_rule                                                */
    int pairs;          /* DME_SPLIT_BF16: bf16 slice products per output of the     */
                        /*    tensor-core products: 10, 13 or 14, or 0 = chosen at    */
                        /*    plan time (see dme_plan); ignored for DME_FP64          */
    int fsal;           /* 1: merge the outer half steps of consecutive Strang steps  */
                        /*    (T_a(h/2) T_a(h/2) = T_a(h) for an exact outer flow; no */
                        /*    F4 outside).  Same result up to rounding, one outer     */
                        /*    sub-flow less per step.  0 = off.  Plans only.          */
    int extrap;         /* q >= 2: extrapolated Strang of order 2q (§2 "higher-order  */
                        /*    schemes"): P <- sum_k gamma_k (S_{h/k})^k P, k = 1..q,  */
                        /*    gamma_k = prod_{j!=k} k^2/(k^2-j^2); q <= 4; Strang of  */
                        /*    exact flows only (no F4).  0 or 1 = plain.  Plans only. */
    int horizon;        /* steps over which the split path's error target must hold  */
                        /*    when pairs = 0 (0: 1024)                                */
    double tol;         /* that target, relative Frobenius error (0: 1e-7)            */
} dme_plan_desc;

typedef struct dme_plan_s* dme_plan_t;
typedef struct dme_server_s* dme_server_t;

/* Build a plan: copy the problem data to the device, form Q = C^T C (if
 * q_is_factor), Bt = B L_R^{-T} with R = L_R L_R^T (so B R^{-1} B^T = Bt Bt^T),
 * and, for every step length t the scheme uses in T1/T12, E_t = e^{tA} and
 * W_t (Eq. full) by [13/13] Pade scaling and squaring of the Van Loan matrix
 * t[[-A^T, Q],[0, A]] (its 1-norm sets the squarings; the exponential is
 * built from its n x n blocks, see dme_expm).
 *   A: n x n.  QorC: n x n or p x n.  B: n x m (NULL unless DRE/GDRE).
 *   R: m x m SPD (NULL unless DRE/GDRE).  S: n x n (NULL unless GDLE/GDRE).
 *   cuda_stream: a cudaStream_t, or NULL for a plan-owned stream.
 * With DME_SPLIT_BF16 every per-step product is an error-free bf16 slice
 * product (a leading 7-bit digit, trailing 9-bit digits; 4 slices of P, 4 or 5
 * of E^T and S).  With pairs = 0 the plan chooses how many slice products to
 * run: it measures the relative error e of one congruence G X G^T of the
 * probe state X = W_t (Q if W_t = 0) against the FP64 congruence (from n = 512
 * the accurate mode's below), for every fixed operand G (E_t^T, S), and the
 * contraction rho of one step (the
 * product of ||E_t||_2^2 over the step's congruences, by power iteration;
 * 1 + t||S||^2 + t^2||S||^4/2 per S-flow), and keeps the first of 10, 13, 14
 * products whose estimate 4 e c (1 + rho + ... + rho^(horizon-1)) is within
 * tol (c congruences per step: every application's error adding up in phase,
 * damped only by the flow); 14 if none is.  dme_plan_split_choice and
 * dme_plan_split_probe report the choice and its inputs.  Above n = 511 the
 * Pade products of the exponential run on the tensor cores too, in an
 * accurate mode (21 slice products with the exact sums of 512-wide K chunks
 * combined in fp64); the denominator solves and the squarings stay FP64.
 * Errors: DME_EINVAL (inconsistent desc), DME_ENOTSPD (R), DME_ENOMEM,
 * DME_ECUDA.  On error *out is NULL. */
dme_status dme_plan(const dme_plan_desc* desc, const double* A, const double* QorC,
                    const double* B, const double* R, const double* S,
                    void* cuda_stream, dme_plan_t* out);

/* A plan for the generalised state-space DRE/DLE of Example 4 (§5.1.4),
 *     M^T P' M = A^T P M + M^T P A + Q - M^T P B R^{-1} B^T P M,
 * which, after cancelling M^T and M, is the standard equation with
 * A~ = A M^{-1} and Q~ = M^{-T} Q M^{-1} (the displayed equation of §5.1.4;
 * its A M^{-1} is taken literally).  A~ and Q~ are formed on the device with
 * an FP64 LU of M (n x n, invertible) and transposed solves; then the plan is
 * built as by dme_plan.  S must be NULL.  DME_EINVAL also for a singular M. */
dme_status dme_plan_mass(const dme_plan_desc* desc, const double* M, const double* A, const double* QorC,
                         const double* B, const double* R, const double* S, void* cuda_stream,
                         dme_plan_t* out);

/* Export E_t = e^{tA} and W_t = int_0^t e^{sA^T} Q e^{sA} ds (Eq. full),
 * computing and caching them if t is new.  E_out / W_out: n x n, host or
 * device, either may be NULL. */
dme_status dme_expm(dme_plan_t plan, double t, double* E_out, double* W_out);

/* Apply one sub-flow T_flow(t) in place to the symmetric n x n state P
 * (device memory).  The result is exactly symmetric. */
dme_status dme_apply(dme_plan_t plan, int flow, double t, double* P);

/* dme_apply without the final synchronisation: the sub-flow is only
 * enqueued on the plan's stream.  Device-side failures (DME_ENOTSPD) are
 * reported by the next dme_sync (or any synchronising call) on the plan. */
dme_status dme_apply_async(dme_plan_t plan, int flow, double t, double* P);

/* Wait for the plan's stream and report any device-side status raised since
 * the last synchronising call. */
dme_status dme_sync(dme_plan_t plan);

/* Advance P (device, n x n, symmetric) by nsteps steps of the plan's
 * composition with the plan's h, in place.  Steps are replayed from a CUDA
 * graph captured on first use for this P. */
dme_status dme_step(dme_plan_t plan, double* P, int nsteps);

/* dme_step without the final synchronisation: the nsteps graph replays are
 * only enqueued on the plan's stream (the first call for a new P captures the
 * graph, as dme_step does).  Device-side failures are reported by the next
 * dme_sync (or any synchronising call) on the plan. */
dme_status dme_step_async(dme_plan_t plan, double* P, int nsteps);

/* P_out = P_N, N = nsteps steps of size h = T/nsteps from P0 (§2).  If
 * T/nsteps differs from desc.h the missing E_t, W_t are built first.
 * P0, P_out: n x n, host or device; P_out may equal P0. */
dme_status dme_solve(dme_plan_t plan, const double* P0, double T, int nsteps, double* P_out);

/* LQR feedback gain K = R^{-1} B^T P (§1: the optimal input is
 * u(t) = -R^{-1} B^T P(T - t) x(t) when P solves the DRE with Q = C^T C).
 * P: n x n symmetric, device memory.  K_out: m x n row-major, host or device.
 * DME_EINVAL for a plan without B and R.  Synchronises the plan's stream. */
dme_status dme_gain(dme_plan_t plan, const double* P, double* K_out);

/* The split path's slice products per output (*pairs; 0 for DME_FP64) and the
 * estimate that chose them (*est = 4 N e of dme_plan, or a negative value when
 * pairs was given explicitly).  Either pointer may be NULL. */
dme_status dme_plan_split_choice(dme_plan_t plan, int* pairs, double* est);

/* What the choice of dme_plan_split_choice rests on (pairs = 0 and
 * DME_SPLIT_BF16 only, else DME_EINVAL): err[0..2] the measured relative
 * errors of one congruence with 10, 13 and 14 slice products (the plan tries
 * them in that order and stops at the first that meets the target, so the
 * ones after it read -1), *rho the contraction of one step.  Either pointer
 * may be NULL. */
dme_status dme_plan_split_probe(dme_plan_t plan, double* err, double* rho);

/* Bytes of device memory the plan holds. */
size_t dme_plan_bytes(dme_plan_t plan);

/* Kernel nodes in the CUDA graph of one step (captured by the last
 * dme_step / dme_solve), or -1 if no step has been captured yet. */
int dme_plan_kernels_per_step(dme_plan_t plan);

/* Kernel kinds for dme_plan_timing. */
enum { DME_KIND_SPLIT_GEMM = 0, DME_KIND_SLICE = 1, DME_KIND_FP64_GEMM = 2, DME_KIND_RICCATI = 3 };

/* Profiling mode (off by default): while enabled, the launches the plan
 * makes outside CUDA-graph replay (dme_apply, dme_apply_async, capture-free
 * work) are bracketed by CUDA events on the plan's stream, per kernel kind.
 * For DME_KIND_FP64_GEMM and DME_KIND_RICCATI one bracket covers the
 * launches of one congruence or one Riccati update. */
dme_status dme_plan_profile(dme_plan_t plan, int enable);

/* Synchronise the plan's stream, then return the milliseconds and bracket
 * count accumulated for `kind` since the last call, and reset them. */
dme_status dme_plan_timing(dme_plan_t plan, int kind, double* ms, int* launches);

dme_status dme_plan_destroy(dme_plan_t plan);

/* ---- low-rank factored path (§2.1-2.3 factor forms, Alg. 1-4) -----------
 * The state is kept as P = L diag(d) L^T (L n x r, d > 0) and never formed
 * during the steps: T1 maps L to E_t^T L, T2 appends C^T with weights t,
 * T12 maps L and appends the compressed Gauss-Legendre factor of W_t (Alg. 2),
 * T3 updates the factor through an m x m eigenproblem ((I + t D L^T B R^-1 B^T L)^-1 D
 * of §2.2 in square-root form), T4 appends sqrt(t) S L and sqrt(t/2) S (sqrt(t) S L)
 * (midpoint) or sqrt(t) S L (Euler).  After every flow that appends columns the
 * factor is compressed: the eigen-decomposition of P on the span of L (a Gram
 * matrix and a Jacobi eigensolver), keeping eigenvalues > tol * max.  E_t is
 * the dense exponential of the plan (n <= 16384; n <= 4096 with DME_SPLIT_BF16,
 * which runs the products with E_t and S on the tensor cores and the rest in
 * FP64).  P0 must be PSD. */
typedef struct dme_lr_s* dme_lr_t;
typedef struct {
    int quad_nodes;     /* Gauss-Legendre nodes for W_t in T12 (0: 7), <= 64       */
    int rmax;           /* column capacity before a compression (0: 224), <= 224  */
    double tol;         /* relative eigenvalue truncation (0: 1e-13)             */
} dme_lr_opts;

/* Plan: as dme_plan with q_is_factor = 1 (C is p x n, Q = C^T C), prec =
 * DME_FP64 or DME_SPLIT_BF16, fsal = 0, extrap <= 1.  opts may be NULL.
 * Errors as dme_plan. */
dme_status dme_lr_plan(const dme_plan_desc* desc, const double* A, const double* C, const double* B,
                       const double* R, const double* S, const dme_lr_opts* opts, void* cuda_stream,
                       dme_lr_t* out);

/* The factored path for a sparse A, which is never formed densely: A in CSR
 * (rowptr n + 1, colidx and vals nnz, 0-based, host or device, copied), C
 * (p x n) and, for a DRE / GDRE, B and R as in dme_plan.  e^{t A^T} L is applied by
 * Newton interpolation at Leja points (the action the paper computes with
 * `expleja`, §3): a Gershgorin interval [a, b] of A^T, A^T = c I + g X with
 * X's spectrum in [-2, 2], substeps of length t with t g <= 4, at most 80
 * Leja points per substep, and the series stopped after two terms below
 * 1e-15 times the partial sum (Frobenius norms).  For GDLE / GDRE, S (of the
 * S P S^T term, Eq. lyapGen; n x n) is given in CSR too (nnz_s, s_rowptr,
 * s_colidx, s_vals, same conventions and checks; ignored for DLE / DRE) and
 * T4 forms S L and S^2 L by a sparse product (§2.3).  desc: q_is_factor = 1,
 * prec = DME_FP64, flows among F1, F2, F12 (W_t by Gauss-Legendre quadrature,
 * each node's exponential again by Leja interpolation), F3 (DRE / GDRE) and
 * F4 (GDLE / GDRE).  n is not limited to 16384; dme_lr_solve's P_out must
 * then be NULL.  DME_EINVAL for a malformed CSR matrix (column index out of
 * range, rowptr not non-decreasing from 0 to nnz). */
dme_status dme_lr_plan_csr(const dme_plan_desc* desc, int nnz, const int* rowptr, const int* colidx,
                           const double* vals, const double* C, const double* B, const double* R, int nnz_s,
                           const int* s_rowptr, const int* s_colidx, const double* s_vals,
                           const dme_lr_opts* opts, void* cuda_stream, dme_lr_t* out);

/* N = nsteps composition steps from P0 = L0 D0 L0^T (L0 n x r0, D0 r0 x r0
 * symmetric PSD, host or device, row-major; r0 = 0 for P0 = 0), h = T/N.
 * P_out (n x n, host or device) receives L diag(d) L^T unless NULL; *r_out the
 * final rank unless NULL.  DME_ENOMEM if a factor outgrows rmax. */
dme_status dme_lr_solve(dme_lr_t plan, const double* L0, const double* D0, int r0, double T, int nsteps,
                        double* P_out, int* r_out);

/* The current factors: L_out (n x r, row-major) and d_out (r), either NULL to skip. */
dme_status dme_lr_factors(dme_lr_t plan, double* L_out, double* d_out, int* r);

dme_status dme_lr_destroy(dme_lr_t plan);

/* ---- serving: continuous batching of independent DRE/DLE solves ----------
 * A server owns one stream and a worker thread.  Requests are admitted into
 * slots while their device footprint (P, E, W and work buffers) fits in
 * hbm_budget_bytes and a slot is free; every resident request advances one
 * composition step per scheduler round through grouped kernels covering all
 * resident requests, so newly admitted requests overlap with running ones. */
dme_status dme_server_create(size_t hbm_budget_bytes, int max_slots, dme_server_t* out);

/* Queue one solve of nsteps steps over [0, T] (h = T/nsteps; desc->h is
 * ignored).  All pointers are host memory and are copied before return.
 * *ticket identifies the request for dme_poll.  DME_EBUSY if the queue is full;
 * DME_ENOMEM if the request alone exceeds the budget. */
dme_status dme_submit(dme_server_t srv, const dme_plan_desc* desc, const double* A,
                      const double* QorC, const double* B, const double* R,
                      const double* S, const double* P0, double T, int nsteps,
                      uint64_t* ticket);

/* Wait up to timeout_us (0: do not wait, < 0: forever) for a request; on
 * completion copy P(T) into P_out (host, n x n, may be NULL) and release the
 * ticket.  DME_ENOTREADY (timeout 0) / DME_ETIMEOUT if still running; the
 * request's own error status (e.g. DME_ENOTSPD) once it has failed. */
dme_status dme_poll(dme_server_t srv, uint64_t ticket, double* P_out, int64_t timeout_us);

/* As dme_submit for a DRE, and the LQR feedback gains along the solve (§1: the
 * optimal input is u = -R^{-1} B^T P(T - t) x): after every step k = 1..nsteps
 * the server forms K_k = R^{-1} B^T P_k (m x n) on the device.  DME_EINVAL
 * unless desc is a DRE/GDRE. */
dme_status dme_submit_gain(dme_server_t server, const dme_plan_desc* desc, const double* A, const double* QorC,
                           const double* B, const double* R, const double* S, const double* P0, double T,
                           int nsteps, uint64_t* ticket);

/* As dme_poll, and K_out (host, nsteps x m x n, row-major, step-major) receives
 * the gains of a request submitted with dme_submit_gain (DME_EINVAL for another
 * request; either output may be NULL). */
dme_status dme_poll_gain(dme_server_t server, uint64_t ticket, double* P_out, double* K_out, int64_t timeout_us);

/* Server statistics as a JSON object (completed, failed, resident, queued,
 * p50/p99 latency in ms, solves/s, rounds, round-graph builds and their host
 * time, the stepper's time blocked on its round batches, plans and their mean
 * time); the string stays valid until the next call. */
const char* dme_server_stats(dme_server_t srv);

dme_status dme_server_destroy(dme_server_t srv);

/* C = A B^T on the split-precision tensor-core path used by DME_SPLIT_BF16:
 * every row of A (M x K) and of B (N x K) is scaled by a power of two, rounded
 * to a fixed-point integer and cut into bf16 digits (a leading digit |d| <= 64,
 * then 9-bit digits |d| <= 256; five slices for A, four for B); the 14 slice
 * products of levels 0..4 are accumulated in fp32 on tcgen05 tensor cores,
 * exactly for level 0 (K <= 4096 keeps every partial sum below 2^24 units),
 * and combined in fp64.  Entry errors are ~2^-34 of the B row scale times the
 * A row scale (times sqrt(K) for random signs).  All matrices are float64
 * row-major device memory; C is M x N.  Synchronises `cuda_stream`.
 * DME_EINVAL unless 1 <= K <= 4096. */
dme_status dme_gemm_split(int M, int N, int K, const double* A, const double* B, double* C,
                          void* cuda_stream);

/* C = A B^T in the accurate split mode the plan uses for the products of the
 * Pade approximant (Eq. full): six bf16 slices of 7-bit digits per row of A
 * and of B (rows rounded at 2^-42 of their scale), the 21 slice products of
 * levels 0..5, K taken in chunks of 512 in which the fp32 sums of levels 0, 1
 * and 2 are exact, the chunk results added in fp64.  Entry errors are ~2^-39
 * of the row scales' product (times sqrt(K)).  Same arguments, layout and
 * errors as dme_gemm_split; synchronises `cuda_stream`. */
dme_status dme_gemm_split_acc(int M, int N, int K, const double* A, const double* B, double* C, void* cuda_stream);

/* B <- M^{-1} B for a dense n x n M and an n x nrhs B (float64, row-major,
 * host or device memory; M is copied and left unchanged): Gauss-Jordan
 * elimination with partial pivoting (largest |entry| of the column, the
 * smallest row on ties), blocked by panels of 16 columns whose trailing
 * update is one pass over the remaining columns (n <= 4096: three launches
 * per panel, the panel factored by a thread-block cluster; larger n: one
 * cooperative launch with 18 grid barriers per panel), the kernels of the
 * plan's Pade step (the denominator systems
 * q R = p of the [13/13] approximant, Eq. full) and of dme_plan_mass.
 * Synchronises `cuda_stream` (NULL: a stream of its own).  DME_EINVAL if
 * n < 1, nrhs < 0, a pointer is NULL, or a pivot column is zero or not finite
 * (M singular; B is then undefined). */
dme_status dme_dense_solve(const double* M, int n, double* B, int nrhs, void* cuda_stream);

/* Self-test of the library's bounded device waits: one GPU block waits at a
 * grid barrier whose release word nothing ever writes, using the same wait as
 * the persistent kernels (a poll limit, then DEV_TIMEOUT in a status word and
 * return).  *timed_out = 1 when the wait gave up and reported it (takes about
 * a second); the context stays usable.  DME_EINVAL if timed_out is NULL. */
dme_status dme_wait_selftest(int* timed_out);

/* dme_gemm_split without any device allocation, for callers that cannot
 * call cudaMalloc: code whose device memory is owned by a host application's
 * own allocator, or loops that must not pay cudaMalloc's implicit device
 * synchronisation.  The paper has no counterpart; it is a library service.
 * Same arguments, arithmetic and results as dme_gemm_split (A, B, C float64
 * row-major device memory, C = A B^T, 1 <= K <= 4096).  Its scratch is an
 * 8 MiB array in the library's device memory, held by every device that
 * loads the library until the process exits:
 *   (5 M + 4 N) * roundup(K, 32) * 2 bytes of slices plus the row scales must
 *   fit in it (e.g. M = N = K = 640), otherwise DME_EINVAL with the sizes.
 * The first call on a device looks up that array's device address (with the
 * device current) and caches it for the life of the process; make that first
 * call before any stream capture.  After a cudaDeviceReset the cached address
 * no longer names the array, so this entry point must not be used across a
 * device reset.  Every call shares the one array and finds the previous call's
 * contents there: calls on the same device that overlap on the GPU (two
 * streams, or two host threads) race and must be serialised by the caller.
 * Each call enqueues its work on `cuda_stream` (NULL: the legacy default
 * stream), then waits for that stream to finish before it returns, to read the
 * kernel's status word. */
dme_status dme_gemm_split_noalloc(int M, int N, int K, const double* A, const double* B, double* C,
                                  void* cuda_stream);

/* Message of the last failed call on this thread ("" if none). */
const char* dme_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DME_H */
