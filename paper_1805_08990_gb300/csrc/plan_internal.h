// Plan internals shared by plan.cu and server.cu (not part of the C ABI).
#pragma once

#include <vector>

#include "dme_internal.h"
#include "split_internal.h"

using dme::SliceBuf;
using dme::GemmProb;

struct EWEntry {
    double tau;
    double* E;
    double* W;
    int s;
    SliceBuf Gsl;   // split path: slices of E^T (rows of E^T = columns of E)
};

enum OpKind { OP_CONG = 0, OP_AXPY = 1, OP_RICC = 2, OP_SFLOW = 3, OP_COPY = 4, OP_COMBINE = 5 };

// States an op acts on: the caller's P, and the two extra states of the
// extrapolated scheme (accumulator and work copy).
enum { BUF_P = 0, BUF_ACC = 1, BUF_WORK = 2 };

struct Op {
    int kind;
    double tau;
    int ew;        // OP_CONG: index of (E, W)
    double wcoef;  // OP_CONG: coefficient of W (1 for T12, 0 for T1)
    double qcoef;  // fused T2: + qcoef Q
    int rule;      // OP_SFLOW: DME_T4_MIDPOINT / DME_T4_EULER
    int buf;       // state the op updates (BUF_*)
    int src;       // OP_COPY: buf <- src.  OP_COMBINE: buf <- c1 buf + c2 src (src < 0: none)
    double c1, c2;
};

// An instantiated CUDA graph of one op list, valid for one state pointer.
struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
    double* P = nullptr;
    int kernels = -1;
};

struct dme_plan_s {
    dme_plan_desc d;
    int n = 0, m = 0;
    cudaStream_t st = nullptr;
    bool own_st = false;
    double* A = nullptr;
    double* Q = nullptr;
    double* Bt = nullptr;
    double* LR = nullptr;      // Cholesky factor of R (m x m, lower)
    double* Kbuf = nullptr;    // m x n LQR gain (allocated on first dme_gain)
    double* S = nullptr;
    double* X = nullptr;       // n x n congruence intermediate
    double* Xs = nullptr;      // n x n S-flow intermediates
    double* Y1 = nullptr;
    double* state = nullptr;   // n x n, dme_solve working state
    double* rwork = nullptr;   // Riccati work
    double* small = nullptr;   // 2n colsums + scalars
    int* status = nullptr;
    double normM = 0.0;
    std::vector<EWEntry> ew;
    std::vector<Op> ops;                          // one step
    std::vector<Op> ops_head, ops_body, ops_tail; // fsal: first, interior and closing parts
    double ops_h = -1.0;
    double* xacc = nullptr;    // extrapolated scheme: accumulator state (n x n)
    double* xwork = nullptr;   // extrapolated scheme with q >= 3: work state (n x n)
    std::vector<void*> allocs;
    size_t bytes = 0;
    GraphSlot g_step, g_head, g_body, g_tail;
    bool split = false;
    int cfg = 2;               // split path: slice-pair configuration (dme::OzCfgId, OZ_P14 by default)
    double cfg_est = -1.0;     // split path: the estimate that chose cfg (< 0: given explicitly)
    double cfg_err[3] = {-1.0, -1.0, -1.0};   // measured one-application errors of P10, P13, P14
    double cfg_rho = 1.0;      // the step's contraction used by the estimate
    SliceBuf psl, usl, Ssl;    // split path: slices of P, of U = G P, and of S
    float2* U = nullptr;       // split path: G P as normalised (hi, lo) pairs
    float2* kws = nullptr;     // split path: split-K workspace of the tail tiles
    int* kcnt = nullptr;       // split path: split-K arrival counters
    // split path with n > 1536 and T3: the Riccati products on the tensor cores
    bool tric = false;
    SliceBuf btsl;             // slices of Bt^T (m rows, 5 slices)
    SliceBuf ysla, yslb;       // slices of Y (n rows, k = m) as A (5) and B (4) operand
    double* Zt = nullptr;      // Z^T = Bt^T P (m x n)
    // profiling: CUDA-event pairs around launches made outside graph capture
    bool prof = false;
    std::vector<cudaEvent_t> evpool;
    struct EvRec {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<EvRec> evrec;
};


namespace dme {

// Build a plan (validated descriptor; pointers host or device).  A serving plan
// (grouped launches, which never split K: at the server's loads splitting only adds
// units and tail work to launches that are already full) holds no split-K workspace.
dme_status plan_create(const dme_plan_desc* d, const double* A, const double* QorC, const double* B,
                       const double* R, const double* S, void* stream, dme_plan_t* out, bool serving = false);
// Free a plan and everything it owns (synchronises its stream).
void free_plan(dme_plan_t p);
// Compile one step of size h into p->ops (computes missing E_t, W_t).
dme_status build_ops(dme_plan_t p, double h);
// Enqueue one op on the plan's stream.
dme_status run_op(dme_plan_t p, const Op& o, double* P);
// Bytes reserved while a plan of this descriptor is built (persistent + transient).
size_t plan_estimate_bytes(const dme_plan_desc& d, bool serving = false);
// E_t, W_t of the plan for step t (computed and cached on first use): index into p->ew.
dme_status plan_ew(dme_plan_t p, double t, int* idx);
// Report (and clear) the plan's device status word after synchronising its stream.
dme_status plan_check(dme_plan_t p, const char* where);
// The descriptor and pointer checks of dme_plan.
dme_status plan_validate(const dme_plan_desc* d, const double* A, const double* QorC, const double* B,
                         const double* R, const double* S);
// One composition step of size h as (flow, t) pairs in application order.
std::vector<std::pair<int, double>> plan_step_sequence(const dme_plan_desc& d, double h);

}  // namespace dme
