// Serving: continuous batching of independent DLE/DRE solves on one GPU.
//
// Host threads share a request table under one mutex:
//  * admission threads (kAdmitThreads of them) take queued requests while a
//    slot is free and the request's device footprint fits in the HBM budget,
//    and build their plans (problem data, Q, Bt, E_t, W_t) each on the plan's
//    own stream, so plans overlap one another and the stepping on the GPU (a
//    small plan is bound by launch latency, not by the GPU's throughput);
//  * the stepper thread owns the resident requests and runs scheduler rounds:
//    each round advances every resident request by one composition step.  The
//    ops of all residents are executed stage by stage with grouped kernels:
//    one grouped GEMM launch per congruence phase (FP64: P E, then E^T X with
//    the W/tQ epilogue; split precision: the tcgen05 slice GEMMs G P and G U^T
//    with the slicing of P and U in between) and one grouped launch per
//    Riccati kernel, covering all residents at that stage.  Requests admitted between rounds join the next
//    round; finished ones leave after it.
// A round is captured once into a CUDA graph for a given set of residents (its
// launch descriptors staged in one device arena) and replayed until the set
// changes; between host checks the stepper replays several rounds back to back
// when no resident finishes and nobody waits for admission.  The FP64 grouped
// GEMM's output tile (32 or 64) is chosen per group size by an online
// autotuner that times both variants on the group's first P E product (which
// only writes scratch); both tiles give bit-identical results.
// Grouped kernels compute each problem's tiles exactly as they would alone
// (no cross-request reduction), so a result is bit-identical alone or in a mix.
// Latency is measured from dme_submit to the end of the round that finished it.
#include "plan_internal.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

using namespace dme;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum ReqState { Q_QUEUED = 0, Q_PLANNING = 1, Q_RESIDENT = 2, Q_DONE = 3 };

struct Req {
    uint64_t id = 0;
    dme_plan_desc desc;
    std::vector<double> A, QC, B, R, S, P0;
    double T = 0;
    int nsteps = 0;
    int state = Q_QUEUED;
    dme_plan_t plan = nullptr;
    double* P = nullptr;
    int slot = -1;
    int done_steps = 0;
    size_t reserved = 0;
    std::vector<double> out;
    bool gain = false;              // record K_k = R^{-1} B^T P_k after every step
    double* Kh = nullptr;           // gain history on the device (nsteps x m x n)
    int* kctr = nullptr;            // steps recorded so far (device)
    std::vector<double> kout;
    dme_status status = DME_OK;
    std::string err;
    double t_submit = 0, t_done = 0;
};

}  // namespace

constexpr int kLanes = 2;   // concurrent lanes of a round

struct dme_server_s {
    size_t budget = 0;
    int max_slots = 0;
    size_t queue_cap = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req*> queue;
    std::vector<Req*> ready;      // planned, waiting for the next round
    std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
    std::vector<int> free_slots;
    size_t reserved = 0;
    uint64_t next_id = 1;
    bool stop = false;
    std::vector<std::thread> admit_thrs;
    std::thread step_thr;
    cudaStream_t st = nullptr;
    // a round runs its residents in kLanes lanes (each its own chain of stages, forked
    // from and joined to st); in a lane the 14-product group's split GEMMs run on the lane's
    // second stream beside the 10/13 group's
    cudaStream_t lane_st[kLanes] = {}, lane_st2[kLanes] = {};
    cudaEvent_t ev_split = nullptr, ev_done[kLanes] = {};
    cudaEvent_t ev_fork[kLanes] = {}, ev_join[kLanes] = {};
    int* dstat = nullptr;         // per-slot device status words
    DescArena arena;              // launch descriptors of the captured round
    GemmProb* tune_desc = nullptr;  // autotuner's descriptor buffer (max_slots)
    cudaGraphExec_t round_exec = nullptr;
    std::vector<uint64_t> round_ids;   // ids of the residents the captured round serves, in order
                                       // (ids, not addresses: a new request may reuse a freed Req's address)
    std::map<int, int> tile_choice;    // autotuner: ceil(log2(64-tiles of a group)) -> tile 32 / 64
    std::vector<double> lat_ms;
    int completed = 0, failed = 0, tuned = 0;
    std::atomic<int> rounds{0}, graph_builds{0};   // written by the stepper, read by dme_server_stats
    double build_s = 0.0;   // host time spent building round graphs (stepper thread; under mu)
    double wait_s = 0.0;    // stepper time blocked on the round batches' completion (under mu)
    double plan_s = 0.0;    // wall time of the admission threads' plan builds, summed (under mu)
    int planned = 0;
    int pairs_hist[3] = {0, 0, 0};   // split plans by slice products chosen: 10, 13, 14 (under mu)
    double t_first = -1, t_last = 0;
    std::string stats;
};

namespace {

void finish(dme_server_t s, Req* r, dme_status st, const std::string& err) {
    // called with s->mu held
    r->status = st;
    r->err = err;
    r->state = Q_DONE;
    r->t_done = now_s();
    if (st == DME_OK) {
        s->completed++;
        s->lat_ms.push_back(1e3 * (r->t_done - r->t_submit));
    } else {
        s->failed++;
    }
    s->t_last = r->t_done;
    s->cv.notify_all();
}

void release(dme_server_t s, Req* r) {
    if (r->P && r->plan) cudaFreeAsync(r->P, r->plan->st);
    r->P = nullptr;
    if (r->Kh && r->plan) cudaFreeAsync(r->Kh, r->plan->st);
    if (r->kctr && r->plan) cudaFreeAsync(r->kctr, r->plan->st);
    r->Kh = nullptr;
    r->kctr = nullptr;
    if (r->plan) free_plan(r->plan);
    r->plan = nullptr;
    std::lock_guard<std::mutex> g(s->mu);
    s->reserved -= r->reserved;
    r->reserved = 0;
    if (r->slot >= 0) s->free_slots.push_back(r->slot);
    r->slot = -1;
    s->cv.notify_all();
}

constexpr int kAdmitThreads = 4;

void admit_loop(dme_server_t s) {
    for (;;) {
        Req* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] {
                if (s->stop) return true;
                if (s->queue.empty() || s->free_slots.empty()) return false;
                return s->reserved + plan_estimate_bytes(s->queue.front()->desc, true) <= s->budget;
            });
            if (s->stop) return;
            r = s->queue.front();
            s->queue.pop_front();
            r->state = Q_PLANNING;
            r->slot = s->free_slots.back();
            s->free_slots.pop_back();
            r->reserved = plan_estimate_bytes(r->desc, true);
            s->reserved += r->reserved;
        }
        set_error("");
        dme_plan_t p = nullptr;
        const double* Bp = r->B.empty() ? nullptr : r->B.data();
        const double* Rp = r->R.empty() ? nullptr : r->R.data();
        const double* Sp = r->S.empty() ? nullptr : r->S.data();
        const double tp0 = now_s();
        dme_status st = plan_create(&r->desc, r->A.data(), r->QC.data(), Bp, Rp, Sp, nullptr, &p, true);
        const double tp1 = now_s();
        const size_t nn = (size_t)r->desc.n * r->desc.n;
        if (st == DME_OK) {
            r->plan = p;
            cudaError_t e = cudaMallocAsync(&r->P, nn * sizeof(double), p->st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(r->P, r->P0.data(), nn * sizeof(double), cudaMemcpyHostToDevice, p->st);
            if (e == cudaSuccess && r->gain) {
                const size_t kn = (size_t)r->nsteps * r->desc.m * r->desc.n;
                e = cudaMallocAsync(&r->Kh, kn * sizeof(double), p->st);
                if (e == cudaSuccess) e = cudaMallocAsync(&r->kctr, sizeof(int), p->st);
                if (e == cudaSuccess) e = cudaMemsetAsync(r->kctr, 0, sizeof(int), p->st);
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
            if (e != cudaSuccess) {
                cudaGetLastError();
                st = DME_ENOMEM;
                set_error(std::string("serving: ") + cudaGetErrorString(e));
            }
        }
        std::string err = get_error();
        if (st != DME_OK) {
            release(s, r);
            std::lock_guard<std::mutex> g(s->mu);
            finish(s, r, st, err);
            continue;
        }
        // free the input copies; keep the measured footprint
        std::vector<double>().swap(r->A);
        std::vector<double>().swap(r->QC);
        std::vector<double>().swap(r->P0);
        std::lock_guard<std::mutex> g(s->mu);
        s->plan_s += tp1 - tp0;
        s->planned++;
        if (p->split) s->pairs_hist[p->cfg == OZ_P10 ? 0 : (p->cfg == OZ_P13 ? 1 : 2)]++;
        const size_t actual = p->bytes + nn * sizeof(double) +
                              (r->gain ? (size_t)r->nsteps * r->desc.m * r->desc.n * sizeof(double) : 0);
        s->reserved = s->reserved - r->reserved + actual;
        r->reserved = actual;
        r->state = Q_RESIDENT;
        s->ready.push_back(r);
        s->cv.notify_all();
    }
}

// Stage-by-stage work lists of one round.
struct StageLists {
    std::vector<GemmProb> g1, g2;
    std::vector<RicItem> ric;
    std::vector<Req*> sc;       // split-precision congruences
    std::vector<Req*> axpy;     // standalone T2
};

dme_status stage_lists(dme_server_t s, std::vector<Req*>& res, size_t k, StageLists& L) {
    for (Req* r : res) {
        if (k >= r->plan->ops.size()) continue;
        const Op& o = r->plan->ops[k];
        dme_plan_t p = r->plan;
        const int n = p->n;
        if (o.kind == OP_CONG && p->split) {
            L.sc.push_back(r);
        } else if (o.kind == OP_CONG) {
            const EWEntry& e = p->ew[o.ew];
            GemmProb a;
            std::memset(&a, 0, sizeof(a));
            a.A = r->P;
            a.B = e.E;
            a.C = p->X;
            a.M = a.N = a.K = n;
            a.lda = a.ldb = a.ldc = a.ldd = n;
            a.alpha = 1.0;
            L.g1.push_back(a);
            GemmProb b;
            std::memset(&b, 0, sizeof(b));
            b.A = e.E;
            b.transA = 1;
            b.B = p->X;
            b.C = r->P;
            b.M = b.N = b.K = n;
            b.lda = b.ldb = b.ldc = b.ldd = n;
            b.alpha = 1.0;
            b.tri = 1;
            if (o.wcoef != 0.0) {
                b.D1 = e.W;
                b.b1 = o.wcoef;
            }
            if (o.qcoef != 0.0) {
                b.D2 = p->Q;
                b.b2 = o.qcoef;
            }
            L.g2.push_back(b);
        } else if (o.kind == OP_RICC) {
            L.ric.push_back(make_ric_item(r->P, p->Bt, n, p->m, o.tau, o.qcoef != 0.0 ? p->Q : nullptr, o.qcoef,
                                          p->rwork, s->dstat + r->slot));
        } else if (o.kind == OP_AXPY) {
            L.axpy.push_back(r);
        } else {
            set_error("serving: unsupported op");
            return DME_EINVAL;
        }
    }
    return DME_OK;
}

size_t round_stages(const std::vector<Req*>& res) {
    size_t stages = 0;
    for (Req* r : res) stages = std::max(stages, r->plan->ops.size());
    return stages;
}

int tile_key(const std::vector<GemmProb>& g) {
    long tiles = 0;
    for (auto& p : g) tiles += (long)((p.M + 63) / 64) * ((p.N + 63) / 64);
    int key = 0;
    while ((1L << key) < tiles) ++key;
    return key;
}

// Autotuner: for every FP64 group size class not seen before, time the grouped
// P E product (it writes only each plan's scratch X) with 32- and 64-wide tiles
// and keep the faster.  Runs eagerly, before the round is captured.
dme_status tune_tiles(dme_server_t s, std::vector<Req*>& res) {
    const size_t stages = round_stages(res);
    for (size_t k = 0; k < stages; ++k) {
        StageLists L;
        DME_TRY(stage_lists(s, res, k, L));
        if (L.g1.empty()) continue;
        const int key = tile_key(L.g1);
        if (s->tile_choice.count(key)) continue;
        cudaEvent_t a = nullptr, b = nullptr;
        DME_CUDA_TRY(cudaEventCreate(&a));
        DME_CUDA_TRY(cudaEventCreate(&b));
        int best = 64;
        float best_ms = 0.0f;
        dme_status st = DME_OK;
        for (int tile : {64, 32}) {
            std::vector<GemmProb> g = L.g1;
            st = gemm64_grouped(g, s->tune_desc, s->st, nullptr, tile);   // warm-up
            float ms = 0.0f;
            for (int rep = 0; rep < 3 && st == DME_OK; ++rep) {
                g = L.g1;
                cudaEventRecord(a, s->st);
                st = gemm64_grouped(g, s->tune_desc, s->st, nullptr, tile);
                cudaEventRecord(b, s->st);
                cudaEventSynchronize(b);
                float t = 0.0f;
                cudaEventElapsedTime(&t, a, b);
                ms = (rep == 0) ? t : std::min(ms, t);
            }
            if (st != DME_OK) break;
            if (tile == 64 || ms < best_ms) {
                best_ms = ms;
                best = tile;
            }
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        DME_TRY(st);
        DME_CUDA_TRY(cudaStreamSynchronize(s->st));
        std::lock_guard<std::mutex> g(s->mu);   // dme_server_stats reads the map
        s->tile_choice[key] = best;
        s->tuned++;
    }
    return DME_OK;
}

void destroy_streams(dme_server_t s) {
    for (int l = 0; l < kLanes; ++l) {
        for (cudaEvent_t ev : {s->ev_done[l], s->ev_fork[l], s->ev_join[l]})
            if (ev) cudaEventDestroy(ev);
        if (s->lane_st[l]) cudaStreamDestroy(s->lane_st[l]);
        if (s->lane_st2[l]) cudaStreamDestroy(s->lane_st2[l]);
    }
    if (s->ev_split) cudaEventDestroy(s->ev_split);
    if (s->st) cudaStreamDestroy(s->st);
}

// The split GEMMs of one stage: the group of 10/13-product plans on the serving stream and,
// when both groups are present, the 14-product group on the second stream at the same time
// (independent problems; the persistent kernels share the SMs neither fills), joined before
// the next stage.
dme_status launch_split_groups(dme_server_t s, int lane, std::vector<OzGroupDesc> (&g)[2]) {
    cudaStream_t st = s->lane_st[lane], st2 = s->lane_st2[lane];
    if (g[0].empty() || g[1].empty()) {
        for (auto& x : g)
            if (!x.empty()) DME_TRY(launch_ozaki_grouped(x, nullptr, st, &s->arena));
        return DME_OK;
    }
    DME_CUDA_TRY(cudaEventRecord(s->ev_fork[lane], st));
    DME_CUDA_TRY(cudaStreamWaitEvent(st2, s->ev_fork[lane], 0));
    DME_TRY(launch_ozaki_grouped(g[1], nullptr, st2, &s->arena));
    DME_TRY(launch_ozaki_grouped(g[0], nullptr, st, &s->arena));
    DME_CUDA_TRY(cudaEventRecord(s->ev_join[lane], st2));
    DME_CUDA_TRY(cudaStreamWaitEvent(st, s->ev_join[lane], 0));
    return DME_OK;
}

// Enqueue one scheduler round over the residents: stage by stage, grouped
// launches, descriptors staged in the arena (no host synchronisation: the
// sequence is captured into a graph).
dme_status run_lane(dme_server_t s, std::vector<Req*>& res, int lane) {
    cudaStream_t st = s->lane_st[lane];
    const size_t stages = round_stages(res);
    for (size_t k = 0; k < stages; ++k) {
        StageLists L;
        DME_TRY(stage_lists(s, res, k, L));
        for (Req* r : L.axpy) {
            const Op& o = r->plan->ops[k];
            launch_axpy_sym(r->P, r->plan->Q, o.qcoef, r->plan->n, r->plan->n, st);
        }
        if (!L.g1.empty()) {
            auto it = s->tile_choice.find(tile_key(L.g1));
            const int tile = it == s->tile_choice.end() ? 64 : it->second;
            DME_TRY(gemm64_grouped(L.g1, nullptr, st, &s->arena, tile));
            DME_TRY(gemm64_grouped(L.g2, nullptr, st, &s->arena, tile));
        }
        if (!L.sc.empty()) {
            // the split congruence G P G^T of every request: slice P, grouped U = G P,
            // slice U, grouped G U^T (upper tiles, FP64 + W / tQ, mirrored)
            std::vector<SliceDesc> s1, s2;
            for (Req* r : L.sc) {
                dme_plan_t p = r->plan;
                const int n = p->n;
                SliceDesc a;
                std::memset(&a, 0, sizeof(a));
                a.X = r->P;
                a.rows = n;
                a.cols = n;
                a.ldx = n;
                a.out = p->psl.data;
                a.Kp = p->psl.Kp;
                a.ns = p->psl.ns;
                a.prow = p->psl.rows;
                a.scale = p->psl.scale;
                s1.push_back(a);
                SliceDesc b = a;
                b.X = nullptr;
                b.Xp = p->U;
                b.out = p->usl.data;
                b.Kp = p->usl.Kp;
                b.ns = p->usl.ns;
                b.prow = p->usl.rows;
                b.scale = p->usl.scale;
                s2.push_back(b);
            }
            DME_TRY(launch_slice_grouped(s1, false, st, &s->arena));
            // one grouped launch for the plans of 10 or 13 slice products (4 x 4 slices), one for
            // those of 14 (each plan chose its own)
            std::vector<OzGroupDesc> o1c[2], o2c[2];
            for (Req* r : L.sc) {
                dme_plan_t p = r->plan;
                const Op& o = p->ops[k];
                const EWEntry& e = p->ew[o.ew];
                const int n = p->n;
                OzGroupDesc a;
                std::memset(&a, 0, sizeof(a));
                a.tmA = oz_tmap_a(e.Gsl, p->cfg);
                a.tmB = oz_tmap_b(p->psl, p->cfg);
                DME_TRY(oz_params(e.Gsl, p->psl, p->cfg, &a.p));
                a.p.mode = OZ_OUT_PAIR;
                a.p.ldc = n;
                a.p.Cp = p->U;
                a.p.status = s->dstat + r->slot;

                o1c[p->cfg == OZ_P14].push_back(a);
                OzGroupDesc b;
                std::memset(&b, 0, sizeof(b));
                b.tmA = oz_tmap_a(e.Gsl, p->cfg);
                b.tmB = oz_tmap_b(p->usl, p->cfg);
                DME_TRY(oz_params(e.Gsl, p->usl, p->cfg, &b.p));
                b.p.mode = OZ_OUT_F64;
                b.p.tri = 1;
                b.p.ldc = n;
                b.p.Cd = r->P;
                b.p.alpha = 1.0;
                if (o.wcoef != 0.0) {
                    b.p.D1 = e.W;
                    b.p.b1 = o.wcoef;
                }
                if (o.qcoef != 0.0) {
                    b.p.D2 = p->Q;
                    b.p.b2 = o.qcoef;
                }
                b.p.status = s->dstat + r->slot;
                o2c[p->cfg == OZ_P14].push_back(b);
                (void)n;
            }
            DME_TRY(launch_split_groups(s, lane, o1c));
            DME_TRY(launch_slice_grouped(s2, true, st, &s->arena));
            DME_TRY(launch_split_groups(s, lane, o2c));
        }
        if (!L.ric.empty()) DME_TRY(launch_riccati_grouped(L.ric, nullptr, st, &s->arena));
    }
    // after the step: the gain of every request that records it (the launches read
    // the device step counter, so the captured round stays valid for every replay)
    for (Req* r : res)
        if (r->gain)
            DME_TRY(launch_lqr_gain_hist(r->P, r->plan->Bt, r->plan->LR, r->plan->n, r->plan->m, r->plan->rwork,
                                         r->Kh, r->kctr, r->nsteps, st));
    DME_CUDA_TRY(cudaGetLastError());
    return DME_OK;
}

// One round: the residents in kLanes lanes of about equal work (largest first, each to the
// lightest lane), each lane its own chain of stages on its own stream, forked from the
// serving stream and joined back; so one lane's slicing and Riccati stages overlap the
// other's GEMMs.  A request's arithmetic does not depend on its lane or group.
dme_status run_round(dme_server_t s, std::vector<Req*>& res) {
    std::vector<Req*> order(res);
    std::stable_sort(order.begin(), order.end(), [](const Req* x, const Req* y) { return x->plan->n > y->plan->n; });
    std::vector<Req*> part[kLanes];
    double w[kLanes] = {};
    for (Req* r : order) {
        const double n = r->plan->n;
        int l = 0;
        for (int q = 1; q < kLanes; ++q)
            if (w[q] < w[l]) l = q;
        part[l].push_back(r);
        w[l] += n * n * n;
    }
    DME_CUDA_TRY(cudaEventRecord(s->ev_split, s->st));
    for (int l = 0; l < kLanes; ++l) {
        DME_CUDA_TRY(cudaStreamWaitEvent(s->lane_st[l], s->ev_split, 0));
        if (!part[l].empty()) DME_TRY(run_lane(s, part[l], l));
        DME_CUDA_TRY(cudaEventRecord(s->ev_done[l], s->lane_st[l]));
    }
    for (int l = 0; l < kLanes; ++l) DME_CUDA_TRY(cudaStreamWaitEvent(s->st, s->ev_done[l], 0));
    return DME_OK;
}

// (Re)capture the round for the current residents and upload its descriptors.
dme_status build_round_graph(dme_server_t s, std::vector<Req*>& res) {
    DME_CUDA_TRY(cudaStreamSynchronize(s->st));
    if (s->round_exec) {
        cudaGraphExecDestroy(s->round_exec);
        s->round_exec = nullptr;
    }
    s->round_ids.clear();
    DME_TRY(tune_tiles(s, res));
    s->arena.host.clear();
    cudaGraph_t g = nullptr;
    DME_CUDA_TRY(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
    dme_status st = run_round(s, res);
    cudaError_t e = cudaStreamEndCapture(s->st, &g);
    if (st != DME_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return set_error(std::string("serving: graph capture: ") + cudaGetErrorString(e)), DME_ECUDA;
    e = cudaGraphInstantiate(&s->round_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return set_error(std::string("serving: graph instantiate: ") + cudaGetErrorString(e)), DME_ECUDA;
    // on the serving stream: the round's launches are ordered after the upload (a plain
    // cudaMemcpy from pageable memory may return before its DMA lands, and the serving
    // stream does not wait for the legacy stream it runs on)
    if (!s->arena.host.empty()) {
        DME_CUDA_TRY(cudaMemcpyAsync(s->arena.dev, s->arena.host.data(), s->arena.host.size(),
                                     cudaMemcpyHostToDevice, s->st));
        DME_CUDA_TRY(cudaStreamSynchronize(s->st));
    }
    for (Req* r : res) s->round_ids.push_back(r->id);
    s->graph_builds++;
    return DME_OK;
}

constexpr int kMaxRoundsPerCheck = 16;

void step_loop(dme_server_t s) {
    std::vector<Req*> res;
    std::vector<int> hstat(s->max_slots);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] { return s->stop || !s->ready.empty() || !res.empty(); });
            if (s->stop) return;
            for (Req* r : s->ready) res.push_back(r);
            s->ready.clear();
        }
        dme_status st = DME_OK;
        bool same = s->round_exec != nullptr && s->round_ids.size() == res.size();
        for (size_t i = 0; same && i < res.size(); ++i) same = s->round_ids[i] == res[i]->id;
        if (!same) {
            const double t0 = now_s();
            st = build_round_graph(s, res);
            std::lock_guard<std::mutex> g(s->mu);
            s->build_s += now_s() - t0;
        }
        // rounds before the next host check: none of the residents finishes
        // earlier, and one round only while a planned request waits to join (a
        // queued one can only be admitted when a slot frees, which the first
        // rule catches, or is being planned, which takes longer than a round)
        int R = kMaxRoundsPerCheck;
        for (Req* r : res) R = std::min(R, r->nsteps - r->done_steps);
        {
            std::lock_guard<std::mutex> g(s->mu);
            if (!s->ready.empty()) R = 1;
        }
        R = std::max(R, 1);
        for (int i = 0; i < R && st == DME_OK; ++i) {
            cudaError_t e = cudaGraphLaunch(s->round_exec, s->st);
            if (e != cudaSuccess) {
                st = DME_ECUDA;
                set_error(std::string("serving: graph launch: ") + cudaGetErrorString(e));
            }
        }
        std::string err = get_error();
        if (st == DME_OK) {
            const double tw = now_s();
            cudaError_t e = cudaMemcpyAsync(hstat.data(), s->dstat, sizeof(int) * s->max_slots,
                                            cudaMemcpyDeviceToHost, s->st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
            {
                std::lock_guard<std::mutex> g(s->mu);
                s->wait_s += now_s() - tw;
            }
            if (e != cudaSuccess) {
                st = DME_ECUDA;
                err = std::string("serving: ") + cudaGetErrorString(e);
            }
        }
        s->rounds += R;
        std::vector<Req*> keep;
        for (Req* r : res) {
            dme_status rs = st;
            std::string rerr = err;
            if (rs == DME_OK && hstat[r->slot]) {
                rs = (hstat[r->slot] & DEV_NOTSPD) ? DME_ENOTSPD : DME_ECUDA;
                rerr = (rs == DME_ENOTSPD) ? "serving: I_m + t Bt^T P Bt is not positive definite"
                                           : "serving: device status " + std::to_string(hstat[r->slot]);
                cudaMemsetAsync(s->dstat + r->slot, 0, sizeof(int), s->st);
            }
            if (rs == DME_OK) r->done_steps += R;
            if (rs != DME_OK || r->done_steps >= r->nsteps) {
                if (rs == DME_OK) {
                    r->out.resize((size_t)r->desc.n * r->desc.n);
                    cudaError_t e = cudaMemcpyAsync(r->out.data(), r->P, r->out.size() * sizeof(double),
                                                    cudaMemcpyDeviceToHost, s->st);
                    if (e == cudaSuccess && r->gain) {
                        r->kout.resize((size_t)r->nsteps * r->desc.m * r->desc.n);
                        e = cudaMemcpyAsync(r->kout.data(), r->Kh, r->kout.size() * sizeof(double),
                                            cudaMemcpyDeviceToHost, s->st);
                    }
                    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
                    if (e != cudaSuccess) {
                        rs = DME_ECUDA;
                        rerr = std::string("serving: ") + cudaGetErrorString(e);
                    }
                }
                release(s, r);
                std::lock_guard<std::mutex> g(s->mu);
                finish(s, r, rs, rerr);
            } else {
                keep.push_back(r);
            }
        }
        res.swap(keep);
    }
}

}  // namespace

extern "C" {

dme_status dme_server_create(size_t hbm_budget_bytes, int max_slots, dme_server_t* out) {
    if (!out) return set_error("out is NULL"), DME_EINVAL;
    *out = nullptr;
    if (max_slots < 1 || max_slots > 4096 || hbm_budget_bytes == 0)
        return set_error("need 1 <= max_slots <= 4096 and a non-zero budget"), DME_EINVAL;
    dme_server_t s = new (std::nothrow) dme_server_s();
    if (!s) return set_error("host allocation failed"), DME_ENOMEM;
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    s->queue_cap = (size_t)max_slots * 64;
    for (int i = max_slots - 1; i >= 0; --i) s->free_slots.push_back(i);
    cudaError_t e = cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_split, cudaEventDisableTiming);
    for (int l = 0; l < kLanes; ++l) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->lane_st[l], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->lane_st2[l], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_done[l], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_fork[l], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_join[l], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMalloc(&s->dstat, sizeof(int) * max_slots);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->dstat, 0, sizeof(int) * max_slots, s->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
    // descriptors of up to kMaxStages stages: two GEMM groups, two split-GEMM
    // groups and one Riccati group per stage, each put 256-byte aligned
    constexpr size_t kMaxStages = 8;
    s->arena.cap = kMaxStages * (2 * sizeof(GemmProb) * max_slots + 2 * sizeof(OzGroupDesc) * max_slots +
                                 2 * sizeof(SliceDesc) * max_slots + riccati_desc_bytes() * max_slots + 7 * 256);
    if (e == cudaSuccess) e = cudaMalloc(&s->arena.dev, s->arena.cap);
    if (e == cudaSuccess) e = cudaMalloc(&s->tune_desc, sizeof(GemmProb) * max_slots);
    if (e != cudaSuccess) {
        set_error(std::string("dme_server_create: ") + cudaGetErrorString(e));
        cudaGetLastError();
        destroy_streams(s);
        cudaFree(s->dstat);
        cudaFree(s->arena.dev);
        cudaFree(s->tune_desc);
        delete s;
        return DME_ECUDA;
    }
    gemm64_prepare();
    if (ozaki_grouped_prepare() != DME_OK) {
        destroy_streams(s);
        cudaFree(s->dstat);
        cudaFree(s->arena.dev);
        cudaFree(s->tune_desc);
        delete s;
        return DME_ECUDA;
    }
    for (int i = 0; i < kAdmitThreads; ++i) s->admit_thrs.emplace_back(admit_loop, s);
    s->step_thr = std::thread(step_loop, s);
    *out = s;
    return DME_OK;
}

}  // extern "C"

namespace {
dme_status submit_impl(dme_server_t s, const dme_plan_desc* desc, const double* A, const double* QorC,
                       const double* B, const double* R, const double* S, const double* P0, double T, int nsteps,
                       bool gain, uint64_t* ticket);
}

extern "C" {

dme_status dme_submit(dme_server_t s, const dme_plan_desc* desc, const double* A, const double* QorC,
                      const double* B, const double* R, const double* S, const double* P0, double T, int nsteps,
                      uint64_t* ticket) {
    return submit_impl(s, desc, A, QorC, B, R, S, P0, T, nsteps, false, ticket);
}

dme_status dme_submit_gain(dme_server_t s, const dme_plan_desc* desc, const double* A, const double* QorC,
                           const double* B, const double* R, const double* S, const double* P0, double T,
                           int nsteps, uint64_t* ticket) {
    if (!desc || (desc->eq != DME_DRE && desc->eq != DME_GDRE))
        return set_error("dme_submit_gain: the gain needs a DRE (B, R)"), DME_EINVAL;
    return submit_impl(s, desc, A, QorC, B, R, S, P0, T, nsteps, true, ticket);
}

}  // extern "C"

namespace {
dme_status submit_impl(dme_server_t s, const dme_plan_desc* desc, const double* A, const double* QorC,
                       const double* B, const double* R, const double* S, const double* P0, double T, int nsteps,
                       bool gain, uint64_t* ticket) {
    if (!s || !desc || !A || !QorC || !P0 || !ticket) return set_error("missing argument"), DME_EINVAL;
    if (!(T > 0.0) || nsteps < 1) return set_error("need T > 0 and nsteps >= 1"), DME_EINVAL;
    if (desc->prec == DME_SPLIT_TF32)
        return set_error("DME_SPLIT_TF32 is not built (an 11-bit TF32 digit breaks exact fp32 accumulation "
                         "beyond K = 4); use DME_SPLIT_BF16"),
               DME_EINVAL;
    if (desc->prec != DME_FP64 && desc->prec != DME_SPLIT_BF16) return set_error("bad prec"), DME_EINVAL;
    if (desc->fsal || desc->extrap > 1) return set_error("fsal and extrapolation are for plans only"), DME_EINVAL;
    if (desc->prec == DME_SPLIT_BF16 && desc->n > 4096) return set_error("split serving needs n <= 4096"), DME_EINVAL;
    for (int i = 0; i < desc->nflows; ++i)
        if (desc->flows[i] == DME_F4) return set_error("serving supports DLE/DRE schemes (no F4)"), DME_EINVAL;
    try {
        auto r = std::make_unique<Req>();
        r->desc = *desc;
        r->desc.h = T / nsteps;
        if (r->desc.horizon == 0) r->desc.horizon = nsteps;     // the split error target holds over the solve
        const int n = desc->n;
        if (n < 1 || n > 16384) return set_error("n must be in [1, 16384]"), DME_EINVAL;
        const size_t nn = (size_t)n * n;
        const int rows_c = desc->q_is_factor ? desc->p : n;
        if (desc->q_is_factor && (desc->p < 1 || desc->p > 16384)) return set_error("bad p"), DME_EINVAL;
        r->A.assign(A, A + nn);
        r->QC.assign(QorC, QorC + (size_t)rows_c * n);
        r->P0.assign(P0, P0 + nn);
        const bool ric = desc->eq == DME_DRE || desc->eq == DME_GDRE;
        if (ric) {
            if (!B || !R || desc->m < 1 || desc->m > 32) return set_error("DRE needs B, R, 1 <= m <= 32"), DME_EINVAL;
            r->B.assign(B, B + (size_t)n * desc->m);
            r->R.assign(R, R + (size_t)desc->m * desc->m);
        }
        if (S) r->S.assign(S, S + nn);
        r->T = T;
        r->nsteps = nsteps;
        r->gain = gain;
        std::lock_guard<std::mutex> g(s->mu);
        if (plan_estimate_bytes(r->desc, true) > s->budget)
            return set_error("request footprint exceeds the server's HBM budget"), DME_ENOMEM;
        if (s->queue.size() >= s->queue_cap) return set_error("queue full"), DME_EBUSY;
        r->id = s->next_id++;
        r->t_submit = now_s();
        if (s->t_first < 0) s->t_first = r->t_submit;
        *ticket = r->id;
        s->queue.push_back(r.get());
        s->reqs[r->id] = std::move(r);
        s->cv.notify_all();
        return DME_OK;
    } catch (const std::bad_alloc&) {
        return set_error("host allocation failed"), DME_ENOMEM;
    }
}

dme_status poll_impl(dme_server_t s, uint64_t ticket, double* P_out, double* K_out, int64_t timeout_us) {
    if (!s) return set_error("server is NULL"), DME_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error("unknown ticket"), DME_EINVAL;
    Req* r = it->second.get();
    auto done = [&] { return r->state == Q_DONE; };
    if (!done()) {
        if (timeout_us == 0) return set_error("not finished"), DME_ENOTREADY;
        if (timeout_us < 0) {
            s->cv.wait(lk, done);
        } else if (!s->cv.wait_for(lk, std::chrono::microseconds(timeout_us), done)) {
            return set_error("timed out"), DME_ETIMEOUT;
        }
    }
    dme_status st = r->status;
    if (st == DME_OK && K_out && !r->gain) {
        set_error("dme_poll_gain: the request was not submitted with dme_submit_gain");
        st = DME_EINVAL;
    }
    if (st == DME_OK && P_out) std::memcpy(P_out, r->out.data(), r->out.size() * sizeof(double));
    if (st == DME_OK && K_out) std::memcpy(K_out, r->kout.data(), r->kout.size() * sizeof(double));
    if (r->status != DME_OK) set_error(r->err);
    s->reqs.erase(it);
    return st;
}

}  // namespace

extern "C" {

dme_status dme_poll(dme_server_t s, uint64_t ticket, double* P_out, int64_t timeout_us) {
    return poll_impl(s, ticket, P_out, nullptr, timeout_us);
}

dme_status dme_poll_gain(dme_server_t s, uint64_t ticket, double* P_out, double* K_out, int64_t timeout_us) {
    return poll_impl(s, ticket, P_out, K_out, timeout_us);
}

const char* dme_server_stats(dme_server_t s) {
    if (!s) return "{}";
    std::lock_guard<std::mutex> g(s->mu);
    std::vector<double> l = s->lat_ms;
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) { return l.empty() ? 0.0 : l[std::min(l.size() - 1, (size_t)(q * (l.size() - 1) + 0.5))]; };
    int resident = 0, queued = (int)s->queue.size();
    for (auto& kv : s->reqs)
        if (kv.second->state == Q_RESIDENT || kv.second->state == Q_PLANNING) ++resident;
    const double span = (s->t_first >= 0 && s->t_last > s->t_first) ? s->t_last - s->t_first : 0.0;
    int t32 = 0;
    for (auto& kv : s->tile_choice) t32 += kv.second == 32;
    char buf[768];
    snprintf(buf, sizeof(buf),
             "{\"completed\": %d, \"failed\": %d, \"resident\": %d, \"queued\": %d, \"rounds\": %d, "
             "\"graph_builds\": %d, \"graph_build_ms\": %.1f, \"round_wait_ms\": %.1f, \"tuned_groups\": %d, "
             "\"tiles32\": %d, "
             "\"p50_ms\": %.3f, \"p99_ms\": %.3f, \"solves_per_s\": %.4f, \"reserved_bytes\": %zu, "
             "\"plans\": %d, \"plan_ms_mean\": %.3f, \"split_pairs_10_13_14\": [%d, %d, %d]}",
             s->completed, s->failed, resident, queued, s->rounds.load(), s->graph_builds.load(), s->build_s * 1e3,
             s->wait_s * 1e3, s->tuned, t32,
             pct(0.5), pct(0.99),
             span > 0 ? s->completed / span : 0.0, s->reserved, s->planned,
             s->planned ? 1e3 * s->plan_s / s->planned : 0.0, s->pairs_hist[0], s->pairs_hist[1], s->pairs_hist[2]);
    s->stats = buf;
    return s->stats.c_str();
}

dme_status dme_server_destroy(dme_server_t s) {
    if (!s) return DME_OK;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    for (auto& t : s->admit_thrs)
        if (t.joinable()) t.join();
    if (s->step_thr.joinable()) s->step_thr.join();
    cudaStreamSynchronize(s->st);
    for (auto& kv : s->reqs) {
        Req* r = kv.second.get();
        if (r->P && r->plan) cudaFreeAsync(r->P, r->plan->st);
        if (r->plan) free_plan(r->plan);
    }
    if (s->round_exec) cudaGraphExecDestroy(s->round_exec);
    cudaFree(s->dstat);
    cudaFree(s->arena.dev);
    cudaFree(s->tune_desc);
    destroy_streams(s);
    delete s;
    return DME_OK;
}

}  // extern "C"
