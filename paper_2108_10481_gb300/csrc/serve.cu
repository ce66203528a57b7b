// a11: request server - continuous batching of boundary-element solves.
//
// Molecules (mesh, charges, eps_int, eps_ext, kappa, formulation,
// preconditioner) arrive with pb_submit. An admission thread takes them in
// arrival order whenever the HBM budget and the slot count allow, loads the
// mesh, builds the FP64 near field and the right-hand side on its own
// non-blocking stream (so near-field builds overlap the other requests'
// iterations), and hands them to the active set. Every pb_server_step then
// advances each active request by one GMRES step: all their operator
// applications go into one persistent launch per row mode over a table of
// work items - (request, target block, source split) of the direct pair sums
// and (request, leaf, list split) of the treecode for requests large enough
// for it - taken by the CTAs most expensive first, followed by each request's
// own preconditioner, Gram-Schmidt and Givens kernels, and one read-back of
// all residual estimates. A request that converges computes its energy,
// reports its result and frees its memory, making room for the next.
//
// Each request keeps the decomposition it has alone, and all its reductions
// run in a fixed order, so its result does not depend on what else is in the
// batch.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <shared_mutex>
#include <thread>

#include "solver.h"

namespace pb {

enum Phase { PH_START = 0, PH_ITER, PH_ENERGY };

static double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct ServeReq {
    uint64_t tag = 0;
    std::vector<double> V, xq, q;
    std::vector<int32_t> T;
    pb_params prm;
    int form = 0, pc = 0;
    pb_solve_opts opts;
    pb_quad_plan plan;
    size_t footprint = 0;
    double t_submit = 0, t_ready = 0;
    // device state
    pb_mesh* m = nullptr;
    pb_near* nf = nullptr;
    double* buf = nullptr;
    double *dxq = nullptr, *dq = nullptr, *rhs = nullptr, *x = nullptr, *rr = nullptr, *dd = nullptr, *w = nullptr;
    Solver S;
    GmresWork G;
    bool mixed = false;
    int mmax = 0;
    int slot = -1;            // row of the server's residual table while active
    StepGraph g_mid, g_tail;  // captured iteration pieces (Calderon middle; preconditioner + Arnoldi)
    // iteration state
    int phase = PH_START;
    int j = 0, outer = 0, total_it = 0;
    double bnorm = 0, rel = 1, prev_rel = 1, inner_tol = 0;
    int status = PB_OK;
};

}  // namespace pb

struct pb_server {
    pb_ctx* ctx = nullptr;
    size_t budget = 0;
    int max_active = 1;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<pb::ServeReq*> waiting;  // submitted, not admitted
    std::deque<pb::ServeReq*> ready;    // set up, not yet in the active set
    std::vector<pb::ServeReq*> active;  // owned by the stepping thread
    std::vector<pb_result> done;
    size_t used = 0;
    int admitted = 0;  // admitted and not finished
    bool stop = false;
    std::vector<std::thread> admit_threads;
    // Held shared by the admission threads while they set requests up (their
    // allocations, frees and synchronisations reach the whole device) and
    // exclusively by the stepping thread while it captures a CUDA graph, which
    // such calls would invalidate.
    std::shared_mutex device_mu;
    cudaStream_t s_main = nullptr;
    std::vector<cudaStream_t> s_setup;  // one per admission thread
    pb::BatchScratch bs;
    double* res_dev = nullptr;   // 4 doubles per slot (max_active slots)
    double* res_host = nullptr;
    std::vector<int> free_slots;
    // per slot: the stream of the active request that holds it (its own kernels, so that the small
    // kernels of different requests overlap on the device) and an event joining it to s_main
    std::vector<cudaStream_t> slot_stream;
    std::vector<cudaEvent_t> slot_event;
};

namespace pb {

static int free_req(ServeReq* r) {
    graph_free(r->g_mid);
    graph_free(r->g_tail);
    solver_release(r->S);
    if (r->buf) cudaFree(r->buf);
    r->buf = nullptr;
    gmres_free(r->G);
    pb_free_near(r->nf);
    pb_free_mesh(r->m);
    r->nf = nullptr;
    r->m = nullptr;
    return PB_OK;
}

// Device bytes a request holds while resident (upper estimates of the
// adjacency sizes: 16 adjacent pairs per triangle, 25 near nonzeros per vertex;
// a distance band of eta radii adds about 18 eta^2 ordered pairs per triangle
// and 15 eta^2 nonzeros per vertex: the synthetic molecules have about 145
// band pairs per triangle and 147 nonzeros per vertex at 3 radii). The near
// build's per-pair blocks (432 bytes per listed pair) are the largest
// transient: about 14 GB on the 5,000-atom molecule.
static size_t footprint(pb_ctx* ctx, int64_t nv, int64_t nt, const pb_quad_plan& plan, int mmax, int64_t nq) {
    const int Q = plan.far_q;
    const double eta = plan.band_eta, band = 18.0 * eta * eta * nt;
    const double np = (double)Q * nt, nadj = 16.0 * nt, npairs = nadj + band, nnz = (25.0 + 15.0 * eta * eta) * nv;
    const double npref = eta > 0.0 ? 6.0 * nt : 0.0;
    double mesh = 24 * nv + 12 * nt + 128 * nt + 64 * np + 32 * npref + 8 * (nv + 1) + 12 * nt + 16 * npairs +
                  12 * nnz + 4 * nv + 4 * (nnz + 1) + 36 * npairs;
    double nearb = 56 * nnz + 56 * nv;
    double near_tmp = 432 * (npairs + nadj) + 4 * nnz;
    double src = 128 * (np + 64);
    int S = far_splits_estimate(ctx, (int64_t)np);
    double part = (double)S * 10 * np * 8;
    double work = src + part + 48 * nt + 48 * nnz + 128 * nv;
    if (ctx->tree_enable && np >= (double)ctx->tree_min_points) {
        work += 330 * np;  // treecode: tree-ordered sources, proxies of about np / 64 clusters, lists
        work += std::max(0.0, 8.0 * 10 * 4 * np - part);  // its partial sums: up to 8 FP32 slices
    }
    double n2 = 2.0 * nv;
    double nchunk = std::ceil(n2 / 2048.0);
    double gm = 8 * ((mmax + 1) * n2 + n2 + (double)(mmax + 1) * mmax + 4 * mmax + 2 + (mmax + 2) * nchunk + 16);
    double bufb = 8 * (4.0 * nq + 10 * nv);
    return (size_t)(mesh + nearb + std::max(near_tmp, work) + gm + bufb);
}

// load, near field, right-hand side and solver state, on the setup stream
static int setup_req(pb_server* srv, ServeReq* r, cudaStream_t s) {
    pb_ctx* ctx = srv->ctx;
    PB_TRY(pb_mesh_load(ctx, r->V.data(), (int64_t)r->V.size() / 3, r->T.data(), (int64_t)r->T.size() / 3,
                        &r->plan, PB_MEM_HOST, &r->m));
    PB_TRY(pb_near_build(ctx, r->m, r->prm.kappa, &r->nf, s));
    const int64_t nv = r->m->nv, nq = (int64_t)r->q.size();
    PB_TRY(dev_alloc((void**)&r->buf, sizeof(double) * (4 * nq + 10 * nv)));
    r->dxq = r->buf;
    r->dq = r->dxq + 3 * nq;
    r->rhs = r->dq + nq;
    r->x = r->rhs + 2 * nv;
    r->rr = r->x + 2 * nv;
    r->dd = r->rr + 2 * nv;
    r->w = r->dd + 2 * nv;
    PB_CUDA(cudaMemcpyAsync(r->dxq, r->xq.data(), sizeof(double) * 3 * nq, cudaMemcpyHostToDevice, s));
    PB_CUDA(cudaMemcpyAsync(r->dq, r->q.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, s));
    const int cprec = r->opts.precision == PB_MIXED ? PB_F32_ACCURATE : PB_F64;  // the charge sums' arithmetic
    PB_TRY(pb_rhs_charges(ctx, r->m, r->dxq, r->dq, nq, &r->prm, r->form, r->opts.alpha, r->opts.beta, r->rhs, cprec,
                          s));
    PB_CUDA(cudaMemsetAsync(r->x, 0, sizeof(double) * 2 * nv, s));
    PB_TRY(setup_solver(r->S, r->m, r->nf, &r->prm, r->form, r->pc, &r->opts, s));
    PB_TRY(gmres_alloc(r->G, 2 * nv, r->mmax));
    PB_CUDA(cudaStreamSynchronize(s));
    r->S.s = srv->s_main;  // until the request holds a slot (and its stream)
    r->mixed = r->opts.precision == PB_MIXED;
    r->phase = PH_START;
    return PB_OK;
}

static void finish(pb_server* srv, ServeReq* r, double dGp, double dGk) {
    pb_result res;
    res.tag = r->tag;
    res.status = r->status;
    res.iters = r->total_it;
    res.outer_iters = r->mixed ? r->outer : 1;
    res.dG_paper = dGp;
    res.dG_kcal = dGk;
    res.rel_residual = r->rel;
    double t = now_ms();
    res.latency_ms = t - r->t_submit;
    res.queue_ms = r->t_ready - r->t_submit;
    free_req(r);
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->used -= r->footprint;
    srv->admitted -= 1;
    srv->done.push_back(res);
    srv->cv.notify_all();
}

static void admission_loop(pb_server* srv, int k) {
    cudaSetDevice(srv->ctx->device);
    for (;;) {
        ServeReq* r = nullptr;
        {
            std::unique_lock<std::mutex> lock(srv->mu);
            srv->cv.wait(lock, [&] {
                return srv->stop || (!srv->waiting.empty() && srv->admitted < srv->max_active &&
                                     srv->used + srv->waiting.front()->footprint <= srv->budget);
            });
            if (srv->stop) return;
            r = srv->waiting.front();
            srv->waiting.pop_front();
            srv->used += r->footprint;
            srv->admitted += 1;
        }
        int rc;
        {
            std::shared_lock<std::shared_mutex> dev_lock(srv->device_mu);
            rc = setup_req(srv, r, srv->s_setup[k]);
        }
        r->t_ready = now_ms();
        if (rc != PB_OK) {
            r->status = rc;
            r->rel = 0.0;
            {
                std::shared_lock<std::shared_mutex> dev_lock(srv->device_mu);
                free_req(r);
            }
            finish(srv, r, 0.0, 0.0);
            delete r;
            continue;
        }
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->ready.push_back(r);
        srv->cv.notify_all();
    }
}

// The operator applications of one round: per precision, one persistent launch
// over the work items of every request (pair items of the direct sums and, for
// FP32 applications of meshes large enough for the treecode, the leaves of
// their trees). The path a request takes, and its decomposition into items,
// depend only on its own size, so its result does not depend on the batch.
static int apply_round(pb_server* srv, std::vector<FarJob>* jobs, cudaStream_t s) {
    for (int p = 0; p < 4; ++p) PB_TRY(apply_blockops_batched(jobs[p], p, srv->bs, s));
    return PB_OK;
}

static int tick(pb_server* srv) {
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        while (!srv->ready.empty()) {
            srv->active.push_back(srv->ready.front());
            srv->ready.pop_front();
        }
    }
    std::vector<ServeReq*>& act = srv->active;
    if (act.empty()) return PB_OK;
    cudaStream_t s = srv->s_main;
    const int n = (int)act.size();
    for (ServeReq* r : act)
        if (r->slot < 0) {
            r->slot = srv->free_slots.back();
            srv->free_slots.pop_back();
            r->S.s = srv->slot_stream[r->slot];
        }
    auto rs_of = [&](const ServeReq* r) { return srv->slot_stream[r->slot]; };
    // an iteration piece from its CUDA graph once the request has run it once
    auto piece = [&](ServeReq* r, StepGraph& g, const std::function<int()>& body) -> int {
        graph_check(g, &r->m->ws_gen);
        if (!srv->ctx->graphs || g.failed) return body();
        if (!g.exec) {
            if (r->j < 1) return body();
            {
                std::unique_lock<std::shared_mutex> dev_lock(srv->device_mu);
                PB_TRY(graph_capture(g, rs_of(r), body, &r->m->ws_gen));
            }
            if (g.failed) return body();
        }
        return graph_replay(g, rs_of(r));
    };
    // a request's combined near values (made on its first application, kept for its solve)
    auto comb_of = [](ServeReq* r, bool calderon) -> const double* {
        const double* c = nullptr;
        return solver_comb(r->S, calderon, &c) == PB_OK ? c : nullptr;
    };
    auto it_prec = [](const ServeReq* r) { return r->mixed ? PB_F32 : PB_F64; };
    auto res_prec = [](const ServeReq* r) { return r->mixed ? PB_F32_ACCURATE : PB_F64; };

    // round A: the system operator for every request that needs one
    std::vector<FarJob> jobs[4];  // by precision
    for (ServeReq* r : act) {
        if (r->phase == PH_ITER)
            jobs[it_prec(r)].push_back({r->m, r->nf, r->S.A, r->G.vin, r->S.t3, rs_of(r), comb_of(r, false)});
        else if (r->phase == PH_START && r->mixed && r->outer > 0)
            jobs[res_prec(r)].push_back({r->m, r->nf, r->S.A, r->x, r->S.t3, rs_of(r), comb_of(r, false)});
    }
    PB_TRY(apply_round(srv, jobs, s));
    for (auto& v : jobs) v.clear();
    // preconditioner input; Calderon requests queue their second operator
    std::vector<const double*> pin(n, nullptr);
    for (int k = 0; k < n; ++k) {
        ServeReq* r = act[k];
        const int64_t n2 = 2 * r->m->nv;
        if (r->phase == PH_ITER) {
            pin[k] = r->S.t3;
            if (r->pc >= PB_PC_CALDERON_FULL) {
                const int ip = it_prec(r);
                PB_TRY(piece(r, r->g_mid, [r, ip] { return calderon_pre(r->S, ip, r->S.t3); }));
                jobs[it_prec(r)].push_back({r->m, r->nf, r->S.C, r->S.t1, r->S.t2, rs_of(r), comb_of(r, true)});
            }
            continue;  // the rest of the iteration follows the batched operators
        } else if (r->phase == PH_START) {
            if (r->mixed && r->outer > 0) {
                vec_sub(n2, r->rhs, r->S.t3, r->rr, rs_of(r));
                pin[k] = r->rr;
            } else {
                pin[k] = r->rhs;
            }
        }
        if (!pin[k]) continue;
        const int prec = r->phase == PH_ITER ? it_prec(r) : res_prec(r);
        if (r->pc >= PB_PC_CALDERON_FULL) {
            PB_TRY(calderon_pre(r->S, prec, pin[k]));
            jobs[prec].push_back({r->m, r->nf, r->S.C, r->S.t1, r->S.t2, rs_of(r), comb_of(r, true)});
        } else {
            PB_TRY(apply_prec(r->S, prec, pin[k], r->w));
        }
    }
    PB_TRY(apply_round(srv, jobs, s));
    for (int k = 0; k < n; ++k) {
        ServeReq* r = act[k];
        if (!pin[k]) continue;
        double* slot = srv->res_dev + 4 * r->slot;
        cudaStream_t rs = rs_of(r);
        if (r->phase == PH_ITER) {
            const int prec = it_prec(r);
            PB_TRY(piece(r, r->g_tail, [r, prec, slot, rs] {
                if (r->pc >= PB_PC_CALDERON_FULL) PB_TRY(calderon_post(r->S, prec, r->w));
                else PB_TRY(apply_prec(r->S, prec, r->S.t3, r->w));
                return gm_step(r->G, r->w, slot, rs);
            }));
        } else {
            if (r->pc >= PB_PC_CALDERON_FULL) PB_TRY(calderon_post(r->S, res_prec(r), r->w));
            gm_norm2(r->G, r->w, slot, rs);
        }
    }
    // every request's estimates, after its own stream's work
    for (ServeReq* r : act) {
        PB_CUDA(cudaEventRecord(srv->slot_event[r->slot], rs_of(r)));
        PB_CUDA(cudaStreamWaitEvent(s, srv->slot_event[r->slot], 0));
    }
    PB_CUDA(cudaMemcpyAsync(srv->res_host, srv->res_dev, sizeof(double) * 4 * srv->max_active,
                            cudaMemcpyDeviceToHost, s));
    PB_CUDA(cudaStreamSynchronize(s));

    // host decisions
    for (int k = 0; k < n; ++k) {
        ServeReq* r = act[k];
        const double* h = srv->res_host + 4 * r->slot;
        const double tol = r->opts.tol;
        if (r->phase == PH_START) {
            const double beta = std::sqrt(h[0]);
            if (!std::isfinite(beta)) {
                r->status = set_error(PB_ENUMERIC, "residual is not finite");
                r->phase = PH_ENERGY;
                continue;
            }
            if (r->outer == 0) r->bnorm = beta;
            r->prev_rel = r->rel;
            r->rel = r->bnorm > 0.0 ? beta / r->bnorm : 0.0;
            // r->inner_tol still holds the last sweep's inner tolerance
            const double next =
                r->mixed && r->rel > 0.0
                    ? refine_inner_tol(r->outer, r->rel, r->prev_rel, r->inner_tol, tol, r->opts.inner_tol)
                    : tol;
            const bool stall = r->mixed && next < 0.0;
            if (beta == 0.0 || (r->mixed && (r->rel <= tol || stall)) || (!r->mixed && r->outer > 0)) {
                if (r->rel > tol) r->status = PB_ENOCONV;
                r->phase = PH_ENERGY;
                continue;
            }
            r->inner_tol = next;
            PB_TRY(gm_begin(r->G, r->w, srv->res_dev + 4 * r->slot, rs_of(r)));
            if (r->mixed) PB_CUDA(cudaMemsetAsync(r->dd, 0, sizeof(double) * 2 * r->m->nv, rs_of(r)));
            r->j = 0;
            r->phase = PH_ITER;
        } else if (r->phase == PH_ITER) {
            const double res = h[0];
            r->total_it += 1;
            r->j += 1;
            if (!std::isfinite(res)) {
                r->status = set_error(PB_ENUMERIC, "residual is not finite");
                r->phase = PH_ENERGY;
                continue;
            }
            const bool conv = res <= r->inner_tol;
            if (conv || h[1] == 0.0 || r->j >= r->mmax || r->total_it >= r->opts.max_it) {
                PB_TRY(gm_finish(r->G, r->j, r->mixed ? r->dd : r->x, rs_of(r)));
                if (r->mixed) {
                    vec_add(2 * r->m->nv, r->dd, r->x, rs_of(r));
                    r->outer += 1;
                    r->phase = r->total_it >= r->opts.max_it || r->outer >= std::max(1, r->opts.max_outer)
                                   ? PH_ENERGY : PH_START;
                    if (r->phase == PH_ENERGY) r->status = PB_ENOCONV;
                } else {
                    r->rel = res;
                    r->outer = 1;
                    if (!conv) r->status = PB_ENOCONV;
                    r->phase = PH_ENERGY;
                }
            }
        }
    }
    // finished requests: energy, result, memory back to the budget
    std::vector<ServeReq*> keep;
    for (ServeReq* r : act) {
        if (r->phase != PH_ENERGY) {
            keep.push_back(r);
            continue;
        }
        double dGp = 0.0, dGk = 0.0;
        int rc = pb_energy(srv->ctx, r->m, r->x, r->form, r->dxq, r->dq, (int64_t)r->q.size(), &r->prm, nullptr, &dGp,
                           &dGk, r->mixed ? PB_F32_ACCURATE : PB_F64, rs_of(r));
        if (rc != PB_OK && r->status == PB_OK) r->status = rc;
        if (r->status == PB_OK) r->status = check_status(r->m, rs_of(r));
        srv->free_slots.push_back(r->slot);
        r->slot = -1;
        finish(srv, r, dGp, dGk);
        delete r;
    }
    act.swap(keep);
    return PB_OK;
}

}  // namespace pb

using namespace pb;

// Admission threads: each sets up one request at a time on its own stream, so
// the host work of one request's mesh ingest overlaps another's near build.
constexpr int ADMIT_THREADS = 2;

static void destroy_streams(pb_server* srv) {
    for (cudaStream_t q : srv->slot_stream)
        if (q) cudaStreamDestroy(q);
    for (cudaEvent_t e : srv->slot_event)
        if (e) cudaEventDestroy(e);
    for (cudaStream_t q : srv->s_setup)
        if (q) cudaStreamDestroy(q);
    if (srv->s_main) cudaStreamDestroy(srv->s_main);
    srv->slot_stream.clear();
    srv->slot_event.clear();
    srv->s_setup.clear();
    srv->s_main = nullptr;
}

extern "C" int pb_server_create(pb_ctx* ctx, int64_t hbm_budget_bytes, int max_active, pb_server** out) {
    if (!ctx || !out || hbm_budget_bytes <= 0 || max_active < 1)
        return set_error(PB_EINVAL, "pb_server_create: bad argument");
    *out = nullptr;
    PB_CUDA(cudaSetDevice(ctx->device));
    pb_server* srv = new pb_server();
    srv->ctx = ctx;
    srv->budget = (size_t)hbm_budget_bytes;
    srv->max_active = max_active;
    srv->s_setup.assign(ADMIT_THREADS, nullptr);
    srv->slot_stream.assign(max_active, nullptr);
    srv->slot_event.assign(max_active, nullptr);
    bool ok = cudaStreamCreateWithFlags(&srv->s_main, cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; ok && k < ADMIT_THREADS; ++k)
        ok = cudaStreamCreateWithFlags(&srv->s_setup[k], cudaStreamNonBlocking) == cudaSuccess;
    // per slot: the active request's stream and its join event
    for (int k = 0; ok && k < max_active; ++k)
        ok = cudaStreamCreateWithFlags(&srv->slot_stream[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&srv->slot_event[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        destroy_streams(srv);
        delete srv;
        return set_error(PB_ECUDA, "pb_server_create: stream creation failed");
    }
    // one residual row per slot, fixed for a request's lifetime (captured graphs write to it)
    if (dev_alloc((void**)&srv->res_dev, sizeof(double) * 4 * max_active) != PB_OK ||
        cudaMallocHost((void**)&srv->res_host, sizeof(double) * 4 * max_active) != cudaSuccess) {
        if (srv->res_dev) cudaFree(srv->res_dev);
        destroy_streams(srv);
        delete srv;
        return set_error(PB_ENOMEM, "pb_server_create: residual table");
    }
    cudaMemset(srv->res_dev, 0, sizeof(double) * 4 * max_active);
    for (int k = max_active - 1; k >= 0; --k) srv->free_slots.push_back(k);
    for (int k = 0; k < ADMIT_THREADS; ++k) srv->admit_threads.emplace_back(admission_loop, srv, k);
    *out = srv;
    return PB_OK;
}

extern "C" int pb_server_destroy(pb_server* srv) {
    if (!srv) return PB_OK;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        srv->stop = true;
        srv->cv.notify_all();
    }
    for (std::thread& t : srv->admit_threads)
        if (t.joinable()) t.join();
    cudaSetDevice(srv->ctx->device);
    cudaDeviceSynchronize();
    for (ServeReq* r : srv->active) { free_req(r); delete r; }
    for (ServeReq* r : srv->ready) { free_req(r); delete r; }
    for (ServeReq* r : srv->waiting) delete r;
    batch_scratch_free(srv->bs);
    if (srv->res_dev) cudaFree(srv->res_dev);
    if (srv->res_host) cudaFreeHost(srv->res_host);
    destroy_streams(srv);
    delete srv;
    return PB_OK;
}

extern "C" int pb_submit(pb_server* srv, const pb_request* req) {
    if (!srv || !req || !req->verts || !req->tris || !req->xq || !req->q || req->n_q < 1 || req->n_verts < 4 ||
        req->n_tris < 4)
        return set_error(PB_EINVAL, "pb_submit: bad request");
    if (req->precond < PB_PC_NONE || req->precond > PB_PC_SCALED_CALDERON_EXT || req->form < PB_DIRECT_INT ||
        req->form > PB_LU)
        return set_error(PB_EINVAL, "pb_submit: unknown formulation or preconditioner");
    ServeReq* r = new ServeReq();
    r->tag = req->tag;
    r->V.assign(req->verts, req->verts + 3 * req->n_verts);
    r->T.assign(req->tris, req->tris + 3 * req->n_tris);
    r->xq.assign(req->xq, req->xq + 3 * req->n_q);
    r->q.assign(req->q, req->q + req->n_q);
    r->prm = req->params;
    r->form = req->form;
    r->pc = req->precond;
    r->opts = req->opts;
    r->plan = req->plan;
    if (r->plan.far_q == 0) r->plan = {6, 4, 0.0, 6};
    if (!(r->opts.tol > 0.0) || r->opts.max_it < 1) {
        delete r;
        return set_error(PB_EINVAL, "pb_submit: need tol > 0 and max_it >= 1");
    }
    r->mmax = r->opts.restart > 0 ? std::min(r->opts.restart, r->opts.max_it) : r->opts.max_it;
    r->footprint = footprint(srv->ctx, req->n_verts, req->n_tris, r->plan, r->mmax, req->n_q);
    if (r->footprint > srv->budget) {
        size_t fp = r->footprint;
        delete r;
        return set_error(PB_ENOMEM, "request needs about %zu bytes, more than the server's budget of %zu", fp,
                         srv->budget);
    }
    r->t_submit = now_ms();
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->waiting.push_back(r);
    srv->cv.notify_all();
    return PB_OK;
}

extern "C" int pb_server_step(pb_server* srv, int* n_active, int* n_pending) {
    if (!srv) return set_error(PB_EINVAL, "pb_server_step: NULL server");
    PB_CUDA(cudaSetDevice(srv->ctx->device));
    int rc = tick(srv);
    std::lock_guard<std::mutex> lock(srv->mu);
    if (n_active) *n_active = (int)srv->active.size();
    // waiting + being set up + set up but not yet stepping
    if (n_pending) *n_pending = (int)srv->waiting.size() + srv->admitted - (int)srv->active.size();
    return rc;
}

extern "C" int pb_poll(pb_server* srv, pb_result* out, int max, int* n_out) {
    if (!srv || !n_out || (max > 0 && !out)) return set_error(PB_EINVAL, "pb_poll: bad argument");
    std::lock_guard<std::mutex> lock(srv->mu);
    int n = std::min(max, (int)srv->done.size());
    for (int i = 0; i < n; ++i) out[i] = srv->done[i];
    srv->done.erase(srv->done.begin(), srv->done.begin() + n);
    *n_out = n;
    return PB_OK;
}
