// pwqt_server: the serving loop of the per-energy solve.  Callers submit solve
// requests (a catalog basis, a device potential, energies, a precision, host output
// buffers) and collect them by ticket.  One library context per catalog basis keeps
// its intrinsic blocks, contact self-energy cache and factor workspaces resident;
// each context has its own CUDA stream and host worker thread, so requests on
// different bases run on the device at the same time.  Continuous batching: when a
// basis' worker starts, every request queued on that basis with the same node count
// and precision joins the batch (up to SLOTS distinct potentials and within the
// budget), and the batch runs as ONE batched solve over all its (potential, energy)
// pairs -- each job with its own potential's node blocks -- so requests that
// arrived while the previous batch was on the device start together as soon as it
// ends.  Admission: a batch starts only while the estimated working sets of the
// running batches plus its own fit the server's device-memory budget
// (scheduler.h).  The worker reuses device output buffers and up to SLOTS
// potentials per basis, so steady-state requests whose energies are already in the
// contact cache allocate nothing.
#include <cmath>
#include <cstring>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "pwqt_internal.cuh"
#include "residual_oz.cuh"
#include "scheduler.h"
#include "sweep_mixed.cuh"

namespace {

constexpr int SLOTS = 8;   // potentials kept assembled per basis (system ids 0..SLOTS-1)

struct SrvReq {
    int basis = 0;
    int N = 0;
    std::vector<double> U, E;
    int precision = 0;
    double *T = nullptr, *R = nullptr, *T_ds = nullptr, *node_n = nullptr, *resid = nullptr;
    int *n_open = nullptr, *iters = nullptr, *status = nullptr;
};

struct Lane {
    pwqt_ctx* ctx = nullptr;
    int n = 0;
    // assembled potentials, most recently used first: (N, U) -> system id
    std::list<std::pair<std::vector<double>, int>> slots;
    // device outputs reused across requests (grow-only)
    void* dev = nullptr;
    size_t dev_bytes = 0;
};

}  // namespace

struct pwqt_server {
    pwqt_server_opts opts{};
    size_t budget = 0;
    std::mutex lanes_m;   // guards the catalog map (workers look their lane up while bases are added)
    std::map<int, std::unique_ptr<Lane>> lanes;
    std::unique_ptr<pwqt::Scheduler<SrvReq>> sched;
    std::mutex err_m;
    std::string err;
    void set_err(const std::string& e) {
        std::lock_guard<std::mutex> g(err_m);
        err = e;
    }
};

namespace {

int srv_fail(pwqt_server* s, int code, const std::string& msg) {
    s->set_err(msg);
    return code;
}

// system id of this potential on the lane's context, assembling it on a miss
int slot_for(Lane& L, const SrvReq& r, int* sys) {
    std::vector<double> key;
    key.reserve(r.U.size() + 1);
    key.push_back((double)r.N);
    key.insert(key.end(), r.U.begin(), r.U.end());
    for (auto it = L.slots.begin(); it != L.slots.end(); ++it)
        if (it->first == key) {
            L.slots.splice(L.slots.begin(), L.slots, it);
            *sys = L.slots.front().second;
            return PWQT_OK;
        }
    int id = (int)L.slots.size();
    if (id >= SLOTS) {   // reuse the least recently used system id
        id = L.slots.back().second;
        L.slots.pop_back();
    }
    const int rc = pwqt_set_extrinsic(L.ctx, id, r.N, r.U.data());
    if (rc != PWQT_OK) return rc;
    L.slots.emplace_front(std::move(key), id);
    *sys = id;
    return PWQT_OK;
}

// One merged batch: the requests' potentials (slots), all their energies in one
// batched solve, results scattered back to each request's host buffers.
void run_batch(pwqt_server* s, int basis, std::vector<SrvReq*>& reqs, std::vector<int>& rcs) {
    Lane* Lp;
    {
        std::lock_guard<std::mutex> g(s->lanes_m);
        Lp = s->lanes.at(basis).get();
    }
    Lane& L = *Lp;
    pwqt_ctx* c = L.ctx;
    auto fail_all = [&](int rc, const std::string& msg) {
        srv_fail(s, rc, msg);
        for (auto& r : rcs) r = rc;
    };
    const int N = reqs[0]->N, precision = reqs[0]->precision;
    std::vector<double> E;
    std::vector<pwqt::System*> of;
    std::vector<size_t> first(reqs.size() + 1, 0);
    for (size_t q = 0; q < reqs.size(); ++q) {
        int sys = 0;
        const int rc = slot_for(L, *reqs[q], &sys);
        if (rc != PWQT_OK) return fail_all(rc, std::string("request potential: ") + pwqt_last_error(c));
        pwqt::System* sp = &c->systems.at(sys);
        for (double e : reqs[q]->E) { E.push_back(e); of.push_back(sp); }
        first[q + 1] = E.size();
    }
    const size_t nE = E.size(), NN = (size_t)N;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_d = up(sizeof(double) * nE), b_nn = up(sizeof(double) * nE * NN * 2), b_i = up(sizeof(int) * nE),
                 b_no = up(sizeof(int) * nE * 2);
    const size_t need = 4 * b_d + b_nn + 2 * b_i + b_no;
    cudaSetDevice(c->dev);
    if (L.dev_bytes < need) {
        if (L.dev) cudaFree(L.dev);
        L.dev = nullptr;
        L.dev_bytes = 0;
        if (cudaMalloc(&L.dev, need) != cudaSuccess) {
            cudaGetLastError();
            return fail_all(PWQT_ERR_OOM, "device output buffers");
        }
        L.dev_bytes = need;
    }
    char* p = static_cast<char*>(L.dev);
    pwqt::SolveOut o;
    o.T = (double*)p; p += b_d;
    o.R = (double*)p; p += b_d;
    o.T_ds = (double*)p; p += b_d;
    o.resid = (double*)p; p += b_d;
    o.node_n = (double*)p; p += b_nn;
    o.iters = (int*)p; p += b_i;
    o.status = (int*)p; p += b_i;
    o.n_open = (int*)p;
    // one system: the plain batched solve; several: every (potential, energy) pair in the
    // same launches (mixed precision needs the sliced residual for that)
    bool several = false;
    for (auto* sp : of) several = several || sp != of[0];
    int rc = pwqt::solve_batch(c, *of[0], (int)nE, E.data(), precision, o, c->stream, nullptr, several ? of.data() : nullptr);
    if (rc != PWQT_OK) return fail_all(rc, std::string("solve: ") + pwqt_last_error(c));
    for (size_t q = 0; q < reqs.size(); ++q) {
        SrvReq& r = *reqs[q];
        const size_t e0 = first[q], ne = first[q + 1] - first[q];
        auto back = [&](void* host, const void* devp, size_t bytes) {
            if (host) cudaMemcpyAsync(host, devp, bytes, cudaMemcpyDeviceToHost, c->stream);
        };
        back(r.T, o.T + e0, sizeof(double) * ne);
        back(r.R, o.R + e0, sizeof(double) * ne);
        back(r.T_ds, o.T_ds + e0, sizeof(double) * ne);
        back(r.resid, o.resid + e0, sizeof(double) * ne);
        back(r.node_n, o.node_n + e0 * NN * 2, sizeof(double) * ne * NN * 2);
        back(r.iters, o.iters + e0, sizeof(int) * ne);
        back(r.status, o.status + e0, sizeof(int) * ne);
        back(r.n_open, o.n_open + 2 * e0, sizeof(int) * ne * 2);
    }
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail_all(PWQT_ERR_CUDA, std::string("copy back: ") + cudaGetErrorString(e));
    for (auto& r : rcs) r = PWQT_OK;
}

// device working set of a request, as the solve would size it (the injected-mode
// count is not known before the contacts are solved: n/4 columns are assumed)
size_t estimate_bytes(const Lane& L, const SrvReq& r) {
    const size_t n = (size_t)L.n, N = (size_t)r.N, m = std::max<size_t>(1, n / 4);
    const size_t nE = r.E.size();
    const size_t batch = std::min<size_t>(nE, L.ctx->opts.batch > 0 ? (size_t)L.ctx->opts.batch : nE);
    size_t per = r.precision == PWQT_FP64 ? sizeof(double2) * (N * n * (n + m) + n * n)
                                          : pwqt::mixed_bytes_per_energy((int)n, (int)N, (int)m);
    size_t panel = 0;   // the potential's slice panels of the tensor-core residual
    if (r.precision != PWQT_FP64 && L.ctx->residual_kind == PWQT_RESIDUAL_SLICED)
        panel = (N + 1) * pwqt::oz::panel_item_bytes((int)n, 3);
    return per * batch + 2 * sizeof(double2) * N * n * n + panel;   // + the potential's node blocks
}

// requests that can share one batched solve: same node count and precision
bool mergeable(const SrvReq& a, const SrvReq& b) { return a.N == b.N && a.precision == b.precision; }

}  // namespace

extern "C" {

int pwqt_server_create(pwqt_server** out, const pwqt_server_opts* o) {
    if (!out) return PWQT_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return PWQT_ERR_NO_DEVICE;
    }
    auto* s = new pwqt_server();
    if (o) s->opts = *o;
    if (s->opts.device < 0 || s->opts.device >= ndev) { delete s; return PWQT_ERR_INVALID_ARG; }
    if (cudaSetDevice(s->opts.device) != cudaSuccess) { delete s; return PWQT_ERR_CUDA; }
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    s->budget = s->opts.hbm_budget_bytes ? s->opts.hbm_budget_bytes : (size_t)(0.7 * (double)free_b);
    const size_t cap = s->opts.queue_capacity > 0 ? (size_t)s->opts.queue_capacity : 4096;
    s->sched = std::make_unique<pwqt::Scheduler<SrvReq>>(
        s->budget, cap, [s](int basis, std::vector<SrvReq*>& b, std::vector<int>& rcs) { run_batch(s, basis, b, rcs); },
        mergeable, (size_t)SLOTS);
    *out = s;
    return PWQT_OK;
}

int pwqt_server_add_basis(pwqt_server* s, int basis, const pwqt_cell* cell, const pwqt_formfactor* ff, double gcut, int n_bands,
                          int* n_out) {
    if (!s) return PWQT_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> g(s->lanes_m);
        if (s->lanes.count(basis)) return srv_fail(s, PWQT_ERR_INVALID_ARG, "basis id already in the catalog");
    }
    pwqt_opts co{};
    co.device = s->opts.device;
    co.hbm_budget_bytes = s->budget;   // one request batches its energies within the server budget
    co.ir_tol = s->opts.ir_tol;
    co.batch = s->opts.batch;
    auto L = std::make_unique<Lane>();
    int rc = pwqt_create(&L->ctx, &co);
    if (rc != PWQT_OK) return srv_fail(s, rc, "context for the basis");
    rc = pwqt_assemble_intrinsic(L->ctx, cell, ff, gcut, n_bands, &L->n);
    if (rc != PWQT_OK) {
        s->set_err(pwqt_last_error(L->ctx));
        pwqt_destroy(L->ctx);
        return rc;
    }
    if (n_out) *n_out = L->n;
    {
        std::lock_guard<std::mutex> g(s->lanes_m);
        s->lanes[basis] = std::move(L);
    }
    if (s->sched->add_key(basis) != 0) return srv_fail(s, PWQT_ERR_STATE, "server is shutting down");
    return PWQT_OK;
}

int pwqt_server_submit(pwqt_server* s, const pwqt_request* q, long long* ticket) {
    if (!s || !q || !ticket) return PWQT_ERR_INVALID_ARG;
    Lane* lane = nullptr;
    {
        std::lock_guard<std::mutex> g(s->lanes_m);
        auto it = s->lanes.find(q->basis);
        if (it != s->lanes.end()) lane = it->second.get();
    }
    if (!lane) return srv_fail(s, PWQT_ERR_INVALID_ARG, "unknown basis");
    if (q->n_nodes < 2 || !q->U || q->n_E < 1 || !q->E)
        return srv_fail(s, PWQT_ERR_INVALID_ARG, "a request needs n_nodes >= 2, U, n_E >= 1 and E");
    if (q->precision != PWQT_FP64 && q->precision != PWQT_MIXED && q->precision != PWQT_FP32)
        return srv_fail(s, PWQT_ERR_INVALID_ARG, "bad precision");
    for (int e = 0; e < q->n_E; ++e)
        if (!std::isfinite(q->E[e])) return srv_fail(s, PWQT_ERR_INVALID_ARG, "non-finite energy");
    for (int i = 0; i < q->n_nodes; ++i)
        if (!std::isfinite(q->U[i])) return srv_fail(s, PWQT_ERR_INVALID_ARG, "non-finite potential");
    SrvReq r;
    r.basis = q->basis;
    r.N = q->n_nodes;
    r.U.assign(q->U, q->U + q->n_nodes);
    r.E.assign(q->E, q->E + q->n_E);
    r.precision = q->precision;
    r.T = q->T; r.R = q->R; r.T_ds = q->T_ds; r.n_open = q->n_open; r.node_n = q->node_n;
    r.resid = q->resid; r.iters = q->iters; r.status = q->status;
    const size_t bytes = estimate_bytes(*lane, r);
    const int rc = s->sched->submit(q->basis, std::move(r), bytes, ticket);
    if (rc == pwqt::Scheduler<SrvReq>::ERR_BUSY) return srv_fail(s, PWQT_ERR_BUSY, "request queue is full");
    if (rc != 0) return srv_fail(s, PWQT_ERR_OOM, "request working set " + std::to_string(bytes) + " bytes exceeds the server budget");
    return PWQT_OK;
}

int pwqt_server_wait(pwqt_server* s, long long ticket, double timeout_s, int* result, double* latency_s) {
    if (!s) return PWQT_ERR_INVALID_ARG;
    const int rc = s->sched->wait(ticket, timeout_s, result, latency_s);
    if (rc == pwqt::Scheduler<SrvReq>::WAIT_TIMEOUT) return PWQT_ERR_TIMEOUT;
    if (rc != 0) return srv_fail(s, PWQT_ERR_INVALID_ARG, "unknown or already collected ticket");
    return PWQT_OK;
}

int pwqt_server_stats(pwqt_server* s, long long* completed, double* p50_s, double* p99_s, size_t* peak_admitted_bytes, int reset) {
    if (!s) return PWQT_ERR_INVALID_ARG;
    s->sched->stats(completed, p50_s, p99_s, peak_admitted_bytes);
    if (reset) s->sched->reset_stats();
    return PWQT_OK;
}

int pwqt_server_batch_stats(pwqt_server* s, long long* batches, long long* requests, long long* largest) {
    if (!s) return PWQT_ERR_INVALID_ARG;
    s->sched->batch_stats(batches, requests, largest);
    return PWQT_OK;
}

const char* pwqt_server_last_error(pwqt_server* s) {
    if (!s) return "null server";
    std::lock_guard<std::mutex> g(s->err_m);
    return s->err.c_str();
}

int pwqt_server_destroy(pwqt_server* s) {
    if (!s) return PWQT_OK;
    s->sched->shutdown();   // finishes the queued requests
    s->sched.reset();
    for (auto& kv : s->lanes) {
        if (kv.second->dev) cudaFree(kv.second->dev);
        pwqt_destroy(kv.second->ctx);
    }
    delete s;
    return PWQT_OK;
}

}  // extern "C"
