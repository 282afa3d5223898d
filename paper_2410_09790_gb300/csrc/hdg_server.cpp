// Serving runtime of the HDG IMEX solver (include/hdg.h, hdg_server_*): a request queue in arrival
// order, admission by device-memory budget and slot limit, continuous batching of the active
// requests (one hdg_batch_step per round: every active request advances one IMEX step, all
// enqueued before any is waited for), and a pool of resident contexts keyed by configuration
// (mesh and parameters) so that a new request reuses the condensed operators and the recorded
// step graph of a finished one. Built only on the public C-ABI and the CUDA runtime.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/hdg.h"

namespace {

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// configuration key: every field of the mesh and the parameters, printed exactly
std::string config_key(const hdg_mesh_desc &m, const hdg_params &p) {
    char b[1024];
    snprintf(b, sizeof b,
             "%d %a %a %d %d | %d %a %a %a %d %a %d %a %d %a %a %d %d %a %a %d %d %d %d %d %d %d %a %a",
             m.n, m.Lx, m.Ly, m.periodic_x, m.periodic_y, p.k, p.alpha, p.tau, p.delta_up, p.tableau, p.dt,
             p.n_richardson, p.richardson_rtol, p.richardson_max, p.trace_rtol, p.stepI_rtol, p.max_iters,
             p.stage_krylov, p.inner_stepI_rtol, p.inner_trace_rtol, p.trace_mg, p.device_loops, p.inner_trace_vcycles,
             p.precision, p.inner_trace_fp32, p.trace_fp32_vcycle, p.inner_gs, p.timeout_ms,
             p.relax_eta);
    return b;
}

struct Slot {                       // a resident context with its stream and staging buffers
    hdg_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;
    std::string key;
    double estimate = 0, last_used = 0;
    int64_t nQ = 0, nP = 0, nL = 0;
    double *dQ = nullptr, *dp = nullptr, *dl = nullptr;
    size_t staging_bytes = 0;
};

struct Request {
    long long id = 0;
    hdg_mesh_desc mesh{};
    hdg_params params{};
    std::vector<double> Q0, Q, p, lam;
    int nsteps = 0, taken = 0;
    double t_submit = 0, t_done = 0;
    Slot *slot = nullptr;
};

void release_slot(Slot *s) {
    if (s->ctx) hdg_destroy(s->ctx);
    if (s->dQ) cudaFree(s->dQ);
    if (s->dp) cudaFree(s->dp);
    if (s->dl) cudaFree(s->dl);
    if (s->st) cudaStreamDestroy(s->st);
    delete s;
}

}  // namespace

struct hdg_server {
    int device = 0;
    double budget = 0;
    int max_active = 1;
    long long next_id = 1;
    std::deque<Request *> queue;
    std::vector<Request *> active;
    std::map<long long, Request *> done;
    std::vector<Slot *> idle, slots;
    hdg_server_stats st{};

    double bytes_in_use() const {
        double b = 0;
        for (const Slot *s : slots) b += std::max((double)hdg_ctx_bytes(s->ctx), s->estimate) + s->staging_bytes;
        return b;
    }
    void drop(Slot *s) {
        slots.erase(std::find(slots.begin(), slots.end(), s));
        release_slot(s);
        st.contexts_released += 1;
    }
};

namespace {

// a slot for the request: an idle one of the same configuration, else a new one if the budget
// allows after releasing idle slots (least recently used first); nullptr if it does not fit
hdg_status acquire_slot(hdg_server *S, Request *r, Slot **out) {
    *out = nullptr;
    const std::string key = config_key(r->mesh, r->params);
    for (size_t i = 0; i < S->idle.size(); ++i)
        if (S->idle[i]->key == key) {
            *out = S->idle[i];
            S->idle.erase(S->idle.begin() + i);
            S->st.contexts_reused += 1;
            return HDG_OK;
        }
    const double need = hdg_estimate_bytes(&r->mesh, &r->params);
    if (!(need > 0)) return HDG_ERR_INVALID_ARG;
    while (S->bytes_in_use() + need > S->budget && !S->idle.empty()) {
        auto lru = std::min_element(S->idle.begin(), S->idle.end(),
                                    [](const Slot *a, const Slot *b) { return a->last_used < b->last_used; });
        Slot *victim = *lru;
        S->idle.erase(lru);
        S->drop(victim);
    }
    if (S->bytes_in_use() + need > S->budget) return HDG_OK;      // wait for memory
    Slot *s = new (std::nothrow) Slot();
    if (!s) return HDG_ERR_OOM;
    s->key = key;
    s->estimate = need;
    if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) {
        release_slot(s);
        return HDG_ERR_CUDA;
    }
    hdg_status e = hdg_setup_mesh(&s->ctx, &r->mesh, &r->params, s->st);
    if (e == HDG_OK) e = hdg_dof_sizes(s->ctx, &s->nQ, &s->nP, &s->nL);
    if (e == HDG_OK) {
        s->staging_bytes = sizeof(double) * (size_t)(s->nQ + s->nP + s->nL);
        if (cudaMalloc(&s->dQ, sizeof(double) * s->nQ) != cudaSuccess ||
            cudaMalloc(&s->dp, sizeof(double) * s->nP) != cudaSuccess ||
            cudaMalloc(&s->dl, sizeof(double) * s->nL) != cudaSuccess)
            e = HDG_ERR_OOM;
    }
    if (e != HDG_OK) {
        release_slot(s);
        return e;
    }
    S->slots.push_back(s);
    S->st.contexts_created += 1;
    *out = s;
    return HDG_OK;
}

}  // namespace

extern "C" {

hdg_status hdg_server_create(hdg_server **out, int device, double mem_budget_bytes, int max_active) {
    if (!out || device < 0 || !(mem_budget_bytes > 0) || max_active < 1) return HDG_ERR_INVALID_ARG;
    *out = nullptr;
    hdg_server *S = new (std::nothrow) hdg_server();
    if (!S) return HDG_ERR_OOM;
    S->device = device;
    S->budget = mem_budget_bytes;
    S->max_active = max_active;
    *out = S;
    return HDG_OK;
}

hdg_status hdg_server_submit(hdg_server *S, const hdg_mesh_desc *mesh, const hdg_params *params,
                             const double *Q0_host, int nsteps, long long *id) {
    if (!S || !mesh || !params || !Q0_host || nsteps < 1 || !id) return HDG_ERR_INVALID_ARG;
    if (!(hdg_estimate_bytes(mesh, params) > 0)) return HDG_ERR_INVALID_ARG;
    int64_t nc = 0, nf = 0;
    hdg_status e = hdg_mesh_counts(mesh, params->k, &nc, &nf);
    if (e != HDG_OK) return e;
    Request *r = new (std::nothrow) Request();
    if (!r) return HDG_ERR_OOM;
    r->id = S->next_id++;
    r->mesh = *mesh;
    r->params = *params;
    const size_t nQ = (size_t)nc * (params->k + 2) * (params->k + 3);
    r->Q0.assign(Q0_host, Q0_host + nQ);
    r->nsteps = nsteps;
    r->t_submit = now_ms();
    S->queue.push_back(r);
    S->st.submitted += 1;
    *id = r->id;
    return HDG_OK;
}

hdg_status hdg_server_progress(hdg_server *S, hdg_server_stats *stats) {
    if (!S) return HDG_ERR_INVALID_ARG;
    if (cudaSetDevice(S->device) != cudaSuccess) return HDG_ERR_CUDA;
    // admission, in arrival order
    while (!S->queue.empty() && (int)S->active.size() < S->max_active) {
        Request *r = S->queue.front();
        Slot *s = nullptr;
        hdg_status e = acquire_slot(S, r, &s);
        if (e != HDG_OK) return e;
        if (!s) break;                                   // the head of the queue waits for memory
        if (cudaMemcpyAsync(s->dQ, r->Q0.data(), sizeof(double) * s->nQ, cudaMemcpyHostToDevice, s->st) != cudaSuccess)
            return HDG_ERR_CUDA;
        e = hdg_set_state(s->ctx, s->dQ, nullptr, nullptr, 0.0);
        if (e == HDG_OK) e = hdg_div_free_project(s->ctx, nullptr);
        if (e != HDG_OK) return e;
        r->slot = s;
        S->queue.pop_front();
        S->active.push_back(r);
        S->st.admitted += 1;
    }
    // one step of every active request, enqueued together
    if (!S->active.empty()) {
        std::vector<hdg_ctx *> ctxs;
        for (Request *r : S->active) ctxs.push_back(r->slot->ctx);
        std::vector<hdg_stats> st(ctxs.size());
        hdg_status e = hdg_batch_step(ctxs.data(), (int)ctxs.size(), 1, st.data());
        if (e != HDG_OK && e != HDG_ERR_NOT_CONVERGED) return e;
        for (size_t i = 0; i < ctxs.size(); ++i) {
            S->active[i]->taken += 1;
            S->st.steps += 1;
            S->st.stage_solves += st[i].stage_solves;
        }
        // retire the requests that have taken their steps; their contexts become idle
        std::vector<Request *> still;
        for (Request *r : S->active) {
            if (r->taken < r->nsteps) {
                still.push_back(r);
                continue;
            }
            Slot *s = r->slot;
            double t = 0;
            e = hdg_get_state(s->ctx, s->dQ, s->dp, s->dl, &t);
            if (e != HDG_OK) return e;
            r->Q.resize(s->nQ); r->p.resize(s->nP); r->lam.resize(s->nL);
            if (cudaMemcpy(r->Q.data(), s->dQ, sizeof(double) * s->nQ, cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(r->p.data(), s->dp, sizeof(double) * s->nP, cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(r->lam.data(), s->dl, sizeof(double) * s->nL, cudaMemcpyDeviceToHost) != cudaSuccess)
                return HDG_ERR_CUDA;
            r->t_done = now_ms();
            s->last_used = r->t_done;
            S->idle.push_back(s);
            r->slot = nullptr;
            S->done[r->id] = r;
            S->st.completed += 1;
        }
        S->active.swap(still);
    }
    S->st.active = (int)S->active.size();
    S->st.queued = (int)S->queue.size();
    S->st.bytes_in_use = S->bytes_in_use();
    if (stats) *stats = S->st;
    return HDG_OK;
}

hdg_status hdg_server_result(hdg_server *S, long long id, double *Q_host, double *p_host, double *lam_host,
                             double *latency_ms) {
    if (!S) return HDG_ERR_INVALID_ARG;
    auto it = S->done.find(id);
    if (it == S->done.end()) return HDG_ERR_INVALID_ARG;
    Request *r = it->second;
    if (Q_host) std::memcpy(Q_host, r->Q.data(), sizeof(double) * r->Q.size());
    if (p_host) std::memcpy(p_host, r->p.data(), sizeof(double) * r->p.size());
    if (lam_host) std::memcpy(lam_host, r->lam.data(), sizeof(double) * r->lam.size());
    if (latency_ms) *latency_ms = r->t_done - r->t_submit;
    S->done.erase(it);
    delete r;
    return HDG_OK;
}

void hdg_server_destroy(hdg_server *S) {
    if (!S) return;
    cudaSetDevice(S->device);
    for (Request *r : S->queue) delete r;
    for (Request *r : S->active) delete r;
    for (auto &kv : S->done) delete kv.second;
    for (Slot *s : S->slots) release_slot(s);
    delete S;
}

}  // extern "C"
