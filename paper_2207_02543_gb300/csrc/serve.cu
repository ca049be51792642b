// Serving worker: a request queue in front of one context. Requests (instance
// values, right-hand side, optional x0) are admitted into free slots between
// CUDA-graph launches of the batched PCG; an instance that converges retires and
// its slot is back-filled by the next waiting request, so work submitted while
// others are on the GPU joins the running batch (continuous batching). The
// FP64 context serves one request at a time on the plain path.
#include "common.cuh"

#include <chrono>
#include <cstring>

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static void finish(pod2g_ctx* c, ServeRequest* r, int status) {
    r->status = status;
    r->t_done = now_s();
    std::lock_guard<std::mutex> g(c->mu);
    c->inflight.erase(r->ticket);
    c->finished[r->ticket] = r;
}

static int serve_plain_one(pod2g_ctx* c, ServeRequest* r) {
    const size_t n = c->n;
    const size_t vb = sizeof(double) * instance_len(c);
    P2G_CUDA(cudaMemcpyAsync(c->d_stage, r->values.data(), vb, cudaMemcpyHostToDevice, c->stream));
    P2G_TRY(setup_instance(c, 0, c->d_stage));
    int st = 0;
    P2G_CUDA(cudaMemcpyAsync(&st, c->d_setup_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    P2G_CUDA(cudaStreamSynchronize(c->stream));
    if (st != POD2G_OK) { finish(c, r, st); return POD2G_OK; }
    P2G_CUDA(cudaMemcpyAsync(c->d_iob, r->b.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    if (r->has_x0)
        P2G_CUDA(cudaMemcpyAsync(c->d_iox, r->x0.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    int status = 0;
    P2G_TRY(plain_solve(c, 0, c->d_iob, r->has_x0 ? c->d_iox : nullptr, r->tol, r->maxit, c->d_iox, &r->iters,
                        &r->relres, &status));
    r->x.resize(n);
    P2G_CUDA(cudaMemcpyAsync(r->x.data(), c->d_iox, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    P2G_CUDA(cudaStreamSynchronize(c->stream));
    finish(c, r, status);
    return POD2G_OK;
}

static void worker_main(pod2g_ctx* c) {
    cudaSetDevice(c->device);
    const size_t n = c->n;
    const size_t vb = sizeof(double) * instance_len(c);
    std::vector<ServeRequest*> lane_req(c->B, nullptr);
    int fatal = POD2G_OK;
    while (true) {
        // ---- admission: free slots take waiting requests
        std::vector<ServeRequest*> joining;
        std::vector<int> jl;
        {
            std::unique_lock<std::mutex> lk(c->mu);
            bool any_active = false;
            for (auto* r : lane_req) any_active = any_active || r;
            if (!any_active && c->queue.empty() && !c->stop)
                c->cv.wait_for(lk, std::chrono::milliseconds(2));
            if (c->stop) break;
            if (c->precision == POD2G_FP64) {
                if (c->queue.empty()) continue;
                ServeRequest* r = c->queue.front();
                c->queue.pop_front();
                c->inflight[r->ticket] = r;
                lk.unlock();
                if (fatal == POD2G_OK) fatal = serve_plain_one(c, r);
                if (fatal != POD2G_OK) finish(c, r, fatal);
                continue;
            }
            for (int b = 0; b < c->B && !c->queue.empty(); ++b) {
                if (lane_req[b]) continue;
                ServeRequest* r = c->queue.front();
                c->queue.pop_front();
                c->inflight[r->ticket] = r;
                r->slot = b;
                lane_req[b] = r;
                joining.push_back(r);
                jl.push_back(b);
            }
        }
        if (fatal != POD2G_OK) {
            for (auto*& r : lane_req)
                if (r) { finish(c, r, fatal); r = nullptr; }
            continue;
        }
        // ---- per-instance set-up of the joining slots, then their initial pass
        if (!joining.empty()) {
            std::vector<ServeRequest*> ok_req;
            std::vector<int> ok_lane;
            for (size_t i = 0; i < joining.size() && fatal == POD2G_OK; ++i) {
                ServeRequest* r = joining[i];
                int b = jl[i];
                const bool ok_setup =
                    r->theta
                        ? cudaMemcpyAsync(c->d_theta + (size_t)b * c->field_m, r->values.data(),
                                          sizeof(double) * c->field_m, cudaMemcpyHostToDevice, c->stream) ==
                                  cudaSuccess &&
                              setup_theta(c, b, c->d_theta + (size_t)b * c->field_m) == POD2G_OK
                        : cudaMemcpyAsync(c->d_stage, r->values.data(), vb, cudaMemcpyHostToDevice, c->stream) ==
                                  cudaSuccess &&
                              setup_instance(c, b, c->d_stage) == POD2G_OK;
                if (!ok_setup) {
                    fatal = POD2G_CUDA_ERROR;
                    break;
                }
                int st = 0;
                cudaMemcpyAsync(&st, c->d_setup_status + b, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
                if (cudaStreamSynchronize(c->stream) != cudaSuccess) { fatal = POD2G_CUDA_ERROR; break; }
                if (st != POD2G_OK) {
                    lane_req[b] = nullptr;
                    finish(c, r, st);
                    continue;
                }
                size_t row = ok_req.size();
                cudaMemcpyAsync(c->d_iob + row * n, r->b.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream);
                if (r->has_x0)
                    cudaMemcpyAsync(c->d_iox + row * n, r->x0.data(), sizeof(double) * n, cudaMemcpyHostToDevice,
                                    c->stream);
                else
                    cudaMemsetAsync(c->d_iox + row * n, 0, sizeof(double) * n, c->stream);
                ok_req.push_back(r);
                ok_lane.push_back(b);
            }
            if (fatal == POD2G_OK && !ok_req.empty()) {
                std::vector<double> tol(ok_req.size());
                std::vector<int> maxit(ok_req.size());
                for (size_t i = 0; i < ok_req.size(); ++i) { tol[i] = ok_req[i]->tol; maxit[i] = ok_req[i]->maxit; }
                fatal = batched_load(c, (int)ok_req.size(), ok_lane.data(), c->d_iob, c->d_iox, tol.data(),
                                     maxit.data());
                if (fatal == POD2G_OK) {
                    cudaMemcpyAsync(c->h_sc, c->d_sc, sizeof(SlotScalars) * c->Bp, cudaMemcpyDeviceToHost, c->stream);
                    if (cudaStreamSynchronize(c->stream) != cudaSuccess) fatal = POD2G_CUDA_ERROR;
                }
            }
            if (fatal != POD2G_OK) continue;
        } else {
            bool any_active = false;
            for (auto* r : lane_req) any_active = any_active || r;
            if (!any_active) continue;
            // ---- one chunk of lockstep iterations for every ACTIVE slot
            fatal = batched_chunk(c);
            if (fatal != POD2G_OK) continue;
        }
        // ---- retire finished slots
        std::vector<int> done;
        for (int b = 0; b < c->B; ++b)
            if (lane_req[b] && c->h_sc[b].state == SLOT_DONE) done.push_back(b);
        if (done.empty()) continue;
        std::vector<int> it(done.size()), st(done.size());
        std::vector<double> rel(done.size());
        fatal = batched_finalize(c, (int)done.size(), done.data(), c->d_iox, it.data(), rel.data(), st.data());
        if (fatal != POD2G_OK) continue;
        for (size_t i = 0; i < done.size(); ++i) {
            ServeRequest* r = lane_req[done[i]];
            r->x.resize(n);
            cudaMemcpyAsync(r->x.data(), c->d_iox + i * n, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream);
        }
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) { fatal = POD2G_CUDA_ERROR; continue; }
        for (size_t i = 0; i < done.size(); ++i) {
            int b = done[i];
            ServeRequest* r = lane_req[b];
            r->iters = it[i];
            r->relres = rel[i];
            c->h_sc[b].state = SLOT_IDLE;
            lane_req[b] = nullptr;
            finish(c, r, st[i]);
        }
        // mark retired lanes IDLE on the device too
        for (int b : done) {
            cudaMemcpyAsync(c->d_sc + b, &c->h_sc[b], sizeof(SlotScalars), cudaMemcpyHostToDevice, c->stream);
        }
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) fatal = POD2G_CUDA_ERROR;
    }
    // shutting down: fail whatever is still running
    for (auto* r : lane_req)
        if (r) finish(c, r, POD2G_NOT_CONVERGED);
}

extern "C" {

int pod2g_serve_start(pod2g_t c, int max_queue) {
    if (!c || max_queue < 1) return POD2G_INVALID_ARG;
    std::lock_guard<std::mutex> g(c->mu);
    if (c->serving) return POD2G_INVALID_ARG;
    c->max_queue = max_queue;
    c->stop = false;
    c->serving = true;
    c->worker = std::thread(worker_main, c);
    return POD2G_OK;
}

int pod2g_submit(pod2g_t c, const double* values, const double* b, const double* x0, double tol, int maxit,
                 uint64_t* ticket) {
    if (!c || !values || !b || !ticket || !(tol >= 0.0) || maxit < 0) return POD2G_INVALID_ARG;
    const size_t n = c->n;
    const size_t nv = instance_len(c);
    {
        std::lock_guard<std::mutex> g(c->mu);
        if (!c->serving) return POD2G_INVALID_ARG;
        if ((int)c->queue.size() >= c->max_queue) return POD2G_ADMISSION;
    }
    ServeRequest* r = new ServeRequest();
    r->values.assign(values, values + nv);
    r->b.assign(b, b + n);
    if (x0) { r->x0.assign(x0, x0 + n); r->has_x0 = true; }
    r->tol = tol;
    r->maxit = maxit;
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> g(c->mu);
        r->ticket = c->next_ticket++;
        *ticket = r->ticket;
        c->queue.push_back(r);
    }
    c->cv.notify_one();
    return POD2G_OK;
}

int pod2g_submit_theta(pod2g_t c, const double* theta, const double* b, const double* x0, double tol, int maxit,
                       uint64_t* ticket) {
    if (!c || !theta || !b || !ticket || !(tol >= 0.0) || maxit < 0) return POD2G_INVALID_ARG;
    if (!c->elem || c->field_m == 0) return POD2G_INVALID_ARG;
    const size_t n = c->n;
    {
        std::lock_guard<std::mutex> g(c->mu);
        if (!c->serving) return POD2G_INVALID_ARG;
        if ((int)c->queue.size() >= c->max_queue) return POD2G_ADMISSION;
    }
    ServeRequest* r = new ServeRequest();
    r->values.assign(theta, theta + c->field_m);
    r->theta = true;
    r->b.assign(b, b + n);
    if (x0) { r->x0.assign(x0, x0 + n); r->has_x0 = true; }
    r->tol = tol;
    r->maxit = maxit;
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> g(c->mu);
        r->ticket = c->next_ticket++;
        *ticket = r->ticket;
        c->queue.push_back(r);
    }
    c->cv.notify_one();
    return POD2G_OK;
}

int pod2g_poll(pod2g_t c, uint64_t ticket, double* x, int* iters, double* relres, int* status, double* latency_s) {
    if (!c) return POD2G_INVALID_ARG;
    ServeRequest* r = nullptr;
    {
        std::lock_guard<std::mutex> g(c->mu);
        auto it = c->finished.find(ticket);
        if (it == c->finished.end()) {
            if (c->inflight.count(ticket)) return POD2G_PENDING;
            for (auto* q : c->queue)
                if (q->ticket == ticket) return POD2G_PENDING;
            return POD2G_INVALID_ARG;
        }
        r = it->second;
        c->finished.erase(it);
    }
    if (x && !r->x.empty()) std::memcpy(x, r->x.data(), sizeof(double) * r->x.size());
    if (iters) *iters = r->iters;
    if (relres) *relres = r->relres;
    if (status) *status = r->status;
    if (latency_s) *latency_s = r->t_done - r->t_submit;
    delete r;
    return POD2G_OK;
}

int pod2g_serve_stop(pod2g_t c) {
    if (!c) return POD2G_INVALID_ARG;
    {
        std::lock_guard<std::mutex> g(c->mu);
        if (!c->serving) return POD2G_OK;
        c->stop = true;
    }
    c->cv.notify_all();
    if (c->worker.joinable()) c->worker.join();
    std::lock_guard<std::mutex> g(c->mu);
    c->serving = false;
    for (auto* r : c->queue) { r->status = POD2G_NOT_CONVERGED; c->finished[r->ticket] = r; }
    c->queue.clear();
    return POD2G_OK;
}

}  // extern "C"
