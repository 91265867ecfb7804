// Serving loop: continuous batching of independent solves over worker handles (declared with
// bm_server_create in bm.h).  Host-side runtime only: every computation goes through the handles'
// kernels.  Admission is first come, first served: the head of the queue waits until a worker is
// free and its device bytes fit beside the bytes of the requests in flight, so a large request is
// never overtaken indefinitely by small ones and the budget is never exceeded.
#include "common.cuh"
#include "kernels.cuh"

#include <chrono>
#include <condition_variable>
#include <deque>
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

namespace {

using clk = std::chrono::steady_clock;

double ms_since(clk::time_point a, clk::time_point b) { return std::chrono::duration<double, std::milli>(b - a).count(); }

struct Job {
    unsigned long long id;
    bm_request req;
    size_t bytes;
    clk::time_point t_submit;
};

}  // namespace

struct bm_server {
    int device = 0;
    int slots = 0;
    size_t budget = 0;
    bm_opts opts{};
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job> queue;
    std::map<unsigned long long, bm_result> done;
    std::map<unsigned long long, bool> collected;
    size_t in_flight_bytes = 0;
    int in_flight = 0;
    unsigned long long next_id = 1, submitted = 0, completed = 0;
    size_t max_bytes = 0;
    int max_in_flight = 0;
    bool stopping = false;
    std::vector<bm_ctx*> handles;
    std::vector<std::thread> workers;
};

namespace {

bm_result run_request(bm_server* s, int slot, const Job& j) {
    bm_ctx* h = s->handles[slot];
    const bm_request& r = j.req;
    bm_result res{};
    res.slot = slot;
    res.bytes = j.bytes;
    bm_status st = bm_assemble(h, &r.curve, r.N, r.k_out, r.k_in, (bm_formulation)r.formulation, &s->opts);
    int info = 0;
    if (st == BM_OK) st = bm_factor(h, &info);
    bm_solve_info si{};
    if (st == BM_OK) st = bm_solve(h, r.nrhs, r.B, r.ldb, r.X, r.ldx, 0, &si);
    res.status = st;
    res.iterations = si.iterations;
    res.backward_error = si.backward_error;
    ctx_release(h);  // the request's memory goes back before the next admission counts on it
    cudaStreamSynchronize(h->stream);
    return res;
}

void worker_loop(bm_server* s, int slot) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        s->cv_work.wait(lk, [&]() {
            if (s->queue.empty()) return s->stopping;
            return s->in_flight_bytes + s->queue.front().bytes <= s->budget;
        });
        if (s->queue.empty()) return;  // stopping and nothing left
        Job j = s->queue.front();
        s->queue.pop_front();
        s->in_flight_bytes += j.bytes;
        s->in_flight += 1;
        s->max_bytes = std::max(s->max_bytes, s->in_flight_bytes);
        s->max_in_flight = std::max(s->max_in_flight, s->in_flight);
        const clk::time_point t_admit = clk::now();
        lk.unlock();
        s->cv_work.notify_all();  // the next head may fit beside this one
        bm_result res = run_request(s, slot, j);
        const clk::time_point t_end = clk::now();
        res.t_queue_ms = ms_since(j.t_submit, t_admit);
        res.t_service_ms = ms_since(t_admit, t_end);
        lk.lock();
        s->in_flight_bytes -= j.bytes;
        s->in_flight -= 1;
        s->completed += 1;
        s->done[j.id] = res;
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
}

}  // namespace

extern "C" bm_status bm_server_create(bm_server** out, int device, const bm_server_opts* o) {
    if (out == nullptr || o == nullptr) return BM_EINVAL;
    *out = nullptr;
    if (o->slots < 1 || o->slots > 32) {
        bm_set_error("bm_server_create: slots must be in [1, 32]");
        return BM_EINVAL;
    }
    BM_CUDA_TRY(cudaSetDevice(device));
    bm_server* s = new bm_server();
    s->device = device;
    s->slots = o->slots;
    s->opts = o->opts;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    s->budget = o->hbm_budget_bytes ? o->hbm_budget_bytes : (size_t)(0.8 * (double)fr);
    for (int i = 0; i < s->slots; ++i) {
        bm_ctx* h = nullptr;
        bm_status st = bm_create(&h, device, nullptr, s->budget);
        if (st != BM_OK) {
            for (bm_ctx* q : s->handles) bm_destroy(q);
            delete s;
            return st;
        }
        s->handles.push_back(h);
    }
    for (int i = 0; i < s->slots; ++i) s->workers.emplace_back(worker_loop, s, i);
    *out = s;
    return BM_OK;
}

extern "C" bm_status bm_server_submit(bm_server* s, const bm_request* r, unsigned long long* ticket) {
    if (s == nullptr || r == nullptr || ticket == nullptr) return BM_EINVAL;
    if (r->N < 8 || r->nrhs < 1 || r->B == nullptr || r->X == nullptr ||
        (r->formulation != BM_MIXED && r->formulation != BM_ORDINARY))
        return BM_EINVAL;
    const int nsys = (r->formulation == BM_MIXED) ? 3 * r->N : 2 * r->N;
    if (r->ldb < nsys || r->ldx < nsys) return BM_EINVAL;
    const size_t bytes = request_bytes(r->N, r->formulation, s->opts.prec, s->opts.nb, r->nrhs);
    if (bytes > s->budget) {
        bm_set_error("bm_server_submit: the request needs " + std::to_string(bytes) + " bytes, more than the budget " +
                     std::to_string(s->budget));
        return BM_ENOMEM;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) return BM_ESTATE;
        Job j{s->next_id++, *r, bytes, clk::now()};
        *ticket = j.id;
        s->queue.push_back(j);
        s->submitted += 1;
    }
    s->cv_work.notify_all();
    return BM_OK;
}

extern "C" bm_status bm_server_wait(bm_server* s, unsigned long long ticket, bm_result* res) {
    if (s == nullptr || ticket == 0) return BM_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (ticket >= s->next_id || s->collected.count(ticket)) {
        bm_set_error("bm_server_wait: unknown or already collected ticket");
        return BM_EINVAL;
    }
    // a second waiter on the same ticket wakes when the first one collects it, instead of waiting
    // for a result that will never come back
    s->cv_done.wait(lk, [&]() { return s->done.count(ticket) != 0 || s->collected.count(ticket) != 0; });
    if (s->done.count(ticket) == 0) {
        bm_set_error("bm_server_wait: ticket collected by another waiter");
        return BM_EINVAL;
    }
    bm_result r = s->done[ticket];
    s->done.erase(ticket);
    s->collected[ticket] = true;
    s->cv_done.notify_all();  // any other waiter on this ticket returns BM_EINVAL
    if (res) *res = r;
    if (r.status != BM_OK) bm_set_error("bm_server: request " + std::to_string(ticket) + " failed with status " +
                                        std::to_string(r.status));
    return (bm_status)r.status;
}

extern "C" bm_status bm_server_stats_get(bm_server* s, bm_server_stats* st) {
    if (s == nullptr || st == nullptr) return BM_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->max_in_flight_bytes = s->max_bytes;
    st->max_in_flight = s->max_in_flight;
    st->budget_bytes = s->budget;
    return BM_OK;
}

extern "C" bm_status bm_server_destroy(bm_server* s) {
    if (s == nullptr) return BM_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    for (auto& t : s->workers) t.join();
    for (bm_ctx* h : s->handles) bm_destroy(h);
    delete s;
    return BM_OK;
}
