// Continuous-batching request server for encrypted matrix products,
// composite sign/ReLU jobs and rotations.
//
// Requests queue on the host.  A dispatcher thread forms a batch from the
// oldest pending request and every other pending request with the same
// signature (context, kind, h or (d, k, relu), level) whenever a lane (a CUDA
// stream with its worker thread) is idle and the batch's estimated device
// memory fits in what the HBM budget leaves after the resident keys.  Lanes run
// their batches concurrently, so requests that arrive while others are on the
// GPU are admitted as lanes and memory free up.  A batch's results are views
// into its output buffer, equal to what the same request computes alone.
// Rotations batch across rings: pending rotations of any contexts and levels
// form one batch, run as one launch per key-switching stage (rotate_jobs).
// A request may carry a deadline: if it is still queued when its deadline
// passes, it completes with HX_ETIMEOUT and no GPU work (a batch already on
// the GPU always runs to the end).
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>

#include "runtime.h"

using namespace hx;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
    uint64_t id = 0;
    int kind = 0;  // 0 matmul, 1 sign, 2 rotation (of any ring: batches span contexts)
    hx_context *ctx = nullptr;
    const hx_keyset *ks = nullptr;
    Cts a, b;
    int h = 0, d = 0, k = 0, relu = 0;
    uint64_t seed = 0;
    int64_t step = 0;
    Clock::time_point t0, deadline = Clock::time_point::max();
    size_t est = 0;
};

struct Done {
    uint64_t id;
    int status;
    hx_context *ctx;
    Cts out;
    double latency_ms;
};

bool same_batch(const Request &x, const Request &y)
{
    if (x.kind == 2 || y.kind == 2) return x.kind == y.kind;  // rotations of every ring batch together
    return x.ctx == y.ctx && x.ks == y.ks && x.kind == y.kind && x.a.limbs == y.a.limbs && x.a.scale == y.a.scale &&
           (x.kind == 0 ? (x.h == y.h && x.b.limbs == y.b.limbs && x.b.scale == y.b.scale)
                        : (x.d == y.d && x.k == y.k && x.relu == y.relu));
}

// conservative device-memory estimate of one batch entry (workspace included)
size_t estimate(const Request &r)
{
    const size_t ct = (size_t)2 * r.a.limbs * r.ctx->N * 8;
    if (r.kind == 2) {  // sigma(c1) and its copy, ModUp's digits, the extended pair, the conversion, the output
        const size_t ext = (size_t)r.a.limbs + r.ctx->K, nd = ((size_t)r.a.limbs + r.ctx->alpha - 1) / r.ctx->alpha;
        return ((size_t)4 * r.a.limbs + (nd + 2) * ext + 2 * (size_t)r.a.limbs) * r.ctx->N * 8 + ct;
    }
    return r.kind == 0 ? 48 * ct : 24 * ct + (size_t)2 * r.ctx->n_q * r.ctx->N * 8;
}

size_t key_bytes(const hx_keyset &ks)
{
    size_t b = ks.relin.buf ? ks.relin.buf->words * 8 : 0;
    for (auto &kv : ks.rot) b += kv.second.buf->words * 8;
    return b;
}

} // namespace

struct hx_server {
    size_t budget = 0, keys = 0, admitted = 0, peak = 0;
    int max_batch = 16;
    std::mutex mu;
    std::condition_variable cv_dispatch, cv_done;
    std::deque<Request> pending;
    std::deque<Done> done;
    uint64_t next_id = 1, n_batches = 0, n_done = 0, max_seen_batch = 0, max_busy = 0, n_inflight = 0;
    uint64_t n_expired = 0;
    bool stop = false, paused = false;
    struct Lane {
        cudaStream_t s = nullptr;
        std::thread th;
        std::vector<Request> batch;
        size_t est = 0;
        bool busy = false;
        std::condition_variable cv;
    };
    std::vector<std::unique_ptr<Lane>> lanes;
    std::thread dispatcher;
    std::vector<const hx_keyset *> registered;
    int device = 0;

    void run_lane(Lane &L);
    void run_dispatch();
    Clock::time_point expire_pending();  // returns the earliest deadline still ahead
};

Clock::time_point hx_server::expire_pending()
{
    const auto now = Clock::now();
    Clock::time_point next = Clock::time_point::max();
    bool any = false;
    for (auto it = pending.begin(); it != pending.end();) {
        if (it->deadline > now) {
            next = std::min(next, it->deadline);
            ++it;
            continue;
        }
        Done d;
        d.id = it->id;
        d.status = HX_ETIMEOUT;
        d.ctx = it->ctx;
        d.latency_ms = std::chrono::duration<double, std::milli>(now - it->t0).count();
        done.push_back(std::move(d));
        n_done++;
        n_expired++;
        any = true;
        it = pending.erase(it);  // drops the request's references to its inputs
    }
    if (any) cv_done.notify_all();
    return next;
}

void hx_server::run_dispatch()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (!stop) {
        const Clock::time_point next = expire_pending();
        auto sleep = [&] {
            if (next == Clock::time_point::max()) cv_dispatch.wait(lk);
            else cv_dispatch.wait_until(lk, next);
        };
        Lane *idle = nullptr;
        for (auto &l : lanes)
            if (!l->busy) {
                idle = l.get();
                break;
            }
        if (pending.empty() || !idle || paused) {
            sleep();
            continue;
        }
        // the oldest request leads; others with its signature join while they fit
        std::vector<Request> batch;
        size_t est = 0;
        for (auto it = pending.begin(); it != pending.end() && (int)batch.size() < max_batch;) {
            if (!batch.empty() && !same_batch(*it, batch[0])) {
                ++it;
                continue;
            }
            if (admitted + est + it->est > budget) break;
            est += it->est;
            batch.push_back(std::move(*it));
            it = pending.erase(it);
        }
        if (batch.empty()) {  // the head does not fit yet: wait for memory to free up
            sleep();
            continue;
        }
        admitted += est;
        peak = std::max(peak, admitted);
        n_batches++;
        max_seen_batch = std::max<uint64_t>(max_seen_batch, batch.size());
        idle->batch = std::move(batch);
        idle->est = est;
        idle->busy = true;
        n_inflight++;
        max_busy = std::max(max_busy, n_inflight);
        idle->cv.notify_one();
    }
}

void hx_server::run_lane(Lane &L)
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        L.cv.wait(lk, [&] { return stop || L.busy; });
        if (stop && !L.busy) return;
        std::vector<Request> batch = std::move(L.batch);
        lk.unlock();
        const Request &r0 = batch[0];
        hx_context &ctx = *r0.ctx;
        int status = HX_OK;
        Cts out;
        std::vector<Cts> rot_out;  // rotations: one result per request, of its own context
        std::shared_ptr<const hx_matmul_plan> plan;
        try {
            if (r0.kind == 2) {
                std::vector<RotateJob> jobs;
                for (auto &r : batch) jobs.push_back(RotateJob{r.ctx, r.ks, r.a, r.step});
                rot_out = rotate_jobs(jobs, L.s);
                HX_CUDA(cudaStreamSynchronize(L.s));
                for (auto &o : rot_out) o.buf->stream = nullptr;  // results outlive the lane's stream
            } else {
                Eval ev(ctx, L.s);
                const int B = (int)batch.size();
                Cts A = ev.alloc(B, 2, r0.a.limbs);
                A.scale = r0.a.scale;
                const size_t N = ctx.N;
                auto pack = [&](Cts &dst, int i, const Cts &src) {
                    for (int c = 0; c < 2; c++)
                        HX_CUDA(cudaMemcpyAsync(dst.d + i * dst.bstride(N) + c * dst.cstride(N),
                                                src.d + c * src.cstride(N), sizeof(uint64_t) * dst.limbs * N,
                                                cudaMemcpyDeviceToDevice, L.s));
                };
                for (int i = 0; i < B; i++) pack(A, i, batch[i].a);
                if (r0.kind == 0) {
                    Cts Bc = ev.alloc(B, 2, r0.b.limbs);
                    Bc.scale = r0.b.scale;
                    for (int i = 0; i < B; i++) pack(Bc, i, batch[i].b);
                    plan = cached_plan(ctx, r0.h, r0.a.limbs);  // held until the lane's stream is done
                    out = matmul_batch(ctx, *r0.ks, *plan, A, Bc, L.s);
                } else {
                    std::vector<uint64_t> seeds;
                    for (auto &r : batch) seeds.push_back(r.seed);
                    out = sign_batch(ctx, *r0.ks, A, r0.d, r0.k, r0.relu != 0, true, seeds, L.s);
                }
                HX_CUDA(cudaStreamSynchronize(L.s));
                out.buf->stream = nullptr;  // results outlive the lane's stream
            }
        } catch (const hx::Error &e) {
            status = e.code;
            cudaStreamSynchronize(L.s);
        }
        const auto t1 = Clock::now();
        plan.reset();
        lk.lock();
        for (size_t i = 0; i < batch.size(); i++) {
            Done d;
            d.id = batch[i].id;
            d.status = status;
            d.ctx = batch[i].ctx;
            if (status == HX_OK && r0.kind == 2) {
                d.out = rot_out[i];
            } else if (status == HX_OK) {
                d.out = out;
                d.out.B = 1;
                d.out.d = out.d + i * out.bstride(ctx.N);
            }
            d.latency_ms = std::chrono::duration<double, std::milli>(t1 - batch[i].t0).count();
            done.push_back(std::move(d));
            n_done++;
        }
        batch.clear();  // drops this lane's references to the inputs
        admitted -= L.est;
        L.busy = false;
        n_inflight--;
        cv_dispatch.notify_one();
        cv_done.notify_all();
    }
}

extern "C" {

hx_status hx_server_create(size_t hbm_budget_bytes, int n_lanes, int max_batch, hx_server **out)
{
    try {
        HX_CHECK(out && n_lanes >= 1 && n_lanes <= 64 && max_batch >= 1 && max_batch <= 4096, HX_EINVAL,
                 "bad server arguments");
        *out = nullptr;
        std::unique_ptr<hx_server> sv(new hx_server);
        sv->budget = hbm_budget_bytes;
        sv->max_batch = max_batch;
        HX_CUDA(cudaGetDevice(&sv->device));
        for (int i = 0; i < n_lanes; i++) {
            sv->lanes.emplace_back(new hx_server::Lane);
            HX_CUDA(cudaStreamCreateWithFlags(&sv->lanes.back()->s, cudaStreamNonBlocking));
        }
        hx_server *p = sv.get();
        for (auto &l : sv->lanes) {
            hx_server::Lane *lp = l.get();
            l->th = std::thread([p, lp] { p->run_lane(*lp); });
        }
        sv->dispatcher = std::thread([p] { p->run_dispatch(); });
        *out = sv.release();
        return HX_OK;
    } catch (const hx::Error &e) {
        set_error(e.msg);
        return e.code;
    }
}

hx_status hx_server_register_keys(hx_server *sv, const hx_keyset *ks)
{
    if (!sv || !ks) return HX_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    for (auto *k : sv->registered)
        if (k == ks) return HX_OK;
    const size_t kb = key_bytes(*ks);
    if (kb > sv->budget) {  // the budget is already net of the keys registered before
        set_error("resident keys exceed the HBM budget");
        return HX_ENOMEM;
    }
    sv->registered.push_back(ks);
    sv->keys += kb;
    sv->budget -= kb;
    return HX_OK;
}

static hx_status submit(hx_server *sv, Request &&r, uint64_t *id)
{
    if (!sv || !id) return HX_EINVAL;
    r.est = estimate(r);
    std::lock_guard<std::mutex> lk(sv->mu);
    if (r.est > sv->budget) {
        set_error("request needs more device memory than the budget allows");
        return HX_ENOMEM;
    }
    r.id = sv->next_id++;
    r.t0 = Clock::now();
    *id = r.id;
    sv->pending.push_back(std::move(r));
    sv->cv_dispatch.notify_one();
    return HX_OK;
}

hx_status hx_server_submit_matmul(hx_server *sv, hx_context *ctx, const hx_keyset *ks, const hx_ct *A,
                                  const hx_ct *B, int h, uint64_t *id)
{
    if (!ctx || !ks || !A || !B) return HX_EINVAL;
    if (ks->ctx != ctx || A->ctx != ctx || B->ctx != ctx) {
        set_error("keys or ciphertexts of another context");
        return HX_EINVAL;
    }
    if (A->c.limbs != B->c.limbs || A->c.comps != 2 || B->c.comps != 2) {
        set_error("A and B must be ciphertexts at one level");
        return HX_ESCALE;
    }
    Request r;
    r.kind = 0;
    r.ctx = ctx;
    r.ks = ks;
    r.a = A->c;
    r.b = B->c;
    r.h = h;
    return submit(sv, std::move(r), id);
}

hx_status hx_server_submit_sign(hx_server *sv, hx_context *ctx, const hx_keyset *ks, const hx_ct *x, int d, int k,
                                int relu, uint64_t refresh_seed, uint64_t *id)
{
    if (!ctx || !ks || !x || x->c.comps != 2) return HX_EINVAL;
    if (ks->ctx != ctx || x->ctx != ctx) {
        set_error("keys or ciphertext of another context");
        return HX_EINVAL;
    }
    Request r;
    r.kind = 1;
    r.ctx = ctx;
    r.ks = ks;
    r.a = x->c;
    r.d = d;
    r.k = k;
    r.relu = relu;
    r.seed = refresh_seed;
    return submit(sv, std::move(r), id);
}

hx_status hx_server_submit_rotate(hx_server *sv, hx_context *ctx, const hx_keyset *ks, const hx_ct *x, int64_t step,
                                  uint64_t *id)
{
    if (!ctx || !ks || !x || x->c.comps != 2) return HX_EINVAL;
    if (ks->ctx != ctx || x->ctx != ctx) {
        set_error("keys or ciphertext of another context");
        return HX_EINVAL;
    }
    Request r;
    r.kind = 2;
    r.ctx = ctx;
    r.ks = ks;
    r.a = x->c;
    r.step = step;
    return submit(sv, std::move(r), id);
}

int hx_server_poll(hx_server *sv, int wait, uint64_t *ids, hx_ct **results, int32_t *status, double *latency_ms,
                   int cap)
{
    if (!sv || cap < 0) return HX_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (wait && sv->done.empty() && (!sv->pending.empty() || sv->n_inflight))
        sv->cv_done.wait(lk, [&] { return !sv->done.empty() || (sv->pending.empty() && !sv->n_inflight); });
    int n = 0;
    while (n < cap && !sv->done.empty()) {
        Done &d = sv->done.front();
        ids[n] = d.id;
        status[n] = d.status;
        latency_ms[n] = d.latency_ms;
        results[n] = nullptr;
        if (d.status == HX_OK) {
            hx_ct *h = new hx_ct;
            h->ctx = d.ctx;
            h->c = d.out;
            results[n] = h;
        }
        sv->done.pop_front();
        n++;
    }
    return n;
}

int hx_server_stats(hx_server *sv, uint64_t *out, int cap)
{
    if (!sv) return HX_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    const uint64_t v[9] = {sv->n_done, sv->n_batches, sv->max_seen_batch, sv->max_busy, sv->peak, sv->keys,
                           sv->budget, (uint64_t)sv->pending.size(), sv->n_expired};
    for (int i = 0; i < 9 && i < cap; i++) out[i] = v[i];
    return 9;
}

hx_status hx_server_set_deadline(hx_server *sv, uint64_t id, double ms)
{
    if (!sv || !(ms >= 0)) return HX_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    for (auto &r : sv->pending)
        if (r.id == id) {
            r.deadline = r.t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double, std::milli>(ms));
            sv->cv_dispatch.notify_one();
            return HX_OK;
        }
    set_error("request " + std::to_string(id) + " is not queued (already dispatched, completed or unknown)");
    return HX_EINVAL;
}

hx_status hx_server_pause(hx_server *sv, int paused)
{
    if (!sv) return HX_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->paused = paused != 0;
    sv->cv_dispatch.notify_one();
    return HX_OK;
}

void hx_server_destroy(hx_server *sv)
{
    if (!sv) return;
    {
        std::unique_lock<std::mutex> lk(sv->mu);
        sv->paused = false;
        sv->cv_dispatch.notify_one();
        sv->cv_done.wait(lk, [&] { return sv->pending.empty() && !sv->n_inflight; });
        sv->stop = true;
        sv->cv_dispatch.notify_all();
        for (auto &l : sv->lanes) l->cv.notify_all();
    }
    sv->dispatcher.join();
    for (auto &l : sv->lanes) {
        l->th.join();
        cudaStreamDestroy(l->s);
    }
    delete sv;
}

} // extern "C"
