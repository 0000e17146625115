// Serving: continuous batching of KSG CMI jobs (te_serve_*).
//
// Jobs are the requests that independent greedy loops emit (a candidate and
// its surrogates for one target; Supporting Information, Run-time on CPU and
// GPU: targets are independent and can run concurrently).  Callers submit
// them from any thread; a scheduler thread admits pending jobs in arrival
// order while their device-memory footprint fits the budget, fuses each
// admitted set into one batch (shared-group fusion and one permutation launch,
// as cmi_ksg_batch) and keeps up to max_inflight batches on the device at
// once, each on its own stream with its own workspaces.  Jobs that arrive
// while batches run join the next batch as soon as a slot and memory free up.
// Results do not depend on which batch a job lands in: every key is exact.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "te_runtime.h"

using namespace teksg;

namespace {

enum JobState { JS_PENDING, JS_RUNNING, JS_DONE, JS_CANCELLED, JS_FAILED };

struct ServeJob {
    te_ticket id = 0;
    const te_data *data = nullptr;
    std::vector<te_var> x, y, z;
    te_ksg_params p{};
    int N = 0, S = 0;
    size_t fp = 0;
    int state = JS_PENDING;
    bool cancel_requested = false;
    te_status err = TE_OK;
    std::vector<int64_t> keys;
    std::vector<double> cmi;
};

struct Slot {
    te_ctx *ctx = nullptr;
    bool busy = false;
    cudaEvent_t done = nullptr;
    std::vector<ServeJob *> jobs;
    std::vector<int> out0;
    int n_out = 0;
    int64_t *keys_pin = nullptr;
    size_t keys_cap = 0;
    size_t fp = 0;
};

// device bytes of one job: permutations and their composed copies (8 S N),
// the X-value rows of the TMA-staged kernel (4 (S + 1) N, rows padded to a
// multiple of 8 points), the order and sorted Y/Z columns, the chunk boxes,
// accumulators, keys and descriptors
size_t footprint(int N, int S, int dyz)
{
    const size_t pitch = (size_t)std::max(32, (N + 7) & ~7);
    return (size_t)S * N * 8 + (size_t)(S + 1) * pitch * 4 + (size_t)N * (4 + 4 * (size_t)dyz) +
           8 * (size_t)dyz * (N / 8 + 1) + 64 * (size_t)(S + 1) + 4096;
}

}  // namespace

struct te_server {
    te_ctx *owner = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ServeJob *> pending;
    std::unordered_map<te_ticket, ServeJob *> jobs;
    std::vector<Slot> slots;
    std::thread th;
    bool stop = false;
    size_t budget = 0, in_use = 0, peak = 0;
    int max_batch = 0;
    te_ticket next = 1;
    te_serve_stats st{};
    std::string err;
};

namespace {

// Build and queue one batch on the slot's stream (no host wait).
te_status launch_batch(Slot &sl)
{
    te_ctx *ctx = sl.ctx;
    te_status st;
    size_t perm_elems = 0;
    int n_out = 0;
    sl.out0.resize(sl.jobs.size());
    std::vector<size_t> perm_at(sl.jobs.size());
    int max_n = 0;
    for (size_t a = 0; a < sl.jobs.size(); ++a) {
        ServeJob *j = sl.jobs[a];
        sl.out0[a] = n_out;
        n_out += j->S + 1;
        perm_at[a] = perm_elems;
        perm_elems += (size_t)j->S * j->N;
        max_n = std::max(max_n, j->N);
    }
    sl.n_out = n_out;
    if ((st = ensure_dev(ctx, ctx->ws_perm, std::max<size_t>(perm_elems, 1) * 4))) return st;
    int32_t *perm = (int32_t *)ctx->ws_perm.p;
    std::vector<PermJob> pj;
    long long total = 0;
    for (size_t a = 0; a < sl.jobs.size(); ++a) {
        ServeJob *j = sl.jobs[a];
        if (j->S == 0) continue;
        PermJob q;
        q.out = perm + perm_at[a];
        q.n = j->N;
        q.n_perm = j->S;
        q.s_first = 1;
        q.seed = j->p.seed;
        q.target = j->p.stream_tag;
        q.stage = 0;
        q.iter = 0;
        q.perm_begin = total;
        total += j->S;
        pj.push_back(q);
    }
    if (!pj.empty()) {
        const size_t bytes = pj.size() * sizeof(PermJob);
        if ((st = ensure_dev(ctx, ctx->ws_stat, bytes + 16))) return st;
        // pageable source: the copy has left pj when the call returns
        CK(cudaMemcpyAsync(ctx->ws_stat.p, pj.data(), bytes, cudaMemcpyHostToDevice, ctx->stream),
           "cudaMemcpyAsync");
        CK(launch_perms_multi((const PermJob *)ctx->ws_stat.p, (int)pj.size(), total, max_n,
                              ctx->stream),
           "permutation launch");
        ctx->stats.launches++;
    }
    std::map<std::vector<long long>, int> gid;
    std::vector<HostGroup> groups;
    for (size_t a = 0; a < sl.jobs.size(); ++a) {
        ServeJob *j = sl.jobs[a];
        std::vector<long long> key{(long long)(uintptr_t)j->data, j->p.max_lag, j->p.k,
                                   j->p.theiler, (long long)j->x.size(), (long long)j->y.size(),
                                   (long long)j->z.size()};
        for (const te_var &v : j->y) key.push_back(((long long)v.proc << 32) | v.lag);
        key.push_back(-1);
        for (const te_var &v : j->z) key.push_back(((long long)v.proc << 32) | v.lag);
        auto it = gid.find(key);
        int g;
        if (it == gid.end()) {
            g = (int)groups.size();
            gid[key] = g;
            HostGroup hg;
            hg.data = j->data;
            hg.max_lag = j->p.max_lag;
            hg.k = j->p.k;
            hg.theiler = j->p.theiler;
            hg.y = j->y;
            hg.z = j->z;
            hg.dx = (int)j->x.size();
            groups.push_back(hg);
        } else {
            g = it->second;
        }
        HostGroup &hg = groups[g];
        const int xfirst = (int)hg.xvars.size();
        hg.xvars.insert(hg.xvars.end(), j->x.begin(), j->x.end());
        for (int s = 0; s <= j->S; ++s)
            hg.members.push_back(HostMember{
                xfirst, s == 0 ? nullptr : perm + perm_at[a] + (size_t)(s - 1) * j->N,
                sl.out0[a] + s});
    }
    if ((st = launch_groups(ctx, groups, n_out))) return st;
    if ((size_t)n_out * 16 > sl.keys_cap) {
        if (sl.keys_pin) {
            CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
            CK(cudaFreeHost(sl.keys_pin), "cudaFreeHost");
            sl.keys_pin = nullptr;
        }
        const size_t want = std::max((size_t)n_out * 16, sl.keys_cap * 2);
        CK(cudaMallocHost(&sl.keys_pin, want), "cudaMallocHost");
        sl.keys_cap = want;
    }
    CK(copy_d2h(ctx, sl.keys_pin, ctx->ws_keys.p, (size_t)n_out * 16), "cudaMemcpyAsync");
    CK(cudaEventRecord(sl.done, ctx->stream), "cudaEventRecord");
    return TE_OK;
}

void serve_loop(te_server *S)
{
    cudaSetDevice(S->owner->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool progressed = false;
        // completions
        for (Slot &sl : S->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) continue;
            lk.unlock();
            const te_status fst = q == cudaSuccess ? finish_groups(sl.ctx) : TE_ECUDA;
            lk.lock();
            for (size_t a = 0; a < sl.jobs.size(); ++a) {
                ServeJob *j = sl.jobs[a];
                if (j->cancel_requested) {
                    j->state = JS_CANCELLED;
                    S->st.cancelled++;
                    continue;
                }
                if (fst) {
                    j->state = JS_FAILED;
                    j->err = fst;
                    continue;
                }
                j->keys.assign(sl.keys_pin + 2 * (size_t)sl.out0[a],
                               sl.keys_pin + 2 * (size_t)(sl.out0[a] + j->S + 1));
                j->cmi.resize(j->S + 1);
                for (int s = 0; s <= j->S; ++s)
                    j->cmi[s] = key_to_cmi(sl.ctx, j->keys[2 * s], (uint64_t)j->keys[2 * s + 1],
                                           j->p.k, j->N);
                j->state = JS_DONE;
                S->st.completed++;
            }
            S->in_use -= sl.fp;
            sl.fp = 0;
            sl.jobs.clear();
            sl.busy = false;
            progressed = true;
            S->cv_done.notify_all();
        }
        // admissions: arrival order, footprint within the budget
        for (Slot &sl : S->slots) {
            if (sl.busy) continue;
            std::vector<ServeJob *> batch;
            size_t fp = 0;
            while (!S->pending.empty() && (int)batch.size() < S->max_batch) {
                ServeJob *j = S->pending.front();
                if (S->in_use + fp + j->fp > S->budget) break;
                S->pending.pop_front();
                fp += j->fp;
                j->state = JS_RUNNING;
                batch.push_back(j);
            }
            if (batch.empty()) break;
            S->in_use += fp;
            S->peak = std::max(S->peak, S->in_use);
            sl.jobs = batch;
            sl.fp = fp;
            sl.busy = true;
            S->st.batches++;
            lk.unlock();
            const te_status lst = launch_batch(sl);
            lk.lock();
            if (lst) {
                for (ServeJob *j : sl.jobs) {
                    j->state = JS_FAILED;
                    j->err = lst;
                }
                S->in_use -= sl.fp;
                sl.fp = 0;
                sl.jobs.clear();
                sl.busy = false;
                S->cv_done.notify_all();
            }
            progressed = true;
        }
        bool any_busy = false;
        for (Slot &sl : S->slots) any_busy |= sl.busy;
        if (S->stop && !any_busy && S->pending.empty()) break;
        if (!progressed) {
            if (any_busy) S->cv_work.wait_for(lk, std::chrono::microseconds(50));
            else S->cv_work.wait(lk);
        }
    }
}

te_status start_server(te_ctx *ctx, const te_serve_config *cfg)
{
    if (ctx->server) return TE_OK;
    te_server *S = new te_server();
    S->owner = ctx;
    S->budget = cfg && cfg->hbm_budget_bytes ? cfg->hbm_budget_bytes : ((size_t)4 << 30);
    int inflight = cfg && cfg->max_inflight ? cfg->max_inflight : 2;
    S->max_batch = cfg && cfg->max_batch_jobs ? cfg->max_batch_jobs : 2048;
    if (inflight < 1 || inflight > 8 || S->max_batch < 1) {
        delete S;
        return fail(ctx, TE_EINVAL, "max_inflight must be 1..8 and max_batch_jobs >= 1");
    }
    S->slots.resize(inflight);
    for (Slot &sl : S->slots) {
        te_status st = te_ctx_create(ctx->device, &sl.ctx);
        if (st == TE_OK && cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess)
            st = TE_ECUDA;
        if (st) {
            for (Slot &o : S->slots) {
                if (o.done) cudaEventDestroy(o.done);
                if (o.ctx) te_ctx_destroy(o.ctx);
            }
            delete S;
            return fail(ctx, st, "could not create the serving streams");
        }
    }
    S->th = std::thread(serve_loop, S);
    ctx->server = S;
    return TE_OK;
}

}  // namespace

extern "C" {

te_status te_serve_start(te_ctx *ctx, const te_serve_config *cfg)
{
    if (!ctx) return TE_EINVAL;
    try {
        if (ctx->server) return fail(ctx, TE_EINVAL, "the server is already running");
        return start_server(ctx, cfg);
    } catch (...) {
        return fail(ctx, TE_ENOMEM, "could not start the server");
    }
}

te_status te_serve_submit(te_ctx *ctx, const te_cmi_job *job, te_ticket *out)
{
    if (!ctx || !job || !out) return TE_EINVAL;
    try {
        te_status st;
        if (!ctx->server) {
            std::lock_guard<std::mutex> g(ctx->serve_start_mu);
            if (!ctx->server && (st = start_server(ctx, nullptr))) return st;
        }
        te_server *S = ctx->server;
        std::string msg;
        st = check_estimate(ctx, job->data, job->x, job->dx, job->y, job->dy, job->z, job->dz,
                            job->params.k, job->params.theiler, job->params.max_lag,
                            job->params.n_surr, msg);
        std::unique_lock<std::mutex> lk(S->mu);
        if (st) {
            S->err = msg;
            return st;
        }
        ServeJob *j = new ServeJob();
        j->data = job->data;
        j->x.assign(job->x, job->x + job->dx);
        j->y.assign(job->y, job->y + job->dy);
        if (job->dz) j->z.assign(job->z, job->z + job->dz);
        j->p = job->params;
        j->N = job->data->T - job->params.max_lag;
        j->S = job->params.n_surr;
        j->fp = footprint(j->N, j->S, job->dy + job->dz);
        if (j->fp > S->budget) {
            delete j;
            S->err = "job footprint exceeds the serving memory budget";
            return TE_EBUSY;
        }
        j->id = S->next++;
        S->jobs[j->id] = j;
        S->pending.push_back(j);
        S->st.submitted++;
        *out = j->id;
        lk.unlock();
        S->cv_work.notify_one();
        return TE_OK;
    } catch (...) {
        return TE_ENOMEM;
    }
}

te_status te_serve_poll(te_ctx *ctx, te_ticket ticket, int32_t timeout_ms, double *out,
                        int64_t *out_key)
{
    if (!ctx || !ctx->server) return TE_EINVAL;
    te_server *S = ctx->server;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return TE_EINVAL;
    ServeJob *j = it->second;
    auto finished = [&] { return j->state >= JS_DONE; };
    if (timeout_ms < 0) {
        S->cv_done.wait(lk, finished);
    } else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), finished)) {
        return TE_ETIMEOUT;
    }
    te_status st = TE_OK;
    if (j->state == JS_CANCELLED) {
        st = TE_ECANCELLED;
    } else if (j->state == JS_FAILED) {
        st = j->err ? j->err : TE_EINTERNAL;
    } else {
        if (out) std::memcpy(out, j->cmi.data(), j->cmi.size() * sizeof(double));
        if (out_key) std::memcpy(out_key, j->keys.data(), j->keys.size() * sizeof(int64_t));
    }
    S->jobs.erase(it);
    delete j;
    return st;
}

te_status te_serve_cancel(te_ctx *ctx, te_ticket ticket)
{
    if (!ctx || !ctx->server) return TE_EINVAL;
    te_server *S = ctx->server;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return TE_EINVAL;
    ServeJob *j = it->second;
    if (j->state == JS_PENDING) {
        S->pending.erase(std::find(S->pending.begin(), S->pending.end(), j));
        j->state = JS_CANCELLED;
        S->st.cancelled++;
        S->cv_done.notify_all();
    } else if (j->state == JS_RUNNING) {
        j->cancel_requested = true;
    } else if (j->state == JS_DONE) {
        j->state = JS_CANCELLED;
        S->st.cancelled++;
    }
    return TE_OK;
}

te_status te_serve_stop(te_ctx *ctx)
{
    if (!ctx) return TE_EINVAL;
    te_server *S = ctx->server;
    if (!S) return TE_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        for (ServeJob *j : S->pending) {
            j->state = JS_CANCELLED;
            S->st.cancelled++;
        }
        S->pending.clear();
    }
    S->cv_work.notify_all();
    S->cv_done.notify_all();
    if (S->th.joinable()) S->th.join();
    for (Slot &sl : S->slots) {
        if (sl.keys_pin) cudaFreeHost(sl.keys_pin);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.ctx) te_ctx_destroy(sl.ctx);
    }
    for (auto &kv : S->jobs) delete kv.second;
    ctx->server = nullptr;
    delete S;
    return TE_OK;
}

te_status te_serve_get_stats(te_ctx *ctx, te_serve_stats *out)
{
    if (!ctx || !out) return TE_EINVAL;
    if (!ctx->server) {
        *out = te_serve_stats{};
        return TE_OK;
    }
    std::lock_guard<std::mutex> lk(ctx->server->mu);
    *out = ctx->server->st;
    out->in_use_bytes = ctx->server->in_use;
    out->peak_bytes = ctx->server->peak;
    out->pending = ctx->server->pending.size();
    return TE_OK;
}

}  // extern "C"
