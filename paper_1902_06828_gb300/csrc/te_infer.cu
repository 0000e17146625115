// Greedy multivariate transfer-entropy network inference (te_network_infer).
//
// Each target runs the paper's four steps (Methods, "Inference algorithm"):
//   stage 1  target past:   repeated maximum-statistic tests over Y^C
//   stage 2  sources past:  repeated maximum-statistic tests over X^C,
//                           conditioned on the selected past
//   stage 3  pruning:       minimum-statistic tests over the selected sources,
//                           each candidate conditioned on all the others
//   stage 4  omnibus test:  collective TE of the selected sources, whose rows
//                           are permuted jointly
//   stage 5  (optional) step-down test after a significant omnibus test
// (Statistical tests: maximum statistic a-d and Table 1, minimum statistic,
// omnibus test; Combining across multiple targets: FDR on omnibus p-values.)
//
// Targets are independent, so every round gathers the next request of every
// unfinished target and evaluates all of them (candidates x surrogates x
// targets) in one fused KSG launch per kernel class, one permutation launch for
// all of the round's permutation sets (one set per request, or per candidate
// with independent surrogates) and one statistics launch; only a few integers per request come back to the host.  With the
// linear-Gaussian estimator each candidate's estimate and surrogates run
// through cmi_gauss's kernels instead, and the statistics compare the
// estimates' order-preserving integer images.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "te_runtime.h"

using namespace teksg;

namespace {

enum Stage { ST_TARGET = 1, ST_SOURCES = 2, ST_PRUNE = 3, ST_OMNIBUS = 4, ST_SEQ = 5, ST_DONE = 6 };

bool var_less(const te_var &a, const te_var &b)
{
    return a.proc != b.proc ? a.proc < b.proc : a.lag < b.lag;
}
bool var_eq(const te_var &a, const te_var &b) { return a.proc == b.proc && a.lag == b.lag; }

struct TargetState {
    int target = 0;
    int stage = ST_TARGET;
    int it = 0;
    bool sources_init = false;
    std::vector<te_var> cand, sel_y, sel_x;
    std::vector<te_var> order;  // candidates of the current request
    // request bookkeeping
    int n_cand = 0, mode = 0, out_base = 0, cnt_off = 0, orig_off = 0;
    double omni_cmi = 0.0, omni_p = 1.0;
    int omni_tested = 0, significant = 0;
    uint64_t n_est = 0;
};

std::vector<te_var> sorted_vars(std::vector<te_var> v)
{
    std::sort(v.begin(), v.end(), var_less);
    return v;
}

// advance through stages with nothing to test; false when the target is done
bool has_request(TargetState &t, int n_proc, const te_infer_params &P)
{
    for (;;) {
        switch (t.stage) {
        case ST_TARGET:
            if (!t.cand.empty()) return true;
            t.stage = ST_SOURCES;
            t.it = 0;
            break;
        case ST_SOURCES:
            if (!t.sources_init) {
                t.cand.clear();
                for (int q = 0; q < n_proc; ++q)
                    if (q != t.target)
                        for (int l = 1; l <= P.max_lag_sources; ++l) t.cand.push_back({q, l});
                t.sources_init = true;
            }
            if (!t.cand.empty()) return true;
            t.stage = ST_PRUNE;
            t.it = 0;
            break;
        case ST_PRUNE:
            if (!t.sel_x.empty()) return true;
            t.stage = ST_OMNIBUS;
            break;
        case ST_OMNIBUS:
            if (!t.sel_x.empty()) return true;
            t.stage = ST_DONE;
            break;
        case ST_SEQ:
            if (P.seq_test && !t.sel_x.empty()) return true;
            t.stage = ST_DONE;
            break;
        default:
            return false;
        }
    }
}

}  // namespace

extern "C" {

te_status te_network_infer(te_ctx *ctx, const te_data *data, const te_infer_params *params,
                           te_network_result **out)
{
    if (!ctx) return TE_EINVAL;
    try {
        ctx->err.clear();
        if (!data || !params || !out) return fail(ctx, TE_EINVAL, "NULL argument");
        if (data->ctx != ctx) return fail(ctx, TE_EINVAL, "data belongs to another context");
        te_infer_params P = *params;
        if (P.estimator != 0 && P.estimator != 1)
            return fail(ctx, TE_EINVAL, "estimator must be 0 (KSG) or 1 (Gaussian)");
        const bool gauss = P.estimator == 1;
        if (gauss && P.theiler != 0)
            return fail(ctx, TE_EINVAL, "the Gaussian estimator has no Theiler window");
        // pooled replications: candidates over the original processes, every
        // variable (p, l) read from the pooled row p * (L + 1) + l at lag 0
        const bool pooled = data->emb_lag >= 0;
        const int n_proc = pooled ? data->n_proc_orig : data->n_proc, T = data->T;
        const int S = P.n_surr;
        if (pooled && P.theiler != 0)
            return fail(ctx, TE_EINVAL, "no Theiler window is defined across pooled trials");
        if (pooled && (P.surr_mode < 0 || P.surr_mode > 2))
            return fail(ctx, TE_EINVAL, "surr_mode must be 0, 1 or 2");
        if (P.max_lag_target < 1 || P.max_lag_sources < 1)
            return fail(ctx, TE_EINVAL, "max lags must be >= 1");
        if (!gauss && (P.k < 1 || P.k > TE_MAX_K))
            return fail(ctx, TE_EINVAL, "k must be in 1..16");
        if (P.theiler < 0) {   // automatic window: largest decay time over the processes
            CK(cudaSetDevice(ctx->device), "cudaSetDevice");
            int32_t w = 0;
            te_status st = autocorr_decay(ctx, data, -1, &w);
            if (st) return st;
            P.theiler = w;
        }
        if (S < 1) return fail(ctx, TE_EINVAL, "n_surr must be >= 1");
        const double alphas[4] = {P.alpha_max, P.alpha_min, P.alpha_omnibus, P.alpha_seq};
        for (int a = 0; a < (P.seq_test ? 4 : 3); ++a)
            if (!(alphas[a] > 0.0 && alphas[a] < 1.0) || !(S * alphas[a] > 1.0))
                return fail(ctx, TE_EINVAL,
                            "every alpha must be in (0, 1) with n_surr * alpha > 1");
        if (P.fdr && !(P.alpha_fdr > 0.0 && P.alpha_fdr < 1.0))
            return fail(ctx, TE_EINVAL, "alpha_fdr must be in (0, 1)");
        const int t0 = std::max(P.max_lag_target, P.max_lag_sources);
        if (pooled && t0 != data->emb_lag)
            return fail(ctx, TE_EINVAL, "max(l_target, l_sources) must equal the trials' max_lag");
        if (!pooled && t0 >= T) return fail(ctx, TE_EINVAL, "max lag must be below T");
        const int t0_est = pooled ? 0 : t0;   // first point of the estimator's columns
        const int N = T - t0_est;
        auto tv = [&](te_var v) {
            return pooled ? te_var{v.proc * (t0 + 1) + v.lag, 0} : v;
        };
        auto tvs = [&](const std::vector<te_var> &vs) {
            std::vector<te_var> o;
            for (const te_var &v : vs) o.push_back(tv(v));
            return o;
        };
        // trial surrogates: 0 = shuffle the trial order, 1 = inside trials
        int trial_mode = 1;
        if (pooled) {
            double orders = 1.0;
            for (int r = 2; r <= data->n_rep; ++r) orders *= r;
            trial_mode = P.surr_mode == 1 ? 0 : P.surr_mode == 2 ? 1 : (orders >= S ? 0 : 1);
        }
        if (!gauss && (long long)N - 1 - 2LL * P.theiler < P.k)
            return fail(ctx, TE_EINVAL, "fewer than k valid neighbours for some point");
        std::vector<int> targets;
        if (P.targets) {
            if (P.n_targets < 1) return fail(ctx, TE_EINVAL, "n_targets must be >= 1");
            targets.assign(P.targets, P.targets + P.n_targets);
        } else {
            for (int q = 0; q < n_proc; ++q) targets.push_back(q);
        }
        {
            std::vector<char> seen(n_proc, 0);
            for (int q : targets) {
                if (q < 0 || q >= n_proc) return fail(ctx, TE_EINVAL, "target outside the data");
                if (seen[q]) return fail(ctx, TE_EINVAL, "target listed twice");
                seen[q] = 1;
            }
        }
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        const auto t_start = std::chrono::steady_clock::now();

        std::vector<TargetState> ts(targets.size());
        for (size_t a = 0; a < targets.size(); ++a) {
            ts[a].target = targets[a];
            for (int l = 1; l <= P.max_lag_target; ++l) ts[a].cand.push_back({targets[a], l});
        }

        te_status st;
        for (;;) {
            std::vector<int> active;
            for (size_t a = 0; a < ts.size(); ++a)
                if (has_request(ts[a], n_proc, P)) active.push_back((int)a);
            if (active.empty()) break;

            // ---- build the round: perms, groups, stat requests ----
            // permutation sets per target: one shared by the test's candidates,
            // or one per candidate with independent surrogates
            std::vector<size_t> set_off(active.size() + 1, 0);
            for (size_t r = 0; r < active.size(); ++r) {
                const TargetState &t = ts[active[r]];
                size_t nc = 1;
                if (P.indep_surr) {
                    if (t.stage == ST_TARGET || t.stage == ST_SOURCES) nc = t.cand.size();
                    else if (t.stage == ST_PRUNE || t.stage == ST_SEQ) nc = t.sel_x.size();
                }
                set_off[r + 1] = set_off[r] + std::max<size_t>(nc, 1);
            }
            const size_t perm_elems = set_off.back() * S * N;
            if ((st = ensure_dev(ctx, ctx->ws_perm, perm_elems * 4))) return st;
            int32_t *perm = (int32_t *)ctx->ws_perm.p;
            std::vector<HostGroup> groups;
            std::vector<StatReq> reqs;
            std::vector<PermJob> pj;   // every plain permutation set of the round
            long long perm_total = 0;
            int n_out = 0, cnt_total = 0, orig_total = 0;
            for (size_t r = 0; r < active.size(); ++r) {
                TargetState &t = ts[active[r]];
                int32_t *pr = perm + set_off[r] * (size_t)S * N;
                const int iter = (t.stage == ST_OMNIBUS || t.stage == ST_SEQ) ? 0 : t.it;
                const size_t n_sets = set_off[r + 1] - set_off[r];
                for (size_t c = 0; c < n_sets; ++c) {
                    const uint64_t s1 = 1 + ((uint64_t)c << 32);
                    if (pooled) {
                        CK(launch_perms_trials(pr + c * (size_t)S * N, data->n_rep,
                                               data->trial_len, P.seed, (uint64_t)t.target,
                                               (uint64_t)t.stage, (uint64_t)iter, s1, S,
                                               trial_mode, ctx->stream),
                           "permutation launch");
                        ctx->stats.launches++;
                    } else {
                        PermJob q{};
                        q.out = pr + c * (size_t)S * N;
                        q.n = N;
                        q.n_perm = S;
                        q.s_first = s1;
                        q.seed = P.seed;
                        q.target = (uint64_t)t.target;
                        q.stage = (uint64_t)t.stage;
                        q.iter = (uint64_t)iter;
                        q.perm_begin = perm_total;
                        perm_total += S;
                        pj.push_back(q);
                    }
                }
                const te_var ypres = tv(te_var{t.target, 0});
                // candidate `c0 + c` of the test uses permutation set c0 + c when
                // every candidate has its own set, set 0 otherwise
                auto add_group = [&](const std::vector<te_var> &z,
                                     const std::vector<std::vector<te_var>> &xs, size_t c0) {
                    HostGroup g;
                    g.data = data;
                    g.max_lag = t0_est;
                    g.k = P.k;
                    g.theiler = P.theiler;
                    g.y = {ypres};
                    g.z = tvs(z);
                    g.dx = (int)xs[0].size();
                    // members surrogate-major, so the members a CTA shares carry
                    // the same permutation; output slots stay candidate-major
                    const int nx = (int)xs.size();
                    for (const auto &x : xs) {
                        const auto xt = tvs(x);
                        g.xvars.insert(g.xvars.end(), xt.begin(), xt.end());
                    }
                    for (int s = 0; s <= S; ++s)
                        for (int c = 0; c < nx; ++c) {
                            const size_t set = n_sets > 1 ? c0 + (size_t)c : 0;
                            g.members.push_back(HostMember{
                                c * g.dx,
                                s == 0 ? nullptr : pr + (set * S + (size_t)(s - 1)) * N,
                                n_out + c * (S + 1) + s});
                        }
                    n_out += nx * (S + 1);
                    groups.push_back(std::move(g));
                };
                t.out_base = n_out;
                if (t.stage == ST_TARGET || t.stage == ST_SOURCES) {
                    t.order = t.cand;
                    std::vector<te_var> z = t.sel_y;
                    if (t.stage == ST_SOURCES) z.insert(z.end(), t.sel_x.begin(), t.sel_x.end());
                    std::vector<std::vector<te_var>> xs;
                    for (const te_var &c : t.order) xs.push_back({c});
                    add_group(z, xs, 0);
                    t.mode = 0;
                } else if (t.stage == ST_PRUNE || t.stage == ST_SEQ) {
                    t.order = sorted_vars(t.sel_x);
                    for (size_t ci = 0; ci < t.order.size(); ++ci) {
                        const te_var &c = t.order[ci];
                        std::vector<te_var> z = t.sel_y;
                        for (const te_var &o : t.order)
                            if (!var_eq(o, c)) z.push_back(o);
                        add_group(z, {{c}}, ci);
                    }
                    t.mode = t.stage == ST_PRUNE ? 1 : 0;
                } else {  // omnibus
                    t.order = sorted_vars(t.sel_x);
                    add_group(t.sel_y, {t.order}, 0);
                    t.mode = 0;
                }
                t.n_cand = t.stage == ST_OMNIBUS ? 1 : (int)t.order.size();
                t.n_est += (uint64_t)t.n_cand * (S + 1);
                t.cnt_off = cnt_total;
                t.orig_off = orig_total;
                cnt_total += 1 + t.n_cand;
                orig_total += t.n_cand;
                reqs.push_back(StatReq{(long long)t.out_base, t.n_cand, S, t.mode, t.cnt_off,
                                       t.orig_off});
            }
            if (!pj.empty()) {   // one launch for the round's permutation sets
                const size_t bytes = pj.size() * sizeof(PermJob);
                if ((st = ensure_dev(ctx, ctx->ws_stat, bytes + 16))) return st;
                CK(copy_h2d(ctx, ctx->ws_stat.p, pj.data(), bytes), "cudaMemcpyAsync");
                CK(launch_perms_multi((const PermJob *)ctx->ws_stat.p, (int)pj.size(), perm_total,
                                      N, ctx->stream),
                   "permutation launch");
                ctx->stats.launches++;
            }
            if ((st = gauss ? run_groups_gauss(ctx, groups, n_out)
                            : run_groups(ctx, groups, n_out)))
                return st;

            // ---- statistics on the device, small readback ----
            const size_t req_bytes = reqs.size() * sizeof(StatReq);
            const size_t ibytes = (size_t)cnt_total * 4;
            const size_t obytes = (size_t)orig_total * 16;
            const size_t ioff = (req_bytes + 15) & ~(size_t)15;
            const size_t ooff = (ioff + ibytes + 15) & ~(size_t)15;
            if ((st = ensure_dev(ctx, ctx->ws_stat, ooff + obytes + 16))) return st;
            if ((st = ensure_pin(ctx, ooff + obytes + 16))) return st;
            char *pin = (char *)ctx->pin;
            std::memcpy(pin, reqs.data(), req_bytes);
            char *dstat = (char *)ctx->ws_stat.p;
            CK(copy_h2d(ctx, dstat, pin, req_bytes), "cudaMemcpyAsync");
            CK(launch_stats((const long long *)ctx->ws_keys.p, (const StatReq *)dstat,
                            (int)reqs.size(), S, (int *)(dstat + ioff), (long long *)(dstat + ooff),
                            ctx->stream),
               "statistics launch");
            ctx->stats.launches++;
            CK(copy_d2h(ctx, pin + ioff, dstat + ioff, ooff - ioff + obytes), "cudaMemcpyAsync");
            CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
            const int *ib = (const int *)(pin + ioff);
            const long long *ob = (const long long *)(pin + ooff);

            // ---- optional trace: every request's keys, before its decision ----
            if (ctx->trace_fn) {
                std::vector<int64_t> kh((size_t)n_out * 2);
                CK(cudaMemcpyAsync(kh.data(), ctx->ws_keys.p, kh.size() * 8,
                                   cudaMemcpyDeviceToHost, ctx->stream),
                   "cudaMemcpyAsync");
                CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
                for (int a : active) {
                    const TargetState &t = ts[a];
                    const int iter = (t.stage == ST_OMNIBUS || t.stage == ST_SEQ) ? 0 : t.it;
                    ctx->trace_fn(ctx->trace_user, t.target, t.stage, iter, t.order.data(),
                                  (int32_t)t.order.size(), t.n_cand, S,
                                  kh.data() + 2 * (size_t)t.out_base);
                }
            }

            // ---- decisions ----
            for (int a : active) {
                TargetState &t = ts[a];
                const int best = ib[t.cnt_off];
                const int *cnt = ib + t.cnt_off + 1;
                if (t.stage == ST_TARGET || t.stage == ST_SOURCES) {
                    const double p = (double)cnt[best] / S;
                    if (p < P.alpha_max) {
                        const te_var c = t.order[best];
                        (t.stage == ST_TARGET ? t.sel_y : t.sel_x).push_back(c);
                        t.cand.erase(t.cand.begin() + best);
                        t.it++;
                    } else {
                        t.cand.clear();  // stop this stage
                    }
                } else if (t.stage == ST_PRUNE) {
                    const double p = (double)cnt[best] / S;
                    if (p < P.alpha_min) {
                        t.stage = ST_OMNIBUS;  // minimum is significant: stop pruning
                    } else {
                        const te_var c = t.order[best];
                        std::vector<te_var> keep;
                        for (const te_var &v : t.sel_x)
                            if (!var_eq(v, c)) keep.push_back(v);
                        t.sel_x = keep;
                        t.it++;
                    }
                } else if (t.stage == ST_OMNIBUS) {
                    const double p = (double)cnt[0] / S;
                    const long long *kk = ob + 2 * t.orig_off;
                    t.omni_cmi = gauss ? gauss_key_value(kk[0], (uint64_t)kk[1])
                                       : key_to_cmi(ctx, kk[0], (uint64_t)kk[1], P.k, N);
                    t.omni_p = p;
                    t.omni_tested = 1;
                    t.significant = p < P.alpha_omnibus;
                    if (!t.significant) t.sel_x.clear();
                    t.stage = (t.significant && P.seq_test) ? ST_SEQ : ST_DONE;
                } else if (t.stage == ST_SEQ) {
                    // step down from the largest contribution
                    std::vector<int> rank(t.n_cand);
                    for (int c = 0; c < t.n_cand; ++c) rank[c] = c;
                    auto key = [&](int c) {
                        const long long *kk = ob + 2 * (t.orig_off + c);
                        return ((__int128)kk[0] << 64) | (__int128)(unsigned long long)kk[1];
                    };
                    std::stable_sort(rank.begin(), rank.end(),
                                     [&](int u, int v) { return key(u) > key(v); });
                    std::vector<te_var> keep;
                    for (int c : rank) {
                        const double p = (double)cnt[c] / S;
                        if (p >= P.alpha_seq) break;
                        keep.push_back(t.order[c]);
                    }
                    t.sel_x = sorted_vars(keep);
                    t.stage = ST_DONE;
                }
            }
        }

        // ---- FDR across targets (optional) ----
        if (P.fdr) {
            std::vector<int> tested;
            for (size_t a = 0; a < ts.size(); ++a)
                if (ts[a].omni_tested) tested.push_back((int)a);
            const int m = (int)tested.size();
            std::vector<int> order(tested);
            std::stable_sort(order.begin(), order.end(), [&](int u, int v) {
                return ts[u].omni_p < ts[v].omni_p;
            });
            int last = 0;
            for (int r = 1; r <= m; ++r)
                if (ts[order[r - 1]].omni_p <= P.alpha_fdr * r / m) last = r;
            for (int r = last + 1; r <= m; ++r) {
                ts[order[r - 1]].sel_x.clear();
                ts[order[r - 1]].significant = 0;
            }
        }

        // ---- result ----
        te_network_result *R = (te_network_result *)std::calloc(1, sizeof(te_network_result));
        if (!R) return fail(ctx, TE_ENOMEM, "host allocation failed");
        R->n_proc = n_proc;
        R->n_targets = (int)ts.size();
        R->targets = (te_target_result *)std::calloc(ts.size(), sizeof(te_target_result));
        R->adjacency = (uint8_t *)std::calloc((size_t)n_proc * n_proc, 1);
        R->min_lag = (int32_t *)std::calloc((size_t)n_proc * n_proc, sizeof(int32_t));
        if (!R->targets || !R->adjacency || !R->min_lag) {
            te_network_result_free(R);
            return fail(ctx, TE_ENOMEM, "host allocation failed");
        }
        for (size_t a = 0; a < ts.size(); ++a) {
            TargetState &t = ts[a];
            te_target_result &o = R->targets[a];
            o.target = t.target;
            const auto sy = sorted_vars(t.sel_y), sx = sorted_vars(t.sel_x);
            o.n_sel_target = (int)sy.size();
            o.n_sel_sources = (int)sx.size();
            o.sel_target = (te_var *)std::calloc(std::max<size_t>(sy.size(), 1), sizeof(te_var));
            o.sel_sources = (te_var *)std::calloc(std::max<size_t>(sx.size(), 1), sizeof(te_var));
            if (!o.sel_target || !o.sel_sources) {
                te_network_result_free(R);
                return fail(ctx, TE_ENOMEM, "host allocation failed");
            }
            std::copy(sy.begin(), sy.end(), o.sel_target);
            std::copy(sx.begin(), sx.end(), o.sel_sources);
            o.omnibus_cmi = t.omni_cmi;
            o.omnibus_p = t.omni_p;
            o.omnibus_tested = t.omni_tested;
            o.significant = t.significant && !sx.empty();
            o.n_estimates = t.n_est;
            R->n_estimates += t.n_est;
            for (const te_var &v : sx) {
                const size_t e = (size_t)v.proc * n_proc + t.target;
                R->adjacency[e] = 1;
                if (R->min_lag[e] == 0 || v.lag < R->min_lag[e]) R->min_lag[e] = v.lag;
            }
        }
        R->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start)
                         .count();
        R->theiler = P.theiler;
        *out = R;
        return TE_OK;
    } catch (const std::bad_alloc &) {
        return fail(ctx, TE_ENOMEM, "host allocation failed");
    } catch (...) {
        return fail(ctx, TE_EINTERNAL, "unexpected C++ exception");
    }
}

te_status te_ctx_set_trace(te_ctx *ctx, te_trace_fn fn, void *user)
{
    if (!ctx) return TE_EINVAL;
    ctx->trace_fn = fn;
    ctx->trace_user = fn ? user : nullptr;
    return TE_OK;
}

void te_network_result_free(te_network_result *res)
{
    if (!res) return;
    if (res->targets) {
        for (int a = 0; a < res->n_targets; ++a) {
            std::free(res->targets[a].sel_target);
            std::free(res->targets[a].sel_sources);
        }
        std::free(res->targets);
    }
    std::free(res->adjacency);
    std::free(res->min_lag);
    std::free(res);
}

}  // extern "C"
