// Host runtime of the KSG engine: contexts, data sets, the digamma table,
// validation, the fused-launch engine and the cmi_ksg* entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <set>
#include <new>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "te_runtime.h"
#include "ksg_tune_table.h"

using namespace teksg;

namespace teksg {

te_status fail(te_ctx *ctx, te_status st, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return st;
}

te_status cuda_fail(te_ctx *ctx, cudaError_t e, const char *what)
{
    std::string m = std::string(what) + " failed: " + cudaGetErrorName(e) + " (" +
                    cudaGetErrorString(e) + ")";
    return fail(ctx, e == cudaErrorMemoryAllocation ? TE_ENOMEM : TE_ECUDA, m);
}

cudaError_t copy_h2d(te_ctx *ctx, void *dst, const void *src, size_t bytes)
{
    ctx->stats.h2d_bytes += bytes;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->stream);
}

cudaError_t copy_d2h(te_ctx *ctx, void *dst, const void *src, size_t bytes)
{
    ctx->stats.d2h_bytes += bytes;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ctx->stream);
}

te_status ensure_dev(te_ctx *ctx, DevBuf &b, size_t bytes)
{
    if (bytes <= b.cap) return TE_OK;
    size_t want = std::max(bytes, b.cap + b.cap / 2);
    want = (want + 255) & ~(size_t)255;
    if (b.p) {
        CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
        CK(cudaFree(b.p), "cudaFree");
        b.p = nullptr;
        b.cap = 0;
    }
    CK(cudaMalloc(&b.p, want), "cudaMalloc");
    b.cap = want;
    return TE_OK;
}

te_status ensure_pin(te_ctx *ctx, size_t bytes)
{
    if (bytes <= ctx->pin_cap) return TE_OK;
    size_t want = std::max(bytes, ctx->pin_cap + ctx->pin_cap / 2);
    if (ctx->pin) {
        CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
        CK(cudaFreeHost(ctx->pin), "cudaFreeHost");
        ctx->pin = nullptr;
        ctx->pin_cap = 0;
    }
    CK(cudaMallocHost(&ctx->pin, want), "cudaMallocHost");
    ctx->pin_cap = want;
    return TE_OK;
}

te_status ensure_aux(te_ctx *ctx)
{
    if (ctx->aux_stream) return TE_OK;
    CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming), "cudaEventCreate");
    CK(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming), "cudaEventCreate");
    CK(cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking), "cudaStreamCreate");
    return TE_OK;
}

// ---- digamma fixed-point table, double-double arithmetic ----------------
// psi(1) = -gamma and psi(n + 1) = psi(n) + 1/n, carried as an unevaluated sum
// hi + lo of two doubles (error-free two-sum; 1/n split with an exact FMA
// residual).  Q[n] = round-to-nearest(2^52 psi(n)).
namespace {

inline void two_sum(double a, double b, double &s, double &e)
{
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

inline void quick_two_sum(double a, double b, double &s, double &e)
{
    s = a + b;
    e = b - (s - a);
}

inline void dd_add(double ah, double al, double bh, double bl, double &rh, double &rl)
{
    double s, e, t, f;
    two_sum(ah, bh, s, e);
    two_sum(al, bl, t, f);
    e += t;
    quick_two_sum(s, e, s, e);
    e += f;
    quick_two_sum(s, e, rh, rl);
}

inline void dd_recip(double n, double &h, double &l)
{
    h = 1.0 / n;
    const double r = std::fma(-h, n, 1.0);  // exact residual 1 - h n
    l = r / n;
}

// divide a double-double by a small integer d
inline void dd_div_int(double ah, double al, double d, double &rh, double &rl)
{
    const double q1 = ah / d;
    const double r = std::fma(-q1, d, ah) + al;
    const double q2 = r / d;
    quick_two_sum(q1, q2, rh, rl);
}

void euler_gamma_dd(double &h, double &l)
{
    // decimal expansion of the Euler-Mascheroni constant, Horner from the end
    static const char *digits = "5772156649015328606065120900824024310421593359399235988057672348848677";
    double xh = 0.0, xl = 0.0;
    for (int p = (int)std::strlen(digits) - 1; p >= 0; --p) {
        double sh, sl;
        dd_add((double)(digits[p] - '0'), 0.0, xh, xl, sh, sl);
        dd_div_int(sh, sl, 10.0, xh, xl);
    }
    h = xh;
    l = xl;
}

int64_t dd_to_q(double h, double l)
{
    const double hs = std::ldexp(h, 52), ls = std::ldexp(l, 52);
    const double ip = std::floor(hs);
    const double fp = hs - ip;  // exact
    const double t = fp + ls;
    return (int64_t)ip + (int64_t)std::floor(t + 0.5);
}

}  // namespace

void digamma_q_fill(int n_max, int64_t *q)
{
    q[0] = 0;
    if (n_max < 1) return;
    double h, l;
    euler_gamma_dd(h, l);
    h = -h;
    l = -l;
    q[1] = dd_to_q(h, l);
    for (int n = 2; n <= n_max; ++n) {
        double rh, rl;
        dd_recip((double)(n - 1), rh, rl);
        dd_add(h, l, rh, rl, h, l);
        q[n] = dd_to_q(h, l);
    }
}

te_status ensure_q(te_ctx *ctx, int n_needed)
{
    if ((int)ctx->q_host.size() <= n_needed) {
        if (ctx->q_host.empty()) {
            ctx->q_host.push_back(0);  // psi has a pole at 0
            double gh, gl;
            euler_gamma_dd(gh, gl);
            ctx->dd_hi = -gh;
            ctx->dd_lo = -gl;
            ctx->q_host.push_back(dd_to_q(ctx->dd_hi, ctx->dd_lo));  // n = 1
        }
        int target = std::max(n_needed + 1, (int)ctx->q_host.size() * 2);
        target = std::max(target, 4096);
        for (int n = (int)ctx->q_host.size(); n < target; ++n) {
            double rh, rl;
            dd_recip((double)(n - 1), rh, rl);
            dd_add(ctx->dd_hi, ctx->dd_lo, rh, rl, ctx->dd_hi, ctx->dd_lo);
            ctx->q_host.push_back(dd_to_q(ctx->dd_hi, ctx->dd_lo));
        }
    }
    if (ctx->q_dev_len <= n_needed) {
        if (ctx->q_dev) {
            CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
            CK(cudaFree(ctx->q_dev), "cudaFree");
            ctx->q_dev = nullptr;
        }
        const size_t bytes = ctx->q_host.size() * sizeof(int64_t);
        CK(cudaMalloc(&ctx->q_dev, bytes), "cudaMalloc");
        CK(copy_h2d(ctx, ctx->q_dev, ctx->q_host.data(), bytes), "cudaMemcpyAsync");
        CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
        ctx->q_dev_len = (int)ctx->q_host.size();
    }
    return TE_OK;
}

double key_to_cmi(const te_ctx *ctx, int64_t hi, uint64_t lo, int k, int N)
{
    const __int128 K = ((__int128)hi << 64) | (__int128)lo;
    const double psi_k = std::ldexp((double)ctx->q_host[k], -52);
    const double t = (double)K;
    const double d = 4503599627370496.0 * (double)N;
    return psi_k + t / d;
}

te_status check_estimate(const te_ctx *ctx, const te_data *data, const te_var *x, int dx,
                         const te_var *y, int dy, const te_var *z, int dz, int k, int theiler,
                         int max_lag, int n_surr, std::string &msg, int max_dims)
{
    if (!data) return (msg = "data is NULL", TE_EINVAL);
    if (data->ctx != ctx) return (msg = "data belongs to another context", TE_EINVAL);
    if (!x || dx < 1) return (msg = "x needs at least one variable", TE_EINVAL);
    if (!y || dy < 1) return (msg = "y needs at least one variable", TE_EINVAL);
    if (dz < 0 || (dz > 0 && !z)) return (msg = "z is NULL with dz > 0", TE_EINVAL);
    if (dx + dy + dz > max_dims)
        return (msg = "dx + dy + dz exceeds " + std::to_string(max_dims), TE_EINVAL);
    if (k < 1 || k > TE_MAX_K) return (msg = "k must be in 1..16", TE_EINVAL);
    if (theiler < 0) return (msg = "theiler window must be >= 0", TE_EINVAL);
    if (n_surr < 0) return (msg = "n_surr must be >= 0", TE_EINVAL);
    if (max_lag < 0 || max_lag >= data->T)
        return (msg = "max_lag must be in 0..T-1", TE_EINVAL);
    const long long N = (long long)data->T - max_lag;
    if (N - 1 - 2LL * theiler < k)
        return (msg = "fewer than k valid neighbours for some point "
                                    "(N - 1 - 2 theiler < k)", TE_EINVAL);
    const te_var *vs[3] = {x, y, z};
    const int ds[3] = {dx, dy, dz};
    for (int s = 0; s < 3; ++s)
        for (int d = 0; d < ds[s]; ++d) {
            const te_var v = vs[s][d];
            if (v.proc < 0 || v.proc >= data->n_proc)
                return (msg = "variable process outside the data", TE_EINVAL);
            if (v.lag < 0 || v.lag > max_lag)
                return (msg = "variable lag outside 0..max_lag", TE_EINVAL);
        }
    return TE_OK;
}

te_status validate_estimate(te_ctx *ctx, const te_data *data, const te_var *x, int dx,
                            const te_var *y, int dy, const te_var *z, int dz, int k, int theiler,
                            int max_lag, int n_surr, int max_dims)
{
    std::string msg;
    const te_status st = check_estimate(ctx, data, x, dx, y, dy, z, dz, k, theiler, max_lag,
                                        n_surr, msg, max_dims);
    if (st) ctx->err = msg;
    return st;
}

// ---- engine ----------------------------------------------------------------
namespace {

struct ClassKey {
    bool dx1;
    bool k4;
    bool operator<(const ClassKey &o) const
    {
        return std::tie(dx1, k4) < std::tie(o.dx1, o.k4);
    }
};

}  // namespace

te_status run_groups(te_ctx *ctx, const std::vector<HostGroup> &groups, int n_out, int dbg_out,
                     float *dbg_eps, int *dbg_nxz, int *dbg_nyz, int *dbg_nz)
{
    te_status st = launch_groups(ctx, groups, n_out, dbg_out, dbg_eps, dbg_nxz, dbg_nyz, dbg_nz);
    if (st) return st;
    return finish_groups(ctx);
}

te_status finish_groups(te_ctx *ctx)
{
    CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    if (!ctx->pend_timed) return TE_OK;
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev_a, ctx->ev_b), "cudaEventElapsedTime");
    ctx->stats.kernel_ms += ms;
    ctx->stats.pair_evals_bruteforce += ctx->pend_pair_evals;
    ctx->stats.pair_evals += ctx->work_host[0];
    ctx->stats.ksg_ops += ctx->work_host[1];
    ctx->stats.estimates += ctx->pend_members;
    ctx->pend_timed = 0;
    if (ctx->work_host[2])
        return fail(ctx, TE_ETIMEOUT, "a KSG tile copy did not complete in time");
    return TE_OK;
}

te_status launch_groups(te_ctx *ctx, const std::vector<HostGroup> &groups, int n_out, int dbg_out,
                        float *dbg_eps, int *dbg_nxz, int *dbg_nyz, int *dbg_nz)
{
    ctx->pend_timed = 0;
    te_status st;
    int max_N = 0;
    for (const HostGroup &g : groups) max_N = std::max(max_N, g.data->T - g.max_lag);
    if ((st = ensure_q(ctx, max_N + 1))) return st;
    if ((st = ensure_dev(ctx, ctx->ws_acc, (size_t)std::max(n_out, 1) * 16))) return st;
    if ((st = ensure_dev(ctx, ctx->ws_keys, (size_t)std::max(n_out, 1) * 16))) return st;
    CK(cudaMemsetAsync(ctx->ws_acc.p, 0, (size_t)n_out * 16, ctx->stream), "cudaMemsetAsync");

    std::map<ClassKey, std::vector<const HostGroup *>> classes;
    for (const HostGroup &g : groups) {
        if (g.members.empty()) continue;
        classes[ClassKey{g.dx == 1, g.k == 4}].push_back(&g);
    }

    // Spatial order for every group without a Theiler window that fits one
    // sorting CTA: sigma [N], sorted coordinates [dyz][N], chunk boxes.
    struct OrderOut {
        size_t sigma, yz, box, tbox;
        int nch, ntl;
    };
    std::map<const HostGroup *, OrderOut> order_of;
    std::vector<const HostGroup *> to_order;
    size_t order_bytes = 0;
    auto align16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    for (const HostGroup &g : groups) {
        const int N = g.data->T - g.max_lag;
        const int dyz = (int)(g.y.size() + g.z.size());
        if (g.members.empty() || g.theiler != 0 || N > kMaxOrderN || N < 16 || dyz > 32)
            continue;
        OrderOut o;
        o.nch = (N + 7) / 8;
        o.sigma = order_bytes;
        order_bytes += align16((size_t)N * 4);
        o.yz = order_bytes;
        order_bytes += align16((size_t)dyz * N * 4);
        o.box = order_bytes;
        order_bytes += align16((size_t)dyz * o.nch * 8);
        o.ntl = (N + 255) / 256;
        o.tbox = order_bytes;
        order_bytes += align16((size_t)dyz * o.ntl * 8);
        order_of[&g] = o;
        to_order.push_back(&g);
    }
    if (!to_order.empty()) {
        if ((st = ensure_dev(ctx, ctx->ws_order, order_bytes))) return st;
    }
    char *obase = (char *)ctx->ws_order.p;

    // every surrogate permutation of a sorted group is composed with the
    // group's order, so kernels index X by position with one load: one
    // composed copy per distinct (group, permutation), found by hashing
    struct ComposeEntry {
        const HostGroup *g;
        const int32_t *perm;
        size_t off;
    };
    std::vector<ComposeEntry> centries;
    std::unordered_map<const HostGroup *, std::vector<size_t>> member_cperm;
    size_t cperm_elems = 0;
    for (const HostGroup *g : to_order) {
        const int N = g->data->T - g->max_lag;
        std::unordered_map<const int32_t *, size_t> seen;
        seen.reserve(g->members.size() * 2);
        std::vector<size_t> &mc = member_cperm[g];
        mc.assign(g->members.size(), SIZE_MAX);
        for (size_t i = 0; i < g->members.size(); ++i) {
            const HostMember &hm = g->members[i];
            if (!hm.perm) continue;
            auto ins = seen.emplace(hm.perm, cperm_elems);
            if (ins.second) {
                centries.push_back(ComposeEntry{g, hm.perm, cperm_elems});
                cperm_elems += ((size_t)N + 3) & ~(size_t)3;
            }
            mc[i] = ins.first->second;
        }
    }
    if (cperm_elems) {
        if ((st = ensure_dev(ctx, ctx->ws_cperm, cperm_elems * 4))) return st;
    }
    int32_t *cbase = (int32_t *)ctx->ws_cperm.p;

    // Sorted groups with an empty Z, one Y and one X variable and no Theiler
    // window count by 1-D range searches: sorted copies of their X columns and
    // of the Y column (one per distinct column of a data set).
    std::map<std::pair<const te_data *, int>, size_t> vsorted_of;
    size_t vs_elems = 0;
    auto col_off = [](const HostGroup *g, te_var v) {
        return v.proc * g->data->T + g->max_lag - v.lag;
    };
    auto want_sorted = [&](const HostGroup *g, int off) {
        auto key = std::make_pair(g->data, off);
        if (!vsorted_of.count(key)) {
            vsorted_of[key] = vs_elems;
            vs_elems += ((size_t)(g->data->T - g->max_lag) + 3) & ~(size_t)3;
        }
    };
    std::vector<const HostGroup *> fast_groups;
    for (const HostGroup *g : to_order) {
        if (!g->z.empty() || g->y.size() != 1 || g->dx != 1 || g->theiler != 0) continue;
        fast_groups.push_back(g);
        want_sorted(g, col_off(g, g->y[0]));
        for (te_var v : g->xvars) want_sorted(g, col_off(g, v));
    }
    if (vs_elems) {
        if ((st = ensure_dev(ctx, ctx->ws_vsort, vs_elems * 4))) return st;
    }
    float *vbase = (float *)ctx->ws_vsort.p;
    std::set<const HostGroup *> fast_set(fast_groups.begin(), fast_groups.end());

    // host tables for every class, staged in one pinned block
    struct Plan {
        KsgVariant v;
        bool dx1;
        int jt;
        size_t smem;
        long long items;
        size_t g_off, m_off, c_off;  // element offsets into the tables
        int n_groups;
        int rows = 0;                // TMA lane kernel: member rows, row pitch (floats),
        long long pitch = 0;         // byte offset of the rows in ws_xval
        size_t xoff = 0;
    };
    size_t xval_bytes = 0;
    std::vector<Plan> plans;
    std::vector<GroupDesc> gdesc;
    std::vector<MemberDesc> mdesc;
    std::vector<int> cols;
    uint64_t pair_evals = 0, members_total = 0;

    for (auto &kv : classes) {
        const bool dx1 = kv.first.dx1, k4 = kv.first.k4;
        auto &gs = kv.second;
        KsgVariant v{4, 4, 128};
        int tune_jt = 256;
        if (dx1) {
            v = KsgVariant{32, k4 ? 4 : 0, kLaneThreads, true};   // member-lane kernel, TMA tiles
            // tile length and members per lane from the tuning table (or the
            // context's forced values); two members per lane only when every
            // group has enough members to fill them
            size_t min_members = SIZE_MAX;
            int tN = 0, tdz = 0;
            for (const HostGroup *g : gs) {
                min_members = std::min(min_members, g->members.size());
                tN = std::max(tN, g->data->T - g->max_lag);
                tdz = std::max(tdz, (int)g->z.size());
            }
            int tune_ms = 1;
            for (const KsgTuneEntry &e : kKsgTune)
                if (tN <= e.n_max && tdz <= e.dz_max && min_members >= (size_t)e.min_members) {
                    tune_jt = e.jt;
                    tune_ms = e.ms;
                    break;
                }
            if (ctx->opt_jt) tune_jt = ctx->opt_jt;
            if (ctx->opt_ms) tune_ms = ctx->opt_ms;
            if (tune_ms == 2 && k4 && min_members >= 64) v.m = 64;
            v.persist = ctx->opt_persistent != 0;
        } else if (!k4) {
            v = KsgVariant{2, 0, 128};
        } else {
            v.m = 4;
        }
        const bool lanek = v.m == 32 || v.m == 64;
        const int qsz = lanek ? kLaneQueries : 128;
        int rows_t = 0, rows_q = 0, maxN = 0;
        for (const HostGroup *g : gs) {
            const int dyz = (int)g->y.size() + (int)g->z.size();
            rows_t = std::max(rows_t, dyz + v.m * g->dx);
            rows_q = std::max(rows_q, dyz + (dx1 ? 0 : v.m * g->dx));
            maxN = std::max(maxN, g->data->T - g->max_lag);
        }
        if (!dx1 && v.m > 2 && (size_t)4 * (rows_t * 64 + rows_q * 128) > 180 * 1024) {
            v.m = 2;
            rows_t = rows_q = 0;
            for (const HostGroup *g : gs) {
                const int dyz = (int)g->y.size() + (int)g->z.size();
                rows_t = std::max(rows_t, dyz + v.m * g->dx);
                rows_q = std::max(rows_q, dyz + v.m * g->dx);
            }
        }
        auto jt_for = [&](size_t budget) {
            long long room = (long long)budget - 4LL * rows_q * 128 - 64 - 8 * 8 * 128;
            long long jt = room / (4LL * rows_t + 8);
            jt &= ~7LL;
            return (int)std::min<long long>(jt, 2048);
        };
        int jt;
        size_t smem;
        if (lanek) {
            int maxdyz = 0;
            for (const HostGroup *g : gs)
                maxdyz = std::max(maxdyz, (int)(g->y.size() + g->z.size()));
            jt = tune_jt;
            if (maxN < jt) jt = std::max(64, (maxN + 63) & ~63);
            smem = ksg_lane_tma_smem_bytes(maxdyz, jt, v.m);
        } else {
            jt = jt_for(40 * 1024);
            if (jt < 64) jt = jt_for(190 * 1024);
            if (jt < 8) return fail(ctx, TE_EINTERNAL, "shared-memory tile does not fit");
            jt = std::min(jt, (maxN + 7) & ~7);
            smem = ksg_smem_bytes(rows_t, rows_q, jt, 128);
        }

        Plan p;
        p.v = v;
        p.dx1 = dx1;
        p.jt = jt;
        p.smem = smem;
        p.g_off = gdesc.size();
        p.m_off = mdesc.size();
        p.c_off = cols.size();
        p.n_groups = (int)gs.size();
        if (v.tma) {
            size_t rows = 0;
            for (const HostGroup *g : gs) rows += g->members.size();
            p.rows = (int)rows;
            p.pitch = std::max(32, (maxN + 3) & ~3);
            p.xoff = xval_bytes;
            xval_bytes += ((size_t)p.rows * (size_t)p.pitch * 4 + 255) & ~(size_t)255;
        }
        long long item = 0;
        for (const HostGroup *g : gs) {
            const te_data *d = g->data;
            const int N = d->T - g->max_lag;
            auto off = [&](te_var vv) { return vv.proc * d->T + g->max_lag - vv.lag; };
            GroupDesc gd{};
            gd.base = d->d_series;
            gd.N = N;
            gd.k = g->k;
            gd.theiler = g->theiler;
            gd.dy = (int)g->y.size();
            gd.dz = (int)g->z.size();
            gd.dx = g->dx;
            gd.ycol = (int)(cols.size() - p.c_off);
            for (te_var vv : g->y) cols.push_back(off(vv));
            gd.zcol = (int)(cols.size() - p.c_off);
            for (te_var vv : g->z) cols.push_back(off(vv));
            const int xbase = (int)(cols.size() - p.c_off);
            for (te_var vv : g->xvars) cols.push_back(off(vv));
            gd.member_begin = (int)(mdesc.size() - p.m_off);
            gd.n_members = (int)g->members.size();
            const bool grp_sorted = order_of.count(g) != 0;
            const bool grp_fast = fast_set.count(g) != 0;
            const std::vector<size_t> *mc = grp_sorted ? &member_cperm[g] : nullptr;
            for (size_t i = 0; i < g->members.size(); ++i) {
                const HostMember &hm = g->members[i];
                MemberDesc md;
                md.perm = hm.perm;
                if (grp_sorted && hm.perm) md.perm = cbase + (*mc)[i];
                md.xsorted = nullptr;
                if (grp_fast)
                    md.xsorted = vbase + vsorted_of[std::make_pair(
                                             g->data, col_off(g, g->xvars[hm.xcol_first]))];
                md.xcol = xbase + hm.xcol_first;
                md.out = hm.out;
                mdesc.push_back(md);
            }
            auto oit = order_of.find(g);
            if (oit != order_of.end()) {
                gd.sigma = (const int *)(obase + oit->second.sigma);
                gd.yz = (const float *)(obase + oit->second.yz);
                gd.box = (const float2 *)(obase + oit->second.box);
                gd.n_chunks8 = oit->second.nch;
                gd.tbox = (const float2 *)(obase + oit->second.tbox);
                gd.n_tiles256 = oit->second.ntl;
                if (fast_set.count(g))
                    gd.ysorted = vbase + vsorted_of[std::make_pair(g->data, col_off(g, g->y[0]))];
            }
            gd.n_qtiles = (N + qsz - 1) / qsz;
            gd.n_mblocks = (gd.n_members + v.m - 1) / v.m;
            gd.item_begin = item;
            item += (long long)gd.n_qtiles * gd.n_mblocks;
            gdesc.push_back(gd);
            pair_evals += (uint64_t)g->members.size() * 2ull * (uint64_t)N * (uint64_t)(N - 1);
            members_total += g->members.size();
        }
        p.items = item;
        plans.push_back(p);
    }
    if (plans.empty()) {
        CK(launch_finalize((const unsigned long long *)ctx->ws_acc.p, (long long *)ctx->ws_keys.p,
                           n_out, ctx->stream),
           "finalize launch");
        return TE_OK;
    }

    std::vector<OrderJob> ojobs;
    for (const HostGroup *g : to_order) {
        const OrderOut &o = order_of[g];
        OrderJob J{};
        J.base = g->data->d_series;
        J.N = g->data->T - g->max_lag;
        J.dyz = (int)(g->y.size() + g->z.size());
        int d = 0;
        for (te_var vv : g->y) J.cols[d++] = vv.proc * g->data->T + g->max_lag - vv.lag;
        for (te_var vv : g->z) J.cols[d++] = vv.proc * g->data->T + g->max_lag - vv.lag;
        J.sigma = (int *)(obase + o.sigma);
        J.yz = (float *)(obase + o.yz);
        J.box = (float2 *)(obase + o.box);
        J.tbox = (float2 *)(obase + o.tbox);
        J.kd = ctx->opt_order == 0 ? (g->members.size() >= kKdOrderMinMembers ? 1 : 0)
                                   : (ctx->opt_order == 2 ? 1 : 0);
        ojobs.push_back(J);
    }
    std::vector<ComposeJob> cjobs;
    int max_cn = 0;
    for (const ComposeEntry &ce : centries) {
        const HostGroup *g = ce.g;
        ComposeJob J;
        J.sigma = (const int *)(obase + order_of[g].sigma);
        J.perm = ce.perm;
        J.out = cbase + ce.off;
        J.N = g->data->T - g->max_lag;
        max_cn = std::max(max_cn, J.N);
        cjobs.push_back(J);
    }
    std::vector<ValueSortJob> vjobs;
    for (auto &kv : vsorted_of) {
        ValueSortJob J;
        J.src = kv.first.first->d_series + kv.first.second;
        J.dst = vbase + kv.second;
        int n = 0;
        for (const HostGroup *g : fast_groups)
            if (g->data == kv.first.first) n = g->data->T - g->max_lag;
        J.N = n;
        vjobs.push_back(J);
    }
    const size_t gbytes = gdesc.size() * sizeof(GroupDesc);
    const size_t mbytes = mdesc.size() * sizeof(MemberDesc);
    const size_t cbytes = cols.size() * sizeof(int);
    const size_t obytes = ojobs.size() * sizeof(OrderJob);
    const size_t jbytes = cjobs.size() * sizeof(ComposeJob);
    const size_t vbytes = vjobs.size() * sizeof(ValueSortJob);
    if ((st = ensure_pin(ctx, gbytes + mbytes + cbytes + obytes + jbytes + vbytes + 64))) return st;
    if ((st = ensure_dev(ctx, ctx->ws_ojobs, obytes + jbytes + vbytes + 16))) return st;
    if ((st = ensure_dev(ctx, ctx->ws_groups, gbytes + 16))) return st;
    if ((st = ensure_dev(ctx, ctx->ws_members, mbytes + 16))) return st;
    if ((st = ensure_dev(ctx, ctx->ws_cols, cbytes + 16))) return st;
    if (xval_bytes && (st = ensure_dev(ctx, ctx->ws_xval, xval_bytes))) return st;
    char *pin = (char *)ctx->pin;
    std::memcpy(pin, gdesc.data(), gbytes);
    std::memcpy(pin + gbytes, mdesc.data(), mbytes);
    std::memcpy(pin + gbytes + mbytes, cols.data(), cbytes);
    CK(copy_h2d(ctx, ctx->ws_groups.p, pin, gbytes), "cudaMemcpyAsync");
    CK(copy_h2d(ctx, ctx->ws_members.p, pin + gbytes, mbytes), "cudaMemcpyAsync");
    if (cbytes) CK(copy_h2d(ctx, ctx->ws_cols.p, pin + gbytes + mbytes, cbytes), "cudaMemcpyAsync");
    if (obytes + jbytes + vbytes) {
        char *jp = pin + gbytes + mbytes + cbytes;
        std::memcpy(jp, ojobs.data(), obytes);
        std::memcpy(jp + obytes, cjobs.data(), jbytes);
        std::memcpy(jp + obytes + jbytes, vjobs.data(), vbytes);
        CK(copy_h2d(ctx, ctx->ws_ojobs.p, jp, obytes + jbytes + vbytes), "cudaMemcpyAsync");
    }

    if (!ctx->prepared) {
        CK(ksg_prepare_attributes(), "cudaFuncSetAttribute");
        ctx->prepared = 1;
    }
    // The batch's device work.  With the graph option it is captured on the
    // stream into a CUDA graph, instantiated and launched as one graph (the
    // timing events then bracket the graph launch).
    const bool graph = ctx->opt_graph != 0;
    auto device_work = [&]() -> te_status {
        if (!ojobs.empty()) {
            CK(launch_order((const OrderJob *)ctx->ws_ojobs.p, (int)ojobs.size(), ctx->stream),
               "order launch");
            ctx->stats.launches++;
        }
        if (!cjobs.empty()) {
            CK(launch_compose((const ComposeJob *)((char *)ctx->ws_ojobs.p + obytes),
                              (int)cjobs.size(), max_cn, ctx->stream),
               "compose launch");
            ctx->stats.launches++;
        }
        if (!vjobs.empty()) {
            CK(launch_value_sort((const ValueSortJob *)((char *)ctx->ws_ojobs.p + obytes + jbytes),
                                 (int)vjobs.size(), ctx->stream),
               "value sort launch");
            ctx->stats.launches++;
        }
        CK(cudaMemsetAsync(ctx->work_dev, 0, 3 * sizeof(unsigned long long), ctx->stream),
           "cudaMemsetAsync");
        if (!graph) CK(cudaEventRecord(ctx->ev_a, ctx->stream), "cudaEventRecord");
        for (const Plan &p : plans) {
            KsgLaunch L{};
            L.groups = (const GroupDesc *)ctx->ws_groups.p + p.g_off;
            L.n_groups = p.n_groups;
            L.members = (const MemberDesc *)ctx->ws_members.p + p.m_off;
            L.cols = (const int *)ctx->ws_cols.p + p.c_off;
            L.q = ctx->q_dev;
            L.acc = (unsigned long long *)ctx->ws_acc.p;
            L.dbg_eps = dbg_eps;
            L.dbg_nxz = dbg_nxz;
            L.dbg_nyz = dbg_nyz;
            L.dbg_nz = dbg_nz;
            L.dbg_out = dbg_out;
            L.jt = p.jt;
            L.work = ctx->work_dev;
            if (p.v.persist) {
                L.item_counter = ctx->work_dev + 3;
                CK(cudaMemsetAsync(L.item_counter, 0, sizeof(unsigned long long), ctx->stream),
                   "cudaMemsetAsync");
            }
            if (p.v.tma) {
                L.xval = (const float *)((char *)ctx->ws_xval.p + p.xoff);
                L.xpitch = p.pitch;
                CUtensorMap map;
                CK(encode_xval_map(&map, L.xval, p.pitch, p.rows, p.v.m), "tensor map encode");
                CK(launch_xval(L, p.rows, ctx->stream), "X-value launch");
                ctx->stats.launches++;
                CK(launch_ksg(L, p.v, p.items, p.dx1, p.smem, ctx->stream, &map),
                   "KSG kernel launch");
            } else {
                CK(launch_ksg(L, p.v, p.items, p.dx1, p.smem, ctx->stream), "KSG kernel launch");
            }
            ctx->stats.launches++;
            ctx->stats.ksg_launches++;
        }
        if (!graph) CK(cudaEventRecord(ctx->ev_b, ctx->stream), "cudaEventRecord");
        CK(copy_d2h(ctx, ctx->work_host, ctx->work_dev, 3 * sizeof(unsigned long long)),
           "cudaMemcpyAsync");
        CK(launch_finalize((const unsigned long long *)ctx->ws_acc.p,
                           (long long *)ctx->ws_keys.p, n_out, ctx->stream),
           "finalize launch");
        ctx->stats.launches++;
        return TE_OK;
    };
    if (!graph) {
        if ((st = device_work())) return st;
    } else {
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal),
           "cudaStreamBeginCapture");
        const te_status ws = device_work();
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
        if (ws) {
            if (g) cudaGraphDestroy(g);
            return ws;
        }
        CK(ce, "cudaStreamEndCapture");
        cudaGraphExec_t ge = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        CK(ie, "cudaGraphInstantiate");
        cudaError_t le = cudaEventRecord(ctx->ev_a, ctx->stream);
        if (le == cudaSuccess) le = cudaGraphLaunch(ge, ctx->stream);
        if (le == cudaSuccess) le = cudaEventRecord(ctx->ev_b, ctx->stream);
        cudaGraphExecDestroy(ge);   // released once the launched graph completes
        CK(le, "cudaGraphLaunch");
    }
    ctx->pend_timed = 1;
    ctx->pend_pair_evals = pair_evals;
    ctx->pend_members = members_total;
    return TE_OK;
}

}  // namespace teksg

// ---- C ABI -------------------------------------------------------------------

#define GUARD_BEGIN try {
#define GUARD_END                                                           \
    }                                                                       \
    catch (const std::bad_alloc &) {                                        \
        return fail(ctx, TE_ENOMEM, "host allocation failed");              \
    }                                                                       \
    catch (...) {                                                           \
        return fail(ctx, TE_EINTERNAL, "unexpected C++ exception");         \
    }

extern "C" {

te_status te_ctx_create(int device, te_ctx **out)
{
    if (!out) return TE_EINVAL;
    te_ctx *ctx = nullptr;
    try {
        ctx = new te_ctx();
    } catch (...) {
        return TE_ENOMEM;
    }
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || device < 0 || device >= n) {
        delete ctx;
        return e != cudaSuccess ? TE_ECUDA : TE_EINVAL;
    }
    ctx->device = device;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&ctx->ev_a) != cudaSuccess || cudaEventCreate(&ctx->ev_b) != cudaSuccess ||
        cudaMalloc(&ctx->work_dev, 4 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost(&ctx->work_host, 3 * sizeof(unsigned long long)) != cudaSuccess) {
        te_ctx_destroy(ctx);
        return TE_ECUDA;
    }
    ctx->stream = ctx->own_stream;
    *out = ctx;
    return TE_OK;
}

te_status te_ctx_set_option(te_ctx *ctx, int32_t option, int64_t value)
{
    if (!ctx) return TE_EINVAL;
    switch (option) {
    case TE_OPT_KSG_TILE:
        if (value != 0 && value != 64 && value != 128 && value != 256)
            return fail(ctx, TE_EINVAL, "the member-lane tile must be 0, 64, 128 or 256 points");
        ctx->opt_jt = (int)value;
        return TE_OK;
    case TE_OPT_KSG_MEMBERS_PER_LANE:
        if (value < 0 || value > 2)
            return fail(ctx, TE_EINVAL, "members per lane must be 0, 1 or 2");
        ctx->opt_ms = (int)value;
        return TE_OK;
    case TE_OPT_PERSISTENT:
    case TE_OPT_GRAPH:
        if (value != 0 && value != 1) return fail(ctx, TE_EINVAL, "the option takes 0 or 1");
        (option == TE_OPT_PERSISTENT ? ctx->opt_persistent : ctx->opt_graph) = (int)value;
        return TE_OK;
    case TE_OPT_KSG_ORDER:
        if (value < 0 || value > 2) return fail(ctx, TE_EINVAL, "the order option takes 0, 1 or 2");
        ctx->opt_order = (int)value;
        return TE_OK;
    default:
        return fail(ctx, TE_EINVAL, "unknown option");
    }
}

te_status te_ctx_set_stream(te_ctx *ctx, void *cuda_stream)
{
    if (!ctx) return TE_EINVAL;
    ctx->stream = cuda_stream ? (cudaStream_t)cuda_stream : ctx->own_stream;
    ctx->err.clear();
    return TE_OK;
}

void te_ctx_destroy(te_ctx *ctx)
{
    if (!ctx) return;
    te_serve_stop(ctx);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->aux_stream) cudaStreamSynchronize(ctx->aux_stream);
    DevBuf *bufs[] = {&ctx->ws_groups, &ctx->ws_members, &ctx->ws_cols,  &ctx->ws_acc,
                      &ctx->ws_keys,   &ctx->ws_perm,    &ctx->ws_stat,  &ctx->ws_dbg,
                      &ctx->ws_order,  &ctx->ws_ojobs,  &ctx->ws_cperm, &ctx->ws_gauss,
                      &ctx->ws_vsort,  &ctx->ws_xval,   &ctx->ws_gtile};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    if (ctx->q_dev) cudaFree(ctx->q_dev);
    if (ctx->pin) cudaFreeHost(ctx->pin);
    if (ctx->work_dev) cudaFree(ctx->work_dev);
    if (ctx->work_host) cudaFreeHost(ctx->work_host);
    if (ctx->ev_a) cudaEventDestroy(ctx->ev_a);
    if (ctx->ev_b) cudaEventDestroy(ctx->ev_b);
    if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
}

const char *te_last_error(const te_ctx *ctx)
{
    if (!ctx) return "no context";
    return ctx->err.c_str();
}

te_status te_data_create(te_ctx *ctx, const float *series, int32_t n_proc, int32_t T,
                         int series_on_device, te_data **out)
{
    if (!ctx) return TE_EINVAL;
    GUARD_BEGIN
    ctx->err.clear();
    if (!series || !out) return fail(ctx, TE_EINVAL, "series or out is NULL");
    if (n_proc < 1 || T < 2) return fail(ctx, TE_EINVAL, "need n_proc >= 1 and T >= 2");
    if ((long long)n_proc * T >= (1LL << 31))
        return fail(ctx, TE_EINVAL, "n_proc * T must be below 2^31");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const size_t bytes = (size_t)n_proc * T * sizeof(float);
    float *d = nullptr;
    CK(cudaMalloc(&d, bytes + sizeof(int)), "cudaMalloc");
    cudaError_t e = series_on_device
                        ? cudaMemcpyAsync(d, series, bytes, cudaMemcpyDeviceToDevice, ctx->stream)
                        : copy_h2d(ctx, d, series, bytes);
    int *flag = (int *)((char *)d + bytes);
    int hflag = 0;
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = launch_check_finite(d, (long long)n_proc * T, flag, ctx->stream);
    if (e == cudaSuccess) e = copy_d2h(ctx, &hflag, flag, sizeof(int));
    ctx->stats.launches++;
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(ctx, e, "te_data_create upload");
    }
    if (hflag) {
        cudaFree(d);
        return fail(ctx, TE_EINVAL, "series holds a non-finite value");
    }
    te_data *D = new te_data{ctx, d, n_proc, T};
    *out = D;
    return TE_OK;
    GUARD_END
}

te_status te_data_create_trials(te_ctx *ctx, const float *series, int32_t n_proc, int32_t n_rep,
                                int32_t T, int32_t max_lag, int series_on_device, te_data **out)
{
    if (!ctx) return TE_EINVAL;
    GUARD_BEGIN
    ctx->err.clear();
    if (!series || !out) return fail(ctx, TE_EINVAL, "series or out is NULL");
    if (n_proc < 1 || n_rep < 1 || max_lag < 0 || T - max_lag < 2)
        return fail(ctx, TE_EINVAL, "need n_proc, n_rep >= 1, 0 <= max_lag and T - max_lag >= 2");
    const long long rows = (long long)n_proc * (max_lag + 1);
    const long long npool = (long long)n_rep * (T - max_lag);
    if ((long long)n_proc * n_rep * T >= (1LL << 31) || rows * npool >= (1LL << 31))
        return fail(ctx, TE_EINVAL, "pooled data must hold fewer than 2^31 values");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    std::vector<float> raw;
    const float *src = series;
    if (series_on_device) {
        raw.resize((size_t)n_proc * n_rep * T);
        CK(cudaMemcpy(raw.data(), series, raw.size() * sizeof(float), cudaMemcpyDeviceToHost),
           "cudaMemcpy");
        src = raw.data();
    }
    // row p * (L + 1) + l, point r * (T - L) + t: process p, trial r, time L + t - l
    const int L = max_lag, n = T - max_lag;
    std::vector<float> pooled((size_t)rows * npool);
    for (int p = 0; p < n_proc; ++p)
        for (int l = 0; l <= L; ++l) {
            float *row = pooled.data() + ((size_t)p * (L + 1) + l) * npool;
            for (int r = 0; r < n_rep; ++r) {
                const float *tr = src + ((size_t)p * n_rep + r) * T + (L - l);
                std::copy(tr, tr + n, row + (size_t)r * n);
            }
        }
    te_data *D = nullptr;
    te_status st = te_data_create(ctx, pooled.data(), (int32_t)rows, (int32_t)npool, 0, &D);
    if (st) return st;
    D->n_rep = n_rep;
    D->trial_len = n;
    D->emb_lag = L;
    D->n_proc_orig = n_proc;
    *out = D;
    return TE_OK;
    GUARD_END
}

void te_data_destroy(te_data *data)
{
    if (!data) return;
    cudaSetDevice(data->ctx->device);
    cudaStreamSynchronize(data->ctx->stream);
    cudaFree(data->d_series);
    delete data;
}

static te_status cmi_common(te_ctx *ctx, const te_data *data, const te_var *x, int32_t dx,
                            const te_var *y, int32_t dy, const te_var *z, int32_t dz,
                            const te_ksg_params *p, double *out_cmi, int64_t *out_key,
                            int32_t dbg_member, float *eps, int32_t *nxz, int32_t *nyz,
                            int32_t *nz)
{
    te_status st;
    if (!p) return fail(ctx, TE_EINVAL, "params is NULL");
    if ((st = validate_estimate(ctx, data, x, dx, y, dy, z, dz, p->k, p->theiler, p->max_lag,
                                p->n_surr)))
        return st;
    if (dbg_member >= 0 && dbg_member > p->n_surr)
        return fail(ctx, TE_EINVAL, "member outside 0..n_surr");
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int N = data->T - p->max_lag;
    const int S = p->n_surr;
    if ((st = ensure_dev(ctx, ctx->ws_perm, (size_t)std::max(S, 1) * N * sizeof(int32_t))))
        return st;
    int32_t *perm = (int32_t *)ctx->ws_perm.p;
    CK(launch_perms(perm, N, N, p->seed, p->stream_tag, 0, 0, 1, S, ctx->stream),
       "permutation launch");
    if (S > 0) ctx->stats.launches++;
    HostGroup g;
    g.data = data;
    g.max_lag = p->max_lag;
    g.k = p->k;
    g.theiler = p->theiler;
    g.y.assign(y, y + dy);
    if (dz) g.z.assign(z, z + dz);
    g.dx = dx;
    g.xvars.assign(x, x + dx);
    for (int s = 0; s <= S; ++s)
        g.members.push_back(HostMember{0, s == 0 ? nullptr : perm + (size_t)(s - 1) * N, s});
    std::vector<HostGroup> gs{g};
    float *d_eps = nullptr;
    int *d_cnt = nullptr;
    if (dbg_member >= 0) {
        if ((st = ensure_dev(ctx, ctx->ws_dbg, (size_t)N * 16))) return st;
        d_eps = (float *)ctx->ws_dbg.p;
        d_cnt = (int *)((char *)ctx->ws_dbg.p + (size_t)N * 4);
    }
    if ((st = run_groups(ctx, gs, S + 1, dbg_member, d_eps, d_cnt, d_cnt + N, d_cnt + 2 * N)))
        return st;
    if (dbg_member >= 0) {
        if (eps)
            CK(copy_d2h(ctx, eps, d_eps, (size_t)N * 4), "cudaMemcpyAsync");
        if (nxz)
            CK(copy_d2h(ctx, nxz, d_cnt, (size_t)N * 4), "cudaMemcpyAsync");
        if (nyz)
            CK(copy_d2h(ctx, nyz, d_cnt + N, (size_t)N * 4), "cudaMemcpyAsync");
        if (nz)
            CK(copy_d2h(ctx, nz, d_cnt + 2 * N, (size_t)N * 4), "cudaMemcpyAsync");
        CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
        return TE_OK;
    }
    std::vector<int64_t> keys((size_t)2 * (S + 1));
    CK(copy_d2h(ctx, keys.data(), ctx->ws_keys.p, keys.size() * 8), "cudaMemcpyAsync");
    CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    for (int s = 0; s <= S; ++s)
        out_cmi[s] = key_to_cmi(ctx, keys[2 * s], (uint64_t)keys[2 * s + 1], p->k, N);
    if (out_key) std::memcpy(out_key, keys.data(), keys.size() * 8);
    return TE_OK;
}

te_status cmi_ksg(te_ctx *ctx, const te_data *data, const te_var *x, int32_t dx, const te_var *y,
                  int32_t dy, const te_var *z, int32_t dz, const te_ksg_params *params,
                  double *out_cmi, int64_t *out_key)
{
    if (!ctx) return TE_EINVAL;
    GUARD_BEGIN
    ctx->err.clear();
    if (!out_cmi) return fail(ctx, TE_EINVAL, "out_cmi is NULL");
    return cmi_common(ctx, data, x, dx, y, dy, z, dz, params, out_cmi, out_key, -1, nullptr,
                      nullptr, nullptr, nullptr);
    GUARD_END
}

te_status cmi_ksg_debug(te_ctx *ctx, const te_data *data, const te_var *x, int32_t dx,
                        const te_var *y, int32_t dy, const te_var *z, int32_t dz,
                        const te_ksg_params *params, int32_t member, float *eps, int32_t *n_xz,
                        int32_t *n_yz, int32_t *n_z)
{
    if (!ctx) return TE_EINVAL;
    GUARD_BEGIN
    ctx->err.clear();
    if (member < 0) return fail(ctx, TE_EINVAL, "member must be >= 0");
    return cmi_common(ctx, data, x, dx, y, dy, z, dz, params, nullptr, nullptr, member, eps,
                      n_xz, n_yz, n_z);
    GUARD_END
}

te_status cmi_ksg_batch(te_ctx *ctx, const te_cmi_job *jobs, int32_t n_jobs, double *out,
                        int64_t *out_key)
{
    if (!ctx) return TE_EINVAL;
    GUARD_BEGIN
    ctx->err.clear();
    te_status st;
    if (n_jobs < 0 || (n_jobs > 0 && (!jobs || !out)))
        return fail(ctx, TE_EINVAL, "jobs or out is NULL");
    if (n_jobs == 0) return TE_OK;
    size_t perm_elems = 0;
    int n_out = 0;
    std::vector<int> job_out(n_jobs), job_N(n_jobs);
    std::vector<size_t> job_perm(n_jobs);
    for (int j = 0; j < n_jobs; ++j) {
        const te_cmi_job &J = jobs[j];
        if ((st = validate_estimate(ctx, J.data, J.x, J.dx, J.y, J.dy, J.z, J.dz, J.params.k,
                                    J.params.theiler, J.params.max_lag, J.params.n_surr))) {
            ctx->err = "job " + std::to_string(j) + ": " + ctx->err;
            return st;
        }
        job_N[j] = J.data->T - J.params.max_lag;
        job_out[j] = n_out;
        n_out += 1 + J.params.n_surr;
        job_perm[j] = perm_elems;
        perm_elems += (size_t)J.params.n_surr * job_N[j];
    }
    CK(cudaSetDevice(ctx->device), "cudaSetDevice");
    if ((st = ensure_dev(ctx, ctx->ws_perm, std::max<size_t>(perm_elems, 1) * 4))) return st;
    int32_t *perm = (int32_t *)ctx->ws_perm.p;
    // jobs with the same data, point set, k, window, Y and Z share a group
    std::map<std::vector<long long>, int> gid;
    std::vector<HostGroup> groups;
    // every job's surrogate permutations in one launch
    std::vector<PermJob> pj;
    long long perm_total = 0;
    int max_n = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const int S = jobs[j].params.n_surr;
        if (S <= 0) continue;
        PermJob q{};
        q.out = perm + job_perm[j];
        q.n = job_N[j];
        q.n_perm = S;
        q.s_first = 1;
        q.seed = jobs[j].params.seed;
        q.target = jobs[j].params.stream_tag;
        q.stage = 0;
        q.iter = 0;
        q.perm_begin = perm_total;
        perm_total += S;
        max_n = std::max(max_n, job_N[j]);
        pj.push_back(q);
    }
    if (!pj.empty()) {
        const size_t bytes = pj.size() * sizeof(PermJob);
        if ((st = ensure_dev(ctx, ctx->ws_stat, bytes + 16))) return st;
        CK(copy_h2d(ctx, ctx->ws_stat.p, pj.data(), bytes), "cudaMemcpyAsync");
        CK(launch_perms_multi((const PermJob *)ctx->ws_stat.p, (int)pj.size(), perm_total, max_n,
                              ctx->stream),
           "permutation launch");
        ctx->stats.launches++;
    }
    for (int j = 0; j < n_jobs; ++j) {
        const te_cmi_job &J = jobs[j];
        const int N = job_N[j], S = J.params.n_surr;
        std::vector<long long> key{(long long)(uintptr_t)J.data, J.params.max_lag, J.params.k,
                                   J.params.theiler, J.dx, J.dy, J.dz};
        for (int d = 0; d < J.dy; ++d) key.push_back(((long long)J.y[d].proc << 32) | J.y[d].lag);
        key.push_back(-1);
        for (int d = 0; d < J.dz; ++d) key.push_back(((long long)J.z[d].proc << 32) | J.z[d].lag);
        auto it = gid.find(key);
        int g;
        if (it == gid.end()) {
            g = (int)groups.size();
            gid[key] = g;
            HostGroup hg;
            hg.data = J.data;
            hg.max_lag = J.params.max_lag;
            hg.k = J.params.k;
            hg.theiler = J.params.theiler;
            hg.y.assign(J.y, J.y + J.dy);
            if (J.dz) hg.z.assign(J.z, J.z + J.dz);
            hg.dx = J.dx;
            groups.push_back(hg);
        } else {
            g = it->second;
        }
        HostGroup &hg = groups[g];
        const int xfirst = (int)hg.xvars.size();
        hg.xvars.insert(hg.xvars.end(), J.x, J.x + J.dx);
        for (int s = 0; s <= S; ++s)
            hg.members.push_back(HostMember{
                xfirst, s == 0 ? nullptr : perm + job_perm[j] + (size_t)(s - 1) * N,
                job_out[j] + s});
    }
    if ((st = run_groups(ctx, groups, n_out))) return st;
    std::vector<int64_t> keys((size_t)2 * n_out);
    CK(copy_d2h(ctx, keys.data(), ctx->ws_keys.p, keys.size() * 8), "cudaMemcpyAsync");
    CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    for (int j = 0; j < n_jobs; ++j)
        for (int s = 0; s <= jobs[j].params.n_surr; ++s) {
            const int o = job_out[j] + s;
            out[o] = key_to_cmi(ctx, keys[2 * o], (uint64_t)keys[2 * o + 1], jobs[j].params.k,
                                job_N[j]);
        }
    if (out_key) std::memcpy(out_key, keys.data(), keys.size() * 8);
    return TE_OK;
    GUARD_END
}

te_status te_get_stats(const te_ctx *ctx, te_stats *out)
{
    if (!ctx || !out) return TE_EINVAL;
    *out = ctx->stats;
    return TE_OK;
}

}  // extern "C"
