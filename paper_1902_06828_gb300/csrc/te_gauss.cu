// cmi_gauss: linear-Gaussian CMI of one estimate and its permutation
// surrogates (the estimator the paper uses for its VAR networks), and the same
// pipeline over the groups of a network-inference round.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "gauss_internal.h"
#include "ksg_internal.h"
#include "te_runtime.h"

using namespace teksg;

namespace {

constexpr int kGaussBatch = 4096;   // estimates per batched launch (grid z)

// Shape of one estimate (N points, S surrogates, X / Y / Z dimensions, the
// points split `splits` ways for the contraction) and the number of doubles
// of its workspace: means, covariance, the two Cholesky factors, their
// inverse norms, scratch, the cross-covariances and their per-split partial
// sums, and with xc the centred X columns.  The estimates and error bounds
// are bound elsewhere.
size_t gauss_shape(GaussArgs &A, int N, int S, int dx, int dy, int dz, int splits,
                   bool xc = false)
{
    A.N = N;
    A.S = S;
    A.dx = dx;
    A.dy = dy;
    A.dw = dy + dz;
    A.d = dx + dy + dz;
    const int nchunks = (N + 31) / 32;
    splits = std::max(1, std::min(splits, nchunks));
    A.chunks_per_split = (nchunks + splits - 1) / splits;
    A.splits = (nchunks + A.chunks_per_split - 1) / A.chunks_per_split;
    const size_t d = (size_t)A.d, dw = (size_t)A.dw;
    return d + d * d + 2 * dw * dw + 2 + kGaussMaxDims +
           (size_t)(S + 1) * dx * dw * (1 + (size_t)A.splits) + (xc ? (size_t)dx * N : 0);
}

// workspace pointers of a shaped estimate, starting at w (xc: as shaped)
void gauss_bind(GaussArgs &A, double *w, bool xc = false)
{
    const size_t d = (size_t)A.d, dw = (size_t)A.dw;
    A.mean = w;
    A.cov = A.mean + d;
    A.LW = A.cov + d * d;
    A.LZ = A.LW + dw * dw;
    A.norms = A.LZ + dw * dw;
    A.scratch = A.norms + 2;
    A.cross = A.scratch + kGaussMaxDims;
    A.cross_part = A.cross + (size_t)(A.S + 1) * A.dx * dw;
    A.xc = xc ? A.cross_part + (size_t)A.splits * (A.S + 1) * A.dx * dw : nullptr;
    A.covw = A.cov;
    A.own_w = 1;
}

// offset of variable v's column at the first point: the value at point t is
// series[col + t]
int gauss_col(const te_data *data, int max_lag, te_var v)
{
    return v.proc * data->T + max_lag - v.lag;
}

}  // namespace

namespace teksg {

double gauss_key_value(int64_t hi, uint64_t lo)
{
    (void)hi;   // the key is the sign extension of lo
    const long long k = (long long)lo;
    const long long b = k >= 0 ? k : (k ^ 0x7fffffffffffffffLL);
    double v;
    std::memcpy(&v, &b, 8);
    return v;
}

te_status run_groups_gauss(te_ctx *ctx, const std::vector<HostGroup> &groups, int n_out)
{
    // One estimate per candidate of a group: its members share X, Y, Z and
    // differ only in the permutation.  Member s of a candidate writes slot
    // slot0 + s and, for s >= 1, reads permutation perms + (s - 1) N.  The
    // test decisions compare these estimates, so the cross-covariances are
    // float-float (dw <= 16) or FP64 sums (gauss_launch_batch_f64), about
    // 1e-13 from an FP64 evaluation: decisions then agree with it except at
    // ties closer than that, where the split-TF32 contraction of cmi_gauss
    // (~1e-7) would flip near-ties.  Estimates run in batches, one launch per
    // kernel per batch; each has its own workspace.
    std::vector<GaussArgs> est;
    std::vector<int> slot0, gid;   // gid: the estimate's group (same W)
    std::vector<int> cols;
    std::vector<size_t> col0;
    for (const HostGroup &g : groups) {
        const int N = g.data->T - g.max_lag;
        const int dy = (int)g.y.size(), dz = (int)g.z.size();
        if (g.dx > kGaussMaxX || g.dx + dy + dz > kGaussMaxDims)
            return fail(ctx, TE_EINVAL,
                        "the Gaussian estimator takes dx <= 8 and dx + dy + dz <= 40");
        if (N <= g.dx + dy + dz + 1)
            return fail(ctx, TE_EINVAL, "need more points than variables + 1");
        std::map<int, std::vector<const HostMember *>> by;
        for (const HostMember &m : g.members) by[m.xcol_first].push_back(&m);
        for (auto &kv : by) {
            auto &ms = kv.second;
            std::sort(ms.begin(), ms.end(),
                      [](const HostMember *a, const HostMember *b) { return a->out < b->out; });
            const int S = (int)ms.size() - 1;
            const int32_t *p1 = S > 0 ? ms[1]->perm : nullptr;
            bool ok = ms[0]->perm == nullptr;
            for (int s = 1; s <= S && ok; ++s)
                ok = ms[s]->out == ms[0]->out + s && ms[s]->perm == p1 + (size_t)(s - 1) * N;
            if (!ok)
                return fail(ctx, TE_EINTERNAL,
                            "Gaussian estimates need consecutive slots and permutations");
            GaussArgs A{};
            A.N = N;
            A.S = S;
            A.dx = g.dx;
            A.dy = dy;
            A.d = g.dx + dy + dz;   // shape completed per batch
            A.base = g.data->d_series;
            A.perms = p1;
            est.push_back(A);
            gid.push_back((int)(&g - groups.data()));
            slot0.push_back(ms[0]->out);
            col0.push_back(cols.size());
            for (int a = 0; a < g.dx; ++a)
                cols.push_back(gauss_col(g.data, g.max_lag, g.xvars[kv.first + a]));
            for (const te_var &v : g.y) cols.push_back(gauss_col(g.data, g.max_lag, v));
            for (const te_var &v : g.z) cols.push_back(gauss_col(g.data, g.max_lag, v));
        }
    }
    // shapes: a batch splits each estimate's points so that the contraction
    // has about eight CTAs per SM in all
    const int n_est = (int)est.size();
    size_t ws = 0;
    std::vector<size_t> off(n_est);
    for (int b0 = 0; b0 < n_est; b0 += kGaussBatch) {
        const int nb = std::min(kGaussBatch, n_est - b0);
        size_t w = 0;
        for (int i = b0; i < b0 + nb; ++i) {
            GaussArgs &A = est[i];
            const int blocks = ((A.S + 1) * A.dx + 127) / 128;
            const int splits = (8 * 152 + nb * blocks - 1) / (nb * blocks);
            off[i] = w;
            w += gauss_shape(A, A.N, A.S, A.dx, A.dy, A.d - A.dx - A.dy, splits, true);
        }
        ws = std::max(ws, w);
    }
    // doubles: batch workspace, then estimates and bounds of all slots;
    // then the batch's argument blocks; ints: status flags, the columns
    const size_t nd = ws + 2 * (size_t)n_out;
    const size_t args_off = nd * 8;
    const size_t int_off = args_off + (size_t)kGaussBatch * sizeof(GaussArgs);
    te_status st;
    if ((st = ensure_dev(ctx, ctx->ws_gauss, int_off + (2 + cols.size()) * 4))) return st;
    if ((st = ensure_dev(ctx, ctx->ws_keys, (size_t)std::max(n_out, 1) * 16))) return st;
    char *base = (char *)ctx->ws_gauss.p;
    double *w = (double *)base;
    double *v_out = w + ws, *v_err = v_out + n_out;
    GaussArgs *args_dev = (GaussArgs *)(base + args_off);
    int *status = (int *)(base + int_off), *cols_dev = status + 2;
    CK(cudaMemsetAsync(status, 0, 2 * sizeof(int), ctx->stream), "cudaMemsetAsync");
    CK(cudaMemsetAsync(v_out, 0, (size_t)n_out * 8, ctx->stream), "cudaMemsetAsync");
    if (!cols.empty())
        CK(copy_h2d(ctx, cols_dev, cols.data(), cols.size() * 4), "cudaMemcpyAsync");
    int src = 0;
    for (int i = 0; i < n_est; ++i) {
        GaussArgs &A = est[i];
        gauss_bind(A, w + off[i], true);
        A.cols = cols_dev + col0[i];
        A.status = status;
        A.out = v_out + slot0[i];
        A.err = v_err + slot0[i];
        // the group's first estimate in each batch forms the W-W covariance and
        // the factors; the group's later ones in the batch use them
        if (i % kGaussBatch == 0 || gid[i] != gid[i - 1]) {
            src = i;
        } else {
            A.own_w = 0;
            A.covw = est[src].cov;
            A.LW = est[src].LW;
            A.LZ = est[src].LZ;
            A.norms = est[src].norms;
        }
        ctx->stats.estimates += (uint64_t)A.S + 1;
    }
    for (int b0 = 0; b0 < n_est; b0 += kGaussBatch) {
        const int nb = std::min(kGaussBatch, n_est - b0);
        // the previous batch's kernels precede this copy on the stream
        CK(copy_h2d(ctx, args_dev, est.data() + b0, (size_t)nb * sizeof(GaussArgs)),
           "cudaMemcpyAsync");
        CK(gauss_launch_batch_f64(args_dev, est.data() + b0, nb, ctx->stream),
           "Gaussian batch launch");
        ctx->stats.launches += 7;
    }
    CK(gauss_launch_keys(v_out, n_out, (long long *)ctx->ws_keys.p, status, ctx->stream),
       "key launch");
    ctx->stats.launches++;
    int flags[2] = {0, 0};
    CK(copy_d2h(ctx, flags, status, sizeof flags), "cudaMemcpyAsync");
    CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    if (flags[1]) return fail(ctx, TE_ETIMEOUT, "tensor-core contraction did not complete in time");
    if (flags[0]) return fail(ctx, TE_EINVAL, "a covariance block of an estimate is singular");
    return TE_OK;
}

}  // namespace teksg

extern "C" te_status cmi_gauss(te_ctx *ctx, const te_data *data, const te_var *x, int32_t dx,
                               const te_var *y, int32_t dy, const te_var *z, int32_t dz,
                               const te_ksg_params *p, double *out_cmi, double *out_err_bound)
{
    if (!ctx) return TE_EINVAL;
    try {
        ctx->err.clear();
        te_status st;
        if (!p || !out_cmi) return fail(ctx, TE_EINVAL, "params or out_cmi is NULL");
        if ((st = validate_estimate(ctx, data, x, dx, y, dy, z, dz, 1, 0, p->max_lag,
                                    p->n_surr, TE_GAUSS_MAX_DIMS)))
            return st;
        if (dx > kGaussMaxX) return fail(ctx, TE_EINVAL, "cmi_gauss supports dx <= 8");
        const int N = data->T - p->max_lag, S = p->n_surr;
        const int d = dx + dy + dz;
        if (N <= d + 1) return fail(ctx, TE_EINVAL, "need more points than variables + 1");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        // workspace: the estimate's doubles, its estimates and bounds, then ints
        GaussArgs A{};
        const size_t ws = gauss_shape(A, N, S, dx, dy, dz, gauss_tc_splits(N));
        const size_t nd = ws + 2 * (size_t)(S + 1);
        if ((st = ensure_dev(ctx, ctx->ws_gauss, nd * 8 + (size_t)(d + 8) * 4))) return st;
        // permutations as 16-bit rows (pitch a multiple of 8 entries) when the
        // points allow: half the bytes for Fisher-Yates to write and the
        // contraction to read, which reads its rows with 16-byte loads
        const bool p16 = N <= kPerm16MaxN;
        const int pitch16 = (N + 7) & ~7;
        const size_t perm_bytes =
            p16 ? (size_t)std::max(S, 1) * pitch16 * 2 : (size_t)std::max(S, 1) * N * 4;
        if ((st = ensure_dev(ctx, ctx->ws_perm, perm_bytes))) return st;
        double *w = (double *)ctx->ws_gauss.p;
        gauss_bind(A, w);
        A.base = data->d_series;
        A.perms = p16 ? nullptr : (const int32_t *)ctx->ws_perm.p;
        A.perms16 = p16 ? (const uint16_t *)ctx->ws_perm.p : nullptr;
        A.perm_pitch = p16 ? pitch16 : 0;
        if ((st = ensure_dev(ctx, ctx->ws_gtile, gauss_tc_workspace(N, dx, dy + dz)))) return st;
        {
            const size_t nchunks = (size_t)(N + 31) / 32;
            const size_t passes = (size_t)(dy + dz + 31) / 32;
            A.btile = (float *)ctx->ws_gtile.p;
            A.xcen = A.btile + passes * nchunks * 2048;
            A.xcen_pitch = (N + 31) & ~31;
        }
        A.out = w + ws;
        A.err = A.out + (S + 1);
        int *ip = (int *)(w + nd);
        A.status = ip;
        int *cols_dev = ip + 2;
        A.cols = cols_dev;
        std::vector<int> cols;
        for (int a = 0; a < dx; ++a) cols.push_back(gauss_col(data, p->max_lag, x[a]));
        for (int a = 0; a < dy; ++a) cols.push_back(gauss_col(data, p->max_lag, y[a]));
        for (int a = 0; a < dz; ++a) cols.push_back(gauss_col(data, p->max_lag, z[a]));
        CK(copy_h2d(ctx, cols_dev, cols.data(), cols.size() * 4), "cudaMemcpyAsync");
        CK(cudaMemsetAsync(A.status, 0, 2 * sizeof(int), ctx->stream), "cudaMemsetAsync");
        // the statistics (means, covariance, FP64 factors) do not depend on
        // the permutations: they run on the auxiliary stream while the
        // permutations are drawn, and the contraction waits for both
        if ((st = ensure_aux(ctx))) return st;
        CK(cudaEventRecord(ctx->ev_fork, ctx->stream), "cudaEventRecord");
        CK(cudaStreamWaitEvent(ctx->aux_stream, ctx->ev_fork, 0), "cudaStreamWaitEvent");
        CK(gauss_launch_stats(A, ctx->aux_stream), "Gaussian statistics launch");
        CK(cudaEventRecord(ctx->ev_join, ctx->aux_stream), "cudaEventRecord");
        if (p16)
            CK(launch_perms16((uint16_t *)ctx->ws_perm.p, pitch16, N, p->seed, p->stream_tag, 0,
                              0, 1, S, ctx->stream),
               "permutation launch");
        else
            CK(launch_perms((int32_t *)ctx->ws_perm.p, N, N, p->seed, p->stream_tag, 0, 0, 1, S,
                            ctx->stream),
               "permutation launch");
        CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0), "cudaStreamWaitEvent");
        CK(gauss_launch_cross_tc(A, ctx->stream), "tensor-core cross-covariance launch");
        const double gamma = gauss_tc_gamma();
        CK(gauss_launch_schur(A, gamma, ctx->stream), "Schur launch");
        ctx->stats.launches += 7;
        std::vector<double> res(2 * (size_t)(S + 1));
        int status[2] = {0, 0};
        CK(copy_d2h(ctx, res.data(), A.out, res.size() * 8), "cudaMemcpyAsync");
        CK(copy_d2h(ctx, status, A.status, 8), "cudaMemcpyAsync");
        CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
        if (status[1])
            return fail(ctx, TE_ETIMEOUT, "tensor-core contraction did not complete in time");
        if (status[0])
            return fail(ctx, TE_EINVAL, "covariance of the conditioning variables is singular");
        std::memcpy(out_cmi, res.data(), (size_t)(S + 1) * 8);
        if (out_err_bound) std::memcpy(out_err_bound, res.data() + S + 1, (size_t)(S + 1) * 8);
        return TE_OK;
    } catch (...) {
        return fail(ctx, TE_EINTERNAL, "unexpected C++ exception");
    }
}
