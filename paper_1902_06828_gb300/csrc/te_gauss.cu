// cmi_gauss: linear-Gaussian CMI of one estimate and its permutation
// surrogates (the estimator the paper uses for its VAR networks).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "gauss_internal.h"
#include "te_runtime.h"

using namespace teksg;

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
                                    p->n_surr)))
            return st;
        if (dx > kGaussMaxX) return fail(ctx, TE_EINVAL, "cmi_gauss supports dx <= 8");
        const int N = data->T - p->max_lag, S = p->n_surr;
        const int d = dx + dy + dz, dw = dy + dz;
        if (N <= d + 1) return fail(ctx, TE_EINVAL, "need more points than variables + 1");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        // workspace layout (doubles first, then ints)
        const int splits = gauss_cross_splits((S + 1) * dx, N);
        const int nchunks = (N + 31) / 32;
        const size_t nd = (size_t)d + (size_t)d * d + 2 * (size_t)dw * dw + 2 + kGaussMaxDims +
                          (size_t)(S + 1) * dx * dw * (1 + (size_t)splits) + 2 * (size_t)(S + 1);
        const size_t bytes = nd * 8 + (size_t)(d + 8) * 4;
        if ((st = ensure_dev(ctx, ctx->ws_gauss, bytes))) return st;
        if ((st = ensure_dev(ctx, ctx->ws_perm, (size_t)std::max(S, 1) * N * 4))) return st;
        double *w = (double *)ctx->ws_gauss.p;
        GaussArgs A{};
        A.base = data->d_series;
        A.N = N;
        A.S = S;
        A.dx = dx;
        A.dy = dy;
        A.dw = dw;
        A.d = d;
        A.perms = (const int32_t *)ctx->ws_perm.p;
        A.mean = w;
        A.cov = A.mean + d;
        A.LW = A.cov + (size_t)d * d;
        A.LZ = A.LW + (size_t)dw * dw;
        A.norms = A.LZ + (size_t)dw * dw;
        A.scratch = A.norms + 2;
        A.cross = A.scratch + kGaussMaxDims;
        A.out = A.cross + (size_t)(S + 1) * dx * dw;
        A.err = A.out + (S + 1);
        A.cross_part = A.err + (S + 1);
        A.splits = splits;
        A.chunks_per_split = (nchunks + splits - 1) / splits;
        A.splits = (nchunks + A.chunks_per_split - 1) / A.chunks_per_split;
        int *ip = (int *)(A.cross_part + (size_t)splits * (S + 1) * dx * dw);
        A.status = ip;
        int *cols_dev = ip + 2;
        A.cols = cols_dev;
        std::vector<int> cols;
        for (int a = 0; a < dx; ++a) cols.push_back(x[a].proc * data->T + p->max_lag - x[a].lag);
        for (int a = 0; a < dy; ++a) cols.push_back(y[a].proc * data->T + p->max_lag - y[a].lag);
        for (int a = 0; a < dz; ++a) cols.push_back(z[a].proc * data->T + p->max_lag - z[a].lag);
        CK(copy_h2d(ctx, cols_dev, cols.data(), cols.size() * 4), "cudaMemcpyAsync");
        CK(launch_perms((int32_t *)ctx->ws_perm.p, N, N, p->seed, p->stream_tag, 0, 0, 1, S,
                        ctx->stream),
           "permutation launch");
        CK(cudaMemsetAsync(A.status, 0, 2 * sizeof(int), ctx->stream), "cudaMemsetAsync");
        CK(gauss_launch_stats(A, ctx->stream), "Gaussian statistics launch");
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
