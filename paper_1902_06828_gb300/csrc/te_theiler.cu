// te_autocorr_decay: the Theiler-window heuristic (Supporting Information,
// dynamic correlation exclusion): the autocorrelation decay time of a
// process, the shortest time shift at which its autocorrelation function has
// dropped by a factor 1/e from the zero-shift value.
//
// r(tau) = sum_{t < T - tau} (x_t - m)(x_{t+tau} - m) / sum_t (x_t - m)^2 with
// m the mean of the whole series (the biased sample estimator), every sum in
// FP64; the decay time is the smallest tau >= 1 with r(tau) <= 1/e (the FP64
// number nearest to e^-1), T - 1 when there is none, 1 for a constant series.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "te_runtime.h"

using namespace teksg;

namespace {

constexpr int kAcfThreads = 1024;
constexpr double kInvE = 0x1.78b56362cef38p-2;   // nearest FP64 to e^-1

// sum over the CTA; every thread gets the result
__device__ double block_sum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();   // red is free (previous readers done)
    if (lane == 0) red[warp] = v;
    __syncthreads();
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// one CTA per requested process
__global__ void __launch_bounds__(kAcfThreads) acf_decay_kernel(const float *series, int T,
                                                                const int *procs, int *out)
{
    __shared__ double red[32];
    const float *x = series + (size_t)procs[blockIdx.x] * T;
    double s = 0.0;
    for (int t = threadIdx.x; t < T; t += blockDim.x) s += (double)x[t];
    const double m = block_sum(s, red) / (double)T;
    double q = 0.0;
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        const double d = (double)x[t] - m;
        q += d * d;
    }
    const double den = block_sum(q, red);
    int result = T - 1;
    if (den == 0.0) {
        result = 1;
    } else {
        for (int tau = 1; tau < T; ++tau) {   // bounded: at most T - 1 shifts
            double p = 0.0;
            for (int t = threadIdx.x; t < T - tau; t += blockDim.x)
                p += ((double)x[t] - m) * ((double)x[t + tau] - m);
            const double num = block_sum(p, red);   // identical in every thread
            if (num / den <= kInvE) {
                result = tau;
                break;
            }
        }
    }
    if (threadIdx.x == 0) out[blockIdx.x] = result;
}

}  // namespace

namespace teksg {

te_status autocorr_decay(te_ctx *ctx, const te_data *data, int32_t proc, int32_t *out_tau)
{
    std::vector<int> procs;
    if (proc >= 0) procs.push_back(proc);
    else
        for (int p = 0; p < data->n_proc; ++p) procs.push_back(p);
    const size_t n = procs.size();
    te_status st;
    if ((st = ensure_dev(ctx, ctx->ws_stat, 2 * n * sizeof(int) + 16))) return st;
    int *d_procs = (int *)ctx->ws_stat.p, *d_out = d_procs + n;
    CK(copy_h2d(ctx, d_procs, procs.data(), n * sizeof(int)), "cudaMemcpyAsync");
    acf_decay_kernel<<<(unsigned)n, kAcfThreads, 0, ctx->stream>>>(data->d_series, data->T,
                                                                    d_procs, d_out);
    CK(cudaGetLastError(), "autocorrelation launch");
    ctx->stats.launches++;
    std::vector<int> taus(n);
    CK(copy_d2h(ctx, taus.data(), d_out, n * sizeof(int)), "cudaMemcpyAsync");
    CK(cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    *out_tau = *std::max_element(taus.begin(), taus.end());
    return TE_OK;
}

}  // namespace teksg

extern "C" te_status te_autocorr_decay(te_ctx *ctx, const te_data *data, int32_t proc,
                                       int32_t *out_tau)
{
    if (!ctx) return TE_EINVAL;
    try {
        ctx->err.clear();
        if (!data || !out_tau) return fail(ctx, TE_EINVAL, "NULL argument");
        if (data->ctx != ctx) return fail(ctx, TE_EINVAL, "data belongs to another context");
        if (proc < -1 || proc >= data->n_proc)
            return fail(ctx, TE_EINVAL, "proc must be -1 (all) or a process index");
        if (data->T < 2) return fail(ctx, TE_EINVAL, "need T >= 2");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        return autocorr_decay(ctx, data, proc, out_tau);
    } catch (...) {
        return fail(ctx, TE_EINTERNAL, "unexpected C++ exception");
    }
}
