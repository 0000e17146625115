// Host-side runtime shared by the C-ABI translation units (not public).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "te_ksg.h"
#include "ksg_internal.h"

namespace teksg {

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

struct HostMember {
    int xcol_first;           // index into the job's column list
    const int32_t *perm;      // device permutation or nullptr
    int out;                  // output slot
};

// One group = members sharing data, point set, k, theiler, Y and Z.
struct HostGroup {
    const te_data *data = nullptr;
    int max_lag = 0;
    int k = 4, theiler = 0;
    std::vector<te_var> y, z;
    int dx = 1;
    std::vector<te_var> xvars;     // dx variables per member, member-major
    std::vector<HostMember> members;
};

struct te_status_error {
    te_status st;
    std::string msg;
};

}  // namespace teksg

struct te_data {
    te_ctx *ctx;
    float *d_series;
    int32_t n_proc, T;
    // pooled replications (te_data_create_trials): the rows are the embedded
    // columns (p, l), p < n_proc_orig, l <= emb_lag, at row p * (emb_lag + 1) + l,
    // each holding n_rep trials of trial_len points; emb_lag < 0 for plain data
    int32_t n_rep = 1, trial_len = 0, emb_lag = -1, n_proc_orig = 0;
};

struct te_ctx {
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    std::string err;
    // digamma fixed-point table Q[0..q_len) on the device, built on the host in
    // double-double arithmetic (psi(n) = -gamma + H_{n-1}).
    std::vector<int64_t> q_host;
    double dd_hi = 0.0, dd_lo = 0.0;   // running psi(q_host.size() - 1) in double-double
    int64_t *q_dev = nullptr;
    int q_dev_len = 0;
    // grow-only device workspaces
    teksg::DevBuf ws_groups, ws_members, ws_cols, ws_acc, ws_keys, ws_perm, ws_stat, ws_dbg;
    teksg::DevBuf ws_order, ws_ojobs, ws_cperm, ws_gauss, ws_vsort;
    teksg::DevBuf ws_xval;   // X-value rows of the TMA-staged lane kernel
    teksg::DevBuf ws_gtile;  // cmi_gauss: the contraction's prepared B tiles and centred X
    // pinned host staging
    void *pin = nullptr;
    size_t pin_cap = 0;
    te_stats stats{};
    // counters of the launch in flight, added to stats by finish_groups
    int pend_timed = 0;
    uint64_t pend_pair_evals = 0, pend_members = 0;
    struct te_server *server = nullptr;   // serving state (te_serve_*), created on demand
    std::mutex serve_start_mu;
    unsigned long long *work_dev = nullptr;   // KSG kernel work counters [2], error flag [1],
                                              // persistent-grid item counter [1]
    unsigned long long *work_host = nullptr;  // pinned copy
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    // second stream for work that overlaps the context's stream (created on
    // first use) and the events that fork to it and join back
    cudaStream_t aux_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int prepared = 0;
    te_trace_fn trace_fn = nullptr;   // te_ctx_set_trace
    void *trace_user = nullptr;
    // te_ctx_set_option: forced member-lane tile / members per lane (0 = the
    // tuning table), persistent member-lane grids, batches captured as graphs
    int opt_jt = 0, opt_ms = 0, opt_persistent = 0, opt_graph = 0, opt_order = 0;
};

namespace teksg {

// status helpers; CK returns from the calling function on a CUDA error
#define CK(call, what)                                                  \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return ::teksg::cuda_fail(ctx, e_, what); \
    } while (0)

te_status fail(te_ctx *ctx, te_status st, const std::string &msg);
// largest autocorrelation decay time over process `proc` (>= 0) or all (-1)
te_status autocorr_decay(te_ctx *ctx, const te_data *data, int32_t proc, int32_t *out_tau);
te_status cuda_fail(te_ctx *ctx, cudaError_t e, const char *what);

te_status ensure_dev(te_ctx *ctx, DevBuf &b, size_t bytes);
te_status ensure_pin(te_ctx *ctx, size_t bytes);
te_status ensure_aux(te_ctx *ctx);   // ctx->aux_stream, ev_fork, ev_join
te_status ensure_q(te_ctx *ctx, int n_needed);   // Q[0..n_needed] on the device
// Q[0..n_max] into a caller buffer (host), same arithmetic as ensure_q
void digamma_q_fill(int n_max, int64_t *q);

// cudaMemcpyAsync on the context's stream, counted in ctx->stats
cudaError_t copy_h2d(te_ctx *ctx, void *dst, const void *src, size_t bytes);
cudaError_t copy_d2h(te_ctx *ctx, void *dst, const void *src, size_t bytes);

// Validate one estimate's variables against its data and parameters: the pure
// form reports through msg (safe from any thread); the other sets ctx->err.
// max_dims: TE_MAX_DIMS for the KSG estimator, TE_GAUSS_MAX_DIMS for the
// linear-Gaussian one.
te_status check_estimate(const te_ctx *ctx, const te_data *data, const te_var *x, int dx,
                         const te_var *y, int dy, const te_var *z, int dz, int k, int theiler,
                         int max_lag, int n_surr, std::string &msg, int max_dims = TE_MAX_DIMS);
te_status validate_estimate(te_ctx *ctx, const te_data *data, const te_var *x, int dx,
                            const te_var *y, int dy, const te_var *z, int dz, int k, int theiler,
                            int max_lag, int n_surr, int max_dims = TE_MAX_DIMS);

// Run every group in fused launches; keys of all n_out slots end up in
// ctx->ws_keys as int64 pairs (hi, lo).  Slots not written by any member are 0.
te_status run_groups(te_ctx *ctx, const std::vector<HostGroup> &groups, int n_out,
                     int dbg_out = -1, float *dbg_eps = nullptr, int *dbg_nxz = nullptr,
                     int *dbg_nyz = nullptr, int *dbg_nz = nullptr);

// The same work in two halves: launch_groups queues everything on ctx->stream
// (keys land in ctx->ws_keys); finish_groups synchronises and updates stats.
te_status launch_groups(te_ctx *ctx, const std::vector<HostGroup> &groups, int n_out,
                        int dbg_out = -1, float *dbg_eps = nullptr, int *dbg_nxz = nullptr,
                        int *dbg_nyz = nullptr, int *dbg_nz = nullptr);
te_status finish_groups(te_ctx *ctx);

double key_to_cmi(const te_ctx *ctx, int64_t hi, uint64_t lo, int k, int N);

// The groups' estimates by the linear-Gaussian estimator (cmi_gauss's
// pipeline with a float-float or FP64 contraction, one estimate per candidate:
// its members must hold consecutive slots and consecutive permutations).
// ctx->ws_keys receives, per slot, the order-preserving int128 image of the
// FP64 estimate, so the test statistics compare estimates; gauss_key_value
// inverts it.  Blocks until done.
te_status run_groups_gauss(te_ctx *ctx, const std::vector<HostGroup> &groups, int n_out);
double gauss_key_value(int64_t hi, uint64_t lo);

}  // namespace teksg
