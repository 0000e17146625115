// Internal interface between the host runtime and the sm_103a kernels.
// Not part of the public ABI (include/te_ksg.h is).
#pragma once

#include <cuda.h>   // CUtensorMap (type only; the encoder is fetched through the runtime)
#include <cuda_runtime.h>
#include <stdint.h>

namespace teksg {

// A group is a set of members (CMI estimates) that share the conditioning
// variables Z, the target variables Y, the point set and k.  Members differ in
// their X variables and in the permutation applied to X.
struct GroupDesc {
    const float *base;      // device series of the group's data set
    int N;                  // points
    int k;                  // neighbours
    int theiler;            // Theiler window
    int dy, dz, dx;         // dims
    int ycol, zcol;         // first index into cols[] of the Y / Z column offsets
    int member_begin;       // first member of the group in members[]
    int n_members;
    int n_qtiles;           // ceil(N / query tile)
    int n_mblocks;          // ceil(n_members / members per thread)
    long long item_begin;   // first CTA of the group in the launch
    // Spatial order (nullptr sigma = time order).  Points are processed in the
    // leaf order of a k-d tree (large groups) or along a Morton curve over the
    // shared (Y, Z) coordinates: position p is
    // time point sigma[p]; yz[d * N + p] holds Y (d < dy) and Z coordinates in
    // that order; box[d * n_chunks8 + c] = (min, max) of dim d over positions
    // 8c .. 8c + 7.  Only used with theiler == 0.
    const int *sigma;
    const float *yz;
    const float2 *box;
    int n_chunks8;
    const float2 *tbox;     // [dy + dz][n_tiles256]: (min, max) per aligned 256-point tile
    int n_tiles256;
    // Empty Z, one Y and one X variable, no Theiler window: the Y column sorted
    // ascending (else nullptr).  Counts then reduce to 1-D range counts.
    const float *ysorted;
};

// One spatial-order job (one CTA): the k-d tree or Morton order of the (Y, Z)
// coordinates of a group, built in shared memory; writes sigma, yz, box and
// tbox as described above.
struct OrderJob {
    const float *base;
    int N, dyz;
    int cols[32];           // column offsets of Y then Z
    int *sigma;
    float *yz;
    float2 *box;
    float2 *tbox;           // boxes of aligned 256-point tiles
    int kd;                 // 1: k-d tree order, 0: Morton curve
};
constexpr int kMaxOrderN = 16384;   // points a CTA can sort in shared memory
// groups of at least this many members take the k-d tree order: its build
// (one sort per tree level, about 2 ms at N = 10^4) pays back in the kernel
// only over many members; smaller groups take the one-sort Morton curve
constexpr size_t kKdOrderMinMembers = 4096;
cudaError_t launch_order(const OrderJob *jobs, int n_jobs, cudaStream_t st);

struct ComposeJob {
    const int *sigma;
    const int32_t *perm;
    int32_t *out;
    int N;
};
cudaError_t launch_compose(const ComposeJob *jobs, int n_jobs, int max_n, cudaStream_t st);

struct MemberDesc {
    const int32_t *perm;    // device permutation of [0, N) applied to X, or nullptr; in a
                            // sorted group it is composed with the order (position ->
                            // time index of X)
    int xcol;               // first index into cols[] of the dx X column offsets
    int out;                // output slot
    const float *xsorted;   // the X column sorted ascending when the group has ysorted
};

// Sort N floats ascending (one CTA per job, N <= kMaxOrderN).
struct ValueSortJob {
    const float *src;
    float *dst;
    int N;
};
cudaError_t launch_value_sort(const ValueSortJob *jobs, int n_jobs, cudaStream_t st);

// A column is addressed as base + off: the value of the column at point i is
// base[off + i], off = proc * T + max_lag - lag.
struct KsgLaunch {
    const GroupDesc *groups;
    int n_groups;
    const MemberDesc *members;
    const int *cols;
    const int64_t *q;              // digamma fixed-point table Q[0..q_len)
    unsigned long long *acc;       // [2 * n_out]: (low-32-bit partial sums, high parts)
    float *dbg_eps;                // per-point debug outputs for member slot dbg_out
    int *dbg_nxz, *dbg_nyz, *dbg_nz;
    int dbg_out;
    int jt;                        // points per staged j tile
    unsigned long long *work;      // [0] += member-pair evaluations executed (both passes),
                                   // [1] += algorithmic ops of those evaluations,
                                   // [2] != 0: a tile copy did not complete in time
    // member-lane kernel with tensor-memory-access staging: X value of member
    // row r (the member's index in this launch) at position j is
    // xval[r * xpitch + j] (positions in the group's order, zero past N)
    const float *xval;
    long long xpitch;
    // persistent member-lane grid (nullptr: one CTA per item): items are taken
    // from this counter, zeroed before the launch; n_items = items of the launch
    unsigned long long *item_counter;
    long long n_items;
};

// Kernel variants: members per thread and k.  kgen = 0 means k is a template
// constant; otherwise a runtime k <= TE_MAX_K.
struct KsgVariant {
    int m;      // members per thread; 32 (64) selects the member-lane kernel with one (two)
                // members per lane
    int kt;     // template k (0 = runtime k)
    int qt;     // threads per CTA
    bool tma;   // member-lane kernel: X tiles copied by the tensor memory accelerator
                // from the launch's X-value rows (false: gathered by the threads)
    bool persist = false;   // member-lane TMA kernel as a persistent grid (KsgLaunch::item_counter)
};

// member-lane kernel (single-variable X): 32 members x 32 query points per CTA
constexpr int kLaneQueries = 32;
constexpr int kLaneThreads = 256;
inline size_t ksg_lane_smem_bytes(int dyz, int jt, int members = 32)
{
    const int warps = kLaneThreads / 32;
    return 4 * ((size_t)dyz * jt + (size_t)members * (jt + 4)) +
           (size_t)warps * (2 * 4 * 8 * 4 + 4 * 4 * (size_t)dyz + 4 * (size_t)(jt / 64));
}

// TMA-staged lane kernel: X tiles are [jt / 32 segments][members][32 points],
// 128-byte swizzled, 1024-byte aligned (hence the slack)
inline size_t ksg_lane_tma_smem_bytes(int dyz, int jt, int members)
{
    const int warps = kLaneThreads / 32;
    return 1024 + 4 * ((size_t)dyz * jt + (size_t)members * jt) +
           (size_t)warps * (2 * 4 * 8 * 4 + 4 * 4 * (size_t)dyz + 4 * (size_t)(jt / 64));
}

// tmap: the 2-D tensor map of L.xval for TMA variants (nullptr otherwise).
// With v.persist (member-lane TMA kernels only; L.item_counter set) the grid is persistent:
// as many CTAs as fit on the device at once, each taking items from the
// counter.
cudaError_t launch_ksg(const KsgLaunch &L, const KsgVariant &v, long long n_items, bool dx1,
                       size_t smem_bytes, cudaStream_t st, const CUtensorMap *tmap = nullptr);
// X-value rows of every member of the launch (L.xval, row pitch L.xpitch floats)
cudaError_t launch_xval(const KsgLaunch &L, int n_rows, cudaStream_t st);
// tensor map over rows x pitch floats at xval, box = 32 points x box_rows rows,
// 128-byte swizzle; cudaErrorNotSupported when the driver lacks the encoder
cudaError_t encode_xval_map(CUtensorMap *map, const float *xval, long long pitch, int rows,
                            int box_rows);
cudaError_t ksg_prepare_attributes();

// dynamic shared memory of the fused kernel: the staged tile, the query-side
// values, per-warp chunk bounds, the staged index row and the per-thread
// (d_Z, d_YZ) scratch of one 8-point chunk
inline size_t ksg_smem_bytes(int rows_t, int rows_q, int jt, int qt)
{
    return 4 * ((size_t)rows_t * jt + (size_t)rows_q * qt) + 8 * (size_t)(qt / 32) * (jt / 8) +
           4 * (size_t)jt + 8 * 8 * (size_t)qt;
}

// Fisher-Yates permutations of [0, n), one per surrogate s = s_first .. s_first +
// n_perm - 1, keyed by SplitMix64 over (seed, target, stage, iter, s).
cudaError_t launch_perms(int32_t *out, long long stride, int n, uint64_t seed, uint64_t target,
                         uint64_t stage, uint64_t iter, uint64_t s_first, int n_perm,
                         cudaStream_t st);

// The same permutations as launch_perms for n <= kPerm16MaxN, as 16-bit rows of
// `pitch` entries (pitch a multiple of 8 and >= n, zeros past n; out 16-byte
// aligned): permutation s - s_first at out + (s - s_first) * pitch.
constexpr int kPerm16MaxN = 65535;
cudaError_t launch_perms16(uint16_t *out, int pitch, int n, uint64_t seed, uint64_t target,
                           uint64_t stage, uint64_t iter, uint64_t s_first, int n_perm,
                           cudaStream_t st);

// Surrogates of R pooled trials of n points (R * n ints per surrogate, n_perm
// of them at out): mode 0 shuffles the trial order, mode 1 the points inside
// each trial, keyed like launch_perms.
cudaError_t launch_perms_trials(int32_t *out, int R, int n, uint64_t seed, uint64_t target,
                                uint64_t stage, uint64_t iter, uint64_t s_first, int n_perm,
                                int mode, cudaStream_t st);

// Many requests of launch_perms in one launch; request r writes n_perm
// permutations of [0, n) at out (stride n) for s = s_first .. s_first+n_perm-1,
// and owns launch CTAs perm_begin .. perm_begin + n_perm - 1.
struct PermJob {
    int32_t *out;
    int n, n_perm;
    uint64_t s_first, seed, target, stage, iter;
    long long perm_begin;
};
cudaError_t launch_perms_multi(const PermJob *jobs, int n_jobs, long long total, int max_n,
                               cudaStream_t st);

// acc (low, high partial sums) -> normalised 128-bit keys (hi, lo) per slot.
cudaError_t launch_finalize(const unsigned long long *acc, long long *keys, int n_out,
                            cudaStream_t st);

// Test statistics over keys laid out [n_cand][S + 1] (slot c * (S + 1) + s
// from req.slot): mode 0 = maximum statistic, 1 = minimum statistic.  One CTA
// per request writes ibuf[cnt_off] = argmax (or argmin) of the originals (ties
// -> lowest index), ibuf[cnt_off + 1 + c] = #{s : null_s > original_c} with
// null_s the max (or min) over candidates of surrogate s, and the originals as
// (hi, lo) pairs at obuf[2 (orig_off + c)].
struct StatReq {
    long long slot;
    int n_cand, S, mode;
    int cnt_off, orig_off;
};
cudaError_t launch_stats(const long long *keys, const StatReq *reqs, int n_req, int max_S,
                         int *ibuf, long long *obuf, cudaStream_t st);

// flag[0] = 1 if any of n values is not finite
cudaError_t launch_check_finite(const float *x, long long n, int *flag, cudaStream_t st);

}  // namespace teksg
