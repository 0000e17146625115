// sm_103a kernels of the KSG conditional-mutual-information engine.
//
// ksg_fused_kernel -- one CTA owns QT query points x M members of one group
// (members share Y, Z and the point set; they differ in X and in the
// permutation of X).  Each thread owns one query point i and M members:
//   pass 1 sweeps every j, builds d_Z(i,j) and d_YZ(i,j) once and, for each
//          member, keeps the k smallest joint distances max(d_X, d_YZ) in
//          registers (ascending min/max insertion network), giving eps_i;
//   pass 2 sweeps every j again and counts d_Z < eps, max(d_X, d_Z) < eps and
//          d_YZ < eps per member (strict <);
//   the thread then forms Q[n_z+1] - Q[n_xz+1] - Q[n_yz+1] (exact int64) and
//   the CTA adds it into the member's 128-bit key with warp shuffles and two
//   64-bit atomics.
// j tiles of Y, Z and the permuted X columns are staged in shared memory;
// every lane of a warp reads the same staged element (broadcast), so the hot
// loop is pure FP32 subtract / max / compare on registers.
// Estimator: Kraskov's I^(1) extended to CMI (Methods, "Coupled logistic maps
// process"); surrogates permute X only (Statistical tests, "Maximum statistic
// test").  Max-norm distances are exact float32 |a - b| (no FMA, no fast-math).
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "ksg_internal.h"

namespace teksg {

namespace {

constexpr int QT = 128;   // query points (threads) per CTA
constexpr int JC = 8;     // j points per register chunk
constexpr int KMAX = 16;  // runtime-k buffer

// Insert D into the ascending buffer b (precondition D < b[K-1]).  New b[a] is
// the a-th smallest of {b, D}: max(b[a-1], min(b[a], D)).
template <int K>
__device__ __forceinline__ void topk_insert(float (&b)[K], float D)
{
#pragma unroll
    for (int a = K - 1; a > 0; --a) b[a] = fmaxf(b[a - 1], fminf(b[a], D));
    b[0] = fminf(b[0], D);
}

template <int K>
__device__ __forceinline__ float topk_at(const float (&b)[K], int idx)
{
    float r = b[0];
#pragma unroll
    for (int a = 1; a < K; ++a) r = (a == idx) ? b[a] : r;
    return r;
}

__device__ __forceinline__ void load8(const float *p, float (&v)[JC])
{
    const float4 a = *reinterpret_cast<const float4 *>(p);
    const float4 b = *reinterpret_cast<const float4 *>(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// Shared-subspace distances for JC consecutive staged points starting at c:
// dzv = max over Z dims (-inf if dz == 0), dyzv = max(dzv, max over Y dims).
__device__ __forceinline__ void shared_dist(const float *tile, const float *qv, int jt, int dy,
                                            int dz, int c, float (&dzv)[JC], float (&dyzv)[JC])
{
#pragma unroll
    for (int u = 0; u < JC; ++u) dzv[u] = -CUDART_INF_F;
    for (int d = 0; d < dz; ++d) {
        const float zi = qv[(dy + d) * QT + threadIdx.x];
        float zj[JC];
        load8(tile + (dy + d) * jt + c, zj);
#pragma unroll
        for (int u = 0; u < JC; ++u) dzv[u] = fmaxf(dzv[u], fabsf(__fsub_rn(zi, zj[u])));
    }
#pragma unroll
    for (int u = 0; u < JC; ++u) dyzv[u] = dzv[u];
    for (int d = 0; d < dy; ++d) {
        const float yi = qv[d * QT + threadIdx.x];
        float yj[JC];
        load8(tile + d * jt + c, yj);
#pragma unroll
        for (int u = 0; u < JC; ++u) dyzv[u] = fmaxf(dyzv[u], fabsf(__fsub_rn(yi, yj[u])));
    }
}

// Member distance d_X for JC staged points (generic dx; X query values in smem).
template <int M>
__device__ __forceinline__ void member_dist(const float *tile, const float *qv, int jt, int dy,
                                            int dz, int dx, int m, int c, float (&dcv)[JC])
{
#pragma unroll
    for (int u = 0; u < JC; ++u) dcv[u] = -CUDART_INF_F;
    for (int d = 0; d < dx; ++d) {
        const int row = dy + dz + m * dx + d;
        const float xq = qv[row * QT + threadIdx.x];
        float xj[JC];
        load8(tile + row * jt + c, xj);
#pragma unroll
        for (int u = 0; u < JC; ++u) dcv[u] = fmaxf(dcv[u], fabsf(__fsub_rn(xq, xj[u])));
    }
}

template <int M, int KT, bool DX1>
__global__ void __launch_bounds__(QT) ksg_fused_kernel(const KsgLaunch L)
{
    constexpr int KB = KT > 0 ? KT : KMAX;
    extern __shared__ __align__(16) float smem[];

    // ---- decode the work item: group, member block, query tile ----
    const long long item = blockIdx.x;
    int glo = 0, ghi = L.n_groups - 1;
    while (glo < ghi) {
        const int mid = (glo + ghi + 1) >> 1;
        if (L.groups[mid].item_begin <= item) glo = mid;
        else ghi = mid - 1;
    }
    const GroupDesc G = L.groups[glo];
    const long long local = item - G.item_begin;
    const int mb = (int)(local / G.n_qtiles);
    const int qtile = (int)(local % G.n_qtiles);
    const int N = G.N, dy = G.dy, dz = G.dz, dx = G.dx, w = G.theiler;
    const int k = KT > 0 ? KT : G.k;
    const int jt = L.jt;
    const float *__restrict__ base = G.base;

    const int rows_t = dy + dz + M * dx;
    float *tile = smem;                       // [rows_t][jt]
    float *qv = smem + rows_t * jt;           // [rows_q][QT]
    __shared__ const int32_t *s_perm[M];
    __shared__ int s_out[M];
    __shared__ int s_valid[M];

    const int tid = threadIdx.x;
    const int i = qtile * QT + tid;
    const bool qvalid = i < N;
    const int ic = qvalid ? i : N - 1;
    const int qlo = qtile * QT;
    const int qhi = min(qlo + QT, N) - 1;

    if (tid < M) {
        const int mi = mb * M + tid;
        const int mc = mi < G.n_members ? mi : G.n_members - 1;
        const MemberDesc md = L.members[G.member_begin + mc];
        s_perm[tid] = md.perm;
        s_out[tid] = md.out;
        s_valid[tid] = mi < G.n_members;
    }
    __syncthreads();

    // query-side values
    for (int d = 0; d < dy; ++d) qv[d * QT + tid] = base[L.cols[G.ycol + d] + ic];
    for (int d = 0; d < dz; ++d) qv[(dy + d) * QT + tid] = base[L.cols[G.zcol + d] + ic];
    float xi[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int mi = min(mb * M + m, G.n_members - 1);
        const MemberDesc md = L.members[G.member_begin + mi];
        const int pi = md.perm ? md.perm[ic] : ic;
        if (DX1) {
            xi[m] = base[L.cols[md.xcol] + pi];
        } else {
            xi[m] = 0.f;
            for (int d = 0; d < dx; ++d)
                qv[(dy + dz + m * dx + d) * QT + tid] = base[L.cols[md.xcol + d] + pi];
        }
    }

    auto stage = [&](int j0) {
        for (int r = 0; r < rows_t; ++r) {
            int off;
            const int32_t *perm = nullptr;
            if (r < dy) {
                off = L.cols[G.ycol + r];
            } else if (r < dy + dz) {
                off = L.cols[G.zcol + r - dy];
            } else {
                const int m = (r - dy - dz) / dx, d = (r - dy - dz) - m * dx;
                const int mi = min(mb * M + m, G.n_members - 1);
                off = L.cols[L.members[G.member_begin + mi].xcol + d];
                perm = s_perm[m];
            }
            for (int jj = tid; jj < jt; jj += QT) {
                const int j = j0 + jj;
                float v = 0.f;
                if (j < N) v = base[off + (perm ? perm[j] : j)];
                tile[r * jt + jj] = v;
            }
        }
    };

    // chunk needs per-pair masking if it reaches past N or meets the Theiler
    // band |i - j| <= w of any query point of this CTA
    auto needs_mask = [&](int j) {
        return (j + JC > N) || (j <= qhi + w && j + JC - 1 >= qlo - w);
    };
    auto apply_mask = [&](int j, float(&dzv)[JC], float(&dyzv)[JC]) {
#pragma unroll
        for (int u = 0; u < JC; ++u) {
            const int jj = j + u;
            const int gap = jj > i ? jj - i : i - jj;
            if (jj >= N || gap <= w) {
                dzv[u] = CUDART_INF_F;
                dyzv[u] = CUDART_INF_F;
            }
        }
    };

    // ---------------- pass 1: k nearest joint distances ----------------
    float buf[M][KB];
    float thr[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
#pragma unroll
        for (int a = 0; a < KB; ++a) buf[m][a] = CUDART_INF_F;
        thr[m] = CUDART_INF_F;
    }

    for (int j0 = 0; j0 < N; j0 += jt) {
        __syncthreads();
        stage(j0);
        __syncthreads();
        const int jn = min(jt, N - j0);
        for (int c = 0; c < jn; c += JC) {
            float dzv[JC], dyzv[JC];
            shared_dist(tile, qv, jt, dy, dz, c, dzv, dyzv);
            if (needs_mask(j0 + c)) apply_mask(j0 + c, dzv, dyzv);
#pragma unroll
            for (int m = 0; m < M; ++m) {
                float dcv[JC];
                if (DX1) {
                    float xj[JC];
                    load8(tile + (dy + dz + m) * jt + c, xj);
#pragma unroll
                    for (int u = 0; u < JC; ++u) dcv[u] = fabsf(__fsub_rn(xi[m], xj[u]));
                } else {
                    member_dist<M>(tile, qv, jt, dy, dz, dx, m, c, dcv);
                }
#pragma unroll
                for (int u = 0; u < JC; ++u) {
                    const float D = fmaxf(dcv[u], dyzv[u]);
                    if (D < thr[m]) {
                        topk_insert<KB>(buf[m], D);
                        thr[m] = KT > 0 ? buf[m][KB - 1] : topk_at<KB>(buf[m], k - 1);
                    }
                }
            }
        }
    }

    // ---------------- pass 2: strict range counts ----------------
    float eps[M];
    int cxz[M], cyz[M], cz[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        eps[m] = thr[m];
        cxz[m] = cyz[m] = cz[m] = 0;
    }
    for (int j0 = 0; j0 < N; j0 += jt) {
        if (N > jt || j0 > 0) {
            __syncthreads();
            stage(j0);
            __syncthreads();
        }
        const int jn = min(jt, N - j0);
        for (int c = 0; c < jn; c += JC) {
            float dzv[JC], dyzv[JC];
            shared_dist(tile, qv, jt, dy, dz, c, dzv, dyzv);
            if (needs_mask(j0 + c)) apply_mask(j0 + c, dzv, dyzv);
#pragma unroll
            for (int m = 0; m < M; ++m) {
                float dcv[JC];
                if (DX1) {
                    float xj[JC];
                    load8(tile + (dy + dz + m) * jt + c, xj);
#pragma unroll
                    for (int u = 0; u < JC; ++u) dcv[u] = fabsf(__fsub_rn(xi[m], xj[u]));
                } else {
                    member_dist<M>(tile, qv, jt, dy, dz, dx, m, c, dcv);
                }
                const float e = eps[m];
#pragma unroll
                for (int u = 0; u < JC; ++u) {
                    const bool pz = dzv[u] < e;
                    cz[m] += pz ? 1 : 0;
                    cxz[m] += (pz && dcv[u] < e) ? 1 : 0;
                    cyz[m] += (dyzv[u] < e) ? 1 : 0;
                }
            }
        }
    }

    // ---------------- digamma key: exact int64 terms, 128-bit sums ----------------
    const int lane = tid & 31;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        long long term = 0;
        if (qvalid)
            term = L.q[cz[m] + 1] - L.q[cxz[m] + 1] - L.q[cyz[m] + 1];
        if (L.dbg_eps && qvalid && s_valid[m] && s_out[m] == L.dbg_out) {
            L.dbg_eps[i] = eps[m];
            L.dbg_nxz[i] = cxz[m];
            L.dbg_nyz[i] = cyz[m];
            L.dbg_nz[i] = cz[m];
        }
        // |term| < 2^57 for N < 2^31, so a 32-lane sum fits in int64
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) term += __shfl_down_sync(0xffffffffu, term, o);
        if (lane == 0 && s_valid[m]) {
            const unsigned long long lo = (unsigned long long)term & 0xffffffffull;
            const long long hi = term >> 32;
            atomicAdd(&L.acc[2 * s_out[m]], lo);
            atomicAdd(&L.acc[2 * s_out[m] + 1], (unsigned long long)hi);
        }
    }
}

// ---------------- SplitMix64 + Fisher-Yates ----------------
__device__ __forceinline__ uint64_t sm64_next(uint64_t &s)
{
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t sm64_once(uint64_t x) { return sm64_next(x); }

__global__ void fisher_yates_kernel(int32_t *out, long long stride, int n, uint64_t seed,
                                    uint64_t target, uint64_t stage, uint64_t iter, int s_first,
                                    int in_smem)
{
    extern __shared__ int32_t sperm[];
    const uint64_t s = (uint64_t)(s_first + (int)blockIdx.x);
    int32_t *p = in_smem ? sperm : out + (long long)blockIdx.x * stride;
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = i;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t h = sm64_once(seed ^ target);
        h = sm64_once(h ^ stage);
        h = sm64_once(h ^ iter);
        uint64_t st = sm64_once(h ^ s);
        for (int i = n - 1; i >= 1; --i) {
            const uint64_t r = sm64_next(st);
            const int j = (int)__umul64hi(r, (uint64_t)(i + 1));
            const int32_t t = p[i];
            p[i] = p[j];
            p[j] = t;
        }
    }
    __syncthreads();
    if (in_smem)
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            out[(long long)blockIdx.x * stride + i] = sperm[i];
}

__global__ void finalize_kernel(const unsigned long long *acc, long long *keys, int n_out)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n_out) return;
    const __int128 K = ((__int128)(long long)acc[2 * o + 1] << 32) + (__int128)acc[2 * o];
    keys[2 * o] = (long long)(K >> 64);
    keys[2 * o + 1] = (long long)(unsigned long long)K;
}

__device__ __forceinline__ __int128 key_at(const long long *keys, long long slot)
{
    return ((__int128)keys[2 * slot] << 64) | (__int128)(unsigned long long)keys[2 * slot + 1];
}

// One CTA per request; null_s kept in dynamic shared memory as 128-bit values.
__global__ void stats_kernel(const long long *keys, const StatReq *reqs, int *ibuf,
                             long long *obuf)
{
    extern __shared__ __int128 snull[];
    const StatReq R = reqs[blockIdx.x];
    const long long stride = R.S + 1;
    const long long *kb = keys + 2 * R.slot;
    if (threadIdx.x == 0) {
        int b = 0;
        __int128 bv = key_at(kb, 0);
        for (int c = 1; c < R.n_cand; ++c) {
            const __int128 v = key_at(kb, c * stride);
            if (R.mode == 0 ? (v > bv) : (v < bv)) {
                bv = v;
                b = c;
            }
        }
        ibuf[R.cnt_off] = b;
    }
    for (int s = threadIdx.x; s < R.S; s += blockDim.x) {
        __int128 v = key_at(kb, 1 + s);
        for (int c = 1; c < R.n_cand; ++c) {
            const __int128 u = key_at(kb, c * stride + 1 + s);
            v = R.mode == 0 ? (u > v ? u : v) : (u < v ? u : v);
        }
        snull[s] = v;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < R.n_cand; c += blockDim.x) {
        const __int128 obs = key_at(kb, c * stride);
        int cnt = 0;
        for (int s = 0; s < R.S; ++s) cnt += snull[s] > obs ? 1 : 0;
        ibuf[R.cnt_off + 1 + c] = cnt;
        obuf[2 * (R.orig_off + c)] = kb[2 * c * stride];
        obuf[2 * (R.orig_off + c) + 1] = kb[2 * c * stride + 1];
    }
}

__global__ void check_finite_kernel(const float *x, long long n, int *flag)
{
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        if (!isfinite(x[t])) atomicOr(flag, 1);
}

template <int M, int KT, bool DX1>
const void *kptr()
{
    return reinterpret_cast<const void *>(&ksg_fused_kernel<M, KT, DX1>);
}

const void *select_kernel(const KsgVariant &v, bool dx1)
{
    if (dx1) {
        if (v.kt == 4) {
            if (v.m == 4) return kptr<4, 4, true>();
            if (v.m == 8) return kptr<8, 4, true>();
            if (v.m == 16) return kptr<16, 4, true>();
        } else if (v.kt == 0 && v.m == 2) {
            return kptr<2, 0, true>();
        }
    } else {
        if (v.kt == 4) {
            if (v.m == 2) return kptr<2, 4, false>();
            if (v.m == 4) return kptr<4, 4, false>();
        } else if (v.kt == 0 && v.m == 2) {
            return kptr<2, 0, false>();
        }
    }
    return nullptr;
}

}  // namespace

size_t ksg_smem_bytes(const KsgVariant &v, int dy, int dz, int dx, bool dx1, int jt)
{
    const size_t rows_t = (size_t)(dy + dz + v.m * dx);
    const size_t rows_q = (size_t)(dy + dz + (dx1 ? 0 : v.m * dx));
    return 4 * (rows_t * (size_t)jt + rows_q * QT);
}

cudaError_t ksg_prepare_attributes()
{
    const KsgVariant vs[] = {{4, 4, QT}, {8, 4, QT}, {16, 4, QT}, {2, 0, QT}, {2, 4, QT}};
    for (const auto &v : vs)
        for (int d = 0; d < 2; ++d) {
            const void *f = select_kernel(v, d == 0);
            if (!f) continue;
            cudaError_t e =
                cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            if (e != cudaSuccess) return e;
        }
    return cudaFuncSetAttribute(reinterpret_cast<const void *>(&stats_kernel),
                                cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t launch_ksg(const KsgLaunch &L, const KsgVariant &v, long long n_items, bool dx1,
                       size_t smem_bytes, cudaStream_t st)
{
    const void *f = select_kernel(v, dx1);
    if (!f) return cudaErrorInvalidValue;
    if (n_items <= 0) return cudaSuccess;
    if (n_items > 0x7fffffffLL) return cudaErrorInvalidValue;
    KsgLaunch arg = L;
    void *args[] = {&arg};
    return cudaLaunchKernel(f, dim3((unsigned)n_items), dim3(QT), args, smem_bytes, st);
}

cudaError_t launch_perms(int32_t *out, long long stride, int n, uint64_t seed, uint64_t target,
                         uint64_t stage, uint64_t iter, int s_first, int n_perm, cudaStream_t st)
{
    if (n_perm <= 0) return cudaSuccess;
    const size_t smem = (size_t)n * sizeof(int32_t);
    const int in_smem = smem <= 200 * 1024;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(&fisher_yates_kernel),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    fisher_yates_kernel<<<n_perm, 256, in_smem ? smem : 0, st>>>(out, stride, n, seed, target,
                                                                stage, iter, s_first, in_smem);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const unsigned long long *acc, long long *keys, int n_out,
                            cudaStream_t st)
{
    if (n_out <= 0) return cudaSuccess;
    finalize_kernel<<<(n_out + 255) / 256, 256, 0, st>>>(acc, keys, n_out);
    return cudaGetLastError();
}

cudaError_t launch_stats(const long long *keys, const StatReq *reqs, int n_req, int max_S,
                         int *ibuf, long long *obuf, cudaStream_t st)
{
    if (n_req <= 0) return cudaSuccess;
    const size_t smem = (size_t)(max_S > 0 ? max_S : 1) * sizeof(__int128);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    stats_kernel<<<n_req, 256, smem, st>>>(keys, reqs, ibuf, obuf);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const float *x, long long n, int *flag, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    long long blocks = (n + 255) / 256;
    if (blocks > 1216) blocks = 1216;
    check_finite_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, n, flag);
    return cudaGetLastError();
}

}  // namespace teksg
