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
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include <cstring>

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

// Compare-exchange: (a, b) <- (min, max).
__device__ __forceinline__ void cmpx(float &a, float &b)
{
    const float lo = fminf(a, b);
    b = fmaxf(a, b);
    a = lo;
}

// b (ascending, 4 values) <- the 4 smallest of b and the 8 values D, ascending,
// with multiplicity: each half of D is sorted by a 5-comparator network, and
// each sorted half is merged into b by taking min(b[i], h[3 - i]) (the 4
// smallest of the two lists, a bitonic sequence) and sorting that by a
// 4-comparator bitonic network.  Comparator networks permute their inputs, so
// the result is exactly the multiset's 4 smallest; when no D is below b[3] it
// returns b unchanged.  Branch-free: 44 min/max operations.
__device__ __forceinline__ void top4_merge8(float (&b)[4], const float (&D)[JC])
{
    float h[2][4];
#pragma unroll
    for (int g = 0; g < 2; ++g) {
#pragma unroll
        for (int i = 0; i < 4; ++i) h[g][i] = D[4 * g + i];
        cmpx(h[g][0], h[g][1]);
        cmpx(h[g][2], h[g][3]);
        cmpx(h[g][0], h[g][2]);
        cmpx(h[g][1], h[g][3]);
        cmpx(h[g][1], h[g][2]);
    }
#pragma unroll
    for (int g = 0; g < 2; ++g) {
#pragma unroll
        for (int i = 0; i < 4; ++i) b[i] = fminf(b[i], h[g][3 - i]);
        cmpx(b[0], b[2]);
        cmpx(b[1], b[3]);
        cmpx(b[0], b[1]);
        cmpx(b[2], b[3]);
    }
}

__device__ __forceinline__ void load8(const float *p, float (&v)[JC])
{
    const float4 a = *reinterpret_cast<const float4 *>(p);
    const float4 b = *reinterpret_cast<const float4 *>(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// M staged X values of one point (members are the fastest index of the tile).
template <int M>
__device__ __forceinline__ void load_members(const float *p, float (&v)[M])
{
    if (M % 4 == 0) {
#pragma unroll
        for (int a = 0; a < M; a += 4) {
            const float4 t = *reinterpret_cast<const float4 *>(p + a);
            v[a] = t.x; v[a + 1] = t.y; v[a + 2] = t.z; v[a + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int a = 0; a < M; a += 2) {
            const float2 t = *reinterpret_cast<const float2 *>(p + a);
            v[a] = t.x; v[a + 1] = t.y;
        }
    }
}

// Strict range counts of one pair for one member, counters in float (exact
// below 2^24): n_z += d_Z < e; n_xz += d_Z < e and d_X < e; n_yz += d_YZ < e.
// The compares run on the ALU pipe, the predicated adds on the FMA pipe.
__device__ __forceinline__ void count3(float &cz, float &cxz, float &cyz, float dz, float dyz,
                                       float dc, float e)
{
    asm("{\n\t.reg .pred pz, pxz, pyz;\n\t"
        "setp.lt.f32 pz, %3, %6;\n\t"
        "setp.lt.and.f32 pxz, %5, %6, pz;\n\t"
        "setp.lt.f32 pyz, %4, %6;\n\t"
        "@pz add.f32 %0, %0, 0f3F800000;\n\t"
        "@pxz add.f32 %1, %1, 0f3F800000;\n\t"
        "@pyz add.f32 %2, %2, 0f3F800000;\n\t}"
        : "+f"(cz), "+f"(cxz), "+f"(cyz)
        : "f"(dz), "f"(dyz), "f"(dc), "f"(e));
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

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <int M, int KT, bool DX1>
__global__ void __launch_bounds__(QT) ksg_fused_kernel(const KsgLaunch L)
{
    constexpr int KB = KT > 0 ? KT : KMAX;
    constexpr int NW = QT / 32;
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
    const int dyz = dy + dz;
    const int k = KT > 0 ? KT : G.k;
    const int jt = L.jt;
    const int cpt = jt >> 3;                  // chunks of 8 per tile
    const float *__restrict__ base = G.base;
    const bool sorted = G.sigma != nullptr;   // spatial order over (Y, Z), theiler == 0

    const int rows_t = dyz + M * dx;
    const int rows_q = dyz + (DX1 ? 0 : M * dx);
    float *tile = smem;                                    // [rows_t][jt]
    float *qv = smem + rows_t * jt;                        // [rows_q][QT]
    float2 *wlb = reinterpret_cast<float2 *>(qv + rows_q * QT);   // [NW][cpt] chunk bounds
    int *sidx = reinterpret_cast<int *>(wlb + NW * cpt);  // [jt] staged point indices
    float2 *scr = reinterpret_cast<float2 *>(sidx + jt) + threadIdx.x;  // [JC][QT] (d_Z, d_YZ)
    float *tx = tile + dyz * jt;   // X part of the tile: [jt][M] (DX1) or [M*dx][jt]
    __shared__ const int32_t *s_perm[M];
    __shared__ int s_xoff[M];
    __shared__ int s_out[M];
    __shared__ int s_valid[M];
    __shared__ int s_shared_perm;
    __shared__ float2 s_wbox[NW][32];
    __shared__ int s_live[2][NW];

    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int i = qtile * QT + tid;
    const bool qvalid = i < N;
    const int ic = qvalid ? i : N - 1;
    const int qlo = qtile * QT;
    const int qhi = min(qlo + QT, N) - 1;
    const int ti = sorted ? G.sigma[ic] : ic;   // time index of the query point

    if (tid < M) {
        const int mi = mb * M + tid;
        const int mc = mi < G.n_members ? mi : G.n_members - 1;
        const MemberDesc md = L.members[G.member_begin + mc];
        s_perm[tid] = md.perm;
        s_xoff[tid] = L.cols[md.xcol];
        s_out[tid] = md.out;
        s_valid[tid] = mi < G.n_members;
    }
    __syncthreads();
    if (tid == 0) {
        int same = 1;
        for (int m = 1; m < M; ++m) same &= (s_perm[m] == s_perm[0]);
        s_shared_perm = same;
    }

    auto yz_off = [&](int d) {
        return d < dy ? L.cols[G.ycol + d] : L.cols[G.zcol + d - dy];
    };

    // query-side values
    for (int d = 0; d < dyz; ++d)
        qv[d * QT + tid] = sorted ? G.yz[(size_t)d * N + ic] : base[yz_off(d) + ic];
    float xi[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int mi = min(mb * M + m, G.n_members - 1);
        const MemberDesc md = L.members[G.member_begin + mi];
        // member permutations of sorted groups are composed with the order:
        // they map a position straight to the time index of X
        const int pi = md.perm ? md.perm[ic] : ti;
        if (DX1) {
            xi[m] = base[L.cols[md.xcol] + pi];
        } else {
            xi[m] = 0.f;
            for (int d = 0; d < dx; ++d)
                qv[(dyz + m * dx + d) * QT + tid] = base[L.cols[md.xcol + d] + pi];
        }
    }
    // per-warp bounding box of the query points in (Y, Z)
    if (sorted) {
        for (int d = 0; d < dyz; ++d) {
            const float v = qv[d * QT + tid];
            const float mn = warp_min(v), mx = warp_max(v);
            if (lane == 0) s_wbox[warp][d] = make_float2(mn, mx);
        }
    }
    __syncthreads();
    const bool shared_perm = s_shared_perm != 0;
    const int32_t *perm0 = s_perm[0];

    auto stage = [&](int j0) {
        const bool use_idx = sorted || shared_perm;
        if (use_idx) {
            for (int jj = tid; jj < jt; jj += QT) {
                const int j = j0 + jj;
                int t = 0;
                if (j < N) t = (shared_perm && perm0) ? perm0[j] : (sorted ? G.sigma[j] : j);
                sidx[jj] = t;
            }
        }
        for (int r = 0; r < dyz; ++r) {
            const int off = sorted ? 0 : yz_off(r);
            const float *src = sorted ? G.yz + (size_t)r * N : base + off;
            for (int jj = tid; jj < jt; jj += QT) {
                const int j = j0 + jj;
                tile[r * jt + jj] = j < N ? src[j] : 0.f;
            }
        }
        if (use_idx) __syncthreads();
        if (DX1) {
            for (int e = tid; e < jt * M; e += QT) {
                const int jj = e / M, m = e - jj * M;
                const int j = j0 + jj;
                float v = 0.f;
                if (j < N) {
                    const int32_t *perm = shared_perm ? nullptr : s_perm[m];
                    const int t = perm ? perm[j] : (use_idx ? sidx[jj] : j);
                    v = base[s_xoff[m] + t];
                }
                tx[e] = v;
            }
        } else {
            for (int r = dyz; r < rows_t; ++r) {
                const int m = (r - dyz) / dx, d = (r - dyz) - m * dx;
                const int mi = min(mb * M + m, G.n_members - 1);
                const int off = L.cols[L.members[G.member_begin + mi].xcol + d];
                const int32_t *perm = shared_perm ? nullptr : s_perm[m];
                for (int jj = tid; jj < jt; jj += QT) {
                    const int j = j0 + jj;
                    float v = 0.f;
                    if (j < N) {
                        const int t = perm ? perm[j] : (use_idx ? sidx[jj] : j);
                        v = base[off + t];
                    }
                    tile[r * jt + jj] = v;
                }
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

    // Lower bounds on d_YZ and d_Z between this warp's query points and each
    // chunk of 8 points of the tile at j0 (sorted mode).  Exact float bounds:
    // rounding is monotone, so fl(z_j - z_i) >= fl(min_chunk - max_query).
    // Returns whether any chunk can still matter for this warp.
    auto chunk_bounds = [&](int j0, int jn, bool pass1, float bound) {
        const int nct = (jn + 7) >> 3;
        bool live = false;
        for (int c = lane; c < nct; c += 32) {
            const int gc = (j0 >> 3) + c;
            float lyz = 0.f, lz = 0.f;
            for (int d = 0; d < dyz; ++d) {
                const float2 b = G.box[(size_t)d * G.n_chunks8 + gc];
                const float2 q = s_wbox[warp][d];
                const float gap = fmaxf(fmaxf(__fsub_rn(b.x, q.y), __fsub_rn(q.x, b.y)), 0.f);
                lyz = fmaxf(lyz, gap);
                if (d >= dy) lz = fmaxf(lz, gap);
            }
            wlb[warp * cpt + c] = make_float2(lyz, lz);
            live |= pass1 ? (lyz < bound) : (lz < bound);
        }
        __syncwarp();
        return __any_sync(0xffffffffu, live);
    };

    const int ntiles = (N + jt - 1) / jt;

    // ---------------- pass 1: k nearest joint distances ----------------
    float buf[M][KB];
    float thr[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
#pragma unroll
        for (int a = 0; a < KB; ++a) buf[m][a] = CUDART_INF_F;
        thr[m] = CUDART_INF_F;
    }
    float tmax_w = CUDART_INF_F;   // max over the warp's lanes and members of thr
    unsigned int executed1 = 0, executed2 = 0;   // 8-point chunks this warp evaluated
    {
        // sorted mode: start at this CTA's own tile and spiral outwards
        const int home = sorted ? min(qlo / jt, ntiles - 1) : 0;
        int up = home + 1, down = home - 1;
        bool toggle = true;
        for (int s = 0; s < ntiles; ++s) {
            int t;
            if (s == 0) t = home;
            else if ((toggle && up < ntiles) || down < 0) t = up++;
            else t = down--;
            toggle = !toggle;
            const int j0 = t * jt;
            const int jn = min(jt, N - j0);
            if (sorted) {
                const bool live = chunk_bounds(j0, jn, true, tmax_w);
                if (lane == 0) s_live[s & 1][warp] = live;
            }
            __syncthreads();
            if (sorted) {
                int any = 0;
#pragma unroll
                for (int a = 0; a < NW; ++a) any |= s_live[s & 1][a];
                if (!any) continue;
            }
            stage(j0);
            __syncthreads();
            for (int c = 0; c < jn; c += JC) {
                if (sorted && wlb[warp * cpt + (c >> 3)].x >= tmax_w) continue;
                ++executed1;
                float dzv[JC], dyzv[JC];
                shared_dist(tile, qv, jt, dy, dz, c, dzv, dyzv);
                if (needs_mask(j0 + c)) apply_mask(j0 + c, dzv, dyzv);
                if (DX1) {
                    // members unrolled, the chunk's points in a loop: compact hot code
#pragma unroll
                    for (int u = 0; u < JC; ++u) scr[u * QT] = make_float2(dzv[u], dyzv[u]);
#pragma unroll 1
                    for (int u = 0; u < JC; ++u) {
                        const float dyzu = scr[u * QT].y;
                        float xv[M];
                        load_members<M>(tx + (c + u) * M, xv);
#pragma unroll
                        for (int m = 0; m < M; ++m) {
                            const float D = fmaxf(fabsf(__fsub_rn(xi[m], xv[m])), dyzu);
                            if (D < thr[m]) {
                                topk_insert<KB>(buf[m], D);
                                thr[m] = KT > 0 ? buf[m][KB - 1] : topk_at<KB>(buf[m], k - 1);
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        float dcv[JC];
                        member_dist<M>(tile, qv, jt, dy, dz, dx, m, c, dcv);
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
            if (sorted) {
                float tm = thr[0];
#pragma unroll
                for (int m = 1; m < M; ++m) tm = fmaxf(tm, thr[m]);
                tmax_w = warp_max(tm);
            }
            __syncthreads();
        }
    }

    // ---------------- pass 2: strict range counts ----------------
    float eps[M];
    float cxz[M], cyz[M], cz[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        eps[m] = thr[m];
        cxz[m] = cyz[m] = cz[m] = 0.f;
    }
    const bool prune2 = sorted && dz > 0;   // with empty Z every j counts in n_xz
    float emax_w = CUDART_INF_F;
    if (prune2) {
        float em = eps[0];
#pragma unroll
        for (int m = 1; m < M; ++m) em = fmaxf(em, eps[m]);
        emax_w = warp_max(em);
    }
    for (int t = 0; t < ntiles; ++t) {
        const int j0 = t * jt;
        const int jn = min(jt, N - j0);
        if (prune2) {
            const bool live = chunk_bounds(j0, jn, false, emax_w);
            if (lane == 0) s_live[t & 1][warp] = live;
        }
        __syncthreads();
        if (prune2) {
            int any = 0;
#pragma unroll
            for (int a = 0; a < NW; ++a) any |= s_live[t & 1][a];
            if (!any) continue;
        }
        stage(j0);
        __syncthreads();
        for (int c = 0; c < jn; c += JC) {
            if (prune2 && wlb[warp * cpt + (c >> 3)].y >= emax_w) continue;
            ++executed2;
            float dzv[JC], dyzv[JC];
            shared_dist(tile, qv, jt, dy, dz, c, dzv, dyzv);
            if (needs_mask(j0 + c)) apply_mask(j0 + c, dzv, dyzv);
            // d_Z is -inf for valid pairs when Z is empty and +inf for masked
            // pairs, so n_z also counts exactly the valid j in that case
            if (DX1) {
#pragma unroll
                for (int u = 0; u < JC; ++u) scr[u * QT] = make_float2(dzv[u], dyzv[u]);
#pragma unroll 1
                for (int u = 0; u < JC; ++u) {
                    const float2 sd = scr[u * QT];
                    float xv[M];
                    load_members<M>(tx + (c + u) * M, xv);
#pragma unroll
                    for (int m = 0; m < M; ++m)
                        count3(cz[m], cxz[m], cyz[m], sd.x, sd.y,
                               fabsf(__fsub_rn(xi[m], xv[m])), eps[m]);
                }
            } else {
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    float dcv[JC];
                    member_dist<M>(tile, qv, jt, dy, dz, dx, m, c, dcv);
#pragma unroll
                    for (int u = 0; u < JC; ++u)
                        count3(cz[m], cxz[m], cyz[m], dzv[u], dyzv[u], dcv[u], eps[m]);
                }
            }
        }
        __syncthreads();
    }

    if (L.work) {
        const unsigned lanes = __popc(__ballot_sync(0xffffffffu, qvalid));
        if (lane == 0) {
            int mv = 0;
#pragma unroll
            for (int m = 0; m < M; ++m) mv += s_valid[m];
            const unsigned long long per = (unsigned long long)JC * lanes * (unsigned)mv;
            // evaluations, and algorithmic ops: 3 per kNN-pass and 7 per count-pass pair
            atomicAdd(&L.work[0], (unsigned long long)(executed1 + executed2) * per);
            atomicAdd(&L.work[1], (3ull * executed1 + 7ull * executed2) * per);
        }
    }

    // ---------------- digamma key: exact int64 terms, 128-bit sums ----------------
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const int nz = (int)cz[m], nxz = (int)cxz[m], nyz = (int)cyz[m];
        long long term = 0;
        if (qvalid) term = L.q[nz + 1] - L.q[nxz + 1] - L.q[nyz + 1];
        if (L.dbg_eps && qvalid && s_valid[m] && s_out[m] == L.dbg_out) {
            L.dbg_eps[ti] = eps[m];
            L.dbg_nxz[ti] = nxz;
            L.dbg_nyz[ti] = nyz;
            L.dbg_nz[ti] = nz;
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

// Number of u with |fl(col[u] - x)| < e over an ascending column: fl(col[u]-x)
// is non-decreasing in u (rounding is monotone), so the set is a contiguous
// run found by two binary searches with exactly the pairwise predicate.
__device__ __forceinline__ int range_count(const float *__restrict__ col, int n, float x, float e)
{
    int lo = 0, hi = n;   // first u with fl(col[u] - x) >= e
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__fsub_rn(__ldg(col + mid), x) >= e) hi = mid;
        else lo = mid + 1;
    }
    const int a = lo;
    lo = 0;
    hi = n;               // first u with fl(col[u] - x) > -e
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (__fsub_rn(__ldg(col + mid), x) > -e) hi = mid;
        else lo = mid + 1;
    }
    return a - lo;
}


// ---------------- member-lane kernel ----------------
// ksg_lane_kernel -- for single-variable X (every candidate of the greedy
// steps).  Lanes are members: a CTA owns 32 members (one per lane) and 32
// query points, 4 per warp.  Every prune decision is taken per query point
// (a warp-uniform branch), against the maximum over the 32 members of that
// point's current k-th distance (pass 1) or eps (pass 2), so the bounds are
// as tight as a single point allows.  d_Z and d_YZ of a chunk are computed
// lane-parallel over (query, point) pairs and read back as broadcasts; the X
// values of a lane's member come from a [member][point] tile in shared memory.
// With TMA = true that tile is copied by the tensor memory accelerator from the
// launch's X-value rows (one 2-D box of 32 points x all CTA members per live
// 32-point segment, 128-byte swizzled); otherwise the threads gather it
// through the members' permutations.
constexpr int LQ = 4;            // query points per warp
constexpr int LW = 8;            // warps per CTA
constexpr int LQC = LQ * LW;     // query points per CTA
constexpr unsigned kTileSpinLimit = 1u << 24;   // bounded waits on a tile copy

__device__ __forceinline__ uint32_t lane_smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// bounded wait for the phase of parity `parity` of the mbarrier at `addr`
__device__ __forceinline__ bool tile_wait(uint32_t addr, uint32_t parity)
{
    for (unsigned it = 0; it < kTileSpinLimit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// One work item of the member-lane kernel: query tile x member block `item`
// of the launch (the CTA's whole job in an ordinary grid; one of many in a
// persistent one).
template <int KT, int MS, bool TMA>
__device__ __forceinline__ void ksg_lane_item(const KsgLaunch &L, const CUtensorMap &tmx,
                                              const long long item)
{
    constexpr int KB = KT > 0 ? KT : KMAX;
    constexpr int MB = 32 * MS;   // members per CTA: MS per lane
    extern __shared__ __align__(16) float smem[];

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
    const int N = G.N, dy = G.dy, dz = G.dz, w = G.theiler;
    const int dyz = dy + dz;
    const int k = KT > 0 ? KT : G.k;
    const int jt = L.jt, jtp = jt + 4, cpt = jt >> 3, wpt = cpt >> 3;
    const float *__restrict__ base = G.base;
    const bool sorted = G.sigma != nullptr;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *t_yz, *t_x, *s_dz;
    if constexpr (TMA) {
        // [jt / 32][MB][32] X tile on a 1024-byte boundary (the swizzle atom)
        const uint32_t pad = (1024u - (lane_smem_u32(smem) & 1023u)) & 1023u;
        t_x = smem + pad / 4;
        t_yz = t_x + MB * jt;                             // [dyz][jt]
        s_dz = t_yz + dyz * jt;                           // [LW][LQ][8]
    } else {
        t_yz = smem;                                      // [dyz][jt]
        t_x = t_yz + dyz * jt;                            // [MB][jtp]
        s_dz = t_x + MB * jtp;                            // [LW][LQ][8]
    }
    float *s_dyz = s_dz + LW * LQ * 8;                    // [LW][LQ][8]
    float *s_q = s_dyz + LW * LQ * 8;                     // [LW][LQ][dyz]
    unsigned *s_bits = reinterpret_cast<unsigned *>(s_q + LW * LQ * dyz);  // [LW][wpt]
    __shared__ const int32_t *s_mperm[MB];
    __shared__ int s_mxoff[MB];
    __shared__ int s_shared_perm;
    __shared__ int s_live[2][LW];
    __shared__ float s_bound[LW][LQ];
    __shared__ long long s_red[LW][MB];
    __shared__ float2 s_cqbox[32];
    // per pass, the lower bound from the CTA's query box to every tile box
    // (pass 1 over (Y, Z), pass 2 over Z): tile t is skipped when it reaches
    // the CTA's largest bound
    __shared__ float s_tlb[2][kMaxOrderN / 256];
    // pass 1 visits the tiles in increasing order of that bound (the home
    // tile first), so that the thresholds fall early
    __shared__ unsigned char s_tord[kMaxOrderN / 256];
    __shared__ __align__(8) unsigned long long s_tbar;   // tile-copy mbarrier (TMA)
    const uint32_t tbar = lane_smem_u32(&s_tbar);
    uint32_t tphase = 0;
    if constexpr (TMA) {
        if (tid == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tbar));
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmx))
                         : "memory");
        }
    }

    // ---- this lane's members: mb * MB + lane + 32 q ----
    bool mvalid[MS];
    MemberDesc md[MS];
#pragma unroll
    for (int q = 0; q < MS; ++q) {
        const int mi = mb * MB + lane + 32 * q;
        mvalid[q] = mi < G.n_members;
        md[q] = L.members[G.member_begin + min(mi, G.n_members - 1)];
    }
    if (!TMA && warp == 0) {
        const unsigned long long p0 =
            __shfl_sync(0xffffffffu, (unsigned long long)(uintptr_t)md[0].perm, 0);
        int same = 1;
#pragma unroll
        for (int q = 0; q < MS; ++q) {
            s_mperm[lane + 32 * q] = md[q].perm;
            s_mxoff[lane + 32 * q] = L.cols[md[q].xcol];
            same &= __all_sync(0xffffffffu, (unsigned long long)(uintptr_t)md[q].perm == p0);
        }
        if (lane == 0) s_shared_perm = same;
    }

    auto yz_off = [&](int d) {
        return d < dy ? L.cols[G.ycol + d] : L.cols[G.zcol + d - dy];
    };
    // The warp's LQ query points are positions qbase + LW a of the CTA's LQC
    // consecutive ones (interleaved, not adjacent): neighbouring points have
    // similar neighbourhoods, so interleaving evens out the warps' work per
    // tile, which the per-tile barrier otherwise pays at the slowest warp.
    const int qbase = qtile * LQC + warp;
    auto qpos = [&](int a) { return qbase + LW * a; };

    // ---- the warp's query points ----
    float xi[LQ][MS];
#pragma unroll
    for (int a = 0; a < LQ; ++a) {
        const int qc = min(qpos(a), N - 1);
#pragma unroll
        for (int q = 0; q < MS; ++q) {
            if constexpr (TMA) {
                const int row = G.member_begin + min(mb * MB + lane + 32 * q, G.n_members - 1);
                xi[a][q] = L.xval[(size_t)row * L.xpitch + qc];
            } else {
                const int32_t *pm = md[q].perm;
                xi[a][q] = base[L.cols[md[q].xcol] + (pm ? pm[qc] : (sorted ? G.sigma[qc] : qc))];
            }
        }
    }
    for (int e = lane; e < LQ * dyz; e += 32) {
        const int a = e / dyz, d = e - a * dyz;
        const int qc = min(qpos(a), N - 1);
        s_q[(warp * LQ + a) * dyz + d] = sorted ? G.yz[(size_t)d * N + qc] : base[yz_off(d) + qc];
    }
    if (lane < LQ) s_bound[warp][lane] = CUDART_INF_F;
    __syncthreads();
    // Coarse test, taken identically by every thread without a barrier: it
    // reads the tile bounds (written before the barrier below) and `bound`, a
    // register snapshot of the CTA's largest per-query bound taken right
    // after a barrier.
    const bool coarse = sorted && jt == 256 && G.tbox != nullptr;
    // bounding box of the CTA's 32 query points, then its lower bound to every
    // tile box for both passes (one warp; N <= kMaxOrderN on this path)
    if (coarse && warp == 0) {
        for (int d = 0; d < dyz; ++d) {
            const float v = s_q[lane * dyz + d];   // query lane of the CTA (warp lane/4, a lane%4)
            const float mn = warp_min(v), mx = warp_max(v);
            if (lane == 0) s_cqbox[d] = make_float2(mn, mx);
        }
        __syncwarp();
        for (int t = lane; t < G.n_tiles256; t += 32) {
            float lb1 = 0.f, lb2 = 0.f;
            for (int d = 0; d < dyz; ++d) {
                const float2 b = G.tbox[(size_t)d * G.n_tiles256 + t];
                const float2 q = s_cqbox[d];
                const float l = fmaxf(fmaxf(__fsub_rn(b.x, q.y), __fsub_rn(q.x, b.y)), 0.f);
                lb1 = fmaxf(lb1, l);
                if (d >= dy) lb2 = fmaxf(lb2, l);
            }
            s_tlb[0][t] = lb1;
            s_tlb[1][t] = lb2;
        }
        __syncwarp();
        const int home = min((qtile * LQC) / jt, G.n_tiles256 - 1);
        for (int t = lane; t < G.n_tiles256; t += 32) {
            const float kt = t == home ? -1.f : s_tlb[0][t];
            int r = 0;
            for (int u = 0; u < G.n_tiles256; ++u) {
                const float ku = u == home ? -1.f : s_tlb[0][u];
                r += ku < kt || (ku == kt && u < t);
            }
            s_tord[r] = (unsigned char)t;
        }
    }
    __syncthreads();
    static_assert(LW * LQ == 32, "one bound per lane");
    auto snapshot = [&]() { return warp_max((&s_bound[0][0])[lane]); };
    auto tile_dead = [&](int t, bool pass1, float bound) {
        return coarse && s_tlb[pass1 ? 0 : 1][t] >= bound;
    };
    const bool shared_perm = s_shared_perm != 0;
    const int32_t *perm0 = s_mperm[0];

    // CTA-wide mask of the tile's chunks that are live for some warp, built
    // by every warp from all warps' bits (identical in every warp; called
    // between the liveness barrier and the staging barrier)
    auto cta_mask = [&](int jn) {
        const int nct = (jn + 7) >> 3;
        unsigned any = 0;
        if (lane < nct)
            for (int b = 0; b < LW; ++b)
                any |= (s_bits[b * wpt + (lane >> 3)] >> (4 * (lane & 7))) & 0xFu;
        return __ballot_sync(0xffffffffu, any != 0);
    };

    // this warp's live chunks of the tile (any of its query points), a subset
    // of the CTA mask: the chunk loop visits only these
    auto warp_mask = [&](int jn) {
        const int nct = (jn + 7) >> 3;
        unsigned any = 0;
        if (lane < nct) any = (s_bits[warp * wpt + (lane >> 3)] >> (4 * (lane & 7))) & 0xFu;
        return __ballot_sync(0xffffffffu, any != 0);
    };

    // stage the live chunks: thread = (member m, point u) for X, (dim, point)
    // for Y and Z; four chunks per round keep several gathers in flight
    auto stage = [&](int j0, unsigned mask) {
        const int m0 = tid >> 3, u = tid & 7;
        unsigned rest = mask;
        while (rest) {
            float xv4[4][MS], yz4[4];
            int cc[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                cc[q] = -1;
                if (rest) {
                    cc[q] = __ffs(rest) - 1;
                    rest &= rest - 1;
                }
                yz4[q] = 0.f;
#pragma unroll
                for (int r = 0; r < MS; ++r) xv4[q][r] = 0.f;
                if (cc[q] >= 0) {
                    const int j = j0 + cc[q] * 8 + u;
                    if (j < N) {
                        const int tj = sorted ? G.sigma[j] : j;
#pragma unroll
                        for (int r = 0; r < MS; ++r) {
                            const int m = m0 + 32 * r;
                            const int32_t *pm = shared_perm ? perm0 : s_mperm[m];
                            xv4[q][r] = base[s_mxoff[m] + (pm ? pm[j] : tj)];
                        }
                        if (tid < dyz * 8) {
                            const int d = tid >> 3;
                            yz4[q] = sorted ? G.yz[(size_t)d * N + j] : base[yz_off(d) + j];
                        }
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (cc[q] < 0) continue;
#pragma unroll
                for (int r = 0; r < MS; ++r) t_x[(m0 + 32 * r) * jtp + cc[q] * 8 + u] = xv4[q][r];
                if (tid < dyz * 8) t_yz[(tid >> 3) * jt + cc[q] * 8 + u] = yz4[q];
            }
        }
    };

    // Stage the tile's live chunks and make them visible to every thread; false
    // (identical in every thread) when a tile copy did not complete in time, in
    // which case the error flag is set and the caller returns.
    auto stage_all = [&](int j0, int jn, unsigned mask) {
        if constexpr (TMA) {
            if (tid == 0) {
                const int nseg = jt >> 5;
                unsigned segs = 0;
                for (int sg = 0; sg < nseg; ++sg)
                    if ((mask >> (4 * sg)) & 0xFu) segs |= 1u << sg;
                const uint32_t bytes = (uint32_t)__popc(segs) * (uint32_t)(MB * 128);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                             ::"r"(tbar), "r"(bytes) : "memory");
                const int row0 = G.member_begin + mb * MB;
                const uint32_t dst0 = lane_smem_u32(t_x);
                while (segs) {
                    const int sg = __ffs(segs) - 1;
                    segs &= segs - 1;
                    asm volatile(
                        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx"
                        "::bytes [%0], [%1, {%2, %3}], [%4];"
                        ::"r"(dst0 + (uint32_t)(sg * MB * 128)),
                          "l"(reinterpret_cast<uint64_t>(&tmx)), "r"(j0 + 32 * sg), "r"(row0),
                          "r"(tbar)
                        : "memory");
                }
            }
            // Y and Z of the whole tile, coalesced (jt <= blockDim); four
            // dimensions' loads are issued before their stores, so that they
            // are in flight together rather than one round trip each
            if (tid < jn)
                for (int d0 = 0; d0 < dyz; d0 += 4) {
                    float v[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (d0 + e < dyz)
                            v[e] = sorted ? G.yz[(size_t)(d0 + e) * N + j0 + tid]
                                          : base[yz_off(d0 + e) + j0 + tid];
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (d0 + e < dyz) t_yz[(d0 + e) * jt + tid] = v[e];
                }
            const bool ok = tile_wait(tbar, tphase);
            tphase ^= 1u;
            if (__syncthreads_or(!ok)) {
                if (tid == 0) {
                    atomicExch(&L.work[2], 1ull);
                    tile_wait(tbar, tphase ^ 1u);   // let copies still in flight land
                }
                return false;
            }
            return true;
        } else {
            stage(j0, mask);
            __syncthreads();
            return true;
        }
    };

    // X values of member slot q (member lane + 32 q) at the 8 points of chunk c
    auto load_x = [&](int c, int q, float (&v)[JC]) {
        if constexpr (TMA) {
            const float *row = t_x + ((c >> 5) * MB + lane + 32 * q) * 32;
            const int k0 = (c & 31) >> 2, sw = lane & 7;
            const float4 lo = *reinterpret_cast<const float4 *>(row + ((k0 ^ sw) << 2));
            const float4 hi = *reinterpret_cast<const float4 *>(row + (((k0 + 1) ^ sw) << 2));
            v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w;
            v[4] = hi.x; v[5] = hi.y; v[6] = hi.z; v[7] = hi.w;
        } else {
            load8(t_x + (lane + 32 * q) * jtp + c, v);
        }
    };

    // liveness of every (query, chunk) of the tile for this warp: bit 4c'+a of
    // word c/8; a lower bound (exact in float, rounding is monotone) on d_YZ
    // (pass 1) or d_Z (pass 2) below the query's bound keeps the chunk
    // (The box loads of all of a tile's rounds of 8 chunks are issued
    // together, dimension by dimension, so that a tile costs one chain of
    // dependent loads per dimension rather than one per round.)
    static_assert(256 / 64 == 4, "at most 4 rounds of 8 chunks per tile (jt <= 256)");
    auto tile_live = [&](int j0, int jn, bool pass1) {
        const int nct = (jn + 7) >> 3;
        const int a = lane & 3;
        float lb[4] = {0.f, 0.f, 0.f, 0.f};
        if (sorted) {
            const float *qc = s_q + (warp * LQ + a) * dyz;
            const int gc0 = (j0 >> 3) + (lane >> 2), gmax = G.n_chunks8 - 1;
#pragma unroll 2
            for (int d = pass1 ? 0 : dy; d < dyz; ++d) {
                const float q = qc[d];
                const float2 *bd = G.box + (size_t)d * G.n_chunks8;
#pragma unroll
                for (int wb = 0; wb < 4; ++wb) {
                    if (wb < wpt) {
                        // past the group's last chunk: a valid address, result unused
                        const float2 b = __ldg(&bd[min(gc0 + 8 * wb, gmax)]);
                        lb[wb] = fmaxf(lb[wb],
                                       fmaxf(fmaxf(__fsub_rn(b.x, q), __fsub_rn(q, b.y)), 0.f));
                    }
                }
            }
        }
        const float bnd = s_bound[warp][a];
        bool any = false;
#pragma unroll
        for (int wb = 0; wb < 4; ++wb) {
            if (wb < wpt) {
                const bool live = wb * 8 + (lane >> 2) < nct && (!sorted || lb[wb] < bnd);
                const unsigned word = __ballot_sync(0xffffffffu, live);
                if (lane == 0) s_bits[warp * wpt + wb] = word;
                any |= word != 0;
            }
        }
        __syncwarp();
        return any;
    };

    // d_Z and d_YZ of the live queries against the 8 points of the chunk at c;
    // lane = (query a, point u); masked pairs (past N, self, Theiler band) = +inf.
    // Returns a byte per query (byte a nonzero: query a stays live): live4
    // without the queries whose 8 points all lie at or beyond the query's bound
    // in the pass's shared subspace (d_YZ in pass 1, d_Z in pass 2); with the
    // bound >= every member's threshold or eps, no member can insert or count
    // one of them.
    // this lane's (query, point) of the distance step: query a = lane / 8 at
    // position qp_lane (clamped to the data), point u = lane % 8 of the chunk
    const int qp_lane = min(qpos(lane >> 3), N - 1);
    auto chunk_dist = [&](int j0, int c, unsigned live4, bool pass1) {
        const int a = lane >> 3, u = lane & 7;
        float dzv = -CUDART_INF_F, dyzv = -CUDART_INF_F;
        bool keep = false;
        if ((live4 >> a) & 1u) {
            const float *qc = s_q + (warp * LQ + a) * dyz;
            const float *tp = t_yz + c + u;
            // two independent running maxima (max is exact in any order), so
            // that the dimensions do not form one chain of dependent operations
            float m1 = -CUDART_INF_F;
            int d = dy;
#pragma unroll 2
            for (; d + 1 < dyz; d += 2) {
                dzv = fmaxf(dzv, fabsf(__fsub_rn(qc[d], tp[d * jt])));
                m1 = fmaxf(m1, fabsf(__fsub_rn(qc[d + 1], tp[(d + 1) * jt])));
            }
            if (d < dyz) dzv = fmaxf(dzv, fabsf(__fsub_rn(qc[d], tp[d * jt])));
            dzv = fmaxf(dzv, m1);
            if (dy == 1) {
                dyzv = fmaxf(dzv, fabsf(__fsub_rn(qc[0], tp[0])));
            } else {
                dyzv = dzv;
#pragma unroll 2
                for (int d = 0; d < dy; ++d)
                    dyzv = fmaxf(dyzv, fabsf(__fsub_rn(qc[d], tp[d * jt])));
            }
            const int j = j0 + c + u;
            const int gap = abs(j - qp_lane);
            if (j >= N || gap <= w) {
                dzv = CUDART_INF_F;
                dyzv = CUDART_INF_F;
            }
            keep = (pass1 ? dyzv : dzv) < s_bound[warp][a];
        }
        // the ballot also orders these stores after every lane's reads of the
        // previous chunk's distances
        const unsigned kb = __ballot_sync(0xffffffffu, keep);
        if (!pass1) s_dz[(warp * LQ + a) * 8 + u] = dzv;   // pass 1 reads d_YZ only
        s_dyz[(warp * LQ + a) * 8 + u] = dyzv;
        __syncwarp();
        return kb;
    };

    const int ntiles = (N + jt - 1) / jt;
    unsigned executed1 = 0, executed2 = 0;
    // s_live is double-buffered by the count of liveness checks taken (not by
    // tile): two checks that use the same buffer always have the barrier of the
    // check between them in between, also when tiles are skipped without one
    int nchk = 0;

    // ---------------- pass 1: k nearest joint distances ----------------
    float buf[LQ][MS][KB];
    float thr[LQ][MS];
#pragma unroll
    for (int a = 0; a < LQ; ++a)
#pragma unroll
        for (int q = 0; q < MS; ++q) {
#pragma unroll
            for (int b = 0; b < KB; ++b) buf[a][q][b] = CUDART_INF_F;
            thr[a][q] = CUDART_INF_F;
        }
    float cbound = CUDART_INF_F;   // snapshot of the CTA's largest bound
    {
        const int home = sorted ? min((qtile * LQC) / jt, ntiles - 1) : 0;
        int up = home + 1, down = home - 1;
        bool toggle = true;
        for (int s = 0; s < ntiles; ++s) {
            int t;
            if (coarse) t = s_tord[s];
            else if (s == 0) t = home;
            else if ((toggle && up < ntiles) || down < 0) t = up++;
            else t = down--;
            toggle = !toggle;
            const int j0 = t * jt;
            const int jn = min(jt, N - j0);
            // in bound order, every later tile is as far and the bound only falls
            if (tile_dead(t, true, cbound)) {
                if (coarse) break;
                continue;
            }
            const bool live = tile_live(j0, jn, true);
            const int buf_i = nchk++ & 1;
            if (lane == 0) s_live[buf_i][warp] = live;
            // Barrier: every warp has finished the previous tile (its compute and
            // its bound updates) before anyone stages or snapshots.
            __syncthreads();
            if (sorted) cbound = snapshot();
            int any = 0;
#pragma unroll
            for (int b = 0; b < LW; ++b) any |= s_live[buf_i][b];
            if (!any) continue;
            const unsigned mask = cta_mask(jn);
            if (!stage_all(j0, jn, mask)) return;
            // The home tile starts with every threshold at +inf: its chunks are
            // visited from the CTA's own positions on (nearest first), so that
            // the thresholds fall early and fewer points are inserted.
            const bool home_tile = s == 0 && sorted;
            const int rot = home_tile ? (((qtile * LQC) - j0) >> 3) & 31 : 0;
            unsigned rest = mask & warp_mask(jn);
            if (rot) rest = (rest >> rot) | (rest << (32 - rot));
            while (rest) {
                const int c = ((__ffs(rest) - 1 + rot) & 31) * JC;
                rest &= rest - 1;
                const unsigned live4 = (s_bits[warp * wpt + (c >> 6)] >> (4 * ((c >> 3) & 7))) & 0xFu;
                if (!live4) continue;
                const unsigned kb = chunk_dist(j0, c, live4, true);
                if (!kb) continue;
                float xv[MS][JC];
#pragma unroll
                for (int q = 0; q < MS; ++q) load_x(c, q, xv[q]);
#pragma unroll
                for (int a = 0; a < LQ; ++a) {
                    if (!((kb >> (8 * a)) & 0xFFu)) continue;
                    ++executed1;
                    float dv[JC];
                    load8(s_dyz + (warp * LQ + a) * 8, dv);
#pragma unroll
                    for (int q = 0; q < MS; ++q) {
                        float D[JC];
#pragma unroll
                        for (int u = 0; u < JC; ++u)
                            D[u] = fmaxf(fabsf(__fsub_rn(xi[a][q], xv[q][u])), dv[u]);
                        // one test for the 8 points; the insertions are the rare path
                        const float mn = fminf(fminf(fminf(D[0], D[1]), fminf(D[2], D[3])),
                                               fminf(fminf(D[4], D[5]), fminf(D[6], D[7])));
                        if constexpr (KT == 4) {
                            // Some lane of the warp has a point below its threshold
                            // on about 70% of the chunks (32 members per warp), so
                            // the whole chunk is merged without branches by every
                            // lane (a no-op for lanes without one).
                            if (__any_sync(0xffffffffu, mn < thr[a][q])) {
                                top4_merge8(buf[a][q], D);
                                thr[a][q] = buf[a][q][3];
                            }
                        } else if (mn < thr[a][q]) {
#pragma unroll
                            for (int u = 0; u < JC; ++u) {
                                if (D[u] < thr[a][q]) {
                                    topk_insert<KB>(buf[a][q], D[u]);
                                    thr[a][q] = KT > 0 ? buf[a][q][KB - 1]
                                                       : topk_at<KB>(buf[a][q], k - 1);
                                }
                            }
                        }
                    }
                }
                __syncwarp();
            }
            if (sorted) {
#pragma unroll
                for (int a = 0; a < LQ; ++a) {
                    float tl = thr[a][0];
#pragma unroll
                    for (int q = 1; q < MS; ++q) tl = fmaxf(tl, thr[a][q]);
                    const float tm = warp_max(tl);
                    if (lane == 0) s_bound[warp][a] = tm;
                }
                __syncwarp();
            }
        }
    }

    // Warps leave pass 1 at different times (coarse skips take no barrier);
    // none may overwrite s_bound with pass-2 values while another still reads
    // it for a pass-1 coarse test.
    __syncthreads();

    // ---------------- pass 2: strict range counts ----------------
    float eps[LQ][MS], cz[LQ][MS], cxz[LQ][MS], cyz[LQ][MS];
#pragma unroll
    for (int a = 0; a < LQ; ++a)
#pragma unroll
        for (int q = 0; q < MS; ++q) {
            eps[a][q] = thr[a][q];
            cz[a][q] = cxz[a][q] = cyz[a][q] = 0.f;
        }
    const bool prune2 = sorted && dz > 0;   // with empty Z every j counts in n_xz
#pragma unroll
    for (int a = 0; a < LQ; ++a) {
        float el = eps[a][0];
#pragma unroll
        for (int q = 1; q < MS; ++q) el = fmaxf(el, eps[a][q]);
        const float em = warp_max(el);
        if (lane == 0) s_bound[warp][a] = prune2 ? em : CUDART_INF_F;
    }
    __syncthreads();   // every warp's pass-2 bounds before the snapshot
    cbound = snapshot();
    // Empty Z with one X and one Y variable and no Theiler window: n_z = N - 1
    // and n_xz, n_yz are 1-D range counts.  The member's X values over the
    // points are the column's values (a permutation only reorders them), so
    // both counts come from sorted columns, minus the point itself (distance 0
    // counts iff eps > 0).  Exactly the counts of the pairwise loop below.
    if (G.ysorted) {
#pragma unroll
        for (int a = 0; a < LQ; ++a)
#pragma unroll
            for (int q = 0; q < MS; ++q) {
                const float e = eps[a][q];
                const int self = e > 0.f ? 1 : 0;
                cz[a][q] = (float)(N - 1);
                cxz[a][q] = (float)(range_count(md[q].xsorted, N, xi[a][q], e) - self);
                cyz[a][q] =
                    (float)(range_count(G.ysorted, N, s_q[(warp * LQ + a) * dyz], e) - self);
            }
    }
    for (int t = 0; t < (G.ysorted ? 0 : ntiles); ++t) {
        const int j0 = t * jt;
        const int jn = min(jt, N - j0);
        bool live = true;
        if (prune2 && tile_dead(t, false, cbound)) continue;
        if (prune2) {
            live = tile_live(j0, jn, false);
        }
        else {
            // no pruning: every chunk below the end of the data is live
            const int nct = (jn + 7) >> 3;
            for (int wb = lane; wb < wpt; wb += 32) {
                const int lo = wb * 8;
                const int n = nct - lo >= 8 ? 8 : (nct - lo > 0 ? nct - lo : 0);
                s_bits[warp * wpt + wb] = n >= 8 ? 0xffffffffu : ((1u << (4 * n)) - 1u);
            }
            __syncwarp();
        }
        const int buf_i = nchk++ & 1;
        if (lane == 0) s_live[buf_i][warp] = live;
        __syncthreads();
        int any = 0;
#pragma unroll
        for (int b = 0; b < LW; ++b) any |= s_live[buf_i][b];
        if (!any) continue;
        const unsigned mask = cta_mask(jn);
        if (!stage_all(j0, jn, mask)) return;
        unsigned rest = mask & warp_mask(jn);
        while (rest) {
            const int c = (__ffs(rest) - 1) * JC;
            rest &= rest - 1;
            const unsigned live4 = (s_bits[warp * wpt + (c >> 6)] >> (4 * ((c >> 3) & 7))) & 0xFu;
            if (!live4) continue;
            const unsigned kb = chunk_dist(j0, c, live4, false);
            if (!kb) continue;
            float xv[MS][JC];
#pragma unroll
            for (int q = 0; q < MS; ++q) load_x(c, q, xv[q]);
#pragma unroll
            for (int a = 0; a < LQ; ++a) {
                if (!((kb >> (8 * a)) & 0xFFu)) continue;
                ++executed2;
                float zv[JC], yv[JC];
                load8(s_dz + (warp * LQ + a) * 8, zv);
                load8(s_dyz + (warp * LQ + a) * 8, yv);
#pragma unroll
                for (int q = 0; q < MS; ++q)
#pragma unroll
                    for (int u = 0; u < JC; ++u)
                        count3(cz[a][q], cxz[a][q], cyz[a][q], zv[u], yv[u],
                               fabsf(__fsub_rn(xi[a][q], xv[q][u])), eps[a][q]);
            }
            __syncwarp();
        }
    }

    // ---------------- work counters, digamma key ----------------
    if (L.work) {
        unsigned mv = 0;
#pragma unroll
        for (int q = 0; q < MS; ++q) mv += __popc(__ballot_sync(0xffffffffu, mvalid[q]));
        if (lane == 0) {
            const unsigned long long per = (unsigned long long)JC * mv;
            atomicAdd(&L.work[0], (unsigned long long)(executed1 + executed2) * per);
            atomicAdd(&L.work[1], (3ull * executed1 + 7ull * executed2) * per);
        }
    }
#pragma unroll
    for (int q = 0; q < MS; ++q) {
        long long term = 0;
#pragma unroll
        for (int a = 0; a < LQ; ++a) {
            const int nz = (int)cz[a][q], nxz = (int)cxz[a][q], nyz = (int)cyz[a][q];
            if (qpos(a) < N) {
                term += L.q[nz + 1] - L.q[nxz + 1] - L.q[nyz + 1];
                if (L.dbg_eps && mvalid[q] && md[q].out == L.dbg_out) {
                    const int tq = sorted ? G.sigma[qpos(a)] : qpos(a);
                    L.dbg_eps[tq] = eps[a][q];
                    L.dbg_nxz[tq] = nxz;
                    L.dbg_nyz[tq] = nyz;
                    L.dbg_nz[tq] = nz;
                }
            }
        }
        s_red[warp][lane + 32 * q] = term;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int q = 0; q < MS; ++q) {
            long long sum = 0;
#pragma unroll
            for (int b = 0; b < LW; ++b) sum += s_red[b][lane + 32 * q];   // |sum| < 32 * 2^57
            if (mvalid[q]) {
                const unsigned long long lo = (unsigned long long)sum & 0xffffffffull;
                const long long hi = sum >> 32;
                atomicAdd(&L.acc[2 * md[q].out], lo);
                atomicAdd(&L.acc[2 * md[q].out + 1], (unsigned long long)hi);
            }
        }
    }
}

template <int KT, int MS, bool TMA>
__global__ void __launch_bounds__(LW * 32, (KT > 0 && MS == 1) ? 3 : 2)
    ksg_lane_kernel(const KsgLaunch L, const __grid_constant__ CUtensorMap tmx)
{
    ksg_lane_item<KT, MS, TMA>(L, tmx, blockIdx.x);
}

template <int KT, int MS, bool TMA>
__global__ void __launch_bounds__(LW * 32, (KT > 0 && MS == 1) ? 3 : 2)
    ksg_lane_persistent_kernel(const KsgLaunch L, const __grid_constant__ CUtensorMap tmx)
{
    // Persistent grid: every CTA takes its next item from a device counter
    // (zeroed before the launch) until none is left, or until a tile copy has
    // timed out somewhere (the error flag is read by one thread and the
    // decision shared, so the CTA leaves together).
    __shared__ long long s_item;
    long long item = blockIdx.x;
    while (item < L.n_items) {
        ksg_lane_item<KT, MS, TMA>(L, tmx, item);
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned long long bad = *(volatile const unsigned long long *)(L.work + 2);
            s_item = bad ? L.n_items
                         : (long long)atomicAdd(L.item_counter, 1ull) + (long long)gridDim.x;
        }
        __syncthreads();
        item = s_item;
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

// Apply the swaps (i, jb[i]) for i = n-1 down to 1 to p, in that order, by
// warp 0 of the CTA.  Steps go in batches of 32 consecutive positions: when
// every draw of a batch lies below the batch's lowest position and no two
// draws are equal, the batch's swaps touch disjoint positions and commute, so
// the 32 lanes apply them at once; otherwise lane 0 applies the batch in
// order.  The result equals the sequential loop exactly.
template <typename P, typename J>
__device__ void fy_apply(P *p, const J *jb, int n)
{
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    for (int hi = n - 1; hi >= 1;) {
        const int lo = hi - 31 > 1 ? hi - 31 : 1;
        const int i = hi - lane;
        const bool valid = i >= lo;
        const int j = valid ? (int)jb[i] : -1 - lane;   // invalid lanes: distinct dummies
        const unsigned same = __match_any_sync(0xffffffffu, j);
        const bool ok = !valid || (j < lo && __popc(same) == 1);
        if (__all_sync(0xffffffffu, ok)) {
            P a = 0, b = 0;
            if (valid) {
                a = p[i];
                b = p[j];
            }
            __syncwarp();
            if (valid) {
                p[i] = b;
                p[j] = a;
            }
            __syncwarp();
        } else {
            if (lane == 0)
                for (int ii = hi; ii >= lo; --ii) {
                    const int jj = (int)jb[ii];
                    const P t = p[ii];
                    p[ii] = p[jj];
                    p[jj] = t;
                }
            __syncwarp();
        }
        hi = lo - 1;
    }
}

// Fisher-Yates shuffle of p[0, n) in place (positions n-1 down to 1, j drawn
// as floor(r (i + 1) / 2^64)) with the SplitMix64 generator whose state starts
// at st.  The k-th output of that generator is mix(st + (k + 1) gamma), so with
// jb (n ints of shared memory) every thread of the CTA computes draws first
// and one thread then runs the swaps; without it one thread does both.  The
// permutation is the same either way.  Called by the whole CTA.
__device__ void fy_shuffle(int32_t *p, int n, uint64_t st, int32_t *jb)
{
    if (jb) {
        for (int i = 1 + threadIdx.x; i < n; i += blockDim.x) {
            uint64_t z = st + (uint64_t)(n - i) * 0x9E3779B97F4A7C15ull;   // draw k = n-1-i
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            jb[i] = (int)__umul64hi(z, (uint64_t)(i + 1));
        }
        __syncthreads();
        fy_apply(p, jb, n);
    } else if (threadIdx.x == 0) {
        for (int i = n - 1; i >= 1; --i) {
            const uint64_t r = sm64_next(st);
            const int j = (int)__umul64hi(r, (uint64_t)(i + 1));
            const int32_t t = p[i];
            p[i] = p[j];
            p[j] = t;
        }
    }
    __syncthreads();
}

// The draw of position i (1 <= i < n): j = floor(r (i + 1) / 2^64) with r the
// (n - 1 - i)-th output of SplitMix64 from state st, mix(st + (n - i) gamma).
__device__ __forceinline__ int fy_draw(uint64_t st, int n, int i)
{
    uint64_t z = st + (uint64_t)(n - i) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (int)__umul64hi(z, (uint64_t)(i + 1));
}

// The same shuffle for n <= 65535 with the permutation as 16-bit values in
// shared memory (2 bytes per point), the result widened into out.  Warp 0
// walks the steps i = n-1 down to 1 in windows of 32, lane l holding step
// hi - l and its draw j.  Each round applies at once the longest leading run
// of steps whose swaps touch pairwise distinct positions: a step with j != i
// allows runs of at most hi - j steps (its j must lie below the run), and a
// draw repeated from an earlier step ends the run before it; disjoint swaps
// commute, so the result equals the sequential loop exactly.  The next
// window's draws come from this window's (shifted) and from draws computed
// one window ahead.  No draw is stored, so a CTA needs only the permutation
// and one warp.  Called by the whole CTA.
__device__ void fy_shuffle16(uint16_t *p, int n, uint64_t st, int32_t *out)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = (uint16_t)i;
    __syncthreads();
    if (threadIdx.x < 32) {
        const unsigned full = 0xffffffffu;
        const int lane = threadIdx.x;
        const unsigned lower = (1u << lane) - 1u;
        int hi = n - 1;
        int jc = (hi - lane >= 1) ? fy_draw(st, n, hi - lane) : 0;
        while (hi >= 1) {
            const int i = hi - lane;
            const bool valid = i >= 1;
            const int j = valid ? jc : -1 - lane;   // invalid lanes: distinct dummies
            // the window below, in case the whole window applies
            const int is = hi - 32 - lane;
            const int js = is >= 1 ? fy_draw(st, n, is) : 0;
            int lim = !valid ? 0 : (j == i ? 32 : hi - j);
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {   // running minimum over lanes 0..lane
                const int t = __shfl_up_sync(full, lim, o);
                if (lane >= o) lim = min(lim, t);
            }
            const unsigned same = __match_any_sync(full, j);
            const unsigned run = __ballot_sync(full, valid && lane < lim && (same & lower) == 0);
            const int k = run == full ? 32 : __ffs(~run) - 1;   // >= 1: step hi always applies
            const bool act = lane < k && j != i;
            uint16_t a = 0, b = 0;
            if (act) {
                a = p[i];
                b = p[j];
            }
            __syncwarp();
            if (act) {
                p[i] = b;
                p[j] = a;
            }
            __syncwarp();
            // next window hi - k: lane l < 32 - k takes lane l + k's draw, the
            // others the draws computed ahead for lane l + k - 32
            const int from_cur = __shfl_down_sync(full, j, k & 31);
            const int from_ahead = __shfl_sync(full, js, (lane + k - 32) & 31);
            jc = lane < 32 - k ? from_cur : from_ahead;
            hi -= k;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) out[i] = (int32_t)p[i];
}

// One round of fy_shuffle16's warp walk for a permutation p (state: the top
// step hi and this lane's draw jc).  Called by the whole warp while hi >= 1.
__device__ __forceinline__ void fy16_round(uint16_t *p, int n, uint64_t st, int &hi, int &jc)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lower = (1u << lane) - 1u;
    const int i = hi - lane;
    const bool valid = i >= 1;
    const int j = valid ? jc : -1 - lane;   // invalid lanes: distinct dummies
    const int is = hi - 32 - lane;
    const int js = is >= 1 ? fy_draw(st, n, is) : 0;
    int lim = !valid ? 0 : (j == i ? 32 : hi - j);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(full, lim, o);
        if (lane >= o) lim = min(lim, t);
    }
    const unsigned same = __match_any_sync(full, j);
    const unsigned run = __ballot_sync(full, valid && lane < lim && (same & lower) == 0);
    const int k = run == full ? 32 : __ffs(~run) - 1;   // >= 1: step hi always applies
    const bool act = lane < k && j != i;
    uint16_t a = 0, b = 0;
    if (act) {
        a = p[i];
        b = p[j];
    }
    __syncwarp();
    if (act) {
        p[i] = b;
        p[j] = a;
    }
    __syncwarp();
    const int from_cur = __shfl_down_sync(full, j, k & 31);
    const int from_ahead = __shfl_sync(full, js, (lane + k - 32) & 31);
    jc = lane < 32 - k ? from_cur : from_ahead;
    hi -= k;
}

// The same permutations as fisher_yates_kernel (16-bit mode), written as
// 16-bit rows of `pitch` entries (a multiple of 8, zeros past n): one warp per
// permutation, the rounds of fy_shuffle16.  (Two walks interleaved in one warp
// were measured 1.5x slower: the rounds' warp collectives and __syncwarp keep
// the two chains from overlapping, and half as many warps remain.)
__global__ void fisher_yates16_kernel(uint16_t *out, int pitch, int n, uint64_t seed,
                                      uint64_t target, uint64_t stage, uint64_t iter,
                                      uint64_t s_first)
{
    extern __shared__ int32_t sperm16[];
    uint16_t *p = reinterpret_cast<uint16_t *>(sperm16);
    uint64_t h = sm64_once(seed ^ target);
    h = sm64_once(h ^ stage);
    h = sm64_once(h ^ iter);
    const uint64_t st = sm64_once(h ^ (s_first + blockIdx.x));
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = (uint16_t)i;
    __syncwarp();
    const int lane = threadIdx.x & 31;
    int hi = n - 1;
    int jc = (hi - lane >= 1) ? fy_draw(st, n, hi - lane) : 0;
    while (hi >= 1) fy16_round(p, n, st, hi, jc);
    __syncwarp();
    uint16_t *o = out + (long long)blockIdx.x * pitch;
    for (int i = 8 * threadIdx.x; i < pitch; i += 8 * blockDim.x) {
        uint16_t v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = i + u < n ? p[i + u] : (uint16_t)0;
        uint4 w;
        w.x = v[0] | ((uint32_t)v[1] << 16);
        w.y = v[2] | ((uint32_t)v[3] << 16);
        w.z = v[4] | ((uint32_t)v[5] << 16);
        w.w = v[6] | ((uint32_t)v[7] << 16);
        *reinterpret_cast<uint4 *>(o + i) = w;
    }
}

// in_smem: bit 0 = the permutation is built in shared memory, bit 1 = the
// draws are computed in parallel into shared memory after it, 4 = the
// permutation as 16-bit values with the draws computed by the swapping warp
// (n <= 65535)
__global__ void fisher_yates_kernel(int32_t *out, long long stride, int n, uint64_t seed,
                                    uint64_t target, uint64_t stage, uint64_t iter,
                                    uint64_t s_first, int in_smem)
{
    extern __shared__ int32_t sperm[];
    const uint64_t s = s_first + blockIdx.x;
    if (in_smem == 4) {
        uint64_t h = sm64_once(seed ^ target);
        h = sm64_once(h ^ stage);
        h = sm64_once(h ^ iter);
        uint16_t *p16 = reinterpret_cast<uint16_t *>(sperm);
        fy_shuffle16(p16, n, sm64_once(h ^ s), out + (long long)blockIdx.x * stride);
        return;
    }
    int32_t *p = (in_smem & 1) ? sperm : out + (long long)blockIdx.x * stride;
    int32_t *jb = (in_smem & 2) ? sperm + ((in_smem & 1) ? n : 0) : nullptr;
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = i;
    __syncthreads();
    uint64_t h = sm64_once(seed ^ target);
    h = sm64_once(h ^ stage);
    h = sm64_once(h ^ iter);
    fy_shuffle(p, n, sm64_once(h ^ s), jb);
    in_smem &= 1;
    if (in_smem)
        for (int i = threadIdx.x; i < n; i += blockDim.x)
            out[(long long)blockIdx.x * stride + i] = sperm[i];
}

// ---------------- spatial order over (Y, Z) ----------------
// The points of a group are processed in a spatial order of their shared
// (Y, Z) coordinates, and every aligned chunk of 8 and tile of 256 ordered
// points carries a bounding box that the pruning tests.  The order only
// affects how much work the pruning saves, never a result.  Two orders:
//  * a Morton curve (per-dimension ranges, keys of interleaved bits, one
//    bitonic sort): cheap to build, for small launches;
//  * the leaf order of a k-d tree: a node of m > 8 points is split at the
//    median of its widest dimension into a first child of `kd_left(m)` points
//    and a second child of the rest; the first child's size is a multiple of
//    256 (nodes above 256 points) or of 8, so every node starts on a multiple
//    of 8 (of 256 above 256 points) and every aligned chunk and tile is a union
//    of whole nodes, whose boxes stay compact in every dimension.  It costs
//    one sort per tree level and pays for large groups, where it cuts the
//    chunks and tiles the pruning must visit.
constexpr int kOrderMaxSeg = 2048;   // nodes that still split at one level (> 8 points: N / 9)
constexpr size_t kOrderSmem = (size_t)kMaxOrderN * 8 + (size_t)kMaxOrderN * 2 +
                              6 * (size_t)kOrderMaxSeg * 4;

// float <-> uint32 with the same order (finite values and infinities)
__device__ __forceinline__ unsigned ordered_u32(float v)
{
    const unsigned b = __float_as_uint(v);
    return b ^ ((b >> 31) ? 0xFFFFFFFFu : 0x80000000u);
}
__device__ __forceinline__ float ordered_f32(unsigned u)
{
    return __uint_as_float(u ^ ((u >> 31) ? 0x80000000u : 0xFFFFFFFFu));
}

// points of the first child of a node of m > 8 points: the multiple of 256
// (m > 256) or of 8 nearest to m / 2, at least one block and below m
__device__ __forceinline__ int kd_left(int m)
{
    const int blk = m > 256 ? 256 : 8;
    const int left = (m + blk) / (2 * blk) * blk;
    return left < blk ? blk : (left > m - 1 ? m - 1 : left);
}


// Ascending bitonic sort of P2 keys in shared memory (one CTA).
__device__ void bitonic_sort_keys(unsigned long long *skeys, int P2)
{
    for (int kk = 2; kk <= P2; kk <<= 1) {
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int t = threadIdx.x; t < (P2 >> 1); t += blockDim.x) {
                const int lo = 2 * jj * (t / jj) + (t % jj);
                const int hi = lo + jj;
                const bool up = (lo & kk) == 0;
                const unsigned long long x = skeys[lo], y = skeys[hi];
                if ((x > y) == up) {
                    skeys[lo] = y;
                    skeys[hi] = x;
                }
            }
            __syncthreads();
        }
    }
}

// Morton order: per-dimension ranges, keys of bits interleaved from the most
// significant (up to 50 bits) packed with the point index, one sort.
__device__ void morton_order(const OrderJob &J, unsigned long long *skeys, int P2)
{
    __shared__ float s_lo[32], s_hi[32];
    __shared__ float s_red[2][32];
    const int N = J.N, D = J.dyz;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nw = blockDim.x >> 5;
    const float *base = J.base;
    for (int d = 0; d < D; ++d) {
        float mn = CUDART_INF_F, mx = -CUDART_INF_F;
        for (int p = tid; p < N; p += blockDim.x) {
            const float v = base[J.cols[d] + p];
            mn = fminf(mn, v);
            mx = fmaxf(mx, v);
        }
        mn = warp_min(mn);
        mx = warp_max(mx);
        if (lane == 0) {
            s_red[0][wid] = mn;
            s_red[1][wid] = mx;
        }
        __syncthreads();
        if (wid == 0) {
            mn = lane < nw ? s_red[0][lane] : CUDART_INF_F;
            mx = lane < nw ? s_red[1][lane] : -CUDART_INF_F;
            mn = warp_min(mn);
            mx = warp_max(mx);
            if (lane == 0) {
                s_lo[d] = mn;
                s_hi[d] = mx;
            }
        }
        __syncthreads();
    }
    int bits = 50 / D;
    if (bits > 24) bits = 24;
    if (bits < 1) bits = 1;
    const float qmax = (float)((1u << bits) - 1u);
    for (int p = tid; p < P2; p += blockDim.x) {
        unsigned long long key = ~0ull;
        if (p < N) {
            unsigned long long mort = 0;
            unsigned int q[32];
            for (int d = 0; d < D; ++d) {
                const float span = s_hi[d] - s_lo[d];
                float f = span > 0.f ? (base[J.cols[d] + p] - s_lo[d]) / span * qmax : 0.f;
                f = fminf(fmaxf(f, 0.f), qmax);
                q[d] = (unsigned int)f;
            }
            for (int b = bits - 1; b >= 0; --b)
                for (int d = 0; d < D; ++d) mort = (mort << 1) | ((q[d] >> b) & 1u);
            key = (mort << 14) | (unsigned long long)p;
        }
        skeys[p] = key;
    }
    __syncthreads();
    bitonic_sort_keys(skeys, P2);
}

// k-d tree order, built level by level over the current order: every node
// that still splits (the active nodes, start-ordered) finds its widest
// dimension from per-dimension extents (segmented warp scans over consecutive
// positions, then shared-memory atomics), and one bitonic sort of the keys
// (node start, coordinate on that dimension, point) orders every active node
// along its dimension at once; points of finished leaves key on their own
// position and stay.
__device__ void kd_order(const OrderJob &J, unsigned long long *skeys, int P2)
{
    short *s_seg = reinterpret_cast<short *>(skeys + kMaxOrderN); // [N] active node of a position, -1 none
    int *s_start = reinterpret_cast<int *>(s_seg + kMaxOrderN);   // [kOrderMaxSeg] active nodes
    int *s_size = s_start + kOrderMaxSeg;
    unsigned *s_lo = reinterpret_cast<unsigned *>(s_size + kOrderMaxSeg);
    unsigned *s_hi = s_lo + kOrderMaxSeg;
    float *s_ext = reinterpret_cast<float *>(s_hi + kOrderMaxSeg);
    int *s_dim = reinterpret_cast<int *>(s_ext + kOrderMaxSeg);
    __shared__ int s_nact;
    const int N = J.N, D = J.dyz;
    const int tid = threadIdx.x, lane = tid & 31;
    const float *base = J.base;
    for (int p = tid; p < P2; p += blockDim.x) skeys[p] = p < N ? (unsigned long long)p : ~0ull;
    if (tid == 0) {
        s_start[0] = 0;
        s_size[0] = N;
        s_nact = N > 8 ? 1 : 0;
    }
    __syncthreads();
    while (s_nact > 0) {
        const int nact = s_nact;
        // the active node of every position (last one starting at or before it)
        for (int p = tid; p < N; p += blockDim.x) {
            int lo = 0, hi = nact - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_start[mid] <= p) lo = mid;
                else hi = mid - 1;
            }
            s_seg[p] = (s_start[lo] <= p && p < s_start[lo] + s_size[lo]) ? (short)lo : (short)-1;
        }
        for (int s = tid; s < nact; s += blockDim.x) {
            s_ext[s] = -1.f;
            s_dim[s] = 0;
        }
        __syncthreads();
        // widest dimension of every active node (first one on ties)
        for (int d = 0; d < D; ++d) {
            for (int s = tid; s < nact; s += blockDim.x) {
                s_lo[s] = 0xFFFFFFFFu;
                s_hi[s] = 0u;
            }
            __syncthreads();
            for (int p0 = 0; p0 < N; p0 += blockDim.x) {   // whole warps: the scan shuffles
                const int p = p0 + tid;
                int sg = -1;
                unsigned v = 0u;
                if (p < N) {
                    sg = s_seg[p];
                    if (sg >= 0) v = ordered_u32(base[J.cols[d] + (int)(skeys[p] & 0x3FFFull)]);
                }
                unsigned mn = v, mx = v;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const unsigned a = __shfl_up_sync(0xffffffffu, mn, off);
                    const unsigned b = __shfl_up_sync(0xffffffffu, mx, off);
                    const int so = __shfl_up_sync(0xffffffffu, sg, off);
                    if (lane >= off && so == sg) {   // nodes are contiguous runs of positions
                        mn = min(mn, a);
                        mx = max(mx, b);
                    }
                }
                const int sn = __shfl_down_sync(0xffffffffu, sg, 1);
                if (sg >= 0 && (lane == 31 || sn != sg)) {
                    atomicMin(&s_lo[sg], mn);
                    atomicMax(&s_hi[sg], mx);
                }
            }
            __syncthreads();
            for (int s = tid; s < nact; s += blockDim.x) {
                const float e = ordered_f32(s_hi[s]) - ordered_f32(s_lo[s]);
                if (e > s_ext[s]) {
                    s_ext[s] = e;
                    s_dim[s] = d;
                }
            }
            __syncthreads();
        }
        // keys: (node start, coordinate on its dimension, point) for active
        // positions, (own position, point) for the others
        for (int p = tid; p < N; p += blockDim.x) {
            const unsigned long long idx = skeys[p] & 0x3FFFull;
            const int sg = s_seg[p];
            unsigned long long key = ((unsigned long long)p << 46) | idx;
            if (sg >= 0) {
                const float v = base[J.cols[s_dim[sg]] + (int)idx];
                key = ((unsigned long long)s_start[sg] << 46) |
                      ((unsigned long long)ordered_u32(v) << 14) | idx;
            }
            skeys[p] = key;
        }
        __syncthreads();
        bitonic_sort_keys(skeys, P2);
        for (int p = tid; p < N; p += blockDim.x) skeys[p] &= 0x3FFFull;
        // the children that still split, in order (one warp; written to the
        // extent arrays, free now, then copied back)
        if (tid < 32) {
            int out = 0;
            for (int c0 = 0; c0 < 2 * nact; c0 += 32) {
                const int c = c0 + lane;
                int st = 0, sz = 0;
                if (c < 2 * nact) {
                    const int s = c >> 1, m = s_size[s], left = kd_left(m);
                    st = s_start[s] + ((c & 1) ? left : 0);
                    sz = (c & 1) ? m - left : left;
                }
                const bool act = sz > 8;
                const unsigned bal = __ballot_sync(0xffffffffu, act);
                if (act) {
                    const int o = out + __popc(bal & ((1u << lane) - 1u));
                    s_lo[o] = (unsigned)st;
                    s_hi[o] = (unsigned)sz;
                }
                out += __popc(bal);
            }
            __syncwarp();
            for (int s = lane; s < out; s += 32) {
                s_start[s] = (int)s_lo[s];
                s_size[s] = (int)s_hi[s];
            }
            if (lane == 0) s_nact = out;
        }
        __syncthreads();
    }
}

// One CTA per group: the order (J.kd: k-d tree, else Morton curve), then the
// sorted coordinates and the bounding box of every aligned chunk of 8 and
// tile of 256 sorted points.
__global__ void __launch_bounds__(1024) order_kernel(const OrderJob *jobs)
{
    extern __shared__ unsigned long long skeys[];
    const OrderJob &J = jobs[blockIdx.x];
    const int N = J.N, D = J.dyz;
    const int tid = threadIdx.x;
    const float *base = J.base;
    int P2 = 1;
    while (P2 < N) P2 <<= 1;
    if (J.kd) kd_order(J, skeys, P2);
    else morton_order(J, skeys, P2);
    for (int p = tid; p < N; p += blockDim.x) {
        const int t = (int)(skeys[p] & 0x3FFFull);
        J.sigma[p] = t;
        for (int d = 0; d < D; ++d) J.yz[(size_t)d * N + p] = base[J.cols[d] + t];
    }
    const int nch = (N + 7) >> 3;
    for (int e = tid; e < nch * D; e += blockDim.x) {
        const int d = e / nch, c = e - d * nch;
        float mn = CUDART_INF_F, mx = -CUDART_INF_F;
        for (int p = 8 * c; p < min(8 * c + 8, N); ++p) {
            const float v = base[J.cols[d] + (int)(skeys[p] & 0x3FFFull)];
            mn = fminf(mn, v);
            mx = fmaxf(mx, v);
        }
        J.box[(size_t)d * nch + c] = make_float2(mn, mx);
    }
    const int ntl = (N + 255) >> 8;
    for (int e = tid; e < ntl * D; e += blockDim.x) {
        const int d = e / ntl, c = e - d * ntl;
        float mn = CUDART_INF_F, mx = -CUDART_INF_F;
        for (int p = 256 * c; p < min(256 * c + 256, N); ++p) {
            const float v = base[J.cols[d] + (int)(skeys[p] & 0x3FFFull)];
            mn = fminf(mn, v);
            mx = fmaxf(mx, v);
        }
        J.tbox[(size_t)d * ntl + c] = make_float2(mn, mx);
    }
}

// Ascending sort of one column (bitonic in shared memory; +inf pads).
__global__ void __launch_bounds__(1024) value_sort_kernel(const ValueSortJob *jobs)
{
    extern __shared__ float sv[];
    const ValueSortJob J = jobs[blockIdx.x];
    int P2 = 1;
    while (P2 < J.N) P2 <<= 1;
    for (int p = threadIdx.x; p < P2; p += blockDim.x) sv[p] = p < J.N ? J.src[p] : CUDART_INF_F;
    __syncthreads();
    for (int kk = 2; kk <= P2; kk <<= 1) {
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int t = threadIdx.x; t < (P2 >> 1); t += blockDim.x) {
                const int lo = 2 * jj * (t / jj) + (t % jj);
                const int hi = lo + jj;
                const bool up = (lo & kk) == 0;
                const float x = sv[lo], y = sv[hi];
                if ((x > y) == up) {
                    sv[lo] = y;
                    sv[hi] = x;
                }
            }
            __syncthreads();
        }
    }
    for (int p = threadIdx.x; p < J.N; p += blockDim.x) J.dst[p] = sv[p];
}

// out[p] = perm[sigma[p]]: a surrogate permutation composed with a group's
// spatial order (index arrays only; the data is never copied)
__global__ void compose_kernel(const ComposeJob *jobs)
{
    const ComposeJob J = jobs[blockIdx.y];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < J.N; p += gridDim.x * blockDim.x)
        J.out[p] = J.perm[J.sigma[p]];
}

// Many permutation requests in one launch: CTA g is permutation g of the
// concatenated request list (binary search over the requests' first index).
__global__ void fisher_yates_multi_kernel(const PermJob *jobs, int n_jobs, int smem_n, int jb_ok)
{
    extern __shared__ int32_t sperm[];
    const long long g = blockIdx.x;
    int lo = 0, hi = n_jobs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].perm_begin <= g) lo = mid;
        else hi = mid - 1;
    }
    const PermJob J = jobs[lo];
    const int r = (int)(g - J.perm_begin);
    const int n = J.n;
    const bool in_smem = n <= smem_n;
    int32_t *dst = J.out + (long long)r * n;
    uint64_t h0 = sm64_once(J.seed ^ J.target);
    h0 = sm64_once(h0 ^ J.stage);
    h0 = sm64_once(h0 ^ J.iter);
    if (in_smem && n <= 65535) {
        uint16_t *p16 = reinterpret_cast<uint16_t *>(sperm);
        fy_shuffle16(p16, n, sm64_once(h0 ^ (J.s_first + (uint64_t)r)), dst);
        return;
    }
    int32_t *p = in_smem ? sperm : dst;
    // smem_n >= 0 holds the permutation; a second smem_n ints hold the draws
    int32_t *jb = (in_smem && jb_ok) ? sperm + smem_n : nullptr;
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = i;
    __syncthreads();
    uint64_t h = sm64_once(J.seed ^ J.target);
    h = sm64_once(h ^ J.stage);
    h = sm64_once(h ^ J.iter);
    fy_shuffle(p, n, sm64_once(h ^ (J.s_first + (uint64_t)r)), jb);
    if (in_smem)
        for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = sperm[i];
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
    if (v.persist) {
        if (!dx1 || !v.tma) return nullptr;
        if (v.m == 32 && v.kt == 4)
            return reinterpret_cast<const void *>(&ksg_lane_persistent_kernel<4, 1, true>);
        if (v.m == 32 && v.kt == 0)
            return reinterpret_cast<const void *>(&ksg_lane_persistent_kernel<0, 1, true>);
        if (v.m == 64 && v.kt == 4)
            return reinterpret_cast<const void *>(&ksg_lane_persistent_kernel<4, 2, true>);
        return nullptr;
    }
    if (dx1 && v.m == 32) {
        if (v.kt == 4)
            return v.tma ? reinterpret_cast<const void *>(&ksg_lane_kernel<4, 1, true>)
                         : reinterpret_cast<const void *>(&ksg_lane_kernel<4, 1, false>);
        if (v.kt == 0)
            return v.tma ? reinterpret_cast<const void *>(&ksg_lane_kernel<0, 1, true>)
                         : reinterpret_cast<const void *>(&ksg_lane_kernel<0, 1, false>);
        return nullptr;
    }
    if (dx1 && v.m == 64) {
        if (v.kt == 4 && v.tma) return reinterpret_cast<const void *>(&ksg_lane_kernel<4, 2, true>);
        return nullptr;
    }
    // single-variable X always runs a member-lane kernel; the fused kernel
    // serves multi-variable X (the omnibus test's block)
    if (!dx1) {
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

// cudaFuncSetAttribute acts on the current device, so a launcher that raises a
// kernel's dynamic shared-memory limit remembers that per device, not per
// process: the first launch on a second GPU sets it again.
constexpr int kAttrDevices = 64;
static cudaError_t smem_attr_once(const void *f, int bytes, bool (&done)[kAttrDevices])
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kAttrDevices && done[dev]) return cudaSuccess;
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < kAttrDevices) done[dev] = true;
    return cudaSuccess;
}

cudaError_t ksg_prepare_attributes()
{
    const KsgVariant vs[] = {{4, 4, QT},  {2, 0, QT},
                             {2, 4, QT},  {32, 4, LW * 32}, {32, 0, LW * 32},
                             {32, 4, LW * 32, true}, {32, 0, LW * 32, true},
                             {64, 4, LW * 32, true}, {32, 4, LW * 32, true, true},
                             {32, 0, LW * 32, true, true}, {64, 4, LW * 32, true, true}};
    for (const auto &v : vs)
        for (int d = 0; d < 2; ++d) {
            const void *f = select_kernel(v, d == 0);
            if (!f) continue;
            cudaError_t e =
                cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            if (e != cudaSuccess) return e;
        }
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(&order_kernel),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kOrderSmem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(reinterpret_cast<const void *>(&stats_kernel),
                                cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

cudaError_t launch_value_sort(const ValueSortJob *jobs, int n_jobs, cudaStream_t st)
{
    if (n_jobs <= 0) return cudaSuccess;
    static bool attr_done[kAttrDevices] = {};
    {
        const cudaError_t e =
            smem_attr_once(reinterpret_cast<const void *>(&value_sort_kernel),
                           kMaxOrderN * 4, attr_done);
        if (e != cudaSuccess) return e;
    }
    value_sort_kernel<<<n_jobs, 1024, kMaxOrderN * 4, st>>>(jobs);
    return cudaGetLastError();
}

cudaError_t launch_compose(const ComposeJob *jobs, int n_jobs, int max_n, cudaStream_t st)
{
    if (n_jobs <= 0) return cudaSuccess;
    const int bx = (max_n + 255) / 256 < 64 ? (max_n + 255) / 256 : 64;
    // one grid row per job; the grid's y extent is at most 65535
    for (int j0 = 0; j0 < n_jobs; j0 += 65535) {
        const int ny = n_jobs - j0 < 65535 ? n_jobs - j0 : 65535;
        compose_kernel<<<dim3(bx, ny), 256, 0, st>>>(jobs + j0);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_order(const OrderJob *jobs, int n_jobs, cudaStream_t st)
{
    if (n_jobs <= 0) return cudaSuccess;
    order_kernel<<<n_jobs, 1024, kOrderSmem, st>>>(jobs);
    return cudaGetLastError();
}

cudaError_t launch_ksg(const KsgLaunch &L, const KsgVariant &v, long long n_items, bool dx1,
                       size_t smem_bytes, cudaStream_t st, const CUtensorMap *tmap)
{
    const void *f = select_kernel(v, dx1);
    if (!f) return cudaErrorInvalidValue;
    if (n_items <= 0) return cudaSuccess;
    if (n_items > 0x7fffffffLL) return cudaErrorInvalidValue;
    const bool lane = dx1 && (v.m == 32 || v.m == 64);
    if (v.tma && (!lane || !tmap || !L.xval || !L.work || L.jt > LW * 32 || (L.jt & 31)))
        return cudaErrorInvalidValue;
    KsgLaunch arg = L;
    arg.n_items = n_items;
    unsigned grid = (unsigned)n_items;
    if (v.persist != (arg.item_counter != nullptr)) return cudaErrorInvalidValue;
    if (v.persist) {
        if (!lane || !arg.work) return cudaErrorInvalidValue;
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, v.qt, smem_bytes);
        if (e != cudaSuccess) return e;
        const long long full = (long long)sms * (per_sm > 0 ? per_sm : 1);
        if (full < n_items) grid = (unsigned)full;
    }
    CUtensorMap map;
    if (tmap) map = *tmap;
    else std::memset(&map, 0, sizeof map);
    void *args[] = {&arg, &map};
    return cudaLaunchKernel(f, dim3(grid), dim3(v.qt), args, smem_bytes, st);
}

// One CTA per member row: the member's X values in its group's point order
// (through the composed permutation, the group's order, or as is), zero from
// N to the row pitch.
__global__ void xval_kernel(const KsgLaunch L, int n_rows)
{
    const int r = blockIdx.x;
    if (r >= n_rows) return;
    int glo = 0, ghi = L.n_groups - 1;
    while (glo < ghi) {
        const int mid = (glo + ghi + 1) >> 1;
        if (L.groups[mid].member_begin <= r) glo = mid;
        else ghi = mid - 1;
    }
    const GroupDesc &G = L.groups[glo];
    const MemberDesc md = L.members[r];
    const float *src = G.base + L.cols[md.xcol];
    float *dst = const_cast<float *>(L.xval) + (size_t)r * L.xpitch;
    for (long long j = threadIdx.x; j < L.xpitch; j += blockDim.x) {
        float v = 0.f;
        if (j < G.N) {
            const int jj = (int)j;
            v = src[md.perm ? md.perm[jj] : (G.sigma ? G.sigma[jj] : jj)];
        }
        dst[j] = v;
    }
}

cudaError_t launch_xval(const KsgLaunch &L, int n_rows, cudaStream_t st)
{
    if (n_rows <= 0) return cudaSuccess;
    xval_kernel<<<n_rows, 256, 0, st>>>(L, n_rows);
    return cudaGetLastError();
}

cudaError_t encode_xval_map(CUtensorMap *map, const float *xval, long long pitch, int rows,
                            int box_rows)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    if (rows < 1 || pitch < 32 || (pitch & 3) || box_rows < 1 || box_rows > 256 ||
        (reinterpret_cast<uintptr_t>(xval) & 15))
        return cudaErrorInvalidValue;
    const cuuint64_t dims[2] = {(cuuint64_t)pitch, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * 4};
    const cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                              const_cast<float *>(xval), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_perms(int32_t *out, long long stride, int n, uint64_t seed, uint64_t target,
                         uint64_t stage, uint64_t iter, uint64_t s_first, int n_perm,
                         cudaStream_t st)
{
    if (n_perm <= 0) return cudaSuccess;
    const size_t smem = (size_t)n * sizeof(int32_t);
    const int in_smem = smem <= 200 * 1024;
    static bool attr_done[kAttrDevices] = {};
    {
        const cudaError_t e =
            smem_attr_once(reinterpret_cast<const void *>(&fisher_yates_kernel),
                           200 * 1024, attr_done);
        if (e != cudaSuccess) return e;
    }
    // permutation and draws in shared memory when both fit, else the
    // permutation alone, else neither
    int mode = 0;
    size_t bytes = 0;
    int threads = 256;
    if (n <= 65535) {
        mode = 4;
        bytes = (size_t)n * 2;   // the permutation alone, one warp per CTA
        threads = 32;
    } else if (2 * smem <= 200 * 1024) {
        mode = 3;
        bytes = 2 * smem;
    } else if (in_smem) {
        mode = 1;
        bytes = smem;
    }
    fisher_yates_kernel<<<n_perm, threads, bytes, st>>>(out, stride, n, seed, target, stage,
                                                        iter, s_first, mode);
    return cudaGetLastError();
}

cudaError_t launch_perms16(uint16_t *out, int pitch, int n, uint64_t seed, uint64_t target,
                           uint64_t stage, uint64_t iter, uint64_t s_first, int n_perm,
                           cudaStream_t st)
{
    if (n_perm <= 0) return cudaSuccess;
    if (n < 1 || n > kPerm16MaxN || pitch < n || (pitch & 7) ||
        (reinterpret_cast<uintptr_t>(out) & 15))
        return cudaErrorInvalidValue;
    static bool attr_done[kAttrDevices] = {};
    {
        const cudaError_t e =
            smem_attr_once(reinterpret_cast<const void *>(&fisher_yates16_kernel),
                           200 * 1024, attr_done);
        if (e != cudaSuccess) return e;
    }
    fisher_yates16_kernel<<<n_perm, 32, (size_t)n * 2, st>>>(out, pitch, n, seed, target, stage,
                                                            iter, s_first);
    return cudaGetLastError();
}

// Surrogates of pooled replications: R trials of n points (point r*n + t).
// One CTA per surrogate s = s_first + blockIdx.x, state keyed as in
// fisher_yates_kernel.  mode 0: Fisher-Yates of the R trials, point r*n + t
// reads sigma[r]*n + t; mode 1: one Fisher-Yates shuffle per trial, trial 0
// first, all from one continuing generator (R = 1 gives the flat permutation).
__global__ void fisher_yates_trials_kernel(int32_t *out, int R, int n, uint64_t seed,
                                           uint64_t target, uint64_t stage, uint64_t iter,
                                           uint64_t s_first, int mode, int in_smem)
{
    extern __shared__ int32_t sbuf[];
    const uint64_t s = s_first + blockIdx.x;
    const long long total = (long long)R * n;
    int32_t *dst = out + (long long)blockIdx.x * total;
    uint64_t h = sm64_once(seed ^ target);
    h = sm64_once(h ^ stage);
    h = sm64_once(h ^ iter);
    uint64_t st = sm64_once(h ^ s);
    if (mode == 0) {
        int32_t *sigma = sbuf;   // [R]
        for (int r = threadIdx.x; r < R; r += blockDim.x) sigma[r] = r;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int i = R - 1; i >= 1; --i) {
                const uint64_t x = sm64_next(st);
                const int j = (int)__umul64hi(x, (uint64_t)(i + 1));
                const int t = sigma[i];
                sigma[i] = sigma[j];
                sigma[j] = t;
            }
        __syncthreads();
        for (long long p = threadIdx.x; p < total; p += blockDim.x) {
            const int r = (int)(p / n), t = (int)(p - (long long)r * n);
            dst[p] = sigma[r] * n + t;
        }
        return;
    }
    int32_t *q = in_smem ? sbuf : dst;
    for (long long p = threadIdx.x; p < total; p += blockDim.x) q[p] = (int32_t)p;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int r = 0; r < R; ++r) {
            int32_t *b = q + (long long)r * n;
            for (int i = n - 1; i >= 1; --i) {
                const uint64_t x = sm64_next(st);
                const int j = (int)__umul64hi(x, (uint64_t)(i + 1));
                const int t = b[i];
                b[i] = b[j];
                b[j] = t;
            }
        }
    __syncthreads();
    if (in_smem)
        for (long long p = threadIdx.x; p < total; p += blockDim.x) dst[p] = q[p];
}

cudaError_t launch_perms_trials(int32_t *out, int R, int n, uint64_t seed, uint64_t target,
                                uint64_t stage, uint64_t iter, uint64_t s_first, int n_perm,
                                int mode, cudaStream_t st)
{
    if (n_perm <= 0) return cudaSuccess;
    if (R < 1 || n < 1 || (mode != 0 && mode != 1) || (long long)R * n >= (1LL << 31))
        return cudaErrorInvalidValue;
    static bool attr_done[kAttrDevices] = {};
    {
        const cudaError_t e =
            smem_attr_once(reinterpret_cast<const void *>(&fisher_yates_trials_kernel),
                           200 * 1024, attr_done);
        if (e != cudaSuccess) return e;
    }
    const size_t whole = (size_t)R * n * sizeof(int32_t);
    size_t smem;
    int in_smem = 0;
    if (mode == 0) {
        smem = (size_t)R * sizeof(int32_t);
        if (smem > 200 * 1024) return cudaErrorInvalidValue;
    } else {
        in_smem = whole <= 200 * 1024;
        smem = in_smem ? whole : 0;
    }
    fisher_yates_trials_kernel<<<n_perm, 256, smem, st>>>(out, R, n, seed, target, stage, iter,
                                                          s_first, mode, in_smem);
    return cudaGetLastError();
}

cudaError_t launch_perms_multi(const PermJob *jobs, int n_jobs, long long total, int max_n,
                               cudaStream_t st)
{
    if (n_jobs <= 0 || total <= 0) return cudaSuccess;
    if (total > 0x7fffffffLL) return cudaErrorInvalidValue;
    static bool attr_done[kAttrDevices] = {};
    {
        const cudaError_t e =
            smem_attr_once(reinterpret_cast<const void *>(&fisher_yates_multi_kernel),
                           200 * 1024, attr_done);
        if (e != cudaSuccess) return e;
    }
    if (max_n <= 65535) {
        // every job shuffles in 16 bits (2 bytes per point), one warp per CTA
        fisher_yates_multi_kernel<<<(unsigned)total, 32, (size_t)max_n * 2, st>>>(jobs, n_jobs,
                                                                                 max_n, 0);
        return cudaGetLastError();
    }
    const int smem_n = max_n * 4 <= 200 * 1024 ? max_n : 0;
    // larger permutations keep their draws beside the permutation when that
    // fits; jobs of at most 65535 points still shuffle in 16 bits
    const int jb_ok = smem_n > 0 && (size_t)max_n * 8 <= 200 * 1024;
    fisher_yates_multi_kernel<<<(unsigned)total, 256, (size_t)smem_n * (jb_ok ? 8 : 4), st>>>(
        jobs, n_jobs, smem_n, jb_ok);
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
