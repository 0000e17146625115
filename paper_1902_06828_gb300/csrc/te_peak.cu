// te_alu_peak: measured ceiling of the KSG kernel's counted operations.
//
// The KSG kernel is bound by plain ALU issue, and its roofline counts three
// operations per evaluated kNN-pass member-pair (subtract, max with d_YZ,
// compare) and seven per count-pass member-pair (subtract, three compares,
// three increments).  These probes run exactly those instruction patterns
// from registers -- the same per-lane shape as the kernel: 4 query points, 2
// members, 8-point blocks -- at full occupancy with no memory traffic, so
// their rate is what the GPU can do with that instruction mix.  A third probe
// measures plain FP32 add issue (the 4 x 32 lanes per SM per clock limit).
#include <cuda_runtime.h>

#include "te_runtime.h"

using namespace teksg;

namespace {

constexpr int kProbeThreads = 256;

// Every probe block takes a loop-carried value v (advanced by one add of a
// runtime delta per block), so no part of it is loop-invariant: the PTX
// assembler would otherwise hoist the distance arithmetic out of the loop.

// kNN pass, one member, one 8-point block: D_u = max(|v - x_u|, d_YZ,u), the
// minimum of the eight, one compare against the member's threshold (taken
// only when the block holds a closer point; the insertion itself is the rare
// path and is left out).  24 counted operations in 26 instructions.
__device__ __forceinline__ void probe_knn8(float &v, float delta, const float (&xv)[8],
                                           const float (&dv)[8], float &thr)
{
    asm volatile(
        "{\n\t.reg .f32 d0, d1, d2, d3, d4, d5, d6, d7;\n\t.reg .pred p;\n\t"
        "add.f32 %1, %1, %2;\n\t"
        "sub.f32 d0, %1, %3;\n\tabs.f32 d0, d0;\n\tmax.f32 d0, d0, %11;\n\t"
        "sub.f32 d1, %1, %4;\n\tabs.f32 d1, d1;\n\tmax.f32 d1, d1, %12;\n\t"
        "sub.f32 d2, %1, %5;\n\tabs.f32 d2, d2;\n\tmax.f32 d2, d2, %13;\n\t"
        "sub.f32 d3, %1, %6;\n\tabs.f32 d3, d3;\n\tmax.f32 d3, d3, %14;\n\t"
        "sub.f32 d4, %1, %7;\n\tabs.f32 d4, d4;\n\tmax.f32 d4, d4, %15;\n\t"
        "sub.f32 d5, %1, %8;\n\tabs.f32 d5, d5;\n\tmax.f32 d5, d5, %16;\n\t"
        "sub.f32 d6, %1, %9;\n\tabs.f32 d6, d6;\n\tmax.f32 d6, d6, %17;\n\t"
        "sub.f32 d7, %1, %10;\n\tabs.f32 d7, d7;\n\tmax.f32 d7, d7, %18;\n\t"
        "min.f32 d0, d0, d1;\n\tmin.f32 d2, d2, d3;\n\tmin.f32 d4, d4, d5;\n\t"
        "min.f32 d6, d6, d7;\n\tmin.f32 d0, d0, d2;\n\tmin.f32 d4, d4, d6;\n\t"
        "min.f32 d0, d0, d4;\n\t"
        "setp.lt.f32 p, d0, %0;\n\t@p mov.f32 %0, d0;\n\t}"
        : "+f"(thr), "+f"(v)
        : "f"(delta), "f"(xv[0]), "f"(xv[1]), "f"(xv[2]), "f"(xv[3]), "f"(xv[4]), "f"(xv[5]),
          "f"(xv[6]), "f"(xv[7]), "f"(dv[0]), "f"(dv[1]), "f"(dv[2]), "f"(dv[3]), "f"(dv[4]),
          "f"(dv[5]), "f"(dv[6]), "f"(dv[7]));
}

// Count pass, one member, one 8-point block: per point the kernel's strict
// range counts (the subtract for d_X, three compares, three predicated
// increments), with v as both the query's X value and its radius.  56 counted
// operations in 57 instructions.
__device__ __forceinline__ void probe_count8(float &v, float delta, const float (&xv)[8],
                                             const float (&zv)[8], const float (&yv)[8],
                                             float &cz, float &cxz, float &cyz)
{
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        if (u == 0)
            asm volatile("add.f32 %0, %0, %1;" : "+f"(v) : "f"(delta));
        asm volatile(
            "{\n\t.reg .f32 dc;\n\t.reg .pred pz, pxz, pyz;\n\t"
            "sub.f32 dc, %3, %4;\n\tabs.f32 dc, dc;\n\t"
            "setp.lt.f32 pz, %5, %3;\n\t"
            "setp.lt.and.f32 pxz, dc, %3, pz;\n\t"
            "setp.lt.f32 pyz, %6, %3;\n\t"
            "@pz add.f32 %0, %0, 0f3F800000;\n\t"
            "@pxz add.f32 %1, %1, 0f3F800000;\n\t"
            "@pyz add.f32 %2, %2, 0f3F800000;\n\t}"
            : "+f"(cz), "+f"(cxz), "+f"(cyz)
            : "f"(v), "f"(xv[u]), "f"(zv[u]), "f"(yv[u]));
    }
}

// Eight independent FP32 add chains: the issue limit of plain FMA-pipe work.
__device__ __forceinline__ void probe_fadd8(float (&a)[8], float b)
{
    asm volatile(
        "add.f32 %0, %0, %8;\n\tadd.f32 %1, %1, %8;\n\tadd.f32 %2, %2, %8;\n\t"
        "add.f32 %3, %3, %8;\n\tadd.f32 %4, %4, %8;\n\tadd.f32 %5, %5, %8;\n\t"
        "add.f32 %6, %6, %8;\n\tadd.f32 %7, %7, %8;"
        : "+f"(a[0]), "+f"(a[1]), "+f"(a[2]), "+f"(a[3]), "+f"(a[4]), "+f"(a[5]), "+f"(a[6]),
          "+f"(a[7])
        : "f"(b));
}

// kind 0: kNN-pass mix, kind 1: count-pass mix, kind 2: FP32 adds.  Per
// iteration each thread evaluates 4 query points x 2 members x 8 points
// (64 member-pairs) or 64 adds.  Inputs come from the thread index, so no
// two lanes hold the same values; delta is 0 at run time but unknown to the
// compiler; the results go to sink so nothing is dead.
template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) alu_probe_kernel(int iters, float delta,
                                                                  float *sink)
{
    const float base = 1e-3f * (float)(threadIdx.x + 7 * blockIdx.x);
    float xv[2][8], zv[8], yv[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        xv[0][u] = base + 0.11f * u;
        xv[1][u] = base - 0.07f * u;
        zv[u] = 0.05f * u;
        yv[u] = 0.06f * u + 0.01f;
    }
    float xq[4][2], st[4][2][3];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            xq[a][q] = base + 0.3f * a - 0.2f * q;
            st[a][q][0] = st[a][q][1] = st[a][q][2] = KIND == 0 ? 1.0f : 0.0f;
        }
    float fa[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) fa[u] = base + u;
    for (int it = 0; it < iters; ++it) {
        if (KIND == 0) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int q = 0; q < 2; ++q) probe_knn8(xq[a][q], delta, xv[q], yv, st[a][q][0]);
        } else if (KIND == 1) {
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int q = 0; q < 2; ++q)
                    probe_count8(xq[a][q], delta, xv[q], zv, yv, st[a][q][0], st[a][q][1],
                                 st[a][q][2]);
        } else {
#pragma unroll
            for (int r = 0; r < 8; ++r) probe_fadd8(fa, 1e-7f);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int q = 0; q < 2; ++q) s += st[a][q][0] + st[a][q][1] + st[a][q][2];
#pragma unroll
    for (int u = 0; u < 8; ++u) s += fa[u];
    sink[blockIdx.x * kProbeThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" te_status te_alu_peak(te_ctx *ctx, int32_t kind, double *out_ops_per_s)
{
    if (!ctx) return TE_EINVAL;
    try {
        ctx->err.clear();
        if (!out_ops_per_s) return fail(ctx, TE_EINVAL, "out_ops_per_s is NULL");
        if (kind < 0 || kind > 2) return fail(ctx, TE_EINVAL, "kind must be 0, 1 or 2");
        CK(cudaSetDevice(ctx->device), "cudaSetDevice");
        int sms = 0, per_sm = 0;
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device),
           "cudaDeviceGetAttribute");
        const void *fn = kind == 0   ? (const void *)&alu_probe_kernel<0>
                         : kind == 1 ? (const void *)&alu_probe_kernel<1>
                                     : (const void *)&alu_probe_kernel<2>;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kProbeThreads, 0),
           "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        const int blocks = sms * (per_sm > 0 ? per_sm : 1);
        te_status st;
        if ((st = ensure_dev(ctx, ctx->ws_dbg, (size_t)blocks * kProbeThreads * 4))) return st;
        float *sink = (float *)ctx->ws_dbg.p;
        // counted operations per thread and iteration: 64 member-pairs x 3
        // (kNN pass) or x 7 (count pass), or 64 adds
        const double ops_it = kind == 0 ? 64.0 * 3 : kind == 1 ? 64.0 * 7 : 64.0;
        auto launch = [&](int iters) {
            if (kind == 0)
                alu_probe_kernel<0><<<blocks, kProbeThreads, 0, ctx->stream>>>(iters, 0.0f, sink);
            else if (kind == 1)
                alu_probe_kernel<1><<<blocks, kProbeThreads, 0, ctx->stream>>>(iters, 0.0f, sink);
            else
                alu_probe_kernel<2><<<blocks, kProbeThreads, 0, ctx->stream>>>(iters, 0.0f, sink);
            return cudaGetLastError();
        };
        CK(launch(64), "probe launch");   // warm-up
        // grow the loop until one launch takes at least 20 ms
        int iters = 1024;
        float ms = 0.f;
        for (int round = 0; round < 12; ++round) {
            CK(cudaEventRecord(ctx->ev_a, ctx->stream), "cudaEventRecord");
            CK(launch(iters), "probe launch");
            CK(cudaEventRecord(ctx->ev_b, ctx->stream), "cudaEventRecord");
            CK(cudaEventSynchronize(ctx->ev_b), "cudaEventSynchronize");
            CK(cudaEventElapsedTime(&ms, ctx->ev_a, ctx->ev_b), "cudaEventElapsedTime");
            ctx->stats.launches += 1;
            if (ms >= 20.f || iters >= (1 << 24)) break;
            iters *= 4;
        }
        ctx->stats.launches += 1;
        *out_ops_per_s = ops_it * (double)iters * (double)blocks * kProbeThreads / (ms * 1e-3);
        return TE_OK;
    } catch (...) {
        return fail(ctx, TE_EINTERNAL, "unexpected C++ exception");
    }
}
