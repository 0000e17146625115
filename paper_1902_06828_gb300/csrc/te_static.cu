// cmi_ksg_static: the KSG estimate of cmi_ksg for callers that must not
// allocate device memory.
//
// Some callers cannot call cudaMalloc: a host framework that has already
// reserved the whole device for its own pool allocator (a new allocation
// would fail or fragment that pool), a serving process that budgets every
// byte of device memory up front, or a latency-critical loop where the
// implicit device synchronisation of cudaMalloc / cudaFree is not acceptable.
// This entry point therefore allocates nothing.  All the scratch memory it
// needs (surrogate permutations, digamma table, launch descriptors,
// accumulators and keys) lives in one file-scope __device__ array of
// kStaticScratchBytes that every GPU which loads this library holds until the
// process exits.
//
// Host code never uses the array's name as an address: the first call on a
// device (with that device current) resolves the array's device address with
// cudaGetSymbolAddress and keeps it for later calls on that device.  No call
// may be made while its stream is being captured into a CUDA graph: every
// call copies from host staging buffers and ends by synchronising the stream,
// and neither is allowed during capture.
//
// Every call shares the array and leaves its contents behind; the parts that
// must start at zero (the key accumulators) are cleared by each call.  Two
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race on the array and give wrong results; callers must serialise
// them.  Host-side staging uses static buffers too, so calls must also not
// overlap on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "te_runtime.h"

using namespace teksg;

namespace {

constexpr size_t kStaticScratchBytes = TE_STATIC_SCRATCH_BYTES;   // 32 MiB per device
constexpr int kStaticMaxN = 1 << 20;                 // points (host digamma staging)
constexpr int kStaticMaxSurr = TE_STATIC_MAX_SURR;   // surrogates per call
constexpr int kStaticMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

void *g_scratch_addr[kStaticMaxDevices];   // device address of g_static_scratch, per device
bool g_ready[kStaticMaxDevices];

// host staging (static: no heap allocation during a call)
int64_t g_q_host[kStaticMaxN + 2];
int g_q_host_n = -1;
unsigned char g_desc_host[sizeof(GroupDesc) + (kStaticMaxSurr + 1) * sizeof(MemberDesc) +
                          4 * TE_MAX_DIMS + 64];
int64_t g_keys_host[2 * (kStaticMaxSurr + 1)];

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
static_assert(sizeof(GroupDesc) <= 256, "the documented scratch size counts 256 bytes for it");
static_assert(sizeof(MemberDesc) == 24, "the documented scratch size counts 24 bytes per member");

te_status setup_device(int dev)
{
    if (dev < 0 || dev >= kStaticMaxDevices) return TE_EINVAL;
    if (g_ready[dev]) return TE_OK;
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return TE_ECUDA;
    if (ksg_prepare_attributes() != cudaSuccess) return TE_ECUDA;
    g_scratch_addr[dev] = p;
    g_ready[dev] = true;
    return TE_OK;
}

}  // namespace

extern "C" te_status cmi_ksg_static(const float *series_dev, int32_t n_proc, int32_t T,
                                    const te_var *x, int32_t dx, const te_var *y, int32_t dy,
                                    const te_var *z, int32_t dz, const te_ksg_params *p,
                                    void *cuda_stream, double *out_cmi, int64_t *out_key)
{
    if (!series_dev || !p || !out_cmi) return TE_EINVAL;
    if (n_proc < 1 || T < 2 || (long long)n_proc * T >= (1LL << 31)) return TE_EINVAL;
    if (!x || dx < 1 || !y || dy < 1 || dz < 0 || (dz > 0 && !z)) return TE_EINVAL;
    if (dx + dy + dz > TE_MAX_DIMS) return TE_EINVAL;
    if (p->k < 1 || p->k > TE_MAX_K || p->theiler < 0 || p->n_surr < 0) return TE_EINVAL;
    if (p->max_lag < 0 || p->max_lag >= T) return TE_EINVAL;
    const int N = T - p->max_lag;
    const int S = p->n_surr;
    if ((long long)N - 1 - 2LL * p->theiler < p->k) return TE_EINVAL;
    const te_var *vs[3] = {x, y, z};
    const int ds[3] = {dx, dy, dz};
    for (int a = 0; a < 3; ++a)
        for (int d = 0; d < ds[a]; ++d)
            if (vs[a][d].proc < 0 || vs[a][d].proc >= n_proc || vs[a][d].lag < 0 ||
                vs[a][d].lag > p->max_lag)
                return TE_EINVAL;
    if (N > kStaticMaxN || S > kStaticMaxSurr) return TE_EINVAL;

    // scratch layout: Q | perms | group | members | cols | acc | keys
    const size_t q_off = 0;
    const size_t perm_off = align256(q_off + (size_t)(N + 2) * 8);
    const size_t grp_off = align256(perm_off + (size_t)S * N * 4);
    const size_t mem_off = align256(grp_off + sizeof(GroupDesc));
    const size_t col_off = align256(mem_off + (size_t)(S + 1) * sizeof(MemberDesc));
    const size_t acc_off = align256(col_off + (size_t)(dx + dy + dz) * 4);
    const size_t key_off = align256(acc_off + (size_t)(S + 1) * 16);
    const size_t total = align256(key_off + (size_t)(S + 1) * 16);
    if (total > kStaticScratchBytes) return TE_EINVAL;   // beyond the static scratch
    const size_t desc_bytes = sizeof(GroupDesc) + (size_t)(S + 1) * sizeof(MemberDesc) +
                              (size_t)(dx + dy + dz) * 4;
    if (desc_bytes > sizeof(g_desc_host)) return TE_EINTERNAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return TE_ECUDA;
    // the series must be device memory of the current device: a pointer into
    // another GPU's memory would be read remotely or fault
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, series_dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return TE_EINVAL;
    }
    if ((pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) ||
        pa.device != dev)
        return TE_EINVAL;
    te_status st = setup_device(dev);
    if (st) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    unsigned char *sc = (unsigned char *)g_scratch_addr[dev];
    int64_t *q = (int64_t *)(sc + q_off);
    int32_t *perms = (int32_t *)(sc + perm_off);
    unsigned long long *acc = (unsigned long long *)(sc + acc_off);
    long long *keys = (long long *)(sc + key_off);

    // digamma table (host double-double, same arithmetic as the context path)
    if (g_q_host_n < N + 1) {
        digamma_q_fill(N + 1, g_q_host);
        g_q_host_n = N + 1;
    }
    if (cudaMemcpyAsync(q, g_q_host, (size_t)(N + 2) * 8, cudaMemcpyHostToDevice, stream) !=
        cudaSuccess)
        return TE_ECUDA;
    if (launch_perms(perms, N, N, p->seed, p->stream_tag, 0, 0, 1, S, stream) != cudaSuccess)
        return TE_ECUDA;

    // one group in time order, members = identity + S surrogates
    const bool dx1 = dx == 1;
    KsgVariant v = dx1 ? KsgVariant{32, p->k == 4 ? 4 : 0, kLaneThreads}
                       : KsgVariant{2, p->k == 4 ? 4 : 0, 128};
    const int qsz = dx1 ? kLaneQueries : 128;
    int jt;
    size_t smem;
    if (dx1) {
        jt = 256;
        if (N < jt) jt = std::max(64, (N + 63) & ~63);
        smem = ksg_lane_smem_bytes(dy + dz, jt);
    } else {
        const int rows_t = dy + dz + v.m * dx, rows_q = rows_t;
        long long room = 40 * 1024 - 4LL * rows_q * 128 - 64 - 8 * 8 * 128;
        jt = (int)std::min<long long>((room / (4LL * rows_t + 8)) & ~7LL, 2048);
        if (jt < 64) {
            room = 190 * 1024 - 4LL * rows_q * 128 - 64 - 8 * 8 * 128;
            jt = (int)std::min<long long>((room / (4LL * rows_t + 8)) & ~7LL, 2048);
        }
        if (jt < 8) return TE_EINVAL;
        jt = std::min(jt, (N + 7) & ~7);
        smem = ksg_smem_bytes(rows_t, rows_q, jt, 128);
    }
    GroupDesc gd{};
    gd.base = series_dev;
    gd.N = N;
    gd.k = p->k;
    gd.theiler = p->theiler;
    gd.dy = dy;
    gd.dz = dz;
    gd.dx = dx;
    gd.ycol = dx;
    gd.zcol = dx + dy;
    gd.member_begin = 0;
    gd.n_members = S + 1;
    gd.n_qtiles = (N + qsz - 1) / qsz;
    gd.n_mblocks = (S + 1 + v.m - 1) / v.m;
    gd.item_begin = 0;
    unsigned char *h = g_desc_host;
    std::memcpy(h, &gd, sizeof gd);
    MemberDesc *hm = (MemberDesc *)(h + sizeof(GroupDesc));
    for (int s = 0; s <= S; ++s) {
        hm[s].perm = s == 0 ? nullptr : perms + (size_t)(s - 1) * N;
        hm[s].xcol = 0;
        hm[s].out = s;
        hm[s].xsorted = nullptr;
    }
    int *hc = (int *)(hm + S + 1);
    int c = 0;
    for (int d = 0; d < dx; ++d) hc[c++] = x[d].proc * T + p->max_lag - x[d].lag;
    for (int d = 0; d < dy; ++d) hc[c++] = y[d].proc * T + p->max_lag - y[d].lag;
    for (int d = 0; d < dz; ++d) hc[c++] = z[d].proc * T + p->max_lag - z[d].lag;
    if (cudaMemcpyAsync(sc + grp_off, h, sizeof(GroupDesc), cudaMemcpyHostToDevice, stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(sc + mem_off, hm, (size_t)(S + 1) * sizeof(MemberDesc),
                        cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaMemcpyAsync(sc + col_off, hc, (size_t)c * 4, cudaMemcpyHostToDevice, stream) !=
            cudaSuccess ||
        cudaMemsetAsync(acc, 0, (size_t)(S + 1) * 16, stream) != cudaSuccess)
        return TE_ECUDA;

    KsgLaunch L{};
    L.groups = (const GroupDesc *)(sc + grp_off);
    L.n_groups = 1;
    L.members = (const MemberDesc *)(sc + mem_off);
    L.cols = (const int *)(sc + col_off);
    L.q = q;
    L.acc = acc;
    L.dbg_out = -1;
    L.jt = jt;
    L.work = nullptr;
    const long long items = (long long)gd.n_qtiles * gd.n_mblocks;
    if (launch_ksg(L, v, items, dx1, smem, stream) != cudaSuccess) return TE_ECUDA;
    if (launch_finalize(acc, keys, S + 1, stream) != cudaSuccess) return TE_ECUDA;

    int64_t *kh = g_keys_host;
    if (cudaMemcpyAsync(kh, keys, (size_t)(S + 1) * 16, cudaMemcpyDeviceToHost, stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return TE_ECUDA;
    if (out_key) std::memcpy(out_key, kh, (size_t)(S + 1) * 16);
    const double psi_k = std::ldexp((double)g_q_host[p->k], -52);
    const double dN = 4503599627370496.0 * (double)N;
    for (int s = 0; s <= S; ++s) {
        const __int128 K = ((__int128)kh[2 * s] << 64) | (__int128)(uint64_t)kh[2 * s + 1];
        out_cmi[s] = psi_k + (double)K / dN;
    }
    return TE_OK;
}
