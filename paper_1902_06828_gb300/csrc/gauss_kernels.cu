// Linear-Gaussian CMI (cmi_gauss) kernels.
//
// Plug-in estimate from the sample covariance (ddof = 1) of the embedded
// variables (Methods, Vector autoregressive process: the Gaussian estimator;
// transfer entropy equals Granger causality for Gaussian variables):
//   I(X;Y|Z) = 1/2 [ln|S_XZ| + ln|S_YZ| - ln|S_Z| - ln|S_XYZ|]
//            = 1/2 [ln|Schur_X|Z| - ln|Schur_X|W|],   W = (Y, Z),
// with Schur_X|V = S_XX - S_XV S_VV^-1 S_VX.  S_XX, S_ZZ and S_WW do not
// depend on the surrogate (a permutation of the rows of X leaves S_XX
// unchanged), so they are formed and factored once in FP64; each surrogate
// only needs its cross-covariance S_XW, a contraction over the N points.
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>

#include "gauss_internal.h"

namespace teksg {

namespace {

__device__ __forceinline__ double block_sum(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int a = 0; a < (int)(blockDim.x >> 5); ++a) s += red[a];
    __syncthreads();
    return s;   // valid in thread 0
}

// column means: block d
__device__ __forceinline__ void gauss_mean_body(const GaussArgs &A, int d)
{
    __shared__ double red[32];
    const float *col = A.base + A.cols[d];
    double s = 0.0;
    for (int t = threadIdx.x; t < A.N; t += blockDim.x) s += (double)col[t];
    s = block_sum(s, red);
    if (threadIdx.x == 0) A.mean[d] = s / (double)A.N;
}

// covariance of columns (i, j), i <= j: block = pair index p
__device__ __forceinline__ void gauss_cov_body(const GaussArgs &A, int p)
{
    __shared__ double red[32];
    int i = 0;
    while (p >= A.d - i) {
        p -= A.d - i;
        ++i;
    }
    if (!A.own_w && i >= A.dx) return;   // a W-W entry: taken from covw
    const int j = i + p;
    const float *ci = A.base + A.cols[i];
    const float *cj = A.base + A.cols[j];
    const double mi = A.mean[i], mj = A.mean[j];
    double s = 0.0;
    for (int t = threadIdx.x; t < A.N; t += blockDim.x)
        s += ((double)ci[t] - mi) * ((double)cj[t] - mj);
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        const double c = s / (double)(A.N - 1);
        A.cov[i * A.d + j] = c;
        A.cov[j * A.d + i] = c;
    }
}

// In-place FP64 Cholesky of an n x n SPD matrix (row-major, lower factor);
// returns false if a pivot is not positive.
__device__ bool chol(double *a, int n, int ld)
{
    for (int j = 0; j < n; ++j) {
        double s = a[j * ld + j];
        for (int k = 0; k < j; ++k) s -= a[j * ld + k] * a[j * ld + k];
        if (!(s > 0.0)) return false;
        const double l = sqrt(s);
        a[j * ld + j] = l;
        for (int i = j + 1; i < n; ++i) {
            double t = a[i * ld + j];
            for (int k = 0; k < j; ++k) t -= a[i * ld + k] * a[j * ld + k];
            a[i * ld + j] = t / l;
        }
    }
    return true;
}

// ||L^-1||_F^2 for lower-triangular L (n x n): sum of squares of the inverse
__device__ double inv_frob2(const double *L, int n, int ld, double *col)
{
    double s = 0.0;
    for (int c = 0; c < n; ++c) {
        for (int i = 0; i < n; ++i) {
            double t = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) t -= L[i * ld + k] * col[k];
            col[i] = i < c ? 0.0 : t / L[i * ld + i];
            s += col[i] * col[i];
        }
    }
    return s;
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// In-place FP64 Cholesky of an n x n SPD matrix (n <= 64, row-major, lower
// factor) by one warp: the pivot's sum is a warp reduction of lane-strided
// partial sums, the column below it one or two rows per lane.  False (in every
// lane) if a pivot is not positive.
__device__ bool chol_warp(double *a, int n, int ld)
{
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < n; ++j) {
        double v = 0.0;
        for (int k = lane; k < j; k += 32) v += a[j * ld + k] * a[j * ld + k];
        const double s = a[j * ld + j] - warp_sum_d(v);
        if (!(s > 0.0)) return false;
        const double l = sqrt(s);
        double t[2] = {0.0, 0.0};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = j + 1 + lane + 32 * h;
            if (i < n) {
                t[h] = a[i * ld + j];
                for (int k = 0; k < j; ++k) t[h] -= a[i * ld + k] * a[j * ld + k];
            }
        }
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = j + 1 + lane + 32 * h;
            if (i < n) a[i * ld + j] = t[h] / l;
        }
        if (lane == 0) a[j * ld + j] = l;
        __syncwarp();
    }
    return true;
}

// Largest blocks the factor kernel holds: W = (Y, Z) has at most
// kGaussMaxDims - 1 columns (X has at least one) and Z at most
// kGaussMaxDims - 2 (Y has at least one).
constexpr int kFacW = kGaussMaxDims - 1;
constexpr int kFacZ = kGaussMaxDims - 2;
constexpr int kFactorThreads = 128;

// Column c's share of ||L^-1||_F^2 for lower-triangular L (n x n, row-major,
// leading dimension ld): forward substitution of L x = e_c, the entries
// x_c .. x_{n-1} kept in xs[0 .. n - c), summed in order of rows.
__device__ double inv_col_sq(const double *L, int n, int ld, int c, double *xs)
{
    double s = 0.0;
    for (int i = c; i < n; ++i) {
        double t = (i == c) ? 1.0 : 0.0;
        for (int k = c; k < i; ++k) t -= L[i * ld + k] * xs[k - c];
        const double x = t / L[i * ld + i];
        xs[i - c] = x;
        s += x * x;
    }
    return s;
}

// Factor S_WW and S_ZZ (one CTA of kFactorThreads threads).  W = the Y then Z
// columns; Z is the trailing block of W.  Warp 0 factors S_WW while warp 1
// factors S_ZZ (GB300's FP64 pipe is narrow, so the two dependent chains run
// on different schedulers); then every column of both inverses is solved by
// a thread of its own (W's columns on threads 0-63, Z's on 64-127).  Writes
// L_W, L_Z (lower, row-major, ld = dw) and ||L^-1||_F^2 of each; status[0] = 1
// if a block is not positive definite (never cleared here, so estimates
// sharing a status word accumulate it).
__device__ __forceinline__ void gauss_factor_body(const GaussArgs &A)
{
    static_assert(kFacW <= 64 && kFacZ <= 64, "one thread per column, 64 per block");
    // the factorisations run in shared memory (a warp's dependent steps would
    // otherwise wait on global memory) and the factors are written back
    __shared__ double sW[kFacW * kFacW], sZ[kFacZ * kFacZ];
    __shared__ double xW[kFacW * (kFacW + 1) / 2], xZ[kFacZ * (kFacZ + 1) / 2];
    __shared__ double s_norm[kFactorThreads / 32];
    __shared__ int s_ok[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int dx = A.dx, dw = A.dw, dy = A.dy, dz = dw - dy, d = A.d;
    for (int e = tid; e < dw * dw; e += blockDim.x) {
        const int r = e / dw, c = e % dw;
        sW[e] = c <= r ? A.cov[(dx + r) * d + dx + c] : 0.0;
    }
    for (int e = tid; e < dz * dz; e += blockDim.x) {
        const int r = e / dz, c = e % dz;
        sZ[e] = c <= r ? A.cov[(dx + dy + r) * d + dx + dy + c] : 0.0;
    }
    __syncthreads();
    if (warp == 0) {
        const bool ok = chol_warp(sW, dw, dw);
        if (lane == 0) s_ok[0] = ok;
    } else if (warp == 1) {
        const bool ok = dz > 0 ? chol_warp(sZ, dz, dz) : true;
        if (lane == 0) s_ok[1] = ok;
    }
    __syncthreads();
    if (!(s_ok[0] && s_ok[1])) {
        if (tid == 0) A.status[0] = 1;
        return;
    }
    for (int e = tid; e < dw * dw; e += blockDim.x) A.LW[e] = sW[e];
    for (int e = tid; e < dz * dz; e += blockDim.x) A.LZ[(e / dz) * dw + e % dz] = sZ[e];
    double s = 0.0;
    if (tid < 64) {
        if (tid < dw) s = inv_col_sq(sW, dw, dw, tid, xW + tid * dw - tid * (tid - 1) / 2);
    } else {
        const int c = tid - 64;
        if (c < dz) s = inv_col_sq(sZ, dz, dz, c, xZ + c * dz - c * (c - 1) / 2);
    }
    s = warp_sum_d(s);
    if (lane == 0) s_norm[warp] = s;
    __syncthreads();
    if (tid == 0) {
        A.norms[0] = s_norm[0] + s_norm[1];
        A.norms[1] = dz > 0 ? s_norm[2] + s_norm[3] : 0.0;
    }
}

// Per surrogate (one thread): Schur complements given Z and given W, their
// log-determinants, the estimate and a first-order bound on its error from
// the cross-covariance error model |dS_XW_ij| <= gamma sqrt(S_ii S_jj), whose
// squared Frobenius norm over (a, r) is gamma^2 tr(S_XX) sum_r S_rr.  One
// thread per surrogate keeps every FP64 lane busy (a warp per surrogate was
// measured slower: GB300's FP64 pipe is narrow, so idle lanes cost more than
// the dependent chain).
// One half of a surrogate's estimate: the Schur complement of X given Z
// (which = 0, the trailing dz entries of W) or given W (which = 1) from the
// factor L (lower, row-major, ld = dw), its log-determinant and the bound
// on its error.
__device__ __forceinline__ void gauss_schur_half(const GaussArgs &A, double gamma, int s,
                                                 int which, const double *L, double &ld_out,
                                                 double &bound_out)
{
    const int dx = A.dx, dw = A.dw, dy = A.dy, dz = dw - dy, d = A.d;
    const double *c = A.cross + (size_t)s * dx * dw;   // [dx][dw]
    double v[kGaussMaxDims], Sm[kGaussMaxX * kGaussMaxX], tmp[kGaussMaxDims];
    double sxx = 0.0;
    for (int a = 0; a < dx; ++a) sxx += A.cov[a * d + a];
    const int n = which == 0 ? dz : dw;
    const int off = which == 0 ? dy : 0;
    // Sm = S_XX - V^T V, V = L^-1 C_V  (column per x dim)
    for (int a = 0; a < dx; ++a)
        for (int b = 0; b < dx; ++b) Sm[a * dx + b] = A.cov[a * d + b];
    double vnorm2 = 0.0, svv = 0.0;
    double vall[kGaussMaxX * kGaussMaxDims];
    for (int r = 0; r < n; ++r) svv += A.covw[(dx + off + r) * d + dx + off + r];
    for (int a = 0; a < dx; ++a) {
        for (int r = 0; r < n; ++r) {
            double t = c[a * dw + off + r];
            for (int k = 0; k < r; ++k) t -= L[r * dw + k] * v[k];
            v[r] = t / L[r * dw + r];
            vnorm2 += v[r] * v[r];
        }
        for (int r = 0; r < n; ++r) vall[a * kGaussMaxDims + r] = v[r];
    }
    const double dcnorm2 = gamma * gamma * sxx * svv;
    for (int a = 0; a < dx; ++a)
        for (int b = 0; b < dx; ++b) {
            double t = 0.0;
            for (int r = 0; r < n; ++r) t += vall[a * kGaussMaxDims + r] * vall[b * kGaussMaxDims + r];
            Sm[a * dx + b] -= t;
        }
    if (!chol(Sm, dx, dx)) {
        ld_out = CUDART_NAN;
        bound_out = CUDART_INF;
        return;
    }
    double l = 0.0;
    for (int a = 0; a < dx; ++a) l += 2.0 * log(Sm[a * dx + a]);
    ld_out = l;
    // d ln|Sm| <= ||Sm^-1||_F ||dSm||_F,  ||dSm||_F <= 2 ||dC||_F ||L^-1||_F ||V||_F
    const double sinv = sqrt(inv_frob2(Sm, dx, dx, tmp));
    const double linv = n > 0 ? sqrt(A.norms[which == 0 ? 1 : 0]) : 0.0;
    bound_out = sinv * 2.0 * sqrt(dcnorm2) * linv * sqrt(vnorm2);
}

__device__ __forceinline__ void gauss_schur_body(const GaussArgs &A, double gamma, int s)
{
    if (s > A.S) return;
    double ld[2], bound[2];
    for (int which = 0; which < 2; ++which)
        gauss_schur_half(A, gamma, s, which, which == 0 ? A.LZ : A.LW, ld[which], bound[which]);
    A.out[s] = 0.5 * (ld[0] - ld[1]);
    // factor 2 for second-order terms
    A.err[s] = 2.0 * 0.5 * (bound[0] + bound[1]);
}

// ---------------- tensor-core cross-covariance (tcgen05, split TF32) ----------------
// cross[s][i][n] = sum_t A[(s, i)][t] B[n][t] with A[(s, i)][t] = x_i(pi_s(t))
// - mean_i (row = (surrogate s, X dim i)) and B[n][t] = w_n(t) - mean_n.  Each
// operand is split in two TF32 parts, a = a_hi + a_lo (a_hi = tf32(a), a_lo =
// tf32(a - a_hi)); the product is a_hi b_hi + a_hi b_lo + a_lo b_hi, three
// tcgen05.mma.kind::tf32 per K step, FP32 accumulation in tensor memory.
//
// What does not depend on the surrogate is prepared once per call
// (gauss_tc_prep_*): W centred in FP64 and split, already laid out as the
// MMA's B tiles (one 8 KB hi + lo tile per 32-point chunk and 32-column pass),
// and X centred in FP64 and rounded to FP32 (one rounding of 2^-24).  A CTA
// owns 128 rows and one FP32 accumulation group of at most kGaussGroup chunks:
// it copies its B tiles with cp.async.bulk, keeps the X column in shared memory
// (one X dimension and N <= kGaussColMax) or reads it through L1, gathers each
// chunk's A operand through the 16-bit permutation rows (loaded one chunk
// ahead), lets one thread issue the MMAs, and at the end reads the accumulator
// once (tcgen05.ld) into its FP64 partial-sum row.  Operands use the canonical
// K-major layout without swizzle: 8-row x 16-byte core matrices, K-adjacent
// core matrices 128 bytes apart (leading byte offset), 8-row groups 1024 bytes
// apart (stride byte offset).
constexpr int kGaussTileM = 128;
constexpr int kGaussTileN = 32;
constexpr int kGaussKC = 32;                     // points per chunk (128 bytes of TF32)
constexpr int kGaussGroup = 4;                   // chunks per FP32 accumulation group
constexpr unsigned kGaussSpinLimit = 1u << 26;   // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t to_tf32(float f)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(f));
    return r;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;   // descriptor version for this architecture
    // base offset 0, absolute LBO mode 0, layout type 0 = no swizzle
    return d;
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity)
{
    for (unsigned it = 0; it < kGaussSpinLimit; ++it) {
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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int a = 0; a < 16; ++a) v[a] = __uint_as_float(r[a]);
}

// byte offset of element (row, k) of a K-major no-swizzle tile with 8 core
// matrices (32 TF32 values) per row group
__device__ __forceinline__ uint32_t cm_offset(int row, int k)
{
    return (uint32_t)(((row >> 3) * 8 + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

constexpr int kGaussColMax = 16384;   // X column points kept in shared memory

// W's B tiles: tile (pass p, chunk c) at btile + (p * nchunks + c) * 2048
// floats, hi then lo, each in the core-matrix layout of 32 columns x 32 points
__global__ void gauss_tc_prep_w(GaussArgs A, int nchunks)
{
    const int c = blockIdx.x, pass = blockIdx.y;
    float *hb = A.btile + ((size_t)pass * nchunks + c) * 2048;
    float *lb = hb + 1024;
    for (int e = threadIdx.x; e < kGaussTileN * kGaussKC; e += blockDim.x) {
        const int n = e / kGaussKC, k = e % kGaussKC;
        const int t = c * kGaussKC + k, col = pass * kGaussTileN + n;
        float hi = 0.f, lo = 0.f;
        if (col < A.dw && t < A.N) {
            const double v = (double)A.base[A.cols[A.dx + col] + t] - A.mean[A.dx + col];
            hi = __uint_as_float(to_tf32((float)v));
            lo = __uint_as_float(to_tf32((float)(v - (double)hi)));
        }
        const uint32_t off = cm_offset(n, k) / 4;
        hb[off] = hi;
        lb[off] = lo;
    }
}

// X centred in FP64, rounded once to FP32: xcen[i * xcen_pitch + t]
__global__ void gauss_tc_prep_x(GaussArgs A)
{
    const int i = blockIdx.y;
    const float *col = A.base + A.cols[i];
    const double m = A.mean[i];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < A.xcen_pitch;
         t += gridDim.x * blockDim.x)
        A.xcen[(size_t)i * A.xcen_pitch + t] = t < A.N ? (float)((double)col[t] - m) : 0.f;
}

// 256 threads: thread (half h = tid / 128, row r = tid % 128) stages points
// 16 h .. 16 h + 15 of every chunk of row r
template <bool COLSMEM>
__global__ void __launch_bounds__(256, 2) gauss_cross_tc_kernel(GaussArgs A, int nchunks)
{
    extern __shared__ unsigned char gsm_raw[];
    unsigned char *gsm = gsm_raw + ((1024u - (smem_u32(gsm_raw) & 1023u)) & 1023u);
    float *sA_hi = reinterpret_cast<float *>(gsm);
    float *sA_lo = sA_hi + kGaussTileM * kGaussKC;
    float *sB = sA_lo + kGaussTileM * kGaussKC;          // [kGaussGroup][2][1024]
    float *scol = sB + kGaussGroup * 2048;               // [xcen_pitch] with COLSMEM
    __shared__ __align__(8) unsigned long long s_mbar_b, s_mbar_m;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int r = tid & (kGaussTileM - 1), half = tid >> 7;
    const int rows = (A.S + 1) * A.dx;
    const int m = blockIdx.x * kGaussTileM + r;   // this thread's row
    const int split = blockIdx.y;
    const bool mvalid = m < rows;
    const int ms = mvalid ? m / A.dx : 0, mi = mvalid ? m % A.dx : 0;
    const uint16_t *perm16 =
        (mvalid && ms > 0 && A.perms16) ? A.perms16 + (size_t)(ms - 1) * A.perm_pitch : nullptr;
    const int32_t *perm32 =
        (mvalid && ms > 0 && !A.perms16) ? A.perms + (size_t)(ms - 1) * A.N : nullptr;
    const float *xg = A.xcen + (size_t)mi * A.xcen_pitch;
    const int w0 = A.w0, pass = w0 / kGaussTileN;
    const int ch0 = split * A.chunks_per_split;
    const int nch = min(nchunks, ch0 + A.chunks_per_split) - ch0;   // 1 .. kGaussGroup
    const uint32_t mbar_b = smem_u32(&s_mbar_b), mbar_m = smem_u32(&s_mbar_m);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&s_tmem)),
                     "r"((uint32_t)kGaussTileN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        s_fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_b));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_m));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // this group's B tiles: one bulk copy of 8 KB per chunk
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar_b),
                     "r"((uint32_t)(nch * 8192))
                     : "memory");
        for (int c = 0; c < nch; ++c) {
            const float *src = A.btile + ((size_t)pass * nchunks + ch0 + c) * 2048;
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], "
                "8192, [%2];" ::"r"(smem_u32(sB + c * 2048)),
                "l"(reinterpret_cast<uint64_t>(src)), "r"(mbar_b)
                : "memory");
        }
    }
    if (COLSMEM) {   // the (single) X column, centred, into shared memory
        const float4 *src = reinterpret_cast<const float4 *>(A.xcen);
        float4 *dst = reinterpret_cast<float4 *>(scol);
        for (int e = tid; e < A.xcen_pitch / 4; e += 256) dst[e] = __ldg(src + e);
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) |
                           ((uint32_t)(kGaussTileN >> 3) << 17) |
                           ((uint32_t)(kGaussTileM >> 4) << 24);
    const uint32_t aHi = smem_u32(sA_hi), aLo = smem_u32(sA_lo);

    // permutation entries of this thread's half chunk: 16 indices (-1 past N)
    uint4 pv[2];
    auto load_perm = [&](int ch) {
        const int k0 = ch * kGaussKC + 16 * half;
        if (perm16) {
            const uint4 *q = reinterpret_cast<const uint4 *>(perm16 + k0);
            pv[0] = __ldg(q);
            pv[1] = __ldg(q + 1);
        }
    };
    auto index_of = [&](int ch, int k) {   // k: 0 .. 15 within the half
        const int t = ch * kGaussKC + 16 * half + k;
        if (!mvalid || t >= A.N) return -1;
        if (perm16) {
            const uint32_t wv = (&pv[k >> 3].x)[(k >> 1) & 3];
            return (int)((wv >> (16 * (k & 1))) & 0xFFFFu);
        }
        return perm32 ? perm32[t] : t;
    };
    load_perm(ch0);
    // the B tiles have landed, or the copy timed out: decided by the whole CTA
    bool failed = __syncthreads_or(!mbar_wait(mbar_b, 0)) != 0;
    uint32_t phase = 0;
    for (int c = 0; c < nch && !failed; ++c) {
        const int ch = ch0 + c;
        // stage A: this thread's half of its row's chunk, all gathers before any use
        {
            unsigned char *hb = reinterpret_cast<unsigned char *>(sA_hi);
            unsigned char *lb = reinterpret_cast<unsigned char *>(sA_lo);
            float xv[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int idx = index_of(ch, k);
                xv[k] = idx < 0 ? 0.f : (COLSMEM ? scol[idx] : __ldg(xg + idx));
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const float hi = __uint_as_float(to_tf32(xv[k]));
                const float lo = __uint_as_float(to_tf32(__fsub_rn(xv[k], hi)));
                const uint32_t off = cm_offset(r, 16 * half + k);
                *reinterpret_cast<float *>(hb + off) = hi;
                *reinterpret_cast<float *>(lb + off) = lo;
            }
        }
        if (c + 1 < nch) load_perm(ch + 1);   // in flight while the MMAs run
        // generic-proxy smem writes -> visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t bHi = smem_u32(sB + c * 2048), bLo = bHi + 4096;
#pragma unroll
            for (int q = 0; q < kGaussKC / 8; ++q) {   // K = 8 TF32 per MMA
                const uint32_t ko = q * 256;            // two core matrices along K
                const uint64_t dAh = smem_desc(aHi + ko, 128, 1024);
                const uint64_t dAl = smem_desc(aLo + ko, 128, 1024);
                const uint64_t dBh = smem_desc(bHi + ko, 128, 1024);
                const uint64_t dBl = smem_desc(bLo + ko, 128, 1024);
                mma_tf32(tmem, dAh, dBh, idesc, (c == 0 && q == 0) ? 0u : 1u);
                mma_tf32(tmem, dAh, dBl, idesc, 1u);
                mma_tf32(tmem, dAl, dBh, idesc, 1u);
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    mbar_m)
                : "memory");
        }
        // every thread waits: the MMAs have read the A tile before it is
        // restaged (and, after the last chunk, written the accumulator)
        if (!mbar_wait(mbar_m, phase)) atomicExch(&s_fail, 1);
        phase ^= 1u;
        __syncthreads();
        if (s_fail) {
            mbar_wait(mbar_m, phase ^ 1u);   // a second bounded wait before TMEM is freed
            failed = true;
        }
    }
    if (failed && tid == 0) atomicExch(A.status + 1, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!failed) {
        // warps w and w + 4 share TMEM lanes 32 (w % 4) ..; each reads 16 columns
        float v[16];
        tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + 16u * half, v);
        if (mvalid) {
            double *part = A.cross_part + ((size_t)split * rows + m) * A.dw + w0 + 16 * half;
#pragma unroll
            for (int n = 0; n < 16; ++n)
                if (w0 + 16 * half + n < A.dw) part[n] = (double)v[n];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"((uint32_t)kGaussTileN));
}

// cross = (sum of the splits' partial sums, in split order) / (N - 1)
__device__ __forceinline__ void gauss_cross_reduce_body(const GaussArgs &A, long long e)
{
    const long long total = (long long)(A.S + 1) * A.dx * A.dw;
    if (e >= total) return;
    double s = 0.0;
    for (int p = 0; p < A.splits; ++p) s += A.cross_part[(size_t)p * total + e];
    A.cross[e] = s * (1.0 / (double)(A.N - 1));
}

// FP64 cross-covariance on the CUDA cores, for estimates whose decisions must
// agree with an FP64 evaluation down to near-ties (network inference): the same
// sums as the tensor-core kernel, every product and addition in FP64.  One
// thread per row (surrogate s, X dim a) holds its dw sums in registers; the
// block stages the centred W values of each 32-point chunk in shared memory
// (read as broadcasts) and each thread gathers its permuted X values.  The
// points are split into A.splits ranges of chunks_per_split chunks (grid y),
// and the tensor-core kernel's reduction adds the splits in order.
constexpr int kF64Rows = 128;
// DW4 = dw rounded up to a multiple of 2: the W values past dw are staged as
// zeros, so the inner loop has no per-column guard (a guarded loop unrolled to
// the 32-column maximum would issue 32 FP64 FMAs per point whatever dw is).
// The X values are gathered already centred (gauss_centre_batch), so a point
// costs one FP64 FMA per column and nothing else on the FP64 pipe.
template <int DW4>
__device__ __forceinline__ void gauss_cross_f64_body(const GaussArgs &A, int bx, int by,
                                                     double (*sW)[kGaussMaxDims])
{
    const int rows = (A.S + 1) * A.dx, dw = A.dw;
    const int row = bx * kF64Rows + threadIdx.x;
    const bool live = row < rows;
    const int s = live ? row / A.dx : 0, a = live ? row % A.dx : 0;
    const int32_t *pi = s > 0 ? A.perms + (size_t)(s - 1) * A.N : nullptr;
    const double *xcol = A.xc + (size_t)a * A.N;
    double acc[DW4];
#pragma unroll
    for (int w = 0; w < DW4; ++w) acc[w] = 0.0;
    const int nchunks = (A.N + kGaussKC - 1) / kGaussKC;
    const int c0 = by * A.chunks_per_split;
    const int c1 = min(nchunks, c0 + A.chunks_per_split);
    for (int c = c0; c < c1; ++c) {
        const int t0 = c * kGaussKC, n = min(kGaussKC, A.N - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < kGaussKC * DW4; e += kF64Rows) {
            const int t = e / DW4, w = e - t * DW4;
            sW[t][w] = (t < n && w < dw)
                           ? (double)A.base[A.cols[A.dx + w] + t0 + t] - A.mean[A.dx + w]
                           : 0.0;
        }
        __syncthreads();
        if (!live) continue;
#pragma unroll 4
        for (int t = 0; t < n; ++t) {
            const int src = pi ? pi[t0 + t] : t0 + t;
            const double xv = xcol[src];
#pragma unroll
            for (int w = 0; w < DW4; ++w) acc[w] = fma(xv, sW[t][w], acc[w]);
        }
    }
    if (!live) return;
    double *dst = A.cross_part + ((size_t)by * rows + row) * dw;
#pragma unroll
    for (int w = 0; w < DW4; ++w)
        if (w < dw) dst[w] = acc[w];
}

// The same sums in float-float arithmetic on the FP32 pipe, for dw <= 16
// (GB300's FP32 pipe is far wider than its FP64 one).  X and W are centred in
// FP64 and split into two floats, v = hi + lo; a product is hi*hi exactly (the
// rounded product and its FMA residual) plus the cross terms hi*lo + lo*hi by
// FMA (lo*lo, about 2^-48 relative, is dropped); the chunk's products are
// added into a float pair by error-free two-sums, and every 32-point chunk the
// pair is flushed into an FP64 sum.  About 3 * 2^-48 relative error per
// product and n^2 * 2^-48 per 32-term window at worst.
template <int DW>
__device__ __forceinline__ void gauss_cross_ff_body(const GaussArgs &A, int bx, int by,
                                                    float2 (*sW)[kGaussMaxDims])
{
    const int rows = (A.S + 1) * A.dx, dw = A.dw;
    const int row = bx * kF64Rows + threadIdx.x;
    const bool live = row < rows;
    const int s = live ? row / A.dx : 0, a = live ? row % A.dx : 0;
    const int32_t *pi = s > 0 ? A.perms + (size_t)(s - 1) * A.N : nullptr;
    const float2 *xcol = reinterpret_cast<const float2 *>(A.xc) + (size_t)a * A.N;
    double acc[DW];
#pragma unroll
    for (int w = 0; w < DW; ++w) acc[w] = 0.0;
    const int nchunks = (A.N + kGaussKC - 1) / kGaussKC;
    const int c0 = by * A.chunks_per_split;
    const int c1 = min(nchunks, c0 + A.chunks_per_split);
    // the float pair sums kGaussFFWindow chunks (128 points) before each FP64
    // flush: the flushes run on GB300's narrow FP64 pipe
    float sh[DW], sl[DW];
#pragma unroll
    for (int w = 0; w < DW; ++w) sh[w] = sl[w] = 0.f;
    for (int c = c0; c < c1; ++c) {
        const int t0 = c * kGaussKC, n = min(kGaussKC, A.N - t0);
        __syncthreads();
        for (int e = threadIdx.x; e < kGaussKC * DW; e += kF64Rows) {
            const int t = e / DW, w = e - t * DW;
            float2 v = make_float2(0.f, 0.f);
            if (t < n && w < dw) {
                const double d = (double)A.base[A.cols[A.dx + w] + t0 + t] - A.mean[A.dx + w];
                v.x = (float)d;
                v.y = (float)(d - (double)v.x);
            }
            sW[t][w] = v;
        }
        __syncthreads();
        if (!live) continue;
        for (int t8 = 0; t8 < n; t8 += 8) {
            // eight permutation entries, then eight X values, before any is used
            int src[8];
            float2 xs[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int t = min(t8 + u, n - 1);   // past n: W is zero there
                src[u] = pi ? pi[t0 + t] : t0 + t;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) xs[u] = xcol[src[u]];
#pragma unroll
            for (int u = 0; u < 8; ++u) {   // t <= 31: t8 <= 24
                const int t = t8 + u;
                const float2 x = xs[u];
#pragma unroll
                for (int w = 0; w < DW; ++w) {
                    const float2 y = sW[t][w];
                    const float p = __fmul_rn(x.x, y.x);
                    float e = __fmaf_rn(x.x, y.x, -p);
                    e = __fmaf_rn(x.x, y.y, e);
                    e = __fmaf_rn(x.y, y.x, e);
                    const float sn = __fadd_rn(sh[w], p);
                    const float bp = __fsub_rn(sn, sh[w]);
                    const float er =
                        __fadd_rn(__fsub_rn(sh[w], __fsub_rn(sn, bp)), __fsub_rn(p, bp));
                    sl[w] = __fadd_rn(sl[w], __fadd_rn(er, e));
                    sh[w] = sn;
                }
            }
        }
        if ((c - c0) % kGaussFFWindow == kGaussFFWindow - 1 || c == c1 - 1) {
#pragma unroll
            for (int w = 0; w < DW; ++w) {
                acc[w] += (double)sh[w] + (double)sl[w];
                sh[w] = sl[w] = 0.f;
            }
        }
    }
    if (!live) return;
    double *dst = A.cross_part + ((size_t)by * rows + row) * dw;
#pragma unroll
    for (int w = 0; w < DW; ++w)
        if (w < dw) dst[w] = acc[w];
}

__device__ __forceinline__ void gauss_cross_f64_any(const GaussArgs &A, int bx, int by)
{
    __shared__ double sW[kGaussKC][kGaussMaxDims];
    float2 (*sF)[kGaussMaxDims] = reinterpret_cast<float2 (*)[kGaussMaxDims]>(sW);
    switch ((A.dw + 1) >> 1) {
    case 0:
    case 1: gauss_cross_ff_body<2>(A, bx, by, sF); return;
    case 2: gauss_cross_ff_body<4>(A, bx, by, sF); return;
    case 3: gauss_cross_ff_body<6>(A, bx, by, sF); return;
    case 4: gauss_cross_ff_body<8>(A, bx, by, sF); return;
    case 5: gauss_cross_ff_body<10>(A, bx, by, sF); return;
    case 6: gauss_cross_ff_body<12>(A, bx, by, sF); return;
    case 7: gauss_cross_ff_body<14>(A, bx, by, sF); return;
    case 8: gauss_cross_ff_body<16>(A, bx, by, sF); return;
    default: break;
    }
    switch ((A.dw + 1) >> 1) {
    case 9: gauss_cross_f64_body<18>(A, bx, by, sW); break;
    case 10: gauss_cross_f64_body<20>(A, bx, by, sW); break;
    case 11: gauss_cross_f64_body<22>(A, bx, by, sW); break;
    case 12: gauss_cross_f64_body<24>(A, bx, by, sW); break;
    case 13: gauss_cross_f64_body<26>(A, bx, by, sW); break;
    case 14: gauss_cross_f64_body<28>(A, bx, by, sW); break;
    case 15: gauss_cross_f64_body<30>(A, bx, by, sW); break;
    case 16: gauss_cross_f64_body<32>(A, bx, by, sW); break;
    case 17: gauss_cross_f64_body<34>(A, bx, by, sW); break;
    case 18: gauss_cross_f64_body<36>(A, bx, by, sW); break;
    case 19: gauss_cross_f64_body<38>(A, bx, by, sW); break;
    default: gauss_cross_f64_body<40>(A, bx, by, sW); break;
    }
}

// Order-preserving integer image of the estimates, in the (hi, lo) int128 form
// the test-statistics kernel compares: key(a) < key(b) exactly when a < b
// (sign-magnitude bits turned into two's complement order; -0 taken as +0).
// A value that is not finite (a singular Schur complement) sets *bad.
__global__ void gauss_keys_kernel(const double *v, int n, long long *keys, int *bad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = v[i] + 0.0;
    if (!isfinite(x)) *bad = 1;
    const long long b = __double_as_longlong(x);
    const long long k = b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
    keys[2 * (size_t)i] = k < 0 ? -1 : 0;
    keys[2 * (size_t)i + 1] = k;
}

__global__ void gauss_mean_kernel(GaussArgs A) { gauss_mean_body(A, blockIdx.x); }
__global__ void gauss_cov_kernel(GaussArgs A) { gauss_cov_body(A, blockIdx.x); }
__global__ void gauss_factor_kernel(GaussArgs A) { gauss_factor_body(A); }
// Single-call Schur step: the two halves of a surrogate run on a pair of
// adjacent threads (the chains are independent and GB300's FP64 pipe is
// narrow, so more threads in flight hide more of their latency), with both
// factors read from shared memory; same arithmetic as gauss_schur_body.
constexpr int kSchurThreads = 64;
__global__ void __launch_bounds__(kSchurThreads) gauss_schur_kernel(GaussArgs A, double gamma)
{
    __shared__ double sL[2][kFacW * kFacW];
    const int dw = A.dw, dz = dw - A.dy;
    for (int e = threadIdx.x; e < dw * dw; e += blockDim.x) {
        sL[0][e] = (e / dw < dz && e % dw < dz) ? A.LZ[e] : 0.0;
        sL[1][e] = A.LW[e];
    }
    __syncthreads();
    const int s = blockIdx.x * (kSchurThreads / 2) + (int)(threadIdx.x >> 1);
    const int which = threadIdx.x & 1;
    double ld = 0.0, bound = 0.0;
    if (s <= A.S) gauss_schur_half(A, gamma, s, which, sL[which], ld, bound);
    const double ld_o = __shfl_xor_sync(0xffffffffu, ld, 1);
    const double bound_o = __shfl_xor_sync(0xffffffffu, bound, 1);
    if (s <= A.S && which == 0) {
        A.out[s] = 0.5 * (ld - ld_o);
        // factor 2 for second-order terms
        A.err[s] = 2.0 * 0.5 * (bound + bound_o);
    }
}
__global__ void gauss_cross_reduce_kernel(GaussArgs A)
{
    gauss_cross_reduce_body(A, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}

// The same kernels over a batch of estimates: estimate blockIdx.z, its
// arguments read from args; blocks beyond the estimate's own grid return.
__global__ void gauss_mean_batch(const GaussArgs *args)
{
    const GaussArgs A = args[blockIdx.z];
    if ((int)blockIdx.x < A.d) gauss_mean_body(A, blockIdx.x);
}
// xc[a][t] = x_a(t) - mean_a in FP64 (as a float pair hi + lo when the
// float-float contraction takes the estimate), grid y = X dim a
__global__ void gauss_centre_batch(const GaussArgs *args)
{
    const GaussArgs A = args[blockIdx.z];
    const int a = blockIdx.y;
    if (a >= A.dx) return;
    const float *col = A.base + A.cols[a];
    const double m = A.mean[a];
    const bool ff = A.dw <= kGaussFFMaxW;   // float pairs for the float-float contraction
    double *dst = A.xc + (size_t)a * A.N;
    float2 *dst2 = reinterpret_cast<float2 *>(A.xc) + (size_t)a * A.N;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < A.N; t += gridDim.x * blockDim.x) {
        const double d = (double)col[t] - m;
        if (ff) {
            const float hi = (float)d;
            dst2[t] = make_float2(hi, (float)(d - (double)hi));
        } else {
            dst[t] = d;
        }
    }
}
__global__ void gauss_cov_batch(const GaussArgs *args)
{
    const GaussArgs A = args[blockIdx.z];
    if ((int)blockIdx.x < A.d * (A.d + 1) / 2) gauss_cov_body(A, blockIdx.x);
}
__global__ void gauss_factor_batch(const GaussArgs *args)
{
    const GaussArgs A = args[blockIdx.z];
    if (A.own_w) gauss_factor_body(A);
}
__global__ void __launch_bounds__(kF64Rows) gauss_cross_f64_batch(const GaussArgs *args)
{
    const GaussArgs A = args[blockIdx.z];
    if ((int)blockIdx.x * kF64Rows < (A.S + 1) * A.dx && (int)blockIdx.y < A.splits)
        gauss_cross_f64_any(A, blockIdx.x, blockIdx.y);
}
__global__ void gauss_cross_reduce_batch(const GaussArgs *args)
{
    const GaussArgs A = args[blockIdx.z];
    gauss_cross_reduce_body(A, blockIdx.x * (long long)blockDim.x + threadIdx.x);
}
__global__ void gauss_schur_f64_batch(const GaussArgs *args)
{
    const GaussArgs A = args[blockIdx.z];
    gauss_schur_body(A, gauss_batch_gamma(A.N, A.dw), blockIdx.x * blockDim.x + threadIdx.x);
}

}  // namespace

cudaError_t gauss_launch_batch_f64(const GaussArgs *args_dev, const GaussArgs *args_host, int n,
                                   cudaStream_t st)
{
    if (n < 1) return cudaSuccess;
    if (n > 65535) return cudaErrorInvalidValue;
    int md = 1, mrb = 1, msp = 1, ms = 1, mdx = 1;
    long long mtot = 1;
    for (int i = 0; i < n; ++i) {
        const GaussArgs &A = args_host[i];
        const int rows = (A.S + 1) * A.dx;
        if (A.splits < 1 || A.splits > 65535) return cudaErrorInvalidValue;
        md = std::max(md, A.d);
        mdx = std::max(mdx, A.dx);
        mrb = std::max(mrb, (rows + kF64Rows - 1) / kF64Rows);
        msp = std::max(msp, A.splits);
        ms = std::max(ms, A.S + 1);
        mtot = std::max(mtot, (long long)rows * A.dw);
    }
    gauss_mean_batch<<<dim3(md, 1, n), 256, 0, st>>>(args_dev);
    gauss_cov_batch<<<dim3(md * (md + 1) / 2, 1, n), 256, 0, st>>>(args_dev);
    gauss_factor_batch<<<dim3(1, 1, n), kFactorThreads, 0, st>>>(args_dev);
    gauss_centre_batch<<<dim3(8, mdx, n), 256, 0, st>>>(args_dev);
    gauss_cross_f64_batch<<<dim3(mrb, msp, n), kF64Rows, 0, st>>>(args_dev);
    gauss_cross_reduce_batch<<<dim3((unsigned)((mtot + 255) / 256), 1, n), 256, 0, st>>>(args_dev);
    gauss_schur_f64_batch<<<dim3((ms + 63) / 64, 1, n), 64, 0, st>>>(args_dev);
    return cudaGetLastError();
}

cudaError_t gauss_launch_keys(const double *v, int n, long long *keys, int *bad, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    gauss_keys_kernel<<<(n + 255) / 256, 256, 0, st>>>(v, n, keys, bad);
    return cudaGetLastError();
}

int gauss_cross_splits(int rows, int N)
{
    // enough CTAs for four resident per SM (each split ends in an FP64
    // partial-sum row that the reduction adds); the SM count is the device's
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1)
        sms = 1;
    const int tiles = (rows + kGaussTileM - 1) / kGaussTileM;
    const int groups = (N + kGaussKC * kGaussGroup - 1) / (kGaussKC * kGaussGroup);
    int splits = (4 * sms + tiles - 1) / tiles;
    return splits < 1 ? 1 : (splits > groups ? groups : splits);
}

cudaError_t gauss_launch_stats(const GaussArgs &A, cudaStream_t st)
{
    gauss_mean_kernel<<<A.d, 256, 0, st>>>(A);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    gauss_cov_kernel<<<A.d * (A.d + 1) / 2, 256, 0, st>>>(A);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    gauss_factor_kernel<<<1, kFactorThreads, 0, st>>>(A);
    return cudaGetLastError();
}

size_t gauss_tc_workspace(int N, int dx, int dw)
{
    const size_t nchunks = (size_t)(N + kGaussKC - 1) / kGaussKC;
    const size_t passes = (size_t)(dw + kGaussTileN - 1) / kGaussTileN;
    const size_t pitch = ((size_t)N + 31) & ~(size_t)31;
    return passes * nchunks * 2048 * 4 + (size_t)dx * pitch * 4;
}

int gauss_tc_splits(int N)
{
    const int nchunks = (N + kGaussKC - 1) / kGaussKC;
    return (nchunks + kGaussGroup - 1) / kGaussGroup;
}

cudaError_t gauss_launch_cross_tc(const GaussArgs &A, cudaStream_t st)
{
    const int rows = (A.S + 1) * A.dx;
    const int nchunks = (A.N + kGaussKC - 1) / kGaussKC;
    if (A.splits < 1 || A.splits > 65535 || A.chunks_per_split > kGaussGroup || !A.btile ||
        !A.xcen || (A.xcen_pitch & 31) || A.xcen_pitch < A.N ||
        (reinterpret_cast<uintptr_t>(A.btile) & 15) || (reinterpret_cast<uintptr_t>(A.xcen) & 15))
        return cudaErrorInvalidValue;
    if (A.perms16 && (A.perm_pitch < A.N || (A.perm_pitch & 7) ||
                      (reinterpret_cast<uintptr_t>(A.perms16) & 15)))
        return cudaErrorInvalidValue;
    const int passes = (A.dw + kGaussTileN - 1) / kGaussTileN;
    gauss_tc_prep_w<<<dim3(nchunks, passes), 256, 0, st>>>(A, nchunks);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    gauss_tc_prep_x<<<dim3((A.xcen_pitch + 255) / 256, A.dx), 256, 0, st>>>(A);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const bool colsmem = A.dx == 1 && A.xcen_pitch <= kGaussColMax;
    const size_t smem = 1024 + (size_t)4 * (2 * kGaussTileM * kGaussKC + kGaussGroup * 2048 +
                                            (colsmem ? A.xcen_pitch : 0));
    const void *f = colsmem ? reinterpret_cast<const void *>(&gauss_cross_tc_kernel<true>)
                            : reinterpret_cast<const void *>(&gauss_cross_tc_kernel<false>);
    static bool attr_done[64][2] = {};
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && !attr_done[dev][colsmem]) {
        if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      200 * 1024)) != cudaSuccess)
            return e;
        attr_done[dev][colsmem] = true;
    }
    // W wider than one 32-column tile: one pass per 32 columns
    for (int w0 = 0; w0 < A.dw; w0 += kGaussTileN) {
        GaussArgs P = A;
        P.w0 = w0;
        int nc = nchunks;
        void *args[] = {&P, &nc};
        e = cudaLaunchKernel(f, dim3((rows + kGaussTileM - 1) / kGaussTileM, A.splits), dim3(256),
                             args, smem, st);
        if (e != cudaSuccess) return e;
    }
    const long long total = (long long)rows * A.dw;
    gauss_cross_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(A);
    return cudaGetLastError();
}

double gauss_tc_gamma()
{
    // split products: 3 * 2^-22 relative; FP32 rounding of the centred X (one,
    // counted twice);
    // FP32 accumulation of at most 3 * kGaussKC * kGaussGroup products per
    // group, 2^-23 per addition
    return 3.0 * std::ldexp(1.0, -22) + 2.0 * std::ldexp(1.0, -24) +
           3.0 * kGaussKC * kGaussGroup * std::ldexp(1.0, -23);
}

cudaError_t gauss_launch_schur(const GaussArgs &A, double gamma, cudaStream_t st)
{
    gauss_schur_kernel<<<(A.S + 1 + kSchurThreads / 2 - 1) / (kSchurThreads / 2), kSchurThreads, 0, st>>>(
        A, gamma);
    return cudaGetLastError();
}

}  // namespace teksg
