// Internal interface of the linear-Gaussian CMI kernels (not public).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace teksg {

constexpr int kGaussMaxDims = 40;   // dx + dy + dz
constexpr int kGaussMaxX = 8;       // dx

// Columns are X (dx), then Y (dy), then Z; W = (Y, Z) has dw = dy + dz
// columns.  The value of column c at point t is base[cols[c] + t].
struct GaussArgs {
    const float *base;
    const int *cols;        // [d] device
    int N, S, dx, dy, dw, d;
    const int32_t *perms;   // [S][N] surrogate permutations of the rows of X
    // the same permutations as 16-bit rows of perm_pitch entries (a multiple
    // of 8), or nullptr: read by the tensor-core contraction when set
    const uint16_t *perms16;
    int perm_pitch;
    int w0;                 // tensor-core contraction: first W column of this pass (32 per pass)
    // tensor-core contraction inputs prepared once per call: W's B tiles
    // (split TF32, core-matrix layout, 8 KB per 32-point chunk and pass) and
    // the centred X columns in FP32, xcen[i * xcen_pitch + t] (pitch a
    // multiple of 32); gauss_tc_workspace bytes in all
    float *btile;
    float *xcen;
    int xcen_pitch;
    double *mean;           // [d]
    double *cov;            // [d][d] sample covariance, ddof = 1
    double *LW, *LZ;        // [dw][dw] lower Cholesky factors of S_WW and S_ZZ
    double *norms;          // ||L_W^-1||_F^2, ||L_Z^-1||_F^2
    double *scratch;        // [kGaussMaxDims]
    int *status;            // [0] 1: a fixed block is not positive definite;
                            // [1] 1: a tensor-core wait timed out
    double *cross;          // [S + 1][dx][dw] cross-covariance of permuted X with W
    double *out, *err;      // [S + 1] estimates and error bounds
    // the W-W block of the covariance and the factors can be another
    // estimate's with the same W (own_w = 0: covw, LW, LZ, norms point there,
    // and this estimate computes only its X rows); own_w = 1: covw = cov
    const double *covw;
    int own_w;
    double *xc;             // [dx][N] X columns centred in FP64, stored as float pairs
                            // (hi, lo) when dw <= kGaussFFMaxW (batched contraction only)
    // the contraction is split along the points: split p sums chunks
    // [p * chunks_per_split, ...) into cross_part[p][S + 1][dx][dw]
    int splits, chunks_per_split;
    double *cross_part;
};
// splits of the points for (S + 1) * dx rows of N points in the batched
// FP64 / float-float contraction (every split keeps at least one accumulation
// group)
int gauss_cross_splits(int rows, int N);
// splits of the tensor-core contraction: one FP32 accumulation group each
int gauss_tc_splits(int N);
// bytes of the tensor-core contraction's prepared inputs (btile, xcen)
size_t gauss_tc_workspace(int N, int dx, int dw);

cudaError_t gauss_launch_stats(const GaussArgs &A, cudaStream_t st);
cudaError_t gauss_launch_cross_tc(const GaussArgs &A, cudaStream_t st);
double gauss_tc_gamma();   // relative error factor of the tensor-core contraction
// relative error factor of the FP64 contraction: a sum of N FP64 products
// errs by at most gamma_N sum |x||w|, gamma_N = N u / (1 - N u), u = 2^-53
// (N + 2 for the centring roundings)
__host__ __device__ inline double gauss_f64_gamma(int N)
{
    const double nu = (double)(N + 2) * 0x1p-53;
    return nu / (1.0 - nu);
}
// estimates with dw <= kGaussFFMaxW take the float-float contraction instead:
// 3 * 2^-48 per product and at most 128^2 * 2^-48 per window of kGaussFFWindow
// 32-point chunks (2^-34 covers both), then the FP64 sums
constexpr int kGaussFFMaxW = 16;
constexpr int kGaussFFWindow = 4;
__host__ __device__ inline double gauss_batch_gamma(int N, int dw)
{
    return gauss_f64_gamma(N) + (dw <= kGaussFFMaxW ? 0x1p-34 : 0.0);
}
// the whole FP64 pipeline (means, covariance, factors, centred X columns into
// xc, FP64 contraction and its reduction, Schur complements) for n <= 65535
// estimates in one launch per kernel: estimate i's arguments at args_dev[i]
// (device) and args_host[i]
cudaError_t gauss_launch_batch_f64(const GaussArgs *args_dev, const GaussArgs *args_host, int n,
                                   cudaStream_t st);
cudaError_t gauss_launch_schur(const GaussArgs &A, double gamma, cudaStream_t st);
// keys[2i], keys[2i + 1] = order-preserving int128 (hi, lo) of v[i]; a value
// that is not finite sets *bad
cudaError_t gauss_launch_keys(const double *v, int n, long long *keys, int *bad, cudaStream_t st);

}  // namespace teksg
