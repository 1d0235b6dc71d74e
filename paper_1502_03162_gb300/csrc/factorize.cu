// factorize.cu -- the small kernels of Algorithm 1's alternating minimisation on the device;
// its matrix products run on the tensor-core GEMM (mlp_gemm_tc.cu, FP32 accuracy) and are
// orchestrated by hrir_factorize (filters_api.cu).  Notation: X (N directions x M taps, the
// HRIRs as rows here), resonance f (Lf = M - Lg + 1 taps), reflections G (N x Lg, >= 0), and
// F~ (M x Lg) the banded Toeplitz matrix of f (Eq. 12), so that row i of G F~^T is f * g_i.
//
//  * fact_diag_kernel: the resonance system of Eqs. 9-11 over the Lf free parameters of
//    Eq. 13 from the products P = G^T G (Lg x Lg) and B = X^T G (M x Lg):
//        a[d] = sum_j P[j][j + d]   (d < Lf; A[l][l'] = a[|l - l'|], symmetric Toeplitz)
//        b[l] = sum_j B[j + l][j]   (l < Lf)
//    each a fixed-order sum in FP64.
//  * fact_solve_kernel: A f = b by Cholesky in FP64 (one CTA; Lf <= 64), f rounded to
//    FP32, and its autocorrelation r[d] = sum_l f[l] f[l + d] (FP64 sums of the FP32 taps),
//    which gives F~^T F~ = Toeplitz(r) (every column of F~ holds the whole of f).
//  * fact_build_kernel: F~ (M x Lg) and Q+ = max(F~^T F~, 0), Q- = max(-F~^T F~, 0) (Lg x Lg).
//  * fact_update_kernel: the multiplicative rule of Eq. 4 with F = F~,
//        G_ij <- G_ij sqrt( (C+_ij + [G Q-]_ij) / (C-_ij + [G Q+]_ij) ),  C = X F~,
//    C+- = (|C| +- C) / 2; entries equal to 0 stay 0 (the denominator is >= G_ij r[0] > 0).
//  * fact_residual_kernel + fact_residual_sum_kernel: ||X - G F~^T||_F^2 straight from the
//    definition (the convolution f * g_i per row in double-float, the differences squared and
//    summed in FP64, partials added in a fixed order).
//  * fact_scale_kernel: the final normalisation f <- f / ||f||, G <- G ||f||.
#include "dfloat.cuh"
#include "kernels.h"

namespace hrir {

namespace {

constexpr int kThreads = 256;

// fixed-order block sum of one FP64 value per thread (result in thread 0)
__device__ __forceinline__ double block_sum(double v, double *red)
{
    const int tid = threadIdx.x;
    red[tid] = v;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
    }
    const double s = red[0];
    __syncthreads();
    return s;
}

// block o < Lf: a[o]; block Lf + l: b[l]
__global__ void __launch_bounds__(kThreads) fact_diag_kernel(const float *__restrict__ P, int ldp,
                                                             const float *__restrict__ B, int ldb, int Lg,
                                                             int Lf, double *__restrict__ a,
                                                             double *__restrict__ b)
{
    __shared__ double red[kThreads];
    const int o = blockIdx.x;
    double s = 0.0;
    if (o < Lf) {
        for (int j = threadIdx.x; j + o < Lg; j += kThreads) s += (double)P[(size_t)j * ldp + j + o];
    } else {
        const int l = o - Lf;
        for (int j = threadIdx.x; j < Lg; j += kThreads) s += (double)B[(size_t)(j + l) * ldb + j];
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        if (o < Lf) a[o] = s;
        else b[o - Lf] = s;
    }
}

// Cholesky of the Lf x Lf Toeplitz system in FP64 by one CTA of kSolveThreads: right-looking
// (column k scaled in parallel, then the trailing matrix updated in parallel), the two
// triangular solves one row at a time with the later right-hand sides updated in parallel;
// f rounded to FP32 and its autocorrelation r (thread d: r[d])
constexpr int kSolveThreads = 64;
__global__ void __launch_bounds__(kSolveThreads) fact_solve_kernel(const double *__restrict__ a,
                                                                   const double *__restrict__ b, int Lf,
                                                                   float *__restrict__ f, float *__restrict__ r,
                                                                   int *status)
{
    __shared__ double A[kFactMaxLf * kFactMaxLf];   // becomes L (lower triangle)
    __shared__ double z[kFactMaxLf];
    __shared__ float fs[kFactMaxLf];
    const int tid = threadIdx.x, n2 = Lf * Lf;
    for (int q = tid; q < n2; q += kSolveThreads) {
        const int i = q / Lf, j = q - i * Lf;
        A[q] = a[i > j ? i - j : j - i];
    }
    for (int i = tid; i < Lf; i += kSolveThreads) z[i] = b[i];
    __syncthreads();
    for (int k = 0; k < Lf; ++k) {
        if (tid == 0) {
            double d = A[k * Lf + k];
            if (!(d > 0.0)) {                          // not positive definite: G carries no energy
                atomicOr(status, DEV_SOLVER);
                d = 1e-300;
            }
            A[k * Lf + k] = sqrt(d);
        }
        __syncthreads();
        const double dk = A[k * Lf + k];
        for (int i = k + 1 + tid; i < Lf; i += kSolveThreads) A[i * Lf + k] /= dk;
        __syncthreads();
        const int m = Lf - k - 1;                      // trailing (m x m), lower triangle used
        for (int q = tid; q < m * m; q += kSolveThreads) {
            const int i = k + 1 + q / m, j = k + 1 + q % m;
            if (j <= i) A[i * Lf + j] -= A[i * Lf + k] * A[j * Lf + k];
        }
        __syncthreads();
    }
    for (int i = 0; i < Lf; ++i) {                     // L z = b
        if (tid == 0) z[i] /= A[i * Lf + i];
        __syncthreads();
        for (int j = i + 1 + tid; j < Lf; j += kSolveThreads) z[j] -= A[j * Lf + i] * z[i];
        __syncthreads();
    }
    for (int i = Lf - 1; i >= 0; --i) {                // L^T f = z
        if (tid == 0) z[i] /= A[i * Lf + i];
        __syncthreads();
        for (int j = tid; j < i; j += kSolveThreads) z[j] -= A[i * Lf + j] * z[i];
        __syncthreads();
    }
    for (int i = tid; i < Lf; i += kSolveThreads) {
        fs[i] = (float)z[i];
        f[i] = fs[i];
    }
    __syncthreads();
    for (int d = tid; d < Lf; d += kSolveThreads) {
        double s = 0.0;
        for (int l = 0; l + d < Lf; ++l) s += (double)fs[l] * (double)fs[l + d];
        r[d] = (float)s;
    }
}

// F~[m][j] = f[m - j] (0 <= m - j < Lf), Qp/Qm[j][j'] = max(+-r[|j - j'|], 0) (|j - j'| < Lf)
__global__ void fact_build_kernel(const float *__restrict__ f, const float *__restrict__ r, int M, int Lg,
                                  int Lf, float *__restrict__ Ft, float *__restrict__ Qp,
                                  float *__restrict__ Qm)
{
    const int64_t nF = (int64_t)M * Lg, nQ = (int64_t)Lg * Lg;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nF + nQ;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < nF) {
            const int m = (int)(i / Lg), j = (int)(i - (int64_t)m * Lg);
            const int l = m - j;
            Ft[i] = (l >= 0 && l < Lf) ? f[l] : 0.f;
        } else {
            const int64_t q = i - nF;
            const int j = (int)(q / Lg), jj = (int)(q - (int64_t)j * Lg);
            const int d = j > jj ? j - jj : jj - j;
            const float v = d < Lf ? r[d] : 0.f;
            Qp[q] = v > 0.f ? v : 0.f;
            Qm[q] = v < 0.f ? -v : 0.f;
        }
    }
}

__global__ void fact_update_kernel(float *__restrict__ G, int64_t ldg, const float *__restrict__ C,
                                   const float *__restrict__ GQp, const float *__restrict__ GQm, int N, int Lg)
{
    const int64_t n = (int64_t)N * Lg;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / Lg;
        const int j = (int)(k - i * Lg);
        float *g = G + i * ldg + j;
        const float gv = *g;
        if (gv > 0.f) {
            const float c = C[k];
            const float num = (c > 0.f ? c : 0.f) + GQm[k];
            const float den = (c < 0.f ? -c : 0.f) + GQp[k];
            *g = gv * sqrtf(num / den);
        }
    }
}

// block x of rows: partial[x] = sum over its rows i and taps m of (x_i[m] - (f * g_i)[m])^2
constexpr int kResRows = 8;
__global__ void __launch_bounds__(kThreads) fact_residual_kernel(const float *__restrict__ X, int64_t ldx,
                                                                 const float *__restrict__ G, int64_t ldg,
                                                                 const float *__restrict__ f, int N, int M,
                                                                 int Lg, int Lf, double *__restrict__ partial)
{
    __shared__ double red[kThreads];
    __shared__ float fs[kFactMaxLf];
    for (int l = threadIdx.x; l < Lf; l += kThreads) fs[l] = f[l];
    __syncthreads();
    double s = 0.0;
    const int i0 = blockIdx.x * kResRows;
    for (int q = threadIdx.x; q < kResRows * M; q += kThreads) {
        const int i = i0 + q / M, m = q % M;
        if (i >= N) break;
        const float *g = G + (int64_t)i * ldg;
        const int l0 = m - (Lg - 1) > 0 ? m - (Lg - 1) : 0;
        const int l1 = m < Lf - 1 ? m : Lf - 1;
        dfl rec = df_make(0.f);                   // (f * g_i)[m] in double-float
        for (int l = l0; l <= l1; ++l) rec = df_fma(rec, fs[l], g[m - l]);
        const dfl d = df_add(df_make(X[(int64_t)i * ldx + m]), df_neg(rec));
        const double dd = (double)d.hi + (double)d.lo;
        s += dd * dd;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// out = sum of n partials in order (one thread per warp lane 0 .. 31 strided, then lanes in
// order), rounded to FP32
__global__ void fact_residual_sum_kernel(const double *__restrict__ partial, int n, float *__restrict__ out)
{
    __shared__ double lanes[32];
    const int t = threadIdx.x;
    double s = 0.0;
    for (int i = t; i < n; i += 32) s += partial[i];
    lanes[t] = s;
    __syncwarp();
    if (t == 0) {
        double tot = 0.0;
        for (int k = 0; k < 32; ++k) tot += lanes[k];
        *out = (float)tot;
    }
}

// s = ||f||; f <- f / s, G <- G s (one CTA per call; G rows with stride ldg)
__global__ void __launch_bounds__(kThreads) fact_scale_kernel(float *__restrict__ f, int Lf, float *__restrict__ G,
                                                              int64_t ldg, int N, int Lg)
{
    __shared__ double red[kThreads];
    double s = 0.0;
    for (int l = threadIdx.x; l < Lf; l += kThreads) s += (double)f[l] * (double)f[l];
    s = sqrt(block_sum(s, red));
    if (!(s > 0.0)) return;
    const float fs = (float)(1.0 / s), gs = (float)s;
    __syncthreads();
    for (int l = threadIdx.x; l < Lf; l += kThreads) f[l] = f[l] * fs;
    for (int64_t k = threadIdx.x; k < (int64_t)N * Lg; k += kThreads) {
        const int64_t i = k / Lg;
        G[i * ldg + (k - i * Lg)] *= gs;
    }
}

unsigned grid_for(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads < 2048 ? (n + kThreads - 1) / kThreads : 2048); }

}  // namespace

cudaError_t launch_fact_diag(const float *P, int ldp, const float *B, int ldb, int Lg, int Lf, double *a, double *b,
                             cudaStream_t st)
{
    fact_diag_kernel<<<2 * Lf, kThreads, 0, st>>>(P, ldp, B, ldb, Lg, Lf, a, b);
    return cudaGetLastError();
}

cudaError_t launch_fact_solve(const double *a, const double *b, int Lf, float *f, float *r, int *status,
                              cudaStream_t st)
{
    if (Lf < 1 || Lf > kFactMaxLf) return cudaErrorInvalidValue;
    fact_solve_kernel<<<1, kSolveThreads, 0, st>>>(a, b, Lf, f, r, status);
    return cudaGetLastError();
}

cudaError_t launch_fact_build(const float *f, const float *r, int M, int Lg, int Lf, float *Ft, float *Qp, float *Qm,
                              cudaStream_t st)
{
    fact_build_kernel<<<grid_for((int64_t)M * Lg + (int64_t)Lg * Lg), kThreads, 0, st>>>(f, r, M, Lg, Lf, Ft, Qp, Qm);
    return cudaGetLastError();
}

cudaError_t launch_fact_update(float *G, int64_t ldg, const float *C, const float *GQp, const float *GQm, int N,
                               int Lg, cudaStream_t st)
{
    fact_update_kernel<<<grid_for((int64_t)N * Lg), kThreads, 0, st>>>(G, ldg, C, GQp, GQm, N, Lg);
    return cudaGetLastError();
}

int fact_residual_blocks(int N) { return (N + kResRows - 1) / kResRows; }

cudaError_t launch_fact_residual(const float *X, int64_t ldx, const float *G, int64_t ldg, const float *f, int N,
                                 int M, int Lg, int Lf, double *partial, float *out, cudaStream_t st)
{
    if (Lf < 1 || Lf > kFactMaxLf) return cudaErrorInvalidValue;
    const int nb = fact_residual_blocks(N);
    fact_residual_kernel<<<nb, kThreads, 0, st>>>(X, ldx, G, ldg, f, N, M, Lg, Lf, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    fact_residual_sum_kernel<<<1, 32, 0, st>>>(partial, nb, out);
    return cudaGetLastError();
}

cudaError_t launch_fact_scale(float *f, int Lf, float *G, int64_t ldg, int N, int Lg, cudaStream_t st)
{
    fact_scale_kernel<<<1, kThreads, 0, st>>>(f, Lf, G, ldg, N, Lg);
    return cudaGetLastError();
}

}  // namespace hrir
