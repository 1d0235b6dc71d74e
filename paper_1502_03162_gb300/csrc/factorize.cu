// factorize.cu -- the alternating minimisation of Algorithm 1 on the GPU, in FP32 with
// double-float (error-free) accumulation where the normal equations need it.
//
// HRIR matrix X (column i = the HRIR x_i of direction i, length M), resonance f of length
// Lf = M - Lg + 1, non-negative reflections G (row i = g_i, length Lg), and the banded
// Toeplitz matrix F~ of f (Eq. 12), so that column i of F~ G^T is f * g_i.  Each round:
//
//  (1) resonance solve (Eqs. 9-11 restricted to the Lf free parameters of Eq. 13): the
//      normal equations A f = b of min_f sum_i ||x_i - f * g_i||^2 with
//          A[l][l'] = a[|l - l'|],  a[d] = sum_i sum_j g_i[j] g_i[j + d]   (symmetric Toeplitz)
//          b[l]     = sum_i sum_j x_i[j + l] g_i[j];
//  (2) reflection update (Eq. 4 with F = F~): F~^T F~ is the symmetric Toeplitz matrix of
//      the autocorrelation r[d] = sum_l f[l] f[l + d] (|d| < Lf), (X^T F~)_ij =
//      sum_l x_i[j + l] f[l], and
//          G_ij <- G_ij sqrt( ((X^T F~)^+_ij + [G (F~^T F~)^-]_ij) /
//                             ((X^T F~)^-_ij + [G (F~^T F~)^+]_ij) ),   Q^+- = (|Q| +- Q) / 2;
//      entries equal to 0 stay 0 (the denominator is >= G_ij ||f||^2 > 0 otherwise);
//  (3) the residual ||X - F~ G^T||_F^2 after the update (and, in the first round, before it).
//
// Kernels: fact_round_kernel, one CTA per (direction, ear): the update of one row of G, the
// row's residual, and the row's contributions to a and b for the next solve, all accumulated
// in double-float and written as per-row partials; fact_solve_kernel, one CTA per ear: the
// partials summed in row order (fixed, deterministic), the Toeplitz system solved by an FP32
// Cholesky factorisation with iterative refinement against the double-float system (so the
// solution has the accuracy of the accumulated system, not of FP32 elimination), and r of
// the new f.  No FP64 arithmetic on the device.
#include "dfloat.cuh"
#include "kernels.h"

namespace hrir {

namespace {

constexpr int kRoundThreads = 256;
constexpr int kSolveThreads = 64;

// ---- per-row kernel --------------------------------------------------------------------------
// partial layout per (ear, row): a[0..Lf), b[0..Lf), residual before, residual after
__global__ void __launch_bounds__(kRoundThreads) fact_round_kernel(const FactArgs a)
{
    extern __shared__ float fsm[];
    const int M = a.M, Lg = a.Lg, Lf = a.Lf;
    float *xs = fsm;                 // [M]
    float *gs = xs + M;              // [Lg] G row before the update
    float *gn = gs + Lg;             // [Lg] after
    float *fs = gn + Lg;             // [Lf]
    float *rs = fs + Lf;             // [Lf] autocorrelation lags of f
    __shared__ dfl red[kRoundThreads / 32];

    const int i = blockIdx.x, e = blockIdx.y, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const size_t row = (size_t)i * a.n_ears + e;
    const float *x = a.X + row * M;
    float *g = a.G + row * Lg;
    for (int m = tid; m < M; m += kRoundThreads) xs[m] = x[m];
    for (int j = tid; j < Lg; j += kRoundThreads) gs[j] = g[j];
    if (a.update || a.res_before) {
        for (int l = tid; l < Lf; l += kRoundThreads) {
            fs[l] = a.f[(size_t)e * Lf + l];
            rs[l] = a.R[(size_t)e * Lf + l];
        }
    }
    __syncthreads();
    dfl *part = reinterpret_cast<dfl *>(a.part) + ((size_t)e * a.n_dirs + i) * (2 * Lf + 2);

    // ||x - f * g||^2 for the row in gv: reconstruction and difference in double-float
    auto residual = [&](const float *gv) -> dfl {
        dfl acc = df_make(0.f);
        for (int m = tid; m < M; m += kRoundThreads) {
            dfl rec = df_make(0.f);
            const int l0 = m - (Lg - 1) > 0 ? m - (Lg - 1) : 0;
            const int l1 = m < Lf - 1 ? m : Lf - 1;
            for (int l = l0; l <= l1; ++l) rec = df_fma(rec, fs[l], gv[m - l]);
            const dfl d = df_add(df_make(xs[m]), df_neg(rec));
            acc = df_fma(acc, d.hi, d.hi);
            acc = df_fma(acc, 2.f * d.hi, d.lo);
        }
        acc = df_warp_sum(acc);
        if (lane == 0) red[warp] = acc;
        __syncthreads();
        dfl tot = red[0];
        for (int w = 1; w < kRoundThreads / 32; ++w) tot = df_add(tot, red[w]);
        __syncthreads();
        return tot;
    };

    if (a.res_before) {
        const dfl r0 = residual(gs);
        if (tid == 0) part[2 * Lf] = r0;
    }
    if (a.update) {
        for (int j = tid; j < Lg; j += kRoundThreads) {
            float gj = gs[j];
            if (gj > 0.f) {
                dfl xtf = df_make(0.f);                        // (X^T F~)_ij
                for (int l = 0; l < Lf; ++l) xtf = df_fma(xtf, xs[j + l], fs[l]);
                const float xf = df_value(xtf);
                float gp = 0.f, gm = 0.f;                      // [G (F~^T F~)^+-]_ij
                const int d0 = j - (Lf - 1) > 0 ? j - (Lf - 1) : 0;
                const int d1 = j + (Lf - 1) < Lg - 1 ? j + (Lf - 1) : Lg - 1;
                for (int jj = d0; jj <= d1; ++jj) {
                    const float r = rs[jj > j ? jj - j : j - jj];
                    const float gv = gs[jj];
                    if (r > 0.f) gp = fmaf(gv, r, gp);
                    else gm = fmaf(gv, -r, gm);
                }
                const float num = (xf > 0.f ? xf : 0.f) + gm;
                const float den = (xf < 0.f ? -xf : 0.f) + gp;
                gj = gj * sqrtf(num / den);
            }
            gn[j] = gj;
            g[j] = gj;
        }
    } else {
        for (int j = tid; j < Lg; j += kRoundThreads) gn[j] = gs[j];
    }
    __syncthreads();
    if (a.update) {
        const dfl r1 = residual(gn);
        if (tid == 0) part[2 * Lf + 1] = r1;
    }
    if (a.partials) {
        // a[d] = sum_j g[j] g[j + d], b[l] = sum_j x[j + l] g[j]: warp w takes outputs w, w + 8, ..
        for (int o = warp; o < 2 * Lf; o += kRoundThreads / 32) {
            dfl acc = df_make(0.f);
            if (o < Lf) {
                for (int j = lane; j + o < Lg; j += 32) acc = df_fma(acc, gn[j], gn[j + o]);
            } else {
                const int l = o - Lf;
                for (int j = lane; j < Lg; j += 32) acc = df_fma(acc, xs[j + l], gn[j]);
            }
            acc = df_warp_sum(acc);
            if (lane == 0) part[o] = acc;
        }
    }
}

// ---- per-ear kernel: sums, Toeplitz solve, autocorrelation ----------------------------------
__global__ void __launch_bounds__(kSolveThreads) fact_solve_kernel(const FactArgs a, int solve,
                                                                   int trace_before, int trace_after)
{
    constexpr int kMaxLf = kFactMaxLf;
    __shared__ dfl sums[2 * kMaxLf + 2];
    __shared__ float L[kMaxLf][kMaxLf + 1];      // Cholesky factor of A (FP32)
    __shared__ dfl fsol[kMaxLf];                 // solution, double-float
    __shared__ float rhs[kMaxLf];                // residual of the current solution (FP32 part)
    __shared__ float z[kMaxLf];
    const int e = blockIdx.x, tid = threadIdx.x, Lf = a.Lf;
    const int W = 2 * Lf + 2;
    const dfl *part = reinterpret_cast<const dfl *>(a.part) + (size_t)e * a.n_dirs * W;
    for (int o = tid; o < W; o += kSolveThreads) {
        dfl acc = df_make(0.f);
        for (int i = 0; i < a.n_dirs; ++i) acc = df_add(acc, part[(size_t)i * W + o]);
        sums[o] = acc;
    }
    __syncthreads();
    if (tid == 0 && a.trace) {
        if (trace_before >= 0) a.trace[(size_t)e * (a.iters + 1) + trace_before] = df_value(sums[2 * Lf]);
        if (trace_after >= 0) a.trace[(size_t)e * (a.iters + 1) + trace_after] = df_value(sums[2 * Lf + 1]);
    }
    if (!solve) return;
    const dfl *acor = sums;          // a[d]
    const dfl *bvec = sums + Lf;     // b[l]
    // Cholesky L L^T = A (FP32, from the leading parts), column by column
    for (int k = 0; k < Lf; ++k) {
        if (tid == 0) {
            float d = acor[0].hi;
            for (int p = 0; p < k; ++p) d = fmaf(-L[k][p], L[k][p], d);
            L[k][k] = sqrtf(d > 0.f ? d : 0.f);
        }
        __syncthreads();
        for (int r = k + 1 + tid; r < Lf; r += kSolveThreads) {
            float v = acor[r - k].hi;
            for (int p = 0; p < k; ++p) v = fmaf(-L[r][p], L[k][p], v);
            L[r][k] = v / L[k][k];
        }
        __syncthreads();
    }
    for (int l = tid; l < Lf; l += kSolveThreads) {
        fsol[l] = df_make(0.f);
        rhs[l] = df_value(bvec[l]);
    }
    __syncthreads();
    // iterative refinement: solve L L^T z = rhs in FP32, f += z, rhs = b - A f in double-float
    for (int it = 0; it < 4; ++it) {
        if (tid == 0) {
            for (int r = 0; r < Lf; ++r) {
                float v = rhs[r];
                for (int p = 0; p < r; ++p) v = fmaf(-L[r][p], z[p], v);
                z[r] = v / L[r][r];
            }
            for (int r = Lf - 1; r >= 0; --r) {
                float v = z[r];
                for (int p = r + 1; p < Lf; ++p) v = fmaf(-L[p][r], z[p], v);
                z[r] = v / L[r][r];
            }
        }
        __syncthreads();
        for (int l = tid; l < Lf; l += kSolveThreads) fsol[l] = df_add(fsol[l], df_make(z[l]));
        __syncthreads();
        for (int l = tid; l < Lf; l += kSolveThreads) {
            dfl r = bvec[l];
            for (int p = 0; p < Lf; ++p) {
                const dfl av = acor[p > l ? p - l : l - p];
                r = df_fma_df(r, df_neg(av), fsol[p].hi);
                r = df_fma_df(r, df_neg(av), fsol[p].lo);
            }
            rhs[l] = df_value(r);
        }
        __syncthreads();
    }
    float *fo = a.f_out + (size_t)e * Lf;
    for (int l = tid; l < Lf; l += kSolveThreads) fo[l] = df_value(fsol[l]);
    __syncthreads();
    // autocorrelation lags of the new (FP32) f for the next update
    for (int d = tid; d < Lf; d += kSolveThreads) {
        dfl acc = df_make(0.f);
        for (int l = 0; l + d < Lf; ++l) acc = df_fma(acc, fo[l], fo[l + d]);
        a.R_out[(size_t)e * Lf + d] = df_value(acc);
    }
}

// s_e = ||f_e|| into a.scale[e], then f_e <- f_e / s_e (one warp per ear)
__global__ void fact_scale_f_kernel(const FactArgs a)
{
    const int e = blockIdx.x, lane = threadIdx.x;
    float *f = a.f_out + (size_t)e * a.Lf;
    dfl ss = df_make(0.f);
    for (int l = lane; l < a.Lf; l += 32) ss = df_fma(ss, f[l], f[l]);
    ss = df_warp_sum(ss);
    const float s = sqrtf(df_value(ss));
    __syncwarp();
    if (lane == 0) a.scale[e] = s > 0.f ? s : 1.f;
    if (s > 0.f)
        for (int l = lane; l < a.Lf; l += 32) f[l] = f[l] / s;
}

// G_e <- G_e s_e (F~ G^T unchanged by the pair of rescalings)
__global__ void fact_scale_g_kernel(const FactArgs a)
{
    const int64_t n = (int64_t)a.n_dirs * a.n_ears * a.Lg;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int e = (int)((k / a.Lg) % a.n_ears);
        a.G[k] = a.G[k] * a.scale[e];
    }
}

}  // namespace

size_t fact_round_smem_bytes(int M, int Lg, int Lf)
{
    return (size_t)(M + 2 * Lg + 2 * Lf) * sizeof(float);
}

cudaError_t launch_fact_round(const FactArgs &a, int update, int res_before, int partials, cudaStream_t st)
{
    FactArgs b = a;
    b.update = update;
    b.res_before = res_before;
    b.partials = partials;
    const size_t smem = fact_round_smem_bytes(a.M, a.Lg, a.Lf);
    cudaError_t e = cudaFuncSetAttribute(fact_round_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fact_round_kernel<<<dim3((unsigned)a.n_dirs, (unsigned)a.n_ears), kRoundThreads, smem, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_fact_solve(const FactArgs &a, int solve, int trace_before, int trace_after, cudaStream_t st)
{
    fact_solve_kernel<<<(unsigned)a.n_ears, kSolveThreads, 0, st>>>(a, solve, trace_before, trace_after);
    return cudaGetLastError();
}

cudaError_t launch_fact_normalise(const FactArgs &a, cudaStream_t st)
{
    fact_scale_f_kernel<<<(unsigned)a.n_ears, 32, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t n = (int64_t)a.n_dirs * a.n_ears * a.Lg;
    const int64_t blocks = (n + 255) / 256;
    fact_scale_g_kernel<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace hrir
