// sparsify.cu -- L1-regularised non-negative least squares per (direction, ear), the
// sparsifying fine-tune of Algorithm 1 (Sec. III-D), on the GPU:
//
//     g_i = argmin_{g >= 0} ||D (F~ g - x_i)||^2 + lambda sum_j g_j                 (Eq. 14)
//
// with the resonance f fixed (F~ its banded Toeplitz matrix, Eq. 12) and D = I or the window
// transform D_W = diag(v(0), .., v(M-1)), v(m) = exp(-m^2 / sigma^2) (Eq. 16); afterwards
// entries <= thresh are set to zero (the paper discards those below 1e-4).
//
// Written as the strictly convex quadratic program  min g^T Q g - 2 c^T g, g >= 0, with
//     Q = F~^T D^2 F~  (Lg x Lg, zero outside the band |j - j'| < Lf),
//     c = F~^T D^2 x - lambda / 2,
// and solved exactly by an active-set method (the scheme of Lawson & Hanson's NNLS applied to
// the normal-equation form): starting from g = 0 and an empty support P, repeatedly add the
// index with the largest positive w = c - Q g, solve the equality-constrained problem on P,
// and, while that solution has a non-positive entry, step towards it as far as g stays
// feasible and drop the entries that reach zero.  It stops when no w_j off the support is
// positive (the KKT conditions of Eq. 14).
//
// Precision: Q and c are formed and every residual is evaluated in double-float (error-free
// transformations, dfloat.cuh); the support systems are factorised by FP32 Cholesky and
// solved with iterative refinement against the double-float system.  One CTA per problem;
// the band of Q (one per ear) is computed once by sparsify_q_kernel.
#include "dfloat.cuh"
#include "kernels.h"

namespace hrir {

namespace {

constexpr int kThreads = 128;
constexpr int kRefine = 3;

// window weight squared, d_m^2 = exp(-2 m^2 / sigma^2) (1 for D = I)
__device__ __forceinline__ float window_sq(int m, float inv_sigma2)
{
    return inv_sigma2 > 0.f ? expf(-2.f * (float)m * (float)m * inv_sigma2) : 1.f;
}

// Q band: q[e][j][d] = Q[j][j + d] = sum_m d_m^2 f[m - j] f[m - j - d], d < Lf, as two
// planes (leading parts, then trailing parts) of a double-float value
__global__ void sparsify_q_kernel(const SparsifyArgs a)
{
    const int e = blockIdx.y;
    const int n = a.Lg * a.Lf;
    const float *f = a.f + (size_t)e * a.Lf;
    float *q_hi = a.q + (size_t)e * n;
    float *q_lo = a.q + (size_t)a.n_ears * n + (size_t)e * n;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int j = k / a.Lf, d = k - j * a.Lf;
        dfl acc = df_make(0.f);
        if (j + d < a.Lg) {
            for (int m = j + d; m < j + a.Lf; ++m) {
                const float w = window_sq(m, a.inv_sigma2);
                const float p = __fmul_rn(w, f[m - j]);
                const dfl wf = {p, fmaf(w, f[m - j], -p)};
                acc = df_fma_df(acc, wf, f[m - j - d]);
            }
        }
        q_hi[k] = acc.hi;
        q_lo[k] = acc.lo;
    }
}

struct Smem {
    float *q_hi;  // [Lg][Lf] band of Q, leading parts
    float *q_lo;  // [Lg][Lf] trailing parts
    float *c_hi;  // [Lg] c, leading parts
    float *c_lo;  // [Lg] trailing parts
    float *g;     // [Lg] current iterate
    float *s;     // [Lg] support solution (entries on P)
    float *xw;    // [M] d^2 x
    float *L;     // [cap][cap + 1] Cholesky factor of Q_PP
    float *rhs;   // [cap]
    float *z;     // [cap]
    int *P;       // [cap] support (row indices of Q)
    int *inP;     // [Lg] 1 when on the support
};

// Q[j][k] from the band (symmetric; zero outside |j - k| < Lf)
__device__ __forceinline__ dfl q_at(const Smem &S, int Lf, int j, int k)
{
    const int d = k > j ? k - j : j - k;
    if (d >= Lf) return df_make(0.f);
    const int o = (j < k ? j : k) * Lf + d;
    return dfl{S.q_hi[o], S.q_lo[o]};
}

// Solve Q_PP s_P = c_P on the support P (np = |P|; all threads of the CTA call it): FP32
// Cholesky of Q_PP, then iterative refinement against the double-float system.  Writes s on P.
__device__ void solve_support(const Smem &S, int np, int Lf, int Lg, int cap)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int k = 0; k < np; ++k) {
        for (int r = k + tid; r < np; r += kThreads) {
            float v = q_at(S, Lf, S.P[r], S.P[k]).hi;
            for (int p = 0; p < k; ++p) v = fmaf(-S.L[r * (cap + 1) + p], S.L[k * (cap + 1) + p], v);
            S.rhs[r] = v;     // column k below (and at) the diagonal, before scaling
        }
        __syncthreads();
        if (tid == 0) S.L[k * (cap + 1) + k] = sqrtf(fmaxf(S.rhs[k], 1e-30f));
        __syncthreads();
        for (int r = k + 1 + tid; r < np; r += kThreads) S.L[r * (cap + 1) + k] = S.rhs[r] / S.L[k * (cap + 1) + k];
        __syncthreads();
    }
    for (int r = tid; r < np; r += kThreads) {
        S.s[S.P[r]] = 0.f;
        S.rhs[r] = __fadd_rn(S.c_hi[S.P[r]], S.c_lo[S.P[r]]);
    }
    __syncthreads();
    for (int it = 0; it <= kRefine; ++it) {
        if (warp == 0) {
            // L y = rhs, then L^T z = y (one warp: lanes split each row's dot product)
            for (int r = 0; r < np; ++r) {
                float v = 0.f;
                for (int p = lane; p < r; p += 32) v = fmaf(S.L[r * (cap + 1) + p], S.z[p], v);
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) S.z[r] = (S.rhs[r] - v) / S.L[r * (cap + 1) + r];
                __syncwarp();
            }
            for (int r = np - 1; r >= 0; --r) {
                float v = 0.f;
                for (int p = r + 1 + lane; p < np; p += 32) v = fmaf(S.L[p * (cap + 1) + r], S.z[p], v);
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) S.z[r] = (S.z[r] - v) / S.L[r * (cap + 1) + r];
                __syncwarp();
            }
        }
        __syncthreads();
        for (int r = tid; r < np; r += kThreads) S.s[S.P[r]] += S.z[r];
        __syncthreads();
        if (it == kRefine) break;
        // rhs = c_P - Q_PP s_P (double-float)
        for (int r = tid; r < np; r += kThreads) {
            const int jr = S.P[r];
            dfl acc = {S.c_hi[jr], S.c_lo[jr]};
            const int k0 = jr - (Lf - 1) > 0 ? jr - (Lf - 1) : 0;
            const int k1 = jr + (Lf - 1) < Lg - 1 ? jr + (Lf - 1) : Lg - 1;
            for (int k = k0; k <= k1; ++k)
                if (S.inP[k]) acc = df_fma_df(acc, df_neg(q_at(S, Lf, jr, k)), S.s[k]);
            S.rhs[r] = df_value(acc);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kThreads) sparsify_kernel(const SparsifyArgs a)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ float red_v[kThreads / 32];
    __shared__ int red_i[kThreads / 32];
    __shared__ int s_np, s_flag, s_arg;
    __shared__ float s_alpha;
    const int Lg = a.Lg, Lf = a.Lf, M = a.M, cap = a.cap;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    Smem S;
    {
        unsigned char *p = smraw;
        S.q_hi = reinterpret_cast<float *>(p);
        p += 4 * (size_t)Lg * Lf;
        S.q_lo = reinterpret_cast<float *>(p);
        p += 4 * (size_t)Lg * Lf;
        S.c_hi = reinterpret_cast<float *>(p);
        p += 4 * (size_t)Lg;
        S.c_lo = reinterpret_cast<float *>(p);
        p += 4 * (size_t)Lg;
        S.g = reinterpret_cast<float *>(p);
        p += 4 * (size_t)Lg;
        S.s = reinterpret_cast<float *>(p);
        p += 4 * (size_t)Lg;
        S.xw = reinterpret_cast<float *>(p);
        p += 4 * (size_t)M;
        S.L = reinterpret_cast<float *>(p);
        p += 4 * (size_t)cap * (cap + 1);
        S.rhs = reinterpret_cast<float *>(p);
        p += 4 * (size_t)cap;
        S.z = reinterpret_cast<float *>(p);
        p += 4 * (size_t)cap;
        S.P = reinterpret_cast<int *>(p);
        p += 4 * (size_t)cap;
        S.inP = reinterpret_cast<int *>(p);
    }
    const int i = blockIdx.x, e = blockIdx.y;
    const size_t row = (size_t)i * a.n_ears + e;
    const float *x = a.X + row * M;
    const float *f = a.f + (size_t)e * Lf;
    const float *qg_hi = a.q + (size_t)e * Lg * Lf;
    const float *qg_lo = a.q + (size_t)a.n_ears * Lg * Lf + (size_t)e * Lg * Lf;
    for (int k = tid; k < Lg * Lf; k += kThreads) {
        S.q_hi[k] = qg_hi[k];
        S.q_lo[k] = qg_lo[k];
    }
    for (int m = tid; m < M; m += kThreads) S.xw[m] = x[m];
    for (int j = tid; j < Lg; j += kThreads) {
        S.g[j] = 0.f;
        S.s[j] = 0.f;
        S.inP[j] = 0;
    }
    if (tid == 0) {
        s_np = 0;
        s_flag = 0;
    }
    __syncthreads();
    // c_j = sum_l d_{j+l}^2 x[j + l] f[l] - lambda / 2
    for (int j = tid; j < Lg; j += kThreads) {
        dfl acc = df_make(0.f);
        for (int l = 0; l < Lf; ++l) {
            const float w = window_sq(j + l, a.inv_sigma2);
            const float p = __fmul_rn(w, S.xw[j + l]);
            const dfl wx = {p, fmaf(w, S.xw[j + l], -p)};
            acc = df_fma_df(acc, wx, f[l]);
        }
        const dfl cj = df_add(acc, df_make(-0.5f * a.lam));
        S.c_hi[j] = cj.hi;
        S.c_lo[j] = cj.lo;
    }
    __syncthreads();
    float cmax = 0.f;
    for (int j = 0; j < Lg; ++j) cmax = fmaxf(cmax, fabsf(S.c_hi[j]));
    const float tol = a.tol * cmax;

    int outer = 0;
    const int max_outer = 4 * Lg + 8;
    const uint64_t t_start = global_timer_ns();
    while (true) {
        // w = c - Q g; the largest w_j off the support (ties: the smaller index)
        float best = -1.f;
        int best_j = -1;
        for (int j = tid; j < Lg; j += kThreads) {
            if (S.inP[j]) continue;
            dfl acc = {S.c_hi[j], S.c_lo[j]};
            const int k0 = j - (Lf - 1) > 0 ? j - (Lf - 1) : 0;
            const int k1 = j + (Lf - 1) < Lg - 1 ? j + (Lf - 1) : Lg - 1;
            for (int k = k0; k <= k1; ++k)
                if (S.g[k] != 0.f) acc = df_fma_df(acc, df_neg(q_at(S, Lf, j, k)), S.g[k]);
            const float wj = df_value(acc);
            if (wj > best) {
                best = wj;
                best_j = j;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oj = __shfl_xor_sync(0xffffffffu, best_j, o);
            if (ov > best || (ov == best && oj >= 0 && (best_j < 0 || oj < best_j))) {
                best = ov;
                best_j = oj;
            }
        }
        if (lane == 0) {
            red_v[warp] = best;
            red_i[warp] = best_j;
        }
        __syncthreads();
        if (tid == 0) {
            float bv = red_v[0];
            int bj = red_i[0];
            for (int w = 1; w < kThreads / 32; ++w)
                if (red_v[w] > bv || (red_v[w] == bv && red_i[w] >= 0 && (bj < 0 || red_i[w] < bj))) {
                    bv = red_v[w];
                    bj = red_i[w];
                }
            s_arg = (bj >= 0 && bv > tol && s_np < cap) ? bj : -1;
            if (bj >= 0 && bv > tol && s_np >= cap) s_flag = 1;    // support larger than the cap
            if (s_arg >= 0 && global_timer_ns() - t_start > kWaitLimitNs) {
                s_arg = -1;                                         // time budget spent
                s_flag = 1;
            }
            if (s_arg >= 0) {
                S.P[s_np] = s_arg;
                S.inP[s_arg] = 1;
                s_np = s_np + 1;
            }
        }
        __syncthreads();
        if (s_arg < 0 || ++outer > max_outer) break;
        // inner loop: keep the solution on P feasible
        for (int inner = 0; inner <= cap; ++inner) {
            const int np = s_np;
            solve_support(S, np, Lf, Lg, cap);
            if (tid == 0) {
                float alpha = 2.f;
                int arg = -1;
                for (int r = 0; r < np; ++r) {
                    const int j = S.P[r];
                    if (S.s[j] <= 0.f) {
                        const float t = S.g[j] / (S.g[j] - S.s[j]);
                        if (t < alpha) {
                            alpha = t;
                            arg = j;
                        }
                    }
                }
                s_alpha = alpha;
                s_arg = arg;
            }
            __syncthreads();
            if (s_arg < 0) {
                for (int r = tid; r < np; r += kThreads) S.g[S.P[r]] = S.s[S.P[r]];
                __syncthreads();
                break;
            }
            const float alpha = s_alpha;
            for (int r = tid; r < np; r += kThreads) {
                const int j = S.P[r];
                S.g[j] = fmaf(alpha, S.s[j] - S.g[j], S.g[j]);
            }
            __syncthreads();
            if (tid == 0) {
                // drop the blocking index and any other entry that reached zero
                int k = 0;
                for (int r = 0; r < np; ++r) {
                    const int j = S.P[r];
                    if (j == s_arg || S.g[j] <= 0.f) {
                        S.g[j] = 0.f;
                        S.s[j] = 0.f;
                        S.inP[j] = 0;
                    } else {
                        S.P[k++] = j;
                    }
                }
                s_np = k;
            }
            __syncthreads();
            if (s_np == 0) break;
        }
    }
    if (tid == 0 && (s_flag || outer > max_outer)) atomicOr(a.status, DEV_SOLVER);
    float *go = a.G + row * Lg;
    int kept = 0;
    for (int j = tid; j < Lg; j += kThreads) {
        const float v = S.g[j] > a.thresh ? S.g[j] : 0.f;
        go[j] = v;
        kept += v > 0.f;
    }
    if (a.nnz) {
        for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
        __syncthreads();
        if (lane == 0) red_i[warp] = kept;
        __syncthreads();
        if (tid == 0) {
            int t = 0;
            for (int w = 0; w < kThreads / 32; ++w) t += red_i[w];
            a.nnz[row] = t;
        }
    }
}

}  // namespace

size_t sparsify_smem_bytes(int M, int Lg, int Lf, int cap)
{
    return sizeof(dfl) * (size_t)Lg * (Lf + 1) + 4 * (size_t)(3 * Lg + M) +
           4 * (size_t)cap * (cap + 4) + 16;
}

cudaError_t launch_sparsify(const SparsifyArgs &a, cudaStream_t st)
{
    const int n = a.Lg * a.Lf;
    sparsify_q_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)a.n_ears), 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = sparsify_smem_bytes(a.M, a.Lg, a.Lf, a.cap);
    e = cudaFuncSetAttribute(sparsify_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    sparsify_kernel<<<dim3((unsigned)a.n_dirs, (unsigned)a.n_ears), kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace hrir
