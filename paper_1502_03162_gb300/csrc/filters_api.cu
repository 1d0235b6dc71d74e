// filters_api.cu -- host side of the filter-production calls of the C ABI (include/hrir.h):
// Algorithm 1's alternating minimisation (hrir_factorize) and its L1-NNLS fine-tune with the
// identity or window transform (hrir_sparsify).
#include <algorithm>
#include <cmath>

#include "api_internal.h"

using namespace hrir;
using namespace hrir_host;

namespace {

int grow_fact_ws(hrir_ctx *ctx, size_t need)
{
    return grow(ctx, &ctx->d_fact_ws, &ctx->fact_ws_bytes, need);
}

GemmArgs product(int64_t M, int N, int K, const float *A, int64_t sam, int64_t sak, const float *B, int64_t sbk,
                 int64_t sbn, float *Z, int k_chunk)
{
    GemmArgs g{};
    g.M = M;
    g.N = N;
    g.K = K;
    g.A = A;
    g.sam = sam;
    g.sak = sak;
    g.B = B;
    g.sbk = sbk;
    g.sbn = sbn;
    g.k_chunk = k_chunk;
    g.Z = Z;
    g.ldz = N;
    return g;
}

// Z = sum over k of A(m, k) B(k, n) with K split over `splits` chunks whose partial products
// (in part) are added in chunk order
int split_product(hrir_ctx *ctx, GemmArgs g, int splits, float *part, cudaStream_t st)
{
    float *Z = g.Z;
    g.k_chunk = (int)round_up((g.K + splits - 1) / splits, 16);
    splits = (g.K + g.k_chunk - 1) / g.k_chunk;
    g.Z = part;
    HRIR_CUDA_TRY(ctx, launch_gemm_tc(3, false, false, g, splits, ctx->d_status, st));
    HRIR_CUDA_TRY(ctx, launch_split_reduce(splits, (int)g.M, g.N, part, Z, st));
    return HRIR_OK;
}

}  // namespace

extern "C" int hrir_factorize(hrir_ctx *ctx, int n_dirs, int n_ears, int hrir_len, int refl_len, const float *X,
                              float *G, float *f, float *trace, int iters, int normalise, void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    const int M = hrir_len, Lg = refl_len, Lf = hrir_len - refl_len + 1, N = n_dirs;
    if (N < 1 || n_ears < 1 || n_ears > 2 || Lg < 1 || Lg > 1024 || Lf < 1 || Lf > kFactMaxLf || iters < 1)
        return fail(ctx, HRIR_EINVAL,
                    "bad sizes (n_dirs=%d n_ears=%d hrir_len=%d refl_len=%d iters=%d; need 1 <= n_ears <= 2, "
                    "1 <= refl_len <= 1024, 1 <= hrir_len - refl_len + 1 <= %d)",
                    n_dirs, n_ears, hrir_len, refl_len, iters, kFactMaxLf);
    if (!X || !G || !f) return fail(ctx, HRIR_EINVAL, "NULL X, G or f");
    if (((uintptr_t)X | (uintptr_t)G | (uintptr_t)f | (uintptr_t)trace) % 4)
        return fail(ctx, HRIR_EINVAL, "X, G, f and trace must be 4-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    HRIR_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    // split-K for the K = n_dirs products: enough CTAs for every SM, at most 64 chunks
    const int64_t tiles = ((Lg + gemm_tc_tile_rows() - 1) / gemm_tc_tile_rows()) *
                          ((Lg + gemm_tc_tile_cols() - 1) / gemm_tc_tile_cols());
    const int splits = (int)std::max<int64_t>(1, std::min<int64_t>(64, std::min<int64_t>(
                                                         (2 * ctx->num_sms + tiles - 1) / tiles, (N + 15) / 16)));
    // workspace (floats, then doubles)
    const size_t nPart = (size_t)splits * M * Lg, nP = (size_t)Lg * Lg, nB = (size_t)M * Lg;
    const size_t nNL = (size_t)N * Lg;
    const size_t n_float = nPart + nP + nB + nB + 2 * nP + 3 * nNL + 2 * (size_t)kFactMaxLf + 4;
    const size_t n_double = (size_t)fact_residual_blocks(N) + 2 * (size_t)kFactMaxLf;
    const size_t off_d = round_up((int64_t)(n_float * sizeof(float)), 256);
    int rc = grow_fact_ws(ctx, off_d + n_double * sizeof(double));
    if (rc) return rc;
    float *ws = static_cast<float *>(ctx->d_fact_ws);
    float *part = ws, *P = part + nPart, *Bm = P + nP, *Ft = Bm + nB, *Qp = Ft + nB, *Qm = Qp + nP;
    float *C = Qm + nP, *GQp = C + nNL, *GQm = GQp + nNL, *fc = GQm + nNL, *rc_ = fc + kFactMaxLf;
    float *tr_scratch = rc_ + kFactMaxLf;
    double *wd = reinterpret_cast<double *>(static_cast<unsigned char *>(ctx->d_fact_ws) + off_d);
    double *res_part = wd, *da = res_part + fact_residual_blocks(N), *db = da + kFactMaxLf;
    const int64_t ldx = (int64_t)n_ears * M, ldg = (int64_t)n_ears * Lg;

    KernelTimer kt(ctx, HRIR_K_FILTERS, st);
    for (int e = 0; e < n_ears; ++e) {
        const float *Xe = X + (size_t)e * M;
        float *Ge = G + (size_t)e * Lg;
        float *tr = trace ? trace + (size_t)e * (iters + 1) : nullptr;
        // the resonance of the current G: A f = b from P = G^T G and B = X^T G (Eqs. 9-11, 13)
        auto solve = [&]() -> int {
            int r = split_product(ctx, product(Lg, Lg, N, Ge, 1, ldg, Ge, ldg, 1, P, 0), splits, part, st);
            if (r) return r;
            r = split_product(ctx, product(M, Lg, N, Xe, 1, ldx, Ge, ldg, 1, Bm, 0), splits, part, st);
            if (r) return r;
            HRIR_CUDA_TRY(ctx, launch_fact_diag(P, Lg, Bm, Lg, Lg, Lf, da, db, st));
            HRIR_CUDA_TRY(ctx, launch_fact_solve(da, db, Lf, fc, rc_, ctx->d_status, st));
            return HRIR_OK;
        };
        if ((rc = solve())) return rc;
        for (int t = 0; t < iters; ++t) {
            // F~ of f_t and the two parts of F~^T F~; C = X F~, G Q+, G Q- (Eq. 4's products)
            HRIR_CUDA_TRY(ctx, launch_fact_build(fc, rc_, M, Lg, Lf, Ft, Qp, Qm, st));
            HRIR_CUDA_TRY(ctx, launch_gemm_tc(3, false, false, product(N, Lg, M, Xe, ldx, 1, Ft, Lg, 1, C, M), 1,
                                              ctx->d_status, st));
            HRIR_CUDA_TRY(ctx, launch_gemm_tc(3, false, false, product(N, Lg, Lg, Ge, ldg, 1, Qp, Lg, 1, GQp, Lg), 1,
                                              ctx->d_status, st));
            HRIR_CUDA_TRY(ctx, launch_gemm_tc(3, false, false, product(N, Lg, Lg, Ge, ldg, 1, Qm, Lg, 1, GQm, Lg), 1,
                                              ctx->d_status, st));
            if (t == 0)
                HRIR_CUDA_TRY(ctx, launch_fact_residual(Xe, ldx, Ge, ldg, fc, N, M, Lg, Lf, res_part,
                                                        tr ? tr : tr_scratch, st));
            HRIR_CUDA_TRY(ctx, launch_fact_update(Ge, ldg, C, GQp, GQm, N, Lg, st));
            HRIR_CUDA_TRY(ctx, launch_fact_residual(Xe, ldx, Ge, ldg, fc, N, M, Lg, Lf, res_part,
                                                    tr ? tr + t + 1 : tr_scratch, st));
            if (t + 1 < iters && (rc = solve())) return rc;
        }
        HRIR_CUDA_TRY(ctx, cudaMemcpyAsync(f + (size_t)e * Lf, fc, (size_t)Lf * sizeof(float),
                                           cudaMemcpyDeviceToDevice, st));
        if (normalise) HRIR_CUDA_TRY(ctx, launch_fact_scale(f + (size_t)e * Lf, Lf, Ge, ldg, N, Lg, st));
    }
    kt.done();
    return HRIR_OK;
}

extern "C" int hrir_sparsify(hrir_ctx *ctx, int n_dirs, int n_ears, int hrir_len, int refl_len,
                             const float *X, const float *f, float lam, float sigma, float thresh,
                             float *G, int32_t *nnz, void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    const int Lf = hrir_len - refl_len + 1;
    if (n_dirs < 1 || n_ears < 1 || n_ears > 2 || refl_len < 1 || Lf < 1 || Lf > kSparsifyMaxLf)
        return fail(ctx, HRIR_EINVAL, "bad sizes (n_dirs=%d n_ears=%d hrir_len=%d refl_len=%d)",
                    n_dirs, n_ears, hrir_len, refl_len);
    if (!(lam >= 0.f) || !std::isfinite(lam) || !std::isfinite(sigma) || !(thresh >= 0.f) ||
        !std::isfinite(thresh))
        return fail(ctx, HRIR_EINVAL, "lambda and thresh must be finite and >= 0, sigma finite");
    if (!X || !f || !G) return fail(ctx, HRIR_EINVAL, "NULL X, f or G");
    if (((uintptr_t)X | (uintptr_t)G | (uintptr_t)f | (uintptr_t)nnz) % 4)
        return fail(ctx, HRIR_EINVAL, "X, f, G and nnz must be 4-byte aligned");
    int cap = std::min(refl_len, 128);
    while (cap > 8 && sparsify_smem_bytes(hrir_len, refl_len, Lf, cap) > 220 * 1024) cap -= 8;
    if (sparsify_smem_bytes(hrir_len, refl_len, Lf, cap) > 220 * 1024)
        return fail(ctx, HRIR_EINVAL, "reflection filters too long for the shared-memory solver");
    cudaStream_t st = (cudaStream_t)stream;
    HRIR_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    int rc = grow_fact_ws(ctx, 2 * (size_t)n_ears * refl_len * Lf * sizeof(float));
    if (rc) return rc;
    SparsifyArgs a{};
    a.n_dirs = n_dirs;
    a.n_ears = n_ears;
    a.M = hrir_len;
    a.Lg = refl_len;
    a.Lf = Lf;
    a.cap = cap;
    a.X = X;
    a.f = f;
    a.lam = lam;
    a.inv_sigma2 = sigma > 0.f ? 1.f / (sigma * sigma) : 0.f;
    a.thresh = thresh;
    a.tol = 1e-6f;
    a.q = static_cast<float *>(ctx->d_fact_ws);
    a.G = G;
    a.nnz = nnz;
    a.status = ctx->d_status;
    KernelTimer kt(ctx, HRIR_K_FILTERS, st);
    HRIR_CUDA_TRY(ctx, launch_sparsify(a, st));
    kt.done();
    return HRIR_OK;
}
