// filters_api.cu -- host side of the filter-production calls of the C ABI (include/hrir.h):
// the alternating minimisation of Algorithm 1 (hrir_factorize) and the L1-NNLS fine-tune
// with the identity or window transform (hrir_sparsify).
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

}  // namespace

extern "C" int hrir_factorize(hrir_ctx *ctx, int n_dirs, int n_ears, int hrir_len, int refl_len,
                              const float *X, float *G, float *f, float *trace, int iters,
                              int normalise, void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    const int Lf = hrir_len - refl_len + 1;
    if (n_dirs < 1 || n_ears < 1 || n_ears > 2 || refl_len < 1 || refl_len > 1024 || Lf < 1 ||
        Lf > kFactMaxLf || iters < 1)
        return fail(ctx, HRIR_EINVAL,
                    "bad sizes (n_dirs=%d n_ears=%d hrir_len=%d refl_len=%d iters=%d; need "
                    "1 <= n_ears <= 2, 1 <= refl_len <= 1024, 1 <= hrir_len - refl_len + 1 <= %d)",
                    n_dirs, n_ears, hrir_len, refl_len, iters, kFactMaxLf);
    if (!X || !G || !f) return fail(ctx, HRIR_EINVAL, "NULL X, G or f");
    if (fact_round_smem_bytes(hrir_len, refl_len, Lf) > 200 * 1024)
        return fail(ctx, HRIR_EINVAL, "filters too long for the shared-memory rows");
    cudaStream_t st = (cudaStream_t)stream;
    HRIR_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const size_t W = 2 * (size_t)Lf + 2;
    const size_t part_bytes = (size_t)n_ears * n_dirs * W * sizeof(float2);
    const size_t r_off = round_up((int64_t)part_bytes, 256);
    const size_t s_off = r_off + round_up((int64_t)n_ears * Lf * 4, 256);
    int rc = grow_fact_ws(ctx, s_off + 256);
    if (rc) return rc;
    unsigned char *ws = static_cast<unsigned char *>(ctx->d_fact_ws);
    FactArgs a{};
    a.n_dirs = n_dirs;
    a.n_ears = n_ears;
    a.M = hrir_len;
    a.Lg = refl_len;
    a.Lf = Lf;
    a.iters = iters;
    a.X = X;
    a.G = G;
    a.f = f;
    a.R = reinterpret_cast<float *>(ws + r_off);
    a.f_out = f;
    a.R_out = reinterpret_cast<float *>(ws + r_off);
    a.part = reinterpret_cast<float2 *>(ws);
    a.trace = trace;
    a.scale = reinterpret_cast<float *>(ws + s_off);
    KernelTimer kt(ctx, HRIR_K_FILTERS, st);
    // the resonance of the starting G, then `iters` rounds of (update G, residuals, partials of
    // the next system; solve for the next f)
    HRIR_CUDA_TRY(ctx, launch_fact_round(a, 0, 0, 1, st));
    HRIR_CUDA_TRY(ctx, launch_fact_solve(a, 1, -1, -1, st));
    for (int t = 0; t < iters; ++t) {
        const bool last = t == iters - 1;
        HRIR_CUDA_TRY(ctx, launch_fact_round(a, 1, t == 0, last ? 0 : 1, st));
        HRIR_CUDA_TRY(ctx, launch_fact_solve(a, last ? 0 : 1, t == 0 ? 0 : -1, t + 1, st));
    }
    if (normalise) HRIR_CUDA_TRY(ctx, launch_fact_normalise(a, st));
    kt.done();
    return HRIR_OK;
}

extern "C" int hrir_sparsify(hrir_ctx *ctx, int n_dirs, int n_ears, int hrir_len, int refl_len,
                             const float *X, const float *f, float lam, float sigma, float thresh,
                             float *G, int32_t *nnz, void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    const int Lf = hrir_len - refl_len + 1;
    if (n_dirs < 1 || n_ears < 1 || n_ears > 2 || refl_len < 1 || Lf < 1 || Lf > kFactMaxLf)
        return fail(ctx, HRIR_EINVAL, "bad sizes (n_dirs=%d n_ears=%d hrir_len=%d refl_len=%d)",
                    n_dirs, n_ears, hrir_len, refl_len);
    if (!(lam >= 0.f) || !std::isfinite(lam) || !std::isfinite(sigma) || !(thresh >= 0.f) ||
        !std::isfinite(thresh))
        return fail(ctx, HRIR_EINVAL, "lambda and thresh must be finite and >= 0, sigma finite");
    if (!X || !f || !G) return fail(ctx, HRIR_EINVAL, "NULL X, f or G");
    int cap = std::min(refl_len, 128);
    while (cap > 8 && sparsify_smem_bytes(hrir_len, refl_len, Lf, cap) > 220 * 1024) cap -= 8;
    if (sparsify_smem_bytes(hrir_len, refl_len, Lf, cap) > 220 * 1024)
        return fail(ctx, HRIR_EINVAL, "reflection filters too long for the shared-memory solver");
    cudaStream_t st = (cudaStream_t)stream;
    HRIR_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    int rc = grow_fact_ws(ctx, (size_t)n_ears * refl_len * Lf * sizeof(float2));
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
    a.q = reinterpret_cast<float2 *>(ctx->d_fact_ws);
    a.G = G;
    a.nnz = nnz;
    a.status = ctx->d_status;
    KernelTimer kt(ctx, HRIR_K_FILTERS, st);
    HRIR_CUDA_TRY(ctx, launch_sparsify(a, st));
    kt.done();
    return HRIR_OK;
}
