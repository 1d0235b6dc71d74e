// filters_api.cu -- host side of the filter-production call of the C ABI (include/hrir.h):
// the L1-NNLS fine-tune of Algorithm 1 with the identity or window transform (hrir_sparsify).
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
