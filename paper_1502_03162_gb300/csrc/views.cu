// views.cu -- rendering of precomputed resonance outputs to several direction sets (the order
// (y * f) * g of Eq. 2): hrir_render_precomputed.
//
// With u_{s,e} = y_s * f_e given (hrir_resonance_per_source), each view v is the mix
//     out_v,e = sum_s u_{s,e} * g_{dir_v[s], e}
// of the reflection taps alone.  The rows of u ([n_src][2][u_ld]: row 2 s + e) are rendered
// by the sparse mixing kernel as 2 n_src one-ear sources: row 2 s + e takes the one-ear
// record 2 dir_v[s] + e (ear e's taps, none for the other ear), and the reduction adds no
// resonance.
#include <algorithm>

#include "api_internal.h"

using namespace hrir;
using namespace hrir_host;

namespace {

// rows[2 s + e] = 2 dir[s] + e, or -1 (silent, flagged by the mixing kernel) for an id out of
// range
__global__ void view_rows_kernel(const int32_t *__restrict__ dir, int n_src, int n_dirs, int32_t *rows)
{
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n_src; s += gridDim.x * blockDim.x) {
        const int d = dir[s];
        const bool ok = (unsigned)d < (unsigned)n_dirs;
        rows[2 * s] = ok ? 2 * d : -1;
        rows[2 * s + 1] = ok ? 2 * d + 1 : -1;
    }
}

}  // namespace

extern "C" int hrir_render_precomputed(hrir_ctx *ctx, int n_src, int64_t len, int64_t u_ld,
                                       const float *u, int n_views, const int32_t *dir, int full,
                                       float *out, int64_t out_ld, int64_t view_ld, void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    if (!ctx->loaded) return fail(ctx, HRIR_ESTATE, "no filters loaded");
    if (n_src < 0 || len < 0 || n_views < 0) return fail(ctx, HRIR_EINVAL, "negative n_src, len or n_views");
    if (n_src > (1 << 29)) return fail(ctx, HRIR_EINVAL, "too many sources");
    const int64_t out_len = full ? (len > 0 ? len + ctx->refl_len - 1 : 0) : len;
    if (out_len == 0 || n_views == 0) return HRIR_OK;
    if (!out || out_ld < out_len || view_ld < 2 * out_ld)
        return fail(ctx, HRIR_EINVAL, "out is NULL, out_ld < %lld or view_ld < 2 out_ld", (long long)out_len);
    cudaStream_t st = (cudaStream_t)stream;
    HRIR_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    if (n_src == 0) {
        for (int v = 0; v < n_views; ++v)
            HRIR_CUDA_TRY(ctx, cudaMemset2DAsync(out + (size_t)v * view_ld, (size_t)out_ld * 4, 0,
                                              (size_t)out_len * 4, 2, st));
        return HRIR_OK;
    }
    if (!u || !dir) return fail(ctx, HRIR_EINVAL, "NULL u or dir");
    if (u_ld < len || ((uintptr_t)u % 16) || (u_ld % 4))
        return fail(ctx, HRIR_EINVAL, "u must be 16-byte aligned with u_ld >= len and u_ld %% 4 == 0");
    if (len > (int64_t)1 << 31) return fail(ctx, HRIR_EINVAL, "len must be < 2^31");
    // the rows of every view, in a workspace of the context
    const size_t need = (size_t)n_views * 2 * n_src * sizeof(int32_t);
    int rc = grow(ctx, &ctx->d_view_ws, &ctx->view_ws_bytes, need);
    if (rc) return rc;
    int32_t *rows = static_cast<int32_t *>(ctx->d_view_ws);
    for (int v = 0; v < n_views; ++v) {
        int32_t *rv = rows + (size_t)v * 2 * n_src;
        const int blocks = std::min((n_src + 255) / 256, 4096);
        view_rows_kernel<<<blocks, 256, 0, st>>>(dir + (size_t)v * n_src, n_src, ctx->n_dirs, rv);
        HRIR_CUDA_TRY(ctx, cudaGetLastError());
        MixJob j;
        j.n_src = 2 * n_src;
        j.len = len;
        j.src_ld = u_ld;
        j.dt = HRIR_F32;
        j.src = u;
        j.dir = rv;
        j.sparse = true;
        j.table = ctx->d_sparse_split;
        j.n_dirs = 2 * ctx->n_dirs;
        j.res = nullptr;
        j.out_len = out_len;
        j.out = out + (size_t)v * view_ld;
        j.out_ld = out_ld;
        rc = mix_render(ctx, j, st);
        if (rc) return rc;
    }
    return HRIR_OK;
}
