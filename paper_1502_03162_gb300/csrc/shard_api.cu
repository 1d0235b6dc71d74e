// shard_api.cu -- source sharding (Sec. II: the renderer is linear in the sources, and the
// resonance f of Eq. 2 is common to all of them): the reflection mix of a source set without
// the resonance (hrir_render_reflections), and the resonance applied once to the sum of the
// reflection mixes of several disjoint source sets (hrir_apply_resonance).  Together they
// equal hrir_render_batch on the union of the sets, up to the order of the FP32 sums.
#include "api_internal.h"

using namespace hrir;
using namespace hrir_host;

extern "C" int hrir_render_reflections(hrir_ctx *ctx, int n_src, int64_t len, int64_t src_ld, hrir_dtype dt,
                                       const void *src, const int32_t *dir, int full, float *z,
                                       int64_t z_ld, void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    if (!ctx->loaded) return fail(ctx, HRIR_ESTATE, "no filters loaded");
    if (n_src < 0 || len < 0) return fail(ctx, HRIR_EINVAL, "negative n_src or len");
    if (dt != HRIR_F32 && dt != HRIR_BF16 && dt != HRIR_F16)
        return fail(ctx, HRIR_EINVAL, "unknown dtype %d", (int)dt);
    const int64_t z_len = full ? (len > 0 ? len + ctx->refl_len - 1 : 0) : len;
    if (z_len == 0) return HRIR_OK;
    if (!z || z_ld < z_len) return fail(ctx, HRIR_EINVAL, "z is NULL or z_ld < %lld", (long long)z_len);
    cudaStream_t st = (cudaStream_t)stream;
    HRIR_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    if (n_src == 0) {
        HRIR_CUDA_TRY(ctx, cudaMemset2DAsync(z, (size_t)z_ld * 4, 0, (size_t)z_len * 4, 2, st));
        return HRIR_OK;
    }
    const size_t es = dtype_size(dt);
    if (!src || !dir) return fail(ctx, HRIR_EINVAL, "NULL src or dir");
    if (src_ld < len || ((uintptr_t)src % 16) || ((src_ld * (int64_t)es) % 16))
        return fail(ctx, HRIR_EINVAL,
                    "src must be 16-byte aligned with src_ld >= len and src_ld*elem_size %% 16 == 0");
    if (len > (int64_t)1 << 31) return fail(ctx, HRIR_EINVAL, "len must be < 2^31");
    MixJob j;
    j.n_src = n_src;
    j.len = len;
    j.src_ld = src_ld;
    j.dt = (int)dt;
    j.src = src;
    j.dir = dir;
    j.sparse = true;
    j.table = ctx->d_sparse;
    j.n_dirs = ctx->n_dirs;
    j.res = nullptr;              // the reflection taps alone
    j.out_len = z_len;
    j.out = z;
    j.out_ld = z_ld;
    return mix_render(ctx, j, st);
}

extern "C" int hrir_apply_resonance(hrir_ctx *ctx, int n_parts, int64_t z_len, int64_t part_ld, const float *z,
                                    int full, float *out, int64_t out_ld, void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    if (!ctx->loaded) return fail(ctx, HRIR_ESTATE, "no filters loaded");
    if (n_parts < 1 || z_len < 0) return fail(ctx, HRIR_EINVAL, "n_parts must be >= 1 and z_len >= 0");
    const int64_t out_len = full ? (z_len > 0 ? z_len + ctx->res_len - 1 : 0) : z_len;
    if (out_len == 0) return HRIR_OK;
    if (!z || part_ld < z_len) return fail(ctx, HRIR_EINVAL, "z is NULL or part_ld < z_len");
    if (!out || out_ld < out_len) return fail(ctx, HRIR_EINVAL, "out is NULL or out_ld < %lld", (long long)out_len);
    cudaStream_t st = (cudaStream_t)stream;
    HRIR_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    KernelTimer kt(ctx, HRIR_K_REDUCE, st);
    HRIR_CUDA_TRY(ctx, launch_parts_fir(z, n_parts, part_ld, z_len, ctx->d_res, ctx->res_len, out_len, out,
                                        out_ld, st));
    kt.done();
    return HRIR_OK;
}
