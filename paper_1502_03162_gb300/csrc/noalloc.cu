// noalloc.cu -- hrir_render_batch_noalloc: the batch render of hrir_render_batch with its
// partial-sum scratch held in a fixed, file-scope device array instead of the context's
// growable workspace, so the call itself allocates nothing.
//
// The scratch is kNoAllocScratchBytes (32 MiB) of device memory.  This file holds no kernel,
// so the array sits in a module of its own; under CUDA's lazy module loading (the default)
// that module is loaded, and its 32 MiB reserved, on the first call made on a device, when
// the array's address is looked up.  From then on the device keeps the array until the
// process exits.  Host code must not pass the array's name to a kernel (on the host it is
// only a stand-in symbol); its device address is fetched once per device with
// cudaGetSymbolAddress, with that device current, and cached.
#include <mutex>

#include "api_internal.h"

using namespace hrir;
using namespace hrir_host;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 128;

static __device__ __align__(256) float g_noalloc_partial[kNoAllocScratchBytes / sizeof(float)];

std::mutex g_scratch_mu;
float *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on ctx->device (that device must be current).
int scratch_address(hrir_ctx *ctx, float **out)
{
    if (ctx->device < 0 || ctx->device >= kMaxDevices)
        return fail(ctx, HRIR_EINVAL, "device ordinal %d out of range for the fixed scratch", ctx->device);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[ctx->device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();   // do not leave the error for the next launch check to report
            return fail(ctx, e == cudaErrorMemoryAllocation ? HRIR_ENOMEM : HRIR_ECUDA,
                        "cudaGetSymbolAddress of the fixed scratch failed: %s",
                        cudaGetErrorString(e));
        }
        g_scratch_addr[ctx->device] = static_cast<float *>(p);
    }
    *out = g_scratch_addr[ctx->device];
    return HRIR_OK;
}

}  // namespace

extern "C" int hrir_render_batch_noalloc(hrir_ctx *ctx, int n_src, int64_t len, int64_t src_ld,
                                         hrir_dtype dt, const void *src, const int32_t *dir,
                                         hrir_mode mode, int full, float *out, int64_t out_ld,
                                         void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    if (!ctx->loaded) return fail(ctx, HRIR_ESTATE, "no filters loaded");
    if (n_src < 0 || len < 0) return fail(ctx, HRIR_EINVAL, "negative n_src or len");
    if (dt != HRIR_F32 && dt != HRIR_BF16 && dt != HRIR_F16)
        return fail(ctx, HRIR_EINVAL, "unknown dtype %d", (int)dt);
    if (mode != HRIR_SPARSE && mode != HRIR_DENSE)
        return fail(ctx, HRIR_EINVAL, "hrir_render_batch_noalloc supports HRIR_SPARSE and HRIR_DENSE");
    const int64_t out_len = full ? (len > 0 ? len + ctx->hrir_len - 1 : 0) : len;
    if (out_len == 0) return HRIR_OK;
    if (!out || out_ld < out_len)
        return fail(ctx, HRIR_EINVAL, "out is NULL or out_ld < %lld", (long long)out_len);
    cudaStream_t st = (cudaStream_t)stream;
    HRIR_CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    float *scratch = nullptr;
    int rc = scratch_address(ctx, &scratch);
    if (rc) return rc;
    if (n_src == 0) {
        HRIR_CUDA_TRY(ctx, cudaMemset2DAsync(out, (size_t)out_ld * 4, 0, (size_t)out_len * 4, 2, st));
        return HRIR_OK;
    }
    const size_t es = dtype_size(dt);
    if (!src || !dir) return fail(ctx, HRIR_EINVAL, "NULL src or dir");
    if (src_ld < len || ((uintptr_t)src % 16) || ((src_ld * (int64_t)es) % 16))
        return fail(ctx, HRIR_EINVAL,
                    "src must be 16-byte aligned with src_ld >= len and src_ld*elem_size %% 16 == 0");
    if (len > (int64_t)1 << 31) return fail(ctx, HRIR_EINVAL, "len must be < 2^31");

    // Every partial slot the reduction reads is written by the mixing kernel of this same
    // call, so nothing in the shared scratch has to be cleared first.  The kernels are not
    // timed (timing would create CUDA events).
    MixJob j;
    j.n_src = n_src;
    j.len = len;
    j.src_ld = src_ld;
    j.dt = (int)dt;
    j.src = src;
    j.dir = dir;
    j.sparse = mode == HRIR_SPARSE;
    j.table = j.sparse ? ctx->d_sparse : reinterpret_cast<const unsigned char *>(ctx->d_dense);
    j.n_dirs = ctx->n_dirs;
    j.res = j.sparse ? ctx->d_res : nullptr;
    j.out_len = out_len;
    j.out = out;
    j.out_ld = out_ld;
    j.scratch = scratch;
    j.scratch_bytes = kNoAllocScratchBytes;
    j.timed = false;
    return mix_render(ctx, j, st);
}
