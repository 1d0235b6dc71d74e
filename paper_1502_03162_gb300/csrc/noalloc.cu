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

    const bool sparse = mode == HRIR_SPARSE;
    const MixShape shape = mix_shape(sparse ? MIX_SPARSE : MIX_DENSE);
    const int tile = shape.tile;
    const int nchunk = sparse ? ctx->sparse_nchunk : ctx->dense_nchunk;
    // history before each tile, a multiple of kMixBox so that tiles start on a source row
    const int halo = (int)round_up((int64_t)nchunk * (sparse ? kSparseSegment : shape.r), kMixBox);
    const int buf_elems = (int)round_up(halo + tile, kMixBox);
    const int rec_bytes = sparse ? ctx->sparse_rec_bytes : 2 * ctx->dense_padded * 4;
    const int64_t mix_len = sparse ? std::min<int64_t>(out_len, len + ctx->refl_len - 1) : out_len;
    const int n_tiles = (int)((mix_len + tile - 1) / tile);

    Partition part;
    part.U = (int64_t)n_tiles * n_src;
    part.P = std::min<int64_t>(ctx->num_sms, part.U);
    part.n_src = n_src;
    part.gs = mix_run_sources(ctx, sparse);
    int slots = 0;
    for (int t = 0; t < n_tiles; ++t) slots = std::max(slots, part.slots(t));
    const size_t need = (size_t)n_tiles * slots * 2 * tile * sizeof(float);
    if (need > kNoAllocScratchBytes)
        return fail(ctx, HRIR_EINVAL,
                    "this render needs %zu bytes of partial-sum scratch; the fixed array of "
                    "hrir_render_batch_noalloc holds %zu (use hrir_render_batch, or fewer sources "
                    "or samples per call)",
                    need, kNoAllocScratchBytes);

    size_t smem = 0;
    const size_t extra = sparse ? (size_t)kSparseRunAccBytes : 0;
    const int stages = pick_stages(buf_elems, (int)es, rec_bytes, extra, &smem);
    if (stages == 0) return fail(ctx, HRIR_EINVAL, "filters too long for the shared-memory pipeline");
    CUtensorMap tmap, tmap3;
    rc = make_source_map(ctx, &tmap, src, (int)dt, len, src_ld, n_src);
    if (rc) return rc;
    rc = make_source_map3(ctx, &tmap3, tmap, src, (int)dt, len, src_ld, n_src, buf_elems / kMixBox);
    if (rc) return rc;

    // Every partial slot the reduction reads is written by the mixing kernel of this same
    // call, so nothing in the shared scratch has to be cleared first.
    MixArgs a;
    a.src = src;
    a.ld = src_ld;
    a.len = len;
    a.n_src = n_src;
    a.dir = dir;
    a.n_dirs = ctx->n_dirs;
    a.table = sparse ? ctx->d_sparse : reinterpret_cast<const unsigned char *>(ctx->d_dense);
    a.rec_bytes = rec_bytes;
    a.nchunk = sparse ? ctx->sparse_nch_pad : nchunk;
    a.nseg = sparse ? ctx->sparse_nchunk : 0;
    a.halo = halo;
    a.buf_elems = buf_elems;
    a.full_rows = (int)(len / kMixBox);
    a.n_tiles = n_tiles;
    a.stages = stages;
    a.runacc_off = (int)(smem - extra);
    a.fold = mix_fold_sources(ctx);
    a.part = part;
    a.partial = scratch;
    a.slots = slots;
    a.status = ctx->d_status;
    HRIR_CUDA_TRY(ctx, launch_mix(sparse ? MIX_SPARSE : MIX_DENSE, (int)dt, tmap, tmap3, a,
                                  (int)part.P, smem, st));
    ReduceArgs r;
    r.partial = scratch;
    r.slots = slots;
    r.n_tiles = n_tiles;
    r.tile = tile;
    r.part = part;
    r.res = sparse ? ctx->d_res : nullptr;
    r.res_len = ctx->res_len;
    r.out_len = out_len;
    r.out = out;
    r.out_ld = out_ld;
    HRIR_CUDA_TRY(ctx, launch_reduce(r, st));
    return HRIR_OK;
}
