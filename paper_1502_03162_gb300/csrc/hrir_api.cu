// hrir_api.cu -- host side of the C ABI declared in include/hrir.h: argument checking,
// filter-table construction, workspace management and kernel launches.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "api_internal.h"

using namespace hrir;

namespace hrir_host {

thread_local std::string g_create_err;

int fail(hrir_ctx *ctx, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    else g_create_err = buf;
    return code;
}

#define CUDA_TRY(ctx, call)                                                                  \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((ctx), HRIR_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));  \
    } while (0)

int grow(hrir_ctx *ctx, void **ptr, size_t *have, size_t need)
{
    if (need <= *have && *ptr) return HRIR_OK;
    if (*ptr) {
        cudaFree(*ptr);
        *ptr = nullptr;
        *have = 0;
    }
    size_t want = need + need / 8;
    if (cudaMalloc(ptr, want) != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return fail(ctx, HRIR_ENOMEM, "workspace allocation of %zu bytes failed", want);
    }
    *have = want;
    return HRIR_OK;
}

int mix_fold_sources(const hrir_ctx *ctx)
{
    return std::max(1, kFoldTerms / std::max(ctx->k_max, 1));
}

int mix_run_sources(const hrir_ctx *ctx, bool sparse)
{
    (void)ctx;
    return sparse ? kRunSources : kDenseRunSources;
}

void free_tables(hrir_ctx *ctx)
{
    cudaFree(ctx->d_sparse);
    cudaFree(ctx->d_sparse_split);
    ctx->d_sparse_split = nullptr;
    cudaFree(ctx->d_dense);
    cudaFree(ctx->d_res);
    cudaFree(ctx->d_tw);
    cudaFree(ctx->d_spec);
    cudaFree(ctx->d_tap_idx);
    cudaFree(ctx->d_tap_w);
    cudaFree(ctx->d_tap_nnz);
    ctx->d_tap_idx = nullptr;
    ctx->d_tap_w = nullptr;
    ctx->d_tap_nnz = nullptr;
    ctx->d_sparse = nullptr;
    ctx->d_dense = nullptr;
    ctx->d_res = nullptr;
    ctx->d_tw = nullptr;
    ctx->d_spec = nullptr;
    ctx->loaded = false;
}

size_t dtype_size(int dt) { return dt == HRIR_F32 ? 4 : 2; }

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Pipeline depth that fits the 227 KB shared-memory limit.
int pick_stages(int buf_elems, int elem_bytes, int rec_bytes, size_t extra, size_t *smem)
{
    for (int st = kMixMaxStages; st >= 2; --st) {
        size_t b = (size_t)round_up((int64_t)mix_smem_bytes(buf_elems, elem_bytes, rec_bytes, st), 16) + extra;
        if (b <= 227 * 1024) {
            *smem = b;
            return st;
        }
    }
    return 0;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link-time libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    }
    return fn;
}

// 2-D tensor map over the sources: dims {len, n_src}, row stride ld elements, box
// {kMixBox, 1}, out-of-range elements read as zero.
int make_source_map(hrir_ctx *ctx, CUtensorMap *m, const void *src, int dt, int64_t len,
                    int64_t ld, int n_src, int box_rows)
{
    auto fn = tensor_map_encoder();
    if (!fn) return fail(ctx, HRIR_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    const CUtensorMapDataType ty = dt == HRIR_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : dt == HRIR_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                     : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const cuuint64_t dims[2] = {(cuuint64_t)len, (cuuint64_t)n_src};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * (int64_t)dtype_size(dt))};
    const cuuint32_t box[2] = {(cuuint32_t)kMixBox, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, ty, 2, const_cast<void *>(src), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, HRIR_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return HRIR_OK;
}

int make_source_map3(hrir_ctx *ctx, CUtensorMap *m, const CUtensorMap &fallback, const void *src,
                     int dt, int64_t len, int64_t ld, int n_src, int box_rows)
{
    const int64_t rows = len / kMixBox;
    if (rows == 0) {
        *m = fallback;
        return HRIR_OK;
    }
    auto fn = tensor_map_encoder();
    if (!fn) return fail(ctx, HRIR_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    const CUtensorMapDataType ty = dt == HRIR_F32    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : dt == HRIR_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                     : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const int64_t es = (int64_t)dtype_size(dt);
    const cuuint64_t dims[3] = {(cuuint64_t)kMixBox, (cuuint64_t)rows, (cuuint64_t)n_src};
    const cuuint64_t strides[2] = {(cuuint64_t)(kMixBox * es), (cuuint64_t)(ld * es)};
    const cuuint32_t box[3] = {(cuuint32_t)kMixBox, (cuuint32_t)box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, ty, 3, const_cast<void *>(src), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, HRIR_ECUDA, "cuTensorMapEncodeTiled (3-D) failed (%d)", (int)r);
    return HRIR_OK;
}

int make_source_rows32_map(hrir_ctx *ctx, CUtensorMap *m, const float *src, int64_t rows, int64_t ld, int n_src,
                           int box_rows)
{
    auto fn = tensor_map_encoder();
    if (!fn) return fail(ctx, HRIR_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    const cuuint64_t dims[3] = {32, (cuuint64_t)rows, (cuuint64_t)n_src};
    const cuuint64_t strides[2] = {32 * 4, (cuuint64_t)(ld * 4)};
    const cuuint32_t box[3] = {32, (cuuint32_t)box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(src), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ctx, HRIR_ECUDA, "cuTensorMapEncodeTiled (32-sample rows) failed (%d)", (int)r);
    return HRIR_OK;
}

cudaEvent_t take_event(hrir_ctx *ctx)
{
    if (!ctx->free_events.empty()) {
        cudaEvent_t e = ctx->free_events.back();
        ctx->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void drop_timing_events(hrir_ctx *ctx)
{
    for (auto &p : ctx->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    ctx->pending.clear();
    for (auto e : ctx->free_events) cudaEventDestroy(e);
    ctx->free_events.clear();
}

// HRIR_FFT: overlap-save frames of P samples, hop B = P - G (G = H - 1 rounded up to 8).
int render_fft(hrir_ctx *ctx, int n_src, int64_t len, int64_t src_ld, hrir_dtype dt,
               const void *src, const int32_t *dir, int64_t out_len, float *out, int64_t out_ld,
               cudaStream_t st)
{
    const int guard = (int)round_up(ctx->hrir_len - 1, 8);
    const int hop = kFftSize - guard;
    const int64_t n_frames64 = (out_len + hop - 1) / hop;
    if (n_frames64 > (1 << 30)) return fail(ctx, HRIR_EINVAL, "too many FFT frames");
    const int n_frames = (int)n_frames64;
    const int n_pairs = (n_src + 1) / 2;
    Partition part;
    part.U = (int64_t)n_frames * n_pairs;
    part.P = std::min<int64_t>((int64_t)ctx->num_sms * kFftCtasPerSm, part.U);
    part.n_src = n_pairs;
    part.gs = kFftPairRun;
    int slots = 0;
    for (int f = 0; f < n_frames; ++f) slots = std::max(slots, part.slots(f));
    const size_t pbytes = (size_t)n_frames * slots * 2 * kFftBinsPadded * sizeof(float2);
    int rc = grow(ctx, (void **)&ctx->d_partial, &ctx->partial_bytes, pbytes);
    if (rc) return rc;
    CUtensorMap tmap;
    rc = make_source_map(ctx, &tmap, src, (int)dt, len, src_ld, n_src, 2);
    if (rc) return rc;
    FftArgs a;
    a.tw = ctx->d_tw;
    a.spec = ctx->d_spec;
    a.dir = dir;
    a.n_src = n_src;
    a.n_dirs = ctx->n_dirs;
    a.hop = hop;
    a.guard = guard;
    a.part = part;
    a.partial = reinterpret_cast<float2 *>(ctx->d_partial);
    a.slots = slots;
    a.status = ctx->d_status;
    {
        KernelTimer kt(ctx, HRIR_K_FFT, st);
        HRIR_CUDA_TRY(ctx, launch_fft_mix((int)dt, tmap, a, (int)part.P,
                                          fft_mix_smem_bytes((int)dtype_size(dt)), st));
        kt.done();
    }
    FftOutArgs o;
    o.partial = a.partial;
    o.slots = slots;
    o.part = part;
    o.tw = ctx->d_tw;
    o.hop = hop;
    o.guard = guard;
    o.out_len = out_len;
    o.out = out;
    o.out_ld = out_ld;
    {
        KernelTimer kt(ctx, HRIR_K_REDUCE, st);
        HRIR_CUDA_TRY(ctx, launch_fft_out(o, n_frames, st));
        kt.done();
    }
    return HRIR_OK;
}

// The direct-convolution render (sparse taps or dense HRIRs): the mixing kernel over
// (tile, source) units writing partial sums, then the fixed-order reduction with the
// resonance FIR.  Shared by hrir_render_batch, hrir_render_batch_noalloc and
// hrir_render_precomputed, so that the three use the same partition, run lengths and
// summation order.
int mix_render(hrir_ctx *ctx, const MixJob &j, cudaStream_t st)
{
    const bool sparse = j.sparse;
    const size_t es = dtype_size(j.dt);
    const int nchunk = sparse ? ctx->sparse_nchunk : ctx->dense_nchunk;
    const MixShape shape = mix_shape(sparse ? MIX_SPARSE : MIX_DENSE);
    const int tile = shape.tile;
    // history before each tile, a multiple of kMixBox so that tiles start on a source row
    const int halo = (int)round_up((int64_t)nchunk * (sparse ? kSparseSegment : shape.r), kMixBox);
    const int buf_elems = (int)round_up(halo + tile, kMixBox);
    const int rec_bytes = sparse ? ctx->sparse_rec_bytes : 2 * ctx->dense_padded * 4;
    const int64_t mix_len = sparse ? std::min<int64_t>(j.out_len, j.len + ctx->refl_len - 1) : j.out_len;
    const int n_tiles = (int)((mix_len + tile - 1) / tile);

    Partition part;
    part.U = (int64_t)n_tiles * j.n_src;
    part.P = std::min<int64_t>(ctx->num_sms, part.U);
    part.n_src = j.n_src;
    part.gs = mix_run_sources(ctx, sparse);
    int slots = 0;
    for (int t = 0; t < n_tiles; ++t) slots = std::max(slots, part.slots(t));
    const size_t pbytes = (size_t)n_tiles * slots * 2 * tile * sizeof(float);
    float *partial = j.scratch;
    if (partial) {
        if (pbytes > j.scratch_bytes)
            return fail(ctx, HRIR_EINVAL,
                        "this render needs %zu bytes of partial-sum scratch; the fixed array holds %zu "
                        "(use hrir_render_batch, or fewer sources or samples per call)",
                        pbytes, j.scratch_bytes);
    } else {
        int rc = grow(ctx, (void **)&ctx->d_partial, &ctx->partial_bytes, pbytes);
        if (rc) return rc;
        partial = ctx->d_partial;
    }
    size_t smem = 0;
    const size_t extra = sparse ? (size_t)kSparseRunAccBytes : 0;
    const int stages = pick_stages(buf_elems, (int)es, rec_bytes, extra, &smem);
    if (stages == 0) return fail(ctx, HRIR_EINVAL, "filters too long for the shared-memory pipeline");
    CUtensorMap tmap, tmap3;
    int rc = make_source_map(ctx, &tmap, j.src, j.dt, j.len, j.src_ld, j.n_src);
    if (rc) return rc;
    rc = make_source_map3(ctx, &tmap3, tmap, j.src, j.dt, j.len, j.src_ld, j.n_src, buf_elems / kMixBox);
    if (rc) return rc;

    MixArgs a;
    a.src = j.src;
    a.ld = j.src_ld;
    a.len = j.len;
    a.n_src = j.n_src;
    a.dir = j.dir;
    a.n_dirs = j.n_dirs;
    a.table = j.table;
    a.rec_bytes = rec_bytes;
    a.nchunk = sparse ? ctx->sparse_nch_pad : nchunk;
    a.nseg = sparse ? ctx->sparse_nchunk : 0;
    a.halo = halo;
    a.buf_elems = buf_elems;
    a.full_rows = (int)(j.len / kMixBox);
    a.n_tiles = n_tiles;
    a.stages = stages;
    a.runacc_off = (int)(smem - extra);
    a.fold = mix_fold_sources(ctx);
    a.part = part;
    a.partial = partial;
    a.slots = slots;
    a.status = ctx->d_status;
    {
        KernelTimer kt(ctx, sparse ? HRIR_K_MIX_SPARSE : HRIR_K_MIX_DENSE, st, j.timed);
        CUDA_TRY(ctx, launch_mix(sparse ? MIX_SPARSE : MIX_DENSE, j.dt, tmap, tmap3, a, (int)part.P, smem, st));
        kt.done();
    }
    ReduceArgs r;
    r.partial = partial;
    r.slots = slots;
    r.n_tiles = n_tiles;
    r.tile = tile;
    r.part = part;
    r.res = j.res;
    r.res_len = ctx->res_len;
    r.out_len = j.out_len;
    r.out = j.out;
    r.out_ld = j.out_ld;
    {
        KernelTimer kt(ctx, HRIR_K_REDUCE, st, j.timed);
        CUDA_TRY(ctx, launch_reduce(r, st));
        kt.done();
    }
    return HRIR_OK;
}

}  // namespace hrir_host

using namespace hrir_host;

extern "C" {

int hrir_version(void) { return (0 << 16) | 1; }

int hrir_create(hrir_ctx **out, int device)
{
    if (!out) return fail(nullptr, HRIR_EINVAL, "out is NULL");
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return fail(nullptr, HRIR_ECUDA, "CUDA device %d not available (%d devices)", device, n);
    }
    if (cudaSetDevice(device) != cudaSuccess)
        return fail(nullptr, HRIR_ECUDA, "cudaSetDevice(%d) failed", device);
    hrir_ctx *ctx = new hrir_ctx();
    ctx->device = device;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&ctx->d_status, sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->d_status, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return fail(nullptr, HRIR_ENOMEM, "status word allocation failed");
    }
    *out = ctx;
    return HRIR_OK;
}

void hrir_destroy(hrir_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    hrir_stream_close(ctx);
    free_tables(ctx);
    drop_timing_events(ctx);
    for (cudaEvent_t &e : ctx->copy_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    cudaFree(ctx->d_partial);
    cudaFree(ctx->d_stage);
    if (ctx->h_dir) cudaFreeHost(ctx->h_dir);
    cudaFree(ctx->d_mlp_ws);
    cudaFree(ctx->d_fact_ws);
    cudaFree(ctx->d_view_ws);
    cudaFree(ctx->d_status);
    delete ctx;
}

int hrir_set_timing(hrir_ctx *ctx, int enable)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    ctx->timing = enable != 0;
    return HRIR_OK;
}

int hrir_kernel_times(hrir_ctx *ctx, double *ms, int64_t *launches, int reset)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    for (auto &p : ctx->pending) {
        CUDA_TRY(ctx, cudaEventSynchronize(p.b));
        float t = 0.f;
        CUDA_TRY(ctx, cudaEventElapsedTime(&t, p.a, p.b));
        ctx->ms[p.kind] += t;
        ctx->launches[p.kind] += 1;
        ctx->free_events.push_back(p.a);
        ctx->free_events.push_back(p.b);
    }
    ctx->pending.clear();
    for (int i = 0; i < HRIR_K_COUNT; ++i) {
        if (ms) ms[i] = ctx->ms[i];
        if (launches) launches[i] = ctx->launches[i];
        if (reset) {
            ctx->ms[i] = 0.0;
            ctx->launches[i] = 0;
        }
    }
    return HRIR_OK;
}

const char *hrir_last_error(const hrir_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

int hrir_sync(hrir_ctx *ctx, void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    CUDA_TRY(ctx, cudaStreamSynchronize((cudaStream_t)stream));
    int st = 0;
    CUDA_TRY(ctx, cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st == 0) return HRIR_OK;
    CUDA_TRY(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)));
    if (st & DEV_TIMEOUT)
        return fail(ctx, HRIR_ETIMEDOUT, "a bounded device wait expired (output incomplete)");
    if (st & DEV_BAD_TAP)
        return fail(ctx, HRIR_EINVAL, "a device tap table held an index >= Lg or a count > k_max (ignored)");
    if (st & DEV_LAYOUT)
        return fail(ctx, HRIR_ECUDA, "a kernel found its shared memory misaligned for its TMA layout "
                                     "(the call produced no output)");
    if (st & DEV_SOLVER)
        return fail(ctx, HRIR_EINVAL, "a filter-production solve failed: an L1-NNLS row outgrew the "
                                      "solver's support or iteration limit (its result is the last "
                                      "feasible iterate), or a resonance system of hrir_factorize was "
                                      "not positive definite");
    return fail(ctx, HRIR_EINVAL, "a direction id was out of range (rendered as silence)");
}

int hrir_selftest_wait_timeout(hrir_ctx *ctx, void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    CUDA_TRY(ctx, launch_wait_timeout_selftest(ctx->d_status, (cudaStream_t)stream));
    return HRIR_OK;
}

int hrir_topk_pack(hrir_ctx *ctx, int n_rows, int refl_len, int k, const float *g, uint16_t *idx,
                   float *w, uint8_t *nnz, void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    if (n_rows < 0 || refl_len < 1 || refl_len > 2048 || k < 0 || k > 255)
        return fail(ctx, HRIR_EINVAL, "bad sizes (n_rows=%d refl_len=%d k=%d)", n_rows, refl_len, k);
    if (n_rows == 0) return HRIR_OK;
    if (!g || !nnz || (k > 0 && (!idx || !w))) return fail(ctx, HRIR_EINVAL, "NULL buffer");
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    KernelTimer kt(ctx, HRIR_K_TABLES, (cudaStream_t)stream);
    CUDA_TRY(ctx, launch_topk(g, n_rows, refl_len, k, idx, w, nnz, (cudaStream_t)stream));
    kt.done();
    return HRIR_OK;
}

int hrir_load_filters(hrir_ctx *ctx, int n_dirs, int n_ears, int refl_len, int k_max,
                      const uint16_t *tap_idx, const float *tap_w, const uint8_t *tap_nnz,
                      int res_len, const float *resonance, int fft_size)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    if (n_dirs < 1 || n_ears != 2 || refl_len < 1 || refl_len > 2048 || k_max < 0 ||
        k_max > 255 || res_len < 1 || res_len > 512)
        return fail(ctx, HRIR_EINVAL, "bad sizes (n_dirs=%d n_ears=%d refl_len=%d k_max=%d res_len=%d)",
                    n_dirs, n_ears, refl_len, k_max, res_len);
    if (!tap_nnz || !resonance || (k_max > 0 && (!tap_idx || !tap_w)))
        return fail(ctx, HRIR_EINVAL, "NULL table pointer");
    const int hrir_len = res_len + refl_len - 1;
    if (fft_size != 0 && fft_size != kFftSize)
        return fail(ctx, HRIR_EINVAL, "fft_size %d: the FFT path implements P = %d (pass 0 or %d)",
                    fft_size, kFftSize, kFftSize);
    if ((int)round_up(hrir_len - 1, 8) >= kFftSize)
        return fail(ctx, HRIR_EINVAL, "HRIR length %d too long for the P = %d FFT frame", hrir_len, kFftSize);
    for (int64_t r = 0; r < (int64_t)n_dirs * 2; ++r) {
        const int k = tap_nnz[r];
        if (k > k_max) return fail(ctx, HRIR_EINVAL, "tap_nnz[%lld]=%d > k_max", (long long)r, k);
        for (int t = 0; t < k; ++t) {
            const int i = tap_idx[r * k_max + t];
            const float v = tap_w[r * k_max + t];
            if (i >= refl_len)
                return fail(ctx, HRIR_EINVAL, "tap index %d >= refl_len at row %lld", i, (long long)r);
            if (t > 0 && i <= tap_idx[r * k_max + t - 1])
                return fail(ctx, HRIR_EINVAL, "tap indices not strictly ascending at row %lld", (long long)r);
            if (!std::isfinite(v) || v < 0.f)
                return fail(ctx, HRIR_EINVAL, "tap weight must be finite and >= 0 (row %lld)", (long long)r);
        }
    }
    for (int i = 0; i < 2 * res_len; ++i)
        if (!std::isfinite(resonance[i])) return fail(ctx, HRIR_EINVAL, "resonance must be finite");

    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    CUDA_TRY(ctx, cudaDeviceSynchronize());
    hrir_stream_close(ctx);  // a stream's graph refers to the old tables
    free_tables(ctx);

    const size_t rows = (size_t)n_dirs * 2;
    const size_t kk = k_max > 0 ? (size_t)k_max : 1;
    uint16_t *d_idx = nullptr;
    float *d_w = nullptr;
    uint8_t *d_nnz = nullptr;
    const int sparse_nseg = (refl_len + kSparseSegment - 1) / kSparseSegment;
    const int sparse_nseg_pad = (int)round_up(sparse_nseg, 2);
    const int sparse_rec =
        (int)round_up(16 + 8 * sparse_nseg_pad + 8 * (2 * (int64_t)k_max + 2 * sparse_nseg + 4), 16);
    const int dense_nchunk = (hrir_len + kDenseR - 1) / kDenseR;
    const int dense_padded = dense_nchunk * kDenseR;
    int rc = HRIR_OK;
    cudaError_t e = cudaSuccess;
    do {
        if ((e = cudaMalloc(&d_idx, rows * kk * 2)) != cudaSuccess) break;
        if ((e = cudaMalloc(&d_w, rows * kk * 4)) != cudaSuccess) break;
        if ((e = cudaMalloc(&d_nnz, rows)) != cudaSuccess) break;
        if ((e = cudaMalloc(&ctx->d_res, 2 * (size_t)res_len * 4)) != cudaSuccess) break;
        if ((e = cudaMalloc(&ctx->d_sparse, (size_t)(n_dirs + 1) * sparse_rec)) != cudaSuccess) break;
        if ((e = cudaMalloc(&ctx->d_dense, (size_t)(n_dirs + 1) * 2 * dense_padded * 4)) != cudaSuccess)
            break;
        if (k_max > 0) {
            if ((e = cudaMemcpy(d_idx, tap_idx, rows * k_max * 2, cudaMemcpyHostToDevice)) != cudaSuccess) break;
            if ((e = cudaMemcpy(d_w, tap_w, rows * k_max * 4, cudaMemcpyHostToDevice)) != cudaSuccess) break;
        }
        if ((e = cudaMemcpy(d_nnz, tap_nnz, rows, cudaMemcpyHostToDevice)) != cudaSuccess) break;
        if ((e = cudaMemcpy(ctx->d_res, resonance, 2 * (size_t)res_len * 4, cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            break;
        if ((e = launch_build_sparse_records(d_idx, d_w, d_nnz, n_dirs, (int)kk, kSparseSegment,
                                             sparse_nseg, sparse_nseg_pad, ctx->d_sparse, sparse_rec,
                                             0)) != cudaSuccess)
            break;
        if ((e = launch_build_dense_records(d_idx, d_w, d_nnz, n_dirs, (int)kk, ctx->d_res, res_len,
                                            hrir_len, dense_padded, ctx->d_dense, 0)) != cudaSuccess)
            break;
        {
            // one-ear records for hrir_render_precomputed: record 2d + e holds ear e's taps of
            // direction d and no taps for the other ear
            const size_t rows2 = 2 * rows;
            std::vector<uint16_t> idx2(rows2 * kk, 0);
            std::vector<float> w2(rows2 * kk, 0.f);
            std::vector<uint8_t> nnz2(rows2, 0);
            for (size_t r = 0; r < rows; ++r) {          // r = 2 d + e of the input tables
                const size_t d = r / 2, ear = r % 2, dst = (2 * d + ear) * 2 + ear;
                nnz2[dst] = tap_nnz[r];
                for (int t = 0; t < k_max; ++t) {
                    idx2[dst * kk + t] = tap_idx[r * k_max + t];
                    w2[dst * kk + t] = tap_w[r * k_max + t];
                }
            }
            uint16_t *d_idx2 = nullptr;
            float *d_w2 = nullptr;
            uint8_t *d_nnz2 = nullptr;
            if ((e = cudaMalloc(&ctx->d_sparse_split, (size_t)(2 * n_dirs + 1) * sparse_rec)) == cudaSuccess &&
                (e = cudaMalloc(&d_idx2, rows2 * kk * 2)) == cudaSuccess &&
                (e = cudaMalloc(&d_w2, rows2 * kk * 4)) == cudaSuccess &&
                (e = cudaMalloc(&d_nnz2, rows2)) == cudaSuccess &&
                (e = cudaMemcpy(d_idx2, idx2.data(), rows2 * kk * 2, cudaMemcpyHostToDevice)) == cudaSuccess &&
                (e = cudaMemcpy(d_w2, w2.data(), rows2 * kk * 4, cudaMemcpyHostToDevice)) == cudaSuccess &&
                (e = cudaMemcpy(d_nnz2, nnz2.data(), rows2, cudaMemcpyHostToDevice)) == cudaSuccess &&
                (e = launch_build_sparse_records(d_idx2, d_w2, d_nnz2, 2 * n_dirs, (int)kk, kSparseSegment,
                                                 sparse_nseg, sparse_nseg_pad, ctx->d_sparse_split,
                                                 sparse_rec, 0)) == cudaSuccess)
                e = cudaDeviceSynchronize();
            cudaFree(d_idx2);
            cudaFree(d_w2);
            cudaFree(d_nnz2);
            if (e != cudaSuccess) break;
        }
        {
            // FFT twiddles exp(-2 pi i k / P), computed in double on the host
            std::vector<float2> tw(kFftSize);
            for (int k = 0; k < kFftSize; ++k) {
                const double ang = -2.0 * 3.14159265358979323846 * (double)k / (double)kFftSize;
                tw[k] = make_float2((float)std::cos(ang), (float)std::sin(ang));
            }
            if ((e = cudaMalloc(&ctx->d_tw, kFftSize * sizeof(float2))) != cudaSuccess) break;
            if ((e = cudaMemcpy(ctx->d_tw, tw.data(), kFftSize * sizeof(float2),
                                cudaMemcpyHostToDevice)) != cudaSuccess)
                break;
            if ((e = cudaMalloc(&ctx->d_spec, (size_t)(n_dirs + 1) * 2 * kFftBinsPadded *
                                                  sizeof(float2))) != cudaSuccess)
                break;
            if ((e = launch_build_spectra(ctx->d_dense, dense_padded, hrir_len, n_dirs + 1, ctx->d_tw,
                                          ctx->d_spec, 0)) != cudaSuccess)
                break;
        }
        e = cudaDeviceSynchronize();
    } while (0);
    if (e != cudaSuccess) {
        cudaFree(d_idx);
        cudaFree(d_w);
        cudaFree(d_nnz);
        free_tables(ctx);
        rc = fail(ctx, e == cudaErrorMemoryAllocation ? HRIR_ENOMEM : HRIR_ECUDA,
                  "filter table construction failed: %s", cudaGetErrorString(e));
        cudaGetLastError();
        return rc;
    }
    ctx->d_tap_idx = d_idx;  // kept for the streaming kernel
    ctx->d_tap_w = d_w;
    ctx->d_tap_nnz = d_nnz;
    ctx->n_dirs = n_dirs;
    ctx->refl_len = refl_len;
    ctx->k_max = k_max;
    ctx->res_len = res_len;
    ctx->hrir_len = hrir_len;
    ctx->fft_size = fft_size;
    ctx->sparse_rec_bytes = sparse_rec;
    ctx->sparse_nchunk = sparse_nseg;
    ctx->sparse_nch_pad = sparse_nseg_pad;
    ctx->dense_nchunk = dense_nchunk;
    ctx->dense_padded = dense_padded;
    ctx->loaded = true;
    return HRIR_OK;
}

int64_t hrir_out_len(const hrir_ctx *ctx, int64_t len, int full)
{
    if (!ctx || !ctx->loaded || len <= 0) return 0;
    return full ? len + ctx->hrir_len - 1 : len;
}

int hrir_render_batch(hrir_ctx *ctx, int n_src, int64_t len, int64_t src_ld, hrir_dtype dt,
                      const void *src, const int32_t *dir, hrir_mode mode, int full, float *out,
                      int64_t out_ld, void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    if (!ctx->loaded) return fail(ctx, HRIR_ESTATE, "no filters loaded");
    if (n_src < 0 || len < 0) return fail(ctx, HRIR_EINVAL, "negative n_src or len");
    if (dt != HRIR_F32 && dt != HRIR_BF16 && dt != HRIR_F16)
        return fail(ctx, HRIR_EINVAL, "unknown dtype %d", (int)dt);
    if (mode != HRIR_SPARSE && mode != HRIR_DENSE && mode != HRIR_FFT)
        return fail(ctx, HRIR_EINVAL, "unknown mode %d", (int)mode);
    const int64_t out_len = full ? (len > 0 ? len + ctx->hrir_len - 1 : 0) : len;
    if (out_len == 0) return HRIR_OK;
    if (!out || out_ld < out_len) return fail(ctx, HRIR_EINVAL, "out is NULL or out_ld < %lld", (long long)out_len);
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    if (n_src == 0) {
        CUDA_TRY(ctx, cudaMemset2DAsync(out, (size_t)out_ld * 4, 0, (size_t)out_len * 4, 2, st));
        return HRIR_OK;
    }
    const size_t es = dtype_size(dt);
    if (!src || !dir) return fail(ctx, HRIR_EINVAL, "NULL src or dir");
    if (src_ld < len || ((uintptr_t)src % 16) || ((src_ld * (int64_t)es) % 16))
        return fail(ctx, HRIR_EINVAL,
                    "src must be 16-byte aligned with src_ld >= len and src_ld*elem_size %% 16 == 0");
    if (len > (int64_t)1 << 31) return fail(ctx, HRIR_EINVAL, "len must be < 2^31");
    if (mode == HRIR_FFT) return render_fft(ctx, n_src, len, src_ld, dt, src, dir, out_len, out, out_ld, st);

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
    return mix_render(ctx, j, st);
}

int hrir_render_batch_host(hrir_ctx *ctx, int n_src, int64_t len, int64_t src_ld, hrir_dtype dt,
                           const void *src, const int32_t *dir, hrir_mode mode, int full, float *out,
                           int64_t out_ld, void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    if (!ctx->loaded) return fail(ctx, HRIR_ESTATE, "no filters loaded");
    if (n_src < 0 || len < 0 || src_ld < len) return fail(ctx, HRIR_EINVAL, "bad n_src/len/src_ld");
    if (dt != HRIR_F32 && dt != HRIR_BF16 && dt != HRIR_F16)
        return fail(ctx, HRIR_EINVAL, "unknown dtype %d", (int)dt);
    const int64_t out_len = full ? (len > 0 ? len + ctx->hrir_len - 1 : 0) : len;
    if (out_len == 0) return HRIR_OK;
    if (!out || out_ld < out_len) return fail(ctx, HRIR_EINVAL, "out is NULL or out_ld too small");
    if (n_src > 0 && (!src || !dir)) return fail(ctx, HRIR_EINVAL, "NULL src or dir");
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(ctx, cudaSetDevice(ctx->device));
    const size_t es = dtype_size(dt);
    const int64_t vec = 16 / (int64_t)es;
    const int64_t dld = round_up(std::max<int64_t>(len, 1), vec);
    const size_t src_bytes = (size_t)n_src * dld * es;
    // The sources go over in up to kHostChunks chunks on the context's copy stream; chunk c is
    // rendered on the caller's stream as soon as it has landed (while the next chunks copy),
    // into its own output planes, and the planes are summed in chunk order (the render is
    // linear in the sources and the resonance follows the mix, Eq. 2).
    constexpr int kHostChunks = 4;
    const int n_chunks = n_src >= 4 * kHostChunks ? kHostChunks : 1;
    const size_t dir_off = round_up((int64_t)src_bytes, 256);
    const size_t out_off = round_up((int64_t)(dir_off + (size_t)n_src * 4), 256);
    const size_t plane = 2 * (size_t)out_len * 4;
    const size_t need = out_off + (size_t)n_chunks * plane;
    int rc = grow(ctx, &ctx->d_stage, &ctx->stage_bytes, need);
    if (rc) return rc;
    unsigned char *base = static_cast<unsigned char *>(ctx->d_stage);
    int32_t *d_dir = reinterpret_cast<int32_t *>(base + dir_off);
    float *d_out = reinterpret_cast<float *>(base + out_off);
    if (n_src == 0) {
        rc = hrir_render_batch(ctx, 0, len, dld, dt, base, d_dir, mode, full, d_out, out_len, stream);
        if (rc) return rc;
    } else {
        if (!ctx->copy_stream) {
            CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
            for (cudaEvent_t &e : ctx->copy_ev) CUDA_TRY(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        }
        cudaStream_t cs = ctx->copy_stream;
        // the direction ids go through a page-locked copy: a copy from pageable memory would
        // wait, inside each chunk's issue, for the chunk copies queued before it.  The copy
        // stream is idle here (every earlier call ended with its synchronize) unless an earlier
        // call failed half-way; the synchronize makes reusing the page-locked copy safe then too.
        CUDA_TRY(ctx, cudaStreamSynchronize(cs));
        const size_t dir_bytes = (size_t)n_src * 4;
        if (ctx->h_dir_bytes < dir_bytes) {
            if (ctx->h_dir) cudaFreeHost(ctx->h_dir);
            ctx->h_dir = nullptr;
            ctx->h_dir_bytes = 0;
            if (cudaHostAlloc(&ctx->h_dir, dir_bytes, cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                ctx->h_dir = nullptr;
                return fail(ctx, HRIR_ENOMEM, "page-locked staging of %zu bytes failed", dir_bytes);
            }
            ctx->h_dir_bytes = dir_bytes;
        }
        std::memcpy(ctx->h_dir, dir, dir_bytes);
        const int32_t *h_dir = static_cast<const int32_t *>(ctx->h_dir);
        // the staging buffers are free once the caller's earlier work on `stream` is done
        CUDA_TRY(ctx, cudaEventRecord(ctx->copy_ev[kHostChunks], st));
        CUDA_TRY(ctx, cudaStreamWaitEvent(cs, ctx->copy_ev[kHostChunks], 0));
        for (int c = 0; c < n_chunks; ++c) {
            const int64_t s0 = (int64_t)n_src * c / n_chunks, s1 = (int64_t)n_src * (c + 1) / n_chunks;
            unsigned char *d_src = base + (size_t)s0 * dld * es;
            const unsigned char *h_src = static_cast<const unsigned char *>(src) + (size_t)s0 * src_ld * es;
            if (dld == src_ld) {
                CUDA_TRY(ctx, cudaMemcpyAsync(d_src, h_src, (size_t)(s1 - s0) * dld * es, cudaMemcpyHostToDevice, cs));
            } else {
                CUDA_TRY(ctx, cudaMemcpy2DAsync(d_src, dld * es, h_src, src_ld * es, len * es, (size_t)(s1 - s0),
                                                cudaMemcpyHostToDevice, cs));
            }
            CUDA_TRY(ctx, cudaMemcpyAsync(d_dir + s0, h_dir + s0, (size_t)(s1 - s0) * 4, cudaMemcpyHostToDevice, cs));
            CUDA_TRY(ctx, cudaEventRecord(ctx->copy_ev[c], cs));
        }
        for (int c = 0; c < n_chunks; ++c) {
            const int64_t s0 = (int64_t)n_src * c / n_chunks, s1 = (int64_t)n_src * (c + 1) / n_chunks;
            CUDA_TRY(ctx, cudaStreamWaitEvent(st, ctx->copy_ev[c], 0));
            rc = hrir_render_batch(ctx, (int)(s1 - s0), len, dld, dt, base + (size_t)s0 * dld * es, d_dir + s0,
                                   mode, full, reinterpret_cast<float *>(reinterpret_cast<unsigned char *>(d_out) + c * plane),
                                   out_len, stream);
            if (rc) return rc;
        }
        // the chunk planes summed in chunk order, in place over the first
        if (n_chunks > 1) CUDA_TRY(ctx, launch_add_parts(d_out, out_len, d_out, n_chunks, out_len, st));
    }
    CUDA_TRY(ctx, cudaMemcpy2DAsync(out, out_ld * 4, d_out, out_len * 4, out_len * 4, 2,
                                    cudaMemcpyDeviceToHost, st));
    return hrir_sync(ctx, stream);
}

}  // extern "C"
