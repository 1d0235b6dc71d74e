// api_internal.h -- context structure and host helpers shared by the C-ABI translation
// units (hrir_api.cu, noalloc.cu).  Not part of the public ABI.
#pragma once

#include <cstdarg>
#include <cstdint>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/hrir.h"
#include "kernels.h"

struct hrir_stream;  // streaming state (stream.cu)

struct hrir_ctx {
    int device = 0;
    int num_sms = 0;
    std::string err;

    bool loaded = false;
    int n_dirs = 0, refl_len = 0, k_max = 0, res_len = 0, hrir_len = 0, fft_size = 0;
    unsigned char *d_sparse = nullptr;  // (n_dirs + 1) sparse tap records
    unsigned char *d_sparse_split = nullptr;  // (2 n_dirs + 1) one-ear records (2 d + e)
    int sparse_rec_bytes = 0;
    int sparse_nchunk = 0;   // window segments of kSparseSegment filter offsets
    int sparse_nch_pad = 0;  // segment-count array length in a record (even)
    float *d_dense = nullptr;           // (n_dirs + 1) x [2][dense_padded]
    int dense_padded = 0, dense_nchunk = 0;
    float *d_res = nullptr;             // [2][res_len]
    uint16_t *d_tap_idx = nullptr;      // [n_dirs][2][k_max] (streaming kernel)
    float *d_tap_w = nullptr;
    uint8_t *d_tap_nnz = nullptr;
    hrir_stream *stream = nullptr;      // open block stream, if any
    float2 *d_tw = nullptr;             // FFT twiddles [kFftSize]
    float2 *d_spec = nullptr;           // (n_dirs + 1) x [2][kFftBinsPadded] HRIR spectra

    float *d_partial = nullptr;
    size_t partial_bytes = 0;
    void *d_stage = nullptr;            // device staging for hrir_render_batch_host
    size_t stage_bytes = 0;
    cudaStream_t copy_stream = nullptr; // host-to-device copies of hrir_render_batch_host
    void *h_dir = nullptr;              // page-locked copy of its direction ids
    size_t h_dir_bytes = 0;
    cudaEvent_t copy_ev[5] = {};        // [chunks]: chunk copied; [chunks]: caller's work before
    void *d_mlp_ws = nullptr;           // learned-filter network workspace
    size_t mlp_ws_bytes = 0;
    void *d_fact_ws = nullptr;          // filter-production workspace (L1-NNLS fine-tune)
    size_t fact_ws_bytes = 0;
    void *d_view_ws = nullptr;          // per-view source rows of hrir_render_precomputed
    size_t view_ws_bytes = 0;
    int *d_status = nullptr;

    // optional kernel timing (hrir_set_timing)
    bool timing = false;
    struct Pending {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> free_events;
    double ms[HRIR_K_COUNT] = {};
    int64_t launches[HRIR_K_COUNT] = {};
};

namespace hrir_host {

// Record a failure message on ctx (or the thread's create-error slot) and return code.
int fail(hrir_ctx *ctx, int code, const char *fmt, ...);
size_t dtype_size(int dt);
// Make *ptr hold at least `need` bytes of device memory (grown with 1/8 slack).
int grow(hrir_ctx *ctx, void **ptr, size_t *have, size_t need);
int64_t round_up(int64_t x, int64_t m);
// Sources per register accumulation run of the sparse (taps of the loaded tables) or dense
// mixing kernel; hrir_render_batch and hrir_render_batch_noalloc use the same value.
int mix_run_sources(const hrir_ctx *ctx, bool sparse);
// Sources per register fold of the sparse mixing kernel (kFoldTerms / k_max, at least 1).
int mix_fold_sources(const hrir_ctx *ctx);
// Pipeline depth (2..kMixMaxStages) that fits the 227 KB shared-memory limit with `extra`
// bytes after the mixing kernel's own layout (16-byte aligned, at *smem - extra); 0 if none.
int pick_stages(int buf_elems, int elem_bytes, int rec_bytes, size_t extra, size_t *smem);
// 2-D tensor map over the sources: dims {len, n_src}, row stride ld, box {kMixBox, 1}.
int make_source_map(hrir_ctx *ctx, CUtensorMap *m, const void *src, int dt, int64_t len,
                    int64_t ld, int n_src, int box_rows = 1);
// 3-D view of the sources {kMixBox, len / kMixBox, n_src} with box {kMixBox, box_rows, 1};
// when len < kMixBox there are no full rows and *m is a copy of the 2-D map `fallback`.
int make_source_map3(hrir_ctx *ctx, CUtensorMap *m, const CUtensorMap &fallback, const void *src,
                     int dt, int64_t len, int64_t ld, int n_src, int box_rows);
// 3-D view {32, rows, n_src} of FP32 sources (rows of 32 samples, row stride 128 bytes, source
// stride ld), box {32, box_rows, 1}, 128-byte swizzle, zero fill outside
int make_source_rows32_map(hrir_ctx *ctx, CUtensorMap *m, const float *src, int64_t rows, int64_t ld, int n_src,
                           int box_rows);
cudaEvent_t take_event(hrir_ctx *ctx);

// Brackets one kernel launch with events when timing is enabled.
struct KernelTimer {
    hrir_ctx *ctx;
    int kind;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    KernelTimer(hrir_ctx *c, int k, cudaStream_t s, bool enabled = true) : ctx(c), kind(k), st(s)
    {
        if (enabled && ctx->timing) {
            a = take_event(ctx);
            cudaEventRecord(a, st);
        }
    }
    void done()
    {
        if (!a) return;
        cudaEvent_t b = take_event(ctx);
        cudaEventRecord(b, st);
        ctx->pending.push_back({kind, a, b});
        a = nullptr;
    }
};

// One direct-convolution render (see mix_render in hrir_api.cu).
struct MixJob {
    int n_src = 0;
    int64_t len = 0, src_ld = 0;
    int dt = 0;
    const void *src = nullptr;          // [n_src][src_ld] of dt, device
    const int32_t *dir = nullptr;       // [n_src] record index per source, device
    bool sparse = true;                 // sparse tap records, else dense HRIR records
    const unsigned char *table = nullptr;
    int n_dirs = 0;                     // records in table (plus one silent record)
    const float *res = nullptr;         // resonance applied after the mix, or nullptr
    int64_t out_len = 0;
    float *out = nullptr;               // [2][out_ld], device
    int64_t out_ld = 0;
    float *scratch = nullptr;           // fixed partial-sum scratch, or nullptr: the workspace
    size_t scratch_bytes = 0;
    bool timed = true;                  // kernels timed by hrir_set_timing
};
int mix_render(hrir_ctx *ctx, const MixJob &j, cudaStream_t st);

}  // namespace hrir_host

#define HRIR_CUDA_TRY(ctx, call)                                                           \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return hrir_host::fail((ctx), HRIR_ECUDA, "%s failed: %s", #call,             \
                                   cudaGetErrorString(e_));                                \
    } while (0)
