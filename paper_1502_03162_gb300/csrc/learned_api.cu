// learned_api.cu -- host side of the learned-filter calls of the C ABI (include/hrir.h):
// the direction -> reflection-filter network (forward, backward, Adam), the moving-source
// render with per-segment filters and a linear crossfade, and the per-source resonance on the
// tensor cores.
#include <algorithm>
#include <cmath>

#include "api_internal.h"

using namespace hrir;
using namespace hrir_host;

namespace {

constexpr int H = kMlpHidden;

// Offsets of the parameter blocks in the flat vector: W1, b1, W2, b2, W3, b3, W4, b4.
struct MlpLayout {
    int64_t W1, b1, W2, b2, W3, b3, W4, b4, total;
    explicit MlpLayout(int refl_len)
    {
        W1 = 0;
        b1 = W1 + (int64_t)H * kMlpIn;
        W2 = b1 + H;
        b2 = W2 + (int64_t)H * H;
        W3 = b2 + H;
        b3 = W3 + (int64_t)H * H;
        W4 = b3 + H;
        b4 = W4 + (int64_t)refl_len * H;
        total = b4 + refl_len;
    }
};

int64_t act_stride(int refl_len) { return round_up(3 * H + refl_len, 4); }

// Rows per forward chunk when the caller keeps no activations.
constexpr int64_t kFwdChunk = 1 << 16;
// Rows per chunk of the tensor-core inference (two BF16 activation buffers of 256 columns).
constexpr int64_t kTcChunk = 1 << 22;

int grow_ws(hrir_ctx *ctx, size_t need)
{
    return grow(ctx, &ctx->d_mlp_ws, &ctx->mlp_ws_bytes, need);
}

GemmArgs gemm_args(int64_t M, int N, int K, const float *A, int64_t sam, int64_t sak, const float *B,
                   int64_t sbk, int64_t sbn)
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
    g.k_chunk = K;
    return g;
}

// CTAs a network GEMM should launch to occupy every SM (two per SM)
int gemm_min_ctas(const hrir_ctx *ctx) { return 2 * std::max(ctx->num_sms, 1); }

// dW[M][N] = sum_b A(m, b) B(b, n) split over the rows b (enough splits to occupy every SM,
// at most 64), partials summed in a fixed order.
int weight_grad(hrir_ctx *ctx, GemmArgs g, bool relu_b, float *P, float *out, cudaStream_t st)
{
    const int64_t rows = g.K;
    const int64_t tiles = ((g.M + gemm_tc_tile_rows() - 1) / gemm_tc_tile_rows()) *
                          ((g.N + gemm_tc_tile_cols() - 1) / gemm_tc_tile_cols());
    const int64_t want = std::max<int64_t>((rows + 511) / 512, (gemm_min_ctas(ctx) + tiles - 1) / tiles);
    int splits = (int)std::min<int64_t>(64, std::max<int64_t>(1, want));
    g.k_chunk = (int)round_up((rows + splits - 1) / splits, 16);
    splits = (int)((rows + g.k_chunk - 1) / g.k_chunk);
    g.Z = P;
    g.ldz = g.N;
    HRIR_CUDA_TRY(ctx, launch_gemm_tc(3, false, relu_b, g, splits, ctx->d_status, st));
    HRIR_CUDA_TRY(ctx, launch_split_reduce(splits, (int)g.M, g.N, P, out, st));
    return HRIR_OK;
}

// The moving-source mix on tensor-memory windows, then the reduction with the resonance.
int render_moving_tmem(hrir_ctx *ctx, int n_src, int64_t len, int64_t src_ld, const float *src, int n_seg,
                       int seg_len, int k_max, const uint16_t *tap_idx, const float *tap_w, const uint8_t *tap_nnz,
                       int64_t mix_len, int64_t out_len, float *out, int64_t out_ld, cudaStream_t st)
{
    const int n_tiles = (int)((mix_len + kMvTile - 1) / kMvTile);
    int stages = kMixMaxStages, runacc_off = 0, prog_off = 0;
    size_t smem = 0;
    for (; stages >= 2; --stages)
        if ((smem = moving_tmem_smem_bytes(stages, k_max, &runacc_off, &prog_off)) != 0) break;
    if (stages < 2) return fail(ctx, HRIR_EINVAL, "the moving-source pipeline does not fit in shared memory");
    Partition part;
    part.U = (int64_t)n_tiles * n_src;
    part.P = std::min<int64_t>(ctx->num_sms, part.U);
    part.n_src = n_src;
    part.gs = kRunSources;
    int slots = 0;
    for (int t = 0; t < n_tiles; ++t) slots = std::max(slots, part.slots(t));
    const size_t pbytes = (size_t)n_tiles * slots * 2 * kMvTile * sizeof(float);
    int rc = grow(ctx, (void **)&ctx->d_partial, &ctx->partial_bytes, pbytes);
    if (rc) return rc;
    CUtensorMap tmap3;
    rc = make_source_rows32_map(ctx, &tmap3, src, len / 32, src_ld, n_src, kMvBufElems / 32);
    if (rc) return rc;
    MovingTmemArgs a{};
    a.src = src;
    a.ld = src_ld;
    a.len = len;
    a.n_src = n_src;
    a.n_seg = n_seg;
    a.seg_len = seg_len;
    a.k_max = k_max;
    a.tap_idx = tap_idx;
    a.tap_w = tap_w;
    a.tap_nnz = tap_nnz;
    a.refl_len = ctx->refl_len;
    a.rows = (int)(len / 32);
    a.stages = stages;
    a.fold = std::max(1, kFoldTerms / k_max);
    a.runacc_off = runacc_off;
    a.prog_off = prog_off;
    a.part = part;
    a.partial = ctx->d_partial;
    a.slots = slots;
    a.status = ctx->d_status;
    {
        KernelTimer kt(ctx, HRIR_K_MOVING, st);
        HRIR_CUDA_TRY(ctx, launch_moving_tmem(tmap3, a, (int)part.P, smem, st));
        kt.done();
    }
    ReduceArgs r;
    r.partial = ctx->d_partial;
    r.slots = slots;
    r.n_tiles = n_tiles;
    r.tile = kMvTile;
    r.part = part;
    r.res = ctx->d_res;
    r.res_len = ctx->res_len;
    r.out_len = out_len;
    r.out = out;
    r.out_ld = out_ld;
    {
        KernelTimer kt(ctx, HRIR_K_REDUCE, st);
        HRIR_CUDA_TRY(ctx, launch_reduce(r, st));
        kt.done();
    }
    return HRIR_OK;
}

}  // namespace

extern "C" {

int64_t hrir_mlp_param_count(int refl_len)
{
    if (refl_len < 1 || refl_len > 2048) return 0;
    return MlpLayout(refl_len).total;
}

int64_t hrir_mlp_act_stride(int refl_len)
{
    if (refl_len < 1 || refl_len > 2048) return 0;
    return act_stride(refl_len);
}

int hrir_mlp_forward(hrir_ctx *ctx, int64_t n_rows, const float *dirs, int refl_len,
                     const float *params, float *out, float *acts, void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    if (n_rows < 0 || refl_len < 1 || refl_len > 2048)
        return fail(ctx, HRIR_EINVAL, "bad sizes (n_rows=%lld refl_len=%d)", (long long)n_rows, refl_len);
    if (n_rows == 0) return HRIR_OK;
    if (!dirs || !params || !out) return fail(ctx, HRIR_EINVAL, "NULL buffer");
    if (n_rows > ((int64_t)1 << 31) - 1) return fail(ctx, HRIR_EINVAL, "n_rows must be < 2^31");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, HRIR_ECUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    const MlpLayout L(refl_len);
    const int64_t ld = act_stride(refl_len);
    const int64_t chunk = acts ? n_rows : std::min<int64_t>(n_rows, kFwdChunk);
    float *z = acts;
    if (!acts) {
        int rc = grow_ws(ctx, (size_t)chunk * ld * sizeof(float));
        if (rc) return rc;
        z = static_cast<float *>(ctx->d_mlp_ws);
    }
    KernelTimer kt(ctx, HRIR_K_MLP, st);
    for (int64_t r0 = 0; r0 < n_rows; r0 += chunk) {
        const int64_t nb = std::min(chunk, n_rows - r0);
        float *zc = acts ? acts + r0 * ld : z;
        HRIR_CUDA_TRY(ctx, launch_features_layer1((int)nb, dirs + r0 * 3, params + L.W1, params + L.b1,
                                                  zc, ld, nullptr, st));
        // layers 2, 3: z_{l+1} = W relu(z_l) + b
        for (int l = 0; l < 2; ++l) {
            GemmArgs g = gemm_args(nb, H, H, zc + l * H, ld, 1, params + (l ? L.W3 : L.W2), 1, H);
            g.bias = params + (l ? L.b3 : L.b2);
            g.Z = zc + (l + 1) * H;
            g.ldz = ld;
            HRIR_CUDA_TRY(ctx, launch_gemm_tc(0, true, false, g, 1, ctx->d_status, st));
        }
        // output layer: z4 = W4 relu(z3) + b4, g = softplus(z4)
        GemmArgs g = gemm_args(nb, refl_len, H, zc + 2 * H, ld, 1, params + L.W4, 1, H);
        g.bias = params + L.b4;
        g.Z = zc + 3 * H;
        g.ldz = ld;
        g.H = out + r0 * refl_len;
        g.ldh = refl_len;
        HRIR_CUDA_TRY(ctx, launch_gemm_tc(1, true, false, g, 1, ctx->d_status, st));
    }
    kt.done();
    return HRIR_OK;
}

int hrir_mlp_forward_bf16(hrir_ctx *ctx, int64_t n_rows, const float *dirs, int refl_len,
                          const float *params, float *out, void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    if (n_rows < 0 || refl_len < 1 || refl_len > 256)
        return fail(ctx, HRIR_EINVAL, "bad sizes (n_rows=%lld refl_len=%d; refl_len <= 256)",
                    (long long)n_rows, refl_len);
    if (n_rows == 0) return HRIR_OK;
    if (!dirs || !params || !out) return fail(ctx, HRIR_EINVAL, "NULL buffer");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, HRIR_ECUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    const MlpLayout L(refl_len);
    const int64_t chunk = std::min<int64_t>(n_rows, kTcChunk);
    // hidden activations in whole 128-row tiles (the tensor-core operand layout)
    const int64_t chunk_rows = round_up(chunk, 128);
    int rc = grow_ws(ctx, (size_t)chunk_rows * H * 2 * sizeof(__nv_bfloat16));
    if (rc) return rc;
    __nv_bfloat16 *h1 = static_cast<__nv_bfloat16 *>(ctx->d_mlp_ws);
    __nv_bfloat16 *h2 = h1 + (size_t)chunk_rows * H;
    KernelTimer kt(ctx, HRIR_K_MLP, st);
    for (int64_t r0 = 0; r0 < n_rows; r0 += chunk) {
        const int64_t nb = std::min(chunk, n_rows - r0);
        const int grid = (int)std::min<int64_t>(ctx->num_sms, (nb + 127) / 128);
        MlpTcArgs a{};
        a.n_rows = nb;
        a.dirs = dirs + r0 * 3;
        a.W1 = params + L.W1;
        a.b1 = params + L.b1;
        a.status = ctx->d_status;
        // layer 2 (layer 1 fused), layer 3, output layer
        for (int l = 0; l < 3; ++l) {
            a.first = l == 0;
            a.last = l == 2;
            a.in = l == 1 ? h1 : h2;
            a.W = params + (l == 0 ? L.W2 : l == 1 ? L.W3 : L.W4);
            a.b = params + (l == 0 ? L.b2 : l == 1 ? L.b3 : L.b4);
            a.N = l == 2 ? refl_len : H;
            a.n_pad = (int)round_up(a.N, 16);
            a.hout = l == 0 ? h1 : h2;
            a.out = out + r0 * refl_len;
            HRIR_CUDA_TRY(ctx, launch_mlp_layer_tc(a, grid, st));
        }
    }
    kt.done();
    return HRIR_OK;
}

int hrir_mlp_backward(hrir_ctx *ctx, int64_t n_rows, const float *dirs, int refl_len,
                      const float *params, const float *acts, const float *out, const float *target,
                      float *grads, float *loss, void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    if (n_rows < 1 || n_rows > (1 << 24) || refl_len < 1 || refl_len > 2048)
        return fail(ctx, HRIR_EINVAL, "bad sizes (n_rows=%lld refl_len=%d; 1 <= n_rows <= 2^24)",
                    (long long)n_rows, refl_len);
    if (!dirs || !params || !acts || !out || !target || !grads)
        return fail(ctx, HRIR_EINVAL, "NULL buffer");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, HRIR_ECUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    const MlpLayout L(refl_len);
    const int64_t ld = act_stride(refl_len);
    const int64_t B = n_rows;
    const int n_partial = (int)std::min<int64_t>(1024, (B * refl_len + 255) / 256);
    const int64_t splits_max = 64;
    const int64_t wmax = std::max<int64_t>(H, refl_len);
    // workspace: D4 [B][Lg], D0, D1 [B][256], X [B][8], P [splits][wmax][256] (also the
    // column sums' chunk partials, kColsumMaxChunks x wmax), loss partials
    static_assert(kColsumMaxChunks <= 64 * H, "column-sum partials fit in P");
    const size_t n4 = (size_t)B * refl_len, nh = (size_t)B * H, nx = (size_t)B * 8;
    const size_t np = (size_t)splits_max * wmax * H;
    const size_t need = (n4 + 2 * nh + nx + np + n_partial + 4) * sizeof(float);
    int rc = grow_ws(ctx, need);
    if (rc) return rc;
    float *D4 = static_cast<float *>(ctx->d_mlp_ws);
    float *D0 = D4 + n4;
    float *D1 = D0 + nh;
    float *X = D1 + nh;
    float *P = X + nx;
    float *part = P + np;
    const float *z1 = acts, *z2 = acts + H, *z3 = acts + 2 * H, *z4 = acts + 3 * H;

    KernelTimer kt(ctx, HRIR_K_MLP, st);
    HRIR_CUDA_TRY(ctx, launch_output_grad(B, refl_len, out, target, z4, ld, (float)(1.0 / (double)B), D4,
                                          part, n_partial, loss, st));
    // output layer
    rc = weight_grad(ctx, gemm_args(refl_len, H, (int)B, D4, 1, refl_len, z3, ld, 1), true, P,
                     grads + L.W4, st);
    if (rc) return rc;
    HRIR_CUDA_TRY(ctx, launch_colsum(B, refl_len, D4, refl_len, P, grads + L.b4, st));
    {
        GemmArgs g = gemm_args(B, H, refl_len, D4, refl_len, 1, params + L.W4, H, 1);
        g.mask = z3;
        g.ldm = ld;
        g.Z = D0;
        g.ldz = H;
        HRIR_CUDA_TRY(ctx, launch_gemm_tc(2, false, false, g, 1, ctx->d_status, st));
    }
    // hidden layers 3 and 2 (dZ in D0 -> weight grads, then dZ of the layer below in D1)
    const float *zin[2] = {z2, z1};
    const float *zmask[2] = {z2, z1};
    const int64_t offW[2] = {L.W3, L.W2}, offb[2] = {L.b3, L.b2};
    float *Dc = D0, *Dn = D1;
    for (int l = 0; l < 2; ++l) {
        rc = weight_grad(ctx, gemm_args(H, H, (int)B, Dc, 1, H, zin[l], ld, 1), true, P, grads + offW[l], st);
        if (rc) return rc;
        HRIR_CUDA_TRY(ctx, launch_colsum(B, H, Dc, H, P, grads + offb[l], st));
        GemmArgs g = gemm_args(B, H, H, Dc, H, 1, params + offW[l], H, 1);
        g.mask = zmask[l];
        g.ldm = ld;
        g.Z = Dn;
        g.ldz = H;
        HRIR_CUDA_TRY(ctx, launch_gemm_tc(2, false, false, g, 1, ctx->d_status, st));
        std::swap(Dc, Dn);
    }
    // first layer: its inputs are the features
    HRIR_CUDA_TRY(ctx, launch_features_layer1((int)B, dirs, params + L.W1, params + L.b1, nullptr, 0, X, st));
    rc = weight_grad(ctx, gemm_args(H, kMlpIn, (int)B, Dc, 1, H, X, 8, 1), false, P, grads + L.W1, st);
    if (rc) return rc;
    HRIR_CUDA_TRY(ctx, launch_colsum(B, H, Dc, H, P, grads + L.b1, st));
    kt.done();
    return HRIR_OK;
}

int hrir_mlp_adam(hrir_ctx *ctx, int64_t n, float *params, const float *grads, float *m, float *v,
                  int step, float lr, float beta1, float beta2, float eps, void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    if (n < 0 || step < 1 || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
        !(eps > 0.f) || !std::isfinite(lr))
        return fail(ctx, HRIR_EINVAL, "bad Adam arguments");
    if (n == 0) return HRIR_OK;
    if (!params || !grads || !m || !v) return fail(ctx, HRIR_EINVAL, "NULL buffer");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, HRIR_ECUDA, "cudaSetDevice failed");
    const double c1 = 1.0 / (1.0 - std::pow((double)beta1, step));
    const double c2 = 1.0 / (1.0 - std::pow((double)beta2, step));
    KernelTimer kt(ctx, HRIR_K_MLP, (cudaStream_t)stream);
    HRIR_CUDA_TRY(ctx, launch_adam(n, params, grads, m, v, lr, beta1, beta2, eps, (float)c1, (float)c2,
                                   (cudaStream_t)stream));
    kt.done();
    return HRIR_OK;
}

int hrir_render_moving(hrir_ctx *ctx, int n_src, int64_t len, int64_t src_ld, const float *src,
                       int n_seg, int seg_len, int k_max, const uint16_t *tap_idx, const float *tap_w,
                       const uint8_t *tap_nnz, int full, float *out, int64_t out_ld, void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    if (!ctx->loaded) return fail(ctx, HRIR_ESTATE, "no filters loaded (the resonance comes from them)");
    if (n_src < 0 || len < 0 || n_seg < 1 || seg_len < 128 || seg_len % 128 != 0 || k_max < 1 ||
        k_max > 255)
        return fail(ctx, HRIR_EINVAL,
                    "bad sizes (n_src=%d len=%lld n_seg=%d seg_len=%d k_max=%d; seg_len a multiple of 128)",
                    n_src, (long long)len, n_seg, seg_len, k_max);
    const int64_t out_len = full ? (len > 0 ? len + ctx->hrir_len - 1 : 0) : len;
    if (out_len == 0) return HRIR_OK;
    if (!out || out_ld < out_len) return fail(ctx, HRIR_EINVAL, "out is NULL or out_ld < %lld", (long long)out_len);
    if (len > ((int64_t)1 << 31) - 8192) return fail(ctx, HRIR_EINVAL, "len must be < 2^31 - 8192");
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, HRIR_ECUDA, "cudaSetDevice failed");
    if (n_src == 0) {
        HRIR_CUDA_TRY(ctx, cudaMemset2DAsync(out, (size_t)out_ld * 4, 0, (size_t)out_len * 4, 2, st));
        return HRIR_OK;
    }
    if (!src || !tap_idx || !tap_w || !tap_nnz) return fail(ctx, HRIR_EINVAL, "NULL buffer");
    if (src_ld < len || ((uintptr_t)src % 16) || (src_ld % 4))
        return fail(ctx, HRIR_EINVAL, "src must be 16-byte aligned with src_ld >= len, src_ld %% 4 == 0");
    const int64_t mix_len = std::min<int64_t>(out_len, len + ctx->refl_len - 1);
    // tensor-memory windows (moving_tmem.cu) where their shape rules hold: whole 32-sample rows
    // (len % 32 == 0), segments of >= 256 samples, <= 16 taps a row in 16-byte table rows,
    // reflection filters within the 224-offset window
    if (seg_len >= 256 && seg_len % 32 == 0 && k_max % 4 == 0 && k_max <= kMvMaxK && ctx->refl_len <= kMvSpan &&
        len % 32 == 0 && len > 0 && ((uintptr_t)tap_idx % 16) == 0 && ((uintptr_t)tap_w % 16) == 0)
        return render_moving_tmem(ctx, n_src, len, src_ld, src, n_seg, seg_len, k_max, tap_idx, tap_w, tap_nnz,
                                  mix_len, out_len, out, out_ld, st);
    const int n_tiles = (int)((mix_len + kMovTile - 1) / kMovTile);
    const int halo = (int)round_up(ctx->refl_len, 4);
    const int n_js = (kMovTile + seg_len - 1) / seg_len + 2;
    if (halo > kMovMaxHalo || (int64_t)n_js * 2 * k_max > kMovMaxTaps || n_js * 2 > 32)
        return fail(ctx, HRIR_EINVAL, "reflection filters too long (Lg <= %d) or too many taps for "
                    "the segment length (%d segments x 2 ears x k_max <= %d)", kMovMaxHalo, n_js, kMovMaxTaps);
    const size_t smem = moving_smem_bytes(halo, n_js, k_max);
    // one resident wave of persistent CTAs (each takes an equal share of the units)
    Partition part;
    part.U = (int64_t)n_tiles * n_src;
    part.P = std::min<int64_t>((int64_t)ctx->num_sms * moving_ctas_per_sm(smem), part.U);
    part.n_src = n_src;
    // each source's taps are summed in fresh registers and its contribution is one term of
    // the run's sum: runs of kRunSources sources are sums of that many terms
    part.gs = kRunSources;
    int slots = 0;
    for (int t = 0; t < n_tiles; ++t) slots = std::max(slots, part.slots(t));
    const size_t pbytes = (size_t)n_tiles * slots * 2 * kMovTile * sizeof(float);
    int rc = grow(ctx, (void **)&ctx->d_partial, &ctx->partial_bytes, pbytes);
    if (rc) return rc;
    MovingArgs a;
    a.src = src;
    a.ld = src_ld;
    a.len = len;
    a.n_src = n_src;
    a.n_seg = n_seg;
    a.seg_len = seg_len;
    a.k_max = k_max;
    a.tap_idx = tap_idx;
    a.tap_w = tap_w;
    a.tap_nnz = tap_nnz;
    a.refl_len = ctx->refl_len;
    a.halo = halo;
    a.n_js = n_js;
    a.bulk_tables = (k_max % 4 == 0) && ((uintptr_t)tap_idx % 16 == 0) && ((uintptr_t)tap_w % 16 == 0);
    a.part = part;
    a.partial = ctx->d_partial;
    a.slots = slots;
    a.status = ctx->d_status;
    {
        KernelTimer kt(ctx, HRIR_K_MOVING, st);
        HRIR_CUDA_TRY(ctx, launch_moving_mix(a, (int)part.P, smem, st));
        kt.done();
    }
    ReduceArgs r;
    r.partial = ctx->d_partial;
    r.slots = slots;
    r.n_tiles = n_tiles;
    r.tile = kMovTile;
    r.part = part;
    r.res = ctx->d_res;
    r.res_len = ctx->res_len;
    r.out_len = out_len;
    r.out = out;
    r.out_ld = out_ld;
    {
        KernelTimer kt(ctx, HRIR_K_REDUCE, st);
        HRIR_CUDA_TRY(ctx, launch_reduce(r, st));
        kt.done();
    }
    return HRIR_OK;
}

int hrir_resonance_per_source(hrir_ctx *ctx, int n_src, int64_t len, int64_t src_ld, hrir_dtype dt,
                              const void *src, int full, float *out, int64_t out_ld, void *stream)
{
    if (!ctx) return fail(nullptr, HRIR_EINVAL, "ctx is NULL");
    if (!ctx->loaded) return fail(ctx, HRIR_ESTATE, "no filters loaded (the resonance comes from them)");
    if (ctx->res_len > kResMaxLf)
        return fail(ctx, HRIR_EINVAL, "resonance length %d > %d", ctx->res_len, kResMaxLf);
    if (dt != HRIR_BF16 && dt != HRIR_F16)
        return fail(ctx, HRIR_EINVAL, "per-source resonance takes BF16 or FP16 sources");
    if (n_src < 0 || len < 0) return fail(ctx, HRIR_EINVAL, "negative n_src or len");
    const int64_t out_len = full ? (len > 0 ? len + ctx->res_len - 1 : 0) : len;
    if (out_len == 0 || n_src == 0) return HRIR_OK;
    if (!src || !out || out_ld < out_len) return fail(ctx, HRIR_EINVAL, "NULL buffer or out_ld too small");
    if (((uintptr_t)out % 16) || (out_ld % 4))
        return fail(ctx, HRIR_EINVAL, "out must be 16-byte aligned with out_ld %% 4 == 0");
    if (src_ld < len || ((uintptr_t)src % 16) || ((src_ld * 2) % 16))
        return fail(ctx, HRIR_EINVAL, "src must be 16-byte aligned with src_ld >= len and src_ld %% 8 == 0");
    if (len > (int64_t)1 << 31) return fail(ctx, HRIR_EINVAL, "len must be < 2^31");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, HRIR_ECUDA, "cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    CUtensorMap tmap;
    int rc = make_source_map(ctx, &tmap, src, (int)dt, len, src_ld, n_src, 1);
    if (rc) return rc;
    ResonanceArgs a;
    a.n_src = n_src;
    a.out_len = out_len;
    a.res = ctx->d_res;
    a.res_len = ctx->res_len;
    a.out = out;
    a.out_ld = out_ld;
    a.status = ctx->d_status;
    const int64_t units = ((out_len + kResTile - 1) / kResTile) * n_src;
    const int grid = (int)std::min<int64_t>(units, (int64_t)ctx->num_sms * 4);
    KernelTimer kt(ctx, HRIR_K_RESONANCE, st);
    HRIR_CUDA_TRY(ctx, launch_resonance_gemm((int)dt, tmap, a, grid, st));
    kt.done();
    return HRIR_OK;
}

}  // extern "C"
