/*
 * hrir.h -- C ABI of the GB300 (sm_103a) sparse factorized HRIR renderer.
 *
 * The method (Luo, Zotkin & Duraiswami, "Sparse Head-Related Impulse Response for
 * Efficient Direct Convolution"):
 *   Eq. 1      every HRIR is x = f * g: a direction-independent resonance filter f
 *              (per ear) convolved with a direction-dependent, sparse, non-negative
 *              reflection filter g;
 *   Eq. 2      y * x = (y * g) * f, so a source y is rendered with the K non-zero taps
 *              of g (direct convolution, Sec. I footnote 2) and the short dense f;
 *   Sec. IV-G  direct convolution costs NNZE multiply-adds per output sample.
 * The renderer mixes many sources, each at its own direction, into one stereo signal:
 *     out_e[n] = sum_s (f_e * g_{dir[s],e} * y_s)[n],   e in {0 = left, 1 = right}.
 * By linearity the resonance filter is applied once, after the mix (Eq. 2 with the sum
 * over sources moved inside).  The same tables also drive two plain-method baselines:
 * direct convolution with the dense HRIR f * g, and overlap-save FFT convolution
 * (Sec. I footnote 3, Sec. IV-G).
 *
 * Notation used below: Lg = reflection length (the paper's K in Eq. 1), K = number of
 * non-zero reflection taps (the paper's NNZE), Lf = resonance length (the paper's
 * M-K+1), H = Lf + Lg - 1 = HRIR length (the paper's M).
 *
 * Conventions
 *  - Every call returns an hrir_status (0 = HRIR_OK, negative = error); nothing aborts,
 *    traps or prints.  hrir_last_error() gives a message for the last failure on ctx.
 *  - "device" pointers are CUDA global-memory pointers on the context's device (for
 *    example torch.Tensor.data_ptr()); "host" pointers are ordinary CPU memory.
 *  - Work is enqueued on the caller's cudaStream_t (passed as void*; NULL = legacy
 *    default stream) and is asynchronous: the call returns before the GPU finishes.
 *  - Errors found on the device (a direction id out of range, a bounded wait that
 *    expired) set a flag in the context; hrir_sync() waits for the stream and returns
 *    the flag (then clears it).
 *  - The caller owns every buffer it passes in.  The library owns its filter tables and
 *    a workspace that it grows on demand and frees in hrir_destroy().
 *  - A context is used by one host thread at a time.
 */
#ifndef HRIR_H
#define HRIR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hrir_ctx hrir_ctx;

typedef enum {
    HRIR_OK = 0,
    HRIR_EINVAL = -1,     /* bad argument (message in hrir_last_error) */
    HRIR_ENOMEM = -2,     /* device or pinned-host allocation failed */
    HRIR_ECUDA = -3,      /* a CUDA runtime call failed */
    HRIR_ETIMEDOUT = -4,  /* a bounded device-side wait expired (kernel returned early) */
    HRIR_EBUSY = -5,      /* resource temporarily unavailable (admission refused) */
    HRIR_ESTATE = -6      /* call not valid in the current state (e.g. no filters loaded) */
} hrir_status;

typedef enum { HRIR_F32 = 0, HRIR_BF16 = 1, HRIR_F16 = 2 } hrir_dtype;

typedef enum {
    HRIR_SPARSE = 0,  /* sparse reflection gather-FMA, mix, then resonance FIR (Eq. 2)  */
    HRIR_DENSE = 1,   /* direct convolution with the dense HRIR f * g (Eq. 1)           */
    HRIR_FFT = 2      /* overlap-save FFT convolution with the dense HRIR (fn. 3)       */
} hrir_mode;

/* Library version, (major << 16) | minor. */
int hrir_version(void);

/* Create a context on CUDA device `device` (cudaSetDevice is called on it).  *out receives
 * the new context or NULL.  HRIR_ECUDA if the device cannot be used. */
int hrir_create(hrir_ctx **out, int device);

/* Free the context, its tables and workspace.  Waits for the context's own work.  NULL ok. */
void hrir_destroy(hrir_ctx *ctx);

/* Message for the most recent failing call on ctx (ctx may be NULL: then the message of the
 * last failing hrir_create on this thread).  Never NULL; valid until the next call. */
const char *hrir_last_error(const hrir_ctx *ctx);

/* Wait for all work enqueued on `stream`, then return and clear any device-side error flag:
 * HRIR_EINVAL (a direction id was out of range, that source rendered as silence, a
 * device tap table of hrir_render_moving held an invalid entry, which was ignored, an
 * hrir_sparsify row hit the solver's limits, or an hrir_factorize resonance system was not
 * positive definite),
 * HRIR_ETIMEDOUT (a bounded wait expired; the output of that call is incomplete), or
 * HRIR_ECUDA if the stream reported a CUDA error. */
int hrir_sync(hrir_ctx *ctx, void *stream);

/* Self-test of the failure path: enqueues on `stream` one thread that waits on a device
 * barrier nothing ever completes, through the same bounded wait the pipelined kernels use.
 * After the wait limit (1 s) it sets the context's timeout flag and returns, so the next
 * hrir_sync(ctx, stream) returns HRIR_ETIMEDOUT (and clears the flag); the context stays
 * usable.  Returns HRIR_OK once enqueued. */
int hrir_selftest_wait_timeout(hrir_ctx *ctx, void *stream);

/* ---------------------------------------------------------------------------------------
 * Filter pack: top-K sparsification of non-negative reflection rows (a device kernel).
 * Follows the NNZE budget of Sec. III-D: from each row of g keep the K largest strictly
 * positive values (larger value first; on equal values the smaller index), then store
 * them in ascending index order, padding unused slots with (0, 0.0f).
 *   g     device, float [n_rows][refl_len], row-major, any values (NaN/negatives are
 *         never selected).  1 <= refl_len <= 2048.
 *   idx   device, uint16 [n_rows][k]    out
 *   w     device, float  [n_rows][k]    out
 *   nnz   device, uint8  [n_rows]       out (number of kept taps, <= k)
 *   0 <= k <= 255.  Bit-exact: indices and weights are copies of input entries.
 * Speed (not the result) depends on the rows' order: each warp walks a contiguous run of rows
 * and starts a row's search from the threshold it found two rows before, which is what the
 * (..., ear) row order of the learned filters offers; refl_len % 8 == 0 (<= 256) with a
 * 16-byte aligned g takes the faster 16-byte loads.
 * ------------------------------------------------------------------------------------- */
int hrir_topk_pack(hrir_ctx *ctx, int n_rows, int refl_len, int k, const float *g,
                   uint16_t *idx, float *w, uint8_t *nnz, void *stream);

/* ---------------------------------------------------------------------------------------
 * Load the factorized filters (Sec. II: f per ear, g per direction and ear).  All
 * pointers are HOST memory; the data is copied (the caller keeps ownership) and the
 * device tables are built by kernels: the sparse tap programs for HRIR_SPARSE, the dense
 * HRIRs x = f * g (Eq. 1) for HRIR_DENSE and their spectra for HRIR_FFT.  Replaces any
 * previously loaded filters; blocks until the tables are ready.
 *   n_dirs     >= 1 directions;  n_ears must be 2.
 *   refl_len   Lg, 1 .. 2048;  k_max 0 .. 255 slots per (direction, ear).
 *   tap_idx    uint16 [n_dirs][2][k_max]: the first nnz entries strictly ascending, < Lg.
 *   tap_w      float  [n_dirs][2][k_max]: finite and >= 0 (g >= 0, Eq. 1).
 *   tap_nnz    uint8  [n_dirs][2]: used slots, <= k_max.
 *   res_len    Lf, 1 .. 512;  resonance float [2][res_len], finite.
 *   fft_size   overlap-save frame P for HRIR_FFT: 0 or 4096 (the frame the FFT kernels
 *              implement; H - 1 rounded up to 8 must be < P), anything else is HRIR_EINVAL.
 * ------------------------------------------------------------------------------------- */
int hrir_load_filters(hrir_ctx *ctx, int n_dirs, int n_ears, int refl_len, int k_max,
                      const uint16_t *tap_idx, const float *tap_w, const uint8_t *tap_nnz,
                      int res_len, const float *resonance, int fft_size);

/* Output length of a render: len + H - 1 when full != 0, else len (the first len
 * samples of the full linear convolution, Sec. I footnote 2).  0 when len == 0. */
int64_t hrir_out_len(const hrir_ctx *ctx, int64_t len, int full);

/* ---------------------------------------------------------------------------------------
 * Render n_src sources into one stereo mix (Eqs. 1-2), on the device.
 *   src     device, [n_src][src_ld] of dtype dt; source s is src[s][0 .. len-1].  The base
 *           must be 16-byte aligned and src_ld*sizeof(dt) a multiple of 16; columns
 *           >= len are never read.  HRIR_BF16/HRIR_F16 sources are widened to FP32 and
 *           all arithmetic is FP32.
 *   dir     device, int32 [n_src], direction of each source (0 .. n_dirs-1; an id out of
 *           range renders that source as silence and flags HRIR_EINVAL for hrir_sync).
 *   mode    HRIR_SPARSE (the method), HRIR_DENSE or HRIR_FFT (plain-method baselines).
 *   full    1: out_len = len + H - 1, 0: out_len = len.
 *   out     device, float [2][out_ld] (row 0 left, row 1 right), out_ld >= out_len;
 *           columns [0, out_len) are overwritten, the rest untouched.
 *   stream  cudaStream_t to enqueue on.
 * Every source is read once per render; the mix is deterministic (fixed summation order
 * for a given device and shape).  Accuracy: no FP32 sum in the mix runs over more than a
 * few hundred products (HRIR_SPARSE: registers folded every ~128 products into per-lane
 * accumulators, flushed every 64 sources; HRIR_DENSE: runs of 8 sources), the runs'
 * partial sums are added with compensation (Kahan) and the resonance stage is a
 * compensated dot product.  n_src == 0 writes zeros; len == 0 writes nothing.
 * ------------------------------------------------------------------------------------- */
int hrir_render_batch(hrir_ctx *ctx, int n_src, int64_t len, int64_t src_ld, hrir_dtype dt,
                      const void *src, const int32_t *dir, hrir_mode mode, int full,
                      float *out, int64_t out_ld, void *stream);

/* Same as hrir_render_batch with HOST buffers: src [n_src][src_ld], dir [n_src] and out
 * [2][out_ld] live in CPU memory (page-locked memory gives the fastest copies).  The
 * call copies the sources to the device on a stream of the context, in up to 4 chunks of
 * sources (16 or more sources; one chunk otherwise); each chunk is rendered on `stream` as
 * soon as it has landed, while the next ones copy, and the chunk mixes are summed in chunk
 * order.  The result equals hrir_render_batch's up to the order of the FP32 sums (and is
 * deterministic); the call returns when `out` holds it.  Device staging space comes from the
 * context workspace; `dir` is first copied into a page-locked buffer the context keeps (grown
 * when a call has more sources than any before it). */
int hrir_render_batch_host(hrir_ctx *ctx, int n_src, int64_t len, int64_t src_ld,
                           hrir_dtype dt, const void *src, const int32_t *dir, hrir_mode mode,
                           int full, float *out, int64_t out_ld, void *stream);

/* ---------------------------------------------------------------------------------------
 * Block streaming with continuous batching: partitioned time-domain convolution, which adds
 * no latency and needs no extra memory when split into blocks (Sec. IV-G), on the filters
 * of Eqs. 1-2.
 *
 * hrir_stream_open  Opens the context's stream: blocks of `block` (128 or 256) samples, at most
 *                   max_slots sources at once, a device pool of pool_bytes for source samples;
 *                   steps run on `stream`.  Captures the step as a CUDA graph.  Closes any
 *                   previous stream; hrir_load_filters also closes it.
 * hrir_stream_admit Admits one source (HOST samples [len], FP32; page-locked memory uploads
 *                   fastest) into session `session` at direction dir.  Returns HRIR_EBUSY when
 *                   no slot is free and HRIR_ENOMEM when the pool has no room: the request was
 *                   not admitted and may be retried after later steps free resources.  The
 *                   upload runs on a copy stream, overlapping earlier steps; the source joins
 *                   the next step (which waits for the upload on the GPU), starting at that
 *                   step's block.  host_src must stay valid until that step has returned.
 *                   Sources of one session are mixed into one stereo stream.
 * hrir_stream_step  Renders one block for every session that has a ready source and waits for
 *                   it.  *out_blocks points to n_out blocks [n_out][2][block] (FP32, row r
 *                   belongs to session (*out_sessions)[r]); both arrays stay valid until the
 *                   next step.  done_ids (capacity max_slots, may be NULL) receives the ids of
 *                   the *n_done requests that finished in this step: a source finishes after
 *                   len + H - 1 samples (its full convolution) have been emitted.
 * hrir_stream_stats Active (rendering) and pending (admitted, not yet stepped) sources and pool
 *                   bytes in use.
 * hrir_stream_close Releases the stream (waits for its work).
 * ------------------------------------------------------------------------------------- */
int hrir_stream_open(hrir_ctx *ctx, int block, int max_slots, size_t pool_bytes, void *stream);
int hrir_stream_admit(hrir_ctx *ctx, int64_t req_id, int64_t session, const float *host_src,
                      int64_t len, int dir);
int hrir_stream_step(hrir_ctx *ctx, const float **out_blocks, const int64_t **out_sessions,
                     int *n_out, int64_t *done_ids, int *n_done);
int hrir_stream_stats(hrir_ctx *ctx, int *active, int *pending, int64_t *pool_used_bytes);
int hrir_stream_close(hrir_ctx *ctx);

/* ---------------------------------------------------------------------------------------
 * hrir_render_batch_noalloc -- the same render as hrir_render_batch (HRIR_SPARSE or
 * HRIR_DENSE, same arguments, same result), for callers that must not allocate device
 * memory while rendering: real-time audio threads, where an allocator call can block for an
 * unbounded time, and hosts that hand the library a fixed device-memory budget up front.
 * The paper has no counterpart to this call; it exists only for those callers.
 *
 * hrir_render_batch keeps its partial sums in a workspace that it grows with cudaMalloc.
 * This call uses instead a fixed 32 MiB array of device memory; it calls no cudaMalloc,
 * cudaFree or other allocating routine.  Renders whose partial sums need more than 32 MiB
 * (about n_tiles * (ceil(n_src / 64) + 2) * 52 KiB, n_tiles = ceil((len + Lg - 1) / 6656)
 * for HRIR_SPARSE; n_tiles * (ceil(n_src / 8) + 2) * 72 KiB, n_tiles = ceil((len + H - 1) /
 * 9216) for HRIR_DENSE) are rejected with HRIR_EINVAL and a message giving the size needed.
 * Set-up on first use: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current).  Under CUDA's lazy module loading (the
 * default) that lookup is also when the driver loads the array and reserves its 32 MiB, so
 * the first call can block in the driver or fail with HRIR_ENOMEM.  Make one call at set-up
 * time, before the real-time phase and before any stream capture; from then on the device
 * holds the array until the process exits and later calls allocate nothing.
 * Every call shares the one array, so calls whose GPU work overlaps in time (on different
 * streams or from different contexts) race on it: serialize them.  Nothing in the array
 * needs to be cleared between calls.  This call's kernels are not timed by hrir_set_timing
 * (timing would create CUDA events).
 * ------------------------------------------------------------------------------------- */
int hrir_render_batch_noalloc(hrir_ctx *ctx, int n_src, int64_t len, int64_t src_ld,
                              hrir_dtype dt, const void *src, const int32_t *dir,
                              hrir_mode mode, int full, float *out, int64_t out_ld,
                              void *stream);

/* ---------------------------------------------------------------------------------------
 * Learned reflection filters.  The paper fits one non-negative reflection filter g per
 * measured direction (Sec. III, Eq. 3 with G >= 0, Algorithm 1).  These calls run a small
 * network that maps a direction to such a filter, so that directions between the measured
 * ones get filters too (moving sources):
 *     x  = (sin az, cos az, sin el, cos el, ear)         ear = -1 (left) or +1 (right)
 *     h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), h3 = relu(W3 h2 + b3)     (256 wide)
 *     g  = softplus(W4 h3 + b4)                           Lg taps, every one > 0
 * trained by least squares on factorized reflection rows T (Algorithm 1 output):
 *     L = 1/(2B) sum_b ||g_b - T_b||^2 over a batch of B rows,
 * with Adam (Kingma & Ba 2015).  All arithmetic is FP32; all pointers are device memory.
 *
 * params  float [hrir_mlp_param_count(Lg)]: W1 [256][5], b1 [256], W2 [256][256], b2,
 *         W3 [256][256], b3, W4 [Lg][256], b4 [Lg], concatenated, matrices row-major.
 * dirs    float [n_rows][3]: {azimuth, elevation (radians), ear (-1 or +1)} per row.
 * acts    float [n_rows][hrir_mlp_act_stride(Lg)]: the pre-activations of the four layers
 *         (z1 | z2 | z3 | z4) that the backward pass needs.
 *
 * hrir_mlp_param_count  number of parameters (184520 for Lg = 200); 0 if Lg is out of range.
 * hrir_mlp_act_stride   row stride of acts (floats).
 * hrir_mlp_forward      out [n_rows][Lg] = g for every row; acts is filled when not NULL
 *                       (otherwise the context workspace holds the activations in chunks).
 * hrir_mlp_forward_bf16 the same filters for inference on the tensor cores: weights and
 *                       activations rounded to BF16, FP32 accumulation, FP32 output; the
 *                       features and the softplus use the hardware approximations of sin,
 *                       cos, exp and log (errors far below the BF16 rounding).  Lg <= 256; the
 *                       hidden activations stay in the context workspace.  For the millions
 *                       of rows of moving sources; agrees with hrir_mlp_forward to BF16
 *                       precision.
 * hrir_mlp_backward     grads [param_count] = dL/dparams for the batch whose forward pass left
 *                       `acts` and `out`; target [n_rows][Lg]; loss (device float, may be
 *                       NULL) = L.  1 <= n_rows <= 2^24.  Deterministic (fixed-order sums).
 * hrir_mlp_adam         one Adam step t = step (>= 1) on n parameters: m and v are the first
 *                       and second moments (zero before step 1), updated in place.
 * Filters for rendering come from hrir_mlp_forward followed by hrir_topk_pack.
 * ------------------------------------------------------------------------------------- */
int64_t hrir_mlp_param_count(int refl_len);
int64_t hrir_mlp_act_stride(int refl_len);
int hrir_mlp_forward(hrir_ctx *ctx, int64_t n_rows, const float *dirs, int refl_len,
                     const float *params, float *out, float *acts, void *stream);
int hrir_mlp_forward_bf16(hrir_ctx *ctx, int64_t n_rows, const float *dirs, int refl_len,
                          const float *params, float *out, void *stream);
int hrir_mlp_backward(hrir_ctx *ctx, int64_t n_rows, const float *dirs, int refl_len,
                      const float *params, const float *acts, const float *out,
                      const float *target, float *grads, float *loss, void *stream);
int hrir_mlp_adam(hrir_ctx *ctx, int64_t n, float *params, const float *grads, float *m,
                  float *v, int step, float lr, float beta1, float beta2, float eps,
                  void *stream);

/* ---------------------------------------------------------------------------------------
 * Moving sources: Eqs. 1-2 with a direction per segment of seg_len samples.  Source s uses
 * the reflection filter g_{s,j} in segment j (samples [j seg_len, (j+1) seg_len)); between
 * segments the reflection output is cross-faded linearly in the output domain:
 *     z[n] = (1 - a) (y * g_{s,j-1})[n] + a (y * g_{s,j})[n],  a = (n - j seg_len + 1) / seg_len,
 * segment 0 uses g_{s,0} alone and outputs past the last segment use g_{s,n_seg-1} alone.
 * The mix over sources is followed by the loaded resonance filter f (hrir_load_filters must
 * have been called: f and Lg come from it); output as in hrir_render_batch.
 *   src       device float [n_src][src_ld], 16-byte aligned, src_ld % 4 == 0.
 *   tap_idx   device uint16 [n_src][n_seg][2][k_max] (indices < Lg, any order),
 *   tap_w     device float  [n_src][n_seg][2][k_max], tap_nnz device uint8 [n_src][n_seg][2]
 *             (the layout hrir_topk_pack writes for rows ordered (source, segment, ear)).
 *             With k_max % 4 == 0 and 16-byte aligned tap_idx and tap_w the tables are
 *             staged by bulk copies; any other k_max works, more slowly.
 *             An index >= Lg or a count > k_max is ignored and flags HRIR_EINVAL for
 *             hrir_sync.
 *   seg_len   a multiple of 128;  1 <= k_max <= 255.
 * With seg_len >= 256, len % 32 == 0, k_max % 4 == 0, k_max <= 16, Lg <= 224 and 16-byte
 * aligned tables the mix runs on tensor-memory windows (per lane quarter, the union of the
 * tap offsets of the segments it spans is applied with each row's weight, 0 where a row lacks
 * an offset); otherwise it gathers the source samples from shared memory.  Both give the
 * same sums up to FP32 rounding order.
 * ------------------------------------------------------------------------------------- */
int hrir_render_moving(hrir_ctx *ctx, int n_src, int64_t len, int64_t src_ld, const float *src,
                       int n_seg, int seg_len, int k_max, const uint16_t *tap_idx,
                       const float *tap_w, const uint8_t *tap_nnz, int full, float *out,
                       int64_t out_ld, void *stream);

/* ---------------------------------------------------------------------------------------
 * The resonance stage applied per source, u_{s,e} = y_s * f_e (Sec. I footnote 2), the
 * first half of Eq. 2 in the order (y * f) * g, which the paper notes can be precomputed
 * when y is known in advance: u can then be rendered to any direction or trajectory with
 * the reflection taps alone.  Computed on the tensor cores as a Toeplitz-block GEMM: every
 * block of 32 outputs is one row of (Hankel window of y) x (Toeplitz matrix of f), with f
 * split into three terms of the source's 16-bit type so that the FP32 accumulation gives
 * y * f to about FP32 accuracy.  Uses the resonance of hrir_load_filters (Lf <= 32).
 *   dt        HRIR_BF16 or HRIR_F16 (the sources' storage type).
 *   src       device [n_src][src_ld] of dt, 16-byte aligned, src_ld % 8 == 0.
 *   full      1: out_len = len + Lf - 1;  0: out_len = len.
 *   out       device float [n_src][2][out_ld] (source s, ear e at out[(2 s + e) out_ld]),
 *             16-byte aligned, out_ld >= out_len and out_ld % 4 == 0.
 * ------------------------------------------------------------------------------------- */
int hrir_resonance_per_source(hrir_ctx *ctx, int n_src, int64_t len, int64_t src_ld,
                              hrir_dtype dt, const void *src, int full, float *out,
                              int64_t out_ld, void *stream);

/* ---------------------------------------------------------------------------------------
 * Filter production on the device: the factorization x_i = f * g_i of a set of HRIRs
 * (Eq. 1) by Algorithm 1's alternating minimisation of ||X - F~ G^T||_F^2 (Eq. 3 with
 * F = F~, the banded Toeplitz matrix of f, Eq. 12), per ear.  Each of `iters` rounds:
 *   (1) the least-squares resonance for the current G: the normal equations of Eqs. 9-11
 *       over the Lf free parameters of Eq. 13, A f = b with A[l][l'] = sum_j (G^T G)[j][j + |l
 *       - l'|] and b[l] = sum_j (X^T G)[j + l][j], solved by Cholesky;
 *   (2) the multiplicative non-negative update of G (Eq. 4):
 *       G_ij <- G_ij sqrt(((X F~)+_ij + [G (F~^T F~)-]_ij) / ((X F~)-_ij + [G (F~^T F~)+]_ij)),
 *       Q+- = (|Q| +- Q) / 2; entries equal to 0 stay 0.
 *   X      device float [n_dirs][n_ears][M], the HRIRs (rows here), M = hrir_len
 *   G      device float [n_dirs][n_ears][Lg]: the start on entry (>= 0; Algorithm 1 draws it
 *          at random, the caller passes it in), the result on return
 *   f      device float [n_ears][Lf] out, Lf = M - Lg + 1 (1 <= Lf <= 64): the resonance of
 *          the last round
 *   trace  device float [n_ears][iters + 1] out (may be NULL): ||X - F~ G^T||_F^2 after the
 *          first solve with the starting G, then after each round's update
 *   normalise != 0: f scaled to unit L2 norm and G by the inverse factor (F~ G^T unchanged).
 * The products (G^T G, X^T G, X F~, G Q+-) run on the tensor cores to FP32 accuracy (each
 * FP32 value split into three BF16 terms, FP32 accumulation), the Toeplitz sums and the
 * Cholesky solve in FP64, the residuals from the definition (f * g per row) summed in FP64.
 * A system that is not positive definite (a G without energy) flags HRIR_EINVAL for
 * hrir_sync.  1 <= n_ears <= 2, 1 <= Lg <= 1024, iters >= 1; workspace from the context.
 * ------------------------------------------------------------------------------------- */
int hrir_factorize(hrir_ctx *ctx, int n_dirs, int n_ears, int hrir_len, int refl_len, const float *X,
                   float *G, float *f, float *trace, int iters, int normalise, void *stream);

/* ---------------------------------------------------------------------------------------
 * The sparsifying fine-tune of Algorithm 1 (Sec. III-D), on the device,
 * so that variable-NNZE tap tables for hrir_load_filters can be made from HRIRs and their
 * factorized resonance without leaving the GPU.  Per direction and ear, with the
 * resonance f fixed (F~ = its banded Toeplitz matrix, Eq. 12):
 *     g_i = argmin_{g >= 0} ||D (F~ g - x_i)||^2 + lam sum_j g_j                   (Eq. 14)
 * with D = I (sigma <= 0) or the window transform D_W = diag(exp(-m^2 / sigma^2)),
 * m = 0..M-1 (Eq. 16), solved exactly by an active-set method (Lawson & Hanson's scheme on
 * the normal-equation form); then entries <= thresh are set to 0 (the paper discards those
 * below 1e-4).  All arrays are device memory, row-major, directions outermost:
 *   X    float [n_dirs][n_ears][M]   the HRIRs, M = hrir_len = Lf + Lg - 1
 *   f    float [n_ears][Lf]          the resonance of each ear (1 <= Lf <= 64)
 *   G    float [n_dirs][n_ears][Lg]  out: the sparse non-negative reflection filters
 *   nnz  int32 [n_dirs][n_ears]      out (may be NULL): non-zeros kept per row
 * FP32 arithmetic; Q = F~^T D^2 F~, c = F~^T D^2 x - lam/2 and every residual are formed in
 * double-float (error-free transformations) and the support systems are solved by FP32
 * Cholesky with iterative refinement, so the result agrees with an FP64 solution to FP32
 * accuracy (no FP64 arithmetic on the device).  A row whose support would exceed the
 * solver's limit (min(Lg, 128), less if shared memory is short) or whose solve runs over
 * 1 s keeps its last feasible iterate and flags HRIR_EINVAL for hrir_sync.
 * 1 <= n_ears <= 2, lam >= 0, thresh >= 0; workspace from the context.  Tap tables follow
 * from G with hrir_topk_pack (k = the largest nnz keeps every non-zero).
 * ------------------------------------------------------------------------------------- */
int hrir_sparsify(hrir_ctx *ctx, int n_dirs, int n_ears, int hrir_len, int refl_len,
                  const float *X, const float *f, float lam, float sigma, float thresh, float *G,
                  int32_t *nnz, void *stream);

/* ---------------------------------------------------------------------------------------
 * Source sharding.  The render is linear in the sources and the resonance f of Eq. 2 is the
 * same for all of them (Sec. II), so a batch can be split into disjoint source sets (for
 * example one per GPU) whose reflection mixes are added once, before f is applied:
 *     out_e = f_e * sum_c z_{c,e},   z_{c,e} = sum_{s in set c} y_s * g_{d(s),e}.
 * hrir_render_reflections(..., full, z, z_ld) followed by hrir_apply_resonance(1 part, full)
 * gives hrir_render_batch(HRIR_SPARSE, full) up to the order of the FP32 sums.
 *
 * hrir_render_reflections  The reflection mix z of one source set with the sparse taps alone
 *                          (the HRIR_SPARSE path without the resonance stage).  Arguments as
 *                          hrir_render_batch; z device float [2][z_ld], z_len = full ? len +
 *                          Lg - 1 : len, columns [0, z_len) overwritten.
 * hrir_apply_resonance     out_e[n] = sum_{l < Lf} f_e[l] z_e[n - l] with z_e = the sum, in part
 *                          order (compensated), of n_parts >= 1 reflection mixes: z device
 *                          float [n_parts][2][part_ld], part c ear e at z + (2 c + e) part_ld,
 *                          z_len samples each (part_ld >= z_len).  out device float [2][out_ld],
 *                          out_len = full ? z_len + Lf - 1 : z_len.  The FIR is the same
 *                          compensated dot product as hrir_render_batch's resonance stage.
 * Both use the filters of hrir_load_filters.
 * ------------------------------------------------------------------------------------- */
int hrir_render_reflections(hrir_ctx *ctx, int n_src, int64_t len, int64_t src_ld, hrir_dtype dt,
                            const void *src, const int32_t *dir, int full, float *z, int64_t z_ld,
                            void *stream);
int hrir_apply_resonance(hrir_ctx *ctx, int n_parts, int64_t z_len, int64_t part_ld, const float *z,
                         int full, float *out, int64_t out_ld, void *stream);

/* ---------------------------------------------------------------------------------------
 * Rendering precomputed resonance outputs to several direction sets: the order (y * f) * g of
 * Eq. 2.  Given u_{s,e} = y_s * f_e for every source (for example from
 * hrir_resonance_per_source, which the paper's remark on precomputing y * f for sources
 * known in advance motivates), each view v mixes the sources at its own directions with the
 * reflection taps alone (no resonance is applied here):
 *     out_v,e[n] = sum_s (u_{s,e} * g_{dir[v][s], e})[n].
 *   u        device float [n_src][2][u_ld] (source s, ear e at u + (2 s + e) u_ld), 16-byte
 *            aligned, u_ld % 4 == 0; u_{s,e}[0 .. len) is read.
 *   dir      device int32 [n_views][n_src]: the direction of each source in each view (an id
 *            out of range renders that source as silence and flags HRIR_EINVAL for hrir_sync).
 *   full     1: out_len = len + Lg - 1, 0: out_len = len.
 *   out      device float, view v at out + v view_ld: [2][out_ld] (row 0 left, row 1 right),
 *            out_ld >= out_len, view_ld >= 2 out_ld; columns [0, out_len) overwritten.
 * Each view reads u once (2 rows per source, one per ear) and applies each source's taps of
 * one ear to each row; the partition, run lengths and fixed summation order are those of
 * hrir_render_batch (deterministic).  Uses the filters of hrir_load_filters.
 * ------------------------------------------------------------------------------------- */
int hrir_render_precomputed(hrir_ctx *ctx, int n_src, int64_t len, int64_t u_ld, const float *u,
                            int n_views, const int32_t *dir, int full, float *out, int64_t out_ld,
                            int64_t view_ld, void *stream);

/* ---------------------------------------------------------------------------------------
 * Optional kernel timing, for benchmarks.  While enabled, the library brackets each of its
 * kernel launches with CUDA events recorded on the launching stream.  hrir_kernel_times
 * waits for those events and writes, per kernel family (hrir_kernel), the accumulated
 * milliseconds and launch counts since the last reset (arrays of HRIR_K_COUNT entries;
 * either may be NULL).  reset != 0 clears the accumulators after reading.
 * ------------------------------------------------------------------------------------- */
typedef enum {
    HRIR_K_MIX_SPARSE = 0,  /* sparse reflection gather-FMA mixing kernel */
    HRIR_K_MIX_DENSE = 1,   /* dense-HRIR direct-convolution mixing kernel */
    HRIR_K_REDUCE = 2,      /* fixed-order partial reduction + resonance FIR */
    HRIR_K_FFT = 3,         /* overlap-save FFT kernels */
    HRIR_K_TABLES = 4,      /* filter-pack kernels (top-K, records) */
    HRIR_K_MLP = 5,         /* learned-filter network kernels (forward, backward, Adam) */
    HRIR_K_MOVING = 6,      /* moving-source crossfade mixing kernel */
    HRIR_K_RESONANCE = 7,   /* per-source resonance on the tensor cores */
    HRIR_K_FILTERS = 8,     /* filter production (L1-NNLS fine-tune) */
    HRIR_K_COUNT = 9
} hrir_kernel;

int hrir_set_timing(hrir_ctx *ctx, int enable);
int hrir_kernel_times(hrir_ctx *ctx, double *ms, int64_t *launches, int reset);

#ifdef __cplusplus
}
#endif

#endif /* HRIR_H */
