// kernels.h -- internal launchers of the sm_103a renderer (not part of the C ABI).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace hrir {

// ---- direct-convolution mixing (sparse reflection taps, or dense HRIR) -----------------
// Outputs per lane and warps per CTA of each mixing kernel.  Dense: all warps compute, warp 0
// also issues the TMA loads, and the tile is warps x 32 lanes x R outputs.
#ifndef HRIR_DENSE_R
#define HRIR_DENSE_R 36
#endif
#ifndef HRIR_DENSE_WARPS
#define HRIR_DENSE_WARPS 8
#endif
// Sparse kernel: windows in tensor memory.  4 TMEM lane quarters x 32 lanes x R = 52
// consecutive outputs per lane (tile 6656); the two tap warps of a lane quarter (one per ear)
// read a window of kSparseTmemCols samples = one segment of kSparseSegment filter offsets
// plus the lane's outputs, which the quarter's copy warp writes, double-buffered in the 512
// TMEM columns (16 tap warps + 4 copy warps + 1 warp that issues the TMA loads).
constexpr int kSparseR = 52, kSparseWarps = 21, kSparseQuarters = 4;
constexpr int kSparseTile = kSparseQuarters * 32 * kSparseR;
constexpr int kSparseTmemCols = 256;
constexpr int kSparseSegment = kSparseTmemCols - kSparseR;  // 204
// per-lane FP32 fold accumulators of the 16 tap warps (26 outputs per lane each)
constexpr int kSparseRunAccBytes = 16 * 32 * (kSparseR / 2) * 4;
constexpr int kDenseR = HRIR_DENSE_R, kDenseWarps = HRIR_DENSE_WARPS;
constexpr int kMixMaxStages = 6;
constexpr int kMixDirCache = 2048;                // unit directions staged in shared memory
// shared memory after the stage ring and its barriers: 16 window barriers (sparse kernel),
// abort flag + TMEM slot (16 B), the per-stage release counters and last issued units, the
// direction cache
constexpr int kMixWindowBars = 16;
constexpr int kMixSmemTail = kMixWindowBars * 8 + 16 + 2 * kMixMaxStages * 4 + kMixDirCache * 4;
constexpr int kMixBox = 256;                      // TMA box width (elements)
constexpr int kRunSources = 64;                   // max sources per partial slot (a run)
// Accuracy of the FP32 mix.  The rounding error of a sequential FP32 sum of n terms grows as
// sqrt(n), and the resonance stage, applied after the mix, can magnify the mix's relative
// error where f attenuates the band that holds the sources' energy.  So every sum is kept
// short or split in two levels:
//  * sparse kernel: its tap registers are folded every kFoldTerms products (fold = max(1,
//    kFoldTerms / K) sources) into a per-lane FP32 accumulator in shared memory, which is
//    flushed to the run's partial slot every kRunSources sources (sums of at most ~128
//    and 64 terms at the two levels);
//  * dense kernel (231 products per source): runs of kDenseRunSources sources;
//  * moving-source kernel: each source's taps are summed in fresh registers, so its runs of
//    kRunSources sources are already sums of kRunSources terms.
constexpr int kFoldTerms = 128;
constexpr int kDenseRunSources = 8;

enum MixMode : int { MIX_SPARSE = 0, MIX_DENSE = 1 };

struct MixArgs {
    const void *src;            // [n_src][ld] sources
    int64_t ld;                 // row stride in elements
    int64_t len;                // samples per source
    int n_src;
    const int32_t *dir;         // [n_src]
    int n_dirs;
    const unsigned char *table; // per-direction records (n_dirs + 1, last one silent)
    int rec_bytes;              // record stride, multiple of 16
    int nchunk;                 // dense: filter span in chunks of R; sparse: length of the
                                // per-segment count array of a record (even)
    int nseg;                   // sparse: window segments per unit (records' segment count)
    int halo;                   // >= nchunk * R samples of history per tile (multiple of 8)
    int buf_elems;              // per-stage source buffer, multiple of kMixBox
    int full_rows;              // floor(len / kMixBox): rows of the 3-D source view
    int n_tiles;
    int stages;                 // pipeline depth (2..kMixMaxStages)
    int runacc_off;             // sparse: byte offset of the per-lane fold accumulators in
                                // dynamic shared memory (kSparseRunAccBytes)
    int fold;                   // sparse: sources per register fold (>= 1)
    Partition part;
    float *partial;             // [n_tiles][slots][2][tile]
    int slots;
    int *status;
};

struct MixShape {
    int r, warps, tile;
};
MixShape mix_shape(int mode);
cudaError_t launch_sparse_tmem(int dtype, const CUtensorMap &tmap, const CUtensorMap &tmap3,
                               const MixArgs &a, int grid, size_t smem, cudaStream_t st);
size_t mix_smem_bytes(int buf_elems, int elem_bytes, int rec_bytes, int stages);
// tmap: 2-D tiled tensor map over the sources ({len, n_src}, box {kMixBox, 1}, zero fill);
// tmap3: 3-D view {kMixBox, len / kMixBox, n_src} with box {kMixBox, buf_elems / kMixBox, 1}
// that loads a whole tile in one request when the tile lies within the full rows.
cudaError_t launch_mix(int mode, int dtype, const CUtensorMap &tmap, const CUtensorMap &tmap3,
                       const MixArgs &a, int grid, size_t smem, cudaStream_t st);

// ---- fixed-order reduction of partial slots + optional resonance FIR -------------------
struct ReduceArgs {
    const float *partial;
    int slots;
    int n_tiles;
    int tile;
    Partition part;
    const float *res;   // [2][res_len] or nullptr for identity
    int res_len;
    int64_t out_len;
    float *out;
    int64_t out_ld;
};
cudaError_t launch_reduce(const ReduceArgs &a, cudaStream_t st);
// a bounded wait that expires (DEV_TIMEOUT into *status after the wait limit): self-test
cudaError_t launch_wait_timeout_selftest(int *status, cudaStream_t st);
// out_e[n] = sum_{l < res_len} res[e][l] z_e[n - l] for n < out_len, z_e[m] = sum over c < n_parts
// of parts[c][e][m] (parts [n_parts][2][part_ld], m < z_len; compensated, in c order)
cudaError_t launch_parts_fir(const float *parts, int n_parts, int64_t part_ld, int64_t z_len, const float *res,
                             int res_len, int64_t out_len, float *out, int64_t out_ld, cudaStream_t st);
// out[e][0, n) (row stride out_ld) = sum over c of parts[c][e][0, n), in c order
cudaError_t launch_add_parts(float *out, int64_t out_ld, const float *parts, int n_parts, int64_t n,
                             cudaStream_t st);

// ---- overlap-save FFT convolution with frequency-domain mixing -------------------------
constexpr int kFftSize = 4096;                    // frame P
constexpr int kFftBinsPadded = kFftSize / 2 + 8;  // P/2 + 1 bins, row stride padded
constexpr int kFftPairRun = 32;                   // source pairs per accumulation run
constexpr int kFftCtasPerSm = 2;                  // two 512-thread CTAs overlap their phases

struct FftArgs {
    const float2 *tw;        // [P] exp(-2 pi i k / P)
    const float2 *spec;      // [(n_dirs + 1)][2][kFftBinsPadded] HRIR spectra (last: silent)
    const int32_t *dir;      // [n_src]
    int n_src;
    int n_dirs;
    int hop;                 // B = P - guard outputs per frame
    int guard;               // G = H - 1 rounded up to 8
    Partition part;          // units = frames x source pairs (part.n_src = pairs)
    float2 *partial;         // [n_frames][slots][2][kFftBinsPadded]
    int slots;
    int *status;
};

struct FftOutArgs {
    const float2 *partial;
    int slots;
    Partition part;
    const float2 *tw;
    int hop;
    int guard;
    int64_t out_len;
    float *out;
    int64_t out_ld;
};

size_t fft_mix_smem_bytes(int elem_bytes);
cudaError_t launch_build_spectra(const float *dense, int padded_len, int hrir_len, int n_records,
                                 const float2 *tw, float2 *spec, cudaStream_t st);
// tmap: 2-D tensor map over the sources with box {256, 2} (one source pair per box)
cudaError_t launch_fft_mix(int dtype, const CUtensorMap &tmap, const FftArgs &a, int grid,
                           size_t smem, cudaStream_t st);
cudaError_t launch_fft_out(const FftOutArgs &a, int n_frames, cudaStream_t st);

// ---- learned reflection filters: direction -> filter network (FP32) -----------------------
constexpr int kMlpIn = 5;        // (sin az, cos az, sin el, cos el, ear)
constexpr int kMlpHidden = 256;  // three hidden layers

// C[m][n] = sum_k A(m, k) B(k, n), A(m, k) = A[m sam + k sak], B(k, n) = B[k sbk + n sbn];
// the K range is split over blockIdx.z in chunks of k_chunk.  Epilogues (epi):
// 0: Z = C + bias; 1: Z = C + bias and H = softplus(Z); 2: Z = C * [mask > 0];
// 3: Z[z][m][n] = C (split-K partial, row stride ldz, M rows per split).
struct GemmArgs {
    int64_t M;
    int N, K;
    const float *A;
    int64_t sam, sak;
    const float *B;
    int64_t sbk, sbn;
    int k_chunk;
    const float *bias;
    float *Z;
    int64_t ldz;
    float *H;
    int64_t ldh;
    const float *mask;
    int64_t ldm;
};
// C[m][n] = sum_k A(m, k) B(k, n) over the strides of GemmArgs on the tensor cores, to FP32
// accuracy (three BF16 terms per operand value), 128-row output tiles; epi: 0 + bias, 1 + bias
// and softplus into H, 2 x [mask > 0], 3 split-K partial (blockIdx.z); relu_a / relu_b: ReLU
// on the operand as it is loaded.  A wait that expires ORs DEV_TIMEOUT into *status.
int gemm_tc_tile_rows();
int gemm_tc_tile_cols();
cudaError_t launch_gemm_tc(int epi, bool relu_a, bool relu_b, const GemmArgs &g, int splits, int *status,
                           cudaStream_t st);
cudaError_t launch_features_layer1(int n_rows, const float *dirs, const float *W1, const float *b1,
                                   float *z1, int64_t ldz, float *xs, cudaStream_t st);
cudaError_t launch_output_grad(int64_t n_rows, int refl_len, const float *g, const float *tgt,
                               const float *z4, int64_t ldz, float inv_b, float *dz, float *partial,
                               int n_partial, float *loss, cudaStream_t st);
// out[n] = sum_b D[b][n] for n < N, deterministic; P: workspace of kColsumMaxChunks * N floats
constexpr int kColsumMaxChunks = 64;
cudaError_t launch_colsum(int64_t rows, int N, const float *D, int64_t ldd, float *P, float *out,
                          cudaStream_t st);
cudaError_t launch_split_reduce(int splits, int M, int N, const float *P, float *out, cudaStream_t st);
cudaError_t launch_adam(int64_t n, float *p, const float *g, float *m, float *v, float lr, float b1,
                        float b2, float eps, float c1, float c2, cudaStream_t st);

// One layer of the network's BF16 tensor-core inference: Z = H W^T + b (K = 256) over 128-row
// tiles; first: H = relu(W1 x + b1) from the rows' features; last: out = softplus(Z) (FP32),
// else hout = relu(Z) (BF16).
struct MlpTcArgs {
    int64_t n_rows;
    const float *dirs;           // [n_rows][3] (first layer only)
    const float *W1, *b1;        // first layer only
    int first, last;
    const __nv_bfloat16 *in;     // (not first) tiles of 128 rows x 256, canonical operand layout
    const float *W;              // [N][256] FP32 (converted to BF16 in shared memory)
    const float *b;              // [N]
    int N, n_pad;                // N <= n_pad <= 256, n_pad % 16 == 0
    __nv_bfloat16 *hout;         // (not last) ceil(n_rows / 128) tiles of 128 x 256, same layout
    float *out;                  // [n_rows][N] (last)
    int stage_out;               // (set by the launcher) output rows staged for coalesced stores
    int *status;
};
size_t mlp_tc_smem_bytes(int n_pad, int stage_out);
cudaError_t launch_mlp_layer_tc(const MlpTcArgs &a, int grid, cudaStream_t st);

// ---- moving sources: per-segment filters with a linear crossfade ---------------------------
constexpr int kMovTile = 1024;   // outputs per (tile, source) unit
constexpr int kMovMaxHalo = 1024;  // history samples per window (Lg rounded up to 4)
constexpr int kMovMaxTaps = 1024;  // taps staged per unit: segments x 2 ears x k_max
struct MovingArgs {
    const float *src;            // [n_src][ld]
    int64_t ld, len;
    int n_src;
    int n_seg, seg_len, k_max;   // tables [n_src][n_seg][2][k_max]
    const uint16_t *tap_idx;
    const float *tap_w;
    const uint8_t *tap_nnz;      // [n_src][n_seg][2]
    int refl_len;
    int halo;                    // round_up(refl_len, 4)
    int n_js;                    // segments staged per unit
    int bulk_tables;             // tables copied by bulk copies (k_max % 4 == 0, 16-byte aligned)
    Partition part;
    float *partial;              // [n_tiles][slots][2][kMovTile]
    int slots;
    int *status;
};
size_t moving_smem_bytes(int halo, int n_js, int k_max);
cudaError_t launch_moving_mix(const MovingArgs &a, int grid, size_t smem, cudaStream_t st);
int moving_ctas_per_sm(size_t smem);   // resident CTAs per SM (>= 1)

// ---- moving sources on tensor-memory windows (moving_tmem.cu) -------------------------------
// 128 TMEM lanes x 32 outputs: a 4096-output tile; a lane never straddles a segment
// (seg_len % 32 == 0).  Each lane's window of 256 samples (224 filter offsets + its 32
// outputs) double-buffered in the 512 TMEM columns; the source tile (4096 + 256 samples)
// arrives by a 3-D TMA load of 32-sample rows with the 128-byte swizzle, so that the copy
// into TMEM reads shared memory without bank conflicts.
constexpr int kMvR = 32, kMvTile = 128 * kMvR, kMvCols = 256, kMvSpan = kMvCols - kMvR;   // 224
constexpr int kMvHalo = 256, kMvBufElems = kMvTile + kMvHalo;   // 4352 samples, 136 rows of 32
constexpr int kMvSegQ = 4;        // segments one lane quarter (1024 outputs) spans, seg_len >= 256
constexpr int kMvMaxK = 16;       // taps per (segment, ear) table row
constexpr int kMvMaxU = 5 * kMvMaxK;   // union of the quarter's <= 5 tables
constexpr int kMvMaxTableSegs = kMvTile / 256 + 2;   // table rows staged per unit
struct MovingTmemArgs {
    const float *src;            // [n_src][ld], ld >= round_up(len, 32)
    int64_t ld, len;
    int n_src, n_seg, seg_len, k_max;   // tables [n_src][n_seg][2][k_max], k_max % 4 == 0
    const uint16_t *tap_idx;
    const float *tap_w;
    const uint8_t *tap_nnz;      // [n_src][n_seg][2]
    int refl_len;                // <= kMvSpan
    int rows;                    // ceil(len / 32): rows of the 3-D source view
    int stages, fold;
    int runacc_off, prog_off;    // shared-memory offsets of the fold accumulators, programs
    Partition part;
    float *partial;              // [n_tiles][slots][2][kMvTile]
    int slots;
    int *status;
};
// shared memory of the pipeline with `stages` stages (0 when it does not fit)
size_t moving_tmem_smem_bytes(int stages, int k_max, int *runacc_off, int *prog_off);
cudaError_t launch_moving_tmem(const CUtensorMap &tmap3, const MovingTmemArgs &a, int grid, size_t smem,
                               cudaStream_t st);

// ---- per-source resonance as a Toeplitz-block GEMM on the tensor cores ----------------------
constexpr int kResTile = 4096;   // outputs per MMA tile (128 blocks of 32)
constexpr int kResMaxLf = 32;    // resonance taps one block row covers
struct ResonanceArgs {
    int n_src;
    int64_t out_len;             // samples of u per (source, ear)
    const float *res;            // [2][res_len], res_len <= kResMaxLf
    int res_len;
    float *out;                  // [n_src][2][out_ld]
    int64_t out_ld;
    int *status;
};
size_t resonance_gemm_smem_bytes(int elem_bytes);
// tmap: 2-D tensor map over the 16-bit sources with box {256, 1}
cudaError_t launch_resonance_gemm(int dtype, const CUtensorMap &tmap, const ResonanceArgs &a,
                                  int grid, cudaStream_t st);

// ---- filter production: L1-NNLS sparsification, Eq. 14 with D_I or D_W (sparsify.cu) ---------
// ---- filter production: the alternating minimisation of Algorithm 1 (factorize.cu; its
// products run on launch_gemm_tc) ----------------------------------------------------------
constexpr int kFactMaxLf = 64;       // resonance taps the FP64 Toeplitz solve supports
// a[d] = sum_j P[j][j + d], b[l] = sum_j B[j + l][j] (d, l < Lf), FP64, fixed order
cudaError_t launch_fact_diag(const float *P, int ldp, const float *B, int ldb, int Lg, int Lf, double *a, double *b,
                             cudaStream_t st);
// Toeplitz(a) f = b by FP64 Cholesky; f (FP32) and its autocorrelation r[0, Lf)
cudaError_t launch_fact_solve(const double *a, const double *b, int Lf, float *f, float *r, int *status,
                              cudaStream_t st);
// F~ [M][Lg] of f; Q+ and Q- [Lg][Lg], the positive and negative parts of Toeplitz(r)
cudaError_t launch_fact_build(const float *f, const float *r, int M, int Lg, int Lf, float *Ft, float *Qp, float *Qm,
                              cudaStream_t st);
// the multiplicative update of Eq. 4 on G (rows of stride ldg) from C = X F~, G Q+, G Q-
cudaError_t launch_fact_update(float *G, int64_t ldg, const float *C, const float *GQp, const float *GQm, int N,
                               int Lg, cudaStream_t st);
// *out = ||X - G F~^T||_F^2 (FP64 sums, fixed order); partial: fact_residual_blocks(N) doubles
int fact_residual_blocks(int N);
cudaError_t launch_fact_residual(const float *X, int64_t ldx, const float *G, int64_t ldg, const float *f, int N,
                                 int M, int Lg, int Lf, double *partial, float *out, cudaStream_t st);
// f <- f / ||f||, G <- G ||f||
cudaError_t launch_fact_scale(float *f, int Lf, float *G, int64_t ldg, int N, int Lg, cudaStream_t st);

constexpr int kSparsifyMaxLf = 64;   // resonance taps of the fixed f
struct SparsifyArgs {
    int n_dirs, n_ears, M, Lg, Lf;  // Lf <= kSparsifyMaxLf
    int cap;                     // largest support the solver holds (<= Lg)
    const float *X;              // [n_dirs][n_ears][M] HRIRs
    const float *f;              // [n_ears][Lf] resonance (fixed)
    float lam;                   // lambda of Eq. 14
    float inv_sigma2;            // 1 / sigma^2 of D_W (Eq. 16), 0 for D = I
    float thresh;                // entries <= thresh are discarded
    float tol;                   // stop when max w off the support <= tol * max |c|
    float *q;                    // 2 planes (leading, trailing parts) of [n_ears][Lg][Lf]:
                                 // the band of Q in double-float (workspace)
    float *G;                    // [n_dirs][n_ears][Lg] out
    int32_t *nnz;                // [n_dirs][n_ears] out, or nullptr
    int *status;                 // DEV_SOLVER when a support outgrew cap or the loop limit
};
size_t sparsify_smem_bytes(int M, int Lg, int Lf, int cap);
cudaError_t launch_sparsify(const SparsifyArgs &a, cudaStream_t st);

// ---- table builders and top-K -------------------------------------------------------------
cudaError_t launch_topk(const float *g, int n_rows, int refl_len, int k, uint16_t *idx, float *w,
                        uint8_t *nnz, cudaStream_t st);
cudaError_t launch_build_sparse_records(const uint16_t *idx, const float *w, const uint8_t *nnz,
                                        int n_dirs, int k_max, int seg_len, int n_seg, int nseg_pad,
                                        unsigned char *rec, int rec_bytes, cudaStream_t st);
cudaError_t launch_build_dense_records(const uint16_t *idx, const float *w, const uint8_t *nnz,
                                       int n_dirs, int k_max, const float *res, int res_len,
                                       int hrir_len, int padded_len, float *rec, cudaStream_t st);

}  // namespace hrir
