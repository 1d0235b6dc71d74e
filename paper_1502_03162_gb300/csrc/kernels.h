// kernels.h -- internal launchers of the sm_103a renderer (not part of the C ABI).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace hrir {

// ---- direct-convolution mixing (sparse reflection taps, or dense HRIR) -----------------
// Outputs per lane (= window chunk width) and warps per CTA of each mixing kernel.  All warps
// compute; warp 0 also issues the TMA loads.  The tile is warps x 32 lanes x R outputs.
#ifndef HRIR_DENSE_R
#define HRIR_DENSE_R 36
#endif
#ifndef HRIR_DENSE_WARPS
#define HRIR_DENSE_WARPS 8
#endif
// Sparse kernel: windows in tensor memory, 8 warps x 32 lanes x 36 outputs (tile 9216); a
// warp's TMEM row holds kSparseTmemCols samples = one segment of kSparseSegment filter
// offsets plus the lane's outputs.
constexpr int kSparseR = 36, kSparseWarps = 8;
constexpr int kSparseTmemCols = 256;
constexpr int kSparseSegment = kSparseTmemCols - kSparseR;  // 220
constexpr int kDenseR = HRIR_DENSE_R, kDenseWarps = HRIR_DENSE_WARPS;
constexpr int kMixMaxR = 36;
constexpr int kMixMaxStages = 4;
constexpr int kMixBox = 256;                      // TMA box width (elements)
constexpr int kRunSources = 64;                   // max sources per register accumulation run

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
    int halo;                   // >= nchunk * R samples of history per tile (multiple of 8)
    int buf_elems;              // per-stage source buffer, multiple of kMixBox
    int full_rows;              // floor(len / kMixBox): rows of the 3-D source view
    int n_tiles;
    int stages;                 // pipeline depth (2..kMixMaxStages)
    Partition part;
    float *partial;             // [n_tiles][slots][2][tile]
    int slots;
    int *status;
};

struct MixShape {
    int r, warps, tile;
};
MixShape mix_shape(int mode);
size_t sparse_smem_bytes(int buf_elems, int elem_bytes, int rec_bytes, int stages);
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
