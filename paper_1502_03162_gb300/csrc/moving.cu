// moving.cu -- moving sources: the sparse reflection mix of Eq. 2 with a direction (and so a
// reflection filter) per segment of seg_len samples and an output-domain linear crossfade:
//
//   z_e[n] = sum_s (1 - a) (y_s * g_{s,j-1,e})[n] + a (y_s * g_{s,j,e})[n],
//            j = n / seg_len, a = (n - j seg_len + 1) / seg_len,
//
// segment 0 using g_0 alone and outputs past the last segment g_{n_seg-1} alone; the
// resonance then follows the mix (linear and direction-independent, Eq. 2), in the same
// fixed-order reduction kernel as the static path.
//
// Per-segment filters make the taps uniform only over a segment, so this kernel gathers from
// shared memory (the static kernel's tensor-memory windows need one filter per 6656-output
// tile): a CTA takes (output tile of 1024, source) units from a balanced contiguous range;
// the tile's source window is staged as four copies shifted by 0..3 samples, so that the 4
// consecutive samples y[n - i .. n - i + 3] a thread needs for its outputs n..n+3 are one
// aligned 16-byte load from the copy (-i) mod 4 for every tap i.  A warp covers 128 outputs
// inside one segment (seg_len is a multiple of 128), so its taps are warp-uniform broadcasts.
// Runs of <= 64 sources accumulate in registers and are flushed to partial slots.
#include "kernels.h"

namespace hrir {

namespace {

constexpr int kThreads = 256;
constexpr int kPer = 4;                        // outputs per thread
constexpr int kTile = kThreads * kPer;         // 1024
static_assert(kTile == kMovTile, "tile");

__global__ void __launch_bounds__(kThreads) moving_mix_kernel(const MovingArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int win = a.halo + kTile;            // samples per shifted copy
    float *Y = reinterpret_cast<float *>(smem);                 // [4][win]
    int2 *taps = reinterpret_cast<int2 *>(Y + 4 * win);         // [n_js][2][k_max]
    int *cnt = reinterpret_cast<int *>(taps + a.n_js * 2 * a.k_max);  // [n_js][2]

    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t u_begin = a.part.first(blockIdx.x);
    const int64_t u_end = a.part.first(blockIdx.x + 1);
    float zr[2][kPer];
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int r = 0; r < kPer; ++r) zr[e][r] = 0.f;
    int cur_t = -1, slot = 0, run_n = 0;

    for (int64_t u = u_begin; u < u_end; ++u) {
        const int t = (int)(u / a.n_src);
        const int s = (int)(u - (int64_t)t * a.n_src);
        if (t != cur_t) {
            cur_t = t;
            slot = a.part.slot_base(blockIdx.x, t);
            run_n = 0;
        }
        const int64_t t0 = (int64_t)t * kTile;
        const int64_t wb = t0 - a.halo;
        // ---- stage the window: Y[c][q] = y[wb + q + c], zero outside [0, len) ----
        const float *ys = a.src + (int64_t)s * a.ld;
        for (int q = tid; q < win + 3; q += kThreads) {
            const int64_t p = wb + q;
            const float v = (p >= 0 && p < a.len) ? __ldg(ys + p) : 0.f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int qq = q - c;
                if (qq >= 0 && qq < win) Y[c * win + qq] = v;
            }
        }
        // ---- stage the taps of the segments this tile touches (and the one before) ----
        // (a tap index >= Lg or a count > k_max is ignored and flagged: the window only
        // holds Lg - 1 samples of history)
        int64_t jl = t0 / a.seg_len - 1;
        jl = jl < 0 ? 0 : jl;
        const int j_lo = (int)(jl < a.n_seg - 1 ? jl : a.n_seg - 1);
        for (int i = tid; i < a.n_js * 2 * a.k_max; i += kThreads) {
            const int jj = i / (2 * a.k_max);
            const int ek = i - jj * 2 * a.k_max;
            const int j = min(j_lo + jj, a.n_seg - 1);
            const int64_t row = ((int64_t)s * a.n_seg + j) * 2 * a.k_max + ek;
            int idx = (int)a.tap_idx[row];
            float w = a.tap_w[row];
            if (idx >= a.refl_len) {
                atomicOr(a.status, DEV_BAD_TAP);
                idx = 0;
                w = 0.f;
            }
            taps[i] = make_int2(idx, __float_as_int(w));
        }
        for (int i = tid; i < a.n_js * 2; i += kThreads) {
            const int jj = i >> 1;
            const int j = min(j_lo + jj, a.n_seg - 1);
            int n = a.tap_nnz[((int64_t)s * a.n_seg + j) * 2 + (i & 1)];
            if (n > a.k_max) {
                atomicOr(a.status, DEV_BAD_TAP);
                n = a.k_max;
            }
            cnt[i] = n;
        }
        __syncthreads();

        // ---- this warp's segment and crossfade ----
        const int64_t nw = t0 + 128 * warp;
        const int64_t jw = nw / a.seg_len;
        const bool tail = jw >= a.n_seg;
        const int jcur = tail ? a.n_seg - 1 : (int)jw;
        const bool fade = !tail && jw >= 1;
        const int lq = kPer * tid + a.halo;    // this thread's first output in the window
        float cur[2][kPer], prv[2][kPer];
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int r = 0; r < kPer; ++r) cur[e][r] = prv[e][r] = 0.f;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int jc = jcur - j_lo;
            const int2 *tc = taps + (jc * 2 + e) * a.k_max;
            const int nc = cnt[jc * 2 + e];
            for (int k = 0; k < nc; ++k) {
                const int2 tp = tc[k];
                const int c = (-tp.x) & 3;
                const float4 v = *reinterpret_cast<const float4 *>(Y + c * win + lq - tp.x - c);
                const float w = __int_as_float(tp.y);
                cur[e][0] = fmaf(w, v.x, cur[e][0]);
                cur[e][1] = fmaf(w, v.y, cur[e][1]);
                cur[e][2] = fmaf(w, v.z, cur[e][2]);
                cur[e][3] = fmaf(w, v.w, cur[e][3]);
            }
            if (fade) {
                const int jp = jc - 1;
                const int2 *tq = taps + (jp * 2 + e) * a.k_max;
                const int np = cnt[jp * 2 + e];
                for (int k = 0; k < np; ++k) {
                    const int2 tp = tq[k];
                    const int c = (-tp.x) & 3;
                    const float4 v = *reinterpret_cast<const float4 *>(Y + c * win + lq - tp.x - c);
                    const float w = __int_as_float(tp.y);
                    prv[e][0] = fmaf(w, v.x, prv[e][0]);
                    prv[e][1] = fmaf(w, v.y, prv[e][1]);
                    prv[e][2] = fmaf(w, v.z, prv[e][2]);
                    prv[e][3] = fmaf(w, v.w, prv[e][3]);
                }
            }
        }
        const int64_t n0 = t0 + kPer * tid;
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const float al = fade ? (float)(n0 + r - jw * a.seg_len + 1) / (float)a.seg_len : 1.f;
#pragma unroll
            for (int e = 0; e < 2; ++e) zr[e][r] += fade ? fmaf(al, cur[e][r] - prv[e][r], prv[e][r]) : cur[e][r];
        }
        __syncthreads();

        ++run_n;
        const bool tile_end = (u + 1 == u_end) || ((u + 1) / a.n_src != t);
        if (run_n == a.part.gs || tile_end) {
            float *p = a.partial + ((size_t)t * a.slots + slot) * 2 * kTile + kPer * tid;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                *reinterpret_cast<float4 *>(p + e * kTile) = make_float4(zr[e][0], zr[e][1], zr[e][2], zr[e][3]);
#pragma unroll
                for (int r = 0; r < kPer; ++r) zr[e][r] = 0.f;
            }
            ++slot;
            run_n = 0;
        }
    }
}

}  // namespace

size_t moving_smem_bytes(int halo, int n_js, int k_max)
{
    return (size_t)4 * (halo + kTile) * 4 + (size_t)n_js * 2 * k_max * 8 + (size_t)n_js * 2 * 4;
}

cudaError_t launch_moving_mix(const MovingArgs &a, int grid, size_t smem, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(moving_mix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    moving_mix_kernel<<<grid, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace hrir
