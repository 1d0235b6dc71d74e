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
// aligned 16-byte load from the copy (-i) mod 4 for every tap i.  The next unit's window and
// taps are loaded into registers while the current unit's taps run (3 CTAs per SM).  A warp
// covers 128 outputs inside one segment (seg_len is a multiple of 128), so its taps are
// warp-uniform broadcasts.
// Runs of <= 64 sources accumulate in registers and are flushed to partial slots.
#include "kernels.h"

namespace hrir {

namespace {

constexpr int kThreads = 256;
constexpr int kPer = 4;                        // outputs per thread
constexpr int kTile = kThreads * kPer;         // 1024
static_assert(kTile == kMovTile, "tile");

// Window chunks (4 samples) a thread prefetches per unit: ceil((halo + kTile) / 4 / kThreads).
constexpr int kMaxChunks = 2;                  // halo <= 1024
constexpr int kMaxTapsPerThread = 4;           // n_js * 2 * k_max <= kThreads * 4

// Loads of one unit kept in registers until the previous unit's taps are done.
struct Prefetch {
    float4 v0[kMaxChunks], v1[kMaxChunks];     // chunk q and q + 1 of the window
    int2 tap[kMaxTapsPerThread];
    int cnt;
};

__device__ __forceinline__ float4 chunk(const float *ys, int64_t p, int64_t len)
{
    // samples p .. p + 3 (p a multiple of 4), zero outside [0, len)
    if (p >= 0 && p + 4 <= len) return __ldg(reinterpret_cast<const float4 *>(ys + p));
    float4 v;
    v.x = (p >= 0 && p < len) ? __ldg(ys + p) : 0.f;
    v.y = (p + 1 >= 0 && p + 1 < len) ? __ldg(ys + p + 1) : 0.f;
    v.z = (p + 2 >= 0 && p + 2 < len) ? __ldg(ys + p + 2) : 0.f;
    v.w = (p + 3 >= 0 && p + 3 < len) ? __ldg(ys + p + 3) : 0.f;
    return v;
}

__global__ void __launch_bounds__(kThreads, 3) moving_mix_kernel(const MovingArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int win = a.halo + kTile;            // samples per shifted copy (multiple of 4)
    const int n_chunks = win / 4;
    float *Y = reinterpret_cast<float *>(smem);                 // [4][win]
    int2 *taps = reinterpret_cast<int2 *>(Y + 4 * win);         // [n_js][2][k_max]
    int *cnt = reinterpret_cast<int *>(taps + a.n_js * 2 * a.k_max);  // [n_js][2]

    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t u_begin = a.part.first(blockIdx.x);
    const int64_t u_end = a.part.first(blockIdx.x + 1);
    const int n_tap = a.n_js * 2 * a.k_max;

    // ---- global loads of the unit at (tile t, source s) into registers ----
    auto fetch = [&](int t, int s, Prefetch &pf) {
        const int t0 = t * kTile;                  // < 2^31: len < 2^31
        const int64_t wb = (int64_t)t0 - a.halo;
        const float *ys = a.src + (int64_t)s * a.ld;
#pragma unroll
        for (int c = 0; c < kMaxChunks; ++c) {
            const int q = tid + c * kThreads;
            if (q < n_chunks) {
                pf.v0[c] = chunk(ys, wb + 4 * q, a.len);
                pf.v1[c] = chunk(ys, wb + 4 * q + 4, a.len);
            }
        }
        int jl = t0 / a.seg_len - 1;
        jl = jl < 0 ? 0 : jl;
        const int j_lo = jl < a.n_seg - 1 ? jl : a.n_seg - 1;
#pragma unroll
        for (int c = 0; c < kMaxTapsPerThread; ++c) {
            const int i = tid + c * kThreads;
            if (i < n_tap) {
                const int jj = i / (2 * a.k_max);
                const int ek = i - jj * 2 * a.k_max;
                const int j = min(j_lo + jj, a.n_seg - 1);
                const int64_t row = ((int64_t)s * a.n_seg + j) * 2 * a.k_max + ek;
                pf.tap[c] = make_int2((int)a.tap_idx[row], __float_as_int(a.tap_w[row]));
            }
        }
        if (tid < a.n_js * 2) {
            const int j = min(j_lo + (tid >> 1), a.n_seg - 1);
            pf.cnt = a.tap_nnz[((int64_t)s * a.n_seg + j) * 2 + (tid & 1)];
        }
    };
    // ---- registers -> shared memory: Y[c][q] = y[wb + q + c]; taps checked ----
    // (a tap index >= Lg or a count > k_max is ignored and flagged: the window only holds
    // Lg - 1 samples of history)
    auto stage = [&](const Prefetch &pf) {
#pragma unroll
        for (int c = 0; c < kMaxChunks; ++c) {
            const int q = tid + c * kThreads;
            if (q < n_chunks) {
                const float4 x = pf.v0[c], y = pf.v1[c];
                float4 *d = reinterpret_cast<float4 *>(Y) + q;
                d[0] = x;
                d[n_chunks] = make_float4(x.y, x.z, x.w, y.x);
                d[2 * n_chunks] = make_float4(x.z, x.w, y.x, y.y);
                d[3 * n_chunks] = make_float4(x.w, y.x, y.y, y.z);
            }
        }
#pragma unroll
        for (int c = 0; c < kMaxTapsPerThread; ++c) {
            const int i = tid + c * kThreads;
            if (i < n_tap) {
                int2 tp = pf.tap[c];
                if (tp.x >= a.refl_len) {
                    atomicOr(a.status, DEV_BAD_TAP);
                    tp = make_int2(0, 0);
                }
                taps[i] = tp;
            }
        }
        if (tid < a.n_js * 2) {
            int n = pf.cnt;
            if (n > a.k_max) {
                atomicOr(a.status, DEV_BAD_TAP);
                n = a.k_max;
            }
            cnt[tid] = n;
        }
    };

    float zr[2][kPer];
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int r = 0; r < kPer; ++r) zr[e][r] = 0.f;
    // unit position (tile t, source s), carried without divisions; units are tile-major
    int t = (int)(u_begin / a.n_src);
    int s = (int)(u_begin - (int64_t)t * a.n_src);
    int slot = a.part.slot_base(blockIdx.x, t), run_n = 0;
    Prefetch pf;
    pf.cnt = 0;
    if (u_begin < u_end) fetch(t, s, pf);

    for (int64_t u = u_begin; u < u_end; ++u) {
        const int t0 = t * kTile;
        __syncthreads();                       // the previous unit's reads of Y and taps are done
        stage(pf);
        __syncthreads();
        if (u + 1 < u_end) {                   // in flight during this unit's taps
            const bool wrap = s + 1 == a.n_src;
            fetch(wrap ? t + 1 : t, wrap ? 0 : s + 1, pf);
        }

        int jl = t0 / a.seg_len - 1;
        jl = jl < 0 ? 0 : jl;
        const int j_lo = jl < a.n_seg - 1 ? jl : a.n_seg - 1;
        // ---- this warp's segment and crossfade ----
        const int nw = t0 + 128 * warp;
        const int jw = nw / a.seg_len;
        const bool tail = jw >= a.n_seg;
        const int jcur = tail ? a.n_seg - 1 : (int)jw;
        const bool fade = !tail && jw >= 1;
        const int lq = kPer * tid + a.halo;    // this thread's first output in the window
        float cur[2][kPer], prv[2][kPer];
#pragma unroll
        for (int e = 0; e < 2; ++e)
#pragma unroll
            for (int r = 0; r < kPer; ++r) cur[e][r] = prv[e][r] = 0.f;
        const int jc = jcur - j_lo;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int2 *tc = taps + (jc * 2 + e) * a.k_max;
            const int nc = cnt[jc * 2 + e];
#pragma unroll 2
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
#pragma unroll 2
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
        const int n0 = t0 + kPer * tid;
#pragma unroll
        for (int r = 0; r < kPer; ++r) {
            const float al = fade ? (float)(n0 + r - jw * a.seg_len + 1) / (float)a.seg_len : 1.f;
#pragma unroll
            for (int e = 0; e < 2; ++e) zr[e][r] += fade ? fmaf(al, cur[e][r] - prv[e][r], prv[e][r]) : cur[e][r];
        }

        ++run_n;
        const bool tile_end = (u + 1 == u_end) || (s + 1 == a.n_src);
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
        if (++s == a.n_src) {
            s = 0;
            ++t;
            if (u + 1 < u_end) {
                slot = a.part.slot_base(blockIdx.x, t);   // the next tile's first slot
                run_n = 0;
            }
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
