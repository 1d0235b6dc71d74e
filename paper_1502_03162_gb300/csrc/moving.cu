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
// tile): a CTA takes (output tile of 1024, source) units from a balanced contiguous range.
// A ring of 3 shared-memory stages, filled by bulk copies (cp.async.bulk, completion on an
// mbarrier), holds each unit's raw source window and the tap tables of the segments the tile
// touches; warp 0 refills a stage as soon as the CTA has read it.  From the raw window the
// CTA builds four copies shifted by 0..3 samples, so that the 4 consecutive samples
// y[n - i .. n - i + 3] a thread needs for its outputs n..n+3 are one aligned 16-byte load
// from the copy (-i) mod 4 for every tap i.  The crossfade needs both the previous and the
// current segment's filter at every output of a segment; their tap lists are merged by offset
// (a direction changes little from one segment to the next, so most offsets are in both),
// and one gather then feeds both filters' FMAs.  The shifted copies and the merged lists are
// double-buffered, so one barrier per unit separates building a unit from using it.  A warp
// covers 128 outputs inside one segment (seg_len is a multiple of 128), so its taps are
// warp-uniform broadcasts.  Runs of <= 64 sources accumulate in registers and are flushed to
// partial slots.
#include "kernels.h"

namespace hrir {

namespace {

constexpr int kThreads = 256;
constexpr int kPer = 4;                        // outputs per thread
constexpr int kTile = kThreads * kPer;         // 1024
static_assert(kTile == kMovTile, "tile");
constexpr int kStages = 3;                     // ring depth

__host__ __device__ inline int align16(int b) { return (b + 15) & ~15; }

// Byte offset, from a thread's first output in the shifted copies, of the 4 samples that tap
// x reads: copy c = (-x) mod 4, element lq - x - c of it.
__device__ __forceinline__ int gather_offset(int x, int win)
{
    const int c = (-x) & 3;
    return 4 * (c * win - x - c);
}

// acc += w * (v0, v1) as one packed FP32 FMA (fma.rn.f32x2: two round-to-nearest FMAs)
__device__ __forceinline__ void fma2(uint64_t &acc, float w, float v0, float v1)
{
    uint64_t ww, vv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(ww) : "f"(w));
    asm("mov.b64 %0, {%1, %2};" : "=l"(vv) : "f"(v0), "f"(v1));
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(ww), "l"(vv));
}

__device__ __forceinline__ float2 unpack2(uint64_t a)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(a));
    return r;
}

// Shared-memory layout of a CTA (byte offsets), computed the same way on host and device.
struct MovLayout {
    int win;       // samples per shifted copy: halo + kTile
    int raw;       // samples of a staged source window: win + 4
    int n_tap;     // tap entries per unit: n_js * 2 * k_max
    int st_idx, st_w, st_nnz, stage;   // within a stage: index, weight, count tables; stage size
    int y, ml, mcnt, lut, bars, flag, total;
    __host__ __device__ MovLayout(int halo, int n_js, int k_max)
    {
        win = halo + kTile;
        raw = win + 4;
        n_tap = n_js * 2 * k_max;
        st_idx = align16(raw * 4);
        st_w = st_idx + align16(n_tap * 2);
        st_nnz = st_w + align16(n_tap * 4);
        stage = st_nnz + align16(n_js * 2);
        y = kStages * stage;                       // [2][4][win] floats
        ml = y + 2 * 4 * win * 4;                  // [2][n_js][2][2 k_max] int4 merged lists
        mcnt = ml + 2 * 2 * n_tap * 16;            // [2][n_js][2] int
        lut = mcnt + 2 * n_js * 2 * 4;             // [8 warps][halo] uint8: offset -> tap + 1
        bars = align16(lut + 8 * halo);            // [kStages] mbarriers
        flag = bars + kStages * 8;                 // abort flag
        total = flag + 16;
    }
};

// What a tile of outputs [t0, t0 + kTile) needs of the per-segment tables, computed once per
// tile (units are tile-major, so it changes once every n_src units): table rows
// [j_lo, j_lo + n_rows) (the previous segment's filter for the crossfade, clamped to the
// table), the merged lists [p_lo, p_hi) its outputs use (2 per segment: ears), and for the
// calling warp's 128 outputs their segment jw, its row jc and whether they crossfade.
struct TileInfo {
    int j_lo, n_rows, p_lo, p_hi, jw, jc;
    bool fade;
    __device__ TileInfo(const MovingArgs &a, int t, int warp)
    {
        const int t0 = t * kTile;
        const int last = a.n_seg - 1;
        int jl = t0 / a.seg_len - 1;
        jl = jl < 0 ? 0 : jl;
        j_lo = jl < last ? jl : last;
        const int j_hi = j_lo + a.n_js - 1 < last ? j_lo + a.n_js - 1 : last;
        n_rows = j_hi - j_lo + 1;
        const int jw_lo = t0 / a.seg_len, jw_hi = (t0 + kTile - 1) / a.seg_len;
        p_lo = 2 * ((jw_lo < last ? jw_lo : last) - j_lo);
        p_hi = 2 * ((jw_hi < last ? jw_hi : last) - j_lo) + 2;
        jw = (t0 + 128 * warp) / a.seg_len;
        const bool tail = jw >= a.n_seg;
        jc = (tail ? last : jw) - j_lo;
        fade = !tail && jw >= 1;
    }
};

// Tap counts of a unit of source s in a tile with table rows from j_lo (n_rows of them), lane
// i holding count i (n_rows * 2 <= 20 lanes), loaded one unit ahead of its staging so that
// their latency never stalls the issuing warp.
__device__ __forceinline__ uint32_t load_counts(const MovingArgs &a, const TileInfo &ti, int s, int lane)
{
    const int64_t row0 = (int64_t)s * a.n_seg + ti.j_lo;
    return lane < ti.n_rows * 2 ? (uint32_t)a.tap_nnz[row0 * 2 + lane] : 0u;
}

// Stage unit (tile t, source s) (all lanes of warp 0): the raw window y[x0, x0 + raw) with
// x0 = t0 - halo by one bulk copy of its part inside [0, len & ~3) and lane stores for the
// rest (zeros, and the last len % 4 samples of the source); the tap tables by bulk copies when
// they are 16-byte aligned, else by lane copies; the counts (loaded earlier, `counts`) by
// lane stores.  The lane stores come before the arrive that publishes them.
__device__ __forceinline__ void issue_unit(const MovingArgs &a, const MovLayout &L, unsigned char *stage,
                                           uint32_t bar, int t, const TileInfo &sr, int s, uint32_t counts,
                                           int lane)
{
    const int t0 = t * kTile;                       // < 2^31: len < 2^31
    const int64_t x0 = (int64_t)t0 - a.halo;        // a multiple of 4
    const int64_t len4 = a.len & ~(int64_t)3;
    const float *ys = a.src + (int64_t)s * a.ld;
    float *raw = reinterpret_cast<float *>(stage);
    const int64_t lo = x0 < 0 ? 0 : x0;
    int64_t hi = x0 + L.raw < len4 ? x0 + L.raw : len4;
    hi = hi < lo ? lo : hi;
    const int r0 = (int)(lo - x0), r1 = (int)(hi - x0);    // bulk-copied: raw[r0, r1)
    for (int i = lane; i < r0; i += 32) raw[i] = 0.f;
    for (int i = r1 + lane; i < L.raw; i += 32) {
        const int64_t p = x0 + i;
        raw[i] = (p >= 0 && p < a.len) ? __ldg(ys + p) : 0.f;
    }
    const int64_t row0 = (int64_t)s * a.n_seg + sr.j_lo;
    const int n_ent = sr.n_rows * 2 * a.k_max;
    uint16_t *idx = reinterpret_cast<uint16_t *>(stage + L.st_idx);
    float *w = reinterpret_cast<float *>(stage + L.st_w);
    uint8_t *nnz = stage + L.st_nnz;
    if (lane < sr.n_rows * 2) nnz[lane] = (uint8_t)counts;
    if (!a.bulk_tables) {
        for (int i = lane; i < n_ent; i += 32) {
            idx[i] = a.tap_idx[row0 * 2 * a.k_max + i];
            w[i] = a.tap_w[row0 * 2 * a.k_max + i];
        }
    }
    fence_proxy_async_smem();   // these stores before later bulk copies into the stage
    __syncwarp();
    if (lane == 0) {
        uint32_t bytes = (uint32_t)(hi - lo) * 4u;
        if (a.bulk_tables) bytes += (uint32_t)n_ent * 6u;
        mbar_arrive_expect_tx(bar, bytes);
        if (hi > lo) tma_load_1d(smem_addr(raw + r0), ys + lo, (uint32_t)(hi - lo) * 4u, bar);
        if (a.bulk_tables) {
            tma_load_1d(smem_addr(idx), a.tap_idx + row0 * 2 * a.k_max, (uint32_t)n_ent * 2u, bar);
            tma_load_1d(smem_addr(w), a.tap_w + row0 * 2 * a.k_max, (uint32_t)n_ent * 4u, bar);
        }
    }
}

__global__ void __launch_bounds__(kThreads, 3) moving_mix_kernel(const MovingArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const MovLayout L(a.halo, a.n_js, a.k_max);
    const int n_chunks = L.win / 4;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bars);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + L.flag);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t u_begin = a.part.first(blockIdx.x);
    const int n_units = (int)(a.part.first(blockIdx.x + 1) - u_begin);
    for (int i = tid; i < 8 * a.halo; i += kThreads) smem[L.lut + i] = 0;
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) mbar_init(smem_addr(&bars[i]), 1);
        *abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();

    // unit position (tile t, source s), carried without divisions; units are tile-major
    int t = (int)(u_begin / a.n_src);
    int s = (int)(u_begin - (int64_t)t * a.n_src);
    int it = t, is = s;                                   // position of the next unit to issue
    int issued = 0;
    TileInfo ti_issue(a, it, warp);                       // of tile it
    uint32_t counts = 0;                                  // its tap counts (warp 0)
    if (warp == 0 && n_units > 0) counts = load_counts(a, ti_issue, is, lane);
    auto issue_next = [&]() {
        issue_unit(a, L, smem + (size_t)(issued % kStages) * L.stage, smem_addr(&bars[issued % kStages]),
                   it, ti_issue, is, counts, lane);
        ++issued;
        if (++is == a.n_src) {
            is = 0;
            ++it;
            ti_issue = TileInfo(a, it, warp);
        }
        if (issued < n_units) counts = load_counts(a, ti_issue, is, lane);
    };
    if (warp == 0)
        while (issued < n_units && issued < kStages) issue_next();

    float zr[2][kPer];
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int r = 0; r < kPer; ++r) zr[e][r] = 0.f;
    int slot = a.part.slot_base(blockIdx.x, t), run_n = 0;
    const float inv_seg = 1.0f / (float)a.seg_len;      // crossfade slope
    TileInfo sr(a, t, warp);                             // of the current unit's tile
    int st = 0;
    uint32_t ph = 0;
    int k = 0;
    for (; k < n_units; ++k) {
        const int t0 = t * kTile;
        const int b = k & 1;
        float *Y = reinterpret_cast<float *>(smem + L.y) + b * 4 * L.win;
        const int row = 2 * a.k_max;                      // merged-list capacity per (segment, ear)
        int4 *ml = reinterpret_cast<int4 *>(smem + L.ml) + b * a.n_js * 2 * row;
        int *mcnt = reinterpret_cast<int *>(smem + L.mcnt) + b * a.n_js * 2;
        // ---- build unit k: shifted copies Y[c][q] = y[t0 - halo + q + c], merged tap lists ----
        bool ok = mbar_wait_bounded(smem_addr(&bars[st]), ph, abort_flag, a.status);
        if (ok) {
            const unsigned char *stage = smem + (size_t)st * L.stage;
            const float4 *raw4 = reinterpret_cast<const float4 *>(stage);
            for (int q = tid; q < n_chunks; q += kThreads) {
                const float4 x = raw4[q], y = raw4[q + 1];
                float4 *d = reinterpret_cast<float4 *>(Y) + q;
                d[0] = x;
                d[n_chunks] = make_float4(x.y, x.z, x.w, y.x);
                d[2 * n_chunks] = make_float4(x.z, x.w, y.x, y.y);
                d[3 * n_chunks] = make_float4(x.w, y.x, y.y, y.z);
            }
            // Merged list of (segment jc, ear e): every tap of segment jc - 1 (the previous
            // filter of the crossfade) and of segment jc, an offset present in both once, as
            // {gather offset, previous weight, current weight}: one gather then serves both
            // filters.  Only the segments the tile's outputs lie in are merged.
            // A tap index >= Lg or a count > k_max is ignored and flagged (the window only
            // holds Lg - 1 samples of history).
            const uint16_t *idx = reinterpret_cast<const uint16_t *>(stage + L.st_idx);
            const float *w = reinterpret_cast<const float *>(stage + L.st_w);
            const uint8_t *nnz = stage + L.st_nnz;
            uint8_t *lut_base = smem + L.lut;
            for (int p = sr.p_lo + warp; p < sr.p_hi; p += kThreads / 32) {
                const int jc = p >> 1, e = p & 1;
                const int jr = jc < sr.n_rows - 1 ? jc : sr.n_rows - 1;
                const int jp = jc < 1 ? -1 : (jc - 1 < sr.n_rows - 1 ? jc - 1 : sr.n_rows - 1);
                auto count = [&](int j) {
                    if (j < 0) return 0;
                    int n = nnz[j * 2 + e];
                    if (n > a.k_max) {
                        if (lane == 0) atomicOr(a.status, DEV_BAD_TAP);
                        n = a.k_max;
                    }
                    return n;
                };
                auto entry = [&](int j, int i) {
                    const int o = (j * 2 + e) * a.k_max + i;
                    int2 tp = make_int2((int)idx[o], __float_as_int(w[o]));
                    if (tp.x >= a.refl_len) {
                        atomicOr(a.status, DEV_BAD_TAP);
                        tp = make_int2(0, 0);
                    }
                    return tp;
                };
                const int nc = count(jr), np = count(jp);
                int4 *out = ml + p * row;
                uint8_t *lut = lut_base + warp * a.halo;
                bool merge = a.k_max <= 32;
                int2 cv = make_int2(-1, 0), pv = make_int2(-2, 0);
                if (merge) {
                    // offset -> previous tap through this warp's lookup table (Lg <= halo
                    // entries, all zero between uses); a repeated offset in either list, which
                    // top-k never gives, leaves the two lists unmerged
                    if (lane < nc) cv = entry(jr, lane);
                    if (lane < np) pv = entry(jp, lane);
                    if (lane < np) lut[pv.x] = (uint8_t)(lane + 1);
                    __syncwarp();
                    const bool dup_p = lane < np && lut[pv.x] != lane + 1;
                    const int jm = lane < nc ? (int)lut[cv.x] - 1 : -1;     // matching previous tap
                    const uint32_t grp = __match_any_sync(0xffffffffu, lane < nc ? cv.x : -1 - lane);
                    const bool dup_c = lane < nc && __popc(grp) > 1;
                    __syncwarp();
                    if (lane < np) lut[pv.x] = 0;
                    merge = !__any_sync(0xffffffffu, dup_p || dup_c);
                    if (merge) {
                        const int pw = __shfl_sync(0xffffffffu, pv.y, jm < 0 ? 0 : jm);
                        if (lane < nc) out[lane] = make_int4(gather_offset(cv.x, L.win), jm < 0 ? 0 : pw, cv.y, 0);
                        const uint32_t matched = __reduce_or_sync(0xffffffffu, jm < 0 ? 0u : 1u << jm);
                        const bool rest = lane < np && !((matched >> lane) & 1u);
                        const uint32_t rm = __ballot_sync(0xffffffffu, rest);
                        if (rest)
                            out[nc + __popc(rm & ((1u << lane) - 1u))] = make_int4(gather_offset(pv.x, L.win), pv.y, 0, 0);
                        if (lane == 0) mcnt[p] = nc + __popc(rm);
                    }
                    __syncwarp();
                }
                if (!merge) {
                    for (int i = lane; i < nc; i += 32) {
                        const int2 c = entry(jr, i);
                        out[i] = make_int4(gather_offset(c.x, L.win), 0, c.y, 0);
                    }
                    for (int i = lane; i < np; i += 32) {
                        const int2 q = entry(jp, i);
                        out[nc + i] = make_int4(gather_offset(q.x, L.win), q.y, 0, 0);
                    }
                    if (lane == 0) mcnt[p] = nc + np;
                }
            }
        }
        // unit k built everywhere (and the stage read everywhere), or a wait expired somewhere
        if (!__syncthreads_and(ok)) break;
        if (warp == 0 && issued < n_units) issue_next();      // into the stage just read
        if (++st == kStages) {
            st = 0;
            ph ^= 1u;
        }

        // ---- this warp's segment and crossfade ----
        const int jw = sr.jw, jc = sr.jc;
        const bool fade = sr.fade;
        // this thread's first output in the shifted copies
        const char *yl = reinterpret_cast<const char *>(Y + kPer * tid + a.halo);
        const int n0 = t0 + kPer * tid;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int4 *m = ml + (jc * 2 + e) * row;
            const int n = mcnt[jc * 2 + e];
            uint64_t cur[2] = {0, 0}, prv[2] = {0, 0};   // outputs (0, 1), (2, 3)
            if (fade) {
#pragma unroll 4
                for (int i = 0; i < n; ++i) {
                    const int4 tp = m[i];
                    const float4 v = *reinterpret_cast<const float4 *>(yl + tp.x);
                    const float wp = __int_as_float(tp.y), wc = __int_as_float(tp.z);
                    fma2(prv[0], wp, v.x, v.y);
                    fma2(prv[1], wp, v.z, v.w);
                    fma2(cur[0], wc, v.x, v.y);
                    fma2(cur[1], wc, v.z, v.w);
                }
            } else {
#pragma unroll 4
                for (int i = 0; i < n; ++i) {
                    const int4 tp = m[i];
                    if (tp.z == 0) continue;              // a tap of the previous filter only
                    const float4 v = *reinterpret_cast<const float4 *>(yl + tp.x);
                    const float wc = __int_as_float(tp.z);
                    fma2(cur[0], wc, v.x, v.y);
                    fma2(cur[1], wc, v.z, v.w);
                }
            }
            const float2 c01 = unpack2(cur[0]), c23 = unpack2(cur[1]);
            const float c4[kPer] = {c01.x, c01.y, c23.x, c23.y};
            if (fade) {
                const float2 p01 = unpack2(prv[0]), p23 = unpack2(prv[1]);
                const float p4[kPer] = {p01.x, p01.y, p23.x, p23.y};
#pragma unroll
                for (int r = 0; r < kPer; ++r) {
                    const float al = (float)(n0 + r - jw * a.seg_len + 1) * inv_seg;
                    zr[e][r] += fmaf(al, c4[r] - p4[r], p4[r]);
                }
            } else {
#pragma unroll
                for (int r = 0; r < kPer; ++r) zr[e][r] += c4[r];
            }
        }

        ++run_n;
        const bool tile_end = (k + 1 == n_units) || (s + 1 == a.n_src);
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
            if (k + 1 < n_units) {
                slot = a.part.slot_base(blockIdx.x, t);   // the next tile's first slot
                run_n = 0;
                sr = TileInfo(a, t, warp);
            }
        }
    }
    // copies still in flight (only after an expired wait): let them land before the CTA exits
    if (warp == 0) {
        for (int u = k; u < issued; ++u) {
            const uint32_t fb = smem_addr(&bars[u % kStages]);
            const uint32_t par = (uint32_t)((u / kStages) & 1);
            const uint64_t t1 = global_timer_ns();
            while (!mbar_try_wait(fb, par) && global_timer_ns() - t1 < kWaitLimitNs) {
            }
        }
    }
}

}  // namespace

size_t moving_smem_bytes(int halo, int n_js, int k_max)
{
    return (size_t)MovLayout(halo, n_js, k_max).total;
}

int moving_ctas_per_sm(size_t smem)
{
    int nb = 0;
    cudaError_t e = cudaFuncSetAttribute(moving_mix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, moving_mix_kernel, kThreads, smem);
    return (e == cudaSuccess && nb > 0) ? nb : 1;
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
