// mix_direct.cu -- direct-convolution mixing kernels for sm_103a.
//
//   sparse (the method, Eq. 2 with the resonance moved after the mix):
//       z_e[n] = sum_s sum_k w_{d(s),e,k} * y_s[n - i_{d(s),e,k}]
//   dense (plain method, direct convolution with the dense HRIR x = f * g, Eq. 1):
//       out_e[n] = sum_s sum_j x_{d(s),e}[j] * y_s[n - j]
// Both follow the direct-convolution definition of Sec. I footnote 2 (0-based).
//
// Design (one CTA per SM, persistent, balanced contiguous ranges of (tile, source) units):
//  * warp 0 streams each source's tile [t0 - halo, t0 + TILE) into a shared-memory ring
//    with 2-D tensor TMA boxes (cp.async.bulk.tensor + mbarrier complete_tx; samples
//    outside [0, len) arrive as hardware zero fill), plus the direction's filter record
//    as a 1-D bulk copy in the same stage;
//  * all eight warps compute; each owns 32 lanes x R = 36 consecutive outputs per lane and keeps
//    a 2R-sample register window of the source: for filter taps with offsets in chunk c,
//    [cR, cR + R), output n + r needs y[n + r - cR - delta] = win[R - delta + r], a fixed
//    register for each (delta, r).  A warp-uniform switch on (ear, delta) picks the code
//    path, so each tap costs R FMAs with no shared-memory traffic; moving to the next
//    chunk reuses half the window and loads R fresh samples (conflict-free LDS.128: the
//    lane stride of 36 floats is an odd number of 16-byte bank groups);
//  * register accumulators are flushed every <= 64 sources into partial slots that the
//    reduction kernel sums in a fixed order (deterministic, bounded FP32 error).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels.h"

namespace hrir {

namespace {

constexpr int R = kMixR;

// ---- window loads (R consecutive samples, widened to FP32) -------------------------------
template <typename T>
struct Window;

template <>
struct Window<float> {
    static __device__ __forceinline__ void load(const float *p, float (&v)[R])
    {
        const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
        for (int i = 0; i < R / 4; ++i) {
            const float4 x = q[i];
            v[4 * i + 0] = x.x;
            v[4 * i + 1] = x.y;
            v[4 * i + 2] = x.z;
            v[4 * i + 3] = x.w;
        }
    }
};

template <>
struct Window<__nv_bfloat16> {
    static __device__ __forceinline__ void load(const __nv_bfloat16 *p, float (&v)[R])
    {
        const uint2 *q = reinterpret_cast<const uint2 *>(p);
#pragma unroll
        for (int i = 0; i < R / 4; ++i) {
            const uint2 x = q[i];
            v[4 * i + 0] = __uint_as_float(x.x << 16);
            v[4 * i + 1] = __uint_as_float(x.x & 0xffff0000u);
            v[4 * i + 2] = __uint_as_float(x.y << 16);
            v[4 * i + 3] = __uint_as_float(x.y & 0xffff0000u);
        }
    }
};

template <>
struct Window<__half> {
    static __device__ __forceinline__ void load(const __half *p, float (&v)[R])
    {
        const uint2 *q = reinterpret_cast<const uint2 *>(p);
#pragma unroll
        for (int i = 0; i < R / 4; ++i) {
            const uint2 x = q[i];
            const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&x.x));
            const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&x.y));
            v[4 * i + 0] = a.x;
            v[4 * i + 1] = a.y;
            v[4 * i + 2] = b.x;
            v[4 * i + 3] = b.y;
        }
    }
};

// ---- one tap of the sparse filter: acc[r] += w * y[n + r - (cR + D)] ----------------------
template <int D>
__device__ __forceinline__ void tap(const float (&lo)[R], const float (&hi)[R], float (&acc)[R],
                                    float w)
{
#pragma unroll
    for (int r = 0; r < R; ++r) {
        constexpr int kBase = R - D;
        const float v = (kBase + r < R) ? lo[(kBase + r) % R] : hi[(kBase + r - R) % R];
        acc[r] = fmaf(w, v, acc[r]);
    }
}

#define HRIR_CASE(D)                    \
    case D:                             \
        tap<D>(lo, hi, accL, w);        \
        break;                          \
    case R + D:                         \
        tap<D>(lo, hi, accR, w);        \
        break;
#define HRIR_CASE4(D) HRIR_CASE(D) HRIR_CASE(D + 1) HRIR_CASE(D + 2) HRIR_CASE(D + 3)

__device__ __forceinline__ void dispatch_tap(int code, float w, const float (&lo)[R],
                                             const float (&hi)[R], float (&accL)[R],
                                             float (&accR)[R])
{
    static_assert(R == 36, "dispatch table is written out for R = 36");
    switch (code) {
        HRIR_CASE4(0)
        HRIR_CASE4(4)
        HRIR_CASE4(8)
        HRIR_CASE4(12)
        HRIR_CASE4(16)
        HRIR_CASE4(20)
        HRIR_CASE4(24)
        HRIR_CASE4(28)
        HRIR_CASE4(32)
        default:
            break;
    }
}
#undef HRIR_CASE4
#undef HRIR_CASE

// Sparse record: int4 {n_taps, max_idx, min_idx, 0}, then n_taps int2 {idx | ear << 16,
// weight bits}, sorted by descending idx.
template <typename T>
__device__ __forceinline__ void sparse_source(const T *yb, int halo, int lane_off,
                                              const unsigned char *rec, float (&accL)[R],
                                              float (&accR)[R])
{
    const int4 hdr = *reinterpret_cast<const int4 *>(rec);
    const int n_taps = hdr.x;
    if (n_taps <= 0) return;
    const int2 *taps = reinterpret_cast<const int2 *>(rec + 16);
    int c = hdr.y / R;
    const int c_min = hdr.z / R;
    const T *base = yb + halo + lane_off;
    float lo[R], hi[R];
    Window<T>::load(base - (c + 1) * R, lo);
    Window<T>::load(base - c * R, hi);
    int ti = 0;
    while (true) {
        const int cb = c * R;
        while (ti < n_taps) {
            const int2 tp = taps[ti];
            const int idx = tp.x & 0xffff;
            if (idx < cb) break;
            const int code = (idx - cb) + ((tp.x >> 16) & 1) * R;
            dispatch_tap(code, __int_as_float(tp.y), lo, hi, accL, accR);
            ++ti;
        }
        if (c <= c_min) break;
        --c;
#pragma unroll
        for (int i = 0; i < R; ++i) lo[i] = hi[i];
        Window<T>::load(base - c * R, hi);
    }
}

// Dense record: float h[2][nchunk * R] (the HRIR of each ear, zero padded).
template <typename T>
__device__ __forceinline__ void dense_source(const T *yb, int halo, int lane_off, int nchunk,
                                             const float *h, float (&accL)[R], float (&accR)[R])
{
    const int hp = nchunk * R;
    int c = nchunk - 1;
    const T *base = yb + halo + lane_off;
    float lo[R], hi[R];
    Window<T>::load(base - (c + 1) * R, lo);
    Window<T>::load(base - c * R, hi);
    while (true) {
        const float *hl = h + c * R;
        const float *hr = h + hp + c * R;
#pragma unroll
        for (int d = 0; d < R; ++d) {
            const float wl = hl[d], wr = hr[d];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int j = R - d + r;
                const float v = (j < R) ? lo[j % R] : hi[(j - R) % R];
                accL[r] = fmaf(wl, v, accL[r]);
                accR[r] = fmaf(wr, v, accR[r]);
            }
        }
        if (c == 0) break;
        --c;
#pragma unroll
        for (int i = 0; i < R; ++i) lo[i] = hi[i];
        Window<T>::load(base - c * R, hi);
    }
}

// Issue the loads of unit u into pipeline stage st (called by all lanes of warp 0):
// the source tile [t0 - halo, t0 - halo + buf_elems) as kMixBox-wide tensor-TMA boxes
// (out-of-range samples arrive as zeros) and the direction's filter record.
template <typename T>
__device__ __forceinline__ void issue_unit(const CUtensorMap *tmap, const MixArgs &a, int64_t u,
                                           int d, T *ybuf, unsigned char *rbuf, uint32_t full_bar,
                                           int lane)
{
    const int t = (int)(u / a.n_src);
    const int s = (int)(u - (int64_t)t * a.n_src);
    const int x0 = t * kMixTile - a.halo;
    const int n_box = a.buf_elems / kMixBox;
    if (lane == 0)
        mbar_arrive_expect_tx(full_bar, (uint32_t)(a.buf_elems * sizeof(T) + a.rec_bytes));
    __syncwarp();
    for (int b = lane; b < n_box; b += 32)
        tma_load_2d(smem_addr(ybuf + b * kMixBox), tmap, x0 + b * kMixBox, s, full_bar);
    if (lane == 0)
        tma_load_1d(smem_addr(rbuf), a.table + (size_t)d * a.rec_bytes, (uint32_t)a.rec_bytes,
                    full_bar);
}

// Direction record index of unit u (the silent record for an id out of range).
__device__ __forceinline__ int unit_dir(const MixArgs &a, int64_t u, int lane)
{
    const int s = (int)(u % a.n_src);
    int d = __ldg(a.dir + s);
    if ((unsigned)d >= (unsigned)a.n_dirs) {
        if (lane == 0) atomicOr(a.status, DEV_BAD_DIR);
        d = a.n_dirs;
    }
    return d;
}

template <int MODE, typename T>
__global__ void __launch_bounds__(kMixThreads, 1)
    mix_kernel(const __grid_constant__ CUtensorMap tmap, const MixArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int stages = a.stages;
    T *ybuf = reinterpret_cast<T *>(smem);
    unsigned char *rbuf = smem + (size_t)stages * a.buf_elems * sizeof(T);
    uint64_t *bars = reinterpret_cast<uint64_t *>(rbuf + (size_t)stages * a.rec_bytes);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 2 * stages);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        prefetch_tensormap(&tmap);
        for (int i = 0; i < stages; ++i) {
            mbar_init(smem_addr(&bars[i]), 1);                   // full: producer + tx bytes
            mbar_init(smem_addr(&bars[stages + i]), kMixWarps);  // empty: one arrive per warp
        }
        *abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();

    const int64_t u_begin = a.part.first(blockIdx.x);
    const int64_t u_end = a.part.first(blockIdx.x + 1);
    const int64_t n_units = u_end - u_begin;

    // prologue: warp 0 fills the pipeline
    int next_dir = 0;        // prefetched direction of the next unit to issue (warp 0)
    int64_t issued = 0;      // units issued so far (warp 0)
    if (warp == 0) {
        const int64_t n0 = n_units < stages ? n_units : stages;
        for (int64_t i = 0; i < n0; ++i) {
            const int d = unit_dir(a, u_begin + i, lane);
            issue_unit<T>(&tmap, a, u_begin + i, d, ybuf + (size_t)i * a.buf_elems,
                          rbuf + (size_t)i * a.rec_bytes, smem_addr(&bars[i]), lane);
        }
        issued = n0;
        if (issued < n_units) next_dir = unit_dir(a, u_begin + issued, lane);
    }

    const int lane_off = (warp * 32 + lane) * R;
    float accL[R], accR[R];
#pragma unroll
    for (int i = 0; i < R; ++i) accL[i] = accR[i] = 0.f;
    int cur_t = -1, slot = 0, run_n = 0;
    int64_t k = 0;  // units consumed
    for (; k < n_units; ++k) {
        const int64_t u = u_begin + k;
        // warp 0: refill the stage freed by unit k-1 with unit k-1+stages
        if (warp == 0 && k >= 1 && issued < n_units) {
            const int st = (int)((k - 1) % stages);
            const uint32_t par = (uint32_t)(((k - 1) / stages) & 1);
            if (!mbar_wait_bounded(smem_addr(&bars[stages + st]), par, abort_flag, a.status)) break;
            issue_unit<T>(&tmap, a, u_begin + issued, next_dir, ybuf + (size_t)st * a.buf_elems,
                          rbuf + (size_t)st * a.rec_bytes, smem_addr(&bars[st]), lane);
            ++issued;
            if (issued < n_units) next_dir = unit_dir(a, u_begin + issued, lane);
        }
        const int t = (int)(u / a.n_src);
        if (t != cur_t) {
            cur_t = t;
            slot = a.part.slot_base(blockIdx.x, t);
            run_n = 0;
        }
        const int st = (int)(k % stages);
        if (!mbar_wait_bounded(smem_addr(&bars[st]), (uint32_t)((k / stages) & 1), abort_flag,
                               a.status))
            break;
        const T *yb = ybuf + (size_t)st * a.buf_elems;
        const unsigned char *rec = rbuf + (size_t)st * a.rec_bytes;
        if (MODE == MIX_SPARSE)
            sparse_source<T>(yb, a.halo, lane_off, rec, accL, accR);
        else
            dense_source<T>(yb, a.halo, lane_off, a.nchunk, reinterpret_cast<const float *>(rec),
                            accL, accR);
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&bars[stages + st]));
        ++run_n;
        const bool tile_end = (u + 1 == u_end) || ((u + 1) / a.n_src != t);
        if (run_n == a.part.gs || tile_end) {
            float *p = a.partial + ((size_t)t * a.slots + slot) * 2 * kMixTile + lane_off;
            float4 *pl = reinterpret_cast<float4 *>(p);
            float4 *pr = reinterpret_cast<float4 *>(p + kMixTile);
#pragma unroll
            for (int i = 0; i < R / 4; ++i) {
                pl[i] = make_float4(accL[4 * i], accL[4 * i + 1], accL[4 * i + 2], accL[4 * i + 3]);
                pr[i] = make_float4(accR[4 * i], accR[4 * i + 1], accR[4 * i + 2], accR[4 * i + 3]);
            }
#pragma unroll
            for (int i = 0; i < R; ++i) accL[i] = accR[i] = 0.f;
            ++slot;
            run_n = 0;
        }
    }
    if (warp == 0 && k < n_units) {
        // aborted: let the copies still in flight land before the CTA exits (bounded)
        for (int64_t j = k; j < issued; ++j) {
            const uint32_t fb = smem_addr(&bars[j % stages]);
            const uint32_t par = (uint32_t)((j / stages) & 1);
            const uint64_t t0 = global_timer_ns();
            while (!mbar_try_wait(fb, par) && global_timer_ns() - t0 < kWaitLimitNs) {
            }
        }
    }
}

}  // namespace

size_t mix_smem_bytes(int buf_elems, int elem_bytes, int rec_bytes, int stages)
{
    return (size_t)stages * ((size_t)buf_elems * elem_bytes + rec_bytes) + 2 * stages * 8 + 16;
}

template <int MODE, typename T>
static cudaError_t launch_one(const CUtensorMap &tmap, const MixArgs &a, int grid, size_t smem,
                              cudaStream_t st)
{
    auto k = mix_kernel<MODE, T>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kMixThreads, smem, st>>>(tmap, a);
    return cudaGetLastError();
}

cudaError_t launch_mix(int mode, int dtype, const CUtensorMap &tmap, const MixArgs &a, int grid,
                       size_t smem, cudaStream_t st)
{
    if (mode == MIX_SPARSE) {
        if (dtype == 0) return launch_one<MIX_SPARSE, float>(tmap, a, grid, smem, st);
        if (dtype == 1) return launch_one<MIX_SPARSE, __nv_bfloat16>(tmap, a, grid, smem, st);
        return launch_one<MIX_SPARSE, __half>(tmap, a, grid, smem, st);
    }
    if (dtype == 0) return launch_one<MIX_DENSE, float>(tmap, a, grid, smem, st);
    if (dtype == 1) return launch_one<MIX_DENSE, __nv_bfloat16>(tmap, a, grid, smem, st);
    return launch_one<MIX_DENSE, __half>(tmap, a, grid, smem, st);
}

}  // namespace hrir
