// mix_direct.cu -- dense-HRIR direct-convolution mixing kernel for sm_103a (plain method 1):
//       out_e[n] = sum_s sum_j x_{d(s),e}[j] * y_s[n - j],   x = f * g  (Eq. 1)
// following the direct-convolution definition of Sec. I footnote 2 (0-based).  The sparse
// method's kernel (mix_sparse_tmem.cu) shares the staging, partition and flush scheme.
//
// Design (one CTA per SM, persistent, balanced contiguous ranges of (tile, source) units):
//  * warp 0 streams each source's tile [t0 - halo, t0 + TILE) into a shared-memory ring
//    with 2-D tensor TMA boxes (cp.async.bulk.tensor + mbarrier complete_tx; samples
//    outside [0, len) arrive as hardware zero fill), plus the direction's filter record
//    as a 1-D bulk copy in the same stage;
//  * all warps compute; each owns 32 lanes x R = 36 consecutive outputs per lane and keeps
//    a 2R-sample register window of the source: for the HRIR taps of chunk c, offsets
//    [cR, cR + R), output n + r needs y[n + r - cR - delta] = win[R - delta + r], a fixed
//    register for each (delta, r), so the fully unrolled chunk is 2 x R x R FMAs with the
//    tap weights broadcast from shared memory; moving to the next chunk reuses half the
//    window and loads R fresh samples (conflict-free LDS.128: the lane stride of R floats
//    is an odd number of 16-byte bank groups);
//  * register accumulators are flushed every <= 64 sources into partial slots that the
//    reduction kernel sums in a fixed order (deterministic, bounded FP32 error).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels.h"

namespace hrir {

namespace {

// ---- window loads (R consecutive samples, widened to FP32) -------------------------------
template <typename T, int R>
struct Window;

template <int R>
struct Window<float, R> {
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

template <int R>
struct Window<__nv_bfloat16, R> {
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

template <int R>
struct Window<__half, R> {
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

// Dense record: float h[2][nchunk * R] (the HRIR of each ear, zero padded).
template <typename T, int R>
__device__ __forceinline__ void dense_source(const T *yb, int halo, int lane_off, int nchunk,
                                             const float *h, float (&accL)[R], float (&accR)[R])
{
    const int hp = nchunk * R;
    int c = nchunk - 1;
    const T *base = yb + halo + lane_off;
    float lo[R], hi[R];
    Window<T, R>::load(base - (c + 1) * R, lo);
    Window<T, R>::load(base - c * R, hi);
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
        Window<T, R>::load(base - c * R, hi);
    }
}

// Issue the loads of unit u into pipeline stage st (called by all lanes of warp 0):
// the source tile [t0 - halo, t0 - halo + buf_elems) as kMixBox-wide tensor-TMA boxes
// (out-of-range samples arrive as zeros) and the direction's filter record.
template <typename T>
__device__ __forceinline__ void issue_unit(const CUtensorMap *tmap, const CUtensorMap *tmap3,
                                           const MixArgs &a, int64_t u, int d, T *ybuf,
                                           unsigned char *rbuf, uint32_t full_bar, int lane,
                                           int tile)
{
    const int t = (int)(u / a.n_src);
    const int s = (int)(u - (int64_t)t * a.n_src);
    const int x0 = t * tile - a.halo;
    const int n_box = a.buf_elems / kMixBox;
    // The tile starts on a row of the 3-D view (x0 % kMixBox == 0), whose rows are the full
    // 256-sample rows of the source.  A window that does not contain the source's ragged last
    // row is one 3-D request (rows before 0 or past the last full row arrive as hardware zero
    // fill).  A window containing the ragged row (at most one per source): one bulk copy of the
    // full rows it covers, one 2-D box for the ragged row (zero fill past len), and 16-byte
    // zero stores here for the other rows, made before the arrive that publishes them.
    const int r0 = x0 >= 0 ? x0 / kMixBox : -((-x0 + kMixBox - 1) / kMixBox);
    const int rr = a.full_rows - r0;                                      // the ragged row, if any
    const bool ragged_in = (int64_t)a.full_rows * kMixBox < a.len && rr >= 0 && rr < n_box;
    if (a.full_rows > 0 && !ragged_in) {
        if (lane == 0) {
            mbar_arrive_expect_tx(full_bar, (uint32_t)(a.buf_elems * sizeof(T) + a.rec_bytes));
            tma_load_3d(smem_addr(ybuf), tmap3, 0, r0, s, full_bar);
        }
    } else {
        const int lo = r0 < 0 ? (-r0 < n_box ? -r0 : n_box) : 0;         // rows before sample 0
        int hi = a.full_rows - r0;                                        // end of the full rows
        hi = hi < lo ? lo : (hi > n_box ? n_box : hi);
        const bool ragged = ragged_in && rr >= lo;
        const int end = ragged ? rr + 1 : hi;                             // rows [lo, end) hold data
        {
            const int per_row = kMixBox * (int)sizeof(T) / 16;
            uint4 *z = reinterpret_cast<uint4 *>(ybuf);                    // 16-byte aligned
            for (int i = lane; i < lo * per_row; i += 32) z[i] = make_uint4(0u, 0u, 0u, 0u);
            for (int i = end * per_row + lane; i < n_box * per_row; i += 32) z[i] = make_uint4(0u, 0u, 0u, 0u);
        }
        fence_proxy_async_smem();   // these stores before any later TMA write to the stage
        __syncwarp();
        if (lane == 0) {
            mbar_arrive_expect_tx(full_bar, (uint32_t)((end - lo) * kMixBox * sizeof(T) + a.rec_bytes));
            if (hi > lo)
                tma_load_1d(smem_addr(ybuf + lo * kMixBox),
                            static_cast<const T *>(a.src) + (int64_t)s * a.ld + (int64_t)(r0 + lo) * kMixBox,
                            (uint32_t)((hi - lo) * kMixBox * sizeof(T)), full_bar);
            if (ragged)
                tma_load_2d(smem_addr(ybuf + rr * kMixBox), tmap, a.full_rows * kMixBox, s, full_bar);
        }
    }
    if (lane == 0)
        tma_load_1d(smem_addr(rbuf), a.table + (size_t)d * a.rec_bytes, (uint32_t)a.rec_bytes,
                    full_bar);
}

// Raw direction id of unit u (the load stays in flight until checked_dir uses it).
__device__ __forceinline__ int raw_dir(const MixArgs &a, int64_t u)
{
    return __ldg(a.dir + (int)(u % a.n_src));
}

// Record index for a direction id: the silent record for an id out of range.
__device__ __forceinline__ int checked_dir(const MixArgs &a, int d, int lane)
{
    if ((unsigned)d >= (unsigned)a.n_dirs) {
        if (lane == 0) atomicOr(a.status, DEV_BAD_DIR);
        d = a.n_dirs;
    }
    return d;
}

template <int MODE, typename T, int R, int NW>
__global__ void __launch_bounds__(NW * 32, 1)
    mix_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap tmap3,
               const MixArgs a)
{
    constexpr int kTile = NW * 32 * R;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int stages = a.stages;
    T *ybuf = reinterpret_cast<T *>(smem);
    unsigned char *rbuf = smem + (size_t)stages * a.buf_elems * sizeof(T);
    uint64_t *bars = reinterpret_cast<uint64_t *>(rbuf + (size_t)stages * a.rec_bytes);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 2 * stages);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        prefetch_tensormap(&tmap);
        prefetch_tensormap(&tmap3);
        for (int i = 0; i < stages; ++i) {
            mbar_init(smem_addr(&bars[i]), 1);                   // full: producer + tx bytes
            mbar_init(smem_addr(&bars[stages + i]), NW);  // empty: one arrive per warp
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
            const int d = checked_dir(a, raw_dir(a, u_begin + i), lane);
            issue_unit<T>(&tmap, &tmap3, a, u_begin + i, d, ybuf + (size_t)i * a.buf_elems,
                          rbuf + (size_t)i * a.rec_bytes, smem_addr(&bars[i]), lane, kTile);
        }
        issued = n0;
        if (issued < n_units) next_dir = raw_dir(a, u_begin + issued);
    }

    const int lane_off = (warp * 32 + lane) * R;
    static_assert(R % 4 == 0 && ((R / 4) & 1), "lane stride must be an odd number of 16-byte groups");
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
            issue_unit<T>(&tmap, &tmap3, a, u_begin + issued, checked_dir(a, next_dir, lane),
                          ybuf + (size_t)st * a.buf_elems, rbuf + (size_t)st * a.rec_bytes,
                          smem_addr(&bars[st]), lane, kTile);
            ++issued;
            if (issued < n_units) next_dir = raw_dir(a, u_begin + issued);
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
        dense_source<T, R>(yb, a.halo, lane_off, a.nchunk, reinterpret_cast<const float *>(rec),
                           accL, accR);
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&bars[stages + st]));
        ++run_n;
        const bool tile_end = (u + 1 == u_end) || ((u + 1) / a.n_src != t);
        if (run_n == a.part.gs || tile_end) {
            float *p = a.partial + ((size_t)t * a.slots + slot) * 2 * kTile + lane_off;
            float4 *pl = reinterpret_cast<float4 *>(p);
            float4 *pr = reinterpret_cast<float4 *>(p + kTile);
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
    return (size_t)stages * ((size_t)buf_elems * elem_bytes + rec_bytes) + 2 * stages * 8 + kMixSmemTail;
}

MixShape mix_shape(int mode)
{
    if (mode == MIX_SPARSE) return {kSparseR, kSparseWarps, kSparseTile};
    return {kDenseR, kDenseWarps, kDenseR * kDenseWarps * 32};
}

template <int MODE, typename T, int R, int NW>
static cudaError_t launch_one(const CUtensorMap &tmap, const CUtensorMap &tmap3, const MixArgs &a,
                              int grid, size_t smem, cudaStream_t st)
{
    auto k = mix_kernel<MODE, T, R, NW>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NW * 32, smem, st>>>(tmap, tmap3, a);
    return cudaGetLastError();
}

template <int MODE, int R, int NW>
static cudaError_t launch_dtype(int dtype, const CUtensorMap &tmap, const CUtensorMap &tmap3,
                                const MixArgs &a, int grid, size_t smem, cudaStream_t st)
{
    if (dtype == 0) return launch_one<MODE, float, R, NW>(tmap, tmap3, a, grid, smem, st);
    if (dtype == 1) return launch_one<MODE, __nv_bfloat16, R, NW>(tmap, tmap3, a, grid, smem, st);
    return launch_one<MODE, __half, R, NW>(tmap, tmap3, a, grid, smem, st);
}

cudaError_t launch_mix(int mode, int dtype, const CUtensorMap &tmap, const CUtensorMap &tmap3,
                       const MixArgs &a, int grid, size_t smem, cudaStream_t st)
{
    if (mode == MIX_SPARSE) return launch_sparse_tmem(dtype, tmap, tmap3, a, grid, smem, st);
    return launch_dtype<MIX_DENSE, kDenseR, kDenseWarps>(dtype, tmap, tmap3, a, grid, smem, st);
}

}  // namespace hrir
