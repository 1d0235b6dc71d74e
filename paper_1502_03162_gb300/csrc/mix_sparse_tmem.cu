// mix_sparse_tmem.cu -- the sparse reflection gather-FMA mix (the method, Eq. 2, with the
// resonance moved after the mix):
//
//     z_e[n] = sum_s sum_k w_{d(s),e,k} * y_s[n - i_{d(s),e,k}]        (Sec. I footnote 2)
//
// with each lane's source window held in tensor memory (TMEM).
//
// Each of the 8 warps owns 32 lanes x R = 36 consecutive outputs per lane (tile 9216).  For
// every (source, tile) unit and every window segment of SW = 220 filter offsets, a lane
// copies the 256 samples y[n - (seg+1) SW .. n - (seg+1) SW + 256) of its window from the
// shared-memory source tile into its own TMEM row (256 columns; the warp's rows are its
// TMEM lane quarter, warps w and w+4 use the two column halves).  A tap at offset o then
// needs y[n + r - o] for r < R, which is the contiguous column range starting at
// (seg+1) SW - o: one tcgen05.ld of 36 columns, warp-uniform address, no branch and no
// register indexing, followed by 36 FMAs.  Left taps accumulate into one register set and
// right taps into the other; the next tap's load is in flight while the current tap's FMAs
// issue.  Staging (TMA), the persistent balanced work partition, run flushes into partial
// slots and bounded waits are as in the dense mixing kernel.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels.h"

namespace hrir {

namespace {

constexpr int R = kSparseR;             // outputs per lane
constexpr int NW = kSparseWarps;        // warps per CTA
constexpr int kTile = NW * 32 * R;      // outputs per tile
constexpr int kCols = kSparseTmemCols;  // TMEM columns per warp
constexpr int SW = kSparseSegment;      // filter offsets per window segment (= kCols - R)
static_assert(SW + R == kCols, "window = segment + outputs per lane");
static_assert(NW == 8 && kCols == 256, "two warps per TMEM lane quarter, 256 columns each");

// ---- 32 consecutive samples, widened to FP32 (conflict-free: lane stride R = 36 elements) --
template <typename T>
struct Load32;

template <>
struct Load32<float> {
    static __device__ __forceinline__ void run(const float *p, uint32_t (&v)[32])
    {
        const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float4 x = q[i];
            v[4 * i + 0] = __float_as_uint(x.x);
            v[4 * i + 1] = __float_as_uint(x.y);
            v[4 * i + 2] = __float_as_uint(x.z);
            v[4 * i + 3] = __float_as_uint(x.w);
        }
    }
};

template <>
struct Load32<__nv_bfloat16> {
    static __device__ __forceinline__ void run(const __nv_bfloat16 *p, uint32_t (&v)[32])
    {
        const uint2 *q = reinterpret_cast<const uint2 *>(p);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint2 x = q[i];
            v[4 * i + 0] = x.x << 16;
            v[4 * i + 1] = x.x & 0xffff0000u;
            v[4 * i + 2] = x.y << 16;
            v[4 * i + 3] = x.y & 0xffff0000u;
        }
    }
};

template <>
struct Load32<__half> {
    static __device__ __forceinline__ void run(const __half *p, uint32_t (&v)[32])
    {
        const uint2 *q = reinterpret_cast<const uint2 *>(p);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint2 x = q[i];
            const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&x.x));
            const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&x.y));
            v[4 * i + 0] = __float_as_uint(a.x);
            v[4 * i + 1] = __float_as_uint(a.y);
            v[4 * i + 2] = __float_as_uint(b.x);
            v[4 * i + 3] = __float_as_uint(b.y);
        }
    }
};

// ---- tensor-memory access (this warp's lane quarter) ----------------------------------------
__device__ __forceinline__ void tm_st32(uint32_t taddr, const uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, "
        "%29, %30, %31, %32};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
        "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]),
        "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]),
        "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]),
        "r"(v[30]), "r"(v[31])
        : "memory");
}

__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// R = 36 columns starting at taddr into v (async; valid after tm_wait_ld(v))
__device__ __forceinline__ void tm_ld36(uint32_t taddr, uint32_t (&v)[R])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
        "%30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35])
                 : "r"(taddr + 32)
                 : "memory");
}

// Wait for this thread's outstanding tcgen05.ld; v is threaded through so that no use of
// the loaded registers can be scheduled before the wait.
__device__ __forceinline__ void tm_wait_ld(uint32_t (&v)[R])
{
    asm volatile(
        "tcgen05.wait::ld.sync.aligned;"
        : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]),
          "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]),
          "+r"(v[14]), "+r"(v[15]), "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]),
          "+r"(v[20]), "+r"(v[21]), "+r"(v[22]), "+r"(v[23]), "+r"(v[24]), "+r"(v[25]),
          "+r"(v[26]), "+r"(v[27]), "+r"(v[28]), "+r"(v[29]), "+r"(v[30]), "+r"(v[31]),
          "+r"(v[32]), "+r"(v[33]), "+r"(v[34]), "+r"(v[35])
        :
        : "memory");
}

__device__ __forceinline__ void fma_slice(float (&acc)[R], const uint32_t (&v)[R], float w)
{
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = fmaf(w, __uint_as_float(v[r]), acc[r]);
}

// Apply n taps {column, weight bits} to acc.  TMEM loads are double-buffered (the next
// tap's slice is in flight while the current tap's FMAs issue) and tap records are read
// from shared memory two taps ahead, so no load feeds an address right away.
__device__ __forceinline__ void apply_taps(float (&acc)[R], uint32_t tw, const int2 *taps, int n)
{
    if (n <= 0) return;
    uint32_t A[R], B[R];
    int2 cur = taps[0];
    int2 nxt = n > 1 ? taps[1] : cur;
    tm_ld36(tw + (uint32_t)cur.x, A);
    int2 nn = n > 2 ? taps[2] : cur;
    tm_wait_ld(A);
    int t = 0;
    while (true) {
        bool more = t + 1 < n;
        if (more) tm_ld36(tw + (uint32_t)nxt.x, B);
        fma_slice(acc, A, __int_as_float(cur.y));
        if (!more) break;
        cur = nxt;
        nxt = nn;
        nn = t + 3 < n ? taps[t + 3] : cur;
        tm_wait_ld(B);
        ++t;
        more = t + 1 < n;
        if (more) tm_ld36(tw + (uint32_t)nxt.x, A);
        fma_slice(acc, B, __int_as_float(cur.y));
        if (!more) break;
        cur = nxt;
        nxt = nn;
        nn = t + 3 < n ? taps[t + 3] : cur;
        tm_wait_ld(A);
        ++t;
    }
}

// Issue the TMA loads of unit u into a pipeline stage (all lanes of warp 0).
template <typename T>
__device__ __forceinline__ void issue_unit(const CUtensorMap *tmap, const CUtensorMap *tmap3,
                                           const MixArgs &a, int64_t u, int d, T *ybuf,
                                           unsigned char *rbuf, uint32_t full_bar, int lane)
{
    const int t = (int)(u / a.n_src);
    const int s = (int)(u - (int64_t)t * a.n_src);
    const int x0 = t * kTile - a.halo;
    const int n_box = a.buf_elems / kMixBox;
    if (lane == 0)
        mbar_arrive_expect_tx(full_bar, (uint32_t)(a.buf_elems * sizeof(T) + a.rec_bytes));
    __syncwarp();
    // The tile starts on a row of the 3-D view (x0 % kMixBox == 0); when every row it covers
    // is a full row of the source, one request loads it (rows before the source read as
    // zeros).  Tiles that reach the ragged last row use one-row boxes of the 2-D map.
    const int r0 = x0 >= 0 ? x0 / kMixBox : -((-x0 + kMixBox - 1) / kMixBox);
    if (r0 + n_box <= a.full_rows) {
        if (lane == 0) tma_load_3d(smem_addr(ybuf), tmap3, 0, r0, s, full_bar);
    } else {
        for (int b = lane; b < n_box; b += 32)
            tma_load_2d(smem_addr(ybuf + b * kMixBox), tmap, x0 + b * kMixBox, s, full_bar);
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

// Record: int4 {n_seg, 0, 0, 0}, int2 cnt[nch_pad] {n_left, n_right} per segment, then per
// segment its left taps and right taps as int2 {TMEM column, weight bits}.
template <typename T>
__global__ void __launch_bounds__(NW * 32, 1)
    sparse_tmem_kernel(const __grid_constant__ CUtensorMap tmap,
                       const __grid_constant__ CUtensorMap tmap3, const MixArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int stages = a.stages;
    T *ybuf = reinterpret_cast<T *>(smem);
    unsigned char *rbuf = smem + (size_t)stages * a.buf_elems * sizeof(T);
    uint64_t *bars = reinterpret_cast<uint64_t *>(rbuf + (size_t)stages * a.rec_bytes);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 2 * stages);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * stages) + 1;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        prefetch_tensormap(&tmap);
        prefetch_tensormap(&tmap3);
        for (int i = 0; i < stages; ++i) {
            mbar_init(smem_addr(&bars[i]), 1);
            mbar_init(smem_addr(&bars[stages + i]), NW);
        }
        *abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         smem_addr(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem_base = *tmem_slot;
    // this warp: TMEM lanes 32*(warp%4).., columns 256*(warp/4)..
    const uint32_t tw = tmem_base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(kCols * (warp >> 2));

    const int64_t u_begin = a.part.first(blockIdx.x);
    const int64_t u_end = a.part.first(blockIdx.x + 1);
    const int64_t n_units = u_end - u_begin;

    int next_dir = 0;
    int64_t issued = 0;
    if (warp == 0) {
        const int64_t n0 = n_units < stages ? n_units : stages;
        for (int64_t i = 0; i < n0; ++i) {
            const int d = checked_dir(a, raw_dir(a, u_begin + i), lane);
            issue_unit<T>(&tmap, &tmap3, a, u_begin + i, d, ybuf + (size_t)i * a.buf_elems,
                          rbuf + (size_t)i * a.rec_bytes, smem_addr(&bars[i]), lane);
        }
        issued = n0;
        if (issued < n_units) next_dir = raw_dir(a, u_begin + issued);
    }

    const int lane_off = (warp * 32 + lane) * R;
    float accL[R], accR[R];
#pragma unroll
    for (int i = 0; i < R; ++i) accL[i] = accR[i] = 0.f;
    int cur_t = -1, slot = 0, run_n = 0;
    int64_t k = 0;
    for (; k < n_units; ++k) {
        const int64_t u = u_begin + k;
        if (warp == 0 && k >= 1 && issued < n_units) {
            const int st = (int)((k - 1) % stages);
            const uint32_t par = (uint32_t)(((k - 1) / stages) & 1);
            if (!mbar_wait_bounded(smem_addr(&bars[stages + st]), par, abort_flag, a.status)) break;
            issue_unit<T>(&tmap, &tmap3, a, u_begin + issued, checked_dir(a, next_dir, lane),
                          ybuf + (size_t)st * a.buf_elems, rbuf + (size_t)st * a.rec_bytes,
                          smem_addr(&bars[st]), lane);
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
        const int n_seg = *reinterpret_cast<const int *>(rec);
        const int2 *cnt = reinterpret_cast<const int2 *>(rec + 16);
        const int2 *taps = reinterpret_cast<const int2 *>(rec + 16 + 8 * a.nchunk);
        for (int seg = 0; seg < n_seg; ++seg) {
            const int2 c = cnt[seg];
            if (c.x + c.y == 0) continue;
            // window of this lane: y[n - (seg+1) SW + j], j < kCols, into its TMEM row
            const T *src = yb + a.halo + lane_off - (seg + 1) * SW;
#pragma unroll 1
            for (int q = 0; q < kCols / 32; ++q) {
                uint32_t v[32];
                Load32<T>::run(src + 32 * q, v);
                tm_st32(tw + 32 * q, v);
            }
            tm_wait_st();
            apply_taps(accL, tw, taps, c.x);
            apply_taps(accR, tw, taps + c.x, c.y);
            taps += c.x + c.y;
        }
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
        // aborted: let the copies still in flight land (bounded)
        for (int64_t j = k; j < issued; ++j) {
            const uint32_t fb = smem_addr(&bars[j % stages]);
            const uint32_t par = (uint32_t)((j / stages) & 1);
            const uint64_t t0 = global_timer_ns();
            while (!mbar_try_wait(fb, par) && global_timer_ns() - t0 < kWaitLimitNs) {
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base) : "memory");
}

}  // namespace

size_t sparse_smem_bytes(int buf_elems, int elem_bytes, int rec_bytes, int stages)
{
    return (size_t)stages * ((size_t)buf_elems * elem_bytes + rec_bytes) + 2 * stages * 8 + 16;
}

template <typename T>
static cudaError_t launch_t(const CUtensorMap &tmap, const CUtensorMap &tmap3, const MixArgs &a,
                            int grid, size_t smem, cudaStream_t st)
{
    auto k = sparse_tmem_kernel<T>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, NW * 32, smem, st>>>(tmap, tmap3, a);
    return cudaGetLastError();
}

cudaError_t launch_sparse_tmem(int dtype, const CUtensorMap &tmap, const CUtensorMap &tmap3,
                               const MixArgs &a, int grid, size_t smem, cudaStream_t st)
{
    if (dtype == 0) return launch_t<float>(tmap, tmap3, a, grid, smem, st);
    if (dtype == 1) return launch_t<__nv_bfloat16>(tmap, tmap3, a, grid, smem, st);
    return launch_t<__half>(tmap, tmap3, a, grid, smem, st);
}

}  // namespace hrir
