// mix_sparse_tmem.cu -- the sparse reflection gather-FMA mix (the method, Eq. 2, with the
// resonance moved after the mix):
//
//     z_e[n] = sum_s sum_k w_{d(s),e,k} * y_s[n - i_{d(s),e,k}]        (Sec. I footnote 2)
//
// with each lane's source window held in tensor memory (TMEM).
//
// A tile of 6656 outputs is split over the 4 TMEM lane quarters x 32 lanes, R = 52
// consecutive outputs per lane.  The two warps of a lane quarter (warp q: left ear, warp
// q + 4: right ear) share that quarter's TMEM rows.  For every (source, tile) unit and every
// window segment of SW = 204 filter offsets, row (lane) holds the 256 samples
// y[n - (seg+1) SW .. n - (seg+1) SW + 256) of its outputs' window.  A tap at offset o then
// needs y[n + r - o] for r < R, the contiguous column range starting at (seg+1) SW - o: one
// warp-uniform tcgen05.ld of 52 columns (no branch, no register indexing) followed by 26
// packed FP32 FMAs (fma.rn.f32x2, two outputs each); the next tap's load is in flight while
// the current tap's FMAs issue.
//
// The window is double-buffered in the 512 TMEM columns: while a pair of warps applies its
// taps to one buffer, each warp copies half of the next window (shared memory -> registers
// -> tcgen05.st) into the other, the left-ear warp before its taps and the right-ear warp
// after them; a named barrier per pair (with
// an AND vote, so that both warps leave together on a timeout) hands the buffers over.
// A ring of up to 6 shared-memory stages holds each unit's source tile (tensor TMA, 256-sample
// halo, hardware zero fill outside [0, len)) and the direction's tap record (bulk copy): the
// last of the 8 warps to release a stage refills it at once with the unit `stages` ahead.
// Work is a persistent balanced range of units per CTA; register accumulators are
// flushed every <= 64 sources into partial slots that the reduction sums in a fixed order.
// All waits are bounded.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels.h"

namespace hrir {

namespace {

constexpr int R = kSparseR;             // outputs per lane
constexpr int NQ = kSparseQuarters;     // TMEM lane quarters
constexpr int NW = kSparseWarps;        // warps: (lane quarter, ear); warp 0 also issues TMA
constexpr int kTile = kSparseTile;      // outputs per tile
constexpr int kCols = kSparseTmemCols;  // TMEM columns per window buffer
constexpr int SW = kSparseSegment;      // filter offsets per window segment (= kCols - R)
constexpr int kHalf = kCols / 2;        // window columns each warp of a pair copies
constexpr int kCopyChunks = kHalf / 32; // tcgen05.st.x32 per warp per window
static_assert(NW == 2 * NQ, "one warp per (lane quarter, ear)");
static_assert(SW + R == kCols && 2 * kCols == 512, "two window buffers fill the 512 columns");
static_assert(R % 4 == 0 && ((R / 4) & 1), "lane stride must be an odd number of 16-byte groups");
static_assert(R == 32 + 16 + 4, "a slice is loaded as x32 + x16 + x4 columns");
static_assert(kTile % kMixBox == 0, "tiles start on a row of the 3-D source view");

// ---- 32 consecutive samples, widened to FP32 (conflict-free: the lane stride R is an odd
// number of 16-byte groups) ------------------------------------------------------------------
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

// R = 52 columns starting at taddr into v (async; valid after tm_wait_ld(v))
__device__ __forceinline__ void tm_ld(uint32_t taddr, uint32_t (&v)[R])
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
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]),
          "=r"(v[38]), "=r"(v[39]), "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]),
          "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47])
        : "r"(taddr + 32)
        : "memory");
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v[48]), "=r"(v[49]), "=r"(v[50]), "=r"(v[51])
                 : "r"(taddr + 48)
                 : "memory");
}

// Accumulators: the R outputs of a lane as R/2 pairs, each a 64-bit register pair that one
// packed FP32 FMA (fma.rn.f32x2: two independent round-to-nearest FMAs, the same results as
// two fmaf) updates, so a tap costs R/2 FMA instructions.
constexpr int RP = R / 2;
static_assert(R % 2 == 0, "outputs per lane in pairs");

// Wait for this thread's outstanding tcgen05.ld.  v and acc are threaded through the
// statements (volatile statements keep their order), so no use of the loaded registers moves
// above the wait and every FMA into acc issued before it stays before it: the FMAs of
// consecutive taps are never interleaved on the same accumulator.
__device__ __forceinline__ void tm_wait_ld(uint32_t (&v)[R], uint64_t (&acc)[RP])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15]), "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]), "+r"(v[22]), "+r"(v[23]), "+r"(v[24]), "+r"(v[25])
                 :
                 : "memory");
    asm volatile(""
                 : "+r"(v[26]), "+r"(v[27]), "+r"(v[28]), "+r"(v[29]), "+r"(v[30]), "+r"(v[31]), "+r"(v[32]), "+r"(v[33]), "+r"(v[34]), "+r"(v[35]), "+r"(v[36]), "+r"(v[37]), "+r"(v[38]), "+r"(v[39]), "+r"(v[40]), "+r"(v[41]), "+r"(v[42]), "+r"(v[43]), "+r"(v[44]), "+r"(v[45]), "+r"(v[46]), "+r"(v[47]), "+r"(v[48]), "+r"(v[49]), "+r"(v[50]), "+r"(v[51])
                 :
                 : "memory");
    asm volatile(""
                 : "+l"(acc[0]), "+l"(acc[1]), "+l"(acc[2]), "+l"(acc[3]), "+l"(acc[4]), "+l"(acc[5]), "+l"(acc[6]), "+l"(acc[7]), "+l"(acc[8]), "+l"(acc[9]), "+l"(acc[10]), "+l"(acc[11]), "+l"(acc[12]), "+l"(acc[13]), "+l"(acc[14]), "+l"(acc[15]), "+l"(acc[16]), "+l"(acc[17]), "+l"(acc[18]), "+l"(acc[19]), "+l"(acc[20]), "+l"(acc[21]), "+l"(acc[22]), "+l"(acc[23]), "+l"(acc[24]), "+l"(acc[25])
                 :
                 : "memory");
}

// Keep every FMA into acc after this point (issued after a TMEM load, so that the load is
// in flight while they run).
__device__ __forceinline__ void tie_acc(uint64_t (&acc)[RP])
{
    asm volatile(""
                 : "+l"(acc[0]), "+l"(acc[1]), "+l"(acc[2]), "+l"(acc[3]), "+l"(acc[4]), "+l"(acc[5]), "+l"(acc[6]), "+l"(acc[7]), "+l"(acc[8]), "+l"(acc[9]), "+l"(acc[10]), "+l"(acc[11]), "+l"(acc[12]), "+l"(acc[13]), "+l"(acc[14]), "+l"(acc[15]), "+l"(acc[16]), "+l"(acc[17]), "+l"(acc[18]), "+l"(acc[19]), "+l"(acc[20]), "+l"(acc[21]), "+l"(acc[22]), "+l"(acc[23]), "+l"(acc[24]), "+l"(acc[25])
                 :
                 : "memory");
}

// acc[i] += w * (v[2i], v[2i+1]) for the R outputs of the lane
__device__ __forceinline__ void fma_slice(uint64_t (&acc)[RP], const uint32_t (&v)[R], uint32_t w)
{
    uint64_t ww;
    asm("mov.b64 %0, {%1, %1};" : "=l"(ww) : "r"(w));
#pragma unroll
    for (int i = 0; i < RP; ++i) {
        uint64_t x;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "r"(v[2 * i]), "r"(v[2 * i + 1]));
        asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc[i]) : "l"(ww), "l"(x));
    }
}

// Barrier of the two warps of lane quarter q (named barrier 1 + q, 64 threads) that also
// returns the AND of `ok` over them; TMEM accesses before it are ordered before those after.
__device__ __forceinline__ bool pair_sync_all(int q, bool ok)
{
    uint32_t r;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    asm volatile(
        "{\n\t.reg .pred p, v;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred v, %2, 64, p;\n\t"
        "selp.u32 %0, 1, 0, v;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)ok), "r"(1 + q)
        : "memory");
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return r != 0;
}

// This warp's half of a window (kHalf columns of its 32 TMEM lanes): shared memory ->
// registers -> tcgen05.st, all loads issued before the first store.
template <typename T>
__device__ __forceinline__ void copy_half(const T *src, uint32_t dst)
{
    uint32_t v[kCopyChunks][32];
#pragma unroll
    for (int c = 0; c < kCopyChunks; ++c) Load32<T>::run(src + 32 * c, v[c]);
#pragma unroll
    for (int c = 0; c < kCopyChunks; ++c) tm_st32(dst + 32 * c, v[c]);
}

// Apply n taps {column, weight bits} of this warp's ear to acc (n even: the lists are padded
// with zero-weight taps, and at least 4 readable entries follow each list).  TMEM loads are
// double-buffered: the next tap's slice is in flight while the current tap's FMAs issue.
__device__ __forceinline__ void apply_taps(uint64_t (&acc)[RP], uint32_t tw, const int2 *taps, int n)
{
    if (n <= 0) return;
    uint32_t A[R], B[R];
    int2 t0 = taps[0], t1 = taps[1];
    tm_ld(tw + (uint32_t)t0.x, A);
    for (int i = 0; i < n; i += 2) {
        const int2 t2 = taps[i + 2], t3 = taps[i + 3];
        tm_wait_ld(A, acc);
        tm_ld(tw + (uint32_t)t1.x, B);
        tie_acc(acc);
        fma_slice(acc, A, (uint32_t)t0.y);
        tm_wait_ld(B, acc);
        if (i + 2 < n) tm_ld(tw + (uint32_t)t2.x, A);
        tie_acc(acc);
        fma_slice(acc, B, (uint32_t)t1.y);
        t0 = t2;
        t1 = t3;
    }
}

// Issue the TMA loads of unit u into a pipeline stage (all lanes of the producer warp).
template <typename T>
__device__ __forceinline__ void issue_unit(const CUtensorMap *tmap, const CUtensorMap *tmap3,
                                           const MixArgs &a, int t, int s, int d, T *ybuf,
                                           unsigned char *rbuf, uint32_t full_bar, int lane)
{
    const int x0 = t * kTile - a.halo;
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

// Position (output tile t, source s) of a unit; units are ordered tile-major.  Advanced by
// small steps without a division (n <= the ring depth).
struct UnitPos {
    int t, s;
    __device__ __forceinline__ void advance(int n, int n_src)
    {
        s += n;
        while (s >= n_src) {
            s -= n_src;
            ++t;
        }
    }
};

// Record index for a direction id: the silent record for an id out of range.
__device__ __forceinline__ int checked_dir(const MixArgs &a, int d, int lane)
{
    if ((unsigned)d >= (unsigned)a.n_dirs) {
        if (lane == 0) atomicOr(a.status, DEV_BAD_DIR);
        d = a.n_dirs;
    }
    return d;
}

// Record: int4 {n_seg, 0, 0, 0}, int2 cnt[nchunk] {n_left, n_right} per segment, then per
// segment its left taps and right taps as int2 {window column, weight bits}, each list padded
// to an even length with zero-weight taps, and 4 padding entries at the end.
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
    int *relcnt = reinterpret_cast<int *>(bars + 2 * stages) + 4;      // [kMixMaxStages]
    int *last_issued = relcnt + kMixMaxStages;                         // [kMixMaxStages]
    int *dircache = last_issued + kMixMaxStages;                       // [kMixDirCache]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        prefetch_tensormap(&tmap);
        prefetch_tensormap(&tmap3);
        for (int i = 0; i < stages; ++i) {
            mbar_init(smem_addr(&bars[i]), 1);              // full: producer + tx bytes
            mbar_init(smem_addr(&bars[stages + i]), NW);    // empty: one arrive per warp
        }
        *abort_flag = 0;
        for (int i = 0; i < kMixMaxStages; ++i) {
            relcnt[i] = 0;
            last_issued[i] = -1;
        }
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

    const int64_t u_begin = a.part.first(blockIdx.x);
    const int64_t u_end = a.part.first(blockIdx.x + 1);
    const int n_units = (int)(u_end - u_begin);
    UnitPos pos0;                                   // position of this CTA's first unit
    pos0.t = (int)(u_begin / a.n_src);
    pos0.s = (int)(u_begin - (int64_t)pos0.t * a.n_src);
    // directions of this CTA's first kMixDirCache units, staged once
    const int n_cached = n_units < kMixDirCache ? n_units : kMixDirCache;
    {
        UnitPos p = pos0;
        p.advance(threadIdx.x, a.n_src);
        for (int i = threadIdx.x; i < n_cached; i += blockDim.x) {
            dircache[i] = __ldg(a.dir + p.s);
            p.advance(blockDim.x, a.n_src);
        }
    }
    __syncthreads();

    // Issue unit k (local index, at position p) into stage st (all lanes of the calling warp).
    auto issue = [&](int k, UnitPos p, int st) {
        const int d = checked_dir(a, k < n_cached ? dircache[k] : __ldg(a.dir + p.s), lane);
        issue_unit<T>(&tmap, &tmap3, a, p.t, p.s, d, ybuf + (size_t)st * a.buf_elems,
                      rbuf + (size_t)st * a.rec_bytes, smem_addr(&bars[st]), lane);
        if (lane == 0) last_issued[st] = k;
    };
    // A warp is done with unit k (at position p, stage st, phase parity ph): arrive on the
    // stage's empty barrier; the last of the NW warps to arrive refills the stage with unit
    // k + stages at once.  Returns false on a timeout.
    auto release = [&](int k, UnitPos p, int st, uint32_t ph) {
        __syncwarp();
        int last = 0;
        if (lane == 0) {
            mbar_arrive(smem_addr(&bars[stages + st]));
            last = atomicAdd(&relcnt[st], 1) == NW - 1;
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (!last) return true;
        if (lane == 0) relcnt[st] = 0;
        if (k + stages >= n_units) return true;
        // every warp has arrived: the phase completes (its acquire orders their reads of the
        // stage before the copy that overwrites it)
        if (!mbar_wait_bounded(smem_addr(&bars[stages + st]), ph, abort_flag, a.status))
            return false;
        p.advance(stages, a.n_src);
        issue(k + stages, p, st);
        return true;
    };

    if (n_units > 0) {
        // ---- compute: warp (q, ear) ----
        const int q = warp & (NQ - 1), ear = warp / NQ;
        const uint32_t tq = tmem_base + ((uint32_t)(32 * q) << 16);
        const int lane_off = (q * 32 + lane) * R;
        const int n_seg = a.nseg;
        const int64_t n_steps = (int64_t)n_units * n_seg;
        uint64_t acc[RP];
#pragma unroll
        for (int i = 0; i < RP; ++i) acc[i] = 0;
        int slot = a.part.slot_base(blockIdx.x, pos0.t), run_n = 0;

        // the window of a step (stage st, segment seg) for this warp's half
        auto window_src = [&](int st, int seg) {
            return ybuf + (size_t)st * a.buf_elems + a.halo + lane_off - (seg + 1) * SW + kHalf * ear;
        };
        // prologue: fill the ring, the first window into buffer 0
        if (warp == 0) {
            UnitPos p = pos0;
            for (int k0 = 0; k0 < n_units && k0 < stages; ++k0) {
                issue(k0, p, k0);
                p.advance(1, a.n_src);
            }
        }
        bool ok = mbar_wait_bounded(smem_addr(&bars[0]), 0u, abort_flag, a.status);
        if (ok) copy_half<T>(window_src(0, 0), tq + (uint32_t)(kHalf * ear));
        tm_wait_st();
        ok = pair_sync_all(q, ok);

        // current step: unit k at position pos, stage st, parity ph; segment seg
        int k = 0, st = 0, seg = 0, toff = 0;
        uint32_t ph = 0;
        UnitPos pos = pos0;
        for (int64_t j = 0; ok && j < n_steps; ++j) {
            // next step
            const bool last_seg = seg == n_seg - 1;
            const int k1 = last_seg ? k + 1 : k;
            const int seg1 = last_seg ? 0 : seg + 1;
            int st1 = st;
            uint32_t ph1 = ph;
            if (last_seg && ++st1 == stages) {
                st1 = 0;
                ph1 ^= 1u;
            }
            const bool have_next = k1 < n_units;
            bool ok_next = true;
            if (have_next && last_seg)
                ok_next = mbar_wait_bounded(smem_addr(&bars[st1]), ph1, abort_flag, a.status);
            // the next window's half: the left-ear warp copies it before its taps, the
            // right-ear warp after them, so that on their shared SM sub-partition one warp's
            // copy overlaps the other's FMAs
            const bool copy = have_next && ok_next;
            const T *nsrc = window_src(copy ? st1 : st, copy ? seg1 : seg);
            const uint32_t ndst = tq + (uint32_t)(kCols * ((j + 1) & 1) + kHalf * ear);
            if (copy && ear == 0) copy_half<T>(nsrc, ndst);
            // taps of this warp's ear in segment seg of unit k
            const unsigned char *rec = rbuf + (size_t)st * a.rec_bytes;
            const int2 c = reinterpret_cast<const int2 *>(rec + 16)[seg];
            const int2 *taps = reinterpret_cast<const int2 *>(rec + 16 + 8 * a.nchunk) + toff +
                               (ear ? c.x : 0);
            apply_taps(acc, tq + (uint32_t)(kCols * (j & 1)), taps, ear ? c.y : c.x);
            toff += c.x + c.y;
            if (last_seg && !release(k, pos, st, ph)) ok_next = false;   // last read of unit k's stage
            if (copy && ear == 1) copy_half<T>(nsrc, ndst);
            tm_wait_st();
            ok = pair_sync_all(q, ok_next);
            if (last_seg) {
                // unit k done: flush the run at its end
                ++run_n;
                const bool tile_end = (k + 1 == n_units) || (pos.s + 1 == a.n_src);
                if (run_n == a.part.gs || tile_end) {
                    float4 *p = reinterpret_cast<float4 *>(
                        a.partial + ((size_t)pos.t * a.slots + slot) * 2 * kTile + ear * kTile + lane_off);
#pragma unroll
                    for (int i = 0; i < R / 4; ++i) {
                        float x0, x1, x2, x3;
                        asm("mov.b64 {%0, %1}, %2;" : "=f"(x0), "=f"(x1) : "l"(acc[2 * i]));
                        asm("mov.b64 {%0, %1}, %2;" : "=f"(x2), "=f"(x3) : "l"(acc[2 * i + 1]));
                        p[i] = make_float4(x0, x1, x2, x3);
                    }
#pragma unroll
                    for (int i = 0; i < RP; ++i) acc[i] = 0;
                    ++slot;
                    run_n = 0;
                }
                toff = 0;
                pos.advance(1, a.n_src);
                if (tile_end && k1 < n_units) {
                    slot = a.part.slot_base(blockIdx.x, pos.t);   // the next tile's first slot
                    run_n = 0;
                }
            }
            k = k1;
            seg = seg1;
            st = st1;
            ph = ph1;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) {
        // let every copy still in flight land before the CTA exits (bounded; immediate unless
        // a wait timed out): the last unit issued into each stage
        for (int st = 0; st < stages; ++st) {
            const int j = last_issued[st];
            if (j < 0) continue;
            const uint32_t fb = smem_addr(&bars[st]);
            const uint32_t par = (uint32_t)((j / stages) & 1);
            const uint64_t t0 = global_timer_ns();
            while (!mbar_try_wait(fb, par) && global_timer_ns() - t0 < kWaitLimitNs) {
            }
        }
    }
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem_base) : "memory");
}

}  // namespace

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
