// mix_sparse_tmem.cu -- the sparse reflection gather-FMA mix (the method, Eq. 2, with the
// resonance moved after the mix):
//
//     z_e[n] = sum_s sum_k w_{d(s),e,k} * y_s[n - i_{d(s),e,k}]        (Sec. I footnote 2)
//
// with each lane's source window held in tensor memory (TMEM).
//
// A tile of 6656 outputs is split over the 4 TMEM lane quarters x 32 lanes, R = 52
// consecutive outputs per lane.  Five warps share each lane quarter q: four tap warps
// q + 4 (ear + 2 half) read its TMEM rows, each for one ear and one half (26 outputs) of every
// lane's outputs, and copy warp q + 16 writes them.  For every (source, tile) unit and every window segment of SW = 204 filter offsets,
// row (lane) holds the 256 samples y[n - (seg+1) SW .. n - (seg+1) SW + 256) of its outputs'
// window.  A tap at offset o then needs y[n + r - o] for r < R, the contiguous column range
// starting at (seg+1) SW - o, of which a tap warp reads its half: one warp-uniform
// tcgen05.ld of 26 columns (no branch, no register indexing) followed by 13 packed FP32 FMAs
// (fma.rn.f32x2, two outputs each).
//
// The window is double-buffered in the 512 TMEM columns.  The copy warp of a quarter fills
// one buffer (shared memory -> registers -> tcgen05.st) while the quarter's tap warps apply
// their taps to the other, so the shared-memory-bound copy and the FMA-bound taps run at the
// same time on different warps; per quarter and buffer a "full" mbarrier (copy warp -> tap
// warps) and an "empty" mbarrier (tap warps -> copy warp) hand the buffers over.
// A ring of up to 6 shared-memory stages holds each unit's source tile (tensor TMA, 256-sample
// halo, hardware zero fill outside [0, len)) and the direction's tap record (bulk copy); a
// producer warp issues every load, refilling each stage with the unit `stages` ahead as soon
// as the 20 compute warps have released it.
// Work is a persistent balanced range of units per CTA; register accumulators are folded
// every few sources (about 128 products per output) into per-lane FP32 accumulators in shared
// memory, which are flushed every <= 64 sources into partial slots that the reduction sums
// in a fixed order (two short sums instead of one long one: the FP32 rounding error grows
// with the square root of a sum's length).
// All waits are bounded: a wait that expires raises the CTA's abort flag, and every other
// wait then returns at once, so all warps leave their loops.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels.h"

namespace hrir {

namespace {

constexpr int R = kSparseR;             // outputs per lane
constexpr int NQ = kSparseQuarters;     // TMEM lane quarters
constexpr int NH = 2;                   // tap warps per (lane quarter, ear), R / NH outputs each
constexpr int RS = R / NH;              // outputs of a lane per tap warp
constexpr int NTW = 2 * NH * NQ;        // tap warps (lane quarter, ear, half)
constexpr int NC = NTW + NQ;            // compute warps: tap warps + one copy warp per quarter
constexpr int NW = kSparseWarps;        // compute warps + the producer warp (TMA issue)
constexpr int kTile = kSparseTile;      // outputs per tile
constexpr int kCols = kSparseTmemCols;  // TMEM columns per window buffer
constexpr int SW = kSparseSegment;      // filter offsets per window segment (= kCols - R)
constexpr int kCopyChunks = 1;          // tcgen05.st.x32 per copy batch (32 columns)
static_assert(NW == NC + 1 && NTW % NQ == 0, "compute warp w works on TMEM lane quarter w % 4");
static_assert(kCols % (32 * kCopyChunks) == 0, "a window is whole copy batches");
static_assert(kMixWindowBars == 4 * NQ, "a full and an empty barrier per quarter and buffer");
static_assert(SW + R == kCols && 2 * kCols == 512, "two window buffers fill the 512 columns");
static_assert(R % 4 == 0 && ((R / 4) & 1), "lane stride must be an odd number of 16-byte groups");
static_assert(RS == 16 + 8 + 2, "a slice is loaded as x16 + x8 + x2 columns");
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

// RS = 26 columns starting at taddr into v (async; valid after tm_wait_ld(v))
__device__ __forceinline__ void tm_ld(uint32_t taddr, uint32_t (&v)[RS])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23])
                 : "r"(taddr + 16)
                 : "memory");
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
                 : "=r"(v[24]), "=r"(v[25])
                 : "r"(taddr + 24)
                 : "memory");
}

// Accumulators: the RS outputs of a lane as RS/2 pairs, each a 64-bit register pair that one
// packed FP32 FMA (fma.rn.f32x2: two independent round-to-nearest FMAs, the same results as
// two fmaf) updates, so a tap costs RS/2 FMA instructions.
constexpr int RP = RS / 2;
static_assert(RS % 2 == 0, "outputs per lane in pairs");

// Wait for this thread's outstanding tcgen05.ld.  v and acc are threaded through the
// statements (volatile statements keep their order), so no use of the loaded registers moves
// above the wait and every FMA into acc issued before it stays before it: the FMAs of
// consecutive taps are never interleaved on the same accumulator.
__device__ __forceinline__ void tm_wait_ld(uint32_t (&v)[RS], uint64_t (&acc)[RP])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15]), "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]), "+r"(v[22]), "+r"(v[23]), "+r"(v[24]), "+r"(v[25])
                 :
                 : "memory");
    asm volatile(""
                 : "+l"(acc[0]), "+l"(acc[1]), "+l"(acc[2]), "+l"(acc[3]), "+l"(acc[4]), "+l"(acc[5]), "+l"(acc[6]), "+l"(acc[7]), "+l"(acc[8]), "+l"(acc[9]), "+l"(acc[10]), "+l"(acc[11]), "+l"(acc[12])
                 :
                 : "memory");
}

// Keep every FMA into acc after this point (issued after a TMEM load, so that the load is
// in flight while they run).
__device__ __forceinline__ void tie_acc(uint64_t (&acc)[RP])
{
    asm volatile(""
                 : "+l"(acc[0]), "+l"(acc[1]), "+l"(acc[2]), "+l"(acc[3]), "+l"(acc[4]), "+l"(acc[5]), "+l"(acc[6]), "+l"(acc[7]), "+l"(acc[8]), "+l"(acc[9]), "+l"(acc[10]), "+l"(acc[11]), "+l"(acc[12])
                 :
                 : "memory");
}

// acc[i] += w * (v[2i], v[2i+1]) for the RS outputs of the lane
__device__ __forceinline__ void fma_slice(uint64_t (&acc)[RP], const uint32_t (&v)[RS], uint32_t w)
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

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// One window (kCols columns of this warp's 32 TMEM lanes): shared memory -> registers ->
// tcgen05.st, in batches of kCopyChunks x 32 columns whose loads all issue before their
// stores.
template <typename T>
__device__ __forceinline__ void copy_window(const T *src, uint32_t dst)
{
#pragma unroll 1
    for (int b = 0; b < kCols; b += 32 * kCopyChunks) {
        uint32_t v[kCopyChunks][32];
#pragma unroll
        for (int c = 0; c < kCopyChunks; ++c) Load32<T>::run(src + b + 32 * c, v[c]);
#pragma unroll
        for (int c = 0; c < kCopyChunks; ++c) tm_st32(dst + (uint32_t)(b + 32 * c), v[c]);
    }
}

// Apply n taps {column, weight bits} of this warp's ear to acc (at least 4 readable entries
// follow each list).  One slice in registers at a time: the load latency of one tap warp is
// covered by the FMAs of the other three tap warps on the same SM sub-partition; the next
// tap's entry is read from shared memory while the current slice is in flight.
__device__ __forceinline__ void apply_taps(uint64_t (&acc)[RP], uint32_t tw, const int2 *taps, int n)
{
    uint32_t A[RS];
    int2 t = taps[0];
#pragma unroll 2
    for (int i = 0; i < n; ++i) {
        tm_ld(tw + (uint32_t)t.x, A);
        const int2 tn = taps[i + 1];
        tm_wait_ld(A, acc);
        fma_slice(acc, A, (uint32_t)t.y);
        tie_acc(acc);      // these FMAs read A before the next load overwrites it
        t = tn;
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
__global__ void __maxnreg__(80)
    sparse_tmem_kernel(const __grid_constant__ CUtensorMap tmap,
                       const __grid_constant__ CUtensorMap tmap3, const MixArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int stages = a.stages;
    T *ybuf = reinterpret_cast<T *>(smem);
    unsigned char *rbuf = smem + (size_t)stages * a.buf_elems * sizeof(T);
    uint64_t *bars = reinterpret_cast<uint64_t *>(rbuf + (size_t)stages * a.rec_bytes);
    uint64_t *wbars = bars + 2 * stages;        // [full, empty][quarter][buffer]
    volatile int *abort_flag = reinterpret_cast<volatile int *>(wbars + kMixWindowBars);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(wbars + kMixWindowBars) + 1;
    int *last_issued = reinterpret_cast<int *>(wbars + kMixWindowBars) + 4;  // [kMixMaxStages]
    int *dircache = last_issued + kMixMaxStages;                       // [kMixDirCache]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        prefetch_tensormap(&tmap);
        prefetch_tensormap(&tmap3);
        for (int i = 0; i < stages; ++i) {
            mbar_init(smem_addr(&bars[i]), 1);              // full: producer + tx bytes
            mbar_init(smem_addr(&bars[stages + i]), NC);    // empty: one arrive per compute warp
        }
        for (int i = 0; i < 2 * NQ; ++i) {
            mbar_init(smem_addr(&wbars[i]), 1);             // window full: the copy warp
            mbar_init(smem_addr(&wbars[2 * NQ + i]), 2 * NH); // window empty: the tap warps
        }
        *abort_flag = 0;
        for (int i = 0; i < kMixMaxStages; ++i) last_issued[i] = -1;
        mbar_fence_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                         smem_addr(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
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
    // A compute warp is done with the stage st of its current unit (every read of it issued
    // and complete): one arrive per compute warp on the stage's empty barrier.
    auto release = [&](int st) {
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&bars[stages + st]));
    };

    if (n_units > 0 && warp == NW - 1) {
        // ---- producer: fills the ring, then refills each stage as soon as the NC compute
        // warps have released it, with the unit `stages` ahead ----
        UnitPos p = pos0;
        for (int k0 = 0; k0 < n_units && k0 < stages; ++k0) {
            issue(k0, p, k0);
            p.advance(1, a.n_src);
        }
        int st = 0;
        uint32_t ph = 0;
        for (int r = 0; r + stages < n_units; ++r) {
            if (!mbar_wait_bounded(smem_addr(&bars[stages + st]), ph, abort_flag, a.status)) break;
            issue(r + stages, p, st);
            p.advance(1, a.n_src);
            if (++st == stages) {
                st = 0;
                ph ^= 1u;
            }
        }
    } else if (n_units > 0) {
        const int q = warp & (NQ - 1);
        const uint32_t tq = tmem_base + ((uint32_t)(32 * q) << 16);
        const int lane_off = (q * 32 + lane) * R;
        const int n_seg = a.nseg;
        const int64_t n_steps = (int64_t)n_units * n_seg;
        const uint32_t win_full = smem_addr(&wbars[q * 2]);           // + 8 * buffer
        const uint32_t win_empty = smem_addr(&wbars[2 * NQ + q * 2]);  // + 8 * buffer

        // step j: unit k at position pos, stage st with phase parity ph, segment seg; window
        // buffer j & 1, used for the (j >> 1)-th time
        int k = 0, st = 0, seg = 0;
        uint32_t ph = 0;
        UnitPos pos = pos0;
        if (warp >= NTW) {
            // ---- copy warp of lane quarter q ----
            for (int64_t j = 0; j < n_steps; ++j) {
                const uint32_t buf = (uint32_t)j & 1u;
                if (seg == 0 && !mbar_wait_bounded(smem_addr(&bars[st]), ph, abort_flag, a.status))
                    break;
                if (j >= 2 && !mbar_wait_bounded(win_empty + 8 * buf, (uint32_t)((j >> 1) - 1) & 1u,
                                                 abort_flag, a.status))
                    break;
                tc_fence_after();
                copy_window<T>(ybuf + (size_t)st * a.buf_elems + a.halo + lane_off - (seg + 1) * SW,
                               tq + kCols * buf);
                tm_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(win_full + 8 * buf);
                if (seg == n_seg - 1) {
                    release(st);                              // last read of unit k's stage
                    pos.advance(1, a.n_src);
                    ++k;
                    seg = 0;
                    if (++st == stages) {
                        st = 0;
                        ph ^= 1u;
                    }
                } else {
                    ++seg;
                }
            }
        } else {
            // ---- tap warp (lane quarter q, ear, half): outputs [RS half, RS half + RS) of
            // each lane ----
            const int ear = (warp / NQ) & 1, half = warp / (2 * NQ);
            uint64_t acc[RP];
#pragma unroll
            for (int i = 0; i < RP; ++i) acc[i] = 0;
            // this lane's fold accumulators in shared memory, [RP][32] packed pairs per warp
            // (a warp's 8-byte accesses are contiguous: conflict-free); only this thread
            // touches them
            uint64_t *racc = reinterpret_cast<uint64_t *>(smem + a.runacc_off) + (size_t)warp * RP * 32 + lane;
#pragma unroll
            for (int i = 0; i < RP; ++i) racc[i * 32] = 0;
            int slot = a.part.slot_base(blockIdx.x, pos0.t), run_n = 0, toff = 0, fold_n = 0;
            for (int64_t j = 0; j < n_steps; ++j) {
                const uint32_t buf = (uint32_t)j & 1u;
                if (seg == 0 && !mbar_wait_bounded(smem_addr(&bars[st]), ph, abort_flag, a.status))
                    break;
                if (!mbar_wait_bounded(win_full + 8 * buf, (uint32_t)(j >> 1) & 1u, abort_flag, a.status))
                    break;
                tc_fence_after();
                // taps of this warp's ear in segment seg of unit k
                const unsigned char *rec = rbuf + (size_t)st * a.rec_bytes;
                const int2 c = reinterpret_cast<const int2 *>(rec + 16)[seg];
                const int2 *taps = reinterpret_cast<const int2 *>(rec + 16 + 8 * a.nchunk) + toff +
                                   (ear ? c.x : 0);
                apply_taps(acc, tq + kCols * buf + RS * half, taps, ear ? c.y : c.x);  // ends with wait::ld
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(win_empty + 8 * buf);
                toff += c.x + c.y;
                if (seg == n_seg - 1) {
                    release(st);                              // last read of unit k's stage
                    // unit k done: every `fold` sources the registers are added into the
                    // shared-memory accumulators; at the end of the run their sum goes to the
                    // run's partial slot
                    ++run_n;
                    ++fold_n;
                    const bool tile_end = (k + 1 == n_units) || (pos.s + 1 == a.n_src);
                    const bool flush = run_n == a.part.gs || tile_end;
                    if (flush || fold_n == a.fold) {
                        fold_n = 0;
                        uint64_t one2;
                        asm("mov.b64 %0, {%1, %1};" : "=l"(one2) : "r"(0x3f800000u));
                        if (flush) {
                            float2 *p = reinterpret_cast<float2 *>(a.partial + ((size_t)pos.t * a.slots + slot) * 2 * kTile +
                                                                   ear * kTile + lane_off + RS * half);
#pragma unroll
                            for (int i = 0; i < RP; ++i) {
                                uint64_t x = racc[i * 32];
                                asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(x) : "l"(one2), "l"(acc[i]));
                                float x0, x1;
                                asm("mov.b64 {%0, %1}, %2;" : "=f"(x0), "=f"(x1) : "l"(x));
                                p[i] = make_float2(x0, x1);
                                racc[i * 32] = 0;
                            }
                            ++slot;
                            run_n = 0;
                        } else {
#pragma unroll
                            for (int i = 0; i < RP; ++i) {
                                uint64_t x = racc[i * 32];
                                asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(x) : "l"(one2), "l"(acc[i]));
                                racc[i * 32] = x;
                            }
                        }
#pragma unroll
                        for (int i = 0; i < RP; ++i) acc[i] = 0;
                    }
                    toff = 0;
                    pos.advance(1, a.n_src);
                    ++k;
                    seg = 0;
                    if (++st == stages) {
                        st = 0;
                        ph ^= 1u;
                    }
                    if (tile_end && k < n_units) {
                        slot = a.part.slot_base(blockIdx.x, pos.t);   // the next tile's first slot
                        run_n = 0;
                    }
                } else {
                    ++seg;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
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
