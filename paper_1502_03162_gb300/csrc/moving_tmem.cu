// moving_tmem.cu -- the mix of moving sources (a direction per segment, Eqs. 1-2 with per-segment
// reflection filters and a linear crossfade between consecutive segments' filters) on
// tensor-memory windows, the scheme of the static sparse kernel (mix_sparse_tmem.cu):
//
//     z_e[n] = sum_s (1 - a_n) (y_s * g_{s,jp(n),e})[n] + a_n (y_s * g_{s,jc(n),e})[n],
//     a_n = (n - j seg_len + 1) / seg_len for n in segment j,
//
// jc = min(j, n_seg - 1), jp = j - 1 for 1 <= j < n_seg and jp = jc otherwise (segment 0 and
// the filter tails use one filter).  Because a_n depends only on n, the sources' "previous"
// and "current" products are summed separately and combined once per output:
//     z_e[n] = (1 - a_n) P[n] + a_n C[n],  P = sum_s y_s * g_{s,jp,e},  C = sum_s y_s * g_{s,jc,e}.
//
// A 4096-output tile is 128 TMEM lanes x 32 outputs; with seg_len % 32 == 0 a lane's outputs
// lie in one segment, so its weights are one (previous, current) pair per tap.  Each lane's
// window of 256 samples (224 filter offsets + its 32 outputs) is double-buffered in the 512
// TMEM columns.  Per (unit = tile x source, lane quarter, ear) the quarter's builder warp makes
// a tap program in shared memory: the union of the tap offsets of the <= 5 table rows the
// quarter's segments use (shared-memory bitmask, ranks by a segmented warp scan; both ears'
// programs side by side), and for each union offset its window column and each row's weight
// (0 where a row lacks the offset).  The quarter's copy warp moves the window from the stage
// into TMEM, and its four tap warps (ear x half) walk the program: a warp-uniform tcgen05.ld
// of 16 columns (the next entry's load in flight while this one's FMAs run, two register
// sets), then 8 packed FMAs into the previous and 8 into the current accumulators with the
// weights of the lane's previous and current rows.  The source tile arrives by one 3-D TMA
// load of 32-sample rows with the 128-byte swizzle (16-byte chunk c of row r at chunk
// c ^ (r % 8)), so the copy warps' per-lane row reads hit distinct banks; the table rows of
// the tile's segments arrive by two bulk copies, issued by quarter 0's builder.  Accumulation
// over sources, folds, partial slots and bounded waits are those of the static kernel.
#include "kernels.h"

namespace hrir {

namespace {

constexpr int R = kMvR;             // outputs per lane
constexpr int RS = R / 2;           // outputs per tap warp (two halves)
constexpr int RP = RS / 2;          // packed pairs per accumulator set
constexpr int NQ = 4;               // TMEM lane quarters
constexpr int NTW = 16;             // tap warps: (quarter, ear, half)
constexpr int NC = NTW + NQ;        // tap and copy warps
constexpr int NB = NQ;              // program builders, one per lane quarter
constexpr int NW = NC + NB;         // (the builder of quarter 0 also issues the loads)
constexpr int kCols = kMvCols;
constexpr int SW = kMvSpan;         // 224 filter offsets per window
constexpr int kWords = (SW + 31) / 32;   // union bitmask words
constexpr int kProgCap = kMvMaxU + 2;    // entries (2 padding entries for the read-ahead)
static_assert(RS == 16 && kCols == 256, "x16 slices of 256-column windows");

constexpr int kRowsQ = kMvSegQ + 1;      // table rows one lane quarter uses
// tap program of one (lane quarter, ear): n entries of window column and, per table row the
// quarter uses (rows jlo .. jlo + 4), the row's weight at that offset (0 where it lacks it)
struct alignas(16) Prog {
    int n, pad[3];
    uint32_t bits[8];                   // union of the offsets, one bit per offset
    float w[kProgCap][kRowsQ];
    float w_pad[4];                     // slack for the 16-byte zeroing stores
    int col[kProgCap];
};
static_assert(offsetof(Prog, w) % 16 == 0 && sizeof(Prog) % 16 == 0,
              "16-byte aligned weight rows in every program of an array");
constexpr int kProgBytes = (int)sizeof(Prog);   // the programs are indexed as an array
constexpr int kProgsBytes = 2 * NQ * 2 * kProgBytes;   // [window buffer][quarter][ear]
constexpr int kRunAccBytes = NTW * 2 * RP * 32 * 8;    // fold accumulators, two sets per tap warp
constexpr int kTableIdxBytes = kMvMaxTableSegs * 2 * kMvMaxK * 2;
constexpr int kTableWBytes = kMvMaxTableSegs * 2 * kMvMaxK * 4;
constexpr int kStageTableBytes = kTableIdxBytes + kTableWBytes;
constexpr int kWinBytes = kMvBufElems * 4;             // 17408 = 17 x 1024
static_assert(kWinBytes % 1024 == 0, "every window buffer 1024-byte aligned (128-byte swizzle)");
static_assert(kTableIdxBytes % 16 == 0 && kStageTableBytes % 16 == 0, "16-byte table blocks");

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

// 16 columns starting at taddr into v (async; valid after tm_wait_ld)
__device__ __forceinline__ void tm_ld16(uint32_t taddr, uint32_t (&v)[RS])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                 : "r"(taddr)
                 : "memory");
}

// wait for this thread's tcgen05.ld; v and both accumulator sets are threaded through so that no
// use of v moves above the wait and no FMA of the previous tap moves below it
__device__ __forceinline__ void tm_wait_ld(uint32_t (&v)[RS], uint64_t (&p)[RP], uint64_t (&c)[RP])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]), "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]), "+r"(v[15])
                 :
                 : "memory");
    asm volatile(""
                 : "+l"(p[0]), "+l"(p[1]), "+l"(p[2]), "+l"(p[3]), "+l"(p[4]), "+l"(p[5]), "+l"(p[6]), "+l"(p[7]),
                   "+l"(c[0]), "+l"(c[1]), "+l"(c[2]), "+l"(c[3]), "+l"(c[4]), "+l"(c[5]), "+l"(c[6]), "+l"(c[7])
                 :
                 : "memory");
}

__device__ __forceinline__ void tie_acc(uint64_t (&p)[RP], uint64_t (&c)[RP])
{
    asm volatile(""
                 : "+l"(p[0]), "+l"(p[1]), "+l"(p[2]), "+l"(p[3]), "+l"(p[4]), "+l"(p[5]), "+l"(p[6]), "+l"(p[7]),
                   "+l"(c[0]), "+l"(c[1]), "+l"(c[2]), "+l"(c[3]), "+l"(c[4]), "+l"(c[5]), "+l"(c[6]), "+l"(c[7])
                 :
                 : "memory");
}

// p[i] += wp * (v[2i], v[2i+1]), c[i] += wc * (v[2i], v[2i+1])   (packed FP32 FMAs)
__device__ __forceinline__ void fma_slice2(uint64_t (&p)[RP], uint64_t (&c)[RP], const uint32_t (&v)[RS], float wp,
                                           float wc)
{
    uint64_t wwp, wwc;
    asm("mov.b64 %0, {%1, %1};" : "=l"(wwp) : "r"(__float_as_uint(wp)));
    asm("mov.b64 %0, {%1, %1};" : "=l"(wwc) : "r"(__float_as_uint(wc)));
#pragma unroll
    for (int i = 0; i < RP; ++i) {
        uint64_t x;
        asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "r"(v[2 * i]), "r"(v[2 * i + 1]));
        asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(p[i]) : "l"(wwp), "l"(x));
        asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(c[i]) : "l"(wwc), "l"(x));
    }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Position (output tile t, source s) of a unit; units are ordered tile-major.
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

// table rows staged for tile t: segments [lo, lo + count)
struct TileRows {
    int lo, count;
};
__device__ __forceinline__ TileRows tile_rows(const MovingTmemArgs &a, int t)
{
    const int64_t n0 = (int64_t)t * kMvTile;
    const int ja = (int)(n0 / a.seg_len), jb = (int)((n0 + kMvTile - 1) / a.seg_len);
    int lo = ja - 1 < 0 ? 0 : ja - 1;
    lo = lo > a.n_seg - 1 ? a.n_seg - 1 : lo;
    const int hi = jb < a.n_seg - 1 ? jb : a.n_seg - 1;
    return {lo, hi - lo + 1};
}

// Issue the loads of unit (t, s) into a stage (lane 0 of the producer warp): the source tile
// with its 256-sample history as 136 swizzled rows of 32 samples (rows outside the source
// arrive as zeros), and the table rows of the tile's segments.
__device__ __forceinline__ void issue_unit(const CUtensorMap *tmap3, const MovingTmemArgs &a, int t, int s,
                                           uint32_t win, uint32_t tbl, uint32_t full_bar)
{
    const TileRows tr = tile_rows(a, t);
    const size_t row0 = ((size_t)s * a.n_seg + tr.lo) * 2 * a.k_max;
    const uint32_t idx_bytes = (uint32_t)(tr.count * 2 * a.k_max * 2);
    const uint32_t w_bytes = (uint32_t)(tr.count * 2 * a.k_max * 4);
    mbar_arrive_expect_tx(full_bar, (uint32_t)kWinBytes + idx_bytes + w_bytes);
    tma_load_3d(win, tmap3, 0, t * (kMvTile / 32) - kMvHalo / 32, s, full_bar);
    tma_load_1d(tbl, a.tap_idx + row0, idx_bytes, full_bar);
    tma_load_1d(tbl + kTableIdxBytes, a.tap_w + row0, w_bytes, full_bar);
}

// The table rows lane quarter q of tile t uses: rows [jlo, jlo + nrows) (<= 5, consecutive),
// and its segments [js0, js0 + nsq) (<= kMvSegQ).
struct QuarterRows {
    int js0, nsq, jlo, nrows;
};
__device__ __forceinline__ int jc_of(const MovingTmemArgs &a, int js) { return js < a.n_seg - 1 ? js : a.n_seg - 1; }
__device__ __forceinline__ int jp_of(const MovingTmemArgs &a, int js)
{
    return (js >= 1 && js < a.n_seg) ? js - 1 : jc_of(a, js);
}
__device__ __forceinline__ QuarterRows quarter_rows(const MovingTmemArgs &a, int t, int q)
{
    const int64_t nq0 = (int64_t)t * kMvTile + (int64_t)q * (kMvTile / NQ);
    const int js0 = (int)(nq0 / a.seg_len), js1 = (int)((nq0 + kMvTile / NQ - 1) / a.seg_len);
    const int jlo = jp_of(a, js0), jhi = jc_of(a, js1);
    return {js0, js1 - js0 + 1, jlo, jhi - jlo + 1};
}

// nnz of the rows of unit (t, s), quarter q: lane 2 r + e holds row jlo + r, ear e (loaded one
// unit ahead of its use, so that the global load's latency is hidden)
__device__ __forceinline__ int load_nnz(const MovingTmemArgs &a, const QuarterRows &qr, int s, int lane)
{
    return lane < 2 * qr.nrows ? (int)a.tap_nnz[((size_t)s * a.n_seg + qr.jlo + (lane >> 1)) * 2 + (lane & 1)] : 0;
}

// Build the tap programs of lane quarter q for unit (t, s) from the staged table rows (the
// quarter's builder warp; every lane calls it).  my_nnz: from load_nnz for this unit.
__device__ __forceinline__ void build_progs(const MovingTmemArgs &a, const TileRows &tr, const QuarterRows &qr,
                                            const int (&er)[3], const int (&ep)[3], const uint16_t *tidx,
                                            const float *tw, Prog *prog0, Prog *prog1, int lane, int my_nnz)
{
    // both ears' programs are built step by step side by side (independent latency chains)
    const int k = a.k_max;
    if (lane < 8) prog0->bits[lane] = 0u;
    else if (lane < 16) prog1->bits[lane - 8] = 0u;
    // this lane's entries (row, offset, weight) per ear; row -1 where there is none
    int ent_o[2][3], ent_r[2][3];
    float ent_w[2][3];
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const int r = er[m], p = ep[m];
            const int nz = __shfl_sync(0xffffffffu, my_nnz, (r < qr.nrows ? r : 0) * 2 + e);
            const bool live = r < qr.nrows && p < nz;
            const int rs = qr.jlo + r - tr.lo;              // staged row
            const int o = live ? (int)tidx[(rs * 2 + e) * k + p] : 0;
            const float wv = live ? tw[(rs * 2 + e) * k + p] : 0.f;
            if (live && ((nz > k && p == 0) || o >= a.refl_len)) atomicOr(a.status, DEV_BAD_TAP);
            const bool ok = live && o < a.refl_len;
            ent_r[e][m] = ok ? r : -1;
            ent_o[e][m] = ok ? o : 0;
            ent_w[e][m] = wv;
        }
    __syncwarp();
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        Prog *pg = e ? prog1 : prog0;
#pragma unroll
        for (int m = 0; m < 3; ++m)
            if (ent_r[e][m] >= 0) atomicOr(&pg->bits[ent_o[e][m] >> 5], 1u << (ent_o[e][m] & 31));
    }
    __syncwarp();
    // lanes 8 e + w (w < kWords): word w of ear e's union and the count of the words below it
    // (one scan in segments of 8 lanes for both ears)
    const int sl = lane & 7;
    const Prog *pl = lane < 8 ? prog0 : prog1;
    const uint32_t word = (lane < 16 && sl < kWords) ? pl->bits[sl] : 0u;
    int incl = __popc(word);
#pragma unroll
    for (int d = 1; d < 8; d <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, d, 8);
        if (sl >= d) incl += v;
    }
    const int excl = incl - __popc(word);
    int n[2];
    n[0] = __shfl_sync(0xffffffffu, incl, kWords - 1);
    n[1] = __shfl_sync(0xffffffffu, incl, 8 + kWords - 1);
    // zero the weight rows of the n entries and of the two padding entries
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        Prog *pg = e ? prog1 : prog0;
        float4 *wz = reinterpret_cast<float4 *>(&pg->w[0][0]);
        for (int i = lane; i < ((n[e] + 2) * kRowsQ + 3) / 4; i += 32) wz[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (lane < 2) pg->col[n[e] + lane] = 0;
        if (lane == 0) pg->n = n[e];
    }
    __syncwarp();
    // entry (row r, offset o) goes to union rank(o) = offsets below o
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        Prog *pg = e ? prog1 : prog0;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const int o = ent_o[e][m], src = 8 * e + (o >> 5);
            const int u = __shfl_sync(0xffffffffu, excl, src) +
                          __popc(__shfl_sync(0xffffffffu, word, src) & ((1u << (o & 31)) - 1u));
            if (ent_r[e][m] >= 0) {
                pg->col[u] = SW - o;
                pg->w[u][ent_r[e][m]] = ent_w[e][m];
            }
        }
    }
    __syncwarp();
}

// Shared memory: [stages] windows (1024-byte aligned), [stages] table blocks, barriers (full,
// empty per stage; full, empty per quarter and window buffer), abort flag, TMEM slot, last
// issued unit per stage, then the tap programs and the fold accumulators at the offsets the
// launcher passes.
// 24 warps put 6 on each SM sub-partition, whose 16384 registers then allow at most 85 a thread
__global__ void __maxnreg__(80) moving_tmem_kernel(const __grid_constant__ CUtensorMap tmap3, const MovingTmemArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int stages = a.stages;
    unsigned char *wins = smem;
    unsigned char *tbls = smem + (size_t)stages * kWinBytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(tbls + (size_t)stages * kStageTableBytes);
    uint64_t *wbars = bars + 2 * stages;            // [full, empty][quarter][buffer]
    volatile int *abort_flag = reinterpret_cast<volatile int *>(wbars + 4 * NQ);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(wbars + 4 * NQ) + 1;
    int *last_issued = reinterpret_cast<int *>(wbars + 4 * NQ) + 4;   // [kMixMaxStages]
    Prog *progs = reinterpret_cast<Prog *>(smem + a.prog_off);        // [buffer][quarter][ear]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (smem_addr(smem) & 1023u) {          // the 128-byte swizzle needs 1024-byte aligned windows
        if (threadIdx.x == 0) atomicOr(a.status, DEV_LAYOUT);
        return;
    }
    if (threadIdx.x == 0) {
        prefetch_tensormap(&tmap3);
        for (int i = 0; i < stages; ++i) {
            mbar_init(smem_addr(&bars[i]), 1);              // full: producer + tx bytes
            mbar_init(smem_addr(&bars[stages + i]), NQ + NB);   // empty: copy warps, builders
        }
        for (int i = 0; i < 2 * NQ; ++i) {
            mbar_init(smem_addr(&wbars[i]), 2);             // window full: copy warp + builder
            mbar_init(smem_addr(&wbars[2 * NQ + i]), 4);    // window empty: the quarter's tap warps
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
    UnitPos pos0;
    pos0.t = (int)(u_begin / a.n_src);
    pos0.s = (int)(u_begin - (int64_t)pos0.t * a.n_src);

    if (n_units > 0) {
        const int q = warp & (NQ - 1);
        const uint32_t tq = tmem_base + ((uint32_t)(32 * q) << 16);
        const int lrow = q * 32 + lane;                      // TMEM lane = tile row
        const uint32_t win_full = smem_addr(&wbars[q * 2]);           // + 8 * buffer
        const uint32_t win_empty = smem_addr(&wbars[2 * NQ + q * 2]);  // + 8 * buffer
        int st = 0;
        uint32_t ph = 0;
        UnitPos pos = pos0;
        if (warp >= NC) {
            // ---- builder of lane quarter q: the quarter's tap programs (both ears) ----
            // this lane's entry slots: i = lane + 32 m -> row i / k_max, position i % k_max
            int er[3], ep[3];
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const int i = lane + 32 * m;
                er[m] = i / a.k_max;
                ep[m] = i - er[m] * a.k_max;
            }
            // the rows of the current tile (integer divisions once per tile, not per unit)
            TileRows tr = tile_rows(a, pos.t);
            QuarterRows qr = quarter_rows(a, pos.t, q);
            int nnz_cur = load_nnz(a, qr, pos.s, lane);
            // quarter 0's builder also fills the ring, then refills the stage of unit k - 1
            // (unit k - 1 + stages) at the start of unit k, once the copy warps and builders
            // released it
            const bool producer = q == 0;
            UnitPos p_iss = pos0;
            int st_r = 0;
            uint32_t ph_r = 0;
            if (producer) {
                for (int k0 = 0; k0 < n_units && k0 < stages; ++k0) {
                    if (lane == 0) {
                        issue_unit(&tmap3, a, p_iss.t, p_iss.s, smem_addr(wins + (size_t)k0 * kWinBytes),
                                   smem_addr(tbls + (size_t)k0 * kStageTableBytes), smem_addr(&bars[k0]));
                        last_issued[k0] = k0;
                    }
                    p_iss.advance(1, a.n_src);
                }
            }
            for (int k = 0; k < n_units; ++k) {
                const uint32_t buf = (uint32_t)k & 1u;
                if (producer && k >= 1 && k - 1 + stages < n_units) {
                    if (!mbar_wait_bounded(smem_addr(&bars[stages + st_r]), ph_r, abort_flag, a.status)) break;
                    if (lane == 0) {
                        issue_unit(&tmap3, a, p_iss.t, p_iss.s, smem_addr(wins + (size_t)st_r * kWinBytes),
                                   smem_addr(tbls + (size_t)st_r * kStageTableBytes), smem_addr(&bars[st_r]));
                        last_issued[st_r] = k - 1 + stages;
                    }
                    __syncwarp();
                    p_iss.advance(1, a.n_src);
                    if (++st_r == stages) {
                        st_r = 0;
                        ph_r ^= 1u;
                    }
                }
                if (!mbar_wait_bounded(smem_addr(&bars[st]), ph, abort_flag, a.status)) break;
                if (k >= 2 && !mbar_wait_bounded(win_empty + 8 * buf, (uint32_t)((k >> 1) - 1) & 1u, abort_flag,
                                                 a.status))
                    break;
                const unsigned char *tb = tbls + (size_t)st * kStageTableBytes;
                build_progs(a, tr, qr, er, ep, reinterpret_cast<const uint16_t *>(tb),
                            reinterpret_cast<const float *>(tb + kTableIdxBytes),
                            progs + (buf * NQ + q) * 2, progs + (buf * NQ + q) * 2 + 1, lane, nnz_cur);
                if (lane == 0) {
                    mbar_arrive(win_full + 8 * buf);                   // programs ready
                    mbar_arrive(smem_addr(&bars[stages + st]));        // tables no longer read
                }
                UnitPos nx = pos;                             // the next unit's nnz, in flight
                nx.advance(1, a.n_src);
                if (k + 1 < n_units && nx.t != pos.t) {
                    tr = tile_rows(a, nx.t);
                    qr = quarter_rows(a, nx.t, q);
                }
                nnz_cur = k + 1 < n_units ? load_nnz(a, qr, nx.s, lane) : 0;
                pos = nx;
                if (++st == stages) {
                    st = 0;
                    ph ^= 1u;
                }
            }
        } else if (warp >= NTW) {
            // ---- copy warp of lane quarter q: the window into TMEM ----
            for (int k = 0; k < n_units; ++k) {
                const uint32_t buf = (uint32_t)k & 1u;
                if (!mbar_wait_bounded(smem_addr(&bars[st]), ph, abort_flag, a.status)) break;
                if (k >= 2 && !mbar_wait_bounded(win_empty + 8 * buf, (uint32_t)((k >> 1) - 1) & 1u, abort_flag,
                                                 a.status))
                    break;
                tc_fence_after();
                // window of TMEM lane lrow: tile rows rr0 .. rr0 + 7 (32 samples each),
                // rr0 = (halo + 32 lrow - SW) / 32; row r's 16-byte chunk c at c ^ (r % 8)
                const unsigned char *wb = wins + (size_t)st * kWinBytes;
                const int rr0 = (kMvHalo + R * lrow - SW) / 32;
#pragma unroll 1
                for (int b = 0; b < kCols / 32; ++b) {
                    const int rr = rr0 + b;
                    uint32_t v[32];
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const float4 x = *reinterpret_cast<const float4 *>(wb + rr * 128 + ((c ^ (rr & 7)) << 4));
                        v[4 * c + 0] = __float_as_uint(x.x);
                        v[4 * c + 1] = __float_as_uint(x.y);
                        v[4 * c + 2] = __float_as_uint(x.z);
                        v[4 * c + 3] = __float_as_uint(x.w);
                    }
                    tm_st32(tq + kCols * buf + (uint32_t)(32 * b), v);
                }
                tm_wait_st();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(win_full + 8 * buf);                   // window ready
                    mbar_arrive(smem_addr(&bars[stages + st]));        // the stage is no longer read
                }
                if (++st == stages) {
                    st = 0;
                    ph ^= 1u;
                }
            }
        } else {
            // ---- tap warp (lane quarter q, ear, half): outputs [16 half, 16 half + 16) of
            // each lane, previous and current products ----
            const int ear = (warp / NQ) & 1, half = warp / (2 * NQ);
            uint64_t accp[RP], accc[RP];
#pragma unroll
            for (int i = 0; i < RP; ++i) accp[i] = accc[i] = 0;
            // fold accumulators in shared memory, [set][RP][32] packed pairs per warp
            uint64_t *racc = reinterpret_cast<uint64_t *>(smem + a.runacc_off) + (size_t)warp * 2 * RP * 32 + lane;
#pragma unroll
            for (int i = 0; i < 2 * RP; ++i) racc[i * 32] = 0;
            int slot = a.part.slot_base(blockIdx.x, pos0.t), run_n = 0, fold_n = 0;
            // per tile: the lane's previous and current table rows relative to the quarter's
            // first, and the position of its first output in its segment
            int rp = 0, rc = 0, pos_in_seg = 0;
            auto tile_setup = [&](int t) {
                const int64_t n_lane0 = (int64_t)t * kMvTile + (int64_t)R * lrow;
                const int js = (int)(n_lane0 / a.seg_len);
                const int jlo = quarter_rows(a, t, q).jlo;
                rp = jp_of(a, js) - jlo;
                rc = jc_of(a, js) - jlo;
                pos_in_seg = (int)(n_lane0 - (int64_t)js * a.seg_len);
            };
            tile_setup(pos.t);
            for (int k = 0; k < n_units; ++k) {
                const uint32_t buf = (uint32_t)k & 1u;
                if (!mbar_wait_bounded(win_full + 8 * buf, (uint32_t)(k >> 1) & 1u, abort_flag, a.status)) break;
                tc_fence_after();
                const Prog *pg = progs + (buf * NQ + q) * 2 + ear;
                const int n = pg->n;
                const uint32_t tw = tq + kCols * buf + RS * half;
                // two register sets: the load of entry u + 1 is in flight while entry u's FMAs
                // run (columns n, n + 1 and weight rows n, n + 1 are zero padding)
                uint32_t A[RS], B[RS];
                tm_ld16(tw + (uint32_t)pg->col[0], A);
                int c_next = pg->col[1];
                float wp = pg->w[0][rp], wc = pg->w[0][rc];
                tm_wait_ld(A, accp, accc);
                int u = 0;
#pragma unroll 1
                for (; u + 1 < n; u += 2) {
                    tm_ld16(tw + (uint32_t)c_next, B);                      // entry u + 1
                    const int c2 = pg->col[u + 2];
                    const float wp1 = pg->w[u + 1][rp], wc1 = pg->w[u + 1][rc];
                    fma_slice2(accp, accc, A, wp, wc);
                    tm_wait_ld(B, accp, accc);
                    tm_ld16(tw + (uint32_t)c2, A);                          // entry u + 2
                    c_next = pg->col[u + 3];
                    wp = pg->w[u + 2][rp];
                    wc = pg->w[u + 2][rc];
                    fma_slice2(accp, accc, B, wp1, wc1);
                    tm_wait_ld(A, accp, accc);
                }
                if (u < n) {
                    fma_slice2(accp, accc, A, wp, wc);
                    tie_acc(accp, accc);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(win_empty + 8 * buf);
                // unit done: folds every a.fold sources, the run's partial slot at its end
                ++run_n;
                ++fold_n;
                const bool tile_end = (k + 1 == n_units) || (pos.s + 1 == a.n_src);
                const bool flush = run_n == a.part.gs || tile_end;
                if (flush || fold_n == a.fold) {
                    fold_n = 0;
                    uint64_t one2;
                    asm("mov.b64 %0, {%1, %1};" : "=l"(one2) : "r"(0x3f800000u));
                    if (flush) {
                        // z = (1 - a_n) P + a_n C per output; a_n from the lane's segment
                        const float inv_seg = 1.0f / (float)a.seg_len;
                        const int base = pos_in_seg + RS * half + 1;
                        float2 *p = reinterpret_cast<float2 *>(a.partial + ((size_t)pos.t * a.slots + slot) * 2 * kMvTile +
                                                               ear * kMvTile + R * lrow + RS * half);
#pragma unroll
                        for (int i = 0; i < RP; ++i) {
                            uint64_t xp = racc[i * 32], xc = racc[(RP + i) * 32];
                            asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(xp) : "l"(one2), "l"(accp[i]));
                            asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(xc) : "l"(one2), "l"(accc[i]));
                            float p0, p1, c0, c1;
                            asm("mov.b64 {%0, %1}, %2;" : "=f"(p0), "=f"(p1) : "l"(xp));
                            asm("mov.b64 {%0, %1}, %2;" : "=f"(c0), "=f"(c1) : "l"(xc));
                            const float a0 = (float)(base + 2 * i) * inv_seg, a1 = (float)(base + 2 * i + 1) * inv_seg;
                            p[i] = make_float2(fmaf(a0, c0 - p0, p0), fmaf(a1, c1 - p1, p1));
                            racc[i * 32] = 0;
                            racc[(RP + i) * 32] = 0;
                        }
                        ++slot;
                        run_n = 0;
                    } else {
#pragma unroll
                        for (int i = 0; i < RP; ++i) {
                            uint64_t xp = racc[i * 32], xc = racc[(RP + i) * 32];
                            asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(xp) : "l"(one2), "l"(accp[i]));
                            asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(xc) : "l"(one2), "l"(accc[i]));
                            racc[i * 32] = xp;
                            racc[(RP + i) * 32] = xc;
                        }
                    }
#pragma unroll
                    for (int i = 0; i < RP; ++i) accp[i] = accc[i] = 0;
                }
                pos.advance(1, a.n_src);
                if (tile_end && k + 1 < n_units) {
                    slot = a.part.slot_base(blockIdx.x, pos.t);   // the next tile's first slot
                    run_n = 0;
                    tile_setup(pos.t);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) {
        // let every copy still in flight land before the CTA exits (bounded)
        for (int s2 = 0; s2 < stages; ++s2) {
            const int j = last_issued[s2];
            if (j < 0) continue;
            const uint32_t fb = smem_addr(&bars[s2]);
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

size_t moving_tmem_smem_bytes(int stages, int k_max, int *runacc_off, int *prog_off)
{
    if (stages < 2 || stages > kMixMaxStages || k_max < 1 || k_max > kMvMaxK) return 0;
    size_t b = (size_t)stages * (kWinBytes + kStageTableBytes);
    b += (size_t)(2 * stages + 4 * NQ) * 8 + 16 + kMixMaxStages * 4;
    b = (b + 15) / 16 * 16;
    const size_t po = b;
    b += kProgsBytes;
    const size_t ro = b;
    b += kRunAccBytes;
    if (b > 227 * 1024) return 0;
    if (prog_off) *prog_off = (int)po;
    if (runacc_off) *runacc_off = (int)ro;
    return b;
}

cudaError_t launch_moving_tmem(const CUtensorMap &tmap3, const MovingTmemArgs &a, int grid, size_t smem,
                               cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(moving_tmem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    moving_tmem_kernel<<<grid, NW * 32, smem, st>>>(tmap3, a);
    return cudaGetLastError();
}

}  // namespace hrir
