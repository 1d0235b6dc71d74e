// common.cuh -- shared device helpers of the sm_103a renderer (PTX wrappers for mbarrier,
// bulk TMA copies and timers, device status codes, the work-partition arithmetic shared by
// the mixing kernels and the reduction kernel).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hrir {

// ---- device-side status bits (OR-ed into the context's status word) -------------------
enum : int {
    DEV_BAD_DIR = 1,    // a direction id was out of range (source rendered as silence)
    DEV_TIMEOUT = 2,    // a bounded mbarrier wait expired; the kernel returned early
    DEV_BAD_TAP = 4,    // a device tap table held an index >= Lg or a count > k_max (ignored)
    DEV_SOLVER = 8,     // an L1-NNLS row hit the solver's limits, or a resonance system was not SPD
    DEV_LAYOUT = 16,    // a kernel found its shared memory misaligned for its TMA layout (did nothing)
};

// Bounded waits give up after this many nanoseconds of %globaltimer.
constexpr uint64_t kWaitLimitNs = 1000ull * 1000ull * 1000ull;  // 1 s

// ---- PTX wrappers ---------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Non-blocking test of phase `parity` (try_wait may suspend the thread for a while; this
// never does).
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the mbarrier at `bar`.  Gives up (returns false) when another
// thread of the CTA raised *abort, or after kWaitLimitNs, in which case it raises *abort
// and ORs DEV_TIMEOUT into *status.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  volatile int *abort, int *status)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort) return false;
        if (global_timer_ns() - t0 > kWaitLimitNs) {
            *abort = 1;
            atomicOr(status, DEV_TIMEOUT);
            return false;
        }
    }
}

// Order this thread's earlier generic-proxy shared-memory accesses before later
// async-proxy (TMA) accesses to the same locations.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 1-D bulk TMA copy global -> shared, completion counted on mbarrier `bar` (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void tma_load_1d(uint32_t dst, const void *src, uint32_t bytes,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// 2-D tiled TMA load of one box at element coordinates (x, y) of the tensor map; elements
// outside the tensor are zero-filled by the hardware.  x * elem_size must be a multiple of 16.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void *tmap, int x, int y,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(tmap), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// 3-D tiled TMA load of one box at element coordinates (x, y, z).
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void *tmap, int x, int y, int z,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const void *tmap)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(tmap) : "memory");
}

// ---- balanced contiguous work partition -------------------------------------------------
// The mixing kernels see the work as U = n_tiles * n_src "units" (one source over one
// output tile), ordered tile-major.  CTA b of P processes units [first(b), first(b+1)),
// first(b) = floor(b U / P), so every CTA gets U/P units to within one.  Within a tile
// the units of one CTA are accumulated in registers in runs of at most `gs` sources
// (bounding FP32 accumulation error), and each run is written to its own partial slot.
// Slots of a tile are numbered in increasing source order, so the reduction kernel sums
// them in a fixed order.
struct Partition {
    int64_t U;     // total units
    int64_t P;     // CTAs (1 <= P <= U)
    int n_src;
    int gs;        // max sources per accumulation run

    __host__ __device__ int64_t first(int64_t b) const { return b * U / P; }
    // CTA that owns unit u: the largest b with first(b) <= u
    __host__ __device__ int64_t owner(int64_t u) const { return ((u + 1) * P - 1) / U; }
    // number of runs CTA b contributes to tile t
    __host__ __device__ int runs(int64_t b, int t) const
    {
        const int64_t ts = (int64_t)t * n_src, te = ts + n_src;
        int64_t lo = first(b), hi = first(b + 1);
        lo = lo > ts ? lo : ts;
        hi = hi < te ? hi : te;
        if (hi <= lo) return 0;
        return (int)((hi - lo + gs - 1) / gs);
    }
    // slot index of the first run of CTA b in tile t
    __host__ __device__ int slot_base(int64_t b, int t) const
    {
        const int64_t b_lo = owner((int64_t)t * n_src);
        int s = 0;
        for (int64_t c = b_lo; c < b; ++c) s += runs(c, t);
        return s;
    }
    // number of slots (runs) in tile t
    __host__ __device__ int slots(int t) const
    {
        const int64_t b_lo = owner((int64_t)t * n_src);
        const int64_t b_hi = owner((int64_t)t * n_src + n_src - 1);
        int s = 0;
        for (int64_t c = b_lo; c <= b_hi; ++c) s += runs(c, t);
        return s;
    }
};

}  // namespace hrir
