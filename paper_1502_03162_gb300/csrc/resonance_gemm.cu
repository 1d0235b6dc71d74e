// resonance_gemm.cu -- the resonance stage of the cascade applied per source (Eq. 2 in the
// order (y * f) * g: "y * f can be precomputed" when y is known in advance), as a
// Toeplitz-block GEMM on the tensor cores (tcgen05.mma, BF16/FP16 operands, FP32
// accumulation in tensor memory):
//
//     u_e[32 b + c] = sum_{l < 32} f_e[l] y[32 b + c - l]          (Sec. I footnote 2)
//                   = sum_{m < 64} A[b][m] T_e[m][c],
//     A[b][m] = y[32 b + m - 32]           (Hankel: block b's 64-sample window)
//     T_e[m][c] = f_e[c - m + 32] for c + 1 <= m <= c + 32, else 0  (Toeplitz of f_e)
//
// One MMA tile is 128 output blocks (4096 samples) x 64 columns (32 per ear).  The sources
// are stored in 16 bits (BF16 or FP16), so A is exact in the MMA's input type; f is split
// into three terms of that type, f = f0 + f1 + f2 (f0 = rn(f), f1 = rn(f - f0), f2 =
// rn(f - f0 - f1)), and the three Toeplitz matrices are stacked along K (K = 192, A repeated),
// so the FP32 accumulator receives y * f to about FP32 accuracy (each product of 16-bit
// operands is exact in FP32).
//
// Per CTA (persistent over (source, tile) units, several CTAs per SM): warp 0 loads the
// source window [t0 - 32, t0 + 4128) with 2-D tensor TMA (zero fill outside [0, len)); all
// threads build A in the canonical no-swizzle K-major layout (8-row x 16-byte core
// matrices); one thread issues the 12 MMAs (K = 16 each) and commits to an mbarrier; the 4
// warps read the accumulator rows (tcgen05.ld, one TMEM lane per output block) and store u
// through shared memory as coalesced warp stores.  Waits are bounded.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels.h"

namespace hrir {

namespace {

constexpr int kRows = 128;                 // output blocks per tile (MMA M)
constexpr int kBlk = 32;                   // outputs per block = resonance taps handled
constexpr int kTileOut = kRows * kBlk;     // 4096
constexpr int kKA = 64;                    // window per block (A's K)
constexpr int kTerms = 3;                  // split of f
constexpr int kK = kKA * kTerms;           // 192
constexpr int kN = 64;                     // 2 ears x 32
constexpr int kThreads = 128;
constexpr int kWin = 4352;                 // staged samples: [t0 - 256, t0 + 4096), 17 boxes
constexpr int kBox = 256;
constexpr uint32_t kTmemCols = 64;
static_assert(kResTile == kTileOut, "tile");

// ---- descriptors ---------------------------------------------------------------------------
// Shared-memory matrix descriptor (no swizzle): start address, leading-dimension byte offset
// (between core matrices adjacent in K), stride-dimension byte offset (between 8-row groups),
// version 1 at bit 46.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: D FP32, A/B BF16 (fmt 1) or FP16 (fmt 0), both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, uint32_t M, uint32_t N)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

template <typename T>
struct Fmt;
template <>
struct Fmt<__nv_bfloat16> {
    static constexpr uint32_t code = 1;
    static __device__ __forceinline__ __nv_bfloat16 rn(float x) { return __float2bfloat16_rn(x); }
    static __device__ __forceinline__ float wide(__nv_bfloat16 x) { return __bfloat162float(x); }
};
template <>
struct Fmt<__half> {
    static constexpr uint32_t code = 0;
    static __device__ __forceinline__ __half rn(float x) { return __float2half_rn(x); }
    static __device__ __forceinline__ float wide(__half x) { return __half2float(x); }
};

// canonical K-major no-swizzle offset (elements) of (row, k) in a matrix with `kc` core
// matrices along K: 8-row groups of kc x 64 elements, 8 x 8 element core matrices
__device__ __forceinline__ int core_off(int row, int k, int kc)
{
    return (row >> 3) * (kc * 64) + (k >> 3) * 64 + (row & 7) * 8 + (k & 7);
}

__device__ __forceinline__ void tm_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
        "%30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) resonance_gemm_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                  const ResonanceArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    T *Bm = reinterpret_cast<T *>(smem);                       // [64 n][192 k] canonical, 24 KB
    T *Am = Bm + kN * kK;                                      // [128 rows][64 k] canonical, 16 KB
    T *yw = Am + kRows * kKA;                                  // [kWin] staged source window
    uint64_t *bars = reinterpret_cast<uint64_t *>(yw + kWin);  // [0] TMA full, [1] MMA done
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2);
    int *abort_flag = reinterpret_cast<int *>(bars + 2) + 1;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        prefetch_tensormap(&tmap);
        mbar_init(smem_addr(&bars[0]), 1);
        mbar_init(smem_addr(&bars[1]), 1);
        *abort_flag = 0;
        mbar_fence_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // B = [T_e(f0) ; T_e(f1) ; T_e(f2)] stacked along K, one column per (ear, c)
    for (int i = tid; i < kN * kK; i += kThreads) {
        const int n = i / kK, k = i - n * kK;
        const int e = n / kBlk, c = n % kBlk;
        const int term = k / kKA, m = k % kKA;
        const int l = c - m + kBlk;
        float v = 0.f;
        if (l >= 0 && l < kBlk && l < a.res_len) {
            const float f = a.res[e * a.res_len + l];
            const float t0 = Fmt<T>::wide(Fmt<T>::rn(f));
            const float t1 = Fmt<T>::wide(Fmt<T>::rn(f - t0));
            const float t2 = f - t0 - t1;
            v = term == 0 ? t0 : term == 1 ? t1 : t2;
        }
        Bm[core_off(n, k, kK / 8)] = Fmt<T>::rn(v);
    }
    fence_proxy_async_smem();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = instr_desc(Fmt<T>::code, kRows, kN);
    const uint32_t a_base = smem_addr(Am), b_base = smem_addr(Bm);

    const int n_tiles = (int)((a.out_len + kTileOut - 1) / kTileOut);
    const int64_t units = (int64_t)n_tiles * a.n_src;
    // ---- stage y[t0 - 256, t0 + 4096) of unit u (hardware zero fill outside [0, len)); the
    // window is staged for the next unit as soon as A has been built from it, so the load
    // overlaps this unit's MMAs and epilogue ----
    auto stage = [&](int64_t u) {
        if (warp != 0) return;
        const int s = (int)(u / n_tiles);
        const int64_t t0 = (u - (int64_t)s * n_tiles) * kTileOut;
        if (lane == 0) mbar_arrive_expect_tx(smem_addr(&bars[0]), kWin * (uint32_t)sizeof(T));
        __syncwarp();
        for (int b = lane; b < kWin / kBox; b += 32)
            tma_load_2d(smem_addr(yw + b * kBox), &tmap, (int)(t0 - kBox + b * kBox), s, smem_addr(&bars[0]));
    };
    uint32_t phase = 0;
    bool in_flight = false;                 // a staged window not yet waited for
    if ((int64_t)blockIdx.x < units) {
        stage(blockIdx.x);
        in_flight = true;
    }
    for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const int s = (int)(u / n_tiles);
        const int t = (int)(u - (int64_t)s * n_tiles);
        const int64_t t0 = (int64_t)t * kTileOut;
        bool ok = mbar_wait_bounded(smem_addr(&bars[0]), phase, abort_flag, a.status);
        if (ok) in_flight = false;
        // ---- A[b][m] = y[t0 + 32 b + m - 32] = yw[256 + 32 b + m - 32] ----
        if (ok) {
            for (int i = tid; i < kRows * kKA / 8; i += kThreads) {
                const int row = i >> 3, kc = i & 7;
                const uint4 v = *reinterpret_cast<const uint4 *>(yw + kBox - kBlk + row * kBlk + kc * 8);
                *reinterpret_cast<uint4 *>(Am + core_off(row, kc * 8, kKA / 8)) = v;
            }
        }
        fence_proxy_async_smem();
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (*abort_flag) break;
        // every thread has read the window: stage the next unit's
        if (u + gridDim.x < units) {
            stage(u + gridDim.x);
            in_flight = true;
        }
        // ---- D[128][64] = sum over 12 K-steps (A's 4 steps, repeated per term) ----
        if (tid == 0) {
#pragma unroll 1
            for (int ks = 0; ks < kK / 16; ++ks) {
                const uint64_t ad = smem_desc(a_base + (ks % (kKA / 16)) * 256, 128, (kKA / 8) * 128);
                const uint64_t bd = smem_desc(b_base + ks * 256, 128, (kK / 8) * 128);
                const uint32_t acc = ks > 0 ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_addr(&bars[1]))
                : "memory");
        }
        ok = mbar_wait_bounded(smem_addr(&bars[1]), phase, abort_flag, a.status);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        phase ^= 1;                          // both barriers complete once per unit
        // ---- epilogue: TMEM lane = output block, 32 columns per ear.  A warp's 32 blocks
        // are 1024 consecutive outputs, so each ear goes through the (now free) A tile in shared
        // memory -- row = block, 16-byte chunk j of row L stored at chunk j ^ (L & 7), so that
        // both the row writes and the contiguous reads are conflict-free -- and leaves as
        // 512-byte coalesced warp stores. ----
        if (ok) {
            float *stg = reinterpret_cast<float *>(Am) + warp * 32 * kBlk;   // 4 KB per warp
            const int64_t n_w = t0 + (int64_t)warp * 32 * kBlk;             // warp's first output
#pragma unroll 1
            for (int e = 0; e < 2; ++e) {
                float v[32];
                tm_ld32(tmem + ((uint32_t)(warp * 32) << 16) + e * kBlk, v);
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    reinterpret_cast<float4 *>(stg + lane * kBlk)[j ^ (lane & 7)] =
                        make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                __syncwarp();
                float *o = a.out + ((int64_t)s * 2 + e) * a.out_ld + n_w;
#pragma unroll
                for (int it = 0; it < 8; ++it) {
                    const int q = it * 32 + lane;                 // float4 chunk of the 1024
                    const int row = q >> 3, j = q & 7;
                    const float4 x = reinterpret_cast<const float4 *>(stg + row * kBlk)[j ^ (row & 7)];
                    const int64_t n = n_w + 4 * q;
                    if (n + 4 <= a.out_len) {
                        *reinterpret_cast<float4 *>(o + 4 * q) = x;
                    } else {
                        if (n < a.out_len) o[4 * q] = x.x;
                        if (n + 1 < a.out_len) o[4 * q + 1] = x.y;
                        if (n + 2 < a.out_len) o[4 * q + 2] = x.z;
                    }
                }
                __syncwarp();
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();   // A, the window and D are reused by the next unit
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!ok) break;
    }
    if (warp == 0) {
        // a staged load still in flight after an abort lands before the CTA exits (bounded):
        // its phase is the one after the last completed window
        const uint64_t t0 = global_timer_ns();
        while (in_flight && !mbar_try_wait(smem_addr(&bars[0]), phase) && global_timer_ns() - t0 < kWaitLimitNs) {
        }
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
}

}  // namespace

size_t resonance_gemm_smem_bytes(int elem_bytes)
{
    return (size_t)(kN * kK + kRows * kKA + kWin) * elem_bytes + 2 * 8 + 16;
}

cudaError_t launch_resonance_gemm(int dtype, const CUtensorMap &tmap, const ResonanceArgs &a, int grid,
                                  cudaStream_t st)
{
    const size_t smem = resonance_gemm_smem_bytes(2);
    if (dtype == 1) {
        auto k = resonance_gemm_kernel<__nv_bfloat16>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<grid, kThreads, smem, st>>>(tmap, a);
    } else if (dtype == 2) {
        auto k = resonance_gemm_kernel<__half>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<grid, kThreads, smem, st>>>(tmap, a);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace hrir
