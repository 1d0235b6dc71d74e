// mlp_gemm_tc.cu -- the FP32 products of the direction -> reflection-filter network
// (training: forward with kept pre-activations, backward dZ W and weight gradients dZ^T X)
// on the tensor cores, to FP32 accuracy.
//
//     C[m][n] = sum_k A(m, k) B(k, n)      (A, B FP32 in HBM, arbitrary element strides)
//
// Every FP32 operand value x is split into three BF16 terms x = x0 + x1 + x2 (x0 = bf16(x),
// x1 = bf16(x - x0), x2 = bf16(x - x0 - x1): 24 significant bits, the FP32 significand), and
// the product is accumulated in FP32 in tensor memory from the six term products whose
// orders sum to at most 2: a2 b0 + a1 b1 + a0 b2 + a1 b0 + a0 b1 + a0 b0 (the dropped ones are
// below 2^-24 relative), in three accumulators (consecutive MMAs independent) that the
// epilogue adds.  Each is one tcgen05.mma kind::f16 (M = 128, N = 64 or 32, K = 16).
//
// One CTA (8 warps) per 128 x 64 (or 128 x 32) output tile and K range (blockIdx.z: a split
// of K whose partial products a second kernel sums in a fixed order).  Per k-step of 64 the warps load
// A (128 x 64) and B (64 x 64) from global memory with the stride-1 index fastest (coalesced),
// apply ReLU where the operand is a hidden layer's pre-activation, split, and store the three
// BF16 planes of each in the canonical no-swizzle K-major layout (8-row x 16-byte core
// matrices) of one of two shared-memory stages; one thread issues the 24 MMAs of the step and
// commits them to the stage's mbarrier, and the warps load the next step's operands into
// registers while they run.  Epilogue: warp (lane quarter q, column half h) reads rows
// 32 q .. 32 q + 31 and its half of the tile's columns from the three accumulators with
// tcgen05.ld, adds them, and applies + bias (and softplus into a second output), x [mask > 0]
// (ReLU'), or writes the split's partial.  Waits are bounded.
#include <cuda_bf16.h>

#include "kernels.h"

namespace hrir {

namespace {

constexpr int kTM = 128;                 // MMA M: output rows per tile
constexpr int kKS = 64;                  // k per step (four MMA k-slices of 16)
constexpr int kThreads = 256;
constexpr int kTerms = 3;                // BF16 terms per FP32 value
constexpr int kPlaneA = kTM * kKS;       // BF16 elements of one A plane

// shared-memory layout for an output tile of TN columns (MMA N; the accumulator takes TN
// TMEM columns): two stages of the three A and three B planes, then the barriers
template <int TN>
struct TileCfg {
    static constexpr int kPlaneB = TN * kKS;
    static constexpr int kStageElems = kTerms * (kPlaneA + kPlaneB);
    static constexpr size_t kSmemBytes = 2 * (size_t)kStageElems * 2 + 64;
    static_assert(TN == 32 || TN == 64, "tile widths with a whole epilogue slice per warp");
};

enum Epi : int { EPI_BIAS = 0, EPI_BIAS_SOFTPLUS = 1, EPI_MASK = 2, EPI_PARTIAL = 3 };

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// kind::f16, D FP32, A and B BF16, both K-major
__host__ __device__ constexpr uint32_t instr_desc_bf16(uint32_t M, uint32_t N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// Element (row, k) of a [rows][kKS] plane in the canonical layout sits at
//     (row / 8) (kKS * 8) + (k / 8) 64 + (row % 8) 8 + k % 8
// (core matrix (row / 8, k / 8) of 8 rows x 8 BF16, a row group's core matrices contiguous
// along k): in bytes, 128 between core matrices adjacent in k (LBO) and kKS * 16 between row
// groups (SBO); a k-slice of 16 is 2 core matrices, 256 bytes.

__device__ __forceinline__ float softplus_f(float z) { return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))); }

// the three BF16 terms of x and y, packed in pairs (x in the low half)
__device__ __forceinline__ void split3(float x, float y, uint32_t (&p)[kTerms])
{
#pragma unroll
    for (int t = 0; t < kTerms; ++t) {
        const __nv_bfloat162 b = __floats2bfloat162_rn(x, y);
        p[t] = *reinterpret_cast<const uint32_t *>(&b);
        if (t + 1 < kTerms) {
            const float2 f = __bfloat1622float2(b);
            x = x - f.x;      // exact: the BF16 rounding of x leaves a representable rest
            y = y - f.y;
        }
    }
}

__device__ __forceinline__ void tm_ld32(uint32_t taddr, uint32_t (&r)[32])
{
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
}

__device__ __forceinline__ void tm_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// The (ROWS x kKS) block of X(row, k) = X[(r0 + row) s_row + (k0 + k) s_k] for k < ke (zero
// outside [0, n_rows) x [k0, ke)), ReLU'd when relu, as three BF16 planes at dst (plane stride
// `plane`).  Each warp fills whole core matrices: 8 rows x 4 pairs of k, lane (row, pair) =
// (lane / 4, lane % 4) when k has stride 1 and (lane % 8, lane / 8) otherwise, so that the
// global loads read whole 32-byte sectors and the 32 lanes store the 32 consecutive words of
// the core matrix (no bank conflicts).  load() fetches this thread's pairs into registers (all
// loads issued before any is used), store() splits and stores them.
template <int ROWS>
struct Operand {
    static constexpr int kCm = (ROWS / 8) * (kKS / 8);      // core matrices of the block
    static constexpr int kPer = kCm / (kThreads / 32);      // per warp: [warp kPer, warp kPer + kPer)
    static_assert(kCm % (kThreads / 32) == 0, "whole passes");
    float x[kPer], y[kPer];

    // core matrix c: row group c / 8, k columns 8 (c % 8) .. + 8
    __device__ __forceinline__ void load(const float *X, int64_t r0, int64_t n_rows, int64_t s_row, int64_t s_k,
                                         int k0, int ke, bool relu)
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const bool k_fast = s_k == 1;
        const int r_in = k_fast ? lane >> 2 : lane & 7;
        const int pr = k_fast ? lane & 3 : lane >> 3;
        const int c0 = warp * kPer;
        // every load is issued unconditionally (all of them in flight at once) from an
        // address clamped into the block's valid range; entries outside it are then zeroed
        float a[kPer], b[kPer];
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int c = c0 + i, rg = c >> 3, kc = c & 7;
            const int64_t r = r0 + rg * 8 + r_in, rc = r < n_rows ? r : n_rows - 1;
            const int k = k0 + kc * 8 + 2 * pr;
            const int ka = k < ke ? k : ke - 1, kb1 = k + 1 < ke ? k + 1 : ke - 1;
            const float *p = X + rc * s_row;
            a[i] = __ldg(p + (int64_t)ka * s_k);
            b[i] = __ldg(p + (int64_t)kb1 * s_k);
        }
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int c = c0 + i, rg = c >> 3, kc = c & 7;
            const int64_t r = r0 + rg * 8 + r_in;
            const int k = k0 + kc * 8 + 2 * pr;
            const float u = r < n_rows && k < ke ? a[i] : 0.f;
            const float v = r < n_rows && k + 1 < ke ? b[i] : 0.f;
            x[i] = relu ? fmaxf(u, 0.f) : u;
            y[i] = relu ? fmaxf(v, 0.f) : v;
        }
    }

    __device__ __forceinline__ void store(__nv_bfloat16 *dst, int plane, bool k_fast) const
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int r_in = k_fast ? lane >> 2 : lane & 7;
        const int pr = k_fast ? lane & 3 : lane >> 3;
        const int c0 = warp * kPer;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int c = c0 + i, rg = c >> 3, kc = c & 7;
            uint32_t t[kTerms];
            split3(x[i], y[i], t);
            const int o = rg * (kKS * 8) + kc * 64 + r_in * 8 + 2 * pr;     // (row, k - k0)
#pragma unroll
            for (int j = 0; j < kTerms; ++j) *reinterpret_cast<uint32_t *>(dst + (size_t)j * plane + o) = t[j];
        }
    }
};

template <int EPI, bool RELU_A, bool RELU_B, int TN>
__global__ void __launch_bounds__(kThreads, 1) gemm_tc_kernel(const GemmArgs g, int *status)
{
    using Cfg = TileCfg<TN>;
    constexpr int kStageElems = Cfg::kStageElems, kPlaneB = Cfg::kPlaneB;
    // three accumulators (term product p goes to p % 3) so that consecutive MMAs do not wait
    // for each other's result; the epilogue adds them
    constexpr int kAcc = 3;
    constexpr uint32_t kTmemCols = TN == 32 ? 128 : 256;
    static_assert(kAcc * TN <= (int)kTmemCols, "accumulators fit the allocation");
    extern __shared__ __align__(1024) unsigned char smem[];
    __nv_bfloat16 *stages = reinterpret_cast<__nv_bfloat16 *>(smem);                      // [2][kStageElems]
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * (size_t)kStageElems * 2);   // [2]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bar + 2) + 1;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t m0 = (int64_t)blockIdx.x * kTM;
    const int n0 = blockIdx.y * TN;
    const int kb = blockIdx.z * g.k_chunk;
    const int ke = min(g.K, kb + g.k_chunk);
    const int n_steps = ke > kb ? (ke - kb + kKS - 1) / kKS : 0;
    if (tid == 0) {
        mbar_init(smem_addr(&bar[0]), 1);
        mbar_init(smem_addr(&bar[1]), 1);
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
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = instr_desc_bf16(kTM, TN);

    // B(k, n) = g.B[k sbk + n sbn] is staged as the K-major plane of rows n.  The operands of
    // step s + 1 are loaded into registers while the MMAs of step s run.
    Operand<kTM> opa;
    Operand<TN> opb;
    if (n_steps > 0) {
        opa.load(g.A, m0, g.M, g.sam, g.sak, kb, ke, RELU_A);
        opb.load(g.B, n0, g.N, g.sbn, g.sbk, kb, ke, RELU_B);
    }
    int issued = 0;      // MMA steps committed
    bool ok = true;
    for (int s = 0; s < n_steps && ok; ++s) {
        const int st = s & 1;
        // the stage's previous MMAs (step s - 2) must have read it
        if (s >= 2) ok = mbar_wait_bounded(smem_addr(&bar[st]), (uint32_t)((s - 2) >> 1) & 1u, abort_flag, status);
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        __nv_bfloat16 *A = stages + (size_t)st * kStageElems, *B = A + kTerms * kPlaneA;
        opa.store(A, kPlaneA, g.sak == 1);
        opb.store(B, kPlaneB, g.sbk == 1);
        fence_proxy_async_smem();       // the generic stores before the MMAs read them
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t a_base = smem_addr(A), b_base = smem_addr(B);
            // term pairs (i, j), smallest first
            constexpr int ti[6] = {2, 1, 0, 1, 0, 0}, tj[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll 1
            for (int ks = 0; ks < kKS / 16; ++ks) {
#pragma unroll
                for (int p = 0; p < 6; ++p) {
                    const uint64_t ad = smem_desc(a_base + (uint32_t)(ti[p] * kPlaneA * 2) + ks * 256, 128, kKS * 16);
                    const uint64_t bd = smem_desc(b_base + (uint32_t)(tj[p] * kPlaneB * 2) + ks * 256, 128, kKS * 16);
                    const uint32_t acc = (s > 0 || ks > 0 || p >= kAcc) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, q;\n\t}" ::"r"(tmem + (uint32_t)((p % kAcc) * TN)),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                        : "memory");
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_addr(&bar[st]))
                : "memory");
        }
        issued = s + 1;
        if (s + 1 < n_steps) {
            const int k1 = kb + (s + 1) * kKS;
            opa.load(g.A, m0, g.M, g.sam, g.sak, k1, ke, RELU_A);
            opb.load(g.B, n0, g.N, g.sbn, g.sbk, k1, ke, RELU_B);
        }
    }
    // the last step's MMAs (and so every earlier one) complete before the epilogue
    if (ok && issued > 0) {
        const int s = issued - 1;
        ok = mbar_wait_bounded(smem_addr(&bar[s & 1]), (uint32_t)(s >> 1) & 1u, abort_flag, status);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (__syncthreads_and(ok)) {
        // warp (lane quarter q, column half h): rows 32 q + lane, columns h TN / 2 .. + TN / 2
        constexpr int kCols = TN / 2;
        const int q = warp & 3, h = warp >> 2;
        const int64_t m = m0 + q * 32 + lane;
        uint32_t v[kCols];
        if (issued > 0) {
            const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(kCols * h);
            float sum[kCols];
#pragma unroll
            for (int a = 0; a < kAcc; ++a) {
                if constexpr (kCols == 32) tm_ld32(ta + (uint32_t)(a * TN), v);
                else tm_ld16(ta + (uint32_t)(a * TN), v);
#pragma unroll
                for (int j = 0; j < kCols; ++j) sum[j] = a ? sum[j] + __uint_as_float(v[j]) : __uint_as_float(v[j]);
            }
#pragma unroll
            for (int j = 0; j < kCols; ++j) v[j] = __float_as_uint(sum[j]);
        } else {
#pragma unroll
            for (int j = 0; j < kCols; ++j) v[j] = 0u;    // empty K range: C = 0
        }
        if (m < g.M) {
#pragma unroll
            for (int j = 0; j < kCols; ++j) {
                const int n = n0 + kCols * h + j;
                if (n >= g.N) break;
                const float c = __uint_as_float(v[j]);
                if (EPI == EPI_BIAS || EPI == EPI_BIAS_SOFTPLUS) {
                    const float z = c + g.bias[n];
                    g.Z[m * g.ldz + n] = z;
                    if (EPI == EPI_BIAS_SOFTPLUS) g.H[m * g.ldh + n] = softplus_f(z);
                } else if (EPI == EPI_MASK) {
                    g.Z[m * g.ldz + n] = g.mask[m * g.ldm + n] > 0.f ? c : 0.f;
                } else {
                    g.Z[((int64_t)blockIdx.z * g.M + m) * g.ldz + n] = c;
                }
            }
        }
    } else if (issued > 0) {
        // a wait expired: let the MMAs in flight finish (bounded) before the dealloc
        const int s = issued - 1;
        const uint64_t t0 = global_timer_ns();
        while (!mbar_try_wait(smem_addr(&bar[s & 1]), (uint32_t)(s >> 1) & 1u) &&
               global_timer_ns() - t0 < kWaitLimitNs) {
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
}

template <int EPI, bool RA, bool RB, int TN>
cudaError_t gemm_tc_tn(const GemmArgs &g, int splits, int *status, cudaStream_t st)
{
    auto k = gemm_tc_kernel<EPI, RA, RB, TN>;
    const size_t smem = TileCfg<TN>::kSmemBytes;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((g.M + kTM - 1) / kTM), (unsigned)((g.N + TN - 1) / TN), (unsigned)splits);
    k<<<grid, kThreads, smem, st>>>(g, status);
    return cudaGetLastError();
}

// 64-column tiles, or 32-column tiles when 64-column ones would leave SMs idle
template <int EPI, bool RA, bool RB>
cudaError_t gemm_tc_t(const GemmArgs &g, int splits, int *status, cudaStream_t st)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        sms = 1;
    const int64_t ctas64 = ((g.M + kTM - 1) / kTM) * ((g.N + 63) / 64) * splits;
    if (ctas64 < sms) return gemm_tc_tn<EPI, RA, RB, 32>(g, splits, status, st);
    return gemm_tc_tn<EPI, RA, RB, 64>(g, splits, status, st);
}

}  // namespace

int gemm_tc_tile_rows() { return kTM; }
int gemm_tc_tile_cols() { return 64; }

cudaError_t launch_gemm_tc(int epi, bool relu_a, bool relu_b, const GemmArgs &g, int splits, int *status,
                           cudaStream_t st)
{
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    if ((g.M + kTM - 1) / kTM > 0x7fffffff || splits < 1 || splits > 65535) return cudaErrorInvalidValue;
#define HRIR_GEMM_TC_CASE(E, A, B)                                                  \
    if (epi == E && relu_a == A && relu_b == B) return gemm_tc_t<E, A, B>(g, splits, status, st);
    HRIR_GEMM_TC_CASE(EPI_BIAS, true, false)
    HRIR_GEMM_TC_CASE(EPI_BIAS_SOFTPLUS, true, false)
    HRIR_GEMM_TC_CASE(EPI_MASK, false, false)
    HRIR_GEMM_TC_CASE(EPI_PARTIAL, false, true)
    HRIR_GEMM_TC_CASE(EPI_PARTIAL, false, false)
#undef HRIR_GEMM_TC_CASE
    return cudaErrorInvalidValue;
}

}  // namespace hrir
