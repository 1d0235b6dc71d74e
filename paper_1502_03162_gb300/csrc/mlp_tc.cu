// mlp_tc.cu -- bulk inference of the direction -> reflection-filter network on the tensor
// cores (BF16 operands, FP32 accumulation in tensor memory), for the millions of
// (source, segment, ear) rows of moving sources.
//
// One kernel per layer l = 2, 3, 4:  Z[r][n] = sum_k H[r][k] W_l[n][k] + b_l[n] (K = 256),
// H = relu(z_{l-1}).  Each CTA (8 warps, persistent over 128-row tiles) keeps W_l in shared
// memory in the canonical no-swizzle K-major layout (8-row x 16-byte core matrices).  Per tile
// it builds the A operand (for layer 2 straight from the features: z1 = W1 x + b1, ReLU, so
// layer 1 is fused on the CUDA cores; for layers 3 and 4 from the previous layer's rows, which
// were loaded into registers during the previous tile), one thread issues 16 tcgen05.mma
// (K = 16 each, M = 128, N = 256 or Lg rounded up to 16) into one of two TMEM accumulators and
// commits to an mbarrier, and while those MMAs run the 8 warps apply the epilogue of the
// previous tile from the other accumulator: warp (lane quarter q, column half) reads its 32
// rows with tcgen05.ld and applies bias + ReLU (hidden layers, stored as BF16 for the next
// layer) or bias + softplus (output layer, stored as FP32).  Waits are bounded.
#include <cuda_bf16.h>

#include "kernels.h"

namespace hrir {

namespace {

constexpr int kRows = 128;                  // MMA M: rows per tile
constexpr int kK = kMlpHidden;              // 256
constexpr int kKc = kK / 8;                 // core matrices along K
constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr uint32_t kTmemCols = 512;         // two accumulators of 256 columns

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

__device__ __forceinline__ int core_off(int row, int k) { return (row >> 3) * (kKc * 64) + (k >> 3) * 64 + (row & 7) * 8 + (k & 7); }

// two floats -> BF16 pair (round to nearest), the first in the low half
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&p);
}

// softplus(z) = max(z, 0) + log(1 + e^-|z|) with the hardware exp2/log2 approximations: an
// absolute error of a few 1e-7, far below the BF16 rounding of the operands
__device__ __forceinline__ float softplus_f(float z) { return fmaxf(z, 0.f) + __logf(1.f + __expf(-fabsf(z))); }

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

__global__ void __launch_bounds__(kThreads, 1) mlp_layer_tc_kernel(const MlpTcArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __nv_bfloat16 *Wm = reinterpret_cast<__nv_bfloat16 *>(smem);        // [n_pad][256] canonical
    __nv_bfloat16 *Am = Wm + (size_t)a.n_pad * kK;                       // [128][256] canonical
    uint64_t *bar = reinterpret_cast<uint64_t *>(Am + kRows * kK);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 1);
    int *abort_flag = reinterpret_cast<int *>(bar + 1) + 1;
    float *bias = reinterpret_cast<float *>(bar + 2);                    // [256] this layer's biases
    float *w1 = bias + kK;                                               // layer 2: W1 [256][5], b1 [256]
    float *stage_out = w1 + kMlpHidden * (kMlpIn + 1);                   // output layer: [8 warps][32][32]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        mbar_init(smem_addr(bar), 1);
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
    // this layer's weights (rows n >= N are zero) as BF16, canonical layout
    for (int i = tid; i < a.n_pad * kK / 4; i += kThreads) {
        const int n = (4 * i) / kK, k = 4 * i - n * kK;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n < a.N) v = __ldg(reinterpret_cast<const float4 *>(a.W + (size_t)n * kK + k));
        *reinterpret_cast<uint2 *>(Wm + core_off(n, k)) = make_uint2(pack_bf16(v.x, v.y), pack_bf16(v.z, v.w));
    }
    for (int i = tid; i < kK; i += kThreads) bias[i] = i < a.N ? a.b[i] : 0.f;
    if (a.first)
        for (int i = tid; i < kMlpHidden * (kMlpIn + 1); i += kThreads)
            w1[i] = i < kMlpHidden * kMlpIn ? a.W1[i] : a.b1[i - kMlpHidden * kMlpIn];
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = instr_desc_bf16(kRows, (uint32_t)a.n_pad);
    const uint32_t a_base = smem_addr(Am), w_base = smem_addr(Wm);
    const int64_t n_tiles = (a.n_rows + kRows - 1) / kRows;

    // ---- A operand of tile t ----
    // layers after the first: the hidden activations are kept in HBM tile by tile in the
    // operand's own canonical layout (128 rows x 256 columns of BF16 = 64 KB a tile, element
    // (row, k) at core_off(row, k)), so tile t is one contiguous block: step j moves 16-byte
    // chunk j kThreads + tid of it (coalesced loads, conflict-free stores).  Loaded into
    // registers two tiles ahead (pre: the next tile, pre2: the one after), so that two tiles
    // are in flight per SM.  The first layer: the direction row of the next tile (dpre).
    constexpr int kTileChunks = kRows * kK / 8;
    static_assert(kTileChunks % kThreads == 0, "whole steps");
    constexpr int kSteps = kTileChunks / kThreads;
    uint4 pre[kSteps], pre2[kSteps];
    float dpre[3] = {0.f, 0.f, 0.f};
    auto load_a = [&](int64_t t, uint4 (&dst)[kSteps]) {
        const uint4 *blk = reinterpret_cast<const uint4 *>(a.in) + t * kTileChunks;
#pragma unroll
        for (int j = 0; j < kSteps; ++j)
            dst[j] = t < n_tiles ? __ldg(blk + j * kThreads + tid) : make_uint4(0, 0, 0, 0);
    };
    auto load_dirs = [&](int64_t t) {
        const int64_t r = t * kRows + (tid & (kRows - 1));
        if (t < n_tiles && r < a.n_rows) {
#pragma unroll
            for (int i = 0; i < 3; ++i) dpre[i] = __ldg(a.dirs + r * 3 + i);
        }
    };
    // the next tile's registers move up: pre <- pre2, and pre2 starts loading tile t
    auto advance = [&](int64_t t) {
        if (a.first) {
            load_dirs(t);
            return;
        }
#pragma unroll
        for (int j = 0; j < kSteps; ++j) pre[j] = pre2[j];
        load_a(t, pre2);
    };
    // the first layer: row tid % 128, hidden units [128 h, 128 h + 128) with h = tid / 128:
    // features, then relu(W1 x + b1)
    auto build_a = [&](int64_t t) {
        if (!a.first) {
#pragma unroll
            for (int j = 0; j < kSteps; ++j) reinterpret_cast<uint4 *>(Am)[j * kThreads + tid] = pre[j];
            return;
        }
        const int row = tid & (kRows - 1), h = tid / kRows;
        const int64_t r = t * kRows + row;
        float sa = 0.f, ca = 0.f, se = 0.f, ce = 0.f, ear = 0.f;
        if (r < a.n_rows) {
            __sincosf(dpre[0], &sa, &ca);  // hardware approximations: the features go
            __sincosf(dpre[1], &se, &ce);  // into BF16 products
            ear = dpre[2];
        }
        const float x[kMlpIn] = {sa, ca, se, ce, ear};
        for (int kc = h * kKc / 2; kc < (h + 1) * kKc / 2; ++kc) {
            uint32_t hv[4];
#pragma unroll
            for (int j = 0; j < 8; j += 2) {
                float z2[2];
#pragma unroll
                for (int jj = 0; jj < 2; ++jj) {
                    const int n = kc * 8 + j + jj;
                    float z = w1[kMlpHidden * kMlpIn + n];
#pragma unroll
                    for (int q = 0; q < kMlpIn; ++q) z = fmaf(w1[n * kMlpIn + q], x[q], z);
                    z2[jj] = r < a.n_rows ? fmaxf(z, 0.f) : 0.f;
                }
                hv[j / 2] = pack_bf16(z2[0], z2[1]);
            }
            *reinterpret_cast<uint4 *>(Am + core_off(row, kc * 8)) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
        }
    };
    // one thread issues the MMAs of the tile in A into accumulator buffer b, then commits
    auto issue_mma = [&](uint32_t b) {
        fence_proxy_async_smem();     // A's generic stores before the MMAs read it
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
#pragma unroll 1
            for (int ks = 0; ks < kK / 16; ++ks) {
                const uint64_t ad = smem_desc(a_base + ks * 256, 128, kKc * 128);
                const uint64_t bd = smem_desc(w_base + ks * 256, 128, kKc * 128);
                const uint32_t acc = ks > 0 ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem + b * 256u),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_addr(bar))
                : "memory");
        }
    };
    // epilogue of tile t from accumulator buffer b: warp (lane quarter warp % 4) takes the
    // 32-column chunks c of parity warp / 4
    // output layer with rows of 16-byte groups at a 16-byte aligned base and room for the
    // staging tiles (set by the launcher): staged, coalesced stores
    const bool vec_out = a.stage_out != 0;
    auto epilogue = [&](int64_t t, uint32_t b) {
        const int q = warp & 3, half = warp >> 2;
        const int row = q * 32 + lane;
        const int64_t r = t * kRows + row;
        for (int c0 = 32 * half; c0 < a.n_pad; c0 += 64) {
            uint32_t v[32];
            tm_ld32(tmem + b * 256u + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, v);
            if (a.last && vec_out) {
                // the warp's 32 rows x 32 columns through shared memory (16-byte chunk j of row
                // L at chunk j ^ (L % 8): conflict-free both ways), then 4 whole 128-byte rows
                // per store instruction
                float *stg = stage_out + warp * 32 * 32;
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    reinterpret_cast<float4 *>(stg + lane * 32)[j ^ (lane & 7)] = make_float4(
                        softplus_f(__uint_as_float(v[4 * j]) + bias[c0 + 4 * j]),
                        softplus_f(__uint_as_float(v[4 * j + 1]) + bias[c0 + 4 * j + 1]),
                        softplus_f(__uint_as_float(v[4 * j + 2]) + bias[c0 + 4 * j + 2]),
                        softplus_f(__uint_as_float(v[4 * j + 3]) + bias[c0 + 4 * j + 3]));
                __syncwarp();
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int rr = 4 * i + (lane >> 3), c = lane & 7;
                    const float4 x = reinterpret_cast<const float4 *>(stg + rr * 32)[c ^ (rr & 7)];
                    const int64_t ro = t * kRows + q * 32 + rr;
                    if (ro < a.n_rows && c0 + 4 * c < a.N)
                        *reinterpret_cast<float4 *>(a.out + ro * a.N + c0 + 4 * c) = x;
                }
                __syncwarp();
                continue;
            }
            if (r >= a.n_rows) continue;
            if (a.last) {
                float *o = a.out + r * a.N;
                if ((a.N & 3) == 0 && ((uintptr_t)a.out & 15) == 0) {   // 16-byte aligned rows: vector stores
#pragma unroll
                    for (int j = 0; j < 32; j += 4)
                        if (c0 + j < a.N)
                            *reinterpret_cast<float4 *>(o + c0 + j) = make_float4(
                                softplus_f(__uint_as_float(v[j]) + bias[c0 + j]),
                                softplus_f(__uint_as_float(v[j + 1]) + bias[c0 + j + 1]),
                                softplus_f(__uint_as_float(v[j + 2]) + bias[c0 + j + 2]),
                                softplus_f(__uint_as_float(v[j + 3]) + bias[c0 + j + 3]));
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (c0 + j < a.N) o[c0 + j] = softplus_f(__uint_as_float(v[j]) + bias[c0 + j]);
                }
            } else {
                uint32_t hv[16];
#pragma unroll
                for (int j = 0; j < 32; j += 2)
                    hv[j / 2] = pack_bf16(fmaxf(__uint_as_float(v[j]) + bias[c0 + j], 0.f),
                                          fmaxf(__uint_as_float(v[j + 1]) + bias[c0 + j + 1], 0.f));
                // the tile's block in the canonical layout: a warp's 32 rows x 16 bytes are four
                // whole 128-byte core matrices
                __nv_bfloat16 *blk = a.hout + t * (int64_t)(kRows * kK);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    *reinterpret_cast<uint4 *>(blk + core_off(row, c0 + 8 * j)) =
                        make_uint4(hv[4 * j], hv[4 * j + 1], hv[4 * j + 2], hv[4 * j + 3]);
            }
        }
    };

    // pipeline: the MMAs of tile t + 1 run while the epilogue of tile t reads the other
    // accumulator
    int64_t t = blockIdx.x;
    uint32_t phase = 0, b = 0;
    if (t < n_tiles) {
        if (a.first) {
            load_dirs(t);
        } else {
            load_a(t, pre);
            load_a(t + gridDim.x, pre2);
        }
        build_a(t);
        issue_mma(0);
        advance(t + (a.first ? 1 : 2) * (int64_t)gridDim.x);
    }
    for (; t < n_tiles; t += gridDim.x) {
        const bool ok = mbar_wait_bounded(smem_addr(bar), phase, abort_flag, a.status);   // MMAs of t
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        phase ^= 1;
        if (!ok) break;
        const int64_t tn = t + gridDim.x;
        if (tn < n_tiles) {
            build_a(tn);                            // A is free: the MMAs of t completed
            issue_mma(b ^ 1u);
            advance(tn + (a.first ? 1 : 2) * (int64_t)gridDim.x);   // in flight during the epilogue
        }
        epilogue(t, b);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();                            // buffer b is read before the MMAs of t + 2
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        b ^= 1u;
    }
    // MMAs still in flight after an expired wait: let them finish (bounded) before the dealloc
    if (t < n_tiles) {
        const uint64_t t0 = global_timer_ns();
        while (!mbar_try_wait(smem_addr(bar), phase ^ 1u) && global_timer_ns() - t0 < kWaitLimitNs) {
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
}

}  // namespace

size_t mlp_tc_smem_bytes(int n_pad, int stage_out)
{
    return (size_t)(n_pad + kRows) * kK * 2 + 16 + (size_t)kK * 4 + (size_t)kMlpHidden * (kMlpIn + 1) * 4 +
           (stage_out ? (size_t)kWarps * 32 * 32 * 4 : 0);
}

cudaError_t launch_mlp_layer_tc(const MlpTcArgs &a, int grid, cudaStream_t st)
{
    if (a.n_pad < 16 || a.n_pad > 256 || a.n_pad % 16 || a.N > a.n_pad) return cudaErrorInvalidValue;
    MlpTcArgs b = a;
    b.stage_out = a.last && (a.N & 3) == 0 && ((uintptr_t)a.out & 15) == 0 &&
                  mlp_tc_smem_bytes(a.n_pad, 1) <= 227 * 1024;
    const size_t smem = mlp_tc_smem_bytes(a.n_pad, b.stage_out);
    cudaError_t e = cudaFuncSetAttribute(mlp_layer_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    mlp_layer_tc_kernel<<<grid, kThreads, smem, st>>>(b);
    return cudaGetLastError();
}

}  // namespace hrir
