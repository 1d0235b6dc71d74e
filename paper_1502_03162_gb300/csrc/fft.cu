// fft.cu -- overlap-save FFT convolution with frequency-domain mixing (plain method 2;
// FFT convolution as in Sec. I footnote 3, partitioned as overlap-save per Sec. IV-G).
//
// Frame j covers outputs [jB, jB + B) and reads the P input samples starting at jB - G,
// G = H - 1 rounded up to 8 (so the TMA start stays 16-byte aligned), B = P - G.  In the
// circular convolution of a frame with an H-tap HRIR, positions >= H - 1 are the linear
// convolution, so output jB + t is frame position G + t.
//
//  * build_spectra_kernel: X_{d,e}[k] = DFT_P(x_{d,e}) for k = 0..P/2 from the dense HRIRs.
//  * fft_mix_kernel: one P-point complex FFT per pair of sources (z = y_a + i y_b), split
//    into the two real spectra, multiplied by each source's HRIR spectra and accumulated per
//    ear in registers (the mix happens in the frequency domain); runs of <= 32 pairs are
//    flushed to partial spectra, like the direct kernels.
//  * fft_out_kernel: per frame, fixed-order compensated sum of the partial spectra, one
//    complex inverse FFT carrying both ears (z = X_L + i X_R), output positions G .. P-1.
// The FFT is a radix-8 Stockham (autosort) transform of P = 4096 points by 512 threads,
// four passes through a padded shared-memory buffer, twiddles from a table.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "kernels.h"

namespace hrir {

namespace {

constexpr int kN = kFftSize;          // 4096
constexpr int kT = kN / 8;            // 512 threads
constexpr int kBins = kN / 2 + 1;     // 2049

__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }
constexpr int kPadded = kN + (kN >> 4);

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by -i
__device__ __forceinline__ float2 mul_mi(float2 a) { return make_float2(a.y, -a.x); }

// In-register forward 8-point DFT (exp(-2 pi i nk / 8)), decimation in frequency; the
// result is returned in natural order.
__device__ __forceinline__ void dft8(float2 (&u)[8])
{
    const float s = 0.70710678118654752f;  // 1/sqrt(2)
    float2 a0 = cadd(u[0], u[4]), a4 = csub(u[0], u[4]);
    float2 a1 = cadd(u[1], u[5]), a5 = csub(u[1], u[5]);
    float2 a2 = cadd(u[2], u[6]), a6 = csub(u[2], u[6]);
    float2 a3 = cadd(u[3], u[7]), a7 = csub(u[3], u[7]);
    a5 = make_float2(s * (a5.x + a5.y), s * (a5.y - a5.x));    // * exp(-i pi/4)
    a6 = mul_mi(a6);                                          // * exp(-i pi/2)
    a7 = make_float2(s * (a7.y - a7.x), -s * (a7.x + a7.y));   // * exp(-3 i pi/4)
    const float2 b0 = cadd(a0, a2), b2 = csub(a0, a2);
    const float2 b1 = cadd(a1, a3), b3 = mul_mi(csub(a1, a3));
    const float2 b4 = cadd(a4, a6), b6 = csub(a4, a6);
    const float2 b5 = cadd(a5, a7), b7 = mul_mi(csub(a5, a7));
    u[0] = cadd(b0, b1);
    u[4] = csub(b0, b1);
    u[2] = cadd(b2, b3);
    u[6] = csub(b2, b3);
    u[1] = cadd(b4, b5);
    u[5] = csub(b4, b5);
    u[3] = cadd(b6, b7);
    u[7] = csub(b6, b7);
}

// Forward FFT of kN points.  On entry u[r] holds input element tid + r*kT; on return buf
// (padded indexing) holds the transform in natural order.  All kT threads must call it.
__device__ __forceinline__ void fft_forward(float2 (&u)[8], float2 *buf, const float2 *__restrict__ tw)
{
    const int i = threadIdx.x;
    // pass p = 1: no twiddles
    dft8(u);
#pragma unroll
    for (int r = 0; r < 8; ++r) buf[pad(i * 8 + r)] = u[r];
    __syncthreads();
#pragma unroll
    for (int p = 8; p < kN; p *= 8) {
        const int k = i & (p - 1);
#pragma unroll
        for (int r = 0; r < 8; ++r) u[r] = buf[pad(i + r * kT)];
        const int step = k * (kN / (8 * p));
#pragma unroll
        for (int r = 1; r < 8; ++r) u[r] = cmul(u[r], __ldg(tw + r * step));
        dft8(u);
        __syncthreads();
        const int j = (i - k) * 8 + k;
#pragma unroll
        for (int r = 0; r < 8; ++r) buf[pad(j + r * p)] = u[r];
        __syncthreads();
    }
}

// Split Z = FFT(a + i b) into the spectra of the real sequences a and b at bin k.
__device__ __forceinline__ void split_real_pair(float2 zk, float2 zm, float2 &ya, float2 &yb)
{
    ya = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    yb = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
}

// ---- HRIR spectra ------------------------------------------------------------------------
__global__ void __launch_bounds__(kT) build_spectra_kernel(const float *__restrict__ dense,
                                                           int padded_len, int hrir_len,
                                                           const float2 *__restrict__ tw,
                                                           float2 *__restrict__ spec)
{
    __shared__ float2 buf[kPadded];
    const int d = blockIdx.x;
    const float *hl = dense + (size_t)d * 2 * padded_len;
    const float *hr = hl + padded_len;
    float2 u[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int n = threadIdx.x + r * kT;
        u[r] = n < hrir_len ? make_float2(hl[n], hr[n]) : make_float2(0.f, 0.f);
    }
    fft_forward(u, buf, tw);
    float2 *sl = spec + (size_t)d * 2 * kFftBinsPadded;
    float2 *sr = sl + kFftBinsPadded;
    for (int k = threadIdx.x; k < kBins; k += kT) {
        float2 a, b;
        split_real_pair(buf[pad(k)], buf[pad((kN - k) & (kN - 1))], a, b);
        sl[k] = a;
        sr[k] = b;
    }
}

template <typename T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }

// ---- forward FFT + frequency-domain mix ------------------------------------------------------
// Shared memory: two TMA stages of [kN/256 boxes][2 rows][256] source samples, the padded
// FFT buffer, two mbarriers.
template <typename T>
__global__ void __launch_bounds__(kT, kFftCtasPerSm)
    fft_mix_kernel(const __grid_constant__ CUtensorMap tmap, const FftArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    T *stage = reinterpret_cast<T *>(smem);                                  // [2][2*kN]
    float2 *buf = reinterpret_cast<float2 *>(smem + 2 * 2 * kN * sizeof(T));  // [kPadded]
    uint64_t *bars = reinterpret_cast<uint64_t *>(buf + kPadded);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bars + 2);
    const int tid = threadIdx.x;
    if (tid == 0) {
        prefetch_tensormap(&tmap);
        mbar_init(smem_addr(&bars[0]), 1);
        mbar_init(smem_addr(&bars[1]), 1);
        *abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();
    const int64_t u_begin = a.part.first(blockIdx.x), u_end = a.part.first(blockIdx.x + 1);
    const int n_pairs = a.part.n_src;

    auto issue = [&](int64_t u, int st) {
        const int j = (int)(u / n_pairs);
        const int p = (int)(u - (int64_t)j * n_pairs);
        const int x0 = j * a.hop - a.guard;
        const uint32_t bar = smem_addr(&bars[st]);
        mbar_arrive_expect_tx(bar, (uint32_t)(2 * kN * sizeof(T)));
        for (int b = 0; b < kN / 256; ++b)
            tma_load_2d(smem_addr(stage + (size_t)st * 2 * kN + b * 512), &tmap, x0 + b * 256, 2 * p, bar);
    };
    if (tid == 0 && u_begin < u_end) issue(u_begin, 0);

    float2 accL[4], accR[4], accL5 = make_float2(0.f, 0.f), accR5 = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) accL[q] = accR[q] = make_float2(0.f, 0.f);
    int cur_f = -1, slot = 0, run_n = 0;
    for (int64_t u = u_begin, k = 0; u < u_end; ++u, ++k) {
        const int st = (int)(k & 1);
        if (tid == 0 && u + 1 < u_end) issue(u + 1, st ^ 1);
        const int f = (int)(u / n_pairs);
        const int p = (int)(u - (int64_t)f * n_pairs);
        if (f != cur_f) {
            cur_f = f;
            slot = a.part.slot_base(blockIdx.x, f);
            run_n = 0;
        }
        const bool ok =
            mbar_wait_bounded(smem_addr(&bars[st]), (uint32_t)((k >> 1) & 1), abort_flag, a.status);
        if (__syncthreads_or(!ok)) {  // every thread leaves together: no one is left at a barrier
            if (tid == 0) {
                // let the copies still in flight (this unit's and the prefetched one) land
                for (int64_t kk = k; kk <= k + 1 && u_begin + kk < u_end; ++kk) {
                    const uint32_t fb = smem_addr(&bars[kk & 1]);
                    const uint64_t t0 = global_timer_ns();
                    while (!mbar_try_wait(fb, (uint32_t)((kk >> 1) & 1)) &&
                           global_timer_ns() - t0 < kWaitLimitNs) {
                    }
                }
            }
            break;
        }
        const T *sa = stage + (size_t)st * 2 * kN;
        float2 v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int n = tid + r * kT;
            const int base = (n >> 8) * 512 + (n & 255);
            v[r] = make_float2(to_f<T>(sa[base]), to_f<T>(sa[base + 256]));
        }
        fft_forward(v, buf, a.tw);
        // directions of the pair (the silent record beyond the last source or out of range)
        const int s0 = 2 * p, s1 = 2 * p + 1;
        int d0 = __ldg(a.dir + s0);
        int d1 = a.n_dirs;  // a missing second source renders as silence
        if ((unsigned)d0 >= (unsigned)a.n_dirs) {
            if (tid == 0) atomicOr(a.status, DEV_BAD_DIR);
            d0 = a.n_dirs;
        }
        if (s1 < a.n_src) {
            d1 = __ldg(a.dir + s1);
            if ((unsigned)d1 >= (unsigned)a.n_dirs) {
                if (tid == 0) atomicOr(a.status, DEV_BAD_DIR);
                d1 = a.n_dirs;
            }
        }
        const float2 *h0 = a.spec + (size_t)d0 * 2 * kFftBinsPadded;
        const float2 *h1 = a.spec + (size_t)d1 * 2 * kFftBinsPadded;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int kb = tid + q * kT;
            float2 y0, y1;
            split_real_pair(buf[pad(kb)], buf[pad((kN - kb) & (kN - 1))], y0, y1);
            accL[q] = cadd(accL[q], cadd(cmul(y0, __ldg(h0 + kb)), cmul(y1, __ldg(h1 + kb))));
            accR[q] = cadd(accR[q], cadd(cmul(y0, __ldg(h0 + kFftBinsPadded + kb)),
                                         cmul(y1, __ldg(h1 + kFftBinsPadded + kb))));
        }
        if (tid == 0) {
            const int kb = kN / 2;
            float2 y0, y1;
            split_real_pair(buf[pad(kb)], buf[pad(kb)], y0, y1);
            accL5 = cadd(accL5, cadd(cmul(y0, __ldg(h0 + kb)), cmul(y1, __ldg(h1 + kb))));
            accR5 = cadd(accR5, cadd(cmul(y0, __ldg(h0 + kFftBinsPadded + kb)),
                                     cmul(y1, __ldg(h1 + kFftBinsPadded + kb))));
        }
        __syncthreads();  // buf is rewritten by the next unit
        ++run_n;
        const bool frame_end = (u + 1 == u_end) || ((u + 1) / n_pairs != f);
        if (run_n == a.part.gs || frame_end) {
            float2 *ps = a.partial + ((size_t)f * a.slots + slot) * 2 * kFftBinsPadded;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ps[tid + q * kT] = accL[q];
                ps[kFftBinsPadded + tid + q * kT] = accR[q];
                accL[q] = accR[q] = make_float2(0.f, 0.f);
            }
            if (tid == 0) {
                ps[kN / 2] = accL5;
                ps[kFftBinsPadded + kN / 2] = accR5;
                accL5 = accR5 = make_float2(0.f, 0.f);
            }
            ++slot;
            run_n = 0;
        }
    }
}

// ---- reduction of partial spectra + inverse FFT per frame -------------------------------
__global__ void __launch_bounds__(kT) fft_out_kernel(const FftOutArgs a)
{
    __shared__ float2 buf[kPadded];
    const int f = blockIdx.x;
    const int ns = a.part.slots(f);
    const float2 *base = a.partial + (size_t)f * a.slots * 2 * kFftBinsPadded;
    // z = conj(Z), Z = X_L + i X_R over all kN bins (Hermitian halves), so that the forward
    // transform of z, conjugated and divided by kN, is the inverse transform of Z.
    for (int k = threadIdx.x; k < kBins; k += kT) {
        float2 xl = make_float2(0.f, 0.f), xr = make_float2(0.f, 0.f);
        float2 cl = xl, cr = xr;
        for (int s = 0; s < ns; ++s) {
            const float2 *ps = base + (size_t)s * 2 * kFftBinsPadded;
            const float2 vl = ps[k], vr = ps[kFftBinsPadded + k];
            float y, t;
            y = vl.x - cl.x; t = xl.x + y; cl.x = (t - xl.x) - y; xl.x = t;
            y = vl.y - cl.y; t = xl.y + y; cl.y = (t - xl.y) - y; xl.y = t;
            y = vr.x - cr.x; t = xr.x + y; cr.x = (t - xr.x) - y; xr.x = t;
            y = vr.y - cr.y; t = xr.y + y; cr.y = (t - xr.y) - y; xr.y = t;
        }
        buf[pad(k)] = make_float2(xl.x - xr.y, -(xl.y + xr.x));
        if (k > 0 && k < kN / 2) buf[pad(kN - k)] = make_float2(xl.x + xr.y, xl.y - xr.x);
    }
    __syncthreads();
    float2 u[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) u[r] = buf[pad(threadIdx.x + r * kT)];
    __syncthreads();
    fft_forward(u, buf, a.tw);
    const float inv = 1.0f / (float)kN;
    const int64_t o0 = (int64_t)f * a.hop;
    for (int t = threadIdx.x; t < a.hop; t += kT) {
        const int64_t n = o0 + t;
        if (n >= a.out_len) break;
        const float2 z = buf[pad(a.guard + t)];
        a.out[n] = z.x * inv;
        a.out[a.out_ld + n] = -z.y * inv;
    }
}

}  // namespace

size_t fft_mix_smem_bytes(int elem_bytes)
{
    return (size_t)2 * 2 * kN * elem_bytes + (size_t)kPadded * sizeof(float2) + 2 * 8 + 16;
}

cudaError_t launch_build_spectra(const float *dense, int padded_len, int hrir_len, int n_records,
                                 const float2 *tw, float2 *spec, cudaStream_t st)
{
    build_spectra_kernel<<<n_records, kT, 0, st>>>(dense, padded_len, hrir_len, tw, spec);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_fft_mix_t(const CUtensorMap &tmap, const FftArgs &a, int grid, size_t smem,
                                    cudaStream_t st)
{
    auto k = fft_mix_kernel<T>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kT, smem, st>>>(tmap, a);
    return cudaGetLastError();
}

cudaError_t launch_fft_mix(int dtype, const CUtensorMap &tmap, const FftArgs &a, int grid,
                           size_t smem, cudaStream_t st)
{
    if (dtype == 0) return launch_fft_mix_t<float>(tmap, a, grid, smem, st);
    if (dtype == 1) return launch_fft_mix_t<__nv_bfloat16>(tmap, a, grid, smem, st);
    return launch_fft_mix_t<__half>(tmap, a, grid, smem, st);
}

cudaError_t launch_fft_out(const FftOutArgs &a, int n_frames, cudaStream_t st)
{
    if (n_frames <= 0) return cudaSuccess;
    fft_out_kernel<<<n_frames, kT, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace hrir
