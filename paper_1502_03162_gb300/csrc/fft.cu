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
// fft_mix_kernel's FFT is a radix-16 Stockham (autosort) transform of P = 4096 points by 256
// threads in three passes (two exchanges through padded shared-memory buffers, ping-pong);
// the spectra builder and the inverse transform use a radix-8 Stockham transform by 512
// threads in four passes.  Twiddles come from a table computed in double on the host.
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
// One (frame, source pair) unit per step of a persistent CTA of 256 threads: the 4096-point
// complex FFT of z = y_a + i y_b as a radix-16 Stockham transform (three passes; thread t holds
// 16 points per pass), the split into the two real spectra, and the multiply-accumulate with
// each source's HRIR spectra per ear (the mix happens in the frequency domain).
constexpr int kT16 = kN / 16;        // 256 threads

// complex addition and subtraction as one packed FP32 instruction each (add/sub.rn.f32x2:
// two independent round-to-nearest operations, the same results as two scalar ones)
__device__ __forceinline__ float2 padd(float2 a, float2 b)
{
    uint64_t x, y, r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b.x), "f"(b.y));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
    float2 o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
    return o;
}
__device__ __forceinline__ float2 psub(float2 a, float2 b)
{
    uint64_t x, y, r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b.x), "f"(b.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
    float2 o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
    return o;
}

// forward 4-point DFT (exp(-2 pi i nk / 4)) in place
__device__ __forceinline__ void dft4(float2 &a, float2 &b, float2 &c, float2 &d)
{
    const float2 t0 = padd(a, c), t1 = psub(a, c), t2 = padd(b, d), t3 = mul_mi(psub(b, d));
    a = padd(t0, t2);
    c = psub(t0, t2);
    b = padd(t1, t3);
    d = psub(t1, t3);
}

// forward 16-point DFT in registers, natural order in and out: four DFT4s over (n, n+4, n+8,
// n+12), twiddles exp(-2 pi i n m / 16), four DFT4s over n; output index m + 4 k
__device__ __forceinline__ void dft16(float2 (&u)[16])
{
    dft4(u[0], u[4], u[8], u[12]);
    dft4(u[1], u[5], u[9], u[13]);
    dft4(u[2], u[6], u[10], u[14]);
    dft4(u[3], u[7], u[11], u[15]);
    // u[n + 4 m] *= w16^(n m), w16^j = (cos(2 pi j / 16), -sin(2 pi j / 16))
    const float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
    u[5] = cmul(u[5], make_float2(c1, -s1));        // n 1, m 1
    u[9] = cmul(u[9], make_float2(h, -h));          // n 1, m 2
    u[13] = cmul(u[13], make_float2(s1, -c1));      // n 1, m 3
    u[6] = cmul(u[6], make_float2(h, -h));          // n 2, m 1
    u[10] = mul_mi(u[10]);                          // n 2, m 2: w16^4 = -i
    u[14] = cmul(u[14], make_float2(-h, -h));       // n 2, m 3: w16^6
    u[7] = cmul(u[7], make_float2(s1, -c1));        // n 3, m 1: w16^3
    u[11] = cmul(u[11], make_float2(-h, -h));       // n 3, m 2: w16^6
    u[15] = cmul(u[15], make_float2(-c1, s1));      // n 3, m 3: w16^9
    dft4(u[0], u[1], u[2], u[3]);
    dft4(u[4], u[5], u[6], u[7]);
    dft4(u[8], u[9], u[10], u[11]);
    dft4(u[12], u[13], u[14], u[15]);
    // now u[m 4 + k] holds X[m + 4 k]: transpose the 4 x 4 index
    float2 t;
    t = u[1]; u[1] = u[4]; u[4] = t;
    t = u[2]; u[2] = u[8]; u[8] = t;
    t = u[3]; u[3] = u[12]; u[12] = t;
    t = u[6]; u[6] = u[9]; u[9] = t;
    t = u[7]; u[7] = u[13]; u[13] = t;
    t = u[11]; u[11] = u[14]; u[14] = t;
}

// Shared memory: one TMA stage [kN/256 boxes][2 rows][256] of source samples, two padded FFT
// buffers (ping-pong), the twiddle tables, an mbarrier.
template <typename T>
__global__ void __launch_bounds__(kT16, kFftCtasPerSm)
    fft_mix_kernel(const __grid_constant__ CUtensorMap tmap, const FftArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    T *stage = reinterpret_cast<T *>(smem);                                  // [2 * kN]
    float2 *bufA = reinterpret_cast<float2 *>(smem + 2 * kN * sizeof(T));     // [kPadded]
    float2 *bufB = bufA + kPadded;                                            // [kPadded]
    // twiddles w = exp(-2 pi i / kN): tw16[r][a] = w^(16 a r), tw1[r][b] = w^(b r), so that
    // pass 2 reads w^(16 (t % 16) r) = tw16[r][t % 16] and pass 3 forms w^(t r) =
    // tw16[r][t / 16] tw1[r][t % 16] (two roundings), both conflict-free or broadcast
    float2 *tw16 = bufB + kPadded;                                            // [16][16]
    float2 *tw1 = tw16 + 256;                                                 // [16][16]
    uint64_t *bar = reinterpret_cast<uint64_t *>(tw1 + 256);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bar + 1);
    const int tid = threadIdx.x;
    if (tid == 0) {
        prefetch_tensormap(&tmap);
        mbar_init(smem_addr(bar), 1);
        *abort_flag = 0;
        mbar_fence_init();
    }
    {
        const int r = tid >> 4, c = tid & 15;
        tw16[tid] = __ldg(a.tw + ((16 * c * r) & (kN - 1)));
        tw1[tid] = __ldg(a.tw + c * r);
    }
    __syncthreads();
    const int64_t u_begin = a.part.first(blockIdx.x), u_end = a.part.first(blockIdx.x + 1);
    const int n_pairs = a.part.n_src;

    auto issue = [&](int64_t u) {
        const int j = (int)(u / n_pairs);
        const int p = (int)(u - (int64_t)j * n_pairs);
        const int x0 = j * a.hop - a.guard;
        mbar_arrive_expect_tx(smem_addr(bar), (uint32_t)(2 * kN * sizeof(T)));
        for (int b = 0; b < kN / 256; ++b)
            tma_load_2d(smem_addr(stage + b * 512), &tmap, x0 + b * 256, 2 * p, smem_addr(bar));
    };
    if (tid == 0 && u_begin < u_end) issue(u_begin);

    float2 accL[8], accR[8], accL8 = make_float2(0.f, 0.f), accR8 = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 8; ++q) accL[q] = accR[q] = make_float2(0.f, 0.f);
    int cur_f = -1, slot = 0, run_n = 0;
    int64_t issued_to = u_begin + 1;     // units whose loads have been issued: [u_begin, issued_to)
    for (int64_t u = u_begin, k = 0; u < u_end; ++u, ++k) {
        const int f = (int)(u / n_pairs);
        const int p = (int)(u - (int64_t)f * n_pairs);
        if (f != cur_f) {
            cur_f = f;
            slot = a.part.slot_base(blockIdx.x, f);
            run_n = 0;
        }
        const bool ok = mbar_wait_bounded(smem_addr(bar), (uint32_t)(k & 1), abort_flag, a.status);
        if (__syncthreads_or(!ok)) {  // every thread leaves together: no one is left at a barrier
            if (tid == 0 && issued_to > u) {
                // let the copy in flight land (bounded)
                const uint64_t t0 = global_timer_ns();
                while (!mbar_try_wait(smem_addr(bar), (uint32_t)(k & 1)) && global_timer_ns() - t0 < kWaitLimitNs) {
                }
            }
            break;
        }
        // The two FFT buffers change roles from unit to unit (X for the first pass's output and
        // the mirror bins, Y for the second pass's output), so that a unit's first stores never
        // touch the buffer the previous unit's multiply-accumulate still reads: three CTA
        // barriers per unit.
        float2 *X = (k & 1) ? bufB : bufA;
        float2 *Y = (k & 1) ? bufA : bufB;
        // pass 1 (p = 1): z[t + 256 r] from the stage, DFT16, to X at 16 t + r
        float2 v[16];
#pragma unroll
        for (int r = 0; r < 16; ++r)
            v[r] = make_float2(to_f<T>(stage[r * 512 + tid]), to_f<T>(stage[r * 512 + 256 + tid]));
        dft16(v);
#pragma unroll
        for (int r = 0; r < 16; ++r) X[pad(16 * tid + r)] = v[r];
        __syncthreads();                                     // stage consumed, X written
        if (tid == 0 && u + 1 < u_end) {
            issue(u + 1);                                    // the next unit's source, now
            issued_to = u + 2;
        }
        // pass 2 (p = 16): X -> Y
        {
            const int kk = tid & 15;
#pragma unroll
            for (int r = 0; r < 16; ++r) v[r] = X[pad(tid + 256 * r)];
#pragma unroll
            for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], tw16[16 * r + kk]);
            dft16(v);
            const int j = (tid - kk) * 16 + kk;
#pragma unroll
            for (int r = 0; r < 16; ++r) Y[pad(j + 16 * r)] = v[r];
        }
        __syncthreads();                                     // Y written
        // pass 3 (p = 256): Y -> registers: v[r] = Z[t + 256 r]
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = Y[pad(tid + 256 * r)];
#pragma unroll
        for (int r = 1; r < 16; ++r)
            v[r] = cmul(v[r], cmul(tw16[16 * r + (tid >> 4)], tw1[16 * r + (tid & 15)]));
        dft16(v);
        // the mirror bins Z[4096 - k] of every k < 2048 lie in the upper halves (r >= 8)
#pragma unroll
        for (int r = 8; r < 16; ++r) X[pad(tid + 256 * r)] = v[r];
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
        // the spectra of the first four bins are requested before the barrier (their latency
        // overlaps it); the other four after
        float2 hp[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int kb = tid + 256 * q;
            hp[q][0] = __ldg(h0 + kb);
            hp[q][1] = __ldg(h1 + kb);
            hp[q][2] = __ldg(h0 + kFftBinsPadded + kb);
            hp[q][3] = __ldg(h1 + kFftBinsPadded + kb);
        }
        __syncthreads();                                     // mirrors written
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int kb = tid + 256 * q;
            const float2 zm = (tid == 0) ? (q == 0 ? v[0] : X[pad(kN - 256 * q)]) : X[pad(kN - kb)];
            float2 y0, y1;
            split_real_pair(v[q], zm, y0, y1);
            float2 g0, g1, g2, g3;
            if (q < 4) {
                g0 = hp[q & 3][0];
                g1 = hp[q & 3][1];
                g2 = hp[q & 3][2];
                g3 = hp[q & 3][3];
            } else {
                g0 = __ldg(h0 + kb);
                g1 = __ldg(h1 + kb);
                g2 = __ldg(h0 + kFftBinsPadded + kb);
                g3 = __ldg(h1 + kFftBinsPadded + kb);
            }
            accL[q] = padd(accL[q], padd(cmul(y0, g0), cmul(y1, g1)));
            accR[q] = padd(accR[q], padd(cmul(y0, g2), cmul(y1, g3)));
        }
        if (tid == 0) {                                      // the Nyquist bin, its own mirror
            const int kb = kN / 2;
            float2 y0, y1;
            split_real_pair(v[8], v[8], y0, y1);
            accL8 = cadd(accL8, cadd(cmul(y0, __ldg(h0 + kb)), cmul(y1, __ldg(h1 + kb))));
            accR8 = cadd(accR8, cadd(cmul(y0, __ldg(h0 + kFftBinsPadded + kb)),
                                     cmul(y1, __ldg(h1 + kFftBinsPadded + kb))));
        }
        ++run_n;
        const bool frame_end = (u + 1 == u_end) || ((u + 1) / n_pairs != f);
        if (run_n == a.part.gs || frame_end) {
            float2 *ps = a.partial + ((size_t)f * a.slots + slot) * 2 * kFftBinsPadded;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                ps[tid + 256 * q] = accL[q];
                ps[kFftBinsPadded + tid + 256 * q] = accR[q];
                accL[q] = accR[q] = make_float2(0.f, 0.f);
            }
            if (tid == 0) {
                ps[kN / 2] = accL8;
                ps[kFftBinsPadded + kN / 2] = accR8;
                accL8 = accR8 = make_float2(0.f, 0.f);
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
    return (size_t)2 * kN * elem_bytes + (2 * (size_t)kPadded + 512) * sizeof(float2) + 8 + 16;
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
    k<<<grid, kT16, smem, st>>>(tmap, a);
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
