// reduce_fir.cu -- deterministic mix reduction fused with the resonance FIR (sm_103a).
//
//   z_e[m]   = sum over the partial slots of tile(m), in slot order, compensated (Kahan)
//   out_e[n] = sum_{l < Lf} f_e[l] z_e[n - l]          (the resonance stage of Eq. 2;
//                                                      identity when no filter is given),
//              a compensated dot product
// Each block produces kBlk outputs of one ear: it first forms z for [n0 - Lf + 1, n0 + kBlk)
// in shared memory (coalesced partial reads, fixed summation order), then applies the FIR.
// parts_fir_kernel does the same for z given as the sum of a few whole reflection mixes (the
// mixes of disjoint source sets, e.g. one per GPU), added in part order.
#include "kernels.h"

namespace hrir {

namespace {

constexpr int kBlk = 2048;
constexpr int kThreads = 256;
constexpr int kMaxRes = 512;
constexpr int kMaxSpanTiles = 16;   // partial tiles one block's z span may touch

// sum_l f[l] z[lf - 1 - l] for l < lf: a compensated dot product (Ogita, Rump & Oishi 2005,
// "Dot2"): the products' and the running sum's rounding errors are carried exactly
// (error-free transformations) and added at the end, so the result is as accurate as a sum
// in twice the working precision; the FIR can cancel most of z where f attenuates z's band,
// which would otherwise magnify its FP32 rounding relative to the output
__device__ __forceinline__ float fir_dot2(const float *fs, const float *z, int lf)
{
    float p = 0.f, c = 0.f;
    for (int l = 0; l < lf; ++l) {
        const float x = fs[l], y = z[lf - 1 - l];
        const float h = __fmul_rn(x, y);
        const float r = fmaf(x, y, -h);               // h + r == x * y exactly
        const float s2 = __fadd_rn(p, h);
        const float bb = __fsub_rn(s2, p);
        const float q = __fadd_rn(__fsub_rn(p, __fsub_rn(s2, bb)), __fsub_rn(h, bb));  // p + h == s2 + q
        p = s2;
        c = __fadd_rn(c, __fadd_rn(q, r));
    }
    return __fadd_rn(p, c);
}

__global__ void __launch_bounds__(kThreads) reduce_fir_kernel(const ReduceArgs a)
{
    __shared__ float zs[kBlk + kMaxRes - 1];
    __shared__ float fs[kMaxRes];
    __shared__ int nslots[kMaxSpanTiles];
    const int e = blockIdx.y;
    const int64_t n0 = (int64_t)blockIdx.x * kBlk;
    const int lf = a.res ? a.res_len : 1;
    const int64_t m_lo = n0 - (lf - 1);
    const int64_t m_hi = n0 + kBlk;  // exclusive
    const int64_t z_len = (int64_t)a.n_tiles * a.tile;
    const int t_lo = (int)((m_lo > 0 ? m_lo : 0) / a.tile);
    for (int k = threadIdx.x; k < kMaxSpanTiles; k += kThreads)
        nslots[k] = t_lo + k < a.n_tiles ? a.part.slots(t_lo + k) : 0;
    for (int l = threadIdx.x; l < lf; l += kThreads) fs[l] = a.res ? a.res[e * a.res_len + l] : 1.0f;
    __syncthreads();
    const int span = (int)(m_hi - m_lo);
    for (int i = threadIdx.x; i < span; i += kThreads) {
        const int64_t m = m_lo + i;
        float sum = 0.f;
        if (m >= 0 && m < z_len) {
            const int t = (int)(m / a.tile);
            const int ns = nslots[t - t_lo];
            const float *p = a.partial + ((size_t)t * a.slots * 2 + e) * a.tile + (m - (int64_t)t * a.tile);
            float c = 0.f;
            for (int j = 0; j < ns; ++j) {
                const float y = p[(size_t)j * 2 * a.tile] - c;
                const float tt = sum + y;
                c = (tt - sum) - y;
                sum = tt;
            }
        }
        zs[i] = sum;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBlk; i += kThreads) {
        const int64_t n = n0 + i;
        if (n >= a.out_len) break;
        a.out[e * a.out_ld + n] = fir_dot2(fs, zs + i, lf);
    }
}

// Blocks of parts_fir_kernel: out_e[n] = sum_l f_e[l] z_e[n - l], z_e[m] = sum_c parts[c][e][m]
// (compensated, in c order; zero outside [0, z_len)).
__global__ void __launch_bounds__(kThreads) parts_fir_kernel(const float *__restrict__ parts, int n_parts,
                                                             int64_t part_ld, int64_t z_len,
                                                             const float *__restrict__ res, int res_len,
                                                             int64_t out_len, float *__restrict__ out,
                                                             int64_t out_ld)
{
    __shared__ float zs[kBlk + kMaxRes - 1];
    __shared__ float fs[kMaxRes];
    const int e = blockIdx.y;
    const int64_t n0 = (int64_t)blockIdx.x * kBlk;
    const int lf = res ? res_len : 1;
    const int64_t m_lo = n0 - (lf - 1);
    for (int l = threadIdx.x; l < lf; l += kThreads) fs[l] = res ? res[e * res_len + l] : 1.0f;
    const int span = (int)(n0 + kBlk - m_lo);
    for (int i = threadIdx.x; i < span; i += kThreads) {
        const int64_t m = m_lo + i;
        float sum = 0.f;
        if (m >= 0 && m < z_len) {
            const float *p = parts + (size_t)e * part_ld + m;
            float c = 0.f;
            for (int j = 0; j < n_parts; ++j) {
                const float y = p[(size_t)j * 2 * part_ld] - c;
                const float tt = sum + y;
                c = (tt - sum) - y;
                sum = tt;
            }
        }
        zs[i] = sum;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBlk; i += kThreads) {
        const int64_t n = n0 + i;
        if (n >= out_len) break;
        out[e * out_ld + n] = fir_dot2(fs, zs + i, lf);
    }
}

// out[e][n] = sum_c parts[c][e][n] in c order (2 planes of n floats per part).
__global__ void add_parts_kernel(float *__restrict__ out, int64_t out_ld, const float *__restrict__ parts,
                                 int n_parts, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * n; i += (int64_t)gridDim.x * blockDim.x) {
        float acc = parts[i];
        for (int c = 1; c < n_parts; ++c) acc += parts[(size_t)c * 2 * n + i];
        const int64_t e = i / n;
        out[e * out_ld + (i - e * n)] = acc;
    }
}

// One thread waits on an mbarrier that nothing arrives on, through the bounded wait every
// pipelined kernel uses: after the wait limit it raises the abort flag and ORs DEV_TIMEOUT
// into *status, then returns (a self-test of the failure path; nothing hangs or traps).
__global__ void wait_timeout_selftest_kernel(int *status)
{
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    mbar_init(smem_addr(&bar), 1);
    abort_flag = 0;
    mbar_fence_init();
    mbar_wait_bounded(smem_addr(&bar), 0u, &abort_flag, status);
}

}  // namespace

cudaError_t launch_wait_timeout_selftest(int *status, cudaStream_t st)
{
    wait_timeout_selftest_kernel<<<1, 1, 0, st>>>(status);
    return cudaGetLastError();
}

cudaError_t launch_add_parts(float *out, int64_t out_ld, const float *parts, int n_parts, int64_t n,
                             cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = (2 * n + 255) / 256;
    add_parts_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(out, out_ld, parts, n_parts, n);
    return cudaGetLastError();
}

cudaError_t launch_parts_fir(const float *parts, int n_parts, int64_t part_ld, int64_t z_len, const float *res,
                             int res_len, int64_t out_len, float *out, int64_t out_ld, cudaStream_t st)
{
    if (out_len <= 0) return cudaSuccess;
    if ((res ? res_len : 1) > kMaxRes || n_parts < 1) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((out_len + kBlk - 1) / kBlk), 2);
    parts_fir_kernel<<<grid, kThreads, 0, st>>>(parts, n_parts, part_ld, z_len, res, res_len, out_len, out, out_ld);
    return cudaGetLastError();
}

cudaError_t launch_reduce(const ReduceArgs &a, cudaStream_t st)
{
    if (a.out_len <= 0) return cudaSuccess;
    if ((a.res ? a.res_len : 1) > kMaxRes || a.tile < 1 ||
        (kBlk + kMaxRes - 2) / a.tile + 2 > kMaxSpanTiles)
        return cudaErrorInvalidValue;
    dim3 grid((unsigned)((a.out_len + kBlk - 1) / kBlk), 2);
    reduce_fir_kernel<<<grid, kThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace hrir
