// tables.cu -- filter-pack kernels (sm_103a): top-K tap selection, the sparse tap records
// consumed by the mixing kernel, and the dense HRIRs x = f * g (Eq. 1) for the baselines.
#include <climits>
#include <type_traits>

#include "kernels.h"

namespace hrir {

namespace {

// ---- top-K: one warp per row at a time ---------------------------------------------------
// Keeps the k largest strictly positive entries (ties -> smaller index), emitted in ascending
// index order, padded with (0, 0).  Lane l holds the contiguous slice [l*per, (l+1)*per) in
// MAXPER registers (the smallest of 8, 16, 32, 64 that holds per = ceil(refl_len / 32)).
// Persistent: each warp walks rows row0, row0 + n_warps, ... and loads the next row's slice
// while it selects from the current one.
constexpr int kTopkMaxPer = 64;  // refl_len <= 32 * 64 = 2048

template <int MAXPER>
__device__ __forceinline__ void topk_load(const float *__restrict__ g, int row, int n_rows, int refl_len,
                                          int per, int j0, float (&v)[MAXPER])
{
    const float *gr = g + (size_t)row * refl_len;
#pragma unroll
    for (int j = 0; j < MAXPER; ++j) {
        const int gi = j0 + j;
        v[j] = (row < n_rows && j < per && gi < refl_len) ? __ldg(gr + gi) : 0.0f;  // 0 is never selected
    }
}

// Rows of a multiple of 8 values at 16-byte aligned addresses: lane l takes the 8 values
// [8 l, 8 l + 8) by two 16-byte loads (lanes past the row take zeros).
__device__ __forceinline__ void topk_load_vec8(const float *__restrict__ g, int row, int n_rows, int refl_len, int j0,
                                               float (&v)[8])
{
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    if (row < n_rows && j0 < refl_len) {
        const float4 *gr = reinterpret_cast<const float4 *>(g + (size_t)row * refl_len + j0);
        a = __ldg(gr);
        b = __ldg(gr + 1);
    }
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// hint: a threshold that separated the k largest keys of an earlier, similar row (0: none);
// it only shortens the search (the selected set does not depend on it).  Returns the
// threshold found for this row (or hint when every positive entry is taken).
template <int MAXPER>
__device__ __forceinline__ uint32_t topk_row(const float (&v)[MAXPER], int row, int j0, int lane, int k,
                                             uint32_t hint, uint16_t *__restrict__ idx, float *__restrict__ w,
                                             uint8_t *__restrict__ nnz)
{
    // Keys: the bits of a strictly positive float order like the float; 0 = not selectable.
    // The selected set is every key above T plus the first ties at T in index order, where T
    // is the k-th largest key: the largest t with #(key >= t) >= k, found by bisection over
    // the key bits (warp-wide counts), stopping early when exactly k keys are >= t.
    using Mask = typename std::conditional<(MAXPER <= 32), uint32_t, uint64_t>::type;
    uint32_t key[MAXPER];
#pragma unroll
    for (int j = 0; j < MAXPER; ++j) key[j] = v[j] > 0.f ? __float_as_uint(v[j]) : 0u;
    auto count_ge = [&](uint32_t t) {
        int c = 0;
#pragma unroll
        for (int j = 0; j < MAXPER; ++j) c += key[j] >= t;
        return (int)__reduce_add_sync(0xffffffffu, (uint32_t)c);
    };
    // first one count at the earlier row's threshold: when exactly k keys lie at or above it
    // (a row whose k-th and (k + 1)-th keys still straddle it) those are the selection
    const int c_hint = hint > 1u ? count_ge(hint) : -1;
    Mask taken = 0;
    int cnt;
    if (c_hint == k) {
#pragma unroll
        for (int j = 0; j < MAXPER; ++j)
            if (key[j] >= hint) taken |= (Mask)1 << j;
        cnt = k;
    } else {
        int n_pos = 0;
        uint32_t kmax = 0;
#pragma unroll
        for (int j = 0; j < MAXPER; ++j) {
            n_pos += key[j] != 0u;
            kmax = key[j] > kmax ? key[j] : kmax;
        }
        const int total = (int)__reduce_add_sync(0xffffffffu, (uint32_t)n_pos);
        if (total <= k) {                       // every positive entry
#pragma unroll
            for (int j = 0; j < MAXPER; ++j)
                if (key[j]) taken |= (Mask)1 << j;
            cnt = total;
        } else {
            uint32_t lo = 1, hi = __reduce_max_sync(0xffffffffu, kmax) + 1u;   // #(>= lo) >= k > #(>= hi)
            bool exact = false;
            if (c_hint >= 0 && hint < hi) {     // the earlier row's threshold as a bound
                if (c_hint > k) lo = hint;
                else hi = hint;
            }
            if (!exact && k <= 32) {
                // a tighter start: the k-th largest lane maximum (k lanes hold a key at least that
                // large), from a bitonic sort of the 32 lane maxima (ascending across the lanes)
                uint32_t x = kmax;
#pragma unroll
                for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
                    for (int stride = size >> 1; stride > 0; stride >>= 1) {
                        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, stride);
                        const bool asc = (lane & size) == 0, lower = (lane & stride) == 0;
                        x = (asc == lower) ? (x < y ? x : y) : (x > y ? x : y);
                    }
                }
                const uint32_t kth = __shfl_sync(0xffffffffu, x, 32 - k);
                lo = kth > lo ? kth : lo;
            }
            while (!exact && hi - lo > 1u) {
                const uint32_t mid = lo + (hi - lo) / 2u;
                const int c = count_ge(mid);
                if (c >= k) {
                    lo = mid;
                    if (c == k) {
                        exact = true;
                        break;
                    }
                } else {
                    hi = mid;
                }
            }
            if (exact) {
#pragma unroll
                for (int j = 0; j < MAXPER; ++j)
                    if (key[j] >= lo) taken |= (Mask)1 << j;
            } else {
                // lo is the k-th largest key: every key above it, then its ties in index order
                int need = k - count_ge(lo + 1u);
                int ties = 0;
#pragma unroll
                for (int j = 0; j < MAXPER; ++j) ties += key[j] == lo;
                int before_t = ties;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int o = __shfl_up_sync(0xffffffffu, before_t, off);
                    if (lane >= off) before_t += o;
                }
                need -= before_t - ties;        // ties already taken by lower lanes
#pragma unroll
                for (int j = 0; j < MAXPER; ++j) {
                    if (key[j] > lo) {
                        taken |= (Mask)1 << j;
                    } else if (key[j] == lo && need > 0) {
                        taken |= (Mask)1 << j;
                        --need;
                    }
                }
            }
            cnt = k;
            hint = lo;                              // a threshold inside this row's gap
        }
    }
    // ascending-index output: lanes hold ascending slices; prefix-count the kept entries
    const int mine = MAXPER <= 32 ? __popc((uint32_t)taken) : __popcll((uint64_t)taken);
    int before = mine;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, before, off);
        if (lane >= off) before += o;
    }
    before -= mine;
    uint16_t *ri = idx + (size_t)row * k;
    float *rw = w + (size_t)row * k;
    int o = before;
#pragma unroll
    for (int j = 0; j < MAXPER; ++j) {
        if ((taken >> j) & 1) {
            ri[o] = (uint16_t)(j0 + j);
            rw[o] = v[j];
            ++o;
        }
    }
    for (int t = cnt + lane; t < k; t += 32) {
        ri[t] = 0;
        rw[t] = 0.f;
    }
    if (lane == 0) nnz[row] = (uint8_t)cnt;
    return hint;
}

template <int MAXPER, bool VEC8>
__global__ void __launch_bounds__(128) topk_kernel(const float *__restrict__ g, int n_rows,
                                                   int refl_len, int k, uint16_t *__restrict__ idx,
                                                   float *__restrict__ w, uint8_t *__restrict__ nnz)
{
    // each warp takes a contiguous run of rows, so that row r - 2 (the same ear of the
    // previous segment or direction in the (.., ear) row order) gives row r's search a start
    const int lane = threadIdx.x & 31;
    const int64_t n_warps = (int64_t)gridDim.x * 4;
    const int64_t chunk = ((int64_t)n_rows + n_warps - 1) / n_warps;
    const int64_t wid = (int64_t)blockIdx.x * 4 + (threadIdx.x >> 5);
    const int r0 = (int)(wid * chunk < n_rows ? wid * chunk : n_rows);
    const int r1 = (int)(r0 + chunk < n_rows ? r0 + chunk : n_rows);
    const int per = VEC8 ? 8 : (refl_len + 31) / 32;
    const int j0 = lane * per;
    auto load = [&](int r, float (&v)[MAXPER]) {
        if constexpr (VEC8) topk_load_vec8(g, r, n_rows, refl_len, j0, v);
        else topk_load<MAXPER>(g, r, n_rows, refl_len, per, j0, v);
    };
    // D rows in flight per warp (the loads of rows row + D .. are issued as each buffer frees)
    constexpr int D = MAXPER <= 16 ? 3 : 1;
    float v[D][MAXPER];
#pragma unroll
    for (int d = 0; d < D; ++d) load(r0 + d < r1 ? r0 + d : n_rows, v[d]);
    uint32_t hint0 = 0u, hint1 = 0u;             // the last thresholds of even and odd rows
    for (int row = r0; row < r1; row += D) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int r = row + d;
            if (r < r1) {
                const uint32_t h = topk_row<MAXPER>(v[d], r, j0, lane, k, (r & 1) ? hint1 : hint0, idx, w, nnz);
                if (r & 1) hint1 = h;
                else hint0 = h;
            }
            load(r + D < r1 ? r + D : n_rows, v[d]);
        }
    }
}

// ---- sparse records ------------------------------------------------------------------------
// Record of one direction for the tensor-memory sparse kernel, whose window covers one
// segment of seg_len filter offsets at a time:
//   int4  {n_seg, 0, 0, 0}
//   int2  cnt[nseg_pad] {left taps, right taps} of each segment
//   int2  tap[...] {TMEM column, weight bits}: per segment, its left then its right taps,
//         each list padded to an even length with a zero-weight tap at column 1, then 4
//         zero-weight entries (the kernel reads two taps ahead)
// A tap at offset o of segment s reads window columns (s+1) seg_len - o onward.
__global__ void build_sparse_records_kernel(const uint16_t *__restrict__ idx,
                                            const float *__restrict__ w,
                                            const uint8_t *__restrict__ nnz, int n_dirs, int k_max,
                                            int seg_len, int n_seg, int nseg_pad,
                                            unsigned char *__restrict__ rec, int rec_bytes)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d > n_dirs) return;
    unsigned char *r0 = rec + (size_t)d * rec_bytes;
    int4 *hdr = reinterpret_cast<int4 *>(r0);
    int2 *cnt = reinterpret_cast<int2 *>(r0 + 16);
    int2 *taps = reinterpret_cast<int2 *>(r0 + 16 + 8 * nseg_pad);
    for (int c = 0; c < nseg_pad; ++c) cnt[c] = make_int2(0, 0);
    if (d == n_dirs) {  // the silent record used for out-of-range direction ids
        *hdr = make_int4(0, 0, 0, 0);
        return;
    }
    int o = 0;
    for (int s = 0; s < n_seg; ++s) {
        const int lo = s * seg_len, hi = lo + seg_len;
        int n_e[2] = {0, 0};
        for (int e = 0; e < 2; ++e) {
            const size_t row = ((size_t)d * 2 + e) * k_max;
            const int k = nnz[(size_t)d * 2 + e];
            for (int t = 0; t < k; ++t) {
                const int i = idx[row + t];
                if (i < lo || i >= hi) continue;
                taps[o++] = make_int2(hi - i, __float_as_int(w[row + t]));
                ++n_e[e];
            }
            if (n_e[e] & 1) {
                taps[o++] = make_int2(1, 0);
                ++n_e[e];
            }
        }
        cnt[s] = make_int2(n_e[0], n_e[1]);
    }
    for (int p = 0; p < 4; ++p) taps[o++] = make_int2(1, 0);
    *hdr = make_int4(n_seg, 0, 0, 0);
}

// ---- dense HRIRs: x_{d,e}[n] = sum_t w_t f_e[n - idx_t] (Eq. 1), zero padded -------------
__global__ void build_dense_records_kernel(const uint16_t *__restrict__ idx,
                                           const float *__restrict__ w,
                                           const uint8_t *__restrict__ nnz, int n_dirs, int k_max,
                                           const float *__restrict__ res, int res_len, int hrir_len,
                                           int padded_len, float *__restrict__ rec)
{
    const int64_t total = (int64_t)(n_dirs + 1) * 2 * padded_len;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int n = (int)(i % padded_len);
        const int64_t de = i / padded_len;
        const int e = (int)(de % 2);
        const int d = (int)(de / 2);
        float acc = 0.f;
        if (d < n_dirs && n < hrir_len) {
            const size_t row = ((size_t)d * 2 + e) * k_max;
            const int k = nnz[(size_t)d * 2 + e];
            for (int t = 0; t < k; ++t) {
                const int l = n - (int)idx[row + t];
                if (l >= 0 && l < res_len) acc = fmaf(w[row + t], res[e * res_len + l], acc);
            }
        }
        rec[i] = acc;
    }
}

}  // namespace

cudaError_t launch_topk(const float *g, int n_rows, int refl_len, int k, uint16_t *idx, float *w,
                        uint8_t *nnz, cudaStream_t st)
{
    if (n_rows <= 0) return cudaSuccess;
    if (refl_len > 32 * kTopkMaxPer) return cudaErrorInvalidValue;
    const int per = (refl_len + 31) / 32;
    // persistent warps: one resident wave of 4-warp blocks, fewer for small inputs
    auto launch = [&](auto kern) {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
            sms = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128, 0) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        const int64_t need = ((int64_t)n_rows + 3) / 4, wave = (int64_t)sms * per_sm;
        kern<<<(unsigned)(need < wave ? need : wave), 128, 0, st>>>(g, n_rows, refl_len, k, idx, w, nnz);
    };
    if (refl_len % 8 == 0 && refl_len <= 256 && (reinterpret_cast<uintptr_t>(g) & 15) == 0)
        launch(topk_kernel<8, true>);          // 8 values a lane, two 16-byte loads
    else if (per <= 8) launch(topk_kernel<8, false>);
    else if (per <= 16) launch(topk_kernel<16, false>);
    else if (per <= 32) launch(topk_kernel<32, false>);
    else launch(topk_kernel<64, false>);
    return cudaGetLastError();
}

cudaError_t launch_build_sparse_records(const uint16_t *idx, const float *w, const uint8_t *nnz,
                                        int n_dirs, int k_max, int seg_len, int n_seg, int nseg_pad,
                                        unsigned char *rec, int rec_bytes, cudaStream_t st)
{
    const int n = n_dirs + 1;
    build_sparse_records_kernel<<<(n + 127) / 128, 128, 0, st>>>(
        idx, w, nnz, n_dirs, k_max, seg_len, n_seg, nseg_pad, rec, rec_bytes);
    return cudaGetLastError();
}

cudaError_t launch_build_dense_records(const uint16_t *idx, const float *w, const uint8_t *nnz,
                                       int n_dirs, int k_max, const float *res, int res_len,
                                       int hrir_len, int padded_len, float *rec, cudaStream_t st)
{
    const int64_t total = (int64_t)(n_dirs + 1) * 2 * padded_len;
    const int blocks = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    build_dense_records_kernel<<<blocks, 256, 0, st>>>(idx, w, nnz, n_dirs, k_max, res, res_len,
                                                       hrir_len, padded_len, rec);
    return cudaGetLastError();
}

}  // namespace hrir
