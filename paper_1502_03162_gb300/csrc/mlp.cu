// mlp.cu -- learned reflection filters: the direction -> filter network (5 -> 256 -> 256 ->
// 256 -> Lg, ReLU, softplus output so every tap is >= 0 like the paper's G >= 0, Eq. 3),
// its backward pass for the least-squares loss against factorized reflection rows
// (Algorithm 1 output), and the Adam update.  FP32 values; the matrix products (forward
// X W^T, backward dZ W, weight gradients dZ^T X) are the tensor-core kernel of
// mlp_gemm_tc.cu, to FP32 accuracy.
//
//  * features_layer1_kernel: x = (sin az, cos az, sin el, cos el, ear) per row, and
//    z1 = W1 x + b1 (K = 5: one thread per output column, rows staged in shared memory).
//  * output_grad_kernel: dz4 = (g - t) / B * sigmoid(z4) and per-block loss partials.
//  * colsum_partial_kernel + split_reduce_kernel: bias gradients, column sums over row
//    chunks, then over the chunks, both in a fixed order.
//  * adam_kernel: the Adam update with host-computed bias corrections.
#include "kernels.h"

namespace hrir {

namespace {

__device__ __forceinline__ float sigmoid_f(float z)
{
    const float e = expf(-fabsf(z));
    return z >= 0.f ? 1.f / (1.f + e) : e / (1.f + e);
}

// z1[b][n] = b1[n] + sum_k W1[n][k] x_b[k] (skipped when z1 == nullptr); also writes x_b
// (5 features, row stride 8) to xs when xs != nullptr.  Rows: {az, el, ear} with ear = -1 (left) or +1 (right).
constexpr int kL1Rows = 16;
__global__ void __launch_bounds__(256) features_layer1_kernel(int n_rows, const float *__restrict__ dirs,
                                                              const float *__restrict__ W1,
                                                              const float *__restrict__ b1,
                                                              float *__restrict__ z1, int64_t ldz,
                                                              float *__restrict__ xs)
{
    __shared__ float x[kL1Rows][kMlpIn];
    const int64_t r0 = (int64_t)blockIdx.x * kL1Rows;
    const int t = threadIdx.x;
    if (t < kL1Rows && r0 + t < n_rows) {
        const float *d = dirs + (r0 + t) * 3;
        float sa, ca, se, ce;
        sincosf(d[0], &sa, &ca);
        sincosf(d[1], &se, &ce);
        x[t][0] = sa;
        x[t][1] = ca;
        x[t][2] = se;
        x[t][3] = ce;
        x[t][4] = d[2];
        if (xs) {
            float *o = xs + (r0 + t) * 8;
            for (int k = 0; k < kMlpIn; ++k) o[k] = x[t][k];
            for (int k = kMlpIn; k < 8; ++k) o[k] = 0.f;
        }
    }
    __syncthreads();
    if (!z1) return;
    for (int n = t; n < kMlpHidden; n += blockDim.x) {
        float w[kMlpIn];
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) w[k] = W1[n * kMlpIn + k];
        const float bias = b1[n];
        for (int r = 0; r < kL1Rows && r0 + r < n_rows; ++r) {
            float v = bias;
#pragma unroll
            for (int k = 0; k < kMlpIn; ++k) v = fmaf(w[k], x[r][k], v);
            z1[(r0 + r) * ldz + n] = v;
        }
    }
}

// dz[b][j] = (g[b][j] - t[b][j]) * inv_b * sigmoid(z4[b][j]); partial[block] = sum (g - t)^2
__global__ void __launch_bounds__(256) output_grad_kernel(int64_t n_rows, int refl_len,
                                                          const float *__restrict__ g,
                                                          const float *__restrict__ tgt,
                                                          const float *__restrict__ z4, int64_t ldz,
                                                          float inv_b, float *__restrict__ dz,
                                                          float *__restrict__ partial)
{
    __shared__ float red[256];
    const int64_t total = n_rows * refl_len;
    float s = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / refl_len;
        const int j = (int)(i - b * refl_len);
        const float d = g[i] - tgt[i];
        s = fmaf(d, d, s);
        dz[i] = d * inv_b * sigmoid_f(z4[b * ldz + j]);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// loss = 0.5 * inv_b * sum partial: one warp, lane l sums partials l, l + 32, .. in order
// (FP64), then a fixed butterfly across the lanes
__global__ void loss_final_kernel(const float *__restrict__ partial, int n, float inv_b,
                                  float *__restrict__ loss)
{
    const int lane = threadIdx.x;
    double s = 0.0;
    for (int i = lane; i < n; i += 32) s += partial[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) *loss = (float)(0.5 * inv_b * s);
}

// Column sums, first pass: block (x, y) sums rows [y rc, (y + 1) rc) of columns
// [32 x, 32 x + 32); warp w takes rows w, w + 8, .. of the chunk in order, then the 8 warp sums
// are added in warp order: P[y][n].  The second pass (split_reduce_kernel with M = 1) adds the
// chunks in order, so the result does not depend on the launch.
constexpr int kColsumWarps = 8;
__global__ void __launch_bounds__(256) colsum_partial_kernel(int64_t rows, int N, const float *__restrict__ D,
                                                             int64_t ldd, int64_t rc, float *__restrict__ P)
{
    __shared__ float red[kColsumWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int n = blockIdx.x * 32 + lane;
    const int64_t r0 = (int64_t)blockIdx.y * rc;
    const int64_t r1 = r0 + rc < rows ? r0 + rc : rows;
    float s = 0.f;
    if (n < N) {
        int64_t r = r0 + w;
        // four loads in flight, added in row order
        for (; r + 3 * kColsumWarps < r1; r += 4 * kColsumWarps) {
            const float a0 = D[r * ldd + n], a1 = D[(r + kColsumWarps) * ldd + n];
            const float a2 = D[(r + 2 * kColsumWarps) * ldd + n], a3 = D[(r + 3 * kColsumWarps) * ldd + n];
            s += a0;
            s += a1;
            s += a2;
            s += a3;
        }
        for (; r < r1; r += kColsumWarps) s += D[r * ldd + n];
    }
    red[w][lane] = s;
    __syncthreads();
    if (w == 0 && n < N) {
        float t = red[0][lane];
        for (int k = 1; k < kColsumWarps; ++k) t += red[k][lane];
        P[(int64_t)blockIdx.y * N + n] = t;
    }
}

// out[m][n] = sum_z P[z][m][n] (z in order)
__global__ void split_reduce_kernel(int splits, int M, int N, const float *__restrict__ P,
                                    float *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t MN = (int64_t)M * N;
    if (i >= MN) return;
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += P[z * MN + i];
    out[i] = s;
}

__global__ void adam_kernel(int64_t n, float *__restrict__ p, const float *__restrict__ g,
                            float *__restrict__ m, float *__restrict__ v, float lr, float b1,
                            float b2, float eps, float c1, float c2)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

}  // namespace

cudaError_t launch_features_layer1(int n_rows, const float *dirs, const float *W1, const float *b1,
                                   float *z1, int64_t ldz, float *xs, cudaStream_t st)
{
    if (n_rows <= 0) return cudaSuccess;
    features_layer1_kernel<<<(n_rows + kL1Rows - 1) / kL1Rows, 256, 0, st>>>(n_rows, dirs, W1, b1, z1,
                                                                              ldz, xs);
    return cudaGetLastError();
}

cudaError_t launch_output_grad(int64_t n_rows, int refl_len, const float *g, const float *tgt,
                               const float *z4, int64_t ldz, float inv_b, float *dz, float *partial,
                               int n_partial, float *loss, cudaStream_t st)
{
    output_grad_kernel<<<n_partial, 256, 0, st>>>(n_rows, refl_len, g, tgt, z4, ldz, inv_b, dz, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !loss) return e;
    loss_final_kernel<<<1, 32, 0, st>>>(partial, n_partial, inv_b, loss);
    return cudaGetLastError();
}

cudaError_t launch_colsum(int64_t rows, int N, const float *D, int64_t ldd, float *P, float *out,
                          cudaStream_t st)
{
    if (N <= 0) return cudaSuccess;
    int64_t chunks = (rows + 255) / 256;
    chunks = chunks < 1 ? 1 : (chunks > kColsumMaxChunks ? kColsumMaxChunks : chunks);
    const int64_t rc = (rows + chunks - 1) / chunks;
    colsum_partial_kernel<<<dim3((unsigned)((N + 31) / 32), (unsigned)chunks), 32 * kColsumWarps, 0, st>>>(
        rows, N, D, ldd, rc, P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_split_reduce((int)chunks, 1, N, P, out, st);
}

cudaError_t launch_split_reduce(int splits, int M, int N, const float *P, float *out, cudaStream_t st)
{
    const int64_t MN = (int64_t)M * N;
    split_reduce_kernel<<<(unsigned)((MN + 255) / 256), 256, 0, st>>>(splits, M, N, P, out);
    return cudaGetLastError();
}

cudaError_t launch_adam(int64_t n, float *p, const float *g, float *m, float *v, float lr, float b1,
                        float b2, float eps, float c1, float c2, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    adam_kernel<<<(unsigned)blocks, 256, 0, st>>>(n, p, g, m, v, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace hrir
