/*
 * hrir_oracle.c -- TEST INFRASTRUCTURE ONLY (the oracle).
 *
 * A plain, slow, obviously-correct FP64 restatement of what the sparse factorized HRIR
 * rendering path computes, written from Luo, Zotkin & Duraiswami, "Sparse Head-Related
 * Impulse Response for Efficient Direct Convolution".  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library, and the CUDA library never calls it.
 *
 * Index conventions are 0-based throughout; the paper's 1-based footnote definitions are
 * shifted by one where noted.  All arithmetic is double precision; inputs that the GPU
 * receives in FP32 are passed here as FP32 and widened exactly to double.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared -o liboracle.so hrir_oracle.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------
 * Direct (time-domain) convolution, Sec. I footnote 2:
 *   (x*y)_i = sum_j x_j y_{i-j+1}  (1-based, zero padded)
 * which in 0-based indexing reads out[n] = sum_j x[j] * y[n-j], n = 0 .. nx+ny-2.
 * ---------------------------------------------------------------------------------- */
void orc_conv_direct(const double *x, int64_t nx, const double *y, int64_t ny, double *out)
{
    if (nx <= 0 || ny <= 0) return;
    int64_t n_out = nx + ny - 1;
    for (int64_t n = 0; n < n_out; ++n) {
        double acc = 0.0;
        for (int64_t j = 0; j < nx; ++j) {
            int64_t m = n - j;
            if (m < 0 || m >= ny) continue;
            acc += x[j] * y[m];
        }
        out[n] = acc;
    }
}

/* ------------------------------------------------------------------------------------
 * Convolution with a sparse reflection filter g of length refl_len given as k
 * (index, weight) pairs -- the same sum as the direct definition above with the zero
 * taps of g skipped (cost proportional to the number of non-zero entries, Sec. II and
 * Sec. IV-G):  out[n] = sum_t w[t] * y[n - idx[t]],  n = 0 .. ny+refl_len-2.
 * ---------------------------------------------------------------------------------- */
void orc_conv_sparse(const int32_t *idx, const double *w, int k, const double *y, int64_t ny,
                     int64_t refl_len, double *out)
{
    if (ny <= 0 || refl_len <= 0) return;
    int64_t n_out = ny + refl_len - 1;
    for (int64_t n = 0; n < n_out; ++n) {
        double acc = 0.0;
        for (int t = 0; t < k; ++t) {
            int64_t m = n - (int64_t)idx[t];
            if (m < 0 || m >= ny) continue;
            acc += w[t] * y[m];
        }
        out[n] = acc;
    }
}

/* ------------------------------------------------------------------------------------
 * Discrete Fourier transform.  Sec. I footnote 3 defines FFT convolution as
 * x*y = F^-1{ F{x} o F{y} }.  F is the DFT X[k] = sum_n x[n] exp(-2 pi i k n / P);
 * the inverse carries the 1/P factor.
 *
 * orc_dft: the O(P^2) definition, for checking the fast transform on small P.
 * orc_fft: iterative radix-2 Cooley-Tukey (decimation in time, bit-reversed input
 *          order), P a power of two; twiddles straight from cos/sin.
 * ---------------------------------------------------------------------------------- */
void orc_dft(const double *re, const double *im, int64_t n, int inverse, double *ore, double *oim)
{
    const double sgn = inverse ? 1.0 : -1.0;
    for (int64_t k = 0; k < n; ++k) {
        double ar = 0.0, ai = 0.0;
        for (int64_t t = 0; t < n; ++t) {
            /* reduce k*t mod n exactly before forming the angle */
            int64_t kt = (k * t) % n;
            double ang = sgn * 2.0 * M_PI * (double)kt / (double)n;
            double c = cos(ang), s = sin(ang);
            ar += re[t] * c - im[t] * s;
            ai += re[t] * s + im[t] * c;
        }
        ore[k] = inverse ? ar / (double)n : ar;
        oim[k] = inverse ? ai / (double)n : ai;
    }
}

int orc_fft(double *re, double *im, int64_t n, int inverse)
{
    if (n <= 0 || (n & (n - 1)) != 0) return -1;
    /* bit-reversal permutation */
    for (int64_t i = 1, j = 0; i < n; ++i) {
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double tr = re[i]; re[i] = re[j]; re[j] = tr;
            double ti = im[i]; im[i] = im[j]; im[j] = ti;
        }
    }
    const double sgn = inverse ? 1.0 : -1.0;
    for (int64_t len = 2; len <= n; len <<= 1) {
        int64_t half = len >> 1;
        for (int64_t j = 0; j < half; ++j) {
            double ang = sgn * 2.0 * M_PI * (double)j / (double)len;
            double wr = cos(ang), wi = sin(ang);
            for (int64_t s = 0; s < n; s += len) {
                int64_t a = s + j, b = s + j + half;
                double br = re[b] * wr - im[b] * wi;
                double bi = re[b] * wi + im[b] * wr;
                re[b] = re[a] - br; im[b] = im[a] - bi;
                re[a] = re[a] + br; im[a] = im[a] + bi;
            }
        }
    }
    if (inverse) {
        for (int64_t i = 0; i < n; ++i) { re[i] /= (double)n; im[i] /= (double)n; }
    }
    return 0;
}

/* FFT convolution (Sec. I footnote 3): zero-pad both operands to the power of two
 * P >= nx+ny-1, transform, multiply pointwise, invert, keep the first nx+ny-1 values. */
int orc_conv_fft(const double *x, int64_t nx, const double *y, int64_t ny, double *out)
{
    if (nx <= 0 || ny <= 0) return 0;
    int64_t n_out = nx + ny - 1, P = 1;
    while (P < n_out) P <<= 1;
    double *buf = (double *)calloc((size_t)(4 * P), sizeof(double));
    if (!buf) return -2;
    double *xr = buf, *xi = buf + P, *yr = buf + 2 * P, *yi = buf + 3 * P;
    memcpy(xr, x, (size_t)nx * sizeof(double));
    memcpy(yr, y, (size_t)ny * sizeof(double));
    orc_fft(xr, xi, P, 0);
    orc_fft(yr, yi, P, 0);
    for (int64_t k = 0; k < P; ++k) {
        double r = xr[k] * yr[k] - xi[k] * yi[k];
        double i = xr[k] * yi[k] + xi[k] * yr[k];
        xr[k] = r; xi[k] = i;
    }
    orc_fft(xr, xi, P, 1);
    memcpy(out, xr, (size_t)n_out * sizeof(double));
    free(buf);
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Binaural rendering of many sources through factorized HRIRs (Sec. II, Eqs. 1-2).
 *
 * Each direction d has, per ear e, a sparse non-negative reflection filter g_{d,e} of
 * length refl_len held as k_max (index, weight) slots of which nnz[d][e] are used, and
 * each ear has a direction-independent resonance filter f_e of length res_len.  The
 * HRIR is x_{d,e} = f_e * g_{d,e} (Eq. 1), of length H = res_len + refl_len - 1.
 * For sources y_s (s < S, length L, row stride ld) placed at directions dir[s]:
 *
 *     out_e = sum_s  y_s * x_{dir[s],e}          n = 0 .. L+H-2   (full linear conv)
 *
 * The three renderers below compute this same quantity three ways:
 *   orc_render_sparse : per source, the cascade of Eq. 2, (y*g)*f  (order 0)
 *                        or (y*f)*g (order 1), then summed over sources;
 *   orc_render_dense  : per source, y * x with x = f*g formed first (Eq. 1);
 *   orc_render_fft    : per source, FFT convolution (footnote 3) of y with x.
 * out is [2][out_ld] (ear-planar), overwritten on [0, L+H-1) of each row.
 * Returns 0, or -1 on a bad argument / direction id, -2 when out of memory.
 * ---------------------------------------------------------------------------------- */
static int check_render_args(int S, int64_t L, const int32_t *dir, int n_dirs, int k_max,
                             const uint16_t *idx, const uint8_t *nnz, int refl_len, int res_len)
{
    if (S < 0 || L < 0 || n_dirs <= 0 || k_max < 0 || refl_len <= 0 || res_len <= 0) return -1;
    for (int s = 0; s < S; ++s)
        if (dir[s] < 0 || dir[s] >= n_dirs) return -1;
    for (int64_t r = 0; r < (int64_t)n_dirs * 2; ++r) {
        if (nnz[r] > k_max) return -1;
        for (int t = 0; t < nnz[r]; ++t)
            if (idx[r * k_max + t] >= refl_len) return -1;
    }
    return 0;
}

/* gather the reflection taps of (direction d, ear e) as int32/double arrays */
static int load_taps(int d, int e, int k_max, const uint16_t *idx, const float *w,
                     const uint8_t *nnz, int32_t *ti, double *tw)
{
    int64_t row = (int64_t)d * 2 + e;
    int k = nnz[row];
    for (int t = 0; t < k; ++t) {
        ti[t] = idx[row * k_max + t];
        tw[t] = (double)w[row * k_max + t];
    }
    return k;
}

int orc_render_sparse(int S, int64_t L, const float *y, int64_t ld, const int32_t *dir, int n_dirs,
                      int k_max, const uint16_t *idx, const float *w, const uint8_t *nnz,
                      int refl_len, int res_len, const float *res, int order,
                      double *out, int64_t out_ld)
{
    if (check_render_args(S, L, dir, n_dirs, k_max, idx, nnz, refl_len, res_len)) return -1;
    int64_t H = (int64_t)res_len + refl_len - 1, n_out = L + H - 1;
    for (int e = 0; e < 2; ++e)
        for (int64_t n = 0; n < n_out; ++n) out[e * out_ld + n] = 0.0;
    if (L == 0) return 0;
    double *ys = (double *)malloc((size_t)L * sizeof(double));
    double *f = (double *)malloc((size_t)res_len * sizeof(double));
    double *t1 = (double *)malloc((size_t)(L + H) * sizeof(double));
    double *t2 = (double *)malloc((size_t)(L + H) * sizeof(double));
    int32_t *ti = (int32_t *)malloc((size_t)(k_max + 1) * sizeof(int32_t));
    double *tw = (double *)malloc((size_t)(k_max + 1) * sizeof(double));
    if (!ys || !f || !t1 || !t2 || !ti || !tw) {
        free(ys); free(f); free(t1); free(t2); free(ti); free(tw);
        return -2;
    }
    for (int s = 0; s < S; ++s) {
        for (int64_t n = 0; n < L; ++n) ys[n] = (double)y[(int64_t)s * ld + n];
        for (int e = 0; e < 2; ++e) {
            for (int l = 0; l < res_len; ++l) f[l] = (double)res[e * res_len + l];
            int k = load_taps(dir[s], e, k_max, idx, w, nnz, ti, tw);
            if (order == 0) {
                /* (y * g) * f */
                orc_conv_sparse(ti, tw, k, ys, L, refl_len, t1);          /* len L+refl_len-1 */
                orc_conv_direct(f, res_len, t1, L + refl_len - 1, t2);    /* len L+H-1 */
            } else {
                /* (y * f) * g */
                orc_conv_direct(f, res_len, ys, L, t1);                   /* len L+res_len-1 */
                orc_conv_sparse(ti, tw, k, t1, L + res_len - 1, refl_len, t2);
            }
            for (int64_t n = 0; n < n_out; ++n) out[e * out_ld + n] += t2[n];
        }
    }
    free(ys); free(f); free(t1); free(t2); free(ti); free(tw);
    return 0;
}

/* Dense HRIR of (direction d, ear e): x = f * g with g written out densely (Eq. 1). */
static void dense_hrir(int d, int e, int k_max, const uint16_t *idx, const float *w,
                       const uint8_t *nnz, int refl_len, int res_len, const float *res,
                       double *g, double *f, double *x)
{
    for (int j = 0; j < refl_len; ++j) g[j] = 0.0;
    int64_t row = (int64_t)d * 2 + e;
    for (int t = 0; t < nnz[row]; ++t) g[idx[row * k_max + t]] += (double)w[row * k_max + t];
    for (int l = 0; l < res_len; ++l) f[l] = (double)res[e * res_len + l];
    orc_conv_direct(f, res_len, g, refl_len, x);
}

/* kind 0: direct convolution with the dense HRIR; kind 1: FFT convolution with it */
static int render_with_hrir(int kind, int S, int64_t L, const float *y, int64_t ld,
                            const int32_t *dir, int n_dirs, int k_max, const uint16_t *idx,
                            const float *w, const uint8_t *nnz, int refl_len, int res_len,
                            const float *res, double *out, int64_t out_ld)
{
    if (check_render_args(S, L, dir, n_dirs, k_max, idx, nnz, refl_len, res_len)) return -1;
    int64_t H = (int64_t)res_len + refl_len - 1, n_out = L + H - 1;
    for (int e = 0; e < 2; ++e)
        for (int64_t n = 0; n < n_out; ++n) out[e * out_ld + n] = 0.0;
    if (L == 0) return 0;
    double *ys = (double *)malloc((size_t)L * sizeof(double));
    double *g = (double *)malloc((size_t)refl_len * sizeof(double));
    double *f = (double *)malloc((size_t)res_len * sizeof(double));
    double *x = (double *)malloc((size_t)H * sizeof(double));
    double *t = (double *)malloc((size_t)n_out * sizeof(double));
    if (!ys || !g || !f || !x || !t) {
        free(ys); free(g); free(f); free(x); free(t);
        return -2;
    }
    int rc = 0;
    for (int s = 0; s < S && rc == 0; ++s) {
        for (int64_t n = 0; n < L; ++n) ys[n] = (double)y[(int64_t)s * ld + n];
        for (int e = 0; e < 2; ++e) {
            dense_hrir(dir[s], e, k_max, idx, w, nnz, refl_len, res_len, res, g, f, x);
            if (kind == 0) orc_conv_direct(x, H, ys, L, t);
            else if (orc_conv_fft(x, H, ys, L, t) != 0) { rc = -2; break; }
            for (int64_t n = 0; n < n_out; ++n) out[e * out_ld + n] += t[n];
        }
    }
    free(ys); free(g); free(f); free(x); free(t);
    return rc;
}

int orc_render_dense(int S, int64_t L, const float *y, int64_t ld, const int32_t *dir, int n_dirs,
                     int k_max, const uint16_t *idx, const float *w, const uint8_t *nnz,
                     int refl_len, int res_len, const float *res, double *out, int64_t out_ld)
{
    return render_with_hrir(0, S, L, y, ld, dir, n_dirs, k_max, idx, w, nnz, refl_len, res_len,
                            res, out, out_ld);
}

int orc_render_fft(int S, int64_t L, const float *y, int64_t ld, const int32_t *dir, int n_dirs,
                   int k_max, const uint16_t *idx, const float *w, const uint8_t *nnz,
                   int refl_len, int res_len, const float *res, double *out, int64_t out_ld)
{
    return render_with_hrir(1, S, L, y, ld, dir, n_dirs, k_max, idx, w, nnz, refl_len, res_len,
                            res, out, out_ld);
}

/* Selected output samples of the same mix, straight from the cascade definition:
 *   out_e[n] = sum_s sum_{l < res_len} f_e[l] sum_t w_{dir s, e, t} y_s[n - l - i_{dir s, e, t}]
 * for the n_pos positions pos[] (any order; positions outside [0, L+H-1) give 0).
 * out is [2][n_pos].  Cost O(n_pos * S * res_len * k_max), independent of L. */
int orc_render_sparse_at(int S, int64_t L, const float *y, int64_t ld, const int32_t *dir,
                         int n_dirs, int k_max, const uint16_t *idx, const float *w,
                         const uint8_t *nnz, int refl_len, int res_len, const float *res,
                         const int64_t *pos, int64_t n_pos, double *out)
{
    if (check_render_args(S, L, dir, n_dirs, k_max, idx, nnz, refl_len, res_len)) return -1;
    for (int64_t p = 0; p < n_pos; ++p) {
        const int64_t n = pos[p];
        for (int e = 0; e < 2; ++e) {
            double acc = 0.0;
            for (int s = 0; s < S; ++s) {
                const int64_t row = (int64_t)dir[s] * 2 + e;
                for (int l = 0; l < res_len; ++l) {
                    double inner = 0.0;
                    for (int t = 0; t < nnz[row]; ++t) {
                        const int64_t m = n - l - (int64_t)idx[row * k_max + t];
                        if (m < 0 || m >= L) continue;
                        inner += (double)w[row * k_max + t] * (double)y[(int64_t)s * ld + m];
                    }
                    acc += (double)res[e * res_len + l] * inner;
                }
            }
            out[e * n_pos + p] = acc;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------------------
 * Top-K sparsification of non-negative reflection rows (the K-tap budget applied after
 * the sparsity-promoting fit of Sec. III-D and the small-tap discard of Sec. III-D).
 * For each row of g ([n_rows][refl_len], FP32 as the device sees it):
 *   candidates are the entries with value > 0 (NaN and negatives are never taps);
 *   keep the k largest, larger value first and the smaller index on equal values;
 *   emit the kept taps in ascending index order; pad unused slots with (0, 0.0);
 *   nnz = number of kept taps.
 * Plain repeated arg-max selection, then insertion sort by index.
 * ---------------------------------------------------------------------------------- */
int orc_topk(const float *g, int n_rows, int refl_len, int k, uint16_t *idx, float *w, uint8_t *nnz)
{
    if (n_rows < 0 || refl_len <= 0 || refl_len > 65535 || k < 0 || k > 255) return -1;
    char *taken = (char *)malloc((size_t)refl_len);
    if (!taken) return -2;
    for (int r = 0; r < n_rows; ++r) {
        const float *row = g + (int64_t)r * refl_len;
        uint16_t *ri = idx + (int64_t)r * k;
        float *rw = w + (int64_t)r * k;
        memset(taken, 0, (size_t)refl_len);
        int cnt = 0;
        for (; cnt < k; ++cnt) {
            int best = -1;
            for (int j = 0; j < refl_len; ++j) {
                double v = (double)row[j];
                if (taken[j] || !(v > 0.0)) continue;
                if (best < 0 || v > (double)row[best]) best = j;  /* strict: first index wins ties */
            }
            if (best < 0) break;
            taken[best] = 1;
            ri[cnt] = (uint16_t)best;
            rw[cnt] = row[best];
        }
        /* ascending index order */
        for (int a = 1; a < cnt; ++a) {
            uint16_t ki = ri[a]; float kw = rw[a];
            int b = a - 1;
            while (b >= 0 && ri[b] > ki) { ri[b + 1] = ri[b]; rw[b + 1] = rw[b]; --b; }
            ri[b + 1] = ki; rw[b + 1] = kw;
        }
        for (int t = cnt; t < k; ++t) { ri[t] = 0; rw[t] = 0.0f; }
        nnz[r] = (uint8_t)cnt;
    }
    free(taken);
    return 0;
}
