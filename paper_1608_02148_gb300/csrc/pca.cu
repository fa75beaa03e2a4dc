// Kernels of the randomized PCA (Algorithm rpca, Sec. 4.2) with the centring
// and scaling of the rpca() interface (Sec. 4.4) applied implicitly.
//
// The data matrix A (observations x variables) is never rewritten.  With
// centre mu and multipliers c_j = 1 / s_j the analysed matrix is
// X = (A - 1 mu^T) diag(c); every product with X is a product with A plus a
// rank-one correction:
//   X P   = A (diag(c) P) - 1 (mu^T diag(c) P)
//   X^T Y = diag(c) (A^T Y - mu (1^T Y))
// (or the transposed forms when the variables are the logical rows).  The
// kernels here compute the per-variable statistics in one pass over A, the
// small vectors h = P^T w of the corrections, and apply
// out_ij = r_i (out_ij - u_i h_j) to a pass result.
#include "internal.cuh"

#include <cuda_bf16.h>

namespace rsvdgb {
namespace {

constexpr int kRun = 16;  // observations accumulated in FP32 before an FP64 add

template <bool BF>
__device__ __forceinline__ float load_elem(const void* S, int64_t off)
{
    if constexpr (BF)
        return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(S)[off]);
    else
        return reinterpret_cast<const float*>(S)[off];
}

// Four consecutive elements (16-byte FP32 or 8-byte BF16 vector load).
template <bool BF>
__device__ __forceinline__ void load4(const void* S, int64_t off, float v[4])
{
    if constexpr (BF) {
        const uint2 w = *reinterpret_cast<const uint2*>(reinterpret_cast<const __nv_bfloat16*>(S) + off);
        v[0] = __uint_as_float(w.x << 16);
        v[1] = __uint_as_float(w.x & 0xFFFF0000u);
        v[2] = __uint_as_float(w.y << 16);
        v[3] = __uint_as_float(w.y & 0xFFFF0000u);
    } else {
        const float4 w = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(S) + off);
        v[0] = w.x;
        v[1] = w.y;
        v[2] = w.z;
        v[3] = w.w;
    }
}

// Statistics of the stored columns (variables = columns of the stored
// row-major matrix S, rows x cols).  Thread t of block (bx, by) owns columns
// [c0, c0 + VEC) and the row chunk by; it sums d = a - x0 and d^2 about the
// column's first element x0 in FP32 runs of kRun rows, then in FP64, and
// writes (s1, s2) to part[by * cols + c].
template <bool BF, int VEC>
__global__ void __launch_bounds__(128) colstats_kernel(const void* __restrict__ S, int64_t lda, int64_t rows,
                                                       int64_t cols, int64_t rows_per_chunk,
                                                       double2* __restrict__ part)
{
    const int64_t c0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * VEC;
    if (c0 >= cols) return;
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
    const int64_t r1 = min(rows, r0 + rows_per_chunk);
    const bool full = (c0 + VEC <= cols);
    float x0[VEC];
    for (int v = 0; v < VEC; ++v) x0[v] = (c0 + v < cols) ? load_elem<BF>(S, c0 + v) : 0.f;
    double s1[VEC], s2[VEC];
    for (int v = 0; v < VEC; ++v) s1[v] = s2[v] = 0.0;
    for (int64_t r = r0; r < r1; r += kRun) {
        float a1[VEC], a2[VEC];
        for (int v = 0; v < VEC; ++v) a1[v] = a2[v] = 0.f;
        const int64_t re = min(r1, r + kRun);
        if (VEC == 4 && full && re - r == kRun) {
#pragma unroll
            for (int t = 0; t < kRun; ++t) {
                float x[4];
                load4<BF>(S, (r + t) * lda + c0, x);
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float d = x[v] - x0[v];
                    a1[v] += d;
                    a2[v] = fmaf(d, d, a2[v]);
                }
            }
        } else {
            for (int64_t i = r; i < re; ++i)
                for (int v = 0; v < VEC; ++v)
                    if (c0 + v < cols) {
                        const float d = load_elem<BF>(S, i * lda + c0 + v) - x0[v];
                        a1[v] += d;
                        a2[v] = fmaf(d, d, a2[v]);
                    }
        }
        for (int v = 0; v < VEC; ++v) {
            s1[v] += (double)a1[v];
            s2[v] += (double)a2[v];
        }
    }
    for (int v = 0; v < VEC; ++v)
        if (c0 + v < cols) part[(int64_t)blockIdx.y * cols + c0 + v] = make_double2(s1[v], s2[v]);
}

// Statistics of the stored rows (variables = rows of S): one block per row,
// sums about the row's first element, block reduction in FP64.
template <bool BF, bool VEC4>
__global__ void __launch_bounds__(256) rowstats_kernel(const void* __restrict__ S, int64_t lda, int64_t cols,
                                                       double2* __restrict__ part)
{
    const int64_t row = blockIdx.x;
    const int64_t base = row * lda;
    const float x0 = load_elem<BF>(S, base);
    double s1 = 0.0, s2 = 0.0;
    float a1 = 0.f, a2 = 0.f;
    int run = 0;
    if (VEC4) {
        const int64_t nv = cols / 4;
        for (int64_t v = threadIdx.x; v < nv; v += blockDim.x) {
            float x[4];
            load4<BF>(S, base + 4 * v, x);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float d = x[e] - x0;
                a1 += d;
                a2 = fmaf(d, d, a2);
            }
            if (++run == kRun / 4) {
                s1 += a1;
                s2 += a2;
                a1 = a2 = 0.f;
                run = 0;
            }
        }
        for (int64_t c = 4 * nv + threadIdx.x; c < cols; c += blockDim.x) {
            const float d = load_elem<BF>(S, base + c) - x0;
            a1 += d;
            a2 = fmaf(d, d, a2);
        }
    } else {
        for (int64_t c = threadIdx.x; c < cols; c += blockDim.x) {
            const float d = load_elem<BF>(S, base + c) - x0;
            a1 += d;
            a2 = fmaf(d, d, a2);
            if (++run == kRun) {
                s1 += a1;
                s2 += a2;
                a1 = a2 = 0.f;
                run = 0;
            }
        }
    }
    s1 += a1;
    s2 += a2;
    __shared__ double r1[8], r2[8];
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        r1[warp] = s1;
        r2[warp] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t1 += r1[w];
            t2 += r2[w];
        }
        part[row] = make_double2(t1, t2);
    }
}

// Per-variable centre and multiplier from the partial sums (chunks x nvar),
// the shifts x0 read again from S, and each block's share of ||X||_F^2.
// Block: 32 variables (lane = variable); warp w sums the chunks c = w mod 8,
// the eight warp sums are added in a fixed order.
//   mean = x0 + s1 / m,  SS = sum (a - mean)^2 = s2 - s1^2 / m
//   centre: mu = mean (or 0);  scale: s = sqrt(SS / (m - 1)) with the centring,
//   sqrt(sum a^2 / (m - 1)) without it; c = 1 / s (0 for s = 0) or 1.
template <bool BF>
__global__ void __launch_bounds__(256) stats_finalize_kernel(const void* __restrict__ S, int64_t shift_stride,
                                                             const double2* __restrict__ part, int chunks,
                                                             int64_t nvar, int64_t m_obs, int center, int scale,
                                                             float* __restrict__ mu, float* __restrict__ cmul,
                                                             float* __restrict__ center_out,
                                                             float* __restrict__ scale_out,
                                                             double* __restrict__ fro2_part)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t j = (int64_t)blockIdx.x * 32 + lane;
    __shared__ double r1[8][32], r2[8][32];
    {
        double a1 = 0.0, a2 = 0.0;
        if (j < nvar)
            for (int c = warp; c < chunks; c += 8) {
                const double2 p = part[(int64_t)c * nvar + j];
                a1 += p.x;
                a2 += p.y;
            }
        r1[warp][lane] = a1;
        r2[warp][lane] = a2;
    }
    __syncthreads();
    if (warp != 0) return;
    double f2 = 0.0;
    if (j < nvar) {
        double s1 = 0.0, s2 = 0.0;
        for (int w = 0; w < 8; ++w) {
            s1 += r1[w][lane];
            s2 += r2[w][lane];
        }
        const double x0 = (double)load_elem<BF>(S, j * shift_stride);
        const double m = (double)m_obs;
        const double mean = x0 + s1 / m;
        const double ss = fmax(s2 - s1 * s1 / m, 0.0);
        // sum a^2 = sum (x0 + d)^2 = m x0^2 + 2 x0 s1 + s2
        const double sq = fmax(m * x0 * x0 + 2.0 * x0 * s1 + s2, 0.0);
        const double spread = center ? ss : sq;  // sum of squares of the (centred) column
        double s = 1.0, c = 1.0;
        if (scale) {
            s = sqrt(spread / (m - 1.0));
            c = (s > 0.0) ? 1.0 / s : 0.0;
        }
        mu[j] = center ? (float)mean : 0.f;
        cmul[j] = (float)c;
        if (center_out) center_out[j] = center ? (float)mean : 0.f;
        if (scale_out) scale_out[j] = scale ? (float)s : 1.f;
        const double cf = (double)(float)c;
        f2 = spread * cf * cf;
    }
    for (int o = 16; o > 0; o >>= 1) f2 += __shfl_xor_sync(0xffffffffu, f2, o);
    if (lane == 0) fro2_part[blockIdx.x] = f2;
}

__global__ void sum_doubles_kernel(const double* __restrict__ part, int count, double* __restrict__ out)
{
    double t = 0.0;
    for (int i = threadIdx.x; i < count; i += 32) t += part[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) *out = t;
}

// part[s * l + j] = sum over rows i of chunk s of X_ij w_i (w null: 1);
// X column-major (ld).  FP32 runs of 8 products, FP64 across runs and lanes.
__global__ void __launch_bounds__(256) affine_dot_kernel(const float* __restrict__ X, int64_t ld, int64_t rows,
                                                         int l, const float* __restrict__ w, int64_t rows_per_chunk,
                                                         double* __restrict__ part)
{
    const int j = blockIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
    const int64_t r1 = min(rows, r0 + rows_per_chunk);
    const float* x = X + (int64_t)j * ld;
    double acc = 0.0;
    // four independent FP32 runs of (at most) 8 terms each, then FP64
    const int64_t step = blockDim.x;
    int64_t i = r0 + threadIdx.x;
    for (; i + 3 * step < r1; i += 32 * step) {
        float run[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int t = 0; t < 8; ++t)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int64_t ii = i + (int64_t)(4 * t + q) * step;
                if (ii < r1) run[q] = w ? fmaf(x[ii], w[ii], run[q]) : run[q] + x[ii];
            }
        acc += (double)run[0] + (double)run[1] + (double)run[2] + (double)run[3];
    }
    for (; i < r1; i += step) acc += w ? (double)(x[i] * w[i]) : (double)x[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        part[(int64_t)blockIdx.y * l + j] = t;
    }
}

// h[j] = sum over the chunk partials of column j (fixed order), for the
// pass epilogue that applies the correction.
__global__ void affine_h_kernel(const double* __restrict__ part, int chunks, int l, float* __restrict__ h)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= l) return;
    double t = 0.0;
    for (int c = 0; c < chunks; ++c) t += part[(int64_t)c * l + j];
    h[j] = (float)t;
}

__device__ __forceinline__ void split_tf32(float x, float& h, float& r)
{
    uint32_t hb, rb;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(x));
    h = __uint_as_float(hb);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(rb) : "f"(x - h));
    r = __uint_as_float(rb);
}

// out_ij = r_i (out_ij - u_i h_j) for i < rows, j < l (column-major, ld),
// h_j = sum of the `chunks` partials of column j (no shift when part is
// null; u null: 1; r null: 1).  hi/lo (optional) receive the TF32 split of
// the result.  Block (bx, j): 1024 rows of column j, 4 per thread (strided
// by the block size, so that each load is coalesced).
__global__ void __launch_bounds__(256) affine_post_kernel(float* __restrict__ out, int64_t ld, int64_t rows, int l,
                                                          const float* __restrict__ r, const float* __restrict__ u,
                                                          const double* __restrict__ part, int chunks,
                                                          float* __restrict__ hi, float* __restrict__ lo)
{
    const int j = blockIdx.y;
    __shared__ float hj;
    if (threadIdx.x < 32) {
        double t = 0.0;
        if (part)
            for (int c = threadIdx.x; c < chunks; c += 32) t += part[(int64_t)c * l + j];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) hj = (float)t;
    }
    __syncthreads();
    const float h = hj;
    const int64_t i0 = (int64_t)blockIdx.x * (4 * blockDim.x) + threadIdx.x;
    float* col = out + (int64_t)j * ld;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int64_t i = i0 + (int64_t)e * blockDim.x;
        if (i >= rows) break;
        float v = col[i];
        if (part) v = fmaf(-(u ? u[i] : 1.f), h, v);
        if (r) v *= r[i];
        col[i] = v;
        if (hi) {
            float a, b;
            split_tf32(v, a, b);
            hi[(int64_t)j * ld + i] = a;
            lo[(int64_t)j * ld + i] = b;
        }
    }
}

// out_ij = r_i in_ij (i < rows, j < l; column-major, ld; in == out allowed),
// with the optional TF32 split of the result; the padding (rows up to ld,
// columns up to l_pad) is written as zero.
__global__ void __launch_bounds__(256) scale_rows_kernel(const float* in, int64_t ld, int64_t rows, int l,
                                                         const float* __restrict__ r, float* out,
                                                         float* __restrict__ hi, float* __restrict__ lo)
{
    const int j = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ld) return;
    const int64_t o = (int64_t)j * ld + i;
    const float v = (i < rows && j < l) ? in[o] * r[i] : 0.f;
    out[o] = v;
    if (hi) {
        float a, b;
        split_tf32(v, a, b);
        hi[o] = a;
        lo[o] = b;
    }
}

// T[i * l + c] *= sigma[c] for c < ncols (l x l row-major small factor).
__global__ void scale_cols_small_kernel(float* __restrict__ T, int l, int ncols, const float* __restrict__ sigma)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (c < ncols) T[i * l + c] *= sigma[c];
}

// Lambda = Sigma^2 / (m - 1) and the standard deviations sqrt(Lambda)
// (Algorithm rpca step 2).
__global__ void pca_values_kernel(const float* __restrict__ sigma, int k, int64_t m_obs, float* __restrict__ eig,
                                  float* __restrict__ sdev)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= k) return;
    const double s = (double)sigma[c];
    const double den = (double)(m_obs - 1);
    eig[c] = (float)(s * s / den);
    if (sdev) sdev[c] = (float)(s / sqrt(den));
}

}  // namespace

int64_t stats_chunks(bool vars_are_cols, int64_t rows_s, int64_t cols_s, int sm_count)
{
    if (!vars_are_cols) return 1;
    // about eight 128-thread blocks per SM
    const int64_t cblocks = ceil_div(cols_s, 128 * 4);
    int64_t chunks = ceil_div(8 * (int64_t)sm_count, cblocks);
    chunks = std::min<int64_t>(chunks, ceil_div(rows_s, kRun));
    return std::max<int64_t>(chunks, 1);
}

void launch_var_stats(cudaStream_t s, int sm_count, const void* S, int64_t lda, int64_t rows_s, int64_t cols_s,
                      int a_bf16, bool vars_are_cols, int center, int scale, double2* part, float* mu, float* cmul,
                      float* center_out, float* scale_out, double* fro2_part, double* fro2)
{
    const int64_t chunks = stats_chunks(vars_are_cols, rows_s, cols_s, sm_count);
    const size_t esz = a_bf16 ? 2 : 4;
    const bool vec = (lda % 4 == 0) && ((uintptr_t)S % (4 * esz) == 0);
    if (vars_are_cols) {
        const int64_t rpc = round_up(ceil_div(rows_s, chunks), kRun);
        const int vecw = vec ? 4 : 1;
        const dim3 grid((unsigned)ceil_div(cols_s, 128 * vecw), (unsigned)ceil_div(rows_s, rpc));
        if (a_bf16) {
            if (vec)
                colstats_kernel<true, 4><<<grid, 128, 0, s>>>(S, lda, rows_s, cols_s, rpc, part);
            else
                colstats_kernel<true, 1><<<grid, 128, 0, s>>>(S, lda, rows_s, cols_s, rpc, part);
        } else {
            if (vec)
                colstats_kernel<false, 4><<<grid, 128, 0, s>>>(S, lda, rows_s, cols_s, rpc, part);
            else
                colstats_kernel<false, 1><<<grid, 128, 0, s>>>(S, lda, rows_s, cols_s, rpc, part);
        }
        count_launches();
        const int used = (int)grid.y;
        const int64_t nvar = cols_s;
        const unsigned fb = (unsigned)ceil_div(nvar, 32);
        if (a_bf16)
            stats_finalize_kernel<true><<<fb, 256, 0, s>>>(S, 1, part, used, nvar, rows_s, center, scale, mu, cmul,
                                                           center_out, scale_out, fro2_part);
        else
            stats_finalize_kernel<false><<<fb, 256, 0, s>>>(S, 1, part, used, nvar, rows_s, center, scale, mu, cmul,
                                                            center_out, scale_out, fro2_part);
        count_launches();
        sum_doubles_kernel<<<1, 32, 0, s>>>(fro2_part, (int)fb, fro2);
        count_launches();
        return;
    }
    const unsigned nb = (unsigned)rows_s;
    if (a_bf16) {
        if (vec)
            rowstats_kernel<true, true><<<nb, 256, 0, s>>>(S, lda, cols_s, part);
        else
            rowstats_kernel<true, false><<<nb, 256, 0, s>>>(S, lda, cols_s, part);
    } else {
        if (vec)
            rowstats_kernel<false, true><<<nb, 256, 0, s>>>(S, lda, cols_s, part);
        else
            rowstats_kernel<false, false><<<nb, 256, 0, s>>>(S, lda, cols_s, part);
    }
    count_launches();
    const int64_t nvar = rows_s;
    const unsigned fb = (unsigned)ceil_div(nvar, 32);
    if (a_bf16)
        stats_finalize_kernel<true><<<fb, 256, 0, s>>>(S, lda, part, 1, nvar, cols_s, center, scale, mu, cmul,
                                                       center_out, scale_out, fro2_part);
    else
        stats_finalize_kernel<false><<<fb, 256, 0, s>>>(S, lda, part, 1, nvar, cols_s, center, scale, mu, cmul,
                                                        center_out, scale_out, fro2_part);
    count_launches();
    sum_doubles_kernel<<<1, 32, 0, s>>>(fro2_part, (int)fb, fro2);
    count_launches();
}

int affine_chunks(int64_t rows, int l, int sm_count)
{
    // about eight 256-thread blocks per SM
    int64_t c = ceil_div(8 * (int64_t)sm_count, std::max(l, 1));
    c = std::min<int64_t>(c, ceil_div(rows, 1024));
    return (int)std::max<int64_t>(std::min<int64_t>(c, kAffineMaxChunks), 1);
}

void launch_affine_dot(cudaStream_t s, int sm_count, const float* X, int64_t ld, int64_t rows, int l, const float* w,
                       double* part, int* chunks_out)
{
    const int chunks = affine_chunks(rows, l, sm_count);
    const int64_t rpc = ceil_div(rows, chunks);
    affine_dot_kernel<<<dim3((unsigned)l, (unsigned)chunks), 256, 0, s>>>(X, ld, rows, l, w, rpc, part);
    count_launches();
    *chunks_out = chunks;
}

void launch_affine_h(cudaStream_t s, const double* part, int chunks, int l, float* h)
{
    affine_h_kernel<<<(unsigned)ceil_div(l, 128), 128, 0, s>>>(part, chunks, l, h);
    count_launches();
}

void launch_affine_post(cudaStream_t s, float* out, int64_t ld, int64_t rows, int l, const float* r, const float* u,
                        const double* part, int chunks, float* hi, float* lo)
{
    const dim3 grid((unsigned)ceil_div(rows, 1024), (unsigned)l);
    affine_post_kernel<<<grid, 256, 0, s>>>(out, ld, rows, l, r, u, part, chunks, hi, lo);
    count_launches();
}

void launch_scale_rows(cudaStream_t s, const float* in, int64_t ld, int64_t rows, int l, int l_pad, const float* r,
                       float* out, float* hi, float* lo)
{
    const dim3 grid((unsigned)ceil_div(ld, 256), (unsigned)l_pad);
    scale_rows_kernel<<<grid, 256, 0, s>>>(in, ld, rows, l, r, out, hi, lo);
    count_launches();
}

void launch_scale_cols_small(cudaStream_t s, float* T, int l, int ncols, const float* sigma)
{
    if (ncols <= 0) return;
    scale_cols_small_kernel<<<dim3((unsigned)ceil_div(ncols, 128), (unsigned)l), 128, 0, s>>>(T, l, ncols, sigma);
    count_launches();
}

void launch_pca_values(cudaStream_t s, const float* sigma, int k, int64_t m_obs, float* eig, float* sdev)
{
    pca_values_kernel<<<(unsigned)ceil_div(k, 128), 128, 0, s>>>(sigma, k, m_obs, eig, sdev);
    count_launches();
}

}  // namespace rsvdgb
