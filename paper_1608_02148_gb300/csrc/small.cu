// Small l x l kernels of the orthonormalisation and of the SVD of B.
//
//  * chol_inv      -- Cholesky G = R^T R of a Gram matrix and R^{-1}, the
//                     factor step of CholeskyQR (the "qr" of Algorithm
//                     sub_iterations and Algorithm rqb step 9).
//  * jacobi_svd    -- one-sided (Hestenes) Jacobi SVD, the deterministic SVD
//                     of the small matrix in Algorithm rSVD step 2.
//  * small helpers -- l x l products, transposes, layout changes, the
//                     finishing kernel that writes d and rsvdgb_info.
//
// Precision: these kernels compute in FP32 with FP64 Gram inputs.  GB300's
// FP64 pipe is far slower than its FP32 pipe, and the Gram matrices they
// factor carry FP32-level error already, so FP64 here would not change the
// result beyond that error; CholeskyQR2 recovers orthogonality to FP32 level.
#include <math.h>

#include "internal.cuh"

namespace rsvdgb {
namespace {

constexpr int kSmallThreads = 1024;

// ---------------------------------------------------------------------------
// Cholesky by symmetric Gaussian elimination on [G | I].
//
// Step j scales pivot row j by 1/sqrt(pivot) and eliminates column j from the
// rows below.  The G half turns into R (upper triangle) and the I half into
// R^{-T} (lower triangle), so R^{-1} = (R^{-T})^T comes out of the same l
// steps.  Both halves share one l x l array: R in the upper triangle
// including the diagonal, R^{-T} strictly below it, its diagonal in dinv.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSmallThreads)
    chol_inv_kernel(const double* __restrict__ G, int l, float shift_rel, float* __restrict__ R,
                    float* __restrict__ T, int* status, int* breakdowns)
{
    extern __shared__ float S[];  // l * l
    __shared__ float dinv[256];
    __shared__ float piv;
    __shared__ float maxdiag;
    __shared__ int broke;
    const int tid = threadIdx.x;
    const int nth = blockDim.x;

    if (tid == 0) {
        float md = 0.f;
        for (int a = 0; a < l; ++a) md = fmaxf(md, (float)G[a * l + a]);
        maxdiag = md;
        broke = 0;
    }
    __syncthreads();

    for (int attempt = 0; attempt < 4; ++attempt) {
        // shift = shift_rel * max diag on the first attempt; after a breakdown
        // the shift grows by 100x per retry (shifted CholeskyQR).
        float shift = shift_rel * maxdiag;
        if (attempt > 0) shift = fmaxf(shift, maxdiag * 1e-6f * powf(100.f, (float)(attempt - 1)));
        for (int e = tid; e < l * l; e += nth) {
            const int a = e / l, b = e % l;
            float v;
            if (b >= a)
                v = (float)G[a * l + b] + (a == b ? shift : 0.f);
            else
                v = 0.f;  // the I half starts as the identity (diagonal kept in dinv)
            S[e] = v;
        }
        __syncthreads();
        bool failed = false;
        for (int j = 0; j < l; ++j) {
            if (tid == 0) {
                const float p = S[j * l + j];
                if (!(p > 0.f) || !isfinite(p)) {
                    broke = 1;
                    piv = 1.f;
                } else {
                    piv = sqrtf(p);
                }
            }
            __syncthreads();
            if (broke) {
                failed = true;
                break;
            }
            const float r = piv;
            const float rinv = 1.0f / r;
            for (int c = tid; c < l; c += nth) {
                if (c == j)
                    S[j * l + j] = r;
                else
                    S[j * l + c] *= rinv;  // c > j: R(j,c); c < j: R^{-T}(j,c)
            }
            if (tid == 0) dinv[j] = rinv;
            __syncthreads();
            // eliminate column j from rows a > j
            const int rows = l - j - 1;
            for (int e = tid; e < rows * l; e += nth) {
                const int a = j + 1 + e / l;
                const int b = e % l;
                const float mult = S[j * l + a];  // R(j, a)
                if (b >= a) {
                    S[a * l + b] -= mult * S[j * l + b];
                } else if (b <= j) {
                    const float lj = (b == j) ? dinv[j] : S[j * l + b];
                    S[a * l + b] -= mult * lj;
                }
            }
            __syncthreads();
        }
        if (!failed) break;
        __syncthreads();
        if (tid == 0) {
            broke = 0;
            if (breakdowns) atomicAdd(breakdowns, 1);
            if (attempt == 3 && status) *status = RSVDGB_ERR_BREAKDOWN;
        }
        __syncthreads();
    }
    for (int e = tid; e < l * l; e += nth) {
        const int a = e / l, b = e % l;
        if (R) R[e] = (b >= a) ? S[e] : 0.f;
        // T = R^{-1} = (R^{-T})^T: T(a, b) = R^{-T}(b, a) for a <= b
        float t = 0.f;
        if (a == b)
            t = dinv[a];
        else if (a < b)
            t = S[b * l + a];
        T[e] = t;
    }
}

__global__ void small_matmul_kernel(const float* __restrict__ A, const float* __restrict__ B, float* __restrict__ C,
                                    int l)
{
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= l || j >= l) return;
    float acc = 0.f;
    for (int t = 0; t < l; ++t) acc = fmaf(A[i * l + t], B[t * l + j], acc);
    C[i * l + j] = acc;
}

__global__ void small_d2f_kernel(const double* __restrict__ in, float* __restrict__ out, int l, int transpose)
{
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= l || j >= l) return;
    out[transpose ? j * l + i : i * l + j] = (float)in[i * l + j];
}

__global__ void small_transpose_kernel(const float* __restrict__ in, float* __restrict__ out, int l)
{
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= l || j >= l) return;
    out[j * l + i] = in[i * l + j];
}

// ---------------------------------------------------------------------------
// One-sided Jacobi SVD of an l x l matrix, parallel (round-robin) ordering:
// in each of the L-1 rounds of a sweep the L/2 disjoint column pairs are
// rotated at once, one warp per pair.  Columns live column-major in Mc and Jc
// (shared memory when they fit, else the global work buffer).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kSmallThreads)
    jacobi_kernel(const float* __restrict__ M, int l, int L, float* __restrict__ sigma, float* __restrict__ Ut,
                  float* __restrict__ Jt, float* __restrict__ gwork, int use_smem)
{
    extern __shared__ float sm[];
    float* Mc = use_smem ? sm : gwork;
    float* Jc = use_smem ? sm + (size_t)L * L : gwork + (size_t)L * L;
    __shared__ int rotated;
    __shared__ float sv[256];
    __shared__ int rank[256];
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;

    // column-major copies, zero padded to L x L
    for (int e = tid; e < L * L; e += blockDim.x) {
        const int c = e / L, i = e % L;
        Mc[e] = (i < l && c < l) ? M[i * l + c] : 0.f;
        Jc[e] = (i == c) ? 1.f : 0.f;
    }
    __syncthreads();

    const float tol = 3e-7f;
    for (int sweep = 0; sweep < 40; ++sweep) {
        if (tid == 0) rotated = 0;
        __syncthreads();
        for (int round = 0; round < L - 1; ++round) {
            for (int t = warp; t < L / 2; t += nwarps) {
                int a, b;
                if (t == 0) {
                    a = L - 1;
                    b = round;
                } else {
                    a = (round + t) % (L - 1);
                    b = (round - t + L - 1) % (L - 1);
                }
                float* ma = Mc + (size_t)a * L;
                float* mb = Mc + (size_t)b * L;
                float al = 0.f, be = 0.f, ga = 0.f;
                for (int i = lane; i < L; i += 32) {
                    const float x = ma[i], y = mb[i];
                    al = fmaf(x, x, al);
                    be = fmaf(y, y, be);
                    ga = fmaf(x, y, ga);
                }
                al = warp_sum(al);
                be = warp_sum(be);
                ga = warp_sum(ga);
                if (ga != 0.f && fabsf(ga) > tol * sqrtf(al * be)) {
                    const float zeta = (be - al) / (2.f * ga);
                    const float tt = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
                    const float c = 1.0f / sqrtf(1.f + tt * tt);
                    const float s = c * tt;
                    for (int i = lane; i < L; i += 32) {
                        const float x = ma[i], y = mb[i];
                        ma[i] = c * x - s * y;
                        mb[i] = s * x + c * y;
                    }
                    float* ja = Jc + (size_t)a * L;
                    float* jb = Jc + (size_t)b * L;
                    for (int i = lane; i < L; i += 32) {
                        const float x = ja[i], y = jb[i];
                        ja[i] = c * x - s * y;
                        jb[i] = s * x + c * y;
                    }
                    if (lane == 0) rotated = 1;
                }
            }
            __syncthreads();
        }
        if (!rotated) break;
        __syncthreads();
    }
    // Singular values.  A rotation computed in FP32 is orthogonal only to
    // rounding, so after many rotations a column of W = M J and the matching
    // column of J carry the same small scale drift; sigma_c = ||W_c|| / ||J_c||
    // cancels it, and J_c is renormalised.
    __shared__ float jn[256];
    __shared__ float wn[256];
    for (int c = warp; c < L; c += nwarps) {
        float s2 = 0.f, j2 = 0.f;
        for (int i = lane; i < L; i += 32) {
            s2 = fmaf(Mc[(size_t)c * L + i], Mc[(size_t)c * L + i], s2);
            j2 = fmaf(Jc[(size_t)c * L + i], Jc[(size_t)c * L + i], j2);
        }
        s2 = warp_sum(s2);
        j2 = warp_sum(j2);
        if (lane == 0) {
            wn[c] = sqrtf(s2);
            jn[c] = sqrtf(j2);
            sv[c] = (j2 > 0.f) ? sqrtf(s2) / sqrtf(j2) : 0.f;
        }
    }
    __syncthreads();
    for (int c = tid; c < L; c += blockDim.x) {
        int r = 0;
        for (int o = 0; o < L; ++o) r += (sv[o] > sv[c]) || (sv[o] == sv[c] && o < c);
        rank[c] = r;
    }
    __syncthreads();
    for (int e = tid; e < L * L; e += blockDim.x) {
        const int c = e / L, i = e % L;
        const int r = rank[c];
        if (r >= l || i >= l) continue;
        const float w = wn[c];
        Ut[i * l + r] = (w > 0.f) ? Mc[(size_t)c * L + i] / w : 0.f;
        Jt[i * l + r] = (jn[c] > 0.f) ? Jc[(size_t)c * L + i] / jn[c] : 0.f;
    }
    for (int c = tid; c < L; c += blockDim.x)
        if (rank[c] < l) sigma[rank[c]] = sv[c];
}

__global__ void finalize_info_kernel(const float* __restrict__ sigma, int l, int k, float* __restrict__ d,
                                     const double* fro2A, const int* status, const int* breakdowns, int q,
                                     int p_used, rsvdgb_info* info)
{
    const int tid = threadIdx.x;
    if (d && sigma)
        for (int i = tid; i < k; i += blockDim.x) d[i] = sigma[i];
    if (tid == 0 && info) {
        double sb = 0.0, sk = 0.0;
        for (int i = 0; sigma && i < l; ++i) {
            const double s = (double)sigma[i];
            sb += s * s;
            if (i < k) sk += s * s;
        }
        const double fa = fro2A ? *fro2A : 0.0;
        int st = status ? *status : 0;
        if (!isfinite(fa)) st = RSVDGB_ERR_NONFINITE;
        info->status = st;
        info->q_used = q;
        info->p_used = p_used;
        info->l = l;
        info->fro2_A = fa;
        info->fro2_B = sb;
        info->err2_QB = fa - sb;
        info->err2_k = fa - sk;
        info->breakdowns = breakdowns ? *breakdowns : 0;
    }
}

__global__ void clear_scalars_kernel(int* status, int* breakdowns, double* fro2)
{
    if (status) *status = 0;
    if (breakdowns) *breakdowns = 0;
    if (fro2) *fro2 = 0.0;
}

__global__ void split_tf32_kernel(const float* __restrict__ in, int64_t ld, int64_t rows, int l, int l_pad,
                                  float* __restrict__ hi, float* __restrict__ lo)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= ld || j >= l_pad) return;
    const int64_t o = (int64_t)j * ld + i;
    float h = 0.f, r = 0.f;
    if (i < rows && j < l) {
        const float x = in[o];
        uint32_t hb, rb;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(x));
        h = __uint_as_float(hb);
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(rb) : "f"(x - h));
        r = __uint_as_float(rb);
    }
    hi[o] = h;
    lo[o] = r;
}

__global__ void col_to_row_kernel(const float* __restrict__ in, int64_t ld, int64_t rows, int cols,
                                  float* __restrict__ out, int64_t ldo)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= rows || j >= cols) return;
    out[i * ldo + j] = in[(int64_t)j * ld + i];
}

__global__ void row_to_col_kernel(const float* __restrict__ in, int64_t ldi, int64_t rows, int cols, int cols_pad,
                                  float* __restrict__ out, int64_t ld)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= ld || j >= cols_pad) return;
    out[(int64_t)j * ld + i] = (i < rows && j < cols) ? in[i * ldi + j] : 0.f;
}

}  // namespace

void launch_chol_inv(cudaStream_t s, const double* G, int l, float shift_rel, float* R, float* T, int* status,
                     int* breakdowns)
{
    const size_t smem = (size_t)l * l * sizeof(float);
    chol_inv_kernel<<<1, kSmallThreads, smem, s>>>(G, l, shift_rel, R, T, status, breakdowns); count_launches();
}

namespace {
template <class K>
int raise_smem_limit(K kernel, int optin)
{
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return RSVDGB_ERR_CUDA;
    const int dyn = optin - (int)fa.sharedSizeBytes;
    if (dyn <= 0 || cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess)
        return RSVDGB_ERR_CUDA;
    return RSVDGB_OK;
}
}  // namespace

int init_small_kernels()
{
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RSVDGB_ERR_CUDA;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return RSVDGB_ERR_CUDA;
    int rc = raise_smem_limit(chol_inv_kernel, optin);
    if (rc) return rc;
    return raise_smem_limit(jacobi_kernel, optin);
}

void launch_small_matmul(cudaStream_t s, const float* A, const float* B, float* C, int l)
{
    dim3 block(16, 16);
    dim3 grid((unsigned)ceil_div(l, 16), (unsigned)ceil_div(l, 16));
    small_matmul_kernel<<<grid, block, 0, s>>>(A, B, C, l); count_launches();
}

void launch_small_d2f(cudaStream_t s, const double* in, float* out, int l, bool transpose)
{
    dim3 block(16, 16);
    dim3 grid((unsigned)ceil_div(l, 16), (unsigned)ceil_div(l, 16));
    small_d2f_kernel<<<grid, block, 0, s>>>(in, out, l, transpose ? 1 : 0);
    count_launches();
}

void launch_small_transpose(cudaStream_t s, const float* in, float* out, int l)
{
    dim3 block(16, 16);
    dim3 grid((unsigned)ceil_div(l, 16), (unsigned)ceil_div(l, 16));
    small_transpose_kernel<<<grid, block, 0, s>>>(in, out, l); count_launches();
}

void launch_jacobi_svd(cudaStream_t s, const float* M, int l, float* sigma, float* Ut, float* Jt, float* work)
{
    const int L = (int)round_up(l, 2);
    const size_t need = (size_t)2 * L * L * sizeof(float);
    const int use_smem = need <= (size_t)216 * 1024;
    jacobi_kernel<<<1, kSmallThreads, use_smem ? need : 0, s>>>(M, l, L, sigma, Ut, Jt, work, use_smem); count_launches();
}

void launch_finalize_info(cudaStream_t s, const float* sigma, int l, int k, float* d, const double* fro2A,
                          const int* status, const int* breakdowns, int q, int p_used, rsvdgb_info* info)
{
    finalize_info_kernel<<<1, 256, 0, s>>>(sigma, l, k, d, fro2A, status, breakdowns, q, p_used, info); count_launches();
}

void launch_clear_scalars(cudaStream_t s, int* status, int* breakdowns, double* fro2)
{
    clear_scalars_kernel<<<1, 1, 0, s>>>(status, breakdowns, fro2); count_launches();
}

void launch_split_tf32(cudaStream_t s, const float* in, int64_t ld, int64_t rows, int l, int l_pad, float* hi,
                       float* lo)
{
    dim3 grid((unsigned)ceil_div(ld, 256), (unsigned)l_pad);
    split_tf32_kernel<<<grid, 256, 0, s>>>(in, ld, rows, l, l_pad, hi, lo);
    count_launches();
}

void launch_colmajor_to_rowmajor(cudaStream_t s, const float* in, int64_t ld, int64_t rows, int cols, float* out,
                                 int64_t ldo)
{
    if (rows == 0 || cols == 0) return;
    dim3 grid((unsigned)ceil_div(rows, 256), (unsigned)cols);
    col_to_row_kernel<<<grid, 256, 0, s>>>(in, ld, rows, cols, out, ldo); count_launches();
}

void launch_rowmajor_to_colmajor(cudaStream_t s, const float* in, int64_t ldi, int64_t rows, int cols, int cols_pad,
                                 float* out, int64_t ld)
{
    dim3 grid((unsigned)ceil_div(ld, 256), (unsigned)cols_pad);
    row_to_col_kernel<<<grid, 256, 0, s>>>(in, ldi, rows, cols, cols_pad, out, ld); count_launches();
}

}  // namespace rsvdgb
