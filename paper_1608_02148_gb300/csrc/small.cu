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
#include <cuda_bf16.h>
#include <math.h>

#include "internal.cuh"

namespace rsvdgb {
namespace {

constexpr int kSmallThreads = 1024;

// ---------------------------------------------------------------------------
// Cholesky by symmetric Gaussian elimination on [G | I].
//
// Step j eliminates column j from the rows below with the pivot row j, then
// scales row j by 1/sqrt(pivot).  The G half turns into R (upper triangle)
// and the I half into R^{-T} (lower triangle), so R^{-1} = (R^{-T})^T comes out
// of the same l steps.  Both halves share one l x l array: R in the upper
// triangle including the diagonal, R^{-T} strictly below it, its diagonal in
// dinv.
//
// The array lives in registers: 1024 threads form a 32 x 32 grid and thread
// (ty, tx) owns rows ty + 32 i and columns tx + 32 j (NB x NB elements,
// NB = ceil(l / 32) <= 7).  Step j publishes the unscaled pivot row through a
// double-buffered shared vector, so each step costs one barrier.
// ---------------------------------------------------------------------------
template <int NB, int TD>  // TD x TD threads, NB x NB elements each (TD * NB >= l)
__global__ void __launch_bounds__(TD * TD)
    chol_inv_kernel(const double* __restrict__ G, int l, float shift_rel, float* __restrict__ R,
                    float* __restrict__ T, int* status, int* breakdowns)
{
    constexpr int kCholThreads = TD * TD;
    __shared__ float rowbuf[2][256];
    __shared__ float dinv[256];
    __shared__ float maxdiag;
    const int tid = threadIdx.x;
    const int tx = tid % TD, ty = tid / TD;

    if (tid < 32) {
        float md = 0.f;
        for (int a = tid; a < l; a += 32) md = fmaxf(md, (float)G[a * l + a]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
        if (tid == 0) maxdiag = md;
    }
    __syncthreads();

    float S[NB][NB];
    for (int attempt = 0; attempt < 4; ++attempt) {
        // shift = shift_rel * max diag on the first attempt; after a breakdown
        // the shift grows by 100x per retry (shifted CholeskyQR).
        float shift = shift_rel * maxdiag;
        if (attempt > 0) shift = fmaxf(shift, maxdiag * 1e-6f * powf(100.f, (float)(attempt - 1)));
#pragma unroll
        for (int i = 0; i < NB; ++i)
#pragma unroll
            for (int jj = 0; jj < NB; ++jj) {
                const int a = ty + TD * i, b = tx + TD * jj;
                float v = 0.f;
                if (a < l && b < l && b >= a) v = (float)G[a * l + b] + (a == b ? shift : 0.f);
                S[i][jj] = v;
            }
        // publish row 0
        if (ty == 0)
#pragma unroll
            for (int jj = 0; jj < NB; ++jj) rowbuf[0][tx + TD * jj] = S[0][jj];
        __syncthreads();
        bool failed = false;
        for (int j = 0; j < l; ++j) {
            const float* u = rowbuf[j & 1];
            const float pv = u[j];
            if (!(pv > 0.f) || !isfinite(pv)) {
                failed = true;  // every thread reads the same pivot
                break;
            }
            // one approximate reciprocal square root per step (relative error
            // a few ulps, far below the FP32 error the factor already carries)
            const float rinv = rsqrtf(pv);
            const float r = pv * rinv;
            const float pinv = rinv * rinv;
            float ub[NB];
#pragma unroll
            for (int jj = 0; jj < NB; ++jj) {
                const int b = tx + TD * jj;
                ub[jj] = (b == j) ? 1.0f : ((b < l) ? u[b] : 0.f);
            }
#pragma unroll
            for (int i = 0; i < NB; ++i) {
                const int a = ty + TD * i;
                if (a > j && a < l) {
                    const float f = u[a] * pinv;
#pragma unroll
                    for (int jj = 0; jj < NB; ++jj) {
                        const int b = tx + TD * jj;
                        if (b >= a || b <= j) S[i][jj] -= f * ub[jj];
                    }
                } else if (a == j) {
                    // scale the pivot row: R(j, b) for b >= j, R^{-T}(j, b) for b < j
#pragma unroll
                    for (int jj = 0; jj < NB; ++jj) {
                        const int b = tx + TD * jj;
                        S[i][jj] = (b == j) ? r : S[i][jj] * rinv;
                    }
                }
            }
            if (tid == 0) dinv[j] = rinv;
            // publish row j + 1 (its owners have just finished their update)
            if (j + 1 < l && ty == ((j + 1) % TD)) {
                const int i1 = (j + 1) / TD;
#pragma unroll
                for (int i = 0; i < NB; ++i)
                    if (i == i1)
#pragma unroll
                        for (int jj = 0; jj < NB; ++jj) rowbuf[(j + 1) & 1][tx + TD * jj] = S[i][jj];
            }
            __syncthreads();
        }
        if (!failed) break;
        __syncthreads();
        if (tid == 0) {
            if (breakdowns) atomicAdd(breakdowns, 1);
            if (attempt == 3 && status) *status = RSVDGB_ERR_BREAKDOWN;
        }
        __syncthreads();
    }
    // R (upper) straight from the registers; T = R^{-1} = (R^{-T})^T needs the
    // transpose of the lower part, so that goes through global memory order:
    // T(b, a) = R^{-T}(a, b) for b < a, T(a, a) = dinv[a].
#pragma unroll
    for (int i = 0; i < NB; ++i)
#pragma unroll
        for (int jj = 0; jj < NB; ++jj) {
            const int a = ty + TD * i, b = tx + TD * jj;
            if (a >= l || b >= l) continue;
            if (R) R[a * l + b] = (b >= a) ? S[i][jj] : 0.f;
            if (b < a) T[b * l + a] = S[i][jj];
            else if (b == a) T[a * l + a] = dinv[a];
            else T[b * l + a] = 0.f;  // T is upper triangular: zero below the diagonal
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

// EPL = ceil(L / 16): column elements per half-warp lane, held in registers
// while a pair is rotated.
//
// The right singular vectors J are needed for kv columns only.  The sweeps
// first run on M alone (half the shared-memory traffic); when the spectrum
// allows it, J_c = M^T U_c / sigma_c for the kv leading columns (its error is
// about u32 sigma_1 / sigma_c, accepted while sigma_kv >= 1e-3 sigma_1).
// Otherwise the sweeps are repeated from the original M with J accumulated.
template <int EPL, int NT>
__global__ void __launch_bounds__(NT)
    jacobi_kernel(const float* __restrict__ M, int l, int L, float* __restrict__ sigma, float* __restrict__ Ut,
                  float* __restrict__ Jt, float* __restrict__ gwork, int use_smem, int* sweeps_out, int kv)
{
    extern __shared__ float sm[];
    float* Mc = use_smem ? sm : gwork;
    float* Jc = use_smem ? sm + (size_t)L * L : gwork + (size_t)L * L;
    __shared__ int rotated;
    __shared__ int need_j;
    __shared__ float sv[256];
    __shared__ int rank[256];
    __shared__ int col_of_rank[256];
    __shared__ float jn[256];
    __shared__ float wn[256];
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int nwarps = NT / 32;
    const int half = lane >> 4, hl = lane & 15;  // half-warp: one column pair

    // rotate a pair only when its cosine exceeds the FP32 noise of the dot
    // products (about sqrt(L) u32); quadratic convergence does the rest.
    // c = 1 / sqrt(1 + t^2) in IEEE arithmetic keeps c^2 + s^2 - 1 at the
    // rounding level, so column norms drift only by a random walk of ulps.
    const float tol = 4.f * sqrtf((float)L) * 5.9604645e-8f;
    const int Lm1 = L - 1;
    int sweep = 0;
    for (int pass = 0; pass < 2; ++pass) {
        const bool accj = (pass == 1);
        // column-major copies, zero padded to L x L
        for (int e = tid; e < L * L; e += NT) {
            const int c = e / L, i = e % L;
            Mc[e] = (i < l && c < l) ? M[i * l + c] : 0.f;
            if (accj) Jc[e] = (i == c) ? 1.f : 0.f;
        }
        __syncthreads();
        for (sweep = 0; sweep < 30; ++sweep) {
            if (tid == 0) rotated = 0;
            __syncthreads();
            for (int round = 0; round < Lm1; ++round) {
                for (int base = 2 * warp; base < L / 2; base += 2 * nwarps) {
                    const int t = base + half;
                    const bool valid = t < L / 2;
                    int a = Lm1, b = round;
                    if (t != 0) {
                        a = round + t;
                        if (a >= Lm1) a -= Lm1;
                        b = round - t;
                        if (b < 0) b += Lm1;
                    }
                    float xa[EPL], xb[EPL];
                    float al = 0.f, be = 0.f, ga = 0.f;
                    if (valid) {
                        const float* ma = Mc + (size_t)a * L;
                        const float* mb = Mc + (size_t)b * L;
#pragma unroll
                        for (int e = 0; e < EPL; ++e) {
                            const int i = hl + 16 * e;
                            xa[e] = (i < L) ? ma[i] : 0.f;
                            xb[e] = (i < L) ? mb[i] : 0.f;
                            al = fmaf(xa[e], xa[e], al);
                            be = fmaf(xb[e], xb[e], be);
                            ga = fmaf(xa[e], xb[e], ga);
                        }
                    }
#pragma unroll
                    for (int o = 8; o > 0; o >>= 1) {
                        al += __shfl_xor_sync(0xffffffffu, al, o);
                        be += __shfl_xor_sync(0xffffffffu, be, o);
                        ga += __shfl_xor_sync(0xffffffffu, ga, o);
                    }
                    if (valid && ga != 0.f && fabsf(ga) > tol * sqrtf(al * be)) {
                        const float zeta = (be - al) / (2.f * ga);
                        const float tt = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
                        const float c = 1.0f / sqrtf(fmaf(tt, tt, 1.f));
                        const float sn = c * tt;
                        float* ma = Mc + (size_t)a * L;
                        float* mb = Mc + (size_t)b * L;
#pragma unroll
                        for (int e = 0; e < EPL; ++e) {
                            const int i = hl + 16 * e;
                            if (i < L) {
                                ma[i] = c * xa[e] - sn * xb[e];
                                mb[i] = sn * xa[e] + c * xb[e];
                            }
                        }
                        if (accj) {
                            float* ja = Jc + (size_t)a * L;
                            float* jb = Jc + (size_t)b * L;
#pragma unroll
                            for (int e = 0; e < EPL; ++e) {
                                const int i = hl + 16 * e;
                                if (i < L) {
                                    const float ya = ja[i], yb = jb[i];
                                    ja[i] = c * ya - sn * yb;
                                    jb[i] = sn * ya + c * yb;
                                }
                            }
                        }
                        if (hl == 0) rotated = 1;
                    }
                }
                __syncthreads();
            }
            if (!rotated) break;
            __syncthreads();
        }
        // singular values.  Rounding in the rotations scales each column of
        // W = M J by a factor close to 1 that accumulates over the sweeps.
        // With J accumulated, sigma_c = ||W_c|| / ||J_c|| cancels it.  Without
        // J, the direction u_c = W_c / ||W_c|| is unaffected and
        // sigma_c = ||M^T u_c||, J_c = M^T u_c / sigma_c (stored in Jc).
        for (int c = warp; c < L; c += nwarps) {
            float s2 = 0.f, j2 = 0.f;
            for (int i = lane; i < L; i += 32) {
                s2 = fmaf(Mc[(size_t)c * L + i], Mc[(size_t)c * L + i], s2);
                if (accj) j2 = fmaf(Jc[(size_t)c * L + i], Jc[(size_t)c * L + i], j2);
            }
            s2 = warp_sum(s2);
            j2 = warp_sum(j2);
            if (lane == 0) {
                wn[c] = sqrtf(s2);
                jn[c] = accj ? sqrtf(j2) : 1.f;
                sv[c] = accj ? ((j2 > 0.f) ? sqrtf(s2) / sqrtf(j2) : 0.f) : sqrtf(s2);
            }
        }
        __syncthreads();
        if (!accj) {
            for (int e = tid; e < L * L; e += NT) {
                const int c = e / L, i = e % L;
                float acc = 0.f;
                if (i < l && c < l && wn[c] > 0.f) {
                    const float* w = Mc + (size_t)c * L;
                    for (int t = 0; t < l; ++t) acc = fmaf(M[t * l + i], w[t], acc);
                    acc /= wn[c];
                }
                Jc[e] = acc;  // x_c = M^T u_c
            }
            __syncthreads();
            for (int c = warp; c < L; c += nwarps) {
                float x2 = 0.f;
                for (int i = lane; i < L; i += 32) x2 = fmaf(Jc[(size_t)c * L + i], Jc[(size_t)c * L + i], x2);
                x2 = warp_sum(x2);
                if (lane == 0) {
                    sv[c] = sqrtf(x2);
                    jn[c] = sqrtf(x2);
                }
            }
            __syncthreads();
        }
        for (int c = tid; c < L; c += NT) {
            int r = 0;
            for (int o = 0; o < L; ++o) r += (sv[o] > sv[c]) || (sv[o] == sv[c] && o < c);
            rank[c] = r;
            col_of_rank[r] = c;
        }
        __syncthreads();
        if (tid == 0 && !accj) {
            const float s1 = sv[col_of_rank[0]];
            const float skv = kv > 0 ? sv[col_of_rank[min(kv, l) - 1]] : s1;
            need_j = (kv > 0 && !(skv >= 1e-3f * s1)) ? 1 : 0;  // stays set after the J pass
        }
        __syncthreads();
        if (!need_j || accj) break;
    }
    if (tid == 0 && sweeps_out) *sweeps_out = sweep + 1;
    for (int e = tid; e < L * L; e += NT) {
        const int c = e / L, i = e % L;
        const int r = rank[c];
        if (r >= l || i >= l) continue;
        const float w = wn[c];
        Ut[i * l + r] = (w > 0.f) ? Mc[(size_t)c * L + i] / w : 0.f;
    }
    for (int c = tid; c < L; c += NT)
        if (rank[c] < l) sigma[rank[c]] = sv[c];
    if (kv <= 0) return;
    // right vectors for the kv leading ranks: accumulated J, or M^T u_c normalised
    for (int e = tid; e < L * L; e += NT) {
        const int c = e / L, i = e % L;
        const int r = rank[c];
        if (r >= kv || r >= l || i >= l) continue;
        Jt[i * l + r] = (jn[c] > 0.f) ? Jc[(size_t)c * L + i] / jn[c] : 0.f;
    }
}

__global__ void finalize_info_kernel(const float* __restrict__ sigma, int l, int k, float* __restrict__ d,
                                     const double* fro2A, const int* status, const int* breakdowns, int q,
                                     int p_used, int engine, const int* sweeps, rsvdgb_info* info)
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
        info->engine = engine;
        info->jacobi_sweeps = sweeps ? *sweeps : 0;
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

__global__ void small_panel_kernel(const float* __restrict__ T, int l, int L, float* __restrict__ hi,
                                   float* __restrict__ lo)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;  // K index (row of T)
    const int j = blockIdx.y;                             // N index (column of T)
    if (c >= L || j >= L) return;
    float h = 0.f, r = 0.f;
    if (c < l && j < l) {
        const float x = T[c * l + j];
        uint32_t hb, rb;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hb) : "f"(x));
        h = __uint_as_float(hb);
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(rb) : "f"(x - h));
        r = __uint_as_float(rb);
    }
    hi[j * L + c] = h;
    lo[j * L + c] = r;
}

__global__ void to_bf16_kernel(const float* __restrict__ in, int64_t ld, int64_t rows, int l, int l_pad,
                               __nv_bfloat16* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= ld || j >= l_pad) return;
    const int64_t o = (int64_t)j * ld + i;
    out[o] = __float2bfloat16_rn((i < rows && j < l) ? in[o] : 0.f);
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
    // 16 x 16 threads while the register tile stays small, 32 x 32 beyond
    if (l <= 16)
        chol_inv_kernel<1, 16><<<1, 256, 0, s>>>(G, l, shift_rel, R, T, status, breakdowns);
    else if (l <= 32)
        chol_inv_kernel<2, 16><<<1, 256, 0, s>>>(G, l, shift_rel, R, T, status, breakdowns);
    else if (l <= 64)
        chol_inv_kernel<4, 16><<<1, 256, 0, s>>>(G, l, shift_rel, R, T, status, breakdowns);
    else if (l <= 96)
        chol_inv_kernel<6, 16><<<1, 256, 0, s>>>(G, l, shift_rel, R, T, status, breakdowns);
    else if (l <= 128)
        chol_inv_kernel<8, 16><<<1, 256, 0, s>>>(G, l, shift_rel, R, T, status, breakdowns);
    else if (l <= 160)
        chol_inv_kernel<5, 32><<<1, 1024, 0, s>>>(G, l, shift_rel, R, T, status, breakdowns);
    else if (l <= 192)
        chol_inv_kernel<6, 32><<<1, 1024, 0, s>>>(G, l, shift_rel, R, T, status, breakdowns);
    else
        chol_inv_kernel<7, 32><<<1, 1024, 0, s>>>(G, l, shift_rel, R, T, status, breakdowns);
    count_launches();
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
    int rc = RSVDGB_OK;
    rc |= raise_smem_limit(jacobi_kernel<1, 1024>, optin);
    rc |= raise_smem_limit(jacobi_kernel<2, 1024>, optin);
    rc |= raise_smem_limit(jacobi_kernel<3, 1024>, optin);
    rc |= raise_smem_limit(jacobi_kernel<4, 1024>, optin);
    rc |= raise_smem_limit(jacobi_kernel<5, 1024>, optin);
    rc |= raise_smem_limit(jacobi_kernel<6, 1024>, optin);
    rc |= raise_smem_limit(jacobi_kernel<7, 1024>, optin);
    rc |= raise_smem_limit(jacobi_kernel<8, 1024>, optin);
    rc |= raise_smem_limit(jacobi_kernel<10, 512>, optin);
    rc |= raise_smem_limit(jacobi_kernel<12, 512>, optin);
    rc |= raise_smem_limit(jacobi_kernel<14, 512>, optin);
    return rc ? RSVDGB_ERR_CUDA : RSVDGB_OK;
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

template <int EPL, int NT>
void launch_jacobi_typed(cudaStream_t s, const float* M, int l, int L, float* sigma, float* Ut, float* Jt,
                         float* work, int* sweeps, int kv)
{
    const size_t need = (size_t)2 * L * L * sizeof(float);
    const int use_smem = need <= (size_t)216 * 1024;
    jacobi_kernel<EPL, NT><<<1, NT, use_smem ? need : 0, s>>>(M, l, L, sigma, Ut, Jt, work, use_smem, sweeps, kv);
}

void launch_jacobi_svd(cudaStream_t s, const float* M, int l, float* sigma, float* Ut, float* Jt, float* work,
                       int* sweeps, int kv)
{
    const int L = (int)round_up(l, 2);
    switch ((L + 15) / 16) {
        case 1: launch_jacobi_typed<1, 1024>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv); break;
        case 2: launch_jacobi_typed<2, 1024>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv); break;
        case 3: launch_jacobi_typed<3, 1024>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv); break;
        case 4: launch_jacobi_typed<4, 1024>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv); break;
        case 5: launch_jacobi_typed<5, 1024>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv); break;
        case 6: launch_jacobi_typed<6, 1024>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv); break;
        case 7: launch_jacobi_typed<7, 1024>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv); break;
        case 8: launch_jacobi_typed<8, 1024>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv); break;
        case 9: case 10: launch_jacobi_typed<10, 512>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv); break;
        case 11: case 12: launch_jacobi_typed<12, 512>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv); break;
        default: launch_jacobi_typed<14, 512>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv); break;
    }
    count_launches();
}

void launch_finalize_info(cudaStream_t s, const float* sigma, int l, int k, float* d, const double* fro2A,
                          const int* status, const int* breakdowns, int q, int p_used, int engine, const int* sweeps,
                          rsvdgb_info* info)
{
    finalize_info_kernel<<<1, 256, 0, s>>>(sigma, l, k, d, fro2A, status, breakdowns, q, p_used, engine, sweeps,
                                           info); count_launches();
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

void launch_small_panel(cudaStream_t s, const float* T, int l, int L, float* hi, float* lo)
{
    dim3 grid((unsigned)ceil_div(L, 128), (unsigned)L);
    small_panel_kernel<<<grid, 128, 0, s>>>(T, l, L, hi, lo);
    count_launches();
}

void launch_to_bf16(cudaStream_t s, const float* in, int64_t ld, int64_t rows, int l, int l_pad, void* out)
{
    dim3 grid((unsigned)ceil_div(ld, 256), (unsigned)l_pad);
    to_bf16_kernel<<<grid, 256, 0, s>>>(in, ld, rows, l, l_pad, (__nv_bfloat16*)out);
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
