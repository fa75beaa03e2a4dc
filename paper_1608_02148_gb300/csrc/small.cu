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
// Precision: these kernels compute in FP32 on FP32 Gram inputs.  GB300's
// FP64 pipe is far slower than its FP32 pipe, and the Gram matrices they
// factor carry FP32-level error already (FP32 accumulation over the rows),
// so FP64 here would not change the result beyond that error; CholeskyQR2
// recovers orthogonality to FP32 level.
#include <cuda_bf16.h>
#include <math.h>

#include "internal.cuh"

namespace rsvdgb {
namespace {

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
    chol_inv_kernel(const float* __restrict__ G, int l, float shift_rel, float* __restrict__ R,
                    float* __restrict__ T, int* status, int* breakdowns)
{
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

// ---------------------------------------------------------------------------
// Blocked form of the same elimination on [G | I], for l <= kCholBlockedMax.
//
// Both halves live in shared memory (row-major, stride ld, the whole
// symmetric G and the whole I half).  For each block of 16 pivot rows
// k0 .. k0 + 15:
//   1. one warp factors the 16 x 16 diagonal block D = R_kk^T R_kk of the
//      current Schur complement in registers and forms R_kk^{-T};
//   2. the block rows are scaled, S_k = R_kk^{-T} [G | I](block rows): their
//      G half becomes rows k0.. of R, their I half rows k0.. of R^{-T};
//   3. the rows below are updated with the scaled block rows,
//      [G | I](r, :) -= sum_m R(k0 + m, r) S_k(m, :),
//      a rank-16 update (packed FP32x2 FMAs, 4 x 4 outputs per thread).
// Only the G columns right of the block and the I columns left of its end
// can be nonzero, so steps 2 and 3 touch exactly those.  Step 1 of the next
// block runs during step 3: warp 0 first updates the next diagonal block
// (16 tiles) and factors it while the other warps update everything else.
// A pivot that is not positive and finite restarts the factorization with a
// larger shift.
// ---------------------------------------------------------------------------
constexpr int kCholBlockedMax = 160;
constexpr int kCholBlockedThreads = 512;

// Step 1 for the block at (k0, k0): lanes 0..15 hold columns of the G half,
// lanes 16..31 the same columns of the I half (identity beyond bk).  The
// pivot column D(:, j) is broadcast from lane j.  Writes R_kk into Gs and
// R_kk^{-T} into Ls; returns true (on every lane) after a bad pivot.
__device__ __noinline__ bool chol_diag_block(float* Gs, int ld, int k0, int bk, float (*Ls)[17], int lane)
{
    const int c = lane & 15;
    const bool gpart = lane < 16;
    float v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r)
        v[r] = (gpart && r < bk && c < bk) ? Gs[(size_t)(k0 + r) * ld + k0 + c] : (r == c ? 1.f : 0.f);
    bool bad = false;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const float pv = __shfl_sync(0xffffffffu, v[j], j);
        if (!(pv > 0.f) || !isfinite(pv)) bad = true;
        const float rinv = rsqrtf(pv);
        const float npinv = -rinv * rinv;
#pragma unroll
        for (int r = j + 1; r < 16; ++r) v[r] = fmaf(__shfl_sync(0xffffffffu, v[r], j) * npinv, v[j], v[r]);
        v[j] *= rinv;
    }
    if (gpart) {
        if (c < bk)
#pragma unroll
            for (int r = 0; r < 16; ++r)
                if (r < bk) Gs[(size_t)(k0 + r) * ld + k0 + c] = v[r];
    } else {
#pragma unroll
        for (int r = 0; r < 16; ++r) Ls[r][c] = v[r];
    }
    return bad;
}

// Step 3 for one 4 x 4 tile: rows r0..r0+3 (>= the block's end) of X (Gs or
// Is), columns cbase..cbase+3, minus sum_m R(k0 + m, r) X(k0 + m, c).
__device__ __forceinline__ void chol_update_tile(const float* Gs, float* X, int ld, int k0, int bk, int r0,
                                                 int cbase, int l)
{
    float2 acc[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = make_float2(0.f, 0.f);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        if (m < bk) {
            const float4 rv = *reinterpret_cast<const float4*>(Gs + (size_t)(k0 + m) * ld + r0);
            const float4 cv = *reinterpret_cast<const float4*>(X + (size_t)(k0 + m) * ld + cbase);
            const float2 c01 = make_float2(cv.x, cv.y), c23 = make_float2(cv.z, cv.w);
            const float rr[4] = {rv.x, rv.y, rv.z, rv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 r2 = make_float2(rr[i], rr[i]);
                acc[i][0] = __ffma2_rn(r2, c01, acc[i][0]);
                acc[i][1] = __ffma2_rn(r2, c23, acc[i][1]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (r0 + i >= l) continue;
        float4* row = reinterpret_cast<float4*>(X + (size_t)(r0 + i) * ld + cbase);
        float4 x = *row;
        x.x -= acc[i][0].x;
        x.y -= acc[i][0].y;
        x.z -= acc[i][1].x;
        x.w -= acc[i][1].y;
        *row = x;
    }
}

__global__ void __launch_bounds__(kCholBlockedThreads, 1)
    chol_blocked_kernel(const float* __restrict__ G, int l, int ld, float shift_rel, float* __restrict__ R,
                        float* __restrict__ T, int* status, int* breakdowns)
{
    extern __shared__ __align__(16) float csm[];
    float* Gs = csm;                  // l x ld
    float* Is = csm + (size_t)l * ld;  // l x ld
    __shared__ float Ls[16][17];      // R_kk^{-T} of the current block
    __shared__ float maxdiag;
    __shared__ int failed;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int NT = kCholBlockedThreads;
    constexpr int NW = NT / 32;

    // zero padding of the G rows (shared memory only)
    for (int a = warp; a < l; a += NW)
        for (int b = l + lane; b < ld; b += 32) Gs[(size_t)a * ld + b] = 0.f;

    for (int attempt = 0; attempt < 4; ++attempt) {
        // G (l x l, contiguous) lands in the I half by 16-byte asynchronous
        // copies, all in flight at once; the upper triangle (+ shift) goes to
        // the G half, the lower triangle is mirrored from it (an exactly
        // symmetric matrix), then the I half is reset to the identity
        {
            const int chunks = (l * l + 3) / 4;
            for (int q = tid; q < chunks; q += NT)
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                                 (uint32_t)__cvta_generic_to_shared(Is + 4 * q)),
                             "l"(G + 4 * q)
                             : "memory");
            asm volatile("cp.async.wait_all;" ::: "memory");
            __syncthreads();
            // shift = shift_rel * max diag on the first attempt; after a
            // breakdown the shift grows by 100x per retry (shifted CholeskyQR)
            float shift = 0.f;
            if (shift_rel > 0.f || attempt > 0) {
                if (warp == 0) {
                    float md = 0.f;
                    for (int a = lane; a < l; a += 32) md = fmaxf(md, Is[a * l + a]);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
                    if (lane == 0) maxdiag = md;
                }
                __syncthreads();
                shift = shift_rel * maxdiag;
                if (attempt > 0) shift = fmaxf(shift, maxdiag * 1e-6f * powf(100.f, (float)(attempt - 1)));
            }
            for (int a = warp; a < l; a += NW)
                for (int b = a + lane; b < l; b += 32)
                    Gs[(size_t)a * ld + b] = Is[a * l + b] + (a == b ? shift : 0.f);
            __syncthreads();
            for (int a = warp; a < l; a += NW)
                for (int b = lane; b < ld; b += 32) Is[(size_t)a * ld + b] = (a == b) ? 1.f : 0.f;
        }
        if (tid == 0) failed = 0;
        __syncthreads();
        for (int a = warp; a < l; a += NW)
            for (int b = lane; b < a; b += 32) Gs[(size_t)a * ld + b] = Gs[(size_t)b * ld + a];
        __syncthreads();
        if (warp == 0 && chol_diag_block(Gs, ld, 0, min(16, l), Ls, lane) && lane == 0) failed = 1;
        __syncthreads();

        for (int k0 = 0; k0 < l; k0 += 16) {
            if (failed) break;
            const int bk = min(16, l - k0);
            const int c_end = k0 + bk;
            const int wG = l - c_end;
            // 2. scale the block rows: columns right of the block (G half) and
            //    left of its end (I half); thread = (column, half of the rows)
            {
                const int task = tid;
                const bool active = task < 2 * l;
                const int half = task / l, t = task - half * l;
                float* X = (t < wG) ? Gs + c_end + t : Is + (t - wG);
                float x[16];
#pragma unroll
                for (int m = 0; m < 16; ++m) x[m] = (active && m < bk) ? X[(size_t)(k0 + m) * ld] : 0.f;
                __syncthreads();
                if (active) {
                    if (half == 0) {
#pragma unroll
                        for (int r = 0; r < 8; ++r) {
                            float acc = 0.f;
#pragma unroll
                            for (int m = 0; m <= r; ++m) acc = fmaf(Ls[r][m], x[m], acc);
                            if (r < bk) X[(size_t)(k0 + r) * ld] = acc;
                        }
                    } else {
#pragma unroll
                        for (int r = 8; r < 16; ++r) {
                            float acc = 0.f;
#pragma unroll
                            for (int m = 0; m <= r; ++m) acc = fmaf(Ls[r][m], x[m], acc);
                            if (r < bk) X[(size_t)(k0 + r) * ld] = acc;
                        }
                    }
                }
            }
            __syncthreads();
            // 3. rank-16 update of the rows below (none after the last block)
            const int h = l - c_end;
            if (h > 0) {
                const int nrt = (h + 3) / 4;
                const int ntG = (wG + 3) / 4, ntI = c_end / 4;
                const int nd = min(4, ntG);  // tiles of the next diagonal block per row
                if (warp == 0) {
                    if (lane < 16) {
                        const int rt = lane >> 2, ct = lane & 3;
                        if (rt < nrt && ct < nd) chol_update_tile(Gs, Gs, ld, k0, bk, c_end + 4 * rt, c_end + 4 * ct, l);
                    }
                    __syncwarp();
                    if (chol_diag_block(Gs, ld, c_end, min(16, h), Ls, lane) && lane == 0) failed = 1;
                } else {
                    for (int tile = tid - 32; tile < nrt * (ntG + ntI); tile += NT - 32) {
                        const int rt = tile / (ntG + ntI), ct = tile - rt * (ntG + ntI);
                        if (rt < 4 && ct < nd) continue;  // warp 0's
                        if (ct < ntG)
                            chol_update_tile(Gs, Gs, ld, k0, bk, c_end + 4 * rt, c_end + 4 * ct, l);
                        else
                            chol_update_tile(Gs, Is, ld, k0, bk, c_end + 4 * rt, 4 * (ct - ntG), l);
                    }
                }
                __syncthreads();
            }
        }
        if (!failed) break;
        if (tid == 0) {
            if (breakdowns) atomicAdd(breakdowns, 1);
            if (attempt == 3 && status) *status = RSVDGB_ERR_BREAKDOWN;
        }
        __syncthreads();
    }
    // R = upper triangle of the G half; T = R^{-1} = (R^{-T})^T from the I half
    for (int a = warp; a < l; a += NW)
        for (int b = lane; b < l; b += 32) {
            if (R) R[(size_t)a * l + b] = (b >= a) ? Gs[(size_t)a * ld + b] : 0.f;
            T[(size_t)a * l + b] = (a <= b) ? Is[(size_t)b * ld + a] : 0.f;  // T(a, b) = R^{-T}(b, a)
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
// rotated at once, eight lanes per pair.  Columns live column-major with a
// padded stride Lp = 8 E (zero rows beyond l) in Mc and Jc (shared memory
// when they fit, else the global work buffer); lane g of a pair holds the E
// contiguous elements [g E, g E + E) of both columns as float2 pairs, so
// loads, dot products and updates run on packed FP32x2 instructions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// The right singular vectors J are needed for kv columns only.  The sweeps
// first run on M alone (half the shared-memory traffic); when the spectrum
// allows it, J_c = M^T U_c / sigma_c for the kv leading columns.  The
// converged columns of W are orthogonal only to the stopping tolerance tol
// (relative), and M^T u_c picks up tol sigma_a / sigma_c of every column a
// with a larger sigma_a, so that route is taken while
// tol sigma_1 / sigma_kv <= 2e-5.  Otherwise the sweeps are repeated from the
// original M with J accumulated (orthogonal to rounding whatever the spectrum).
//
// MODE 0: columns in the global work buffer; 1: columns in shared memory;
// 2: also a staged copy of M (rows padded to a multiple of 4); 3: the columns
// of M in shared memory, J (accumulated or M^T u) in global memory.  MODE is a
// template parameter so that shared-memory columns get shared-memory loads.
template <int E, int NT, int MODE>
__global__ void __launch_bounds__(NT, 1)
    jacobi_kernel(const float* __restrict__ M, int l, int L, float* __restrict__ sigma, float* __restrict__ Ut,
                  float* __restrict__ Jt, float* __restrict__ gwork, int* sweeps_out, int kv)
{
    static_assert(E % 2 == 0, "E float2 pairs");
    constexpr int Lp = 8 * E;
    constexpr int E2 = E / 2;
    constexpr int use_smem = MODE;
    extern __shared__ __align__(16) float sm[];
    float* Mc = MODE ? sm : gwork;
    float* Jc = (MODE == 1 || MODE == 2) ? sm + (size_t)L * Lp : gwork + (size_t)L * Lp;
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
    constexpr int ngrp = NT / 8;
    const int grp = tid >> 3, gl = tid & 7;  // pair group, lane in the group
    const int P = L / 2;

    // rotate a pair only when its cosine exceeds the FP32 noise of the dot
    // products (about sqrt(L) u32); quadratic convergence does the rest.
    const float tol = 4.f * sqrtf((float)L) * 5.9604645e-8f;
    const int Lm1 = L - 1;
    int sweep = 0;
    for (int pass = 0; pass < 2; ++pass) {
        const bool accj = (pass == 1);
        // column-major copies, zero padded to Lp rows (rows of M read
        // contiguously, one warp per row)
        for (int i = warp; i < Lp; i += nwarps)
            for (int c = lane; c < L; c += 32) {
                Mc[(size_t)c * Lp + i] = (i < l && c < l) ? M[i * l + c] : 0.f;
                if (accj) Jc[(size_t)c * Lp + i] = (i == c) ? 1.f : 0.f;
            }
        __syncthreads();
        for (sweep = 0; sweep < 30; ++sweep) {
            if (tid == 0) rotated = 0;
            __syncthreads();
            for (int round = 0; round < Lm1; ++round) {
                for (int t0 = 0; t0 < P; t0 += ngrp) {
                    const int t = t0 + grp;
                    const bool valid = t < P;
                    int a = Lm1, b = round;
                    if (t != 0) {
                        a = round + t;
                        if (a >= Lm1) a -= Lm1;
                        b = round - t;
                        if (b < 0) b += Lm1;
                    }
                    float2 xa[E2], xb[E2];
                    float2 al2 = make_float2(0.f, 0.f), be2 = al2, ga2 = al2;
                    if (valid) {
                        const float2* ma = reinterpret_cast<const float2*>(Mc + (size_t)a * Lp + gl * E);
                        const float2* mb = reinterpret_cast<const float2*>(Mc + (size_t)b * Lp + gl * E);
#pragma unroll
                        for (int e = 0; e < E2; ++e) {
                            xa[e] = ma[e];
                            xb[e] = mb[e];
                            al2 = __ffma2_rn(xa[e], xa[e], al2);
                            be2 = __ffma2_rn(xb[e], xb[e], be2);
                            ga2 = __ffma2_rn(xa[e], xb[e], ga2);
                        }
                    }
                    float al = al2.x + al2.y, be = be2.x + be2.y, ga = ga2.x + ga2.y;
#pragma unroll
                    for (int o = 4; o > 0; o >>= 1) {
                        al += __shfl_xor_sync(0xffffffffu, al, o);
                        be += __shfl_xor_sync(0xffffffffu, be, o);
                        ga += __shfl_xor_sync(0xffffffffu, ga, o);
                    }
                    // al, be > 0 whenever ga != 0, so the rsqrt factors are finite
                    if (valid && ga != 0.f && fabsf(ga) * rsqrtf(al) * rsqrtf(be) > tol) {
                        // Rutishauser's rotation: zeta = cot(2 theta), t = tan(theta)
                        // = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2).
                        // The angle may be off by a few ulps (hardware reciprocal
                        // and rsqrt), which only moves the pair's off-diagonal a
                        // little; what must hold to rounding level is
                        // c^2 (1 + t^2) = 1, so c gets one Newton step for
                        // x^(-1/2) (r <- r + r (1 - x r^2) / 2) after the rsqrt.
                        const float zeta = __fdividef(be - al, 2.f * ga);
                        const float az = fabsf(zeta);
                        float tt;
                        if (az < 1e18f) {
                            const float h2 = fmaf(az, az, 1.f);
                            tt = __fdividef(1.f, az + h2 * rsqrtf(h2));
                        } else {
                            tt = __fdividef(0.5f, az);
                        }
                        tt = copysignf(tt, zeta);
                        const float x = fmaf(tt, tt, 1.f);
                        const float r0 = rsqrtf(x);
                        const float c = fmaf(0.5f * r0, fmaf(-x * r0, r0, 1.f), r0);
                        const float sn = c * tt;
                        const float2 c2 = make_float2(c, c), s2 = make_float2(sn, sn), ns2 = make_float2(-sn, -sn);
                        float2* ma = reinterpret_cast<float2*>(Mc + (size_t)a * Lp + gl * E);
                        float2* mb = reinterpret_cast<float2*>(Mc + (size_t)b * Lp + gl * E);
#pragma unroll
                        for (int e = 0; e < E2; ++e) {
                            ma[e] = __ffma2_rn(ns2, xb[e], __fmul2_rn(c2, xa[e]));
                            mb[e] = __ffma2_rn(s2, xa[e], __fmul2_rn(c2, xb[e]));
                        }
                        if (accj) {
                            float2* ja = reinterpret_cast<float2*>(Jc + (size_t)a * Lp + gl * E);
                            float2* jb = reinterpret_cast<float2*>(Jc + (size_t)b * Lp + gl * E);
#pragma unroll
                            for (int e = 0; e < E2; ++e) {
                                const float2 ya = ja[e], yb = jb[e];
                                ja[e] = __ffma2_rn(ns2, yb, __fmul2_rn(c2, ya));
                                jb[e] = __ffma2_rn(s2, ya, __fmul2_rn(c2, yb));
                            }
                        }
                        if (gl == 0) rotated = 1;
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
                s2 = fmaf(Mc[(size_t)c * Lp + i], Mc[(size_t)c * Lp + i], s2);
                if (accj) j2 = fmaf(Jc[(size_t)c * Lp + i], Jc[(size_t)c * Lp + i], j2);
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
            // x_c = M^T u_c for all columns at once, 4 x 4 outputs per thread;
            // M row-major, staged in shared memory (rows padded to Lq) when
            // there is room, else read from global memory.
            const int Lq = (L + 3) & ~3;
            const float* Ms = M;
            int ldm = l;
            if (use_smem == 2) {
                float* st = sm + 2 * (size_t)L * Lp;
                for (int e = tid; e < l * Lq; e += NT) {
                    const int t = e / Lq, i = e % Lq;
                    st[e] = (i < l) ? M[t * l + i] : 0.f;
                }
                __syncthreads();
                Ms = st;
                ldm = Lq;
            }
            const int nb = Lq / 4;
            for (int blk = tid; blk < nb * nb; blk += NT) {
                const int ib = blk % nb, cb = blk / nb;
                float acc[4][4] = {};
                for (int t = 0; t < l; ++t) {
                    float mv[4], wv[4];
                    if (use_smem == 2) {
                        const float4 m4 = *(const float4*)&Ms[(size_t)t * ldm + 4 * ib];
                        mv[0] = m4.x;
                        mv[1] = m4.y;
                        mv[2] = m4.z;
                        mv[3] = m4.w;
                    } else {
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int i = 4 * ib + k;
                            mv[k] = (i < l) ? Ms[(size_t)t * ldm + i] : 0.f;
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int c = 4 * cb + k;
                        wv[k] = (c < L) ? Mc[(size_t)c * Lp + t] : 0.f;
                    }
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(mv[a], wv[b], acc[a][b]);
                }
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int c = 4 * cb + b;
                    if (c >= L) continue;
                    const float rw = (c < l && wn[c] > 0.f) ? 1.f / wn[c] : 0.f;
#pragma unroll
                    for (int a = 0; a < 4; ++a) {
                        const int i = 4 * ib + a;
                        if (i < L) Jc[(size_t)c * Lp + i] = (i < l) ? acc[a][b] * rw : 0.f;
                    }
                }
            }
            __syncthreads();
            for (int c = warp; c < L; c += nwarps) {
                float x2 = 0.f;
                for (int i = lane; i < L; i += 32) x2 = fmaf(Jc[(size_t)c * Lp + i], Jc[(size_t)c * Lp + i], x2);
                x2 = warp_sum(x2);
                if (lane == 0) {
                    sv[c] = sqrtf(x2);
                    jn[c] = sqrtf(x2);
                }
            }
            __syncthreads();
        }
        // ranks by descending sigma, ties by column; a NaN sigma (non-finite
        // input) ranks as -1, so the ranks always form a permutation
        for (int c = tid; c < L; c += NT) {
            const float kc = (sv[c] == sv[c]) ? sv[c] : -1.f;
            int r = 0;
            for (int o = 0; o < L; ++o) {
                const float ko = (sv[o] == sv[o]) ? sv[o] : -1.f;
                r += (ko > kc) || (ko == kc && o < c);
            }
            rank[c] = r;
            col_of_rank[r] = c;
        }
        __syncthreads();
        if (tid == 0 && !accj) {
            const float s1 = sv[col_of_rank[0]];
            const float skv = kv > 0 ? sv[col_of_rank[min(kv, l) - 1]] : s1;
            need_j = (kv > 0 && !(skv * 2e-5f >= tol * s1)) ? 1 : 0;  // stays set after the J pass
        }
        __syncthreads();
        if (!need_j || accj) break;
    }
    if (tid == 0 && sweeps_out) *sweeps_out = sweep + 1;
    // outputs row by row (contiguous stores): Ut(i, r) = u_c(i), c of rank r
    for (int i = warp; i < l; i += nwarps)
        for (int r = lane; r < l; r += 32) {
            const int c = col_of_rank[r];
            const float w = wn[c];
            Ut[i * l + r] = (w > 0.f) ? Mc[(size_t)c * Lp + i] / w : 0.f;
        }
    for (int c = tid; c < L; c += NT)
        if (rank[c] < l) sigma[rank[c]] = sv[c];
    if (kv <= 0) return;
    // right vectors for the kv leading ranks: accumulated J, or M^T u_c normalised
    const int kr = min(kv, l);
    for (int i = warp; i < l; i += nwarps)
        for (int r = lane; r < kr; r += 32) {
            const int c = col_of_rank[r];
            Jt[i * l + r] = (jn[c] > 0.f) ? Jc[(size_t)c * Lp + i] / jn[c] : 0.f;
        }
}

// max_ij |G_ij - delta_ij| of an l x l row-major Gram (one CTA)
__global__ void orth_err_kernel(const float* __restrict__ G, int l, float* __restrict__ out)
{
    __shared__ float red[8];
    float mx = 0.f;
    for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
        const int i = e / l, j = e - i * l;
        mx = fmaxf(mx, fabsf(G[e] - (i == j ? 1.f : 0.f)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
        *out = fmaxf(red[0], mx);
    }
}

__global__ void finalize_info_kernel(const float* __restrict__ sigma, int l, int k, float* __restrict__ d,
                                     const double* fro2A, const int* status, const int* breakdowns, int q,
                                     int p_used, int engine, const int* sweeps, rsvdgb_info* info,
                                     const float* orth)
{
    const int tid = threadIdx.x;
    if (d && sigma)
        for (int i = tid; i < k; i += blockDim.x) d[i] = sigma[i];
    if (tid >= 32 || !info) return;
    // sum of squares over the l (and the first k) singular values: one warp,
    // lane-strided loads in flight together, FP64 shuffle reduction
    double sb = 0.0, sk = 0.0;
    for (int i = tid; sigma && i < l; i += 32) {
        const double s = (double)sigma[i];
        sb += s * s;
        if (i < k) sk += s * s;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
        sk += __shfl_xor_sync(0xffffffffu, sk, o);
    }
    if (tid == 0) {
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
        info->orth_max = orth ? *orth : -1.f;
    }
}

__global__ void clear_scalars_kernel(int* status, int* breakdowns, double* fro2, unsigned int* amax, float* fillv,
                                     int nfill, float fillval, unsigned int* zerov, int nzero)
{
    for (int i = threadIdx.x; i < nzero; i += blockDim.x) zerov[i] = 0u;
    if (threadIdx.x == 0) {
        if (status) *status = 0;
        if (breakdowns) *breakdowns = 0;
        if (fro2) *fro2 = 0.0;
        if (amax) *amax = 0u;
    }
    for (int i = threadIdx.x; i < nfill; i += blockDim.x) fillv[i] = fillval;
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

void launch_chol_inv(cudaStream_t s, const float* G, int l, float shift_rel, float* R, float* T, int* status,
                     int* breakdowns)
{
    if (l <= kCholBlockedMax) {
        // rows padded to a multiple of 4 (+4 to spread banks) for float4 tiles
        const int ld = ((l + 3) & ~3) + 4;
        const size_t bytes = (size_t)2 * l * ld * sizeof(float);
        chol_blocked_kernel<<<1, kCholBlockedThreads, bytes, s>>>(G, l, ld, shift_rel, R, T, status, breakdowns);
        count_launches();
        return;
    }
    // wider sketches: the register-tile elimination on 32 x 32 threads
    if (l <= 192)
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
    rc |= raise_smem_limit(chol_blocked_kernel, optin);
    rc |= raise_smem_limit(jacobi_kernel<2, 512, 2>, optin);
    rc |= raise_smem_limit(jacobi_kernel<4, 512, 2>, optin);
    rc |= raise_smem_limit(jacobi_kernel<6, 512, 2>, optin);
    rc |= raise_smem_limit(jacobi_kernel<8, 512, 2>, optin);
    rc |= raise_smem_limit(jacobi_kernel<10, 512, 2>, optin);
    rc |= raise_smem_limit(jacobi_kernel<12, 512, 2>, optin);
    rc |= raise_smem_limit(jacobi_kernel<14, 448, 2>, optin);
    rc |= raise_smem_limit(jacobi_kernel<16, 512, 2>, optin);
    rc |= raise_smem_limit(jacobi_kernel<20, 512, 1>, optin);
    rc |= raise_smem_limit(jacobi_kernel<24, 512, 3>, optin);
    rc |= raise_smem_limit(jacobi_kernel<28, 512, 3>, optin);
    return rc ? RSVDGB_ERR_CUDA : RSVDGB_OK;
}

void launch_small_matmul(cudaStream_t s, const float* A, const float* B, float* C, int l)
{
    dim3 block(16, 16);
    dim3 grid((unsigned)ceil_div(l, 16), (unsigned)ceil_div(l, 16));
    small_matmul_kernel<<<grid, block, 0, s>>>(A, B, C, l); count_launches();
}

void launch_small_transpose(cudaStream_t s, const float* in, float* out, int l)
{
    dim3 block(16, 16);
    dim3 grid((unsigned)ceil_div(l, 16), (unsigned)ceil_div(l, 16));
    small_transpose_kernel<<<grid, block, 0, s>>>(in, out, l); count_launches();
}

template <int E, int NT, int MODE>
void launch_jacobi_typed(cudaStream_t s, const float* M, int l, int L, float* sigma, float* Ut, float* Jt,
                         float* work, int* sweeps, int kv)
{
    const size_t Lp = 8 * E;
    const size_t cols = (size_t)2 * L * Lp * sizeof(float);
    const size_t bytes = MODE == 2   ? cols + (size_t)l * ((L + 3) & ~3) * sizeof(float)
                         : MODE == 1 ? cols
                         : MODE == 3 ? cols / 2
                                     : 0;
    jacobi_kernel<E, NT, MODE><<<1, NT, bytes, s>>>(M, l, L, sigma, Ut, Jt, work, sweeps, kv);
}

// Columns of L = l rounded up to even rows; E elements per lane of the eight
// lanes of a pair, so the padded column stride 8 E covers L.  Up to L = 128
// the columns and a staged M fit in shared memory (MODE 2), up to 160 the
// columns alone (MODE 1); wider sketches keep M's columns in shared memory and
// J in global memory (MODE 3).  At E = 14 (L in [98, 112]) the 56 pairs fill
// 448 threads exactly: no idle warps issue the round's instructions or wait
// at its barrier (512 threads measured 9-20 us slower per SVD at l = 110).
void launch_jacobi_svd(cudaStream_t s, const float* M, int l, float* sigma, float* Ut, float* Jt, float* work,
                       int* sweeps, int kv)
{
    const int L = (int)round_up(l, 2);
    const int e = (int)round_up(ceil_div(L, 8), 2);
    if (e <= 2) launch_jacobi_typed<2, 512, 2>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv);
    else if (e <= 4) launch_jacobi_typed<4, 512, 2>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv);
    else if (e <= 6) launch_jacobi_typed<6, 512, 2>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv);
    else if (e <= 8) launch_jacobi_typed<8, 512, 2>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv);
    else if (e <= 10) launch_jacobi_typed<10, 512, 2>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv);
    else if (e <= 12) launch_jacobi_typed<12, 512, 2>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv);
    else if (e <= 14) launch_jacobi_typed<14, 448, 2>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv);
    else if (e <= 16) launch_jacobi_typed<16, 512, 2>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv);
    else if (e <= 20) launch_jacobi_typed<20, 512, 1>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv);
    else if (e <= 24) launch_jacobi_typed<24, 512, 3>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv);
    else launch_jacobi_typed<28, 512, 3>(s, M, l, L, sigma, Ut, Jt, work, sweeps, kv);
    count_launches();
}

void launch_finalize_info(cudaStream_t s, const float* sigma, int l, int k, float* d, const double* fro2A,
                          const int* status, const int* breakdowns, int q, int p_used, int engine, const int* sweeps,
                          rsvdgb_info* info, const float* orth)
{
    finalize_info_kernel<<<1, 256, 0, s>>>(sigma, l, k, d, fro2A, status, breakdowns, q, p_used, engine, sweeps,
                                           info, orth);
    count_launches();
}

void launch_orth_err(cudaStream_t s, const float* G, int l, float* out)
{
    orth_err_kernel<<<1, 256, 0, s>>>(G, l, out);
    count_launches();
}

void launch_clear_scalars(cudaStream_t s, int* status, int* breakdowns, double* fro2, unsigned int* amax,
                          float* fillv, int nfill, float fillval, unsigned int* zerov, int nzero)
{
    clear_scalars_kernel<<<1, 256, 0, s>>>(status, breakdowns, fro2, amax, fillv, fillv ? nfill : 0, fillval, zerov,
                                           zerov ? nzero : 0);
    count_launches();
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
