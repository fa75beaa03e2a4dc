// Batched randomized SVD of many small matrices of uneven shapes (l = k + p <= 32).
//
// Every step of Algorithm rSVD (Sec. 3.3) with subspace iterations (Algorithm
// sub_iterations) runs as one grouped kernel over the whole batch:
//   * pass kernels (Y = A X, W = A^T Y) pull (matrix, 128-row block) or
//     (matrix, 64-column block) work items from a device queue (an item array
//     and an atomic cursor), so CTAs stay busy whatever the shape mix;
//   * tall x small kernels (X T, Gram partials) use the same row-block items;
//   * per-matrix kernels (Gram reduction + Cholesky + inverse, 32 x 32 products,
//     one-sided Jacobi SVD) give one warp to each matrix.
// The stage sequence is captured once per batch layout in a CUDA graph and
// replayed with a single cudaGraphLaunch.  A small autotuner picks the number
// of resident CTAs per SM for the pass kernels on the first call.
// Arithmetic is FP32 (FMA) with the same Philox test matrix as the
// single-matrix path; tall matrices are stored row-major with 32 columns.
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.cuh"
#include "philox.cuh"

namespace rsvdgb {
namespace batched {

constexpr int LB = 32;   // panel width
constexpr int RB = 128;  // rows per row-block item
constexpr int CB = 64;   // columns per column-block item
constexpr int NT = 256;  // threads per CTA of the grouped kernels

struct MatDev {
    const float* A;
    int64_t lda;
    int64_t M, N;         // logical rows >= logical columns
    int trans;            // logical = stored^T
    int l;                // sketch width
    int64_t offM, offN;   // first row in the M-side / N-side pools
    int64_t slot0;        // first Gram-partial slot of this matrix
    float* d;
    float* Ulog;          // logical left vectors (user's U, or V when swapped)
    int64_t ldUl;
    int nUl;
    float* Vlog;          // logical right vectors
    int64_t ldVl;
    int nVl;
    int k;
};

struct Item {
    int32_t b;
    int32_t blk;
};

__device__ __forceinline__ float aget(const MatDev& D, int64_t i, int64_t j)
{
    return D.trans ? D.A[j * D.lda + i] : D.A[i * D.lda + j];
}

// ------------------------------------------------------------------ Omega
__global__ void omega_kernel(const MatDev* __restrict__ D, const int64_t* __restrict__ qoff, int B, int64_t nquads,
                             uint64_t seed, int sdist, float* __restrict__ P)
{
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nquads;
         g += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = B - 1;
        while (lo < hi) {  // last b with qoff[b] <= g
            const int mid = (lo + hi + 1) >> 1;
            if (qoff[mid] <= g)
                lo = mid;
            else
                hi = mid - 1;
        }
        const MatDev& M = D[lo];
        const int64_t r = g - qoff[lo];
        for (int j = 0; j < LB; ++j) {
            float v[4] = {0.f, 0.f, 0.f, 0.f};
            if (j < M.l) philox::omega4(seed, r, j, sdist, v);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int64_t i = 4 * r + t;
                if (i < M.N) P[(M.offN + i) * LB + j] = v[t];
            }
        }
    }
}

// ------------------------------------------------------------------ Gram partial of a RB x 32 tile in smem
// Ts: RB rows of 33 floats; writes G = Ts^T Ts (32 x 32) to out.
__device__ __forceinline__ void tile_gram(const float* Ts, int rows, float* __restrict__ out)
{
    for (int e = threadIdx.x; e < LB * LB; e += NT) {
        const int a = e >> 5, c = e & 31;
        float acc = 0.f;
        for (int i = 0; i < rows; ++i) acc = fmaf(Ts[i * 33 + a], Ts[i * 33 + c], acc);
        out[e] = acc;
    }
}

// Cross Gram X^T Y of two RB x 32 tiles.
__device__ __forceinline__ void tile_cross(const float* Xs, const float* Ys, int rows, float* __restrict__ out)
{
    for (int e = threadIdx.x; e < LB * LB; e += NT) {
        const int a = e >> 5, c = e & 31;
        float acc = 0.f;
        for (int i = 0; i < rows; ++i) acc = fmaf(Xs[i * 33 + a], Ys[i * 33 + c], acc);
        out[e] = acc;
    }
}

// ------------------------------------------------------------------ Y = A_log P  (row-block items)
// Y[i][:] = sum_j A_log(i, j) P[j][:] for RB logical rows; optional Gram partial
// of the tile and ||A||_F^2 accumulation (per matrix, FP64 atomics).
__global__ void __launch_bounds__(NT, 3) pass_a_kernel(const MatDev* __restrict__ D, const Item* __restrict__ items,
                                                    int nitems, int* cursor, const float* __restrict__ P,
                                                    float* __restrict__ Y, float* __restrict__ part,
                                                    double* __restrict__ fro2)
{
    __shared__ __align__(16) float As[32][RB + 4];
    __shared__ __align__(16) float Ps[32][LB];
    __shared__ float Ts[RB * 33];
    __shared__ int cur;
    const int tid = threadIdx.x;
    const int ty = tid >> 3, tx = tid & 7;  // 32 x 8 threads: rows 4ty.., cols 4tx..
    for (;;) {
        if (tid == 0) cur = atomicAdd(cursor, 1);
        __syncthreads();
        const int it = cur;
        __syncthreads();
        if (it >= nitems) break;
        const Item item = items[it];
        const MatDev Mt = D[item.b];
        const int64_t r0 = (int64_t)item.blk * RB;
        const int rows = (int)min((int64_t)RB, Mt.M - r0);
        float acc[4][4] = {};
        float sq = 0.f;
        // next chunk in registers while the current one is multiplied
        constexpr int EA = RB * 32 / NT, EP = 32 * LB / NT;
        float ra[EA], rp[EP];
        auto load_chunk = [&](int64_t k0) {
#pragma unroll
            for (int q = 0; q < EA; ++q) {
                const int e = tid + q * NT;
                int i, kk;
                if (Mt.trans) {  // logical row i = stored column: contiguous over i
                    i = e % RB;
                    kk = e / RB;
                } else {
                    kk = e % 32;
                    i = e / 32;
                }
                ra[q] = (i < rows && k0 + kk < Mt.N) ? aget(Mt, r0 + i, k0 + kk) : 0.f;
            }
#pragma unroll
            for (int q = 0; q < EP; ++q) {
                const int e = tid + q * NT;
                const int kk = e >> 5, c = e & 31;
                rp[q] = (k0 + kk < Mt.N) ? P[(Mt.offN + k0 + kk) * LB + c] : 0.f;
            }
        };
        load_chunk(0);
        for (int64_t k0 = 0; k0 < Mt.N; k0 += 32) {
            // A chunk: RB rows x 32 columns of the logical matrix, k-major in smem
#pragma unroll
            for (int q = 0; q < EA; ++q) {
                const int e = tid + q * NT;
                int i, kk;
                if (Mt.trans) {
                    i = e % RB;
                    kk = e / RB;
                } else {
                    kk = e % 32;
                    i = e / 32;
                }
                As[kk][i] = ra[q];
                sq = fmaf(ra[q], ra[q], sq);
            }
#pragma unroll
            for (int q = 0; q < EP; ++q) {
                const int e = tid + q * NT;
                Ps[e >> 5][e & 31] = rp[q];
            }
            __syncthreads();
            if (k0 + 32 < Mt.N) load_chunk(k0 + 32);
#pragma unroll 8
            for (int kk = 0; kk < 32; ++kk) {
                const float4 a4 = *(const float4*)&As[kk][4 * ty];
                const float4 p4 = *(const float4*)&Ps[kk][4 * tx];
                const float av[4] = {a4.x, a4.y, a4.z, a4.w};
                const float pv[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[i][c] = fmaf(av[i], pv[c], acc[i][c]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = 4 * ty + i;
#pragma unroll
            for (int c = 0; c < 4; ++c) Ts[r * 33 + 4 * tx + c] = (r < rows) ? acc[i][c] : 0.f;
        }
        __syncthreads();
        for (int e = tid; e < rows * LB; e += NT) {
            const int r = e >> 5, c = e & 31;
            Y[(Mt.offM + r0 + r) * LB + c] = Ts[r * 33 + c];
        }
        if (part) tile_gram(Ts, rows, part + (Mt.slot0 + item.blk) * (int64_t)(LB * LB));
        if (fro2) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
            if ((tid & 31) == 0) atomicAdd(&fro2[item.b], (double)sq);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ W = A_log^T Y (column-block items)
// W[c][:] = sum_i A_log(i, c) Y[i][:] for CB logical columns over all rows;
// optional right factor T (Z = W T) and Gram partial of the result.
__global__ void __launch_bounds__(NT) pass_at_kernel(const MatDev* __restrict__ D, const Item* __restrict__ items,
                                                     int nitems, int* cursor, const float* __restrict__ Y,
                                                     const float* __restrict__ T, float* __restrict__ W,
                                                     float* __restrict__ part)
{
    __shared__ __align__(16) float As[32][CB + 4];
    __shared__ __align__(16) float Ys[32][LB];
    __shared__ float Ts[CB * 33];
    __shared__ float Tm[LB * LB];
    __shared__ int cur;
    const int tid = threadIdx.x;
    const int ty = tid >> 3, tx = tid & 7;  // 32 x 8: columns 2ty.., outputs 4tx..
    for (;;) {
        if (tid == 0) cur = atomicAdd(cursor, 1);
        __syncthreads();
        const int it = cur;
        __syncthreads();
        if (it >= nitems) break;
        const Item item = items[it];
        const MatDev Mt = D[item.b];
        const int64_t c0 = (int64_t)item.blk * CB;
        const int cols = (int)min((int64_t)CB, Mt.N - c0);
        float acc[2][4] = {};
        constexpr int EA = 32 * CB / NT, EY = 32 * LB / NT;
        float ra[EA], ry[EY];
        auto load_chunk = [&](int64_t i0) {
#pragma unroll
            for (int q = 0; q < EA; ++q) {
                const int e = tid + q * NT;
                int ii, c;
                if (Mt.trans) {  // A_log(i, c) = S[c][i]: contiguous over i
                    ii = e % 32;
                    c = e / 32;
                } else {
                    c = e % CB;
                    ii = e / CB;
                }
                ra[q] = (c < cols && i0 + ii < Mt.M) ? aget(Mt, i0 + ii, c0 + c) : 0.f;
            }
#pragma unroll
            for (int q = 0; q < EY; ++q) {
                const int e = tid + q * NT;
                const int ii = e >> 5, c = e & 31;
                ry[q] = (i0 + ii < Mt.M) ? Y[(Mt.offM + i0 + ii) * LB + c] : 0.f;
            }
        };
        load_chunk(0);
        for (int64_t i0 = 0; i0 < Mt.M; i0 += 32) {
#pragma unroll
            for (int q = 0; q < EA; ++q) {
                const int e = tid + q * NT;
                int ii, c;
                if (Mt.trans) {
                    ii = e % 32;
                    c = e / 32;
                } else {
                    c = e % CB;
                    ii = e / CB;
                }
                As[ii][c] = ra[q];
            }
#pragma unroll
            for (int q = 0; q < EY; ++q) {
                const int e = tid + q * NT;
                Ys[e >> 5][e & 31] = ry[q];
            }
            __syncthreads();
            if (i0 + 32 < Mt.M) load_chunk(i0 + 32);
            // each 32-row chunk is summed on its own and then added to the
            // running sum: the FP32 error grows like 32 + M / 32, not M
            float cacc[2][4] = {};
#pragma unroll 8
            for (int ii = 0; ii < 32; ++ii) {
                const float2 a2 = *(const float2*)&As[ii][2 * ty];
                const float4 y4 = *(const float4*)&Ys[ii][4 * tx];
                const float av[2] = {a2.x, a2.y};
                const float yv[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) cacc[a][c] = fmaf(av[a], yv[c], cacc[a][c]);
            }
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][c] += cacc[a][c];
            __syncthreads();
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) Ts[(2 * ty + a) * 33 + 4 * tx + c] = (2 * ty + a < cols) ? acc[a][c] : 0.f;
        if (T)
            for (int e = tid; e < LB * LB; e += NT) Tm[e] = T[(int64_t)item.b * LB * LB + e];
        __syncthreads();
        if (T) {
            // Z = W T, row by row (CB x 32 times 32 x 32)
            float z[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = tid + q * NT;
                const int r = e >> 5, c = e & 31;
                float s = 0.f;
                for (int t = 0; t < LB; ++t) s = fmaf(Ts[r * 33 + t], Tm[t * LB + c], s);
                z[q] = s;
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = tid + q * NT;
                Ts[(e >> 5) * 33 + (e & 31)] = z[q];
            }
            __syncthreads();
        }
        for (int e = tid; e < cols * LB; e += NT) {
            const int r = e >> 5, c = e & 31;
            W[(Mt.offN + c0 + r) * LB + c] = Ts[r * 33 + c];
        }
        if (part) tile_gram(Ts, cols, part + (Mt.slot0 + item.blk) * (int64_t)(LB * LB));
        __syncthreads();
    }
}

// ------------------------------------------------------------------ X T on row blocks (M side or N side)
// out = in T (rows x 32) for RB-row items; writes out when it is non-null
// (in place allowed); Gram partial of the product (part) and/or cross Gram
// out^T x2 (part2 with x2 a second pool on the same side).
__global__ void __launch_bounds__(NT) tall_small_kernel(const MatDev* __restrict__ D, const Item* __restrict__ items,
                                                        int nitems, int* cursor, int nside, const float* in,
                                                        const float* __restrict__ T, float* out, float* part,
                                                        const float* __restrict__ x2, float* part2)
{
    __shared__ float Ts[RB * 33];
    __shared__ float Xs[RB * 33];
    __shared__ float Tm[LB * LB];
    __shared__ int cur;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) cur = atomicAdd(cursor, 1);
        __syncthreads();
        const int it = cur;
        __syncthreads();
        if (it >= nitems) break;
        const Item item = items[it];
        const MatDev Mt = D[item.b];
        const int64_t rows_all = nside ? Mt.N : Mt.M;
        const int64_t off = nside ? Mt.offN : Mt.offM;
        const int64_t r0 = (int64_t)item.blk * RB;
        const int rows = (int)min((int64_t)RB, rows_all - r0);
        for (int e = tid; e < LB * LB; e += NT) Tm[e] = T[(int64_t)item.b * LB * LB + e];
        for (int e = tid; e < RB * LB; e += NT) {
            const int r = e >> 5, c = e & 31;
            Xs[r * 33 + c] = (r < rows) ? in[(off + r0 + r) * LB + c] : 0.f;
        }
        __syncthreads();
        for (int e = tid; e < RB * LB; e += NT) {
            const int r = e >> 5, c = e & 31;
            float s = 0.f;
            for (int t = 0; t < LB; ++t) s = fmaf(Xs[r * 33 + t], Tm[t * LB + c], s);
            Ts[r * 33 + c] = (r < rows) ? s : 0.f;
        }
        __syncthreads();
        if (out)
            for (int e = tid; e < rows * LB; e += NT) {
                const int r = e >> 5, c = e & 31;
                out[(off + r0 + r) * LB + c] = Ts[r * 33 + c];
            }
        if (part) tile_gram(Ts, rows, part + (Mt.slot0 + item.blk) * (int64_t)(LB * LB));
        if (part2) {
            for (int e = tid; e < RB * LB; e += NT) {
                const int r = e >> 5, c = e & 31;
                Xs[r * 33 + c] = (r < rows) ? x2[(off + r0 + r) * LB + c] : 0.f;
            }
            __syncthreads();
            tile_cross(Ts, Xs, rows, part2 + (Mt.slot0 + item.blk) * (int64_t)(LB * LB));
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ per-matrix small kernels (one warp each)
// Sum of the nslots partials (32 x 32) of matrix b into column `lane` (g[t] = G[t][lane]).
__device__ __forceinline__ void reduce_parts(const float* __restrict__ part, int64_t slot0, int nslots, int lane,
                                             float (&g)[LB])
{
#pragma unroll
    for (int t = 0; t < LB; ++t) g[t] = 0.f;
    for (int s = 0; s < nslots; ++s) {
        const float* p = part + (slot0 + s) * (int64_t)(LB * LB);
#pragma unroll
        for (int t = 0; t < LB; ++t) g[t] += p[t * LB + lane];
    }
}

// Cholesky of the reduced Gram (+ shift on breakdown) and T = R^{-1}; also R.
// nside / block: which row blocking produced the partials.
__global__ void chol_kernel(const MatDev* __restrict__ D, int B, const float* __restrict__ part, int nside,
                            int block, float* __restrict__ Tout, float* __restrict__ Rout, int* status,
                            int* breakdowns)
{
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= B) return;
    const MatDev Mt = D[b];
    const int64_t rows = nside ? Mt.N : Mt.M;
    const int nslots = (int)((rows + block - 1) / block);
    float g[LB];
    reduce_parts(part, Mt.slot0, nslots, lane, g);
    // pad outside the l x l leading block with the identity
#pragma unroll
    for (int t = 0; t < LB; ++t)
        if (t >= Mt.l || lane >= Mt.l) g[t] = (t == lane) ? 1.f : 0.f;
    float maxd = 0.f;
#pragma unroll
    for (int t = 0; t < LB; ++t)
        if (t == lane) maxd = g[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxd = fmaxf(maxd, __shfl_xor_sync(0xffffffffu, maxd, o));
    float c[LB];
    bool ok = false;
    for (int attempt = 0; attempt < 4 && !ok; ++attempt) {
        const float shift = attempt == 0 ? 0.f : maxd * 1e-6f * powf(100.f, (float)(attempt - 1));
#pragma unroll
        for (int t = 0; t < LB; ++t) c[t] = (t <= lane) ? g[t] + ((t == lane) ? shift : 0.f) : 0.f;
        bool bad = false;
#pragma unroll
        for (int i = 0; i < LB; ++i) {
            const float piv = __shfl_sync(0xffffffffu, c[i], i);
            if (!(piv > 0.f) || !isfinite(piv)) bad = true;
            const float rinv = rsqrtf(fmaxf(piv, 1e-30f));
            if (lane > i) c[i] *= rinv;
            if (lane == i) c[i] = piv * rinv;
#pragma unroll
            for (int t = i + 1; t < LB; ++t) {
                const float rt = __shfl_sync(0xffffffffu, c[i], t);  // R(i, t)
                if (lane >= t) c[t] -= rt * c[i];
            }
        }
        ok = !bad;
        if (bad && lane == 0) {
            atomicAdd(breakdowns, 1);
            if (attempt == 3) atomicExch(status, RSVDGB_ERR_BREAKDOWN);
        }
    }
    // c[t] = R(t, lane).  T = R^{-1}: lane j solves R x = e_j by back substitution.
    float x[LB];
#pragma unroll
    for (int t = 0; t < LB; ++t) x[t] = 0.f;
#pragma unroll
    for (int i = LB - 1; i >= 0; --i) {
        float acc = (i == lane) ? 1.f : 0.f;
#pragma unroll
        for (int t = i + 1; t < LB; ++t) {
            const float rit = __shfl_sync(0xffffffffu, c[i], t);  // R(i, t) lives in lane t
            acc -= rit * x[t];
        }
        const float rii = __shfl_sync(0xffffffffu, c[i], i);
        x[i] = (i <= lane) ? acc / rii : 0.f;
    }
    float* To = Tout + (int64_t)b * LB * LB;
#pragma unroll
    for (int t = 0; t < LB; ++t) To[t * LB + lane] = x[t];
    if (Rout) {
        float* Ro = Rout + (int64_t)b * LB * LB;
#pragma unroll
        for (int t = 0; t < LB; ++t) Ro[t * LB + lane] = c[t];
    }
}

// C = A B for 32 x 32 per-matrix factors.
__global__ void small_mul_kernel(int B, const float* __restrict__ A, const float* __restrict__ Bm,
                                 float* __restrict__ C)
{
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= B) return;
    const float* a = A + (int64_t)b * LB * LB;
    const float* bm = Bm + (int64_t)b * LB * LB;
    float* cc = C + (int64_t)b * LB * LB;
    for (int i = 0; i < LB; ++i) {
        float acc = 0.f;
        for (int t = 0; t < LB; ++t) acc = fmaf(a[i * LB + t], bm[t * LB + lane], acc);
        cc[i * LB + lane] = acc;
    }
}

// One-sided Jacobi SVD of M = R_B^T (R_B reduced from the cross-Gram partials),
// one warp per matrix, lanes over rows; outputs sorted sigma, Ut (l x l) and
// J (right vectors), row-major 32 x 32 per matrix.
__global__ void jacobi_kernel(const MatDev* __restrict__ D, int B, const float* __restrict__ part, int block,
                              float* __restrict__ sigma, float* __restrict__ Ut, float* __restrict__ Jt,
                              int* sweeps_max)
{
    const int wib = threadIdx.x >> 5;
    const int b = blockIdx.x * (blockDim.x >> 5) + wib;
    const int lane = threadIdx.x & 31;
    extern __shared__ float sh[];
    float* Mc = sh + wib * 2 * LB * (LB + 1);  // column-major, 33 stride
    float* Jc = Mc + LB * (LB + 1);
    if (b >= B) return;
    const MatDev Mt = D[b];
    const int nslots = (int)((Mt.N + block - 1) / block);
    float g[LB];
    reduce_parts(part, Mt.slot0, nslots, lane, g);  // g[t] = R_B(t, lane)  (R_B = Q_B^T B^T)
    // M = R_B^T: column c of M = row c of R_B; element (i, c) = R_B(c, i)
#pragma unroll
    for (int t = 0; t < LB; ++t) {
        // lane holds column `lane` of R_B = row `lane` of M; store M(lane, t) = R_B(t, lane)
        Mc[t * (LB + 1) + lane] = (t < Mt.l && lane < Mt.l) ? g[t] : 0.f;
        Jc[t * (LB + 1) + lane] = (t == lane) ? 1.f : 0.f;
    }
    __syncwarp();
    const float tol = 4.f * sqrtf((float)LB) * 5.9604645e-8f;
    int sweep = 0;
    for (; sweep < 30; ++sweep) {
        bool any = false;
        for (int round = 0; round < LB - 1; ++round) {
            for (int t = 0; t < LB / 2; ++t) {
                int a = LB - 1, bb = round;
                if (t != 0) {
                    a = round + t;
                    if (a >= LB - 1) a -= LB - 1;
                    bb = round - t;
                    if (bb < 0) bb += LB - 1;
                }
                const float x = Mc[a * (LB + 1) + lane], y = Mc[bb * (LB + 1) + lane];
                float al = x * x, be = y * y, ga = x * y;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    al += __shfl_xor_sync(0xffffffffu, al, o);
                    be += __shfl_xor_sync(0xffffffffu, be, o);
                    ga += __shfl_xor_sync(0xffffffffu, ga, o);
                }
                if (ga != 0.f && fabsf(ga) > tol * sqrtf(al * be)) {
                    const float zeta = (be - al) / (2.f * ga);
                    const float tt = copysignf(1.f, zeta) / (fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
                    const float cs = 1.0f / sqrtf(fmaf(tt, tt, 1.f));
                    const float sn = cs * tt;
                    Mc[a * (LB + 1) + lane] = cs * x - sn * y;
                    Mc[bb * (LB + 1) + lane] = sn * x + cs * y;
                    const float ja = Jc[a * (LB + 1) + lane], jb = Jc[bb * (LB + 1) + lane];
                    Jc[a * (LB + 1) + lane] = cs * ja - sn * jb;
                    Jc[bb * (LB + 1) + lane] = sn * ja + cs * jb;
                    any = true;
                }
                __syncwarp();
            }
        }
        if (!any) break;
    }
    if (lane == 0) atomicMax(sweeps_max, sweep + 1);
    // sigma_c = ||W_c|| / ||J_c||, ranks by descending value
    float wn = 0.f, jn = 0.f;
    for (int i = 0; i < LB; ++i) {
        const float w = Mc[lane * (LB + 1) + i], j = Jc[lane * (LB + 1) + i];
        wn = fmaf(w, w, wn);
        jn = fmaf(j, j, jn);
    }
    wn = sqrtf(wn);
    jn = sqrtf(jn);
    const float sv = (jn > 0.f) ? wn / jn : 0.f;
    // ranks by descending sigma, ties by column; NaN ranks as -1 so the ranks
    // form a permutation
    const float key = (sv == sv) ? sv : -1.f;
    int rank = 0;
    for (int o = 0; o < LB; ++o) {
        const float so = __shfl_sync(0xffffffffu, key, o);
        rank += (so > key) || (so == key && o < lane);
    }
    float* sg = sigma + (int64_t)b * LB;
    float* ut = Ut + (int64_t)b * LB * LB;
    float* jt = Jt + (int64_t)b * LB * LB;
    sg[rank] = sv;
    for (int i = 0; i < LB; ++i) {
        ut[i * LB + rank] = (wn > 0.f) ? Mc[lane * (LB + 1) + i] / wn : 0.f;
        jt[i * LB + rank] = (jn > 0.f) ? Jc[lane * (LB + 1) + i] / jn : 0.f;
    }
}

// ------------------------------------------------------------------ outputs
// Row-block items on the M side write U_log = Q Ut (first nUl columns) and
// the singular values; on the N side V_log = Q_B J (first nVl columns).
__global__ void __launch_bounds__(NT) output_kernel(const MatDev* __restrict__ D, const Item* __restrict__ items,
                                                    int nitems, int nside, const float* __restrict__ X,
                                                    const float* __restrict__ S, const float* __restrict__ sigma)
{
    __shared__ float Sm[LB * LB];
    const int it = blockIdx.x;
    if (it >= nitems) return;
    const Item item = items[it];
    const MatDev Mt = D[item.b];
    const int64_t rows_all = nside ? Mt.N : Mt.M;
    const int64_t off = nside ? Mt.offN : Mt.offM;
    const int ncol = nside ? Mt.nVl : Mt.nUl;
    float* out = nside ? Mt.Vlog : Mt.Ulog;
    const int64_t ld = nside ? Mt.ldVl : Mt.ldUl;
    for (int e = threadIdx.x; e < LB * LB; e += NT) Sm[e] = S[(int64_t)item.b * LB * LB + e];
    __syncthreads();
    if (!nside && item.blk == 0)
        for (int i = threadIdx.x; i < Mt.k; i += NT) Mt.d[i] = sigma[(int64_t)item.b * LB + i];
    if (ncol <= 0 || !out) return;
    const int64_t r0 = (int64_t)item.blk * RB;
    const int rows = (int)min((int64_t)RB, rows_all - r0);
    for (int e = threadIdx.x; e < rows * ncol; e += NT) {
        const int r = e / ncol, c = e % ncol;
        const float* x = X + (off + r0 + r) * LB;
        float s = 0.f;
        for (int t = 0; t < Mt.l; ++t) s = fmaf(x[t], Sm[t * LB + c], s);
        out[(r0 + r) * ld + c] = s;
    }
}

__global__ void finalize_kernel(const MatDev* __restrict__ D, int B, const float* __restrict__ sigma,
                                const double* __restrict__ fro2, const int* status, const int* breakdowns,
                                const int* sweeps, int q, rsvdgb_info* infos)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B || !infos) return;
    const MatDev Mt = D[b];
    double sb = 0.0, sk = 0.0;
    for (int i = 0; i < Mt.l; ++i) {
        const double s = sigma[(int64_t)b * LB + i];
        sb += s * s;
        if (i < Mt.k) sk += s * s;
    }
    rsvdgb_info inf{};
    inf.status = *status;
    if (!isfinite(fro2[b])) inf.status = RSVDGB_ERR_NONFINITE;
    inf.q_used = q;
    inf.p_used = Mt.l - Mt.k;
    inf.l = Mt.l;
    inf.fro2_A = fro2[b];
    inf.fro2_B = sb;
    inf.err2_QB = fro2[b] - sb;
    inf.err2_k = fro2[b] - sk;
    inf.breakdowns = *breakdowns;
    inf.engine = RSVDGB_ENGINE_SIMT;
    inf.jacobi_sweeps = *sweeps;
    inf.orth_max = -1.f;  // not measured in the batched call
    infos[b] = inf;
}

}  // namespace batched

// ===================================================================== host plan
namespace {
struct HostItemLists {
    std::vector<batched::Item> mrows, nrows, ncols;
};
}  // namespace

struct BatchedPlan {
    // key
    std::vector<rsvdgb_matrix_desc> descs;
    std::vector<rsvdgb_result_desc> outs;
    int k = 0, p = 0, q = 0, sdist = 0;
    uint64_t seed = 0;
    int device = -1;
    // device memory (one allocation)
    void* mem = nullptr;
    size_t mem_bytes = 0;
    batched::MatDev* D = nullptr;
    batched::Item *it_m = nullptr, *it_nr = nullptr, *it_nc = nullptr;
    int n_m = 0, n_nr = 0, n_nc = 0;
    int64_t* qoff = nullptr;
    int64_t nquads = 0;
    float *P = nullptr, *Y = nullptr, *W = nullptr, *Z = nullptr, *part = nullptr, *part2 = nullptr;
    float *T = nullptr, *T1 = nullptr, *T2 = nullptr, *Tc = nullptr, *sig = nullptr, *Ut = nullptr, *Jt = nullptr;
    double* fro2 = nullptr;
    int *cursors = nullptr, *status = nullptr, *breakdowns = nullptr, *sweeps = nullptr;
    rsvdgb_info* infos_dev = nullptr;
    // tuned launch shape of the grouped kernels
    int ctas_per_sm = 2;
    bool tuned = false;
    cudaGraphExec_t graph = nullptr;
    rsvdgb_info* graph_infos = nullptr;  // infos pointer baked into the graph
    cudaStream_t graph_stream = nullptr;
    int B = 0;
    int kernels_per_run = 0;
};

void destroy_plan(BatchedPlan* pl)
{
    if (!pl) return;
    if (pl->graph) cudaGraphExecDestroy(pl->graph);
    if (pl->mem) cudaFree(pl->mem);
    delete pl;
}

namespace {

int build_plan(BatchedPlan* pl, int B, const rsvdgb_matrix_desc* descs, int k, const rsvdgb_opts& o,
               const rsvdgb_result_desc* outs, int device)
{
    using namespace batched;
    pl->B = B;
    pl->descs.assign(descs, descs + B);
    pl->outs.assign(outs, outs + B);
    pl->k = k;
    pl->p = o.p;
    pl->q = o.q;
    pl->sdist = o.sdist;
    pl->seed = o.seed;
    pl->device = device;
    // order: largest matrices first (their items enter the queues first)
    std::vector<int> order(B);
    for (int b = 0; b < B; ++b) order[b] = b;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return descs[x].m * descs[x].n > descs[y].m * descs[y].n;
    });
    std::vector<MatDev> hd(B);
    std::vector<int64_t> qoff(B);
    int64_t offM = 0, offN = 0, slot = 0, quads = 0;
    HostItemLists L;
    for (int b = 0; b < B; ++b) {
        const rsvdgb_matrix_desc& ds = descs[b];
        const rsvdgb_result_desc& rs = outs[b];
        MatDev& m = hd[b];
        m.A = (const float*)ds.A;
        m.lda = ds.lda;
        m.trans = ds.m < ds.n;
        m.M = std::max(ds.m, ds.n);
        m.N = std::min(ds.m, ds.n);
        m.l = (int)std::min<int64_t>((int64_t)k + o.p, m.N);
        m.k = k;
        m.offM = offM;
        m.offN = offN;
        m.slot0 = slot;
        m.d = rs.d;
        if (!m.trans) {
            m.Ulog = rs.U; m.ldUl = rs.ldu; m.nUl = rs.U ? k : 0;
            m.Vlog = rs.V; m.ldVl = rs.ldv; m.nVl = rs.V ? k : 0;
        } else {
            m.Ulog = rs.V; m.ldUl = rs.ldv; m.nUl = rs.V ? k : 0;
            m.Vlog = rs.U; m.ldVl = rs.ldu; m.nVl = rs.U ? k : 0;
        }
        offM += m.M;
        offN += m.N;
        slot += std::max(ceil_div(m.M, RB), ceil_div(m.N, CB));
        qoff[b] = quads;
        quads += ceil_div(m.N, 4);
    }
    for (int oi = 0; oi < B; ++oi) {
        const int b = order[oi];
        for (int64_t r = 0; r < ceil_div(hd[b].M, RB); ++r) L.mrows.push_back({b, (int32_t)r});
        for (int64_t r = 0; r < ceil_div(hd[b].N, RB); ++r) L.nrows.push_back({b, (int32_t)r});
        for (int64_t c = 0; c < ceil_div(hd[b].N, CB); ++c) L.ncols.push_back({b, (int32_t)c});
    }
    pl->n_m = (int)L.mrows.size();
    pl->n_nr = (int)L.nrows.size();
    pl->n_nc = (int)L.ncols.size();
    pl->nquads = quads;
    // one allocation for everything
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (size_t)round_up((int64_t)off, 256);
        const size_t at = off;
        off += bytes;
        return at;
    };
    const size_t oD = take(sizeof(MatDev) * B);
    const size_t oIm = take(sizeof(Item) * pl->n_m);
    const size_t oInr = take(sizeof(Item) * pl->n_nr);
    const size_t oInc = take(sizeof(Item) * pl->n_nc);
    const size_t oQ = take(sizeof(int64_t) * B);
    const size_t oP = take(sizeof(float) * offN * LB);
    const size_t oY = take(sizeof(float) * offM * LB);
    const size_t oW = take(sizeof(float) * offN * LB);
    const size_t oZ = take(sizeof(float) * offN * LB);
    const size_t oPart = take(sizeof(float) * slot * LB * LB);
    const size_t oPart2 = take(sizeof(float) * slot * LB * LB);
    const size_t oT = take(sizeof(float) * B * LB * LB);
    const size_t oT1 = take(sizeof(float) * B * LB * LB);
    const size_t oT2 = take(sizeof(float) * B * LB * LB);
    const size_t oTc = take(sizeof(float) * B * LB * LB);
    const size_t oSig = take(sizeof(float) * B * LB);
    const size_t oUt = take(sizeof(float) * B * LB * LB);
    const size_t oJt = take(sizeof(float) * B * LB * LB);
    const size_t oF = take(sizeof(double) * B);
    const size_t oC = take(sizeof(int) * 64);
    const size_t oInf = take(sizeof(rsvdgb_info) * B);
    if (cudaMalloc(&pl->mem, off) != cudaSuccess) {
        cudaGetLastError();
        return RSVDGB_ERR_NOMEM;
    }
    pl->mem_bytes = off;
    char* base = (char*)pl->mem;
    pl->D = (MatDev*)(base + oD);
    pl->it_m = (Item*)(base + oIm);
    pl->it_nr = (Item*)(base + oInr);
    pl->it_nc = (Item*)(base + oInc);
    pl->qoff = (int64_t*)(base + oQ);
    pl->P = (float*)(base + oP);
    pl->Y = (float*)(base + oY);
    pl->W = (float*)(base + oW);
    pl->Z = (float*)(base + oZ);
    pl->part = (float*)(base + oPart);
    pl->part2 = (float*)(base + oPart2);
    pl->T = (float*)(base + oT);
    pl->T1 = (float*)(base + oT1);
    pl->T2 = (float*)(base + oT2);
    pl->Tc = (float*)(base + oTc);
    pl->sig = (float*)(base + oSig);
    pl->Ut = (float*)(base + oUt);
    pl->Jt = (float*)(base + oJt);
    pl->fro2 = (double*)(base + oF);
    pl->cursors = (int*)(base + oC);
    pl->status = pl->cursors + 40;
    pl->breakdowns = pl->cursors + 41;
    pl->sweeps = pl->cursors + 42;
    pl->infos_dev = (rsvdgb_info*)(base + oInf);
    RSVDGB_CUDA_TRY(cudaMemset(pl->mem, 0, off));
    RSVDGB_CUDA_TRY(cudaMemcpy(pl->D, hd.data(), sizeof(MatDev) * B, cudaMemcpyHostToDevice));
    RSVDGB_CUDA_TRY(cudaMemcpy(pl->it_m, L.mrows.data(), sizeof(Item) * pl->n_m, cudaMemcpyHostToDevice));
    RSVDGB_CUDA_TRY(cudaMemcpy(pl->it_nr, L.nrows.data(), sizeof(Item) * pl->n_nr, cudaMemcpyHostToDevice));
    RSVDGB_CUDA_TRY(cudaMemcpy(pl->it_nc, L.ncols.data(), sizeof(Item) * pl->n_nc, cudaMemcpyHostToDevice));
    RSVDGB_CUDA_TRY(cudaMemcpy(pl->qoff, qoff.data(), sizeof(int64_t) * B, cudaMemcpyHostToDevice));
    const int jsmem = 8 * 2 * LB * (LB + 1) * (int)sizeof(float);
    RSVDGB_CUDA_TRY(cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, jsmem));
    return RSVDGB_OK;
}

// Queue all stages of the batched rSVD on stream s.
void enqueue(BatchedPlan* pl, cudaStream_t s, int sm_count, rsvdgb_info* infos)
{
    using namespace batched;
    const int B = pl->B;
    const int grid = sm_count * pl->ctas_per_sm;
    const int warps_blocks = (B + 7) / 8;  // one warp per matrix, 8 per CTA
    int cur = 0;                           // next cursor slot
    auto cursor = [&]() { return pl->cursors + (cur++); };
    cudaMemsetAsync(pl->cursors, 0, sizeof(int) * 64, s);
    cudaMemsetAsync(pl->fro2, 0, sizeof(double) * B, s);

    omega_kernel<<<sm_count * 4, 256, 0, s>>>(pl->D, pl->qoff, B, pl->nquads, pl->seed, pl->sdist, pl->P);
    // step 3: Y = A Omega, Gram partials, ||A||_F^2
    pass_a_kernel<<<grid, NT, 0, s>>>(pl->D, pl->it_m, pl->n_m, cursor(), pl->P, pl->Y, pl->part, pl->fro2);
    chol_kernel<<<warps_blocks, 256, 0, s>>>(pl->D, B, pl->part, 0, RB, pl->T, nullptr, pl->status, pl->breakdowns);
    int launches = 3;
    for (int it = 0; it < pl->q; ++it) {
        // Q = Y T in place (one Cholesky step; only the span is carried
        // forward), then Z = A^T Q with the Gram partials of Z.  Forming Q
        // first keeps the directions of small singular values at their
        // relative accuracy (A^T Y T would carry them at sigma^2 / sigma_1^2
        // of A^T Y's columns).
        tall_small_kernel<<<grid, NT, 0, s>>>(pl->D, pl->it_m, pl->n_m, cursor(), 0, pl->Y, pl->T, pl->Y, nullptr,
                                              nullptr, nullptr);
        pass_at_kernel<<<grid, NT, 0, s>>>(pl->D, pl->it_nc, pl->n_nc, cursor(), pl->Y, nullptr, pl->Z, pl->part);
        chol_kernel<<<warps_blocks, 256, 0, s>>>(pl->D, B, pl->part, 1, CB, pl->T1, nullptr, pl->status,
                                                 pl->breakdowns);
        // Gram of Z T1 (not stored), then T2 and Tc = T1 T2
        tall_small_kernel<<<grid, NT, 0, s>>>(pl->D, pl->it_nr, pl->n_nr, cursor(), 1, pl->Z, pl->T1, nullptr,
                                              pl->part, nullptr, nullptr);
        chol_kernel<<<warps_blocks, 256, 0, s>>>(pl->D, B, pl->part, 1, RB, pl->T2, nullptr, pl->status,
                                                 pl->breakdowns);
        small_mul_kernel<<<warps_blocks, 256, 0, s>>>(B, pl->T1, pl->T2, pl->Tc);
        // Q_n = Z Tc into the panel
        tall_small_kernel<<<grid, NT, 0, s>>>(pl->D, pl->it_nr, pl->n_nr, cursor(), 1, pl->Z, pl->Tc, pl->P,
                                              nullptr, nullptr, nullptr);
        // Y = A Q_n
        pass_a_kernel<<<grid, NT, 0, s>>>(pl->D, pl->it_m, pl->n_m, cursor(), pl->P, pl->Y, pl->part, nullptr);
        chol_kernel<<<warps_blocks, 256, 0, s>>>(pl->D, B, pl->part, 0, RB, pl->T, nullptr, pl->status,
                                                 pl->breakdowns);
        launches += 9;
    }
    // step 9: Q = qr(Y) by CholeskyQR2: Gram of Y T (not stored), T2, Q = Y (T T2) in place
    tall_small_kernel<<<grid, NT, 0, s>>>(pl->D, pl->it_m, pl->n_m, cursor(), 0, pl->Y, pl->T, nullptr, pl->part,
                                          nullptr, nullptr);
    chol_kernel<<<warps_blocks, 256, 0, s>>>(pl->D, B, pl->part, 0, RB, pl->T2, nullptr, pl->status,
                                             pl->breakdowns);
    small_mul_kernel<<<warps_blocks, 256, 0, s>>>(B, pl->T, pl->T2, pl->Tc);
    tall_small_kernel<<<grid, NT, 0, s>>>(pl->D, pl->it_m, pl->n_m, cursor(), 0, pl->Y, pl->Tc, pl->Y, nullptr,
                                          nullptr, nullptr);
    // step 10: B^T = A^T Q with Gram partials
    pass_at_kernel<<<grid, NT, 0, s>>>(pl->D, pl->it_nc, pl->n_nc, cursor(), pl->Y, nullptr, pl->W, pl->part);
    chol_kernel<<<warps_blocks, 256, 0, s>>>(pl->D, B, pl->part, 1, CB, pl->T1, nullptr, pl->status,
                                             pl->breakdowns);
    tall_small_kernel<<<grid, NT, 0, s>>>(pl->D, pl->it_nr, pl->n_nr, cursor(), 1, pl->W, pl->T1, nullptr, pl->part,
                                          nullptr, nullptr);
    chol_kernel<<<warps_blocks, 256, 0, s>>>(pl->D, B, pl->part, 1, RB, pl->T2, nullptr, pl->status,
                                             pl->breakdowns);
    small_mul_kernel<<<warps_blocks, 256, 0, s>>>(B, pl->T1, pl->T2, pl->Tc);
    // Q_B = B^T Tc (panel pool) and R_B = Q_B^T B^T (cross-Gram partials)
    tall_small_kernel<<<grid, NT, 0, s>>>(pl->D, pl->it_nr, pl->n_nr, cursor(), 1, pl->W, pl->Tc, pl->P, nullptr,
                                          pl->W, pl->part2);
    // SVD of the small factor, then U = Q Ut and V = Q_B J
    const size_t jsmem = 8 * 2 * LB * (LB + 1) * sizeof(float);
    jacobi_kernel<<<warps_blocks, 256, jsmem, s>>>(pl->D, B, pl->part2, RB, pl->sig, pl->Ut, pl->Jt, pl->sweeps);
    output_kernel<<<pl->n_m, NT, 0, s>>>(pl->D, pl->it_m, pl->n_m, 0, pl->Y, pl->Ut, pl->sig);
    output_kernel<<<pl->n_nr, NT, 0, s>>>(pl->D, pl->it_nr, pl->n_nr, 1, pl->P, pl->Jt, pl->sig);
    finalize_kernel<<<(B + 127) / 128, 128, 0, s>>>(pl->D, B, pl->sig, pl->fro2, pl->status, pl->breakdowns,
                                                     pl->sweeps, pl->q, infos);
    launches += 16;
    pl->kernels_per_run = launches;
}

}  // namespace

// Entry used by the C ABI (rsvd.cu).  Builds (or reuses) the plan for this
// batch layout, tunes the grouped-kernel grid on first use, captures the
// stages in a CUDA graph and launches it on `stream`.
int batched_rsvd(BatchedPlan** cache, int device, int sm_count, cudaStream_t stream, int B,
                 const rsvdgb_matrix_desc* descs, int k, const rsvdgb_opts& o, const rsvdgb_result_desc* outs,
                 rsvdgb_info* infos)
{
    BatchedPlan* pl = *cache;
    bool same = pl && pl->B == B && pl->k == k && pl->p == o.p && pl->q == o.q && pl->sdist == o.sdist &&
                pl->seed == o.seed && pl->device == device &&
                std::memcmp(pl->descs.data(), descs, sizeof(rsvdgb_matrix_desc) * B) == 0 &&
                std::memcmp(pl->outs.data(), outs, sizeof(rsvdgb_result_desc) * B) == 0;
    if (!same) {
        destroy_plan(pl);
        *cache = nullptr;
        pl = new BatchedPlan();
        const int rc = build_plan(pl, B, descs, k, o, outs, device);
        if (rc) {
            destroy_plan(pl);
            return rc;
        }
        *cache = pl;
    }
    if (!pl->tuned) {
        // the tuning runs read A on a private stream: let the caller's stream
        // finish producing it first
        RSVDGB_CUDA_TRY(cudaStreamSynchronize(stream));
        // autotune: resident CTAs per SM of the grouped kernels (1, 2 or 4),
        // one timed run each on a private stream
        cudaStream_t ts;
        RSVDGB_CUDA_TRY(cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking));
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        int best_c = 2;
        const int cands[3] = {2, 3, 4};
        for (int ci = 0; ci < 3; ++ci) {
            pl->ctas_per_sm = cands[ci];
            enqueue(pl, ts, sm_count, pl->infos_dev);  // warm
            cudaEventRecord(e0, ts);
            enqueue(pl, ts, sm_count, pl->infos_dev);
            cudaEventRecord(e1, ts);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) {
                best = ms;
                best_c = cands[ci];
            }
        }
        pl->ctas_per_sm = best_c;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaStreamDestroy(ts);
        pl->tuned = true;
        RSVDGB_CUDA_TRY(cudaGetLastError());
    }
    if (o.batched_eager == 1) {
        // eager mode (no graph): every stage launched on the caller's stream
        enqueue(pl, stream, sm_count, infos);
        count_launches(pl->kernels_per_run);
        RSVDGB_CUDA_TRY(cudaGetLastError());
        return RSVDGB_OK;
    }
    if (!pl->graph || pl->graph_infos != infos) {
        if (pl->graph) {
            cudaGraphExecDestroy(pl->graph);
            pl->graph = nullptr;
        }
        cudaStream_t cs;
        RSVDGB_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g;
        RSVDGB_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        enqueue(pl, cs, sm_count, infos);
        RSVDGB_CUDA_TRY(cudaStreamEndCapture(cs, &g));
        const cudaError_t e = cudaGraphInstantiate(&pl->graph, g, 0);
        cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        RSVDGB_CUDA_TRY(e);
        pl->graph_infos = infos;
    }
    RSVDGB_CUDA_TRY(cudaGraphLaunch(pl->graph, stream));
    count_launches(pl->kernels_per_run);
    return RSVDGB_OK;
}

}  // namespace rsvdgb
