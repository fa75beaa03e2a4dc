// Interpolative and CUR decompositions (Algorithms id, rid and rcur, Sec. 7).
//
// rid: [~, B] = rqb(A, k, p, q); the column ID of the l x n factor B by QR
// with column pivoting stopped after k steps; T = S11^{-1} S12; Z(:, P) =
// [I, T]; C = A(:, J).  rcur adds the row pivots of C^T (the same pivoted QR
// on the k x m matrix C^T), R = A(I, :) and U = Z pinv(R).
//
// The pivoted QR runs as one cooperative kernel over all SMs: each CTA owns a
// contiguous range of columns, keeps their residual norms (FP64, downdated
// by the square of each new row of R), and every step ends at a grid
// barrier after which all CTAs take the same argmax of the per-CTA maxima.
// The new direction q_t is the pivot column made orthogonal to q_0..q_{t-1}
// by classical Gram-Schmidt applied twice; every CTA computes it from the
// same data in the same order, so all hold the same q_t, each in its own
// shared-memory copy of Q (r x k).
// Row t of R is q_t^T x_j for all columns, which equals the Householder R of
// the same pivots up to the sign of each row.  Every wait is bounded.
#include "internal.cuh"

#include <cuda_bf16.h>

#include "ptx.cuh"

namespace rsvdgb {
namespace {

constexpr int kPqrThreads = 256;
constexpr int kPqrWarps = kPqrThreads / 32;

struct PqrArgs {
    const float* X;  // r x N: column j at X + j * ldx (r contiguous floats)
    int64_t ldx;
    int r;
    int64_t N;
    int k;
    int* piv;          // k pivots (CTA 0 writes; -1 after a breakdown)
    float* R;          // k x N row-major (ld N), or null
    double* nrm;       // N residual norms^2; -inf marks a chosen column
    double* slot_val;  // per-CTA maxima, two buffers of gridDim.x (by barrier parity)
    int64_t* slot_idx;
    unsigned int* bar;  // grid barrier counter (zero at launch)
    int* status;
    long long spin_limit;  // bound of each barrier wait in clock64 ticks
    int absent_cta;        // test hook: this CTA skips its arrival at the first barrier (-1: none)
};

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// (v, i) beats (bv, bi): larger value, ties to the lower index; i < 0 never wins
__device__ __forceinline__ bool better(double v, int64_t i, double bv, int64_t bi)
{
    if (i < 0) return false;
    if (bi < 0) return true;
    return v > bv || (v == bv && i < bi);
}

// Grid-wide barrier on a monotone counter; bounded (spin_limit ticks, about
// 2 s by default), on expiry RSVDGB_ERR_TIMEOUT is recorded and false
// returned.  arrive = false (a test hook) waits without arriving.
__device__ bool grid_barrier(unsigned int* bar, unsigned int target, int* status, volatile int* flag,
                             long long spin_limit, bool arrive = true)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (arrive) atomicAdd(bar, 1u);
        const long long t0 = clock64();
        bool ok = true;
        while (*(volatile unsigned int*)bar < target) {
            if (clock64() - t0 > spin_limit) {
                ok = false;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        if (!ok) atomicExch(status, RSVDGB_ERR_TIMEOUT);
        *flag = ok ? 1 : 0;
    }
    __syncthreads();
    return *flag != 0;
}

// One stage of a butterfly reduce-scatter over the warp: lanes with bit O
// set keep the upper half of their 2 O partial sums, the others the lower
// half, each adding the partner's copy of the half it keeps.
template <int O>
__device__ __forceinline__ void reduce_scatter_stage(float (&v)[32], int lane)
{
    const bool up = (lane & O) != 0;
#pragma unroll
    for (int k = 0; k < O; ++k) {
        const float send = up ? v[k] : v[k + O];
        const float keep = up ? v[k + O] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, O);
    }
}

// For the 32 columns j0 .. j0 + 31 of X (those below c1): w^T x_j with w
// (r floats, shared memory), or ||x_j||^2 when SQ.  Each lane sums its rows
// i = lane (mod 32) of all 32 columns (one coalesced 128-byte load per
// column and row block); five reduce-scatter stages (31 shuffles) then
// leave column j0 + L's total in lane L.  Called by whole warps.
template <bool SQ>
__device__ __forceinline__ float dots32(const PqrArgs& a, const float* w, int64_t j0, int64_t c1, int lane)
{
    float v[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = 0.f;
    const float* x0 = a.X + j0 * a.ldx;
    for (int i = lane; i < a.r; i += 32) {
        const float wi = SQ ? 0.f : w[i];
#pragma unroll
        for (int c = 0; c < 32; ++c)
            if (j0 + c < c1) {
                const float x = x0[(int64_t)c * a.ldx + i];
                v[c] = fmaf(SQ ? x : wi, x, v[c]);
            }
    }
    reduce_scatter_stage<16>(v, lane);
    reduce_scatter_stage<8>(v, lane);
    reduce_scatter_stage<4>(v, lane);
    reduce_scatter_stage<2>(v, lane);
    reduce_scatter_stage<1>(v, lane);
    return v[0];
}

// Block-wide argmax of per-warp candidates; thread 0 writes the CTA slot of
// buffer buf.  The maxima gathered after barrier e sit in buffer e & 1: a CTA
// that runs ahead cannot overwrite them before every CTA has read them, since
// it writes that buffer again only after the next barrier.
__device__ void block_argmax_to_slot(double v, int64_t i, double* wv, int64_t* wi, const PqrArgs& a, int buf)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int64_t oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (better(ov, oi, v, i)) {
            v = ov;
            i = oi;
        }
    }
    if (lane == 0) {
        wv[warp] = v;
        wi[warp] = i;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bv = -1.0;
        int64_t bi = -1;
        for (int w = 0; w < kPqrWarps; ++w)
            if (better(wv[w], wi[w], bv, bi)) {
                bv = wv[w];
                bi = wi[w];
            }
        a.slot_val[(int64_t)buf * gridDim.x + blockIdx.x] = bv;
        a.slot_idx[(int64_t)buf * gridDim.x + blockIdx.x] = bi;
    }
}

__global__ void __launch_bounds__(kPqrThreads, 1) pqr_kernel(PqrArgs a)
{
    extern __shared__ float sm[];  // Q (r x k, column t = q_t), then r floats for the new column
    float* Qs = sm;
    float* qs = sm + (size_t)a.r * a.k;
    __shared__ float coef[256];
    __shared__ double wv[kPqrWarps];
    __shared__ int64_t wi[kPqrWarps];
    __shared__ double red[kPqrWarps];
    __shared__ int64_t piv_sh;
    __shared__ double norm_sh;
    __shared__ volatile int flag;
    const int G = gridDim.x, b = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = a.r;
    const int64_t c0 = a.N * b / G, c1 = a.N * (b + 1) / G;
    unsigned int epoch = 0;
    // CTA 0 writes the pivots (only it does, and only after this): -1 until
    // a step chooses one, so that a launch left early (a barrier wait that
    // ran out) hands the gathers and the ID solve only -1 entries
    if (b == 0)
        for (int u = threadIdx.x; u < a.k; u += kPqrThreads) a.piv[u] = -1;

    // residual norms of this CTA's columns (lane L of a warp owns column
    // j0 + L of each 32-column block), and their maximum
    double bv = -1.0;
    int64_t bi = -1;
    for (int64_t j0 = c0 + 32 * warp; j0 < c1; j0 += 32 * kPqrWarps) {
        const float s = dots32<true>(a, nullptr, j0, c1, lane);
        const int64_t j = j0 + lane;
        if (j < c1) {
            const double sd = (double)s;
            a.nrm[j] = sd;
            if (better(sd, j, bv, bi)) {
                bv = sd;
                bi = j;
            }
        }
    }
    block_argmax_to_slot(bv, bi, wv, wi, a, (int)((epoch + 1) & 1));
    if (!grid_barrier(a.bar, ++epoch * (unsigned)G, a.status, &flag, a.spin_limit, (int)blockIdx.x != a.absent_cta))
        return;

    for (int t = 0; t < a.k; ++t) {
        {
            // global argmax of the per-CTA maxima, block-parallel
            double gv = -1.0;
            int64_t gi = -1;
            const int64_t base = (int64_t)(epoch & 1) * G;
            for (int c = threadIdx.x; c < G; c += kPqrThreads) {
                const double v = __ldcg(a.slot_val + base + c);
                const int64_t i = __ldcg(a.slot_idx + base + c);
                if (better(v, i, gv, gi)) {
                    gv = v;
                    gi = i;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, gv, o);
                const int64_t oi = __shfl_xor_sync(0xffffffffu, gi, o);
                if (better(ov, oi, gv, gi)) {
                    gv = ov;
                    gi = oi;
                }
            }
            if (lane == 0) {
                wv[warp] = gv;
                wi[warp] = gi;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double fv = -1.0;
                int64_t fi = -1;
                for (int w = 0; w < kPqrWarps; ++w)
                    if (better(wv[w], wi[w], fv, fi)) {
                        fv = wv[w];
                        fi = wi[w];
                    }
                piv_sh = (fi >= 0 && fv > 0.0) ? fi : -1;
            }
            __syncthreads();
        }
        const int64_t p = piv_sh;
        if (p < 0) {
            // every remaining column is (numerically) in the span already
            if (b == 0 && threadIdx.x == 0) {
                for (int u = t; u < a.k; ++u) a.piv[u] = -1;
                atomicExch(a.status, RSVDGB_ERR_BREAKDOWN);
            }
            return;
        }
        if (b == 0 && threadIdx.x == 0) a.piv[t] = (int)p;
        for (int i = threadIdx.x; i < r; i += kPqrThreads) qs[i] = a.X[p * a.ldx + i];
        __syncthreads();
        // classical Gram-Schmidt against q_0 .. q_{t-1}, twice
        for (int pass = 0; pass < 2; ++pass) {
            for (int s = warp; s < t; s += kPqrWarps) {
                const float* qv = Qs + (int64_t)s * r;
                float d = 0.f;
                for (int i = lane; i < r; i += 32) d = fmaf(qv[i], qs[i], d);
                d = warp_sum_f(d);
                if (lane == 0) coef[s] = d;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < r; i += kPqrThreads) {
                float acc = qs[i];
                for (int s = 0; s < t; ++s) acc = fmaf(-coef[s], Qs[(int64_t)s * r + i], acc);
                qs[i] = acc;
            }
            __syncthreads();
        }
        {
            float s2 = 0.f;
            for (int i = threadIdx.x; i < r; i += kPqrThreads) s2 = fmaf(qs[i], qs[i], s2);
            const double w2 = warp_sum_d((double)s2);
            if (lane == 0) red[warp] = w2;
            __syncthreads();
            if (threadIdx.x == 0) {
                double tot = 0.0;
                for (int w = 0; w < kPqrWarps; ++w) tot += red[w];
                norm_sh = sqrt(tot);
            }
            __syncthreads();
        }
        const double nq = norm_sh;
        if (!(nq > 0.0)) {
            if (b == 0 && threadIdx.x == 0) {
                for (int u = t; u < a.k; ++u) a.piv[u] = -1;
                atomicExch(a.status, RSVDGB_ERR_BREAKDOWN);
            }
            return;
        }
        const float inv = (float)(1.0 / nq);
        for (int i = threadIdx.x; i < r; i += kPqrThreads) {
            qs[i] *= inv;
            Qs[(int64_t)t * r + i] = qs[i];
        }
        __syncthreads();
        // row t of R for this CTA's columns; downdate their residual norms,
        // each lane its own column (the FP64 work is not repeated across
        // the warp: GB300's FP64 pipe is a small fraction of its FP32 one)
        bv = -1.0;
        bi = -1;
        for (int64_t j0 = c0 + 32 * warp; j0 < c1; j0 += 32 * kPqrWarps) {
            const float du = dots32<false>(a, qs, j0, c1, lane);
            const int64_t j = j0 + lane;
            if (j >= c1) continue;
            const double cur = a.nrm[j];
            if (cur == -INFINITY) {  // a pivot of an earlier step
                if (a.R) a.R[(int64_t)t * a.N + j] = 0.f;
                continue;
            }
            double nn = fmax(cur - (double)du * (double)du, 0.0);
            if (j == p) nn = -INFINITY;
            if (a.R) a.R[(int64_t)t * a.N + j] = du;
            a.nrm[j] = nn;
            if (j != p && better(nn, j, bv, bi)) {
                bv = nn;
                bi = j;
            }
        }
        block_argmax_to_slot(bv, bi, wv, wi, a, (int)((epoch + 1) & 1));
        if (!grid_barrier(a.bar, ++epoch * (unsigned)G, a.status, &flag, a.spin_limit)) return;
    }
}

// Z (k x N, row-major ld ldz): Z(:, piv[t]) = e_t; other columns solve
// S11 z = R(:, j) with S11(a, b) = R(a, piv[b]) upper triangular, by back
// substitution: one warp per column, the lanes sharing each row's dot
// product; z in shared memory (k floats per warp).  A pivot list cut short
// by a breakdown (entries -1) leaves Z = 0.
constexpr int kSolveWarps = 4;
__global__ void __launch_bounds__(32 * kSolveWarps) id_solve_kernel(const float* __restrict__ R, int64_t N, int k,
                                                                     const int* __restrict__ piv,
                                                                     float* __restrict__ Z, int64_t ldz, int* status)
{
    extern __shared__ int pv[];  // k pivots, then kSolveWarps x k floats
    float* zs = reinterpret_cast<float*>(pv + k);
    for (int t = threadIdx.x; t < k; t += blockDim.x) pv[t] = piv[t];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t j = (int64_t)blockIdx.x * kSolveWarps + warp;
    if (j >= N) return;
    float* z = zs + warp * k;
    int pos = -1;
    bool short_piv = false;  // the pivoted QR stopped early (status already set)
    for (int t = lane; t < k; t += 32) {
        if (pv[t] == (int)j) pos = t;
        short_piv |= pv[t] < 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pos = max(pos, __shfl_xor_sync(0xffffffffu, pos, o));
    if (__any_sync(0xffffffffu, short_piv)) {
        for (int a = lane; a < k; a += 32) Z[(int64_t)a * ldz + j] = 0.f;
        return;
    }
    if (pos >= 0) {
        for (int a = lane; a < k; a += 32) Z[(int64_t)a * ldz + j] = (a == pos) ? 1.f : 0.f;
        return;
    }
    for (int a = k - 1; a >= 0; --a) {
        const float* Ra = R + (int64_t)a * N;
        float s = 0.f;
        for (int c = a + 1 + lane; c < k; c += 32) s = fmaf(__ldg(Ra + pv[c]), z[c], s);
        s = warp_sum_f(s);
        const float d = __ldg(Ra + pv[a]);
        const float za = (__ldg(Ra + j) - s) / d;
        if (lane == 0) {
            z[a] = za;
            Z[(int64_t)a * ldz + j] = za;
            if (!isfinite(za)) atomicExch(status, RSVDGB_ERR_BREAKDOWN);
        }
        __syncwarp();
    }
}

template <bool BF>
__device__ __forceinline__ float elem(const void* S, int64_t off)
{
    if constexpr (BF)
        return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(S)[off]);
    else
        return reinterpret_cast<const float*>(S)[off];
}

// C (rows x k, row-major ldc) = columns idx of the logical matrix
// (logical(i, j) = S[i * lda + j], or S[j * lda + i] when trans).
template <bool BF>
__global__ void gather_cols_kernel(const void* __restrict__ S, int64_t lda, bool trans, int64_t rows,
                                   const int* __restrict__ idx, int k, float* __restrict__ C, int64_t ldc)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * k) return;
    int64_t i, t;
    if (trans) {  // consecutive threads along the stored row of column idx[t]
        t = e / rows;
        i = e % rows;
    } else {
        i = e / k;
        t = e % k;
    }
    const int64_t j = idx[t];  // -1 after a pivoted-QR breakdown: zero column
    C[i * ldc + t] = j < 0 ? 0.f : elem<BF>(S, trans ? j * lda + i : i * lda + j);
}

// R (k x cols, row-major ldr) = rows idx of the logical matrix; Rt (if not
// null) receives the transpose column-major (Rt[t * ldt + j]).
template <bool BF>
__global__ void gather_rows_kernel(const void* __restrict__ S, int64_t lda, bool trans, int64_t cols,
                                   const int* __restrict__ idx, int k, float* __restrict__ R, int64_t ldr,
                                   float* __restrict__ Rt, int64_t ldt)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cols * k) return;
    const int64_t t = e / cols, j = e % cols;
    const int64_t i = idx[t];  // -1 after a pivoted-QR breakdown: zero row
    const float v = i < 0 ? 0.f : elem<BF>(S, trans ? j * lda + i : i * lda + j);
    if (R) R[t * ldr + j] = v;
    if (Rt) Rt[t * ldt + j] = v;
}

// Xc (column-major r x N, ld ldx) = transpose of the column-major N x r Bt (ld ldb).
__global__ void transpose_cm_kernel(const float* __restrict__ Bt, int64_t ldb, int64_t N, int r,
                                    float* __restrict__ X, int64_t ldx)
{
    __shared__ float tile[32][33];
    const int64_t j0 = (int64_t)blockIdx.x * 32;
    const int t0 = blockIdx.y * 32;
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int t = t0 + dy;
        const int64_t j = j0 + threadIdx.x;
        tile[dy][threadIdx.x] = (t < r && j < N) ? Bt[(int64_t)t * ldb + j] : 0.f;
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
        const int64_t j = j0 + dy;
        const int t = t0 + threadIdx.x;
        if (j < N && t < r) X[j * ldx + t] = tile[threadIdx.x][dy];
    }
}

// W (k x k row-major) = Z Q with Z (k x N row-major, ld ldz) and Q (N x k
// column-major, ld ldq): warp per output, FP32 runs then FP64.
__global__ void zq_kernel(const float* __restrict__ Z, int64_t ldz, const float* __restrict__ Q, int64_t ldq,
                          int64_t N, int k, float* __restrict__ W)
{
    const int lane = threadIdx.x & 31;
    const int o = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (o >= k * k) return;
    const int a = o / k, c = o % k;
    const float* z = Z + (int64_t)a * ldz;
    const float* q = Q + (int64_t)c * ldq;
    double acc = 0.0;
    for (int64_t j0 = 0; j0 < N; j0 += 32 * 8) {
        float run = 0.f;
        for (int u = 0; u < 8; ++u) {
            const int64_t j = j0 + u * 32 + lane;
            if (j < N) run = fmaf(z[j], q[j], run);
        }
        acc += run;
    }
    acc = warp_sum_d(acc);
    if (lane == 0) W[a * k + c] = (float)acc;
}

__global__ void piv_to_i64_kernel(const int* __restrict__ piv, int k, int64_t* __restrict__ out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < k) out[t] = piv[t];
}

}  // namespace

int pqr_max_ctas(int sm_count, size_t smem)
{
    int per_sm = 0;
    if (cudaFuncSetAttribute(pqr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pqr_kernel, kPqrThreads, smem) != cudaSuccess)
        return 0;
    return std::min(per_sm, 4) * sm_count;
}

int launch_pqr(cudaStream_t s, int sm_count, const float* X, int64_t ldx, int r, int64_t N, int k, int* piv,
               float* R, double* nrm, double* slot_val, int64_t* slot_idx, int max_slots, unsigned int* bar,
               int* status, long long spin_limit, int absent_cta)
{
    if (r < 1 || r > 256 || k < 1 || k > r || k > 256 || N < k) return RSVDGB_ERR_INVALID_ARG;
    const size_t smem = ((size_t)r * k + r) * sizeof(float);
    if (smem > 200 * 1024) return RSVDGB_ERR_UNSUPPORTED;
    const int cap = pqr_max_ctas(sm_count, smem);
    if (cap <= 0) return RSVDGB_ERR_CUDA;
    // one 32-column block per warp and step where the columns allow it:
    // fewer CTAs make the per-step barrier cheaper
    int G = (int)std::min<int64_t>(std::min<int64_t>(cap, max_slots / 2), ceil_div(N, 32 * kPqrWarps));
    G = std::max(G, 1);
    if (cudaMemsetAsync(bar, 0, sizeof(unsigned int), s) != cudaSuccess) return RSVDGB_ERR_CUDA;
    PqrArgs a{X, ldx, r, N, k, piv, R, nrm, slot_val, slot_idx, bar, status,
              spin_limit > 0 ? spin_limit : dev::kSpinLimit, absent_cta};
    void* params[] = {&a};
    if (cudaLaunchCooperativeKernel((const void*)pqr_kernel, dim3(G), dim3(kPqrThreads), params, smem, s) !=
        cudaSuccess)
        return RSVDGB_ERR_CUDA;
    count_launches();
    return RSVDGB_OK;
}

void launch_id_solve(cudaStream_t s, const float* R, int64_t N, int k, const int* piv, float* Z, int64_t ldz,
                     int* status)
{
    const size_t smem = (size_t)k * sizeof(int) + (size_t)kSolveWarps * k * sizeof(float);
    id_solve_kernel<<<(unsigned)ceil_div(N, kSolveWarps), 32 * kSolveWarps, smem, s>>>(R, N, k, piv, Z, ldz,
                                                                                        status);
    count_launches();
}

void launch_gather_cols(cudaStream_t s, const void* S, int64_t lda, int a_bf16, bool trans, int64_t rows,
                        const int* idx, int k, float* C, int64_t ldc)
{
    const unsigned nb = (unsigned)ceil_div(rows * k, 256);
    if (a_bf16)
        gather_cols_kernel<true><<<nb, 256, 0, s>>>(S, lda, trans, rows, idx, k, C, ldc);
    else
        gather_cols_kernel<false><<<nb, 256, 0, s>>>(S, lda, trans, rows, idx, k, C, ldc);
    count_launches();
}

void launch_gather_rows(cudaStream_t s, const void* S, int64_t lda, int a_bf16, bool trans, int64_t cols,
                        const int* idx, int k, float* R, int64_t ldr, float* Rt, int64_t ldt)
{
    const unsigned nb = (unsigned)ceil_div(cols * k, 256);
    if (a_bf16)
        gather_rows_kernel<true><<<nb, 256, 0, s>>>(S, lda, trans, cols, idx, k, R, ldr, Rt, ldt);
    else
        gather_rows_kernel<false><<<nb, 256, 0, s>>>(S, lda, trans, cols, idx, k, R, ldr, Rt, ldt);
    count_launches();
}

void launch_transpose_cm(cudaStream_t s, const float* Bt, int64_t ldb, int64_t N, int r, float* X, int64_t ldx)
{
    transpose_cm_kernel<<<dim3((unsigned)ceil_div(N, 32), (unsigned)ceil_div(r, 32)), dim3(32, 8), 0, s>>>(
        Bt, ldb, N, r, X, ldx);
    count_launches();
}

void launch_zq(cudaStream_t s, const float* Z, int64_t ldz, const float* Q, int64_t ldq, int64_t N, int k, float* W)
{
    zq_kernel<<<(unsigned)ceil_div((int64_t)k * k, 8), 256, 0, s>>>(Z, ldz, Q, ldq, N, k, W);
    count_launches();
}

void launch_piv_to_i64(cudaStream_t s, const int* piv, int k, int64_t* out)
{
    piv_to_i64_kernel<<<(unsigned)ceil_div(k, 128), 128, 0, s>>>(piv, k, out);
    count_launches();
}

}  // namespace rsvdgb
