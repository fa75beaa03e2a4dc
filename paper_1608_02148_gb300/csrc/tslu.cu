// Pivoted LU of a tall sketch for the normalized power iterations
// (Algorithm norm_iterations, Sec. 2.2.2): [L, ~] = lu(Y), L = P^T L0 with L0
// unit lower trapezoidal.  L spans Y, so only its role as a well-scaled basis
// matters (|L| stays small with pivoting); it is formed as L = Y U^{-1} from
// the U of l pivot rows.
//
// Partial pivoting over all m rows needs l sequential searches down the whole
// column; on the GPU the l pivot rows are chosen by tournament pivoting
// instead (the communication-avoiding "tall-skinny LU"): every CTA factors a
// block of rows by Gaussian elimination with partial pivoting in shared
// memory and proposes the l rows it pivoted on; groups of up to kGroup
// proposals are factored again, level by level, until one set remains.  The
// LU of that set's rows gives U (and the growth stays bounded as with partial
// pivoting in practice).  The pivots differ from partial pivoting over all
// rows, so L does too, but span(L) = span(Y) either way.
//
// One CTA per block; rows are staged row-major in shared memory (stride l + 1
// against bank conflicts); each elimination step: a block-wide argmax of the
// pivot column, the row swap, the column scaling and the rank-one update of
// the trailing block.
#include <algorithm>

#include "internal.cuh"

namespace rsvdgb {
namespace {

constexpr int kLuThreads = 256;
constexpr int kLuWarps = kLuThreads / 32;
constexpr int kBlock0 = 128;  // rows per block at the first level (>= l)
constexpr int kGroup = 4;     // proposals combined per CTA at later levels

// X column-major rows x l (ld).  Level 0 (cand_in null): CTA b takes rows
// [b * kBlock0, ...).  Later levels: CTA b takes the valid (>= 0) row ids of
// proposals [b * kGroup, b * kGroup + kGroup) of cand_in (l ids each, nsets of
// them).  Writes its l proposals to cand_out + b * l (-1 where it had fewer
// than l rows); when U is non-null (the last level, one CTA) also U = the
// upper triangle (l x l, row-major) and *status = RSVDGB_ERR_BREAKDOWN on a
// zero pivot.
__global__ void __launch_bounds__(kLuThreads) tslu_kernel(const float* __restrict__ X, int64_t ld, int64_t rows, int l,
                                                          const int* __restrict__ cand_in, int nsets,
                                                          int* __restrict__ cand_out, float* __restrict__ U,
                                                          int* status)
{
    extern __shared__ float S[];  // R rows of l + 1 floats, then R row ids
    const int LS = l + 1;
    const int R_max = (cand_in ? kGroup * l : kBlock0);
    int* rid = (int*)(S + (size_t)R_max * LS);
    __shared__ int nrows;
    __shared__ float wv[kLuWarps];
    __shared__ int wi[kLuWarps];
    __shared__ int piv_row;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b = blockIdx.x;

    // the rows of this CTA
    if (tid == 0) {
        int R = 0;
        if (!cand_in) {
            const int64_t r0 = (int64_t)b * kBlock0;
            R = (int)((rows - r0 < (int64_t)kBlock0) ? rows - r0 : (int64_t)kBlock0);
            for (int r = 0; r < R; ++r) rid[r] = (int)(r0 + r);
        } else {
            for (int g = 0; g < kGroup; ++g) {
                const int set = b * kGroup + g;
                if (set >= nsets) break;
                for (int t = 0; t < l; ++t) {
                    const int id = cand_in[(int64_t)set * l + t];
                    if (id >= 0) rid[R++] = id;
                }
            }
        }
        nrows = R;
    }
    __syncthreads();
    const int R = nrows;
    for (int e = tid; e < R * l; e += kLuThreads) {
        const int r = e % R, c = e / R;  // consecutive threads: consecutive rows of one column
        S[r * LS + c] = X[(int64_t)c * ld + rid[r]];
    }
    __syncthreads();

    const int steps = min(l, R);
    for (int j = 0; j < steps; ++j) {
        // pivot: the largest magnitude in column j at or below row j (ties to
        // the lower position)
        float bv = -1.f;
        int bi = R;
        for (int r = j + tid; r < R; r += kLuThreads) {
            const float v = fabsf(S[r * LS + j]);
            if (v > bv) {
                bv = v;
                bi = r;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) {
                bv = ov;
                bi = oi;
            }
        }
        if (lane == 0) {
            wv[warp] = bv;
            wi[warp] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            float v = wv[0];
            int i = wi[0];
            for (int w = 1; w < kLuWarps; ++w)
                if (wv[w] > v || (wv[w] == v && wi[w] < i)) {
                    v = wv[w];
                    i = wi[w];
                }
            piv_row = (i < R) ? i : j;
        }
        __syncthreads();
        const int p = piv_row;
        if (p != j) {
            for (int c = tid; c < l; c += kLuThreads) {
                const float t = S[j * LS + c];
                S[j * LS + c] = S[p * LS + c];
                S[p * LS + c] = t;
            }
            if (tid == 0) {
                const int t = rid[j];
                rid[j] = rid[p];
                rid[p] = t;
            }
        }
        __syncthreads();
        const float piv = S[j * LS + j];
        if (piv == 0.f) {
            if (U && tid == 0) atomicExch(status, RSVDGB_ERR_BREAKDOWN);
            continue;  // the column is zero at and below j: nothing to eliminate
        }
        const float inv = 1.f / piv;
        for (int r = j + 1 + tid; r < R; r += kLuThreads) S[r * LS + j] *= inv;
        __syncthreads();
        // rank-one update of the trailing block: a warp per row, lanes along it
        for (int r = j + 1 + warp; r < R; r += kLuWarps) {
            const float f = S[r * LS + j];
            for (int c = j + 1 + lane; c < l; c += 32) S[r * LS + c] = fmaf(-f, S[j * LS + c], S[r * LS + c]);
        }
        __syncthreads();
    }
    for (int t = tid; t < l; t += kLuThreads) cand_out[(int64_t)b * l + t] = (t < R) ? rid[t] : -1;
    if (U)
        for (int e = tid; e < l * l; e += kLuThreads) {
            const int r = e / l, c = e % l;
            U[e] = (c >= r && r < R) ? S[r * LS + c] : 0.f;
        }
}

// T = U^{-1} for an l x l row-major upper triangular U (back substitution,
// one thread per column of T); a zero diagonal entry gives T's column the
// unit vector (the sketch is rank-deficient there; the status is already set).
__global__ void tri_inv_kernel(const float* __restrict__ U, int l, float* __restrict__ T)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= l) return;
    for (int i = 0; i < l; ++i) T[i * l + j] = 0.f;
    if (U[j * l + j] == 0.f) {
        T[j * l + j] = 1.f;
        return;
    }
    T[j * l + j] = 1.f / U[j * l + j];
    for (int i = j - 1; i >= 0; --i) {
        float s = 0.f;
        for (int c = i + 1; c <= j; ++c) s = fmaf(U[i * l + c], T[c * l + j], s);
        const float d = U[i * l + i];
        T[i * l + j] = (d != 0.f) ? -s / d : 0.f;
    }
}

}  // namespace

bool tslu_supported(int l) { return l >= 1 && l <= 112; }

int64_t tslu_scratch_ints(int64_t rows, int l) { return 2 * ceil_div(rows, kBlock0) * (int64_t)l; }

int launch_tslu(cudaStream_t s, const float* X, int64_t ld, int64_t rows, int l, int* scratch, float* U, float* T,
                int* status)
{
    if (!tslu_supported(l) || rows < l) return RSVDGB_ERR_UNSUPPORTED;
    const size_t smem0 = (size_t)kBlock0 * (l + 1) * sizeof(float) + kBlock0 * sizeof(int);
    const size_t smemg = (size_t)kGroup * l * (l + 1) * sizeof(float) + (size_t)kGroup * l * sizeof(int);
    if (cudaFuncSetAttribute(tslu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)std::max(smem0, smemg)) != cudaSuccess)
        return RSVDGB_ERR_CUDA;
    int64_t nsets = ceil_div(rows, kBlock0);
    int* a = scratch;
    int* b = scratch + nsets * l;
    tslu_kernel<<<(unsigned)nsets, kLuThreads, smem0, s>>>(X, ld, rows, l, nullptr, 0, a, nsets == 1 ? U : nullptr,
                                                           status);
    count_launches();
    while (nsets > 1) {
        const int64_t nn = ceil_div(nsets, kGroup);
        tslu_kernel<<<(unsigned)nn, kLuThreads, smemg, s>>>(X, ld, rows, l, a, (int)nsets, b,
                                                            nn == 1 ? U : nullptr, status);
        count_launches();
        std::swap(a, b);
        nsets = nn;
    }
    tri_inv_kernel<<<(unsigned)ceil_div(l, 128), 128, 0, s>>>(U, l, T);
    count_launches();
    return cudaGetLastError() == cudaSuccess ? RSVDGB_OK : RSVDGB_ERR_CUDA;
}

}  // namespace rsvdgb
