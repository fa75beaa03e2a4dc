// Z = X T for a tall column-major X (rows x l, leading dimension ld) and a
// small l x l row-major T that is upper triangular (a Cholesky factor's
// inverse): the basis change of CholeskyQR, Q = Y R^{-1} (the "qr" of
// Algorithm sub_iterations and of Algorithm rqb step 9), in FP32 FMA.
//
// The product reads X once and writes Z once (plus, optionally, Z's split
// for the pass that reads it next: TF32 hi / lo floats, or the FP16 hi / lo
// of a fixed power-of-two multiple of Z).  Its arithmetic, rows * l^2 / 2
// FMA, is a few microseconds of the SM's packed FP32x2 FMA rate, so it is
// bound by the 3 (or 5) m x l streams.  One CTA keeps T in shared memory and
// walks 128-row tiles of X: the tile is staged column by column (coalesced)
// in shared memory, each thread accumulates 4 rows x 14 columns (warp w owns
// columns [14 w, 14 w + 14)), and the sum over k stops at the diagonal of T.
// Rows beyond `rows` (up to ld) and columns l..l_pad-1 of the outputs are
// written as zero.
#include <algorithm>

#include "internal.cuh"
#include "ptx.cuh"

namespace rsvdgb {
namespace {
using namespace dev;

constexpr int kXtRows = 128;     // rows per tile
constexpr int kXtThreads = 256;  // 8 warps
constexpr int kXtCols = 14;      // columns per warp (8 x 14 = 112 >= l_pad)
constexpr int kXtMaxL = 8 * kXtCols;

template <int SPLIT>  // 0 none, 1 TF32 hi / lo floats, 2 FP16 hi / lo (uint16) of sc * Z
__global__ void __launch_bounds__(kXtThreads) xt_kernel(const float* __restrict__ X, int64_t ld, int64_t rows, int l,
                                                        int l_pad, const float* __restrict__ T, float* __restrict__ Z,
                                                        void* __restrict__ Zh, void* __restrict__ Zl, float sc)
{
    extern __shared__ __align__(16) float sm[];
    float* Ts = sm;                               // l x kXtMaxL (row k, column j), zero padded
    float* Xs = sm + (size_t)l * kXtMaxL;         // l x kXtRows: column k of the tile at k * kXtRows
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < l * kXtMaxL; e += kXtThreads) {
        const int k = e / kXtMaxL, j = e % kXtMaxL;
        Ts[e] = (j < l) ? T[k * l + j] : 0.f;
    }
    const int c0 = warp * kXtCols;
    // T is upper triangular: column j collects k <= j only
    const int kend = min(l, c0 + kXtCols);
    const int64_t ntiles = (ld + kXtRows - 1) / kXtRows;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r0 = tile * kXtRows;
        __syncthreads();  // previous tile's Xs reads done (and Ts written, first time)
        for (int e = tid; e < l * kXtRows; e += kXtThreads) {
            const int k = e / kXtRows, r = e % kXtRows;
            const int64_t i = r0 + r;
            Xs[e] = (i < rows) ? X[(int64_t)k * ld + i] : 0.f;
        }
        __syncthreads();
        float2 acc[4][kXtCols / 2];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < kXtCols / 2; ++c) acc[a][c] = make_float2(0.f, 0.f);
        for (int k = 0; k < kend; ++k) {
            const float* tk = Ts + k * kXtMaxL + c0;
            float2 t2[kXtCols / 2];
#pragma unroll
            for (int c = 0; c < kXtCols / 2; ++c) t2[c] = *(const float2*)(tk + 2 * c);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float x = Xs[k * kXtRows + lane + 32 * a];
                const float2 x2 = make_float2(x, x);
#pragma unroll
                for (int c = 0; c < kXtCols / 2; ++c) acc[a][c] = __ffma2_rn(x2, t2[c], acc[a][c]);
            }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int64_t i = r0 + lane + 32 * a;
            if (i >= ld) continue;
#pragma unroll
            for (int c = 0; c < kXtCols; ++c) {
                const int j = c0 + c;
                if (j >= l_pad) continue;
                const float v = (i < rows && j < l) ? ((c & 1) ? acc[a][c / 2].y : acc[a][c / 2].x) : 0.f;
                const int64_t o = (int64_t)j * ld + i;
                Z[o] = v;
                if (SPLIT == 1) {
                    const uint32_t h = tf32_rna(v);
                    ((float*)Zh)[o] = __uint_as_float(h);
                    ((float*)Zl)[o] = __uint_as_float(tf32_rna(v - __uint_as_float(h)));
                } else if (SPLIT == 2) {
                    uint32_t h, w;
                    split_f16_pair(v * sc, 0.f, h, w);
                    ((uint16_t*)Zh)[o] = (uint16_t)(h & 0xFFFFu);
                    ((uint16_t*)Zl)[o] = (uint16_t)(w & 0xFFFFu);
                }
            }
        }
    }
}

template <int SPLIT>
int launch_xt_typed(cudaStream_t s, int sm_count, const float* X, int64_t ld, int64_t rows, int l, int l_pad,
                    const float* T, float* Z, void* Zh, void* Zl, float sc)
{
    const size_t smem = sizeof(float) * (size_t)l * (kXtMaxL + kXtRows);
    if (cudaFuncSetAttribute(xt_kernel<SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return RSVDGB_ERR_CUDA;
    const int64_t ntiles = ceil_div(ld, kXtRows);
    const int per_sm = smem <= 110 * 1024 ? 2 : 1;
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)per_sm * sm_count);
    xt_kernel<SPLIT><<<grid, kXtThreads, smem, s>>>(X, ld, rows, l, l_pad, T, Z, Zh, Zl, sc);
    count_launches();
    return cudaGetLastError() == cudaSuccess ? RSVDGB_OK : RSVDGB_ERR_CUDA;
}

}  // namespace

bool xt_supported(int l_pad) { return l_pad <= kXtMaxL; }

int launch_xt(cudaStream_t s, int sm_count, const float* X, int64_t ld, int64_t rows, int l, int l_pad, const float* T,
              float* Z, int split, void* Zh, void* Zl, float sc)
{
    if (l_pad > kXtMaxL || l > l_pad) return RSVDGB_ERR_UNSUPPORTED;
    switch (split) {
        case 0: return launch_xt_typed<0>(s, sm_count, X, ld, rows, l, l_pad, T, Z, nullptr, nullptr, sc);
        case 1: return launch_xt_typed<1>(s, sm_count, X, ld, rows, l, l_pad, T, Z, Zh, Zl, sc);
        case 2: return launch_xt_typed<2>(s, sm_count, X, ld, rows, l, l_pad, T, Z, Zh, Zl, sc);
        default: return RSVDGB_ERR_INVALID_ARG;
    }
}

}  // namespace rsvdgb
