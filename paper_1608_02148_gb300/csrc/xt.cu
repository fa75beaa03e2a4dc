// Z = X T for a tall column-major X (rows x l, leading dimension ld) and a
// small l x l row-major T that is upper triangular (a Cholesky factor's
// inverse): the basis change of CholeskyQR, Q = Y R^{-1} (the "qr" of
// Algorithm sub_iterations and of Algorithm rqb step 9), in FP32 FMA.
//
// The product reads X once and writes Z once (plus, optionally, Z's split
// for the pass that reads it next: TF32 hi / lo floats, or the FP16 hi / lo
// of a fixed power-of-two multiple of Z).  Its arithmetic, rows * l^2 / 2
// FMA, is a few microseconds of the SM's packed FP32x2 FMA rate, so it is
// bound by the 3 (or 5) m x l streams.  One CTA per SM keeps T in shared
// memory and walks 128-row tiles of X, double-buffered: the next tile is in
// flight (16-byte asynchronous copies, zero-filled past `rows`) while the
// current one is multiplied.  The columns form blocks of 8; warp w owns
// blocks w and nb - 1 - w, so that with the sum over k stopping at T's
// diagonal every warp runs the same number of steps.  A thread accumulates
// 4 rows x 8 columns of a block at a time, over k in increasing order.
// Rows beyond `rows` (up to ld) and columns l..l_pad-1 of the outputs are
// written as zero.
#include <algorithm>

#include "internal.cuh"
#include "ptx.cuh"

namespace rsvdgb {
namespace {
using namespace dev;

constexpr int kXtRows = 128;  // rows per tile
constexpr int kXtBlk = 8;     // columns per block
constexpr int kXtMaxL = 112;  // widest l_pad: 14 blocks, 7 warps
constexpr int kXtMaxThreads = 32 * kXtMaxL / (2 * kXtBlk);

__device__ __forceinline__ void cp_async16_zfill(float* dst, const float* src, int bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(bytes)
                 : "memory");
}

template <int SPLIT>  // 0 none, 1 TF32 hi / lo floats, 2 FP16 hi / lo (uint16) of sc * Z
__global__ void __launch_bounds__(kXtMaxThreads, 1)
    xt_kernel(const float* __restrict__ X, int64_t ld, int64_t rows, int l, int l_pad, const float* __restrict__ T,
              float* __restrict__ Z, void* __restrict__ Zh, void* __restrict__ Zl, float sc)
{
    extern __shared__ __align__(16) float sm[];
    float* Ts = sm;                          // l x kXtMaxL (row k, column j), zero padded
    float* Xb0 = sm + (size_t)l * kXtMaxL;   // two tiles: column k at k * kXtRows
    float* Xb1 = Xb0 + (size_t)l * kXtRows;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthreads = blockDim.x;
    const int nb = l_pad / kXtBlk;
    // T into shared memory, eight loads in flight per thread before the stores
    for (int e0 = tid; e0 < l * kXtMaxL; e0 += 8 * nthreads) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * nthreads;
            const int k = e / kXtMaxL, j = e - k * kXtMaxL;
            v[u] = (e < l * kXtMaxL && j < l) ? T[k * l + j] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int e = e0 + u * nthreads;
            if (e < l * kXtMaxL) Ts[e] = v[u];
        }
    }
    const int64_t ntiles = (ld + kXtRows - 1) / kXtRows;
    // one commit group per tile: 16-byte chunks of each column, zero-filled
    // past `rows` (a chunk wholly past it reads nothing)
    auto issue = [&](int64_t tile, float* buf) {
        const int64_t r0 = tile * kXtRows;
        constexpr int q4 = kXtRows / 4;
        for (int q = tid; q < l * q4; q += nthreads) {
            const int k = q / q4, c = q - k * q4;
            const int64_t i = r0 + 4 * c;
            const int64_t left = rows - i;
            const int bytes = left >= 4 ? 16 : (left > 0 ? (int)left * 4 : 0);
            cp_async16_zfill(buf + k * kXtRows + 4 * c, bytes ? X + (int64_t)k * ld + i : X, bytes);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    int64_t tile = blockIdx.x;
    if (tile < ntiles) issue(tile, Xb0);
    for (int it = 0; tile < ntiles; ++it, tile += gridDim.x) {
        const float* cur = (it & 1) ? Xb1 : Xb0;
        float* nxt = (it & 1) ? Xb0 : Xb1;
        __syncthreads();  // the previous tile's reads of nxt are done (and Ts is written)
        if (tile + gridDim.x < ntiles)
            issue(tile + gridDim.x, nxt);
        else
            asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();  // every thread's copies of the current tile have landed
        const int64_t r0 = tile * kXtRows;
#pragma unroll 1
        for (int half = 0; half < 2; ++half) {
            const int b = half ? nb - 1 - warp : warp;
            const int c0 = b * kXtBlk;
            // T is upper triangular: column j collects k <= j only
            const int kend = min(l, c0 + kXtBlk);
            float2 acc[4][kXtBlk / 2];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < kXtBlk / 2; ++c) acc[a][c] = make_float2(0.f, 0.f);
            for (int k = 0; k < kend; ++k) {
                const float4 ta = *(const float4*)(Ts + k * kXtMaxL + c0);
                const float4 tb = *(const float4*)(Ts + k * kXtMaxL + c0 + 4);
                const float2 t2[4] = {make_float2(ta.x, ta.y), make_float2(ta.z, ta.w), make_float2(tb.x, tb.y),
                                      make_float2(tb.z, tb.w)};
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const float x = cur[k * kXtRows + lane + 32 * a];
                    const float2 x2 = make_float2(x, x);
#pragma unroll
                    for (int c = 0; c < kXtBlk / 2; ++c) acc[a][c] = __ffma2_rn(x2, t2[c], acc[a][c]);
                }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int64_t i = r0 + lane + 32 * a;
                if (i >= ld) continue;
#pragma unroll
                for (int c = 0; c < kXtBlk; ++c) {
                    const int j = c0 + c;
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
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

template <int SPLIT>
int launch_xt_typed(cudaStream_t s, int sm_count, const float* X, int64_t ld, int64_t rows, int l, int l_pad,
                    const float* T, float* Z, void* Zh, void* Zl, float sc)
{
    const size_t smem = sizeof(float) * (size_t)l * (kXtMaxL + 2 * kXtRows);
    if (cudaFuncSetAttribute(xt_kernel<SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return RSVDGB_ERR_CUDA;
    const int64_t ntiles = ceil_div(ld, kXtRows);
    const int grid = (int)std::min<int64_t>(ntiles, (int64_t)sm_count);
    const int threads = 32 * (l_pad / (2 * kXtBlk));
    xt_kernel<SPLIT><<<grid, threads, smem, s>>>(X, ld, rows, l, l_pad, T, Z, Zh, Zl, sc);
    count_launches();
    return cudaGetLastError() == cudaSuccess ? RSVDGB_OK : RSVDGB_ERR_CUDA;
}

}  // namespace

bool xt_supported(int l_pad) { return l_pad >= 16 && l_pad <= kXtMaxL && l_pad % 16 == 0; }

int launch_xt(cudaStream_t s, int sm_count, const float* X, int64_t ld, int64_t rows, int l, int l_pad, const float* T,
              float* Z, int split, void* Zh, void* Zl, float sc)
{
    if (!xt_supported(l_pad) || l > l_pad || ld % 4 != 0 || ((uintptr_t)X & 15) != 0) return RSVDGB_ERR_UNSUPPORTED;
    switch (split) {
        case 0: return launch_xt_typed<0>(s, sm_count, X, ld, rows, l, l_pad, T, Z, nullptr, nullptr, sc);
        case 1: return launch_xt_typed<1>(s, sm_count, X, ld, rows, l, l_pad, T, Z, Zh, Zl, sc);
        case 2: return launch_xt_typed<2>(s, sm_count, X, ld, rows, l, l_pad, T, Z, Zh, Zl, sc);
        default: return RSVDGB_ERR_INVALID_ARG;
    }
}

}  // namespace rsvdgb
