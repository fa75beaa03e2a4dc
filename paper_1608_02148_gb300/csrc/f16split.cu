// Operands of the scaled FP16x3 passes over A (see tc_pass.cu):
//   * the split of a column-major panel into FP16 hi and lo parts, column j
//     multiplied first by the power of two 2^ej that brings its largest
//     magnitude into [2^13, 2^14), with 2^-ej kept for the pass's epilogue;
//   * max|A| of a stored matrix, for the products that are not preceded by
//     a first pass measuring it (the C-ABI pass entry points).
#include <algorithm>

#include "internal.cuh"
#include "ptx.cuh"

namespace rsvdgb {
namespace {
using namespace dev;

constexpr int kSplitThreads = 256;

__device__ __forceinline__ float block_max(float v, float* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) red[0] = v;
    }
    __syncthreads();
    const float r = red[0];
    __syncthreads();
    return r;
}

// One CTA per column j < l_pad.  Rows rows..ld-1 and columns l..l_pad-1 are
// written as zero (the tensor maps read them).
__global__ void __launch_bounds__(kSplitThreads) panel_f16_kernel(const float* __restrict__ in, int64_t ld,
                                                                  int64_t rows, int l, uint16_t* __restrict__ hi,
                                                                  uint16_t* __restrict__ lo, float* __restrict__ pinv)
{
    __shared__ float red[32];
    const int j = blockIdx.x;
    const float* col = in + (int64_t)j * ld;
    float mx = 0.f;
    if (j < l)
        for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) mx = fmaxf(mx, fabsf(col[i]));
    mx = block_max(mx, red);
    const float sc = pow2_scale_below(mx);
    uint16_t* h = hi + (int64_t)j * ld;
    uint16_t* w = lo + (int64_t)j * ld;
    // pairs of rows (ld is even): 32-bit stores
    for (int64_t i = 2 * threadIdx.x; i < ld; i += 2 * blockDim.x) {
        const float x0 = (j < l && i < rows) ? col[i] * sc : 0.f;
        const float x1 = (j < l && i + 1 < rows) ? col[i + 1] * sc : 0.f;
        uint32_t ph, pl;
        split_f16_pair(x0, x1, ph, pl);
        *(uint32_t*)(h + i) = ph;
        *(uint32_t*)(w + i) = pl;
    }
    if (threadIdx.x == 0) pinv[j] = 1.f / sc;
}

// max|a| over a row-major rows x cols matrix (FP32 or BF16 bits), as float
// bits accumulated with atomicMax into *amax (zeroed beforehand).
__global__ void __launch_bounds__(kSplitThreads) absmax_kernel(const void* __restrict__ A, int64_t lda, int a_bf16,
                                                               int64_t rows, int64_t cols, unsigned int* amax)
{
    __shared__ float red[32];
    float mx = 0.f;
    const int64_t total = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / cols, c = e % cols;
        const float v = a_bf16 ? __uint_as_float((uint32_t)((const uint16_t*)A)[i * lda + c] << 16)
                               : ((const float*)A)[i * lda + c];
        mx = fmaxf(mx, fabsf(v));
    }
    mx = block_max(mx, red);
    if (threadIdx.x == 0) atomicMax(amax, __float_as_uint(mx));
}

}  // namespace

void launch_panel_f16(cudaStream_t s, const float* in, int64_t ld, int64_t rows, int l, int l_pad, uint16_t* hi,
                      uint16_t* lo, float* pinv)
{
    panel_f16_kernel<<<l_pad, kSplitThreads, 0, s>>>(in, ld, rows, l, hi, lo, pinv);
    count_launches();
}

void launch_absmax(cudaStream_t s, int sm_count, const void* A, int64_t lda, int a_bf16, int64_t rows, int64_t cols,
                   unsigned int* amax)
{
    const int64_t want = ceil_div(rows * cols, kSplitThreads * 8);
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, 4 * (int64_t)sm_count));
    absmax_kernel<<<blocks, kSplitThreads, 0, s>>>(A, lda, a_bf16, rows, cols, amax);
    count_launches();
}

}  // namespace rsvdgb
