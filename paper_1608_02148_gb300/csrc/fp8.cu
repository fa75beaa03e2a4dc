// FP8 (E4M3) operands for the power passes of the mixed-precision rSVD: the
// power iterations only carry the span of the sketch (Algorithm
// sub_iterations), so their products may be coarse while the projection
// B = Q^T A stays FP32-accurate.
//
// A is quantised once, row by row: row i is multiplied by 2^-e_i, the power
// of two that brings max_j |a_ij| to at most 448 (the largest finite E4M3
// value), and rounded to nearest E4M3 (saturating); e_i is kept.  The
// factors come out of the products exactly: (A P)_ij = 2^e_i (A8 P)_ij on
// the A side, and A^T Q = A8^T (S Q) with S = diag(2^e_i) on the A^T side,
// where S Q is quantised like a panel.  Panels (K x l, column-major) are
// quantised per column the same way.  A8 is stored twice, row-major and
// transposed (column-major), so that both products read K-major tiles.
#include <algorithm>

#include "internal.cuh"
#include "ptx.cuh"

namespace rsvdgb {
namespace {
using namespace dev;

constexpr float kE4M3Max = 448.f;

// Power of two p with max / p <= 448 (p = 1 for a zero or non-finite max).
__device__ __forceinline__ float e4m3_scale(float mx)
{
    if (!(mx > 0.f) || !(mx <= 3.4e38f)) return 1.f;
    int e;
    frexpf(mx / kE4M3Max, &e);  // mx / 448 < 2^e
    return ldexpf(1.f, max(-126, min(127, e)));
}

// Two floats to two E4M3 bytes (round to nearest, saturating): lo_elem in
// the low byte.
__device__ __forceinline__ uint16_t pack_e4m3(float lo_elem, float hi_elem)
{
    uint16_t r;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi_elem), "f"(lo_elem));
    return r;
}

template <bool BF>
__device__ __forceinline__ float load_a(const void* A, int64_t off)
{
    if (BF) return __uint_as_float((uint32_t)((const uint16_t*)A)[off] << 16);
    return ((const float*)A)[off];
}

// One warp per row: the row's max (first read), then the quantised row
// (second read, mostly from L2), its scale 2^e_i, its sum of squares and max
// (FP64 atomics / bit atomicMax for ||A||_F^2 and max|A|).
template <bool BF>
__global__ void __launch_bounds__(256) fp8_rows_kernel(const void* __restrict__ A, int64_t lda, int64_t m, int64_t n,
                                                       uint8_t* __restrict__ A8, int64_t ld8, float* __restrict__ rs,
                                                       double* fro2, unsigned int* amax)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= m) return;
    const int64_t base = i * lda;
    float mx = 0.f;
    double sq = 0.0;
    float sqf = 0.f;
    int cnt = 0;
    for (int64_t c = lane; c < n; c += 32) {
        const float v = load_a<BF>(A, base + c);
        mx = fmaxf(mx, fabsf(v));
        sqf = fmaf(v, v, sqf);
        if (++cnt == 64) {  // FP32 runs of 64, FP64 across runs
            sq += sqf;
            sqf = 0.f;
            cnt = 0;
        }
    }
    sq += sqf;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
    }
    const float sc = e4m3_scale(mx);
    const float inv = 1.f / sc;
    // pairs of columns: 16-bit stores
    uint8_t* row8 = A8 + i * ld8;
    for (int64_t c = 2 * lane; c < ld8; c += 64) {
        const float v0 = (c < n) ? load_a<BF>(A, base + c) * inv : 0.f;
        const float v1 = (c + 1 < n) ? load_a<BF>(A, base + c + 1) * inv : 0.f;
        *(uint16_t*)(row8 + c) = pack_e4m3(v0, v1);
    }
    if (lane == 0) {
        rs[i] = sc;
        if (fro2) atomicAdd(fro2, sq);
        if (amax) atomicMax(amax, __float_as_uint(mx));
    }
}

// Byte transpose: At8 (n x m stored column-major, i.e. At8[c * ldt + i]) from
// A8 (m x n row-major, ld8); 64 x 64 tiles through shared memory.  Rows of
// At8 beyond m (up to ldt) are zero.
__global__ void __launch_bounds__(256) transpose_u8_kernel(const uint8_t* __restrict__ A8, int64_t ld8, int64_t m,
                                                           int64_t n, uint8_t* __restrict__ At8, int64_t ldt)
{
    __shared__ uint8_t t[64][65];
    const int64_t i0 = (int64_t)blockIdx.y * 64, c0 = (int64_t)blockIdx.x * 64;
    for (int e = threadIdx.x; e < 64 * 64; e += 256) {
        const int r = e / 64, c = e % 64;
        const int64_t i = i0 + r, cc = c0 + c;
        t[r][c] = (i < m && cc < n) ? A8[i * ld8 + cc] : 0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * 64; e += 256) {
        const int c = e / 64, r = e % 64;
        const int64_t i = i0 + r, cc = c0 + c;
        if (cc < n && i < ldt) At8[cc * ldt + i] = t[r][c];
    }
}

// Panel quantisation, one CTA per column j < l_pad: P (K x l column-major,
// ld) with optional row factors r (K floats; the A^T side's S Q); column j
// becomes P8[j * ld8 + k] = e4m3(r_k P_kj / t_j) with t_j the column's power of
// two, written to ts[j]; rows K..ld8-1 and columns >= l are zero (ts = 1).
__global__ void __launch_bounds__(256) fp8_panel_kernel(const float* __restrict__ P, int64_t ld, int64_t K, int l,
                                                        const float* __restrict__ r, uint8_t* __restrict__ P8,
                                                        int64_t ld8, float* __restrict__ ts)
{
    __shared__ float red[8];
    const int j = blockIdx.x;
    const float* col = P + (int64_t)j * ld;
    float mx = 0.f;
    if (j < l)
        for (int64_t k = threadIdx.x; k < K; k += 256) mx = fmaxf(mx, fabsf(col[k] * (r ? r[k] : 1.f)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = red[0];
    for (int w = 1; w < 8; ++w) mx = fmaxf(mx, red[w]);
    const float sc = e4m3_scale(mx);
    const float inv = 1.f / sc;
    uint8_t* c8 = P8 + (int64_t)j * ld8;
    for (int64_t k = 2 * threadIdx.x; k < ld8; k += 512) {
        const float v0 = (j < l && k < K) ? col[k] * (r ? r[k] : 1.f) * inv : 0.f;
        const float v1 = (j < l && k + 1 < K) ? col[k + 1] * (r ? r[k + 1] : 1.f) * inv : 0.f;
        *(uint16_t*)(c8 + k) = pack_e4m3(v0, v1);
    }
    if (threadIdx.x == 0) ts[j] = sc;
}

}  // namespace

void launch_fp8_prep(cudaStream_t s, const void* A, int64_t lda, int a_bf16, int64_t m, int64_t n, uint8_t* A8,
                     int64_t ld8, uint8_t* At8, int64_t ldt, float* rs, double* fro2, unsigned int* amax)
{
    const unsigned nb = (unsigned)ceil_div(m, 8);
    if (a_bf16)
        fp8_rows_kernel<true><<<nb, 256, 0, s>>>(A, lda, m, n, A8, ld8, rs, fro2, amax);
    else
        fp8_rows_kernel<false><<<nb, 256, 0, s>>>(A, lda, m, n, A8, ld8, rs, fro2, amax);
    transpose_u8_kernel<<<dim3((unsigned)ceil_div(n, 64), (unsigned)ceil_div(ldt, 64)), 256, 0, s>>>(A8, ld8, m, n,
                                                                                                   At8, ldt);
    count_launches(2);
}

void launch_fp8_panel(cudaStream_t s, const float* P, int64_t ld, int64_t K, int l, int l_pad, const float* r,
                      uint8_t* P8, int64_t ld8, float* ts)
{
    fp8_panel_kernel<<<l_pad, 256, 0, s>>>(P, ld, K, l, r, P8, ld8, ts);
    count_launches();
}

}  // namespace rsvdgb
