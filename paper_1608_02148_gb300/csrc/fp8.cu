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

constexpr int kPrepRows = 32;      // rows of A per CTA: one 32-byte sector of each At8 column
constexpr int kPrepThreads = 256;  // 8 warps, 4 rows each
constexpr int kPrepCols = 2048;    // columns per chunk: 64 values per lane

// Bytes e of the four words w[0..3], gathered into one word (w[0]'s byte
// lowest): the 4 x 4 byte transpose.
__device__ __forceinline__ void transpose4x4(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, uint32_t* c)
{
    const uint32_t t0 = __byte_perm(w0, w1, 0x5140), t1 = __byte_perm(w2, w3, 0x5140);
    const uint32_t t2 = __byte_perm(w0, w1, 0x7362), t3 = __byte_perm(w2, w3, 0x7362);
    c[0] = __byte_perm(t0, t1, 0x5410);
    c[1] = __byte_perm(t0, t1, 0x7632);
    c[2] = __byte_perm(t2, t3, 0x5410);
    c[3] = __byte_perm(t2, t3, 0x7632);
}

// A (m x n row-major, lda) -> A8 (row-major, ld8), At8 (column-major,
// At8[c * ldt + i]) and rs, for 32 rows per CTA.  A warp takes 4 rows in
// turn: each lane loads EPL consecutive columns per load (a float4 or eight
// BF16 values when VEC), 2048 columns per chunk.  When n <= 2048 the row
// stays in registers, so A is read once: its max gives the row's power of
// two, then the quantised bytes go to A8 and to a 32 x 2048 shared tile;
// wider rows are read twice (max, then quantise, chunk by chunk).  The tile
// is written out transposed, 32 bytes (the CTA's rows) per column of At8.
// Rows m..ldt-1 of At8 come out zero, as do columns n..ld8-1 of A8.  The CTA
// adds its sum of squares (FP32 over at most 64 values per lane, FP64 above)
// to *fro2 and its max to *amax.
template <bool BF, bool VEC>
__global__ void __launch_bounds__(kPrepThreads, 2)
    fp8_prep_kernel(const void* __restrict__ A, int64_t lda, int64_t m, int64_t n, uint8_t* __restrict__ A8,
                    int64_t ld8, uint8_t* __restrict__ At8, int64_t ldt, float* __restrict__ rs, double* fro2,
                    unsigned int* amax)
{
    extern __shared__ __align__(16) uint8_t tile[];  // kPrepRows x kPrepCols bytes
    __shared__ double wsq[kPrepThreads / 32];
    __shared__ float wmx[kPrepThreads / 32];
    constexpr int EPL = BF ? 8 : 4;  // elements per lane and load
    constexpr int NT = 64 / EPL;     // loads per lane and chunk
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i0 = (int64_t)blockIdx.x * kPrepRows;
    const int nch = (int)((ld8 + kPrepCols - 1) / kPrepCols);
    float v[NT][EPL];

    auto load = [&](int64_t i, int ch) {
        const int64_t base = i * lda;
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int64_t c = (int64_t)ch * kPrepCols + EPL * (lane + 32 * t);
            if (VEC && c + EPL <= n) {
                if (BF) {
                    const uint4 q = __ldcs((const uint4*)((const uint16_t*)A + base + c));
                    const uint32_t u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        v[t][2 * e] = __uint_as_float(u[e] << 16);
                        v[t][2 * e + 1] = __uint_as_float(u[e] & 0xFFFF0000u);
                    }
                } else {
                    const float4 q = __ldcs((const float4*)((const float*)A + base + c));
                    v[t][0] = q.x;
                    v[t][1] = q.y;
                    v[t][2] = q.z;
                    v[t][3] = q.w;
                }
            } else {
#pragma unroll
                for (int e = 0; e < EPL; ++e) v[t][e] = (c + e < n) ? load_a<BF>(A, base + c + e) : 0.f;
            }
        }
    };
    // max and sum of squares of the loaded chunk, over the warp
    auto reduce = [&](float& mx, double& sq) {
        float m1 = 0.f, s1 = 0.f;
#pragma unroll
        for (int t = 0; t < NT; ++t)
#pragma unroll
            for (int e = 0; e < EPL; ++e) {
                m1 = fmaxf(m1, fabsf(v[t][e]));
                s1 = fmaf(v[t][e], v[t][e], s1);
            }
        double s2 = s1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        mx = fmaxf(mx, m1);
        sq += s2;
    };
    // quantise the loaded chunk of row r (global row i) into the tile and A8
    auto quant = [&](int r, int64_t i, int ch, float inv) {
#pragma unroll
        for (int t = 0; t < NT; ++t) {
            const int c = EPL * (lane + 32 * t);
            const int64_t gc = (int64_t)ch * kPrepCols + c;
            uint32_t q[EPL / 4];
#pragma unroll
            for (int e = 0; e < EPL / 4; ++e)
                q[e] = (uint32_t)pack_e4m3(v[t][4 * e] * inv, v[t][4 * e + 1] * inv) |
                       ((uint32_t)pack_e4m3(v[t][4 * e + 2] * inv, v[t][4 * e + 3] * inv) << 16);
            if (BF) {
                *(uint2*)(tile + r * kPrepCols + c) = make_uint2(q[0], q[EPL / 4 - 1]);
                if (gc < ld8) *(uint2*)(A8 + i * ld8 + gc) = make_uint2(q[0], q[EPL / 4 - 1]);
            } else {
                *(uint32_t*)(tile + r * kPrepCols + c) = q[0];
                if (gc < ld8) *(uint32_t*)(A8 + i * ld8 + gc) = q[0];
            }
        }
    };
    auto zero_row = [&](int r) {
        for (int c = 4 * lane; c < kPrepCols; c += 128) *(uint32_t*)(tile + r * kPrepCols + c) = 0u;
    };
    // the tile's columns [ch * 2048, ...) < n -> At8, 32 (or 16 at the end) bytes each
    auto store_t = [&](int ch) {
        const int64_t c0 = (int64_t)ch * kPrepCols;
        const int cc = (int)((n - c0 < kPrepCols) ? n - c0 : kPrepCols);
        const bool full = i0 + kPrepRows <= ldt;
        for (int g = threadIdx.x; 4 * g < cc; g += kPrepThreads) {
            uint32_t col[4][8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                uint32_t w[4], c4[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) w[r] = *(const uint32_t*)(tile + (4 * q + r) * kPrepCols + 4 * g);
                transpose4x4(w[0], w[1], w[2], w[3], c4);
#pragma unroll
                for (int e = 0; e < 4; ++e) col[e][q] = c4[e];
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (4 * g + e >= cc) break;
                uint8_t* dst = At8 + (c0 + 4 * g + e) * ldt + i0;
                *(uint4*)dst = make_uint4(col[e][0], col[e][1], col[e][2], col[e][3]);
                if (full) *(uint4*)(dst + 16) = make_uint4(col[e][4], col[e][5], col[e][6], col[e][7]);
            }
        }
    };

    float cmx = 0.f;
    double csq = 0.0;
    if (nch == 1) {
        for (int j = 0; j < kPrepRows / 8; ++j) {
            const int r = warp * (kPrepRows / 8) + j;
            const int64_t i = i0 + r;
            if (i < m) {
                load(i, 0);
                float mx = 0.f;
                double sq = 0.0;
                reduce(mx, sq);
                const float sc = e4m3_scale(mx);
                if (lane == 0) rs[i] = sc;
                cmx = fmaxf(cmx, mx);
                csq += sq;
                quant(r, i, 0, 1.f / sc);
            } else {
                zero_row(r);
            }
        }
        __syncthreads();
        store_t(0);
    } else {
        float inv[kPrepRows / 8];
        for (int j = 0; j < kPrepRows / 8; ++j) {
            const int64_t i = i0 + warp * (kPrepRows / 8) + j;
            inv[j] = 1.f;
            if (i >= m) continue;
            float mx = 0.f;
            double sq = 0.0;
            for (int ch = 0; ch < nch; ++ch) {
                load(i, ch);
                reduce(mx, sq);
            }
            const float sc = e4m3_scale(mx);
            if (lane == 0) rs[i] = sc;
            inv[j] = 1.f / sc;
            cmx = fmaxf(cmx, mx);
            csq += sq;
        }
        for (int ch = 0; ch < nch; ++ch) {
            for (int j = 0; j < kPrepRows / 8; ++j) {
                const int r = warp * (kPrepRows / 8) + j;
                const int64_t i = i0 + r;
                if (i < m) {
                    load(i, ch);
                    quant(r, i, ch, inv[j]);
                } else {
                    zero_row(r);
                }
            }
            __syncthreads();
            store_t(ch);
            __syncthreads();
        }
    }
    if (lane == 0) {
        wsq[warp] = csq;
        wmx[warp] = cmx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        float mx = 0.f;
        for (int w = 0; w < kPrepThreads / 32; ++w) {
            s += wsq[w];
            mx = fmaxf(mx, wmx[w]);
        }
        if (fro2) atomicAdd(fro2, s);
        if (amax) atomicMax(amax, __float_as_uint(mx));
    }
}

constexpr int kPanelRows = 1024;  // rows per CTA of the panel kernels: a float4 per thread
constexpr int kPanelCols = 16;    // columns per CTA of the column-max kernel

// Column maxima of the panel P (K x l column-major, ld a multiple of 4, rows
// scaled by r_k when r is given): CTA (x, y) takes rows [1024 x, ...) of
// columns [16 y, ...) and folds its maxima into cm[j] (float bits, atomicMax;
// the values are non-negative).  The last CTA to finish (counted in
// cm[l_pad]) turns them into the column powers of two ts[j] (1 for columns
// >= l) and zeroes cm[0..l_pad] for the next panel.
__global__ void __launch_bounds__(256) panel_max_kernel(const float* __restrict__ P, int64_t ld, int64_t K, int l,
                                                        int l_pad, const float* __restrict__ r,
                                                        unsigned int* cm, float* __restrict__ ts)
{
    __shared__ float red[kPanelCols][8];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * kPanelRows + 4 * threadIdx.x;
    const int j0 = blockIdx.y * kPanelCols;
    float rk[4] = {1.f, 1.f, 1.f, 1.f};
    if (r)
#pragma unroll
        for (int e = 0; e < 4; ++e) rk[e] = (k + e < K) ? r[k + e] : 0.f;
    float x[kPanelCols][4];
#pragma unroll
    for (int c = 0; c < kPanelCols; ++c) {
        const int j = j0 + c;
        if (j < l && k + 3 < K) {
            const float4 q = *(const float4*)(P + (int64_t)j * ld + k);
            x[c][0] = q.x;
            x[c][1] = q.y;
            x[c][2] = q.z;
            x[c][3] = q.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) x[c][e] = (j < l && k + e < K) ? P[(int64_t)j * ld + k + e] : 0.f;
        }
    }
#pragma unroll
    for (int c = 0; c < kPanelCols; ++c) {
        float mx = 0.f;
#pragma unroll
        for (int e = 0; e < 4; ++e) mx = fmaxf(mx, fabsf(x[c][e] * rk[e]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) red[c][warp] = mx;
    }
    __syncthreads();
    if (threadIdx.x < kPanelCols && j0 + (int)threadIdx.x < l) {
        float mx = red[threadIdx.x][0];
        for (int w = 1; w < 8; ++w) mx = fmaxf(mx, red[threadIdx.x][w]);
        atomicMax(&cm[j0 + threadIdx.x], __float_as_uint(mx));
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&cm[l_pad], 1u) == gridDim.x * gridDim.y - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int j = threadIdx.x; j < l_pad; j += blockDim.x) {
        const float mx = __uint_as_float(__ldcg(&cm[j]));
        ts[j] = (j < l) ? e4m3_scale(mx) : 1.f;
        cm[j] = 0u;
    }
    if (threadIdx.x == 0) cm[l_pad] = 0u;
}

// P8[j * ld8 + k] = e4m3(r_k P_kj / ts_j) for k < ld8, j < l_pad (zero
// outside K x l); four rows per thread.
__global__ void __launch_bounds__(256) panel_quant_kernel(const float* __restrict__ P, int64_t ld, int64_t K, int l,
                                                          const float* __restrict__ r, const float* __restrict__ ts,
                                                          uint8_t* __restrict__ P8, int64_t ld8)
{
    const int64_t k = (int64_t)blockIdx.x * kPanelRows + 4 * threadIdx.x;
    const int j = blockIdx.y;
    if (k >= ld8) return;
    float x[4] = {0.f, 0.f, 0.f, 0.f};
    if (j < l) {
        if (k + 3 < K) {
            const float4 q = *(const float4*)(P + (int64_t)j * ld + k);
            x[0] = q.x;
            x[1] = q.y;
            x[2] = q.z;
            x[3] = q.w;
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) x[e] = (k + e < K) ? P[(int64_t)j * ld + k + e] : 0.f;
        }
        const float inv = 1.f / ts[j];
#pragma unroll
        for (int e = 0; e < 4; ++e) x[e] *= (r && k + e < K ? r[k + e] : 1.f) * inv;
    }
    *(uint32_t*)(P8 + (int64_t)j * ld8 + k) =
        (uint32_t)pack_e4m3(x[0], x[1]) | ((uint32_t)pack_e4m3(x[2], x[3]) << 16);
}

template <bool BF, bool VEC>
void prep_typed(cudaStream_t s, const void* A, int64_t lda, int64_t m, int64_t n, uint8_t* A8, int64_t ld8,
                uint8_t* At8, int64_t ldt, float* rs, double* fro2, unsigned int* amax)
{
    const int smem = kPrepRows * kPrepCols;
    cudaFuncSetAttribute(fp8_prep_kernel<BF, VEC>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    fp8_prep_kernel<BF, VEC><<<(unsigned)ceil_div(ldt, kPrepRows), kPrepThreads, smem, s>>>(A, lda, m, n, A8, ld8,
                                                                                            At8, ldt, rs, fro2, amax);
}

}  // namespace

void launch_fp8_prep(cudaStream_t s, const void* A, int64_t lda, int a_bf16, int64_t m, int64_t n, uint8_t* A8,
                     int64_t ld8, uint8_t* At8, int64_t ldt, float* rs, double* fro2, unsigned int* amax)
{
    const int epl = a_bf16 ? 8 : 4;
    const bool vec = lda % epl == 0 && ((uintptr_t)A & 15) == 0;
    if (a_bf16) {
        if (vec)
            prep_typed<true, true>(s, A, lda, m, n, A8, ld8, At8, ldt, rs, fro2, amax);
        else
            prep_typed<true, false>(s, A, lda, m, n, A8, ld8, At8, ldt, rs, fro2, amax);
    } else {
        if (vec)
            prep_typed<false, true>(s, A, lda, m, n, A8, ld8, At8, ldt, rs, fro2, amax);
        else
            prep_typed<false, false>(s, A, lda, m, n, A8, ld8, At8, ldt, rs, fro2, amax);
    }
    count_launches();
}

void launch_fp8_panel(cudaStream_t s, const float* P, int64_t ld, int64_t K, int l, int l_pad, const float* r,
                      uint8_t* P8, int64_t ld8, float* ts, unsigned int* cm)
{
    panel_max_kernel<<<dim3((unsigned)ceil_div(K, kPanelRows), (unsigned)ceil_div(l, kPanelCols)), 256, 0, s>>>(
        P, ld, K, l, l_pad, r, cm, ts);
    panel_quant_kernel<<<dim3((unsigned)ceil_div(ld8, kPanelRows), (unsigned)l_pad), 256, 0, s>>>(P, ld, K, l, r, ts,
                                                                                                 P8, ld8);
    count_launches(2);
}

}  // namespace rsvdgb
