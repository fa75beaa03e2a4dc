// FP32 FMA (SIMT) tall-skinny products for the passes over A and for the
// small Gram / basis-change products of CholeskyQR.
//
// This family is FP32 throughout: it is the accuracy reference of the GPU
// path and the fallback engine for shapes the tensor-core kernels do not take.
// Tile: 64 x 64 outputs per 256-thread CTA, 4 x 4 per thread, K step 16.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace rsvdgb {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <bool AT, bool A_BF16>
__device__ __forceinline__ float load_a(const void* A, int64_t lda, int64_t i, int64_t k)
{
    const int64_t off = AT ? k * lda + i : i * lda + k;
    if (A_BF16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(A)[off]);
    return reinterpret_cast<const float*>(A)[off];
}

template <bool AT, bool BT, bool CT, bool A_BF16>
__global__ void __launch_bounds__(NT) simt_gemm_kernel(GemmArgs g, int64_t ntiles_n, int64_t k_per_split)
{
    __shared__ __align__(16) float As[BK][BM + 4];
    __shared__ __align__(16) float Bs[BK][BN + 4];

    const int tid = threadIdx.x;
    const int tx = tid & 15;  // i group
    const int ty = tid >> 4;  // j group
    const int64_t tile = blockIdx.x;
    const int64_t tn = tile % ntiles_n;
    const int64_t tm = tile / ntiles_n;
    const int64_t i0 = tm * BM, j0 = tn * BN;
    const int64_t kbeg = (int64_t)blockIdx.z * k_per_split;
    const int64_t kend = min(g.K, kbeg + k_per_split);
    const bool do_fro = (g.fro2 != nullptr) && tn == 0;

    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    float fro = 0.f;

    for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
        // ---- stage op(A) tile (BM x BK) into As[k][i]
#pragma unroll
        for (int e = 0; e < (BM * BK) / NT; ++e) {
            const int idx = tid + e * NT;
            int r, c;  // r: i offset, c: k offset
            if (AT) {  // consecutive threads walk i (contiguous in memory)
                r = idx % BM;
                c = idx / BM;
            } else {  // consecutive threads walk k
                c = idx % BK;
                r = idx / BK;
            }
            const int64_t i = i0 + r, k = k0 + c;
            float v = 0.f;
            if (i < g.M && k < kend) v = load_a<AT, A_BF16>(g.A, g.lda, i, k);
            As[c][r] = v;
            fro += v * v;
        }
        // ---- stage op(B) tile (BK x BN) into Bs[k][j]
#pragma unroll
        for (int e = 0; e < (BN * BK) / NT; ++e) {
            const int idx = tid + e * NT;
            int c, r;  // c: j offset, r: k offset
            if (BT) {
                r = idx % BK;
                c = idx / BK;
            } else {
                c = idx % BN;
                r = idx / BN;
            }
            const int64_t j = j0 + c, k = k0 + r;
            float v = 0.f;
            if (j < g.N && k < kend) v = BT ? g.B[j * g.ldb + k] : g.B[k * g.ldb + j];
            Bs[r][c] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a4 = *reinterpret_cast<const float4*>(&As[kk][tx * 4]);
            const float4 b4 = *reinterpret_cast<const float4*>(&Bs[kk][ty * 4]);
            const float av[4] = {a4.x, a4.y, a4.z, a4.w};
            const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }

    float* C = g.C + (int64_t)blockIdx.z * g.split_stride;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t i = i0 + tx * 4 + a;
        if (i >= g.M) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t j = j0 + ty * 4 + b;
            if (j >= g.N) continue;
            if (CT)
                C[j * g.ldc + i] = acc[a][b];
            else
                C[i * g.ldc + j] = acc[a][b];
        }
    }

    if (do_fro) {
        // block reduction of the squares, then one FP64 atomic per CTA
        __shared__ float red[NT / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
        if ((tid & 31) == 0) red[tid >> 5] = fro;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < NT / 32; ++w) t += (double)red[w];
            atomicAdd(g.fro2, t);
        }
    }
}

template <bool AT, bool BT, bool CT>
void launch_typed(cudaStream_t s, const GemmArgs& g)
{
    const int64_t ntn = ceil_div(g.N, BN), ntm = ceil_div(g.M, BM);
    const int splits = g.splits < 1 ? 1 : g.splits;
    int64_t kps = ceil_div(g.K, splits);
    kps = round_up(kps, BK);
    dim3 grid((unsigned)(ntn * ntm), 1, (unsigned)splits);
    if (g.a_bf16)
        simt_gemm_kernel<AT, BT, CT, true><<<grid, NT, 0, s>>>(g, ntn, kps);
    else
        simt_gemm_kernel<AT, BT, CT, false><<<grid, NT, 0, s>>>(g, ntn, kps);
    count_launches();
}

// out = sum over the splits of part (rows x cols, leading dimension ld, split
// s at part + s * split_stride).  A CTA takes one row and 32 consecutive
// columns; warp w sums splits w, w + 8, ... with four independent
// accumulators (all loads of a lane in flight together), then the eight warp
// sums are added in a fixed order, so the result does not depend on timing.
__global__ void __launch_bounds__(256) reduce_splits_kernel(const float* __restrict__ part, int splits,
                                                            int64_t split_stride, int64_t rows, int64_t cols,
                                                            int64_t ld, float* __restrict__ out, int64_t ld_out)
{
    __shared__ float red[8][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t ncb = (cols + 31) / 32;
    const int64_t r = blockIdx.x / ncb;
    const int64_t c = (blockIdx.x % ncb) * 32 + lane;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    if (c < cols) {
        const float* src = part + r * ld + c;
        int s = warp;
        for (; s + 24 < splits; s += 32) {
            a0 += src[(int64_t)s * split_stride];
            a1 += src[(int64_t)(s + 8) * split_stride];
            a2 += src[(int64_t)(s + 16) * split_stride];
            a3 += src[(int64_t)(s + 24) * split_stride];
        }
        for (; s < splits; s += 8) a0 += src[(int64_t)s * split_stride];
    }
    red[warp][lane] = (a0 + a1) + (a2 + a3);
    __syncthreads();
    if (warp == 0 && c < cols) {
        const float t = ((red[0][lane] + red[1][lane]) + (red[2][lane] + red[3][lane])) +
                        ((red[4][lane] + red[5][lane]) + (red[6][lane] + red[7][lane]));
        out[r * ld_out + c] = t;
    }
}

}  // namespace

void launch_simt_gemm(cudaStream_t s, bool AT, bool BT, bool CT, const GemmArgs& g)
{
    const int key = (AT ? 4 : 0) | (BT ? 2 : 0) | (CT ? 1 : 0);
    switch (key) {
        case 0: launch_typed<false, false, false>(s, g); break;
        case 1: launch_typed<false, false, true>(s, g); break;
        case 2: launch_typed<false, true, false>(s, g); break;
        case 3: launch_typed<false, true, true>(s, g); break;
        case 4: launch_typed<true, false, false>(s, g); break;
        case 5: launch_typed<true, false, true>(s, g); break;
        case 6: launch_typed<true, true, false>(s, g); break;
        default: launch_typed<true, true, true>(s, g); break;
    }
}

void launch_reduce_splits(cudaStream_t s, const float* part, int splits, int64_t split_stride, int64_t rows,
                          int64_t cols, int64_t ld, float* out, int64_t ld_out)
{
    if (rows * cols == 0) return;
    const int64_t blocks = rows * ((cols + 31) / 32);
    reduce_splits_kernel<<<(unsigned)blocks, 256, 0, s>>>(part, splits, split_stride, rows, cols, ld, out, ld_out);
    count_launches();
}

}  // namespace rsvdgb
