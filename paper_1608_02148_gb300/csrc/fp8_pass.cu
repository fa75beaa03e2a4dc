// FP8 (E4M3) passes over A on the tensor cores (tcgen05.mma kind::f8f6f4,
// FP32 accumulation) for the power iterations of the mixed-precision rSVD:
//   A side  (TRANS = false): Y = A P, lanes = rows of A8 (row-major copy);
//   A^T side (TRANS = true): Z = A^T Q, lanes = rows of At8 (the transposed
//                            copy), K split across CTAs, partials summed
//                            afterwards.
// Both operands are K-major E4M3 tiles that TMA brings into shared memory
// with the 128-byte swizzle (128 K values per row); the MMA reads them there
// directly (no conversion step), four MMAs of K = 32 per stage.  Tensor
// memory holds only accumulators, two sets of G x l_pad columns, so the
// epilogue of one tile set overlaps the products of the next.  The epilogue
// multiplies column j by the panel's power of two and, on the A side, row i
// by A's row power of two (both exact).
// Roles (192 threads): warp 0 issues the TMA loads, warp 1 allocates tensor
// memory and issues the MMAs (one lane), warps 2..5 drain the accumulators
// (one TMEM lane quarter each).  Every mbarrier wait is bounded; on expiry the
// kernel records RSVDGB_ERR_TIMEOUT, waits (bounded) for its copies and MMAs
// in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "internal.cuh"
#include "ptx.cuh"

namespace rsvdgb {
namespace {
using namespace dev;

constexpr int kF8Threads = 192;
constexpr int kF8K = 128;      // K (bytes) per stage: one 128-byte swizzle row
constexpr int kF8Rows = 128;   // accumulator lanes per tile
constexpr int kF8MaxStages = 8;

struct F8Params {
    int64_t lanes;         // rows of the lane-major copy (m for A8, n for At8)
    int64_t k_total;       // K extent
    int64_t k_per_split;   // K per split (multiple of kF8K)
    int64_t num_tiles;     // 128-lane tiles
    int l_pad;
    int stages;
    float* out;            // column-major lanes x l_pad (ld_out); split s at out + s * split_stride
    int64_t ld_out;
    int64_t split_stride;
    const float* row_scale;  // per lane factor (A side: 2^e_i), or null
    const float* col_scale;  // per column factor (l_pad floats)
    int* status;
};

__device__ __forceinline__ void mma_f8_ss(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Instruction descriptor of kind::f8f6f4: A and B E4M3 (both K-major), D FP32.
__device__ __forceinline__ uint32_t e4m3_idesc(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int G>
__global__ void __launch_bounds__(kF8Threads, 1)
    f8_pass_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmP, F8Params p)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full_bar[kF8MaxStages], empty_bar[kF8MaxStages];
    __shared__ uint64_t accf_bar[2], acce_bar[2];
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = p.stages, l_pad = p.l_pad;
    const uint32_t a_tile = kF8Rows * kF8K;                 // 16 KB
    const uint32_t p_tile = (uint32_t)l_pad * kF8K;         // l_pad x 128 bytes
    const uint32_t stage_bytes = G * a_tile + p_tile;

    // work of this CTA: lane tiles [tile_begin, tile_end), K range
    const int64_t units = (p.num_tiles + G - 1) / G;
    const int64_t tile_begin = units * blockIdx.x / gridDim.x * G;
    const int64_t tile_end = std::min<int64_t>(p.num_tiles, units * (blockIdx.x + 1) / gridDim.x * G);
    const int64_t k_begin = (int64_t)blockIdx.y * p.k_per_split;
    const int64_t k_end = std::min<int64_t>(p.k_total, k_begin + p.k_per_split);
    const int64_t num_sets = (tile_end - tile_begin + G - 1) / G;
    const int64_t nk = (k_end > k_begin) ? (k_end - k_begin + kF8K - 1) / kF8K : 0;
    const uint32_t tmem_cols = 512;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf_bar[b], 1);
            mbar_init(&acce_bar[b], 4);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tmem = tmem_base_sh;

    if (warp == 0) {
        // =========================== TMA producer
        if (lane == 0 && nk > 0) {
            int64_t it = 0;
            bool ok = true;
            for (int64_t set = 0; set < num_sets && ok; ++set) {
                const int64_t t0 = tile_begin + set * G;
                const int gv = (int)std::min<int64_t>(G, tile_end - t0);
                for (int64_t c = 0; c < nk; ++c, ++it) {
                    const int s = (int)(it % S);
                    const uint32_t ph = (uint32_t)((it / S) & 1);
                    if (!(ok = mbar_wait(&empty_bar[s], ph ^ 1, &abort_flag, p.status))) break;
                    uint8_t* st = smem + (size_t)s * stage_bytes;
                    const int kc = (int)(k_begin + c * kF8K);
                    mbar_expect_tx(&full_bar[s], gv * a_tile + p_tile);
                    for (int g = 0; g < gv; ++g)
                        tma_load_2d(&tmA, &full_bar[s], st + g * a_tile, kc, (int)((t0 + g) * kF8Rows));
                    tma_load_2d(&tmP, &full_bar[s], st + G * a_tile, kc, 0);
                }
            }
            if (!ok) {
                const long long t0 = clock64();
                for (int64_t j = (it > S ? it - S : 0); j < it; ++j) {
                    const int s = (int)(j % S);
                    const uint32_t ph = (uint32_t)((j / S) & 1);
                    while (!mbar_test(&full_bar[s], ph) && clock64() - t0 < kSpinLimit) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // =========================== MMA issuer
        if (lane == 0 && nk > 0) {
            const uint32_t idesc = e4m3_idesc(kF8Rows, l_pad);
            int64_t it = 0;
            bool ok = true;
            for (int64_t set = 0; set < num_sets && ok; ++set) {
                const int64_t t0 = tile_begin + set * G;
                const int gv = (int)std::min<int64_t>(G, tile_end - t0);
                const int b = (int)(set & 1);
                // this accumulator set is free once the epilogue of two sets ago drained it
                if (!(ok = mbar_wait(&acce_bar[b], ((uint32_t)(set >> 1) & 1) ^ 1, &abort_flag, p.status))) break;
                tmem_fence_after();
                for (int64_t c = 0; c < nk; ++c, ++it) {
                    const int s = (int)(it % S);
                    const uint32_t ph = (uint32_t)((it / S) & 1);
                    if (!(ok = mbar_wait(&full_bar[s], ph, &abort_flag, p.status))) break;
                    tmem_fence_after();
                    const uint32_t st = smem_u32(smem + (size_t)s * stage_bytes);
                    const uint32_t pp = st + G * a_tile;
                    for (int g = 0; g < gv; ++g) {
                        const uint32_t d = tmem + (uint32_t)((b * G + g) * l_pad);
#pragma unroll
                        for (int kk = 0; kk < kF8K / 32; ++kk)
                            mma_f8_ss(d, sw128_desc(st + g * a_tile + kk * 32), sw128_desc(pp + kk * 32), idesc,
                                      (c > 0 || kk > 0) ? 1u : 0u);
                    }
                    mma_commit(&empty_bar[s]);
                }
                if (!ok) break;
                mma_commit(&accf_bar[b]);
            }
            if (!ok) {
                __shared__ uint64_t drain_bar;
                mbar_init(&drain_bar, 1);
                asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
                mma_commit(&drain_bar);
                const long long t0 = clock64();
                while (!mbar_test(&drain_bar, 0) && clock64() - t0 < kSpinLimit) {
                }
            }
        }
    } else {
        // =========================== epilogue (warps 2..5)
        const int q = warp & 3;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        float* out = p.out + (int64_t)blockIdx.y * p.split_stride;
        for (int64_t set = 0; set < num_sets && nk > 0; ++set) {
            const int64_t t0 = tile_begin + set * G;
            const int gv = (int)std::min<int64_t>(G, tile_end - t0);
            const int b = (int)(set & 1);
            if (!mbar_wait_warp(&accf_bar[b], (uint32_t)(set >> 1) & 1, &abort_flag, p.status)) break;
            tmem_fence_after();
            for (int g = 0; g < gv; ++g) {
                const int64_t idx = (t0 + g) * kF8Rows + q * 32 + lane;
                const float rs = (p.row_scale && idx < p.lanes) ? p.row_scale[idx] : 1.f;
                for (int j0 = 0; j0 < l_pad; j0 += 16) {
                    uint32_t v[16];
                    tmem_ld16(tmem + (uint32_t)((b * G + g) * l_pad + j0) + lane_off, v);
                    tmem_wait_ld();
                    if (idx < p.lanes) {
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            out[(int64_t)(j0 + e) * p.ld_out + idx] = __uint_as_float(v[e]) * rs * p.col_scale[j0 + e];
                    }
                }
            }
            tmem_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce_bar[b]);
        }
    }

    tmem_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tmem_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
    }
}

template <int G>
int launch_f8_typed(cudaStream_t s, const CUtensorMap& mA, const CUtensorMap& mP, const F8Params& p, dim3 grid,
                    size_t smem)
{
    if (cudaFuncSetAttribute(f8_pass_kernel<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return RSVDGB_ERR_CUDA;
    f8_pass_kernel<G><<<grid, kF8Threads, smem, s>>>(mA, mP, p);
    count_launches();
    return cudaGetLastError() == cudaSuccess ? RSVDGB_OK : RSVDGB_ERR_CUDA;
}

}  // namespace

int launch_f8_pass(cudaStream_t s, int sm_count, bool trans, const uint8_t* A8, int64_t lanes, int64_t k_total,
                   int64_t ld_a8, const uint8_t* P8, int64_t ld_p8, int l_pad, const float* row_scale,
                   const float* col_scale, float* out, int64_t ld_out, float* partial, int64_t* splits_out,
                   int* status)
{
    if (l_pad < 16 || l_pad > 256 || (l_pad % 16) || (ld_a8 % 16) || (ld_p8 % 16)) return RSVDGB_ERR_UNSUPPORTED;
    const int G = l_pad <= 128 ? 2 : 1;
    const size_t stage = (size_t)G * kF8Rows * kF8K + (size_t)l_pad * kF8K;
    const int stages = (int)std::min<size_t>(kF8MaxStages, (220 * 1024) / stage);
    if (stages < 2) return RSVDGB_ERR_UNSUPPORTED;
    const size_t smem = stages * stage + 1024;
    CUtensorMap mA, mP;
    bool ok = encode_2d(&mA, A8, k_total, lanes, ld_a8, kF8K, kF8Rows, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_DATA_TYPE_UINT8);
    ok = ok && encode_2d(&mP, P8, k_total, l_pad, ld_p8, kF8K, l_pad, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_DATA_TYPE_UINT8);
    if (!ok) return RSVDGB_ERR_CUDA;
    F8Params p{};
    p.lanes = lanes;
    p.k_total = k_total;
    p.num_tiles = ceil_div(lanes, kF8Rows);
    p.l_pad = l_pad;
    p.stages = stages;
    p.ld_out = ld_out;
    p.row_scale = row_scale;
    p.col_scale = col_scale;
    p.status = status;
    const int64_t units = ceil_div(p.num_tiles, G);
    int64_t splits = 1;
    if (trans) {
        splits = std::max<int64_t>(1, (int64_t)sm_count / std::max<int64_t>(units, 1));
        splits = std::min<int64_t>(splits, std::max<int64_t>(1, k_total / (4 * kF8K)));
    }
    p.k_per_split = round_up(ceil_div(k_total, splits), kF8K);
    splits = ceil_div(k_total, p.k_per_split);
    dim3 grid;
    if (splits == 1) {
        p.out = out;
        p.split_stride = 0;
        grid = dim3((unsigned)std::min<int64_t>(units, sm_count), 1);
    } else {
        if (!partial) return RSVDGB_ERR_INVALID_ARG;
        p.out = partial;
        p.split_stride = (int64_t)l_pad * ld_out;
        grid = dim3((unsigned)units, (unsigned)splits);
    }
    if (splits_out) *splits_out = splits == 1 ? 0 : splits;
    return G == 2 ? launch_f8_typed<2>(s, mA, mP, p, grid, smem) : launch_f8_typed<1>(s, mA, mP, p, grid, smem);
}

int64_t f8_pass_max_splits(int64_t lanes, int64_t k_total, int l_pad, int sm_count)
{
    const int G = l_pad <= 128 ? 2 : 1;
    const int64_t units = ceil_div(ceil_div(lanes, kF8Rows), G);
    int64_t splits = std::max<int64_t>(1, (int64_t)sm_count / std::max<int64_t>(units, 1));
    splits = std::min<int64_t>(splits, std::max<int64_t>(1, k_total / (4 * kF8K)));
    const int64_t kps = round_up(ceil_div(k_total, splits), kF8K);
    return ceil_div(k_total, kps);
}

}  // namespace rsvdgb
