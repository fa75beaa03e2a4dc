// Gram matrices G = X^T X and cross products G = X^T Z of tall column-major
// FP32 matrices (rows x l, l <= 128) on the tensor cores, FP32-accurate
// (3xTF32), reading each input once.
//
// These are the Gram steps of CholeskyQR (the "qr" of Algorithm
// sub_iterations and Algorithm rqb step 9) and the cross product
// R_B = Q_B^T B^T of the small SVD.  Column j of X is contiguous, so X^T
// stored by columns is K-major: one TMA box of 32 rows of X and all l
// columns lands in shared memory as an l x 32 K-major tile with the 128-byte
// swizzle, which is at the same time the A operand (M = 128 rows, the rows
// beyond l kept at zero) and the B operand (N = l_pad) of
// tcgen05.mma.kind::tf32.  Converter warps split the tile in place,
// x = x_hi + x_lo (x_hi = x with the low 13 mantissa bits cleared, x_lo the
// exact FP32 remainder), and the MMA warp issues x_hi z_hi + x_hi z_lo +
// x_lo z_hi per K step of 8, accumulating in FP32 in tensor memory; each
// product is within 2^-19 |x||z| (the same split and bound as the passes
// over A).  The tensor core's FP32 accumulation does not round to nearest:
// each accumulate step drops the low bits toward zero, so a long chain of
// accumulations shrinks a sum of positive terms (a Gram diagonal) by a
// relative bias that grows with the chain (about 5e-5 after 500 MMAs).  So
// every two 32-row stages accumulate into a fresh tensor-memory accumulator
// (four in rotation), and the epilogue warps add it into FP32 registers
// (round to nearest) one such chunk later, while the tensor core runs on.  Every CTA takes a range of rows and
// writes its l x l partial; the partials are summed by the split reduction.
//
// Roles (320 threads): warp 0 issues the TMA loads, warp 1 allocates tensor
// memory and issues the MMAs, warps 2..9 convert and run the epilogue: a
// converter splits half of its row of the tile (four of its eight 16-byte
// chunks), and in the drain each of the two warps of a TMEM lane quarter
// sums half of the accumulator's columns.  All
// mbarrier waits are bounded (see ptx.cuh); on expiry the kernel records
// RSVDGB_ERR_TIMEOUT and leaves after its copies and MMAs in flight drain.
#include <algorithm>

#include "internal.cuh"
#include "ptx.cuh"

namespace rsvdgb {
namespace {
using namespace dev;

constexpr int kBK = 32;       // rows of X per stage (one 128-byte swizzle row of FP32)
constexpr int kRows = 128;    // tile rows (columns of X, padded): the MMA's M
constexpr int kConvWarps = 8;
constexpr int kThreads = 64 + 32 * kConvWarps;
constexpr int kMaxStages = 8;
constexpr uint32_t kTile = kRows * kBK * 4;  // 16 KB

struct GramParams {
    int64_t rows;       // K extent (rows of X)
    int l;              // rows / columns of the partial that are written
    int l_pad;          // MMA N: multiple of 16, <= 128
    int64_t k_per_cta;  // multiple of kBK
    int stages;
    float* part;        // CTA c writes part + c * l_pad * l_pad (row-major, ld l_pad)
    int* status;
};

template <bool CROSS>
__global__ void __launch_bounds__(kThreads, 1)
    tc_gram_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmZ, GramParams p)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    // stage: X tile (FP32, converted in place to x_hi), x_lo [, Z tile, z_lo]
    constexpr uint32_t kStage = (CROSS ? 4 : 2) * kTile;
    __shared__ uint64_t full_bar[kMaxStages], conv_bar[kMaxStages], empty_bar[kMaxStages];
    constexpr int kAcc = 4;  // accumulators in rotation
    constexpr int kSpa = 2;  // stages per accumulator chunk (24 MMAs)
    constexpr int kLag = 1;  // chunk ch is drained once chunk ch + kLag is converted
    __shared__ uint64_t acc_bar, accf_bar[kAcc], acce_bar[kAcc];
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = p.stages;
    const int l_pad = p.l_pad;
    const int64_t k_begin = (int64_t)blockIdx.x * p.k_per_cta;
    const int64_t k_end = min(p.rows, k_begin + p.k_per_cta);
    const int64_t nk = (k_end > k_begin) ? (k_end - k_begin + kBK - 1) / kBK : 0;
    const uint32_t load_bytes = (uint32_t)l_pad * kBK * 4;  // one TMA box: l_pad rows of 128 B
    constexpr uint32_t kTmemCols = 512;  // four accumulators of 128 columns

    // rows l_pad..127 of every tile stay zero (TMA and the converters only
    // touch rows < l_pad)
    for (int s = 0; s < S; ++s)
        for (int t = 0; t < (CROSS ? 4 : 2); ++t) {
            float4* tile = (float4*)(smem + (size_t)s * kStage + t * kTile);
            for (int e = l_pad * 8 + threadIdx.x; e < kRows * 8; e += kThreads) tile[e] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&conv_bar[s], kConvWarps);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&acc_bar, 1);
        for (int a = 0; a < kAcc; ++a) {
            mbar_init(&accf_bar[a], 1);
            mbar_init(&acce_bar[a], kConvWarps);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_sh)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_proxy_async();  // the zeroed rows are read by the tensor cores
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tmem = tmem_base_sh;

    if (warp == 0) {
        // =========================== TMA producer
        if (lane == 0) {
            bool ok = true;
            int64_t c = 0;
            for (; c < nk; ++c) {
                const int s = (int)(c % S);
                const uint32_t ph = (uint32_t)((c / S) & 1);
                if (!(ok = mbar_wait(&empty_bar[s], ph ^ 1, &abort_flag, p.status))) break;
                uint8_t* st = smem + (size_t)s * kStage;
                const int kc = (int)(k_begin + c * kBK);
                mbar_expect_tx(&full_bar[s], (CROSS ? 2 : 1) * load_bytes);
                tma_load_2d(&tmX, &full_bar[s], st, kc, 0);
                if (CROSS) tma_load_2d(&tmZ, &full_bar[s], st + 2 * kTile, kc, 0);
            }
            if (!ok) {
                // wait (bounded) for the copies already issued
                const long long t0 = clock64();
                for (int64_t j = (c > S ? c - S : 0); j < c; ++j) {
                    const int s = (int)(j % S);
                    const uint32_t ph = (uint32_t)((j / S) & 1);
                    while (!mbar_test(&full_bar[s], ph) && clock64() - t0 < kSpinLimit) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // =========================== MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tf32_idesc(kRows, l_pad);
            bool ok = true;
            for (int64_t c = 0; c < nk; ++c) {
                const int s = (int)(c % S);
                const uint32_t ph = (uint32_t)((c / S) & 1);
                const int64_t ch = c / kSpa;
                const int a = (int)(ch % kAcc);  // accumulator of this chunk
                // accumulator a was last used by chunk ch - kAcc: wait until it is drained
                if (c % kSpa == 0 && ch >= kAcc &&
                    !(ok = mbar_wait(&acce_bar[a], (uint32_t)((ch / kAcc - 1) & 1), &abort_flag, p.status)))
                    break;
                if (!(ok = mbar_wait(&conv_bar[s], ph, &abort_flag, p.status))) break;
                tmem_fence_after();
                const uint32_t d = tmem + (uint32_t)(a * kRows);
                const uint32_t xhi = smem_u32(smem + (size_t)s * kStage);
                const uint32_t xlo = xhi + kTile;
                const uint32_t zhi = CROSS ? xhi + 2 * kTile : xhi;
                const uint32_t zlo = CROSS ? zhi + kTile : xlo;
#pragma unroll
                for (int kk = 0; kk < kBK / 8; ++kk) {
                    const uint32_t acc = (c % kSpa > 0 || kk > 0) ? 1u : 0u;
                    mma_tf32_ss(d, sw128_desc(xhi + kk * 32), sw128_desc(zhi + kk * 32), idesc, acc);
                    mma_tf32_ss(d, sw128_desc(xhi + kk * 32), sw128_desc(zlo + kk * 32), idesc, 1u);
                    mma_tf32_ss(d, sw128_desc(xlo + kk * 32), sw128_desc(zhi + kk * 32), idesc, 1u);
                }
                mma_commit(&empty_bar[s]);
                if (c % kSpa == kSpa - 1 || c == nk - 1) mma_commit(&accf_bar[a]);
            }
            // arrives once every MMA issued above has completed (at once if none)
            mma_commit(&acc_bar);
            (void)ok;
        }
    } else {
        // =========================== converters + epilogue (warps 2..9)
        const int cw = warp - 2;                // converter warp 0..7
        const int half = cw >> 2;               // half of each row (converter) / of the columns (drain)
        const int t = (cw & 3) * 32 + lane;     // tile row (column of X) of this thread
        // TMEM lane quarter warp % 4 holds accumulator rows 32 (warp % 4) ..;
        // this thread sums row r over the stages in FP32 registers
        const int q = warp & 3;
        const int r = q * 32 + lane;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        float sum[kRows / 2];  // this warp's half of the columns: half * 64 + j
#pragma unroll
        for (int j = 0; j < kRows / 2; ++j) sum[j] = 0.f;
        const int c0 = half * (kRows / 2);
        // add the accumulator of chunk ch into sum and hand it back to the MMA warp
        auto drain = [&](int64_t ch) -> bool {
            const int a = (int)(ch % kAcc);
            if (!mbar_wait_warp(&accf_bar[a], (uint32_t)((ch / kAcc) & 1), &abort_flag, p.status)) return false;
            tmem_fence_after();
            // two batches of four 16-column loads, one wait each
            {
                uint32_t v[4][16];
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (c0 + 16 * t < l_pad) tmem_ld16(tmem + (uint32_t)(a * kRows + c0 + 16 * t) + lane_off, v[t]);
                tmem_wait_ld();
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (c0 + 16 * t < l_pad) {
                        tmem_regs_ready(v[t]);
#pragma unroll
                        for (int e = 0; e < 16; ++e) sum[16 * t + e] += __uint_as_float(v[t][e]);
                    }
            }
            tmem_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce_bar[a]);
            return true;
        };
        bool ok = true;
        for (int64_t c = 0; c < nk; ++c) {
            const int s = (int)(c % S);
            const uint32_t ph = (uint32_t)((c / S) & 1);
            if (!(ok = mbar_wait_warp(&full_bar[s], ph, &abort_flag, p.status))) break;
            if (t < l_pad) {
#pragma unroll
                for (int mtx = 0; mtx < (CROSS ? 2 : 1); ++mtx) {
                    // row t: 8 chunks of 16 bytes; the split keeps the layout.
                    // Chunk j is visited as j ^ (t & 7) so that the 32 rows of a
                    // warp spread over all banks (rows are 128 bytes apart).
                    float4* hi = (float4*)(smem + (size_t)s * kStage + mtx * 2 * kTile + t * 128);
                    float4* lo = (float4*)((uint8_t*)hi + kTile);
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        const int ch = (half * 4 + jj) ^ (t & 7);
                        const float4 v = hi[ch];
                        float4 h, r;
                        h.x = __uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u);
                        h.y = __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u);
                        h.z = __uint_as_float(__float_as_uint(v.z) & 0xFFFFE000u);
                        h.w = __uint_as_float(__float_as_uint(v.w) & 0xFFFFE000u);
                        r.x = v.x - h.x;
                        r.y = v.y - h.y;
                        r.z = v.z - h.z;
                        r.w = v.w - h.w;
                        hi[ch] = h;
                        lo[ch] = r;
                    }
                }
            }
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&conv_bar[s]);
            // at the end of chunk ch: drain chunk ch - kLag (the tensor core has
            // the chunks after it queued meanwhile)
            if ((c % kSpa == kSpa - 1 || c == nk - 1) && c / kSpa >= kLag && !(ok = drain(c / kSpa - kLag))) break;
        }
        const int64_t nch = (nk + kSpa - 1) / kSpa;
        for (int64_t ch = (nch > kLag ? nch - kLag : 0); ok && ch < nch; ++ch) ok = drain(ch);
        // ---- epilogue: row r of the partial from the FP32 sums
        float* out = p.part + (int64_t)blockIdx.x * l_pad * l_pad;
        if (ok && r < l_pad) {
#pragma unroll
            for (int j0 = 0; j0 < kRows / 2; j0 += 16)
                if (c0 + j0 < l_pad)
#pragma unroll
                    for (int e = 0; e < 16; ++e) out[(int64_t)r * l_pad + c0 + j0 + e] = sum[j0 + e];
        }
        if (!ok) {
            // the MMA warp's final commit tells when its work has drained
            const long long t0 = clock64();
            while (!mbar_test(&acc_bar, 0) && clock64() - t0 < kSpinLimit) {
            }
        }
    }

    tmem_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tmem_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

}  // namespace

bool tc_gram_supported(const float* X, const float* Z, int64_t ld, int l_pad)
{
    if (l_pad < 16 || l_pad > kRows || (l_pad % 16)) return false;
    if ((ld * 4) % 16 || ((uintptr_t)X % 16) || (Z && ((uintptr_t)Z % 16))) return false;
    return get_encoder() != nullptr;
}

int64_t tc_gram_max_ctas(int sm_count) { return sm_count; }

int launch_tc_gram(cudaStream_t s, int sm_count, const float* X, const float* Z, int64_t rows, int64_t ld, int l,
                   int l_pad, float* part, float* G, int* status)
{
    if (!tc_gram_supported(X, Z, ld, l_pad) || rows < 1 || l < 1 || l > l_pad) return RSVDGB_ERR_UNSUPPORTED;
    const bool cross = Z != nullptr && Z != X;
    CUtensorMap mX, mZ;
    bool ok = encode_2d(&mX, X, (uint64_t)rows, (uint64_t)l_pad, (uint64_t)ld * 4, kBK, (uint32_t)l_pad,
                        CU_TENSOR_MAP_SWIZZLE_128B);
    if (cross)
        ok = ok && encode_2d(&mZ, Z, (uint64_t)rows, (uint64_t)l_pad, (uint64_t)ld * 4, kBK, (uint32_t)l_pad,
                             CU_TENSOR_MAP_SWIZZLE_128B);
    else
        mZ = mX;
    if (!ok) return RSVDGB_ERR_CUDA;

    GramParams p{};
    p.rows = rows;
    p.l = l;
    p.l_pad = l_pad;
    const int64_t nk_total = ceil_div(rows, kBK);
    const int64_t steps = ceil_div(nk_total, (int64_t)std::max(sm_count, 1));
    p.k_per_cta = steps * kBK;
    const int64_t grid = ceil_div(nk_total, steps);
    const size_t stage = (cross ? 4 : 2) * (size_t)kTile;
    p.stages = (int)std::min<int64_t>(kMaxStages, std::min<int64_t>(std::max<int64_t>(steps, 2), (192 * 1024) / stage));
    p.part = part;
    p.status = status;
    const size_t smem = p.stages * stage + 1024;
    auto kern = cross ? tc_gram_kernel<true> : tc_gram_kernel<false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return RSVDGB_ERR_CUDA;
    kern<<<(unsigned)grid, kThreads, smem, s>>>(mX, mZ, p);
    count_launches();
    if (cudaGetLastError() != cudaSuccess) return RSVDGB_ERR_CUDA;
    launch_reduce_splits(s, part, (int)grid, (int64_t)l_pad * l_pad, l, l, l_pad, G, l);
    return RSVDGB_OK;
}

}  // namespace rsvdgb
