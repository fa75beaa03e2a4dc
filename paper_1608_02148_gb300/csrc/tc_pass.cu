// Tensor-core (tcgen05 + TMA) passes over A with FP32-accurate products.
//
// One kernel serves both products of the method:
//   AX  (TRANS = false): Y = A X      -- sketch Y = A Omega (Eq. YAQ) and the
//                                        power step Y = A Q (Algorithm
//                                        sub_iterations step 4);
//   AtX (TRANS = true) : Z = A^T Y    -- power step A^T Q (step 3) and the
//                                        projection B = Q^T A = (A^T Q)^T
//                                        (Eq. BQA).
// The MMA is D[128 x N] += A_op[128 x K] * P[K x N] with N = l_pad:
//   * the 128 accumulator lanes are 128 rows of A (AX) or 128 columns of A
//     (AtX); each CTA keeps G such accumulators in tensor memory (TMEM);
//   * the panel P (Omega, Q_n or Q; column-major, i.e. K-major) is streamed by
//     TMA into shared memory, already split into hi and lo parts;
//   * A is streamed by TMA into shared memory once; sixteen "converter" warps
//     read each element once, split it into hi and lo parts and store both
//     into TMEM, where the MMA reads its A operand (tcgen05.mma ... [a_tmem]);
//     a ring of up to four converted stages in TMEM decouples the converters
//     from the tensor core.
// Two FP32-accurate forms:
//   * 3xTF32 (H = false): a_hi = a with the low 13 mantissa bits cleared
//     (exact TF32), a_lo = a - a_hi (exact in FP32, |a_lo| < 2^-10 |a|); the
//     panel split by round-to-nearest TF32 (hi, then lo of the remainder);
//     three kind::tf32 MMAs per K step of 8, a_hi p_hi + a_hi p_lo + a_lo p_hi.
//     Whether the tensor core rounds or truncates a_lo to TF32, and with the
//     dropped a_lo p_lo term, each product is within 2^-19 |a||p|.
//   * scaled FP16x3 (H = true): A is multiplied by 2^eA, which brings max|A|
//     (measured by the first pass) into [2^13, 2^14), and column j of the
//     panel by its own 2^ej; both are split into FP16 hi + lo, each part with
//     11 significant bits (A: hi = the scaled value truncated to 11 bits,
//     exact in FP16, lo = the remainder rounded, so a = hi + lo within
//     2^-21 |a|; the panel: round to nearest twice, within 2^-22), and
//     within 2^-24 of the scaled unit where the parts fall below FP16's
//     normal range; three kind::f16 MMAs per K step of 16, a_hi p_hi + a_hi
//     p_lo + a_lo p_hi, each product exact in FP32; the epilogue multiplies
//     column j by 2^-(eA + ej).  Each product is within 2^-19 |a||p| (the
//     dropped a_lo p_lo, at most 2^-20, and the two roundings of the lo
//     parts, 2^-21 each) plus the FP16 underflow term.  The same bound as
//     3xTF32 at half the tensor time
//     (K = 16 per FP16 MMA, 8 per TF32 MMA, same issue rate), and a 16-bit A
//     operand takes half the TMEM, so the converted-A ring is twice as deep.
//     BF16-stored A is exact in FP16 after the scaling, so only a p_hi +
//     a p_lo remain.
//   * the tensor core's FP32 accumulation drops low bits toward zero at each
//     step, so a long chain shrinks the sum by a relative bias that grows
//     with its length (about 1.7e-8 per MMA on sums of random sign).  Where
//     the scale of the result matters (the projection B = Q^T A, Grams, the
//     C-ABI products) the K range is cut into chunks of chunk_stages stages:
//     each chunk starts a fresh accumulator, the first chunk's result is
//     stored and the later ones are added in FP32 (round to nearest) with
//     reductions -- 16-byte ones into row-major split partials, which the
//     launch then sums, when the product has split partials and an output.
// Roles (640 threads): warp 0 issues the TMA loads of A, warp 18 those of the
// panel, warps 1 and 19 issue MMAs (one elected lane each; even and odd
// accumulator groups), warps 2..17 convert A and run the epilogue.  The
// converters form two groups of eight that take alternate stages, so two
// stages are converted at once (a group's turn is bounded by its barrier
// waits and TMEM stores, not by its arithmetic); in a group, two warps per
// TMEM lane quarter each take half of the stage's K columns.  All sixteen run
// the epilogue, each taking every fourth 16-column chunk of its lane quarter.  A tiles and
// panel tiles sit in separate shared-memory rings: an A tile is released as
// soon as it is converted, a panel tile when the MMAs that read it complete.
// Every mbarrier wait is bounded; on expiry the kernel records
// RSVDGB_ERR_TIMEOUT, stops issuing work, waits (bounded) for its copies and
// MMAs in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.cuh"
#include "ptx.cuh"

namespace rsvdgb {
namespace {
using namespace dev;

constexpr int kBK = 32;            // K elements per stage (one 128-byte swizzle row)
constexpr int kTileRows = 128;     // accumulator lanes
constexpr int kConvWarps = 16;     // converter / epilogue warps (four per TMEM lane quarter)
constexpr int kGroupWarps = 8;     // converter warps per group; the two groups take alternate stages
constexpr int kThreads = 128 + 32 * kConvWarps;  // + TMA(A), 2 x MMA, TMA(panel) warps
constexpr int kMmaWarp1 = 3 + kConvWarps;        // second MMA issuer (odd groups)
constexpr int kMaxAStages = 6;
constexpr int kMaxPStages = 6;
constexpr int kPanelStages = 3;    // panel ring depth wanted (fewer when shared memory is short)
constexpr int kMaxTmemStages = 4;  // converted-A ring in TMEM (as deep as the columns allow)

struct TcParams {
    int64_t m, n;          // stored A: row-major m x n
    int l_pad;             // MMA N (multiple of 16, <= 256)
    int64_t num_tiles;     // 128-wide tiles along the lane dimension
    int64_t k_total;       // extent of K (n for AX, m for AtX)
    int64_t k_per_split;   // AtX: K rows per split (multiple of kBK); AX: k_total
    int a_stages;          // shared-memory ring of A tiles (released by the converters)
    int p_stages;          // shared-memory ring of panel tiles (released by the MMAs)
    float* out;            // AX: Yt (column-major, ld_out); AtX: partial base
    float* out_hi;         // AX: TF32 hi part of Y (may be null)
    float* out_lo;         // AX: TF32 lo part of Y (may be null)
    int64_t ld_out;
    int out_rowmajor;      // direct output stored row-major: out[idx * ld_out + j], j < out_cols
    int out_vec4;          // row-major output 16-byte aligned (float4 stores)
    int out_cols;
    int64_t split_stride;  // AtX: floats between partials
    int chunk_stages;      // > 0: accumulate at most this many K stages in TMEM before adding to the output
    const float* aff_h;    // direct column-major output only: out = r_i (acc - u_i h_j)
    const float* aff_u;    //   (h null: no shift; u, r null: 1)
    const float* aff_r;
    int part_rm;           // partials row-major (part + split * lanes * l_pad + idx * l_pad + j): chunks
                           // after the first are added with 16-byte vector reductions
    int* status;
    double* fro2;          // if set: ||A||_F^2 is accumulated by the converters
    int tmem_stages;       // depth of the converted-A ring in TMEM (2..kMaxTmemStages)
    unsigned int* amax_out;       // SQ: bits of max|a| accumulated by the converters (atomicMax)
    const unsigned int* amax_in;  // H: bits of max|A|, which sets A's scale 2^eA
    const float* pinv;     // H: per panel column, the inverse 2^-ej of its scale (l_pad floats)
    // FP16 hi / lo copy of a direct column-major output (the panel of a later
    // FP16x3 pass), column j scaled by split_sc[j] (or split_sc_const)
    uint16_t* out_h16;
    uint16_t* out_l16;
    const float* split_sc;
    float split_sc_const;
};

// ----------------------------------------------------------------- the kernel
template <bool TRANS, int G, bool SQ, bool BF, bool ABF, bool H>
__global__ void __launch_bounds__(kThreads, 1)
    tc_pass_kernel(const __grid_constant__ CUtensorMap tmapA, const __grid_constant__ CUtensorMap tmapPhi,
                   const __grid_constant__ CUtensorMap tmapPlo, TcParams p)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte aligned base for the swizzled tiles
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);

    __shared__ uint64_t afull_bar[kMaxAStages], aempty_bar[kMaxAStages];
    __shared__ uint64_t pfull_bar[kMaxPStages], pempty_bar[kMaxPStages];
    const int TS = p.tmem_stages;
    __shared__ uint64_t conv_bar[kMaxTmemStages], tfree_bar[kMaxTmemStages];
    __shared__ uint64_t accf_bar, acce_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int SA = p.a_stages, SP = p.p_stages;
    const int l_pad = p.l_pad;
    const uint32_t a_tile_bytes = kTileRows * kBK * (ABF ? 2 : 4);  // 16 KB (8 KB for BF16 A)
    // panel tile: l_pad rows x kBK elements (TF32 hi + lo: 128 B rows each;
    // BF16: one 64 B row; FP16 hi + lo: 64 B rows each)
    const uint32_t p_tile_bytes = (uint32_t)l_pad * kBK * ((BF || H) ? 2 : 4);
    const uint32_t a_stage_bytes = G * a_tile_bytes;
    const uint32_t p_stage_bytes = (BF ? 1 : 2) * p_tile_bytes;
    // TMEM columns of one converted A tile: BF16 pairs; TF32 hi + lo; FP16
    // pairs hi + lo; or hi alone for BF16 A, which TF32 and (scaled) FP16
    // hold exactly (a_lo = 0)
    constexpr uint32_t kAcols = BF ? kBK / 2 : (H ? (ABF ? kBK / 2 : kBK) : (ABF ? kBK : 2 * kBK));
    uint8_t* a_ring = smem;
    uint8_t* p_ring = smem + (size_t)SA * a_stage_bytes;

    // ---- work of this CTA: a range of lane tiles and a K range
    int64_t tile_begin, tile_end, k_begin, k_end;
    if (!TRANS) {
        tile_begin = p.num_tiles * blockIdx.x / gridDim.x;
        tile_end = p.num_tiles * (blockIdx.x + 1) / gridDim.x;
        k_begin = (int64_t)blockIdx.y * p.k_per_split;
        k_end = min(p.k_total, k_begin + p.k_per_split);
    } else {
        // sets of G lane tiles; a grid narrower than the sets makes the CTAs
        // persistent over a range of them
        const int64_t units = (p.num_tiles + G - 1) / G;
        tile_begin = units * blockIdx.x / gridDim.x * G;
        tile_end = min(p.num_tiles, units * (blockIdx.x + 1) / gridDim.x * G);
        k_begin = (int64_t)blockIdx.y * p.k_per_split;
        k_end = min(p.k_total, k_begin + p.k_per_split);
    }
    const int64_t num_sets = (tile_end - tile_begin + G - 1) / G;
    const int64_t nk = (k_end > k_begin) ? (k_end - k_begin + kBK - 1) / kBK : 0;
    // K chunks of each set (one accumulator chain each)
    const int64_t chunk = (p.chunk_stages > 0 && p.chunk_stages < nk) ? p.chunk_stages : (nk > 0 ? nk : 1);
    const int64_t nch = (nk + chunk - 1) / chunk;

    // ---- TMEM columns: G accumulators of l_pad, then A buffers
    const uint32_t acc_cols = (uint32_t)G * l_pad;
    const uint32_t a_col0 = (acc_cols + 31) & ~31u;
    const uint32_t need = a_col0 + TS * G * kAcols;
    uint32_t tmem_cols = 32;
    while (tmem_cols < need) tmem_cols <<= 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SA; ++s) {
            mbar_init(&afull_bar[s], 1);
            mbar_init(&aempty_bar[s], kGroupWarps);
        }
        for (int s = 0; s < SP; ++s) {
            mbar_init(&pfull_bar[s], 1);
            mbar_init(&pempty_bar[s], 2);  // one commit per MMA issuer
        }
        for (int s = 0; s < TS; ++s) {
            mbar_init(&conv_bar[s], kGroupWarps);
            mbar_init(&tfree_bar[s], 2);
        }
        mbar_init(&accf_bar, 2);
        mbar_init(&acce_bar, kConvWarps);
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

    if (warp == 0 || warp == 2 + kConvWarps) {
        // =========================== TMA producers: A tiles (warp 0), panel tiles (last warp)
        const bool is_a = (warp == 0);
        if (lane == 0) {
            const int S = is_a ? SA : SP;
            uint64_t* fullb = is_a ? afull_bar : pfull_bar;
            uint64_t* emptyb = is_a ? aempty_bar : pempty_bar;
            int64_t it = 0;
            bool ok = true;
            for (int64_t set = 0; set < num_sets && ok; ++set) {
                const int64_t t0 = tile_begin + set * G;
                const int gv = (int)min((int64_t)G, tile_end - t0);
                for (int64_t c = 0; c < nk && ok; ++c, ++it) {
                    const int s = (int)(it % S);
                    const uint32_t ph = (uint32_t)((it / S) & 1);
                    if (!(ok = mbar_wait(&emptyb[s], ph ^ 1, &abort_flag, p.status))) break;
                    const int kc = (int)(k_begin + c * kBK);
                    if (is_a) {
                        uint8_t* st = a_ring + (size_t)s * a_stage_bytes;
                        mbar_expect_tx(&fullb[s], gv * a_tile_bytes);
                        for (int g = 0; g < gv; ++g) {
                            const int lane0 = (int)((t0 + g) * kTileRows);
                            if (!TRANS)
                                tma_load_2d(&tmapA, &fullb[s], st + g * a_tile_bytes, kc, lane0);  // {col k, row}
                            else
                                tma_load_2d(&tmapA, &fullb[s], st + g * a_tile_bytes, lane0, kc);  // {col, row k}
                        }
                    } else {
                        uint8_t* st = p_ring + (size_t)s * p_stage_bytes;
                        mbar_expect_tx(&fullb[s], p_stage_bytes);
                        tma_load_2d(&tmapPhi, &fullb[s], st, kc, 0);
                        if (!BF) tma_load_2d(&tmapPlo, &fullb[s], st + p_tile_bytes, kc, 0);
                    }
                }
            }
            if (!ok) {
                // drain: wait (bounded) for the copies already issued
                const long long t0 = clock64();
                for (int64_t j = (it > S ? it - S : 0); j < it; ++j) {
                    const int s = (int)(j % S);
                    const uint32_t ph = (uint32_t)((j / S) & 1);
                    while (!mbar_test(&fullb[s], ph) && clock64() - t0 < kSpinLimit) {
                    }
                }
            }
        }
    } else if (warp == 1 || warp == kMmaWarp1) {
        // =========================== MMA issuers: warp 1 even groups, the other odd groups
        const int gpar = (warp == 1) ? 0 : 1;
        if (lane == 0) {
            const uint32_t idesc = BF  ? bf16_idesc(kTileRows, l_pad)
                                   : H ? f16_idesc(kTileRows, l_pad)
                                       : tf32_idesc(kTileRows, l_pad);
            int64_t it = 0, item = 0;
            bool ok = true;
            for (int64_t set = 0; set < num_sets && ok; ++set) {
                const int64_t t0 = tile_begin + set * G;
                const int gv = (int)min((int64_t)G, tile_end - t0);
              for (int64_t ch = 0; ch < nch && ok; ++ch, ++item) {
                const int64_t c0 = ch * chunk, c1 = min(nk, c0 + chunk);
                // the accumulators are free once the previous item's epilogue read them
                if (!(ok = mbar_wait(&acce_bar, ((uint32_t)item & 1) ^ 1, &abort_flag, p.status))) break;
                tmem_fence_after();
                for (int64_t c = c0; c < c1; ++c, ++it) {
                    const int s = (int)(it % SP);
                    const uint32_t ph = (uint32_t)((it / SP) & 1);
                    const int ts = (int)(it % TS);
                    const uint32_t tph = (uint32_t)((it / TS) & 1);
                    if (!(ok = mbar_wait(&conv_bar[ts], tph, &abort_flag, p.status))) break;
                    if (!(ok = mbar_wait(&pfull_bar[s], ph, &abort_flag, p.status))) break;
                    tmem_fence_after();
                    const uint32_t phi = smem_u32(p_ring + (size_t)s * p_stage_bytes);
                    const uint32_t plo = phi + p_tile_bytes;
                    for (int g = gpar; g < gv; g += 2) {
                        const uint32_t d = tmem + (uint32_t)(g * l_pad);
                        const uint32_t ahi = tmem + a_col0 + (uint32_t)(ts * G + g) * kAcols;
                        const uint32_t alo = ahi + kBK;
                        if (BF) {
                            // one BF16 product per K step of 16 (8 TMEM columns, 32 bytes of panel row)
#pragma unroll
                            for (int kk = 0; kk < kBK / 16; ++kk) {
                                const uint32_t acc = (c > c0 || kk > 0) ? 1u : 0u;
                                mma_kf16_tmemA(d, ahi + kk * 8, sw64_desc(phi + kk * 32), idesc, acc);
                            }
                            continue;
                        }
                        if (H) {
                            // per K step of 16: a_hi p_hi + a_hi p_lo (+ a_lo p_hi); the
                            // hi pairs sit in the tile's first kBK / 2 TMEM columns, lo after
#pragma unroll
                            for (int kk = 0; kk < kBK / 16; ++kk) {
                                const uint32_t acc = (c > c0 || kk > 0) ? 1u : 0u;
                                const uint32_t ah = ahi + kk * 8;
                                mma_kf16_tmemA(d, ah, sw64_desc(phi + kk * 32), idesc, acc);
                                mma_kf16_tmemA(d, ah, sw64_desc(plo + kk * 32), idesc, 1u);
                                if (!ABF) mma_kf16_tmemA(d, ah + kBK / 2, sw64_desc(phi + kk * 32), idesc, 1u);
                            }
                            continue;
                        }
#pragma unroll
                        for (int kk = 0; kk < kBK / 8; ++kk) {
                            const uint64_t bhi = sw128_desc(phi + kk * 32);
                            const uint64_t blo = sw128_desc(plo + kk * 32);
                            const uint32_t acc = (c > c0 || kk > 0) ? 1u : 0u;
                            mma_tf32_tmemA(d, ahi + kk * 8, bhi, idesc, acc);
                            mma_tf32_tmemA(d, ahi + kk * 8, blo, idesc, 1u);
                            if (!ABF) mma_tf32_tmemA(d, alo + kk * 8, bhi, idesc, 1u);
                        }
                    }
                    mma_commit(&pempty_bar[s]);
                    mma_commit(&tfree_bar[ts]);
                }
                if (!ok) break;
                mma_commit(&accf_bar);
              }
            }
            if (!ok) {
                // wait (bounded) for the MMAs already issued before TMEM is freed
                __shared__ uint64_t drain_bar[2];
                mbar_init(&drain_bar[gpar], 1);
                asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
                mma_commit(&drain_bar[gpar]);
                const long long t0 = clock64();
                while (!mbar_test(&drain_bar[gpar], 0) && clock64() - t0 < kSpinLimit) {
                }
            }
        }
    } else {
        // =========================== converters + epilogue (warps 2..9)
        const int q = warp & 3;                 // TMEM lane quarter of this warp
        const int ew = (warp - 2) >> 2;         // which quarter of the 16-column output chunks
        const int cg = (warp - 2) >> 3;         // converter group: stages it with it % 2 == cg
        const int hk = ew & 1;                  // which half of a stage's K columns
        const int r = q * 32 + lane;            // lane (row of the tile) of this thread
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        constexpr int KH = kBK / 2;             // K columns converted by this warp
        float sq = 0.f;  // sum of squares of the A elements this thread converted
        float mx = 0.f;  // and their largest magnitude
        // scale 2^eA of A in the FP16x3 form (max|A| from the first pass)
        const float sA = H ? pow2_scale_below(__uint_as_float(*p.amax_in)) : 1.f;
        const float inv_sA = 1.f / sA;
        // Epilogue of one (tile set, K chunk) item: 16-column chunks alternate
        // between the two warps of a quarter; the first chunk stores, later
        // chunks add.  It runs after the first stage of the next item has been
        // converted, so the tensor core restarts as soon as TMEM is drained.
        auto epilogue = [&](int64_t e_item) -> bool {
                const int64_t e_ch = e_item % nch;
                const int64_t e_t0 = tile_begin + (e_item / nch) * G;
                const int e_gv = (int)min((int64_t)G, tile_end - e_t0);
                const bool e_first = (e_ch == 0), e_last = (e_ch == nch - 1);
                if (!mbar_wait_warp(&accf_bar, (uint32_t)e_item & 1, &abort_flag, p.status)) return false;
                tmem_fence_after();
                for (int g = 0; g < e_gv; ++g) {
                    const int64_t idx = (e_t0 + g) * kTileRows + r;  // row (AX) or column (AtX) of A
                    const int64_t lim = TRANS ? p.n : p.m;
                    // rank-one correction and row scale of an affine map (centred /
                    // scaled data): y = r_i (acc - u_i h_j)
                    const float au = (p.aff_u && idx < lim) ? p.aff_u[idx] : 1.f;
                    const float ar = (p.aff_r && idx < lim) ? p.aff_r[idx] : 1.f;
                    float* out = p.out + (int64_t)blockIdx.y * p.split_stride;
                    for (int j0 = 16 * ew; j0 < l_pad; j0 += 64) {
                        uint32_t v[16];
                        tmem_ld16(tmem + (uint32_t)(g * l_pad + j0) + lane_off, v);
                        tmem_wait_ld();
                        if (H) {
                            // undo the scales of A and of the panel columns (powers of two: exact)
#pragma unroll
                            for (int e = 0; e < 16; ++e)
                                v[e] = __float_as_uint(__uint_as_float(v[e]) * (inv_sA * p.pinv[j0 + e]));
                        }
                        if (idx < lim) {
                            if (p.out_rowmajor) {
                                // a row of the output per thread: 16-byte stores when aligned
                                float* orow = out + idx * p.ld_out + j0;
                                if (p.out_vec4 && j0 + 16 <= p.out_cols) {
#pragma unroll
                                    for (int e = 0; e < 4; ++e) {
                                        float4 y = make_float4(__uint_as_float(v[4 * e]), __uint_as_float(v[4 * e + 1]),
                                                               __uint_as_float(v[4 * e + 2]), __uint_as_float(v[4 * e + 3]));
                                        if (!e_first) {
                                            const float4 o4 = *(const float4*)(orow + 4 * e);
                                            y.x += o4.x;
                                            y.y += o4.y;
                                            y.z += o4.z;
                                            y.w += o4.w;
                                        }
                                        *(float4*)(orow + 4 * e) = y;
                                    }
                                } else {
#pragma unroll
                                    for (int e = 0; e < 16; ++e)
                                        if (j0 + e < p.out_cols)
                                            orow[e] = e_first ? __uint_as_float(v[e]) : orow[e] + __uint_as_float(v[e]);
                                }
                            } else if (p.part_rm) {
                                float* prow = out + idx * l_pad + j0;
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    const float4 y =
                                        make_float4(__uint_as_float(v[4 * e]), __uint_as_float(v[4 * e + 1]),
                                                    __uint_as_float(v[4 * e + 2]), __uint_as_float(v[4 * e + 3]));
                                    if (e_first)
                                        *(float4*)(prow + 4 * e) = y;
                                    else
                                        red_add_v4(prow + 4 * e, y);
                                }
                            } else {
#pragma unroll
                                for (int e = 0; e < 16; ++e) {
                                    const int64_t o = (int64_t)(j0 + e) * p.ld_out + idx;
                                    if (!e_first && !p.out_hi && !p.out_h16) {
                                        // later chunks: a reduction (round to nearest) that
                                        // returns nothing, so the warp does not wait on it;
                                        // each address has one writer, in program order
                                        atomicAdd(out + o, __uint_as_float(v[e]));
                                        continue;
                                    }
                                    float y = e_first ? __uint_as_float(v[e]) : out[o] + __uint_as_float(v[e]);
                                    if (p.aff_h) y = fmaf(-au, p.aff_h[j0 + e], y);
                                    if (p.aff_r) y *= ar;
                                    out[o] = y;
                                    if (p.out_hi && e_last) {
                                        const uint32_t h = tf32_rna(y);
                                        p.out_hi[o] = __uint_as_float(h);
                                        p.out_lo[o] = __uint_as_float(tf32_rna(y - __uint_as_float(h)));
                                    }
                                    if (p.out_h16 && e_last) {
                                        // scaled FP16 hi / lo (the panel of a later FP16x3 pass)
                                        const float sc = p.split_sc ? p.split_sc[j0 + e] : p.split_sc_const;
                                        uint32_t h, lw;
                                        split_f16_pair(y * sc, 0.f, h, lw);
                                        p.out_h16[o] = (uint16_t)(h & 0xFFFFu);
                                        p.out_l16[o] = (uint16_t)(lw & 0xFFFFu);
                                    }
                                }
                            }
                        }
                    }
                }
                tmem_fence_before();
                __syncwarp();
                tmem_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acce_bar);
                return true;
        };
        int64_t it = 0, item = 0;
        bool ok = true;
        for (int64_t set = 0; set < num_sets && ok; ++set) {
            const int64_t t0 = tile_begin + set * G;
            const int gv = (int)min((int64_t)G, tile_end - t0);
          for (int64_t ch = 0; ch < nch && ok; ++ch, ++item) {
            const int64_t c0 = ch * chunk, c1 = min(nk, c0 + chunk);
            for (int64_t c = c0; c < c1; ++c, ++it) {
                const int s = (int)(it % SA);
                const uint32_t ph = (uint32_t)((it / SA) & 1);
                const int ts = (int)(it % TS);
                const uint32_t tph = (uint32_t)((it / TS) & 1);
                if ((int)(it & 1) != cg) {
                    // the other group's stage; the epilogue is shared by both groups
                    if (c == c0 && item > 0 && !(ok = epilogue(item - 1))) break;
                    continue;
                }
                if (!(ok = mbar_wait_warp(&afull_bar[s], ph, &abort_flag, p.status))) break;
                if (!(ok = mbar_wait_warp(&tfree_bar[ts], tph ^ 1, &abort_flag, p.status))) break;
                tmem_fence_after();
                const uint8_t* st = a_ring + (size_t)s * a_stage_bytes;
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    if (g >= gv) continue;
                    const float* tile = (const float*)(st + g * a_tile_bytes);
                    float a8[KH];  // this warp's KH = 16 K values of lane r in tile g
                    if (ABF) {
                        // BF16 A, exact in FP32 (BF16 is a prefix of FP32 and of TF32)
                        const uint16_t* tb = (const uint16_t*)tile;
                        if (!TRANS) {
                            // row r of a 128 x 32 tile, 64-byte rows, 64-byte swizzle:
                            // 16-byte chunk c of row r sits at chunk (c ^ ((r >> 1) & 3));
                            // this warp takes chunks 2hk, 2hk+1
#pragma unroll
                            for (int cc = 0; cc < 2; ++cc) {
                                const int ch = 2 * hk + cc;
                                const uint4 v = *(const uint4*)((const uint8_t*)tile + r * 64 +
                                                                ((ch ^ ((r >> 1) & 3)) << 4));
                                const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    a8[cc * 8 + 2 * e] = __uint_as_float(w4[e] << 16);
                                    a8[cc * 8 + 2 * e + 1] = __uint_as_float(w4[e] & 0xFFFF0000u);
                                }
                            }
                        } else {
                            // column r of a 32 x 128 tile (rows of 256 bytes, no swizzle)
#pragma unroll
                            for (int kk = 0; kk < KH; ++kk)
                                a8[kk] = __uint_as_float((uint32_t)tb[(KH * hk + kk) * kTileRows + r] << 16);
                        }
                    } else if (!TRANS) {
                        // row r of a 128 x 32 tile, 128-byte swizzle: 16-byte chunk c of
                        // row r sits at chunk (c ^ (r & 7)); this warp takes chunks 4hk..4hk+3
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) {
                            const int ch = 4 * hk + cc;
                            const float4 v =
                                *(const float4*)((const uint8_t*)tile + r * 128 + ((ch ^ (r & 7)) << 4));
                            a8[cc * 4 + 0] = v.x;
                            a8[cc * 4 + 1] = v.y;
                            a8[cc * 4 + 2] = v.z;
                            a8[cc * 4 + 3] = v.w;
                        }
                    } else {
                        // column r of a 32 x 128 tile (rows of 512 bytes, no swizzle)
#pragma unroll
                        for (int kk = 0; kk < KH; ++kk) a8[kk] = tile[(KH * hk + kk) * kTileRows + r];
                    }
                    if (SQ) {
#pragma unroll
                        for (int kk = 0; kk < KH; ++kk) {
                            sq = fmaf(a8[kk], a8[kk], sq);
                            mx = fmaxf(mx, fabsf(a8[kk]));
                        }
                    }
                    if (g == gv - 1) {
                        // the stage is in registers: hand its shared-memory slot back to TMA
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&aempty_bar[s]);
                    }
                    uint32_t hi[KH], lo[KH];
                    if (BF) {
                        // BF16 pairs (round to nearest; exact for BF16 A)
#pragma unroll
                        for (int e = 0; e < KH / 2; ++e) hi[e] = pack_bf16(a8[2 * e], a8[2 * e + 1]);
                    } else if (H) {
                        // scaled FP16 pairs.  hi = the scaled value with its 13 low
                        // mantissa bits cleared: 11 significant bits, exact in FP16
                        // (in its normal range); lo = the exact remainder rounded to
                        // FP16, so a = hi + lo within 2^-21 |a| (BF16 A: lo = 0)
#pragma unroll
                        for (int e = 0; e < KH / 2; ++e) {
                            const float2 x = __fmul2_rn(make_float2(a8[2 * e], a8[2 * e + 1]), make_float2(sA, sA));
                            if (ABF) {
                                hi[e] = pack_f16(x.x, x.y);
                            } else {
                                const float2 h = make_float2(__uint_as_float(__float_as_uint(x.x) & 0xFFFFE000u),
                                                             __uint_as_float(__float_as_uint(x.y) & 0xFFFFE000u));
                                const float2 w = __fadd2_rn(x, make_float2(-h.x, -h.y));
                                hi[e] = pack_f16(h.x, h.y);
                                lo[e] = pack_f16(w.x, w.y);
                            }
                        }
                    } else if (ABF) {
#pragma unroll
                        for (int kk = 0; kk < KH; ++kk) hi[kk] = __float_as_uint(a8[kk]);
                    } else {
                        // TF32 hi = a with the low 13 mantissa bits cleared, lo = the rest
#pragma unroll
                        for (int kk = 0; kk < KH; ++kk) {
                            const uint32_t h = __float_as_uint(a8[kk]) & 0xFFFFE000u;
                            hi[kk] = h;
                            lo[kk] = __float_as_uint(a8[kk] - __uint_as_float(h));
                        }
                    }
                    const uint32_t base = tmem + a_col0 + (uint32_t)(ts * G + g) * kAcols + lane_off;
                    if (BF || H) {
                        // 16-bit pairs: this warp's 16 K values in 8 columns (hi; then lo
                        // kBK / 2 columns further on)
                        uint32_t pk[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) pk[e] = hi[e];
                        tmem_st8(base + (uint32_t)(8 * hk), pk);
                        if (H && !ABF) {
#pragma unroll
                            for (int e = 0; e < 8; ++e) pk[e] = lo[e];
                            tmem_st8(base + (uint32_t)(kBK / 2 + 8 * hk), pk);
                        }
                        continue;
                    }
                    tmem_st16(base + (uint32_t)(KH * hk), hi);
                    if (!ABF) tmem_st16(base + (uint32_t)(kBK + KH * hk), lo);
                }
                tmem_wait_st();
                tmem_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&conv_bar[ts]);
                // the previous item's epilogue, once this item's first stage is
                // converted (the tensor core restarts as soon as TMEM is read)
                if (c == c0 && item > 0 && !(ok = epilogue(item - 1))) break;
            }
            if (!ok) break;
          }
        }
        if (ok && item > 0) ok = epilogue(item - 1);
        if (SQ && p.fro2) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
            if (lane == 0) atomicAdd(p.fro2, (double)sq);
        }
        if (SQ && p.amax_out) {
            // bits of a non-negative float order like the float
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) atomicMax(p.amax_out, __float_as_uint(mx));
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

// Sum of row-major split partials part[s][idx][j] (rows x l_pad each) into the
// column-major output out[j * ld_out + idx], splits added in order (FP32).
// Block: kRedRows rows, staged through shared memory so that the stores of a
// column are contiguous.
constexpr int kRedRows = 16;
__global__ void __launch_bounds__(256) reduce_rm_kernel(const float* __restrict__ part, int splits, int64_t rows,
                                                        int l_pad, float* __restrict__ out, int64_t ld_out)
{
    extern __shared__ float tile[];  // kRedRows x (l_pad + 1)
    const int64_t r0 = (int64_t)blockIdx.x * kRedRows;
    const int nr = (int)min((int64_t)kRedRows, rows - r0);
    const int64_t stride = rows * l_pad;
    for (int e = threadIdx.x; e < nr * l_pad; e += blockDim.x) {
        const float* src = part + r0 * l_pad + e;
        float acc = 0.f;
        for (int s = 0; s < splits; ++s) acc += src[(int64_t)s * stride];
        tile[(e / l_pad) * (l_pad + 1) + e % l_pad] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kRedRows * l_pad; e += blockDim.x) {
        const int j = e / kRedRows, rr = e % kRedRows;
        if (rr < nr) out[(int64_t)j * ld_out + r0 + rr] = tile[rr * (l_pad + 1) + j];
    }
}

// ----------------------------------------------------------------- host side
template <bool TRANS, int G, bool BF, bool ABF, bool H>
int launch_typed(cudaStream_t s, const CUtensorMap& mA, const CUtensorMap& mhi, const CUtensorMap& mlo,
                 TcParams p, dim3 grid, size_t smem)
{
    // the statistics of A (||A||_F^2, max|A|) are taken by the first pass, never an FP16x3 one
    const bool sq = !H && (p.fro2 || p.amax_out);
    auto kern = sq ? tc_pass_kernel<TRANS, G, !H, BF, ABF, H> : tc_pass_kernel<TRANS, G, false, BF, ABF, H>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return RSVDGB_ERR_CUDA;
    kern<<<grid, kThreads, smem, s>>>(mA, mhi, mlo, p);
    count_launches();
    return cudaGetLastError() == cudaSuccess ? RSVDGB_OK : RSVDGB_ERR_CUDA;
}

template <bool TRANS, bool BF, bool ABF, bool H>
int launch_g(int G, cudaStream_t s, const CUtensorMap& mA, const CUtensorMap& mhi, const CUtensorMap& mlo,
             const TcParams& p, dim3 grid, size_t smem)
{
    switch (G) {
        case 1: return launch_typed<TRANS, 1, BF, ABF, H>(s, mA, mhi, mlo, p, grid, smem);
        case 2: return launch_typed<TRANS, 2, BF, ABF, H>(s, mA, mhi, mlo, p, grid, smem);
        case 3: return launch_typed<TRANS, 3, BF, ABF, H>(s, mA, mhi, mlo, p, grid, smem);
        default: return RSVDGB_ERR_UNSUPPORTED;
    }
}

template <bool TRANS, bool ABF>
int launch_prec(int G, bool bf, bool h, cudaStream_t s, const CUtensorMap& mA, const CUtensorMap& mhi,
                const CUtensorMap& mlo, const TcParams& p, dim3 grid, size_t smem)
{
    if (bf) return launch_g<TRANS, true, ABF, false>(G, s, mA, mhi, mlo, p, grid, smem);
    if (h) return launch_g<TRANS, false, ABF, true>(G, s, mA, mhi, mlo, p, grid, smem);
    return launch_g<TRANS, false, ABF, false>(G, s, mA, mhi, mlo, p, grid, smem);
}

// TMEM plan: G accumulators of l_pad columns (32-aligned), then a ring of TS
// stages x G converted A tiles, within the SM's 512 columns.  The most
// accumulator groups that still leave a ring of two, then the deepest ring
// (up to four) that fits.
void tmem_plan(int l_pad, bool bf, bool abf, bool h, int* G_out, int* TS_out)
{
    const int acols = bf ? kBK / 2 : (h ? (abf ? kBK / 2 : kBK) : (abf ? kBK : 2 * kBK));
    int g = 3, ts = 0;
    for (; g >= 1; --g) {
        const int acc = (g * l_pad + 31) / 32 * 32;
        ts = std::min(kMaxTmemStages, (512 - acc) / (g * acols));
        if (ts >= 2) break;
    }
    *G_out = std::max(g, 1);
    *TS_out = std::max(ts, 2);
}

int groups_for(int l_pad, bool bf, bool abf = false, bool h = false)
{
    int G, TS;
    tmem_plan(l_pad, bf, abf, h, &G, &TS);
    return G;
}

}  // namespace

bool tc_pass_supported(int64_t m, int64_t n, int64_t lda, int l_pad, const void* A, int a_bf16)
{
    if (l_pad < 16 || l_pad > 256 || (l_pad % 16)) return false;
    if ((lda * (a_bf16 ? 2 : 4)) % 16 || ((uintptr_t)A % 16)) return false;
    if (m > 0x7fffffff || n > 0x7fffffff) return false;
    return get_encoder() != nullptr;
}

int launch_tc_gemm(cudaStream_t s, int sm_count, bool trans, const float* A, int64_t m, int64_t n, int64_t lda,
                   const float* Phi, const float* Plo, int64_t ldp, int l_pad, float* out, float* out_hi,
                   float* out_lo, int64_t ld_out, float* partial, int64_t want_splits, int64_t* splits_out,
                   int* status, double* fro2, int out_rowmajor, int out_cols, int bf16_panel, int a_bf16,
                   int chunk_stages, const float* aff_h, const float* aff_u, const float* aff_r, const TcExtra* x)
{
    static const TcExtra none{};
    if (!x) x = &none;
    const bool bf = bf16_panel != 0;
    const bool abf = a_bf16 != 0;
    const bool h = x->h16 != 0;
    if (h && (bf || !x->amax_in || !x->pinv)) return RSVDGB_ERR_INVALID_ARG;
    int G, TS;
    tmem_plan(l_pad, bf, abf, h, &G, &TS);
    const size_t a_stage = (size_t)G * kTileRows * kBK * (abf ? 2 : 4);
    // panel stage: TF32 hi + lo (4-byte elements), BF16 alone, FP16 hi + lo
    const size_t p_stage = (bf ? 2 : (h ? 4 : 8)) * (size_t)l_pad * kBK;
    const size_t budget = 224 * 1024;  // dynamic shared memory, 1 KB kept for alignment
    int sp = kPanelStages;
    while (sp > 2 && sp * p_stage + 2 * a_stage > budget) --sp;
    int sa = (int)std::min<size_t>(kMaxAStages, (budget - sp * p_stage) / a_stage);
    if (sa < 2) return RSVDGB_ERR_UNSUPPORTED;
    const size_t smem = sa * a_stage + sp * p_stage + 1024;

    CUtensorMap mA, mhi, mlo;
    const int64_t k_total = trans ? m : n;
    bool ok;
    if (abf) {
        // BF16 A: 64-byte rows of 32 K values (A side) or 256-byte rows (A^T side)
        if (!trans)
            ok = encode_2d(&mA, A, n, m, lda * 2, kBK, kTileRows, CU_TENSOR_MAP_SWIZZLE_64B,
                           CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
        else
            ok = encode_2d(&mA, A, n, m, lda * 2, kTileRows, kBK, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    } else if (!trans)
        ok = encode_2d(&mA, A, n, m, lda * 4, kBK, kTileRows, CU_TENSOR_MAP_SWIZZLE_128B);
    else
        ok = encode_2d(&mA, A, n, m, lda * 4, kTileRows, kBK, CU_TENSOR_MAP_SWIZZLE_NONE);
    if (bf) {
        ok = ok && encode_2d(&mhi, Phi, k_total, l_pad, ldp * 2, kBK, l_pad, CU_TENSOR_MAP_SWIZZLE_64B,
                             CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
        mlo = mhi;
    } else if (h) {
        // FP16 hi / lo panels: 64-byte rows of 32 K values
        ok = ok && encode_2d(&mhi, Phi, k_total, l_pad, ldp * 2, kBK, l_pad, CU_TENSOR_MAP_SWIZZLE_64B,
                             CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
        ok = ok && encode_2d(&mlo, Plo, k_total, l_pad, ldp * 2, kBK, l_pad, CU_TENSOR_MAP_SWIZZLE_64B,
                             CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
    } else {
        ok = ok && encode_2d(&mhi, Phi, k_total, l_pad, ldp * 4, kBK, l_pad, CU_TENSOR_MAP_SWIZZLE_128B);
        ok = ok && encode_2d(&mlo, Plo, k_total, l_pad, ldp * 4, kBK, l_pad, CU_TENSOR_MAP_SWIZZLE_128B);
    }
    if (!ok) return RSVDGB_ERR_CUDA;

    TcParams p{};
    p.m = m;
    p.n = n;
    p.l_pad = l_pad;
    p.k_total = k_total;
    p.a_stages = sa;
    p.p_stages = sp;
    p.tmem_stages = TS;
    p.status = status;
    p.fro2 = fro2;
    p.amax_out = x->amax_out;
    p.amax_in = x->amax_in;
    p.pinv = x->pinv;
    p.ld_out = ld_out;
    // each chunk boundary stalls the tensor core while the accumulators are
    // read out, so chunks are at least 16 stages (512 K elements)
    p.chunk_stages = chunk_stages > 0 ? std::max(chunk_stages, 16) : 0;
    p.num_tiles = ceil_div(trans ? n : m, kTileRows);
    // K splits: fill the GPU when the lane tiles alone do not
    const int64_t units = trans ? ceil_div(p.num_tiles, G) : p.num_tiles;
    int64_t splits = want_splits;
    if (splits <= 0) {
        splits = std::max<int64_t>(1, (int64_t)sm_count / std::max<int64_t>(units, 1));
        splits = std::min<int64_t>(splits, std::max<int64_t>(1, k_total / (4 * kBK)));
    }
    p.k_per_split = round_up(ceil_div(k_total, splits), kBK);
    splits = ceil_div(k_total, p.k_per_split);
    const bool direct = (splits == 1) && out != nullptr;
    if (!direct && !partial) return RSVDGB_ERR_INVALID_ARG;
    p.out = direct ? out : partial;
    p.out_hi = direct ? out_hi : nullptr;
    p.out_lo = direct ? out_lo : nullptr;
    p.out_h16 = direct ? x->out_h16 : nullptr;
    p.out_l16 = direct ? x->out_l16 : nullptr;
    p.split_sc = x->split_sc;
    p.split_sc_const = x->split_sc_const;
    if (x->out_h16 && (!direct || out_rowmajor || !x->out_l16 || (!x->split_sc && !(x->split_sc_const > 0.f))))
        return RSVDGB_ERR_INVALID_ARG;
    p.split_stride = direct ? 0 : (int64_t)l_pad * ld_out;
    // chunked split products with an output: row-major partials, vector
    // reductions, and the split sum done here
    const int64_t lanes = trans ? n : m;
    p.part_rm = (!direct && p.chunk_stages > 0 && out != nullptr && !out_rowmajor) ? 1 : 0;
    if (p.part_rm) p.split_stride = lanes * l_pad;
    p.out_rowmajor = direct ? out_rowmajor : 0;
    p.out_cols = out_cols > 0 ? out_cols : l_pad;
    p.out_vec4 = (p.out_rowmajor && ((uintptr_t)p.out % 16) == 0 && (ld_out % 4) == 0) ? 1 : 0;
    if (out_rowmajor && !direct) return RSVDGB_ERR_INVALID_ARG;
    // the affine epilogue needs the whole sum in one place: direct, unchunked, column-major
    if ((aff_h || aff_r) && (!direct || p.chunk_stages > 0 || out_rowmajor)) return RSVDGB_ERR_UNSUPPORTED;
    p.aff_h = aff_h;
    p.aff_u = aff_u;
    p.aff_r = aff_r;
    dim3 grid;
    if (!trans)
        grid = dim3((unsigned)std::min<int64_t>(std::max<int64_t>(sm_count / splits, 1), p.num_tiles),
                    (unsigned)splits);
    else if (direct)
        grid = dim3((unsigned)std::min<int64_t>(units, sm_count), 1);  // persistent over the sets
    else
        grid = dim3((unsigned)units, (unsigned)splits);
    if (splits_out) *splits_out = (direct || p.part_rm) ? 0 : splits;
    int rc;
    if (trans)
        rc = abf ? launch_prec<true, true>(G, bf, h, s, mA, mhi, mlo, p, grid, smem)
                 : launch_prec<true, false>(G, bf, h, s, mA, mhi, mlo, p, grid, smem);
    else
        rc = abf ? launch_prec<false, true>(G, bf, h, s, mA, mhi, mlo, p, grid, smem)
                 : launch_prec<false, false>(G, bf, h, s, mA, mhi, mlo, p, grid, smem);
    if (rc != RSVDGB_OK || !p.part_rm) return rc;
    const size_t red_smem = kRedRows * (size_t)(l_pad + 1) * sizeof(float);
    reduce_rm_kernel<<<(unsigned)ceil_div(lanes, kRedRows), 256, red_smem, s>>>(partial, (int)splits, lanes, l_pad,
                                                                                out, ld_out);
    count_launches();
    return cudaGetLastError() == cudaSuccess ? RSVDGB_OK : RSVDGB_ERR_CUDA;
}


int64_t tc_pass_max_splits(int64_t m, int64_t n, int l_pad, int sm_count)
{
    // automatic split count of an A^T X launch on an m x n matrix
    int G = 1;
    for (int mode = 0; mode < 8; ++mode) {
        const bool bf = mode & 1, abf = mode & 2, h = mode & 4;
        if (!(bf && h)) G = std::max(G, groups_for(l_pad, bf, abf, h));
    }
    const int64_t units = ceil_div(ceil_div(n, kTileRows), G);
    int64_t splits = std::max<int64_t>(1, (int64_t)sm_count / units);
    splits = std::min<int64_t>(splits, std::max<int64_t>(1, m / (4 * kBK)));
    const int64_t kps = round_up(ceil_div(m, splits), kBK);
    return ceil_div(m, kps);
}

int64_t tc_split_count(int64_t k_total, int64_t units, int sm_count)
{
    int64_t splits = std::max<int64_t>(1, (int64_t)sm_count / std::max<int64_t>(units, 1));
    splits = std::min<int64_t>(splits, std::max<int64_t>(1, k_total / (4 * kBK)));
    const int64_t kps = round_up(ceil_div(k_total, splits), kBK);
    return ceil_div(k_total, kps);
}

}  // namespace rsvdgb
