// Tensor-core (tcgen05 + TMA) passes over A with FP32-accurate 3xTF32 products.
//
// One kernel serves both products of the method:
//   AX  (TRANS = false): Y = A X      -- sketch Y = A Omega (Eq. YAQ) and the
//                                        power step Y = A Q (Algorithm
//                                        sub_iterations step 4);
//   AtX (TRANS = true) : Z = A^T Y    -- power step A^T Q (step 3) and the
//                                        projection B = Q^T A = (A^T Q)^T
//                                        (Eq. BQA).
// The MMA is D[128 x N] += A_op[128 x 8] * P[8 x N] with N = l_pad:
//   * the 128 accumulator lanes are 128 rows of A (AX) or 128 columns of A
//     (AtX); each CTA keeps G such accumulators in tensor memory (TMEM);
//   * the panel P (Omega, Q_n or Y; column-major, i.e. K-major) is streamed by
//     TMA into shared memory, already split into TF32 hi and lo parts;
//   * A is streamed by TMA into shared memory once; four "converter" warps read
//     each element once, split it a = a_hi + a_lo (a_hi = TF32 round-to-
//     nearest of a, a_lo = TF32 of the remainder) and store both into TMEM,
//     where the MMA reads its A operand (tcgen05.mma ... [a_tmem]);
//   * three MMAs per K step, a_hi p_hi + a_hi p_lo + a_lo p_hi, accumulate in
//     FP32.  a_hi is a with the low 13 mantissa bits cleared (exact TF32) and
//     a_lo = a - a_hi (exact in FP32, |a_lo| < 2^-10 |a|); whether the tensor
//     core rounds or truncates a_lo to TF32, and with the dropped a_lo p_lo
//     term, each product is within 2^-19 |a||p| (p_hi, p_lo are split by
//     round-to-nearest beforehand);
//   * the tensor core's FP32 accumulation drops low bits toward zero at each
//     step, so a long chain shrinks the sum by a relative bias that grows
//     with its length (about 1.7e-8 per MMA on sums of random sign).  Where
//     the scale of the result matters (the projection B = Q^T A, Grams, the
//     C-ABI products) the K range is cut into chunks of chunk_stages stages:
//     each chunk starts a fresh accumulator, the first chunk's result is
//     stored and the later ones are added in FP32 (round to nearest) with
//     reductions -- 16-byte ones into row-major split partials, which the
//     launch then sums, when the product has split partials and an output.
// Roles (352 threads): warp 0 issues the TMA loads of A, warp 10 those of the
// panel, warp 1 allocates TMEM and issues MMAs (one elected lane), warps 2..9
// convert A and run the epilogue (two warps per TMEM lane quarter, each taking
// half of the K columns).  A tiles and panel tiles sit in separate shared-
// memory rings: an A tile is released as soon as it is converted, a panel
// tile when the MMAs that read it complete.  Every
// mbarrier wait is bounded; on expiry the kernel records RSVDGB_ERR_TIMEOUT,
// stops issuing work, waits (bounded) for its copies and MMAs in flight, frees
// its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.cuh"
#include "ptx.cuh"

namespace rsvdgb {
namespace {
using namespace dev;

constexpr int kBK = 32;            // K elements per stage (one 128-byte swizzle row)
constexpr int kTileRows = 128;     // accumulator lanes
constexpr int kConvWarps = 8;      // converter / epilogue warps (two per TMEM lane quarter)
constexpr int kThreads = 128 + 32 * kConvWarps;  // + TMA(A), 2 x MMA, TMA(panel) warps
constexpr int kMmaWarp1 = 3 + kConvWarps;        // second MMA issuer (odd groups)
constexpr int kMaxAStages = 6;
constexpr int kMaxPStages = 6;
constexpr int kPanelStages = 3;    // panel ring depth wanted (fewer when shared memory is short)
constexpr int kTmemStages = 2;     // A-operand buffers in TMEM

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
};

// ----------------------------------------------------------------- the kernel
template <bool TRANS, int G, bool SQ, bool BF, bool ABF>
__global__ void __launch_bounds__(kThreads, 1)
    tc_pass_kernel(const __grid_constant__ CUtensorMap tmapA, const __grid_constant__ CUtensorMap tmapPhi,
                   const __grid_constant__ CUtensorMap tmapPlo, TcParams p)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte aligned base for the swizzled tiles
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);

    __shared__ uint64_t afull_bar[kMaxAStages], aempty_bar[kMaxAStages];
    __shared__ uint64_t pfull_bar[kMaxPStages], pempty_bar[kMaxPStages];
    constexpr int TS = kTmemStages;
    __shared__ uint64_t conv_bar[TS], tfree_bar[TS];
    __shared__ uint64_t accf_bar, acce_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int SA = p.a_stages, SP = p.p_stages;
    const int l_pad = p.l_pad;
    const uint32_t a_tile_bytes = kTileRows * kBK * (ABF ? 2 : 4);  // 16 KB (8 KB for BF16 A)
    // panel tile: l_pad rows x kBK elements (TF32 hi + lo: 128 B rows each; BF16: one 64 B row)
    const uint32_t p_tile_bytes = (uint32_t)l_pad * kBK * (BF ? 2 : 4);
    const uint32_t a_stage_bytes = G * a_tile_bytes;
    const uint32_t p_stage_bytes = (BF ? 1 : 2) * p_tile_bytes;
    // TMEM columns of one converted A tile: BF16 pairs; TF32 hi + lo; or hi
    // alone for BF16 A, which TF32 holds exactly (a_lo = 0)
    constexpr uint32_t kAcols = BF ? kBK / 2 : (ABF ? kBK : 2 * kBK);
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
            mbar_init(&aempty_bar[s], kConvWarps);
        }
        for (int s = 0; s < SP; ++s) {
            mbar_init(&pfull_bar[s], 1);
            mbar_init(&pempty_bar[s], 2);  // one commit per MMA issuer
        }
        for (int s = 0; s < TS; ++s) {
            mbar_init(&conv_bar[s], kConvWarps);
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
            const uint32_t idesc = BF ? bf16_idesc(kTileRows, l_pad) : tf32_idesc(kTileRows, l_pad);
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
                                mma_bf16_tmemA(d, ahi + kk * 8, sw64_desc(phi + kk * 32), idesc, acc);
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
        const int hk = (warp - 2) >> 2;         // which half of the K columns / output chunks
        const int r = q * 32 + lane;            // lane (row of the tile) of this thread
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        constexpr int KH = kBK / 2;             // K columns converted by this warp
        float sq = 0.f;  // sum of squares of the A elements this thread converted
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
                    for (int j0 = 16 * hk; j0 < l_pad; j0 += 32) {
                        uint32_t v[16];
                        tmem_ld16(tmem + (uint32_t)(g * l_pad + j0) + lane_off, v);
                        tmem_wait_ld();
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
                                    if (!e_first && !p.out_hi) {
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
                if (!(ok = mbar_wait_warp(&afull_bar[s], ph, &abort_flag, p.status))) break;
                if (!(ok = mbar_wait_warp(&tfree_bar[ts], tph ^ 1, &abort_flag, p.status))) break;
                tmem_fence_after();
                const uint8_t* st = a_ring + (size_t)s * a_stage_bytes;
                uint32_t hi[G][kBK / 2], lo[G][kBK / 2];
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    if (g >= gv) continue;
                    const float* tile = (const float*)(st + g * a_tile_bytes);
                    if (ABF) {
                        // BF16 A: this warp's 16 K values as FP32 (exact: BF16 is a
                        // prefix of FP32 and of TF32)
                        float a16[KH];
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
                                    a16[cc * 8 + 2 * e] = __uint_as_float(w4[e] << 16);
                                    a16[cc * 8 + 2 * e + 1] = __uint_as_float(w4[e] & 0xFFFF0000u);
                                }
                            }
                        } else {
                            // column r of a 32 x 128 tile (rows of 256 bytes, no swizzle)
#pragma unroll
                            for (int kk = 0; kk < KH; ++kk)
                                a16[kk] = __uint_as_float((uint32_t)tb[(KH * hk + kk) * kTileRows + r] << 16);
                        }
                        if (BF) {
#pragma unroll
                            for (int e = 0; e < KH / 2; ++e) {
                                if (SQ) sq = fmaf(a16[2 * e], a16[2 * e], fmaf(a16[2 * e + 1], a16[2 * e + 1], sq));
                                hi[g][e] = pack_bf16(a16[2 * e], a16[2 * e + 1]);  // exact
                            }
                        } else {
#pragma unroll
                            for (int kk = 0; kk < KH; ++kk) {
                                if (SQ) sq = fmaf(a16[kk], a16[kk], sq);
                                hi[g][kk] = __float_as_uint(a16[kk]);
                            }
                        }
                        continue;
                    }
                    if (BF) {
                        // BF16 (round to nearest) of this warp's 16 K values, packed in pairs
                        float a16[KH];
                        if (!TRANS) {
#pragma unroll
                            for (int cc = 0; cc < 4; ++cc) {
                                const int ch = 4 * hk + cc;
                                const float4 v =
                                    *(const float4*)((const uint8_t*)tile + r * 128 + ((ch ^ (r & 7)) << 4));
                                a16[cc * 4 + 0] = v.x;
                                a16[cc * 4 + 1] = v.y;
                                a16[cc * 4 + 2] = v.z;
                                a16[cc * 4 + 3] = v.w;
                            }
                        } else {
#pragma unroll
                            for (int kk = 0; kk < KH; ++kk) a16[kk] = tile[(KH * hk + kk) * kTileRows + r];
                        }
#pragma unroll
                        for (int e = 0; e < KH / 2; ++e) {
                            if (SQ) sq = fmaf(a16[2 * e], a16[2 * e], fmaf(a16[2 * e + 1], a16[2 * e + 1], sq));
                            hi[g][e] = pack_bf16(a16[2 * e], a16[2 * e + 1]);
                        }
                        continue;
                    }
                    if (!TRANS) {
                        // row r of a 128 x 32 tile, 128-byte swizzle: 16-byte chunk c of
                        // row r sits at chunk (c ^ (r & 7)); this warp takes chunks 4hk..4hk+3
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) {
                            const int ch = 4 * hk + cc;
                            const float4 v =
                                *(const float4*)((const uint8_t*)tile + r * 128 + ((ch ^ (r & 7)) << 4));
                            const float a4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                if (SQ) sq = fmaf(a4[e], a4[e], sq);
                                const uint32_t h = __float_as_uint(a4[e]) & 0xFFFFE000u;
                                hi[g][cc * 4 + e] = h;
                                lo[g][cc * 4 + e] = __float_as_uint(a4[e] - __uint_as_float(h));
                            }
                        }
                    } else {
                        // column r of a 32 x 128 tile (rows of 512 bytes, no swizzle)
#pragma unroll
                        for (int kk = 0; kk < KH; ++kk) {
                            const float a = tile[(KH * hk + kk) * kTileRows + r];
                            if (SQ) sq = fmaf(a, a, sq);
                            const uint32_t h = __float_as_uint(a) & 0xFFFFE000u;
                            hi[g][kk] = h;
                            lo[g][kk] = __float_as_uint(a - __uint_as_float(h));
                        }
                    }
                }
                // the A tile is in registers: hand its shared-memory slot back to TMA
                __syncwarp();
                if (lane == 0) mbar_arrive(&aempty_bar[s]);
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    if (g >= gv) continue;
                    if (BF) {
                        const uint32_t col = tmem + a_col0 + (uint32_t)(ts * G + g) * kAcols + (uint32_t)(8 * hk);
                        uint32_t pk[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) pk[e] = hi[g][e];
                        tmem_st8(col + lane_off, pk);
                        continue;
                    }
                    const uint32_t col = tmem + a_col0 + (uint32_t)(ts * G + g) * kAcols + (uint32_t)(KH * hk);
                    tmem_st16(col + lane_off, hi[g]);
                    if (!ABF) tmem_st16(col + kBK + lane_off, lo[g]);
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
template <bool TRANS, int G, bool BF, bool ABF>
int launch_typed(cudaStream_t s, const CUtensorMap& mA, const CUtensorMap& mhi, const CUtensorMap& mlo,
                 TcParams p, dim3 grid, size_t smem)
{
    auto kern = p.fro2 ? tc_pass_kernel<TRANS, G, true, BF, ABF> : tc_pass_kernel<TRANS, G, false, BF, ABF>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return RSVDGB_ERR_CUDA;
    kern<<<grid, kThreads, smem, s>>>(mA, mhi, mlo, p);
    count_launches();
    return cudaGetLastError() == cudaSuccess ? RSVDGB_OK : RSVDGB_ERR_CUDA;
}

int groups_for(int l_pad, bool bf, bool abf = false)
{
    // TMEM: G accumulators of l_pad columns + 2 stages x G converted A tiles <= 512
    const int acols = bf ? kBK / 2 : (abf ? kBK : 2 * kBK);
    int g = 3;
    while (g > 1 && ((g * l_pad + 31) / 32 * 32 + kTmemStages * g * acols) > 512) --g;
    return g;
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
                   int chunk_stages, const float* aff_h, const float* aff_u, const float* aff_r)
{
    const bool bf = bf16_panel != 0;
    const bool abf = a_bf16 != 0;
    const int G = groups_for(l_pad, bf, abf);
    const size_t a_stage = (size_t)G * kTileRows * kBK * (abf ? 2 : 4);
    const size_t p_stage = (bf ? 2 : 8) * (size_t)l_pad * kBK;
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
    p.status = status;
    p.fro2 = fro2;
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
    int rc = RSVDGB_OK;
    switch ((abf ? 32 : 0) + (bf ? 16 : 0) + (trans ? 8 : 0) + G) {
        case 1: rc = launch_typed<false, 1, false, false>(s, mA, mhi, mlo, p, grid, smem); break;
        case 2: rc = launch_typed<false, 2, false, false>(s, mA, mhi, mlo, p, grid, smem); break;
        case 3: rc = launch_typed<false, 3, false, false>(s, mA, mhi, mlo, p, grid, smem); break;
        case 9: rc = launch_typed<true, 1, false, false>(s, mA, mhi, mlo, p, grid, smem); break;
        case 10: rc = launch_typed<true, 2, false, false>(s, mA, mhi, mlo, p, grid, smem); break;
        case 11: rc = launch_typed<true, 3, false, false>(s, mA, mhi, mlo, p, grid, smem); break;
        case 17: rc = launch_typed<false, 1, true, false>(s, mA, mhi, mlo, p, grid, smem); break;
        case 18: rc = launch_typed<false, 2, true, false>(s, mA, mhi, mlo, p, grid, smem); break;
        case 19: rc = launch_typed<false, 3, true, false>(s, mA, mhi, mlo, p, grid, smem); break;
        case 25: rc = launch_typed<true, 1, true, false>(s, mA, mhi, mlo, p, grid, smem); break;
        case 26: rc = launch_typed<true, 2, true, false>(s, mA, mhi, mlo, p, grid, smem); break;
        case 27: rc = launch_typed<true, 3, true, false>(s, mA, mhi, mlo, p, grid, smem); break;
        case 33: rc = launch_typed<false, 1, false, true>(s, mA, mhi, mlo, p, grid, smem); break;
        case 34: rc = launch_typed<false, 2, false, true>(s, mA, mhi, mlo, p, grid, smem); break;
        case 35: rc = launch_typed<false, 3, false, true>(s, mA, mhi, mlo, p, grid, smem); break;
        case 41: rc = launch_typed<true, 1, false, true>(s, mA, mhi, mlo, p, grid, smem); break;
        case 42: rc = launch_typed<true, 2, false, true>(s, mA, mhi, mlo, p, grid, smem); break;
        case 43: rc = launch_typed<true, 3, false, true>(s, mA, mhi, mlo, p, grid, smem); break;
        case 49: rc = launch_typed<false, 1, true, true>(s, mA, mhi, mlo, p, grid, smem); break;
        case 50: rc = launch_typed<false, 2, true, true>(s, mA, mhi, mlo, p, grid, smem); break;
        case 51: rc = launch_typed<false, 3, true, true>(s, mA, mhi, mlo, p, grid, smem); break;
        case 57: rc = launch_typed<true, 1, true, true>(s, mA, mhi, mlo, p, grid, smem); break;
        case 58: rc = launch_typed<true, 2, true, true>(s, mA, mhi, mlo, p, grid, smem); break;
        case 59: rc = launch_typed<true, 3, true, true>(s, mA, mhi, mlo, p, grid, smem); break;
        default: return RSVDGB_ERR_UNSUPPORTED;
    }
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
    const int G = std::max(std::max(groups_for(l_pad, false), groups_for(l_pad, true)), groups_for(l_pad, false, true));
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
